#include <algorithm>
// Set-up kernels (step A0), the adjoint contractions (step A10) and the
// per-user SINR / sum rate of the precoder (eq. (rate)).
#include "kz_device.cuh"

namespace {

// Row k of the caller's packed H (vr_len[k] entries at in_off[k]) into the
// aligned layout [a_k, a_k + len2_k) at rptr[k], zero-filled outside the VR;
// optionally a BF16 (re, im) copy rounded to nearest even.
__global__ void pack_rows_kernel(const float2* __restrict__ Hin, const int* __restrict__ in_off,
                                 const int4* __restrict__ rows, const int* __restrict__ rptr, float2* Hc,
                                 __nv_bfloat162* Hb) {
    const int k = blockIdx.x;
    const int4 rd = rows[k];  // {a, len2, o, e}
    const int src = in_off[k], dst = rptr[k];
    for (int p = threadIdx.x; p < rd.y; p += blockDim.x) {
        const int n = rd.x + p;
        const float2 h = (n >= rd.z && n < rd.w) ? Hin[src + (n - rd.z)] : make_float2(0.f, 0.f);
        Hc[dst + p] = h;
        if (Hb) Hb[dst + p] = __float22bfloat162_rn(h);
    }
}

// The same packing from a dense K x Nt row-major matrix: row k's VR [o, e)
// is read from Hd[k * Nt + n]; entries outside the VR are never read (the
// channel is zero there, eq. (3)).
__global__ void pack_dense_kernel(const float2* __restrict__ Hd, int Nt, const int4* __restrict__ rows,
                                  const int* __restrict__ rptr, float2* Hc, __nv_bfloat162* Hb) {
    const int k = blockIdx.x;
    const int4 rd = rows[k];  // {a, len2, o, e}
    const float2* src = Hd + (int64_t)k * Nt;
    const int dst = rptr[k];
    for (int p = threadIdx.x; p < rd.y; p += blockDim.x) {
        const int n = rd.x + p;
        const float2 h = (n >= rd.z && n < rd.w) ? src[n] : make_float2(0.f, 0.f);
        Hc[dst + p] = h;
        if (Hb) Hb[dst + p] = __float22bfloat162_rn(h);
    }
}

// ||h_k||^2 (one block per row) with Dot2-compensated FP32 sums: each thread
// carries (sum, error) words, the warps and then the block combine them with
// TwoSum in a fixed order; the result is about as accurate as an FP64 sum
// (GB300's FP64 rate is a small fraction of FP32's).
__device__ __forceinline__ void dot2_add(float a, float b, float& s, float& c);

__device__ double row_norm2(const float2* __restrict__ h, int len) {
    __shared__ float2 part[32];
    float s0 = 0.f, c0 = 0.f, s1 = 0.f, c1 = 0.f;
    for (int p = threadIdx.x; p < len; p += blockDim.x) {
        const float2 v = h[p];
        dot2_add(v.x, v.x, s0, c0);
        dot2_add(v.y, v.y, s1, c1);
    }
    float s, e;
    two_sum(s0, s1, s, e);
    float c = (c0 + c1) + e;
    for (int o = 16; o > 0; o >>= 1) {
        const float rs = __shfl_xor_sync(KZ_FULL, s, o), rc = __shfl_xor_sync(KZ_FULL, c, o);
        float t;
        two_sum(s, rs, s, t);
        c = (c + rc) + t;
    }
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = make_float2(s, c);
    __syncthreads();
    double out = 0.0;
    if (threadIdx.x == 0) {
        float hi = 0.f, lo = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            float t;
            two_sum(hi, part[w].x, hi, t);
            lo += part[w].y + t;
        }
        out = (double)hi + (double)lo;
    }
    return out;  // valid in thread 0
}

// The FP16 copy of row k (len2 entries at h): every entry times 1 / hs_k,
// hs_k the power of two at or above ||h_k|| (so each scaled entry is below 1
// and the row's largest entries keep FP16's full 11-bit precision), rounded to
// nearest even; hs_k = 1 for a zero or non-finite norm.  Called by every
// thread of the block after the norm t (FP64) is known to all of them.
__device__ void row_to_f16(const float2* __restrict__ h, int len, double t, __half2* hh, float* hs_k) {
    int ex = 0;
    if (t > 0.0 && t < 1e300) (void)frexp(sqrt(t), &ex);  // sqrt(t) < 2^ex
    ex = max(-126, min(126, ex));
    const float inv = ldexpf(1.f, -ex);
    for (int p = threadIdx.x; p < len; p += blockDim.x) {
        const float2 v = h[p];
        hh[p] = __float22half2_rn(make_float2(v.x * inv, v.y * inv));
    }
    if (threadIdx.x == 0) *hs_k = ldexpf(1.f, ex);
}

__global__ void row_norms_kernel(const float2* __restrict__ Hc, const int4* __restrict__ rows,
                                 const int* __restrict__ rptr, double* out_d, float* out_f, __half2* Hh, float* hs) {
    __shared__ double s_t;
    const int k = blockIdx.x;
    const double t = row_norm2(Hc + rptr[k], rows[k].y);
    if (threadIdx.x == 0) {
        out_d[k] = t;
        out_f[k] = (float)t;
        s_t = t;
    }
    if (Hh) {
        __syncthreads();
        row_to_f16(Hc + rptr[k], rows[k].y, s_t, Hh + rptr[k], hs + k);
    }
}

// Entries of the Gram matrix G = H H^H on the pattern of the overlap sets
// (G_kl is zero when the VRs of k and l are disjoint, Lemma 1): entry e of
// row k's CSR list (l = xidx[e]) gets the sum over the overlap of the two VRs
// of H[k, n] conj(H[l, n]).  Each lane sums its share with Ogita, Rump and
// Oishi's Dot2 (error-free TwoProduct by FMA and TwoSum, errors carried in a
// second word), the lanes' (sum, error) pairs are combined with compensated
// additions, and the result is rounded once: about as accurate as an FP64
// sum, on the FP32 units (GB300's FP64 rate is a small fraction of FP32).
// One block per row, one warp per entry of the upper half (l >= k); the
// lower half is the conjugate of the upper (G is Hermitian).
__device__ __forceinline__ void dot2_add(float a, float b, float& s, float& c) {
    const float p = a * b;
    const float pe = fmaf(a, b, -p);  // a b = p + pe exactly
    float e;
    two_sum(s, p, s, e);
    c += pe + e;
}

// One entry: sum over [lo, hi) of a[n] conj(b[n]) by one warp, four
// independent Dot2 chains (re re, im im, im re, -re im) with two elements in
// flight per lane; the value is returned in every lane.
__device__ __forceinline__ float2 overlap_entry(const float2* __restrict__ hk, const float2* __restrict__ hl, int lo,
                                                int hi) {
    const int lane = threadIdx.x & 31;
    float s0 = 0.f, c0 = 0.f, s1 = 0.f, c1 = 0.f, s2 = 0.f, c2 = 0.f, s3 = 0.f, c3 = 0.f;
    int n = lo + lane;
    for (; n + 32 < hi; n += 64) {
        const float2 a0 = hk[n], b0 = hl[n], a1 = hk[n + 32], b1 = hl[n + 32];
        dot2_add(a0.x, b0.x, s0, c0);
        dot2_add(a0.y, b0.y, s1, c1);
        dot2_add(a0.y, b0.x, s2, c2);
        dot2_add(-a0.x, b0.y, s3, c3);
        dot2_add(a1.x, b1.x, s0, c0);
        dot2_add(a1.y, b1.y, s1, c1);
        dot2_add(a1.y, b1.x, s2, c2);
        dot2_add(-a1.x, b1.y, s3, c3);
    }
    if (n < hi) {
        const float2 a0 = hk[n], b0 = hl[n];
        dot2_add(a0.x, b0.x, s0, c0);
        dot2_add(a0.y, b0.y, s1, c1);
        dot2_add(a0.y, b0.x, s2, c2);
        dot2_add(-a0.x, b0.y, s3, c3);
    }
    float sx, sy, ex, ey;
    two_sum(s0, s1, sx, ex);
    two_sum(s2, s3, sy, ey);
    float cx = (c0 + c1) + ex, cy = (c2 + c3) + ey;
    for (int o = 16; o > 0; o >>= 1) {
        const float rsx = __shfl_xor_sync(KZ_FULL, sx, o), rcx = __shfl_xor_sync(KZ_FULL, cx, o);
        const float rsy = __shfl_xor_sync(KZ_FULL, sy, o), rcy = __shfl_xor_sync(KZ_FULL, cy, o);
        float t;
        two_sum(sx, rsx, sx, t);
        cx = (cx + rcx) + t;
        two_sum(sy, rsy, sy, t);
        cy = (cy + rcy) + t;
    }
    return make_float2(sx + cx, sy + cy);
}

// Row k's entries G_kl for l >= k (G is Hermitian: the others are mirrored
// by gram_mirror), one warp per entry.
__device__ __forceinline__ void gram_row_upper(const float2* __restrict__ Hc, const int4* __restrict__ rows,
                                               const int* __restrict__ rptr, const int* __restrict__ xptr,
                                               const int* __restrict__ xidx, float2* __restrict__ G, int k) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int4 rk = rows[k];
    const float2* hk = Hc + rptr[k] - rk.x;
    const int e0 = xptr[k], e1 = xptr[k + 1];
    // first entry with l >= k (xidx is sorted and holds k)
    int lo = e0, hi = e1;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (xidx[mid] < k) lo = mid + 1;
        else hi = mid;
    }
    for (int e = lo + warp; e < e1; e += nw) {
        const int l = xidx[e];
        const int4 rl = rows[l];
        const float2* hl = Hc + rptr[l] - rl.x;
        const float2 v = overlap_entry(hk, hl, max(rk.z, rl.z), min(rk.w, rl.w));
        if (lane == 0) G[e] = v;
    }
}

// Row k's entries G_kl for l < k: conj(G_lk), found by binary search in X_l.
__device__ __forceinline__ void gram_row_mirror(const int* __restrict__ xptr, const int* __restrict__ xidx,
                                                float2* __restrict__ G, int k) {
    for (int e = xptr[k] + threadIdx.x; e < xptr[k + 1]; e += blockDim.x) {
        const int l = xidx[e];
        if (l >= k) break;
        int lo = xptr[l], hi = xptr[l + 1];
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (xidx[mid] < k) lo = mid + 1;
            else hi = mid;
        }
        const float2 v = G[lo];
        G[e] = make_float2(v.x, -v.y);
    }
}

__global__ void gram_kernel(const float2* __restrict__ Hc, const int4* __restrict__ rows, const int* __restrict__ rptr,
                            const int* __restrict__ xptr, const int* __restrict__ xidx, float2* __restrict__ G) {
    gram_row_upper(Hc, rows, rptr, xptr, xidx, G, blockIdx.x);
}

__global__ void gram_mirror_kernel(const int* __restrict__ xptr, const int* __restrict__ xidx, float2* __restrict__ G) {
    gram_row_mirror(xptr, xidx, G, blockIdx.x);
}

// Batched set-up (kz_batch_update): block i handles row rowmap[i].y of item
// rowmap[i].x of the instance table, whose packed channel starts at
// H_cat + hoff[item].  phase 0 packs the row (as pack_rows_kernel), phase 1
// forms its norm (as row_norms_kernel), phase 2 its inner products with the
// overlapping rows of higher index (as gram_kernel), phase 3 mirrors the
// others (as gram_mirror_kernel); the phases are separate launches.
__global__ void batch_update_kernel(const KzInst* __restrict__ insts, const int2* __restrict__ rowmap,
                                    const long long* __restrict__ hoff, const float2* __restrict__ H_cat, int row0,
                                    int phase) {
    const int2 ir = rowmap[row0 + blockIdx.x];
    const KzInst& I = insts[ir.x];
    const int k = ir.y;
    const int4 rd = I.rows[k];  // {a, len2, o, e}
    if (phase == 0) {
        const float2* src = H_cat + hoff[ir.x] + I.in_off[k];
        float2* Hc = const_cast<float2*>(I.Hc) + I.rptr[k];
        __nv_bfloat162* Hb = I.Hb ? const_cast<__nv_bfloat162*>(I.Hb) + I.rptr[k] : nullptr;
        for (int p = threadIdx.x; p < rd.y; p += blockDim.x) {
            const int n = rd.x + p;
            const float2 h = (n >= rd.z && n < rd.w) ? src[n - rd.z] : make_float2(0.f, 0.f);
            Hc[p] = h;
            if (Hb) Hb[p] = __float22bfloat162_rn(h);
        }
    } else if (phase == 1) {
        __shared__ double s_t;
        const double t = row_norm2(I.Hc + I.rptr[k], rd.y);
        if (threadIdx.x == 0) {
            const_cast<double*>(I.nrmd)[k] = t;
            const_cast<float*>(I.nrm)[k] = (float)t;
            s_t = t;
        }
        if (I.Hh) {
            __syncthreads();
            row_to_f16(I.Hc + I.rptr[k], rd.y, s_t, const_cast<__half2*>(I.Hh) + I.rptr[k], const_cast<float*>(I.hs) + k);
        }
    } else if (phase == 2) {
        gram_row_upper(I.Hc, I.rows, I.rptr, I.xptr, I.xidx, const_cast<float2*>(I.G), k);
    } else {
        gram_row_mirror(I.xptr, I.xidx, const_cast<float2*>(I.G), k);
    }
}

// Subarray-wise precoder (eq. (precoding2)): for the antennas n of subarray s
// (n in [s Nt / S, (s + 1) Nt / S)), F[n, j] = sum_{k in Q_s} conj(H[k, n]) V[k, j],
// Q_s the users whose VR meets the subarray.  Block (s, column chunk of 32):
// V's rows of Q_s staged in shared memory 64 at a time, one thread per
// antenna; the block's sum of |F|^2 goes to part[] for the normalisation.
__global__ void subarray_precoder_kernel(const __grid_constant__ KzInst I, const int* __restrict__ qptr,
                                         const int* __restrict__ qidx, int S, const float2* __restrict__ V, int ncols,
                                         float2* __restrict__ F, double* __restrict__ part) {
    __shared__ float2 sv[64 * 32];
    __shared__ int sk[64];
    __shared__ double red[32];
    const int s = blockIdx.x, c0 = blockIdx.y * 32, nc = min(32, ncols - c0);
    const int K = I.K, Nt = I.Nt;
    const int n0 = (int)((long long)s * Nt / S), n1 = (int)((long long)(s + 1) * Nt / S);
    const int q0 = qptr[s], q1 = qptr[s + 1];
    double ss = 0.0;
    for (int nb = n0; nb < n1; nb += blockDim.x) {
        const int n = nb + threadIdx.x;
        float2 acc[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) acc[j] = make_float2(0.f, 0.f);
        for (int qb = q0; qb < q1; qb += 64) {
            const int nq = min(64, q1 - qb);
            __syncthreads();
            for (int e = threadIdx.x; e < nq * 32; e += blockDim.x) {
                const int r = e % nq, j = e / nq;
                sv[r * 32 + j] = j < nc ? V[(size_t)(c0 + j) * K + qidx[qb + r]] : make_float2(0.f, 0.f);
            }
            for (int r = threadIdx.x; r < nq; r += blockDim.x) sk[r] = qidx[qb + r];
            __syncthreads();
            if (n < n1) {
                for (int r = 0; r < nq; ++r) {
                    const int k = sk[r];
                    const int4 rd = I.rows[k];  // {a, len2, o, e}
                    if (n < rd.z || n >= rd.w) continue;
                    const float2 h = I.Hc[I.rptr[k] + (n - rd.x)];
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const float2 v = sv[r * 32 + j];
                        acc[j].x = fmaf(h.x, v.x, fmaf(h.y, v.y, acc[j].x));
                        acc[j].y = fmaf(h.x, v.y, fmaf(-h.y, v.x, acc[j].y));
                    }
                }
            }
        }
        if (n < n1) {
            for (int j = 0; j < nc; ++j) {
                F[(size_t)(c0 + j) * Nt + n] = acc[j];
                ss += (double)acc[j].x * acc[j].x + (double)acc[j].y * acc[j].y;
            }
        }
    }
    ss = warp_sum_d(ss);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ss;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        part[blockIdx.x * gridDim.y + blockIdx.y] = t;
    }
}

// beta = 1 / sqrt(sum of the blocks' partial sums, in block order).
__global__ void precoder_beta_kernel(const double* __restrict__ part, int n, float* __restrict__ beta) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < n; ++i) t += part[i];
        *beta = t > 0.0 ? (float)(1.0 / sqrt(t)) : 0.f;
    }
}

__global__ void scale_kernel(float2* __restrict__ F, long long n, const float* __restrict__ beta) {
    const float b = *beta;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float2 f = F[i];
        F[i] = make_float2(f.x * b, f.y * b);
    }
}

// Reverse pass through T recorded row steps (the unrolled adjoint of a
// fixed-iteration RK / GRK / VR-OGRK solve; only the selected rows and step
// lengths were kept).  Forward step t of a column: i = row, gamma = (s_i -
// h_i m - xi q_i) / d_i with d_i = ||h_i||^2 + xi, m += gamma conj(h_i),
// q_i += gamma.  With adjoints mb, qb of the state after the step (PyTorch's
// convention: dL = Re sum conj(G) dz), the step's reverse is
//   gb = sum_n mb_n h_in + qb_i                      (adjoint of gamma)
//   dL/dh_in += gamma conj(mb_n) - gb conj(m_n) / d_i - (2 / d_i) Re(conj(gb) gamma) h_in
//   mb_n -= gb conj(h_in) / d_i,   qb_i -= xi gb / d_i,   sb_i += gb / d_i,
//   dL/dxi += -Re(conj(gb) (q_i + gamma)) / d_i
// where m_n, q_i are the state BEFORE the step, rebuilt from the state after
// it (m -= gamma conj(h_i), q_i -= gamma) starting from the solve's x and v.
// One CTA per column: m, mb (Nt) and q, qb, sb (K) in shared memory; the H
// gradient is added with atomics (its summation order over columns varies).
__global__ void unrolled_adjoint_kernel(const __grid_constant__ KzInst I, int nrhs, int T, const int* __restrict__ iters,
                                        const int* __restrict__ hrow, const float2* __restrict__ hgam,
                                        const float2* __restrict__ X, const float2* __restrict__ Vq,
                                        const float2* __restrict__ GX, const float2* __restrict__ GV,
                                        float2* __restrict__ gH, double* __restrict__ gxi, float2* __restrict__ gS) {
    extern __shared__ __align__(16) unsigned char ua_smem[];
    const int K = I.K, Nt = I.Nt, j = blockIdx.x;
    float2* m = reinterpret_cast<float2*>(ua_smem);
    float2* mb = m + Nt;
    float2* q = mb + Nt;
    float2* qb = q + K;
    float2* sb = qb + K;
    __shared__ float2 red[32];
    __shared__ float2 s_gb;
    const float xi = I.xi;
    for (int n = threadIdx.x; n < Nt; n += blockDim.x) {
        m[n] = X[(size_t)j * Nt + n];
        mb[n] = GX ? GX[(size_t)j * Nt + n] : make_float2(0.f, 0.f);
    }
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        q[k] = Vq[(size_t)j * K + k];
        qb[k] = GV ? GV[(size_t)j * K + k] : make_float2(0.f, 0.f);
        sb[k] = make_float2(0.f, 0.f);
    }
    __syncthreads();
    double gx = 0.0;
    const int steps = min(iters[j], T);
    for (int t = steps - 1; t >= 0; --t) {
        const int i = hrow[(size_t)t * nrhs + j];
        if (i < 0) continue;
        const float2 g = hgam[(size_t)t * nrhs + j];
        const int4 rd = I.rows[i];  // {a, len2, o, e}
        const float2* h = I.Hc + I.rptr[i] - rd.x;
        const float d = I.nrm[i] + xi;
        // rebuild m before the step; gb = sum mb h (+ qb_i)
        float ax = 0.f, ay = 0.f;
        for (int n = rd.z + threadIdx.x; n < rd.w; n += blockDim.x) {
            const float2 hn = h[n];
            float2 mn = m[n];
            mn.x -= g.x * hn.x + g.y * hn.y;
            mn.y -= g.y * hn.x - g.x * hn.y;
            m[n] = mn;
            const float2 b = mb[n];
            ax = fmaf(b.x, hn.x, fmaf(-b.y, hn.y, ax));
            ay = fmaf(b.x, hn.y, fmaf(b.y, hn.x, ay));
        }
        ax = warp_sum(ax);
        ay = warp_sum(ay);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = make_float2(ax, ay);
        __syncthreads();
        if (threadIdx.x == 0) {
            float2 a = qb[i];
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
                a.x += red[w].x;
                a.y += red[w].y;
            }
            s_gb = a;
        }
        __syncthreads();
        const float2 gb = s_gb;
        const float id = 1.f / d;
        const float c2 = 2.f * id * (gb.x * g.x + gb.y * g.y);
        float2* gh = gH + I.in_off[i] - rd.z;
        for (int n = rd.z + threadIdx.x; n < rd.w; n += blockDim.x) {
            const float2 hn = h[n], mn = m[n], b = mb[n];
            const float2 dh = make_float2((g.x * b.x + g.y * b.y) - id * (gb.x * mn.x + gb.y * mn.y) - c2 * hn.x,
                                          (g.y * b.x - g.x * b.y) - id * (gb.y * mn.x - gb.x * mn.y) - c2 * hn.y);
            atomicAdd(&gh[n].x, dh.x);
            atomicAdd(&gh[n].y, dh.y);
            mb[n] = make_float2(b.x - id * (gb.x * hn.x + gb.y * hn.y), b.y - id * (gb.y * hn.x - gb.x * hn.y));
        }
        if (threadIdx.x == 0) {
            const float2 qp = make_float2(q[i].x - g.x, q[i].y - g.y);
            gx -= ((double)gb.x * (qp.x + g.x) + (double)gb.y * (qp.y + g.y)) / d;
            sb[i].x += gb.x * id;
            sb[i].y += gb.y * id;
            qb[i].x -= xi * gb.x * id;
            qb[i].y -= xi * gb.y * id;
            q[i] = qp;
        }
        __syncthreads();
    }
    for (int k = threadIdx.x; k < K; k += blockDim.x) gS[(size_t)j * K + k] = sb[k];
    if (threadIdx.x == 0) atomicAdd(gxi, gx);
}

__global__ void double_to_float_kernel(const double* a, float* b) { *b = (float)*a; }

// Gt[:, j] = G_Q[:, j] + H G_X[:, j]   (one block per row, one warp per column).
__global__ void adjoint_rhs_kernel(const __grid_constant__ KzInst I, int nrhs, const float2* __restrict__ G_Q,
                                   const float2* __restrict__ G_X, float2* __restrict__ Gt) {
    const int i = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int4 rd = I.rows[i];
    const int base = I.rptr[i];
    for (int j = warp; j < nrhs; j += nw) {
        const float2* g = G_X + (size_t)j * I.Nt;
        float ax = 0.f, ay = 0.f;
        for (int n = rd.z + lane; n < rd.w; n += 32) {
            const float2 h = I.Hc[base + (n - rd.x)];
            const float2 v = g[n];
            ax = fmaf(h.x, v.x, fmaf(-h.y, v.y, ax));
            ay = fmaf(h.x, v.y, fmaf(h.y, v.x, ay));
        }
        ax = warp_sum(ax);
        ay = warp_sum(ay);
        if (lane == 0) {
            const float2 q = G_Q ? G_Q[(size_t)j * I.K + i] : make_float2(0.f, 0.f);
            Gt[(size_t)j * I.K + i] = make_float2(q.x + ax, q.y + ay);
        }
    }
}

// grad_H[k, n] = sum_j Q_kj conj(GX_nj) - Lam_kj conj(X_nj) - Q_kj conj(Y_nj) on row k's VR,
// written in the caller's packed layout (row k at in_off[k]).
__global__ void adjoint_grad_h_kernel(const __grid_constant__ KzInst I, int nrhs, const float2* __restrict__ Q,
                                      const float2* __restrict__ X, const float2* __restrict__ GX,
                                      const float2* __restrict__ Lam, const float2* __restrict__ Y,
                                      const int* __restrict__ in_off, float2* __restrict__ gH) {
    const int k = blockIdx.x;
    const int4 rd = I.rows[k];
    for (int n = rd.z + threadIdx.x; n < rd.w; n += blockDim.x) {
        float gx = 0.f, gy = 0.f;
        for (int j = 0; j < nrhs; ++j) {
            const float2 q = Q[(size_t)j * I.K + k];
            const float2 l = Lam[(size_t)j * I.K + k];
            const size_t o = (size_t)j * I.Nt + n;
            const float2 a = GX ? GX[o] : make_float2(0.f, 0.f);
            const float2 x = X[o];
            const float2 y = Y[o];
            // q conj(a - y) - l conj(x)
            const float2 c = make_float2(a.x - y.x, a.y - y.y);
            gx += q.x * c.x + q.y * c.y - (l.x * x.x + l.y * x.y);
            gy += q.y * c.x - q.x * c.y - (l.y * x.x - l.x * x.y);
        }
        gH[in_off[k] + (n - rd.z)] = make_float2(gx, gy);
    }
}

// grad_xi = -Re sum conj(Lam) Q  (single block, FP64 accumulation).
__global__ void adjoint_grad_xi_kernel(int count, const float2* __restrict__ Q, const float2* __restrict__ Lam,
                                       float* out) {
    __shared__ double part[32];
    double a = 0.0;
    for (int e = threadIdx.x; e < count; e += blockDim.x) {
        const float2 q = Q[e], l = Lam[e];
        a += (double)l.x * q.x + (double)l.y * q.y;
    }
    a = warp_sum_d(a);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
        *out = (float)(-t);
    }
}

// Batched forms: grid (item, row group); block y takes rows y, y + gridDim.y, ...
// of its item.
__global__ void adjoint_rhs_batched_kernel(const KzInst* __restrict__ insts, const KzAdjItem* __restrict__ adj,
                                           int nrhs) {
    const KzInst& I = insts[blockIdx.x];
    const KzAdjItem A = adj[blockIdx.x];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    float2* Gt = const_cast<float2*>(I.s);
    for (int i = blockIdx.y; i < I.K; i += gridDim.y) {
        const int4 rd = I.rows[i];
        const int base = I.rptr[i];
        for (int j = warp; j < nrhs; j += nw) {
            float ax = 0.f, ay = 0.f;
            if (A.G_X) {
                const float2* g = A.G_X + (size_t)j * I.Nt;
                for (int n = rd.z + lane; n < rd.w; n += 32) {
                    const float2 h = I.Hc[base + (n - rd.x)];
                    const float2 v = g[n];
                    ax = fmaf(h.x, v.x, fmaf(-h.y, v.y, ax));
                    ay = fmaf(h.x, v.y, fmaf(h.y, v.x, ay));
                }
                ax = warp_sum(ax);
                ay = warp_sum(ay);
            }
            if (lane == 0) {
                const float2 q = A.G_Q ? A.G_Q[(size_t)j * I.K + i] : make_float2(0.f, 0.f);
                Gt[(size_t)j * I.K + i] = make_float2(q.x + ax, q.y + ay);
            }
        }
    }
}

// Lambda = I.v and Y = H^H Lambda = I.x are the adjoint batch's outputs.
__global__ void adjoint_grad_h_batched_kernel(const KzInst* __restrict__ insts, const KzAdjItem* __restrict__ adj,
                                              int nrhs) {
    const KzInst& I = insts[blockIdx.x];
    const KzAdjItem A = adj[blockIdx.x];
    const float2* Lam = I.v;
    const float2* Y = I.x;
    for (int k = blockIdx.y; k < I.K; k += gridDim.y) {
        const int4 rd = I.rows[k];
        for (int n = rd.z + threadIdx.x; n < rd.w; n += blockDim.x) {
            float gx = 0.f, gy = 0.f;
            for (int j = 0; j < nrhs; ++j) {
                const float2 q = A.Q[(size_t)j * I.K + k];
                const float2 l = Lam[(size_t)j * I.K + k];
                const size_t o = (size_t)j * I.Nt + n;
                const float2 a = A.G_X ? A.G_X[o] : make_float2(0.f, 0.f);
                const float2 x = A.X[o];
                const float2 y = Y[o];
                const float2 c = make_float2(a.x - y.x, a.y - y.y);
                gx += q.x * c.x + q.y * c.y - (l.x * x.x + l.y * x.y);
                gy += q.y * c.x - q.x * c.y - (l.y * x.x - l.x * x.y);
            }
            A.grad_H[I.in_off[k] + (n - rd.z)] = make_float2(gx, gy);
        }
    }
}

__global__ void adjoint_grad_xi_batched_kernel(const KzInst* __restrict__ insts, const KzAdjItem* __restrict__ adj,
                                               int nrhs) {
    __shared__ double part[32];
    const KzInst& I = insts[blockIdx.x];
    const KzAdjItem A = adj[blockIdx.x];
    const int count = I.K * nrhs;
    double a = 0.0;
    for (int e = threadIdx.x; e < count; e += blockDim.x) {
        const float2 q = A.Q[e], l = I.v[e];
        a += (double)l.x * q.x + (double)l.y * q.y;
    }
    a = warp_sum_d(a);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
        *A.grad_xi = (float)(-t);
    }
}

// Per-user SINR and sum rate of F = X / ||X||_F (eq. (rate)) for one channel
// per block; X is Nt x K column-major (column k: user k's precoder).  Each
// warp owns whole rows k and sweeps the K columns in order (G_kj = h_k . x_j
// over row k's VR, FP32 lane sums combined with compensated additions,
// |G_kj|^2 summed in FP64), so every sum has a fixed order.
__device__ void sum_rate_block(const KzInst& I, const float2* __restrict__ X, double snr_lin, double* sinr,
                               double* rate, double* sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int K = I.K, Nt = I.Nt;
    double* sig = sm;          // K
    double* itf = sm + K;      // K
    double* part = sm + 2 * K; // 32 per-warp partials
    for (int k = warp; k < K; k += nw) {
        const int4 rd = I.rows[k];  // {a, len2, o, e}
        const float2* h = I.Hc + I.rptr[k] - rd.x;
        double acc_itf = 0.0, acc_sig = 0.0;
        for (int j = 0; j < K; ++j) {
            const float2* xj = X + (size_t)j * Nt;
            float gx = 0.f, gy = 0.f;
            for (int n = rd.z + lane; n < rd.w; n += 32) {
                const float2 a = h[n], b = xj[n];
                gx = fmaf(a.x, b.x, fmaf(-a.y, b.y, gx));
                gy = fmaf(a.x, b.y, fmaf(a.y, b.x, gy));
            }
            float hx, lx, hy, ly;
            warp_sum_c(gx, hx, lx);
            warp_sum_c(gy, hy, ly);
            const double re = (double)hx + lx, im = (double)hy + ly;
            const double g2 = re * re + im * im;
            if (j == k) acc_sig = g2;
            else acc_itf += g2;
        }
        if (lane == 0) {
            sig[k] = acc_sig;
            itf[k] = acc_itf;
        }
    }
    // ||X||_F^2, fixed order: per-thread sums, then per warp, then warp 0
    double f = 0.0;
    for (size_t e = threadIdx.x; e < (size_t)K * Nt; e += blockDim.x) {
        const float2 v = X[e];
        f += (double)v.x * v.x + (double)v.y * v.y;
    }
    f = warp_sum_d(f);
    if (lane == 0) part[warp] = f;
    __syncthreads();
    if (warp == 0) {
        double fr = 0.0;
        for (int w = 0; w < nw; ++w) fr += part[w];
        const double beta2 = fr > 0.0 ? 1.0 / fr : 0.0;
        double r = 0.0;
        for (int k = lane; k < K; k += 32) {
            const double g = beta2 * sig[k] / (beta2 * itf[k] + 1.0 / snr_lin);
            if (sinr) sinr[k] = g;
            r += log2(1.0 + g);
        }
        r = warp_sum_d(r);
        if (lane == 0 && rate) *rate = r;
    }
}

__global__ void sum_rate_kernel(const __grid_constant__ KzInst I, const float2* X, double snr_lin, double* sinr,
                                double* rate) {
    extern __shared__ double kz_sr_smem[];
    sum_rate_block(I, X, snr_lin, sinr, rate, kz_sr_smem);
}

// Batched: block b takes channel b of the batch and its x buffer; SINRs of
// channel b at sinr[b * K_max ...], its rate at rate[b].
__global__ void sum_rate_batched_kernel(const KzInst* __restrict__ insts, int K_max, double snr_lin, double* sinr,
                                        double* rate) {
    extern __shared__ double kz_sr_smem[];
    const KzInst& I = insts[blockIdx.x];
    sum_rate_block(I, I.x, snr_lin, sinr ? sinr + (size_t)blockIdx.x * K_max : nullptr,
                   rate ? rate + blockIdx.x : nullptr, kz_sr_smem);
}

}  // namespace

cudaError_t kz_sum_rate(const KzInst& I, const float2* X, double snr_lin, double* sinr, double* rate,
                        cudaStream_t st) {
    const size_t smem = (2 * (size_t)I.K + 32) * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(sum_rate_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    sum_rate_kernel<<<1, 1024, smem, st>>>(I, X, snr_lin, sinr, rate);
    return cudaGetLastError();
}

cudaError_t kz_sum_rate_batched(const KzInst* insts, int n, int K_max, double snr_lin, double* sinr, double* rate,
                                cudaStream_t st) {
    const size_t smem = (2 * (size_t)K_max + 32) * sizeof(double);
    cudaError_t e =
        cudaFuncSetAttribute(sum_rate_batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    sum_rate_batched_kernel<<<n, 1024, smem, st>>>(insts, K_max, snr_lin, sinr, rate);
    return cudaGetLastError();
}

cudaError_t kz_adjoint_rhs_batched(const KzInst* insts, const KzAdjItem* adj, int n, int K_max, int nrhs,
                                   cudaStream_t st) {
    adjoint_rhs_batched_kernel<<<dim3(n, std::min(K_max, 65535)), 256, 0, st>>>(insts, adj, nrhs);
    return cudaGetLastError();
}

cudaError_t kz_adjoint_contract_batched(const KzInst* insts, const KzAdjItem* adj, int n, int K_max, int nrhs,
                                        cudaStream_t st) {
    adjoint_grad_h_batched_kernel<<<dim3(n, std::min(K_max, 65535)), 256, 0, st>>>(insts, adj, nrhs);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    adjoint_grad_xi_batched_kernel<<<n, 1024, 0, st>>>(insts, adj, nrhs);
    return cudaGetLastError();
}

cudaError_t kz_pack_rows(const float2* Hin, const int* in_off, const int4* rows, const int* rptr, int K,
                         int64_t total2, float2* Hc, __nv_bfloat162* Hb, cudaStream_t st) {
    (void)total2;
    pack_rows_kernel<<<K, 256, 0, st>>>(Hin, in_off, rows, rptr, Hc, Hb);
    return cudaGetLastError();
}

cudaError_t kz_pack_dense(const float2* Hd, int Nt, const int4* rows, const int* rptr, int K, float2* Hc,
                          __nv_bfloat162* Hb, cudaStream_t st) {
    pack_dense_kernel<<<K, 256, 0, st>>>(Hd, Nt, rows, rptr, Hc, Hb);
    return cudaGetLastError();
}

cudaError_t kz_row_norms(const float2* Hc, const int4* rows, const int* rptr, int K, double* out_d, float* out_f,
                         __half2* Hh, float* hs, cudaStream_t st) {
    row_norms_kernel<<<K, 256, 0, st>>>(Hc, rows, rptr, out_d, out_f, Hh, hs);
    return cudaGetLastError();
}

__global__ void coupling_kernel(const KzInst* __restrict__ insts, float* __restrict__ mu) {
    const KzInst& I = insts[blockIdx.x];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __shared__ float s_max[32];
    float best = 0.f;
    for (int k = warp; k < I.K; k += nw) {
        const float dk = I.nrm[k] + I.xi;
        float a = 0.f;
        for (int e = I.xptr[k] + lane; e < I.xptr[k + 1]; e += 32) {
            const int l = I.xidx[e];
            if (l == k) continue;
            const float2 g = I.G[e];
            a += (g.x * g.x + g.y * g.y) / (dk * (I.nrm[l] + I.xi));
        }
        best = fmaxf(best, warp_sum(a));
    }
    if (lane == 0) s_max[warp] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = 0.f;
        for (int w = 0; w < nw; ++w) m = fmaxf(m, s_max[w]);
        mu[blockIdx.x] = m;
    }
}

cudaError_t kz_coupling(const KzInst* insts, int n, float* mu, cudaStream_t st) {
    coupling_kernel<<<n, 256, 0, st>>>(insts, mu);
    return cudaGetLastError();
}

cudaError_t kz_gram(const float2* Hc, const int4* rows, const int* rptr, const int* xptr, const int* xidx, int K,
                    float2* G, cudaStream_t st) {
    gram_kernel<<<K, 256, 0, st>>>(Hc, rows, rptr, xptr, xidx, G);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    gram_mirror_kernel<<<K, 128, 0, st>>>(xptr, xidx, G);
    return cudaGetLastError();
}

cudaError_t kz_batch_update_rows(const KzInst* insts, const int2* rowmap, int row0, int nrows, const long long* hoff,
                                 const float2* H_cat, cudaStream_t st) {
    if (nrows <= 0) return cudaSuccess;
    for (int phase = 0; phase < 4; ++phase) {
        batch_update_kernel<<<nrows, phase == 3 ? 128 : 256, 0, st>>>(insts, rowmap, hoff, H_cat, row0, phase);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t kz_subarray_precoder(const KzInst& I, const int* qptr, const int* qidx, int S, const float2* V, int ncols,
                                 float2* F, double* part, float* beta, cudaStream_t st) {
    const dim3 grid(S, (ncols + 31) / 32);
    subarray_precoder_kernel<<<grid, 128, 0, st>>>(I, qptr, qidx, S, V, ncols, F, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !beta) return e;
    precoder_beta_kernel<<<1, 32, 0, st>>>(part, (int)(grid.x * grid.y), beta);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const long long n = (long long)I.Nt * ncols;
    scale_kernel<<<(int)std::min<long long>((n + 255) / 256, 4096), 256, 0, st>>>(F, n, beta);
    return cudaGetLastError();
}

size_t kz_smem_unrolled(int Nt, int K) { return (size_t)(2 * Nt + 3 * K) * sizeof(float2); }

cudaError_t kz_unrolled_adjoint(const KzInst& I, int nrhs, int T, const int* iters, const int* hrow, const float2* hgam,
                                const float2* X, const float2* Vq, const float2* GX, const float2* GV, float2* gH,
                                double* gxi, float2* gS, float* gxi_out, cudaStream_t st) {
    const size_t smem = kz_smem_unrolled(I.Nt, I.K);
    cudaError_t e = cudaFuncSetAttribute(unrolled_adjoint_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    unrolled_adjoint_kernel<<<nrhs, 256, smem, st>>>(I, nrhs, T, iters, hrow, hgam, X, Vq, GX, GV, gH, gxi, gS);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    double_to_float_kernel<<<1, 1, 0, st>>>(gxi, gxi_out);
    return cudaGetLastError();
}

cudaError_t kz_adjoint_rhs(const KzInst& I, int nrhs, const float2* G_Q, const float2* G_X, float2* Gt,
                           cudaStream_t st) {
    adjoint_rhs_kernel<<<I.K, 256, 0, st>>>(I, nrhs, G_Q, G_X, Gt);
    return cudaGetLastError();
}

cudaError_t kz_adjoint_contract(const KzInst& I, int nrhs, const float2* Q, const float2* X, const float2* G_X,
                                const float2* Lam, const float2* Y, const int* in_off, float2* grad_H,
                                float* grad_xi, cudaStream_t st) {
    adjoint_grad_h_kernel<<<I.K, 256, 0, st>>>(I, nrhs, Q, X, G_X, Lam, Y, in_off, grad_H);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    adjoint_grad_xi_kernel<<<1, 1024, 0, st>>>(I.K * nrhs, Q, Lam, grad_xi);
    return cudaGetLastError();
}
