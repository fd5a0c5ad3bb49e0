// Small-channel kernel: every method on one channel of at most 32 users and
// 511 antennas, one CTA of 8 warps per right-hand side, the whole state in
// shared memory (the channel's aligned complex64 rows, m, and r, q, d, s per
// row).  A step is a few short phases separated by block barriers:
//
//   residuals   r_k = s_k - h_k m - xi q_k for the rows the method needs
//               (Alg. 1 step 8: all rows for GRK / AHK, X_{i(t-1)} for VR-OGRK
//               (Alg. 2 step 8), one row for RK), rows spread over the warps,
//               each row's VR over the lanes of its warp;
//   selection   warp 0 (lane k holds row k): inverse-CDF draws (Sec. III-A,
//               IV-A), the Bai-Wu greedy set, argmax with the lowest index on
//               ties; the stopping test on ||r||;
//   projection  m[Gamma_i] += gamma conj(h_i) over all threads (eq. (update));
//               the orthogonal set F with each warp taking whole rows (their
//               VRs are disjoint, Prop. 1); the aggregate u = H_V^H phi_V with
//               one thread per antenna (eqs. (update4), (coefficient)).
//
// Stopping as in the other kernels: tested where the method has its residual
// (RK: every K projections; GRK / VR-OGRK: before every selection; AHK: before
// every step; VR-OAHK: after the orthogonal half-step), every pass confirmed
// on the true residual rebuilt from m = H^H q with compensated FP32 sums.
#include "kz_device.cuh"

namespace {

constexpr int SNT = 256, SNW = 8, SU = 2;  // threads, warps, antennas per thread (Ntp <= 512)

// Inverse-CDF draw when lane k holds row k's weight w (lanes >= K hold 0): the
// smallest k whose running sum (FP64, inclusive scan over the lanes) exceeds
// u * total; the last positive weight when rounding leaves none; -1 when every
// weight is zero.  Every lane of the warp takes part.
__device__ __forceinline__ int lane_pick(double w, double u) {
    const int lane = threadIdx.x & 31;
    double incl = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double y = __shfl_up_sync(KZ_FULL, incl, o);
        if (lane >= o) incl += y;
    }
    const double total = __shfl_sync(KZ_FULL, incl, 31);
    const unsigned hit = __ballot_sync(KZ_FULL, total > 0.0 && incl > u * total);
    if (hit) return __ffs(hit) - 1;
    const unsigned pos = __ballot_sync(KZ_FULL, w > 0.0);
    return pos ? 31 - __clz(pos) : -1;
}

// Argmax of the lanes' values (lanes >= K pass -1), lowest lane on ties; -1 if
// none is >= 0.  *best (if given) receives the maximum.
__device__ __forceinline__ int lane_argmax(double v, double* best) {
    int bi = threadIdx.x & 31;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(KZ_FULL, v, o);
        const int oi = __shfl_xor_sync(KZ_FULL, bi, o);
        if (ov > v || (ov == v && oi < bi)) {
            v = ov;
            bi = oi;
        }
    }
    if (best) *best = v;
    return v >= 0.0 ? bi : -1;
}

__device__ __forceinline__ void dot2_acc(float a, float b, float& s, float& c) {
    const float p = a * b;
    const float pe = fmaf(a, b, -p);
    float e;
    two_sum(s, p, s, e);
    c += pe + e;
}

__global__ void __launch_bounds__(SNT, 1) kz_small_kernel(const __grid_constant__ KzLaunch L) {
    extern __shared__ __align__(16) unsigned char s_smem[];
    __shared__ float2 r_s[32], q_s[32], sv_s[32], ph_s[32];
    __shared__ float d_s[32];
    __shared__ int drawn_s[32];
    __shared__ double red_d[SNW];
    __shared__ double s_a, s_num, s_pn;
    __shared__ int s_sel;
    __shared__ float2 s_g;

    const KzInst& I = L.single;
    const int K = I.K, Nt = I.Nt, Ntp = I.Ntp;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int col = blockIdx.x;
    const int total2 = I.rptr[K - 1] + I.rows[K - 1].y;
    float2* Hs = reinterpret_cast<float2*>(s_smem);
    int4* rows_s = reinterpret_cast<int4*>(Hs + ((total2 + 1) & ~1));
    int* rptr_s = reinterpret_cast<int*>(rows_s + K);
    float2* m = reinterpret_cast<float2*>(rptr_s + ((K + 3) & ~3));
    const float xi = I.xi;
    const int algo = L.algo;

    for (int e = tid; e < total2; e += SNT) Hs[e] = I.Hc[e];
    for (int n = tid; n < Ntp; n += SNT) m[n] = make_float2(0.f, 0.f);
    if (tid < K) {
        rows_s[tid] = I.rows[tid];
        rptr_s[tid] = I.rptr[tid];
        const float2 sv = I.s[(size_t)col * K + tid];
        sv_s[tid] = sv;
        r_s[tid] = sv;
        q_s[tid] = make_float2(0.f, 0.f);
        d_s[tid] = I.nrm[tid] + xi;
        drawn_s[tid] = -1;
    }
    unsigned fmask = 0u;  // the orthogonal set F (rows of I.order[0, nF))
    for (int f = 0; f < I.nF; ++f) fmask |= 1u << I.order[f];
    const unsigned allmask = (K == 32) ? 0xffffffffu : ((1u << K) - 1u);
    const unsigned vmask = allmask & ~fmask;
    __syncthreads();
    double sn2 = 0.0, sumd = 0.0;  // ||s||^2 and ||B||_F^2 (warp 0 forms them, all read)
    if (warp == 0) {
        const float2 sv = lane < K ? sv_s[lane] : make_float2(0.f, 0.f);
        const double a = warp_sum_d((double)sv.x * sv.x + (double)sv.y * sv.y);
        const double b = warp_sum_d(lane < K ? I.nrmd[lane] : 0.0);
        if (lane == 0) {
            s_a = a;
            s_num = b + (double)K * xi;
        }
    }
    __syncthreads();
    sn2 = s_a;
    sumd = s_num;
    __syncthreads();  // s_a and s_num are reused below
    const double tol2 = L.tol * L.tol * sn2;

    // residuals of the rows in `mask` from the current m (plain or compensated sums)
    auto resid = [&](unsigned mask, bool comp) {
        for (int k = warp; k < K; k += SNW) {
            if (!((mask >> k) & 1u)) continue;
            const int4 rk = rows_s[k];
            const float2* h = Hs + rptr_s[k];
            const float2* v = m + rk.x;
            if (!comp) {
                float ax = 0.f, ay = 0.f;
                for (int p = lane; p < rk.y; p += 32) {
                    const float2 hh = h[p], vv = v[p];
                    ax = fmaf(hh.x, vv.x, fmaf(-hh.y, vv.y, ax));
                    ay = fmaf(hh.x, vv.y, fmaf(hh.y, vv.x, ay));
                }
                ax = warp_sum(ax);
                ay = warp_sum(ay);
                if (lane == 0) {
                    const float2 sv = sv_s[k], qv = q_s[k];
                    r_s[k] = make_float2(sv.x - ax - xi * qv.x, sv.y - ay - xi * qv.y);
                }
            } else {
                float sx = 0.f, cx = 0.f, sy = 0.f, cy = 0.f;
                for (int p = lane; p < rk.y; p += 32) {
                    const float2 hh = h[p], vv = v[p];
                    dot2_acc(hh.x, vv.x, sx, cx);
                    dot2_acc(-hh.y, vv.y, sx, cx);
                    dot2_acc(hh.x, vv.y, sy, cy);
                    dot2_acc(hh.y, vv.x, sy, cy);
                }
                float hx, lx, hy, ly;
                warp_sum_c(sx, hx, lx);
                warp_sum_c(sy, hy, ly);
                lx += warp_sum(cx);
                ly += warp_sum(cy);
                if (lane == 0) r_s[k] = true_resid(sv_s[k], make_float2(hx, hy), make_float2(lx, ly), q_s[k], xi);
            }
        }
        __syncthreads();
    };
    // ||r||^2 over the rows of `mask` (warp 0), every thread gets it
    auto norm2 = [&](unsigned mask) -> double {
        if (warp == 0) {
            const float2 rv = lane < K ? r_s[lane] : make_float2(0.f, 0.f);
            const double a = warp_sum_d(((mask >> lane) & 1u) ? (double)rv.x * rv.x + (double)rv.y * rv.y : 0.0);
            if (lane == 0) s_a = a;
        }
        __syncthreads();
        const double a = s_a;
        __syncthreads();
        return a;
    };
    // m = H^H q, one thread per antenna
    auto rebuild = [&]() {
        for (int c = 0; c < SU; ++c) {
            const int n = tid + c * SNT;
            if (n >= Ntp) continue;
            float2 acc = make_float2(0.f, 0.f);
            for (int k = 0; k < K; ++k) {
                const int4 rk = rows_s[k];
                if (n < rk.x || n >= rk.x + rk.y) continue;
                const float2 h = Hs[rptr_s[k] + (n - rk.x)], qk = q_s[k];
                acc.x = fmaf(h.x, qk.x, fmaf(h.y, qk.y, acc.x));
                acc.y = fmaf(h.x, qk.y, fmaf(-h.y, qk.x, acc.y));
            }
            m[n] = acc;
        }
        __syncthreads();
    };
    auto confirm = [&]() -> double {
        rebuild();
        resid(allmask, true);
        return norm2(allmask);
    };
    // m[Gamma_i] += g conj(h_i) on row i's true VR, all threads
    auto project = [&](int i, float2 g) {
        const int4 ri = rows_s[i];
        const float2* h = Hs + rptr_s[i];
        for (int p = tid; p < ri.y; p += SNT) {
            const int n = ri.x + p;
            if (n < ri.z || n >= ri.w) continue;
            const float2 hh = h[p];
            float2 v = m[n];
            v.x = fmaf(g.x, hh.x, fmaf(g.y, hh.y, v.x));
            v.y = fmaf(g.y, hh.x, fmaf(-g.x, hh.y, v.y));
            m[n] = v;
        }
        __syncthreads();
    };
    // aggregate step on the rows of `mask` (eq. (update4)) with phi = r / d
    auto aggregate = [&](unsigned mask) {
        if (warp == 0) {
            const bool in = lane < K && ((mask >> lane) & 1u);
            const float2 rv = in ? r_s[lane] : make_float2(0.f, 0.f);
            const float dk = lane < K ? d_s[lane] : 1.f;
            const float2 ph = in ? make_float2(rv.x / dk, rv.y / dk) : make_float2(0.f, 0.f);
            if (lane < K) ph_s[lane] = ph;
            const double num = warp_sum_d(in ? ((double)rv.x * rv.x + (double)rv.y * rv.y) / dk : 0.0);
            const double pn = warp_sum_d((double)ph.x * ph.x + (double)ph.y * ph.y);
            if (lane == 0) {
                s_num = num;
                s_pn = pn;
            }
        }
        __syncthreads();
        float2 u[SU];
        double un = 0.0;
#pragma unroll
        for (int c = 0; c < SU; ++c) {
            const int n = tid + c * SNT;
            float2 acc = make_float2(0.f, 0.f);
            if (n < Ntp) {
                for (int k = 0; k < K; ++k) {
                    if (!((mask >> k) & 1u)) continue;
                    const int4 rk = rows_s[k];
                    if (n < rk.x || n >= rk.x + rk.y) continue;
                    const float2 h = Hs[rptr_s[k] + (n - rk.x)], pk = ph_s[k];
                    acc.x = fmaf(h.x, pk.x, fmaf(h.y, pk.y, acc.x));
                    acc.y = fmaf(h.x, pk.y, fmaf(-h.y, pk.x, acc.y));
                }
            }
            u[c] = acc;
            un += (double)acc.x * acc.x + (double)acc.y * acc.y;
        }
        un = warp_sum_d(un);
        if (lane == 0) red_d[warp] = un;
        __syncthreads();
        if (tid == 0) {
            double a = 0.0;
            for (int w = 0; w < SNW; ++w) a += red_d[w];
            const double den = a + (double)xi * s_pn;
            s_g = make_float2((s_num > 0.0 && den > 0.0) ? (float)(s_num / den) : 0.f, 0.f);
        }
        __syncthreads();
        const float g = s_g.x;
#pragma unroll
        for (int c = 0; c < SU; ++c) {
            const int n = tid + c * SNT;
            if (n < Ntp) {
                m[n].x = fmaf(g, u[c].x, m[n].x);
                m[n].y = fmaf(g, u[c].y, m[n].y);
            }
        }
        if (tid < K && ((mask >> tid) & 1u)) {
            q_s[tid].x = fmaf(g, ph_s[tid].x, q_s[tid].x);
            q_s[tid].y = fmaf(g, ph_s[tid].y, q_s[tid].y);
        }
        __syncthreads();
    };

    int t = 0, since = 0;
    bool conv = false, numeric = false;
    const bool zero = !(sn2 > 0.0);
    if (!(sn2 == sn2) || isinf(sn2)) numeric = true;
    const bool is_rk = (algo == KZ_RK_ENERGY || algo == KZ_RK_UNIFORM || algo == KZ_RK_SWOR);
    const bool oahk = (algo == KZ_VR_OAHK), ahk = (algo == KZ_AHK), ogrk = (algo == KZ_VR_OGRK);
    const int refresh = L.refresh;
    if (zero || numeric) {
        conv = zero && !numeric;
    } else if (is_rk) {
        while (true) {
            if (t % K == 0) {
                resid(allmask, false);
                const double a = norm2(allmask);
                if (!(a == a) || isinf(a)) {
                    numeric = true;
                    break;
                }
                if (a <= tol2 && confirm() <= tol2) {
                    conv = true;
                    break;
                }
            }
            if (t >= L.max_iter) break;
            if (warp == 0) {  // draw a row, then its residual (lanes over its VR)
                const double uu = kz_uniform(L.seed, I.inst, col, t);
                const int sweep = t / K;
                const double dk = lane < K ? (double)d_s[lane] : 0.0;
                int sel;
                if (algo == KZ_RK_ENERGY)
                    sel = lane_pick(dk, uu);
                else if (algo == KZ_RK_SWOR)
                    sel = lane_pick(lane < K && drawn_s[lane] != sweep ? dk : 0.0, uu);
                else
                    sel = lane_pick(lane < K ? 1.0 : 0.0, uu);
                float2 g = make_float2(0.f, 0.f);
                if (sel >= 0) {
                    const int4 ri = rows_s[sel];
                    const float2* h = Hs + rptr_s[sel];
                    float ax = 0.f, ay = 0.f;
                    for (int p = lane; p < ri.y; p += 32) {
                        const float2 hh = h[p], vv = m[ri.x + p];
                        ax = fmaf(hh.x, vv.x, fmaf(-hh.y, vv.y, ax));
                        ay = fmaf(hh.x, vv.y, fmaf(hh.y, vv.x, ay));
                    }
                    ax = warp_sum(ax);
                    ay = warp_sum(ay);
                    const float2 sv = sv_s[sel], qv = q_s[sel];
                    const float ds = d_s[sel];
                    g = make_float2((sv.x - ax - xi * qv.x) / ds, (sv.y - ay - xi * qv.y) / ds);
                }
                __syncwarp();
                if (lane == 0) {
                    s_sel = sel;
                    s_g = g;
                    if (sel >= 0) {
                        drawn_s[sel] = sweep;
                        q_s[sel].x += g.x;
                        q_s[sel].y += g.y;
                    }
                }
            }
            __syncthreads();
            const int sel = s_sel;
            if (sel < 0) break;
            project(sel, s_g);
            ++t;
            if (++since >= refresh) {
                since = 0;
                rebuild();
            }
        }
    } else if (!ahk && !oahk) {  // GRK / VR-OGRK (GK arrives as GRK with argmax)
        int prev = -1;
        bool full = true;
        while (true) {
            unsigned mask = allmask;
            if (ogrk && !full) {
                mask = 0u;
                if (prev >= 0)
                    for (int e = I.xptr[prev]; e < I.xptr[prev + 1]; ++e) mask |= 1u << I.xidx[e];
            }
            full = false;
            if (mask) resid(mask, false);
            const double a = norm2(allmask);
            if (!(a == a) || isinf(a)) {
                numeric = true;
                break;
            }
            if (a <= tol2 && confirm() <= tol2) {
                conv = true;
                break;
            }
            if (t >= L.max_iter) break;
            if (warp == 0) {
                const double uu = kz_uniform(L.seed, I.inst, col, t);
                const float2 rv = lane < K ? r_s[lane] : make_float2(0.f, 0.f);
                const double a2 = (double)rv.x * rv.x + (double)rv.y * rv.y;
                const double ratio = lane < K ? a2 / (double)d_s[lane] : -1.0;
                int sel;
                if (L.sel == KZ_SEL_ARGMAX) {
                    sel = lane_argmax(ratio, nullptr);
                } else if (L.sel == KZ_SEL_PAPER) {
                    sel = lane_pick(a2, uu);
                } else {
                    double mx = 0.0;
                    (void)lane_argmax(ratio, &mx);
                    const double tot = warp_sum_d(a2);
                    const double thr = 0.5 * (mx + fmin(tot / sumd, mx));
                    sel = lane_pick(lane < K && ratio >= thr ? a2 : 0.0, uu);
                }
                if (lane == 0) {
                    s_sel = sel;
                    if (sel >= 0) {
                        const float2 rs = r_s[sel];
                        const float ds = d_s[sel];
                        const float2 g = make_float2(rs.x / ds, rs.y / ds);
                        s_g = g;
                        q_s[sel].x += g.x;
                        q_s[sel].y += g.y;
                    }
                }
            }
            __syncthreads();
            const int sel = s_sel;
            if (sel < 0) {
                conv = true;  // every residual is exactly zero
                break;
            }
            project(sel, s_g);
            prev = sel;
            ++t;
            if (++since >= refresh) {
                since = 0;
                rebuild();
                full = ogrk;  // carried residuals refer to the old m
            }
        }
    } else if (ahk) {
        while (true) {
            resid(allmask, false);
            const double a = norm2(allmask);
            if (!(a == a) || isinf(a)) {
                numeric = true;
                break;
            }
            if (a <= tol2 && confirm() <= tol2) {
                conv = true;
                break;
            }
            if (t >= L.max_iter) break;
            aggregate(allmask);
            ++t;
            if (++since >= refresh) {
                since = 0;
                rebuild();
            }
        }
    } else {  // VR-OAHK
        while (t < L.max_iter) {
            ++t;
            // orthogonal half-step: each warp projects whole rows of F (disjoint VRs)
            if (fmask) {
                resid(fmask, false);
                int idx = 0;
                for (unsigned fm = fmask; fm; fm &= fm - 1, ++idx) {
                    if (idx % SNW != warp) continue;
                    const int f = __ffs(fm) - 1;
                    const float2 rf = r_s[f];
                    const float df = d_s[f];
                    const float2 g = make_float2(rf.x / df, rf.y / df);
                    const int4 ri = rows_s[f];
                    const float2* h = Hs + rptr_s[f];
                    for (int p = lane; p < ri.y; p += 32) {
                        const int n = ri.x + p;
                        if (n < ri.z || n >= ri.w) continue;
                        const float2 hh = h[p];
                        float2 v = m[n];
                        v.x = fmaf(g.x, hh.x, fmaf(g.y, hh.y, v.x));
                        v.y = fmaf(g.y, hh.x, fmaf(-g.x, hh.y, v.y));
                        m[n] = v;
                    }
                    if (lane == 0) {
                        q_s[f].x += g.x;
                        q_s[f].y += g.y;
                    }
                }
                __syncthreads();
            }
            if (vmask) resid(vmask, false);
            const double a = norm2(vmask);
            if (!(a == a) || isinf(a)) {
                numeric = true;
                break;
            }
            if (a <= tol2 && confirm() <= tol2) {
                conv = true;
                break;
            }
            if (vmask) aggregate(vmask);
            if (++since >= refresh) {
                since = 0;
                rebuild();
            }
        }
    }
    // outputs: x = H^H q, the true residual, v = q
    const double rn2 = (zero || numeric) ? 0.0 : confirm();
    for (int n = tid; n < Nt; n += SNT) I.x[(size_t)col * Nt + n] = zero ? make_float2(0.f, 0.f) : m[n];
    if (I.v && tid < K) I.v[(size_t)col * K + tid] = q_s[tid];
    if (tid == 0) {
        I.iters[col] = t;
        I.resid[col] = zero ? 0.0 : (numeric ? (double)NAN : sqrt(rn2 / sn2));
        if (numeric || !(rn2 == rn2)) kz_flag(L.status, KZ_STATUS_BIT_NUMERIC);
        else if (!conv) kz_flag(L.status, KZ_STATUS_BIT_NOT_CONVERGED);
    }
}

}  // namespace

size_t kz_smem_small(int total2, int K, int Ntp) {
    return (size_t)((total2 + 1) & ~1) * sizeof(float2) + (size_t)K * sizeof(int4) + (size_t)((K + 3) & ~3) * sizeof(int) +
           (size_t)Ntp * sizeof(float2);
}

cudaError_t kz_launch_small(const KzLaunch& L, int grid, size_t smem, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(kz_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kz_small_kernel<<<grid, SNT, smem, st>>>(L);
    return cudaGetLastError();
}
