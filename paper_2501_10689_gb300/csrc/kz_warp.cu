// Warp kernel: every method on one small channel (K <= 32 users, at most 512
// antennas), one warp per right-hand side, no block-wide barrier inside the
// iteration.  Lane k owns row k of B = [H, sqrt(xi) I]: its residual r_k, q_k,
// d_k = ||h_k||^2 + xi and s_k stay in registers; the sets X_k and F are
// 32-bit masks; the channel (aligned complex64 rows) is staged once per CTA in
// shared memory, next to each warp's iterate m.
//
//   residual of own row  r_k = s_k - h_k m - xi q_k, each lane over its VR
//                        (Alg. 1 step 8; all rows for GRK / AHK, the rows of
//                        X_{i(t-1)} for VR-OGRK (Alg. 2 step 8), one row for RK)
//   selection            warp shuffles: inverse-CDF draws (Sec. III-A, IV-A),
//                        the Bai-Wu greedy set, argmax (lowest index on ties)
//   projection           m[Gamma_i] += gamma conj(h_i), lanes striding the VR
//                        (eq. (update)); the orthogonal set F row by row
//                        (Prop. 1); u = H_V^H phi_V with one lane per antenna
//                        (eqs. (update4), (coefficient))
//
// Stopping follows the other kernels: the test is made where the method has
// its residual (RK: every K projections; GRK / VR-OGRK: before every
// selection; AHK: before every step; VR-OAHK: after the orthogonal half-step)
// and every pass is confirmed on the true residual, rebuilt from m = H^H q
// with compensated FP32 sums (TwoProduct and TwoSum).
#include "kz_device.cuh"

namespace {

constexpr int WU = 16;  // antennas per lane in the aggregate: Ntp <= 512

// Inverse-CDF draw when lane k holds row k's weight w (lanes >= K hold 0):
// the smallest k whose running sum (FP64, inclusive scan over the lanes)
// exceeds u * total; the last positive weight when rounding leaves none; -1
// when every weight is zero.  Every lane takes part and gets the result.
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

// Argmax of the lanes' values v (lanes >= K pass -1), lowest lane on ties; -1 if
// no value is >= 0.  *best (if given) receives the maximum.
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

template <int NWC>
__global__ void __launch_bounds__(NWC * 32, 1) kz_warp_kernel(const __grid_constant__ KzLaunch L) {
    extern __shared__ __align__(16) unsigned char w_smem[];
    const KzInst& I = L.single;
    const int K = I.K, Nt = I.Nt, Ntp = I.Ntp;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int total2 = I.rptr[K - 1] + I.rows[K - 1].y;
    float2* Hs = reinterpret_cast<float2*>(w_smem);
    int4* rows_s = reinterpret_cast<int4*>(Hs + ((total2 + 1) & ~1));
    int* rptr_s = reinterpret_cast<int*>(rows_s + K);
    float2* m_all = reinterpret_cast<float2*>(rptr_s + ((K + 3) & ~3));
    for (int e = tid; e < total2; e += blockDim.x) Hs[e] = I.Hc[e];
    for (int k = tid; k < K; k += blockDim.x) {
        rows_s[k] = I.rows[k];
        rptr_s[k] = I.rptr[k];
    }
    __syncthreads();

    const int col = blockIdx.x * NWC + warp;
    if (col >= I.ld) return;
    float2* m = m_all + (size_t)warp * Ntp;
    const float xi = I.xi;
    const int algo = L.algo;
    const bool own = lane < K;
    const int4 rd = own ? rows_s[lane] : make_int4(0, 0, 0, 0);  // {a, len2, o, e}
    const int base = own ? rptr_s[lane] : 0;
    const float dk = own ? I.nrm[lane] + xi : 1.f;
    const float2 sk = own ? I.s[(size_t)col * K + lane] : make_float2(0.f, 0.f);
    unsigned xmask = 0u;  // X_k of this lane's row (k included)
    if (own)
        for (int e = I.xptr[lane]; e < I.xptr[lane + 1]; ++e) xmask |= 1u << I.xidx[e];
    unsigned fmask = 0u;  // the orthogonal set F
    for (int f = 0; f < I.nF; ++f) fmask |= 1u << I.order[f];
    const unsigned allmask = (K == 32) ? 0xffffffffu : ((1u << K) - 1u);
    const bool inF = own && ((fmask >> lane) & 1u);
    for (int n = lane; n < Ntp; n += 32) m[n] = make_float2(0.f, 0.f);
    __syncwarp();

    float2 q = make_float2(0.f, 0.f), r = sk;
    const double sn2 = warp_sum_d(own ? (double)sk.x * sk.x + (double)sk.y * sk.y : 0.0);
    const double tol2 = L.tol * L.tol * sn2;
    double sumd = warp_sum_d(own ? (double)I.nrmd[lane] : 0.0) + (double)K * xi;  // ||B||_F^2

    // r = s - h_k m - xi q on this lane's row (plain FP32 sums)
    auto own_resid = [&]() {
        float ax = 0.f, ay = 0.f;
        for (int p = 0; p < rd.y; ++p) {
            const float2 h = Hs[base + p], v = m[rd.x + p];
            ax = fmaf(h.x, v.x, fmaf(-h.y, v.y, ax));
            ay = fmaf(h.x, v.y, fmaf(h.y, v.x, ay));
        }
        return make_float2(sk.x - ax - xi * q.x, sk.y - ay - xi * q.y);
    };
    // m = H^H q (one lane per antenna), then the true residual of every row
    // with compensated sums; returns ||r||^2 and leaves the residual in r
    auto confirm = [&]() -> double {
        __syncwarp();
        for (int n0 = 0; n0 < Ntp; n0 += 32) {
            const int n = n0 + lane;
            float2 acc = make_float2(0.f, 0.f);
            for (int k = 0; k < K; ++k) {
                const float2 qk = make_float2(__shfl_sync(KZ_FULL, q.x, k), __shfl_sync(KZ_FULL, q.y, k));
                const int4 rk = rows_s[k];
                if (n < Ntp && n >= rk.x && n < rk.x + rk.y) {
                    const float2 h = Hs[rptr_s[k] + (n - rk.x)];
                    acc.x = fmaf(h.x, qk.x, fmaf(h.y, qk.y, acc.x));
                    acc.y = fmaf(h.x, qk.y, fmaf(-h.y, qk.x, acc.y));
                }
            }
            if (n < Ntp) m[n] = acc;
        }
        __syncwarp();
        if (own) {
            float sx = 0.f, cx = 0.f, sy = 0.f, cy = 0.f;
            for (int p = 0; p < rd.y; ++p) {
                const float2 h = Hs[base + p], v = m[rd.x + p];
                dot2_acc(h.x, v.x, sx, cx);
                dot2_acc(-h.y, v.y, sx, cx);
                dot2_acc(h.x, v.y, sy, cy);
                dot2_acc(h.y, v.x, sy, cy);
            }
            r = true_resid(sk, make_float2(sx, sy), make_float2(cx, cy), q, xi);
        } else {
            r = make_float2(0.f, 0.f);
        }
        return warp_sum_d((double)r.x * r.x + (double)r.y * r.y);
    };
    // residual of row i from the current m, all lanes (warp-wide dot)
    auto row_resid = [&](int i) {
        const int4 ri = rows_s[i];
        const int bi = rptr_s[i];
        float ax = 0.f, ay = 0.f;
        for (int p = lane; p < ri.y; p += 32) {
            const float2 h = Hs[bi + p], v = m[ri.x + p];
            ax = fmaf(h.x, v.x, fmaf(-h.y, v.y, ax));
            ay = fmaf(h.x, v.y, fmaf(h.y, v.x, ay));
        }
        ax = warp_sum(ax);
        ay = warp_sum(ay);
        const float2 si = make_float2(__shfl_sync(KZ_FULL, sk.x, i), __shfl_sync(KZ_FULL, sk.y, i));
        const float2 qi = make_float2(__shfl_sync(KZ_FULL, q.x, i), __shfl_sync(KZ_FULL, q.y, i));
        return make_float2(si.x - ax - xi * qi.x, si.y - ay - xi * qi.y);
    };
    // m[Gamma_i] += g conj(h_i) on the true VR, lanes striding the row
    auto project = [&](int i, float2 g) {
        __syncwarp();
        const int4 ri = rows_s[i];
        const int bi = rptr_s[i];
        for (int p = lane; p < ri.y; p += 32) {
            const int n = ri.x + p;
            if (n < ri.z || n >= ri.w) continue;
            const float2 h = Hs[bi + p];
            float2 v = m[n];
            v.x = fmaf(g.x, h.x, fmaf(g.y, h.y, v.x));
            v.y = fmaf(g.y, h.x, fmaf(-g.x, h.y, v.y));
            m[n] = v;
        }
        __syncwarp();
    };
    // aggregate step on the rows of `mask` with phi = r / d (eq. (update4)):
    // u = H^H phi, gamma = (phi^H r) / (||u||^2 + xi ||phi||^2), m += gamma u, q += gamma phi
    auto aggregate = [&](unsigned mask) {
        const bool in = own && ((mask >> lane) & 1u);
        const float2 ph = in ? make_float2(r.x / dk, r.y / dk) : make_float2(0.f, 0.f);
        const double num = warp_sum_d(in ? ((double)r.x * r.x + (double)r.y * r.y) / dk : 0.0);
        const double pn = warp_sum_d((double)ph.x * ph.x + (double)ph.y * ph.y);
        float2 u[WU];
        double un = 0.0;
#pragma unroll
        for (int c = 0; c < WU; ++c) {
            const int n = c * 32 + lane;
            float2 acc = make_float2(0.f, 0.f);
            if (c * 32 < Ntp) {
                for (int k = 0; k < K; ++k) {
                    const float2 pk = make_float2(__shfl_sync(KZ_FULL, ph.x, k), __shfl_sync(KZ_FULL, ph.y, k));
                    if (!((mask >> k) & 1u)) continue;
                    const int4 rk = rows_s[k];
                    if (n < Ntp && n >= rk.x && n < rk.x + rk.y) {
                        const float2 h = Hs[rptr_s[k] + (n - rk.x)];
                        acc.x = fmaf(h.x, pk.x, fmaf(h.y, pk.y, acc.x));
                        acc.y = fmaf(h.x, pk.y, fmaf(-h.y, pk.x, acc.y));
                    }
                }
            }
            u[c] = acc;
            un += (double)acc.x * acc.x + (double)acc.y * acc.y;
        }
        un = warp_sum_d(un);
        const double den = un + (double)xi * pn;
        const float g = (num > 0.0 && den > 0.0) ? (float)(num / den) : 0.f;
        __syncwarp();
#pragma unroll
        for (int c = 0; c < WU; ++c) {
            const int n = c * 32 + lane;
            if (c * 32 < Ntp && n < Ntp) {
                m[n].x = fmaf(g, u[c].x, m[n].x);
                m[n].y = fmaf(g, u[c].y, m[n].y);
            }
        }
        __syncwarp();
        q.x = fmaf(g, ph.x, q.x);
        q.y = fmaf(g, ph.y, q.y);
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
        int drawn_sweep = -1;  // SWOR: the sweep this lane's row was last drawn in
        while (true) {
            if (t % K == 0) {
                if (own) r = own_resid();
                const double a = warp_sum_d(own ? (double)r.x * r.x + (double)r.y * r.y : 0.0);
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
            const double uu = kz_uniform(L.seed, I.inst, col, t);
            const int sweep = t / K;
            int sel;
            if (algo == KZ_RK_ENERGY)
                sel = lane_pick(own ? (double)dk : 0.0, uu);
            else if (algo == KZ_RK_SWOR)
                sel = lane_pick(own && drawn_sweep != sweep ? (double)dk : 0.0, uu);
            else
                sel = lane_pick(own ? 1.0 : 0.0, uu);
            if (sel < 0) break;
            if (lane == sel) drawn_sweep = sweep;
            const float2 rs = row_resid(sel);
            const float ds = __shfl_sync(KZ_FULL, dk, sel);
            const float2 g = make_float2(rs.x / ds, rs.y / ds);
            project(sel, g);
            if (lane == sel) {
                q.x += g.x;
                q.y += g.y;
            }
            ++t;
            if (++since >= refresh) {
                since = 0;
                (void)confirm();  // rebuild m = H^H q
            }
        }
    } else if (!ahk && !oahk) {  // GRK / VR-OGRK (GK arrives as GRK with argmax)
        int prev = -1;
        bool full = true;
        while (true) {
            if (own && (algo == KZ_GRK || full || (prev >= 0 && ((xmask >> prev) & 1u)))) r = own_resid();
            full = false;
            const double a = warp_sum_d(own ? (double)r.x * r.x + (double)r.y * r.y : 0.0);
            if (!(a == a) || isinf(a)) {
                numeric = true;
                break;
            }
            if (a <= tol2) {
                if (confirm() <= tol2) {
                    conv = true;
                    break;
                }
            }
            if (t >= L.max_iter) break;
            const double uu = kz_uniform(L.seed, I.inst, col, t);
            // the residual weights as the other kernels take them: squares in FP64
            const double a2 = own ? (double)r.x * r.x + (double)r.y * r.y : 0.0;
            const double ratio = own ? a2 / (double)dk : -1.0;
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
                sel = lane_pick(own && ratio >= thr ? a2 : 0.0, uu);
            }
            if (sel < 0) {
                conv = true;  // every residual is exactly zero
                break;
            }
            const float ds = __shfl_sync(KZ_FULL, dk, sel);
            const float2 rs = make_float2(__shfl_sync(KZ_FULL, r.x, sel), __shfl_sync(KZ_FULL, r.y, sel));
            const float2 g = make_float2(rs.x / ds, rs.y / ds);
            project(sel, g);
            if (lane == sel) {
                q.x += g.x;
                q.y += g.y;
            }
            prev = sel;
            ++t;
            if (++since >= refresh) {
                since = 0;
                (void)confirm();
                full = ogrk;  // carried residuals refer to the old m
            }
        }
    } else if (ahk) {
        while (true) {
            if (own) r = own_resid();
            const double a = warp_sum_d(own ? (double)r.x * r.x + (double)r.y * r.y : 0.0);
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
                (void)confirm();
            }
        }
    } else {  // VR-OAHK
        const unsigned vmask = allmask & ~fmask;
        while (t < L.max_iter) {
            ++t;
            // orthogonal half-step: phi_F = r_F / d_F, unit step row by row
            if (inF) r = own_resid();
            for (unsigned fm = fmask; fm; fm &= fm - 1) {
                const int f = __ffs(fm) - 1;
                const float df = __shfl_sync(KZ_FULL, dk, f);
                const float2 rf = make_float2(__shfl_sync(KZ_FULL, r.x, f), __shfl_sync(KZ_FULL, r.y, f));
                const float2 g = make_float2(rf.x / df, rf.y / df);
                project(f, g);
                if (lane == f) {
                    q.x += g.x;
                    q.y += g.y;
                }
            }
            const bool inV = own && !inF;
            if (inV) r = own_resid();
            const double a = warp_sum_d(inV ? (double)r.x * r.x + (double)r.y * r.y : 0.0);
            if (!(a == a) || isinf(a)) {
                numeric = true;
                break;
            }
            if (a <= tol2) {
                if (confirm() <= tol2) {
                    conv = true;
                    break;
                }
            }
            if (vmask) aggregate(vmask);
            if (++since >= refresh) {
                since = 0;
                (void)confirm();
            }
        }
    }
    // outputs: x = H^H q, the true residual, v = q
    const double rn2 = (zero || numeric) ? (numeric ? (double)NAN : 0.0) : confirm();
    for (int n = lane; n < Nt; n += 32) I.x[(size_t)col * Nt + n] = zero ? make_float2(0.f, 0.f) : m[n];
    if (I.v && own) I.v[(size_t)col * K + lane] = q;
    if (lane == 0) {
        I.iters[col] = t;
        I.resid[col] = zero ? 0.0 : sqrt(rn2 / sn2);
        if (numeric || !(rn2 == rn2)) kz_flag(L.status, KZ_STATUS_BIT_NUMERIC);
        else if (!conv) kz_flag(L.status, KZ_STATUS_BIT_NOT_CONVERGED);
    }
}

}  // namespace

size_t kz_smem_warp(int nwc, int total2, int K, int Ntp) {
    return (size_t)((total2 + 1) & ~1) * sizeof(float2) + (size_t)K * sizeof(int4) + (size_t)((K + 3) & ~3) * sizeof(int) +
           (size_t)nwc * Ntp * sizeof(float2);
}

cudaError_t kz_launch_warp(const KzLaunch& L, int nwc, int grid, size_t smem, cudaStream_t st) {
    auto go = [&](auto kern) -> cudaError_t {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<grid, nwc * 32, smem, st>>>(L);
        return cudaGetLastError();
    };
    if (nwc == 1) return go(kz_warp_kernel<1>);
    if (nwc == 4) return go(kz_warp_kernel<4>);
    return cudaErrorInvalidValue;
}
