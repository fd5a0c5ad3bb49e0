// Small-channel kernel: every method on one channel of at most 32 users and
// 511 antennas, one CTA of 8 warps per right-hand side, the whole state in
// shared memory: the channel as a dense K x Ntp complex64 array (zero outside
// each VR, so the aggregate's per-antenna sums need no index lookups), m, and
// |r|^2, phi = r / d, q, s, 1/d per row.  Built for the latency of one solve, so a
// step is as few short phases between block barriers as the method allows:
//
//   residuals   r_k = s_k - h_k m - xi q_k for the rows the method needs
//               (Alg. 1 step 8: all rows for GRK / AHK, X_{i(t-1)} for VR-OGRK
//               (Alg. 2 step 8)), up to four rows per warp, each row's VR over
//               the lanes, the rows' warp sums interleaved;
//   selection   every warp on its own (lane k holds row k), so no barrier
//               follows it: inverse-CDF draws (Sec. III-A, IV-A), the Bai-Wu
//               greedy set, argmax with the lowest index on ties; the
//               stopping test on ||r||;
//   projection  m[Gamma_i] += gamma conj(h_i) over all threads (eq. (update));
//               RK's selected row, whose residual is taken in the same phase,
//               by warp 0 alone between the every-K-step tests; the
//               orthogonal set F with each warp taking whole rows (their VRs
//               are disjoint, Prop. 1); the aggregate u = H_V^H phi_V with one
//               thread per antenna (eqs. (update4), (coefficient)).
//
// All per-step arithmetic is FP32 (FP64 runs at a small fraction of the FP32
// rate on this GPU and its latency dominated a step): selection weights,
// their running sums and the draw u (the top 24 bits of the same
// counter-based SplitMix64 stream the other kernels use) are FP32.  Each
// column is scaled on entry by the power of two that brings its RMS into
// [0.5, 1); that is exact, so the iterates are exactly those of the unscaled
// column while squared residuals cannot underflow, and the outputs are scaled
// back exactly.
//
// Stopping as in the other kernels: tested where the method has its residual
// (RK: every K projections; GRK / VR-OGRK: before every selection; AHK: before
// every step; VR-OAHK: after the orthogonal half-step), every pass confirmed
// on the true residual rebuilt from m = H^H q with compensated FP32 sums.
#include "kz_device.cuh"

namespace {

constexpr int SNT = 256, SNW = 8, SU = 2, RPW = 4;  // threads, warps, antennas per thread, rows per warp

// Inclusive running sum over the lanes (lane k holds row k's weight).
__device__ __forceinline__ float lane_scan(float w) {
    const int lane = threadIdx.x & 31;
    float incl = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float y = __shfl_up_sync(KZ_FULL, incl, o);
        if (lane >= o) incl += y;
    }
    return incl;
}

// Inverse-CDF draw from a running sum: the smallest lane whose running sum
// exceeds u * total; the last positive weight when rounding leaves none; -1
// when every weight is zero.
__device__ __forceinline__ int pick_scan(float incl, float w, float u) {
    const float total = __shfl_sync(KZ_FULL, incl, 31);
    const unsigned hit = __ballot_sync(KZ_FULL, total > 0.f && incl > u * total);
    if (hit) return __ffs(hit) - 1;
    const unsigned pos = __ballot_sync(KZ_FULL, w > 0.f);
    return pos ? 31 - __clz(pos) : -1;
}

// Argmax of the lanes' values (lanes outside pass -1), lowest lane on ties;
// -1 if none is >= 0.  *best receives the maximum.
__device__ __forceinline__ int lane_argmax_f(float v, float* best) {
    int bi = threadIdx.x & 31;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_xor_sync(KZ_FULL, v, o);
        const int oi = __shfl_xor_sync(KZ_FULL, bi, o);
        if (ov > v || (ov == v && oi < bi)) {
            v = ov;
            bi = oi;
        }
    }
    *best = v;
    return v >= 0.f ? bi : -1;
}

// u in [0, 1): the top 24 bits of draw t of a column's SplitMix64 stream
// (key = kz_mix64(seed + counter * golden), as in kz_uniform).
__device__ __forceinline__ float draw24(unsigned long long key, int t) {
    const unsigned long long z = kz_mix64(key + (unsigned long long)(t + 1) * KZ_GOLDEN);
    return (float)(unsigned)(z >> 40) * 5.9604644775390625e-8f;
}

__device__ __forceinline__ void dot2_acc(float a, float b, float& s, float& c) {
    const float p = a * b;
    const float pe = fmaf(a, b, -p);
    float e;
    two_sum(s, p, s, e);
    c += pe + e;
}

__device__ __forceinline__ bool bad(float a) { return !(a == a) || isinf(a); }

__global__ void __launch_bounds__(SNT, 1) kz_small_kernel(const __grid_constant__ KzLaunch L) {
    extern __shared__ __align__(16) unsigned char s_smem[];
    __shared__ float2 ph_s[32], cf_s[32], q_s[32], sv_s[32];
    __shared__ float a2_s[32], dinv_s[32];
    __shared__ int2 vr_s[32];
    __shared__ unsigned xm_s[32];
    __shared__ float red_s[SNW];
    __shared__ double s_sn2, s_sumd;
    __shared__ int s_stop, s_tstop;

    const KzInst& I = L.single;
    const int K = I.K, Nt = I.Nt, Ntp = I.Ntp;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int col = blockIdx.x;
    float2* Hd = reinterpret_cast<float2*>(s_smem);  // Hd[k * Ntp + n]
    float2* m = Hd + (size_t)K * Ntp;
    const float xi = I.xi;
    const int algo = L.algo;

    for (int e = tid; e < K * Ntp; e += SNT) {
        const int k = e / Ntp, n = e - k * Ntp;
        const int4 rk = __ldg(I.rows + k);
        Hd[e] = (n >= rk.z && n < rk.w) ? I.Hc[__ldg(I.rptr + k) + (n - rk.x)] : make_float2(0.f, 0.f);
    }
    for (int n = tid; n < Ntp; n += SNT) m[n] = make_float2(0.f, 0.f);
    if (tid < K) {
        const int4 rk = I.rows[tid];
        vr_s[tid] = make_int2(rk.z, rk.w);
        unsigned xm = 0u;  // X_k (k included)
        for (int e = I.xptr[tid]; e < I.xptr[tid + 1]; ++e) xm |= 1u << I.xidx[e];
        xm_s[tid] = xm;
        const float dk = I.nrm[tid] + xi;
        dinv_s[tid] = dk > 0.f ? 1.f / dk : 0.f;
        q_s[tid] = make_float2(0.f, 0.f);
        ph_s[tid] = make_float2(0.f, 0.f);
        cf_s[tid] = make_float2(0.f, 0.f);  // rows outside the aggregate step keep 0
    }
    if (tid == 0) s_stop = 0;
    if (warp == 0) {  // ||s||^2, ||B||_F^2 and the column's scale, once, in FP64
        const float2 sv = lane < K ? I.s[(size_t)col * K + lane] : make_float2(0.f, 0.f);
        const double a = warp_sum_d((double)sv.x * sv.x + (double)sv.y * sv.y);
        const double b = warp_sum_d(lane < K ? I.nrmd[lane] : 0.0);
        int ex = 0;
        if (a > 0.0 && isfinite(a)) {
            (void)frexp(sqrt(a / K), &ex);
            ex = max(-120, min(120, ex));
        }
        const float sc = ldexpf(1.f, -ex);
        if (lane < K) {
            const float2 ss = make_float2(sv.x * sc, sv.y * sc);
            sv_s[lane] = ss;
            a2_s[lane] = ss.x * ss.x + ss.y * ss.y;
        }
        if (lane == 0) {
            s_sn2 = a;
            s_sumd = b + (double)K * xi;
            red_s[0] = sc;
        }
    }
    __syncthreads();
    const float sc = red_s[0];
    const float unsc = 1.f / sc;  // exact: sc is a power of two
    const double sn2 = s_sn2;     // unscaled ||s||^2
    const double sn2s = sn2 * (double)sc * (double)sc;
    const float tol2f = (float)(L.tol * L.tol * sn2s);
    const float inv_sumd = (float)(1.0 / s_sumd);
    __syncthreads();  // red_s is reused below

    unsigned fmask = 0u;  // the orthogonal set F (rows of I.order[0, nF))
    for (int f = 0; f < I.nF; ++f) fmask |= 1u << I.order[f];
    const unsigned allmask = (K == 32) ? 0xffffffffu : ((1u << K) - 1u);
    const unsigned vmask = allmask & ~fmask;
    const unsigned amask = algo == KZ_VR_OAHK ? vmask : allmask;  // rows the aggregate step takes

    // lane 0 of a warp stores row k's residual as |r_k|^2 and phi_k = r_k / d_k
    // (cf_k = phi_k on the rows the aggregate step takes, else 0)
    auto put_r = [&](int k, float2 r) {
        const float di = dinv_s[k];
        const float2 ph = make_float2(r.x * di, r.y * di);
        a2_s[k] = r.x * r.x + r.y * r.y;
        ph_s[k] = ph;
        cf_s[k] = ((amask >> k) & 1u) ? ph : make_float2(0.f, 0.f);
    };
    // r for the rows of `mask` from the current m (plain FP32 sums): a warp's
    // rows (up to four) advance together over their VRs, so their chains and
    // then their warp sums interleave
    auto resid = [&](unsigned mask) {
        float2 acc[RPW];
        int2 vr[RPW];
        int imax = 0;
#pragma unroll
        for (int j = 0; j < RPW; ++j) {
            acc[j] = make_float2(0.f, 0.f);
            const int k = warp + SNW * j;
            vr[j] = (k < K && ((mask >> k) & 1u)) ? vr_s[k] : make_int2(0, 0);
            imax = max(imax, (vr[j].y - vr[j].x + 31) >> 5);
        }
        for (int i = 0; i < imax; ++i) {
#pragma unroll
            for (int j = 0; j < RPW; ++j) {
                const int n = vr[j].x + lane + 32 * i;
                if (n < vr[j].y) {
                    const float2 hh = Hd[(size_t)(warp + SNW * j) * Ntp + n], vv = m[n];
                    acc[j].x = fmaf(hh.x, vv.x, fmaf(-hh.y, vv.y, acc[j].x));
                    acc[j].y = fmaf(hh.x, vv.y, fmaf(hh.y, vv.x, acc[j].y));
                }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
            for (int j = 0; j < RPW; ++j) {
                if (warp + SNW * j >= K) continue;
                acc[j].x += __shfl_xor_sync(KZ_FULL, acc[j].x, o);
                acc[j].y += __shfl_xor_sync(KZ_FULL, acc[j].y, o);
            }
        }
        if (lane == 0) {
#pragma unroll
            for (int j = 0; j < RPW; ++j) {
                const int k = warp + SNW * j;
                if (k >= K || !((mask >> k) & 1u)) continue;
                const float2 sv = sv_s[k], qv = q_s[k];
                put_r(k, make_float2(sv.x - acc[j].x - xi * qv.x, sv.y - acc[j].y - xi * qv.y));
            }
        }
        __syncthreads();
    };
    // the true residual of every row (compensated sums), for confirmation
    auto resid_true = [&]() {
        for (int k = warp; k < K; k += SNW) {
            const int2 vr = vr_s[k];
            const float2* h = Hd + (size_t)k * Ntp;
            float sx = 0.f, cx = 0.f, sy = 0.f, cy = 0.f;
            for (int n = vr.x + lane; n < vr.y; n += 32) {
                const float2 hh = h[n], vv = m[n];
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
            if (lane == 0) put_r(k, true_resid(sv_s[k], make_float2(hx, hy), make_float2(lx, ly), q_s[k], xi));
        }
        __syncthreads();
    };
    // ||r||^2 over the rows of `mask`, every warp on its own
    auto wnorm = [&](unsigned mask) -> float {
        return warp_sum((lane < K && ((mask >> lane) & 1u)) ? a2_s[lane] : 0.f);
    };
    // sum over all rows of conj(h_k[n]) c_k for this thread's antennas (rows
    // in two interleaved partial sums; zero coefficients drop rows out)
    auto gather = [&](const float2* c, float2 (&u)[SU]) {
        float2 ua[SU], ub[SU];
#pragma unroll
        for (int a = 0; a < SU; ++a) ua[a] = ub[a] = make_float2(0.f, 0.f);
        int k = 0;
#pragma unroll 2
        for (; k + 1 < K; k += 2) {
            const float2 c0 = c[k], c1 = c[k + 1];
            const float2* h0 = Hd + (size_t)k * Ntp;
            const float2* h1 = h0 + Ntp;
#pragma unroll
            for (int a = 0; a < SU; ++a) {
                const int n = tid + a * SNT;
                if (n < Ntp) {
                    const float2 x0 = h0[n], x1 = h1[n];
                    ua[a].x = fmaf(x0.x, c0.x, fmaf(x0.y, c0.y, ua[a].x));
                    ua[a].y = fmaf(x0.x, c0.y, fmaf(-x0.y, c0.x, ua[a].y));
                    ub[a].x = fmaf(x1.x, c1.x, fmaf(x1.y, c1.y, ub[a].x));
                    ub[a].y = fmaf(x1.x, c1.y, fmaf(-x1.y, c1.x, ub[a].y));
                }
            }
        }
        if (k < K) {
            const float2 c0 = c[k];
            const float2* h0 = Hd + (size_t)k * Ntp;
#pragma unroll
            for (int a = 0; a < SU; ++a) {
                const int n = tid + a * SNT;
                if (n < Ntp) {
                    const float2 x0 = h0[n];
                    ua[a].x = fmaf(x0.x, c0.x, fmaf(x0.y, c0.y, ua[a].x));
                    ua[a].y = fmaf(x0.x, c0.y, fmaf(-x0.y, c0.x, ua[a].y));
                }
            }
        }
#pragma unroll
        for (int a = 0; a < SU; ++a) u[a] = make_float2(ua[a].x + ub[a].x, ua[a].y + ub[a].y);
    };
    // m = H^H q
    auto rebuild = [&]() {
        float2 u[SU];
        gather(q_s, u);
#pragma unroll
        for (int a = 0; a < SU; ++a) {
            const int n = tid + a * SNT;
            if (n < Ntp) m[n] = u[a];
        }
        __syncthreads();
    };
    auto confirm = [&]() -> float {
        rebuild();
        resid_true();
        return wnorm(allmask);
    };
    // m[Gamma_i] += g conj(h_i) on row i's VR, all threads
    auto project = [&](int i, float2 g) {
        const int2 vr = vr_s[i];
        const float2* h = Hd + (size_t)i * Ntp;
        for (int n = vr.x + tid; n < vr.y; n += SNT) {
            const float2 hh = h[n];
            float2 v = m[n];
            v.x = fmaf(g.x, hh.x, fmaf(g.y, hh.y, v.x));
            v.y = fmaf(g.y, hh.x, fmaf(-g.x, hh.y, v.y));
            m[n] = v;
        }
        __syncthreads();
    };
    // one warp: row i's residual over its VR, the step g = r_i / d_i, and the
    // projection on the lanes' own entries; returns g
    auto warp_row_step = [&](int i) -> float2 {
        const int2 vr = vr_s[i];
        const float2* h = Hd + (size_t)i * Ntp;
        float ax = 0.f, ay = 0.f;
#pragma unroll 4
        for (int n = vr.x + lane; n < vr.y; n += 32) {
            const float2 hh = h[n], vv = m[n];
            ax = fmaf(hh.x, vv.x, fmaf(-hh.y, vv.y, ax));
            ay = fmaf(hh.x, vv.y, fmaf(hh.y, vv.x, ay));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ax += __shfl_xor_sync(KZ_FULL, ax, o);
            ay += __shfl_xor_sync(KZ_FULL, ay, o);
        }
        const float2 sv = sv_s[i], qv = q_s[i];
        const float di = dinv_s[i];
        const float2 g = make_float2((sv.x - ax - xi * qv.x) * di, (sv.y - ay - xi * qv.y) * di);
#pragma unroll 4
        for (int n = vr.x + lane; n < vr.y; n += 32) {
            const float2 hh = h[n];
            float2 v = m[n];
            v.x = fmaf(g.x, hh.x, fmaf(g.y, hh.y, v.x));
            v.y = fmaf(g.y, hh.x, fmaf(-g.x, hh.y, v.y));
            m[n] = v;
        }
        return g;
    };
    // aggregate step on the rows of `mask` (eq. (update4)), phi = r / d:
    // gamma = phi^H r / (||H^H phi||^2 + xi ||phi||^2)
    auto aggregate = [&](unsigned mask) {
        float2 u[SU];
        gather(cf_s, u);
        float un = 0.f;
#pragma unroll
        for (int a = 0; a < SU; ++a) un += u[a].x * u[a].x + u[a].y * u[a].y;
        // phi^H r = sum |r_k|^2 / d_k and ||phi||^2, lane k holding row k
        const bool in = lane < K && ((mask >> lane) & 1u);
        const float dl = in ? dinv_s[lane] : 0.f, al = in ? a2_s[lane] * dl : 0.f;
        float num = al, pn = al * dl;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            un += __shfl_xor_sync(KZ_FULL, un, o);
            num += __shfl_xor_sync(KZ_FULL, num, o);
            pn += __shfl_xor_sync(KZ_FULL, pn, o);
        }
        if (lane == 0) red_s[warp] = un;
        __syncthreads();
        float ut = 0.f;
#pragma unroll
        for (int w = 0; w < SNW; ++w) ut += red_s[w];
        const float den = ut + xi * pn;
        const float g = (num > 0.f && den > 0.f) ? num / den : 0.f;
#pragma unroll
        for (int a = 0; a < SU; ++a) {
            const int n = tid + a * SNT;
            if (n < Ntp) {
                m[n].x = fmaf(g, u[a].x, m[n].x);
                m[n].y = fmaf(g, u[a].y, m[n].y);
            }
        }
        if (tid < K && ((mask >> tid) & 1u)) {
            q_s[tid].x = fmaf(g, ph_s[tid].x, q_s[tid].x);
            q_s[tid].y = fmaf(g, ph_s[tid].y, q_s[tid].y);
        }
        __syncthreads();
    };

    const unsigned long long key =
        kz_mix64(L.seed + (((unsigned long long)(unsigned)I.inst << 32) + (unsigned long long)(unsigned)col + 1ull) *
                              KZ_GOLDEN);
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
        // fixed weights: their running sum once; SWOR-ERK re-scans each draw
        const float wl = lane < K ? (algo == KZ_RK_UNIFORM ? 1.f : I.nrm[lane] + xi) : 0.f;
        const float incl = lane_scan(wl);
        int drawn = -1;  // SWOR: the sweep in which this lane's row was last drawn (warp 0)
        while (true) {
            if (t % K == 0) {
                resid(allmask);
                const float a = wnorm(allmask);
                if (bad(a)) {
                    numeric = true;
                    break;
                }
                if (a <= tol2f && confirm() <= tol2f) {
                    conv = true;
                    break;
                }
            }
            if (t >= L.max_iter) break;
            const int seg = min(min(K - t % K, L.max_iter - t), refresh - since);
            if (warp == 0) {  // seg projections by warp 0 alone
                for (int st = 0; st < seg; ++st) {
                    const int tt = t + st;
                    const float u = draw24(key, tt);
                    int sel;
                    if (algo == KZ_RK_SWOR) {
                        const int sweep = tt / K;
                        const float w = drawn != sweep ? wl : 0.f;
                        sel = pick_scan(lane_scan(w), w, u);
                        if (lane == sel) drawn = sweep;
                    } else {
                        sel = pick_scan(incl, wl, u);
                    }
                    if (sel < 0) {
                        if (lane == 0) {
                            s_stop = 1;
                            s_tstop = tt;
                        }
                        break;
                    }
                    const float2 g = warp_row_step(sel);
                    __syncwarp();
                    if (lane == 0) {
                        q_s[sel].x += g.x;
                        q_s[sel].y += g.y;
                    }
                    __syncwarp();
                }
            }
            __syncthreads();
            if (s_stop) {  // every weight is zero: nothing left to project
                t = s_tstop;
                break;
            }
            t += seg;
            since += seg;
            if (since >= refresh) {
                since = 0;
                rebuild();
            }
        }
    } else if (!ahk && !oahk) {  // GRK / VR-OGRK (GK arrives as GRK with argmax)
        int prev = -1;
        bool full = true;
        while (true) {
            const unsigned mask = (ogrk && !full) ? xm_s[prev] : allmask;
            full = false;
            const float u = draw24(key, t);  // ahead of the residual phase, off the selection's path
            resid(mask);
            float a = wnorm(allmask);
            if (bad(a)) {
                numeric = true;
                break;
            }
            if (a <= tol2f) {
                const float ac = confirm();
                if (ac <= tol2f) {
                    conv = true;
                    break;
                }
                a = ac;
            }
            if (t >= L.max_iter) break;
            // selection, every warp on its own
            const float a2 = lane < K ? a2_s[lane] : 0.f;
            const float ratio = lane < K ? a2 * dinv_s[lane] : -1.f;
            int sel;
            if (L.sel == KZ_SEL_ARGMAX) {
                float mx;
                sel = lane_argmax_f(ratio, &mx);
            } else if (L.sel == KZ_SEL_PAPER) {
                sel = pick_scan(lane_scan(a2), a2, u);
            } else {  // Bai-Wu: rows with |r_k|^2 / d_k >= (max + ||r||^2 / ||B||_F^2) / 2
                float mx;
                (void)lane_argmax_f(ratio, &mx);
                const float thr = 0.5f * (mx + fminf(a * inv_sumd, mx));
                const float w = (lane < K && ratio >= thr) ? a2 : 0.f;
                sel = pick_scan(lane_scan(w), w, u);
            }
            if (sel < 0) {
                conv = true;  // every residual is exactly zero
                break;
            }
            const float2 g = ph_s[sel];
            if (tid == 0) {
                q_s[sel].x += g.x;
                q_s[sel].y += g.y;
            }
            project(sel, g);
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
            resid(allmask);
            const float a = wnorm(allmask);
            if (bad(a)) {
                numeric = true;
                break;
            }
            if (a <= tol2f && confirm() <= tol2f) {
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
            // orthogonal half-step: each warp takes whole rows of F (disjoint
            // VRs: a row's residual and projection touch only its own entries)
            if (fmask) {
                int idx = 0;
                for (unsigned fm = fmask; fm; fm &= fm - 1, ++idx) {
                    if (idx % SNW != warp) continue;
                    const int f = __ffs(fm) - 1;
                    const float2 g = warp_row_step(f);
                    if (lane == 0) {
                        q_s[f].x += g.x;
                        q_s[f].y += g.y;
                    }
                }
                __syncthreads();
            }
            if (vmask) resid(vmask);
            const float a = wnorm(vmask);
            if (bad(a)) {
                numeric = true;
                break;
            }
            if (a <= tol2f && confirm() <= tol2f) {
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
    // outputs: x = H^H q, the true residual, v = q (scaled back exactly)
    const float rn2 = (zero || numeric) ? 0.f : confirm();
    for (int n = tid; n < Nt; n += SNT) {
        const float2 v = m[n];
        I.x[(size_t)col * Nt + n] = zero ? make_float2(0.f, 0.f) : make_float2(v.x * unsc, v.y * unsc);
    }
    if (I.v && tid < K) I.v[(size_t)col * K + tid] = make_float2(q_s[tid].x * unsc, q_s[tid].y * unsc);
    if (tid == 0) {
        I.iters[col] = t;
        I.resid[col] = zero ? 0.0 : (numeric ? (double)NAN : sqrt((double)rn2 / sn2s));
        if (numeric || bad(rn2)) kz_flag(L.status, KZ_STATUS_BIT_NUMERIC);
        else if (!conv) kz_flag(L.status, KZ_STATUS_BIT_NOT_CONVERGED);
    }
}


// ---------------------------------------------------------------------------
// Register-resident variant for every method but RK on channels with
// K <= KMAX (16 or 32) and Ntp <= 256 AU: thread n keeps antenna n's column of
// H (and of m) in registers, so
//
//   residuals   each thread forms h_k[n] m[n] for all rows at once; a warp
//               reduces the 2 KMAX partial sums by recursive halving (31
//               shuffles for 32 values, every lane ending with one row
//               component), the 8 warps' sums meet in shared memory across
//               one block barrier, and every warp then finishes r_k, |r_k|^2,
//               phi_k for all rows on its own (lane k holds row k; r, q and
//               phi are replicated per warp, computed identically);
//   aggregate   u[n] = sum_k conj(h_k[n]) c_k from the warp's own copy of the
//               coefficients, ||u||^2 over one more barrier, then m[n] and q_k
//               update in registers;
//   projection  m[n] += g conj(h_i[n]) from the dense shared-memory copy of
//               row i, no barrier (GRK); the orthogonal set F as one gather
//               with coefficients r_f / d_f (disjoint VRs: one term per
//               antenna).
//
// Block barriers per step: GRK / VR-OGRK 1, AHK 2, VR-OAHK 3.  The
// confirmation stages m in shared memory and takes the rows' true residuals
// with compensated sums, as in the shared-memory kernel above.
// Recursive halving: v[32] per lane -> this lane's value of index `lane`
// summed over the warp (fixed order).
__device__ __forceinline__ float halving_sum32(float (&v)[32]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 16, w = 16; o > 0; o >>= 1, w >>= 1) {
        const bool hi = lane & o;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            if (i >= w) break;
            const float send = hi ? v[i] : v[i + w];
            const float keep = hi ? v[i + w] : v[i];
            v[i] = keep + __shfl_xor_sync(KZ_FULL, send, o);
        }
    }
    return v[0];
}

template <int KMAX, int AU>
__global__ void __launch_bounds__(SNT, 1) kz_small_reg_kernel(const __grid_constant__ KzLaunch L) {
    constexpr int NB = (2 * KMAX) / 32;  // banks of 32 partial sums: re parts, then im parts
    extern __shared__ __align__(16) unsigned char s_smem[];
    __shared__ float part_s[2][SNW][2 * KMAX];
    __shared__ float red_s[2][SNW];
    __shared__ float2 cw_s[SNW][KMAX];
    __shared__ float2 rt_s[32];
    __shared__ unsigned xm_s[32];
    __shared__ int2 vr_s[32];
    __shared__ double s_sn2, s_sumd;
    __shared__ float s_sc;

    const KzInst& I = L.single;
    const int K = I.K, Nt = I.Nt, Ntp = I.Ntp;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int col = blockIdx.x;
    float2* Hd = reinterpret_cast<float2*>(s_smem);  // Hd[k * Ntp + n], zero outside each VR
    float2* m_s = Hd + (size_t)K * Ntp;                // m staged for the confirmation
    const float xi = I.xi;
    const int algo = L.algo;

    for (int e = tid; e < K * Ntp; e += SNT) {
        const int k = e / Ntp, n = e - k * Ntp;
        const int4 rk = __ldg(I.rows + k);
        Hd[e] = (n >= rk.z && n < rk.w) ? I.Hc[__ldg(I.rptr + k) + (n - rk.x)] : make_float2(0.f, 0.f);
    }
    if (tid < K) {
        const int4 rk = I.rows[tid];
        vr_s[tid] = make_int2(rk.z, rk.w);
        unsigned xm = 0u;  // X_k (k included)
        for (int e = I.xptr[tid]; e < I.xptr[tid + 1]; ++e) xm |= 1u << I.xidx[e];
        xm_s[tid] = xm;
    }
    if (warp == 0) {  // ||s||^2, ||B||_F^2 and the column's scale, once, in FP64
        const float2 sv = lane < K ? I.s[(size_t)col * K + lane] : make_float2(0.f, 0.f);
        const double a = warp_sum_d((double)sv.x * sv.x + (double)sv.y * sv.y);
        const double b = warp_sum_d(lane < K ? I.nrmd[lane] : 0.0);
        int ex = 0;
        if (a > 0.0 && isfinite(a)) {
            (void)frexp(sqrt(a / K), &ex);
            ex = max(-120, min(120, ex));
        }
        if (lane == 0) {
            s_sn2 = a;
            s_sumd = b + (double)K * xi;
            s_sc = ldexpf(1.f, -ex);
        }
    }
    __syncthreads();
    const float sc = s_sc, unsc = 1.f / sc;  // exact: sc is a power of two
    const double sn2 = s_sn2;
    const double sn2s = sn2 * (double)sc * (double)sc;
    const float tol2f = (float)(L.tol * L.tol * sn2s);
    const float inv_sumd = (float)(1.0 / s_sumd);

    // this thread's antennas: H column and m in registers
    float2 h[AU][KMAX], m[AU];
#pragma unroll
    for (int a = 0; a < AU; ++a) {
        const int n = tid + a * SNT;
        m[a] = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < KMAX; ++k) h[a][k] = (k < K && n < Ntp) ? Hd[(size_t)k * Ntp + n] : make_float2(0.f, 0.f);
    }
    // lane k's row (replicated in every warp)
    const bool own = lane < K;
    const float2 sv = own ? make_float2(I.s[(size_t)col * K + lane].x * sc, I.s[(size_t)col * K + lane].y * sc)
                          : make_float2(0.f, 0.f);
    const float dk = own ? I.nrm[lane] + xi : 0.f;
    const float dinv = dk > 0.f ? 1.f / dk : 0.f;
    float2 q = make_float2(0.f, 0.f), ph = make_float2(0.f, 0.f);
    float a2 = sv.x * sv.x + sv.y * sv.y;

    unsigned fmask = 0u;
    for (int f = 0; f < I.nF; ++f) fmask |= 1u << I.order[f];
    const unsigned allmask = (K == 32) ? 0xffffffffu : ((1u << K) - 1u);
    const unsigned vmask = allmask & ~fmask;

    int pp = 0, rp = 0;  // parities of the double-buffered partial sums
    auto set_r = [&](float2 r) {
        a2 = r.x * r.x + r.y * r.y;
        ph = make_float2(r.x * dinv, r.y * dinv);
    };
    // r for the rows of `mask` (others keep theirs)
    auto resid = [&](unsigned mask) {
        float v[NB][32];
#pragma unroll
        for (int k = 0; k < KMAX; ++k) {
            float px = 0.f, py = 0.f;
            if ((mask >> k) & 1u) {
#pragma unroll
                for (int a = 0; a < AU; ++a) {
                    px = fmaf(h[a][k].x, m[a].x, fmaf(-h[a][k].y, m[a].y, px));
                    py = fmaf(h[a][k].x, m[a].y, fmaf(h[a][k].y, m[a].x, py));
                }
            }
            v[k / 32][k % 32] = px;
            v[(KMAX + k) / 32][(KMAX + k) % 32] = py;
        }
        float* ps = part_s[pp][warp];
#pragma unroll
        for (int b = 0; b < NB; ++b) ps[b * 32 + lane] = halving_sum32(v[b]);
        __syncthreads();
        if (own && ((mask >> lane) & 1u)) {
            float hx = 0.f, hy = 0.f;
#pragma unroll
            for (int w = 0; w < SNW; ++w) {
                hx += part_s[pp][w][lane];
                hy += part_s[pp][w][KMAX + lane];
            }
            set_r(make_float2(sv.x - hx - xi * q.x, sv.y - hy - xi * q.y));
        }
        pp ^= 1;
    };
    auto rnorm = [&](unsigned mask) -> float { return warp_sum((own && ((mask >> lane) & 1u)) ? a2 : 0.f); };
    // u[a] = sum_k conj(h_k[n]) c_k with c from lane k of this warp
    auto gather = [&](float2 c, float2 (&u)[AU]) {
        __syncwarp();
        if (lane < KMAX) cw_s[warp][lane] = own ? c : make_float2(0.f, 0.f);
        __syncwarp();
        float2 ua[AU], ub[AU];
#pragma unroll
        for (int a = 0; a < AU; ++a) ua[a] = ub[a] = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < KMAX; k += 2) {
            const float2 c0 = cw_s[warp][k], c1 = cw_s[warp][k + 1];
#pragma unroll
            for (int a = 0; a < AU; ++a) {
                ua[a].x = fmaf(h[a][k].x, c0.x, fmaf(h[a][k].y, c0.y, ua[a].x));
                ua[a].y = fmaf(h[a][k].x, c0.y, fmaf(-h[a][k].y, c0.x, ua[a].y));
                ub[a].x = fmaf(h[a][k + 1].x, c1.x, fmaf(h[a][k + 1].y, c1.y, ub[a].x));
                ub[a].y = fmaf(h[a][k + 1].x, c1.y, fmaf(-h[a][k + 1].y, c1.x, ub[a].y));
            }
        }
#pragma unroll
        for (int a = 0; a < AU; ++a) u[a] = make_float2(ua[a].x + ub[a].x, ua[a].y + ub[a].y);
    };
    auto rebuild = [&]() {  // m = H^H q
        float2 u[AU];
        gather(q, u);
#pragma unroll
        for (int a = 0; a < AU; ++a) m[a] = u[a];
    };
    // the true residual of every row: m rebuilt, staged, compensated row sums
    auto confirm = [&]() -> float {
        rebuild();
#pragma unroll
        for (int a = 0; a < AU; ++a) {
            const int n = tid + a * SNT;
            if (n < Ntp) m_s[n] = m[a];
        }
        __syncthreads();
        for (int k = warp; k < K; k += SNW) {
            const int2 vr = vr_s[k];
            const float2* hk = Hd + (size_t)k * Ntp;
            float sx = 0.f, cx = 0.f, sy = 0.f, cy = 0.f;
            for (int n = vr.x + lane; n < vr.y; n += 32) {
                const float2 hh = hk[n], vv = m_s[n];
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
            const float2 sk = make_float2(__shfl_sync(KZ_FULL, sv.x, k), __shfl_sync(KZ_FULL, sv.y, k));
            const float2 qk = make_float2(__shfl_sync(KZ_FULL, q.x, k), __shfl_sync(KZ_FULL, q.y, k));
            if (lane == 0) rt_s[k] = true_resid(sk, make_float2(hx, hy), make_float2(lx, ly), qk, xi);
        }
        __syncthreads();
        if (own) set_r(rt_s[lane]);
        __syncthreads();  // rt_s and m_s are rewritten by the next confirmation only after this
        return rnorm(allmask);
    };
    // aggregate step on the rows of `mask` (eq. (update4))
    auto aggregate = [&](unsigned mask) {
        const bool in = own && ((mask >> lane) & 1u);
        float2 u[AU];
        gather(in ? ph : make_float2(0.f, 0.f), u);
        float un = 0.f;
#pragma unroll
        for (int a = 0; a < AU; ++a) un += u[a].x * u[a].x + u[a].y * u[a].y;
        const float al = in ? a2 * dinv : 0.f;
        float num = al, pn = al * dinv;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            un += __shfl_xor_sync(KZ_FULL, un, o);
            num += __shfl_xor_sync(KZ_FULL, num, o);
            pn += __shfl_xor_sync(KZ_FULL, pn, o);
        }
        if (lane == 0) red_s[rp][warp] = un;
        __syncthreads();
        float ut = 0.f;
#pragma unroll
        for (int w = 0; w < SNW; ++w) ut += red_s[rp][w];
        rp ^= 1;
        const float den = ut + xi * pn;
        const float g = (num > 0.f && den > 0.f) ? num / den : 0.f;
#pragma unroll
        for (int a = 0; a < AU; ++a) {
            m[a].x = fmaf(g, u[a].x, m[a].x);
            m[a].y = fmaf(g, u[a].y, m[a].y);
        }
        if (in) {
            q.x = fmaf(g, ph.x, q.x);
            q.y = fmaf(g, ph.y, q.y);
        }
    };

    const unsigned long long key =
        kz_mix64(L.seed + (((unsigned long long)(unsigned)I.inst << 32) + (unsigned long long)(unsigned)col + 1ull) *
                              KZ_GOLDEN);
    int t = 0, since = 0;
    bool conv = false, numeric = false;
    const bool zero = !(sn2 > 0.0);
    if (!(sn2 == sn2) || isinf(sn2)) numeric = true;
    const bool oahk = (algo == KZ_VR_OAHK), ahk = (algo == KZ_AHK), ogrk = (algo == KZ_VR_OGRK);
    const int refresh = L.refresh;
    if (zero || numeric) {
        conv = zero && !numeric;
    } else if (!ahk && !oahk) {  // GRK / VR-OGRK (GK arrives as GRK with argmax)
        int prev = -1;
        bool full = true;
        while (true) {
            const unsigned mask = (ogrk && !full) ? xm_s[prev] : allmask;
            full = false;
            const float u = draw24(key, t);
            resid(mask);
            // the paper's rule draws from the running sum of |r_k|^2, whose
            // total is ||r||^2: one scan serves the stopping test and the draw
            const bool paper = L.sel == KZ_SEL_PAPER;
            float incl = paper ? lane_scan(own ? a2 : 0.f) : 0.f;
            float a = paper ? __shfl_sync(KZ_FULL, incl, 31) : rnorm(allmask);
            if (bad(a)) {
                numeric = true;
                break;
            }
            if (a <= tol2f) {
                const float ac = confirm();
                if (ac <= tol2f) {
                    conv = true;
                    break;
                }
                a = ac;
                if (paper) incl = lane_scan(own ? a2 : 0.f);  // the confirmed residuals
            }
            if (t >= L.max_iter) break;
            const float w2 = own ? a2 : 0.f;
            const float ratio = own ? a2 * dinv : -1.f;
            int sel;
            if (L.sel == KZ_SEL_ARGMAX) {
                float mx;
                sel = lane_argmax_f(ratio, &mx);
            } else if (paper) {
                sel = pick_scan(incl, w2, u);
            } else {  // Bai-Wu
                float mx;
                (void)lane_argmax_f(ratio, &mx);
                const float thr = 0.5f * (mx + fminf(a * inv_sumd, mx));
                const float w = (own && ratio >= thr) ? a2 : 0.f;
                sel = pick_scan(lane_scan(w), w, u);
            }
            if (sel < 0) {
                conv = true;  // every residual is exactly zero
                break;
            }
            const float2 g = make_float2(__shfl_sync(KZ_FULL, ph.x, sel), __shfl_sync(KZ_FULL, ph.y, sel));
            if (lane == sel) {
                q.x += g.x;
                q.y += g.y;
            }
            const float2* hs = Hd + (size_t)sel * Ntp;
#pragma unroll
            for (int a = 0; a < AU; ++a) {
                const int n = tid + a * SNT;
                if (n < Ntp) {
                    const float2 hh = hs[n];
                    m[a].x = fmaf(g.x, hh.x, fmaf(g.y, hh.y, m[a].x));
                    m[a].y = fmaf(g.y, hh.x, fmaf(-g.x, hh.y, m[a].y));
                }
            }
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
            resid(allmask);
            const float a = rnorm(allmask);
            if (bad(a)) {
                numeric = true;
                break;
            }
            if (a <= tol2f && confirm() <= tol2f) {
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
            if (fmask) {  // orthogonal half-step: unit steps on F, one gather (disjoint VRs)
                resid(fmask);
                const bool inF = own && ((fmask >> lane) & 1u);
                const float2 g = inF ? ph : make_float2(0.f, 0.f);
                if (inF) {
                    q.x += g.x;
                    q.y += g.y;
                }
                float2 u[AU];
                gather(g, u);
#pragma unroll
                for (int a = 0; a < AU; ++a) {
                    m[a].x += u[a].x;
                    m[a].y += u[a].y;
                }
            }
            if (vmask) resid(vmask);
            const float a = rnorm(vmask);
            if (bad(a)) {
                numeric = true;
                break;
            }
            if (a <= tol2f && confirm() <= tol2f) {
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
    // outputs: x = H^H q, the true residual, v = q (scaled back exactly)
    const float rn2 = (zero || numeric) ? 0.f : confirm();
#pragma unroll
    for (int a = 0; a < AU; ++a) {
        const int n = tid + a * SNT;
        if (n < Nt) I.x[(size_t)col * Nt + n] = zero ? make_float2(0.f, 0.f) : make_float2(m[a].x * unsc, m[a].y * unsc);
    }
    if (I.v && warp == 0 && own) I.v[(size_t)col * K + lane] = make_float2(q.x * unsc, q.y * unsc);
    if (tid == 0) {
        I.iters[col] = t;
        I.resid[col] = zero ? 0.0 : (numeric ? (double)NAN : sqrt((double)rn2 / sn2s));
        if (numeric || bad(rn2)) kz_flag(L.status, KZ_STATUS_BIT_NUMERIC);
        else if (!conv) kz_flag(L.status, KZ_STATUS_BIT_NOT_CONVERGED);
    }
}

}  // namespace

size_t kz_smem_small(int K, int Ntp) { return (size_t)(K + 1) * Ntp * sizeof(float2); }

cudaError_t kz_launch_small(const KzLaunch& L, int grid, size_t smem, cudaStream_t st) {
    auto go = [&](auto kern) -> cudaError_t {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<grid, SNT, smem, st>>>(L);
        return cudaGetLastError();
    };
    const int K = L.single.K, Ntp = L.single.Ntp;
    const bool rk = (L.algo == KZ_RK_ENERGY || L.algo == KZ_RK_UNIFORM || L.algo == KZ_RK_SWOR);
    if (!rk && K <= 16 && Ntp <= SNT) return go(kz_small_reg_kernel<16, 1>);
    if (!rk && K <= 16 && Ntp <= 2 * SNT) return go(kz_small_reg_kernel<16, 2>);
    if (!rk && K <= 32 && Ntp <= SNT) return go(kz_small_reg_kernel<32, 1>);
    return go(kz_small_kernel);
}
