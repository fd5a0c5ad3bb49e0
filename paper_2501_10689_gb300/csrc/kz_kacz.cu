// Persistent RK / GRK / VR-OGRK solver (steps A1-A3 and A7).
//
// One CTA owns one work item (one channel, J right-hand-side columns); m
// stays in shared memory.  Each column runs its own sequence of single-row
// projections (eq. (update)):
//
//   residuals  GRK: every row (Sec. IV-A);  VR-OGRK: only rows of
//              X_{i(t-1)} (Alg. 2 step 8; the others keep their value by
//              Theorem 2), starting from r = s;  RK: only the drawn row, plus
//              every row each K steps for the stopping test;
//   selection  one warp per column: RK draws p_i = d_i / sum d or 1/K;
//              SWOR-ERK draws p_i proportional to d_i over the rows not yet
//              drawn in the current sweep of K steps (without replacement);
//              GRK / VR-OGRK use the PAPER, BAIWU or ARGMAX rule;
//   projection gamma = r_i / d_i,  m[Gamma_i] += gamma conj(h_i),  q_i += gamma
//              (Alg. 1 steps 9-11).
//
// Different columns may select different rows in the same step; each column
// updates only its own m column, so the projections never conflict.
#include "kz_device.cuh"

namespace {

template <int J, int NW>
__global__ void __launch_bounds__(NW * 32) kz_kacz_kernel(const __grid_constant__ KzLaunch L) {
    extern __shared__ __align__(16) unsigned char kz_smem[];
    __shared__ KzInst sI;
    __shared__ double s_sn2[J];
    __shared__ float2 s_gam[J];
    __shared__ int s_sel[J];
    __shared__ int s_iters[J];
    __shared__ int s_active;
    __shared__ int s_pending;
    __shared__ int s_full;
    __shared__ int s_item;
    __shared__ double s_sumd;
    __shared__ double s_partd[NW][J];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NT = NW * 32;
    float2* m_s = reinterpret_cast<float2*>(kz_smem);
    float2* b_s = m_s + (size_t)J * L.Ntp_max;
    float2* q_s = b_s + (size_t)L.K_max * J;
    float2* r_s = q_s + (size_t)L.K_max * J;
    float* d_s = reinterpret_cast<float*>(r_s + (size_t)L.K_max * J);
    int* stamp = reinterpret_cast<int*>(d_s + L.K_max);
    int* swor = stamp + L.K_max;  // [K][J]: the sweep in which (row, column) was last drawn
    const int algo = L.algo;
    const bool is_rk = (algo == KZ_RK_ENERGY || algo == KZ_RK_UNIFORM || algo == KZ_RK_SWOR);
    const bool ogrk = (algo == KZ_VR_OGRK);

    int static_item = blockIdx.x;
    for (;;) {
        if (tid == 0) s_item = L.queue ? atomicAdd(L.queue, 1) : static_item;
        static_item += gridDim.x;
        __syncthreads();
        const int item = s_item;
        if (item >= L.n_items) break;
        int2 it;
        if (L.insts) {
            it = L.items[item];
            load_inst(sI, L.insts + it.x);
        } else {
            it = make_int2(0, item * J);
            load_inst(sI, &L.single);
        }
        __syncthreads();
        const KzInst& I = sI;
        const int K = I.K, Nt = I.Nt, Ntp = I.Ntp;
        const int col0 = KZ_ITEM_COL(it.y), ncols = min(J, I.ld - col0);
        const float xi = I.xi;
        const int4* trow4 = I.trow4;

        for (int e = tid; e < J * Ntp; e += NT) m_s[e] = make_float2(0.f, 0.f);
        for (int e = tid; e < K * J; e += NT) {
            const int i = e / J, j = e % J;
            const float2 sv = (j < ncols) ? I.s[(size_t)(col0 + j) * K + i] : make_float2(0.f, 0.f);
            b_s[e] = sv;
            r_s[e] = sv;  // r = s at w = 0 (Alg. 2 step 3)
            q_s[e] = make_float2(0.f, 0.f);
        }
        for (int i = tid; i < K; i += NT) {
            d_s[i] = I.nrm[i] + xi;
            stamp[i] = -1;
        }
        for (int e = tid; e < K * J; e += NT) swor[e] = -1;
        __syncthreads();
        if (warp < J) {
            double a = 0.0;
            for (int i = lane; i < K; i += 32) {
                const float2 v = b_s[i * J + warp];
                a += (double)v.x * v.x + (double)v.y * v.y;
            }
            a = warp_sum_d(a);
            if (lane == 0) s_sn2[warp] = a;
        }
        if (warp == NW - 1) {  // ||B||_F^2 = sum_k ||h_k||^2 + K xi, in FP64
            double a = 0.0;
            for (int i = lane; i < K; i += 32) a += I.nrmd[i];
            a = warp_sum_d(a);
            if (lane == 0) s_sumd = a + (double)K * xi;
        }
        __syncthreads();
        if (tid == 0) {
            int act = 0;
            for (int j = 0; j < ncols; ++j) {
                s_iters[j] = L.max_iter;
                s_sel[j] = -1;
                if (s_sn2[j] > 0.0 && isfinite(s_sn2[j])) {
                    act |= 1 << j;
                } else {  // a zero column is solved by x = 0; a NaN / Inf one is reported
                    s_iters[j] = 0;
                    if (!(s_sn2[j] == 0.0)) kz_flag(L.status, KZ_STATUS_BIT_NUMERIC);
                }
            }
            s_active = act;
            s_pending = 0;
            s_full = 0;
        }
        __syncthreads();

        int t = 0, since_refresh = 0;
        while (s_active) {
            // ---------------- residual phase
            const bool full = (algo == KZ_GRK) || (is_rk && (t % K) == 0) || (ogrk && s_full);
            if (full) {
                for (int i = warp; i < K; i += NW) {
                    float2 acc[J];
                    row_dot<J, false>(I, I.rows, I.rptr, i, m_s, Ntp, acc);
                    if (lane == 0) {
#pragma unroll
                        for (int j = 0; j < J; ++j) {
                            const float2 bv = b_s[i * J + j], qv = q_s[i * J + j];
                            r_s[i * J + j] = make_float2(bv.x - acc[j].x - xi * qv.x, bv.y - acc[j].y - xi * qv.y);
                        }
                    }
                }
            } else if (ogrk && t > 0) {
                // stamp X_{i(t-1)} of every column, then recompute those rows
                for (int j = 0; j < ncols; ++j) {
                    const int sel = s_sel[j];
                    if (sel < 0) continue;
                    for (int k = I.xptr[sel] + tid; k < I.xptr[sel + 1]; k += NT) stamp[I.xidx[k]] = t;
                }
                __syncthreads();
                for (int i = warp; i < K; i += NW) {
                    if (stamp[i] != t) continue;
                    float2 acc[J];
                    row_dot<J, false>(I, I.rows, I.rptr, i, m_s, Ntp, acc);
                    if (lane == 0) {
#pragma unroll
                        for (int j = 0; j < J; ++j) {
                            const float2 bv = b_s[i * J + j], qv = q_s[i * J + j];
                            r_s[i * J + j] = make_float2(bv.x - acc[j].x - xi * qv.x, bv.y - acc[j].y - xi * qv.y);
                        }
                    }
                }
            }
            __syncthreads();
            if (tid == 0) s_full = 0;
            // ---------------- tentative stopping test (one warp per column)
            if (warp < ncols && ((s_active >> warp) & 1) && (!is_rk || (t % K) == 0)) {
                const int j = warp;
                double a = 0.0;
                for (int i = lane; i < K; i += 32) {
                    const float2 r = r_s[i * J + j];
                    a += (double)r.x * r.x + (double)r.y * r.y;
                }
                a = warp_sum_d(a);
                if (lane == 0) {
                    if (!(a == a) || isinf(a)) {
                        s_iters[j] = t;
                        kz_flag(L.status, KZ_STATUS_BIT_NUMERIC);
                        atomicAnd(&s_active, ~(1 << j));
                    } else if (a <= L.tol * L.tol * s_sn2[j]) {
                        atomicOr(&s_pending, 1 << j);
                    }
                }
            }
            __syncthreads();
            // ---------------- confirmation: m = H^H q, every residual recomputed
            // with compensated FP32 sums, then the test again on those residuals
            if (s_pending) {
                for (int tile = warp; tile < I.ntiles; tile += NW) {
                    float2 u0[J], u1[J];
                    tile_accum<J, false>(I, trow4, tile, I.tptr[tile], I.tptr[tile + 1], q_s, u0, u1);
                    const int n = tile * KZ_TILE + 2 * lane;
#pragma unroll
                    for (int j = 0; j < J; ++j) {
                        m_s[j * Ntp + n] = u0[j];
                        m_s[j * Ntp + n + 1] = u1[j];
                    }
                }
                __syncthreads();
                for (int i = warp; i < K; i += NW) {
                    float2 hi[J], lo[J];
                    row_dot_c<J>(I, I.rows, I.rptr, i, m_s, Ntp, hi, lo);
                    if (lane == 0) {
#pragma unroll
                        for (int j = 0; j < J; ++j)
                            r_s[i * J + j] = true_resid(b_s[i * J + j], hi[j], lo[j], q_s[i * J + j], xi);
                    }
                }
                since_refresh = 0;
                __syncthreads();
                if (warp < ncols && ((s_pending >> warp) & 1)) {
                    const int j = warp;
                    double a = 0.0;
                    for (int i = lane; i < K; i += 32) {
                        const float2 r = r_s[i * J + j];
                        a += (double)r.x * r.x + (double)r.y * r.y;
                    }
                    a = warp_sum_d(a);
                    if (lane == 0 && a <= L.tol * L.tol * s_sn2[j]) {
                        s_iters[j] = t;
                        atomicAnd(&s_active, ~(1 << j));
                    }
                }
                __syncthreads();
                if (tid == 0) s_pending = 0;
                __syncthreads();
            }
            // ---------------- selection and the dual update (one warp per column)
            if (warp < ncols) {
                const int j = warp;
                int sel = -1;
                float2 gam = make_float2(0.f, 0.f);
                if ((s_active >> j) & 1) {
                    if (t >= L.max_iter) {
                        if (lane == 0) {
                            kz_flag(L.status, KZ_STATUS_BIT_NOT_CONVERGED);
                            atomicAnd(&s_active, ~(1 << j));
                        }
                    } else {
                        const double u = kz_uniform(L.seed, I.inst, col0 + j, t);
                        float2 r;
                        if (is_rk) {
                            if (algo == KZ_RK_ENERGY) {
                                sel = warp_pick(K, u, [&](int i) { return (double)d_s[i]; });
                            } else if (algo == KZ_RK_SWOR) {
                                const int sweep = t / K;
                                sel = warp_pick(K, u, [&](int i) {
                                    return swor[i * J + j] == sweep ? 0.0 : (double)d_s[i];
                                });
                                if (lane == 0 && sel >= 0) swor[sel * J + j] = sweep;
                            } else {
                                sel = warp_pick(K, u, [&](int i) { return 1.0; });
                            }
                            // no positive weight (every d_i NaN): sel < 0 stops the column below
                            const int4 rd = sel >= 0 ? I.rows[sel] : make_int4(0, 0, 0, 0);
                            const int base = sel >= 0 ? I.rptr[sel] : 0;
                            float ax = 0.f, ay = 0.f;
                            for (int p = 2 * lane; p < rd.y; p += 64) {
                                const float4 h = h_pair<false>(I, base + p);
                                const float4 mm = *reinterpret_cast<const float4*>(m_s + j * Ntp + rd.x + p);
                                ax = fmaf(h.x, mm.x, fmaf(-h.y, mm.y, fmaf(h.z, mm.z, fmaf(-h.w, mm.w, ax))));
                                ay = fmaf(h.x, mm.y, fmaf(h.y, mm.x, fmaf(h.z, mm.w, fmaf(h.w, mm.z, ay))));
                            }
                            ax = warp_sum(ax);
                            ay = warp_sum(ay);
                            const float2 bv = sel >= 0 ? b_s[sel * J + j] : make_float2(0.f, 0.f);
                            const float2 qv = sel >= 0 ? q_s[sel * J + j] : make_float2(0.f, 0.f);
                            r = make_float2(bv.x - ax - xi * qv.x, bv.y - ay - xi * qv.y);
                        } else {
                            if (L.sel == KZ_SEL_ARGMAX) {
                                sel = warp_argmax(K, [&](int i) {
                                    const float2 rr = r_s[i * J + j];
                                    return ((double)rr.x * rr.x + (double)rr.y * rr.y) / (double)d_s[i];
                                }, nullptr);
                            } else if (L.sel == KZ_SEL_PAPER) {
                                sel = warp_pick(K, u, [&](int i) {
                                    const float2 rr = r_s[i * J + j];
                                    return (double)rr.x * rr.x + (double)rr.y * rr.y;
                                });
                            } else {
                                // Bai-Wu greedy set: ratio_i >= (max_ratio + min(||r||^2 / ||B||_F^2, max_ratio)) / 2
                                double mx = 0.0;
                                (void)warp_argmax(K, [&](int i) {
                                    const float2 rr = r_s[i * J + j];
                                    return ((double)rr.x * rr.x + (double)rr.y * rr.y) / (double)d_s[i];
                                }, &mx);
                                double a = 0.0;
                                for (int i = lane; i < K; i += 32) {
                                    const float2 rr = r_s[i * J + j];
                                    a += (double)rr.x * rr.x + (double)rr.y * rr.y;
                                }
                                a = warp_sum_d(a);
                                const double thr = 0.5 * (mx + fmin(a / s_sumd, mx));
                                sel = warp_pick(K, u, [&](int i) {
                                    const float2 rr = r_s[i * J + j];
                                    const double a2 = (double)rr.x * rr.x + (double)rr.y * rr.y;
                                    return (a2 / (double)d_s[i] >= thr) ? a2 : 0.0;
                                });
                            }
                            r = (sel >= 0) ? r_s[sel * J + j] : make_float2(0.f, 0.f);
                        }
                        if (sel < 0) {  // every weight zero: the residual is already zero
                            if (lane == 0) {
                                s_iters[j] = t;
                                atomicAnd(&s_active, ~(1 << j));
                            }
                        } else {
                            const float di = d_s[sel];
                            gam = make_float2(r.x / di, r.y / di);
                            if (lane == 0) {
                                q_s[sel * J + j].x += gam.x;
                                q_s[sel * J + j].y += gam.y;
                            }
                        }
                    }
                }
                if (lane == 0) {
                    s_sel[j] = sel;
                    s_gam[j] = gam;
                    if (L.hist_row && t < L.hist_T) {  // the selected-row history (step t, this column)
                        L.hist_row[(size_t)t * L.hist_ld + col0 + j] = sel;
                        L.hist_gam[(size_t)t * L.hist_ld + col0 + j] = gam;
                    }
                }
            }
            __syncthreads();
            if (!s_active) break;
            // ---------------- projection of each column onto its selected row
            for (int j = 0; j < ncols; ++j) {
                const int sel = s_sel[j];
                if (sel < 0) continue;
                const float2 g1[1] = {s_gam[j]};
                row_axpy<1, false>(I, I.rows, I.rptr, sel, m_s + j * Ntp, Ntp, g1, tid, NT);
            }
            ++t;
            ++since_refresh;
            __syncthreads();
            if (L.refresh > 0 && since_refresh >= L.refresh) {
                since_refresh = 0;
                for (int tile = warp; tile < I.ntiles; tile += NW) {
                    float2 u0[J], u1[J];
                    tile_accum<J, false>(I, trow4, tile, I.tptr[tile], I.tptr[tile + 1], q_s, u0, u1);
                    const int n = tile * KZ_TILE + 2 * lane;
#pragma unroll
                    for (int j = 0; j < J; ++j) {
                        m_s[j * Ntp + n] = u0[j];
                        m_s[j * Ntp + n + 1] = u1[j];
                    }
                }
                if (tid == 0) s_full = 1;  // VR-OGRK: carried residuals refer to the old m
                __syncthreads();
            }
        }

        // ---- finalise: x = H^H q, true residual with compensated FP32 sums
        for (int tile = warp; tile < I.ntiles; tile += NW) {
            float2 u0[J], u1[J];
            tile_accum<J, false>(I, trow4, tile, I.tptr[tile], I.tptr[tile + 1], q_s, u0, u1);
            const int n = tile * KZ_TILE + 2 * lane;
#pragma unroll
            for (int j = 0; j < J; ++j) {
                m_s[j * Ntp + n] = u0[j];
                m_s[j * Ntp + n + 1] = u1[j];
            }
        }
        __syncthreads();
        {
            float rp[J];
#pragma unroll
            for (int j = 0; j < J; ++j) rp[j] = 0.f;
            for (int i = warp; i < K; i += NW) {
                float2 hi[J], lo[J];
                row_dot_c<J>(I, I.rows, I.rptr, i, m_s, Ntp, hi, lo);
#pragma unroll
                for (int j = 0; j < J; ++j) {
                    const float2 r = true_resid(b_s[i * J + j], hi[j], lo[j], q_s[i * J + j], xi);
                    rp[j] += r.x * r.x + r.y * r.y;
                }
            }
            if (lane == 0) {
#pragma unroll
                for (int j = 0; j < J; ++j) s_partd[warp][j] = rp[j];
            }
        }
        for (int j = 0; j < ncols; ++j) {
            float2* xc = I.x + (size_t)(col0 + j) * Nt;
            for (int n = tid; n < Nt; n += NT) xc[n] = m_s[j * Ntp + n];
            if (I.v) {
                float2* vc = I.v + (size_t)(col0 + j) * K;
                for (int i = tid; i < K; i += NT) vc[i] = q_s[i * J + j];
            }
        }
        __syncthreads();
        if (tid < ncols) {
            double rn2 = 0.0;
            for (int w = 0; w < NW; ++w) rn2 += s_partd[w][tid];
            const double sn2 = s_sn2[tid];
            I.resid[col0 + tid] = sn2 > 0.0 ? sqrt(rn2 / sn2) : 0.0;
            I.iters[col0 + tid] = s_iters[tid];
            if (!(rn2 == rn2)) kz_flag(L.status, KZ_STATUS_BIT_NUMERIC);
        }
        __syncthreads();
    }
}

template <int J, int NW>
cudaError_t launch_t(const KzLaunch& L, int grid, size_t smem, cudaStream_t st) {
    auto k = kz_kacz_kernel<J, NW>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, NW * 32, smem, st>>>(L);
    return cudaGetLastError();
}

template <int J, int NW>
int occ_t(size_t smem) {
    auto k = kz_kacz_kernel<J, NW>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, NW * 32, smem) != cudaSuccess) return 0;
    return n;
}

template <int NW>
cudaError_t launch_j(const KzLaunch& L, int J, int grid, size_t smem, cudaStream_t st) {
    switch (J) {
        case 1: return launch_t<1, NW>(L, grid, smem, st);
        case 2: return launch_t<2, NW>(L, grid, smem, st);
        case 4: return launch_t<4, NW>(L, grid, smem, st);
        case 8: return launch_t<8, NW>(L, grid, smem, st);
        default: return cudaErrorInvalidValue;
    }
}

template <int NW>
int occ_j(int J, size_t smem) {
    switch (J) {
        case 1: return occ_t<1, NW>(smem);
        case 2: return occ_t<2, NW>(smem);
        case 4: return occ_t<4, NW>(smem);
        case 8: return occ_t<8, NW>(smem);
        default: return 0;
    }
}

}  // namespace

size_t kz_smem_kacz(int J, int Ntp, int K) {
    return (size_t)J * Ntp * sizeof(float2) + 3 * (size_t)K * J * sizeof(float2) + (size_t)K * sizeof(float) +
           (size_t)K * sizeof(int) + (size_t)K * J * sizeof(int) + 16;
}

cudaError_t kz_launch_kacz(const KzLaunch& L, int J, int nw, int grid, size_t smem, cudaStream_t st) {
    if (nw == 8) return launch_j<8>(L, J, grid, smem, st);
    if (nw == 16) return launch_j<16>(L, J, grid, smem, st);
    return cudaErrorInvalidValue;
}

int kz_occupancy_kacz(int J, int nw, size_t smem) {
    if (nw == 8) return occ_j<8>(J, smem);
    if (nw == 16) return occ_j<16>(J, smem);
    return 0;
}
