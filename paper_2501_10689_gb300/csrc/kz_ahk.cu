// Persistent AHK / VR-OAHK solver (steps A1, A4-A7 and A9).
//
// One CTA owns one work item: one channel and J of its right-hand-side
// columns.  The iterate m (J x Ntp complex) lives in shared memory for the
// whole solve; only H is streamed from L2 / HBM.  Per iteration of Alg. 3:
//
//   F half-step (eq. (updateor), unit step of Prop. 1): one warp per row of
//     the orthogonal set computes r_i = b_i - h_i . m - xi q_i, then
//     m += (r_i / d_i) conj(h_i) on its VR and q_i += r_i / d_i.  F rows have
//     disjoint VRs, so warps never touch the same m entries.
//   V half-step (eq. (updatenor)): one warp per V row computes r_i and
//     phi_i = r_i / d_i; the aggregate u = H_V^H phi_V is formed antenna-major
//     (each thread owns an antenna pair and loops over the covering V rows of
//     its 64-antenna tile, no scatter); gamma = phi^H r / (||u||^2 + xi ||phi||^2);
//     m += gamma u, q_V += gamma phi_V.
// AHK (eq. (update4) with eq. (coefficient)) is the V half-step over every row.
//
// The right-hand side of the row equations is b (= s for C64).  In BF16_MIXED
// the iteration reads the BF16 copy of H and works in correction form: at
// each refresh m_ref = H^H q and b = s - H m_ref are recomputed from the
// complex64 H (compensated FP32 sums), m restarts at 0, so the inner residual
// b - H_bf16 m - xi q differs from the true one only by (H - H_bf16) times the
// correction.  The refresh's true residual drives the stopping test.
//
// The tensor-core mode (MODE 2) runs the same correction form on the
// complex64 H, with the two contractions of every iteration on the tensor
// cores (FP16 products, FP32 sums): the V-row residuals as 8-row blocks
// (rows sorted by VR centre, so a block's rows share most of their union
// interval) and the aggregate H_V^H phi per tile.  They read the plan's FP16
// copy of H (row k scaled by 1 / hs_k, a power of two at or above ||h_k||),
// half the bytes of complex64.  The F half-step, the refresh and every
// stopping decision stay in FP32 on the CUDA cores and the complex64 H.  Its
// correction m is held in FP16 as m / sigma_j (sigma_j: the column's relative
// residual at the last refresh times an estimate of the RMS of H^H D^-1 s_j,
// fixed between refreshes), half the shared memory of FP32, so eight columns
// of a 4096-antenna channel fit one CTA, and read by the MMAs as stored.
#include "kz_device.cuh"

namespace {

constexpr int ALGO_OAHK = KZ_VR_OAHK;

// MODE 0: complex64, FP32 CUDA-core products; 1: BF16_MIXED (correction
// form on the BF16 copy); 2: tensor-core correction form on complex64.
template <int J, int NW, int MODE>
__global__ void __launch_bounds__(NW * 32, (J <= 2 ? 2 : 1) * (512 / (NW * 32))) kz_ahk_kernel(const __grid_constant__ KzLaunch L) {
    constexpr bool BF16 = (MODE == 1);
    constexpr bool TC = (MODE == 2);
    constexpr bool CORR = (MODE != 0);  // correction form with periodic refresh
    static_assert(!TC || J == 4 || J == 8, "tensor-core mode takes 4 or 8 columns");
    extern __shared__ __align__(16) unsigned char kz_smem[];
    __shared__ KzInst sI;
    // per column: ||r_V||^2, phi^H r, ||phi||^2 and (tensor-core mode) the
    // sum of hs_i^2 |phi_i|^2 that scales phi for the FP16 products
    __shared__ float s_part[NW][4 * J];
    __shared__ float s_tot[4 * J];
    __shared__ float s_partd[NW][J];  // per-warp sums of |r|^2 of the true residual
    __shared__ double s_sn2[J];
    __shared__ double s_thr[J];  // tol^2 ||s_j||^2
    __shared__ float s_isn2[J];  // 1 / ||s_j||^2 (tensor-core mode: the storage scale)
    __shared__ int s_conf[J];    // the true residual passed the test at the last refresh
    __shared__ float s_sn2f[J];  // ||s_j||^2 tol^2 for the tentative test
    __shared__ float s_rn2[J];
    __shared__ float s_gamma[J];
    __shared__ float s_kap[J];  // tensor-core mode: RMS of H^H D^-1 s_j
    __shared__ float s_sig[J];  // tensor-core mode: storage scale of column j of m
    __shared__ int s_iters[J];
    __shared__ int s_wait[J];  // iterations a column spent waiting for its confirmation
    __shared__ int s_active;
    __shared__ int s_pending;
    __shared__ int s_item;
    // tensor-core mode, F half-step: the rows of the orthogonal set cut into
    // at most FCAP chunks of whole 256-entry steps {F index, first entry, end,
    // first chunk of the row | end chunk << 16}, dealt to all warps
    constexpr int FCAP = TC ? 2 * NW : 1;
    __shared__ int4 fch_s[FCAP];
    __shared__ float2 fpart_s[FCAP][J];  // partial dots per chunk
    __shared__ float2 fb_s[FCAP][J];     // b - xi q of every F row
    __shared__ int s_nfch;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NT = NW * 32;
    // shared-memory carve-up: every array starts at a 16-byte aligned offset
    // (the int4 descriptors and the float4 iterate loads need it)
    size_t off = 0;
    auto carve = [&](size_t bytes) {
        unsigned char* p = kz_smem + off;
        off += (bytes + 15) & ~(size_t)15;
        return p;
    };
    // iterate columns; the tensor-core mode pads each by KZ_TC_PAD entries so
    // the columns read by one MMA fragment fall in different banks
    // (FP16 pairs in the tensor-core mode)
    float2* m_s = reinterpret_cast<float2*>(
        carve((L.m_elems ? (size_t)L.m_elems : (size_t)J * (L.Ntp_max + (TC ? KZ_TC_PAD : 0))) *
              (TC ? sizeof(__half2) : sizeof(float2))));
    __half2* m16 = reinterpret_cast<__half2*>(m_s);
    float2* b_s = reinterpret_cast<float2*>(carve((size_t)L.K_max * J * sizeof(float2)));
    float2* q_s = reinterpret_cast<float2*>(carve((size_t)L.K_max * J * sizeof(float2)));
    float2* p_s = reinterpret_cast<float2*>(carve((size_t)L.K_max * J * sizeof(float2)));
    float* d_s = reinterpret_cast<float*>(carve((size_t)L.K_max * sizeof(float)));
    // per-channel descriptors staged once per item (no dependent global loads
    // in front of every row): row intervals, offsets, solve order, 1 / d
    int4* rows_s = reinterpret_cast<int4*>(carve((size_t)L.K_max * sizeof(int4)));
    int* rptr_s = reinterpret_cast<int*>(carve((size_t)L.K_max * sizeof(int)));
    int* order_s = reinterpret_cast<int*>(carve((size_t)L.K_max * sizeof(int)));
    float* dinv_s = reinterpret_cast<float*>(carve((size_t)L.K_max * sizeof(float)));
    int* tptr_s = reinterpret_cast<int*>(carve((size_t)(L.Ntp_max / KZ_TILE + 1) * sizeof(int)));
    int* tnv_s = reinterpret_cast<int*>(carve((size_t)(L.Ntp_max / KZ_TILE) * sizeof(int)));
    int* vs_s = TC ? reinterpret_cast<int*>(carve((size_t)L.K_max * sizeof(int))) : nullptr;
    // correction form: CSR offsets of the overlap sets (the refresh's row passes)
    int* xptr_s = CORR ? reinterpret_cast<int*>(carve((size_t)(L.K_max + 1) * sizeof(int))) : nullptr;
    float* hs_s = TC ? reinterpret_cast<float*>(carve((size_t)L.K_max * sizeof(float))) : nullptr;  // FP16 row scales
    // tensor-core V residual: every 8-row block's union interval is cut in
    // two parts (tasks); part 0 sums into p_s, part 1 into pb_s, and the two
    // are added in that order.  Tasks are dealt to warps largest first, each
    // to the least loaded warp (fixed per item, so results are reproducible).
    const int ntask_max = TC ? 2 * ((L.K_max + 7) / 8) : 0;
    float2* pb_s = TC ? reinterpret_cast<float2*>(carve((size_t)L.K_max * J * sizeof(float2))) : nullptr;
    int4* task_s = TC ? reinterpret_cast<int4*>(carve((size_t)ntask_max * sizeof(int4))) : nullptr;
    int* tcost_s = TC ? reinterpret_cast<int*>(carve((size_t)ntask_max * sizeof(int))) : nullptr;
    int* wlist_s = TC ? reinterpret_cast<int*>(carve((size_t)ntask_max * sizeof(int))) : nullptr;
    __shared__ int s_wptr[NW + 1];
    // tensor-core aggregate: the row index of every covering-list entry of the
    // channel, staged once per item (the intervals and offsets come from
    // rows_s / rptr_s), so no list entry is read from L2 in the iteration
    unsigned short* trow_s =
        (TC && L.trow_max) ? reinterpret_cast<unsigned short*>(carve((size_t)L.trow_max * sizeof(unsigned short)))
                           : nullptr;
    const bool oahk = (L.algo == ALGO_OAHK);

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
        const int K = I.K, Nt = I.Nt, Ntp = I.Ntp, nF = oahk ? I.nF : 0;
        const int MS = TC ? Ntp + KZ_TC_PAD : Ntp;  // column stride of m_s
        // an item may be narrower than J (W columns): a wide channel whose J
        // iterate columns would not fit shared memory
        const int W = KZ_ITEM_WIDTH(it.y, J);
        const int col0 = KZ_ITEM_COL(it.y), ncols = min(W, I.ld - col0);
        const float xi = I.xi;
        const int4* trow4 = I.trow4;
        // x holds u between the aggregate and its application; whole 128-byte
        // lines of the item's columns may be dropped from L2 after that
        const bool xdisc = (Nt & 15) == 0 && ((reinterpret_cast<uintptr_t>(I.x + (size_t)col0 * Nt) & 127) == 0);
        // True residual s - H H^H q - xi q of every row: per-warp sums of |r|^2
        // per column into s_partd; with store_b also the correction right-hand
        // side b = s - H H^H q.  In correction form through the Gram matrix on
        // the overlap pattern (one pass over each row's overlap set, not its
        // VR); in MODE 0 through the iterate m = H^H q just recomputed in m_s,
        // the quantity the iteration itself carries (on ill-conditioned
        // channels the two FP32 routes differ near 1e-7).  Four or eight
        // columns: two rows per warp at a time and a compensated
        // reduce-scatter, the s entries each lane needs fetched first.
        auto true_residual_pass = [&](bool store_b) {
            if constexpr (CORR) {
                // rows i and i + NW of a warp together (rows warp, warp + NW,
                // warp + 2 NW, ... in that order); lanes j < J own column j
                // (its s entries are fetched before the rows' sums)
                float rpl = 0.f;
                const int j = lane % J;
                for (int i0 = warp; i0 < K; i0 += 2 * NW) {
                    const int i1 = i0 + NW < K ? i0 + NW : -1;
                    const bool mine = lane < J && j < ncols;
                    const float2 sv0 = mine ? I.s[(size_t)(col0 + j) * K + i0] : make_float2(0.f, 0.f);
                    const float2 sv1 = (mine && i1 >= 0) ? I.s[(size_t)(col0 + j) * K + i1] : make_float2(0.f, 0.f);
                    float2 hi[2], lo[2];
                    gram_rows_t<J>(I, xptr_s, i0, i1, q_s, W, hi, lo);
                    if (lane < J) {
#pragma unroll
                        for (int r = 0; r < 2; ++r) {
                            const int i = r ? i1 : i0;
                            if (i < 0) continue;
                            const float2 sv = r ? sv1 : sv0;
                            const float2 rr = true_resid(sv, hi[r], lo[r], q_s[i * J + j], xi);
                            rpl += rr.x * rr.x + rr.y * rr.y;
                            if (store_b)
                                b_s[i * J + j] = make_float2((sv.x - hi[r].x) - lo[r].x, (sv.y - hi[r].y) - lo[r].y);
                        }
                    }
                }
                if (lane < J) s_partd[warp][lane] = rpl;
            } else if constexpr (J >= 4) {
                constexpr int LPV = 32 / (4 * J);
                const int idx = lane / LPV;
                const int mw = idx / (2 * J), mj = (idx % (2 * J)) / 2;
                const bool slot = (idx % 2 == 0) && (lane % LPV == 0);
                float rpl = 0.f;
                for (int k = warp; k < K; k += 2 * NW) {
                    const int i0 = k, i1 = (k + NW < K) ? k + NW : -1;
                    const int i = mw ? i1 : i0;
                    const bool mine = slot && i >= 0;
                    const float2 sv = (mine && mj < ncols) ? I.s[(size_t)(col0 + mj) * K + i] : make_float2(0.f, 0.f);
                    float2 hi, lo;
                    int which, jj;
                    bool own;
                    row_dot_c2<J>(I, rows_s, rptr_s, i0, i1, m_s, MS, W, hi, lo, which, jj, own);
                    if (mine) {
                        const float2 r = true_resid(sv, hi, lo, q_s[i * J + mj], xi);
                        rpl += r.x * r.x + r.y * r.y;
                        if (store_b) b_s[i * J + mj] = make_float2((sv.x - hi.x) - lo.x, (sv.y - hi.y) - lo.y);
                    }
                }
#pragma unroll
                for (int j = 0; j < J; ++j) {
                    const float t = warp_sum(mj == j ? rpl : 0.f);
                    if (lane == 0) s_partd[warp][j] = t;
                }
            } else {
                float rp[J];
#pragma unroll
                for (int j = 0; j < J; ++j) rp[j] = 0.f;
                for (int i = warp; i < K; i += NW) {
                    float2 hi[J], lo[J];
                    row_dot_c<J>(I, rows_s, rptr_s, i, m_s, MS, hi, lo, W);
#pragma unroll
                    for (int j = 0; j < J; ++j) {
                        const float2 sv = (j < ncols) ? I.s[(size_t)(col0 + j) * K + i] : make_float2(0.f, 0.f);
                        const float2 r = true_resid(sv, hi[j], lo[j], q_s[i * J + j], xi);
                        rp[j] += r.x * r.x + r.y * r.y;
                        if (store_b && lane == 0)
                            b_s[i * J + j] = make_float2((sv.x - hi[j].x) - lo[j].x, (sv.y - hi[j].y) - lo[j].y);
                    }
                }
                if (lane == 0) {
#pragma unroll
                    for (int j = 0; j < J; ++j) s_partd[warp][j] = rp[j];
                }
            }
        };

        // ---- initialise: m = 0, q = 0, b = s, d = ||h||^2 + xi
        if (TC)
            for (int e = tid; e < W * MS; e += NT) reinterpret_cast<unsigned*>(m16)[e] = 0u;
        else
            for (int e = tid; e < W * MS; e += NT) m_s[e] = make_float2(0.f, 0.f);
        for (int e = tid; e < K * J; e += NT) {
            const int i = e / J, j = e % J;
            b_s[e] = (j < ncols) ? I.s[(size_t)(col0 + j) * K + i] : make_float2(0.f, 0.f);
            q_s[e] = make_float2(0.f, 0.f);
            p_s[e] = make_float2(0.f, 0.f);
        }
        for (int i = tid; i < K; i += NT) {
            const float d = I.nrm[i] + xi;
            d_s[i] = d;
            dinv_s[i] = 1.f / d;
            rows_s[i] = I.rows[i];
            rptr_s[i] = I.rptr[i];
            order_s[i] = I.order[i];
            if (TC) hs_s[i] = I.hs[i];
        }
        if (CORR)
            for (int i = tid; i <= K; i += NT) xptr_s[i] = I.xptr[i];
        for (int t2 = tid; t2 <= I.ntiles; t2 += NT) {
            tptr_s[t2] = I.tptr[t2];
            if (t2 < I.ntiles) tnv_s[t2] = I.tnv[t2];
        }
        if (TC) {  // V rows by VR centre (all rows for AHK)
            const int* src = I.vsort + (oahk ? 0 : K - I.nF);
            for (int v = tid; v < K - nF; v += NT) vs_s[v] = src[v];
            if (trow_s)
                for (int e = tid; e < __ldg(I.tptr + I.ntiles); e += NT) trow_s[e] = (unsigned short)I.trow4[e].x;
        }
        __syncthreads();
        if (TC) {
            const int nv = K - nF, nblk = (nv + 7) >> 3;
            for (int b = tid; b < nblk; b += NT) {
                int lo = 0x7fffffff, hi = 0;
                for (int r = 8 * b; r < min(8 * b + 8, nv); ++r) {
                    const int4 rd = rows_s[vs_s[r]];
                    lo = min(lo, rd.x);
                    hi = max(hi, rd.x + rd.y);
                }
                const int lo16 = lo & ~15;
                const int steps = (hi - lo16 + 63) >> 6;  // steps of 64 antennas
                const int cut = lo16 + 64 * ((steps + 1) >> 1);
                task_s[2 * b] = make_int4(lo16, min(cut, hi), b, 0);
                task_s[2 * b + 1] = make_int4(cut, max(cut, hi), b, 1);
                tcost_s[2 * b] = (steps + 1) >> 1;
                tcost_s[2 * b + 1] = steps >> 1;
            }
            __syncthreads();
            // greedy longest-first assignment to warps: tasks ranked by
            // (cost descending, index ascending) in parallel into wlist_s,
            // then warp 0 gives each, in that order, to the least loaded
            // warp (lowest index on ties)
            const int nt = 2 * nblk;
            for (int t2 = tid; t2 < nt; t2 += NT) {
                const int c2 = tcost_s[t2];
                int rank = 0;
                for (int t3 = 0; t3 < nt; ++t3) {
                    const int c3 = tcost_s[t3];
                    rank += (c3 > c2) || (c3 == c2 && t3 < t2);
                }
                wlist_s[rank] = t2;
            }
            __syncthreads();
            if (warp == 0) {
                int load = 0, cnt = 0;  // of warp `lane` (lanes < NW)
                for (int q = 0; q < nt; ++q) {
                    const int t2 = wlist_s[q];
                    const int c2 = tcost_s[t2];
                    const int key = lane < NW ? (load << 5) | lane : 0x7fffffff;
                    const int w0 = __reduce_min_sync(KZ_FULL, key) & 31;
                    if (lane == w0) {
                        load += c2;
                        ++cnt;
                    }
                    __syncwarp();
                    if (lane == 0) tcost_s[t2] = -1 - w0;  // taken, by warp w0
                }
                int incl = cnt;  // prefix sums of the counts
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int v = __shfl_up_sync(KZ_FULL, incl, o);
                    if (lane >= o) incl += v;
                }
                if (lane < NW) s_wptr[lane + 1] = incl;
                if (lane == 0) s_wptr[0] = 0;
                __syncwarp();
            }
            if (tid == 0) {
                int cnt[NW];
                for (int w = 0; w < NW; ++w) cnt[w] = s_wptr[w];
                for (int t2 = 0; t2 < nt; ++t2) wlist_s[cnt[-1 - tcost_s[t2]]++] = t2;
                // F chunks: c steps each, c chosen so that the rows' chunks
                // number at most FCAP (a row has ceil(u / c) of them); only
                // when a row of three or more steps would hold one warp while
                // the others wait (with shorter rows the extra barrier costs
                // as much as the balance saves)
                int nch = 0;
                int U = 0, umax = 0;
                for (int f = 0; f < nF; ++f) {
                    const int u = (rows_s[order_s[f]].y + 255) >> 8;
                    U += u;
                    umax = max(umax, u);
                }
                if (oahk && nF > 0 && nF <= FCAP && umax >= 3) {
                    const int c = (nF == FCAP) ? max(1, umax) : max(1, (U + FCAP - nF - 1) / (FCAP - nF));
                    for (int f = 0; f < nF; ++f) {
                        const int u = max(1, (rows_s[order_s[f]].y + 255) >> 8);
                        const int c0 = nch;
                        for (int a = 0; a < u; a += c) fch_s[nch++] = make_int4(f, 256 * a, 256 * min(u, a + c), 0);
                        for (int k = c0; k < nch; ++k) fch_s[k].w = c0 | (nch << 16);
                    }
                }
                s_nfch = nch;
            }
            // the scale of the solution: kappa_j^2 = (1 / Nt) sum_i |s_ij|^2
            // ||h_i||^2 / d_i^2, the diagonal part of ||H^H D^-1 s_j||^2 (one
            // Jacobi step from 0; the storage scale only needs its order of
            // magnitude)
            if (warp < J) {
                float a = 0.f;
                for (int i = lane; i < K; i += 32) {
                    const float2 bv = b_s[i * J + warp];
                    const float di = dinv_s[i];
                    a += (bv.x * bv.x + bv.y * bv.y) * (d_s[i] - xi) * di * di;
                }
                a = warp_sum(a);
                if (lane == 0) {
                    const float kap = sqrtf(a / (float)Nt);
                    s_kap[warp] = (kap > 0.f && isfinite(kap)) ? kap : 1.f;
                    s_sig[warp] = s_kap[warp];
                }
            }
            __syncthreads();
        }
        if (warp < J) {
            double a = 0.0;
            for (int i = lane; i < K; i += 32) {
                const float2 v = b_s[i * J + warp];
                a += (double)v.x * v.x + (double)v.y * v.y;
            }
            a = warp_sum_d(a);
            if (lane == 0) {
                s_sn2[warp] = a;
                s_sn2f[warp] = (float)(a * L.tol * L.tol);
                s_thr[warp] = a * L.tol * L.tol;
                s_isn2[warp] = a > 0.0 ? (float)(1.0 / a) : 0.f;
            }
        }
        __syncthreads();
        if (tid == 0) {
            int act = 0;
            for (int j = 0; j < ncols; ++j) {
                s_iters[j] = L.max_iter;
                s_wait[j] = 0;
                if (s_sn2[j] > 0.0 && isfinite(s_sn2[j])) {
                    act |= 1 << j;
                } else {  // a zero column is solved by x = 0; a NaN / Inf one is reported
                    s_iters[j] = 0;
                    if (!(s_sn2[j] == 0.0)) kz_flag(L.status, KZ_STATUS_BIT_NUMERIC);
                }
            }
            s_active = act;
            s_pending = 0;
        }
        __syncthreads();

        int t = 0, since_refresh = 0;
        while (s_active) {
            // correction form: a column whose residual passed the test waits,
            // without stepping, for the next refresh to confirm it
            const int act = CORR ? (s_active & ~s_pending) : s_active;
            // ---------------- F half-step (VR-OAHK only)
            if (oahk) {
                ++t;
                const int nch = TC ? s_nfch : 0;
                if (TC && nch > 0) {
                    // chunked: partial dots of every chunk (the warp of a
                    // row's first chunk also keeps b - xi q of the row), then
                    // each chunk's step from its row's sum (chunks in order:
                    // the same sum in every warp of a row), the first chunk's
                    // warp updating q
                    for (int ch = warp; ch < nch; ch += NW) {
                        const int4 e = fch_s[ch];
                        const int i = order_s[e.x];
                        float2 acc[J];
                        row_dot_h<J>(I, rows_s, rptr_s, i, m16, MS, acc, W, e.y, e.z);
                        if (lane == 0) {
                            const bool first = (e.w & 0xffff) == ch;
#pragma unroll
                            for (int j = 0; j < J; ++j) {
                                fpart_s[ch][j] = acc[j];
                                if (first) {
                                    const float2 bv = b_s[i * J + j], qv = q_s[i * J + j];
                                    fb_s[e.x][j] = make_float2(bv.x - xi * qv.x, bv.y - xi * qv.y);
                                }
                            }
                        }
                    }
                    __syncthreads();
                    for (int ch = warp; ch < nch; ch += NW) {
                        const int4 e = fch_s[ch];
                        const int f = e.x, i = order_s[f], c0 = e.w & 0xffff, c1 = e.w >> 16;
                        const float di = d_s[i];
                        float2 g[J], gs[J];
#pragma unroll
                        for (int j = 0; j < J; ++j) {
                            float2 a = make_float2(0.f, 0.f);
                            for (int c = c0; c < c1; ++c) {
                                a.x += fpart_s[c][j].x;
                                a.y += fpart_s[c][j].y;
                            }
                            const float sg = s_sig[j];
                            const float2 bq = fb_s[f][j];
                            const float rx = bq.x - a.x * sg;
                            const float ry = bq.y - a.y * sg;
                            const bool on = (act >> j) & 1;
                            g[j] = on ? make_float2(rx / di, ry / di) : make_float2(0.f, 0.f);
                            gs[j] = make_float2(g[j].x / sg, g[j].y / sg);
                        }
                        row_axpy_h<J>(I, rows_s, rptr_s, i, m16, MS, gs, W, e.y, e.z);
                        if (ch == c0 && lane == 0) {
#pragma unroll
                            for (int j = 0; j < J; ++j) {
                                q_s[i * J + j].x += g[j].x;
                                q_s[i * J + j].y += g[j].y;
                            }
                        }
                    }
                }
                if constexpr (TC) {
                    // few short rows: each row's columns split between two
                    // warps (both read the row; no cross-warp sums)
                    constexpr int JH = J > 1 ? J / 2 : 1;
                    if (nch == 0 && 2 * nF <= NW && warp < 2 * nF) {
                        const int f = warp >> 1, j0 = (warp & 1) * JH;
                        const int i = order_s[f];
                        const int jn = min(JH, W - j0);
                        float2 acc[JH];
                        row_dot_h<JH>(I, rows_s, rptr_s, i, m16 + j0 * MS, MS, acc, jn, 0, 0x7fffffff);
                        const float di = d_s[i];
                        float2 g[JH], gs[JH];
#pragma unroll
                        for (int jj = 0; jj < JH; ++jj) {
                            const int j = j0 + jj;
                            const float sg = s_sig[j];
                            const float2 bv = b_s[i * J + j], qv = q_s[i * J + j];
                            const float rx = bv.x - acc[jj].x * sg - xi * qv.x;
                            const float ry = bv.y - acc[jj].y * sg - xi * qv.y;
                            const bool on = jj < jn && ((act >> j) & 1);
                            g[jj] = on ? make_float2(rx / di, ry / di) : make_float2(0.f, 0.f);
                            const float r = 1.f / sg;
                            gs[jj] = make_float2(g[jj].x * r, g[jj].y * r);
                        }
                        row_axpy_h<JH>(I, rows_s, rptr_s, i, m16 + j0 * MS, MS, gs, jn, 0, 0x7fffffff);
                        if (lane == 0) {
#pragma unroll
                            for (int jj = 0; jj < JH; ++jj) {
                                q_s[i * J + j0 + jj].x += g[jj].x;
                                q_s[i * J + j0 + jj].y += g[jj].y;
                            }
                        }
                    }
                }
                for (int f = (TC && (nch > 0 || 2 * nF <= NW)) ? nF : warp; f < nF; f += NW) {
                    const int i = order_s[f];
                    float2 acc[J];
                    if constexpr (TC) {
                        row_dot_h<J>(I, rows_s, rptr_s, i, m16, MS, acc, W, 0, 0x7fffffff);
#pragma unroll
                        for (int j = 0; j < J; ++j) {
                            acc[j].x *= s_sig[j];
                            acc[j].y *= s_sig[j];
                        }
                    } else {
                        row_dot<J, BF16>(I, rows_s, rptr_s, i, m_s, MS, acc, W);
                    }
                    float2 g[J];
                    const float di = d_s[i];
#pragma unroll
                    for (int j = 0; j < J; ++j) {
                        const float2 bv = b_s[i * J + j], qv = q_s[i * J + j];
                        const float rx = bv.x - acc[j].x - xi * qv.x;
                        const float ry = bv.y - acc[j].y - xi * qv.y;
                        const bool on = (act >> j) & 1;
                        g[j] = on ? make_float2(rx / di, ry / di) : make_float2(0.f, 0.f);
                    }
                    if constexpr (TC) {
                        float2 gs[J];
#pragma unroll
                        for (int j = 0; j < J; ++j) {
                            const float r = 1.f / s_sig[j];
                            gs[j] = make_float2(g[j].x * r, g[j].y * r);
                        }
                        row_axpy_h<J>(I, rows_s, rptr_s, i, m16, MS, gs, W, 0, 0x7fffffff);
                    } else {
                        row_axpy<J, BF16>(I, rows_s, rptr_s, i, m_s, MS, g, lane, 32, W);
                    }
                    if (lane == 0) {
#pragma unroll
                        for (int j = 0; j < J; ++j) {
                            q_s[i * J + j].x += g[j].x;
                            q_s[i * J + j].y += g[j].y;
                        }
                    }
                }
                __syncthreads();
            }
            // ---------------- V residual, phi = r / d and the scalars of the step
            const int v0 = nF, vcount = K - nF;
            float pr[J], pn[J], pp[J];
#pragma unroll
            for (int j = 0; j < J; ++j) pr[j] = pn[j] = pp[j] = 0.f;
            if constexpr (TC) {
                // 8-row blocks on the tensor cores, each in two parts
                {
                    const int g = lane >> 2, c = lane & 3;
                    for (int q = s_wptr[warp]; q < s_wptr[warp + 1]; ++q) {
                        const int4 tk = task_s[wlist_s[q]];
                        float d[4];
                        tc_row_part<J>(I.Hh, rows_s, rptr_s, vs_s, vcount, tk.z, tk.x, tk.y, m16, MS, W, d);
                        float2* dst = tk.w ? pb_s : p_s;
                        const int k = 8 * tk.z + 2 * c;
                        if (g < W) {  // true units: times the row's hs and the column's sigma
                            const float sg = s_sig[g];
                            if (k < vcount) {
                                const int r = vs_s[k];
                                const float f = sg * hs_s[r];
                                dst[r * J + g] = make_float2(d[0] * f, d[2] * f);
                            }
                            if (k + 1 < vcount) {
                                const int r = vs_s[k + 1];
                                const float f = sg * hs_s[r];
                                dst[r * J + g] = make_float2(d[1] * f, d[3] * f);
                            }
                        }
                    }
                }
                __syncthreads();
                // residuals, phi and the column sums; thread tid always has
                // column j = tid % J (J divides the block size)
                float spr = 0.f, spn = 0.f, spp = 0.f, sph = 0.f;
                const int j = tid % J;
                const bool on = (act >> j) & 1;
                for (int e = tid; e < vcount * J; e += NT) {
                    const int i = vs_s[e / J];
                    float2 ph = make_float2(0.f, 0.f);
                    if (j < W) {
                        const float2 p0 = p_s[i * J + j], p1 = pb_s[i * J + j];
                        const float2 bv = b_s[i * J + j], qv = q_s[i * J + j];
                        const float rx = bv.x - (p0.x + p1.x) - xi * qv.x;
                        const float ry = bv.y - (p0.y + p1.y) - xi * qv.y;
                        const float r2 = rx * rx + ry * ry;
                        const float di = dinv_s[i];
                        ph = on ? make_float2(rx * di, ry * di) : make_float2(0.f, 0.f);
                        spr += r2;
                        spn += on ? r2 * di : 0.f;
                        const float p2 = ph.x * ph.x + ph.y * ph.y;
                        spp += p2;
                        sph += p2 * (hs_s[i] * hs_s[i]);
                    }
                    p_s[i * J + j] = ph;
                }
#pragma unroll
                for (int o = J; o < 32; o <<= 1) {
                    spr += __shfl_xor_sync(KZ_FULL, spr, o);
                    spn += __shfl_xor_sync(KZ_FULL, spn, o);
                    spp += __shfl_xor_sync(KZ_FULL, spp, o);
                    sph += __shfl_xor_sync(KZ_FULL, sph, o);
                }
                if (lane < J) {
                    s_part[warp][lane] = spr;
                    s_part[warp][J + lane] = spn;
                    s_part[warp][2 * J + lane] = spp;
                    s_part[warp][3 * J + lane] = sph;
                }
            } else {
            // rows v and v + NW go to the same warp together (two loads streams)
            for (int v = warp; v < vcount; v += 2 * NW) {
                const int i0 = order_s[v0 + v];
                const int i1 = (v + NW < vcount) ? order_s[v0 + v + NW] : -1;
                float2 acc0[J], acc1[J];
                row_dot2<J, BF16>(I, rows_s, rptr_s, i0, i1, m_s, MS, acc0, acc1);
#pragma unroll
                for (int rr = 0; rr < 2; ++rr) {
                    const int i = rr ? i1 : i0;
                    if (i < 0) continue;
                    const float di = dinv_s[i];
#pragma unroll
                    for (int j = 0; j < J; ++j) {
                        const float2 a = rr ? acc1[j] : acc0[j];
                        const float2 bv = b_s[i * J + j], qv = q_s[i * J + j];
                        const float rx = bv.x - a.x - xi * qv.x;
                        const float ry = bv.y - a.y - xi * qv.y;
                        const float r2 = rx * rx + ry * ry;
                        const bool on = (act >> j) & 1;
                        const float2 ph = on ? make_float2(rx * di, ry * di) : make_float2(0.f, 0.f);
                        pr[j] += r2;
                        pn[j] += on ? r2 * di : 0.f;
                        pp[j] += ph.x * ph.x + ph.y * ph.y;
                        if (lane == 0) p_s[i * J + j] = ph;
                    }
                }
            }
            if (lane == 0) {
#pragma unroll
                for (int j = 0; j < J; ++j) {
                    s_part[warp][j] = pr[j];
                    s_part[warp][J + j] = pn[j];
                    s_part[warp][2 * J + j] = pp[j];
                }
            }
            }
            __syncthreads();
            if (tid < (TC ? 4 : 3) * J) {
                float a = 0.f;
                for (int w = 0; w < NW; ++w) a += s_part[w][tid];
                s_tot[tid] = a;
            }
            __syncthreads();
            // ---------------- stopping test on the residual at hand (tentative:
            // a column that passes is confirmed on the true residual first)
            if (tid == 0) {
                int a2 = s_active, pend = 0;
                for (int j = 0; j < ncols; ++j)
                    if (((a2 & ~act) >> j) & 1) ++s_wait[j];  // reported iterations count steps taken
                for (int j = 0; j < ncols; ++j) {
                    if (!((a2 >> j) & 1)) continue;
                    const float rn2 = s_tot[j];
                    if (!(rn2 == rn2) || isinf(rn2)) {
                        a2 &= ~(1 << j);
                        s_iters[j] = t - s_wait[j];
                        kz_flag(L.status, KZ_STATUS_BIT_NUMERIC);
                    } else if (rn2 <= s_sn2f[j]) {
                        pend |= 1 << j;
                    } else if (!oahk && t >= L.max_iter) {
                        a2 &= ~(1 << j);  // AHK: t steps done and still above tol
                        kz_flag(L.status, KZ_STATUS_BIT_NOT_CONVERGED);
                    }
                }
                s_active = a2;
                s_pending = pend;
            }
            __syncthreads();
            // ---------------- confirmation: m = H^H q from the complex64 H, the
            // true residual s - H m - xi q with compensated sums, and the test
            // again; in correction form also the refresh that sets b = s - H m
            // and restarts m at 0.  At once for a tentative stop in MODE 0; in
            // correction form when every active column waits, at the refresh
            // period, or at the last iteration.
            const bool last = t >= L.max_iter;
            if ((!CORR && s_pending) ||
                (CORR && ((s_pending && (s_pending == s_active || last)) || since_refresh >= L.refresh))) {
                since_refresh = 0;
                if (!CORR) {  // the iterate itself restarts from m = H^H q (drift correction)
                    for (int tile = warp; tile < I.ntiles; tile += NW) {
                        float2 u0[J], u1[J];
                        tile_accum<J, false>(I, trow4, tile, tptr_s[tile], tptr_s[tile + 1], q_s, u0, u1);
                        const int n = tile * KZ_TILE + 2 * lane;
#pragma unroll
                        for (int j = 0; j < J; ++j) {
                            if (j >= W) continue;
                            m_s[j * MS + n] = u0[j];
                            m_s[j * MS + n + 1] = u1[j];
                        }
                    }
                }
                __syncthreads();
                true_residual_pass(CORR);
                __syncthreads();
                if (tid < J) {  // the columns' squared residual norms and tests, one thread each
                    float a = 0.f;
                    for (int w = 0; w < NW; ++w) a += s_partd[w][tid];
                    s_rn2[tid] = a;
                    s_conf[tid] = (double)a <= s_thr[tid];
                    if (TC) {  // the next correction is about rho_j times the solution's scale
                        const float rho = s_isn2[tid] > 0.f ? sqrtf(a * s_isn2[tid]) : 1.f;
                        const float sg = rho * s_kap[tid];
                        s_sig[tid] = (sg > 1e-30f && isfinite(sg)) ? sg : 1e-30f;
                    }
                }
                __syncthreads();
                if (tid == 0) {
                    int a2 = s_active;
                    const int tested = CORR ? a2 : s_pending;
                    for (int j = 0; j < ncols; ++j) {
                        if (!((tested >> j) & 1) || !((a2 >> j) & 1)) continue;
                        const float rn2 = s_rn2[j];
                        if (!(rn2 == rn2) || isinf(rn2)) {
                            a2 &= ~(1 << j);
                            s_iters[j] = t - s_wait[j];
                            kz_flag(L.status, KZ_STATUS_BIT_NUMERIC);
                        } else if (s_conf[j]) {
                            a2 &= ~(1 << j);
                            s_iters[j] = t - s_wait[j];
                        } else if (!oahk && t >= L.max_iter) {
                            a2 &= ~(1 << j);
                            kz_flag(L.status, KZ_STATUS_BIT_NOT_CONVERGED);
                        }
                    }
                    s_active = a2;
                    s_pending = 0;
                }
                if (TC)
                    for (int e = tid; e < W * MS; e += NT) reinterpret_cast<unsigned*>(m16)[e] = 0u;
                else if (CORR)
                    for (int e = tid; e < W * MS; e += NT) m_s[e] = make_float2(0.f, 0.f);
                __syncthreads();
            }
            if (!s_active) break;
            // columns that take the aggregate step this iteration (a column whose
            // confirmation failed keeps iterating, so nothing stalls)
            const int stepmask = (!oahk && t >= L.max_iter) ? 0 : (CORR ? (s_active & ~s_pending) : s_active);
            // ---------------- aggregate u = H_V^H phi_V (antenna-major), ||u||^2
            if (stepmask) {
                if constexpr (TC) {
                    constexpr int NB = J / 4;
                    const int g = lane >> 2, c = lane & 3;
                    float uu[2 * NB];
#pragma unroll
                    for (int j = 0; j < 2 * NB; ++j) uu[j] = 0.f;
                    // phi enters the FP16 products as hs_i phi_ij / tau_j, tau_j the
                    // RMS of hs_i phi_ij over the V rows (0: a zero column); this
                    // lane's B column 4 nb + (g & 3), its output columns 4 nb + 2c
                    // and 4 nb + 2c + 1 (c < 2)
                    const float rv = 1.f / (float)max(vcount, 1);
                    auto itau_of = [&](int j) {
                        const float a = s_tot[3 * J + j] * rv;
                        return a > 0.f ? rsqrtf(a) : 0.f;
                    };
                    float itl[NB], tl0[NB], tl1[NB];
#pragma unroll
                    for (int nb = 0; nb < NB; ++nb) {
                        itl[nb] = itau_of(4 * nb + (g & 3));
                        const float i0 = itau_of(4 * nb + 2 * (c & 1)), i1 = itau_of(4 * nb + 2 * (c & 1) + 1);
                        tl0[nb] = i0 > 0.f ? 1.f / i0 : 0.f;
                        tl1[nb] = i1 > 0.f ? 1.f / i1 : 0.f;
                    }
                    // tasks: tile halves (32 antennas each)
                    for (int task = warp; task < 2 * I.ntiles; task += NW) {
                        const int tile = task >> 1, part = task & 1;
                        const int k0 = tptr_s[tile];
                        const int k1 = oahk ? k0 + tnv_s[tile] : tptr_s[tile + 1];
                        if (k0 == k1) continue;
                        float acc[4][NB][4];
                        if (trow_s)
                            tc_tile_aggr<J, true>(I.Hh, trow4, trow_s, rows_s, rptr_s, hs_s, tile, part, k0, k1, p_s,
                                                  itl, acc);
                        else
                            tc_tile_aggr<J, false>(I.Hh, trow4, trow_s, rows_s, rptr_s, hs_s, tile, part, k0, k1, p_s,
                                                   itl, acc);
                        // lane (g, c < 2) holds u at antennas n .. n + 3 (n =
                        // s + 4 g) for columns j and j + 1: two 16-byte stores per
                        // column, after the factor tau_j
#pragma unroll
                        for (int q2 = 0; q2 < 4; q2 += 2) {
                            const int n = tile * KZ_TILE + 32 * part + 4 * g + q2;
#pragma unroll
                            for (int nb = 0; nb < NB; ++nb) {
                                float2 u0a, u1a, u0b, u1b;
                                tc_u_combine(acc[q2][nb], u0a, u1a);
                                tc_u_combine(acc[q2 + 1][nb], u0b, u1b);
                                const int j = 4 * nb + 2 * c;
                                if (c < 2) {
                                    const float t0 = tl0[nb], t1 = tl1[nb];
                                    u0a = make_float2(u0a.x * t0, u0a.y * t0);
                                    u0b = make_float2(u0b.x * t0, u0b.y * t0);
                                    u1a = make_float2(u1a.x * t1, u1a.y * t1);
                                    u1b = make_float2(u1b.x * t1, u1b.y * t1);
                                    if (n < Nt) {
                                        kz_store_pair(I.x, Nt, col0 + j, n, j < ncols, u0a, u0b);
                                        kz_store_pair(I.x, Nt, col0 + j + 1, n, j + 1 < ncols, u1a, u1b);
                                    }
                                    uu[2 * nb] += u0a.x * u0a.x + u0a.y * u0a.y + u0b.x * u0b.x + u0b.y * u0b.y;
                                    uu[2 * nb + 1] += u1a.x * u1a.x + u1a.y * u1a.y + u1b.x * u1b.x + u1b.y * u1b.y;
                                }
                            }
                        }
                    }
#pragma unroll
                    for (int j = 0; j < 2 * NB; ++j) {
#pragma unroll
                        for (int o = 4; o < 32; o <<= 1) uu[j] += __shfl_xor_sync(KZ_FULL, uu[j], o);
                    }
                    if (g == 0 && c < 2) {
#pragma unroll
                        for (int nb = 0; nb < NB; ++nb) {
                            s_part[warp][4 * nb + 2 * c] = uu[2 * nb];
                            s_part[warp][4 * nb + 2 * c + 1] = uu[2 * nb + 1];
                        }
                    }
                } else {
                float uu[J];
#pragma unroll
                for (int j = 0; j < J; ++j) uu[j] = 0.f;
                for (int tile = warp; tile < I.ntiles; tile += NW) {
                    const int k0 = tptr_s[tile];
                    const int k1 = oahk ? k0 + tnv_s[tile] : tptr_s[tile + 1];
                    if (k0 == k1) continue;
                    float2 u0[J], u1[J];
                    tile_accum<J, BF16>(I, trow4, tile, k0, k1, p_s, u0, u1);
                    const int n = tile * KZ_TILE + 2 * lane;
#pragma unroll
                    for (int j = 0; j < J; ++j) {
                        if (j < ncols) {
                            float2* xc = I.x + (size_t)(col0 + j) * Nt;
                            if (n < Nt) xc[n] = u0[j];
                            if (n + 1 < Nt) xc[n + 1] = u1[j];
                        }
                        uu[j] += u0[j].x * u0[j].x + u0[j].y * u0[j].y + u1[j].x * u1[j].x + u1[j].y * u1[j].y;
                    }
                }
#pragma unroll
                for (int j = 0; j < J; ++j) uu[j] = warp_sum(uu[j]);
                if (lane == 0) {
#pragma unroll
                    for (int j = 0; j < J; ++j) s_part[warp][j] = uu[j];
                }
                }
                __syncthreads();
                if (tid < J) {
                    float a = 0.f;
                    for (int w = 0; w < NW; ++w) a += s_part[w][tid];
                    const float num = s_tot[J + tid];
                    const float den = a + xi * s_tot[2 * J + tid];
                    const bool on = (stepmask >> tid) & 1;
                    s_gamma[tid] = (on && num > 0.f && den > 0.f) ? num / den : 0.f;
                }
                __syncthreads();
                // ---------------- m += gamma u ; q_V += gamma phi_V
                // (u of all J columns of a tile read before any is applied)
                for (int tile = warp; tile < I.ntiles; tile += NW) {
                    const int k0 = tptr_s[tile];
                    const int k1 = oahk ? k0 + tnv_s[tile] : tptr_s[tile + 1];
                    if (k0 == k1) continue;
                    const int n = tile * KZ_TILE + 2 * lane;
                    float2 ua[J], ub[J];
#pragma unroll
                    for (int j = 0; j < J; ++j) {
                        const float2* xc = I.x + (size_t)(col0 + j) * Nt;
                        const bool on = j < ncols && s_gamma[j] != 0.f;
                        // one 16-byte load when the pair is inside the column
                        // and 16-byte aligned (the buffer need only be 8-byte
                        // aligned), else two 8-byte loads
                        const bool vec = n + 1 < Nt && (reinterpret_cast<uintptr_t>(xc + n) & 15) == 0;
                        if (on && vec) {
                            const float4 v = *reinterpret_cast<const float4*>(xc + n);
                            ua[j] = make_float2(v.x, v.y);
                            ub[j] = make_float2(v.z, v.w);
                        } else {
                            ua[j] = (on && n < Nt) ? xc[n] : make_float2(0.f, 0.f);
                            ub[j] = (on && n + 1 < Nt) ? xc[n + 1] : make_float2(0.f, 0.f);
                        }
                    }
#pragma unroll
                    for (int j = 0; j < J; ++j) {
                        const float g = s_gamma[j];
                        if constexpr (TC) {
                            if (j < ncols && g != 0.f) {
                                const float gs = g / s_sig[j];
                                __half2* mp = m16 + j * MS + n;
                                if (n + 1 < Nt) {  // both entries: one 8-byte access
                                    uint2 raw = *reinterpret_cast<const uint2*>(mp);
                                    float2 v = __half22float2(*reinterpret_cast<const __half2*>(&raw.x));
                                    float2 w = __half22float2(*reinterpret_cast<const __half2*>(&raw.y));
                                    v.x = fmaf(gs, ua[j].x, v.x);
                                    v.y = fmaf(gs, ua[j].y, v.y);
                                    w.x = fmaf(gs, ub[j].x, w.x);
                                    w.y = fmaf(gs, ub[j].y, w.y);
                                    const __half2 a = __float22half2_rn(v), b = __float22half2_rn(w);
                                    raw.x = *reinterpret_cast<const unsigned*>(&a);
                                    raw.y = *reinterpret_cast<const unsigned*>(&b);
                                    *reinterpret_cast<uint2*>(mp) = raw;
                                    continue;
                                }
                                if (n < Nt) {  // the last antenna of an odd Nt
                                    float2 v = __half22float2(mp[0]);
                                    v.x = fmaf(gs, ua[j].x, v.x);
                                    v.y = fmaf(gs, ua[j].y, v.y);
                                    mp[0] = __float22half2_rn(v);
                                }
                            }
                            continue;
                        }
                        if (j < ncols && g != 0.f) {
                            float2* mp = m_s + j * MS + n;
                            if (n < Nt) {
                                mp[0].x = fmaf(g, ua[j].x, mp[0].x);
                                mp[0].y = fmaf(g, ua[j].y, mp[0].y);
                            }
                            if (n + 1 < Nt) {
                                mp[1].x = fmaf(g, ub[j].x, mp[1].x);
                                mp[1].y = fmaf(g, ub[j].y, mp[1].y);
                            }
                        }
                    }
                    // u in x is dead once applied (the next aggregate rewrites
                    // every entry of the tile before it is read, the final
                    // x = H^H q every entry): its L2 lines are dropped without
                    // a write-back, so their space goes back to H.  Only whole
                    // lines of this item's own columns (Nt a multiple of 16,
                    // the first column 128-byte aligned), each by the first
                    // lane of the eight that read it, after all eight have.
                    if (xdisc) {
                        __syncwarp();
                        const int nl = tile * KZ_TILE + 2 * lane;
                        if ((lane & 7) == 0 && nl + 16 <= Nt)
                            for (int j = 0; j < ncols; ++j) kz_discard_l2(I.x + (size_t)(col0 + j) * Nt + nl);
                    }
                }
                for (int e = tid; e < vcount * J; e += NT) {
                    const int i = order_s[v0 + e / J], j = e % J;
                    const float g = s_gamma[j];
                    const float2 ph = p_s[i * J + j];
                    q_s[i * J + j].x = fmaf(g, ph.x, q_s[i * J + j].x);
                    q_s[i * J + j].y = fmaf(g, ph.y, q_s[i * J + j].y);
                }
            }
            if (!oahk) ++t;
            ++since_refresh;
            __syncthreads();
            // ---------------- periodic drift correction m = H^H q (C64)
            if (!CORR && L.refresh > 0 && since_refresh >= L.refresh) {
                since_refresh = 0;
                for (int tile = warp; tile < I.ntiles; tile += NW) {
                    float2 u0[J], u1[J];
                    tile_accum<J, false>(I, trow4, tile, tptr_s[tile], tptr_s[tile + 1], q_s, u0, u1);
                    const int n = tile * KZ_TILE + 2 * lane;
#pragma unroll
                    for (int j = 0; j < J; ++j) {
                        if (j >= W) continue;
                        m_s[j * MS + n] = u0[j];
                        m_s[j * MS + n + 1] = u1[j];
                    }
                }
                __syncthreads();
            }
            if (oahk && t >= L.max_iter) {
                if (tid == 0) {
                    for (int j = 0; j < ncols; ++j)
                        if ((s_active >> j) & 1) kz_flag(L.status, KZ_STATUS_BIT_NOT_CONVERGED);
                    s_active = 0;
                }
                __syncthreads();
                break;
            }
        }

        // ---- finalise: x = m = H^H q (complex64), true residual with compensated
        // sums; the tensor-core mode writes x straight to global memory
        for (int tile = warp; tile < I.ntiles; tile += NW) {
            float2 u0[J], u1[J];
            tile_accum<J, false>(I, trow4, tile, tptr_s[tile], tptr_s[tile + 1], q_s, u0, u1);
            const int n = tile * KZ_TILE + 2 * lane;
#pragma unroll
            for (int j = 0; j < J; ++j) {
                if (j >= W) continue;
                if constexpr (TC) {
                    if (j < ncols) {
                        float2* xc = I.x + (size_t)(col0 + j) * Nt;
                        if (n < Nt) xc[n] = u0[j];
                        if (n + 1 < Nt) xc[n + 1] = u1[j];
                    }
                } else {
                    m_s[j * MS + n] = u0[j];
                    m_s[j * MS + n + 1] = u1[j];
                }
            }
        }
        __syncthreads();
        true_residual_pass(false);
        for (int j = 0; j < ncols; ++j) {
            float2* xc = I.x + (size_t)(col0 + j) * Nt;
            if (!TC)
                for (int n = tid; n < Nt; n += NT) xc[n] = m_s[j * MS + n];
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

template <int J, int NW, int MODE>
cudaError_t launch_t(const KzLaunch& L, int grid, size_t smem, cudaStream_t st) {
    auto k = kz_ahk_kernel<J, NW, MODE>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, NW * 32, smem, st>>>(L);
    return cudaGetLastError();
}

template <int J, int NW, int MODE>
int occ_t(size_t smem) {
    auto k = kz_ahk_kernel<J, NW, MODE>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, NW * 32, smem) != cudaSuccess) return 0;
    return n;
}

template <int NW, int MODE>
cudaError_t launch_j(const KzLaunch& L, int J, int grid, size_t smem, cudaStream_t st) {
    if constexpr (MODE == 2) {
        switch (J) {
            case 4: return launch_t<4, NW, MODE>(L, grid, smem, st);
            case 8: return launch_t<8, NW, MODE>(L, grid, smem, st);
            default: return cudaErrorInvalidValue;
        }
    } else {
        switch (J) {
            case 1: return launch_t<1, NW, MODE>(L, grid, smem, st);
            case 2: return launch_t<2, NW, MODE>(L, grid, smem, st);
            case 4: return launch_t<4, NW, MODE>(L, grid, smem, st);
            case 8: return launch_t<8, NW, MODE>(L, grid, smem, st);
            default: return cudaErrorInvalidValue;
        }
    }
}

template <int NW, int MODE>
int occ_j(int J, size_t smem) {
    if constexpr (MODE == 2) {
        switch (J) {
            case 4: return occ_t<4, NW, MODE>(smem);
            case 8: return occ_t<8, NW, MODE>(smem);
            default: return 0;
        }
    } else {
        switch (J) {
            case 1: return occ_t<1, NW, MODE>(smem);
            case 2: return occ_t<2, NW, MODE>(smem);
            case 4: return occ_t<4, NW, MODE>(smem);
            case 8: return occ_t<8, NW, MODE>(smem);
            default: return 0;
        }
    }
}

template <int MODE>
cudaError_t launch_nw(const KzLaunch& L, int J, int nw, int grid, size_t smem, cudaStream_t st) {
    if (nw == 8) return launch_j<8, MODE>(L, J, grid, smem, st);
    if (nw == 16) return launch_j<16, MODE>(L, J, grid, smem, st);
    return cudaErrorInvalidValue;
}

template <int MODE>
int occ_nw(int J, int nw, size_t smem) {
    if (nw == 8) return occ_j<8, MODE>(J, smem);
    if (nw == 16) return occ_j<16, MODE>(J, smem);
    return 0;
}

}  // namespace

size_t kz_smem_ahk(int J, int Ntp, int K, int prec) {
    auto r16 = [](size_t b) { return (b + 15) & ~(size_t)15; };
    return r16((size_t)J * Ntp * sizeof(float2)) + 3 * r16((size_t)K * J * sizeof(float2)) +
           r16((size_t)K * sizeof(float)) + r16((size_t)K * sizeof(int4)) + 3 * r16((size_t)K * sizeof(int)) +
           r16((size_t)(Ntp / KZ_TILE + 1) * sizeof(int)) + r16((size_t)(Ntp / KZ_TILE) * sizeof(int)) +
           (prec == KZ_BF16_MIXED ? r16((size_t)(K + 1) * sizeof(int)) : 0);  // correction form: xptr
}

size_t kz_smem_ahk_tc(int J, int m_elems, int Ntp_max, int K, int trow) {
    auto r16 = [](size_t b) { return (b + 15) & ~(size_t)15; };
    const size_t ntask = 2 * (size_t)((K + 7) / 8);
    return kz_smem_ahk(J, Ntp_max, K, KZ_C64) - r16((size_t)J * Ntp_max * sizeof(float2)) +
           r16((size_t)m_elems * sizeof(__half2)) + r16((size_t)K * sizeof(int)) + r16((size_t)K * sizeof(float)) +
           r16((size_t)(K + 1) * sizeof(int)) +
           r16((size_t)K * J * sizeof(float2)) + r16(ntask * sizeof(int4)) + 2 * r16(ntask * sizeof(int)) +
           r16((size_t)trow * sizeof(unsigned short));
}

cudaError_t kz_launch_ahk(const KzLaunch& L, int J, int nw, int grid, size_t smem, cudaStream_t st) {
    if (L.tc) return L.prec == KZ_C64 ? launch_nw<2>(L, J, nw, grid, smem, st) : cudaErrorInvalidValue;
    return L.prec == KZ_BF16_MIXED ? launch_nw<1>(L, J, nw, grid, smem, st) : launch_nw<0>(L, J, nw, grid, smem, st);
}

int kz_occupancy_ahk(int J, int nw, size_t smem, int prec) {
    return prec == KZ_BF16_MIXED ? occ_nw<1>(J, nw, smem) : occ_nw<0>(J, nw, smem);
}

int kz_occupancy_ahk_tc(int J, int nw, size_t smem) { return occ_nw<2>(J, nw, smem); }
