// AHK / VR-OAHK in residual-update form with shared-memory H tiles.
//
// The iterate is kept in the dual variable q (w = B^H q with B = [H, sqrt(xi) I],
// so m = H^H q is never stored) together with its residual r = s - B B^H q.
// One aggregate step of eq. (update4) with coefficients phi (eq. (coefficient))
// changes them by
//     u = H^H phi,   z = H u + xi phi  (= B B^H phi),
//     q += gamma phi,   r -= gamma z,   gamma = phi^H r / (||u||^2 + xi ||phi||^2),
// the same iterates as the projection written with m, since B^H phi = [u; sqrt(xi) phi].
// The orthogonal half-step of Alg. 3 is the same update with phi restricted
// to F and gamma = 1 (Prop. 1); the V half-step restricts phi to V.
//
// One CTA owns one channel and J columns.  A pass over the channel visits
// its 64-antenna tiles once: the rows covering a tile are staged in shared
// memory (each row's tile segment is one coalesced read), u_tile =
// H_tile^H phi is formed from the staged rows, and z += H_tile u_tile goes to
// the rows' accumulators, all from shared memory.  H is read from L2 / HBM
// once per pass for all J columns.
//
// Recursive residuals drift by rounding; a pass with phi = q recomputes the
// true residual s - H (H^H q) - xi q.  It confirms every tentative stop, runs
// every `refresh` iterations, and the final pass with phi = q also writes
// x = H^H q.
#include "kz_device.cuh"

namespace {

constexpr int HSTR = KZ_TILE + 1;  // staged row stride (complex): odd, so row-wise reads spread over banks
constexpr int JT = 4;              // columns per thread in the u product
constexpr int JZ = 2;              // columns per thread in the z product (more tasks: every warp busy)

enum PassKind { PASS_F = 0, PASS_V = 1, PASS_ALL = 2 };

// Sum over the lanes of a warp that share lane % J (J a power of two <= 32):
// afterwards lane l < J holds the sum for column l.
template <int J>
__device__ __forceinline__ float seg_sum(float v) {
#pragma unroll
    for (int o = 16; o >= J; o >>= 1) v += __shfl_xor_sync(KZ_FULL, v, o);
    return v;
}
template <int J>
__device__ __forceinline__ double seg_sum_d(double v) {
#pragma unroll
    for (int o = 16; o >= J; o >>= 1) v += __shfl_xor_sync(KZ_FULL, v, o);
    return v;
}

template <int J, int NW>
struct DualSmem {
    float2* hs;     // [CS][HSTR] staged rows of one tile (chunk)
    int* hrow;      // [CS] row index of each staged slot, -1 if empty
    int* huse;      // [CS] 1 if the slot's row contributes to u in this pass
    float2* up;     // [RG][J][KZ_TILE] partial u per row group (antenna fastest: conflict-free stores)
    float2* us;     // [J][KZ_TILE] u of the tile
    float2* r_s;    // [K][J]
    float2* q_s;    // [K][J]
    float2* p_s;    // [K][J] phi
    float2* z_s;    // [K][J] H u accumulators of the pass
    float* d_s;     // [K]
};

// 8-byte asynchronous global -> shared copy; `valid == false` writes zeros
// (source size 0) without reading the source.
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem, bool valid) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    const int nbytes = valid ? 8 : 0;
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(sa), "l"(gmem), "r"(nbytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Asynchronous version of stage_rows: the copies complete at the next
// cp_async_wait; hrow / huse are plain stores (visible after the barrier).
template <int NW>
__device__ __forceinline__ void stage_rows_async(const KzInst& I, const int4* __restrict__ trow4, int tile, int k0,
                                                 int n, int ku0, int ku1, float2* hs, int* hrow, int* huse) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nb = tile * KZ_TILE + 2 * lane;
    for (int sl = warp; sl < n; sl += NW) {
        const int4 e = __ldg(trow4 + k0 + sl);
        const bool in = (nb >= e.z && nb < e.w);
        const float2* src = in ? (I.Hc + e.y + nb) : I.Hc;
        float2* dst = hs + sl * HSTR + 2 * lane;
        cp_async8(dst, src, in);
        cp_async8(dst + 1, src + 1, in);
        if (lane == 0) {
            hrow[sl] = e.x;
            huse[sl] = (k0 + sl >= ku0 && k0 + sl < ku1) ? 1 : 0;
        }
    }
}

// Stage the covering-row entries [k0, k0 + n) of `tile` into slots 0..n-1.
template <int NW>
__device__ __forceinline__ void stage_rows(const KzInst& I, const int4* __restrict__ trow4, int tile, int k0, int n,
                                           int ku0, int ku1, float2* hs, int* hrow, int* huse) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nb = tile * KZ_TILE + 2 * lane;
    for (int sl = warp; sl < n; sl += NW) {
        const int4 e = __ldg(trow4 + k0 + sl);
        float4 h = make_float4(0.f, 0.f, 0.f, 0.f);
        if (nb >= e.z && nb < e.w) h = h_pair<false>(I, e.y + nb);
        float2* dst = hs + sl * HSTR + 2 * lane;
        dst[0] = make_float2(h.x, h.y);
        dst[1] = make_float2(h.z, h.w);
        if (lane == 0) {
            hrow[sl] = e.x;
            huse[sl] = (k0 + sl >= ku0 && k0 + sl < ku1) ? 1 : 0;
        }
    }
}

// z[row] += H_tile[row, :] u_tile for the n staged rows: one thread per
// (staged row, JZ columns), rows over lanes (padded stride: conflict-free),
// u_tile read as broadcasts.
template <int J, int NW>
__device__ __forceinline__ void z_tile(const DualSmem<J, NW>& S, const float2* hs, const int* hrow, int n) {
    constexpr int CZ = J / JZ;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ntask = ((n + 31) / 32) * CZ;
    for (int task = warp; task < ntask; task += NW) {
        const int sl = (task / CZ) * 32 + lane;
        const int g = task % CZ;
        if (sl < n) {
            float2 acc[JZ];
#pragma unroll
            for (int t = 0; t < JZ; ++t) acc[t] = make_float2(0.f, 0.f);
            const float2* hp = hs + sl * HSTR;
#pragma unroll 8
            for (int nn = 0; nn < KZ_TILE; ++nn) {
                const float2 h = hp[nn];
                const float2* up = S.us + (g * JZ) * KZ_TILE + nn;
#pragma unroll
                for (int t = 0; t < JZ; ++t) {
                    const float2 u = up[t * KZ_TILE];
                    acc[t].x = fmaf(h.x, u.x, fmaf(-h.y, u.y, acc[t].x));
                    acc[t].y = fmaf(h.x, u.y, fmaf(h.y, u.x, acc[t].y));
                }
            }
            float2* zp = S.z_s + hrow[sl] * J + g * JZ;
#pragma unroll
            for (int t = 0; t < JZ; ++t) {
                zp[t].x += acc[t].x;
                zp[t].y += acc[t].y;
            }
        }
    }
}

// One pass: z = H (H^H coef) restricted as `kind` says, ||u||^2 per column.
// kind PASS_V: u from V rows (list head), PASS_F: from F rows (list tail),
// PASS_ALL: from every row.  If xout != nullptr, u is also written to
// x (columns col0.., leading dimension Nt).  z_s must be zero on entry.
// u-phase contribution of n staged rows (rows of this warp's row group that
// are flagged for u), per thread 2 antennas x JT columns.
template <int J, int NW>
__device__ __forceinline__ void u_rows(const float2* hs, const int* hrow, const int* huse, int n, const float2* coef,
                                       float2 (&a0)[JT], float2 (&a1)[JT]) {
    constexpr int CG = J / JT, RG = NW / CG;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int cg = warp % CG, rg = warp / CG;
    for (int sl = rg; sl < n; sl += RG) {
        if (!huse[sl]) continue;
        const float2* hp = hs + sl * HSTR + 2 * lane;
        const float2 h0 = hp[0], h1 = hp[1];
        const float2* cp = coef + hrow[sl] * J + cg * JT;
#pragma unroll
        for (int t = 0; t < JT; ++t) {
            const float2 cv = cp[t];
            a0[t].x = fmaf(h0.x, cv.x, fmaf(h0.y, cv.y, a0[t].x));
            a0[t].y = fmaf(h0.x, cv.y, fmaf(-h0.y, cv.x, a0[t].y));
            a1[t].x = fmaf(h1.x, cv.x, fmaf(h1.y, cv.y, a1[t].x));
            a1[t].y = fmaf(h1.x, cv.y, fmaf(-h1.y, cv.x, a1[t].y));
        }
    }
}

// Combine the row groups' partial u of one tile into us, add ||u||^2 of
// column tid / 32 to uacc and optionally write u to x.  Ends with us ready.
template <int J, int NW>
__device__ __forceinline__ void finish_u(const DualSmem<J, NW>& S, int tile, int Nt, const float2 (&a0)[JT],
                                         const float2 (&a1)[JT], float& uacc, float2* xout, int col0, int ncols) {
    constexpr int CG = J / JT, RG = NW / CG;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int cg = warp % CG, rg = warp / CG;
    float2* upp = S.up + (size_t)rg * KZ_TILE * J;
#pragma unroll
    for (int t = 0; t < JT; ++t) {
        upp[(cg * JT + t) * KZ_TILE + 2 * lane] = a0[t];
        upp[(cg * JT + t) * KZ_TILE + 2 * lane + 1] = a1[t];
    }
    __syncthreads();
    for (int e = tid; e < KZ_TILE * J; e += NW * 32) {
        float2 u = make_float2(0.f, 0.f);
        for (int g = 0; g < RG; ++g) {
            const float2 v = S.up[(size_t)g * KZ_TILE * J + e];
            u.x += v.x;
            u.y += v.y;
        }
        S.us[e] = u;
    }
    __syncthreads();
    if (tid < 32 * J) {
        const int j = tid / 32, l = tid % 32;
        const float2 u0 = S.us[j * KZ_TILE + 2 * l], u1 = S.us[j * KZ_TILE + 2 * l + 1];
        uacc += u0.x * u0.x + u0.y * u0.y + u1.x * u1.x + u1.y * u1.y;
        if (xout && j < ncols) {
            const int nn = tile * KZ_TILE + 2 * l;
            float2* xc = xout + (size_t)(col0 + j) * Nt;
            if (nn < Nt) xc[nn] = u0;
            if (nn + 1 < Nt) xc[nn + 1] = u1;
        }
    }
}

// Pass with the next tile's rows copied (cp.async) into the other staging
// buffer while the current tile computes; every tile's rows fit one buffer.
template <int J, int NW>
__device__ float dual_pass_pipe(const KzInst& I, const DualSmem<J, NW>& S, int CS, int kind, const float2* coef,
                                float2* xout, int col0, int ncols) {
    const int tid = threadIdx.x;
    const int4* trow4 = I.trow4;
    const int Nt = I.Nt;
    float uacc = 0.f;
    auto has_u = [&](int tile, int& k0, int& k1, int& ku0, int& ku1) {
        k0 = I.tptr[tile];
        k1 = I.tptr[tile + 1];
        const int nv = I.tnv[tile];
        ku0 = k0;
        ku1 = k1;
        if (kind == PASS_V) ku1 = k0 + nv;
        if (kind == PASS_F) ku0 = k0 + nv;
        return ku0 < ku1;
    };
    auto next_tile = [&](int t) {
        for (int tt = t + 1; tt < I.ntiles; ++tt) {
            int k0, k1, ku0, ku1;
            if (has_u(tt, k0, k1, ku0, ku1)) return tt;
            if (xout && tid < 32 * J && tid / 32 < ncols) {  // u = 0 on an uncovered tile
                const int nn = tt * KZ_TILE + 2 * (tid % 32);
                float2* xc = xout + (size_t)(col0 + tid / 32) * Nt;
                if (nn < Nt) xc[nn] = make_float2(0.f, 0.f);
                if (nn + 1 < Nt) xc[nn + 1] = make_float2(0.f, 0.f);
            }
        }
        return -1;
    };
    int t = next_tile(-1), b = 0;
    if (t >= 0) {
        int k0, k1, ku0, ku1;
        has_u(t, k0, k1, ku0, ku1);
        stage_rows_async<NW>(I, trow4, t, k0, k1 - k0, ku0, ku1, S.hs, S.hrow, S.huse);
    }
    cp_async_commit();
    while (t >= 0) {
        const int tn = next_tile(t);
        if (tn >= 0) {
            int k0, k1, ku0, ku1;
            has_u(tn, k0, k1, ku0, ku1);
            stage_rows_async<NW>(I, trow4, tn, k0, k1 - k0, ku0, ku1, S.hs + (b ^ 1) * CS * HSTR,
                                 S.hrow + (b ^ 1) * CS, S.huse + (b ^ 1) * CS);
        }
        cp_async_commit();
        cp_async_wait<1>();  // this tile's copies are done (the prefetch may still fly)
        __syncthreads();
        const int n = I.tptr[t + 1] - I.tptr[t];
        const float2* hs = S.hs + b * CS * HSTR;
        const int* hrow = S.hrow + b * CS;
        const int* huse = S.huse + b * CS;
        float2 a0[JT], a1[JT];
#pragma unroll
        for (int q = 0; q < JT; ++q) a0[q] = a1[q] = make_float2(0.f, 0.f);
        u_rows<J, NW>(hs, hrow, huse, n, coef, a0, a1);
        finish_u<J, NW>(S, t, Nt, a0, a1, uacc, xout, col0, ncols);
        z_tile<J, NW>(S, hs, hrow, n);
        __syncthreads();  // buffers of this tile free before they are refilled
        t = tn;
        b ^= 1;
    }
    cp_async_wait<0>();
    __syncthreads();
    return uacc;
}

template <int J, int NW>
__device__ float dual_pass(const KzInst& I, const DualSmem<J, NW>& S, int CS, int kind, const float2* coef,
                           float2* xout, int col0, int ncols) {
    if (I.cmax <= CS) return dual_pass_pipe<J, NW>(I, S, CS, kind, coef, xout, col0, ncols);
    constexpr int CG = J / JT;        // column groups
    constexpr int RG = NW / CG;       // row groups in the u phase
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int4* trow4 = I.trow4;
    const int Nt = I.Nt;
    const int cg = warp % CG, rg = warp / CG;
    float uacc = 0.f;  // ||u||^2 of column tid / 32 (threads tid < 32 J)
    for (int tile = 0; tile < I.ntiles; ++tile) {
        const int k0 = I.tptr[tile], k1 = I.tptr[tile + 1];
        const int nv = I.tnv[tile];
        int ku0 = k0, ku1 = k1;
        if (kind == PASS_V) ku1 = k0 + nv;
        if (kind == PASS_F) ku0 = k0 + nv;
        if (ku0 >= ku1) {  // u = 0 on this tile: nothing changes
            if (xout && tid < 32 * J && tid / 32 < ncols) {
                const int nn = tile * KZ_TILE + 2 * (tid % 32);
                float2* xc = xout + (size_t)(col0 + tid / 32) * Nt;
                if (nn < Nt) xc[nn] = make_float2(0.f, 0.f);
                if (nn + 1 < Nt) xc[nn + 1] = make_float2(0.f, 0.f);
            }
            continue;
        }
        const int c = k1 - k0;
        const int nchunk = (c + CS - 1) / CS;
        // ---- u phase: accumulate over chunks, per thread 2 antennas x JT columns
        float2 a0[JT], a1[JT];
#pragma unroll
        for (int t = 0; t < JT; ++t) a0[t] = a1[t] = make_float2(0.f, 0.f);
        for (int ch = 0; ch < nchunk; ++ch) {
            const int kc = k0 + ch * CS, n = min(CS, k1 - kc);
            __syncthreads();  // previous users of the staging buffer are done
            stage_rows<NW>(I, trow4, tile, kc, n, ku0, ku1, S.hs, S.hrow, S.huse);
            __syncthreads();
            for (int sl = rg; sl < n; sl += RG) {
                if (!S.huse[sl]) continue;
                const float2* hp = S.hs + sl * HSTR + 2 * lane;
                const float2 h0 = hp[0], h1 = hp[1];
                const float2* cp = coef + S.hrow[sl] * J + cg * JT;
#pragma unroll
                for (int t = 0; t < JT; ++t) {
                    const float2 cv = cp[t];
                    a0[t].x = fmaf(h0.x, cv.x, fmaf(h0.y, cv.y, a0[t].x));
                    a0[t].y = fmaf(h0.x, cv.y, fmaf(-h0.y, cv.x, a0[t].y));
                    a1[t].x = fmaf(h1.x, cv.x, fmaf(h1.y, cv.y, a1[t].x));
                    a1[t].y = fmaf(h1.x, cv.y, fmaf(-h1.y, cv.x, a1[t].y));
                }
            }
        }
        // partial u of this row group -> up[rg]
        {
            float2* upp = S.up + (size_t)rg * KZ_TILE * J;
#pragma unroll
            for (int t = 0; t < JT; ++t) {
                upp[(cg * JT + t) * KZ_TILE + 2 * lane] = a0[t];
                upp[(cg * JT + t) * KZ_TILE + 2 * lane + 1] = a1[t];
            }
        }
        __syncthreads();
        for (int e = tid; e < KZ_TILE * J; e += NW * 32) {
            float2 u = make_float2(0.f, 0.f);
            for (int g = 0; g < RG; ++g) {
                const float2 v = S.up[(size_t)g * KZ_TILE * J + e];
                u.x += v.x;
                u.y += v.y;
            }
            S.us[e] = u;
        }
        __syncthreads();
        // ||u||^2 and the optional x output (thread per antenna pair x column)
        if (tid < 32 * J) {
            const int j = tid / 32, l = tid % 32;
            const float2 u0 = S.us[j * KZ_TILE + 2 * l], u1 = S.us[j * KZ_TILE + 2 * l + 1];
            const float p = u0.x * u0.x + u0.y * u0.y + u1.x * u1.x + u1.y * u1.y;
            uacc += p;
            if (xout && j < ncols) {
                const int nn = tile * KZ_TILE + 2 * l;
                float2* xc = xout + (size_t)(col0 + j) * Nt;
                if (nn < Nt) xc[nn] = u0;
                if (nn + 1 < Nt) xc[nn + 1] = u1;
            }
        }
        // ---- z phase: z[row] += H_tile[row, :] u_tile, thread per (staged row, JT columns)
        for (int ch = 0; ch < nchunk; ++ch) {
            const int kc = k0 + ch * CS, n = min(CS, k1 - kc);
            if (nchunk > 1) {
                __syncthreads();
                stage_rows<NW>(I, trow4, tile, kc, n, ku0, ku1, S.hs, S.hrow, S.huse);
                __syncthreads();
            }
            z_tile<J, NW>(S, S.hs, S.hrow, n);
        }
        __syncthreads();  // z and us settled before the next tile reuses the buffers
    }
    return uacc;
}

template <int J, int NW>
__global__ void __launch_bounds__(NW * 32, 1) kz_dual_kernel(const __grid_constant__ KzLaunch L) {
    static_assert(J % JT == 0, "J must be a multiple of JT");
    static_assert(32 * J <= NW * 32, "one thread per (antenna pair, column) in the norm step");
    extern __shared__ __align__(16) unsigned char kz_smem[];
    __shared__ KzInst sI;
    __shared__ float s_part[NW][3 * J];
    __shared__ float s_tot[3 * J];
    __shared__ double s_partd[NW][J];
    __shared__ double s_sn2[J];
    __shared__ float s_gamma[J];
    __shared__ int s_iters[J];
    __shared__ int s_active, s_pending, s_item;

    constexpr int CG = J / JT, RG = NW / CG;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NT = NW * 32;
    const int CS = L.cs;
    DualSmem<J, NW> S;
    {
        unsigned char* p = kz_smem;
        S.hs = reinterpret_cast<float2*>(p);
        p += 2 * (size_t)CS * HSTR * sizeof(float2);
        S.up = reinterpret_cast<float2*>(p);
        p += (size_t)RG * KZ_TILE * J * sizeof(float2);
        S.us = reinterpret_cast<float2*>(p);
        p += (size_t)KZ_TILE * J * sizeof(float2);
        S.r_s = reinterpret_cast<float2*>(p);
        p += (size_t)L.K_max * J * sizeof(float2);
        S.q_s = reinterpret_cast<float2*>(p);
        p += (size_t)L.K_max * J * sizeof(float2);
        S.p_s = reinterpret_cast<float2*>(p);
        p += (size_t)L.K_max * J * sizeof(float2);
        S.z_s = reinterpret_cast<float2*>(p);
        p += (size_t)L.K_max * J * sizeof(float2);
        S.d_s = reinterpret_cast<float*>(p);
        p += (size_t)L.K_max * sizeof(float);
        S.hrow = reinterpret_cast<int*>(p);
        p += 2 * (size_t)CS * sizeof(int);
        S.huse = reinterpret_cast<int*>(p);
    }
    const float tol2 = (float)(L.tol * L.tol);
    const bool oahk = (L.algo == KZ_VR_OAHK);

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
        const int K = I.K, nF = oahk ? I.nF : 0;
        const int col0 = KZ_ITEM_COL(it.y), ncols = min(J, I.ld - col0);
        const float xi = I.xi;

        // r = s, q = 0 at w = 0
        for (int e = tid; e < K * J; e += NT) {
            const int i = e / J, j = e % J;
            S.r_s[e] = (j < ncols) ? I.s[(size_t)(col0 + j) * K + i] : make_float2(0.f, 0.f);
            S.q_s[e] = make_float2(0.f, 0.f);
            S.p_s[e] = make_float2(0.f, 0.f);
            S.z_s[e] = make_float2(0.f, 0.f);
        }
        for (int i = tid; i < K; i += NT) S.d_s[i] = I.nrm[i] + xi;
        __syncthreads();
        if (warp < J) {
            double a = 0.0;
            for (int i = lane; i < K; i += 32) {
                const float2 v = S.r_s[i * J + warp];
                a += (double)v.x * v.x + (double)v.y * v.y;
            }
            a = warp_sum_d(a);
            if (lane == 0) s_sn2[warp] = a;
        }
        __syncthreads();
        if (tid == 0) {
            int act = 0;
            for (int j = 0; j < ncols; ++j) {
                s_iters[j] = L.max_iter;
                if (s_sn2[j] > 0.0) act |= 1 << j;
                else s_iters[j] = 0;
            }
            s_active = act;
            s_pending = 0;
        }
        __syncthreads();

        // block-wide helpers -------------------------------------------------
        // apply r -= g z + g xi phi and q += g phi on rows [r0, r1) of `order`
        // (or every row when order_rows is false), clear z, and sum ||r||^2 (float)
        // Squared residual norm per column: thread tid only ever visits column
        // tid % J (NT is a multiple of J), so each keeps one scalar.
        auto residual_norms = [&](void) {
            float a = 0.f;
            for (int e = tid; e < K * J; e += NT) {
                const float2 r = S.r_s[e];
                a += r.x * r.x + r.y * r.y;
            }
            a = seg_sum<J>(a);
            if (lane < J) s_part[warp][lane] = a;
            __syncthreads();
            if (tid < J) {
                float t = 0.f;
                for (int w = 0; w < NW; ++w) t += s_part[w][tid];
                s_tot[tid] = t;
            }
            __syncthreads();
        };
        // True residual r = s - H (H^H q) - xi q (FP32 tile products, squared
        // norm summed in FP64 into s_partd); optionally writes x = H^H q.
        auto true_residual = [&](float2* xo) {
            (void)dual_pass<J, NW>(I, S, CS, PASS_ALL, S.q_s, xo, col0, ncols);
            double rp = 0.0;
            for (int e = tid; e < K * J; e += NT) {
                const int i = e / J, j = e % J;
                const float2 sv = (j < ncols) ? I.s[(size_t)(col0 + j) * K + i] : make_float2(0.f, 0.f);
                const float2 z = S.z_s[e], q = S.q_s[e];
                const float2 r = make_float2(sv.x - z.x - xi * q.x, sv.y - z.y - xi * q.y);
                S.r_s[e] = r;
                S.z_s[e] = make_float2(0.f, 0.f);
                rp += (double)r.x * r.x + (double)r.y * r.y;
            }
            rp = seg_sum_d<J>(rp);
            if (lane < J) s_partd[warp][lane] = rp;
            __syncthreads();
        };

        int t = 0, since_refresh = 0;
        while (s_active) {
            const int act = s_active;
            if (oahk) {
                ++t;
                // ---- orthogonal half-step: phi_F = r_F / d_F, unit step (Prop. 1)
                for (int e = tid; e < nF * J; e += NT) {
                    const int i = I.order[e / J], j = e % J;
                    const float2 r = S.r_s[i * J + j];
                    const float di = S.d_s[i];
                    S.p_s[i * J + j] = ((act >> j) & 1) ? make_float2(r.x / di, r.y / di) : make_float2(0.f, 0.f);
                }
                __syncthreads();
                (void)dual_pass<J, NW>(I, S, CS, PASS_F, S.p_s, nullptr, col0, ncols);
                // r -= z + xi phi_F ; q_F += phi_F ; z = 0 ; phi_F = 0
                for (int e = tid; e < K * J; e += NT) {
                    const float2 z = S.z_s[e];
                    S.r_s[e].x -= z.x;
                    S.r_s[e].y -= z.y;
                    S.z_s[e] = make_float2(0.f, 0.f);
                }
                __syncthreads();
                for (int e = tid; e < nF * J; e += NT) {
                    const int i = I.order[e / J], j = e % J;
                    const float2 ph = S.p_s[i * J + j];
                    S.r_s[i * J + j].x -= xi * ph.x;
                    S.r_s[i * J + j].y -= xi * ph.y;
                    S.q_s[i * J + j].x += ph.x;
                    S.q_s[i * J + j].y += ph.y;
                    S.p_s[i * J + j] = make_float2(0.f, 0.f);
                }
                __syncthreads();
            }
            // ---- residual norm of the current iterate (r_F = 0 after the F step)
            residual_norms();
            if (tid == 0) {
                int a2 = s_active, pend = 0;
                for (int j = 0; j < ncols; ++j) {
                    if (!((a2 >> j) & 1)) continue;
                    const float rn2 = s_tot[j];
                    if (!(rn2 == rn2) || isinf(rn2)) {
                        a2 &= ~(1 << j);
                        s_iters[j] = t;
                        kz_flag(L.status, KZ_STATUS_BIT_NUMERIC);
                    } else if ((double)rn2 <= (double)tol2 * s_sn2[j]) {
                        pend |= 1 << j;
                    } else if (!oahk && t >= L.max_iter) {
                        a2 &= ~(1 << j);
                        kz_flag(L.status, KZ_STATUS_BIT_NOT_CONVERGED);
                    }
                }
                s_active = a2;
                s_pending = pend;
            }
            __syncthreads();
            // ---- confirmation of tentative stops on the true residual
            if (s_pending) {
                since_refresh = 0;
                true_residual(nullptr);
                if (tid == 0) {
                    int a2 = s_active;
                    for (int j = 0; j < ncols; ++j) {
                        if (!((s_pending >> j) & 1) || !((a2 >> j) & 1)) continue;
                        double rn2 = 0.0;
                        for (int w = 0; w < NW; ++w) rn2 += s_partd[w][j];
                        if (rn2 <= L.tol * L.tol * s_sn2[j]) {
                            a2 &= ~(1 << j);
                            s_iters[j] = t;
                        } else if (!oahk && t >= L.max_iter) {
                            a2 &= ~(1 << j);
                            kz_flag(L.status, KZ_STATUS_BIT_NOT_CONVERGED);
                        }
                    }
                    s_active = a2;
                    s_pending = 0;
                }
                __syncthreads();
            }
            if (!s_active) break;
            const int stepmask = (!oahk && t >= L.max_iter) ? 0 : s_active;
            // ---- aggregate step on V (all rows for AHK)
            if (stepmask) {
                const int v0 = nF, vcount = K - nF;
                float pn = 0.f, pp = 0.f;  // column tid % J
                for (int e = tid; e < vcount * J; e += NT) {
                    const int i = I.order[v0 + e / J], j = e % J;
                    const float2 r = S.r_s[i * J + j];
                    const float di = S.d_s[i];
                    const bool on = (stepmask >> j) & 1;
                    const float2 ph = on ? make_float2(r.x / di, r.y / di) : make_float2(0.f, 0.f);
                    S.p_s[i * J + j] = ph;
                    pn += on ? (r.x * r.x + r.y * r.y) / di : 0.f;
                    pp += ph.x * ph.x + ph.y * ph.y;
                }
                pn = seg_sum<J>(pn);
                pp = seg_sum<J>(pp);
                if (lane < J) {
                    s_part[warp][J + lane] = pn;
                    s_part[warp][2 * J + lane] = pp;
                }
                __syncthreads();
                // ||u||^2: thread tid < 32 J holds column tid / 32, so warp w < J sums column w
                float usq = dual_pass<J, NW>(I, S, CS, oahk ? PASS_V : PASS_ALL, S.p_s, nullptr, col0, ncols);
                usq = warp_sum(usq);
                if (lane == 0) s_part[warp][0] = usq;
                __syncthreads();
                if (tid < J) {
                    const float a = s_part[tid][0];  // warp tid's sum is column tid's ||u||^2
                    float num = 0.f, phin = 0.f;
                    for (int w = 0; w < NW; ++w) {
                        num += s_part[w][J + tid];
                        phin += s_part[w][2 * J + tid];
                    }
                    const float den = a + xi * phin;
                    const bool on = (stepmask >> tid) & 1;
                    s_gamma[tid] = (on && num > 0.f && den > 0.f) ? num / den : 0.f;
                }
                __syncthreads();
                // r -= gamma (z + xi phi) ; q += gamma phi ; z = 0 ; phi = 0
                for (int e = tid; e < K * J; e += NT) {
                    const int j = e % J;
                    const float g = s_gamma[j];
                    const float2 z = S.z_s[e], ph = S.p_s[e];
                    S.r_s[e].x -= g * (z.x + xi * ph.x);
                    S.r_s[e].y -= g * (z.y + xi * ph.y);
                    S.q_s[e].x = fmaf(g, ph.x, S.q_s[e].x);
                    S.q_s[e].y = fmaf(g, ph.y, S.q_s[e].y);
                    S.z_s[e] = make_float2(0.f, 0.f);
                    S.p_s[e] = make_float2(0.f, 0.f);
                }
                __syncthreads();
            }
            if (!oahk) ++t;
            ++since_refresh;
            if (L.refresh > 0 && since_refresh >= L.refresh) {
                since_refresh = 0;
                true_residual(nullptr);
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

        // ---- finalise: x = H^H q (written by the pass), true residual
        true_residual(I.x);
        for (int j = 0; j < ncols; ++j) {
            if (I.v) {
                float2* vc = I.v + (size_t)(col0 + j) * K;
                for (int i = tid; i < K; i += NT) vc[i] = S.q_s[i * J + j];
            }
        }
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
    auto k = kz_dual_kernel<J, NW>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, NW * 32, smem, st>>>(L);
    return cudaGetLastError();
}

template <int J, int NW>
int occ_t(size_t smem) {
    auto k = kz_dual_kernel<J, NW>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, NW * 32, smem) != cudaSuccess) return 0;
    return n;
}

}  // namespace

// Shared memory of the dual kernel with CS staged rows per chunk.
size_t kz_smem_dual(int J, int nw, int CS, int K) {
    const int CG = J / JT, RG = nw / CG;
    return 2 * (size_t)CS * HSTR * sizeof(float2) + (size_t)RG * KZ_TILE * J * sizeof(float2) +
           (size_t)KZ_TILE * J * sizeof(float2) + 4 * (size_t)K * J * sizeof(float2) + (size_t)K * sizeof(float) +
           4 * (size_t)CS * sizeof(int) + 16;
}

cudaError_t kz_launch_dual(const KzLaunch& L, int J, int nw, int grid, size_t smem, cudaStream_t st) {
    if (J == 8 && nw == 8) return launch_t<8, 8>(L, grid, smem, st);
    if (J == 8 && nw == 16) return launch_t<8, 16>(L, grid, smem, st);
    if (J == 16 && nw == 16) return launch_t<16, 16>(L, grid, smem, st);
    return cudaErrorInvalidValue;
}

int kz_occupancy_dual(int J, int nw, size_t smem) {
    if (J == 8 && nw == 8) return occ_t<8, 8>(smem);
    if (J == 8 && nw == 16) return occ_t<8, 16>(smem);
    if (J == 16 && nw == 16) return occ_t<16, 16>(smem);
    return 0;
}
