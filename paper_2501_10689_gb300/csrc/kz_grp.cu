// Group kernel: AHK / VR-OAHK (eqs. (update4), (coefficient); Alg. 3) on ONE
// channel whose right-hand sides share H (Remark 2), with the two
// contractions of every half-step on the Blackwell tensor cores (tcgen05.mma,
// accumulators in tensor memory).
//
// Work split.  The antenna axis is cut into blocks of 128 antennas and the
// right-hand sides into groups of NC columns.  CTA (b, g) = (blockIdx.x,
// blockIdx.y) owns antenna block b of the iterate correction for column group
// g, and holds in shared memory -- for the whole solve, loaded once by a bulk
// (TMA) copy -- the block's "tile": every row whose VR meets the block,
// restricted to the block, as 16-bit (FP16 or BF16) real and imaginary planes.
// The AB CTAs of one column group form the "group"; they synchronise through a
// cluster barrier (AB <= 16, one cluster per group) or, for larger channels,
// through a grid barrier of a cooperative launch.  Per half-step:
//
//   P = H dM       tile (K-major, M = rows) x correction (MN-major, N = columns);
//                  each CTA writes its rows' partial sums, and the owner of row
//                  k (rows are dealt to the group's CTAs) adds the partials of
//                  the blocks the row meets: r = b_ref - P - xi dq;
//   U = H^H Phi    the same tile read as an MN-major operand (M = antennas,
//                  K = rows) x Phi (MN-major, N = columns), gathered from the
//                  owners' phi = r / d;
//   complex products as four real products on planes, one with negated B.
//
// Correction form (the iteration cannot reach 1e-6 on 16-bit operands alone):
// the owners keep q (FP32) and b_ref = s - H H^H q - xi q, recomputed every
// `refresh` iterations from the inner products of overlapping rows (the X_k
// pattern, compensated FP32 sums); between refreshes the kernel iterates on
// the correction (dM, dq) with dM's FP32 master in tensor memory and its
// 16-bit copy (scaled per column) as the MMA operand.  Every stop is
// confirmed on the refreshed true residual, and x = H^H q is formed at the end
// from the complex64 rows.  The cross-CTA sums (residual partials, column
// norms) are added in a fixed order, so results do not depend on timing.
#include <algorithm>

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "kz_device.cuh"
#include "kz_internal.h"
#include "kz_tc5.cuh"

namespace {

constexpr int GT = 256;     // threads per CTA
constexpr int GBN = 128;    // antennas per block
constexpr int GNCMAX = 64;  // columns per group, at most
enum { Q_RV2 = 0, Q_NUM, Q_PHIN, Q_U2, Q_RT2, Q_SN2, Q_KAP, NQ };
constexpr unsigned long long WAIT_NS = 2000000000ull;  // 2 s bound on any wait

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait on an mbarrier phase.
__device__ __forceinline__ bool wait_phase(uint64_t* bar, uint32_t parity) {
    const unsigned long long t0 = gtimer();
    for (long i = 0; i < (1L << 30); ++i) {
        if (kz5::bar_test(bar, parity)) return true;
        if ((i & 1023) == 1023 && gtimer() - t0 > WAIT_NS) return false;
    }
    return false;
}

__device__ __forceinline__ uint32_t pack2(float a, float b, int fmt) {
    if (fmt) {
        __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<uint32_t*>(&h);
    }
    __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
}

__device__ __forceinline__ void two_prod_acc(float a, float b, float& hi, float& lo) {
    const float p = a * b;
    const float pe = fmaf(a, b, -p);
    const float s = hi + p;
    const float bb = s - hi;
    const float e = (hi - (s - bb)) + (p - bb);
    hi = s;
    lo += e + pe;
}

// ---------------------------------------------------------------------------
// Set-up: max |Re|, |Im| over the channel (the 16-bit tiles hold H / sigma_H
// with sigma_H a power of two, so every entry is at most 1 in magnitude) and
// the mean row norm (scales of the 16-bit right-hand-side operand).
__global__ void grp_stats_kernel(const float2* __restrict__ Hc, long long total2, const float* __restrict__ nrm, int K,
                                 float* stat) {
    __shared__ float smax[32];
    __shared__ double ssum[32];
    float m = 0.f;
    double a = 0.0;
    for (long long i = threadIdx.x; i < total2; i += blockDim.x) {
        const float2 h = Hc[i];
        m = fmaxf(m, fmaxf(fabsf(h.x), fabsf(h.y)));
    }
    for (int k = threadIdx.x; k < K; k += blockDim.x) a += (double)nrm[k];
    for (int o = 16; o > 0; o >>= 1) {
        m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        a += __shfl_xor_sync(0xffffffffu, a, o);
    }
    if ((threadIdx.x & 31) == 0) {
        smax[threadIdx.x >> 5] = m;
        ssum[threadIdx.x >> 5] = a;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float mm = 0.f;
        double aa = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            mm = fmaxf(mm, smax[w]);
            aa += ssum[w];
        }
        int ex = 0;
        (void)frexpf(mm > 0.f && isfinite(mm) ? mm : 1.f, &ex);  // mm = f 2^ex with f in [0.5, 1)
        stat[0] = ldexpf(1.f, ex);                                // sigma_H
        stat[1] = (float)(aa / K);                                // mean ||h_k||^2
    }
}

// Tile images: block b's image is two planes (Re, Im) of RT_b rows x 128
// antennas; element (slot r, antenna n) at plane * RT_b * 256 + (r / 8) * 2048
// + (n / 8) * 128 + (r % 8) * 16 + (n % 8) * 2 bytes.  One thread writes one
// 16-byte row chunk (8 antennas).
__global__ void grp_fill_kernel(KzGrpChan C, const float2* __restrict__ Hc, const int4* __restrict__ rows,
                                const int* __restrict__ rptr, const float* __restrict__ stat, int fmt) {
    const int b = blockIdx.x;
    const int RT = 128 * C.blk_nrt[b];
    const float inv = 1.f / stat[0];
    uint8_t* img = const_cast<uint8_t*>(C.tiles) + C.blk_toff[b];
    for (int c = threadIdx.x; c < 2 * RT * 16; c += blockDim.x) {
        const int plane = c / (RT * 16), rem = c % (RT * 16), r = rem / 16, ng = rem % 16;
        const int k = C.slot_row[b * 256 + r];
        float v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int n = b * GBN + ng * 8 + i;
            float x = 0.f;
            if (k >= 0) {
                const int4 rd = rows[k];  // {a, len2, o, e}
                if (n >= rd.z && n < rd.w) {
                    const float2 h = Hc[rptr[k] + (n - rd.x)];
                    x = (plane ? h.y : h.x) * inv;
                }
            }
            v[i] = x;
        }
        uint4 w;
        w.x = pack2(v[0], v[1], fmt);
        w.y = pack2(v[2], v[3], fmt);
        w.z = pack2(v[4], v[5], fmt);
        w.w = pack2(v[6], v[7], fmt);
        *reinterpret_cast<uint4*>(img + (size_t)plane * RT * 256 + (r / 8) * 2048 + ng * 128 + (r % 8) * 16) = w;
    }
}

// ---------------------------------------------------------------------------
// Group synchronisation.  Cluster: hardware barrier with release / acquire.
// Grid: a monotone arrival counter per group (the group's AB CTAs of the
// cooperative launch; the groups decide their refreshes and their end on
// their own columns, so they take different numbers of barriers), polled
// with acquire loads for at most WAIT_NS; a timeout raises the status bit and
// the group's abort flag, which every CTA of the group reads right after each
// barrier.
__device__ __forceinline__ void flag(int* status, int bit) {
    if (status) atomicOr(status, bit);
}

// Abort protocol: a CTA that meets a failure after completing `gen` group
// barriers stores the epoch gen + 1 (atomicMin) in the abort word; every CTA
// reads the word right after each barrier and stops once the epoch is at most
// the number of barriers it has completed.  A failure is thus acted on by all
// CTAs at the same barrier, so none is left waiting for the others.
template <bool CLUSTER>
__device__ __forceinline__ void group_sync(const KzGrpLaunch& L, unsigned& gen, unsigned nctas, unsigned* abort_word) {
    ++gen;
    if constexpr (CLUSTER) {
        kz5::cluster_sync();
    } else {
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned* counter = L.gbar + blockIdx.y;  // this group's arrivals
            kz5::red_release_gpu_add(counter, 1u);  // publishes the CTA's writes (ordered by the barrier above)
            const unsigned target = gen * nctas;
            const unsigned long long t0 = gtimer();
            long i = 0;
            while (kz5::ld_acquire_gpu(counter) < target) {
                __nanosleep(32);
                if ((++i & 255) == 0 && gtimer() - t0 > WAIT_NS) {
                    flag(L.status, KZ_STATUS_BIT_TIMEOUT);
                    atomicMin(abort_word, gen);
                    break;
                }
            }
            // the acquire load that saw every arrival orders this CTA's later
            // reads (through the barrier below) after the other CTAs' writes
        }
        __syncthreads();
    }
}

template <bool CLUSTER>
__global__ void __launch_bounds__(GT, 1) kz_grp_kernel(const KzGrpLaunch L) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ uint64_t bar_ld, bar_mma;
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort, s_refresh;
    __shared__ double c_sn2[GNCMAX], c_rt2[GNCMAX], c_sum[3 * GNCMAX];
    __shared__ float c_tmp[3 * GNCMAX * 8];  // chunk sums of sum_partials (AB <= 128)
    __shared__ float c_sumf[3 * GNCMAX], c_thr[GNCMAX];
    __shared__ float c_kap[GNCMAX], c_sig[GNCMAX], c_isig[GNCMAX], c_tau[GNCMAX], c_gam[GNCMAX], c_coef[GNCMAX];
    __shared__ int c_act[GNCMAX], c_wait[GNCMAX], c_iters[GNCMAX];
    __shared__ float c_numv[GNCMAX], c_phinv[GNCMAX];
    __shared__ float red[4][GNCMAX];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int quarter = warp & 3, half = warp >> 2;
    const int b = blockIdx.x, g = blockIdx.y;
    const KzGrpChan& C = L.C;
    const int AB = C.AB, K = C.K, Nt = C.Nt, NC = L.NC;
    const int col0 = g * NC;
    const int ncols = min(NC, L.nrhs - col0);
    const unsigned nctas = gridDim.x;  // CTAs of one group
    const int fmt = L.fmt;
    const bool oahk = (L.algo == KZ_VR_OAHK);
    const float xi = L.xi;
    const int nrt = C.blk_nrt[b], RT = 128 * nrt, nb = C.blk_nb[b], coff = C.blk_coff[b];
    const int rtrows = 128 * L.rtmax;
    const int rpc = L.rpc, k0 = b * rpc, nown = max(0, min(K - k0, rpc));

    // shared memory carve-up
    uint8_t* sH = smem;                                          // tile: 2 planes x RT x 256 bytes
    uint8_t* sOp = smem + (size_t)2 * rtrows * 256;              // 16-bit B operand (dM or Phi)
    const int szop = max(512 * NC, 4 * NC * rtrows);
    float2* o_s = reinterpret_cast<float2*>(sOp + szop);         // owner state, [rpc][NC] each
    float2* o_rref = o_s + rpc * NC;
    float2* o_dq = o_rref + rpc * NC;
    float2* o_q = o_dq + rpc * NC;
    float2* o_phi = o_q + rpc * NC;
    float* ubuf = reinterpret_cast<float*>(o_phi + rpc * NC);   // [3][rpc][NC] per-unit values
    int* s_slot = reinterpret_cast<int*>(ubuf + 3 * rpc * NC);   // [rtrows]
    int* s_cidx = s_slot + rtrows;                               // [rpc * AB] partial slots of the owned rows
    int* s_cptr = s_cidx + rpc * AB;                             // [rpc + 1], relative to the owned rows' first

    const int PSH = RT * 256;           // tile plane bytes
    const int Tn = NC * 16;             // operand stride between 8-row groups along K
    const int PSd = 16 * Tn;            // dM operand plane bytes (128 antennas)
    const int PSf = (RT / 8) * Tn;      // Phi operand plane bytes (RT rows)
    const uint32_t P0 = 0, U0 = (uint32_t)(L.rtmax * 2 * NC), M0 = U0 + 2 * NC;
    const uint32_t idP = kz5::idesc_f16(128, NC, fmt, 0, 1, 0), idPn = kz5::idesc_f16(128, NC, fmt, 0, 1, 1);
    const uint32_t idU = kz5::idesc_f16(128, NC, fmt, 1, 1, 0), idUn = kz5::idesc_f16(128, NC, fmt, 1, 1, 1);
    unsigned* abort_word = L.gbar + L.CG + g;
    unsigned gen = 0;
    uint32_t mma_par = 0;
    bool mma_late = false;

    // ---------------- set-up
    if (tid == 0) {
        kz5::bar_init(&bar_ld, 1);
        kz5::bar_init(&bar_mma, 1);
        kz5::bar_init_fence();
        s_abort = 0;
    }
    if (warp == 0) kz5::tmem_alloc(&s_tmem, (uint32_t)L.tmem_cols);
    for (int r = tid; r < rtrows; r += GT) s_slot[r] = (r < RT) ? C.slot_row[b * 256 + r] : -1;
    {
        const int c0 = nown ? C.cptr[k0] : 0;
        for (int i = tid; i <= nown; i += GT) s_cptr[i] = C.cptr[k0 + i] - c0;
        const int nc = nown ? C.cptr[k0 + nown] - c0 : 0;
        for (int i = tid; i < nc; i += GT) s_cidx[i] = C.cidx[c0 + i];
    }
    kz5::fence_async_smem();
    kz5::fence_before();
    __syncthreads();
    kz5::fence_after();
    const uint32_t tmem = s_tmem;
    const uint32_t tl = tmem + ((uint32_t)(32 * quarter) << 16);  // this warp's TMEM lanes
    if (tid == 0) {
        const uint32_t bytes = (uint32_t)(2 * PSH);
        kz5::bar_expect_tx(&bar_ld, bytes);
        for (uint32_t o = 0; o < bytes; o += 32768u)
            kz5::bulk_g2s(sH + o, C.tiles + C.blk_toff[b] + o, min(32768u, bytes - o), &bar_ld);
    }
    const float sigH = C.stat[0], dmean = C.stat[1] + xi;

    // owner rows: b_ref = s (q = 0), and the column sums ||s||^2 and the
    // storage-scale estimate sum_k |s_k|^2 ||h_k||^2 / d_k^2
    for (int u = tid; u < nown * NC; u += GT) {
        const int kk = u / NC, j = u % NC, k = k0 + kk;
        const float2 sv = (j < ncols) ? L.s[(size_t)(col0 + j) * K + k] : make_float2(0.f, 0.f);
        o_s[u] = sv;
        o_rref[u] = sv;
        o_dq[u] = make_float2(0.f, 0.f);
        o_q[u] = make_float2(0.f, 0.f);
        o_phi[u] = make_float2(0.f, 0.f);
        const float a2 = sv.x * sv.x + sv.y * sv.y, d = C.nrm[k] + xi;
        ubuf[u] = a2;
        ubuf[rpc * NC + u] = a2 * C.nrm[k] / (d * d);
    }
    __syncthreads();
    float* cp = L.colpart + (size_t)g * NQ * AB * NC;  // this group's partials [NQ][NC][AB]
    auto put_partial = [&](int q, int which) {         // column sums over the owned rows, in row order
        if (tid < NC) {
            float a = 0.f;
            for (int kk = 0; kk < nown; ++kk) a += ubuf[which * rpc * NC + kk * NC + tid];
            cp[((size_t)q * NC + tid) * AB + b] = a;
        }
    };
    put_partial(Q_SN2, 0);
    put_partial(Q_KAP, 1);

    // fixed-order sums of partials over the group's AB CTAs into c_sum[qi * NC + j]
    // (and c_sumf, its float value) (nq <= 3): every (quantity, column) pair's
    // AB partials (contiguous) are cut into chunks of 16 added by one thread
    // each (four 16-byte loads), then the chunk sums are added in chunk order;
    // FP32 with TwoSum compensation throughout (no FP64 arithmetic, whose rate
    // on this GPU is a small fraction of FP32's).  With the abort word read
    // here too, this is where every CTA learns of a failure (at the same
    // barrier).
    auto sum_partials = [&](const int* qs, int nq) {
        const int pairs = nq * NC, nch = (AB + 15) / 16, tasks = pairs * nch;
        if (tid == 0) s_abort = (__ldcg(abort_word) <= gen) ? 1 : 0;
#pragma unroll 2
        for (int tk = tid; tk < tasks; tk += GT) {
            const int p = tk / nch, c = tk % nch;
            const float* src = cp + ((size_t)qs[p / NC] * NC + (p % NC)) * AB + 16 * c;
            const int n = min(16, AB - 16 * c);
            float hi = 0.f, lo = 0.f;
            auto add = [&](float v) {
                float sm, e;
                two_sum(hi, v, sm, e);
                hi = sm;
                lo += e;
            };
            if (n == 16 && (AB & 3) == 0) {
                float4 x[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) x[i] = __ldcg(reinterpret_cast<const float4*>(src) + i);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    add(x[i].x);
                    add(x[i].y);
                    add(x[i].z);
                    add(x[i].w);
                }
            } else {
                for (int i = 0; i < n; ++i) add(__ldcg(src + i));
            }
            c_tmp[tk] = hi + lo;
        }
        __syncthreads();
        for (int p = tid; p < pairs; p += GT) {
            float hi = 0.f, lo = 0.f;
            for (int c = 0; c < nch; ++c) {
                float sm, e;
                two_sum(hi, c_tmp[p * nch + c], sm, e);
                hi = sm;
                lo += e;
            }
            c_sum[p] = (double)hi + (double)lo;
            c_sumf[p] = hi + lo;
        }
        __syncthreads();
    };
    auto sync = [&]() { group_sync<CLUSTER>(L, gen, nctas, abort_word); };
    auto fail_later = [&]() {  // acted on by every CTA after the next barrier
        flag(L.status, KZ_STATUS_BIT_TIMEOUT);
        atomicMin(abort_word, gen + 1);
    };

    sync();
    {
        const int qs[2] = {Q_SN2, Q_KAP};
        sum_partials(qs, 2);
    }
    if (tid < NC) {
        const int j = tid;
        const double sn2 = c_sum[j], kap2 = c_sum[NC + j];
        c_sn2[j] = sn2;
        c_thr[j] = (float)(L.tol * L.tol * sn2);
        c_rt2[j] = sn2;
        const bool bad = !(sn2 == sn2) || isinf(sn2);
        c_act[j] = (j < ncols) && sn2 > 0.0 && !bad;
        if (j < ncols && bad && b == 0) flag(L.status, KZ_STATUS_BIT_NUMERIC);
        c_wait[j] = 0;
        c_iters[j] = 0;
        const float kap = (float)sqrt(kap2 / Nt);
        c_kap[j] = (kap > 0.f && isfinite(kap)) ? kap : 1.f;
        c_sig[j] = c_kap[j];
        c_isig[j] = 1.f / c_sig[j];
        const float tau = (float)(sqrt(sn2 / K) / dmean);
        c_tau[j] = (tau > 1e-30f && isfinite(tau)) ? tau : 1.f;
        c_gam[j] = 0.f;
    }
    // the tile
    if (!wait_phase(&bar_ld, 0) && tid == 0) fail_later();
    __syncthreads();

    // ---------------- building blocks
    // the product's rows (slot r of row tile rt) -> compact partial index
    auto mma_wait = [&]() {
        if (!wait_phase(&bar_mma, mma_par)) {
            mma_late = true;
            if (tid == 0) fail_later();
        }
        mma_par ^= 1u;
        kz5::fence_after();
    };
    const int chunks = (NC / 2) / 8;  // 8-column chunks per half
    // P = H dM for the rows of this block -> partial sums (scaled to true units)
    auto gemm_p = [&]() {
        if (tid == 0) {
            kz5::fence_after();
            const uint32_t aH = kz5::smem_u32(sH), aD = kz5::smem_u32(sOp);
            for (int rt = 0; rt < nrt; ++rt) {
                const uint32_t dre = tmem + P0 + rt * 2 * NC, dim = dre + NC;
                for (int s = 0; s < 8; ++s) {
                    const uint64_t are = kz5::desc(aH + rt * 16 * 2048 + s * 256, 128, 2048);
                    const uint64_t aim = kz5::desc(aH + PSH + rt * 16 * 2048 + s * 256, 128, 2048);
                    const uint64_t bre = kz5::desc(aD + s * 2 * Tn, Tn, 128);
                    const uint64_t bim = kz5::desc(aD + PSd + s * 2 * Tn, Tn, 128);
                    kz5::mma(dre, are, bre, idP, s > 0);
                    kz5::mma(dre, aim, bim, idPn, 1u);
                    kz5::mma(dim, are, bim, idP, s > 0);
                    kz5::mma(dim, aim, bre, idP, 1u);
                }
            }
            kz5::mma_commit(&bar_mma);
        }
        mma_wait();
        for (int rt = 0; rt < nrt; ++rt) {
            const int r = rt * 128 + 32 * quarter + lane;
            for (int c = 0; c < chunks; ++c) {
                const int j0 = half * (NC / 2) + 8 * c;
                float vr[8], vi[8];
                kz5::tmem_ld8(tl + P0 + rt * 2 * NC + j0, vr);
                kz5::tmem_ld8(tl + P0 + rt * 2 * NC + NC + j0, vi);
                kz5::tmem_ld_wait();
                if (r < nb) {
                    float4* dst = reinterpret_cast<float4*>(L.Ppart + ((size_t)g * C.n_slots + coff + r) * NC + j0);
#pragma unroll
                    for (int i = 0; i < 8; i += 2) {
                        const float s0 = sigH * c_sig[j0 + i], s1 = sigH * c_sig[j0 + i + 1];
                        dst[i / 2] = make_float4(vr[i] * s0, vi[i] * s0, vr[i + 1] * s1, vi[i + 1] * s1);
                    }
                }
            }
        }
        kz5::fence_before();
    };
    // U = H^H Phi for this block's antennas (left in tensor memory)
    auto gemm_u = [&]() {
        const int nch = RT * 2 * (NC / 8);  // 16-byte chunks of the Phi operand
        const uint16_t* phg = L.Phi + (size_t)g * K * 2 * NC;
        for (int c = tid; c < nch; c += GT) {
            const int r = c % RT, pj = c / RT, plane = pj / (NC / 8), jg = pj % (NC / 8);
            const int k = s_slot[r];
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (k >= 0) v = __ldcg(reinterpret_cast<const uint4*>(phg + ((size_t)k * 2 + plane) * NC + 8 * jg));
            *reinterpret_cast<uint4*>(sOp + plane * PSf + (r / 8) * Tn + jg * 128 + (r % 8) * 16) = v;
        }
        kz5::fence_async_smem();
        kz5::fence_before();
        __syncthreads();
        if (tid == 0) {
            kz5::fence_after();
            const uint32_t aH = kz5::smem_u32(sH), aF = kz5::smem_u32(sOp);
            const uint32_t ure = tmem + U0, uim = ure + NC;
            for (int s = 0; s < RT / 16; ++s) {
                const uint64_t are = kz5::desc(aH + s * 2 * 2048, 2048, 128);
                const uint64_t aim = kz5::desc(aH + PSH + s * 2 * 2048, 2048, 128);
                const uint64_t bre = kz5::desc(aF + s * 2 * Tn, Tn, 128);
                const uint64_t bim = kz5::desc(aF + PSf + s * 2 * Tn, Tn, 128);
                kz5::mma(ure, are, bre, idU, s > 0);
                kz5::mma(ure, aim, bim, idU, 1u);
                kz5::mma(uim, are, bim, idU, s > 0);
                kz5::mma(uim, aim, bre, idUn, 1u);
            }
            kz5::mma_commit(&bar_mma);
        }
        mma_wait();
    };
    // ||U_j||^2 partials of this block (true units)
    auto u_norms = [&]() {
        for (int c = 0; c < chunks; ++c) {
            const int j0 = half * (NC / 2) + 8 * c;
            float vr[8], vi[8];
            kz5::tmem_ld8(tl + U0 + j0, vr);
            kz5::tmem_ld8(tl + U0 + NC + j0, vi);
            kz5::tmem_ld_wait();
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const float a = warp_sum(vr[i] * vr[i] + vi[i] * vi[i]);
                if (lane == 0) red[quarter][j0 + i] = a;
            }
        }
        kz5::fence_before();
        __syncthreads();
        if (tid < NC) {
            const float sc = sigH * c_tau[tid];
            const float a = ((red[0][tid] + red[1][tid]) + (red[2][tid] + red[3][tid])) * sc * sc;
            cp[((size_t)Q_U2 * NC + tid) * AB + b] = a;
        }
    };
    // dM += coef_j U (FP32 master in tensor memory), then the 16-bit operand dM / sigma_j
    auto dm_update = [&]() {
        const int n = 32 * quarter + lane;
        for (int c = 0; c < chunks; ++c) {
            const int j0 = half * (NC / 2) + 8 * c;
            float ur[8], ui[8], mr[8], mi[8];
            kz5::tmem_ld8(tl + U0 + j0, ur);
            kz5::tmem_ld8(tl + U0 + NC + j0, ui);
            kz5::tmem_ld8(tl + M0 + j0, mr);
            kz5::tmem_ld8(tl + M0 + NC + j0, mi);
            kz5::tmem_ld_wait();
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const float cf = c_coef[j0 + i];
                mr[i] = fmaf(cf, ur[i], mr[i]);
                mi[i] = fmaf(cf, ui[i], mi[i]);
            }
            kz5::tmem_st8(tl + M0 + j0, mr);
            kz5::tmem_st8(tl + M0 + NC + j0, mi);
            float wr[8], wi[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                wr[i] = mr[i] * c_isig[j0 + i];
                wi[i] = mi[i] * c_isig[j0 + i];
            }
            const uint4 pr = make_uint4(pack2(wr[0], wr[1], fmt), pack2(wr[2], wr[3], fmt), pack2(wr[4], wr[5], fmt),
                                        pack2(wr[6], wr[7], fmt));
            const uint4 pi = make_uint4(pack2(wi[0], wi[1], fmt), pack2(wi[2], wi[3], fmt), pack2(wi[4], wi[5], fmt),
                                        pack2(wi[6], wi[7], fmt));
            uint8_t* dst = sOp + (n / 8) * Tn + (j0 / 8) * 128 + (n % 8) * 16;
            *reinterpret_cast<uint4*>(dst) = pr;
            *reinterpret_cast<uint4*>(dst + PSd) = pi;
        }
        kz5::tmem_st_wait();
        kz5::fence_async_smem();
        kz5::fence_before();
        __syncthreads();
    };
    auto dm_zero = [&]() {
        float z[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int c = 0; c < chunks; ++c) {
            const int j0 = half * (NC / 2) + 8 * c;
            kz5::tmem_st8(tl + M0 + j0, z);
            kz5::tmem_st8(tl + M0 + NC + j0, z);
        }
        kz5::tmem_st_wait();
        kz5::fence_before();
        __syncthreads();
    };
    // owner residual of unit u (row k0 + kk, column j): b_ref - P - xi dq
    auto owner_resid = [&](int kk, int j, int u, bool dirty) {
        float2 r = o_rref[u];
        if (dirty) {
            const float2* pp = L.Ppart + (size_t)g * C.n_slots * NC + j;
            const int e0 = s_cptr[kk], e1 = s_cptr[kk + 1];
            float px = 0.f, py = 0.f;
            for (int e = e0; e < e1; e += 8) {  // eight loads in flight, added in order
                float2 v[8];
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    v[i] = (e + i < e1) ? __ldcg(pp + (size_t)s_cidx[e + i] * NC) : make_float2(0.f, 0.f);
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    px += v[i].x;
                    py += v[i].y;
                }
            }
            r.x -= px;
            r.y -= py;
        }
        const float2 dq = o_dq[u];
        r.x = fmaf(-xi, dq.x, r.x);
        r.y = fmaf(-xi, dq.y, r.y);
        return r;
    };
    auto put_phi = [&](int kk, int j, float2 ph) {  // 16-bit Phi (scaled by 1 / tau_j), both planes
        const int k = k0 + kk;
        uint16_t* base = L.Phi + ((size_t)g * K + k) * 2 * NC + j;
        const float it = 1.f / c_tau[j];
        if (fmt) {
            base[0] = __bfloat16_as_ushort(__float2bfloat16_rn(ph.x * it));
            base[NC] = __bfloat16_as_ushort(__float2bfloat16_rn(ph.y * it));
        } else {
            base[0] = __half_as_ushort(__float2half_rn(ph.x * it));
            base[NC] = __half_as_ushort(__float2half_rn(ph.y * it));
        }
    };

    // ---------------- refresh: q += dq; publish q; b_ref = s - H H^H q - xi q
    // through the inner products of overlapping rows (compensated sums); the
    // stopping test on that true residual.  `last`: columns still above tol
    // stop as not converged.  Returns 0: columns remain, 1: none, 2: abort.
    int t = 0;
    auto refresh = [&](bool last) -> int {
        float2* qg = L.Qg + (size_t)g * K * NC;
        for (int u = tid; u < nown * NC; u += GT) {
            const int kk = u / NC, j = u % NC, k = k0 + kk;
            o_q[u].x += o_dq[u].x;
            o_q[u].y += o_dq[u].y;
            o_dq[u] = make_float2(0.f, 0.f);
            qg[(size_t)k * NC + j] = o_q[u];
        }
        sync();
        for (int u = tid; u < nown * NC; u += GT) {
            const int kk = u / NC, j = u % NC, k = k0 + kk;
            float hx = 0.f, lx = 0.f, hy = 0.f, ly = 0.f;
            const int e1 = C.xptr[k + 1];
            for (int e = C.xptr[k]; e < e1; e += 8) {  // eight entries' loads in flight
                float2 gk[8], ql[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const bool in = e + i < e1;
                    gk[i] = in ? __ldg(C.G + e + i) : make_float2(0.f, 0.f);
                    ql[i] = in ? __ldcg(qg + (size_t)__ldg(C.xidx + e + i) * NC + j) : make_float2(0.f, 0.f);
                }
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    two_prod_acc(gk[i].x, ql[i].x, hx, lx);
                    two_prod_acc(-gk[i].y, ql[i].y, hx, lx);
                    two_prod_acc(gk[i].x, ql[i].y, hy, ly);
                    two_prod_acc(gk[i].y, ql[i].x, hy, ly);
                }
            }
            const float2 sv = o_s[u], qv = o_q[u];
            float2 r;
            r.x = fmaf(-xi, qv.x, (sv.x - hx) - lx);
            r.y = fmaf(-xi, qv.y, (sv.y - hy) - ly);
            o_rref[u] = r;
            ubuf[u] = r.x * r.x + r.y * r.y;
        }
        __syncthreads();
        put_partial(Q_RT2, 0);
        sync();
        {
            const int qs[1] = {Q_RT2};
            sum_partials(qs, 1);
        }
        if (s_abort) return 2;
        if (tid < NC) {
            const int j = tid;
            if (c_act[j]) {
                const double rt2 = c_sum[j];
                c_rt2[j] = rt2;
                if (!(rt2 == rt2) || isinf(rt2)) {
                    c_act[j] = 0;
                    c_iters[j] = t;
                    if (b == 0) flag(L.status, KZ_STATUS_BIT_NUMERIC);
                } else if (rt2 <= L.tol * L.tol * c_sn2[j]) {
                    c_act[j] = 0;
                    c_iters[j] = t;
                } else {
                    c_wait[j] = 0;
                    if (last) {
                        c_act[j] = 0;
                        c_iters[j] = t;
                        if (b == 0) flag(L.status, KZ_STATUS_BIT_NOT_CONVERGED);
                    }
                }
                // the next correction is about rho_j times the solution's scale
                const double rho = sqrt(rt2 / c_sn2[j]);
                const float sg = (float)(rho * c_kap[j]);
                c_sig[j] = (sg > 1e-30f && isfinite(sg)) ? sg : 1e-30f;
                c_isig[j] = 1.f / c_sig[j];
                const float tau = (float)(sqrt(rt2 / K) / dmean);
                c_tau[j] = (tau > 1e-30f && isfinite(tau)) ? tau : 1e-30f;
            }
        }
        __syncthreads();
        if (tid == 0) {
            int any = 0;
            for (int j = 0; j < NC; ++j) any |= c_act[j];
            s_refresh = any;
        }
        dm_zero();  // ends with a block barrier
        return s_refresh ? 0 : 1;
    };

    // ---------------- the iteration
    int since = 0;
    bool dirty = false, resume_v = false;
    if (!s_abort) {
        dm_zero();
        while (true) {
            if (!resume_v) {
                ++t;
                if (oahk) {
                    // orthogonal half-step: phi_F = r_F / d_F, unit step (Prop. 1)
                    if (dirty) {
                        gemm_p();
                        sync();
                    }
                    for (int u = tid; u < nown * NC; u += GT) {
                        const int kk = u / NC, j = u % NC, k = k0 + kk;
                        float2 ph = make_float2(0.f, 0.f);
                        if (C.inF[k] && c_act[j] && !c_wait[j]) {
                            const float2 r = owner_resid(kk, j, u, dirty);
                            const float di = 1.f / (C.nrm[k] + xi);
                            ph = make_float2(r.x * di, r.y * di);
                            o_dq[u].x += ph.x;
                            o_dq[u].y += ph.y;
                        }
                        put_phi(kk, j, ph);
                    }
                    sync();
                    if (tid < NC) c_coef[tid] = (c_act[tid] && !c_wait[tid]) ? sigH * c_tau[tid] : 0.f;
                    gemm_u();
                    dm_update();
                    dirty = true;
                }
            }
            // a V half-step right after a refresh tests nothing (the true residual
            // was just tested) and always steps, so every refresh is followed by
            // progress
            const bool resumed = resume_v;
            resume_v = false;
            // residual of V (all rows for AHK) on the current iterate
            if (dirty) {
                gemm_p();
                sync();
            }
            for (int u = tid; u < nown * NC; u += GT) {
                const int kk = u / NC, j = u % NC, k = k0 + kk;
                float2 ph = make_float2(0.f, 0.f);
                float rv2 = 0.f, num = 0.f, pn = 0.f;
                if (!(oahk && C.inF[k]) && c_act[j]) {
                    const float2 r = owner_resid(kk, j, u, dirty);
                    rv2 = r.x * r.x + r.y * r.y;
                    if (!c_wait[j]) {
                        const float di = 1.f / (C.nrm[k] + xi);
                        ph = make_float2(r.x * di, r.y * di);
                        num = rv2 * di;
                        pn = ph.x * ph.x + ph.y * ph.y;
                    }
                }
                o_phi[u] = ph;
                put_phi(kk, j, ph);
                ubuf[u] = rv2;
                ubuf[rpc * NC + u] = num;
                ubuf[2 * rpc * NC + u] = pn;
            }
            __syncthreads();
            put_partial(Q_RV2, 0);
            put_partial(Q_NUM, 1);
            put_partial(Q_PHIN, 2);
            sync();
            {
                const int qs[3] = {Q_RV2, Q_NUM, Q_PHIN};
                sum_partials(qs, 3);
            }
            if (s_abort) break;
            // tentative stopping test on the running residual
            if (tid < NC) {
                const int j = tid;
                if (!resumed && c_act[j] && !c_wait[j]) {
                    const float rv2 = c_sumf[j];
                    if (!(rv2 == rv2) || isinf(rv2)) {
                        c_act[j] = 0;
                        c_iters[j] = t;
                        if (b == 0) flag(L.status, KZ_STATUS_BIT_NUMERIC);
                    } else if (rv2 <= c_thr[j]) {
                        c_wait[j] = 1;
                    }
                }
                c_numv[j] = c_sumf[NC + j];
                c_phinv[j] = c_sumf[2 * NC + j];
            }
            __syncthreads();
            if (tid == 0) {
                bool all_wait = true;
                for (int j = 0; j < NC; ++j)
                    if (c_act[j] && !c_wait[j]) all_wait = false;
                s_refresh = !resumed && ((since + 1 >= L.refresh) || all_wait);
            }
            __syncthreads();
            if (s_refresh) {
                const int rc = refresh(false);
                dirty = false;
                since = 0;
                if (rc) break;
                resume_v = true;  // the V half-step, now on the refreshed residual
                continue;
            }
            // aggregate step on V (eq. (updatenor)): u = H_V^H phi_V, gamma, update
            gemm_u();
            u_norms();
            sync();
            {
                const int qs[1] = {Q_U2};
                sum_partials(qs, 1);
            }
            if (s_abort) break;
            // gamma = Re(phi_V^H r_V) / (||u||^2 + xi ||phi_V||^2) (eq. (coefficient)); 0 skips the step
            if (tid < NC) {
                const int j = tid;
                float gm = 0.f;
                if (c_act[j] && !c_wait[j] && c_numv[j] > 0.f) {
                    const float den = c_sumf[j] + xi * c_phinv[j];
                    gm = den > 0.f ? c_numv[j] / den : 0.f;
                }
                c_gam[j] = gm;
                c_coef[j] = gm * sigH * c_tau[j];
            }
            __syncthreads();
            dm_update();
            dirty = true;
            for (int u = tid; u < nown * NC; u += GT) {
                const float gm = c_gam[u % NC];
                o_dq[u].x = fmaf(gm, o_phi[u].x, o_dq[u].x);
                o_dq[u].y = fmaf(gm, o_phi[u].y, o_dq[u].y);
            }
            since += 1;
            if (t >= L.max_iter) {  // max_iter full iterations taken: the last true residual decides
                __syncthreads();
                (void)refresh(true);
                break;
            }
        }
    }
    // ---------------- outputs (after the last refresh every column is inactive)
    // x = H^H q from the complex64 rows; q of the block's rows staged in shared memory
    if (!s_abort) {
        float2* qs = reinterpret_cast<float2*>(sH);
        const float2* qg = L.Qg + (size_t)g * K * NC;
        for (int e = tid; e < nb * NC; e += GT) qs[e] = __ldcg(qg + (size_t)s_slot[e / NC] * NC + (e % NC));
        __syncthreads();
        const int n = b * GBN + (tid & 127);
        const int jlo = (tid >> 7) * (NC / 2), jhi = jlo + NC / 2;
        if (n < Nt) {
            float2 acc[GNCMAX / 2];
#pragma unroll
            for (int i = 0; i < GNCMAX / 2; ++i) acc[i] = make_float2(0.f, 0.f);
            for (int r = 0; r < nb; ++r) {
                const int k = s_slot[r];
                const int4 rd = C.rows[k];
                if (n < rd.z || n >= rd.w) continue;
                const float2 h = __ldg(C.Hc + C.rptr[k] + (n - rd.x));
#pragma unroll
                for (int i = 0; i < GNCMAX / 2; ++i) {
                    if (i < NC / 2) {
                        const float2 q = qs[r * NC + jlo + i];
                        acc[i].x = fmaf(h.x, q.x, fmaf(h.y, q.y, acc[i].x));
                        acc[i].y = fmaf(h.x, q.y, fmaf(-h.y, q.x, acc[i].y));
                    }
                }
            }
            for (int i = 0; i < NC / 2; ++i)
                if (jlo + i < ncols) L.x[(size_t)(col0 + jlo + i) * Nt + n] = acc[i];
        }
        (void)jhi;
        for (int u = tid; u < nown * NC; u += GT) {
            const int kk = u / NC, j = u % NC;
            if (j < ncols && L.v) L.v[(size_t)(col0 + j) * K + k0 + kk] = o_q[u];
        }
        if (b == 0 && tid < ncols) {
            L.iters[col0 + tid] = c_iters[tid];
            L.resid[col0 + tid] = c_sn2[tid] > 0.0 ? sqrt(c_rt2[tid] / c_sn2[tid]) : 0.0;
        }
    }
    // a product that did not complete in time is waited for (bounded) before
    // its tensor memory is released
    if (mma_late && !wait_phase(&bar_mma, mma_par ^ 1u)) flag(L.status, KZ_STATUS_BIT_TIMEOUT);
    kz5::fence_before();
    __syncthreads();
    kz5::fence_after();
    if (warp == 0) kz5::tmem_dealloc(tmem, (uint32_t)L.tmem_cols);
}

}  // namespace

// ---------------------------------------------------------------------------
// Host side.

cudaError_t kz_grp_prepare(const KzGrpChan& C, const float2* Hc, long long total2, const int4* rows, const int* rptr,
                           const float* nrm, float* stat, int fmt, cudaStream_t st) {
    grp_stats_kernel<<<1, 1024, 0, st>>>(Hc, total2, nrm, C.K, stat);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    grp_fill_kernel<<<C.AB, 256, 0, st>>>(C, Hc, rows, rptr, stat, fmt);
    return cudaGetLastError();
}

size_t kz_grp_smem(int NC, int rtmax, int rpc, int AB) {
    const int rtrows = 128 * rtmax;
    const size_t szop = (size_t)std::max(512 * NC, 4 * NC * rtrows);
    return (size_t)2 * rtrows * 256 + szop + (size_t)5 * rpc * NC * sizeof(float2) + (size_t)3 * rpc * NC * sizeof(float) +
           (size_t)(rtrows + rpc * AB + rpc + 1) * sizeof(int);
}

// Whether AB x CG CTAs can run: cluster mode needs one resident cluster of AB
// CTAs; grid mode needs every CTA resident at once (cooperative launch).
bool kz_grp_fits(int AB, int CG, bool cluster, size_t smem) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return false;
    if (cluster) {
        auto fn = kz_grp_kernel<true>;
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return false;
        if (AB > 8 && cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
            return false;
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = AB;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(AB, CG);
        cfg.blockDim = dim3(GT);
        cfg.dynamicSmemBytes = smem;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int nclusters = 0;
        if (cudaOccupancyMaxActiveClusters(&nclusters, fn, &cfg) != cudaSuccess) {
            (void)cudaGetLastError();
            return false;
        }
        return nclusters >= 1;
    }
    auto fn = kz_grp_kernel<false>;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return false;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, GT, smem) != cudaSuccess) return false;
    return (long)AB * CG <= (long)occ * sms;
}

cudaError_t kz_launch_grp(const KzGrpLaunch& L, bool cluster, size_t smem, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    cfg.gridDim = dim3(L.C.AB, L.CG);
    cfg.blockDim = dim3(GT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (cluster) {
        auto fn = kz_grp_kernel<true>;
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess && L.C.AB > 8) e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = L.C.AB;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        return cudaLaunchKernelEx(&cfg, fn, L);
    }
    auto fn = kz_grp_kernel<false>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    return cudaLaunchKernelEx(&cfg, fn, L);
}
