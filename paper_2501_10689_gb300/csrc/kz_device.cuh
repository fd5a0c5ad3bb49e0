// Device building blocks of the Kaczmarz sweep over the rows of B = [H, sqrt(xi) I].
//
// Shared-memory layouts inside one CTA working on J columns:
//   m_s[j * Ntp + n]  iterate m (or its correction), antenna-fastest per column;
//   b_s, q_s, p_s     K x J arrays, element (i, j) at [i * J + j].
// All reductions run in a fixed order so deterministic methods are bitwise
// reproducible.
#pragma once

#include "kz_internal.h"

#define KZ_FULL 0xffffffffu

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(KZ_FULL, v, o);
    return v;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(KZ_FULL, v, o);
    return v;
}

// Antenna pair (n, n+1) of a row: {re_n, im_n, re_n+1, im_n+1}.  `off` is the
// aligned complex offset (even), so the load is 16-byte (C64) / 8-byte (BF16).
template <bool BF16>
__device__ __forceinline__ float4 h_pair(const KzInst& I, int off);

template <>
__device__ __forceinline__ float4 h_pair<false>(const KzInst& I, int off) {
    return __ldg(reinterpret_cast<const float4*>(I.Hc + off));
}

template <>
__device__ __forceinline__ float4 h_pair<true>(const KzInst& I, int off) {
    const uint2 raw = __ldg(reinterpret_cast<const uint2*>(I.Hb + off));
    const __nv_bfloat162 a = *reinterpret_cast<const __nv_bfloat162*>(&raw.x);
    const __nv_bfloat162 b = *reinterpret_cast<const __nv_bfloat162*>(&raw.y);
    const float2 fa = __bfloat1622float2(a);
    const float2 fb = __bfloat1622float2(b);
    return make_float4(fa.x, fa.y, fb.x, fb.y);
}

// acc[j] = sum_n H[i, n] m[j][n] over row i's aligned interval (warp-wide;
// every lane holds the result).  Products and sums in FP32.  Four antenna
// pairs per lane are loaded before they are used, so each lane keeps four
// independent 16-byte loads in flight.
template <int J, bool BF16>
__device__ __forceinline__ void cmac_pair(const float4& h, const float4& mm, float2& acc) {
    acc.x = fmaf(h.x, mm.x, acc.x);
    acc.x = fmaf(-h.y, mm.y, acc.x);
    acc.x = fmaf(h.z, mm.z, acc.x);
    acc.x = fmaf(-h.w, mm.w, acc.x);
    acc.y = fmaf(h.x, mm.y, acc.y);
    acc.y = fmaf(h.y, mm.x, acc.y);
    acc.y = fmaf(h.z, mm.w, acc.y);
    acc.y = fmaf(h.w, mm.z, acc.y);
}

// Columns j >= jn (a narrower work item) are neither read nor written.
template <int J, bool BF16>
__device__ __forceinline__ void row_dot(const KzInst& I, const int4* rows, const int* rptr, int i,
                                        const float2* __restrict__ m_s, int Ntp, float2 (&acc)[J], int jn = J) {
    const int lane = threadIdx.x & 31;
    const int4 rd = rows[i];
    const int base = rptr[i];
    const int pend = rd.y;
#pragma unroll
    for (int j = 0; j < J; ++j) acc[j] = make_float2(0.f, 0.f);
    // four antenna pairs per lane per step, all loads issued first; the last
    // step is predicated, so a short row costs one round trip to memory
    for (int p = 2 * lane; p < pend; p += 256) {
        float4 h[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
            h[u] = (p + 64 * u < pend) ? h_pair<BF16>(I, base + p + 64 * u) : make_float4(0.f, 0.f, 0.f, 0.f);
        const int n = rd.x + p;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (p + 64 * u >= pend) continue;
#pragma unroll
            for (int j = 0; j < J; ++j) {
                if (j >= jn) continue;
                const float4 mm = *reinterpret_cast<const float4*>(m_s + j * Ntp + n + 64 * u);
                cmac_pair<J, BF16>(h[u], mm, acc[j]);
            }
        }
    }
#pragma unroll
    for (int j = 0; j < J; ++j) {
        acc[j].x = warp_sum(acc[j].x);
        acc[j].y = warp_sum(acc[j].y);
    }
}

// Two rows per warp at once: acc0[j] = h_{i0} . m_j and acc1[j] = h_{i1} . m_j
// (i1 < 0: only i0).  Both rows' loads are in flight together, four antenna
// pairs per row per lane, which doubles the independent loads of a warp.
template <int J, bool BF16>
__device__ __forceinline__ void row_dot2(const KzInst& I, const int4* rows, const int* rptr, int i0, int i1,
                                         const float2* __restrict__ m_s, int Ntp, float2 (&acc0)[J],
                                         float2 (&acc1)[J]) {
    const int lane = threadIdx.x & 31;
    const int4 r0 = rows[i0];
    const int b0 = rptr[i0];
    int4 r1 = make_int4(0, 0, 0, 0);
    int b1 = 0;
    if (i1 >= 0) {
        r1 = rows[i1];
        b1 = rptr[i1];
    }
#pragma unroll
    for (int j = 0; j < J; ++j) acc0[j] = acc1[j] = make_float2(0.f, 0.f);
    const int len = max(r0.y, r1.y);
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int p = 2 * lane; p < len; p += 256) {
        float4 h0[4], h1[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int q = p + 64 * u;
            h0[u] = (q < r0.y) ? h_pair<BF16>(I, b0 + q) : z4;
            h1[u] = (q < r1.y) ? h_pair<BF16>(I, b1 + q) : z4;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int q = p + 64 * u;
            if (q < r0.y) {
#pragma unroll
                for (int j = 0; j < J; ++j)
                    cmac_pair<J, BF16>(h0[u], *reinterpret_cast<const float4*>(m_s + j * Ntp + r0.x + q), acc0[j]);
            }
            if (q < r1.y) {
#pragma unroll
                for (int j = 0; j < J; ++j)
                    cmac_pair<J, BF16>(h1[u], *reinterpret_cast<const float4*>(m_s + j * Ntp + r1.x + q), acc1[j]);
            }
        }
    }
#pragma unroll
    for (int j = 0; j < J; ++j) {
        acc0[j].x = warp_sum(acc0[j].x);
        acc0[j].y = warp_sum(acc0[j].y);
        acc1[j].x = warp_sum(acc1[j].x);
        acc1[j].y = warp_sum(acc1[j].y);
    }
}

// ---------------------------------------------------------------------------
// FP16 iterate of the tensor-core mode.  The correction m of the correction
// form is stored per column as m / sigma_j in FP16 (re, im) pairs, sigma_j the
// column's relative residual at the last refresh, so the stored values keep
// the scale of the solution however small the correction gets; the MMAs
// take it as stored (FP16 operands).  Antenna pair (n, n+1) of a column,
// n even: one 8-byte load (as FP32 for the CUDA-core half-step).
__device__ __forceinline__ float4 m16_pair(const __half2* p) {
    const uint2 raw = *reinterpret_cast<const uint2*>(p);
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&raw.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&raw.y));
    return make_float4(a.x, a.y, b.x, b.y);
}

// row_dot on the FP16 iterate (the caller scales by sigma_j), over the
// packed entries [p0, p1) of row i (p0 a multiple of 256).
template <int J>
__device__ __forceinline__ void row_dot_h(const KzInst& I, const int4* rows, const int* rptr, int i,
                                          const __half2* __restrict__ m16, int MS, float2 (&acc)[J], int jn,
                                          int p0, int p1) {
    const int lane = threadIdx.x & 31;
    const int4 rd = rows[i];
    const int base = rptr[i];
    const int pend = min(rd.y, p1);
#pragma unroll
    for (int j = 0; j < J; ++j) acc[j] = make_float2(0.f, 0.f);
    for (int p = p0 + 2 * lane; p < pend; p += 256) {
        float4 h[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
            h[u] = (p + 64 * u < pend) ? h_pair<false>(I, base + p + 64 * u) : make_float4(0.f, 0.f, 0.f, 0.f);
        const int n = rd.x + p;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (p + 64 * u >= pend) continue;
#pragma unroll
            for (int j = 0; j < J; ++j) {
                if (j >= jn) continue;
                cmac_pair<J, false>(h[u], m16_pair(m16 + j * MS + n + 64 * u), acc[j]);
            }
        }
    }
#pragma unroll
    for (int j = 0; j < J; ++j) {
        acc[j].x = warp_sum(acc[j].x);
        acc[j].y = warp_sum(acc[j].y);
    }
}

// m16[j][n] += g[j] conj(H[i, n]) on row i's true VR (g already divided by
// sigma_j), warp-wide, over the packed entries [p0, p1) (p0 a multiple of
// 256).  Both entries of a pair are read and written together when both
// lie in the true VR (one 8-byte access).
template <int J>
__device__ __forceinline__ void row_axpy_h(const KzInst& I, const int4* rows, const int* rptr, int i,
                                           __half2* __restrict__ m16, int MS, const float2 (&g)[J], int jn, int p0,
                                           int p1) {
    const int lane = threadIdx.x & 31;
    const int4 rd = rows[i];
    const int base = rptr[i];
    const int pend = min(rd.y, p1);
    auto apply = [&](const float4& h, int p) {
        const int n = rd.x + p;
        const bool in0 = (n >= rd.z) && (n < rd.w);
        const bool in1 = (n + 1 >= rd.z) && (n + 1 < rd.w);
#pragma unroll
        for (int j = 0; j < J; ++j) {
            if (j >= jn) continue;
            __half2* mp = m16 + j * MS + n;
            if (in0 && in1) {
                uint2 raw = *reinterpret_cast<const uint2*>(mp);
                float2 v = __half22float2(*reinterpret_cast<const __half2*>(&raw.x));
                float2 w = __half22float2(*reinterpret_cast<const __half2*>(&raw.y));
                v.x = fmaf(h.x, g[j].x, fmaf(h.y, g[j].y, v.x));
                v.y = fmaf(h.x, g[j].y, fmaf(-h.y, g[j].x, v.y));
                w.x = fmaf(h.z, g[j].x, fmaf(h.w, g[j].y, w.x));
                w.y = fmaf(h.z, g[j].y, fmaf(-h.w, g[j].x, w.y));
                const __half2 a = __float22half2_rn(v), b = __float22half2_rn(w);
                raw.x = *reinterpret_cast<const unsigned*>(&a);
                raw.y = *reinterpret_cast<const unsigned*>(&b);
                *reinterpret_cast<uint2*>(mp) = raw;
                continue;
            }
            if (in0) {
                float2 v = __half22float2(mp[0]);
                v.x = fmaf(h.x, g[j].x, fmaf(h.y, g[j].y, v.x));
                v.y = fmaf(h.x, g[j].y, fmaf(-h.y, g[j].x, v.y));
                mp[0] = __float22half2_rn(v);
            }
            if (in1) {
                float2 v = __half22float2(mp[1]);
                v.x = fmaf(h.z, g[j].x, fmaf(h.w, g[j].y, v.x));
                v.y = fmaf(h.z, g[j].y, fmaf(-h.w, g[j].x, v.y));
                mp[1] = __float22half2_rn(v);
            }
        }
    };
    for (int p = p0 + 2 * lane; p < pend; p += 256) {
        float4 h[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
            h[u] = (p + 64 * u < pend) ? h_pair<false>(I, base + p + 64 * u) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (p + 64 * u < pend) apply(h[u], p + 64 * u);
    }
}

// Knuth's TwoSum: s = fl(a + b) and the exact rounding error e (s + e == a + b).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// Compensated warp sum: hi + lo is the sum of the 32 lane values to about
// twice FP32 precision (each butterfly level adds exactly with TwoSum and
// carries the error terms in lo).  Partners combine in the same order, so
// every lane ends with the same hi and lo.
__device__ __forceinline__ void warp_sum_c(float v, float& hi, float& lo) {
    float s = v, c = 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float so = __shfl_xor_sync(KZ_FULL, s, o), co = __shfl_xor_sync(KZ_FULL, c, o);
        float e;
        two_sum(s, so, s, e);
        c = (c + co) + e;
    }
    hi = s;
    lo = c;
}

// True-residual variant (complex64 H): each lane sums its share of the row in
// FP32 (the VR is split over 32 lanes, so a lane adds at most a few dozen
// products), and the 32 lane sums are combined with compensated FP32
// additions: hi[j] + lo[j] = h_i . m_j.  No FP64 arithmetic, which runs at a
// small fraction of the FP32 rate on this GPU.
template <int J>
__device__ __forceinline__ void row_dot_c(const KzInst& I, const int4* rows, const int* rptr, int i,
                                          const float2* __restrict__ m_s, int Ntp, float2 (&hi)[J],
                                          float2 (&lo)[J], int jn = J) {
    float2 acc[J];
    const int lane = threadIdx.x & 31;
    const int4 rd = rows[i];
    const int base = rptr[i];
#pragma unroll
    for (int j = 0; j < J; ++j) acc[j] = make_float2(0.f, 0.f);
    int p = 2 * lane;
    for (; p + 192 < rd.y; p += 256) {
        float4 h[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) h[u] = h_pair<false>(I, base + p + 64 * u);
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int j = 0; j < J; ++j)
                if (j < jn)
                    cmac_pair<J, false>(h[u], *reinterpret_cast<const float4*>(m_s + j * Ntp + rd.x + p + 64 * u),
                                        acc[j]);
    }
    for (; p < rd.y; p += 64) {
        const float4 h = h_pair<false>(I, base + p);
#pragma unroll
        for (int j = 0; j < J; ++j)
            if (j < jn) cmac_pair<J, false>(h, *reinterpret_cast<const float4*>(m_s + j * Ntp + rd.x + p), acc[j]);
    }
#pragma unroll
    for (int j = 0; j < J; ++j) {
        warp_sum_c(acc[j].x, hi[j].x, lo[j].x);
        warp_sum_c(acc[j].y, hi[j].y, lo[j].y);
    }
}

// Compensated reduce-scatter of NV (a power of two, 2 <= NV <= 32) per-lane
// values: on return lane l holds in hi + lo the sum over the 32 lanes of
// value l / (32 / NV).  Each level halves the values a lane keeps (its half
// chosen by one lane bit) and adds the partner's copy of that half with
// TwoSum, carrying the rounding errors in the compensation terms; the last
// levels add the single remaining value.  Partners add in the same order, so
// both hold identical sums.  NV - 1 shuffle pairs instead of 5 NV.
template <int NV>
__device__ __forceinline__ void warp_rs_c(float (&v)[NV], float& hi, float& lo) {
    const int lane = threadIdx.x & 31;
    float c[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) c[k] = 0.f;
#pragma unroll
    for (int n = NV, o = 16; n > 1; n >>= 1, o >>= 1) {
        const bool upper = lane & o;
#pragma unroll
        for (int k = 0; k < n / 2; ++k) {
            const float sh = upper ? v[k] : v[k + n / 2], sc = upper ? c[k] : c[k + n / 2];
            const float kh = upper ? v[k + n / 2] : v[k], kc = upper ? c[k + n / 2] : c[k];
            const float rh = __shfl_xor_sync(KZ_FULL, sh, o), rc = __shfl_xor_sync(KZ_FULL, sc, o);
            float e;
            two_sum(kh, rh, v[k], e);
            c[k] = (kc + rc) + e;
        }
    }
    float sv = v[0], cv = c[0];
#pragma unroll
    for (int o = 16 / NV; o > 0; o >>= 1) {
        const float rh = __shfl_xor_sync(KZ_FULL, sv, o), rc = __shfl_xor_sync(KZ_FULL, cv, o);
        float e;
        two_sum(sv, rh, sv, e);
        cv = (cv + rc) + e;
    }
    hi = sv;
    lo = cv;
}

// True-residual products of two rows at once (i1 < 0: row i0 only), J = 4 or
// 8 columns: FP32 lane sums of both rows (four antenna pairs per row in
// flight), then one compensated reduce-scatter of the 4 J values.  The lane
// with own = true holds row `which` (0: i0, 1: i1), column j: hi + lo = h . m_j
// (each (row, column) has exactly one owner).  Columns j >= jn read nothing.
template <int J>
__device__ __forceinline__ void row_dot_c2(const KzInst& I, const int4* rows, const int* rptr, int i0, int i1,
                                           const float2* __restrict__ m_s, int Ntp, int jn, float2& hi, float2& lo,
                                           int& which, int& j, bool& own) {
    static_assert(J == 4 || J == 8, "row_dot_c2 takes 4 or 8 columns");
    constexpr int NV = 4 * J;        // (row, column, re / im)
    constexpr int LPV = 32 / NV;     // lanes holding each value after the scatter
    const int lane = threadIdx.x & 31;
    const int4 r0 = rows[i0];
    const int b0 = rptr[i0];
    int4 r1 = make_int4(0, 0, 0, 0);
    int b1 = 0;
    if (i1 >= 0) {
        r1 = rows[i1];
        b1 = rptr[i1];
    }
    float2 acc0[J], acc1[J];
#pragma unroll
    for (int jj = 0; jj < J; ++jj) acc0[jj] = acc1[jj] = make_float2(0.f, 0.f);
    const int len = max(r0.y, r1.y);
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int p = 2 * lane; p < len; p += 256) {
        float4 h0[4], h1[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int q = p + 64 * u;
            h0[u] = (q < r0.y) ? h_pair<false>(I, b0 + q) : z4;
            h1[u] = (q < r1.y) ? h_pair<false>(I, b1 + q) : z4;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int q = p + 64 * u;
#pragma unroll
            for (int jj = 0; jj < J; ++jj) {
                if (jj >= jn) continue;
                if (q < r0.y)
                    cmac_pair<J, false>(h0[u], *reinterpret_cast<const float4*>(m_s + jj * Ntp + r0.x + q), acc0[jj]);
                if (q < r1.y)
                    cmac_pair<J, false>(h1[u], *reinterpret_cast<const float4*>(m_s + jj * Ntp + r1.x + q), acc1[jj]);
            }
        }
    }
    float v[NV];
#pragma unroll
    for (int jj = 0; jj < J; ++jj) {
        v[2 * jj] = acc0[jj].x;
        v[2 * jj + 1] = acc0[jj].y;
        v[2 * J + 2 * jj] = acc1[jj].x;
        v[2 * J + 2 * jj + 1] = acc1[jj].y;
    }
    float h, l;
    warp_rs_c<NV>(v, h, l);
    const int idx = lane / LPV;
    // the imaginary part sits LPV lanes above the real part
    const float him = __shfl_down_sync(KZ_FULL, h, LPV), lim = __shfl_down_sync(KZ_FULL, l, LPV);
    hi = make_float2(h, him);
    lo = make_float2(l, lim);
    which = idx / (2 * J);
    j = (idx % (2 * J)) / 2;
    own = (idx % 2 == 0) && (lane % LPV == 0) && (which == 0 || i1 >= 0);
}

// (H H^H q)_i = sum over l in X_i of G_il q_l through the Gram matrix on the
// overlap pattern (the VRs of rows outside X_i are disjoint from row i's, so
// their entries are zero): the same sum as h_i . (H^H q) from one pass over
// the row's overlap set instead of its VR, for two rows i0 and i1 of a warp
// at once (i1 < 0: none).  Lane (slot, j) = (lane / J, lane % J) takes column
// j of every (32 / J)-th entry: the warp loads 32 entries (index and G value)
// at a time, coalesced, and hands them round by shuffles, so the q reads of a
// pass hit consecutive shared-memory words.  The loads of up to four such
// groups of 32 entries of both rows are in flight together (a row's overlap
// set rarely has more than 128 entries, so one L2 round trip per two rows);
// xptr: the CSR offsets of the overlap sets (shared memory).  FP32 complex
// products, each row's entries added in list order; the 32 / J lanes of a
// column are then added with compensated sums.  Every lane returns hi + lo
// for its column j of each row (columns j >= jn are not read and return 0).
template <int J>
__device__ __forceinline__ void gram_rows_t(const KzInst& I, const int* xptr, int i0, int i1,
                                            const float2* __restrict__ q_s, int jn, float2 (&hi)[2],
                                            float2 (&lo)[2]) {
    constexpr int EPP = 32 / J;  // entries per pass
    constexpr int CH = 4;        // groups of 32 entries of a row loaded together
    const int lane = threadIdx.x & 31, slot = lane / J, j = lane % J;
    float ax[2] = {0.f, 0.f}, ay[2] = {0.f, 0.f};
    int eb[2], ee[2];
    eb[0] = xptr[i0];
    ee[0] = xptr[i0 + 1];
    eb[1] = i1 >= 0 ? xptr[i1] : 0;
    ee[1] = i1 >= 0 ? xptr[i1 + 1] : 0;
    for (int round = 0; eb[0] + 32 * CH * round < ee[0] || eb[1] + 32 * CH * round < ee[1]; ++round) {
        int l[2][CH];
        float2 g[2][CH];
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                const int e = eb[r] + 32 * (CH * round + c) + lane;
                l[r][c] = 0;
                g[r][c] = make_float2(0.f, 0.f);
                if (e < ee[r]) {
                    l[r][c] = __ldg(I.xidx + e);
                    g[r][c] = __ldg(I.G + e);
                }
            }
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                const int b0 = eb[r] + 32 * (CH * round + c);
                if (b0 >= ee[r]) break;  // the same in every lane
#pragma unroll
                for (int p = 0; p < J; ++p) {
                    const int src = p * EPP + slot;
                    const int ls = __shfl_sync(KZ_FULL, l[r][c], src);
                    const float gx = __shfl_sync(KZ_FULL, g[r][c].x, src), gy = __shfl_sync(KZ_FULL, g[r][c].y, src);
                    if (b0 + src < ee[r] && j < jn) {
                        const float2 q = q_s[ls * J + j];
                        ax[r] = fmaf(gx, q.x, fmaf(-gy, q.y, ax[r]));
                        ay[r] = fmaf(gx, q.y, fmaf(gy, q.x, ay[r]));
                    }
                }
            }
    }
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        float sx = ax[r], sy = ay[r], cx = 0.f, cy = 0.f;
#pragma unroll
        for (int o = J; o < 32; o <<= 1) {
            const float rx = __shfl_xor_sync(KZ_FULL, sx, o), rcx = __shfl_xor_sync(KZ_FULL, cx, o);
            const float ry = __shfl_xor_sync(KZ_FULL, sy, o), rcy = __shfl_xor_sync(KZ_FULL, cy, o);
            float e;
            two_sum(sx, rx, sx, e);
            cx = (cx + rcx) + e;
            two_sum(sy, ry, sy, e);
            cy = (cy + rcy) + e;
        }
        hi[r] = make_float2(sx, sy);
        lo[r] = make_float2(cx, cy);
    }
}

// b - h_i . m - xi q from row_dot_c's hi + lo: b - hi is exact when the two
// nearly cancel, and xi q enters through one fused multiply-add.
__device__ __forceinline__ float2 true_resid(float2 b, float2 hi, float2 lo, float2 q, float xi) {
    return make_float2(fmaf(-xi, q.x, (b.x - hi.x) - lo.x), fmaf(-xi, q.y, (b.y - hi.y) - lo.y));
}

// m[j][n] += g[j] * conj(H[i, n]) on row i's true VR [o, e) (warp-wide).
// Restricting to the true VR keeps rows of the orthogonal set, whose aligned
// intervals may share an edge pair, from writing the same element.
template <int J, bool BF16>
__device__ __forceinline__ void row_axpy(const KzInst& I, const int4* rows, const int* rptr, int i,
                                         float2* __restrict__ m_s, int Ntp, const float2 (&g)[J], int lane,
                                         int nlanes, int jn = J) {
    const int4 rd = rows[i];
    const int base = rptr[i];
    const int pend = rd.y;
    auto apply = [&](const float4& h, int p) {
        const int n = rd.x + p;
        const bool in0 = (n >= rd.z) && (n < rd.w);
        const bool in1 = (n + 1 >= rd.z) && (n + 1 < rd.w);
#pragma unroll
        for (int j = 0; j < J; ++j) {
            if (j >= jn) continue;
            float2* mp = m_s + j * Ntp + n;
            if (in0) {
                float2 v = mp[0];
                v.x = fmaf(h.x, g[j].x, fmaf(h.y, g[j].y, v.x));
                v.y = fmaf(h.x, g[j].y, fmaf(-h.y, g[j].x, v.y));
                mp[0] = v;
            }
            if (in1) {
                float2 v = mp[1];
                v.x = fmaf(h.z, g[j].x, fmaf(h.w, g[j].y, v.x));
                v.y = fmaf(h.z, g[j].y, fmaf(-h.w, g[j].x, v.y));
                mp[1] = v;
            }
        }
    };
    const int step = 2 * nlanes;
    // four antenna pairs per lane in flight before they are applied; the last
    // step is predicated
    for (int p = 2 * lane; p < pend; p += 4 * step) {
        float4 h[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
            h[u] = (p + u * step < pend) ? h_pair<BF16>(I, base + p + u * step) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (p + u * step < pend) apply(h[u], p + u * step);
    }
}

// u[j] at antennas (n, n+1), n = 64 * tile + 2 * lane:
//   u_n = sum_{k in [k0, k1)} conj(H[i_k, n]) * coef[i_k][j]
// over the covering-row list entries k0..k1 of the tile (antenna-major, no
// scatter).  trow4[k] = {row, rptr - a, a, a + len2}.  Four rows are fetched
// before they are used (independent loads in flight).
template <int J>
__device__ __forceinline__ void cmac_conj(const float4& h, const float2& c, float2& u0, float2& u1) {
    u0.x = fmaf(h.x, c.x, fmaf(h.y, c.y, u0.x));
    u0.y = fmaf(h.x, c.y, fmaf(-h.y, c.x, u0.y));
    u1.x = fmaf(h.z, c.x, fmaf(h.w, c.y, u1.x));
    u1.y = fmaf(h.z, c.y, fmaf(-h.w, c.x, u1.y));
}

template <int J, bool BF16>
__device__ __forceinline__ void tile_accum(const KzInst& I, const int4* __restrict__ trow4, int tile, int k0,
                                           int k1, const float2* __restrict__ coef, float2 (&u0)[J],
                                           float2 (&u1)[J]) {
    const int lane = threadIdx.x & 31;
    const int n = tile * KZ_TILE + 2 * lane;
#pragma unroll
    for (int j = 0; j < J; ++j) u0[j] = u1[j] = make_float2(0.f, 0.f);
    const int4 none = make_int4(0, 0, 0, 0);  // empty interval: never matches
    int4 en[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) en[u] = (k0 + u < k1) ? __ldg(trow4 + k0 + u) : none;
    for (int k = k0; k < k1; k += 4) {
        int4 e[4];
        float4 h[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) e[u] = en[u];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const bool in = (n >= e[u].z) && (n < e[u].w);
            h[u] = in ? h_pair<BF16>(I, e[u].y + n) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        // descriptors of the next batch, in flight while this batch is used
#pragma unroll
        for (int u = 0; u < 4; ++u) en[u] = (k + 4 + u < k1) ? __ldg(trow4 + k + 4 + u) : none;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (k + u < k1) {
#pragma unroll
                for (int j = 0; j < J; ++j) cmac_conj<J>(h[u], coef[e[u].x * J + j], u0[j], u1[j]);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Tensor-core inner products (warp-level mma.sync m16n8k16, FP16 operands,
// FP32 accumulation).  Every operand carries FP16's 11-bit significand: the
// channel from its FP16 copy (each row scaled by a power of two, so its
// entries keep full precision), the correction iterate as stored (FP16,
// scaled per column) and phi scaled per column by its RMS.  These products
// serve the inner iteration of the correction form only: its right-hand side
// b = s - H m_ref is recomputed from the complex64 H at every refresh, and
// stops are confirmed on that true residual.
//
// Fragment ownership (lane = 4 g + c; two FP16 values per register, the
// lower K index in the low half): A (16 x 16, row-major) a0 = (g, 2c | 2c + 1),
// a1 = (g + 8, 2c | 2c + 1), a2 = (g, 2c + 8 | 2c + 9), a3 = (g + 8, 2c + 8 | 2c + 9);
// B (16 x 8) b0 = (2c | 2c + 1, g), b1 = (2c + 8 | 2c + 9, g); D (16 x 8, FP32)
// d0 = (g, 2c), d1 = (g, 2c + 1), d2 = (g + 8, 2c), d3 = (g + 8, 2c + 1).
__device__ __forceinline__ void mma_f16(float (&d)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                        unsigned b0, unsigned b1) {
    asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// An FP16 pair {re, im} as {re, -im} (sign bit of the high half) and as
// {im, re} (halves swapped).
__device__ __forceinline__ unsigned h2_conj(unsigned v) { return v ^ 0x80000000u; }
__device__ __forceinline__ unsigned h2_swap(unsigned v) { return __byte_perm(v, 0u, 0x1032); }

__device__ __forceinline__ unsigned h2_pack(float lo, float hi) {
    const __half2 t = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<const unsigned*>(&t);
}

// Products H m_j for a block of 8 rows, vs[8 b .. 8 b + 8) (fewer at the end
// of the list, nv entries), over the antenna range [nbeg, nend) (nbeg a
// multiple of 16, nend of 4; a block's union interval is cut into such parts),
// sixteen antennas per pair of MMAs, K = (antenna, re | im):
//   A[(j, re)][(n, re | im)] = {Re, -Im} m_j(n),  A[(j, im)][(n, re | im)] = {Im, Re} m_j(n)
// (row j of the 16 for (j, re), row j + 8 for (j, im); j < W, the rest zero),
// B[(n, re | im)][row] = {Re, Im} H[row, n] (zero outside the row's interval),
// so D[(j, re | im)][row] = Re | Im (H m_j)[row] over the range, in the units
// of the FP16 copies (times hs_row sigma_j in true units).  Lane (g, c) loads
// antennas n .. n + 3 (n = n0 + 4c) of row g and of m_g as one 16-byte load
// each: the first MMA takes n (K = 2c, 2c + 1) and n + 1 (K = 2c + 8, 2c + 9),
// the second n + 2 and n + 3.  (Aligned intervals start and end on multiples
// of four antennas, so the four antennas of a load are inside or outside a
// row together.)  Lane (g, c) returns column j = g of rows 2c (d[0] + i d[2])
// and 2c + 1 (d[1] + i d[3]) of the block.  m16: the FP16 iterate, column
// stride MS (a multiple of 4; columns 16-byte aligned).
template <int J>
__device__ __forceinline__ void tc_row_part(const __half2* __restrict__ Hh, const int4* rows, const int* rptr,
                                            const int* vs, int nv, int b, int nbeg, int nend,
                                            const __half2* __restrict__ m16, int MS, int W, float (&d)[4]) {
    const int lane = threadIdx.x & 31, g = lane >> 2, c = lane & 3;
    const int k = 8 * b + g;
    int a = 0, len = 0, hb = 0;
    if (k < nv) {
        const int row = vs[k];
        const int4 rd = rows[row];
        a = rd.x;
        len = rd.y;
        hb = rptr[row] - rd.x;
    }
    // four accumulator sets (first / second MMA of a load x even / odd step
    // u), so no MMA waits on the one before it
    float e[4] = {0.f, 0.f, 0.f, 0.f}, d2[4] = {0.f, 0.f, 0.f, 0.f}, e2[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int u = 0; u < 4; ++u) d[u] = 0.f;
    const bool jok = g < W;  // W <= J columns of this item
    const __half2* mj = m16 + (jok ? g : 0) * MS;
    const uint4 z = make_uint4(0u, 0u, 0u, 0u);
    // eight 16-byte H loads per lane per step (128 antennas of the row), all
    // in flight before the first MMA of the step; the iterate is read from
    // shared memory next to its MMAs.  Entries at or beyond nend are zero on
    // both sides.
    constexpr int U = 8;
    for (int n0 = nbeg; n0 < nend; n0 += 16 * U) {
        uint4 h[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int n = n0 + 16 * u + 4 * c;
            h[u] = (n < nend && (unsigned)(n - a) < (unsigned)len)
                       ? __ldg(reinterpret_cast<const uint4*>(Hh + hb + n))
                       : z;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int n = n0 + 16 * u + 4 * c;
            const uint4 m = (jok && n < nend) ? *reinterpret_cast<const uint4*>(mj + n) : z;
            if (u & 1) {
                mma_f16(d2, h2_conj(m.x), h2_swap(m.x), h2_conj(m.y), h2_swap(m.y), h[u].x, h[u].y);
                mma_f16(e2, h2_conj(m.z), h2_swap(m.z), h2_conj(m.w), h2_swap(m.w), h[u].z, h[u].w);
            } else {
                mma_f16(d, h2_conj(m.x), h2_swap(m.x), h2_conj(m.y), h2_swap(m.y), h[u].x, h[u].y);
                mma_f16(e, h2_conj(m.z), h2_swap(m.z), h2_conj(m.w), h2_swap(m.w), h[u].z, h[u].w);
            }
        }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) d[u] = (d[u] + e[u]) + (d2[u] + e2[u]);
}

// u = H_V^H phi on one half (32 antennas, part 0 or 1) of a 64-antenna
// tile, antenna-major, sixteen covering rows (list entries k0..k1 of the
// tile) per step, four MMAs per block of four columns:
//   A[(n, re)][row] = Re H[row, n],  A[(n, im)][row] = Im H[row, n]
//   (rows g and g + 8 of the 16 for antenna n = s + 4 g + q of MMA q < 4),
//   B[row][(j, re | im)] = {Re, Im} phi[row][j] hs_row / tau_j
//   (columns 4 nb .. 4 nb + 3 per block nb of the 8 N entries).
// Lane (g, c) loads antennas s + 4 g .. s + 4 g + 3 of the step's covering
// rows 2c, 2c + 1, 2c + 8 and 2c + 9 (its K indices), one 16-byte load each,
// and pairs two rows' real (imaginary) parts of an antenna in one register;
// acc[q][nb] holds the products of antenna s + 4 g + q, whose sums and
// differences give u / tau_j (tc_u_combine).  coef: K x J phi in shared
// memory (FP32); hs: the rows' scales; itau[nb] = 1 / tau_j for this lane's
// column j = 4 nb + (g & 3) (0 for a column whose phi is zero).
// STAGED: the entries' row indices come from trow_s and their intervals and
// offsets from rows / rptr (shared memory) instead of trow4 (global).
template <int J, bool STAGED>
__device__ __forceinline__ void tc_tile_aggr(const __half2* __restrict__ Hh, const int4* __restrict__ trow4,
                                             const unsigned short* trow_s, const int4* rows, const int* rptr,
                                             const float* hs, int tile, int part, int k0, int k1,
                                             const float2* __restrict__ coef, const float (&itau)[J / 4],
                                             float (&acc)[4][J / 4][4]) {
    constexpr int NB = J / 4;
    const int lane = threadIdx.x & 31, g = lane >> 2, c = lane & 3;
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int nb = 0; nb < NB; ++nb)
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[q][nb][u] = 0.f;
    const int4 none = make_int4(0, 0, 0, 0);  // empty interval: never matches
    const uint4 z4 = make_uint4(0u, 0u, 0u, 0u);
    const int n = tile * KZ_TILE + 32 * part + 4 * g;
    auto entry = [&](int kk) -> int4 {
        if (kk >= k1) return none;
        if constexpr (STAGED) {
            const int r = trow_s[kk];
            const int4 rd = rows[r];
            return make_int4(r, rptr[r] - rd.x, rd.x, rd.x + rd.y);
        } else {
            return __ldg(trow4 + kk);
        }
    };
    // list offsets of this lane's four rows in a step
    int off[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) off[i] = 2 * c + (i & 1) + 8 * (i >> 1);
    int4 nxt[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) nxt[i] = entry(k0 + off[i]);
    for (int k = k0; k < k1; k += 16) {
        int4 e[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) e[i] = nxt[i];
        uint4 h[4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
            h[i] = (n >= e[i].z && n < e[i].w) ? __ldg(reinterpret_cast<const uint4*>(Hh + e[i].y + n)) : z4;
        // descriptors of the next step, in flight while this one is used
#pragma unroll
        for (int i = 0; i < 4; ++i) nxt[i] = entry(k + 16 + off[i]);
        // B: the four rows' phi in this lane's column slots, scaled by the
        // row's hs and the column's 1 / tau (0 for a list entry past the end)
        float sc[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) sc[i] = (k + off[i] < k1) ? hs[e[i].x] : 0.f;
        unsigned b0[NB], b1[NB];
#pragma unroll
        for (int nb = 0; nb < NB; ++nb) {
            const int j = 4 * nb + (g & 3);
            float v[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float2 p = sc[i] != 0.f ? coef[e[i].x * J + j] : make_float2(0.f, 0.f);
                v[i] = ((g >> 2) ? p.y : p.x) * (sc[i] * itau[nb]);
            }
            b0[nb] = h2_pack(v[0], v[1]);
            b1[nb] = h2_pack(v[2], v[3]);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const unsigned w0 = q == 0 ? h[0].x : q == 1 ? h[0].y : q == 2 ? h[0].z : h[0].w;
            const unsigned w1 = q == 0 ? h[1].x : q == 1 ? h[1].y : q == 2 ? h[1].z : h[1].w;
            const unsigned w2 = q == 0 ? h[2].x : q == 1 ? h[2].y : q == 2 ? h[2].z : h[2].w;
            const unsigned w3 = q == 0 ? h[3].x : q == 1 ? h[3].y : q == 2 ? h[3].z : h[3].w;
            const unsigned a0 = __byte_perm(w0, w1, 0x5410), a1 = __byte_perm(w0, w1, 0x7632);
            const unsigned a2 = __byte_perm(w2, w3, 0x5410), a3 = __byte_perm(w2, w3, 0x7632);
#pragma unroll
            for (int nb = 0; nb < NB; ++nb) mma_f16(acc[q][nb], a0, a1, a2, a3, b0[nb], b1[nb]);
        }
    }
}

// Sums and differences of tc_tile_aggr's products (all lanes take part):
// lanes c < 2 return u at the products' antenna for columns
// j = 4 nb + 2c (u0) and j + 1 (u1).  With the partner lane c + 2 (which
// holds the Im phi products):  Re u = Re H Re phi + Im H Im phi,
// Im u = Re H Im phi - Im H Re phi.
__device__ __forceinline__ void tc_u_combine(const float (&a)[4], float2& u0, float2& u1) {
    const float e0 = __shfl_xor_sync(KZ_FULL, a[0], 2), e1 = __shfl_xor_sync(KZ_FULL, a[1], 2);
    const float e2 = __shfl_xor_sync(KZ_FULL, a[2], 2), e3 = __shfl_xor_sync(KZ_FULL, a[3], 2);
    u0 = make_float2(a[0] + e2, e0 - a[2]);
    u1 = make_float2(a[1] + e3, e1 - a[3]);
}

// Drops the 128-byte L2 line at p (128-byte aligned) without writing it back:
// for scratch whose content is dead and is rewritten before it is read again.
__device__ __forceinline__ void kz_discard_l2(const void* p) {
    asm volatile("discard.global.L2 [%0], 128;" ::"l"(p) : "memory");
}

// Column `col` of an Nt-long complex output: entries n and n + 1 (n < Nt).
// One 16-byte store when the pair is inside the column and its address is
// 16-byte aligned (the caller's buffer need only be 8-byte aligned), else
// two 8-byte stores.
__device__ __forceinline__ void kz_store_pair(float2* out, int Nt, int col, int n, bool on, float2 a, float2 b) {
    if (!on) return;
    float2* p = out + (size_t)col * Nt + n;
    if (n + 1 < Nt && (reinterpret_cast<uintptr_t>(p) & 15) == 0) {
        *reinterpret_cast<float4*>(p) = make_float4(a.x, a.y, b.x, b.y);
    } else {
        p[0] = a;
        if (n + 1 < Nt) p[1] = b;
    }
}

// ---------------------------------------------------------------------------
// SplitMix64 (Steele, Lea & Flood 2014): counter-based uniform draws keyed by
// (seed, instance, column, iteration).
#define KZ_GOLDEN 0x9E3779B97F4A7C15ull

__device__ __forceinline__ unsigned long long kz_mix64(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ double kz_uniform(unsigned long long seed, int inst, int col, int t) {
    const unsigned long long ctr = ((unsigned long long)(unsigned)inst << 32) + (unsigned long long)(unsigned)col + 1ull;
    const unsigned long long key = kz_mix64(seed + ctr * KZ_GOLDEN);
    const unsigned long long z = kz_mix64(key + (unsigned long long)(t + 1) * KZ_GOLDEN);
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

// Warp-wide inverse-CDF draw: the smallest i with (running sum of w up to i)
// > u * total, weights given per row by `wfun(i)` (FP64).  Each lane owns a
// contiguous block of rows.  Returns -1 when every weight is zero.
template <class WF>
__device__ __forceinline__ int warp_pick(int K, double u, WF wfun) {
    const int lane = threadIdx.x & 31;
    const int C = (K + 31) / 32;
    const int lo = min(lane * C, K), hi = min(lo + C, K);
    double local = 0.0;
    int lastpos = -1;
    for (int i = lo; i < hi; ++i) {
        const double w = wfun(i);
        local += w;
        if (w > 0.0) lastpos = i;
    }
    // inclusive scan over lanes
    double incl = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double y = __shfl_up_sync(KZ_FULL, incl, o);
        if (lane >= o) incl += y;
    }
    const double total = __shfl_sync(KZ_FULL, incl, 31);
    const double target = u * total;
    int cand = K;
    if (total > 0.0 && incl > target) {
        double cum = incl - local;
        for (int i = lo; i < hi; ++i) {
            cum += wfun(i);
            if (cum > target) {
                cand = i;
                break;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cand = min(cand, __shfl_xor_sync(KZ_FULL, cand, o));
    if (cand == K) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) lastpos = max(lastpos, __shfl_xor_sync(KZ_FULL, lastpos, o));
        cand = lastpos;
    }
    return cand;
}

// Warp-wide argmax of ratio(i) with the lowest index on ties.
template <class RF>
__device__ __forceinline__ int warp_argmax(int K, RF rfun, double* best_out) {
    const int lane = threadIdx.x & 31;
    double best = -1.0;
    int bi = K;
    for (int i = lane; i < K; i += 32) {
        const double v = rfun(i);
        if (v > best) {
            best = v;
            bi = i;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(KZ_FULL, best, o);
        const int oi = __shfl_xor_sync(KZ_FULL, bi, o);
        if (ob > best || (ob == best && oi < bi)) {
            best = ob;
            bi = oi;
        }
    }
    if (best_out) *best_out = best;
    return bi < K ? bi : -1;
}

__device__ __forceinline__ void kz_flag(int* status, int bit) {
    if (status) atomicOr(status, bit);
}

// Copy an instance descriptor into shared memory (block-wide; caller syncs).
__device__ __forceinline__ void load_inst(KzInst& dst, const KzInst* src) {
    const int nwords = (int)(sizeof(KzInst) / 4);
    const int* s = reinterpret_cast<const int*>(src);
    int* d = reinterpret_cast<int*>(&dst);
    for (int w = threadIdx.x; w < nwords; w += blockDim.x) d[w] = s[w];
}
