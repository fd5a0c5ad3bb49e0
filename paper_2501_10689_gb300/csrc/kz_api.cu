// C-ABI of libkzprecode: argument checking, the per-channel host set-up
// (step A0) and the launches.  See include/kzprecode.h for the contract.
#include <atomic>
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "kz_internal.h"

namespace {

thread_local std::string g_err;

// Dynamic shared memory budget per CTA: the 227 KiB opt-in maximum less room
// for the kernels' static shared memory (at most 6 KiB).
constexpr size_t kSmemLimit = 227 * 1024 - 8 * 1024;

template <class T>
cudaError_t upload(T** dst, const std::vector<T>& v, cudaStream_t st) {
    *dst = nullptr;
    const size_t bytes = std::max<size_t>(v.size(), 1) * sizeof(T);
    cudaError_t e = cudaMalloc((void**)dst, bytes);
    if (e != cudaSuccess) return e;
    if (!v.empty()) e = cudaMemcpyAsync(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st);
    return e;
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

int sm_count() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
    return std::max(n, 1);
}

}  // namespace

void kz_set_error(const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
}

// Set-up of the group kernel (built on its first use): per 128-antenna block
// the rows meeting it and their 16-bit tile image, the compact index of the
// residual partial sums, and the kernel's scratch (grown on demand).
struct GrpPlan {
    bool built = false;
    int fmt = -1, AB = 0, rtmax = 1, n_slots = 0;
    int *d_slot = nullptr, *d_nrt = nullptr, *d_nb = nullptr, *d_coff = nullptr, *d_cptr = nullptr,
        *d_cidx = nullptr;
    long long* d_toff = nullptr;
    unsigned char* d_inF = nullptr;
    uint8_t* d_tiles = nullptr;
    float* d_stat = nullptr;
    void* d_scr = nullptr;
    size_t scr_bytes = 0;
    void release() {
        void* ps[] = {d_slot, d_nrt, d_nb, d_coff, d_cptr, d_cidx, d_toff, d_inF, d_tiles, d_stat, d_scr};
        for (void* p : ps)
            if (p) cudaFree(p);
        *this = GrpPlan();
    }
};

struct kz_plan {
    int K = 0, Nt = 0, Ntp = 0, ntiles = 0, nF = 0;
    int cmax = 0;  // largest number of rows covering one tile
    int n_trow = 0;  // covering-list entries over all tiles
    int64_t sumL = 0, total2 = 0;
    kz_prec prec = KZ_C64;
    std::vector<int> F, xptr, xidx;
    // device
    int4* d_rows = nullptr;
    int* d_rptr = nullptr;
    int* d_in_off = nullptr;
    float* d_nrm = nullptr;
    double* d_nrmd = nullptr;
    int* d_order = nullptr;
    int* d_xptr = nullptr;
    int* d_xidx = nullptr;
    int* d_tptr = nullptr;
    int* d_tnv = nullptr;
    int4* d_trow4 = nullptr;
    int* d_vsort = nullptr;
    float2* d_G = nullptr;  // H H^H on the X_k pattern
    float2* d_Hc = nullptr;
    __nv_bfloat162* d_Hb = nullptr;
    __half2* d_Hh = nullptr;  // complex64 plans: FP16 rows scaled by 1 / hs (tensor-core contractions)
    float* d_hs = nullptr;
    float2* d_scratch = nullptr;  // adjoint right-hand side G~ (grown on demand)
    size_t scratch_elems = 0;
    int sms = 1;
    std::vector<int> vr_off, vr_len;  // the caller's VRs
    GrpPlan grp;
    // kz_precoder_matrix: Q_s of the last subarray count used, and partial sums
    int q_S = 0;
    int *d_qptr = nullptr, *d_qidx = nullptr;
    double* d_qpart = nullptr;
    size_t qpart_n = 0;

    ~kz_plan() {
        void* ps[] = {d_rows, d_rptr, d_in_off, d_nrm, d_nrmd, d_order, d_xptr, d_xidx,
                      d_tptr, d_tnv, d_trow4, d_vsort, d_G, d_Hc, d_Hb, d_Hh, d_hs, d_scratch};
        for (void* p : ps)
            if (p) cudaFree(p);
        grp.release();
        void* qs[] = {d_qptr, d_qidx, d_qpart};
        for (void* p : qs)
            if (p) cudaFree(p);
    }

    KzInst inst() const {
        KzInst I;
        memset(&I, 0, sizeof(I));
        I.K = K;
        I.Nt = Nt;
        I.Ntp = Ntp;
        I.ntiles = ntiles;
        I.nF = nF;
        I.rows = d_rows;
        I.rptr = d_rptr;
        I.nrm = d_nrm;
        I.order = d_order;
        I.xptr = d_xptr;
        I.xidx = d_xidx;
        I.tptr = d_tptr;
        I.tnv = d_tnv;
        I.trow4 = d_trow4;
        I.Hc = d_Hc;
        I.Hb = d_Hb;
        I.Hh = d_Hh;
        I.hs = d_hs;
        I.nrmd = d_nrmd;
        I.in_off = d_in_off;
        I.vsort = d_vsort;
        I.G = d_G;
        I.cmax = cmax;
        return I;
    }
};

struct kz_batch {
    int n = 0, nrhs = 0, J = 1, nw = 16, grid = 1, n_items = 0, Ntp_max = 0, K_max = 0;
    int kernel = KZ_KERNEL_RESIDENT, cmax = 0;
    int m_elems = 0;               // tensor-core kernel: shared iterate entries per CTA
    int trow_max = 0, trow_max2 = 0;  // tensor-core kernel: staged covering-list entries (0: none)
    std::vector<int> Ntp_of;       // per instance
    std::vector<double> cost;  // per-instance work estimate ((aligned entries + 4 Nt) x (0.036 + coupling))
    size_t smem = 0;
    kz_algo algo = KZ_VR_OAHK;
    kz_prec prec = KZ_C64;
    KzInst* d_insts = nullptr;
    int2* d_items = nullptr;
    int* d_queue = nullptr;
    KzAdjItem* d_adj = nullptr;  // adjoint item table (allocated on first use)
    int2* d_rowmap = nullptr;    // kz_batch_update: {item, row} of every row of every item
    long long* d_hoff = nullptr; // kz_batch_update: item b's offset in the concatenated channels
    int n_rows = 0;
    std::vector<int> row_start;  // kz_batch_update: first rowmap entry of every item (n + 1)
    bool all_v = true;           // every item has a v buffer
    bool gk = false;             // prepared as KZ_GK: GRK with the argmax rule
    std::vector<const kz_plan*> plans;  // the items' plans, fixed at preparation
    std::vector<KzInst> h_insts;        // host copy of the instance table
    // Tensor-core kernel at J = 8 over channels of both widths: the 4-column
    // items run as a second launch of the J = 4 kernel, on an auxiliary stream
    // forked from and joined to the caller's.
    int2* d_items2 = nullptr;
    int n_items2 = 0, grid2 = 0, m_elems2 = 0;
    size_t smem2 = 0;
    cudaStream_t aux = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    ~kz_batch() {
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (ev_join) cudaEventDestroy(ev_join);
        if (aux) cudaStreamDestroy(aux);
        if (d_items2) cudaFree(d_items2);
        if (d_adj) cudaFree(d_adj);
        if (d_rowmap) cudaFree(d_rowmap);
        if (d_hoff) cudaFree(d_hoff);
        if (d_insts) cudaFree(d_insts);
        if (d_items) cudaFree(d_items);
        if (d_queue) cudaFree(d_queue);
    }
};

namespace {

bool is_ahk_family(kz_algo a) { return a == KZ_AHK || a == KZ_VR_OAHK; }

bool valid_algo(int a) { return a >= KZ_RK_ENERGY && a <= KZ_GK; }

// Refresh period: the drift correction of C64, the correction-form refresh
// of BF16_MIXED and of the tensor-core kernel (whose FP16 products slow the
// iteration when the correction grows for longer; on the 512-channel batch
// periods 7 to 10 are within 1% of each other).
int default_refresh(kz_algo a, kz_prec p, bool tc = false) {
    if (is_ahk_family(a)) return tc ? 8 : (p == KZ_BF16_MIXED ? 6 : 16);
    return 512;
}

size_t smem_for(kz_algo a, int J, int Ntp, int K, kz_prec p) {
    return is_ahk_family(a) ? kz_smem_ahk(J, Ntp, K, p) : kz_smem_kacz(J, Ntp, K);
}

int occupancy_for(kz_algo a, int J, int nw, size_t smem, kz_prec p) {
    return is_ahk_family(a) ? kz_occupancy_ahk(J, nw, smem, p) : kz_occupancy_kacz(J, nw, smem);
}

// J (columns per CTA): the largest of {8, 4, 2, 1} that fits shared memory
// and still gives every SM a work item; 1 when there are few columns.
int choose_J(kz_algo a, int nrhs_total_items_base, int Ntp, int K, kz_prec p, int sms, int per_inst_cols) {
    for (int J : {8, 4, 2}) {
        if (J > per_inst_cols) continue;
        if (smem_for(a, J, Ntp, K, p) > kSmemLimit / 2 + 8 * 1024) continue;
        const long items = (long)nrhs_total_items_base * ((per_inst_cols + J - 1) / J);
        if (items >= 2L * sms) return J;
    }
    return 1;
}

int choose_nw(int Ntp) { return (Ntp / KZ_TILE) >= 16 ? 16 : 8; }

// Work items of a batch for J columns per CTA and nw warps: {instance, first
// column} ordered by estimated cost, largest first; grid = resident CTAs.
cudaError_t batch_layout_k(kz_batch* B, int kernel, int J, int nw, int sms, cudaStream_t st);
cudaError_t batch_layout(kz_batch* B, int J, int nw, int sms, cudaStream_t st) {
    return batch_layout_k(B, KZ_KERNEL_RESIDENT, J, nw, sms, st);
}
// Tensor-core kernel: the width (columns) of instance b's items, the largest
// of J, J / 2, ... (at least 4) whose iterate columns fit shared memory next to
// the widest other instance's; 0 if even 4 do not fit.
// The covering lists' row indices are staged in shared memory when they fit
// next to everything else (16-bit indices: K below 65536).
bool tc_stage_ok(int J, int m_elems, int Ntp_max, int K_max, int trow) {
    return trow > 0 && K_max < 65536 && kz_smem_ahk_tc(J, m_elems, Ntp_max, K_max, trow) <= kSmemLimit;
}

int tc_width(int J, int Ntp, int Ntp_max, int K_max) {
    for (int W = J; W >= 4; W /= 2)
        if (kz_smem_ahk_tc(J, W * (Ntp + KZ_TC_PAD), Ntp_max, K_max) <= kSmemLimit) return W;
    return 0;
}

cudaError_t batch_layout_k(kz_batch* B, int kernel, int J, int nw, int sms, cudaStream_t st) {
    // work items {instance, first column | width << 24} with a cost estimate;
    // tensor-core items narrower than J go to the second list
    std::vector<std::pair<double, int2>> work, work2;
    int m_elems = 0, m_elems2 = 0, trow1 = 0, trow2 = 0;
    double cost1 = 0.0, cost2 = 0.0;
    for (int b = 0; b < B->n; ++b) {
        int W = J;
        if (kernel == KZ_KERNEL_TC) {
            W = tc_width(J, B->Ntp_of[b], B->Ntp_max, B->K_max);
            if (W == 0) return cudaErrorInvalidValue;
        }
        const bool second = (W < J);
        if (kernel == KZ_KERNEL_TC) (second ? trow2 : trow1) = std::max(second ? trow2 : trow1, B->plans[b]->n_trow);
        for (int c = 0; c < B->nrhs; c += W) {
            // a CTA-iteration costs about the same at either width, so the
            // cost of an item is its channel's
            (second ? work2 : work).push_back({B->cost[b], make_int2(b, c | (W << 24))});
            (second ? cost2 : cost1) += B->cost[b];
        }
        (second ? m_elems2 : m_elems) = std::max(second ? m_elems2 : m_elems, W * (B->Ntp_of[b] + KZ_TC_PAD));
    }
    if (work.empty()) {  // every channel is narrower than J: one launch at that width
        work.swap(work2);
        m_elems = m_elems2;
        trow1 = trow2;
        J = 4;
        cost1 = cost2;
        cost2 = 0.0;
    }
    auto sorted_items = [](std::vector<std::pair<double, int2>>& w) {
        std::stable_sort(w.begin(), w.end(), [](const auto& x, const auto& y) { return x.first > y.first; });
        std::vector<int2> out(w.size());
        for (size_t i = 0; i < w.size(); ++i) out[i] = w[i].second;
        return out;
    };
    std::vector<int2> witems = sorted_items(work), witems2 = sorted_items(work2);
    if (B->d_items) cudaFree(B->d_items);
    B->d_items = nullptr;
    if (B->d_items2) cudaFree(B->d_items2);
    B->d_items2 = nullptr;
    B->n_items2 = 0;
    cudaError_t e = upload(&B->d_items, witems, st);
    if (e != cudaSuccess) return e;
    if (!witems2.empty()) {
        e = upload(&B->d_items2, witems2, st);
        if (e == cudaSuccess && !B->aux) e = cudaStreamCreateWithFlags(&B->aux, cudaStreamNonBlocking);
        if (e == cudaSuccess && !B->ev_fork) e = cudaEventCreateWithFlags(&B->ev_fork, cudaEventDisableTiming);
        if (e == cudaSuccess && !B->ev_join) e = cudaEventCreateWithFlags(&B->ev_join, cudaEventDisableTiming);
        if (e != cudaSuccess) return e;
        B->n_items2 = (int)witems2.size();
        B->m_elems2 = m_elems2;
        B->trow_max2 = tc_stage_ok(4, m_elems2, B->Ntp_max, B->K_max, trow2) ? trow2 : 0;
        B->smem2 = kz_smem_ahk_tc(4, m_elems2, B->Ntp_max, B->K_max, B->trow_max2);
    }
    B->J = J;
    B->nw = nw;
    B->kernel = kernel;
    B->n_items = (int)witems.size();
    int occ = 1;
    if (kernel == KZ_KERNEL_TC) {
        B->m_elems = m_elems;
        B->trow_max = tc_stage_ok(J, m_elems, B->Ntp_max, B->K_max, trow1) ? trow1 : 0;
        B->smem = kz_smem_ahk_tc(J, m_elems, B->Ntp_max, B->K_max, B->trow_max);
        occ = std::max(1, kz_occupancy_ahk_tc(J, nw, B->smem));
    } else {
        B->smem = smem_for(B->algo, J, B->Ntp_max, B->K_max, B->prec);
        occ = std::max(1, occupancy_for(B->algo, J, nw, B->smem, B->prec));
    }
    B->grid = std::min(B->n_items, sms * occ);
    if (B->n_items2) {
        // both launches get the whole GPU: the narrow one (the widest channels,
        // the longest items) is issued first and holds every SM; CTAs of the
        // second start on the SMs it releases, so its work fills the first's tail
        const int occ2 = std::max(1, kz_occupancy_ahk_tc(4, nw, B->smem2));
        B->grid2 = std::min(B->n_items2, sms * occ2);
    }
    (void)cost1;
    (void)cost2;
    return cudaSuccess;
}

bool tc_ok(kz_algo a, kz_prec p) { return is_ahk_family(a) && p == KZ_C64; }

kz_status check_launch(cudaError_t e, const char* what) {
    if (e != cudaSuccess) {
        kz_set_error("%s: %s", what, cudaGetErrorString(e));
        return KZ_ERR_CUDA;
    }
    return KZ_OK;
}

KzGrpChan grp_chan(const kz_plan* P) {
    const GrpPlan& G = P->grp;
    KzGrpChan C;
    memset(&C, 0, sizeof(C));
    C.K = P->K;
    C.Nt = P->Nt;
    C.AB = G.AB;
    C.n_slots = G.n_slots;
    C.slot_row = G.d_slot;
    C.blk_nrt = G.d_nrt;
    C.blk_nb = G.d_nb;
    C.blk_coff = G.d_coff;
    C.blk_toff = G.d_toff;
    C.tiles = G.d_tiles;
    C.cptr = G.d_cptr;
    C.cidx = G.d_cidx;
    C.nrm = P->d_nrm;
    C.inF = G.d_inF;
    C.xptr = P->d_xptr;
    C.xidx = P->d_xidx;
    C.G = P->d_G;
    C.Hc = P->d_Hc;
    C.rows = P->d_rows;
    C.rptr = P->d_rptr;
    C.stat = G.d_stat;
    return C;
}

// The group kernel's set-up for operand format fmt (0 FP16, 1 BF16): rows per
// 128-antenna block from the VRs, tile images filled on `st`.
kz_status build_grp(kz_plan* P, int fmt, cudaStream_t st) {
    GrpPlan& G = P->grp;
    if (G.built && G.fmt == fmt) return KZ_OK;
    const int K = P->K, AB = (P->Nt + 127) / 128;
    std::vector<int> nb(AB, 0);
    for (int k = 0; k < K; ++k)
        for (int b = P->vr_off[k] / 128; b <= (P->vr_off[k] + P->vr_len[k] - 1) / 128; ++b) ++nb[b];
    for (int b = 0; b < AB; ++b)
        if (nb[b] > 256) {
            kz_set_error("group kernel: antennas [%d, %d) are seen by %d users (at most 256 per 128-antenna block)",
                         128 * b, 128 * b + 128, nb[b]);
            return KZ_ERR_UNSUPPORTED;
        }
    std::vector<int> nrt(AB), coff(AB), cnt(AB, 0), slot((size_t)AB * 256, -1), cptr(K + 1, 0), cidx;
    std::vector<long long> toff(AB);
    int rtmax = 1, n_slots = 0;
    long long bytes = 0;
    for (int b = 0; b < AB; ++b) {
        nrt[b] = std::max(1, (nb[b] + 127) / 128);
        rtmax = std::max(rtmax, nrt[b]);
        coff[b] = n_slots;
        n_slots += nb[b];
        toff[b] = bytes;
        bytes += 2LL * 128 * nrt[b] * 256;
    }
    for (int k = 0; k < K; ++k) {
        for (int b = P->vr_off[k] / 128; b <= (P->vr_off[k] + P->vr_len[k] - 1) / 128; ++b) {
            slot[(size_t)b * 256 + cnt[b]] = k;
            cidx.push_back(coff[b] + cnt[b]);
            ++cnt[b];
        }
        cptr[k + 1] = (int)cidx.size();
    }
    std::vector<unsigned char> inF(K, 0);
    for (int k : P->F) inF[k] = 1;
    G.release();
    cudaError_t e = cudaSuccess;
#define GRP_TRY(x)              \
    do {                        \
        e = (x);                \
        if (e != cudaSuccess) { \
            G.release();        \
            return check_launch(e, "group kernel set-up"); \
        }                       \
    } while (0)
    GRP_TRY(upload(&G.d_slot, slot, st));
    GRP_TRY(upload(&G.d_nrt, nrt, st));
    GRP_TRY(upload(&G.d_nb, nb, st));
    GRP_TRY(upload(&G.d_coff, coff, st));
    GRP_TRY(upload(&G.d_toff, toff, st));
    GRP_TRY(upload(&G.d_cptr, cptr, st));
    GRP_TRY(upload(&G.d_cidx, cidx, st));
    GRP_TRY(upload(&G.d_inF, inF, st));
    GRP_TRY(cudaMalloc((void**)&G.d_tiles, (size_t)bytes));
    GRP_TRY(cudaMalloc((void**)&G.d_stat, 2 * sizeof(float)));
    G.AB = AB;
    G.rtmax = rtmax;
    G.n_slots = n_slots;
    G.fmt = fmt;
    GRP_TRY(kz_grp_prepare(grp_chan(P), P->d_Hc, P->total2, P->d_rows, P->d_rptr, P->d_nrm, G.d_stat, fmt, st));
    GRP_TRY(cudaStreamSynchronize(st));  // the host vectors above are released on return
#undef GRP_TRY
    G.built = true;
    return KZ_OK;
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// One group-kernel solve (possibly several launches over column chunks).
kz_status run_grp(kz_plan* P, const kz_cf32* s, int nrhs, float xi, kz_algo algo, double tol, int max_iter,
                  kz_cf32* x, kz_cf32* v, int32_t* iters, double* resid, int32_t* status, int rhs_per_cta,
                  int refresh, cudaStream_t st) {
    const int fmt = (P->prec == KZ_BF16_MIXED) ? 1 : 0;
    kz_status rc = build_grp(P, fmt, st);
    if (rc != KZ_OK) return rc;
    GrpPlan& G = P->grp;
    const int AB = G.AB, sms = P->sms;
    const bool cluster = AB <= 16;
    const int rpc = (P->K + AB - 1) / AB;
    const size_t smem_limit = 227 * 1024 - 16 * 1024;  // the kernel's static shared memory is below 16 KiB
    int NC = 0;
    for (int nc : {16, 32, 64}) {
        if (rhs_per_cta && nc != rhs_per_cta) continue;
        if ((G.rtmax + 2) * 2 * nc > 512 || kz_grp_smem(nc, G.rtmax, rpc, AB) > smem_limit) continue;
        NC = nc;
        if (rhs_per_cta || (long)AB * ((nrhs + nc - 1) / nc) <= sms) break;  // smallest width that fills the GPU once
    }
    if (NC == 0) {
        kz_set_error("group kernel: %s", rhs_per_cta ? "rhs_per_cta must be 0, 16, 32 or 64 and fit" :
                                                       "the channel's tiles do not fit shared memory");
        return rhs_per_cta ? KZ_ERR_INVALID_ARG : KZ_ERR_UNSUPPORTED;
    }
    int tcols = 32;
    while (tcols < (G.rtmax + 2) * 2 * NC) tcols *= 2;
    // A CTA that holds more than half of the SM's 512 tensor-memory columns
    // must never share its SM (a second CTA's allocation would wait for the
    // first, which may wait for it at a group barrier): its shared memory is
    // padded past half of the SM's 228 KiB.
    const size_t smem = std::max(kz_grp_smem(NC, G.rtmax, rpc, AB), tcols > 256 ? (size_t)120 * 1024 : (size_t)0);
    const int CG_all = (nrhs + NC - 1) / NC;
    const int CG = cluster ? CG_all : std::min(CG_all, sms / AB);
    if (CG < 1 || !kz_grp_fits(AB, cluster ? 1 : CG, cluster, smem)) {
        kz_set_error("group kernel: %d blocks of 128 antennas cannot be resident at once", AB);
        return KZ_ERR_UNSUPPORTED;
    }
    // scratch
    const size_t b_pp = align256((size_t)CG * G.n_slots * NC * sizeof(float2));
    const size_t b_phi = align256((size_t)CG * P->K * 2 * NC * sizeof(uint16_t));
    const size_t b_q = align256((size_t)CG * P->K * NC * sizeof(float2));
    const size_t b_cp = align256((size_t)CG * 7 * AB * NC * sizeof(float));
    const size_t b_bar = align256((size_t)(2 * CG) * sizeof(unsigned));
    const size_t need = b_pp + b_phi + b_q + b_cp + b_bar;
    if (G.scr_bytes < need) {
        if (G.d_scr) cudaFree(G.d_scr);
        G.d_scr = nullptr;
        G.scr_bytes = 0;
        cudaError_t e = cudaMalloc(&G.d_scr, need);
        if (e != cudaSuccess) {
            kz_set_error("group kernel scratch: %s", cudaGetErrorString(e));
            return KZ_ERR_NOMEM;
        }
        G.scr_bytes = need;
    }
    uint8_t* base = static_cast<uint8_t*>(G.d_scr);
    KzGrpLaunch L;
    memset(&L, 0, sizeof(L));
    L.C = grp_chan(P);
    L.xi = xi;
    L.NC = NC;
    L.algo = algo;
    L.fmt = fmt;
    L.tol = tol;
    L.max_iter = max_iter;
    L.refresh = refresh ? refresh : 16;  // swept on configs 2 and 4: 8 -> 16 saves 4-6%, iterations +2%
    L.status = status;
    L.Ppart = reinterpret_cast<float2*>(base);
    L.Phi = reinterpret_cast<uint16_t*>(base + b_pp);
    L.Qg = reinterpret_cast<float2*>(base + b_pp + b_phi);
    L.colpart = reinterpret_cast<float*>(base + b_pp + b_phi + b_q);
    L.gbar = reinterpret_cast<unsigned*>(base + b_pp + b_phi + b_q + b_cp);
    L.rpc = rpc;
    L.rtmax = G.rtmax;
    L.tmem_cols = tcols;
    // column chunks of CG groups, one launch each
    for (int c0 = 0; c0 < nrhs; c0 += CG * NC) {
        const int n = std::min(nrhs - c0, CG * NC);
        L.nrhs = n;
        L.CG = (n + NC - 1) / NC;
        L.s = reinterpret_cast<const float2*>(s) + (size_t)c0 * P->K;
        L.x = reinterpret_cast<float2*>(x) + (size_t)c0 * P->Nt;
        L.v = v ? reinterpret_cast<float2*>(v) + (size_t)c0 * P->K : nullptr;
        L.iters = iters + c0;
        L.resid = resid + c0;
        cudaError_t e = cudaMemsetAsync(L.gbar, 0, (size_t)L.CG * sizeof(unsigned), st);
        if (e == cudaSuccess) e = cudaMemsetAsync(L.gbar + L.CG, 0xff, (size_t)L.CG * sizeof(unsigned), st);
        if (e == cudaSuccess) e = kz_launch_grp(L, cluster, smem, st);
        if (e != cudaSuccess) return check_launch(e, "group kernel launch");
    }
    return KZ_OK;
}

}  // namespace

extern "C" {

const char* kz_last_error(void) { return g_err.c_str(); }

int32_t kz_version(void) { return 1 * 10000 + 0 * 100 + 0; }

}  // extern "C"

// Step A0 for kz_plan_create (H given packed) and kz_plan_dense (H given as a
// dense K x Nt matrix): exactly one of H_packed / H_dense is non-NULL.
static kz_status plan_build(const char* fn, kz_plan** out, int32_t K, int32_t Nt, const int32_t* vr_offset,
                            const int32_t* vr_len, const kz_cf32* H_packed, const kz_cf32* H_dense, kz_prec prec,
                            void* stream) {
    g_err.clear();
    if (!out) {
        kz_set_error("%s: out is NULL", fn);
        return KZ_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (K < 1 || Nt < 2 || K >= Nt) {
        kz_set_error("%s: need 1 <= K < Nt (got K=%d, Nt=%d)", fn, K, Nt);
        return KZ_ERR_INVALID_ARG;
    }
    const kz_cf32* Hin = H_packed ? H_packed : H_dense;
    if (!vr_offset || !vr_len || !Hin) {
        kz_set_error("%s: NULL vr_offset, vr_len or H", fn);
        return KZ_ERR_INVALID_ARG;
    }
    if (!aligned(Hin, 8)) {
        kz_set_error("%s: H must be 8-byte aligned", fn);
        return KZ_ERR_INVALID_ARG;
    }
    if (prec != KZ_C64 && prec != KZ_BF16_MIXED) {
        kz_set_error("%s: unknown precision %d", fn, (int)prec);
        return KZ_ERR_INVALID_ARG;
    }
    for (int k = 0; k < K; ++k) {
        const long o = vr_offset[k], L = vr_len[k];
        if (L < 1 || o < 0 || o + L > Nt) {
            kz_set_error("%s: VR of user %d is [%ld, %ld), outside [0, %d) or empty", fn, k, o, o + L, Nt);
            return KZ_ERR_INVALID_ARG;
        }
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    kz_plan* P = new kz_plan();
    P->K = K;
    P->Nt = Nt;
    P->prec = prec;
    P->sms = sm_count();
    P->Ntp = ((Nt + (Nt & 1)) + KZ_TILE - 1) / KZ_TILE * KZ_TILE;
    P->ntiles = P->Ntp / KZ_TILE;

    // aligned rows: intervals on multiples of four antennas (one 16-byte load
    // of the FP16 copy is inside a row or outside it), zero-filled outside the VR
    std::vector<int4> rows(K);
    std::vector<int> rptr(K), in_off(K);
    int64_t acc = 0, acc_in = 0;
    for (int k = 0; k < K; ++k) {
        const int o = vr_offset[k], e = vr_offset[k] + vr_len[k];
        const int a = o & ~3, b = (e + 3) & ~3;
        rows[k] = make_int4(a, b - a, o, e);
        rptr[k] = (int)acc;
        in_off[k] = (int)acc_in;
        acc += b - a;
        acc_in += vr_len[k];
    }
    if (acc >= (int64_t)1 << 31) {
        delete P;
        kz_set_error("%s: channel too large (%lld aligned entries)", fn, (long long)acc);
        return KZ_ERR_UNSUPPORTED;
    }
    P->total2 = acc;
    P->sumL = acc_in;
    P->vr_off.assign(vr_offset, vr_offset + K);
    P->vr_len.assign(vr_len, vr_len + K);

    // orthogonal set F: earliest-end greedy on the VR intervals (exact maximum
    // independent set of an interval graph); ties: later start, then lower index.
    std::vector<int> idx(K);
    std::iota(idx.begin(), idx.end(), 0);
    std::sort(idx.begin(), idx.end(), [&](int x, int y) {
        const int ex = vr_offset[x] + vr_len[x], ey = vr_offset[y] + vr_len[y];
        if (ex != ey) return ex < ey;
        if (vr_offset[x] != vr_offset[y]) return vr_offset[x] > vr_offset[y];
        return x < y;
    });
    std::vector<char> inF(K, 0);
    long last_end = -1;
    for (int k : idx) {
        if (last_end < 0 || vr_offset[k] >= last_end) {
            inF[k] = 1;
            last_end = vr_offset[k] + vr_len[k];
        }
    }
    for (int k = 0; k < K; ++k)
        if (inF[k]) P->F.push_back(k);
    P->nF = (int)P->F.size();
    // solve order: F rows then V rows, each by decreasing VR length (balances
    // the round-robin assignment of rows to warps)
    std::vector<int> order;
    std::vector<int> Vrows;
    for (int k = 0; k < K; ++k)
        if (!inF[k]) Vrows.push_back(k);
    auto by_len = [&](int x, int y) { return vr_len[x] != vr_len[y] ? vr_len[x] > vr_len[y] : x < y; };
    order = P->F;
    std::sort(order.begin(), order.end(), by_len);
    std::sort(Vrows.begin(), Vrows.end(), by_len);
    order.insert(order.end(), Vrows.begin(), Vrows.end());
    // V rows, then all rows, each by the centre of the aligned interval (the
    // tensor-core residual takes rows in blocks of 8 consecutive entries, whose
    // union interval is then short)
    auto by_centre = [&](int x, int y) {
        const long cx = 2L * rows[x].x + rows[x].y, cy = 2L * rows[y].x + rows[y].y;
        return cx != cy ? cx < cy : x < y;
    };
    std::vector<int> vsort(Vrows), all(K);
    std::iota(all.begin(), all.end(), 0);
    std::sort(vsort.begin(), vsort.end(), by_centre);
    std::sort(all.begin(), all.end(), by_centre);
    vsort.insert(vsort.end(), all.begin(), all.end());

    // X_k: users whose VR overlaps user k's (k included), via a sweep over starts
    std::vector<int> by_start(K);
    std::iota(by_start.begin(), by_start.end(), 0);
    std::sort(by_start.begin(), by_start.end(), [&](int x, int y) { return vr_offset[x] < vr_offset[y]; });
    std::vector<std::vector<int>> X(K);
    for (int k = 0; k < K; ++k) X[k].push_back(k);
    for (int ii = 0; ii < K; ++ii) {
        const int x = by_start[ii];
        const long ex = (long)vr_offset[x] + vr_len[x];
        for (int jj = ii + 1; jj < K; ++jj) {
            const int y = by_start[jj];
            if (vr_offset[y] >= ex) break;
            X[x].push_back(y);
            X[y].push_back(x);
        }
    }
    P->xptr.assign(K + 1, 0);
    for (int k = 0; k < K; ++k) {
        std::sort(X[k].begin(), X[k].end());
        P->xptr[k + 1] = P->xptr[k] + (int)X[k].size();
    }
    P->xidx.reserve(P->xptr[K]);
    for (int k = 0; k < K; ++k) P->xidx.insert(P->xidx.end(), X[k].begin(), X[k].end());

    // covering lists per 64-antenna tile (aligned intervals), V rows first
    std::vector<std::vector<int>> tv(P->ntiles), tf(P->ntiles);
    for (int k = 0; k < K; ++k) {
        const int a = rows[k].x, b = rows[k].x + rows[k].y;
        for (int t = a / KZ_TILE; t <= (b - 1) / KZ_TILE; ++t) (inF[k] ? tf[t] : tv[t]).push_back(k);
    }
    std::vector<int> tptr(P->ntiles + 1, 0), tnv(P->ntiles, 0);
    std::vector<int4> trow4;
    for (int t = 0; t < P->ntiles; ++t) {
        tnv[t] = (int)tv[t].size();
        P->cmax = std::max(P->cmax, (int)(tv[t].size() + tf[t].size()));
        for (int pass = 0; pass < 2; ++pass)
            for (int k : (pass == 0 ? tv[t] : tf[t])) trow4.push_back(make_int4(k, rptr[k] - rows[k].x, rows[k].x, rows[k].x + rows[k].y));
        tptr[t + 1] = (int)trow4.size();
    }
    P->n_trow = (int)trow4.size();

    cudaError_t e = cudaSuccess;
#define KZ_TRY(x)                                            \
    do {                                                     \
        e = (x);                                             \
        if (e != cudaSuccess) {                              \
            kz_set_error("%s: %s", fn, cudaGetErrorString(e)); \
            delete P;                                        \
            return e == cudaErrorMemoryAllocation ? KZ_ERR_NOMEM : KZ_ERR_CUDA; \
        }                                                    \
    } while (0)
    KZ_TRY(upload(&P->d_rows, rows, st));
    KZ_TRY(upload(&P->d_rptr, rptr, st));
    KZ_TRY(upload(&P->d_in_off, in_off, st));
    KZ_TRY(upload(&P->d_order, order, st));
    KZ_TRY(upload(&P->d_xptr, P->xptr, st));
    KZ_TRY(upload(&P->d_xidx, P->xidx, st));
    KZ_TRY(upload(&P->d_tptr, tptr, st));
    KZ_TRY(upload(&P->d_tnv, tnv, st));
    KZ_TRY(upload(&P->d_trow4, trow4, st));
    KZ_TRY(upload(&P->d_vsort, vsort, st));
    KZ_TRY(cudaMalloc((void**)&P->d_Hc, std::max<int64_t>(acc, 2) * sizeof(float2)));
    if (prec == KZ_BF16_MIXED) KZ_TRY(cudaMalloc((void**)&P->d_Hb, std::max<int64_t>(acc, 2) * sizeof(__nv_bfloat162)));
    if (prec == KZ_C64) {
        KZ_TRY(cudaMalloc((void**)&P->d_Hh, std::max<int64_t>(acc, 4) * sizeof(__half2)));
        KZ_TRY(cudaMalloc((void**)&P->d_hs, K * sizeof(float)));
    }
    KZ_TRY(cudaMalloc((void**)&P->d_nrm, K * sizeof(float)));
    KZ_TRY(cudaMalloc((void**)&P->d_nrmd, K * sizeof(double)));
    if (H_packed)
        KZ_TRY(kz_pack_rows(reinterpret_cast<const float2*>(H_packed), P->d_in_off, P->d_rows, P->d_rptr, K, acc,
                            P->d_Hc, P->d_Hb, st));
    else
        KZ_TRY(kz_pack_dense(reinterpret_cast<const float2*>(H_dense), Nt, P->d_rows, P->d_rptr, K, P->d_Hc, P->d_Hb,
                             st));
    KZ_TRY(kz_row_norms(P->d_Hc, P->d_rows, P->d_rptr, K, P->d_nrmd, P->d_nrm, P->d_Hh, P->d_hs, st));
    KZ_TRY(cudaMalloc((void**)&P->d_G, std::max<size_t>(P->xidx.size(), 1) * sizeof(float2)));
    KZ_TRY(kz_gram(P->d_Hc, P->d_rows, P->d_rptr, P->d_xptr, P->d_xidx, K, P->d_G, st));
    KZ_TRY(cudaStreamSynchronize(st));
#undef KZ_TRY
    *out = P;
    return KZ_OK;
}

extern "C" {

kz_status kz_plan_create(kz_plan** out, int32_t K, int32_t Nt, const int32_t* vr_offset, const int32_t* vr_len,
                         const kz_cf32* H_packed, kz_prec prec, void* stream) {
    if (!H_packed) {
        g_err.clear();
        kz_set_error("kz_plan_create: H_packed is NULL");
        return KZ_ERR_INVALID_ARG;
    }
    return plan_build("kz_plan_create", out, K, Nt, vr_offset, vr_len, H_packed, nullptr, prec, stream);
}

kz_status kz_plan_dense(kz_plan** out, int32_t K, int32_t Nt, const int32_t* vr_offset, const int32_t* vr_len,
                        const kz_cf32* H_dense, kz_prec prec, void* stream) {
    if (!H_dense) {
        g_err.clear();
        kz_set_error("kz_plan_dense: H_dense is NULL");
        return KZ_ERR_INVALID_ARG;
    }
    if ((int64_t)K * Nt >= ((int64_t)1 << 40)) {
        g_err.clear();
        kz_set_error("kz_plan_dense: K x Nt too large");
        return KZ_ERR_UNSUPPORTED;
    }
    return plan_build("kz_plan_dense", out, K, Nt, vr_offset, vr_len, nullptr, H_dense, prec, stream);
}

kz_status kz_plan_update(kz_plan* P, const kz_cf32* H_packed, void* stream) {
    g_err.clear();
    if (!P || !H_packed || !aligned(H_packed, 8)) {
        kz_set_error("kz_plan_update: need a plan and an 8-byte aligned H_packed");
        return KZ_ERR_INVALID_ARG;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = kz_pack_rows(reinterpret_cast<const float2*>(H_packed), P->d_in_off, P->d_rows, P->d_rptr, P->K,
                                 P->total2, P->d_Hc, P->d_Hb, st);
    if (e == cudaSuccess)
        e = kz_row_norms(P->d_Hc, P->d_rows, P->d_rptr, P->K, P->d_nrmd, P->d_nrm, P->d_Hh, P->d_hs, st);
    if (e == cudaSuccess) e = kz_gram(P->d_Hc, P->d_rows, P->d_rptr, P->d_xptr, P->d_xidx, P->K, P->d_G, st);
    if (e == cudaSuccess && P->grp.built)
        e = kz_grp_prepare(grp_chan(P), P->d_Hc, P->total2, P->d_rows, P->d_rptr, P->d_nrm, P->grp.d_stat, P->grp.fmt, st);
    return check_launch(e, "kz_plan_update");
}

void kz_plan_destroy(kz_plan* plan) { delete plan; }

kz_status kz_plan_query(const kz_plan* P, int32_t* K, int32_t* Nt, int64_t* sum_len, int32_t* nF, int32_t* F,
                        int32_t* X_ptr, int32_t* X_idx) {
    g_err.clear();
    if (!P) {
        kz_set_error("kz_plan_query: plan is NULL");
        return KZ_ERR_INVALID_ARG;
    }
    if (K) *K = P->K;
    if (Nt) *Nt = P->Nt;
    if (sum_len) *sum_len = P->sumL;
    if (nF) *nF = P->nF;
    if (F) std::copy(P->F.begin(), P->F.end(), F);
    if (X_ptr) std::copy(P->xptr.begin(), P->xptr.end(), X_ptr);
    if (X_idx) std::copy(P->xidx.begin(), P->xidx.end(), X_idx);
    return KZ_OK;
}

static kz_status check_solve_args(const char* fn, const kz_plan* plan, int nrhs, float xi, int algo, int sel,
                                  double tol, int max_iter, int J, int refresh) {
    if (!plan) {
        kz_set_error("%s: plan is NULL", fn);
        return KZ_ERR_INVALID_ARG;
    }
    if (nrhs < 1) {
        kz_set_error("%s: nrhs must be >= 1", fn);
        return KZ_ERR_INVALID_ARG;
    }
    if (!(xi > 0.f) || !std::isfinite(xi)) {
        kz_set_error("%s: xi must be positive and finite", fn);
        return KZ_ERR_INVALID_ARG;
    }
    if (!valid_algo(algo)) {
        kz_set_error("%s: unknown algorithm %d", fn, algo);
        return KZ_ERR_INVALID_ARG;
    }
    if (sel < KZ_SEL_PAPER || sel > KZ_SEL_ARGMAX) {
        kz_set_error("%s: unknown selection rule %d", fn, sel);
        return KZ_ERR_INVALID_ARG;
    }
    if (!(tol >= 0.0) || max_iter < 1) {
        kz_set_error("%s: need tol >= 0 and max_iter >= 1", fn);
        return KZ_ERR_INVALID_ARG;
    }
    if (J != 0 && J != 1 && J != 2 && J != 4 && J != 8) {
        kz_set_error("%s: rhs_per_cta must be 0, 1, 2, 4 or 8", fn);
        return KZ_ERR_INVALID_ARG;
    }
    if (refresh < 0) {
        kz_set_error("%s: refresh must be >= 0", fn);
        return KZ_ERR_INVALID_ARG;
    }
    return KZ_OK;
}

kz_status kz_precode(kz_plan* plan, const kz_cf32* s, int32_t nrhs, float xi, kz_algo algo, kz_select sel,
                     double tol, int32_t max_iter, uint64_t seed, kz_cf32* x, kz_cf32* v, int32_t* iters,
                     double* resid, int32_t* status, int32_t rhs_per_cta, int32_t refresh, void* stream) {
    return kz_precode_ex(plan, s, nrhs, xi, algo, sel, tol, max_iter, seed, x, v, iters, resid, status,
                         KZ_KERNEL_AUTO, rhs_per_cta, refresh, stream);
}

}  // extern "C"

// kz_precode_ex, optionally recording the selected-row history of a row-action
// method (hist_row / hist_gam: T x nrhs, step t of column c at t * nrhs + c).
static kz_status precode_impl(kz_plan* plan, const kz_cf32* s, int32_t nrhs, float xi, kz_algo algo, kz_select sel,
                              double tol, int32_t max_iter, uint64_t seed, kz_cf32* x, kz_cf32* v, int32_t* iters,
                              double* resid, int32_t* status, kz_kernel kernel, int32_t rhs_per_cta, int32_t refresh,
                              void* stream, int32_t* hist_row, kz_cf32* hist_gam, int32_t hist_T) {
    g_err.clear();
    if (kernel == KZ_KERNEL_TC) {
        if (rhs_per_cta != 0 && rhs_per_cta != 4 && rhs_per_cta != 8) {
            kz_set_error("kz_precode_ex: the tensor-core kernel takes 0, 4 or 8 columns per CTA");
            return KZ_ERR_INVALID_ARG;
        }
    } else if (kernel == KZ_KERNEL_SMALL) {
        if (rhs_per_cta != 0 && rhs_per_cta != 1) {
            kz_set_error("kz_precode_ex: the small-channel kernel takes 0 or 1 column per CTA");
            return KZ_ERR_INVALID_ARG;
        }
    } else if (kernel == KZ_KERNEL_GROUP) {
        if (rhs_per_cta != 0 && rhs_per_cta != 16 && rhs_per_cta != 32 && rhs_per_cta != 64) {
            kz_set_error("kz_precode_ex: the group kernel takes 0, 16, 32 or 64 columns per group");
            return KZ_ERR_INVALID_ARG;
        }
    } else if (kernel != KZ_KERNEL_AUTO && kernel != KZ_KERNEL_RESIDENT) {
        kz_set_error("kz_precode_ex: unknown kernel %d", (int)kernel);
        return KZ_ERR_INVALID_ARG;
    }
    kz_status rc = check_solve_args("kz_precode", plan, nrhs, xi, algo, sel, tol, max_iter,
                                    (kernel == KZ_KERNEL_TC || kernel == KZ_KERNEL_GROUP || kernel == KZ_KERNEL_SMALL)
                                        ? 0
                                        : rhs_per_cta,
                                    refresh);
    if (rc != KZ_OK) return rc;
    if (!s || !x || !iters || !resid) {
        kz_set_error("kz_precode: s, x, iters and resid are required");
        return KZ_ERR_INVALID_ARG;
    }
    if (!aligned(s, 8) || !aligned(x, 8) || (v && !aligned(v, 8)) || !aligned(resid, 8) || !aligned(iters, 4)) {
        kz_set_error("kz_precode: misaligned output or input pointer");
        return KZ_ERR_INVALID_ARG;
    }
    if (algo == KZ_GK) {  // GK is GRK with the maximal-residual rule
        algo = KZ_GRK;
        sel = KZ_SEL_ARGMAX;
    }
    const kz_prec prec = plan->prec;
    const bool bf = (prec == KZ_BF16_MIXED);
    if (bf && !is_ahk_family(algo)) {
        kz_set_error("kz_precode: BF16_MIXED is provided for AHK and VR_OAHK only");
        return KZ_ERR_UNSUPPORTED;
    }
    if (kernel == KZ_KERNEL_TC && !tc_ok(algo, prec)) {
        kz_set_error("kz_precode_ex: the tensor-core kernel runs AHK / VR_OAHK on C64 plans");
        return KZ_ERR_UNSUPPORTED;
    }
    // AUTO on a small channel with at most one column per SM and no fixed
    // column count per CTA: the small-channel kernel (3-4x less time per
    // iteration than RESIDENT on 16 users and 256 antennas)
    if (kernel == KZ_KERNEL_AUTO && rhs_per_cta == 0 && prec == KZ_C64 && plan->K <= 32 && plan->Ntp <= 512 &&
        !hist_row && nrhs <= plan->sms && kz_smem_small(plan->K, plan->Ntp) <= kSmemLimit)
        kernel = KZ_KERNEL_SMALL;
    if (kernel == KZ_KERNEL_SMALL) {
        if (prec != KZ_C64 || plan->K > 32 || plan->Ntp > 512 || hist_row) {
            kz_set_error("kz_precode_ex: the small-channel kernel needs a C64 plan with K <= 32 and Nt <= 511");
            return KZ_ERR_UNSUPPORTED;
        }
        const size_t smem = kz_smem_small(plan->K, plan->Ntp);
        if (smem > kSmemLimit) {
            kz_set_error("kz_precode_ex: the channel does not fit the small-channel kernel's shared memory");
            return KZ_ERR_UNSUPPORTED;
        }
        KzLaunch L;
        memset(&L, 0, sizeof(L));
        L.single = plan->inst();
        L.single.xi = xi;
        L.single.ld = nrhs;
        L.single.s = reinterpret_cast<const float2*>(s);
        L.single.x = reinterpret_cast<float2*>(x);
        L.single.v = reinterpret_cast<float2*>(v);
        L.single.iters = iters;
        L.single.resid = resid;
        L.algo = algo;
        L.sel = sel;
        L.prec = prec;
        L.tol = tol;
        L.max_iter = max_iter;
        L.refresh = refresh ? refresh : default_refresh(algo, prec);
        L.seed = seed;
        L.status = status;
        return check_launch(kz_launch_small(L, nrhs, smem, static_cast<cudaStream_t>(stream)),
                            "kz_precode small-channel kernel");
    }
    // AUTO on a large channel (4096 antennas or more) for AHK / VR-OAHK: the
    // group kernel (measured 1.3-11x faster than RESIDENT from 4096 to 16384
    // antennas, 16-256 columns); a channel it cannot hold falls back
    if (kernel == KZ_KERNEL_AUTO && rhs_per_cta == 0 && is_ahk_family(algo) && !hist_row && plan->Ntp >= 4096) {
        const kz_status rc = run_grp(plan, s, nrhs, xi, algo, tol, max_iter, x, v, iters, resid, status, 0, refresh,
                                     static_cast<cudaStream_t>(stream));
        if (rc != KZ_ERR_UNSUPPORTED) return rc;
        g_err.clear();
    }
    if (kernel == KZ_KERNEL_GROUP) {
        if (!is_ahk_family(algo)) {
            kz_set_error("kz_precode_ex: the group kernel runs AHK / VR_OAHK");
            return KZ_ERR_UNSUPPORTED;
        }
        return run_grp(plan, s, nrhs, xi, algo, tol, max_iter, x, v, iters, resid, status, rhs_per_cta, refresh,
                       static_cast<cudaStream_t>(stream));
    }
    int J, nw, trow_single = 0;
    size_t smem;
    if (kernel == KZ_KERNEL_TC) {
        // 8 columns per CTA only when that still gives every SM a work item
        J = rhs_per_cta ? rhs_per_cta
                        : ((nrhs + 7) / 8 >= plan->sms &&
                                   kz_smem_ahk_tc(8, 8 * (plan->Ntp + KZ_TC_PAD), plan->Ntp, plan->K) <= kSmemLimit
                               ? 8
                               : 4);
        nw = choose_nw(plan->Ntp);
        trow_single = tc_stage_ok(J, J * (plan->Ntp + KZ_TC_PAD), plan->Ntp, plan->K, plan->n_trow) ? plan->n_trow : 0;
        smem = kz_smem_ahk_tc(J, J * (plan->Ntp + KZ_TC_PAD), plan->Ntp, plan->K, trow_single);
    } else {
        J = rhs_per_cta ? rhs_per_cta : choose_J(algo, 1, plan->Ntp, plan->K, prec, plan->sms, nrhs);
        nw = choose_nw(plan->Ntp);
        smem = smem_for(algo, J, plan->Ntp, plan->K, prec);
    }
    if (smem > kSmemLimit) {
        kz_set_error("kz_precode: channel needs %zu bytes of shared memory per CTA (limit %zu); use fewer columns per CTA",
                     smem, kSmemLimit);
        return KZ_ERR_UNSUPPORTED;
    }
    KzLaunch L;
    memset(&L, 0, sizeof(L));
    L.single = plan->inst();
    L.single.xi = xi;
    L.single.ld = nrhs;
    L.single.s = reinterpret_cast<const float2*>(s);
    L.single.x = reinterpret_cast<float2*>(x);
    L.single.v = reinterpret_cast<float2*>(v);
    L.single.iters = iters;
    L.single.resid = resid;
    L.insts = nullptr;
    L.items = nullptr;
    L.n_items = (nrhs + J - 1) / J;
    L.queue = nullptr;
    L.algo = algo;
    L.sel = sel;
    L.prec = prec;
    L.tol = tol;
    L.max_iter = max_iter;
    L.refresh = refresh ? refresh : default_refresh(algo, prec, kernel == KZ_KERNEL_TC);
    L.seed = seed;
    L.status = status;
    L.Ntp_max = plan->Ntp;
    L.K_max = plan->K;
    L.hist_row = hist_row;
    L.hist_gam = reinterpret_cast<float2*>(hist_gam);
    L.hist_ld = nrhs;
    L.hist_T = hist_T;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (kernel == KZ_KERNEL_TC) {
        L.tc = 1;
        L.trow_max = trow_single;
        const int occ = std::max(1, kz_occupancy_ahk_tc(J, nw, smem));
        e = kz_launch_ahk(L, J, nw, std::min(L.n_items, plan->sms * occ), smem, st);
    } else {
        const int occ = std::max(1, occupancy_for(algo, J, nw, smem, prec));
        const int grid = std::min(L.n_items, plan->sms * occ);
        e = is_ahk_family(algo) ? kz_launch_ahk(L, J, nw, grid, smem, st) : kz_launch_kacz(L, J, nw, grid, smem, st);
    }
    return check_launch(e, "kz_precode launch");
}

extern "C" {

kz_status kz_precode_ex(kz_plan* plan, const kz_cf32* s, int32_t nrhs, float xi, kz_algo algo, kz_select sel,
                        double tol, int32_t max_iter, uint64_t seed, kz_cf32* x, kz_cf32* v, int32_t* iters,
                        double* resid, int32_t* status, kz_kernel kernel, int32_t rhs_per_cta, int32_t refresh,
                        void* stream) {
    return precode_impl(plan, s, nrhs, xi, algo, sel, tol, max_iter, seed, x, v, iters, resid, status, kernel,
                        rhs_per_cta, refresh, stream, nullptr, nullptr, 0);
}

kz_status kz_precode_record(kz_plan* plan, const kz_cf32* s, int32_t nrhs, float xi, kz_algo algo, kz_select sel,
                            int32_t T, uint64_t seed, kz_cf32* x, kz_cf32* v, int32_t* iters, double* resid,
                            int32_t* hist_row, kz_cf32* hist_gam, int32_t* status, void* stream) {
    g_err.clear();
    if (is_ahk_family(algo) || !valid_algo(algo)) {
        kz_set_error("kz_precode_record: records the row-action methods (RK, GRK, GK, VR_OGRK, SWOR-ERK)");
        return KZ_ERR_UNSUPPORTED;
    }
    if (T < 1 || !hist_row || !hist_gam || !v || !aligned(hist_gam, 8) || !aligned(hist_row, 4)) {
        kz_set_error("kz_precode_record: need T >= 1, v and the history buffers");
        return KZ_ERR_INVALID_ARG;
    }
    if (plan && plan->prec != KZ_C64) {
        kz_set_error("kz_precode_record: needs a C64 plan");
        return KZ_ERR_UNSUPPORTED;
    }
    // refresh T + 1: m is never rebuilt from q inside the T steps
    return precode_impl(plan, s, nrhs, xi, algo, sel, 0.0, T, seed, x, v, iters, resid, status, KZ_KERNEL_AUTO, 0,
                        T + 1, stream, hist_row, hist_gam, T);
}

kz_status kz_unrolled_adjoint(kz_plan* plan, int32_t nrhs, float xi, int32_t T, const int32_t* iters,
                              const int32_t* hist_row, const kz_cf32* hist_gam, const kz_cf32* x, const kz_cf32* v,
                              const kz_cf32* G_X, const kz_cf32* G_V, kz_cf32* grad_H_packed, float* grad_xi,
                              kz_cf32* grad_s, void* stream) {
    g_err.clear();
    if (!plan || nrhs < 1 || T < 1 || !(xi > 0.f) || !iters || !hist_row || !hist_gam || !x || !v || (!G_X && !G_V) ||
        !grad_H_packed || !grad_xi || !grad_s) {
        kz_set_error("kz_unrolled_adjoint: need a plan, nrhs >= 1, T >= 1, xi > 0, the history, x, v, one of "
                     "G_X / G_V and the gradient outputs");
        return KZ_ERR_INVALID_ARG;
    }
    if (kz_smem_unrolled(plan->Nt, plan->K) > kSmemLimit) {
        kz_set_error("kz_unrolled_adjoint: Nt = %d, K = %d do not fit one CTA's shared memory", plan->Nt, plan->K);
        return KZ_ERR_UNSUPPORTED;
    }
    if (!plan->d_scratch || plan->scratch_elems < 1) {  // one double for the xi gradient
        if (plan->d_scratch) cudaFree(plan->d_scratch);
        plan->d_scratch = nullptr;
        plan->scratch_elems = 0;
        cudaError_t e = cudaMalloc((void**)&plan->d_scratch, sizeof(float2));
        if (e != cudaSuccess) {
            kz_set_error("kz_unrolled_adjoint: %s", cudaGetErrorString(e));
            return KZ_ERR_NOMEM;
        }
        plan->scratch_elems = 1;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    KzInst I = plan->inst();
    I.xi = xi;
    I.ld = nrhs;
    double* acc = reinterpret_cast<double*>(plan->d_scratch);
    cudaError_t e = cudaMemsetAsync(grad_H_packed, 0, (size_t)plan->sumL * sizeof(kz_cf32), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(acc, 0, sizeof(double), st);
    if (e == cudaSuccess)
        e = kz_unrolled_adjoint(I, nrhs, T, iters, hist_row, reinterpret_cast<const float2*>(hist_gam),
                                reinterpret_cast<const float2*>(x), reinterpret_cast<const float2*>(v),
                                reinterpret_cast<const float2*>(G_X), reinterpret_cast<const float2*>(G_V),
                                reinterpret_cast<float2*>(grad_H_packed), acc, reinterpret_cast<float2*>(grad_s),
                                grad_xi, st);
    return check_launch(e, "kz_unrolled_adjoint");
}

kz_status kz_batch_prepare(kz_batch** out, const kz_batch_item* items, int32_t n, int32_t nrhs, kz_algo algo,
                           kz_prec prec, int32_t rhs_per_cta, void* stream) {
    g_err.clear();
    if (!out || !items || n < 1 || nrhs < 1) {
        kz_set_error("kz_batch_prepare: need out, items, n >= 1 and nrhs >= 1");
        return KZ_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (!valid_algo(algo) || (prec != KZ_C64 && prec != KZ_BF16_MIXED)) {
        kz_set_error("kz_batch_prepare: unknown algorithm or precision");
        return KZ_ERR_INVALID_ARG;
    }
    if (prec == KZ_BF16_MIXED && !is_ahk_family(algo)) {
        kz_set_error("kz_batch_prepare: BF16_MIXED is provided for AHK and VR_OAHK only");
        return KZ_ERR_UNSUPPORTED;
    }
    if (rhs_per_cta != 0 && rhs_per_cta != 1 && rhs_per_cta != 2 && rhs_per_cta != 4 && rhs_per_cta != 8) {
        kz_set_error("kz_batch_prepare: rhs_per_cta must be 0, 1, 2, 4 or 8");
        return KZ_ERR_INVALID_ARG;
    }
    int Ntp_max = 0, K_max = 0, cmax = 0, sms = sm_count();
    for (int b = 0; b < n; ++b) {
        const kz_batch_item& it = items[b];
        if (!it.plan || !it.s || !it.x || !it.iters || !it.resid || !(it.xi > 0.f)) {
            kz_set_error("kz_batch_prepare: item %d is missing a plan, buffer or positive xi", b);
            return KZ_ERR_INVALID_ARG;
        }
        if (!aligned(it.s, 8) || !aligned(it.x, 8) || (it.v && !aligned(it.v, 8)) || !aligned(it.resid, 8) ||
            !aligned(it.iters, 4)) {
            kz_set_error("kz_batch_prepare: item %d has a misaligned buffer", b);
            return KZ_ERR_INVALID_ARG;
        }
        if (prec == KZ_BF16_MIXED && it.plan->prec != KZ_BF16_MIXED) {
            kz_set_error("kz_batch_prepare: item %d's plan has no BF16 copy", b);
            return KZ_ERR_INVALID_ARG;
        }
        Ntp_max = std::max(Ntp_max, it.plan->Ntp);
        K_max = std::max(K_max, it.plan->K);
        cmax = std::max(cmax, it.plan->cmax);
    }
    kz_batch* B = new kz_batch();
    B->n = n;
    B->nrhs = nrhs;
    B->gk = (algo == KZ_GK);
    B->algo = B->gk ? KZ_GRK : algo;
    B->prec = prec;
    B->Ntp_max = Ntp_max;
    B->K_max = K_max;
    B->cmax = cmax;
    B->J = rhs_per_cta ? rhs_per_cta : choose_J(algo, n, Ntp_max, K_max, prec, sms, nrhs);
    B->nw = choose_nw(Ntp_max);
    B->smem = smem_for(algo, B->J, Ntp_max, K_max, prec);
    if (B->smem > kSmemLimit) {
        delete B;
        kz_set_error("kz_batch_prepare: largest channel needs %zu bytes of shared memory per CTA", smem_for(algo, rhs_per_cta ? rhs_per_cta : 1, Ntp_max, K_max, prec));
        return KZ_ERR_UNSUPPORTED;
    }
    std::vector<KzInst> insts(n);
    B->cost.resize(n);
    for (int b = 0; b < n; ++b) {
        const kz_batch_item& it = items[b];
        KzInst I = it.plan->inst();
        I.inst = b;
        I.xi = it.xi;
        I.ld = nrhs;
        I.s = reinterpret_cast<const float2*>(it.s);
        I.x = reinterpret_cast<float2*>(it.x);
        I.v = reinterpret_cast<float2*>(it.v);
        I.iters = it.iters;
        I.resid = it.resid;
        insts[b] = I;
        if (!it.v) B->all_v = false;
        B->cost[b] = (double)it.plan->total2 + 4.0 * it.plan->Ntp;
        B->plans.push_back(it.plan);
        B->Ntp_of.push_back(it.plan->Ntp);
    }
    B->h_insts = insts;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = upload(&B->d_insts, insts, st);
    // work estimate of a channel: aligned entries + 4 Nt per iteration, times
    // the expected iterations, taken as proportional to 0.036 + mu (mu the
    // largest squared off-diagonal row mass of the row-normalised system, the
    // worst-coupled user; least-squares fit of the iterations of near-field
    // channels of 1024-4096 antennas: 2.7 + 75 mu).  It only orders the queue.
    if (e == cudaSuccess) {
        float* d_mu = nullptr;
        std::vector<float> mu(n, 0.f);
        e = cudaMalloc((void**)&d_mu, n * sizeof(float));
        if (e == cudaSuccess) e = kz_coupling(B->d_insts, n, d_mu, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(mu.data(), d_mu, n * sizeof(float), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (d_mu) cudaFree(d_mu);
        if (e == cudaSuccess)
            for (int b = 0; b < n; ++b)
                if (std::isfinite(mu[b])) B->cost[b] *= 0.036 + (double)mu[b];
    }
    if (e == cudaSuccess) e = cudaMalloc((void**)&B->d_queue, 2 * sizeof(int));
    if (e == cudaSuccess) e = batch_layout(B, B->J, B->nw, sms, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        delete B;
        kz_set_error("kz_batch_prepare: %s", cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? KZ_ERR_NOMEM : KZ_ERR_CUDA;
    }
    *out = B;
    return KZ_OK;
}

kz_status kz_batch_rebind(kz_batch* B, const kz_batch_item* items, void* stream) {
    g_err.clear();
    if (!B || !items) {
        kz_set_error("kz_batch_rebind: need a batch and its items");
        return KZ_ERR_INVALID_ARG;
    }
    std::vector<KzInst> insts = B->h_insts;
    bool all_v = true;
    for (int b = 0; b < B->n; ++b) {
        const kz_batch_item& it = items[b];
        if (it.plan != B->plans[b]) {
            kz_set_error("kz_batch_rebind: item %d names another plan than at preparation", b);
            return KZ_ERR_INVALID_ARG;
        }
        if (!it.s || !it.x || !it.iters || !it.resid || !(it.xi > 0.f)) {
            kz_set_error("kz_batch_rebind: item %d is missing a buffer or positive xi", b);
            return KZ_ERR_INVALID_ARG;
        }
        if (!aligned(it.s, 8) || !aligned(it.x, 8) || (it.v && !aligned(it.v, 8)) || !aligned(it.resid, 8) ||
            !aligned(it.iters, 4)) {
            kz_set_error("kz_batch_rebind: item %d has a misaligned buffer", b);
            return KZ_ERR_INVALID_ARG;
        }
        KzInst& I = insts[b];
        I.xi = it.xi;
        I.s = reinterpret_cast<const float2*>(it.s);
        I.x = reinterpret_cast<float2*>(it.x);
        I.v = reinterpret_cast<float2*>(it.v);
        I.iters = it.iters;
        I.resid = it.resid;
        if (!it.v) all_v = false;
    }
    // pageable source: staged before return, so the host vector may go away
    cudaError_t e = cudaMemcpyAsync(B->d_insts, insts.data(), insts.size() * sizeof(KzInst), cudaMemcpyHostToDevice,
                                    static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return check_launch(e, "kz_batch_rebind");
    B->h_insts.swap(insts);
    B->all_v = all_v;
    return KZ_OK;
}

kz_status kz_precode_batched(kz_batch* B, kz_select sel, double tol, int32_t max_iter, uint64_t seed,
                             int32_t refresh, int32_t* status, void* stream) {
    g_err.clear();
    if (!B) {
        kz_set_error("kz_precode_batched: batch is NULL");
        return KZ_ERR_INVALID_ARG;
    }
    if (sel < KZ_SEL_PAPER || sel > KZ_SEL_ARGMAX || !(tol >= 0.0) || max_iter < 1 || refresh < 0) {
        kz_set_error("kz_precode_batched: bad selection rule, tol, max_iter or refresh");
        return KZ_ERR_INVALID_ARG;
    }
    if (B->gk) sel = KZ_SEL_ARGMAX;
    KzLaunch L;
    memset(&L, 0, sizeof(L));
    L.insts = B->d_insts;
    L.items = B->d_items;
    L.n_items = B->n_items;
    L.queue = B->d_queue;
    L.algo = B->algo;
    L.sel = sel;
    L.prec = B->prec;
    L.tol = tol;
    L.max_iter = max_iter;
    L.refresh = refresh ? refresh : default_refresh(B->algo, B->prec, B->kernel == KZ_KERNEL_TC);
    L.seed = seed;
    L.status = status;
    L.Ntp_max = B->Ntp_max;
    L.K_max = B->K_max;
    L.tc = (B->kernel == KZ_KERNEL_TC);
    L.m_elems = L.tc ? B->m_elems : 0;
    L.trow_max = L.tc ? B->trow_max : 0;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(B->d_queue, 0, 2 * sizeof(int), st);
    if (e != cudaSuccess) return check_launch(e, "kz_precode_batched memset");
    if (B->n_items2) {  // fork: the narrow items run on the auxiliary stream
        e = cudaEventRecord(B->ev_fork, st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(B->aux, B->ev_fork, 0);
        if (e != cudaSuccess) return check_launch(e, "kz_precode_batched fork");
    }
    if (B->n_items2) {  // the narrow items first, on the auxiliary stream
        KzLaunch L2 = L;
        L2.items = B->d_items2;
        L2.n_items = B->n_items2;
        L2.queue = B->d_queue + 1;
        L2.m_elems = B->m_elems2;
        L2.trow_max = B->trow_max2;
        e = kz_launch_ahk(L2, 4, B->nw, B->grid2, B->smem2, B->aux);
        if (e == cudaSuccess) e = cudaEventRecord(B->ev_join, B->aux);
        if (e != cudaSuccess) return check_launch(e, "kz_precode_batched second launch");
    }
    e = is_ahk_family(B->algo) ? kz_launch_ahk(L, B->J, B->nw, B->grid, B->smem, st)
                               : kz_launch_kacz(L, B->J, B->nw, B->grid, B->smem, st);
    if (e != cudaSuccess) return check_launch(e, "kz_precode_batched launch");
    if (B->n_items2) {
        e = cudaStreamWaitEvent(st, B->ev_join, 0);  // join
        if (e != cudaSuccess) return check_launch(e, "kz_precode_batched join");
    }
    return KZ_OK;
}

void kz_batch_destroy(kz_batch* batch) { delete batch; }

kz_status kz_batch_tune(kz_batch* B, kz_select sel, double tol, int32_t max_iter, uint64_t seed, int32_t* chosen,
                        void* stream) {
    g_err.clear();
    if (!B) {
        kz_set_error("kz_batch_tune: batch is NULL");
        return KZ_ERR_INVALID_ARG;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int sms = sm_count();
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        kz_set_error("kz_batch_tune: cudaEventCreate failed");
        return KZ_ERR_CUDA;
    }
    float best_ms = 1e30f;
    int best_J = B->J, best_nw = B->nw;
    kz_status rc = KZ_OK;
    int best_kernel = B->kernel;
    struct Cand {
        int kernel, J, nw;
    };
    std::vector<Cand> cands;
    for (int J : {1, 2, 4, 8}) {
        if (J > B->nrhs) continue;
        if (smem_for(B->algo, J, B->Ntp_max, B->K_max, B->prec) > kSmemLimit) continue;
        for (int nw : {8, 16}) cands.push_back({KZ_KERNEL_RESIDENT, J, nw});
    }
    if (tc_ok(B->algo, B->prec)) {
        for (int J : {4, 8}) {
            if (J == 8 && B->nrhs < 8) continue;
            if (tc_width(J, B->Ntp_max, B->Ntp_max, B->K_max) == 0) continue;  // the widest fits at >= 4
            for (int nw : {8, 16}) cands.push_back({KZ_KERNEL_TC, J, nw});
        }
    }
    for (const Cand& cd : cands) {
        const int J = cd.J, nw = cd.nw;
        {
            cudaError_t e = batch_layout_k(B, cd.kernel, J, nw, sms, st);
            if (e != cudaSuccess) {
                rc = check_launch(e, "kz_batch_tune layout");
                break;
            }
            float ms = 0.f;
            bool skip = false;
            for (int rep = 0; rep < 3 && rc == KZ_OK; ++rep) {
                if (rep == 1) cudaEventRecord(e0, st);
                rc = kz_precode_batched(B, sel, tol, max_iter, seed, 0, nullptr, stream);
                if (rc == KZ_ERR_CUDA) {  // a launch this device rejects: not a candidate
                    (void)cudaGetLastError();
                    rc = KZ_OK;
                    skip = true;
                    break;
                }
            }
            if (rc != KZ_OK) break;
            if (skip) continue;
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                rc = KZ_ERR_CUDA;
                kz_set_error("kz_batch_tune: timing failed");
                break;
            }
            if (ms < best_ms) {
                best_ms = ms;
                best_J = J;
                best_nw = nw;
                best_kernel = cd.kernel;
            }
        }
        if (rc != KZ_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != KZ_OK) return rc;
    cudaError_t e = batch_layout_k(B, best_kernel, best_J, best_nw, sms, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return check_launch(e, "kz_batch_tune");
    if (chosen) {
        chosen[0] = best_kernel;
        chosen[1] = best_J;
        chosen[2] = best_nw * 32;
    }
    return KZ_OK;
}

kz_status kz_batch_query(const kz_batch* B, int32_t* kernel, int32_t* rhs_per_cta, int32_t* threads,
                         int32_t* launches) {
    g_err.clear();
    if (!B) {
        kz_set_error("kz_batch_query: null batch");
        return KZ_ERR_INVALID_ARG;
    }
    if (kernel) *kernel = B->kernel;
    if (rhs_per_cta) *rhs_per_cta = B->J;
    if (threads) *threads = B->nw * 32;
    if (launches) *launches = B->n_items2 ? 2 : 1;
    return KZ_OK;
}

kz_status kz_batch_set_launch(kz_batch* B, kz_kernel kernel, int32_t rhs_per_cta, int32_t threads, void* stream) {
    g_err.clear();
    if (!B || (threads != 256 && threads != 512)) {
        kz_set_error("kz_batch_set_launch: need a batch and threads of 256 or 512");
        return KZ_ERR_INVALID_ARG;
    }
    const int nw = threads / 32;
    if (kernel == KZ_KERNEL_TC) {
        if (!tc_ok(B->algo, B->prec) || (rhs_per_cta != 4 && rhs_per_cta != 8) ||
            tc_width(rhs_per_cta, B->Ntp_max, B->Ntp_max, B->K_max) == 0) {
            kz_set_error("kz_batch_set_launch: the tensor-core kernel needs AHK / VR_OAHK on C64 with 4 or 8 "
                         "columns that fit shared memory");
            return KZ_ERR_UNSUPPORTED;
        }
    } else if (kernel == KZ_KERNEL_RESIDENT || kernel == KZ_KERNEL_AUTO) {
        if ((rhs_per_cta != 1 && rhs_per_cta != 2 && rhs_per_cta != 4 && rhs_per_cta != 8) ||
            smem_for(B->algo, rhs_per_cta, B->Ntp_max, B->K_max, B->prec) > kSmemLimit) {
            kz_set_error("kz_batch_set_launch: resident kernel needs 1, 2, 4 or 8 columns that fit shared memory");
            return KZ_ERR_UNSUPPORTED;
        }
        kernel = KZ_KERNEL_RESIDENT;
    } else {
        kz_set_error("kz_batch_set_launch: unknown kernel %d", (int)kernel);
        return KZ_ERR_INVALID_ARG;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = batch_layout_k(B, kernel, rhs_per_cta, nw, sm_count(), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return check_launch(e, "kz_batch_set_launch");
}

static kz_status batch_update_range(kz_batch* B, const kz_cf32* H_cat, int first, int count, void* stream,
                                    const char* fn) {
    g_err.clear();
    if (!B || !H_cat || !aligned(H_cat, 8)) {
        kz_set_error("%s: need a batch and an 8-byte aligned H_cat", fn);
        return KZ_ERR_INVALID_ARG;
    }
    if (first < 0 || count < 1 || first > B->n - count) {
        kz_set_error("%s: items [%d, %d) are not within the batch's %d items", fn, first, first + count, B->n);
        return KZ_ERR_INVALID_ARG;
    }
    for (int b = 0; b < B->n; ++b)
        for (int c = 0; c < b; ++c)
            if (B->plans[b] == B->plans[c]) {
                kz_set_error("%s: items %d and %d name the same plan", fn, c, b);
                return KZ_ERR_INVALID_ARG;
            }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    if (!B->d_rowmap) {
        std::vector<int2> rm;
        std::vector<long long> hoff(B->n);
        std::vector<int> rs(B->n + 1, 0);
        long long acc = 0;
        for (int b = 0; b < B->n; ++b) {
            hoff[b] = acc;
            acc += B->plans[b]->sumL;
            rs[b] = (int)rm.size();
            for (int k = 0; k < B->plans[b]->K; ++k) rm.push_back(make_int2(b, k));
        }
        rs[B->n] = (int)rm.size();
        e = upload(&B->d_rowmap, rm, st);
        if (e == cudaSuccess) e = upload(&B->d_hoff, hoff, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the host vectors go out of scope
        if (e != cudaSuccess) {
            if (B->d_rowmap) cudaFree(B->d_rowmap);
            if (B->d_hoff) cudaFree(B->d_hoff);
            B->d_rowmap = nullptr;
            B->d_hoff = nullptr;
            return check_launch(e, fn);
        }
        B->n_rows = (int)rm.size();
        B->row_start = rs;
    }
    const int r0 = B->row_start[first], r1 = B->row_start[first + count];
    e = kz_batch_update_rows(B->d_insts, B->d_rowmap, r0, r1 - r0, B->d_hoff, reinterpret_cast<const float2*>(H_cat),
                             st);
    if (e != cudaSuccess) return check_launch(e, fn);
    for (int b = first; b < first + count; ++b) {  // a plan that also serves the group kernel keeps its tiles current
        kz_plan* P = const_cast<kz_plan*>(B->plans[b]);
        if (P->grp.built) {
            e = kz_grp_prepare(grp_chan(P), P->d_Hc, P->total2, P->d_rows, P->d_rptr, P->d_nrm, P->grp.d_stat,
                               P->grp.fmt, st);
            if (e != cudaSuccess) return check_launch(e, fn);
        }
    }
    return KZ_OK;
}

kz_status kz_batch_update(kz_batch* B, const kz_cf32* H_cat, void* stream) {
    return batch_update_range(B, H_cat, 0, B ? B->n : 0, stream, "kz_batch_update");
}

kz_status kz_batch_update_items(kz_batch* B, const kz_cf32* H_cat, int32_t first, int32_t count, void* stream) {
    return batch_update_range(B, H_cat, first, count, stream, "kz_batch_update_items");
}

kz_status kz_precode_adjoint_batched(kz_batch* B, const kz_adjoint_item* items, double tol, int32_t max_iter,
                                     int32_t* status, void* stream) {
    g_err.clear();
    if (!B || !items) {
        kz_set_error("kz_precode_adjoint_batched: need a batch and its items");
        return KZ_ERR_INVALID_ARG;
    }
    if (B->algo != KZ_VR_OAHK || B->prec != KZ_C64 || !B->all_v) {
        kz_set_error("kz_precode_adjoint_batched: the batch must run VR_OAHK on C64 plans with a v buffer per item");
        return KZ_ERR_INVALID_ARG;
    }
    if (!(tol >= 0.0) || max_iter < 1) {
        kz_set_error("kz_precode_adjoint_batched: need tol >= 0 and max_iter >= 1");
        return KZ_ERR_INVALID_ARG;
    }
    std::vector<KzAdjItem> adj(B->n);
    for (int b = 0; b < B->n; ++b) {
        const kz_adjoint_item& it = items[b];
        if (!it.Q || !it.X || !it.grad_H_packed || !it.grad_xi || (!it.G_Q && !it.G_X)) {
            kz_set_error("kz_precode_adjoint_batched: item %d needs Q, X, grad_H_packed, grad_xi and G_Q or G_X", b);
            return KZ_ERR_INVALID_ARG;
        }
        adj[b] = KzAdjItem{reinterpret_cast<const float2*>(it.Q), reinterpret_cast<const float2*>(it.X),
                           reinterpret_cast<const float2*>(it.G_Q), reinterpret_cast<const float2*>(it.G_X),
                           reinterpret_cast<float2*>(it.grad_H_packed), it.grad_xi};
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    if (!B->d_adj) e = cudaMalloc((void**)&B->d_adj, (size_t)B->n * sizeof(KzAdjItem));
    if (e != cudaSuccess) {
        kz_set_error("kz_precode_adjoint_batched: %s", cudaGetErrorString(e));
        return KZ_ERR_NOMEM;
    }
    // staged copy from pageable memory: the host table may be reused on return
    e = cudaMemcpyAsync(B->d_adj, adj.data(), (size_t)B->n * sizeof(KzAdjItem), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = kz_adjoint_rhs_batched(B->d_insts, B->d_adj, B->n, B->K_max, B->nrhs, st);
    if (e != cudaSuccess) return check_launch(e, "kz_precode_adjoint_batched right-hand side");
    kz_status rc = kz_precode_batched(B, KZ_SEL_ARGMAX, tol, max_iter, 0, 0, status, stream);
    if (rc != KZ_OK) return rc;
    e = kz_adjoint_contract_batched(B->d_insts, B->d_adj, B->n, B->K_max, B->nrhs, st);
    return check_launch(e, "kz_precode_adjoint_batched contraction");
}

kz_status kz_precoder_matrix(kz_plan* P, const kz_cf32* V, int32_t ncols, int32_t S, int32_t normalise, kz_cf32* F,
                             float* beta, void* stream) {
    g_err.clear();
    if (!P || !V || !F || ncols < 1 || S < 1 || S > P->Nt || (normalise && !beta) || !aligned(V, 8) ||
        !aligned(F, 8) || (beta && !aligned(beta, 4))) {
        kz_set_error("kz_precoder_matrix: need a plan, V and F (8-byte aligned), ncols >= 1, 1 <= S <= Nt, and beta "
                     "when normalising");
        return KZ_ERR_INVALID_ARG;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    if (P->q_S != S) {  // Q_s: users whose VR meets subarray s
        std::vector<int> qptr(S + 1, 0), qidx;
        for (int s = 0; s < S; ++s) {
            const long n0 = (long)s * P->Nt / S, n1 = (long)(s + 1) * P->Nt / S;
            for (int k = 0; k < P->K; ++k)
                if (P->vr_off[k] < n1 && P->vr_off[k] + P->vr_len[k] > n0) qidx.push_back(k);
            qptr[s + 1] = (int)qidx.size();
        }
        if (P->d_qptr) cudaFree(P->d_qptr);
        if (P->d_qidx) cudaFree(P->d_qidx);
        P->d_qptr = P->d_qidx = nullptr;
        P->q_S = 0;
        e = upload(&P->d_qptr, qptr, st);
        if (e == cudaSuccess) e = upload(&P->d_qidx, qidx, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the host vectors go out of scope
        if (e != cudaSuccess) return check_launch(e, "kz_precoder_matrix set-up");
        P->q_S = S;
    }
    const size_t need = (size_t)S * ((ncols + 31) / 32);
    if (P->qpart_n < need) {
        if (P->d_qpart) cudaFree(P->d_qpart);
        P->d_qpart = nullptr;
        P->qpart_n = 0;
        e = cudaMalloc((void**)&P->d_qpart, need * sizeof(double));
        if (e != cudaSuccess) {
            kz_set_error("kz_precoder_matrix: %s", cudaGetErrorString(e));
            return KZ_ERR_NOMEM;
        }
        P->qpart_n = need;
    }
    e = kz_subarray_precoder(P->inst(), P->d_qptr, P->d_qidx, S, reinterpret_cast<const float2*>(V), ncols,
                             reinterpret_cast<float2*>(F), P->d_qpart, normalise ? beta : nullptr, st);
    return check_launch(e, "kz_precoder_matrix");
}

kz_status kz_plan_flops(const kz_plan* P, int32_t scheme, int32_t S, double T, double* flops) {
    g_err.clear();
    if (!P || !flops || S < 1 || S > (P ? P->Nt : 1) || !(T >= 0.0)) {
        kz_set_error("kz_plan_flops: need a plan, flops, 1 <= S <= Nt and T >= 0");
        return KZ_ERR_INVALID_ARG;
    }
    const double K = P->K, Nt = P->Nt;
    const double M = (double)P->sumL / K;                           // mean |Gamma_k|
    const double X = (double)P->xidx.size() / K - 1.0;              // mean |X_k| without k itself
    const double F = P->nF, V = K - P->nF;
    double Qsum = 0.0;                                              // mean |Q_s| over the S subarrays
    for (int s = 0; s < S; ++s) {
        const long n0 = (long)s * P->Nt / S, n1 = (long)(s + 1) * P->Nt / S;
        for (int k = 0; k < P->K; ++k)
            if (P->vr_off[k] < n1 && P->vr_off[k] + P->vr_len[k] > n0) Qsum += 1.0;
    }
    const double Q = Qsum / S;
    double f;
    switch (scheme) {
        case -1: f = 8 * K * K * K + 9 * K * K + 12 * Nt * K * K - 3 * K; break;
        case KZ_RK_UNIFORM: f = 8 * Nt * K * K + 4 * Nt * K + T * (16 * Nt - 4); break;
        case KZ_RK_SWOR: f = 8 * Nt * K * K + 4 * Nt * K + K - 1 + T * (16 * Nt + K + 8); break;
        case KZ_GK: f = 8 * Nt * K * K + 4 * Nt * K - K + T * (8 * Nt * (K + 1) + K - 5); break;
        case KZ_VR_OGRK: f = 8 * Nt * K * (Q + 0.5) - K + T * (8 * M * (X + 1) + K - 5); break;
        case KZ_VR_OAHK: f = 8 * Nt * K * (Q + 0.5) + T * (8 * M * (2 * V + F + 2) + 24 * V + 14 * Nt + 5); break;
        default:
            kz_set_error("kz_plan_flops: Table I has no row for scheme %d", scheme);
            return KZ_ERR_UNSUPPORTED;
    }
    *flops = f;
    return KZ_OK;
}

kz_status kz_sum_rate(const kz_plan* plan, const kz_cf32* X, double snr_lin, double* sinr, double* rate,
                      void* stream) {
    g_err.clear();
    if (!plan || !X || !aligned(X, 8) || !(snr_lin > 0.0) || (!sinr && !rate) || (sinr && !aligned(sinr, 8)) ||
        (rate && !aligned(rate, 8))) {
        kz_set_error("kz_sum_rate: need a plan, an 8-byte aligned X, snr_lin > 0 and an output");
        return KZ_ERR_INVALID_ARG;
    }
    if ((2 * (size_t)plan->K + 32) * sizeof(double) > kSmemLimit) {
        kz_set_error("kz_sum_rate: K = %d users exceed the kernel's shared memory", plan->K);
        return KZ_ERR_UNSUPPORTED;
    }
    cudaError_t e = kz_sum_rate(plan->inst(), reinterpret_cast<const float2*>(X), snr_lin, sinr, rate,
                                static_cast<cudaStream_t>(stream));
    return check_launch(e, "kz_sum_rate");
}

kz_status kz_sum_rate_batched(const kz_batch* B, double snr_lin, double* sinr, double* rate, void* stream) {
    g_err.clear();
    if (!B || !(snr_lin > 0.0) || (!sinr && !rate) || (sinr && !aligned(sinr, 8)) || (rate && !aligned(rate, 8))) {
        kz_set_error("kz_sum_rate_batched: need a batch, snr_lin > 0 and an output");
        return KZ_ERR_INVALID_ARG;
    }
    for (int b = 0; b < B->n; ++b)
        if (B->plans[b]->K != B->nrhs) {
            kz_set_error("kz_sum_rate_batched: item %d has K = %d users but %d columns", b, B->plans[b]->K, B->nrhs);
            return KZ_ERR_INVALID_ARG;
        }
    if ((2 * (size_t)B->K_max + 32) * sizeof(double) > kSmemLimit) {
        kz_set_error("kz_sum_rate_batched: K = %d users exceed the kernel's shared memory", B->K_max);
        return KZ_ERR_UNSUPPORTED;
    }
    cudaError_t e = kz_sum_rate_batched(B->d_insts, B->n, B->K_max, snr_lin, sinr, rate,
                                        static_cast<cudaStream_t>(stream));
    return check_launch(e, "kz_sum_rate_batched");
}

kz_status kz_precode_adjoint(kz_plan* plan, int32_t nrhs, float xi, const kz_cf32* Q, const kz_cf32* X,
                             const kz_cf32* G_Q, const kz_cf32* G_X, double tol, int32_t max_iter, kz_cf32* lambda,
                             kz_cf32* y, kz_cf32* grad_H_packed, float* grad_xi, int32_t* iters, double* resid,
                             int32_t* status, void* stream) {
    g_err.clear();
    kz_status rc = check_solve_args("kz_precode_adjoint", plan, nrhs, xi, KZ_VR_OAHK, KZ_SEL_ARGMAX, tol, max_iter, 0, 0);
    if (rc != KZ_OK) return rc;
    if (!Q || !X || !lambda || !y || !grad_H_packed || !grad_xi || !iters || !resid || (!G_Q && !G_X)) {
        kz_set_error("kz_precode_adjoint: Q, X, lambda, y, grad_H_packed, grad_xi, iters, resid and one of G_Q / G_X are required");
        return KZ_ERR_INVALID_ARG;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t need = (size_t)plan->K * nrhs;
    if (plan->scratch_elems < need) {
        if (plan->d_scratch) cudaFree(plan->d_scratch);
        plan->d_scratch = nullptr;
        plan->scratch_elems = 0;
        cudaError_t e = cudaMalloc((void**)&plan->d_scratch, need * sizeof(float2));
        if (e != cudaSuccess) {
            kz_set_error("kz_precode_adjoint: %s", cudaGetErrorString(e));
            return KZ_ERR_NOMEM;
        }
        plan->scratch_elems = need;
    }
    KzInst I = plan->inst();
    I.xi = xi;
    I.ld = nrhs;
    cudaError_t e;
    if (G_X) {
        e = kz_adjoint_rhs(I, nrhs, reinterpret_cast<const float2*>(G_Q), reinterpret_cast<const float2*>(G_X),
                           plan->d_scratch, st);
    } else {
        e = cudaMemcpyAsync(plan->d_scratch, G_Q, need * sizeof(float2), cudaMemcpyDeviceToDevice, st);
    }
    if (e != cudaSuccess) return check_launch(e, "kz_precode_adjoint right-hand side");
    rc = kz_precode(plan, reinterpret_cast<const kz_cf32*>(plan->d_scratch), nrhs, xi, KZ_VR_OAHK, KZ_SEL_ARGMAX, tol,
                    max_iter, 0, y, lambda, iters, resid, status, 0, 0, stream);
    if (rc != KZ_OK) return rc;
    e = kz_adjoint_contract(I, nrhs, reinterpret_cast<const float2*>(Q), reinterpret_cast<const float2*>(X),
                            reinterpret_cast<const float2*>(G_X), reinterpret_cast<const float2*>(lambda),
                            reinterpret_cast<const float2*>(y), plan->d_in_off, reinterpret_cast<float2*>(grad_H_packed),
                            grad_xi, st);
    return check_launch(e, "kz_precode_adjoint contraction");
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free adjoint.  Some callers cannot allocate device memory at the
// time they differentiate: a real-time loop that must not block in the
// driver's allocator, a process whose device memory is all reserved up front
// by another allocator (so a cudaMalloc would fail), or a runtime that forbids
// allocation after start-up.  For them the right-hand side G~ = G_Q + H G_X,
// the only scratch of the adjoint, lives in this file-scope device array
// instead of plan-owned memory.  Each device's context holds its own copy.
namespace {

constexpr int64_t kNoAllocMaxElems = 262144;  // K * nrhs complex entries (2 MiB)
static __device__ __align__(256) float2 g_kz_adjoint_scratch[kNoAllocMaxElems];

constexpr int kNoAllocMaxDevices = 64;
// Cached device address of the array, per device.  Atomic so that two host
// threads making their first call on one device do not race: both may look
// the address up, and both store the same value.
std::atomic<float2*> g_noalloc_ptr[kNoAllocMaxDevices];

// Host code cannot use the array's name as a device address; fetch the
// address once per device, with that device current.
kz_status noalloc_scratch(float2** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return check_launch(e, "kz_precode_adjoint_noalloc cudaGetDevice");
    if (dev < 0 || dev >= kNoAllocMaxDevices) {
        kz_set_error("kz_precode_adjoint_noalloc: device %d is beyond the supported %d", dev, kNoAllocMaxDevices);
        return KZ_ERR_UNSUPPORTED;
    }
    float2* p = g_noalloc_ptr[dev].load(std::memory_order_acquire);
    if (!p) {
        void* a = nullptr;
        e = cudaGetSymbolAddress(&a, g_kz_adjoint_scratch);
        if (e != cudaSuccess) return check_launch(e, "kz_precode_adjoint_noalloc cudaGetSymbolAddress");
        p = static_cast<float2*>(a);
        g_noalloc_ptr[dev].store(p, std::memory_order_release);
    }
    *out = p;
    return KZ_OK;
}

}  // namespace

extern "C" kz_status kz_precode_adjoint_noalloc(kz_plan* plan, int32_t nrhs, float xi, const kz_cf32* Q,
                                                const kz_cf32* X, const kz_cf32* G_Q, const kz_cf32* G_X,
                                                double tol, int32_t max_iter, kz_cf32* lambda, kz_cf32* y,
                                                kz_cf32* grad_H_packed, float* grad_xi, int32_t* iters,
                                                double* resid, int32_t* status, void* stream) {
    g_err.clear();
    kz_status rc = check_solve_args("kz_precode_adjoint_noalloc", plan, nrhs, xi, KZ_VR_OAHK, KZ_SEL_ARGMAX, tol,
                                    max_iter, 0, 0);
    if (rc != KZ_OK) return rc;
    if (!Q || !X || !lambda || !y || !grad_H_packed || !grad_xi || !iters || !resid || (!G_Q && !G_X)) {
        kz_set_error("kz_precode_adjoint_noalloc: Q, X, lambda, y, grad_H_packed, grad_xi, iters, resid and one of "
                     "G_Q / G_X are required");
        return KZ_ERR_INVALID_ARG;
    }
    const int64_t need = (int64_t)plan->K * nrhs;
    if (need > kNoAllocMaxElems) {
        kz_set_error("kz_precode_adjoint_noalloc: K * nrhs = %lld exceeds the static scratch of %lld entries",
                     (long long)need, (long long)kNoAllocMaxElems);
        return KZ_ERR_INVALID_ARG;
    }
    float2* scratch = nullptr;
    rc = noalloc_scratch(&scratch);
    if (rc != KZ_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    KzInst I = plan->inst();
    I.xi = xi;
    I.ld = nrhs;
    // every entry of G~ that the solve reads is written first, so nothing is cleared
    cudaError_t e;
    if (G_X) {
        e = kz_adjoint_rhs(I, nrhs, reinterpret_cast<const float2*>(G_Q), reinterpret_cast<const float2*>(G_X),
                           scratch, st);
    } else {
        e = cudaMemcpyAsync(scratch, G_Q, (size_t)need * sizeof(float2), cudaMemcpyDeviceToDevice, st);
    }
    if (e != cudaSuccess) return check_launch(e, "kz_precode_adjoint_noalloc right-hand side");
    rc = kz_precode(plan, reinterpret_cast<const kz_cf32*>(scratch), nrhs, xi, KZ_VR_OAHK, KZ_SEL_ARGMAX, tol,
                    max_iter, 0, y, lambda, iters, resid, status, 0, 0, stream);
    if (rc != KZ_OK) return rc;
    e = kz_adjoint_contract(I, nrhs, reinterpret_cast<const float2*>(Q), reinterpret_cast<const float2*>(X),
                            reinterpret_cast<const float2*>(G_X), reinterpret_cast<const float2*>(lambda),
                            reinterpret_cast<const float2*>(y), plan->d_in_off,
                            reinterpret_cast<float2*>(grad_H_packed), grad_xi, st);
    return check_launch(e, "kz_precode_adjoint_noalloc contraction");
}
