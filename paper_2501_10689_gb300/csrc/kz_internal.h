// Internal definitions shared by the libkzprecode translation units.
//
// Device layout of one channel (a "plan"):
//   * Row k's VR [o_k, e_k) (e_k = o_k + vr_len[k]) is stored over the
//     aligned interval [a_k, b_k) with a_k = o_k rounded down to even and
//     b_k = e_k rounded up to even, zero-filled outside [o_k, e_k).  Row k
//     starts at complex offset rptr[k] (even), so every pair of antennas
//     (2p, 2p+1) of a row is one 16-byte load, aligned with the same pair of
//     the iterate m.  Padding entries are exact zeros and contribute nothing
//     to any product.
//   * The antenna axis is cut into tiles of KZ_TILE = 64 antennas; tile t
//     lists the rows whose aligned interval meets it (V rows first, then F
//     rows), so H^H phi is formed antenna-major with no scatter (each
//     thread owns one antenna pair and loops over the covering rows).
//   * Ntp = Nt + 1 rounded up to a whole tile: the length of each iterate
//     column in shared memory (b_k <= Nt + 1).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "../../include/kzprecode.h"

#define KZ_TILE 64
// Tensor-core mode: padding of each iterate column in shared memory (entries
// of 4 bytes), so that the two columns one 8-lane phase of a 16-byte fragment
// load reads start 64 bytes (16 banks) apart
#define KZ_TC_PAD 16

struct KzInst {
    // --- channel (fixed at plan creation) ---
    int K, Nt, Ntp, ntiles, nF;
    int inst;                  // instance number: keys the random streams
    const int4* rows;          // {a, len2, o, e} per row
    const int* rptr;           // aligned complex offset of each row
    const float* nrm;          // ||h_k||^2 (rounded from an FP64 sum)
    const int* order;          // F rows then V rows, each by decreasing VR length
    const int* xptr;           // CSR of X_k (k included)
    const int* xidx;
    const int* tptr;           // CSR of covering rows per tile
    const int* tnv;            // number of V rows at the head of each tile list
    const int4* trow4;         // per entry {row, rptr - a, a, a + len2}
    const float2* Hc;          // aligned complex64 rows
    const __nv_bfloat162* Hb;  // aligned BF16 (re, im) rows, or nullptr
    // aligned FP16 (re, im) rows scaled by 1 / hs[k] (complex64 plans; the
    // tensor-core contractions), and hs[k] = the power of two at or above
    // ||h_k|| (every scaled entry below 1 in magnitude)
    const __half2* Hh;
    const float* hs;
    const double* nrmd;        // ||h_k||^2 in FP64
    const int* in_off;         // row k's offset in the caller's packed layout
    const int* vsort;          // V rows (K - nF), then all K rows, each by VR centre
    const float2* G;           // H H^H on the CSR pattern of X_k (compensated FP32 sums)
    int cmax;                  // most rows covering one tile
    // --- call ---
    float xi;
    int ld;                    // number of columns of s / x / v
    const float2* s;
    float2* x;
    float2* v;
    int* iters;
    double* resid;
};

struct KzLaunch {
    const KzInst* insts;  // batched: device table; nullptr: use `single`
    KzInst single;
    const int2* items;    // batched: {instance, first column}; nullptr: item k = columns [kJ, kJ+J)
    int n_items;
    int* queue;           // work-queue counter (zeroed before the launch), or nullptr
    int algo, sel, prec;
    double tol;
    int max_iter;
    int refresh;
    unsigned long long seed;
    int* status;
    int Ntp_max, K_max;
    int tc;               // resident kernel: tensor-core inner products (correction form)
    int m_elems;          // resident kernel: shared iterate entries per CTA (0: J x (Ntp_max + pad))
    int trow_max;         // tensor-core kernel: covering-list entries staged in shared memory (0: none)
    // row kernel: selected-row history (row index and step gamma of step t of
    // column c at [t * hist_ld + c], t < hist_T), or nullptr
    int* hist_row;
    float2* hist_gam;
    int hist_ld, hist_T;
};

// Work item {instance, first column | (columns << 24)}: the column count of
// an item (its width, at most the kernel's J) is 0 for "J".
#define KZ_ITEM_COL(y) ((y) & 0xffffff)
#define KZ_ITEM_WIDTH(y, J) (((y) >> 24) ? ((y) >> 24) : (J))

// Host-side launchers (kz_ahk.cu / kz_kacz.cu).
cudaError_t kz_launch_ahk(const KzLaunch& L, int J, int nw, int grid, size_t smem, cudaStream_t st);
cudaError_t kz_launch_kacz(const KzLaunch& L, int J, int nw, int grid, size_t smem, cudaStream_t st);
// Small-channel kernel (kz_small.cu): single channel with K <= 32 and
// Ntp <= 512, one CTA of 8 warps per column.
cudaError_t kz_launch_small(const KzLaunch& L, int grid, size_t smem, cudaStream_t st);
size_t kz_smem_small(int K, int Ntp);
size_t kz_smem_ahk(int J, int Ntp, int K, int prec);
size_t kz_smem_kacz(int J, int Ntp, int K);
int kz_occupancy_ahk(int J, int nw, size_t smem, int prec);
// Tensor-core mode: m_elems shared iterate entries (columns of Ntp + KZ_TC_PAD) and
// trow covering-list row indices staged as 16-bit entries.
size_t kz_smem_ahk_tc(int J, int m_elems, int Ntp_max, int K, int trow = 0);
int kz_occupancy_ahk_tc(int J, int nw, size_t smem);
int kz_occupancy_kacz(int J, int nw, size_t smem);

// Auxiliary kernels (kz_aux.cu).
cudaError_t kz_pack_rows(const float2* Hin, const int* in_off, const int4* rows, const int* rptr, int K,
                         int64_t total2, float2* Hc, __nv_bfloat162* Hb, cudaStream_t st);
cudaError_t kz_pack_dense(const float2* Hd, int Nt, const int4* rows, const int* rptr, int K, float2* Hc,
                          __nv_bfloat162* Hb, cudaStream_t st);
// Row norms; with Hh, also the scaled FP16 copy of every row and its scale hs.
cudaError_t kz_row_norms(const float2* Hc, const int4* rows, const int* rptr, int K, double* out_d,
                         float* out_f, __half2* Hh, float* hs, cudaStream_t st);
cudaError_t kz_gram(const float2* Hc, const int4* rows, const int* rptr, const int* xptr, const int* xidx, int K,
                    float2* G, cudaStream_t st);
// Re-pack items of a batch from H_cat (item b's packed channel at
// H_cat + hoff[b]): packing, row norms and inner products of overlapping rows
// (upper half, then the mirror), one launch each over the (item, row) pairs
// rowmap[row0, row0 + nrows).
cudaError_t kz_batch_update_rows(const KzInst* insts, const int2* rowmap, int row0, int nrows, const long long* hoff,
                                 const float2* H_cat, cudaStream_t st);
// Subarray-wise precoder F = H^H V over S subarrays (Q_s in CSR qptr / qidx);
// with beta non-NULL, F is scaled by beta = 1 / ||F||_F (part: S x ceil(ncols / 32) doubles).
cudaError_t kz_subarray_precoder(const KzInst& I, const int* qptr, const int* qidx, int S, const float2* V, int ncols,
                                 float2* F, double* part, float* beta, cudaStream_t st);
// Reverse pass through a recorded row-action solve (kz_aux.cu): one CTA per
// column; gradients with respect to the packed H (accumulated, caller zeroes
// it), xi (accumulated into *gxi) and s.
cudaError_t kz_unrolled_adjoint(const KzInst& I, int nrhs, int T, const int* iters, const int* hrow, const float2* hgam,
                                const float2* X, const float2* Vq, const float2* GX, const float2* GV, float2* gH,
                                double* gxi, float2* gS, float* gxi_out, cudaStream_t st);
size_t kz_smem_unrolled(int Nt, int K);
// Coupling of every channel of a batch: mu[b] = max_k sum_{l in X_k, l != k}
// |G_kl|^2 / (d_k d_l), d = ||h||^2 + xi (the largest squared off-diagonal
// row mass of the row-normalised system), one block per channel.
cudaError_t kz_coupling(const KzInst* insts, int n, float* mu, cudaStream_t st);
cudaError_t kz_adjoint_rhs(const KzInst& I, int nrhs, const float2* G_Q, const float2* G_X, float2* Gt,
                           cudaStream_t st);
cudaError_t kz_adjoint_contract(const KzInst& I, int nrhs, const float2* Q, const float2* X,
                                const float2* G_X, const float2* Lam, const float2* Y,
                                const int* in_off, float2* grad_H, float* grad_xi, cudaStream_t st);

// Batched adjoint pieces: item b's channel is insts[b] (its s / x / v are the
// adjoint right-hand side G~, y = H^H Lambda and Lambda), its gradients and
// forward outputs are in adj[b].
struct KzAdjItem {
    const float2* Q;
    const float2* X;
    const float2* G_Q;
    const float2* G_X;
    float2* grad_H;
    float* grad_xi;
};
cudaError_t kz_adjoint_rhs_batched(const KzInst* insts, const KzAdjItem* adj, int n, int K_max, int nrhs,
                                   cudaStream_t st);
cudaError_t kz_adjoint_contract_batched(const KzInst* insts, const KzAdjItem* adj, int n, int K_max, int nrhs,
                                        cudaStream_t st);

// Per-user SINR and sum rate of F = X / ||X||_F (kz_aux.cu): one channel, or
// every channel of a batch (its items' x, SINRs at b * K_max).
cudaError_t kz_sum_rate(const KzInst& I, const float2* X, double snr_lin, double* sinr, double* rate,
                        cudaStream_t st);
cudaError_t kz_sum_rate_batched(const KzInst* insts, int n, int K_max, double snr_lin, double* sinr, double* rate,
                                cudaStream_t st);

// Group kernel (kz_grp.cu): one channel, the CTAs of a column group share it
// by antenna blocks of 128; contractions on tcgen05 tensor cores.
struct KzGrpChan {
    int K, Nt, AB, n_slots;
    const int* slot_row;        // [AB][256] row of slot r of block b (-1: padding), rows ascending
    const int* blk_nrt;         // [AB] row tiles of 128 slots (1 or 2)
    const int* blk_nb;          // [AB] rows meeting the block
    const int* blk_coff;        // [AB] first compact partial slot of the block
    const long long* blk_toff;  // [AB] byte offset of the block's tile image
    const uint8_t* tiles;       // 16-bit tile images
    const int* cptr;            // [K + 1] CSR over rows: compact partial slots of the blocks row k meets
    const int* cidx;
    const float* nrm;           // ||h_k||^2
    const unsigned char* inF;   // [K] 1: row k is in the orthogonal set F
    const int* xptr;            // X_k pattern and H H^H on it (refresh)
    const int* xidx;
    const float2* G;
    const float2* Hc;           // aligned complex64 rows (x = H^H q at the end)
    const int4* rows;
    const int* rptr;
    const float* stat;          // [2] sigma_H (power of two, tiles hold H / sigma_H), mean ||h_k||^2
};

struct KzGrpLaunch {
    KzGrpChan C;
    float xi;
    int nrhs;               // columns of s / x / v handled by this launch
    int NC, CG;             // columns per group, groups (gridDim.y)
    int algo, fmt;          // KZ_AHK / KZ_VR_OAHK; 0 FP16, 1 BF16 operands
    double tol;
    int max_iter, refresh;
    const float2* s;        // K x nrhs (column-major), x Nt x nrhs, v K x nrhs (may be NULL)
    float2* x;
    float2* v;
    int* iters;
    double* resid;
    int* status;            // may be NULL
    // scratch (device)
    float2* Ppart;          // [CG][n_slots][NC] residual partial sums
    uint16_t* Phi;          // [CG][K][2][NC] 16-bit phi / tau
    float2* Qg;             // [CG][K][NC] q at the last refresh
    float* colpart;         // [CG][7][AB][NC] per-CTA column partials
    unsigned* gbar;         // [g] group g's grid barrier counter (0), [CG + g] its abort epoch (0xffffffff)
    int rpc, rtmax, tmem_cols;
};

cudaError_t kz_grp_prepare(const KzGrpChan& C, const float2* Hc, long long total2, const int4* rows, const int* rptr,
                           const float* nrm, float* stat, int fmt, cudaStream_t st);
size_t kz_grp_smem(int NC, int rtmax, int rpc, int AB);
bool kz_grp_fits(int AB, int CG, bool cluster, size_t smem);
cudaError_t kz_launch_grp(const KzGrpLaunch& L, bool cluster, size_t smem, cudaStream_t st);

// Thread-local last-error text (kz_api.cu).
void kz_set_error(const char* fmt, ...);
