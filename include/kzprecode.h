/*
 * libkzprecode -- Kaczmarz-type RZF precoders for near-field multiuser
 * systems with spatial non-stationarity, on one GB300 (sm_103a).
 *
 * The library solves, for each right-hand side s (a K-vector of symbols),
 *
 *     x = H^H (H H^H + xi I)^-1 s                        (eq. (precoding), Thm. 1)
 *
 * without forming or inverting the Gram matrix: it runs a Kaczmarz sweep over
 * the rows of the consistent system B w = s, B = [H, sqrt(xi) I_K] (eq. (SLE)),
 * from w = 0, and reads x = m and v = q off w = [m; sqrt(xi) q] (Remark 1).
 *
 * Conventions shared by every call:
 *   - H is K x Nt; row k is user k's channel, non-zero only on its visibility
 *     region (VR), the contiguous antenna interval
 *     [vr_offset[k], vr_offset[k] + vr_len[k]) (eqs. (3)-(4), Sec. IV-B).
 *   - H_packed stores row k's VR slice (vr_len[k] entries) at element
 *     sum_{j<k} vr_len[j]; entries are interleaved complex64 (kz_cf32).
 *   - Matrices of right-hand sides and solutions are column-major:
 *     s is K x nrhs (element (k, j) at s[k + K j]), x is Nt x nrhs,
 *     v is K x nrhs.  Column j is one independent system (Remark 2).
 *   - Device pointers are CUDA device memory of the current device; the
 *     caller owns them.  Host pointers are plain host memory.
 *   - "stream" is a cudaStream_t passed as void*; NULL means the legacy
 *     default stream.  Solve calls are asynchronous on that stream: their
 *     device outputs are valid once the stream has been synchronised.
 *   - Functions return kz_status.  KZ_ERR_INVALID_ARG is returned before any
 *     work is enqueued; kz_last_error() gives a one-line reason (thread-local).
 *     Nothing is thrown across this interface.
 *   - Convergence: every method stops per right-hand side once its relative
 *     residual ||s - B w|| / ||s|| <= tol (the paper stops on an NMSE against
 *     the RZF answer, which a solver cannot know) or after max_iter
 *     iterations.  The per-call device status word (optional) receives
 *     KZ_STATUS_BIT_NOT_CONVERGED and/or KZ_STATUS_BIT_NUMERIC.
 */
#ifndef KZPRECODE_H
#define KZPRECODE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    float re, im;
} kz_cf32;

typedef enum {
    KZ_OK = 0,
    KZ_NOT_CONVERGED = 1,    /* some column reached max_iter (outputs still written) */
    KZ_ERR_INVALID_ARG = 2,  /* bad size, VR, pointer alignment or enum */
    KZ_ERR_NUMERIC = 3,      /* NaN or Inf in a residual */
    KZ_ERR_CUDA = 4,         /* a CUDA runtime call failed */
    KZ_ERR_NOMEM = 5,        /* device allocation failed */
    KZ_ERR_UNSUPPORTED = 6   /* combination not provided (e.g. BF16 with a row method) */
} kz_status;

/* Bits the kernels OR into the optional device status word. */
#define KZ_STATUS_BIT_NOT_CONVERGED 1
#define KZ_STATUS_BIT_NUMERIC 2
#define KZ_STATUS_BIT_TIMEOUT 4  /* a bounded device wait expired (the call's outputs are not valid) */

/* Methods.  RK_ENERGY / RK_UNIFORM: Alg. 1 with p_i = ||b_i||^2/||B||_F^2 or 1/K
 * (Sec. III-A; RK_UNIFORM is the URK of Table I).  GRK: greedy selection
 * with every residual recomputed (Sec. IV-A).  VR_OGRK: Alg. 2, residuals
 * recomputed only on X_{i(t-1)}.  AHK: aggregation-hyperplane step on all
 * rows (eqs. (update4), (coefficient)).  VR_OAHK: Alg. 3, unit step on the
 * orthogonal set F (Prop. 1) followed by an AHK step on the rest V.
 * RK_SWOR (SWOR-ERK of Table I): energy weights, each sweep of K steps
 * drawing rows without replacement (p_i proportional to ||b_i||^2 over the
 * rows not yet drawn in the sweep).  GK (Table I): GRK with the maximal-
 * residual rule, i.e. KZ_SEL_ARGMAX whatever `sel` says. */
typedef enum {
    KZ_RK_ENERGY = 0,
    KZ_RK_UNIFORM = 1,
    KZ_GRK = 2,
    KZ_AHK = 3,
    KZ_VR_OGRK = 4,
    KZ_VR_OAHK = 5,
    KZ_RK_SWOR = 6,
    KZ_GK = 7
} kz_algo;

/* Row selection for GRK / VR_OGRK.  PAPER: sample p_i = |r_i|^2/||r||^2
 * (Sec. IV-A, Alg. 2 step 4).  BAIWU: the same sampling restricted to the
 * greedy set of Bai & Wu cited in Sec. IV-A.  ARGMAX: i = argmax |r_i|^2/||b_i||^2,
 * lowest index on ties.  Random draws use the SplitMix64 counter-based
 * generator keyed by (seed, instance, column, iteration). */
typedef enum { KZ_SEL_PAPER = 0, KZ_SEL_BAIWU = 1, KZ_SEL_ARGMAX = 2 } kz_select;

/* Storage / arithmetic of the iteration.  C64: complex64 H, FP32 arithmetic.
 * BF16_MIXED (AHK / VR_OAHK only): the residual and projection read a BF16
 * copy of H with FP32 accumulation, in correction form against a true
 * residual recomputed from the complex64 H (FP32 products, compensated
 * sums) every refresh period; that recomputation drives the stopping test. */
typedef enum { KZ_C64 = 0, KZ_BF16_MIXED = 1 } kz_prec;

/* Which kernel runs AHK / VR_OAHK.  RESIDENT keeps the iterate m of J
 * columns in shared memory and streams H per column group (every method,
 * both precisions).  TC (AHK / VR_OAHK, C64, 4 or 8 columns) is
 * RESIDENT in correction form with the two contractions of each iteration
 * (the V-row residuals and H_V^H phi) on the tensor cores with FP16 operands
 * and FP32 sums, reading an FP16 copy of H that every C64 plan keeps (each
 * row scaled by a power of two at or above its norm; 4 bytes per stored
 * entry beside the 8 of complex64); the right-hand side b = s - H m_ref is
 * recomputed from the complex64 H every `refresh` iterations and every stop
 * is confirmed on the true residual, so results meet the same tolerance as
 * RESIDENT.  GROUP (AHK /
 * VR_OAHK, one channel shared by many columns) spreads one channel over a
 * group of CTAs -- each owns a 128-antenna block of the iterate for 16, 32
 * or 64 columns and keeps the block's rows in shared memory -- and runs both
 * contractions of each half-step on the Blackwell tensor cores (tcgen05.mma,
 * FP32 accumulators in tensor memory) with 16-bit operands: FP16 (H scaled
 * by a power of two) on C64 plans, BF16 on BF16_MIXED plans; in correction
 * form with the refresh through the plan's inner products of overlapping
 * rows, every stop confirmed on the true residual.  A group is one cluster of
 * CTAs for channels up to 2048 antennas, else every CTA of a cooperative
 * launch (then one launch serves at most SMs / blocks groups; more columns
 * take further launches).  KZ_ERR_UNSUPPORTED when a 128-antenna block is
 * seen by more than 256 users.  SMALL (every method, C64, channels of at
 * most 32 users and 511 antennas whose rows fit shared memory): one CTA of 8
 * warps per column with the whole state in shared memory and a few short
 * phases per step, for the latency of single small solves (rhs_per_cta 0
 * or 1).  AUTO for kz_precode (with rhs_per_cta 0): SMALL when it applies
 * and nrhs is at most the GPU's SM count; GROUP for AHK / VR_OAHK on
 * channels of 4096 antennas or more (RESIDENT if the group kernel cannot
 * hold the channel); else RESIDENT.  The batch default is RESIDENT until
 * kz_batch_tune or kz_batch_set_launch chooses. */
typedef enum {
    KZ_KERNEL_AUTO = 0,
    KZ_KERNEL_RESIDENT = 1,
    KZ_KERNEL_TC = 3,
    KZ_KERNEL_GROUP = 4,
    KZ_KERNEL_SMALL = 5
} kz_kernel;

typedef struct kz_plan kz_plan;
typedef struct kz_batch kz_batch;

/* Build the per-channel set-up (step A0): row norms ||h_k||^2, the VR overlap
 * graph, the non-orthogonal sets X_k (Sec. IV-B, k included), the orthogonal
 * set F as a maximum independent set of the overlap graph (eq. (max_set);
 * exact for contiguous VRs by the earliest-end rule), the antenna-tile
 * covering lists and the device copies of H in the solver's aligned layout
 * (each row's VR widened to multiples of four antennas, zero-filled):
 * complex64, plus BF16 when prec == KZ_BF16_MIXED, plus, when prec ==
 * KZ_C64, an FP16 copy for the tensor-core kernel (each row scaled by a power
 * of two at or above its norm; 4 bytes per stored entry against 8).
 *   K, Nt: users and antennas, 1 <= K < Nt (Sec. II).
 *   vr_offset, vr_len: host int32[K]; every VR must satisfy
 *     vr_len >= 1 and 0 <= vr_offset, vr_offset + vr_len <= Nt.
 *   H_packed: device kz_cf32[sum vr_len] (layout above), 8-byte aligned.
 *     It is copied; the caller may free it after this call returns.
 *   stream: the copies and set-up kernels are enqueued there and the call
 *     waits for them before returning.
 * On success *out owns all device memory of the plan until kz_plan_destroy. */
kz_status kz_plan_create(kz_plan** out, int32_t K, int32_t Nt, const int32_t* vr_offset,
                         const int32_t* vr_len, const kz_cf32* H_packed, kz_prec prec, void* stream);

/* kz_plan_create from a dense channel matrix: H_dense is device kz_cf32
 * [K * Nt], row-major (entry (k, n) at H_dense[k * Nt + n]), 8-byte aligned.
 * Only the entries inside each user's VR are read; the channel is zero
 * outside it by the VR model h_k = hbar_k (.) u_k (Sec. II, eqs. (3)-(4)),
 * whatever H_dense holds there.  Every other argument, the resulting plan and
 * the errors are those of kz_plan_create; the plan is the one kz_plan_create
 * builds from the same VR entries packed (so kz_plan_update and the adjoint's
 * packed gradient keep the packed layout).  H_dense is not retained. */
kz_status kz_plan_dense(kz_plan** out, int32_t K, int32_t Nt, const int32_t* vr_offset,
                        const int32_t* vr_len, const kz_cf32* H_dense, kz_prec prec, void* stream);

/* Replace the channel of an existing plan (same K, Nt and VRs): re-pack
 * H_packed (device, layout as in kz_plan_create, 8-byte aligned) into the
 * plan's aligned copy (and its BF16 or FP16 copy) and recompute the row norms
 * and the inner products of overlapping rows, as kernels
 * on `stream`; nothing else of the plan changes and no host synchronisation
 * happens, so prepared batches that name the plan stay valid.  Calls that use
 * the plan must be ordered after this one on the stream. */
kz_status kz_plan_update(kz_plan* plan, const kz_cf32* H_packed, void* stream);

/* Release a plan (NULL is ignored).  Not stream-ordered: the caller makes
 * sure no call using the plan is still running. */
void kz_plan_destroy(kz_plan* plan);

/* Sizes and sets of a plan, for inspection and tests (host outputs; any
 * pointer may be NULL).  F receives the orthogonal set (ascending, *nF entries,
 * room for K); X_ptr (K+1) and X_idx (room for K*K) receive the CSR sets X_k. */
kz_status kz_plan_query(const kz_plan* plan, int32_t* K, int32_t* Nt, int64_t* sum_len, int32_t* nF,
                        int32_t* F, int32_t* X_ptr, int32_t* X_idx);

/* Solve nrhs independent systems that share one channel (steps A1-A7).
 *   s: device K x nrhs;  x: device Nt x nrhs (output, also used as the
 *   solver's per-iteration aggregate buffer);  v: device K x nrhs output of
 *   the auxiliary vectors (may be NULL);  iters: device int32[nrhs] (row
 *   projections for the RK family, iterations for AHK / VR_OAHK);  resid:
 *   device double[nrhs], the final true relative residual;  status: device
 *   int32 word the kernel ORs KZ_STATUS_BIT_* into (may be NULL; the caller
 *   zeroes it).
 *   xi > 0; tol >= 0; max_iter >= 1; nrhs >= 1.  rhs_per_cta in {0,1,2,4,8}
 *   (0 = the plan's tuned choice).  refresh: recompute m = H^H q every
 *   `refresh` iterations (0 = default: 16 for AHK / VR_OAHK on C64, 6 for
 *   BF16_MIXED, 8 with KZ_KERNEL_TC, 16 with KZ_KERNEL_GROUP, 512 for the RK
 *   family).
 * Returns KZ_OK once the work is enqueued. */
kz_status kz_precode(kz_plan* plan, const kz_cf32* s, int32_t nrhs, float xi, kz_algo algo,
                     kz_select sel, double tol, int32_t max_iter, uint64_t seed, kz_cf32* x,
                     kz_cf32* v, int32_t* iters, double* resid, int32_t* status, int32_t rhs_per_cta,
                     int32_t refresh, void* stream);

/* kz_precode with an explicit kernel (see kz_kernel).  With KZ_KERNEL_TC,
 * rhs_per_cta must be 0, 4 or 8 (0: 8 when nrhs >= 8 and it fits, else 4)
 * and algo AHK or VR_OAHK on a C64 plan (else KZ_ERR_UNSUPPORTED). */
kz_status kz_precode_ex(kz_plan* plan, const kz_cf32* s, int32_t nrhs, float xi, kz_algo algo,
                        kz_select sel, double tol, int32_t max_iter, uint64_t seed, kz_cf32* x,
                        kz_cf32* v, int32_t* iters, double* resid, int32_t* status, kz_kernel kernel,
                        int32_t rhs_per_cta, int32_t refresh, void* stream);

/* A fixed number of iterations of a row-action method (RK_ENERGY,
 * RK_UNIFORM, RK_SWOR, GRK, GK, VR_OGRK) -- the fixed-T precoders of the
 * paper's spectral-efficiency comparisons (Sec. VII, T = 15) -- recording
 * the selected-row history for kz_unrolled_adjoint: hist_row (device
 * int32[T * nrhs]) and hist_gam (device kz_cf32[T * nrhs]) receive the row
 * and the step gamma of step t of column c at t * nrhs + c (row -1: the
 * column had stopped; a column stops early only when its residual is
 * exactly zero).  The solve takes T row projections per column (tol = 0),
 * so the status word receives KZ_STATUS_BIT_NOT_CONVERGED by design; x, v,
 * iters (the projections taken) and resid are those of kz_precode, v is
 * required.  C64 plans only.  The history is all the reverse pass keeps:
 * O(T) per column instead of the T iterates. */
kz_status kz_precode_record(kz_plan* plan, const kz_cf32* s, int32_t nrhs, float xi, kz_algo algo,
                            kz_select sel, int32_t T, uint64_t seed, kz_cf32* x, kz_cf32* v,
                            int32_t* iters, double* resid, int32_t* hist_row, kz_cf32* hist_gam,
                            int32_t* status, void* stream);

/* Gradient of a real loss through a recorded fixed-iteration solve (the
 * unrolled adjoint; the paper has no gradient).  Given x, v and the history of
 * kz_precode_record and the loss's gradients G_X (Nt x nrhs) and / or G_V
 * (K x nrhs) (PyTorch's convention: dL = Re sum conj(G) dZ; either may be
 * NULL, not both), it replays the steps in reverse -- each iterate before a
 * step is rebuilt from the one after it and the recorded gamma, so no iterate
 * is stored -- and writes dL/dH (grad_H_packed, packed like H_packed), dL/dxi
 * (grad_xi, one float) and dL/ds (grad_s, K x nrhs), treating the selected
 * rows as fixed (the selection is piecewise constant in H).  All pointers are
 * device memory.  One CTA per column holds m and its adjoint: needs
 * (2 Nt + 3 K) * 8 bytes of shared memory (KZ_ERR_UNSUPPORTED beyond 219
 * KiB).  The H gradient is accumulated with atomic additions, so its last
 * bits may vary between calls.  The first call allocates 8 bytes owned by
 * the plan. */
kz_status kz_unrolled_adjoint(kz_plan* plan, int32_t nrhs, float xi, int32_t T, const int32_t* iters,
                              const int32_t* hist_row, const kz_cf32* hist_gam, const kz_cf32* x,
                              const kz_cf32* v, const kz_cf32* G_X, const kz_cf32* G_V,
                              kz_cf32* grad_H_packed, float* grad_xi, kz_cf32* grad_s, void* stream);

/* One item of a batch: a plan with its own right-hand sides and outputs
 * (layouts as in kz_precode, all device pointers, nrhs columns each). */
typedef struct {
    const kz_plan* plan;
    const kz_cf32* s;
    kz_cf32* x;
    kz_cf32* v;      /* may be NULL */
    int32_t* iters;
    double* resid;
    float xi;
} kz_batch_item;

/* Prepare one persistent launch over n instances of uneven K, Nt and VR
 * lengths (step A8): copies the instance table to the device, orders the
 * work (one item = one instance x rhs_per_cta columns) by estimated cost,
 * largest first, and allocates the work-queue counters.  The estimate is the
 * per-iteration work (aligned VR entries + 4 Nt) times a predicted iteration
 * count that grows with the coupling of the users (the largest squared
 * off-diagonal row mass of the row-normalised system, from the plan's inner
 * products of overlapping rows and the item's xi); it only orders the queue
 * and is fixed here (kz_batch_rebind and kz_plan_update keep the order).
 * rhs_per_cta and threads as in kz_precode (0 = tuned).  The plans and
 * buffers named by the items must stay valid while the batch is used.
 * Synchronous. */
kz_status kz_batch_prepare(kz_batch** out, const kz_batch_item* items, int32_t n, int32_t nrhs,
                           kz_algo algo, kz_prec prec, int32_t rhs_per_cta, void* stream);

/* Point every item of a prepared batch at new buffers and a new xi (the
 * plans and nrhs stay those of kz_batch_prepare; items[b].plan must be the
 * plan item b was prepared with).  The instance table is copied on `stream`,
 * ordered after earlier launches of the batch on that stream; a CUDA graph
 * captured earlier replays with the new buffers.  items: host array of
 * batch->n entries, free to reuse on return. */
kz_status kz_batch_rebind(kz_batch* batch, const kz_batch_item* items, void* stream);

/* A new channel for every item of a prepared batch at once (step A0 over
 * step A8): H_cat (device, 8-byte aligned) holds the items' packed channels
 * (layout of kz_plan_create) concatenated in item order, item b's at
 * sum_{c<b} sum(vr_len of item c).  Every item's plan is updated as
 * kz_plan_update would (packing, row norms, inner products of overlapping
 * rows), in four kernel launches for the whole batch, asynchronously on
 * `stream` (the first call also uploads a small row table owned by the
 * batch, synchronously).  The items must name distinct plans
 * (KZ_ERR_INVALID_ARG otherwise).  The batch's queue order is kept. */
kz_status kz_batch_update(kz_batch* batch, const kz_cf32* H_cat, void* stream);

/* kz_batch_update for the items [first, first + count) only (step A0 for
 * part of a batch): H_cat has the layout of kz_batch_update (all items'
 * packed channels in item order), but only the range's channels are read, so
 * a caller can upload the channels of later items while the set-up of
 * earlier ones runs (the launches of one range go to `stream`).  The items
 * must name distinct plans; an empty or out-of-range item range returns
 * KZ_ERR_INVALID_ARG.  Asynchronous on `stream` (the first call of either
 * form uploads the batch's row table, synchronously). */
kz_status kz_batch_update_items(kz_batch* batch, const kz_cf32* H_cat, int32_t first, int32_t count,
                                void* stream);

/* Run a prepared batch: one kernel launch after an 8-byte memset of the
 * queue counters (two launches, the second on a stream forked from `stream`
 * and joined back, when a tensor-core batch holds channels whose columns per
 * CTA do not fit shared memory: those run at 4 columns), no host
 * synchronisation, so it can be captured in a CUDA graph.  status as in
 * kz_precode (may be NULL). */
kz_status kz_precode_batched(kz_batch* batch, kz_select sel, double tol, int32_t max_iter,
                             uint64_t seed, int32_t refresh, int32_t* status, void* stream);

void kz_batch_destroy(kz_batch* batch);

/* Autotune a prepared batch (step A8's launch shape): time every feasible
 * launch on the batch itself -- the RESIDENT kernel with columns-per-CTA in
 * {1, 2, 4, 8} and 256 or 512 threads, and for AHK / VR_OAHK on C64 the TC
 * kernel with 4 or 8 columns (256 or 512 threads) -- three runs each,
 * the last two timed with CUDA events on `stream`; keep the fastest and write
 * it to chosen (host int32[3]: kernel, columns per CTA, threads; may be
 * NULL).  It solves the batch repeatedly, so the batch's outputs hold a
 * valid result afterwards.  Synchronous. */
kz_status kz_batch_tune(kz_batch* batch, kz_select sel, double tol, int32_t max_iter, uint64_t seed,
                        int32_t* chosen, void* stream);

/* Fix a batch's launch: kernel (RESIDENT or TC), columns per CTA
 * (RESIDENT: 1, 2, 4, 8; TC: 4, 8) and threads (256 or 512).  Rebuilds the
 * work list; synchronous.
 * KZ_ERR_UNSUPPORTED if the combination does not fit shared memory or the
 * batch's method. */
kz_status kz_batch_set_launch(kz_batch* batch, kz_kernel kernel, int32_t rhs_per_cta, int32_t threads,
                              void* stream);

/* The launch a batch runs (host outputs, each may be NULL): kernel, columns
 * per CTA, threads, and the number of kernel launches one kz_precode_batched
 * issues (1, or 2 for a tensor-core batch split by shared memory). */
kz_status kz_batch_query(const kz_batch* batch, int32_t* kernel, int32_t* rhs_per_cta, int32_t* threads,
                         int32_t* launches);

/* Adjoint (implicit differentiation) of Q = (H H^H + xi I)^-1 S, X = H^H Q for
 * a real loss L.  Given the gradients G_Q (K x nrhs) and G_X (Nt x nrhs) of L
 * with respect to Q and X (PyTorch's convention for complex tensors: the
 * first-order change is dL = Re sum conj(G) dZ), it
 *   1. forms G~ = G_Q + H G_X,
 *   2. solves (H H^H + xi I) Lambda = G~ with the same Kaczmarz operator
 *      (VR-OAHK), giving Lambda (K x nrhs) and Y = H^H Lambda (written to y),
 *   3. contracts grad_H = Q G_X^H - Lambda X^H - Q Y^H on the VR entries only
 *      (packed like H_packed) and grad_xi = -Re sum conj(Lambda) Q.
 * Lambda is also dL/dS.  All pointers are device memory; grad_xi is one
 * float.  tol / max_iter / iters / resid / status as in kz_precode.  The
 * paper has no gradient; this follows from dA = dxi I + dH H^H + H dH^H. */
kz_status kz_precode_adjoint(kz_plan* plan, int32_t nrhs, float xi, const kz_cf32* Q,
                             const kz_cf32* X, const kz_cf32* G_Q, const kz_cf32* G_X, double tol,
                             int32_t max_iter, kz_cf32* lambda, kz_cf32* y, kz_cf32* grad_H_packed,
                             float* grad_xi, int32_t* iters, double* resid, int32_t* status,
                             void* stream);

/* The adjoint above without any device allocation.  The paper has no
 * counterpart; this entry exists for callers that cannot allocate device memory
 * when they differentiate: a real-time loop that must not block in the
 * driver's allocator, a process whose device memory is all reserved up front by
 * another allocator (so a cudaMalloc would fail), or a runtime that forbids
 * allocation after start-up.
 * kz_precode_adjoint keeps its right-hand side G~ (K x nrhs) in plan-owned
 * memory that it allocates on first use; this variant keeps G~ in one
 * file-scope device array of 262144 complex entries (2 MiB), which every GPU
 * that loads the library holds until the process exits.
 *   Arguments, outputs and errors are those of kz_precode_adjoint (the plan
 *   itself is created beforehand with kz_plan_create).  K * nrhs above 262144
 *   returns KZ_ERR_INVALID_ARG with a message; nothing is enqueued then.
 *   The first call on a device looks up the array's device address (with that
 *   device current) and caches it; make that first call before any stream
 *   capture.  cudaDeviceReset on a device invalidates the cached address:
 *   do not call this entry on that device again in the same process.
 *   Each device has its own copy of the array.  On one device all calls share
 *   it, and it keeps the last call's contents: calls that overlap on the GPU
 *   (through different streams, for example) race on it, so serialise them.
 *   Every entry of G~ the solve reads is written first, so nothing needs
 *   clearing. */
kz_status kz_precode_adjoint_noalloc(kz_plan* plan, int32_t nrhs, float xi, const kz_cf32* Q,
                                     const kz_cf32* X, const kz_cf32* G_Q, const kz_cf32* G_X,
                                     double tol, int32_t max_iter, kz_cf32* lambda, kz_cf32* y,
                                     kz_cf32* grad_H_packed, float* grad_xi, int32_t* iters,
                                     double* resid, int32_t* status, void* stream);

/* One channel of a batched adjoint (device pointers; layouts as in
 * kz_precode_adjoint). */
typedef struct {
    const kz_cf32* Q;        /* K x nrhs: the forward's v */
    const kz_cf32* X;        /* Nt x nrhs: the forward's x */
    const kz_cf32* G_Q;      /* K x nrhs gradient of the loss w.r.t. Q, or NULL */
    const kz_cf32* G_X;      /* Nt x nrhs gradient w.r.t. X, or NULL (not both) */
    kz_cf32* grad_H_packed;  /* sum vr_len: gradient w.r.t. the packed H */
    float* grad_xi;          /* one float: gradient w.r.t. xi */
} kz_adjoint_item;

/* kz_precode_adjoint for every channel of a batch at once (step A10 over
 * step A8): `batch` is prepared with algo VR_OAHK and C64, and its items'
 * s / x / v buffers receive G~ = G_Q + H G_X (written here), y = H^H Lambda
 * and Lambda; its xi are the forward's.  One kernel forms all right-hand
 * sides, one persistent launch solves all adjoint systems, two kernels form
 * all gradients.  items: host array of batch->n entries (copied on the
 * stream before return).  The first call allocates a small device table
 * owned by the batch. */
kz_status kz_precode_adjoint_batched(kz_batch* batch, const kz_adjoint_item* items, double tol,
                                     int32_t max_iter, int32_t* status, void* stream);

/* Precoder matrix from the auxiliary matrix V by the subarray-wise form
 * (Sec. IV-B, eq. (precoding2)): the array is cut into S subarrays of
 * consecutive antennas (subarray s = antennas [s Nt / S, (s + 1) Nt / S)),
 * Q_s is the set of users whose VR meets subarray s, and the rows of F on
 * subarray s are [H_s]_{Q_s} [V]_{Q_s}, i.e. F[n, :] = sum_{k in Q_s}
 * conj(H[k, n]) V[k, :] -- the product H^H V at O(Nt |Q| ncols) instead of
 * O(Nt K ncols).  V: device K x ncols column-major (the v of a solve with
 * identity right-hand sides gives the RZF precoder); F: device Nt x ncols
 * column-major (output).  normalise != 0: F is scaled by beta = 1 / ||F||_F
 * (eq. (power) with equality) and beta (device float) receives it; else F =
 * H^H V and beta may be NULL.  FP32 products and sums; the norm in FP64, in
 * a fixed order.  The plan caches Q_s for the last S used and a small partial
 * buffer (allocated on first use).  Asynchronous on `stream`. */
kz_status kz_precoder_matrix(kz_plan* plan, const kz_cf32* V, int32_t ncols, int32_t S, int32_t normalise,
                             kz_cf32* F, float* beta, void* stream);

/* The paper's computational complexity in FLOPs (Table I) for this plan:
 * scheme -1 is RZF; KZ_RK_UNIFORM (URK), KZ_RK_SWOR (SWOR-ERK), KZ_GK,
 * KZ_VR_OGRK and KZ_VR_OAHK are the table's other rows (the precoder-matrix
 * setup plus T times the per-iteration cost; T: the iteration count, e.g.
 * the mean of a solve's iters).  The table's per-user set sizes are means
 * over the plan's users: |Q| over S subarrays (as in kz_precoder_matrix),
 * |M| the VR length |Gamma_k| (the table's |M| in the VR rows is read as
 * |Gamma|), |X| the size of X_k without k, |F| and |V| the orthogonal set
 * and its complement.  Host only; KZ_ERR_UNSUPPORTED for a method the table
 * does not list. */
kz_status kz_plan_flops(const kz_plan* plan, int32_t scheme, int32_t S, double T, double* flops);

/* Per-user SINR and spectral efficiency of the precoder (eq. (rate)):
 * F = beta X with beta = 1 / ||X||_F (the power budget ||F||_F^2 <= 1 of
 * eq. (power) met with equality), SINR_k = |h_k^H f_k|^2 /
 * (sum_{i != k} |h_k^H f_i|^2 + 1 / snr_lin), rate = sum_k log2(1 + SINR_k).
 * X: device, Nt x K column-major (column k is user k's precoder: the x of a
 * solve with identity right-hand sides), 8-byte aligned; snr_lin = rho /
 * sigma^2 > 0; sinr: device double[K] or NULL; rate: device double or NULL
 * (not both NULL).  h_k^H f_i is summed in FP32 with compensated
 * cross-lane additions, every square and sum after that in FP64, in a fixed
 * order.  Asynchronous on `stream`. */
kz_status kz_sum_rate(const kz_plan* plan, const kz_cf32* X, double snr_lin, double* sinr, double* rate,
                      void* stream);

/* kz_sum_rate for every channel of a batch, one launch, on the items' x
 * buffers (the batch's column count must equal every item's K).  sinr:
 * device double[n * K_max], channel b's users at b * K_max (K_max = largest K
 * of the batch), or NULL; rate: device double[n] or NULL. */
kz_status kz_sum_rate_batched(const kz_batch* batch, double snr_lin, double* sinr, double* rate, void* stream);

/* One-line description of the last error on this thread ("" if none). */
const char* kz_last_error(void);

/* Library version, as major*10000 + minor*100 + patch. */
int32_t kz_version(void);

#ifdef __cplusplus
}
#endif

#endif /* KZPRECODE_H */
