/*
 * recon.h -- C ABI of the GB300 IRLS reconstruction of damped-exponential image series by
 * structured low-rank matrix completion (Balachandrasekaran, Magnotta, Jacob, arXiv 1704.04511).
 *
 * Problem (Sec. II-D, Eq. problem-formulation-relaxed, solved by Algorithm 1 of Sec. III):
 *     x* = argmin_x  ||T(F x)||_p  +  (1/lam) * ||A x - b||^2-style data term,
 * implemented as the IRLS alternation of Eq. x-update / Eq. weight-update:
 *     weight:  G = T^H T (Gram of the lifted matrix),  H = (G + eps I)^(p/2 - 1)
 *     x-step:  (A^H A + lam W_H) x = A^H b by a fixed number of CG steps, warm-started,
 * with x0 = A^H b, eps0 = eps0_frac * lambda_max(G(x0)), eps <- eps / gamma per iteration
 * (Sec. III-C).
 *
 * Conventions shared by every entry point:
 *  - Image series and k-space are [T][P][Q] arrays (Q fastest) of complex64 (interleaved
 *    float re, im). k-space may instead be bfloat16 pairs (kspace_bf16 = 1).
 *  - F is the unitary 2-D DFT per frame, forward sign e^{-2 pi i}, natural frequency order
 *    (DC at index 0, no fftshift). A = mask * F per frame (one coil, Eq. measurement-ij).
 *  - Masks are [T][P][Q] uint8, nonzero = sampled (treated as exactly 1).
 *  - Filter support N1 x N2 spatial taps x M frame taps (s = N1 N2 M columns of the lifted
 *    matrix; column index a = (m N1 + l1) N2 + l2). The lifting is circular in space and a valid
 *    linear convolution over frames (the hybrid approximation of Sec. III-A), k = T - M + 1.
 *  - Every data pointer is a DEVICE pointer on the context's device unless stated otherwise,
 *    owned by the caller, and must stay valid until the call returns. Calls are synchronous:
 *    they return after the device work finished (results readable). Image, k-space, mask,
 *    coil, S and G arrays start on a 16-byte boundary (every cudaMalloc / PyTorch allocation
 *    does; a view starting at an odd complex64 element does not): RECON_EINVAL otherwise.
 *  - Supported sizes: P, Q in {16, 32, 64, 128, 192, 256, 512}; 1 <= M <= 6, M <= T;
 *    1 <= N1 <= P, 1 <= N2 <= Q; T * Q <= 8533 (fused row/W pass).
 *  - Return value: RECON_OK (0) or a negative RECON_E* code; recon_last_error() describes it.
 *    A failed call never reports partial output as valid.
 */
#ifndef RECON_H
#define RECON_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RECON_OK 0
#define RECON_EINVAL (-1)   /* bad dims / filter / parameters / null pointer            */
#define RECON_ENOMEM (-2)   /* request exceeds the context budget or allocation failed  */
#define RECON_ECUDA (-3)    /* CUDA runtime or library error                            */
#define RECON_ENUMERIC (-4) /* NaN / Inf in the iteration, or eigensolver failure       */
#define RECON_ETIMEOUT (-5) /* a bounded device-wide wait (grid barrier) gave up         */
#define RECON_EBUSY (-6)    /* serving: no free request slot or workspace budget; retry  */

/* How the weight H = (G + eps I)^(p/2-1) is formed (recon_params.weight_method):
 * RECON_WEIGHT_AUTO: p = 0 -> FP64 Hermitian sweep inverse (G + eps I)^-1 and a Lanczos
 *                    lambda_max for eps0; p > 0 -> FP64 eigendecomposition.
 * RECON_WEIGHT_EIG:  always the FP64 eigendecomposition (cuSOLVER zheevd). */
#define RECON_WEIGHT_AUTO 0
#define RECON_WEIGHT_EIG 1

typedef struct recon_ctx recon_ctx;

typedef struct {
    int P, Q, T; /* grid P x Q (Q fastest), T frames */
} recon_dims;

typedef struct {
    int N1, N2, M; /* filter support: N1 x N2 spatial taps, M frame taps */
} recon_filter;

typedef struct {
    int irls;         /* IRLS iterations (Algorithm 1 outer loop), >= 0            */
    int cg;           /* CG steps per IRLS iteration (Algorithm 1, step 2), >= 1   */
    double lambda;    /* weight of the structured penalty, > 0                     */
    double p;         /* Schatten-p exponent, 0 <= p <= 1 (Eq. problem-formulation-relaxed) */
    double gamma;     /* eps decay factor, > 1 (Sec. III-C uses 1.4)               */
    double eps0_frac; /* eps0 = eps0_frac * lambda_max(G(x0)) (Sec. III-C uses 0.01) */
    int kspace_bf16;  /* 1: kspace holds bfloat16 (re, im) pairs; 0: complex64      */
    int weight_method; /* RECON_WEIGHT_AUTO or RECON_WEIGHT_EIG                      */
} recon_params;

/* Create a context on `device`. It owns device workspace (grown on demand, never beyond
 * mem_budget_bytes; 0 = no limit), the twiddle tables and an eigensolver handle, and issues all
 * work on `cuda_stream` (a cudaStream_t; NULL = a stream the context creates). One context must
 * not be used by two host threads at once. Returns RECON_OK and sets *out, or an error code. */
int recon_create(recon_ctx** out, int device, size_t mem_budget_bytes, void* cuda_stream);

/* Release the context and all its device memory. NULL is ignored. */
void recon_destroy(recon_ctx* c);

/* Description of the last error on this context (static storage; never NULL). */
const char* recon_last_error(const recon_ctx* c);

/* Device bytes of workspace recon_solve needs for this problem (the admission formula). */
size_t recon_bytes_needed(recon_dims d, recon_filter f, int kspace_bf16);

/* Full reconstruction, Algorithm 1 (Sec. III): x0 = A^H b, then prm->irls iterations of
 * [Gram (Eq. P-ij-modified) -> FP64 eigendecomposition -> weight (Eq. weight-update) ->
 * per-pixel S(r) -> prm->cg CG steps on Eq. grad-ls]. kspace: [T][P][Q] complex64 or bf16
 * pairs; masks: [T][P][Q] uint8; image_out: [T][P][Q] complex64, receives x. */
int recon_solve(recon_ctx* c, recon_dims d, const void* kspace, const uint8_t* masks,
                recon_filter f, const recon_params* prm, void* image_out);

/* Batched reconstruction: n independent problems of the same dims, filter and parameters
 * (slot i reads kspace[i] and masks[i] and writes image_out[i], all device pointers), each
 * solved exactly as recon_solve would, concurrently on n streams of the context, each with its
 * own workspace (the budget covers all slots). IRLS iterations are issued interleaved across
 * the slots, so that the latency-bound phases of one problem (FP64 weight, small reductions)
 * overlap with the others' work. Results are bitwise identical to solving each problem alone
 * (fixed launch shapes and reduction orders). 1 <= n <= RECON_MAX_BATCH; synchronous. */
#define RECON_MAX_BATCH 16
int recon_solve_batch(recon_ctx* c, int n, recon_dims d, const void* const* kspace,
                      const uint8_t* const* masks, recon_filter f, const recon_params* prm,
                      void* const* image_out);

/* recon_solve_batch with the problems in host memory: kspace[i], masks[i] and image_out[i] are
 * host pointers (same layouts and types as recon_solve_batch). Slot i copies its k-space and
 * masks into device buffers of its own workspace on its own stream, solves, and copies its image
 * back, so that the copies of one slot overlap the other slots' solves: with page-locked host
 * memory (cudaHostAlloc, or a pinned torch tensor) the copies run asynchronously; pageable memory
 * works but its copies do not overlap. Each slot's workspace grows by (8 or 4) T P Q + T P Q +
 * 8 T P Q bytes (k-space, masks, image) on top of recon_bytes_needed. Results are bitwise those of
 * recon_solve_batch on the same inputs. The call returns when every image_out[i] holds its
 * result; on an error nothing queued is still running. 1 <= n <= RECON_MAX_BATCH. */
int recon_solve_batch_host(recon_ctx* c, int n, recon_dims d, const void* const* kspace,
                           const uint8_t* const* masks, recon_filter f, const recon_params* prm,
                           void* const* image_out);

/* Batched reconstruction of uneven problems: problem i has its own dims d[i] and filter f[i]
 * (grid, frame count and filter support may all differ; the parameters prm are shared), slot i
 * reading kspace[i], masks[i] and writing image_out[i]. Run as recon_solve_batch runs its slots:
 * independent slots by default; with RECON_OPT_BATCH_GROUP = g the whole batch is one CUDA graph
 * and every g consecutive slots share one Lanczos, one eps and one FP64 sweep launch per IRLS
 * iteration, each matrix of its own size s_i = N1 N2 M (the sweep runs as many pivot steps as
 * the largest needs). Results are bitwise identical to solving each problem alone.
 * 1 <= n <= RECON_MAX_BATCH; synchronous. */
int recon_solve_many(recon_ctx* c, int n, const recon_dims* d, const recon_filter* f,
                     const void* const* kspace, const uint8_t* const* masks,
                     const recon_params* prm, void* const* image_out);

/* ---- serving: asynchronous requests (continuous batching) ----
 * recon_submit queues one reconstruction (arguments as recon_solve; buffers must stay valid
 * until the request completes) on a free request slot -- its own stream and workspace -- and
 * returns at once with a ticket. Requests in flight overlap on the device; a new one can be
 * submitted whenever a slot is free and its workspace (recon_bytes_needed) fits the context's
 * budget next to the requests in flight (idle slots return their cached workspace first).
 * Otherwise RECON_EBUSY: poll and retry. Up to RECON_MAX_BATCH requests in flight. Results are
 * bitwise identical to recon_solve of the same request. Not for use from several host threads
 * at once (like every call on one context). */
int recon_submit(recon_ctx* c, recon_dims d, const void* kspace, const uint8_t* masks,
                 recon_filter f, const recon_params* prm, void* image_out, int* ticket);
/* Non-blocking completion check: *done = 0 while the request runs; once it finished, *done = 1,
 * the ticket is released and the return value is the request's own status (RECON_OK or the
 * error recon_solve would have returned). */
int recon_poll(recon_ctx* c, int ticket, int* done);

/* Context options (value 0 = off, 1 = on unless stated):
 * RECON_OPT_GRAPHS: recon_solve and recon_solve_batch capture a whole solve (every launch of
 *   Algorithm 1) into a CUDA graph on first use and replay it while the shapes, parameters,
 *   buffer pointers and workspace stay the same (one graph per slot). Not used for the
 *   eigensolver-library path or while launch classes are timed.
 * RECON_OPT_AUTOTUNE: on the first solve of each shape (P, Q, T, R, coils) the context times the
 *   column passes of the CG operator with tiles of 8, 16 and 32 columns (CUDA events on its own
 *   stream, a few milliseconds at most) and keeps the fastest; off = the built-in widths. The
 *   width changes launch shapes only: results are bitwise the same either way.
 * Option numbers 2 and 4 are retired (a cluster operator for square frames and a three-pass CG
 *   step, both measured slower than the four-pass step): setting them gives RECON_EINVAL. */
#define RECON_OPT_GRAPHS 1      /* default on  */
#define RECON_OPT_AUTOTUNE 3    /* default on  */
/* RECON_OPT_INJECT_BARRIER_FAULT (testing): the next solve on this context that forms its weight
 *   by the FP64 sweep (p = 0, RECON_WEIGHT_AUTO) starts with the error word of the sweep's grid
 *   barrier set from the host, as a CTA whose bounded wait gave up would leave it; every sweep of that solve returns at its first barrier and reports it, the
 *   solve returns RECON_ETIMEOUT and re-arms the barrier, and the following solve runs normally.
 *   One-shot (cleared when used). No kernel waits, traps or faults for it. */
#define RECON_OPT_INJECT_BARRIER_FAULT 5
/* RECON_OPT_TEST_WITHHOLD_ARRIVAL (testing): in the next solve on this context that forms its
 *   weight by the FP64 sweep (p = 0, RECON_WEIGHT_AUTO), CTA 1 of every Lanczos and sweep launch
 *   leaves at its first grid barrier without arriving, as a lost CTA would, and the bounded waits
 *   of the other CTAs give up after 4096 polls (about a millisecond) instead of the default limit
 *   of seconds. The waits run out for real: the kernels record the failure and return, the solve
 *   returns RECON_ETIMEOUT and re-arms the barriers, and the following solve runs normally. That
 *   solve is issued as direct launches (no graph). One-shot (cleared when used). */
#define RECON_OPT_TEST_WITHHOLD_ARRIVAL 6
/* RECON_OPT_BATCH_GROUP (value g, 0 <= g <= RECON_MAX_BATCH; default 0): how recon_solve_batch runs
 *   the FP64 weight of its solves on the sweep path (p = 0, RECON_WEIGHT_AUTO, graphs on).
 *   0: every solve has its own graph and stream, its weight launches its own (independent slots).
 *   g >= 1: the whole batch is one CUDA graph; every IRLS iteration the solves of each group of g
 *   consecutive slots join for ONE Lanczos (first iteration), one eps and ONE sweep launch that
 *   serve all of them (one grid barrier per pivot step for the group), then continue on their
 *   own streams; with several groups the groups' weight launches take turns, so each overlaps
 *   the other groups' CG. Results are bitwise identical to solving each problem alone. */
#define RECON_OPT_BATCH_GROUP 7
/* RECON_OPT_AUTOTUNE_FFT (default off): with RECON_OPT_AUTOTUNE on, the autotuner also picks the
 *   radix schedule of the column passes' Stockham transforms (lengths other than the register
 *   transforms' 128 and 256): schedule 0 takes radix 8 whenever the remaining length allows
 *   (fewest passes), schedule 1 takes radix 4 before 8 (more passes, fewer registers per
 *   butterfly). Each (tile width, schedule) pair is timed on the first solve of a shape. Unlike
 *   the tile width, the schedule changes the order of the FP32 operations, so results move at
 *   the FP32 rounding level with the choice (each schedule is parity-tested against the FP64
 *   reference); a cache file (recon_tile_cache) makes the choice reproducible.
 * RECON_OPT_FFT_SCHEDULE (testing; default -1): -1 uses the tuned (or default) schedule, 0 or 1
 *   forces that schedule on the column passes of the CG operator. */
#define RECON_OPT_AUTOTUNE_FFT 8
#define RECON_OPT_FFT_SCHEDULE 9
int recon_set_option(recon_ctx* c, int option, int value);


/* ---- stage entry points (the same kernels recon_solve runs; used for parity checks) ---- */

/* x = A^H b = F^H (mask * b) (Sec. II-A). */
int recon_adjoint(recon_ctx* c, recon_dims d, const void* kspace, int kspace_bf16,
                  const uint8_t* masks, void* x_out);

/* y = F x (inverse = 0) or F^H x (inverse = 1), every frame; x and y complex64 [T][P][Q];
 * y may equal x. */
int recon_fft2(recon_ctx* c, recon_dims d, const void* x, void* y, int inverse);

/* Gram matrix of the lifted matrix of F x (Sec. III-B, Eq. block-expression-for-R,
 * Eq. P-ij-modified): G_out, s x s complex128 column-major (both triangles written);
 * lags_out (may be NULL): npair x (2N1-1) x (2N2-1) complex128, pair (a <= b) at index
 * a(2M-a+1)/2 + (b-a), lag (d1, d2) at offset (N1-1, N2-1):
 * lag_ab[d] = sum_r sum_{j<k} conj(x_{j+M-1-a}(r)) x_{j+M-1-b}(r) e^{-2 pi i (d1 r1/P + d2 r2/Q)}.
 * G is exactly Hermitian: lag_aa[-d] is written as conj(lag_aa[d]) and lag_aa[0] is real. */
int recon_gram(recon_ctx* c, recon_dims d, recon_filter f, const void* x, void* G_out,
               void* lags_out);

/* Weight step (Sec. III-B, Eq. weight-update) on G_in (s x s complex128, column-major,
 * Hermitian positive semi-definite; not modified; the inverse and the eigendecomposition read its
 * lower triangle, the diagonal as real), all in FP64:
 * H = (G + eps I)^(p/2-1) -- by the eigendecomposition H = U diag((lambda+eps)^(p/2-1)) U^H, or
 * for p = 0 with method RECON_WEIGHT_AUTO by the Hermitian sweep inverse (G + eps I)^-1 --,
 * then the summed diagonals d_ab[delta] = sum_{l-l'=delta} H[(l',b),(l,a)] and the per-pixel
 * weight S_ab(r) = sum_delta d_ab[delta] e^{-2 pi i (delta.r)}.
 * eps: if eps_in >= 0 it is used; else eps = -eps_in * lambda_max(G) (so -0.01 gives the
 * Sec. III-C initial value). S_out: npair x P x Q complex64 (pair layout as above);
 * dsum_out (may be NULL): npair x (2N1-1) x (2N2-1) complex128; evals_out (may be NULL; only
 * with the eigendecomposition): s doubles ascending; eps_out (host pointer, may be NULL)
 * receives the eps used. */
int recon_weight(recon_ctx* c, recon_dims d, recon_filter f, const void* G_in, double eps_in,
                 double p, int method, void* S_out, void* dsum_out, void* evals_out,
                 double* eps_out);

/* y = (A^H A + lambda W_S) x with W_S the per-pixel banded frame operator of Eq. grad-ls:
 * (W x)_n(r) = sum_{a: 0 <= n-M+1+a < k} sum_b S_ab(r) x_{n+a-b}(r). S as from recon_weight.
 * lambda = 0 gives A^H A x. y must not alias x. */
int recon_apply_normal(recon_ctx* c, recon_dims d, recon_filter f, const uint8_t* masks,
                       const void* S, double lambda, const void* x, void* y);

/* y = W_S x (no lambda, no data term). y must not alias x. */
int recon_apply_w(recon_ctx* c, recon_dims d, recon_filter f, const void* S, const void* x,
                  void* y);

/* One least-squares step of Algorithm 1 as recon_solve runs it: residual carry
 * r <- (S_old == NULL ? 0 : r) + lambda W_{S_old - S_new} x   (S_old == NULL: r = -lambda W x,
 * valid when x = A^H b), then n_cg CG steps on (A^H A + lambda W_{S_new}) with x, r updated in
 * place. rr_hist (host, may be NULL) receives n_cg + 1 values |r_c|^2. */
int recon_cg(recon_ctx* c, recon_dims d, recon_filter f, const uint8_t* masks,
             const void* S_old, const void* S_new, double lambda, void* x, void* r, int n_cg,
             double* rr_hist);

/* ---- Gram matrix without device allocation ----
 *
 * Some callers may not allocate device memory once they are running: a reconstruction service
 * whose device memory is planned when it starts and must not grow, or a program that shares the
 * GPU with other streams and cannot accept the device-wide synchronisation that cudaMalloc and
 * cudaFree can cause. recon_gram_static gives them the same Gram matrix and lags as recon_gram
 * (same kernels) without a context: its scratch (per-row pruned DFTs and twiddle tables)
 * lives in one fixed device array of RECON_GRAM_STATIC_BYTES inside the library, which every
 * GPU that loads the library holds until the process exits. The paper has no counterpart; this
 * is a deployment aid, not part of the method.
 *  - Arguments as for recon_gram, plus cuda_stream (a cudaStream_t; NULL = the default stream);
 *    x, G_out, lags_out are device pointers on the current device. The call is synchronous.
 *  - The first call on each device is a warm-up. With the device current it looks up the array's
 *    device address (cudaGetSymbolAddress) and caches it for that device's context. Under CUDA's
 *    lazy module loading (the default since CUDA 12.2) this first call is also what loads the
 *    library's Gram code on that device and commits the RECON_GRAM_STATIC_BYTES array, which can
 *    allocate device memory and synchronise the device. Make it once at start-up, before any
 *    stream capture; only the calls after it allocate nothing. After a device reset
 *    (cudaDeviceReset, a new primary context) the next call is a first call again: the cached
 *    address belongs to the old context and is looked up anew.
 *  - A problem whose scratch exceeds RECON_GRAM_STATIC_BYTES is rejected with RECON_EINVAL and a
 *    message naming the bytes it needs (recon_last_error(NULL)); use recon_gram for it. The
 *    256x256x16 series with a 9x9x3 filter needs about 0.42 MB.
 *  - Every call uses the same array and it keeps the last call's contents; each call writes
 *    everything it reads first. Calls that overlap on the GPU (other host threads or streams)
 *    race on the array and must be serialised by the caller.
 *  - After the warm-up call, allocates no device memory (no cudaMalloc / cudaFree or allocating
 *    library call). */
#define RECON_GRAM_STATIC_BYTES (4u * 1024u * 1024u)
int recon_gram_static(recon_dims d, recon_filter f, const void* x, void* G_out, void* lags_out,
                      void* cuda_stream);

/* ---- multi-coil measurements (Eq. measurement-ij with receiver sensitivities) ----
 * b[c][n] = mask_n * F (C_c * x_n) + noise for coils c < n_coils: the paper's S_i F C_j F^* acting
 * on the k-space of frame i is the multiplication of the image by C_j. A^H b =
 * sum_c conj(C_c) F^H (mask_n b[c][n]); the normal operator of the least-squares step becomes
 * sum_c conj(C_c) F^H mask F (C_c x) + lambda W x. Layouts (all device, caller-owned):
 *  - kspace: coil-major [n_coils][T][P][Q] complex64 (bf16 storage is not offered here);
 *  - coils: [n_coils][P][Q] complex64 sensitivities (any normalisation; the tests use
 *    sum_c |C_c|^2 = 1);
 *  - masks, x, image_out: as for the single-coil calls ([T][P][Q]).
 * The workspace holds n_coils transform series (8 n_coils T P Q bytes) instead of one, on top of
 * recon_bytes_needed; serving (recon_submit) is single-coil. */
#define RECON_MAX_COILS 64
int recon_solve_coils(recon_ctx* c, recon_dims d, const void* kspace, const uint8_t* masks,
                      const void* coils, int n_coils, recon_filter f, const recon_params* prm,
                      void* image_out);
/* x = A^H b with coils. */
int recon_adjoint_coils(recon_ctx* c, recon_dims d, const void* kspace, const uint8_t* masks,
                        const void* coils, int n_coils, void* x_out);
/* y = (A^H A + lambda W) x with coils; S as for recon_apply_normal. */
int recon_apply_normal_coils(recon_ctx* c, recon_dims d, recon_filter f, const uint8_t* masks,
                             const void* coils, int n_coils, const void* S, double lambda,
                             const void* x, void* y);

/* Mono-exponential T2 map of a recovered series (Sec. IV-A: the paper fits a mono-exponential
 * model to every pixel of the reconstructed series for its T2 maps). Over the foreground pixels
 * |x_0(r)| > fg_frac * max |x_0|: |x_n(r)| ~ A(r) exp(-t_n / T2(r)), log-linear least squares for
 * the start, then n_gn Gauss-Newton steps on the un-logged residual, 1/T2 >= 1e-4 per ms; FP32.
 * The foreground test is computed in FP32 with separately rounded operations (reproducible on a
 * host in FP32).
 *  - x: device [T][P][Q] complex64 (e.g. recon_solve's output), 2 <= T <= 64.
 *  - times_ms: HOST array of the T echo times in ms, read during the call.
 *  - t2_out: device [P][Q] float32, T2 in ms, NaN outside the foreground; amp_out: device
 *    [P][Q] float32 amplitude A, or NULL.
 *  - 0 <= fg_frac < 1, 0 <= n_gn <= 1000, else RECON_EINVAL. Synchronous. */
int recon_t2fit(recon_ctx* c, recon_dims d, const void* x, const double* times_ms, double fg_frac,
                int n_gn, float* t2_out, float* amp_out);

/* ---- image volumes ----
 * The method on series of 3-D volumes: the signal model of Sec. II-B holds per voxel, and the
 * lifting of Sec. III-A gains a third spatial axis, circular like the other two. The paper
 * builds the lifting for P x Q frames (a 3-D k-t dataset, Sec. II-C) and motivates its FFT
 * approximations by larger multidimensional problems (Sec. I); these calls carry the same
 * formulas along one more spatial axis. Conventions as above, except:
 *  - series, k-space and masks are [T][R][P][Q] (Q fastest): T volumes of R slices of P x Q;
 *  - F is the unitary 3-D DFT of each volume (sign e^{-2 pi i}, natural order); A = mask * F;
 *  - the filter has N1 x N2 x N3 spatial taps (rows, columns, depth) x M frame taps,
 *    s = N1 N2 N3 M, column index ((m N3 + l3) N1 + l1) N2 + l2;
 *  - lags and summed diagonals are npair x (2N3-1) x (2N1-1) x (2N2-1) complex128 (lag (d3, d1,
 *    d2) at offset (N3-1, N1-1, N2-1)), with the extra factor e^{-2 pi i d3 r3 / R};
 *  - S is npair x R x P x Q complex64;
 *  - R = 1 or R in {16, 32, 64, 128, 192, 256, 512}; 1 <= N3 <= R. With R = N3 = 1 every call
 *    computes what its 2-D counterpart does.
 * Single coil; no batched or serving form. */
typedef struct {
    int P, Q, R, T; /* volume R x P x Q (Q fastest), T frames */
} recon_dims3;

typedef struct {
    int N1, N2, N3, M; /* N1 x N2 x N3 spatial taps (rows, columns, depth), M frame taps */
} recon_filter3;

size_t recon_bytes_needed3(recon_dims3 d, recon_filter3 f, int kspace_bf16);
/* Algorithm 1 on volumes (as recon_solve). */
int recon_solve3(recon_ctx* c, recon_dims3 d, const void* kspace, const uint8_t* masks,
                 recon_filter3 f, const recon_params* prm, void* image_out);
/* x = A^H b = F^H (mask * b), 3-D. */
int recon_adjoint3(recon_ctx* c, recon_dims3 d, const void* kspace, int kspace_bf16,
                   const uint8_t* masks, void* x_out);
/* y = F x or F^H x (unitary 3-D DFT per volume); y may equal x. */
int recon_fft3(recon_ctx* c, recon_dims3 d, const void* x, void* y, int inverse);
/* Gram matrix and lags of the 3-D lifting (as recon_gram). */
int recon_gram3(recon_ctx* c, recon_dims3 d, recon_filter3 f, const void* x, void* G_out,
                void* lags_out);
/* Weight step (as recon_weight), S_out npair x R x P x Q. */
int recon_weight3(recon_ctx* c, recon_dims3 d, recon_filter3 f, const void* G_in, double eps_in,
                  double p, int method, void* S_out, void* dsum_out, void* evals_out,
                  double* eps_out);
/* y = (A^H A + lambda W_S) x on volumes (W_S per voxel, as recon_apply_normal). */
int recon_apply_normal3(recon_ctx* c, recon_dims3 d, recon_filter3 f, const uint8_t* masks,
                        const void* S, double lambda, const void* x, void* y);

/* ---- comparison methods (Sec. IV) ----
 * The methods the paper compares against, on the same forward model and parameters as
 * recon_solve, for reproducing its qualitative comparison on synthetic data:
 *  RECON_VARIANT_PROPOSED   the method of recon_solve;
 *  RECON_VARIANT_GIRAF      the lifting circular along the frames as well (the GIRAF
 *                           approximation, Sec. III-A): T windows, window j taking frames
 *                           (j + M - 1 - m) mod T; Gram, weight and W otherwise as proposed;
 *  RECON_VARIANT_HLR_VOXEL  the pixel-wise Toeplitz prior (Sec. II-D, Eq. MORASA-objective):
 *                           per pixel r the k x M matrix T_r[j][m] = x_{j+M-1-m}(r) (image
 *                           domain), its Gram G_r and weight H_r = (G_r + eps_r I)^(p/2-1) (FP64
 *                           Jacobi eigendecomposition per pixel), eps_r^(0) = eps0_frac *
 *                           lambda_max(G_r(x0)), eps_r <- eps_r / gamma; W uses S(r) = H_r^T.
 *                           The filter must have N1 = N2 = 1;
 *  RECON_VARIANT_DIRECT     IRLS without the FFT approximations (Sec. IV-A): the exact multi-fold
 *                           Toeplitz matrix, valid in space and time, (T-M+1)(P-N1+1)(Q-N2+1) x s,
 *                           of the centred k-space C F x (C moves DC to (P/2, Q/2); the valid
 *                           lifting is not shift invariant and the grid of Sec. II-B is centred
 *                           on k = 0), formed explicitly (complex128 for its Gram, a library Hermitian
 *                           rank-k product; complex64 for the CG, a library GEMM per step); the
 *                           workspace holds (T-M+1)(P-N1+1)(Q-N2+1) s 16 bytes for it. */
#define RECON_VARIANT_PROPOSED 0
#define RECON_VARIANT_GIRAF 1
#define RECON_VARIANT_HLR_VOXEL 2
#define RECON_VARIANT_DIRECT 3
/* Algorithm 1 with the chosen variant (arguments as recon_solve). */
int recon_solve_variant(recon_ctx* c, recon_dims d, const void* kspace, const uint8_t* masks,
                        recon_filter f, const recon_params* prm, int variant, void* image_out);
/* Gram of the variant's lifting of F x: PROPOSED / GIRAF / DIRECT: s x s complex128 column-major;
 * HLR_VOXEL: the per-pixel Grams G_r, [P][Q][M][M] complex128 (row-major M x M). */
int recon_gram_variant(recon_ctx* c, recon_dims d, recon_filter f, int variant, const void* x,
                       void* G_out);
/* HLR-Voxel weight of x: per pixel G_r, its FP64 eigendecomposition, H_r with eps[r] (device
 * [P][Q] doubles, > 0) and S(r) = H_r^T into S_out (npair x P x Q complex64, the pair layout of
 * recon_weight); lmax_out (device [P][Q] doubles, may be NULL) receives lambda_max(G_r). */
int recon_voxel_weight(recon_ctx* c, recon_dims d, int M, const void* x, const double* eps,
                       double p, void* S_out, double* lmax_out);
/* IRLS-direct weight: H = (G + eps I)^(p/2-1) as a full s x s complex128 column-major matrix
 * (eps as in recon_weight; the FP64 sweep inverse for p = 0 with RECON_WEIGHT_AUTO, else the
 * eigendecomposition). */
int recon_weight_direct(recon_ctx* c, recon_dims d, recon_filter f, const void* G_in,
                        double eps_in, double p, int method, void* H_out, double* eps_out);
/* y = (A^H A + lambda W) x of the variant: W is S (npair x P x Q complex64) for PROPOSED, GIRAF and
 * HLR_VOXEL, and H (s x s complex128 column-major) for DIRECT, where
 * W x = F^H C^H T^*(T(C F x) H). */
int recon_apply_normal_variant(recon_ctx* c, recon_dims d, recon_filter f, int variant,
                               const uint8_t* masks, const void* W, double lambda, const void* x,
                               void* y);

/* ---- autotuner (RECON_OPT_AUTOTUNE) ----
 * Autotuner cache file: reads the choices stored in `path` (lines "P Q T R coils colC depthC
 * [colS depthS]"; a missing file is an empty cache) into the context and appends every new
 * choice to it. NULL stops appending. RECON_EINVAL on a malformed entry. */
int recon_tile_cache(recon_ctx* c, const char* path);
/* The tile widths the context uses for a shape (R = 1 for image series; 0 = not tuned yet). */
int recon_tile_choice(recon_ctx* c, recon_dims3 d, int n_coils, int* colC, int* depthC);
/* The radix schedules (0 or 1) of the length-P and depth column passes the context uses for a
 * shape; -1 = not tuned yet. Cache lines carry them as two more fields ("... colC depthC colS
 * depthS"); lines without them mean schedule 0. */
int recon_fft_schedule_choice(recon_ctx* c, recon_dims3 d, int n_coils, int* colS, int* depthS);

/* ---- measurement ---- */

/* Launch classes timed by recon_profile (one pair of CUDA events on the context's stream around
 * every launch of the class; the eigensolver class brackets the whole library call). */
#define RECON_PROF_ADJOINT 0      /* x0 = A^H b: column + row pass                       */
#define RECON_PROF_GRAM 1         /* Gram lags + fill of G                                */
#define RECON_PROF_EIG 2          /* FP64 eigendecomposition (cuSOLVER zheevd)            */
#define RECON_PROF_EPS 3          /* eps schedule                                         */
#define RECON_PROF_DIAG 4         /* summed diagonals of H (FP64)                         */
#define RECON_PROF_S 5            /* per-pixel S(r)                                       */
#define RECON_PROF_RESID 6        /* residual carry between IRLS iterations               */
#define RECON_PROF_CG_ROWFWD 7    /* CG pass A: p update + row FFT                        */
#define RECON_PROF_CG_COL 8       /* CG pass B: column FFT, mask, column IFFT             */
#define RECON_PROF_CG_ROWINVW 9   /* CG pass C: row IFFT + lambda W p + <p, q> partials    */
#define RECON_PROF_CG_UPDATE 10   /* CG pass D: x, r update + |r|^2 partials               */
#define RECON_PROF_LANCZOS 11     /* lambda_max of G for eps0 (p = 0 path)                 */
#define RECON_PROF_INV 12         /* FP64 sweep inverse (G + eps I)^-1 (p = 0 path)        */
#define RECON_PROF_KINDS 13

#define RECON_PROF_ALL ((1u << RECON_PROF_KINDS) - 1u)

/* Time the launch classes whose bit (1u << kind) is set in kind_mask (0 = off,
 * RECON_PROF_ALL = every class); resets the totals. Only the selected classes pay for the event
 * records. */
int recon_profile(recon_ctx* c, unsigned int kind_mask);
/* Total device milliseconds and launch count of one class since the last recon_profile call
 * (waits for the recorded events). */
int recon_profile_read(recon_ctx* c, int kind, double* total_ms, long long* launches);
/* Name of a launch class ("" if out of range). */
const char* recon_profile_name(int kind);

#ifdef __cplusplus
}
#endif

#endif /* RECON_H */
