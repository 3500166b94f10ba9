// Internal launch interface between the C-ABI layer (recon.cu) and the kernel files.
// Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>

namespace recon {

// Most matrices (solves) one batched weight launch serves.
constexpr int kMaxHpdBatch = 16;

// Geometry of one problem: image series [T][P][Q] complex64 (or volumes [T][R][P][Q] when
// R > 1), filter N1 x N2 (x N3) x M taps. A volume is laid out as R * P image rows of length Q,
// so the row passes, the pixel-wise W and the CG vectors see rows() = R * P rows.
struct Dims {
    int T, P, Q;
    int N1, N2, M;
    int nc = 1;  // receiver coils (Eq. measurement-ij); the transform buffer holds nc series
    int R = 1;   // depth of a volume (third spatial axis, circular like the other two)
    int N3 = 1;  // filter taps along the depth
    int circ = 0;  // 1: lifting circular in time as well (the fully circulant GIRAF form)
    int colC = 0, depthC = 0;  // column tiles of the column / depth passes (0 = default)
    int colS = 0, depthS = 0;  // radix schedules of their Stockham passes (fft_radix_at)
    int k() const { return circ ? T : T - M + 1; }
    int npair() const { return M * (M + 1) / 2; }
    int L1() const { return 2 * N1 - 1; }
    int L2() const { return 2 * N2 - 1; }
    int L3() const { return 2 * N3 - 1; }
    int s() const { return N1 * N2 * N3 * M; }
    int rows() const { return R * P; }
    size_t nlag() const { return (size_t)npair() * L1() * L2() * L3(); }
    size_t pixels() const { return (size_t)R * P * Q; }
    size_t elems() const { return (size_t)T * R * P * Q; }
};

// Twiddle tables e^{-2 pi i j / n}, j < n, for the grid lengths (device memory).
struct Twiddles {
    const float2* twP;   // length P, FP32
    const float2* twQ;   // length Q, FP32
    const double2* twPd; // length P, FP64
    const double2* twQd; // length Q, FP64
    const float2* twR = nullptr;   // length R (volumes), FP32
    const double2* twRd = nullptr; // length R (volumes), FP64
};

// Grid-wide deterministic reduction slot: one partial per block, finished by the last block.
// `counter` must be zero before the first use; each reduction leaves it zero again.
struct RedSlot {
    double* parts;          // max_parts() doubles
    unsigned int* counter;  // one word
};

// Per-CTA partial sums of one grid-wide dot product, left by the producing kernel for its
// consumers to add up (sum_partials: fixed order, so every consumer gets the same value).
struct Partials {
    double* parts;  // max_parts() doubles
    int n;          // partials written (the producer's grid), set by the producer's launcher
};

// Launch `kern` with programmatic stream serialization (see pdl_wait in common.cuh).
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// SM count of the current device (cached per device).
int num_sms();

bool fft_size_supported(int n);
// Column tile the length-P (depth = false) or depth passes of `d` use (fft.cu).
int col_tile_for(const Dims& d, bool depth);
// Radix schedule of those passes' Stockham transforms (0 or 1, see fft_radix_at).
int col_sched_for(const Dims& d, bool depth);
constexpr int kFftSchedules = 2;
// True where the column stage of the CG operator runs register transforms without tiles.
bool col_register(const Dims& d, bool depth);
// True for volumes of 128 x 128 slices and depth 64 (single coil): the row pass of a CG step also
// runs the first half of the length-P DFT and the column stage is two launches (fft.cu).
bool vol_fold(const Dims& d);
// Message returned by recon_last_error(NULL) (calls that have no context).
void set_context_free_error(const std::string& msg);
int w_max_M();
int w_max_frames_times_q();  // bound on T * Q for the fused row/W kernel

// ---- fft.cu ----
// t = F^H (mask * b) / sqrt(PQ) (adjoint, Sec. II-A); b may be complex64 or bf16 pairs.
cudaError_t launch_adjoint(const Dims& d, const Twiddles& tw, const void* b, int b_bf16,
                           const uint8_t* mask, float2* t, float2* x, cudaStream_t st);
// y = unitary forward (inv = 0) or inverse (inv = 1) 2-D DFT of every frame of x (in place ok)
cudaError_t launch_fft2(const Dims& d, const Twiddles& tw, const float2* x, float2* y, int inv,
                        cudaStream_t st);
// CG step, pass A: p = r (first) or r + beta p with beta = |r|^2 / *rr_prev, |r|^2 the sum of
// the update pass's partials `rr` (also stored to *rr_out); t = row-FFT(p).
cudaError_t launch_row_fwd_pupdate(const Dims& d, const Twiddles& tw, const float2* r, float2* p,
                                   float2* t, const Partials& rr, const double* rr_prev,
                                   double* rr_out, int first, cudaStream_t st);
// CG step, pass B: t = column-IFFT(mask * column-FFT(t)) / (PQ), in place.
cudaError_t launch_col_mask(const Dims& d, const Twiddles& tw, float2* t, const uint8_t* mask,
                            cudaStream_t st);

// ---- cg.cu ----
// CG step, pass C: q = row-IFFT(t) + lam W p written over t; partials of Re <p, q> to *pq.
cudaError_t launch_row_inv_w(const Dims& d, const Twiddles& tw, float2* t, const float2* p,
                             const float2* S, float lam, Partials* pq, cudaStream_t st);
// CG step, pass D: alpha = *rr_in / Re <p, q> (sum of `pq`); x += alpha p; r -= alpha q;
// partials of |r|^2 to *rr.
cudaError_t launch_cg_update(const Dims& d, float2* x, float2* r, const float2* p,
                             const float2* q, const double* rr_in, const Partials& pq,
                             Partials* rr, cudaStream_t st);
// *out = the sum of the partials `in` (one warp).
cudaError_t launch_sum_partials(const Partials& in, double* out, cudaStream_t st);
// Residual carry: r = (first ? r0 : r) + lam W_{S_old - S_new} x (S_old ignored when first),
// r0 = 0 or, when aha_x = A^H A x is given, x - aha_x; *rr_out = |r|^2.
cudaError_t launch_resid_carry(const Dims& d, float2* r, const float2* x, const float2* S_old,
                               const float2* S_new, float lam, int first, const RedSlot& rs,
                               double* rr_out, cudaStream_t st, const float2* aha_x = nullptr);
// y = W_S x alone (tests)
cudaError_t launch_apply_w(const Dims& d, const float2* x, const float2* S, float2* y,
                           cudaStream_t st);
int max_parts();  // partial-sum slots a RedSlot must provide

// ---- gram.cu ----
// Lags of the Gram matrix (Sec. III-B): per-block partials then deterministic reduction and
// Hermitian fill of G (column-major s x s complex128).
size_t gram_smem(const Dims& d);  // shared memory of the Gram row kernel
size_t gram_scratch_bytes(const Dims& d, int nblocks);
int gram_blocks(const Dims& d);
cudaError_t launch_gram(const Dims& d, const Twiddles& tw, const float2* x, double2* lag_part,
                        int nblocks, double2* lags, double2* G, cudaStream_t st);

// ---- weight.cu ----
// eps update: first -> eps = frac * lambda_max (read from *lmax), else eps /= gamma
cudaError_t launch_eps(const double* lmax, double* eps, int first, double frac, double gamma,
                       cudaStream_t st);
// The same for n solves in one launch (n <= kMaxHpdBatch).
cudaError_t launch_eps_batch(const double* const* lmax, double* const* eps, int n, int first,
                             double frac, double gamma, cudaStream_t st);
// Summed diagonals of H = U diag((lambda + eps)^(p/2-1)) U^H: d[pair][L1][L2] (complex128)
size_t diag_scratch_bytes(const Dims& d);
cudaError_t launch_diag_sums(const Dims& d, const double2* U, const double* evals,
                             const double* eps, double p, double2* dpart, double2* dsum,
                             cudaStream_t st);
// S[pair][P][Q] (complex64) from the summed diagonals
size_t s_scratch_bytes(const Dims& d);
cudaError_t launch_weight_S(const Dims& d, const Twiddles& tw, const double2* dsum, double2* Z,
                            float2* S, cudaStream_t st);

// ---- hpdinv.cu (p = 0: H = (G + eps I)^-1 by a blocked Hermitian sweep, FP64) ----
// The first kCoopBarrierBytes of the sweep and Lanczos scratch hold the grid barrier of their
// cooperative launch. A launch that completed leaves it ready for the next one; zero it when the
// scratch is allocated and after a launch reported a barrier failure (err_flag_out = 1).
constexpr size_t kCoopBarrierBytes = 256;
// Sets the error word of the grid barrier at the head of `scratch` (stream-ordered memset; host-side
// fault injection for tests).
cudaError_t set_barrier_error(void* scratch, cudaStream_t st);
// Test hook of the cooperative weight kernels (host-directed failure, no fault): CTA `withhold`
// (> 0; 0 = none) leaves at its first grid barrier without arriving, and every wait gives up after
// `polls` polls (0 = the default limit of seconds), so that the others' bounded waits run out,
// the launch reports 1 and returns.
struct CoopFault {
    int withhold = 0;
    long long polls = 0;
};
size_t hpd_scratch_bytes(const Dims& d);
size_t lanczos_scratch_bytes(const Dims& d, int grid_max);
// G (s x s, column-major, Hermitian) is replaced by H = (G + eps I)^-1. The kernel writes
// *err_flag_out itself (device int, may be NULL): 0 when it completed, 1 when a grid barrier
// gave up. The same holds for launch_lanczos_lmax.
cudaError_t launch_hpd_inverse(const Dims& d, double2* G, const double* eps, void* scratch,
                               int* err_flag_out, cudaStream_t st, CoopFault fault = {});
// Several matrices in one cooperative launch (one grid barrier per pivot step serves all): job b
// inverts its G (s_b x s_b) with its own eps, scratch (hpd_scratch_bytes of its s) and status
// word. barrier_scratch: the scratch whose barrier header the launch uses (launches sharing it
// must be stream-ordered). Results are bitwise those of launching each matrix alone.
struct HpdJob {
    double2* G;
    const double* eps;
    void* scratch;
    int* err_out;
    int s;
};
cudaError_t launch_hpd_inverse_batch(const HpdJob* jobs, int n, void* barrier_scratch,
                                     cudaStream_t st, CoopFault fault = {});
// d_ab[delta] (summed diagonals) from an explicit H
cudaError_t launch_hdiag(const Dims& d, const double2* H, double2* dsum, cudaStream_t st);
// *lmax = largest eigenvalue of G (Lanczos, FP64)
cudaError_t launch_lanczos_lmax(const Dims& d, const double2* G, void* scratch, double* lmax,
                                int* err_flag_out, cudaStream_t st, CoopFault fault = {});
// Several matrices in one cooperative launch (two grid barriers per step serve all): job b writes
// lambda_max of its G (s_b x s_b) to its *lmax, using its scratch (lanczos_scratch_bytes of its
// s). Bitwise the value of launching the matrix alone.
struct LanczosJob {
    const double2* G;
    void* scratch;
    double* lmax;
    int* err_out;
    int s;
};
cudaError_t launch_lanczos_batch(const LanczosJob* jobs, int n, void* barrier_scratch,
                                 cudaStream_t st, CoopFault fault = {});

// ---- coils (Eq. measurement-ij with receiver sensitivities C_c; d.nc coils, coil-major) ----
// Pass A: p = r (first) or r + beta p (as launch_row_fwd_pupdate); t[c] = row-FFT(C_c * p).
cudaError_t launch_coil_row_fwd(const Dims& d, const Twiddles& tw, const float2* r, float2* p,
                                float2* t, const float2* coils, const Partials& rr,
                                const double* rr_prev, double* rr_out, int first, cudaStream_t st);
// Pass C: q = sum_c conj(C_c) row-IFFT(t[c]) + lam W p over coil 0's plane of t; partials of
// Re <p, q> to *pq.
cudaError_t launch_coil_row_inv_w(const Dims& d, const Twiddles& tw, float2* t, const float2* p,
                                  const float2* coils, const float2* S, float lam, Partials* pq,
                                  cudaStream_t st);
// Adjoint: t[c][n] = column-IFFT(mask_n * b[c][n]) / sqrt(PQ), then
// x = sum_c conj(C_c) row-IFFT(t[c]).
cudaError_t launch_adjoint_coils_cols(const Dims& d, const Twiddles& tw, const void* b,
                                      const uint8_t* mask, float2* t, cudaStream_t st);
cudaError_t launch_coil_combine(const Dims& d, const Twiddles& tw, float2* t, const float2* coils,
                                float2* x, cudaStream_t st);

// *dev = max | |C|^2 - 1 | of the first coil map (float bits; zeroed here).
cudaError_t launch_coil_unimodular(const Dims& d, const float2* coils, unsigned int* dev,
                                   cudaStream_t st);

// ---- t2fit.cu ----
constexpr int kT2MaxT = 64;
struct T2Times {
    float t[kT2MaxT];  // echo times in ms (passed to the kernel by value)
};
// T2 and amplitude maps of a series: max |x_0| into *amax_scratch (one word, zeroed here), then
// the per-pixel fit (NaN outside the foreground |x_0| > frac max |x_0|); amp may be null.
cudaError_t launch_t2fit(const Dims& d, const float2* x, const T2Times& tm, float frac, int n_gn,
                         unsigned int* amax_scratch, float* t2, float* amp, cudaStream_t st);

// ---- variants.cu (comparison methods of Sec. IV) ----
// HLR-Voxel weight per pixel (S = H_r^T into [pair][P][Q]); eps_mode 0: eps_r = eps_in[px];
// 1: no weight, the largest lambda_max(G_r) over the pixels into *lmax_max (atomic max of the
// FP64 bits; zero it first); 2: eps_r = eps_in[0] for every pixel. G_out / lmax_out may be null.
cudaError_t launch_voxel_weight(const Dims& d, const float2* x, double p, const double* eps_in,
                                double* lmax_max, int eps_mode, float2* S, double2* G_out,
                                double* lmax_out, cudaStream_t st);
// IRLS-direct: rows of the exact (valid) lifting, (T-M+1)(P-N1+1)(Q-N2+1)
size_t direct_rows(const Dims& d);
// Tm (rows x s, column-major) of x_hat; complex128 when fp64, else complex64
cudaError_t launch_direct_lift(const Dims& d, const float2* xh, void* Tm, int fp64, cudaStream_t st);
// z = mask * yh (mask may be null: no data term) + lam T^*(Y)
cudaError_t launch_direct_unlift(const Dims& d, const float2* Y, const float2* yh,
                                 const uint8_t* mask, float lam, float2* z, cudaStream_t st);
cudaError_t launch_herm_fill(double2* G, int s, cudaStream_t st);
cudaError_t launch_form_H(const double2* U, const double* evals, const double* eps, double p,
                          int s, double2* H, cudaStream_t st);
cudaError_t launch_h_delta(const double2* H_new, const double2* H_old, float2* delta, float2* h32,
                           size_t n, cudaStream_t st);
cudaError_t launch_dcg_dot(const float2* a, const float2* b, size_t n, const RedSlot& rs,
                           double* out, cudaStream_t st);
cudaError_t launch_dcg_resid(float2* r, const float2* w, int first, size_t n, const RedSlot& rs,
                             double* rr_out, cudaStream_t st);
cudaError_t launch_dcg_update(float2* x, float2* r, const float2* p, const float2* q, size_t n,
                              const double* rr, const double* pq, const RedSlot& rs,
                              double* rr_out, cudaStream_t st);
cudaError_t launch_dcg_pupdate(float2* p, const float2* r, size_t n, const double* rr_new,
                               const double* rr_old, int first, cudaStream_t st);

}  // namespace recon
