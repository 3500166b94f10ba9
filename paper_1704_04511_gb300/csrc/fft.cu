// Row and column passes of the unitary 2-D DFT used by the forward model A = mask * F
// (Sec. II-A, Eq. measurement-ij with one coil) and by the CG operator (Sec. III-A, Eq. grad-ls).
//
// Layout: frames [T][P][Q] complex64, Q contiguous. A row pass transforms length-Q rows
// (ROWS rows per CTA, staged in shared memory); a column pass transforms a P x 8 tile of
// 8 adjacent columns of one frame (64-byte row segments), optionally applying the
// sampling mask between a forward and an inverse transform so that A^H A needs one column pass.
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"
#include "regfft.cuh"

namespace recon {

namespace {

constexpr int kThreads = 256;
constexpr int kColTile = 8;

template <int N>
__host__ __device__ constexpr int rows_per_cta() { return N >= 1024 ? 1 : 1024 / N; }

// Columns per CTA of the column passes: 8, 16 or 32 (64- to 256-byte row segments). The default
// for the volume passes is about 2048 elements per CTA (8 per thread, 33 KB of shared memory,
// six CTAs per SM); the image-series passes default to 8. The autotuner of recon.cu may choose
// another width per shape: the width changes the launch shape, not the arithmetic of any column.
int wide_cols(int n) { return n <= 64 ? 32 : (n <= 128 ? 16 : 8); }
template <int N, int C>
constexpr bool col_tile_ok() { return (size_t)(2 * N * C + N) * sizeof(float2) <= 100 * 1024; }

enum ColMode { COL_FWD = 0, COL_INV = 1, COL_MASK_OP = 2, COL_ADJ_C64 = 3, COL_ADJ_BF16 = 4 };

template <int N, bool INV>
__global__ void __launch_bounds__(kThreads)
row_fft_kernel(const float2* in, float2* out, int nrows, float scale,
               const float2* __restrict__ tw_g) {
    constexpr int ROWS = rows_per_cta<N>();
    extern __shared__ float2 sm[];
    float2* a = sm;
    float2* b = a + ROWS * N;
    float2* tw = b + ROWS * N;
    for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = tw_g[i];
    const int row0 = blockIdx.x * ROWS;
    const int nr = min(ROWS, nrows - row0);
    const size_t base = (size_t)row0 * N;
    for (int e = threadIdx.x; e < nr * N; e += blockDim.x) a[e] = in[base + e];
    __syncthreads();
    float2* res = fft_smem<N, INV, false>(a, b, nr, N, 1, tw);
    for (int e = threadIdx.x; e < nr * N; e += blockDim.x) out[base + e] = cscale(res[e], scale);
}

// Pass A of a CG step: p = r (first) or r + beta p with beta = |r_c|^2 / |r_{c-1}|^2, |r_c|^2
// summed here from the update pass's per-CTA partials (CTA 0 also stores it); p is written back
// and its row FFT goes to t.
template <int N>
__global__ void __launch_bounds__(kThreads)
row_fwd_pupdate_kernel(const float2* __restrict__ r, float2* __restrict__ p,
                       float2* __restrict__ t, int nrows, const double* __restrict__ rr_parts,
                       int n_rr, const double* __restrict__ rr_prev, double* __restrict__ rr_out,
                       int first, const float2* __restrict__ tw_g) {
    constexpr int ROWS = rows_per_cta<N>();
    extern __shared__ float2 sm[];
    __shared__ float beta_s;
    __shared__ double s_rr;
    float2* a = sm;
    float2* b = a + ROWS * N;
    float2* tw = b + ROWS * N;
    for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = tw_g[i];
    pdl_wait();
    float beta = 0.f;
    if (!first) {
        const double rr_new = sum_partials(rr_parts, n_rr, &s_rr);
        if (threadIdx.x == 0) {
            beta_s = (float)(rr_new * rcp_nr(rr_prev[0]));
            if (blockIdx.x == 0) rr_out[0] = rr_new;
        }
        __syncthreads();
        beta = beta_s;
    }
    const int row0 = blockIdx.x * ROWS;
    const int nr = min(ROWS, nrows - row0);
    const size_t base = (size_t)row0 * N;
    for (int e = threadIdx.x; e < nr * N; e += blockDim.x) {
        float2 v = r[base + e];
        if (!first) {
            const float2 pv = p[base + e];
            v.x = fmaf(beta, pv.x, v.x);
            v.y = fmaf(beta, pv.y, v.y);
        }
        p[base + e] = v;
        a[e] = v;
    }
    __syncthreads();
    float2* res = fft_smem<N, false, false>(a, b, nr, N, 1, tw);
    pdl_trigger();
    for (int e = threadIdx.x; e < nr * N; e += blockDim.x) t[base + e] = res[e];
}

// Pass A of a CG step with coils (Eq. measurement-ij): p = r (first) or r + beta p as in
// row_fwd_pupdate_kernel, then for every coil c the row FFT of C_c * p goes to the coil-major
// transform buffer t[c][n] (rows of the T x P row space; coil maps [nc][P][Q]).
template <int N>
__global__ void __launch_bounds__(kThreads)
coil_row_fwd_kernel(const float2* __restrict__ r, float2* __restrict__ p, float2* __restrict__ t,
                    const float2* __restrict__ coils, int nrows, int P, int nc,
                    const double* __restrict__ rr_parts, int n_rr,
                    const double* __restrict__ rr_prev, double* __restrict__ rr_out, int first,
                    const float2* __restrict__ tw_g) {
    constexpr int ROWS = rows_per_cta<N>();
    extern __shared__ float2 sm[];
    __shared__ float beta_s;
    __shared__ double s_rr;
    float2* a = sm;
    float2* b = a + ROWS * N;
    float2* pk = b + ROWS * N;
    float2* tw = pk + ROWS * N;
    for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = tw_g[i];
    pdl_wait();
    float beta = 0.f;
    if (!first) {
        const double rr_new = sum_partials(rr_parts, n_rr, &s_rr);
        if (threadIdx.x == 0) {
            beta_s = (float)(rr_new * rcp_nr(rr_prev[0]));
            if (blockIdx.x == 0) rr_out[0] = rr_new;
        }
        __syncthreads();
        beta = beta_s;
    }
    const int row0 = blockIdx.x * ROWS;
    const int nr = min(ROWS, nrows - row0);
    const size_t base = (size_t)row0 * N;
    const size_t series = (size_t)nrows * N;  // one coil's T x P x Q block
    for (int e = threadIdx.x; e < nr * N; e += blockDim.x) {
        float2 v = r[base + e];
        if (!first) {
            const float2 pv = p[base + e];
            v.x = fmaf(beta, pv.x, v.x);
            v.y = fmaf(beta, pv.y, v.y);
        }
        p[base + e] = v;
        pk[e] = v;
    }
    for (int c = 0; c < nc; ++c) {
        __syncthreads();  // pk written / a, b free again
        for (int e = threadIdx.x; e < nr * N; e += blockDim.x) {
            const int row = row0 + e / N;
            const float2 cv = coils[((size_t)c * P + row % P) * N + e % N];
            a[e] = cmul(cv, pk[e]);
        }
        __syncthreads();
        float2* res = fft_smem<N, false, false>(a, b, nr, N, 1, tw);
        if (c == nc - 1) pdl_trigger();
        for (int e = threadIdx.x; e < nr * N; e += blockDim.x) t[c * series + base + e] = res[e];
    }
}

// Column pass over an N x C tile (frame blockIdx.y, columns C*blockIdx.x ..), Stockham passes
// in radix schedule S (fft_radix_at).
template <int N, int MODE, int C, int S>
__global__ void __launch_bounds__(kThreads)
col_kernel(const void* in_, float2* out, const uint8_t* __restrict__ mask,
           int Q, int mask_frames, float scale, const float2* __restrict__ tw_g) {
    extern __shared__ float2 sm[];
    float2* a = sm;
    float2* b = a + N * C;
    float2* tw = b + N * C;
    for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = tw_g[i];
    pdl_wait();
    const int c0 = blockIdx.x * C;
    const size_t fbase = (size_t)blockIdx.y * N * Q;
    // coil-major series: frame blockIdx.y is coil blockIdx.y / T of frame blockIdx.y % T
    const size_t mbase = (size_t)(blockIdx.y % mask_frames) * N * Q;
    for (int e = threadIdx.x; e < N * C; e += blockDim.x) {
        const int i = e / C, c = e % C;
        const size_t g = fbase + (size_t)i * Q + c0 + c;
        const size_t gm = mbase + (size_t)i * Q + c0 + c;
        float2 v;
        if constexpr (MODE == COL_ADJ_BF16) {
            const __nv_bfloat162 h = reinterpret_cast<const __nv_bfloat162*>(in_)[g];
            v = __bfloat1622float2(h);
        } else {
            v = reinterpret_cast<const float2*>(in_)[g];
        }
        if constexpr (MODE == COL_ADJ_C64 || MODE == COL_ADJ_BF16) {
            v = mask[gm] ? cscale(v, scale) : make_float2(0.f, 0.f);
        }
        a[e] = v;
    }
    __syncthreads();
    float2* res;
    if constexpr (MODE == COL_FWD) {
        res = fft_smem<N, false, true, 1, S>(a, b, C, 1, C, tw);
    } else if constexpr (MODE == COL_INV || MODE == COL_ADJ_C64 || MODE == COL_ADJ_BF16) {
        res = fft_smem<N, true, true, 1, S>(a, b, C, 1, C, tw);
    } else {  // COL_MASK_OP
        float2* f = fft_smem<N, false, true, 1, S>(a, b, C, 1, C, tw);
        for (int e = threadIdx.x; e < N * C; e += blockDim.x) {
            const int i = e / C, c = e % C;
            const uint8_t m = mask[mbase + (size_t)i * Q + c0 + c];
            f[e] = m ? cscale(f[e], scale) : make_float2(0.f, 0.f);
        }
        __syncthreads();
        res = fft_smem<N, true, true, 1, S>(f, f == a ? b : a, C, 1, C, tw);
    }
    pdl_trigger();
    const float osc = (MODE == COL_FWD || MODE == COL_INV) ? scale : 1.f;
    for (int e = threadIdx.x; e < N * C; e += blockDim.x) {
        const int i = e / C, c = e % C;
        out[fbase + (size_t)i * Q + c0 + c] = cscale(res[e], osc);
    }
}

// ---- 256-point specialisations: transforms held in registers (regfft.cuh) ----
constexpr int kR256Rows = 4;  // rows per 64-thread CTA, one half-warp per row

// Pass A of a CG step for 256-point rows (same contract as row_fwd_pupdate_kernel).
__global__ void __launch_bounds__(64)
row_fwd_pupdate_256_kernel(const float2* __restrict__ r, float2* __restrict__ p,
                           float2* __restrict__ t, int nrows, const double* __restrict__ rr_parts,
                           int n_rr, const double* __restrict__ rr_prev,
                           double* __restrict__ rr_out, int first,
                           const float2* __restrict__ tw_g) {
    __shared__ float2 tw2[256];
    __shared__ float2 sx[kR256Rows][16 * 17];
    __shared__ float beta_s;
    fill_tw256(tw2, tw_g);
    pdl_wait();
    const int lr = threadIdx.x / 16, j = threadIdx.x % 16;
    const int row = blockIdx.x * kR256Rows + lr;
    const bool ok = row < nrows;
    const size_t base = (size_t)row * 256 + j;
    float2 u[16], pv[16];
    if (ok) {
#pragma unroll
        for (int n1 = 0; n1 < 16; ++n1) u[n1] = r[base + 16 * n1];
        if (!first) {
#pragma unroll
            for (int n1 = 0; n1 < 16; ++n1) pv[n1] = p[base + 16 * n1];
        }
    } else {
#pragma unroll
        for (int n1 = 0; n1 < 16; ++n1) u[n1] = make_float2(0.f, 0.f);
    }
    if (!first && threadIdx.x < 32) {  // |r|^2 from the update pass's partials, loads in flight
        const double rr_new = warp0_sum_array(rr_parts, n_rr);
        if (threadIdx.x == 0) {
            beta_s = (float)(rr_new * rcp_nr(rr_prev[0]));
            if (blockIdx.x == 0) rr_out[0] = rr_new;
        }
    }
    __syncthreads();  // tw2, beta
    if (!first) {
        const float beta = beta_s;
#pragma unroll
        for (int n1 = 0; n1 < 16; ++n1) {
            u[n1].x = fmaf(beta, pv[n1].x, u[n1].x);
            u[n1].y = fmaf(beta, pv[n1].y, u[n1].y);
        }
    }
    if (ok) {
#pragma unroll
        for (int n1 = 0; n1 < 16; ++n1) p[base + 16 * n1] = u[n1];
    }
    row_dft256<false>(u, sx[lr], tw2, j);
    pdl_trigger();
    if (ok) {
#pragma unroll
        for (int k2 = 0; k2 < 16; ++k2) t[base + 16 * k2] = u[k2];
    }
}

// Pass A of a CG step for 128-point rows (same contract as row_fwd_pupdate_kernel): 8 rows per
// 64-thread CTA, 8 lanes per row (row_dft128 in regfft.cuh).
constexpr int kR128Rows = 8;

__global__ void __launch_bounds__(64)
row_fwd_pupdate_128_kernel(const float2* __restrict__ r, float2* __restrict__ p,
                           float2* __restrict__ t, int nrows, const double* __restrict__ rr_parts,
                           int n_rr, const double* __restrict__ rr_prev,
                           double* __restrict__ rr_out, int first,
                           const float2* __restrict__ tw_g) {
    __shared__ float2 tw8[128];
    __shared__ float2 sx[kR128Rows][kX128];
    __shared__ float beta_s;
    fill_tw128(tw8, tw_g);
    pdl_wait();
    const int lr = threadIdx.x / 8, j = threadIdx.x % 8;
    const int row = blockIdx.x * kR128Rows + lr;
    const bool ok = row < nrows;
    const size_t base = (size_t)row * 128 + j;
    float2 u[16], pv[16];
    if (ok) {
#pragma unroll
        for (int n1 = 0; n1 < 16; ++n1) u[n1] = r[base + 8 * n1];
        if (!first) {
#pragma unroll
            for (int n1 = 0; n1 < 16; ++n1) pv[n1] = p[base + 8 * n1];
        }
    } else {
#pragma unroll
        for (int n1 = 0; n1 < 16; ++n1) u[n1] = make_float2(0.f, 0.f);
    }
    if (!first && threadIdx.x < 32) {  // |r|^2 from the update pass's partials, loads in flight
        const double rr_new = warp0_sum_array(rr_parts, n_rr);
        if (threadIdx.x == 0) {
            beta_s = (float)(rr_new * rcp_nr(rr_prev[0]));
            if (blockIdx.x == 0) rr_out[0] = rr_new;
        }
    }
    __syncthreads();  // tw8, beta
    if (!first) {
        const float beta = beta_s;
#pragma unroll
        for (int n1 = 0; n1 < 16; ++n1) {
            u[n1].x = fmaf(beta, pv[n1].x, u[n1].x);
            u[n1].y = fmaf(beta, pv[n1].y, u[n1].y);
        }
    }
    if (ok) {
#pragma unroll
        for (int n1 = 0; n1 < 16; ++n1) p[base + 8 * n1] = u[n1];
    }
    float2 a[8], b[8];
    row_dft128<false>(u, a, b, sx[lr], tw8, j);
    pdl_trigger();
    if (ok) {
        float2* out = t + (size_t)row * 128 + 2 * j;
#pragma unroll
        for (int k2 = 0; k2 < 8; ++k2) {
            out[16 * k2] = a[k2];
            out[16 * k2 + 1] = b[k2];
        }
    }
}

// Column pass with the sampling mask for 256-point columns: 8 adjacent columns of one frame per
// 128-thread CTA, thread (c, j) holding rows j + 16 n1 of column c. Forward DFT, mask and the
// 1/(PQ) scale, inverse DFT, all in registers; two exchanges through shared memory, laid out as
// c + 8 (17 a + b) so that both the writes and the reads are conflict-free.
__global__ void __launch_bounds__(128)
col_mask_256_kernel(float2* t, const uint8_t* __restrict__ mask, int Q, int mask_frames,
                    float scale, const float2* __restrict__ tw_g) {
    __shared__ float2 tw2[256];
    __shared__ float2 buf[8 * 17 * 16];
    fill_tw256(tw2, tw_g);
    pdl_wait();
    const int c = threadIdx.x % 8, j = threadIdx.x / 8;
    const int col = blockIdx.x * 8 + c;
    const size_t fbase = (size_t)blockIdx.y * 256 * Q;
    const size_t mbase = (size_t)(blockIdx.y % mask_frames) * 256 * Q;  // coil-major series
    float2 u[16];
#pragma unroll
    for (int n1 = 0; n1 < 16; ++n1) u[n1] = t[fbase + (size_t)(16 * n1 + j) * Q + col];
    uint8_t mk[16];
#pragma unroll
    for (int k2 = 0; k2 < 16; ++k2) mk[k2] = mask[mbase + (size_t)(j + 16 * k2) * Q + col];
    __syncthreads();  // tw2
    dft16<false>(u);
    twiddle256<false>(u, tw2, j);
#pragma unroll
    for (int k1 = 0; k1 < 16; ++k1) buf[c + 8 * (17 * k1 + j)] = u[k1];
    __syncthreads();
#pragma unroll
    for (int n2 = 0; n2 < 16; ++n2) u[n2] = buf[c + 8 * (17 * j + n2)];
    dft16<false>(u);  // u[k2] = X[j + 16 k2]
#pragma unroll
    for (int k2 = 0; k2 < 16; ++k2) u[k2] = mk[k2] ? cscale(u[k2], scale) : make_float2(0.f, 0.f);
    dft16<true>(u);  // u[n1] = sum_k2 X[j + 16 k2] w16^(-k2 n1)
    twiddle256<true>(u, tw2, j);
    __syncthreads();  // first exchange fully read
#pragma unroll
    for (int n1 = 0; n1 < 16; ++n1) buf[c + 8 * (17 * n1 + j)] = u[n1];
    __syncthreads();
#pragma unroll
    for (int k1 = 0; k1 < 16; ++k1) u[k1] = buf[c + 8 * (17 * j + k1)];
    dft16<true>(u);  // u[n2] = x[j + 16 n2]
    pdl_trigger();
#pragma unroll
    for (int n2 = 0; n2 < 16; ++n2) t[fbase + (size_t)(j + 16 * n2) * Q + col] = u[n2];
}

// ---- register-transform column passes of the volume column stage ----
// 128-point columns (the length-P passes, slices of a volume): 16 columns per 128-thread CTA, 8
// lanes per column in different warps; lane j loads x[8 n1 + j] (n1 < 16), runs the 16-point
// DFT and the twiddles w128^(j k1), and after one exchange through shared memory (layout
// [k1][j][column], conflict-free) runs two 8-point DFTs for k1 = 2j and 2j + 1: it then holds
// X[k1 + 16 k2]. Unnormalised, forward or inverse, in place (each CTA owns its columns).
template <bool INV>
__global__ void __launch_bounds__(128)
col128_kernel(float2* t, int Q, const float2* __restrict__ tw_g) {
    constexpr int C = 16;
    __shared__ float2 tw8[128];
    __shared__ float2 buf[16 * 8 * C];
    fill_tw128(tw8, tw_g);
    pdl_wait();
    const int c = threadIdx.x % C, j = threadIdx.x / C;
    const int col = blockIdx.x * C + c;
    const size_t fbase = (size_t)blockIdx.y * 128 * Q;
    float2 u[16];
#pragma unroll
    for (int n1 = 0; n1 < 16; ++n1) u[n1] = t[fbase + (size_t)(8 * n1 + j) * Q + col];
    __syncthreads();  // tw8
    dft16<INV>(u);
#pragma unroll
    for (int k1 = 1; k1 < 16; ++k1) {
        float2 w = tw8[k1 * 8 + j];
        if (INV) w.y = -w.y;
        u[k1] = cmul(u[k1], w);
    }
#pragma unroll
    for (int k1 = 0; k1 < 16; ++k1) buf[(k1 * 8 + j) * C + c] = u[k1];
    __syncthreads();
    float2 a[8], b[8];
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) {
        a[jj] = buf[((2 * j) * 8 + jj) * C + c];
        b[jj] = buf[((2 * j + 1) * 8 + jj) * C + c];
    }
    SmallDFT<8, INV>::run(a);
    SmallDFT<8, INV>::run(b);
    pdl_trigger();
#pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) {
        t[fbase + (size_t)(2 * j + 16 * k2) * Q + col] = a[k2];
        t[fbase + (size_t)(2 * j + 1 + 16 * k2) * Q + col] = b[k2];
    }
}

// 128-point column pass with the mask (image series of 128 rows, any coil count): the forward
// transform of col128_kernel, the mask and the 1/(PQ) scale on X[k1 + 16 k2] (k1 = 2j, 2j + 1),
// then the inverse in the mirrored order -- two 8-point IDFTs over k2, twiddles w128^(-n2 k1),
// an exchange, a 16-point IDFT over k1 -- so that lane j ends holding y[j + 8 n1], the elements
// it loaded. Frame blockIdx.y uses mask frame blockIdx.y % mask_frames (coil-major series).
__global__ void __launch_bounds__(128)
col_mask_128_kernel(float2* t, const uint8_t* __restrict__ mask, int Q, int mask_frames,
                    float scale, const float2* __restrict__ tw_g) {
    constexpr int C = 16;
    __shared__ float2 tw8[128];
    __shared__ float2 buf[16 * 8 * C];
    fill_tw128(tw8, tw_g);
    pdl_wait();
    const int c = threadIdx.x % C, j = threadIdx.x / C;
    const int col = blockIdx.x * C + c;
    const size_t fbase = (size_t)blockIdx.y * 128 * Q;
    const size_t mbase = (size_t)(blockIdx.y % mask_frames) * 128 * Q;
    float2 u[16];
#pragma unroll
    for (int n1 = 0; n1 < 16; ++n1) u[n1] = t[fbase + (size_t)(8 * n1 + j) * Q + col];
    uint8_t ma[8], mb[8];
#pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) {
        ma[k2] = mask[mbase + (size_t)(2 * j + 16 * k2) * Q + col];
        mb[k2] = mask[mbase + (size_t)(2 * j + 1 + 16 * k2) * Q + col];
    }
    __syncthreads();  // tw8
    dft16<false>(u);
#pragma unroll
    for (int k1 = 1; k1 < 16; ++k1) u[k1] = cmul(u[k1], tw8[k1 * 8 + j]);
#pragma unroll
    for (int k1 = 0; k1 < 16; ++k1) buf[(k1 * 8 + j) * C + c] = u[k1];
    __syncthreads();
    float2 a[8], b[8];
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) {
        a[jj] = buf[((2 * j) * 8 + jj) * C + c];
        b[jj] = buf[((2 * j + 1) * 8 + jj) * C + c];
    }
    SmallDFT<8, false>::run(a);  // a[k2] = X[2j + 16 k2], b[k2] = X[2j + 1 + 16 k2]
    SmallDFT<8, false>::run(b);
#pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) {
        a[k2] = ma[k2] ? cscale(a[k2], scale) : make_float2(0.f, 0.f);
        b[k2] = mb[k2] ? cscale(b[k2], scale) : make_float2(0.f, 0.f);
    }
    SmallDFT<8, true>::run(a);   // a[n2] = sum_k2 Y[2j + 16 k2] w8^(-k2 n2)
    SmallDFT<8, true>::run(b);
#pragma unroll
    for (int n2 = 1; n2 < 8; ++n2) {  // w128^(-n2 k1) for k1 = 2j and 2j + 1
        float2 wa = tw8[(2 * j) * 8 + n2], wb = tw8[(2 * j + 1) * 8 + n2];
        wa.y = -wa.y;
        wb.y = -wb.y;
        a[n2] = cmul(a[n2], wa);
        b[n2] = cmul(b[n2], wb);
    }
    __syncthreads();  // the first exchange is read
#pragma unroll
    for (int n2 = 0; n2 < 8; ++n2) {
        buf[((2 * j) * 8 + n2) * C + c] = a[n2];
        buf[((2 * j + 1) * 8 + n2) * C + c] = b[n2];
    }
    __syncthreads();
#pragma unroll
    for (int k1 = 0; k1 < 16; ++k1) u[k1] = buf[(k1 * 8 + j) * C + c];
    dft16<true>(u);  // u[n1] = y[j + 8 n1]
    pdl_trigger();
#pragma unroll
    for (int n1 = 0; n1 < 16; ++n1) t[fbase + (size_t)(8 * n1 + j) * Q + col] = u[n1];
}

// 64-point depth pass with the mask (volumes of depth 64): 32 columns per 256-thread CTA, 8
// lanes per column; lane j loads x[8 n1 + j], and after the 8-point DFT, the twiddles w64^(j k1)
// and one exchange it holds X[j + 8 k2]; it applies the mask and the 1/(PQR) scale, then runs the
// inverse in the mirrored order (8-point IDFT over k2, twiddles w64^(-n2 j), exchange, 8-point
// IDFT) and ends holding y[j + 8 n1] -- the elements it loaded.
__global__ void __launch_bounds__(256)
col_mask_64_kernel(float2* t, const uint8_t* __restrict__ mask, int Q, float scale,
                   const float2* __restrict__ tw_g) {
    constexpr int C = 32;
    __shared__ float2 tw8[64];
    __shared__ float2 buf[8 * 8 * C];
    for (int e = threadIdx.x; e < 64; e += blockDim.x) tw8[e] = tw_g[(e / 8) * (e % 8)];
    pdl_wait();
    const int c = threadIdx.x % C, j = threadIdx.x / C;
    const int col = blockIdx.x * C + c;
    const size_t fbase = (size_t)blockIdx.y * 64 * Q;
    float2 u[8];
    uint8_t mk[8];
#pragma unroll
    for (int n1 = 0; n1 < 8; ++n1) u[n1] = t[fbase + (size_t)(8 * n1 + j) * Q + col];
#pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) mk[k2] = mask[fbase + (size_t)(j + 8 * k2) * Q + col];
    __syncthreads();  // tw8
    SmallDFT<8, false>::run(u);
#pragma unroll
    for (int k1 = 1; k1 < 8; ++k1) u[k1] = cmul(u[k1], tw8[k1 * 8 + j]);
#pragma unroll
    for (int k1 = 0; k1 < 8; ++k1) buf[(k1 * 8 + j) * C + c] = u[k1];
    __syncthreads();
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) u[jj] = buf[(j * 8 + jj) * C + c];
    SmallDFT<8, false>::run(u);  // u[k2] = X[j + 8 k2]
#pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) u[k2] = mk[k2] ? cscale(u[k2], scale) : make_float2(0.f, 0.f);
    SmallDFT<8, true>::run(u);   // u[n2] = sum_k2 Y[j + 8 k2] w8^(-k2 n2)
#pragma unroll
    for (int n2 = 1; n2 < 8; ++n2) {
        float2 w = tw8[n2 * 8 + j];
        w.y = -w.y;
        u[n2] = cmul(u[n2], w);
    }
    __syncthreads();  // the first exchange is read
#pragma unroll
    for (int n2 = 0; n2 < 8; ++n2) buf[(n2 * 8 + j) * C + c] = u[n2];
    __syncthreads();
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) u[jj] = buf[(j * 8 + jj) * C + c];
    SmallDFT<8, true>::run(u);   // u[n1] = y[j + 8 n1]
    pdl_trigger();
#pragma unroll
    for (int n1 = 0; n1 < 8; ++n1) t[fbase + (size_t)(j + 8 * n1) * Q + col] = u[n1];
}

// ---- volumes of 128 x 128 slices and depth 64: the length-P DFT split over two passes ----
// With p = 8 p1 + p2 and kp = k1 + 16 k2 the length-128 column DFT is
//   X[k1 + 16 k2] = sum_p2 w8^(p2 k2) Y[k1][p2],  Y[k1][p2] = w128^(p2 k1) sum_p1 x[8 p1 + p2] w16^(p1 k1),
// and its inverse, with p = p2 + 8 p1,
//   x[p2 + 8 p1] = sum_k1 w16^(-p1 k1) Z[k1][p2],  Z[k1][p2] = w128^(-p2 k1) sum_k2 X[k1 + 16 k2] w8^(-p2 k2).
// The row pass of a CG step, holding the 16 rows 8 p1 + p2 of one slice (one p2), computes Y and
// stores Y[k1][p2] at row 8 k1 + p2. The depth pass, holding the rows 8 k1 + p2 of one k1 in every
// slice of a frame for 8 columns, runs the 8-point DFT over p2 (giving X), the depth DFT, the
// mask, the depth IDFT and the 8-point IDFT over k2, and stores Z[k1][p2] at row 8 k1 + p2 again.
// The last pass runs the 16-point IDFT over k1 in place. The column stage is then two launches
// (33 E bytes) instead of three (49 E): the length-P forward pass is folded away.
// vol_fold selects this path.

// Pass A of a CG step for such volumes: p = r + beta p and the row DFT of 16 rows of one slice
// (rows 8 p1 + p2, p2 = blockIdx.x % 8, 8 lanes per row as in row_fwd_pupdate_128_kernel), then the
// 16-point DFT over p1 of each of the 128 columns and the twiddle w128^(p2 k1) (P = Q = 128, so the
// one length-128 table serves both directions); Y[k1][p2] goes to row 8 k1 + p2 of t.
__global__ void __launch_bounds__(128)
row_fwd_col1_128_kernel(const float2* __restrict__ r, float2* __restrict__ p,
                        float2* __restrict__ t, const double* __restrict__ rr_parts, int n_rr,
                        const double* __restrict__ rr_prev, double* __restrict__ rr_out,
                        int first, const float2* __restrict__ tw_g) {
    __shared__ float2 tw8[128];
    __shared__ float2 sx[16][kX128];
    __shared__ __align__(16) float2 cb[16][128];
    __shared__ float beta_s;
    fill_tw128(tw8, tw_g);
    pdl_wait();
    const int p1 = threadIdx.x / 8, j = threadIdx.x % 8;
    const int p2 = blockIdx.x % 8;
    const size_t sbase = (size_t)(blockIdx.x / 8) * 128 * 128;
    const size_t base = sbase + (size_t)(8 * p1 + p2) * 128 + j;
    float2 u[16], pv[16];
#pragma unroll
    for (int n1 = 0; n1 < 16; ++n1) u[n1] = r[base + 8 * n1];
    if (!first) {
#pragma unroll
        for (int n1 = 0; n1 < 16; ++n1) pv[n1] = p[base + 8 * n1];
    }
    if (!first && threadIdx.x < 32) {  // |r|^2 from the update pass's partials, loads in flight
        const double rr_new = warp0_sum_array(rr_parts, n_rr);
        if (threadIdx.x == 0) {
            beta_s = (float)(rr_new * rcp_nr(rr_prev[0]));
            if (blockIdx.x == 0) rr_out[0] = rr_new;
        }
    }
    __syncthreads();  // tw8, beta
    if (!first) {
        const float beta = beta_s;
#pragma unroll
        for (int n1 = 0; n1 < 16; ++n1) {
            u[n1].x = fmaf(beta, pv[n1].x, u[n1].x);
            u[n1].y = fmaf(beta, pv[n1].y, u[n1].y);
        }
    }
#pragma unroll
    for (int n1 = 0; n1 < 16; ++n1) p[base + 8 * n1] = u[n1];
    float2 a[8], b[8];
    row_dft128<false>(u, a, b, sx[p1], tw8, j);  // a[k2] = X[2j + 16 k2], b[k2] = X[2j + 1 + 16 k2]
#pragma unroll
    for (int k2 = 0; k2 < 8; ++k2)  // one 16-byte store per pair: eight lanes fill 128 bytes
        *reinterpret_cast<float4*>(&cb[p1][2 * j + 16 * k2]) =
            make_float4(a[k2].x, a[k2].y, b[k2].x, b[k2].y);
    __syncthreads();
    const int kq = threadIdx.x;
    float2 v[16];
#pragma unroll
    for (int n = 0; n < 16; ++n) v[n] = cb[n][kq];
    dft16<false>(v);  // v[k1] = sum_p1 x[8 p1 + p2] w16^(p1 k1) in column kq
#pragma unroll
    for (int k1 = 1; k1 < 16; ++k1) v[k1] = cmul(v[k1], tw8[k1 * 8 + p2]);
    pdl_trigger();
#pragma unroll
    for (int k1 = 0; k1 < 16; ++k1) t[sbase + (size_t)(8 * k1 + p2) * 128 + kq] = v[k1];
}

// The depth pass of the split: one frame, one k1 (blockIdx.y), 8 columns (blockIdx.x), all 64
// slices; 256 threads. Stage A: thread (q, d) holds rows 8 k1 + p2 (p2 < 8) of depths d and d + 32
// and runs the 8-point DFT over p2 -> X[k1 + 16 k2]. Stage B: the 64 columns (k2, q) of 64 depths
// get the depth DFT, mask, 1/(PQR) scale and depth IDFT of col_mask_64_kernel (lane j holding depths
// 8 n1 + j of columns c and c + 32). Stage A again: the 8-point IDFT over k2 and the twiddle
// w128^(-p2 k1), stored at rows 8 k1 + p2 (the rows loaded). The exchange buffer holds a depth row
// of 64 columns every 72 float2, so that every exchange is free of bank conflicts; the mask bytes
// of the 8 columns arrive in 8-byte runs into shared memory while stage A loads.
constexpr int kFoldPitch = 72;

constexpr int kFoldQ = 128;  // P and Q of the volumes the split serves

__global__ void __launch_bounds__(256, 4)  // 64 registers: four CTAs per SM
depth_fold_64_kernel(float2* t, const uint8_t* __restrict__ mask, float scale,
                     const float2* __restrict__ twP_g, const float2* __restrict__ twR_g) {
    constexpr int Q = kFoldQ;
    constexpr size_t PQ = (size_t)128 * Q;
    __shared__ float2 tw8[128];  // w128^(j k1) at [k1 * 8 + j]
    __shared__ float2 tw64[64];  // w64^(j k1) at [k1 * 8 + j]
    __shared__ float2 E[64 * kFoldPitch];
    __shared__ __align__(8) uint8_t Mk[64 * 64];  // mask at depth frequency kr, column (k2, q): [kr * 64 + 8 k2 + q]
    fill_tw128(tw8, twP_g);
    for (int e = threadIdx.x; e < 64; e += blockDim.x) tw64[e] = twR_g[(e / 8) * (e % 8)];
    pdl_wait();
    const int q0 = blockIdx.x * 8, k1 = blockIdx.y;
    const size_t fbase = (size_t)blockIdx.z * 64 * PQ;
    const int qa = threadIdx.x % 8, da = threadIdx.x / 8;  // stage A: column q0 + qa, depths da, da + 32
    const int cb = threadIdx.x % 32, jb = threadIdx.x / 32;  // stage B: columns cb, cb + 32; lane jb
    float2 x0[8], x1[8];
    const size_t a0 = fbase + (size_t)da * PQ + (size_t)(8 * k1) * Q + q0 + qa;
    const size_t a1 = a0 + 32 * PQ;
#pragma unroll
    for (int p2 = 0; p2 < 8; ++p2) {
        x0[p2] = t[a0 + (size_t)p2 * Q];
        x1[p2] = t[a1 + (size_t)p2 * Q];
    }
    {   // the mask bytes of the CTA's 8 columns: 512 runs of 8 (depth frequency kr, k2), each an
        // aligned 8-byte load (the entry points take 16-byte aligned masks; q0 is a multiple of 8)
        const uint8_t* mb = mask + fbase + (size_t)k1 * Q + q0;
#pragma unroll
        for (int i = threadIdx.x; i < 512; i += 256) {
            const int kr = i / 8, k2 = i % 8;
            const uint8_t* src = mb + (size_t)kr * PQ + (size_t)(16 * k2) * Q;
            *reinterpret_cast<uint2*>(&Mk[kr * 64 + 8 * k2]) =
                __ldg(reinterpret_cast<const uint2*>(src));
        }
    }
    __syncthreads();  // tables
    SmallDFT<8, false>::run(x0);  // x0[k2] = X[k1 + 16 k2] at depth da
    SmallDFT<8, false>::run(x1);
#pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) {
        E[da * kFoldPitch + 8 * k2 + qa] = x0[k2];
        E[(da + 32) * kFoldPitch + 8 * k2 + qa] = x1[k2];
    }
    __syncthreads();
    float2 u0[8], u1[8];
#pragma unroll
    for (int n1 = 0; n1 < 8; ++n1) {
        u0[n1] = E[(8 * n1 + jb) * kFoldPitch + cb];
        u1[n1] = E[(8 * n1 + jb) * kFoldPitch + cb + 32];
    }
    SmallDFT<8, false>::run(u0);
    SmallDFT<8, false>::run(u1);
#pragma unroll
    for (int kd = 1; kd < 8; ++kd) {
        const float2 w = tw64[kd * 8 + jb];
        u0[kd] = cmul(u0[kd], w);
        u1[kd] = cmul(u1[kd], w);
    }
    __syncthreads();  // stage A rows read
#pragma unroll
    for (int kd = 0; kd < 8; ++kd) {
        E[(kd * 8 + jb) * kFoldPitch + cb] = u0[kd];
        E[(kd * 8 + jb) * kFoldPitch + cb + 32] = u1[kd];
    }
    __syncthreads();
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) {
        u0[jj] = E[(jb * 8 + jj) * kFoldPitch + cb];
        u1[jj] = E[(jb * 8 + jj) * kFoldPitch + cb + 32];
    }
    SmallDFT<8, false>::run(u0);  // u0[m] = X[jb + 8 m] along the depth
    SmallDFT<8, false>::run(u1);
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        const uint8_t* mk = &Mk[(jb + 8 * m) * 64 + cb];
        u0[m] = mk[0] ? cscale(u0[m], scale) : make_float2(0.f, 0.f);
        u1[m] = mk[32] ? cscale(u1[m], scale) : make_float2(0.f, 0.f);
    }
    SmallDFT<8, true>::run(u0);  // u0[n2] = sum_m Y[jb + 8 m] w8^(-m n2)
    SmallDFT<8, true>::run(u1);
#pragma unroll
    for (int n2 = 1; n2 < 8; ++n2) {
        float2 w = tw64[n2 * 8 + jb];
        w.y = -w.y;
        u0[n2] = cmul(u0[n2], w);
        u1[n2] = cmul(u1[n2], w);
    }
    __syncthreads();  // the depth exchange is read
#pragma unroll
    for (int n2 = 0; n2 < 8; ++n2) {
        E[(n2 * 8 + jb) * kFoldPitch + cb] = u0[n2];
        E[(n2 * 8 + jb) * kFoldPitch + cb + 32] = u1[n2];
    }
    __syncthreads();
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) {
        u0[jj] = E[(jb * 8 + jj) * kFoldPitch + cb];
        u1[jj] = E[(jb * 8 + jj) * kFoldPitch + cb + 32];
    }
    SmallDFT<8, true>::run(u0);  // u0[n1] = y at depth jb + 8 n1
    SmallDFT<8, true>::run(u1);
    __syncthreads();  // the second depth exchange is read
#pragma unroll
    for (int n1 = 0; n1 < 8; ++n1) {
        E[(jb + 8 * n1) * kFoldPitch + cb] = u0[n1];
        E[(jb + 8 * n1) * kFoldPitch + cb + 32] = u1[n1];
    }
    __syncthreads();
#pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) {
        x0[k2] = E[da * kFoldPitch + 8 * k2 + qa];
        x1[k2] = E[(da + 32) * kFoldPitch + 8 * k2 + qa];
    }
    SmallDFT<8, true>::run(x0);  // x0[p2] = sum_k2 X[k1 + 16 k2] w8^(-p2 k2)
    SmallDFT<8, true>::run(x1);
#pragma unroll
    for (int p2 = 1; p2 < 8; ++p2) {
        float2 w = tw8[k1 * 8 + p2];
        w.y = -w.y;
        x0[p2] = cmul(x0[p2], w);
        x1[p2] = cmul(x1[p2], w);
    }
    pdl_trigger();
#pragma unroll
    for (int p2 = 0; p2 < 8; ++p2) {
        t[a0 + (size_t)p2 * Q] = x0[p2];
        t[a1 + (size_t)p2 * Q] = x1[p2];
    }
}

// The last pass of the split: lane j of column c loads Z[k1][j] from rows 8 k1 + j (k1 < 16), runs
// the 16-point IDFT over k1 and stores x[j + 8 p1] at rows 8 p1 + j, the rows it loaded. 16 columns
// of one slice per 128-thread CTA, unnormalised.
__global__ void __launch_bounds__(128)
col_fold_inv_kernel(float2* t) {
    constexpr int Q = kFoldQ;
    pdl_wait();
    const int c = threadIdx.x % 16, j = threadIdx.x / 16;
    const size_t base = (size_t)blockIdx.y * 128 * Q + (size_t)j * Q + blockIdx.x * 16 + c;
    float2 u[16];
#pragma unroll
    for (int n = 0; n < 16; ++n) u[n] = t[base + (size_t)(8 * n) * Q];
    dft16<true>(u);
    pdl_trigger();
#pragma unroll
    for (int n = 0; n < 16; ++n) t[base + (size_t)(8 * n) * Q] = u[n];
}

template <int N>
size_t row_smem() { return (size_t)(2 * rows_per_cta<N>() * N + N) * sizeof(float2); }
template <int N, int C>
size_t col_smem() { return (size_t)(2 * N * C + N) * sizeof(float2); }

template <typename K>
cudaError_t set_smem(K kern, size_t bytes) {
    if (bytes > 48 * 1024)
        return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    return cudaSuccess;
}

// ---- size dispatch ----
#define RECON_FFT_SIZES(X) X(16) X(32) X(64) X(128) X(192) X(256) X(512)

template <bool INV>
cudaError_t row_fft(int n, const float2* in, float2* out, int nrows, float scale,
                    const float2* tw, cudaStream_t st) {
    switch (n) {
#define CASE(N)                                                                          \
    case N: {                                                                            \
        auto k = row_fft_kernel<N, INV>;                                                 \
        cudaError_t e = set_smem(k, row_smem<N>());                                      \
        if (e != cudaSuccess) return e;                                                  \
        const int grid = (nrows + rows_per_cta<N>() - 1) / rows_per_cta<N>();            \
        k<<<grid, kThreads, row_smem<N>(), st>>>(in, out, nrows, scale, tw);             \
        return cudaGetLastError();                                                       \
    }
        RECON_FFT_SIZES(CASE)
#undef CASE
        default: return cudaErrorInvalidValue;
    }
}

template <int N, int MODE, int C, int S>
cudaError_t col_launch(int Q, int T, int mask_frames, const void* in, float2* out,
                       const uint8_t* mask, float scale, const float2* tw, cudaStream_t st) {
    auto k = col_kernel<N, MODE, C, S>;
    cudaError_t e = set_smem(k, col_smem<N, C>());
    if (e != cudaSuccess) return e;
    dim3 grid(Q / C, T);
    return launch_pdl(k, grid, dim3(kThreads), col_smem<N, C>(), st, in, out, mask, Q, mask_frames,
                      scale, tw);
}

// Tile width C (rounded down to what Q and the shared memory allow; 8 at least) and radix
// schedule S (the adjoint's one-off passes keep schedule 0).
template <int N, int MODE, int S>
cudaError_t col_launch_cs(int C, int Q, int T, int mask_frames, const void* in, float2* out,
                          const uint8_t* mask, float scale, const float2* tw, cudaStream_t st) {
    if constexpr (col_tile_ok<N, 32>()) {
        if (C >= 32 && Q % 32 == 0)
            return col_launch<N, MODE, 32, S>(Q, T, mask_frames, in, out, mask, scale, tw, st);
    }
    if constexpr (col_tile_ok<N, 16>()) {
        if (C >= 16 && Q % 16 == 0)
            return col_launch<N, MODE, 16, S>(Q, T, mask_frames, in, out, mask, scale, tw, st);
    }
    return col_launch<N, MODE, kColTile, S>(Q, T, mask_frames, in, out, mask, scale, tw, st);
}

template <int N, int MODE>
cudaError_t col_launch_c(int C, int S, int Q, int T, int mask_frames, const void* in, float2* out,
                         const uint8_t* mask, float scale, const float2* tw, cudaStream_t st) {
    if constexpr (MODE == COL_FWD || MODE == COL_INV || MODE == COL_MASK_OP) {
        if (S == 1)
            return col_launch_cs<N, MODE, 1>(C, Q, T, mask_frames, in, out, mask, scale, tw, st);
    }
    return col_launch_cs<N, MODE, 0>(C, Q, T, mask_frames, in, out, mask, scale, tw, st);
}

// `T` transforms (frames), the mask of frame f being mask frame f % mask_frames; tiles of C
// columns, radix schedule S.
template <int MODE>
cudaError_t col_pass(int n, int C, int S, int Q, int T, int mask_frames, const void* in,
                     float2* out, const uint8_t* mask, float scale, const float2* tw,
                     cudaStream_t st) {
    switch (n) {
#define CASE(N)                                                                              \
    case N:                                                                                  \
        return col_launch_c<N, MODE>(C, S, Q, T, mask_frames, in, out, mask, scale, tw, st);
        RECON_FFT_SIZES(CASE)
#undef CASE
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

bool fft_size_supported(int n) {
    switch (n) {
#define CASE(N) case N: return true;
        RECON_FFT_SIZES(CASE)
#undef CASE
        default: return false;
    }
}

// Volumes (R > 1): the depth transforms reuse the column kernel with the depth as the transform
// axis and the P * Q voxels of a depth slice as its "columns" (stride P * Q between depth
// samples); the length-P column passes then run over the T * R slices.
// Column tile for the length-P passes (depth = false) or the depth passes of a volume: the
// width the caller chose in Dims (autotuner), else 8 for image series and the wide default for
// volumes.
int col_sched_for(const Dims& d, bool depth) { return depth ? d.depthS : d.colS; }

int col_tile_for(const Dims& d, bool depth) {
    const int chosen = depth ? d.depthC : d.colC;
    if (chosen > 0) return chosen;
    if (d.R == 1) return kColTile;
    return wide_cols(depth ? d.R : d.P);
}

bool vol_fold(const Dims& d) { return d.R == 64 && d.P == 128 && d.Q == 128 && d.nc == 1; }

bool col_register(const Dims& d, bool depth) {
    if (depth) return d.R == 64 && (d.P * d.Q) % 32 == 0;
    if (d.R == 1 && d.P == 256) return true;
    return d.P == 128 && d.Q % 16 == 0;
}

cudaError_t launch_fft2(const Dims& d, const Twiddles& tw, const float2* x, float2* y, int inv,
                        cudaStream_t st) {
    const float sq = 1.0f / sqrtf((float)d.Q), sp = 1.0f / sqrtf((float)d.P);
    const int slices = d.T * d.R;
    const int cP = col_tile_for(d, false), cR = col_tile_for(d, true);
    cudaError_t e = inv ? row_fft<true>(d.Q, x, y, slices * d.P, sq, tw.twQ, st)
                        : row_fft<false>(d.Q, x, y, slices * d.P, sq, tw.twQ, st);
    if (e != cudaSuccess) return e;
    e = inv ? col_pass<COL_INV>(d.P, cP, 0, d.Q, slices, slices, y, y, nullptr, sp, tw.twP, st)
            : col_pass<COL_FWD>(d.P, cP, 0, d.Q, slices, slices, y, y, nullptr, sp, tw.twP, st);
    if (e != cudaSuccess || d.R == 1) return e;
    const float sr = 1.0f / sqrtf((float)d.R);
    const int pq = d.P * d.Q;
    return inv ? col_pass<COL_INV>(d.R, cR, 0, pq, d.T, d.T, y, y, nullptr, sr, tw.twR, st)
               : col_pass<COL_FWD>(d.R, cR, 0, pq, d.T, d.T, y, y, nullptr, sr, tw.twR, st);
}

cudaError_t launch_adjoint(const Dims& d, const Twiddles& tw, const void* b, int b_bf16,
                           const uint8_t* mask, float2* t, float2* x, cudaStream_t st) {
    const float sc = 1.0f / sqrtf((float)d.P * (float)d.Q * (float)d.R);
    cudaError_t e;
    if (d.R > 1) {
        // masked depth IDFT (with the whole 1/sqrt(PQR)), then the column IDFT of every slice
        const int pq = d.P * d.Q, slices = d.T * d.R;
        const int cP = col_tile_for(d, false), cR = col_tile_for(d, true);
        e = b_bf16 ? col_pass<COL_ADJ_BF16>(d.R, cR, 0, pq, d.T, d.T, b, t, mask, sc, tw.twR, st)
                   : col_pass<COL_ADJ_C64>(d.R, cR, 0, pq, d.T, d.T, b, t, mask, sc, tw.twR, st);
        if (e != cudaSuccess) return e;
        e = col_pass<COL_INV>(d.P, cP, 0, d.Q, slices, slices, t, t, nullptr, 1.0f, tw.twP, st);
    } else {
        const int cP = col_tile_for(d, false);
        e = b_bf16 ? col_pass<COL_ADJ_BF16>(d.P, cP, 0, d.Q, d.T, d.T, b, t, mask, sc, tw.twP, st)
                   : col_pass<COL_ADJ_C64>(d.P, cP, 0, d.Q, d.T, d.T, b, t, mask, sc, tw.twP, st);
    }
    if (e != cudaSuccess) return e;
    return row_fft<true>(d.Q, t, x, d.T * d.rows(), 1.0f, tw.twQ, st);
}

cudaError_t launch_row_fwd_pupdate(const Dims& d, const Twiddles& tw, const float2* r, float2* p,
                                   float2* t, const Partials& rr, const double* rr_prev,
                                   double* rr_out, int first, cudaStream_t st) {
    const int nrows = d.T * d.rows();
    if (vol_fold(d))  // the row DFT and the first half of the length-P DFT (see vol_fold)
        return launch_pdl(row_fwd_col1_128_kernel, dim3(d.T * d.R * 8), dim3(128), 0, st, r, p, t,
                          (const double*)rr.parts, rr.n, rr_prev, rr_out, first, tw.twQ);
    if (d.Q == 256) {
        const int grid = (nrows + kR256Rows - 1) / kR256Rows;
        return launch_pdl(row_fwd_pupdate_256_kernel, dim3(grid), dim3(64), 0, st, r, p, t, nrows,
                          (const double*)rr.parts, rr.n, rr_prev, rr_out, first, tw.twQ);
    }
    if (d.Q == 128) {
        const int grid = (nrows + kR128Rows - 1) / kR128Rows;
        return launch_pdl(row_fwd_pupdate_128_kernel, dim3(grid), dim3(64), 0, st, r, p, t, nrows,
                          (const double*)rr.parts, rr.n, rr_prev, rr_out, first, tw.twQ);
    }
    switch (d.Q) {
#define CASE(N)                                                                              \
    case N: {                                                                                \
        auto k = row_fwd_pupdate_kernel<N>;                                                  \
        cudaError_t e = set_smem(k, row_smem<N>());                                          \
        if (e != cudaSuccess) return e;                                                      \
        const int grid = (nrows + rows_per_cta<N>() - 1) / rows_per_cta<N>();                \
        return launch_pdl(k, dim3(grid), dim3(kThreads), row_smem<N>(), st, r, p, t, nrows,  \
                          (const double*)rr.parts, rr.n, rr_prev, rr_out, first, tw.twQ);    \
    }
        RECON_FFT_SIZES(CASE)
#undef CASE
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_coil_row_fwd(const Dims& d, const Twiddles& tw, const float2* r, float2* p,
                                float2* t, const float2* coils, const Partials& rr,
                                const double* rr_prev, double* rr_out, int first, cudaStream_t st) {
    const int nrows = d.T * d.P;
    switch (d.Q) {
#define CASE(N)                                                                              \
    case N: {                                                                                \
        auto k = coil_row_fwd_kernel<N>;                                                     \
        const size_t smem = (size_t)(3 * rows_per_cta<N>() * N + N) * sizeof(float2);       \
        cudaError_t e = set_smem(k, smem);                                                   \
        if (e != cudaSuccess) return e;                                                      \
        const int grid = (nrows + rows_per_cta<N>() - 1) / rows_per_cta<N>();                \
        return launch_pdl(k, dim3(grid), dim3(kThreads), smem, st, r, p, t, coils, nrows,    \
                          d.P, d.nc, (const double*)rr.parts, rr.n, rr_prev, rr_out, first,  \
                          tw.twQ);                                                           \
    }
        RECON_FFT_SIZES(CASE)
#undef CASE
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_adjoint_coils_cols(const Dims& d, const Twiddles& tw, const void* b,
                                      const uint8_t* mask, float2* t, cudaStream_t st) {
    const float sc = 1.0f / sqrtf((float)d.P * (float)d.Q);
    return col_pass<COL_ADJ_C64>(d.P, col_tile_for(d, false), 0, d.Q, d.T * d.nc, d.T, b, t, mask,
                                 sc, tw.twP, st);
}

cudaError_t launch_col_mask(const Dims& d, const Twiddles& tw, float2* t, const uint8_t* mask,
                            cudaStream_t st) {
    if (d.R > 1) {
        // volumes: column DFT of every slice, depth DFT + mask + depth IDFT (with the 1/(PQR)
        // of the two unnormalised transforms), column IDFT of every slice
        const int pq = d.P * d.Q, slices = d.T * d.R;
        const float sc3 = 1.0f / ((float)d.P * (float)d.Q * (float)d.R);
        if (vol_fold(d)) {  // the row pass did the first half of the length-P DFT
            cudaError_t e = launch_pdl(depth_fold_64_kernel, dim3(d.Q / 8, 16, d.T), dim3(256), 0,
                                       st, t, mask, sc3, tw.twP, tw.twR);
            if (e != cudaSuccess) return e;
            return launch_pdl(col_fold_inv_kernel, dim3(d.Q / 16, slices), dim3(128), 0, st, t);
        }
        const int cP = col_tile_for(d, false), cR = col_tile_for(d, true);
        const bool reg128 = col_register(d, false);  // register transforms where they exist
        const bool reg64 = col_register(d, true);
        cudaError_t e =
            reg128 ? launch_pdl(col128_kernel<false>, dim3(d.Q / 16, slices), dim3(128), 0, st, t,
                                d.Q, tw.twP)
                   : col_pass<COL_FWD>(d.P, cP, d.colS, d.Q, slices, slices, t, t, nullptr, 1.0f, tw.twP, st);
        if (e != cudaSuccess) return e;
        e = reg64 ? launch_pdl(col_mask_64_kernel, dim3(pq / 32, d.T), dim3(256), 0, st, t, mask, pq,
                               sc3, tw.twR)
                  : col_pass<COL_MASK_OP>(d.R, cR, d.depthS, pq, d.T, d.T, t, t, mask, sc3, tw.twR, st);
        if (e != cudaSuccess) return e;
        return reg128 ? launch_pdl(col128_kernel<true>, dim3(d.Q / 16, slices), dim3(128), 0, st, t,
                                   d.Q, tw.twP)
                      : col_pass<COL_INV>(d.P, cP, d.colS, d.Q, slices, slices, t, t, nullptr, 1.0f,
                                          tw.twP, st);
    }
    const float sc = 1.0f / ((float)d.P * (float)d.Q);
    const int frames = d.T * d.nc;  // coil-major: the mask of frame f is mask frame f % T
    if (d.P == 256)
        return launch_pdl(col_mask_256_kernel, dim3(d.Q / kColTile, frames), dim3(128), 0, st, t,
                          mask, d.Q, d.T, sc, tw.twP);
    if (col_register(d, false))
        return launch_pdl(col_mask_128_kernel, dim3(d.Q / 16, frames), dim3(128), 0, st, t, mask,
                          d.Q, d.T, sc, tw.twP);
    return col_pass<COL_MASK_OP>(d.P, col_tile_for(d, false), d.colS, d.Q, frames, d.T, t, t, mask,
                                 sc, tw.twP, st);
}

}  // namespace recon
