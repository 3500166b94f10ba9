// CG operator tail, CG vector updates and the warm-start residual carry (Sec. III-A,
// Eq. grad-ls; Algorithm 1, step 2).
//
// The sum-of-squares weight acts per pixel r as a banded frame operator built from the M x M
// Hermitian matrix S(r) (the precomputed G of Eq. grad-ls, the sum of k shifted copies of one
// block product):
//     (W x)_n(r) = sum_{a : 0 <= n-M+1+a < k} sum_b S_ab(r) x_{n+a-b}(r),
// which is sum_j E_j^T S(r) E_j x(r) with (E_j x)(r)[m] = x_{j+M-1-m}(r). S is stored as its
// upper triangle, pair (a <= b) at index a(2M-a+1)/2 + (b-a), layout [pair][P][Q] complex64.
#include "common.cuh"
#include "kernels.h"
#include "regfft.cuh"

namespace recon {

namespace {

constexpr int kThreads = 256;
constexpr int kMaxM = 6;
constexpr int kMaxParts = 4096;  // partial-sum slots (largest grid of a reducing kernel)
constexpr int kUpdVec = 2;       // float4 per thread per iteration in the update pass
constexpr int kUpdThreads = 512;
constexpr int kUpdPerSM = 2;     // update CTAs per SM (few partials for the next pass to add)

// Load S(r) (full M x M from the stored upper triangle) into registers.
template <int M>
RECON_DEV void load_S(const float2* __restrict__ S, size_t npix, size_t px, float2 (&s)[M][M]) {
#pragma unroll
    for (int a = 0; a < M; ++a)
#pragma unroll
        for (int b = a; b < M; ++b) {
            const float2 v = S[(size_t)(a * (2 * M - a + 1) / 2 + (b - a)) * npix + px];
            s[a][b] = v;
            s[b][a] = cconj(v);
        }
}

// Diagonal sums of the per-pixel block: c[M - 1 + d] = sum_{a - b = d} s[a][b], d = -(M-1) ..
// M-1. A frame n whose M windows n - M + 1 + a all exist (every frame of the circular lifting)
// has (W x)_n = sum_d c[M - 1 + d] x_{n+d}: 2M - 1 products instead of M^2. s is Hermitian, so
// c[M - 1 - d] = conj(c[M - 1 + d]).
template <int M>
RECON_DEV void s_diagonals(const float2 (&s)[M][M], float2 (&c)[2 * M - 1]) {
#pragma unroll
    for (int d = 0; d < M; ++d) {
        float2 v = make_float2(0.f, 0.f);
#pragma unroll
        for (int a = d; a < M; ++a) v = cadd(v, s[a][a - d]);
        c[M - 1 + d] = v;
        if (d > 0) c[M - 1 - d] = cconj(v);
    }
}

// (W x)_n at one pixel, from the frame values xs[f * stride] (0 <= f < T), the block s and its
// diagonal sums c: the diagonal form where all M windows of frame n exist (for 3 <= M <= 5,
// where it saves products and the block and its sums fit the registers; the circular lifting
// always), else the window sum.
template <int M, bool CIRC>
RECON_DEV float2 w_frame(const float2 (&s)[M][M], const float2 (&c)[2 * M - 1],
                         const float2* xs, int stride, int n, int T, int k) {
    float2 w = make_float2(0.f, 0.f);
    if (CIRC || (M >= 3 && M <= 5 && n >= M - 1 && n < k)) {
#pragma unroll
        for (int d = 0; d < 2 * M - 1; ++d) {
            const int f = n + d - (M - 1);
            w = cfma(c[d], xs[(CIRC ? wrap_frame(f, T) : f) * stride], w);
        }
        return w;
    }
#pragma unroll
    for (int a = 0; a < M; ++a) {
        const int j = n - M + 1 + a;
        if (j < 0 || j >= k) continue;
#pragma unroll
        for (int b = 0; b < M; ++b) w = cfma(s[a][b], xs[(n + a - b) * stride], w);
    }
    return w;
}

// Pass C of a CG step. One CTA per image row r1 holds that row of every frame: it inverse-
// transforms the k-space rows of t (giving A^H A p; the 1/(PQ) scale was applied with the mask),
// adds lam W p from the p rows, writes q over t and emits the partial Re <p, q> of its row.
template <int N, int M, bool CIRC>
__global__ void __launch_bounds__(kThreads)
row_inv_w_kernel(float2* t, const float2* __restrict__ p, const float2* __restrict__ S,
                 float lam, int T, int P, double* __restrict__ pq_parts,
                 const float2* __restrict__ tw_g) {
    extern __shared__ float2 sm[];
    __shared__ double red[kThreads / 32];
    float2* a = sm;
    float2* b = a + (size_t)T * N;
    float2* pt = b + (size_t)T * N;
    float2* tw = pt + (size_t)T * N;
    const size_t npix = (size_t)P * N;
    for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = tw_g[i];
    pdl_wait();
    const int k = CIRC ? T : T - M + 1;
    float acc = 0.f, comp = 0.f;  // Kahan-compensated per-thread partial of Re <p, q>
    for (int r1 = blockIdx.x; r1 < P; r1 += gridDim.x) {
    __syncthreads();  // the previous row's results are stored
    for (int e = threadIdx.x; e < T * N; e += blockDim.x) {
        const int n = e / N, c = e % N;
        const size_t g = (size_t)n * npix + (size_t)r1 * N + c;
        a[e] = t[g];
        pt[e] = p[g];
    }
    __syncthreads();
    float2* res = fft_smem<N, true, false>(a, b, T, N, 1, tw);
    for (int c = threadIdx.x; c < N; c += blockDim.x) {
        float2 s[M][M];
        load_S<M>(S, npix, (size_t)r1 * N + c, s);
        float2 cs[2 * M - 1];
        s_diagonals<M>(s, cs);
        for (int n = 0; n < T; ++n) {
            const float2 w = w_frame<M, CIRC>(s, cs, pt + c, N, n, T, k);
            float2 q = res[n * N + c];
            q.x = fmaf(lam, w.x, q.x);
            q.y = fmaf(lam, w.y, q.y);
            res[n * N + c] = q;
            const float2 pv = pt[n * N + c];
            const float term = fmaf(pv.x, q.x, pv.y * q.y) - comp;
            const float sum = acc + term;
            comp = (sum - acc) - term;
            acc = sum;
        }
    }
    __syncthreads();  // every column of q written
    if (r1 + (int)gridDim.x >= P) pdl_trigger();
    for (int e = threadIdx.x; e < T * N; e += blockDim.x) {
        const int n = e / N, c = e % N;
        t[(size_t)n * npix + (size_t)r1 * N + c] = res[e];
    }
    }
    const double tot = block_sum_f_t0(acc, red);
    if (threadIdx.x == 0) pq_parts[blockIdx.x] = tot;
}

// Pass C for 256-point rows: one CTA per image row r1 with 16 threads per frame; the inverse row
// transforms run in registers (regfft.cuh), the rest as in row_inv_w_kernel. The block is padded
// to a multiple of 16 frames (256 threads), at least 32: warps without a frame skip the
// transform, and the W phase gives each column blockDim / 256 threads, each with a contiguous
// range of frames. Shared memory: p rows [T][256], then the exchange buffers [T'][16 x 17] (T' = T
// rounded up to even, the frames of the warps that transform) which afterwards hold the
// transformed rows [T][256].
template <int M>
__global__ void __launch_bounds__(1024)
row_inv_w_256_kernel(float2* t, const float2* __restrict__ p, const float2* __restrict__ S,
                     float lam, int T, int P, double* __restrict__ pq_parts,
                     const float2* __restrict__ tw_g) {
    constexpr int N = 256;
    extern __shared__ float2 sm[];
    __shared__ float2 tw2[256];
    __shared__ double red[32];
    float2* pt = sm;
    float2* res = sm + (size_t)T * N;
    fill_tw256(tw2, tw_g);
    pdl_wait();
    const int n = threadIdx.x / 16, j = threadIdx.x % 16;
    const bool live = n < T;                            // the block is padded (see the launch)
    const bool warp_live = (threadIdx.x / 32) * 2 < T;  // a warp holds frames 2w and 2w + 1
    const size_t npix = (size_t)P * N;
    const int k = T - M + 1;
    float acc = 0.f, comp = 0.f;  // Kahan-compensated per-thread partial of Re <p, q>
    for (int r1 = blockIdx.x; r1 < P; r1 += gridDim.x) {
    __syncthreads();  // the previous row's results are stored
    const size_t g0 = (size_t)n * npix + (size_t)r1 * N + j;
    float2 u[16];
#pragma unroll
    for (int n1 = 0; n1 < 16; ++n1) {
        u[n1] = make_float2(0.f, 0.f);
        if (live) {
            u[n1] = t[g0 + 16 * n1];
            pt[n * N + 16 * n1 + j] = p[g0 + 16 * n1];
        }
    }
    __syncthreads();  // tw2
    if (warp_live) row_dft256<true>(u, res + n * (16 * 17), tw2, j);  // warp-uniform
    __syncthreads();  // every exchange buffer read
    if (live) {
#pragma unroll
        for (int k2 = 0; k2 < 16; ++k2) res[n * N + j + 16 * k2] = u[k2];
    }
    __syncthreads();
    {   // W phase: column c, frames [f0, f1) of this thread's group (blockDim.x = ng N)
        const int c = threadIdx.x % N, ng = blockDim.x / N, g = threadIdx.x / N;
        const int f0 = g * T / ng, f1 = (g + 1) * T / ng;
        float2 s[M][M];
        load_S<M>(S, npix, (size_t)r1 * N + c, s);
        float2 cs[2 * M - 1];
        s_diagonals<M>(s, cs);
        for (int nn = f0; nn < f1; ++nn) {
            const float2 w = w_frame<M, false>(s, cs, pt + c, N, nn, T, k);
            float2 q = res[nn * N + c];
            q.x = fmaf(lam, w.x, q.x);
            q.y = fmaf(lam, w.y, q.y);
            res[nn * N + c] = q;
            const float2 pv = pt[nn * N + c];
            const float term = fmaf(pv.x, q.x, pv.y * q.y) - comp;
            const float sum = acc + term;
            comp = (sum - acc) - term;
            acc = sum;
        }
    }
    __syncthreads();  // every column of q written
    if (r1 + (int)gridDim.x >= P) pdl_trigger();
    for (int e = threadIdx.x; e < T * N; e += blockDim.x) {
        const int nn = e / N, c = e % N;
        t[(size_t)nn * npix + (size_t)r1 * N + c] = res[e];
    }
    }
    const double tot = block_sum_f_t0(acc, red);
    if (threadIdx.x == 0) pq_parts[blockIdx.x] = tot;
}

// Pass C for 128-point rows: as row_inv_w_256_kernel with 8 threads per frame (row_dft128), the
// block padded to at least 16 frames (128 threads, one column each in the W phase) and at most
// 64; warps without a frame skip the transform. A CTA usually owns several rows (volumes have
// R P rows), so the inputs of its next row are staged into shared memory by asynchronous copies
// while the current one is processed: the p rows (double-buffered) as the row starts, the t rows
// once the current ones are in registers, the S row once the current one has been used. Shared
// memory: p rows [2][T][128], t rows [T][128], S row [npair][128], then the exchange buffers
// [T4][kX128] (T4 = T rounded up to whole warps) which afterwards hold the transformed rows.
template <int M>
__global__ void __launch_bounds__(512)
row_inv_w_128_kernel(float2* t, const float2* __restrict__ p, const float2* __restrict__ S,
                     float lam, int T, int P, double* __restrict__ pq_parts,
                     const float2* __restrict__ tw_g) {
    constexpr int N = 128;
    constexpr int NP = M * (M + 1) / 2;
    extern __shared__ __align__(16) float2 sm[];
    __shared__ float2 tw8[128];
    __shared__ double red[32];
    const int TN = T * N;
    float2* pst = sm;             // [2][T][N]
    float2* tst = sm + 2 * TN;    // [T][N]
    float2* sst = tst + TN;       // [NP][N]
    float2* res = sst + NP * N;   // [T4][kX128]
    fill_tw128(tw8, tw_g);
    pdl_wait();
    const int n = threadIdx.x / 8, j = threadIdx.x % 8;
    const bool live = n < T;
    const bool warp_live = (threadIdx.x / 32) * 4 < T;  // a warp holds frames 4w .. 4w + 3
    const size_t npix = (size_t)P * N;
    const int k = T - M + 1;
    // 16-byte copies of `rows` rows of N values, row f from src + f * stride, to dst + f * N
    auto stage = [&](float2* dst, const float2* src, size_t stride, int rows) {
        for (int e = threadIdx.x; e < rows * (N / 2); e += blockDim.x) {
            const int f = e / (N / 2), c2 = 2 * (e % (N / 2));
            cp_async16(dst + f * N + c2, src + f * stride + c2);
        }
        cp_async_commit();
    };
    float acc = 0.f, comp = 0.f;  // Kahan-compensated per-thread partial of Re <p, q>
    int buf = 0;
    if ((int)blockIdx.x < P) {
        const size_t r0 = (size_t)blockIdx.x * N;
        stage(pst, p + r0, npix, T);
        stage(tst, t + r0, npix, T);
        stage(sst, S + r0, npix, NP);
    }
    for (int r1 = blockIdx.x; r1 < P; r1 += gridDim.x, buf ^= 1) {
    const int nxt = r1 + gridDim.x;
    const size_t rn = (size_t)nxt * N;
    cp_async_wait<0>();
    __syncthreads();  // this row's copies landed (every thread's); tw8; the previous row stored
    // the other p buffer was last read before the previous row's final barrier
    if (nxt < P) stage(pst + (buf ^ 1) * TN, p + rn, npix, T);
    float2 a[8], b[8];
    if (warp_live) {  // warp-uniform
        float2 u[16];
#pragma unroll
        for (int n1 = 0; n1 < 16; ++n1) u[n1] = live ? tst[n * N + 8 * n1 + j] : make_float2(0.f, 0.f);
        row_dft128<true>(u, a, b, res + n * kX128, tw8, j);
    }
    __syncthreads();  // every exchange buffer read; every t row in registers
    if (nxt < P) stage(tst, t + rn, npix, T);
    if (live) {
#pragma unroll
        for (int k2 = 0; k2 < 8; ++k2) {
            res[n * N + 2 * j + 16 * k2] = a[k2];
            res[n * N + 2 * j + 1 + 16 * k2] = b[k2];
        }
    }
    __syncthreads();
    const float2* pt = pst + buf * TN;
    for (int c = threadIdx.x; c < N; c += blockDim.x) {
        float2 s[M][M];  // S(r) from the staged row, pair (a <= b) at a(2M-a+1)/2 + (b-a)
#pragma unroll
        for (int aa = 0; aa < M; ++aa)
#pragma unroll
            for (int bb = aa; bb < M; ++bb) {
                const float2 v = sst[(aa * (2 * M - aa + 1) / 2 + (bb - aa)) * N + c];
                s[aa][bb] = v;
                s[bb][aa] = cconj(v);
            }
        float2 cs[2 * M - 1];
        s_diagonals<M>(s, cs);
        for (int nn = 0; nn < T; ++nn) {
            const float2 w = w_frame<M, false>(s, cs, pt + c, N, nn, T, k);
            float2 q = res[nn * N + c];
            q.x = fmaf(lam, w.x, q.x);
            q.y = fmaf(lam, w.y, q.y);
            res[nn * N + c] = q;
            const float2 pv = pt[nn * N + c];
            const float term = fmaf(pv.x, q.x, pv.y * q.y) - comp;
            const float sum = acc + term;
            comp = (sum - acc) - term;
            acc = sum;
        }
    }
    __syncthreads();  // every column of q written; the S row used
    if (nxt < P) stage(sst, S + rn, npix, NP);
    else pdl_trigger();
    float2* trow = t + (size_t)r1 * N;
    for (int e = threadIdx.x; e < TN; e += blockDim.x) {
        const int nn = e / N, c = e % N;
        trow[nn * npix + c] = res[e];
    }
    }
    const double tot = block_sum_f_t0(acc, red);
    if (threadIdx.x == 0) pq_parts[blockIdx.x] = tot;
}

// Pass C of a CG step with coils (ADJ = false), or the coil combination of the adjoint
// (ADJ = true). One CTA per image row r1 holds that row of every frame: for each coil c it
// inverse-transforms the rows t[c][n][r1] and accumulates conj(C_c) * (...) (Eq.
// measurement-ij: A^H = sum_c conj(C_c) F^H mask). ADJ: the sum is x[n][r1]. Otherwise lam W p is
// added from the p rows, q goes over coil 0's plane of t (rows r1, read by this CTA only) and the
// row's partial Re <p, q> to pq_parts.
template <int N, int M, bool ADJ>
__global__ void __launch_bounds__(kThreads)
coil_row_inv_kernel(float2* t, const float2* __restrict__ p, const float2* __restrict__ coils,
                    const float2* __restrict__ S, float lam, int T, int P, int nc,
                    double* __restrict__ pq_parts, float2* __restrict__ x_out,
                    const float2* __restrict__ tw_g) {
    extern __shared__ float2 sm[];
    __shared__ double red[kThreads / 32];
    float2* a = sm;
    float2* b = a + (size_t)T * N;
    float2* acc = b + (size_t)T * N;
    float2* pt = acc + (size_t)T * N;
    float2* tw = pt + (size_t)T * N;
    const int r1 = blockIdx.x;
    const size_t npix = (size_t)P * N;
    const size_t series = (size_t)T * npix;
    for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = tw_g[i];
    pdl_wait();
    for (int e = threadIdx.x; e < T * N; e += blockDim.x) {
        acc[e] = make_float2(0.f, 0.f);
        if (!ADJ) pt[e] = p[(size_t)(e / N) * npix + (size_t)r1 * N + e % N];
    }
    for (int c = 0; c < nc; ++c) {
        __syncthreads();  // a, b free again
        for (int e = threadIdx.x; e < T * N; e += blockDim.x)
            a[e] = t[c * series + (size_t)(e / N) * npix + (size_t)r1 * N + e % N];
        __syncthreads();
        float2* res = fft_smem<N, true, false>(a, b, T, N, 1, tw);
        for (int e = threadIdx.x; e < T * N; e += blockDim.x) {
            const float2 cv = coils[((size_t)c * P + r1) * N + e % N];
            acc[e] = cfmacj(cv, res[e], acc[e]);
        }
    }
    __syncthreads();
    if constexpr (ADJ) {
        pdl_trigger();
        for (int e = threadIdx.x; e < T * N; e += blockDim.x)
            x_out[(size_t)(e / N) * npix + (size_t)r1 * N + e % N] = acc[e];
        return;
    } else {
        const int k = T - M + 1;
        float accd = 0.f, comp = 0.f;  // Kahan-compensated per-thread partial of Re <p, q>
        for (int c = threadIdx.x; c < N; c += blockDim.x) {
            float2 s[M][M];
            load_S<M>(S, npix, (size_t)r1 * N + c, s);
            for (int n = 0; n < T; ++n) {
                float2 w = make_float2(0.f, 0.f);
#pragma unroll
                for (int aa = 0; aa < M; ++aa) {
                    const int j = n - M + 1 + aa;
                    if (j < 0 || j >= k) continue;
#pragma unroll
                    for (int bb = 0; bb < M; ++bb)
                    w = cfma(s[aa][bb], pt[wrap_frame(n + aa - bb, T) * N + c], w);
                }
                float2 q = acc[n * N + c];
                q.x = fmaf(lam, w.x, q.x);
                q.y = fmaf(lam, w.y, q.y);
                acc[n * N + c] = q;
                const float2 pv = pt[n * N + c];
                const float term = fmaf(pv.x, q.x, pv.y * q.y) - comp;
                const float sum = accd + term;
                comp = (sum - accd) - term;
                accd = sum;
            }
        }
        const double tot = block_sum_f_t0(accd, red);
        pdl_trigger();
        for (int e = threadIdx.x; e < T * N; e += blockDim.x)
            t[(size_t)(e / N) * npix + (size_t)r1 * N + e % N] = acc[e];
        if (threadIdx.x == 0) pq_parts[blockIdx.x] = tot;
    }
}

// Pass D: alpha = |r|^2 / Re <p, q> (Re <p, q> summed here from pass C's partials); x += alpha p;
// r -= alpha q; per-CTA partials of |r_new|^2 for the next pass A.
__global__ void __launch_bounds__(kUpdThreads, kUpdPerSM)
cg_update_kernel(float4* __restrict__ x, float4* __restrict__ r, const float4* __restrict__ p,
                 const float4* __restrict__ q, size_t n4, const double* __restrict__ rr_in,
                 const double* __restrict__ pq_parts, int n_pq, double* __restrict__ rr_parts) {
    __shared__ double red[kUpdThreads / 32];
    __shared__ double s_pq;
    __shared__ float alpha_s;
    pdl_wait();
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    size_t i0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    float4 xv[kUpdVec], rv[kUpdVec], pv[kUpdVec], qv[kUpdVec];
    // the first loads go out before alpha is known (they do not depend on it)
#pragma unroll
    for (int u = 0; u < kUpdVec; ++u) {
        const size_t i = i0 + (size_t)u * stride;
        if (i < n4) { xv[u] = x[i]; rv[u] = r[i]; pv[u] = p[i]; qv[u] = q[i]; }
    }
    const double pq = sum_partials(pq_parts, n_pq, &s_pq);
    if (threadIdx.x == 0) alpha_s = (float)(rr_in[0] * rcp_nr(pq));
    __syncthreads();
    const float alpha = alpha_s;
    float acc = 0.f, comp = 0.f;
    for (; i0 < n4; i0 += stride * kUpdVec) {
#pragma unroll
        for (int u = 0; u < kUpdVec; ++u) {
            const size_t i = i0 + (size_t)u * stride;
            if (i >= n4) continue;
            xv[u].x = fmaf(alpha, pv[u].x, xv[u].x);
            xv[u].y = fmaf(alpha, pv[u].y, xv[u].y);
            xv[u].z = fmaf(alpha, pv[u].z, xv[u].z);
            xv[u].w = fmaf(alpha, pv[u].w, xv[u].w);
            rv[u].x = fmaf(-alpha, qv[u].x, rv[u].x);
            rv[u].y = fmaf(-alpha, qv[u].y, rv[u].y);
            rv[u].z = fmaf(-alpha, qv[u].z, rv[u].z);
            rv[u].w = fmaf(-alpha, qv[u].w, rv[u].w);
            x[i] = xv[u];
            r[i] = rv[u];
            const float4 w = rv[u];
            const float term = fmaf(w.x, w.x, fmaf(w.y, w.y, fmaf(w.z, w.z, w.w * w.w))) - comp;
            const float sum = acc + term;
            comp = (sum - acc) - term;
            acc = sum;
        }
        const size_t nx = i0 + stride * kUpdVec;
#pragma unroll
        for (int u = 0; u < kUpdVec; ++u) {
            const size_t i = nx + (size_t)u * stride;
            if (i < n4) { xv[u] = x[i]; rv[u] = r[i]; pv[u] = p[i]; qv[u] = q[i]; }
        }
    }
    pdl_trigger();
    const double tot = block_sum_f_t0(acc, red);
    if (threadIdx.x == 0) rr_parts[blockIdx.x] = tot;
}

__global__ void sum_partials_kernel(const double* __restrict__ parts, int n, double* __restrict__ out) {
    const double v = warp0_sum_array(parts, n);
    if (threadIdx.x == 0) out[0] = v;
}

// Residual carry between IRLS iterations: r = (first ? r0 : r) + lam W_{dS} x with
// dS = S_old - S_new (or -S_new when first); partial |r|^2. One thread per pixel, all frames.
// r0 = A^H b - A^H A x0 = x0 - A^H A x0 for x0 = A^H b: zero for one coil and 0/1 masks (A A^H
// is then a projection), x0 - aha_x when A^H A x0 is supplied (coils).
template <int M>
__global__ void __launch_bounds__(kThreads)
resid_carry_kernel(float2* __restrict__ r, const float2* __restrict__ x,
                   const float2* __restrict__ aha_x, const float2* __restrict__ S_old,
                   const float2* __restrict__ S_new, float lam, int first, int T, int circ,
                   size_t npix,
                   double* __restrict__ parts, unsigned int* counter,
                   double* __restrict__ rr_out) {
    __shared__ double red[kThreads / 32];
    const int k = circ ? T : T - M + 1;
    float acc = 0.f, comp = 0.f;
    for (size_t px = (size_t)blockIdx.x * blockDim.x + threadIdx.x; px < npix;
         px += (size_t)gridDim.x * blockDim.x) {
        float2 s[M][M];
        load_S<M>(S_new, npix, px, s);
        if (first) {
#pragma unroll
            for (int a = 0; a < M; ++a)
#pragma unroll
                for (int b = 0; b < M; ++b) s[a][b] = make_float2(-s[a][b].x, -s[a][b].y);
        } else {
            float2 so[M][M];
            load_S<M>(S_old, npix, px, so);
#pragma unroll
            for (int a = 0; a < M; ++a)
#pragma unroll
                for (int b = 0; b < M; ++b) s[a][b] = csub(so[a][b], s[a][b]);
        }
        for (int n = 0; n < T; ++n) {
            float2 w = make_float2(0.f, 0.f);
#pragma unroll
            for (int a = 0; a < M; ++a) {
                const int j = n - M + 1 + a;
                if (!circ && (j < 0 || j >= k)) continue;  // circ: every window
#pragma unroll
                for (int b = 0; b < M; ++b)
                    w = cfma(s[a][b], x[(size_t)wrap_frame(n + a - b, T) * npix + px], w);
            }
            float2 rv = make_float2(0.f, 0.f);
            if (!first) {
                rv = r[(size_t)n * npix + px];
            } else if (aha_x) {  // x0 - A^H A x0 (coils: A A^H is no projection)
                const float2 xv = x[(size_t)n * npix + px], av = aha_x[(size_t)n * npix + px];
                rv = make_float2(xv.x - av.x, xv.y - av.y);
            }
            rv.x = fmaf(lam, w.x, rv.x);
            rv.y = fmaf(lam, w.y, rv.y);
            r[(size_t)n * npix + px] = rv;
            const float term = fmaf(rv.x, rv.x, rv.y * rv.y) - comp;
            const float sum = acc + term;
            comp = (sum - acc) - term;
            acc = sum;
        }
    }
    const double tot = block_sum_f_t0(acc, red);
    last_block_sum(tot, parts, counter, rr_out);
}

// max_r | |C(r)|^2 - 1 | of one coil map into *dev (non-negative float bits: atomicMax exact).
__global__ void __launch_bounds__(kThreads)
coil_unimodular_kernel(const float2* __restrict__ C, size_t npix, unsigned int* __restrict__ dev) {
    float m = 0.f;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < npix;
         i += (size_t)gridDim.x * blockDim.x) {
        const float2 v = C[i];
        m = fmaxf(m, fabsf(fmaf(v.x, v.x, v.y * v.y) - 1.f));
    }
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 16));
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 8));
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 4));
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 2));
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 1));
    if ((threadIdx.x & 31) == 0) atomicMax(dev, __float_as_uint(m));
}

// y = W_S x (no lambda); parity tests only.
template <int M>
__global__ void __launch_bounds__(kThreads)
apply_w_kernel(const float2* __restrict__ x, const float2* __restrict__ S, float2* __restrict__ y,
               int T, int circ, size_t npix) {
    const int k = circ ? T : T - M + 1;
    for (size_t px = (size_t)blockIdx.x * blockDim.x + threadIdx.x; px < npix;
         px += (size_t)gridDim.x * blockDim.x) {
        float2 s[M][M];
        load_S<M>(S, npix, px, s);
        for (int n = 0; n < T; ++n) {
            float2 w = make_float2(0.f, 0.f);
#pragma unroll
            for (int a = 0; a < M; ++a) {
                const int j = n - M + 1 + a;
                if (!circ && (j < 0 || j >= k)) continue;  // circ: every window
#pragma unroll
                for (int b = 0; b < M; ++b)
                    w = cfma(s[a][b], x[(size_t)wrap_frame(n + a - b, T) * npix + px], w);
            }
            y[(size_t)n * npix + px] = w;
        }
    }
}

// Grid of a row kernel: one CTA per row while the rows fit one resident wave, else one wave
// (the CTAs then loop over rows), so that the pass leaves at most a wave of partials.
template <typename K>
cudaError_t row_grid(K kern, int threads, size_t smem, int rows, int* grid) {
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    if (e != cudaSuccess) return e;
    long long wave = (long long)(per_sm < 1 ? 1 : per_sm) * num_sms();
    if (wave > kMaxParts) wave = kMaxParts;
    *grid = rows < wave ? rows : (int)wave;
    return cudaSuccess;
}

template <int N, int M>
cudaError_t launch_row_inv_w_NM(const Dims& d, const Twiddles& tw, float2* t, const float2* p,
                                const float2* S, float lam, Partials* pq, cudaStream_t st) {
    const int rows = d.rows();
    int grid = 0;
    if (N == 128 && !d.circ) {  // register transforms for the valid (non-circular) lifting
        // whole warps, and at least 128 threads so that the W phase has one column per thread
        const int tpad = d.T <= 16 ? 16 : (d.T + 3) / 4 * 4;
        const int t4 = (d.T + 3) / 4 * 4;  // frames of the warps that transform
        const size_t smem128 =
            ((size_t)3 * d.T * N + (size_t)d.M * (d.M + 1) / 2 * N + (size_t)t4 * kX128) * sizeof(float2);
        if (tpad * 8 <= 512 && smem128 <= 200 * 1024) {
            auto k = row_inv_w_128_kernel<M>;
            if (smem128 > 48 * 1024) {
                cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     (int)smem128);
                if (e != cudaSuccess) return e;
            }
            cudaError_t e = row_grid(k, tpad * 8, smem128, rows, &grid);
            if (e != cudaSuccess) return e;
            pq->n = grid;
            return launch_pdl(k, dim3(grid), dim3(tpad * 8), smem128, st, t, p, S, lam, d.T, rows,
                              pq->parts, tw.twQ);
        }
    }
    if (N == 256 && !d.circ) {  // the register kernel serves the valid (non-circular) lifting
        const int t2 = (d.T + 1) / 2 * 2;                          // frames that transform
        const int tpad = d.T <= 32 ? 32 : (d.T + 15) / 16 * 16;   // frames of the block
        const size_t smem256 = ((size_t)d.T * N + (size_t)t2 * 16 * 17) * sizeof(float2);
        if (tpad * 16 <= 1024 && smem256 <= 200 * 1024) {
            auto k = row_inv_w_256_kernel<M>;
            if (smem256 > 48 * 1024) {
                cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     (int)smem256);
                if (e != cudaSuccess) return e;
            }
            cudaError_t e = row_grid(k, tpad * 16, smem256, rows, &grid);
            if (e != cudaSuccess) return e;
            pq->n = grid;
            return launch_pdl(k, dim3(grid), dim3(tpad * 16), smem256, st, t, p, S, lam, d.T, rows,
                              pq->parts, tw.twQ);
        }
    }
    auto k = d.circ ? row_inv_w_kernel<N, M, true> : row_inv_w_kernel<N, M, false>;
    const size_t smem = ((size_t)3 * d.T * N + N) * sizeof(float2);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = row_grid(k, kThreads, smem, rows, &grid);
    if (e != cudaSuccess) return e;
    pq->n = grid;
    return launch_pdl(k, dim3(grid), dim3(kThreads), smem, st, t, p, S, lam, d.T, rows,
                      pq->parts, tw.twQ);
}

template <int N>
cudaError_t launch_row_inv_w_N(const Dims& d, const Twiddles& tw, float2* t, const float2* p,
                               const float2* S, float lam, Partials* pq, cudaStream_t st) {
    switch (d.M) {
        case 1: return launch_row_inv_w_NM<N, 1>(d, tw, t, p, S, lam, pq, st);
        case 2: return launch_row_inv_w_NM<N, 2>(d, tw, t, p, S, lam, pq, st);
        case 3: return launch_row_inv_w_NM<N, 3>(d, tw, t, p, S, lam, pq, st);
        case 4: return launch_row_inv_w_NM<N, 4>(d, tw, t, p, S, lam, pq, st);
        case 5: return launch_row_inv_w_NM<N, 5>(d, tw, t, p, S, lam, pq, st);
        case 6: return launch_row_inv_w_NM<N, 6>(d, tw, t, p, S, lam, pq, st);
        default: return cudaErrorInvalidValue;
    }
}

int pix_grid(size_t npix) {
    const size_t g = (npix + kThreads - 1) / kThreads;
    return (int)(g < (size_t)kMaxParts ? g : (size_t)kMaxParts);
}

// One resident wave: kUpdPerSM CTAs per SM (fewer for small problems), grid-stride inside.
int upd_grid(size_t n4) {
    const size_t per = (size_t)kUpdThreads * kUpdVec;
    const size_t need = (n4 + per - 1) / per;
    size_t g = (size_t)num_sms() * kUpdPerSM;
    if (need < g) g = need;
    return (int)(g < 1 ? 1 : (g < (size_t)kMaxParts ? g : (size_t)kMaxParts));
}

template <int N, int M, bool ADJ>
cudaError_t launch_coil_inv_NM(const Dims& d, const Twiddles& tw, float2* t, const float2* p,
                               const float2* coils, const float2* S, float lam, double* pq_parts,
                               float2* x_out, cudaStream_t st) {
    auto k = coil_row_inv_kernel<N, M, ADJ>;
    const size_t smem = ((size_t)4 * d.T * N + N) * sizeof(float2);
    if (smem > 220 * 1024) return cudaErrorInvalidValue;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    return launch_pdl(k, dim3(d.P), dim3(kThreads), smem, st, t, p, coils, S, lam, d.T, d.P, d.nc,
                      pq_parts, x_out, tw.twQ);
}

template <int N, bool ADJ>
cudaError_t launch_coil_inv_N(const Dims& d, const Twiddles& tw, float2* t, const float2* p,
                              const float2* coils, const float2* S, float lam, double* pq_parts,
                              float2* x_out, cudaStream_t st) {
    if constexpr (ADJ) {
        return launch_coil_inv_NM<N, 1, true>(d, tw, t, p, coils, S, lam, pq_parts, x_out, st);
    } else {
        switch (d.M) {
#define CASE(MM) \
    case MM: return launch_coil_inv_NM<N, MM, false>(d, tw, t, p, coils, S, lam, pq_parts, x_out, st);
            CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6)
#undef CASE
            default: return cudaErrorInvalidValue;
        }
    }
}

template <bool ADJ>
cudaError_t launch_coil_inv(const Dims& d, const Twiddles& tw, float2* t, const float2* p,
                            const float2* coils, const float2* S, float lam, double* pq_parts,
                            float2* x_out, cudaStream_t st) {
    if (d.P > kMaxParts) return cudaErrorInvalidValue;
    switch (d.Q) {
#define CASE(NN) \
    case NN: return launch_coil_inv_N<NN, ADJ>(d, tw, t, p, coils, S, lam, pq_parts, x_out, st);
        CASE(16) CASE(32) CASE(64) CASE(128) CASE(192) CASE(256) CASE(512)
#undef CASE
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

int num_sms() {
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 132;
    if (!cache[dev]) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 132;
        cache[dev] = n;
    }
    return cache[dev];
}

int w_max_M() { return kMaxM; }
int w_max_frames_times_q() { return (200 * 1024) / (3 * (int)sizeof(float2)); }
int max_parts() { return kMaxParts; }

cudaError_t launch_row_inv_w(const Dims& d, const Twiddles& tw, float2* t, const float2* p,
                             const float2* S, float lam, Partials* pq, cudaStream_t st) {
    switch (d.Q) {
        case 16: return launch_row_inv_w_N<16>(d, tw, t, p, S, lam, pq, st);
        case 32: return launch_row_inv_w_N<32>(d, tw, t, p, S, lam, pq, st);
        case 64: return launch_row_inv_w_N<64>(d, tw, t, p, S, lam, pq, st);
        case 128: return launch_row_inv_w_N<128>(d, tw, t, p, S, lam, pq, st);
        case 192: return launch_row_inv_w_N<192>(d, tw, t, p, S, lam, pq, st);
        case 256: return launch_row_inv_w_N<256>(d, tw, t, p, S, lam, pq, st);
        case 512: return launch_row_inv_w_N<512>(d, tw, t, p, S, lam, pq, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_coil_row_inv_w(const Dims& d, const Twiddles& tw, float2* t, const float2* p,
                                  const float2* coils, const float2* S, float lam, Partials* pq,
                                  cudaStream_t st) {
    pq->n = d.P;
    return launch_coil_inv<false>(d, tw, t, p, coils, S, lam, pq->parts, nullptr, st);
}

cudaError_t launch_coil_combine(const Dims& d, const Twiddles& tw, float2* t, const float2* coils,
                                float2* x, cudaStream_t st) {
    return launch_coil_inv<true>(d, tw, t, nullptr, coils, nullptr, 0.f, nullptr, x, st);
}

cudaError_t launch_cg_update(const Dims& d, float2* x, float2* r, const float2* p,
                             const float2* q, const double* rr_in, const Partials& pq,
                             Partials* rr, cudaStream_t st) {
    const size_t n4 = d.elems() / 2;  // two complex values per float4
    const int grid = upd_grid(n4);
    rr->n = grid;
    return launch_pdl(cg_update_kernel, dim3(grid), dim3(kUpdThreads), 0, st,
                      reinterpret_cast<float4*>(x), reinterpret_cast<float4*>(r),
                      reinterpret_cast<const float4*>(p), reinterpret_cast<const float4*>(q), n4,
                      rr_in, (const double*)pq.parts, pq.n, rr->parts);
}

cudaError_t launch_sum_partials(const Partials& in, double* out, cudaStream_t st) {
    sum_partials_kernel<<<1, 32, 0, st>>>(in.parts, in.n, out);
    return cudaGetLastError();
}

cudaError_t launch_resid_carry(const Dims& d, float2* r, const float2* x, const float2* S_old,
                               const float2* S_new, float lam, int first, const RedSlot& rs,
                               double* rr_out, cudaStream_t st, const float2* aha_x) {
    const int g = pix_grid(d.pixels());
#define CASE(MM)                                                                              \
    case MM:                                                                                  \
        resid_carry_kernel<MM><<<g, kThreads, 0, st>>>(r, x, aha_x, S_old, S_new, lam, first, \
                                                       d.T, d.circ, d.pixels(), rs.parts,     \
                                                       rs.counter,                            \
                                                       rr_out);                               \
        break;
    switch (d.M) {
        CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6)
        default: return cudaErrorInvalidValue;
    }
#undef CASE
    return cudaGetLastError();
}

cudaError_t launch_coil_unimodular(const Dims& d, const float2* coils, unsigned int* dev,
                                   cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(dev, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) return e;
    coil_unimodular_kernel<<<pix_grid(d.pixels()), kThreads, 0, st>>>(coils, d.pixels(), dev);
    return cudaGetLastError();
}

cudaError_t launch_apply_w(const Dims& d, const float2* x, const float2* S, float2* y,
                           cudaStream_t st) {
    const int g = pix_grid(d.pixels());
#define CASE(MM)                                                                        \
    case MM: apply_w_kernel<MM><<<g, kThreads, 0, st>>>(x, S, y, d.T, d.circ, d.pixels()); break;
    switch (d.M) {
        CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6)
        default: return cudaErrorInvalidValue;
    }
#undef CASE
    return cudaGetLastError();
}

}  // namespace recon
