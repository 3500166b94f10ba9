// CG operator on square frames with thread-block clusters (Sec. III-A, Eq. grad-ls):
//
//   frame_aha_kernel:  p = r (+ beta p);  t = F^H (mask * F p) per frame, the whole 2-D transform
//                      of one frame done by one 8-CTA cluster: each CTA holds N/8 rows in shared
//                      memory, transforms them, and the clusters exchange column blocks through
//                      distributed shared memory (DSMEM) for the column transforms and back.
//                      One pass over r, p and t instead of a row pass plus a strided column pass.
//   w_combine_kernel:  q = t + lam W p per pixel over all frames (W: the banded frame operator of
//                      the per-pixel S(r), see cg.cu), written over t; per-CTA partials of
//                      Re <p, q> for the update pass. All frames of a pixel block are staged in
//                      shared memory first so that every load is in flight at once.
//
// Used for P = Q in {32, 64, 128, 192, 256} (two (N/8) x (N+1) complex buffers per CTA fit in
// shared memory) when the context option asks for it; other shapes, and the default, use the
// row / column passes of fft.cu and cg.cu. Measured at 256 x 256 x 16: 70 us per operator pass
// against ~22 us for the row + column passes, because only 15 such clusters are co-resident
// (16 frames take two waves) and the Stockham stages conflict on shared-memory banks.
#include <cooperative_groups.h>

#include "common.cuh"
#include "kernels.h"

namespace cg = cooperative_groups;

namespace recon {

namespace {

constexpr int kThreads = 1024;  // one Stockham butterfly per thread per stage at N = 256
constexpr int kCluster = 8;
constexpr int kPixBlock = 128;  // pixels per CTA in w_combine
constexpr int kMaxM = 6;

template <int N>
constexpr int frame_smem_floats2() { return 2 * (N / kCluster) * (N + 1) + 2 * N; }

template <int N>
__global__ void __launch_bounds__(kThreads)
frame_aha_kernel(const float2* __restrict__ r, float2* __restrict__ p, float2* __restrict__ t,
                 const uint8_t* __restrict__ mask, const double* __restrict__ rr_parts, int n_rr,
                 const double* __restrict__ rr_prev, double* __restrict__ rr_out, int first,
                 float scale, const float2* __restrict__ tw_g) {
    constexpr int R = N / kCluster;   // rows (and columns) this CTA owns
    constexpr int S = N + 1;          // padded stride of a row / a column in shared memory
    extern __shared__ float2 sm[];
    float2* buf0 = sm;
    float2* buf1 = sm + R * S;
    float2* tw = sm + 2 * R * S;
    __shared__ float beta_s;
    __shared__ double s_rr;
    cg::cluster_group cluster = cg::this_cluster();
    const int j = (int)cluster.block_rank();
    const size_t fbase = (size_t)blockIdx.y * N * N;
    for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = tw_g[i];
    pdl_wait();
    float beta = 0.f;
    if (!first) {
        const double rr_new = sum_partials(rr_parts, n_rr, &s_rr);
        if (threadIdx.x == 0) {
            beta_s = (float)(rr_new * rcp_nr(rr_prev[0]));
            if (blockIdx.x == 0 && blockIdx.y == 0) rr_out[0] = rr_new;
        }
        __syncthreads();
        beta = beta_s;
    }
    // rows j*R .. j*R+R-1 of this frame: p update, kept in buf0 (row-major, stride S)
    for (int e = threadIdx.x; e < R * N; e += blockDim.x) {
        const int rl = e / N, c = e % N;
        const size_t g = fbase + (size_t)(j * R + rl) * N + c;
        float2 v = r[g];
        if (!first) {
            const float2 pv = p[g];
            v.x = fmaf(beta, pv.x, v.x);
            v.y = fmaf(beta, pv.y, v.y);
        }
        p[g] = v;
        buf0[rl * S + c] = v;
    }
    __syncthreads();
    // forward transforms of the rows
    float2* rowres = fft_smem<N, false, false>(buf0, buf1, R, S, 1, tw);
    float2* other = rowres == buf0 ? buf1 : buf0;
    cluster.sync();
    // exchange: gather column block j of every CTA's rows, column-major (stride S)
    for (int e = threadIdx.x; e < kCluster * R * R; e += blockDim.x) {
        const int cl = e % R, rl = (e / R) % R, m = e / (R * R);
        const float2* src = cluster.map_shared_rank(rowres, m);
        other[cl * S + m * R + rl] = src[rl * S + j * R + cl];
    }
    cluster.sync();
    // column transforms, mask (and the 1/(PQ) of the two unitary transforms), inverse
    float2* colres = fft_smem<N, false, false>(other, rowres, R, S, 1, tw);
    for (int e = threadIdx.x; e < R * N; e += blockDim.x) {
        const int cl = e % R, i = e / R;
        const uint8_t mk = mask[fbase + (size_t)i * N + j * R + cl];
        float2& v = colres[cl * S + i];
        v = mk ? cscale(v, scale) : make_float2(0.f, 0.f);
    }
    __syncthreads();
    float2* colinv = fft_smem<N, true, false>(colres, colres == buf0 ? buf1 : buf0, R, S, 1, tw);
    float2* other2 = colinv == buf0 ? buf1 : buf0;
    cluster.sync();
    // exchange back: row block j of every CTA's columns, row-major (stride S)
    for (int e = threadIdx.x; e < kCluster * R * R; e += blockDim.x) {
        const int rl = e % R, cl = (e / R) % R, m = e / (R * R);
        const float2* src = cluster.map_shared_rank(colinv, m);
        other2[rl * S + m * R + cl] = src[cl * S + j * R + rl];
    }
    cluster.sync();
    float2* rowinv = fft_smem<N, true, false>(other2, colinv, R, S, 1, tw);
    pdl_trigger();
    for (int e = threadIdx.x; e < R * N; e += blockDim.x) {
        const int rl = e / N, c = e % N;
        t[fbase + (size_t)(j * R + rl) * N + c] = rowinv[rl * S + c];
    }
}

template <int M>
__global__ void __launch_bounds__(kPixBlock)
w_combine_kernel(float2* t, const float2* __restrict__ p, const float2* __restrict__ S, float lam,
                 int T, size_t npix, double* __restrict__ pq_parts) {
    extern __shared__ float2 sm[];
    float2* sp = sm;                       // [T][kPixBlock]
    float2* sa = sm + (size_t)T * kPixBlock;  // [T][kPixBlock]
    __shared__ double red[kPixBlock / 32];
    const size_t px = (size_t)blockIdx.x * kPixBlock + threadIdx.x;
    const bool ok = px < npix;
    float2 s[M][M];
    pdl_wait();
    if (ok) {
#pragma unroll
        for (int a = 0; a < M; ++a)
#pragma unroll
            for (int b = a; b < M; ++b) {
                const float2 v = S[(size_t)(a * (2 * M - a + 1) / 2 + (b - a)) * npix + px];
                s[a][b] = v;
                s[b][a] = cconj(v);
            }
        for (int n = 0; n < T; ++n) {
            sp[n * kPixBlock + threadIdx.x] = p[(size_t)n * npix + px];
            sa[n * kPixBlock + threadIdx.x] = t[(size_t)n * npix + px];
        }
    }
    const int k = T - M + 1;
    float acc = 0.f, comp = 0.f;
    if (ok) {
        for (int n = 0; n < T; ++n) {
            float2 w = make_float2(0.f, 0.f);
#pragma unroll
            for (int a = 0; a < M; ++a) {
                const int jw = n - M + 1 + a;
                if (jw < 0 || jw >= k) continue;
#pragma unroll
                for (int b = 0; b < M; ++b) w = cfma(s[a][b], sp[(n + a - b) * kPixBlock + threadIdx.x], w);
            }
            float2 q = sa[n * kPixBlock + threadIdx.x];
            q.x = fmaf(lam, w.x, q.x);
            q.y = fmaf(lam, w.y, q.y);
            t[(size_t)n * npix + px] = q;
            const float2 pv = sp[n * kPixBlock + threadIdx.x];
            const float term = fmaf(pv.x, q.x, pv.y * q.y) - comp;
            const float sum = acc + term;
            comp = (sum - acc) - term;
            acc = sum;
        }
    }
    pdl_trigger();
    const double tot = block_sum_f_t0(acc, red);
    if (threadIdx.x == 0) pq_parts[blockIdx.x] = tot;
}

template <int N>
cudaError_t launch_frame_N(const Dims& d, const Twiddles& tw, const float2* r, float2* p,
                           float2* t, const uint8_t* mask, const Partials& rr,
                           const double* rr_prev, double* rr_out, int first, cudaStream_t st) {
    auto kern = frame_aha_kernel<N>;
    const size_t smem = (size_t)frame_smem_floats2<N>() * sizeof(float2);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kCluster, d.T);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kCluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    const float scale = 1.0f / ((float)N * (float)N);
    const float2* twp = tw.twQ;
    return cudaLaunchKernelEx(&cfg, kern, r, p, t, mask, (const double*)rr.parts, rr.n, rr_prev,
                              rr_out, first, scale, twp);
}

}  // namespace

bool frame_op_supported(const Dims& d) {
    if (d.P != d.Q || d.R != 1 || d.nc != 1 || d.circ) return false;
    switch (d.P) {
        case 32: case 64: case 128: case 192: case 256: return true;
        default: return false;
    }
}

cudaError_t launch_frame_aha(const Dims& d, const Twiddles& tw, const float2* r, float2* p,
                             float2* t, const uint8_t* mask, const Partials& rr,
                             const double* rr_prev, double* rr_out, int first, cudaStream_t st) {
    switch (d.P) {
        case 32: return launch_frame_N<32>(d, tw, r, p, t, mask, rr, rr_prev, rr_out, first, st);
        case 64: return launch_frame_N<64>(d, tw, r, p, t, mask, rr, rr_prev, rr_out, first, st);
        case 128: return launch_frame_N<128>(d, tw, r, p, t, mask, rr, rr_prev, rr_out, first, st);
        case 192: return launch_frame_N<192>(d, tw, r, p, t, mask, rr, rr_prev, rr_out, first, st);
        case 256: return launch_frame_N<256>(d, tw, r, p, t, mask, rr, rr_prev, rr_out, first, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_w_combine(const Dims& d, float2* t, const float2* p, const float2* S, float lam,
                             Partials* pq, cudaStream_t st) {
    const size_t npix = d.pixels();
    const int grid = (int)((npix + kPixBlock - 1) / kPixBlock);
    if (grid > max_parts()) return cudaErrorInvalidValue;
    pq->n = grid;
    const size_t smem = (size_t)2 * d.T * kPixBlock * sizeof(float2);
#define CASE(MM)                                                                                  \
    case MM: {                                                                                    \
        auto kern = w_combine_kernel<MM>;                                                         \
        if (smem > 48 * 1024) {                                                                   \
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                                 (int)smem);                                      \
            if (e != cudaSuccess) return e;                                                       \
        }                                                                                         \
        return launch_pdl(kern, dim3(grid), dim3(kPixBlock), smem, st, t, p, S, lam, d.T, npix,   \
                          pq->parts);                                                             \
    }
    switch (d.M) {
        CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6)
        default: return cudaErrorInvalidValue;
    }
#undef CASE
}

}  // namespace recon
