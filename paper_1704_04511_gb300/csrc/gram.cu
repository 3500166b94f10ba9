// Gram matrix of the lifted matrix without forming it (Sec. III-B, Eq. gram-matrix,
// Eq. block-expression-for-R and Eq. P-ij-modified).
//
// G[(l, a), (l', b)] = lag_ab[l - l'],  lag_ab[d] = sum_r q_ab(r) e^{-2 pi i (d1 r1/P + d2 r2/Q)},
// q_ab(r) = sum_{j<k} conj(x_{j+M-1-a}(r)) x_{j+M-1-b}(r),   0 <= a <= b < M.
//
// The paper reads these lags out of the FFT of each product image. Only the (2N1-1) x (2N2-1)
// lags around zero are used, so this kernel evaluates exactly those DFT outputs directly,
// separably: per image row, a pruned length-Q DFT of the pair products (FP32, warp-tree sums),
// then the row's contribution to the length-P direction in FP64. Each CTA accumulates its rows
// and writes one partial; a second kernel adds the partials in a fixed order (deterministic)
// and fills G (column-major s x s complex128, both triangles).
#include "common.cuh"
#include "kernels.h"

namespace recon {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

__global__ void __launch_bounds__(kThreads)
gram_rows_kernel(const float2* __restrict__ x, int T, int P, int Q, int N1, int N2, int M,
                 const float2* __restrict__ twQ, const double2* __restrict__ twPd,
                 double2* __restrict__ lag_part) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int k = T - M + 1, npair = M * (M + 1) / 2;
    const int L1 = 2 * N1 - 1, L2 = 2 * N2 - 1;
    const int nlag = npair * L1 * L2;
    double2* acc = reinterpret_cast<double2*>(smraw);               // [npair][L1][L2]
    float2* xs = reinterpret_cast<float2*>(acc + nlag);             // [T][Q]
    float2* qp = xs + (size_t)T * Q;                                // [npair][Q]
    float2* tw = qp + (size_t)npair * Q;                            // [Q]
    int* pa = reinterpret_cast<int*>(tw + Q);                       // [npair] a
    int* pb = pa + npair;                                           // [npair] b
    for (int i = threadIdx.x; i < nlag; i += blockDim.x) acc[i] = make_double2(0.0, 0.0);
    for (int i = threadIdx.x; i < Q; i += blockDim.x) tw[i] = twQ[i];
    if (threadIdx.x == 0) {
        int e = 0;
        for (int a = 0; a < M; ++a)
            for (int b = a; b < M; ++b) { pa[e] = a; pb[e] = b; ++e; }
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nout = npair * L2;
    for (int r1 = blockIdx.x; r1 < P; r1 += gridDim.x) {
        __syncthreads();
        for (int e = threadIdx.x; e < T * Q; e += blockDim.x) {
            const int n = e / Q, c = e % Q;
            xs[e] = x[((size_t)n * P + r1) * Q + c];
        }
        __syncthreads();
        for (int e = threadIdx.x; e < npair * Q; e += blockDim.x) {
            const int pr = e / Q, c = e % Q;
            const int a = pa[pr], b = pb[pr];
            float2 s = make_float2(0.f, 0.f);
            for (int j = 0; j < k; ++j)
                s = cfmacj(xs[(j + M - 1 - a) * Q + c], xs[(j + M - 1 - b) * Q + c], s);
            qp[e] = s;
        }
        __syncthreads();
        // Y[pair][d2] = sum_r2 q[pair][r2] w_Q^{d2 r2}; one warp per output, lanes stride r2.
        for (int o = warp; o < nout; o += kWarps) {
            const int pr = o / L2, i2 = o % L2;
            const int d2 = i2 - (N2 - 1);
            const int d2m = ((d2 % Q) + Q) % Q;
            const float2* qrow = qp + (size_t)pr * Q;
            int idx = (int)(((long long)d2m * lane) % Q);
            const int step = (int)(((long long)d2m * 32) % Q);
            float2 y = make_float2(0.f, 0.f);
            for (int c = lane; c < Q; c += 32) {
                y = cfma(qrow[c], tw[idx], y);
                idx += step;
                if (idx >= Q) idx -= Q;
            }
            y.x = warp_sum(y.x);
            y.y = warp_sum(y.y);
            // this row's contribution to lag[pair][d1][d2] for every d1 (FP64), lanes over d1
            const double2 yd = make_double2((double)y.x, (double)y.y);
            for (int i1 = lane; i1 < L1; i1 += 32) {
                const int d1 = i1 - (N1 - 1);
                const int ti = (int)((((long long)d1 % P + P) % P * r1) % P);
                double2* dst = acc + ((size_t)pr * L1 + i1) * L2 + i2;
                *dst = zfma(yd, twPd[ti], *dst);
            }
        }
    }
    __syncthreads();
    double2* out = lag_part + (size_t)blockIdx.x * nlag;
    for (int i = threadIdx.x; i < nlag; i += blockDim.x) out[i] = acc[i];
}

// One warp per lag: lanes add the per-block partials (fixed order, then a fixed shuffle tree)
// and scatter the lag over the (l, l') pairs it fills in G.
__global__ void gram_fill_kernel(const double2* __restrict__ lag_part, int nblocks, int N1,
                                 int N2, int M, double2* __restrict__ lags,
                                 double2* __restrict__ G) {
    const int L1 = 2 * N1 - 1, L2 = 2 * N2 - 1, npair = M * (M + 1) / 2;
    const int nlag = npair * L1 * L2;
    const int s = N1 * N2 * M;
    const int o = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (o >= nlag) return;
    double2 v = make_double2(0.0, 0.0);
    for (int bI = lane; bI < nblocks; bI += 32) v = zadd(v, lag_part[(size_t)bI * nlag + o]);
    v.x = warp_sum(v.x);
    v.y = warp_sum(v.y);
    if (lags && lane == 0) lags[o] = v;
    const int pr = o / (L1 * L2), rem = o % (L1 * L2);
    const int d1 = rem / L2 - (N1 - 1), d2 = rem % L2 - (N2 - 1);
    int a = 0, e = pr;
    while (e >= M - a) { e -= M - a; ++a; }
    const int b = a + e;
    const int lo1 = max(0, -d1), hi1 = min(N1, N1 - d1);
    const int lo2 = max(0, -d2), hi2 = min(N2, N2 - d2);
    const int n2 = hi2 - lo2, cnt = (hi1 - lo1) * n2;
    for (int t = lane; t < cnt; t += 32) {
        const int lp1 = lo1 + t / n2, lp2 = lo2 + t % n2;
        const int l1 = lp1 + d1, l2 = lp2 + d2;
        const size_t i = ((size_t)a * N1 + l1) * N2 + l2;
        const size_t j = ((size_t)b * N1 + lp1) * N2 + lp2;
        G[i + j * s] = v;
        if (a != b) G[j + i * s] = zconj(v);
    }
}

size_t gram_smem(const Dims& d) {
    const size_t nlag = (size_t)d.npair() * d.L1() * d.L2();
    return nlag * sizeof(double2) + ((size_t)d.T * d.Q + (size_t)d.npair() * d.Q + d.Q) * sizeof(float2) +
           2 * d.npair() * sizeof(int);
}

}  // namespace

int gram_blocks(const Dims& d) { return d.P < 128 ? d.P : 128; }

size_t gram_scratch_bytes(const Dims& d, int nblocks) {
    return (size_t)nblocks * d.npair() * d.L1() * d.L2() * sizeof(double2);
}

cudaError_t launch_gram(const Dims& d, const Twiddles& tw, const float2* x, double2* lag_part,
                        int nblocks, double2* lags, double2* G, cudaStream_t st) {
    const size_t smem = gram_smem(d);
    if (smem > 220 * 1024) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(gram_rows_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    gram_rows_kernel<<<nblocks, kThreads, smem, st>>>(x, d.T, d.P, d.Q, d.N1, d.N2, d.M, tw.twQ,
                                                      tw.twPd, lag_part);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int nlag = d.npair() * d.L1() * d.L2();
    gram_fill_kernel<<<(nlag + 7) / 8, 256, 0, st>>>(lag_part, nblocks, d.N1, d.N2, d.M, lags, G);
    return cudaGetLastError();
}

}  // namespace recon
