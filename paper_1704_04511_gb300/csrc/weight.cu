// Weight update after the FP64 eigendecomposition G = U diag(lambda) U^H (Sec. III-B; epsilon
// schedule of Sec. III-C):
//   H = U diag((lambda_i + eps)^(p/2 - 1)) U^H                                 (Eq. weight-update)
//   d_ab[delta] = sum_{l - l' = delta} H[(l', b), (l, a)]                        (summed diagonals)
//   S_ab(r) = sum_delta d_ab[delta] e^{-2 pi i (delta1 r1 / P + delta2 r2 / Q)}    (per-pixel S)
// d is formed straight from the eigenvectors, V = U diag(sqrt f):
//   d_ab[delta] = sum_i sum_{l'} V[(l', b), i] conj(V[(l' + delta, a), i]),
// in FP64, in chunks of eigenvectors (one CTA per chunk and pair), then reduced in a fixed
// order. S is a pruned 2-D DFT evaluated separably: FP64 along Q, FP32 along P.
// Volumes (depth R, N3 depth taps): d carries a third lag d3 (layout [pair][d3][d1][d2]) and S a
// third factor e^{-2 pi i d3 r3 / R}: the Q and P stages run over the pair x d3 planes, then an
// FP32 depth stage forms S[pair][r3][r1][r2].
#include "common.cuh"
#include "kernels.h"

namespace recon {

namespace {

constexpr int kThreads = 256;
constexpr int kChunk = 2;  // eigenvectors per CTA
constexpr int kMaxL1 = 1024;  // 2 N1 - 1 <= 2 P - 1 < 1024

__global__ void eps_kernel(const double* __restrict__ lmax, double* eps, int first, double frac,
                           double gamma) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        if (first) eps[0] = frac * lmax[0];
        else eps[0] = eps[0] / gamma;
    }
}

// The eps schedule of several solves in one launch (thread b: solve b).
struct EpsBatch {
    const double* lmax[kMaxHpdBatch];
    double* eps[kMaxHpdBatch];
    int n;
};
__global__ void eps_batch_kernel(EpsBatch bt, int first, double frac, double gamma) {
    const int b = threadIdx.x;
    if (blockIdx.x == 0 && b < bt.n) {
        if (first) bt.eps[b][0] = frac * bt.lmax[b][0];
        else bt.eps[b][0] = bt.eps[b][0] / gamma;
    }
}

__global__ void __launch_bounds__(kThreads)
diag_part_kernel(const double2* __restrict__ U, const double* __restrict__ evals,
                 const double* __restrict__ eps_p, double p, int N1, int N2, int N3, int M,
                 double2* __restrict__ dpart) {
    extern __shared__ __align__(16) unsigned char smraw[];
    double2* V = reinterpret_cast<double2*>(smraw);  // [kChunk][s]
    const int s = N1 * N2 * N3 * M;
    const int L1 = 2 * N1 - 1, L2 = 2 * N2 - 1, L3 = 2 * N3 - 1;
    const int i0 = blockIdx.x * kChunk;
    const int nc = min(kChunk, s - i0);
    const int pr = blockIdx.y;
    int a = 0, e = pr;
    while (e >= M - a) { e -= M - a; ++a; }
    const int b = a + e;
    const double eps = eps_p[0];
    for (int t = threadIdx.x; t < nc * s; t += blockDim.x) {
        const int c = t / s, row = t % s;
        const double lam = evals[i0 + c] + eps;
        // sqrt((lambda + eps)^(p/2 - 1)) = (lambda + eps)^(p/4 - 1/2)
        const double sf = (p == 0.0) ? 1.0 / sqrt(lam) : pow(lam, 0.25 * p - 0.5);
        const double2 u = U[(size_t)(i0 + c) * s + row];
        V[t] = make_double2(u.x * sf, u.y * sf);
    }
    __syncthreads();
    const int nlag = L3 * L1 * L2;
    double2* out = dpart + ((size_t)blockIdx.x * gridDim.y + pr) * nlag;
    for (int o = threadIdx.x; o < nlag; o += blockDim.x) {
        const int d2 = o % L2 - (N2 - 1), d1 = (o / L2) % L1 - (N1 - 1), d3 = o / (L2 * L1) - (N3 - 1);
        double2 acc = make_double2(0.0, 0.0);
        for (int c = 0; c < nc; ++c) {
            const double2* v = V + (size_t)c * s;
            for (int lp3 = max(0, -d3); lp3 < min(N3, N3 - d3); ++lp3)
                for (int lp1 = max(0, -d1); lp1 < min(N1, N1 - d1); ++lp1)
                    for (int lp2 = max(0, -d2); lp2 < min(N2, N2 - d2); ++lp2) {
                        const double2 vb = v[(((size_t)b * N3 + lp3) * N1 + lp1) * N2 + lp2];
                        const double2 va =
                            v[(((size_t)a * N3 + lp3 + d3) * N1 + lp1 + d1) * N2 + lp2 + d2];
                        acc = zfmacj2(vb, va, acc);
                    }
        }
        out[o] = acc;
    }
}

// one warp per output: lanes add the chunk partials, then a fixed shuffle tree
__global__ void diag_reduce_kernel(const double2* __restrict__ dpart, int nchunks, int nout,
                                   double2* __restrict__ dsum) {
    const int o = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (o >= nout) return;
    double2 v = make_double2(0.0, 0.0);
    for (int c = lane; c < nchunks; c += 32) v = zadd(v, dpart[(size_t)c * nout + o]);
    v.x = warp_sum(v.x);
    v.y = warp_sum(v.y);
    if (lane == 0) dsum[o] = v;
}

// Z[pair][i1][r2] = sum_{d2} d[pair][i1][d2] w_Q^{d2 r2}  (FP64, rounded to FP32 on store);
// the twiddle index (d2 r2) mod Q advances by r2 per lag (int arithmetic, no division).
__global__ void __launch_bounds__(kThreads)
s_stage1_kernel(const double2* __restrict__ dsum, int N1, int N2, int Q,
                const double2* __restrict__ twQd, float2* __restrict__ Z) {
    const int L2 = 2 * N2 - 1;
    const int row = blockIdx.x;  // pair * L1 + i1
    const double2* drow = dsum + (size_t)row * L2;
    const int d2m0 = (Q - (N2 - 1) % Q) % Q;  // (-(N2 - 1)) mod Q
    for (int r2 = blockIdx.y * blockDim.x + threadIdx.x; r2 < Q; r2 += blockDim.x * gridDim.y) {
        double2 acc = make_double2(0.0, 0.0);
        int ti = (d2m0 * r2) % Q;
        for (int i2 = 0; i2 < L2; ++i2) {
            acc = zfma(drow[i2], twQd[ti], acc);
            ti += r2;
            if (ti >= Q) ti -= Q;
        }
        Z[(size_t)row * Q + r2] = make_float2((float)acc.x, (float)acc.y);
    }
}

// S[pair][r1][r2] = sum_{d1} Z[pair][d1][r2] w_P^{d1 r1}  (FP32), for L1 <= kL1Reg: thread
// (pair, column r2, block of kRB rows r1) holds the L1 values Z[pair][.][r2] in registers and
// forms its kRB outputs, each summed in d1 order with the twiddles of s_stage2_kernel (the same
// bits); Z is read once instead of once per image row.
constexpr int kL1Reg = 20;
constexpr int kRB = 8;
__global__ void __launch_bounds__(kThreads)
s_stage2_reg_kernel(const float2* __restrict__ Z, int N1, int P, int Q, int npair,
                    const float2* __restrict__ twP, float2* __restrict__ S) {
    __shared__ float2 tws[kMaxL1];
    for (int i = threadIdx.x; i < P; i += blockDim.x) tws[i] = twP[i];
    __syncthreads();
    const int L1 = 2 * N1 - 1;
    const int nrb = (P + kRB - 1) / kRB;
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (long long)npair * nrb * Q) return;
    const int r2 = (int)(g % Q), rb = (int)((g / Q) % nrb), pr = (int)(g / ((long long)Q * nrb));
    const float2* zp = Z + (size_t)pr * L1 * Q + r2;
    float2 z[kL1Reg];
#pragma unroll
    for (int i1 = 0; i1 < kL1Reg; ++i1) z[i1] = i1 < L1 ? zp[(size_t)i1 * Q] : make_float2(0.f, 0.f);
    const int d1m0 = (P - (N1 - 1) % P) % P;  // (-(N1 - 1)) mod P
    for (int u = 0; u < kRB; ++u) {
        const int r1 = rb * kRB + u;
        if (r1 >= P) break;
        int ti = (d1m0 * r1) % P;
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int i1 = 0; i1 < kL1Reg; ++i1) {
            if (i1 < L1) {
                acc = cfma(z[i1], tws[ti], acc);
                ti += r1;
                if (ti >= P) ti -= P;
            }
        }
        S[((size_t)pr * P + r1) * Q + r2] = acc;
    }
}

// The same for any L1: one CTA per image row r1, its L1 twiddles in shared memory, every pair
// and column.
__global__ void __launch_bounds__(kThreads)
s_stage2_kernel(const float2* __restrict__ Z, int N1, int P, int Q, int npair,
                const float2* __restrict__ twP, float2* __restrict__ S) {
    __shared__ float2 w1[kMaxL1];
    const int L1 = 2 * N1 - 1;
    const int r1 = blockIdx.x;
    if (threadIdx.x == 0) {
        int ti = (((P - (N1 - 1) % P) % P) * r1) % P;
        for (int i1 = 0; i1 < L1; ++i1) {
            w1[i1] = twP[ti];
            ti += r1;
            if (ti >= P) ti -= P;
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < npair * Q; e += blockDim.x) {
        const int pr = e / Q, r2 = e % Q;
        const float2* zp = Z + (size_t)pr * L1 * Q + r2;
        float2 acc = make_float2(0.f, 0.f);
        int i1 = 0;
        for (; i1 + 8 <= L1; i1 += 8) {  // eight loads in flight, then the products in order
            float2 z[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) z[u] = zp[(size_t)(i1 + u) * Q];
#pragma unroll
            for (int u = 0; u < 8; ++u) acc = cfma(z[u], w1[i1 + u], acc);
        }
        for (; i1 < L1; ++i1) acc = cfma(zp[(size_t)i1 * Q], w1[i1], acc);
        S[((size_t)pr * P + r1) * Q + r2] = acc;
    }
}

// S[pair][r3][px] = sum_{d3} Z2[pair][d3][px] w_R^{d3 r3} (FP32): one thread per voxel of depth
// slice r3 (blockIdx.y = pair * R + r3), the L3 twiddles in shared memory.
__global__ void __launch_bounds__(kThreads)
s_stage3_kernel(const float2* __restrict__ Z2, int N3, int R, size_t npx,
                const float2* __restrict__ twR, float2* __restrict__ S) {
    __shared__ float2 w3[kMaxL1];
    const int L3 = 2 * N3 - 1;
    const int pr = blockIdx.y / R, r3 = blockIdx.y % R;
    if (threadIdx.x == 0) {
        int ti = (((R - (N3 - 1) % R) % R) * r3) % R;
        for (int i3 = 0; i3 < L3; ++i3) {
            w3[i3] = twR[ti];
            ti += r3;
            if (ti >= R) ti -= R;
        }
    }
    __syncthreads();
    const float2* zp = Z2 + (size_t)pr * L3 * npx;
    float2* out = S + ((size_t)pr * R + r3) * npx;
    for (size_t px = (size_t)blockIdx.x * blockDim.x + threadIdx.x; px < npx;
         px += (size_t)gridDim.x * blockDim.x) {
        float2 acc = make_float2(0.f, 0.f);
        int i3 = 0;
        for (; i3 + 4 <= L3; i3 += 4) {  // four loads in flight, then the products in order
            float2 z[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) z[u] = zp[(size_t)(i3 + u) * npx + px];
#pragma unroll
            for (int u = 0; u < 4; ++u) acc = cfma(z[u], w3[i3 + u], acc);
        }
        for (; i3 < L3; ++i3) acc = cfma(zp[(size_t)i3 * npx + px], w3[i3], acc);
        out[px] = acc;
    }
}

int nchunks(const Dims& d) { return (d.s() + kChunk - 1) / kChunk; }

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace

cudaError_t launch_eps(const double* lmax, double* eps, int first, double frac, double gamma,
                       cudaStream_t st) {
    eps_kernel<<<1, 32, 0, st>>>(lmax, eps, first, frac, gamma);
    return cudaGetLastError();
}

cudaError_t launch_eps_batch(const double* const* lmax, double* const* eps, int n, int first,
                             double frac, double gamma, cudaStream_t st) {
    if (n < 1 || n > kMaxHpdBatch) return cudaErrorInvalidValue;
    EpsBatch bt = {};
    bt.n = n;
    for (int b = 0; b < n; ++b) {
        bt.lmax[b] = lmax[b];
        bt.eps[b] = eps[b];
    }
    eps_batch_kernel<<<1, 32, 0, st>>>(bt, first, frac, gamma);
    return cudaGetLastError();
}

size_t diag_scratch_bytes(const Dims& d) {
    return (size_t)nchunks(d) * d.nlag() * sizeof(double2);
}

cudaError_t launch_diag_sums(const Dims& d, const double2* U, const double* evals,
                             const double* eps, double p, double2* dpart, double2* dsum,
                             cudaStream_t st) {
    const size_t smem = (size_t)kChunk * d.s() * sizeof(double2);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(diag_part_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    dim3 grid(nchunks(d), d.npair());
    diag_part_kernel<<<grid, kThreads, smem, st>>>(U, evals, eps, p, d.N1, d.N2, d.N3, d.M, dpart);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int nout = (int)d.nlag();
    diag_reduce_kernel<<<(nout + 7) / 8, 256, 0, st>>>(dpart, nchunks(d), nout, dsum);
    return cudaGetLastError();
}

size_t s_scratch_bytes(const Dims& d) {
    size_t b = align256((size_t)d.npair() * d.L3() * d.L1() * d.Q * sizeof(float2));
    if (d.R > 1) b += (size_t)d.npair() * d.L3() * d.P * d.Q * sizeof(float2);
    return b;
}

cudaError_t launch_weight_S(const Dims& d, const Twiddles& tw, const double2* dsum, double2* Z_,
                            float2* S, cudaStream_t st) {
    float2* Z = reinterpret_cast<float2*>(Z_);
    const int planes = d.npair() * d.L3();  // (pair, d3) planes of the summed diagonals
    // FP64 sums: two CTAs of 128 columns per (plane, d1) row where the columns allow, so that
    // the FP64 work spreads over more SMs
    const int s1_threads = d.Q >= 256 ? 128 : kThreads;
    const dim3 s1_grid(planes * d.L1(), (d.Q + s1_threads - 1) / s1_threads);
    s_stage1_kernel<<<s1_grid, s1_threads, 0, st>>>(dsum, d.N1, d.N2, d.Q, tw.twQd, Z);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (d.L1() > kMaxL1 || d.L3() > kMaxL1 || d.P > kMaxL1) return cudaErrorInvalidValue;
    auto stage2 = [&](int np, float2* out) {
        if (d.L1() <= kL1Reg) {
            const long long n = (long long)np * ((d.P + kRB - 1) / kRB) * d.Q;
            s_stage2_reg_kernel<<<(unsigned)((n + kThreads - 1) / kThreads), kThreads, 0, st>>>(
                Z, d.N1, d.P, d.Q, np, tw.twP, out);
        } else {
            s_stage2_kernel<<<d.P, kThreads, 0, st>>>(Z, d.N1, d.P, d.Q, np, tw.twP, out);
        }
        return cudaGetLastError();
    };
    if (d.R == 1) return stage2(d.npair(), S);
    float2* Z2 = reinterpret_cast<float2*>(reinterpret_cast<unsigned char*>(Z) +
                                           align256((size_t)planes * d.L1() * d.Q * sizeof(float2)));
    e = stage2(planes, Z2);
    if (e != cudaSuccess) return e;
    const size_t npx = (size_t)d.P * d.Q;
    const int gx = (int)((npx + kThreads - 1) / kThreads);
    s_stage3_kernel<<<dim3(gx < 64 ? gx : 64, d.npair() * d.R), kThreads, 0, st>>>(
        Z2, d.N3, d.R, npx, tw.twR, S);
    return cudaGetLastError();
}

}  // namespace recon
