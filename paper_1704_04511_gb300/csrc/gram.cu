// Gram matrix of the lifted matrix without forming it (Sec. III-B, Eq. gram-matrix,
// Eq. block-expression-for-R and Eq. P-ij-modified).
//
// G[(l, a), (l', b)] = lag_ab[l - l'],  lag_ab[d] = sum_r q_ab(r) e^{-2 pi i (d1 r1/P + d2 r2/Q)},
// q_ab(r) = sum_{j<k} conj(x_{j+M-1-a}(r)) x_{j+M-1-b}(r),   0 <= a <= b < M.
//
// The paper reads these lags out of the FFT of each product image. Only the (2N1-1) x (2N2-1)
// lags around zero are used, so they are evaluated directly as a pruned separable DFT:
//   gram_rows_kernel: one CTA per image row r1: the pair products of the row (a sliding window
//                     over the frames, all pairs per column in registers) and their pruned
//                     length-Q DFT Y[pair][d2][r1] (FP32 products with compensated sums: each
//                     accumulation carries the rounding errors of its additions in a second
//                     float, through the window sums, the DFT terms and the warp tree, and the
//                     pair becomes one FP64 value);
//   gram_fill_kernel: one warp per lag: the length-P direction sum_r1 Y[pair][d2][r1] w_P^(d1 r1)
//                     in FP64 (fixed order, deterministic), then the lag scattered over the
//                     (l, l') pairs it fills in G (column-major s x s complex128, both triangles).
// Volumes (depth R, N3 depth taps; lag_ab[d] also carries w_R^(d3 r3)): the row kernel runs over
// the R * P rows unchanged, then the length-P and length-R directions are separated:
//   gram_depth_kernel: Z[pair][d2][d1][r3] = sum_r1 Y[pair][d2][r3 P + r1] w_P^(d1 r1)  (FP64);
//   gram_fill3_kernel: one warp per 3-D lag: sum_r3 Z[..][r3] w_R^(d3 r3) (FP64), scattered over
//                      the tap pairs of G with column index ((m N3 + l3) N1 + l1) N2 + l2.
#include "common.cuh"
#include "kernels.h"

namespace recon {

namespace {

// Threads of the row kernel: 512 (its DFT outputs spread over 16 warps) while the window sums of
// all pairs fit in the registers that leaves; 256 for M >= 5 (15 or 21 compensated pairs).
__host__ __device__ constexpr int row_threads(int M) { return M >= 5 ? 256 : 512; }

// kLo = false (only where the low parts do not fit in shared memory: M = 6 with 512-point rows
// and more than 12 frames): each window sum is rounded once to FP32 (hi + lo) before the DFT,
// whose terms and tree stay compensated. tab: the twiddles of every output lag d2 are laid out
// contiguously in c ([L2][Q], built once per CTA), so that the lanes of a warp read consecutive
// entries; otherwise lane c reads w^(d2 c mod Q) from the length-Q table (bank conflicts for
// even d2). The same values either way.
template <int M, bool kLo>
__global__ void __launch_bounds__(row_threads(M))
gram_rows_kernel(const float2* __restrict__ x, int T, int P, int Q, int N2, int circ, int tab,
                 const float2* __restrict__ twQ, double2* __restrict__ Y) {
    constexpr int NP = M * (M + 1) / 2;
    extern __shared__ float2 sm[];
    // circ: T windows with frame indices taken mod T (the fully circulant lifting)
    const int k = circ ? T : T - M + 1, L2 = 2 * N2 - 1;
    float2* xs = sm;                         // [T][Q] row r1 of every frame
    float2* qp = xs + (size_t)T * Q;         // [NP][Q] pair products (compensated sum, high part)
    float2* ql = qp + (size_t)NP * Q;        // [NP][Q] their low parts (kLo)
    float2* tw = ql + (kLo ? (size_t)NP * Q : 0);  // [Q]
    float2* dtab = tw + Q;                   // [L2][Q] (tab)
    const int r1 = blockIdx.x;
    for (int i = threadIdx.x; i < Q; i += blockDim.x) tw[i] = twQ[i];
    for (int e = threadIdx.x; e < T * Q; e += blockDim.x) {
        const int n = e / Q, c = e % Q;
        xs[e] = x[((size_t)n * P + r1) * Q + c];
    }
    __syncthreads();
    if (tab) {  // from the shared copy of the table (no further global loads)
        for (int e = threadIdx.x; e < L2 * Q; e += blockDim.x) {
            const int i2 = e / Q, c = e % Q;
            const int d2m = (i2 - (N2 - 1) + Q) % Q;
            dtab[e] = tw[(d2m * c) % Q];  // d2m, c < Q <= 512: no overflow in 32 bits
        }
    }
    // q_ab(c) = sum_j conj(x_{j+M-1-a}(c)) x_{j+M-1-b}(c): window w[m] = x_{j+M-1-m}(c)
    for (int c = threadIdx.x; c < Q; c += blockDim.x) {
        float2 w[M], acc[NP], lo[NP];
#pragma unroll
        for (int e = 0; e < NP; ++e) acc[e] = lo[e] = make_float2(0.f, 0.f);
#pragma unroll
        for (int m = 1; m < M; ++m) w[m] = xs[(M - 1 - m) * Q + c];
        for (int j = 0; j < k; ++j) {
            w[0] = xs[wrap_frame(j + M - 1, T) * Q + c];
            int e = 0;
#pragma unroll
            for (int a = 0; a < M; ++a)
#pragma unroll
                for (int b = a; b < M; ++b, ++e) {
                    const float2 t = cmulcj(w[a], w[b]);
                    comp_add(acc[e].x, lo[e].x, t.x);
                    comp_add(acc[e].y, lo[e].y, t.y);
                }
#pragma unroll
            for (int m = M - 1; m > 0; --m) w[m] = w[m - 1];
        }
#pragma unroll
        for (int e = 0; e < NP; ++e) {
            if (kLo) {
                qp[e * Q + c] = acc[e];
                ql[e * Q + c] = lo[e];
            } else {
                qp[e * Q + c] = make_float2(__fadd_rn(acc[e].x, lo[e].x), __fadd_rn(acc[e].y, lo[e].y));
            }
        }
    }
    __syncthreads();
    // Y[pair][d2] = sum_c q[pair][c] w_Q^(d2 c); one warp per output, lanes stride c, each term
    // (hi + lo) w added to a compensated (hi, lo) pair, then a TwoSum shuffle tree
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nout = NP * L2;
    for (int o = warp; o < nout; o += row_threads(M) / 32) {
        const int pr = o / L2, i2 = o % L2;
        const int d2m = (i2 - (N2 - 1) + Q) % Q;
        const float2* qrow = qp + (size_t)pr * Q;
        const float2* qlow = ql + (size_t)pr * Q;
        const float2* trow = dtab + (size_t)i2 * Q;
        int idx = (d2m * lane) % Q;
        const int step = (d2m * 32) % Q;
        float2 y = make_float2(0.f, 0.f), yl = make_float2(0.f, 0.f);
        for (int c = lane; c < Q; c += 32) {
            const float2 wt = tab ? trow[c] : tw[idx];
            const float2 t = cmul(qrow[c], wt);
            comp_add(y.x, yl.x, t.x);
            comp_add(y.y, yl.y, t.y);
            if (kLo) {
                const float2 tl = cmul(qlow[c], wt);
                yl.x = __fadd_rn(yl.x, tl.x);
                yl.y = __fadd_rn(yl.y, tl.y);
            }
            idx += step;
            if (idx >= Q) idx -= Q;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const float hx = __shfl_xor_sync(0xffffffffu, y.x, off);
            const float lx = __shfl_xor_sync(0xffffffffu, yl.x, off);
            const float hy = __shfl_xor_sync(0xffffffffu, y.y, off);
            const float ly = __shfl_xor_sync(0xffffffffu, yl.y, off);
            float sx, ex, sy, ey;
            two_sum(y.x, hx, sx, ex);
            two_sum(y.y, hy, sy, ey);
            y = make_float2(sx, sy);
            yl.x = __fadd_rn(__fadd_rn(yl.x, lx), ex);
            yl.y = __fadd_rn(__fadd_rn(yl.y, ly), ey);
        }
        if (lane == 0)
            Y[(size_t)o * P + r1] = make_double2((double)y.x + (double)yl.x, (double)y.y + (double)yl.y);
    }
}

// One warp per lag (pair, d1, d2): the length-P direction in FP64 (lanes over r1 in a fixed
// order, then a fixed shuffle tree), then the lag scattered over the (l, l') pairs of G.
__global__ void gram_fill_kernel(const double2* __restrict__ Y, int P, int N1, int N2, int M,
                                 const double2* __restrict__ twPd, double2* __restrict__ lags,
                                 double2* __restrict__ G) {
    const int L1 = 2 * N1 - 1, L2 = 2 * N2 - 1, npair = M * (M + 1) / 2;
    const int nlag = npair * L1 * L2;
    const int s = N1 * N2 * M;
    const int o = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (o >= nlag) return;
    const int pr = o / (L1 * L2), rem = o % (L1 * L2);
    const int i1 = rem / L2, i2 = rem % L2;
    const int d1 = i1 - (N1 - 1), d2 = i2 - (N2 - 1);
    const int d1m = (d1 + P) % P;
    int a = 0, e = pr;
    while (e >= M - a) { e -= M - a; ++a; }
    const int b = a + e;
    // a frame with itself: lag_aa[-d] = conj(lag_aa[d]) exactly, so the warp of the lag in the
    // non-negative half (d1 > 0, or d1 = 0 and d2 >= 0) writes both and G is exactly Hermitian
    const bool self = a == b;
    if (self && (d1 < 0 || (d1 == 0 && d2 < 0))) return;
    const double2* yrow = Y + ((size_t)pr * L2 + i2) * P;
    double2 v = make_double2(0.0, 0.0);
    for (int r1 = lane; r1 < P; r1 += 32) v = zfma(yrow[r1], twPd[(d1m * r1) % P], v);
    v.x = warp_sum(v.x);
    v.y = warp_sum(v.y);
    if (self && d1 == 0 && d2 == 0) v.y = 0.0;  // sum of |x|^2
    if (lags && lane == 0) {
        lags[o] = v;
        if (self) lags[(size_t)pr * L1 * L2 + (size_t)(L1 - 1 - i1) * L2 + (L2 - 1 - i2)] = zconj(v);
    }
    const int lo1 = max(0, -d1), hi1 = min(N1, N1 - d1);
    const int lo2 = max(0, -d2), hi2 = min(N2, N2 - d2);
    const int n2 = hi2 - lo2, cnt = (hi1 - lo1) * n2;
    for (int t = lane; t < cnt; t += 32) {
        const int lp1 = lo1 + t / n2, lp2 = lo2 + t % n2;
        const int l1 = lp1 + d1, l2 = lp2 + d2;
        const size_t i = ((size_t)a * N1 + l1) * N2 + l2;
        const size_t j = ((size_t)b * N1 + lp1) * N2 + lp2;
        G[i + j * s] = v;
        if (i != j) G[j + i * s] = zconj(v);
    }
}

// One warp per (pair, d2, d1, r3): the length-P direction of depth slice r3 (FP64, lanes over r1
// in a fixed order, then a fixed shuffle tree).
__global__ void gram_depth_kernel(const double2* __restrict__ Y, int P, int R, int N1, int N2,
                                  int npair, const double2* __restrict__ twPd,
                                  double2* __restrict__ Z) {
    const int L1 = 2 * N1 - 1, L2 = 2 * N2 - 1;
    const long long nout = (long long)npair * L2 * L1 * R;
    const long long o = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (o >= nout) return;
    const int r3 = (int)(o % R);
    const long long q = o / R;  // (pair * L2 + i2) * L1 + i1
    const int i1 = (int)(q % L1);
    const long long pi2 = q / L1;  // pair * L2 + i2
    const int d1m = ((i1 - (N1 - 1)) % P + P) % P;
    const double2* yrow = Y + (size_t)pi2 * R * P + (size_t)r3 * P;
    double2 v = make_double2(0.0, 0.0);
    for (int r1 = lane; r1 < P; r1 += 32) v = zfma(yrow[r1], twPd[(d1m * r1) % P], v);
    v.x = warp_sum(v.x);
    v.y = warp_sum(v.y);
    if (lane == 0) Z[o] = v;
}

// One warp per 3-D lag (pair, d3, d1, d2): the length-R direction in FP64, then the lag
// scattered over the tap pairs (l, l') with l - l' = d that it fills in G.
__global__ void gram_fill3_kernel(const double2* __restrict__ Z, int R, int N1, int N2, int N3,
                                  int M, const double2* __restrict__ twRd,
                                  double2* __restrict__ lags, double2* __restrict__ G) {
    const int L1 = 2 * N1 - 1, L2 = 2 * N2 - 1, L3 = 2 * N3 - 1, npair = M * (M + 1) / 2;
    const int nlag = npair * L3 * L1 * L2;
    const int s = N1 * N2 * N3 * M;
    const int o = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (o >= nlag) return;
    const int i2 = o % L2, i1 = (o / L2) % L1, i3 = (o / (L2 * L1)) % L3, pr = o / (L2 * L1 * L3);
    const int d1 = i1 - (N1 - 1), d2 = i2 - (N2 - 1), d3 = i3 - (N3 - 1);
    const int d3m = (d3 % R + R) % R;
    int a = 0, e = pr;
    while (e >= M - a) { e -= M - a; ++a; }
    const int b = a + e;
    // a frame with itself: only the non-negative half of the lags (d3 > 0, or d3 = 0 and
    // (d1, d2) non-negative as in 2-D) is summed; it writes the mirrored lag as its conjugate
    const bool self = a == b;
    if (self && (d3 < 0 || (d3 == 0 && (d1 < 0 || (d1 == 0 && d2 < 0))))) return;
    const double2* zrow = Z + (((size_t)pr * L2 + i2) * L1 + i1) * R;
    double2 v = make_double2(0.0, 0.0);
    for (int r3 = lane; r3 < R; r3 += 32) v = zfma(zrow[r3], twRd[(d3m * r3) % R], v);
    v.x = warp_sum(v.x);
    v.y = warp_sum(v.y);
    if (self && d3 == 0 && d1 == 0 && d2 == 0) v.y = 0.0;
    if (lags && lane == 0) {
        lags[o] = v;
        if (self)
            lags[(((size_t)pr * L3 + (L3 - 1 - i3)) * L1 + (L1 - 1 - i1)) * L2 + (L2 - 1 - i2)] = zconj(v);
    }
    const int lo1 = max(0, -d1), hi1 = min(N1, N1 - d1);
    const int lo2 = max(0, -d2), hi2 = min(N2, N2 - d2);
    const int lo3 = max(0, -d3), hi3 = min(N3, N3 - d3);
    const int n1 = hi1 - lo1, n2 = hi2 - lo2, cnt = (hi3 - lo3) * n1 * n2;
    for (int t = lane; t < cnt; t += 32) {
        const int lp2 = lo2 + t % n2, lp1 = lo1 + (t / n2) % n1, lp3 = lo3 + t / (n2 * n1);
        const size_t i = (((size_t)a * N3 + lp3 + d3) * N1 + lp1 + d1) * N2 + lp2 + d2;
        const size_t j = (((size_t)b * N3 + lp3) * N1 + lp1) * N2 + lp2;
        G[i + j * s] = v;
        if (i != j) G[j + i * s] = zconj(v);
    }
}

constexpr size_t kGramSmemMax = 220 * 1024;

size_t gram_smem_cfg(const Dims& d, bool lo, bool tab) {
    return ((size_t)d.T * d.Q + (lo ? 2 : 1) * (size_t)d.npair() * d.Q + d.Q +
            (tab ? (size_t)d.L2() * d.Q : 0)) * sizeof(float2);
}

// The shared-memory layout of the row kernel: the low parts first (accuracy), then the twiddle
// rows (speed), each where it fits.
void gram_cfg(const Dims& d, bool* lo, bool* tab) {
    *lo = gram_smem_cfg(d, true, false) <= kGramSmemMax;
    *tab = gram_smem_cfg(d, *lo, true) <= kGramSmemMax;
}

}  // namespace

size_t gram_smem(const Dims& d) {
    bool lo, tab;
    gram_cfg(d, &lo, &tab);
    return gram_smem_cfg(d, lo, tab);
}

// One CTA per image row; the scratch holds the row DFTs Y[pair][d2][row] (complex128) and, for
// volumes, the depth-slice sums Z[pair][d2][d1][r3] after them.
int gram_blocks(const Dims& d) { return d.rows(); }

size_t gram_scratch_bytes(const Dims& d, int nblocks) {
    size_t b = (size_t)nblocks * d.npair() * d.L2() * sizeof(double2);
    if (d.R > 1) b += (size_t)d.npair() * d.L2() * d.L1() * d.R * sizeof(double2);
    return b;
}

cudaError_t launch_gram(const Dims& d, const Twiddles& tw, const float2* x, double2* lag_part,
                        int nblocks, double2* lags, double2* G, cudaStream_t st) {
    if (nblocks != d.rows()) return cudaErrorInvalidValue;
    const size_t smem = gram_smem(d);
    if (smem > kGramSmemMax) return cudaErrorInvalidValue;
    bool lo, tab;
    gram_cfg(d, &lo, &tab);
#define CASE(MM)                                                                                 \
    case MM: {                                                                                   \
        auto k = lo ? gram_rows_kernel<MM, true> : gram_rows_kernel<MM, false>;                  \
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,     \
                                             (int)smem);                                         \
        if (e != cudaSuccess) return e;                                                          \
        k<<<d.rows(), row_threads(MM), smem, st>>>(x, d.T, d.rows(), d.Q, d.N2, d.circ, (int)tab,\
                                               tw.twQ, lag_part);                                \
        break;                                                                                   \
    }
    switch (d.M) {
        CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6)
        default: return cudaErrorInvalidValue;
    }
#undef CASE
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (d.R > 1) {
        double2* Z = lag_part + (size_t)nblocks * d.npair() * d.L2();
        const long long nz = (long long)d.npair() * d.L2() * d.L1() * d.R;
        gram_depth_kernel<<<(unsigned)((nz + 7) / 8), 256, 0, st>>>(lag_part, d.P, d.R, d.N1, d.N2,
                                                                    d.npair(), tw.twPd, Z);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        const int nlag3 = (int)d.nlag();
        gram_fill3_kernel<<<(nlag3 + 7) / 8, 256, 0, st>>>(Z, d.R, d.N1, d.N2, d.N3, d.M, tw.twRd,
                                                           lags, G);
        return cudaGetLastError();
    }
    const int nlag = d.npair() * d.L1() * d.L2();
    gram_fill_kernel<<<(nlag + 7) / 8, 256, 0, st>>>(lag_part, d.P, d.N1, d.N2, d.M, tw.twPd, lags, G);
    return cudaGetLastError();
}

}  // namespace recon
