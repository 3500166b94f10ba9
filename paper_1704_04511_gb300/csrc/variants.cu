// Kernels of the comparison methods of Sec. IV (the GIRAF form reuses every kernel of the
// proposed path with the time-circular flag of Dims):
//
// HLR-Voxel (Sec. II-D, Eq. MORASA-objective): one k x M Toeplitz matrix of the temporal signal
// per pixel, T_r[j][m] = x_{j+M-1-m}(r). voxel_weight_kernel forms, per pixel and in FP64, the
// Gram G_r = T_r^H T_r, its eigendecomposition by cyclic complex Jacobi rotations, the weight
// H_r = U diag((lambda + eps)^(p/2-1)) U^H and the banded-W matrix S(r) = H_r^T (so that
// Re <x, W x> = sum_r Tr(H_r G_r)); the CG then runs on the proposed path's kernels. The penalty
// sum_r ||T_r||_p is one objective with one smoothing eps, scheduled as in Sec. III-C from the
// largest lambda_max(G_r(x0)) over the pixels (a first launch reduces it, the weight launch
// reads the one eps).
//
// IRLS-direct (Sec. IV-A: Eq. x-update and Eq. weight-update without the FFT approximations):
// the exact multi-fold Toeplitz matrix, valid in all three dimensions, of the centred k-space
// (DC at (P/2, Q/2): the valid lifting is not shift invariant and the grid of Sec. II-B is
// centred on k = 0) is formed explicitly (direct_lift_kernel), its Gram is a library Hermitian
// rank-k product, and the penalty gradient F^H C^H T^*(T(C F p) H) is a library GEMM between the
// lifting and its adjoint (direct_unlift_kernel, a gather: each element of T(C F p) H goes back
// to the k-space sample it was copied from). The centring C is folded into the index maps
// (P and Q are even, so it is the half-grid shift both ways).
#include "common.cuh"
#include "kernels.h"

namespace recon {

namespace {

constexpr int kThreads = 256;
constexpr int kVoxThreads = 128;
constexpr int kJacobiSweeps = 16;

// Per-pixel HLR-Voxel weight. eps_mode: 0 = eps_r = eps_in[px] (one eps per pixel); 1 = no
// weight: the largest lambda_max(G_r) over the pixels goes to *lmax_max (FP64 bits, atomic max;
// zero it first); 2 = eps_r = eps_in[0] (one eps for every pixel). G_out (may be null):
// [npix][M][M] complex128 row-major; lmax_out (may be null): [npix].
template <int M>
__global__ void __launch_bounds__(kVoxThreads)
voxel_weight_kernel(const float2* __restrict__ x, int T, size_t npix, double p,
                    const double* __restrict__ eps_in, unsigned long long* __restrict__ lmax_max,
                    int eps_mode, float2* __restrict__ S, double2* __restrict__ G_out,
                    double* __restrict__ lmax_out) {
    const int k = T - M + 1;
    for (size_t px = (size_t)blockIdx.x * blockDim.x + threadIdx.x; px < npix;
         px += (size_t)gridDim.x * blockDim.x) {
        // G_r[a][b] = sum_j conj(x_{j+M-1-a}) x_{j+M-1-b}, window w[m] = x_{j+M-1-m}
        double2 A[M][M], w[M];
#pragma unroll
        for (int a = 0; a < M; ++a)
#pragma unroll
            for (int b = 0; b < M; ++b) A[a][b] = make_double2(0.0, 0.0);
#pragma unroll
        for (int m = 1; m < M; ++m) {
            const float2 v = x[(size_t)(M - 1 - m) * npix + px];
            w[m] = make_double2(v.x, v.y);
        }
        for (int j = 0; j < k; ++j) {
            const float2 v = x[(size_t)(j + M - 1) * npix + px];
            w[0] = make_double2(v.x, v.y);
#pragma unroll
            for (int a = 0; a < M; ++a)
#pragma unroll
                for (int b = a; b < M; ++b) A[a][b] = zfmacj2(w[b], w[a], A[a][b]);
#pragma unroll
            for (int m = M - 1; m > 0; --m) w[m] = w[m - 1];
        }
#pragma unroll
        for (int a = 0; a < M; ++a) {
            A[a][a].y = 0.0;
#pragma unroll
            for (int b = a + 1; b < M; ++b) A[b][a] = zconj(A[a][b]);
        }
        if (G_out) {
#pragma unroll
            for (int a = 0; a < M; ++a)
#pragma unroll
                for (int b = 0; b < M; ++b) G_out[(px * M + a) * M + b] = A[a][b];
        }
        // cyclic Jacobi: A <- J^H A J with J = diag(1, conj(e)) x real rotation on (p, q)
        double2 V[M][M];
#pragma unroll
        for (int a = 0; a < M; ++a)
#pragma unroll
            for (int b = 0; b < M; ++b) V[a][b] = make_double2(a == b ? 1.0 : 0.0, 0.0);
        for (int sweep = 0; sweep < kJacobiSweeps; ++sweep) {
            double off = 0.0, dg = 0.0;
#pragma unroll
            for (int a = 0; a < M; ++a) {
                dg += A[a][a].x * A[a][a].x;
#pragma unroll
                for (int b = a + 1; b < M; ++b) off += A[a][b].x * A[a][b].x + A[a][b].y * A[a][b].y;
            }
            if (off <= 1e-30 * dg) break;
#pragma unroll
            for (int pp = 0; pp < M; ++pp)
#pragma unroll
                for (int qq = pp + 1; qq < M; ++qq) {
                    const double2 apq = A[pp][qq];
                    const double mag = hypot(apq.x, apq.y);
                    if (mag == 0.0) continue;
                    const double2 e = make_double2(apq.x / mag, apq.y / mag);
                    const double2 ec = zconj(e);
                    const double th = (A[qq][qq].x - A[pp][pp].x) / (2.0 * mag);
                    const double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
                    const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
#pragma unroll
                    for (int i = 0; i < M; ++i) {
                        const double2 aip = A[i][pp], aiq = zmul(ec, A[i][qq]);
                        A[i][pp] = make_double2(c * aip.x - s * aiq.x, c * aip.y - s * aiq.y);
                        A[i][qq] = make_double2(s * aip.x + c * aiq.x, s * aip.y + c * aiq.y);
                        const double2 vip = V[i][pp], viq = zmul(ec, V[i][qq]);
                        V[i][pp] = make_double2(c * vip.x - s * viq.x, c * vip.y - s * viq.y);
                        V[i][qq] = make_double2(s * vip.x + c * viq.x, s * vip.y + c * viq.y);
                    }
#pragma unroll
                    for (int j = 0; j < M; ++j) {
                        const double2 apj = A[pp][j], aqj = zmul(e, A[qq][j]);
                        A[pp][j] = make_double2(c * apj.x - s * aqj.x, c * apj.y - s * aqj.y);
                        A[qq][j] = make_double2(s * apj.x + c * aqj.x, s * apj.y + c * aqj.y);
                    }
                    A[pp][qq] = make_double2(0.0, 0.0);
                    A[qq][pp] = make_double2(0.0, 0.0);
                    A[pp][pp].y = 0.0;
                    A[qq][qq].y = 0.0;
                }
        }
        double lmax = A[0][0].x;
#pragma unroll
        for (int a = 1; a < M; ++a) lmax = fmax(lmax, A[a][a].x);
        if (lmax_out) lmax_out[px] = lmax;
        if (eps_mode == 1) {
            // lambda_max >= 0 (PSD Gram): the bit patterns of non-negative doubles order as the
            // values do
            atomicMax(lmax_max, (unsigned long long)__double_as_longlong(fmax(lmax, 0.0)));
            continue;
        }
        const double eps = eps_mode == 0 ? eps_in[px] : eps_in[0];
        double alpha[M];
#pragma unroll
        for (int i = 0; i < M; ++i) {
            const double l = A[i][i].x + eps;
            alpha[i] = p == 0.0 ? 1.0 / l : pow(l, 0.5 * p - 1.0);
        }
        // S_ab = H_ba = sum_i V[b][i] alpha_i conj(V[a][i]), stored for a <= b
        int e = 0;
#pragma unroll
        for (int a = 0; a < M; ++a)
#pragma unroll
            for (int b = a; b < M; ++b, ++e) {
                double2 h = make_double2(0.0, 0.0);
#pragma unroll
                for (int i = 0; i < M; ++i) {
                    const double2 t2 = zmul(V[b][i], zconj(V[a][i]));
                    h.x += alpha[i] * t2.x;
                    h.y += alpha[i] * t2.y;
                }
                S[(size_t)e * npix + px] = make_float2((float)h.x, (float)h.y);
            }
    }
}

// Tm[col * m + row] with row = (j nr1 + c1) nr2 + c2, col = (mm N1 + l1) N2 + l2:
// centred x_hat[j + M - 1 - mm][c1 + N1 - 1 - l1][c2 + N2 - 1 - l2] (grid.y = column); centred
// index u is natural index (u + P/2) mod P.
template <typename TOut>
__global__ void __launch_bounds__(kThreads)
direct_lift_kernel(const float2* __restrict__ xh, int T, int P, int Q, int N1, int N2, int M,
                   TOut* __restrict__ Tm) {
    const int nr1 = P - N1 + 1, nr2 = Q - N2 + 1, k = T - M + 1;
    const size_t m = (size_t)k * nr1 * nr2;
    const int col = blockIdx.y;
    const int l2 = col % N2, l1 = (col / N2) % N1, mm = col / (N2 * N1);
    for (size_t row = (size_t)blockIdx.x * blockDim.x + threadIdx.x; row < m;
         row += (size_t)gridDim.x * blockDim.x) {
        const int c2 = (int)(row % nr2);
        const int c1 = (int)((row / nr2) % nr1);
        const int j = (int)(row / ((size_t)nr2 * nr1));
        const int k1 = (c1 + N1 - 1 - l1 + P / 2) % P, k2 = (c2 + N2 - 1 - l2 + Q / 2) % Q;
        const float2 v = xh[((size_t)(j + M - 1 - mm) * P + k1) * Q + k2];
        if constexpr (sizeof(TOut) == sizeof(double2)) {
            Tm[(size_t)col * m + row] = make_double2(v.x, v.y);
        } else {
            Tm[(size_t)col * m + row] = v;
        }
    }
}

// z[n][k1][k2] = (mask ? mask * yh : 0) + lam * sum of Y over the lifted entries copied from
// x_hat[n][k1][k2] (the adjoint of direct_lift_kernel, as a gather; natural order in and out).
__global__ void __launch_bounds__(kThreads)
direct_unlift_kernel(const float2* __restrict__ Y, int T, int P, int Q, int N1, int N2, int M,
                     const float2* __restrict__ yh, const uint8_t* __restrict__ mask, float lam,
                     float2* __restrict__ z) {
    const int nr1 = P - N1 + 1, nr2 = Q - N2 + 1, k = T - M + 1;
    const size_t m = (size_t)k * nr1 * nr2;
    const size_t n_el = (size_t)T * P * Q;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_el;
         i += (size_t)gridDim.x * blockDim.x) {
        const int k2 = (int)(i % Q), k1 = (int)((i / Q) % P), n = (int)(i / ((size_t)Q * P));
        const int u1 = (k1 + P / 2) % P, u2 = (k2 + Q / 2) % Q;  // centred position
        float2 acc = make_float2(0.f, 0.f);
        for (int mm = 0; mm < M; ++mm) {
            const int j = n - (M - 1 - mm);
            if (j < 0 || j >= k) continue;
            for (int l1 = 0; l1 < N1; ++l1) {
                const int c1 = u1 - (N1 - 1 - l1);
                if (c1 < 0 || c1 >= nr1) continue;
                for (int l2 = 0; l2 < N2; ++l2) {
                    const int c2 = u2 - (N2 - 1 - l2);
                    if (c2 < 0 || c2 >= nr2) continue;
                    const size_t row = ((size_t)j * nr1 + c1) * nr2 + c2;
                    const size_t col = ((size_t)mm * N1 + l1) * N2 + l2;
                    const float2 y = Y[col * m + row];
                    acc.x += y.x;
                    acc.y += y.y;
                }
            }
        }
        float2 out = make_float2(lam * acc.x, lam * acc.y);
        if (mask && mask[i]) {
            const float2 v = yh[i];
            out.x += v.x;
            out.y += v.y;
        }
        z[i] = out;
    }
}

// Upper triangle of a Hermitian s x s column-major matrix from its lower triangle.
__global__ void herm_fill_kernel(double2* G, int s) {
    const size_t n = (size_t)s * s;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(idx % s), c = (int)(idx / s);
        if (r < c) G[idx] = zconj(G[c + (size_t)r * s]);
        else if (r == c) G[idx].y = 0.0;
    }
}

// H = U diag((lambda + eps)^(p/2-1)) U^H (s x s column-major) from the eigenpairs.
__global__ void form_H_kernel(const double2* __restrict__ U, const double* __restrict__ evals,
                              const double* __restrict__ eps_p, double p, int s,
                              double2* __restrict__ H) {
    const size_t n = (size_t)s * s;
    const double eps = eps_p[0];
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int a = (int)(idx % s), b = (int)(idx / s);
        double2 acc = make_double2(0.0, 0.0);
        for (int i = 0; i < s; ++i) {
            const double l = evals[i] + eps;
            const double al = p == 0.0 ? 1.0 / l : pow(l, 0.5 * p - 1.0);
            const double2 t = zmul(U[a + (size_t)i * s], zconj(U[b + (size_t)i * s]));
            acc.x += al * t.x;
            acc.y += al * t.y;
        }
        H[idx] = acc;
    }
}

// delta = H_old - H_new (or -H_new without H_old) and h32 = H_new, both rounded to complex64.
__global__ void h_delta_kernel(const double2* __restrict__ H_new, const double2* __restrict__ H_old,
                               float2* __restrict__ delta, float2* __restrict__ h32, size_t n) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const double2 hn = H_new[i];
        double2 d = make_double2(-hn.x, -hn.y);
        if (H_old) {
            d.x += H_old[i].x;
            d.y += H_old[i].y;
        }
        delta[i] = make_float2((float)d.x, (float)d.y);
        h32[i] = make_float2((float)hn.x, (float)hn.y);
    }
}

// ---- plain CG of the direct variant (scalars on the device) ----

// *out = Re <a, b> (FP32 Kahan per thread, FP64 across threads and blocks).
__global__ void __launch_bounds__(kThreads)
dcg_dot_kernel(const float2* __restrict__ a, const float2* __restrict__ b, size_t n,
               double* __restrict__ parts, unsigned int* counter, double* __restrict__ out) {
    __shared__ double red[kThreads / 32];
    float acc = 0.f, comp = 0.f;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const float2 u = a[i], v = b[i];
        const float term = fmaf(u.x, v.x, u.y * v.y) - comp;
        const float sum = acc + term;
        comp = (sum - acc) - term;
        acc = sum;
    }
    const double tot = block_sum_f_t0(acc, red);
    last_block_sum(tot, parts, counter, out);
}

// r = (first ? 0 : r) + w, *rr_out = |r|^2
__global__ void __launch_bounds__(kThreads)
dcg_resid_kernel(float2* __restrict__ r, const float2* __restrict__ w, int first, size_t n,
                 double* __restrict__ parts, unsigned int* counter, double* __restrict__ rr_out) {
    __shared__ double red[kThreads / 32];
    float acc = 0.f, comp = 0.f;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        float2 v = w[i];
        if (!first) {
            const float2 o = r[i];
            v.x += o.x;
            v.y += o.y;
        }
        r[i] = v;
        const float term = fmaf(v.x, v.x, v.y * v.y) - comp;
        const float sum = acc + term;
        comp = (sum - acc) - term;
        acc = sum;
    }
    const double tot = block_sum_f_t0(acc, red);
    last_block_sum(tot, parts, counter, rr_out);
}

// alpha = *rr / *pq; x += alpha p; r -= alpha q; *rr_out = |r|^2
__global__ void __launch_bounds__(kThreads)
dcg_update_kernel(float2* __restrict__ x, float2* __restrict__ r, const float2* __restrict__ p,
                  const float2* __restrict__ q, size_t n, const double* __restrict__ rr,
                  const double* __restrict__ pq, double* __restrict__ parts, unsigned int* counter,
                  double* __restrict__ rr_out) {
    __shared__ double red[kThreads / 32];
    const float alpha = (float)(rr[0] / pq[0]);
    float acc = 0.f, comp = 0.f;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        float2 xv = x[i], rv = r[i];
        const float2 pv = p[i], qv = q[i];
        xv.x = fmaf(alpha, pv.x, xv.x);
        xv.y = fmaf(alpha, pv.y, xv.y);
        rv.x = fmaf(-alpha, qv.x, rv.x);
        rv.y = fmaf(-alpha, qv.y, rv.y);
        x[i] = xv;
        r[i] = rv;
        const float term = fmaf(rv.x, rv.x, rv.y * rv.y) - comp;
        const float sum = acc + term;
        comp = (sum - acc) - term;
        acc = sum;
    }
    const double tot = block_sum_f_t0(acc, red);
    last_block_sum(tot, parts, counter, rr_out);
}

// p = r (first) or r + (*rr_new / *rr_old) p
__global__ void __launch_bounds__(kThreads)
dcg_pupdate_kernel(float2* __restrict__ p, const float2* __restrict__ r, size_t n,
                   const double* __restrict__ rr_new, const double* __restrict__ rr_old,
                   int first) {
    const float beta = first ? 0.f : (float)(rr_new[0] / rr_old[0]);
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        float2 v = r[i];
        if (!first) {
            const float2 o = p[i];
            v.x = fmaf(beta, o.x, v.x);
            v.y = fmaf(beta, o.y, v.y);
        }
        p[i] = v;
    }
}

int grid_for(size_t n, int cap) {
    const size_t g = (n + kThreads - 1) / kThreads;
    return (int)(g < (size_t)cap ? (g < 1 ? 1 : g) : (size_t)cap);
}

}  // namespace

size_t direct_rows(const Dims& d) {
    return (size_t)(d.T - d.M + 1) * (d.P - d.N1 + 1) * (d.Q - d.N2 + 1);
}

cudaError_t launch_voxel_weight(const Dims& d, const float2* x, double p, const double* eps_in,
                                double* lmax_max, int eps_mode, float2* S, double2* G_out,
                                double* lmax_out, cudaStream_t st) {
    const size_t npix = d.pixels();
    const int g = grid_for(npix * 2, 4 * num_sms() * 4);
    const int grid = (int)((npix + kVoxThreads - 1) / kVoxThreads) < g
                         ? (int)((npix + kVoxThreads - 1) / kVoxThreads) : g;
    unsigned long long* mx = reinterpret_cast<unsigned long long*>(lmax_max);
#define CASE(MM)                                                                               \
    case MM:                                                                                   \
        voxel_weight_kernel<MM><<<grid, kVoxThreads, 0, st>>>(x, d.T, npix, p, eps_in, mx,      \
                                                              eps_mode, S, G_out, lmax_out);   \
        break;
    switch (d.M) {
        CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6)
        default: return cudaErrorInvalidValue;
    }
#undef CASE
    return cudaGetLastError();
}

cudaError_t launch_direct_lift(const Dims& d, const float2* xh, void* Tm, int fp64,
                               cudaStream_t st) {
    const size_t m = direct_rows(d);
    dim3 grid((unsigned)grid_for(m, 1024), (unsigned)d.s());
    if (fp64)
        direct_lift_kernel<double2><<<grid, kThreads, 0, st>>>(xh, d.T, d.P, d.Q, d.N1, d.N2, d.M,
                                                              (double2*)Tm);
    else
        direct_lift_kernel<float2><<<grid, kThreads, 0, st>>>(xh, d.T, d.P, d.Q, d.N1, d.N2, d.M,
                                                             (float2*)Tm);
    return cudaGetLastError();
}

cudaError_t launch_direct_unlift(const Dims& d, const float2* Y, const float2* yh,
                                 const uint8_t* mask, float lam, float2* z, cudaStream_t st) {
    direct_unlift_kernel<<<grid_for(d.elems(), 8 * num_sms()), kThreads, 0, st>>>(
        Y, d.T, d.P, d.Q, d.N1, d.N2, d.M, yh, mask, lam, z);
    return cudaGetLastError();
}

cudaError_t launch_herm_fill(double2* G, int s, cudaStream_t st) {
    herm_fill_kernel<<<grid_for((size_t)s * s, 1024), kThreads, 0, st>>>(G, s);
    return cudaGetLastError();
}

cudaError_t launch_form_H(const double2* U, const double* evals, const double* eps, double p,
                          int s, double2* H, cudaStream_t st) {
    form_H_kernel<<<grid_for((size_t)s * s, 4096), kThreads, 0, st>>>(U, evals, eps, p, s, H);
    return cudaGetLastError();
}

cudaError_t launch_h_delta(const double2* H_new, const double2* H_old, float2* delta, float2* h32,
                           size_t n, cudaStream_t st) {
    h_delta_kernel<<<grid_for(n, 1024), kThreads, 0, st>>>(H_new, H_old, delta, h32, n);
    return cudaGetLastError();
}

cudaError_t launch_dcg_dot(const float2* a, const float2* b, size_t n, const RedSlot& rs,
                           double* out, cudaStream_t st) {
    dcg_dot_kernel<<<grid_for(n, max_parts()), kThreads, 0, st>>>(a, b, n, rs.parts, rs.counter, out);
    return cudaGetLastError();
}

cudaError_t launch_dcg_resid(float2* r, const float2* w, int first, size_t n, const RedSlot& rs,
                             double* rr_out, cudaStream_t st) {
    dcg_resid_kernel<<<grid_for(n, max_parts()), kThreads, 0, st>>>(r, w, first, n, rs.parts,
                                                                   rs.counter, rr_out);
    return cudaGetLastError();
}

cudaError_t launch_dcg_update(float2* x, float2* r, const float2* p, const float2* q, size_t n,
                              const double* rr, const double* pq, const RedSlot& rs,
                              double* rr_out, cudaStream_t st) {
    dcg_update_kernel<<<grid_for(n, max_parts()), kThreads, 0, st>>>(x, r, p, q, n, rr, pq, rs.parts,
                                                                    rs.counter, rr_out);
    return cudaGetLastError();
}

cudaError_t launch_dcg_pupdate(float2* p, const float2* r, size_t n, const double* rr_new,
                               const double* rr_old, int first, cudaStream_t st) {
    dcg_pupdate_kernel<<<grid_for(n, 8 * num_sms()), kThreads, 0, st>>>(p, r, n, rr_new, rr_old,
                                                                       first);
    return cudaGetLastError();
}

}  // namespace recon
