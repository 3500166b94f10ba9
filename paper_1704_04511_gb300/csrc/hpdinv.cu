// FP64 weight for p = 0 without an eigendecomposition (Sec. III-B, Eq. weight-update):
//   H = (G + eps I)^(p/2 - 1) = (G + eps I)^(-1)   when p = 0,
// and eps0 = eps0_frac * lambda_max(G) (Sec. III-C) from a Lanczos iteration.
//
// The inverse is a blocked Hermitian sweep (Gauss-Jordan without pivoting, stable for Hermitian
// positive-definite matrices) over 8 x 8 tiles, run as ONE cooperative kernel over every SM
// (each CTA works four tiles at once in 64-thread groups with named barriers):
//   per pivot block K:  D^-1 = (A_KK)^-1 (computed one step ahead by the CTA that owns A_KK),
//                       W_KJ = D^-1 A_KJ,  C_IK = A_IK            (phase A, whole grid)
//                       A_IJ -= C_IK W_KJ,  A_IK <- C_IK D^-1,  A_KJ <- W_KJ,  A_KK <- -D^-1
//                                                                 (phase B, lower tiles only)
// Sweeping every pivot leaves -A^{-1}; the Hermitian symmetry is kept at each step, so only the
// lower tiles (and the full diagonal tiles) are updated. Grid barriers are bounded spin-waits:
// on timeout the kernel records an error flag and returns.
#include "common.cuh"
#include "kernels.h"

namespace recon {

namespace {

constexpr int kThreads = 256;
constexpr int kB = 8;                        // tile edge
constexpr int kTileT = kB * kB;              // threads per tile group
constexpr int kGroups = kThreads / kTileT;   // tiles a CTA works on at once
constexpr long long kSpinLimit = 1LL << 26;  // polls (~1 us each at most) before giving up

struct GridBar {
    unsigned int count;
    unsigned int gen;
    int err;
    int pad;
};

RECON_DEV unsigned int ld_acquire(const unsigned int* p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
RECON_DEV int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Generation barrier over gridDim.x co-resident CTAs (cooperative launch). Thread 0 of each CTA
// arrives with one atomic and then polls the generation word with plain acquire loads. Returns
// false (and sets gb->err) if the wait exceeded kSpinLimit polls; after a failure every later
// call returns false at once so the kernel can unwind.
RECON_DEV bool grid_barrier(GridBar* gb) {
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = (ld_acquire(&gb->err) == 0);
        if (ok) {
            const unsigned int g = ld_acquire(&gb->gen);
            __threadfence();
            const unsigned int arrived = atomicAdd(&gb->count, 1u) + 1u;
            if (arrived == gridDim.x) {
                atomicExch(&gb->count, 0u);
                __threadfence();
                atomicAdd(&gb->gen, 1u);
            } else {
                long long it = 0;
                while (ld_acquire(&gb->gen) == g) {
                    if (++it > kSpinLimit) {
                        atomicExch(&gb->err, 1);
                        ok = 0;
                        break;
                    }
                    if ((it & 1023) == 0 && ld_acquire(&gb->err) != 0) {
                        ok = 0;
                        break;
                    }
                }
            }
            __threadfence();
        }
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

// Synchronise the 64 threads of tile group g (named barrier g + 1; 0 is __syncthreads).
RECON_DEV void group_sync(int g) {
    asm volatile("bar.sync %0, %1;" ::"r"(g + 1), "r"(kTileT) : "memory");
}

// Inverse of a Hermitian positive-definite 8 x 8 tile held (full, column-major) in the group's
// shared memory, by 8 scalar sweeps (which leave -T^{-1}); the negated result goes to `out`.
// Called by the 64 threads of one tile group.
RECON_DEV void tile_inverse(double2* T, double2* out, double* s_inv, double2* s_row, int g) {
    const int e = threadIdx.x % kTileT, i = e % kB, j = e / kB;
    for (int k = 0; k < kB; ++k) {
        if (e == 0) *s_inv = rcp_nr(T[k + k * kB].x);  // one reciprocal per pivot
        group_sync(g);
        const double inv = *s_inv;
        if (e < kB) {
            const double2 t = T[k + e * kB];  // row k, scaled once
            s_row[e] = make_double2(t.x * inv, t.y * inv);
        }
        const double2 tij = T[i + j * kB], tik = T[i + k * kB];
        group_sync(g);
        double2 v;
        if (i == k && j == k) v = make_double2(-inv, 0.0);
        else if (i == k) v = s_row[j];
        else if (j == k) v = make_double2(tik.x * inv, tik.y * inv);
        else v = zfms(tik, s_row[j], tij);
        T[i + j * kB] = v;
        group_sync(g);
    }
    const double2 v = T[i + j * kB];
    out[i + j * kB] = make_double2(-v.x, -v.y);
    group_sync(g);
}

__global__ void __launch_bounds__(kThreads)
hpd_sweep_kernel(double2* G, int s, const double* __restrict__ eps_p, int np,
                 double2* __restrict__ A, double2* __restrict__ Dinv2, double2* __restrict__ W,
                 double2* __restrict__ C, GridBar* gb) {
    __shared__ double2 ta[kGroups][kTileT];
    __shared__ double2 tb[kGroups][kTileT];
    __shared__ double s_inv[kGroups];
    __shared__ double2 s_row[kGroups][kB];
    const int nt = np / kB;
    const double eps = eps_p[0];
    const int tid = threadIdx.x;
    const int g = tid / kTileT, e = tid % kTileT;
    const int ii = e % kB, jj = e / kB;
    const size_t gtid = (size_t)blockIdx.x * blockDim.x + tid;
    const size_t gstride = (size_t)gridDim.x * blockDim.x;
    // interleaved index: consecutive work items go to different CTAs (spreads the FP64 work)
    const size_t itid = (size_t)tid * gridDim.x + blockIdx.x;

    // A = pad(G + eps I): lower tiles and full diagonal tiles are the live part
    for (size_t idx = gtid; idx < (size_t)np * np; idx += gstride) {
        const int i = (int)(idx % np), j = (int)(idx / np);
        double2 v = make_double2(i == j ? 1.0 : 0.0, 0.0);
        if (i < s && j < s) {
            v = G[i + (size_t)j * s];
            if (i == j) v.x += eps;
        }
        A[idx] = v;
    }
    if (!grid_barrier(gb)) return;
    if (blockIdx.x == 0 && g == 0) {
        ta[0][e] = A[ii + (size_t)jj * np];
        group_sync(0);
        tile_inverse(ta[0], Dinv2, &s_inv[0], s_row[0], 0);
    }
    if (!grid_barrier(gb)) return;

    const int nlt = nt * (nt + 1) / 2;
    const int ngroups = gridDim.x * kGroups;
    for (int K = 0; K < nt; ++K) {
        const double2* D = Dinv2 + (K & 1) * kTileT;
        double2* Dnext = Dinv2 + ((K + 1) & 1) * kTileT;
        const int k0 = K * kB;
        // ---- phase A: W = D^-1 A_K,: (8 x np) and C = A_:,K (np x 8), old values
        if (itid < (size_t)np * kB) {
            const int m = (int)(itid % kB);       // pivot-local index
            const int col = (int)(itid / kB);     // global column (for W) / row (for C)
            const int J = col / kB;
            double2 acc = make_double2(0.0, 0.0);
            if (J != K) {
#pragma unroll
                for (int q = 0; q < kB; ++q) {
                    const double2 a = (J < K) ? A[(k0 + q) + (size_t)col * np]
                                              : zconj(A[col + (size_t)(k0 + q) * np]);
                    acc = zfma(D[m + q * kB], a, acc);
                }
            }
            W[m + (size_t)col * kB] = acc;
            C[col + (size_t)m * np] = (J >= K) ? A[col + (size_t)(k0 + m) * np]
                                               : zconj(A[(k0 + m) + (size_t)col * np]);
        }
        if (!grid_barrier(gb)) return;
        // ---- phase B: lower tiles, one per 64-thread group; the group that owns tile
        // (K+1, K+1) also inverts it (look-ahead pivot)
        for (int t = blockIdx.x * kGroups + g; t < nlt; t += ngroups) {
            int I = 0, rem = t;
            while (rem > I) { rem -= I + 1; ++I; }
            const int J = rem;                    // J <= I
            const int row = I * kB + ii, col = J * kB + jj;
            double2 v;
            if (I == K && J == K) {
                const double2 dd = D[ii + jj * kB];
                v = make_double2(-dd.x, -dd.y);
            } else if (I == K) {
                v = W[ii + (size_t)col * kB];
            } else if (J == K) {
                double2 acc = make_double2(0.0, 0.0);
#pragma unroll
                for (int q = 0; q < kB; ++q) acc = zfma(C[row + (size_t)q * np], D[q + jj * kB], acc);
                v = acc;
            } else {
                ta[g][e] = C[(I * kB + ii) + (size_t)jj * np];
                tb[g][e] = W[ii + (size_t)(J * kB + jj) * kB];
                group_sync(g);
                double2 acc = A[row + (size_t)col * np];
#pragma unroll
                for (int q = 0; q < kB; ++q) acc = zfms(ta[g][ii + q * kB], tb[g][q + jj * kB], acc);
                v = acc;
                group_sync(g);
            }
            A[row + (size_t)col * np] = v;
            if (I == J && I == K + 1) {
                ta[g][e] = v;
                group_sync(g);
                tile_inverse(ta[g], Dnext, &s_inv[g], s_row[g], g);
            }
        }
        if (!grid_barrier(gb)) return;
    }
    // ---- H = -A (s x s, full, column-major) written over G
    for (size_t idx = gtid; idx < (size_t)s * s; idx += gstride) {
        const int i = (int)(idx % s), j = (int)(idx / s);
        const int I = i / kB, J = j / kB;
        const double2 v = (I >= J) ? A[i + (size_t)j * np] : zconj(A[j + (size_t)i * np]);
        G[idx] = make_double2(-v.x, -v.y);
    }
}

// d_ab[delta] = sum_{l - l' = delta} H[(l', b), (l, a)] from H (s x s column-major).
__global__ void hdiag_kernel(const double2* __restrict__ H, int N1, int N2, int M,
                             double2* __restrict__ dsum) {
    const int L1 = 2 * N1 - 1, L2 = 2 * N2 - 1;
    const int npair = M * (M + 1) / 2;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= npair * L1 * L2) return;
    const int pr = warp / (L1 * L2), rem = warp % (L1 * L2);
    const int d1 = rem / L2 - (N1 - 1), d2 = rem % L2 - (N2 - 1);
    int a = 0, e = pr;
    while (e >= M - a) { e -= M - a; ++a; }
    const int b = a + e;
    const int s = N1 * N2 * M;
    const int lo1 = max(0, -d1), hi1 = min(N1, N1 - d1);
    const int lo2 = max(0, -d2), hi2 = min(N2, N2 - d2);
    const int n2 = hi2 - lo2;
    const int cnt = (hi1 - lo1) * n2;
    double2 acc = make_double2(0.0, 0.0);
    for (int t = lane; t < cnt; t += 32) {
        const int lp1 = lo1 + t / n2, lp2 = lo2 + t % n2;
        const size_t rowi = ((size_t)b * N1 + lp1) * N2 + lp2;
        const size_t coli = ((size_t)a * N1 + lp1 + d1) * N2 + lp2 + d2;
        acc = zadd(acc, H[rowi + coli * s]);
    }
    acc.x = warp_sum(acc.x);
    acc.y = warp_sum(acc.y);
    if (lane == 0) dsum[warp] = acc;
}

// ---- Lanczos estimate of lambda_max(G), FP64, m steps, then multisection on the tridiagonal.
__global__ void __launch_bounds__(kThreads)
lanczos_kernel(const double2* __restrict__ G, int s, int m, double2* __restrict__ u,
               double2* __restrict__ vprev, double* __restrict__ part, double* __restrict__ ab,
               double* __restrict__ lmax_out, GridBar* gb) {
    __shared__ double red[kThreads / 32];
    __shared__ double s_beta, s_ib, s_alpha;
    __shared__ double sh_lo, sh_hi;
    __shared__ int s_m;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nw = gridDim.x * (kThreads / 32);
    const int gw = blockIdx.x * (kThreads / 32) + warp;
    // deterministic start vector, unnormalised: u_i = 1 + 0.5 sin(i) + i 0.25 i cos(3 i) / s
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < s; i += gridDim.x * blockDim.x) {
        u[i] = make_double2(1.0 + 0.5 * sin((double)i), 0.25 * cos(3.0 * i) * i / s);
        vprev[i] = make_double2(0.0, 0.0);
    }
    if (!grid_barrier(gb)) return;
    if (warp == 0) {
        double acc = 0.0;
        for (int i = lane; i < s; i += 32) acc += u[i].x * u[i].x + u[i].y * u[i].y;
        acc = warp_sum(acc);
        if (lane == 0) {
            s_beta = sqrt(acc);
            s_ib = rcp_nr(s_beta);
            s_m = m;
        }
    }
    __syncthreads();
    for (int k = 0; k < m; ++k) {
        // v_k = u / beta_{k-1};  w = G v_k - alpha_k v_k - beta_{k-1} v_{k-1};  beta_k = |w|
        const double beta = s_beta, ib = s_ib;
        double* pa = part + (size_t)(k & 1) * 2 * gridDim.x;   // alpha partials (ping-pong)
        double* pb = pa + gridDim.x;                            // beta partials
        double ap = 0.0;
        double2 yrow[4];
        int nrow = 0;
        for (int i = gw; i < s && nrow < 4; i += nw, ++nrow) {
            // row i of the Hermitian G is the conjugate of column i (contiguous)
            double2 acc = make_double2(0.0, 0.0);
            const double2* gcol = G + (size_t)i * s;
            for (int j = lane; j < s; j += 32) {
                const double2 g = gcol[j], uj = u[j];
                acc.x = fma(g.x, uj.x, acc.x);
                acc.x = fma(g.y, uj.y, acc.x);
                acc.y = fma(g.x, uj.y, acc.y);
                acc.y = fma(-g.y, uj.x, acc.y);
            }
            acc.x = warp_sum(acc.x) * ib;
            acc.y = warp_sum(acc.y) * ib;
            yrow[nrow] = acc;
            const double2 vi = make_double2(u[i].x * ib, u[i].y * ib);
            ap += vi.x * acc.x + vi.y * acc.y;
        }
        __syncthreads();
        if (lane == 0) red[warp] = ap;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < kThreads / 32; ++w) t += red[w];
            pa[blockIdx.x] = t;
        }
        if (!grid_barrier(gb)) return;
        if (warp == 0) {
            const double al = warp0_sum_array(pa, gridDim.x);
            if (lane == 0) s_alpha = al;
        }
        __syncthreads();
        const double alpha = s_alpha;
        double bp = 0.0;
        nrow = 0;
        for (int i = gw; i < s && nrow < 4; i += nw, ++nrow) {
            if (lane == 0) {
                const double2 vi = make_double2(u[i].x * ib, u[i].y * ib);
                const double2 vp = vprev[i];
                const double2 un = make_double2(yrow[nrow].x - alpha * vi.x - beta * vp.x,
                                                yrow[nrow].y - alpha * vi.y - beta * vp.y);
                bp += un.x * un.x + un.y * un.y;
                vprev[i] = vi;
                u[i] = un;
            }
        }
        if (lane == 0) red[warp] = bp;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < kThreads / 32; ++w) t += red[w];
            pb[blockIdx.x] = t;
        }
        if (!grid_barrier(gb)) return;
        if (warp == 0) {
            const double b2 = warp0_sum_array(pb, gridDim.x);
            if (lane == 0) {
                const double bnew = sqrt(b2);
                if (blockIdx.x == 0) {
                    ab[2 * k] = alpha;
                    ab[2 * k + 1] = bnew;
                }
                s_beta = bnew;
                s_ib = rcp_nr(bnew);
                if (!(bnew > 1e-300 * fabs(alpha) + 1e-300)) s_m = k + 1;
            }
        }
        __syncthreads();
        if (s_m == k + 1) break;
    }
    m = s_m;
    // Largest eigenvalue of the m x m tridiagonal (alpha_k, beta_k) by multisection with Sturm
    // counts (CTA 0): FP32 rounds over the whole block to 1e-4 relative (FP32 counts are exact
    // for x farther than ~m eps32 |T| from an eigenvalue), then FP64 rounds on
    // one warp (FP64 divisions are expensive here, so few threads evaluate them).
    if (blockIdx.x != 0) return;
    __shared__ int best;
    __syncthreads();
    if (threadIdx.x == 0) {
        double lo = 1e300, hi = -1e300;
        for (int k = 0; k < m; ++k) {
            const double r = (k > 0 ? fabs(ab[2 * k - 1]) : 0.0) + (k + 1 < m ? fabs(ab[2 * k + 1]) : 0.0);
            lo = fmin(lo, ab[2 * k] - r);
            hi = fmax(hi, ab[2 * k] + r);
        }
        const double pad = 1e-6 * fmax(fabs(lo), fabs(hi));
        sh_lo = lo - pad;
        sh_hi = hi + pad;
    }
    __syncthreads();
    for (int round = 0; round < 24; ++round) {
        const bool fp32 = (sh_hi - sh_lo) > 1e-4 * fabs(sh_hi);
        const int nthr = fp32 ? (int)blockDim.x : 32;
        const double lo = sh_lo, hi = sh_hi;
        int cnt = m;
        if ((int)threadIdx.x < nthr) {
            const double x = lo + (hi - lo) * (threadIdx.x + 1) / (double)(nthr + 1);
            cnt = 0;
            if (fp32) {
                const float xf = (float)x;
                float d = 1.f;
                for (int k = 0; k < m; ++k) {
                    const float bb = k > 0 ? (float)(ab[2 * k - 1] * ab[2 * k - 1]) : 0.f;
                    d = ((float)ab[2 * k] - xf) - (k > 0 ? bb * __frcp_rn(d) : 0.f);
                    if (d == 0.f) d = -1e-30f;
                    if (d < 0.f) ++cnt;
                }
            } else {
                double d = 1.0;
                for (int k = 0; k < m; ++k) {
                    const double bb = k > 0 ? ab[2 * k - 1] * ab[2 * k - 1] : 0.0;
                    d = (ab[2 * k] - x) - (k > 0 ? bb * rcp_nr(d) : 0.0);
                    if (d == 0.0) d = -1e-300;
                    if (d < 0.0) ++cnt;
                }
            }
        }
        // the largest eigenvalue lies above the largest sample x with cnt < m
        if (threadIdx.x == 0) best = -1;
        __syncthreads();
        if ((int)threadIdx.x < nthr && cnt < m) atomicMax(&best, (int)threadIdx.x);
        __syncthreads();
        if (threadIdx.x == 0) {
            const double step = (hi - lo) / (double)(nthr + 1);
            const double nlo = lo + step * (best + 1);
            // FP32 counts near the root may be off by rounding: keep one step of margin
            sh_lo = fp32 ? fmax(lo, nlo - step) : nlo;
            sh_hi = fp32 ? fmin(hi, nlo + 2 * step) : nlo + step;
        }
        __syncthreads();
        if (sh_hi - sh_lo <= 2e-16 * fabs(sh_hi)) break;
    }
    if (threadIdx.x == 0) lmax_out[0] = 0.5 * (sh_lo + sh_hi);
}

int coop_grid(const void* kern, int* grid) {
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kThreads, 0) != cudaSuccess) return -1;
    if (per < 1) return -1;
    *grid = sms;  // one CTA per SM
    return 0;
}

int padded(int s) { return (s + kB - 1) / kB * kB; }

// Cooperative launch (all CTAs co-resident, required by the grid barriers) through
// cudaLaunchKernelEx so that it can be captured into a CUDA graph.
template <typename... KArgs, typename... Args>
cudaError_t launch_coop(void (*kern)(KArgs...), int grid, cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kThreads);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

}  // namespace

size_t hpd_scratch_bytes(const Dims& d) {
    const size_t np = (size_t)padded(d.s());
    return 256 + np * np * sizeof(double2) + 2 * kB * kB * sizeof(double2) +
           2 * np * kB * sizeof(double2) + 1024;
}

size_t lanczos_scratch_bytes(const Dims& d, int grid_max) {
    return 256 + 2 * (size_t)d.s() * sizeof(double2) + 4 * (size_t)grid_max * sizeof(double) +
           2 * 96 * sizeof(double) + 1024;
}

cudaError_t launch_hpd_inverse(const Dims& d, double2* G, const double* eps, void* scratch,
                               int* err_flag_out, cudaStream_t st) {
    const int s = d.s(), np = padded(s);
    unsigned char* p = reinterpret_cast<unsigned char*>(scratch);
    GridBar* gb = reinterpret_cast<GridBar*>(p);
    p += 256;
    double2* A = reinterpret_cast<double2*>(p);
    p += (size_t)np * np * sizeof(double2);
    double2* Dinv2 = reinterpret_cast<double2*>(p);
    p += 2 * kB * kB * sizeof(double2);
    double2* W = reinterpret_cast<double2*>(p);
    p += (size_t)np * kB * sizeof(double2);
    double2* C = reinterpret_cast<double2*>(p);
    cudaError_t e = cudaMemsetAsync(gb, 0, sizeof(GridBar), st);
    if (e != cudaSuccess) return e;
    int grid = 0;
    if (coop_grid((const void*)hpd_sweep_kernel, &grid)) return cudaErrorInvalidConfiguration;
    e = launch_coop(hpd_sweep_kernel, grid, st, G, s, eps, np, A, Dinv2, W, C, gb);
    if (e != cudaSuccess) return e;
    if (err_flag_out) {
        // fold the barrier error into the caller's flag (max)
        e = cudaMemcpyAsync(err_flag_out, &gb->err, sizeof(int), cudaMemcpyDeviceToDevice, st);
    }
    return e;
}

cudaError_t launch_hdiag(const Dims& d, const double2* H, double2* dsum, cudaStream_t st) {
    const int nout = d.npair() * d.L1() * d.L2();
    const int warps_per_block = 8;
    hdiag_kernel<<<(nout + warps_per_block - 1) / warps_per_block, 32 * warps_per_block, 0, st>>>(
        H, d.N1, d.N2, d.M, dsum);
    return cudaGetLastError();
}

cudaError_t launch_lanczos_lmax(const Dims& d, const double2* G, void* scratch, double* lmax,
                                int* err_flag_out, cudaStream_t st) {
    int grid = 0;
    if (coop_grid((const void*)lanczos_kernel, &grid)) return cudaErrorInvalidConfiguration;
    const int s = d.s();
    int m = s < 96 ? s : 96;
    unsigned char* p = reinterpret_cast<unsigned char*>(scratch);
    GridBar* gb = reinterpret_cast<GridBar*>(p);
    p += 256;
    double2* u = reinterpret_cast<double2*>(p);
    p += (size_t)s * sizeof(double2);
    double2* vprev = reinterpret_cast<double2*>(p);
    p += (size_t)s * sizeof(double2);
    double* part = reinterpret_cast<double*>(p);
    p += 4 * (size_t)grid * sizeof(double);
    double* ab = reinterpret_cast<double*>(p);
    cudaError_t e = cudaMemsetAsync(gb, 0, sizeof(GridBar), st);
    if (e != cudaSuccess) return e;
    e = launch_coop(lanczos_kernel, grid, st, G, s, m, u, vprev, part, ab, lmax, gb);
    if (e != cudaSuccess) return e;
    if (err_flag_out) e = cudaMemcpyAsync(err_flag_out, &gb->err, sizeof(int), cudaMemcpyDeviceToDevice, st);
    return e;
}

}  // namespace recon
