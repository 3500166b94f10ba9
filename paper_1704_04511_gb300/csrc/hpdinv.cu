// FP64 weight for p = 0 without an eigendecomposition (Sec. III-B, Eq. weight-update):
//   H = (G + eps I)^(p/2 - 1) = (G + eps I)^(-1)   when p = 0,
// and eps0 = eps0_frac * lambda_max(G) (Sec. III-C) from a Lanczos iteration.
//
// The inverse is a blocked Hermitian sweep (Gauss-Jordan without pivoting, stable for Hermitian
// positive-definite matrices) over 8 x 8 tiles of the padded matrix. Sweeping pivot block K with
// D = (A_KK)^-1 maps, for I, J != K,
//     A_IJ -> A_IJ - A_IK D A_KJ,   A_IK -> A_IK D,   A_KJ -> D A_KJ,   A_KK -> -D,
// and sweeping every pivot leaves -A^{-1}. Hermitian symmetry holds after every step, so only the
// lower tiles are kept (tile-major, 1 KB per tile). The kernel is ONE cooperative launch, one grid
// barrier per pivot step, the lower tiles ping-ponging between two buffers so that a step reads
// only the previous step's values:
//   - "diagonal" CTAs own the diagonal tiles; the owner of tile (K+1, K+1) updates it first with
//     the whole CTA and inverts it (the next pivot, D_{K+1}) while its other warps update the
//     CTA's remaining diagonal tiles, so the serial pivot chain never waits behind bulk work;
//   - the other CTAs each own chunks of up to four tiles of one tile row I: the chunk forms
//     X = A_IK D_K once (split over the CTA's eight warps) and each 64-thread group applies
//     A_IJ - X A_KJ to its tile.
// FP64 on this part issues one warp instruction per ~19 cycles per SM whatever the active lanes,
// so the products use full warps and the work is spread over every SM. Grid barriers are bounded
// spin-waits: on timeout the kernel records an error flag and returns.
#include "common.cuh"
#include "kernels.h"

namespace recon {

namespace {

constexpr int kThreads = 256;
constexpr int kB = 8;                        // tile edge
constexpr int kTileT = kB * kB;              // elements of a tile = threads of a tile group
constexpr int kGroups = kThreads / kTileT;   // tile groups per CTA
constexpr int kChunk = 4;                    // off-diagonal tiles of one row handled per CTA pass
constexpr int kMaxChunks = 128;              // chunks one off-diagonal CTA may own
constexpr long long kSpinLimit = 1LL << 26;  // polls (~1 us each at most) before giving up

struct GridBar {
    unsigned int word;  // bit 31 flips when the last CTA arrives; bits 0-30 count arrivals
    int err;
    unsigned int pad[2];
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
RECON_DEV unsigned int atom_add_release(unsigned int* p, unsigned int v) {
    unsigned int old;
    asm volatile("atom.add.release.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

// Barrier over gridDim.x co-resident CTAs (cooperative launch) with one atomic per CTA: CTA 0 adds
// 2^31 - (gridDim.x - 1) and every other CTA adds 1, so bit 31 of the word flips exactly when the
// last CTA arrives and the low bits return to zero. Thread 0 of each CTA then polls the word with
// acquire loads. Returns false (and sets gb->err) if the wait exceeded kSpinLimit polls; after a
// failure every later call returns false at once so the kernel can unwind.
RECON_DEV bool grid_barrier(GridBar* gb) {
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = (ld_acquire(&gb->err) == 0);
        if (ok) {
            __threadfence();
            const unsigned int inc = blockIdx.x == 0 ? 0x80000000u - (gridDim.x - 1u) : 1u;
            const unsigned int old = atom_add_release(&gb->word, inc);
            long long it = 0;
            while (((ld_acquire(&gb->word) ^ old) & 0x80000000u) == 0u) {
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

// Lower tile (I, J), J <= I: offset of its 64 elements, element (i, j) at i + 8 j.
RECON_DEV size_t tile_off(int I, int J) { return ((size_t)I * (I + 1) / 2 + J) * kTileT; }

// Element e = i + 8 q of the block (I, K) of the full Hermitian matrix held as lower tiles.
RECON_DEV double2 block_elem(const double2* A, int I, int K, int e) {
    if (I >= K) return A[tile_off(I, K) + e];
    return zconj(A[tile_off(K, I) + e / kB + kB * (e % kB)]);
}

// (I, J) of lower tile number t in row-major order of the lower triangle.
RECON_DEV void tile_ij(int t, int* I, int* J) {
    int r = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
    while (r * (r + 1) / 2 > t) --r;
    while ((r + 1) * (r + 2) / 2 <= t) ++r;
    *I = r;
    *J = t - r * (r + 1) / 2;
}

struct SweepSmem {
    double2 D[kTileT];              // D_K
    double2 P[kGroups][kTileT];     // A_IK per group (diagonal CTAs) / per chunk (slot 0)
    double2 B[kGroups][kTileT];     // A_KJ per group
    double2 X[kGroups][kTileT];     // X = A_IK D_K per group / per chunk (slot 0)
    double2 Xp[kGroups][kTileT];    // partial products over quarters of q
    double s_inv[kGroups];
    double2 s_row[kGroups][kB];
    int chunk[kMaxChunks];          // (I << 16) | (J0 << 4) | nj of this CTA's chunks
    int nchunk;
};

// One diagonal tile I at step K by the 64-thread group g (not the next pivot).
RECON_DEV void diag_tile_group(SweepSmem& sm, const double2* Ain, double2* Aout, const double2* DK,
                               int I, int K, int g) {
    const int e = threadIdx.x % kTileT, i = e % kB, j = e / kB;
    if (I == K) {
        const double2 d = DK[e];
        Aout[tile_off(K, K) + e] = make_double2(-d.x, -d.y);
        return;
    }
    const double2 own = Ain[tile_off(I, I) + e];
    sm.P[g][e] = block_elem(Ain, I, K, e);
    sm.B[g][e] = DK[e];
    group_sync(g);
    double2 x = make_double2(0.0, 0.0);
#pragma unroll
    for (int q = 0; q < kB; ++q) x = zfma(sm.P[g][i + kB * q], sm.B[g][q + kB * j], x);
    sm.X[g][e] = x;
    group_sync(g);
    // A_KI = (A_IK)^H:  new = own - X (A_IK)^H
    double2 v = own;
#pragma unroll
    for (int q = 0; q < kB; ++q) v = zfms(sm.X[g][i + kB * q], zconj(sm.P[g][j + kB * q]), v);
    Aout[tile_off(I, I) + e] = v;
    group_sync(g);
}

__global__ void __launch_bounds__(kThreads, 2)
hpd_sweep_kernel(double2* G, int s, const double* __restrict__ eps_p, int nt, int ndc,
                 double2* __restrict__ A0, double2* __restrict__ A1, double2* __restrict__ Dbuf,
                 GridBar* gb) {
    __shared__ SweepSmem sm;
    const int tid = threadIdx.x;
    const int g = tid / kTileT, e = tid % kTileT;
    const int i = e % kB, j = e / kB;
    const int h = g;  // quarter of the q range in the split products
    const int nlt = nt * (nt + 1) / 2;
    const double eps = eps_p[0];
    const bool diag_cta = (int)blockIdx.x < ndc;
    const int noc = (int)gridDim.x - ndc;

    // this CTA's off-diagonal chunks: row I (1..nt-1), columns J0 .. J0 + nj - 1 (J0 < I)
    if (tid == 0) {
        int n = 0;
        if (!diag_cta) {
            int ch = 0;
            for (int I = 1; I < nt; ++I)
                for (int J0 = 0; J0 < I; J0 += kChunk, ++ch)
                    if (ch % noc == (int)blockIdx.x - ndc && n < kMaxChunks)
                        sm.chunk[n++] = (I << 16) | (J0 << 4) | min(kChunk, I - J0);
        }
        sm.nchunk = n;
    }
    // A0 = pad(G + eps I), lower tiles; padding is the identity
    for (int t = blockIdx.x * kGroups + g; t < nlt; t += gridDim.x * kGroups) {
        int I, J;
        tile_ij(t, &I, &J);
        const int r = I * kB + i, c = J * kB + j;
        double2 v = make_double2(r == c ? 1.0 : 0.0, 0.0);
        if (r < s && c < s) {
            v = G[r + (size_t)c * s];
            if (r == c) v.x += eps;
        }
        A0[tile_off(I, J) + e] = v;
    }
    if (!grid_barrier(gb)) return;
    if (blockIdx.x == 0 && g == 0) {  // D_0, by the owner of tile (0, 0)
        sm.X[0][e] = A0[e];
        group_sync(0);
        tile_inverse(sm.X[0], Dbuf, &sm.s_inv[0], sm.s_row[0], 0);
    }
    if (!grid_barrier(gb)) return;

    for (int K = 0; K < nt; ++K) {
        const double2* Ain = (K & 1) ? A1 : A0;
        double2* Aout = (K & 1) ? A0 : A1;
        const double2* DK = Dbuf + (K & 1) * kTileT;
        double2* Dnext = Dbuf + ((K + 1) & 1) * kTileT;
        if (diag_cta) {
            const int c = blockIdx.x;
            const int piv = K + 1;
            const bool has_piv = piv < nt && piv % ndc == c;
            if (has_piv) {
                // next pivot tile (K+1, K+1) with all eight warps: X = A_{K+1,K} D_K (quarters
                // of q), then new = own - X (A_{K+1,K})^H, then its inverse D_{K+1}
                if (tid < kTileT) sm.D[e] = DK[e];
                else if (tid < 2 * kTileT) sm.P[0][e] = Ain[tile_off(piv, K) + e];
                const double2 own = Ain[tile_off(piv, piv) + e];
                __syncthreads();
                double2 x = make_double2(0.0, 0.0);
#pragma unroll
                for (int q = 2 * h; q < 2 * h + 2; ++q) x = zfma(sm.P[0][i + kB * q], sm.D[q + kB * j], x);
                sm.Xp[h][e] = x;
                __syncthreads();
                if (tid < kTileT)
                    sm.X[0][e] = zadd(zadd(sm.Xp[0][e], sm.Xp[1][e]), zadd(sm.Xp[2][e], sm.Xp[3][e]));
                __syncthreads();
                double2 u = make_double2(0.0, 0.0);
#pragma unroll
                for (int q = 2 * h; q < 2 * h + 2; ++q)
                    u = zfma(sm.X[0][i + kB * q], zconj(sm.P[0][j + kB * q]), u);
                sm.Xp[h][e] = u;
                __syncthreads();
                if (tid < kTileT) {
                    const double2 sum = zadd(zadd(sm.Xp[0][e], sm.Xp[1][e]), zadd(sm.Xp[2][e], sm.Xp[3][e]));
                    const double2 v = make_double2(own.x - sum.x, own.y - sum.y);
                    Aout[tile_off(piv, piv) + e] = v;
                    sm.Xp[0][e] = v;  // the same thread read slot (0, e) above
                }
                __syncthreads();
                if (g == 0) {
                    tile_inverse(sm.Xp[0], Dnext, &sm.s_inv[0], sm.s_row[0], 0);
                } else {
                    // the CTA's other diagonal tiles on groups 1..3 meanwhile
                    int m = 0;
                    for (int I = c; I < nt; I += ndc) {
                        if (I == piv) continue;
                        if (m++ % (kGroups - 1) == g - 1) diag_tile_group(sm, Ain, Aout, DK, I, K, g);
                    }
                }
            } else {
                int m = 0;
                for (int I = c; I < nt; I += ndc)
                    if (m++ % kGroups == g) diag_tile_group(sm, Ain, Aout, DK, I, K, g);
            }
        } else {
            for (int ci = 0; ci < sm.nchunk; ++ci) {
                const int code = sm.chunk[ci];
                const int I = code >> 16, J0 = (code >> 4) & 0xfff, nj = code & 15;
                const int J = J0 + g;
                const bool mine = g < nj;
                if (tid < kTileT) sm.D[e] = DK[e];
                else if (tid < 2 * kTileT && I != K) sm.P[0][e] = block_elem(Ain, I, K, e);
                double2 own = make_double2(0.0, 0.0);
                if (mine) {
                    own = Ain[tile_off(I, J) + e];
                    if (I == K) sm.B[g][e] = own;
                    else if (J != K) sm.B[g][e] = block_elem(Ain, K, J, e);
                }
                __syncthreads();
                if (I == K) {
                    // row K: new = D_K A_KJ
                    if (mine) {
                        double2 v = make_double2(0.0, 0.0);
#pragma unroll
                        for (int q = 0; q < kB; ++q) v = zfma(sm.D[i + kB * q], sm.B[g][q + kB * j], v);
                        Aout[tile_off(I, J) + e] = v;
                    }
                } else {
                    double2 x = make_double2(0.0, 0.0);
#pragma unroll
                    for (int q = 2 * h; q < 2 * h + 2; ++q) x = zfma(sm.P[0][i + kB * q], sm.D[q + kB * j], x);
                    sm.Xp[h][e] = x;
                    __syncthreads();
                    if (tid < kTileT)
                        sm.X[0][e] = zadd(zadd(sm.Xp[0][e], sm.Xp[1][e]), zadd(sm.Xp[2][e], sm.Xp[3][e]));
                    __syncthreads();
                    if (mine) {
                        double2 v;
                        if (J == K) {
                            v = sm.X[0][e];  // column K: new = A_IK D_K
                        } else {
                            v = own;
#pragma unroll
                            for (int q = 0; q < kB; ++q) v = zfms(sm.X[0][i + kB * q], sm.B[g][q + kB * j], v);
                        }
                        Aout[tile_off(I, J) + e] = v;
                    }
                }
                __syncthreads();
            }
        }
        if (!grid_barrier(gb)) return;
    }
    // H = -A (s x s, full, column-major) written over G
    const double2* Af = (nt & 1) ? A1 : A0;
    const size_t gtid = (size_t)blockIdx.x * blockDim.x + tid;
    const size_t gstride = (size_t)gridDim.x * blockDim.x;
    for (size_t idx = gtid; idx < (size_t)s * s; idx += gstride) {
        const int r = (int)(idx % s), c = (int)(idx / s);
        const int I = r / kB, J = c / kB;
        const double2 v = (I >= J) ? Af[tile_off(I, J) + r % kB + kB * (c % kB)]
                                   : zconj(Af[tile_off(J, I) + c % kB + kB * (r % kB)]);
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

int tiles_per_side(int s) { return (s + kB - 1) / kB; }

// Diagonal CTAs of the sweep: two diagonal tiles each where the grid allows.
int sweep_diag_ctas(int nt, int grid) { return max(1, min((nt + 1) / 2, grid / 8)); }

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
    const size_t nt = (size_t)tiles_per_side(d.s());
    const size_t nlt = nt * (nt + 1) / 2;
    return 256 + 2 * nlt * kTileT * sizeof(double2) + 2 * kTileT * sizeof(double2) + 1024;
}

size_t lanczos_scratch_bytes(const Dims& d, int grid_max) {
    return 256 + 2 * (size_t)d.s() * sizeof(double2) + 4 * (size_t)grid_max * sizeof(double) +
           2 * 96 * sizeof(double) + 1024;
}

cudaError_t launch_hpd_inverse(const Dims& d, double2* G, const double* eps, void* scratch,
                               int* err_flag_out, cudaStream_t st) {
    const int s = d.s(), nt = tiles_per_side(s);
    const size_t nlt = (size_t)nt * (nt + 1) / 2;
    int grid = 0;
    if (coop_grid((const void*)hpd_sweep_kernel, &grid) || grid < 2) return cudaErrorInvalidConfiguration;
    const int ndc = sweep_diag_ctas(nt, grid);
    // every off-diagonal chunk must fit the per-CTA chunk table
    long long nch = 0;
    for (int I = 1; I < nt; ++I) nch += (I + kChunk - 1) / kChunk;
    if ((nch + (grid - ndc) - 1) / (grid - ndc) > kMaxChunks) return cudaErrorInvalidValue;
    unsigned char* p = reinterpret_cast<unsigned char*>(scratch);
    GridBar* gb = reinterpret_cast<GridBar*>(p);
    p += 256;
    double2* A0 = reinterpret_cast<double2*>(p);
    p += nlt * kTileT * sizeof(double2);
    double2* A1 = reinterpret_cast<double2*>(p);
    p += nlt * kTileT * sizeof(double2);
    double2* Dbuf = reinterpret_cast<double2*>(p);
    cudaError_t e = cudaMemsetAsync(gb, 0, sizeof(GridBar), st);
    if (e != cudaSuccess) return e;
    e = launch_coop(hpd_sweep_kernel, grid, st, G, s, eps, nt, ndc, A0, A1, Dbuf, gb);
    if (e != cudaSuccess) return e;
    if (err_flag_out) {
        // fold the barrier error into the caller's flag
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
