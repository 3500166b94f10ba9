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
// only the previous step's values and any CTA may update any tile:
//   - CTA 0 carries the serial chain alone: at step K it updates tile (K+1, K+1) and inverts it
//     (the next pivot, D_{K+1}) with no other FP64 work on its SM, one barrier ahead of the
//     others: it arrives at each barrier without waiting for its release;
//   - CTA 1, its helper, forms the chain's next input tiles (row K+2 after step K) right after
//     each release, with the workers' arithmetic, and hands them over through a flag;
//   - the other CTAs own fixed work items (chunks of up to four tiles of one tile row, which
//     form X = A_IK D_K once and apply A_IJ - X A_KJ per tile, the last chunk of a row carrying
//     its diagonal tile), dealt so that the FP64 work per SM is even.
// FP64 on this part issues one warp instruction per ~19 cycles per SM whatever the active lanes,
// and one warp at most one per ~64 cycles, so the products use full warps spread over every SM
// and the pivot chain keeps its SM to itself. Grid barriers and the helper's flag are bounded
// spin-waits: on timeout the kernel records an error flag and returns. (With n matrices in one
// launch, CTAs 0..n-1 are their pivot CTAs and CTAs n..2n-1 their helpers.)
#include <cstddef>

#include "common.cuh"
#include "kernels.h"

namespace recon {

namespace {

constexpr int kThreads = 256;
// The Lanczos kernel: four warps per CTA (so that up to four launches fit on an SM at once, as
// when several solves start together), each warp holding up to kLancRows rows of a matrix.
constexpr int kLancThreads = 128;
constexpr int kLancRows = 8;
constexpr int kB = 8;                        // tile edge
constexpr int kTileT = kB * kB;              // elements of a tile = threads of a tile group
constexpr int kGroups = kThreads / kTileT;   // tile groups per CTA
constexpr int kChunk = 4;                    // off-diagonal tiles of one row handled per CTA pass
constexpr int kMaxItems = 128;               // work items one CTA may own
constexpr long long kSpinLimit = 1LL << 24;  // polls (~1 us each at most) before giving up
// Lanczos steps (tridiagonal order) at most. lambda_max of a Gram of image series converges to
// rounding by ~16 steps (a dominant top eigenvalue); Grams of random series, whose relative top
// gap is ~0.2 %, by ~40 (plain Lanczos from the start vector below, checked in FP64 on the CPU).
constexpr int kLanczosMax = 64;

struct alignas(8) GridBar {
    unsigned int word;  // bit 31 flips when the last CTA arrives; bits 0-30 count arrivals
    int err;            // read with `word` in one 8-byte load
    unsigned int pad[2];
};
static_assert(sizeof(GridBar) <= kCoopBarrierBytes, "grid barrier exceeds its scratch header");

// The barrier word and the error word in one acquire load (GridBar: word at offset 0, err at 4).
RECON_DEV unsigned long long ld_acquire_pair(const GridBar* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
RECON_DEV unsigned int atom_add_acq_rel(unsigned int* p, unsigned int v) {
    unsigned int old;
    asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

// Barrier over gridDim.x co-resident CTAs (cooperative launch) with one atomic per CTA: CTA 0 adds
// 2^31 - (gridDim.x - 1) and every other CTA adds 1, so bit 31 of the word flips exactly when the
// last CTA arrives and the low bits return to zero. The barrier only looks at the flip, so a
// launch that completed every barrier leaves a valid starting state for the next one: the word
// is zeroed once when its scratch is allocated and again by the host after a reported failure,
// not before every launch. Thread 0 of each CTA arrives at once (no load before its atomic: the
// last arrival, which releases the others, then costs one round trip); the arrival that flips
// bit 31 goes on without reading anything, the others poll the word and the error word together
// (one acquire load per poll). Returns false (and sets gb->err) if the wait exceeded `polls`
// polls, or false when a poll finds the error word set, so that after a failure every CTA leaves
// at its next barrier that it does not complete last (a CTA that completes one goes on to the
// next, where the error stops it). Test hook: the CTA numbered `fault.withhold` (> 0) returns
// false at once without arriving, as a CTA that was lost would, so that the others' waits run
// out.
RECON_DEV bool grid_barrier(GridBar* gb, const CoopFault& fault) {
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = !(fault.withhold > 0 && (int)blockIdx.x == fault.withhold);
        if (ok) {
            __threadfence();
            const unsigned int inc = blockIdx.x == 0 ? 0x80000000u - (gridDim.x - 1u) : 1u;
            const unsigned int old = atom_add_acq_rel(&gb->word, inc);
            const bool last = (((old + inc) ^ old) & 0x80000000u) != 0u;
            const long long limit = fault.polls > 0 ? fault.polls : kSpinLimit;
            long long it = 0;
            while (!last) {
                const unsigned long long we = ld_acquire_pair(gb);
                if ((unsigned int)(we >> 32) != 0u) {  // gb->err
                    ok = 0;
                    break;
                }
                if ((((unsigned int)we ^ old) & 0x80000000u) != 0u) break;
                if (++it > limit) {
                    atomicExch(&gb->err, 1);
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

// The two halves of grid_barrier for a CTA that arrives at one barrier and waits for its release
// later or not at all (the pivot CTAs of the sweep). A CTA may arrive at the next barrier only
// after the previous one was released; every arrival then carries the previous flip, and bit 31
// flips once per barrier as in grid_barrier. barrier_arrive: thread 0, after a __syncthreads
// that follows the CTA's writes; returns the word before its add. barrier_wait: one thread;
// false when the error word is set or the wait exceeded its poll limit (which sets it).
RECON_DEV unsigned int barrier_arrive(GridBar* gb) {
    __threadfence();
    const unsigned int inc = blockIdx.x == 0 ? 0x80000000u - (gridDim.x - 1u) : 1u;
    return atom_add_acq_rel(&gb->word, inc);
}
// The arrival alone, for a CTA that never waits for this barrier: an acquire-release fence and a
// relaxed reduction (together a release of the CTA's writes ordered before it by the caller's
// __syncthreads), which does not wait for the word's old value to come back.
RECON_DEV void barrier_arrive_only(GridBar* gb) {
    const unsigned int inc = blockIdx.x == 0 ? 0x80000000u - (gridDim.x - 1u) : 1u;
    asm volatile("fence.acq_rel.gpu;\n\tred.relaxed.gpu.global.add.u32 [%0], %1;"
                 ::"l"(&gb->word), "r"(inc) : "memory");
}
RECON_DEV bool barrier_wait(GridBar* gb, unsigned int old, const CoopFault& fault) {
    const long long limit = fault.polls > 0 ? fault.polls : kSpinLimit;
    for (long long it = 0;; ++it) {
        const unsigned long long we = ld_acquire_pair(gb);
        if ((unsigned int)(we >> 32) != 0u) return false;
        if ((((unsigned int)we ^ old) & 0x80000000u) != 0u) break;
        if (it > limit) {
            atomicExch(&gb->err, 1);
            return false;
        }
    }
    __threadfence();
    return true;
}

// Wait (one thread) until *flag >= want, bounded like the barrier waits; false when the error
// word of gb is set meanwhile or the wait ran out (which sets it).
RECON_DEV bool flag_wait(const unsigned int* flag, unsigned int want, GridBar* gb,
                         const CoopFault& fault) {
    const long long limit = fault.polls > 0 ? fault.polls : kSpinLimit;
    for (long long it = 0;; ++it) {
        unsigned int v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(flag) : "memory");
        if (v >= want) return true;
        if ((it & 255) == 255) {
            const unsigned long long we = ld_acquire_pair(gb);
            if ((unsigned int)(we >> 32) != 0u) return false;
        }
        if (it > limit) {
            atomicExch(&gb->err, 1);
            return false;
        }
    }
}

// Synchronise the 64 threads of tile group g (named barrier g + 1; 0 is __syncthreads).
RECON_DEV void group_sync(int g) {
    asm volatile("bar.sync %0, %1;" ::"r"(g + 1), "r"(kTileT) : "memory");
}

// 1 / a for a pivot of a positive-definite matrix: the FP64 approximate reciprocal instruction
// as the seed, then one cubic Newton-Raphson step r (1 + e + e^2), e = 1 - a r (the error goes
// from e to e^3). Three dependent FMAs after the seed; no range test (pivots are positive,
// normal numbers). Checked against the division on the GPU: within about 1 ulp. (A seed from
// the rounded FP32 reciprocal costs two conversions on the pivot chain, 264 vs 237 us per sweep
// at s = 243, for the same results.)
RECON_DEV double rcp_pivot(double a) {
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(a));
    const double e = fma(-a, r, 1.0);
    return fma(r, fma(e, e, e), r);
}

// Inverse of a Hermitian positive-definite 8 x 8 tile (full, column-major) by 8 scalar sweeps,
// which leave -T^{-1}; the negated result goes to `out`. Run by the 64 threads of group 0, one
// element each, ping-ponging between T0 and T1 so that one barrier per pivot suffices. Each sweep
// is one rank-1 update v = t' - c_i r_j with t' = 0 on the pivot row and column, c = column k
// with c_k = -1 and r = row k / a_kk with r_k = -1 / a_kk, which gives the row (a_kj / a_kk), the
// column (a_ik / a_kk) and the pivot (-1 / a_kk) without branches. It is evaluated as
// v = t' - (c_i rr_j) / a_kk with rr = row k (rr_k = -1): the complex product c_i rr_j is formed
// while the reciprocal is being computed, so that one FMA per component follows it on the
// dependent chain. Every thread forms the reciprocal itself: a warp issues the same FP64
// instructions for one lane or for 32.
RECON_DEV void tile_inverse(double2* T0, double2* T1, double2* out, double2* out_smem = nullptr) {
    const int e = threadIdx.x % kTileT, i = e % kB, j = e / kB;
    double2* a = T0;
    double2* b = T1;
#pragma unroll 1
    for (int k = 0; k < kB; ++k) {
        const double akk = a[k + k * kB].x;
        const double2 aij = a[i + j * kB], aik = a[i + k * kB], akj = a[k + j * kB];
        const double2 t = (i == k || j == k) ? make_double2(0.0, 0.0) : aij;
        const double2 c = (i == k) ? make_double2(-1.0, 0.0) : aik;
        const double2 rr = (j == k) ? make_double2(-1.0, 0.0) : akj;
        const double2 ca = zmul(c, rr);
        const double inv = rcp_pivot(akk);
        b[i + j * kB] = make_double2(fma(-ca.x, inv, t.x), fma(-ca.y, inv, t.y));
        group_sync(0);
        double2* sw = a;
        a = b;
        b = sw;
    }
    // The Hermitian part of the result: the tile (a Schur complement updated in floating point)
    // and its computed inverse are Hermitian only up to rounding, while the sweep keeps the lower
    // tiles alone and reads an upper block as the conjugate transpose of the lower one. An inverse
    // that is not exactly Hermitian would make the two halves disagree by its anti-Hermitian part
    // times the block, an inconsistency that late pivots (inverses of nearly singular Schur
    // complements) amplify step after step; its Hermitian part keeps them consistent and is as
    // accurate.
    const double2 v = a[i + j * kB], w = a[j + i * kB];
    const double2 d = make_double2(-0.5 * (v.x + w.x), -0.5 * (v.y - w.y));
    out[i + j * kB] = d;
    if (out_smem) out_smem[i + j * kB] = d;  // the pivot CTA's own copy for its next chain
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

// One matrix of a batched sweep launch (passed by value in the kernel parameters).
struct SweepMat {
    double2* G;            // s x s column-major; H = (G + eps I)^-1 written over it
    const double* eps;     // device scalar
    double2 *A0, *A1;      // lower tiles, ping-pong
    double2* Dbuf;         // three pivot inverses (D_K in slot K mod 3)
    double2* hand;         // the helper's tiles for the chain, two slots of two tiles
    unsigned int* flag;    // the helper's step count (set to K + 1 once step K's tiles are out)
    int* err_out;          // status word (may be null)
    int s, nt;
};
struct SweepBatch {
    int n, nt_max;
    SweepMat m[kMaxHpdBatch];
};

// Status of the launch for the host, per matrix (thread 0 of CTA 0): 0 when the kernel completed,
// 1 when a barrier gave up (every CTA then fails its next barrier and returns).
RECON_DEV void report_batch(const SweepBatch& bt, int v) {
    if (blockIdx.x == 0 && threadIdx.x == 0)
        for (int b = 0; b < bt.n; ++b)
            if (bt.m[b].err_out) *bt.m[b].err_out = v;
}

// Failure status of a batched Lanczos launch (thread 0 of CTA 0, every matrix); on success each
// matrix's CTA writes 0 after its multisection.
struct LancBatch;
RECON_DEV void report_lanc(const LancBatch& bt, int v);

struct SweepSmem {
    double2 D[kTileT];            // D_K
    double2 P[kTileT];            // A_IK of the current item
    double2 B[kGroups][kTileT];   // A_KJ of each group's tile
    double2 X[kTileT];            // X = A_IK D_K
    double2 Xp[kGroups][kTileT];  // partial products over quarters of q
    double2 T1[kTileT];           // second buffer of the pivot inverse
    int item[kMaxItems];          // (I << 16) | (J0 << 4) | nj of this CTA's work items
    int nitem;
};

// A pivot CTA's inputs for its next chain: A_{K+1,K} and A_{K+1,K+1} after step K - 1, ping-pong
// over K; its last arrival and a failure flag.
struct PivotSmem {
    double2 tp[2][2][kTileT];
    double2 D[kTileT];  // D_K, as written to Dbuf
    unsigned int old;
    int fail;
};

// Work items of the non-pivot CTAs: chunks of up to four tiles (I, J0 .. J0 + nj - 1) of one tile
// row, J0 + nj <= I + 1, for every matrix b of the launch: full chunks of four off-diagonal tiles,
// then the rest of each row together with its diagonal tile (which shares the row's X = A_IK D_K),
// then the diagonal tiles of the rows that have no rest (I a multiple of four) alone. Listed
// largest first and dealt to the worker CTAs in a snake order (forward, backward, ...), which
// balances the FP64 work per SM; at s = 243 that makes 136 items for 150 workers, one pass each
// (with every diagonal tile an item of its own, 159 items left 8 CTAs two passes per step). Every
// CTA runs this enumeration and keeps its own items.
// Item code: (b << 26) | (I << 16) | (J0 << 4) | nj.
struct ItemDeal {
    int workers, me, idx, n, cap;
    int* out;
};

RECON_HD void deal_item(ItemDeal& d, int code) {
    const int rnd = d.idx / d.workers, pos = d.idx % d.workers;
    const int w = (rnd & 1) ? d.workers - 1 - pos : pos;
    if (w == d.me) {
        if (d.out && d.n < d.cap) d.out[d.n] = code;
        ++d.n;
    }
    ++d.idx;
}

RECON_HD int item_code(int b, int I, int J0, int nj) { return (b << 26) | (I << 16) | (J0 << 4) | nj; }

// Items of worker `me` (0-based among the worker CTAs) into out[0 .. cap); returns their count.
// nts[b]: tile rows of matrix b. With me < 0 it returns the largest count of any worker (host
// capacity check).
RECON_HD int sweep_items(const int* nts, int nmat, int workers, int me, int* out, int cap) {
    ItemDeal d{workers, me, 0, 0, cap, out};
    for (int b = 0; b < nmat; ++b)
        for (int I = 1; I < nts[b]; ++I)
            for (int J0 = 0; J0 + kChunk <= I; J0 += kChunk) deal_item(d, item_code(b, I, J0, kChunk));
    for (int nj = kChunk - 1; nj >= 1; --nj)
        for (int b = 0; b < nmat; ++b)
            for (int I = 1; I < nts[b]; ++I)
                if (I % kChunk == nj) deal_item(d, item_code(b, I, I - nj, nj + 1));
    for (int b = 0; b < nmat; ++b)
        for (int I = 0; I < nts[b]; I += kChunk) deal_item(d, item_code(b, I, I, 1));
    return me < 0 ? (d.idx + workers - 1) / workers : d.n;
}

// One work item at step K by the whole CTA (uniform control flow). Chunk: X = A_IK D_K is formed
// once (quarters of q on the four groups), then group g updates tile (I, J0 + g):
//   I == K:  new = D_K A_KJ;   J == K:  new = X;   otherwise  new = A_IJ - X A_KJ.
// Diagonal tile (I, I) (the last tile of its row's item): -D_K when I == K, skipped when
// I == K + 1 (the pivot CTA has it), otherwise new = A_II - X A_KI with A_KI = (A_IK)^H.
RECON_DEV void sweep_item(SweepSmem& sm, int code, int K, int nt, const double2* Ain,
                          double2* Aout, const double2* DK) {
    const int tid = threadIdx.x, g = tid / kTileT, e = tid % kTileT;
    const int i = e % kB, j = e / kB;
    const int I = (code >> 16) & 0x3ff, J0 = (code >> 4) & 0xfff, nj = code & 15;
    const bool diag = (J0 == I);  // the diagonal tile alone
    if (diag && I == K + 1) return;
    if (diag && I == K) {
        if (g == 0) {
            const double2 d = DK[e];
            Aout[tile_off(K, K) + e] = make_double2(-d.x, -d.y);
        }
        return;
    }
    const int J = J0 + g;
    const bool dtile = (J == I);  // the row's diagonal tile at the end of a chunk
    const bool mine = g < nj && !(dtile && I == K + 1);
    if (tid < kTileT) sm.D[e] = DK[e];
    else if (tid < 2 * kTileT && I != K) sm.P[e] = block_elem(Ain, I, K, e);
    double2 own = make_double2(0.0, 0.0);
    if (mine) {
        own = Ain[tile_off(I, J) + e];
        if (I == K) sm.B[g][e] = own;
        else if (J != K) sm.B[g][e] = block_elem(Ain, K, J, e);
    }
    __syncthreads();
    if (I == K) {
        if (mine) {
            double2 v = make_double2(0.0, 0.0);
            if (dtile) {
                v = make_double2(-sm.D[e].x, -sm.D[e].y);
            } else {
#pragma unroll
                for (int q = 0; q < kB; ++q) v = zfma(sm.D[i + kB * q], sm.B[g][q + kB * j], v);
            }
            Aout[tile_off(I, J) + e] = v;
        }
    } else {
        double2 x = make_double2(0.0, 0.0);
#pragma unroll
        for (int q = 2 * g; q < 2 * g + 2; ++q) x = zfma(sm.P[i + kB * q], sm.D[q + kB * j], x);
        sm.Xp[g][e] = x;
        __syncthreads();
        if (tid < kTileT) sm.X[e] = zadd(zadd(sm.Xp[0][e], sm.Xp[1][e]), zadd(sm.Xp[2][e], sm.Xp[3][e]));
        __syncthreads();
        if (mine) {
            double2 v;
            if (J == K) {
                v = sm.X[e];
            } else {
                v = own;
#pragma unroll
                for (int q = 0; q < kB; ++q) v = zfms(sm.X[i + kB * q], sm.B[g][q + kB * j], v);
            }
            Aout[tile_off(I, J) + e] = v;
        }
    }
    __syncthreads();
}

// The pivot CTA at step K, first half: the next pivot tile's Schur update with all eight warps,
// X = A_{K+1,K} D_K and S = A_{K+1,K+1} - X (A_{K+1,K})^H (quarters of q), into sm.X; the 8 x 8
// inverse of S (D_{K+1}) follows on group 0. tp = {A_{K+1,K}, A_{K+1,K+1}} after step K - 1, from
// the matrix's helper CTA (or the initial matrix at K = 0). The tile's swept value itself is never
// read again (step K+1 writes -D_{K+1} there).
RECON_DEV void sweep_pivot(SweepSmem& sm, const double2* DK, const double2 (*tp)[kTileT]) {
    const int tid = threadIdx.x, g = tid / kTileT, e = tid % kTileT;
    const int i = e % kB, j = e / kB;
    if (tid < kTileT) sm.D[e] = DK[e];
    else if (tid < 2 * kTileT) sm.P[e] = tp[0][e];
    const double2 own = tid < kTileT ? tp[1][e] : make_double2(0.0, 0.0);
    __syncthreads();
    double2 x = make_double2(0.0, 0.0);
#pragma unroll
    for (int q = 2 * g; q < 2 * g + 2; ++q) x = zfma(sm.P[i + kB * q], sm.D[q + kB * j], x);
    sm.Xp[g][e] = x;
    __syncthreads();
    if (tid < kTileT) sm.X[e] = zadd(zadd(sm.Xp[0][e], sm.Xp[1][e]), zadd(sm.Xp[2][e], sm.Xp[3][e]));
    __syncthreads();
    double2 u = make_double2(0.0, 0.0);
#pragma unroll
    for (int q = 2 * g; q < 2 * g + 2; ++q) u = zfma(sm.X[i + kB * q], zconj(sm.P[j + kB * q]), u);
    sm.Xp[g][e] = u;
    __syncthreads();
    if (tid < kTileT) {
        const double2 sum = zadd(zadd(sm.Xp[0][e], sm.Xp[1][e]), zadd(sm.Xp[2][e], sm.Xp[3][e]));
        sm.X[e] = make_double2(own.x - sum.x, own.y - sum.y);  // the same thread read X[e] above
    }
}

// The helper CTA of a matrix at step K: the tiles (K+2, K+1) and (K+2, K+2) after step K, from
// A = the matrix after step K - 1 and D_K, by the arithmetic of the workers' items (X = A_{K+2,K} D_K
// from the same four quarter partials added in the same order, then new = A_{K+2,J} - X A_{K,J}),
// so that they are bitwise the tiles the workers write; out: the two tiles, the next chain's
// inputs. Run on an SM of its own so that the chain keeps its SM's FP64 pipe.
RECON_DEV void helper_tiles(SweepSmem& sm, int K, const double2* A, const double2* DK,
                            double2* out) {
    const int tid = threadIdx.x, g = tid / kTileT, e = tid % kTileT;
    const int i = e % kB, j = e / kB;
    const int R = K + 2;
    if (g == 0) sm.D[e] = DK[e];
    else if (g == 1) sm.P[e] = A[tile_off(R, K) + e];
    double2 own = make_double2(0.0, 0.0);
    if (g < 2) {
        own = A[tile_off(R, K + 1 + g) + e];
        sm.B[g][e] = block_elem(A, K, K + 1 + g, e);
    }
    __syncthreads();
    double2 x = make_double2(0.0, 0.0);
#pragma unroll
    for (int q = 2 * g; q < 2 * g + 2; ++q) x = zfma(sm.P[i + kB * q], sm.D[q + kB * j], x);
    sm.Xp[g][e] = x;
    __syncthreads();
    if (g == 0) sm.X[e] = zadd(zadd(sm.Xp[0][e], sm.Xp[1][e]), zadd(sm.Xp[2][e], sm.Xp[3][e]));
    __syncthreads();
    if (g < 2) {
        double2 v = own;
#pragma unroll
        for (int q = 0; q < kB; ++q) v = zfms(sm.X[i + kB * q], sm.B[g][q + kB * j], v);
        out[g * kTileT + e] = v;
    }
}

// One cooperative launch sweeps every matrix of the batch: one grid barrier per pivot step serves
// all of them (the largest tile count sets the number of steps; a matrix with fewer tiles is done
// earlier and its CTAs skip its later steps). CTA b (< n) carries matrix b's pivot chain, CTA
// n + b is its helper, the other CTAs share the work items of all matrices. Every tile is computed
// by the same arithmetic as in a launch of its matrix alone, so the results do not depend on the
// batch.
__global__ void __launch_bounds__(kThreads, 2)
hpd_sweep_kernel(SweepBatch bt, GridBar* gb, CoopFault fault) {
    __shared__ SweepSmem sm;
    __shared__ PivotSmem ps;
    const int tid = threadIdx.x;
    const int g = tid / kTileT, e = tid % kTileT;
    const int i = e % kB, j = e / kB;
    const int n = bt.n;

    if (tid == 0) {
        int nts[kMaxHpdBatch];
        for (int b = 0; b < n; ++b) nts[b] = bt.m[b].nt;
        sm.nitem = (int)blockIdx.x < 2 * n
                       ? 0 : sweep_items(nts, n, gridDim.x - 2 * n, blockIdx.x - 2 * n, sm.item,
                                         kMaxItems);
        if ((int)blockIdx.x < n) *bt.m[blockIdx.x].flag = 0u;  // before the first barrier
        if (sm.nitem > kMaxItems) sm.nitem = kMaxItems;  // the host refuses such sizes
    }
    // A0 = pad(G + eps I), lower tiles; padding is the identity. Only the lower triangle of G is
    // read (the upper half of a diagonal tile is taken as the conjugate of the lower, the
    // diagonal as real), as the FP64 eigensolver reads it: the sweep assumes an exactly Hermitian
    // matrix, and a G whose halves differ by rounding would make its pivots' inverses disagree
    // with the mirrored off-diagonal tiles by far more than rounding at large condition numbers.
    for (int b = 0; b < n; ++b) {
        const SweepMat& mt = bt.m[b];
        const int nlt = mt.nt * (mt.nt + 1) / 2, s = mt.s;
        const double eps = mt.eps[0];
        for (int t = blockIdx.x * kGroups + g; t < nlt; t += gridDim.x * kGroups) {
            int I, J;
            tile_ij(t, &I, &J);
            const int r = I * kB + i, c = J * kB + j;
            double2 v = make_double2(r == c ? 1.0 : 0.0, 0.0);
            if (r < s && c < s) {
                v = r >= c ? mt.G[r + (size_t)c * s] : zconj(mt.G[c + (size_t)r * s]);
                if (r == c) v = make_double2(v.x + eps, 0.0);
            }
            mt.A0[tile_off(I, J) + e] = v;
        }
    }
    if (!grid_barrier(gb, fault)) return report_batch(bt, 1);
    if ((int)blockIdx.x < n && g == 0) {  // D_0 of matrix blockIdx.x
        const SweepMat& mt = bt.m[blockIdx.x];
        sm.X[e] = mt.A0[e];
        group_sync(0);
        tile_inverse(sm.X, sm.T1, mt.Dbuf, ps.D);
    }
    if (!grid_barrier(gb, fault)) return report_batch(bt, 1);

    if ((int)blockIdx.x < n) {
        // Pivot CTA of matrix blockIdx.x, one barrier ahead of the workers. Step K: the chain (the
        // Schur update of tile (K+1, K+1) on all warps, then its inverse D_{K+1} on group 0) needs
        // D_K and the row-(K+1) tiles after step K - 1, which the matrix's helper CTA formed
        // during step K - 1; meanwhile group 1 waits for the helper's step-K tiles (the helper
        // forms them once it has seen the release of the barrier that ended step K - 1, so they
        // also tell that this CTA may arrive at the next barrier). Then the CTA arrives at the
        // barrier that ends step K without waiting for its release: the release latency leaves
        // the chain's path. D_K lives in slot K mod 3 of Dbuf (the chain writes D_{K+2} while slow
        // workers may still read D_K).
        const SweepMat& mt = bt.m[blockIdx.x];
        if (mt.nt > 1 && tid < 2 * kTileT) ps.tp[0][tid / kTileT][e] = mt.A0[tile_off(1, tid / kTileT) + e];
        if (tid == 0) ps.fail = 0;
        __syncthreads();
        for (int K = 0; K < bt.nt_max; ++K) {
            const bool chain = K + 1 < mt.nt;
            if (chain) sweep_pivot(sm, ps.D, ps.tp[K & 1]);
            if (g == 0) {
                if (chain) {
                    group_sync(0);
                    tile_inverse(sm.X, sm.T1, mt.Dbuf + ((K + 1) % 3) * kTileT, ps.D);
                }
            } else if (g == 1) {
                if (e == 0 && !flag_wait(mt.flag, (unsigned int)(K + 1), gb, fault)) ps.fail = 1;
                group_sync(1);
                if (!ps.fail && K + 2 < mt.nt) {
                    const double2* h = mt.hand + ((K + 1) & 1) * 2 * kTileT;
                    ps.tp[(K + 1) & 1][0][e] = h[e];
                    ps.tp[(K + 1) & 1][1][e] = h[kTileT + e];
                }
            }
            __syncthreads();
            if (ps.fail) return report_batch(bt, 1);
            // only the last arrival's old value is needed (its release is waited for below)
            if (tid == 0) {
                if (K + 1 < bt.nt_max) barrier_arrive_only(gb);
                else ps.old = barrier_arrive(gb);
            }
            __syncthreads();
        }
        if (tid == 0 && !barrier_wait(gb, ps.old, fault)) ps.fail = 1;
        __syncthreads();
        if (ps.fail) return report_batch(bt, 1);
    } else if ((int)blockIdx.x < 2 * n) {
        // Helper CTA of matrix blockIdx.x - n: after the release of the barrier that ended step
        // K - 1, the row-(K+2) tiles after step K for the pivot CTA's next chain, then its flag.
        const SweepMat& mt = bt.m[blockIdx.x - n];
        for (int K = 0; K < bt.nt_max; ++K) {
            if (K + 2 < mt.nt)
                helper_tiles(sm, K, (K & 1) ? mt.A1 : mt.A0, mt.Dbuf + (K % 3) * kTileT,
                             mt.hand + ((K + 1) & 1) * 2 * kTileT);
            __syncthreads();
            if (tid == 0) {
                __threadfence();
                asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(mt.flag),
                             "r"((unsigned int)(K + 1)) : "memory");
            }
            if (!grid_barrier(gb, fault)) return report_batch(bt, 1);
        }
    } else {
        for (int K = 0; K < bt.nt_max; ++K) {
            for (int it = 0; it < sm.nitem; ++it) {
                const int code = sm.item[it];
                const SweepMat& mt = bt.m[code >> 26];
                if (K < mt.nt)
                    sweep_item(sm, code, K, mt.nt, (K & 1) ? mt.A1 : mt.A0, (K & 1) ? mt.A0 : mt.A1,
                               mt.Dbuf + (K % 3) * kTileT);
            }
            if (!grid_barrier(gb, fault)) return report_batch(bt, 1);
        }
    }
    // H = -A (s x s, full, column-major) written over G
    const size_t gtid = (size_t)blockIdx.x * blockDim.x + tid;
    const size_t gstride = (size_t)gridDim.x * blockDim.x;
    for (int b = 0; b < n; ++b) {
        const SweepMat& mt = bt.m[b];
        const int s = mt.s;
        const double2* Af = (mt.nt & 1) ? mt.A1 : mt.A0;
        for (size_t idx = gtid; idx < (size_t)s * s; idx += gstride) {
            // from the lower triangle (within a diagonal tile too): H exactly Hermitian
            const int r = (int)(idx % s), c = (int)(idx / s);
            const double2 v = (r >= c) ? Af[tile_off(r / kB, c / kB) + r % kB + kB * (c % kB)]
                                       : zconj(Af[tile_off(c / kB, r / kB) + c % kB + kB * (r % kB)]);
            mt.G[idx] = make_double2(-v.x, r == c ? 0.0 : -v.y);
        }
    }
    report_batch(bt, 0);
}

// d_ab[delta] = sum_{l - l' = delta} H[(l', b), (l, a)] from H (s x s column-major); taps
// l = (l3, l1, l2) at column index ((m N3 + l3) N1 + l1) N2 + l2, output [pair][d3][d1][d2].
__global__ void hdiag_kernel(const double2* __restrict__ H, int N1, int N2, int N3, int M,
                             double2* __restrict__ dsum) {
    const int L1 = 2 * N1 - 1, L2 = 2 * N2 - 1, L3 = 2 * N3 - 1;
    const int npair = M * (M + 1) / 2;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= npair * L3 * L1 * L2) return;
    const int pr = warp / (L3 * L1 * L2), rem = warp % (L3 * L1 * L2);
    const int d3 = rem / (L1 * L2) - (N3 - 1);
    const int d1 = (rem / L2) % L1 - (N1 - 1), d2 = rem % L2 - (N2 - 1);
    int a = 0, e = pr;
    while (e >= M - a) { e -= M - a; ++a; }
    const int b = a + e;
    const int s = N1 * N2 * N3 * M;
    const int lo1 = max(0, -d1), hi1 = min(N1, N1 - d1);
    const int lo2 = max(0, -d2), hi2 = min(N2, N2 - d2);
    const int lo3 = max(0, -d3), hi3 = min(N3, N3 - d3);
    const int n1 = hi1 - lo1, n2 = hi2 - lo2;
    const int cnt = (hi3 - lo3) * n1 * n2;
    double2 acc = make_double2(0.0, 0.0);
    for (int t = lane; t < cnt; t += 32) {
        const int lp2 = lo2 + t % n2, lp1 = lo1 + (t / n2) % n1, lp3 = lo3 + t / (n2 * n1);
        const size_t rowi = (((size_t)b * N3 + lp3) * N1 + lp1) * N2 + lp2;
        const size_t coli = (((size_t)a * N3 + lp3 + d3) * N1 + lp1 + d1) * N2 + lp2 + d2;
        acc = zadd(acc, H[rowi + coli * s]);
    }
    acc.x = warp_sum(acc.x);
    acc.y = warp_sum(acc.y);
    if (lane == 0) dsum[warp] = acc;
}

// ---- Lanczos estimate of lambda_max(G), FP64, m steps, then multisection on the tridiagonal.
// One matrix of a batched Lanczos launch (by value in the kernel parameters).
struct LancMat {
    const double2* G;      // s x s column-major, Hermitian
    double2 *u, *vprev;    // Lanczos vectors (s each)
    double* part;          // 4 x grid partial sums (alpha, beta; ping-pong)
    double* ab;            // alpha_k, beta_k
    double* lmax_out;      // device scalar
    int* err_out;          // status word (may be null)
    int s, m;              // order, steps (<= kLanczosMax)
};
struct LancBatch {
    int n, m_max;
    LancMat mt[kMaxHpdBatch];
};

RECON_DEV void report_lanc(const LancBatch& bt, int v) {
    if (blockIdx.x == 0 && threadIdx.x == 0)
        for (int b = 0; b < bt.n; ++b)
            if (bt.mt[b].err_out) *bt.mt[b].err_out = v;
}

// Several matrices per launch, two grid barriers per step for all of them. Row i of matrix b goes
// to global warp i mod (warps of the grid), as in a launch of that matrix alone, and every sum is
// taken in the same order, so each matrix's lambda_max is bitwise the one its own launch gives.
__global__ void __launch_bounds__(kLancThreads, 4)
lanczos_kernel(LancBatch bt, GridBar* gb, CoopFault fault) {
    __shared__ double red[kMaxHpdBatch][kLancThreads / 32];
    __shared__ double2 ys[kMaxHpdBatch][kLancRows][kLancThreads / 32];  // G v of the warp's rows (lane 0)
    __shared__ double s_beta[kMaxHpdBatch], s_ib[kMaxHpdBatch], s_alpha[kMaxHpdBatch];
    __shared__ int s_m[kMaxHpdBatch];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nw = gridDim.x * (kLancThreads / 32);
    const int gw = warp * gridDim.x + blockIdx.x;  // rows spread over every SM (FP64 unit per SM)
    const int n = bt.n;
    // deterministic start vector, unnormalised: u_i = 1 + 0.5 sin(i) + i 0.25 i cos(3 i) / s
    for (int b = 0; b < n; ++b) {
        const LancMat& L = bt.mt[b];
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < L.s; i += gridDim.x * blockDim.x) {
            L.u[i] = make_double2(1.0 + 0.5 * sin((double)i), 0.25 * cos(3.0 * i) * i / L.s);
            L.vprev[i] = make_double2(0.0, 0.0);
        }
    }
    if (!grid_barrier(gb, fault)) return report_lanc(bt, 1);
    for (int b = warp; b < n; b += kLancThreads / 32) {
        const LancMat& L = bt.mt[b];
        double acc = 0.0;
        for (int i = lane; i < L.s; i += 32) acc += L.u[i].x * L.u[i].x + L.u[i].y * L.u[i].y;
        acc = warp_sum(acc);
        if (lane == 0) {
            s_beta[b] = sqrt(acc);
            s_ib[b] = rcp_nr(s_beta[b]);
            s_m[b] = L.m;
        }
    }
    __syncthreads();
    for (int k = 0; k < bt.m_max; ++k) {
        // v_k = u / beta_{k-1};  w = G v_k - alpha_k v_k - beta_{k-1} v_{k-1};  beta_k = |w|
        bool any = false;
        for (int b = 0; b < n; ++b) {
            const LancMat& L = bt.mt[b];
            const bool act = k < s_m[b];
            any = any || act;
            double ap = 0.0;
            if (act) {
                const double ib = s_ib[b];
                int nrow = 0;
                for (int i = gw; i < L.s && nrow < kLancRows; i += nw, ++nrow) {
                    // row i of the Hermitian G is the conjugate of column i (contiguous)
                    double2 acc = make_double2(0.0, 0.0);
                    const double2* gcol = L.G + (size_t)i * L.s;
                    int j = lane;
                    for (; j + 32 * 3 < L.s; j += 32 * 4) {  // four loads of each in flight
                        double2 g[4], uj[4];
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            g[q] = gcol[j + 32 * q];
                            uj[q] = L.u[j + 32 * q];
                        }
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            acc.x = fma(g[q].x, uj[q].x, acc.x);
                            acc.x = fma(g[q].y, uj[q].y, acc.x);
                            acc.y = fma(g[q].x, uj[q].y, acc.y);
                            acc.y = fma(-g[q].y, uj[q].x, acc.y);
                        }
                    }
                    for (; j < L.s; j += 32) {
                        const double2 g = gcol[j], uj = L.u[j];
                        acc.x = fma(g.x, uj.x, acc.x);
                        acc.x = fma(g.y, uj.y, acc.x);
                        acc.y = fma(g.x, uj.y, acc.y);
                        acc.y = fma(-g.y, uj.x, acc.y);
                    }
                    acc.x = warp_sum(acc.x) * ib;
                    acc.y = warp_sum(acc.y) * ib;
                    if (lane == 0) ys[b][nrow][warp] = acc;
                    const double2 vi = make_double2(L.u[i].x * ib, L.u[i].y * ib);
                    ap += vi.x * acc.x + vi.y * acc.y;
                }
            }
            if (lane == 0) red[b][warp] = ap;
        }
        if (!any) break;
        __syncthreads();
        if ((int)threadIdx.x < n && k < s_m[threadIdx.x]) {
            const int b = threadIdx.x;
            double t = 0.0;
            for (int w = 0; w < kLancThreads / 32; ++w) t += red[b][w];
            bt.mt[b].part[(size_t)(k & 1) * 2 * gridDim.x + blockIdx.x] = t;
        }
        if (!grid_barrier(gb, fault)) return report_lanc(bt, 1);
        for (int b = warp; b < n; b += kLancThreads / 32) {
            if (k >= s_m[b]) continue;
            const double* pa = bt.mt[b].part + (size_t)(k & 1) * 2 * gridDim.x;
            const double v = warp_sum(lane_sum(pa, lane, (int)gridDim.x));
            if (lane == 0) s_alpha[b] = v;
        }
        __syncthreads();
        for (int b = 0; b < n; ++b) {
            const LancMat& L = bt.mt[b];
            double bp = 0.0;
            if (k < s_m[b] && lane == 0) {
                const double alpha = s_alpha[b], beta = s_beta[b], ib = s_ib[b];
                int nrow = 0;
                for (int i = gw; i < L.s && nrow < kLancRows; i += nw, ++nrow) {
                    const double2 vi = make_double2(L.u[i].x * ib, L.u[i].y * ib);
                    const double2 vp = L.vprev[i], yi = ys[b][nrow][warp];
                    const double2 un = make_double2(yi.x - alpha * vi.x - beta * vp.x,
                                                    yi.y - alpha * vi.y - beta * vp.y);
                    bp += un.x * un.x + un.y * un.y;
                    L.vprev[i] = vi;
                    L.u[i] = un;
                }
            }
            if (lane == 0) red[b][warp] = bp;
        }
        __syncthreads();
        if ((int)threadIdx.x < n && k < s_m[threadIdx.x]) {
            const int b = threadIdx.x;
            double t = 0.0;
            for (int w = 0; w < kLancThreads / 32; ++w) t += red[b][w];
            bt.mt[b].part[(size_t)(k & 1) * 2 * gridDim.x + gridDim.x + blockIdx.x] = t;
        }
        if (!grid_barrier(gb, fault)) return report_lanc(bt, 1);
        for (int b = warp; b < n; b += kLancThreads / 32) {
            if (k >= s_m[b]) continue;
            const double* pb = bt.mt[b].part + (size_t)(k & 1) * 2 * gridDim.x + gridDim.x;
            const double b2 = warp_sum(lane_sum(pb, lane, (int)gridDim.x));
            if (lane == 0) {
                const double bnew = sqrt(b2);
                if ((int)blockIdx.x == b) {  // the CTA that reads them for the multisection
                    bt.mt[b].ab[2 * k] = s_alpha[b];
                    bt.mt[b].ab[2 * k + 1] = bnew;
                }
                const double al = s_alpha[b];
                s_beta[b] = bnew;
                s_ib[b] = rcp_nr(bnew);
                if (!(bnew > 1e-300 * fabs(al) + 1e-300)) s_m[b] = k + 1;
            }
        }
        __syncthreads();
    }
    // matrix b's tridiagonal on CTA b
    if ((int)blockIdx.x >= n) return;
    const LancMat& L = bt.mt[blockIdx.x];
    const double* ab = L.ab;
    const int m = s_m[blockIdx.x];
    __shared__ double sh_lo, sh_hi;
    // Largest eigenvalue of the m x m tridiagonal (alpha_k, beta_k) by multisection with Sturm
    // counts (one CTA per matrix): FP32 rounds over the whole block to 1e-4 relative (FP32 counts are exact
    // for x farther than ~m eps32 |T| from an eigenvalue), then FP64 rounds on three warps. The
    // FP64 count follows the characteristic polynomials p_k = (alpha_k - x) p_{k-1} -
    // beta_{k-1}^2 p_{k-2} (the number of sign changes of p_0 .. p_m is the number of eigenvalues
    // below x), rescaled by exact powers of two when the exponent drifts: two dependent FP64
    // operations per step instead of a reciprocal.
    __shared__ int best;
    __shared__ float sa32[kLanczosMax], sb32[kLanczosMax];
    __shared__ double sa64[kLanczosMax], sb64[kLanczosMax];
    for (int k = threadIdx.x; k < m; k += blockDim.x) {
        const double a = ab[2 * k], b2 = k > 0 ? ab[2 * k - 1] * ab[2 * k - 1] : 0.0;
        sa64[k] = a;
        sb64[k] = b2;
        sa32[k] = (float)a;
        sb32[k] = (float)b2;
    }
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
        const int nthr = fp32 ? (int)blockDim.x : 96;
        const double lo = sh_lo, hi = sh_hi;
        int cnt = m;
        if ((int)threadIdx.x < nthr) {
            const double x = lo + (hi - lo) * (threadIdx.x + 1) / (double)(nthr + 1);
            cnt = 0;
            if (fp32) {
                const float xf = (float)x;
                float d = 1.f;
                for (int k = 0; k < m; ++k) {
                    d = (sa32[k] - xf) - (k > 0 ? sb32[k] * __frcp_rn(d) : 0.f);
                    if (d == 0.f) d = -1e-30f;
                    if (d < 0.f) ++cnt;
                }
            } else {
                double p0 = 1.0, p1 = sa64[0] - x;
                if (p1 == 0.0) p1 = -1e-300;
                cnt = p1 < 0.0;
                for (int k = 1; k < m; ++k) {
                    double p2 = fma(-sb64[k], p0, (sa64[k] - x) * p1);
                    if (p2 == 0.0) p2 = p1 < 0.0 ? 1e-300 : -1e-300;  // a zero counts as a change
                    cnt += (p2 < 0.0) != (p1 < 0.0);
                    p0 = p1;
                    p1 = p2;
                    const int ex = max((int)((__double_as_longlong(p0) >> 52) & 0x7ff),
                                       (int)((__double_as_longlong(p1) >> 52) & 0x7ff));
                    if (ex > 1023 + 480 || ex < 1023 - 480) {  // keep the larger one near 1
                        const double sc = __longlong_as_double((long long)(2046 - ex) << 52);
                        p0 *= sc;
                        p1 *= sc;
                    }
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
    if (threadIdx.x == 0) {
        L.lmax_out[0] = 0.5 * (sh_lo + sh_hi);
        if (L.err_out) *L.err_out = 0;
    }
}


int coop_grid(const void* kern, int threads, int* grid) {
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, threads, 0) != cudaSuccess) return -1;
    if (per < 1) return -1;
    *grid = sms;  // one CTA per SM
    return 0;
}

int tiles_per_side(int s) { return (s + kB - 1) / kB; }

// Cooperative launch (all CTAs co-resident, required by the grid barriers) through
// cudaLaunchKernelEx so that it can be captured into a CUDA graph.
template <typename... KArgs, typename... Args>
cudaError_t launch_coop(void (*kern)(KArgs...), int grid, int threads, cudaStream_t st,
                        Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(threads);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

}  // namespace

cudaError_t set_barrier_error(void* scratch, cudaStream_t st) {
    return cudaMemsetAsync(reinterpret_cast<unsigned char*>(scratch) + offsetof(GridBar, err), 1,
                           sizeof(int), st);
}

size_t hpd_scratch_bytes(const Dims& d) {
    const size_t nt = (size_t)tiles_per_side(d.s());
    const size_t nlt = nt * (nt + 1) / 2;
    return kCoopBarrierBytes + 2 * nlt * kTileT * sizeof(double2) + 7 * kTileT * sizeof(double2) + 1024;
}

size_t lanczos_scratch_bytes(const Dims& d, int grid_max) {
    return kCoopBarrierBytes + 2 * (size_t)d.s() * sizeof(double2) + 4 * (size_t)grid_max * sizeof(double) +
           2 * kLanczosMax * sizeof(double) + 1024;
}

cudaError_t launch_hpd_inverse_batch(const HpdJob* jobs, int n, void* barrier_scratch,
                                     cudaStream_t st, CoopFault fault) {
    if (n < 1 || n > kMaxHpdBatch || !barrier_scratch) return cudaErrorInvalidValue;
    int grid = 0;
    if (coop_grid((const void*)hpd_sweep_kernel, kThreads, &grid) || grid < 2 * n + 1)
        return cudaErrorInvalidConfiguration;
    SweepBatch bt = {};
    bt.n = n;
    int nts[kMaxHpdBatch];
    for (int b = 0; b < n; ++b) {
        const int s = jobs[b].s, nt = tiles_per_side(s);
        if (s < 1 || nt >= 1024 || !jobs[b].G || !jobs[b].eps || !jobs[b].scratch)
            return cudaErrorInvalidValue;
        const size_t nlt = (size_t)nt * (nt + 1) / 2;
        unsigned char* p = reinterpret_cast<unsigned char*>(jobs[b].scratch) + kCoopBarrierBytes;
        SweepMat& mt = bt.m[b];
        mt.G = jobs[b].G;
        mt.eps = jobs[b].eps;
        mt.A0 = reinterpret_cast<double2*>(p);
        p += nlt * kTileT * sizeof(double2);
        mt.A1 = reinterpret_cast<double2*>(p);
        p += nlt * kTileT * sizeof(double2);
        mt.Dbuf = reinterpret_cast<double2*>(p);
        p += 3 * kTileT * sizeof(double2);
        mt.hand = reinterpret_cast<double2*>(p);
        p += 4 * kTileT * sizeof(double2);
        mt.flag = reinterpret_cast<unsigned int*>(p);
        mt.err_out = jobs[b].err_out;
        mt.s = s;
        mt.nt = nt;
        nts[b] = nt;
        if (nt > bt.nt_max) bt.nt_max = nt;
    }
    // every work item must fit the per-CTA item table
    if (sweep_items(nts, n, grid - 2 * n, -1, nullptr, 0) > kMaxItems) return cudaErrorInvalidValue;
    GridBar* gb = reinterpret_cast<GridBar*>(barrier_scratch);
    return launch_coop(hpd_sweep_kernel, grid, kThreads, st, bt, gb, fault);
}

cudaError_t launch_hpd_inverse(const Dims& d, double2* G, const double* eps, void* scratch,
                               int* err_flag_out, cudaStream_t st, CoopFault fault) {
    const HpdJob job{G, eps, scratch, err_flag_out, d.s()};
    return launch_hpd_inverse_batch(&job, 1, scratch, st, fault);
}

cudaError_t launch_hdiag(const Dims& d, const double2* H, double2* dsum, cudaStream_t st) {
    const int nout = (int)d.nlag();
    const int warps_per_block = 8;
    hdiag_kernel<<<(nout + warps_per_block - 1) / warps_per_block, 32 * warps_per_block, 0, st>>>(
        H, d.N1, d.N2, d.N3, d.M, dsum);
    return cudaGetLastError();
}

cudaError_t launch_lanczos_batch(const LanczosJob* jobs, int n, void* barrier_scratch,
                                 cudaStream_t st, CoopFault fault) {
    if (n < 1 || n > kMaxHpdBatch || !barrier_scratch) return cudaErrorInvalidValue;
    int grid = 0;
    if (coop_grid((const void*)lanczos_kernel, kLancThreads, &grid) || grid < n)
        return cudaErrorInvalidConfiguration;
    const int nw = grid * (kLancThreads / 32);
    LancBatch bt = {};
    bt.n = n;
    for (int b = 0; b < n; ++b) {
        const int s = jobs[b].s;
        // each warp holds at most kLancRows rows of a matrix
        if (s < 1 || s > kLancRows * nw || !jobs[b].G || !jobs[b].scratch || !jobs[b].lmax)
            return cudaErrorInvalidValue;
        unsigned char* p = reinterpret_cast<unsigned char*>(jobs[b].scratch) + kCoopBarrierBytes;
        LancMat& L = bt.mt[b];
        L.G = jobs[b].G;
        L.u = reinterpret_cast<double2*>(p);
        p += (size_t)s * sizeof(double2);
        L.vprev = reinterpret_cast<double2*>(p);
        p += (size_t)s * sizeof(double2);
        L.part = reinterpret_cast<double*>(p);
        p += 4 * (size_t)grid * sizeof(double);
        L.ab = reinterpret_cast<double*>(p);
        L.lmax_out = jobs[b].lmax;
        L.err_out = jobs[b].err_out;
        L.s = s;
        L.m = s < kLanczosMax ? s : kLanczosMax;
        if (L.m > bt.m_max) bt.m_max = L.m;
    }
    GridBar* gb = reinterpret_cast<GridBar*>(barrier_scratch);
    return launch_coop(lanczos_kernel, grid, kLancThreads, st, bt, gb, fault);
}

cudaError_t launch_lanczos_lmax(const Dims& d, const double2* G, void* scratch, double* lmax,
                                int* err_flag_out, cudaStream_t st, CoopFault fault) {
    const LanczosJob job{G, scratch, lmax, err_flag_out, d.s()};
    return launch_lanczos_batch(&job, 1, scratch, st, fault);
}

}  // namespace recon
