// Device helpers shared by the recon kernels: complex arithmetic, warp reductions and the
// in-shared-memory Stockham FFT used by the row and column passes.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define RECON_DEV __device__ __forceinline__
#define RECON_HD __host__ __device__ inline

// Programmatic dependent launch: a kernel launched with programmatic stream serialization may
// start while its predecessor is finishing; it must wait before touching the predecessor's
// results (no-op when launched normally). Every such kernel calls pdl_wait() on every path, so
// completion stays transitive along the stream.
RECON_DEV void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
RECON_DEV void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Asynchronous 16-byte global -> shared copies (cp.async, cached in L2 only). Both addresses must
// be 16-byte aligned. A thread's copies are grouped by commit; wait<N> returns once at most the N
// most recent groups of this thread are still in flight (the copies always complete), after which
// a barrier makes the landed data visible to the other threads of the CTA.
RECON_DEV void cp_async16(void* smem_dst, const void* gmem_src) {
    const unsigned int d = static_cast<unsigned int>(__cvta_generic_to_shared(smem_dst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gmem_src) : "memory");
}
RECON_DEV void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
RECON_DEV void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Frame index of the banded W / the pair products, wrapped into [0, T) for the fully circulant
// (time-circular) lifting; for the valid lifting every index already lies in [0, T).
RECON_DEV int wrap_frame(int f, int T) {
    f += f < 0 ? T : 0;
    return f >= T ? f - T : f;
}

// ------------------------------------------------------------------------------------------
// complex helpers (float2 / double2 hold (re, im))
// ------------------------------------------------------------------------------------------
RECON_DEV float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
RECON_DEV float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
RECON_DEV float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
RECON_DEV float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// conj(a) * b
RECON_DEV float2 cmulcj(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.x, b.y, -a.y * b.x));
}
RECON_DEV float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
// acc += a * b
RECON_DEV float2 cfma(float2 a, float2 b, float2 acc) {
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(a.y, b.x, acc.y);
    return acc;
}
// acc += conj(a) * b
RECON_DEV float2 cfmacj(float2 a, float2 b, float2 acc) {
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(-a.y, b.x, acc.y);
    return acc;
}

// Error-free sum (Knuth's TwoSum): s + e == a + b exactly in round-to-nearest; the explicit
// rounding intrinsics keep the compiler from contracting or reassociating it.
RECON_DEV void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// Compensated accumulation: hi + lo += v, the rounding error of every addition to hi kept in lo.
RECON_DEV void comp_add(float& hi, float& lo, float v) {
    float s, e;
    two_sum(hi, v, s, e);
    hi = s;
    lo = __fadd_rn(lo, e);
}

RECON_DEV double2 zadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
RECON_DEV double2 zmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
RECON_DEV double2 zfma(double2 a, double2 b, double2 acc) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
    return acc;
}
// acc += a * conj(b)
RECON_DEV double2 zfmacj2(double2 a, double2 b, double2 acc) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(a.y, b.x, acc.y);
    acc.y = fma(-a.x, b.y, acc.y);
    return acc;
}
RECON_DEV double2 zconj(double2 a) { return make_double2(a.x, -a.y); }
// acc -= a * b with four FMAs
RECON_DEV double2 zfms(double2 a, double2 b, double2 acc) {
    acc.x = fma(-a.x, b.x, acc.x);
    acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(-a.x, b.y, acc.y);
    acc.y = fma(-a.y, b.x, acc.y);
    return acc;
}

// 1 / a in FP64 by Newton-Raphson on f(r) = 1/r - a, r <- r (2 - a r), from the FP32 reciprocal
// (24 correct bits; two steps give >= 48, within about 1 ulp of the rounded quotient). An IEEE
// FP64 division costs several hundred cycles of the narrow FP64 pipe on this part; this is four
// dependent FMAs. Falls back to the division outside the FP32 exponent range.
RECON_DEV double rcp_nr(double a) {
    const double aa = fabs(a);
    if (!(aa > 1e-30 && aa < 1e30)) return 1.0 / a;
    double r = (double)__frcp_rn((float)a);
    double e = fma(-a, r, 1.0);
    r = fma(r, e, r);
    e = fma(-a, r, 1.0);
    r = fma(r, e, r);
    return r;
}

RECON_DEV float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
RECON_DEV double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum of one double per thread (fixed tree order -> deterministic). `red` needs
// blockDim.x / 32 doubles of shared memory. Every thread gets the result.
RECON_DEV double block_sum(double v, double* red) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double t = 0.0;
    if (wid == 0) {
        t = lane < nw ? red[lane] : 0.0;
        t = warp_sum(t);
        if (lane == 0) red[0] = t;
    }
    __syncthreads();
    t = red[0];
    __syncthreads();
    return t;
}

// Deterministic sum of n doubles in global memory by the whole block (every thread gets it).
RECON_DEV double block_sum_array(const double* a, int n, double* red) {
    double v = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) v += a[i];
    return block_sum(v, red);
}

// Block sum of one float per thread: FP32 shuffle tree inside each warp, FP64 shuffle tree over
// the warps' sums in warp 0 (fixed order). Only thread 0 holds the result. Keeps the FP64 work to
// a few instructions of one warp (the FP64 pipe is ~60x narrower than FP32 on this part).
RECON_DEV double block_sum_f_t0(float v, double* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = (double)v;
    __syncthreads();
    double t = 0.0;
    if (wid == 0) {
        t = lane < nw ? red[lane] : 0.0;
        t = warp_sum(t);
    }
    return t;
}

// Grid-wide sum of one double per block, finished by the last block to arrive: every block
// stores its partial (thread 0), the block that takes the last ticket adds all partials in a
// fixed order (so the total does not depend on which block finished last), writes *out and
// re-arms the counter. `partial` is read from thread 0 only. Must be reached by all threads.
RECON_DEV void last_block_sum(double partial, double* parts, unsigned int* counter, double* out) {
    __shared__ unsigned int s_ticket;
    __shared__ double s_red[32];
    if (threadIdx.x == 0) {
        parts[blockIdx.x] = partial;
        __threadfence();
        s_ticket = atomicAdd(counter, 1u);
    }
    __syncthreads();
    if (s_ticket != gridDim.x - 1) return;
    __threadfence();
    double v = 0.0;
    for (unsigned int i = threadIdx.x; i < gridDim.x; i += blockDim.x) v += __ldcg(parts + i);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (unsigned int w = 0; w < (blockDim.x >> 5); ++w) t += s_red[w];
        *out = t;
        *counter = 0u;
        __threadfence();
    }
}

// Lane-strided sum of a[lane], a[lane + 32], ... (i < n) in that order, with the loads issued
// B at a time before their additions (the order of the additions is the plain loop's: the same
// bits). Used by the Lanczos kernel, whose grid-wide sums wait on nothing else.
template <int B = 8>
RECON_DEV double lane_sum(const double* a, int lane, int n) {
    double v = 0.0;
    int i = lane;
    for (; i + 32 * (B - 1) < n; i += 32 * B) {
        double t[B];
#pragma unroll
        for (int k = 0; k < B; ++k) t[k] = a[i + 32 * k];
#pragma unroll
        for (int k = 0; k < B; ++k) v += t[k];
    }
    double t[B];
#pragma unroll
    for (int k = 0; k < B; ++k) t[k] = i + 32 * k < n ? a[i + 32 * k] : 0.0;
#pragma unroll
    for (int k = 0; k < B; ++k)
        if (i + 32 * k < n) v += t[k];
    return v;
}

// Deterministic sum of n doubles in global memory by warp 0 alone (FP64 in 32 lanes only);
// the result is valid in every lane of warp 0. (The plain loop: in the CG passes, whose own
// loads are in flight meanwhile, lane_sum's batched loads measured slower.)
RECON_DEV double warp0_sum_array(const double* a, int n) {
    double v = 0.0;
    for (int i = threadIdx.x; i < n; i += 32) v += a[i];
    return warp_sum(v);
}

// Sum of a producer kernel's per-CTA partials (fixed order, warp 0), returned to every thread
// of the block: the consumer finishes the reduction instead of the producer's last block, which
// takes the atomic ticket and the serial tail off the critical path. Must be reached by all
// threads of the block.
RECON_DEV double sum_partials(const double* parts, int n, double* s_slot) {
    if (threadIdx.x < 32) {
        const double v = warp0_sum_array(parts, n);
        if (threadIdx.x == 0) *s_slot = v;
    }
    __syncthreads();
    return *s_slot;
}

// ------------------------------------------------------------------------------------------
// Small DFTs in registers: U[f] = sum_t u[t] e^{s 2 pi i t f / R}, s = -1 forward, +1 inverse.
// ------------------------------------------------------------------------------------------
template <bool INV>
RECON_DEV float2 mul_mi(float2 a) {  // a * (-i) forward, a * (+i) inverse
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

template <int R, bool INV>
struct SmallDFT;

template <bool INV>
struct SmallDFT<2, INV> {
    RECON_DEV static void run(float2* u) {
        float2 a = u[0], b = u[1];
        u[0] = cadd(a, b);
        u[1] = csub(a, b);
    }
};

template <bool INV>
struct SmallDFT<3, INV> {
    RECON_DEV static void run(float2* u) {
        const float c = 0.86602540378443864676f;  // sqrt(3)/2
        float2 s = cadd(u[1], u[2]);
        float2 d = csub(u[1], u[2]);
        float2 t = make_float2(u[0].x - 0.5f * s.x, u[0].y - 0.5f * s.y);
        float2 id = mul_mi<INV>(d);              // -i d forward
        u[0] = cadd(u[0], s);
        u[1] = make_float2(t.x + c * id.x, t.y + c * id.y);
        u[2] = make_float2(t.x - c * id.x, t.y - c * id.y);
    }
};

template <bool INV>
struct SmallDFT<4, INV> {
    RECON_DEV static void run(float2* u) {
        float2 a0 = cadd(u[0], u[2]), a1 = csub(u[0], u[2]);
        float2 a2 = cadd(u[1], u[3]), a3 = mul_mi<INV>(csub(u[1], u[3]));
        u[0] = cadd(a0, a2);
        u[2] = csub(a0, a2);
        u[1] = cadd(a1, a3);
        u[3] = csub(a1, a3);
    }
};

template <bool INV>
struct SmallDFT<8, INV> {
    RECON_DEV static void run(float2* u) {
        float2 e[4] = {u[0], u[2], u[4], u[6]};
        float2 o[4] = {u[1], u[3], u[5], u[7]};
        SmallDFT<4, INV>::run(e);
        SmallDFT<4, INV>::run(o);
        const float h = 0.70710678118654752440f;
        // w8^f for f = 0..3, w8 = e^{-i pi/4} forward
        float2 o1 = INV ? make_float2(h * (o[1].x - o[1].y), h * (o[1].x + o[1].y))
                        : make_float2(h * (o[1].x + o[1].y), h * (o[1].y - o[1].x));
        float2 o2 = mul_mi<INV>(o[2]);
        float2 o3 = INV ? make_float2(-h * (o[3].x + o[3].y), h * (o[3].x - o[3].y))
                        : make_float2(h * (o[3].y - o[3].x), -h * (o[3].x + o[3].y));
        u[0] = cadd(e[0], o[0]);
        u[4] = csub(e[0], o[0]);
        u[1] = cadd(e[1], o1);
        u[5] = csub(e[1], o1);
        u[2] = cadd(e[2], o2);
        u[6] = csub(e[2], o2);
        u[3] = cadd(e[3], o3);
        u[7] = csub(e[3], o3);
    }
};

// Radix schedules of the Stockham passes: the radix of the pass at span p for length n.
// Schedule 0: radix 8 whenever the remaining length allows it, then 4, 3, 2 (fewest passes).
// Schedule 1: radix 4 before 8 (more passes over shared memory, fewer registers and fewer bank
// conflicts per butterfly). Both are exact factorisations of the same DFT; results differ only
// in FP32 rounding.
__host__ __device__ constexpr int fft_radix_at(int n, int p, int sched = 0) {
    return sched == 1
               ? (((n / p) % 4 == 0) ? 4 : ((n / p) % 8 == 0) ? 8 : ((n / p) % 3 == 0) ? 3 : 2)
               : (((n / p) % 8 == 0) ? 8 : ((n / p) % 4 == 0) ? 4 : ((n / p) % 3 == 0) ? 3 : 2);
}
__host__ __device__ constexpr int fft_num_stages(int n, int p = 1, int sched = 0) {
    return p >= n ? 0 : 1 + fft_num_stages(n, p * fft_radix_at(n, p, sched), sched);
}


// One Stockham autosort pass (radix R, span p) over `nseq` independent length-N sequences.
// Element e of sequence s lives at buf[s * ss + e * es]. `tw` holds e^{-2 pi i j / N}, j < N,
// in shared memory. SEQ_FAST selects the thread mapping: sequence index fastest (column
// layouts, es > 1) or butterfly index fastest (row layouts, es == 1).
template <int N, int R, bool INV, bool SEQ_FAST>
RECON_DEV void stockham_pass(const float2* __restrict__ src, float2* __restrict__ dst, int p,
                             int nseq, int ss, int es, const float2* __restrict__ tw) {
    constexpr int NR = N / R;
    const int total = nseq * NR;
    for (int w = threadIdx.x; w < total; w += blockDim.x) {
        int s, i;
        if (SEQ_FAST) { s = w % nseq; i = w / nseq; }
        else          { s = w / NR;   i = w % NR; }
        const int k = i % p;
        const float2* in = src + s * ss;
        float2 u[R];
#pragma unroll
        for (int t = 0; t < R; ++t) u[t] = in[(i + t * NR) * es];
        if (p > 1) {
            const int step = N / (p * R);
#pragma unroll
            for (int t = 1; t < R; ++t) {
                float2 w_ = tw[t * k * step];
                if (INV) w_.y = -w_.y;
                u[t] = cmul(u[t], w_);
            }
        }
        SmallDFT<R, INV>::run(u);
        const int j = (i - k) * R + k;
        float2* out = dst + s * ss;
#pragma unroll
        for (int t = 0; t < R; ++t) out[(j + t * p) * es] = u[t];
    }
}

// Full length-N FFT of nseq sequences, ping-ponging between a and b (both in shared memory).
// Returns the buffer that holds the result. Ends with __syncthreads().
template <int N, bool INV, bool SEQ_FAST, int P = 1, int SCHED = 0>
RECON_DEV float2* fft_smem(float2* a, float2* b, int nseq, int ss, int es, const float2* tw) {
    if constexpr (P >= N) {
        return a;
    } else {
        constexpr int R = fft_radix_at(N, P, SCHED);
        stockham_pass<N, R, INV, SEQ_FAST>(a, b, P, nseq, ss, es, tw);
        __syncthreads();
        return fft_smem<N, INV, SEQ_FAST, P * R, SCHED>(b, a, nseq, ss, es, tw);
    }
}
