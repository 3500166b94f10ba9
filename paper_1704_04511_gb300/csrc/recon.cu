// C ABI (include/recon.h): context, workspace, argument checks and the IRLS orchestration of
// Algorithm 1 (Sec. III) over the kernels of fft.cu, gram.cu, weight.cu and cg.cu.
//
// Per IRLS iteration n (all on the context's stream, no host synchronisation):
//   Gram of x^(n-1) -> G (FP64)                                  [gram.cu]
//   G = U diag(lambda) U^H, FP64 (cuSOLVER zheevd)                [library call]
//   eps: n = 1 -> eps0_frac * lambda_max, else eps / gamma        [Sec. III-C]
//   summed diagonals of H, per-pixel S(r)                         [weight.cu]
//   residual carry, then `cg` CG steps (4 passes each)            [cg.cu, fft.cu]
// The CG warm-start residual is carried from the previous iteration's CG,
//   r0^(1) = -lam W^(1) x0   (A^H A A^H b = A^H b for 0/1 masks),
//   r0^(n+1) = r_end^(n) + lam (W^(n) - W^(n+1)) x^(n),
// which equals A^H b - (A^H A + lam W^(n+1)) x^(n) in exact arithmetic but avoids forming it by
// cancellation in FP32 (the two terms agree to ~1e-5 relative near convergence).
#include <cuda_runtime.h>
#include <cublas_v2.h>
#include <cusolverDn.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <cstdint>
#include <fstream>
#include <initializer_list>
#include <map>
#include <sstream>
#include <tuple>
#include <string>
#include <vector>

#include "../../include/recon.h"
#include "kernels.h"

using recon::Dims;
using recon::Twiddles;

namespace {

struct Buf {
    void* ptr = nullptr;
    size_t bytes = 0;
};

struct TwTable {
    float2* f = nullptr;
    double2* d = nullptr;
};

// Timing events captured into a solve's CUDA graph (event-record nodes): the launch class and
// the event pair of every timed launch, and how many replays have run / been read.
struct GraphProf {
    std::vector<std::tuple<int, cudaEvent_t, cudaEvent_t>> ev;
    unsigned long replays = 0, collected = 0;
    ~GraphProf() {
        for (auto& t : ev) {
            cudaEventDestroy(std::get<1>(t));
            cudaEventDestroy(std::get<2>(t));
        }
    }
};

thread_local std::string g_create_error;

}  // namespace

namespace recon {
void set_context_free_error(const std::string& msg) { g_create_error = msg; }
}  // namespace recon

struct recon_ctx {
    int device = 0;
    size_t budget = 0;
    size_t allocated = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cusolverDnHandle_t solver = nullptr;
    cublasHandle_t blas = nullptr;  // library GEMMs of the IRLS-direct variant (slot 0 stream)
    std::string err;
    std::map<int, TwTable> tw;
    std::map<std::string, Buf> bufs;
    // Batch slots: each has its own stream, workspace and eigensolver handle. The fields
    // stream / bufs / solver above always hold the ACTIVE slot's; the others are parked here.
    unsigned long ws_gen = 0;          // bumped when the active slot's workspace moves
    struct GraphKey {
        int T, P, Q, N1, N2, M, irls, cg, bf16, method, R, N3;
        double lambda, p, gamma, eps0_frac;
        const void *kspace, *masks, *out, *coils;
        int nc, coil_proj, circ, variant, colC, depthC, colS, depthS;
        unsigned int prof;
        unsigned long ws_gen;
    };
    GraphKey gkey = {};
    cudaGraphExec_t gexec = nullptr;   // the active slot's captured solve
    GraphProf* gprof = nullptr;        // its timing events (launch classes timed when captured)
    GraphProf* capturing = nullptr;    // set while a solve with timed classes is being captured
    bool graphs = true;
    // autotuner: column tile widths per problem shape (P, Q, T, R, coils), timed on first use
    bool autotune = true;
    bool inject_barrier_fault = false; // next solve: sweep barrier starts failed (RECON_OPT_INJECT_BARRIER_FAULT)
    bool withhold_arrival = false;     // next solve: one CTA withholds its barrier arrival (RECON_OPT_TEST_WITHHOLD_ARRIVAL)
    // lockstep batches (RECON_OPT_BATCH_GROUP): one graph over every slot of recon_solve_batch
    int batch_group = 0;               // solves per shared weight launch; 0 = independent slots
    cudaGraphExec_t batch_gexec = nullptr;
    GraphProf* batch_gprof = nullptr;
    std::vector<unsigned char> batch_key;
    std::vector<cudaEvent_t> batch_ev;  // fork / join events of the capture
    bool autotune_fft = false;         // the autotuner also picks the radix schedule (RECON_OPT_AUTOTUNE_FFT)
    int fft_sched = -1;                // forced radix schedule of the column passes (-1 = tuned / 0)
    struct TileChoice {
        int colC = 0, depthC = 0, colS = 0, depthS = 0;
    };
    std::map<std::tuple<int, int, int, int, int>, TileChoice> tiles;
    std::string tile_cache;            // file the tuned choices are appended to (may be empty)
    struct Slot {
        cudaStream_t stream = nullptr;
        bool own_stream = false;
        std::map<std::string, Buf> bufs;
        cusolverDnHandle_t solver = nullptr;
        unsigned long ws_gen = 0;
        GraphKey gkey = {};
        cudaGraphExec_t gexec = nullptr;
        GraphProf* gprof = nullptr;
    };
    std::vector<Slot> slots;  // slots[i] valid while i != active
    int active = 0;
    // asynchronous requests (recon_submit / recon_poll) use slots 1..RECON_MAX_BATCH
    struct Pending;
    std::vector<Pending*> pending;
    // optional per-launch CUDA-event timing (recon_profile): bit k times launch class k
    unsigned int prof = 0;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    std::vector<std::pair<int, size_t>> prof_pending;  // (kind, index of start event)
    double prof_ms[RECON_PROF_KINDS] = {0};
    long long prof_n[RECON_PROF_KINDS] = {0};
};

namespace {

int fail(recon_ctx* c, int code, const std::string& msg) {
    if (c) c->err = msg;
    return code;
}

// Device arrays handed to the library start on a 16-byte boundary: the vector passes move two
// complex64 values per access and the row passes stage rows with 16-byte asynchronous copies.
constexpr const char* kAlignMsg = "device arrays must be 16-byte aligned";
bool misaligned(std::initializer_list<const void*> ptrs) {
    for (const void* p : ptrs)
        if (reinterpret_cast<uintptr_t>(p) & 15u) return true;
    return false;
}

int cuda_fail(recon_ctx* c, cudaError_t e, const char* where) {
    return fail(c, RECON_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define RC_CUDA(call)                                                \
    do {                                                             \
        cudaError_t e_ = (call);                                     \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, #call);       \
    } while (0)

// Bracket one launch of `kind` with two events when profiling is on. While a solve is being
// captured into a CUDA graph the events become event-record nodes of the graph (read after each
// replay by prof_collect); otherwise they come from the context's pool.
struct ProfScope {
    recon_ctx* c;
    int kind;
    size_t i0 = 0;
    bool on = false;
    cudaEvent_t g0 = nullptr, g1 = nullptr;
    ProfScope(recon_ctx* c_, int kind_) : c(c_), kind(kind_) {
        if (!(c->prof & (1u << kind))) return;
        if (c->capturing) {
            if (cudaEventCreate(&g0) != cudaSuccess) return;
            if (cudaEventCreate(&g1) != cudaSuccess) {
                cudaEventDestroy(g0);
                return;
            }
            cudaEventRecordWithFlags(g0, c->stream, cudaEventRecordExternal);
            on = true;
            return;
        }
        if (c->ev_used + 2 > c->ev_pool.size()) {
            for (int k = 0; k < 256; ++k) {
                cudaEvent_t e;
                if (cudaEventCreate(&e) != cudaSuccess) return;
                c->ev_pool.push_back(e);
            }
        }
        i0 = c->ev_used;
        c->ev_used += 2;
        cudaEventRecord(c->ev_pool[i0], c->stream);
        on = true;
    }
    ~ProfScope() {
        if (!on) return;
        if (g0) {
            cudaEventRecordWithFlags(g1, c->stream, cudaEventRecordExternal);
            c->capturing->ev.emplace_back(kind, g0, g1);
            return;
        }
        cudaEventRecord(c->ev_pool[i0 + 1], c->stream);
        c->prof_pending.push_back({kind, i0});
    }
};

void collect_graph(recon_ctx* c, GraphProf* gp) {
    if (!gp || gp->replays == gp->collected) return;
    for (auto& t : gp->ev) {  // the most recent replay's launches
        float ms = 0.f;
        cudaEventSynchronize(std::get<2>(t));
        if (cudaEventElapsedTime(&ms, std::get<1>(t), std::get<2>(t)) == cudaSuccess) {
            c->prof_ms[std::get<0>(t)] += ms;
            c->prof_n[std::get<0>(t)] += 1;
        }
    }
    gp->collected = gp->replays;
}

// Fold the recorded event pairs into the per-kind totals (synchronises on the events); for solves
// replayed from a graph, the launches of the latest replay not yet read.
void prof_collect(recon_ctx* c) {
    collect_graph(c, c->gprof);
    for (auto& sl : c->slots) collect_graph(c, sl.gprof);
    collect_graph(c, c->batch_gprof);
    for (auto& pk : c->prof_pending) {
        float ms = 0.f;
        cudaEventSynchronize(c->ev_pool[pk.second + 1]);
        if (cudaEventElapsedTime(&ms, c->ev_pool[pk.second], c->ev_pool[pk.second + 1]) == cudaSuccess) {
            c->prof_ms[pk.first] += ms;
            c->prof_n[pk.first] += 1;
        }
    }
    c->prof_pending.clear();
    c->ev_used = 0;
}

// Device buffer `name` of at least `bytes` (contents undefined on growth).
int ensure(recon_ctx* c, const char* name, size_t bytes, void** out) {
    Buf& b = c->bufs[name];
    if (b.bytes >= bytes && b.ptr) {
        *out = b.ptr;
        return RECON_OK;
    }
    if (b.ptr) {
        cudaFree(b.ptr);
        c->allocated -= b.bytes;
        b = Buf{};
    }
    ++c->ws_gen;  // captured solves that point into this workspace are stale now
    const size_t want = bytes < 256 ? 256 : bytes;
    if (c->budget && c->allocated + want > c->budget)
        return fail(c, RECON_ENOMEM, std::string("workspace budget exceeded allocating ") + name);
    cudaError_t e = cudaMalloc(&b.ptr, want);
    if (e != cudaSuccess) {
        b = Buf{};
        cudaGetLastError();
        return fail(c, RECON_ENOMEM, std::string("cudaMalloc failed for ") + name + ": " +
                                         cudaGetErrorString(e));
    }
    b.bytes = want;
    c->allocated += want;
    *out = b.ptr;
    return RECON_OK;
}

int twiddles(recon_ctx* c, int n, TwTable* out) {
    auto it = c->tw.find(n);
    if (it != c->tw.end()) {
        *out = it->second;
        return RECON_OK;
    }
    std::vector<float2> hf(n);
    std::vector<double2> hd(n);
    for (int j = 0; j < n; ++j) {
        // e^{-2 pi i j / n}; exact at the quarter points
        double cr, ci;
        if ((4 * j) % n == 0) {
            const int q = (4 * j) / n;
            const double cs[4] = {1.0, 0.0, -1.0, 0.0}, sn[4] = {0.0, -1.0, 0.0, 1.0};
            cr = cs[q];
            ci = sn[q];
        } else {
            const double ang = 2.0 * M_PI * (double)j / (double)n;
            cr = std::cos(ang);
            ci = -std::sin(ang);
        }
        hd[j] = make_double2(cr, ci);
        hf[j] = make_float2((float)cr, (float)ci);
    }
    TwTable t;
    RC_CUDA(cudaMalloc(&t.f, n * sizeof(float2)));
    RC_CUDA(cudaMalloc(&t.d, n * sizeof(double2)));
    RC_CUDA(cudaMemcpy(t.f, hf.data(), n * sizeof(float2), cudaMemcpyHostToDevice));
    RC_CUDA(cudaMemcpy(t.d, hd.data(), n * sizeof(double2), cudaMemcpyHostToDevice));
    c->tw[n] = t;
    *out = t;
    return RECON_OK;
}

int get_twiddles(recon_ctx* c, const Dims& d, Twiddles* tw) {
    TwTable tp, tq;
    int rc = twiddles(c, d.P, &tp);
    if (rc) return rc;
    rc = twiddles(c, d.Q, &tq);
    if (rc) return rc;
    tw->twP = tp.f;
    tw->twQ = tq.f;
    tw->twPd = tp.d;
    tw->twQd = tq.d;
    if (d.R > 1) {
        TwTable tr;
        rc = twiddles(c, d.R, &tr);
        if (rc) return rc;
        tw->twR = tr.f;
        tw->twRd = tr.d;
    }
    return RECON_OK;
}

size_t gram_smem_bytes(const Dims& d) { return recon::gram_smem(d); }

// Geometry checks shared by the image-series (R = 1) and volume entry points; f = NULL for calls
// without a filter.
int check_geometry(recon_ctx* c, int T, int R, int P, int Q, const recon_filter3* f, Dims* d) {
    if (P <= 0 || Q <= 0 || T <= 0 || R <= 0)
        return fail(c, RECON_EINVAL, "P, Q, R, T must be positive");
    if (!recon::fft_size_supported(P) || !recon::fft_size_supported(Q))
        return fail(c, RECON_EINVAL, "P and Q must be one of 16, 32, 64, 128, 192, 256, 512");
    if (R > 1 && !recon::fft_size_supported(R))
        return fail(c, RECON_EINVAL, "R must be 1 or one of 16, 32, 64, 128, 192, 256, 512");
    *d = Dims{};
    d->T = T;
    d->P = P;
    d->Q = Q;
    d->R = R;
    d->N1 = d->N2 = d->N3 = d->M = 1;
    if (f) {
        if (f->M < 1 || f->M > recon::w_max_M() || f->M > T)
            return fail(c, RECON_EINVAL, "need 1 <= M <= min(6, T)");
        if (f->N1 < 1 || f->N1 > P || f->N2 < 1 || f->N2 > Q)
            return fail(c, RECON_EINVAL, "need 1 <= N1 <= P and 1 <= N2 <= Q");
        if (f->N3 < 1 || f->N3 > R) return fail(c, RECON_EINVAL, "need 1 <= N3 <= R");
        d->N1 = f->N1;
        d->N2 = f->N2;
        d->N3 = f->N3;
        d->M = f->M;
        if (gram_smem_bytes(*d) > 220 * 1024)
            return fail(c, RECON_EINVAL, "filter / frame count too large for the Gram kernel");
    }
    if ((long long)T * Q > recon::w_max_frames_times_q())
        return fail(c, RECON_EINVAL, "T * Q too large for the fused row pass");
    if ((long long)T * R * P > (1LL << 30)) return fail(c, RECON_EINVAL, "problem too large");
    return RECON_OK;
}

int check_dims(recon_ctx* c, recon_dims dd, const recon_filter* f, Dims* d) {
    if (!f) return check_geometry(c, dd.T, 1, dd.P, dd.Q, nullptr, d);
    const recon_filter3 f3{f->N1, f->N2, 1, f->M};
    return check_geometry(c, dd.T, 1, dd.P, dd.Q, &f3, d);
}

int check_dims3(recon_ctx* c, recon_dims3 dd, const recon_filter3* f, Dims* d) {
    return check_geometry(c, dd.T, dd.R, dd.P, dd.Q, f, d);
}

struct Work {
    float2 *r, *p, *t, *S0, *S1;
    double2 *G, *lag_part, *lags, *dpart, *dsum, *Z, *eigwork;
    double *evals, *parts, *rparts, *rr, *pq, *eps, *lmax;
    unsigned int* counter;
    int *info, *kerr;
    void *hpd = nullptr, *lanc = nullptr;
    int lwork;
    int gblocks;
    int n_status;
    bool use_eig;
    recon::CoopFault fault;  // test hook of the cooperative weight kernels (default: none)
};

int eig_lwork(recon_ctx* c, int s, double2* G, double* evals, int* lwork) {
    cusolverStatus_t st = cusolverDnZheevd_bufferSize(
        c->solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, s,
        reinterpret_cast<cuDoubleComplex*>(G), s, evals, lwork);
    if (st != CUSOLVER_STATUS_SUCCESS) return fail(c, RECON_ECUDA, "zheevd_bufferSize failed");
    return RECON_OK;
}

// Weight method: the p = 0 weight (G + eps I)^-1 is formed by the FP64 sweep inverse unless the
// eigendecomposition is asked for (or p > 0, which needs the eigenvalues).
bool wants_eig(double p, int method) { return method == RECON_WEIGHT_EIG || p != 0.0; }

// Allocate (or reuse) the workspace of one solve. n_iter: number of weight steps to record.
int get_work(recon_ctx* c, const Dims& d, int n_cg, int n_iter, bool vectors, bool use_eig,
             Work* w) {
    void* ptr;
    int rc;
    const size_t vec = d.elems() * sizeof(float2);
    const size_t sbytes = (size_t)d.npair() * d.pixels() * sizeof(float2);
    const int s = d.s();
    const size_t nlag = d.nlag();
    const int ni = n_iter < 1 ? 1 : n_iter;
    w->gblocks = recon::gram_blocks(d);
    w->use_eig = use_eig;
#define GET(name, bytes, field, type)                         \
    rc = ensure(c, name, (bytes), &ptr);                      \
    if (rc) return rc;                                        \
    w->field = reinterpret_cast<type>(ptr);
    if (vectors) {
        GET("r", vec, r, float2*);
        GET("p", vec, p, float2*);
        GET("t", vec * (size_t)d.nc, t, float2*);  // one series per coil
        GET("S0", sbytes, S0, float2*);
        GET("S1", sbytes, S1, float2*);
    }
    GET("G", (size_t)s * s * sizeof(double2), G, double2*);
    GET("lag_part", recon::gram_scratch_bytes(d, w->gblocks), lag_part, double2*);
    GET("lags", nlag * sizeof(double2), lags, double2*);
    GET("dsum", nlag * sizeof(double2), dsum, double2*);
    GET("Z", recon::s_scratch_bytes(d), Z, double2*);
    GET("parts", (size_t)recon::max_parts() * sizeof(double), parts, double*);
    GET("rparts", (size_t)recon::max_parts() * sizeof(double), rparts, double*);
    GET("counter", 256, counter, unsigned int*);
    GET("rr", (size_t)(n_cg + 1) * sizeof(double), rr, double*);
    GET("pq", (size_t)(n_cg + 1) * sizeof(double), pq, double*);
    GET("eps", 2 * sizeof(double), eps, double*);
    w->lmax = w->eps + 1;
    GET("info", (size_t)ni * sizeof(int), info, int*);
    GET("kerr", (size_t)2 * ni * sizeof(int), kerr, int*);
    if (use_eig) {
        GET("evals", (size_t)s * sizeof(double), evals, double*);
        GET("dpart", recon::diag_scratch_bytes(d), dpart, double2*);
        rc = eig_lwork(c, s, w->G, w->evals, &w->lwork);
        if (rc) return rc;
        GET("eigwork", (size_t)(w->lwork < 1 ? 1 : w->lwork) * sizeof(double2), eigwork, double2*);
    } else {
        int dev = 0, sms = 0;
        RC_CUDA(cudaGetDevice(&dev));
        RC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        // the grid barriers of the cooperative kernels start zeroed (see kCoopBarrierBytes)
        unsigned long gen0 = c->ws_gen;
        GET("hpd", recon::hpd_scratch_bytes(d), hpd, void*);
        if (c->ws_gen != gen0) RC_CUDA(cudaMemsetAsync(w->hpd, 0, recon::kCoopBarrierBytes, c->stream));
        gen0 = c->ws_gen;
        GET("lanc", recon::lanczos_scratch_bytes(d, sms), lanc, void*);
        if (c->ws_gen != gen0) RC_CUDA(cudaMemsetAsync(w->lanc, 0, recon::kCoopBarrierBytes, c->stream));
    }
#undef GET
    w->n_status = ni;
    return RECON_OK;
}

// Reset the counters and status words of a workspace (stream-ordered; part of a captured solve).
int reset_status(recon_ctx* c, Work& w) {
    RC_CUDA(cudaMemsetAsync(w.counter, 0, sizeof(unsigned int), c->stream));
    RC_CUDA(cudaMemsetAsync(w.info, 0, (size_t)w.n_status * sizeof(int), c->stream));
    RC_CUDA(cudaMemsetAsync(w.kerr, 0, (size_t)2 * w.n_status * sizeof(int), c->stream));
    return RECON_OK;
}

int run_eig(recon_ctx* c, int s, Work& w, int* info) {
    cusolverStatus_t st = cusolverDnZheevd(
        c->solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, s,
        reinterpret_cast<cuDoubleComplex*>(w.G), s, w.evals,
        reinterpret_cast<cuDoubleComplex*>(w.eigwork), w.lwork, info);
    if (st != CUSOLVER_STATUS_SUCCESS) return fail(c, RECON_ECUDA, "cusolverDnZheevd failed");
    return RECON_OK;
}

// Weight step on w.G (consumed): eps update, H (eigendecomposition or sweep inverse), summed
// diagonals, S. `it` indexes the per-iteration status slots (eigensolver info, barrier flags).
int weight_step(recon_ctx* c, const Dims& d, const Twiddles& tw, Work& w, double p, int eps_first,
                double eps_frac, double gamma, int eps_mode_set, double eps_value, float2* S,
                int it) {
    if (eps_mode_set)
        RC_CUDA(cudaMemcpyAsync(w.eps, &eps_value, sizeof(double), cudaMemcpyHostToDevice, c->stream));
    if (w.use_eig) {
        {
            ProfScope ps(c, RECON_PROF_EIG);
            int rc = run_eig(c, d.s(), w, w.info + it);
            if (rc) return rc;
        }
        if (!eps_mode_set) {
            ProfScope ps(c, RECON_PROF_EPS);
            RC_CUDA(recon::launch_eps(w.evals + d.s() - 1, w.eps, eps_first, eps_frac, gamma, c->stream));
        }
        ProfScope ps(c, RECON_PROF_DIAG);
        RC_CUDA(recon::launch_diag_sums(d, w.G, w.evals, w.eps, p, w.dpart, w.dsum, c->stream));
    } else {
        if (!eps_mode_set) {
            if (eps_first) {
                ProfScope ps(c, RECON_PROF_LANCZOS);
                RC_CUDA(recon::launch_lanczos_lmax(d, w.G, w.lanc, w.lmax, w.kerr + 2 * it + 1, c->stream,
                                                   w.fault));
            }
            ProfScope ps(c, RECON_PROF_EPS);
            RC_CUDA(recon::launch_eps(w.lmax, w.eps, eps_first, eps_frac, gamma, c->stream));
        }
        {
            ProfScope ps(c, RECON_PROF_INV);
            RC_CUDA(recon::launch_hpd_inverse(d, w.G, w.eps, w.hpd, w.kerr + 2 * it, c->stream, w.fault));
        }
        ProfScope ps(c, RECON_PROF_DIAG);
        RC_CUDA(recon::launch_hdiag(d, w.G, w.dsum, c->stream));
    }
    {
        ProfScope ps(c, RECON_PROF_S);
        RC_CUDA(recon::launch_weight_S(d, tw, w.dsum, w.Z, S, c->stream));
    }
    return RECON_OK;
}

// After the stream finished: eigensolver status and device-wait flags of n_iter weight steps.
int check_status(recon_ctx* c, Work& w, int n_iter) {
    if (n_iter < 1) return RECON_OK;
    std::vector<int> info(n_iter), kerr(2 * (size_t)n_iter);
    RC_CUDA(cudaMemcpy(info.data(), w.info, n_iter * sizeof(int), cudaMemcpyDeviceToHost));
    RC_CUDA(cudaMemcpy(kerr.data(), w.kerr, 2 * (size_t)n_iter * sizeof(int), cudaMemcpyDeviceToHost));
    for (int e : kerr)
        if (e != 0) {
            // re-arm the grid barriers for the next solve (a failed launch leaves them set)
            if (w.hpd) RC_CUDA(cudaMemset(w.hpd, 0, recon::kCoopBarrierBytes));
            if (w.lanc) RC_CUDA(cudaMemset(w.lanc, 0, recon::kCoopBarrierBytes));
            RC_CUDA(cudaDeviceSynchronize());
            return fail(c, RECON_ETIMEOUT, "a bounded device-wide barrier timed out");
        }
    for (int e : info)
        if (e != 0) return fail(c, RECON_ENUMERIC, "eigensolver failed (info != 0)");
    return RECON_OK;
}

// Residual carry + n_cg CG steps on x (in place).
int cg_block(recon_ctx* c, const Dims& d, const Twiddles& tw, Work& w, const uint8_t* mask,
             const float2* S_old, const float2* S_new, float lam, float2* x, int first, int n_cg,
             const float2* coils = nullptr, bool coil_proj = false) {
    const recon::RedSlot rs{w.parts, w.counter};
    {
        ProfScope ps(c, RECON_PROF_RESID);
        const float2* aha_x = nullptr;
        if (first && coils && !coil_proj) {
            // with coils A A^H is no projection: the first residual needs A^H A x0 (in coil 0's
            // plane of t, from the operator passes with lambda = 0). One coil of unit modulus
            // keeps the projection, and the exact identity avoids the FP32 cancellation.
            const recon::Partials none{nullptr, 0};
            recon::Partials scratch{w.rparts, 0};
            RC_CUDA(recon::launch_coil_row_fwd(d, tw, x, w.p, w.t, coils, none, nullptr, nullptr, 1,
                                               c->stream));
            RC_CUDA(recon::launch_col_mask(d, tw, w.t, mask, c->stream));
            RC_CUDA(recon::launch_coil_row_inv_w(d, tw, w.t, w.p, coils, S_new, 0.f, &scratch,
                                                 c->stream));
            aha_x = w.t;
        }
        RC_CUDA(recon::launch_resid_carry(d, w.r, x, S_old, S_new, lam, first, rs, w.rr, c->stream,
                                          aha_x));
    }
    // Dot products travel as per-CTA partials: pass C leaves those of Re <p, q> in w.parts for
    // the update pass; the update pass leaves those of |r|^2 in w.rparts for the next pass A,
    // which also stores the sum in rr[it] (rr[0] comes from the residual carry).
    recon::Partials pq{w.parts, 0}, rr{w.rparts, 0};
    for (int it = 0; it < n_cg; ++it) {
        const double* rr_prev = it > 0 ? w.rr + it - 1 : w.rr;
        {
            ProfScope ps(c, RECON_PROF_CG_ROWFWD);
            if (coils)
                RC_CUDA(recon::launch_coil_row_fwd(d, tw, w.r, w.p, w.t, coils, rr, rr_prev,
                                                   w.rr + it, it == 0, c->stream));
            else
                RC_CUDA(recon::launch_row_fwd_pupdate(d, tw, w.r, w.p, w.t, rr, rr_prev,
                                                      w.rr + it, it == 0, c->stream));
        }
        {
            ProfScope ps(c, RECON_PROF_CG_COL);
            RC_CUDA(recon::launch_col_mask(d, tw, w.t, mask, c->stream));
        }
        {
            ProfScope ps(c, RECON_PROF_CG_ROWINVW);
            if (coils)
                RC_CUDA(recon::launch_coil_row_inv_w(d, tw, w.t, w.p, coils, S_new, lam, &pq,
                                                     c->stream));
            else
                RC_CUDA(recon::launch_row_inv_w(d, tw, w.t, w.p, S_new, lam, &pq, c->stream));
        }
        ProfScope ps(c, RECON_PROF_CG_UPDATE);
        RC_CUDA(recon::launch_cg_update(d, x, w.r, w.p, w.t, w.rr + it, pq, &rr, c->stream));
    }
    if (n_cg > 0) RC_CUDA(recon::launch_sum_partials(rr, w.rr + n_cg, c->stream));
    return RECON_OK;
}

int select_slot(recon_ctx* c, int i);

// Every entry point starts here: the context's device current and slot 0 (the context's own
// stream and workspace) active.
int set_device(recon_ctx* c) {
    RC_CUDA(cudaSetDevice(c->device));
    return select_slot(c, 0);
}

// Make slot i active (creating it on first use: own non-blocking stream, no workspace yet).
int select_slot(recon_ctx* c, int i) {
    if ((int)c->slots.size() < i + 1) c->slots.resize(i + 1);
    if (i == c->active) return RECON_OK;
    auto& park = c->slots[c->active];
    park.stream = c->stream;
    park.own_stream = c->own_stream;
    park.bufs = std::move(c->bufs);
    park.solver = c->solver;
    park.ws_gen = c->ws_gen;
    park.gkey = c->gkey;
    park.gexec = c->gexec;
    park.gprof = c->gprof;
    auto& next = c->slots[i];
    if (!next.stream) {
        cudaError_t e = cudaStreamCreateWithFlags(&next.stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            c->bufs = std::move(park.bufs);
            return cuda_fail(c, e, "cudaStreamCreateWithFlags");
        }
        next.own_stream = true;
    }
    c->stream = next.stream;
    c->own_stream = next.own_stream;
    c->bufs = std::move(next.bufs);
    c->solver = next.solver;
    c->ws_gen = next.ws_gen;
    c->gkey = next.gkey;
    c->gexec = next.gexec;
    c->gprof = next.gprof;
    next = recon_ctx::Slot{};
    c->active = i;
    return RECON_OK;
}

int ensure_solver(recon_ctx* c) {
    if (c->solver) return RECON_OK;
    if (cusolverDnCreate(&c->solver) != CUSOLVER_STATUS_SUCCESS)
        return fail(c, RECON_ECUDA, "cusolverDnCreate failed");
    if (cusolverDnSetStream(c->solver, c->stream) != CUSOLVER_STATUS_SUCCESS)
        return fail(c, RECON_ECUDA, "cusolverDnSetStream failed");
    return RECON_OK;
}

int check_prm(recon_ctx* c, const recon_params* prm) {
    if (prm->irls < 0 || prm->cg < 1) return fail(c, RECON_EINVAL, "need irls >= 0, cg >= 1");
    if (!(prm->lambda > 0.0) || !std::isfinite(prm->lambda))
        return fail(c, RECON_EINVAL, "lambda must be positive and finite");
    if (!(prm->p >= 0.0 && prm->p <= 1.0)) return fail(c, RECON_EINVAL, "need 0 <= p <= 1");
    if (!(prm->gamma >= 1.0) || !std::isfinite(prm->gamma)) return fail(c, RECON_EINVAL, "need gamma >= 1");
    if (!(prm->eps0_frac > 0.0) || !std::isfinite(prm->eps0_frac))
        return fail(c, RECON_EINVAL, "eps0_frac must be positive");
    if (prm->weight_method != RECON_WEIGHT_AUTO && prm->weight_method != RECON_WEIGHT_EIG)
        return fail(c, RECON_EINVAL, "unknown weight method");
    return RECON_OK;
}

int check_params(recon_ctx* c, recon_dims dd, recon_filter f, const recon_params* prm, Dims* d) {
    int rc = check_dims(c, dd, &f, d);
    return rc ? rc : check_prm(c, prm);
}

// One solve in flight on the active slot's stream.
struct Solve {
    Dims d;
    Twiddles tw;
    Work w;
    float2* x;
    const void* kspace;
    const uint8_t* masks;
    const recon_params* prm;
    const float2* coils = nullptr;  // [nc][P][Q] for the multi-coil operator
    bool coil_proj = false;         // one coil with |C| = 1: A A^H is a projection
    int variant = RECON_VARIANT_PROPOSED;  // HLR-Voxel: per-pixel weights instead of the Gram
};

// Autotuner of the column passes: on the first solve of a shape (P, Q, T, R, coils) the context
// times the column stage of the CG operator (launch_col_mask, one warm-up and three timed
// launches per candidate, CUDA events on the solve's stream) for tile widths of 8, 16 and 32
// columns -- first for the length-P passes, then, for volumes, for the depth passes -- and keeps
// the fastest. The width changes only the launch shape: every column is transformed by the same
// arithmetic, so results do not depend on the choice. Choices are cached per context and, when a
// cache file is set (recon_tile_cache), appended to it and read back by later contexts.
int autotune_tiles(recon_ctx* c, Dims* d, const Twiddles& tw, float2* t, const uint8_t* mask) {
    const auto key = std::make_tuple(d->P, d->Q, d->T, d->R, d->nc);
    auto apply_forced = [&]() {
        if (c->fft_sched >= 0) d->colS = d->depthS = c->fft_sched;
    };
    auto it = c->tiles.find(key);
    if (it != c->tiles.end()) {
        d->colC = it->second.colC;
        d->depthC = it->second.depthC;
        d->colS = it->second.colS;
        d->depthS = it->second.depthS;
        apply_forced();
        return RECON_OK;
    }
    if (!c->autotune) {
        apply_forced();
        return RECON_OK;
    }
    cudaEvent_t e0, e1;
    RC_CUDA(cudaEventCreate(&e0));
    RC_CUDA(cudaEventCreate(&e1));
    auto time_it = [&](Dims& dd, float* ms) -> cudaError_t {
        cudaError_t e = recon::launch_col_mask(dd, tw, t, mask, c->stream);
        if (e != cudaSuccess) return e;
        e = cudaEventRecord(e0, c->stream);
        for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = recon::launch_col_mask(dd, tw, t, mask, c->stream);
        if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
        return e;
    };
    cudaError_t err = cudaSuccess;
    const int cand[3] = {8, 16, 32};
    // radix schedules tried (the Stockham passes' factorisation order), when asked for
    const int nsched = c->autotune_fft ? recon::kFftSchedules : 1;
    Dims dd = *d;
    // the length-P passes (those in register transforms have no tiles or schedules to choose)
    if (!recon::col_register(*d, false)) {
        float best = 1e30f;
        int bestC = recon::col_tile_for(*d, false), bestS = 0;
        for (int S = 0; S < nsched && err == cudaSuccess; ++S)
            for (int C : cand) {
                if (d->Q % C) continue;
                dd.colC = C;
                dd.colS = S;
                float ms = 0.f;
                err = time_it(dd, &ms);
                if (err != cudaSuccess) break;
                if (ms < best) { best = ms; bestC = C; bestS = S; }
            }
        dd.colC = bestC;
        dd.colS = bestS;
    }
    if (err == cudaSuccess && d->R > 1 && !recon::col_register(*d, true)) {
        float best = 1e30f;
        int bestC = recon::col_tile_for(*d, true), bestS = 0;
        for (int S = 0; S < nsched && err == cudaSuccess; ++S)
            for (int C : cand) {
                if ((d->P * d->Q) % C) continue;
                dd.depthC = C;
                dd.depthS = S;
                float ms = 0.f;
                err = time_it(dd, &ms);
                if (err != cudaSuccess) break;
                if (ms < best) { best = ms; bestC = C; bestS = S; }
            }
        dd.depthC = bestC;
        dd.depthS = bestS;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) return cuda_fail(c, err, "autotuner");
    d->colC = dd.colC;
    d->depthC = dd.depthC;
    d->colS = dd.colS;
    d->depthS = dd.depthS;
    c->tiles[key] = {d->colC, d->depthC, d->colS, d->depthS};
    if (!c->tile_cache.empty()) {
        std::ofstream f(c->tile_cache, std::ios::app);
        if (f) f << d->P << ' ' << d->Q << ' ' << d->T << ' ' << d->R << ' ' << d->nc << ' '
                 << d->colC << ' ' << d->depthC << ' ' << d->colS << ' ' << d->depthS << '\n';
    }
    apply_forced();
    return RECON_OK;
}

// Twiddles, eigensolver handle and workspace of one solve on the active slot (no stream work).
int solve_prepare(recon_ctx* c, const Dims& d, const void* kspace, const uint8_t* masks,
                  const recon_params* prm, void* image_out, Solve* sv) {
    sv->d = d;
    sv->kspace = kspace;
    sv->masks = masks;
    sv->prm = prm;
    sv->x = reinterpret_cast<float2*>(image_out);
    int rc = get_twiddles(c, d, &sv->tw);
    if (rc) return rc;
    const bool eig = wants_eig(prm->p, prm->weight_method);
    if (eig) {
        rc = ensure_solver(c);
        if (rc) return rc;
    }
    rc = get_work(c, d, prm->cg, prm->irls, true, eig, &sv->w);
    if (rc) return rc;
    if (c->inject_barrier_fault && sv->w.hpd) {
        // host-side fault injection: the sweep's barrier error word set, as a peer that gave up
        // would leave it; the sweeps then return at their first barrier and report it
        c->inject_barrier_fault = false;
        RC_CUDA(recon::set_barrier_error(sv->w.hpd, c->stream));
    }
    if (c->withhold_arrival && sv->w.hpd) {
        // host-directed lost peer: CTA 1 of the Lanczos and sweep launches of this solve leaves
        // at its first grid barrier without arriving; the others' waits give up after 4096 polls
        c->withhold_arrival = false;
        sv->w.fault.withhold = 1;
        sv->w.fault.polls = 4096;
    }
    return autotune_tiles(c, &sv->d, sv->tw, sv->w.t, masks);
}

// HLR-Voxel: per-pixel weights instead of the Gram (after solve_prepare).
int prepare_voxel(recon_ctx* c, Solve* sv) {
    (void)c;
    sv->variant = RECON_VARIANT_HLR_VOXEL;
    return RECON_OK;
}

// Status reset and x0 = A^H b (Algorithm 1 initialisation). Enqueues only.
int solve_begin(recon_ctx* c, Solve* sv) {
    int rc = reset_status(c, sv->w);
    if (rc) return rc;
    ProfScope ps(c, RECON_PROF_ADJOINT);
    if (sv->coils) {
        RC_CUDA(recon::launch_adjoint_coils_cols(sv->d, sv->tw, sv->kspace, sv->masks, sv->w.t,
                                                 c->stream));
        RC_CUDA(recon::launch_coil_combine(sv->d, sv->tw, sv->w.t, sv->coils, sv->x, c->stream));
        return RECON_OK;
    }
    RC_CUDA(recon::launch_adjoint(sv->d, sv->tw, sv->kspace, sv->prm->kspace_bf16, sv->masks,
                                  sv->w.t, sv->x, c->stream));
    return RECON_OK;
}

// IRLS iteration n of Algorithm 1: Gram, weight, residual carry, CG. Enqueues only.
int solve_iter(recon_ctx* c, Solve& sv, int n) {
    const Dims& d = sv.d;
    Work& w = sv.w;
    float2* S[2] = {w.S0, w.S1};
    float2* S_new = S[n & 1];
    const float2* S_old = n == 0 ? nullptr : S[(n + 1) & 1];
    if (sv.variant == RECON_VARIANT_HLR_VOXEL) {
        // one M x M Gram, eigendecomposition and weight per pixel with one eps for the whole
        // penalty: eps0 = eps0_frac * (largest lambda_max(G_r(x0)) over the pixels), then
        // eps <- eps / gamma (Sec. III-C)
        ProfScope ps(c, RECON_PROF_S);
        if (n == 0) {
            RC_CUDA(cudaMemsetAsync(w.lmax, 0, sizeof(double), c->stream));
            RC_CUDA(recon::launch_voxel_weight(d, sv.x, sv.prm->p, nullptr, w.lmax, 1, nullptr,
                                               nullptr, nullptr, c->stream));
        }
        RC_CUDA(recon::launch_eps(w.lmax, w.eps, n == 0, sv.prm->eps0_frac, sv.prm->gamma, c->stream));
        RC_CUDA(recon::launch_voxel_weight(d, sv.x, sv.prm->p, w.eps, nullptr, 2, S_new, nullptr,
                                           nullptr, c->stream));
    } else {
        {
            ProfScope ps(c, RECON_PROF_GRAM);
            RC_CUDA(recon::launch_gram(d, sv.tw, sv.x, w.lag_part, w.gblocks, nullptr, w.G,
                                       c->stream));
        }
        int rc = weight_step(c, d, sv.tw, w, sv.prm->p, n == 0, sv.prm->eps0_frac, sv.prm->gamma,
                             0, 0.0, S_new, n);
        if (rc) return rc;
    }
    return cg_block(c, d, sv.tw, w, sv.masks, S_old, S_new, (float)sv.prm->lambda, sv.x, n == 0,
                    sv.prm->cg, sv.coils, sv.coil_proj);
}

// The key of a solve's graph (shapes, parameters, buffers, workspace generation, options).
recon_ctx::GraphKey graph_key(recon_ctx* c, const Solve& sv) {
    const recon_params* prm = sv.prm;
    recon_ctx::GraphKey k;
    std::memset(&k, 0, sizeof(k));
    k.T = sv.d.T; k.P = sv.d.P; k.Q = sv.d.Q; k.N1 = sv.d.N1; k.N2 = sv.d.N2; k.M = sv.d.M;
    k.R = sv.d.R; k.N3 = sv.d.N3;
    k.irls = prm->irls; k.cg = prm->cg; k.bf16 = prm->kspace_bf16; k.method = prm->weight_method;
    k.lambda = prm->lambda; k.p = prm->p; k.gamma = prm->gamma; k.eps0_frac = prm->eps0_frac;
    k.kspace = sv.kspace; k.masks = sv.masks; k.out = sv.x; k.ws_gen = c->ws_gen;
    k.coils = sv.coils; k.nc = sv.d.nc; k.coil_proj = sv.coil_proj;
    k.circ = sv.d.circ; k.variant = sv.variant; k.colC = sv.d.colC; k.depthC = sv.d.depthC;
    k.colS = sv.d.colS; k.depthS = sv.d.depthS;
    k.prof = c->prof;
    return k;
}

// Enqueue a whole solve on the active slot's stream: as one replay of a captured CUDA graph
// (captured on first use, cached per slot and keyed by shapes, parameters, buffers and the
// workspace generation), or as direct launches when graphs are off, when the eigensolver
// library path is used, or while launch classes are being timed.
int solve_enqueue_all(recon_ctx* c, Solve& sv) {
    const recon_params* prm = sv.prm;
    const bool direct = !c->graphs || wants_eig(prm->p, prm->weight_method) || sv.w.fault.withhold;
    if (direct) {
        int rc = solve_begin(c, &sv);
        for (int n = 0; n < prm->irls && !rc; ++n) rc = solve_iter(c, sv, n);
        return rc;
    }
    const recon_ctx::GraphKey k = graph_key(c, sv);
    if (!c->gexec || std::memcmp(&k, &c->gkey, sizeof(k)) != 0) {
        if (c->gexec) {
            cudaGraphExecDestroy(c->gexec);
            c->gexec = nullptr;
        }
        delete c->gprof;
        c->gprof = c->prof ? new GraphProf() : nullptr;
        c->capturing = c->gprof;
        RC_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed));
        int rc = solve_begin(c, &sv);
        for (int n = 0; n < prm->irls && !rc; ++n) rc = solve_iter(c, sv, n);
        cudaGraph_t g = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(c->stream, &g);
        c->capturing = nullptr;
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (ec != cudaSuccess) return cuda_fail(c, ec, "cudaStreamEndCapture");
        const cudaError_t ei = cudaGraphInstantiate(&c->gexec, g, 0);
        cudaGraphDestroy(g);
        if (ei != cudaSuccess) {
            c->gexec = nullptr;
            return cuda_fail(c, ei, "cudaGraphInstantiate");
        }
        c->gkey = k;
    }
    RC_CUDA(cudaGraphLaunch(c->gexec, c->stream));
    if (c->gprof) ++c->gprof->replays;
    return RECON_OK;
}

// ---- lockstep batches: the weight steps of a group of solves share their launches ----

// Gram of x^(n-1) into the solve's G (active slot's stream).
int iter_gram(recon_ctx* c, Solve& sv) {
    ProfScope ps(c, RECON_PROF_GRAM);
    RC_CUDA(recon::launch_gram(sv.d, sv.tw, sv.x, sv.w.lag_part, sv.w.gblocks, nullptr, sv.w.G,
                               c->stream));
    return RECON_OK;
}

// The FP64 weight of a group of solves (p = 0 sweep path) in shared launches on the active
// stream: at n = 0 one Lanczos launch for every lambda_max, then one eps launch and one sweep
// launch for all. The group leader's scratch holds the barriers of the shared launches.
int group_weight(recon_ctx* c, Solve* grp, int cnt, int n) {
    if (n == 0) {
        recon::LanczosJob jobs[recon::kMaxHpdBatch];
        for (int b = 0; b < cnt; ++b)
            jobs[b] = {grp[b].w.G, grp[b].w.lanc, grp[b].w.lmax, grp[b].w.kerr + 2 * n + 1, grp[b].d.s()};
        ProfScope ps(c, RECON_PROF_LANCZOS);
        RC_CUDA(recon::launch_lanczos_batch(jobs, cnt, grp[0].w.lanc, c->stream, grp[0].w.fault));
    }
    {
        const double* lmax[recon::kMaxHpdBatch];
        double* eps[recon::kMaxHpdBatch];
        for (int b = 0; b < cnt; ++b) {
            lmax[b] = grp[b].w.lmax;
            eps[b] = grp[b].w.eps;
        }
        ProfScope ps(c, RECON_PROF_EPS);
        RC_CUDA(recon::launch_eps_batch(lmax, eps, cnt, n == 0, grp[0].prm->eps0_frac,
                                        grp[0].prm->gamma, c->stream));
    }
    recon::HpdJob jobs[recon::kMaxHpdBatch];
    for (int b = 0; b < cnt; ++b)
        jobs[b] = {grp[b].w.G, grp[b].w.eps, grp[b].w.hpd, grp[b].w.kerr + 2 * n, grp[b].d.s()};
    ProfScope ps(c, RECON_PROF_INV);
    RC_CUDA(recon::launch_hpd_inverse_batch(jobs, cnt, grp[0].w.hpd, c->stream, grp[0].w.fault));
    return RECON_OK;
}

// After the weight: summed diagonals of H, S(r), residual carry and the CG steps (active slot).
int iter_post_weight(recon_ctx* c, Solve& sv, int n) {
    Work& w = sv.w;
    float2* S[2] = {w.S0, w.S1};
    float2* S_new = S[n & 1];
    const float2* S_old = n == 0 ? nullptr : S[(n + 1) & 1];
    {
        ProfScope ps(c, RECON_PROF_DIAG);
        RC_CUDA(recon::launch_hdiag(sv.d, w.G, w.dsum, c->stream));
    }
    {
        ProfScope ps(c, RECON_PROF_S);
        RC_CUDA(recon::launch_weight_S(sv.d, sv.tw, w.dsum, w.Z, S_new, c->stream));
    }
    return cg_block(c, sv.d, sv.tw, w, sv.masks, S_old, S_new, (float)sv.prm->lambda, sv.x, n == 0,
                    sv.prm->cg);
}

// Capture body of a lockstep batch (slot 0 active and capturing): every solve runs on its own
// slot stream; per IRLS iteration the solves' Grams join on their group leader's stream for the
// shared weight launches, then fork back for the summed diagonals, S(r) and CG. With several
// groups the weight launches take turns (each waits for the previous group's), so that the FP64
// launches of one group overlap the other groups' CG instead of each other.
int batch_capture(recon_ctx* c, std::vector<Solve>& sv, int group) {
    const int n = (int)sv.size();
    const int ngroups = (n + group - 1) / group;
    cudaEvent_t ev_start = c->batch_ev[0], ev_tok = c->batch_ev[1];
    auto ev = [&](int i) { return c->batch_ev[2 + i]; };
    RC_CUDA(cudaEventRecord(ev_start, c->stream));
    int rc = RECON_OK;
    for (int i = 1; i < n && !rc; ++i) {
        rc = select_slot(c, i);
        if (!rc) RC_CUDA(cudaStreamWaitEvent(c->stream, ev_start, 0));
    }
    for (int i = 0; i < n && !rc; ++i) {
        rc = select_slot(c, i);
        if (!rc) rc = solve_begin(c, &sv[i]);
    }
    bool tok = false;
    for (int it = 0; it < sv[0].prm->irls && !rc; ++it) {
        for (int i = 0; i < n && !rc; ++i) {
            rc = select_slot(c, i);
            if (!rc) rc = iter_gram(c, sv[i]);
            if (!rc) RC_CUDA(cudaEventRecord(ev(i), c->stream));
        }
        for (int g0 = 0; g0 < n && !rc; g0 += group) {
            const int cnt = std::min(group, n - g0);
            rc = select_slot(c, g0);
            for (int i = g0 + 1; i < g0 + cnt && !rc; ++i)
                RC_CUDA(cudaStreamWaitEvent(c->stream, ev(i), 0));
            if (!rc && tok) RC_CUDA(cudaStreamWaitEvent(c->stream, ev_tok, 0));
            if (!rc) rc = group_weight(c, &sv[g0], cnt, it);
            if (!rc) RC_CUDA(cudaEventRecord(ev(g0), c->stream));
            if (!rc && ngroups > 1) {
                RC_CUDA(cudaEventRecord(ev_tok, c->stream));
                tok = true;
            }
            for (int i = g0; i < g0 + cnt && !rc; ++i) {
                rc = select_slot(c, i);
                if (!rc && i != g0) RC_CUDA(cudaStreamWaitEvent(c->stream, ev(g0), 0));
                if (!rc) rc = iter_post_weight(c, sv[i], it);
            }
        }
    }
    for (int i = 1; i < n && !rc; ++i) {
        rc = select_slot(c, i);
        if (!rc) RC_CUDA(cudaEventRecord(ev(i), c->stream));
        if (!rc) rc = select_slot(c, 0);
        if (!rc) RC_CUDA(cudaStreamWaitEvent(c->stream, ev(i), 0));
    }
    return rc;
}

// Enqueue a lockstep batch on slot 0's stream as one replay of its captured graph (captured on
// first use, cached while every solve's key, the group size and the slots' workspaces stay).
int batch_enqueue_lockstep(recon_ctx* c, std::vector<Solve>& sv, int group) {
    const int n = (int)sv.size();
    std::vector<unsigned char> key(sizeof(int) * 2);
    std::memcpy(key.data(), &n, sizeof(int));
    std::memcpy(key.data() + sizeof(int), &group, sizeof(int));
    for (int i = 0; i < n; ++i) {
        int rc = select_slot(c, i);
        if (rc) return rc;
        const recon_ctx::GraphKey k = graph_key(c, sv[i]);
        const unsigned char* kb = reinterpret_cast<const unsigned char*>(&k);
        key.insert(key.end(), kb, kb + sizeof(k));
    }
    int rc = select_slot(c, 0);
    if (rc) return rc;
    if (!c->batch_gexec || key != c->batch_key) {
        if (c->batch_gexec) {
            cudaGraphExecDestroy(c->batch_gexec);
            c->batch_gexec = nullptr;
        }
        while ((int)c->batch_ev.size() < RECON_MAX_BATCH + 2) {
            cudaEvent_t e;
            RC_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            c->batch_ev.push_back(e);
        }
        delete c->batch_gprof;
        c->batch_gprof = c->prof ? new GraphProf() : nullptr;
        c->capturing = c->batch_gprof;
        RC_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed));
        rc = batch_capture(c, sv, group);
        const int rc0 = select_slot(c, 0);
        cudaGraph_t g = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(c->stream, &g);
        c->capturing = nullptr;
        if (!rc) rc = rc0;
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (ec != cudaSuccess) return cuda_fail(c, ec, "cudaStreamEndCapture");
        const cudaError_t ei = cudaGraphInstantiate(&c->batch_gexec, g, 0);
        cudaGraphDestroy(g);
        if (ei != cudaSuccess) {
            c->batch_gexec = nullptr;
            return cuda_fail(c, ei, "cudaGraphInstantiate");
        }
        c->batch_key = key;
    }
    RC_CUDA(cudaGraphLaunch(c->batch_gexec, c->stream));
    if (c->batch_gprof) ++c->batch_gprof->replays;
    return RECON_OK;
}

// After the slot's stream finished: status flags, finite residual and eps.
int solve_check(recon_ctx* c, Solve& sv);
int solve_check(recon_ctx* c, Solve& sv) {
    int rc = check_status(c, sv.w, sv.prm->irls);
    if (rc) return rc;
    if (sv.prm->irls > 0) {
        double rr = 0.0, eps = 0.0;
        RC_CUDA(cudaMemcpy(&rr, sv.w.rr + sv.prm->cg, sizeof(double), cudaMemcpyDeviceToHost));
        RC_CUDA(cudaMemcpy(&eps, sv.w.eps, sizeof(double), cudaMemcpyDeviceToHost));
        if (!std::isfinite(rr) || !std::isfinite(eps))
            return fail(c, RECON_ENUMERIC, "non-finite residual or eps in the iteration");
    }
    return RECON_OK;
}

}  // namespace

// One asynchronous request in flight on slot `slot`.
struct recon_ctx::Pending {
    int slot = 0;
    bool busy = false;
    recon_params prm = {};
    Solve sv;
    cudaEvent_t done = nullptr;
};

namespace {

// Free the workspaces of serving slots that have nothing in flight (memory-based admission).
void release_idle(recon_ctx* c) {
    for (size_t k = 0; k < c->pending.size(); ++k) {
        recon_ctx::Pending* pd = c->pending[k];
        if (!pd || pd->busy) continue;
        const int i = pd->slot;
        if (i == c->active || i >= (int)c->slots.size()) continue;
        auto& sl = c->slots[i];
        for (auto& kv : sl.bufs)
            if (kv.second.ptr) {
                cudaFree(kv.second.ptr);
                c->allocated -= kv.second.bytes;
            }
        sl.bufs.clear();
        ++sl.ws_gen;
    }
}

}  // namespace

namespace {

size_t bytes_needed(const Dims& d) {
    if (d.T <= 0 || d.P <= 0 || d.Q <= 0 || d.R <= 0 || d.M <= 0 || d.N1 <= 0 || d.N2 <= 0 ||
        d.N3 <= 0)
        return 0;
    const size_t vec = d.elems() * sizeof(float2);
    const size_t s = d.s();
    const size_t nlag = d.nlag();
    size_t b = 3 * vec + 2 * (size_t)d.npair() * d.pixels() * sizeof(float2);
    b += s * s * sizeof(double2) * 3 + s * sizeof(double);  // G + eigensolver work (estimate)
    b += recon::gram_scratch_bytes(d, recon::gram_blocks(d)) + recon::diag_scratch_bytes(d) +
         2 * nlag * sizeof(double2) + recon::s_scratch_bytes(d);
    b += (size_t)(recon::max_parts() + 512) * sizeof(double);
    return b;
}

// A solve that fails part-way through being enqueued may have work queued on the active slot's
// stream that still writes the caller's buffers: wait for it before the error is returned (the
// error stays the one reported).
int drain_on_fail(recon_ctx* c, int rc) {
    if (rc) cudaStreamSynchronize(c->stream);
    return rc;
}

int solve_impl(recon_ctx* c, const Dims& d, const void* kspace, const uint8_t* masks,
               const recon_params* prm, void* image_out, int variant = RECON_VARIANT_PROPOSED) {
    int rc = set_device(c);
    if (rc) return rc;
    rc = select_slot(c, 0);
    if (rc) return rc;
    Solve sv;
    rc = solve_prepare(c, d, kspace, masks, prm, image_out, &sv);
    if (rc) return drain_on_fail(c, rc);
    if (variant == RECON_VARIANT_HLR_VOXEL) {
        rc = prepare_voxel(c, &sv);
        if (rc) return drain_on_fail(c, rc);
    }
    rc = solve_enqueue_all(c, sv);
    if (rc) return drain_on_fail(c, rc);
    RC_CUDA(cudaStreamSynchronize(c->stream));
    return solve_check(c, sv);
}

// ---- IRLS-direct (Sec. IV-A): the exact valid lifting, explicit, with library GEMMs ----

int ensure_blas(recon_ctx* c) {
    if (!c->blas && cublasCreate(&c->blas) != CUBLAS_STATUS_SUCCESS) {
        c->blas = nullptr;
        return fail(c, RECON_ECUDA, "cublasCreate failed");
    }
    if (cublasSetStream(c->blas, c->stream) != CUBLAS_STATUS_SUCCESS)
        return fail(c, RECON_ECUDA, "cublasSetStream failed");
    return RECON_OK;
}

#define RC_BLAS(call)                                                          \
    do {                                                                       \
        if ((call) != CUBLAS_STATUS_SUCCESS) return fail(c, RECON_ECUDA, #call); \
    } while (0)

// Buffers of the direct variant (slot 0).
struct DirectWork {
    float2 *yh, *z, *h32, *hd32;
    double2 *H, *Hold;
    void* lift;  // rows x s complex128 for the Gram, or two rows x s complex64 (lifting, product)
};

int get_direct_work(recon_ctx* c, const Dims& d, DirectWork* dw) {
    void* ptr;
    int rc;
    const size_t vec = d.elems() * sizeof(float2);
    const size_t ss = (size_t)d.s() * d.s();
#define GETD(name, bytes, field, type)    \
    rc = ensure(c, name, (bytes), &ptr); \
    if (rc) return rc;                   \
    dw->field = reinterpret_cast<type>(ptr);
    GETD("d_yh", vec, yh, float2*);
    GETD("d_z", vec, z, float2*);
    GETD("d_h32", ss * sizeof(float2), h32, float2*);
    GETD("d_hd32", ss * sizeof(float2), hd32, float2*);
    GETD("d_H", ss * sizeof(double2), H, double2*);
    GETD("d_Hold", ss * sizeof(double2), Hold, double2*);
    GETD("d_lift", recon::direct_rows(d) * d.s() * sizeof(double2), lift, void*);
#undef GETD
    return RECON_OK;
}

// G = T^H T of the exact lifting of F x (lower triangle by the library rank-k product, then the
// upper triangle filled).
int direct_gram(recon_ctx* c, const Dims& d, const Twiddles& tw, DirectWork& dw, const float2* x,
                double2* G) {
    const int s = d.s();
    const long long m = (long long)recon::direct_rows(d);
    RC_CUDA(recon::launch_fft2(d, tw, x, dw.yh, 0, c->stream));
    RC_CUDA(recon::launch_direct_lift(d, dw.yh, dw.lift, 1, c->stream));
    const double one = 1.0, zero = 0.0;
    RC_BLAS(cublasZherk(c->blas, CUBLAS_FILL_MODE_LOWER, CUBLAS_OP_C, s, (int)m, &one,
                        reinterpret_cast<const cuDoubleComplex*>(dw.lift), (int)m, &zero,
                        reinterpret_cast<cuDoubleComplex*>(G), s));
    RC_CUDA(recon::launch_herm_fill(G, s, c->stream));
    return RECON_OK;
}

// out = F^H( mask * F v + lam T^*(T(F v) h) ), h complex64 s x s; mask = NULL drops the data term.
int direct_op(recon_ctx* c, const Dims& d, const Twiddles& tw, DirectWork& dw, const float2* v,
              const float2* h, const uint8_t* mask, float lam, float2* out) {
    const int s = d.s();
    const long long m = (long long)recon::direct_rows(d);
    float2* Tm = reinterpret_cast<float2*>(dw.lift);
    float2* Y = Tm + (size_t)m * s;
    RC_CUDA(recon::launch_fft2(d, tw, v, dw.yh, 0, c->stream));
    RC_CUDA(recon::launch_direct_lift(d, dw.yh, Tm, 0, c->stream));
    const cuComplex one = make_cuComplex(1.f, 0.f), zero = make_cuComplex(0.f, 0.f);
    RC_BLAS(cublasCgemm(c->blas, CUBLAS_OP_N, CUBLAS_OP_N, (int)m, s, s, &one,
                        reinterpret_cast<const cuComplex*>(Tm), (int)m,
                        reinterpret_cast<const cuComplex*>(h), s, &zero,
                        reinterpret_cast<cuComplex*>(Y), (int)m));
    RC_CUDA(recon::launch_direct_unlift(d, Y, dw.yh, mask, lam, dw.z, c->stream));
    RC_CUDA(recon::launch_fft2(d, tw, dw.z, out, 1, c->stream));
    return RECON_OK;
}

// H = (G + eps I)^(p/2-1) into dw.H from G (consumed). eps: the Sec. III-C schedule (first:
// eps0_frac * lambda_max, else eps / gamma) unless eps_set.
int direct_weight(recon_ctx* c, const Dims& d, Work& w, DirectWork& dw, double p, int first,
                  double frac, double gamma, int eps_set, double eps_value, int it) {
    const int s = d.s();
    const size_t gbytes = (size_t)s * s * sizeof(double2);
    if (eps_set)
        RC_CUDA(cudaMemcpyAsync(w.eps, &eps_value, sizeof(double), cudaMemcpyHostToDevice, c->stream));
    if (w.use_eig) {
        int rc = run_eig(c, s, w, w.info + it);
        if (rc) return rc;
        if (!eps_set) RC_CUDA(recon::launch_eps(w.evals + s - 1, w.eps, first, frac, gamma, c->stream));
        RC_CUDA(recon::launch_form_H(w.G, w.evals, w.eps, p, s, dw.H, c->stream));
    } else {
        if (!eps_set) {
            if (first)
                RC_CUDA(recon::launch_lanczos_lmax(d, w.G, w.lanc, w.lmax, w.kerr + 2 * it + 1, c->stream,
                                                   w.fault));
            RC_CUDA(recon::launch_eps(w.lmax, w.eps, first, frac, gamma, c->stream));
        }
        RC_CUDA(recon::launch_hpd_inverse(d, w.G, w.eps, w.hpd, w.kerr + 2 * it, c->stream));
        RC_CUDA(cudaMemcpyAsync(dw.H, w.G, gbytes, cudaMemcpyDeviceToDevice, c->stream));
    }
    return RECON_OK;
}

int direct_prepare(recon_ctx* c, const Dims& d, const recon_params* prm, int n_cg, Twiddles* tw,
                   Work* w, DirectWork* dw) {
    int rc = set_device(c);
    if (rc) return rc;
    rc = get_twiddles(c, d, tw);
    if (rc) return rc;
    rc = ensure_blas(c);
    if (rc) return rc;
    const bool eig = prm ? wants_eig(prm->p, prm->weight_method) : false;
    if (eig) {
        rc = ensure_solver(c);
        if (rc) return rc;
    }
    rc = get_work(c, d, n_cg, prm ? prm->irls : 1, true, eig, w);
    if (rc) return rc;
    return get_direct_work(c, d, dw);
}

// Algorithm 1 with the exact lifting: x0 = A^H b; per iteration the Gram, the weight H, the
// carried residual r += lam W_{H_old - H_new} x (r0 = -lam W x0), n_cg plain CG steps.
int solve_direct(recon_ctx* c, const Dims& d, const void* kspace, const uint8_t* masks,
                 const recon_params* prm, void* image_out) {
    Twiddles tw;
    Work w;
    DirectWork dw;
    int rc = direct_prepare(c, d, prm, prm->cg, &tw, &w, &dw);
    if (rc) return rc;
    rc = reset_status(c, w);
    if (rc) return rc;
    float2* x = reinterpret_cast<float2*>(image_out);
    const size_t n = d.elems();
    const size_t ss = (size_t)d.s() * d.s();
    const float lam = (float)prm->lambda;
    const recon::RedSlot rs{w.parts, w.counter};
    RC_CUDA(recon::launch_adjoint(d, tw, kspace, prm->kspace_bf16, masks, w.t, x, c->stream));
    for (int it = 0; it < prm->irls; ++it) {
        rc = direct_gram(c, d, tw, dw, x, w.G);
        if (rc) return rc;
        rc = direct_weight(c, d, w, dw, prm->p, it == 0, prm->eps0_frac, prm->gamma, 0, 0.0, it);
        if (rc) return rc;
        RC_CUDA(recon::launch_h_delta(dw.H, it == 0 ? nullptr : dw.Hold, dw.hd32, dw.h32, ss,
                                      c->stream));
        RC_CUDA(cudaMemcpyAsync(dw.Hold, dw.H, ss * sizeof(double2), cudaMemcpyDeviceToDevice,
                                c->stream));
        // residual carry: r = (first ? 0 : r) + lam W_{H_old - H_new} x
        rc = direct_op(c, d, tw, dw, x, dw.hd32, nullptr, lam, w.t);
        if (rc) return rc;
        RC_CUDA(recon::launch_dcg_resid(w.r, w.t, it == 0, n, rs, w.rr, c->stream));
        for (int k = 0; k < prm->cg; ++k) {
            RC_CUDA(recon::launch_dcg_pupdate(w.p, w.r, n, w.rr + k, k > 0 ? w.rr + k - 1 : w.rr,
                                              k == 0, c->stream));
            rc = direct_op(c, d, tw, dw, w.p, dw.h32, masks, lam, w.t);
            if (rc) return rc;
            RC_CUDA(recon::launch_dcg_dot(w.p, w.t, n, rs, w.pq + k, c->stream));
            RC_CUDA(recon::launch_dcg_update(x, w.r, w.p, w.t, n, w.rr + k, w.pq + k, rs,
                                             w.rr + k + 1, c->stream));
        }
    }
    RC_CUDA(cudaStreamSynchronize(c->stream));
    rc = check_status(c, w, prm->irls);
    if (rc) return rc;
    if (prm->irls > 0) {
        double rr = 0.0;
        RC_CUDA(cudaMemcpy(&rr, w.rr + prm->cg, sizeof(double), cudaMemcpyDeviceToHost));
        if (!std::isfinite(rr)) return fail(c, RECON_ENUMERIC, "non-finite residual in the iteration");
    }
    return RECON_OK;
}

int adjoint_impl(recon_ctx* c, const Dims& d, const void* kspace, int kspace_bf16,
                 const uint8_t* masks, void* x_out) {
    int rc = set_device(c);
    if (rc) return rc;
    Twiddles tw;
    rc = get_twiddles(c, d, &tw);
    if (rc) return rc;
    void* t;
    rc = ensure(c, "t", d.elems() * sizeof(float2), &t);
    if (rc) return rc;
    RC_CUDA(recon::launch_adjoint(d, tw, kspace, kspace_bf16, masks, (float2*)t, (float2*)x_out,
                                  c->stream));
    RC_CUDA(cudaStreamSynchronize(c->stream));
    return RECON_OK;
}

int fft_impl(recon_ctx* c, const Dims& d, const void* x, void* y, int inverse) {
    int rc = set_device(c);
    if (rc) return rc;
    Twiddles tw;
    rc = get_twiddles(c, d, &tw);
    if (rc) return rc;
    RC_CUDA(recon::launch_fft2(d, tw, (const float2*)x, (float2*)y, inverse, c->stream));
    RC_CUDA(cudaStreamSynchronize(c->stream));
    return RECON_OK;
}

int gram_impl(recon_ctx* c, const Dims& d, const void* x, void* G_out, void* lags_out) {
    int rc = set_device(c);
    if (rc) return rc;
    Twiddles tw;
    rc = get_twiddles(c, d, &tw);
    if (rc) return rc;
    void* lp;
    const int nb = recon::gram_blocks(d);
    rc = ensure(c, "lag_part", recon::gram_scratch_bytes(d, nb), &lp);
    if (rc) return rc;
    RC_CUDA(recon::launch_gram(d, tw, (const float2*)x, (double2*)lp, nb, (double2*)lags_out,
                               (double2*)G_out, c->stream));
    RC_CUDA(cudaStreamSynchronize(c->stream));
    return RECON_OK;
}

int weight_impl(recon_ctx* c, const Dims& d, const void* G_in, double eps_in, double p,
                int method, void* S_out, void* dsum_out, void* evals_out, double* eps_out) {
    int rc = set_device(c);
    if (rc) return rc;
    Twiddles tw;
    rc = get_twiddles(c, d, &tw);
    if (rc) return rc;
    Work w;
    rc = get_work(c, d, 1, 1, false, wants_eig(p, method), &w);
    if (rc) return rc;
    rc = reset_status(c, w);
    if (rc) return rc;
    const size_t gbytes = (size_t)d.s() * d.s() * sizeof(double2);
    RC_CUDA(cudaMemcpyAsync(w.G, G_in, gbytes, cudaMemcpyDeviceToDevice, c->stream));
    const bool set = eps_in >= 0.0;
    rc = weight_step(c, d, tw, w, p, 1, set ? 0.0 : -eps_in, 1.0, set, eps_in, (float2*)S_out, 0);
    if (rc) return rc;
    if (dsum_out)
        RC_CUDA(cudaMemcpyAsync(dsum_out, w.dsum, d.nlag() * sizeof(double2),
                                cudaMemcpyDeviceToDevice, c->stream));
    if (evals_out)
        RC_CUDA(cudaMemcpyAsync(evals_out, w.evals, (size_t)d.s() * sizeof(double),
                                cudaMemcpyDeviceToDevice, c->stream));
    RC_CUDA(cudaStreamSynchronize(c->stream));
    rc = check_status(c, w, 1);
    if (rc) return rc;
    if (eps_out) RC_CUDA(cudaMemcpy(eps_out, w.eps, sizeof(double), cudaMemcpyDeviceToHost));
    return RECON_OK;
}

int weight_args(recon_ctx* c, const void* G_in, double eps_in, double p, int method,
                const void* S_out, const void* evals_out) {
    if (!G_in || !S_out) return fail(c, RECON_EINVAL, "null pointer");
    if (misaligned({G_in, S_out})) return fail(c, RECON_EINVAL, kAlignMsg);
    if (method != RECON_WEIGHT_AUTO && method != RECON_WEIGHT_EIG)
        return fail(c, RECON_EINVAL, "unknown weight method");
    if (evals_out && !wants_eig(p, method))
        return fail(c, RECON_EINVAL, "eigenvalues are only formed by RECON_WEIGHT_EIG or p > 0");
    if (!std::isfinite(eps_in) || !(p >= 0.0 && p <= 1.0)) return fail(c, RECON_EINVAL, "bad eps or p");
    return RECON_OK;
}

int apply_normal_impl(recon_ctx* c, const Dims& d0, const uint8_t* masks, const void* S,
                      double lambda, const void* x, void* y) {
    Dims d = d0;
    if (c->fft_sched >= 0) d.colS = d.depthS = c->fft_sched;  // forced radix schedule (tests)
    int rc;
    rc = set_device(c);
    if (rc) return rc;
    Twiddles tw;
    rc = get_twiddles(c, d, &tw);
    if (rc) return rc;
    void *pp, *parts;
    rc = ensure(c, "p", d.elems() * sizeof(float2), &pp);
    if (rc) return rc;
    rc = ensure(c, "parts", (size_t)recon::max_parts() * sizeof(double), &parts);
    if (rc) return rc;
    recon::Partials pq{(double*)parts, 0};
    const recon::Partials none{nullptr, 0};
    // the CG operator passes with first = 1 (p = x); y receives (A^H A + lambda W) x
    RC_CUDA(recon::launch_row_fwd_pupdate(d, tw, (const float2*)x, (float2*)pp, (float2*)y, none,
                                          nullptr, nullptr, 1, c->stream));
    RC_CUDA(recon::launch_col_mask(d, tw, (float2*)y, masks, c->stream));
    RC_CUDA(recon::launch_row_inv_w(d, tw, (float2*)y, (const float2*)pp, (const float2*)S,
                                    (float)lambda, &pq, c->stream));
    RC_CUDA(cudaStreamSynchronize(c->stream));
    return RECON_OK;
}

int check_variant(recon_ctx* c, int variant, const recon_filter& f) {
    if (variant < RECON_VARIANT_PROPOSED || variant > RECON_VARIANT_DIRECT)
        return fail(c, RECON_EINVAL, "unknown variant");
    if (variant == RECON_VARIANT_HLR_VOXEL && (f.N1 != 1 || f.N2 != 1))
        return fail(c, RECON_EINVAL, "HLR-Voxel has no spatial taps: need N1 = N2 = 1");
    return RECON_OK;
}

}  // namespace

extern "C" {

int recon_create(recon_ctx** out, int device, size_t mem_budget_bytes, void* cuda_stream) {
    if (!out) return RECON_EINVAL;
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || device < 0 || device >= ndev) {
        g_create_error = "no such CUDA device";
        return RECON_ECUDA;
    }
    recon_ctx* c = new recon_ctx();
    c->device = device;
    c->budget = mem_budget_bytes;
    if (cudaSetDevice(device) != cudaSuccess) {
        g_create_error = "cudaSetDevice failed";
        delete c;
        return RECON_ECUDA;
    }
    if (cuda_stream) {
        c->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            g_create_error = "cudaStreamCreate failed";
            delete c;
            return RECON_ECUDA;
        }
        c->own_stream = true;
    }
    if (cusolverDnCreate(&c->solver) != CUSOLVER_STATUS_SUCCESS ||
        cusolverDnSetStream(c->solver, c->stream) != CUSOLVER_STATUS_SUCCESS) {
        g_create_error = "cusolverDnCreate failed";
        if (c->own_stream) cudaStreamDestroy(c->stream);
        delete c;
        return RECON_ECUDA;
    }
    *out = c;
    return RECON_OK;
}

void recon_destroy(recon_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    select_slot(c, 0);
    for (auto& sl : c->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.gexec) cudaGraphExecDestroy(sl.gexec);
        delete sl.gprof;
        for (auto& kv : sl.bufs)
            if (kv.second.ptr) cudaFree(kv.second.ptr);
        if (sl.solver) cusolverDnDestroy(sl.solver);
        if (sl.own_stream && sl.stream) cudaStreamDestroy(sl.stream);
    }
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (auto& kv : c->bufs)
        if (kv.second.ptr) cudaFree(kv.second.ptr);
    for (auto& kv : c->tw) {
        cudaFree(kv.second.f);
        cudaFree(kv.second.d);
    }
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    for (auto* pd : c->pending) {
        if (pd && pd->done) cudaEventDestroy(pd->done);
        delete pd;
    }
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    delete c->gprof;
    if (c->batch_gexec) cudaGraphExecDestroy(c->batch_gexec);
    delete c->batch_gprof;
    for (cudaEvent_t e : c->batch_ev) cudaEventDestroy(e);
    if (c->solver) cusolverDnDestroy(c->solver);
    if (c->blas) cublasDestroy(c->blas);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
}

const char* recon_last_error(const recon_ctx* c) {
    if (!c) return g_create_error.c_str();
    return c->err.c_str();
}

size_t recon_bytes_needed(recon_dims dd, recon_filter f, int kspace_bf16) {
    (void)kspace_bf16;  // k-space stays in the caller's buffer
    Dims d{dd.T, dd.P, dd.Q, f.N1, f.N2, f.M};
    return bytes_needed(d);
}

size_t recon_bytes_needed3(recon_dims3 dd, recon_filter3 f, int kspace_bf16) {
    (void)kspace_bf16;
    Dims d{dd.T, dd.P, dd.Q, f.N1, f.N2, f.M};
    d.R = dd.R;
    d.N3 = f.N3;
    return bytes_needed(d);
}

int recon_solve(recon_ctx* c, recon_dims dd, const void* kspace, const uint8_t* masks,
                recon_filter f, const recon_params* prm, void* image_out) {
    if (!c) return RECON_EINVAL;
    if (!kspace || !masks || !prm || !image_out) return fail(c, RECON_EINVAL, "null pointer");
    if (misaligned({kspace, masks, image_out})) return fail(c, RECON_EINVAL, kAlignMsg);
    Dims d;
    int rc = check_params(c, dd, f, prm, &d);
    if (rc) return rc;
    return solve_impl(c, d, kspace, masks, prm, image_out);
}

int recon_solve3(recon_ctx* c, recon_dims3 dd, const void* kspace, const uint8_t* masks,
                 recon_filter3 f, const recon_params* prm, void* image_out) {
    if (!c) return RECON_EINVAL;
    if (!kspace || !masks || !prm || !image_out) return fail(c, RECON_EINVAL, "null pointer");
    if (misaligned({kspace, masks, image_out})) return fail(c, RECON_EINVAL, kAlignMsg);
    Dims d;
    int rc = check_dims3(c, dd, &f, &d);
    if (!rc) rc = check_prm(c, prm);
    if (rc) return rc;
    return solve_impl(c, d, kspace, masks, prm, image_out);
}

int recon_solve_coils(recon_ctx* c, recon_dims dd, const void* kspace, const uint8_t* masks,
                      const void* coils, int n_coils, recon_filter f, const recon_params* prm,
                      void* image_out) {
    if (!c) return RECON_EINVAL;
    if (!kspace || !masks || !coils || !prm || !image_out) return fail(c, RECON_EINVAL, "null pointer");
    if (misaligned({kspace, masks, coils, image_out})) return fail(c, RECON_EINVAL, kAlignMsg);
    if (n_coils < 1 || n_coils > RECON_MAX_COILS)
        return fail(c, RECON_EINVAL, "need 1 <= n_coils <= RECON_MAX_COILS");
    if (prm->kspace_bf16) return fail(c, RECON_EINVAL, "multi-coil k-space must be complex64");
    Dims d;
    int rc = check_params(c, dd, f, prm, &d);
    if (rc) return rc;
    d.nc = n_coils;
    rc = set_device(c);
    if (rc) return rc;
    rc = select_slot(c, 0);
    if (rc) return rc;
    Solve sv;
    rc = solve_prepare(c, d, kspace, masks, prm, image_out, &sv);
    if (rc) return drain_on_fail(c, rc);
    sv.coils = reinterpret_cast<const float2*>(coils);
    if (n_coils == 1) {  // unit modulus (to FP32 rounding) keeps A A^H a projection
        void* dev = nullptr;
        rc = ensure(c, "coildev", 256, &dev);
        if (rc) return rc;
        RC_CUDA(recon::launch_coil_unimodular(d, sv.coils, (unsigned int*)dev, c->stream));
        unsigned int bits = 0;
        RC_CUDA(cudaMemcpyAsync(&bits, dev, sizeof(bits), cudaMemcpyDeviceToHost, c->stream));
        RC_CUDA(cudaStreamSynchronize(c->stream));
        float m;
        std::memcpy(&m, &bits, sizeof(m));
        sv.coil_proj = m <= 1e-6f;
    }
    rc = solve_enqueue_all(c, sv);
    if (rc) return drain_on_fail(c, rc);
    RC_CUDA(cudaStreamSynchronize(c->stream));
    return solve_check(c, sv);
}

int recon_adjoint_coils(recon_ctx* c, recon_dims dd, const void* kspace, const uint8_t* masks,
                        const void* coils, int n_coils, void* x_out) {
    if (!c) return RECON_EINVAL;
    if (!kspace || !masks || !coils || !x_out) return fail(c, RECON_EINVAL, "null pointer");
    if (misaligned({kspace, masks, coils, x_out})) return fail(c, RECON_EINVAL, kAlignMsg);
    if (n_coils < 1 || n_coils > RECON_MAX_COILS)
        return fail(c, RECON_EINVAL, "need 1 <= n_coils <= RECON_MAX_COILS");
    Dims d;
    int rc = check_dims(c, dd, nullptr, &d);
    if (rc) return rc;
    d.nc = n_coils;
    rc = set_device(c);
    if (rc) return rc;
    Twiddles tw;
    rc = get_twiddles(c, d, &tw);
    if (rc) return rc;
    void* t;
    rc = ensure(c, "t", d.elems() * (size_t)d.nc * sizeof(float2), &t);
    if (rc) return rc;
    RC_CUDA(recon::launch_adjoint_coils_cols(d, tw, kspace, masks, (float2*)t, c->stream));
    RC_CUDA(recon::launch_coil_combine(d, tw, (float2*)t, (const float2*)coils, (float2*)x_out,
                                       c->stream));
    RC_CUDA(cudaStreamSynchronize(c->stream));
    return RECON_OK;
}

int recon_apply_normal_coils(recon_ctx* c, recon_dims dd, recon_filter f, const uint8_t* masks,
                             const void* coils, int n_coils, const void* S, double lambda,
                             const void* x, void* y) {
    if (!c) return RECON_EINVAL;
    if (!masks || !coils || !S || !x || !y) return fail(c, RECON_EINVAL, "null pointer");
    if (misaligned({masks, coils, S, x, y})) return fail(c, RECON_EINVAL, kAlignMsg);
    if (x == y) return fail(c, RECON_EINVAL, "y must not alias x");
    if (n_coils < 1 || n_coils > RECON_MAX_COILS)
        return fail(c, RECON_EINVAL, "need 1 <= n_coils <= RECON_MAX_COILS");
    Dims d;
    int rc = check_dims(c, dd, &f, &d);
    if (rc) return rc;
    d.nc = n_coils;
    rc = set_device(c);
    if (rc) return rc;
    Twiddles tw;
    rc = get_twiddles(c, d, &tw);
    if (rc) return rc;
    void *pp, *t, *parts;
    rc = ensure(c, "p", d.elems() * sizeof(float2), &pp);
    if (rc) return rc;
    rc = ensure(c, "t", d.elems() * (size_t)d.nc * sizeof(float2), &t);
    if (rc) return rc;
    rc = ensure(c, "parts", (size_t)recon::max_parts() * sizeof(double), &parts);
    if (rc) return rc;
    recon::Partials pq{(double*)parts, 0};
    const recon::Partials none{nullptr, 0};
    // the coil passes with first = 1 (p = x); q lands in coil 0's plane of t
    RC_CUDA(recon::launch_coil_row_fwd(d, tw, (const float2*)x, (float2*)pp, (float2*)t,
                                       (const float2*)coils, none, nullptr, nullptr, 1, c->stream));
    RC_CUDA(recon::launch_col_mask(d, tw, (float2*)t, masks, c->stream));
    RC_CUDA(recon::launch_coil_row_inv_w(d, tw, (float2*)t, (const float2*)pp, (const float2*)coils,
                                         (const float2*)S, (float)lambda, &pq, c->stream));
    RC_CUDA(cudaMemcpyAsync(y, t, d.elems() * sizeof(float2), cudaMemcpyDeviceToDevice, c->stream));
    RC_CUDA(cudaStreamSynchronize(c->stream));
    return RECON_OK;
}

namespace {

// n solves with their own geometry (dims[i]) and shared parameters: independent slots (each its
// own stream, workspace and graph), or lockstep groups sharing their weight launches
// (RECON_OPT_BATCH_GROUP), or direct launches (graphs off / eigensolver path). Arguments checked
// by the callers.
// host_io: kspace, masks and image_out are host pointers; slot i copies its inputs into device
// buffers of its own workspace on its own stream before its solve and its image back after it,
// so that one slot's copies overlap the other slots' work (one cudaMemcpyAsync per buffer).
int solve_many_impl(recon_ctx* c, int n, const Dims* dims, const void* const* kspace,
                    const uint8_t* const* masks, const recon_params* prm, void* const* image_out,
                    bool host_io = false) {
    int rc = set_device(c);
    if (rc) return rc;
    rc = select_slot(c, 0);
    if (rc) return rc;
    std::vector<void*> out_dev(n, nullptr);
    auto image_bytes = [&](int i) { return dims[i].elems() * sizeof(float2); };
    // slot streams start after the work already queued on the context's stream
    cudaEvent_t start = nullptr;
    RC_CUDA(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
    std::vector<cudaEvent_t> done(n, nullptr);
    auto cleanup = [&]() {
        select_slot(c, 0);
        cudaEventDestroy(start);
        for (cudaEvent_t e : done)
            if (e) cudaEventDestroy(e);
    };
    std::vector<Solve> sv(n);
    rc = RECON_OK;
    cudaError_t e = cudaEventRecord(start, c->stream);
    const bool direct = !c->graphs || wants_eig(prm->p, prm->weight_method);
    // lockstep: one graph over all slots, the weight steps of each group of solves in shared
    // launches (p = 0 sweep path, more than one solve, no test hook pending)
    const bool lockstep = !direct && c->batch_group > 0 && n > 1 && !c->withhold_arrival &&
                          !c->inject_barrier_fault;
    for (int i = 0; i < n && !rc && e == cudaSuccess; ++i) {
        rc = select_slot(c, i);
        if (!rc) e = cudaStreamWaitEvent(c->stream, start, 0);
        const void* kd = kspace[i];
        const uint8_t* md = masks[i];
        void* od = image_out[i];
        if (host_io && !rc && e == cudaSuccess) {
            const size_t ne = dims[i].elems();
            const size_t kb = ne * (prm->kspace_bf16 ? 4 : 8);
            void *kdev = nullptr, *mdev = nullptr;
            rc = ensure(c, "io_kspace", kb, &kdev);
            if (!rc) rc = ensure(c, "io_masks", ne, &mdev);
            if (!rc) rc = ensure(c, "io_image", image_bytes(i), &out_dev[i]);
            if (!rc) e = cudaMemcpyAsync(kdev, kspace[i], kb, cudaMemcpyHostToDevice, c->stream);
            if (!rc && e == cudaSuccess)
                e = cudaMemcpyAsync(mdev, masks[i], ne, cudaMemcpyHostToDevice, c->stream);
            kd = kdev;
            md = reinterpret_cast<const uint8_t*>(mdev);
            od = out_dev[i];
        }
        if (!rc && e == cudaSuccess) rc = solve_prepare(c, dims[i], kd, md, prm, od, &sv[i]);
        if (!rc && e == cudaSuccess && !direct && !lockstep) rc = solve_enqueue_all(c, sv[i]);
        if (!rc && e == cudaSuccess && direct) rc = solve_begin(c, &sv[i]);
        // the set-up work of the slot (workspace clears, tuning) precedes the lockstep graph
        if (!rc && e == cudaSuccess && lockstep && i > 0) {
            e = cudaEventCreateWithFlags(&done[i], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventRecord(done[i], c->stream);
        }
    }
    if (lockstep && !rc && e == cudaSuccess) {
        rc = select_slot(c, 0);
        for (int i = 1; i < n && !rc && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(c->stream, done[i], 0);
        if (!rc && e == cudaSuccess) rc = batch_enqueue_lockstep(c, sv, c->batch_group);
        for (int i = 0; host_io && i < n && !rc && e == cudaSuccess; ++i)
            e = cudaMemcpyAsync(image_out[i], out_dev[i], image_bytes(i), cudaMemcpyDeviceToHost,
                                c->stream);
    }
    // direct launches: iterations interleaved over the slots so that every stream has work
    // queued early
    for (int it = 0; direct && it < prm->irls && !rc && e == cudaSuccess; ++it)
        for (int i = 0; i < n && !rc; ++i) {
            rc = select_slot(c, i);
            if (!rc) rc = solve_iter(c, sv[i], it);
        }
    for (int i = 0; i < n && !rc && e == cudaSuccess && !lockstep; ++i) {
        rc = select_slot(c, i);
        if (!rc && host_io)
            e = cudaMemcpyAsync(image_out[i], out_dev[i], image_bytes(i), cudaMemcpyDeviceToHost,
                                c->stream);
        if (!rc && e == cudaSuccess) e = cudaEventCreateWithFlags(&done[i], cudaEventDisableTiming);
        if (!rc && e == cudaSuccess) e = cudaEventRecord(done[i], c->stream);
    }
    if (!rc && e == cudaSuccess) {
        rc = select_slot(c, 0);
        for (int i = 1; i < n && !rc && e == cudaSuccess && !lockstep; ++i)
            e = cudaStreamWaitEvent(c->stream, done[i], 0);
        if (!rc && e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    }
    for (int i = 0; i < n && !rc && e == cudaSuccess; ++i) {
        rc = select_slot(c, i);
        if (!rc) rc = solve_check(c, sv[i]);
    }
    if (rc || e != cudaSuccess)  // nothing queued for the caller's buffers outlives the call
        for (int i = 0; i < n && i < (int)c->slots.size(); ++i)
            if (select_slot(c, i) == RECON_OK) cudaStreamSynchronize(c->stream);
    cleanup();
    if (e != cudaSuccess) return cuda_fail(c, e, "batched solve");
    return rc;
}

int check_many_ptrs(recon_ctx* c, int n, const void* const* kspace, const uint8_t* const* masks,
                    const recon_params* prm, void* const* image_out) {
    if (n < 1 || n > RECON_MAX_BATCH) return fail(c, RECON_EINVAL, "need 1 <= n <= RECON_MAX_BATCH");
    if (!kspace || !masks || !prm || !image_out) return fail(c, RECON_EINVAL, "null pointer");
    for (int i = 0; i < n; ++i) {
        if (!kspace[i] || !masks[i] || !image_out[i]) return fail(c, RECON_EINVAL, "null pointer");
        if (misaligned({kspace[i], masks[i], image_out[i]})) return fail(c, RECON_EINVAL, kAlignMsg);
    }
    return RECON_OK;
}

}  // namespace

int recon_solve_batch(recon_ctx* c, int n, recon_dims dd, const void* const* kspace,
                      const uint8_t* const* masks, recon_filter f, const recon_params* prm,
                      void* const* image_out) {
    if (!c) return RECON_EINVAL;
    int rc = check_many_ptrs(c, n, kspace, masks, prm, image_out);
    if (rc) return rc;
    Dims d;
    rc = check_params(c, dd, f, prm, &d);
    if (rc) return rc;
    std::vector<Dims> dims(n, d);
    return solve_many_impl(c, n, dims.data(), kspace, masks, prm, image_out);
}

int recon_solve_batch_host(recon_ctx* c, int n, recon_dims dd, const void* const* kspace,
                           const uint8_t* const* masks, recon_filter f, const recon_params* prm,
                           void* const* image_out) {
    if (!c) return RECON_EINVAL;
    if (n < 1 || n > RECON_MAX_BATCH) return fail(c, RECON_EINVAL, "need 1 <= n <= RECON_MAX_BATCH");
    if (!kspace || !masks || !prm || !image_out) return fail(c, RECON_EINVAL, "null pointer");
    for (int i = 0; i < n; ++i)
        if (!kspace[i] || !masks[i] || !image_out[i]) return fail(c, RECON_EINVAL, "null pointer");
    Dims d;
    int rc = check_params(c, dd, f, prm, &d);
    if (rc) return rc;
    std::vector<Dims> dims(n, d);
    return solve_many_impl(c, n, dims.data(), kspace, masks, prm, image_out, true);
}

int recon_solve_many(recon_ctx* c, int n, const recon_dims* dd, const recon_filter* f,
                     const void* const* kspace, const uint8_t* const* masks,
                     const recon_params* prm, void* const* image_out) {
    if (!c) return RECON_EINVAL;
    int rc = check_many_ptrs(c, n, kspace, masks, prm, image_out);
    if (rc) return rc;
    if (!dd || !f) return fail(c, RECON_EINVAL, "null pointer");
    std::vector<Dims> dims(n);
    for (int i = 0; i < n; ++i) {
        rc = check_params(c, dd[i], f[i], prm, &dims[i]);
        if (rc) return rc;
    }
    return solve_many_impl(c, n, dims.data(), kspace, masks, prm, image_out);
}

int recon_submit(recon_ctx* c, recon_dims dd, const void* kspace, const uint8_t* masks,
                 recon_filter f, const recon_params* prm, void* image_out, int* ticket) {
    if (!c) return RECON_EINVAL;
    if (!kspace || !masks || !prm || !image_out || !ticket) return fail(c, RECON_EINVAL, "null pointer");
    if (misaligned({kspace, masks, image_out})) return fail(c, RECON_EINVAL, kAlignMsg);
    Dims d;
    int rc = check_params(c, dd, f, prm, &d);
    if (rc) return rc;
    rc = set_device(c);
    if (rc) return rc;
    if (c->pending.empty()) {
        c->pending.resize(RECON_MAX_BATCH, nullptr);
        for (int k = 0; k < RECON_MAX_BATCH; ++k) {
            c->pending[k] = new recon_ctx::Pending();
            c->pending[k]->slot = k + 1;
        }
    }
    recon_ctx::Pending* pd = nullptr;
    for (auto* q : c->pending)
        if (!q->busy) { pd = q; break; }
    if (!pd) return fail(c, RECON_EBUSY, "every request slot is in flight; poll and retry");
    // admission by memory: the request's workspace must fit the budget next to the requests in
    // flight; idle slots give their cached workspaces back first
    if (c->budget) {
        const size_t need = recon_bytes_needed(dd, f, prm->kspace_bf16);
        if (need > c->budget) return fail(c, RECON_ENOMEM, "request larger than the whole budget");
        if (c->allocated + need > c->budget) release_idle(c);
        if (c->allocated + need > c->budget)
            return fail(c, RECON_EBUSY, "not enough workspace budget while other requests run");
    }
    pd->prm = *prm;
    rc = select_slot(c, pd->slot);
    if (!rc) rc = solve_prepare(c, d, kspace, masks, &pd->prm, image_out, &pd->sv);
    if (rc == RECON_ENOMEM && c->budget) {
        // the workspace did not fit next to the requests in flight: give idle slots' memory
        // back and try once more, else report a transient refusal
        select_slot(c, 0);
        release_idle(c);
        rc = select_slot(c, pd->slot);
        if (!rc) rc = solve_prepare(c, d, kspace, masks, &pd->prm, image_out, &pd->sv);
        if (rc == RECON_ENOMEM) {
            select_slot(c, 0);
            return fail(c, RECON_EBUSY, "not enough workspace budget while other requests run");
        }
    }
    if (!rc) {
        rc = solve_begin(c, &pd->sv);
        for (int n = 0; n < pd->prm.irls && !rc; ++n) rc = solve_iter(c, pd->sv, n);
    }
    if (!rc && !pd->done) {
        cudaError_t e = cudaEventCreateWithFlags(&pd->done, cudaEventDisableTiming);
        if (e != cudaSuccess) rc = cuda_fail(c, e, "cudaEventCreate");
    }
    if (!rc) {
        cudaError_t e = cudaEventRecord(pd->done, c->stream);
        if (e != cudaSuccess) rc = cuda_fail(c, e, "cudaEventRecord");
    }
    drain_on_fail(c, rc);  // a request that failed part-way leaves nothing running
    const int rc0 = select_slot(c, 0);
    if (rc) {
        if (rc == RECON_ENOMEM) c->err += " (request not admitted)";
        return rc;
    }
    if (rc0) return rc0;
    pd->busy = true;
    *ticket = pd->slot;
    return RECON_OK;
}

int recon_poll(recon_ctx* c, int ticket, int* done) {
    if (!c || !done) return RECON_EINVAL;
    *done = 0;
    if (ticket < 1 || ticket > (int)c->pending.size() || !c->pending[ticket - 1]->busy)
        return fail(c, RECON_EINVAL, "no request in flight with this ticket");
    recon_ctx::Pending* pd = c->pending[ticket - 1];
    int rc = set_device(c);
    if (rc) return rc;
    const cudaError_t q = cudaEventQuery(pd->done);
    if (q == cudaErrorNotReady) return RECON_OK;
    pd->busy = false;
    *done = 1;
    if (q != cudaSuccess) return cuda_fail(c, q, "request stream");
    rc = select_slot(c, pd->slot);
    if (!rc) rc = solve_check(c, pd->sv);
    const int rc0 = select_slot(c, 0);
    return rc ? rc : rc0;
}

int recon_adjoint(recon_ctx* c, recon_dims dd, const void* kspace, int kspace_bf16,
                  const uint8_t* masks, void* x_out) {
    if (!c) return RECON_EINVAL;
    if (!kspace || !masks || !x_out) return fail(c, RECON_EINVAL, "null pointer");
    if (misaligned({kspace, masks, x_out})) return fail(c, RECON_EINVAL, kAlignMsg);
    Dims d;
    int rc = check_dims(c, dd, nullptr, &d);
    return rc ? rc : adjoint_impl(c, d, kspace, kspace_bf16, masks, x_out);
}

int recon_adjoint3(recon_ctx* c, recon_dims3 dd, const void* kspace, int kspace_bf16,
                   const uint8_t* masks, void* x_out) {
    if (!c) return RECON_EINVAL;
    if (!kspace || !masks || !x_out) return fail(c, RECON_EINVAL, "null pointer");
    if (misaligned({kspace, masks, x_out})) return fail(c, RECON_EINVAL, kAlignMsg);
    Dims d;
    int rc = check_dims3(c, dd, nullptr, &d);
    return rc ? rc : adjoint_impl(c, d, kspace, kspace_bf16, masks, x_out);
}

int recon_fft2(recon_ctx* c, recon_dims dd, const void* x, void* y, int inverse) {
    if (!c) return RECON_EINVAL;
    if (!x || !y) return fail(c, RECON_EINVAL, "null pointer");
    if (misaligned({x, y})) return fail(c, RECON_EINVAL, kAlignMsg);
    Dims d;
    int rc = check_dims(c, dd, nullptr, &d);
    return rc ? rc : fft_impl(c, d, x, y, inverse);
}

int recon_fft3(recon_ctx* c, recon_dims3 dd, const void* x, void* y, int inverse) {
    if (!c) return RECON_EINVAL;
    if (!x || !y) return fail(c, RECON_EINVAL, "null pointer");
    if (misaligned({x, y})) return fail(c, RECON_EINVAL, kAlignMsg);
    Dims d;
    int rc = check_dims3(c, dd, nullptr, &d);
    return rc ? rc : fft_impl(c, d, x, y, inverse);
}

int recon_gram(recon_ctx* c, recon_dims dd, recon_filter f, const void* x, void* G_out,
               void* lags_out) {
    if (!c) return RECON_EINVAL;
    if (!x || !G_out) return fail(c, RECON_EINVAL, "null pointer");
    if (misaligned({x, G_out})) return fail(c, RECON_EINVAL, kAlignMsg);
    Dims d;
    int rc = check_dims(c, dd, &f, &d);
    return rc ? rc : gram_impl(c, d, x, G_out, lags_out);
}

int recon_gram3(recon_ctx* c, recon_dims3 dd, recon_filter3 f, const void* x, void* G_out,
                void* lags_out) {
    if (!c) return RECON_EINVAL;
    if (!x || !G_out) return fail(c, RECON_EINVAL, "null pointer");
    if (misaligned({x, G_out})) return fail(c, RECON_EINVAL, kAlignMsg);
    Dims d;
    int rc = check_dims3(c, dd, &f, &d);
    return rc ? rc : gram_impl(c, d, x, G_out, lags_out);
}

int recon_weight(recon_ctx* c, recon_dims dd, recon_filter f, const void* G_in, double eps_in,
                 double p, int method, void* S_out, void* dsum_out, void* evals_out,
                 double* eps_out) {
    if (!c) return RECON_EINVAL;
    int rc = weight_args(c, G_in, eps_in, p, method, S_out, evals_out);
    if (rc) return rc;
    Dims d;
    rc = check_dims(c, dd, &f, &d);
    return rc ? rc : weight_impl(c, d, G_in, eps_in, p, method, S_out, dsum_out, evals_out, eps_out);
}

int recon_weight3(recon_ctx* c, recon_dims3 dd, recon_filter3 f, const void* G_in, double eps_in,
                  double p, int method, void* S_out, void* dsum_out, void* evals_out,
                  double* eps_out) {
    if (!c) return RECON_EINVAL;
    int rc = weight_args(c, G_in, eps_in, p, method, S_out, evals_out);
    if (rc) return rc;
    Dims d;
    rc = check_dims3(c, dd, &f, &d);
    return rc ? rc : weight_impl(c, d, G_in, eps_in, p, method, S_out, dsum_out, evals_out, eps_out);
}

int recon_apply_normal(recon_ctx* c, recon_dims dd, recon_filter f, const uint8_t* masks,
                       const void* S, double lambda, const void* x, void* y) {
    if (!c) return RECON_EINVAL;
    if (!masks || !S || !x || !y) return fail(c, RECON_EINVAL, "null pointer");
    if (misaligned({masks, S, x, y})) return fail(c, RECON_EINVAL, kAlignMsg);
    if (x == y) return fail(c, RECON_EINVAL, "y must not alias x");
    Dims d;
    int rc = check_dims(c, dd, &f, &d);
    return rc ? rc : apply_normal_impl(c, d, masks, S, lambda, x, y);
}

int recon_apply_normal3(recon_ctx* c, recon_dims3 dd, recon_filter3 f, const uint8_t* masks,
                        const void* S, double lambda, const void* x, void* y) {
    if (!c) return RECON_EINVAL;
    if (!masks || !S || !x || !y) return fail(c, RECON_EINVAL, "null pointer");
    if (misaligned({masks, S, x, y})) return fail(c, RECON_EINVAL, kAlignMsg);
    if (x == y) return fail(c, RECON_EINVAL, "y must not alias x");
    Dims d;
    int rc = check_dims3(c, dd, &f, &d);
    return rc ? rc : apply_normal_impl(c, d, masks, S, lambda, x, y);
}

// ---- comparison methods (Sec. IV) ----

int recon_solve_variant(recon_ctx* c, recon_dims dd, const void* kspace, const uint8_t* masks,
                        recon_filter f, const recon_params* prm, int variant, void* image_out) {
    if (!c) return RECON_EINVAL;
    if (!kspace || !masks || !prm || !image_out) return fail(c, RECON_EINVAL, "null pointer");
    if (misaligned({kspace, masks, image_out})) return fail(c, RECON_EINVAL, kAlignMsg);
    Dims d;
    int rc = check_params(c, dd, f, prm, &d);
    if (!rc) rc = check_variant(c, variant, f);
    if (rc) return rc;
    if (variant == RECON_VARIANT_DIRECT) return solve_direct(c, d, kspace, masks, prm, image_out);
    d.circ = variant == RECON_VARIANT_GIRAF;
    return solve_impl(c, d, kspace, masks, prm, image_out, variant);
}

int recon_gram_variant(recon_ctx* c, recon_dims dd, recon_filter f, int variant, const void* x,
                       void* G_out) {
    if (!c) return RECON_EINVAL;
    if (!x || !G_out) return fail(c, RECON_EINVAL, "null pointer");
    if (misaligned({x, G_out})) return fail(c, RECON_EINVAL, kAlignMsg);
    Dims d;
    int rc = check_dims(c, dd, &f, &d);
    if (!rc) rc = check_variant(c, variant, f);
    if (rc) return rc;
    if (variant == RECON_VARIANT_PROPOSED || variant == RECON_VARIANT_GIRAF) {
        d.circ = variant == RECON_VARIANT_GIRAF;
        return gram_impl(c, d, x, G_out, nullptr);
    }
    rc = set_device(c);
    if (rc) return rc;
    if (variant == RECON_VARIANT_HLR_VOXEL) {
        void* st;
        rc = ensure(c, "veps_g", sizeof(double), &st);
        if (rc) return rc;
        RC_CUDA(cudaMemsetAsync(st, 0, sizeof(double), c->stream));
        RC_CUDA(recon::launch_voxel_weight(d, (const float2*)x, 0.0, nullptr, (double*)st, 1,
                                           nullptr, (double2*)G_out, nullptr, c->stream));
        RC_CUDA(cudaStreamSynchronize(c->stream));
        return RECON_OK;
    }
    Twiddles tw;
    Work w;
    DirectWork dw;
    rc = direct_prepare(c, d, nullptr, 1, &tw, &w, &dw);
    if (rc) return rc;
    rc = direct_gram(c, d, tw, dw, (const float2*)x, (double2*)G_out);
    if (rc) return rc;
    RC_CUDA(cudaStreamSynchronize(c->stream));
    return RECON_OK;
}

int recon_voxel_weight(recon_ctx* c, recon_dims dd, int M, const void* x, const double* eps,
                       double p, void* S_out, double* lmax_out) {
    if (!c) return RECON_EINVAL;
    if (!x || !eps || !S_out) return fail(c, RECON_EINVAL, "null pointer");
    if (misaligned({x, S_out})) return fail(c, RECON_EINVAL, kAlignMsg);
    if (!(p >= 0.0 && p <= 1.0)) return fail(c, RECON_EINVAL, "need 0 <= p <= 1");
    Dims d;
    const recon_filter f{1, 1, M};
    int rc = check_dims(c, dd, &f, &d);
    if (rc) return rc;
    rc = set_device(c);
    if (rc) return rc;
    RC_CUDA(recon::launch_voxel_weight(d, (const float2*)x, p, eps, nullptr, 0, (float2*)S_out,
                                       nullptr, lmax_out, c->stream));
    RC_CUDA(cudaStreamSynchronize(c->stream));
    return RECON_OK;
}

int recon_weight_direct(recon_ctx* c, recon_dims dd, recon_filter f, const void* G_in,
                        double eps_in, double p, int method, void* H_out, double* eps_out) {
    if (!c) return RECON_EINVAL;
    int rc = weight_args(c, G_in, eps_in, p, method, H_out, nullptr);
    if (rc) return rc;
    Dims d;
    rc = check_dims(c, dd, &f, &d);
    if (rc) return rc;
    recon_params prm{};
    prm.irls = 1;
    prm.cg = 1;
    prm.p = p;
    prm.weight_method = method;
    Twiddles tw;
    Work w;
    DirectWork dw;
    rc = direct_prepare(c, d, &prm, 1, &tw, &w, &dw);
    if (rc) return rc;
    rc = reset_status(c, w);
    if (rc) return rc;
    const size_t gbytes = (size_t)d.s() * d.s() * sizeof(double2);
    RC_CUDA(cudaMemcpyAsync(w.G, G_in, gbytes, cudaMemcpyDeviceToDevice, c->stream));
    const bool set = eps_in >= 0.0;
    rc = direct_weight(c, d, w, dw, p, 1, set ? 0.0 : -eps_in, 1.0, set, eps_in, 0);
    if (rc) return rc;
    RC_CUDA(cudaMemcpyAsync(H_out, dw.H, gbytes, cudaMemcpyDeviceToDevice, c->stream));
    RC_CUDA(cudaStreamSynchronize(c->stream));
    rc = check_status(c, w, 1);
    if (rc) return rc;
    if (eps_out) RC_CUDA(cudaMemcpy(eps_out, w.eps, sizeof(double), cudaMemcpyDeviceToHost));
    return RECON_OK;
}

int recon_apply_normal_variant(recon_ctx* c, recon_dims dd, recon_filter f, int variant,
                               const uint8_t* masks, const void* W, double lambda, const void* x,
                               void* y) {
    if (!c) return RECON_EINVAL;
    if (!masks || !W || !x || !y) return fail(c, RECON_EINVAL, "null pointer");
    if (misaligned({masks, W, x, y})) return fail(c, RECON_EINVAL, kAlignMsg);
    if (x == y) return fail(c, RECON_EINVAL, "y must not alias x");
    Dims d;
    int rc = check_dims(c, dd, &f, &d);
    if (!rc) rc = check_variant(c, variant, f);
    if (rc) return rc;
    if (variant != RECON_VARIANT_DIRECT) {
        d.circ = variant == RECON_VARIANT_GIRAF;
        return apply_normal_impl(c, d, masks, W, lambda, x, y);
    }
    Twiddles tw;
    Work w;
    DirectWork dw;
    rc = direct_prepare(c, d, nullptr, 1, &tw, &w, &dw);
    if (rc) return rc;
    const size_t ss = (size_t)d.s() * d.s();
    RC_CUDA(recon::launch_h_delta((const double2*)W, nullptr, dw.hd32, dw.h32, ss, c->stream));
    rc = direct_op(c, d, tw, dw, (const float2*)x, dw.h32, masks, (float)lambda, (float2*)y);
    if (rc) return rc;
    RC_CUDA(cudaStreamSynchronize(c->stream));
    return RECON_OK;
}

int recon_apply_w(recon_ctx* c, recon_dims dd, recon_filter f, const void* S, const void* x,
                  void* y) {
    if (!c) return RECON_EINVAL;
    if (!S || !x || !y) return fail(c, RECON_EINVAL, "null pointer");
    if (misaligned({S, x, y})) return fail(c, RECON_EINVAL, kAlignMsg);
    if (x == y) return fail(c, RECON_EINVAL, "y must not alias x");
    Dims d;
    int rc = check_dims(c, dd, &f, &d);
    if (rc) return rc;
    rc = set_device(c);
    if (rc) return rc;
    RC_CUDA(recon::launch_apply_w(d, (const float2*)x, (const float2*)S, (float2*)y, c->stream));
    RC_CUDA(cudaStreamSynchronize(c->stream));
    return RECON_OK;
}

int recon_cg(recon_ctx* c, recon_dims dd, recon_filter f, const uint8_t* masks, const void* S_old,
             const void* S_new, double lambda, void* x, void* r, int n_cg, double* rr_hist) {
    if (!c) return RECON_EINVAL;
    if (!masks || !S_new || !x || !r) return fail(c, RECON_EINVAL, "null pointer");
    if (misaligned({masks, S_new, x, r})) return fail(c, RECON_EINVAL, kAlignMsg);
    if (n_cg < 0) return fail(c, RECON_EINVAL, "n_cg must be >= 0");
    Dims d;
    int rc = check_dims(c, dd, &f, &d);
    if (rc) return rc;
    rc = set_device(c);
    if (rc) return rc;
    Twiddles tw;
    rc = get_twiddles(c, d, &tw);
    if (rc) return rc;
    Work w;
    rc = get_work(c, d, n_cg, 1, true, false, &w);
    if (rc) return rc;
    rc = reset_status(c, w);
    if (rc) return rc;
    // the caller's r is the residual buffer for this call
    float2* r_save = w.r;
    w.r = (float2*)r;
    rc = cg_block(c, d, tw, w, masks, (const float2*)S_old, (const float2*)S_new, (float)lambda,
                  (float2*)x, S_old == nullptr, n_cg);
    w.r = r_save;
    if (rc) return rc;
    RC_CUDA(cudaStreamSynchronize(c->stream));
    if (rr_hist)
        RC_CUDA(cudaMemcpy(rr_hist, w.rr, (size_t)(n_cg + 1) * sizeof(double), cudaMemcpyDeviceToHost));
    return RECON_OK;
}

int recon_t2fit(recon_ctx* c, recon_dims dd, const void* x, const double* times_ms, double fg_frac,
                int n_gn, float* t2_out, float* amp_out) {
    if (!c) return RECON_EINVAL;
    if (!x || !times_ms || !t2_out) return fail(c, RECON_EINVAL, "null pointer");
    if (misaligned({x})) return fail(c, RECON_EINVAL, kAlignMsg);
    if (dd.P <= 0 || dd.Q <= 0 || dd.T < 2 || dd.T > recon::kT2MaxT)
        return fail(c, RECON_EINVAL, "need P, Q > 0 and 2 <= T <= 64");
    if (!(fg_frac >= 0.0 && fg_frac < 1.0)) return fail(c, RECON_EINVAL, "need 0 <= fg_frac < 1");
    if (n_gn < 0 || n_gn > 1000) return fail(c, RECON_EINVAL, "need 0 <= n_gn <= 1000");
    recon::T2Times tm{};
    for (int n = 0; n < dd.T; ++n) {
        if (!std::isfinite(times_ms[n])) return fail(c, RECON_EINVAL, "echo times must be finite");
        tm.t[n] = (float)times_ms[n];
    }
    int rc = set_device(c);
    if (rc) return rc;
    void* amax = nullptr;
    rc = ensure(c, "t2amax", 256, &amax);
    if (rc) return rc;
    recon::Dims d;
    d.T = dd.T;
    d.P = dd.P;
    d.Q = dd.Q;
    d.N1 = d.N2 = d.M = 1;
    RC_CUDA(recon::launch_t2fit(d, (const float2*)x, tm, (float)fg_frac, n_gn, (unsigned int*)amax,
                                t2_out, amp_out, c->stream));
    RC_CUDA(cudaStreamSynchronize(c->stream));
    return RECON_OK;
}

int recon_set_option(recon_ctx* c, int option, int value) {
    if (!c) return RECON_EINVAL;
    switch (option) {
        case RECON_OPT_GRAPHS: c->graphs = value != 0; return RECON_OK;
        case RECON_OPT_AUTOTUNE: c->autotune = value != 0; return RECON_OK;
        case RECON_OPT_INJECT_BARRIER_FAULT: c->inject_barrier_fault = value != 0; return RECON_OK;
        case RECON_OPT_TEST_WITHHOLD_ARRIVAL: c->withhold_arrival = value != 0; return RECON_OK;
        case RECON_OPT_AUTOTUNE_FFT: c->autotune_fft = value != 0; return RECON_OK;
        case RECON_OPT_FFT_SCHEDULE:
            if (value < -1 || value >= recon::kFftSchedules)
                return fail(c, RECON_EINVAL, "radix schedule must be -1 (tuned), 0 or 1");
            c->fft_sched = value;
            return RECON_OK;
        case RECON_OPT_BATCH_GROUP:
            if (value < 0 || value > RECON_MAX_BATCH) return fail(c, RECON_EINVAL, "need 0 <= group <= RECON_MAX_BATCH");
            c->batch_group = value;
            return RECON_OK;
        default: return fail(c, RECON_EINVAL, "unknown option");
    }
}

int recon_tile_cache(recon_ctx* c, const char* path) {
    if (!c) return RECON_EINVAL;
    if (!path) {
        c->tile_cache.clear();
        return RECON_OK;
    }
    std::ifstream f(path);
    std::string line;
    auto width_ok = [](int v) { return v == 0 || v == 8 || v == 16 || v == 32; };
    auto sched_ok = [](int v) { return v >= 0 && v < recon::kFftSchedules; };
    while (f && std::getline(f, line)) {
        std::istringstream ls(line);
        int P, Q, T, R, nc, colC, depthC, colS = 0, depthS = 0;
        if (!(ls >> P >> Q >> T >> R >> nc >> colC >> depthC) || !width_ok(colC) || !width_ok(depthC))
            return fail(c, RECON_EINVAL, "tile cache: malformed entry in " + std::string(path));
        // the radix schedules (two more fields) are optional: entries without them use schedule 0
        if (ls >> colS) {
            if (!(ls >> depthS) || !sched_ok(colS) || !sched_ok(depthS))
                return fail(c, RECON_EINVAL, "tile cache: malformed entry in " + std::string(path));
        }
        c->tiles[std::make_tuple(P, Q, T, R, nc)] = {colC, depthC, colS, depthS};
    }
    c->tile_cache = path;
    return RECON_OK;
}

int recon_tile_choice(recon_ctx* c, recon_dims3 dd, int n_coils, int* colC, int* depthC) {
    if (!c || !colC || !depthC) return RECON_EINVAL;
    auto it = c->tiles.find(std::make_tuple(dd.P, dd.Q, dd.T, dd.R, n_coils));
    if (it == c->tiles.end()) {
        *colC = *depthC = 0;
        return RECON_OK;
    }
    *colC = it->second.colC;
    *depthC = it->second.depthC;
    return RECON_OK;
}

int recon_fft_schedule_choice(recon_ctx* c, recon_dims3 dd, int n_coils, int* colS, int* depthS) {
    if (!c || !colS || !depthS) return RECON_EINVAL;
    auto it = c->tiles.find(std::make_tuple(dd.P, dd.Q, dd.T, dd.R, n_coils));
    if (it == c->tiles.end()) {
        *colS = *depthS = -1;
        return RECON_OK;
    }
    *colS = it->second.colS;
    *depthS = it->second.depthS;
    return RECON_OK;
}

int recon_profile(recon_ctx* c, unsigned int kind_mask) {
    if (!c) return RECON_EINVAL;
    prof_collect(c);  // drop what was recorded so far (the totals are reset below)
    for (int k = 0; k < RECON_PROF_KINDS; ++k) {
        c->prof_ms[k] = 0.0;
        c->prof_n[k] = 0;
    }
    c->prof = kind_mask & ((1u << RECON_PROF_KINDS) - 1u);
    return RECON_OK;
}

int recon_profile_read(recon_ctx* c, int kind, double* total_ms, long long* launches) {
    if (!c) return RECON_EINVAL;
    if (kind < 0 || kind >= RECON_PROF_KINDS || !total_ms || !launches)
        return fail(c, RECON_EINVAL, "bad profile kind or null pointer");
    prof_collect(c);
    *total_ms = c->prof_ms[kind];
    *launches = c->prof_n[kind];
    return RECON_OK;
}

const char* recon_profile_name(int kind) {
    static const char* names[RECON_PROF_KINDS] = {
        "adjoint", "gram", "eig", "eps", "diag_sums", "weight_S", "resid_carry",
        "cg_row_fwd", "cg_col_mask", "cg_row_inv_w", "cg_update", "lanczos", "hpd_inverse"};
    return (kind >= 0 && kind < RECON_PROF_KINDS) ? names[kind] : "";
}

}  // extern "C"
