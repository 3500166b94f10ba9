// recon_gram_static: the Gram matrix of recon_gram for callers that must not allocate device
// memory, e.g. a scanner-side reconstruction service whose device memory is planned up front and
// may not grow, or a host program that shares the GPU with other work and cannot afford the
// device-wide synchronisation that cudaMalloc / cudaFree can cause. Instead of the context's
// workspace, the per-row pruned DFTs and the twiddle tables live in one file-scope device
// array of fixed size, which every GPU that loads the library keeps until the process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>
#include <string>

#include "../../include/recon.h"
#include "common.cuh"
#include "kernels.h"

namespace {

// The scratch array. In host code this name is only a host-side stand-in for the device symbol;
// its device address comes from cudaGetSymbolAddress (see scratch_on_device).
static __device__ __align__(256) unsigned char g_gram_scratch[RECON_GRAM_STATIC_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {nullptr};
unsigned long long g_ctx_id[kMaxDevices] = {0};

int static_fail(int code, const std::string& msg) {
    recon::set_context_free_error(msg);  // read back with recon_last_error(NULL)
    return code;
}

// Identity of the calling thread's current context (a driver context id, unique for the life of
// the process), 0 when there is none yet or the driver does not offer the query. The two driver
// calls are reached through the runtime's entry-point lookup, so the library does not link the
// driver library itself.
typedef int (*CtxGetCurrentFn)(void** ctx);
typedef int (*CtxGetIdFn)(void* ctx, unsigned long long* id);
unsigned long long current_context_id() {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        looked_up = true;
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(f);
    }
    if (!get_current || !get_id) return 0;
    void* ctx = nullptr;
    unsigned long long id = 0;
    if (get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
    return id;
}

// Device address of the scratch array on the current device, looked up once per device and
// context: a device reset gives the device a new primary context, whose array lives elsewhere.
// Without a context id (no current context yet, or no driver query) it is looked up every call.
int scratch_on_device(int dev, unsigned char** out) {
    std::lock_guard<std::mutex> lk(g_mu);
    const unsigned long long id = current_context_id();
    if (!g_addr[dev] || id == 0 || id != g_ctx_id[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_gram_scratch);
        if (e != cudaSuccess)
            return static_fail(RECON_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_addr[dev] = p;
        // the lookup creates the context when the thread had none: read its id now
        g_ctx_id[dev] = id != 0 ? id : current_context_id();
    }
    *out = reinterpret_cast<unsigned char*>(g_addr[dev]);
    return RECON_OK;
}

// e^{-2 pi i j / n}: FP32 table for length Q, FP64 table for length P (the two the Gram uses).
__global__ void static_twiddle_kernel(int P, int Q, float2* twQ, double2* twPd) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < Q) {
        double s, c;
        sincospi(2.0 * (double)i / (double)Q, &s, &c);
        twQ[i] = make_float2((float)c, (float)-s);
    }
    if (i < P) {
        double s, c;
        sincospi(2.0 * (double)i / (double)P, &s, &c);
        twPd[i] = make_double2(c, -s);
    }
}

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace

extern "C" int recon_gram_static(recon_dims dd, recon_filter f, const void* x, void* G_out,
                                 void* lags_out, void* cuda_stream) {
    if (!x || !G_out) return static_fail(RECON_EINVAL, "null pointer");
    if ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(G_out) |
         reinterpret_cast<uintptr_t>(lags_out)) & 15u)
        return static_fail(RECON_EINVAL, "device arrays must be 16-byte aligned");
    if (dd.P <= 0 || dd.Q <= 0 || dd.T <= 0 || !recon::fft_size_supported(dd.P) ||
        !recon::fft_size_supported(dd.Q))
        return static_fail(RECON_EINVAL, "P and Q must be one of 16, 32, 64, 128, 192, 256, 512");
    if (f.M < 1 || f.M > dd.T || f.N1 < 1 || f.N1 > dd.P || f.N2 < 1 || f.N2 > dd.Q)
        return static_fail(RECON_EINVAL, "need 1 <= M <= T, 1 <= N1 <= P, 1 <= N2 <= Q");
    recon::Dims d{dd.T, dd.P, dd.Q, f.N1, f.N2, f.M};
    const int nb = recon::gram_blocks(d);
    const size_t part = align256(recon::gram_scratch_bytes(d, nb));
    const size_t twq = align256((size_t)d.Q * sizeof(float2));
    const size_t twp = align256((size_t)d.P * sizeof(double2));
    if (part + twq + twp > (size_t)RECON_GRAM_STATIC_BYTES)
        return static_fail(RECON_EINVAL,
                           "problem needs " + std::to_string(part + twq + twp) +
                               " bytes of Gram scratch, more than the fixed " +
                               std::to_string((size_t)RECON_GRAM_STATIC_BYTES) +
                               " (RECON_GRAM_STATIC_BYTES); use recon_gram");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return static_fail(RECON_ECUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return static_fail(RECON_ECUDA, "device index out of range");
    unsigned char* base = nullptr;
    int rc = scratch_on_device(dev, &base);
    if (rc) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
    double2* lag_part = reinterpret_cast<double2*>(base);
    float2* twQ = reinterpret_cast<float2*>(base + part);
    double2* twPd = reinterpret_cast<double2*>(base + part + twq);
    // Every byte the Gram kernels read from the array is written first in this call (twiddles
    // here, each image row's pruned DFTs by that row's block), so no clearing is needed.
    const int n = d.P > d.Q ? d.P : d.Q;
    static_twiddle_kernel<<<(n + 255) / 256, 256, 0, st>>>(d.P, d.Q, twQ, twPd);
    e = cudaGetLastError();
    if (e != cudaSuccess) return static_fail(RECON_ECUDA, cudaGetErrorString(e));
    recon::Twiddles tw{nullptr, twQ, twPd, nullptr};
    e = recon::launch_gram(d, tw, reinterpret_cast<const float2*>(x), lag_part, nb,
                           reinterpret_cast<double2*>(lags_out), reinterpret_cast<double2*>(G_out), st);
    if (e == cudaErrorInvalidValue)
        return static_fail(RECON_EINVAL, "filter / frame count too large for the Gram kernel");
    if (e != cudaSuccess) return static_fail(RECON_ECUDA, cudaGetErrorString(e));
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return static_fail(RECON_ECUDA, cudaGetErrorString(e));
    return RECON_OK;
}
