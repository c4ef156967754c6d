// goat_noalloc.cu -- a Sinkhorn entry point that allocates nothing.
//
// Some callers cannot allocate device memory while they run this step: code
// that runs under an allocator it does not own (a framework's caching
// allocator, a real-time loop with a fixed memory budget, a host thread that
// must not synchronise with the device as cudaMalloc/cudaFree can), or code
// that has no way to hand us a workspace.  goat_sinkhorn_noalloc serves them: its
// scratch (the device state block and the column partial sums) lives in one
// file-scope device array that every GPU loading the library holds until exit,
// and it neither allocates nor synchronises with the device.
#include <cstring>
#include <mutex>

#include "goat_common.cuh"
#include "goat_internal.h"

namespace goat {

// Largest n this entry point accepts; the scratch below is sized for it.
constexpr int kNoallocMaxN = 4096;
// Largest max_iter: every iteration slot is queued up front (about five launches each).
constexpr int kNoallocMaxIter = 1000;
// DevState (rounded to 16 KiB) + at most ceil(n / 64) row chunks x n FP64 column partials.
constexpr size_t kNoallocStateBytes = 16384;
constexpr size_t kNoallocScratchBytes = kNoallocStateBytes + (size_t)(kNoallocMaxN / 64) * kNoallocMaxN * 8;

static_assert(sizeof(DevState) <= kNoallocStateBytes, "state block does not fit its slot");
// the partial sums above are laid out for the two-pass iteration (ceil(n / 64) row chunks)
static_assert(kNoallocMaxN < kSkFusedMinN, "the fused iteration's partial sums need more room");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

// Identity of the calling thread's current CUDA context (0 if none or unknown),
// through the driver's cuCtxGetCurrent / cuCtxGetId entry points.
static unsigned long long current_context_id() {
    typedef int (*get_current_fn)(void **);
    typedef int (*get_id_fn)(void *, unsigned long long *);
    static get_current_fn get_current = nullptr;
    static get_id_fn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<get_current_fn>(p);
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<get_id_fn>(p);
        cudaGetLastError();
    });
    void *ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
    return id;
}

// Device address of g_noalloc_scratch in the current context (the host-side symbol
// is a stand-in, not a device address).  Looked up once per device, with that
// device current, and again only if the device's context has changed since (after
// a cudaDeviceReset the array lives at a new address).
static unsigned char *noalloc_scratch_address(int *status) {
    static std::mutex mu;
    static unsigned char *addr[64] = {};
    static unsigned long long ctx_of[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        *status = GOAT_ERR_CUDA;
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(mu);
    const unsigned long long ctx = current_context_id();
    if (!addr[dev] || ctx == 0 || ctx != ctx_of[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            *status = GOAT_ERR_CUDA;
            return nullptr;
        }
        addr[dev] = static_cast<unsigned char *>(p);
        ctx_of[dev] = current_context_id();  // the lookup above makes the primary context current
    }
    *status = GOAT_OK;
    return addr[dev];
}

__global__ void k_noalloc_state_init(DevState *st) {
    st->eps_rel = 0.03f;
    st->maximize = 1;
    st->eps = 1.0f;
    st->c = 1.4426950408889634f;
}

__global__ void k_noalloc_report(const DevState *st, int *iters_out, float *resid_out, int *status_out) {
    if (iters_out) *iters_out = st->sk_iters;
    if (resid_out) *resid_out = st->sk_resid;
    if (status_out) *status_out = st->error;
}

}  // namespace goat

using namespace goat;

extern "C" {

int goat_sinkhorn_noalloc(const float *G, int n, float eps, float tol, int max_iter, float *f_out, float *g_io,
                          int *iters_out, float *resid_out, int *status_out, goat_stream_t stream) {
    if (!G || !f_out || !g_io || n < 1 || !(eps > 0.0f) || !(tol >= 0.0f) || max_iter < 1)
        return GOAT_ERR_INVALID_ARG;
    if (n > kNoallocMaxN) return GOAT_ERR_INVALID_ARG;            // beyond the static scratch
    if (max_iter > kNoallocMaxIter) return GOAT_ERR_INVALID_ARG;  // bounded launch queue
    int dev = 0, major = 0, minor = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess) {
        cudaGetLastError();
        return GOAT_ERR_CUDA;
    }
    if (major != 10 || minor != 3) return GOAT_ERR_UNSUPPORTED;
    int status = GOAT_OK;
    unsigned char *scratch = noalloc_scratch_address(&status);
    if (!scratch) return status;
    cudaStream_t s = (cudaStream_t)stream;
    DevState *st = reinterpret_cast<DevState *>(scratch);
    double *partial = reinterpret_cast<double *>(scratch + kNoallocStateBytes);
    // the array keeps the previous call's contents: the state block must start at zero
    // (the partial sums are fully rewritten by every iteration before they are read)
    if (cudaMemsetAsync(st, 0, sizeof(DevState), s) != cudaSuccess) {
        cudaGetLastError();
        return GOAT_ERR_CUDA;
    }
    k_noalloc_state_init<<<1, 1, 0, s>>>(st);
    note_launches(1);
    sinkhorn_begin(st, eps, tol, nullptr, n, s);
    sinkhorn_queue_fixed(G, n, n, f_out, g_io, partial, st, max_iter, s);
    k_noalloc_report<<<1, 1, 0, s>>>(st, iters_out, resid_out, status_out);
    note_launches(1);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GOAT_OK : GOAT_ERR_CUDA;
}

}  // extern "C"
