// fz_noalloc.cu -- counting without any device allocation.
//
// Some callers cannot call cudaMalloc: code that runs while a stream is being
// captured into a CUDA graph (allocation calls are not permitted there),
// latency-critical loops that must not hit the allocator's implicit device
// synchronisation, and processes whose device memory is entirely reserved by
// another allocator.  fz_count_upto_noalloc serves them: it computes the same
// |Z(r, g)|, r = 0..n_max, as fz_count_upto, but its two rolling count rows
// and the blocked-scan scratch live in one fixed array compiled into this
// library, so the call itself allocates nothing.
//
// That array is a file-scope __device__ variable: every GPU that loads the
// library holds it (NOALLOC_WORDS * 8 bytes, about 4.4 MB) until the process
// exits.  Its address is looked up with cudaGetSymbolAddress the first time
// a device's context is current here (host code must never pass the
// variable's host-side name to a kernel), and looked up again whenever that
// context changes: after cudaDeviceReset, or a reset of the primary context
// by other code, the module is loaded afresh and the old address is stale.
// The context is identified by the driver's context id (cuCtxGetId, reached
// through the runtime's driver entry point, so the library still links no
// libcuda), which is never reused within a process.
// All calls share it, so calls that overlap on the GPU (other streams, other
// host threads) race on it; every word a call reads it has written first in
// the same call, so nothing needs clearing between calls.
#include <mutex>

#include "fz_internal.cuh"

namespace fz {
namespace {

constexpr int64_t NOALLOC_MAX_N = FZ_NOALLOC_MAX_N;
constexpr int64_t NOALLOC_ROW = NOALLOC_MAX_N + 1;
constexpr int64_t NOALLOC_TMP = 20000;  // >= blocked-scan scratch for any g at NOALLOC_ROW
constexpr int64_t NOALLOC_WORDS = 2 * NOALLOC_ROW + NOALLOC_TMP;

__device__ __align__(256) uint64_t g_noalloc_scratch[NOALLOC_WORDS];

constexpr int MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
struct ScratchAddr {
    unsigned long long ctx_id = 0;  // 0: not looked up yet
    uint64_t *ptr = nullptr;
};
ScratchAddr g_noalloc_addr[MAX_DEVICES];

// Driver calls, fetched once through cudaGetDriverEntryPointByVersion.
typedef int (*CtxGetCurrentFn)(void **ctx);
typedef int (*CtxGetIdFn)(void *ctx, unsigned long long *id);
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;
bool g_driver_fns_tried = false;

// Id of the context current on this thread, 0 when none is current yet (or
// the driver entry points are unavailable).  Caller holds g_noalloc_mu.
unsigned long long current_ctx_id() {
    if (!g_driver_fns_tried) {
        g_driver_fns_tried = true;
        cudaDriverEntryPointQueryResult q1, q2;
        void *f1 = nullptr, *f2 = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault,
                                             &q1) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault,
                                             &q2) == cudaSuccess &&
            q2 == cudaDriverEntryPointSuccess) {
            g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
            g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(f2);
        }
        cudaGetLastError();
    }
    if (!g_ctx_get_current || !g_ctx_get_id) return 0;
    void *ctx = nullptr;
    unsigned long long id = 0;
    if (g_ctx_get_current(&ctx) != 0 || !ctx) return 0;
    if (g_ctx_get_id(ctx, &id) != 0) return 0;
    return id;
}

// Device address of the scratch array in the current device's context,
// looked up on the first call made in that context.
int noalloc_scratch(uint64_t **out) {
    int dev = 0;
    FZ_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= MAX_DEVICES)
        return set_error(FZ_EINVAL, "count_upto_noalloc: device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    ScratchAddr &a = g_noalloc_addr[dev];
    const unsigned long long id = current_ctx_id();
    if (!a.ptr || id == 0 || id != a.ctx_id) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(scratch)");
        a.ptr = static_cast<uint64_t *>(p);
        // the lookup makes the primary context current if none was
        a.ctx_id = id ? id : current_ctx_id();
    }
    *out = a.ptr;
    return FZ_OK;
}

}  // namespace
}  // namespace fz

using namespace fz;

extern "C" int fz_count_upto_noalloc(const int32_t *g, int d, int32_t n_max,
                                     uint64_t *counts_dev, void *stream) {
    int rc = validate_gens(g, d);
    if (rc != FZ_OK) return rc;
    if (n_max < 0) return set_error(FZ_EINVAL, "n must be >= 0");
    if ((int64_t)n_max > NOALLOC_MAX_N)
        return set_error(FZ_EINVAL,
                         "count_upto_noalloc: n_max exceeds FZ_NOALLOC_MAX_N (262143); "
                         "use fz_count_upto");
    if (!counts_dev) return set_error(FZ_EINVAL, "counts_dev: null pointer");
    if (count_table_tmp_words(g, d, n_max) > NOALLOC_TMP)
        return set_error(FZ_EINTERNAL, "count_upto_noalloc: scratch budget too small");
    uint64_t *base = nullptr;
    rc = noalloc_scratch(&base);
    if (rc != FZ_OK) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint64_t *a = base, *b = base + NOALLOC_ROW, *tmp = base + 2 * NOALLOC_ROW, *res = nullptr;
    rc = launch_count_rolling(g, d, n_max, a, b, tmp, &res, s);
    if (rc != FZ_OK) return rc;
    FZ_CUDA_TRY(cudaMemcpyAsync(counts_dev, res, ((size_t)n_max + 1) * sizeof(uint64_t),
                                cudaMemcpyDeviceToDevice, s));
    return FZ_OK;
}
