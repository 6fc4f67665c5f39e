// fz_api.cu -- the C ABI declared in include/fz.h: error state, counting,
// memo construction, plans (resident count table + memo per instance) and
// the one-shot enumeration calls.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "fz_internal.cuh"

namespace fz {

namespace {
thread_local std::string g_last_error;
std::atomic<uint64_t> g_launches{0};
}

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

int set_error(int status, const std::string &msg) {
    g_last_error = msg;
    return status;
}

int cuda_error(cudaError_t e, const char *what) {
    std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" +
                    cudaGetErrorString(e) + ")";
    if (e == cudaErrorMemoryAllocation) return set_error(FZ_ENOMEM, m);
    return set_error(FZ_ECUDA, m);
}

int device_props(DeviceProps *out) {
    static std::mutex mu;
    static DeviceProps cache[64];
    int dev = 0;
    FZ_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    if (dev >= 0 && dev < 64 && cache[dev].device == dev) {
        *out = cache[dev];
        return FZ_OK;
    }
    DeviceProps p;
    p.device = dev;
    FZ_CUDA_TRY(cudaDeviceGetAttribute(&p.sms, cudaDevAttrMultiProcessorCount, dev));
    FZ_CUDA_TRY(cudaDeviceGetAttribute(&p.max_smem_optin,
                                       cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    if (dev >= 0 && dev < 64) cache[dev] = p;
    *out = p;
    return FZ_OK;
}

int validate_gens(const int32_t *g, int d) {
    if (!g) return set_error(FZ_EINVAL, "generators: null pointer");
    if (d < 1 || d > FZ_MAX_D) return set_error(FZ_EINVAL, "d must be in 1..16");
    for (int i = 0; i < d; ++i)
        if (g[i] < 1) return set_error(FZ_EINVAL, "generators must be >= 1");
    return FZ_OK;
}

namespace {

// RAII device buffer (cudaMalloc / cudaFree).
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { release(); }
    int alloc(size_t b) {
        release();
        if (b == 0) b = 16;
        cudaError_t e = cudaMalloc(&p, b);
        if (e != cudaSuccess) {
            p = nullptr;
            return cuda_error(e, "cudaMalloc");
        }
        bytes = b;
        return FZ_OK;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    template <class T>
    T *as() const {
        return static_cast<T *>(p);
    }
};

int status_to_fz(int dev_status) {
    switch (dev_status) {
        case DEV_OK: return FZ_OK;
        case DEV_TIMEOUT: return set_error(FZ_ETIMEOUT, "a bounded device wait expired");
        default: return set_error(FZ_EINTERNAL, "device-side consistency check failed");
    }
}

bool mul_overflows(uint64_t a, uint64_t b, uint64_t *out) {
    if (a != 0 && b > ~0ull / a) return true;
    *out = a * b;
    return false;
}

cudaStream_t as_stream(void *s) { return static_cast<cudaStream_t>(s); }

}  // namespace
}  // namespace fz

using namespace fz;

// ---------------------------------------------------------------------------
// plan
// ---------------------------------------------------------------------------
struct fz_plan_s {
    int d = 0;
    int32_t n = 0;
    int32_t g[FZ_MAX_D] = {};
    int K = 0;
    int32_t top = 0;
    uint64_t count = 0;
    uint64_t memo_rows = 0;
    uint64_t slice_rows = 0;
    int64_t tmp_words = 0;
    DevBuf base;   // C, tmp, O, status, bar, counter
    DevBuf memo;   // map + rows
    DevBuf runs;   // runs table for work-balanced slicing
    DevBuf runm;   // memo in run order + class starts (full memo, k <= 3)
    int4 *run_memo = nullptr;
    uint64_t *cls_beg = nullptr;
    uint64_t *RT = nullptr;
    int lam_r = 0;
    int clamp_row = -1;
    uint64_t W = 0;
    uint64_t total_runs = 0;
    int ctas_per_sm = 0;
    uint64_t *C = nullptr, *tmp = nullptr, *O = nullptr, *map = nullptr;
    int32_t *rows = nullptr;
    int *status = nullptr;
    unsigned *bar = nullptr;
    unsigned long long *counter = nullptr;
};

struct fz_memo_s {
    int k = 0;
    int32_t top = 0;
    uint64_t rows = 0;
    DevBuf buf;       // offsets
    DevBuf rows_buf;  // rows
    uint64_t *O = nullptr;
    int32_t *R = nullptr;
};

namespace fz {
namespace {

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

// FZ_RUN_COST overrides W (tuning only).
void balance_level(int d, int K, int top, int n, bool run_order, int *lam_r, uint64_t *W,
                   int *clamp_row) {
    static const long long forced = [] {
        const char *e = getenv("FZ_RUN_COST");
        return e ? atoll(e) : 0ll;
    }();
    const bool memo = K >= 1 && K <= d - 1 && top > 0;
    *clamp_row = -1;
    if (run_order) {
        // the run-order walk visits every prefix of the leading d - K - 1
        // coordinates (empty or not) and copies its run
        *lam_r = d - K - 1;
        *W = 64;
    } else if (memo && top > n) {
        // full memo: the leaves are the memo leaves, evaluated 32 at a time
        *lam_r = d - K;
        *W = 16;
    } else if (K == 1 || !walk_progression_enabled()) {
        // walk leaves evaluated candidate by candidate: count the candidates
        *lam_r = d - 1;
        *W = 16;
    } else {
        // walk runs: prefixes of length d - 2, each an advance to the next
        // prefix plus a progression; a memo leaf (a prefix of length d - K
        // with remainder below top) is one unit whatever lies under it
        *lam_r = d - 2;
        *W = 64;
        if (memo && K > 2) *clamp_row = d - K;
    }
    if (*lam_r < 0) *lam_r = 0;
    if (forced > 0) *W = (uint64_t)forced;
}

// FZ_RUN_MEMO=0 keeps full memos in element order only, in plans and
// batches (tuning only).
bool run_memo_enabled() {
    static const bool on = [] {
        const char *e = getenv("FZ_RUN_MEMO");
        return !(e && e[0] == '0');
    }();
    return on;
}

namespace {

// Enqueue the memo of plan p (offsets scan, gather map, fill, run order).
int plan_enqueue_memo(fz_plan_s *p, cudaStream_t s) {
    if (p->K < 1 || p->top < 1) return FZ_OK;
    const int64_t cs = (int64_t)p->n + 1;
    const uint64_t *crow = p->C + (int64_t)(p->d - p->K) * cs;
    int rc = launch_exclusive_scan_tmp(crow, p->O, p->top, p->tmp, s);
    if (rc != FZ_OK) return rc;
    if (p->memo_rows == 0) return FZ_OK;
    MemoBuffers mb;
    mb.Ct = crow;
    mb.cs = cs;
    mb.O = p->O;
    mb.map = p->map;
    mb.rows = p->rows;
    mb.status = p->status;
    mb.bar = p->bar;
    // an enumeration capped below full occupancy leaves room for a small build
    mb.small_ctas = p->ctas_per_sm > 0 && p->ctas_per_sm <= 3;
    // depth 1 and 2: the closed form of the tail sets (same rows as the
    // dynamic pass, no dependent batches); deeper memos: the dynamic pass
    if (p->K <= 2)
        rc = launch_memo_closed(p->g + (p->d - p->K), p->K, p->top, p->O, p->rows, p->status, s);
    else
        rc = launch_memo_build(p->g + (p->d - p->K), p->K, p->top, p->memo_rows, mb, s);
    if (rc != FZ_OK || !p->run_memo) return rc;
    const int lam = p->d - p->K - 1;
    return launch_run_memo(p->C, cs, lam, p->n, p->g[lam], p->O, p->rows, p->K, p->memo_rows,
                           p->cls_beg, p->run_memo, p->status, s);
}

int read_status(int *status_dev, cudaStream_t s) {
    int h = 0;
    FZ_CUDA_TRY(cudaMemcpyAsync(&h, status_dev, sizeof(int), cudaMemcpyDeviceToHost, s));
    FZ_CUDA_TRY(cudaStreamSynchronize(s));
    if (h != 0) {
        FZ_CUDA_TRY(cudaMemsetAsync(status_dev, 0, sizeof(int), s));
        FZ_CUDA_TRY(cudaStreamSynchronize(s));
    }
    return status_to_fz(h);
}

// Memo rows of depth k with full top = n + 1, from row d - k of the table
// (exclusive scan into p->O, then one 8-byte read).  Synchronises.
int memo_rows_for(fz_plan_s *p, int k, int32_t top, uint64_t *rows, cudaStream_t s) {
    const int64_t cs = (int64_t)p->n + 1;
    const uint64_t *crow = p->C + (int64_t)(p->d - k) * cs;
    int rc = launch_exclusive_scan_tmp(crow, p->O, top, p->tmp, s);
    if (rc != FZ_OK) return rc;
    FZ_CUDA_TRY(cudaMemcpyAsync(rows, p->O + top, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
    FZ_CUDA_TRY(cudaStreamSynchronize(s));
    return FZ_OK;
}

// Memo depth chosen automatically: the deepest k in 2..min(d-1, 4) whose full
// memo stays small next to the output and needs a bounded number of
// elementwise batches; k = 0 (plain walk) when none qualifies.
int choose_k(fz_plan_s *p, cudaStream_t s, int *k_out) {
    *k_out = 0;
    const uint64_t out_bytes = p->count * (uint64_t)p->d * 4ull;
    const uint64_t budget = std::max<uint64_t>(8ull << 20, out_bytes / 8);
    for (int k = std::min(p->d - 1, 4); k >= 2; --k) {
        int32_t tmin = p->g[p->d - k];
        for (int i = p->d - k; i < p->d; ++i) tmin = std::min(tmin, p->g[i]);
        const int64_t batches = ((int64_t)p->n + 1 + tmin - 1) / tmin;
        if (batches > 4096) continue;
        uint64_t rows = 0;
        int rc = memo_rows_for(p, k, p->n + 1, &rows, s);
        if (rc != FZ_OK) return rc;
        if (rows == ~0ull || rows > MEMO_MAX_ROWS) continue;
        const uint64_t bytes = rows * (uint64_t)(4 * k + 8);
        if (bytes > budget) continue;
        *k_out = k;
        return FZ_OK;
    }
    return FZ_OK;
}

// Measured options by (device, g, n), filled by fz_autotune.
std::mutex g_tune_mu;
std::map<std::vector<int32_t>, fz_opts_t> g_tune;

std::vector<int32_t> tune_key(const int32_t *g, int d, int32_t n) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::vector<int32_t> key(g, g + d);
    key.push_back(n);
    key.push_back(dev);
    return key;
}

bool autotune_lookup(const int32_t *g, int d, int32_t n, fz_opts_t *out) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(tune_key(g, d, n));
    if (it == g_tune.end()) return false;
    *out = it->second;
    return true;
}

int plan_create_impl(const int32_t *g, int d, int32_t n, const fz_opts_t *opt, fz_plan_s *p,
                     cudaStream_t s) {
    int rc = validate_gens(g, d);
    if (rc != FZ_OK) return rc;
    if (n < 0) return set_error(FZ_EINVAL, "n must be >= 0");
    if (opt && opt->flags != 0) return set_error(FZ_EINVAL, "opts.flags must be 0");
    if (opt && (opt->k != FZ_AUTO && (opt->k < 0 || opt->k > d)))
        return set_error(FZ_EINVAL, "opts.k must be FZ_AUTO or in 0..d");
    if (opt && opt->top != FZ_AUTO && opt->top < 0)
        return set_error(FZ_EINVAL, "opts.top must be FZ_AUTO or >= 0");
    if (opt && opt->slice_rows < 0) return set_error(FZ_EINVAL, "opts.slice_rows must be >= 0");
    p->d = d;
    p->n = n;
    for (int i = 0; i < d; ++i) p->g[i] = g[i];
    const int64_t cs = (int64_t)n + 1;
    uint64_t table_words;
    if (mul_overflows((uint64_t)(d + 1), (uint64_t)cs, &table_words))
        return set_error(FZ_EOVERFLOW, "count table size");
    p->tmp_words = std::max(count_table_tmp_words(g, d, n), exclusive_scan_tmp_words(cs));
    const size_t off_C = 0;
    const size_t off_tmp = align256(off_C + table_words * 8);
    const size_t off_O = align256(off_tmp + (size_t)p->tmp_words * 8);
    const size_t off_status = align256(off_O + (size_t)(cs + 1) * 8);
    const size_t off_bar = off_status + 256;
    const size_t off_counter = off_bar + 256;
    const size_t total = off_counter + 256;
    rc = p->base.alloc(total);
    if (rc != FZ_OK) return rc;
    char *b = p->base.as<char>();
    p->C = reinterpret_cast<uint64_t *>(b + off_C);
    p->tmp = reinterpret_cast<uint64_t *>(b + off_tmp);
    p->O = reinterpret_cast<uint64_t *>(b + off_O);
    p->status = reinterpret_cast<int *>(b + off_status);
    p->bar = reinterpret_cast<unsigned *>(b + off_bar);
    p->counter = reinterpret_cast<unsigned long long *>(b + off_counter);
    FZ_CUDA_TRY(cudaMemsetAsync(b + off_status, 0, 768, s));

    rc = launch_count_table_tmp(g, d, n, p->C, p->tmp, s);
    if (rc != FZ_OK) return rc;
    FZ_CUDA_TRY(cudaMemcpyAsync(&p->count, p->C + n, sizeof(uint64_t), cudaMemcpyDeviceToHost,
                                s));
    FZ_CUDA_TRY(cudaStreamSynchronize(s));
    if (p->count == ~0ull) return set_error(FZ_EOVERFLOW, "|Z(n)| does not fit in 64 bits");

    // memo depth and top: the caller's, else a measured choice cached by
    // fz_autotune for this (g, n), else the size heuristic
    int k = opt ? opt->k : FZ_AUTO;
    int32_t tuned_slice = 0;
    if (k == FZ_AUTO) {
        fz_opts_t cached;
        if (autotune_lookup(g, d, n, &cached)) {
            k = cached.k;
            tuned_slice = cached.slice_rows;
        } else {
            rc = choose_k(p, s, &k);
            if (rc != FZ_OK) return rc;
        }
    }
    int64_t top = (opt && opt->top != FZ_AUTO) ? opt->top : (int64_t)n + 1;
    if (top > (int64_t)n + 1) top = (int64_t)n + 1;
    if (k == 0) top = 0;
    p->K = k;
    p->top = (int32_t)top;
    if (k >= 1 && top >= 1) {
        rc = memo_rows_for(p, k, p->top, &p->memo_rows, s);
        if (rc != FZ_OK) return rc;
        if (p->memo_rows == ~0ull || p->memo_rows > MEMO_MAX_ROWS)
            return set_error(FZ_EINVAL, "memo too large (more than 2^30 rows); lower k or top");
        const size_t off_rows = align256(p->memo_rows * 8);
        rc = p->memo.alloc(off_rows + p->memo_rows * (size_t)k * 4 + 16);
        if (rc != FZ_OK) return rc;
        p->map = p->memo.as<uint64_t>();
        p->rows = reinterpret_cast<int32_t *>(p->memo.as<char>() + off_rows);
        // full memo of depth <= 3: also keep it in run order (16 bytes per
        // row), which lets the enumeration copy whole subtrees of the last
        // walked coordinate as one contiguous range
        if (p->top > n && k <= 3 && k <= d - 1 && run_memo_enabled()) {
            const int32_t glam = p->g[d - k - 1];
            const int64_t G = glam < (int64_t)n + 1 ? glam : (int64_t)n + 1;
            const size_t rm_bytes = align256(p->memo_rows * 16);
            if (p->runm.alloc(rm_bytes + (size_t)(G + 1) * 8) == FZ_OK) {
                p->run_memo = p->runm.as<int4>();
                p->cls_beg = reinterpret_cast<uint64_t *>(p->runm.as<char>() + rm_bytes);
            } else {
                cudaGetLastError();  // optional: without it the leaf-by-leaf copy runs
            }
        }
        rc = plan_enqueue_memo(p, s);
        if (rc != FZ_OK) return rc;
        rc = read_status(p->status, s);
        if (rc != FZ_OK) return rc;
    }
    // runs table for work-balanced slicing (not needed when the output is a
    // single block: d == 1 or k == d with a full memo)
    const bool single_block = d == 1 || (p->K == d && p->top > n);
    if (!single_block && p->count > 0) {
        balance_level(d, p->K, p->top, n, p->run_memo != nullptr, &p->lam_r, &p->W,
                      &p->clamp_row);
        rc = p->runs.alloc((size_t)(p->lam_r + 1) * cs * 8);
        if (rc != FZ_OK) return rc;
        p->RT = p->runs.as<uint64_t>();
        rc = launch_runs_table(p->g, p->lam_r, n, p->RT, p->tmp, p->clamp_row, p->top, s);
        if (rc != FZ_OK) return rc;
        FZ_CUDA_TRY(cudaMemcpyAsync(&p->total_runs, p->RT + n, 8, cudaMemcpyDeviceToHost, s));
        FZ_CUDA_TRY(cudaStreamSynchronize(s));
        uint64_t wr = 0;
        if (mul_overflows(p->W, p->total_runs, &wr) || p->count + wr < p->count) {
            p->RT = nullptr;  // costs would not fit in 64 bits: slice by rows
            p->runs.release();
        }
    }
    DeviceProps dp;
    rc = device_props(&dp);
    if (rc != FZ_OK) return rc;
    if (opt && opt->slice_rows > 0)
        p->slice_rows = ((uint64_t)opt->slice_rows + 3) & ~3ull;
    else if (tuned_slice > 0)
        p->slice_rows = (uint64_t)tuned_slice;
    else
        p->slice_rows = default_slice_rows(p->count, dp.sms);
    return FZ_OK;
}

EnumLaunch launch_of(const fz_plan_s *p) {
    EnumLaunch L;
    L.C = p->C;
    L.cs = (int64_t)p->n + 1;
    L.O = p->O;
    L.memo = p->rows;
    L.memo_rows = p->memo_rows;
    L.status = p->status;
    L.slice_counter = p->counter;
    L.n = p->n;
    L.d = p->d;
    L.K = p->K;
    L.top = p->top;
    L.g = p->g;
    L.ctas_per_sm = p->ctas_per_sm;
    L.run_memo = p->run_memo;
    L.cls_beg = p->cls_beg;
    if (p->RT) {
        L.RT = p->RT;
        L.W = p->W;
        L.lam_r = p->lam_r;
        L.total_rows = p->count;
        L.total_cost = p->count + p->W * p->total_runs;
    }
    return L;
}

uint64_t rows_in(const fz_plan_s *p, uint64_t b, uint64_t e) {
    if (e > p->count) e = p->count;
    return b < e ? e - b : 0;
}

// ---------------------------------------------------------------------------
// Streamed delivery into pageable host memory (the role of the paper's
// copyDeviceBufferToHostAndClear flushes, Section 3.2, made asynchronous).
//
// A kernel cannot write pageable memory, and a copy-engine transfer into
// pageable memory returns only when it has finished, so the rows are made in
// chunks: chunk i is written by the enumeration kernel straight into
// page-locked, mapped staging buffer i mod HOST_STAGES (over the host link,
// as for pinned output), and host worker threads copy every finished stage
// into the caller's array while the GPU fills the next ones.  The host
// enqueues chunk i only once the workers have emptied its stage (chunk
// i - HOST_STAGES), so the GPU runs at most HOST_STAGES - 1 chunks ahead of
// the host copies and the output may be far larger than device memory.
// The staging buffers are kept between calls (one pool per process, grown
// on demand: pinning memory costs far more than copying one chunk) and are
// used by one call at a time; a call that finds the pool busy pins its own.
// ---------------------------------------------------------------------------
constexpr int HOST_STAGES = 3;

// True when the current device reads and writes pageable host memory through
// the host's page tables (cudaDevAttrPageableMemoryAccess and
// ...UsesHostPageTables both 1).  FZ_HOST_DIRECT=0 turns the direct path off
// (tuning and testing only).
bool pageable_direct_ok() {
    static const bool allowed = [] {
        const char *e = std::getenv("FZ_HOST_DIRECT");
        return !(e && e[0] == '0');
    }();
    if (!allowed) return false;
    int dev = 0, pma = 0, hpt = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&pma, cudaDevAttrPageableMemoryAccess, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&hpt, cudaDevAttrPageableMemoryAccessUsesHostPageTables, dev) !=
            cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return pma == 1 && hpt == 1;
}

struct StagePool {
    std::mutex mu;  // held by the call using the pool
    char *base = nullptr;
    size_t bytes = 0;
};
StagePool g_stage_pool;

int host_copy_threads() {
    static const int t = [] {
        const char *e = std::getenv("FZ_HOST_COPY_THREADS");
        int v = e ? std::atoi(e) : 0;
        if (v <= 0) {
            const unsigned hc = std::thread::hardware_concurrency();
            v = hc >= 4 ? (int)(hc / 2) : 1;
            if (v > 8) v = 8;
        }
        return v > 64 ? 64 : v;
    }();
    return t;
}

// Default chunk: 128 MB of rows.
uint64_t default_host_chunk_rows(int d) {
    return std::max<uint64_t>(1u << 14, (128ull << 20) / (4ull * (uint64_t)d));
}

struct CopyJob {
    const char *src;
    char *dst;
    size_t bytes;
    int stage;
    cudaEvent_t ev;
};

int stream_to_pageable(fz_plan_s *p, uint64_t rank_begin, uint64_t rows, int32_t *out_host,
                       uint64_t chunk_rows, cudaStream_t s) {
    const int d = p->d;
    if (chunk_rows == 0) chunk_rows = default_host_chunk_rows(d);
    if (chunk_rows > rows) chunk_rows = rows;
    const size_t stage_bytes = align256(chunk_rows * (size_t)d * 4);
    const size_t pool_bytes = HOST_STAGES * stage_bytes;

    // staging buffers: the process pool when it is free, else this call's own
    std::unique_lock<std::mutex> pool_lk(g_stage_pool.mu, std::try_to_lock);
    char *base = nullptr;
    bool own = false;
    if (pool_lk.owns_lock()) {
        if (g_stage_pool.bytes < pool_bytes) {
            if (g_stage_pool.base) cudaFreeHost(g_stage_pool.base);
            g_stage_pool.base = nullptr;
            g_stage_pool.bytes = 0;
            void *h = nullptr;
            if (cudaHostAlloc(&h, pool_bytes, cudaHostAllocMapped | cudaHostAllocPortable) !=
                cudaSuccess) {
                cudaGetLastError();
                return set_error(FZ_ENOMEM, "cudaHostAlloc (staging buffers)");
            }
            g_stage_pool.base = static_cast<char *>(h);
            g_stage_pool.bytes = pool_bytes;
        }
        base = g_stage_pool.base;
    } else {
        void *h = nullptr;
        if (cudaHostAlloc(&h, pool_bytes, cudaHostAllocMapped | cudaHostAllocPortable) !=
            cudaSuccess) {
            cudaGetLastError();
            return set_error(FZ_ENOMEM, "cudaHostAlloc (staging buffers)");
        }
        base = static_cast<char *>(h);
        own = true;
    }
    void *dbase_v = nullptr;
    cudaEvent_t ev[HOST_STAGES] = {};
    int rc = FZ_OK;
    if (cudaHostGetDevicePointer(&dbase_v, base, 0) != cudaSuccess)
        rc = set_error(FZ_ECUDA, "cudaHostGetDevicePointer (staging buffers)");
    for (int j = 0; j < HOST_STAGES && rc == FZ_OK; ++j)
        if (cudaEventCreateWithFlags(&ev[j], cudaEventDisableTiming | cudaEventBlockingSync) !=
            cudaSuccess)
            rc = set_error(FZ_ECUDA, "cudaEventCreate");
    char *dbase = static_cast<char *>(dbase_v);

    std::mutex mu;
    std::condition_variable cv_work, cv_free;
    std::deque<CopyJob> jobs;
    int pending[HOST_STAGES] = {};
    bool stop = false;
    int worker_err = FZ_OK;
    std::vector<std::thread> workers;
    auto work = [&] {
        for (;;) {
            CopyJob job;
            {
                std::unique_lock<std::mutex> lk(mu);
                cv_work.wait(lk, [&] { return stop || !jobs.empty(); });
                if (jobs.empty()) return;
                job = jobs.front();
                jobs.pop_front();
            }
            const bool ok = cudaEventSynchronize(job.ev) == cudaSuccess;
            if (ok) std::memcpy(job.dst, job.src, job.bytes);
            {
                std::lock_guard<std::mutex> lk(mu);
                if (!ok && worker_err == FZ_OK) worker_err = FZ_ECUDA;
                if (--pending[job.stage] == 0 || !ok) cv_free.notify_all();
            }
        }
    };
    const int nthreads = host_copy_threads();
    if (rc == FZ_OK)
        for (int t = 0; t < nthreads; ++t) workers.emplace_back(work);

    DeviceProps dp;
    if (rc == FZ_OK) rc = device_props(&dp);
    EnumLaunch L = launch_of(p);
    L.plain_stores = true;
    uint64_t done = 0;
    for (uint64_t i = 0; rc == FZ_OK && done < rows; ++i) {
        const int j = (int)(i % HOST_STAGES);
        const uint64_t now = std::min(chunk_rows, rows - done);
        {
            std::unique_lock<std::mutex> lk(mu);
            cv_free.wait(lk, [&] { return pending[j] == 0 || worker_err != FZ_OK; });
            if (worker_err != FZ_OK) {
                rc = set_error(worker_err, "staging copy: event wait failed");
                break;
            }
        }
        const uint64_t slice = std::min<uint64_t>(p->slice_rows, default_slice_rows(now, dp.sms));
        rc = launch_enumerate(L, rank_begin + done, now,
                              reinterpret_cast<int32_t *>(dbase + (size_t)j * stage_bytes), slice,
                              s);
        if (rc != FZ_OK) break;
        if (cudaEventRecord(ev[j], s) != cudaSuccess) {
            rc = set_error(FZ_ECUDA, "cudaEventRecord");
            break;
        }
        // one job per worker, each a multiple of 4 KB (the last takes the rest)
        const size_t bytes = (size_t)now * d * 4;
        const char *src = base + (size_t)j * stage_bytes;
        char *dst = reinterpret_cast<char *>(out_host) + (size_t)done * d * 4;
        size_t part = (bytes + nthreads - 1) / nthreads;
        part = (part + 4095) & ~size_t(4095);
        if (part < (1u << 20)) part = 1u << 20;
        {
            std::lock_guard<std::mutex> lk(mu);
            for (size_t off = 0; off < bytes; off += part) {
                jobs.push_back({src + off, dst + off, std::min(part, bytes - off), j, ev[j]});
                pending[j]++;
            }
        }
        cv_work.notify_all();
        done += now;
    }
    {
        std::lock_guard<std::mutex> lk(mu);
        stop = true;
    }
    cv_work.notify_all();
    for (std::thread &t : workers) t.join();
    if (rc == FZ_OK && worker_err != FZ_OK)
        rc = set_error(worker_err, "staging copy: event wait failed");
    for (int j = 0; j < HOST_STAGES; ++j)
        if (ev[j]) cudaEventDestroy(ev[j]);
    if (own) cudaFreeHost(base);
    return rc;
}

}  // namespace

int plan_launch_for(fz_plan_t p, int32_t n, EnumLaunch *L) {
    if (!p || n < 0 || n > p->n) return set_error(FZ_EINVAL, "element outside the plan");
    *L = launch_of(p);
    L->n = n;  // tables have stride p->n + 1 and serve every n <= p->n
    return FZ_OK;
}

int plan_host_rows(fz_plan_t p, uint64_t *count_row, std::vector<uint64_t> *runs_row,
                   cudaStream_t s) {
    const size_t len = (size_t)p->n + 1;
    FZ_CUDA_TRY(cudaMemcpyAsync(count_row, p->C, len * 8, cudaMemcpyDeviceToHost, s));
    if (runs_row) {
        runs_row->clear();
        if (p->RT) {
            runs_row->resize(len);
            FZ_CUDA_TRY(cudaMemcpyAsync(runs_row->data(), p->RT, len * 8, cudaMemcpyDeviceToHost, s));
        }
    }
    FZ_CUDA_TRY(cudaStreamSynchronize(s));
    return FZ_OK;
}

}  // namespace fz

namespace fz {
namespace {
// Two blocks wait at the monotonic grid barrier for the arrivals of a grid
// ten times larger: the wait can only end by its time limit.
__global__ void bounded_wait_selftest_kernel(unsigned *count, int *status, uint64_t limit_ns) {
    grid_barrier_mono(count, 9u, status, limit_ns);
}
}  // namespace
}  // namespace fz

extern "C" {

int fz_version(void) { return 100; }

uint64_t fz_kernel_launches(void) { return fz::g_launches.load(std::memory_order_relaxed); }


int fz_selftest_bounded_wait(uint32_t limit_ms, int *status_seen, void *stream) {
    if (!status_seen) return fz::set_error(FZ_EINVAL, "status_seen: null pointer");
    if (limit_ms < 1 || limit_ms > 2000) return fz::set_error(FZ_EINVAL, "limit_ms must be 1..2000");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    void *buf = nullptr;
    if (cudaMalloc(&buf, 256) != cudaSuccess) {
        cudaGetLastError();
        return fz::set_error(FZ_ENOMEM, "self-test buffer");
    }
    unsigned *count = static_cast<unsigned *>(buf);
    int *status = reinterpret_cast<int *>(static_cast<char *>(buf) + 128);
    int rc = FZ_OK;
    if (cudaMemsetAsync(buf, 0, 256, s) != cudaSuccess) rc = fz::set_error(FZ_ECUDA, "memset");
    if (rc == FZ_OK) {
        fz::bounded_wait_selftest_kernel<<<2, 32, 0, s>>>(count, status,
                                                          (uint64_t)limit_ms * 1000000ull);
        fz::note_launch();
        if (cudaGetLastError() != cudaSuccess) rc = fz::set_error(FZ_ECUDA, "self-test launch");
    }
    int h = 0;
    if (rc == FZ_OK && (cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, s) !=
                            cudaSuccess ||
                        cudaStreamSynchronize(s) != cudaSuccess))
        rc = fz::set_error(FZ_ECUDA, "self-test status");
    cudaFree(buf);
    if (rc != FZ_OK) return rc;
    *status_seen = fz::status_to_fz(h);
    fz::set_error(FZ_OK, "");
    return FZ_OK;
}

int fz_write_probe(int32_t *out_dev, uint64_t words, void *stream) {
    if (words == 0) return FZ_OK;
    if (!out_dev || ((uintptr_t)out_dev & 15u) != 0)
        return fz::set_error(FZ_EINVAL, "write probe: null or unaligned output");
    int rc = fz::launch_write_probe(out_dev, words, static_cast<cudaStream_t>(stream));
    return rc;
}

const char *fz_last_error_string(void) { return fz::g_last_error.c_str(); }

const char *fz_status_string(int status) {
    switch (status) {
        case FZ_OK: return "FZ_OK";
        case FZ_EINVAL: return "FZ_EINVAL";
        case FZ_EOVERFLOW: return "FZ_EOVERFLOW";
        case FZ_ENOSPC: return "FZ_ENOSPC";
        case FZ_ENOMEM: return "FZ_ENOMEM";
        case FZ_EAGAIN: return "FZ_EAGAIN";
        case FZ_ETIMEOUT: return "FZ_ETIMEOUT";
        case FZ_ECUDA: return "FZ_ECUDA";
        case FZ_ENOTFOUND: return "FZ_ENOTFOUND";
        case FZ_EINTERNAL: return "FZ_EINTERNAL";
        case FZ_ECANCELED: return "FZ_ECANCELED";
        default: return "FZ_UNKNOWN";
    }
}

// ----------------------------------------------------------------- counting
int fz_count_upto(const int32_t *g, int d, int32_t n_max, uint64_t *counts, void *stream) {
    int rc = validate_gens(g, d);
    if (rc != FZ_OK) return rc;
    if (n_max < 0) return set_error(FZ_EINVAL, "n must be >= 0");
    if (!counts) return set_error(FZ_EINVAL, "counts: null pointer");
    cudaStream_t s = as_stream(stream);
    const int64_t len = (int64_t)n_max + 1;
    int64_t tmpw = count_table_tmp_words(g, d, n_max);
    DevBuf buf;
    rc = buf.alloc((size_t)(2 * len + tmpw) * 8);
    if (rc != FZ_OK) return rc;
    uint64_t *a = buf.as<uint64_t>(), *b = a + len, *tmp = b + len, *res = nullptr;
    rc = launch_count_rolling(g, d, n_max, a, b, tmp, &res, s);
    if (rc != FZ_OK) return rc;
    FZ_CUDA_TRY(cudaMemcpyAsync(counts, res, (size_t)len * 8, cudaMemcpyDeviceToHost, s));
    FZ_CUDA_TRY(cudaStreamSynchronize(s));
    return FZ_OK;
}

int fz_count(const int32_t *g, int d, int32_t n, uint64_t *count, void *stream) {
    int rc = validate_gens(g, d);
    if (rc != FZ_OK) return rc;
    if (n < 0) return set_error(FZ_EINVAL, "n must be >= 0");
    if (!count) return set_error(FZ_EINVAL, "count: null pointer");
    cudaStream_t s = as_stream(stream);
    const int64_t len = (int64_t)n + 1;
    int64_t tmpw = count_table_tmp_words(g, d, n);
    DevBuf buf;
    rc = buf.alloc((size_t)(2 * len + tmpw) * 8);
    if (rc != FZ_OK) return rc;
    uint64_t *a = buf.as<uint64_t>(), *b = a + len, *tmp = b + len, *res = nullptr;
    rc = launch_count_rolling(g, d, n, a, b, tmp, &res, s);
    if (rc != FZ_OK) return rc;
    uint64_t h = 0;
    FZ_CUDA_TRY(cudaMemcpyAsync(&h, res + n, 8, cudaMemcpyDeviceToHost, s));
    FZ_CUDA_TRY(cudaStreamSynchronize(s));
    *count = h;
    if (h == ~0ull) return set_error(FZ_EOVERFLOW, "|Z(n)| does not fit in 64 bits");
    return FZ_OK;
}

int fz_count_table(const int32_t *g, int d, int32_t n, uint64_t *table_dev, void *stream) {
    int rc = validate_gens(g, d);
    if (rc != FZ_OK) return rc;
    if (n < 0) return set_error(FZ_EINVAL, "n must be >= 0");
    if (!table_dev) return set_error(FZ_EINVAL, "table: null pointer");
    cudaStream_t s = as_stream(stream);
    int64_t tmpw = count_table_tmp_words(g, d, n);
    uint64_t *tmp = nullptr;
    if (tmpw > 0) FZ_CUDA_TRY(cudaMallocAsync((void **)&tmp, (size_t)tmpw * 8, s));
    rc = launch_count_table_tmp(g, d, n, table_dev, tmp, s);
    if (tmp) cudaFreeAsync(tmp, s);
    return rc;
}

// --------------------------------------------------------------------- memo
static int memo_common(const int32_t *tail, int k, int32_t top, cudaStream_t s, DevBuf &table,
                       uint64_t **C, int64_t *tmpw_out) {
    int rc = validate_gens(tail, k);
    if (rc != FZ_OK) return rc;
    if (top < 0) return set_error(FZ_EINVAL, "top must be >= 0");
    const int32_t n = top > 0 ? top - 1 : 0;
    const int64_t cs = (int64_t)n + 1;
    int64_t tmpw = std::max(count_table_tmp_words(tail, k, n), exclusive_scan_tmp_words(cs));
    rc = table.alloc((size_t)((k + 1) * cs + tmpw + 64) * 8);
    if (rc != FZ_OK) return rc;
    *C = table.as<uint64_t>();
    *tmpw_out = tmpw;
    rc = launch_count_table_tmp(tail, k, n, *C, *C + (k + 1) * cs, s);
    return rc;
}

int fz_memo_rows(const int32_t *tail, int k, int32_t top, uint64_t *rows, void *stream) {
    if (!rows) return set_error(FZ_EINVAL, "rows: null pointer");
    cudaStream_t s = as_stream(stream);
    if (top == 0) {
        int rc = validate_gens(tail, k);
        if (rc == FZ_OK) *rows = 0;
        return rc;
    }
    DevBuf table, off;
    uint64_t *C = nullptr;
    int64_t tmpw = 0;
    int rc = memo_common(tail, k, top, s, table, &C, &tmpw);
    if (rc != FZ_OK) return rc;
    rc = off.alloc((size_t)(top + 1) * 8);
    if (rc != FZ_OK) return rc;
    const int64_t cs = (int64_t)top;
    rc = launch_exclusive_scan_tmp(C, off.as<uint64_t>(), top, C + (k + 1) * cs, s);
    if (rc != FZ_OK) return rc;
    uint64_t h = 0;
    FZ_CUDA_TRY(cudaMemcpyAsync(&h, off.as<uint64_t>() + top, 8, cudaMemcpyDeviceToHost, s));
    FZ_CUDA_TRY(cudaStreamSynchronize(s));
    *rows = h;
    if (h == ~0ull) return set_error(FZ_EOVERFLOW, "memo rows do not fit in 64 bits");
    return FZ_OK;
}

static int build_memo_to(const int32_t *tail, int k, int32_t top, uint64_t *O, int32_t **R,
                         uint64_t rows_capacity, uint64_t *rows_needed, DevBuf *own_rows,
                         cudaStream_t s, int schedule = FZ_MEMO_BATCHED) {
    DevBuf table, work;
    uint64_t *C = nullptr;
    int64_t tmpw = 0;
    int rc = memo_common(tail, k, top, s, table, &C, &tmpw);
    if (rc != FZ_OK) return rc;
    const int64_t cs = (int64_t)top;
    uint64_t *tmp = C + (k + 1) * cs;
    rc = launch_exclusive_scan_tmp(C, O, top, tmp, s);
    if (rc != FZ_OK) return rc;
    uint64_t rows = 0;
    FZ_CUDA_TRY(cudaMemcpyAsync(&rows, O + top, 8, cudaMemcpyDeviceToHost, s));
    FZ_CUDA_TRY(cudaStreamSynchronize(s));
    if (rows_needed) *rows_needed = rows;
    if (rows == ~0ull) return set_error(FZ_EOVERFLOW, "memo rows do not fit in 64 bits");
    if (own_rows) {
        rc = own_rows->alloc(rows * (size_t)k * 4 + 16);
        if (rc != FZ_OK) return rc;
        *R = own_rows->as<int32_t>();
    } else if (rows > rows_capacity) {
        return set_error(FZ_ENOSPC, "memo rows exceed rows_capacity");
    }
    if (rows == 0) return FZ_OK;
    // gather map + status + barrier words
    const size_t map_bytes = align256(rows * 8);
    rc = work.alloc(map_bytes + 512);
    if (rc != FZ_OK) return rc;
    MemoBuffers mb;
    mb.Ct = C;
    mb.cs = cs;
    mb.O = O;
    mb.rows = *R;
    mb.map = work.as<uint64_t>();
    mb.status = reinterpret_cast<int *>(work.as<char>() + map_bytes);
    mb.bar = reinterpret_cast<unsigned *>(work.as<char>() + map_bytes + 256);
    FZ_CUDA_TRY(cudaMemsetAsync(work.as<char>() + map_bytes, 0, 512, s));
    rc = launch_memo_build(tail, k, top, rows, mb, s, schedule);
    if (rc != FZ_OK) return rc;
    return read_status(mb.status, s);
}

int fz_build_memo_into(const int32_t *tail, int k, int32_t top, uint64_t *offsets_dev,
                       int32_t *rows_dev, uint64_t rows_capacity, uint64_t *rows_needed,
                       void *stream) {
    return fz_build_memo_schedule(tail, k, top, FZ_MEMO_BATCHED, offsets_dev, rows_dev,
                                  rows_capacity, rows_needed, stream);
}

int fz_build_memo_schedule(const int32_t *tail, int k, int32_t top, int schedule,
                           uint64_t *offsets_dev, int32_t *rows_dev, uint64_t rows_capacity,
                           uint64_t *rows_needed, void *stream) {
    if (schedule != FZ_MEMO_BATCHED && schedule != FZ_MEMO_PER_BATCH &&
        schedule != FZ_MEMO_PER_COPY)
        return set_error(FZ_EINVAL, "unknown memo schedule");
    if (!offsets_dev || (!rows_dev && rows_capacity > 0))
        return set_error(FZ_EINVAL, "memo buffers: null pointer");
    if (top == 0) {
        int rc = validate_gens(tail, k);
        if (rc != FZ_OK) return rc;
        if (rows_needed) *rows_needed = 0;
        FZ_CUDA_TRY(cudaMemsetAsync(offsets_dev, 0, 8, as_stream(stream)));
        FZ_CUDA_TRY(cudaStreamSynchronize(as_stream(stream)));
        return FZ_OK;
    }
    int32_t *R = rows_dev;
    return build_memo_to(tail, k, top, offsets_dev, &R, rows_capacity, rows_needed, nullptr,
                         as_stream(stream), schedule);
}

int fz_build_memo(const int32_t *tail, int k, int32_t top, fz_memo_t *memo, void *stream) {
    if (!memo) return set_error(FZ_EINVAL, "memo: null pointer");
    int rc = validate_gens(tail, k);
    if (rc != FZ_OK) return rc;
    if (top < 0) return set_error(FZ_EINVAL, "top must be >= 0");
    fz_memo_s *m = new (std::nothrow) fz_memo_s;
    if (!m) return set_error(FZ_ENOMEM, "host allocation");
    m->k = k;
    m->top = top;
    cudaStream_t s = as_stream(stream);
    rc = m->buf.alloc((size_t)(top + 1) * 8);
    if (rc == FZ_OK) {
        m->O = m->buf.as<uint64_t>();
        if (top == 0) {
            if (cudaMemsetAsync(m->O, 0, 8, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess)
                rc = set_error(FZ_ECUDA, "memset");
        } else {
            rc = build_memo_to(tail, k, top, m->O, &m->R, 0, &m->rows, &m->rows_buf, s);
        }
    }
    if (rc != FZ_OK) {
        delete m;
        return rc;
    }
    *memo = m;
    return FZ_OK;
}

int fz_memo_info(fz_memo_t memo, fz_memo_info_t *info) {
    if (!memo || !info) return set_error(FZ_EINVAL, "null pointer");
    info->k = memo->k;
    info->top = memo->top;
    info->rows = memo->rows;
    info->offsets_dev = memo->O;
    info->rows_dev = memo->R;
    return FZ_OK;
}

int fz_memo_release(fz_memo_t memo) {
    if (!memo) return set_error(FZ_EINVAL, "null pointer");
    delete memo;
    return FZ_OK;
}

// ----------------------------------------------------------------- tuning
// One timed pass of a plan: its rebuild (count tables + memo), then the
// enumeration of ranks [0, rows) in windows of at most `wrows` rows, all
// written to the same buffer (each window a full launch over the GPU).
static int time_pass(fz_plan_t p, int32_t *buf, uint64_t wrows, uint64_t rows, cudaStream_t s,
                     double *build_ms, double *enum_ms) {
    cudaEvent_t e0, e1, e2;
    FZ_CUDA_TRY(cudaEventCreate(&e0));
    FZ_CUDA_TRY(cudaEventCreate(&e1));
    FZ_CUDA_TRY(cudaEventCreate(&e2));
    cudaEventRecord(e0, s);
    int rc = fz_plan_rebuild(p, s);
    cudaEventRecord(e1, s);
    for (uint64_t b = 0; b < rows && rc == FZ_OK; b += wrows) {
        uint64_t got = 0;
        const uint64_t e = std::min(rows, b + wrows);
        rc = fz_plan_enumerate(p, b, e, buf, wrows, &got, s);
    }
    cudaEventRecord(e2, s);
    if (rc == FZ_OK) rc = fz_plan_sync(p, s);
    float b_ms = 0, en_ms = 0;
    cudaEventElapsedTime(&b_ms, e0, e1);
    cudaEventElapsedTime(&en_ms, e1, e2);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaEventDestroy(e2);
    *build_ms = b_ms;
    *enum_ms = en_ms;
    return rc;
}

int fz_autotune_report(const int32_t *g, int d, int32_t n, fz_tune_entry_t *entries,
                       int capacity, int *n_entries, fz_opts_t *best, double *best_ms,
                       void *stream) {
    if (!best) return set_error(FZ_EINVAL, "best: null pointer");
    if (capacity < 0 || (capacity > 0 && !entries))
        return set_error(FZ_EINVAL, "entries: null pointer");
    if (n_entries) *n_entries = 0;
    cudaStream_t s = as_stream(stream);
    // the heuristic plan gives the count and the first depth to try
    fz_plan_t p0 = nullptr;
    fz_opts_t o0{FZ_AUTO, FZ_AUTO, 0, 0};
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune.erase(tune_key(g, d, n));
    }
    int rc = fz_plan_create(g, d, n, &o0, &p0, stream);
    if (rc != FZ_OK) return rc;
    const uint64_t count = p0->count;
    const int k0 = p0->K;
    fz_plan_destroy(p0);
    *best = fz_opts_t{k0, FZ_AUTO, 0, 0};
    if (best_ms) *best_ms = 0;
    if (count == 0 || d == 1) return FZ_OK;
    // Candidates are timed on the whole set: a sample of small windows
    // leaves most warps idle and favours small work items.  The output goes
    // to one scratch buffer of the whole set when it fits in a third of the
    // free device memory, else to windows of that size.
    size_t fr = 0, tot = 0;
    FZ_CUDA_TRY(cudaMemGetInfo(&fr, &tot));
    uint64_t wrows = std::min<uint64_t>(count, (uint64_t)(fr / 3) / (4ull * d));
    wrows = std::max<uint64_t>(32, wrows & ~31ull);
    DevBuf buf;
    rc = buf.alloc(wrows * (size_t)d * 4 + 256);
    if (rc != FZ_OK) return rc;
    double best_t = 1e300;
    fz_opts_t best_o = *best;
    int found = 0;
    // the size rule's depth first (a good time early lets slow candidates
    // be screened out after one pass), then every other depth that fits
    std::vector<int> ks{k0};
    for (int k = std::min(d - 1, 4); k >= 0; --k)
        if (k != k0) ks.push_back(k);
    for (int k : ks) {
        fz_opts_t o{k, FZ_AUTO, 0, 0};
        fz_plan_t p = nullptr;
        if (fz_plan_create(g, d, n, &o, &p, stream) != FZ_OK) {  // memo too large
            cudaGetLastError();
            continue;
        }
        if (p->memo_rows * (uint64_t)(4 * k + 8) > std::max<uint64_t>(64ull << 20, count * d)) {
            fz_plan_destroy(p);
            continue;
        }
        const uint64_t base_slice = p->slice_rows;
        for (uint64_t sl : {base_slice, base_slice / 2, base_slice * 2}) {
            if (sl < 1024) continue;
            p->slice_rows = (sl + 31) & ~31ull;
            // screening pass (also the warm-up): one window, scaled to the set
            double b_ms = 0, e_ms = 0;
            const uint64_t first = std::min(count, wrows);
            rc = time_pass(p, buf.as<int32_t>(), wrows, first, s, &b_ms, &e_ms);
            if (rc != FZ_OK) {
                fz_plan_destroy(p);
                return rc;
            }
            const double screen = b_ms + e_ms * (double)count / (double)first;
            double t = screen, bsum = 0, esum = 0;
            const bool hopeless = best_t < 1e300 && screen > 4.0 * best_t;
            if (!hopeless) {
                for (int rep = 0; rep < 2 && rc == FZ_OK; ++rep) {
                    rc = time_pass(p, buf.as<int32_t>(), wrows, count, s, &b_ms, &e_ms);
                    bsum += b_ms;
                    esum += e_ms;
                }
                if (rc != FZ_OK) {
                    fz_plan_destroy(p);
                    return rc;
                }
                t = (bsum + esum) / 2;
            }
            if (found < capacity) {
                fz_tune_entry_t &E = entries[found];
                E.k = k;
                E.slice_rows = (int32_t)p->slice_rows;
                E.run_order = p->run_memo ? 1 : 0;
                E.screened_out = hopeless ? 1 : 0;
                E.memo_rows = p->memo_rows;
                E.build_ms = hopeless ? b_ms : bsum / 2;
                E.enum_ms = hopeless ? e_ms * (double)count / (double)first : esum / 2;
                E.total_ms = t;
            }
            ++found;
            if (!hopeless && t < best_t) {
                best_t = t;
                best_o = fz_opts_t{k, FZ_AUTO, (int32_t)p->slice_rows, 0};
            }
            if (hopeless) break;  // other work-item sizes will not rescue this depth
        }
        fz_plan_destroy(p);
    }
    if (n_entries) *n_entries = std::min(found, capacity);
    *best = best_o;
    if (best_ms) *best_ms = best_t;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[tune_key(g, d, n)] = best_o;
    return FZ_OK;
}

int fz_autotune(const int32_t *g, int d, int32_t n, fz_opts_t *best, double *best_ms,
                void *stream) {
    return fz_autotune_report(g, d, n, nullptr, 0, nullptr, best, best_ms, stream);
}

// -------------------------------------------------------------------- plans
int fz_plan_create(const int32_t *g, int d, int32_t n, const fz_opts_t *opt, fz_plan_t *plan,
                   void *stream) {
    if (!plan) return set_error(FZ_EINVAL, "plan: null pointer");
    fz_plan_s *p = new (std::nothrow) fz_plan_s;
    if (!p) return set_error(FZ_ENOMEM, "host allocation");
    int rc = plan_create_impl(g, d, n, opt, p, as_stream(stream));
    if (rc != FZ_OK) {
        cudaStreamSynchronize(as_stream(stream));
        delete p;
        return rc;
    }
    *plan = p;
    return FZ_OK;
}

int fz_plan_info(fz_plan_t p, fz_plan_info_t *info) {
    if (!p || !info) return set_error(FZ_EINVAL, "null pointer");
    info->count = p->count;
    info->d = p->d;
    info->n = p->n;
    info->k = p->K;
    info->top = p->top;
    info->memo_rows = p->memo_rows;
    info->device_bytes = p->base.bytes + p->memo.bytes + p->runs.bytes;
    info->slice_rows = (int32_t)p->slice_rows;
    info->run_order = p->run_memo ? 1 : 0;
    return FZ_OK;
}

int fz_plan_set_enum_ctas_per_sm(fz_plan_t p, int32_t ctas) {
    if (!p) return set_error(FZ_EINVAL, "plan: null pointer");
    if (ctas < 0) return set_error(FZ_EINVAL, "ctas must be >= 0");
    p->ctas_per_sm = ctas;
    return FZ_OK;
}

int fz_plan_rebuild(fz_plan_t p, void *stream) {
    if (!p) return set_error(FZ_EINVAL, "plan: null pointer");
    cudaStream_t s = as_stream(stream);
    int rc = launch_count_table_tmp(p->g, p->d, p->n, p->C, p->tmp, s);
    if (rc != FZ_OK) return rc;
    if (p->RT) {
        rc = launch_runs_table(p->g, p->lam_r, p->n, p->RT, p->tmp, p->clamp_row, p->top, s);
        if (rc != FZ_OK) return rc;
    }
    return plan_enqueue_memo(p, s);
}

int fz_plan_enumerate(fz_plan_t p, uint64_t rank_begin, uint64_t rank_end, int32_t *out_dev,
                      uint64_t out_capacity_rows, uint64_t *written, void *stream) {
    if (!p) return set_error(FZ_EINVAL, "plan: null pointer");
    const uint64_t rows = rows_in(p, rank_begin, rank_end);
    if (written) *written = rows;
    if (rows == 0) return FZ_OK;
    if (!out_dev) return set_error(FZ_EINVAL, "out: null pointer");
    if (((uintptr_t)out_dev & 3u) != 0) return set_error(FZ_EINVAL, "out must be 4-byte aligned");
    if (out_capacity_rows < rows) return set_error(FZ_ENOSPC, "output capacity too small");
    return launch_enumerate(launch_of(p), rank_begin, rows, out_dev, p->slice_rows,
                            as_stream(stream));
}

int fz_plan_unrank(fz_plan_t p, const uint64_t *ranks_dev, uint64_t m, int32_t *out_dev,
                   void *stream) {
    if (!p) return set_error(FZ_EINVAL, "plan: null pointer");
    if (m == 0) return FZ_OK;
    if (!ranks_dev || !out_dev) return set_error(FZ_EINVAL, "null pointer");
    return launch_unrank(launch_of(p), ranks_dev, m, out_dev, as_stream(stream));
}

int fz_plan_sync(fz_plan_t p, void *stream) {
    if (!p) return set_error(FZ_EINVAL, "plan: null pointer");
    cudaStream_t s = as_stream(stream);
    FZ_CUDA_TRY(cudaStreamSynchronize(s));
    return read_status(p->status, s);
}

int fz_plan_destroy(fz_plan_t p) {
    if (!p) return set_error(FZ_EINVAL, "plan: null pointer");
    delete p;
    return FZ_OK;
}

// ---------------------------------------------------------------- one-shot
int fz_enumerate(const int32_t *g, int d, int32_t n, const fz_opts_t *opt, uint64_t rank_begin,
                 uint64_t rank_end, int32_t *out_dev, uint64_t out_capacity_rows,
                 uint64_t *written, void *stream) {
    fz_plan_t p = nullptr;
    int rc = fz_plan_create(g, d, n, opt, &p, stream);
    if (rc != FZ_OK) return rc;
    rc = fz_plan_enumerate(p, rank_begin, rank_end, out_dev, out_capacity_rows, written, stream);
    if (rc == FZ_OK) rc = fz_plan_sync(p, stream);
    fz_plan_destroy(p);
    return rc;
}

int fz_enumerate_host(const int32_t *g, int d, int32_t n, const fz_opts_t *opt,
                      uint64_t rank_begin, uint64_t rank_end, int32_t *out_host,
                      uint64_t out_capacity_rows, uint64_t *written, void *stream) {
    return fz_enumerate_host_chunks(g, d, n, opt, rank_begin, rank_end, out_host,
                                    out_capacity_rows, 0, written, stream);
}

int fz_enumerate_host_chunks(const int32_t *g, int d, int32_t n, const fz_opts_t *opt,
                             uint64_t rank_begin, uint64_t rank_end, int32_t *out_host,
                             uint64_t out_capacity_rows, uint64_t chunk_rows,
                             uint64_t *written, void *stream) {
    fz_plan_t p = nullptr;
    int rc = fz_plan_create(g, d, n, opt, &p, stream);
    if (rc != FZ_OK) return rc;
    const uint64_t rows = rows_in(p, rank_begin, rank_end);
    if (written) *written = rows;
    if (rows > 0 && !out_host) rc = set_error(FZ_EINVAL, "out: null pointer");
    if (rc == FZ_OK && out_capacity_rows < rows)
        rc = set_error(FZ_ENOSPC, "output capacity too small");
    if (rc != FZ_OK || rows == 0) {
        fz_plan_destroy(p);
        return rc;
    }
    cudaStream_t s = as_stream(stream);
    // Pinned (page-locked, mapped) host memory is written by the kernel
    // itself over the host link: no staging buffer, no copy.
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, out_host) == cudaSuccess &&
        attr.type == cudaMemoryTypeHost && attr.devicePointer) {
        EnumLaunch L = launch_of(p);
        L.plain_stores = true;
        rc = launch_enumerate(L, rank_begin, rows, static_cast<int32_t *>(attr.devicePointer),
                              p->slice_rows, s);
        if (rc == FZ_OK) rc = fz_plan_sync(p, stream);
        fz_plan_destroy(p);
        return rc;
    }
    cudaGetLastError();  // pageable memory: the query above may have set an error
    // Devices that reach pageable host memory through the host's own page
    // tables (address translation services over a coherent link, as on
    // Grace-Blackwell) are written directly by the kernel, as pinned memory
    // is; elsewhere, or when a chunk size is asked for, the rows go through
    // the staging ring.
    if (chunk_rows == 0 && pageable_direct_ok()) {
        EnumLaunch L = launch_of(p);
        L.plain_stores = true;
        rc = launch_enumerate(L, rank_begin, rows, out_host, p->slice_rows, s);
        if (rc == FZ_OK) rc = fz_plan_sync(p, stream);
        fz_plan_destroy(p);
        return rc;
    }
    rc = stream_to_pageable(p, rank_begin, rows, out_host, chunk_rows, s);
    const int rc2 = fz_plan_sync(p, stream);
    if (rc == FZ_OK) rc = rc2;
    fz_plan_destroy(p);
    return rc;
}

}  // extern "C"
