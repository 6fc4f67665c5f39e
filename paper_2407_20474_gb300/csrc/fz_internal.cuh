// fz_internal.cuh -- device helpers and host utilities shared by the fz
// library's translation units (count DP, memo build, enumeration, C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "../../include/fz.h"
#include "fz_host_math.h"

namespace fz {

constexpr unsigned FULL = 0xffffffffu;
constexpr uint64_t SAT = ~0ull;

// ---------------------------------------------------------------------------
// Error reporting (host).  The message is thread-local; see fz_api.cu.
// ---------------------------------------------------------------------------
int set_error(int status, const std::string &msg);
// Count one kernel launch (fz_kernel_launches).
void note_launch();
int cuda_error(cudaError_t e, const char *what);
#define FZ_CUDA_TRY(expr)                                   \
    do {                                                    \
        cudaError_t fz_e_ = (expr);                         \
        if (fz_e_ != cudaSuccess) return ::fz::cuda_error(fz_e_, #expr); \
    } while (0)

// Device-side status codes written into a per-handle status word.
enum DevStatus : int {
    DEV_OK = 0,
    DEV_TIMEOUT = 1,    // a bounded wait gave up
    DEV_INTERNAL = 2,   // a consistency check failed
};

// ---------------------------------------------------------------------------
// Saturating 64-bit arithmetic and warp scans.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t sat_add(uint64_t a, uint64_t b) {
    uint64_t s = a + b;
    return s < a ? SAT : s;
}

__device__ __forceinline__ uint64_t shfl_u64(uint64_t v, int src) {
    return __shfl_sync(FULL, v, src);
}

// Inclusive warp scan with saturation (min(sum, 2^64-1) is associative).
__device__ __forceinline__ uint64_t warp_incl_scan_sat(uint64_t v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint64_t t = __shfl_up_sync(FULL, v, o);
        if (lane >= o) v = sat_add(v, t);
    }
    return v;
}

__device__ __forceinline__ uint64_t warp_incl_scan(uint64_t v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint64_t t = __shfl_up_sync(FULL, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// ---------------------------------------------------------------------------
// Memory-model helpers.
// ---------------------------------------------------------------------------
// L2-only load (bypasses L1, which is not coherent with writes made by other
// SMs during the same kernel).
__device__ __forceinline__ int32_t ld_cg_s32(const int32_t *p) {
    int32_t v;
    asm volatile("ld.global.cg.s32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

__device__ __forceinline__ uint64_t ld_cg_u64(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.global.cg.u64 %0, [%1];" : "=l"(v) : "l"(p));
    return v;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u32(unsigned *p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ---------------------------------------------------------------------------
// Bulk (TMA) stores from shared to global memory.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Makes this thread's generic-proxy writes to shared memory visible to the
// async proxy (the bulk copy engine).
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// dst and src 16-byte aligned, bytes a positive multiple of 16.
__device__ __forceinline__ void bulk_store(void *gdst, const void *ssrc, uint32_t bytes,
                                           uint64_t pol) {
    asm volatile(
        "cp.async.bulk.global.shared::cta.bulk_group.L2::cache_hint [%0], [%1], %2, %3;" ::"l"(
            gdst),
        "r"(smem_addr(ssrc)), "r"(bytes), "l"(pol)
        : "memory");
}

__device__ __forceinline__ void bulk_commit() {
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

// Wait until every committed bulk group of this thread has finished reading
// its shared-memory source.
__device__ __forceinline__ void bulk_wait_read_all() {
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

// Wait until at most N of this thread's committed bulk groups are still
// reading their shared-memory source.
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
    asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}

// Wait until every committed bulk group of this thread has completed.
__device__ __forceinline__ void bulk_wait_all() {
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// Limits of every bounded device-side wait.
constexpr uint64_t BARRIER_TIMEOUT_NS = 2000000000ull;  // 2 s
constexpr uint32_t BARRIER_MAX_POLLS = 1u << 26;

// ---------------------------------------------------------------------------
// Bounded monotonic grid barrier for cooperative launches: *count (zeroed
// before the launch) counts arrivals; the i-th barrier (i = 0, 1, ...)
// completes when it reaches (i + 1) * gridDim.  One atomic and one poll per
// barrier.  A block whose wait runs past the limit records DEV_TIMEOUT and
// returns false (the others then time out too, each on its own).
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool grid_barrier_mono(unsigned *count, unsigned index, int *status,
                                                  uint64_t timeout_ns = BARRIER_TIMEOUT_NS) {
    __shared__ int ok_flag_m;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned target = (index + 1u) * (gridDim.x * gridDim.y * gridDim.z);
        // release-add: the block's writes (ordered before this thread by the
        // __syncthreads above) are visible to whoever acquires the count
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(count) : "memory");
        uint64_t t0 = 0;
        uint32_t polls = 0;
        while (ld_acquire_u32(count) < target) {
            if (polls == 0) t0 = globaltimer_ns();
            if (++polls >= BARRIER_MAX_POLLS ||
                ((polls & 255u) == 0 && globaltimer_ns() - t0 > timeout_ns)) {
                atomicExch(status, (int)DEV_TIMEOUT);
                ok = 0;
                break;
            }
            __nanosleep(20);
        }
        ok_flag_m = ok;
    }
    __syncthreads();
    return ok_flag_m != 0;
}


// The two halves of grid_barrier_mono, for a block that has work needing no
// other block's writes to do between them: grid_arrive releases the block's
// writes (ordered before thread 0 by the __syncthreads) with one add to the
// count; grid_wait polls (thread 0, bounded like grid_barrier_mono) until
// the count reaches (index + 1) x blocks, then orders the block after it.
__device__ __forceinline__ void grid_arrive(unsigned *count) {
    __syncthreads();
    if (threadIdx.x == 0)
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(count) : "memory");
}

__device__ __forceinline__ bool grid_wait(unsigned *count, unsigned index, int *status,
                                          uint64_t timeout_ns = BARRIER_TIMEOUT_NS) {
    __shared__ int ok_flag_w;
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned target = (index + 1u) * (gridDim.x * gridDim.y * gridDim.z);
        uint64_t t0 = 0;
        uint32_t polls = 0;
        while (ld_acquire_u32(count) < target) {
            if (polls == 0) t0 = globaltimer_ns();
            if (++polls >= BARRIER_MAX_POLLS ||
                ((polls & 255u) == 0 && globaltimer_ns() - t0 > timeout_ns)) {
                atomicExch(status, (int)DEV_TIMEOUT);
                ok = 0;
                break;
            }
            __nanosleep(20);
        }
        ok_flag_w = ok;
    }
    __syncthreads();
    return ok_flag_w != 0;
}

// ---------------------------------------------------------------------------
// Host helpers.
// ---------------------------------------------------------------------------
// Per-device flags for host-side steps done once per kernel and device
// (function attributes), safe when several host threads launch: the
// serving thread and its callers.
struct DeviceOnce {
    std::atomic<bool> done[64];
    bool is_set(int dev) const {
        return dev >= 0 && dev < 64 && done[dev].load(std::memory_order_acquire);
    }
    void set(int dev) {
        if (dev >= 0 && dev < 64) done[dev].store(true, std::memory_order_release);
    }
};

struct DeviceProps {
    int device = -1;
    int sms = 0;
    int max_smem_optin = 0;
};
int device_props(DeviceProps *out);

int validate_gens(const int32_t *g, int d);

// Count DP (fz_count.cu).  Writes C[j][r], j = 0..d, r = 0..n, row stride
// n + 1, into table (device), using `tmp` (count_table_tmp_words words) as
// scratch.  Asynchronous; saturates at 2^64 - 1.
int64_t count_table_tmp_words(const int32_t *g, int d, int32_t n);
int launch_count_table_tmp(const int32_t *g, int d, int32_t n, uint64_t *table, uint64_t *tmp,
                           cudaStream_t s);
// Only row 0 (|Z(r, g)|, r = 0..n) with two rolling rows a, b (n + 1 words
// each); returns which of them holds the result.
int launch_count_rolling(const int32_t *g, int d, int32_t n, uint64_t *a, uint64_t *b,
                         uint64_t *tmp, uint64_t **result, cudaStream_t s);

// Batched strided scans (fz_count.cu): one row per job, CTA tasks per launch.
struct ScanJob {
    const uint64_t *in;  // row below (scan input)
    uint64_t *out;       // row to write
    int64_t len;         // entries in the row
    int64_t g;           // stride
    uint64_t *S;         // block sums (blocked jobs), else null
    uint64_t *Sincl;     // their strided inclusive scan
    int64_t slen;        // entries of S
    int64_t ones_below;  // entries r < ones_below of out are written as 1
    // strided view: logical entry r of in/out is entry off + r * es (es = 0
    // means 1); the one chain of a row that is ever read
    // TK_PAIR: out = row d-2 of a count table, out + len = row d-1 (written
    // only when ones_below != 0), for the last two generators g (= this g)
    // and h, e = gcd(g, h), h1 = h / e, g1 = g / e, inv = g1^-1 mod h1 (0 when
    // h1 = 1)
    int64_t h, e, h1, g1, inv;
    int64_t off, es;
    // entries per block of a blocked scan (0: scan_block_rows()); long
    // chains take larger blocks so their chains of block sums stay within
    // the direct-scan limit
    int64_t rb;
};
enum ScanTaskKind : int {
    TK_DIRECT = 0,  // chains [begin, end) of in -> out, one warp each
    TK_BSUM = 1,    // block sums S[begin..end)
    TK_SSCAN = 2,   // chains [begin, end) of S -> Sincl
    TK_APPLY = 3,   // blocks [begin, end): out = carry + running sum
    TK_DELTA = 4,   // out[begin..end) = [i == 0]
    TK_ONES = 5,    // out[begin..end) = 1
    TK_PAIR = 6,    // rows d-2 and d-1 of a count table in closed form
    TK_LINEAR = 7,  // out[x] = x / g + 1 (a runs-table row above the ones row)
    TK_LANES = 8    // chains [begin, end) of in -> out, 32 neighbouring chains a warp
};
struct ScanTask {
    int job;
    int kind;
    int64_t begin, end;
};
int launch_scan_tasks(const ScanJob *jobs, const ScanTask *tasks, int ntasks, cudaStream_t s);
int64_t scan_direct_limit();  // chains up to this length are scanned directly
int64_t scan_lane_limit();    // chains up to this length, 32 or more of them: a lane each
int64_t scan_blocks_per_task();  // block sums a TK_BSUM / TK_APPLY task covers
int scan_block_rows();        // entries per block of a blocked scan

// out[0] = 0, out[r + 1] = in[0] + ... + in[r] for r < len (saturating).
int64_t exclusive_scan_tmp_words(int64_t len);
int launch_exclusive_scan_tmp(const uint64_t *in, uint64_t *out, int64_t len, uint64_t *tmp,
                              cudaStream_t s);

// Memo build (fz_memo.cu).
struct MemoBuffers {
    const uint64_t *Ct = nullptr;  // count table rows 0..k of the tail, stride cs
    int64_t cs = 0;
    const uint64_t *O = nullptr;   // top + 1 offsets (already scanned)
    uint64_t *map = nullptr;       // rows entries (gather map)
    int32_t *rows = nullptr;       // rows * k
    int *status = nullptr;         // device status word
    unsigned *bar = nullptr;       // grid-barrier arrival count (zeroed before each fill)
    bool small_ctas = false;       // fill with small CTAs (beside a capped enumeration)
};
// Memo of depth 1 or 2 written in closed form from its offsets O (one warp
// per element; no gather map, no batches).  Asynchronous.
int launch_memo_closed(const int32_t *tail, int k, int32_t top, const uint64_t *O,
                       int32_t *rows, int *status, cudaStream_t s);
// Gather map + batched copy-and-increment fill.  Asynchronous.
// schedule: FZ_MEMO_BATCHED (one launch), FZ_MEMO_PER_BATCH or FZ_MEMO_PER_COPY.
int launch_memo_build(const int32_t *tail, int k, int32_t top, uint64_t rows,
                      const MemoBuffers &mb, cudaStream_t s, int schedule = FZ_MEMO_BATCHED);
// Many small memos, one CTA each (fz_memo.cu).
struct MemoJob {
    const uint64_t *Ct;  // tail count table rows 0..k, stride cs (row 0: |Z(r, tail)|)
    int64_t cs;
    uint64_t *O;         // top + 1 offsets (written by the build)
    int32_t *R;          // rows * k int32
    uint64_t rows;       // expected row count (consistency check)
    int top, k, b;
    int t[FZ_MAX_D];
};
int launch_memo_sizes(const MemoJob *jobs, int njobs, uint64_t *rows_out, cudaStream_t s);

// The memo of a full plan (tail = g_{lam+1}..g_{d-1}, every element 0..n) in
// run order: the rows of the elements p = c, c + g_lam, c + 2 g_lam, ... of
// each residue class c mod g_lam, classes in increasing order, each row as
// int4 (p div g_lam, its k <= 3 memo words, zero padding).  For a prefix
// with remainder r at level lam, the rows of its whole subtree over a_lam are
// then the contiguous range [cls_beg[r mod g_lam], + C[lam][r]), and a_lam =
// r div g_lam - (first word).  cls_beg: G = min(g_lam, n + 1) class starts.
int launch_run_memo(const uint64_t *C, int64_t cs, int lam, int32_t n, int32_t g_lam,
                    const uint64_t *O, const int32_t *rows, int k, uint64_t memo_rows,
                    uint64_t *cls_beg, int4 *run_memo, int *status, cudaStream_t s);
// The memos of a batch, one per job (jobs sorted longest first): the first
// ncoop jobs each by a thread-block cluster, the rest one per CTA (claim: a
// device counter the launch zeroes).  memo_coop_count picks ncoop (0: the
// one-CTA launch for every job).
int memo_coop_count(const MemoJob *sorted, int njobs);
int launch_memo_cta_build(const MemoJob *jobs, int njobs, int ncoop, unsigned *claim,
                          int *status, cudaStream_t s);

// One run-order memo of a batch (the layout of launch_run_memo) for the
// elements 0..n: its rows come from an element-order memo of depth k <= 3
// (O, rows), or, with O null, from the closed form of the tail: k = 1, the
// one row p / ta when ta divides p (ta = g_{d-1}); k = 2, the pair (t0, t1)
// = (g_{d-2}, g_{d-1}), whose rows for element p have a_{d-2} = a_top - o h1
// (o = 0, 1, ...) as in launch_memo_closed.
struct RunJob {
    const uint64_t *Clam;   // count-table row lam of the source instance, n + 1 entries
    const uint64_t *Cnext;  // row lam + 1: |Z(p, tail)|
    const uint64_t *O;      // element-order memo offsets, or null (closed form)
    const int32_t *rows;    // element-order memo rows (k int32 each), or null
    uint64_t *cls_beg;      // G + 1 class starts
    int4 *out;              // run-order rows
    uint64_t out_rows;      // capacity of out (bounds guard)
    uint64_t expect_rows;   // closed form: sum over p <= n of |Z(p, tail)|
    int32_t n, g, G, k;     // last element, g_lam, G = min(g_lam, n + 1), depth
    int64_t t0, t1, e, h1, inv;
    int64_t ta;             // closed form, k = 1: the tail's generator
    uint64_t blk0;          // first block of this job in the row kernel
};
// Builds every job's class starts, then its rows: `blocks` blocks of 256
// threads, job j owning ceil((n_j + 1) / 256) of them from blk0 on (zero
// skips the launch).
int launch_run_memo_batch(const RunJob *jobs, int njobs, uint64_t blocks, int *status,
                          cudaStream_t s);

// out[w] = w for w < words, 16-byte stores (fz_write_probe; fz_count.cu).
int launch_write_probe(int32_t *out, uint64_t words, cudaStream_t s);

// Enumeration (fz_enum.cu).
// Walk leaves are produced as a progression (FZ_WALK_PROGRESSION != 0).
bool walk_progression_enabled();

// Work balancing: the level lam_r whose prefixes the candidates table counts
// and the cost W of one such prefix in rows, for an instance of d generators
// with memo depth K and top (top > n: full memo); run_order: the memo is kept
// in run order.  Walk runs (the last two coordinates as a progression) and
// run-order runs cost a chain of dependent loads each (W = 64); memo leaves
// and candidates evaluated 32 at a time cost W = 16.
// *clamp_row >= 0: the table row whose entries below top are set to 1 (a
// memo leaf is one unit, whatever lies under it), else -1.
bool run_memo_enabled();
void balance_level(int d, int K, int top, int n, bool run_order, int *lam_r, uint64_t *W,
                   int *clamp_row);

struct EnumLaunch {
    const uint64_t *C = nullptr;   // count table rows 0..d, stride cs = n + 1
    int64_t cs = 0;
    const uint64_t *O = nullptr;   // memo offsets
    const int32_t *memo = nullptr; // memo rows
    uint64_t memo_rows = 0;
    int *status = nullptr;
    unsigned long long *slice_counter = nullptr;
    int n = 0, d = 0, K = 0, top = 0;
    const int32_t *g = nullptr;    // host generators
    // work-balanced slicing (optional): runs table rows 0..lam_r, the cost of
    // one run in rows, and the totals over the whole set
    const uint64_t *RT = nullptr;
    uint64_t W = 0;
    int lam_r = 0;
    uint64_t total_cost = 0, total_rows = 0;
    // the output is host memory reached over the host link: flush rows with
    // plain coalesced stores instead of bulk (TMA) stores
    bool plain_stores = false;
    // at most this many CTAs of the enumeration kernel per SM (0 = as many as
    // fit), leaving room for other kernels to run beside it
    int ctas_per_sm = 0;
    // full memo of depth K <= 3 in run order (see launch_run_memo), or null
    const int4 *run_memo = nullptr;
    const uint64_t *cls_beg = nullptr;
    // K == 2, full: the memo is the closed form of Z(p, (g_{d-2}, g_{d-1}))
    // (no table; O and memo may be null)
    bool pair_memo = false;
};
// Runs table: RT[lam][x] = 1, RT[j][x] = sum_t RT[j+1][x - t g_j]
// (fz_count.cu); if clamp_row >= 0, RT[clamp_row][x] = 1 for x < clamp_top
// (before the rows above it are summed).
int launch_runs_table(const int32_t *g, int lam, int32_t n, uint64_t *RT, uint64_t *tmp,
                      int clamp_row, int64_t clamp_top,
                      cudaStream_t s);
int launch_enumerate(const EnumLaunch &L, uint64_t rank_begin, uint64_t nrows, int32_t *out,
                     uint64_t slice_rows, cudaStream_t s);
int launch_unrank(const EnumLaunch &L, const uint64_t *ranks, uint64_t m, int32_t *out,
                  cudaStream_t s);
uint64_t default_slice_rows(uint64_t nrows, int sms);
// Batched enumeration (fz_enum.cu): per-instance parameter images, then one
// persistent launch over all work items.
size_t enum_params_bytes();
void fill_batch_params(const EnumLaunch &L, int32_t *out, uint64_t count, uint64_t slice_rows,
                       uint64_t slice_cost, void *dst);
int launch_enumerate_batch(const void *params_dev, const uint64_t *item0_dev, int count,
                           uint64_t nitems, unsigned long long *item_counter, int32_t *out_base,
                           cudaStream_t s, int ctas_per_sm = 0);

// Plans as seen by the batch and serve layers (fz_api.cu): the launch
// description of a plan for an element n <= its n, and host copies of row 0
// of its count table (n + 1 entries) and runs table (empty if none).
int plan_launch_for(fz_plan_t plan, int32_t n, EnumLaunch *L);
int plan_host_rows(fz_plan_t plan, uint64_t *count_row, std::vector<uint64_t> *runs_row,
                   cudaStream_t s);

// Largest memo the library builds (rows); keeps memo row indices in 32 bits.
constexpr uint64_t MEMO_MAX_ROWS = 1ull << 30;

}  // namespace fz
