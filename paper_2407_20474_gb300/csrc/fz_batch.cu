// fz_batch.cu -- many instances Z(n_i, g_i) in one set of launches.
//
// A batch keeps, for every instance, its count table and runs table (for
// work-balanced slicing) and, per distinct tail, one memo shared by the
// instances with that tail.  A rebuild is: one initialisation launch and
// three launches per table level for all instances' tables together (the
// batched strided scans of fz_count.cu), then one launch that builds every
// memo (one CTA per memo, the elementwise dynamic pass of Section 2).  The
// enumeration is one persistent launch over (instance, slice) work items
// (fz_enum.cu).  Everything after creation is asynchronous, so a rebuild plus
// an enumeration can be captured in a CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "fz_internal.cuh"

namespace fz {
namespace {

struct DevArena {
    void *p = nullptr;
    size_t bytes = 0;
    ~DevArena() {
        if (p) cudaFree(p);
    }
    int alloc(size_t b) {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
        if (b == 0) b = 256;
        cudaError_t e = cudaMalloc(&p, b);
        if (e != cudaSuccess) {
            p = nullptr;
            return cuda_error(e, "cudaMalloc (batch)");
        }
        bytes = b;
        return FZ_OK;
    }
};

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

// Elementwise batches a batch memo may take (its top is cut to this many
// batches of min(tail) elements; larger remainders take the ordinary step).
// FZ_BATCH_MEMO_BATCHES=b overrides it (tuning only).
int64_t batch_memo_batches() {
    static const int64_t v = [] {
        const char *e = getenv("FZ_BATCH_MEMO_BATCHES");
        const long long x = e ? atoll(e) : 0;
        return x >= 16 && x <= 65536 ? (int64_t)x : (int64_t)512;
    }();
    return v;
}
constexpr double BATCH_MEMO_MAX_ROWS = 1 << 20;

struct Inst {
    int d = 0, n = 0, K = 0, top = 0, lam_r = 0, clamp_row = -1;
    bool pair = false;  // K = 2 kept as the closed form (no memo table)
    bool run = false;   // full memo copied in run order (RunJob run_job)
    int run_job = -1;
    const int4 *run_memo = nullptr;
    const uint64_t *cls_beg = nullptr;
    uint64_t run_rows = 0;
    int32_t g[FZ_MAX_D] = {};
    size_t off_C = 0, off_RT = 0;  // word offsets into the table arena
    int memo = -1;                 // memo job index
    uint64_t count = 0, runs = 0;
    uint64_t W = 16;  // cost of one prefix counted by the runs table, in rows
    uint64_t word_off = 0;
    uint64_t items = 0, slice_cost = 0, slice_rows = 0;
};

}  // namespace
}  // namespace fz

using namespace fz;

struct fz_batch_s {
    int count = 0;
    std::vector<Inst> inst;
    DevArena tables;   // all count and runs tables
    DevArena scratch;  // block sums of blocked scans
    DevArena memos;    // memo offsets and rows
    DevArena meta;     // jobs, tasks, memo jobs, params, item prefix, counters
    DevArena runs;     // run-order memos: jobs, rows, class starts
    // scan launches: (first task, number of tasks) per launch, in order
    std::vector<std::pair<int, int>> scan_launches;
    ScanJob *jobs_dev = nullptr;
    ScanTask *tasks_dev = nullptr;
    MemoJob *memo_jobs_dev = nullptr;
    int nmemo = 0;
    int memo_ncoop = 0;              // memos built by a cluster
    unsigned *memo_claim = nullptr;  // claim counter of the memo build
    std::vector<MemoJob> memo_jobs;
    RunJob *run_jobs_dev = nullptr;
    int nrun = 0, run_inst = 0;
    uint64_t run_blocks = 0;  // blocks of the run-row kernel
    int ctas_per_sm = 0;      // cap of the enumeration kernel (0: as many as fit)
    void *params_dev = nullptr;       // EnumParams images (out = word offset)
    uint64_t *item0_dev = nullptr;
    unsigned long long *counter_dev = nullptr;
    int *status_dev = nullptr;
    uint64_t nitems = 0;
    uint64_t total_rows = 0, total_words = 0;
    std::vector<unsigned char> params_host;
};

namespace fz {
namespace {

// Row 0 of an instance's count and runs tables is only ever read along the
// chain n, n - g_1, n - 2 g_1, ... (unranking, the walk at the first
// coordinate, the costs and the totals): its jobs cover that chain alone,
// as a strided view of n div g_1 + 1 entries.  For d = 3 with the pair memo
// the same holds for row 1, which only feeds row 0's chain.
void chain_view(ScanJob &J, const Inst &I) {
    J.off = I.n % I.g[0];
    J.es = I.g[0];
    J.len = I.n / I.g[0] + 1;
}

int build_scan_plan(fz_batch_s *b, uint64_t *table_base, std::vector<ScanJob> &jobs,
                    std::vector<ScanTask> &tasks, size_t *scratch_words) {
    const int64_t DIRECT = scan_direct_limit();
    const int64_t LANE_LIMIT = scan_lane_limit();
    const int64_t BS_TASK = scan_blocks_per_task();
    const int RBk = scan_block_rows();
    int maxlev = 0;
    for (const Inst &I : b->inst) maxlev = std::max(maxlev, std::max(I.d, I.lam_r));
    // Initialisation launch.  Rows nothing reads are not written (the poison
    // fill of a new arena would turn a wrong omission into an error): the
    // delta row C[d] (it only fed the scan of C[d-1], now closed form),
    // C[d-1] unless a memo is built from this table or the candidates table
    // is counted at level d - 1, and the runs table's ones row RT[lam_r] when
    // the row above it is closed form.
    {
        const int first = (int)tasks.size();
        for (const Inst &I : b->inst) {
            const int64_t len = (int64_t)I.n + 1;
            if (I.d < 2) {
                ScanJob jd{};
                jd.out = table_base + I.off_C + (size_t)I.d * len;
                jd.len = len;
                jobs.push_back(jd);
                for (int64_t a = 0; a < len; a += 8192)
                    tasks.push_back({(int)jobs.size() - 1, TK_DELTA, a, std::min(len, a + 8192)});
            } else {
                // rows d-2 and d-1 in closed form (no scans)
                ScanJob jp{};
                jp.out = table_base + I.off_C + (size_t)(I.d - 2) * len;
                jp.len = len;
                jp.g = I.g[I.d - 2];
                jp.h = I.g[I.d - 1];
                // row d-1 is read by a memo build from this table, or as the
                // leaf row of a candidates table counted at level d - 1
                jp.ones_below = ((I.K > 0 && !I.pair) || I.lam_r >= I.d - 1) ? 1 : 0;
                pair_params(jp.g, jp.h, &jp.e, &jp.h1, &jp.g1, &jp.inv);
                if (!jp.ones_below && (I.d == 2 || (I.d == 3 && I.pair))) chain_view(jp, I);
                jobs.push_back(jp);
                for (int64_t a = 0; a < jp.len; a += 8192)
                    tasks.push_back(
                        {(int)jobs.size() - 1, TK_PAIR, a, std::min(jp.len, a + 8192)});
            }
            if (I.lam_r >= 0 && I.off_RT != (size_t)-1) {
                if (I.lam_r == 0) {
                    ScanJob jo{};
                    jo.out = table_base + I.off_RT + (size_t)I.lam_r * len;
                    jo.len = len;
                    jobs.push_back(jo);
                    for (int64_t a = 0; a < len; a += 8192)
                        tasks.push_back(
                            {(int)jobs.size() - 1, TK_ONES, a, std::min(len, a + 8192)});
                }
                if (I.lam_r >= 1) {
                    // the row above the ones row: x / g + 1
                    ScanJob jl{};
                    const int j = I.lam_r - 1;
                    jl.out = table_base + I.off_RT + (size_t)j * len;
                    jl.len = len;
                    jl.g = I.g[j];
                    if (j == I.clamp_row) jl.ones_below = I.top;
                    if (j == 0) chain_view(jl, I);
                    jobs.push_back(jl);
                    for (int64_t a = 0; a < jl.len; a += 8192)
                        tasks.push_back(
                            {(int)jobs.size() - 1, TK_LINEAR, a, std::min(jl.len, a + 8192)});
                }
            }
        }
        b->scan_launches.push_back({first, (int)tasks.size() - first});
    }
    size_t max_scratch = 0;
    for (int t = 0; t < maxlev; ++t) {
        // jobs of this level: count row d-1-t (from d-3 on), runs row lam_r-2-t
        std::vector<int> step_jobs;
        for (const Inst &I : b->inst) {
            const int64_t len = (int64_t)I.n + 1;
            if (I.d > t && (I.d < 2 || I.d - 1 - t < I.d - 2)) {  // rows d-2, d-1: closed form
                const int j = I.d - 1 - t;
                ScanJob J{};
                J.in = table_base + I.off_C + (size_t)(j + 1) * len;
                J.out = table_base + I.off_C + (size_t)j * len;
                J.len = len;
                J.g = I.g[j];
                if (j == 0) {
                    chain_view(J, I);
                    J.g = 1;  // consecutive entries of the chain
                }
                jobs.push_back(J);
                step_jobs.push_back((int)jobs.size() - 1);
            }
            if (I.off_RT != (size_t)-1 && I.lam_r > t + 1) {
                // rows lam_r - 2, lam_r - 3, ..., 0 (lam_r and lam_r - 1 are
                // written in closed form by the initialisation launch)
                const int j = I.lam_r - 2 - t;
                ScanJob J{};
                J.in = table_base + I.off_RT + (size_t)(j + 1) * len;
                J.out = table_base + I.off_RT + (size_t)j * len;
                J.len = len;
                J.g = I.g[j];
                if (j == I.clamp_row) J.ones_below = I.top;
                if (j == 0) {
                    chain_view(J, I);
                    J.g = 1;
                }
                jobs.push_back(J);
                step_jobs.push_back((int)jobs.size() - 1);
            }
        }
        // scratch for blocked jobs of this level (reused by every level)
        size_t sw = 0;
        for (int ji : step_jobs) {
            ScanJob &J = jobs[ji];
            const int64_t T = (J.len + J.g - 1) / J.g;
            if (T > DIRECT) {
                // blocks of at least RBk entries, more for long chains, so
                // that each chain of block sums is scanned directly
                J.rb = std::max<int64_t>(RBk, (T + DIRECT - 1) / DIRECT);
                const int64_t nrb = (T + J.rb - 1) / J.rb;
                J.slen = nrb * J.g;
                J.S = reinterpret_cast<uint64_t *>(sw);  // offset, fixed up below
                J.Sincl = reinterpret_cast<uint64_t *>(sw + (size_t)J.slen);
                sw += 2 * (size_t)J.slen;
            }
        }
        max_scratch = std::max(max_scratch, sw);
        int first = (int)tasks.size();
        for (int ji : step_jobs) {
            const ScanJob &J = jobs[ji];
            if (!J.slen) {
                const int64_t chains = std::min<int64_t>(J.g, J.len);
                const int64_t T = (J.len + J.g - 1) / J.g;
                if (chains >= 32 && T <= LANE_LIMIT) {
                    // 256 chains a task, one a lane
                    for (int64_t a = 0; a < chains; a += 256)
                        tasks.push_back({ji, TK_LANES, a, std::min(chains, a + 256)});
                } else {
                    for (int64_t a = 0; a < chains; a += 8)
                        tasks.push_back({ji, TK_DIRECT, a, std::min(chains, a + 8)});
                }
            } else {
                // one block sum a thread: a block is rb strided entries
                for (int64_t a = 0; a < J.slen; a += BS_TASK)
                    tasks.push_back({ji, TK_BSUM, a, std::min(J.slen, a + BS_TASK)});
            }
        }
        b->scan_launches.push_back({first, (int)tasks.size() - first});
        first = (int)tasks.size();
        for (int ji : step_jobs) {
            const ScanJob &J = jobs[ji];
            if (J.slen)
                for (int64_t a = 0; a < J.g; a += 8)
                    tasks.push_back({ji, TK_SSCAN, a, std::min<int64_t>(J.g, a + 8)});
        }
        b->scan_launches.push_back({first, (int)tasks.size() - first});
        first = (int)tasks.size();
        for (int ji : step_jobs) {
            const ScanJob &J = jobs[ji];
            if (J.slen)
                for (int64_t a = 0; a < J.slen; a += BS_TASK)
                    tasks.push_back({ji, TK_APPLY, a, std::min(J.slen, a + BS_TASK)});
        }
        b->scan_launches.push_back({first, (int)tasks.size() - first});
    }
    *scratch_words = max_scratch;
    return FZ_OK;
}

int batch_enqueue_rebuild(fz_batch_s *b, cudaStream_t s) {
    for (const auto &L : b->scan_launches) {
        int rc = launch_scan_tasks(b->jobs_dev, b->tasks_dev + L.first, L.second, s);
        if (rc != FZ_OK) return rc;
    }
    int rc = launch_memo_cta_build(b->memo_jobs_dev, b->nmemo, b->memo_ncoop, b->memo_claim,
                                   b->status_dev, s);
    if (rc != FZ_OK) return rc;
    return launch_run_memo_batch(b->run_jobs_dev, b->nrun, b->run_blocks, b->status_dev, s);
}

__global__ void gather_kernel(const uint64_t *const *ptrs, uint64_t *out, int count) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) out[i] = ptrs[i] ? *ptrs[i] : 0ull;
}

int gather(const std::vector<const uint64_t *> &ptrs, std::vector<uint64_t> &out,
           cudaStream_t s) {
    const int count = (int)ptrs.size();
    out.assign(count, 0);
    if (!count) return FZ_OK;
    DevArena tmp;
    int rc = tmp.alloc(a256((size_t)count * 8) * 2);
    if (rc != FZ_OK) return rc;
    const uint64_t **dp = static_cast<const uint64_t **>(tmp.p);
    uint64_t *dv = reinterpret_cast<uint64_t *>(static_cast<char *>(tmp.p) + a256((size_t)count * 8));
    FZ_CUDA_TRY(cudaMemcpyAsync(dp, ptrs.data(), (size_t)count * 8, cudaMemcpyHostToDevice, s));
    gather_kernel<<<(count + 255) / 256, 256, 0, s>>>(dp, dv, count);
    note_launch();
    FZ_CUDA_TRY(cudaGetLastError());
    FZ_CUDA_TRY(cudaMemcpyAsync(out.data(), dv, (size_t)count * 8, cudaMemcpyDeviceToHost, s));
    FZ_CUDA_TRY(cudaStreamSynchronize(s));
    return FZ_OK;
}

// Memo depth of a batch instance, chosen for the largest element n_set
// asked of the same generators in the batch (so instances of one generator
// set share one memo).  A memo's rows are estimated by the volume
// top^K / (K! prod tail), with top = min(n_set + 1, batch_memo_batches()
// elementwise batches of min(tail) elements).  Preferred: the deepest full
// memo (top > n_set) of depth >= 3 within BATCH_MEMO_MAX_ROWS rows and
// cap_rows times the instance's estimated rows (volume n^(d-1) / ((d-1)!
// prod g)) -- the deeper the memo, the fewer prefixes the walk visits.  Otherwise, for
// d >= 5, a partial memo of depth 3 within BATCH_MEMO_MAX_ROWS rows (the
// pair memo's leaves, prefixes of length d - 2, would be mostly empty
// there: the d = 5 instances of a 4096-instance batch took 11.3 ms with it,
// 2 ms with depth
// 3).  Otherwise the pair memo: depth 2, full, as the closed form of
// Z(p, (g_{d-2}, g_{d-1})) -- no table to build, and its leaves are
// evaluated 32 at a time.
// Estimated |Z(n, g)|: the volume n^(d-1) / ((d-1)! prod g).
double volume_rows(const Inst &I, int n) {
    double count = 1.0 / (double)I.g[I.d - 1];
    for (int i = 0; i < I.d - 1; ++i) count *= (double)n / (double)(i + 1) / (double)I.g[i];
    return count;
}

// Run-order memos of the pair's closed form are kept within this many times
// the instance's estimated rows: they cost 16 bytes a row, built in one
// fully parallel pass, and replace memo leaves of one to three rows that
// cost about 12 warp instructions per output row.
constexpr double RUN_PAIR_CAP = 2.0;

// FZ_BATCH_ORDER=0 numbers the work items in the caller's instance order
// (tuning only; see the item numbering in batch_create_impl).
bool batch_item_order_enabled() {
    static const bool on = [] {
        const char *e = getenv("FZ_BATCH_ORDER");
        return !(e && e[0] == '0');
    }();
    return on;
}

// How a batch chooses memos, per tuple width d: the memo rows allowed per
// estimated instance row (cap_rows, see choose_batch_memo) and whether full
// memos of depth <= 3 are also kept in run order.  The defaults are the
// hand-set rule; fz_batch_autotune replaces them per device by the fastest
// measured candidates.
struct BatchPolicy {
    double cap_rows[FZ_MAX_D + 1];
    bool run_order[FZ_MAX_D + 1];
};

BatchPolicy default_policy() {
    BatchPolicy P;
    for (int d = 0; d <= FZ_MAX_D; ++d) {
        // the batch walk pays per memo leaf, so deeper memos (fewer, larger
        // leaves) repaid their build at d >= 6 up to ~4x the instance's rows
        // (4096 mixed instances: d = 6..8 enumeration 11.9 -> 4.1 ms for
        // 1.6 ms more build); at d <= 5 they did not
        P.cap_rows[d] = d >= 6 ? 4.0 : 1.0;
        P.run_order[d] = true;
    }
    return P;
}

std::mutex g_policy_mu;
std::map<int, BatchPolicy> g_policy;  // by device ordinal, set by fz_batch_autotune

BatchPolicy current_policy() {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_policy_mu);
    auto it = g_policy.find(dev);
    return it == g_policy.end() ? default_policy() : it->second;
}

void choose_batch_memo(Inst &I, int n_set, double cap_rows) {
    I.K = 0;
    I.top = 0;
    I.pair = false;
    if (I.d < 3) return;
    double count = 1.0 / (double)I.g[I.d - 1];
    for (int i = 0; i < I.d - 1; ++i) count *= (double)n_set / (double)(i + 1) / (double)I.g[i];
    int64_t part_top = 0;
    for (int k = I.d - 1; k >= 3; --k) {
        int32_t tmin = I.g[I.d - k];
        double prod = 1.0;
        for (int i = I.d - k; i < I.d; ++i) {
            tmin = std::min(tmin, I.g[i]);
            prod *= I.g[i];
        }
        const int64_t top = std::min<int64_t>((int64_t)n_set + 1, batch_memo_batches() * tmin);
        double rows = 1.0;
        for (int i = 0; i < k; ++i) rows *= (double)top / (i + 1);
        rows /= prod;
        if (rows > BATCH_MEMO_MAX_ROWS) continue;
        if (top > n_set && rows <= cap_rows * count + 4096.0) {
            I.K = k;
            I.top = (int)std::min<int64_t>((int64_t)I.n + 1, top);
            return;
        }
        if (k == 3 && I.d >= 5) part_top = top;
    }
    if (part_top > 0) {
        I.K = 3;
        I.top = (int)std::min<int64_t>((int64_t)I.n + 1, part_top);
        return;
    }
    I.K = 2;
    I.top = I.n + 1;
    I.pair = true;
}

}  // namespace
}  // namespace fz

extern "C" {

namespace fz {
namespace {

int batch_create_impl(const fz_instance_t *inst, int count, const fz_opts_t *opt,
                      const BatchPolicy &pol, fz_batch_t *batch, cudaStream_t s);

}  // namespace
}  // namespace fz

int fz_batch_create(const fz_instance_t *inst, int count, const fz_opts_t *opt,
                    fz_batch_t *batch, void *stream) {
    return batch_create_impl(inst, count, opt, current_policy(), batch,
                             static_cast<cudaStream_t>(stream));
}

}  // extern "C"

namespace fz {
namespace {

int batch_create_impl(const fz_instance_t *inst, int count, const fz_opts_t *opt,
                      const BatchPolicy &pol, fz_batch_t *batch, cudaStream_t s) {
    if (!batch) return set_error(FZ_EINVAL, "batch: null pointer");
    if (count < 0 || (count > 0 && !inst)) return set_error(FZ_EINVAL, "instances");
    if (opt && opt->flags != 0) return set_error(FZ_EINVAL, "opts.flags must be 0");
    fz_batch_s *b = new (std::nothrow) fz_batch_s;
    if (!b) return set_error(FZ_ENOMEM, "host allocation");
    auto fail = [&](int rc) {
        cudaStreamSynchronize(s);
        delete b;
        return rc;
    };
    b->count = count;
    b->inst.resize(count);
    size_t words = 0;
    // largest element asked of each generator set (memo depth per set)
    std::map<std::vector<int32_t>, int> n_set;
    for (int i = 0; i < count; ++i) {
        if (inst[i].d < 1 || inst[i].d > FZ_MAX_D || !inst[i].g) continue;  // validated below
        std::vector<int32_t> key(inst[i].g, inst[i].g + inst[i].d);
        int &m = n_set[key];
        m = std::max(m, inst[i].n);
    }
    for (int i = 0; i < count; ++i) {
        const fz_instance_t &x = inst[i];
        int rc = validate_gens(x.g, x.d);
        if (rc != FZ_OK) return fail(rc);
        if (x.n < 0) return fail(set_error(FZ_EINVAL, "n must be >= 0"));
        Inst &I = b->inst[i];
        I.d = x.d;
        I.n = x.n;
        for (int j = 0; j < x.d; ++j) I.g[j] = x.g[j];
        choose_batch_memo(I, n_set[std::vector<int32_t>(x.g, x.g + x.d)], pol.cap_rows[x.d]);
        if (opt && opt->k != FZ_AUTO) {
            if (opt->k < 0 || opt->k > x.d - 1)
                return fail(set_error(FZ_EINVAL, "opts.k must be in 0..d-1 for every instance"));
            I.pair = false;
            I.K = opt->k;
            int32_t tmin = I.K ? I.g[I.d - I.K] : 1;
            for (int j = I.d - I.K; j < I.d; ++j) tmin = std::min(tmin, I.g[j]);
            I.top = I.K ? (int)std::min<int64_t>((int64_t)I.n + 1, batch_memo_batches() * tmin) : 0;
        }
        if (opt && opt->top != FZ_AUTO && I.K > 0) {
            I.top = std::min(I.top, opt->top);
            if (I.top <= I.n) I.pair = false;  // a partial memo is a table
        }
        if (I.K > 0 && I.top <= 0) I.K = 0;
        if (I.K == 0) I.top = 0;
        // run order: a full memo of depth 1..3 under at least one walked
        // coordinate, width <= 8 (the batch walk's run copy); the pair's
        // closed form gets a run-order table when that stays small
        I.run = false;
        if (run_memo_enabled() && pol.run_order[I.d] && I.K >= 1 && I.K <= 3 && I.top > I.n &&
            I.d <= 8 &&
            I.d - I.K - 1 >= 1) {
            if (!I.pair) {
                I.run = true;
            } else {
                const int ns = n_set[std::vector<int32_t>(x.g, x.g + x.d)];
                const int64_t t0 = I.g[I.d - 2], t1 = I.g[I.d - 1];
                if ((int64_t)ns / t0 < (int64_t)BATCH_MEMO_MAX_ROWS) {
                    const double rows = (double)pair_rows_upto(ns, t0, t1);
                    I.run = rows <= BATCH_MEMO_MAX_ROWS &&
                            rows <= RUN_PAIR_CAP * volume_rows(I, ns) + 4096.0;
                }
            }
        }
        const size_t len = (size_t)I.n + 1;
        I.off_C = words;
        words += (size_t)(I.d + 1) * len;
        I.off_RT = (size_t)-1;
        if (I.d >= 2) {
            balance_level(I.d, I.K, I.top, I.n, I.run, &I.lam_r, &I.W, &I.clamp_row);
            I.off_RT = words;
            words += (size_t)(I.lam_r + 1) * len;
        } else {
            I.lam_r = -1;
        }
    }
    int rc = b->tables.alloc(words * 8);
    if (rc != FZ_OK) return fail(rc);
    uint64_t *tb = static_cast<uint64_t *>(b->tables.p);
    // every table entry is written by each rebuild; poison them first so an
    // entry the build missed shows up as an error instead of stale zeros
    FZ_CUDA_TRY(cudaMemsetAsync(tb, 0xff, words * 8, s));

    std::vector<ScanJob> jobs;
    std::vector<ScanTask> tasks;
    size_t scratch_words = 0;
    rc = build_scan_plan(b, tb, jobs, tasks, &scratch_words);
    if (rc != FZ_OK) return fail(rc);
    rc = b->scratch.alloc(scratch_words * 8);
    if (rc != FZ_OK) return fail(rc);
    for (ScanJob &J : jobs) {
        if (J.slen) {
            J.S = static_cast<uint64_t *>(b->scratch.p) + reinterpret_cast<size_t>(J.S);
            J.Sincl = static_cast<uint64_t *>(b->scratch.p) + reinterpret_cast<size_t>(J.Sincl);
        }
    }

    // memo jobs, one per distinct (tail, k); top = the largest asked for
    std::map<std::vector<int32_t>, int> memo_of;
    std::vector<std::vector<int32_t>> memo_tail;
    std::vector<int> memo_src;  // instance whose table rows feed the memo
    for (int i = 0; i < count; ++i) {
        Inst &I = b->inst[i];
        // run-order instances of depth 1 and 2 take their rows from the
        // tail's closed form: no element-order memo
        if (I.K <= 0 || I.pair || (I.run && I.K <= 2)) continue;
        std::vector<int32_t> key(I.g + (I.d - I.K), I.g + I.d);
        auto it = memo_of.find(key);
        int m;
        if (it == memo_of.end()) {
            m = (int)b->memo_jobs.size();
            memo_of[key] = m;
            memo_tail.push_back(key);
            memo_src.push_back(i);
            MemoJob J{};
            J.k = I.K;
            J.top = I.top;
            b->memo_jobs.push_back(J);
        } else {
            m = it->second;
            if (I.top > b->memo_jobs[m].top) b->memo_jobs[m].top = I.top;
            if (I.n > b->inst[memo_src[m]].n) memo_src[m] = i;
        }
        I.memo = m;
    }
    b->nmemo = (int)b->memo_jobs.size();
    for (int m = 0; m < b->nmemo; ++m) {
        MemoJob &J = b->memo_jobs[m];
        const Inst &S = b->inst[memo_src[m]];
        J.Ct = tb + S.off_C + (size_t)(S.d - J.k) * ((size_t)S.n + 1);
        J.cs = (int64_t)S.n + 1;
        int32_t tmin = memo_tail[m][0];
        for (int c = 0; c < J.k; ++c) {
            J.t[c] = memo_tail[m][c];
            tmin = std::min(tmin, J.t[c]);
        }
        J.b = tmin;
        if (J.top > S.n + 1) J.top = S.n + 1;
    }

    // metadata arena: jobs, tasks, memo jobs, params, item prefix, counters
    const size_t pbytes = enum_params_bytes();
    const size_t o_jobs = 0;
    const size_t o_tasks = a256(o_jobs + jobs.size() * sizeof(ScanJob));
    const size_t o_mjobs = a256(o_tasks + tasks.size() * sizeof(ScanTask));
    const size_t o_params = a256(o_mjobs + (size_t)b->nmemo * sizeof(MemoJob));
    const size_t o_item0 = a256(o_params + (size_t)count * pbytes);
    const size_t o_misc = a256(o_item0 + ((size_t)count + 1) * 8);
    const size_t o_mrows = a256(o_misc + 256);
    rc = b->meta.alloc(a256(o_mrows + (size_t)b->nmemo * 8) + 256);
    if (rc != FZ_OK) return fail(rc);
    char *mb = static_cast<char *>(b->meta.p);
    b->jobs_dev = reinterpret_cast<ScanJob *>(mb + o_jobs);
    b->tasks_dev = reinterpret_cast<ScanTask *>(mb + o_tasks);
    b->memo_jobs_dev = reinterpret_cast<MemoJob *>(mb + o_mjobs);
    b->params_dev = mb + o_params;
    b->item0_dev = reinterpret_cast<uint64_t *>(mb + o_item0);
    b->counter_dev = reinterpret_cast<unsigned long long *>(mb + o_misc);
    b->status_dev = reinterpret_cast<int *>(mb + o_misc + 64);
    b->memo_claim = reinterpret_cast<unsigned *>(mb + o_misc + 128);
    uint64_t *mrows_dev = reinterpret_cast<uint64_t *>(mb + o_mrows);
    FZ_CUDA_TRY(cudaMemsetAsync(mb + o_misc, 0, 256, s));
    if (!jobs.empty())
        FZ_CUDA_TRY(cudaMemcpyAsync(b->jobs_dev, jobs.data(), jobs.size() * sizeof(ScanJob),
                                    cudaMemcpyHostToDevice, s));
    if (!tasks.empty())
        FZ_CUDA_TRY(cudaMemcpyAsync(b->tasks_dev, tasks.data(), tasks.size() * sizeof(ScanTask),
                                    cudaMemcpyHostToDevice, s));
    // count and runs tables
    for (const auto &L : b->scan_launches) {
        rc = launch_scan_tasks(b->jobs_dev, b->tasks_dev + L.first, L.second, s);
        if (rc != FZ_OK) return fail(rc);
    }
    // memo sizes, then allocation and build
    std::vector<uint64_t> mrows(b->nmemo, 0);
    if (b->nmemo) {
        FZ_CUDA_TRY(cudaMemcpyAsync(b->memo_jobs_dev, b->memo_jobs.data(),
                                    b->memo_jobs.size() * sizeof(MemoJob),
                                    cudaMemcpyHostToDevice, s));
        rc = launch_memo_sizes(b->memo_jobs_dev, b->nmemo, mrows_dev, s);
        if (rc != FZ_OK) return fail(rc);
        FZ_CUDA_TRY(cudaMemcpyAsync(mrows.data(), mrows_dev, (size_t)b->nmemo * 8,
                                    cudaMemcpyDeviceToHost, s));
        FZ_CUDA_TRY(cudaStreamSynchronize(s));
        size_t mwords = 0;
        for (int m = 0; m < b->nmemo; ++m) {
            if (mrows[m] > MEMO_MAX_ROWS) return fail(set_error(FZ_EINVAL, "batch memo too large"));
            mwords += a256(((size_t)b->memo_jobs[m].top + 1) * 8) / 8;
            mwords += a256((size_t)mrows[m] * b->memo_jobs[m].k * 4 + 16) / 8;
        }
        rc = b->memos.alloc(mwords * 8);
        if (rc != FZ_OK) return fail(rc);
        char *base = static_cast<char *>(b->memos.p);
        size_t off = 0;
        for (int m = 0; m < b->nmemo; ++m) {
            MemoJob &J = b->memo_jobs[m];
            J.O = reinterpret_cast<uint64_t *>(base + off);
            off += a256(((size_t)J.top + 1) * 8);
            J.R = reinterpret_cast<int32_t *>(base + off);
            off += a256((size_t)mrows[m] * J.k * 4 + 16);
            J.rows = mrows[m];
        }
        // the build launches one CTA per memo in job order and far more memos
        // than fit on the GPU at once: longest first (rows copied plus a
        // barrier's worth per elementwise batch), so the long ones start in
        // the first wave and the short ones fill in behind them
        std::vector<MemoJob> by_work(b->memo_jobs);
        auto work = [](const MemoJob &J) {
            const double nbatch = ((double)J.top + J.b - 1) / (double)J.b;
            return (double)J.rows * J.k + 4096.0 * nbatch;
        };
        std::stable_sort(by_work.begin(), by_work.end(),
                         [&](const MemoJob &x, const MemoJob &y) { return work(x) > work(y); });
        FZ_CUDA_TRY(cudaMemcpyAsync(b->memo_jobs_dev, by_work.data(),
                                    by_work.size() * sizeof(MemoJob), cudaMemcpyHostToDevice, s));
        FZ_CUDA_TRY(cudaStreamSynchronize(s));  // by_work is a host temporary
        b->memo_ncoop = memo_coop_count(by_work.data(), b->nmemo);
        rc = launch_memo_cta_build(b->memo_jobs_dev, b->nmemo, b->memo_ncoop, b->memo_claim,
                                   b->status_dev, s);
        if (rc != FZ_OK) return fail(rc);
    }
    // run-order memos, one per distinct (g_lam, tail) and source (memo or
    // closed form), built for the largest element asked of it
    {
        std::map<std::vector<int32_t>, int> run_of;
        std::vector<int> run_src;
        for (int i = 0; i < count; ++i) {
            Inst &I = b->inst[i];
            if (!I.run) continue;
            std::vector<int32_t> key(I.g + (I.d - I.K - 1), I.g + I.d);
            key.push_back(I.pair ? -1 : I.K);
            auto it = run_of.find(key);
            if (it == run_of.end()) {
                I.run_job = (int)run_src.size();
                run_of[key] = I.run_job;
                run_src.push_back(i);
            } else {
                I.run_job = it->second;
                if (I.n > b->inst[run_src[I.run_job]].n) run_src[I.run_job] = i;
            }
            ++b->run_inst;
        }
        b->nrun = (int)run_src.size();
        std::vector<RunJob> rj(b->nrun);
        size_t bytes = a256((size_t)b->nrun * sizeof(RunJob));
        for (int j = 0; j < b->nrun; ++j) {
            const Inst &S = b->inst[run_src[j]];
            RunJob &R = rj[j];
            const int lam = S.d - S.K - 1;
            const size_t len = (size_t)S.n + 1;
            R.Clam = tb + S.off_C + (size_t)lam * len;
            R.Cnext = tb + S.off_C + (size_t)(lam + 1) * len;
            R.n = S.n;
            R.g = S.g[lam];
            R.G = (int32_t)std::min<int64_t>(R.g, (int64_t)S.n + 1);
            R.k = S.K;
            // depth 1 and 2: the tail's closed form (k = 1, one row when ta
            // divides p; k = 2, the pair (t0, t1)); depth 3: rows copied from
            // the element-order memo
            if (S.K == 2) {
                R.t0 = S.g[S.d - 2];
                R.t1 = S.g[S.d - 1];
                int64_t g1;
                pair_params(R.t0, R.t1, &R.e, &R.h1, &g1, &R.inv);
                R.expect_rows = pair_rows_upto(S.n, R.t0, R.t1);
            } else if (S.K == 1) {
                R.ta = S.g[S.d - 1];
                R.expect_rows = (uint64_t)(S.n / R.ta) + 1;
            } else if (S.K == 3) {
                if (S.memo < 0 || b->memo_jobs[S.memo].top < S.n + 1)
                    return fail(set_error(FZ_EINTERNAL, "run-order memo without its full memo"));
                const MemoJob &M = b->memo_jobs[S.memo];
                R.O = M.O;
                R.rows = M.R;
                R.expect_rows = M.rows;
            } else {
                return fail(set_error(FZ_EINTERNAL, "run-order memo of depth > 3"));
            }
            R.out_rows = R.expect_rows;
            if (R.out_rows > MEMO_MAX_ROWS)
                return fail(set_error(FZ_EINVAL, "batch run-order memo too large"));
            bytes += a256((size_t)R.out_rows * 16 + 16) + a256(((size_t)R.G + 1) * 8);
        }
        if (b->nrun) {
            rc = b->runs.alloc(bytes);
            if (rc != FZ_OK) return fail(rc);
            char *base = static_cast<char *>(b->runs.p);
            size_t off = a256((size_t)b->nrun * sizeof(RunJob));
            for (RunJob &R : rj) {
                R.out = reinterpret_cast<int4 *>(base + off);
                off += a256((size_t)R.out_rows * 16 + 16);
                R.cls_beg = reinterpret_cast<uint64_t *>(base + off);
                off += a256(((size_t)R.G + 1) * 8);
            }
            // block ranges of the row kernel (256 threads a block, a thread
            // per element)
            uint64_t bt = 0;
            for (RunJob &R : rj) {
                R.blk0 = bt;
                bt += ((uint64_t)R.n + 256) / 256;
            }
            if (bt > 0x7fffffffull)
                return fail(set_error(FZ_EINVAL, "batch run-order memos too large"));
            b->run_blocks = bt;
            b->run_jobs_dev = reinterpret_cast<RunJob *>(base);
            FZ_CUDA_TRY(cudaMemcpyAsync(b->run_jobs_dev, rj.data(), rj.size() * sizeof(RunJob),
                                        cudaMemcpyHostToDevice, s));
            rc = launch_run_memo_batch(b->run_jobs_dev, b->nrun, b->run_blocks, b->status_dev, s);
            if (rc != FZ_OK) return fail(rc);
            FZ_CUDA_TRY(cudaStreamSynchronize(s));  // rj is a host temporary
        }
        for (int i = 0; i < count; ++i) {
            Inst &I = b->inst[i];
            if (!I.run) continue;
            const RunJob &R = rj[I.run_job];
            I.run_memo = R.out;
            I.cls_beg = R.cls_beg;
            I.run_rows = R.out_rows;
        }
    }
    // counts and run totals
    std::vector<const uint64_t *> pc(count), pr(count);
    for (int i = 0; i < count; ++i) {
        const Inst &I = b->inst[i];
        pc[i] = tb + I.off_C + I.n;
        pr[i] = I.off_RT != (size_t)-1 ? tb + I.off_RT + I.n : nullptr;
    }
    std::vector<uint64_t> cnt, runs;
    rc = gather(pc, cnt, s);
    if (rc == FZ_OK) rc = gather(pr, runs, s);
    if (rc != FZ_OK) return fail(rc);
    int hstatus = 0;
    FZ_CUDA_TRY(cudaMemcpyAsync(&hstatus, b->status_dev, 4, cudaMemcpyDeviceToHost, s));
    FZ_CUDA_TRY(cudaStreamSynchronize(s));
    if (hstatus != 0) return fail(set_error(FZ_EINTERNAL, "batch memo build check failed"));

    // layout, work items, per-instance parameter images
    DeviceProps dp;
    rc = device_props(&dp);
    if (rc != FZ_OK) return fail(rc);
    uint64_t total_cost = 0;
    uint64_t word = 0;
    for (int i = 0; i < count; ++i) {
        Inst &I = b->inst[i];
        I.count = cnt[i];
        if (I.count == ~0ull) return fail(set_error(FZ_EOVERFLOW, "|Z(n)| does not fit"));
        I.runs = runs[i];
        word = (word + 31) & ~31ull;  // every instance starts on a 128-byte line
        I.word_off = word;
        word += I.count * (uint64_t)I.d;
        b->total_rows += I.count;
        total_cost += I.count + I.W * I.runs;
    }
    b->total_words = word;
    const uint64_t warps = (uint64_t)dp.sms * 16;
    const uint64_t target = std::max<uint64_t>(4096, total_cost / (warps * 8 + 1));
    std::vector<uint64_t> item0(count + 1, 0);
    b->params_host.resize((size_t)count * pbytes);
    // Work items are numbered instance by instance in an order grouped by
    // code path (run copy, walk up to width 8, wider walk) and then by width,
    // so that warps taking consecutive items run the same code: warps of
    // one SM mixing the paths evict each other's instructions.  The output
    // layout (word offsets) keeps the caller's order.
    std::vector<int> order(count);
    for (int i = 0; i < count; ++i) order[i] = i;
    if (batch_item_order_enabled()) {
        auto path = [&](const Inst &I) { return I.run ? 0 : (I.d <= 8 ? 1 : 2); };
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
            const Inst &A = b->inst[x], &B = b->inst[y];
            if (path(A) != path(B)) return path(A) < path(B);
            return A.d < B.d;
        });
    }
    for (int pos = 0; pos < count; ++pos) {
        const int i = order[pos];
        Inst &I = b->inst[i];
        const uint64_t cost = I.count + I.W * I.runs;
        I.items = I.count == 0 ? 0 : std::max<uint64_t>(1, (cost + target - 1) / target);
        I.slice_cost = I.items ? (cost + I.items - 1) / I.items : 64;
        I.slice_rows = I.items ? std::max<uint64_t>(4, (I.count + I.items - 1) / I.items) : 4;
        item0[pos + 1] = item0[pos] + I.items;
        EnumLaunch L;
        L.C = tb + I.off_C;
        L.cs = (int64_t)I.n + 1;
        L.n = I.n;
        L.d = I.d;
        L.K = I.K;
        L.top = I.top;
        L.g = I.g;
        L.status = b->status_dev;
        L.slice_counter = b->counter_dev;
        L.pair_memo = I.pair;
        if (I.memo >= 0) {
            L.O = b->memo_jobs[I.memo].O;
            L.memo = b->memo_jobs[I.memo].R;
            L.memo_rows = b->memo_jobs[I.memo].rows;
        }
        if (I.run) {
            // the run copy reads the run-order rows only: memo_rows bounds them
            L.run_memo = I.run_memo;
            L.cls_beg = I.cls_beg;
            L.memo_rows = I.run_rows;
        }
        if (I.off_RT != (size_t)-1) {
            L.RT = tb + I.off_RT;
            L.W = I.W;
            L.lam_r = I.lam_r;
        }
        // out holds the word offset; the kernel adds the output base
        fill_batch_params(L, reinterpret_cast<int32_t *>(I.word_off * 4), I.count, I.slice_rows,
                          I.slice_cost, b->params_host.data() + (size_t)pos * pbytes);
    }
    b->nitems = item0[count];
    if (count) {
        FZ_CUDA_TRY(cudaMemcpyAsync(b->params_dev, b->params_host.data(), b->params_host.size(),
                                    cudaMemcpyHostToDevice, s));
        FZ_CUDA_TRY(cudaMemcpyAsync(b->item0_dev, item0.data(), item0.size() * 8,
                                    cudaMemcpyHostToDevice, s));
    }
    FZ_CUDA_TRY(cudaStreamSynchronize(s));
    *batch = b;
    return FZ_OK;
}

}  // namespace
}  // namespace fz

extern "C" {

int fz_batch_info(fz_batch_t b, fz_batch_info_t *info) {
    if (!b || !info) return set_error(FZ_EINVAL, "null pointer");
    info->count = b->count;
    info->memos = b->nmemo;
    info->total_rows = b->total_rows;
    info->total_words = b->total_words;
    info->device_bytes =
        b->tables.bytes + b->scratch.bytes + b->memos.bytes + b->meta.bytes + b->runs.bytes;
    info->work_items = b->nitems;
    info->run_order = b->run_inst;
    info->run_memos = b->nrun;
    info->coop_memos = b->memo_ncoop;
    info->reserved = 0;
    return FZ_OK;
}

int fz_batch_layout(fz_batch_t b, uint64_t *rows, uint64_t *word_offsets, int32_t *k,
                    int32_t *top) {
    if (!b) return set_error(FZ_EINVAL, "batch: null pointer");
    for (int i = 0; i < b->count; ++i) {
        if (rows) rows[i] = b->inst[i].count;
        if (word_offsets) word_offsets[i] = b->inst[i].word_off;
        if (k) k[i] = b->inst[i].K;
        if (top) top[i] = b->inst[i].top;
    }
    if (word_offsets) word_offsets[b->count] = b->total_words;
    return FZ_OK;
}

int fz_batch_set_enum_ctas_per_sm(fz_batch_t b, int32_t ctas) {
    if (!b) return set_error(FZ_EINVAL, "batch: null pointer");
    if (ctas < 0) return set_error(FZ_EINVAL, "ctas must be >= 0");
    b->ctas_per_sm = ctas;
    return FZ_OK;
}

int fz_batch_rebuild(fz_batch_t b, void *stream) {
    if (!b) return set_error(FZ_EINVAL, "batch: null pointer");
    return batch_enqueue_rebuild(b, static_cast<cudaStream_t>(stream));
}

int fz_batch_enumerate(fz_batch_t b, int32_t *out_dev, uint64_t out_capacity_words,
                       void *stream) {
    if (!b) return set_error(FZ_EINVAL, "batch: null pointer");
    if (b->total_words == 0) return FZ_OK;
    if (!out_dev) return set_error(FZ_EINVAL, "out: null pointer");
    if (((uintptr_t)out_dev & 3u) != 0) return set_error(FZ_EINVAL, "out must be 4-byte aligned");
    if (out_capacity_words < b->total_words) return set_error(FZ_ENOSPC, "output capacity too small");
    return launch_enumerate_batch(b->params_dev, b->item0_dev, b->count, b->nitems,
                                  b->counter_dev, out_dev, static_cast<cudaStream_t>(stream),
                                  b->ctas_per_sm);
}

int fz_batch_sync(fz_batch_t b, void *stream) {
    if (!b) return set_error(FZ_EINVAL, "batch: null pointer");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int h = 0;
    FZ_CUDA_TRY(cudaMemcpyAsync(&h, b->status_dev, 4, cudaMemcpyDeviceToHost, s));
    FZ_CUDA_TRY(cudaStreamSynchronize(s));
    if (h != 0) {
        FZ_CUDA_TRY(cudaMemsetAsync(b->status_dev, 0, 4, s));
        FZ_CUDA_TRY(cudaStreamSynchronize(s));
        return set_error(h == DEV_TIMEOUT ? FZ_ETIMEOUT : FZ_EINTERNAL,
                         "device-side check failed in the batch");
    }
    return FZ_OK;
}

int fz_batch_destroy(fz_batch_t b) {
    if (!b) return set_error(FZ_EINVAL, "batch: null pointer");
    delete b;
    return FZ_OK;
}

int fz_plan_batch(const fz_instance_t *inst, int count, const fz_opts_t *opt,
                  uint64_t *word_offsets, uint64_t *rows, uint64_t *words_needed,
                  void *stream) {
    fz_batch_t b = nullptr;
    int rc = fz_batch_create(inst, count, opt, &b, stream);
    if (rc != FZ_OK) return rc;
    if (words_needed) *words_needed = b->total_words;
    fz_batch_layout(b, rows, word_offsets, nullptr, nullptr);
    fz_batch_destroy(b);
    return FZ_OK;
}

int fz_enumerate_batch(const fz_instance_t *inst, int count, const fz_opts_t *opt,
                       uint64_t *word_offsets, int32_t *out_dev, uint64_t out_capacity_words,
                       uint64_t *words_needed, void *stream) {
    fz_batch_t b = nullptr;
    int rc = fz_batch_create(inst, count, opt, &b, stream);
    if (rc != FZ_OK) return rc;
    if (words_needed) *words_needed = b->total_words;
    if (word_offsets) fz_batch_layout(b, nullptr, word_offsets, nullptr, nullptr);
    rc = fz_batch_enumerate(b, out_dev, out_capacity_words, stream);
    if (rc == FZ_OK) rc = fz_batch_sync(b, stream);
    fz_batch_destroy(b);
    return rc;
}

int fz_batch_autotune(const fz_instance_t *inst, int count, fz_batch_tune_entry_t *entries,
                      int capacity, int *n_entries, void *stream) {
    if (count < 0 || (count > 0 && !inst)) return set_error(FZ_EINVAL, "instances");
    if (capacity < 0 || (capacity > 0 && !entries))
        return set_error(FZ_EINVAL, "entries: null pointer");
    if (n_entries) *n_entries = 0;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    for (int i = 0; i < count; ++i) {
        int rc = validate_gens(inst[i].g, inst[i].d);
        if (rc != FZ_OK) return rc;
        if (inst[i].n < 0) return set_error(FZ_EINVAL, "n must be >= 0");
    }
    BatchPolicy tuned = current_policy();
    const BatchPolicy base = tuned;
    static const double caps[] = {0.0, 0.25, 1.0, 4.0, 16.0};
    int found = 0;
    cudaEvent_t e0, e1, e2;
    FZ_CUDA_TRY(cudaEventCreate(&e0));
    FZ_CUDA_TRY(cudaEventCreate(&e1));
    FZ_CUDA_TRY(cudaEventCreate(&e2));
    int rc = FZ_OK;
    DevArena out;
    // rebuild + enumeration of a created batch, mean of 3 after a warm-up
    auto time_batch = [&](fz_batch_s *b, double *build_ms, double *enum_ms) -> int {
        if (out.bytes < b->total_words * 4 + 256) {
            const int r = out.alloc(b->total_words * 4 + 256);
            if (r != FZ_OK) return r;
        }
        double bsum = 0, esum = 0;
        int r = FZ_OK;
        for (int rep = 0; rep < 4 && r == FZ_OK; ++rep) {  // rep 0 warms up
            cudaEventRecord(e0, s);
            r = fz_batch_rebuild(b, s);
            cudaEventRecord(e1, s);
            if (r == FZ_OK)
                r = fz_batch_enumerate(b, static_cast<int32_t *>(out.p), b->total_words, s);
            cudaEventRecord(e2, s);
            if (r == FZ_OK) r = fz_batch_sync(b, s);
            float b_ms = 0, e_ms = 0;
            cudaEventElapsedTime(&b_ms, e0, e1);
            cudaEventElapsedTime(&e_ms, e1, e2);
            if (rep > 0) {
                bsum += b_ms;
                esum += e_ms;
            }
        }
        *build_ms = bsum / 3;
        *enum_ms = esum / 3;
        return r;
    };
    // per width: the default's time and the fastest candidate's
    std::vector<double> width_gain(FZ_MAX_D + 1, 0.0), width_base(FZ_MAX_D + 1, 0.0);
    for (int d = 3; d <= FZ_MAX_D && rc == FZ_OK; ++d) {
        // the instances of this width (up to 1024, spread over the list):
        // memo builds run one CTA per memo in waves and the enumeration's
        // tail depends on the work available, so timings of small samples
        // do not add up to the whole batch; whole widths nearly do
        std::vector<fz_instance_t> all;
        for (int i = 0; i < count; ++i)
            if (inst[i].d == d) all.push_back(inst[i]);
        if (all.empty()) continue;
        std::vector<fz_instance_t> sub;
        const size_t step = (all.size() + 1023) / 1024;
        for (size_t i = 0; i < all.size(); i += step) sub.push_back(all[i]);
        double best_t = 1e300, base_t = -1;
        double best_cap = base.cap_rows[d];
        bool best_run = base.run_order[d];
        std::vector<std::pair<double, bool>> cands;
        for (double c : caps) cands.push_back({c, true});
        for (double c : caps) cands.push_back({c, false});
        std::vector<std::vector<int>> seen;  // memo depth and layout choices already timed
        std::vector<double> seen_t;
        std::vector<int> base_key;
        {
            fz_batch_t b0 = nullptr;
            if (batch_create_impl(sub.data(), (int)sub.size(), nullptr, base, &b0, s) == FZ_OK) {
                for (const Inst &I : b0->inst) {
                    base_key.push_back(I.K);
                    base_key.push_back(I.top);
                    base_key.push_back(I.pair ? 1 : 0);
                    base_key.push_back(I.run ? 1 : 0);
                }
                fz_batch_destroy(b0);
            }
            cudaGetLastError();
        }
        for (auto &cand : cands) {
            BatchPolicy pol = tuned;
            pol.cap_rows[d] = cand.first;
            pol.run_order[d] = cand.second;
            fz_batch_t b = nullptr;
            rc = batch_create_impl(sub.data(), (int)sub.size(), nullptr, pol, &b, s);
            if (rc == FZ_ENOMEM || rc == FZ_EINVAL) {  // too large for this device: skip
                cudaGetLastError();
                rc = FZ_OK;
                continue;
            }
            if (rc != FZ_OK) break;
            // candidates that choose the same memos as one already timed are
            // not timed again
            std::vector<int> key;
            for (const Inst &I : b->inst) {
                key.push_back(I.K);
                key.push_back(I.top);
                key.push_back(I.pair ? 1 : 0);
                key.push_back(I.run ? 1 : 0);
            }
            bool dup = false;
            for (auto &k : seen) dup = dup || k == key;
            if (dup) {
                fz_batch_destroy(b);
                continue;
            }
            double b_ms = 0, e_ms = 0;
            rc = time_batch(b, &b_ms, &e_ms);
            if (rc == FZ_OK) {
                const double t = b_ms + e_ms;
                seen.push_back(key);
                seen_t.push_back(t);
                if (key == base_key) base_t = t;
                if (found < capacity) {
                    fz_batch_tune_entry_t &E = entries[found];
                    E.d = d;
                    E.run_order = cand.second ? 1 : 0;
                    E.instances = (int32_t)sub.size();
                    E.memos = b->nmemo;
                    E.cap_rows = cand.first;
                    E.rows = b->total_rows;
                    uint64_t mr = 0;
                    for (const MemoJob &J : b->memo_jobs) mr += J.rows;
                    E.memo_rows = mr;
                    E.build_ms = b_ms;
                    E.enum_ms = e_ms;
                    E.total_ms = t;
                }
                ++found;
                if (t < best_t) {
                    best_t = t;
                    best_cap = cand.first;
                    best_run = cand.second;
                }
            }
            fz_batch_destroy(b);
        }
        tuned.cap_rows[d] = best_cap;
        tuned.run_order[d] = best_run;
        if (base_t > 0 && best_t < base_t) {
            width_gain[d] = base_t - best_t;
            width_base[d] = base_t;
        }
    }
    // The widths' fastest choices need not combine: the enumeration of a
    // mixed batch shares the GPU, its L2 and its instruction cache among
    // widths.  So they are applied greedily on the whole batch: starting
    // from the policy in force, each width's fastest choice (widths in
    // decreasing order of their own gain, gains of 3 % or more) is tried on
    // top of the choices kept so far and kept only if the whole batch's
    // rebuild + enumeration gets faster by 1 % or more.
    auto time_whole = [&](const BatchPolicy &pol, int tag, double *t) -> int {
        *t = 1e300;
        fz_batch_t b = nullptr;
        int r = batch_create_impl(inst, count, nullptr, pol, &b, s);
        if (r == FZ_ENOMEM || r == FZ_EINVAL) {  // too large for this device
            cudaGetLastError();
            return FZ_OK;
        }
        if (r != FZ_OK) return r;
        double b_ms = 0, e_ms = 0;
        r = time_batch(b, &b_ms, &e_ms);
        if (r == FZ_OK) {
            *t = b_ms + e_ms;
            if (found < capacity) {
                fz_batch_tune_entry_t &E = entries[found];
                E.d = 0;            // the whole batch
                E.run_order = tag;  // 0: the starting policy; w: after trying width w
                E.instances = count;
                E.memos = b->nmemo;
                E.cap_rows = -1.0;
                E.rows = b->total_rows;
                uint64_t mr = 0;
                for (const MemoJob &J : b->memo_jobs) mr += J.rows;
                E.memo_rows = mr;
                E.build_ms = b_ms;
                E.enum_ms = e_ms;
                E.total_ms = *t;
            }
            ++found;
        }
        fz_batch_destroy(b);
        return r;
    };
    BatchPolicy kept = base;
    double kept_t = 1e300;
    if (rc == FZ_OK) rc = time_whole(kept, 0, &kept_t);
    std::vector<int> order;
    for (int d = 3; d <= FZ_MAX_D; ++d)
        if (width_gain[d] > 0) order.push_back(d);
    std::sort(order.begin(), order.end(),
              [&](int x, int y) { return width_gain[x] > width_gain[y]; });
    for (int d : order) {
        if (rc != FZ_OK || kept_t >= 1e300) break;
        if (width_gain[d] < 0.03 * width_base[d]) continue;  // under 3 % of the width's time
        BatchPolicy trial = kept;
        trial.cap_rows[d] = tuned.cap_rows[d];
        trial.run_order[d] = tuned.run_order[d];
        double t = 1e300;
        rc = time_whole(trial, d, &t);
        if (rc == FZ_OK && t < 0.99 * kept_t) {
            kept = trial;
            kept_t = t;
        }
    }
    tuned = kept;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaEventDestroy(e2);
    if (rc != FZ_OK) return rc;
    if (n_entries) *n_entries = std::min(found, capacity);
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_policy_mu);
    g_policy[dev] = tuned;
    return FZ_OK;
}

int fz_batch_policy(int32_t d, double *cap_rows, int32_t *run_order) {
    if (d < 1 || d > FZ_MAX_D) return set_error(FZ_EINVAL, "d out of range");
    const BatchPolicy P = current_policy();
    if (cap_rows) *cap_rows = P.cap_rows[d];
    if (run_order) *run_order = P.run_order[d] ? 1 : 0;
    return FZ_OK;
}

int fz_batch_policy_reset(void) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_policy_mu);
    g_policy.erase(dev);
    return FZ_OK;
}

}  // extern "C"
