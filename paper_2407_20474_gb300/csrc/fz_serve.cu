// fz_serve.cu -- a request loop that keeps generator sets resident on the
// device and serves Z(n, g) queries with continuous batching.
//
// Registering a set builds its plan once (count table, runs table and memo
// for every n up to n_max; the tables depend on the generators only) and
// mirrors row 0 of its count and runs tables on the host, so the exact size
// of any later query is known at submission without touching the device.
// A background thread admits queued requests in arrival order whenever a
// slot and enough output memory (exact bytes, from a first-fit arena carved
// out of one device allocation) are free.  By default every request admitted
// in one pass of the loop is launched as one group: one persistent launch of
// the batch enumeration kernel with a work-item range per request (its
// parameters and item prefix staged in page-locked memory and copied in one
// transfer), one copy back of the group's status words and one completion
// callback, on the next of several streams, so groups admitted while others
// run overlap on the GPU.  With FZ_SERVE_PER_REQUEST every request is its
// own launch of the single-instance kernel (and so is a request whose plan
// the batch kernel does not serve: run order wider than 8).  Completion is recorded by a host callback on the
// request's stream (cudaLaunchHostFunc), which frees the slot, stamps the
// completion time and reads the request's own device status word (copied to
// page-locked host memory just before the callback), so a device-side check
// that failed marks that request, and only it, as failed.  The output stays
// valid until the client releases it.  A queued request can be cancelled;
// one already on the device runs to completion.
#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <cstdlib>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "fz_internal.cuh"

struct fz_server_s;

namespace fz {
namespace {

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator over [0, size) with 256-byte granules and coalescing.
class Arena {
   public:
    void init(uint64_t size) {
        free_.clear();
        size_ = size & ~255ull;
        if (size_) free_[0] = size_;
        used_ = 0;
    }
    bool alloc(uint64_t bytes, uint64_t *off) {
        bytes = (bytes + 255) & ~255ull;
        if (bytes == 0) bytes = 256;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const uint64_t rest = it->second - bytes;
                const uint64_t at = it->first + bytes;
                free_.erase(it);
                if (rest) free_[at] = rest;
                used_ += bytes;
                return true;
            }
        }
        return false;
    }
    void release(uint64_t off, uint64_t bytes) {
        bytes = (bytes + 255) & ~255ull;
        if (bytes == 0) bytes = 256;
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto next = std::next(it);
        if (next != free_.end() && it->first + it->second == next->first) {
            it->second += next->second;
            free_.erase(next);
        }
        if (it != free_.begin()) {
            auto prev = std::prev(it);
            if (prev->first + prev->second == it->first) {
                prev->second += it->second;
                free_.erase(it);
            }
        }
    }
    uint64_t used() const { return used_; }
    uint64_t size() const { return size_; }

   private:
    std::map<uint64_t, uint64_t> free_;
    uint64_t size_ = 0, used_ = 0;
};

struct SetRec {
    fz_plan_t plan = nullptr;
    int d = 0;
    int32_t n_max = 0;
    std::vector<int32_t> g;           // generators, in the caller's order
    std::vector<uint64_t> count_row;  // |Z(r)|, r = 0..n_max
    std::vector<uint64_t> runs_row;   // runs under the root, r = 0..n_max (if any)
};

struct Req;

struct CallbackCtx {
    fz_server_s *srv;
    Req *req;
};

// A launch group (grouped mode): device and page-locked staging buffers for
// up to max_group requests, used by one launch at a time.
struct Group {
    cudaStream_t st = nullptr;
    char *dev = nullptr;      // params | item0 | status | counter
    char *stage = nullptr;    // page-locked: params | item0 | status (zeros), copied up
    int *status_host = nullptr;  // page-locked: the status words, copied back
    size_t o_item0 = 0, o_status = 0, o_counter = 0, bytes = 0;
    std::vector<Req *> reqs;
    fz_server_s *srv = nullptr;
    int index = 0;
};

struct Req {
    uint64_t ticket = 0;
    int set = 0;
    int32_t n = 0;
    uint64_t count = 0, bytes = 0, off = 0;
    int slot = -1;   // per-request mode: its slot; grouped mode: its group
    int status = FZ_SERVE_QUEUED;  // or FZ_SERVE_RUNNING / DONE, or a negative fz_status
    bool has_mem = false;
    double t_submit = 0, t_admit = 0, t_done = 0;
    CallbackCtx cb;
};

}  // namespace
}  // namespace fz

using namespace fz;

struct fz_server_s {
    std::mutex mu;
    std::condition_variable cv;       // wakes the server thread
    std::condition_variable done_cv;  // wakes waiters
    std::thread th;
    bool stop = false;
    int device = 0;
    fz_serve_cfg_t cfg{};
    std::vector<cudaStream_t> streams;
    int next_stream = 0;
    void *arena_base = nullptr;
    Arena arena;
    unsigned long long *counters = nullptr;  // work-item counter, one per slot
    int *slot_status = nullptr;              // device status word, one per slot
    int *slot_status_host = nullptr;         // page-locked copies, read by on_done
    std::vector<int> free_slots;
    std::vector<SetRec> sets;
    std::deque<Req *> queue;
    std::unordered_map<uint64_t, Req *> reqs;
    uint64_t next_ticket = 1;
    uint64_t admitted = 0, completed = 0;
    int launch_error = FZ_OK;
    bool grouped = true;
    int max_group = 0, in_flight = 0;
    std::vector<Group> groups;
    std::vector<int> free_groups;
};

namespace fz {
namespace {

void CUDART_CB on_done(void *p) {
    CallbackCtx *c = static_cast<CallbackCtx *>(p);
    fz_server_s *s = c->srv;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        c->req->t_done = now_s();
        // the status word of this request's slot, copied back on its stream
        // before this callback (no CUDA call is allowed in here)
        const int dev = s->slot_status_host[c->req->slot];
        if (dev == DEV_OK) {
            c->req->status = FZ_SERVE_DONE;
        } else {
            c->req->status = dev == DEV_TIMEOUT ? FZ_ETIMEOUT : FZ_EINTERNAL;
            s->launch_error = c->req->status;
        }
        s->free_slots.push_back(c->req->slot);
        c->req->slot = -1;
        s->completed++;
    }
    s->cv.notify_one();
    s->done_cv.notify_all();
}

// Enqueue one admitted request (called by the server thread, lock not held).
int launch_request(fz_server_s *s, Req *r, cudaStream_t st) {
    const SetRec &S = s->sets[r->set];
    fz_plan_info_t info;
    int rc = fz_plan_info(S.plan, &info);
    if (rc != FZ_OK) return rc;
    int32_t *out = reinterpret_cast<int32_t *>(static_cast<char *>(s->arena_base) + r->off);
    // the slot is free, so no copy into its host word is pending
    s->slot_status_host[r->slot] = DEV_OK;
    if (r->count > 0) {
        EnumLaunch L;
        rc = plan_launch_for(S.plan, r->n, &L);
        if (rc != FZ_OK) return rc;
        L.slice_counter = s->counters + r->slot;
        L.status = s->slot_status + r->slot;
        FZ_CUDA_TRY(cudaMemsetAsync(L.status, 0, sizeof(int), st));
        if (L.RT) {
            L.total_rows = r->count;
            L.total_cost = r->count + L.W * S.runs_row[r->n];
        }
        DeviceProps dp;
        rc = device_props(&dp);
        if (rc != FZ_OK) return rc;
        rc = launch_enumerate(L, 0, r->count, out, default_slice_rows(r->count, dp.sms), st);
        if (rc != FZ_OK) return rc;
        FZ_CUDA_TRY(cudaMemcpyAsync(s->slot_status_host + r->slot, L.status, sizeof(int),
                                    cudaMemcpyDeviceToHost, st));
    }
    r->cb.srv = s;
    r->cb.req = r;
    FZ_CUDA_TRY(cudaLaunchHostFunc(st, on_done, &r->cb));
    return FZ_OK;
}

// Grouped mode: the completion of a group (its status words were copied
// back on the group's stream before this callback).
void CUDART_CB on_group_done(void *p) {
    Group *G = static_cast<Group *>(p);
    fz_server_s *s = G->srv;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        const double t = now_s();
        for (size_t j = 0; j < G->reqs.size(); ++j) {
            Req *r = G->reqs[j];
            r->t_done = t;
            const int dev = G->status_host[j];
            if (dev == DEV_OK) {
                r->status = FZ_SERVE_DONE;
            } else {
                r->status = dev == DEV_TIMEOUT ? FZ_ETIMEOUT : FZ_EINTERNAL;
                s->launch_error = r->status;
            }
            r->slot = -1;
            s->completed++;
        }
        s->in_flight -= (int)G->reqs.size();
        G->reqs.clear();
        s->free_groups.push_back(G->index);
    }
    s->cv.notify_one();
    s->done_cv.notify_all();
}

// Requests of at least this many rows are launched with their plan's own
// kernel after the group's batch kernel (FZ_SERVE_DIRECT_ROWS overrides it;
// tuning only).
uint64_t serve_direct_rows() {
    static const uint64_t v = [] {
        const char *e = std::getenv("FZ_SERVE_DIRECT_ROWS");
        const long long x = e ? std::atoll(e) : -1;
        return x >= 0 ? (uint64_t)x : (uint64_t)(1u << 22);
    }();
    return v;
}

// Whether the batch kernel serves a launch of this shape (its run-order
// copy takes widths up to 8 with at least one walked coordinate).
bool batch_kernel_serves(const EnumLaunch &L) {
    if (!L.run_memo) return true;
    return L.d <= 8 && L.d - L.K - 1 >= 1 && L.K >= 1 && L.K <= 3;
}

// Enqueue a group of admitted requests (called by the server thread, lock
// not held): one batch launch over all of them (request j's items follow
// request j-1's, equal-cost items as in batches), requests the batch kernel
// does not serve launched one by one after it, then the status words back
// and the completion callback.
int launch_group(fz_server_s *s, Group &G) {
    const size_t pb = enum_params_bytes();
    const int m = (int)G.reqs.size();
    DeviceProps dp;
    int rc = device_props(&dp);
    if (rc != FZ_OK) return rc;
    std::vector<EnumLaunch> Ls(m);
    std::vector<uint64_t> cost(m, 0);
    std::vector<char> direct(m, 0);
    uint64_t total_cost = 0;
    for (int j = 0; j < m; ++j) {
        const Req *r = G.reqs[j];
        const SetRec &S = s->sets[r->set];
        rc = plan_launch_for(S.plan, r->n, &Ls[j]);
        if (rc != FZ_OK) return rc;
        EnumLaunch &L = Ls[j];
        L.status = reinterpret_cast<int *>(G.dev + G.o_status) + j;
        L.slice_counter = reinterpret_cast<unsigned long long *>(G.dev + G.o_counter);
        cost[j] = r->count;
        if (L.RT) {
            L.total_rows = r->count;
            L.total_cost = r->count + L.W * S.runs_row[r->n];
            cost[j] = L.total_cost;
        }
        // large requests take their plan's own kernel (its compiled-in walk
        // or run copy writes faster than the batch kernel's generic one);
        // so do those the batch kernel does not serve
        direct[j] = (!batch_kernel_serves(L) || r->count >= serve_direct_rows()) ? 1 : 0;
        if (!direct[j]) total_cost += cost[j];
    }
    const uint64_t warps = (uint64_t)dp.sms * 16;
    const uint64_t target = std::max<uint64_t>(4096, total_cost / (warps * 8 + 1));
    uint64_t *item0 = reinterpret_cast<uint64_t *>(G.stage + G.o_item0);
    item0[0] = 0;
    for (int j = 0; j < m; ++j) {
        const Req *r = G.reqs[j];
        uint64_t items = 0, slice_cost = 64, slice_rows = 4;
        if (!direct[j] && r->count > 0) {
            items = std::max<uint64_t>(1, (cost[j] + target - 1) / target);
            slice_cost = (cost[j] + items - 1) / items;
            slice_rows = std::max<uint64_t>(4, (r->count + items - 1) / items);
        }
        // out holds the byte offset of the request's rows in the arena
        fill_batch_params(Ls[j], reinterpret_cast<int32_t *>((uintptr_t)r->off), r->count,
                          slice_rows, slice_cost, G.stage + (size_t)j * pb);
        item0[j + 1] = item0[j] + items;
        reinterpret_cast<int *>(G.stage + G.o_status)[j] = DEV_OK;
    }
    // parameters, item prefix and zeroed status words: one transfer
    FZ_CUDA_TRY(cudaMemcpyAsync(G.dev, G.stage, G.o_status + (size_t)m * sizeof(int),
                                cudaMemcpyHostToDevice, G.st));
    int32_t *base = static_cast<int32_t *>(s->arena_base);
    rc = launch_enumerate_batch(G.dev, reinterpret_cast<const uint64_t *>(G.dev + G.o_item0), m,
                                item0[m], reinterpret_cast<unsigned long long *>(G.dev + G.o_counter),
                                base, G.st);
    if (rc != FZ_OK) return rc;
    for (int j = 0; j < m; ++j) {
        if (!direct[j] || G.reqs[j]->count == 0) continue;
        const Req *r = G.reqs[j];
        int32_t *out = reinterpret_cast<int32_t *>(static_cast<char *>(s->arena_base) + r->off);
        rc = launch_enumerate(Ls[j], 0, r->count, out, default_slice_rows(r->count, dp.sms), G.st);
        if (rc != FZ_OK) return rc;
    }
    FZ_CUDA_TRY(cudaMemcpyAsync(G.status_host, G.dev + G.o_status, (size_t)m * sizeof(int),
                                cudaMemcpyDeviceToHost, G.st));
    FZ_CUDA_TRY(cudaLaunchHostFunc(G.st, on_group_done, &G));
    return FZ_OK;
}

void server_loop_grouped(fz_server_s *s) {
    std::unique_lock<std::mutex> lk(s->mu);
    while (!s->stop) {
        bool launched = false;
        // admit in arrival order into a free group while requests may be in
        // flight and the exact output bytes are free
        while (!s->free_groups.empty() && !s->queue.empty() &&
               s->in_flight < s->cfg.max_in_flight) {
            const int gi = s->free_groups.back();
            Group &G = s->groups[gi];
            G.reqs.clear();
            while (!s->queue.empty() && (int)G.reqs.size() < s->max_group &&
                   s->in_flight < s->cfg.max_in_flight) {
                Req *r = s->queue.front();
                uint64_t off = 0;
                if (!s->arena.alloc(r->bytes, &off)) break;
                s->queue.pop_front();
                r->off = off;
                r->has_mem = true;
                r->slot = gi;
                r->status = FZ_SERVE_RUNNING;
                r->t_admit = now_s();
                s->admitted++;
                s->in_flight++;
                G.reqs.push_back(r);
            }
            if (G.reqs.empty()) break;  // waiting for output memory
            s->free_groups.pop_back();
            lk.unlock();
            const int rc = launch_group(s, G);
            lk.lock();
            if (rc != FZ_OK) {
                // nothing of this group reaches its callback: fail its requests
                for (Req *r : G.reqs) {
                    r->status = rc;
                    r->t_done = now_s();
                    r->slot = -1;
                }
                s->in_flight -= (int)G.reqs.size();
                G.reqs.clear();
                s->free_groups.push_back(gi);
                s->launch_error = rc;
                s->done_cv.notify_all();
            }
            launched = true;
        }
        if (!launched) s->cv.wait_for(lk, std::chrono::microseconds(200));
    }
}

void server_loop(fz_server_s *s) {
    cudaSetDevice(s->device);
    if (s->grouped) {
        server_loop_grouped(s);
        return;
    }
    std::unique_lock<std::mutex> lk(s->mu);
    while (!s->stop) {
        // admit in arrival order while a slot and the exact output bytes are free
        std::vector<std::pair<Req *, cudaStream_t>> go;
        while (!s->queue.empty() && !s->free_slots.empty()) {
            Req *r = s->queue.front();
            uint64_t off = 0;
            if (!s->arena.alloc(r->bytes, &off)) break;
            s->queue.pop_front();
            r->off = off;
            r->has_mem = true;
            r->slot = s->free_slots.back();
            s->free_slots.pop_back();
            r->status = FZ_SERVE_RUNNING;
            r->t_admit = now_s();
            s->admitted++;
            go.push_back({r, s->streams[s->next_stream]});
            s->next_stream = (s->next_stream + 1) % (int)s->streams.size();
        }
        if (!go.empty()) {
            lk.unlock();
            for (auto &x : go) {
                int rc = launch_request(s, x.first, x.second);
                if (rc != FZ_OK) {
                    std::lock_guard<std::mutex> g2(s->mu);
                    x.first->status = rc;
                    x.first->t_done = now_s();
                    s->free_slots.push_back(x.first->slot);
                    x.first->slot = -1;
                    s->launch_error = rc;
                    s->done_cv.notify_all();
                }
            }
            lk.lock();
            continue;
        }
        s->cv.wait_for(lk, std::chrono::microseconds(200));
    }
}

}  // namespace
}  // namespace fz

extern "C" {

int fz_serve_create(const fz_serve_cfg_t *cfg, fz_server_t *srv) {
    if (!cfg || !srv) return set_error(FZ_EINVAL, "null pointer");
    if ((cfg->flags & ~FZ_SERVE_PER_REQUEST) != 0 || cfg->max_in_flight < 1 || cfg->streams < 1 ||
        cfg->max_queue < 1)
        return set_error(FZ_EINVAL, "serve config");
    fz_server_s *s = new (std::nothrow) fz_server_s;
    if (!s) return set_error(FZ_ENOMEM, "host allocation");
    s->cfg = *cfg;
    s->grouped = (cfg->flags & FZ_SERVE_PER_REQUEST) == 0;
    auto fail = [&](int rc) {
        for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
        if (s->arena_base) cudaFree(s->arena_base);
        if (s->counters) cudaFree(s->counters);
        if (s->slot_status_host) cudaFreeHost(s->slot_status_host);
        for (Group &G : s->groups) {
            if (G.dev) cudaFree(G.dev);
            if (G.stage) cudaFreeHost(G.stage);
            if (G.status_host) cudaFreeHost(G.status_host);
        }
        delete s;
        return rc;
    };
    cudaError_t e = cudaGetDevice(&s->device);
    if (e != cudaSuccess) return fail(cuda_error(e, "cudaGetDevice"));
    uint64_t mem = cfg->memory_bytes;
    if (mem == 0) {
        size_t fr = 0, tot = 0;
        cudaMemGetInfo(&fr, &tot);
        mem = fr / 4;
    }
    e = cudaMalloc(&s->arena_base, mem);
    if (e != cudaSuccess) return fail(cuda_error(e, "cudaMalloc (serve arena)"));
    s->arena.init(mem);
    const size_t cbytes = (size_t)cfg->max_in_flight * (8 + 4);
    e = cudaMalloc((void **)&s->counters, cbytes);
    if (e != cudaSuccess) return fail(cuda_error(e, "cudaMalloc (serve counters)"));
    s->slot_status = reinterpret_cast<int *>(s->counters + cfg->max_in_flight);
    e = cudaMemset(s->counters, 0, cbytes);
    if (e != cudaSuccess) return fail(cuda_error(e, "cudaMemset (serve counters)"));
    e = cudaHostAlloc((void **)&s->slot_status_host, (size_t)cfg->max_in_flight * 4,
                      cudaHostAllocDefault);
    if (e != cudaSuccess) return fail(cuda_error(e, "cudaHostAlloc (serve status)"));
    for (int i = 0; i < cfg->max_in_flight; ++i) s->slot_status_host[i] = DEV_OK;
    for (int i = 0; i < cfg->streams; ++i) {
        cudaStream_t st;
        e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e != cudaSuccess) return fail(cuda_error(e, "cudaStreamCreate"));
        s->streams.push_back(st);
    }
    for (int i = cfg->max_in_flight - 1; i >= 0; --i) s->free_slots.push_back(i);
    if (s->grouped) {
        // one launch group per stream, each for up to max_in_flight requests
        s->max_group = cfg->max_in_flight;
        const size_t pb = enum_params_bytes();
        s->groups.resize(cfg->streams);
        for (int i = 0; i < cfg->streams; ++i) {
            Group &G = s->groups[i];
            G.st = s->streams[i];
            G.srv = s;
            G.index = i;
            G.o_item0 = ((size_t)s->max_group * pb + 255) & ~size_t(255);
            G.o_status = (G.o_item0 + ((size_t)s->max_group + 1) * 8 + 255) & ~size_t(255);
            G.o_counter = (G.o_status + (size_t)s->max_group * 4 + 255) & ~size_t(255);
            G.bytes = G.o_counter + 256;
            e = cudaMalloc((void **)&G.dev, G.bytes);
            if (e != cudaSuccess) return fail(cuda_error(e, "cudaMalloc (serve group)"));
            e = cudaHostAlloc((void **)&G.stage, G.o_counter, cudaHostAllocDefault);
            if (e != cudaSuccess) return fail(cuda_error(e, "cudaHostAlloc (serve group)"));
            e = cudaHostAlloc((void **)&G.status_host, (size_t)s->max_group * 4,
                              cudaHostAllocDefault);
            if (e != cudaSuccess) return fail(cuda_error(e, "cudaHostAlloc (serve group)"));
        }
        for (int i = cfg->streams - 1; i >= 0; --i) s->free_groups.push_back(i);
    }
    s->th = std::thread(server_loop, s);
    *srv = s;
    return FZ_OK;
}

int fz_serve_register(fz_server_t s, const int32_t *g, int d, int32_t n_max, int32_t *set_id) {
    if (!s || !set_id) return set_error(FZ_EINVAL, "null pointer");
    SetRec rec;
    rec.d = d;
    rec.n_max = n_max;
    if (g && d > 0 && d <= FZ_MAX_D) rec.g.assign(g, g + d);
    fz_opts_t opt{FZ_AUTO, FZ_AUTO, 0, 0};
    int rc = fz_plan_create(g, d, n_max, &opt, &rec.plan, s->streams[0]);
    if (rc != FZ_OK) return rc;
    rec.count_row.resize((size_t)n_max + 1);
    rc = plan_host_rows(rec.plan, rec.count_row.data(), &rec.runs_row, s->streams[0]);
    if (rc != FZ_OK) {
        fz_plan_destroy(rec.plan);
        return rc;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    s->sets.push_back(std::move(rec));
    *set_id = (int32_t)s->sets.size() - 1;
    return FZ_OK;
}

int fz_serve_submit(fz_server_t s, int32_t set_id, int32_t n, uint64_t *ticket) {
    if (!s || !ticket) return set_error(FZ_EINVAL, "null pointer");
    Req *r = nullptr;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (set_id < 0 || set_id >= (int32_t)s->sets.size())
            return set_error(FZ_ENOTFOUND, "unknown generator set");
        const SetRec &S = s->sets[set_id];
        if (n < 0 || n > S.n_max) return set_error(FZ_EINVAL, "n outside [0, n_max] of the set");
        if ((int)s->queue.size() >= s->cfg.max_queue) return set_error(FZ_EAGAIN, "queue full");
        const uint64_t count = S.count_row[n];
        uint64_t bytes = 0;
        if (count == ~0ull || count > (~0ull / 4) / (uint64_t)S.d)
            return set_error(FZ_EOVERFLOW, "output size");
        bytes = count * (uint64_t)S.d * 4;
        if (bytes > s->arena.size()) return set_error(FZ_ENOMEM, "larger than the output budget");
        r = new (std::nothrow) Req;
        if (!r) return set_error(FZ_ENOMEM, "host allocation");
        r->ticket = s->next_ticket++;
        r->set = set_id;
        r->n = n;
        r->count = count;
        r->bytes = bytes;
        r->t_submit = now_s();
        s->reqs[r->ticket] = r;
        s->queue.push_back(r);
        *ticket = r->ticket;
    }
    s->cv.notify_one();
    return FZ_OK;
}

int fz_serve_submit_gens(fz_server_t s, const int32_t *g, int d, int32_t n, uint64_t *ticket) {
    if (!s || !ticket) return set_error(FZ_EINVAL, "null pointer");
    int rc = validate_gens(g, d);
    if (rc != FZ_OK) return rc;
    if (n < 0) return set_error(FZ_EINVAL, "n must be >= 0");
    int32_t set_id = -1;
    {
        // a registered set with the same generators, in the same order
        // (the order defines the lexicographic order), covering n
        std::lock_guard<std::mutex> lk(s->mu);
        for (size_t i = 0; i < s->sets.size() && set_id < 0; ++i) {
            const SetRec &S = s->sets[i];
            if (S.d != d || S.n_max < n) continue;
            bool same = true;
            for (int j = 0; j < d && same; ++j) same = S.g[j] == g[j];
            if (same) set_id = (int32_t)i;
        }
    }
    if (set_id < 0) {
        rc = fz_serve_register(s, g, d, n, &set_id);
        if (rc != FZ_OK) return rc;
    }
    return fz_serve_submit(s, set_id, n, ticket);
}

int fz_serve_cancel(fz_server_t s, uint64_t ticket) {
    if (!s) return set_error(FZ_EINVAL, "null pointer");
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->reqs.find(ticket);
        if (it == s->reqs.end()) return set_error(FZ_ENOTFOUND, "unknown ticket");
        Req *r = it->second;
        if (r->status == FZ_SERVE_RUNNING)
            return set_error(FZ_EAGAIN, "request already on the device; wait, then release");
        if (r->status != FZ_SERVE_QUEUED) return FZ_OK;  // finished or failed: nothing to do
        for (auto q = s->queue.begin(); q != s->queue.end(); ++q) {
            if (*q == r) {
                s->queue.erase(q);
                break;
            }
        }
        r->status = FZ_ECANCELED;
        r->t_done = now_s();
    }
    s->done_cv.notify_all();
    s->cv.notify_one();  // the request may have been blocking admission of later ones
    return FZ_OK;
}

static void fill_result(fz_server_t s, const Req *r, fz_result_t *out) {
    out->status = r->status;
    out->d = s->sets[r->set].d;
    out->count = r->count;
    out->rows_dev = r->status == FZ_SERVE_DONE
                        ? reinterpret_cast<const int32_t *>(static_cast<char *>(s->arena_base) + r->off)
                        : nullptr;
    out->t_submit = r->t_submit;
    out->t_admit = r->t_admit;
    out->t_done = r->t_done;
}

int fz_serve_poll(fz_server_t s, uint64_t ticket, fz_result_t *res) {
    if (!s || !res) return set_error(FZ_EINVAL, "null pointer");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return set_error(FZ_ENOTFOUND, "unknown ticket");
    fill_result(s, it->second, res);
    return FZ_OK;
}

int fz_serve_wait(fz_server_t s, uint64_t ticket, int32_t timeout_ms, fz_result_t *res) {
    if (!s || !res) return set_error(FZ_EINVAL, "null pointer");
    std::unique_lock<std::mutex> lk(s->mu);
    const auto deadline =
        std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms);
    for (;;) {
        // looked up again after every wakeup: another thread may have
        // released (and so freed) the request meanwhile
        auto it = s->reqs.find(ticket);
        if (it == s->reqs.end()) return set_error(FZ_ENOTFOUND, "unknown or released ticket");
        if (it->second->status <= 0) {
            fill_result(s, it->second, res);
            return FZ_OK;
        }
        if (timeout_ms < 0)
            s->done_cv.wait(lk);
        else if (s->done_cv.wait_until(lk, deadline) == std::cv_status::timeout &&
                 std::chrono::steady_clock::now() >= deadline) {
            auto again = s->reqs.find(ticket);
            if (again == s->reqs.end())
                return set_error(FZ_ENOTFOUND, "unknown or released ticket");
            if (again->second->status <= 0) {
                fill_result(s, again->second, res);
                return FZ_OK;
            }
            return set_error(FZ_EAGAIN, "not done yet");
        }
    }
}

int fz_serve_copy(fz_server_t s, uint64_t ticket, int32_t *dst, uint64_t capacity_words,
                  void *stream) {
    if (!s) return set_error(FZ_EINVAL, "null pointer");
    const void *src = nullptr;
    uint64_t words = 0;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->reqs.find(ticket);
        if (it == s->reqs.end()) return set_error(FZ_ENOTFOUND, "unknown ticket");
        const Req *r = it->second;
        if (r->status < 0) return set_error(r->status, "request failed or was cancelled");
        if (r->status != FZ_SERVE_DONE) return set_error(FZ_EAGAIN, "request not done");
        words = r->count * (uint64_t)s->sets[r->set].d;
        src = static_cast<char *>(s->arena_base) + r->off;
    }
    if (words == 0) return FZ_OK;
    if (!dst) return set_error(FZ_EINVAL, "dst: null pointer");
    if (capacity_words < words) return set_error(FZ_ENOSPC, "capacity too small");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    FZ_CUDA_TRY(cudaMemcpyAsync(dst, src, words * 4, cudaMemcpyDefault, st));
    FZ_CUDA_TRY(cudaStreamSynchronize(st));
    return FZ_OK;
}

int fz_serve_release(fz_server_t s, uint64_t ticket) {
    if (!s) return set_error(FZ_EINVAL, "null pointer");
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->reqs.find(ticket);
        if (it == s->reqs.end()) return set_error(FZ_ENOTFOUND, "unknown ticket");
        Req *r = it->second;
        if (r->status > 0) return set_error(FZ_EAGAIN, "request still queued or running");
        if (r->has_mem) s->arena.release(r->off, r->bytes);
        s->reqs.erase(it);
        delete r;
    }
    s->cv.notify_one();
    return FZ_OK;
}

int fz_serve_replay(fz_server_t s, const int32_t *set_ids, const int32_t *ns,
                    const double *arrival_s, int count, double *latency_s, uint64_t *rows,
                    double *span_s) {
    if (!s || count < 0 || (count > 0 && (!set_ids || !ns || !arrival_s || !latency_s)))
        return set_error(FZ_EINVAL, "null pointer");
    std::vector<uint64_t> tickets((size_t)count, 0);
    std::atomic<int> submitted{0};
    std::atomic<int> drain_rc{FZ_OK};
    double first_submit = 0, last_done = 0;
    // drain: wait for the requests in submission order, record, release
    std::thread drain([&] {
        for (int i = 0; i < count; ++i) {
            while (submitted.load(std::memory_order_acquire) <= i) {
                if (drain_rc.load() != FZ_OK) return;
                std::this_thread::yield();
            }
            fz_result_t r;
            int rc = fz_serve_wait(s, tickets[i], -1, &r);
            if (rc != FZ_OK || r.status != FZ_SERVE_DONE) {
                drain_rc.store(rc != FZ_OK ? rc : r.status);
                return;
            }
            latency_s[i] = r.t_done - r.t_submit;
            if (rows) rows[i] = r.count;
            if (i == 0) first_submit = r.t_submit;
            if (r.t_done > last_done) last_done = r.t_done;
            fz_serve_release(s, tickets[i]);
        }
    });
    const double t0 = now_s();
    int rc = FZ_OK;
    for (int i = 0; i < count && rc == FZ_OK; ++i) {
        while (now_s() < t0 + arrival_s[i]) {
        }
        for (;;) {
            rc = fz_serve_submit(s, set_ids[i], ns[i], &tickets[i]);
            if (rc != FZ_EAGAIN) break;  // queue full: retry
            std::this_thread::yield();
        }
        if (rc == FZ_OK) submitted.store(i + 1, std::memory_order_release);
    }
    if (rc != FZ_OK) drain_rc.store(rc);
    drain.join();
    if (rc != FZ_OK) return rc;
    if (drain_rc.load() != FZ_OK) return set_error(drain_rc.load(), "replayed request failed");
    if (span_s) *span_s = count > 0 ? last_done - first_submit : 0.0;
    return FZ_OK;
}

int fz_serve_stats(fz_server_t s, fz_serve_stats_t *st) {
    if (!s || !st) return set_error(FZ_EINVAL, "null pointer");
    std::lock_guard<std::mutex> lk(s->mu);
    st->queued = s->queue.size();
    st->admitted = s->admitted;
    st->completed = s->completed;
    st->bytes_in_use = s->arena.used();
    st->bytes_budget = s->arena.size();
    st->sets = (int32_t)s->sets.size();
    st->last_error = s->launch_error;
    return FZ_OK;
}

int fz_serve_destroy(fz_server_t s) {
    if (!s) return set_error(FZ_EINVAL, "null pointer");
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->th.joinable()) s->th.join();
    for (cudaStream_t st : s->streams) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    for (auto &kv : s->reqs) delete kv.second;
    for (SetRec &r : s->sets) fz_plan_destroy(r.plan);
    cudaFree(s->arena_base);
    cudaFree(s->counters);
    cudaFreeHost(s->slot_status_host);
    for (Group &G : s->groups) {
        cudaFree(G.dev);
        cudaFreeHost(G.stage);
        cudaFreeHost(G.status_host);
    }
    delete s;
    // device-side failures were reported on the requests they hit
    return FZ_OK;
}

}  // extern "C"
