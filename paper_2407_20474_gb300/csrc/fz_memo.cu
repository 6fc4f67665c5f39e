// fz_memo.cu -- the memo of tail sets, built by the dynamic
// FactorizationsUpToElement pass of Section 2.
//
// For a tail (t_0..t_{k-1}) and top, Memo[r] = Z(r, tail) for r = 0..top-1,
// each list in descending lexicographic order, stored as a CSR (offsets O,
// k int32 per row).  The lists come from the disjoint, lexicographically
// ordered recurrence (Lemma "disjlex", Section 2.1):
//
//   Z(m) = incr_0(Z_{>=0}(m - t_0)) ++ ... ++ incr_{k-1}(Z_{>=k-1}(m - t_{k-1}))
//
// where Z_{>=i}(x), the rows of Z(x) with zeros left of i, is the last
// |Z_{>=i}(x)| = Ct[i][x] rows of Z(x).  Saving those cardinalities (Section
// 2.3) pre-assigns every copy its source and destination; this build writes
// the assignment out as a gather map (one entry per memo row: source row and
// incremented coordinate) in a fully parallel pre-pass.  The copies then run
// elementwise in batches of b = min(tail) consecutive elements (Section 2.2):
// elements m+1..m+b depend only on elements <= m, so every batch is one
// parallel copy-and-increment step (the kernel copyAndIncrementIndex of
// Section 2.4), and batches are separated by a bounded grid barrier inside one
// cooperative launch.  Empty batches need no barrier.
#include <cstdlib>
#include <cstring>
#include <vector>

#include "fz_internal.cuh"

namespace fz {

namespace {

constexpr uint64_t MAP_ZERO = ~0ull;  // the row of Z(0): all zeros
constexpr int THREADS = 256;

struct MapParams {
    const uint64_t *Ct;  // tail count table rows 0..k, stride cs
    int64_t cs;
    const uint64_t *O;
    uint64_t *map;
    int *status;
    int top;
    int k;
    int skip0;  // leave block 0's entries out (the phase fill never reads them)
    int t[FZ_MAX_D];
};

// One warp per element m: lay out the blocks incr_i(Z_{>=i}(m - t_i)).
__global__ void __launch_bounds__(THREADS) memo_map_kernel(MapParams P) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t m = warp; m < P.top; m += nwarps) {
        uint64_t dst = __ldg(P.O + m);
        const uint64_t end = __ldg(P.O + m + 1);
        if (m == 0) {
            if (lane == 0 && end == dst + 1) P.map[dst] = MAP_ZERO;
            if (lane == 0 && end != dst + 1) atomicExch(P.status, (int)DEV_INTERNAL);
            continue;
        }
        for (int i = 0; i < P.k; ++i) {
            const int64_t src_m = m - (int64_t)P.t[i];
            if (src_m < 0) continue;
            const uint64_t len = __ldg(P.Ct + (int64_t)i * P.cs + src_m);
            if (len == 0) continue;
            const uint64_t src = __ldg(P.O + src_m + 1) - len;  // suffix Z_{>=i}(src_m)
            if (dst + len > end) {  // bounds guard: the counts must tile Z(m) exactly
                if (lane == 0) atomicExch(P.status, (int)DEV_INTERNAL);
                break;
            }
            if (i > 0 || !P.skip0)
                for (uint64_t r = lane; r < len; r += 32)
                    P.map[dst + r] = ((src + r) << 4) | (uint64_t)i;
            dst += len;
        }
        if (lane == 0 && dst != end) atomicExch(P.status, (int)DEV_INTERNAL);
    }
}

struct FillParams {
    const uint64_t *O;
    const uint64_t *map;
    int32_t *rows;
    int *status;
    unsigned *bar;  // arrival count of the monotonic grid barrier (zero at launch)
    int top;
    int k;
    int b;        // elements per batch
    int nbatch;
    int L;        // phase fill: elements a phase (the least of t_1..t_{k-1})
};

// The copies run over memo WORDS: word w is coordinate w % k of row w / k.
// A thread first loads the source words of all the words it owns in the
// batch and only then stores them (sources precede the batch, so the loads
// cannot alias the stores): one L2 round trip per batch, not one per row.
constexpr int FILL_W = 4;  // words per thread per pass

struct WordPos {
    uint64_t R;  // row
    uint32_t c;  // coordinate
};

__device__ __forceinline__ WordPos word_pos(uint64_t w, int k) {
    WordPos p;
    p.R = w / (uint64_t)k;
    p.c = (uint32_t)(w - p.R * (uint64_t)k);
    return p;
}

// advance by `nthreads` words, nthreads = qn * k + rn
__device__ __forceinline__ void word_step(WordPos &p, uint64_t qn, uint32_t rn, int k) {
    p.R += qn;
    p.c += rn;
    if (p.c >= (uint32_t)k) {
        p.c -= (uint32_t)k;
        p.R += 1;
    }
}

// Value of one word of a copied row: the source row's word, plus one on the
// incremented coordinate.  False if the map names a source inside the batch.
// LOCAL: every row was written by this CTA (ordered by __syncthreads), so
// the source may come from L1; otherwise it is read from L2 (ld.cg).
template <bool LOCAL>
__device__ __forceinline__ bool word_value(const FillParams &P, uint64_t e, uint32_t c,
                                           uint64_t R0, int32_t &v) {
    if (e == MAP_ZERO) {
        v = 0;
        return true;
    }
    const uint64_t sr = e >> 4;
    if (sr >= R0) return false;  // bounds guard: sources precede the batch
    const int32_t *src = P.rows + sr * (uint64_t)P.k + c;
    v = (LOCAL ? *src : ld_cg_s32(src)) + (c == (uint32_t)(e & 15u) ? 1 : 0);
    return true;
}

// One pass over words base, base + nthreads, ... (FILL_W of them, < W1),
// with the map entries already in e[] when `have_map`.
template <bool HAVE_MAP, bool LOCAL = false>
__device__ __forceinline__ void fill_pass(const FillParams &P, uint64_t base, uint64_t W1,
                                          uint64_t R0, uint64_t nthreads, uint64_t qn,
                                          uint32_t rn, uint64_t (&e)[FILL_W]) {
    const int k = P.k;
    WordPos pos = word_pos(base, k);
    uint32_t c[FILL_W];
#pragma unroll
    for (int j = 0; j < FILL_W; ++j) {
        c[j] = pos.c;
        if (!HAVE_MAP) e[j] = base + j * nthreads < W1 ? __ldg(P.map + pos.R) : MAP_ZERO;
        word_step(pos, qn, rn, k);
    }
    int32_t v[FILL_W];
    unsigned ok = 0;
#pragma unroll
    for (int j = 0; j < FILL_W; ++j)
        if (base + j * nthreads < W1 && word_value<LOCAL>(P, e[j], c[j], R0, v[j]))
            ok |= 1u << j;
#pragma unroll
    for (int j = 0; j < FILL_W; ++j) {
        const uint64_t w = base + j * nthreads;
        if (w < W1) {
            if (ok >> j & 1u)
                P.rows[w] = v[j];
            else
                atomicExch(P.status, (int)DEV_INTERNAL);
        }
    }
}

// Batches of b elements over the whole grid; bounded grid barrier between
// non-empty batches.  One CTA of GRID_THREADS per SM, so a barrier has one
// arrival per SM, and a batch of up to FILL_W * GRID_THREADS * SMs words
// (about 620k words on 152 SMs) is one pass.  The gather-map entries of the
// next batch's first pass do not depend on this batch: they are loaded
// before the barrier.
constexpr int GRID_THREADS = 1024;

__global__ void __launch_bounds__(GRID_THREADS) memo_fill_kernel(FillParams P) {
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t nthreads = (uint64_t)gridDim.x * blockDim.x;
    const int k = P.k;
    const uint64_t qn = nthreads / (uint64_t)k;
    const uint32_t rn = (uint32_t)(nthreads - qn * (uint64_t)k);
    uint64_t e[FILL_W];
    bool have = false;  // e[] holds the map entries of this batch's first pass
    unsigned nbar = 0;  // barriers passed
    uint64_t R0 = __ldg(P.O + 0);
    for (int q = 0; q < P.nbatch; ++q) {
        const int64_t m0 = (int64_t)q * P.b;
        int64_t m1 = m0 + P.b;
        if (m1 > P.top) m1 = P.top;
        const uint64_t R1 = __ldg(P.O + m1);  // R0 carried over from the previous batch
        if (R1 == R0) {
            have = false;
            continue;
        }
        const uint64_t W1 = R1 * (uint64_t)k;
        uint64_t base = R0 * (uint64_t)k + tid;
        if (have && base < W1) {
            fill_pass<true>(P, base, W1, R0, nthreads, qn, rn, e);
            base += FILL_W * nthreads;
        }
        for (; base < W1; base += FILL_W * nthreads) fill_pass<false>(P, base, W1, R0, nthreads, qn, rn, e);
        have = false;
        if (q + 1 < P.nbatch) {
            // prefetch the next batch's first-pass map entries (the map and
            // the offsets are read-only here)
            int64_t n1 = m1 + P.b;
            if (n1 > P.top) n1 = P.top;
            const uint64_t NR1 = __ldg(P.O + n1);
            const uint64_t NW1 = NR1 * (uint64_t)k;
            const uint64_t nbase = R1 * (uint64_t)k + tid;
            if (NR1 > R1 && nbase < NW1) {
                WordPos pos = word_pos(nbase, k);
#pragma unroll
                for (int j = 0; j < FILL_W; ++j) {
                    e[j] = nbase + j * nthreads < NW1 ? __ldg(P.map + pos.R) : MAP_ZERO;
                    word_step(pos, qn, rn, k);
                }
                have = true;
            }
            if (!grid_barrier_mono(P.bar, nbar++, P.status)) return;
        }
        R0 = R1;
    }
}

// Phase fill.  Block 0 of Z(m) is Z(m - t_0) with coordinate 0 raised by
// one, row for row (Corollary "resultislex" orders the blocks by i), so word
// w of element m, while w < |Z(m - t_0)| k, is word w of element m - t_0 plus
// one when w is coordinate 0; every other word's source lies at least L =
// min(t_1..t_{k-1}) elements back.  Along a class m mod t_0 the element sizes
// never shrink (block 0 is the previous element), so a (class, word) chain is
// born once and stays.  Each chain belongs to one thread for the whole fill
// (a fixed bound per class: its last element's words), and the memo is
// filled in phases of L elements:
//   pass A: the chains alive when the phase starts hold only block-0 words
//     in it, computed from the thread's own last word of the chain (kept for
//     its first PH_J chains, else re-read from its own store);
//   wait at the grid barrier of the previous phase;
//   pass B: the chains born in the phase, their first word from the gather
//     map (sources L or more elements back, so in earlier phases), the rest
//     block 0;
//   arrive at this phase's barrier.
// Pass A needs no other thread's writes, so it overlaps the barrier.  With
// t_1 >= 2 t_0 there are L / t_0 times fewer barriers than batches of t_0
// elements (the d = 5 memo with tail (4, 20, 22, 31, 39): 75 instead of 375).
constexpr int PH_J = 32;

__global__ void __launch_bounds__(GRID_THREADS) memo_fill_phase_kernel(FillParams P) {
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t nthreads = (uint64_t)gridDim.x * blockDim.x;
    const uint32_t uk = (uint32_t)P.k;
    const int64_t t0 = P.b;
    const int64_t ncl = P.top < t0 ? P.top : t0;
    uint64_t wc = 0;  // words of the widest class's last element
    for (int64_t e = 0; e < ncl; ++e) {
        const int64_t ml = e + ((P.top - 1 - e) / t0) * t0;
        const uint64_t sz = __ldg(P.O + ml + 1) - __ldg(P.O + ml);
        if (sz > wc) wc = sz;
    }
    wc *= uk;
    // chain ch: word w = 32 (ch / 32 div ncl) + ch mod 32 of class (ch / 32)
    // mod ncl -- a warp's lanes take 32 neighbouring words of one class, and
    // a thread's chains (ch = tid + j nthreads) grow in w with j, so a phase
    // stops at its widest element
    // (32-bit chain indices: the host launches this fill only when
    // t_0 x rows x k stays below 2^31)
    const uint32_t nblk = (uint32_t)((wc + 31) / 32);
    const uint32_t ucl = (uint32_t)ncl, ut0 = (uint32_t)t0;
    const uint32_t nch = ucl * nblk * 32u;
    const uint32_t nth = (uint32_t)nthreads, utid = (uint32_t)tid;
    const uint32_t J = (nch + nth - 1) / nth;
    int32_t last[PH_J];
    unsigned nbar = 0;
    for (int64_t ma = 0; ma < P.top; ma += P.L) {
        const int64_t mb = ma + P.L < P.top ? ma + P.L : P.top;
        const uint32_t mr = (uint32_t)(ma % t0);
        // the phase's widest element: sizes never shrink along a class, so
        // it is one of the classes' last elements in the phase
        uint64_t wp = 0;
        for (int64_t e = 0; e < ncl; ++e) {
            const int64_t ml = mb - 1 - (int64_t)(((uint32_t)((mb - 1) % t0) - (uint32_t)e + ut0) % ut0);
            if (ml < ma) continue;
            const uint64_t sz = __ldg(P.O + ml + 1) - __ldg(P.O + ml);
            if (sz > wp) wp = sz;
        }
        wp *= uk;
        // pass A
        for (uint32_t j = 0; j < J; ++j) {
            const uint32_t ch = utid + j * nth;
            if (ch >= nch) break;
            const uint32_t q = ch >> 5;
            const uint32_t qd = q / ucl;
            const int64_t e = (int64_t)(q - qd * ucl);
            const uint64_t w = (uint64_t)qd * 32u + (ch & 31u);
            if (w >= wp) break;
            const int64_t m1 = ma + (int64_t)(((uint32_t)e - mr + ut0) % ut0);  // the class's first element here
            if (m1 >= mb || m1 < t0) continue;
            const uint64_t op = __ldg(P.O + m1 - t0);
            if (w >= (__ldg(P.O + m1 - t0 + 1) - op) * uk) continue;  // not alive yet
            int32_t prev = j < PH_J ? last[j] : P.rows[op * uk + w];
            const int32_t inc = ((uint32_t)w % uk) == 0 ? 1 : 0;
            for (int64_t m = m1; m < mb; m += t0) {
                prev += inc;
                P.rows[__ldg(P.O + m) * uk + w] = prev;
            }
            if (j < PH_J) last[j] = prev;
        }
        if (ma > 0 && !grid_wait(P.bar, nbar - 1, P.status)) return;
        // pass B
        const uint64_t R0 = __ldg(P.O + ma);
        for (uint32_t j = 0; j < J; ++j) {
            const uint32_t ch = utid + j * nth;
            if (ch >= nch) break;
            const uint32_t q = ch >> 5;
            const uint32_t qd = q / ucl;
            const int64_t e = (int64_t)(q - qd * ucl);
            const uint64_t w = (uint64_t)qd * 32u + (ch & 31u);
            if (w >= wp) break;
            const int64_t m1 = ma + (int64_t)(((uint32_t)e - mr + ut0) % ut0);
            if (m1 >= mb) continue;
            if (m1 >= t0 && w < (__ldg(P.O + m1 - t0 + 1) - __ldg(P.O + m1 - t0)) * uk)
                continue;  // alive: done in pass A
            const uint32_t c = (uint32_t)w % uk;
            int32_t prev = 0;
            bool have = false;
            for (int64_t m = m1; m < mb; m += t0) {
                const uint64_t o = __ldg(P.O + m);
                if (w >= (__ldg(P.O + m + 1) - o) * uk) continue;  // not born yet
                int32_t v;
                if (have) {
                    v = prev + (c == 0 ? 1 : 0);  // block 0 after the birth
                } else if (!word_value<false>(P, __ldg(P.map + o + w / uk), c, R0, v)) {
                    atomicExch(P.status, (int)DEV_INTERNAL);
                    v = 0;
                }
                P.rows[o * uk + w] = v;
                prev = v;
                have = true;
            }
            if (have && j < PH_J) last[j] = prev;
        }
        if (mb < P.top) {
            grid_arrive(P.bar);
            ++nbar;
        }
    }
}

// ---------------------------------------------------------------------------
// Memos of depth 1 and 2 in closed form (plans only; the dynamic pass above
// builds the same rows).  Z(m, (t0)) is the row (m / t0) when t0 divides m;
// Z(m, (t0, t1)) is the progression a0 = a_top, a_top - h1, ... (descending,
// so the rows come out in the memo's order) with a1 = (m - a0 t0) / t1, h1 =
// t1 / gcd, a_top the largest a0 <= m / t0 with t1 | m - a0 t0.  One warp per
// element; offsets O from the count scan.  A row count that disagrees with
// the closed form is recorded as DEV_INTERNAL.
// ---------------------------------------------------------------------------
struct ClosedParams {
    const uint64_t *O;
    int32_t *rows;
    int *status;
    int top, k;
    int64_t t0, t1, e, h1, g1, inv;
};

__global__ void __launch_bounds__(THREADS) memo_closed_kernel(ClosedParams P) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t m = warp; m < P.top; m += nwarps) {
        const uint64_t beg = __ldg(P.O + m);
        const uint64_t cnt = __ldg(P.O + m + 1) - beg;
        if (P.k == 1) {
            const uint64_t want = (m % P.t0 == 0) ? 1u : 0u;
            if (lane == 0) {
                if (cnt != want)
                    atomicExch(P.status, (int)DEV_INTERNAL);
                else if (cnt)
                    P.rows[beg] = (int32_t)(m / P.t0);
            }
            continue;
        }
        int64_t atop = -1;
        uint64_t want = 0;
        if (m % P.e == 0) {
            const int64_t astar = ((m / P.e) % P.h1) * P.inv % P.h1;
            const int64_t q = m / P.t0;
            if (q >= astar) {
                atop = q - (q - astar) % P.h1;
                want = (uint64_t)(atop / P.h1) + 1;
            }
        }
        if (cnt != want) {
            if (lane == 0) atomicExch(P.status, (int)DEV_INTERNAL);
            continue;
        }
        for (uint64_t j = lane; j < cnt; j += 32) {
            const int64_t a0 = atop - (int64_t)j * P.h1;
            P.rows[(beg + j) * 2] = (int32_t)a0;
            P.rows[(beg + j) * 2 + 1] = (int32_t)((m - a0 * P.t0) / P.t1);
        }
    }
}

}  // namespace

int launch_memo_closed(const int32_t *tail, int k, int32_t top, const uint64_t *O,
                       int32_t *rows, int *status, cudaStream_t s) {
    if (top <= 0) return FZ_OK;
    if (k != 1 && k != 2) return set_error(FZ_EINTERNAL, "closed-form memo: depth 1 or 2 only");
    ClosedParams P{};
    P.O = O;
    P.rows = rows;
    P.status = status;
    P.top = top;
    P.k = k;
    P.t0 = tail[0];
    P.t1 = k == 2 ? tail[1] : 1;
    P.e = 1;
    P.h1 = 1;
    if (k == 2) pair_params(P.t0, P.t1, &P.e, &P.h1, &P.g1, &P.inv);
    int64_t blocks = ((int64_t)top * 32 + THREADS - 1) / THREADS;
    if (blocks > 4096) blocks = 4096;
    memo_closed_kernel<<<(int)blocks, THREADS, 0, s>>>(P);
    note_launch();
    FZ_CUDA_TRY(cudaGetLastError());
    return FZ_OK;
}

namespace {

// ---------------------------------------------------------------------------
// Cluster variant: one thread-block cluster runs every batch.  Between
// batches the CTAs meet at the hardware cluster barrier; the arrive and the
// wait are split so that the gather-map entries of the next batch's first
// pass (which do not depend on the current batch) are loaded while the
// barrier completes.  Source words written by other CTAs of the cluster are
// read from L2 (ld.cg).  ONE_CTA: a single CTA (no cluster) for memos whose
// batches are a few rows each -- __syncthreads between batches and sources
// from L1.  Instances: 16 x 1024 threads; 16 x 256 threads at <= 48
// registers (fits beside an enumeration capped at 3 CTAs per SM); 1 x 1024.
// ---------------------------------------------------------------------------
constexpr int CL_THREADS = 1024;
constexpr int CL_SMALL_THREADS = 256;
constexpr uint64_t ONE_CTA_MAX_WORDS = 2048;  // average words per batch

__device__ __forceinline__ unsigned cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ unsigned cluster_size() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ void cluster_arrive_release() {
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}

__device__ __forceinline__ void cluster_wait_acquire() {
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ void prefetch_map(const FillParams &P, uint64_t base, uint64_t W1,
                                             uint64_t nthreads, uint64_t qn, uint32_t rn,
                                             uint64_t (&e)[FILL_W]) {
    WordPos pos = word_pos(base, P.k);
#pragma unroll
    for (int j = 0; j < FILL_W; ++j) {
        e[j] = base + j * nthreads < W1 ? __ldg(P.map + pos.R) : MAP_ZERO;
        word_step(pos, qn, rn, P.k);
    }
}

template <int MAXT, int MINB, bool ONE_CTA>
__global__ void __launch_bounds__(MAXT, MINB) memo_fill_cluster_kernel(FillParams P) {
    const uint64_t tid = (ONE_CTA ? 0u : (uint64_t)cluster_rank() * blockDim.x) + threadIdx.x;
    const uint64_t nthreads = (ONE_CTA ? 1u : (uint64_t)cluster_size()) * blockDim.x;
    const int k = P.k;
    const uint64_t qn = nthreads / (uint64_t)k;
    const uint32_t rn = (uint32_t)(nthreads - qn * (uint64_t)k);
    // batch 0 boundaries and map entries
    uint64_t R0 = __ldg(P.O), R1 = __ldg(P.O + (P.b < P.top ? P.b : P.top));
    uint64_t e[FILL_W];
    prefetch_map(P, R0 * k + tid, R1 * k, nthreads, qn, rn, e);
    for (int q = 0; q < P.nbatch; ++q) {
        const uint64_t W0 = R0 * (uint64_t)k, W1 = R1 * (uint64_t)k;
        if (W1 != W0) {
            fill_pass<true, ONE_CTA>(P, W0 + tid, W1, R0, nthreads, qn, rn, e);
            for (uint64_t base = W0 + tid + FILL_W * nthreads; base < W1;
                 base += FILL_W * nthreads)
                fill_pass<false, ONE_CTA>(P, base, W1, R0, nthreads, qn, rn, e);
        }
        // next batch's boundaries and first map entries (independent of this batch)
        const bool more = q + 1 < P.nbatch;
        uint64_t N1 = R1;
        if (more) {
            int64_t m1 = (int64_t)(q + 2) * P.b;
            if (m1 > P.top) m1 = P.top;
            N1 = __ldg(P.O + m1);
        }
        if (ONE_CTA) {
            prefetch_map(P, R1 * k + tid, N1 * k, nthreads, qn, rn, e);
            if (W1 != W0 && more) __syncthreads();
        } else {
            if (W1 != W0 && more) cluster_arrive_release();
            prefetch_map(P, R1 * k + tid, N1 * k, nthreads, qn, rn, e);
            if (W1 != W0 && more) cluster_wait_acquire();
        }
        R0 = R1;
        R1 = N1;
    }
}

// ---------------------------------------------------------------------------
// Launch-per-step schedules (Section 2.2 and the factorizationwise parallel
// algorithm of Section 2.4), kept for comparison with the single-launch
// build above.
//
// Per batch ("both" parallelism): one launch per elementwise batch, covering
// every copy of the batch; consecutive launches on one stream order the
// batches.
__global__ void __launch_bounds__(THREADS) memo_batch_kernel(FillParams P, int q) {
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t nthreads = (uint64_t)gridDim.x * blockDim.x;
    const int k = P.k;
    const uint64_t qn = nthreads / (uint64_t)k;
    const uint32_t rn = (uint32_t)(nthreads - qn * (uint64_t)k);
    const int64_t m0 = (int64_t)q * P.b;
    int64_t m1 = m0 + P.b;
    if (m1 > P.top) m1 = P.top;
    const uint64_t R0 = __ldg(P.O + m0), R1 = __ldg(P.O + m1);
    const uint64_t W1 = R1 * (uint64_t)k;
    for (uint64_t base = R0 * (uint64_t)k + tid; base < W1; base += FILL_W * nthreads) {
        uint64_t e[FILL_W];
        fill_pass<false>(P, base, W1, R0, nthreads, qn, rn, e);
    }
}

// Per copy (factorizationwise): one launch per (m, i), the kernel
// copyAndIncrementIndex -- `len` rows from row `src` to row `dst`, coordinate
// `inc` plus one, one thread per word.
__global__ void __launch_bounds__(THREADS) copy_and_increment_kernel(int32_t *rows, int k,
                                                                     uint64_t dst, uint64_t src,
                                                                     uint64_t len, int inc) {
    const uint64_t words = len * (uint64_t)k;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t w = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; w < words; w += stride) {
        const uint64_t r = w / (uint64_t)k;
        const int c = (int)(w - r * (uint64_t)k);
        rows[dst * k + w] = rows[src * k + w] + (c == inc ? 1 : 0);
    }
}

__global__ void zero_row_kernel(int32_t *rows, int k) {
    if (threadIdx.x < (unsigned)k) rows[threadIdx.x] = 0;
}

int coop_grid(const void *kernel, int threads) {
    DeviceProps dp;
    if (device_props(&dp) != FZ_OK) return -1;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) !=
        cudaSuccess)
        return -1;
    if (per_sm < 1) return -1;
    if (per_sm > 1) per_sm = 1;  // one CTA per SM: one barrier arrival per SM
    return per_sm * dp.sms;
}

// One cluster of 16 CTAs (8 if 16 cannot be co-scheduled).  Returns
// FZ_ECUDA without launching if no cluster shape fits.
template <int MAXT, int MINB>
static int launch_fill_cluster_t(FillParams fp, int threads, cudaStream_t s) {
    auto kern = memo_fill_cluster_kernel<MAXT, MINB, false>;
    static DeviceOnce attr_set;
    int dev = 0;
    FZ_CUDA_TRY(cudaGetDevice(&dev));
    if (!attr_set.is_set(dev)) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        attr_set.set(dev);
    }
    for (int csize : {16, 8}) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(csize);
        cfg.blockDim = dim3(threads);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = csize;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int nclusters = 0;
        if (cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg) != cudaSuccess ||
            nclusters < 1) {
            cudaGetLastError();
            continue;
        }
        cudaError_t e = cudaLaunchKernelEx(&cfg, kern, fp);
        if (e != cudaSuccess) return cuda_error(e, "memo fill (cluster) launch");
        note_launch();
        return FZ_OK;
    }
    return set_error(FZ_ECUDA, "memo fill: no cluster shape fits");
}

int launch_fill_cluster(FillParams fp, bool small_ctas, cudaStream_t s) {
    // FZ_MEMO_CL_THREADS=256|512|1024 sets the CTA size of the large
    // variant (tuning only)
    static const int threads = [] {
        const char *e = getenv("FZ_MEMO_CL_THREADS");
        const int t = e ? atoi(e) : CL_THREADS;
        return (t == 256 || t == 512 || t == 1024) ? t : CL_THREADS;
    }();
    if (small_ctas)
        return launch_fill_cluster_t<CL_SMALL_THREADS, 5>(fp, CL_SMALL_THREADS, s);
    return launch_fill_cluster_t<CL_THREADS, 1>(fp, threads, s);
}

int launch_fill_one_cta(FillParams fp, cudaStream_t s) {
    memo_fill_cluster_kernel<CL_THREADS, 1, true><<<1, CL_THREADS, 0, s>>>(fp);
    note_launch();
    FZ_CUDA_TRY(cudaGetLastError());
    return FZ_OK;
}

// ---------------------------------------------------------------------------
// Many small memos at once (batched instances): one CTA per memo runs the
// whole dynamic pass for it -- the offsets by a block-wide scan of the tail's
// row counts, then the elementwise batches of b = min(tail) elements, each a
// set of copy-and-increment steps incr_i(Z_{>=i}(m - t_i)) with warps over
// elements and lanes over rows, separated by __syncthreads (all the data of
// one memo stays inside one CTA, so CTA-scope ordering suffices).
// ---------------------------------------------------------------------------
constexpr int MB_THREADS = 256;

__device__ uint64_t block_exclusive_scan(uint64_t v, uint64_t *smem_warp_sums,
                                         uint64_t *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    uint64_t incl = warp_incl_scan(v, lane);
    if (lane == 31) smem_warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint64_t x = lane < nwarps ? smem_warp_sums[lane] : 0ull;
        uint64_t xi = warp_incl_scan(x, lane);
        if (lane < nwarps) smem_warp_sums[lane] = xi - x;  // exclusive
        if (lane == nwarps - 1) smem_warp_sums[32] = xi;
    }
    __syncthreads();
    const uint64_t r = smem_warp_sums[warp] + incl - v;
    *total = smem_warp_sums[32];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(MB_THREADS) memo_sizes_kernel(const MemoJob *__restrict__ jobs,
                                                                uint64_t *__restrict__ rows_out) {
    __shared__ uint64_t sums[33];
    const MemoJob J = jobs[blockIdx.x];
    uint64_t acc = 0;
    for (int r = threadIdx.x; r < J.top; r += blockDim.x) acc += __ldg(J.Ct + r);
    uint64_t total;
    block_exclusive_scan(acc, sums, &total);
    if (threadIdx.x == 0) rows_out[blockIdx.x] = total;
}

// One CTA of T threads per memo.  Inside an elementwise batch each warp
// copies whole (element, generator) blocks as flat word copies; a lane loads
// MB_ILP words before it stores them, so a block of W words costs about
// W / (32 MB_ILP) L2 round trips.  The kernel needs 57 registers a thread
// (64 allocated), so 1024 threads fit on an SM: one CTA of 1024, or several
// smaller CTAs, each building its own memo.
constexpr int MB_ILP = 8;
constexpr int MB_CTA_THREADS_DEFAULT = 512;

// PAR: lanes 0..k-1 load the lengths and source offsets of an element's k
// blocks at once (one round of loads per element) instead of each block's
// before its copy (two dependent rounds per block).
template <bool PAR>
__device__ __forceinline__ void memo_cta_build_body(const MemoJob &J, uint64_t *sums,
                                                    int *status) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int k = J.k;
    // offsets: O[0] = 0, O[m+1] = O[m] + |Z(m, tail)| (chunked block scan)
    uint64_t carry = 0;
    for (int base = 0; base < J.top; base += blockDim.x) {
        const int m = base + threadIdx.x;
        const uint64_t v = m < J.top ? __ldg(J.Ct + m) : 0ull;
        uint64_t tot;
        const uint64_t ex = block_exclusive_scan(v, sums, &tot);
        if (m < J.top) J.O[m] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) J.O[J.top] = carry;
    __syncthreads();
    if (carry != J.rows) {
        if (threadIdx.x == 0) atomicExch(status, (int)DEV_INTERNAL);
        return;
    }
    // elementwise batches of b elements
    for (int m0 = 0; m0 < J.top; m0 += J.b) {
        const int m1 = m0 + J.b < J.top ? m0 + J.b : J.top;
        for (int m = m0 + warp; m < m1; m += nwarps) {
            uint64_t dst = J.O[m];
            if (m == 0) {
                if (lane < k) J.R[lane] = 0;
                continue;
            }
            uint64_t plen = 0, psrc = 0;
            if (PAR && lane < k) {
                const int sm = m - J.t[lane];
                if (sm >= 0) {
                    plen = __ldg(J.Ct + (int64_t)lane * J.cs + sm);
                    psrc = J.O[sm + 1] - plen;  // suffix Z_{>=lane}(sm)
                }
            }
            for (int i = 0; i < k; ++i) {
                uint64_t len, src;
                if (PAR) {
                    len = shfl_u64(plen, i);
                    src = shfl_u64(psrc, i);
                    if (len == 0) continue;
                } else {
                    const int src_m = m - J.t[i];
                    if (src_m < 0) continue;
                    len = __ldg(J.Ct + (int64_t)i * J.cs + src_m);
                    if (len == 0) continue;
                    src = J.O[src_m + 1] - len;  // suffix Z_{>=i}(src_m)
                }
                // the block is a flat copy of len * k words with one added to
                // every word of coordinate i: word w of the block is
                // coordinate w mod k of row w div k
                const uint64_t W = len * (uint64_t)k;
                const int32_t *a = J.R + src * (uint64_t)k;
                int32_t *b = J.R + dst * (uint64_t)k;
                const uint32_t step = (uint32_t)(32 % k);
                uint32_t c0 = (uint32_t)(lane % k);  // coordinate of word lane
                for (uint64_t w0 = lane; w0 < W; w0 += 32 * MB_ILP) {
                    int32_t v[MB_ILP];
#pragma unroll
                    for (int u = 0; u < MB_ILP; ++u)
                        if (w0 + 32 * u < W) v[u] = a[w0 + 32 * u];
                    uint32_t c = c0;
#pragma unroll
                    for (int u = 0; u < MB_ILP; ++u) {
                        if (w0 + 32 * u < W) b[w0 + 32 * u] = v[u] + (c == (uint32_t)i ? 1 : 0);
                        c += step;
                        if (c >= (uint32_t)k) c -= (uint32_t)k;
                    }
                    c0 = c;
                }
                dst += len;
            }
        }
        __syncthreads();
    }
}

template <int T, bool PAR>
__global__ void __launch_bounds__(T, 1024 / T) memo_cta_build_kernel(
    const MemoJob *__restrict__ jobs, int *status) {
    __shared__ uint64_t sums[33];
    const MemoJob J = jobs[blockIdx.x];
    memo_cta_build_body<PAR>(J, sums, status);
}

// Element groups.  Most elements of a batch memo are a few rows (a batch of
// 4096 instances of widths 3..8: 95 % of 1.7e7 elements hold at most 256
// words), and a warp that takes them one at a time pays a chain of
// dependent loads (the element's offset, then its blocks' lengths and
// sources, then the copy) for a handful of words.
// Here each warp owns a contiguous run of the batch's elements and takes
// them G = floor(32 / k) at a time: lane j loads the length and source of
// block j mod k of element j div k, all in one round; a warp scan of the
// lengths gives every block its first row (the group's rows are contiguous,
// so the scan total must meet the next element's offset).  A group of at
// most MG_FLAT_WORDS words is then copied as one flat range: each word finds
// its block by a binary search over the lanes' first rows (shuffles; empty
// blocks share their successor's first row and are never the last block
// starting at or before a row).  Larger groups copy block by block, as the
// one-element build does.  One __syncthreads per elementwise batch: a
// warp's groups never read rows of its own batch.
constexpr uint64_t MG_FLAT_WORDS = 4 * 32 * MB_ILP;

__device__ __forceinline__ uint32_t warp_incl_scan_u32(uint32_t v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(FULL, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

__device__ __forceinline__ void memo_group_build_body(const MemoJob &J, uint64_t *sums,
                                                      int32_t *s_t, int *status) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int k = J.k;
    uint64_t carry = 0;
    for (int base = 0; base < J.top; base += blockDim.x) {
        const int m = base + threadIdx.x;
        const uint64_t v = m < J.top ? __ldg(J.Ct + m) : 0ull;
        uint64_t tot;
        const uint64_t ex = block_exclusive_scan(v, sums, &tot);
        if (m < J.top) J.O[m] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) J.O[J.top] = carry;
    if (threadIdx.x < FZ_MAX_D) s_t[threadIdx.x] = (int)threadIdx.x < k ? J.t[threadIdx.x] : 0;
    __syncthreads();
    if (carry != J.rows || k < 1 || k > FZ_MAX_D) {
        if (threadIdx.x == 0) atomicExch(status, (int)DEV_INTERNAL);
        return;
    }
    const int G = 32 / k;                          // elements per group
    const int je = lane / k, ji = lane - je * k;   // lane's (element, block) in a group
    const uint32_t uk = (uint32_t)k, rstep = 32u / uk, cstep = 32u % uk;
    int32_t *R = J.R;
    for (int m0 = 0; m0 < J.top; m0 += J.b) {
        const int m1 = m0 + J.b < J.top ? m0 + J.b : J.top;
        const int ne = m1 - m0;
        const int e_lo = m0 + (int)(((int64_t)warp * ne) / nwarps);
        const int e_hi = m0 + (int)(((int64_t)(warp + 1) * ne) / nwarps);
        for (int eb = e_lo; eb < e_hi; eb += G) {
            const int ge = e_hi - eb < G ? e_hi - eb : G;
            const int npair = ge * k;
            uint32_t len = 0, src = 0;
            if (lane < npair) {
                const int sm = eb + je - s_t[ji];
                if (sm >= 0) {
                    const uint64_t l = __ldg(J.Ct + (int64_t)ji * J.cs + sm);
                    len = (uint32_t)l;
                    src = (uint32_t)(J.O[sm + 1] - l);  // suffix Z_{>=ji}(sm)
                }
            }
            const uint32_t ob = (uint32_t)J.O[eb], oe = (uint32_t)J.O[eb + ge];
            const uint32_t z = eb == 0 ? 1u : 0u;  // Z(0): one zero row before the blocks
            const uint32_t incl = warp_incl_scan_u32(len, lane);
            const uint32_t rbeg = ob + z;
            const uint32_t dst = rbeg + incl - len;
            if (rbeg + __shfl_sync(FULL, incl, 31) != oe) {
                if (lane == 0) atomicExch(status, (int)DEV_INTERNAL);
                continue;
            }
            if (z && lane < k) R[lane] = 0;
            const uint64_t W = (uint64_t)(oe - rbeg) * uk;
            if (W <= MG_FLAT_WORDS) {
                const uint32_t key = lane < npair ? dst : 0xffffffffu;
                const uint64_t obase = (uint64_t)rbeg * uk;
                for (uint32_t w0 = 0; w0 < (uint32_t)W; w0 += 32u * MB_ILP) {
                    const uint32_t wl = w0 + (uint32_t)lane;
                    uint32_t r = rbeg + wl / uk, c = wl % uk;
                    int32_t v[MB_ILP];
                    uint32_t inc = 0;
#pragma unroll
                    for (int u = 0; u < MB_ILP; ++u) {
                        int p = 0;  // the last block starting at or before row r
#pragma unroll
                        for (int st = 16; st >= 1; st >>= 1)
                            if (__shfl_sync(FULL, key, p + st) <= r) p += st;
                        const uint32_t sp = __shfl_sync(FULL, src, p);
                        const uint32_t dp = __shfl_sync(FULL, dst, p);
                        const int ip = __shfl_sync(FULL, ji, p);
                        if (wl + 32u * u < (uint32_t)W) {
                            v[u] = R[(uint64_t)(sp + (r - dp)) * uk + c];
                            if (c == (uint32_t)ip) inc |= 1u << u;
                        }
                        r += rstep;
                        c += cstep;
                        if (c >= uk) {
                            c -= uk;
                            ++r;
                        }
                    }
#pragma unroll
                    for (int u = 0; u < MB_ILP; ++u)
                        if (wl + 32u * u < (uint32_t)W)
                            R[obase + wl + 32u * u] = v[u] + (int32_t)((inc >> u) & 1u);
                }
            } else {
                for (int j = 0; j < npair; ++j) {
                    const uint32_t l = __shfl_sync(FULL, len, j);
                    if (l == 0) continue;
                    const uint32_t sj = __shfl_sync(FULL, src, j);
                    const uint32_t dj = __shfl_sync(FULL, dst, j);
                    const uint32_t i = (uint32_t)(j % k);
                    const uint64_t Wb = (uint64_t)l * uk;
                    const int32_t *a = R + (uint64_t)sj * uk;
                    int32_t *b = R + (uint64_t)dj * uk;
                    uint32_t c0 = (uint32_t)lane % uk;
                    for (uint64_t w0 = lane; w0 < Wb; w0 += 32 * MB_ILP) {
                        int32_t v[MB_ILP];
#pragma unroll
                        for (int u = 0; u < MB_ILP; ++u)
                            if (w0 + 32 * u < Wb) v[u] = a[w0 + 32 * u];
                        uint32_t c = c0;
#pragma unroll
                        for (int u = 0; u < MB_ILP; ++u) {
                            if (w0 + 32 * u < Wb) b[w0 + 32 * u] = v[u] + (c == i ? 1 : 0);
                            c += cstep;
                            if (c >= uk) c -= uk;
                        }
                        c0 = c;
                    }
                }
            }
        }
        __syncthreads();
    }
}

template <int T>
__global__ void __launch_bounds__(T, 1024 / T) memo_group_cta_kernel(
    const MemoJob *__restrict__ jobs, int *status) {
    __shared__ uint64_t sums[33];
    __shared__ int32_t s_t[FZ_MAX_D];
    const MemoJob J = jobs[blockIdx.x];
    memo_group_build_body(J, sums, s_t, status);
}

// One memo built by all CTAs of a thread-block cluster: the same elementwise
// batches as the one-CTA build, with the elements of a batch spread over the
// warps of the whole cluster (wpe warps to an element, interleaving its words,
// when a batch has fewer elements than the cluster has warps) and the
// hardware cluster barrier (release/acquire) between batches.  Every CTA
// computes the offsets; rank 0 stores them.  Offsets and sources, stored by
// other CTAs, are read from L2 (ld.global.cg): a line of L1 could hold rows
// of a batch that another CTA was still writing.  All CTAs of the cluster
// pass the same sequence of barriers: the batch loop and the one early
// return depend only on the job.
__device__ __forceinline__ void memo_coop_build_body(const MemoJob &J, unsigned part,
                                                     unsigned nparts, uint64_t *sums,
                                                     int *status) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int k = J.k;
    uint64_t carry = 0;
    for (int base = 0; base < J.top; base += blockDim.x) {
        const int m = base + threadIdx.x;
        const uint64_t v = m < J.top ? __ldg(J.Ct + m) : 0ull;
        uint64_t tot;
        const uint64_t ex = block_exclusive_scan(v, sums, &tot);
        if (part == 0 && m < J.top) J.O[m] = carry + ex;
        carry += tot;
    }
    if (part == 0 && threadIdx.x == 0) J.O[J.top] = carry;
    __syncthreads();
    if (carry != J.rows) {
        if (part == 0 && threadIdx.x == 0) atomicExch(status, (int)DEV_INTERNAL);
        return;
    }
    cluster_arrive_release();
    cluster_wait_acquire();
    const int tw = (int)nparts * nwarps;  // warps of the cluster
    const int gw = (int)part * nwarps + warp;
    for (int m0 = 0; m0 < J.top; m0 += J.b) {
        const int m1 = m0 + J.b < J.top ? m0 + J.b : J.top;
        const int ne = m1 - m0;
        const int wpe = tw >= 2 * ne ? tw / ne : 1;
        const int groups = tw / wpe;
        const int sub = gw % wpe;
        const uint32_t stride = 32u * (uint32_t)wpe;
        const uint32_t step = stride % (uint32_t)k;
        for (int e = gw / wpe; e < ne && gw < groups * wpe; e += groups) {
            const int m = m0 + e;
            uint64_t dst = __ldcg(J.O + m);
            if (m == 0) {
                if (sub == 0 && lane < k) J.R[lane] = 0;
                continue;
            }
            uint64_t plen = 0, psrc = 0;
            if (lane < k) {
                const int sm = m - J.t[lane];
                if (sm >= 0) {
                    plen = __ldg(J.Ct + (int64_t)lane * J.cs + sm);
                    psrc = __ldcg(J.O + sm + 1) - plen;  // suffix Z_{>=lane}(sm)
                }
            }
            for (int i = 0; i < k; ++i) {
                const uint64_t len = shfl_u64(plen, i);
                const uint64_t src = shfl_u64(psrc, i);
                if (len == 0) continue;
                const uint64_t W = len * (uint64_t)k;
                const int32_t *a = J.R + src * (uint64_t)k;
                int32_t *b = J.R + dst * (uint64_t)k;
                const uint64_t first = (uint64_t)sub * 32u + (uint64_t)lane;
                uint32_t c0 = (uint32_t)(first % (uint64_t)k);
                for (uint64_t w0 = first; w0 < W; w0 += (uint64_t)stride * MB_ILP) {
                    int32_t v[MB_ILP];
#pragma unroll
                    for (int u = 0; u < MB_ILP; ++u)
                        if (w0 + (uint64_t)stride * u < W) v[u] = __ldcg(a + w0 + (uint64_t)stride * u);
                    uint32_t c = c0;
#pragma unroll
                    for (int u = 0; u < MB_ILP; ++u) {
                        if (w0 + (uint64_t)stride * u < W)
                            b[w0 + (uint64_t)stride * u] = v[u] + (c == (uint32_t)i ? 1 : 0);
                        c += step;
                        if (c >= (uint32_t)k) c -= (uint32_t)k;
                    }
                    c0 = c;
                }
                dst += len;
            }
        }
        cluster_arrive_release();
        cluster_wait_acquire();
    }
}

// Persistent build of a batch's memos, jobs sorted longest first: cluster c
// < ncoop builds job c cooperatively, then every CTA claims the remaining
// jobs one at a time (claim counter zeroed before the launch), so the short
// memos fill in behind the long ones as in the one-CTA launch.  Clusters
// need not be co-resident with one another: a CTA waits only on its own
// cluster's barrier.
template <int T, bool GROUP>
__global__ void __launch_bounds__(T, 1024 / T) memo_cluster_build_kernel(
    const MemoJob *__restrict__ jobs, int njobs, int ncoop, unsigned *claim, int *status) {
    __shared__ uint64_t sums[33];
    __shared__ int32_t s_t[FZ_MAX_D];
    __shared__ int s_job;
    const unsigned nparts = cluster_size();
    const int cl = (int)(blockIdx.x / nparts);
    if (cl < ncoop) {
        const MemoJob J = jobs[cl];
        memo_coop_build_body(J, cluster_rank(), nparts, sums, status);
    }
    for (;;) {
        __syncthreads();  // s_job of the previous claim has been read
        if (threadIdx.x == 0) s_job = ncoop + (int)atomicAdd(claim, 1u);
        __syncthreads();
        const int j = s_job;
        if (j >= njobs) break;
        const MemoJob J = jobs[j];
        if (GROUP) memo_group_build_body(J, sums, s_t, status);
        else memo_cta_build_body<true>(J, sums, status);
    }
}

// ---------------------------------------------------------------------------
// The memo in run order (declared in fz_internal.cuh).  The element p of
// class c = p mod g_lam, q = p div g_lam, starts at
//   cls_beg[c] + sum_{p' = c mod g, p' < p} |Z(p', tail)|
//             = cls_beg[c] + C[lam][p] - C[lam+1][p]
// because the rows of a class up to p are exactly Z(p, (g_lam, tail)).
// ---------------------------------------------------------------------------
constexpr int RUN_CB_THREADS = 1024;

__global__ void __launch_bounds__(RUN_CB_THREADS) run_class_begin_kernel(
    const uint64_t *__restrict__ Clam, const uint64_t *__restrict__ O, int32_t n, int32_t g,
    int32_t G, uint64_t *__restrict__ cls_beg, int *status) {
    __shared__ uint64_t sums[33];
    uint64_t carry = 0;
    for (int base = 0; base < G; base += blockDim.x) {
        const int c = base + (int)threadIdx.x;
        uint64_t v = 0;
        if (c < G) {
            const int64_t last = c + (int64_t)((n - c) / g) * g;  // last element of class c
            v = __ldg(Clam + last);
        }
        uint64_t total;
        const uint64_t ex = block_exclusive_scan(v, sums, &total);
        if (c < G) cls_beg[c] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) {
        cls_beg[G] = carry;
        if (carry != __ldg(O + (int64_t)n + 1)) atomicExch(status, (int)DEV_INTERNAL);
    }
}

// One warp per element: its rows, with q = p div g_lam in front, to their
// place in run order.
__global__ void __launch_bounds__(THREADS) run_memo_kernel(
    const uint64_t *__restrict__ Clam, const uint64_t *__restrict__ Cnext,
    const uint64_t *__restrict__ O, const int32_t *__restrict__ rows, int k, int32_t n,
    int32_t g, const uint64_t *__restrict__ cls_beg, int4 *__restrict__ out, uint64_t out_rows,
    int *status) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t p = warp; p <= n; p += nwarps) {
        const int64_t q = p / g, c = p - q * g;
        const uint64_t o0 = __ldg(O + p), len = __ldg(O + p + 1) - o0;
        const uint64_t tail_rows = __ldg(Cnext + p);
        const uint64_t dst = __ldg(cls_beg + c) + __ldg(Clam + p) - tail_rows;
        if (len != tail_rows || dst + len > out_rows) {  // the tables must agree
            if (lane == 0) atomicExch(status, (int)DEV_INTERNAL);
            continue;
        }
        const int32_t *src = rows + o0 * (uint64_t)k;
        for (uint64_t r = lane; r < len; r += 32) {
            const int32_t *s = src + r * (uint64_t)k;
            int4 v;
            v.x = (int)q;
            v.y = k > 0 ? s[0] : 0;
            v.z = k > 1 ? s[1] : 0;
            v.w = k > 2 ? s[2] : 0;
            out[dst + r] = v;
        }
    }
}

// Batches: one CTA per run job for its class starts.  The total must be the
// memo's rows up to n (O[n + 1]), or the closed form's count.
__global__ void __launch_bounds__(RUN_CB_THREADS) run_class_begin_batch_kernel(
    const RunJob *__restrict__ jobs, int *status) {
    __shared__ uint64_t sums[33];
    const RunJob &J = jobs[blockIdx.x];
    const uint64_t *Clam = J.Clam;
    const int32_t n = J.n, g = J.g, G = J.G;
    uint64_t carry = 0;
    for (int base = 0; base < G; base += blockDim.x) {
        const int c = base + (int)threadIdx.x;
        uint64_t v = 0;
        if (c < G) {
            const int64_t last = c + (int64_t)((n - c) / g) * g;
            v = __ldg(Clam + last);
        }
        uint64_t total;
        const uint64_t ex = block_exclusive_scan(v, sums, &total);
        if (c < G) J.cls_beg[c] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) {
        J.cls_beg[G] = carry;
        const uint64_t want = J.O ? __ldg(J.O + (int64_t)n + 1) : J.expect_rows;
        if (carry != want || carry > J.out_rows) atomicExch(status, (int)DEV_INTERNAL);
    }
}

// Batches: a thread per element (these elements hold a few rows each), each
// job owning the blocks [blk0, blk0 + ceil((n + 1) / 256)) of the launch.
// Rows come from the element-order memo (O, rows), or from the closed form:
// k = 1, the one row p / ta when ta divides p; k = 2, the progression of the
// pair (t0, t1).
__device__ __forceinline__ uint32_t pair_first(const RunJob &J, int64_t r, int64_t *atop) {
    // rows of Z(r, (t0, t1)): a_{d-2} = atop, atop - h1, ..., >= 0 (none if
    // atop < 0); r, t0 and h1 fit in 32 bits
    *atop = -1;
    if (r < 0) return 0;
    const uint32_t ru = (uint32_t)r, e = (uint32_t)J.e, h1 = (uint32_t)J.h1;
    const uint32_t re = ru / e;
    if (re * e != ru) return 0;
    const uint32_t astar = (uint32_t)((uint64_t)(re % h1) * (uint64_t)J.inv % h1);
    const uint32_t q0 = ru / (uint32_t)J.t0;
    if (q0 < astar) return 0;
    const uint32_t top = q0 - (q0 - astar) % h1;
    *atop = top;
    return top / h1 + 1u;
}

// The job of block `blk` for a kernel whose jobs own the consecutive block
// ranges [blk0(j), blk0(j + 1)) (blk0 non-decreasing; jobs owning no block
// have equal starts): the last job whose range starts at or before blk.
template <class F>
__device__ __forceinline__ int job_of_block(int njobs, uint64_t blk, F blk0) {
    int lo = 0, hi = njobs;  // blk0(lo) <= blk < blk0(hi) (blk0(njobs) = total)
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (blk0(mid) <= blk)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

__global__ void __launch_bounds__(THREADS) run_rows_batch_kernel(const RunJob *__restrict__ jobs,
                                                                 int njobs, int *status) {
    __shared__ int s_job;
    if (threadIdx.x == 0)
        s_job = job_of_block(njobs, blockIdx.x, [&](int j) { return jobs[j].blk0; });
    __syncthreads();
    {
        const RunJob &J = jobs[s_job];
        const int64_t g = J.g;
        const int64_t p = (int64_t)(blockIdx.x - J.blk0) * blockDim.x + threadIdx.x;
        if (p <= J.n) {
            const int64_t q = p / g, c = p - q * g;
            const uint64_t tail_rows = __ldg(J.Cnext + p);
            const uint64_t dst = __ldg(J.cls_beg + c) + __ldg(J.Clam + p) - tail_rows;
            if (dst + tail_rows > J.out_rows) {
                atomicExch(status, (int)DEV_INTERNAL);
                return;
            }
            int4 *o = J.out + dst;
            if (J.O) {
                const uint64_t o0 = __ldg(J.O + p), len = __ldg(J.O + p + 1) - o0;
                if (len != tail_rows) {
                    atomicExch(status, (int)DEV_INTERNAL);
                    return;
                }
                const int k = J.k;
                const int32_t *s = J.rows + o0 * (uint64_t)k;
                // four rows' loads before their stores
                uint64_t r = 0;
                for (; r + 4 <= len; r += 4, s += 4 * k) {
                    int4 v[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        v[u] = make_int4((int)q, __ldg(s + u * k), k > 1 ? __ldg(s + u * k + 1) : 0,
                                         k > 2 ? __ldg(s + u * k + 2) : 0);
#pragma unroll
                    for (int u = 0; u < 4; ++u) o[r + u] = v[u];
                }
                for (; r < len; ++r, s += k)
                    o[r] = make_int4((int)q, __ldg(s), k > 1 ? __ldg(s + 1) : 0,
                                     k > 2 ? __ldg(s + 2) : 0);
            } else if (J.k == 1) {
                const uint64_t want = p % J.ta == 0 ? 1u : 0u;
                if (want != tail_rows) {
                    atomicExch(status, (int)DEV_INTERNAL);
                    return;
                }
                if (want) o[0] = make_int4((int)q, (int)(p / J.ta), 0, 0);
            } else {
                int64_t atop;
                const uint64_t want = pair_first(J, p, &atop);
                if (want != tail_rows) {
                    atomicExch(status, (int)DEV_INTERNAL);
                    return;
                }
                // a0 falls by h1 = t1 / e a row, so the last coordinate
                // (p - a0 t0) / t1 rises by t0 / e: one division an element
                if (want > 0) {
                    int64_t a0 = atop, b0 = (p - atop * J.t0) / J.t1;
                    const int64_t bstep = J.t0 / J.e;
                    for (uint64_t r = 0; r < want; ++r, a0 -= J.h1, b0 += bstep)
                        o[r] = make_int4((int)q, (int)a0, (int)b0, 0);
                }
            }
        }
    }
}

}  // namespace

int launch_run_memo_batch(const RunJob *jobs, int njobs, uint64_t blocks, int *status,
                          cudaStream_t s) {
    if (njobs <= 0) return FZ_OK;
    if (!jobs || !status) return set_error(FZ_EINTERNAL, "run memo batch: missing device buffer");
    run_class_begin_batch_kernel<<<njobs, RUN_CB_THREADS, 0, s>>>(jobs, status);
    note_launch();
    if (blocks > 0) {
        run_rows_batch_kernel<<<(unsigned)blocks, THREADS, 0, s>>>(jobs, njobs, status);
        note_launch();
    }
    FZ_CUDA_TRY(cudaGetLastError());
    return FZ_OK;
}

int launch_run_memo(const uint64_t *C, int64_t cs, int lam, int32_t n, int32_t g_lam,
                    const uint64_t *O, const int32_t *rows, int k, uint64_t memo_rows,
                    uint64_t *cls_beg, int4 *run_memo, int *status, cudaStream_t s) {
    if (k < 1 || k > 3 || g_lam < 1 || n < 0)
        return set_error(FZ_EINTERNAL, "run memo: unsupported shape");
    if (!C || !O || !rows || !cls_beg || !run_memo || !status)
        return set_error(FZ_EINTERNAL, "run memo: missing device buffer");
    const uint64_t *Clam = C + (int64_t)lam * cs;
    const uint64_t *Cnext = C + (int64_t)(lam + 1) * cs;
    const int32_t G = g_lam < n + 1 ? g_lam : n + 1;
    run_class_begin_kernel<<<1, RUN_CB_THREADS, 0, s>>>(Clam, O, n, g_lam, G, cls_beg, status);
    note_launch();
    int64_t blocks = ((int64_t)n + 1) * 32 / THREADS + 1;
    if (blocks > 4096) blocks = 4096;
    run_memo_kernel<<<(int)blocks, THREADS, 0, s>>>(Clam, Cnext, O, rows, k, n, g_lam, cls_beg,
                                                    run_memo, memo_rows, status);
    note_launch();
    FZ_CUDA_TRY(cudaGetLastError());
    return FZ_OK;
}

int launch_memo_sizes(const MemoJob *jobs, int njobs, uint64_t *rows_out, cudaStream_t s) {
    if (njobs <= 0) return FZ_OK;
    memo_sizes_kernel<<<njobs, MB_THREADS, 0, s>>>(jobs, rows_out);
    note_launch();
    FZ_CUDA_TRY(cudaGetLastError());
    return FZ_OK;
}

// Descriptor loads of the batch memo build: FZ_MEMO_DESC=serial loads each
// block's before its copy (tuning only).
static bool memo_desc_parallel() {
    static const bool on = [] {
        const char *e = getenv("FZ_MEMO_DESC");
        return !(e && strcmp(e, "serial") == 0);
    }();
    return on;
}

// CTA size of the batch memo build: FZ_MEMO_CTA_THREADS=256|512|1024
// (tuning only).
static int memo_cta_threads() {
    static const int t = [] {
        const char *e = getenv("FZ_MEMO_CTA_THREADS");
        const int v = e ? atoi(e) : 0;
        return (v == 256 || v == 512 || v == 1024) ? v : MB_CTA_THREADS_DEFAULT;
    }();
    return t;
}

// The one-CTA batch memo build: element groups (default) or
// FZ_MEMO_BUILD=element, one element per warp at a time (tuning only).
static bool memo_build_groups() {
    static const bool on = [] {
        const char *e = getenv("FZ_MEMO_BUILD");
        return !(e && strcmp(e, "element") == 0);
    }();
    return on;
}

// Cluster size of the cooperative batch memo build: FZ_MEMO_COOP=0 turns it
// off, 2|4|8 set the size (tuning only).
constexpr int MEMO_COOP_CL_DEFAULT = 2;
static int memo_coop_cluster() {
    static const int c = [] {
        const char *e = getenv("FZ_MEMO_COOP");
        if (!e) return MEMO_COOP_CL_DEFAULT;
        const int v = atoi(e);
        return (v == 0 || v == 2 || v == 4 || v == 8) ? v : MEMO_COOP_CL_DEFAULT;
    }();
    return c;
}

static cudaLaunchConfig_t coop_config(int grid, int csize, cudaLaunchAttribute *attr,
                                      cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(MB_CTA_THREADS_DEFAULT);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = csize;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

// Clusters of the cooperative build that fit on the device at once (0 if
// the shape does not fit).
static int coop_resident_clusters(int csize) {
    static DeviceOnce done[3];
    static int cached[3][64];
    const int slot = csize == 2 ? 0 : csize == 4 ? 1 : 2;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    if (!done[slot].is_set(dev)) {
        cudaLaunchAttribute attr[1];
        cudaLaunchConfig_t cfg = coop_config(csize, csize, attr, 0);
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(
                &n, memo_cluster_build_kernel<MB_CTA_THREADS_DEFAULT, true>, &cfg) !=
            cudaSuccess) {
            cudaGetLastError();
            n = 0;
        }
        cached[slot][dev] = n;
        done[slot].set(dev);
    }
    return cached[slot][dev];
}

// The build takes as long as its longest memo when that memo alone outlasts
// an even share of all the work: a one-CTA memo costs about its words plus
// MEMO_BATCH_WORDS per elementwise batch (the dependent round trips and the
// barrier).  Jobs sorted longest first; every job above the even share over
// the device's CTA slots is built by a cluster, at most half the clusters
// that fit at once.
constexpr double MEMO_BATCH_WORDS = 16000.0;

int memo_coop_count(const MemoJob *sorted, int njobs) {
    const int csize = memo_coop_cluster();
    if (csize == 0 || njobs < 2) return 0;
    const int clusters = coop_resident_clusters(csize);
    if (clusters < 2) return 0;
    const double slots = (double)clusters * csize;
    std::vector<double> w((size_t)njobs);
    double sum = 0;
    for (int j = 0; j < njobs; ++j) {
        const MemoJob &J = sorted[j];
        const double nbatch = ((double)J.top + J.b - 1) / (double)J.b;
        w[(size_t)j] = (double)J.rows * J.k + MEMO_BATCH_WORDS * nbatch;
        sum += w[(size_t)j];
    }
    const double share = sum / slots;
    int n = 0;
    while (n < njobs && n < clusters / 2 && w[(size_t)n] > share) ++n;
    return n;
}

int launch_memo_cta_build(const MemoJob *jobs, int njobs, int ncoop, unsigned *claim,
                          int *status, cudaStream_t s) {
    if (njobs <= 0) return FZ_OK;
    const int csize = memo_coop_cluster();
    if (ncoop > 0 && csize > 0) {
        const int clusters = coop_resident_clusters(csize);
        if (ncoop > clusters) return set_error(FZ_EINTERNAL, "memo build: too many clusters");
        // enough CTAs for every slot, none beyond the jobs they can take
        int grid_cl = clusters;
        const int need = ncoop + (njobs - ncoop + csize - 1) / csize;
        if (grid_cl > need) grid_cl = need;
        FZ_CUDA_TRY(cudaMemsetAsync(claim, 0, sizeof(unsigned), s));
        cudaLaunchAttribute attr[1];
        cudaLaunchConfig_t cfg = coop_config(grid_cl * csize, csize, attr, s);
        cudaError_t e =
            memo_build_groups()
                ? cudaLaunchKernelEx(&cfg, memo_cluster_build_kernel<MB_CTA_THREADS_DEFAULT, true>,
                                     jobs, njobs, ncoop, claim, status)
                : cudaLaunchKernelEx(&cfg, memo_cluster_build_kernel<MB_CTA_THREADS_DEFAULT, false>,
                                     jobs, njobs, ncoop, claim, status);
        if (e != cudaSuccess) return cuda_error(e, "memo build (cluster) launch");
        note_launch();
        return FZ_OK;
    }
    if (memo_build_groups()) {
        memo_group_cta_kernel<MB_CTA_THREADS_DEFAULT>
            <<<njobs, MB_CTA_THREADS_DEFAULT, 0, s>>>(jobs, status);
        note_launch();
        FZ_CUDA_TRY(cudaGetLastError());
        return FZ_OK;
    }
    const bool par = memo_desc_parallel();
    switch (memo_cta_threads()) {
        case 256:
            if (par) memo_cta_build_kernel<256, true><<<njobs, 256, 0, s>>>(jobs, status);
            else memo_cta_build_kernel<256, false><<<njobs, 256, 0, s>>>(jobs, status);
            break;
        case 1024:
            if (par) memo_cta_build_kernel<1024, true><<<njobs, 1024, 0, s>>>(jobs, status);
            else memo_cta_build_kernel<1024, false><<<njobs, 1024, 0, s>>>(jobs, status);
            break;
        default:
            if (par) memo_cta_build_kernel<512, true><<<njobs, 512, 0, s>>>(jobs, status);
            else memo_cta_build_kernel<512, false><<<njobs, 512, 0, s>>>(jobs, status);
            break;
    }
    note_launch();
    FZ_CUDA_TRY(cudaGetLastError());
    return FZ_OK;
}

// Factorizationwise schedule: the host walks m and i in the algorithm's
// order with the saved cardinalities (copied to the host once) and launches
// one copy per non-empty block.
static int launch_memo_per_copy(const int32_t *tail, int k, int32_t top, uint64_t rows,
                                const MemoBuffers &mb, cudaStream_t s) {
    std::vector<uint64_t> O((size_t)top + 1), Ct((size_t)k * (size_t)mb.cs);
    FZ_CUDA_TRY(cudaMemcpyAsync(O.data(), mb.O, O.size() * 8, cudaMemcpyDeviceToHost, s));
    FZ_CUDA_TRY(cudaMemcpyAsync(Ct.data(), mb.Ct, Ct.size() * 8, cudaMemcpyDeviceToHost, s));
    FZ_CUDA_TRY(cudaStreamSynchronize(s));
    if (O[top] != rows) return set_error(FZ_EINTERNAL, "memo build: offsets disagree");
    DeviceProps dp;
    int rc = device_props(&dp);
    if (rc != FZ_OK) return rc;
    zero_row_kernel<<<1, 32, 0, s>>>(mb.rows, k);  // Z(0) = [0]
    note_launch();
    for (int64_t m = 1; m < top; ++m) {
        uint64_t dst = O[m];
        for (int i = 0; i < k; ++i) {
            const int64_t sm = m - (int64_t)tail[i];
            if (sm < 0) continue;
            const uint64_t len = Ct[(size_t)i * mb.cs + sm];
            if (len == 0) continue;
            const uint64_t src = O[sm + 1] - len;  // Z_{>=i}(m - t_i): the last len rows
            if (dst + len > O[m + 1]) return set_error(FZ_EINTERNAL, "memo build: block overflow");
            uint64_t blocks = (len * (uint64_t)k + THREADS - 1) / THREADS;
            if (blocks > (uint64_t)dp.sms * 8) blocks = (uint64_t)dp.sms * 8;
            copy_and_increment_kernel<<<(unsigned)blocks, THREADS, 0, s>>>(mb.rows, k, dst, src,
                                                                          len, i);
            note_launch();
            dst += len;
        }
        if (dst != O[m + 1]) return set_error(FZ_EINTERNAL, "memo build: blocks do not tile");
    }
    FZ_CUDA_TRY(cudaGetLastError());
    return FZ_OK;
}

int launch_memo_build(const int32_t *tail, int k, int32_t top, uint64_t rows,
                      const MemoBuffers &mb, cudaStream_t s, int schedule) {
    if (top <= 0 || rows == 0) return FZ_OK;
    if (schedule == FZ_MEMO_PER_COPY) {
        if (!mb.Ct || !mb.O || !mb.rows) return set_error(FZ_EINTERNAL, "memo build: missing device buffer");
        return launch_memo_per_copy(tail, k, top, rows, mb, s);
    }
    if (!mb.Ct || !mb.O || !mb.map || !mb.rows || !mb.status || !mb.bar)
        return set_error(FZ_EINTERNAL, "memo build: missing device buffer");
    MapParams mp{};
    mp.Ct = mb.Ct;
    mp.cs = mb.cs;
    mp.O = mb.O;
    mp.map = mb.map;
    mp.status = mb.status;
    mp.top = top;
    mp.k = k;
    int tmin = tail[0];
    for (int i = 0; i < k; ++i) {
        mp.t[i] = tail[i];
        if (tail[i] < tmin) tmin = tail[i];
    }
    FillParams fp{};
    fp.O = mb.O;
    fp.map = mb.map;
    fp.rows = mb.rows;
    fp.status = mb.status;
    fp.bar = mb.bar;
    fp.top = top;
    fp.k = k;
    fp.b = tmin;
    fp.nbatch = (int)(((int64_t)top + tmin - 1) / tmin);
    // FZ_MEMO_FILL=cta|cluster|grid|phase forces one fill (tuning only)
    static const int forced = [] {
        const char *e = getenv("FZ_MEMO_FILL");
        if (!e) return 0;
        if (!strcmp(e, "cta")) return 1;
        if (!strcmp(e, "cluster")) return 2;
        if (!strcmp(e, "grid")) return 3;
        if (!strcmp(e, "phase")) return 4;
        return 0;
    }();
    // phases of L elements when block 0's generator is the tail's first and
    // every other generator is at least twice it (a phase spans >= 2 batches)
    {
        int L = top;
        for (int i = 1; i < k; ++i) L = tail[i] < L ? tail[i] : L;
        const bool fits32 = (double)tail[0] * (double)(rows + 32) * k < 2147483648.0;
        fp.L = (tail[0] == tmin && L >= 2 * tail[0] && fits32) ? L : 0;
    }
    // the gather map: every memo row's source row and incremented coordinate
    auto launch_map = [&](int skip0) -> int {
        mp.skip0 = skip0;
        int64_t warps = top;
        int64_t blocks = (warps * 32 + THREADS - 1) / THREADS;
        if (blocks > 4096) blocks = 4096;
        memo_map_kernel<<<(int)blocks, THREADS, 0, s>>>(mp);
        note_launch();
        FZ_CUDA_TRY(cudaGetLastError());
        return FZ_OK;
    };
    if (schedule == FZ_MEMO_PER_BATCH) {
        DeviceProps dp;
        int rc = device_props(&dp);
        if (rc != FZ_OK) return rc;
        rc = launch_map(0);
        if (rc != FZ_OK) return rc;
        for (int q = 0; q < fp.nbatch; ++q) {
            memo_batch_kernel<<<dp.sms * 4, THREADS, 0, s>>>(fp, q);
            note_launch();
        }
        FZ_CUDA_TRY(cudaGetLastError());
        return FZ_OK;
    }
    const uint64_t avg_batch_rows = rows / (uint64_t)fp.nbatch;
    // a few rows per batch: one CTA (its barrier and L1 beat a cluster's);
    // batches of modest size: one cluster; else the whole GPU, in phases
    // when the tail allows them (then block 0 needs no map entries)
    const bool one_cta =
        (forced == 0 && avg_batch_rows * (uint64_t)k <= ONE_CTA_MAX_WORDS) || forced == 1;
    const bool cluster = !one_cta &&
                         ((forced == 0 && avg_batch_rows <= (uint64_t)64 * 1024) || forced == 2);
    const bool phase = !one_cta && !cluster && fp.L > 0 && forced != 3;
    {
        int rc = launch_map(phase ? 1 : 0);
        if (rc != FZ_OK) return rc;
    }
    if (one_cta) return launch_fill_one_cta(fp, s);
    if (cluster) {
        int rc = launch_fill_cluster(fp, mb.small_ctas, s);
        if (rc == FZ_OK) return rc;
    }
    const void *kern = phase ? (const void *)memo_fill_phase_kernel : (const void *)memo_fill_kernel;
    int grid = coop_grid(kern, GRID_THREADS);
    if (grid <= 0) return set_error(FZ_ECUDA, "memo build: no cooperative occupancy");
    FZ_CUDA_TRY(cudaMemsetAsync(mb.bar, 0, sizeof(unsigned), s));
    void *args[] = {&fp};
    FZ_CUDA_TRY(cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(GRID_THREADS), args, 0, s));
    note_launch();
    return FZ_OK;
}

}  // namespace fz
