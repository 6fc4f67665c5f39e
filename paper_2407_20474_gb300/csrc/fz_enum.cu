// fz_enum.cu -- lexicographic enumeration of Z(n, g) with low-dimension
// tabulation (Section 3.1), sliced by exact ranks.
//
// The output list (descending lexicographic order) is the depth-first walk of
// the tree whose depth-c nodes are prefixes (a_0..a_{c-1}) with remainder
// rem = n - phi(prefix) >= 0; the children of a node are a_c = floor(rem/g_c)
// down to 0 (the order in which the next-candidate step of Algorithm 3.1
// visits them).  The subtree of the child a_c = v holds C[c+1][rem - v g_c]
// rows, and the rows of all children with a_c >= v number C[c][rem - v g_c]
// (count table, fz_count.cu), so any rank is located by searching one table
// row per level.
//
// Leaves ("blocks"), as in the dynamic next-candidate step:
//  * memo leaf: a prefix of length L = d - K whose remainder p is < top;
//    its rows are Memo[p] = Z(p, (g_L..g_{d-1})) with the prefix prepended
//    (the block copy of Section 3.1; the walk then continues from
//    (prefix, 0, ..., 0), the observation of Section 3.1);
//  * walk leaf: a prefix of length d - 1 (reached when no memo applies);
//    its one row, if g_{d-1} divides p, is the candidate of Algorithm 3.1's
//    ordinary step with a_d = p / g_d.
//
// Work split: each warp takes slices of S consecutive ranks (an atomic
// counter hands them out), finds the leaf holding its first rank by table
// search (this replaces the paper's splitWork with exact bounds), and walks
// from there.  A run of sibling leaves is processed 32 at a time: every lane
// evaluates one candidate, the table gives each lane its cumulative row end
// directly, and lanes then fill rows: each lane finds the leaf of its row by
// a 5-step shuffle search.  Rows are assembled in a per-warp shared-memory
// ring of two halves and each full half is written to HBM with one bulk
// (TMA) store, so the stream is written with 16-byte aligned, fully
// coalesced transactions while the warp generates the next half.
#include <cstring>

#include <cstdlib>

#include "fz_internal.cuh"

namespace fz {

constexpr int ENUM_WARPS = 8;
constexpr int ENUM_THREADS = ENUM_WARPS * 32;
constexpr int RING_BYTES_PER_WARP = 6 * 1024;  // two halves; 4 CTAs of 8 warps per SM
constexpr uint32_t CAP32 = 0xffffffffu;

// Division and remainder of a 32-bit value by a fixed divisor via one
// precomputed 64-bit multiplier (Lemire, Kaser and Kurz, "Faster remainder by
// direct computation", 2019): M = floor((2^64 - 1) / g) + 1, a / g =
// hi64(M * a), a % g = hi64(lo64(M * a) * g), exact for all a, g < 2^32, g > 1.
struct FastDiv {
    uint64_t M;
    uint32_t g;
};
__host__ __device__ inline FastDiv make_fastdiv(uint32_t g) {
    FastDiv f;
    f.g = g;
    f.M = g > 1 ? ~0ull / g + 1 : 0ull;
    return f;
}
__device__ __forceinline__ uint32_t fd_div(uint32_t a, FastDiv f) {
    return f.g > 1 ? (uint32_t)__umul64hi(f.M, a) : a;
}

struct EnumParams {
    const uint64_t *C;     // count table rows 0..d, stride cs
    int64_t cs;
    const uint64_t *O;     // memo CSR offsets (top + 1), or null
    const int32_t *memo;   // memo rows, K int32 each, or null
    uint64_t memo_rows;    // rows in memo (bounds guard)
    int32_t *out;          // row 0 = rank rank_begin
    int *status;
    unsigned long long *slice_counter;
    uint64_t rank_begin;   // absolute rank of out row 0
    uint64_t nrows;        // rows to write
    uint64_t slice_rows;   // S (multiple of 4), used when RT is null
    uint64_t nslices;
    const uint64_t *RT;    // candidates table rows 0..lam_r (stride cs), or null
    uint64_t W;            // cost of one unit of walk work (a prefix of length lam_r), in rows
    uint64_t slice_cost;   // cost units per work item when RT is set
    int lam_r;             // one past the leaf coordinate (RT[lam_r] = 1)
    int n, d, K, top;
    int lam_m;             // coordinate whose children are memo leaves (d-K-1), or -1
    int lam_w;             // coordinate whose children are walk leaves (d-2)
    int half_rows;         // B: rows per ring half (multiple of 32)
    int aligned;           // out is 16-byte aligned
    int ctas_per_sm;       // occupancy cap of the launch (0 = none)
    int dense_min;         // memo batches with >= dense_min rows per leaf go leaf by leaf
    const int4 *run_memo;  // full memo in run order (k <= 3), or null
    const uint64_t *cls_beg;
    int g[FZ_MAX_D];
    FastDiv glast;         // division by g_{d-1} (walk leaves)
    // Walk leaves as a progression: with e = gcd(g_{d-2}, g_{d-1}), the
    // candidates a_{d-2} = v of remainder r with g_{d-1} | r - v g_{d-2} are
    // v = v* (mod h1), h1 = g_{d-1}/e, v* = (r/e) inv (mod h1), inv the inverse
    // of g1 = g_{d-2}/e mod h1 (0 when h1 = 1); e must divide r.  Along the
    // progression a_{d-1} grows by g1.  wl_h1 = 0: candidate by candidate.
    int wl_e, wl_h1, wl_g1, wl_inv;
    // Pair memo: a full memo of depth 2 kept as a formula, no table.  Memo
    // leaf p (remainder at depth d-2) holds Z(p, (g_{d-2}, g_{d-1})): row o
    // is a_{d-2} = a_top - o h1, a_{d-1} = (p - a_{d-2} g_{d-2}) / g_{d-1},
    // with a_top the largest valid a_{d-2} (the progression above).
    int pair_memo;
    FastDiv fd_e, fd_h1, fd_g2;  // division by e, h1 and g_{d-2}
};

__device__ __forceinline__ uint32_t fd_mod(uint32_t a, FastDiv f) {
    return a - fd_div(a, f) * f.g;
}

// First a_{d-2} of pair-memo leaf p (meaningful when the leaf is not empty):
// 32-bit divisions by precomputed multipliers; the product (p/e mod h1) inv
// fits 32 bits when h1 < 2^16, else it takes a 64-bit remainder.
__device__ __forceinline__ uint32_t pair_top(const EnumParams &P, int p) {
    const uint32_t up = (uint32_t)p;
    const uint32_t h1 = (uint32_t)P.wl_h1;
    const uint32_t xr = fd_mod(fd_div(up, P.fd_e), P.fd_h1);
    const uint32_t astar = h1 < 65536u
                               ? fd_mod(xr * (uint32_t)P.wl_inv, P.fd_h1)
                               : (uint32_t)((uint64_t)xr * (uint32_t)P.wl_inv % h1);
    const uint32_t q = fd_div(up, P.fd_g2);
    return q >= astar ? q - fd_mod(q - astar, P.fd_h1) : 0u;
}

struct WarpPath {
    int a[FZ_MAX_D];      // a_0..a_{lam-1}
    int r[FZ_MAX_D + 1];  // r[0] = n, r[c+1] = r[c] - a[c] g[c]
};

enum LeafType : int { T_NONE = 0, T_MEMO = 1, T_WALK = 2, T_INTERNAL = 3 };

// Largest u in [0, umax] with F(u) <= R, F(u) = C[c][rem - (umax + 1 - u) g_c]
// (rows in the children with a_c > umax - u), searched 32 probes at a time.
// Returns the child a_c = umax - u holding relative rank R and the rows
// before it.  Requires R < C[c][rem].
__device__ __forceinline__ void find_child(const EnumParams &P, int c, int rem, uint64_t R,
                                           int lane, int &v_out, uint64_t &before_out) {
    const long long g = P.g[c];
    const long long umax = rem / g;
    const long long base = (long long)rem - (umax + 1) * g;
    const uint64_t *row = P.C + (long long)c * P.cs;
    long long lo = 0, hi = umax + 1;
    uint64_t flo = 0;
    while (hi - lo > 1) {
        const long long step = (hi - lo + 31) >> 5;
        const long long u = lo + (long long)(lane + 1) * step;
        bool ok = false;
        uint64_t fu = 0;
        if (u < hi) {
            const long long idx = base + u * g;
            fu = idx >= 0 ? __ldg(row + idx) : 0ull;
            ok = fu <= R;
        }
        const unsigned m = __ballot_sync(FULL, ok);
        const int cnt = __popc(m);
        const uint64_t fsel = shfl_u64(fu, cnt > 0 ? cnt - 1 : 0);
        if (cnt > 0) {
            flo = fsel;
            lo += (long long)cnt * step;
        }
        const long long nh = lo + step;
        if (nh < hi) hi = nh;
    }
    v_out = (int)(umax - lo);
    before_out = flo;
}

// Walk state of one warp (warp-uniform).
struct RunState {
    int lam;          // coordinate of the current run of sibling leaves
    int inwalk;       // inside the subtree of a memo-level child with p >= top
    long long vcur;   // next candidate value of a_lam (descending)
    uint64_t base;    // rows in the siblings before vcur
};

// Choose the first live child at depths c_from..c_to-1 (path stored by lane 0).
__device__ __forceinline__ void descend(const EnumParams &P, WarpPath *wp, int c_from,
                                        int c_to, int lane) {
    int rem = wp->r[c_from];
    for (int c = c_from; c < c_to; ++c) {
        int v = rem / P.g[c];
        // usually the largest child is live (one load); else search
        if (__ldg(P.C + (long long)(c + 1) * P.cs + (rem - v * P.g[c])) == 0ull) {
            uint64_t before;
            find_child(P, c, rem, 0ull, lane, v, before);
        }
        rem -= v * P.g[c];
        if (lane == 0) {
            wp->a[c] = v;
            wp->r[c + 1] = rem;
        }
    }
    __syncwarp();
}

// Position the warp on the leaf holding absolute rank R.  Returns the offset
// of R inside that leaf.  Sets *ok = false if the table is inconsistent.
__device__ uint64_t unrank_to_leaf(const EnumParams &P, WarpPath *wp, uint64_t R, int lane,
                                   RunState &st, bool *ok) {
    int rem = P.n;
    if (lane == 0) wp->r[0] = rem;
    int inwalk = 0;
    const bool memo = P.lam_m >= 0;
    *ok = true;
    for (int c = 0; c < P.d; ++c) {
        const int runlev = (memo && !inwalk) ? P.lam_m : P.lam_w;
        const uint64_t total = __ldg(P.C + (long long)c * P.cs + rem);
        if (R >= total) {
            *ok = false;
            break;
        }
        int v;
        uint64_t before;
        find_child(P, c, rem, R, lane, v, before);
        R -= before;
        const int p = rem - v * P.g[c];
        if (c == runlev) {
            if (memo && !inwalk && p >= P.top && P.lam_m < P.lam_w) {
                // memo-level child beyond the memo: walk its subtree
                if (lane == 0) {
                    wp->a[c] = v;
                    wp->r[c + 1] = p;
                }
                rem = p;
                inwalk = 1;
                continue;
            }
            st.lam = c;
            st.inwalk = inwalk;
            st.vcur = v;
            st.base = before;
            __syncwarp();
            return R;
        }
        if (lane == 0) {
            wp->a[c] = v;
            wp->r[c + 1] = p;
        }
        rem = p;
    }
    __syncwarp();
    *ok = false;
    return 0;
}

// Move to the next run after the current one is exhausted.  Returns false at
// the end of the stream.
__device__ bool advance(const EnumParams &P, WarpPath *wp, int lane, RunState &st) {
    const bool memo = P.lam_m >= 0;
    for (int j = st.lam - 1; j >= 0; --j) {
        const int rem = wp->r[j];
        const int aj = wp->a[j];
        const uint64_t *row = P.C + (long long)j * P.cs;
        const uint64_t R = __ldg(row + (rem - aj * P.g[j]));  // rows in children >= aj
        const uint64_t total = __ldg(row + rem);
        if (R >= total) continue;
        // usually the next smaller value is live (one load); else search
        int v = aj - 1;
        if (__ldg(P.C + (long long)(j + 1) * P.cs + (rem - v * P.g[j])) == 0ull) {
            uint64_t before;
            find_child(P, j, rem, R, lane, v, before);
        }
        const int p = rem - v * P.g[j];
        if (lane == 0) {
            wp->a[j] = v;
            wp->r[j + 1] = p;
        }
        __syncwarp();
        int nw;
        if (memo && j < P.lam_m)
            nw = 0;
        else if (memo)
            nw = 1;  // at or below the memo level: inside a walked subtree
        else
            nw = 0;
        const int newlam = (memo && !nw) ? P.lam_m : P.lam_w;
        descend(P, wp, j + 1, newlam, lane);
        st.lam = newlam;
        st.inwalk = nw;
        st.vcur = wp->r[newlam] / P.g[newlam];
        st.base = 0;
        return true;
    }
    return false;
}

// ---------------------------------------------------------------------------
// Work-balanced slicing.  The cost of a subtree is its rows plus W for every
// unit of walk work in it -- a leaf candidate, a walk run or a run-order run,
// i.e. a prefix of length lam_r the walk evaluates, live or not (balance_level
// picks lam_r and W); RT[j][x] counts those prefixes (RT[lam_r] = 1, and row j
// is row j+1 strided-summed with stride g_j, like the count table; a memo
// leaf above level lam_r is clamped to one unit), so the cost of the
// children a_j >= v of a node is
// C[j][x] + W RT[j][x] with x = rem - v g_j.  Work items are equal cost ranges, located by the same
// 32-probe search as ranks, then snapped to ranks that are multiples of 32
// from rank_begin: 32 rows are 128 d bytes, so every bulk store of a slice
// starts on a 128-byte line when the output is 128-byte aligned.
// ---------------------------------------------------------------------------
// A memo leaf above the counted level (a partial memo of depth K > 2 whose
// runs table counts walk runs): the node at depth j is one unit of cost.
__device__ __forceinline__ bool is_memo_unit(const EnumParams &P, int j, int rem) {
    return P.lam_m >= 0 && j == P.lam_m + 1 && j < P.lam_r && rem < P.top;
}

__device__ __forceinline__ uint64_t cost_at(const EnumParams &P, int j, long long idx) {
    if (idx < 0) return 0ull;
    return __ldg(P.C + (long long)j * P.cs + idx) + P.W * __ldg(P.RT + (long long)j * P.cs + idx);
}

// Rank of the first row whose cumulative cost reaches `target` (clamped to
// the total row count).
__device__ uint64_t cost_to_rank(const EnumParams &P, uint64_t target, int lane) {
    int rem = P.n;
    uint64_t rank = 0;
    if (target >= cost_at(P, 0, rem)) return __ldg(P.C + rem);
    int lev = P.lam_r;
    for (int j = 0; j < P.lam_r; ++j) {
        if (is_memo_unit(P, j, rem)) {
            lev = j;
            break;
        }
        const long long g = P.g[j];
        const long long umax = rem / g;
        const long long base = (long long)rem - (umax + 1) * g;
        long long lo = 0, hi = umax + 1;
        uint64_t flo = 0;
        while (hi - lo > 1) {
            const long long step = (hi - lo + 31) >> 5;
            const long long u = lo + (long long)(lane + 1) * step;
            bool ok = false;
            uint64_t fu = 0;
            if (u < hi) {
                fu = cost_at(P, j, base + u * g);
                ok = fu <= target;
            }
            const int cnt = __popc(__ballot_sync(FULL, ok));
            const uint64_t fsel = shfl_u64(fu, cnt > 0 ? cnt - 1 : 0);
            if (cnt > 0) {
                flo = fsel;
                lo += (long long)cnt * step;
            }
            const long long nh = lo + step;
            if (nh < hi) hi = nh;
        }
        const long long idx = base + lo * g;
        rank += idx >= 0 ? __ldg(P.C + (long long)j * P.cs + idx) : 0ull;
        target -= flo;
        rem = (int)(rem - (umax - lo) * g);
    }
    const uint64_t rows = __ldg(P.C + (long long)lev * P.cs + rem);
    const uint64_t t = target > P.W ? target - P.W : 0ull;
    return rank + (t < rows ? t : rows);
}

// Cumulative cost of everything before rank R.
__device__ uint64_t rank_to_cost(const EnumParams &P, uint64_t R, int lane) {
    int rem = P.n;
    if (R >= __ldg(P.C + rem)) return cost_at(P, 0, rem);
    uint64_t cost = 0;
    for (int j = 0; j < P.lam_r; ++j) {
        if (is_memo_unit(P, j, rem)) break;
        int v;
        uint64_t before;
        find_child(P, j, rem, R, lane, v, before);
        cost += before + P.W * (rem - (long long)(v + 1) * P.g[j] >= 0
                                    ? __ldg(P.RT + (long long)j * P.cs +
                                            (rem - (long long)(v + 1) * P.g[j]))
                                    : 0ull);
        R -= before;
        rem -= v * P.g[j];
    }
    return cost + P.W + R;
}

// Rows [row0, row1) (relative to out) of work item s.  With a candidates
// table the items are cost ranges of [cost_lo, cost_hi) snapped to multiples
// of 32 rows: the first four fifths of the cost in items of slice_cost, the
// rest in items of an eighth of that, so the warps that take the last items
// finish close together.  Otherwise equal-row ranges.  Returns 0 when s is
// past the last item, 1 when the item is empty, 2 otherwise.
__device__ __forceinline__ int item_rows(const EnumParams &P, uint64_t s, uint64_t cost_lo,
                                         uint64_t cost_hi, int lane, uint64_t &row0,
                                         uint64_t &row1) {
    if (P.RT) {
        const uint64_t sc = P.slice_cost;
        const uint64_t n1 = (cost_hi - cost_lo) / sc * 4 / 5;  // large items
        const uint64_t sc_t = sc / 8 > 64 ? sc / 8 : 64;
        uint64_t c0, c1;
        if (s < n1) {
            c0 = cost_lo + s * sc;
            c1 = c0 + sc;
        } else {
            const uint64_t t = s - n1;
            const uint64_t base = cost_lo + n1 * sc;
            if (t >= (cost_hi - base + sc_t - 1) / sc_t) return 0;
            c0 = base + t * sc_t;
            c1 = c0 + sc_t;
        }
        if (c0 >= cost_hi) return 0;
        row0 = 0;
        if (s > 0) {
            const uint64_t r = cost_to_rank(P, c0, lane);
            row0 = r > P.rank_begin ? ((r - P.rank_begin) & ~31ull) : 0ull;
            if (row0 > P.nrows) row0 = P.nrows;
        }
        row1 = P.nrows;
        if (c1 < cost_hi) {
            const uint64_t r = cost_to_rank(P, c1, lane);
            row1 = r > P.rank_begin ? ((r - P.rank_begin) & ~31ull) : 0ull;
            if (row1 > P.nrows) row1 = P.nrows;
        }
        return row1 > row0 ? 2 : 1;
    }
    if (s >= P.nslices) return 0;
    row0 = s * P.slice_rows;
    row1 = row0 + P.slice_rows < P.nrows ? row0 + P.slice_rows : P.nrows;
    return 2;
}

__device__ __forceinline__ void flush_rows(const EnumParams &P, const int32_t *src,
                                           uint64_t out_row, uint32_t nrows, int d, int lane,
                                           uint64_t pol) {
    int32_t *gdst = P.out + out_row * (uint64_t)d;
    const uint32_t words = nrows * (uint32_t)d;
    if (P.aligned) {
        const uint32_t bytes = words * 4u;
        const uint32_t bulk = bytes & ~15u;
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0 && bulk) {
            bulk_store(gdst, src, bulk, pol);
            bulk_commit();
        }
        const uint32_t rem_words = (bytes - bulk) >> 2;
        if ((uint32_t)lane < rem_words) gdst[(bulk >> 2) + lane] = src[(bulk >> 2) + lane];
    } else {
        // plain stores (unaligned output, or host memory over the host link):
        // 16-byte vectors when both sides allow it
        __syncwarp();
        uint32_t w0 = 0;
        if ((((uintptr_t)gdst | (uintptr_t)src) & 15u) == 0) {
            const uint32_t nv = words >> 2;
            const int4 *s4 = reinterpret_cast<const int4 *>(src);
            int4 *g4 = reinterpret_cast<int4 *>(gdst);
            for (uint32_t v = lane; v < nv; v += 32) g4[v] = s4[v];
            w0 = nv << 2;
        }
        for (uint32_t w = w0 + lane; w < words; w += 32) gdst[w] = src[w];
        __syncwarp();
    }
}

// 4-byte global -> shared copy that does not hold a register (cp.async).
// No memory clobber: the source (memo) is read-only, the destination word is
// touched by nothing else until cp.async.wait_group (which has the clobber),
// and volatile keeps issue order with the commit and the wait.
__device__ __forceinline__ void cp_async4(int32_t *sdst, const int32_t *gsrc) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(sdst)), "l"(gsrc));
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Rounds a completed ring half waits before its bulk store, so that the
// cp.async copies of its last rows have landed without stalling the warp.
constexpr int FLUSH_LAG = 2;

// One work item: rows [row0, row1) of the output (relative to P.out),
// produced by unranking row0 and walking from there.  D > 0: tuple width known
// at compile time; D == 0: width P.d (at most FZ_MAX_D).  LAMF >= 0: every run
// is a memo run at coordinate LAMF (full memo, k = D-1-LAMF) fixed at compile
// time; LAMF < 0: generic (runtime run level, walk leaves).  Returns false if
// a device-side consistency check failed (status already recorded).  DMAX:
// with D == 0, the largest width the call serves (shorter row loops and
// prefix arrays for narrow tuples).
template <int D, int LAMF, int DMAX = FZ_MAX_D>
__device__ __forceinline__ bool enum_slice(const EnumParams &P, WarpPath *wp, int32_t *ring,
                                           uint32_t B, uint64_t row0, uint64_t row1,
                                           uint64_t pol, int lane) {
    constexpr int DM = D > 0 ? D : DMAX;
    const int d = D > 0 ? D : P.d;
    constexpr int KF = LAMF >= 0 ? D - 1 - LAMF : 0;
    uint32_t rows_left = (uint32_t)(row1 - row0);

    RunState st;
    bool ok;
    uint64_t skip = unrank_to_leaf(P, wp, P.rank_begin + row0, lane, st, &ok);
    if (!ok) {
        if (lane == 0) atomicExch(P.status, (int)DEV_INTERNAL);
        return false;
    }

    // ring: rows go to half `half` at position hpos; `nfull` halves of
    // this slice are complete; a completed half is flushed FLUSH_LAG
    // rounds later (pend_rounds counts them).
    uint32_t hpos = 0, half = 0, nfull = 0, pend_rounds = 0;
    bool pend = false;

    int pre[DM];
#pragma unroll
    for (int c = 0; c < DM; ++c) pre[c] = (c < st.lam) ? wp->a[c] : 0;

    // ring bookkeeping after a round of cnt rows (both paths)
    auto after_round = [&](uint32_t cnt) {
        cp_async_commit();
        hpos += cnt;
        if (pend && ++pend_rounds >= (uint32_t)FLUSH_LAG) {
            cp_async_wait<FLUSH_LAG>();
            flush_rows(P, ring + (size_t)(half ^ 1u) * B * d,
                          row0 + (uint64_t)(nfull - 1) * B, B, d, lane, pol);
            pend = false;
        }
        if (hpos == B) {
            if (pend) {  // (only if a half holds fewer than FLUSH_LAG rounds)
                cp_async_wait<0>();
                flush_rows(P, ring + (size_t)(half ^ 1u) * B * d,
                              row0 + (uint64_t)(nfull - 1) * B, B, d, lane, pol);
            }
            pend = true;
            pend_rounds = 0;
            ++nfull;
            half ^= 1u;
            hpos = 0;
        }
    };
    auto before_round = [&]() {
        if (hpos == 0 && nfull >= 2) {
            // re-entering a half: its bulk store (the most recent bulk
            // group) must have finished reading it
            if (lane == 0) bulk_wait_read_all();
            __syncwarp();
        }
    };
    while (rows_left > 0) {
        const int lam = LAMF >= 0 ? LAMF : st.lam;
        const int rem = wp->r[lam];
        const int glam = P.g[lam];
        const bool memo_run =
            LAMF >= 0 ? true : ((P.lam_m >= 0) && !st.inwalk && lam == P.lam_m);
        if (LAMF < 0 && !memo_run && lam == P.lam_w && P.wl_h1 > 0) {
            // A run of walk leaves (the ordinary step at the last two
            // coordinates): only the candidates a_{d-2} = v whose remainder
            // g_{d-1} divides hold a row, and they form a progression, so
            // rows are produced directly -- v from the largest valid value
            // <= st.vcur down by h1, a_{d-1} up by g1 -- with no candidate
            // that holds no row evaluated.
            long long vtop = -1;
            if (rem % P.wl_e == 0) {
                const long long h1 = P.wl_h1;
                const long long vstar = (long long)((rem / P.wl_e) % h1) * P.wl_inv % h1;
                if (st.vcur >= vstar) vtop = st.vcur - (st.vcur - vstar) % h1;
            }
            const uint32_t nrun = vtop >= 0 ? (uint32_t)(vtop / P.wl_h1) + 1u : 0u;
            const int wtop =
                vtop >= 0 ? (int)(((long long)rem - vtop * glam) / P.g[d - 1]) : 0;
            uint64_t qe = skip + rows_left;
            if (qe > nrun) qe = nrun;
            const uint32_t q_end = (uint32_t)qe;
            for (uint32_t q0 = (uint32_t)skip; q0 < q_end;) {
                uint32_t cnt = q_end - q0;
                if (cnt > 32u) cnt = 32u;
                if (cnt > B - hpos) cnt = B - hpos;
                before_round();
                if ((uint32_t)lane < cnt) {
                    const int q = (int)(q0 + lane);
                    int32_t *dst = ring + (size_t)(half * B + hpos + lane) * d;
#pragma unroll
                    for (int c = 0; c < DM; ++c) {
                        if (c >= d - 2) break;
                        dst[c] = pre[c];
                    }
                    dst[d - 2] = (int)(vtop - (long long)q * P.wl_h1);
                    dst[d - 1] = wtop + q * P.wl_g1;
                }
                q0 += cnt;
                after_round(cnt);
            }
            const uint32_t emitted = q_end > (uint32_t)skip ? q_end - (uint32_t)skip : 0u;
            rows_left -= emitted;
            if (rows_left == 0) break;
            skip = 0;
            st.vcur = -1;
            if (!advance(P, wp, lane, st)) {
                if (lane == 0) atomicExch(P.status, (int)DEV_INTERNAL);
                ok = false;
                break;
            }
#pragma unroll
            for (int c = 0; c < DM; ++c) pre[c] = (c < st.lam) ? wp->a[c] : 0;
            continue;
        }
        const long long vl = st.vcur - lane;
        const bool valid = vl >= 0;
        int p = 0;
        uint64_t incl = 0;
        int type = T_NONE;
        // a run of walk leaves: candidate v is valid iff g_{d-1} divides the
        // remainder (the ordinary step's test); row ends by counting, no table
        const bool walk_run = LAMF < 0 && !memo_run && lam == P.lam_w;
        uint32_t wq = 0;
        bool wvalid = false;
        if (valid) {
            p = (int)((long long)rem - vl * glam);
            if (p < 0 || p > P.n) {  // cannot happen for 0 <= vl <= rem / glam
                atomicExch(P.status, (int)DEV_INTERNAL);
                p = 0;
            }
            if (walk_run) {
                wq = fd_div((uint32_t)p, P.glast);
                wvalid = (uint32_t)p - wq * P.glast.g == 0u;
            } else {
                incl = __ldg(P.C + (long long)lam * P.cs + p);
            }
            if (memo_run && (LAMF >= 0 || p < P.top))
                type = T_MEMO;
            else if (lam == P.lam_w)
                type = T_WALK;
            else
                type = T_INTERNAL;
        }
        if (walk_run) {
            const unsigned vm = __ballot_sync(FULL, wvalid);
            incl = st.base + (uint64_t)__popc(vm & (0xffffffffu >> (31 - lane)));
        }
        uint64_t prev = __shfl_up_sync(FULL, incl, 1);
        if (lane == 0) prev = st.base;
        const uint64_t size = valid ? incl - prev : 0ull;
        const unsigned im = __ballot_sync(FULL, type == T_INTERNAL && size > 0);
        const int first_int = im ? __ffs(im) - 1 : 32;
        const int nvalid = st.vcur + 1 < 32 ? (int)(st.vcur + 1) : 32;
        const int consumed = first_int < nvalid ? first_int : nvalid;
        const uint64_t last_incl = consumed > 0 ? shfl_u64(incl, consumed - 1) : st.base;
        const uint64_t batch_rows = last_incl - st.base;
        uint32_t E32 = CAP32, X32 = 0;
        if (lane < consumed) {
            const uint64_t e = incl - st.base;
            E32 = e < (uint64_t)CAP32 ? (uint32_t)e : CAP32;
            if (type == T_MEMO)
                X32 = (LAMF < 0 && P.pair_memo) ? pair_top(P, p) : (uint32_t)__ldg(P.O + p);
            else if (type == T_WALK)
                X32 = walk_run ? wq : fd_div((uint32_t)p, P.glast);
        }
        uint64_t q_end64 = skip + rows_left;
        if (q_end64 > batch_rows) q_end64 = batch_rows;
        const uint32_t q_begin = (uint32_t)skip;
        const uint32_t q_end = (uint32_t)q_end64;
        // Dense batches of memo leaves: rounds follow the leaves, so every
        // lane of a round copies a row of the same leaf (no per-row search).
        const bool all_memo = __all_sync(FULL, lane >= consumed || type == T_MEMO);
        const bool dense = memo_run && all_memo && consumed > 0 &&
                           batch_rows >= (uint64_t)P.dense_min * (uint64_t)consumed;
        if (dense && q_end > q_begin) {
            const int lfirst = __popc(__ballot_sync(FULL, E32 <= q_begin));
            for (int j = lfirst; j < consumed; ++j) {
                const uint32_t ej = __shfl_sync(FULL, E32, j);
                uint32_t sj = __shfl_sync(FULL, E32, j > 0 ? j - 1 : 0);
                if (j == 0) sj = 0;
                const uint32_t lo = sj > q_begin ? sj : q_begin;
                const uint32_t hi = ej < q_end ? ej : q_end;
                if (lo < hi) {
                    const uint32_t xj = __shfl_sync(FULL, X32, j);
                    const int pj = __shfl_sync(FULL, p, j);
                    const int vj = (int)(st.vcur - j);
                    const bool pair = LAMF < 0 && P.pair_memo;
                    if (!pair && (uint64_t)xj + (hi - sj) > P.memo_rows) {  // bounds guard
                        if (lane == 0) atomicExch(P.status, (int)DEV_INTERNAL);
                        break;
                    }
                    const int kk = LAMF >= 0 ? KF : P.K;
                    const int32_t *mbase = pair ? P.memo : P.memo + (size_t)xj * (size_t)kk;
                    for (uint32_t q0 = lo; q0 < hi;) {
                        uint32_t cnt = hi - q0;
                        if (cnt > 32u) cnt = 32u;
                        if (cnt > B - hpos) cnt = B - hpos;
                        before_round();
                        if ((uint32_t)lane < cnt) {
                            int32_t *dst = ring + (size_t)(half * B + hpos + lane) * d;
                            const int32_t *mrow =
                                pair ? mbase : mbase + (size_t)(q0 + lane - sj) * (size_t)kk;
                            if (pair) {
                                // pair memo: the row from the progression
                                const int o = (int)(q0 + lane - sj);
                                const int av = (int)xj - o * P.wl_h1;
#pragma unroll
                                for (int c = 0; c < DM; ++c) {
                                    if (c >= lam) break;
                                    dst[c] = pre[c];
                                }
                                dst[lam] = vj;
                                dst[lam + 1] = av;
                                dst[lam + 2] = (int)fd_div(
                                    (uint32_t)(pj - av * P.g[d - 2]), P.glast);
                            } else if constexpr (LAMF >= 0) {
#pragma unroll
                                for (int c = 0; c < LAMF; ++c) dst[c] = pre[c];
                                dst[LAMF] = vj;
#pragma unroll
                                for (int c = 0; c < KF; ++c)
                                    cp_async4(dst + LAMF + 1 + c, mrow + c);
                            } else {
#pragma unroll
                                for (int c = 0; c < DM; ++c) {
                                    if (c >= d)
                                        break;
                                    if (c < lam)
                                        dst[c] = pre[c];
                                    else if (c == lam)
                                        dst[c] = vj;
                                    else
                                        cp_async4(dst + c, mrow + (c - lam - 1));
                                }
                            }
                        }
                        q0 += cnt;
                        after_round(cnt);
                    }
                }
                if (ej >= q_end) break;
            }
        } else {
        for (uint32_t q0 = q_begin; q0 < q_end;) {
            uint32_t cnt = q_end - q0;
            if (cnt > 32u) cnt = 32u;
            if (cnt > B - hpos) cnt = B - hpos;  // rounds never cross a half boundary
            before_round();
            const bool act = (uint32_t)lane < cnt;
            const uint32_t q_last = q0 + cnt - 1;
            const uint32_t q = act ? q0 + lane : q_last;  // idle lanes map a row of the round
            // owning leaf of row q: l = number of leaves ending at or before q
            const int lcur = __popc(__ballot_sync(FULL, E32 <= q0));
            const int nb = __popc(__ballot_sync(FULL, E32 > q0 && E32 <= q_last));
            int l = lcur;
            if (nb <= 3) {
                for (int t = 0; t < nb; ++t) {
                    const uint32_t e = __shfl_sync(FULL, E32, lcur + t);
                    if (e <= q) ++l;
                }
            } else {
                l = 0;
#pragma unroll
                for (int sft = 16; sft >= 1; sft >>= 1) {
                    const uint32_t e = __shfl_sync(FULL, E32, l + sft - 1);
                    if (e <= q) l += sft;
                }
            }
            uint32_t eprev = __shfl_sync(FULL, E32, l > 0 ? l - 1 : 0);
            if (l == 0) eprev = 0;
            const uint32_t o = q - eprev;
            const int pl = __shfl_sync(FULL, p, l);
            const uint32_t xl = __shfl_sync(FULL, X32, l);
            const int vrow = (int)(st.vcur - l);
            bool mleaf = memo_run && (LAMF >= 0 || pl < P.top);
            const bool pair = LAMF < 0 && P.pair_memo && mleaf;
            if (act && mleaf && !pair && (uint64_t)xl + o >= P.memo_rows) {  // bounds guard
                atomicExch(P.status, (int)DEV_INTERNAL);
                mleaf = false;
            }
            if (act) {
                int32_t *dst = ring + (size_t)(half * B + hpos + lane) * d;
                if constexpr (LAMF >= 0) {
#pragma unroll
                    for (int c = 0; c < LAMF; ++c) dst[c] = pre[c];
                    dst[LAMF] = vrow;
                    const int32_t *mrow = P.memo + (size_t)(xl + o) * (size_t)KF;
                    if (mleaf) {
#pragma unroll
                        for (int c = 0; c < KF; ++c) cp_async4(dst + LAMF + 1 + c, mrow + c);
                    } else {
#pragma unroll
                        for (int c = 0; c < KF; ++c) dst[LAMF + 1 + c] = 0;
                    }
                } else if (pair) {
                    // pair memo: the row from the progression
                    const int av = (int)xl - (int)o * P.wl_h1;
#pragma unroll
                    for (int c = 0; c < DM; ++c) {
                        if (c >= lam) break;
                        dst[c] = pre[c];
                    }
                    dst[lam] = vrow;
                    dst[lam + 1] = av;
                    dst[lam + 2] = (int)fd_div((uint32_t)(pl - av * P.g[d - 2]), P.glast);
                } else {
                    const int32_t *mrow =
                        mleaf ? P.memo + (size_t)(xl + o) * (size_t)P.K : nullptr;
#pragma unroll
                    for (int c = 0; c < DM; ++c) {
                        if (c >= d)
                            break;
                        if (c < lam)
                            dst[c] = pre[c];
                        else if (c == lam)
                            dst[c] = vrow;
                        else if (mleaf)
                            cp_async4(dst + c, mrow + (c - lam - 1));
                        else
                            dst[c] = (int)xl;
                    }
                }
            }
            q0 += cnt;
            after_round(cnt);
        }
        }
        const uint32_t emitted = q_end > q_begin ? q_end - q_begin : 0u;
        rows_left -= emitted;
        if (rows_left == 0) break;
        skip = 0;
        if (first_int < nvalid) {
            // the next child is a memo-level prefix beyond the memo: walk it
            const int ve = (int)(st.vcur - first_int);
            const int pe = rem - ve * glam;
            if (lane == 0) {
                wp->a[lam] = ve;
                wp->r[lam + 1] = pe;
            }
            __syncwarp();
            descend(P, wp, lam + 1, P.lam_w, lane);
            st.lam = P.lam_w;
            st.inwalk = 1;
            st.vcur = wp->r[P.lam_w] / P.g[P.lam_w];
            st.base = 0;
        } else {
            st.base = last_incl;
            st.vcur -= consumed;
            if (st.vcur < 0 && !advance(P, wp, lane, st)) {
                if (lane == 0) atomicExch(P.status, (int)DEV_INTERNAL);
                ok = false;
                break;
            }
        }
#pragma unroll
        for (int c = 0; c < DM; ++c) pre[c] = (c < st.lam) ? wp->a[c] : 0;
    }
    cp_async_wait<0>();
    if (pend)
        flush_rows(P, ring + (size_t)(half ^ 1u) * B * d,
                      row0 + (uint64_t)(nfull - 1) * B, B, d, lane, pol);
    if (hpos > 0)
        flush_rows(P, ring + (size_t)half * B * d, row0 + (uint64_t)nfull * B, hpos, d,
                      lane, pol);
    if (lane == 0) bulk_wait_read_all();
    __syncwarp();
    return ok;
}

// Rows are handed out as work items (equal-cost ranges when the runs table
// is present, else equal-row ranges) from an atomic counter.
template <int D, int LAMF>
__global__ void __launch_bounds__(ENUM_THREADS, 4)
    fz_enum_kernel(const __grid_constant__ EnumParams P) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const uint32_t B = (uint32_t)P.half_rows;
    int32_t *ring = reinterpret_cast<int32_t *>(smem_raw) + (size_t)wid * 2 * B * D;
    WarpPath *wp =
        reinterpret_cast<WarpPath *>(smem_raw + (size_t)ENUM_WARPS * 2 * B * D * 4) + wid;
    const uint64_t pol = policy_evict_first();

    // cost range of the requested ranks (work-balanced slicing)
    uint64_t cost_lo = 0, cost_hi = 0;
    if (P.RT) {
        cost_lo = rank_to_cost(P, P.rank_begin, lane);
        cost_hi = rank_to_cost(P, P.rank_begin + P.nrows, lane);
    }
    for (;;) {
        unsigned long long s = 0;
        if (lane == 0) s = atomicAdd(P.slice_counter, 1ull);
        s = __shfl_sync(FULL, s, 0);
        uint64_t row0 = 0, row1 = 0;  // relative to out
        const int it = item_rows(P, s, cost_lo, cost_hi, lane, row0, row1);
        if (it == 0) break;
        if (it == 1) continue;
        if (!enum_slice<D, LAMF>(P, wp, ring, B, row0, row1, pol, lane)) break;
    }
    cp_async_wait<0>();
    if (lane == 0) bulk_wait_all();
    __syncwarp();
}

// ---------------------------------------------------------------------------
// Full memo of depth K <= 3 in run order.  The walk covers the leading LAMF
// coordinates only: for a prefix (a_0..a_{LAMF-1}) with remainder r, the
// rows of its whole subtree -- every a_LAMF from r div g down to 0, each with
// Memo[r - a_LAMF g] -- are the contiguous run-memo range
// [cls_beg[r mod g], + C[LAMF][r]) with a_LAMF = r div g - (first word).  A
// round is then one 16-byte load and one row store per lane.
// ---------------------------------------------------------------------------
template <int D, int LAMF, int K>
__device__ __forceinline__ void run_store_row(int32_t *dst, const int (&a)[LAMF > 0 ? LAMF : 1],
                                              int vmax, int4 m) {
    int32_t w[D];
#pragma unroll
    for (int c = 0; c < LAMF; ++c) w[c] = a[c];
    w[LAMF] = vmax - m.x;
    if constexpr (K >= 1) w[LAMF + 1] = m.y;
    if constexpr (K >= 2) w[LAMF + 2] = m.z;
    if constexpr (K >= 3) w[LAMF + 3] = m.w;
    if constexpr (D % 2 == 0) {  // row starts are 8-byte aligned: 8-byte stores
#pragma unroll
        for (int c = 0; c < D; c += 2)
            *reinterpret_cast<int2 *>(dst + c) = make_int2(w[c], w[c + 1]);
    } else {
#pragma unroll
        for (int c = 0; c < D; ++c) dst[c] = w[c];
    }
}

template <int D, int LAMF, int K>
__device__ __forceinline__ bool runs_slice(const EnumParams &P, int32_t *ring, uint32_t B,
                                           uint64_t row0, uint64_t row1, uint64_t pol,
                                           int lane) {
    // unrank the first row: the prefix, its remainder and the offset in its run
    int a[LAMF > 0 ? LAMF : 1];
    int r[LAMF + 1];
    uint64_t R = P.rank_begin + row0;
    r[0] = P.n;
    a[0] = 0;
#pragma unroll
    for (int j = 0; j < LAMF; ++j) {
        int v;
        uint64_t before;
        find_child(P, j, r[j], R, lane, v, before);
        a[j] = v;
        R -= before;
        r[j + 1] = r[j] - v * P.g[j];
    }
    uint64_t off = R;
    uint64_t left = row1 - row0;
    uint32_t hpos = 0, half = 0, nfull = 0;
    const int glam = P.g[LAMF];
    bool ok = true;
    for (;;) {
        const int rem = r[LAMF];
        const uint64_t run_rows = __ldg(P.C + (long long)LAMF * P.cs + rem);
        if (off < run_rows) {
            const int vmax = rem / glam;
            const int cls = rem - vmax * glam;
            const uint64_t src64 = __ldg(P.cls_beg + cls) + off;
            uint64_t take64 = run_rows - off;
            if (take64 > left) take64 = left;
            if (src64 + take64 > P.memo_rows) {  // bounds guard: the run lies in the memo
                if (lane == 0) atomicExch(P.status, (int)DEV_INTERNAL);
                ok = false;
                break;
            }
            left -= take64;
            // the run lies in the memo (< 2^30 rows): 32-bit row indices
            uint32_t src = (uint32_t)src64, take = (uint32_t)take64;
            // Rounds of up to 64 rows (never across a ring half); lane l
            // stores rows l and l + 32 of a round.  The memo rows of the next
            // round are loaded before this round's rows are stored.  The loop
            // is unrolled twice so the two register sets swap roles without
            // moves.
            uint32_t c0 = take < 64u ? take : 64u;
            if (c0 > B - hpos) c0 = B - hpos;
            int4 x0 = make_int4(0, 0, 0, 0), x1 = x0, y0 = x0, y1 = x0;
            {
                const int4 *ms = P.run_memo + src;
                if ((uint32_t)lane < c0) x0 = __ldg(ms + lane);
                if ((uint32_t)lane + 32u < c0) x1 = __ldg(ms + 32 + lane);
            }
            auto round = [&](const int4 &cur0, const int4 &cur1, int4 &nxt0, int4 &nxt1) {
                const uint32_t hp1 = hpos + c0 == B ? 0u : hpos + c0;
                const uint32_t t1 = take - c0;
                uint32_t c1 = t1 < 64u ? t1 : 64u;
                if (c1 > B - hp1) c1 = B - hp1;
                const int4 *ns = P.run_memo + (src + c0);
                if ((uint32_t)lane < c1) nxt0 = __ldg(ns + lane);
                if ((uint32_t)lane + 32u < c1) nxt1 = __ldg(ns + 32 + lane);
                if (hpos == 0 && nfull >= 2) {
                    // re-entering a half: the bulk store issued from it two
                    // flushes ago must have finished reading it
                    if (lane == 0) bulk_wait_read<1>();
                    __syncwarp();
                }
                int32_t *dst = ring + (size_t)(half * B + hpos + lane) * D;
                if ((uint32_t)lane < c0) run_store_row<D, LAMF, K>(dst, a, vmax, cur0);
                if ((uint32_t)lane + 32u < c0)
                    run_store_row<D, LAMF, K>(dst + 32 * D, a, vmax, cur1);
                if (hp1 == 0) {
                    flush_rows(P, ring + (size_t)half * B * D, row0 + (uint64_t)nfull * B, B, D,
                               lane, pol);
                    ++nfull;
                    half ^= 1u;
                }
                hpos = hp1;
                src += c0;
                take = t1;
                c0 = c1;
            };
            for (;;) {
                round(x0, x1, y0, y1);
                if (take == 0) break;
                round(y0, y1, x0, x1);
                if (take == 0) break;
            }
            if (left == 0) break;
        }
        off = 0;
        // the next prefix in descending order: decrement the deepest positive
        // coordinate, reset the ones after it to their maxima
        int jj = -1;
#pragma unroll
        for (int j = 0; j < LAMF; ++j)
            if (a[j] > 0) jj = j;
        if (jj < 0) {  // past the last prefix with rows still owed
            if (lane == 0) atomicExch(P.status, (int)DEV_INTERNAL);
            ok = false;
            break;
        }
#pragma unroll
        for (int j = 0; j < LAMF; ++j) {
            if (j == jj) {
                a[j] -= 1;
                r[j + 1] = r[j] - a[j] * P.g[j];
            } else if (j > jj) {
                a[j] = r[j] / P.g[j];
                r[j + 1] = r[j] - a[j] * P.g[j];
            }
        }
    }
    if (hpos > 0)
        flush_rows(P, ring + (size_t)half * B * D, row0 + (uint64_t)nfull * B, hpos, D, lane,
                   pol);
    if (lane == 0) bulk_wait_read_all();
    __syncwarp();
    return ok;
}

// Work items from an atomic counter: equal-cost ranges when the plan has a
// candidates table counted at level LAMF (each walked prefix costs W rows, so
// the items at the start of the order, where prefixes hold few rows each, are
// short), else equal-row ranges.
template <int D, int LAMF, int K>
__global__ void __launch_bounds__(ENUM_THREADS, 4)
    fz_enum_runs_kernel(const __grid_constant__ EnumParams P) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const uint32_t B = (uint32_t)P.half_rows;
    int32_t *ring = reinterpret_cast<int32_t *>(smem_raw) + (size_t)wid * 2 * B * D;
    const uint64_t pol = policy_evict_first();
    uint64_t cost_lo = 0, cost_hi = 0;
    if (P.RT) {
        cost_lo = rank_to_cost(P, P.rank_begin, lane);
        cost_hi = rank_to_cost(P, P.rank_begin + P.nrows, lane);
    }
    for (;;) {
        unsigned long long s = 0;
        if (lane == 0) s = atomicAdd(P.slice_counter, 1ull);
        s = __shfl_sync(FULL, s, 0);
        uint64_t row0 = 0, row1 = 0;
        const int it = item_rows(P, s, cost_lo, cost_hi, lane, row0, row1);
        if (it == 0) break;
        if (it == 1) continue;
        if (!runs_slice<D, LAMF, K>(P, ring, B, row0, row1, pol, lane)) break;
    }
    if (lane == 0) bulk_wait_all();
    __syncwarp();
}

// The run-order copy with the tuple width D <= 8 and the memo depth
// 1 <= K <= 3 read at run time (batches): the rounds of runs_slice, with the
// prefix a_0..a_{LAMF-1} (LAMF = D - K - 1 <= 6) kept in registers through
// loops unrolled to their maxima and guarded by the run-time bounds.
constexpr int RT_LAMF_MAX = 6;

__device__ __forceinline__ void run_store_row_rt(int32_t *dst, const int (&a)[RT_LAMF_MAX], int D,
                                                 int LAMF, int vmax, int4 m) {
    int w[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int t = c - LAMF;
        int v = c < RT_LAMF_MAX ? a[c] : 0;
        if (t == 0)
            v = vmax - m.x;
        else if (t == 1)
            v = m.y;
        else if (t == 2)
            v = m.z;
        else if (t == 3)
            v = m.w;
        w[c] = v;
    }
    if ((D & 3) == 0) {  // row starts 16-byte aligned
#pragma unroll
        for (int c = 0; c < 8; c += 4)
            if (c < D)
                *reinterpret_cast<int4 *>(dst + c) = make_int4(w[c], w[c + 1], w[c + 2], w[c + 3]);
    } else if ((D & 1) == 0) {  // 8-byte aligned
#pragma unroll
        for (int c = 0; c < 8; c += 2)
            if (c < D) *reinterpret_cast<int2 *>(dst + c) = make_int2(w[c], w[c + 1]);
    } else {
#pragma unroll
        for (int c = 0; c < 8; ++c)
            if (c < D) dst[c] = w[c];
    }
}

__device__ __noinline__ bool runs_slice_rt(const EnumParams &P, int32_t *ring, uint32_t B,
                                           uint64_t row0, uint64_t row1, uint64_t pol,
                                           int lane) {
    const int D = P.d;
    const int LAMF = P.d - P.K - 1;
    if (LAMF < 1 || D > 8 || P.K < 1 || P.K > 3) {  // shapes the host never sends here
        if (lane == 0) atomicExch(P.status, (int)DEV_INTERNAL);
        return false;
    }
    // unrank the first row: the prefix, its remainder and the offset in its run
    int a[RT_LAMF_MAX];
#pragma unroll
    for (int c = 0; c < RT_LAMF_MAX; ++c) a[c] = 0;
    uint64_t R = P.rank_begin + row0;
    int rem = P.n;
#pragma unroll 1
    for (int j = 0; j < LAMF; ++j) {
        int v;
        uint64_t before;
        find_child(P, j, rem, R, lane, v, before);
        R -= before;
        rem -= v * P.g[j];
#pragma unroll
        for (int c = 0; c < RT_LAMF_MAX; ++c)
            if (c == j) a[c] = v;
    }
    uint64_t off = R;
    uint64_t left = row1 - row0;
    uint32_t hpos = 0, half = 0, nfull = 0;
    const int glam = P.g[LAMF];
    bool ok = true;
    for (;;) {
        const uint64_t run_rows = __ldg(P.C + (long long)LAMF * P.cs + rem);
        if (off < run_rows) {
            const int vmax = rem / glam;
            const int cls = rem - vmax * glam;
            const uint64_t src64 = __ldg(P.cls_beg + cls) + off;
            uint64_t take64 = run_rows - off;
            if (take64 > left) take64 = left;
            if (src64 + take64 > P.memo_rows) {  // bounds guard: the run lies in the memo
                if (lane == 0) atomicExch(P.status, (int)DEV_INTERNAL);
                ok = false;
                break;
            }
            left -= take64;
            uint32_t src = (uint32_t)src64, take = (uint32_t)take64;
            uint32_t c0 = take < 64u ? take : 64u;
            if (c0 > B - hpos) c0 = B - hpos;
            int4 x0 = make_int4(0, 0, 0, 0), x1 = x0, y0 = x0, y1 = x0;
            {
                const int4 *ms = P.run_memo + src;
                if ((uint32_t)lane < c0) x0 = __ldg(ms + lane);
                if ((uint32_t)lane + 32u < c0) x1 = __ldg(ms + 32 + lane);
            }
            auto round = [&](const int4 &cur0, const int4 &cur1, int4 &nxt0, int4 &nxt1) {
                const uint32_t hp1 = hpos + c0 == B ? 0u : hpos + c0;
                const uint32_t t1 = take - c0;
                uint32_t c1 = t1 < 64u ? t1 : 64u;
                if (c1 > B - hp1) c1 = B - hp1;
                const int4 *ns = P.run_memo + (src + c0);
                if ((uint32_t)lane < c1) nxt0 = __ldg(ns + lane);
                if ((uint32_t)lane + 32u < c1) nxt1 = __ldg(ns + 32 + lane);
                if (hpos == 0 && nfull >= 2) {
                    if (lane == 0) bulk_wait_read<1>();
                    __syncwarp();
                }
                int32_t *dst = ring + (size_t)(half * B + hpos + lane) * D;
                if ((uint32_t)lane < c0) run_store_row_rt(dst, a, D, LAMF, vmax, cur0);
                if ((uint32_t)lane + 32u < c0) run_store_row_rt(dst + 32 * D, a, D, LAMF, vmax, cur1);
                if (hp1 == 0) {
                    flush_rows(P, ring + (size_t)half * B * D, row0 + (uint64_t)nfull * B, B, D,
                               lane, pol);
                    ++nfull;
                    half ^= 1u;
                }
                hpos = hp1;
                src += c0;
                take = t1;
                c0 = c1;
            };
            for (;;) {
                round(x0, x1, y0, y1);
                if (take == 0) break;
                round(y0, y1, x0, x1);
                if (take == 0) break;
            }
            if (left == 0) break;
        }
        off = 0;
        // the next prefix in descending order: decrement the deepest positive
        // coordinate, reset the ones after it to their maxima (the remainder
        // is carried forward from r_0 = n)
        int jj = -1;
#pragma unroll
        for (int j = 0; j < RT_LAMF_MAX; ++j)
            if (j < LAMF && a[j] > 0) jj = j;
        if (jj < 0) {
            if (lane == 0) atomicExch(P.status, (int)DEV_INTERNAL);
            ok = false;
            break;
        }
        int rr = P.n;
#pragma unroll
        for (int j = 0; j < RT_LAMF_MAX; ++j) {
            if (j < LAMF) {
                if (j == jj)
                    a[j] -= 1;
                else if (j > jj)
                    a[j] = rr / P.g[j];
                rr -= a[j] * P.g[j];
            }
        }
        rem = rr;
    }
    if (hpos > 0)
        flush_rows(P, ring + (size_t)half * B * D, row0 + (uint64_t)nfull * B, hpos, D, lane,
                   pol);
    if (lane == 0) bulk_wait_read_all();
    __syncwarp();
    return ok;
}

// ---------------------------------------------------------------------------
// Many instances in one persistent launch.  Work items (instance, slice) are
// numbered consecutively, instance i owning items [item0[i], item0[i+1]); a
// warp takes the next item from an atomic counter, finds its instance by a
// binary search over item0, copies that instance's parameters into its own
// shared-memory slot (when it changes) and runs the same slice routine as the
// single-instance kernel with the tuple width read at run time.
// ---------------------------------------------------------------------------
struct BatchEnumParams {
    const EnumParams *inst;   // per-instance parameters; `out` holds a byte offset
    int32_t *out_base;        // output base the offsets are added to
    const uint64_t *item0;    // count + 1 prefix of work items
    int count;
    uint64_t nitems;
    unsigned long long *item_counter;
};

constexpr size_t BATCH_RING_BYTES = RING_BYTES_PER_WARP;

__global__ void __launch_bounds__(ENUM_THREADS, 4)
    fz_enum_batch_kernel(const __grid_constant__ BatchEnumParams BP) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    int32_t *ring = reinterpret_cast<int32_t *>(smem_raw + (size_t)wid * BATCH_RING_BYTES);
    EnumParams *ep =
        reinterpret_cast<EnumParams *>(smem_raw + (size_t)ENUM_WARPS * BATCH_RING_BYTES) + wid;
    WarpPath *wp = reinterpret_cast<WarpPath *>(smem_raw + (size_t)ENUM_WARPS * BATCH_RING_BYTES +
                                                ENUM_WARPS * sizeof(EnumParams)) +
                   wid;
    const uint64_t pol = policy_evict_first();
    int cur = -1;
    for (;;) {
        unsigned long long item = 0;
        if (lane == 0) item = atomicAdd(BP.item_counter, 1ull);
        item = __shfl_sync(FULL, item, 0);
        if (item >= BP.nitems) break;
        // largest i with item0[i] <= item
        int lo = 0, hi = BP.count;  // item0[lo] <= item < item0[hi]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (__ldg(BP.item0 + mid) <= item)
                lo = mid;
            else
                hi = mid;
        }
        if (lo != cur) {
            const uint32_t *src = reinterpret_cast<const uint32_t *>(BP.inst + lo);
            uint32_t *dst = reinterpret_cast<uint32_t *>(ep);
            for (int w = lane; w < (int)(sizeof(EnumParams) / 4); w += 32) dst[w] = __ldg(src + w);
            __syncwarp();
            if (lane == 0) {
                int32_t *o = reinterpret_cast<int32_t *>(reinterpret_cast<char *>(BP.out_base) +
                                                         reinterpret_cast<uintptr_t>(ep->out));
                ep->out = o;
                ep->aligned = ((uintptr_t)o & 15u) == 0;
            }
            __syncwarp();
            cur = lo;
        }
        const EnumParams &P = *ep;
        const uint64_t s = item - __ldg(BP.item0 + lo);
        uint64_t row0, row1;
        if (P.RT) {
            const uint64_t cost_hi = cost_at(P, 0, P.n);
            const uint64_t c0 = s * P.slice_cost;
            if (c0 >= cost_hi) continue;
            const uint64_t c1 = c0 + P.slice_cost;
            row0 = 0;
            if (s > 0) {
                row0 = cost_to_rank(P, c0, lane) & ~31ull;
                if (row0 > P.nrows) row0 = P.nrows;
            }
            row1 = P.nrows;
            if (c1 < cost_hi) {
                row1 = cost_to_rank(P, c1, lane) & ~31ull;
                if (row1 > P.nrows) row1 = P.nrows;
            }
        } else {
            row0 = s * P.slice_rows;
            row1 = row0 + P.slice_rows < P.nrows ? row0 + P.slice_rows : P.nrows;
        }
        if (row1 <= row0) continue;
        if (P.d == 1 || (P.K == P.d && P.top > P.n)) {
            // a single block: d == 1 or the output is Memo[n] itself
            if (P.d == 1) {
                if (lane == 0 && row0 == 0) P.out[0] = P.n / P.g[0];
            } else {
                const uint64_t src0 = (__ldg(P.O + P.n) + row0) * (uint64_t)P.d;
                for (uint64_t w = lane; w < (row1 - row0) * (uint64_t)P.d; w += 32)
                    P.out[row0 * (uint64_t)P.d + w] = __ldg(P.memo + src0 + w);
            }
            continue;
        }
        // full memos in run order take the run copy; otherwise one walk for
        // every width up to 8 (row loops unrolled to 8), the 16-wide one
        // beyond: three code paths at most, so warps of different instances
        // share the instruction cache
        bool ok;
        if (P.run_memo)
            ok = runs_slice_rt(P, ring, (uint32_t)P.half_rows, row0, row1, pol, lane);
        else if (P.d <= 8)
            ok = enum_slice<0, -1, 8>(P, wp, ring, (uint32_t)P.half_rows, row0, row1, pol, lane);
        else
            ok = enum_slice<0, -1>(P, wp, ring, (uint32_t)P.half_rows, row0, row1, pol, lane);
        if (!ok) break;
    }
    cp_async_wait<0>();
    if (lane == 0) bulk_wait_all();
    __syncwarp();
}

size_t enum_batch_smem_bytes() {
    return (size_t)ENUM_WARPS * (BATCH_RING_BYTES + sizeof(EnumParams) + sizeof(WarpPath));
}

// Tuples of given ranks (one warp per rank).
template <int D>
__global__ void __launch_bounds__(ENUM_THREADS)
    fz_unrank_kernel(const __grid_constant__ EnumParams P,
                                                                 const uint64_t *ranks,
                                                                 uint64_t m) {
    __shared__ WarpPath paths[ENUM_WARPS];
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    WarpPath *wp = &paths[wid];
    const uint64_t nw = (uint64_t)gridDim.x * ENUM_WARPS;
    for (uint64_t i = (uint64_t)blockIdx.x * ENUM_WARPS + wid; i < m; i += nw) {
        const uint64_t R = ranks[i];
        RunState st;
        bool ok;
        const uint64_t off = unrank_to_leaf(P, wp, R, lane, st, &ok);
        if (!ok) {
            if (lane < D) P.out[i * D + lane] = -1;
            if (lane == 0) atomicExch(P.status, (int)DEV_INTERNAL);
            continue;
        }
        const int lam = st.lam;
        const int v = (int)st.vcur;
        const int p = wp->r[lam] - v * P.g[lam];
        bool mleaf = (P.lam_m >= 0) && !st.inwalk && lam == P.lam_m && p < P.top;
        if (mleaf && __ldg(P.O + p) + off >= P.memo_rows) {  // bounds guard
            if (lane == 0) atomicExch(P.status, (int)DEV_INTERNAL);
            mleaf = false;
        }
        if (lane < D) {
            int x;
            if (lane < lam)
                x = wp->a[lane];
            else if (lane == lam)
                x = v;
            else if (mleaf)
                x = __ldg(P.memo + (size_t)(__ldg(P.O + p) + off) * P.K + (lane - lam - 1));
            else
                x = (int)fd_div((uint32_t)p, P.glast);
            P.out[i * D + lane] = x;
        }
        __syncwarp();
    }
}

// Whole output taken from one place: d == 1 (one candidate) or k == d (the
// output is Memo[n] itself).  mode 1: copy memo rows; mode 2: single row.
__global__ void fz_direct_kernel(const EnumParams P, int mode) {
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t nt = (uint64_t)gridDim.x * blockDim.x;
    if (mode == 1) {
        const uint64_t src0 = (__ldg(P.O + P.n) + P.rank_begin) * (uint64_t)P.d;
        const uint64_t words = P.nrows * (uint64_t)P.d;
        if (src0 + words > P.memo_rows * (uint64_t)P.d) {  // bounds guard
            if (tid == 0) atomicExch(P.status, (int)DEV_INTERNAL);
            return;
        }
        for (uint64_t w = tid; w < words; w += nt) P.out[w] = __ldg(P.memo + src0 + w);
    } else if (tid == 0 && P.nrows > 0) {
        P.out[0] = P.n / P.g[0];
    }
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
static int half_rows_for(int d, int ring_bytes = RING_BYTES_PER_WARP) {
    int b = ring_bytes / (8 * d);
    b = (b / 32) * 32;
    return b < 32 ? 32 : b;
}

// Ring bytes per warp for an occupancy cap: fewer resident warps get larger
// rings, so the bytes in flight per SM stay about the same.
// FZ_ENUM_RING_KB overrides (tuning only).
static int ring_bytes_for(int ctas_per_sm) {
    static const int forced = [] {
        const char *e = getenv("FZ_ENUM_RING_KB");
        const int kb = e ? atoi(e) : 0;
        return (kb >= 4 && kb <= 24) ? kb * 1024 : 0;
    }();
    if (forced) return forced;
    if (ctas_per_sm <= 0 || ctas_per_sm >= 4) return RING_BYTES_PER_WARP;
    const int b = (192 * 1024) / (ctas_per_sm * ENUM_WARPS);
    return b > 16 * 1024 ? 16 * 1024 : (b / 1024) * 1024;
}

constexpr int ENUM_MAX_SMEM = 200 * 1024;

template <typename Kern>
static int launch_enum_kernel(Kern kern, const EnumParams &P, int D, cudaStream_t s, int sms,
                              DeviceOnce &attr_set) {
    const size_t smem = (size_t)ENUM_WARPS * 2 * P.half_rows * D * 4 +
                        (size_t)ENUM_WARPS * sizeof(WarpPath);
    if (smem > (size_t)ENUM_MAX_SMEM) return set_error(FZ_EINTERNAL, "enumerate: ring too large");
    int dev = 0;
    FZ_CUDA_TRY(cudaGetDevice(&dev));
    if (!attr_set.is_set(dev)) {
        FZ_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         ENUM_MAX_SMEM));
        attr_set.set(dev);
    }
    int per_sm = 0;
    FZ_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, ENUM_THREADS, smem));
    if (P.ctas_per_sm > 0 && per_sm > P.ctas_per_sm) per_sm = P.ctas_per_sm;
    if (per_sm < 1) per_sm = 1;
    uint64_t want = (P.nslices + ENUM_WARPS - 1) / ENUM_WARPS;
    uint64_t grid = (uint64_t)per_sm * sms;
    if (want < grid) grid = want;
    if (grid < 1) grid = 1;
    FZ_CUDA_TRY(cudaMemsetAsync(P.slice_counter, 0, sizeof(unsigned long long), s));
    kern<<<(unsigned)grid, ENUM_THREADS, smem, s>>>(P);
    note_launch();
    FZ_CUDA_TRY(cudaGetLastError());
    return FZ_OK;
}

template <int D, int LAMF>
static int launch_enum_dl(const EnumParams &P, cudaStream_t s, int sms) {
    static DeviceOnce attr_set;
    return launch_enum_kernel(fz_enum_kernel<D, LAMF>, P, D, s, sms, attr_set);
}

template <int D, int LAMF, int K>
static int launch_enum_runs(const EnumParams &P, cudaStream_t s, int sms) {
    static DeviceOnce attr_set;
    return launch_enum_kernel(fz_enum_runs_kernel<D, LAMF, K>, P, D, s, sms, attr_set);
}

// Full memo of depth 2, 3 or 4: every run is a memo run at a fixed
// coordinate; use the compile-time specialisation.  Otherwise generic.
template <int D>
static int launch_enum_d(const EnumParams &P, cudaStream_t s, int sms) {
    const bool full = P.lam_m >= 0 && P.top > P.n;
    const int K = P.K;
    if (full && P.run_memo && P.cls_beg) {
        if (K == 1 && D >= 2) return launch_enum_runs<D, (D >= 2 ? D - 2 : 0), 1>(P, s, sms);
        if (K == 2 && D >= 3) return launch_enum_runs<D, (D >= 3 ? D - 3 : 0), 2>(P, s, sms);
        if (K == 3 && D >= 4) return launch_enum_runs<D, (D >= 4 ? D - 4 : 0), 3>(P, s, sms);
    }
    if (full && K == 2 && D >= 3) return launch_enum_dl<D, (D >= 3 ? D - 3 : 0)>(P, s, sms);
    if (full && K == 3 && D >= 4) return launch_enum_dl<D, (D >= 4 ? D - 4 : 0)>(P, s, sms);
    if (full && K == 4 && D >= 5) return launch_enum_dl<D, (D >= 5 ? D - 5 : 0)>(P, s, sms);
    return launch_enum_dl<D, -1>(P, s, sms);
}

template <int D>
static int launch_unrank_d(const EnumParams &P, const uint64_t *ranks, uint64_t m,
                           cudaStream_t s) {
    uint64_t blocks = (m + ENUM_WARPS - 1) / ENUM_WARPS;
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    fz_unrank_kernel<D><<<(unsigned)blocks, ENUM_THREADS, 0, s>>>(P, ranks, m);
    note_launch();
    FZ_CUDA_TRY(cudaGetLastError());
    return FZ_OK;
}

// FZ_WALK_PROGRESSION=0 evaluates walk leaves candidate by candidate as the
// ordinary step does (tuning and testing only).
bool walk_progression_enabled() {
    static const bool on = [] {
        const char *e = getenv("FZ_WALK_PROGRESSION");
        return !(e && e[0] == '0');
    }();
    return on;
}

// Rows per leaf from which a batch of memo leaves is copied leaf by leaf:
// 16 for plans, 64 for batches (a 4096-instance batch of widths 3..8:
// 11.8 ms at 16, 11.3 at 64 and 256, 11.6 never leaf by leaf, 12.3 at 4).
// FZ_ENUM_DENSE_MIN overrides both (tuning only).
static int dense_min_for(bool batch) {
    static const int forced = [] {
        const char *e = getenv("FZ_ENUM_DENSE_MIN");
        const int v = e ? atoi(e) : -1;
        return v >= 0 ? v : -1;
    }();
    if (forced >= 0) return forced;
    return batch ? 64 : 16;
}

static EnumParams make_params(const EnumLaunch &L) {
    EnumParams P{};
    P.C = L.C;
    P.cs = L.cs;
    P.O = L.O;
    P.memo = L.memo;
    P.memo_rows = L.memo_rows;
    P.ctas_per_sm = L.ctas_per_sm;
    P.dense_min = dense_min_for(false);
    P.RT = L.RT;
    P.W = L.W;
    P.lam_r = L.lam_r;
    P.status = L.status;
    P.slice_counter = L.slice_counter;
    P.n = L.n;
    P.d = L.d;
    P.K = L.K;
    P.top = L.top;
    for (int i = 0; i < L.d; ++i) P.g[i] = L.g[i];
    P.glast = make_fastdiv((uint32_t)L.g[L.d - 1]);
    P.wl_e = 1;
    P.wl_h1 = P.wl_g1 = P.wl_inv = 0;
    P.fd_e = P.fd_h1 = P.fd_g2 = make_fastdiv(1u);
    P.pair_memo = L.pair_memo && L.K == 2 && L.d >= 3 && L.top > L.n;
    if (L.d >= 2 && (walk_progression_enabled() || P.pair_memo)) {
        int64_t e, h1, g1, inv;
        pair_params(L.g[L.d - 2], L.g[L.d - 1], &e, &h1, &g1, &inv);
        P.wl_e = (int)e;
        P.wl_h1 = (int)h1;
        P.wl_g1 = (int)g1;
        P.wl_inv = (int)inv;
        P.fd_e = make_fastdiv((uint32_t)e);
        P.fd_h1 = make_fastdiv((uint32_t)h1);
        P.fd_g2 = make_fastdiv((uint32_t)L.g[L.d - 2]);
    }
    const bool memo = L.K >= 1 && L.K <= L.d - 1 && L.top > 0;
    P.lam_m = memo ? L.d - L.K - 1 : -1;
    P.lam_w = L.d - 2;
    if (!memo) {
        P.K = 0;
        P.top = 0;
    }
    // the run-order memo serves full memos of depth 1..3
    const bool runs = memo && L.top > L.n && L.K <= 3 && L.run_memo && L.cls_beg;
    P.run_memo = runs ? L.run_memo : nullptr;
    P.cls_beg = runs ? L.cls_beg : nullptr;
    // the run walk's candidates are the prefixes of its LAMF = d - K - 1
    // leading coordinates; a table counted at another level cannot balance it
    if (runs && P.lam_r != L.d - L.K - 1) P.RT = nullptr;
    return P;
}

#define FZ_DISPATCH_D(d, FN, ...)                 \
    switch (d) {                                  \
        case 2: return FN<2>(__VA_ARGS__);        \
        case 3: return FN<3>(__VA_ARGS__);        \
        case 4: return FN<4>(__VA_ARGS__);        \
        case 5: return FN<5>(__VA_ARGS__);        \
        case 6: return FN<6>(__VA_ARGS__);        \
        case 7: return FN<7>(__VA_ARGS__);        \
        case 8: return FN<8>(__VA_ARGS__);        \
        case 9: return FN<9>(__VA_ARGS__);        \
        case 10: return FN<10>(__VA_ARGS__);      \
        case 11: return FN<11>(__VA_ARGS__);      \
        case 12: return FN<12>(__VA_ARGS__);      \
        case 13: return FN<13>(__VA_ARGS__);      \
        case 14: return FN<14>(__VA_ARGS__);      \
        case 15: return FN<15>(__VA_ARGS__);      \
        case 16: return FN<16>(__VA_ARGS__);      \
        default: return set_error(FZ_EINVAL, "d out of range"); \
    }

// Enumerate ranks [rank_begin, rank_begin + nrows) into out.  Asynchronous.
int launch_enumerate(const EnumLaunch &L, uint64_t rank_begin, uint64_t nrows, int32_t *out,
                     uint64_t slice_rows, cudaStream_t s) {
    if (nrows == 0) return FZ_OK;
    if (!out || !L.C || !L.status || !L.slice_counter || (L.K >= 1 && L.top > 0 && !L.O) ||
        (L.K >= 1 && L.top > 0 && L.memo_rows > 0 && !L.memo))
        return set_error(FZ_EINTERNAL, "enumerate: missing device buffer");
    EnumParams P = make_params(L);
    P.out = out;
    P.rank_begin = rank_begin;
    P.nrows = nrows;
    P.aligned = ((uintptr_t)out & 15u) == 0 && !L.plain_stores;
    if (L.d == 1 || (L.K == L.d && L.top > L.n)) {
        const int mode = (L.d == 1 && !(L.K == 1 && L.top > L.n)) ? 2 : 1;
        uint64_t words = nrows * (uint64_t)L.d;
        uint64_t blocks = (words + 255) / 256;
        if (blocks > 4096) blocks = 4096;
        if (blocks < 1) blocks = 1;
        fz_direct_kernel<<<(unsigned)blocks, 256, 0, s>>>(P, mode);
        note_launch();
        FZ_CUDA_TRY(cudaGetLastError());
        return FZ_OK;
    }
    DeviceProps dp;
    int rc = device_props(&dp);
    if (rc != FZ_OK) return rc;
    if (slice_rows < 4) slice_rows = 4;
    slice_rows = (slice_rows + 3) & ~3ull;
    P.slice_rows = slice_rows;
    P.nslices = (nrows + slice_rows - 1) / slice_rows;
    if (P.RT) {
        // equal-cost work items; about as many as equal-row items would be
        const uint64_t cost = L.total_cost ? L.total_cost : 1;
        const uint64_t rows = L.total_rows ? L.total_rows : 1;
        const double per_row = (double)cost / (double)rows;
        uint64_t sc = (uint64_t)((double)slice_rows * per_row);
        P.slice_cost = sc < 64 ? 64 : sc;
    }
    P.half_rows = half_rows_for(L.d, ring_bytes_for(L.ctas_per_sm));
    FZ_DISPATCH_D(L.d, launch_enum_d, P, s, dp.sms);
}

int launch_unrank(const EnumLaunch &L, const uint64_t *ranks, uint64_t m, int32_t *out,
                  cudaStream_t s) {
    if (m == 0) return FZ_OK;
    if (!out || !ranks || !L.C || !L.status || (L.K >= 1 && L.top > 0 && !L.O))
        return set_error(FZ_EINTERNAL, "unrank: missing device buffer");
    EnumParams P = make_params(L);
    P.out = out;
    if (L.d == 1 || (L.K == L.d && L.top > L.n))
        return set_error(FZ_EINVAL, "unrank: d == 1 or k == d has a single block; use enumerate");
    FZ_DISPATCH_D(L.d, launch_unrank_d, P, ranks, m, s);
}

size_t enum_params_bytes() { return sizeof(EnumParams); }

// EnumParams of one batch instance (host-side image, copied to the device).
void fill_batch_params(const EnumLaunch &L, int32_t *out, uint64_t count, uint64_t slice_rows,
                       uint64_t slice_cost, void *dst) {
    EnumParams P = make_params(L);
    P.dense_min = dense_min_for(true);
    P.out = out;
    P.rank_begin = 0;
    P.nrows = count;
    P.aligned = ((uintptr_t)out & 15u) == 0;
    P.slice_rows = slice_rows < 4 ? 4 : ((slice_rows + 3) & ~3ull);
    P.nslices = (count + P.slice_rows - 1) / P.slice_rows;
    P.half_rows = half_rows_for(L.d);
    P.slice_cost = slice_cost < 64 ? 64 : slice_cost;
    memcpy(dst, &P, sizeof(P));
}

int launch_enumerate_batch(const void *params_dev, const uint64_t *item0_dev, int count,
                           uint64_t nitems, unsigned long long *item_counter, int32_t *out_base,
                           cudaStream_t s, int ctas_per_sm) {
    if (nitems == 0) return FZ_OK;
    DeviceProps dp;
    int rc = device_props(&dp);
    if (rc != FZ_OK) return rc;
    const size_t smem = enum_batch_smem_bytes();
    static DeviceOnce attr_set;
    if (!attr_set.is_set(dp.device)) {
        FZ_CUDA_TRY(cudaFuncSetAttribute(fz_enum_batch_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr_set.set(dp.device);
    }
    int per_sm = 0;
    FZ_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fz_enum_batch_kernel,
                                                              ENUM_THREADS, smem));
    if (per_sm < 1) per_sm = 1;
    if (ctas_per_sm > 0 && ctas_per_sm < per_sm) per_sm = ctas_per_sm;
    uint64_t grid = (uint64_t)per_sm * dp.sms;
    const uint64_t want = (nitems + ENUM_WARPS - 1) / ENUM_WARPS;
    if (want < grid) grid = want;
    BatchEnumParams BP;
    BP.inst = static_cast<const EnumParams *>(params_dev);
    BP.out_base = out_base;
    BP.item0 = item0_dev;
    BP.count = count;
    BP.nitems = nitems;
    BP.item_counter = item_counter;
    FZ_CUDA_TRY(cudaMemsetAsync(item_counter, 0, sizeof(unsigned long long), s));
    fz_enum_batch_kernel<<<(unsigned)grid, ENUM_THREADS, smem, s>>>(BP);
    note_launch();
    FZ_CUDA_TRY(cudaGetLastError());
    return FZ_OK;
}

uint64_t default_slice_rows(uint64_t nrows, int sms) {
    // about eight work items per resident warp, between 1024 and 65536 rows
    uint64_t warps = (uint64_t)sms * 2 * ENUM_WARPS;
    uint64_t s = nrows / (warps * 8 + 1);
    if (s < 1024) s = 1024;
    if (s > 65536) s = 65536;
    return (s + 31) & ~31ull;
}

}  // namespace fz
