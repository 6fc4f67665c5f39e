/*
 * fz.h -- C ABI of the GB300 (sm_103a) library for exact, lexicographically
 * ordered factorization sets in numerical semigroups (arXiv 2407.20474).
 *
 *   Z(n, (g_1..g_d)) = { a in N^d : sum_i a_i g_i = n }            (Section 1)
 *
 * Every list this library writes is in DESCENDING lexicographic order: a_1
 * first, greatest first (Lemma "disjlex" and its corollary, Section 2.1; the
 * lexicographically greatest next-candidate step of Algorithm 3.1, Section 3).
 * Rank 0 is the greatest tuple.  Tuples are int32, row-major: row t of an
 * output holds a_1..a_d at out[t*d + 0 .. t*d + d-1].
 *
 * Conventions shared by every call
 * --------------------------------
 * - Return value: FZ_OK (0) or a negative fz_status.  No call traps, aborts
 *   or exits; device-side failures are reported through status words that
 *   the library reads back at its next synchronising call.
 * - Generators: 1 <= d <= FZ_MAX_D, every g_i >= 1.  The caller's order is
 *   kept (never sorted): it defines the lexicographic order.  Repeated values
 *   and a gcd > 1 are allowed (they give distinct tuples / empty sets).
 * - Elements: 0 <= n <= INT32_MAX.  Z(0) = {0}; an n that is not a
 *   combination of the generators has |Z(n)| = 0 (not an error).
 * - Counts and offsets are uint64.  A count that does not fit (>= 2^64 - 1)
 *   gives FZ_EOVERFLOW.
 * - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *   stream).  Calls documented as asynchronous only enqueue work on it.
 * - Pointers ending in _dev are device memory owned by the caller; the
 *   library never frees caller memory.  Handles (fz_plan_t, fz_memo_t) own
 *   library-allocated device memory until destroyed.
 * - Output buffers (out_dev) should be 16-byte aligned: that enables the
 *   bulk (TMA) store path.  Other 4-byte aligned pointers are accepted and
 *   use plain stores.
 * - Thread safety: distinct handles may be used from distinct host threads;
 *   one handle must not be used by two threads at once.
 */
#ifndef FZ_H
#define FZ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FZ_MAX_D 16
#define FZ_AUTO (-1)

typedef enum fz_status {
    FZ_OK = 0,
    FZ_EINVAL = -1,     /* bad argument: d, g_i, n, k, top, null pointer, alignment */
    FZ_EOVERFLOW = -2,  /* a count or a byte size does not fit in 64 bits */
    FZ_ENOSPC = -3,     /* output capacity smaller than needed (*written and *rows_needed still set) */
    FZ_ENOMEM = -4,     /* device or host allocation failed */
    FZ_EAGAIN = -5,     /* serving: request deferred, queue full */
    FZ_ETIMEOUT = -6,   /* a bounded device-side wait gave up */
    FZ_ECUDA = -7,      /* other CUDA failure; see fz_last_error_string() */
    FZ_ENOTFOUND = -8,  /* unknown ticket or handle */
    FZ_EINTERNAL = -9,  /* a device-side consistency check failed */
    FZ_ECANCELED = -10  /* serving: the request was cancelled before it ran */
} fz_status;

/* Implementation options.  Every field accepts FZ_AUTO (or 0 for slice_rows). */
typedef struct fz_opts {
    int32_t k;          /* memo depth, the paper's memoDim (Section 3.1): the
                           last k coordinates are copied from the memo.
                           0 = no memo (plain next-candidate walk of
                           Algorithm 3.1); 1..d; FZ_AUTO = autotuned. */
    int32_t top;        /* memo covers remainders p in [0, top) (the paper's
                           topOfMemo); larger p take the ordinary step.
                           FZ_AUTO = n + 1 (fully populated memo). */
    int32_t slice_rows; /* output rows per warp work item (rounded up to a
                           multiple of 4); 0 = default */
    int32_t flags;      /* reserved, must be 0 */
} fz_opts_t;

/* Library version as 10000*major + 100*minor + patch. */
int fz_version(void);

/* Human-readable text of the last error raised on the calling host thread. */
const char *fz_last_error_string(void);

/* Static name of a status code ("FZ_EINVAL", ...). */
const char *fz_status_string(int status);

/* Number of CUDA kernels this library has enqueued in this process, over
 * all threads and devices (a tracing counter; memsets and copies are not
 * counted). */
uint64_t fz_kernel_launches(void);

/* Measurement utility (the paper has no counterpart): writes out_dev[w] = w
 * for w < words with 16-byte stores, one pass, so a caller can time the
 * write-only bandwidth the device reaches for distinct data of the same
 * size as an enumeration (constant fills are written faster than distinct
 * data by this GPU's memory system, so they overstate that ceiling).
 * out_dev: caller-owned device memory, 16-byte aligned (may be null when
 * words == 0, which does nothing).  Asynchronous.
 * Errors: FZ_EINVAL (null or unaligned pointer), FZ_ECUDA. */
int fz_write_probe(int32_t *out_dev, uint64_t words, void *stream);

/* Self-test of the bounded device-side waits (the paper has no counterpart):
 * two blocks wait at the library's grid barrier for arrivals that never
 * come; after limit_ms (1..2000) each gives up, records the timeout status
 * and returns, as every wait in the library does instead of hanging.
 * *status_seen (host) receives the status the host then reports: FZ_ETIMEOUT
 * when the mechanism works.  The context stays usable.  Synchronises.
 * Errors: FZ_EINVAL (null pointer, limit out of range), FZ_ENOMEM,
 * FZ_ECUDA. */
int fz_selftest_bounded_wait(uint32_t limit_ms, int *status_seen, void *stream);

/* ------------------------------------------------------------------------
 * Counting (the saved subset cardinalities of Section 2.3, generalised).
 *
 * C[j][r] = |Z(r, (g_{j+1}..g_d))| for j = 0..d, r = 0..n (0-based j), with
 * C[d][r] = [r == 0] and C[j][r] = C[j+1][r] + C[j][r - g_{j+1}].  By the
 * disjoint recurrence of Section 2 (Lemma "disjdyn"), C[i-1][r] = |Z_{>=i}(r)|
 * is the size of the block incr_i(Z_{>=i}(r)) = Z_{=i}(r + g_i).
 * ---------------------------------------------------------------------- */

/* |Z(n, g)| into *count (host).  `g` is host memory.  Synchronises `stream`.
 * Errors: FZ_EINVAL, FZ_EOVERFLOW, FZ_ENOMEM, FZ_ECUDA. */
int fz_count(const int32_t *g, int d, int32_t n, uint64_t *count, void *stream);

/* counts[r] = |Z(r, g)| for r = 0..n_max into a host array of n_max + 1
 * entries.  Entries that do not fit are UINT64_MAX (saturated).
 * Synchronises `stream`.  Errors: FZ_EINVAL, FZ_ENOMEM, FZ_ECUDA. */
int fz_count_upto(const int32_t *g, int d, int32_t n_max, uint64_t *counts,
                  void *stream);

/* Allocation-free variant of fz_count_upto, for callers that cannot call
 * cudaMalloc (while a stream is being captured, in loops that must not wait
 * on the allocator, or when another allocator owns all device memory).  The
 * paper has no counterpart; it only concerns how this library gets scratch.
 * counts_dev (caller device memory, n_max + 1 uint64) receives |Z(r, g)| for
 * r = 0..n_max, saturated at UINT64_MAX.  `g` is host memory.  All scratch
 * is one fixed device array inside the library (about 4.4 MB, held by every
 * GPU that loads the library until the process exits), so n_max is limited
 * to FZ_NOALLOC_MAX_N; larger n_max gives FZ_EINVAL.  The first call made
 * with a given device current looks up that array's device address
 * (cudaGetSymbolAddress), and so does the first call after that device's
 * context was reset (cudaDeviceReset); make such a first call before any
 * stream capture.  counts_dev must hold n_max + 1 uint64 (the call cannot
 * check a raw pointer's size).  Every call shares the array: calls that
 * overlap on the GPU (other streams or host threads) race on it.
 * Asynchronous; calls no allocating routine.
 * Errors: FZ_EINVAL, FZ_ECUDA. */
#define FZ_NOALLOC_MAX_N 262143
int fz_count_upto_noalloc(const int32_t *g, int d, int32_t n_max,
                          uint64_t *counts_dev, void *stream);

/* The full table C (layout [d+1][n+1], row-major, uint64) into caller device
 * memory `table_dev`.  Asynchronous; saturating at UINT64_MAX.
 * Errors: FZ_EINVAL, FZ_ECUDA. */
int fz_count_table(const int32_t *g, int d, int32_t n, uint64_t *table_dev,
                   void *stream);

/* ------------------------------------------------------------------------
 * Memo of tail sets, built by the dynamic FactorizationsUpToElement pass:
 * the lists Z(r, tail), r = 0..top-1, each in descending order, computed
 * elementwise in batches of min(tail) elements (Section 2.2), every batch a
 * set of copy-and-increment steps incr_i(Z_{>=i}(r - t_i)) written to
 * pre-assigned offsets (Sections 2.3 and 2.4).  The layout is a CSR:
 * offsets[r] .. offsets[r+1] are the rows of Z(r, tail), k int32 per row.
 * ---------------------------------------------------------------------- */

/* Number of memo rows sum_{r<top} |Z(r, tail)| into *rows (host).
 * Synchronises `stream`.  Errors: FZ_EINVAL, FZ_EOVERFLOW, FZ_ENOMEM, FZ_ECUDA. */
int fz_memo_rows(const int32_t *tail, int k, int32_t top, uint64_t *rows,
                 void *stream);

/* Build the memo into caller memory: offsets_dev (top + 1 uint64) and
 * rows_dev (rows_capacity rows of k int32).  *rows_needed receives the row
 * count; if it exceeds rows_capacity nothing is written and FZ_ENOSPC is
 * returned.  Synchronises `stream`.  Errors: FZ_EINVAL, FZ_ENOSPC,
 * FZ_EOVERFLOW, FZ_ENOMEM, FZ_ETIMEOUT, FZ_ECUDA. */
int fz_build_memo_into(const int32_t *tail, int k, int32_t top,
                       uint64_t *offsets_dev, int32_t *rows_dev,
                       uint64_t rows_capacity, uint64_t *rows_needed,
                       void *stream);

/* Launch schedules of the memo build (Section 2.2 names the two kinds of
 * parallelism of the dynamic pass; Section 2.4 gives the factorizationwise
 * algorithm).  All give the same memo.
 *   FZ_MEMO_BATCHED    elementwise batches of min(tail) elements, each batch
 *                      factorizationwise parallel, all in ONE launch (batches
 *                      separated by a cluster or bounded grid barrier); the
 *                      schedule every other call uses, except that plans
 *                      fill memos of depth 1 and 2 from their closed forms
 *                      (the same rows, with no dependent batches).
 *   FZ_MEMO_PER_BATCH  the same batches, one kernel launch per batch ("both"
 *                      parallelism, ordered by the stream).
 *   FZ_MEMO_PER_COPY   the factorizationwise parallel algorithm of Section
 *                      2.4: one copyAndIncrementIndex launch per element m and
 *                      generator i with a non-empty block, sized from the
 *                      saved cardinalities (host copies of the count table
 *                      and offsets).  top * k launches at most: for
 *                      comparison, not for large tops. */
#define FZ_MEMO_BATCHED 0
#define FZ_MEMO_PER_BATCH 1
#define FZ_MEMO_PER_COPY 2

/* fz_build_memo_into with an explicit schedule.  Errors: those of
 * fz_build_memo_into; FZ_EINVAL for an unknown schedule. */
int fz_build_memo_schedule(const int32_t *tail, int k, int32_t top, int schedule,
                           uint64_t *offsets_dev, int32_t *rows_dev,
                           uint64_t rows_capacity, uint64_t *rows_needed,
                           void *stream);

typedef struct fz_memo_s *fz_memo_t;
typedef struct fz_memo_info {
    int32_t k, top;
    uint64_t rows;                /* total rows */
    const uint64_t *offsets_dev;  /* top + 1 entries, owned by the memo */
    const int32_t *rows_dev;      /* rows * k entries, owned by the memo */
} fz_memo_info_t;

/* Library-owned memo (same contents as fz_build_memo_into).  Synchronises.
 * Release with fz_memo_release. */
int fz_build_memo(const int32_t *tail, int k, int32_t top, fz_memo_t *memo,
                  void *stream);
int fz_memo_info(fz_memo_t memo, fz_memo_info_t *info);
int fz_memo_release(fz_memo_t memo);

/* ------------------------------------------------------------------------
 * Plans: one instance Z(n, g) with its count table and memo resident on the
 * device, enumerated by rank ranges.
 *
 * The enumeration is the dynamic next-candidate walk (Section 3.1): leading
 * coordinates a_1..a_{d-k} are walked in descending order; each prefix with
 * p = n - phi(prefix) < top emits Memo[p] with the prefix prepended, and the
 * state is left at (prefix, 0, ..., 0); prefixes with p >= top continue with
 * the ordinary step of Algorithm 3.1 (at the last two coordinates its
 * candidates that hold a row form one residue class and are generated
 * directly).  With a full memo of depth <= 3 the memo is also kept in run
 * order and a prefix's whole subtree over the last walked coordinate is
 * copied as one contiguous run.  Work is split by exact rank ranges
 * from the count table (each warp unranks the start of its range), which
 * plays the role of the paper's splitWork.
 * ---------------------------------------------------------------------- */
typedef struct fz_plan_s *fz_plan_t;
typedef struct fz_plan_info {
    uint64_t count;         /* |Z(n, g)| */
    int32_t d, n, k, top;   /* resolved memo depth and top */
    uint64_t memo_rows;     /* rows in the memo (0 if k == 0) */
    uint64_t device_bytes;  /* device memory held by the plan */
    int32_t slice_rows;     /* resolved rows per warp work item */
    int32_t run_order;      /* 1 when the memo is also kept in run order and
                               the subtree-run kernel enumerates, else 0 */
} fz_plan_info_t;

/* Count (device), choose k and top (opts or autotune), allocate, build the
 * memo.  `g` is host memory.  Synchronises `stream`.
 * Errors: FZ_EINVAL, FZ_EOVERFLOW, FZ_ENOMEM, FZ_ETIMEOUT, FZ_ECUDA. */
int fz_plan_create(const int32_t *g, int d, int32_t n, const fz_opts_t *opt,
                   fz_plan_t *plan, void *stream);
int fz_plan_info(fz_plan_t plan, fz_plan_info_t *info);

/* Cap the enumeration kernel of this plan at `ctas` blocks per SM (0 = as
 * many as fit; the kernel fits 4).  Leaving room lets other kernels run
 * beside it, e.g. another plan's rebuild overlapping this enumeration.
 * Errors: FZ_EINVAL. */
int fz_plan_set_enum_ctas_per_sm(fz_plan_t plan, int32_t ctas);

/* Empirical tuning of the implementation options for Z(n, g): each memo
 * depth k = 0..min(d-1, 4) whose memo fits (and three work-item sizes for
 * each) is built and timed on the device -- its rebuild plus the
 * enumeration of the whole set into a scratch buffer (of the whole output
 * when it fits in a third of the free device memory, else windows of that
 * size), averaged over two passes after a first pass that also screens:
 * a candidate whose first pass, scaled to the set, takes over four times
 * the best time so far is not timed further.  The fastest is written to
 * *best (and its ms per step to *best_ms, may be NULL) and remembered for
 * this (g, n) and device: later plans created with k = FZ_AUTO use it.
 * Synchronises.  Errors: as fz_plan_create. */
int fz_autotune(const int32_t *g, int d, int32_t n, fz_opts_t *best, double *best_ms,
                void *stream);

/* One measured candidate of the tuning above. */
typedef struct fz_tune_entry {
    int32_t k;            /* memo depth */
    int32_t slice_rows;   /* rows per work item */
    int32_t run_order;    /* 1 when the memo is kept in run order */
    int32_t screened_out; /* 1: timed once only (over 4x the best so far) */
    uint64_t memo_rows;
    double build_ms;      /* rebuild: count tables + memo (measured) */
    double enum_ms;       /* enumeration of the whole set (measured; for a
                             screened-out candidate its first window, scaled) */
    double total_ms;      /* build_ms + enum_ms: what the choice minimises */
} fz_tune_entry_t;

/* fz_autotune that also reports every candidate it timed: up to `capacity`
 * entries into `entries` (host; may be NULL when capacity is 0), their
 * number into *n_entries (may be NULL).  Same choice, same memory of it.
 * Errors: as fz_autotune; FZ_EINVAL (entries null with capacity > 0). */
int fz_autotune_report(const int32_t *g, int d, int32_t n, fz_tune_entry_t *entries,
                       int capacity, int *n_entries, fz_opts_t *best, double *best_ms,
                       void *stream);

/* Recompute the count table and rebuild the memo in the plan's buffers.
 * Asynchronous (no host synchronisation), so it can be captured in a CUDA
 * graph.  Errors surface at fz_plan_sync. */
int fz_plan_rebuild(fz_plan_t plan, void *stream);

/* Rows with rank in [rank_begin, min(rank_end, count)) into out_dev (row 0
 * of out_dev is rank rank_begin).  rank_end = UINT64_MAX means "to the end".
 * *written (host) is set before launching.  Asynchronous.
 * Errors: FZ_EINVAL, FZ_ENOSPC (capacity < *written; nothing launched),
 * FZ_ECUDA. */
int fz_plan_enumerate(fz_plan_t plan, uint64_t rank_begin, uint64_t rank_end,
                      int32_t *out_dev, uint64_t out_capacity_rows,
                      uint64_t *written, void *stream);

/* Tuples of the given ranks: ranks_dev[m] (device, each < count) ->
 * out_dev[m*d ..].  Asynchronous.  Errors: FZ_EINVAL, FZ_ECUDA. */
int fz_plan_unrank(fz_plan_t plan, const uint64_t *ranks_dev, uint64_t m,
                   int32_t *out_dev, void *stream);

/* Synchronise `stream` and report device-side errors of earlier calls on
 * this plan (FZ_ETIMEOUT, FZ_EINTERNAL, FZ_ECUDA), clearing them. */
int fz_plan_sync(fz_plan_t plan, void *stream);
int fz_plan_destroy(fz_plan_t plan);

/* ------------------------------------------------------------------------
 * Batches: many instances Z(n_i, g_i) of possibly different d_i in one set
 * of launches -- batched counting tables, one memo per distinct tail shared
 * by the instances that have it (each built by the elementwise dynamic pass,
 * Sections 2.2-2.4, cut to at most 512 element batches; larger
 * remainders take the ordinary next-candidate step, Section 3.1; a memo of
 * depth 2 over the last two generators is kept as its closed form, with no
 * table), and one persistent enumeration launch over (instance, slice) work
 * items.  Full memos of depth 1..3 (widths d <= 8 with at least one walked
 * coordinate above the memo) are also kept in run order, as in plans, so a
 * prefix's whole subtree is one contiguous copy; for the closed form that
 * table is computed from the formula when it stays small.  The memo depth
 * of each generator set is chosen by the library unless opts.k is given.
 * Output: instance i's rows (d_i int32 each, descending lexicographic order)
 * start at word word_offsets[i] of the output buffer (multiples of 32 words,
 * so 128-byte aligned when the buffer is); word_offsets[count] is the total.
 * ---------------------------------------------------------------------- */
typedef struct fz_instance {
    const int32_t *g;  /* host generators, d of them */
    int32_t d;
    int32_t n;
} fz_instance_t;

typedef struct fz_batch_s *fz_batch_t;
typedef struct fz_batch_info {
    int32_t count;         /* instances */
    int32_t memos;         /* distinct memos (shared tails counted once) */
    uint64_t total_rows;   /* sum of |Z(n_i, g_i)| */
    uint64_t total_words;  /* output words needed (with alignment padding) */
    uint64_t device_bytes; /* device memory held by the batch */
    uint64_t work_items;   /* (instance, slice) items of one enumeration */
    int32_t run_order;     /* instances whose full memo is copied in run order */
    int32_t run_memos;     /* distinct run-order memos */
    int32_t coop_memos;    /* memos built by a thread-block cluster (the
                              longest, when one alone would outlast an even
                              share of the build) */
    int32_t reserved;
} fz_batch_info_t;

/* Validate, count every instance (device), choose each memo depth (opts->k
 * applies to all instances when not FZ_AUTO), build the memos.  Synchronises.
 * Errors: FZ_EINVAL, FZ_EOVERFLOW, FZ_ENOMEM, FZ_EINTERNAL, FZ_ECUDA. */
int fz_batch_create(const fz_instance_t *inst, int count, const fz_opts_t *opt,
                    fz_batch_t *batch, void *stream);
int fz_batch_info(fz_batch_t batch, fz_batch_info_t *info);
/* Host arrays (any may be NULL): rows[count], word_offsets[count + 1],
 * k[count], top[count]. */
int fz_batch_layout(fz_batch_t batch, uint64_t *rows, uint64_t *word_offsets,
                    int32_t *k, int32_t *top);
/* Recompute every table and memo in place.  Asynchronous (capturable). */
int fz_batch_rebuild(fz_batch_t batch, void *stream);
/* Cap the batch's enumeration kernel at `ctas` blocks per SM (0 = as many
 * as fit; it fits 4), leaving room for other kernels beside it, e.g. the
 * rebuild of another batch overlapping this enumeration.
 * Errors: FZ_EINVAL. */
int fz_batch_set_enum_ctas_per_sm(fz_batch_t batch, int32_t ctas);
/* All instances' rows into out_dev (capacity in int32 words).  Asynchronous,
 * one persistent kernel.  Errors: FZ_EINVAL, FZ_ENOSPC, FZ_ECUDA. */
int fz_batch_enumerate(fz_batch_t batch, int32_t *out_dev,
                       uint64_t out_capacity_words, void *stream);
/* Synchronise and report device-side errors (FZ_ETIMEOUT, FZ_EINTERNAL). */
int fz_batch_sync(fz_batch_t batch, void *stream);
int fz_batch_destroy(fz_batch_t batch);

/* The exact layout of a batch before any output exists: word_offsets (host,
 * count + 1) and rows (host, count; may be NULL) receive what
 * fz_enumerate_batch will use for the same instances and options, and
 * *words_needed (may be NULL) the total.  Costs one fz_batch_create (the
 * counts come from the batch's own tables); callers that go on to enumerate
 * should keep a batch instead (fz_batch_create + fz_batch_layout).
 * Synchronises.  Errors: as fz_batch_create. */
int fz_plan_batch(const fz_instance_t *inst, int count, const fz_opts_t *opt,
                  uint64_t *word_offsets, uint64_t *rows, uint64_t *words_needed,
                  void *stream);

/* Measured choice of memos for batches (the memo depth, Section 3.1's
 * memoDim, and the memo layout).  A batch chooses per generator set the
 * deepest full memo whose estimated rows stay within cap_rows times the
 * instance's estimated rows (else a partial depth-3 memo for d >= 5, else
 * the closed form of the last two generators), and keeps full memos of
 * depth <= 3 in run order when run_order is set; both are per tuple width.
 * fz_batch_autotune times, on the device, the given instances of each width
 * >= 3 (up to 1024 of them, spread over the list) under cap_rows in
 * {0, 1/4, 1, 4, 16}
 * with run order on and off (rebuild + enumeration, mean of 3 after a
 * warm-up; candidates that choose the same memos are timed once).  The
 * widths' fastest choices need not combine well, so they are then applied
 * greedily on the whole batch of the given instances: starting from the
 * policy in force before the call, each width's fastest choice (widths in
 * decreasing order of their own gain) is tried on top of the choices kept
 * so far and kept only if the whole batch gets 1 % faster or more.  The
 * result is kept for later fz_batch_create calls on this device (with
 * opts.k = FZ_AUTO).  Up to `capacity` timed candidates go to `entries`
 * (host, may be NULL when capacity is 0), their number to *n_entries; the
 * whole-batch timings are the entries with d = 0 and cap_rows = -1, with
 * run_order = 0 for the starting policy and w after trying width w's
 * choice.  Synchronises.  Errors: as fz_batch_create. */
typedef struct fz_batch_tune_entry {
    int32_t d;          /* tuple width of the sample */
    int32_t run_order;  /* layout candidate: 1 = run order allowed */
    int32_t instances;  /* sampled instances */
    int32_t memos;      /* distinct memos built */
    double cap_rows;    /* depth candidate: memo rows per instance row */
    uint64_t rows;      /* output rows of the sample */
    uint64_t memo_rows; /* memo rows built */
    double build_ms;    /* rebuild: tables + memos (measured) */
    double enum_ms;     /* enumeration (measured) */
    double total_ms;
} fz_batch_tune_entry_t;
int fz_batch_autotune(const fz_instance_t *inst, int count, fz_batch_tune_entry_t *entries,
                      int capacity, int *n_entries, void *stream);
/* The policy in force for width d on the current device (measured by
 * fz_batch_autotune, else the hand-set default: cap_rows 4 for d >= 6, 1
 * below, run order on).  Either pointer may be NULL.  Errors: FZ_EINVAL. */
int fz_batch_policy(int32_t d, double *cap_rows, int32_t *run_order);
/* Forget the measured policy of the current device (back to the default). */
int fz_batch_policy_reset(void);

/* One-shot: create + enumerate + sync + destroy.  word_offsets (host,
 * count + 1, may be NULL) and *words_needed receive the layout.  Errors: as
 * above; FZ_ENOSPC when out_capacity_words is too small (nothing written). */
int fz_enumerate_batch(const fz_instance_t *inst, int count, const fz_opts_t *opt,
                       uint64_t *word_offsets, int32_t *out_dev,
                       uint64_t out_capacity_words, uint64_t *words_needed,
                       void *stream);

/* ------------------------------------------------------------------------
 * Serving: a request loop over generator sets kept resident on the device.
 *
 * fz_serve_register builds a set's plan once for every n <= n_max (count and
 * runs tables and memo depend on the generators only) and mirrors its count
 * row on the host, so fz_serve_submit knows the exact output bytes of a
 * query at once.  A background thread admits queued requests in arrival
 * order as soon as a slot (max_in_flight) and the exact bytes are free in the
 * output budget, and launches them on the next of `streams` CUDA streams:
 * requests that arrive while others run are admitted as slots and memory
 * free up, and their work overlaps on the GPU (continuous batching).  The
 * requests admitted together are one launch (see FZ_SERVE_PER_REQUEST).  A
 * result stays valid until fz_serve_release.  Times are seconds on the host
 * steady clock; t_done is stamped when the request's stream reaches it.
 * Each request in flight has its own device status word, read back with
 * the request: a device-side check that fails marks that request's status
 * FZ_EINTERNAL (or FZ_ETIMEOUT), not the server or other requests.
 * The paper serves no requests; this is the deployment layer around the
 * enumeration of Section 3.1.
 * ---------------------------------------------------------------------- */
typedef struct fz_serve_cfg {
    uint64_t memory_bytes;  /* device bytes for request outputs; 0 = a quarter
                               of the free memory at creation */
    int32_t max_in_flight;  /* requests on the device at once (slots) */
    int32_t streams;        /* CUDA streams the server launches on (grouped
                               mode: at most one group in flight on each) */
    int32_t max_queue;      /* queued requests before FZ_EAGAIN */
    int32_t flags;          /* 0 or FZ_SERVE_PER_REQUEST */
} fz_serve_cfg_t;

/* fz_serve_cfg_t.flags: launch every request on its own instead of in
 * groups.  By default (flags 0) the requests admitted in one pass of the
 * server loop are launched together: one launch of the batch enumeration
 * kernel with a range of work items per request, one transfer of their
 * parameters and one completion callback per group; requests of 2^22 rows
 * or more, whose plan's own kernel writes them faster, are launched with it
 * right after the group's kernel on the same stream. */
#define FZ_SERVE_PER_REQUEST 1

typedef struct fz_server_s *fz_server_t;

#define FZ_SERVE_DONE 0
#define FZ_SERVE_QUEUED 1
#define FZ_SERVE_RUNNING 2

typedef struct fz_result {
    int32_t status;          /* FZ_SERVE_DONE / QUEUED / RUNNING, or a negative fz_status
                                (FZ_ECANCELED, FZ_EINTERNAL, FZ_ETIMEOUT, ...) */
    int32_t d;
    uint64_t count;          /* rows */
    const int32_t *rows_dev; /* count * d int32 (when done), owned by the server */
    double t_submit, t_admit, t_done;
} fz_result_t;

typedef struct fz_serve_stats {
    uint64_t queued, admitted, completed;
    uint64_t bytes_in_use, bytes_budget;
    int32_t sets;
    int32_t last_error;
} fz_serve_stats_t;

/* Start a server on the current device.  Errors: FZ_EINVAL, FZ_ENOMEM, FZ_ECUDA. */
int fz_serve_create(const fz_serve_cfg_t *cfg, fz_server_t *srv);
/* Make generator set g (host, d entries) resident for n <= n_max.
 * Synchronous.  *set_id receives its index. */
int fz_serve_register(fz_server_t srv, const int32_t *g, int d, int32_t n_max,
                      int32_t *set_id);
/* Queue Z(n, set).  Errors: FZ_ENOTFOUND (set), FZ_EINVAL (n > n_max),
 * FZ_EAGAIN (queue full), FZ_ENOMEM (larger than the whole budget). */
int fz_serve_submit(fz_server_t srv, int32_t set_id, int32_t n, uint64_t *ticket);
/* Queue Z(n, g) by its generators (host, d entries, in the caller's order):
 * the request goes to a registered set with the same generators in the same
 * order and n_max >= n; when there is none, the set is first registered
 * (synchronously, with n_max = n) and later queries reuse it.  This is the
 * submit-by-instance form; fz_serve_submit with a set id skips the lookup.
 * Errors: those of fz_serve_register and fz_serve_submit. */
int fz_serve_submit_gens(fz_server_t srv, const int32_t *g, int d, int32_t n,
                         uint64_t *ticket);
/* Current state of a request (non-blocking). */
int fz_serve_poll(fz_server_t srv, uint64_t ticket, fz_result_t *result);
/* Block until the request is done, failed or cancelled (timeout_ms < 0: no
 * limit; FZ_EAGAIN on timeout; FZ_ENOTFOUND if another thread releases the
 * ticket meanwhile). */
int fz_serve_wait(fz_server_t srv, uint64_t ticket, int32_t timeout_ms,
                  fz_result_t *result);
/* Copy a finished request's rows into dst (host or device memory, at least
 * count * d int32 words).  Synchronises `stream`.  Errors: FZ_ENOTFOUND,
 * FZ_EAGAIN (not done), FZ_ENOSPC (capacity_words too small), the request's
 * own negative status if it failed or was cancelled, FZ_ECUDA. */
int fz_serve_copy(fz_server_t srv, uint64_t ticket, int32_t *dst, uint64_t capacity_words,
                  void *stream);
/* Free a finished, failed or cancelled request's output and forget its
 * ticket (FZ_EAGAIN while queued or running). */
int fz_serve_release(fz_server_t srv, uint64_t ticket);
/* Cancel a queued request: it leaves the queue without running, its status
 * becomes FZ_ECANCELED (release it as usual), and requests queued behind it
 * may be admitted at once.  A request already on the device is not stopped:
 * FZ_EAGAIN (wait for it, then release).  A finished request is left as it
 * is (FZ_OK).  Errors: FZ_ENOTFOUND, FZ_EAGAIN. */
int fz_serve_cancel(fz_server_t srv, uint64_t ticket);
int fz_serve_stats(fz_server_t srv, fz_serve_stats_t *stats);
/* Measurement utility (the paper has no counterpart): replays a request
 * stream against the server from native threads, so that a client's own
 * overhead does not bound the measured rate.  Request i (set set_ids[i],
 * element ns[i]) is submitted at arrival_s[i] seconds after the call starts
 * (busy wait; a full queue is retried); a second thread waits for the
 * requests in submission order and releases them.  latency_s[i] receives
 * t_done - t_submit, rows[i] (may be NULL) the request's row count, and
 * *span_s (may be NULL) the time from the first submission to the last
 * completion.  All arrays are host memory of `count` entries.  Returns when
 * every request is done.  Errors: FZ_EINVAL, those of fz_serve_submit, and
 * the status of a request that failed. */
int fz_serve_replay(fz_server_t srv, const int32_t *set_ids, const int32_t *ns,
                    const double *arrival_s, int count, double *latency_s, uint64_t *rows,
                    double *span_s);
/* Stop the loop, wait for running requests, free everything.  Requests still
 * queued are dropped. */
int fz_serve_destroy(fz_server_t srv);

/* ------------------------------------------------------------------------
 * One-shot calls.
 * ---------------------------------------------------------------------- */

/* fz_plan_create + fz_plan_enumerate + fz_plan_sync + fz_plan_destroy.
 * `opt` may be NULL (autotune).  Synchronises.  Errors: as those calls. */
int fz_enumerate(const int32_t *g, int d, int32_t n, const fz_opts_t *opt,
                 uint64_t rank_begin, uint64_t rank_end, int32_t *out_dev,
                 uint64_t out_capacity_rows, uint64_t *written, void *stream);

/* As fz_enumerate, but out_host is host memory: the asynchronous form of
 * the device-to-host buffer flushes of the paper's driver (Section 3.2).
 * Page-locked (pinned, mapped) memory is written by the enumeration kernel
 * itself over the host link, and so is pageable memory on devices that
 * reach it through the host's page tables (cudaDevAttrPageableMemoryAccess
 * and cudaDevAttrPageableMemoryAccessUsesHostPageTables both 1, as on
 * Grace-Blackwell).  Other pageable memory is filled in chunks: each chunk
 * is enumerated into one of three page-locked staging buffers while host
 * threads copy the previous, finished chunks into out_host.  Either way the
 * output may be larger than device memory.  The staging buffers (3 chunks)
 * are kept for later calls; a call that finds them in use by another
 * thread pins its own.  Synchronises.
 * Errors: those of fz_enumerate; FZ_ENOMEM (staging buffers). */
int fz_enumerate_host(const int32_t *g, int d, int32_t n, const fz_opts_t *opt,
                      uint64_t rank_begin, uint64_t rank_end, int32_t *out_host,
                      uint64_t out_capacity_rows, uint64_t *written,
                      void *stream);

/* fz_enumerate_host with the chunk size for pageable output given in rows:
 * chunk_rows > 0 always takes the staging ring with chunks of that many
 * rows; 0 = the default (direct writes where the device can make them,
 * else the ring with 128 MB chunks).  Ignored for page-locked output. */
int fz_enumerate_host_chunks(const int32_t *g, int d, int32_t n, const fz_opts_t *opt,
                             uint64_t rank_begin, uint64_t rank_end, int32_t *out_host,
                             uint64_t out_capacity_rows, uint64_t chunk_rows,
                             uint64_t *written, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* FZ_H */
