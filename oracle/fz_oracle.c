/*
 * fz_oracle.c -- plain CPU oracle for the factorization set
 *
 *     Z(n, (g_1..g_d)) = { a in N^d : sum_i a_i g_i = n }          (Section 1)
 *
 * listed in descending lexicographic order (a_1 first, then a_2, ...), the
 * order fixed by the disjoint recurrence (Lemma "disjlex") and its corollary
 * that concatenating the blocks incr_i(Z_{>=i}(n - g_i)) keeps the list
 * sorted (Section 2.1), and walked by the lexicographically greatest
 * next-candidate step (Algorithm 3.1 of Section 3).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline leg (and bench.py --impl reference) use it.  It shares no code,
 * header or table with the CUDA library.
 *
 * The enumeration is the definition written out: a depth-first recursion
 * that fixes a_1 = floor(n/g_1) down to 0, then a_2, ..., and at the last
 * coordinate keeps the tuple iff g_d divides what is left.  No counting
 * tables, no memo, no pruning beyond rem >= 0.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#define FZO_MAX_D 64

typedef struct {
    const int32_t *g;
    int d;
    int64_t a[FZO_MAX_D];
    /* rank window [begin, end) to copy out; rows outside it are counted only */
    uint64_t rank;
    uint64_t begin, end;
    int32_t *out;       /* row-major, d int32 per row, NULL = do not store */
    uint64_t written;
    uint64_t checksum;  /* order-sensitive digest of the emitted rows */
    int stop;           /* set once rank reaches end (no further row needed) */
} fzo_state;

/* One emitted row.  The digest mixes every coordinate with the row's rank so
 * that a permutation of rows changes it. */
static void fzo_emit(fzo_state *s)
{
    if (s->rank >= s->begin && s->rank < s->end) {
        if (s->out) {
            int32_t *row = s->out + (size_t)s->written * (size_t)s->d;
            for (int i = 0; i < s->d; ++i) row[i] = (int32_t)s->a[i];
        }
        uint64_t h = s->rank * 0x9E3779B97F4A7C15ULL;
        for (int i = 0; i < s->d; ++i) {
            h ^= (uint64_t)s->a[i] + 0x632BE59BD9B4E019ULL + (h << 6) + (h >> 2);
        }
        s->checksum += h;
        s->written += 1;
    }
    s->rank += 1;
    if (s->rank >= s->end) s->stop = 1;
}

/* Coordinates i..d-1 of the tuples with sum_{j>=i} a_j g_j = rem, greatest
 * a_i first (descending lexicographic order). */
static void fzo_rec(fzo_state *s, int i, int64_t rem)
{
    const int64_t gi = s->g[i];
    if (i == s->d - 1) {
        if (rem % gi == 0) {
            s->a[i] = rem / gi;
            fzo_emit(s);
        }
        return;
    }
    for (int64_t v = rem / gi; v >= 0 && !s->stop; --v) {
        s->a[i] = v;
        fzo_rec(s, i + 1, rem - v * gi);
    }
}

static int fzo_check(const int32_t *g, int d, int64_t n)
{
    if (!g || d < 1 || d > FZO_MAX_D || n < 0) return -1;
    for (int i = 0; i < d; ++i)
        if (g[i] <= 0) return -1;
    return 0;
}

/*
 * Rows of Z(n, g) with rank in [rank_begin, rank_end), rank 0 being the
 * lexicographically greatest tuple.  `out` (may be NULL) receives the rows
 * row-major.  Returns the number of rows copied, or -1 on bad arguments.
 * If `total` is non-NULL it receives |Z(n, g)| when the walk ran to the end
 * (rank_end == UINT64_MAX), else the number of ranks visited.
 * `checksum` (may be NULL) receives the order-sensitive digest.
 */
int64_t fzo_enumerate(const int32_t *g, int d, int64_t n, uint64_t rank_begin,
                      uint64_t rank_end, int32_t *out, uint64_t *total,
                      uint64_t *checksum)
{
    if (fzo_check(g, d, n)) return -1;
    fzo_state s;
    memset(&s, 0, sizeof s);
    s.g = g;
    s.d = d;
    s.begin = rank_begin;
    s.end = rank_end;
    s.out = out;
    if (rank_begin < rank_end) fzo_rec(&s, 0, n);
    if (total) *total = s.rank;
    if (checksum) *checksum = s.checksum;
    return (int64_t)s.written;
}

/* |Z(n, g)| by walking the whole set (the definition, no formula). */
int64_t fzo_count(const int32_t *g, int d, int64_t n)
{
    if (fzo_check(g, d, n)) return -1;
    fzo_state s;
    memset(&s, 0, sizeof s);
    s.g = g;
    s.d = d;
    s.begin = 0;
    s.end = UINT64_MAX;
    fzo_rec(&s, 0, n);
    return (int64_t)s.rank;
}

/* ---------------------------------------------------------------------------
 * Timing driver for the CPU baseline: the rows of Z(n, g) whose first
 * coordinate a_1 lies in a given list of values, each such subtree walked by
 * the same plain recursion on one of `nthreads` POSIX threads (the a_1 values
 * are handed out one at a time).  Rows are digested, not stored.
 * ------------------------------------------------------------------------- */
typedef struct {
    const int32_t *g;
    int d;
    int64_t n;
    const int64_t *a1;
    const uint64_t *first;  /* rank of each subtree's first row, or NULL (0) */
    int na1;
    int next;
    pthread_mutex_t mu;
    uint64_t rows;
    uint64_t checksum;
} fzo_pool;

static void *fzo_worker(void *arg)
{
    fzo_pool *p = (fzo_pool *)arg;
    uint64_t rows = 0, sum = 0;
    for (;;) {
        pthread_mutex_lock(&p->mu);
        int j = p->next++;
        pthread_mutex_unlock(&p->mu);
        if (j >= p->na1) break;
        int64_t v = p->a1[j];
        int64_t rem = p->n - v * (int64_t)p->g[0];
        if (rem < 0) continue;
        fzo_state s;
        memset(&s, 0, sizeof s);
        s.g = p->g;
        s.d = p->d;
        s.begin = 0;
        s.end = UINT64_MAX;
        s.rank = p->first ? p->first[j] : 0;
        s.a[0] = v;
        if (p->d == 1) {
            if (rem == 0) fzo_emit(&s);
        } else {
            fzo_rec(&s, 1, rem);
        }
        rows += s.written;
        sum += s.checksum;
    }
    pthread_mutex_lock(&p->mu);
    p->rows += rows;
    p->checksum += sum;
    pthread_mutex_unlock(&p->mu);
    return NULL;
}

static int fzo_pool_run(const int32_t *g, int d, int64_t n, const int64_t *a1_values,
                        const uint64_t *first, int na1, int nthreads, uint64_t *rows,
                        uint64_t *checksum)
{
    if (fzo_check(g, d, n) || na1 < 0 || (na1 && !a1_values)) return -1;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 1024) nthreads = 1024;
    fzo_pool p;
    memset(&p, 0, sizeof p);
    p.g = g;
    p.d = d;
    p.n = n;
    p.a1 = a1_values;
    p.first = first;
    p.na1 = na1;
    pthread_mutex_init(&p.mu, NULL);
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!th) return -1;
    int started = 0;
    for (int t = 0; t < nthreads; ++t) {
        if (pthread_create(&th[t], NULL, fzo_worker, &p) != 0) break;
        ++started;
    }
    if (started == 0) fzo_worker(&p);
    for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
    free(th);
    pthread_mutex_destroy(&p.mu);
    if (rows) *rows = p.rows;
    if (checksum) *checksum = p.checksum;
    return started == 0 ? 1 : started;
}

int fzo_sample(const int32_t *g, int d, int64_t n, const int64_t *a1_values,
               int na1, int nthreads, uint64_t *rows, uint64_t *checksum)
{
    return fzo_pool_run(g, d, n, a1_values, NULL, na1, nthreads, rows, checksum);
}

/*
 * The order-sensitive digest of fzo_enumerate over whole subtrees walked in
 * parallel: subtree j (a_1 = a1_values[j]) starts at global rank first[j],
 * which the caller takes from the sizes of the subtrees of the larger a_1
 * values (the list is descending, Lemma "disjlex").  The digest is a sum over
 * rows, so the subtrees may run in any order.  Returns as fzo_sample.
 */
int fzo_digest_subtrees(const int32_t *g, int d, int64_t n, const int64_t *a1_values,
                        const uint64_t *first, int na1, int nthreads, uint64_t *rows,
                        uint64_t *checksum)
{
    if (!first && na1) return -1;
    return fzo_pool_run(g, d, n, a1_values, first, na1, nthreads, rows, checksum);
}

/*
 * The memo lists Z(m, tail), m = 0..top-1, by the single-threaded dynamic
 * list algorithm of Section 2.1 (LexicographicFactorizationListsUpToElement):
 * F[0] = [0]; F[m] is the concatenation over i of incr_i(a) for the rows a
 * of F[m - t_i] whose coordinates left of i are all zero.  Each row is
 * tested one by one (no saved cardinalities).  offsets receives top + 1
 * entries; rows holds at most `capacity` rows of k int32.  Returns the row
 * count, -1 for bad arguments, -2 if the rows do not fit.
 */
int64_t fzo_lex_lists(const int32_t *tail, int k, int64_t top, uint64_t *offsets,
                      int32_t *rows, uint64_t capacity)
{
    if (k < 1 || k > FZO_MAX_D || top < 0 || !tail || !offsets) return -1;
    for (int i = 0; i < k; ++i)
        if (tail[i] < 1) return -1;
    uint64_t total = 0;
    offsets[0] = 0;
    for (int64_t m = 0; m < top; ++m) {
        if (m == 0) {
            if (capacity < 1 || !rows) return -2;
            for (int c = 0; c < k; ++c) rows[c] = 0;
            total = 1;
            offsets[1] = 1;
            continue;
        }
        for (int i = 0; i < k; ++i) {
            const int64_t src = m - tail[i];
            if (src < 0) continue;
            for (uint64_t r = offsets[src]; r < offsets[src + 1]; ++r) {
                const int32_t *a = rows + r * (uint64_t)k;
                int zero_left = 1;
                for (int j = 0; j < i; ++j)
                    if (a[j] != 0) {
                        zero_left = 0;
                        break;
                    }
                if (!zero_left) continue;
                if (total >= capacity) return -2;
                int32_t *b = rows + total * (uint64_t)k;
                for (int c = 0; c < k; ++c) b[c] = a[c] + (c == i ? 1 : 0);
                ++total;
            }
        }
        offsets[m + 1] = total;
    }
    return (int64_t)total;
}
