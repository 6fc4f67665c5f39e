"""Oracle for exact lexicographic factorization-set enumeration (arXiv 2407.20474).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s ``cpu_baseline`` leg (and ``bench.py --impl reference``) may
import, call, link or execute anything in this package.  The product path
(the CUDA library and its Python binding) never does, and this package never
imports the product.  The two share no code: only the seeded input generators
(``paper_2407_20474_gb300.workloads``, which holds none of the method's
arithmetic) serve both.

What is computed here, each written from the paper:

* :func:`enumerate_desc` -- Z(n, g) = {a in N^d : sum a_i g_i = n} (Section 1)
  as the list sorted in descending lexicographic order (Lemma "disjlex" and
  its corollary, Section 2.1).  Plain C recursion (``fz_oracle.c``).
* :func:`count` / :func:`count_table` -- |Z(r, (g_j..g_d))| for all r, as the
  coefficients of the series prod_{i>=j} 1/(1 - x^{g_i}), i.e. the size of the
  sets of Section 1; the blocks |Z_{>=i}| of Section 2.3 are columns of it.
* :func:`unrank` -- the tuple at a given rank of the sorted list, found by
  skipping whole blocks of equal leading coordinates (their sizes from the
  table above).
* :func:`lex_lists` -- Algorithm "LexicographicFactorizationListsUpToElement"
  (Section 2.1), lists of Z(0..n) built by concatenating incr_i of the
  suffixes with zeros left of i.
* :func:`fwpar_lists` -- Algorithm "LexFacListsUpToElement_Factorizationwise
  Parallel" (Section 2.4), the same lists built from saved cardinalities
  (Section 2.3) with one copy-and-increment per (m, i), run sequentially.
* :func:`memo_csr` -- the memo of Section 3.1: Z(r, tail) for r < top as a
  CSR (offsets, rows), each r enumerated by the definition.
* :func:`nc_enumerate` / :func:`ncd_enumerate` -- the next-candidate walk
  (Algorithm 3.1 of Section 3) and its dynamic variant with low-dimension
  tabulation (Section 3.1), driven from the first candidate to the end of the
  stream.  Used only to pin the order on tiny inputs.

Readings of the paper that these functions adopt (where it is silent, garbled
or self-contradictory) are listed in the module docstrings of the functions
that use them.
"""
from __future__ import annotations

import ctypes
import os
from typing import List, Optional, Sequence, Tuple

import numpy as np

from . import build as _build

__all__ = [
    "enumerate_desc", "count", "count_table", "count_upto", "unrank",
    "lex_lists", "fwpar_lists", "memo_csr", "nc_enumerate", "ncd_enumerate",
    "sample_a1", "digest",
]

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build_oracle()
        lib = ctypes.CDLL(path)
        lib.fzo_enumerate.restype = ctypes.c_int64
        lib.fzo_enumerate.argtypes = [
            ctypes.POINTER(ctypes.c_int32), ctypes.c_int, ctypes.c_int64,
            ctypes.c_uint64, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int32),
            ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]
        lib.fzo_count.restype = ctypes.c_int64
        lib.fzo_count.argtypes = [ctypes.POINTER(ctypes.c_int32), ctypes.c_int,
                                  ctypes.c_int64]
        lib.fzo_sample.restype = ctypes.c_int
        lib.fzo_sample.argtypes = [
            ctypes.POINTER(ctypes.c_int32), ctypes.c_int, ctypes.c_int64,
            ctypes.POINTER(ctypes.c_int64), ctypes.c_int, ctypes.c_int,
            ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]
        lib.fzo_digest_subtrees.restype = ctypes.c_int
        lib.fzo_digest_subtrees.argtypes = [
            ctypes.POINTER(ctypes.c_int32), ctypes.c_int, ctypes.c_int64,
            ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_uint64), ctypes.c_int,
            ctypes.c_int, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]
        lib.fzo_lex_lists.restype = ctypes.c_int64
        lib.fzo_lex_lists.argtypes = [
            ctypes.POINTER(ctypes.c_int32), ctypes.c_int, ctypes.c_int64,
            ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_int32), ctypes.c_uint64]
        _lib = lib
    return _lib


def _gens(g: Sequence[int]) -> np.ndarray:
    arr = np.ascontiguousarray(np.asarray(g, dtype=np.int64))
    if arr.ndim != 1 or arr.size < 1:
        raise ValueError("need at least one generator")
    if (arr <= 0).any():
        raise ValueError("generators must be positive")
    return arr.astype(np.int32)


# ---------------------------------------------------------------------------
# The set itself (Section 1), in descending lexicographic order (Section 2.1).
# ---------------------------------------------------------------------------
def enumerate_desc(g: Sequence[int], n: int, rank_begin: int = 0,
                   rank_end: Optional[int] = None) -> np.ndarray:
    """Rows of Z(n, g) with rank in [rank_begin, rank_end), greatest first.

    Rank 0 is the lexicographically greatest tuple.  Returns an int32 array of
    shape (rows, d).  With ``rank_end=None`` the whole tail of the list is
    returned (its length is found by a first counting walk).
    """
    gg = _gens(g)
    d = gg.size
    if n < 0:
        return np.zeros((0, d), dtype=np.int32)
    lib = _load()
    gp = gg.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    if rank_end is None:
        rank_end = int(lib.fzo_count(gp, d, n))
    rows = max(0, int(rank_end) - int(rank_begin))
    out = np.zeros((rows, d), dtype=np.int32)
    if rows == 0:
        return out
    got = lib.fzo_enumerate(gp, d, n, int(rank_begin), int(rank_end),
                            out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                            None, None)
    if got < 0:
        raise ValueError("oracle rejected its arguments")
    return out[:got]


def digest(g: Sequence[int], n: int, rank_begin: int = 0,
           rank_end: Optional[int] = None) -> Tuple[int, int]:
    """(rows, order-sensitive digest) of the rows with rank in [begin, end)."""
    gg = _gens(g)
    lib = _load()
    total = ctypes.c_uint64(0)
    cs = ctypes.c_uint64(0)
    end = (1 << 64) - 1 if rank_end is None else int(rank_end)
    got = lib.fzo_enumerate(gg.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                            gg.size, n, int(rank_begin), end, None,
                            ctypes.byref(total), ctypes.byref(cs))
    return int(got), int(cs.value)


def sample_a1(g: Sequence[int], n: int, a1_values: Sequence[int],
              threads: int = 1) -> Tuple[int, int, int]:
    """Walk the subtrees of Z(n, g) whose first coordinate is in ``a1_values``.

    Each subtree is the plain recursion on one of ``threads`` POSIX threads.
    Returns (rows, digest, threads actually used).  Used to time the oracle on a
    bounded sample of a workload.
    """
    gg = _gens(g)
    vals = np.ascontiguousarray(np.asarray(a1_values, dtype=np.int64))
    lib = _load()
    rows = ctypes.c_uint64(0)
    cs = ctypes.c_uint64(0)
    used = lib.fzo_sample(gg.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                          gg.size, n,
                          vals.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                          int(vals.size), int(threads), ctypes.byref(rows),
                          ctypes.byref(cs))
    if used < 0:
        raise ValueError("oracle rejected its arguments")
    return int(rows.value), int(cs.value), int(used)


def digest_parallel(g: Sequence[int], n: int, threads: int = 1) -> Tuple[int, int]:
    """(rows, digest) of the whole of Z(n, g): the digest of ``digest`` (same
    value), computed by walking the subtree of each first coordinate a_1 on
    one of ``threads`` POSIX threads, each from its global rank.  The list is
    descending in a_1 and the subtree of a_1 = v holds |Z(n - v g_1, (g_2..g_d))|
    rows, so the subtree of v starts after those of every larger value."""
    gg = _gens(g)
    if gg.size == 1 or n < 0:
        return digest(g, n)
    T = count_table(gg[1:], n)[0]  # uint64 (exact: wrap-around is detected)
    g1 = int(gg[0])
    vals = list(range(n // g1, -1, -1))
    sizes = [int(T[n - v * g1]) for v in vals]
    first, acc = [], 0
    for c in sizes:
        first.append(acc)
        acc += c
    if acc >= 1 << 64:
        raise ValueError("more than 2^64 rows")
    # largest subtrees first, so the threads finish together
    order = sorted(range(len(vals)), key=lambda j: -sizes[j])
    v_arr = np.ascontiguousarray(np.array([vals[j] for j in order], dtype=np.int64))
    f_arr = np.ascontiguousarray(np.array([first[j] for j in order], dtype=np.uint64))
    lib = _load()
    rows = ctypes.c_uint64(0)
    cs = ctypes.c_uint64(0)
    used = lib.fzo_digest_subtrees(gg.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), gg.size,
                                   n, v_arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                   f_arr.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                   int(v_arr.size), int(threads), ctypes.byref(rows),
                                   ctypes.byref(cs))
    if used < 0:
        raise ValueError("oracle rejected its arguments")
    return int(rows.value), int(cs.value)


# ---------------------------------------------------------------------------
# Sizes: coefficients of prod 1/(1 - x^{g_i}).
# ---------------------------------------------------------------------------
def _times_geometric(series, gj: int):
    """Multiply a power series (list of Python ints) by 1/(1 - x^gj)."""
    out = list(series)
    for r in range(gj, len(out)):
        out[r] += out[r - gj]
    return out


def count_table(g: Sequence[int], n: int, exact: bool = False) -> List:
    """T[j][r] = |Z(r, (g_j, ..., g_d))| for j = 0..d (0-based), r = 0..n.

    T[d] is the series of the empty product (1 at r = 0).  Row j is row j+1
    times 1/(1 - x^{g_j}), which counts the ways to add any number of g_j's.
    With ``exact=False`` the rows are numpy uint64 arrays built with a strided
    cumulative sum per residue class modulo g_j (a library step); an overflow
    of 64 bits is detected (a cumulative sum that decreases) and the table is
    then recomputed with Python integers.  ``exact=True`` always uses Python
    integers (lists).
    """
    gg = [int(x) for x in _gens(g)]
    d = len(gg)
    if n < 0:
        raise ValueError("n must be >= 0")
    if exact:
        rows = [None] * (d + 1)
        rows[d] = [1] + [0] * n
        for j in range(d - 1, -1, -1):
            rows[j] = _times_geometric(rows[j + 1], gg[j])
        return rows
    rows = [None] * (d + 1)
    last = np.zeros(n + 1, dtype=np.uint64)
    last[0] = 1
    rows[d] = last
    for j in range(d - 1, -1, -1):
        src = rows[j + 1]
        cur = np.empty_like(src)
        gj = gg[j]
        for rho in range(min(gj, n + 1)):
            col = src[rho::gj]
            acc = np.cumsum(col, dtype=np.uint64)
            # a running sum of non-negative terms never decreases; a decrease
            # means the 64-bit sum wrapped around
            if acc.size > 1 and (acc[1:] < acc[:-1]).any():
                return count_table(g, n, exact=True)
            cur[rho::gj] = acc
        rows[j] = cur
    # Sanity guard against silent wrap-around: every entry of the top row must
    # be at least the corresponding entry below it (adding a generator only
    # adds factorizations).
    for j in range(d):
        if (rows[j] < rows[j + 1]).any():
            return count_table(g, n, exact=True)
    return rows


def count_upto(g: Sequence[int], n_max: int) -> np.ndarray:
    """|Z(r, g)| for r = 0..n_max as a uint64 array (object array on overflow)."""
    t = count_table(g, n_max)
    top = t[0]
    if isinstance(top, list):
        return np.array(top, dtype=object)
    return top


def count(g: Sequence[int], n: int) -> int:
    """|Z(n, g)| exactly (Python int)."""
    if n < 0:
        return 0
    t = count_table(g, n)
    return int(t[0][n])


# ---------------------------------------------------------------------------
# Tuple at a given rank.
# ---------------------------------------------------------------------------
def unrank(g: Sequence[int], n: int, rank: int, table=None) -> Tuple[int, ...]:
    """The tuple of rank ``rank`` (0 = greatest) of Z(n, g) in descending order.

    The tuples with a given first coordinate v form one contiguous run of the
    sorted list, of size |Z(n - v g_1, (g_2..g_d))|, and the runs come in the
    order v = floor(n/g_1), ..., 0.  Skipping whole runs fixes a_1; the same on
    the remaining coordinates fixes the rest.
    """
    gg = [int(x) for x in _gens(g)]
    d = len(gg)
    if table is None:
        table = count_table(gg, n)
    total = int(table[0][n])
    if not 0 <= rank < total:
        raise IndexError("rank %d outside [0, %d)" % (rank, total))
    a = [0] * d
    rem = n
    r = int(rank)
    for j in range(d - 1):
        gj = gg[j]
        vs = np.arange(rem // gj, -1, -1, dtype=np.int64)
        sub = table[j + 1]
        if isinstance(sub, list):
            sizes = [sub[rem - int(v) * gj] for v in vs]
            acc = 0
            for v, s in zip(vs, sizes):
                if r < acc + s:
                    a[j] = int(v)
                    r -= acc
                    break
                acc += s
            else:
                raise AssertionError("rank not found")
        else:
            sizes = sub[rem - vs * gj].astype(np.uint64)
            csum = np.cumsum(sizes, dtype=np.uint64)
            idx = int(np.searchsorted(csum, np.uint64(r), side="right"))
            a[j] = int(vs[idx])
            r -= 0 if idx == 0 else int(csum[idx - 1])
        rem -= a[j] * gj
    assert rem % gg[d - 1] == 0 and r == 0
    a[d - 1] = rem // gg[d - 1]
    return tuple(a)


# ---------------------------------------------------------------------------
# Algorithm "LexicographicFactorizationListsUpToElement" (Section 2.1).
# ---------------------------------------------------------------------------
def lex_lists(g: Sequence[int], n: int) -> List[List[Tuple[int, ...]]]:
    """F[m] for m = 0..n: the list of Z(m, g) built by the list recurrence.

    F[0] = [0].  For m > 0, F[m] concatenates, for i = 1..d with m - g_i >= 0,
    incr_i applied to those a in F[m - g_i] that are zero left of index i
    (isAllZeroesLeftOfIndex).  The membership test of the original set
    algorithm is relaxed to m - g_i >= 0 (Section 2, remark after the
    original algorithm), so gaps of the semigroup get empty lists.
    Pure Python: small n only.
    """
    gg = [int(x) for x in _gens(g)]
    d = len(gg)
    F: List[List[Tuple[int, ...]]] = [[] for _ in range(n + 1)]
    if n >= 0:
        F[0] = [tuple([0] * d)]
    for m in range(1, n + 1):
        Z: List[Tuple[int, ...]] = []
        for i in range(d):
            if m - gg[i] >= 0:
                for a in F[m - gg[i]]:
                    if all(a[j] == 0 for j in range(i)):
                        b = list(a)
                        b[i] += 1
                        Z.append(tuple(b))
        F[m] = Z
    return F


# ---------------------------------------------------------------------------
# Algorithm "LexFacListsUpToElement_FactorizationwiseParallel" (Section 2.4).
# ---------------------------------------------------------------------------
def fwpar_lists(g: Sequence[int], n: int) -> Tuple[np.ndarray, np.ndarray]:
    """Z(0..n, g) as a CSR (offsets uint64[n+2], rows int32[total, d]).

    Follows the factorizationwise algorithm with saved cardinalities: for each
    m and each i with m - g_i >= 0, the rows of Z(m - g_i) that are zero left
    of i -- a contiguous suffix of that list, starting after the blocks
    Z_{=j}, j < i -- are copied with coordinate i incremented to the running
    position of Z(m), and the size of the copied run is saved as
    card[m][i] = |Z_{=i}(m)|.

    Reading adopted for the initialisation ``cardinalities[0] = [1,...,1]``,
    which would make the suffix sum for m - g_i = 0 equal d - i + 1 instead
    of 1: Z(0) = [0] is treated as the footnote of Section 2.3 states it,
    |Z_{>=i}(0)| = 1 for every i with start index 0.  Each copy is one numpy
    slice (a library step); m and i are plain loops.
    """
    gg = [int(x) for x in _gens(g)]
    d = len(gg)
    card = np.zeros((n + 1, d), dtype=np.int64)      # |Z_{=i}(m)|
    sizes = np.zeros(n + 1, dtype=np.int64)
    lists: List[np.ndarray] = [None] * (n + 1)
    lists[0] = np.zeros((1, d), dtype=np.int32)
    sizes[0] = 1
    for m in range(1, n + 1):
        parts = []
        for i in range(d):
            src_m = m - gg[i]
            if src_m < 0:
                continue
            if src_m == 0:
                start, cnt = 0, 1
            else:
                start = int(card[src_m, :i].sum())
                cnt = int(card[src_m, i:].sum())
            if cnt == 0:
                continue
            block = lists[src_m][start:start + cnt].copy()
            block[:, i] += 1
            parts.append(block)
            card[m, i] = cnt
        lists[m] = (np.concatenate(parts, axis=0) if parts
                    else np.zeros((0, d), dtype=np.int32))
        sizes[m] = lists[m].shape[0]
    offsets = np.zeros(n + 2, dtype=np.uint64)
    offsets[1:] = np.cumsum(sizes).astype(np.uint64)
    rows = (np.concatenate(lists, axis=0) if n >= 0
            else np.zeros((0, d), dtype=np.int32))
    return offsets, rows.astype(np.int32)


# ---------------------------------------------------------------------------
# The memo of low-dimension tabulation (Section 3.1).
# ---------------------------------------------------------------------------
def memo_csr(tail: Sequence[int], top: int) -> Tuple[np.ndarray, np.ndarray]:
    """Memo[r] = Z(r, tail) in descending order for r = 0..top-1, as a CSR.

    Returns (offsets uint64[top+1], rows int32[total, k]).  Every Memo[r] is
    enumerated by the definition (:func:`enumerate_desc`).
    """
    tt = _gens(tail)
    k = tt.size
    parts = []
    offsets = np.zeros(max(top, 0) + 1, dtype=np.uint64)
    total = 0
    for r in range(max(top, 0)):
        rows = enumerate_desc(tt, r)
        parts.append(rows)
        total += rows.shape[0]
        offsets[r + 1] = total
    rows = (np.concatenate(parts, axis=0) if parts
            else np.zeros((0, k), dtype=np.int32))
    return offsets, rows


def lex_lists_c(tail: Sequence[int], top: int) -> Tuple[np.ndarray, np.ndarray]:
    """The memo CSR of :func:`memo_csr` by the single-threaded dynamic list
    algorithm of Section 2.1, in C (the CPU memo population the paper times
    beside its GPU one).  Returns (offsets uint64[top+1], rows int32[total, k])."""
    tt = _gens(tail)
    k = tt.size
    top = max(int(top), 0)
    cap = int(sum(int(x) for x in count_upto(tt, top - 1))) if top > 0 else 0
    offsets = np.zeros(top + 1, dtype=np.uint64)
    rows = np.zeros((max(cap, 1), k), dtype=np.int32)
    got = _load().fzo_lex_lists(tt.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), k, top,
                                offsets.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                rows.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), cap)
    if got < 0:
        raise ValueError("oracle rejected its arguments (%d)" % got)
    return offsets, rows[:got]


# ---------------------------------------------------------------------------
# The next-candidate walk (Algorithm 3.1, Section 3) and its dynamic variant
# with low-dimension tabulation (Section 3.1).
# ---------------------------------------------------------------------------
def _phi(a, g):
    return sum(x * y for x, y in zip(a, g))


def _initial_candidate(g, n):
    """First candidate (ceil(n/g_1), 0, ..., 0); valid iff g_1 divides n.

    The paper calls setInitialCandidate without defining it; this is the
    candidate the successor step itself produces for a prefix of length 0.
    """
    d = len(g)
    a = [0] * d
    a[0] = -(-n // g[0])
    return a, (n % g[0] == 0)


def _next_candidate(n, g, a, b, state):
    """One step of the lexicographically greatest next candidate (in place).

    ``state`` is a dict with keys ``valid`` and ``end``.  Readings: the search
    for the rightmost nonzero index runs over 1..d-1 (the text says it
    excludes the final index); ``b`` is the lower bound of the stream.
    """
    d = len(g)
    if state["end"]:
        return
    i = 0
    for j in range(1, d):            # 1-based j = 1..d-1
        if a[j - 1] > 0:
            i = j
    if i == 0:
        state["end"] = True
        return
    a[d - 1] = 0
    a[i - 1] -= 1
    p = n - _phi(a, g)
    m = p // g[i]
    r = p - m * g[i]
    state["valid"] = True
    if r != 0:
        m += 1
        state["valid"] = False
    a[i] = m
    if tuple(a) <= tuple(b):
        state["end"] = True


def nc_enumerate(g: Sequence[int], n: int) -> List[Tuple[int, ...]]:
    """Z(n, g) as produced by repeated next-candidate steps from the first
    candidate, keeping the candidates flagged valid (one worker, lower bound
    below every tuple).  Pure Python: tiny inputs only."""
    gg = [int(x) for x in _gens(g)]
    d = len(gg)
    a, valid = _initial_candidate(gg, n)
    b = tuple([-1] + [0] * (d - 1))
    out = []
    if valid:
        out.append(tuple(a))
    st = {"valid": valid, "end": False}
    while True:
        _next_candidate(n, gg, a, b, st)
        if st["end"]:
            break
        if st["valid"]:
            out.append(tuple(a))
    return out


def _next_candidate_dynamic(n, g, a, b, state, memo, memo_dim, top, outputs):
    """One step of the dynamic next candidate (in place).

    Readings: the rightmost nonzero index is searched over 1..d-1; the memo
    test uses p = n - phi(a) computed right after the decrement (the printed
    step tests p before defining it); Memo[p] exists for 0 <= p < top and any
    larger p takes the ordinary step.
    """
    d = len(g)
    if state["end"]:
        return
    i = 0
    for j in range(1, d):
        if a[j - 1] > 0:
            i = j
    if i == 0:
        state["end"] = True
        return
    a[d - 1] = 0
    a[i - 1] -= 1
    p = n - _phi(a, g)
    if memo_dim > 0 and i == d - memo_dim and p < top:
        prefix = tuple(a[:d - memo_dim])
        for row in memo[p]:
            outputs.append(prefix + tuple(row))
        state["valid"] = False
    else:
        m = p // g[i]
        r = p - m * g[i]
        state["valid"] = True
        if r != 0:
            m += 1
            state["valid"] = False
        a[i] = m
    if tuple(a) <= tuple(b):
        state["end"] = True


def ncd_enumerate(g: Sequence[int], n: int, memo_dim: int,
                  top: int) -> List[Tuple[int, ...]]:
    """Z(n, g) produced by repeated dynamic next-candidate steps.

    The memo holds Z(r, (g_{d-memo_dim+1}..g_d)) for r < top, each built with
    :func:`lex_lists` (the paper populates the memo with the dynamic
    algorithm).  Rows copied out of the memo and candidates flagged valid are
    collected in the order the steps produce them.  Pure Python: tiny inputs.
    """
    gg = [int(x) for x in _gens(g)]
    d = len(gg)
    memo = []
    if memo_dim > 0 and top > 0:
        memo = lex_lists(gg[d - memo_dim:], top - 1)
    a, valid = _initial_candidate(gg, n)
    b = tuple([-1] + [0] * (d - 1))
    out: List[Tuple[int, ...]] = []
    if valid:
        out.append(tuple(a))
    st = {"valid": valid, "end": False}
    while True:
        outputs: List[Tuple[int, ...]] = []
        _next_candidate_dynamic(n, gg, a, b, st, memo, memo_dim, top, outputs)
        out.extend(outputs)
        if st["end"]:
            break
        if st["valid"]:
            out.append(tuple(a))
    return out
