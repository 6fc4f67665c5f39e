"""Pins for the oracle: checks against what the paper and the mathematics fix.

Each check is a function taking the implementation under test, so that
``test_oracle_mutations.py`` can run the same checks on deliberately broken
copies of the oracle and show that they fail.

* brute force over the box prod [0, floor(n/g_i)], filtered by the defining
  equation of Z(n, g) (Section 1) and sorted descending (Section 2.1);
* closed forms: d = 1; g = (1,...,1) (stars and bars); g = (1, 2);
  Popoviciu's formula for two coprime generators;
* the num_results column of Table 1 (22 of its 23 distinct (d, n) rows);
* invariants: every row sums to n, strictly descending order, the blocks
  Z_{=i}(n) = incr_i(Z_{>=i}(n - g_i)) in the order of Lemma "disjlex";
* the paper's own algorithms (Algorithm 3.1's next-candidate walk, its
  dynamic variant of Section 3.1, the list algorithm of Section 2.1 and the
  factorizationwise algorithm of Section 2.4) give the same lists.
"""
import itertools
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


# ---------------------------------------------------------------------------
# independent references (no oracle code)
# ---------------------------------------------------------------------------
def brute_force(g, n):
    """All tuples of the box with sum a_i g_i == n, sorted descending."""
    ranges = [range(n // x + 1) for x in g]
    rows = [t for t in itertools.product(*ranges)
            if sum(a * b for a, b in zip(t, g)) == n]
    rows.sort(reverse=True)
    return rows


def popoviciu(a, b, n):
    """Number of (x, y) >= 0 with a x + b y = n for coprime a, b."""
    ap = pow(a, -1, b)       # a * ap == 1 (mod b)
    bp = pow(b, -1, a)       # b * bp == 1 (mod a)
    frac = lambda q: q - math.floor(q)
    v = Fraction(n, a * b) - frac(Fraction(bp * n, a)) - frac(Fraction(ap * n, b)) + 1
    assert v.denominator == 1
    return int(v)


def table1_rows():
    rows = []
    with open(os.path.join(HERE, "golden", "table1_counts.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            rows.append((int(parts[0]), int(parts[1]), int(parts[2]),
                         int(parts[3]), len(parts) > 4 and parts[4] == "x"))
    return rows


TABLE1_G = (13, 37, 38, 40, 41, 42, 43, 44, 45)


def small_cases(seed=7, count=160):
    rng = np.random.Generator(np.random.PCG64(seed))
    cases = [((1,), 0), ((1,), 5), ((2,), 5), ((3,), 9), ((2, 2), 6),
             ((4, 6), 14), ((4, 6), 15), ((1, 1, 1), 6), ((5, 3, 2), 17),
             ((7, 7, 7), 21), ((2, 3, 5, 7), 30), ((3, 5), 0), ((6, 10, 15), 60)]
    while len(cases) < count:
        d = int(rng.integers(1, 6))
        g = tuple(int(x) for x in rng.integers(1, 13, size=d))
        n = int(rng.integers(0, 61))
        box = 1
        for x in g:
            box *= n // x + 1
        if box > 300_000:
            continue
        cases.append((g, n))
    return cases


# ---------------------------------------------------------------------------
# reusable checks
# ---------------------------------------------------------------------------
def check_enumeration(enum_fn, cases):
    for g, n in cases:
        got = [tuple(int(v) for v in r) for r in enum_fn(g, n)]
        assert got == brute_force(g, n), (g, n)


def check_counts_small(count_fn, cases):
    for g, n in cases:
        assert count_fn(g, n) == len(brute_force(g, n)), (g, n)


def check_closed_forms(count_fn):
    for g in (1, 2, 3, 7):
        for n in range(0, 40):
            assert count_fn((g,), n) == (1 if n % g == 0 else 0)
    for d in range(1, 6):
        for n in (0, 1, 5, 17, 40):
            assert count_fn((1,) * d, n) == math.comb(n + d - 1, d - 1)
    for n in range(0, 200, 7):
        assert count_fn((1, 2), n) == n // 2 + 1
    for a, b in ((3, 5), (4, 9), (7, 11), (13, 37), (56, 93)):
        if math.gcd(a, b) != 1:
            continue
        for n in list(range(0, 120)) + [1000, 4321, 99991]:
            assert count_fn((a, b), n) == popoviciu(a, b, n), (a, b, n)


def check_table1(count_fn):
    for d, _k, n, num, excluded in table1_rows():
        if excluded:
            continue
        assert count_fn(TABLE1_G[:d], n) == num, (d, n)


def check_invariants(enum_fn, count_fn, g, n):
    rows = np.asarray(enum_fn(g, n), dtype=np.int64)
    d = len(g)
    assert rows.shape == (count_fn(g, n), d)
    if rows.shape[0] == 0:
        return
    assert (rows >= 0).all()
    assert (rows @ np.asarray(g, dtype=np.int64) == n).all()
    # strictly descending lexicographic order
    diff = rows[:-1] - rows[1:]
    nz = diff != 0
    assert nz.any(axis=1).all(), "duplicate rows"
    first = nz.argmax(axis=1)
    assert (diff[np.arange(diff.shape[0]), first] > 0).all(), "not descending"
    # blocks Z_{=i}(n) = incr_i(Z_{>=i}(n - g_i)) in the order i = 1..d
    lead = (rows != 0).argmax(axis=1)
    if n > 0:
        assert (np.diff(lead) >= 0).all()
        for i in range(d):
            block = rows[lead == i]
            assert block.shape[0] == (count_fn(g[i:], n - g[i]) if n - g[i] >= 0 else 0)
            if block.shape[0]:
                back = block.copy()
                back[:, i] -= 1
                assert (back[:, :i] == 0).all()
                assert (back @ np.asarray(g, dtype=np.int64) == n - g[i]).all()
    if n % g[0] == 0:
        assert tuple(rows[0]) == (n // g[0],) + (0,) * (d - 1)


# ---------------------------------------------------------------------------
# tests on the oracle itself
# ---------------------------------------------------------------------------
def test_enumerate_matches_brute_force():
    check_enumeration(oracle.enumerate_desc, small_cases())


def test_count_matches_brute_force():
    check_counts_small(oracle.count, small_cases())


def test_count_closed_forms():
    check_closed_forms(oracle.count)


def test_count_exact_path_matches_fast_path():
    for g, n in (((13, 37, 38), 5000), ((3, 5, 7, 11), 700), ((1, 1, 2), 300)):
        fast = oracle.count_table(g, n)
        slow = oracle.count_table(g, n, exact=True)
        for a, b in zip(fast, slow):
            assert [int(x) for x in a] == b


def test_count_overflow_falls_back_to_exact():
    # |Z(n, (1,)*8)| = C(n+7, 7) exceeds 2^64 at n = 2^11.
    n = 2100
    assert oracle.count((1,) * 8, n) == math.comb(n + 7, 7)
    assert math.comb(n + 7, 7) > 2**64


def test_table1_counts():
    check_table1(oracle.count)


def test_table1_row_4_15000():
    """The paper prints 779252 for Z(15000, (13,37,38,40)).  Count it without
    the oracle: for every (a1, a2, a3) in the box, a4 is forced."""
    g = (13, 37, 38, 40)
    n = 15000
    total = 0
    a3 = np.arange(n // 38 + 1, dtype=np.int64)
    for a1 in range(n // 13 + 1):
        for a2 in range((n - 13 * a1) // 37 + 1):
            rem = n - 13 * a1 - 37 * a2 - 38 * a3
            total += int(((rem >= 0) & (rem % 40 == 0)).sum())
    assert total == 779257
    assert oracle.count(g, n) == total


def test_config1_count_by_brute_force():
    g, n = (5, 8, 11, 14), 500
    a = np.arange(n // 5 + 1)[:, None, None]
    b = np.arange(n // 8 + 1)[None, :, None]
    c = np.arange(n // 11 + 1)[None, None, :]
    rem = n - 5 * a - 8 * b - 11 * c
    total = int(((rem >= 0) & (rem % 14 == 0)).sum())
    assert total == 3783
    assert oracle.count(g, n) == 3783
    assert len(oracle.enumerate_desc(g, n)) == 3783


@pytest.mark.parametrize("g,n", [((5, 8, 11, 14), 500), ((13, 37, 38, 40), 5000),
                                 ((3, 5, 7, 11, 13), 300), ((2, 2, 3), 150),
                                 ((4, 6, 10), 301), ((6, 10, 15), 600),
                                 ((17,), 340), ((1, 1, 1, 1), 40)])
def test_invariants(g, n):
    check_invariants(oracle.enumerate_desc, oracle.count, g, n)


def test_next_candidate_walk_matches():
    for g, n in small_cases(seed=11, count=60):
        assert oracle.nc_enumerate(g, n) == brute_force(g, n), (g, n)


def test_dynamic_next_candidate_matches_every_memo_dim_and_top():
    rng = np.random.Generator(np.random.PCG64(5))
    for g, n in small_cases(seed=13, count=40):
        ref = brute_force(g, n)
        d = len(g)
        for k in range(0, d + 1):
            for top in (0, 1, int(rng.integers(0, n + 2)), n + 1):
                assert oracle.ncd_enumerate(g, n, k, top) == ref, (g, n, k, top)


def test_list_algorithms_match_definition():
    for g, n in (((3, 5, 7), 60), ((2, 2, 5), 40), ((4, 6), 50), ((1, 3, 4, 9), 45),
                 ((5,), 30)):
        F = oracle.lex_lists(g, n)
        off, rows = oracle.fwpar_lists(g, n)
        for m in range(n + 1):
            ref = [tuple(int(v) for v in r) for r in oracle.enumerate_desc(g, m)]
            assert F[m] == ref, (g, m)
            seg = [tuple(int(v) for v in r) for r in rows[int(off[m]):int(off[m + 1])]]
            assert seg == ref, (g, m)


def test_c_lex_lists_match_definition():
    """The C single-threaded dynamic list build equals the definition."""
    for tail, top in (((4, 9, 10), 80), ((2, 2, 5), 41), ((7,), 50), ((1, 3, 4, 9), 46),
                      ((13, 37, 38), 300), ((6, 4), 61), ((3, 5, 7), 0), ((3, 5, 7), 1)):
        off, rows = oracle.lex_lists_c(tail, top)
        ref_off, ref_rows = oracle.memo_csr(tail, top)
        assert np.array_equal(off, ref_off), tail
        assert np.array_equal(rows, ref_rows), tail


def test_memo_csr_matches_brute_force():
    tail = (4, 9, 10)
    off, rows = oracle.memo_csr(tail, 50)
    assert off.shape == (51,)
    for r in range(50):
        seg = [tuple(int(v) for v in x) for x in rows[int(off[r]):int(off[r + 1])]]
        assert seg == brute_force(tail, r)


def test_unrank_matches_enumeration():
    for g, n in (((5, 8, 11, 14), 500), ((3, 5, 7), 90), ((2, 2, 3), 40),
                 ((7,), 49), ((1, 1, 1, 1, 1), 9)):
        rows = oracle.enumerate_desc(g, n)
        T = oracle.count_table(g, n)
        for r in range(rows.shape[0]):
            assert oracle.unrank(g, n, r, T) == tuple(int(v) for v in rows[r])


def test_unrank_exact_table_path():
    g, n = (5, 8, 11, 14), 200
    rows = oracle.enumerate_desc(g, n)
    T = oracle.count_table(g, n, exact=True)
    for r in range(0, rows.shape[0], 7):
        assert oracle.unrank(g, n, r, T) == tuple(int(v) for v in rows[r])


def test_rank_window_and_digest():
    g, n = (5, 8, 11, 14), 500
    full = oracle.enumerate_desc(g, n)
    part = oracle.enumerate_desc(g, n, 100, 250)
    assert (part == full[100:250]).all()
    rows, h = oracle.digest(g, n)
    assert rows == full.shape[0]
    rows2, h2 = oracle.digest(g, n, 0, 3783)
    assert (rows2, h2) == (rows, h)
    # a_1-subtree sampling sees exactly the rows with that leading value
    vals = [100, 50, 7, 0]
    got, _, used = oracle.sample_a1(g, n, vals, threads=2)
    assert got == int(np.isin(full[:, 0], vals).sum())
    assert used >= 1


def test_empty_and_degenerate():
    assert oracle.count((2, 4), 7) == 0
    assert oracle.enumerate_desc((2, 4), 7).shape == (0, 2)
    assert oracle.enumerate_desc((3, 5, 7), 0).tolist() == [[0, 0, 0]]
    assert oracle.count((3, 5, 7), 0) == 1
    with pytest.raises(ValueError):
        oracle.enumerate_desc((0, 3), 5)
