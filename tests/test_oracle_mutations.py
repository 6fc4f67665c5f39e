"""Planted mistakes: the oracle pins must catch plausible bugs.

Each mutant below is a copy of an oracle function with one deliberate slip of
the kinds a reader could miss (a dropped term, a wrong index, an off-by-one
bound, a reversed order, a transposed operand).  The checks of
``test_oracle_pins.py`` are run on each and must fail.  All of it is CPU-only.
"""
import pytest

import oracle
from test_oracle_pins import (brute_force, check_closed_forms, check_counts_small,
                              check_enumeration, check_table1, small_cases)


def _series_count(g, n, mutate):
    """|Z(n, g)| from the series prod 1/(1 - x^{g_i}) with a planted slip."""
    d = len(g)
    row = [1] + [0] * n
    for j in range(d - 1, -1, -1):
        if mutate == "drop_last_factor" and j == d - 1 and d > 1:
            continue
        gj = g[j + 1] if (mutate == "wrong_index" and j + 1 < d) else g[j]
        start = gj + 1 if mutate == "off_by_one" else gj
        out = list(row)
        for r in range(start, n + 1):
            out[r] += out[r - gj]
        row = out
    return row[n]


def _fails(check, *args):
    try:
        check(*args)
    except AssertionError:
        return True
    return False


@pytest.mark.parametrize("mutate", ["drop_last_factor", "wrong_index", "off_by_one"])
def test_count_mutants_are_caught(mutate):
    fn = lambda g, n: _series_count(g, n, mutate)
    caught = (_fails(check_counts_small, fn, small_cases(count=60))
              or _fails(check_closed_forms, fn) or _fails(check_table1, fn))
    assert caught
    # and the unmutated copy passes everything
    ok = lambda g, n: _series_count(g, n, None)
    check_counts_small(ok, small_cases(count=60))
    check_closed_forms(ok)


def _enum_ascending(g, n):
    return oracle.enumerate_desc(g, n)[::-1]


def _enum_skip_top(g, n):
    rows = oracle.enumerate_desc(g, n)
    return rows[rows[:, 0] != n // g[0]] if rows.size else rows


def _enum_transposed(g, n):
    # generators taken in reverse order, coordinates put back: same set, wrong order
    rows = oracle.enumerate_desc(tuple(reversed(g)), n)
    return rows[:, ::-1]


def _enum_swapped_coords(g, n):
    rows = oracle.enumerate_desc(g, n).copy()
    if rows.shape[1] > 1:
        rows[:, [0, 1]] = rows[:, [1, 0]]
    return rows


@pytest.mark.parametrize("mutant", [_enum_ascending, _enum_skip_top, _enum_transposed,
                                    _enum_swapped_coords])
def test_enumeration_mutants_are_caught(mutant):
    assert _fails(check_enumeration, mutant, small_cases(count=60))


def _unrank_wrong_table_row(g, n, rank, table):
    # looks up the run sizes one level too high
    d = len(g)
    a = [0] * d
    rem, r = n, rank
    for j in range(d - 1):
        for v in range(rem // g[j], -1, -1):
            s = int(table[j][rem - v * g[j]])
            if r < s:
                a[j] = v
                break
            r -= s
        rem -= a[j] * g[j]
    a[d - 1] = rem // g[d - 1]
    return tuple(a)


def test_unrank_mutant_is_caught():
    g, n = (5, 8, 11, 14), 200
    rows = oracle.enumerate_desc(g, n)
    T = oracle.count_table(g, n)
    bad = [r for r in range(rows.shape[0])
           if _unrank_wrong_table_row(g, n, r, T) != tuple(int(v) for v in rows[r])]
    assert bad
    good = [r for r in range(rows.shape[0])
            if oracle.unrank(g, n, r, T) != tuple(int(v) for v in rows[r])]
    assert not good


def test_brute_force_reference_is_not_the_oracle():
    # the brute-force reference enumerates the whole box; sanity-check it on a
    # hand-countable case: 2a + 3b = 12 -> (6,0), (3,2), (0,4)
    assert brute_force((2, 3), 12) == [(6, 0), (3, 2), (0, 4)]
