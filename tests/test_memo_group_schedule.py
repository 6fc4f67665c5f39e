"""The element-group batch memo build, restated on the CPU and checked
against the oracle (no GPU).

Z(m) = incr_0(Z_{>=0}(m - t_0)) ++ ... ++ incr_{k-1}(Z_{>=k-1}(m - t_{k-1}))
(Lemma "disjlex", Section 2.1), elementwise in batches of b = min(tail)
elements (Section 2.2).  In the batch build each warp owns a contiguous run
of a batch's elements and takes them G = floor(32 / k) at a time: lane j
describes block j mod k of element j div k (its length from the tail's count
table, its source the suffix Z_{>=i}(m - t_i)), a warp scan of the lengths
places the blocks, and a group of at most 1024 words is copied as one flat
range, each word finding its block by a binary search over the lanes' first
rows (five shuffle steps; lanes past the group hold an all-ones key);
larger groups copy block by block.  This test runs that schedule for a few
warps, checks that every word is written once from a source before the
batch, and requires the oracle's memo; planted mistakes must be caught.
"""
import numpy as np
import pytest

import oracle

ILP = 8
FLAT = 4 * 32 * ILP
KEY_NONE = 0xFFFFFFFF


def _group_build(tail, top, nwarps=16, flat=FLAT, mistake=None):
    k = len(tail)
    b = min(tail)
    Ct = [[int(x) for x in row] for row in oracle.count_table(tail, top)]
    O = [0] * (top + 1)
    for m in range(top):
        O[m + 1] = O[m] + Ct[0][m]
    R = [None] * (O[top] * k)
    G = 32 // k
    rstep, cstep = 32 // k, 32 % k
    for m0 in range(0, top, b):
        m1 = min(m0 + b, top)
        ne = m1 - m0
        writes = []
        for warp in range(nwarps):
            lo = m0 + (warp * ne) // nwarps
            hi = m0 + ((warp + 1) * ne) // nwarps
            for eb in range(lo, hi, G):
                ge = min(G, hi - eb)
                npair = ge * k
                lens, srcs, jis = [0] * 32, [0] * 32, [0] * 32
                for lane in range(32):
                    je, ji = divmod(lane, k)
                    jis[lane] = ji
                    if lane < npair:
                        sm = eb + je - tail[ji]
                        if sm >= 0:
                            lens[lane] = Ct[ji][sm]
                            srcs[lane] = O[sm + 1] - Ct[ji][sm]
                z = 1 if eb == 0 else 0
                incl = list(np.cumsum(lens))
                rbeg = O[eb] + z
                excl = [x - y for x, y in zip(incl, lens)]
                if mistake == "inclusive_scan":
                    excl = incl
                dsts = [rbeg + x for x in excl]
                assert rbeg + incl[31] == O[eb + ge], "blocks do not tile the group"
                if z:
                    writes += [(i, 0) for i in range(k)]
                W = (O[eb + ge] - rbeg) * k
                if W <= flat:
                    key = [dsts[l] if l < npair else KEY_NONE for l in range(32)]
                    for w0 in range(0, W, 32 * ILP):
                        for lane in range(32):
                            wl = w0 + lane
                            r, c = rbeg + wl // k, wl % k
                            for u in range(ILP):
                                p = 0
                                for st in (16, 8, 4, 2, 1):
                                    take = key[p + st] < r if mistake == "strict_search" \
                                        else key[p + st] <= r
                                    if take:
                                        p += st
                                if wl + 32 * u < W:
                                    sr = srcs[p] + (r - dsts[p])
                                    a = sr * k + c
                                    assert a < O[m0] * k and R[a] is not None, "source not ready"
                                    inc = 1 if c == jis[p] else 0
                                    writes.append((rbeg * k + wl + 32 * u, R[a] + inc))
                                r += rstep
                                c += cstep if mistake != "coordinate_step" else cstep + 1
                                if c >= k:
                                    c -= k
                                    r += 1
                else:
                    for j in range(npair):
                        ln = lens[j]
                        if ln == 0:
                            continue
                        i = j % k
                        for w in range(ln * k):
                            a = srcs[j] * k + w
                            assert a < O[m0] * k and R[a] is not None, "source not ready"
                            writes.append((dsts[j] * k + w, R[a] + (1 if w % k == i else 0)))
        for a, v in writes:
            assert R[a] is None, "word written twice"
            R[a] = v
    assert all(x is not None for x in R), "word never written"
    return np.asarray(O, dtype=np.uint64), np.asarray(R).reshape(-1, k)


CASES = [((3, 5, 7), 150, 16, FLAT), ((2, 3), 60, 4, FLAT), ((5, 8, 11, 14), 220, 16, 64),
         ((1, 1, 1), 25, 16, FLAT), ((7,), 60, 16, FLAT), ((37, 41, 43, 47), 500, 16, FLAT),
         ((3, 4, 5, 6, 7, 8), 45, 16, FLAT), ((140, 150, 160), 1000, 16, FLAT),
         ((2, 5), 40, 2, 32), ((4, 6, 9, 10), 300, 16, 0)]


@pytest.mark.parametrize("tail,top,nwarps,flat", CASES)
def test_group_schedule_matches_the_oracle(tail, top, nwarps, flat):
    O, R = _group_build(tail, top, nwarps, flat)
    ref_off, ref_rows = oracle.memo_csr(tail, top)
    assert np.array_equal(O, ref_off)
    assert np.array_equal(R, ref_rows)


def test_widest_tail():
    """k = 16: two elements a group, one lane per block."""
    tail = tuple(range(2, 18))
    O, R = _group_build(tail, 30)
    ref_off, ref_rows = oracle.memo_csr(tail, 30)
    assert np.array_equal(R, ref_rows)


@pytest.mark.parametrize("mistake", ["inclusive_scan", "strict_search", "coordinate_step"])
def test_planted_group_mistakes_are_caught(mistake):
    """Block starts from the inclusive scan, a search that skips a block
    starting exactly at the row, a wrong coordinate step: each fails a check
    or the comparison with the oracle on at least one case."""
    caught = False
    for tail, top, nwarps, flat in CASES:
        try:
            O, R = _group_build(tail, top, nwarps, flat, mistake=mistake)
            ref_off, ref_rows = oracle.memo_csr(tail, top)
            caught = not (np.array_equal(O, ref_off) and np.array_equal(R, ref_rows))
        except (AssertionError, IndexError, TypeError):
            caught = True
        if caught:
            break
    assert caught, mistake
