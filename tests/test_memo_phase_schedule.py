"""The phase fill of the memo build, restated on the CPU and checked against
the oracle (no GPU).

For a tail (t_0, ..., t_{k-1}) whose first generator is its least and whose
others are all at least 2 t_0, Z(m) = incr_0(Z(m - t_0)) ++ incr_1(...) ++
... (Lemma "disjlex" and Corollary "resultislex", Section 2.1): block 0 is
Z(m - t_0) with coordinate 0 raised, row for row, and every other block's
source lies L = min(t_1..t_{k-1}) or more elements back.  The whole-GPU fill
owns (class m mod t_0, word w) chains, one thread each for the whole fill,
chains ordered by 32-word block and then class, and fills phases of L
elements: pass A writes the block-0 words of chains alive at the phase start
from the thread's own last word (before waiting at the previous phase's
barrier), pass B the chains born in the phase (first word from the gather
map).  This test runs that schedule with a few simulated threads, checks the
dependencies it relies on (pass A reads only the thread's own writes, pass B
only earlier phases, every word written once) and requires the oracle's memo;
planted mistakes in the schedule must each be caught.
"""
import numpy as np
import pytest

import oracle

ZERO = None


def _map(tail, top, O, Ct):
    """Gather map: memo row -> (source row, incremented coordinate)."""
    k = len(tail)
    mp = {0: ZERO}
    for m in range(1, top):
        dst = O[m]
        for i in range(k):
            sm = m - tail[i]
            if sm < 0 or Ct[i][sm] == 0:
                continue
            ln = Ct[i][sm]
            src = O[sm + 1] - ln
            for r in range(ln):
                mp[dst + r] = (src + r, i)
            dst += ln
        assert dst == O[m + 1]
    return mp


def _phase_fill(tail, top, nthreads, cache=4, mistake=None):
    k = len(tail)
    t0 = tail[0]
    L = min(tail[1:]) if k > 1 else top
    if mistake == "long_phase":
        L += 1
    Ct = [[int(x) for x in row] for row in oracle.count_table(tail, top)]
    O = [0] * (top + 1)
    for m in range(top):
        O[m + 1] = O[m] + Ct[0][m]
    mp = _map(tail, top, O, Ct)

    def size(m):
        return O[m + 1] - O[m]

    R = [None] * (O[top] * k)
    writer = [None] * len(R)
    phase_of = [None] * len(R)
    ncl = min(t0, top)
    wc = max(size(e + ((top - 1 - e) // t0) * t0) for e in range(ncl)) * k
    nch = ncl * (-(-wc // 32)) * 32
    J = -(-nch // nthreads)
    last = {}
    for ph, ma in enumerate(range(0, top, L)):
        mb = min(ma + L, top)
        wp = max(size(m) for m in range(ma, mb)) * k
        for pas in "AB":
            for tid in range(nthreads):
                owner = tid
                if mistake == "remap" and ph % 2:
                    owner = (tid + 1) % nthreads  # chains move between threads
                for j in range(J):
                    ch = owner + j * nthreads
                    if ch >= nch:
                        break
                    q = ch >> 5
                    e, w = q % ncl, (q // ncl) * 32 + (ch & 31)
                    if w >= wp:
                        break
                    c = w % k
                    m1 = ma + (e - ma % t0) % t0
                    if m1 >= mb:
                        continue
                    ref = m1 if mistake == "alive_test" else m1 - t0
                    alive = m1 >= t0 and w < size(ref) * k
                    if (pas == "A") != alive:
                        continue
                    have, prev = False, None
                    if alive:
                        a = O[m1 - t0] * k + w
                        if j < cache and (tid, j) in last:
                            prev = last[(tid, j)]
                        else:
                            assert writer[a] == tid, "pass A read another thread's word"
                            prev = R[a]
                        have = True
                    for m in range(m1, mb, t0):
                        if w >= size(m) * k:
                            continue
                        if have:
                            hit = c == (1 if mistake == "coordinate" else 0)
                            v = prev + (1 if hit else 0)
                        else:
                            assert pas == "B"
                            ent = mp[O[m] + w // k]
                            if ent is ZERO:
                                v = 0
                            else:
                                sr, inc = ent
                                a = sr * k + c
                                assert R[a] is not None and phase_of[a] < ph, \
                                    "pass B read a word of this phase"
                                v = R[a] + (1 if c == inc else 0)
                        a = O[m] * k + w
                        assert R[a] is None, "word written twice"
                        R[a], writer[a], phase_of[a] = v, tid, ph
                        prev, have = v, True
                    if have and j < cache:
                        if mistake != "stale_cache" or (tid, j) not in last:
                            last[(tid, j)] = prev
    assert all(x is not None for x in R), "word never written"
    return np.asarray(O, dtype=np.uint64), np.asarray(R).reshape(-1, k)


CASES = [((4, 9, 10), 300, 64), ((3, 7, 8, 20), 200, 32), ((2, 5), 200, 96), ((5,), 40, 32),
         ((4, 20, 22, 31, 39), 200, 128), ((2, 4), 80, 32), ((3, 6, 6), 90, 64)]


@pytest.mark.parametrize("tail,top,nthreads", CASES)
def test_phase_schedule_matches_the_oracle(tail, top, nthreads):
    O, R = _phase_fill(tail, top, nthreads)
    ref_off, ref_rows = oracle.memo_csr(tail, top)
    assert np.array_equal(O, ref_off)
    assert np.array_equal(R, ref_rows)


@pytest.mark.parametrize("mistake", ["long_phase", "coordinate", "alive_test", "remap",
                                     "stale_cache"])
def test_planted_schedule_mistakes_are_caught(mistake):
    """A phase one element too long, the increment on the wrong coordinate,
    the alive test against the wrong element, chains that change threads
    between phases, a cached word not refreshed: each fails a dependency
    check or the comparison with the oracle on at least one case."""
    caught = False
    for tail, top, nthreads in CASES:
        try:
            O, R = _phase_fill(tail, top, nthreads, mistake=mistake)
            ref_off, ref_rows = oracle.memo_csr(tail, top)
            if not (np.array_equal(O, ref_off) and np.array_equal(R, ref_rows)):
                caught = True
        except (AssertionError, KeyError, TypeError, IndexError):
            caught = True
        if caught:
            break
    assert caught, mistake
