"""The run-order memo layout and the run walk, restated on the CPU and
checked against the oracle (no GPU).

For a full memo of depth K under lam = d - K - 1 walked coordinates, the
rows of the elements p = c, c + g_lam, c + 2 g_lam, ... of each residue
class c mod g_lam are stored one after another (classes in increasing
order), each row as (p div g_lam, the K memo words).  The subtree of a
prefix with remainder r over a_lam (a_lam from r div g_lam down to 0, each
followed by Memo[r - a_lam g_lam], the tabulated tail of Section 3.1) is
then the contiguous range [cls_beg[r mod g_lam], + C[lam][r]), and element
p starts at cls_beg[c] + C[lam][p] - C[lam + 1][p].  A pair memo (K = 2,
no table) holds the progression a_{d-2} = a_top - o h1 of the last two
generators.  This test builds the layout from those formulas, walks it the
way the run copy does (prefix by prefix in descending order, any rank
window), and requires the oracle's list: it pins the index arithmetic the
kernels use, so a change to it can be checked here before it runs on a GPU.
"""
import math
import random

import numpy as np

import oracle


def _pair_params(g, h):
    e = math.gcd(g, h)
    h1 = h // e
    inv = pow(g // e, -1, h1) if h1 > 1 else 0
    return e, h1, inv


def _layout(g, n, K, pair):
    d = len(g)
    lam = d - K - 1
    C = [[int(v) for v in row] for row in oracle.count_table(g, n, exact=True)]
    gl = g[lam]
    G = min(gl, n + 1)
    cls = [0] * (G + 1)
    for c in range(G):
        last = c + ((n - c) // gl) * gl
        cls[c + 1] = cls[c] + C[lam][last]
    rows = [None] * cls[G]
    if not pair:
        O, R = oracle.memo_csr(g[d - K:], n + 1)
        O = [int(x) for x in O]
        R = np.asarray(R).reshape(-1, K)
        assert O[n + 1] == cls[G]
    else:
        t0, t1 = g[d - 2], g[d - 1]
        e, h1, inv = _pair_params(t0, t1)
        # the lattice points under t0 x + t1 y <= n
        assert cls[G] == sum((n - t0 * x) // t1 + 1 for x in range(n // t0 + 1))
    for p in range(n + 1):
        q, c = divmod(p, gl)
        cnt = C[lam + 1][p]
        dst = cls[c] + C[lam][p] - cnt
        if pair:
            body = []
            if p % e == 0:
                astar = (p // e) % h1 * inv % h1 if h1 > 1 else 0
                q0 = p // t0
                if q0 >= astar:
                    atop = q0 - (q0 - astar) % h1
                    body = [(atop - o * h1, (p - (atop - o * h1) * t0) // t1)
                            for o in range(atop // h1 + 1)]
        else:
            body = [tuple(int(v) for v in R[i]) for i in range(O[p], O[p + 1])]
        assert len(body) == cnt, (g, n, K, p)
        for o, words in enumerate(body):
            assert rows[dst + o] is None
            rows[dst + o] = (q,) + tuple(words)
    assert all(r is not None for r in rows)
    return C, cls, rows


def _find_child(C, g, j, rem, R):
    before = 0
    for v in range(rem // g[j], -1, -1):
        k = C[j + 1][rem - v * g[j]]
        if R < before + k:
            return v, before
        before += k
    raise AssertionError("rank past the subtree")


def _walk(g, n, K, C, cls, rows, row0, row1):
    """Rows [row0, row1) by the run walk: unrank the first row to a
    lam-prefix and an offset in its run, copy runs, step to the next
    prefix (decrement the deepest positive coordinate, reset the later
    ones to their maxima)."""
    d = len(g)
    lam = d - K - 1
    a = [0] * lam
    rem, R = n, row0
    for j in range(lam):
        v, before = _find_child(C, g, j, rem, R)
        a[j], R, rem = v, R - before, rem - v * g[j]
    off, left, out = R, row1 - row0, []
    while True:
        run = C[lam][rem]
        if off < run:
            vmax, c = divmod(rem, g[lam])
            take = min(run - off, left)
            for m in rows[cls[c] + off:cls[c] + off + take]:
                out.append(tuple(a) + (vmax - m[0],) + m[1:])
            left -= take
            if left == 0:
                return out
        off = 0
        jj = max(j for j in range(lam) if a[j] > 0)
        rr = n
        for j in range(lam):
            if j == jj:
                a[j] -= 1
            elif j > jj:
                a[j] = rr // g[j]
            rr -= a[j] * g[j]
        rem = rr


def test_run_order_layout_and_walk_match_the_oracle():
    rng = random.Random(5)
    done = 0
    while done < 200:
        d = rng.randint(3, 8)
        pair = d >= 4 and rng.random() < 0.5
        # depth 1..3 as built (one int4 per row); deeper memos keep the
        # same layout with wider rows
        K = 2 if pair else rng.randint(1, d - 2)
        g = tuple(rng.randint(1, 12) for _ in range(d))
        n = rng.randint(0, 70 if d <= 5 else 40)
        ref = oracle.enumerate_desc(g, n)
        if len(ref) == 0:
            continue
        C, cls, rows = _layout(g, n, K, pair)
        cuts = sorted({0, len(ref)} | {rng.randint(0, len(ref)) for _ in range(4)})
        got = []
        for r0, r1 in zip(cuts, cuts[1:]):
            got += _walk(g, n, K, C, cls, rows, r0, r1)
        assert np.array_equal(np.array(got, dtype=np.int64).reshape(-1, d),
                              ref.astype(np.int64)), (g, n, K, pair)
        done += 1


def _closed_rows(tail, p):
    """Rows of Z(p, tail), depth 1 or 2, from the tail's closed form as the
    batch's run-order build writes them: depth 1, the row p / t when t
    divides p; depth 2, the pair progression a = a_top, a_top - h1, ... with
    the last coordinate (p - a t0) / t1."""
    K = len(tail)
    if K == 1:
        return [(p // tail[0],)] if p % tail[0] == 0 else []
    t0, t1 = tail
    e, h1, inv = _pair_params(t0, t1)
    if p % e:
        return []
    astar = (p // e) % h1 * inv % h1 if h1 > 1 else 0
    q0 = p // t0
    if q0 < astar:
        return []
    atop = q0 - (q0 - astar) % h1
    return [(atop - o * h1, (p - (atop - o * h1) * t0) // t1) for o in range(atop // h1 + 1)]


def test_closed_form_tail_rows_match_the_memo():
    """The closed forms of tails of depth 1 and 2 (what the batch writes in
    run order instead of building an element-order memo) give every
    element's list of the oracle's memo, and the row totals the host
    allocates for them are the memo's size."""
    rng = random.Random(11)
    for _ in range(150):
        K = rng.randint(1, 2)
        tail = tuple(rng.randint(1, 30) for _ in range(K))
        top = rng.randint(1, 400)
        O, R = oracle.memo_csr(tail, top)
        R = np.asarray(R).reshape(-1, K)
        for p in range(top):
            got = _closed_rows(tail, p)
            want = [tuple(int(v) for v in R[i]) for i in range(int(O[p]), int(O[p + 1]))]
            assert got == want, (tail, p)
        n = top - 1
        if K == 1:
            total = n // tail[0] + 1
        else:
            t0, t1 = tail
            total = sum((n - t0 * x) // t1 + 1 for x in range(n // t0 + 1))
        assert total == int(O[top]), (tail, top)
