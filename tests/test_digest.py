"""The digest the full-size GPU tests compare with the oracle's, pinned on
the CPU: tests/gpu_checks.rows_digest over the oracle's own rows equals
oracle.digest (whole lists and rank windows), and oracle.digest_parallel
(subtrees of the first coordinate on several threads, each from its global
rank) equals the single-threaded walk."""
import random

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
from gpu_checks import rows_digest  # noqa: E402


def test_rows_digest_equals_the_oracle():
    rng = random.Random(7)
    for _ in range(120):
        d = rng.randint(1, 7)
        g = tuple(rng.randint(1, 15) for _ in range(d))
        n = rng.randint(0, 150)
        if oracle.count(g, n) > 100_000:
            continue
        ref = oracle.enumerate_desc(g, n)
        rows, dig = oracle.digest(g, n)
        assert rows == ref.shape[0]
        chunk = rng.choice([7, 64]) if rows <= 500 else rng.choice([rows // 3 + 1, 1 << 22])
        assert rows_digest(torch.from_numpy(ref), chunk=chunk) == dig
        if rows > 2:
            b, e = sorted(rng.sample(range(rows + 1), 2))
            _, wdig = oracle.digest(g, n, b, e)
            assert rows_digest(torch.from_numpy(np.ascontiguousarray(ref[b:e])), rank0=b) == wdig


def test_digest_is_order_sensitive():
    g, n = (3, 5, 7), 60
    ref = oracle.enumerate_desc(g, n)
    dig = rows_digest(torch.from_numpy(ref))
    swapped = ref.copy()
    swapped[[3, 4]] = swapped[[4, 3]]
    assert rows_digest(torch.from_numpy(swapped)) != dig
    bumped = ref.copy()
    bumped[10, 1] += 1
    assert rows_digest(torch.from_numpy(bumped)) != dig


def test_parallel_digest_equals_the_walk():
    for g, n in (((5, 8, 11, 14), 2000), ((56, 90, 96, 127, 146, 178), 4000), ((7,), 49)):
        assert oracle.digest_parallel(g, n, threads=4) == oracle.digest(g, n)
    rng = random.Random(8)
    for _ in range(150):
        d = rng.randint(1, 6)
        g = tuple(rng.randint(1, 15) for _ in range(d))
        n = rng.randint(0, 150)
        if oracle.count(g, n) > 100_000:
            continue
        assert oracle.digest_parallel(g, n, threads=rng.randint(1, 6)) == oracle.digest(g, n)
