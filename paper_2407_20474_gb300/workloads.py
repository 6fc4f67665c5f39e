"""Seeded synthetic workloads for the factorization-set path.

This module draws generator sets, element targets and request streams from a
seed.  It holds none of the method's arithmetic: where a workload is defined
by a size ("the smallest n with |Z(n)| >= T"), the caller passes in its own
counting function and :func:`find_n` only searches the values it returns.
Both the oracle side (tests) and the CUDA side (bench) use these generators.

The paper's only workload family is generators (13, 37, 38, 40, ..., 45)
(Table 1); it names no dataset.  The configurations below are synthetic
stand-ins with the shapes stated beside each function.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Callable, List, Sequence, Tuple

import numpy as np

# Generators of the paper's runtime table: the first d of these (Table 1).
TABLE1_GENERATORS = (13, 37, 38, 40, 41, 42, 43, 44, 45)


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _gcd_all(values: Sequence[int]) -> int:
    g = 0
    for v in values:
        g = math.gcd(g, int(v))
    return g


def draw_generators(rng: np.random.Generator, d: int, lo: int, hi: int,
                    distinct: bool = True, sort: bool = True) -> Tuple[int, ...]:
    """d generators uniform in [lo, hi], redrawn until their gcd is 1.

    ``distinct`` redraws sets with repeated values; ``sort`` returns them in
    ascending order (the order fixes the lexicographic order of the output).
    """
    if d == 1:
        return (1,) if lo <= 1 <= hi else (int(rng.integers(lo, hi + 1)),)
    while True:
        g = [int(x) for x in rng.integers(lo, hi + 1, size=d)]
        if distinct and len(set(g)) != d:
            continue
        if _gcd_all(g) != 1:
            continue
        return tuple(sorted(g)) if sort else tuple(g)


def find_n(counts_upto: Callable[[Sequence[int], int], Sequence[int]],
           g: Sequence[int], target: int, n_hint: int = 64) -> int:
    """Smallest n with counts_upto(g, N)[n] >= target.

    ``counts_upto(g, N)`` must return |Z(r, g)| for r = 0..N (any exact
    counting implementation).  N starts at ``n_hint`` and doubles until some
    entry reaches the target.
    """
    n_max = max(1, int(n_hint))
    while True:
        c = counts_upto(g, n_max)
        arr = np.asarray([int(x) for x in c], dtype=object) \
            if not isinstance(c, np.ndarray) or c.dtype == object else c
        hits = np.nonzero(arr >= target)[0]
        if hits.size:
            return int(hits[0])
        n_max *= 2
        if n_max > 2**31 - 1:
            raise ValueError("target not reached below 2^31")


# ---------------------------------------------------------------------------
# Configurations.
# ---------------------------------------------------------------------------
CONFIG1 = dict(name="single element, plain method: g=(5,8,11,14), n=500, d=4, k=2",
               g=(5, 8, 11, 14), n=500, k=2)


def config2_generators(seed: int = 0) -> Tuple[int, ...]:
    """Single large element: d=6 distinct generators uniform in [50, 200],
    sorted ascending, redrawn until gcd = 1.  n is then the smallest n with
    |Z(n)| >= 5e8 (resolved by the caller with :func:`find_n`)."""
    return draw_generators(rng_for(seed), 6, 50, 200)


CONFIG2_TARGET = 500_000_000


def config3_generators(seed: int = 1) -> Tuple[int, ...]:
    """Dynamic build of all Z(0..N): d=5 distinct generators uniform in
    [3, 40], gcd = 1, sorted ascending; N = 1500."""
    return draw_generators(rng_for(seed), 5, 3, 40)


CONFIG3_N = 1500


@dataclass
class BatchInstance:
    g: Tuple[int, ...]
    target: int


def config4_instances(seed: int = 2, count: int = 4096) -> List[BatchInstance]:
    """Batched: ``count`` instances, d uniform in 3..8, distinct generators
    uniform in [2, 300] with gcd = 1 (sorted ascending), target size
    T = 10^U(2, 6); each instance's n is the smallest with |Z(n)| >= T."""
    rng = rng_for(seed)
    out = []
    for _ in range(count):
        d = int(rng.integers(3, 9))
        g = draw_generators(rng, d, 2, 300)
        t = int(round(10 ** rng.uniform(2.0, 6.0)))
        out.append(BatchInstance(g=g, target=t))
    return out


@dataclass
class ServeStream:
    sets: List[Tuple[int, ...]]
    arrivals_s: np.ndarray      # arrival time of each request (seconds)
    set_index: np.ndarray       # which generator set each request uses
    targets: np.ndarray         # target |Z| of each request
    rate: float = 2000.0
    duration_s: float = 10.0
    extra: dict = field(default_factory=dict)


def config5_stream(seed: int = 3, n_sets: int = 64, rate: float = 2000.0,
                   duration_s: float = 10.0) -> ServeStream:
    """Served: ``n_sets`` generator sets (d uniform in 4..7, distinct
    generators uniform in [5, 500], gcd = 1, sorted ascending); an open-loop
    Poisson stream at ``rate`` requests/s for ``duration_s`` seconds; each
    request picks a set uniformly and a target |Z| = 10^U(3, 7)."""
    rng = rng_for(seed)
    sets = []
    for _ in range(n_sets):
        d = int(rng.integers(4, 8))
        sets.append(draw_generators(rng, d, 5, 500))
    gaps = rng.exponential(1.0 / rate, size=int(rate * duration_s * 1.5) + 16)
    t = np.cumsum(gaps)
    t = t[t < duration_s]
    idx = rng.integers(0, n_sets, size=t.size)
    targets = np.round(10 ** rng.uniform(3.0, 7.0, size=t.size)).astype(np.int64)
    return ServeStream(sets=sets, arrivals_s=t, set_index=idx, targets=targets,
                       rate=rate, duration_s=duration_s)


def random_small_instance(rng: np.random.Generator, max_d: int = 8,
                          max_g: int = 50, max_n: int = 2000,
                          allow_repeats: bool = True) -> Tuple[Tuple[int, ...], int]:
    """A small (g, n) for parity sweeps: d in 1..max_d, generators in
    1..max_g (repeats and gcd > 1 allowed), n in 0..max_n.  No size control:
    callers bound the output by their own count."""
    d = int(rng.integers(1, max_d + 1))
    g = tuple(int(x) for x in rng.integers(1, max_g + 1, size=d))
    if not allow_repeats:
        g = tuple(sorted(set(g)))
    n = int(rng.integers(0, max_n + 1))
    return g, n
