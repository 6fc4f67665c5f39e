"""Host-side integer helpers of the closed forms (csrc/fz_host_math.h),
compiled on their own with the host compiler and checked against brute
force: the extended-Euclid parameters of the last two generators (which
give the progression of valid a_{d-2}, Section 3's ordinary step solved in
closed form) and the lattice-point count that sizes a pair memo's
run-order table."""
import math
import os
import random
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2407_20474_gb300", "csrc")

DRIVER = r"""
#include <cstdio>
#include "fz_host_math.h"
int main() {
    char op;
    while (std::scanf(" %c", &op) == 1) {
        if (op == 'P') {
            long long g, h;
            std::scanf("%lld %lld", &g, &h);
            int64_t e, h1, g1, inv;
            fz::pair_params(g, h, &e, &h1, &g1, &inv);
            std::printf("%lld %lld %lld %lld\n", (long long)e, (long long)h1, (long long)g1,
                        (long long)inv);
        } else if (op == 'R') {
            long long n, t0, t1;
            std::scanf("%lld %lld %lld", &n, &t0, &t1);
            std::printf("%llu\n", (unsigned long long)fz::pair_rows_upto(n, t0, t1));
        } else if (op == 'F') {
            unsigned long long c, m, a, b;
            std::scanf("%llu %llu %llu %llu", &c, &m, &a, &b);
            unsigned __int128 s = fz::floor_sum(c, m, a, b);
            std::printf("%llu %llu\n", (unsigned long long)(s >> 64), (unsigned long long)s);
        }
    }
    return 0;
}
"""


@pytest.fixture(scope="module")
def run(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("hostmath")
    src = d / "driver.cpp"
    src.write_text(DRIVER)
    exe = d / "driver"
    subprocess.run([cxx, "-std=c++17", "-O2", "-I", CSRC, str(src), "-o", str(exe)], check=True)

    def call(lines):
        r = subprocess.run([str(exe)], input="\n".join(lines) + "\n", capture_output=True,
                           text=True, check=True, timeout=120)
        return r.stdout.split("\n")[:len(lines)]
    return call


def test_pair_params_give_the_progression(run):
    rng = random.Random(1)
    cases = [(1, 1), (1, 7), (7, 1), (6, 4), (4, 6), (12, 18), (300, 299), (2, 2), (35, 49)]
    cases += [(rng.randint(1, 300), rng.randint(1, 300)) for _ in range(400)]
    out = run(["P %d %d" % c for c in cases])
    for (g, h), line in zip(cases, out):
        e, h1, g1, inv = map(int, line.split())
        assert e == math.gcd(g, h) and h1 == h // e and g1 == g // e
        assert 0 <= inv < max(h1, 1)
        if h1 > 1:
            assert g1 * inv % h1 == 1
        # the valid a_{d-2} of Z(p, (g, h)) form the class (p/e) inv mod h1
        pool = range(0, 3 * g * h + 1)
        for p in rng.sample(pool, min(6, len(pool))) + [0, g * h]:
            valid = [v for v in range(p // g + 1) if (p - v * g) % h == 0]
            if p % e:
                assert valid == []
                continue
            astar = (p // e) % h1 * inv % h1 if h1 > 1 else 0
            assert valid == [v for v in range(p // g + 1) if v % h1 == astar], (g, h, p)


def test_floor_sum_brute_force(run):
    rng = random.Random(2)
    cases = [(0, 1, 0, 0), (1, 1, 0, 0), (5, 3, 0, 7), (10, 1, 1, 0)]
    cases += [(rng.randint(0, 60), rng.randint(1, 40), rng.randint(0, 90), rng.randint(0, 90))
              for _ in range(500)]
    out = run(["F %d %d %d %d" % c for c in cases])
    for (c, m, a, b), line in zip(cases, out):
        hi, lo = map(int, line.split())
        assert (hi << 64 | lo) == sum((a * i + b) // m for i in range(c)), (c, m, a, b)


def test_pair_rows_upto_counts_lattice_points(run):
    rng = random.Random(3)
    cases = [(0, 1, 1), (0, 5, 7), (4, 5, 7), (35, 5, 7), (100, 1, 1), (1000, 2, 3)]
    cases += [(rng.randint(0, 3000), rng.randint(1, 60), rng.randint(1, 60)) for _ in range(300)]
    out = run(["R %d %d %d" % c for c in cases])
    for (n, t0, t1), line in zip(cases, out):
        brute = sum((n - t0 * x) // t1 + 1 for x in range(n // t0 + 1))
        assert int(line) == brute, (n, t0, t1)
    # the largest element: (n + 1)(n + 2) / 2 points for t0 = t1 = 1
    n = 2 ** 31 - 1
    out = run(["R %d 1 1" % n, "R %d 1 2" % n])
    assert int(out[0]) == (n + 1) * (n + 2) // 2
    # t0 = 1, t1 = 2: sum over j <= n of floor(j / 2) + 1, n odd
    M = (n - 1) // 2
    assert int(out[1]) == M * (M + 1) + n + 1
