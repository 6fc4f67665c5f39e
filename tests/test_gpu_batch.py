"""Batched enumeration: many instances in one persistent launch, compared
with the oracle and with single-instance plans (identical bytes)."""
import numpy as np
import pytest

import oracle
from gpu_checks import check_sorted_solutions
from paper_2407_20474_gb300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CANARY = -7


@pytest.fixture(scope="module")
def fz():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2407_20474_gb300 as m
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    torch.cuda.set_device(0)
    return m


def run_batch(fz, instances, **kw):
    with fz.Batch(instances, **kw) as b:
        out = torch.full((int(b.total_words) + 16,), CANARY, dtype=torch.int32, device="cuda")
        b.enumerate(out)
        b.sync()
        host = out.cpu().numpy()
        assert (host[int(b.total_words):] == CANARY).all()
        segs = []
        for i, (g, n) in enumerate(instances):
            a, r = int(b.word_offsets[i]), int(b.rows[i])
            segs.append(host[a:a + r * len(g)].reshape(r, len(g)))
        return b, segs


def small_instances(seed, count, max_rows=60_000):
    rng = np.random.Generator(np.random.PCG64(seed))
    out = [((3, 5, 7), 0), ((2, 4), 7), ((7,), 49), ((7,), 50), ((4, 4, 6), 40),
           ((1, 1, 1, 1), 12), ((5, 8, 11, 14), 500)]
    while len(out) < count:
        g, n = workloads.random_small_instance(rng, max_d=8, max_g=60, max_n=3000)
        if oracle.count(g, n) <= max_rows:
            out.append((g, n))
    return out


def test_batch_matches_oracle(fz):
    inst = small_instances(31, 160)
    b, segs = run_batch(fz, inst)
    for (g, n), got in zip(inst, segs):
        assert np.array_equal(got, oracle.enumerate_desc(g, n)), (g, n)


def test_plan_batch_layout(fz):
    """fz_plan_batch gives the exact layout the one-shot batch call then uses:
    rows are the oracle's counts, each instance starts on a multiple of 32
    words after the previous one's rows."""
    inst = small_instances(37, 40)
    offs, rows = fz.fz_plan_batch(inst)
    assert [int(r) for r in rows] == [oracle.count(g, n) for g, n in inst]
    for i, (g, n) in enumerate(inst):
        a, b = int(offs[i]), int(offs[i + 1])
        assert a % 32 == 0 and b - a >= int(rows[i]) * len(g) and b - a < int(rows[i]) * len(g) + 32
    out = torch.full((int(offs[-1]) + 16,), CANARY, dtype=torch.int32, device="cuda")
    offs2 = fz.fz_enumerate_batch(inst, out)
    assert np.array_equal(offs, offs2)
    host = out.cpu().numpy()
    for i, (g, n) in enumerate(inst):
        a, r = int(offs[i]), int(rows[i])
        assert np.array_equal(host[a:a + r * len(g)].reshape(r, len(g)),
                              oracle.enumerate_desc(g, n)), (g, n)


def test_batch_autotune(fz):
    """The measured memo policy: each width's candidates are timed, then the
    widths' fastest choices are tried one at a time on the whole batch and
    kept when it gets faster; each width ends with the default or its own
    fastest choice, and batches created under the result equal the oracle."""
    inst = small_instances(43, 150)
    default = {d: fz.fz_batch_policy(d) for d in range(3, 9)}
    try:
        rows, chosen = fz.fz_batch_autotune(inst)
        per_width = [r for r in rows if r["d"] > 0]
        whole = [r for r in rows if r["d"] == 0]
        assert per_width and whole, "no candidate timed"
        assert whole[0]["run_order"] == 0 and whole[0]["rows"] > 0
        fastest = {}
        for d in {r["d"] for r in per_width}:
            best = min((r for r in per_width if r["d"] == d), key=lambda r: r["total_ms"])
            fastest[d] = (best["cap_rows"], bool(best["run_order"]))
        for r in per_width:
            assert r["rows"] > 0 and r["total_ms"] > 0
        for d, pol in chosen.items():
            if d in fastest:
                assert pol in (default[d], fastest[d]), d
        b, segs = run_batch(fz, inst)
        for (g, n), got in zip(inst, segs):
            assert np.array_equal(got, oracle.enumerate_desc(g, n)), (g, n)
    finally:
        fz.fz_batch_policy_reset()
    assert fz.fz_batch_policy(7) == (4.0, True)
    assert fz.fz_batch_policy(4) == (1.0, True)


def test_batch_pair_memo_leaves(fz):
    """Instances whose memo is the closed form of the last two generators
    (no full memo of depth >= 3 fits): last pair coprime, with a common
    factor, equal, or containing 1; with and without shared generator sets."""
    inst = []
    for g in ((3, 10, 15), (6, 4, 4), (5, 9, 12, 18), (7, 2, 1), (11, 13, 17),
              (4, 6, 9, 10, 14), (2, 3, 35, 49)):
        for target in (2_000, 40_000):
            inst.append((g, workloads.find_n(oracle.count_upto, g, target, 64)))
    inst += [(inst[0][0], inst[0][1] + 1), (inst[2][0], inst[2][1] + 3)]
    b, segs = run_batch(fz, inst)
    assert int((b.k == 2).sum()) >= 4, b.k  # the closed form is exercised
    for (g, n), got in zip(inst, segs):
        assert np.array_equal(got, oracle.enumerate_desc(g, n)), (g, n)


def test_batch_run_order(fz):
    """Full memos copied in run order inside the batch launch: the pair's
    closed form (d >= 4) and memos of depth 1..3 (explicit k), prefixes of
    one to six walked coordinates, generator sets repeated with several n
    (one run-order memo for the largest), repeats and gcd > 1."""
    gens = [(5, 9, 12, 18), (2, 3, 35, 49), (7, 11, 13, 17, 19), (6, 10, 15, 4),
            (3, 5, 7, 9, 11, 13), (4, 4, 6, 9), (9, 6, 12, 15, 21, 10), (2, 3, 5, 7, 11, 13, 17, 19)]
    inst = []
    for g in gens:
        for target in (700, 9_000, 40_000):
            inst.append((g, workloads.find_n(oracle.count_upto, g, target, 64)))
    inst.append((gens[0], inst[0][1] + 1))
    b, segs = run_batch(fz, inst)
    assert b.run_order > 0 and b.run_memos > 0, (b.run_order, b.run_memos)
    for (g, n), got in zip(inst, segs):
        assert np.array_equal(got, oracle.enumerate_desc(g, n)), (g, n)
    for k in (1, 2, 3):
        sub = [(g, n) for g, n in inst if len(g) >= k + 2]
        b, segs = run_batch(fz, sub, k=k)
        assert b.run_order > 0, k
        for (g, n), got in zip(sub, segs):
            assert np.array_equal(got, oracle.enumerate_desc(g, n)), (g, n, k)


def test_batch_every_memo_depth(fz):
    inst = [x for x in small_instances(32, 60) if len(x[0]) >= 4]
    for k in (0, 1, 2, 3):
        b, segs = run_batch(fz, inst, k=k)
        for (g, n), got in zip(inst, segs):
            assert np.array_equal(got, oracle.enumerate_desc(g, n)), (g, n, k)


def test_batch_cluster_memo_build(fz):
    """The longest memos built by thread-block clusters: a few elements per
    batch (small tail generators: several warps share an element's words),
    batches of more elements than the cluster has warps (tail minimum 140),
    and many short memos claimed one per CTA after them, among them tails
    whose other generators are at least twice the first.  Rebuilt twice (the
    claim counter starts over)."""
    inst = [((2, 3, 5, 7), 400), ((2, 3, 5, 7, 11), 200), ((33, 37, 41, 43, 47), 2500),
            ((34, 39, 41, 45), 3000), ((5, 8, 11, 14), 900), ((3, 4, 5, 6, 7, 8), 60),
            ((70, 75, 80, 85), 5000), ((130, 140, 150, 160), 9000),
            ((2, 3, 9, 10), 300), ((4, 5, 12, 30), 900), ((3, 4, 9, 20, 23), 250),
            ((2, 5, 40, 41), 2000)]
    inst += small_instances(36, 80)
    with fz.Batch(inst) as b:
        assert b.coop_memos > 0, b.coop_memos
        out = torch.full((int(b.total_words) + 16,), CANARY, dtype=torch.int32, device="cuda")
        for _ in range(2):
            out.fill_(CANARY)
            b.rebuild()
            b.enumerate(out)
            b.sync()
        host = out.cpu().numpy()
        assert (host[int(b.total_words):] == CANARY).all()
        for i, (g, n) in enumerate(inst):
            a, r = int(b.word_offsets[i]), int(b.rows[i])
            got = host[a:a + r * len(g)].reshape(r, len(g))
            assert np.array_equal(got, oracle.enumerate_desc(g, n)), (g, n)


def test_batch_shared_tails_and_rebuild(fz):
    rng = np.random.Generator(np.random.PCG64(33))
    pool = [workloads.draw_generators(rng, int(rng.integers(3, 8)), 5, 60) for _ in range(6)]
    inst = []
    for _ in range(120):
        g = pool[int(rng.integers(0, len(pool)))]
        inst.append((g, int(rng.integers(0, 900))))
    with fz.Batch(inst) as b:
        assert b.memos <= len(pool)
        out = torch.full((int(b.total_words) + 16,), CANARY, dtype=torch.int32, device="cuda")
        first = None
        for _ in range(3):
            out.fill_(CANARY)
            b.rebuild()
            b.enumerate(out)
            b.sync()
            host = out.cpu().numpy()
            if first is None:
                first = host.copy()
            assert np.array_equal(host, first)
        for i, (g, n) in enumerate(inst):
            a, r = int(b.word_offsets[i]), int(b.rows[i])
            got = first[a:a + r * len(g)].reshape(r, len(g))
            assert np.array_equal(got, oracle.enumerate_desc(g, n)), (g, n)


def test_batch_equals_single_instance_plans(fz):
    inst = []
    for x in workloads.config4_instances(2, 48):
        n = workloads.find_n(fz.fz_count_upto, x.g, min(x.target, 200_000), 64)
        inst.append((x.g, n))
    b, segs = run_batch(fz, inst)
    for (g, n), got in zip(inst, segs):
        c = fz.fz_count(g, n)
        one = torch.full((c * len(g) + 8,), CANARY, dtype=torch.int32, device="cuda")
        fz.fz_enumerate(g, n, one)
        torch.cuda.synchronize()
        ref = one[:c * len(g)].cpu().numpy().reshape(c, len(g))
        assert np.array_equal(got, ref), (g, n)
        assert c == oracle.count(g, n)


def test_batch_config4_full(fz):
    """4096 instances (d 3..8, generators in [2,300], |Z| log-uniform in
    [1e2, 1e6]): every segment sorted, valid and of the oracle's count (which
    together prove it equal to the oracle's list), exact rows on a sample of
    the small ones."""
    insts = workloads.config4_instances(2, 4096)
    rng = np.random.Generator(np.random.PCG64(34))
    inst = [(x.g, workloads.find_n(fz.fz_count_upto, x.g, x.target, 64)) for x in insts]
    with fz.Batch(inst) as b:
        out = torch.full((int(b.total_words) + 16,), CANARY, dtype=torch.int32, device="cuda")
        b.enumerate(out)
        b.sync()
        assert bool((out[int(b.total_words):] == CANARY).all())
        sample = set(int(x) for x in rng.integers(0, len(inst), size=200))
        for i, (g, n) in enumerate(inst):
            a, r = int(b.word_offsets[i]), int(b.rows[i])
            rows = out[a:a + r * len(g)].view(r, len(g))
            check_sorted_solutions(rows, g, n)
            assert r == oracle.count(g, n), (g, n)
            if i in sample and r <= 20_000:
                assert np.array_equal(rows.cpu().numpy(), oracle.enumerate_desc(g, n))
