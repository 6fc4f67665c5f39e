"""GPU parity: the CUDA path (through the C ABI) against the oracle.

Exact integer work: the comparison is bit-exact, tuple for tuple and in
order, with no tolerance.  Small and medium cases are compared element by
element; the full-size workloads are checked by properties that prove
equality (sorted, valid, right count; see gpu_checks.py) plus sampled ranks
the oracle computes one by one, and the 5e8-row set also by an order-sensitive
digest of every row against the oracle's (its walk split over host cores).
"""
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
from gpu_checks import check_csr_segments, check_sorted_solutions, rows_digest
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


def run_enum(fz, g, n, rank_begin=0, rank_end=None, pad=16, offset_words=0, **kw):
    """Enumerate into a canary-filled buffer; return (rows, tail canary ok)."""
    d = len(g)
    total = oracle.count(g, n)
    end = total if rank_end is None else min(rank_end, total)
    rows = max(0, end - rank_begin)
    buf = torch.full(((rows + pad) * d + offset_words,), CANARY, dtype=torch.int32,
                     device="cuda")
    view = buf[offset_words:]
    try:
        written = fz.fz_enumerate(g, n, view, rank_begin=rank_begin,
                                  rank_end=rank_end, capacity_rows=rows + pad, **kw)
    except fz.FzError as e:
        raise AssertionError("g=%s n=%d ranks=[%d,%s) %s: %s"
                             % (g, n, rank_begin, rank_end, kw, e)) from e
    torch.cuda.synchronize()
    assert written == rows
    host = buf.cpu().numpy()
    assert (host[:offset_words] == CANARY).all(), "write before the output"
    got = host[offset_words:offset_words + rows * d].reshape(rows, d)
    assert (host[offset_words + rows * d:] == CANARY).all(), "write past the output"
    return got


# --------------------------------------------------------------------------
# counting
# --------------------------------------------------------------------------
def test_count_matches_oracle(fz):
    rng = np.random.Generator(np.random.PCG64(21))
    for _ in range(40):
        g, n = workloads.random_small_instance(rng, max_d=8, max_g=60, max_n=3000)
        assert fz.fz_count(g, n) == oracle.count(g, n), (g, n)
    for g, n in (((13, 37, 38), 300000), ((1, 2), 12345), ((7,), 49), ((7,), 50),
                 ((2, 4), 7), ((3, 5, 7), 0)):
        assert fz.fz_count(g, n) == oracle.count(g, n), (g, n)


def test_count_upto_long_chains(fz):
    # chains longer than one warp pass: the blocked strided scan is used
    for g, n in (((2, 3, 5), 400000), ((1, 1, 2), 150000), ((3,), 200000)):
        got = fz.fz_count_upto(g, n)
        ref = oracle.count_upto(g, n)
        assert np.array_equal(got, ref.astype(np.uint64)), g


def test_count_table_rows(fz):
    g, n = (5, 8, 11, 14), 500
    d = len(g)
    t = torch.zeros((d + 1) * (n + 1), dtype=torch.int64, device="cuda")
    fz.fz_count_table(g, n, t)
    torch.cuda.synchronize()
    got = t.cpu().numpy().view(np.uint64).reshape(d + 1, n + 1)
    ref = oracle.count_table(g, n)
    for j in range(d + 1):
        assert np.array_equal(got[j], ref[j]), j


def test_count_overflow_is_reported(fz):
    # |Z(n, (1,)*16)| = C(n+15, 15) > 2^64 for n = 2^14
    with pytest.raises(fz.FzError) as e:
        fz.fz_count((1,) * 16, 1 << 14)
    assert e.value.status == fz.FZ_EOVERFLOW
    assert fz.fz_count((1,) * 16, 40) == oracle.count((1,) * 16, 40)


def test_table1_counts_on_gpu(fz):
    rows = [(3, 100000, 273793), (4, 10000, 232364), (5, 10000, 14375415),
            (6, 5000, 22955008), (7, 2000, 2369185), (8, 2000, 17552389),
            (9, 1500, 13936185)]
    for d, n, num in rows:
        assert fz.fz_count(workloads.TABLE1_GENERATORS[:d], n) == num


# --------------------------------------------------------------------------
# enumeration, element by element
# --------------------------------------------------------------------------
def test_config1_exact(fz):
    g, n = workloads.CONFIG1["g"], workloads.CONFIG1["n"]
    got = run_enum(fz, g, n, k=2)
    ref = oracle.enumerate_desc(g, n)
    assert got.shape == (3783, 4)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("k", [0, 1, 2, 3, 4])
def test_config1_every_depth(fz, k):
    g, n = workloads.CONFIG1["g"], workloads.CONFIG1["n"]
    assert np.array_equal(run_enum(fz, g, n, k=k), oracle.enumerate_desc(g, n))


def _random_cases(seed, count, max_rows=150_000):
    rng = np.random.Generator(np.random.PCG64(seed))
    cases = []
    while len(cases) < count:
        g, n = workloads.random_small_instance(rng, max_d=8, max_g=50, max_n=2000)
        c = oracle.count(g, n)
        if c > max_rows:
            continue
        cases.append((g, n))
    return cases


def test_random_instances_every_depth_and_top(fz):
    rng = np.random.Generator(np.random.PCG64(99))
    for g, n in _random_cases(5, 45):
        ref = oracle.enumerate_desc(g, n)
        d = len(g)
        for k in sorted({0, 1, min(2, d), min(3, d), d, int(rng.integers(0, d + 1))}):
            tops = {-1, 0, int(rng.integers(0, n + 2))}
            for top in sorted(tops):
                got = run_enum(fz, g, n, k=k, top=top)
                assert np.array_equal(got, ref), (g, n, k, top)


def test_autotuned_random_instances(fz):
    for g, n in _random_cases(6, 40):
        assert np.array_equal(run_enum(fz, g, n), oracle.enumerate_desc(g, n)), (g, n)


def test_measured_autotune(fz):
    """Options measured on the device are remembered and give the same output."""
    for g, n in (((7, 11, 13, 17, 19), 900), ((5, 8, 11, 14), 700), ((3, 4), 50), ((3,), 30)):
        k, slice_rows, est_ms = fz.fz_autotune(g, n)
        assert 0 <= k <= len(g) and est_ms >= 0
        with fz.Plan(g, n) as plan:
            assert plan.k == k
            if slice_rows > 0:
                assert plan.slice_rows == slice_rows
        assert np.array_equal(run_enum(fz, g, n), oracle.enumerate_desc(g, n)), (g, n)


def test_autotune_report(fz):
    """Every candidate the tuner timed is reported; the best one is the
    fastest candidate not screened out, and plans then use it."""
    g = (56, 90, 96, 127, 146, 178)
    n = 16000
    (k, slice_rows, ms), cands = fz.fz_autotune_report(g, n)
    assert cands, "no candidate timed"
    timed = [c for c in cands if not c["screened_out"]]
    fastest = min(timed, key=lambda c: c["total_ms"])
    assert (k, slice_rows) == (fastest["k"], fastest["slice_rows"])
    assert abs(ms - fastest["total_ms"]) < 1e-9
    for c in cands:
        assert c["build_ms"] >= 0 and c["enum_ms"] > 0
        assert abs(c["total_ms"] - c["build_ms"] - c["enum_ms"]) < 1e-6 * max(1.0, c["total_ms"])
    with fz.Plan(g, n) as plan:
        assert (plan.k, plan.slice_rows) == (k, slice_rows)
    assert np.array_equal(run_enum(fz, g, n), oracle.enumerate_desc(g, n))


@pytest.mark.parametrize("d", [2, 3, 5, 6, 7, 9, 12, 16])
def test_small_slices_ring_boundaries(fz, d):
    """Tiny slices and many ring halves: every flush path, every tuple width."""
    rng = np.random.Generator(np.random.PCG64(100 + d))
    g = tuple(sorted(int(x) for x in rng.integers(2, 9, size=d)))
    n = workloads.find_n(oracle.count_upto, g, 20000)
    ref = oracle.enumerate_desc(g, n)
    for k in (0, min(2, d - 1), min(3, d - 1)):
        for slice_rows in (4, 36, 1000, 0):
            got = run_enum(fz, g, n, k=k, slice_rows=slice_rows)
            assert np.array_equal(got, ref), (g, n, k, slice_rows)


@pytest.mark.parametrize("g", [(6, 10), (4, 9, 6, 15), (5, 8, 12, 18), (3, 7, 7),
                               (9, 14, 1, 5), (11, 4, 4), (13, 6, 21, 35), (2, 3, 5, 1, 1)])
def test_walk_leaves_as_progression(fz, g):
    """Walk leaves produced directly along the progression of valid a_{d-2}
    values: last two generators coprime, with a common factor, equal, or 1;
    no memo and partial memos; windows and tiny slices that start work items
    inside a run of walk leaves."""
    n = workloads.find_n(oracle.count_upto, g, 3000)
    ref = oracle.enumerate_desc(g, n)
    total = ref.shape[0]
    d = len(g)
    for k, top in ((0, -1), (2, 7), (min(3, d - 1), 25), (2, -1)):
        if k > d:
            continue
        for slice_rows in (4, 52, 0):
            got = run_enum(fz, g, n, k=k, top=top, slice_rows=slice_rows)
            assert np.array_equal(got, ref), (g, n, k, top, slice_rows)
    rng = np.random.Generator(np.random.PCG64(sum(g)))
    for _ in range(8):
        a = int(rng.integers(0, total))
        b = int(rng.integers(a, total + 1))
        got = run_enum(fz, g, n, rank_begin=a, rank_end=b, k=0, slice_rows=8)
        assert np.array_equal(got, ref[a:b]), (g, n, a, b)
    for n2 in (n + 1, n + 7):  # other residues (some not divisible by the gcd)
        assert np.array_equal(run_enum(fz, g, n2, k=0), oracle.enumerate_desc(g, n2)), (g, n2)


def test_bounded_device_wait_times_out(fz):
    """A device wait that can never complete gives up after its limit and the
    host reads FZ_ETIMEOUT; the context stays usable (no fault, no hang)."""
    import time
    for limit_ms in (5, 50):
        t0 = time.perf_counter()
        st = fz.fz_selftest_bounded_wait(limit_ms)
        dt = time.perf_counter() - t0
        assert st == fz.FZ_ETIMEOUT, fz.status_string(st)
        assert dt >= limit_ms / 1e3, dt
        assert dt < 10.0, dt
    with pytest.raises(fz.FzError):
        fz.fz_selftest_bounded_wait(0)
    g, n = (5, 8, 11, 14), 500
    assert np.array_equal(run_enum(fz, g, n, k=2), oracle.enumerate_desc(g, n))


def test_write_probe(fz):
    """The measurement utility writes out[w] = w and nothing past the end."""
    for words in (0, 1, 5, 1023, 1 << 20, (1 << 20) + 3):
        buf = torch.full((words + 64,), CANARY, dtype=torch.int32, device="cuda")
        fz.fz_write_probe(buf[:words] if words else buf[:0])
        torch.cuda.synchronize()
        host = buf.cpu().numpy()
        assert np.array_equal(host[:words], np.arange(words, dtype=np.int32)), words
        assert (host[words:] == CANARY).all(), words
    with pytest.raises(fz.FzError):
        fz.fz_write_probe(torch.zeros(9, dtype=torch.int32, device="cuda")[1:])  # unaligned


def test_rank_windows_and_unaligned_output(fz):
    g, n = (7, 11, 13, 17, 19), 420
    ref = oracle.enumerate_desc(g, n)
    total = ref.shape[0]
    rng = np.random.Generator(np.random.PCG64(3))
    windows = [(0, total), (1, total), (3, 4), (total - 1, total), (5, 5),
               (0, None), (total - 5, total + 100), (total, total + 3)]
    for _ in range(20):
        a = int(rng.integers(0, total))
        b = int(rng.integers(a, total + 1))
        windows.append((a, b))
    for a, b in windows:
        for offset_words in (0, 1, 3):
            got = run_enum(fz, g, n, rank_begin=a, rank_end=b, k=2, slice_rows=64,
                           offset_words=offset_words)
            end = total if b is None else min(b, total)
            assert np.array_equal(got, ref[a:end]), (a, b, offset_words)


def test_plan_reuse_rebuild_and_unrank(fz):
    g, n = (9, 10, 14, 15, 21), 600
    ref = oracle.enumerate_desc(g, n)
    total = ref.shape[0]
    with fz.Plan(g, n, k=3) as plan:
        assert plan.count == total
        out = torch.full((total, len(g)), CANARY, dtype=torch.int32, device="cuda")
        for _ in range(3):
            out.fill_(CANARY)
            plan.rebuild()
            assert plan.enumerate(out) == total
            plan.sync()
            assert np.array_equal(out.cpu().numpy(), ref)
        ranks = torch.tensor(list(range(0, total, 97)) + [total - 1], dtype=torch.int64,
                             device="cuda")
        tup = torch.zeros((ranks.numel(), len(g)), dtype=torch.int32, device="cuda")
        plan.unrank(ranks, tup)
        plan.sync()
        idx = ranks.cpu().numpy()
        assert np.array_equal(tup.cpu().numpy(), ref[idx])


def test_partial_memo_unrank(fz):
    g, n = (6, 7, 9, 10, 13, 15), 260
    ref = oracle.enumerate_desc(g, n)
    for k, top in ((2, 40), (3, 100), (4, 1), (1, 50)):
        with fz.Plan(g, n, k=k, top=top) as plan:
            ranks = torch.arange(0, ref.shape[0], 13, dtype=torch.int64, device="cuda")
            tup = torch.zeros((ranks.numel(), len(g)), dtype=torch.int32, device="cuda")
            plan.unrank(ranks, tup)
            plan.sync()
            assert np.array_equal(tup.cpu().numpy(), ref[ranks.cpu().numpy()]), (k, top)


def test_degenerate_inputs(fz):
    # n = 0: one all-zero tuple; empty sets; d = 1; k = d (output is Memo[n])
    assert np.array_equal(run_enum(fz, (3, 5, 7), 0), np.zeros((1, 3), np.int32))
    assert run_enum(fz, (2, 4), 7).shape == (0, 2)
    assert fz.fz_count((2, 4), 7) == 0
    assert np.array_equal(run_enum(fz, (7,), 49), np.array([[7]], np.int32))
    assert run_enum(fz, (7,), 50).shape == (0, 1)
    assert np.array_equal(run_enum(fz, (7,), 49, k=1), np.array([[7]], np.int32))
    g, n = (3, 4, 5), 60
    ref = oracle.enumerate_desc(g, n)
    assert np.array_equal(run_enum(fz, g, n, k=3), ref)
    assert np.array_equal(run_enum(fz, g, n, k=3, rank_begin=5, rank_end=17), ref[5:17])
    assert np.array_equal(run_enum(fz, g, n, k=3, top=10), ref)
    # repeated generators and gcd > 1
    for g, n in (((4, 4, 6), 40), ((6, 10, 15, 6), 90), ((1, 1, 1, 1), 12)):
        assert np.array_equal(run_enum(fz, g, n), oracle.enumerate_desc(g, n))


def test_argument_errors(fz):
    out = torch.zeros(64, dtype=torch.int32, device="cuda")
    with pytest.raises(fz.FzError) as e:
        fz.fz_enumerate((5, 8, 11, 14), 500, out, capacity_rows=16)
    assert e.value.status == fz.FZ_ENOSPC
    with pytest.raises(fz.FzError) as e:
        fz.fz_enumerate((5, 8, 11, 14), 500, out, k=7)
    assert e.value.status == fz.FZ_EINVAL
    with pytest.raises(fz.FzError) as e:
        fz.Plan((5, 8, 11, 14), -3)
    assert e.value.status == fz.FZ_EINVAL


def test_enumerate_host(fz):
    g, n = (5, 8, 11, 14), 700
    ref = oracle.enumerate_desc(g, n)
    out = np.full(ref.size + 8, CANARY, dtype=np.int32)
    w = fz.fz_enumerate_host(g, n, out)
    assert w == ref.shape[0]
    assert np.array_equal(out[:ref.size].reshape(ref.shape), ref)
    assert (out[ref.size:] == CANARY).all()


def test_enumerate_host_pinned_direct(fz):
    """Page-locked host output is written by the kernel itself."""
    g, n = (5, 8, 11, 14), 900
    ref = oracle.enumerate_desc(g, n)
    out = torch.full((ref.size + 8,), CANARY, dtype=torch.int32).pin_memory()
    w = fz.fz_enumerate_host(g, n, out)
    torch.cuda.synchronize()
    host = out.numpy()
    assert w == ref.shape[0]
    assert np.array_equal(host[:ref.size].reshape(ref.shape), ref)
    assert (host[ref.size:] == CANARY).all()
    w2 = fz.fz_enumerate_host(g, n, out[4:], rank_begin=7, rank_end=1000)
    assert np.array_equal(out.numpy()[4:4 + w2 * 4].reshape(w2, 4), ref[7:1000])


@pytest.mark.parametrize("g,n,chunk,begin,end", [
    # 3 staging buffers: 7+ chunks wrap the ring twice, the last chunk is short
    ((5, 8, 11, 14), 700, 997, 0, None),
    ((5, 8, 11, 14), 700, 613, 1234, 9001),          # window not starting at 0
    ((3, 7, 8, 10, 13, 20), 260, 4099, 11, None),    # d = 6, odd chunk
    ((2, 5), 50001, 1, 3, 40),                        # one row per chunk
])
def test_enumerate_host_streamed_many_chunks(fz, g, n, chunk, begin, end):
    """Pageable host output streamed through the page-locked staging ring:
    many chunks (ring wrap, short last chunk, rank windows), byte for byte
    against the oracle, nothing written outside the window's rows."""
    ref = oracle.enumerate_desc(g, n)
    stop = ref.shape[0] if end is None else min(end, ref.shape[0])
    want = ref[begin:stop]
    d = len(g)
    chunks = -(-want.shape[0] // chunk)
    assert chunks >= 7 or want.shape[0] < 7 * chunk
    out = np.full(want.size + 2 * d + 5, CANARY, dtype=np.int32)
    w = fz.fz_enumerate_host(g, n, out[d:], rank_begin=begin, rank_end=end, chunk_rows=chunk)
    assert w == want.shape[0]
    assert (out[:d] == CANARY).all(), "write before the output"
    assert np.array_equal(out[d:d + want.size].reshape(want.shape), want)
    assert (out[d + want.size:] == CANARY).all(), "write past the output"
    # a second call reuses the staging pool and gives the same bytes
    again = np.full(want.size, CANARY, dtype=np.int32)
    assert fz.fz_enumerate_host(g, n, again, rank_begin=begin, rank_end=end,
                                chunk_rows=chunk) == want.shape[0]
    assert np.array_equal(again.reshape(want.shape), want)


@pytest.mark.parametrize("chunk", [0, 5_000_000])
def test_enumerate_host_streamed_large(fz, chunk):
    """A pageable output of 1.09 GB (45,216,350 rows): the default path
    (direct writes where the device reaches pageable memory through the
    host's page tables, else 128 MB chunks through the staging ring) and the
    ring with nine chunks of 5,000,000 rows; every row checked against the
    oracle's digest, plus the first rows element by element."""
    g = (56, 90, 96, 127, 146, 178)
    n = 24000
    total = oracle.count(g, n)
    out = np.empty(total * len(g), dtype=np.int32)
    w = fz.fz_enumerate_host(g, n, out, chunk_rows=chunk)
    assert w == total
    rows = out.reshape(total, len(g))
    head = oracle.enumerate_desc(g, n, 0, 20000)
    assert np.array_equal(rows[:20000], head)
    dev = torch.from_numpy(rows).cuda()
    assert rows_digest(dev) == oracle.digest_parallel(g, n, threads=os.cpu_count() or 1)[1]


# --------------------------------------------------------------------------
# memo build (the dynamic FactorizationsUpToElement pass)
# --------------------------------------------------------------------------
def _memo_on_gpu(fz, tail, top):
    rows = fz.fz_memo_rows(tail, top)
    off = torch.zeros(top + 1, dtype=torch.int64, device="cuda")
    buf = torch.full(((rows + 4) * len(tail),), CANARY, dtype=torch.int32, device="cuda")
    got_rows = fz.fz_build_memo_into(tail, top, off, buf, rows)
    torch.cuda.synchronize()
    assert got_rows == rows
    host = buf.cpu().numpy()
    assert (host[rows * len(tail):] == CANARY).all()
    return off.cpu().numpy().view(np.uint64), host[:rows * len(tail)].reshape(rows, len(tail))


@pytest.mark.parametrize("tail,top", [((11, 14), 501), ((4, 9, 10), 300), ((3, 5, 7, 8), 120),
                                      ((1, 2, 3), 60), ((5,), 40), ((6, 10, 15), 200),
                                      ((2, 2, 3), 50)])
def test_memo_matches_definition(fz, tail, top):
    off, rows = _memo_on_gpu(fz, tail, top)
    ref_off, ref_rows = oracle.memo_csr(tail, top)
    assert np.array_equal(off, ref_off)
    assert np.array_equal(rows, ref_rows)


def test_memo_matches_factorizationwise_algorithm(fz):
    g = workloads.config3_generators(1)
    N = 200
    off, rows = _memo_on_gpu(fz, g, N + 1)
    ref_off, ref_rows = oracle.fwpar_lists(g, N)
    assert np.array_equal(off, ref_off)
    assert np.array_equal(rows, ref_rows)


@pytest.mark.parametrize("schedule", [1, 2])
def test_memo_launch_schedules(fz, schedule):
    """One launch per batch and one launch per (m, i) copy give the same memo."""
    for tail, top in (((11, 14), 501), ((4, 9, 10), 300), ((2, 2, 3), 50), ((5,), 40),
                      ((13, 37, 38, 40), 400)):
        ref_off, ref_rows = oracle.lex_lists_c(tail, top)
        rows = int(ref_off[-1])
        k = len(tail)
        off = torch.zeros(top + 1, dtype=torch.int64, device="cuda")
        buf = torch.full(((rows + 4) * k,), CANARY, dtype=torch.int32, device="cuda")
        got = fz.fz_build_memo_schedule(tail, top, schedule, off, buf, rows)
        torch.cuda.synchronize()
        assert got == rows
        host = buf.cpu().numpy()
        assert (host[rows * k:] == CANARY).all()
        assert np.array_equal(off.cpu().numpy().view(np.uint64), ref_off), (tail, schedule)
        assert np.array_equal(host[:rows * k].reshape(rows, k), ref_rows), (tail, schedule)
    with pytest.raises(fz.FzError) as e:
        fz.fz_build_memo_schedule((3, 4), 10, 7, off, buf, rows)
    assert e.value.status == fz.FZ_EINVAL


def test_memo_library_owned_handle(fz):
    m = fz.fz_build_memo((4, 9, 10), 100)
    ref_off, _ = oracle.memo_csr((4, 9, 10), 100)
    assert m.rows == int(ref_off[-1]) and m.k == 3 and m.top == 100
    m.close()


# --------------------------------------------------------------------------
# full-size workloads (the launch configuration bench.py times)
# --------------------------------------------------------------------------
def test_config2_full_size(fz):
    """Single large element, |Z| ~ 5e8 (12 GB of int32 tuples)."""
    g = workloads.config2_generators(0)
    n = workloads.find_n(oracle.count_upto, g, workloads.CONFIG2_TARGET, 4096)
    total = oracle.count(g, n)
    d = len(g)
    with fz.Plan(g, n) as plan:
        assert plan.count == total
        out = torch.empty((total + 64) * d, dtype=torch.int32, device="cuda")
        out[total * d:].fill_(CANARY)
        assert plan.enumerate(out) == total
        plan.sync()
        rows = out[:total * d].view(total, d)
        assert bool((out[total * d:] == CANARY).all())
        check_sorted_solutions(rows, g, n)
        # sampled ranks: both ends, slice boundaries, random
        rng = np.random.Generator(np.random.PCG64(11))
        S = plan.slice_rows
        picks = set(range(0, 2000)) | set(range(total - 2000, total))
        for s in range(1, 200):
            for off in (-2, -1, 0, 1):
                r = s * S + off
                if 0 <= r < total:
                    picks.add(r)
        picks |= set(int(x) for x in rng.integers(0, total, size=2000))
        picks = sorted(picks)
        T = oracle.count_table(g, n)
        ref = np.array([oracle.unrank(g, n, r, T) for r in picks], dtype=np.int32)
        idx = torch.tensor(picks, dtype=torch.int64, device="cuda")
        got = rows.index_select(0, idx).cpu().numpy()
        assert np.array_equal(got, ref)
        # the oracle's own walk over the first ranks
        head = oracle.enumerate_desc(g, n, 0, 50000)
        assert np.array_equal(rows[:50000].cpu().numpy(), head)
        # every row: the order-sensitive digest of the whole output against
        # the oracle's, its first-coordinate subtrees walked on all host cores
        rows_o, dig = oracle.digest_parallel(g, n, threads=os.cpu_count() or 1)
        assert rows_o == total
        assert rows_digest(rows) == dig
        # the launch configuration bench.py times: the enumeration capped at
        # 3 or 2 CTAs per SM (larger rings) while another plan of the same
        # element rebuilds on a second stream; the bytes must not change
        out2 = torch.empty_like(out)
        side = torch.cuda.Stream()
        main = torch.cuda.current_stream()
        with fz.Plan(g, n, k=plan.k) as other:
            for cap in (3, 2):
                out2.fill_(CANARY)
                plan.set_enum_ctas_per_sm(cap)
                side.wait_stream(main)
                other.rebuild(stream=side)
                assert plan.enumerate(out2) == total
                torch.cuda.synchronize()
                plan.sync()
                other.sync()
                assert torch.equal(out2, out), cap
            plan.set_enum_ctas_per_sm(0)
        del out, out2


_FORCED_FILL = r"""
import sys, numpy as np, torch
sys.path.insert(0, sys.argv[1])
import oracle
import paper_2407_20474_gb300 as fz
torch.cuda.set_device(0)
for tail, top in (((4, 9, 10), 300), ((3, 7, 8, 20), 200), ((2, 5), 200), ((5,), 40),
                  ((4, 20, 22, 31, 39), 240), ((2, 4), 80), ((3, 6, 6), 90), ((11, 14), 501)):
    rows = fz.fz_memo_rows(tail, top)
    off = torch.zeros(top + 1, dtype=torch.int64, device="cuda")
    buf = torch.full(((rows + 4) * len(tail),), -7, dtype=torch.int32, device="cuda")
    assert fz.fz_build_memo_into(tail, top, off, buf, rows) == rows
    torch.cuda.synchronize()
    host = buf.cpu().numpy()
    assert (host[rows * len(tail):] == -7).all(), tail
    ref_off, ref_rows = oracle.memo_csr(tail, top)
    assert np.array_equal(off.cpu().numpy().view(np.uint64), ref_off), tail
    assert np.array_equal(host[:rows * len(tail)].reshape(rows, len(tail)), ref_rows), tail
print("forced fill ok")
"""


@pytest.mark.parametrize("variant", ["phase", "grid"])
def test_memo_fill_forced_variant(fz, variant):
    """The whole-GPU fills forced on small memos (FZ_MEMO_FILL is read once
    per process, so each runs in a child): phases of min(t_1..) elements
    where the tail allows them (t_1 >= 2 t_0), batches of t_0 elements
    otherwise, both equal to the oracle's memo."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, FZ_MEMO_FILL=variant)
    r = subprocess.run([sys.executable, "-c", _FORCED_FILL, root], env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    assert "forced fill ok" in r.stdout


def test_config3_full_memo_build(fz):
    """Dynamic build of all Z(0..1500) for d=5 generators in [3, 40]."""
    g = workloads.config3_generators(1)
    N = workloads.CONFIG3_N
    counts = oracle.count_upto(g, N)
    total = int(counts.astype(np.float64).sum())
    rows_needed = fz.fz_memo_rows(g, N + 1)
    assert rows_needed == total
    off = torch.zeros(N + 2, dtype=torch.int64, device="cuda")
    buf = torch.full(((total + 4) * len(g),), CANARY, dtype=torch.int32, device="cuda")
    assert fz.fz_build_memo_into(g, N + 1, off, buf, total) == total
    torch.cuda.synchronize()
    assert bool((buf[total * len(g):] == CANARY).all())
    rows = buf[:total * len(g)].view(total, len(g))
    check_csr_segments(off, rows, g, counts)
    o = off.cpu().numpy()
    rng = np.random.Generator(np.random.PCG64(12))
    for m in [0, 1, 4, 5, 40, N - 1, N] + [int(x) for x in rng.integers(0, N + 1, size=12)]:
        ref = oracle.enumerate_desc(g, m)
        got = rows[int(o[m]):int(o[m + 1])].cpu().numpy()
        assert np.array_equal(got, ref), m


def test_table1_instances_every_row(fz):
    """The paper's own workload (Table 1: g = the first d of (13, 37, 38,
    40..45), each n at the memo depth the paper used): every row of every
    instance against the oracle by the order-sensitive digest, the count
    against the printed one where it is a pin."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                        "table1_counts.txt")
    cases = []
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        cases.append((int(f[0]), int(f[1]), int(f[2]), int(f[3]), len(f) == 4))
    assert len(cases) == 31
    threads = os.cpu_count() or 1
    oracle_digest = {}
    for d, k, n, printed, pin in cases:
        g = workloads.TABLE1_GENERATORS[:d]
        c = fz.fz_count(g, n)
        if pin:
            assert c == printed, (d, n)
        out = torch.empty((c + 16) * d, dtype=torch.int32, device="cuda")
        out[c * d:].fill_(CANARY)
        assert fz.fz_enumerate(g, n, out, k=k) == c
        torch.cuda.synchronize()
        assert bool((out[c * d:] == CANARY).all())
        if (d, n) not in oracle_digest:
            oracle_digest[(d, n)] = oracle.digest_parallel(g, n, threads=threads)
        rows_o, dig = oracle_digest[(d, n)]
        assert rows_o == c, (d, n)
        assert rows_digest(out[:c * d].view(c, d)) == dig, (d, k, n)
        del out
