"""Serving: requests over resident generator sets with continuous batching.
Every result produced in the mix is byte-identical to the same query run
alone (exact integer output: tolerance 0)."""
import numpy as np
import pytest

import oracle
from paper_2407_20474_gb300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fz():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2407_20474_gb300 as m
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    torch.cuda.set_device(0)
    return m


def rows_of(srv, ticket, res):
    words = int(res.count) * int(res.d)
    out = torch.empty(max(words, 1), dtype=torch.int32)
    srv.copy(ticket, out)
    return out[:words].numpy().reshape(int(res.count), int(res.d))


def alone(fz, g, n):
    c = fz.fz_count(g, n)
    out = torch.empty(max(c, 1) * len(g), dtype=torch.int32, device="cuda")
    fz.fz_enumerate(g, n, out)
    torch.cuda.synchronize()
    return out[:c * len(g)].cpu().numpy().reshape(c, len(g))


@pytest.mark.parametrize("per_request", [False, True])
def test_mix_equals_alone(fz, per_request):
    """Requests launched in groups (default) or one by one: every result
    equals the same query run alone, and the oracle's list where small."""
    rng = np.random.Generator(np.random.PCG64(41))
    sets = [workloads.draw_generators(rng, int(rng.integers(4, 8)), 5, 60) for _ in range(5)]
    n_max = 700
    with fz.Server(max_in_flight=16, streams=4, per_request=per_request) as srv:
        ids = [srv.register(g, n_max) for g in sets]
        reqs = []
        for _ in range(150):
            s = int(rng.integers(0, len(sets)))
            n = int(rng.integers(0, n_max + 1))
            reqs.append((s, n, srv.submit(ids[s], n)))
        for s, n, t in reqs:
            res = srv.wait(t, 60000)
            assert res.status == fz.FZ_SERVE_DONE
            assert res.t_submit <= res.t_admit <= res.t_done
            got = rows_of(srv, t, res)
            g = sets[s]
            assert int(res.count) == oracle.count(g, n)
            assert np.array_equal(got, alone(fz, g, n)), (g, n)
            if res.count <= 20000:
                assert np.array_equal(got, oracle.enumerate_desc(g, n))
            srv.release(t)
        st = srv.stats()
        assert st.completed == len(reqs) and st.bytes_in_use == 0


def test_admission_by_exact_bytes_and_queue_limit(fz):
    g = (7, 9, 11, 13, 17)
    n = 300
    c = fz.fz_count(g, n)
    size = c * len(g) * 4
    budget = ((size + 255) // 256) * 256          # room for exactly one result
    with fz.Server(memory_bytes=budget, max_in_flight=8, streams=2, max_queue=2) as srv:
        sid = srv.register(g, 400)
        t1 = srv.submit(sid, n)
        r1 = srv.wait(t1, 60000)
        assert r1.status == fz.FZ_SERVE_DONE
        t2 = srv.submit(sid, n)                    # waits for memory: t1 not released
        t3 = srv.submit(sid, n)
        with pytest.raises(fz.FzError) as e:
            srv.submit(sid, n)                     # queue holds two: full
        assert e.value.status == fz.FZ_EAGAIN
        assert srv.poll(t2).status == fz.FZ_SERVE_QUEUED
        assert srv.stats().bytes_in_use <= budget
        ref = rows_of(srv, t1, r1)
        srv.release(t1)                            # frees the bytes: t2 then t3 run
        for t in (t2, t3):
            r = srv.wait(t, 60000)
            assert r.status == fz.FZ_SERVE_DONE
            assert np.array_equal(rows_of(srv, t, r), ref)
            srv.release(t)
        with pytest.raises(fz.FzError) as e:
            srv.submit(sid, 400)                   # larger than the whole budget
        assert e.value.status == fz.FZ_ENOMEM
        with pytest.raises(fz.FzError) as e:
            srv.submit(sid, 401)                   # beyond the set's n_max
        assert e.value.status == fz.FZ_EINVAL
        with pytest.raises(fz.FzError) as e:
            srv.poll(123456789)
        assert e.value.status == fz.FZ_ENOTFOUND


def test_config5_sets_large_requests(fz):
    """Requests at the upper sizes of the served workload (|Z| about 10^6 and
    10^7 rows, generator sets of the served workload's draw), several in
    flight at once: every served result equals the oracle's list, checked by
    its count and an order-sensitive digest of every row against the
    oracle's walk, and the 10^6-row results also equal the same query run
    alone."""
    import os
    from gpu_checks import rows_digest
    stream = workloads.config5_stream(3, n_sets=4, rate=2000.0, duration_s=0.05)
    threads = os.cpu_count() or 1
    with fz.Server(max_in_flight=32, streams=8) as srv:
        for g in stream.sets:
            n7 = workloads.find_n(oracle.count_upto, g, 10_000_000, n_hint=1024)
            n6 = workloads.find_n(oracle.count_upto, g, 1_000_000, n_hint=1024)
            sid = srv.register(g, n7)
            ns = (n7, n6, n7 - 1, 0)
            ts = [srv.submit(sid, m) for m in ns]
            for m, t in zip(ns, ts):
                r = srv.wait(t, 120000)
                assert r.status == fz.FZ_SERVE_DONE
                assert int(r.count) == oracle.count(g, m)
                words = int(r.count) * len(g)
                dev = torch.empty(max(words, 1), dtype=torch.int32, device="cuda")
                srv.copy(t, dev)
                rows = dev[:words].view(int(r.count), len(g))
                assert rows_digest(rows) == oracle.digest_parallel(g, m, threads)[1], (g, m)
                if m == n6:
                    assert np.array_equal(rows.cpu().numpy(), alone(fz, g, m)), (g, m)
                srv.release(t)


def test_cancel_queued_request(fz):
    """A queued request can be cancelled: it never runs, reports FZ_ECANCELED,
    and the request queued behind it is admitted once memory frees up."""
    g = (7, 9, 11, 13, 17)
    n = 300
    c = fz.fz_count(g, n)
    budget = ((c * len(g) * 4 + 255) // 256) * 256   # room for exactly one result
    with fz.Server(memory_bytes=budget, max_in_flight=8, streams=2, max_queue=8) as srv:
        sid = srv.register(g, n)
        t1 = srv.submit(sid, n)
        r1 = srv.wait(t1, 60000)
        assert r1.status == fz.FZ_SERVE_DONE
        t2 = srv.submit(sid, n)                    # queued: t1 holds the memory
        t3 = srv.submit(sid, n)
        assert srv.poll(t2).status == fz.FZ_SERVE_QUEUED
        srv.cancel(t2)
        r2 = srv.poll(t2)
        assert r2.status == fz.FZ_ECANCELED and r2.t_done >= r2.t_submit
        with pytest.raises(fz.FzError) as e:
            srv.copy(t2, torch.empty(c * len(g), dtype=torch.int32))
        assert e.value.status == fz.FZ_ECANCELED
        srv.release(t2)                            # a cancelled ticket is released as usual
        with pytest.raises(fz.FzError) as e:
            srv.poll(t2)
        assert e.value.status == fz.FZ_ENOTFOUND
        ref = rows_of(srv, t1, r1)
        srv.release(t1)                            # t3 (behind the cancelled t2) runs
        r3 = srv.wait(t3, 60000)
        assert r3.status == fz.FZ_SERVE_DONE
        assert np.array_equal(rows_of(srv, t3, r3), ref)
        assert np.array_equal(ref, oracle.enumerate_desc(g, n))
        srv.cancel(t3)                             # finished: left as it is
        assert srv.poll(t3).status == fz.FZ_SERVE_DONE
        srv.release(t3)
        st = srv.stats()
        assert st.bytes_in_use == 0 and st.queued == 0
        assert st.completed == 2                   # t1 and t3; t2 never ran


def test_submit_by_generators(fz):
    """fz_serve_submit_gens registers a set on first use and reuses it for
    queries it covers; results equal the oracle."""
    with fz.Server(max_in_flight=8, streams=2) as srv:
        g = (6, 9, 20)
        t1 = srv.submit_gens(g, 500)
        t2 = srv.submit_gens(g, 450)                # covered by the first registration
        assert srv.stats().sets == 1
        t3 = srv.submit_gens((9, 6, 20), 450)       # another order is another set
        t4 = srv.submit_gens(g, 800)                # beyond n_max: a new registration
        assert srv.stats().sets == 3
        for t, gg, n in ((t1, g, 500), (t2, g, 450), (t3, (9, 6, 20), 450), (t4, g, 800)):
            r = srv.wait(t, 60000)
            assert r.status == fz.FZ_SERVE_DONE
            assert np.array_equal(rows_of(srv, t, r), oracle.enumerate_desc(gg, n)), (gg, n)
            srv.release(t)
        with pytest.raises(fz.FzError) as e:
            srv.wait(t1, 10)                        # released: unknown ticket
        assert e.value.status == fz.FZ_ENOTFOUND


def test_grouped_server_wide_run_order_plan(fz):
    """A width-9 set whose plan keeps a depth-2 memo in run order (the deeper
    memos exceed the plan's memo budget): the batch kernel's run copy serves
    widths up to 8, so the grouped server launches these requests on their
    own after its group kernel.  Mixed with requests of a narrow set, every
    result equals the oracle's list."""
    wide = (1000, 1001, 1002, 1003, 1004, 3, 4, 5, 7)
    narrow = (6, 9, 20)
    with fz.Plan(wide, 1200) as p:
        assert p.d == 9 and p.k == 2 and p.run_order, (p.k, p.run_order)
    with fz.Server(max_in_flight=16, streams=2) as srv:
        w = srv.register(wide, 1200)
        s = srv.register(narrow, 600)
        reqs = [(wide, w, 1200), (narrow, s, 600), (wide, w, 1000), (narrow, s, 0),
                (wide, w, 3), (narrow, s, 599), (wide, w, 1199)]
        ts = [(g, n, srv.submit(sid, n)) for g, sid, n in reqs]
        for g, n, t in ts:
            r = srv.wait(t, 60000)
            assert r.status == fz.FZ_SERVE_DONE, (g, n, r.status)
            assert np.array_equal(rows_of(srv, t, r), oracle.enumerate_desc(g, n)), (g, n)
            srv.release(t)


def test_native_replay(fz):
    """fz_serve_replay submits a stream from native threads: every request
    completes, its row count is the oracle's, latencies are positive, and
    the server is empty afterwards."""
    g1, g2 = (7, 11, 13, 17), (5, 8, 11, 14)
    with fz.Server(max_in_flight=8, streams=2) as srv:
        a = srv.register(g1, 400)
        b = srv.register(g2, 500)
        ids = [a, b] * 20
        ns = [int(x) for x in np.linspace(0, 400, 40)]
        arr = np.arange(40) * 1e-4
        lat, rows, span = srv.replay(ids, ns, arr)
        gs = [g1, g2] * 20
        assert [int(r) for r in rows] == [oracle.count(g, n) for g, n in zip(gs, ns)]
        assert (lat > 0).all() and span > 0
        st = srv.stats()
        assert st.completed == 40 and st.bytes_in_use == 0 and st.queued == 0
