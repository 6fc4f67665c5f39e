"""The N > 1 launch path on CPU: two ranks over gloo (no GPU).

bench.py under torchrun runs one replica per rank and rank 0 alone prints;
times are the maximum over ranks.  These tests run that path with
world_size 2 on the CPU: the reference arm (the oracle, gloo) through
torchrun, the max-over-ranks reduction with two spawned processes, and a
rank that leaves between steps (the other's next collective must end with
an error, not hang).
"""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_reference_arm_two_ranks_prints_one_line():
    env = dict(os.environ)
    env.pop("CUDA_VISIBLE_DEVICES", None)
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", "--master-port=%d" % free_port(),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
           "--steps", "1", "--warmup", "0", "--cpu-seconds", "0.3", "--target", "2000000"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                       timeout=600)
    assert r.returncode == 0, r.stderr.decode()[-2000:]
    lines = [l for l in r.stdout.decode().splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout.decode()
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference" and rec["n_gpus"] == 2
    assert rec["value"] > 0 and rec["cpu_baseline"]["kind"] == "oracle"
    assert rec["e2e"]["h2d_bytes_per_step"] == 0


def _worker(rank, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE="2")
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=2)
    v = bench.max_over_ranks(dist, float(10 * (rank + 1)))
    bench.barrier(dist)
    out.put((rank, v))
    dist.destroy_process_group()


def test_max_over_ranks_gloo():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    ps = [ctx.Process(target=_worker, args=(r, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    got = dict(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got == {0: 20.0, 1: 20.0}


def _leaving_worker(rank, port, out):
    import argparse
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE="2", LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    args = argparse.Namespace(impl="reference", pg_timeout=10.0)
    world, r, _, pg = bench.dist_setup(args)
    assert world == 2 and r == rank
    bench.barrier(pg)  # one step together
    if rank == 1:
        # leaves between steps, with nothing in flight
        out.put((rank, "left"))
        out.close()
        out.join_thread()
        os._exit(3)
    import time
    t0 = time.monotonic()
    try:
        bench.max_over_ranks(pg, 1.0)
        res = "no error"
    except Exception:
        res = "error"
    out.put((rank, res, time.monotonic() - t0))
    out.close()
    out.join_thread()
    os._exit(0)


def test_rank_leaving_ends_the_next_collective():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    ps = [ctx.Process(target=_leaving_worker, args=(r, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    got = {}
    for _ in ps:
        item = q.get(timeout=120)
        got[item[0]] = item[1:]
    for p in ps:
        p.join(timeout=60)
    assert got[1] == ("left",)
    assert got[0][0] == "error", got
    assert got[0][1] < 60.0  # the process-group timeout (10 s) or the closed connection
    assert ps[0].exitcode == 0 and ps[1].exitcode == 3
