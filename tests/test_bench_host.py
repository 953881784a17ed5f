"""Host-side checks of bench.py (no GPU): the JSON contract of the
reference arm (the FP64 oracle on the host cores), the silent non-zero
ranks under torchrun, and the max-over-ranks timing reduction with two
gloo processes (the replicas-only multi-GPU mode)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(args, env=None, timeout=600):
    e = dict(os.environ)
    e.update(env or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, capture_output=True,
                          text=True, env=e, timeout=timeout, cwd=ROOT)


def test_reference_arm_prints_one_json_line():
    r = _run(["--impl", "reference", "--steps", "1", "--warmup", "0", "--workload", "advection2d_sine_16x16_N3"])
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["config"]["workload"] == "advection2d_sine_16x16_N3"


def test_reference_arm_other_ranks_are_silent():
    r = _run(["--impl", "reference", "--steps", "1", "--warmup", "0"], env={"WORLD_SIZE": "2", "RANK": "1"})
    assert r.returncode == 0 and r.stdout.strip() == ""


def _rank(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    q.put((rank, bench._max_over_ranks(10.0 + 7.0 * rank, world, device="cpu")))
    dist.destroy_process_group()


def test_max_over_ranks_with_two_gloo_processes():
    import multiprocessing as mp
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    got = dict(q.get(timeout=5) for _ in range(2))
    assert got == {0: 17.0, 1: 17.0}


def _rank_failing(rank, world, port, q):
    """Rank 1 fails before the collective; rank 0 must get an error from the
    process group's timeout instead of waiting forever."""
    import datetime

    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=5))
    if rank == 1:
        q.put((1, "raised"))
        raise SystemExit(3)  # the failing rank leaves between steps
    import bench
    try:
        bench._max_over_ranks(1.0, world, device="cpu")
        q.put((0, "returned"))
    except Exception as e:  # the collective fails on the host, nothing hangs
        q.put((0, "error: " + type(e).__name__))


def test_a_failing_rank_surfaces_as_an_error_not_a_hang():
    import multiprocessing as mp
    import socket
    import time
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_rank_failing, args=(r, 2, port, q)) for r in range(2)]
    t0 = time.time()
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
    got = dict(q.get(timeout=5) for _ in range(2))
    assert ps[1].exitcode == 3
    assert got[1] == "raised" and got[0].startswith("error"), got
    assert time.time() - t0 < 100
