"""The multi-process path of bench.py on CPU (gloo, world size 2): the path
shards into independent replicas (one right-hand side per rank, no
data-path collective), so the only cross-rank step is the timing reduction.
Checks the max-over-ranks reduction and whole-job throughput, and that the
reference arm under torchrun prints one line from rank 0 while rank 1 exits
cleanly without work."""

import importlib.util
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    b = _bench()
    out = b.max_over_ranks([1.0 + rank, 10.0 * rank, 5.0], dist, device="cpu")
    q.put((rank, out, b.replica_throughput(3, max(out[0], 1.0), world)))
    dist.destroy_process_group()


def test_max_over_ranks_gloo():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = [q.get(timeout=120) for _ in ps]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, out, thr in res:
        assert out == [2.0, 10.0, 5.0]
        assert thr == pytest.approx(3 * 2 / 2.0)


def test_single_process_is_identity():
    b = _bench()
    assert b.max_over_ranks([3.5, 1.0]) == [3.5, 1.0]
    assert b.replica_throughput(5, 2.0, 1) == 2.5


def test_reference_arm_under_torchrun():
    env = dict(os.environ)
    env["OMP_NUM_THREADS"] = "4"
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
           "127.0.0.1", "--master-port", str(_free_port()), os.path.join(ROOT, "bench.py"), "--impl", "reference",
           "--gpus", "2", "--steps", "2", "--warmup", "0", "--ref-chunk", "1"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0
