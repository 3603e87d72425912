"""The multi-GPU path is replicas only: every rank runs its own chain and the
only collective is the max-over-ranks time. Its host side runs here on CPU
with world_size-2 gloo process groups."""

import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = bench.WORKLOADS["L24_mixed"]
    rp = bench.replica(w, rank)
    slowest = bench.max_over_ranks(10.0 + rank, dist, "cpu")
    out.put((rank, rp["seed"], rp["chain"], slowest))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_seeds_and_max_over_ranks_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, c0, m0), (r1, s1, c1, m1) = res
    assert (s0, c0) != (s1, c1)                 # independent chains
    assert m0 == m1 == 11.0                     # both ranks see the slowest time


def test_reference_arm_under_torchrun_prints_once():
    """`bench.py --impl reference` launched by torchrun with two ranks: rank 0
    alone times the oracle (small workload here) and prints one JSON line."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "L4_fp64",
           "--steps", "1", "--warmup", "0", "--gpus", "2"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    import json
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0


def test_bench_options_are_parsed_and_recorded():
    """`--option key=value` reaches the JSON line's config (reference arm,
    one process, small workload); a malformed option stops the run."""
    import json
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "L4_fp64",
           "--steps", "1", "--warmup", "0", "--option", "pipeline=0", "--option", "metro_reserve=0"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    d = json.loads([ln for ln in r.stdout.splitlines() if ln.startswith("{")][0])
    assert d["config"]["options"] == {"pipeline": 0.0, "metro_reserve": 0.0}
    bad = subprocess.run(cmd[:-2] + ["--option", "pipeline"], capture_output=True, text=True, timeout=600,
                         cwd=ROOT)
    assert bad.returncode != 0 and "key=value" in (bad.stderr + bad.stdout)
