"""The N > 1 host logic of bench.py on CPU with the gloo backend (world size 2).

Replicas are independent (no data-path collective); ranks only meet in a
barrier and in the max-over-ranks reduction of the timed region, and rank 0
alone prints the JSON line.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(
        MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank)
    )
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist

    class Args:
        impl = "reference"

    w, r, lr = bench.init_dist(Args)
    bench.barrier(w)
    got = bench.allmax(w, float(10 * (rank + 1)))
    out.put((rank, w, got))
    dist.destroy_process_group()


def test_allmax_and_barrier_over_two_gloo_ranks():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [(0, 2, 20.0), (1, 2, 20.0)]


def test_reference_arm_under_torchrun_prints_one_line_from_rank_zero():
    port = _free_port()
    cmd = [
        sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
        "--master-addr", "127.0.0.1", "--master-port", str(port),
        "bench.py", "--impl", "reference", "--gpus", "2", "--size", "64", "--steps", "1", "--warmup", "0",
    ]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0


def test_oracle_host_pool_replicas_and_saved_step(tmp_path):
    # bench.py's host-oracle legs: spawned processes, one replica each, aligned by a
    # barrier; replica 0's result is the oracle's step of the same workload.
    sys.path.insert(0, ROOT)
    import bench
    import numpy as np

    import oracle as O

    rate, secs, w = bench.oracle_on_host("hex", 32, 2, 1, workers=2, save_dir=str(tmp_path))
    assert w == 2 and secs > 0
    assert rate == pytest.approx(2 * 3 * 32 * 32 * 2 / secs, rel=1e-12)
    eta, L, h, P = bench._oracle_input("hex", 32)
    for _ in range(3):
        eta, zeta = O.step(eta, 1.0, P, L, h)
    assert np.array_equal(np.load(tmp_path / "eta.npy"), eta)
    assert np.array_equal(np.load(tmp_path / "zeta.npy"), zeta)
