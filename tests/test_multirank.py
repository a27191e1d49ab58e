"""The multi-rank path of the benchmark on the CPU (no GPU): replicas with
their own draws, the slowest rank's time over a gloo process group of two
ranks, and the reference arm under torchrun, where rank 0 alone prints."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _reduce_worker(rank, world, port, out):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        got = bench.reduce_max(10.0 * (rank + 1), dist, "cpu")
        out[rank] = got
    finally:
        dist.destroy_process_group()


def test_reduce_max_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_reduce_worker, args=(2, port, out), nprocs=2, join=True)
        assert dict(out) == {0: 20.0, 1: 20.0}
    assert bench.reduce_max(3.5) == 3.5


@pytest.mark.parametrize("name", ["stabilized20x25", "batch64"])
def test_replicas_draw_their_own_instances(name):
    """Weak scaling: each rank factors its own draws (batch64: its own
    scenarios too) on the same kind of workload."""
    import itertools
    spec = bench.workload_spec(name, None)
    a = list(itertools.islice(bench.iter_patterns(name, 0), 3))
    b = list(itertools.islice(bench.iter_patterns(name, 1), 3))
    assert len(a) == len(b)
    va = next(bench.iter_values(name, a, spec, 0, 0))
    vb = next(bench.iter_values(name, b, spec, 0, 1))
    assert not np.array_equal(va.Sigma, vb.Sigma)
    if name == "batch64":
        assert any(pa.nnz_J != pb.nnz_J for pa, pb in zip(a, b))


def test_reference_arm_under_torchrun_prints_once():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "1", "--workload", "stabilized20x25", "--cpu-budget", "0.2"]
    out = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
