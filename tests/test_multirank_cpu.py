"""The N > 1 paths of bench.py on CPU: world-size-2 gloo ranks.

The single-instance path runs replicas (no data-path collective); the only
cross-rank step is the timing reduction, max over ranks of the timed region,
and the reference arm runs on rank 0 alone.
"""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, port, out):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=2)
    local_ms = 100.0 if rank == 0 else 250.0  # rank 1 is the slower one
    value, ms = bench.aggregate_over_ranks(local_ms, points_per_rank=1000, steps=4, dist=dist, device="cpu")
    out[rank] = (value, ms)
    dist.barrier()
    dist.destroy_process_group()


def test_value_uses_all_points_and_the_slowest_rank():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(port, out), nprocs=2, join=True)
        res = dict(out)
    for r in (0, 1):
        value, ms = res[r]
        assert ms == 250.0
        assert value == pytest.approx(2 * 1000 * 4 / 0.25)


def test_single_rank_aggregation_is_local():
    import bench
    value, ms = bench.aggregate_over_ranks(50.0, 8, 10)
    assert ms == 50.0 and value == pytest.approx(8 * 10 / 0.05)


@pytest.mark.parametrize("rank", [0, 1])
def test_reference_arm_prints_on_rank0_only(rank):
    env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank), OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--grid", "16", "--steps", "1",
                        "--warmup", "3"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    if rank == 0:
        d = json.loads(lines[-1])
        assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
        assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
    else:
        assert lines == []
