"""The N > 1 host path of the benchmark on the CPU: two ranks over gloo (127.0.0.1).

The path shards by independent realisations (one seed per rank, no data-path collective);
the only cross-rank step is the whole-job rate, the updates of all ranks over the slowest
rank's time.  The reference arm prints on rank 0 only.
"""
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        updates = [3.0e9, 5.0e9][rank]
        ms = [120.0, 150.0][rank]
        out[rank] = bench.job_throughput(updates, ms, dist, device="cpu")
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_whole_job_rate_over_two_gloo_ranks():
    world = 2
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_worker, args=(world, free_port(), out), nprocs=world, join=True)
        res = dict(out)
    expect = ((3.0e9 + 5.0e9) / 0.150, 150.0)
    for rank in range(world):
        assert res[rank][0] == pytest.approx(expect[0], rel=1e-12)
        assert res[rank][1] == expect[1]


def test_single_rank_rate_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    v, ms = bench.job_throughput(4.0e9, 200.0)
    assert v == pytest.approx(2.0e10) and ms == 200.0


def test_reference_arm_prints_on_rank_zero_only():
    """Under torchrun the reference arm runs and prints on rank 0; rank 1 exits 0 without
    work (a tiny lattice keeps the oracle's sample short)."""
    outs = []
    for rank in (0, 1):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank))
        r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1",
                            "--warmup", "0", "--Lx", "32", "--Ly", "32"], cwd=ROOT, env=env,
                           capture_output=True, text=True, timeout=300)
        assert r.returncode == 0, r.stderr[-2000:]
        outs.append(r.stdout.strip())
    assert '"impl": "reference"' in outs[0] and '"n_gpus": 2' in outs[0]
    assert outs[1] == ""
