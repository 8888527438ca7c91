"""The N > 1 path of bench.py on the CPU: two gloo ranks (replicas, no
data-path collective).  The job's time is the maximum over ranks and its
work the sum over ranks; the reference arm runs on rank 0 only."""
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench

    t, units = bench._reduce(dist, 10.0 * (rank + 1), 1000.0 + rank)
    q.put((rank, t, units))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_reduction_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, t, units in got:
        assert t == 20.0 and units == 2001.0


def test_reference_arm_runs_on_rank_zero_only(tmp_path):
    """Rank 1 of a two-rank reference run exits 0 without work or output."""
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], env=env, capture_output=True, text=True, timeout=120, cwd=str(tmp_path))
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_profile_traffic_read_from_the_committed_summary():
    """The roofline's traffic figure comes from the committed ncu summary of
    the pair kernel, and only while that summary's source hash is current."""
    import bench

    path = os.path.join(ROOT, "profiles", "pair_kernel_rpy6_n32768.txt")
    vals = dict(line.split(":", 1) for line in open(path) if ":" in line)
    current = vals["kernel_source_sha256_16"].split()[0] == bench.pair_kernel_source_hash()
    t = bench.profile_traffic("rpy6")
    if current:
        assert t == float(vals["dram_bytes_per_launch"].split()[0]) and t > 0
    else:
        assert t is None
