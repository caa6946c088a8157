"""The multi-rank host path of bench.py on CPU, world size 2 over gloo: the job
time is the slowest rank's (max over ranks), the whole-job rate counts every
rank's units (replicas, weak scaling), and under a two-process launcher the
reference arm prints one line from rank 0 while rank 1 exits without work.
No GPU."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = [120.0, 95.5][rank]                   # each rank's own total time
        job_ms = bench.max_over_ranks(local_ms, world, torch.device("cpu"))
        rate = bench.job_throughput(1920, world, 20, job_ms)
        dist.barrier()
        with open(os.path.join(out, f"r{rank}.json"), "w") as f:
            json.dump({"job_ms": job_ms, "rate": rate}, f)
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_rate_gloo(tmp_path):
    world = 2
    mp.spawn(_rank_main, args=(world, free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / f"r{r}.json")) for r in range(world)]
    for r in res:
        assert r["job_ms"] == 120.0
        assert r["rate"] == pytest.approx(2 * 1920 * 20 / 0.120)


def test_single_rank_helpers():
    assert bench.max_over_ranks(3.5, 1, None) == 3.5
    assert bench.job_throughput(100, 1, 10, 500.0) == pytest.approx(2000.0)


def test_reference_arm_two_ranks_prints_once():
    """bench.py --impl reference under a two-process launcher: rank 0 times the
    oracle and prints one JSON line; rank 1 exits 0 without work."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
           "--steps", "1", "--warmup", "0"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    p = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, p.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"


def test_traffic_record_is_taken_only_for_its_workload_and_sources(tmp_path, monkeypatch):
    """bench.kernel_traffic returns a record's DRAM bytes only when the record
    names the benchmarked workload and its kernel sources are unchanged."""
    src = tmp_path / "k.cu"
    src.write_bytes(b"kernel v1")
    prof = tmp_path / "profiles"
    prof.mkdir()
    import hashlib
    rec = {"workload": "cell_A, one launch", "sources": ["k.cu"],
           "source_sha256": hashlib.sha256(b"kernel v1").hexdigest(),
           "dram_bytes_per_launch": {"mixed": 123.0}}
    (prof / "t.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.kernel_traffic("mixed", "t.json", "cell_A") == 123.0
    assert bench.kernel_traffic("mixed", "t.json", "cell_B") is None
    assert bench.kernel_traffic("fp64", "t.json", "cell_A") is None
    src.write_bytes(b"kernel v2")
    assert bench.kernel_traffic("mixed", "t.json", "cell_A") is None
