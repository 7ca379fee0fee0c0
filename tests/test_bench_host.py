"""Host-side logic of the benchmark: the replica aggregation over ranks
(world_size 2 over gloo on the CPU), distinct replica inputs per rank, and the
reference arm's JSON line (the CPU oracle on the small workload)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r ran 100 + r iterations in 1 + r seconds
    it, t = bench.whole_job(100 + rank, 1.0 + rank, dist, "cpu", torch)
    out[rank] = (it, t)
    dist.destroy_process_group()


def test_whole_job_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    port = 29500 + (os.getpid() % 2000)
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    # iterations summed over ranks, time of the slowest rank, on every rank
    assert res[0] == res[1] == (201.0, 2.0)


def test_single_rank_whole_job():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.whole_job(7, 0.5, None, "cpu", torch) == (7.0, 0.5)


def test_replicas_draw_distinct_inputs():
    sys.path.insert(0, ROOT)
    import bench
    a, sa = bench.make_system("tiny", 0)
    b, sb = bench.make_system("tiny", 1)
    assert sa != sb and a.m == b.m
    assert not np.array_equal(a.values, b.values)


def test_reference_arm_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "tiny", "--steps", "1", "--warmup", "3"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "iter/s" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["higher_is_better"] is True


def test_captured_traffic_follows_the_kernel_sources(tmp_path, monkeypatch):
    """The roofline's DRAM traffic is read from a committed capture summary
    only while the kernel sources hash to the value recorded beside it."""
    sys.path.insert(0, ROOT)
    import bench
    h = bench.kernel_source_hash()
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "cap.md").write_text(
        "notes\n`traffic: k_aprod2_fused workload=medium dram_bytes_per_launch=1.5e9 "
        "source_sha256=%s`\ntraffic: k_aprod1 workload=medium dram_bytes_per_launch=2e9 "
        "source_sha256=0000000000000000\n" % h)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: h)
    assert bench.captured_traffic("k_aprod2_fused", "medium") == (1.5e9, "profiles/cap.md")
    assert bench.captured_traffic("k_aprod2_fused", "tiny") == (None, None)
    assert bench.captured_traffic("k_aprod1", "medium") == (None, None)  # stale hash
