"""The benchmark's multi-process path on the CPU (gloo, world size 2): the time reported is the
slowest rank's and the throughput is the whole job's; under torchrun the reference arm prints one
line from rank 0 while the other ranks exit without work."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        slowest = bench.max_over_ranks(10.0 + 5.0 * rank, world)  # rank 1 is the slow one
        rate = bench.whole_job_rate(1000.0, world, slowest)
        with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
            json.dump({"slowest": slowest, "rate": rate}, f)
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate_gloo(tmp_path):
    import torch.multiprocessing as mp

    port = free_port()
    mp.spawn(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        got = json.load(open(tmp_path / f"r{r}.json"))
        assert got["slowest"] == 15.0
        assert got["rate"] == pytest.approx(2 * 1000.0 / 15.0)


def test_reference_arm_under_torchrun_prints_one_line():
    port = free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
           "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"), "--impl", "reference",
           "--workload", "heightfield256", "--steps", "1", "--warmup", "0", "--gpus", "2"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"


def test_sort_pass_roofline_weighs_each_pass_by_its_item_size():
    """The dominant kernel's algorithmic bytes come from each launch's own item size (a call that
    sorts by key prefix first moves 16-byte records, then maybe whole (S+4)-byte items); skipped
    passes do not count."""
    sys.path.insert(0, ROOT)
    import bench

    U = 1000
    recs = [dict(name="tile_scatter", skipped=False, ms=1.0, item_bytes=16) for _ in range(8)]
    recs += [dict(name="tile_scatter", skipped=True, ms=0.01, item_bytes=36) for _ in range(32)]
    recs += [dict(name="head_scan", skipped=False, ms=5.0, item_bytes=0)]
    kname, per_launch, avg_ms, item_bytes, n = bench.sort_pass_roofline(recs, U)
    assert (kname, per_launch, avg_ms, item_bytes, n) == ("tile_scatter", 2 * U * 16, 1.0, 16, 8)
    recs[8]["skipped"] = False  # one whole-key pass moved data too
    recs[8]["ms"] = 2.0
    kname, per_launch, avg_ms, item_bytes, n = bench.sort_pass_roofline(recs, U)
    assert n == 9 and item_bytes == [16, 36]
    assert per_launch == (8 * 2 * U * 16 + 2 * U * 36) / 9 and avg_ms == 10.0 / 9
    kname, *_ = bench.sort_pass_roofline([dict(name="onesweep", skipped=False, ms=1.0, item_bytes=16)], U)
    assert kname == "onesweep"
