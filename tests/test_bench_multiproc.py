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


def _rec(name, item_bytes=0, skipped=0):
    return {"name": name, "item_bytes": item_bytes, "skipped": skipped, "ms": 0.1, "digit": -1}


def test_path_model_counts_the_kernels_that_ran():
    """The path byte model: a full-key call is the fixed model minus its skipped passes plus the
    digit planes; a prefix-sort call counts its own kernels and nothing after the gate."""
    sys.path.insert(0, ROOT)
    import bench

    N, S, M, U, D = 1000, 12, 900, 900, 300
    W = S + 4
    full = [_rec("clear"), _rec("used_flags"), _rec("compact_hist"), _rec("sort_plan")]
    for p in range(12):
        sk = int(p in (0, 4))
        full += [_rec("tile_count", W, sk), _rec("tile_offsets", W, sk), _rec("chunk_scatter", W, sk)]
    full += [_rec("head_scan"), _rec("remap"), _rec("finalize")]
    got, gated = bench.path_model_bytes(full, N, S, M, U, D)
    want = 4 * M + (N / 8 + N * S + U * W + U) + 10 * (U + 2 * U * W + U) + (U * W + 4 * U + D * S) + 12 * M
    assert gated == 0 and abs(got - want) < 1e-6
    S = 32
    pre = [_rec("clear"), _rec("used_flags"), _rec("key_masks"), _rec("sort_plan"), _rec("compact_hist")]
    pre += [_rec("tile_count", 16), _rec("tile_offsets", 16), _rec("chunk_scatter", 16)] * 8
    pre += [_rec("head_scan"), _rec("prefix_check"), _rec("clear"), _rec("prefix_gate"), _rec("used_flags"),
            _rec("compact_hist"), _rec("sort_plan"), _rec("chunk_scatter", 36), _rec("head_scan"), _rec("remap"),
            _rec("finalize")]
    got, gated = bench.path_model_bytes(pre * 2, N, S, M, U, D)  # two calls
    want = 2 * (4 * M + (N * S + N / 8) + (N / 8 + N * S + 16 * U + U) + 8 * (U + 2 * U * 16 + U)
                + (16 * U + 4 * U + 2 * D * S) + (N / 8 + N * S + 4 * N + D * S) + 12 * M)
    assert gated == 2 * 5 and abs(got - want) < 1e-6


def test_hash_path_models():
    """The hash path: its path bytes count the table clear, the hash kernel, the sort and the head
    scan on the D distinct keys, resolve and remap; the roofline goes to hash_dedup only while it
    takes longer than the radix passes together, and then charges one 32-byte sector per probe and
    per compare on top of the streamed bytes; the sort pass is charged for D items."""
    sys.path.insert(0, ROOT)
    import bench

    N, S, M, U, D = 1000, 12, 900, 900, 150
    W = S + 4
    call = [_rec("clear"), _rec("used_flags"), _rec("clear"), _rec("hash_dedup"), _rec("sort_plan")]
    for p in range(12):
        sk = int(p in (0, 4))
        call += [_rec("tile_count", W, sk), _rec("tile_offsets", W, sk), _rec("chunk_scatter", W, sk)]
    call += [_rec("head_scan"), _rec("resolve"), _rec("remap"), _rec("finalize")]  # (batched-style: a resolve pass)
    got, gated = bench.path_model_bytes(call, N, S, M, U, D)
    slots = bench.dedup_table_slots(N, M)
    assert slots == 2048  # the smallest power of two >= 1.25 * 900 + 1
    want = (4 * M + 4 * slots + (N / 8 + N * S + 4 * (U - D) + D * W + D) + 10 * (D + 2 * D * W + D)
            + (D * W + 4 * D + D * S) + (N / 8 + 4 * U + 8 * (U - D)) + 12 * M)
    assert gated == 0 and abs(got - want) < 1e-6
    # the roofline: hash_dedup dominates when it outlasts the ten passes
    for r in call:
        r["ms"] = 1.0 if r["name"] == "hash_dedup" else 0.01
    roof = bench.step_roofline(call, N, S, M, U, D, 1, "none", 1000.0, "test")
    comp = N / 8 + N * S + 4 * (U - D) + D * (S + 5)
    assert roof["kernel"] == "hash_dedup" and roof["compulsory_bytes_per_launch"] == comp
    assert roof["algorithmic_bytes_per_launch"] == comp + 32 * (2 * U - D)
    assert abs(roof["frac"] - (comp + 32 * (2 * U - D)) / 1e-3 / 1e9 / 1000.0) < 1e-12
    assert roof["sort_pass"]["items_sorted"] == D
    assert roof["sort_pass"]["algorithmic_bytes_per_launch"] == 2 * D * W
    for r in call:
        r["ms"] = 0.5 if r["name"] == "chunk_scatter" else 0.01
    roof = bench.step_roofline(call, N, S, M, U, D, 1, "none", 1000.0, "test")
    assert roof["kernel"] == "chunk_scatter" and roof["items_sorted"] == D


def test_hash_and_prefix_path_model():
    """Hash table plus prefix sort (keys of 12 bytes and wider): the hash kernel writes the
    representatives' bitmask instead of items, the prefix path's kernels count on the D
    representatives, the gated full-key sort counts 0, and the remap adds the copies' second look-up."""
    sys.path.insert(0, ROOT)
    import bench

    N, S, M, U, D = 1000, 32, 900, 900, 150
    call = [_rec("clear"), _rec("used_flags"), _rec("clear"), _rec("hash_dedup"), _rec("sort_plan"),
            _rec("compact_hist")]
    call += [_rec("tile_count", 16), _rec("tile_offsets", 16), _rec("chunk_scatter", 16)] * 8
    call += [_rec("head_scan"), _rec("prefix_check"), _rec("clear"), _rec("prefix_gate"), _rec("used_flags"),
             _rec("compact_hist"), _rec("sort_plan"), _rec("chunk_scatter", 36, 1), _rec("head_scan"),
             _rec("remap"), _rec("finalize")]  # (a gated pass is recorded as skipped)
    got, gated = bench.path_model_bytes(call, N, S, M, U, D)
    want = (4 * M + 4 * bench.dedup_table_slots(N, M) + (N / 8 + N * S + 4 * (U - D) + N / 8)
            + (N / 8 + N * S + 16 * D + D) + 8 * (D + 2 * D * 16 + D) + (16 * D + 4 * D + 2 * D * S)
            + (N / 8 + N * S + 4 * N + D * S) + 12 * M + 4 * (U - D))
    assert gated == 5 and abs(got - want) < 1e-6
    for r in call:
        r["ms"] = 1.0 if r["name"] == "hash_dedup" else 0.01
    roof = bench.step_roofline(call, N, S, M, U, D, 1, "none", 1000.0, "test")
    assert roof["kernel"] == "hash_dedup"
    assert roof["compulsory_bytes_per_launch"] == N / 8 + N * S + 4 * (U - D) + N / 8
    assert roof["sort_pass"]["items_sorted"] == D and roof["sort_pass"]["item_bytes"] == 16
