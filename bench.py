"""Throughput benchmark of GB300 mesh re-indexing (input elements re-indexed per second).

Default workload: the 2048 x 2048-cell heightfield triangle soup (8,388,608 triangles, each
emitting its own 3 float32 xyz vertices, plus 5% unreferenced vertices, vertex array randomly
permuted; 26,424,115 vertices, int32 indices, 3 per element), seed 2.

One step = one full pass of the pipeline (used flags, compaction + digit histograms, sort plan,
onesweep radix passes, fused head scan / oldToNew scatter / unique gather, remap) on that mesh.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME]

Prints one JSON line.  `value` is device-resident throughput (inputs already in HBM, workspace
preallocated); `e2e` is the same metric through the host-buffer C entry point with the copies
inside the timed region.  Under torchrun each rank runs an independent replica of the workload
(no collective on the data path); the time is the max over ranks.  `--impl reference` times the
serial CPU oracle on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (description, builder args)
    "heightfield2048": ("heightfield triangle soup 2048x2048 cells (8,388,608 tris, 25,165,824 soup vertices "
                        "float32 xyz + 5% unused = 26,424,115 vertices, permuted), int32 idx x3, seed 2", 2),
    "heightfield256": ("heightfield triangle soup 256x256 cells (131,072 tris, 393,216 soup vertices float32 xyz "
                       "+ 10% unused = 432,538 vertices, permuted), int32 idx x3, seed 1", 1),
    "tet128": ("tetrahedral soup 128^3 hex cells x 5 tets (10,485,760 tets, 41,943,040 soup vertices of 16 B "
               "+ 3% unused = 43,201,331 vertices, permuted), int32 idx x4, seed 3", 3),
    "batched4096": ("4096 independent heightfield triangle soups (float32 xyz, int32 idx x3), triangle counts "
                    "log-uniform in [64, 200000], 0-10% unused vertices each, each permuted, seed 4; one "
                    "reindex_meshes launch sequence replayed as a CUDA graph vs one reindex_mesh_ws call per mesh", 4),
    "serving20000": ("serving: Poisson arrivals of 20,000 re-index requests, element counts log-uniform in "
                     "[1e3, 4e6] (70% heightfield triangle soups, float32 xyz, 3 idx; 30% tet soups, 16-B vertices, "
                     "4 idx), 0-10% unused, generated on the device just before arrival, admitted against a 40 GB "
                     "HBM budget and coalesced into reindex_meshes batches on 2 streams", 5),
    # The paper's own evaluation workload (Section 3.5, Table 1): n x n quads, float2 vertices,
    # 4 corners + 1 unused centre per quad; its GPU times (RTX 3090, thrust + CUDA) are context.
    "quadgrid1024": ("quad grid 1024x1024 (Table 1 workload: 1,048,576 quads, float2 vertices, 5 per quad, "
                     "every fifth unused), int32 idx x4", ("quad", 1024)),
    "quadgrid4096": ("quad grid 4096x4096 (Table 1 workload: 16,777,216 quads, float2 vertices, 5 per quad, "
                     "every fifth unused), int32 idx x4", ("quad", 4096)),
    "quadgrid8192": ("quad grid 8192x8192 (Table 1 workload: 67,108,864 quads, float2 vertices, 5 per quad, "
                     "every fifth unused), int32 idx x4", ("quad", 8192)),
    # The paper's other uses (Section 3): merging meshes and extracting a subset
    "merge16": ("merging (Section 3.2): 16 heightfield soup patches of 512x512 cells (4x4 tiling of the 2048x2048 "
                "field, float32 xyz, 5% unused each, each permuted, seed 2) into one mesh; vertices on shared patch "
                "edges are duplicates across meshes (8,388,608 tris; 2049^2 unique vertices)", ("merge", 512, 4)),
    "submesh30": ("subset (Section 3.4): the 2048x2048 heightfield soup (seed 2) with 30% of its triangles "
                  "selected by a seeded hash, re-indexed against the full vertex array", ("submesh", 0.30)),
    # wider vertices: the 2048^2 soup with attribute words per lattice point (position + 3 normal-like
    # words + 2 texture coordinates = 32 bytes; 24 bytes without the texture coordinates)
    "heightfield2048_s32": ("heightfield triangle soup 2048x2048 cells with 32-byte vertices (float32 xyz + 3 "
                            "normal-like words in [-1,1) + 2 texture coordinates in [0,1), each a hash of the "
                            "position; 25,165,824 soup vertices + 5% unused, permuted), int32 idx x3, seed 2",
                            (2048, 0.05, 2, 32)),
    "heightfield2048_s24": ("heightfield triangle soup 2048x2048 cells with 24-byte vertices (float32 xyz + 3 "
                            "normal-like words in [-1,1), each a hash of the position; 25,165,824 soup vertices "
                            "+ 5% unused, permuted), int32 idx x3, seed 2", (2048, 0.05, 2, 24)),
    "heightfield2048_s64": ("heightfield triangle soup 2048x2048 cells with 64-byte vertices (float32 xyz + 3 "
                            "normal-like words in [-1,1) + 10 more attribute words in [0,1) (texture coordinates, "
                            "tangent...), each a hash of the position; 25,165,824 soup vertices + 5% unused, permuted), "
                            "int32 idx x3, seed 2", (2048, 0.05, 2, 64)),
    "heightfield2048_s48": ("heightfield triangle soup 2048x2048 cells with 48-byte vertices (float32 xyz + 3 "
                            "normal-like words in [-1,1) + 6 more attribute words in [0,1), each a hash of the "
                            "position; 25,165,824 soup vertices + 5% unused, permuted), int32 idx x3, seed 2",
                            (2048, 0.05, 2, 48)),
    "heightfield1448_s32": ("heightfield triangle soup 1448x1448 cells with 32-byte vertices (as heightfield2048_s32), "
                            "for profiler captures", (1448, 0.05, 2, 32)),
    # a half-size case of the 2048^2 workload, for profiler captures (still larger than L2)
    "heightfield1448": ("heightfield triangle soup 1448x1448 cells (4,193,408 tris, 12,580,224 soup vertices "
                        "float32 xyz + 5% unused, permuted), int32 idx x3, seed 2", (1448, 0.05, 2)),
}
METRIC = "input elements re-indexed/sec"
# The paper's GPU times for its quad-grid workload (Table 1), as elements (quads) per second.
PAPER_RATE = {"quadgrid1024": 1048576 / 9.2e-3, "quadgrid4096": 16777216 / 92e-3, "quadgrid8192": 67108864 / 338e-3}
UNIT = "elements/s"


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def source_digest(paths):
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


# The radix-pass kernels (the dominant kernel of a step) and the sources their code comes from.
SORT_KERNEL_SOURCES = {
    "onesweep": ["paper_2109_09812_gb300/csrc/k_onesweep.cu", "paper_2109_09812_gb300/csrc/radix.cuh",
                 "paper_2109_09812_gb300/csrc/common.cuh"],
    "tile_scatter": ["paper_2109_09812_gb300/csrc/k_radix_tiles.cu", "paper_2109_09812_gb300/csrc/radix.cuh",
                     "paper_2109_09812_gb300/csrc/common.cuh"],
    "chunk_scatter": ["paper_2109_09812_gb300/csrc/k_radix_chunk.cu", "paper_2109_09812_gb300/csrc/radix.cuh",
                      "paper_2109_09812_gb300/csrc/tma.cuh", "paper_2109_09812_gb300/csrc/common.cuh"],
    # the duplicate-removal kernel (the dominant kernel when it runs)
    "hash_dedup": ["paper_2109_09812_gb300/csrc/k_dedup.cu", "paper_2109_09812_gb300/csrc/common.cuh"],
}


def ncu_traffic(kernel, workload, item_bytes=None):
    """Per-launch DRAM bytes of a radix-pass kernel from the committed ncu summary
    (profiles/<kernel>_traffic.json), if it was taken on the current kernel source with items of
    the same size (else None)."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
        if rec.get("source_digest") != source_digest(SORT_KERNEL_SOURCES[kernel]):
            return None
        if item_bytes is not None and rec.get("item_bytes") not in (None, item_bytes):
            return None
        return rec.get("per_launch_bytes_full", {}).get(workload)
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms around the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu_index = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu_index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not self.path:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for _, _, r in rows for k in range(4) if r[k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1 and args.impl == "ours":
        import torch.distributed as dist

        backend = "gloo" if args.impl == "reference" else "nccl"
        if backend == "nccl":
            import torch

            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return world, rank, local


def max_over_ranks(x: float, world: int, device=None) -> float:
    """The largest value over all ranks (the slowest rank's time); no-op for one process."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Throughput of the whole job: every rank processed units_per_rank in at most `seconds`."""
    return world * units_per_rank / seconds


def oracle_rate(mesh, repeats=1):
    """Serial oracle (std::sort over (key, index) pairs) on the host: elements/s, seconds."""
    import oracle

    oracle.lib()
    t0 = time.perf_counter()
    for _ in range(repeats):
        oracle.reindex_sort(mesh.vtx, mesh.idx)
    dt = (time.perf_counter() - t0) / repeats
    return mesh.n_elem / dt, dt


def run_reference(args, world, rank):
    """The reference arm: the serial CPU oracle as it stands, on a bounded sample per step."""
    if rank != 0:
        return
    from paper_2109_09812_gb300 import synth

    cfg = WORKLOADS[args.workload][1]
    if args.workload == "batched4096":
        meshes = synth.batched_heightfield(64, seed=4)
        sample = synth.Mesh(vtx=None, idx=None)
        sample_desc = "the first 64 meshes of the 4096-mesh batch (same sizes and seeds), one oracle call each"
    elif isinstance(cfg, tuple) and cfg[0] == "quad":
        qn = min(cfg[1], 1024)
        sample = synth.quad_grid(qn)
        sample_desc = f"quad grid {qn}x{qn}, the same construction ({qn * qn:,} quads)"
    elif isinstance(cfg, tuple) and cfg[0] == "merge":
        sample = usecase_sample(cfg)
        sample_desc = sample.name + " (merging = re-indexing the concatenation with offset indices)"
    elif isinstance(cfg, tuple) and cfg[0] == "submesh":
        sample = usecase_sample(cfg)
        sample_desc = sample.name
    elif isinstance(cfg, tuple) and len(cfg) == 4:
        sample = synth.heightfield_soup_attrs(1024, 1024, cfg[1], cfg[2], stride=cfg[3])
        sample_desc = f"heightfield soup 1024^2 cells with {cfg[3]}-byte vertices, same construction"
    elif isinstance(cfg, tuple):
        sample = synth.heightfield_soup(min(cfg[0], 1024), min(cfg[0], 1024), cfg[1], cfg[2])
        sample_desc = f"heightfield soup {min(cfg[0], 1024)}^2 cells, same construction"
    elif cfg == 3:
        sample = synth.tet_soup(48, 0.03, 3)
        sample_desc = "tetrahedral soup 48^3 cells x 5 tets, same construction (552,960 tets)"
    else:
        g = 1024 if cfg == 2 else 256
        sample = synth.heightfield_soup(g, g, 0.05 if cfg == 2 else 0.10, cfg)
        sample_desc = f"heightfield soup {g}x{g} cells, same construction ({2 * g * g:,} tris)"
    import oracle

    oracle.lib()
    work = [(m.vtx, m.idx) for m in meshes] if args.workload == "batched4096" else [(sample.vtx, sample.idx)]
    n_elem = sum(w[1].shape[0] for w in work)

    def one_step():
        for v, i in work:
            oracle.reindex_sort(v, i)

    for _ in range(args.warmup):
        one_step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        one_step()
    dt = (time.perf_counter() - t0) / args.steps
    value = n_elem / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload][0], "sample": sample_desc},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample_desc + ", serial std::sort oracle, one thread"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def tet_measure(rx, torch, dev, local, steps, autotune=True):
    """The 128^3 tetrahedral soup (16-byte vertices, 4 indices per element), generated on the
    device (bit-identical to the host generator): device-resident step time with the configuration
    the autotuner picks for 16-byte vertices on this mesh (else the default, the prefix sort),
    unique count checked against the closed form."""
    from paper_2109_09812_gb300 import synth

    v, i = synth.tet_soup_gpu(128, 0.03, 3, device=dev)
    v = v.view(torch.int32)
    n_vtx, n_elem = int(v.shape[0]), int(i.shape[0])
    ws = torch.empty(rx.reindex_workspace_size(n_vtx, 16, n_elem, 4), dtype=torch.uint8, device=dev)
    out_v, out_n, out_i = torch.empty_like(v), torch.empty(1, dtype=torch.int64, device=dev), torch.empty_like(i)
    if autotune:
        rx.reindex_autotune(v, i, ws, reps=3)
    for _ in range(3):
        rx.reindex_mesh_ws(v, i, ws, out_v, out_n, out_i)
    torch.cuda.synchronize(dev)
    D = int(out_n.item())
    if D != 129 ** 3:
        raise SystemExit(f"tet soup: unexpected unique count {D}")
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clocks:
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(steps):
            rx.reindex_mesh_ws(v, i, ws, out_v, out_n, out_i)
        e1.record(stream)
        torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / steps
    return {"workload": WORKLOADS["tet128"][0], "ms_per_step": ms, "value": n_elem / (ms / 1e3), "unit": UNIT,
            "unique_out": D, "steps": steps, "tuning": rx.reindex_tuning_get(16), "clocks": clocks.summary()}


class BatchedTuning:
    """Sets a tuning spec for the key sizes of batched calls (S + 4 bytes: mesh id and vertex, for
    4- to 16-byte vertices) and restores the previous settings on exit; spec "default" leaves the
    library's configuration.  The autotuner times single-mesh calls, so batched calls and serving
    are configured here, explicitly; `desc` is the configuration in force for 16-byte keys (12-byte
    vertices), reported with the records."""

    def __init__(self, rx, spec):
        self.rx, self.spec, self.saved = rx, spec, {}

    def __enter__(self):
        if self.spec and self.spec != "default":
            for S in (8, 12, 16, 20):
                self.saved[S] = self.rx.reindex_tuning_get(S)
                self.rx.reindex_tuning_set(S, self.spec)
        self.desc = self.rx.reindex_tuning_get(16)
        return self

    def __exit__(self, *exc):
        for S, t in self.saved.items():
            self.rx.reindex_tuning_set(S, t)
        return False


def batched_measure(rx, torch, dev, local, steps, warmup):
    """Batched path on the 4096-mesh workload (generated on the device, bit-identical to the host
    generator): one CUDA-graph replay of reindex_meshes over all meshes vs one reindex_mesh_ws
    call per mesh (same library, preallocated workspace, one stream).  Returns a dict."""
    import ctypes

    from paper_2109_09812_gb300 import synth

    specs = synth.batched_heightfield_sizes(4096, seed=4)
    parts = [synth.heightfield_soup_gpu(g, gy, uf, sd, device=dev) for (g, gy, uf, sd) in specs]
    nv = np.array([int(v.shape[0]) for v, _ in parts], dtype=np.int64)
    ne = np.array([int(i.shape[0]) for _, i in parts], dtype=np.int64)
    vtx = torch.cat([v for v, _ in parts]).view(torch.int32)
    idx = torch.cat([i for _, i in parts])
    del parts
    voff = np.concatenate([[0], np.cumsum(nv)]).astype(np.int64)
    eoff = np.concatenate([[0], np.cumsum(ne)]).astype(np.int64)
    N, E, k, S = int(voff[-1]), int(eoff[-1]), 3, 12
    vo, eo = torch.from_numpy(voff).to(dev), torch.from_numpy(eoff).to(dev)
    ws = torch.empty(rx.reindex_meshes_workspace_size(len(nv), N, S, E, k), dtype=torch.uint8, device=dev)
    out_v = torch.empty((min(N, E * k), 3), dtype=torch.int32, device=dev)
    out_off = torch.empty(len(nv) + 1, dtype=torch.int64, device=dev)
    out_i = torch.empty_like(idx)
    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        rx.reindex_meshes(vtx, vo, idx, eo, ws, out_v, out_off, out_i, stream=stream)
    torch.cuda.synchronize(dev)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        rx.reindex_meshes(vtx, vo, idx, eo, ws, out_v, out_off, out_i, stream=stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):  # CUDAGraph.replay launches on the current stream
        for _ in range(max(warmup, 1)):
            graph.replay()
        torch.cuda.synchronize(dev)
        with ClockSampler(local) as clocks:
            torch.cuda.synchronize(dev)
            e0.record(stream)
            for _ in range(steps):
                graph.replay()
            e1.record(stream)
            torch.cuda.synchronize(dev)
    ms_batched = e0.elapsed_time(e1) / steps
    D = int(out_off[-1].item())
    if D < 0:
        raise SystemExit(f"batched run reported device error {-D}")

    # one call per mesh through the C ABI (pointers precomputed; one shared workspace)
    L = rx.lib()
    per_ws = torch.empty(max(rx.reindex_workspace_size(int(a), S, int(b), k) for a, b in zip(nv, ne)),
                         dtype=torch.uint8, device=dev)
    pv = torch.empty((N, 3), dtype=torch.int32, device=dev)
    pn = torch.empty(len(nv), dtype=torch.int64, device=dev)
    pi = torch.empty_like(out_i)
    h = ctypes.c_void_p(stream.cuda_stream)
    calls = []
    for m in range(len(nv)):
        calls.append((ctypes.c_void_p(vtx.data_ptr() + int(voff[m]) * S), int(nv[m]), S,
                      ctypes.c_void_p(idx.data_ptr() + int(eoff[m]) * k * 4), int(ne[m]), k,
                      ctypes.c_void_p(pv.data_ptr() + int(voff[m]) * S), ctypes.c_void_p(pn.data_ptr() + 8 * m),
                      ctypes.c_void_p(pi.data_ptr() + int(eoff[m]) * k * 4), ctypes.c_void_p(per_ws.data_ptr()),
                      per_ws.numel(), h))

    def loop():
        for c in calls:
            rc = L.reindex_mesh_ws(*c)
            if rc:
                raise SystemExit(f"reindex_mesh_ws failed: {rc}")

    loop()
    torch.cuda.synchronize(dev)
    loop_steps = max(2, min(steps, 5))
    t0 = time.perf_counter()
    for _ in range(loop_steps):
        loop()
    torch.cuda.synchronize(dev)
    ms_loop = (time.perf_counter() - t0) / loop_steps * 1e3
    # untimed check: every mesh identical in both paths
    counts = pn.cpu().numpy()
    offs = out_off.cpu().numpy()
    same = bool(np.array_equal(np.diff(offs), counts) and torch.equal(out_i, pi))
    if same:
        ov, pv_h = out_v.cpu().numpy(), pv.cpu().numpy()
        same = all(np.array_equal(ov[offs[m]:offs[m + 1]], pv_h[voff[m]:voff[m] + counts[m]]) for m in range(len(nv)))
    return {"n_meshes": int(len(nv)), "n_vtx": N, "n_elem": E, "unique_out": D, "ms_graph_replay": ms_batched,
            "value": E / (ms_batched / 1e3), "unit": UNIT,
            "per_mesh_loop": {"value": E / (ms_loop / 1e3), "unit": UNIT, "ms_per_step": ms_loop,
                              "launch_sequences": int(len(nv))},
            "batched_vs_per_mesh": ms_loop / ms_batched, "identical_results": same,
            "l2": f"inputs larger than L2 ({(N * S + E * k * 4) / 1e9:.2f} GB)", "clocks": clocks.summary()}


def run_batched_bench(args, world, rank, local):
    """Batched path: one CUDA-graph replay of reindex_meshes over all meshes vs one
    reindex_mesh_ws call per mesh (same library, preallocated workspace, one stream)."""
    import torch

    import paper_2109_09812_gb300 as rx
    from paper_2109_09812_gb300 import build as rxbuild

    rxbuild.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    with BatchedTuning(rx, args.batched_tuning) as bt:
        b = batched_measure(rx, torch, dev, local, args.steps, args.warmup)
    line = {
        "metric": METRIC, "value": b["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": b["ms_graph_replay"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic (generated on the device)",
        "config": {"workload": WORKLOADS[args.workload][0], "n_meshes": b["n_meshes"], "n_vtx": b["n_vtx"],
                   "n_elem": b["n_elem"], "unique_out": b["unique_out"], "parallelism": f"replicas x{world}",
                   "l2": b["l2"]},
        "per_mesh_loop": b["per_mesh_loop"], "batched_vs_per_mesh": b["batched_vs_per_mesh"],
        "identical_results": b["identical_results"], "clocks": b["clocks"], "tuning": bt.desc,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def serving_measure(rx, torch, dev, local, n_req, loads, calib_n=2000):
    """Serving: capacity from a closed-loop run of calib_n requests, then open-loop Poisson
    arrivals of the first n_req requests at the given fractions of that capacity; latency =
    completion - arrival (host monotonic clock, as the library's).  Returns a dict."""
    import collections

    from paper_2109_09812_gb300 import synth

    specs = synth.serving_requests(max(n_req, calib_n), seed=5)
    elems = np.array([sp["n_elem"] for sp in specs], dtype=np.float64)
    gen_stream = torch.cuda.Stream(dev)

    def gen(r):
        with torch.cuda.stream(gen_stream):
            v, i = synth.generate_request(specs[r], device=dev, stream=gen_stream)
            ev = torch.cuda.Event()
            ev.record(gen_stream)
        return v.view(torch.int32), i, ev

    def run(rate_rps, n):
        """Submit requests 0..n-1 at Poisson times (rate_rps <= 0: all at once); returns stats."""
        rng = np.random.default_rng(12345)
        gaps = rng.exponential(1.0 / rate_rps, size=n) if rate_rps > 0 else np.zeros(n)
        arrive = np.cumsum(gaps)
        lat, inflight, ahead = [], {}, collections.deque()
        srv = rx.Server(hbm_budget_bytes=40 << 30, max_batch_requests=256, num_streams=2, device=local)
        state = {"done": 0, "last_us": 0.0}

        def take(results):
            for res in results:
                _, _, a = inflight.pop(res["id"])
                if res["status"] != 0:
                    raise SystemExit(f"request failed with status {res['status']}")
                lat.append(res["done_us"] / 1e6 - a)
                state["last_us"] = max(state["last_us"], res["done_us"])
                srv.release(res["id"])
                state["done"] += 1

        try:
            t0 = time.perf_counter()
            nxt = 0
            for r in range(n):
                while nxt < n and nxt < r + 32:  # inputs prepared shortly before they arrive
                    ahead.append((nxt,) + gen(nxt))
                    nxt += 1
                rr, v, i, ev = ahead.popleft()
                while time.perf_counter() - t0 < arrive[r]:
                    take(srv.poll(wait_ms=0))
                ev.synchronize()
                rid = srv.submit(v, i)
                inflight[rid] = (v, i, t0 + arrive[r])
                take(srv.poll(wait_ms=0))
            while state["done"] < n:
                take(srv.poll(wait_ms=20))
            st = srv.stats()
        finally:
            srv.close()
        span = state["last_us"] / 1e6 - t0
        lat_ms = np.array(lat) * 1e3
        return {"requests": n, "elements": float(elems[:n].sum()), "seconds": span,
                "elements_per_s": float(elems[:n].sum() / span), "p50_ms": float(np.percentile(lat_ms, 50)),
                "p99_ms": float(np.percentile(lat_ms, 99)), "max_ms": float(lat_ms.max()),
                "batches": st["batches"], "failed": st["requests_failed"]}

    run(0, min(64, n_req))  # warm-up (kernels, allocator)
    cap = run(0, min(calib_n, len(specs)))
    capacity_eps = cap["elements_per_s"]
    mean_elems = float(elems[:n_req].mean())
    out = {}
    for frac in loads:
        out[f"{frac:.2f}"] = run(frac * capacity_eps / mean_elems, n_req)
    return {"capacity_closed_loop": cap, "loads": out, "mean_elements": mean_elems}


def run_serving_bench(args, world, rank, local):
    """Serving: capacity from a closed-loop run, then open-loop Poisson arrivals at fractions of
    that capacity (the 20,000-request stream by default)."""
    import torch

    import paper_2109_09812_gb300 as rx
    from paper_2109_09812_gb300 import build as rxbuild

    rxbuild.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    with BatchedTuning(rx, args.batched_tuning) as bt:
        m = serving_measure(rx, torch, dev, local, args.requests, [float(x) for x in args.loads.split(",")])
    loads = m["loads"]
    head = loads.get("0.70") or next(iter(loads.values()))
    line = {
        "metric": METRIC, "value": head["elements_per_s"], "unit": UNIT, "n_gpus": world, "steps": 1,
        "warmup": 1, "ms_per_step": head["seconds"] * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic (generated on the device)",
        "config": {"workload": WORKLOADS[args.workload][0], "requests": args.requests,
                   "mean_elements": m["mean_elements"], "parallelism": f"replicas x{world}", "headline_load": 0.7},
        "latency_ms": {"p50": head["p50_ms"], "p99": head["p99_ms"], "max": head["max_ms"]},
        "capacity_closed_loop": m["capacity_closed_loop"], "loads": loads, "tuning": bt.desc,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def build_mesh(workload):
    """(mesh, mesh the CPU baseline times) of a single-mesh workload."""
    from paper_2109_09812_gb300 import synth

    cfg = WORKLOADS[workload][1]
    if isinstance(cfg, tuple) and cfg[0] == "quad":
        # the oracle on 268M used vertices would take minutes: time it on the 2048^2 grid
        return synth.quad_grid(cfg[1]), (synth.quad_grid(min(cfg[1], 2048)) if cfg[1] > 2048 else None)
    if isinstance(cfg, tuple) and len(cfg) == 4:
        # wide vertices, made by the device generators (bit-identical to synth.heightfield_soup_attrs,
        # which is slow on the host at this size); the oracle is timed on 1024^2 cells
        def gen(G):
            import torch

            v, i = synth.heightfield_soup_gpu(G, G, cfg[1], cfg[2])
            w = synth.with_attributes_gpu(v.view(torch.int32), (cfg[3] - 12) // 4, cfg[2])
            return synth.Mesh(vtx=w.cpu().numpy().view(np.uint32), idx=i.cpu().numpy(),
                              name=f"heightfield soup {G}^2 cells, {cfg[3]}-byte vertices",
                              expected_unique=(G + 1) ** 2)

        return gen(cfg[0]), gen(1024)
    if isinstance(cfg, tuple):
        return synth.heightfield_soup(cfg[0], cfg[0], cfg[1], cfg[2]), None
    return synth.config_mesh(cfg), None


def sort_pass_roofline(recs, U):
    """The radix scatter's roofline from the per-launch records: (kernel, algorithmic bytes per
    launch, average launch ms, item bytes, launches).  One pass reads and writes every (key, old
    index) item once: 2 * U * item bytes, averaged over the passes that moved data (a call that
    sorts by key prefix first has 12-byte items in those passes).  U is the number of items sorted:
    the used vertices, or the distinct keys when duplicates were removed first."""
    names = {r["name"] for r in recs}
    kname = next((k for k in ("chunk_scatter", "tile_scatter") if k in names), "onesweep")
    sw = [r for r in recs if r["name"] == kname and not r["skipped"]]
    if not sw:
        return kname, float("nan"), float("nan"), None, 0
    total_bytes = sum(2 * U * r["item_bytes"] for r in sw)
    avg_ms = sum(r["ms"] for r in sw) / len(sw)
    sizes = sorted({r["item_bytes"] for r in sw})
    return kname, total_bytes / len(sw), avg_ms, sizes[0] if len(sizes) == 1 else sizes, len(sw)


def dedup_table_slots(N, M):
    """Slots of the duplicate-removal hash table, as the library sizes it: the smallest power of two
    of at least 1.25 slots per possible used vertex (min(N, M)), and at least 64."""
    umax = min(N, M)
    need, p = umax + umax // 4 + 1, 64
    while p < need:
        p *= 2
    return p


def hash_dedup_bytes(N, S, U, D, repmask=False):
    """Compulsory bytes of one hash_dedup launch: the bitmask N/8 and the vertex array N*S read;
    oldToNew of every copy 4(U-D) written, then either the representatives' items D(S+4) and their
    digit plane D, or (when the prefix path sorts them) the representatives' bitmask N/8."""
    return N / 8 + N * S + 4 * (U - D) + (N / 8 if repmask else D * (S + 4) + D)


def step_roofline(recs, N, S, M, U, D, steps, workload, peak, peak_kind):
    """The dominant kernel's roofline: the radix scatter, or hash_dedup when duplicates are removed
    before the sort and it takes longer than all the radix passes together."""
    dedup = any(r["name"] == "hash_dedup" for r in recs)
    repmask = dedup and any(r["name"] == "prefix_check" for r in recs)  # the prefix path sorts the representatives
    items = D if dedup else U
    kname, alg_bytes, avg_ms, item_bytes, n_sweeps = sort_pass_roofline(recs, items)
    per_pass, count_pass = {}, {}
    for r in recs:
        if r["name"] == kname and not r["skipped"]:
            per_pass.setdefault(f'{r["digit"]}/{r["item_bytes"]}B', []).append(r["ms"])
        if r["name"] == "tile_count" and not r["skipped"]:
            count_pass.setdefault(f'{r["digit"]}/{r["item_bytes"]}B', []).append(r["ms"])
    achieved = alg_bytes / (avg_ms / 1e3) / 1e9
    sort = {"kernel": kname, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "per_pass_ms": {d: round(sum(v) / len(v), 4) for d, v in sorted(per_pass.items())},
            "count_per_pass_ms": {d: round(sum(v) / len(v), 4) for d, v in sorted(count_pass.items())},
            "frac": achieved / peak, "peak_kind": f"{peak_kind} hbm_gbs (copy)",
            "traffic": None if dedup else ncu_traffic(kname, workload, item_bytes),
            "algorithmic_bytes_per_launch": alg_bytes, "item_bytes": item_bytes, "items_sorted": items,
            "avg_launch_ms": avg_ms, "passes_per_step": n_sweeps / steps}
    hd = [r for r in recs if r["name"] == "hash_dedup" and not r["skipped"]]
    sort_ms = sum(r["ms"] for r in recs if r["name"] == kname and not r["skipped"])
    if not hd or sum(r["ms"] for r in hd) <= sort_ms:
        return sort
    h_ms = sum(r["ms"] for r in hd) / len(hd)
    comp = hash_dedup_bytes(N, S, U, D, repmask)
    rand = 32 * (2 * U - D)
    h_bytes = comp + rand
    h_ach = h_bytes / (h_ms / 1e3) / 1e9
    return {"kernel": "hash_dedup", "bound": "hbm", "achieved": h_ach, "peak": peak, "unit": "GB/s",
            "frac": h_ach / peak, "peak_kind": f"{peak_kind} hbm_gbs (copy)",
            "traffic": ncu_traffic("hash_dedup", workload), "algorithmic_bytes_per_launch": h_bytes,
            "avg_launch_ms": h_ms, "launches_per_step": len(hd) / steps,
            "compulsory_bytes_per_launch": comp, "random_sector_bytes_per_launch": rand,
            "compulsory_frac": comp / (h_ms / 1e3) / 1e9 / peak,
            "basis": "streamed bytes (bitmask and vertex array read; copies' oldToNew, and the representatives' "
                     "items and digit plane D(S+5) -- or their bitmask N/8 when the prefix path sorts them -- "
                     "written) plus one random 32-byte sector per table probe (one per used vertex) and per "
                     "key compare (one per copy): N/8 + N*S + 4(U-D) + [D(S+5) | N/8] + 32(2U-D)",
            "sort_pass": sort}


def step_model_bytes(N, S, M, U, D):
    """Bytes a re-indexing step must move under a fixed model: 8-bit digits, all S radix passes
    (no credit for skipped ones), items of W = S + 4 bytes.  Used-flag scatter 4M + N/8; compaction
    N*S + N/8 + U*W; sort 2*S*U*W; run heads, scan, scatter and gather U*W + 4U + D*S; remap 12M."""
    W = S + 4
    return (4 * M + N / 8) + (N * S + N / 8 + U * W) + 2 * S * U * W + (U * W + 4 * U + D * S) + 12 * M


def path_model_bytes(recs, N, S, M, U, D):
    """Algorithmic bytes of the kernels that actually ran (per-launch records of whole calls, in
    launch order), for soups (U = M used vertices, each referenced once).  Full-key path: used flags
    4M; compaction N/8 + N*S + U*W + U (items and the digit plane); per radix pass that moved data
    2*U*w + U (items of w bytes read and written, plane) and U (its digit count reads the plane);
    run heads, scan, scatter and gather U*W + 4U + D*S; remap 12M.  Prefix sort: key masks N*S + N/8;
    compaction into 16-byte records N/8 + N*S + 16U + U; its head scan 16U + 4U + 2*D*S (the run
    heads' whole keys are read from the vertex array); the check N/8 + N*S + 4N + D*S; the full-key
    sort's kernels after the gate count nothing (they return at once when the check passed).
    Returns (bytes in all, launches counted as no-ops after the gate)."""
    W = S + 4
    total, gated_all = 0.0, 0
    calls, cur = [], []
    for r in recs:  # split into calls (each ends with its finalize launch)
        cur.append(r)
        if r["name"] == "finalize":
            calls.append(cur)
            cur = []
    for call in calls:
        prefix = any(r["name"] == "prefix_check" for r in call)
        if any(r["name"] == "hash_dedup" for r in call):
            clears, gated = 0, False
            for r in call:
                if r["name"] == "prefix_gate":
                    gated = True
                    continue
                if gated and r["name"] not in ("remap", "finalize"):
                    gated_all += 1
                    continue
                table = r["name"] == "clear" and clears == 1  # the first clear zeroes the counters
                clears += r["name"] == "clear"
                total += _dedup_launch_bytes(r, table, N, S, W, M, U, D, prefix,
                                             hop2=not any(x["name"] == "resolve" for x in call))
            continue
        gated = False
        for r in call:
            n = r["name"]
            if n == "prefix_gate":
                gated = True
                continue
            if gated and n not in ("remap", "finalize"):
                gated_all += 1
                continue
            total += _launch_bytes(r, n, prefix, N, S, W, M, U, D)
    return total, gated_all


def _dedup_launch_bytes(r, table, N, S, W, M, U, D, prefix=False, hop2=True):
    """Algorithmic bytes of one launch of a call that removed duplicates before the sort: the table
    clear 4*slots (written), hash_dedup (compulsory bytes, hash_dedup_bytes), the sort and the head
    scan on the D distinct keys (with the prefix path: its compaction, 16-byte records, head scan and
    check on the D representatives; the gated full-key sort counts 0), resolve N/8 + 4U + 8(U-D)
    (bitmask, used oldToNew entries, each copy's representative read and its entry rewritten), remap
    12M (+ 4(U-D) for the copies' second look-up when no resolve pass ran)."""
    n = r["name"]
    if r["skipped"]:
        return 0.0
    if n == "clear":
        return 4 * dedup_table_slots(N, M) if table else 0.0
    if n == "hash_dedup":
        return hash_dedup_bytes(N, S, U, D, prefix)
    if n == "resolve":
        return N / 8 + 4 * U + 8 * (U - D)
    if n == "remap":
        return 12 * M + (4 * (U - D) if hop2 else 0)
    return _launch_bytes(r, n, prefix, N, S, W, M, D, D)


def _launch_bytes(r, n, prefix, N, S, W, M, U, D):
    """Algorithmic bytes of one launch (see path_model_bytes); 0 for a radix pass that moved nothing."""
    if r["skipped"]:
        return 0.0
    if n == "used_flags":
        return 4 * M
    if n == "key_masks":
        return N * S + N / 8
    if n == "compact_hist":
        return N / 8 + N * S + (16 * U if prefix else U * W) + U
    if n == "tile_count":
        return U
    if n in ("tile_scatter", "chunk_scatter"):
        return 2 * U * r["item_bytes"] + U
    if n == "onesweep":
        return 2 * U * r["item_bytes"]
    if n == "head_scan":
        return (16 * U + 4 * U + 2 * D * S) if prefix else (U * W + 4 * U + D * S)
    if n == "prefix_check":
        return N / 8 + N * S + 4 * N + D * S
    if n == "remap":
        return 12 * M
    return 0.0


def record_traffic(csv_path, kernel, capture, capture_items):
    """Writes profiles/<kernel>_traffic.json from an ncu CSV log (metrics dram__bytes_read.sum and
    dram__bytes_write.sum of one launch of the radix-pass kernel, captured on a workload sorting
    capture_items 16-byte records, or of hash_dedup on a workload of capture_items used vertices),
    scaled to each full workload by its used vertices, with the digest of the kernel's current
    sources."""
    import csv

    scale = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}
    vals = {}
    with open(csv_path) as f:
        rows = [r for r in csv.reader(f) if len(r) > 5]
    head = rows[0]
    mi, ui, vi = head.index("Metric Name"), head.index("Metric Unit"), head.index("Metric Value")
    for r in rows[1:]:
        if r[mi] in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
            vals[r[mi]] = float(r[vi].replace(",", "")) * scale[r[ui]]
    per = vals["dram__bytes_read.sum"] + vals["dram__bytes_write.sum"]
    full_items = {"heightfield2048": 25165824, "heightfield2048_s24": 25165824, "heightfield2048_s32": 25165824,
                  "tet128": 41943040}
    if kernel == "hash_dedup":  # scales only to a mesh of the same stride and copies per key
        full_items = {"heightfield2048": 25165824}
    rec = {"kernel": kernel, "source_digest": source_digest(SORT_KERNEL_SOURCES[kernel]),
           "item_bytes": None if kernel == "hash_dedup" else 16,
           "capture": capture, "capture_items": capture_items,
           "dram_read_bytes": vals["dram__bytes_read.sum"], "dram_write_bytes": vals["dram__bytes_write.sum"],
           "per_launch_bytes_capture": per,
           "per_launch_bytes_full": {w: round(per * u / capture_items) for w, u in full_items.items()},
           "scaling": (f"traffic grows with the used vertices: x U / {capture_items:,} (the 2048^2 soup's table "
                       "and keys exceed L2 more than the capture's: a lower bound there)") if kernel == "hash_dedup"
           else f"traffic grows with the records sorted: x U / {capture_items:,}"}
    out = os.path.join(ROOT, "profiles", f"{kernel}_traffic.json")
    with open(out, "w") as f:
        json.dump(rec, f, indent=1)
    print(json.dumps(rec))


def merge_patches(P, T, seed=2, unused=0.05):
    """T x T heightfield patches of P x P cells tiling one field: (vtx, vtx_off, idx (local), elem_off)."""
    from paper_2109_09812_gb300 import synth

    meshes = [synth.heightfield_soup(P, P, unused, seed, origin=(P * i, P * j)) for j in range(T) for i in range(T)]
    vtx = np.concatenate([m.vtx for m in meshes])
    idx = np.concatenate([m.idx for m in meshes])
    voff = np.concatenate([[0], np.cumsum([m.n_vtx for m in meshes])]).astype(np.int64)
    eoff = np.concatenate([[0], np.cumsum([m.n_elem for m in meshes])]).astype(np.int64)
    return vtx, voff, idx, eoff


def subset_list(n_elem, frac, seed=2):
    """Sorted element ids selected by a seeded hash (fraction frac)."""
    from paper_2109_09812_gb300 import synth

    u = synth.unit_float(synth.hash_u64(seed, 7, np.arange(n_elem, dtype=np.int64)))
    return np.nonzero(u < np.float32(frac))[0].astype(np.int32)


def usecase_sample(cfg):
    """The bounded oracle sample of a merging / subset workload (a quarter-size instance)."""
    from paper_2109_09812_gb300 import synth

    if cfg[0] == "merge":
        P, T = cfg[1] // 4, cfg[2]
        v, voff, i, eoff = merge_patches(P, T)
        gidx = (i + np.repeat(voff[:-1], np.diff(eoff))[:, None]).astype(np.int32)
        return synth.Mesh(vtx=v, idx=gidx, expected_unique=(P * T + 1) ** 2,
                          name=f"merge of {T * T} patches of {P}^2 cells ({int(i.shape[0]):,} tris)")
    small = synth.heightfield_soup(1024, 1024, 0.05, 2)
    ssel = subset_list(small.n_elem, cfg[1])
    return synth.Mesh(vtx=small.vtx, idx=small.idx[ssel], name=f"heightfield 1024^2 cells with {cfg[1]:.0%} of its "
                      f"triangles ({int(ssel.shape[0]):,} tris)")


def run_usecase(args, world, rank, local):
    """Merging and subset workloads: the same timing, per-kernel breakdown and baselines as the
    single-mesh workloads, through reindex_merge_meshes / reindex_submesh."""
    import torch

    import paper_2109_09812_gb300 as rx
    from paper_2109_09812_gb300 import build as rxbuild
    from paper_2109_09812_gb300 import synth

    if rank == 0 or world == 1:
        rxbuild.build()
    if world > 1:
        torch.distributed.barrier()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    cfg = WORKLOADS[args.workload][1]
    if cfg[0] == "merge":
        P, T = cfg[1], cfg[2]
        vtx_h, voff_h, idx_h, eoff_h = merge_patches(P, T)
        vtx = torch.from_numpy(vtx_h.view(np.int32)).to(dev)
        idx = torch.from_numpy(idx_h).to(dev)
        voff, eoff = torch.from_numpy(voff_h).to(dev), torch.from_numpy(eoff_h).to(dev)
        n_elem, expected = int(idx_h.shape[0]), (P * T + 1) ** 2
        U, S, n_vtx = int(idx_h.size), 12, int(vtx_h.shape[0])
        ws = torch.empty(rx.lib().reindex_merge_workspace_size(T * T, n_vtx, S, n_elem, 3), dtype=torch.uint8, device=dev)
        out_v = torch.empty((min(n_vtx, 3 * n_elem), 3), dtype=torch.int32, device=dev)
        out_n = torch.empty(1, dtype=torch.int64, device=dev)
        out_i = torch.empty_like(idx)
        step = lambda: rx.reindex_merge_meshes(vtx, voff, idx, eoff, ws=ws, out_vtx=out_v, out_nVtx=out_n,
                                               out_idx=out_i)
        sample_mesh = usecase_sample(cfg)
    else:
        mesh = synth.config_mesh(2)
        sel = subset_list(mesh.n_elem, cfg[1])
        vtx = torch.from_numpy(mesh.vtx.view(np.int32)).to(dev)
        idx = torch.from_numpy(mesh.idx).to(dev)
        elist = torch.from_numpy(sel).to(dev)
        n_elem, n_vtx, S = int(sel.shape[0]), mesh.n_vtx, 12
        keys = mesh.vtx.reshape(-1, 3)[mesh.idx[sel].reshape(-1)]
        expected = int(np.unique(keys.view(np.dtype((np.void, 12)))).shape[0])
        U = int(np.unique(mesh.idx[sel].reshape(-1)).shape[0])
        ws = torch.empty(rx.lib().reindex_submesh_workspace_size(n_vtx, S, n_elem, 3), dtype=torch.uint8, device=dev)
        out_v = torch.empty((min(n_vtx, 3 * n_elem), 3), dtype=torch.int32, device=dev)
        out_n = torch.empty(1, dtype=torch.int64, device=dev)
        out_i = torch.empty((n_elem, 3), dtype=torch.int32, device=dev)
        step = lambda: rx.reindex_submesh(vtx, idx, elist, ws=ws, out_vtx=out_v, out_nVtx=out_n, out_idx=out_i)
        sample_mesh = usecase_sample(cfg)
    stream = torch.cuda.current_stream(dev)
    for _ in range(max(args.warmup, 1)):
        step()
    torch.cuda.synchronize(dev)
    D = int(out_n.item())
    if D != expected:
        raise SystemExit(f"unexpected unique count {D} (expected {expected})")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clocks:
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        if world > 1:
            torch.distributed.barrier()
        ms = e0.elapsed_time(e1) / args.steps
        rx.profile_collect()
        rx.profile_enable(True)
        for _ in range(args.steps):
            step()
        torch.cuda.synchronize(dev)
        rx.profile_enable(False)
    recs = rx.profile_collect()
    ms = max_over_ranks(ms, world, dev)
    value = whole_job_rate(n_elem, world, ms / 1e3)
    per_kernel = {}
    for r in recs:
        key = r["name"] + (" (skipped)" if r["skipped"] else "")
        a = per_kernel.setdefault(key, [0, 0.0])
        a[0] += 1
        a[1] += r["ms"]
    peak, peak_kind = load_peaks()
    roofline = step_roofline(recs, n_vtx, S, 3 * n_elem, U, D, args.steps, args.workload, peak, peak_kind)
    if rank != 0:
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        rate, secs = oracle_rate(sample_mesh)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{sample_mesh.name} ({sample_mesh.n_elem:,} elements, {secs:.1f} s), serial std::sort "
                         "oracle, one thread"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload][0], "n_vtx": n_vtx, "n_elem": n_elem, "stride_bytes": S,
                   "idx_per_elem": 3, "unique_out": D, "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2"},
        "roofline": roofline, "cpu_baseline": cpu, "e2e": None, "tuning": rx.reindex_tuning_get(S),
        "gpu_launches": len(recs),
        "kernels": {k_: {"launches": v[0], "ms_per_step": v[1] / args.steps} for k_, v in sorted(per_kernel.items())},
        "clocks": clocks.summary(),
    }
    print(json.dumps(line), flush=True)


def run_ours(args, world, rank, local):
    import torch

    import paper_2109_09812_gb300 as rx
    from paper_2109_09812_gb300 import build as rxbuild
    from paper_2109_09812_gb300 import synth

    if rank == 0 or world == 1:
        rxbuild.build()
    if world > 1:
        torch.distributed.barrier()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    mesh, cpu_sample = build_mesh(args.workload)
    S, k, n_vtx, n_elem = mesh.stride_bytes, mesh.idx_per_elem, mesh.n_vtx, mesh.n_elem
    M = n_elem * k
    U = M  # soups: every soup vertex is referenced exactly once
    vtx = torch.from_numpy(mesh.vtx.view(np.int32)).to(dev)
    idx = torch.from_numpy(mesh.idx).to(dev)
    ws = torch.empty(rx.reindex_workspace_size(n_vtx, S, n_elem, k), dtype=torch.uint8, device=dev)
    out_v = torch.empty((min(n_vtx, M), S // 4), dtype=torch.int32, device=dev)
    out_n = torch.empty(1, dtype=torch.int64, device=dev)
    out_i = torch.empty_like(idx)
    stream = torch.cuda.current_stream(dev)

    tuning = rx.reindex_autotune(vtx, idx, ws, reps=5) if not args.no_autotune else rx.reindex_tuning_get(S)
    for _ in range(max(args.warmup, 1)):
        rx.reindex_mesh_ws(vtx, idx, ws, out_v, out_n, out_i)
    torch.cuda.synchronize(dev)
    D = int(out_n.item())
    if D != mesh.expected_unique:
        raise SystemExit(f"unexpected unique count {D} (expected {mesh.expected_unique})")
    # one call captured into a CUDA graph (the library's workspace variant allocates nothing and
    # never synchronises): a replay issues the whole launch sequence at once, as a caller that
    # re-indexes meshes of one size in a loop would
    graph = None
    if not args.no_graph:
        gs = torch.cuda.Stream(dev)
        gs.wait_stream(stream)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=gs):
            rx.reindex_mesh_ws(vtx, idx, ws, out_v, out_n, out_i, stream=gs)
        stream.wait_stream(gs)
        out_n.fill_(-1)
        graph.replay()
        torch.cuda.synchronize(dev)
        if int(out_n.item()) != D:
            raise SystemExit("graph replay: unexpected unique count")

    # ---- timed region: device-resident inputs (inputs larger than L2)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clocks:
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(args.steps):
            if graph is not None:
                graph.replay()
            else:
                rx.reindex_mesh_ws(vtx, idx, ws, out_v, out_n, out_i)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        if world > 1:
            torch.distributed.barrier()
        ms = e0.elapsed_time(e1) / args.steps
        ms_stream = None
        if graph is not None:  # the same steps launched call by call, for reference
            torch.cuda.synchronize(dev)
            e0.record(stream)
            for _ in range(args.steps):
                rx.reindex_mesh_ws(vtx, idx, ws, out_v, out_n, out_i)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms_stream = e0.elapsed_time(e1) / args.steps
        # the same steps again with a pair of events around every kernel launch: per-kernel
        # durations for the breakdown and the roofline (the events add a little time per launch,
        # so the step time above is taken without them)
        rx.profile_collect()
        rx.profile_enable(True)
        for _ in range(args.steps):
            rx.reindex_mesh_ws(vtx, idx, ws, out_v, out_n, out_i)
        torch.cuda.synchronize(dev)
        rx.profile_enable(False)
    recs = rx.profile_collect()
    ms = max_over_ranks(ms, world, dev)
    value = whole_job_rate(n_elem, world, ms / 1e3)

    # ---- per-kernel breakdown and the dominant kernel's roofline
    per_kernel = {}
    for r in recs:
        key = r["name"] + (" (skipped)" if r["skipped"] else "")
        a = per_kernel.setdefault(key, [0, 0.0])
        a[0] += 1
        a[1] += r["ms"]
    peak, peak_kind = load_peaks()
    roofline = step_roofline(recs, n_vtx, S, M, U, D, args.steps, args.workload, peak, peak_kind)

    # the whole step against two byte models: the fixed one (8-bit digits, all S passes of W-byte
    # items: the full-key method, whatever the call skips) and the bytes the kernels that ran move
    model = step_model_bytes(n_vtx, S, M, U, D)
    path_total, gated = path_model_bytes(recs, n_vtx, S, M, U, D)
    path = path_total / args.steps
    prefix_ran = any(r["name"] == "prefix_check" for r in recs)
    dedup_ran = any(r["name"] == "hash_dedup" for r in recs)
    fixed = {"bytes": model, "achieved": model / (ms / 1e3) / 1e9,
             "frac": None if prefix_ran or dedup_ran else model / (ms / 1e3) / 1e9 / peak,
             "basis": "the full-key method: 8-bit digits, all S passes of (S+4)-byte items"}
    if prefix_ran or dedup_ran:
        fixed["note"] = ("not a roofline here: the " + ("hash-table duplicate removal" if dedup_ran else "prefix sort")
                         + " moves far fewer bytes than the full-key method (see path)")
    step_model = {"path": {"bytes": path, "achieved": path / (ms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                           "frac": path / (ms / 1e3) / 1e9 / peak,
                           "basis": "algorithmic bytes of the kernels that ran in this configuration (passes that "
                                    "moved data, digit planes, prefix check; the gated full-key sort counts 0)",
                           "noop_launches_after_gate_per_step": gated / args.steps},
                  "fixed": fixed,
                  "compulsory_frac": (n_vtx * S + 8 * M + D * S) / (ms / 1e3) / 1e9 / peak}

    # ---- end to end through the host-buffer entry point
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(rx, torch, mesh, world, dev, args)

    # ---- the batched path and the serving loop (the metric's other two parts), on this GPU
    sub = {}
    if world == 1 and args.workload == "heightfield2048" and not args.no_sub:
        sub["tet128"] = tet_measure(rx, torch, dev, local, max(3, min(args.steps, 10)), not args.no_autotune)
        with BatchedTuning(rx, args.batched_tuning) as bt:
            sub["batched"] = batched_measure(rx, torch, dev, local, max(3, min(args.steps, 10)), 3)
            srv = serving_measure(rx, torch, dev, local, args.serving_requests, [0.7], calib_n=args.serving_requests)
        sub["batched"]["tuning"] = bt.desc
        load = srv["loads"]["0.70"]
        sub["serving"] = {"requests": args.serving_requests, "load": 0.7, "mean_elements": srv["mean_elements"],
                          "latency_ms": {"p50": load["p50_ms"], "p99": load["p99_ms"], "max": load["max_ms"]},
                          "elements_per_s": load["elements_per_s"], "batches": load["batches"],
                          "failed": load["failed"], "capacity_closed_loop": srv["capacity_closed_loop"],
                          "stream": "the first requests of the 20,000-request stream (sizes log-uniform in "
                                    "[1e3, 4e6] elements, 70% triangle / 30% tet soups), Poisson arrivals at 0.7 "
                                    "of the closed-loop capacity measured on the same requests",
                          "tuning": bt.desc}
    if rank != 0:
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        rate, secs = oracle_rate(cpu_sample if cpu_sample is not None else mesh)
        what = (f"the same construction at {cpu_sample.name} ({cpu_sample.n_elem:,} elements)" if cpu_sample is not None
                else "the full workload once")
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{what} ({secs:.1f} s), serial std::sort oracle, one thread"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": (value / PAPER_RATE[args.workload]) if args.workload in PAPER_RATE else None,
        "dtype": "u32", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload][0], "n_vtx": n_vtx, "n_elem": n_elem, "stride_bytes": S,
                   "idx_per_elem": k, "unique_out": D, "parallelism": f"replicas x{world}",
                   "l2": f"inputs larger than L2 ({(n_vtx * S + M * 4) / 1e6:.0f} MB read per step)",
                   "launch": ("one CUDA graph replay per step (one reindex_mesh_ws call, captured once)"
                              if graph is not None else "one reindex_mesh_ws call per step")},
        "ms_per_step_stream_launched": ms_stream,
        "roofline": roofline, "step_model": step_model, "cpu_baseline": cpu, "e2e": e2e, "tuning": tuning,
        **sub,
        "gpu_launches": len(recs),
        "kernels": {k_: {"launches": v[0], "ms_per_step": v[1] / args.steps} for k_, v in sorted(per_kernel.items())},
        "clocks": clocks.summary(),
    }
    print(json.dumps(line), flush=True)


def run_e2e(rx, torch, mesh, world, dev, args):
    """Same metric through reindex_mesh_host: pinned host buffers in, results back in host memory."""
    S, M, n_vtx, n_elem = mesh.stride_bytes, mesh.n_elem * mesh.idx_per_elem, mesh.n_vtx, mesh.n_elem
    hv = torch.from_numpy(mesh.vtx.view(np.int32)).pin_memory()
    hi = torch.from_numpy(mesh.idx).pin_memory()
    ho_v = torch.empty((min(n_vtx, M), S // 4), dtype=torch.int32).pin_memory()
    ho_i = torch.empty_like(hi).pin_memory()
    for _ in range(2):
        rx.reindex_mesh_host(hv, hi, ho_v, ho_i)
    if world > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    e2e_steps = max(3, min(args.steps, 10))
    for _ in range(e2e_steps):
        rv, _ = rx.reindex_mesh_host(hv, hi, ho_v, ho_i)
    e2e_s = max_over_ranks((time.perf_counter() - t0) / e2e_steps, world, dev)
    return {"value": whole_job_rate(n_elem, world, e2e_s), "unit": UNIT, "h2d_bytes_per_step": n_vtx * S + M * 4,
            "d2h_bytes_per_step": rv.shape[0] * S + M * 4 + 8, "ms_per_step": e2e_s * 1e3}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="heightfield2048")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--requests", type=int, default=20000, help="serving workload: number of requests")
    ap.add_argument("--loads", default="0.5,0.7,0.9", help="serving workload: offered loads (fractions of capacity)")
    ap.add_argument("--no-sub", action="store_true", help="default workload: skip the batched and serving records")
    ap.add_argument("--no-graph", action="store_true",
                    help="time the call launched on the stream each step instead of a captured CUDA graph's replay")
    ap.add_argument("--batched-tuning", default="dedup=hash,dpub=off",
                    help="tuning spec of batched calls and serving (keys of 8-20 bytes), or 'default'")
    ap.add_argument("--serving-requests", type=int, default=2000,
                    help="default workload: requests of the serving record")
    ap.add_argument("--record-traffic", default=None,
                    help="write profiles/<--traffic-kernel>_traffic.json from this ncu CSV log and exit")
    ap.add_argument("--traffic-kernel", default="chunk_scatter")
    ap.add_argument("--traffic-capture", default="heightfield1448, one pass")
    ap.add_argument("--traffic-items", type=int, default=12580224)
    args = ap.parse_args()
    if args.record_traffic:
        record_traffic(args.record_traffic, args.traffic_kernel, args.traffic_capture, args.traffic_items)
        return
    world, rank, local = dist_setup(args)
    try:
        if args.impl == "reference":
            run_reference(args, world, rank)
        elif args.workload == "batched4096":
            run_batched_bench(args, world, rank, local)
        elif args.workload == "serving20000":
            run_serving_bench(args, world, rank, local)
        elif args.workload in ("merge16", "submesh30"):
            run_usecase(args, world, rank, local)
        else:
            run_ours(args, world, rank, local)
    finally:
        if world > 1 and args.impl == "ours":
            import torch.distributed as dist

            dist.destroy_process_group()


if __name__ == "__main__":
    main()
