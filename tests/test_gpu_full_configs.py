"""Element-by-element oracle parity at the full batched and serving workloads.

- The 4096-mesh batch (heightfield triangle soups of 64 .. 200,000 triangles, 0-10 % unused
  vertices each, generated on the device): one CUDA-graph replay of reindex_meshes, then every
  mesh's unique vertices, their count and every remapped index against the serial oracle on that
  mesh alone (meshes stay independent: Section 3.2 is the opposite, merging, use).
- The serving mix (triangle soups with 12-byte vertices and tet soups with 16-byte vertices,
  1,000 .. 4,000,000 elements, 0-10 % unused): a few hundred requests, including the smallest and
  the largest of each class, submitted to the server at Poisson arrival times so that batches
  overlap on the device; every request's result against the oracle on that request alone.

The oracle calls run in host threads (the C oracle holds no global state and ctypes releases the
interpreter lock during each call).
"""
import concurrent.futures as cf
import os
import time

import numpy as np
import pytest

import oracle
from paper_2109_09812_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

THREADS = max(1, min(32, os.cpu_count() or 1))


@pytest.fixture(scope="module")
def rx():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2109_09812_gb300 import build

    build.build()
    import paper_2109_09812_gb300 as rx

    oracle.lib()
    return rx


def _compare(job):
    """(name, vtx words, idx, gpu unique vertices, gpu indices) -> None, or a message."""
    name, vtx, idx, gv, gi = job
    ov, oi = oracle.reindex_sort(vtx, idx)
    if gv.shape[0] != ov.shape[0]:
        return f"{name}: D {gv.shape[0]} vs oracle {ov.shape[0]}"
    if not np.array_equal(gv, ov):
        return f"{name}: unique vertices differ"
    if not np.array_equal(gi.reshape(-1), oi):
        return f"{name}: indices differ"
    return None


def _run_jobs(jobs):
    with cf.ThreadPoolExecutor(THREADS) as ex:
        bad = [m for m in ex.map(_compare, jobs) if m]
    assert not bad, f"{len(bad)} mismatches, first: {bad[:3]}"


@pytest.mark.parametrize("tuning", [None, "dedup=hash,dpub=off"])
def test_batched_4096_meshes_match_oracle_mesh_by_mesh(rx, tuning):
    """All 4,096 meshes after one graph replay, each against the oracle; with the library's
    default configuration for 16-byte (mesh id, vertex) keys, and with duplicates removed by the
    hash table first."""
    saved = rx.reindex_tuning_get(16)
    if tuning:
        rx.reindex_tuning_set(16, tuning)
    try:
        _batched_4096(rx)
    finally:
        rx.reindex_tuning_set(16, saved)


def _batched_4096(rx):
    specs = synth.batched_heightfield_sizes(4096, seed=4)
    parts = [synth.heightfield_soup_gpu(g, gy, uf, s) for (g, gy, uf, s) in specs]
    nv = np.array([int(v.shape[0]) for v, _ in parts], dtype=np.int64)
    ne = np.array([int(i.shape[0]) for _, i in parts], dtype=np.int64)
    vtx = torch.cat([v for v, _ in parts]).view(torch.int32)
    idx = torch.cat([i for _, i in parts])
    del parts
    voff_h = np.concatenate([[0], np.cumsum(nv)]).astype(np.int64)
    eoff_h = np.concatenate([[0], np.cumsum(ne)]).astype(np.int64)
    voff, eoff = torch.from_numpy(voff_h).cuda(), torch.from_numpy(eoff_h).cuda()
    N, E = int(voff_h[-1]), int(eoff_h[-1])
    assert len(specs) == 4096 and E > 50_000_000  # the full workload, not a sample
    ws = torch.empty(rx.reindex_meshes_workspace_size(4096, N, 12, E, 3), dtype=torch.uint8, device="cuda")
    out_v = torch.empty((min(N, 3 * E), 3), dtype=torch.int32, device="cuda")
    out_off = torch.empty(4097, dtype=torch.int64, device="cuda")
    out_i = torch.full_like(idx, -1)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):  # warm-up outside the capture
        rx.reindex_meshes(vtx, voff, idx, eoff, ws, out_v, out_off, out_i, stream=stream)
    torch.cuda.synchronize()
    out_i.fill_(-1)
    out_off.fill_(-7)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        rx.reindex_meshes(vtx, voff, idx, eoff, ws, out_v, out_off, out_i, stream=stream)
    with torch.cuda.stream(stream):
        graph.replay()
    torch.cuda.synchronize()
    offs = out_off.cpu().numpy()
    assert offs[0] == 0 and offs[-1] > 0
    gv_all = out_v[: int(offs[-1])].cpu().numpy().view(np.uint32)
    gi_all = out_i.cpu().numpy()
    v_all = vtx.cpu().numpy().view(np.uint32)
    i_all = idx.cpu().numpy()
    jobs = [(f"mesh {m}", v_all[voff_h[m]:voff_h[m + 1]], i_all[eoff_h[m]:eoff_h[m + 1]],
             gv_all[offs[m]:offs[m + 1]], gi_all[eoff_h[m]:eoff_h[m + 1]]) for m in range(4096)]
    _run_jobs(jobs)


def _serving_sample(n_pick=256):
    """Specs from the 20,000-request stream: the smallest and largest request of each class, then
    the first requests in arrival order up to n_pick."""
    specs = synth.serving_requests(20000, seed=5)
    pick = set()
    for kind in ("tri", "tet"):
        ks = [r for r, sp in enumerate(specs) if sp["kind"] == kind]
        ks.sort(key=lambda r: specs[r]["n_elem"])
        pick.update(ks[:2] + ks[-2:])
    r = 0
    while len(pick) < n_pick:
        pick.add(r)
        r += 1
    return [specs[r] for r in sorted(pick)]


@pytest.mark.parametrize("tuning", [None, "dedup=hash"])
def test_serving_mix_matches_oracle_request_by_request(rx, tuning):
    """256 requests of the serving mix at Poisson arrivals, each against the oracle; with the default
    configuration, and with duplicates removed by the hash table first (keys of 16 and 20 bytes:
    triangle and tet requests with their mesh ids)."""
    saved = {S: rx.reindex_tuning_get(S) for S in (16, 20)}
    if tuning:
        for S in saved:
            rx.reindex_tuning_set(S, tuning)
    try:
        _serving_mix(rx)
    finally:
        for S, t in saved.items():
            rx.reindex_tuning_set(S, t)


def _serving_mix(rx):
    specs = _serving_sample()
    assert {sp["kind"] for sp in specs} == {"tri", "tet"}
    sizes = [sp["n_elem"] for sp in specs]
    assert min(sizes) < 2_000 and max(sizes) > 3_000_000
    reqs = []
    for sp in specs:
        v, i = synth.generate_request(sp)
        reqs.append((v.view(torch.int32), i))
    torch.cuda.synchronize()
    rng = np.random.default_rng(5)
    gaps = rng.exponential(1.0 / 2000.0, size=len(reqs))  # ~2,000 requests/s: batches overlap
    results = {}
    with rx.Server(hbm_budget_bytes=40 << 30, max_batch_requests=256, num_streams=2) as srv:
        ids = []
        t0 = time.perf_counter()
        due = np.cumsum(gaps)
        for r, (v, i) in enumerate(reqs):
            while time.perf_counter() - t0 < due[r]:
                time.sleep(0.0001)
            ids.append(srv.submit(v, i))
        deadline = time.time() + 600
        while len(results) < len(ids):
            for res in srv.poll(wait_ms=50):
                assert res["status"] == 0, f"request {res['id']} failed: {res['status']}"
                results[res["id"]] = (res["out_vtx"].cpu().numpy().view(np.uint32),
                                      res["out_idx"].cpu().numpy())
                srv.release(res["id"])
            assert time.time() < deadline, f"only {len(results)} of {len(ids)} finished"
        st = srv.stats()
        assert st["requests_failed"] == 0 and st["batches"] >= 2
    jobs = []
    for rid, (v, i) in zip(ids, reqs):
        gv, gi = results[rid]
        jobs.append((f"request {rid}", v.cpu().numpy().view(np.uint32), i.cpu().numpy(), gv, gi))
    _run_jobs(jobs)
