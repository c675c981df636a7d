"""The paper's use cases beyond plain duplicate removal (Section 3): merging meshes that share
vertices (3.2) and extracting a subset of a mesh's elements (3.4), each checked bit for bit
against the oracle applied to the construction the paper describes."""
import numpy as np
import pytest

import oracle
from paper_2109_09812_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rx():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2109_09812_gb300 import build

    build.build()
    import paper_2109_09812_gb300 as rx

    return rx


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("S", [4, 8, 12, 16, 20, 24, 32, 48, 64])
def test_merge_equals_concatenate_offset_dedup(rx, S):
    """Section 3.2: concatenate the vertex arrays, add each mesh's vertex offset to its indices,
    then remove duplicates -- here across meshes."""
    rng = np.random.default_rng(S)
    K = S // 4
    pool = rng.integers(0, 2**32, size=(300, K), dtype=np.uint64).astype(np.uint32)  # shared vertices
    meshes = []
    for m in range(9):
        nv = int(rng.integers(1, 2500))
        ne = 0 if m == 4 else int(rng.integers(1, 1500))
        vtx = pool[rng.integers(0, pool.shape[0], size=nv)]
        meshes.append((vtx, rng.integers(0, nv, size=(ne, 3)).astype(np.int32)))
    vtx = np.concatenate([m[0] for m in meshes])
    idx_local = np.concatenate([m[1] for m in meshes])
    voff = np.concatenate([[0], np.cumsum([m[0].shape[0] for m in meshes])]).astype(np.int64)
    eoff = np.concatenate([[0], np.cumsum([m[1].shape[0] for m in meshes])]).astype(np.int64)
    idx_global = np.concatenate([m[1] + voff[j] for j, m in enumerate(meshes)]).astype(np.int32)
    ov, oi = oracle.reindex_sort(vtx, idx_global)
    out_v, out_n, out_i = rx.reindex_merge_meshes(dev(vtx.view(np.int32)), dev(voff), dev(idx_local), dev(eoff))
    torch.cuda.synchronize()
    D = int(out_n.item())
    assert D == ov.shape[0] and D <= 300
    np.testing.assert_array_equal(out_v[:D].cpu().numpy().view(np.uint32), ov)
    np.testing.assert_array_equal(out_i.cpu().numpy().reshape(-1), oi)


def test_merge_of_identical_meshes_is_one_mesh(rx):
    m = synth.heightfield_soup(30, 20, 0.1, seed=4)
    vtx = np.concatenate([m.vtx] * 3)
    idx = np.concatenate([m.idx] * 3)
    voff = np.array([0, m.n_vtx, 2 * m.n_vtx, 3 * m.n_vtx], np.int64)
    eoff = np.array([0, m.n_elem, 2 * m.n_elem, 3 * m.n_elem], np.int64)
    out_v, out_n, out_i = rx.reindex_merge_meshes(dev(vtx.view(np.int32)), dev(voff), dev(idx), dev(eoff))
    torch.cuda.synchronize()
    assert int(out_n.item()) == 31 * 21
    single_v, single_i = oracle.reindex_sort(m.vtx, m.idx)
    np.testing.assert_array_equal(out_i.cpu().numpy(), np.concatenate([single_i.reshape(-1, 3)] * 3))


@pytest.mark.parametrize("keep", [0.0, 0.01, 0.3, 1.0])
def test_submesh_equals_copy_of_selected_elements(rx, keep):
    """Section 3.4: a mesh with the full vertex array but only the selected elements, re-indexed."""
    m = synth.heightfield_soup(80, 70, 0.05, seed=8)
    rng = np.random.default_rng(int(keep * 100))
    sel = np.flatnonzero(rng.random(m.n_elem) < keep).astype(np.int32)
    if keep == 1.0:
        sel = np.concatenate([sel, sel[:17]])  # repeats are allowed and kept
    ov, oi = oracle.reindex_sort(m.vtx, m.idx[sel])
    out_v, out_n, out_i = rx.reindex_submesh(dev(m.vtx.view(np.int32)), dev(m.idx), dev(sel))
    torch.cuda.synchronize()
    D = int(out_n.item())
    assert D == ov.shape[0]
    np.testing.assert_array_equal(out_v[:D].cpu().numpy().view(np.uint32), ov)
    np.testing.assert_array_equal(out_i.cpu().numpy().reshape(-1), oi)


@pytest.mark.parametrize("S", [16, 32])
def test_merge_and_submesh_with_prefix_sort(rx, S):
    """Merging and subset extraction of wide vertices go through the prefix sort (its first pass
    rewrites the indices in place, so the full-key sort, when needed, must see them intact)."""
    meshes = [synth.heightfield_soup_attrs(40, 30, 0.05, seed=3, stride=S)] * 2
    m0 = meshes[0]
    vtx = np.concatenate([m0.vtx, m0.vtx])
    voff = np.array([0, m0.n_vtx, 2 * m0.n_vtx], np.int64)
    eoff = np.array([0, m0.n_elem, 2 * m0.n_elem], np.int64)
    idx = np.concatenate([m0.idx, m0.idx])
    ov, oi = oracle.reindex_sort(vtx, np.concatenate([m0.idx, m0.idx + m0.n_vtx]))
    out_v, out_n, out_i = rx.reindex_merge_meshes(dev(vtx.view(np.int32)), dev(voff), dev(idx), dev(eoff))
    torch.cuda.synchronize()
    D = int(out_n.item())
    assert D == ov.shape[0] == 41 * 31
    np.testing.assert_array_equal(out_v[:D].cpu().numpy().view(np.uint32), ov)
    np.testing.assert_array_equal(out_i.cpu().numpy().reshape(-1), oi)
    # subset of a mesh whose keys share prefixes (few values per word): the full-key sort runs
    rng = np.random.default_rng(S)
    pool = rng.integers(0, 2**32, size=(5, S // 4), dtype=np.uint64).astype(np.uint32)
    wv = pool[rng.integers(0, 5, size=(6000, S // 4)), np.arange(S // 4)]
    widx = rng.integers(0, 6000, size=(4000, 3)).astype(np.int32)
    sel = np.flatnonzero(rng.random(4000) < 0.4).astype(np.int32)
    ov, oi = oracle.reindex_sort(wv, widx[sel])
    out_v, out_n, out_i = rx.reindex_submesh(dev(wv.view(np.int32)), dev(widx), dev(sel))
    torch.cuda.synchronize()
    D = int(out_n.item())
    assert D == ov.shape[0]
    np.testing.assert_array_equal(out_v[:D].cpu().numpy().view(np.uint32), ov)
    np.testing.assert_array_equal(out_i.cpu().numpy().reshape(-1), oi)


@pytest.mark.parametrize("S,pub", [(8, "on"), (12, "off"), (16, "on"), (32, "off")])
def test_merge_and_submesh_hash_path(rx, S, pub):
    """Merging (indices offset into the concatenated vertex array, then the single-mesh hash path)
    and subset extraction with duplicates removed by the hash table first: two identical patches
    merge into one, and a subset equals the oracle on the selected elements."""
    saved = {k: rx.reindex_tuning_get(k) for k in (S, S + 4)}
    for k in saved:
        rx.reindex_tuning_set(k, f"dedup=hash,dpub={pub}")
    try:
        m0 = synth.heightfield_soup_attrs(40, 30, 0.05, seed=4, stride=S) if S >= 12 else None
        if m0 is None:  # 8-byte vertices: x, y of the heightfield soup
            h = synth.heightfield_soup(40, 30, 0.05, seed=4)
            vtx1, idx1 = np.ascontiguousarray(h.vtx[:, :2]), h.idx
        else:
            vtx1, idx1 = m0.vtx, m0.idx
        vtx = np.concatenate([vtx1, vtx1])
        n1, e1 = vtx1.shape[0], idx1.shape[0]
        voff = np.array([0, n1, 2 * n1], np.int64)
        eoff = np.array([0, e1, 2 * e1], np.int64)
        idx = np.concatenate([idx1, idx1])
        ov, oi = oracle.reindex_sort(vtx, np.concatenate([idx1, idx1 + n1]))
        out_v, out_n, out_i = rx.reindex_merge_meshes(dev(vtx.view(np.int32)), dev(voff), dev(idx), dev(eoff))
        torch.cuda.synchronize()
        D = int(out_n.item())
        assert D == ov.shape[0]
        np.testing.assert_array_equal(out_v[:D].cpu().numpy().view(np.uint32), ov)
        np.testing.assert_array_equal(out_i.cpu().numpy().reshape(-1), oi)
        rng = np.random.default_rng(40 + S)
        sel = np.flatnonzero(rng.random(e1) < 0.3).astype(np.int32)
        ov, oi = oracle.reindex_sort(vtx1, idx1[sel])
        out_v, out_n, out_i = rx.reindex_submesh(dev(vtx1.view(np.int32)), dev(idx1), dev(sel))
        torch.cuda.synchronize()
        D = int(out_n.item())
        assert D == ov.shape[0]
        np.testing.assert_array_equal(out_v[:D].cpu().numpy().view(np.uint32), ov)
        np.testing.assert_array_equal(out_i.cpu().numpy().reshape(-1), oi)
    finally:
        for k, t in saved.items():
            rx.reindex_tuning_set(k, t)


def test_submesh_bad_element_id(rx):
    m = synth.heightfield_soup(10, 10, 0.0, seed=2)
    sel = np.array([0, 5, m.n_elem], np.int32)
    rx.reindex_stream_status()
    out_v, out_n, out_i = rx.reindex_submesh(dev(m.vtx.view(np.int32)), dev(m.idx), dev(sel))
    assert rx.reindex_stream_status() == rx.REINDEX_ERR_INDEX_RANGE
    assert int(out_n.item()) == -rx.REINDEX_ERR_INDEX_RANGE


# ------------------------------------------------------------------------------------ autotuner


def test_autotune_keeps_results_exact_and_persists(rx, tmp_path):
    import os
    import subprocess
    import sys

    m = synth.heightfield_soup(400, 300, 0.05, seed=21)
    v, i = dev(m.vtx.view(np.int32)), dev(m.idx)
    cache = tmp_path / "tune.txt"
    os.environ["REINDEX_TUNE_CACHE"] = str(cache)
    try:
        chosen = rx.reindex_autotune(v, i, reps=2)
    finally:
        del os.environ["REINDEX_TUNE_CACHE"]
    assert chosen.startswith("sort=") and "grid=" in chosen
    assert rx.reindex_tuning_get(12) == chosen
    ov, oi = oracle.reindex_sort(m.vtx, m.idx)
    out_v, out_n, out_i = rx.reindex_mesh(v, i)
    torch.cuda.synchronize()
    D = int(out_n.item())
    np.testing.assert_array_equal(out_v[:D].cpu().numpy().view(np.uint32), ov)
    np.testing.assert_array_equal(out_i.cpu().numpy().reshape(-1), oi)
    # explicit settings round-trip, and every variant stays exact
    for spec in ["sort=pipe,rank=match,hist=peel,grid=tile,swaves=tile,pack=on,prefix=off,chunk=wide,cocc=max,cgrid=0,"
                 "dbits=8,dedup=off,dpub=on",
                 "sort=regs,rank=ballot,hist=match,grid=persist,swaves=4,pack=off,prefix=on,chunk=big,cocc=1,cgrid=0,"
                 "dbits=8,dedup=off,dpub=off",
                 "sort=tiles,rank=ballot,hist=uniform,grid=persist,swaves=1,pack=off,prefix=auto,chunk=small,cocc=max,"
                 "cgrid=0,dbits=8,dedup=off,dpub=on",
                 "sort=tiles,rank=vary,hist=uniform,grid=persist,swaves=tile,pack=on,prefix=off,chunk=deep,cocc=max,"
                 "cgrid=0,dbits=8,dedup=off,dpub=on",
                 "sort=chunk,rank=match,hist=uniform,grid=persist,swaves=tile,pack=on,prefix=off,chunk=wide,cocc=1,"
                 "cgrid=4,dbits=7,dedup=hash,dpub=off",
                 "sort=chunk,rank=ballot,hist=uniform,grid=persist,swaves=tile,pack=off,prefix=auto,chunk=big,cocc=max,"
                 "cgrid=0,dbits=6,dedup=off,dpub=on"]:
        rx.reindex_tuning_set(12, spec)
        assert rx.reindex_tuning_get(12) == spec
        out_v, out_n, out_i = rx.reindex_mesh(v, i)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out_i.cpu().numpy().reshape(-1), oi)
    rx.reindex_tuning_set(12, chosen)
    # a new process starts from the cached choice
    assert cache.read_text().strip().endswith("|12|" + chosen)
    code = ("import paper_2109_09812_gb300 as rx, torch; torch.zeros(1, device='cuda'); "
            "print(rx.reindex_tuning_get(12))")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300,
                       env=dict(os.environ, REINDEX_TUNE_CACHE=str(cache)), cwd=os.path.dirname(os.path.dirname(__file__)))
    assert r.stdout.strip().splitlines()[-1] == chosen, r.stderr[-2000:]
