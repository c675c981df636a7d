"""Batched path (reindex_meshes): every mesh's result must be bitwise identical to re-indexing it
alone -- checked against reindex_mesh and against the oracle -- and duplicates must never merge
across meshes."""
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


def concat(meshes):
    K = meshes[0][0].shape[1]
    k = meshes[0][1].shape[1]
    vtx = np.concatenate([m[0] for m in meshes]).reshape(-1, K).astype(np.uint32)
    idx = np.concatenate([m[1] for m in meshes]).reshape(-1, k).astype(np.int32)
    voff = np.concatenate([[0], np.cumsum([m[0].shape[0] for m in meshes])]).astype(np.int64)
    eoff = np.concatenate([[0], np.cumsum([m[1].shape[0] for m in meshes])]).astype(np.int64)
    return vtx, idx, voff, eoff


def run_batched(rx, vtx, idx, voff, eoff):
    out_v, out_off, out_i = rx.reindex_meshes(torch.from_numpy(vtx.view(np.int32)).cuda(), torch.from_numpy(voff).cuda(),
                                              torch.from_numpy(idx).cuda(), torch.from_numpy(eoff).cuda())
    torch.cuda.synchronize()
    return out_v.cpu().numpy().view(np.uint32), out_off.cpu().numpy(), out_i.cpu().numpy()


def check_against_oracle(meshes, out_v, out_off, out_i):
    assert out_off[0] == 0
    for m, (v, i) in enumerate(meshes):
        ov, oi = oracle.reindex_sort(v, i)
        lo, hi = out_off[m], out_off[m + 1]
        assert hi - lo == ov.shape[0], f"mesh {m}: {hi - lo} vs {ov.shape[0]}"
        np.testing.assert_array_equal(out_v[lo:hi], ov)
        e0 = sum(x[1].shape[0] for x in meshes[:m])
        np.testing.assert_array_equal(out_i[e0:e0 + i.shape[0]].reshape(-1), oi)


def random_meshes(rng, n, K, k, with_empty=True):
    meshes = []
    pool = rng.integers(0, 2**32, size=(64, K), dtype=np.uint64).astype(np.uint32)  # shared across meshes
    for m in range(n):
        nv = int(rng.integers(1, 3000))
        ne = int(rng.integers(0, 2000))
        if with_empty and m % 7 == 3:
            ne = 0  # vertices but no elements
        vtx = pool[rng.integers(0, pool.shape[0], size=nv)] if m % 2 else \
            rng.integers(0, 2**32, size=(nv, K), dtype=np.uint64).astype(np.uint32)
        idx = rng.integers(0, nv, size=(ne, k)).astype(np.int32)
        meshes.append((vtx, idx))
    return meshes


@pytest.mark.parametrize("S", [4, 8, 12, 16])
def test_batched_equals_oracle_per_mesh(rx, S):
    rng = np.random.default_rng(100 + S)
    meshes = random_meshes(rng, 37, S // 4, 3)
    out_v, out_off, out_i = run_batched(rx, *concat(meshes))
    check_against_oracle(meshes, out_v, out_off, out_i)


@pytest.mark.parametrize("spec", ["sort=regs,grid=persist", "sort=tiles,swaves=1,pack=off", "sort=tiles,swaves=tile,pack=on",
                                  "sort=chunk,chunk=wide,cgrid=3,dbits=8", "sort=chunk,chunk=small,cgrid=2,dbits=7",
                                  "sort=chunk,chunk=big,dbits=6,rank=match"])
@pytest.mark.parametrize("S", [4, 16])
def test_batched_sort_variants(rx, spec, S):
    """The batched path sorts (S + 4)-byte keys with the variant configured for that key size."""
    saved = rx.reindex_tuning_get(S + 4)
    rx.reindex_tuning_set(S + 4, spec)
    try:
        rng = np.random.default_rng(300 + S)
        meshes = random_meshes(rng, 29, S // 4, 3)
        out_v, out_off, out_i = run_batched(rx, *concat(meshes))
        check_against_oracle(meshes, out_v, out_off, out_i)
    finally:
        rx.reindex_tuning_set(S + 4, saved)


@pytest.mark.parametrize("pub", ["on", "off"])
@pytest.mark.parametrize("S", [4, 8, 12, 16])
def test_batched_dedup_hash(rx, S, pub):
    """Duplicates removed by the hash table before the sort, with the mesh id in the key: every
    mesh equals the oracle, and equal vertices of different meshes (a shared pool, identical meshes)
    never merge."""
    saved = rx.reindex_tuning_get(S + 4)
    rx.reindex_tuning_set(S + 4, f"dedup=hash,dpub={pub}")
    try:
        rng = np.random.default_rng(500 + S)
        meshes = random_meshes(rng, 31, S // 4, 3)
        out_v, out_off, out_i = run_batched(rx, *concat(meshes))
        check_against_oracle(meshes, out_v, out_off, out_i)
        m = synth.heightfield_soup(20, 17, 0.1, seed=3)
        vtx = m.vtx if S == 12 else np.ascontiguousarray(
            np.resize(m.vtx.reshape(-1), (m.vtx.shape[0], S // 4)).astype(np.uint32))
        same = [(vtx, m.idx)] * 5
        out_v, out_off, out_i = run_batched(rx, *concat(same))
        check_against_oracle(same, out_v, out_off, out_i)
    finally:
        rx.reindex_tuning_set(S + 4, saved)


def test_batched_equals_single_calls(rx):
    meshes = [(m.vtx, m.idx) for m in synth.batched_heightfield(24, seed=9, min_tris=64, max_tris=20_000)]
    out_v, out_off, out_i = run_batched(rx, *concat(meshes))
    e0 = 0
    for m, (v, i) in enumerate(meshes):
        sv, sn, si = rx.reindex_mesh(torch.from_numpy(v.view(np.int32)).cuda(), torch.from_numpy(i).cuda())
        torch.cuda.synchronize()
        D = int(sn.item())
        np.testing.assert_array_equal(out_v[out_off[m]:out_off[m + 1]], sv[:D].cpu().numpy().view(np.uint32))
        np.testing.assert_array_equal(out_i[e0:e0 + i.shape[0]], si.cpu().numpy())
        e0 += i.shape[0]


def test_identical_meshes_do_not_merge(rx):
    m = synth.heightfield_soup(20, 17, 0.1, seed=3)
    meshes = [(m.vtx, m.idx)] * 5
    out_v, out_off, out_i = run_batched(rx, *concat(meshes))
    D = 21 * 18
    np.testing.assert_array_equal(out_off, np.arange(6) * D)
    check_against_oracle(meshes, out_v, out_off, out_i)


def test_single_mesh_batch_and_trailing_empty_meshes(rx):
    rng = np.random.default_rng(5)
    v = rng.integers(0, 50, size=(500, 3)).astype(np.uint32)
    i = rng.integers(0, 500, size=(300, 3)).astype(np.int32)
    empty = (np.zeros((0, 3), np.uint32), np.zeros((0, 3), np.int32))
    meshes = [empty, (v, i), empty, empty]
    out_v, out_off, out_i = run_batched(rx, *concat(meshes))
    ov, oi = oracle.reindex_sort(v, i)
    np.testing.assert_array_equal(out_off, [0, 0, ov.shape[0], ov.shape[0], ov.shape[0]])
    check_against_oracle(meshes, out_v, out_off, out_i)


def test_batched_local_index_out_of_range(rx):
    rng = np.random.default_rng(6)
    meshes = random_meshes(rng, 5, 3, 3, with_empty=False)
    vtx, idx, voff, eoff = concat(meshes)
    j = int(eoff[2]) * 3 + 1  # an index of mesh 2, pointing just past its own vertices
    idx.reshape(-1)[j] = int(voff[3] - voff[2])
    rx.reindex_stream_status()
    out_v, out_off, out_i = run_batched(rx, vtx, idx, voff, eoff)
    assert out_off[-1] == -rx.REINDEX_ERR_INDEX_RANGE
    assert rx.reindex_stream_status() == rx.REINDEX_ERR_INDEX_RANGE


def test_batched_bad_offsets(rx):
    rng = np.random.default_rng(7)
    meshes = random_meshes(rng, 4, 3, 3, with_empty=False)
    vtx, idx, voff, eoff = concat(meshes)
    voff[2], voff[1] = voff[1], voff[2] + 1  # decreasing
    rx.reindex_stream_status()
    out_v, out_off, out_i = run_batched(rx, vtx, idx, voff, eoff)
    assert out_off[-1] == -rx.REINDEX_ERR_INVALID_ARG
    assert rx.reindex_stream_status() == rx.REINDEX_ERR_INVALID_ARG


def test_batched_graph_capture_replay(rx):
    meshes = [(m.vtx, m.idx) for m in synth.batched_heightfield(16, seed=11, min_tris=64, max_tris=5_000)]
    vtx, idx, voff, eoff = concat(meshes)
    v, i = torch.from_numpy(vtx.view(np.int32)).cuda(), torch.from_numpy(idx).cuda()
    vo, eo = torch.from_numpy(voff).cuda(), torch.from_numpy(eoff).cuda()
    ws = torch.empty(rx.reindex_meshes_workspace_size(len(meshes), vtx.shape[0], 12, idx.shape[0], 3),
                     dtype=torch.uint8, device="cuda")
    out_v = torch.empty((min(vtx.shape[0], idx.size), 3), dtype=torch.int32, device="cuda")
    out_off = torch.empty(len(meshes) + 1, dtype=torch.int64, device="cuda")
    out_i = torch.empty_like(i)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        rx.reindex_meshes(v, vo, i, eo, ws, out_v, out_off, out_i)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        rx.reindex_meshes(v, vo, i, eo, ws, out_v, out_off, out_i, stream=s)
    out_i.zero_()
    out_off.zero_()
    g.replay()
    torch.cuda.synchronize()
    check_against_oracle(meshes, out_v.cpu().numpy().view(np.uint32), out_off.cpu().numpy(), out_i.cpu().numpy())


# ------------------------------------------------------------------------- device generators


@pytest.mark.parametrize("G,Gy,frac,seed", [(1, 1, 0.0, 1), (7, 3, 0.1, 2), (64, 50, 0.05, 9), (256, 256, 0.10, 1)])
def test_device_heightfield_generator_matches_host(rx, G, Gy, frac, seed):
    m = synth.heightfield_soup(G, Gy, frac, seed)
    v, i = synth.heightfield_soup_gpu(G, Gy, frac, seed)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(v.cpu().numpy().view(np.uint32), m.vtx)
    np.testing.assert_array_equal(i.cpu().numpy(), m.idx)


@pytest.mark.parametrize("L,frac,seed", [(1, 0.0, 3), (5, 0.03, 4), (24, 0.03, 3)])
def test_device_tet_generator_matches_host(rx, L, frac, seed):
    m = synth.tet_soup(L, frac, seed)
    v, i = synth.tet_soup_gpu(L, frac, seed)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(v.cpu().numpy().view(np.uint32), m.vtx)
    np.testing.assert_array_equal(i.cpu().numpy(), m.idx)
