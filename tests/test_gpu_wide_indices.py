"""Index width: int64 index arrays (reindex_mesh64 / reindex_mesh64_ws) and vertex arrays of more
than 2^30 vertices, compared element by element with the serial oracle.

Section 3.5 of the paper expects the method to carry over to other formats; the int64 entry points
take 8-byte index buffers (no 2^31 cap on the index count) and every path accepts up to 2^31 - 1
vertices (31-bit look-back counts)."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SIZES = [(1, 3), (33, 30), (2047, 2047), (2049, 6000), (4097, 4097), (12289, 9000), (70001, 70001),
         (150_000, 40_000)]


@pytest.fixture(scope="module")
def rx():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2109_09812_gb300 import build

    build.build()
    import paper_2109_09812_gb300 as rx

    return rx


def _mesh(rng, n, m, K):
    pool = rng.integers(0, 2**32, size=(max(2, n // 4), K), dtype=np.uint64).astype(np.uint32)
    vtx = pool[rng.integers(0, pool.shape[0], size=n)]
    idx = rng.integers(0, n, size=m).astype(np.int64)
    return vtx, idx


@pytest.mark.parametrize("S", [4, 12, 16, 32])
def test_int64_indices_match_oracle(rx, S):
    rng = np.random.default_rng(500 + S)
    for n, m in SIZES:
        vtx, idx = _mesh(rng, n, m * 3 if n > 1 else 3, S // 4)
        v = torch.from_numpy(vtx.view(np.int32)).cuda()
        i = torch.from_numpy(idx.reshape(-1, 3)).cuda()
        out_v, out_n, out_i = rx.reindex_mesh(v, i)  # int64 indices: reindex_mesh64
        torch.cuda.synchronize()
        assert out_i.dtype == torch.int64
        D = int(out_n.item())
        ov, oi = oracle.reindex_sort(vtx, idx.astype(np.int32))
        assert D == ov.shape[0]
        np.testing.assert_array_equal(out_v[:D].cpu().numpy().view(np.uint32), ov)
        np.testing.assert_array_equal(out_i.cpu().numpy().reshape(-1), oi.astype(np.int64))


@pytest.mark.parametrize("S,pub", [(8, "off"), (12, "on"), (16, "off"), (32, "on")])
def test_int64_indices_hash_path(rx, S, pub):
    """int64 indices with duplicates removed by the hash table before the sort."""
    saved = rx.reindex_tuning_get(S)
    rx.reindex_tuning_set(S, f"dedup=hash,dpub={pub}")
    try:
        _int64_cases(rx, S)
    finally:
        rx.reindex_tuning_set(S, saved)


def _int64_cases(rx, S):
    rng = np.random.default_rng(700 + S)
    for n, m in SIZES:
        vtx, idx = _mesh(rng, n, m * 3 if n > 1 else 3, S // 4)
        v = torch.from_numpy(vtx.view(np.int32)).cuda()
        i = torch.from_numpy(idx.reshape(-1, 3)).cuda()
        out_v, out_n, out_i = rx.reindex_mesh(v, i)
        torch.cuda.synchronize()
        D = int(out_n.item())
        ov, oi = oracle.reindex_sort(vtx, idx.astype(np.int32))
        assert D == ov.shape[0]
        np.testing.assert_array_equal(out_v[:D].cpu().numpy().view(np.uint32), ov)
        np.testing.assert_array_equal(out_i.cpu().numpy().reshape(-1), oi.astype(np.int64))


def test_int64_workspace_variant_in_place(rx):
    rng = np.random.default_rng(7)
    vtx, idx = _mesh(rng, 50_000, 60_000, 3)
    v = torch.from_numpy(vtx.view(np.int32)).cuda()
    i = torch.from_numpy(idx.reshape(-1, 3)).cuda()
    ws = torch.empty(rx.lib().reindex_workspace_size64(v.shape[0], 12, i.shape[0], 3), dtype=torch.uint8,
                     device="cuda")
    out_v, out_n, out_i = rx.reindex_mesh_ws(v, i, ws, out_idx=i)  # in place
    torch.cuda.synchronize()
    ov, oi = oracle.reindex_sort(vtx, idx.astype(np.int32))
    D = int(out_n.item())
    assert D == ov.shape[0] and out_i.data_ptr() == i.data_ptr()
    np.testing.assert_array_equal(out_v[:D].cpu().numpy().view(np.uint32), ov)
    np.testing.assert_array_equal(i.cpu().numpy().reshape(-1), oi.astype(np.int64))


@pytest.mark.parametrize("bad", [-1, 1000, 2**32 + 3, -(2**32), 2**62])
def test_int64_index_out_of_range_is_reported(rx, bad):
    """An int64 index outside [0, nVtx) is an error even when its low 32 bits are in range."""
    rng = np.random.default_rng(9)
    vtx, idx = _mesh(rng, 1000, 3000, 3)
    idx[1234] = bad
    v = torch.from_numpy(vtx.view(np.int32)).cuda()
    i = torch.from_numpy(idx.reshape(-1, 3)).cuda()
    rx.reindex_stream_status()
    out_v, out_n, out_i = rx.reindex_mesh(v, i)
    assert rx.reindex_stream_status() == rx.REINDEX_ERR_INDEX_RANGE
    assert int(out_n.item()) == -rx.REINDEX_ERR_INDEX_RANGE
    idx[1234] = 5
    ov, oi = oracle.reindex_sort(vtx, idx.astype(np.int32))
    i = torch.from_numpy(idx.reshape(-1, 3)).cuda()
    out_v, out_n, out_i = rx.reindex_mesh(v, i)  # the next call is exact again
    torch.cuda.synchronize()
    assert int(out_n.item()) == ov.shape[0]
    np.testing.assert_array_equal(out_i.cpu().numpy().reshape(-1), oi.astype(np.int64))


def _vertex_value(i):
    """Vertex i's 4-byte value: a multiplicative hash reduced to 4,096 values (many duplicates)."""
    return ((np.asarray(i, dtype=np.int64) * 0x9E3779B1) >> 7) & 0xFFF


@pytest.mark.parametrize("wide,words", [(False, 1), (True, 1), (True, 2)])
def test_more_than_2_30_vertices(rx, wide, words):
    """nVtx = 2^30 + 5,000 four-byte vertices (filled on the device), 300,000 indices spread over
    the whole range including both sides of 2^30 and the last vertex.  Only the used vertices
    matter to the result, so the oracle runs on them alone: the referenced vertices' values and the
    indices renumbered to positions in that list (a relabelling that changes neither the unique
    values nor the rank each index resolves to)."""
    n = (1 << 30) + 5000
    rng = np.random.default_rng(31)
    idx = rng.integers(0, n, size=300_000).astype(np.int64)
    idx[:6] = [0, (1 << 30) - 1, 1 << 30, (1 << 30) + 1, n - 1, n - 2]
    ar = torch.arange(n, device="cuda", dtype=torch.int64)
    v = (((ar * 0x9E3779B1) >> 7) & 0xFFF).to(torch.int32).reshape(n, 1)
    del ar
    if words == 2:  # 8-byte vertices (value, 0) on the hash path: owner indices beyond 2^30 in the table
        v = torch.cat([v, torch.zeros_like(v)], dim=1)
    i = torch.from_numpy(idx.reshape(-1, 3) if wide else idx.astype(np.int32).reshape(-1, 3)).cuda()
    saved = rx.reindex_tuning_get(4 * words)
    if words == 2:
        rx.reindex_tuning_set(8, "dedup=hash")
    try:
        out_v, out_n, out_i = rx.reindex_mesh(v, i)
        torch.cuda.synchronize()
    finally:
        rx.reindex_tuning_set(4 * words, saved)
    D = int(out_n.item())
    used, pos = np.unique(idx, return_inverse=True)
    uv = _vertex_value(used).astype(np.uint32).reshape(-1, 1)
    if words == 2:
        uv = np.concatenate([uv, np.zeros_like(uv)], axis=1)
    ov, oi = oracle.reindex_sort(uv, pos.astype(np.int32))
    assert D == ov.shape[0]
    np.testing.assert_array_equal(out_v[:D].cpu().numpy().view(np.uint32), ov)
    np.testing.assert_array_equal(out_i.cpu().numpy().reshape(-1), oi)


@pytest.mark.parametrize("words,tuning", [(1, None), (2, "dedup=hash")])
def test_more_than_2_31_vertices(rx, words, tuning):
    """nVtx = 2^31 + 5,000 vertices (beyond INT32_MAX: re-indexed in vertex ranges of 2^30, then the
    ranges' unique vertices once more), 300,000 int64 indices reaching both sides of every range
    boundary and the last vertex; only 4,096 distinct values, so every range shares keys with the
    others.  The oracle runs on the used vertices alone, relabelled (as for 2^30 + 5,000).  Then one
    index past the end: REINDEX_ERR_INDEX_RANGE."""
    n = (1 << 31) + 5000
    rng = np.random.default_rng(37)
    idx = rng.integers(0, n, size=300_000).astype(np.int64)
    edges = [0, (1 << 30) - 1, 1 << 30, (1 << 30) + 1, (1 << 31) - 1, 1 << 31, (1 << 31) + 1, n - 1, n - 2]
    idx[: len(edges)] = edges
    ar = torch.arange(n, device="cuda", dtype=torch.int64)
    v = (((ar * 0x9E3779B1) >> 7) & 0xFFF).to(torch.int32).reshape(n, 1)
    del ar
    if words == 2:
        v = torch.cat([v, torch.zeros_like(v)], dim=1)
    i = torch.from_numpy(idx.reshape(-1, 3)).cuda()
    S = 4 * words
    saved = rx.reindex_tuning_get(S)
    if tuning:
        rx.reindex_tuning_set(S, tuning)
    try:
        out_v, out_n, out_i = rx.reindex_mesh(v, i)
        torch.cuda.synchronize()
        D = int(out_n.item())
        used, pos = np.unique(idx, return_inverse=True)
        uv = _vertex_value(used).astype(np.uint32).reshape(-1, 1)
        if words == 2:
            uv = np.concatenate([uv, np.zeros_like(uv)], axis=1)
        ov, oi = oracle.reindex_sort(uv, pos.astype(np.int32))
        assert D == ov.shape[0]
        np.testing.assert_array_equal(out_v[:D].cpu().numpy().view(np.uint32), ov)
        np.testing.assert_array_equal(out_i.cpu().numpy().reshape(-1), oi)
        bad = idx.copy()
        bad[4321] = n
        with pytest.raises(rx.ReindexError) as ei:
            rx.reindex_mesh(v, torch.from_numpy(bad.reshape(-1, 3)).cuda())
        assert ei.value.code == rx.REINDEX_ERR_INDEX_RANGE
        rx.reindex_stream_status()  # clear the sticky word
    finally:
        rx.reindex_tuning_set(S, saved)
