"""Bit-exact parity of the CUDA path (through the C ABI) with the serial oracle.

Every comparison is element by element on the same seeded inputs: the unique vertex array,
its length D and every remapped index.  Sizes straddle the kernels' tiles (2048 vertices per
compaction tile, 4096 items per sort and head-scan tile) and end in ragged tails.
"""
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


def to_dev(vtx_words: np.ndarray, idx: np.ndarray):
    v = torch.from_numpy(np.ascontiguousarray(vtx_words).view(np.int32)).cuda()
    i = torch.from_numpy(np.ascontiguousarray(idx, dtype=np.int32)).cuda()
    return v, i


def run_gpu(rx, vtx_words, idx, k=None):
    idx2 = idx.reshape(-1, k) if k else (idx if idx.ndim == 2 else idx.reshape(-1, 1))
    v, i = to_dev(vtx_words, idx2)
    out_v, out_n, out_i = rx.reindex_mesh(v, i)
    torch.cuda.synchronize()
    D = int(out_n.item())
    return D, out_v[: max(D, 0)].cpu().numpy().view(np.uint32), out_i.cpu().numpy().reshape(-1)


def assert_parity(rx, vtx_words, idx, k=None):
    ov, oi = oracle.reindex_sort(vtx_words, idx)
    D, gv, gi = run_gpu(rx, vtx_words, idx, k)
    assert D == ov.shape[0], f"D: gpu {D} vs oracle {ov.shape[0]}"
    np.testing.assert_array_equal(gv, ov)
    np.testing.assert_array_equal(gi, oi)
    return D


def random_mesh(rng, n, m, K, mode):
    if mode == "random":
        vtx = rng.integers(0, 2**32, size=(n, K), dtype=np.uint64).astype(np.uint32)
    elif mode == "dups":  # few distinct values per word -> many duplicates, all digits vary
        pool = rng.integers(0, 2**32, size=(7,), dtype=np.uint64).astype(np.uint32)
        vtx = pool[rng.integers(0, 7, size=(n, K))]
    elif mode == "floats":  # +-0, NaN payloads, negatives, integers
        pool = np.array([0x00000000, 0x80000000, 0x7FC00000, 0x7FC00001, 0xBF800000, 0x3F800000, 0x40400000],
                        dtype=np.uint32)
        vtx = pool[rng.integers(0, len(pool), size=(n, K))]
    elif mode == "hibyte":  # lowest key byte constant, varying bits in several runs per word
        vtx = (rng.integers(0, 2**32, size=(n, K), dtype=np.uint64).astype(np.uint32) & np.uint32(0xF0F0FF00))
        vtx |= np.uint32(0x00000A05)
    else:  # "const": a few constant words -> trivial radix passes get skipped
        vtx = np.zeros((n, K), dtype=np.uint32)
        vtx[:, -1] = rng.integers(0, 300, size=n).astype(np.uint32)
    idx = rng.integers(0, n, size=m).astype(np.int32)
    return vtx, idx


SIZES = [(1, 3), (2, 4), (33, 30), (2047, 2047), (2049, 6000), (4096, 4096), (4097, 4097), (12289, 9000),
         (70001, 70001), (150_000, 40_000)]


@pytest.mark.parametrize("S", [4, 8, 12, 16, 20, 24, 32, 48, 64])
@pytest.mark.parametrize("mode", ["random", "dups", "floats", "const"])
def test_random_meshes(rx, S, mode):
    rng = np.random.default_rng(1000 + S * 10 + ["random", "dups", "floats", "const"].index(mode))
    for n, m in SIZES:
        assert_parity(rx, *random_mesh(rng, n, m, S // 4, mode))


def test_worked_example(rx):
    from test_oracle import load_worked_example

    rows, letters, ints, words = load_worked_example()
    vtx, idx = words("vtx"), ints("idx").astype(np.int32)
    D, gv, gi = run_gpu(rx, vtx, idx, 3)
    assert D == 6
    np.testing.assert_array_equal(gv, words("newVtx"))
    np.testing.assert_array_equal(gi, ints("idxNew"))


def test_config1_heightfield_256(rx):
    m = synth.config_mesh(1)
    assert assert_parity(rx, m.vtx, m.idx.reshape(-1), 3) == 66_049


@pytest.mark.parametrize("n", [8, 64, 1024])
def test_table1_quad_grid(rx, n):
    m = synth.quad_grid(n)
    assert assert_parity(rx, m.vtx, m.idx.reshape(-1), 4) == (n + 1) ** 2


@pytest.mark.slow
def test_config2_heightfield_2048_full(rx):
    m = synth.config_mesh(2)
    assert assert_parity(rx, m.vtx, m.idx.reshape(-1), 3) == 4_198_401


@pytest.mark.slow
def test_config3_tet_soup_128_full(rx):
    m = synth.config_mesh(3)
    assert assert_parity(rx, m.vtx, m.idx.reshape(-1), 4) == 2_146_689


# ------------------------------------------------------------------------------- edge cases


def test_no_elements(rx):
    v, _ = to_dev(np.arange(12, dtype=np.uint32).reshape(4, 3), np.zeros((0, 3), np.int32))
    i = torch.zeros((0, 3), dtype=torch.int32, device="cuda")
    out_v, out_n, out_i = rx.reindex_mesh(v, i)
    assert int(out_n.item()) == 0 and out_i.numel() == 0


def test_single_vertex_all_indices(rx):
    vtx = np.arange(3 * 5000, dtype=np.uint32).reshape(5000, 3)
    idx = np.full(9999, 4321, np.int32)
    assert assert_parity(rx, vtx, idx, 3) == 1


def test_all_vertices_bitwise_equal(rx):
    vtx = np.tile(np.array([[0xDEADBEEF, 7, 0x80000000, 1]], np.uint32), (20000, 1))
    idx = np.random.default_rng(3).integers(0, 20000, size=(30000,)).astype(np.int32)
    assert assert_parity(rx, vtx, idx, 3) == 1


@pytest.mark.parametrize("bad", [-1, 1000, 2**31 - 1])
def test_index_out_of_range_is_reported(rx, bad):
    vtx = np.arange(3000, dtype=np.uint32).reshape(1000, 3)
    idx = np.arange(999, dtype=np.int32)
    idx[517] = bad
    v, i = to_dev(vtx, idx.reshape(-1, 3))
    rx.reindex_stream_status()  # clear anything left over
    out_v, out_n, out_i = rx.reindex_mesh(v, i)
    assert rx.reindex_stream_status() == rx.REINDEX_ERR_INDEX_RANGE
    assert int(out_n.item()) == -rx.REINDEX_ERR_INDEX_RANGE
    assert rx.reindex_stream_status() == rx.REINDEX_OK  # sticky word was cleared
    # the context stays usable
    idx[517] = 5
    assert_parity(rx, vtx, idx, 3)


def test_in_place_remap(rx):
    rng = np.random.default_rng(8)
    vtx, idx = random_mesh(rng, 30000, 45000, 3, "dups")
    ov, oi = oracle.reindex_sort(vtx, idx)
    v, i = to_dev(vtx, idx.reshape(-1, 3))
    out_v, out_n, out_i = rx.reindex_mesh(v, i, out_idx=i)
    assert int(out_n.item()) == ov.shape[0]
    np.testing.assert_array_equal(i.cpu().numpy().reshape(-1), oi)


def test_unaligned_index_buffers(rx):
    """int32 index arrays that are only 4-byte aligned take the scalar load path."""
    rng = np.random.default_rng(9)
    vtx, idx = random_mesh(rng, 20000, 30003, 3, "dups")
    ov, oi = oracle.reindex_sort(vtx, idx)
    v = torch.from_numpy(vtx.view(np.int32)).cuda()
    big = torch.zeros(30003 + 1, dtype=torch.int32, device="cuda")
    big[1:] = torch.from_numpy(idx).cuda()
    i = big[1:].view(-1, 3)
    outbig = torch.zeros_like(big)
    o = outbig[1:].view(-1, 3)
    assert i.data_ptr() % 16 != 0 and o.data_ptr() % 16 != 0
    out_v, out_n, _ = rx.reindex_mesh(v, i, out_idx=o)
    assert int(out_n.item()) == ov.shape[0]
    np.testing.assert_array_equal(o.cpu().numpy().reshape(-1), oi)
    np.testing.assert_array_equal(out_v[: ov.shape[0]].cpu().numpy().view(np.uint32), ov)


def test_workspace_variant_and_determinism(rx):
    m = synth.heightfield_soup(300, 200, 0.07, seed=42)
    v, i = to_dev(m.vtx, m.idx)
    ws = torch.empty(rx.reindex_workspace_size(m.n_vtx, 12, m.n_elem, 3), dtype=torch.uint8, device="cuda")
    a = rx.reindex_mesh(v, i)
    b = rx.reindex_mesh_ws(v, i, ws)
    c = rx.reindex_mesh_ws(v, i, ws)
    torch.cuda.synchronize()
    D = int(a[1].item())
    assert D == 301 * 201 == int(b[1].item()) == int(c[1].item())
    for x, y in ((a, b), (b, c)):
        assert torch.equal(x[0][:D], y[0][:D]) and torch.equal(x[2], y[2])


def test_cuda_graph_capture_of_workspace_variant(rx):
    m = synth.heightfield_soup(120, 90, 0.1, seed=5)
    ov, oi = oracle.reindex_sort(m.vtx, m.idx)
    v, i = to_dev(m.vtx, m.idx)
    ws = torch.empty(rx.reindex_workspace_size(m.n_vtx, 12, m.n_elem, 3), dtype=torch.uint8, device="cuda")
    out_v = torch.empty((min(m.n_vtx, i.numel()), 3), dtype=torch.int32, device="cuda")
    out_n = torch.empty(1, dtype=torch.int64, device="cuda")
    out_i = torch.empty_like(i)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        rx.reindex_mesh_ws(v, i, ws, out_v, out_n, out_i)  # warm-up outside capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        rx.reindex_mesh_ws(v, i, ws, out_v, out_n, out_i, stream=s)
    out_i.zero_()
    out_n.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert int(out_n.item()) == ov.shape[0]
    np.testing.assert_array_equal(out_v[: ov.shape[0]].cpu().numpy().view(np.uint32), ov)
    np.testing.assert_array_equal(out_i.cpu().numpy().reshape(-1), oi)


@pytest.mark.parametrize("G,pinned_in,pinned_out,tets", [(200, True, True, False), (1200, True, True, False),
                                                          (64, False, True, False), (300, True, False, False),
                                                          (24, True, True, True)])
def test_host_buffer_variant(rx, G, pinned_in, pinned_out, tets):
    """Host buffers in and out, page-locked or not: staged through device memory, the vertex upload
    and the unique-vertex download overlapping kernels on a second stream.  1200^2 cells: large
    enough for the large-mesh sort; tet soups take the prefix sort."""
    m = synth.tet_soup(G, 0.03, seed=6) if tets else synth.heightfield_soup(G, (3 * G) // 4, 0.05, seed=6)
    ov, oi = oracle.reindex_sort(m.vtx, m.idx)
    hv = torch.from_numpy(m.vtx.view(np.int32))
    hi = torch.from_numpy(m.idx)
    if pinned_in:
        hv, hi = hv.pin_memory(), hi.pin_memory()
    for _ in range(2):  # twice: nothing left over from the first call
        out_v = torch.empty((min(m.n_vtx, m.idx.size), hv.shape[1]), dtype=torch.int32, pin_memory=pinned_out)
        out_i = torch.empty_like(hi, pin_memory=pinned_out)
        got_v, got_i = rx.reindex_mesh_host(hv, hi, out_v, out_i)
        np.testing.assert_array_equal(got_v.numpy().view(np.uint32), ov)
        np.testing.assert_array_equal(got_i.numpy().reshape(-1), oi)


@pytest.mark.parametrize("G,pinned,tets,pub", [(7, True, False, "off"), (1200, True, False, "off"),
                                             (300, False, False, "on"), (24, True, True, "on")])
def test_host_buffer_variant_hash_path(rx, G, pinned, tets, pub):
    """The host-buffer entry point on the hash path: indices first, then the vertex array in
    chunks, each chunk inserted into the hash table as soon as it has arrived (7^2 cells: fewer
    vertices than chunks of 32 rows)."""
    S = 16 if tets else 12
    m = synth.tet_soup(G, 0.03, seed=6) if tets else synth.heightfield_soup(G, (3 * G) // 4, 0.05, seed=6)
    ov, oi = oracle.reindex_sort(m.vtx, m.idx)
    hv = torch.from_numpy(m.vtx.view(np.int32))
    hi = torch.from_numpy(m.idx)
    if pinned:
        hv, hi = hv.pin_memory(), hi.pin_memory()
    saved = rx.reindex_tuning_get(S)
    rx.reindex_tuning_set(S, f"dedup=hash,dpub={pub}")
    try:
        for _ in range(2):
            got_v, got_i = rx.reindex_mesh_host(hv, hi)
            np.testing.assert_array_equal(got_v.numpy().view(np.uint32), ov)
            np.testing.assert_array_equal(got_i.numpy().reshape(-1), oi)
    finally:
        rx.reindex_tuning_set(S, saved)


def test_host_buffer_variant_reports_device_errors(rx):
    m = synth.heightfield_soup(64, 64, 0.0, seed=7)
    idx = m.idx.copy()
    idx.reshape(-1)[12345] = m.n_vtx + 5  # out of range
    hv = torch.from_numpy(m.vtx.view(np.int32)).pin_memory()
    hi = torch.from_numpy(idx).pin_memory()
    with pytest.raises(rx.ReindexError) as ei:
        rx.reindex_mesh_host(hv, hi)
    assert ei.value.code == rx.REINDEX_ERR_INDEX_RANGE
    rx.reindex_stream_status()  # clear the sticky word
    out_v, out_i = rx.reindex_mesh_host(hv, torch.from_numpy(m.idx).pin_memory())  # and the next call works
    ov, oi = oracle.reindex_sort(m.vtx, m.idx)
    np.testing.assert_array_equal(out_v.numpy().view(np.uint32), ov)


SORT_KERNELS = {"regs": ["onesweep"], "tiles,pack=off": ["tile_count", "tile_offsets", "tile_scatter"],
                "tiles,pack=on": ["tile_count", "tile_offsets", "tile_scatter", "key_masks"],
                "chunk,pack=off": ["tile_count", "tile_offsets", "chunk_scatter"],
                "chunk,pack=on": ["tile_count", "tile_offsets", "chunk_scatter", "key_masks"]}


@pytest.mark.parametrize("sort", ["regs", "tiles,pack=off", "tiles,pack=on", "chunk,pack=off", "chunk,pack=on"])
def test_profile_records_every_kernel(rx, sort):
    m = synth.config_mesh(1)
    v, i = to_dev(m.vtx, m.idx)
    saved = rx.reindex_tuning_get(12)
    rx.reindex_tuning_set(12, f"sort={sort},prefix=off,dedup=off")
    rx.profile_collect()
    rx.profile_enable(True)
    try:
        rx.reindex_mesh(v, i)
        torch.cuda.synchronize()
    finally:
        rx.profile_enable(False)
        rx.reindex_tuning_set(12, saved)
    recs = rx.profile_collect()
    names = [r["name"] for r in recs]
    mine = SORT_KERNELS[sort]
    for k in mine:
        assert names.count(k) == (1 if k == "key_masks" else 12)
    others = {k for ks in SORT_KERNELS.values() for k in ks} - set(mine)
    assert set(names) == (set(rx.KERNEL_NAMES) - {"seg_prepare", "seg_offsets", "prefix_gate", "prefix_check",
                                                   "hash_dedup", "resolve"} - others)
    # x and y are integers 0..256 as float32: their lowest byte is always zero -> skipped passes
    # (packed keys: the skipped passes are the top digit positions instead)
    sk = {r["digit"]: r["skipped"] for r in recs if r["name"] == mine[0]}
    assert sum(sk.values()) >= 2 and not sk[0]
    if not sort.endswith("pack=on"):
        assert sk[8] and sk[4]


# Every radix-pass variant (and grid shape) must give the same bit-exact result.
SORT_VARIANTS = ["sort=regs,rank=ballot,grid=persist,prefix=off", "sort=regs,rank=match,grid=tile",
                 "sort=pipe,rank=ballot,grid=persist,prefix=off", "sort=tiles,rank=ballot,swaves=1,pack=on",
                 "sort=tiles,rank=match,swaves=tile,pack=off,prefix=off", "sort=tiles,rank=ballot,swaves=4,pack=off",
                 "sort=tiles,rank=vary,swaves=tile,pack=on,prefix=off", "sort=tiles,rank=ballot,pack=auto",
                 "sort=chunk,chunk=big,pack=off,prefix=off", "sort=chunk,chunk=small,pack=on,prefix=off",
                 "sort=chunk,chunk=big,cgrid=3,pack=auto", "sort=chunk,chunk=small,cgrid=5,cocc=1,pack=off",
                 "sort=chunk,chunk=wide,cgrid=7,rank=match,pack=on", "sort=chunk,chunk=deep,cgrid=2,pack=off,prefix=off",
                 "sort=chunk,chunk=wide,cgrid=3,dbits=7,rank=ballot,prefix=off",
                 "sort=chunk,chunk=small,dbits=6,rank=vary,prefix=auto", "sort=chunk,chunk=big,cgrid=5,dbits=6,rank=match",
                 "dedup=hash,sort=auto", "dedup=hash,dpub=off,sort=tiles,rank=match",
                 "dedup=hash,sort=chunk,chunk=big,cgrid=3", "dedup=hash,dbits=7,sort=regs",
                 "dedup=hash,prefix=off,sort=chunk", "dedup=hash,prefix=on,dpub=on,sort=tiles"]


@pytest.mark.parametrize("spec", SORT_VARIANTS)
@pytest.mark.parametrize("S", [4, 8, 12, 16, 20])
def test_sort_variants_bit_exact(rx, spec, S):
    saved = rx.reindex_tuning_get(S)
    rx.reindex_tuning_set(S, spec)
    try:
        rng = np.random.default_rng(7000 + S + 100 * SORT_VARIANTS.index(spec))
        for mode in ["random", "dups", "const", "hibyte"]:
            for n, m in SIZES:
                assert_parity(rx, *random_mesh(rng, n, m, S // 4, mode))
        if S == 12:
            mesh = synth.config_mesh(1)
            assert assert_parity(rx, mesh.vtx, mesh.idx, 3) == mesh.expected_unique
    finally:
        rx.reindex_tuning_set(S, saved)


WIDE_VARIANTS = ["pack=off,swaves=tile,prefix=off", "pack=on,swaves=tile,prefix=off", "pack=auto,swaves=1",
                 "pack=on,swaves=4", "sort=chunk,chunk=big,cgrid=4,prefix=off", "sort=chunk,chunk=small,prefix=auto",
                 "sort=chunk,chunk=wide,cgrid=3,prefix=off", "sort=chunk,chunk=deep,prefix=auto",
                 "sort=chunk,chunk=big,cgrid=4,dbits=7,prefix=auto", "sort=chunk,chunk=wide,dbits=6,prefix=off",
                 "dedup=hash,sort=chunk", "dedup=hash,dpub=off,sort=tiles,cgrid=2",
                 "dedup=hash,prefix=off,sort=chunk,cgrid=3", "dedup=hash,prefix=off,dpub=on"]


@pytest.mark.parametrize("spec", WIDE_VARIANTS)
@pytest.mark.parametrize("S", [24, 32, 48, 64])
def test_wide_vertices_bit_exact(rx, spec, S):
    """24- and 32-byte vertices (always the "tiles" sort): random words, many duplicates, constant
    low bytes, and a heightfield whose vertices carry normal and texture-coordinate words."""
    saved = rx.reindex_tuning_get(S)
    rx.reindex_tuning_set(S, spec)
    try:
        rng = np.random.default_rng(9100 + S + 10 * WIDE_VARIANTS.index(spec))
        for mode in ["random", "dups", "const", "hibyte"]:
            for n, m in SIZES:
                assert_parity(rx, *random_mesh(rng, n, m, S // 4, mode))
        mesh = synth.heightfield_soup_attrs(300, 170, 0.05, seed=12, stride=S)
        assert assert_parity(rx, mesh.vtx, mesh.idx.reshape(-1), 3) == mesh.expected_unique
    finally:
        rx.reindex_tuning_set(S, saved)


@pytest.mark.parametrize("S", [24, 32, 48, 64])
def test_wide_vertices_large_heightfield(rx, S):
    """A 1448^2-cell heightfield with attribute words (12.6 M soup vertices of 24 or 32 bytes, the
    prefix sort's default path): D = 1449^2, and every unique vertex and every index equals the
    oracle's, element by element."""
    vtx, idx = synth.heightfield_soup_gpu(1448, 1448, 0.05, seed=2)
    wide = synth.with_attributes_gpu(vtx.view(torch.int32), (S - 12) // 4, seed=2)
    out_v, out_n, out_i = rx.reindex_mesh(wide, idx)
    torch.cuda.synchronize()
    D = int(out_n.item())
    assert D == 1449 * 1449
    ov, oi = oracle.reindex_sort(wide.cpu().numpy().view(np.uint32), idx.cpu().numpy())
    assert ov.shape[0] == D
    np.testing.assert_array_equal(out_v[:D].cpu().numpy().view(np.uint32), ov)
    np.testing.assert_array_equal(out_i.reshape(-1).cpu().numpy(), oi)


def test_lookback_wait_runs_out_and_reports_timeout(rx):
    """A compaction tile that never publishes its status (test hook): the waits after it give up
    after their iteration limit, the call reports REINDEX_ERR_TIMEOUT, and the next call works."""
    import time

    m = synth.heightfield_soup(64, 64, 0.05, seed=31)  # 25,805 vertices: 13 compaction tiles
    v, i = to_dev(m.vtx, m.idx)
    rx.reindex_stream_status()
    rx.lib().reindex_debug_stall_tile(5)
    try:
        t0 = time.time()
        out_v, out_n, out_i = rx.reindex_mesh(v, i)
        status = rx.reindex_stream_status()
        elapsed = time.time() - t0
    finally:
        rx.lib().reindex_debug_stall_tile(-1)
    assert status == rx.REINDEX_ERR_TIMEOUT
    assert int(out_n.item()) == -rx.REINDEX_ERR_TIMEOUT
    assert elapsed < 60
    assert assert_parity(rx, m.vtx, m.idx.reshape(-1), 3) == 65 * 65


def test_attribute_generator_device_matches_host(rx):
    """The device attribute generator writes the same bits as the host one (inputs only)."""
    m = synth.heightfield_soup(50, 40, 0.1, seed=23)
    for n_attr in (3, 5):
        host = synth.with_attributes(m.vtx, n_attr, 23)
        dev = synth.with_attributes_gpu(torch.from_numpy(m.vtx.view(np.int32)).cuda(), n_attr, 23)
        np.testing.assert_array_equal(dev.cpu().numpy().view(np.uint32), host)


def _sort_records(rx, S, spec, vtx, idx):
    """Per-launch records of one call under tuning `spec` for stride S."""
    saved = rx.reindex_tuning_get(S)
    rx.reindex_tuning_set(S, spec)
    v, i = to_dev(vtx, idx.reshape(-1, 3))
    rx.profile_collect()
    rx.profile_enable(True)
    try:
        out_v, out_n, out_i = rx.reindex_mesh(v, i)
        torch.cuda.synchronize()
    finally:
        rx.profile_enable(False)
        rx.reindex_tuning_set(S, saved)
    return rx.profile_collect(), int(out_n.item()), out_v, out_i


@pytest.mark.parametrize("S", [12, 16, 24, 32, 48, 64])
def test_prefix_sort_skips_the_full_key_sort(rx, S):
    """Vertices whose 64 most significant varying bits already tell them apart (a heightfield's x, y
    and the top of z): the prefix sort gives the result and every pass of the full-key sort is
    skipped.  Keys that share prefixes (few values per word) run the full-key sort; both bit-exact."""
    m = synth.heightfield_soup_attrs(200, 130, 0.05, seed=3, stride=S) if S > 12 else \
        synth.heightfield_soup(200, 130, 0.05, seed=3)
    if S == 16:
        m = synth.Mesh(vtx=m.vtx[:, :4], idx=m.idx)
    ov, oi = oracle.reindex_sort(m.vtx, m.idx.reshape(-1))
    sort, kname = ("chunk", "chunk_scatter") if S >= 48 else ("tiles", "tile_scatter")  # 48, 64: chunk only
    recs, D, out_v, out_i = _sort_records(rx, S, f"prefix=on,sort={sort}", m.vtx, m.idx)
    assert D == ov.shape[0]
    np.testing.assert_array_equal(out_v[:D].cpu().numpy().view(np.uint32), ov)
    np.testing.assert_array_equal(out_i.cpu().numpy().reshape(-1), oi)
    sc = [r for r in recs if r["name"] == kname]  # in launch order: the prefix sort's 8 passes first
    pre, full = sc[:8], sc[8:]
    assert len(full) == S and all(r["item_bytes"] == 16 for r in pre) and all(r["item_bytes"] == S + 4 for r in full)
    assert sum(not r["skipped"] for r in pre) >= 6
    assert all(r["skipped"] for r in full)
    assert [r["name"] for r in recs].count("prefix_gate") == 1
    assert [r["name"] for r in recs].count("prefix_check") == 1

    rng = np.random.default_rng(S)
    vtx, idx = random_mesh(rng, 30000, 30000, S // 4, "dups")  # 7 values per word: prefixes collide
    ov, oi = oracle.reindex_sort(vtx, idx)
    recs, D, out_v, out_i = _sort_records(rx, S, f"prefix=on,sort={sort}", vtx, idx[: 30000 // 3 * 3])
    ov, oi = oracle.reindex_sort(vtx, idx[: 30000 // 3 * 3])
    assert D == ov.shape[0]
    np.testing.assert_array_equal(out_v[:D].cpu().numpy().view(np.uint32), ov)
    np.testing.assert_array_equal(out_i.cpu().numpy().reshape(-1), oi)
    full = [r for r in recs if r["name"] == kname][8:]
    assert sum(not r["skipped"] for r in full) >= 8


@pytest.mark.parametrize("S", [16, 32])
def test_prefix_sort_reports_device_errors(rx, S):
    """An index out of range, and a look-back wait that runs out, inside the prefix sort: the call
    reports the error (the full-key sort is skipped), and the next call is exact."""
    import time

    m = synth.heightfield_soup_attrs(64, 64, 0.05, seed=31, stride=S)  # 25,805 vertices: 13 compaction tiles
    idx = m.idx.copy()
    idx.reshape(-1)[777] = m.n_vtx
    v, i = to_dev(m.vtx, idx)
    rx.reindex_stream_status()
    out_v, out_n, out_i = rx.reindex_mesh(v, i)
    assert rx.reindex_stream_status() == rx.REINDEX_ERR_INDEX_RANGE
    assert int(out_n.item()) == -rx.REINDEX_ERR_INDEX_RANGE
    v, i = to_dev(m.vtx, m.idx)
    rx.lib().reindex_debug_stall_tile(5)
    try:
        t0 = time.time()
        out_v, out_n, out_i = rx.reindex_mesh(v, i)
        status = rx.reindex_stream_status()
        elapsed = time.time() - t0
    finally:
        rx.lib().reindex_debug_stall_tile(-1)
    assert status == rx.REINDEX_ERR_TIMEOUT and int(out_n.item()) == -rx.REINDEX_ERR_TIMEOUT
    assert elapsed < 60
    assert assert_parity(rx, m.vtx, m.idx.reshape(-1), 3) == 65 * 65


@pytest.mark.parametrize("S", [16, 32])
def test_prefix_sort_host_buffers_and_graph_capture(rx, S):
    """The host-buffer entry point and a captured CUDA graph of the workspace variant, both on
    the prefix sort."""
    m = synth.heightfield_soup_attrs(150, 90, 0.05, seed=5, stride=S)
    ov, oi = oracle.reindex_sort(m.vtx, m.idx)
    hv = torch.from_numpy(m.vtx.view(np.int32)).pin_memory()
    hi = torch.from_numpy(m.idx).pin_memory()
    out_v, out_i = rx.reindex_mesh_host(hv, hi)
    np.testing.assert_array_equal(out_v.numpy().view(np.uint32), ov)
    np.testing.assert_array_equal(out_i.numpy().reshape(-1), oi)
    v, i = to_dev(m.vtx, m.idx)
    ws = torch.empty(rx.reindex_workspace_size(m.n_vtx, S, m.n_elem, 3), dtype=torch.uint8, device="cuda")
    out_v = torch.empty((min(m.n_vtx, i.numel()), S // 4), dtype=torch.int32, device="cuda")
    out_n = torch.empty(1, dtype=torch.int64, device="cuda")
    out_i = torch.empty_like(i)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        rx.reindex_mesh_ws(v, i, ws, out_v, out_n, out_i)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        rx.reindex_mesh_ws(v, i, ws, out_v, out_n, out_i, stream=s)
    out_i.zero_()
    out_n.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert int(out_n.item()) == ov.shape[0]
    np.testing.assert_array_equal(out_v[: ov.shape[0]].cpu().numpy().view(np.uint32), ov)
    np.testing.assert_array_equal(out_i.cpu().numpy().reshape(-1), oi)


@pytest.mark.parametrize("S,kind,pub", [(12, "soup", "on"), (12, "soup", "off"), (16, "tets", "on"),
                                        (16, "tets", "on,prefix=off"), (32, "attrs", "on"),
                                        (32, "attrs", "off,prefix=off"), (64, "attrs", "off")])
def test_dedup_hash_full_size(rx, S, kind, pub):
    """Duplicate removal with the hash table before the sort, on full-size soups (about six copies of
    every vertex in the triangle soups, twenty in the tet soup), with and without the published item
    positions, and for 16-byte keys and wider with the prefix sort of the representatives (the
    default) or the full-key sort of them: every output element against the oracle."""
    saved = rx.reindex_tuning_get(S)
    rx.reindex_tuning_set(S, f"dedup=hash,dpub={pub}")
    try:
        if kind == "soup":
            v, i = synth.heightfield_soup_gpu(2048, 2048, 0.05, seed=2)
            v = v.view(torch.int32)
        elif kind == "tets":
            v, i = synth.tet_soup_gpu(96, 0.03, seed=3)
            v = v.view(torch.int32)
        else:
            v0, i = synth.heightfield_soup_gpu(1024, 1024, 0.05, seed=2)
            v = synth.with_attributes_gpu(v0.view(torch.int32), (S - 12) // 4, seed=2)
        rx.profile_collect()
        rx.profile_enable(True)
        try:
            out_v, out_n, out_i = rx.reindex_mesh(v, i)
            torch.cuda.synchronize()
        finally:
            rx.profile_enable(False)
        names = [r["name"] for r in rx.profile_collect()]
        assert "hash_dedup" in names and "resolve" not in names  # copies resolve in the remap
        if S == 12 or "prefix=off" in pub:  # hash path: the sort of the representatives' full keys
            assert "prefix_check" not in names
        else:  # the prefix path sorts the representatives
            assert "prefix_check" in names
        D = int(out_n.item())
        ov, oi = oracle.reindex_sort(v.cpu().numpy().view(np.uint32), i.cpu().numpy())
        assert D == ov.shape[0]
        np.testing.assert_array_equal(out_v[:D].cpu().numpy().view(np.uint32), ov)
        np.testing.assert_array_equal(out_i.cpu().numpy().reshape(-1), oi)
    finally:
        rx.reindex_tuning_set(S, saved)
