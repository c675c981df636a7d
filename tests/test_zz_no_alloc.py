"""reindex_mesh_noalloc: the entry point for callers that cannot allocate device memory.

Such callers (a program that reserved its whole device-memory budget up front, a real-time loop
in which cudaMalloc/cudaFree would synchronise the device, a plugin whose host forbids hidden
allocations) get the same result as reindex_mesh from a fixed scratch array inside the library.
These tests call the entry point through the C ABI several times in a row and check every result
bit for bit against the serial oracle and against reindex_mesh on the same input; a later call
would expose anything an earlier call left behind in the shared scratch array (a small mesh, then
a larger one of the same stride, then the small one again).  They also check that a call, once
the library is warm on the device, allocates nothing (the device's default memory pool and the
device's free memory are unchanged), and that meshes over the stated limit are refused.

The file name makes pytest collect it last.
"""
import ctypes
import glob
import os

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MAX_VTX = 262_144  # REINDEX_NOALLOC_MAX_VTX


@pytest.fixture(scope="module")
def rx():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2109_09812_gb300 import build

    build.build()
    import paper_2109_09812_gb300 as rx

    L = rx.lib()
    L.reindex_mesh_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p,
                                       ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p]
    L.reindex_mesh_noalloc.restype = ctypes.c_int
    return rx


def _mesh(seed, n_vtx, n_elem, k, words):
    rng = np.random.default_rng(seed)
    pool = rng.integers(0, 2**32, size=(n_vtx // 3 + 1, words), dtype=np.uint64).astype(np.uint32)
    vtx = pool[rng.integers(0, pool.shape[0], size=n_vtx)]  # many exact duplicates
    idx = rng.integers(0, n_vtx, size=(n_elem, k)).astype(np.int32)  # some vertices unused
    return vtx, idx


def _dev(vtx, idx):
    return torch.from_numpy(vtx.view(np.int32)).cuda(), torch.from_numpy(idx).cuda()


def _noalloc(rx, v, i, out=None):
    S = v.shape[1] * 4
    cap = min(v.shape[0], i.numel())
    if out is None:
        out = (torch.full((max(cap, 1), v.shape[1]), -1, dtype=torch.int32, device="cuda"),
               torch.full((1,), -99, dtype=torch.int64, device="cuda"), torch.full_like(i, -1))
    out_v, out_n, out_i = out
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = rx.lib().reindex_mesh_noalloc(ctypes.c_void_p(v.data_ptr()), v.shape[0], S, ctypes.c_void_p(i.data_ptr()),
                                       i.shape[0], i.shape[1], ctypes.c_void_p(out_v.data_ptr()),
                                       ctypes.c_void_p(out_n.data_ptr()), ctypes.c_void_p(out_i.data_ptr()), st)
    return rc, out_v, out_n, out_i


def _check(rx, vtx, idx):
    """One no-allocation call, compared with the oracle and with reindex_mesh, element by element."""
    v, i = _dev(vtx, idx)
    rc, nv, nn, ni = _noalloc(rx, v, i)
    assert rc == rx.REINDEX_OK
    torch.cuda.synchronize()
    D = int(nn.item())
    ov, oi = oracle.reindex_sort(vtx, idx)
    assert D == ov.shape[0] > 0
    np.testing.assert_array_equal(nv[:D].cpu().numpy().view(np.uint32), ov)
    np.testing.assert_array_equal(ni.cpu().numpy().reshape(-1), oi)
    rv, rn, ri = rx.reindex_mesh(v, i)
    torch.cuda.synchronize()
    assert int(rn.item()) == D
    assert torch.equal(nv[:D], rv[:D]) and torch.equal(ni, ri)


def test_noalloc_matches_oracle_on_calls_in_a_row(rx):
    small = _mesh(1, 30_001, 12_000, 3, 3)
    large = _mesh(2, 200_000, 150_000, 3, 3)
    other = _mesh(3, 90_001, 40_000, 4, 4)
    for vtx, idx in (small, large, small, other, small):  # same stride small -> large -> small, then another
        _check(rx, vtx, idx)


@pytest.mark.parametrize("words", [6, 8])
def test_noalloc_wide_vertices_at_the_limit(rx, words):
    """24- and 32-byte vertices at the largest size the static scratch holds."""
    _check(rx, *_mesh(4, MAX_VTX, 87_381, 3, words))


@pytest.mark.parametrize("words,pub", [(3, "on"), (3, "off"), (8, "off")])
def test_noalloc_hash_path(rx, words, pub):
    """With duplicates removed by the hash table before the sort (its table in the same scratch
    array; 32-byte vertices: the prefix sort of the representatives): calls in a row, small, large
    and small again, each against the oracle."""
    S = 4 * words
    saved = rx.reindex_tuning_get(S)
    rx.reindex_tuning_set(S, f"dedup=hash,dpub={pub}")
    try:
        small = _mesh(11, 30_001, 12_000, 3, words)
        large = _mesh(12, 200_000, 150_000, 3, words)
        for vtx, idx in (small, large, small):
            _check(rx, vtx, idx)
    finally:
        rx.reindex_tuning_set(S, saved)


def _cudart():
    """The CUDA runtime library as a separate handle, for the memory-pool queries."""
    cands = ["libcudart.so", "libcudart.so.13", "/usr/local/cuda/lib64/libcudart.so"]
    cands += sorted(glob.glob("/usr/local/cuda*/lib64/libcudart.so*"))
    cands += sorted(glob.glob(os.path.join(os.path.dirname(torch.__file__), "lib", "libcudart*.so*")))
    for c in cands:
        try:
            return ctypes.CDLL(c)
        except OSError:
            continue
    pytest.fail("no CUDA runtime library found for the memory-pool queries")


def test_noalloc_call_allocates_nothing(rx):
    """Once the library is warm on the device, a call changes neither the default memory pool's
    usage (not even transiently: its high-water mark is reset first) nor the device's free memory."""
    rt = _cudart()
    dev = torch.cuda.current_device()
    pool = ctypes.c_void_p()
    assert rt.cudaDeviceGetDefaultMemPool(ctypes.byref(pool), dev) == 0
    USED_CURRENT, USED_HIGH, RESERVED_CURRENT, RESERVED_HIGH = 7, 8, 5, 6

    def attr(a):
        v = ctypes.c_uint64(0)
        assert rt.cudaMemPoolGetAttribute(pool, a, ctypes.byref(v)) == 0
        return v.value

    vtx, idx = _mesh(5, 150_000, 100_000, 3, 3)
    v, i = _dev(vtx, idx)
    out = (torch.empty((150_000, 3), dtype=torch.int32, device="cuda"), torch.empty(1, dtype=torch.int64,
                                                                                      device="cuda"),
           torch.empty_like(i))
    assert _noalloc(rx, v, i, out)[0] == rx.REINDEX_OK  # warm: scratch resolved, kernels loaded
    torch.cuda.synchronize()
    used0, reserved0 = attr(USED_CURRENT), attr(RESERVED_CURRENT)
    zero = ctypes.c_uint64(0)
    assert rt.cudaMemPoolSetAttribute(pool, USED_HIGH, ctypes.byref(zero)) == 0  # reset the high-water marks
    assert rt.cudaMemPoolSetAttribute(pool, RESERVED_HIGH, ctypes.byref(zero)) == 0
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        assert _noalloc(rx, v, i, out)[0] == rx.REINDEX_OK
    torch.cuda.synchronize()
    assert attr(USED_HIGH) <= used0, "a no-allocation call took memory from the default pool"
    assert attr(RESERVED_HIGH) <= reserved0 and attr(RESERVED_CURRENT) == reserved0
    assert torch.cuda.mem_get_info()[0] == free0, "device free memory changed across no-allocation calls"
    ov, oi = oracle.reindex_sort(vtx, idx)
    D = int(out[1].item())
    assert D == ov.shape[0]
    np.testing.assert_array_equal(out[0][:D].cpu().numpy().view(np.uint32), ov)
    np.testing.assert_array_equal(out[2].cpu().numpy().reshape(-1), oi)


def test_noalloc_refuses_meshes_over_the_limit(rx):
    n = MAX_VTX + 1
    v = torch.zeros((n, 3), dtype=torch.int32, device="cuda")
    i = torch.zeros((10, 3), dtype=torch.int32, device="cuda")
    rc, *_ = _noalloc(rx, v, i)
    assert rc == rx.REINDEX_ERR_UNSUPPORTED


def _largest_fitting(rx, S, scratch=20 << 20):
    """The largest nVtx whose workspace (with as many indices as vertices) fits the scratch."""
    lo, hi = 1, MAX_VTX
    while lo < hi:
        mid = (lo + hi + 1) // 2
        if rx.reindex_workspace_size(mid, S, mid, 1) <= scratch:
            lo = mid
        else:
            hi = mid - 1
    return lo


@pytest.mark.parametrize("words", [12, 16])
def test_noalloc_48_and_64_byte_vertices(rx, words):
    """48- and 64-byte vertices: taken up to the largest mesh whose workspace fits the scratch."""
    n = _largest_fitting(rx, 4 * words)
    _check(rx, *_mesh(6, n, n // 3, 3, words))
    v = torch.zeros((n + 2000, words), dtype=torch.int32, device="cuda")
    i = torch.zeros(((n + 2000) // 3 + 1, 3), dtype=torch.int32, device="cuda")
    rc, *_ = _noalloc(rx, v, i)
    assert rc == rx.REINDEX_ERR_UNSUPPORTED
