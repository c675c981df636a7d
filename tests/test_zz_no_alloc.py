"""reindex_mesh_noalloc: the entry point for callers that cannot allocate device memory.

Such callers (a program that reserved its whole device-memory budget up front, a real-time loop
in which cudaMalloc/cudaFree would synchronise the device, a plugin whose host forbids hidden
allocations) get the same result as reindex_mesh from scratch memory the library reserved when
it was loaded.  This test calls the entry point through the C ABI twice in a row, on two
different meshes, and checks each result bit for bit against reindex_mesh on the same input;
the second call would expose anything the first call left behind in the shared scratch array.
It also checks that meshes over the stated limit are refused.

The file name makes pytest collect it last.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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
    return (torch.from_numpy(vtx.view(np.int32)).cuda(), torch.from_numpy(idx).cuda())


def _noalloc(rx, v, i):
    S = v.shape[1] * 4
    cap = min(v.shape[0], i.numel())
    out_v = torch.full((cap, v.shape[1]), -1, dtype=torch.int32, device="cuda")
    out_n = torch.full((1,), -99, dtype=torch.int64, device="cuda")
    out_i = torch.full_like(i, -1)
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = rx.lib().reindex_mesh_noalloc(ctypes.c_void_p(v.data_ptr()), v.shape[0], S, ctypes.c_void_p(i.data_ptr()),
                                       i.shape[0], i.shape[1], ctypes.c_void_p(out_v.data_ptr()),
                                       ctypes.c_void_p(out_n.data_ptr()), ctypes.c_void_p(out_i.data_ptr()), st)
    return rc, out_v, out_n, out_i


def test_noalloc_matches_reindex_mesh_twice_in_a_row(rx):
    meshes = [_mesh(1, 200_000, 150_000, 3, 3), _mesh(2, 90_001, 40_000, 4, 4)]
    for v, i in meshes:  # two calls in a row, different strides and sizes
        rc, nv, nn, ni = _noalloc(rx, v, i)
        assert rc == rx.REINDEX_OK
        rv, rn, ri = rx.reindex_mesh(v, i)
        torch.cuda.synchronize()
        D = int(rn.item())
        assert D > 0 and int(nn.item()) == D
        assert torch.equal(nv[:D], rv[:D])
        assert torch.equal(ni, ri)


@pytest.mark.parametrize("words", [6, 8])
def test_noalloc_wide_vertices_at_the_limit(rx, words):
    """24- and 32-byte vertices at the largest size the static scratch holds."""
    v, i = _mesh(3, 262_144, 87_381, 3, words)
    rc, nv, nn, ni = _noalloc(rx, v, i)
    assert rc == rx.REINDEX_OK
    rv, rn, ri = rx.reindex_mesh(v, i)
    torch.cuda.synchronize()
    D = int(rn.item())
    assert D > 0 and int(nn.item()) == D
    assert torch.equal(nv[:D], rv[:D]) and torch.equal(ni, ri)


def test_noalloc_refuses_meshes_over_the_limit(rx):
    n = 262_144 + 1
    v = torch.zeros((n, 3), dtype=torch.int32, device="cuda")
    i = torch.zeros((10, 3), dtype=torch.int32, device="cuda")
    rc, *_ = _noalloc(rx, v, i)
    assert rc == rx.REINDEX_ERR_UNSUPPORTED
