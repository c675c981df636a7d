"""The C ABI library builds, loads on a machine without a GPU, exports every entry point that
include/reindex.h declares, and rejects bad arguments on the host before touching the GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2109_09812_gb300 as rx
from paper_2109_09812_gb300 import build as rxbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "reindex.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_][\w\s\*]*?\b(reindex_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def L():
    rxbuild.build()
    return rx.lib()


def test_library_exports_every_declared_function(L):
    names = declared_functions()
    assert len(names) >= 9
    for n in names:
        assert hasattr(L, n), f"{n} declared in include/reindex.h but not exported"
    assert sorted(rx.EXPORTED) == sorted(names)


def test_status_strings(L):
    for code, name in [(0, "REINDEX_OK"), (1, "REINDEX_ERR_INVALID_ARG"), (2, "REINDEX_ERR_UNSUPPORTED"),
                       (3, "REINDEX_ERR_OOM"), (4, "REINDEX_ERR_INDEX_RANGE"), (5, "REINDEX_ERR_TIMEOUT"),
                       (6, "REINDEX_ERR_CUDA"), (7, "REINDEX_ERR_INTERNAL")]:
        assert rx.reindex_status_string(code) == name
    assert rx.reindex_status_string(99) == "REINDEX_ERR_UNKNOWN"
    assert [L.reindex_kernel_name(i).decode() for i in range(len(rx.KERNEL_NAMES))] == rx.KERNEL_NAMES


def test_workspace_size_model(L):
    # two item buffers of (S+4) bytes per potentially used vertex + a 1-byte digit plane per item
    # + oldToNew + bitmask + tables
    n, S, ne, k = 26_424_115, 12, 8_388_608, 3
    b = rx.reindex_workspace_size(n, S, ne, k)
    U = min(n, ne * k)
    assert 2 * U * (S + 4) + U + 4 * n <= b <= 2 * U * (S + 4) + U + 4 * n + 64 * 2**20
    for S in (24, 32):  # wide vertices: the same model
        b = rx.reindex_workspace_size(n, S, ne, k)
        assert 2 * U * (S + 4) + U + 4 * n <= b <= 2 * U * (S + 4) + U + 4 * n + 64 * 2**20
    for S in (5, 28, 36, 64):  # unsupported strides
        assert rx.reindex_workspace_size(n, S, ne, k) == 0
    assert rx.reindex_meshes_workspace_size(2, n, 24, ne, k) == 0  # batched: up to 16 bytes
    assert rx.reindex_workspace_size(-1, 12, ne, k) == 0
    assert rx.reindex_workspace_size(10, 12, 0, 3) > 0


def test_host_side_argument_checks(L):
    z = ctypes.c_void_p(0)
    fake = ctypes.c_void_p(1 << 20)  # never dereferenced: every call below fails its host checks
    # unsupported stride
    assert L.reindex_mesh(fake, 10, 6, fake, 3, 3, fake, fake, fake, z) == rx.REINDEX_ERR_UNSUPPORTED
    # negative sizes, zero arity
    assert L.reindex_mesh(fake, -1, 12, fake, 3, 3, fake, fake, fake, z) == rx.REINDEX_ERR_INVALID_ARG
    assert L.reindex_mesh(fake, 10, 12, fake, 3, 0, fake, fake, fake, z) == rx.REINDEX_ERR_INVALID_ARG
    # too many vertices for 30-bit look-back counts; too many indices for int32
    assert L.reindex_mesh(fake, 1 << 30, 12, fake, 3, 3, fake, fake, fake, z) == rx.REINDEX_ERR_UNSUPPORTED
    assert L.reindex_mesh(fake, 10, 12, fake, 1 << 30, 3, fake, fake, fake, z) == rx.REINDEX_ERR_UNSUPPORTED
    # null output count, null idx
    assert L.reindex_mesh(fake, 10, 12, fake, 3, 3, fake, z, fake, z) == rx.REINDEX_ERR_INVALID_ARG
    assert L.reindex_mesh(fake, 10, 12, z, 3, 3, fake, fake, fake, z) == rx.REINDEX_ERR_INVALID_ARG
    # misaligned 16-, 24- and 32-byte vertices (16-, 8- and 16-byte alignment)
    for S, off in ((16, 4), (24, 4), (32, 8)):
        assert L.reindex_mesh(ctypes.c_void_p((1 << 20) + off), 10, S, fake, 3, 3, fake, fake, fake, z) \
            == rx.REINDEX_ERR_INVALID_ARG
    assert L.reindex_mesh(fake, 10, 28, fake, 3, 3, fake, fake, fake, z) == rx.REINDEX_ERR_UNSUPPORTED
    # no vertices but some indices: every index is out of range
    assert L.reindex_mesh(z, 0, 12, fake, 3, 3, fake, fake, fake, z) == rx.REINDEX_ERR_INDEX_RANGE
    # workspace too small
    assert L.reindex_mesh_ws(fake, 10, 12, fake, 3, 3, fake, fake, fake, fake, 16, z) == rx.REINDEX_ERR_INVALID_ARG


@pytest.mark.parametrize("seed,size", [(1, 1 << 20), (2, 1 << 28), (3, 12345 * 256), (4, 256)])
def test_server_arena_allocator_host_check(L, seed, size):
    """The serving arena allocator (first fit, coalescing, 256-byte alignment) against a brute-force
    model: no overlaps, no refusal while a large enough gap exists, full coalescing at the end."""
    assert rx.debug_arena_check(seed, 5000, size) == 0


@pytest.mark.parametrize("K", [1, 2, 3, 4, 5, 6, 8])
def test_prefix_sort_bit_selection(L, K):
    """The prefix sort keeps the most significant varying key bits: the bits it selects are exactly
    the first ones of the varying bits listed from word 0's bit 31 down (64 of them, or fewer when
    the 16-run limit or the key runs out), described as runs least significant first, each placed
    right above the previous one.  Keys whose prefixes differ then compare like their prefixes."""
    import random

    rnd = random.Random(100 + K)
    for trial in range(200):
        kor, knand = [], []
        for _ in range(K):
            style = rnd.randrange(4)
            if style == 0:
                m = 0
            elif style == 1:
                m = 0xFFFFFFFF
            elif style == 2:  # a few runs
                m = 0
                for _ in range(rnd.randrange(1, 4)):
                    lo = rnd.randrange(32)
                    hi = rnd.randrange(lo, 32)
                    m |= ((1 << (hi - lo + 1)) - 1) << lo
            else:
                m = rnd.getrandbits(32)
            const = rnd.getrandbits(32) & ~m
            kor.append(m | const)
            knand.append(m | (~const & 0xFFFFFFFF & ~m))
        p = rx.debug_prefix_pack(np.array(kor, np.uint32), np.array(knand, np.uint32))
        varying = [(w, b) for w in range(K) for b in range(31, -1, -1) if ((kor[w] & knand[w]) >> b) & 1]
        selected = set()
        for r in range(p["nruns"]):
            assert 1 <= p["len"][r] and p["shift"][r] + p["len"][r] <= 32
            selected |= {(p["word"][r], b) for b in range(p["shift"][r], p["shift"][r] + p["len"][r])}
            assert p["pos"][r] == sum(p["len"][:r])
        n = p["nbits"]
        assert p["returned"] == n == len(selected) <= 64 and p["nruns"] <= 16 and p["on"] == 1
        assert selected == set(varying[:n])
        if p["nruns"] < 16:
            assert n == min(64, len(varying))
        # runs least significant first: each run lies below the next in significance order
        order = {wb: i for i, wb in enumerate(varying)}
        for r in range(p["nruns"] - 1):
            assert order[(p["word"][r], p["shift"][r])] > order[(p["word"][r + 1], p["shift"][r + 1] + p["len"][r + 1] - 1)]
        words_with_runs = [p["word"][r] for r in range(p["nruns"])]
        assert p["simple"] == (len(set(words_with_runs)) == len(words_with_runs))
        if p["simple"]:
            for r in range(p["nruns"]):
                assert (p["wshift"][p["word"][r]], p["wlen"][p["word"][r]]) == (p["shift"][r], p["len"][r])
        # order preservation on random keys with these masks
        for _ in range(20):
            a = [(kor[w] & ~knand[w]) | (rnd.getrandbits(32) & kor[w] & knand[w]) for w in range(K)]
            b = [(kor[w] & ~knand[w]) | (rnd.getrandbits(32) & kor[w] & knand[w]) for w in range(K)]

            def prefix(k):
                return [(k[w] >> bit) & 1 for (w, bit) in varying[:n]]

            if prefix(a) != prefix(b):
                assert (prefix(a) < prefix(b)) == (a < b)
