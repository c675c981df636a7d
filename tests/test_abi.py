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
    for S in (48, 64):  # position + normal + texture coordinates + tangent: the same model
        b = rx.reindex_workspace_size(n, S, ne, k)
        assert 2 * U * (S + 4) + U + 4 * n <= b <= 2 * U * (S + 4) + U + 4 * n + 64 * 2**20
    for S in (5, 28, 36, 40, 128):  # unsupported strides
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
    # too many vertices for 31-bit look-back counts; too many indices for int32
    assert L.reindex_mesh(fake, 1 << 31, 12, fake, 3, 3, fake, fake, fake, z) == rx.REINDEX_ERR_UNSUPPORTED
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


def _masks_and_keys(rnd, K, n, max_runs=16):
    """Per-word varying-bit masks (at most max_runs runs in all), constant bits, and n keys."""
    while True:
        masks = []
        for _ in range(K):
            style = rnd.randrange(4)
            if style == 0:
                m = 0
            elif style == 1:
                m = 0xFFFFFFFF
            elif style == 2:
                m = 0
                for _ in range(rnd.randrange(1, 4)):
                    lo = rnd.randrange(32)
                    hi = rnd.randrange(lo, 32)
                    m |= ((1 << (hi - lo + 1)) - 1) << lo
            else:
                m = rnd.getrandbits(32) & rnd.getrandbits(32)
            masks.append(m)
        runs = [(w, lo, ln) for w in range(K - 1, -1, -1) for (lo, ln) in _runs_of(masks[w])]
        if len(runs) <= max_runs and sum(r[2] for r in runs) <= 255:  # positions are bytes
            break
    const = [rnd.getrandbits(32) & ~m & 0xFFFFFFFF for m in masks]
    pool = [[const[w] | (rnd.getrandbits(32) & masks[w]) for w in range(K)] for _ in range(max(1, n // 3))]
    keys = np.array([rnd.choice(pool) for _ in range(n)], dtype=np.uint32)  # with repeats
    return masks, const, runs, keys


def _runs_of(m):
    out, b = [], 0
    while b < 32:
        if not (m >> b) & 1:
            b += 1
            continue
        e = b
        while e < 32 and (m >> e) & 1:
            e += 1
        out.append((b, e - b))
        b = e
    return out


def _keypack_bytes(runs, K):
    """The 104-byte packing description (layout of reindex_debug_prefix_pack) for runs listed least
    significant first as (word, lowest bit, length)."""
    b = bytearray(104)
    b[0] = 1
    b[1] = sum(r[2] for r in runs) & 0xFF
    b[2] = len(runs)
    pos = 0
    per_word = {}
    for i, (w, lo, ln) in enumerate(runs):
        b[3 + i], b[19 + i], b[35 + i], b[51 + i] = w, lo, ln, pos
        pos += ln
        per_word.setdefault(w, []).append((lo, ln))
    b[67] = int(all(len(v) == 1 for v in per_word.values()))
    for w, v in per_word.items():
        if len(v) == 1:
            b[68 + w], b[84 + w] = v[0]
    return bytes(b)


@pytest.mark.parametrize("K", [1, 2, 3, 4, 5, 6, 8, 12, 16])
def test_key_packing_roundtrip_and_order(L, K):
    """The kernels' key packing, run on the host: packing keeps only the varying bits and keeps
    their order, so packed keys compare exactly like the keys (equal iff equal); unpacking with
    the constant bits restores every key; the one-run-per-word variant agrees with the general one;
    word 0 (a batched call's mesh id) is read back from the packed bits alone."""
    import random

    rnd = random.Random(7 + K)
    for trial in range(60):
        masks, const, runs, keys = _masks_and_keys(rnd, K, 64)
        pack = _keypack_bytes(runs, K)
        nbits = sum(r[2] for r in runs)
        packed = rx.debug_pack_keys(pack, keys, 0)
        if pack[67]:
            np.testing.assert_array_equal(rx.debug_pack_keys(pack, keys, 1), packed)
        np.testing.assert_array_equal(rx.debug_pack_keys(pack, packed, 2, const), keys)
        np.testing.assert_array_equal(rx.debug_pack_keys(pack, packed, 3, const), keys[:, 0])
        for q in range(K):  # nothing above the packed bits
            lo_bit = 32 * (K - 1 - q)
            if lo_bit >= nbits:
                assert not packed[:, q].any()
            elif nbits - lo_bit < 32:
                assert not (packed[:, q] >> np.uint32(nbits - lo_bit)).any()
        kt = [tuple(int(x) for x in r) for r in keys]
        pt = [tuple(int(x) for x in r) for r in packed]
        for i in range(0, 64, 2):
            a, b = i, (i * 7 + 3) % 64
            assert (kt[a] < kt[b]) == (pt[a] < pt[b]) and (kt[a] == kt[b]) == (pt[a] == pt[b])


@pytest.mark.parametrize("K", [3, 4, 6, 8])
def test_prefix_packing_of_keys(L, K):
    """The prefix sort's packing (the chosen bits, then the kernels' packing): the prefix sits in
    the low two words, equal keys get equal prefixes, and keys with different prefixes compare
    like their prefixes."""
    import random

    rnd = random.Random(70 + K)
    for trial in range(60):
        masks, const, runs, keys = _masks_and_keys(rnd, K, 64, max_runs=64)
        kor = np.array([m | c for m, c in zip(masks, const)], np.uint32)
        knand = np.array([m | (~c & ~m & 0xFFFFFFFF) for m, c in zip(masks, const)], np.uint32)
        p = rx.debug_prefix_pack(kor, knand)
        packed = rx.debug_pack_keys(p["raw"], keys, 1 if p["simple"] else 0)
        assert not packed[:, : K - 2].any()
        kt = [tuple(int(x) for x in r) for r in keys]
        pre = [tuple(int(x) for x in r[K - 2:]) for r in packed]
        for a in range(64):
            b = (a * 5 + 1) % 64
            if kt[a] == kt[b]:
                assert pre[a] == pre[b]
            elif pre[a] != pre[b]:
                assert (pre[a] < pre[b]) == (kt[a] < kt[b])


def test_noalloc_scratch_holds_the_largest_accepted_mesh(L):
    """reindex_mesh_noalloc accepts every mesh of up to REINDEX_NOALLOC_MAX_VTX vertices, whatever
    its stride and element count; its fixed scratch must hold the workspace of each of them."""
    src = open(HEADER).read()
    max_vtx = int(re.search(r"#define REINDEX_NOALLOC_MAX_VTX (\d+)", src).group(1))
    m = re.search(r"#define REINDEX_NOALLOC_SCRATCH_BYTES \((\d+)u << (\d+)\)", src)
    scratch = int(m.group(1)) << int(m.group(2))
    for S in (4, 8, 12, 16, 20, 24, 32):
        for k in (1, 3, 4):
            for n_elem in (1, max_vtx // k, max_vtx, 10 * max_vtx):
                b = rx.reindex_workspace_size(max_vtx, S, n_elem, k)
                assert 0 < b <= scratch, (S, k, n_elem, b, scratch)


def test_int64_entry_points_host_checks(L):
    """The int64-index entry points: 8-byte aligned index arrays, no 2^31 cap on the index count (the
    workspace grows with min(nVtx, indices) only); reindex_mesh64 takes up to 2^40 vertices (in
    vertex ranges), its workspace variant up to 2^31 - 1."""
    z = ctypes.c_void_p(0)
    fake = ctypes.c_void_p(1 << 20)  # never dereferenced: every call below fails its host checks
    assert L.reindex_mesh64(fake, (1 << 40) + 1, 12, fake, 3, 3, fake, fake, fake, z) == rx.REINDEX_ERR_UNSUPPORTED
    assert L.reindex_mesh64_ws(fake, 1 << 31, 12, fake, 3, 3, fake, fake, fake, fake, ctypes.c_size_t(1 << 40), z) \
        == rx.REINDEX_ERR_UNSUPPORTED
    assert rx.lib().reindex_workspace_size64(1 << 31, 12, 3, 3) == 0
    assert L.reindex_mesh64(fake, 10, 6, fake, 3, 3, fake, fake, fake, z) == rx.REINDEX_ERR_UNSUPPORTED
    assert L.reindex_mesh64(fake, 10, 12, ctypes.c_void_p((1 << 20) + 4), 3, 3, fake, fake, fake, z) \
        == rx.REINDEX_ERR_INVALID_ARG  # int64 indices must be 8-byte aligned
    assert L.reindex_mesh64(fake, 10, 12, fake, (1 << 40) // 3 + 1, 3, fake, fake, fake, z) \
        == rx.REINDEX_ERR_UNSUPPORTED
    n = 1000
    big = rx.lib().reindex_workspace_size64(n, 12, 1 << 33, 3)  # 2^33 elements: more than 2^31 indices
    assert big == rx.reindex_workspace_size(n, 12, 1000, 3) > 0
    assert rx.lib().reindex_workspace_size64((1 << 31) - 1, 4, 10, 3) > 0
    assert rx.reindex_workspace_size((1 << 31) - 1, 4, 10, 3) > 0
    assert rx.reindex_workspace_size(1 << 31, 4, 10, 3) == 0


def test_noalloc_limits_stated_for_48_and_64_byte_vertices(L):
    """The header's stated no-allocation limits for 48- and 64-byte vertices are the largest meshes
    whose workspace (with as many indices as vertices: the largest case) fits the scratch."""
    src = open(HEADER).read()
    m = re.search(r"every mesh of up to ([\d,]+) or ([\d,]+) vertices does", src)
    stated = [int(m.group(1).replace(",", "")), int(m.group(2).replace(",", ""))]
    scratch = 20 << 20
    for S, n in zip((48, 64), stated):
        assert rx.reindex_workspace_size(n, S, n, 1) <= scratch < rx.reindex_workspace_size(n + 1, S, n + 1, 1)
