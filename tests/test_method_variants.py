"""The library's restructurings of the method, checked on the CPU against the plain definition
(the oracle's reindex_sort), independently of the CUDA path: each is built here from the oracle
itself, with its free choices made at random, and must give the plain definition's result.

- Duplicates removed first (the hash path): any copy of a key may become its representative; the
  representatives alone are sorted; every copy then takes its representative's new index.
- Vertex ranges (meshes beyond 2^31 - 1 vertices): each range's used vertices are re-indexed on
  their own, the ranges' unique vertices concatenated and re-indexed once more, and the two maps
  composed for every index.
"""
import numpy as np
import pytest

import oracle


def _mesh(rng, n, m, K, values):
    pool = rng.integers(0, 2**32, size=(values, K), dtype=np.uint64).astype(np.uint32)
    vtx = pool[rng.integers(0, values, size=n)]
    idx = rng.integers(0, n, size=m).astype(np.int32)
    return vtx, idx


def _rank_of_used(vtx, used):
    """(unique keys, rank of each vertex in `used`) by the plain definition on the used vertices."""
    uv, ui = oracle.reindex_sort(vtx, used.astype(np.int32))
    return uv, ui


@pytest.mark.parametrize("K,values", [(1, 7), (3, 50), (3, 5000), (8, 11)])
def test_duplicates_removed_first(K, values):
    rng = np.random.default_rng(100 * K + values)
    for n, m in [(1, 1), (40, 100), (3000, 5000)]:
        vtx, idx = _mesh(rng, n, m, K, values)
        want_v, want_i = oracle.reindex_sort(vtx, idx)
        used = np.unique(idx)
        # a representative per distinct key, chosen at random among the key's used copies
        keys = vtx[used].view(np.dtype((np.void, 4 * K))).reshape(-1)
        order = rng.permutation(used.size)
        rep_of_key = {}
        for j in order:
            rep_of_key.setdefault(keys[j].tobytes(), used[j])
        reps = np.array(sorted(rep_of_key.values()), dtype=np.int64)
        # sort the representatives alone; their new indices
        uv, rank = _rank_of_used(vtx, reps)
        new_of_rep = dict(zip(reps.tolist(), rank.tolist()))
        # every copy takes its representative's new index
        rep_of = {int(v): int(rep_of_key[k.tobytes()]) for v, k in zip(used, keys)}
        got_i = np.array([new_of_rep[rep_of[int(v)]] for v in idx], dtype=np.int32)
        np.testing.assert_array_equal(uv, want_v)
        np.testing.assert_array_equal(got_i, want_i)


@pytest.mark.parametrize("K,values,width", [(1, 7, 16), (3, 40, 37), (3, 4000, 64), (2, 300, 1000)])
def test_vertex_ranges_compose_to_the_single_level_result(K, values, width):
    rng = np.random.default_rng(7 * K + values + width)
    for n, m in [(1, 1), (50, 120), (5000, 4000)]:
        vtx, idx = _mesh(rng, n, m, K, values)
        want_v, want_i = oracle.reindex_sort(vtx, idx)
        # level 1: each range [lo, lo + width) on its own: its used vertices' ranks, its unique keys
        rank = np.full(n, -1, dtype=np.int64)
        cat, off = [], [0]
        for lo in range(0, n, width):
            hi = min(n, lo + width)
            used = np.unique(idx[(idx >= lo) & (idx < hi)])
            if used.size == 0:
                off.append(off[-1])
                continue
            uv, r = _rank_of_used(vtx, used)
            rank[used] = r
            cat.append(uv)
            off.append(off[-1] + uv.shape[0])
        cat = np.concatenate(cat)
        # level 2: the concatenated range-unique keys with identity indices
        fv, map2 = oracle.reindex_sort(cat, np.arange(cat.shape[0], dtype=np.int32))
        # composition: index -> its range's unique key -> its final index
        got_i = map2[np.array(off)[idx // width] + rank[idx]]
        np.testing.assert_array_equal(fv, want_v)
        np.testing.assert_array_equal(got_i, want_i)


def _prefix64(keys):
    """The 64 most significant varying bits of each key (K uint32 words, word 0 most significant),
    in order, as one uint64 per key: an order-preserving prefix of the key (the bits left out are
    constant over the keys or less significant than every bit kept)."""
    K = keys.shape[1]
    bits = np.unpackbits(keys.astype(">u4").view(np.uint8).reshape(keys.shape[0], 4 * K), axis=1)  # MSB first
    varying = np.flatnonzero(bits.max(axis=0) != bits.min(axis=0))[:64]
    p = np.zeros(keys.shape[0], dtype=np.uint64)
    for b in varying:
        p = (p << np.uint64(1)) | bits[:, b].astype(np.uint64)
    return p << np.uint64(64 - len(varying)) if len(varying) < 64 else p


def _prefix_path(vtx, idx):
    """Sort the used vertices by prefix (stable); each run of equal prefixes gives one unique
    vertex (its first key); the check: every used vertex equals its run's key.  Returns the result,
    or None when the check fails (two keys share a prefix: the full-key sort must run)."""
    used = np.unique(idx)
    keys = vtx[used]
    pre = _prefix64(keys)
    order = np.argsort(pre, kind="stable")
    sp = pre[order]
    head = np.ones(sp.size, dtype=bool)
    head[1:] = sp[1:] != sp[:-1]
    run = np.cumsum(head) - 1  # run rank of each sorted used vertex
    heads = keys[order][head]
    if not np.array_equal(keys[order], heads[run]):
        return None
    rank = np.empty(used.size, dtype=np.int64)
    rank[order] = run
    new = np.full(vtx.shape[0], -1, dtype=np.int64)
    new[used] = rank
    return heads, new[idx].astype(np.int32)


@pytest.mark.parametrize("K,values,collide", [(4, 5000, False), (8, 3000, False), (4, 7, True), (8, 5, True)])
def test_prefix_sort_with_check_and_fallback(K, values, collide):
    """The prefix sort: when the check passes its result is the plain definition's; keys built to
    share their 64-bit prefixes fail the check (the full-key sort then runs)."""
    rng = np.random.default_rng(31 * K + values)
    fallbacks = 0
    for n, m in [(1, 1), (60, 150), (4000, 6000)]:
        if collide:  # few values per word, all words varying: more than 64 varying bits
            pool = rng.integers(0, 2**32, size=(values,), dtype=np.uint64).astype(np.uint32)
            vtx = pool[rng.integers(0, values, size=(n, K))]
        else:
            vtx = _mesh(rng, n, 1, K, values)[0]
        idx = rng.integers(0, n, size=m).astype(np.int32)
        want_v, want_i = oracle.reindex_sort(vtx, idx)
        got = _prefix_path(vtx, idx)
        if got is None:
            fallbacks += 1
            got = oracle.reindex_sort(vtx, idx)  # the full-key sort
        np.testing.assert_array_equal(got[0], want_v)
        np.testing.assert_array_equal(got[1], want_i)
    if collide:
        assert fallbacks >= 1
