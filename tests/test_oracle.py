"""Pins for the serial CPU oracle, against facts the paper and mathematics fix.

None of these compares the oracle with itself: the worked example's printed arrays
(Section 2), an O(n^2) brute force written from the definition, numpy.unique as an
independent library routine, closed-form unique counts of the generators (Table 1's
"vertices (out)" row among them), and invariants of any correct result.
"""
import os
import random
import struct

import numpy as np
import pytest

import oracle
from paper_2109_09812_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "worked_example.txt")


def f32_bits(x: float) -> int:
    return struct.unpack("<I", struct.pack("<f", x))[0]


def load_worked_example():
    rows = {}
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        name, vals = line.split(":", 1)
        rows[name.strip()] = vals.split()
    letters = {k.split(".")[1]: [f32_bits(float(v)) for v in vals] for k, vals in rows.items() if k.startswith("letters.")}
    ints = lambda name: np.array([int(v) for v in rows[name]], dtype=np.int64)
    words = lambda name: np.array([letters[c] for c in rows[name]], dtype=np.uint32)
    return rows, letters, ints, words


# --------------------------------------------------------------------------- worked example


def test_worked_example_paper_steps(oracle_lib):
    """Every intermediate array printed in Sections 2.1-2.4 (tie-independent ones)."""
    rows, letters, ints, words = load_worked_example()
    vtx, idx = words("vtx"), ints("idx").astype(np.int32)
    r = oracle.paper_steps(vtx, idx)
    np.testing.assert_array_equal(r["isUsed"], ints("isUsed"))
    np.testing.assert_array_equal(r["vtxAfterStep1"], words("vtxAfterStep1"))
    np.testing.assert_array_equal(r["vtxAfterStep1"][r["sortedOrgID"]], words("sortedVtx"))
    np.testing.assert_array_equal(r["nodup"], ints("nodup"))
    np.testing.assert_array_equal(r["newIdxInclusive"], ints("newIdxInclusive"))
    np.testing.assert_array_equal(r["newIdx"], ints("newIdx"))
    assert r["newN"] == int(rows["newN"][0])
    np.testing.assert_array_equal(r["newVtx"], words("newVtx"))
    np.testing.assert_array_equal(r["idxNew"], ints("idxNew"))
    # Section 2.5: the new triangles are the old ones, vertex for vertex.
    np.testing.assert_array_equal(r["newVtx"][r["idxNew"]], words("trisNew"))
    np.testing.assert_array_equal(r["newVtx"][r["idxNew"]], vtx[idx])


def test_worked_example_paper_perm_is_a_valid_tie_order(oracle_lib):
    """The paper's perm (Section 2.4) comes from another tie order of the unstable sort; composed
    with newIdx it must give the same old->new map as the oracle's stable order."""
    rows, letters, ints, words = load_worked_example()
    vtx, idx = words("vtx"), ints("idx").astype(np.int32)
    r = oracle.paper_steps(vtx, idx)
    paper_perm = ints("paperPerm")
    assert sorted(paper_perm.tolist()) == list(range(10))
    newIdx = ints("newIdx")
    np.testing.assert_array_equal(newIdx[paper_perm][idx], ints("idxNew"))
    np.testing.assert_array_equal(newIdx[r["perm"]][idx], ints("idxNew"))
    # perm is the inverse of the sorted orgID array
    np.testing.assert_array_equal(r["perm"][r["sortedOrgID"]], np.arange(10))


@pytest.mark.parametrize("fn", ["sort", "map"])
def test_worked_example_final_result(oracle_lib, fn):
    rows, letters, ints, words = load_worked_example()
    vtx, idx = words("vtx"), ints("idx").astype(np.int32)
    out_v, out_i = oracle.reindex_sort(vtx, idx) if fn == "sort" else oracle.reindex_map(vtx, idx, True)
    assert out_v.shape[0] == int(rows["newN"][0]) == 6
    np.testing.assert_array_equal(out_v, words("newVtx"))
    np.testing.assert_array_equal(out_i, ints("idxNew"))


def test_worked_example_map_first_occurrence(oracle_lib):
    """Section 1's map numbers vertices in first-occurrence order; permuting the elements changes
    that numbering but not the canonical result."""
    rows, letters, ints, words = load_worked_example()
    vtx, idx = words("vtx"), ints("idx").astype(np.int32).reshape(4, 3)
    idx2 = idx[[2, 3, 0, 1]].reshape(-1)  # (C,E,F)(C,F,D)(A,B,C)(A,C,D)
    v, i = oracle.reindex_map(vtx, idx2, canonical=False)
    np.testing.assert_array_equal(v, np.array([letters[c] for c in "CEFDAB"], np.uint32))
    np.testing.assert_array_equal(i, [0, 1, 2, 0, 2, 3, 4, 5, 0, 4, 0, 3])
    vc, ic = oracle.reindex_map(vtx, idx2, canonical=True)
    np.testing.assert_array_equal(vc, words("newVtx"))
    np.testing.assert_array_equal(vc[ic], vtx[idx2])


# --------------------------------------------------------------------------- brute force


def brute_force(vtx_words, idx):
    """O(n^2) from the definition: keys as tuples of unsigned ints; a used key's new index is the
    number of distinct used keys strictly less than it (tuples compare lexicographically)."""
    keys = [tuple(int(w) for w in row) for row in vtx_words]
    used = []
    for j in idx:
        k = keys[j]
        if all(k != u for u in used):
            used.append(k)
    rank = {}
    for k in used:
        rank[k] = sum(1 for u in used if u < k)
    out = [None] * len(used)
    for k, r in rank.items():
        out[r] = k
    return np.array(out, dtype=np.uint32).reshape(len(used), len(keys[0]) if keys else 0), \
        np.array([rank[keys[j]] for j in idx], dtype=np.int32)


ALPHABET = [0x00000000, 0x80000000, 0x7FC00000, 0x7FC00001, 0xFFC00000, 0x3F800000, 0xBF800000,
            0x00000001, 0x7F800000, 0xFFFFFFFF, 0x40000000]  # +0, -0, NaNs, 1, -1, denormal, inf, ...


@pytest.mark.parametrize("K", [1, 2, 3, 4, 5, 6, 8])
@pytest.mark.parametrize("trial", range(12))
def test_brute_force_tiny(oracle_lib, K, trial):
    rng = random.Random(1000 * K + trial)
    n = rng.randint(1, 48)
    alpha = ALPHABET[: rng.randint(2, len(ALPHABET))]
    vtx = np.array([[rng.choice(alpha) for _ in range(K)] for _ in range(n)], dtype=np.uint32)
    k = rng.randint(1, 4)
    m = k * rng.randint(1, 16)
    idx = np.array([rng.randrange(n) for _ in range(m)], dtype=np.int32)
    bv, bi = brute_force(vtx, idx)
    for fn in (oracle.reindex_sort, lambda v, i: oracle.reindex_map(v, i, True)):
        ov, oi = fn(vtx, idx)
        np.testing.assert_array_equal(ov, bv)
        np.testing.assert_array_equal(oi, bi)
    r = oracle.paper_steps(vtx, idx)
    np.testing.assert_array_equal(r["newVtx"], bv)
    np.testing.assert_array_equal(r["idxNew"], bi)


@pytest.mark.parametrize("stride", [24, 32, 48, 64])
def test_wide_vertices_extend_the_narrow_result(oracle_lib, stride):
    """Attribute words that are a function of the position words change neither the order nor the
    equality of the vertices: the wide result is the 12-byte result with its attributes appended
    (and D keeps its closed form (G+1)(Gy+1))."""
    m = synth.heightfield_soup(37, 23, 0.1, seed=19)
    w = synth.heightfield_soup_attrs(37, 23, 0.1, seed=19, stride=stride)
    ov, oi = oracle.reindex_sort(m.vtx, m.idx)
    wv, wi = oracle.reindex_sort(w.vtx, w.idx)
    assert wv.shape == (38 * 24, stride // 4)
    np.testing.assert_array_equal(wv[:, :3], ov)
    np.testing.assert_array_equal(wv, synth.with_attributes(ov, stride // 4 - 3, 19))
    np.testing.assert_array_equal(wi, oi)
    mv, mi = oracle.reindex_map(w.vtx, w.idx, canonical=True)
    np.testing.assert_array_equal(mv, wv)
    np.testing.assert_array_equal(mi, wi)


# --------------------------------------------------------------------------- order and equality


def test_raw_bit_equality_and_order(oracle_lib):
    """+0.0 and -0.0 differ; equal NaN payloads merge, different ones do not; order is unsigned
    raw-bit order with word 0 most significant, so negative floats sort after positive ones."""
    vals = [0.0, -0.0, 1.0, -1.0, 2.0]
    vtx = np.array([[f32_bits(v), 0] for v in vals] + [[0x7FC00000, 0], [0x7FC00000, 0], [0x7FC00001, 0],
                                                        [0, 5], [1, 0]], dtype=np.uint32)
    idx = np.arange(vtx.shape[0], dtype=np.int32)
    ov, oi = oracle.reindex_sort(vtx, idx)
    assert ov.shape[0] == vtx.shape[0] - 1  # only the two identical NaNs merge
    assert oi[5] == oi[6] and oi[6] != oi[7]
    assert oi[0] != oi[1]  # +0 vs -0
    expected_order = sorted(set(tuple(r) for r in vtx.tolist()))
    np.testing.assert_array_equal(ov, np.array(expected_order, dtype=np.uint32))
    assert [tuple(r) for r in ov.tolist()].index((0, 5)) < [tuple(r) for r in ov.tolist()].index((1, 0))
    assert oi[3] > oi[4] > oi[2]  # -1.0 (0xBF800000) after 2.0 (0x40000000) after 1.0


def test_numpy_unique_agrees(oracle_lib):
    """numpy.unique over rows sorts lexicographically with unsigned fields: an independent routine."""
    m = synth.heightfield_soup(40, 31, 0.1, seed=77)
    ov, oi = oracle.reindex_sort(m.vtx, m.idx)
    u, inv = np.unique(m.vtx[m.idx.reshape(-1)], axis=0, return_inverse=True)
    np.testing.assert_array_equal(ov, u)
    np.testing.assert_array_equal(oi, inv.reshape(-1))


# --------------------------------------------------------------------------- closed forms


@pytest.mark.parametrize("n,expected", [(8, 81), (64, 4225)])
def test_table1_quad_grid_unique_counts(oracle_lib, n, expected):
    """Table 1, 'vertices (out)': 81 for N=8 and 4.22K for N=64 ((N+1)^2)."""
    m = synth.quad_grid(n)
    assert m.vtx.shape[0] == 5 * n * n  # 'vertices (in)': 320 and 20.48K
    ov, oi = oracle.reindex_sort(m.vtx, m.idx)
    assert ov.shape[0] == expected
    mv, mi = oracle.reindex_map(m.vtx, m.idx, False)
    assert mv.shape[0] == expected


def test_config1_closed_form(oracle_lib):
    m = synth.config_mesh(1)
    assert (m.n_vtx, m.n_elem * m.idx_per_elem) == (432_538, 393_216)
    ov, oi = oracle.reindex_sort(m.vtx, m.idx)
    assert ov.shape[0] == 257 * 257 == m.expected_unique
    check_invariants(m, ov, oi)
    mv, mi = oracle.reindex_map(m.vtx, m.idx, True)
    np.testing.assert_array_equal(mv, ov)
    np.testing.assert_array_equal(mi, oi)


@pytest.mark.parametrize("L", [3, 9])
def test_tet_soup_closed_form(oracle_lib, L):
    m = synth.tet_soup(L, 0.03, seed=11)
    assert m.n_elem == 5 * L ** 3
    ov, oi = oracle.reindex_sort(m.vtx, m.idx)
    assert ov.shape[0] == (L + 1) ** 3
    check_invariants(m, ov, oi)


def check_invariants(m, ov, oi):
    idx = m.idx.reshape(-1)
    D = ov.shape[0]
    assert D <= min(m.n_vtx, idx.size)
    # strictly ascending (lexicographic, unsigned) => no duplicates
    if D > 1:
        a, b = ov[:-1], ov[1:]
        diff = a != b
        first = np.argmax(diff, axis=1)
        assert diff.any(axis=1).all()
        assert (a[np.arange(D - 1), first] < b[np.arange(D - 1), first]).all()
    # every element resolves to bitwise the same vertices
    np.testing.assert_array_equal(ov[oi], m.vtx[idx])
    # every output vertex is referenced
    assert np.bincount(oi, minlength=D).min() >= 1


# --------------------------------------------------------------------------- special cases


def test_no_duplicates_no_unused_is_sort_permutation(oracle_lib):
    rng = np.random.default_rng(5)
    vtx = rng.permutation(1000).astype(np.uint32).reshape(-1, 1) * np.uint32(7919)
    idx = np.arange(1000, dtype=np.int32)
    ov, oi = oracle.reindex_sort(vtx, idx)
    np.testing.assert_array_equal(ov[:, 0], np.sort(vtx[:, 0]))
    np.testing.assert_array_equal(ov[oi], vtx)


def test_all_indices_one_vertex(oracle_lib):
    vtx = np.arange(30, dtype=np.uint32).reshape(10, 3)
    idx = np.full(12, 7, dtype=np.int32)
    ov, oi = oracle.reindex_sort(vtx, idx)
    assert ov.shape[0] == 1 and (oi == 0).all()
    np.testing.assert_array_equal(ov[0], vtx[7])


def test_all_vertices_equal(oracle_lib):
    vtx = np.tile(np.array([[5, 6, 7, 8]], np.uint32), (50, 1))
    idx = np.arange(48, dtype=np.int32)[::-1].copy()
    ov, oi = oracle.reindex_sort(vtx, idx)
    assert ov.shape[0] == 1 and (oi == 0).all()


def test_identity_soup_k1_is_sort_unique(oracle_lib):
    rng = np.random.default_rng(9)
    vtx = rng.integers(0, 40, size=(500, 2), dtype=np.uint32)
    idx = np.arange(500, dtype=np.int32)
    ov, oi = oracle.reindex_sort(vtx, idx)
    u = sorted(set(map(tuple, vtx.tolist())))
    np.testing.assert_array_equal(ov, np.array(u, dtype=np.uint32))


def test_empty_elements(oracle_lib):
    vtx = np.arange(12, dtype=np.uint32).reshape(4, 3)
    ov, oi = oracle.reindex_sort(vtx, np.zeros(0, np.int32))
    assert ov.shape[0] == 0 and oi.size == 0
    assert oracle.paper_steps(vtx, np.zeros(0, np.int32))["newN"] == 0


@pytest.mark.parametrize("bad", [-1, 4, 1 << 30])
def test_index_out_of_range(oracle_lib, bad):
    vtx = np.arange(12, dtype=np.uint32).reshape(4, 3)
    idx = np.array([0, 1, bad], dtype=np.int32)
    for fn in (oracle.reindex_sort, oracle.reindex_map, oracle.paper_steps):
        with pytest.raises(oracle.OracleError) as e:
            fn(vtx, idx)
        assert e.value.code == oracle.INDEX_RANGE


def test_unused_duplicate_of_used_vertex(oracle_lib):
    """An unused vertex that is a bit copy of a used one changes nothing (Step 1's overwrite
    makes every unused vertex such a copy)."""
    vtx = np.array([[1, 2], [3, 4], [1, 2], [9, 9]], dtype=np.uint32)
    idx = np.array([1, 0, 1], dtype=np.int32)
    ov, oi = oracle.reindex_sort(vtx, idx)
    np.testing.assert_array_equal(ov, [[1, 2], [3, 4]])
    np.testing.assert_array_equal(oi, [1, 0, 1])
