"""Seeded synthetic mesh generators (inputs only; no re-indexing arithmetic).

This module builds the vertex and index arrays that both the CUDA path and the
CPU oracle consume.  It holds none of the method's arithmetic: it never marks,
sorts, compares or renumbers vertices.  Every random draw comes from one
counter-based generator, SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), keyed by (seed, tag, coordinates),
and every float is produced by IEEE float32 ``+ - *`` in a fixed order (numpy
never contracts to FMA), so the bytes are identical on any host.

Workloads
---------
* ``heightfield_soup(G, Gy, unused_frac, seed)`` -- a G x Gy heightfield grid with
  two triangles per cell.  Every triangle emits its own three float32 xyz
  vertices ("soup to mesh", Section 3.3), then unreferenced random vertices are
  appended and the whole vertex array is permuted with the indices fixed up.
  Lattice points are bit-identical wherever they are emitted, so the number of
  distinct used vertices is exactly (G+1)(Gy+1).
* ``tet_soup(L, unused_frac, seed)`` -- L^3 hexahedral cells split into five
  tetrahedra each; every tet emits its own four 16-byte vertices
  (jittered xyz + scalar field).  Distinct used vertices: (L+1)^3.
* ``quad_grid(n)`` -- the generator of the paper's evaluation (Section 3.5):
  n x n quads, each emitting its four corners plus one unreferenced centre
  vertex (float2 vertices, four indices per element).  Distinct used vertices:
  (n+1)^2, the "vertices (out)" row of Table 1.
* ``batched_heightfield_sizes(n_meshes, ...)`` / ``batched_heightfield(...)`` --
  thousands of independent heightfield soups with log-uniform triangle counts.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_U64 = np.uint64
_GOLDEN = _U64(0x9E3779B97F4A7C15)
_M1 = _U64(0xBF58476D1CE4E5B9)
_M2 = _U64(0x94D049BB133111EB)

# Stream tags: one per independent use of the generator.
TAG_NOISE = 1
TAG_EXTRA = 2
TAG_PERM = 3
TAG_JITTER = 4
TAG_FIELD = 5
TAG_SIZES = 6
TAG_ATTR = 7


def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser applied elementwise to a uint64 array (wrapping arithmetic)."""
    x = np.asarray(x, dtype=_U64)
    with np.errstate(over="ignore"):
        z = x + _GOLDEN
        z = (z ^ (z >> _U64(30))) * _M1
        z = (z ^ (z >> _U64(27))) * _M2
        return z ^ (z >> _U64(31))


def hash_u64(seed: int, tag: int, *coords) -> np.ndarray:
    """Counter-based 64-bit hash of (seed, tag, c0, c1, ...); coords broadcast."""
    h = splitmix64(np.array([(seed * 0x100000001B3 + tag) & 0xFFFFFFFFFFFFFFFF], dtype=_U64))[0]
    h = np.asarray(h, dtype=_U64)
    for c in coords:
        c = np.asarray(c).astype(np.int64).astype(_U64)
        h = splitmix64(h ^ c)
    return h


def unit_float(h: np.ndarray) -> np.ndarray:
    """Top 24 bits of a hash as an exact float32 in [0, 1)."""
    return (h >> _U64(40)).astype(np.float32) * np.float32(1.0 / 16777216.0)


def _feistel(x: np.ndarray, half_bits: int, seed: int) -> np.ndarray:
    """Four-round balanced Feistel network on 2*half_bits-bit integers (a bijection), round
    function = low half_bits of hash(seed, TAG_PERM, round, right half)."""
    mask = _U64((1 << half_bits) - 1)
    hb = _U64(half_bits)
    left, right = x >> hb, x & mask
    for rnd in range(4):
        f = hash_u64(seed, TAG_PERM, rnd, right.astype(np.int64)) & mask
        left, right = right, left ^ f
    return (left << hb) | right


def permutation_dest(n: int, seed: int, i: np.ndarray) -> np.ndarray:
    """Destination of position i under a random permutation of [0, n): a Feistel network on the
    smallest even-bit-width power-of-two domain >= n, with cycle walking into [0, n) (Black and
    Rogaway, "Ciphers with arbitrary finite domains", CT-RSA 2002).  Counter-based: every
    position is computed on its own, so a GPU computes the same permutation element by element."""
    bits = max(2, int(n - 1).bit_length() if n > 1 else 1)
    bits += bits & 1
    x = np.asarray(i, dtype=_U64).copy()
    pending = np.ones(x.shape, dtype=bool)
    nn = _U64(n)
    while pending.any():
        x[pending] = _feistel(x[pending], bits // 2, seed)
        pending = x >= nn
    return x.astype(np.int64)


def permutation(n: int, seed: int) -> np.ndarray:
    """src array of a random permutation of [0, n): position p receives element src[p]."""
    dst = permutation_dest(n, seed, np.arange(n, dtype=np.int64))
    src = np.empty(n, dtype=np.int64)
    src[dst] = np.arange(n, dtype=np.int64)
    return src


@dataclass
class Mesh:
    """An indexed mesh: ``vtx`` is (nVtx, S/4) uint32 raw words, ``idx`` is (nElem, k) int32."""

    vtx: np.ndarray
    idx: np.ndarray
    name: str = ""
    expected_unique: int | None = None
    meta: dict = field(default_factory=dict)

    @property
    def n_vtx(self) -> int:
        return int(self.vtx.shape[0])

    @property
    def stride_bytes(self) -> int:
        return int(self.vtx.shape[1]) * 4

    @property
    def n_elem(self) -> int:
        return int(self.idx.shape[0])

    @property
    def idx_per_elem(self) -> int:
        return int(self.idx.shape[1])


def _value_noise_2d(a: np.ndarray, b: np.ndarray, seed: int) -> np.ndarray:
    """Four octaves of bilinearly interpolated hashed lattice values in [-1, 1);
    cell sizes 64/32/16/8, amplitudes 1, 1/2, 1/4, 1/8.  Depends only on (a, b)."""
    h = np.zeros(np.broadcast(a, b).shape, dtype=np.float32)
    for octave, (cs, amp) in enumerate(((64, 1.0), (32, 0.5), (16, 0.25), (8, 0.125))):
        ca, cb = a // cs, b // cs
        fa = (a % cs).astype(np.float32) * np.float32(1.0 / cs)
        fb = (b % cs).astype(np.float32) * np.float32(1.0 / cs)
        two, one = np.float32(2.0), np.float32(1.0)
        v00 = unit_float(hash_u64(seed, TAG_NOISE, octave, ca, cb)) * two - one
        v10 = unit_float(hash_u64(seed, TAG_NOISE, octave, ca + 1, cb)) * two - one
        v01 = unit_float(hash_u64(seed, TAG_NOISE, octave, ca, cb + 1)) * two - one
        v11 = unit_float(hash_u64(seed, TAG_NOISE, octave, ca + 1, cb + 1)) * two - one
        v0 = v00 + (v10 - v00) * fa
        v1 = v01 + (v11 - v01) * fa
        v = v0 + (v1 - v0) * fb
        h = h + np.float32(amp) * v
    return h.astype(np.float32)


def _append_unused_and_permute(soup: np.ndarray, n_extra: int, extra_fn, seed: int, permute: bool):
    """Append ``n_extra`` unreferenced vertices, then permute all vertices and fix up the indices.

    Returns (vtx, idx_flat) where soup vertex j is referenced by idx_flat[j]."""
    m = soup.shape[0]
    if n_extra:
        extra = extra_fn(np.arange(n_extra, dtype=np.int64))
        vtx = np.concatenate([soup, extra], axis=0)
    else:
        vtx = soup
    n = vtx.shape[0]
    if not permute:
        return np.ascontiguousarray(vtx), np.arange(m, dtype=np.int32)
    dst = permutation_dest(n, seed, np.arange(n, dtype=np.int64))  # vertex i moves to dst[i]
    out = np.empty_like(vtx)
    out[dst] = vtx
    return out, dst[:m].astype(np.int32)


def heightfield_soup(G: int, Gy: int | None = None, unused_frac: float = 0.10, seed: int = 1,
                     permute: bool = True, origin: tuple = (0, 0)) -> Mesh:
    """Triangle soup of a G x Gy-cell heightfield (2 tris per cell, float32 xyz, 3 int32 indices).

    Vertex p(a, b) = (float(a), float(b), noise(a, b)); cell (i, j) emits the triangles
    (p(i,j), p(i+1,j), p(i+1,j+1)) and (p(i,j), p(i+1,j+1), p(i,j+1)), cells in row-major
    order (j outer).  round(unused_frac * 6*G*Gy) unreferenced vertices uniform in
    [0,G] x [0,Gy] x [-2,2) are appended, then the vertex array is permuted.  origin = (a0, b0)
    places the patch at cells [a0, a0+G) x [b0, b0+Gy) of the same field, so that adjacent patches
    share the vertices of their common edge bit for bit."""
    Gy = G if Gy is None else Gy
    a0, b0 = int(origin[0]), int(origin[1])
    i = np.arange(G, dtype=np.int64)[None, :]
    j = np.arange(Gy, dtype=np.int64)[:, None]
    i = np.broadcast_to(i, (Gy, G)).reshape(-1)
    j = np.broadcast_to(j, (Gy, G)).reshape(-1)
    # corner lattice coordinates of the 6 soup vertices of each cell, in emission order
    da = np.array([0, 1, 1, 0, 1, 0], dtype=np.int64)
    db = np.array([0, 0, 1, 0, 1, 1], dtype=np.int64)
    a = (i[:, None] + da[None, :]).reshape(-1)
    b = (j[:, None] + db[None, :]).reshape(-1)
    # evaluate the field once per lattice point, then gather (identical bits by construction)
    la = np.arange(a0, a0 + G + 1, dtype=np.int64)[None, :]
    lb = np.arange(b0, b0 + Gy + 1, dtype=np.int64)[:, None]
    zlat = _value_noise_2d(np.broadcast_to(la, (Gy + 1, G + 1)), np.broadcast_to(lb, (Gy + 1, G + 1)), seed)
    soup = np.empty((a.shape[0], 3), dtype=np.float32)
    soup[:, 0] = (a + a0).astype(np.float32)
    soup[:, 1] = (b + b0).astype(np.float32)
    soup[:, 2] = zlat[b, a]
    m = soup.shape[0]
    n_extra = int(math.floor(unused_frac * m + 0.5))

    def extra_fn(e):
        ux = unit_float(hash_u64(seed, TAG_EXTRA, 0, e))
        uy = unit_float(hash_u64(seed, TAG_EXTRA, 1, e))
        uz = unit_float(hash_u64(seed, TAG_EXTRA, 2, e))
        out = np.empty((e.shape[0], 3), dtype=np.float32)
        out[:, 0] = ux * np.float32(G) + np.float32(a0)
        out[:, 1] = uy * np.float32(Gy) + np.float32(b0)
        out[:, 2] = uz * np.float32(4.0) - np.float32(2.0)
        return out

    vtx, idx = _append_unused_and_permute(soup, n_extra, extra_fn, seed, permute)
    return Mesh(vtx=vtx.view(np.uint32).reshape(-1, 3), idx=idx.reshape(-1, 3),
                name=f"heightfield_soup_{G}x{Gy}", expected_unique=(G + 1) * (Gy + 1),
                meta=dict(G=G, Gy=Gy, unused_frac=unused_frac, seed=seed, n_extra=n_extra))


def with_attributes(vtx_words: np.ndarray, n_attr: int, seed: int) -> np.ndarray:
    """Appends n_attr float32 attribute words to every vertex (e.g. 3 -> a 24-byte position +
    normal vertex, 5 -> 32 bytes with texture coordinates).  Attribute q of a vertex is a function
    of its key words only, so bit-identical vertices stay bit-identical and the unique count is
    unchanged:  h = hash(seed, TAG_ATTR, q, w0, w1, ...);  q < 3: unit_float(h) * 2 - 1 (a
    normal-like component in [-1, 1)),  q >= 3: unit_float(h) (a texture coordinate in [0, 1))."""
    vtx_words = np.ascontiguousarray(vtx_words, dtype=np.uint32)
    n, k0 = vtx_words.shape
    out = np.empty((n, k0 + n_attr), dtype=np.uint32)
    out[:, :k0] = vtx_words
    cols = [vtx_words[:, c].astype(np.int64) for c in range(k0)]
    for q in range(n_attr):
        u = unit_float(hash_u64(seed, TAG_ATTR, q, *cols))
        if q < 3:
            u = u * np.float32(2.0) - np.float32(1.0)
        out[:, k0 + q] = u.astype(np.float32).view(np.uint32)
    return out


def heightfield_soup_attrs(G: int, Gy: int | None = None, unused_frac: float = 0.10, seed: int = 1,
                           stride: int = 32, permute: bool = True) -> Mesh:
    """heightfield_soup with (stride - 12) / 4 attribute words per vertex (with_attributes)."""
    m = heightfield_soup(G, Gy, unused_frac, seed, permute)
    vtx = with_attributes(m.vtx, (stride - 12) // 4, seed)
    return Mesh(vtx=vtx, idx=m.idx, name=f"{m.name}_s{stride}", expected_unique=m.expected_unique,
                meta=dict(m.meta, stride=stride))


def _value_noise_3d(a, b, c, seed: int, cs: int = 16) -> np.ndarray:
    ca, cb, cc = a // cs, b // cs, c // cs
    inv = np.float32(1.0 / cs)
    fa = (a % cs).astype(np.float32) * inv
    fb = (b % cs).astype(np.float32) * inv
    fc = (c % cs).astype(np.float32) * inv
    two, one = np.float32(2.0), np.float32(1.0)

    def v(oa, ob, oc):
        return unit_float(hash_u64(seed, TAG_FIELD, ca + oa, cb + ob, cc + oc)) * two - one

    x00 = v(0, 0, 0) + (v(1, 0, 0) - v(0, 0, 0)) * fa
    x10 = v(0, 1, 0) + (v(1, 1, 0) - v(0, 1, 0)) * fa
    x01 = v(0, 0, 1) + (v(1, 0, 1) - v(0, 0, 1)) * fa
    x11 = v(0, 1, 1) + (v(1, 1, 1) - v(0, 1, 1)) * fa
    y0 = x00 + (x10 - x00) * fb
    y1 = x01 + (x11 - x01) * fb
    return (y0 + (y1 - y0) * fc).astype(np.float32)


# Five-tetrahedron split of a cube; corner k = dx + 2*dy + 4*dz.
_TETS_EVEN = np.array([[0, 1, 2, 4], [3, 1, 2, 7], [5, 1, 4, 7], [6, 2, 4, 7], [1, 2, 4, 7]], dtype=np.int64)
_TETS_ODD = np.array([[1, 0, 3, 5], [2, 0, 3, 6], [4, 0, 5, 6], [7, 3, 5, 6], [0, 3, 5, 6]], dtype=np.int64)


def tet_soup(L: int, unused_frac: float = 0.03, seed: int = 3, permute: bool = True) -> Mesh:
    """Tetrahedral soup over L^3 hex cells, 5 tets per cell, 16-byte vertices.

    Lattice point (a, b, c) maps to (a + jx, b + jy, c + jz, s) with hashed jitters in
    [-0.25, 0.25) and s a trilinear value-noise field, all per lattice point.  The
    split alternates with the parity of (i + j + k).  Each tet emits its own 4 vertices."""
    P = L + 1
    la = np.arange(P, dtype=np.int64)
    A, B, C = np.meshgrid(la, la, la, indexing="ij")  # A[a,b,c] = a
    A, B, C = A.reshape(-1), B.reshape(-1), C.reshape(-1)  # lattice id = (a*P + b)*P + c
    half, quarter = np.float32(0.5), np.float32(0.25)
    lat = np.empty((A.shape[0], 4), dtype=np.float32)
    for axis, coord in enumerate((A, B, C)):
        jit = unit_float(hash_u64(seed, TAG_JITTER, axis, A, B, C)) * half - quarter
        lat[:, axis] = coord.astype(np.float32) + jit
    lat[:, 3] = _value_noise_3d(A, B, C, seed)
    cells = np.arange(L, dtype=np.int64)
    K, J, I = np.meshgrid(cells, cells, cells, indexing="ij")  # k outer, i inner
    I, J, K = I.reshape(-1), J.reshape(-1), K.reshape(-1)
    odd = ((I + J + K) & 1).astype(bool)
    corners = np.where(odd[:, None, None], _TETS_ODD[None], _TETS_EVEN[None])  # (cells, 5, 4)
    dx, dy, dz = corners & 1, (corners >> 1) & 1, (corners >> 2) & 1
    lid = ((I[:, None, None] + dx) * P + (J[:, None, None] + dy)) * P + (K[:, None, None] + dz)
    soup = lat[lid.reshape(-1)]
    m = soup.shape[0]
    n_extra = int(math.floor(unused_frac * m + 0.5))

    def extra_fn(e):
        out = np.empty((e.shape[0], 4), dtype=np.float32)
        for axis in range(3):
            out[:, axis] = unit_float(hash_u64(seed, TAG_EXTRA, axis, e)) * np.float32(L)
        out[:, 3] = unit_float(hash_u64(seed, TAG_EXTRA, 3, e)) * np.float32(2.0) - np.float32(1.0)
        return out

    vtx, idx = _append_unused_and_permute(soup, n_extra, extra_fn, seed, permute)
    return Mesh(vtx=vtx.view(np.uint32).reshape(-1, 4), idx=idx.reshape(-1, 4),
                name=f"tet_soup_{L}^3", expected_unique=P ** 3,
                meta=dict(L=L, unused_frac=unused_frac, seed=seed, n_extra=n_extra))


def quad_grid(n: int) -> Mesh:
    """The paper's evaluation generator (Section 3.5): n x n quads, float2 vertices.

    Quad (i, j) emits its corners (i,j), (i+1,j), (i+1,j+1), (i,j+1) and then an unused centre
    vertex, so every fifth vertex is unreferenced; indices are four per quad."""
    i = np.broadcast_to(np.arange(n, dtype=np.int64)[None, :], (n, n)).reshape(-1)
    j = np.broadcast_to(np.arange(n, dtype=np.int64)[:, None], (n, n)).reshape(-1)
    q = i.shape[0]
    v = np.empty((q, 5, 2), dtype=np.float32)
    fi, fj = i.astype(np.float32), j.astype(np.float32)
    one, half = np.float32(1.0), np.float32(0.5)
    v[:, 0, 0], v[:, 0, 1] = fi, fj
    v[:, 1, 0], v[:, 1, 1] = fi + one, fj
    v[:, 2, 0], v[:, 2, 1] = fi + one, fj + one
    v[:, 3, 0], v[:, 3, 1] = fi, fj + one
    v[:, 4, 0], v[:, 4, 1] = fi + half, fj + half
    base = (np.arange(q, dtype=np.int64) * 5)[:, None]
    idx = (base + np.arange(4, dtype=np.int64)[None, :]).astype(np.int32)
    return Mesh(vtx=v.reshape(-1, 2).view(np.uint32).reshape(-1, 2), idx=idx,
                name=f"quad_grid_{n}", expected_unique=(n + 1) ** 2, meta=dict(n=n))


def batched_heightfield_sizes(n_meshes: int, seed: int = 4, min_tris: int = 64, max_tris: int = 200_000,
                              max_unused: float = 0.10):
    """Per-mesh (G, Gy, unused_frac, seed) for the batched workload: triangle counts
    log-uniform in [min_tris, max_tris], grid G x ceil(T / 2G) with G = round(sqrt(T/2))."""
    m = np.arange(n_meshes, dtype=np.int64)
    u = unit_float(hash_u64(seed, TAG_SIZES, 0, m)).astype(np.float64)
    uf = unit_float(hash_u64(seed, TAG_SIZES, 1, m)).astype(np.float64)
    lo, hi = math.log(min_tris), math.log(max_tris)
    out = []
    for k in range(n_meshes):
        t = int(round(math.exp(lo + (hi - lo) * u[k])))
        g = max(1, int(round(math.sqrt(t / 2.0))))
        gy = max(1, -(-t // (2 * g)))
        out.append((g, gy, float(max_unused * uf[k]), seed * 1_000_000 + k))
    return out


def batched_heightfield(n_meshes: int, seed: int = 4, **kw) -> list[Mesh]:
    """Independent heightfield soups for the batched workload (see ``batched_heightfield_sizes``)."""
    return [heightfield_soup(g, gy, uf, s) for (g, gy, uf, s) in batched_heightfield_sizes(n_meshes, seed, **kw)]


# ---------------------------------------------------------------------------------------------
# Device generators (libsynth.so): bit-identical to the functions above, for workloads too large
# to build on the host.  They return torch CUDA tensors and never touch the re-indexing library.
_synth_lib = None


def _gpu_lib():
    global _synth_lib
    if _synth_lib is None:
        import ctypes
        import os

        path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libsynth.so")
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with `python -m paper_2109_09812_gb300.build`")
        L = ctypes.CDLL(path)
        vp, i64 = ctypes.c_void_p, ctypes.c_int64
        L.synth_heightfield.argtypes = [vp, vp, i64, i64, i64, ctypes.c_uint64, ctypes.c_int, vp]
        L.synth_heightfield.restype = ctypes.c_int
        L.synth_tets.argtypes = [vp, vp, i64, i64, ctypes.c_uint64, ctypes.c_int, vp]
        L.synth_tets.restype = ctypes.c_int
        L.synth_attributes.argtypes = [vp, i64, ctypes.c_int, vp, ctypes.c_int, ctypes.c_uint64, vp]
        L.synth_attributes.restype = ctypes.c_int
        _synth_lib = L
    return _synth_lib


def _stream_ptr(torch, stream):
    import ctypes

    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def heightfield_soup_gpu(G: int, Gy: int | None = None, unused_frac: float = 0.10, seed: int = 1, device="cuda",
                         permute: bool = True, stream=None):
    """heightfield_soup on the GPU: returns (vtx float32 (N, 3), idx int32 (2*G*Gy, 3)) CUDA tensors."""
    import ctypes

    import torch

    Gy = G if Gy is None else Gy
    m = 6 * G * Gy
    n_extra = int(math.floor(unused_frac * m + 0.5))
    vtx = torch.empty((m + n_extra, 3), dtype=torch.float32, device=device)
    idx = torch.empty((2 * G * Gy, 3), dtype=torch.int32, device=device)
    rc = _gpu_lib().synth_heightfield(ctypes.c_void_p(vtx.data_ptr()), ctypes.c_void_p(idx.data_ptr()), G, Gy, n_extra,
                                      seed, int(permute), _stream_ptr(torch, stream))
    if rc:
        raise RuntimeError(f"synth_heightfield: CUDA error {rc}")
    return vtx, idx


def with_attributes_gpu(vtx, n_attr: int, seed: int, stream=None):
    """with_attributes on the GPU: vtx is a CUDA tensor (N, k0) of 4-byte words; returns an int32
    (N, k0 + n_attr) CUDA tensor, bit-identical to the host generator."""
    import ctypes

    import torch

    vtx = vtx.contiguous()
    n, k0 = int(vtx.shape[0]), int(vtx.shape[1])
    out = torch.empty((n, k0 + n_attr), dtype=torch.int32, device=vtx.device)
    rc = _gpu_lib().synth_attributes(ctypes.c_void_p(vtx.data_ptr()), n, k0, ctypes.c_void_p(out.data_ptr()),
                                     k0 + n_attr, seed, _stream_ptr(torch, stream))
    if rc:
        raise RuntimeError(f"synth_attributes: CUDA error {rc}")
    return out


def tet_soup_gpu(L: int, unused_frac: float = 0.03, seed: int = 3, device="cuda", permute: bool = True, stream=None):
    """tet_soup on the GPU: returns (vtx float32 (N, 4), idx int32 (5*L^3, 4)) CUDA tensors."""
    import ctypes

    import torch

    m = 20 * L ** 3
    n_extra = int(math.floor(unused_frac * m + 0.5))
    vtx = torch.empty((m + n_extra, 4), dtype=torch.float32, device=device)
    idx = torch.empty((5 * L ** 3, 4), dtype=torch.int32, device=device)
    rc = _gpu_lib().synth_tets(ctypes.c_void_p(vtx.data_ptr()), ctypes.c_void_p(idx.data_ptr()), L, n_extra, seed,
                               int(permute), _stream_ptr(torch, stream))
    if rc:
        raise RuntimeError(f"synth_tets: CUDA error {rc}")
    return vtx, idx


def serving_requests(n: int, seed: int = 5, min_tris: int = 1000, max_tris: int = 4_000_000, tet_frac: float = 0.3,
                     max_unused: float = 0.10):
    """Request specs of the serving workload: element counts log-uniform in [min_tris, max_tris];
    a fraction tet_frac are tet soups (16-byte vertices, 4 indices), the rest heightfield triangle
    soups (12-byte vertices, 3 indices); unused fraction uniform in [0, max_unused); one seed each.
    Returns a list of dicts(kind, size, unused, seed, n_elem)."""
    r = np.arange(n, dtype=np.int64)
    u_size = unit_float(hash_u64(seed, TAG_SIZES, 10, r)).astype(np.float64)
    u_kind = unit_float(hash_u64(seed, TAG_SIZES, 11, r)).astype(np.float64)
    u_unused = unit_float(hash_u64(seed, TAG_SIZES, 12, r)).astype(np.float64)
    lo, hi = math.log(min_tris), math.log(max_tris)
    out = []
    for k in range(n):
        t = int(round(math.exp(lo + (hi - lo) * u_size[k])))
        if u_kind[k] < tet_frac:
            L = max(1, int(round((t / 5.0) ** (1.0 / 3.0))))
            out.append(dict(kind="tet", size=(L,), unused=float(max_unused * u_unused[k]), seed=seed * 1_000_000 + k,
                            n_elem=5 * L ** 3))
        else:
            g = max(1, int(round(math.sqrt(t / 2.0))))
            gy = max(1, -(-t // (2 * g)))
            out.append(dict(kind="tri", size=(g, gy), unused=float(max_unused * u_unused[k]),
                            seed=seed * 1_000_000 + k, n_elem=2 * g * gy))
    return out


def generate_request(spec: dict, device="cuda", host: bool = False, stream=None):
    """The mesh of one serving request: on the device (torch tensors) or, with host=True, the
    identical Mesh built on the host."""
    if spec["kind"] == "tet":
        (L,) = spec["size"]
        if host:
            return tet_soup(L, spec["unused"], spec["seed"])
        return tet_soup_gpu(L, spec["unused"], spec["seed"], device=device, stream=stream)
    g, gy = spec["size"]
    if host:
        return heightfield_soup(g, gy, spec["unused"], spec["seed"])
    return heightfield_soup_gpu(g, gy, spec["unused"], spec["seed"], device=device, stream=stream)


def config_mesh(cfg: int) -> Mesh:
    """The single-mesh workloads: 1 = 256^2 heightfield soup + 10% unused (seed 1);
    2 = 2048^2 heightfield soup + 5% unused (seed 2); 3 = 128^3 tet soup + 3% unused (seed 3)."""
    if cfg == 1:
        return heightfield_soup(256, 256, 0.10, 1)
    if cfg == 2:
        return heightfield_soup(2048, 2048, 0.05, 2)
    if cfg == 3:
        return tet_soup(128, 0.03, 3)
    raise ValueError(f"unknown single-mesh workload {cfg}")
