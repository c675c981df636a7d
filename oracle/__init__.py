"""Python binding of the serial CPU oracle (``reindex_oracle.cpp``).

TEST INFRASTRUCTURE ONLY: imported by the test suite, the smoke check and the
benchmark's CPU-baseline leg.  The product path (the CUDA library and its binding)
never imports this package, and this package imports nothing from the product path.

All wrappers take a vertex array as an (nVtx, S/4) uint32 array of raw words and an
index array of int32 (any shape; flattened), and return numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "reindex_oracle.cpp")
_LIB = os.path.join(_HERE, "libreindex_oracle.so")
_lock = threading.Lock()
_lib = None

OK, BAD_ARG, INDEX_RANGE = 0, -1, -2


class OracleError(RuntimeError):
    def __init__(self, code: int):
        super().__init__({BAD_ARG: "invalid argument", INDEX_RANGE: "index out of range"}.get(code, str(code)))
        self.code = code


def build(force: bool = False) -> str:
    """Compile the oracle with the host C++ compiler (plain -O2; no vector intrinsics)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    """Load the oracle library.  ``REINDEX_ORACLE_LIB`` names another build of the same source
    (the mutation tests use it to load deliberately broken copies)."""
    global _lib
    with _lock:
        if _lib is None:
            path = os.environ.get("REINDEX_ORACLE_LIB") or build()
            L = ctypes.CDLL(path)
            vp, i64, i32p, i64p, u8p = ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p
            L.oracle_reindex_sort.argtypes = [vp, i64, ctypes.c_int, i32p, i64, vp, i64p, i32p]
            L.oracle_reindex_map.argtypes = [vp, i64, ctypes.c_int, i32p, i64, ctypes.c_int, vp, i64p, i32p]
            L.oracle_paper_steps.argtypes = [vp, i64, ctypes.c_int, i32p, i64, u8p, vp, i32p, u8p, i32p, i32p,
                                             i32p, vp, i64p, i32p]
            for f in (L.oracle_reindex_sort, L.oracle_reindex_map, L.oracle_paper_steps):
                f.restype = ctypes.c_int
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data) if a.size else ctypes.c_void_p(0)


def _prep(vtx: np.ndarray, idx: np.ndarray):
    vtx = np.ascontiguousarray(vtx, dtype=np.uint32)
    if vtx.ndim != 2:
        raise ValueError("vtx must be (nVtx, S/4) uint32 words")
    idx = np.ascontiguousarray(idx, dtype=np.int32).reshape(-1)
    return vtx, idx


def reindex_sort(vtx: np.ndarray, idx: np.ndarray):
    """Plain definition: returns (out_vtx (D, K) uint32, out_idx (M,) int32)."""
    vtx, idx = _prep(vtx, idx)
    n, K = vtx.shape
    out_v = np.zeros((max(min(n, idx.size), 1), K), dtype=np.uint32)
    out_i = np.zeros(idx.size, dtype=np.int32)
    D = ctypes.c_int64(-1)
    rc = lib().oracle_reindex_sort(_ptr(vtx), n, 4 * K, _ptr(idx), idx.size, _ptr(out_v), ctypes.byref(D), _ptr(out_i))
    if rc:
        raise OracleError(rc)
    return out_v[: D.value].copy(), out_i


def reindex_map(vtx: np.ndarray, idx: np.ndarray, canonical: bool = True):
    """Section 1's std::map method; canonical=True relabels to ascending key order."""
    vtx, idx = _prep(vtx, idx)
    n, K = vtx.shape
    out_v = np.zeros((max(min(n, idx.size), 1), K), dtype=np.uint32)
    out_i = np.zeros(idx.size, dtype=np.int32)
    D = ctypes.c_int64(-1)
    rc = lib().oracle_reindex_map(_ptr(vtx), n, 4 * K, _ptr(idx), idx.size, int(canonical), _ptr(out_v),
                                  ctypes.byref(D), _ptr(out_i))
    if rc:
        raise OracleError(rc)
    return out_v[: D.value].copy(), out_i


def paper_steps(vtx: np.ndarray, idx: np.ndarray) -> dict:
    """Steps 1-4 of Section 2 with every intermediate array (see reindex_oracle.cpp)."""
    vtx, idx = _prep(vtx, idx)
    n, K = vtx.shape
    r = dict(
        isUsed=np.zeros(n, np.uint8), vtxAfterStep1=np.zeros((n, K), np.uint32), sortedOrgID=np.zeros(n, np.int32),
        nodup=np.zeros(n, np.uint8), newIdxInclusive=np.zeros(n, np.int32), newIdx=np.zeros(n, np.int32),
        perm=np.zeros(n, np.int32), newVtx=np.zeros((max(n, 1), K), np.uint32), idxNew=np.zeros(idx.size, np.int32))
    nn = ctypes.c_int64(-1)
    rc = lib().oracle_paper_steps(_ptr(vtx), n, 4 * K, _ptr(idx), idx.size, _ptr(r["isUsed"]),
                                  _ptr(r["vtxAfterStep1"]), _ptr(r["sortedOrgID"]), _ptr(r["nodup"]),
                                  _ptr(r["newIdxInclusive"]), _ptr(r["newIdx"]), _ptr(r["perm"]), _ptr(r["newVtx"]),
                                  ctypes.byref(nn), _ptr(r["idxNew"]))
    if rc:
        raise OracleError(rc)
    r["newN"] = nn.value
    r["newVtx"] = r["newVtx"][: nn.value].copy()
    return r
