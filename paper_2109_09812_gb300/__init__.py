"""GB300-native mesh re-indexing with duplicate- and unused-vertex removal.

Thin Python binding (ctypes) of ``libreindex.so``, whose C ABI is ``include/reindex.h``.
Every step of the method runs in the library's CUDA kernels; this module only checks that
tensors are on the GPU, contiguous and of the right element size, and passes their pointers
and the current CUDA stream.  PyTorch provides device memory and streams only.

There is no CPU fallback: if ``libreindex.so`` is missing, every entry point raises.
Build it with ``python -m paper_2109_09812_gb300.build``.

Method: Wald, "GPGPU-Parallel Re-indexing of Triangle Meshes with Duplicate-Vertex and
Unused-Vertex Removal" (arXiv 2109.09812), Sections 2.1-2.4.

Usage::

    import torch
    import paper_2109_09812_gb300 as rx

    vtx = torch.rand(n, 3, device="cuda")                          # one vertex per row
    idx = torch.randint(0, n, (m, 3), dtype=torch.int32, device="cuda")
    new_vtx, new_idx = rx.reindex(vtx, idx)                        # reads the unique count once
    out_vtx, out_n, out_idx = rx.reindex_mesh(vtx, idx)            # fully asynchronous
    ws = torch.empty(rx.reindex_workspace_size(n, 12, m, 3), dtype=torch.uint8, device="cuda")
    rx.reindex_mesh_ws(vtx, idx, ws, out_vtx, out_n, out_idx)      # no allocation: graph-capturable

Unique vertices come out in ascending raw-bit order, so the result does not depend on the
input's vertex order or on the GPU; new_idx[j] points at the unique copy of vtx[idx[j]].
"""
from __future__ import annotations

import ctypes
import math
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libreindex.so")

REINDEX_OK = 0
REINDEX_ERR_INVALID_ARG = 1
REINDEX_ERR_UNSUPPORTED = 2
REINDEX_ERR_OOM = 3
REINDEX_ERR_INDEX_RANGE = 4
REINDEX_ERR_TIMEOUT = 5
REINDEX_ERR_CUDA = 6
REINDEX_ERR_INTERNAL = 7

# Size of the key-packing description the debug hooks exchange (see reindex_debug_prefix_pack).
KEYPACK_BYTES = 104

KERNEL_NAMES = ["clear", "used_flags", "compact_hist", "sort_plan", "onesweep", "head_scan", "remap", "finalize",
                "seg_prepare", "seg_offsets", "tile_count", "tile_offsets", "tile_scatter", "key_masks", "prefix_gate",
                "prefix_check", "chunk_scatter", "hash_dedup", "resolve"]

# Symbols declared in include/reindex.h (checked by the ABI test).
EXPORTED = ["reindex_status_string", "reindex_workspace_size", "reindex_mesh", "reindex_mesh_ws",
            "reindex_mesh_host", "reindex_stream_status", "reindex_profile_enable", "reindex_profile_collect",
            "reindex_kernel_name", "reindex_mesh_noalloc", "reindex_meshes", "reindex_meshes_workspace_size",
            "reindex_server_create", "reindex_server_submit", "reindex_server_poll", "reindex_server_release",
            "reindex_server_drain", "reindex_server_get_stats", "reindex_server_destroy", "reindex_debug_arena_check",
            "reindex_merge_workspace_size", "reindex_merge_meshes", "reindex_submesh_workspace_size",
            "reindex_submesh", "reindex_autotune", "reindex_tuning_get", "reindex_tuning_set",
            "reindex_debug_stall_tile", "reindex_debug_prefix_pack", "reindex_debug_pack_keys",
            "reindex_workspace_size64", "reindex_mesh64", "reindex_mesh64_ws"]

_lock = threading.Lock()
_lib = None


class ReindexError(RuntimeError):
    def __init__(self, code: int, where: str = ""):
        self.code = int(code)
        super().__init__(f"{where}: {reindex_status_string(self.code)}" if where else reindex_status_string(self.code))


class _ServerConfig(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("max_batch_requests", ctypes.c_int),
                ("num_streams", ctypes.c_int), ("device", ctypes.c_int)]


class _Request(ctypes.Structure):
    _fields_ = [("vtx", ctypes.c_void_p), ("nVtx", ctypes.c_int64), ("vtxStrideBytes", ctypes.c_int),
                ("idx", ctypes.c_void_p), ("nElem", ctypes.c_int64), ("idxPerElem", ctypes.c_int)]


class _Result(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int64), ("status", ctypes.c_int), ("nVtxOut", ctypes.c_int64),
                ("out_vtx", ctypes.c_void_p), ("out_idx", ctypes.c_void_p), ("submit_us", ctypes.c_double),
                ("start_us", ctypes.c_double), ("done_us", ctypes.c_double)]


class _ServerStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("requests_submitted", "requests_started", "requests_done",
                                               "requests_failed", "requests_rejected", "batches", "batches_split",
                                               "arena_bytes_in_use", "pending")]


class _ProfileRecord(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int), ("digit", ctypes.c_int), ("skipped", ctypes.c_int), ("ms", ctypes.c_float),
                ("item_bytes", ctypes.c_int)]


def lib() -> ctypes.CDLL:
    """Load libreindex.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2109_09812_gb300.build` "
                                   "(there is no CPU fallback)")
            L = ctypes.CDLL(LIB_PATH)
            vp, i64, ci = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
            L.reindex_status_string.argtypes = [ci]
            L.reindex_status_string.restype = ctypes.c_char_p
            L.reindex_workspace_size.argtypes = [i64, ci, i64, ci]
            L.reindex_workspace_size.restype = ctypes.c_size_t
            mesh_args = [vp, i64, ci, vp, i64, ci, vp, vp, vp]
            L.reindex_mesh.argtypes = mesh_args + [vp]
            L.reindex_mesh.restype = ci
            L.reindex_mesh_ws.argtypes = mesh_args + [vp, ctypes.c_size_t, vp]
            L.reindex_mesh_ws.restype = ci
            L.reindex_mesh_host.argtypes = mesh_args + [vp]
            L.reindex_mesh64.argtypes = mesh_args + [vp]
            L.reindex_mesh64.restype = ci
            L.reindex_mesh64_ws.argtypes = mesh_args + [vp, ctypes.c_size_t, vp]
            L.reindex_mesh64_ws.restype = ci
            L.reindex_workspace_size64.argtypes = [i64, ci, i64, ci]
            L.reindex_workspace_size64.restype = ctypes.c_size_t
            L.reindex_mesh_host.restype = ci
            L.reindex_stream_status.argtypes = [vp]
            L.reindex_stream_status.restype = ci
            L.reindex_profile_enable.argtypes = [ci]
            L.reindex_profile_enable.restype = None
            L.reindex_profile_collect.argtypes = [ctypes.POINTER(_ProfileRecord), ci]
            L.reindex_profile_collect.restype = ci
            L.reindex_kernel_name.argtypes = [ci]
            L.reindex_kernel_name.restype = ctypes.c_char_p
            L.reindex_meshes_workspace_size.argtypes = [ci, i64, ci, i64, ci]
            L.reindex_meshes_workspace_size.restype = ctypes.c_size_t
            L.reindex_meshes.argtypes = [vp, vp, ci, vp, vp, ci, ci, i64, i64, vp, vp, vp, vp, ctypes.c_size_t, vp]
            L.reindex_meshes.restype = ci
            L.reindex_server_create.argtypes = [ctypes.POINTER(_ServerConfig), ctypes.POINTER(vp)]
            L.reindex_server_create.restype = ci
            L.reindex_server_submit.argtypes = [vp, ctypes.POINTER(_Request), ctypes.POINTER(i64)]
            L.reindex_server_submit.restype = ci
            L.reindex_server_poll.argtypes = [vp, ctypes.POINTER(_Result), ci, ci]
            L.reindex_server_poll.restype = ci
            L.reindex_server_release.argtypes = [vp, i64]
            L.reindex_server_release.restype = ci
            L.reindex_server_drain.argtypes = [vp, ci]
            L.reindex_server_drain.restype = ci
            L.reindex_server_get_stats.argtypes = [vp, ctypes.POINTER(_ServerStats)]
            L.reindex_server_get_stats.restype = ci
            L.reindex_server_destroy.argtypes = [vp]
            L.reindex_server_destroy.restype = None
            L.reindex_merge_workspace_size.argtypes = [ci, i64, ci, i64, ci]
            L.reindex_merge_workspace_size.restype = ctypes.c_size_t
            L.reindex_merge_meshes.argtypes = [vp, vp, ci, vp, vp, ci, ci, i64, i64, vp, vp, vp, vp, ctypes.c_size_t, vp]
            L.reindex_merge_meshes.restype = ci
            L.reindex_submesh_workspace_size.argtypes = [i64, ci, i64, ci]
            L.reindex_submesh_workspace_size.restype = ctypes.c_size_t
            L.reindex_submesh.argtypes = [vp, i64, ci, vp, i64, ci, vp, i64, vp, vp, vp, vp, ctypes.c_size_t, vp]
            L.reindex_submesh.restype = ci
            L.reindex_autotune.argtypes = [vp, i64, ci, vp, i64, ci, vp, vp, vp, vp, ctypes.c_size_t, ci, vp,
                                           ctypes.c_char_p, ci]
            L.reindex_autotune.restype = ci
            L.reindex_tuning_get.argtypes = [ci, ctypes.c_char_p, ci]
            L.reindex_tuning_get.restype = ci
            L.reindex_tuning_set.argtypes = [ci, ctypes.c_char_p]
            L.reindex_tuning_set.restype = ci
            L.reindex_debug_stall_tile.argtypes = [i64]
            L.reindex_debug_stall_tile.restype = None
            L.reindex_debug_arena_check.argtypes = [ctypes.c_uint64, ci, ctypes.c_size_t]
            L.reindex_debug_arena_check.restype = ci
            L.reindex_debug_prefix_pack.argtypes = [vp, vp, ci, vp, ci]
            L.reindex_debug_prefix_pack.restype = ci
            L.reindex_debug_pack_keys.argtypes = [vp, ci, ci, vp, vp, i64, ci, vp]
            L.reindex_debug_pack_keys.restype = ci
            _lib = L
    return _lib


def reindex_status_string(code: int) -> str:
    try:
        return lib().reindex_status_string(int(code)).decode()
    except RuntimeError:
        return f"status {code}"


def reindex_workspace_size(n_vtx: int, stride_bytes: int, n_elem: int, idx_per_elem: int) -> int:
    return int(lib().reindex_workspace_size(n_vtx, stride_bytes, n_elem, idx_per_elem))


def _torch():
    import torch

    return torch


def _stream_handle(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _mesh_geometry(vtx, idx, wide_ok=False):
    """(nVtx, strideBytes, nElem, k) from a (nVtx, ...) tensor with one vertex per row and an
    (nElem, k) int32 (or, where wide_ok, int64) index tensor."""
    torch = _torch()
    if vtx.dim() < 1 or not vtx.is_contiguous():
        raise ValueError("vtx must be a contiguous tensor with one vertex per row")
    ok = (torch.int32, torch.int64) if wide_ok else (torch.int32,)
    if idx.dtype not in ok or idx.dim() != 2 or not idx.is_contiguous():
        raise ValueError("idx must be a contiguous (nElem, idxPerElem) " + (
            "int32 or int64" if wide_ok else "int32") + " tensor")
    stride = math.prod(vtx.shape[1:]) * vtx.element_size()
    return int(vtx.shape[0]), int(stride), int(idx.shape[0]), int(idx.shape[1])


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr() if t is not None and t.numel() else 0)


def reindex_mesh(vtx, idx, out_vtx=None, out_nVtx=None, out_idx=None, stream=None):
    """Asynchronously re-index one mesh on the GPU (workspace from the stream-ordered pool).

    vtx: CUDA tensor (nVtx, ...) with one vertex of 4, 8, 12, 16, 20, 24 or 32 bytes per row
    (any dtype; the raw bits are the key).  idx: CUDA int32 or int64 tensor (nElem, k) (int64:
    reindex_mesh64).  Returns (out_vtx, out_nVtx, out_idx): out_vtx has min(nVtx, nElem*k) rows of
    which the first D = out_nVtx.item() are valid; out_nVtx is a 1-element int64 CUDA tensor
    (negative status on a device error); out_idx has idx's dtype."""
    torch = _torch()
    n_vtx, S, n_elem, k = _mesh_geometry(vtx, idx, wide_ok=True)
    if not (vtx.is_cuda and idx.is_cuda):
        raise ValueError("vtx and idx must be CUDA tensors (use reindex_mesh_host for host buffers)")
    cap = min(n_vtx, n_elem * k)
    if out_vtx is None:
        out_vtx = torch.empty((cap,) + tuple(vtx.shape[1:]), dtype=vtx.dtype, device=vtx.device)
    if out_nVtx is None:
        out_nVtx = torch.empty(1, dtype=torch.int64, device=vtx.device)
    if out_idx is None:
        out_idx = torch.empty_like(idx)
    fn = lib().reindex_mesh64 if idx.dtype == torch.int64 else lib().reindex_mesh
    rc = fn(_ptr(vtx), n_vtx, S, _ptr(idx), n_elem, k, _ptr(out_vtx), _ptr(out_nVtx), _ptr(out_idx),
            _stream_handle(stream))
    if rc:
        raise ReindexError(rc, "reindex_mesh")
    return out_vtx, out_nVtx, out_idx


def reindex_mesh_ws(vtx, idx, ws, out_vtx=None, out_nVtx=None, out_idx=None, stream=None):
    """Like reindex_mesh with a caller-supplied workspace (a CUDA uint8 tensor of at least
    reindex_workspace_size(...) bytes); performs no allocation, so it can be graph-captured
    when the outputs are preallocated."""
    torch = _torch()
    n_vtx, S, n_elem, k = _mesh_geometry(vtx, idx, wide_ok=True)
    cap = min(n_vtx, n_elem * k)
    if out_vtx is None:
        out_vtx = torch.empty((cap,) + tuple(vtx.shape[1:]), dtype=vtx.dtype, device=vtx.device)
    if out_nVtx is None:
        out_nVtx = torch.empty(1, dtype=torch.int64, device=vtx.device)
    if out_idx is None:
        out_idx = torch.empty_like(idx)
    fn = lib().reindex_mesh64_ws if idx.dtype == torch.int64 else lib().reindex_mesh_ws
    rc = fn(_ptr(vtx), n_vtx, S, _ptr(idx), n_elem, k, _ptr(out_vtx), _ptr(out_nVtx), _ptr(out_idx), _ptr(ws),
            ws.numel() * ws.element_size(), _stream_handle(stream))
    if rc:
        raise ReindexError(rc, "reindex_mesh_ws")
    return out_vtx, out_nVtx, out_idx


def reindex_mesh_host(vtx, idx, out_vtx=None, out_idx=None, stream=None):
    """Blocking end-to-end call on HOST tensors (pinned for full copy bandwidth): copies in,
    re-indexes, copies the D unique vertices and the indices back.  Returns (out_vtx[:D], out_idx)."""
    torch = _torch()
    n_vtx, S, n_elem, k = _mesh_geometry(vtx, idx)
    if vtx.is_cuda or idx.is_cuda:
        raise ValueError("reindex_mesh_host takes host tensors")
    cap = min(n_vtx, n_elem * k)
    if out_vtx is None:
        out_vtx = torch.empty((cap,) + tuple(vtx.shape[1:]), dtype=vtx.dtype, pin_memory=True)
    if out_idx is None:
        out_idx = torch.empty_like(idx, pin_memory=True)
    D = ctypes.c_int64(-1)
    rc = lib().reindex_mesh_host(_ptr(vtx), n_vtx, S, _ptr(idx), n_elem, k, _ptr(out_vtx),
                                 ctypes.cast(ctypes.pointer(D), ctypes.c_void_p), _ptr(out_idx),
                                 _stream_handle(stream))
    if rc:
        raise ReindexError(rc, "reindex_mesh_host")
    return out_vtx[: D.value], out_idx


def reindex_meshes_workspace_size(n_meshes: int, n_vtx_total: int, stride_bytes: int, n_elem_total: int,
                                  idx_per_elem: int) -> int:
    return int(lib().reindex_meshes_workspace_size(n_meshes, n_vtx_total, stride_bytes, n_elem_total, idx_per_elem))


def reindex_meshes(vtx, vtx_offsets, idx, elem_offsets, ws=None, out_vtx=None, out_offsets=None, out_idx=None,
                   stream=None):
    """Re-index many independent meshes in one launch sequence (asynchronous, allocation-free
    inside the C call, graph-capturable when ws and the outputs are given).

    vtx: CUDA tensor (nVtxTotal, ...) of concatenated vertices; idx: CUDA int32 (nElemTotal, k)
    of concatenated elements with mesh-local indices; vtx_offsets / elem_offsets: CUDA int64
    tensors of nMeshes+1 offsets.  Returns (out_vtx, out_offsets, out_idx): mesh m's unique
    vertices are out_vtx[out_offsets[m]:out_offsets[m+1]] and its indices are local to them."""
    torch = _torch()
    n_vtx, S, n_elem, k = _mesh_geometry(vtx, idx)
    n_meshes = int(vtx_offsets.numel()) - 1
    if elem_offsets.numel() != n_meshes + 1 or vtx_offsets.dtype != torch.int64 or elem_offsets.dtype != torch.int64:
        raise ValueError("vtx_offsets and elem_offsets must be int64 tensors of nMeshes+1 entries")
    if ws is None:
        ws = torch.empty(max(1, reindex_meshes_workspace_size(n_meshes, n_vtx, S, n_elem, k)), dtype=torch.uint8,
                         device=vtx.device)
    if out_vtx is None:
        out_vtx = torch.empty((min(n_vtx, n_elem * k),) + tuple(vtx.shape[1:]), dtype=vtx.dtype, device=vtx.device)
    if out_offsets is None:
        out_offsets = torch.empty(n_meshes + 1, dtype=torch.int64, device=vtx.device)
    if out_idx is None:
        out_idx = torch.empty_like(idx)
    rc = lib().reindex_meshes(_ptr(vtx), _ptr(vtx_offsets), S, _ptr(idx), _ptr(elem_offsets), k, n_meshes, n_vtx,
                              n_elem, _ptr(out_vtx), _ptr(out_offsets), _ptr(out_idx), _ptr(ws),
                              ws.numel() * ws.element_size(), _stream_handle(stream))
    if rc:
        raise ReindexError(rc, "reindex_meshes")
    return out_vtx, out_offsets, out_idx


def reindex_merge_meshes(vtx, vtx_offsets, idx, elem_offsets, ws=None, out_vtx=None, out_nVtx=None, out_idx=None,
                         stream=None):
    """Merge meshes (Section 3.2): one output mesh, duplicates removed across meshes.  Inputs as for
    reindex_meshes; returns (out_vtx, out_nVtx, out_idx) as reindex_mesh does."""
    torch = _torch()
    n_vtx, S, n_elem, k = _mesh_geometry(vtx, idx)
    n_meshes = int(vtx_offsets.numel()) - 1
    if ws is None:
        ws = torch.empty(max(1, int(lib().reindex_merge_workspace_size(n_meshes, n_vtx, S, n_elem, k))),
                         dtype=torch.uint8, device=vtx.device)
    if out_vtx is None:
        out_vtx = torch.empty((min(n_vtx, n_elem * k),) + tuple(vtx.shape[1:]), dtype=vtx.dtype, device=vtx.device)
    if out_nVtx is None:
        out_nVtx = torch.empty(1, dtype=torch.int64, device=vtx.device)
    if out_idx is None:
        out_idx = torch.empty_like(idx)
    rc = lib().reindex_merge_meshes(_ptr(vtx), _ptr(vtx_offsets), S, _ptr(idx), _ptr(elem_offsets), k, n_meshes,
                                    n_vtx, n_elem, _ptr(out_vtx), _ptr(out_nVtx), _ptr(out_idx), _ptr(ws),
                                    ws.numel() * ws.element_size(), _stream_handle(stream))
    if rc:
        raise ReindexError(rc, "reindex_merge_meshes")
    return out_vtx, out_nVtx, out_idx


def reindex_submesh(vtx, idx, elem_list, ws=None, out_vtx=None, out_nVtx=None, out_idx=None, stream=None):
    """Subset of a mesh (Section 3.4): the elements listed in elem_list (CUDA int32) with the full
    vertex array, compacted.  Returns (out_vtx, out_nVtx, out_idx) with out_idx (nSel, k)."""
    torch = _torch()
    n_vtx, S, n_elem, k = _mesh_geometry(vtx, idx)
    n_sel = int(elem_list.numel())
    if elem_list.dtype != torch.int32 or not elem_list.is_contiguous():
        raise ValueError("elem_list must be a contiguous int32 tensor")
    if ws is None:
        ws = torch.empty(max(1, int(lib().reindex_submesh_workspace_size(n_vtx, S, n_sel, k))), dtype=torch.uint8,
                         device=vtx.device)
    if out_vtx is None:
        out_vtx = torch.empty((min(n_vtx, n_sel * k),) + tuple(vtx.shape[1:]), dtype=vtx.dtype, device=vtx.device)
    if out_nVtx is None:
        out_nVtx = torch.empty(1, dtype=torch.int64, device=vtx.device)
    if out_idx is None:
        out_idx = torch.empty((n_sel, k), dtype=torch.int32, device=vtx.device)
    rc = lib().reindex_submesh(_ptr(vtx), n_vtx, S, _ptr(idx), n_elem, k, _ptr(elem_list), n_sel, _ptr(out_vtx),
                               _ptr(out_nVtx), _ptr(out_idx), _ptr(ws), ws.numel() * ws.element_size(),
                               _stream_handle(stream))
    if rc:
        raise ReindexError(rc, "reindex_submesh")
    return out_vtx, out_nVtx, out_idx


def reindex_autotune(vtx, idx, ws=None, reps: int = 3, stream=None) -> str:
    """Time the kernel variants on this mesh and keep the fastest for its stride (blocking).
    Returns the chosen configuration."""
    torch = _torch()
    n_vtx, S, n_elem, k = _mesh_geometry(vtx, idx)
    if ws is None:
        ws = torch.empty(max(1, reindex_workspace_size(n_vtx, S, n_elem, k)), dtype=torch.uint8, device=vtx.device)
    out_vtx = torch.empty((min(n_vtx, n_elem * k),) + tuple(vtx.shape[1:]), dtype=vtx.dtype, device=vtx.device)
    out_n = torch.empty(1, dtype=torch.int64, device=vtx.device)
    out_idx = torch.empty_like(idx)
    buf = ctypes.create_string_buffer(512)
    rc = lib().reindex_autotune(_ptr(vtx), n_vtx, S, _ptr(idx), n_elem, k, _ptr(out_vtx), _ptr(out_n), _ptr(out_idx),
                                _ptr(ws), ws.numel() * ws.element_size(), reps, _stream_handle(stream), buf, len(buf))
    if rc:
        raise ReindexError(rc, "reindex_autotune")
    return buf.value.decode()


def reindex_tuning_get(stride_bytes: int) -> str:
    buf = ctypes.create_string_buffer(512)
    lib().reindex_tuning_get(stride_bytes, buf, len(buf))
    return buf.value.decode()


def reindex_tuning_set(stride_bytes: int, spec: str) -> None:
    rc = lib().reindex_tuning_set(stride_bytes, spec.encode())
    if rc:
        raise ReindexError(rc, "reindex_tuning_set")


def reindex_stream_status(stream=None) -> int:
    """Synchronise the stream; return and clear the device's sticky device-side error (0 = none)."""
    return int(lib().reindex_stream_status(_stream_handle(stream)))


def reindex(vtx, idx, stream=None):
    """Convenience wrapper: re-index and return (new_vtx[:D], new_idx), synchronising to read D."""
    out_vtx, out_n, out_idx = reindex_mesh(vtx, idx, stream=stream)
    D = int(out_n.item())
    if D < 0:
        raise ReindexError(-D, "reindex (device)")
    return out_vtx[:D], out_idx


def profile_enable(on: bool = True) -> None:
    lib().reindex_profile_enable(1 if on else 0)


def profile_collect(max_records: int = 1 << 16):
    """Per-launch records since the last collect: list of dicts(kernel, name, digit, skipped, ms)."""
    buf = (_ProfileRecord * max_records)()
    n = lib().reindex_profile_collect(buf, max_records)
    if n < 0:
        raise ReindexError(REINDEX_ERR_CUDA, "reindex_profile_collect")
    return [dict(kernel=r.kernel, name=KERNEL_NAMES[r.kernel], digit=r.digit, skipped=bool(r.skipped), ms=r.ms,
                 item_bytes=r.item_bytes)
            for r in buf[: min(n, max_records)]]


class _DeviceArray:
    """A view of device memory owned by the server (exposes __cuda_array_interface__)."""

    def __init__(self, ptr, shape, typestr, keep):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (int(ptr or 0), False),
                                         "version": 3, "strides": None}
        self._keep = keep


class Server:
    """Request loop with continuous batching (reindex_server_* in the C ABI).

    submit(vtx, idx) takes CUDA tensors that must stay alive and unchanged until the request
    finishes; poll() returns finished requests as dicts with zero-copy torch views of the outputs
    (valid until release(id))."""

    def __init__(self, hbm_budget_bytes: int, max_batch_requests: int = 256, num_streams: int = 2, device: int = 0):
        cfg = _ServerConfig(hbm_budget_bytes, max_batch_requests, num_streams, device)
        h = ctypes.c_void_p()
        rc = lib().reindex_server_create(ctypes.byref(cfg), ctypes.byref(h))
        if rc:
            raise ReindexError(rc, "reindex_server_create")
        self._h = h
        self._inputs = {}  # id -> (vtx, idx, stride, shape info) kept alive until finished

    def submit(self, vtx, idx) -> int:
        n_vtx, S, n_elem, k = _mesh_geometry(vtx, idx)
        req = _Request(_ptr(vtx), n_vtx, S, _ptr(idx), n_elem, k)
        rid = ctypes.c_int64(-1)
        rc = lib().reindex_server_submit(self._h, ctypes.byref(req), ctypes.byref(rid))
        if rc:
            raise ReindexError(rc, "reindex_server_submit")
        self._inputs[rid.value] = (vtx, idx, S, tuple(vtx.shape[1:]), vtx.dtype)
        return rid.value

    def poll(self, max_results: int = 1024, wait_ms: int = 0):
        torch = _torch()
        buf = (_Result * max_results)()
        n = lib().reindex_server_poll(self._h, buf, max_results, wait_ms)
        out = []
        for r in buf[:max(n, 0)]:
            vtx, idx, S, vshape, vdtype = self._inputs.pop(r.id)
            res = dict(id=r.id, status=r.status, n_out=r.nVtxOut, submit_us=r.submit_us, start_us=r.start_us,
                       done_us=r.done_us, out_vtx=None, out_idx=None)
            if r.status == REINDEX_OK:
                res["out_idx"] = torch.as_tensor(_DeviceArray(r.out_idx, tuple(idx.shape), "<i4", self),
                                                 device=idx.device)
                words = _DeviceArray(r.out_vtx if r.nVtxOut else 0, (r.nVtxOut, S // 4), "<i4", self)
                res["out_vtx"] = torch.as_tensor(words, device=vtx.device)
            out.append(res)
        return out

    def release(self, rid: int) -> None:
        rc = lib().reindex_server_release(self._h, rid)
        if rc:
            raise ReindexError(rc, "reindex_server_release")

    def drain(self, timeout_ms: int = 600_000) -> None:
        rc = lib().reindex_server_drain(self._h, timeout_ms)
        if rc:
            raise ReindexError(rc, "reindex_server_drain")

    def stats(self) -> dict:
        st = _ServerStats()
        lib().reindex_server_get_stats(self._h, ctypes.byref(st))
        return {n: getattr(st, n) for n, _ in _ServerStats._fields_}

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib().reindex_server_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def debug_prefix_pack(kor, knand) -> dict:
    """Host-only: the prefix sort's choice of key bits for per-word masks (test hook)."""
    import numpy as np

    kor = np.ascontiguousarray(kor, dtype=np.uint32)
    knand = np.ascontiguousarray(knand, dtype=np.uint32)
    buf = ctypes.create_string_buffer(KEYPACK_BYTES)
    nbits = lib().reindex_debug_prefix_pack(kor.ctypes.data, knand.ctypes.data, int(kor.shape[0]), buf,
                                            KEYPACK_BYTES)
    if nbits < 0:
        raise ValueError("bad masks")
    b = buf.raw
    n = b[2]
    return dict(on=b[0], nbits=b[1], nruns=n, word=list(b[3:3 + n]), shift=list(b[19:19 + n]),
                len=list(b[35:35 + n]), pos=list(b[51:51 + n]), simple=b[67], wshift=list(b[68:84]),
                wlen=list(b[84:100]), returned=nbits, raw=b)


def debug_pack_keys(pack: bytes, keys, mode: int, kconst=None):
    """Host-only: the kernels' key packing applied to keys (n, K) uint32 (test hook); mode 0/1
    pack (general / one run per word), 2 unpacks with kconst, 3 returns word 0 of the unpacked keys."""
    import numpy as np

    keys = np.ascontiguousarray(keys, dtype=np.uint32)
    n, K = keys.shape
    out = np.zeros(n if mode == 3 else (n, K), dtype=np.uint32)
    kc = np.ascontiguousarray(kconst if kconst is not None else np.zeros(K), dtype=np.uint32)
    buf = ctypes.create_string_buffer(bytes(pack), len(pack))
    rc = lib().reindex_debug_pack_keys(buf, len(pack), K, kc.ctypes.data, keys.ctypes.data, n, mode, out.ctypes.data)
    if rc:
        raise ValueError("bad arguments")
    return out


def debug_arena_check(seed: int, ops: int, size: int) -> int:
    """Host-only self-check of the server's arena allocator (0 = no inconsistency)."""
    return int(lib().reindex_debug_arena_check(seed, ops, size))
