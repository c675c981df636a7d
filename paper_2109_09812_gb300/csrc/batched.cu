// Batched re-indexing of many independent meshes in one launch sequence (reindex_meshes).
//
// The meshes are concatenated: mesh m owns vertices [vtxOff[m], vtxOff[m+1]) and indices
// [elemOff[m]*k, elemOff[m+1]*k), its indices local to its own vertices.  The pipeline of the
// single-mesh path runs once over everything with the mesh id as the most significant key word:
//   k_seg_prepare  position -> mesh lookup tables (one entry per 1024 positions), offsets check,
//                  output offsets set to "unknown"
//   k_seg_flags    local -> global index (range-checked against the mesh's own vertex count),
//                  used-vertex bits (Section 2.1); the global indices are kept in out_idx
//   (compaction, sort, head scan of the single-mesh path, with the mesh word in the key: equal
//    vertices of different meshes stay distinct, and each mesh's unique vertices come out
//    contiguous and ascending; the head scan records each mesh's first output vertex)
//   k_seg_offsets  meshes without used vertices take the next mesh's offset; last = D
//   k_seg_remap    out_idx[j] = oldToNew[global index] - first output vertex of j's mesh (a copy's
//                  entry on the hash path through its representative's)
// Every mesh's result is therefore identical to re-indexing it alone.
#include "internal.h"

namespace reindex {

constexpr uint32_t kErrInvalidArg = 1;

// Largest m in [0, nMeshes) with off[m] * scale <= pos.
__device__ __forceinline__ uint32_t seg_search(const int64_t* off, int32_t nMeshes, int64_t scale, int64_t pos) {
  int32_t lo = 0, hi = nMeshes - 1;
  while (lo < hi) {
    const int32_t mid = (lo + hi + 1) >> 1;
    if (__ldg(off + mid) * scale <= pos) lo = mid; else hi = mid - 1;
  }
  return (uint32_t)lo;
}

__global__ void __launch_bounds__(kThreads) k_seg_prepare(SegArgs seg, int64_t nVtx, int64_t M, uint32_t* blkV,
                                                           uint32_t* blkI, Control* ctrl) {
  const int64_t nbV = (nVtx + kSegBlock - 1) / kSegBlock, nbI = (M + kSegBlock - 1) / kSegBlock;
  const int64_t t0 = blockIdx.x * (int64_t)kThreads + threadIdx.x, stride = (int64_t)gridDim.x * kThreads;
  bool bad = false;
  for (int64_t m = t0; m <= seg.nMeshes; m += stride) {
    seg.outOff[m] = -1;  // unknown until the head scan (or the fix-up) sets it
    if (m < seg.nMeshes) {
      bad |= seg.vtxOff[m] > seg.vtxOff[m + 1] || seg.elemOff[m] > seg.elemOff[m + 1];
    } else {
      bad |= seg.vtxOff[0] != 0 || seg.elemOff[0] != 0 || seg.vtxOff[m] != nVtx || seg.elemOff[m] * seg.k != M;
    }
  }
  if (bad) record_error(ctrl, kErrInvalidArg);
  for (int64_t b = t0; b < nbV; b += stride) blkV[b] = seg_search(seg.vtxOff, seg.nMeshes, 1, b * kSegBlock);
  for (int64_t b = t0; b < nbI; b += stride) blkI[b] = seg_search(seg.elemOff, seg.nMeshes, seg.k, b * kSegBlock);
}

// Local -> global indices with the per-mesh range check, and the used-vertex bits.
__global__ void __launch_bounds__(kThreads) k_seg_flags(const int32_t* idx, int32_t* gidx, int64_t M, SegArgs seg,
                                                         uint32_t* bitmask, Control* ctrl) {
  if (ctrl->err) return;  // bad offsets
  bool bad = false;
  const int64_t t0 = blockIdx.x * (int64_t)kThreads + threadIdx.x, stride = (int64_t)gridDim.x * kThreads;
  for (int64_t j = t0; j < M; j += stride) {
    const uint32_t m = seg_mesh(j, seg.elemOff, seg.k, seg.blkI, seg.nMeshes);
    const int64_t v0 = __ldg(seg.vtxOff + m), nv = __ldg(seg.vtxOff + m + 1) - v0;
    const int32_t local = idx[j];
    if (local < 0 || (int64_t)local >= nv) {
      bad = true;
    } else {
      const uint32_t g = (uint32_t)(v0 + local);
      atomicOr(bitmask + (g >> 5), 1u << (g & 31u));
      gidx[j] = (int32_t)g;
    }
  }
  if (bad) record_error(ctrl, kErrIndexRange);
}

// Meshes without used vertices (no elements) get the offset of the next mesh; outOff[n] = D.
__global__ void __launch_bounds__(1024) k_seg_offsets(SegArgs seg, const Control* ctrl) {
  __shared__ int64_t s_first[1024];
  if (ctrl->err) return;
  const int n = seg.nMeshes, t = threadIdx.x;
  const int chunk = (n + 1023) / 1024;
  const int lo = min(n, t * chunk), hi = min(n, lo + chunk);
  int64_t first = -1;  // leftmost known offset in this thread's chunk
  for (int m = lo; m < hi && first < 0; ++m) first = seg.outOff[m];
  s_first[t] = first;
  __syncthreads();
  if (t == 0) {  // carry for each chunk: the nearest known offset to its right (the last is D)
    int64_t carry = seg.outOff[n];
    for (int q = 1023; q >= 0; --q) {
      const int64_t f = s_first[q];
      s_first[q] = carry;
      if (f >= 0) carry = f;
    }
  }
  __syncthreads();
  int64_t carry = s_first[t];
  for (int m = hi - 1; m >= lo; --m) {
    const int64_t v = seg.outOff[m];
    if (v < 0) seg.outOff[m] = carry; else carry = v;
  }
}

// out_idx[j] = oldToNew[global index] - first output vertex of j's mesh (in place over gidx).
__global__ void __launch_bounds__(kThreads) k_seg_remap(int32_t* io, int64_t M, SegArgs seg,
                                                         const uint32_t* __restrict__ o2n, const Control* ctrl) {
  if (ctrl->err) return;
  const int64_t t0 = blockIdx.x * (int64_t)kThreads + threadIdx.x, stride = (int64_t)gridDim.x * kThreads;
  for (int64_t j = t0; j < M; j += stride) {
    const uint32_t m = seg_mesh(j, seg.elemOff, seg.k, seg.blkI, seg.nMeshes);
    uint32_t v = __ldg(o2n + (uint32_t)io[j]);
    if (v & kRepTag) v = __ldg(o2n + (v & ~kRepTag));  // a copy (hash path): its representative's
    io[j] = (int32_t)((int64_t)v - seg.outOff[m]);
  }
}

static int grid_for(int64_t items, const LaunchCfg& c) {
  int64_t g = (items + kThreads - 1) / kThreads;
  const int64_t cap = (int64_t)c.sms * 8;
  if (g > cap) g = cap;
  return g < 1 ? 1 : (int)g;
}

cudaError_t launch_seg_prepare(const SegArgs& seg, int64_t nVtx, int64_t M, uint32_t* blkV, uint32_t* blkI,
                               Control* ctrl, const LaunchCfg& c, cudaStream_t st) {
  const int64_t work = (nVtx + M) / kSegBlock + seg.nMeshes + 2;
  k_seg_prepare<<<grid_for(work, c), kThreads, 0, st>>>(seg, nVtx, M, blkV, blkI, ctrl);
  return cudaGetLastError();
}

cudaError_t launch_seg_flags(const int32_t* idx, int32_t* gidx, int64_t M, const SegArgs& seg, WsPtrs ws,
                             const LaunchCfg& c, cudaStream_t st) {
  if (M == 0) return cudaSuccess;
  k_seg_flags<<<grid_for(M, c), kThreads, 0, st>>>(idx, gidx, M, seg, ws.bitmask, ws.ctrl);
  return cudaGetLastError();
}

cudaError_t launch_seg_offsets(const SegArgs& seg, const Control* ctrl, cudaStream_t st) {
  k_seg_offsets<<<1, 1024, 0, st>>>(seg, ctrl);
  return cudaGetLastError();
}

cudaError_t launch_seg_remap(int32_t* out_idx, int64_t M, const SegArgs& seg, WsPtrs ws, const LaunchCfg& c,
                             cudaStream_t st) {
  if (M == 0) return cudaSuccess;
  k_seg_remap<<<grid_for(M, c), kThreads, 0, st>>>(out_idx, M, seg, ws.old2new, ws.ctrl);
  return cudaGetLastError();
}

}  // namespace reindex
