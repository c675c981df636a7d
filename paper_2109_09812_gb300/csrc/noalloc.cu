// reindex_mesh_noalloc: re-index one small mesh with scratch memory that lives inside the library,
// so that the call itself allocates nothing.
//
// Who needs this: callers that cannot (or must not) allocate device memory at call time -- a
// host program that committed its whole device-memory budget up front and accounts for every
// byte, a real-time loop in which cudaMalloc/cudaFree would synchronise the device and stall
// its other streams, or a plugin whose host application forbids allocations behind its back.
// They pass inputs and outputs as usual; the scratch is the static array below.
//
// The array is a file-scope __device__ variable (REINDEX_NOALLOC_SCRATCH_BYTES), held on a device
// from the moment the CUDA runtime loads this file's device code there until the process exits.
// With lazy module loading (the CUDA default) that moment is the first call on the device, whose
// cudaGetSymbolAddress loads the code: that first call reserves the 20 MiB (and may synchronise).
// Host code only sees a stand-in for the array's name; the real device address is looked up once
// per device (with that device current) and cached.  Every call shares the array: the pipeline's
// first kernel zeroes the parts that must start at zero, and calls whose work overlaps on the GPU
// (for example two calls on two streams without ordering between them) race on it.
#include <mutex>

#include "internal.h"
#include "reindex.h"

namespace {

constexpr size_t kScratchBytes = REINDEX_NOALLOC_SCRATCH_BYTES;

// The scratch holds the workspace of the largest mesh the entry point accepts, for every stride
// (the workspace grows with min(nVtx, nElem * idxPerElem), so nElem * idxPerElem = nVtx is the
// largest case).  A change of the workspace layout that breaks this fails to compile.
constexpr bool fits_every_stride() {
  const int strides[] = {4, 8, 12, 16, 20, 24, 32};
  for (int S : strides)
    if (reindex::ws_bytes(REINDEX_NOALLOC_MAX_VTX, S, REINDEX_NOALLOC_MAX_VTX) > kScratchBytes) return false;
  return true;
}
static_assert(fits_every_stride(), "the no-allocation scratch must hold the workspace of the largest accepted mesh");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once per device).
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> g(g_mu);
  if (g_addr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    if (p == nullptr) return cudaErrorInvalidSymbol;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" reindex_status reindex_mesh_noalloc(const void* vtx, int64_t nVtx, int vtxStrideBytes,
                                               const int32_t* idx, int64_t nElem, int idxPerElem,
                                               void* out_vtx, int64_t* out_nVtx, int32_t* out_idx,
                                               reindex_stream_t stream) {
  if (nVtx > REINDEX_NOALLOC_MAX_VTX) return REINDEX_ERR_UNSUPPORTED;
  const size_t need = reindex_workspace_size(nVtx, vtxStrideBytes, nElem, idxPerElem);
  if (need == 0) return nVtx < 0 || nElem < 0 || idxPerElem < 1 ? REINDEX_ERR_INVALID_ARG : REINDEX_ERR_UNSUPPORTED;
  if (need > kScratchBytes) return REINDEX_ERR_UNSUPPORTED;
  void* ws = nullptr;
  if (scratch_address(&ws) != cudaSuccess) return REINDEX_ERR_CUDA;
  return reindex_mesh_ws(vtx, nVtx, vtxStrideBytes, idx, nElem, idxPerElem, out_vtx, out_nVtx, out_idx, ws,
                         kScratchBytes, stream);
}
