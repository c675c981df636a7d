// Steps 4-7 of the pipeline fused into one pass over the sorted (key, old index) items:
//   nodup[j]  = j == 0 || key[j] != key[j-1]                 (Section 2.2, run heads)
//   newIdx[j] = number of run heads before j, minus one unless j is itself a head
//             = inclusive prefix sum of nodup minus one      (Section 2.2 and its footnote)
//   oldToNew[orgID[j]] = newIdx[j]                           (Section 2.4: perm composed with newIdx)
//   newVtx[newIdx[j]] = key[j] for every head j              (Section 2.3)
//   *out_nVtx = total number of heads                        (Section 2.3, newN)
// The prefix sum is a decoupled look-back scan over tiles of 2048 items (256 threads x 8; up to
// four CTAs per SM, so that the others keep working while one waits in its look-back);
// neither nodup nor newIdx is materialised.  If the radix sort packed the keys (their varying
// bits only), run heads are found on the packed keys (equal exactly when the keys are) and only
// the keys written out are restored; a mesh id (batched mode) is read from its packed bits.
#include <atomic>

#include "internal.h"

namespace reindex {

constexpr int kHeadWarps = kHeadThreads / 32;

// S is the item key size.  In batched mode (kSeg) key word 0 is the mesh id: only words 1.. are
// written to out_vtx, and the first item of each mesh records that mesh's first output vertex.
// kMayPack: the sort may have packed the keys (the call allows packing); else they are never packed.
//
// SV > 0 (prefix sort; S = 12 with key word 0 zero): the items carry the 64 most significant
// varying bits of SV-byte vertex keys; run heads are where that prefix changes, and each head
// writes its whole key, read from the vertex array by its old index (loaded before the scan, so
// that the look-back wait covers the latency of these random reads).  k_prefix_check then
// confirms that equal prefixes meant equal keys.
template <int S, bool kSeg, bool kMayPack, int SV = 0>
__global__ void __launch_bounds__(kHeadThreads, (S >= 16 || SV > 0) ? 2 : 4)
    k_head_scan(WsPtrs ws, void* __restrict__ out_vtx, int64_t* __restrict__ out_nVtx, uint32_t nVtx, SegArgs seg,
                const void* __restrict__ vtx) {
  constexpr int K = S / 4;
  constexpr bool kVerify = SV > 0;
  constexpr int KV = kVerify ? SV / 4 : 1;
  // the heads' whole keys are loaded before the scan (their latency hidden by the look-back) up to
  // 32-byte vertices; wider ones are read when stored (eight 16-word keys would not fit in registers)
  constexpr bool kPrefetchKeys = kVerify && SV <= 32;
  __shared__ uint32_t s_warp[kHeadWarps];
  __shared__ uint32_t s_tile, s_prefix;
  __shared__ KeyPack s_pack;
  __shared__ uint32_t s_kconst[K];
  Control* ctrl = ws.ctrl;
  const Plan* plan = ws.plan;
  if (kMayPack && threadIdx.x == 0) {
    s_pack = plan->pack;
#pragma unroll
    for (int q = 0; q < K; ++q) s_kconst[q] = plan->kconst[q];
  }
  if (block_error(ctrl)) return;  // (its barriers also publish s_pack and s_kconst)
  const bool packed = kMayPack && s_pack.on != 0;
  const uint32_t U = plan->U;
  const int64_t ntiles = ((int64_t)U + kHeadTile - 1) / kHeadTile;
  const unsigned char* buf = plan->final_sel ? ws.itemsB : ws.itemsA;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const uint64_t keep = l2_policy_evict_last();
  if (U == 0) {
    if (blockIdx.x == 0 && t == 0) *out_nVtx = 0;
    return;
  }

  for (;;) {
    if (t == 0) s_tile = atomicAdd(&ctrl->ctr[1 + kMaxDigits], 1u);
    __syncthreads();
    const int64_t tile = s_tile;
    if (tile >= ntiles) break;
    const int64_t wbase = tile * kHeadTile + (int64_t)w * 32 * kHeadIpt;

    Item<S> it[kHeadIpt];
#pragma unroll
    for (int r = 0; r < kHeadIpt; ++r) {
      const int64_t j = wbase + r * 32 + lane;
      if (j < U) ItemIO<S>::load_cs(buf, ws.idoff, j, it[r]);
    }
    uint32_t prevk[K];
#pragma unroll
    for (int q = 0; q < K; ++q) prevk[q] = 0;
    if (lane == 0 && wbase > 0 && wbase < U) {
      Item<S> p;
      ItemIO<S>::load(buf, ws.idoff, wbase - 1, p);
#pragma unroll
      for (int q = 0; q < K; ++q) prevk[q] = p.k[q];
    }

    uint32_t within[kHeadIpt];
    uint32_t heads = 0, cnt = 0, firsts = 0;
    uint32_t hkey[kPrefetchKeys ? kHeadIpt : 1][KV];  // whole keys of the heads (prefetched)
#pragma unroll
    for (int r = 0; r < kHeadIpt; ++r) {
      const int64_t j = wbase + r * 32 + lane;
      bool diff = false, mesh_diff = false;
      uint32_t pks[K];  // the preceding item's key
#pragma unroll
      for (int q = 0; q < K; ++q) {
        const uint32_t up = __shfl_up_sync(0xffffffffu, it[r].k[q], 1);
        uint32_t pk;
        if (r == 0) {
          pk = lane ? up : prevk[q];
        } else {
          const uint32_t last = __shfl_sync(0xffffffffu, it[r - 1].k[q], 31);
          pk = lane ? up : last;
        }
        diff |= it[r].k[q] != pk;
        pks[q] = pk;
      }
      if constexpr (kSeg) {  // the mesh id is key word 0 (restored from its packed bits when packed)
        mesh_diff = packed ? unpacked_word0<K>(it[r].k, s_pack, 0u) != unpacked_word0<K>(pks, s_pack, 0u)
                           : it[r].k[0] != pks[0];
      }
      const bool head = (j < U) && (j == 0 || diff);
      if constexpr (kPrefetchKeys)  // the head's whole key, loaded now: in flight during the scan
        if (head && it[r].id < nVtx) load_key_ro<SV>(vtx, it[r].id, hkey[r]);
      const uint32_t m = __ballot_sync(0xffffffffu, head);
      within[r] = cnt + __popc(m & lanemask_lt());
      heads |= (uint32_t)head << r;
      if (kSeg) firsts |= (uint32_t)((j < U) && (j == 0 || mesh_diff)) << r;
      cnt += __popc(m);
    }
    if (lane == 0) s_warp[w] = cnt;
    __syncthreads();
    uint32_t woff = 0, total = 0;
#pragma unroll
    for (int q = 0; q < kHeadWarps; ++q) {
      const uint32_t c = s_warp[q];
      woff += (q < w) ? c : 0u;
      total += c;
    }
    if (w == 0) {
      uint32_t prefix = 0;
      uint32_t* my = ws.lb_head + tile * kLbPad;
      if (tile == 0) {
        if (lane == 0) st_relaxed(my, lb_pre(total));
      } else {
        if (lane == 0) st_relaxed(my, lb_agg(total));
        prefix = warp_lookback(ws.lb_head, tile, ctrl);
        if (lane == 0) st_relaxed(my, lb_pre(prefix + total));
      }
      if (lane == 0) {
        s_prefix = prefix;
        if (tile == ntiles - 1) *out_nVtx = (int64_t)(prefix + total);
      }
    }
    __syncthreads();
    const uint32_t ebase = s_prefix + woff;
#pragma unroll
    for (int r = 0; r < kHeadIpt; ++r) {
      const int64_t j = wbase + r * 32 + lane;
      if (j < U) {
        const bool head = (heads >> r) & 1u;
        const uint32_t e = ebase + within[r];  // heads strictly before j
        const uint32_t nid = head ? e : e - 1u;
        if (it[r].id < nVtx) {
          st_u32_hint(ws.old2new + it[r].id, nid, keep);
          if constexpr (kPrefetchKeys) {
            if (head) store_key<SV>(out_vtx, nid, hkey[r]);  // the unique vertex
          } else if constexpr (kVerify) {
            if (head) {
              load_key_ro<SV>(vtx, it[r].id, hkey[0]);
              store_key<SV>(out_vtx, nid, hkey[0]);
            }
          } else if (head || (kSeg && ((firsts >> r) & 1u))) {
            uint32_t key[K];
#pragma unroll
            for (int q = 0; q < K; ++q) key[q] = it[r].k[q];
            if (packed) unpack_key<K>(key, s_pack, s_kconst);
            if constexpr (kSeg) {
              if (head) {
                uint32_t v[K - 1];
#pragma unroll
                for (int q = 1; q < K; ++q) v[q - 1] = key[q];
                store_key<S - 4>(out_vtx, nid, v);
              }
              if ((firsts >> r) & 1u) seg.outOff[key[0]] = (int64_t)nid;
            } else {
              store_key<S>(out_vtx, nid, key);
            }
          }
        } else {
          record_error(ctrl, kErrInternal);  // corrupted item: never write out of range
        }
      }
    }
    __syncthreads();  // s_tile / s_warp / s_prefix reuse
  }
}

template <int S>
static int occ() {
  int n = 0, m = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_head_scan<S, false, false>, kHeadThreads, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&m, k_head_scan<S, false, true>, kHeadThreads, 0);
  n = min(n, m);
  return n < 1 ? 1 : n;
}

template <int S>
static int occ_unpacked() {
  int n = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_head_scan<S, false, false>, kHeadThreads, 0);
  return n < 1 ? 1 : n;
}

// Resident CTAs per SM of the prefix-sort variant (queried once per stride).
template <int SV>
static int occ_verify() {
  static std::atomic<int> cached{0};
  int n = cached.load(std::memory_order_relaxed);
  if (n == 0) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_head_scan<kPrefixItem, false, false, SV>, kHeadThreads, 0);
    if (n < 1) n = 1;
    cached.store(n, std::memory_order_relaxed);
  }
  return n;
}

template <int SV>
static void launch_verify(int64_t tiles, const LaunchCfg& c, WsPtrs ws, const void* vtx, void* out_vtx,
                          int64_t* out_nVtx, uint32_t nVtx, cudaStream_t st) {
  int64_t g = c.grid_per_tile ? tiles : (int64_t)c.sms * occ_verify<SV>();
  if (g > tiles) g = tiles;
  if (g < 1) g = 1;
  k_head_scan<kPrefixItem, false, false, SV><<<(int)g, kHeadThreads, 0, st>>>(ws, out_vtx, out_nVtx, nVtx,
                                                                                  SegArgs{}, vtx);
}

cudaError_t launch_head_scan_prefix(int S, WsPtrs ws, const void* vtx, void* out_vtx, int64_t* out_nVtx,
                                    uint32_t nVtx, const LaunchCfg& c, cudaStream_t st) {
  const int64_t tiles = (ws.Umax + kHeadTile - 1) / kHeadTile;
  switch (S) {
    case 12: launch_verify<12>(tiles, c, ws, vtx, out_vtx, out_nVtx, nVtx, st); break;
    case 16: launch_verify<16>(tiles, c, ws, vtx, out_vtx, out_nVtx, nVtx, st); break;
    case 20: launch_verify<20>(tiles, c, ws, vtx, out_vtx, out_nVtx, nVtx, st); break;
    case 24: launch_verify<24>(tiles, c, ws, vtx, out_vtx, out_nVtx, nVtx, st); break;
    case 32: launch_verify<32>(tiles, c, ws, vtx, out_vtx, out_nVtx, nVtx, st); break;
    case 48: launch_verify<48>(tiles, c, ws, vtx, out_vtx, out_nVtx, nVtx, st); break;
    case 64: launch_verify<64>(tiles, c, ws, vtx, out_vtx, out_nVtx, nVtx, st); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

int occupancy_head(int S) {
  switch (S) {
    case 4: return occ<4>();
    case 8: return occ<8>();
    case 12: return occ<12>();
    case 16: return occ<16>();
    case 20: return occ<20>();
    case 24: return occ<24>();
    case 48: return occ_unpacked<48>();
    case 64: return occ_unpacked<64>();
    default: return occ<32>();
  }
}

template <int S, bool kSeg>
static void launch_s(int g, WsPtrs ws, void* out_vtx, int64_t* out_nVtx, uint32_t nVtx, const SegArgs& seg,
                     bool may_pack, cudaStream_t st) {
  if (may_pack)
    k_head_scan<S, kSeg, true><<<g, kHeadThreads, 0, st>>>(ws, out_vtx, out_nVtx, nVtx, seg, nullptr);
  else
    k_head_scan<S, kSeg, false><<<g, kHeadThreads, 0, st>>>(ws, out_vtx, out_nVtx, nVtx, seg, nullptr);
}

cudaError_t launch_head_scan(int S, WsPtrs ws, void* out_vtx, int64_t* out_nVtx, uint32_t nVtx,
                             const LaunchCfg& c, const SegArgs* seg, cudaStream_t st) {
  int64_t tiles = (ws.Umax + kHeadTile - 1) / kHeadTile;
  int64_t g = c.grid_per_tile ? tiles : (int64_t)c.sms * c.occ_head;
  if (g > tiles) g = tiles;
  if (g < 1) g = 1;
  const SegArgs none{};
  const bool may_pack = uses_plane(c.sort_kernel) && c.pack_keys != 0;
  if (seg) {
    switch (S) {
      case 8: launch_s<8, true>((int)g, ws, out_vtx, out_nVtx, nVtx, *seg, may_pack, st); break;
      case 12: launch_s<12, true>((int)g, ws, out_vtx, out_nVtx, nVtx, *seg, may_pack, st); break;
      case 16: launch_s<16, true>((int)g, ws, out_vtx, out_nVtx, nVtx, *seg, may_pack, st); break;
      default: launch_s<20, true>((int)g, ws, out_vtx, out_nVtx, nVtx, *seg, may_pack, st); break;
    }
  } else {
    switch (S) {
      case 4: launch_s<4, false>((int)g, ws, out_vtx, out_nVtx, nVtx, none, may_pack, st); break;
      case 8: launch_s<8, false>((int)g, ws, out_vtx, out_nVtx, nVtx, none, may_pack, st); break;
      case 12: launch_s<12, false>((int)g, ws, out_vtx, out_nVtx, nVtx, none, may_pack, st); break;
      case 16: launch_s<16, false>((int)g, ws, out_vtx, out_nVtx, nVtx, none, may_pack, st); break;
      case 20: launch_s<20, false>((int)g, ws, out_vtx, out_nVtx, nVtx, none, may_pack, st); break;
      case 24: launch_s<24, false>((int)g, ws, out_vtx, out_nVtx, nVtx, none, may_pack, st); break;
      case 32: launch_s<32, false>((int)g, ws, out_vtx, out_nVtx, nVtx, none, may_pack, st); break;
      case 48:  // 48- and 64-byte keys are never packed
        k_head_scan<48, false, false><<<(int)g, kHeadThreads, 0, st>>>(ws, out_vtx, out_nVtx, nVtx, none, nullptr);
        break;
      case 64:
        k_head_scan<64, false, false><<<(int)g, kHeadThreads, 0, st>>>(ws, out_vtx, out_nVtx, nVtx, none, nullptr);
        break;
      default: return cudaErrorInvalidValue;
    }
  }
  return cudaGetLastError();
}

}  // namespace reindex
