// Stable compaction of the used vertices into (key, old index) sort items, fused with the
// upfront digit histograms of the radix sort.
//
// The paper (Section 2.1) instead overwrites every unused vertex with a used one and then sorts
// all nVtx vertices.  An overwritten vertex is a copy of a used key, so the set of distinct keys
// and every used vertex's new index are unchanged; dropping the unused vertices here gives the
// same result while sorting U <= nVtx items instead of nVtx.
//
// Tiles of 2048 vertices (8 warps x 8 rows x 32 lanes); a tile's output offset comes from a
// decoupled look-back over per-tile used counts, so items keep vertex order.  The same pass
// counts, per byte digit d of the key, how many used vertices have each digit value; or, for the
// "tiles" sort (kHistNone, after k_key_masks and the plan), it packs each key's varying bits when
// the plan packs them and writes each item's digit of the first radix pass into the digit plane.
//
// k_key_masks (tiles sort, before the plan): the OR of every key word over the used vertices and
// the OR of its complement; a bit varies between used vertices iff it is set in both.
#include <algorithm>
#include <atomic>

#include "internal.h"

namespace reindex {

// S is the vertex stride.  In batched mode (kSeg) the item key is the owning mesh's id followed
// by the vertex words (SI = S + 4 bytes), so that one sort groups the items by mesh.
// stall_tile >= 0 (a test hook, -1 otherwise): that tile never publishes its look-back status, so
// its successors' bounded waits run out and the call ends with REINDEX_ERR_TIMEOUT.
template <int S, int kHist, bool kSeg>
__global__ void __launch_bounds__(kThreads) k_compact(const void* __restrict__ vtx, int64_t nVtx, WsPtrs ws,
                                                       int64_t tilesV, SegArgs seg, int64_t stall_tile) {
  constexpr bool kPrefix = kHist == kHistPrefix;  // items keep the 8-byte prefix of the packed key
  constexpr int KL = kSeg ? S / 4 + 1 : S / 4;     // key words loaded per vertex
  constexpr int SI = kPrefix ? kPrefixItem : 4 * KL;  // item key bytes
  constexpr int K = SI / 4;
  constexpr int P = 4 * KL;  // byte digits per key
  constexpr bool kCount = kHist != kHistNone && kHist != kHistMasks && !kPrefix;
  constexpr bool kMasks = kHist == kHistMasks;  // tiles sort without packing: the plan comes after
  constexpr bool kPacks = kHist == kHistNone || kPrefix;  // the plan ran first (packing known)
  __shared__ uint32_t s_hist[kCount ? P * kRadix : 1];
  __shared__ uint32_t s_warp[kWarps];
  __shared__ uint32_t s_tile, s_prefix;
  __shared__ KeyPack s_pack;
  __shared__ int s_first;
  __shared__ uint32_t s_dmask;
  Control* ctrl = ws.ctrl;
  if (kPacks && threadIdx.x == 0) {
    s_pack = ws.plan->pack;
    s_first = ws.plan->first;
    s_dmask = (1u << ws.plan->dbits) - 1u;  // the first digit: the packed key's low dbits bits
  }
  if (block_error(ctrl)) return;  // an invalid index was seen: nothing downstream is meaningful
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  if constexpr (kCount)
    for (int i = t; i < P * kRadix; i += kThreads) s_hist[i] = 0;
  // digit of the first radix pass (tiles sort): byte 0 of the packed key, or a byte of the key
  // (kHistMasks: key byte 0, the first pass's digit unless that byte is constant)
  const bool packed = kPacks && s_pack.on;
  const int first = kMasks ? 0 : (kCount ? -1 : s_first);
  const int fword = packed ? K - 1 : K - 1 - (first >> 2), fshift = packed ? 0 : (first & 3) * 8;
  uint32_t kor[K], knand[K];  // kHistMasks: this thread's OR of each key word and of its complement
#pragma unroll
  for (int q = 0; q < K; ++q) kor[q] = knand[q] = 0;

  for (;;) {
    if (t == 0) s_tile = atomicAdd(&ctrl->ctr[0], 1u);
    __syncthreads();
    const int64_t tile = s_tile;
    if (tile >= tilesV) break;
    const int64_t vbase = tile * kCompactTile + (int64_t)w * kCompactRows * 32;

    // Used bits of this warp's 8 rows of 32 vertices (bits past nVtx are never set).
    uint32_t myword = 0;
    if (lane < kCompactRows) {
      const int64_t wi = (vbase >> 5) + lane;
      if (wi * 32 < nVtx) myword = ws.bitmask[wi];
    }
    uint32_t k[kCompactRows][KL];
    uint32_t pos[kCompactRows];
    uint32_t used = 0, cnt = 0;
#pragma unroll
    for (int r = 0; r < kCompactRows; ++r) {
      const uint32_t word = __shfl_sync(0xffffffffu, myword, r);
      const uint32_t u = (word >> lane) & 1u;
      if (u) {
        const int64_t v = vbase + r * 32 + lane;
        if constexpr (kSeg) {
          uint32_t kv[S / 4];
          load_key<S>(vtx, v, kv);
          k[r][0] = seg_mesh(v, seg.vtxOff, 1, seg.blkV, seg.nMeshes);
#pragma unroll
          for (int q = 0; q < S / 4; ++q) k[r][1 + q] = kv[q];
        } else {
          load_key<S>(vtx, v, k[r]);
        }
      }
      pos[r] = cnt + __popc(word & lanemask_lt());
      cnt += __popc(word);
      used |= u << r;
    }
    if (lane == 0) s_warp[w] = cnt;
    __syncthreads();
    uint32_t woff = 0, total = 0;
#pragma unroll
    for (int q = 0; q < kWarps; ++q) {
      const uint32_t c = s_warp[q];
      woff += (q < w) ? c : 0u;
      total += c;
    }
    if (w == 0 && tile != stall_tile) {
      uint32_t prefix = 0;
      uint32_t* my = ws.lb_compact + tile * kLbPad;
      if (tile == 0) {
        if (lane == 0) st_relaxed(my, lb_pre(total));
      } else {
        if (lane == 0) st_relaxed(my, lb_agg(total));
        prefix = warp_lookback(ws.lb_compact, tile, ctrl);
        if (lane == 0) st_relaxed(my, lb_pre(prefix + total));
      }
      if (lane == 0) {
        s_prefix = prefix;
        if (tile == tilesV - 1) {
          ctrl->U = prefix + total;
          if (kPacks) ws.plan->U = prefix + total;  // the plan ran before the compaction
        }
      }
    }
    if (tile == stall_tile && t == 0) s_prefix = 0;  // the stalled tile writes at [0, total): in bounds
    __syncthreads();
    const int64_t obase = (int64_t)s_prefix + woff;

#pragma unroll
    for (int r = 0; r < kCompactRows; ++r) {
      const uint32_t u = (used >> r) & 1u;
      const uint32_t umask = __ballot_sync(0xffffffffu, u);
      if (umask == 0) continue;  // warp-uniform
      if (u) {
        Item<SI> it;
        it.id = (uint32_t)(vbase + r * 32 + lane);
        if constexpr (kPrefix) {  // pack the whole key; its low 8 bytes are the prefix's bits
          uint32_t full[KL];
#pragma unroll
          for (int q = 0; q < KL; ++q) full[q] = k[r][q];
          if (s_pack.simple)
            pack_key_simple<KL>(full, s_pack);
          else
            pack_key<KL>(full, s_pack);
          it.k[0] = 0;
          it.k[1] = full[KL - 2];
          it.k[2] = full[KL - 1];
        } else {
#pragma unroll
          for (int q = 0; q < K; ++q) it.k[q] = k[r][q];
        }
        if constexpr (!kCount) {
          if (packed && !kPrefix) {
            if (s_pack.simple)
              pack_key_simple<K>(it.k, s_pack);
            else
              pack_key<K>(it.k, s_pack);
          }
          if (first >= 0)
            ws.digits[obase + pos[r]] =
                (uint8_t)((key_word<K>(it.k, fword) >> fshift) & (kPacks ? s_dmask : 0xFFu));
        }
        if constexpr (kMasks) {
#pragma unroll
          for (int q = 0; q < K; ++q) {
            kor[q] |= it.k[q];
            knand[q] |= ~it.k[q];
          }
        }
        ItemIO<SI>::store(ws.itemsA, ws.idoff, obase + pos[r], it);
      }
      if constexpr (!kCount) continue;
      // Histograms.  Many key bytes are heavily skewed (exponent bytes, the zero low bytes of
      // small integers), and lanes adding to the same bin in one instruction serialise, so the
      // lanes that share a digit are combined first (three variants, chosen per device).
      const int leader = __ffs(umask) - 1;
#pragma unroll
      for (int d = 0; d < P; ++d) {
        const uint32_t dig = u ? key_digit<KL>(k[r], d) : 0u;
        if (kHist == kHistMatchAny) {
          const uint32_t peers = __match_any_sync(0xffffffffu, u ? dig : 0x100u);
          if (u && (peers & lanemask_lt()) == 0) atomicAdd(&s_hist[d * kRadix + dig], (uint32_t)__popc(peers));
        } else if (kHist == kHistPeel) {
          const uint32_t d0 = __shfl_sync(0xffffffffu, dig, leader);
          const bool same = u && dig == d0;
          const uint32_t same_mask = __ballot_sync(0xffffffffu, same);
          if (lane == leader) atomicAdd(&s_hist[d * kRadix + d0], (uint32_t)__popc(same_mask));
          if (u && !same) atomicAdd(&s_hist[d * kRadix + dig], 1u);
        } else {
          const uint32_t d0 = __shfl_sync(0xffffffffu, dig, leader);
          if (__all_sync(0xffffffffu, !u || dig == d0)) {
            if (lane == leader) atomicAdd(&s_hist[d * kRadix + d0], (uint32_t)__popc(umask));
          } else if (u) {
            atomicAdd(&s_hist[d * kRadix + dig], 1u);
          }
        }
      }
    }
    __syncthreads();  // s_tile, s_warp and s_prefix are rewritten by the next tile
  }
  __syncthreads();
  if constexpr (kCount) {
    for (int i = t; i < P * kRadix; i += kThreads) {
      const uint32_t c = s_hist[i];
      if (c) atomicAdd(ws.hist + i, c);
    }
  }
  if constexpr (kMasks) {
#pragma unroll
    for (int q = 0; q < K; ++q) {
      const uint32_t a = __reduce_or_sync(0xffffffffu, kor[q]), b = __reduce_or_sync(0xffffffffu, knand[q]);
      if (lane == 0) {
        if (a) atomicOr(&ctrl->kor[q], a);
        if (b) atomicOr(&ctrl->knand[q], b);
      }
    }
  }
}

// kVec: the vertex array is 16-byte aligned, so a thread reads 4 consecutive vertices (S words of
// 16 bytes) with vector loads; the tail and unaligned arrays go one vertex at a time.
template <int S, bool kSeg, bool kVec>
__global__ void __launch_bounds__(kThreads) k_key_masks(const void* __restrict__ vtx, int64_t nVtx, WsPtrs ws,
                                                         SegArgs seg) {
  constexpr int K = kSeg ? S / 4 + 1 : S / 4;
  constexpr int KV = S / 4;  // words per vertex
  if (block_error(ws.ctrl)) return;
  uint32_t kor[K], knand[K];
#pragma unroll
  for (int q = 0; q < K; ++q) kor[q] = knand[q] = 0;
  const int64_t stride = (int64_t)gridDim.x * kThreads;
  int64_t done = 0;
  if constexpr (kVec) {
    const uint4* v4 = reinterpret_cast<const uint4*>(vtx);
    const int64_t n4 = nVtx >> 2;  // groups of 4 vertices = KV vectors
    for (int64_t g = blockIdx.x * (int64_t)kThreads + threadIdx.x; g < n4; g += stride) {
      // vertex loads first (independent of the used bits, so both are in flight together)
      uint32_t wds[4 * KV];
#pragma unroll
      for (int i = 0; i < KV; ++i) {
        const uint4 x = __ldcs(v4 + g * KV + i);
        wds[4 * i] = x.x; wds[4 * i + 1] = x.y; wds[4 * i + 2] = x.z; wds[4 * i + 3] = x.w;
      }
      const uint32_t bits = (__ldg(ws.bitmask + (g >> 3)) >> ((g & 7) * 4)) & 0xFu;  // used bits of the 4
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (!((bits >> j) & 1u)) continue;
        uint32_t k[K];
        if constexpr (kSeg) {
          k[0] = seg_mesh(g * 4 + j, seg.vtxOff, 1, seg.blkV, seg.nMeshes);
#pragma unroll
          for (int q = 0; q < KV; ++q) k[1 + q] = wds[j * KV + q];
        } else {
#pragma unroll
          for (int q = 0; q < KV; ++q) k[q] = wds[j * KV + q];
        }
#pragma unroll
        for (int q = 0; q < K; ++q) {
          kor[q] |= k[q];
          knand[q] |= ~k[q];
        }
      }
    }
    done = n4 << 2;
  }
  for (int64_t v = done + blockIdx.x * (int64_t)kThreads + threadIdx.x; v < nVtx; v += stride) {
    if (!((__ldg(ws.bitmask + (v >> 5)) >> (v & 31)) & 1u)) continue;
    uint32_t k[K];
    if constexpr (kSeg) {
      uint32_t kv[S / 4];
      load_key<S>(vtx, v, kv);
      k[0] = seg_mesh(v, seg.vtxOff, 1, seg.blkV, seg.nMeshes);
#pragma unroll
      for (int q = 0; q < S / 4; ++q) k[1 + q] = kv[q];
    } else {
      load_key<S>(vtx, v, k);
    }
#pragma unroll
    for (int q = 0; q < K; ++q) {
      kor[q] |= k[q];
      knand[q] |= ~k[q];
    }
  }
#pragma unroll
  for (int q = 0; q < K; ++q) {
    const uint32_t a = __reduce_or_sync(0xffffffffu, kor[q]), b = __reduce_or_sync(0xffffffffu, knand[q]);
    if ((threadIdx.x & 31) == 0) {
      if (a) atomicOr(&ws.ctrl->kor[q], a);
      if (b) atomicOr(&ws.ctrl->knand[q], b);
    }
  }
}

// Prefix sort check: every used vertex's key must equal the unique vertex it was given
// (out_vtx[oldToNew[i]], written by the head scan).  Then each run of equal prefixes held one
// key, runs with different prefixes hold different keys, and the runs are in key order: the
// result is exact.  Otherwise ctrl->amb is set and the full-key sort runs.  The vertex array is
// streamed (four vertices per thread with vector loads when 16-byte aligned); the unique vertices
// are gathered (a fraction of the vertex array, largely served by L2).
template <int S, bool kVec>
__global__ void __launch_bounds__(kThreads) k_prefix_check(const void* __restrict__ vtx, int64_t nVtx,
                                                            const void* __restrict__ out_vtx, WsPtrs ws) {
  constexpr int KV = S / 4;
  if (block_error(ws.ctrl)) return;
  const uint32_t U = ws.plan->U;  // unique vertices are fewer (an index past it fails the check)
  bool bad = false;
  const int64_t stride = (int64_t)gridDim.x * kThreads;
  int64_t done = 0;
  if constexpr (kVec) {
    const uint4* v4 = reinterpret_cast<const uint4*>(vtx);
    const int64_t n4 = nVtx >> 2;
    for (int64_t g = blockIdx.x * (int64_t)kThreads + threadIdx.x; g < n4; g += stride) {
      // the four vertices, their used bits and their new indices, all loads in flight together
      uint32_t wds[4 * KV];
#pragma unroll
      for (int i = 0; i < KV; ++i) {
        const uint4 x = __ldcs(v4 + g * KV + i);
        wds[4 * i] = x.x; wds[4 * i + 1] = x.y; wds[4 * i + 2] = x.z; wds[4 * i + 3] = x.w;
      }
      const uint4 n4 = __ldg(reinterpret_cast<const uint4*>(ws.old2new) + g);
      const uint32_t nids[4] = {n4.x, n4.y, n4.z, n4.w};
      const uint32_t bits = (__ldg(ws.bitmask + (g >> 3)) >> ((g & 7) * 4)) & 0xFu;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (!((bits >> j) & 1u)) continue;
        if (nids[j] >= U) {
          bad = true;
          continue;
        }
        uint32_t u[KV];
        load_key_ro<S>(out_vtx, nids[j], u);
#pragma unroll
        for (int q = 0; q < KV; ++q) bad |= u[q] != wds[j * KV + q];
      }
    }
    done = n4 << 2;
  }
  for (int64_t v = done + blockIdx.x * (int64_t)kThreads + threadIdx.x; v < nVtx; v += stride) {
    if (!((__ldg(ws.bitmask + (v >> 5)) >> (v & 31)) & 1u)) continue;
    const uint32_t nid = __ldg(ws.old2new + v);
    if (nid >= U) {
      bad = true;
      continue;
    }
    uint32_t k[KV], u[KV];
    load_key<S>(vtx, v, k);
    load_key_ro<S>(out_vtx, nid, u);
#pragma unroll
    for (int q = 0; q < KV; ++q) bad |= u[q] != k[q];
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&ws.ctrl->amb, 1u);
}

template <int S>
static int occ() {
  int a = 0, b = 0, c = 0;
  int n = 0;
  if constexpr (S >= kHugeMin) {  // 48- and 64-byte keys: unpacked keys, masks mode only
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_compact<S, kHistMasks, false>, kThreads, 0);
    return n < 1 ? 1 : n;
  }
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_compact<S, kHistNone, false>, kThreads, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_compact<S, kHistMasks, false>, kThreads, 0);
  n = min(a, b);
  if constexpr (S < kWideMin) {  // upfront histograms (onesweep sort) for keys of up to 20 bytes
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_compact<S, kHistUniform, false>, kThreads, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_compact<S, kHistPeel, false>, kThreads, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c, k_compact<S, kHistMatchAny, false>, kThreads, 0);
    n = min(n, min(a, min(b, c)));
  }
  if constexpr (S <= 16) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_compact<S, kHistUniform, true>, kThreads, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_compact<S, kHistNone, true>, kThreads, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c, k_compact<S, kHistMasks, true>, kThreads, 0);
    n = min(n, min(a, min(b, c)));
  }
  return n < 1 ? 1 : n;
}

int occupancy_compact(int S) {
  switch (S) {
    case 4: return occ<4>();
    case 8: return occ<8>();
    case 12: return occ<12>();
    case 16: return occ<16>();
    case 20: return occ<20>();
    case 24: return occ<24>();
    case 48: return occ<48>();
    case 64: return occ<64>();
    default: return occ<32>();
  }
}

// Resident CTAs per SM of one compaction variant (queried once; persistent grids are sized by it).
template <int S, int kHist, bool kSeg>
static int occ_variant() {
  static std::atomic<int> cached{0};
  int n = cached.load(std::memory_order_relaxed);
  if (n == 0) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_compact<S, kHist, kSeg>, kThreads, 0);
    if (n < 1) n = 1;
    cached.store(n, std::memory_order_relaxed);
  }
  return n;
}

template <int S, int kHist, bool kSeg>
static void launch_v(int64_t g, int sms, bool persistent, const void* vtx, int64_t nVtx, WsPtrs ws, int64_t tilesV,
                     const SegArgs& seg, cudaStream_t st) {
  if (persistent) g = std::min<int64_t>(g, (int64_t)sms * occ_variant<S, kHist, kSeg>());
  k_compact<S, kHist, kSeg><<<(int)g, kThreads, 0, st>>>(vtx, nVtx, ws, tilesV, seg, debug_stall_tile());
}

template <int S, bool kSeg>
static void launch_s(int64_t g, int sms, bool persistent, const void* vtx, int64_t nVtx, WsPtrs ws, int64_t tilesV,
                     int mode, const SegArgs& seg, cudaStream_t st) {
  if (mode == kHistNone)
    launch_v<S, kHistNone, kSeg>(g, sms, persistent, vtx, nVtx, ws, tilesV, seg, st);
  else if (mode == kHistMasks || S >= kWideMin)  // 24- and 32-byte keys: "tiles" sort only
    launch_v<S, kHistMasks, kSeg>(g, sms, persistent, vtx, nVtx, ws, tilesV, seg, st);
  else if constexpr (S >= kWideMin)
    return;
  else if (kSeg || mode == kHistUniform)
    launch_v<S, kHistUniform, kSeg>(g, sms, persistent, vtx, nVtx, ws, tilesV, seg, st);
  else if (mode == kHistMatchAny)
    launch_v<S, kHistMatchAny, kSeg>(g, sms, persistent, vtx, nVtx, ws, tilesV, seg, st);
  else
    launch_v<S, kHistPeel, kSeg>(g, sms, persistent, vtx, nVtx, ws, tilesV, seg, st);
}

cudaError_t launch_compact(int S, const void* vtx, int64_t nVtx, WsPtrs ws, int64_t tilesV, const LaunchCfg& c,
                           const SegArgs* seg, cudaStream_t st) {
  if (tilesV == 0) return cudaSuccess;
  const int64_t g = tilesV;  // capped at SMs x the variant's occupancy unless one CTA per tile
  const bool persistent = !c.grid_per_tile;
  const SegArgs none{};
  // the "tiles" sort counts digits per pass and needs no upfront histograms
  const int mode = uses_plane(c.sort_kernel) ? (c.pack_keys ? kHistNone : kHistMasks) : c.hist_mode;
  if (seg) {
    switch (S) {
      case 4: launch_s<4, true>(g, c.sms, persistent, vtx, nVtx, ws, tilesV, mode, *seg, st); break;
      case 8: launch_s<8, true>(g, c.sms, persistent, vtx, nVtx, ws, tilesV, mode, *seg, st); break;
      case 12: launch_s<12, true>(g, c.sms, persistent, vtx, nVtx, ws, tilesV, mode, *seg, st); break;
      default: launch_s<16, true>(g, c.sms, persistent, vtx, nVtx, ws, tilesV, mode, *seg, st); break;
    }
  } else {
    switch (S) {
      case 4: launch_s<4, false>(g, c.sms, persistent, vtx, nVtx, ws, tilesV, mode, none, st); break;
      case 8: launch_s<8, false>(g, c.sms, persistent, vtx, nVtx, ws, tilesV, mode, none, st); break;
      case 12: launch_s<12, false>(g, c.sms, persistent, vtx, nVtx, ws, tilesV, mode, none, st); break;
      case 16: launch_s<16, false>(g, c.sms, persistent, vtx, nVtx, ws, tilesV, mode, none, st); break;
      case 20: launch_s<20, false>(g, c.sms, persistent, vtx, nVtx, ws, tilesV, mode, none, st); break;
      case 24: launch_s<24, false>(g, c.sms, persistent, vtx, nVtx, ws, tilesV, mode, none, st); break;
      case 32: launch_s<32, false>(g, c.sms, persistent, vtx, nVtx, ws, tilesV, mode, none, st); break;
      case 48: launch_v<48, kHistMasks, false>(g, c.sms, persistent, vtx, nVtx, ws, tilesV, none, st); break;
      case 64: launch_v<64, kHistMasks, false>(g, c.sms, persistent, vtx, nVtx, ws, tilesV, none, st); break;
      default: return cudaErrorInvalidValue;
    }
  }
  return cudaGetLastError();
}

cudaError_t launch_compact_prefix(int S, const void* vtx, int64_t nVtx, WsPtrs ws, int64_t tilesV, const LaunchCfg& c,
                                  cudaStream_t st) {
  if (tilesV == 0) return cudaSuccess;
  const bool persistent = !c.grid_per_tile;
  const SegArgs none{};
  switch (S) {
    case 12: launch_v<12, kHistPrefix, false>(tilesV, c.sms, persistent, vtx, nVtx, ws, tilesV, none, st); break;
    case 16: launch_v<16, kHistPrefix, false>(tilesV, c.sms, persistent, vtx, nVtx, ws, tilesV, none, st); break;
    case 20: launch_v<20, kHistPrefix, false>(tilesV, c.sms, persistent, vtx, nVtx, ws, tilesV, none, st); break;
    case 24: launch_v<24, kHistPrefix, false>(tilesV, c.sms, persistent, vtx, nVtx, ws, tilesV, none, st); break;
    case 32: launch_v<32, kHistPrefix, false>(tilesV, c.sms, persistent, vtx, nVtx, ws, tilesV, none, st); break;
    case 48: launch_v<48, kHistPrefix, false>(tilesV, c.sms, persistent, vtx, nVtx, ws, tilesV, none, st); break;
    case 64: launch_v<64, kHistPrefix, false>(tilesV, c.sms, persistent, vtx, nVtx, ws, tilesV, none, st); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_prefix_check(int S, const void* vtx, int64_t nVtx, const void* out_vtx, WsPtrs ws,
                                const LaunchCfg& c, cudaStream_t st) {
  if (nVtx == 0) return cudaSuccess;
  int64_t g = (nVtx / 4 + kThreads - 1) / kThreads;
  if (g > (int64_t)c.sms * 8) g = (int64_t)c.sms * 8;
  if (g < 1) g = 1;
  const bool vec = (reinterpret_cast<uintptr_t>(vtx) & 15) == 0;
#define REINDEX_PC(SS)                                                                           \
  (vec ? k_prefix_check<SS, true><<<(int)g, kThreads, 0, st>>>(vtx, nVtx, out_vtx, ws)          \
       : k_prefix_check<SS, false><<<(int)g, kThreads, 0, st>>>(vtx, nVtx, out_vtx, ws))
  switch (S) {
    case 12: REINDEX_PC(12); break;
    case 16: REINDEX_PC(16); break;
    case 20: REINDEX_PC(20); break;
    case 24: REINDEX_PC(24); break;
    case 32: REINDEX_PC(32); break;
    case 48: REINDEX_PC(48); break;
    case 64: REINDEX_PC(64); break;
    default: return cudaErrorInvalidValue;
  }
#undef REINDEX_PC
  return cudaGetLastError();
}

cudaError_t launch_key_masks(int S, const void* vtx, int64_t nVtx, WsPtrs ws, const LaunchCfg& c,
                             const SegArgs* seg, cudaStream_t st) {
  if (nVtx == 0) return cudaSuccess;
  int64_t g = (nVtx + kThreads - 1) / kThreads;
  if (g > (int64_t)c.sms * 8) g = (int64_t)c.sms * 8;
  const bool vec = (reinterpret_cast<uintptr_t>(vtx) & 15) == 0;
  const SegArgs none{};
  const SegArgs& sg = seg ? *seg : none;
#define REINDEX_KM(SS, SEG)                                                                 \
  (vec ? k_key_masks<SS, SEG, true><<<(int)g, kThreads, 0, st>>>(vtx, nVtx, ws, sg)       \
       : k_key_masks<SS, SEG, false><<<(int)g, kThreads, 0, st>>>(vtx, nVtx, ws, sg))
  if (seg) {
    switch (S) {
      case 4: REINDEX_KM(4, true); break;
      case 8: REINDEX_KM(8, true); break;
      case 12: REINDEX_KM(12, true); break;
      default: REINDEX_KM(16, true); break;
    }
  } else {
    switch (S) {
      case 4: REINDEX_KM(4, false); break;
      case 8: REINDEX_KM(8, false); break;
      case 12: REINDEX_KM(12, false); break;
      case 16: REINDEX_KM(16, false); break;
      case 20: REINDEX_KM(20, false); break;
      case 24: REINDEX_KM(24, false); break;
      case 32: REINDEX_KM(32, false); break;
      case 48: REINDEX_KM(48, false); break;
      case 64: REINDEX_KM(64, false); break;
      default: return cudaErrorInvalidValue;
    }
  }
#undef REINDEX_KM
  return cudaGetLastError();
}

}  // namespace reindex
