// Duplicate removal before the sort (the "hash" variant of steps 2-4; beyond the paper, same
// result).  The paper sorts every used vertex and finds duplicates as equal neighbours; when most
// used vertices are copies (a triangle soup repeats each lattice point about six times, a tet soup
// about twenty), it is cheaper to find the copies first and sort one representative per distinct
// key:
//   k_hash_dedup  every used vertex inserts its key into an open-addressing table (linear probing;
//                 a slot is claimed by compare-and-swap for the first vertex that reaches it empty).
//                 A vertex that claims an empty slot is its key's representative and appends its
//                 (key, index) item for the sort, with the item's first-pass digit and the key bit
//                 masks (as the compaction does) -- or, when the prefix path sorts the
//                 representatives, marks itself in the used bits instead; any other vertex finds
//                 the slot whose owner's key equals its own (raw bits) and records that
//                 representative in oldToNew, tagged;
//   (sort, run heads, scan, oldToNew scatter, gather: unchanged, on the D distinct keys -- every
//    item is a run head, and oldToNew[rep] = its new index)
//   k_remap_rep   out = oldToNew[idx], a tagged entry through its representative's (single meshes;
//                 batched calls: k_seg_remap does the same);
//   k_resolve     every tagged oldToNew entry takes its representative's new index (callers that
//                 read oldToNew itself).
// Keys compare by raw bits, so the set of representatives' keys is exactly the set of distinct
// used keys, and the sorted result (unique vertices in ascending key order, each index's rank) is
// the paper's, bit for bit, whichever copy became a representative.  The table lives in the sort's
// second item buffer, idle until the first radix pass.
#include "internal.h"

namespace reindex {

// Table slot values: 0 (empty); owner index + 1 (claimed by a representative whose item is not
// published: below 2^31); kPosFlag | item position (published, in the publishing variant).
constexpr uint32_t kPosFlag = 0x80000000u;

template <int K>
__device__ __forceinline__ uint32_t key_hash(const uint32_t (&k)[K]) {
  uint64_t h = 0x9E3779B97F4A7C15ull;
#pragma unroll
  for (int q = 0; q < K; ++q) {
    h = (h ^ k[q]) * 0xBF58476D1CE4E5B9ull;
    h ^= h >> 29;
  }
  h *= 0x94D049BB133111EBull;
  return (uint32_t)(h >> 32);
}

// L2 policy for the random accesses (table slots, the keys compared against): keep them in L2 in
// preference to the streamed lines (the vertex array, read once, and the oldToNew stores, which go
// evict-first).
__device__ __forceinline__ uint64_t l2_keep_policy() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint32_t ld_slot(const uint32_t* a, uint64_t pol) {  // through L2 only
  uint32_t v;
  asm("ld.global.cg.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(a), "l"(pol));
  return v;
}
// Slot read of the publishing variant: kept before the acquire fence that follows it.
__device__ __forceinline__ uint32_t ld_slot_ordered(const uint32_t* a, uint64_t pol) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(a), "l"(pol) : "memory");
  return v;
}
__device__ __forceinline__ void fence_acq_rel() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

// An owner's key from the vertex array (read-only input: no ordering needed).
template <int S>
__device__ __forceinline__ void load_key_keep(const void* vtx, uint32_t i, uint32_t (&k)[S / 4], uint64_t pol) {
  if constexpr (S % 16 == 0) {
    const uint4* p = reinterpret_cast<const uint4*>(vtx) + (size_t)i * (S / 16);
#pragma unroll
    for (int h = 0; h < S / 16; ++h)
      asm("ld.global.nc.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
          : "=r"(k[4 * h]), "=r"(k[4 * h + 1]), "=r"(k[4 * h + 2]), "=r"(k[4 * h + 3])
          : "l"(p + h), "l"(pol));
  } else if constexpr (S % 8 == 0) {
    const uint2* p = reinterpret_cast<const uint2*>(vtx) + (size_t)i * (S / 8);
#pragma unroll
    for (int h = 0; h < S / 8; ++h)
      asm("ld.global.nc.L2::cache_hint.v2.u32 {%0,%1}, [%2], %3;"
          : "=r"(k[2 * h]), "=r"(k[2 * h + 1])
          : "l"(p + h), "l"(pol));
  } else {
    const uint32_t* p = reinterpret_cast<const uint32_t*>(vtx) + (size_t)i * (S / 4);
#pragma unroll
    for (int q = 0; q < S / 4; ++q)
      asm("ld.global.nc.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(k[q]) : "l"(p + q), "l"(pol));
  }
}

// The key and vertex index of the item at `pos` of the first item buffer (written in this launch
// by another warp; read after the acquire fence, in program order).
template <int S>
__device__ __forceinline__ void load_item_key(const WsPtrs& ws, uint32_t pos, uint32_t (&k)[S / 4], uint32_t& id,
                                              uint64_t pol) {
  constexpr int K = S / 4;
  if constexpr (soa_items(S)) {
    const unsigned char* kp = ws.itemsA + (size_t)pos * S;
    if constexpr (S % 16 == 0) {
#pragma unroll
      for (int h = 0; h < S / 16; ++h)
        asm volatile("ld.global.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
                     : "=r"(k[4 * h]), "=r"(k[4 * h + 1]), "=r"(k[4 * h + 2]), "=r"(k[4 * h + 3])
                     : "l"(kp + 16 * h), "l"(pol)
                     : "memory");
    } else {
#pragma unroll
      for (int h = 0; h < S / 8; ++h)
        asm volatile("ld.global.L2::cache_hint.v2.u32 {%0,%1}, [%2], %3;"
                     : "=r"(k[2 * h]), "=r"(k[2 * h + 1])
                     : "l"(kp + 8 * h), "l"(pol)
                     : "memory");
    }
    asm volatile("ld.global.L2::cache_hint.u32 %0, [%1], %2;"
                 : "=r"(id)
                 : "l"(ws.itemsA + ws.idoff + (size_t)pos * 4), "l"(pol)
                 : "memory");
  } else if constexpr (S == 12) {  // {k0, k1, k2, id}: one 16-byte vector
    asm volatile("ld.global.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
                 : "=r"(k[0]), "=r"(k[1]), "=r"(k[2]), "=r"(id)
                 : "l"(ws.itemsA + (size_t)pos * 16), "l"(pol)
                 : "memory");
  } else {  // 4 and 20 bytes: {k..., id} in 8-byte vectors
    uint32_t w[K + 1];
#pragma unroll
    for (int h = 0; h < (K + 1) / 2; ++h)
      asm volatile("ld.global.L2::cache_hint.v2.u32 {%0,%1}, [%2], %3;"
                   : "=r"(w[2 * h]), "=r"(w[2 * h + 1])
                   : "l"(ws.itemsA + (size_t)pos * (S + 4) + 8 * h), "l"(pol)
                   : "memory");
#pragma unroll
    for (int q = 0; q < K; ++q) k[q] = w[q];
    id = w[K];
  }
}

// CTAs per SM the register budget is set for (the grid is one wave of them); SI = key bytes
__host__ __device__ constexpr int dedup_ctas_per_sm(int SI, bool pub, bool seg) {
  return SI <= 24 && !((pub || seg) && SI == 12) ? 4 : 3;
}

// Each warp keeps R rows of 32 vertices in flight (R = 4 for keys of up to 12 bytes, 2 up to 32,
// else 1): their keys load together, their first table slots load together, and the keys they
// compare against load together, so that a warp waits on R independent chains of random accesses
// at a time instead of one.  A slot changes from 0 only by compare-and-swap, so a stale 0 merely
// sends the vertex to the compare-and-swap, which returns the slot's value.  One counter add per
// warp and batch hands out the representatives' item positions.
//
// kPub: a representative publishes its item position in its slot (one batch later, after the
// acquire-release fence that every batch with a published slot or a pending publication takes), so
// that most copies compare against the dense item array rather than the owner's key scattered over
// the vertex array.  A copy that finds a claim not yet published compares against the owner's key
// in the vertex array.  Message passing: item stores, fence, slot store (relaxed) by the
// representative; slot load (relaxed) or compare-and-swap, fence, item loads by the copy.
//
// kSeg (batched calls): the key is (mesh id, vertex), the mesh id its most significant word, as in
// the batched compaction; a copy compares the owner's mesh id too (looked up from its index).
// kRepMask (single meshes of 12-byte vertices and wider whose sort runs on key prefixes):
// representatives append nothing; each row's used-bit word is replaced by the bits of its
// representatives (the warp that reads a row's word is the only one that touches it), so that the
// prefix path's compaction, sort, check and fallback take the representatives as the used
// vertices; copies still record theirs.
// A launch inserts the used vertices of rows [row_lo, row_hi) (32 vertices a row): a call may insert
// the vertex array chunk by chunk, as the chunks arrive, in any order -- the result does not depend
// on which copy of a key claims its slot first.
template <int S, bool kPub, bool kSeg, bool kRepMask = false>
__global__ void __launch_bounds__(kThreads, dedup_ctas_per_sm(S + (kSeg ? 4 : 0), kPub, kSeg))
    k_hash_dedup(const void* __restrict__ vtx, int64_t nVtx, WsPtrs ws, uint32_t* __restrict__ table, uint32_t mask,
                 uint32_t cap, SegArgs seg, int64_t row_lo, int64_t row_hi) {
  constexpr int KV = S / 4;             // vertex words
  constexpr int K = KV + (kSeg ? 1 : 0);  // key words
  constexpr int SI = 4 * K;             // key bytes of an item
  constexpr int R = K <= 3 ? 4 : (K <= 8 ? 2 : 1);
  Control* ctrl = ws.ctrl;
  if (block_error(ctrl)) return;
  const int lane = threadIdx.x & 31;
  const int64_t rows = row_hi;
  const int64_t warp0 = (blockIdx.x * (int64_t)kThreads + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * kThreads) >> 5;
  uint32_t kor[K], knand[K];
#pragma unroll
  for (int q = 0; q < K; ++q) kor[q] = knand[q] = 0;
  bool bad = false;  // a consistency check failed
  const uint64_t keep = l2_keep_policy();
  bool pend[R];  // kPub: this lane's representatives of the previous batch, not yet published
  uint32_t pend_h[R], pend_pos[R];
#pragma unroll
  for (int r = 0; r < R; ++r) pend[r] = false;
  for (int64_t row0 = row_lo + warp0 * R; row0 < rows; row0 += nwarps * R) {
    uint32_t k[R][K], h[R];
    bool act[R], rep[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {  // keys load whether used or not: no wait on the bitmask first
      const int64_t i = (row0 + r) * 32 + lane;
      const uint32_t used = row0 + r < rows ? __ldg(ws.bitmask + row0 + r) : 0u;
      act[r] = (used >> lane) & 1u;
      rep[r] = false;
      if (i < nVtx) {
        uint32_t kv[KV];
        load_key<S>(vtx, i, kv);
#pragma unroll
        for (int q = 0; q < KV; ++q) k[r][K - KV + q] = kv[q];
        if constexpr (kSeg) k[r][0] = seg_mesh(i, seg.vtxOff, 1, seg.blkV, seg.nMeshes);
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) h[r] = act[r] ? key_hash<K>(k[r]) & mask : 0u;
    for (uint32_t probes = 0;; ++probes) {
      bool any = false;
#pragma unroll
      for (int r = 0; r < R; ++r) any |= act[r];
      if (!any) break;
      if (probes > mask) {  // the table is full: cannot happen (it has 1.25 slots per used vertex)
        bad = true;
        break;
      }
      uint32_t o[R];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if constexpr (kPub)
          o[r] = act[r] ? ld_slot_ordered(table + h[r], keep) : 1u;
        else
          o[r] = act[r] ? ld_slot(table + h[r], keep) : 1u;
      }
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (act[r] && o[r] == 0) {
          o[r] = atomicCAS(table + h[r], 0u, (uint32_t)((row0 + r) * 32 + lane) + 1u);
          if (o[r] == 0) {
            rep[r] = true;
            act[r] = false;
          }
        }
      uint32_t ok[R][K], oid[R];
      if constexpr (kPub) {
        bool fence = false;
#pragma unroll
        for (int r = 0; r < R; ++r) fence |= (act[r] && (o[r] & kPosFlag)) || pend[r];
        if (fence) {
          fence_acq_rel();
#pragma unroll
          for (int r = 0; r < R; ++r)
            if (pend[r]) {
              st_relaxed(table + pend_h[r], kPosFlag | pend_pos[r]);
              pend[r] = false;
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r)
          if (act[r] && (o[r] & kPosFlag)) {
            if ((o[r] & ~kPosFlag) >= cap) {  // not an item position: a bug
              bad = true;
              act[r] = false;
            } else {
              load_item_key<SI>(ws, o[r] & ~kPosFlag, ok[r], oid[r], keep);
              if ((int64_t)oid[r] >= nVtx) {
                bad = true;
                act[r] = false;
              }
            }
          }
      }
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (act[r] && !(kPub && (o[r] & kPosFlag))) {
          if ((int64_t)(o[r] - 1u) >= nVtx) {  // not an owner index (a table left uncleared): a bug
            bad = true;
            act[r] = false;
          } else {
            uint32_t kv[KV];
            load_key_keep<S>(vtx, o[r] - 1u, kv, keep);
#pragma unroll
            for (int q = 0; q < KV; ++q) ok[r][K - KV + q] = kv[q];
            if constexpr (kSeg) ok[r][0] = seg_mesh(o[r] - 1u, seg.vtxOff, 1, seg.blkV, seg.nMeshes);
            oid[r] = o[r] - 1u;
          }
        }
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (act[r]) {
          bool same = true;
#pragma unroll
          for (int q = 0; q < K; ++q) same &= ok[r][q] == k[r][q];
          if (same) {
            __stcs(ws.old2new + (row0 + r) * 32 + lane, kRepTag | oid[r]);
            act[r] = false;
          } else {
            h[r] = (h[r] + 1u) & mask;
          }
        }
    }
    // representatives append their items (one counter add per warp and batch)
    uint32_t b[R], tot = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      b[r] = __ballot_sync(0xffffffffu, rep[r]);
      tot += __popc(b[r]);
    }
    if constexpr (kRepMask) {  // the rows' used bits become their representatives' bits
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (lane == 0 && row0 + r < rows) ws.bitmask[row0 + r] = b[r];
        if (rep[r]) {
#pragma unroll
          for (int q = 0; q < K; ++q) {
            kor[q] |= k[r][q];
            knand[q] |= ~k[r][q];
          }
        }
      }
      continue;
    }
    if (tot == 0) continue;  // warp-uniform
    uint32_t base = 0;
    if (lane == 0) base = atomicAdd(&ctrl->U, tot);
    base = __shfl_sync(0xffffffffu, base, 0);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (rep[r]) {
        const uint32_t pos = base + __popc(b[r] & lanemask_lt());
        Item<SI> it;
#pragma unroll
        for (int q = 0; q < K; ++q) it.k[q] = k[r][q];
        it.id = (uint32_t)((row0 + r) * 32 + lane);
        ItemIO<SI>::store(ws.itemsA, ws.idoff, pos, it);
        ws.digits[pos] = (uint8_t)(k[r][K - 1] & 0xFFu);  // the first pass's digit: key byte 0
#pragma unroll
        for (int q = 0; q < K; ++q) {  // key bit masks: over the representatives, i.e. every distinct key
          kor[q] |= k[r][q];
          knand[q] |= ~k[r][q];
        }
        if constexpr (kPub) {  // (a representative of the previous batch in this row is published by now)
          pend[r] = true;
          pend_h[r] = h[r];
          pend_pos[r] = pos;
        }
      }
      base += __popc(b[r]);
    }
  }
  if (bad) record_error(ctrl, kErrInternal);
#pragma unroll
  for (int q = 0; q < K; ++q) {
    const uint32_t a = __reduce_or_sync(0xffffffffu, kor[q]), c = __reduce_or_sync(0xffffffffu, knand[q]);
    if (lane == 0) {
      if (a) atomicOr(&ctrl->kor[q], a);
      if (c) atomicOr(&ctrl->knand[q], c);
    }
  }
}

// Copies take their representative's new index (written by the head scan).
__global__ void __launch_bounds__(kThreads) k_resolve(int64_t nVtx, WsPtrs ws) {
  const uint32_t err = ws.ctrl->err;
  if (err && err != kErrSkip) return;
  const int lane = threadIdx.x & 31;
  const int64_t rows = (nVtx + 31) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * kThreads) >> 5;
  for (int64_t row = (blockIdx.x * (int64_t)kThreads + threadIdx.x) >> 5; row < rows; row += nwarps) {
    const uint32_t used = __ldg(ws.bitmask + row);
    if (!((used >> lane) & 1u)) continue;
    const int64_t i = row * 32 + lane;
    const uint32_t v = ws.old2new[i];
    if (!(v & kRepTag)) continue;
    if ((int64_t)(v & ~kRepTag) >= nVtx) {  // not a vertex index: a bug; record it, skip the load
      record_error(ws.ctrl, kErrInternal);
      continue;
    }
    ws.old2new[i] = __ldcg(ws.old2new + (v & ~kRepTag));
  }
}

// Slots of the table: the smallest power of two of at least 1.25 slots per possible used vertex
// (so that the table is at most 80 % full, whatever the duplicates), and at least 64 (the table is
// cleared in whole 16-byte vectors), within the second item buffer (always 256 bytes or more).
uint32_t dedup_table_slots(const WsLayout& L) {
  const uint64_t need = (uint64_t)L.Umax + (uint64_t)L.Umax / 4 + 1;
  const uint64_t room = (uint64_t)L.items_bytes / 4;
  uint64_t p = 64;
  while (p < need && p * 2 <= room && p < (1ull << 31)) p *= 2;
  return (uint32_t)p;
}

static int grid_rows(int64_t nVtx, const LaunchCfg& c) {
  int64_t g = ((nVtx + 31) / 32 * 32 + kThreads - 1) / kThreads;
  const int64_t cap = (int64_t)c.sms * 8;
  if (g > cap) g = cap;
  return g < 1 ? 1 : (int)g;
}

static cudaError_t hash_repmask_s(int S, int g, const void* vtx, int64_t nVtx, WsPtrs ws, uint32_t* table,
                                  uint32_t mask, uint32_t cap, int64_t rlo, int64_t rhi, cudaStream_t st) {
  const SegArgs none{};
  switch (S) {
    case 12: k_hash_dedup<12, false, false, true><<<g, kThreads, 0, st>>>(vtx, nVtx, ws, table, mask, cap, none, rlo, rhi); break;
    case 16: k_hash_dedup<16, false, false, true><<<g, kThreads, 0, st>>>(vtx, nVtx, ws, table, mask, cap, none, rlo, rhi); break;
    case 20: k_hash_dedup<20, false, false, true><<<g, kThreads, 0, st>>>(vtx, nVtx, ws, table, mask, cap, none, rlo, rhi); break;
    case 24: k_hash_dedup<24, false, false, true><<<g, kThreads, 0, st>>>(vtx, nVtx, ws, table, mask, cap, none, rlo, rhi); break;
    case 32: k_hash_dedup<32, false, false, true><<<g, kThreads, 0, st>>>(vtx, nVtx, ws, table, mask, cap, none, rlo, rhi); break;
    case 48: k_hash_dedup<48, false, false, true><<<g, kThreads, 0, st>>>(vtx, nVtx, ws, table, mask, cap, none, rlo, rhi); break;
    case 64: k_hash_dedup<64, false, false, true><<<g, kThreads, 0, st>>>(vtx, nVtx, ws, table, mask, cap, none, rlo, rhi); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <bool kPub>
static cudaError_t hash_dedup_s(int S, int g, const void* vtx, int64_t nVtx, WsPtrs ws, uint32_t* table,
                                uint32_t mask, uint32_t cap, const SegArgs* seg, int64_t rlo, int64_t rhi,
                                cudaStream_t st) {
  if (seg) {  // batched: S is the vertex stride (4 to 16 bytes), keys are S + 4 bytes
    switch (S) {
      case 4: k_hash_dedup<4, kPub, true><<<g, kThreads, 0, st>>>(vtx, nVtx, ws, table, mask, cap, *seg, rlo, rhi); break;
      case 8: k_hash_dedup<8, kPub, true><<<g, kThreads, 0, st>>>(vtx, nVtx, ws, table, mask, cap, *seg, rlo, rhi); break;
      case 12: k_hash_dedup<12, kPub, true><<<g, kThreads, 0, st>>>(vtx, nVtx, ws, table, mask, cap, *seg, rlo, rhi); break;
      case 16: k_hash_dedup<16, kPub, true><<<g, kThreads, 0, st>>>(vtx, nVtx, ws, table, mask, cap, *seg, rlo, rhi); break;
      default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
  }
  const SegArgs none{};
  switch (S) {
    case 8: k_hash_dedup<8, kPub, false><<<g, kThreads, 0, st>>>(vtx, nVtx, ws, table, mask, cap, none, rlo, rhi); break;
    case 12: k_hash_dedup<12, kPub, false><<<g, kThreads, 0, st>>>(vtx, nVtx, ws, table, mask, cap, none, rlo, rhi); break;
    case 16: k_hash_dedup<16, kPub, false><<<g, kThreads, 0, st>>>(vtx, nVtx, ws, table, mask, cap, none, rlo, rhi); break;
    case 20: k_hash_dedup<20, kPub, false><<<g, kThreads, 0, st>>>(vtx, nVtx, ws, table, mask, cap, none, rlo, rhi); break;
    case 24: k_hash_dedup<24, kPub, false><<<g, kThreads, 0, st>>>(vtx, nVtx, ws, table, mask, cap, none, rlo, rhi); break;
    case 32: k_hash_dedup<32, kPub, false><<<g, kThreads, 0, st>>>(vtx, nVtx, ws, table, mask, cap, none, rlo, rhi); break;
    case 48: k_hash_dedup<48, kPub, false><<<g, kThreads, 0, st>>>(vtx, nVtx, ws, table, mask, cap, none, rlo, rhi); break;
    case 64: k_hash_dedup<64, kPub, false><<<g, kThreads, 0, st>>>(vtx, nVtx, ws, table, mask, cap, none, rlo, rhi); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_hash_dedup(int S, const void* vtx, int64_t nVtx, WsPtrs ws, uint32_t slots, uint32_t cap,
                              const LaunchCfg& c, cudaStream_t st, const SegArgs* seg, int64_t vlo, int64_t vhi,
                              bool repmask) {
  if (vhi < 0 || vhi > nVtx) vhi = nVtx;
  if (vlo < 0) vlo = 0;
  if (vlo % 32 != 0) return cudaErrorInvalidValue;  // whole rows
  if (vhi <= vlo) return cudaSuccess;
  const int64_t rlo = vlo / 32, rhi = (vhi + 31) / 32;
  uint32_t* table = reinterpret_cast<uint32_t*>(ws.itemsB);
  const uint32_t mask = slots - 1u;
  // one wave: as many CTAs as the register cap of the kernel lets every SM hold
  int g = grid_rows(vhi - vlo, c);
  const bool pub = c.dedup_pub != 0 && !repmask;  // (no items to publish with repmask)
  const int wave = c.sms * dedup_ctas_per_sm(S + (seg ? 4 : 0), pub, seg != nullptr);
  if (g > wave) g = wave;
  if (repmask) return seg ? cudaErrorInvalidValue : hash_repmask_s(S, g, vtx, nVtx, ws, table, mask, cap, rlo, rhi, st);
  return c.dedup_pub ? hash_dedup_s<true>(S, g, vtx, nVtx, ws, table, mask, cap, seg, rlo, rhi, st)
                     : hash_dedup_s<false>(S, g, vtx, nVtx, ws, table, mask, cap, seg, rlo, rhi, st);
}

// out[j] = oldToNew[idx[j]], through the representative for a copy (tagged entry): the remap of a
// call whose representatives were sorted by the prefix path (no resolve pass).  After a full-key
// fallback every used vertex holds its new index and the second look-up never happens.
template <typename I>
__global__ void __launch_bounds__(kThreads) k_remap_rep(const I* idx, I* out, int64_t M, const uint32_t* o2n,
                                                        const Control* ctrl) {
  const uint32_t err = ctrl->err;
  if (err && err != kErrSkip) return;
  constexpr int kB = 4;
  const int64_t stride = (int64_t)gridDim.x * kThreads;
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < M; i += stride * kB) {
    I q[kB];
    uint32_t v[kB];
#pragma unroll
    for (int b = 0; b < kB; ++b)
      if (i + b * stride < M) q[b] = __ldcs(idx + i + b * stride);
#pragma unroll
    for (int b = 0; b < kB; ++b)
      if (i + b * stride < M) v[b] = __ldg(o2n + q[b]);
#pragma unroll
    for (int b = 0; b < kB; ++b)
      if (i + b * stride < M && (v[b] & kRepTag)) v[b] = __ldg(o2n + (v[b] & ~kRepTag));
#pragma unroll
    for (int b = 0; b < kB; ++b)
      if (i + b * stride < M) __stcs(out + i + b * stride, (I)v[b]);
  }
}

cudaError_t launch_remap_rep(const void* idx, void* out, bool wide, int64_t M, WsPtrs ws, const LaunchCfg& c,
                             cudaStream_t st) {
  if (M == 0) return cudaSuccess;
  int64_t g = (M + kThreads - 1) / kThreads;
  if (g > (int64_t)c.sms * 8) g = (int64_t)c.sms * 8;
  if (wide)
    k_remap_rep<int64_t><<<(int)g, kThreads, 0, st>>>(static_cast<const int64_t*>(idx), static_cast<int64_t*>(out),
                                                      M, ws.old2new, ws.ctrl);
  else
    k_remap_rep<int32_t><<<(int)g, kThreads, 0, st>>>(static_cast<const int32_t*>(idx), static_cast<int32_t*>(out),
                                                      M, ws.old2new, ws.ctrl);
  return cudaGetLastError();
}

cudaError_t launch_resolve(int64_t nVtx, WsPtrs ws, const LaunchCfg& c, cudaStream_t st) {
  if (nVtx == 0) return cudaSuccess;
  k_resolve<<<grid_rows(nVtx, c), kThreads, 0, st>>>(nVtx, ws);
  return cudaGetLastError();
}

}  // namespace reindex
