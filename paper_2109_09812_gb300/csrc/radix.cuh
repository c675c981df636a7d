// Pieces shared by the radix-pass kernels (k_onesweep.cu, k_radix_tiles.cu): shared-memory
// staging of a tile in digit order, the per-CTA shared-memory budget and the warp-level digit
// matching used to rank items stably.
#pragma once

#include "internal.h"

namespace reindex {

// Shared-memory staging of one tile: a vector per item (the key words, plus the old index for
// the array-of-structures layouts) and, for S = 8, 16, 24 and 32, a separate old-index plane.
template <int S>
struct Stage;

template <>
struct Stage<4> {
  static constexpr size_t bytes = (size_t)kSortTile * 8;
  static __device__ __forceinline__ void put(unsigned char* sm, int p, const Item<4>& it) {
    reinterpret_cast<uint2*>(sm)[p] = make_uint2(it.k[0], it.id);
  }
  static __device__ __forceinline__ void get(const unsigned char* sm, int p, Item<4>& it) {
    const uint2 v = reinterpret_cast<const uint2*>(sm)[p];
    it.k[0] = v.x; it.id = v.y;
  }
};
template <>
struct Stage<12> {
  static constexpr size_t bytes = (size_t)kSortTile * 16;
  static __device__ __forceinline__ void put(unsigned char* sm, int p, const Item<12>& it) {
    reinterpret_cast<uint4*>(sm)[p] = make_uint4(it.k[0], it.k[1], it.k[2], it.id);
  }
  static __device__ __forceinline__ void get(const unsigned char* sm, int p, Item<12>& it) {
    const uint4 v = reinterpret_cast<const uint4*>(sm)[p];
    it.k[0] = v.x; it.k[1] = v.y; it.k[2] = v.z; it.id = v.w;
  }
};
template <>
struct Stage<8> {
  static constexpr size_t bytes = (size_t)kSortTile * 12;
  static __device__ __forceinline__ void put(unsigned char* sm, int p, const Item<8>& it) {
    reinterpret_cast<uint2*>(sm)[p] = make_uint2(it.k[0], it.k[1]);
    reinterpret_cast<uint32_t*>(sm + (size_t)kSortTile * 8)[p] = it.id;
  }
  static __device__ __forceinline__ void get(const unsigned char* sm, int p, Item<8>& it) {
    const uint2 v = reinterpret_cast<const uint2*>(sm)[p];
    it.k[0] = v.x; it.k[1] = v.y;
    it.id = reinterpret_cast<const uint32_t*>(sm + (size_t)kSortTile * 8)[p];
  }
};
template <>
struct Stage<16> {
  static constexpr size_t bytes = (size_t)kSortTile * 20;
  static __device__ __forceinline__ void put(unsigned char* sm, int p, const Item<16>& it) {
    reinterpret_cast<uint4*>(sm)[p] = make_uint4(it.k[0], it.k[1], it.k[2], it.k[3]);
    reinterpret_cast<uint32_t*>(sm + (size_t)kSortTile * 16)[p] = it.id;
  }
  static __device__ __forceinline__ void get(const unsigned char* sm, int p, Item<16>& it) {
    const uint4 v = reinterpret_cast<const uint4*>(sm)[p];
    it.k[0] = v.x; it.k[1] = v.y; it.k[2] = v.z; it.k[3] = v.w;
    it.id = reinterpret_cast<const uint32_t*>(sm + (size_t)kSortTile * 16)[p];
  }
};

template <>
struct Stage<20> {
  static constexpr size_t bytes = (size_t)kSortTile * 24;
  static __device__ __forceinline__ void put(unsigned char* sm, int p, const Item<20>& it) {
    uint2* q = reinterpret_cast<uint2*>(sm) + 3 * p;
    q[0] = make_uint2(it.k[0], it.k[1]);
    q[1] = make_uint2(it.k[2], it.k[3]);
    q[2] = make_uint2(it.k[4], it.id);
  }
  static __device__ __forceinline__ void get(const unsigned char* sm, int p, Item<20>& it) {
    const uint2* q = reinterpret_cast<const uint2*>(sm) + 3 * p;
    const uint2 a = q[0], b = q[1], c = q[2];
    it.k[0] = a.x; it.k[1] = a.y; it.k[2] = b.x; it.k[3] = b.y; it.k[4] = c.x; it.id = c.y;
  }
};

// 24- and 32-byte keys: key vectors, then the old-index plane.
template <>
struct Stage<24> {
  static constexpr size_t bytes = (size_t)kSortTile * 28;
  static __device__ __forceinline__ void put(unsigned char* sm, int p, const Item<24>& it) {
    uint2* q = reinterpret_cast<uint2*>(sm) + 3 * p;
    q[0] = make_uint2(it.k[0], it.k[1]);
    q[1] = make_uint2(it.k[2], it.k[3]);
    q[2] = make_uint2(it.k[4], it.k[5]);
    reinterpret_cast<uint32_t*>(sm + (size_t)kSortTile * 24)[p] = it.id;
  }
  static __device__ __forceinline__ void get(const unsigned char* sm, int p, Item<24>& it) {
    const uint2* q = reinterpret_cast<const uint2*>(sm) + 3 * p;
    const uint2 a = q[0], b = q[1], c = q[2];
    it.k[0] = a.x; it.k[1] = a.y; it.k[2] = b.x; it.k[3] = b.y; it.k[4] = c.x; it.k[5] = c.y;
    it.id = reinterpret_cast<const uint32_t*>(sm + (size_t)kSortTile * 24)[p];
  }
};
template <>
struct Stage<32> {
  static constexpr size_t bytes = (size_t)kSortTile * 36;
  static __device__ __forceinline__ void put(unsigned char* sm, int p, const Item<32>& it) {
    uint4* q = reinterpret_cast<uint4*>(sm) + 2 * p;
    q[0] = make_uint4(it.k[0], it.k[1], it.k[2], it.k[3]);
    q[1] = make_uint4(it.k[4], it.k[5], it.k[6], it.k[7]);
    reinterpret_cast<uint32_t*>(sm + (size_t)kSortTile * 32)[p] = it.id;
  }
  static __device__ __forceinline__ void get(const unsigned char* sm, int p, Item<32>& it) {
    const uint4* q = reinterpret_cast<const uint4*>(sm) + 2 * p;
    const uint4 a = q[0], b = q[1];
    it.k[0] = a.x; it.k[1] = a.y; it.k[2] = a.z; it.k[3] = a.w;
    it.k[4] = b.x; it.k[5] = b.y; it.k[6] = b.z; it.k[7] = b.w;
    it.id = reinterpret_cast<const uint32_t*>(sm + (size_t)kSortTile * 32)[p];
  }
};

constexpr int kSortWarps = kSortThreads / 32;

template <int S>
struct SortSmem {
  static constexpr size_t stage = Stage<S>::bytes;
  static constexpr size_t whist = (size_t)kSortWarps * kRadix * 4;
  static constexpr size_t bytes = stage + whist + 2 * kRadix * 4 + 32 * 4;
};

// Mask of the lanes whose 8-bit digit equals this lane's (and whose validity matches), from
// match.any, from 8 ballots (one per digit bit), or (kRankBallotVary) from ballots on the bits in
// `vary` only: the digit bits that differ between items anywhere in the array (the others are
// equal in every valid lane; the branches are warp-uniform).
// kAllValid: every lane holds an item (a full row), so no validity vote is needed.
template <int kMode, bool kAllValid = false>
__device__ __forceinline__ uint32_t match_digit(uint32_t dig, bool valid, uint32_t vary) {
  if (kMode == kRankMatchAny) {
    return __match_any_sync(0xffffffffu, (kAllValid || valid) ? dig : 0x100u);
  } else {
    uint32_t peers = 0xffffffffu;
    if (!kAllValid) {
      peers = __ballot_sync(0xffffffffu, valid);
      if (!valid) peers = ~peers;
    }
#pragma unroll
    for (int b = 0; b < kRadixBits; ++b) {
      if (kMode == kRankBallotVary && !((vary >> b) & 1u)) continue;
      const bool bit = (dig >> b) & 1u;
      const uint32_t vote = __ballot_sync(0xffffffffu, bit);
      peers &= bit ? vote : ~vote;
    }
    return peers;
  }
}

// Per-pass values of the plan, read once by thread 0 and shared, together with the error word
// (so that every thread of the CTA takes the same early exit).
struct PassInfo {
  uint32_t U, run, src, next, vary;
  uint32_t bits;  // digit width (8, or 6 / 7 bits of a packed key)
  uint32_t keys;  // k_tile_count reads digit d from the keys: a first pass whose digit is not in the
                  // compaction's plane (unpacked keys whose byte 0 is constant)
};

// A skipped pass exits without a barrier: every thread reads the skip flag through the read-only
// cache (written by an earlier kernel), so the CTAs of a skipped pass cost almost nothing.
template <bool kCount = false>
__device__ __forceinline__ PassInfo pass_info(const WsPtrs& ws, int d) {
  __shared__ PassInfo s_pi;
  if (__ldg(ws.plan->skip + d)) return PassInfo{0, 0, 0, 0, 0, 8, 0};
  if (threadIdx.x == 0) {
    const Plan* plan = ws.plan;
    const uint32_t skip = plan->skip[d], U = plan->U, src = plan->src[d];
    const int next = plan->next[d];
    const uint32_t err = *(volatile const uint32_t*)&ws.ctrl->err;
    s_pi.U = U;
    s_pi.run = (!skip && err == 0) ? 1u : 0u;
    s_pi.src = src;
    s_pi.next = (uint32_t)(int32_t)next;
    s_pi.vary = plan->vary[d];
    s_pi.bits = plan->dbits;
    if (kCount) {
      const int first = plan->first;
      s_pi.keys = (d == first && d != 0 && !plan->plane_first) ? 1u : 0u;
    }
  }
  __syncthreads();
  const PassInfo pi = s_pi;
  __syncthreads();
  return pi;
}

// Word `word` of item i's key, read from an item buffer.
template <int S>
__device__ __forceinline__ uint32_t item_key_word(const unsigned char* buf, int64_t i, int word) {
  constexpr int kStride = soa_items(S) ? S / 4 : S / 4 + 1;  // words per item in the key array
  return reinterpret_cast<const uint32_t*>(buf)[i * kStride + word];
}

// Where digit d of a K-word key lies: bits [d * bits, d * bits + bits) counted from the least
// significant bit of word K - 1 (word 0 is the most significant).  A digit of fewer than 8 bits may
// straddle two words: its high part is then the low bits of the next more significant word.
struct DigitLoc {
  int word, shift;
  bool straddle;
  uint32_t mask;
};
template <int K>
__device__ __forceinline__ DigitLoc digit_loc(int d, uint32_t bits) {
  const int o = d * (int)bits;
  DigitLoc L;
  L.word = K - 1 - (o >> 5);
  L.shift = o & 31;
  L.straddle = L.shift + (int)bits > 32 && L.word > 0;
  L.mask = (1u << bits) - 1u;
  return L;
}
// The digit from its low word and the next more significant one (used only when straddling).
__device__ __forceinline__ uint32_t digit_from(uint32_t lo, uint32_t hi, const DigitLoc& L) {
  return (L.straddle ? __funnelshift_r(lo, hi, L.shift) : lo >> L.shift) & L.mask;
}
// Digit d of a key held in registers.
template <int K>
__device__ __forceinline__ uint32_t key_digit_loc(const uint32_t (&k)[K], const DigitLoc& L) {
  return digit_from(key_word<K>(k, L.word), L.straddle ? key_word<K>(k, L.word - 1) : 0u, L);
}

}  // namespace reindex
