// One LSD radix pass of the (key, old index) sort (Section 2.2's key-value sort) in which the
// offset of every tile within every digit is known before the pass moves any item, so that no
// tile waits for another (the "tiles" sort variant).  Three launches per digit position d:
//   k_tile_count    per tile of 4096 items, how many carry each digit value, and the pass's
//                   digit totals.  It reads a byte plane holding each item's digit d at the
//                   item's position, written by the previous pass (for the first pass, by the
//                   compaction);
//   k_tile_offsets  per digit value v, the exclusive scan of its counts over the tiles plus the
//                   number of items whose digit is below v;
//   k_tile_scatter  loads a tile, ranks its digits inside each warp (stable), stages the tile in
//                   digit order in shared memory and writes it out in runs; every item also
//                   writes its digit of the next non-trivial pass into the byte plane.
// Every pass is the same stable pass as k_onesweep, so the result is identical.  No upfront
// histograms are needed: trivial passes are known from the key bit masks, and when many key bits
// are constant the compaction packs the varying ones (KeyPack), so the passes sort fewer bytes.
// Extra traffic per item and pass: one byte written and one read.
#include <algorithm>

#include "radix.cuh"

namespace reindex {

// Tile counts (then offsets) live in sort look-back area 0, digit-major: cnt[v * tilesS + tile].
// The pass's digit totals accumulate in the histogram row of digit d.
__device__ __forceinline__ uint32_t* tile_counts(const WsPtrs& ws, int v) {
  return ws.lb_sort + (size_t)v * (size_t)ws.tilesS;
}

// k_tile_count: a CTA counts 16 consecutive tiles, each warp two whole tiles into its own
// histogram row (so warps never contend), then the CTA writes every digit's 16 counts as one
// contiguous 64-byte run.  Rows are padded by one word so that reading a column is conflict-free.
constexpr int kCntTiles = 16;
constexpr int kHPad = kRadix + 1;
constexpr int kLaneDigits = kSortTile / 32;  // 128 digits of a tile per lane
static_assert(kCntTiles == 2 * kWarps, "two tiles per warp");

template <int S>
__global__ void __launch_bounds__(kThreads, 4) k_tile_count(WsPtrs ws, int d) {
  __shared__ uint32_t h[kCntTiles * kHPad];
  pdl_wait();
  pdl_trigger();
  const PassInfo pi = pass_info<true>(ws, d);
  if (!pi.run) return;
  const uint32_t U = pi.U;
  const uint32_t ntiles = (U + kSortTile - 1) / kSortTile;
  const uint32_t t0 = blockIdx.x * kCntTiles;
  if (t0 >= ntiles) return;
  const unsigned char* items = pi.src ? ws.itemsB : ws.itemsA;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  for (int i = t; i < kCntTiles * kHPad; i += kThreads) h[i] = 0;
  __syncthreads();
#pragma unroll 1
  for (int k = 0; k < 2; ++k) {
    const int tl = w + k * kWarps;
    const uint32_t tile = t0 + tl;
    if (tile >= ntiles) break;
    const uint32_t base = tile * kSortTile;
    const int n = (int)min((uint32_t)kSortTile, U - base);
    uint32_t* hr = h + tl * kHPad;
    if (pi.keys) {
      const int word = S / 4 - 1 - (d >> 2), sh = (d & 3) * 8;
      for (int i = lane; i < n; i += 32)
        atomicAdd(hr + ((item_key_word<S>(items, (int64_t)base + i, word) >> sh) & 0xFFu), 1u);
      continue;
    }
    // lane's 128 digits: 8 chunks of 16, chunk c at c*512 + lane*16; all loads issued first
    uint4 v[kLaneDigits / 16];
#pragma unroll
    for (int c = 0; c < kLaneDigits / 16; ++c) {
      const int p = c * 512 + lane * 16;
      v[c] = p < n ? __ldcs(reinterpret_cast<const uint4*>(ws.digits + base + p)) : make_uint4(0, 0, 0, 0);
    }
#pragma unroll
    for (int c = 0; c < kLaneDigits / 16; ++c) {
      const int p = c * 512 + lane * 16;
      const uint32_t q4[4] = {v[c].x, v[c].y, v[c].z, v[c].w};
#pragma unroll
      for (int i = 0; i < 16; ++i)
        if (p + i < n) atomicAdd(hr + ((q4[i >> 2] >> ((i & 3) * 8)) & 0xFFu), 1u);
    }
  }
  __syncthreads();
  // digit rows: half-warp per row, lane -> tile t0 + (lane & 15)
  const uint32_t myt = t0 + (lane & 15);
#pragma unroll 4
  for (int r = 0; r < kRadix / (2 * kWarps); ++r) {
    const int v = w * (kRadix / kWarps) + 2 * r + (lane >> 4);
    if (myt < ntiles) tile_counts(ws, v)[myt] = h[(lane & 15) * kHPad + v];
  }
  uint32_t total = 0;  // digit t over this CTA's tiles
#pragma unroll
  for (int i = 0; i < kCntTiles; ++i) total += h[i * kHPad + t];
  if (total) atomicAdd(ws.hist + d * kRadix + t, total);
}

constexpr int kOffThreads = 512;
constexpr int kOffWarps = kOffThreads / 32;
constexpr int kOffBatch = 8;  // rows of 32 counts loaded together per warp

// One CTA per digit value v: cnt[v][tile] -> (items with a digit below v) + sum of
// cnt[v][0 .. tile) (or the same over the chunks of the chunk sort).  Warp w owns a contiguous segment of the column and walks it in rows of 32
// consecutive tiles (coalesced): a first sweep sums the segment, one barrier gives the segment
// starts, and a second sweep scans each row and writes the offsets.
__global__ void __launch_bounds__(kOffThreads, 2) k_tile_offsets(WsPtrs ws, int d, int cols) {
  __shared__ uint32_t s_seg[kOffWarps];
  __shared__ uint32_t s_below[kRadix / 32];
  pdl_wait();
  pdl_trigger();
  const PassInfo pi = pass_info(ws, d);
  if (!pi.run) return;
  // tiles sort: one count per 4096-item tile, column v at v * tilesS; chunk sort (cols > 0): one
  // count per chunk, column v at v * cols
  const uint32_t ntiles = cols > 0 ? (uint32_t)cols : (pi.U + kSortTile - 1) / kSortTile;
  const int v = blockIdx.x, t = threadIdx.x, lane = t & 31, w = t >> 5;
  uint32_t* col = cols > 0 ? ws.lb_sort + (size_t)v * cols : tile_counts(ws, v);
  const uint32_t rows = (ntiles + 32 * kOffWarps - 1) / (32 * kOffWarps);  // rows of 32 per warp
  const uint32_t seg0 = (uint32_t)w * rows * 32;
  uint32_t below = (t < v) ? ws.hist[d * kRadix + t] : 0u;  // items whose digit is smaller than v
  uint32_t acc = 0;
  for (uint32_t r0 = 0; r0 < rows; r0 += kOffBatch) {
    uint32_t x[kOffBatch];
#pragma unroll
    for (int i = 0; i < kOffBatch; ++i) {
      const uint32_t q = seg0 + (r0 + i) * 32 + lane;
      x[i] = (r0 + i < rows && q < ntiles) ? col[q] : 0u;
    }
#pragma unroll
    for (int i = 0; i < kOffBatch; ++i) acc += x[i];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    acc += __shfl_xor_sync(0xffffffffu, acc, o);
    below += __shfl_xor_sync(0xffffffffu, below, o);
  }
  if (lane == 0) {
    s_seg[w] = acc;
    if (w < kRadix / 32) s_below[w] = below;
  }
  __syncthreads();
  uint32_t carry = 0;
#pragma unroll
  for (int q = 0; q < kRadix / 32; ++q) carry += s_below[q];
  for (int q = 0; q < w; ++q) carry += s_seg[q];
  for (uint32_t r0 = 0; r0 < rows; r0 += kOffBatch) {
    uint32_t x[kOffBatch];
#pragma unroll
    for (int i = 0; i < kOffBatch; ++i) {
      const uint32_t q = seg0 + (r0 + i) * 32 + lane;
      x[i] = (r0 + i < rows && q < ntiles) ? col[q] : 0u;
    }
#pragma unroll
    for (int i = 0; i < kOffBatch; ++i) {
      const uint32_t q = seg0 + (r0 + i) * 32 + lane;
      const uint32_t incl = warp_incl_scan(x[i]);
      if (r0 + i < rows && q < ntiles) col[q] = carry + incl - x[i];
      carry += __shfl_sync(0xffffffffu, incl, 31);
    }
  }
}

// Selects word `word` (runtime) of a key held in registers.
template <int K>
__device__ __forceinline__ uint32_t pick_word(const uint32_t (&k)[K], int word) {
  uint32_t x = k[0];
#pragma unroll
  for (int q = 1; q < K; ++q)
    if (q == word) x = k[q];
  return x;
}

template <int S, int kWord, int kMode>
__global__ void __launch_bounds__(kSortThreads, S >= 20 ? 1 : 2) k_tile_scatter(WsPtrs ws, int d) {
  constexpr int K = S / 4;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  unsigned char* stage = sm_raw;
  uint32_t* whist = reinterpret_cast<uint32_t*>(sm_raw + SortSmem<S>::stage);  // [warps][256]
  int32_t* goff = reinterpret_cast<int32_t*>(whist + kSortWarps * kRadix);     // [256] global - local pos
  uint32_t* s_misc = reinterpret_cast<uint32_t*>(goff + 2 * kRadix);          // [32]

  pdl_wait();
  pdl_trigger();
  const PassInfo pi = pass_info(ws, d);
  if (!pi.run) return;
  Control* ctrl = ws.ctrl;
  const uint32_t U = pi.U;
  const uint32_t ntiles = (U + kSortTile - 1) / kSortTile;
  const unsigned char* src = pi.src ? ws.itemsB : ws.itemsA;
  unsigned char* dst = pi.src ? ws.itemsA : ws.itemsB;
  const int nd = (int)pi.next;
  const int nword = nd >= 0 ? K - 1 - (nd >> 2) : 0, nshift = nd >= 0 ? (nd & 3) * 8 : 0;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const bool digit_thread = t < kRadix;
  const int shift = (d & 3) * 8;
  uint32_t* wh = whist + w * kRadix;
  const int wbase = w * 32 * kSortIpt;
  const uint32_t* col = digit_thread ? tile_counts(ws, t) : nullptr;

  for (uint32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const uint32_t base = tile * kSortTile;
    const int n = (int)min((uint32_t)kSortTile, U - base);
    const uint32_t toff = digit_thread ? col[tile] : 0u;  // global start of this tile's digit-t items

    // 1. load (warp-striped: row r of warp w is 32 consecutive items)
    Item<S> it[kSortIpt];
#pragma unroll
    for (int r = 0; r < kSortIpt; ++r) {
      const int local = wbase + r * 32 + lane;
      if (local < n) ItemIO<S>::load_cs(src, ws.idoff, (int64_t)(base + local), it[r]);
    }
#pragma unroll
    for (int i = lane; i < kRadix; i += 32) wh[i] = 0;
    __syncwarp();

    // 2. warp-level ranking (stable: row-major, lane order)
    uint32_t rank[kSortIpt / 2];
#pragma unroll
    for (int r = 0; r < kSortIpt; ++r) {
      const bool valid = wbase + r * 32 + lane < n;
      const uint32_t dig = (it[r].k[kWord] >> shift) & 0xFFu;
      const uint32_t peers = match_digit<kMode>(dig, valid, pi.vary);
      const uint32_t lt = peers & lanemask_lt();
      const int leader = __ffs(peers) - 1;
      uint32_t old = 0;
      if (valid && lt == 0) old = atomicAdd(wh + dig, (uint32_t)__popc(peers));
      old = __shfl_sync(0xffffffffu, old, leader);
      const uint32_t rk = old + __popc(lt);
      if (r & 1)
        rank[r >> 1] |= rk << 16;
      else
        rank[r >> 1] = rk;
    }
    __syncthreads();

    // 3. tile-local digit starts and per-(warp, digit) offsets
    uint32_t cnt = 0;
    if (digit_thread) {
#pragma unroll
      for (int q = 0; q < kSortWarps; ++q) cnt += whist[q * kRadix + t];
    }
    const uint32_t incl = warp_incl_scan(cnt);
    if (lane == 31 && digit_thread) s_misc[w] = incl;
    __syncthreads();
    if (digit_thread) {
      uint32_t ts = incl - cnt;
#pragma unroll
      for (int q = 0; q < kRadix / 32; ++q) ts += (q < w) ? s_misc[q] : 0u;
      uint32_t run = ts;
#pragma unroll
      for (int q = 0; q < kSortWarps; ++q) {
        const uint32_t c = whist[q * kRadix + t];
        whist[q * kRadix + t] = run;
        run += c;
      }
      goff[t] = (int32_t)toff - (int32_t)ts;
    }
    __syncthreads();

    // 4. stage in digit order
#pragma unroll
    for (int r = 0; r < kSortIpt; ++r) {
      if (wbase + r * 32 + lane < n) {
        const uint32_t dig = (it[r].k[kWord] >> shift) & 0xFFu;
        const uint32_t rk = (rank[r >> 1] >> ((r & 1) * 16)) & 0xFFFFu;
        Stage<S>::put(stage, (int)(wh[dig] + rk), it[r]);
      }
    }
    __syncthreads();

    // 5. coalesced scatter, with the next pass's digit into the byte plane
#pragma unroll
    for (int r = 0; r < kSortIpt; ++r) {
      const int i = r * kSortThreads + t;
      if (i < n) {
        Item<S> o;
        Stage<S>::get(stage, i, o);
        const uint32_t gpos = (uint32_t)(goff[(o.k[kWord] >> shift) & 0xFFu] + i);
        if (gpos < U) {
          ItemIO<S>::store(dst, ws.idoff, (int64_t)gpos, o);
          if (nd >= 0) ws.digits[gpos] = (uint8_t)(pick_word<K>(o.k, nword) >> nshift);
        } else {
          record_error(ctrl, kErrInternal);  // counts/ranking inconsistency: never write out of range
        }
      }
    }
    __syncthreads();
  }
}

template <int S, int kWord, int kMode>
static int occ_one() {
  cudaFuncSetAttribute(k_tile_scatter<S, kWord, kMode>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)SortSmem<S>::bytes);
  int n = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_tile_scatter<S, kWord, kMode>, kSortThreads,
                                                SortSmem<S>::bytes);
  return n < 1 ? 1 : n;
}

template <int S, int kMode, int kWord = 0>
static int occ_mode() {
  const int n = occ_one<S, kWord, kMode>();
  if constexpr (kWord + 1 < S / 4) return min(n, occ_mode<S, kMode, kWord + 1>());
  return n;
}

// 24- and 32-byte keys are ranked with the vary ballots only.
template <int S>
static int occ() {
  if constexpr (S >= kWideMin)
    return occ_mode<S, kRankBallotVary>();
  else
    return min(occ_mode<S, kRankBallot>(), min(occ_mode<S, kRankMatchAny>(), occ_mode<S, kRankBallotVary>()));
}

int occupancy_tiles(int S) {
  switch (S) {
    case 4: return occ<4>();
    case 8: return occ<8>();
    case 12: return occ<12>();
    case 16: return occ<16>();
    case 20: return occ<20>();
    case 24: return occ<24>();
    default: return occ<32>();
  }
}

cudaError_t launch_tile_count(int S, int digit, WsPtrs ws, const LaunchCfg& c, cudaStream_t st) {
  const int64_t tiles = (ws.Umax + kSortTile - 1) / kSortTile;
  if (tiles < 1) return cudaSuccess;
  const int g = (int)((tiles + kCntTiles - 1) / kCntTiles);
  switch (S) {
    case 4: return launch_pdl(k_tile_count<4>, g, kThreads, 0, st, ws, digit);
    case 8: return launch_pdl(k_tile_count<8>, g, kThreads, 0, st, ws, digit);
    case 12: return launch_pdl(k_tile_count<12>, g, kThreads, 0, st, ws, digit);
    case 16: return launch_pdl(k_tile_count<16>, g, kThreads, 0, st, ws, digit);
    case 20: return launch_pdl(k_tile_count<20>, g, kThreads, 0, st, ws, digit);
    case 24: return launch_pdl(k_tile_count<24>, g, kThreads, 0, st, ws, digit);
    case 32: return launch_pdl(k_tile_count<32>, g, kThreads, 0, st, ws, digit);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_tile_offsets(int digit, WsPtrs ws, cudaStream_t st, int chunks) {
  if (ws.Umax < 1) return cudaSuccess;
  return launch_pdl(k_tile_offsets, kRadix, kOffThreads, 0, st, ws, digit, chunks);
}

// The pass over key word `word` (word 0 is the most significant), one instantiation per word.
template <int S, int kMode, int kWord = 0>
static cudaError_t scatter_word(int word, int g, int digit, WsPtrs ws, cudaStream_t st) {
  if (word == kWord)
    return launch_pdl(k_tile_scatter<S, kWord, kMode>, g, kSortThreads, SortSmem<S>::bytes, st, ws, digit);
  if constexpr (kWord + 1 < S / 4) return scatter_word<S, kMode, kWord + 1>(word, g, digit, ws, st);
  return cudaErrorInvalidValue;
}

template <int S>
static cudaError_t scatter_s(int g, int digit, WsPtrs ws, int mode, cudaStream_t st) {
  const int word = S / 4 - 1 - (digit >> 2);
  if constexpr (S >= kWideMin) {
    if (mode != kRankBallotVary) return cudaErrorInvalidValue;
    return scatter_word<S, kRankBallotVary>(word, g, digit, ws, st);
  } else {
    if (mode == kRankMatchAny) return scatter_word<S, kRankMatchAny>(word, g, digit, ws, st);
    if (mode == kRankBallotVary) return scatter_word<S, kRankBallotVary>(word, g, digit, ws, st);
    return scatter_word<S, kRankBallot>(word, g, digit, ws, st);
  }
}

cudaError_t launch_tile_scatter(int S, int digit, WsPtrs ws, const LaunchCfg& c, cudaStream_t st) {
  const int64_t tiles = (ws.Umax + kSortTile - 1) / kSortTile;
  if (tiles < 1) return cudaSuccess;
  // one CTA per tile (the block scheduler overlaps retiring and starting CTAs), or a few waves of
  // CTAs that stride over the tiles
  const int g = (int)std::min<int64_t>(tiles, c.scatter_waves ? (int64_t)c.scatter_waves * c.sms * c.occ_tiles : tiles);
  switch (S) {
    case 4: return scatter_s<4>(g, digit, ws, c.rank_mode, st);
    case 8: return scatter_s<8>(g, digit, ws, c.rank_mode, st);
    case 12: return scatter_s<12>(g, digit, ws, c.rank_mode, st);
    case 16: return scatter_s<16>(g, digit, ws, c.rank_mode, st);
    case 20: return scatter_s<20>(g, digit, ws, c.rank_mode, st);
    case 24: return scatter_s<24>(g, digit, ws, c.rank_mode, st);
    case 32: return scatter_s<32>(g, digit, ws, c.rank_mode, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace reindex
