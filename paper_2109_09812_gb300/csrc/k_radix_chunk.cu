// One LSD radix pass of the (key, old index) sort (Section 2.2's key-value sort), "chunk"
// variant.  The U items of the pass are cut into G contiguous chunks of whole tiles, one chunk per
// CTA of a single resident wave (G = SMs x resident CTAs per SM, at most one chunk per tile).
// Three launches per digit position d:
//   k_chunk_count    per chunk, how many items carry each digit value (from the byte plane that
//                    holds each item's digit d at the item's position), and the pass's totals;
//   k_tile_offsets   per digit value v, the exclusive scan of its chunk counts plus the number of
//                    items whose digit is below v (k_radix_tiles.cu, chunk columns);
//   k_chunk_scatter  each CTA walks its chunk tile by tile, in order.  The Tensor Memory
//                    Accelerator copies tile k+1 (cp.async.bulk, completion on an mbarrier) into
//                    one shared-memory buffer while tile k is ranked straight from the other
//                    (ballots find the lanes of a warp with equal digits; each warp counts into
//                    its own shared histogram, rows in order, so ranks are stable), its inverse
//                    permutation is built (sorted slot -> original slot and digit), and it is
//                    written out in digit order: sorted slot i goes to run[v] + (i - start of v in
//                    the tile), where run[v] is the CTA's running offset of digit v in the output
//                    (the chunk's offset from the scan, advanced by each tile's count).  Every
//                    item also writes its digit of the next non-trivial pass into the byte plane.
// No CTA waits for another, there is no per-tile offset table (G x 256 counts per pass instead of
// one row per tile), and consecutive tiles of a CTA fill each digit's output run contiguously.
// The result of a pass is that of every other variant: a stable pass on digit d.
#include <algorithm>

#include "radix.cuh"
#include "tma.cuh"

namespace reindex {

// Tiles [t0, t1) of chunk c for U items in tiles of T (the same split in all three kernels).
__device__ __forceinline__ void chunk_tiles(uint32_t U, uint32_t T, uint32_t G, uint32_t c, uint32_t& t0,
                                            uint32_t& t1) {
  const uint32_t ntiles = (U + T - 1) / T;
  const uint32_t tpc = (ntiles + G - 1) / G;
  t0 = min(c * tpc, ntiles);
  t1 = min(t0 + tpc, ntiles);
}

// ---------------------------------------------------------------------------------------------
// k_chunk_count: one CTA per chunk; each warp counts into its own padded histogram row, then the
// CTA writes the chunk's 256 counts (digit-major table cnt[v * G + c], every entry, zeros
// included) and adds them to the pass's digit totals.
constexpr int kChunkCountThreads = 512;
constexpr int kChunkCountWarps = kChunkCountThreads / 32;
constexpr int kCPad = kRadix + 1;
constexpr int kCountBatch = 4;

template <int S>
__global__ void __launch_bounds__(kChunkCountThreads) k_chunk_count(WsPtrs ws, int d, int G, int T) {
  __shared__ uint32_t h[kChunkCountWarps * kCPad];
  pdl_wait();
  pdl_trigger();
  const PassInfo pi = pass_info<true>(ws, d);
  if (!pi.run) return;
  const uint32_t U = pi.U;
  uint32_t t0, t1;
  chunk_tiles(U, (uint32_t)T, (uint32_t)G, blockIdx.x, t0, t1);
  const uint32_t lo = t0 * (uint32_t)T, hi = min(t1 * (uint32_t)T, U);
  const int t = threadIdx.x, w = t >> 5;
  for (int i = t; i < kChunkCountWarps * kCPad; i += kChunkCountThreads) h[i] = 0;
  __syncthreads();
  uint32_t* hr = h + w * kCPad;
  if (pi.keys) {  // the first pass's digit is not in the plane: read it from the keys
    const unsigned char* items = pi.src ? ws.itemsB : ws.itemsA;
    const int word = S / 4 - 1 - (d >> 2), sh = (d & 3) * 8;
    for (uint32_t i = lo + t; i < hi; i += kChunkCountThreads)
      atomicAdd(hr + ((item_key_word<S>(items, (int64_t)i, word) >> sh) & 0xFFu), 1u);
  } else {  // lo is a multiple of T (>= 2048), so 16-byte vectors of the plane are aligned
    // kCountBatch vectors in flight per thread (one at a time left the loads' latency exposed)
    constexpr uint32_t kStep = 16u * kChunkCountThreads;
    for (uint32_t p0 = lo + 16u * t; p0 < hi; p0 += kStep * kCountBatch) {
      uint4 v[kCountBatch];
#pragma unroll
      for (int b = 0; b < kCountBatch; ++b) {
        const uint32_t p = p0 + b * kStep;
        v[b] = p < hi ? __ldcs(reinterpret_cast<const uint4*>(ws.digits + p)) : make_uint4(0, 0, 0, 0);
      }
#pragma unroll
      for (int b = 0; b < kCountBatch; ++b) {
        const uint32_t p = p0 + b * kStep;
        const uint32_t q4[4] = {v[b].x, v[b].y, v[b].z, v[b].w};
        if (p + 16 <= hi) {
#pragma unroll
          for (int i = 0; i < 16; ++i) atomicAdd(hr + ((q4[i >> 2] >> ((i & 3) * 8)) & 0xFFu), 1u);
        } else if (p < hi) {
#pragma unroll
          for (int i = 0; i < 16; ++i)
            if (p + i < hi) atomicAdd(hr + ((q4[i >> 2] >> ((i & 3) * 8)) & 0xFFu), 1u);
        }
      }
    }
  }
  __syncthreads();
  if (t < kRadix) {
    uint32_t total = 0;
#pragma unroll
    for (int q = 0; q < kChunkCountWarps; ++q) total += h[q * kCPad + t];
    ws.lb_sort[(size_t)t * G + blockIdx.x] = total;
    if (total) atomicAdd(ws.hist + d * kRadix + t, total);
  }
}

// ---------------------------------------------------------------------------------------------
// k_chunk_scatter
template <int S, int T, int NT, int NB>
struct ChunkSmem {
  static constexpr int NW = NT / 32, R = T / NT;  // rows of 32 items per warp
  static constexpr bool kAos = !soa_items(S);
  static constexpr size_t stride = kAos ? S + 4 : S;       // bytes per item in the key array
  static constexpr size_t buf = align_up((size_t)T * (S + 4), 128);
  static constexpr size_t ids = kAos ? 0 : (size_t)T * S;  // id plane inside a buffer (SoA)
  static constexpr size_t off_inv = NB * buf;
  static constexpr size_t off_whist = off_inv + (size_t)T * 4;
  static constexpr size_t off_run = off_whist + (size_t)NW * kRadix * 4;
  static constexpr size_t off_goff = off_run + kRadix * 4;
  static constexpr size_t off_misc = off_goff + kRadix * 4;
  static constexpr size_t off_bar = off_misc + 32 * 4;
  static constexpr size_t bytes = off_bar + NB * 8;
  static_assert(T % NT == 0 && NT % 32 == 0 && NT >= kRadix && R >= 1 && R <= 32, "tile shape");
  static_assert(T % 16 == 0 && T <= (1 << 16), "tile size (16-byte aligned copies, 16-bit slots)");
  static_assert(buf % 16 == 0 && ids % 16 == 0 && off_inv % 16 == 0 && off_bar % 8 == 0, "alignment");
};

// Bulk copy of tile `tile` of the item buffer `src` (keys, then the id plane for SoA layouts).
// Addresses are 16-byte aligned: tiles start at multiples of T items, the id plane at a 256-byte
// aligned offset; sizes are rounded up to 16 bytes inside the workspace's spare bytes.
template <int S, int T, int NT, int NB>
__device__ __forceinline__ void chunk_load(unsigned char* dst, const unsigned char* src, int64_t idoff, uint32_t tile,
                                           uint32_t U, uint64_t* bar) {
  using P = ChunkSmem<S, T, NT, NB>;
  const uint32_t base = tile * (uint32_t)T;
  const uint32_t n = min((uint32_t)T, U - base);
  if (P::kAos) {
    const uint32_t b = round16(n * (S + 4));
    mbar_expect_tx(bar, b);
    bulk_load(dst, src + (size_t)base * (S + 4), b, bar);
  } else {
    const uint32_t kb = round16(n * S), ib = round16(n * 4);
    mbar_expect_tx(bar, kb + ib);
    bulk_load(dst, src + (size_t)base * S, kb, bar);
    bulk_load(dst + P::ids, src + idoff + (size_t)base * 4, ib, bar);
  }
}

template <int S, int T>
__device__ __forceinline__ void chunk_item(const unsigned char* buf, int i, Item<S>& it) {
  if constexpr (S == 4) {
    const uint2 v = reinterpret_cast<const uint2*>(buf)[i];
    it.k[0] = v.x; it.id = v.y;
  } else if constexpr (S == 12) {
    const uint4 v = reinterpret_cast<const uint4*>(buf)[i];
    it.k[0] = v.x; it.k[1] = v.y; it.k[2] = v.z; it.id = v.w;
  } else if constexpr (S == 20) {
    const uint2* q = reinterpret_cast<const uint2*>(buf) + 3 * i;
    const uint2 a = q[0], b = q[1], c = q[2];
    it.k[0] = a.x; it.k[1] = a.y; it.k[2] = b.x; it.k[3] = b.y; it.k[4] = c.x; it.id = c.y;
  } else {  // SoA: S/8 8-byte or S/16 16-byte key vectors, then the id plane
    if constexpr (S % 16 == 0) {
      const uint4* q = reinterpret_cast<const uint4*>(buf) + (S / 16) * i;
#pragma unroll
      for (int h = 0; h < S / 16; ++h) {
        const uint4 v = q[h];
        it.k[4 * h] = v.x; it.k[4 * h + 1] = v.y; it.k[4 * h + 2] = v.z; it.k[4 * h + 3] = v.w;
      }
    } else {
      const uint2* q = reinterpret_cast<const uint2*>(buf) + (S / 8) * i;
#pragma unroll
      for (int h = 0; h < S / 8; ++h) {
        const uint2 v = q[h];
        it.k[2 * h] = v.x; it.k[2 * h + 1] = v.y;
      }
    }
    it.id = reinterpret_cast<const uint32_t*>(buf + (size_t)T * S)[i];
  }
}

// Stable ranks of one tile's items inside each warp: digit of item i from shared memory, lanes
// with equal digits from the digit matcher, each group counted into the warp's histogram in row
// order (rank = the warp's earlier count of that digit + lanes below with the same digit).
template <int S, int kMode, int T, int NT, int NB, bool kFull>
__device__ __forceinline__ void chunk_rank(const unsigned char* cb, int n, int w, int lane, const DigitLoc& dl,
                                           uint32_t vary, uint32_t* wh, uint32_t (&dig)[T / NT],
                                           uint32_t (&rk)[T / NT]) {
  using P = ChunkSmem<S, T, NT, NB>;
  constexpr int R = T / NT;
  const unsigned char* base = cb + (size_t)(w * R * 32 + lane) * P::stride + 4 * dl.word;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const bool valid = kFull || (w * R + r) * 32 + lane < n;
    const uint32_t* q = reinterpret_cast<const uint32_t*>(base + (size_t)r * 32 * P::stride);
    dig[r] = valid ? digit_from(q[0], dl.straddle ? q[-1] : 0u, dl) : 0u;
    const uint32_t peers = match_digit<kMode, kFull>(dig[r], valid, vary);
    const uint32_t lt = peers & lanemask_lt();
    uint32_t old = 0;
    if (valid && lt == 0) old = atomicAdd(wh + dig[r], (uint32_t)__popc(peers));
    rk[r] = __shfl_sync(0xffffffffu, old, __ffs(peers) - 1) + __popc(lt);  // rows in order: stable
  }
}

// Write-out of one tile in digit order: sorted slot i = r * NT + t reads its item through the
// inverse permutation and stores it at goff[digit] + i, with the next pass's digit into the plane.
template <int S, int T, int NT, bool kFull>
__device__ __forceinline__ void chunk_write(const unsigned char* cb, const uint32_t* inv, const uint32_t* goff, int n,
                                            int t, uint32_t U, unsigned char* dst, const WsPtrs& ws, int nd,
                                            const DigitLoc& ndl, Control* ctrl) {
  constexpr int K = S / 4, R = T / NT;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = r * NT + t;
    if (kFull || i < n) {
      const uint32_t e = inv[i];
      Item<S> o;
      chunk_item<S, T>(cb, (int)(e >> 8), o);
      const uint32_t gpos = goff[e & 0xFFu] + (uint32_t)i;
      if (gpos < U) {
        ItemIO<S>::store(dst, ws.idoff, (int64_t)gpos, o);
        if (nd >= 0) ws.digits[gpos] = (uint8_t)key_digit_loc<K>(o.k, ndl);
      } else {
        record_error(ctrl, kErrInternal);  // counts/ranking inconsistency: never write out of range
      }
    }
  }
}

template <int S, int kMode, int T, int NT, int NB, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_chunk_scatter(WsPtrs ws, int d, int G) {
  using P = ChunkSmem<S, T, NT, NB>;
  constexpr int K = S / 4, NW = P::NW, R = P::R;
  extern __shared__ __align__(128) unsigned char sm[];
  uint32_t* inv = reinterpret_cast<uint32_t*>(sm + P::off_inv);     // [T] sorted slot -> (slot << 8) | digit
  uint32_t* whist = reinterpret_cast<uint32_t*>(sm + P::off_whist); // [NW][256]
  uint32_t* run = reinterpret_cast<uint32_t*>(sm + P::off_run);     // [256] running output offsets
  uint32_t* goff = reinterpret_cast<uint32_t*>(sm + P::off_goff);   // [256] run - tile-local start
  uint32_t* misc = reinterpret_cast<uint32_t*>(sm + P::off_misc);   // [8] scan partials
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + P::off_bar);     // [NB]

  pdl_wait();
  pdl_trigger();
  const PassInfo pi = pass_info(ws, d);
  if (!pi.run) return;
  Control* ctrl = ws.ctrl;
  const uint32_t U = pi.U;
  uint32_t t0, t1;
  chunk_tiles(U, (uint32_t)T, (uint32_t)G, blockIdx.x, t0, t1);
  if (t0 >= t1) return;  // same in every thread
  const uint32_t nt = t1 - t0;
  const unsigned char* src = pi.src ? ws.itemsB : ws.itemsA;
  unsigned char* dst = pi.src ? ws.itemsA : ws.itemsB;
  const int nd = (int)pi.next;
  const DigitLoc dl = digit_loc<K>(d, pi.bits), ndl = digit_loc<K>(nd >= 0 ? nd : 0, pi.bits);
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const bool digit_thread = t < kRadix;
  if (digit_thread) run[t] = ws.lb_sort[(size_t)t * G + blockIdx.x];  // the chunk's offset of digit t
  if (t == 0) {
    for (int b = 0; b < NB; ++b) mbar_init(bar + b, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");  // barriers visible to the copy engine
    fence_proxy_async();
    for (uint32_t j = 0; j < (uint32_t)NB && j < nt; ++j)
      chunk_load<S, T, NT, NB>(sm + j * P::buf, src, ws.idoff, t0 + j, U, bar + j);
  }
  __syncthreads();
  uint32_t* wh = whist + w * kRadix;

  for (uint32_t k = 0; k < nt; ++k) {
    const uint32_t b = k % NB, tile = t0 + k;
    unsigned char* cb = sm + b * P::buf;
    const int n = (int)min((uint32_t)T, U - tile * (uint32_t)T);
    wait_tile(bar + b, (k / NB) & 1u, ctrl);

    // 1. rank: warp w owns rows w*R .. w*R+R-1 (items in original order)
#pragma unroll
    for (int i = lane; i < kRadix; i += 32) wh[i] = 0;
    __syncwarp();
    uint32_t dig[R], rk[R];
    if (n == T)
      chunk_rank<S, kMode, T, NT, NB, true>(cb, n, w, lane, dl, pi.vary, wh, dig, rk);
    else
      chunk_rank<S, kMode, T, NT, NB, false>(cb, n, w, lane, dl, pi.vary, wh, dig, rk);
    __syncthreads();

    // 2. tile counts -> tile-local digit starts -> per-(warp, digit) starts; output offsets
    uint32_t cnt = 0;
    if (digit_thread) {
#pragma unroll
      for (int q = 0; q < NW; ++q) cnt += whist[q * kRadix + t];
    }
    const uint32_t incl = warp_incl_scan(cnt);
    if (lane == 31 && digit_thread) misc[w] = incl;
    __syncthreads();
    if (digit_thread) {
      uint32_t ts = incl - cnt;
#pragma unroll
      for (int q = 0; q < kRadix / 32; ++q) ts += (q < w) ? misc[q] : 0u;
      uint32_t s = ts;
#pragma unroll
      for (int q = 0; q < NW; ++q) {
        const uint32_t c = whist[q * kRadix + t];
        whist[q * kRadix + t] = s;
        s += c;
      }
      goff[t] = run[t] - ts;
      run[t] += cnt;
    }
    __syncthreads();

    // 3. inverse permutation: sorted slot -> (original slot, digit)
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int i = (w * R + r) * 32 + lane;
      if (i < n) inv[wh[dig[r]] + rk[r]] = ((uint32_t)i << 8) | dig[r];
    }
    __syncthreads();

    // 4. write out in digit order (consecutive threads write consecutive slots of a digit run),
    //    with the next pass's digit into the byte plane
    if (n == T)
      chunk_write<S, T, NT, true>(cb, inv, goff, n, t, U, dst, ws, nd, ndl, ctrl);
    else
      chunk_write<S, T, NT, false>(cb, inv, goff, n, t, U, dst, ws, nd, ndl, ctrl);
    __syncthreads();  // buffer b and inv are free

    // 5. start the copy of the tile NB ahead into the freed buffer
    if (t == 0 && k + NB < nt) {
      fence_proxy_async();  // the generic-proxy reads of buffer b happen before the async write
      chunk_load<S, T, NT, NB>(cb, src, ws.idoff, tile + NB, U, bar + b);
    }
  }
}

// Tile shapes (two shared-memory tile buffers each):
//   cfg 0 "big":   4096-item tiles (2048 for items over 20 bytes), 512 threads, 1 CTA per SM;
//   cfg 1 "small": 2048-item tiles, 256 threads, up to 2 CTAs per SM;
//   cfg 2 "wide":  2048-item tiles, 512 threads, 2 CTAs per SM (registers capped at 64);
//   cfg 3 "deep":  4096-item tiles (2048 over 20 bytes), 1024 threads, 1 CTA per SM (64 registers).
template <int S, int C>
struct ChunkCfg;
// Largest tile of S-byte keys whose two buffers fit beside the tables: 4096 items up to 20-byte
// items, 2048 up to 36 bytes, 1024 for the 52- and 68-byte items of 48- and 64-byte keys.
constexpr int chunk_tile_max(int S) { return S + 4 <= 20 ? 4096 : (S + 4 <= 36 ? 2048 : 1024); }
template <int S>
struct ChunkCfg<S, 0> {
  static constexpr int T = chunk_tile_max(S), NT = 512, NB = 2, MINB = 1;
};
template <int S>
struct ChunkCfg<S, 1> {
  static constexpr int T = chunk_tile_max(S) < 2048 ? chunk_tile_max(S) : 2048, NT = 256, NB = 2, MINB = 1;
};
template <int S>
struct ChunkCfg<S, 2> {
  static constexpr int T = chunk_tile_max(S) < 2048 ? chunk_tile_max(S) : 2048, NT = 512, NB = 2, MINB = 2;
};
template <int S>
struct ChunkCfg<S, 3> {
  static constexpr int T = chunk_tile_max(S), NT = 1024, NB = 2, MINB = 1;
};

// Digit matching: for keys up to 12 bytes 8 ballots, match.any, or ballots on the varying digit
// bits only (the one that skips the ballots of bits a narrower digit does not have); wider keys
// always the last (the per-stride default of the other radix passes).
template <int S>
constexpr int chunk_mode(int mode) {
  return S >= 16 ? kRankBallotVary : mode;
}

template <int S, int C, int kMode = kRankBallot>
static auto chunk_kernel() {
  using F = ChunkCfg<S, C>;
  return k_chunk_scatter<S, chunk_mode<S>(kMode), F::T, F::NT, F::NB, F::MINB>;
}

template <int S, int C>
static size_t chunk_smem() {
  using F = ChunkCfg<S, C>;
  return ChunkSmem<S, F::T, F::NT, F::NB>::bytes;
}

template <int S, int C>
static int chunk_occ_one() {
  int best = 0;
  for (int m = 0; m < (S <= 12 ? 3 : 1); ++m) {  // every matcher for keys up to 12 bytes
    auto k = m == 0 ? chunk_kernel<S, C, kRankBallot>()
                    : (m == 1 ? chunk_kernel<S, C, kRankMatchAny>() : chunk_kernel<S, C, kRankBallotVary>());
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)chunk_smem<S, C>()) != cudaSuccess)
      return 0;
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, ChunkCfg<S, C>::NT, chunk_smem<S, C>());
    best = m ? std::min(best, n) : n;
  }
  return best;
}

template <int S>
static int chunk_occ_s(int cfg) {
  switch (cfg) {
    case 1: return chunk_occ_one<S, 1>();
    case 2: return chunk_occ_one<S, 2>();
    case 3: return chunk_occ_one<S, 3>();
    default: return chunk_occ_one<S, 0>();
  }
}

int occupancy_chunk(int S, int cfg) {
  switch (S) {
    case 4: return chunk_occ_s<4>(cfg);
    case 8: return chunk_occ_s<8>(cfg);
    case 12: return chunk_occ_s<12>(cfg);
    case 16: return chunk_occ_s<16>(cfg);
    case 20: return chunk_occ_s<20>(cfg);
    case 24: return chunk_occ_s<24>(cfg);
    case 32: return chunk_occ_s<32>(cfg);
    case 48: return chunk_occ_s<48>(cfg);
    case 64: return chunk_occ_s<64>(cfg);
    default: return 0;
  }
}

int chunk_tile_items(int S, int cfg) {
  const int t = chunk_tile_max(S);
  return (cfg == 1 || cfg == 2) ? std::min(t, 2048) : t;
}

int chunk_grid(int S, const LaunchCfg& c, int64_t Umax) {
  const int T = chunk_tile_items(S, c.chunk_cfg);
  const int occ = c.occ_chunk[c.chunk_cfg];
  int per_sm = occ < 1 ? 1 : occ;
  if (c.chunk_occ > 0 && c.chunk_occ < per_sm) per_sm = c.chunk_occ;
  const int64_t tiles = (Umax + T - 1) / T;
  int64_t g = std::min<int64_t>((int64_t)c.sms * per_sm, tiles);
  if (c.chunk_grid_cap > 0) g = std::min<int64_t>(g, c.chunk_grid_cap);
  return (int)std::max<int64_t>(1, g);
}

cudaError_t launch_chunk_count(int S, int digit, WsPtrs ws, int G, int T, cudaStream_t st) {
  if (ws.Umax < 1) return cudaSuccess;
  switch (S) {
    case 4: return launch_pdl(k_chunk_count<4>, G, kChunkCountThreads, 0, st, ws, digit, G, T);
    case 8: return launch_pdl(k_chunk_count<8>, G, kChunkCountThreads, 0, st, ws, digit, G, T);
    case 12: return launch_pdl(k_chunk_count<12>, G, kChunkCountThreads, 0, st, ws, digit, G, T);
    case 16: return launch_pdl(k_chunk_count<16>, G, kChunkCountThreads, 0, st, ws, digit, G, T);
    case 20: return launch_pdl(k_chunk_count<20>, G, kChunkCountThreads, 0, st, ws, digit, G, T);
    case 24: return launch_pdl(k_chunk_count<24>, G, kChunkCountThreads, 0, st, ws, digit, G, T);
    case 32: return launch_pdl(k_chunk_count<32>, G, kChunkCountThreads, 0, st, ws, digit, G, T);
    case 48: return launch_pdl(k_chunk_count<48>, G, kChunkCountThreads, 0, st, ws, digit, G, T);
    case 64: return launch_pdl(k_chunk_count<64>, G, kChunkCountThreads, 0, st, ws, digit, G, T);
    default: return cudaErrorInvalidValue;
  }
}

template <int S, int C>
static cudaError_t scatter_c(int mode, int G, int digit, WsPtrs ws, cudaStream_t st) {
  constexpr int NT = ChunkCfg<S, C>::NT;
  if (S <= 12 && mode == kRankMatchAny)
    return launch_pdl(chunk_kernel<S, C, kRankMatchAny>(), G, NT, chunk_smem<S, C>(), st, ws, digit, G);
  if (S <= 12 && mode == kRankBallotVary)
    return launch_pdl(chunk_kernel<S, C, kRankBallotVary>(), G, NT, chunk_smem<S, C>(), st, ws, digit, G);
  return launch_pdl(chunk_kernel<S, C, kRankBallot>(), G, NT, chunk_smem<S, C>(), st, ws, digit, G);
}

template <int S>
static cudaError_t scatter_s(int cfg, int mode, int G, int digit, WsPtrs ws, cudaStream_t st) {
  switch (cfg) {
    case 1: return scatter_c<S, 1>(mode, G, digit, ws, st);
    case 2: return scatter_c<S, 2>(mode, G, digit, ws, st);
    case 3: return scatter_c<S, 3>(mode, G, digit, ws, st);
    default: return scatter_c<S, 0>(mode, G, digit, ws, st);
  }
}

cudaError_t launch_chunk_scatter(int S, int digit, WsPtrs ws, const LaunchCfg& c, int G, cudaStream_t st) {
  if (ws.Umax < 1) return cudaSuccess;
  const int cfg = c.chunk_cfg;
  // narrower digits: ballots on the digit's bits only
  const int mode = (c.digit_bits < 8 && c.rank_mode == kRankBallot) ? kRankBallotVary : c.rank_mode;
  switch (S) {
    case 4: return scatter_s<4>(cfg, mode, G, digit, ws, st);
    case 8: return scatter_s<8>(cfg, mode, G, digit, ws, st);
    case 12: return scatter_s<12>(cfg, mode, G, digit, ws, st);
    case 16: return scatter_s<16>(cfg, mode, G, digit, ws, st);
    case 20: return scatter_s<20>(cfg, mode, G, digit, ws, st);
    case 24: return scatter_s<24>(cfg, mode, G, digit, ws, st);
    case 32: return scatter_s<32>(cfg, mode, G, digit, ws, st);
    case 48: return scatter_s<48>(cfg, mode, G, digit, ws, st);
    case 64: return scatter_s<64>(cfg, mode, G, digit, ws, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace reindex
