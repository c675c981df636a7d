// Software-pipelined variant of the onesweep radix pass (same result as k_onesweep; Section 2.2's
// key-value sort, one stable 8-bit LSD pass).
//
// One persistent CTA per SM keeps three tiles in flight in a ring of three shared-memory
// buffers:
//   - tile k+2 is being copied in by the Tensor Memory Accelerator (cp.async.bulk, completion on
//     an mbarrier), issued two iterations before it is needed;
//   - tile k is ranked straight from shared memory (8 ballots per row find the lanes with equal
//     digits; the group's lowest lane adds the group size to the warp's counter) and its
//     per-digit counts are published;
//   - tile k-1, whose look-back finished in the previous iteration, is written out: output slot
//     i (in digit order) reads its item through a 16-bit inverse permutation, so consecutive
//     threads write consecutive addresses of one digit run.
// The decoupled look-back of tile k runs at the end of the iteration: each warp resolves a group
// of digits over the 32 nearest predecessors at once (warp_lookback_tiles).  Items never pass
// through registers between phases, so the CTA can run 1024 threads.
#include "internal.h"
#include "tma.cuh"

namespace reindex {

template <int S>
struct Pipe;
template <>
struct Pipe<4> {
  static constexpr int kThreads = 1024, kTile = 4096;
};
template <>
struct Pipe<8> {
  static constexpr int kThreads = 1024, kTile = 4096;
};
template <>
struct Pipe<12> {
  static constexpr int kThreads = 1024, kTile = 3072;
};
template <>
struct Pipe<16> {
  static constexpr int kThreads = 512, kTile = 3072;
};
template <>
struct Pipe<20> {
  static constexpr int kThreads = 512, kTile = 2048;
};

template <int S>
struct PipeSmem {
  static constexpr int T = Pipe<S>::kTile, NT = Pipe<S>::kThreads, NW = NT / 32;
  static constexpr bool kAos = (S == 4 || S == 12 || S == 20);
  static constexpr int kRows = T / NT;  // 32-item rows per warp
  static constexpr size_t buf = kAos ? (size_t)T * (S + 4) : (size_t)T * (S + 4);
  static constexpr size_t ids = kAos ? 0 : (size_t)T * S;  // id plane offset inside a buffer (SoA)
  static constexpr size_t off_inv = 3 * buf;
  static constexpr size_t off_whist = off_inv + 2 * (size_t)T * 2;
  static constexpr size_t off_goff = off_whist + (size_t)NW * kRadix * 4;
  static constexpr size_t off_cnt = off_goff + 2 * kRadix * 4;      // tcnt, tstart, gbase
  static constexpr size_t off_bar = off_cnt + 3 * kRadix * 4;
  static constexpr size_t off_misc = off_bar + 4 * 8;
  static constexpr size_t bytes = off_misc + 32 * 4;
  static_assert(T % NT == 0 && T <= 65536 && T >= kSortTileMin, "tile shape");
  static_assert(buf % 16 == 0 && off_inv % 16 == 0 && off_whist % 16 == 0, "bulk-copy alignment");
};

// Issue the bulk copy of tile `tile` (< ntiles) of the item buffer `src` into shared buffer dst.
template <int S>
__device__ __forceinline__ void load_tile(unsigned char* dst, const unsigned char* src, int64_t idoff, uint32_t tile,
                                          uint32_t U, uint64_t* bar) {
  using P = PipeSmem<S>;
  const uint32_t base = tile * (uint32_t)P::T;
  const uint32_t n = min((uint32_t)P::T, U - base);
  if (P::kAos) {
    const uint32_t bytes = round16(n * (S + 4));
    mbar_expect_tx(bar, bytes);
    bulk_load(dst, src + (size_t)base * (S + 4), bytes, bar);
  } else {
    const uint32_t kb = round16(n * S), ib = round16(n * 4);
    mbar_expect_tx(bar, kb + ib);
    bulk_load(dst, src + (size_t)base * S, kb, bar);
    bulk_load(dst + P::ids, src + idoff + (size_t)base * 4, ib, bar);
  }
}

template <int S, int kWord>
__device__ __forceinline__ uint32_t smem_word(const unsigned char* buf, int i) {
  return *reinterpret_cast<const uint32_t*>(buf + (size_t)i * (PipeSmem<S>::kAos ? S + 4 : S) + 4 * kWord);
}

template <int S>
__device__ __forceinline__ void smem_item(const unsigned char* buf, int i, Item<S>& it) {
  if constexpr (S == 4) {
    const uint2 v = reinterpret_cast<const uint2*>(buf)[i];
    it.k[0] = v.x; it.id = v.y;
  } else if constexpr (S == 12) {
    const uint4 v = reinterpret_cast<const uint4*>(buf)[i];
    it.k[0] = v.x; it.k[1] = v.y; it.k[2] = v.z; it.id = v.w;
  } else if constexpr (S == 8) {
    const uint2 v = reinterpret_cast<const uint2*>(buf)[i];
    it.k[0] = v.x; it.k[1] = v.y;
    it.id = reinterpret_cast<const uint32_t*>(buf + PipeSmem<S>::ids)[i];
  } else if constexpr (S == 16) {
    const uint4 v = reinterpret_cast<const uint4*>(buf)[i];
    it.k[0] = v.x; it.k[1] = v.y; it.k[2] = v.z; it.k[3] = v.w;
    it.id = reinterpret_cast<const uint32_t*>(buf + PipeSmem<S>::ids)[i];
  } else {
    const uint2* q = reinterpret_cast<const uint2*>(buf) + 3 * i;
    const uint2 a = q[0], b = q[1], c = q[2];
    it.k[0] = a.x; it.k[1] = a.y; it.k[2] = b.x; it.k[3] = b.y; it.k[4] = c.x; it.id = c.y;
  }
}

template <int S, int kWord>
__global__ void __launch_bounds__(Pipe<S>::kThreads, 1) k_onesweep_pipe(WsPtrs ws, int d) {
  using P = PipeSmem<S>;
  constexpr int T = P::T, NT = P::NT, NW = P::NW, R = P::kRows;
  extern __shared__ __align__(128) unsigned char sm[];
  uint16_t* inv = reinterpret_cast<uint16_t*>(sm + P::off_inv);       // [2][T]
  uint32_t* whist = reinterpret_cast<uint32_t*>(sm + P::off_whist);   // [NW][256]
  int32_t* goff = reinterpret_cast<int32_t*>(sm + P::off_goff);       // [2][256]
  uint32_t* tcnt = reinterpret_cast<uint32_t*>(sm + P::off_cnt);     // [256] tile digit counts
  uint32_t* tstart = tcnt + kRadix;                                   // [256] tile-local starts
  uint32_t* gbase = tstart + kRadix;                                  // [256] pass digit offsets
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + P::off_bar);       // [3]
  uint32_t* misc = reinterpret_cast<uint32_t*>(sm + P::off_misc);     // [0..2] tile ring, [4..11] scan

  const Plan* plan = ws.plan;
  if (plan->skip[d]) return;
  Control* ctrl = ws.ctrl;
  if (block_error(ctrl)) return;
  const uint32_t U = plan->U;
  const uint32_t ntiles = (U + T - 1) / T;
  const bool fromB = plan->src[d] != 0;
  const unsigned char* src = fromB ? ws.itemsB : ws.itemsA;
  unsigned char* dst = fromB ? ws.itemsA : ws.itemsB;
  const size_t area = (size_t)ws.tilesS * kRadix;
  uint32_t* lb = ws.lb_sort + (size_t)plan->area[d] * area;
  uint32_t* lb_next = ws.lb_sort + (size_t)(plan->area[d] ^ 1) * area;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const bool digit_thread = t < kRadix;
  if (digit_thread) gbase[t] = plan->base[d][t];
  const int shift = (d & 3) * 8;
  uint32_t* wh = whist + w * kRadix;

  if (t == 0) {
    for (int b = 0; b < 3; ++b) mbar_init(bar + b, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");  // barriers visible to the copy engine
    fence_proxy_async();
    for (int j = 0; j < 2; ++j) {
      const uint32_t tile = atomicAdd(&ctrl->ctr[1 + d], 1u);
      misc[j] = tile;
      if (tile < ntiles) load_tile<S>(sm + j * P::buf, src, ws.idoff, tile, U, bar + j);
    }
  }
  __syncthreads();

  uint32_t prev = 0xFFFFFFFFu;  // tile written out this iteration (its look-back is done)
  for (uint32_t k = 0;; ++k) {
    const uint32_t b = k % 3, pb = (k + 2) % 3;
    const uint32_t cur = misc[b];
    const bool has_cur = cur < ntiles, has_prev = prev != 0xFFFFFFFFu;
    if (!has_cur && !has_prev) break;
    unsigned char* cbuf = sm + b * P::buf;
    const int n = has_cur ? (int)min((uint32_t)T, U - cur * T) : 0;

    // 1. rank tile k straight from shared memory
    uint32_t dig[R], rank[R];
    if (has_cur) {
      wait_tile(bar + b, (k / 3) & 1u, ctrl);
#pragma unroll
      for (int i = lane; i < kRadix; i += 32) wh[i] = 0;
      __syncwarp();
      uint32_t grp[R];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int i = (w * R + r) * 32 + lane;
        const bool valid = i < n;
        dig[r] = valid ? (smem_word<S, kWord>(cbuf, i) >> shift) & 0xFFu : 0u;
        uint32_t peers = __ballot_sync(0xffffffffu, valid);
        if (!valid) peers = ~peers;
#pragma unroll
        for (int bit = 0; bit < kRadixBits; ++bit) {
          const bool one = (dig[r] >> bit) & 1u;
          const uint32_t vote = __ballot_sync(0xffffffffu, one);
          peers &= one ? vote : ~vote;
        }
        const uint32_t lt = peers & lanemask_lt();
        grp[r] = (uint32_t)(__ffs(peers) - 1) | ((uint32_t)__popc(lt) << 8);
        rank[r] = 0;
        if (valid && lt == 0) rank[r] = atomicAdd(wh + dig[r], (uint32_t)__popc(peers));
        __syncwarp();  // rows add to the counters in row order: stable ranks
      }
#pragma unroll
      for (int r = 0; r < R; ++r) rank[r] = __shfl_sync(0xffffffffu, rank[r], grp[r] & 31u) + (grp[r] >> 8);
    }
    __syncthreads();

    // 2. per-digit tile counts (published as the tile's aggregate) and local starts
    uint32_t cnt = 0;
    if (has_cur && digit_thread) {
#pragma unroll 8
      for (int q = 0; q < NW; ++q) cnt += whist[q * kRadix + t];
      tcnt[t] = cnt;
      st_relaxed(lb + (size_t)cur * kRadix + t, cur == 0 ? lb_pre(cnt) : lb_agg(cnt));
      lb_next[(size_t)cur * kRadix + t] = 0;  // the next non-trivial pass uses the other area
    }
    const uint32_t incl = warp_incl_scan(cnt);
    if (lane == 31 && digit_thread) misc[4 + w] = incl;
    __syncthreads();
    if (has_cur && digit_thread) {
      uint32_t ts = 0;
#pragma unroll
      for (int q = 0; q < kRadix / 32; ++q) ts += (q < w) ? misc[4 + q] : 0u;
      ts += incl - cnt;
      tstart[t] = ts;
      uint32_t run = ts;
#pragma unroll 8
      for (int q = 0; q < NW; ++q) {  // -> tile-local start of (warp q, digit t)
        const uint32_t c = whist[q * kRadix + t];
        whist[q * kRadix + t] = run;
        run += c;
      }
    }
    __syncthreads();

    // 3. inverse permutation of tile k; scatter of tile k-1
    if (has_cur) {
      uint16_t* cinv = inv + (k & 1) * T;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int i = (w * R + r) * 32 + lane;
        if (i < n) cinv[wh[dig[r]] + rank[r]] = (uint16_t)i;
      }
    }
    if (has_prev) {
      const unsigned char* pbuf = sm + pb * P::buf;
      const uint16_t* pinv = inv + ((k + 1) & 1) * T;
      const int32_t* pgoff = goff + ((k + 1) & 1) * kRadix;
      const int pn = (int)min((uint32_t)T, U - prev * T);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int i = r * NT + t;
        if (i < pn) {
          Item<S> o;
          smem_item<S>(pbuf, pinv[i], o);
          const uint32_t gpos = (uint32_t)(pgoff[(o.k[kWord] >> shift) & 0xFFu] + i);
          if (gpos < U)
            ItemIO<S>::store(dst, ws.idoff, (int64_t)gpos, o);
          else
            record_error(ctrl, kErrInternal);  // histogram/ranking inconsistency: never write out of range
        }
      }
    }
    __syncthreads();  // buffer pb, inv and goff of tile k-1 are free

    // 4. acquire tile k+2 and start its copy into the freed buffer
    if (t == 0) {
      const uint32_t tile = atomicAdd(&ctrl->ctr[1 + d], 1u);
      misc[pb] = tile;
      if (tile < ntiles) {
        fence_proxy_async();  // generic-proxy reads of buffer pb happen before the async write
        load_tile<S>(sm + pb * P::buf, src, ws.idoff, tile, U, bar + pb);
      }
    }

    // 5. look-back of tile k: warp w resolves digits w*DPW .. (w+1)*DPW-1 on the digit-major table
    if (has_cur) {
      constexpr int DPW = kRadix / NW;
      const uint32_t excl = cur > 0 ? warp_lookback_tiles<DPW>(lb, cur, w * DPW, ctrl) : 0u;
      if (lane < DPW) {
        const int dd = w * DPW + lane;
        if (cur > 0) st_relaxed(lb + (size_t)cur * kRadix + dd, lb_pre(excl + tcnt[dd]));
        goff[(k & 1) * kRadix + dd] = (int32_t)(gbase[dd] + excl) - (int32_t)tstart[dd];
      }
    }
    prev = has_cur ? cur : 0xFFFFFFFFu;
    __syncthreads();  // misc[pb], goff of tile k visible to every thread
  }
}

template <int S, int kWord>
static int occ_one() {
  cudaFuncSetAttribute(k_onesweep_pipe<S, kWord>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)PipeSmem<S>::bytes);
  int n = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_onesweep_pipe<S, kWord>, Pipe<S>::kThreads,
                                                PipeSmem<S>::bytes);
  return n;
}

template <int S>
static int occ() {
  int n = occ_one<S, 0>();
  if constexpr (S >= 8) n = min(n, occ_one<S, 1>());
  if constexpr (S >= 12) n = min(n, occ_one<S, 2>());
  if constexpr (S >= 16) n = min(n, occ_one<S, 3>());
  if constexpr (S >= 20) n = min(n, occ_one<S, 4>());
  return n;
}

int occupancy_sort_pipe(int S) {
  switch (S) {
    case 4: return occ<4>();
    case 8: return occ<8>();
    case 12: return occ<12>();
    case 16: return occ<16>();
    case 20: return occ<20>();
    default: return 0;  // 24- and 32-byte keys use the "tiles" sort only
  }
}

template <int S>
static void launch_s(int g, int digit, WsPtrs ws, cudaStream_t st) {
  const int word = S / 4 - 1 - (digit >> 2);  // word 0 is the most significant
  const size_t sm = PipeSmem<S>::bytes;
  constexpr int NT = Pipe<S>::kThreads;
  switch (word) {
    case 0: k_onesweep_pipe<S, 0><<<g, NT, sm, st>>>(ws, digit); break;
    case 1: if constexpr (S >= 8) k_onesweep_pipe<S, 1><<<g, NT, sm, st>>>(ws, digit); break;
    case 2: if constexpr (S >= 12) k_onesweep_pipe<S, 2><<<g, NT, sm, st>>>(ws, digit); break;
    case 3: if constexpr (S >= 16) k_onesweep_pipe<S, 3><<<g, NT, sm, st>>>(ws, digit); break;
    default: if constexpr (S >= 20) k_onesweep_pipe<S, 4><<<g, NT, sm, st>>>(ws, digit); break;
  }
}

cudaError_t launch_onesweep_pipe(int S, int digit, WsPtrs ws, const LaunchCfg& c, cudaStream_t st) {
  int64_t g = (int64_t)c.sms * c.occ_sort_pipe;
  if (g > ws.tilesS) g = ws.tilesS;
  if (g < 1) return cudaSuccess;
  switch (S) {
    case 4: launch_s<4>((int)g, digit, ws, st); break;
    case 8: launch_s<8>((int)g, digit, ws, st); break;
    case 12: launch_s<12>((int)g, digit, ws, st); break;
    case 16: launch_s<16>((int)g, digit, ws, st); break;
    case 20: launch_s<20>((int)g, digit, ws, st); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace reindex
