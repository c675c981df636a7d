// One pass of the LSD radix sort of (key, old index) items on one 8-bit digit (Section 2.2's
// key-value sort), in the single-pass "onesweep" form: the global digit offsets come from the
// upfront histograms (k_compact + k_sort_plan), and each tile's offset within a digit from a
// decoupled look-back over per-tile digit counts, so every item is read and written once per pass.
//
// Per tile of 4096 items (512 threads x 8 items, warp-striped so loads are coalesced):
//   1. load items;
//   2. rank digits inside each warp: find the lanes holding the same digit (8 ballots, one per
//      digit bit, or one match.any), the group's lowest lane adds the group size to the warp's
//      shared-memory counter for that digit and broadcasts the old value (stable: row-major,
//      lane order);
//   3. per-digit tile counts; publish them (aggregate) and load the preceding tile's status;
//      tile-local digit starts and per-(warp, digit) offsets;
//   4. stage the items in shared memory in digit order while that load is in flight, then walk
//      back (one earlier tile per step) to the nearest inclusive prefix and publish this tile's;
//   5. write the items out so that consecutive threads write consecutive addresses of one run.
// The pass is stable, so the composition of passes sorts by the whole key (ties keep vertex order).
// A pass whose digit is constant over all items is skipped (it would be the identity).
#include "internal.h"
#include "radix.cuh"

namespace reindex {

// 20-byte items need more registers and shared memory: one CTA per SM.
template <int S, int kWord, int kMode>
__global__ void __launch_bounds__(kSortThreads, S >= 20 ? 1 : 2) k_onesweep(WsPtrs ws, int d) {
  constexpr int K = S / 4;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  unsigned char* stage = sm_raw;                                               // tile in digit order
  uint32_t* whist = reinterpret_cast<uint32_t*>(sm_raw + SortSmem<S>::stage);  // [warps][256]
  int32_t* goff = reinterpret_cast<int32_t*>(whist + kSortWarps * kRadix);     // [256] global - local pos
  uint32_t* gbase = reinterpret_cast<uint32_t*>(goff + kRadix);                // [256] pass digit offsets
  uint32_t* s_misc = gbase + kRadix;                                           // [32]

  const Plan* plan = ws.plan;
  if (plan->skip[d]) return;
  Control* ctrl = ws.ctrl;
  if (block_error(ctrl)) return;
  const uint32_t U = plan->U;
  const uint32_t ntiles = (U + kSortTile - 1) / kSortTile;
  const bool fromB = plan->src[d] != 0;
  const unsigned char* src = fromB ? ws.itemsB : ws.itemsA;
  unsigned char* dst = fromB ? ws.itemsA : ws.itemsB;
  const size_t area = (size_t)ws.tilesS * kRadix;
  uint32_t* lb = ws.lb_sort + (size_t)plan->area[d] * area;
  uint32_t* lb_next = ws.lb_sort + (size_t)(plan->area[d] ^ 1) * area;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const bool digit_thread = t < kRadix;  // threads 0..255 own digit value t
  if (digit_thread) gbase[t] = plan->base[d][t];
  const int shift = (d & 3) * 8;
  const uint32_t vary = plan->vary[d];
  uint32_t* wh = whist + w * kRadix;
  const int wbase = w * 32 * kSortIpt;

  for (;;) {
    if (t == 0) s_misc[0] = atomicAdd(&ctrl->ctr[1 + d], 1u);
    __syncthreads();
    const uint32_t tile = s_misc[0];
    if (tile >= ntiles) break;
    const uint32_t base = tile * kSortTile;
    const int n = (int)min((uint32_t)kSortTile, U - base);

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

    // 2. warp-level ranking
    uint32_t rank[kSortIpt / 2];  // two 16-bit ranks per register (ranks < 4096)
#pragma unroll
    for (int r = 0; r < kSortIpt; ++r) {
      const bool valid = wbase + r * 32 + lane < n;
      const uint32_t dig = (it[r].k[kWord] >> shift) & 0xFFu;
      const uint32_t peers = match_digit<kMode>(dig, valid, vary);
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

    // 3. per-digit tile count, aggregate publication, first look-back load, local digit start
    uint32_t cnt = 0, s_prev = lb_pre(0);
    if (digit_thread) {
#pragma unroll
      for (int q = 0; q < kSortWarps; ++q) cnt += whist[q * kRadix + t];
      st_relaxed(lb + (size_t)tile * kRadix + t, tile == 0 ? lb_pre(cnt) : lb_agg(cnt));
      lb_next[(size_t)tile * kRadix + t] = 0;  // the next non-trivial pass uses the other area
      if (tile > 0) s_prev = ld_relaxed(lb + (size_t)(tile - 1) * kRadix + t);  // consumed after staging
    }
    const uint32_t incl = warp_incl_scan(cnt);
    if (lane == 31 && digit_thread) s_misc[1 + w] = incl;
    __syncthreads();
    uint32_t ts = 0;
    if (digit_thread) {
#pragma unroll
      for (int q = 0; q < kRadix / 32; ++q) ts += (q < w) ? s_misc[1 + q] : 0u;
      ts += incl - cnt;  // tile-local start of digit t
      uint32_t run = ts;
#pragma unroll
      for (int q = 0; q < kSortWarps; ++q) {  // -> tile-local start of (warp q, digit t)
        const uint32_t c = whist[q * kRadix + t];
        whist[q * kRadix + t] = run;
        run += c;
      }
    }
    __syncthreads();

    // 4. stage in digit order (the first look-back load is in flight meanwhile), then walk back
#pragma unroll
    for (int r = 0; r < kSortIpt; ++r) {
      if (wbase + r * 32 + lane < n) {
        const uint32_t dig = (it[r].k[kWord] >> shift) & 0xFFu;
        const uint32_t rk = (rank[r >> 1] >> ((r & 1) * 16)) & 0xFFFFu;
        Stage<S>::put(stage, (int)(wh[dig] + rk), it[r]);
      }
    }
    if (digit_thread) {
      uint32_t excl = 0;
      if (tile > 0) {
        uint32_t s = s_prev;
        if (!lb_ready(s)) s = wait_status(lb + (size_t)(tile - 1) * kRadix + t, ctrl);
        excl = lb_val(s);
        for (int64_t q = (int64_t)tile - 2; !lb_is_pre(s); --q) {
          s = wait_status(lb + (size_t)q * kRadix + t, ctrl);
          excl += lb_val(s);
        }
        st_relaxed(lb + (size_t)tile * kRadix + t, lb_pre(excl + cnt));
      }
      goff[t] = (int32_t)(gbase[t] + excl) - (int32_t)ts;
    }
    __syncthreads();

    // 5. coalesced scatter
#pragma unroll
    for (int r = 0; r < kSortIpt; ++r) {
      const int i = r * kSortThreads + t;
      if (i < n) {
        Item<S> o;
        Stage<S>::get(stage, i, o);
        const uint32_t gpos = (uint32_t)(goff[(o.k[kWord] >> shift) & 0xFFu] + i);
        if (gpos < U)
          ItemIO<S>::store(dst, ws.idoff, (int64_t)gpos, o);
        else
          record_error(ctrl, kErrInternal);  // histogram/ranking inconsistency: never write out of range
      }
    }
    __syncthreads();
  }
}

template <int S, int kWord, int kMode>
static int occ_one() {
  cudaFuncSetAttribute(k_onesweep<S, kWord, kMode>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)SortSmem<S>::bytes);
  int n = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_onesweep<S, kWord, kMode>, kSortThreads,
                                                SortSmem<S>::bytes);
  return n < 1 ? 1 : n;
}

template <int S, int kMode>
static int occ_mode() {
  int n = occ_one<S, 0, kMode>();
  if constexpr (S >= 8) n = min(n, occ_one<S, 1, kMode>());
  if constexpr (S >= 12) n = min(n, occ_one<S, 2, kMode>());
  if constexpr (S >= 16) n = min(n, occ_one<S, 3, kMode>());
  if constexpr (S >= 20) n = min(n, occ_one<S, 4, kMode>());
  return n;
}

template <int S>
static int occ() {
  return min(occ_mode<S, kRankBallot>(), occ_mode<S, kRankMatchAny>());
}

int occupancy_sort(int S) {
  switch (S) {
    case 4: return occ<4>();
    case 8: return occ<8>();
    case 12: return occ<12>();
    case 16: return occ<16>();
    case 20: return occ<20>();
    default: return 1;  // 24- and 32-byte keys use the "tiles" sort only
  }
}

template <int S, int kMode>
static void launch_mode(int g, int digit, WsPtrs ws, cudaStream_t st) {
  const int word = S / 4 - 1 - (digit >> 2);  // word 0 is the most significant
  switch (word) {
    case 0: k_onesweep<S, 0, kMode><<<g, kSortThreads, SortSmem<S>::bytes, st>>>(ws, digit); break;
    case 1: if constexpr (S >= 8) k_onesweep<S, 1, kMode><<<g, kSortThreads, SortSmem<S>::bytes, st>>>(ws, digit); break;
    case 2: if constexpr (S >= 12) k_onesweep<S, 2, kMode><<<g, kSortThreads, SortSmem<S>::bytes, st>>>(ws, digit); break;
    case 3: if constexpr (S >= 16) k_onesweep<S, 3, kMode><<<g, kSortThreads, SortSmem<S>::bytes, st>>>(ws, digit); break;
    default: if constexpr (S >= 20) k_onesweep<S, 4, kMode><<<g, kSortThreads, SortSmem<S>::bytes, st>>>(ws, digit); break;
  }
}

template <int S>
static void launch_s(int g, int digit, WsPtrs ws, int mode, cudaStream_t st) {
  if (mode == kRankMatchAny)
    launch_mode<S, kRankMatchAny>(g, digit, ws, st);
  else
    launch_mode<S, kRankBallot>(g, digit, ws, st);
}

cudaError_t launch_onesweep(int S, int digit, WsPtrs ws, const LaunchCfg& c, cudaStream_t st) {
  int64_t g = c.grid_per_tile ? (ws.Umax + kSortTile - 1) / kSortTile : (int64_t)c.sms * c.occ_sort;
  if (g > ws.tilesS) g = ws.tilesS;
  if (g < 1) return cudaSuccess;
  switch (S) {
    case 4: launch_s<4>((int)g, digit, ws, c.rank_mode, st); break;
    case 8: launch_s<8>((int)g, digit, ws, c.rank_mode, st); break;
    case 12: launch_s<12>((int)g, digit, ws, c.rank_mode, st); break;
    case 16: launch_s<16>((int)g, digit, ws, c.rank_mode, st); break;
    case 20: launch_s<20>((int)g, digit, ws, c.rank_mode, st); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace reindex
