// One pass of the LSD radix sort of (key, old index) items on one 8-bit digit (Section 2.2's
// key-value sort), in the single-pass "onesweep" form: the global digit offsets come from the
// upfront histograms (k_compact + k_sort_plan), and each tile's offset within a digit from a
// decoupled look-back over per-tile digit counts, so every item is read and written once per pass.
//
// Per tile of 4096 items (256 threads x 16 items, warp-striped so loads are coalesced):
//   1. load items; 2. rank digits inside each warp with __match_any_sync (stable: row-major,
//   lane order); 3. per-digit tile counts and warp offsets; publish the counts (aggregate) and
//   look back for each digit's exclusive prefix over earlier tiles, then publish the inclusive
//   prefix; 4. stage the items in shared memory in digit order; 5. write them out so that
//   consecutive threads write consecutive addresses of the same digit run.
// The pass is stable, so the composition of passes sorts by the whole key (ties keep vertex order).
// A pass whose digit is constant over all items is skipped (it would be the identity).
#include "internal.h"

namespace reindex {

template <int S>
struct SortSmem {
  static constexpr int K = S / 4;
  static constexpr size_t planes = (size_t)(K + 1) * kSortTile * 4;
  static constexpr size_t whist = (size_t)kWarps * kRadix * 4;
  static constexpr size_t bytes = planes + whist + 2 * kRadix * 4 + 16 * 4;
};

template <int S>
__global__ void __launch_bounds__(kThreads, 2) k_onesweep(WsPtrs ws, int d) {
  constexpr int K = S / 4;
  extern __shared__ __align__(16) uint32_t sm[];
  uint32_t* planes = sm;                                   // [K+1][kSortTile]
  uint32_t* whist = planes + (K + 1) * kSortTile;          // [kWarps][256]
  uint32_t* tstart = whist + kWarps * kRadix;              // [256] digit start inside the tile
  int32_t* goff = reinterpret_cast<int32_t*>(tstart + kRadix);  // [256] global pos - local pos
  uint32_t* s_misc = reinterpret_cast<uint32_t*>(goff + kRadix);  // [16]

  const Plan* plan = ws.plan;
  if (plan->skip[d]) return;
  Control* ctrl = ws.ctrl;
  if (block_error(ctrl)) return;
  const uint32_t U = plan->U;
  const int64_t ntiles = ((int64_t)U + kSortTile - 1) / kSortTile;
  const bool fromB = plan->src[d] != 0;
  const unsigned char* src = fromB ? ws.itemsB : ws.itemsA;
  unsigned char* dst = fromB ? ws.itemsA : ws.itemsB;
  const size_t area = (size_t)ws.tilesS * kRadix;
  uint32_t* lb = ws.lb_sort + (size_t)plan->area[d] * area;
  uint32_t* lb_next = ws.lb_sort + (size_t)(plan->area[d] ^ 1) * area;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const uint32_t gbase = plan->base[d][t];  // thread t owns digit value t

  for (;;) {
    if (t == 0) s_misc[0] = atomicAdd(&ctrl->ctr[1 + d], 1u);
    __syncthreads();
    const int64_t tile = s_misc[0];
    if (tile >= ntiles) break;
    const int64_t base = tile * kSortTile;
    const int n = (int)min((int64_t)kSortTile, (int64_t)U - base);

    // 1. load (warp-striped)
    Item<S> it[kSortIpt];
#pragma unroll
    for (int r = 0; r < kSortIpt; ++r) {
      const int local = w * 32 * kSortIpt + r * 32 + lane;
      if (local < n) ItemIO<S>::load(src, ws.Umax, base + local, it[r]);
    }
    uint32_t* wh = whist + w * kRadix;
#pragma unroll
    for (int i = lane; i < kRadix; i += 32) wh[i] = 0;
    __syncwarp();

    // 2. warp-level ranking
    uint32_t rank[kSortIpt];
#pragma unroll
    for (int r = 0; r < kSortIpt; ++r) {
      const int local = w * 32 * kSortIpt + r * 32 + lane;
      const bool valid = local < n;
      const uint32_t dig = valid ? key_digit<K>(it[r].k, d) : (uint32_t)kRadix;
      const uint32_t peers = __match_any_sync(0xffffffffu, dig);
      const uint32_t lt = peers & lanemask_lt();
      const uint32_t pre = valid ? wh[dig] : 0u;
      __syncwarp();
      if (valid && lt == 0) wh[dig] = pre + __popc(peers);
      __syncwarp();
      rank[r] = pre + __popc(lt);
    }
    __syncthreads();

    // 3. per-digit tile count (thread t = digit t), warp offsets, aggregate publication
    uint32_t cnt = 0;
#pragma unroll
    for (int q = 0; q < kWarps; ++q) {
      const uint32_t c = whist[q * kRadix + t];
      whist[q * kRadix + t] = cnt;
      cnt += c;
    }
    uint32_t* my = lb + tile * kRadix + t;
    st_relaxed(my, (tile == 0 ? kFlagPre : kFlagAgg) | cnt);
    lb_next[tile * kRadix + t] = 0;  // the next non-trivial pass uses the other area
    const uint32_t incl = warp_incl_scan(cnt);
    if (lane == 31) s_misc[1 + w] = incl;
    __syncthreads();
    uint32_t woff = 0;
#pragma unroll
    for (int q = 0; q < kWarps; ++q) woff += (q < w) ? s_misc[1 + q] : 0u;
    const uint32_t ts = woff + incl - cnt;
    tstart[t] = ts;
    uint32_t excl = 0;
    if (tile > 0) {
      for (int64_t k = tile - 1;; --k) {
        const uint32_t s = wait_status(lb + k * kRadix + t, ctrl);
        excl += s & kValMask;
        if ((s & kFlagMask) == kFlagPre) break;
      }
      st_relaxed(my, kFlagPre | ((excl + cnt) & kValMask));
    }
    goff[t] = (int32_t)(gbase + excl) - (int32_t)ts;
    __syncthreads();

    // 4. stage in digit order
#pragma unroll
    for (int r = 0; r < kSortIpt; ++r) {
      const int local = w * 32 * kSortIpt + r * 32 + lane;
      if (local < n) {
        const uint32_t dig = key_digit<K>(it[r].k, d);
        const uint32_t p = tstart[dig] + wh[dig] + rank[r];
#pragma unroll
        for (int q = 0; q < K; ++q) planes[q * kSortTile + p] = it[r].k[q];
        planes[K * kSortTile + p] = it[r].id;
      }
    }
    __syncthreads();

    // 5. coalesced scatter
#pragma unroll
    for (int r = 0; r < kSortIpt; ++r) {
      const int i = r * kThreads + t;
      if (i < n) {
        Item<S> o;
#pragma unroll
        for (int q = 0; q < K; ++q) o.k[q] = planes[q * kSortTile + i];
        o.id = planes[K * kSortTile + i];
        const uint32_t dig = key_digit<K>(o.k, d);
        const int64_t gpos = (int64_t)goff[dig] + i;
        if (gpos >= 0 && gpos < (int64_t)U)
          ItemIO<S>::store(dst, ws.Umax, gpos, o);
        else
          record_error(ctrl, kErrInternal);  // histogram/ranking inconsistency: never write out of range
      }
    }
    __syncthreads();
  }
}

template <int S>
static int occ() {
  cudaFuncSetAttribute(k_onesweep<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SortSmem<S>::bytes);
  int n = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_onesweep<S>, kThreads, SortSmem<S>::bytes);
  return n < 1 ? 1 : n;
}

int occupancy_sort(int S) {
  switch (S) {
    case 4: return occ<4>();
    case 8: return occ<8>();
    case 12: return occ<12>();
    default: return occ<16>();
  }
}

cudaError_t launch_onesweep(int S, int digit, WsPtrs ws, const LaunchCfg& c, cudaStream_t st) {
  int64_t g = (int64_t)c.sms * c.occ_sort;
  if (g > ws.tilesS) g = ws.tilesS;
  if (g < 1) return cudaSuccess;
  switch (S) {
    case 4: k_onesweep<4><<<(int)g, kThreads, SortSmem<4>::bytes, st>>>(ws, digit); break;
    case 8: k_onesweep<8><<<(int)g, kThreads, SortSmem<8>::bytes, st>>>(ws, digit); break;
    case 12: k_onesweep<12><<<(int)g, kThreads, SortSmem<12>::bytes, st>>>(ws, digit); break;
    default: k_onesweep<16><<<(int)g, kThreads, SortSmem<16>::bytes, st>>>(ws, digit); break;
  }
  return cudaGetLastError();
}

}  // namespace reindex
