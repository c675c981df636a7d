// Streaming kernels of the re-indexing pipeline:
//   k_clear       zero the workspace tables that must start at zero
//   k_used_flags  Section 2.1: isUsed[idx[j]] = true, as one bit per vertex, with range check
//   k_sort_plan   exclusive digit offsets of the upfront histograms; which radix passes are
//                 trivial (digit constant over all items) and the buffer each pass reads
//   k_remap       Section 2.4: out_idx[j] = oldToNew[idx[j]]
//   k_finalize    propagate a device-detected error into *out_nVtx and the sticky word
#include <algorithm>
#include <cstring>

#include "internal.h"

namespace reindex {

// Device-wide sticky error (one per device context); see reindex_stream_status.
__device__ uint32_t g_sticky_err;
__device__ uint32_t g_sticky_out;

__global__ void __launch_bounds__(kThreads) k_clear(uint4* p, int64_t n16) {
  const uint4 z = make_uint4(0, 0, 0, 0);
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n16; i += (int64_t)gridDim.x * kThreads)
    p[i] = z;
}

__device__ __forceinline__ void mark_used(int32_t v, uint32_t nVtx, uint32_t* bitmask, bool& bad) {
  if ((uint32_t)v >= nVtx) {  // negative indices wrap to >= 2^31 > nVtx
    bad = true;
  } else {
    atomicOr(bitmask + ((uint32_t)v >> 5), 1u << ((uint32_t)v & 31u));  // result unused -> RED.OR
  }
}

// One bit per vertex, set by every index that references it (Section 2.1).  Indices are read
// with 128-bit loads when the array is 16-byte aligned, kBatch vectors per thread at a time so
// that enough loads are in flight.
constexpr int kBatch = 4;

template <bool kVec>
__global__ void __launch_bounds__(kThreads) k_used_flags(const int32_t* idx, int64_t M, uint32_t nVtx,
                                                          uint32_t* bitmask, Control* ctrl) {
  if (*(volatile const uint32_t*)&ctrl->err) return;  // skipped full-key sort (or an earlier error)
  bool bad = false;
  const int64_t t0 = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * kThreads;
  int64_t done = 0;
  if (kVec) {
    const int4* v4 = reinterpret_cast<const int4*>(idx);
    const int64_t n4 = M >> 2;
    for (int64_t i = t0; i < n4; i += stride * kBatch) {
      int4 q[kBatch];
#pragma unroll
      for (int b = 0; b < kBatch; ++b)
        if (i + b * stride < n4) q[b] = __ldcs(v4 + i + b * stride);
#pragma unroll
      for (int b = 0; b < kBatch; ++b) {
        if (i + b * stride < n4) {
          mark_used(q[b].x, nVtx, bitmask, bad);
          mark_used(q[b].y, nVtx, bitmask, bad);
          mark_used(q[b].z, nVtx, bitmask, bad);
          mark_used(q[b].w, nVtx, bitmask, bad);
        }
      }
    }
    done = n4 << 2;
  }
  for (int64_t i = done + t0; i < M; i += stride) mark_used(__ldcs(idx + i), nVtx, bitmask, bad);
  if (bad) record_error(ctrl, kErrIndexRange);
}

// The same for int64 indices: any value outside [0, nVtx) -- negative or past the vertex array,
// however large -- is an index-range error (no index is truncated to 32 bits).
__device__ __forceinline__ void mark_used64(int64_t v, uint32_t nVtx, uint32_t* bitmask, bool& bad) {
  if ((uint64_t)v >= (uint64_t)nVtx) {
    bad = true;
  } else {
    atomicOr(bitmask + ((uint32_t)v >> 5), 1u << ((uint32_t)v & 31u));
  }
}

template <bool kVec>
__global__ void __launch_bounds__(kThreads) k_used_flags64(const int64_t* idx, int64_t M, uint32_t nVtx,
                                                            uint32_t* bitmask, Control* ctrl) {
  if (*(volatile const uint32_t*)&ctrl->err) return;
  bool bad = false;
  const int64_t t0 = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * kThreads;
  int64_t done = 0;
  if (kVec) {  // 16-byte vectors of two indices, kBatch vectors in flight per thread
    const longlong2* v2 = reinterpret_cast<const longlong2*>(idx);
    const int64_t n2 = M >> 1;
    for (int64_t i = t0; i < n2; i += stride * kBatch) {
      longlong2 q[kBatch];
#pragma unroll
      for (int b = 0; b < kBatch; ++b)
        if (i + b * stride < n2) q[b] = __ldcs(v2 + i + b * stride);
#pragma unroll
      for (int b = 0; b < kBatch; ++b) {
        if (i + b * stride < n2) {
          mark_used64(q[b].x, nVtx, bitmask, bad);
          mark_used64(q[b].y, nVtx, bitmask, bad);
        }
      }
    }
    done = n2 << 1;
  }
  for (int64_t i = done + t0; i < M; i += stride) mark_used64(__ldcs(idx + i), nVtx, bitmask, bad);
  if (bad) record_error(ctrl, kErrIndexRange);
}

// Meshes of more than 2^31 - 1 vertices (int64 indices) are re-indexed in vertex ranges (see api.cu):
// k_used_flags_range64 sets the used bits of range [lo, lo + n) only, from all the indices (relative
// to lo); with `check` it also records indices outside [0, N) as an index-range error.
__global__ void __launch_bounds__(kThreads) k_used_flags_range64(const int64_t* __restrict__ idx, int64_t M,
                                                                  int64_t lo, int64_t n, int64_t N,
                                                                  uint32_t* bitmask, Control* ctrl, int check) {
  bool bad = false;
  const int64_t stride = (int64_t)gridDim.x * kThreads;
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < M; i += stride) {
    const int64_t v = __ldcs(idx + i);
    if ((uint64_t)v >= (uint64_t)N) {
      bad = true;
    } else if (v >= lo && v < lo + n) {
      const uint32_t r = (uint32_t)(v - lo);
      atomicOr(bitmask + (r >> 5), 1u << (r & 31u));
    }
  }
  if (bad && check) record_error(ctrl, kErrIndexRange);
}

// out[j] = j (the identity indices of the second level).
__global__ void __launch_bounds__(kThreads) k_iota(int32_t* out, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * kThreads;
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n; i += stride) out[i] = (int32_t)i;
}

// out[j] = map2[part_off[v >> shift] + rank[v]] for v = idx[j]: the vertex's rank among its range's
// unique vertices, then that range's unique vertex's final index (indices already range-checked).
__global__ void __launch_bounds__(kThreads) k_remap_two_level(const int64_t* __restrict__ idx,
                                                               int64_t* __restrict__ out, int64_t M,
                                                               const uint32_t* __restrict__ rank,
                                                               const int64_t* __restrict__ part_off,
                                                               const int32_t* __restrict__ map2, int shift) {
  const int64_t stride = (int64_t)gridDim.x * kThreads;
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < M; i += stride) {
    const int64_t v = __ldcs(idx + i);
    __stcs(out + i, (int64_t)__ldg(map2 + __ldg(part_off + (v >> shift)) + __ldg(rank + v)));
  }
}

// Digit offsets and pass plan (one CTA of 256 threads; thread t owns digit value t).
// The radix-sort plan for the P byte positions of a P-byte key.  With upfront histograms
// (onesweep sort): a byte is trivial if one value holds all U items; exclusive digit offsets from
// the histogram.  From the key bit masks (tiles sort, no histograms): if packing the varying bits
// (KeyPack) saves at least one pass, the passes sort the bytes of the packed key and the positions
// past its last byte are trivial; otherwise the raw bytes without a varying bit are trivial.
//
// Prefix sort (prefix_words = K > 0 words of key masks, P = 12): the packing keeps only the 64 most
// significant varying bits of the K-word key (the top part of a run that straddles the cut), so
// the items sort by an order-preserving 8-byte prefix of the packed key (digits 8-11 are zero).
//
// After a device-detected error (or in a skipped full-key sort) every pass is marked trivial.
// kor[q] / knand[q]: OR of key word q over the used vertices and of its complement.
__host__ __device__ void plan_prefix_pack(const uint32_t* kor, const uint32_t* knand, int K, KeyPack& kp,
                                          int& nbits) {
  uint8_t rw[kMaxPackRuns], rs[kMaxPackRuns], rl[kMaxPackRuns];  // most significant run first
  int n = 0, need = 8 * kPrefixBytes;
  for (int wd = 0; wd < K && need > 0 && n < kMaxPackRuns; ++wd) {
    const uint32_t m = kor[wd] & knand[wd];
    for (int b = 31; b >= 0 && need > 0 && n < kMaxPackRuns;) {
      if (!((m >> b) & 1u)) {
        --b;
        continue;
      }
      int e = b;
      while (e >= 0 && ((m >> e) & 1u)) --e;  // run = bits e+1 .. b
      int len = b - e, lo = e + 1;
      if (len > need) {  // keep the run's most significant bits
        lo = b - need + 1;
        len = need;
      }
      rw[n] = (uint8_t)wd;
      rs[n] = (uint8_t)lo;
      rl[n] = (uint8_t)len;
      ++n;
      need -= len;
      b = e;
    }
  }
  kp = KeyPack{};
  kp.on = 1;
  kp.simple = 1;
  int pos = 0;
  for (int i = n - 1; i >= 0; --i) {  // least significant first
    const int r = n - 1 - i;
    kp.word[r] = rw[i];
    kp.shift[r] = rs[i];
    kp.len[r] = rl[i];
    kp.pos[r] = (uint8_t)pos;
    pos += rl[i];
    if (kp.wlen[rw[i]]) kp.simple = 0;  // two runs in one word
    kp.wshift[rw[i]] = rs[i];
    kp.wlen[rw[i]] = rl[i];
  }
  kp.nruns = (uint8_t)n;
  kp.nbits = (uint8_t)pos;
  nbits = pos;
}

// dbits: digit width when the keys are packed (8; 6 or 7 for the chunk sort: digit d is then bits
// [d * dbits, (d + 1) * dbits) of the packed key); npass: the passes the host launches (>= P when
// digits are narrower than bytes).
__global__ void __launch_bounds__(kRadix) k_sort_plan(WsPtrs ws, int P, int from_masks, int allow_pack,
                                                      int prefix_words, int dbits, int npass) {
  __shared__ uint32_t s_warp[kRadix / 32];
  __shared__ uint32_t s_or[kRadix / 32], s_and[kRadix / 32];
  __shared__ int s_np;  // digits of the packed key, or -1 (keys not packed)
  __shared__ int s_b;   // digit width
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const uint32_t U = ws.ctrl->U;
  Plan* plan = ws.plan;
  const int K = P / 4;
  if (*(volatile const uint32_t*)&ws.ctrl->err != 0) {  // same value in every thread (written before launch)
    if (t < kMaxDigits) {
      plan->skip[t] = 1;
      plan->next[t] = -1;
    }
    if (t == 0) {
      plan->first = -1;
      plan->pack.on = 0;
      plan->U = 0;
      plan->dbits = 8;
    }
    return;
  }
  if (t == 0) {
    int np = -1, b = dbits;
    plan->pack.on = 0;
    if (prefix_words > 0) {
      KeyPack kp;
      int nbits = 0;
      plan_prefix_pack(ws.ctrl->kor, ws.ctrl->knand, prefix_words, kp, nbits);
      plan->pack = kp;
      np = (nbits + b - 1) / b;
    } else if (from_masks && allow_pack) {
      KeyPack kp{};
      int pos = 0, nraw = 0;
      bool fits = true;
      kp.simple = 1;
      for (int wd = K - 1; wd >= 0; --wd) {  // least significant word first
        const uint32_t m = ws.ctrl->kor[wd] & ws.ctrl->knand[wd];
        plan->kconst[wd] = ws.ctrl->kor[wd] & ~m;
        const int first_run = kp.nruns;
        for (int i = 0; i < 4; ++i) nraw += ((m >> (8 * i)) & 0xFFu) != 0;
        for (int b = 0; b < 32;) {  // runs of varying bits
          if (!((m >> b) & 1u)) {
            ++b;
            continue;
          }
          int e = b;
          while (e < 32 && ((m >> e) & 1u)) ++e;
          if (kp.nruns == kMaxPackRuns) {
            fits = false;
          } else {
            kp.word[kp.nruns] = (uint8_t)wd;
            kp.shift[kp.nruns] = (uint8_t)b;
            kp.len[kp.nruns] = (uint8_t)(e - b);
            kp.pos[kp.nruns] = (uint8_t)pos;
            ++kp.nruns;
          }
          pos += e - b;
          b = e;
        }
        const int runs_here = kp.nruns - first_run;
        if (runs_here > 1) kp.simple = 0;
        kp.wshift[wd] = runs_here == 1 ? kp.shift[first_run] : 0;
        kp.wlen[wd] = runs_here == 1 ? kp.len[first_run] : 0;
      }
      if (pos > 255) fits = false;  // run positions are bytes
      kp.nbits = (uint8_t)pos;
      const int packed = (pos + b - 1) / b;
      // packing when it saves at least one pass; always for digits narrower than bytes (else they
      // fall back to bytes of the unpacked key)
      if (allow_pack && fits && (b < 8 || packed < nraw)) {
        kp.on = 1;
        plan->pack = kp;
        np = packed;
      } else {
        b = 8;
      }
    } else {
      b = 8;
    }
    if (np > npass) {  // cannot happen for the pass counts the host launches; keep the passes exact
      np = -1;
      b = 8;
      plan->pack.on = 0;
    }
    s_np = np;
    s_b = b;
    plan->dbits = (uint8_t)b;
  }
  __syncthreads();
  const int np = s_np;
  const uint32_t nbits = np >= 0 ? plan->pack.nbits : 0u, b = (uint32_t)s_b;
  uint32_t sel = 0, q = 0;  // identical in every thread
  const int nloop = np >= 0 ? npass : P;  // byte digits of the unpacked key, or the packed key's digits
  for (int d = 0; d < nloop; ++d) {
    const uint32_t c = ws.hist[d * kRadix + t];
    // A digit whose value is the same for all U items: that pass is the identity.
    int trivial;
    uint32_t vary;  // digit bits that are not the same in every item
    if (from_masks && np >= 0) {
      trivial = d >= np;
      vary = trivial ? 0u : ((d == np - 1 && (nbits % b)) ? (1u << (nbits % b)) - 1u : (1u << b) - 1u);
      __syncthreads();
    } else if (from_masks) {
      const int q = P / 4 - 1 - (d >> 2);
      vary = ((ws.ctrl->kor[q] & ws.ctrl->knand[q]) >> ((d & 3) * 8)) & 0xFFu;
      trivial = vary == 0;
      __syncthreads();
    } else {
      // from the histogram: OR and AND over the digit values that occur
      const uint32_t o = __reduce_or_sync(0xffffffffu, c ? (uint32_t)t : 0u);
      const uint32_t a = __reduce_and_sync(0xffffffffu, c ? (uint32_t)t : 0xFFu);
      if (lane == 0) s_or[w] = o, s_and[w] = a;
      trivial = __syncthreads_or(c == U);
      uint32_t oo = 0, aa = 0xFFu;
      for (int k = 0; k < kRadix / 32; ++k) oo |= s_or[k], aa &= s_and[k];
      vary = (oo ^ aa) & 0xFFu;
      __syncthreads();  // s_or / s_and are rewritten for the next digit
    }
    const uint32_t incl = warp_incl_scan(c);
    if (lane == 31) s_warp[w] = incl;
    __syncthreads();
    uint32_t off = 0;
    for (int k = 0; k < w; ++k) off += s_warp[k];
    plan->base[d][t] = off + incl - c;
    __syncthreads();
    if (t == 0) {
      plan->skip[d] = (uint8_t)trivial;
      plan->src[d] = (uint8_t)sel;
      plan->area[d] = (uint8_t)(q & 1u);
      plan->vary[d] = (uint8_t)vary;
    }
    if (!trivial) {
      sel ^= 1u;
      ++q;
    }
  }
  if (t == 0) {
    for (int d = nloop; d < kMaxDigits; ++d) plan->skip[d] = 1;
    int nxt = -1;
    for (int d = kMaxDigits - 1; d >= 0; --d) {
      plan->next[d] = (int8_t)nxt;
      if (!plan->skip[d]) nxt = d;
    }
    plan->first = (int8_t)nxt;
    plan->U = allow_pack ? 0u : U;  // packing: the plan runs first and the compaction writes U
    plan->plane_first = allow_pack ? 1 : 0;
    plan->final_sel = sel;
  }
}

// out_idx[j] = oldToNew[idx[j]] (Section 2.4).  Safe in place: each slot is read and written
// by the same thread.  kBatch index vectors are loaded before their 4*kBatch gathers are issued.
template <bool kVec>
__global__ void __launch_bounds__(kThreads) k_remap(const int32_t* idx, int32_t* out, int64_t M,
                                                     const uint32_t* __restrict__ o2n, const Control* ctrl) {
  const uint32_t err = ctrl->err;
  if (err && err != kErrSkip) return;  // outputs are unspecified after a device-detected error
  const int64_t t0 = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * kThreads;
  int64_t done = 0;
  if (kVec) {
    const int4* in4 = reinterpret_cast<const int4*>(idx);
    int4* out4 = reinterpret_cast<int4*>(out);
    const int64_t n4 = M >> 2;
    for (int64_t i = t0; i < n4; i += stride * kBatch) {
      int4 q[kBatch];
#pragma unroll
      for (int b = 0; b < kBatch; ++b)
        if (i + b * stride < n4) q[b] = __ldcs(in4 + i + b * stride);
#pragma unroll
      for (int b = 0; b < kBatch; ++b) {
        if (i + b * stride < n4) {
          int4 r;
          r.x = (int32_t)__ldg(o2n + q[b].x);
          r.y = (int32_t)__ldg(o2n + q[b].y);
          r.z = (int32_t)__ldg(o2n + q[b].z);
          r.w = (int32_t)__ldg(o2n + q[b].w);
          q[b] = r;
        }
      }
#pragma unroll
      for (int b = 0; b < kBatch; ++b)
        if (i + b * stride < n4) __stcs(out4 + i + b * stride, q[b]);
    }
    done = n4 << 2;
  }
  for (int64_t i = done + t0; i < M; i += stride) out[i] = (int32_t)__ldg(o2n + idx[i]);
}

// out_idx[j] = oldToNew[idx[j]] for int64 indices (already range-checked by k_used_flags64).
template <bool kVec>
__global__ void __launch_bounds__(kThreads) k_remap64(const int64_t* idx, int64_t* out, int64_t M,
                                                       const uint32_t* __restrict__ o2n, const Control* ctrl) {
  const uint32_t err = ctrl->err;
  if (err && err != kErrSkip) return;  // outputs are unspecified after a device-detected error
  const int64_t t0 = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * kThreads;
  int64_t done = 0;
  if (kVec) {
    const longlong2* in2 = reinterpret_cast<const longlong2*>(idx);
    longlong2* out2 = reinterpret_cast<longlong2*>(out);
    const int64_t n2 = M >> 1;
    for (int64_t i = t0; i < n2; i += stride * kBatch) {
      longlong2 q[kBatch];
#pragma unroll
      for (int b = 0; b < kBatch; ++b)
        if (i + b * stride < n2) q[b] = __ldcs(in2 + i + b * stride);
#pragma unroll
      for (int b = 0; b < kBatch; ++b) {
        if (i + b * stride < n2) {
          q[b].x = (long long)__ldg(o2n + q[b].x);
          q[b].y = (long long)__ldg(o2n + q[b].y);
        }
      }
#pragma unroll
      for (int b = 0; b < kBatch; ++b)
        if (i + b * stride < n2) __stcs(out2 + i + b * stride, q[b]);
    }
    done = n2 << 1;
  }
  for (int64_t i = done + t0; i < M; i += stride) out[i] = (int64_t)__ldg(o2n + idx[i]);
}

// Subset of a mesh (Section 3.4): out[s*k + q] = idx[list[s]*k + q] for the selected elements.
__global__ void __launch_bounds__(kThreads) k_gather_elements(const int32_t* idx, int k, int64_t nElem,
                                                               const int32_t* list, int64_t nSel, int32_t* out,
                                                               Control* ctrl) {
  bool bad = false;
  const int64_t n = nSel * k;
  for (int64_t j = blockIdx.x * (int64_t)kThreads + threadIdx.x; j < n; j += (int64_t)gridDim.x * kThreads) {
    const int64_t s = j / k;
    const int32_t e = __ldg(list + s);
    if (e < 0 || (int64_t)e >= nElem) {
      bad = true;
      out[j] = 0;
    } else {
      out[j] = __ldg(idx + (int64_t)e * k + (j - s * k));
    }
  }
  if (bad) record_error(ctrl, kErrIndexRange);
}

__global__ void k_finalize(Control* ctrl, int64_t* out_nVtx) {
  const uint32_t e = ctrl->err;
  if (e && e != kErrSkip) {
    *out_nVtx = -(int64_t)e;
    atomicCAS(&g_sticky_err, 0u, e);
  }
}

__global__ void k_set_count(int64_t* out_nVtx, int64_t v) { *out_nVtx = v; }

__global__ void k_take_sticky() { g_sticky_out = atomicExch(&g_sticky_err, 0u); }

static int grid_for(int64_t work_items, const LaunchCfg& c, int per_sm) {
  int64_t g = (work_items + kThreads - 1) / kThreads;
  const int64_t cap = (int64_t)c.sms * per_sm;
  if (g > cap) g = cap;
  return g < 1 ? 1 : (int)g;
}

cudaError_t launch_clear(void* p, size_t bytes, const LaunchCfg& c, cudaStream_t st) {
  const int64_t n16 = (int64_t)(bytes / 16);
  if (n16 == 0) return cudaSuccess;
  k_clear<<<grid_for(n16, c, 8), kThreads, 0, st>>>(static_cast<uint4*>(p), n16);
  return cudaGetLastError();
}

cudaError_t launch_used_flags(const int32_t* idx, int64_t M, int64_t nVtx, WsPtrs ws, const LaunchCfg& c,
                              cudaStream_t st) {
  if (M == 0) return cudaSuccess;
  const bool vec = (reinterpret_cast<uintptr_t>(idx) & 15) == 0;
  const int g = grid_for(vec ? (M + 3) / 4 : M, c, 8);
  if (vec)
    k_used_flags<true><<<g, kThreads, 0, st>>>(idx, M, (uint32_t)nVtx, ws.bitmask, ws.ctrl);
  else
    k_used_flags<false><<<g, kThreads, 0, st>>>(idx, M, (uint32_t)nVtx, ws.bitmask, ws.ctrl);
  return cudaGetLastError();
}

cudaError_t launch_used_flags64(const int64_t* idx, int64_t M, int64_t nVtx, WsPtrs ws, const LaunchCfg& c,
                                cudaStream_t st) {
  if (M == 0) return cudaSuccess;
  const bool vec = (reinterpret_cast<uintptr_t>(idx) & 15) == 0;
  const int g = grid_for(vec ? (M + 1) / 2 : M, c, 8);
  if (vec)
    k_used_flags64<true><<<g, kThreads, 0, st>>>(idx, M, (uint32_t)nVtx, ws.bitmask, ws.ctrl);
  else
    k_used_flags64<false><<<g, kThreads, 0, st>>>(idx, M, (uint32_t)nVtx, ws.bitmask, ws.ctrl);
  return cudaGetLastError();
}

cudaError_t launch_used_flags_range64(const int64_t* idx, int64_t M, int64_t lo, int64_t n, int64_t N, WsPtrs ws,
                                      bool check, const LaunchCfg& c, cudaStream_t st) {
  if (M == 0) return cudaSuccess;
  k_used_flags_range64<<<grid_for(M, c, 8), kThreads, 0, st>>>(idx, M, lo, n, N, ws.bitmask, ws.ctrl, check ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_iota(int32_t* out, int64_t n, const LaunchCfg& c, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_iota<<<grid_for(n, c, 8), kThreads, 0, st>>>(out, n);
  return cudaGetLastError();
}

cudaError_t launch_remap_two_level(const int64_t* idx, int64_t* out, int64_t M, const uint32_t* rank,
                                   const int64_t* part_off, const int32_t* map2, int shift, const LaunchCfg& c,
                                   cudaStream_t st) {
  if (M == 0) return cudaSuccess;
  k_remap_two_level<<<grid_for(M, c, 8), kThreads, 0, st>>>(idx, out, M, rank, part_off, map2, shift);
  return cudaGetLastError();
}

int sort_passes(int keyBytes, int dbits) { return dbits >= 8 ? keyBytes : std::min(kMaxDigits, (8 * keyBytes + dbits - 1) / dbits); }

cudaError_t launch_sort_plan(int S, WsPtrs ws, bool from_masks, bool allow_pack, cudaStream_t st, int dbits) {
  k_sort_plan<<<1, kRadix, 0, st>>>(ws, S, from_masks ? 1 : 0, allow_pack ? 1 : 0, 0, dbits,
                                    sort_passes(S, dbits));
  return cudaGetLastError();
}

cudaError_t launch_prefix_plan(int S, WsPtrs ws, cudaStream_t st, int dbits) {
  k_sort_plan<<<1, kRadix, 0, st>>>(ws, kPrefixItem, 1, 1, S / 4, dbits, prefix_passes(dbits));
  return cudaGetLastError();
}

// The full-key sort of a prefix-sorted call runs only where the prefix sort found two different
// keys with one prefix; a device error of the prefix sort skips it and is reported by it.
__global__ void k_prefix_gate(const Control* pre, Control* full) {
  const uint32_t e = pre->err;
  if (e)
    full->err = e;
  else if (!pre->amb)
    full->err = kErrSkip;
}

cudaError_t launch_prefix_gate(WsPtrs pre, WsPtrs full, cudaStream_t st) {
  k_prefix_gate<<<1, 1, 0, st>>>(pre.ctrl, full.ctrl);
  return cudaGetLastError();
}

cudaError_t launch_remap(const int32_t* idx, int32_t* out_idx, int64_t M, WsPtrs ws, const LaunchCfg& c,
                         cudaStream_t st) {
  if (M == 0) return cudaSuccess;
  const bool vec = ((reinterpret_cast<uintptr_t>(idx) | reinterpret_cast<uintptr_t>(out_idx)) & 15) == 0;
  const int g = grid_for(vec ? (M + 3) / 4 : M, c, 8);
  if (vec)
    k_remap<true><<<g, kThreads, 0, st>>>(idx, out_idx, M, ws.old2new, ws.ctrl);
  else
    k_remap<false><<<g, kThreads, 0, st>>>(idx, out_idx, M, ws.old2new, ws.ctrl);
  return cudaGetLastError();
}

cudaError_t launch_remap64(const int64_t* idx, int64_t* out_idx, int64_t M, WsPtrs ws, const LaunchCfg& c,
                           cudaStream_t st) {
  if (M == 0) return cudaSuccess;
  const bool vec = ((reinterpret_cast<uintptr_t>(idx) | reinterpret_cast<uintptr_t>(out_idx)) & 15) == 0;
  const int g = grid_for(vec ? (M + 1) / 2 : M, c, 8);
  if (vec)
    k_remap64<true><<<g, kThreads, 0, st>>>(idx, out_idx, M, ws.old2new, ws.ctrl);
  else
    k_remap64<false><<<g, kThreads, 0, st>>>(idx, out_idx, M, ws.old2new, ws.ctrl);
  return cudaGetLastError();
}

cudaError_t launch_gather_elements(const int32_t* idx, int k, int64_t nElem, const int32_t* list, int64_t nSel,
                                  int32_t* out, WsPtrs ws, const LaunchCfg& c, cudaStream_t st) {
  if (nSel == 0) return cudaSuccess;
  k_gather_elements<<<grid_for(nSel * k, c, 8), kThreads, 0, st>>>(idx, k, nElem, list, nSel, out, ws.ctrl);
  return cudaGetLastError();
}

cudaError_t launch_finalize(WsPtrs ws, int64_t* out_nVtx, cudaStream_t st) {
  k_finalize<<<1, 1, 0, st>>>(ws.ctrl, out_nVtx);
  return cudaGetLastError();
}

cudaError_t launch_set_count(int64_t* out_nVtx, int64_t value, cudaStream_t st) {
  k_set_count<<<1, 1, 0, st>>>(out_nVtx, value);
  return cudaGetLastError();
}

cudaError_t read_and_clear_sticky(uint32_t* value, cudaStream_t st) {
  k_take_sticky<<<1, 1, 0, st>>>();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = cudaMemcpyFromSymbolAsync(value, g_sticky_out, sizeof(uint32_t), 0, cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(st);
}

}  // namespace reindex

// Host test hook (include/reindex.h): the prefix sort's packing for given key masks.
extern "C" int reindex_debug_prefix_pack(const uint32_t* kor, const uint32_t* knand, int K, void* out, int outBytes) {
  using namespace reindex;
  if (K < 1 || K > kMaxKeyWords || !kor || !knand || !out || outBytes < (int)sizeof(KeyPack)) return -1;
  KeyPack kp;
  int nbits = 0;
  plan_prefix_pack(kor, knand, K, kp, nbits);
  std::memcpy(out, &kp, sizeof(KeyPack));
  return nbits;
}

// Host test hook (include/reindex.h): the key packing arithmetic of the compaction and the head
// scan (the same inline functions the kernels use) applied to n keys of K words on the host.
namespace {
template <int K>
void debug_pack_k(const reindex::KeyPack& P, const uint32_t* kconst, const uint32_t* keys, int64_t n, int mode,
                  uint32_t* out) {
  using namespace reindex;
  for (int64_t i = 0; i < n; ++i) {
    uint32_t k[K];
    for (int q = 0; q < K; ++q) k[q] = keys[i * K + q];
    if (mode == 3) {
      out[i] = unpacked_word0<K>(k, P, kconst[0]);
      continue;
    }
    if (mode == 0)
      pack_key<K>(k, P);
    else if (mode == 1)
      pack_key_simple<K>(k, P);
    else
      unpack_key<K>(k, P, kconst);
    for (int q = 0; q < K; ++q) out[i * K + q] = k[q];
  }
}
}  // namespace

extern "C" int reindex_debug_pack_keys(const void* pack, int packBytes, int K, const uint32_t* kconst,
                                       const uint32_t* keys, int64_t n, int mode, uint32_t* out) {
  using namespace reindex;
  if (!pack || packBytes < (int)sizeof(KeyPack) || K < 1 || K > kMaxKeyWords || n < 0 || mode < 0 || mode > 3 ||
      (n > 0 && (!keys || !out)) || ((mode >= 2) && !kconst))
    return -1;
  KeyPack P;
  std::memcpy(&P, pack, sizeof(KeyPack));
  if (P.nruns > kMaxPackRuns) return -1;
  switch (K) {
    case 1: debug_pack_k<1>(P, kconst, keys, n, mode, out); break;
    case 2: debug_pack_k<2>(P, kconst, keys, n, mode, out); break;
    case 3: debug_pack_k<3>(P, kconst, keys, n, mode, out); break;
    case 4: debug_pack_k<4>(P, kconst, keys, n, mode, out); break;
    case 5: debug_pack_k<5>(P, kconst, keys, n, mode, out); break;
    case 6: debug_pack_k<6>(P, kconst, keys, n, mode, out); break;
    case 7: debug_pack_k<7>(P, kconst, keys, n, mode, out); break;
    case 8: debug_pack_k<8>(P, kconst, keys, n, mode, out); break;
    case 12: debug_pack_k<12>(P, kconst, keys, n, mode, out); break;
    case 16: debug_pack_k<16>(P, kconst, keys, n, mode, out); break;
    default: return -1;  // key sizes the library does not use
  }
  return 0;
}
