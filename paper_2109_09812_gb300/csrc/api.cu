// C ABI of the re-indexing library (include/reindex.h): argument checks, workspace layout,
// the launch sequence of the pipeline, the pool-allocating and host-buffer variants, the
// sticky error query and the per-launch timing facility.
#include <atomic>
#include <cstdlib>
#include <algorithm>
#include <cstring>
#include <functional>
#include <string>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "reindex.h"
#include "internal.h"

namespace reindex {

// ---------------------------------------------------------------------------------------------
// Per-device launch configuration.
static std::mutex g_cfg_mu;
static std::map<std::pair<int, int>, LaunchCfg> g_cfg;

// Applies "sort=regs|pipe|tiles|chunk|auto,rank=ballot|match|vary,hist=uniform|peel|match,grid=persist|tile,
// swaves=tile|1|4,pack=auto|on|off,prefix=auto|on|off,chunk=big|small|wide|deep,cocc=max|1|2,cgrid=N,
// dbits=6|7|8,dedup=hash|off,dpub=on|off" (any subset, in any order).  Every variant computes the same
// result.
void apply_tuning(LaunchCfg& c, const char* spec) {
  if (!spec) return;
  if (std::strstr(spec, "grid=tile")) c.grid_per_tile = 1;
  if (std::strstr(spec, "grid=persist")) c.grid_per_tile = 0;
  if (std::strstr(spec, "sort=regs")) c.sort_kernel = kSortRegs;
  if (std::strstr(spec, "sort=pipe") && c.occ_sort_pipe > 0) c.sort_kernel = kSortPipe;
  if (std::strstr(spec, "sort=tiles")) c.sort_kernel = kSortTiles;
  if (std::strstr(spec, "sort=auto")) c.sort_kernel = kSortAuto;
  if (std::strstr(spec, "sort=chunk")) c.sort_kernel = kSortChunk;
  if (std::strstr(spec, "chunk=big")) c.chunk_cfg = 0;
  if (std::strstr(spec, "chunk=small")) c.chunk_cfg = 1;
  if (std::strstr(spec, "chunk=wide")) c.chunk_cfg = 2;
  if (std::strstr(spec, "chunk=deep")) c.chunk_cfg = 3;
  if (std::strstr(spec, "cocc=max")) c.chunk_occ = 0;
  if (std::strstr(spec, "cocc=1")) c.chunk_occ = 1;
  if (std::strstr(spec, "cocc=2")) c.chunk_occ = 2;
  if (const char* g = std::strstr(spec, "cgrid=")) c.chunk_grid_cap = std::atoi(g + 6);
  if (const char* g = std::strstr(spec, "dbits=")) {
    const int b = std::atoi(g + 6);
    if (b >= 6 && b <= 8) c.digit_bits = b;
  }
  if (std::strstr(spec, "dedup=hash")) c.dedup = 1;
  if (std::strstr(spec, "dedup=off")) c.dedup = 0;
  if (std::strstr(spec, "dpub=on")) c.dedup_pub = 1;
  if (std::strstr(spec, "dpub=off")) c.dedup_pub = 0;
  if (std::strstr(spec, "rank=match")) c.rank_mode = kRankMatchAny;
  if (std::strstr(spec, "rank=ballot")) c.rank_mode = kRankBallot;
  if (std::strstr(spec, "rank=vary")) c.rank_mode = kRankBallotVary;
  if (std::strstr(spec, "hist=uniform")) c.hist_mode = kHistUniform;
  if (std::strstr(spec, "hist=peel")) c.hist_mode = kHistPeel;
  if (std::strstr(spec, "hist=match")) c.hist_mode = kHistMatchAny;
  if (std::strstr(spec, "swaves=tile")) c.scatter_waves = 0;
  if (std::strstr(spec, "swaves=1")) c.scatter_waves = 1;
  if (std::strstr(spec, "swaves=4")) c.scatter_waves = 4;
  if (std::strstr(spec, "pack=on")) c.pack_keys = 1;
  if (std::strstr(spec, "pack=off")) c.pack_keys = 0;
  if (std::strstr(spec, "pack=auto")) c.pack_keys = -1;
  if (std::strstr(spec, "prefix=on")) c.prefix = 1;
  if (std::strstr(spec, "prefix=off")) c.prefix = 0;
  if (std::strstr(spec, "prefix=auto")) c.prefix = -1;
}

std::string describe_tuning(const LaunchCfg& c) {
  const char* sorts[] = {"sort=regs", "sort=pipe", "sort=tiles", "sort=auto", "sort=chunk"};
  std::string d = sorts[c.sort_kernel];
  d += c.rank_mode == kRankMatchAny ? ",rank=match" : (c.rank_mode == kRankBallotVary ? ",rank=vary" : ",rank=ballot");
  d += c.hist_mode == kHistMatchAny ? ",hist=match" : (c.hist_mode == kHistPeel ? ",hist=peel" : ",hist=uniform");
  d += c.grid_per_tile ? ",grid=tile" : ",grid=persist";
  d += c.scatter_waves ? ",swaves=" + std::to_string(c.scatter_waves) : std::string(",swaves=tile");
  d += c.pack_keys < 0 ? ",pack=auto" : (c.pack_keys ? ",pack=on" : ",pack=off");
  d += c.prefix < 0 ? ",prefix=auto" : (c.prefix ? ",prefix=on" : ",prefix=off");
  const char* shapes[] = {",chunk=big", ",chunk=small", ",chunk=wide", ",chunk=deep"};
  d += shapes[c.chunk_cfg & 3];
  d += c.chunk_occ ? ",cocc=" + std::to_string(c.chunk_occ) : std::string(",cocc=max");
  d += ",cgrid=" + std::to_string(c.chunk_grid_cap);  // 0: no cap (always written, so specs round-trip)
  d += ",dbits=" + std::to_string(c.digit_bits);
  d += c.dedup ? ",dedup=hash" : ",dedup=off";
  d += c.dedup_pub ? ",dpub=on" : ",dpub=off";
  return d;
}

static LaunchCfg& launch_cfg_locked(int S) {
  int dev = 0;
  cudaGetDevice(&dev);
  auto it = g_cfg.find({dev, S});
  if (it != g_cfg.end()) return it->second;
  LaunchCfg c;
  cudaDeviceGetAttribute(&c.sms, cudaDevAttrMultiProcessorCount, dev);
  if (c.sms < 1) c.sms = 1;
  c.occ_compact = occupancy_compact(S);
  c.occ_sort = occupancy_sort(S);
  c.occ_head = occupancy_head(S);
  c.occ_sort_pipe = occupancy_sort_pipe(S);
  c.occ_tiles = occupancy_tiles(S);
  for (int k = 0; k < 4; ++k) c.occ_chunk[k] = occupancy_chunk(S, k);
  if (c.occ_sort_pipe < 1 && c.sort_kernel == kSortPipe) c.sort_kernel = kSortRegs;  // too little shared memory
  // 16- to 32-byte keys rank faster without the ballots of constant digit bits (register pressure
  // of the wider items); 4- to 12-byte keys with all eight (measured on GB300)
  if (S >= 16) c.rank_mode = kRankBallotVary;
  // Defaults are the variants measured fastest on GB300; a tuning cache (written by the
  // autotuner) and then REINDEX_TUNE override them.
  apply_tuning(c, tuning_from_cache(dev, c.sms, S).c_str());
  apply_tuning(c, std::getenv("REINDEX_TUNE"));
  return g_cfg.emplace(std::make_pair(dev, S), c).first->second;
}

LaunchCfg launch_cfg(int S) {
  std::lock_guard<std::mutex> g(g_cfg_mu);
  return launch_cfg_locked(S);  // copied under the lock
}

void set_launch_cfg(int S, const LaunchCfg& c) {
  std::lock_guard<std::mutex> g(g_cfg_mu);
  launch_cfg_locked(S) = c;
}

// ---------------------------------------------------------------------------------------------
// Per-launch timing (off by default).
namespace prof {
struct Pending {
  int kernel, digit;
  int item_bytes;       // bytes per sort item (key + old index) of a sort pass, else 0
  cudaEvent_t a, b;
  const uint8_t* skip;  // pinned host copy of the plan's skip flags (sort passes only)
};
static std::mutex mu;
static bool enabled = false;
static std::vector<Pending> pending;
static std::vector<uint8_t*> pinned;

struct Scope {
  bool on;
  Pending p;
  cudaStream_t st;
  Scope(int kernel, int digit, cudaStream_t s, const uint8_t* skip = nullptr, int item_bytes = 0)
      : on(false), st(s) {
    {
      std::lock_guard<std::mutex> g(mu);
      on = enabled;
    }
    if (!on) return;
    p.kernel = kernel;
    p.digit = digit;
    p.item_bytes = item_bytes;
    p.skip = skip;
    cudaEventCreate(&p.a);
    cudaEventCreate(&p.b);
    cudaEventRecord(p.a, st);
  }
  ~Scope() {
    if (!on) return;
    cudaEventRecord(p.b, st);
    std::lock_guard<std::mutex> g(mu);
    pending.push_back(p);
  }
};

static uint8_t* skip_buffer(const Plan* plan, cudaStream_t st) {
  {
    std::lock_guard<std::mutex> g(mu);
    if (!enabled) return nullptr;
  }
  uint8_t* h = nullptr;
  if (cudaMallocHost(&h, kMaxDigits) != cudaSuccess) return nullptr;
  cudaMemcpyAsync(h, plan->skip, kMaxDigits, cudaMemcpyDeviceToHost, st);
  std::lock_guard<std::mutex> g(mu);
  pinned.push_back(h);
  return h;
}
}  // namespace prof

static std::atomic<int64_t> g_stall_tile{-1};
int64_t debug_stall_tile() { return g_stall_tile.load(); }

static reindex_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return REINDEX_OK;
  if (e == cudaErrorMemoryAllocation) return REINDEX_ERR_OOM;
  return REINDEX_ERR_CUDA;
}

#define REINDEX_TRY(expr)                          \
  do {                                             \
    cudaError_t e__ = (expr);                      \
    if (e__ != cudaSuccess) return cuda_status(e__); \
  } while (0)

static bool aligned(const void* p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

static uintptr_t vtx_alignment(int S) { return S % 16 == 0 ? 16 : (S % 8 == 0 ? 8 : 4); }

// Host-side checks shared by every entry point.  Sets M.
// Vertex strides of single meshes: 4-32 bytes on every sort, 48 and 64 bytes through the prefix
// sort with the chunk sort as its full-key fallback.
static bool stride_supported(int S) {
  return S == 4 || S == 8 || S == 12 || S == 16 || S == 20 || S == 24 || S == 32 || S == 48 || S == 64;
}

static reindex_status check_args(int64_t nVtx, int S, int64_t nElem, int k, int64_t* M) {
  if (!stride_supported(S)) return REINDEX_ERR_UNSUPPORTED;
  if (nVtx < 0 || nElem < 0 || k < 1) return REINDEX_ERR_INVALID_ARG;
  if (nVtx > kMaxCount) return REINDEX_ERR_UNSUPPORTED;
  if (nElem > (int64_t)INT32_MAX / k) return REINDEX_ERR_UNSUPPORTED;
  *M = nElem * (int64_t)k;
  return REINDEX_OK;
}

// int64 indices: the same vertex limit; up to 2^40 index entries (nElem * idxPerElem).
// Vertex ranges of meshes beyond kMaxCount vertices (reindex_mesh64 only)
constexpr int kRangeShift = 30;
constexpr int64_t kMaxLargeVtx = int64_t(1) << 40;

static reindex_status check_args64(int64_t nVtx, int S, int64_t nElem, int k, int64_t* M, bool large_ok = false) {
  if (!stride_supported(S)) return REINDEX_ERR_UNSUPPORTED;
  if (nVtx < 0 || nElem < 0 || k < 1) return REINDEX_ERR_INVALID_ARG;
  if (nVtx > (large_ok ? kMaxLargeVtx : kMaxCount)) return REINDEX_ERR_UNSUPPORTED;
  if (nElem > (int64_t(1) << 40) / k) return REINDEX_ERR_UNSUPPORTED;
  *M = nElem * (int64_t)k;
  return REINDEX_OK;
}

static reindex_status check_ptrs(const void* vtx, int64_t nVtx, int S, const void* idx, int64_t M,
                                 const void* out_vtx, const int64_t* out_nVtx, const void* out_idx,
                                 uintptr_t idx_align = 4) {
  if (out_nVtx == nullptr || !aligned(out_nVtx, 8)) return REINDEX_ERR_INVALID_ARG;
  if (M == 0) return REINDEX_OK;
  if (!idx || !out_idx || !out_vtx || (nVtx > 0 && !vtx)) return REINDEX_ERR_INVALID_ARG;
  if (!aligned(idx, idx_align) || !aligned(out_idx, idx_align)) return REINDEX_ERR_INVALID_ARG;
  if ((nVtx > 0 && !aligned(vtx, vtx_alignment(S))) || !aligned(out_vtx, vtx_alignment(S)))
    return REINDEX_ERR_INVALID_ARG;
  return REINDEX_OK;
}

// Optional steps around the single-mesh sequence: `pre` runs right after the workspace is
// cleared (it may record device errors), and with `flags_done` it has already set the used bits.
struct PipeExtras {
  std::function<cudaError_t(const WsPtrs&, const LaunchCfg&)> pre;
  bool flags_done = false;
  cudaEvent_t vtx_ready = nullptr;   // the vertex array is complete once this event has fired
  cudaEvent_t heads_done = nullptr;  // recorded once the unique vertices and *out_nVtx are written
  // hash path: the vertex array arrives in chunks of chunk_vtx vertices (a multiple of 32), chunk c
  // complete once chunk_ready[c] has fired; each chunk is inserted as soon as it is there
  int n_chunks = 0;
  int64_t chunk_vtx = 0;
  const cudaEvent_t* chunk_ready = nullptr;
  bool no_prefix = false;  // the caller's indices are not available for the prefix sort's fallback
  bool o2n_out = false;    // the caller reads oldToNew after the call (every entry a new index)
};

// One radix pass (digit d) with the configured kernel variant.
static cudaError_t sort_pass(int S, int d, const WsPtrs& p, const LaunchCfg& c, cudaStream_t st,
                             const uint8_t* skip) {
  if (c.sort_kernel == kSortChunk) {
    const int G = chunk_grid(S, c, p.Umax);  // the same chunks in the three kernels
    {
      prof::Scope s(REINDEX_K_TILE_COUNT, d, st, skip, S + 4);
      cudaError_t e = launch_chunk_count(S, d, p, G, chunk_tile_items(S, c.chunk_cfg), st);
      if (e != cudaSuccess) return e;
    }
    {
      prof::Scope s(REINDEX_K_TILE_OFFSETS, d, st, skip, S + 4);
      cudaError_t e = launch_tile_offsets(d, p, st, G);
      if (e != cudaSuccess) return e;
    }
    prof::Scope s(REINDEX_K_CHUNK_SCATTER, d, st, skip, S + 4);
    return launch_chunk_scatter(S, d, p, c, G, st);
  }
  if (c.sort_kernel == kSortTiles) {
    {
      prof::Scope s(REINDEX_K_TILE_COUNT, d, st, skip, S + 4);
      cudaError_t e = launch_tile_count(S, d, p, c, st);
      if (e != cudaSuccess) return e;
    }
    {
      prof::Scope s(REINDEX_K_TILE_OFFSETS, d, st, skip, S + 4);
      cudaError_t e = launch_tile_offsets(d, p, st);
      if (e != cudaSuccess) return e;
    }
    prof::Scope s(REINDEX_K_TILE_SCATTER, d, st, skip, S + 4);
    return launch_tile_scatter(S, d, p, c, st);
  }
  prof::Scope s(REINDEX_K_ONESWEEP, d, st, skip, S + 4);
  return c.sort_kernel == kSortPipe ? launch_onesweep_pipe(S, d, p, c, st) : launch_onesweep(S, d, p, c, st);
}

// Index arrays of a call: int32 (every entry point but reindex_mesh64*) or int64.
struct Indices {
  const void* idx;
  void* out;
  bool wide;  // int64
};

static cudaError_t used_flags(const Indices& ix, int64_t M, int64_t nVtx, const WsPtrs& p, const LaunchCfg& c,
                              cudaStream_t st) {
  return ix.wide ? launch_used_flags64(static_cast<const int64_t*>(ix.idx), M, nVtx, p, c, st)
                 : launch_used_flags(static_cast<const int32_t*>(ix.idx), M, nVtx, p, c, st);
}

static cudaError_t remap(const Indices& ix, int64_t M, const WsPtrs& p, const LaunchCfg& c, cudaStream_t st) {
  return ix.wide ? launch_remap64(static_cast<const int64_t*>(ix.idx), static_cast<int64_t*>(ix.out), M, p, c, st)
                 : launch_remap(static_cast<const int32_t*>(ix.idx), static_cast<int32_t*>(ix.out), M, p, c, st);
}

// The launch sequence (all on `st`, no host synchronisation).
static reindex_status run_pipeline(const void* vtx, int64_t nVtx, int S, const Indices& ix, int64_t M,
                                   void* out_vtx, int64_t* out_nVtx, void* ws, const WsLayout& L, cudaStream_t st,
                                   const PipeExtras* extra = nullptr) {
  LaunchCfg c0 = launch_cfg(S);
  if (extra && extra->no_prefix) c0.prefix = 0;
  LaunchCfg c = resolve_cfg(c0, S, L.Umax);  // one configuration for the whole call
  const WsPtrs p = ws_ptrs(ws, L);
  // Prefix sort first: items keep the 64 most significant varying key bits; the full-key sort
  // below then runs only if two different keys shared a prefix (else every kernel of it returns
  // at once).  Both write the same outputs; the remap and the finalize come once, at the end.
  const bool prefix = c.prefix && S > kPrefixBytes;
  const WsPtrs pp = prefix ? ws_ptrs_prefix(ws, L) : p;
  {
    prof::Scope s(REINDEX_K_CLEAR, -1, st);
    REINDEX_TRY(launch_clear(ws, L.zero_bytes + (prefix ? sizeof(Control) : 0), c, st));  // + the prefix control block
  }
  if (extra && extra->pre) {
    prof::Scope s(extra->flags_done ? REINDEX_K_USED_FLAGS : REINDEX_K_SEG_PREPARE, -1, st);
    REINDEX_TRY(extra->pre(pp, c));
  }
  if (!(extra && extra->flags_done)) {
    prof::Scope s(REINDEX_K_USED_FLAGS, -1, st);
    REINDEX_TRY(used_flags(ix, M, nVtx, pp, c, st));
  }
  const bool chunked = c.dedup && extra && extra->n_chunks > 0;
  if (extra && extra->vtx_ready && !chunked) REINDEX_TRY(cudaStreamWaitEvent(st, extra->vtx_ready, 0));
  // the hash table's insertion: each chunk of the vertex array as it arrives, or all at once
  auto hash_insert = [&](const WsPtrs& w, uint32_t slots, bool repmask) -> cudaError_t {
    if (chunked) {
      for (int ch = 0; ch < extra->n_chunks; ++ch) {
        cudaError_t e = cudaStreamWaitEvent(st, extra->chunk_ready[ch], 0);
        if (e != cudaSuccess) return e;
        prof::Scope s(REINDEX_K_HASH_DEDUP, -1, st);
        e = launch_hash_dedup(S, vtx, nVtx, w, slots, (uint32_t)L.Umax, c, st, nullptr, ch * extra->chunk_vtx,
                              (ch + 1) * extra->chunk_vtx, repmask);
        if (e != cudaSuccess) return e;
      }
      return extra->vtx_ready ? cudaStreamWaitEvent(st, extra->vtx_ready, 0) : cudaSuccess;
    }
    prof::Scope s(REINDEX_K_HASH_DEDUP, -1, st);
    return launch_hash_dedup(S, vtx, nVtx, w, slots, (uint32_t)L.Umax, c, st, nullptr, 0, -1, repmask);
  };
  if (c.dedup && !prefix) {  // distinct keys first (hash table), then the method on them; see k_dedup.cu
    const uint32_t slots = dedup_table_slots(L);
    {
      prof::Scope s(REINDEX_K_CLEAR, -1, st);
      REINDEX_TRY(launch_clear(p.itemsB, (size_t)slots * 4, c, st));
    }
    REINDEX_TRY(hash_insert(p, slots, false));
    {
      prof::Scope s(REINDEX_K_SORT_PLAN, -1, st);
      REINDEX_TRY(launch_sort_plan(S, p, true, false, st));
    }
    const uint8_t* skip = prof::skip_buffer(p.plan, st);
    for (int d = 0; d < S; ++d) REINDEX_TRY(sort_pass(S, d, p, c, st, skip));
    {
      prof::Scope s(REINDEX_K_HEAD_SCAN, -1, st);
      REINDEX_TRY(launch_head_scan(S, p, out_vtx, out_nVtx, (uint32_t)nVtx, c, nullptr, st));
    }
    if (extra && extra->heads_done) REINDEX_TRY(cudaEventRecord(extra->heads_done, st));
    if (extra && extra->o2n_out) {  // oldToNew is itself a product: every copy takes its new index
      prof::Scope s(REINDEX_K_RESOLVE, -1, st);
      REINDEX_TRY(launch_resolve(nVtx, p, c, st));
    }
    {  // copies go through their representative (a second look-up: cheaper than a resolve pass)
      prof::Scope s(REINDEX_K_REMAP, -1, st);
      REINDEX_TRY(launch_remap_rep(ix.idx, ix.out, ix.wide, M, p, c, st));
    }
    prof::Scope s(REINDEX_K_FINALIZE, -1, st);
    REINDEX_TRY(launch_finalize(p, out_nVtx, st));
    return REINDEX_OK;
  }
  if (prefix) {
    LaunchCfg cp = c;  // the passes sort 12-byte keys (8 varying bytes) with the tiles or chunk sort
    cp.sort_kernel = c.sort_kernel == kSortChunk ? kSortChunk : kSortTiles;
    const LaunchCfg c12 = launch_cfg(kPrefixItem);
    cp.occ_tiles = c12.occ_tiles;
    for (int k = 0; k < 4; ++k) cp.occ_chunk[k] = c12.occ_chunk[k];
    if (c.dedup) {  // the representatives become the used vertices; the key masks come with them
      const uint32_t slots = dedup_table_slots(L);
      {
        prof::Scope s(REINDEX_K_CLEAR, -1, st);
        REINDEX_TRY(launch_clear(p.itemsB, (size_t)slots * 4, c, st));
      }
      REINDEX_TRY(hash_insert(pp, slots, true));
    } else {
      prof::Scope s(REINDEX_K_KEY_MASKS, -1, st);
      REINDEX_TRY(launch_key_masks(S, vtx, nVtx, pp, c, nullptr, st));
    }
    {
      prof::Scope s(REINDEX_K_SORT_PLAN, -1, st);
      REINDEX_TRY(launch_prefix_plan(S, pp, st, cp.digit_bits));
    }
    {
      prof::Scope s(REINDEX_K_COMPACT, -1, st);
      REINDEX_TRY(launch_compact_prefix(S, vtx, nVtx, pp, L.tilesV, c, st));
    }
    const uint8_t* pskip = prof::skip_buffer(pp.plan, st);
    for (int d = 0; d < prefix_passes(cp.digit_bits); ++d) REINDEX_TRY(sort_pass(kPrefixItem, d, pp, cp, st, pskip));
    {
      prof::Scope s(REINDEX_K_HEAD_SCAN, -1, st);
      REINDEX_TRY(launch_head_scan_prefix(S, pp, vtx, out_vtx, out_nVtx, (uint32_t)nVtx, c, st));
    }
    {
      prof::Scope s(REINDEX_K_PREFIX_CHECK, -1, st);
      REINDEX_TRY(launch_prefix_check(S, vtx, nVtx, out_vtx, pp, c, st));
    }
    {
      prof::Scope s(REINDEX_K_CLEAR, -1, st);
      REINDEX_TRY(launch_clear(ws, L.zero_bytes, c, st));  // the full-key sort's tables
    }
    {
      prof::Scope s(REINDEX_K_PREFIX_GATE, -1, st);
      REINDEX_TRY(launch_prefix_gate(pp, p, st));
    }
    prof::Scope s(REINDEX_K_USED_FLAGS, -1, st);
    REINDEX_TRY(used_flags(ix, M, nVtx, p, c, st));
    c.scatter_waves = 1;  // the full-key sort's passes: few CTAs, cheap when skipped
  }
  if (uses_plane(c.sort_kernel) && c.pack_keys) {  // bit masks -> plan (key packing) -> compaction
    {
      prof::Scope s(REINDEX_K_KEY_MASKS, -1, st);
      REINDEX_TRY(launch_key_masks(S, vtx, nVtx, p, c, nullptr, st));
    }
    {
      prof::Scope s(REINDEX_K_SORT_PLAN, -1, st);
      REINDEX_TRY(launch_sort_plan(S, p, true, true, st, c.digit_bits));
    }
    prof::Scope s(REINDEX_K_COMPACT, -1, st);
    REINDEX_TRY(launch_compact(S, vtx, nVtx, p, L.tilesV, c, nullptr, st));
  } else {  // compaction (upfront histograms, or key bit masks) -> plan
    {
      prof::Scope s(REINDEX_K_COMPACT, -1, st);
      REINDEX_TRY(launch_compact(S, vtx, nVtx, p, L.tilesV, c, nullptr, st));
    }
    prof::Scope s(REINDEX_K_SORT_PLAN, -1, st);
    REINDEX_TRY(launch_sort_plan(S, p, uses_plane(c.sort_kernel), false, st));
  }
  const uint8_t* skip = prof::skip_buffer(p.plan, st);
  for (int d = 0; d < sort_passes(S, c.digit_bits); ++d) REINDEX_TRY(sort_pass(S, d, p, c, st, skip));
  {
    prof::Scope s(REINDEX_K_HEAD_SCAN, -1, st);
    REINDEX_TRY(launch_head_scan(S, p, out_vtx, out_nVtx, (uint32_t)nVtx, c, nullptr, st));
  }
  if (extra && extra->heads_done) REINDEX_TRY(cudaEventRecord(extra->heads_done, st));
  {
    prof::Scope s(REINDEX_K_REMAP, -1, st);
    if (c.dedup)  // the prefix path sorted the representatives: copies go through theirs
      REINDEX_TRY(launch_remap_rep(ix.idx, ix.out, ix.wide, M, p, c, st));
    else
      REINDEX_TRY(remap(ix, M, p, c, st));
  }
  {
    prof::Scope s(REINDEX_K_FINALIZE, -1, st);
    REINDEX_TRY(launch_finalize(p, out_nVtx, st));
  }
  return REINDEX_OK;
}

static reindex_status run_pipeline(const void* vtx, int64_t nVtx, int S, const int32_t* idx, int64_t M,
                                   void* out_vtx, int64_t* out_nVtx, int32_t* out_idx, void* ws,
                                   const WsLayout& L, cudaStream_t st, const PipeExtras* extra = nullptr) {
  return run_pipeline(vtx, nVtx, S, Indices{idx, out_idx, false}, M, out_vtx, out_nVtx, ws, L, st, extra);
}

// Workspace of the batched path: the single-mesh layout for (S + 4)-byte keys over all vertices
// and indices, followed by the two position -> mesh lookup tables.
struct SegLayout {
  WsLayout L;
  size_t off_blkV = 0, off_blkI = 0, total = 0;
  void compute(int64_t n, int s, int64_t m) {
    L.compute(n, s + 4, m);
    size_t o = L.total;
    off_blkV = o;
    o = align_up(o + (size_t)((n + kSegBlock - 1) / kSegBlock + 1) * 4, 256);
    off_blkI = o;
    o = align_up(o + (size_t)((m + kSegBlock - 1) / kSegBlock + 1) * 4, 256);
    total = o;
  }
};

static reindex_status run_batched(const void* vtx, int64_t nVtx, int S, const int32_t* idx, int64_t M, int k,
                                  const int64_t* vtxOff, const int64_t* elemOff, int nMeshes, void* out_vtx,
                                  int64_t* outOff, int32_t* out_idx, void* ws, const SegLayout& SL,
                                  cudaStream_t st) {
  const LaunchCfg cS = launch_cfg(S);
  const LaunchCfg c = resolve_cfg(launch_cfg(S + 4), S + 4, SL.L.Umax, true);
  const WsPtrs p = ws_ptrs(ws, SL.L);
  unsigned char* b = static_cast<unsigned char*>(ws);
  SegArgs seg;
  seg.vtxOff = vtxOff;
  seg.elemOff = elemOff;
  seg.outOff = outOff;
  seg.blkV = reinterpret_cast<const uint32_t*>(b + SL.off_blkV);
  seg.blkI = reinterpret_cast<const uint32_t*>(b + SL.off_blkI);
  seg.nMeshes = nMeshes;
  seg.k = k;
  int64_t* total = outOff + nMeshes;  // D, or -status after a device-detected error
  {
    prof::Scope sc(REINDEX_K_CLEAR, -1, st);
    REINDEX_TRY(launch_clear(ws, SL.L.zero_bytes, c, st));
  }
  {
    prof::Scope sc(REINDEX_K_SEG_PREPARE, -1, st);
    REINDEX_TRY(launch_seg_prepare(seg, nVtx, M, reinterpret_cast<uint32_t*>(b + SL.off_blkV),
                                   reinterpret_cast<uint32_t*>(b + SL.off_blkI), p.ctrl, c, st));
  }
  {
    prof::Scope sc(REINDEX_K_USED_FLAGS, -1, st);
    REINDEX_TRY(launch_seg_flags(idx, out_idx, M, seg, p, c, st));
  }
  if (c.dedup) {  // distinct (mesh id, vertex) keys first (hash table), then the method on them
    const uint32_t slots = dedup_table_slots(SL.L);
    {
      prof::Scope sc(REINDEX_K_CLEAR, -1, st);
      REINDEX_TRY(launch_clear(p.itemsB, (size_t)slots * 4, c, st));
    }
    {
      prof::Scope sc(REINDEX_K_HASH_DEDUP, -1, st);
      REINDEX_TRY(launch_hash_dedup(S, vtx, nVtx, p, slots, (uint32_t)SL.L.Umax, c, st, &seg));
    }
    {
      prof::Scope sc(REINDEX_K_SORT_PLAN, -1, st);
      REINDEX_TRY(launch_sort_plan(S + 4, p, true, false, st));
    }
    const uint8_t* skip = prof::skip_buffer(p.plan, st);
    for (int d = 0; d < S + 4; ++d) REINDEX_TRY(sort_pass(S + 4, d, p, c, st, skip));
    {
      prof::Scope sc(REINDEX_K_HEAD_SCAN, -1, st);
      REINDEX_TRY(launch_head_scan(S + 4, p, out_vtx, total, (uint32_t)nVtx, c, &seg, st));
    }
    {
      prof::Scope sc(REINDEX_K_SEG_OFFSETS, -1, st);
      REINDEX_TRY(launch_seg_offsets(seg, p.ctrl, st));
    }
    {
      prof::Scope sc(REINDEX_K_REMAP, -1, st);
      REINDEX_TRY(launch_seg_remap(out_idx, M, seg, p, c, st));
    }
    prof::Scope sc(REINDEX_K_FINALIZE, -1, st);
    REINDEX_TRY(launch_finalize(p, total, st));
    return REINDEX_OK;
  }
  LaunchCfg cc = cS;  // the sort (configured for S + 4) decides whether histograms are taken
  cc.sort_kernel = c.sort_kernel;
  cc.pack_keys = c.pack_keys;
  if (uses_plane(c.sort_kernel) && c.pack_keys) {  // bit masks -> plan (key packing) -> compaction
    {
      prof::Scope sc(REINDEX_K_KEY_MASKS, -1, st);
      REINDEX_TRY(launch_key_masks(S, vtx, nVtx, p, cc, &seg, st));
    }
    {
      prof::Scope sc(REINDEX_K_SORT_PLAN, -1, st);
      REINDEX_TRY(launch_sort_plan(S + 4, p, true, true, st, c.digit_bits));
    }
    prof::Scope sc(REINDEX_K_COMPACT, -1, st);
    REINDEX_TRY(launch_compact(S, vtx, nVtx, p, SL.L.tilesV, cc, &seg, st));
  } else {  // compaction (upfront histograms, or key bit masks) -> plan
    {
      prof::Scope sc(REINDEX_K_COMPACT, -1, st);
      REINDEX_TRY(launch_compact(S, vtx, nVtx, p, SL.L.tilesV, cc, &seg, st));
    }
    prof::Scope sc(REINDEX_K_SORT_PLAN, -1, st);
    REINDEX_TRY(launch_sort_plan(S + 4, p, uses_plane(c.sort_kernel), false, st));
  }
  const uint8_t* skip = prof::skip_buffer(p.plan, st);
  for (int d = 0; d < sort_passes(S + 4, c.digit_bits); ++d) REINDEX_TRY(sort_pass(S + 4, d, p, c, st, skip));
  {
    prof::Scope sc(REINDEX_K_HEAD_SCAN, -1, st);
    REINDEX_TRY(launch_head_scan(S + 4, p, out_vtx, total, (uint32_t)nVtx, c, &seg, st));
  }
  {
    prof::Scope sc(REINDEX_K_SEG_OFFSETS, -1, st);
    REINDEX_TRY(launch_seg_offsets(seg, p.ctrl, st));
  }
  {
    prof::Scope sc(REINDEX_K_REMAP, -1, st);
    REINDEX_TRY(launch_seg_remap(out_idx, M, seg, p, c, st));
  }
  {
    prof::Scope sc(REINDEX_K_FINALIZE, -1, st);
    REINDEX_TRY(launch_finalize(p, total, st));
  }
  return REINDEX_OK;
}

static void set_pool_threshold() {
  static std::mutex mu;
  static std::map<int, bool> done;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> g(mu);
  if (done[dev]) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;  // keep freed blocks cached in the pool between calls
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  done[dev] = true;
}

}  // namespace reindex

using namespace reindex;

extern "C" {

const char* reindex_status_string(reindex_status s) {
  switch (s) {
    case REINDEX_OK: return "REINDEX_OK";
    case REINDEX_ERR_INVALID_ARG: return "REINDEX_ERR_INVALID_ARG";
    case REINDEX_ERR_UNSUPPORTED: return "REINDEX_ERR_UNSUPPORTED";
    case REINDEX_ERR_OOM: return "REINDEX_ERR_OOM";
    case REINDEX_ERR_INDEX_RANGE: return "REINDEX_ERR_INDEX_RANGE";
    case REINDEX_ERR_TIMEOUT: return "REINDEX_ERR_TIMEOUT";
    case REINDEX_ERR_CUDA: return "REINDEX_ERR_CUDA";
    case REINDEX_ERR_INTERNAL: return "REINDEX_ERR_INTERNAL";
  }
  return "REINDEX_ERR_UNKNOWN";
}

size_t reindex_workspace_size(int64_t nVtx, int vtxStrideBytes, int64_t nElem, int idxPerElem) {
  int64_t M = 0;
  if (check_args(nVtx, vtxStrideBytes, nElem, idxPerElem, &M) != REINDEX_OK) return 0;
  WsLayout L;
  L.compute(nVtx, vtxStrideBytes, M);
  return L.total;
}

reindex_status reindex_mesh_ws(const void* vtx, int64_t nVtx, int S, const int32_t* idx, int64_t nElem, int k,
                               void* out_vtx, int64_t* out_nVtx, int32_t* out_idx, void* ws, size_t wsBytes,
                               reindex_stream_t stream) {
  int64_t M = 0;
  reindex_status r = check_args(nVtx, S, nElem, k, &M);
  if (r != REINDEX_OK) return r;
  if ((r = check_ptrs(vtx, nVtx, S, idx, M, out_vtx, out_nVtx, out_idx)) != REINDEX_OK) return r;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (M == 0) return cuda_status(launch_set_count(out_nVtx, 0, st));
  if (nVtx == 0) return REINDEX_ERR_INDEX_RANGE;
  WsLayout L;
  L.compute(nVtx, S, M);
  if (ws == nullptr || !aligned(ws, 256) || wsBytes < L.total) return REINDEX_ERR_INVALID_ARG;
  return run_pipeline(vtx, nVtx, S, idx, M, out_vtx, out_nVtx, out_idx, ws, L, st);
}

reindex_status reindex_mesh(const void* vtx, int64_t nVtx, int S, const int32_t* idx, int64_t nElem, int k,
                            void* out_vtx, int64_t* out_nVtx, int32_t* out_idx, reindex_stream_t stream) {
  int64_t M = 0;
  reindex_status r = check_args(nVtx, S, nElem, k, &M);
  if (r != REINDEX_OK) return r;
  if ((r = check_ptrs(vtx, nVtx, S, idx, M, out_vtx, out_nVtx, out_idx)) != REINDEX_OK) return r;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (M == 0) return cuda_status(launch_set_count(out_nVtx, 0, st));
  if (nVtx == 0) return REINDEX_ERR_INDEX_RANGE;
  WsLayout L;
  L.compute(nVtx, S, M);
  set_pool_threshold();
  void* ws = nullptr;
  cudaError_t e = cudaMallocAsync(&ws, L.total, st);
  if (e != cudaSuccess) return cuda_status(e);
  r = run_pipeline(vtx, nVtx, S, idx, M, out_vtx, out_nVtx, out_idx, ws, L, st);
  e = cudaFreeAsync(ws, st);
  if (r == REINDEX_OK && e != cudaSuccess) r = cuda_status(e);
  return r;
}

size_t reindex_workspace_size64(int64_t nVtx, int vtxStrideBytes, int64_t nElem, int idxPerElem) {
  int64_t M = 0;
  if (check_args64(nVtx, vtxStrideBytes, nElem, idxPerElem, &M) != REINDEX_OK) return 0;
  WsLayout L;
  L.compute(nVtx, vtxStrideBytes, M);
  return L.total;
}

reindex_status reindex_mesh64_ws(const void* vtx, int64_t nVtx, int S, const int64_t* idx, int64_t nElem, int k,
                                 void* out_vtx, int64_t* out_nVtx, int64_t* out_idx, void* ws, size_t wsBytes,
                                 reindex_stream_t stream) {
  int64_t M = 0;
  reindex_status r = check_args64(nVtx, S, nElem, k, &M);
  if (r != REINDEX_OK) return r;
  if ((r = check_ptrs(vtx, nVtx, S, idx, M, out_vtx, out_nVtx, out_idx, 8)) != REINDEX_OK) return r;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (M == 0) return cuda_status(launch_set_count(out_nVtx, 0, st));
  if (nVtx == 0) return REINDEX_ERR_INDEX_RANGE;
  WsLayout L;
  L.compute(nVtx, S, M);
  if (ws == nullptr || !aligned(ws, 256) || wsBytes < L.total) return REINDEX_ERR_INVALID_ARG;
  return run_pipeline(vtx, nVtx, S, Indices{idx, out_idx, true}, M, out_vtx, out_nVtx, ws, L, st);
}

// Meshes of more than kMaxCount vertices (int64 indices): the look-back counts, the 32-bit old-index
// payload and oldToNew cover at most kMaxCount vertices, so the vertex array is re-indexed in ranges
// of 2^30 vertices.  Range p takes the used vertices in [p * 2^30, (p + 1) * 2^30) -- its used bits
// set from all the indices -- through the single-mesh path (no remap), which leaves each of them its
// rank among the range's unique vertices and writes those unique vertices, sorted, after the previous
// ranges'.  The concatenated unique vertices (fewer than 2^31, or REINDEX_ERR_UNSUPPORTED) are then
// re-indexed once more with identity indices, which merges keys that occur in several ranges and
// gives each range-unique vertex its final index; a last kernel composes the two maps for every
// index.  The result is the single-level one: the unique vertices are the distinct used keys in key
// order, and every index resolves to its key's rank.  Synchronises the stream once per range.
static reindex_status run_large64(const void* vtx, int64_t N, int S, const int64_t* idx, int64_t M, void* out_vtx,
                                  int64_t* out_nVtx, int64_t* out_idx, cudaStream_t st) {
  const int64_t part = int64_t(1) << kRangeShift;
  const int P = (int)((N + part - 1) / part);
  const int64_t cap = std::min(N, M);  // unique vertices of all ranges together, at most
  WsLayout Lp;
  Lp.compute(part, S, std::min(part, M));
  const size_t b_rank = align_up((size_t)N * 4, 256), b_cat = align_up((size_t)cap * S, 256),
               b_off = align_up((size_t)(P + 1) * 8, 256);
  set_pool_threshold();
  unsigned char* d = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&d), b_rank + b_cat + b_off + 256 + Lp.total, st);
  if (e != cudaSuccess) return cuda_status(e);
  uint32_t* rank = reinterpret_cast<uint32_t*>(d);
  unsigned char* cat = d + b_rank;
  int64_t* part_off = reinterpret_cast<int64_t*>(d + b_rank + b_cat);
  int64_t* cnt = reinterpret_cast<int64_t*>(d + b_rank + b_cat + b_off);
  void* ws = d + b_rank + b_cat + b_off + 256;
  std::vector<int64_t> off(P + 1, 0);
  reindex_status r = REINDEX_OK;
  const LaunchCfg c0 = launch_cfg(S);
  for (int pi = 0; pi < P && r == REINDEX_OK && e == cudaSuccess; ++pi) {
    const int64_t lo = pi * part, n = std::min(part, N - lo);
    WsLayout L;
    L.compute(n, S, std::min(n, M));
    PipeExtras ex;
    ex.flags_done = true;
    ex.no_prefix = true;
    ex.o2n_out = true;
    ex.pre = [&](const WsPtrs& w, const LaunchCfg& c) {
      return launch_used_flags_range64(idx, M, lo, n, N, w, pi == 0, c, st);
    };
    r = run_pipeline(static_cast<const unsigned char*>(vtx) + (size_t)lo * S, n, S, Indices{nullptr, nullptr, true},
                     0, cat + (size_t)off[pi] * S, cnt, ws, L, st, &ex);
    if (r != REINDEX_OK) break;
    if ((e = cudaMemcpyAsync(rank + lo, static_cast<unsigned char*>(ws) + L.off_old2new, (size_t)n * 4,
                             cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
      break;
    int64_t Dp = 0;
    if ((e = cudaMemcpyAsync(&Dp, cnt, 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess) break;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) break;
    if (Dp < 0) {  // a device-detected error (an index out of range, found with range 0)
      e = launch_set_count(out_nVtx, Dp, st);
      r = (reindex_status)(-Dp);
      break;
    }
    off[pi + 1] = off[pi] + Dp;
  }
  const int64_t N2 = off[P];
  if (r == REINDEX_OK && e == cudaSuccess && N2 > kMaxCount) r = REINDEX_ERR_UNSUPPORTED;
  if (r == REINDEX_OK && e == cudaSuccess) {
    WsLayout L2;
    L2.compute(N2, S, N2);
    const size_t b_map = align_up((size_t)N2 * 4, 256);
    unsigned char* d2 = nullptr;
    e = cudaMallocAsync(reinterpret_cast<void**>(&d2), 2 * b_map + L2.total, st);
    if (e == cudaSuccess) {
      int32_t* iota = reinterpret_cast<int32_t*>(d2);
      int32_t* map2 = reinterpret_cast<int32_t*>(d2 + b_map);
      do {
        if ((e = cudaMemcpyAsync(part_off, off.data(), (size_t)(P + 1) * 8, cudaMemcpyHostToDevice, st)) !=
            cudaSuccess)
          break;
        if ((e = launch_iota(iota, N2, c0, st)) != cudaSuccess) break;
        r = run_pipeline(cat, N2, S, Indices{iota, map2, false}, N2, out_vtx, out_nVtx, d2 + 2 * b_map, L2, st);
        if (r != REINDEX_OK) break;
        e = launch_remap_two_level(idx, out_idx, M, rank, part_off, map2, kRangeShift, c0, st);
      } while (0);
      // the host copy of the offsets must outlive the transfer above
      cudaError_t es = cudaStreamSynchronize(st);
      if (e == cudaSuccess) e = es;
      cudaError_t ef = cudaFreeAsync(d2, st);
      if (e == cudaSuccess) e = ef;
    }
  }
  cudaError_t ef = cudaFreeAsync(d, st);
  if (e == cudaSuccess) e = ef;
  if (r != REINDEX_OK) return r;
  return e == cudaSuccess ? REINDEX_OK : cuda_status(e);
}

reindex_status reindex_mesh64(const void* vtx, int64_t nVtx, int S, const int64_t* idx, int64_t nElem, int k,
                              void* out_vtx, int64_t* out_nVtx, int64_t* out_idx, reindex_stream_t stream) {
  int64_t M = 0;
  reindex_status r = check_args64(nVtx, S, nElem, k, &M, true);
  if (r != REINDEX_OK) return r;
  if ((r = check_ptrs(vtx, nVtx, S, idx, M, out_vtx, out_nVtx, out_idx, 8)) != REINDEX_OK) return r;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (M == 0) return cuda_status(launch_set_count(out_nVtx, 0, st));
  if (nVtx == 0) return REINDEX_ERR_INDEX_RANGE;
  if (nVtx > kMaxCount) return run_large64(vtx, nVtx, S, idx, M, out_vtx, out_nVtx, out_idx, st);
  WsLayout L;
  L.compute(nVtx, S, M);
  set_pool_threshold();
  void* ws = nullptr;
  cudaError_t e = cudaMallocAsync(&ws, L.total, st);
  if (e != cudaSuccess) return cuda_status(e);
  r = run_pipeline(vtx, nVtx, S, Indices{idx, out_idx, true}, M, out_vtx, out_nVtx, ws, L, st);
  e = cudaFreeAsync(ws, st);
  if (r == REINDEX_OK && e != cudaSuccess) r = cuda_status(e);
  return r;
}

reindex_status reindex_mesh_host(const void* host_vtx, int64_t nVtx, int S, const int32_t* host_idx,
                                 int64_t nElem, int k, void* host_out_vtx, int64_t* host_out_nVtx,
                                 int32_t* host_out_idx, reindex_stream_t stream) {
  int64_t M = 0;
  reindex_status r = check_args(nVtx, S, nElem, k, &M);
  if (r != REINDEX_OK) return r;
  if (host_out_nVtx == nullptr) return REINDEX_ERR_INVALID_ARG;
  if (M == 0) {
    *host_out_nVtx = 0;
    return REINDEX_OK;
  }
  if (!host_idx || !host_out_idx || !host_out_vtx || !host_vtx) return REINDEX_ERR_INVALID_ARG;
  if (nVtx == 0) return REINDEX_ERR_INDEX_RANGE;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  WsLayout L;
  L.compute(nVtx, S, M);
  // The hash path inserts the vertex array chunk by chunk as it arrives (indices first: the used
  // flags must be complete before the first insertion); the other paths sort after the whole array.
  const bool dedup = resolve_cfg(launch_cfg(S), S, L.Umax).dedup != 0;
  constexpr int kMaxChunks = 8;
  const int64_t chunk_vtx = align_up((size_t)((nVtx + kMaxChunks - 1) / kMaxChunks), 32);
  const int n_chunks = dedup ? (int)((nVtx + chunk_vtx - 1) / chunk_vtx) : 0;
  const size_t b_vtx = align_up((size_t)nVtx * S, 256), b_idx = align_up((size_t)M * 4, 256);
  const size_t b_out = align_up((size_t)L.Umax * S, 256);
  const size_t total = b_vtx + 2 * b_idx + b_out + 256 + L.total;
  set_pool_threshold();
  // A second stream carries the vertex upload (while the used flags are set from the indices) and
  // the download of the unique vertices (while the indices are remapped).
  cudaStream_t cs = nullptr;
  cudaEvent_t ev_alloc = nullptr, ev_vtx = nullptr, ev_heads = nullptr, ev_cs = nullptr, ev_idx = nullptr;
  cudaEvent_t ev_chunk[kMaxChunks] = {};
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  for (cudaEvent_t* ev : {&ev_alloc, &ev_vtx, &ev_heads, &ev_cs, &ev_idx})
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
  for (int ch = 0; ch < n_chunks; ++ch)
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_chunk[ch], cudaEventDisableTiming);
  unsigned char* d = nullptr;
  if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void**>(&d), total, st);
  int64_t D = -1, Dfinal = -1;
  bool allocated = e == cudaSuccess;
  if (allocated) {
    void* d_vtx = d;
    int32_t* d_idx = reinterpret_cast<int32_t*>(d + b_vtx);
    int32_t* d_oidx = reinterpret_cast<int32_t*>(d + b_vtx + b_idx);
    void* d_ovtx = d + b_vtx + 2 * b_idx;
    int64_t* d_n = reinterpret_cast<int64_t*>(d + b_vtx + 2 * b_idx + b_out);
    void* d_ws = d + b_vtx + 2 * b_idx + b_out + 256;
    PipeExtras ex;
    ex.vtx_ready = ev_vtx;
    ex.heads_done = ev_heads;
    ex.n_chunks = n_chunks;
    ex.chunk_vtx = chunk_vtx;
    ex.chunk_ready = ev_chunk;
    do {
      if ((e = cudaEventRecord(ev_alloc, st)) != cudaSuccess) break;
      if ((e = cudaStreamWaitEvent(cs, ev_alloc, 0)) != cudaSuccess) break;
      if (n_chunks > 0) {  // indices, then the vertex array chunk by chunk, on the copy stream
        if ((e = cudaMemcpyAsync(d_idx, host_idx, (size_t)M * 4, cudaMemcpyHostToDevice, cs)) != cudaSuccess) break;
        if ((e = cudaEventRecord(ev_idx, cs)) != cudaSuccess) break;
        for (int ch = 0; ch < n_chunks && e == cudaSuccess; ++ch) {
          const int64_t lo = ch * chunk_vtx, hi = std::min(nVtx, lo + chunk_vtx);
          e = cudaMemcpyAsync(static_cast<unsigned char*>(d_vtx) + (size_t)lo * S,
                              static_cast<const unsigned char*>(host_vtx) + (size_t)lo * S, (size_t)(hi - lo) * S,
                              cudaMemcpyHostToDevice, cs);
          if (e == cudaSuccess) e = cudaEventRecord(ev_chunk[ch], cs);
        }
        if (e != cudaSuccess) break;
        if ((e = cudaEventRecord(ev_vtx, cs)) != cudaSuccess) break;
        if ((e = cudaStreamWaitEvent(st, ev_idx, 0)) != cudaSuccess) break;
      } else {
        if ((e = cudaMemcpyAsync(d_vtx, host_vtx, (size_t)nVtx * S, cudaMemcpyHostToDevice, cs)) != cudaSuccess)
          break;
        if ((e = cudaEventRecord(ev_vtx, cs)) != cudaSuccess) break;
        if ((e = cudaMemcpyAsync(d_idx, host_idx, (size_t)M * 4, cudaMemcpyHostToDevice, st)) != cudaSuccess) break;
      }
      if ((e = cudaMemsetAsync(d_n, 0xFF, 8, st)) != cudaSuccess) break;  // -1 unless the head scan runs
      r = run_pipeline(d_vtx, nVtx, S, d_idx, M, d_ovtx, d_n, d_oidx, d_ws, L, st, &ex);
      if (r != REINDEX_OK) break;
      if ((e = cudaMemcpyAsync(host_out_idx, d_oidx, (size_t)M * 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess) break;
      // the unique count, then the unique vertices, on the second stream while the remap runs
      if ((e = cudaStreamWaitEvent(cs, ev_heads, 0)) != cudaSuccess) break;
      if ((e = cudaMemcpyAsync(&D, d_n, 8, cudaMemcpyDeviceToHost, cs)) != cudaSuccess) break;
      if ((e = cudaStreamSynchronize(cs)) != cudaSuccess) break;
      if (D > 0 && D <= L.Umax &&
          (e = cudaMemcpyAsync(host_out_vtx, d_ovtx, (size_t)D * S, cudaMemcpyDeviceToHost, cs)) != cudaSuccess)
        break;
      if ((e = cudaEventRecord(ev_cs, cs)) != cudaSuccess) break;
      if ((e = cudaStreamWaitEvent(st, ev_cs, 0)) != cudaSuccess) break;
      // the final count: k_finalize replaces it by -status after a device-detected error
      if ((e = cudaMemcpyAsync(&Dfinal, d_n, 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess) break;
    } while (0);
    cudaError_t ef = cudaFreeAsync(d, st);
    if (e == cudaSuccess) e = ef;
  }
  cudaError_t es = cudaStreamSynchronize(st);
  cudaError_t es2 = cs ? cudaStreamSynchronize(cs) : cudaSuccess;
  D = Dfinal;
  for (cudaEvent_t ev : {ev_alloc, ev_vtx, ev_heads, ev_cs, ev_idx})
    if (ev) cudaEventDestroy(ev);
  for (int ch = 0; ch < n_chunks; ++ch)
    if (ev_chunk[ch]) cudaEventDestroy(ev_chunk[ch]);
  if (cs) cudaStreamDestroy(cs);
  if (r != REINDEX_OK) return r;
  if (e != cudaSuccess) return cuda_status(e);
  if (es != cudaSuccess) return cuda_status(es);
  if (es2 != cudaSuccess) return cuda_status(es2);
  *host_out_nVtx = D;
  if (D < 0) return (reindex_status)(-D);
  return REINDEX_OK;
}

static reindex_status check_batched(int64_t nVtxTotal, int S, int64_t nElemTotal, int k, int nMeshes, int64_t* M) {
  if (S != 4 && S != 8 && S != 12 && S != 16) return REINDEX_ERR_UNSUPPORTED;
  if (nMeshes < 1) return REINDEX_ERR_INVALID_ARG;
  return check_args(nVtxTotal, S, nElemTotal, k, M);
}

size_t reindex_meshes_workspace_size(int nMeshes, int64_t nVtxTotal, int vtxStrideBytes, int64_t nElemTotal,
                                     int idxPerElem) {
  int64_t M = 0;
  if (check_batched(nVtxTotal, vtxStrideBytes, nElemTotal, idxPerElem, nMeshes, &M) != REINDEX_OK) return 0;
  SegLayout SL;
  SL.compute(nVtxTotal, vtxStrideBytes, M);
  return SL.total;
}

reindex_status reindex_meshes(const void* vtx, const int64_t* vtxOffsets, int vtxStrideBytes, const int32_t* idx,
                              const int64_t* elemOffsets, int idxPerElem, int nMeshes, int64_t nVtxTotal,
                              int64_t nElemTotal, void* out_vtx, int64_t* out_vtxOffsets, int32_t* out_idx,
                              void* ws, size_t wsBytes, reindex_stream_t stream) {
  int64_t M = 0;
  const int S = vtxStrideBytes;
  reindex_status r = check_batched(nVtxTotal, S, nElemTotal, idxPerElem, nMeshes, &M);
  if (r != REINDEX_OK) return r;
  if (!vtxOffsets || !elemOffsets || !out_vtxOffsets || !aligned(vtxOffsets, 8) || !aligned(elemOffsets, 8) ||
      !aligned(out_vtxOffsets, 8))
    return REINDEX_ERR_INVALID_ARG;
  if ((r = check_ptrs(vtx, nVtxTotal, S, idx, M, out_vtx, out_vtxOffsets, out_idx)) != REINDEX_OK) return r;
  if (M > 0 && nVtxTotal == 0) return REINDEX_ERR_INDEX_RANGE;
  SegLayout SL;
  SL.compute(nVtxTotal, S, M);
  if (ws == nullptr || !aligned(ws, 256) || wsBytes < SL.total) return REINDEX_ERR_INVALID_ARG;
  return run_batched(vtx, nVtxTotal, S, idx, M, idxPerElem, vtxOffsets, elemOffsets, nMeshes, out_vtx,
                     out_vtxOffsets, out_idx, ws, SL, reinterpret_cast<cudaStream_t>(stream));
}

// ---- mesh merging (Section 3.2) --------------------------------------------------------------
// Workspace: the single-mesh layout over the concatenation, the two lookup tables of the batched
// path, and nMeshes+1 offsets of scratch.
struct MergeLayout {
  WsLayout L;
  size_t off_blkV = 0, off_blkI = 0, off_scratch = 0, total = 0;
  void compute(int64_t n, int s, int64_t m, int nMeshes) {
    L.compute(n, s, m);
    size_t o = L.total;
    off_blkV = o;
    o = align_up(o + (size_t)((n + kSegBlock - 1) / kSegBlock + 1) * 4, 256);
    off_blkI = o;
    o = align_up(o + (size_t)((m + kSegBlock - 1) / kSegBlock + 1) * 4, 256);
    off_scratch = o;
    o = align_up(o + (size_t)(nMeshes + 1) * 8, 256);
    total = o;
  }
};

size_t reindex_merge_workspace_size(int nMeshes, int64_t nVtxTotal, int vtxStrideBytes, int64_t nElemTotal,
                                    int idxPerElem) {
  int64_t M = 0;
  if (nMeshes < 1 || check_args(nVtxTotal, vtxStrideBytes, nElemTotal, idxPerElem, &M) != REINDEX_OK) return 0;
  MergeLayout ML;
  ML.compute(nVtxTotal, vtxStrideBytes, M, nMeshes);
  return ML.total;
}

reindex_status reindex_merge_meshes(const void* vtx, const int64_t* vtxOffsets, int S, const int32_t* idx,
                                    const int64_t* elemOffsets, int k, int nMeshes, int64_t nVtxTotal,
                                    int64_t nElemTotal, void* out_vtx, int64_t* out_nVtx, int32_t* out_idx, void* ws,
                                    size_t wsBytes, reindex_stream_t stream) {
  int64_t M = 0;
  reindex_status r = check_args(nVtxTotal, S, nElemTotal, k, &M);
  if (r != REINDEX_OK) return r;
  if (nMeshes < 1 || !vtxOffsets || !elemOffsets || !aligned(vtxOffsets, 8) || !aligned(elemOffsets, 8))
    return REINDEX_ERR_INVALID_ARG;
  if ((r = check_ptrs(vtx, nVtxTotal, S, idx, M, out_vtx, out_nVtx, out_idx)) != REINDEX_OK) return r;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (M == 0) return cuda_status(launch_set_count(out_nVtx, 0, st));
  if (nVtxTotal == 0) return REINDEX_ERR_INDEX_RANGE;
  MergeLayout ML;
  ML.compute(nVtxTotal, S, M, nMeshes);
  if (ws == nullptr || !aligned(ws, 256) || wsBytes < ML.total) return REINDEX_ERR_INVALID_ARG;
  unsigned char* b = static_cast<unsigned char*>(ws);
  SegArgs seg;
  seg.vtxOff = vtxOffsets;
  seg.elemOff = elemOffsets;
  seg.outOff = reinterpret_cast<int64_t*>(b + ML.off_scratch);
  seg.blkV = reinterpret_cast<const uint32_t*>(b + ML.off_blkV);
  seg.blkI = reinterpret_cast<const uint32_t*>(b + ML.off_blkI);
  seg.nMeshes = nMeshes;
  seg.k = k;
  PipeExtras ex;
  ex.flags_done = true;  // the concatenation step marks the used vertices itself
  ex.pre = [&](const WsPtrs& p, const LaunchCfg& c) -> cudaError_t {
    // concatenate: local -> global indices (offset by the mesh's first vertex), range-checked
    cudaError_t e = launch_seg_prepare(seg, nVtxTotal, M, reinterpret_cast<uint32_t*>(b + ML.off_blkV),
                                       reinterpret_cast<uint32_t*>(b + ML.off_blkI), p.ctrl, c, st);
    if (e != cudaSuccess) return e;
    return launch_seg_flags(idx, out_idx, M, seg, p, c, st);
  };
  // Then the single-mesh method over the concatenation, reading the global indices in out_idx.
  return run_pipeline(vtx, nVtxTotal, S, out_idx, M, out_vtx, out_nVtx, out_idx, ws, ML.L, st, &ex);
}

// ---- subset of a mesh (Section 3.4) ---------------------------------------------------------------
size_t reindex_submesh_workspace_size(int64_t nVtx, int vtxStrideBytes, int64_t nSel, int idxPerElem) {
  return reindex_workspace_size(nVtx, vtxStrideBytes, nSel, idxPerElem);
}

reindex_status reindex_submesh(const void* vtx, int64_t nVtx, int S, const int32_t* idx, int64_t nElem, int k,
                               const int32_t* elemList, int64_t nSel, void* out_vtx, int64_t* out_nVtx,
                               int32_t* out_idx, void* ws, size_t wsBytes, reindex_stream_t stream) {
  int64_t M = 0, Mall = 0;
  reindex_status r = check_args(nVtx, S, nSel, k, &M);
  if (r != REINDEX_OK) return r;
  if ((r = check_args(nVtx, S, nElem, k, &Mall)) != REINDEX_OK) return r;
  if (nSel > 0 && (!elemList || !aligned(elemList, 4) || !idx)) return REINDEX_ERR_INVALID_ARG;
  if ((r = check_ptrs(vtx, nVtx, S, out_idx, M, out_vtx, out_nVtx, out_idx)) != REINDEX_OK) return r;
  if (out_idx == idx) return REINDEX_ERR_INVALID_ARG;  // the selection is gathered into out_idx first
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (M == 0) return cuda_status(launch_set_count(out_nVtx, 0, st));
  if (nVtx == 0) return REINDEX_ERR_INDEX_RANGE;
  WsLayout L;
  L.compute(nVtx, S, M);
  if (ws == nullptr || !aligned(ws, 256) || wsBytes < L.total) return REINDEX_ERR_INVALID_ARG;
  PipeExtras ex;
  ex.pre = [&](const WsPtrs& p, const LaunchCfg& c) -> cudaError_t {
    return launch_gather_elements(idx, k, nElem, elemList, nSel, out_idx, p, c, st);
  };
  // The selected elements, with the full vertex array, go through the method unchanged: the
  // vertices no selected element uses drop out as unused ones.
  return run_pipeline(vtx, nVtx, S, out_idx, M, out_vtx, out_nVtx, out_idx, ws, L, st, &ex);
}

reindex_status reindex_stream_status(reindex_stream_t stream) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return REINDEX_ERR_CUDA;
  uint32_t v = 0;
  if (read_and_clear_sticky(&v, st) != cudaSuccess) return REINDEX_ERR_CUDA;
  return (reindex_status)v;
}

void reindex_profile_enable(int on) {
  std::lock_guard<std::mutex> g(prof::mu);
  prof::enabled = on != 0;
}

int reindex_profile_collect(reindex_profile_record* out, int maxRecords) {
  std::vector<prof::Pending> recs;
  std::vector<uint8_t*> pins;
  {
    std::lock_guard<std::mutex> g(prof::mu);
    recs.swap(prof::pending);
    pins.swap(prof::pinned);
  }
  int bad = 0;
  for (size_t i = 0; i < recs.size(); ++i) {
    const prof::Pending& p = recs[i];
    float ms = 0.f;
    if (cudaEventSynchronize(p.b) != cudaSuccess || cudaEventElapsedTime(&ms, p.a, p.b) != cudaSuccess) bad = 1;
    if (out && (int)i < maxRecords) {
      out[i].kernel = p.kernel;
      out[i].digit = p.digit;
      out[i].skipped = (p.skip && p.digit >= 0) ? (int)p.skip[p.digit] : 0;
      out[i].item_bytes = p.item_bytes;
      out[i].ms = ms;
    }
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  for (uint8_t* h : pins) cudaFreeHost(h);
  return bad ? -1 : (int)recs.size();
}

void reindex_debug_stall_tile(int64_t tile) { g_stall_tile.store(tile < 0 ? -1 : tile); }

const char* reindex_kernel_name(int kernel) {
  static const char* names[REINDEX_K_COUNT] = {"clear",     "used_flags", "compact_hist", "sort_plan",
                                               "onesweep",  "head_scan",  "remap",        "finalize",
                                               "seg_prepare", "seg_offsets", "tile_count", "tile_offsets",
                                               "tile_scatter", "key_masks", "prefix_gate", "prefix_check",
                                               "chunk_scatter", "hash_dedup", "resolve"};
  return (kernel >= 0 && kernel < REINDEX_K_COUNT) ? names[kernel] : "unknown";
}

}  // extern "C"
