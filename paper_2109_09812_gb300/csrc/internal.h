// Host-side launch wrappers of the re-indexing kernels (one translation unit per kernel
// family so that they compile in parallel).  Internal; the public ABI is include/reindex.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "common.cuh"

namespace reindex {

struct LaunchCfg {
  int sms = 0;          // multiprocessors of the current device
  int occ_compact = 0;  // resident CTAs per SM of each persistent kernel
  int occ_sort = 0;
  int occ_head = 0;
  int occ_sort_pipe = 0;
  int occ_tiles = 0;
  int sort_kernel = kSortAuto;  // kSortRegs (k_onesweep), kSortPipe (k_onesweep_pipe), kSortTiles, kSortChunk,
                                // kSortAuto
  int rank_mode = kRankBallot;  // digit matching of the radix passes (kRank*; onesweep: ballot or match)
  int hist_mode = kHistUniform; // compaction histogram method (kHist*)
  int grid_per_tile = 0;        // 1: one CTA per tile; 0: persistent CTAs (SMs x occupancy)
  int scatter_waves = 0;        // "tiles" scatter: 0 one CTA per tile, else CTAs = waves x SMs x occupancy
  int pack_keys = -1;           // "tiles" sort: pack the varying key bits when that saves a pass
                                // (1 on, 0 off, -1 auto: keys of up to 8 bytes and batched calls)
  int prefix = -1;              // single meshes of 12- to 32-byte vertices: sort by the 64 most
                                // significant varying key bits first (1 on, 0 off, -1 auto: 16 bytes
                                // and wider)
  int chunk_cfg = 2;            // "chunk" sort tile shape: 0 big (4096-item tiles, 512 threads; 2048
                                // for items over 20 bytes), 1 small (2048-item tiles, 256 threads),
                                // 2 wide (2048-item tiles, 512 threads, 2 CTAs per SM), 3 deep
                                // (4096-item tiles, 1024 threads)
  int chunk_occ = 0;            // "chunk" sort: resident CTAs per SM to launch (0: as many as fit)
  int occ_chunk[4] = {0, 0, 0, 0};  // resident CTAs per SM of the chunk scatter, per tile shape
  int digit_bits = 8;           // "chunk" sort: radix digit width, 6, 7 or 8 bits (narrower digits take
                                // bit fields of the packed key: more passes, fewer ballots per pass,
                                // longer output runs); every other sort uses 8
  int chunk_grid_cap = 0;       // "chunk" sort: at most this many chunks (0: no cap; small caps give
                                // every CTA many tiles, e.g. to test the pipeline on small meshes)
  int dedup = 0;                // 1: remove duplicates with a hash table before the sort (keys of 8
                                // bytes and wider); the sort then orders the distinct keys only
  int dedup_pub = 1;            // 1: representatives publish their item positions in the hash table
};

// The "tiles" and "chunk" sorts take no upfront histograms: the compaction writes the first pass's
// digit plane (and the key bit masks), and each pass counts its digits itself.
inline bool uses_plane(int sort_kernel) { return sort_kernel == kSortTiles || sort_kernel == kSortChunk; }

// The configuration for one call: kSortAuto resolved for S-byte keys and up to Umax items.
// batched: the call sorts (mesh id, vertex) keys, whose mesh-id bytes are mostly constant.
// Large meshes take the "chunk" sort, small ones the onesweep sort (fewer launches); 24- and
// 32-byte keys take the "tiles" or "chunk" sort with vary ranking (the only variants built).
inline LaunchCfg resolve_cfg(LaunchCfg c, int S, int64_t Umax, bool batched = false) {
  if (S >= kWideMin) {
    if (c.sort_kernel != kSortChunk && c.sort_kernel != kSortTiles)
      c.sort_kernel = (c.sort_kernel == kSortAuto && Umax >= kTilesMinItems) ? kSortChunk : kSortTiles;
    c.rank_mode = kRankBallotVary;
  }
  if (S >= kHugeMin) {  // 48- and 64-byte keys: chunk sort of unpacked byte digits only
    c.sort_kernel = kSortChunk;
    c.pack_keys = 0;
    c.digit_bits = 8;
  }
  if (c.sort_kernel == kSortAuto) c.sort_kernel = Umax >= kTilesMinItems ? kSortChunk : kSortRegs;
  if (c.sort_kernel != kSortChunk || c.digit_bits < 6 || c.digit_bits > 8) c.digit_bits = 8;
  if (c.digit_bits < 8) c.pack_keys = 1;  // narrower digits are bit fields of the packed key
  if (c.pack_keys < 0) c.pack_keys = (batched || S <= 8) ? 1 : 0;
  if (batched || S <= kPrefixBytes)
    c.prefix = 0;
  else if (c.prefix < 0)  // 12-byte keys: the two passes saved do not pay for the check (GB300)
    c.prefix = S >= 16 ? 1 : 0;
  if (S < 8) c.dedup = 0;
  if (c.dedup && !c.prefix) {  // the hash table writes the plane of key byte 0 and the masks: unpacked
    c.pack_keys = 0;           // 8-bit digits (with the prefix sort, it marks the representatives and
    c.digit_bits = 8;          // the prefix path sorts them instead)
    if (!uses_plane(c.sort_kernel)) c.sort_kernel = kSortChunk;
  }
  return c;
}

// Launch with programmatic dependent launch: the kernel may be scheduled while the previous kernel
// on the stream finishes; it must call pdl_wait() before reading anything that kernel wrote.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), unsigned grid, unsigned block, size_t smem, cudaStream_t st,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Per-device launch configuration (computed once per device and stride, thread-safe).
LaunchCfg launch_cfg(int S);
void set_launch_cfg(int S, const LaunchCfg& c);
void apply_tuning(LaunchCfg& c, const char* spec);
std::string describe_tuning(const LaunchCfg& c);
// Tuning cache file (REINDEX_TUNE_CACHE): the spec stored for this device and stride, or "".
std::string tuning_from_cache(int dev, int sms, int S);

cudaError_t launch_clear(void* p, size_t bytes, const LaunchCfg& c, cudaStream_t st);
cudaError_t launch_used_flags(const int32_t* idx, int64_t M, int64_t nVtx, WsPtrs ws, const LaunchCfg& c,
                              cudaStream_t st);
// seg == nullptr: single mesh; otherwise batched, S being the vertex stride (items carry S + 4 bytes).
cudaError_t launch_compact(int S, const void* vtx, int64_t nVtx, WsPtrs ws, int64_t tilesV, const LaunchCfg& c,
                           const SegArgs* seg, cudaStream_t st);
// from_masks: trivial passes from the key bit masks (the "tiles" sort takes no upfront histograms).
// dbits < 8: digits of dbits bits of the packed key (chunk sort only; packing is forced).
cudaError_t launch_sort_plan(int S, WsPtrs ws, bool from_masks, bool allow_pack, cudaStream_t st, int dbits = 8);
// Radix passes the host launches for keyBytes-byte keys at a digit width (passes past the plan's
// last digit exit at once), and for the prefix sort's 64-bit prefixes.
int sort_passes(int keyBytes, int dbits);
inline int prefix_passes(int dbits) { return dbits >= 8 ? kPrefixBytes : (8 * kPrefixBytes + dbits - 1) / dbits; }
// Prefix sort (single meshes, S > 8): the plan keeping the 64 most significant varying key bits,
// the compaction into (prefix, old index) items, the head scan that checks whole keys, and the
// gate that skips the full-key sort unless two different keys shared a prefix.
cudaError_t launch_prefix_plan(int S, WsPtrs ws, cudaStream_t st, int dbits = 8);
cudaError_t launch_compact_prefix(int S, const void* vtx, int64_t nVtx, WsPtrs ws, int64_t tilesV, const LaunchCfg& c,
                                  cudaStream_t st);
cudaError_t launch_head_scan_prefix(int S, WsPtrs ws, const void* vtx, void* out_vtx, int64_t* out_nVtx,
                                    uint32_t nVtx, const LaunchCfg& c, cudaStream_t st);
cudaError_t launch_prefix_check(int S, const void* vtx, int64_t nVtx, const void* out_vtx, WsPtrs ws,
                                const LaunchCfg& c, cudaStream_t st);
cudaError_t launch_prefix_gate(WsPtrs pre, WsPtrs full, cudaStream_t st);
// Key bit masks over the used vertices (tiles sort; S is the vertex stride, seg as for the compaction).
cudaError_t launch_key_masks(int S, const void* vtx, int64_t nVtx, WsPtrs ws, const LaunchCfg& c, const SegArgs* seg,
                             cudaStream_t st);
cudaError_t launch_onesweep(int S, int digit, WsPtrs ws, const LaunchCfg& c, cudaStream_t st);
cudaError_t launch_onesweep_pipe(int S, int digit, WsPtrs ws, const LaunchCfg& c, cudaStream_t st);
// The "tiles" radix pass (k_radix_tiles.cu): per-tile digit counts, their scan, the scatter.
cudaError_t launch_tile_count(int S, int digit, WsPtrs ws, const LaunchCfg& c, cudaStream_t st);
cudaError_t launch_tile_offsets(int digit, WsPtrs ws, cudaStream_t st, int chunks = 0);
// The "chunk" radix pass (k_radix_chunk.cu): per-chunk digit counts, their scan (launch_tile_offsets
// with chunks = G), the pipelined scatter.  G = chunk_grid(...) for the whole call.
int chunk_tile_items(int S, int cfg);
int chunk_grid(int S, const LaunchCfg& c, int64_t Umax);
cudaError_t launch_chunk_count(int S, int digit, WsPtrs ws, int G, int T, cudaStream_t st);
cudaError_t launch_chunk_scatter(int S, int digit, WsPtrs ws, const LaunchCfg& c, int G, cudaStream_t st);
cudaError_t launch_tile_scatter(int S, int digit, WsPtrs ws, const LaunchCfg& c, cudaStream_t st);
// seg != nullptr: batched, S being the item key size (vertex stride + 4); writes seg->outOff.
cudaError_t launch_head_scan(int S, WsPtrs ws, void* out_vtx, int64_t* out_nVtx, uint32_t nVtx,
                             const LaunchCfg& c, const SegArgs* seg, cudaStream_t st);
// Batched helpers (batched.cu).
cudaError_t launch_seg_prepare(const SegArgs& seg, int64_t nVtx, int64_t M, uint32_t* blkV, uint32_t* blkI,
                               Control* ctrl, const LaunchCfg& c, cudaStream_t st);
cudaError_t launch_seg_flags(const int32_t* idx, int32_t* gidx, int64_t M, const SegArgs& seg, WsPtrs ws,
                             const LaunchCfg& c, cudaStream_t st);
cudaError_t launch_seg_offsets(const SegArgs& seg, const Control* ctrl, cudaStream_t st);
cudaError_t launch_seg_remap(int32_t* out_idx, int64_t M, const SegArgs& seg, WsPtrs ws, const LaunchCfg& c,
                             cudaStream_t st);
cudaError_t launch_remap(const int32_t* idx, int32_t* out_idx, int64_t M, WsPtrs ws, const LaunchCfg& c,
                         cudaStream_t st);
// int64 indices (reindex_mesh64*): the same two steps on 8-byte indices.
cudaError_t launch_used_flags64(const int64_t* idx, int64_t M, int64_t nVtx, WsPtrs ws, const LaunchCfg& c,
                                cudaStream_t st);
cudaError_t launch_remap64(const int64_t* idx, int64_t* out_idx, int64_t M, WsPtrs ws, const LaunchCfg& c,
                           cudaStream_t st);
cudaError_t launch_finalize(WsPtrs ws, int64_t* out_nVtx, cudaStream_t st);
// Duplicate removal before the sort (k_dedup.cu): the table takes the second item buffer.  A copy's
// oldToNew entry holds kRepTag | its representative's index until the remap looks that up (new
// indices stay below 2^31, so an untagged entry is a new index).
constexpr uint32_t kRepTag = 0x80000000u;
uint32_t dedup_table_slots(const WsLayout& L);
// seg: batched calls ((mesh id, vertex) keys of S + 4 bytes; S = 4 to 16).  [vlo, vhi): the vertices
// this launch inserts (vlo a multiple of 32; vhi < 0: to the end).
// repmask: representatives replace the used bits instead of appending items (single meshes whose
// sort runs on key prefixes: 12-byte keys and wider; the prefix path then sorts them).
cudaError_t launch_hash_dedup(int S, const void* vtx, int64_t nVtx, WsPtrs ws, uint32_t slots, uint32_t cap,
                              const LaunchCfg& c, cudaStream_t st, const SegArgs* seg = nullptr, int64_t vlo = 0,
                              int64_t vhi = -1, bool repmask = false);
// out = oldToNew[idx], a tagged entry through its representative (int32 or, with wide, int64 indices)
cudaError_t launch_remap_rep(const void* idx, void* out, bool wide, int64_t M, WsPtrs ws, const LaunchCfg& c,
                             cudaStream_t st);
cudaError_t launch_resolve(int64_t nVtx, WsPtrs ws, const LaunchCfg& c, cudaStream_t st);
// Meshes of more than 2^31 - 1 vertices, re-indexed in vertex ranges (k_simple.cu)
cudaError_t launch_used_flags_range64(const int64_t* idx, int64_t M, int64_t lo, int64_t n, int64_t N, WsPtrs ws,
                                      bool check, const LaunchCfg& c, cudaStream_t st);
cudaError_t launch_iota(int32_t* out, int64_t n, const LaunchCfg& c, cudaStream_t st);
cudaError_t launch_remap_two_level(const int64_t* idx, int64_t* out, int64_t M, const uint32_t* rank,
                                   const int64_t* part_off, const int32_t* map2, int shift, const LaunchCfg& c,
                                   cudaStream_t st);
cudaError_t launch_gather_elements(const int32_t* idx, int k, int64_t nElem, const int32_t* list, int64_t nSel,
                                  int32_t* out, WsPtrs ws, const LaunchCfg& c, cudaStream_t st);
cudaError_t launch_set_count(int64_t* out_nVtx, int64_t value, cudaStream_t st);

// Test hook: compaction tile that withholds its look-back status (-1: none).
int64_t debug_stall_tile();

// Occupancy queries for the persistent kernels (per template instantiation).
int occupancy_compact(int S);
int occupancy_sort(int S);
int occupancy_sort_pipe(int S);
int occupancy_tiles(int S);
int occupancy_chunk(int S, int cfg);
int occupancy_head(int S);

// Device-wide sticky error word (read and cleared by reindex_stream_status).
cudaError_t read_and_clear_sticky(uint32_t* value, cudaStream_t st);

}  // namespace reindex
