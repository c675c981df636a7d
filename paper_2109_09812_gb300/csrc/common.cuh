// Internal definitions shared by the kernels and the host orchestration of the re-indexing
// library: workspace layout, item layouts of the sort, decoupled look-back primitives and
// warp/block scans.  Nothing here is part of the public ABI (include/reindex.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace reindex {

// ---------------------------------------------------------------------------------------------
// Tunables (compile-time tile shapes; the look-back tables are sized from them).
constexpr int kThreads = 256;              // threads per CTA for every tiled kernel
constexpr int kWarps = kThreads / 32;
constexpr int kCompactRows = 8;            // 32-vertex rows per warp in the compaction
constexpr int kCompactTile = kWarps * kCompactRows * 32;   // 2048 vertices per tile
constexpr int kSortThreads = 512;          // threads per CTA of a sort pass
constexpr int kSortIpt = 8;                // items per thread in a sort pass
constexpr int kSortTile = kSortThreads * kSortIpt;         // 4096 items per tile
constexpr int kSortTileMin = 2048;         // smallest sort tile of any variant (sizes the look-back)
constexpr int kHeadThreads = 256;          // threads per CTA of the head scan
constexpr int kHeadIpt = 8;                // items per thread in the head scan
constexpr int kHeadTile = kHeadThreads * kHeadIpt;         // 2048 items per tile
constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;    // 256 digit values (narrower digits use the low bins)
constexpr int kMaxDigits = 64;             // 64-byte keys -> 64 byte digits
constexpr int kMaxKeyWords = kMaxDigits / 4;  // 16 words per key at most
constexpr int kHugeMin = 48;               // keys of 48 and 64 bytes: prefix sort, chunk-sort fallback only
constexpr int kPrefixBytes = 8;           // prefix sort: keys cut to their 64 most significant varying bits,
constexpr int kPrefixItem = 12;           // held in 12-byte item keys (word 0 zero: 16-byte records)
constexpr int kWideMin = 24;               // keys of 24 and 32 bytes (single meshes) use the "tiles"
                                           // sort with vary ranking only (fewer kernel variants)

// Kernel variants (chosen per device by launch_cfg; see REINDEX_TUNE in api.cu).
constexpr int kSortRegs = 0;      // radix pass with items in registers (k_onesweep)
constexpr int kSortPipe = 1;      // radix pass pipelined through shared memory (k_onesweep_pipe)
constexpr int kSortTiles = 2;     // radix pass with precounted tile offsets (k_radix_tiles.cu)
constexpr int kSortAuto = 3;      // per call: kSortChunk for large meshes, else kSortRegs (the faster
                                  // on GB300 for each)
constexpr int kSortChunk = 4;     // radix pass over contiguous chunks with bulk-copied tiles (k_radix_chunk.cu)
constexpr int64_t kTilesMinItems = 1 << 21;  // below this, launch count favours kSortRegs
constexpr int kRankBallot = 0;    // digit peers from 8 ballots
constexpr int kRankMatchAny = 1;  // digit peers from match.any
constexpr int kRankBallotVary = 2;  // ballots on the digit bits that vary only
constexpr int kHistUniform = 0;   // histogram: one atomic per warp when the digit is warp-uniform
constexpr int kHistPeel = 1;      // histogram: the first lane's digit group counted with one atomic
constexpr int kHistMatchAny = 2;  // histogram: one atomic per distinct digit (match.any)
constexpr int kHistNone = 3;      // no histograms: packed keys and the first pass's digit plane instead
constexpr int kHistMasks = 4;     // no histograms: key bit masks and the plane of key byte 0 instead
                                  // (the "tiles" sort counts digits per pass itself)
constexpr int kHistPrefix = 5;    // prefix sort: items carry the 64 most significant varying key bits

// Look-back status word (one 32-bit word, zeroed before use):
//   0                      not published yet;
//   top bit clear, v > 0   the tile's aggregate only, v - 1 (an aggregate is at most a tile);
//   top bit set            the inclusive prefix through the tile, in the low 31 bits.
// Counts up to 2^31 - 1 fit, so meshes of up to INT32_MAX vertices can be re-indexed.
constexpr uint32_t kPreBit = 1u << 31;
constexpr uint32_t kValMask = kPreBit - 1;
constexpr int64_t kMaxCount = (int64_t)kValMask;  // largest count a status word can carry
__host__ __device__ constexpr uint32_t lb_agg(uint32_t count) { return count + 1u; }
__host__ __device__ constexpr uint32_t lb_pre(uint32_t count) { return kPreBit | (count & kValMask); }
__host__ __device__ constexpr bool lb_ready(uint32_t s) { return s != 0u; }
__host__ __device__ constexpr bool lb_is_pre(uint32_t s) { return (s & kPreBit) != 0u; }
__host__ __device__ constexpr uint32_t lb_val(uint32_t s) { return lb_is_pre(s) ? (s & kValMask) : s - 1u; }
static_assert(!lb_ready(0u) && lb_ready(lb_agg(0)) && lb_ready(lb_pre(0)), "published statuses are non-zero");
static_assert(lb_val(lb_agg(0)) == 0 && lb_val(lb_agg(65536)) == 65536 && !lb_is_pre(lb_agg(65536)), "aggregates");
static_assert(lb_val(lb_pre(0)) == 0 && lb_val(lb_pre((uint32_t)kMaxCount)) == (uint32_t)kMaxCount &&
                  lb_is_pre(lb_pre((uint32_t)kMaxCount)) && kMaxCount == 2147483647,
              "inclusive prefixes up to INT32_MAX");

// Bounded spin: every wait on another CTA gives up after this many polls, records
// REINDEX_ERR_TIMEOUT and publishes a (meaningless) prefix so that no successor waits forever.
constexpr uint32_t kSpinLimit = 1u << 20;
// Single-counter look-back tables (compaction, head scan) keep each tile's status word in its own
// kLbPad-word slot (one 128-byte line), so that the hundreds of CTAs polling recent tiles do not
// all hit one L2 line (packed status words made both kernels about 1.5x slower).
constexpr int kLbPad = 32;

// Device-side error codes (same numbers as reindex_status).
constexpr uint32_t kErrIndexRange = 4;
constexpr uint32_t kErrTimeout = 5;
constexpr uint32_t kErrInternal = 7;
// Not an error: set in the control block of a call's full-key sort when its prefix sort already
// produced the result (every kernel of the full-key sort then returns at once).
constexpr uint32_t kErrSkip = 0x100;

// ---------------------------------------------------------------------------------------------
// Workspace.
struct Control {             // zeroed at the start of every call
  uint32_t err;              // first device-detected error (0 = none)
  uint32_t U;                // number of used vertices (written by the last compaction tile)
  uint32_t ctr[2 + kMaxDigits];  // atomic tile counters: [0] compaction, [1 + d] sort digit d,
                                 // [1 + kMaxDigits] head scan
  uint32_t kor[kMaxKeyWords];     // OR of key word q over the used vertices (compaction, kHistNone)
  uint32_t knand[kMaxKeyWords];   // OR of the complement: bit b varies iff set in both masks
  uint32_t amb;                   // prefix sort: two different keys share a prefix (1)
  uint32_t pad[27];
};
static_assert(sizeof(Control) == 512, "Control block is two 256-byte lines");

// Key packing for the "tiles" sort.  Bits that are equal in every item do not affect the order,
// so the compaction can pack the varying bits of each key (runs of consecutive bits, least
// significant first) into the low bits of the key, and the radix passes sort byte digits of that
// packed key: fewer passes when many bits are constant (integer coordinates, exponent bits, the
// high bytes of a mesh id).  Packed keys are equal exactly when the keys are; the head scan
// restores the keys it writes out.
constexpr int kMaxPackRuns = 16;
struct KeyPack {
  uint8_t on;                      // 1: the keys are packed
  uint8_t nbits;                   // varying bits in all
  uint8_t nruns;                   // runs, least significant first
  uint8_t word[kMaxPackRuns];      // key word of run r (word 0 is the most significant)
  uint8_t shift[kMaxPackRuns];     // lowest bit of the run within that word
  uint8_t len[kMaxPackRuns];       // run length in bits
  uint8_t pos[kMaxPackRuns];       // where the run starts in the packed key
  uint8_t simple;                  // 1: at most one run per word (wshift / wlen describe them)
  uint8_t wshift[kMaxKeyWords];    // word q's run: lowest bit
  uint8_t wlen[kMaxKeyWords];      //               and length (0: no varying bit)
  uint8_t pad[4];
};
static_assert(sizeof(KeyPack) == 104, "KeyPack layout");

struct Plan {                // written by the sort-plan kernel
  uint32_t U;
  uint32_t final_sel;        // 0: sorted items end in buffer A, 1: in buffer B
  uint8_t skip[kMaxDigits];  // 1: digit d is constant over all items; its pass moves nothing
  uint8_t src[kMaxDigits];   // buffer the pass for digit d reads (0 = A, 1 = B)
  uint8_t area[kMaxDigits];  // which of the two look-back areas the pass uses
  int8_t next[kMaxDigits];   // the next non-trivial digit after d, or -1
  int8_t first;              // the first non-trivial digit, or -1
  uint8_t plane_first;       // tiles sort: the compaction's digit plane holds the first pass's digit
                             // (else key byte 0)
  uint8_t dbits;             // digit width: 8 (key bytes), or 6 / 7 bits of a packed key (chunk sort)
  uint8_t pad[9];
  uint8_t vary[kMaxDigits];  // bits of digit d that differ between items (the others are constant)
  uint8_t pad2[12];
  KeyPack pack;                      // packing of the keys (pack.on == 0: not packed)
  uint32_t kconst[kMaxKeyWords];     // values of the constant key bits (to restore packed keys)
  uint32_t base[kMaxDigits][kRadix];  // exclusive prefix of the digit histogram
};

constexpr size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Item buffers of S-byte keys: structure of arrays (a key plane, then an id plane) for S = 8, 16,
// 24 and 32; array of structures {key, id} for S = 4, 12 and 20.
__host__ __device__ constexpr bool soa_items(int S) { return S % 8 == 0; }

struct WsLayout {
  int S = 0, K = 0, P = 0;
  int64_t nVtx = 0, M = 0, Umax = 0;
  int64_t tilesV = 0, tilesS = 0, tilesH = 0;
  size_t off_ctrl = 0, off_hist = 0, off_lb_compact = 0, off_lb_head = 0, off_lb_sort = 0,
         off_bitmask = 0, zero_bytes = 0;
  size_t off_plan = 0, off_itemsA = 0, off_itemsB = 0, items_bytes = 0, idoff = 0, off_old2new = 0, off_digits = 0,
         total = 0;
  size_t off_ctrl_pre = 0;  // prefix sort: its control block

  constexpr void compute(int64_t n, int s, int64_t m) {
    S = s; K = s / 4; P = s; nVtx = n; M = m;
    Umax = n < m ? n : m;
    tilesV = (n + kCompactTile - 1) / kCompactTile;
    tilesS = (Umax + kSortTileMin - 1) / kSortTileMin;  // enough for every sort kernel variant
    tilesH = (Umax + kHeadTile - 1) / kHeadTile;
    size_t o = 0;
    off_ctrl = o;        o += sizeof(Control);
    off_hist = o;        o = align_up(o + (size_t)kMaxDigits * kRadix * 4, 256);  // a row per pass
    off_lb_compact = o;  o = align_up(o + (size_t)tilesV * 4 * kLbPad, 256);
    off_lb_head = o;     o = align_up(o + (size_t)tilesH * 4 * kLbPad, 256);
    off_lb_sort = o;     o = align_up(o + (size_t)2 * tilesS * kRadix * 4, 256);
    off_bitmask = o;     o = align_up(o + (size_t)((n + 31) / 32) * 4, 256);
    zero_bytes = o;
    off_ctrl_pre = o;    o += sizeof(Control);  // the prefix sort's control block (outside the full sort's zeroing)
    off_plan = o;        o = align_up(o + sizeof(Plan), 256);
    // SoA layouts keep the id plane 256-byte aligned; 256 spare bytes let bulk copies of a
    // ragged last tile round their size up to 16 bytes without leaving the buffer.
    idoff = soa_items(S) ? align_up((size_t)Umax * S, 256) : 0;
    items_bytes = soa_items(S) ? idoff + align_up((size_t)Umax * 4, 256) + 256
                               : align_up((size_t)Umax * (size_t)(S + 4), 256) + 256;
    if (S > kPrefixBytes) {  // the prefix sort's items (16-byte records) share the item buffers
      const size_t pre = align_up((size_t)Umax * (kPrefixItem + 4), 256) + 256;
      if (pre > items_bytes) items_bytes = pre;
    }
    off_itemsA = o;      o += items_bytes;
    off_itemsB = o;      o += items_bytes;
    off_old2new = o;     o = align_up(o + (size_t)n * 4, 256);
    off_digits = o;      o = align_up(o + (size_t)align_up((size_t)Umax, kSortTile), 256);  // whole tiles
    total = o;
  }
};

// Workspace bytes of one single-mesh call (usable in constant expressions).
constexpr size_t ws_bytes(int64_t n, int s, int64_t m) {
  WsLayout L{};
  L.compute(n, s, m);
  return L.total;
}

// Device views of the workspace, passed by value to the kernels.
struct WsPtrs {
  Control* ctrl;
  uint32_t* hist;        // [kMaxDigits][256]: digit totals of each pass
  uint32_t* lb_compact;  // [tilesV * kLbPad]: status of tile q at q * kLbPad
  uint32_t* lb_head;     // [tilesH * kLbPad]
  uint32_t* lb_sort;     // [2][tilesS][256]
  uint32_t* bitmask;     // [ceil(nVtx/32)]
  Plan* plan;
  unsigned char* itemsA;
  unsigned char* itemsB;
  uint32_t* old2new;     // [nVtx]
  uint8_t* digits;       // [Umax rounded up to whole sort tiles]: each item's digit of the next radix
                         // pass (of the first one: written by the compaction)
  int64_t tilesS;        // capacity of the sort look-back table, in tiles
  int64_t Umax;          // capacity of each item buffer, in items
  int64_t idoff;         // byte offset of the id plane inside an item buffer (S = 8, 16, 24, 32)
};

inline WsPtrs ws_ptrs(void* ws, const WsLayout& L) {
  unsigned char* b = static_cast<unsigned char*>(ws);
  WsPtrs p;
  p.ctrl = reinterpret_cast<Control*>(b + L.off_ctrl);
  p.hist = reinterpret_cast<uint32_t*>(b + L.off_hist);
  p.lb_compact = reinterpret_cast<uint32_t*>(b + L.off_lb_compact);
  p.lb_head = reinterpret_cast<uint32_t*>(b + L.off_lb_head);
  p.lb_sort = reinterpret_cast<uint32_t*>(b + L.off_lb_sort);
  p.bitmask = reinterpret_cast<uint32_t*>(b + L.off_bitmask);
  p.plan = reinterpret_cast<Plan*>(b + L.off_plan);
  p.itemsA = b + L.off_itemsA;
  p.itemsB = b + L.off_itemsB;
  p.old2new = reinterpret_cast<uint32_t*>(b + L.off_old2new);
  p.digits = b + L.off_digits;
  p.tilesS = L.tilesS;
  p.Umax = L.Umax;
  p.idoff = (int64_t)L.idoff;
  return p;
}

// The prefix sort's view: its own control block, 16-byte {0, prefix, old index} records in the
// same item buffers; the other tables are shared with the full-key sort, which runs (or is
// skipped) after it.
inline WsPtrs ws_ptrs_prefix(void* ws, const WsLayout& L) {
  WsPtrs p = ws_ptrs(ws, L);
  p.ctrl = reinterpret_cast<Control*>(static_cast<unsigned char*>(ws) + L.off_ctrl_pre);
  p.idoff = 0;  // array of structures
  return p;
}

// ---------------------------------------------------------------------------------------------
// Batched (segmented) re-indexing: many meshes concatenated, mesh m owning vertices
// [vtxOff[m], vtxOff[m+1]) and indices [elemOff[m]*k, elemOff[m+1]*k).  The mesh id becomes the
// most significant key word, so one sort orders all items by (mesh, vertex key).
constexpr int kSegBlock = 1024;  // granularity of the position -> mesh lookup tables

struct SegArgs {
  const int64_t* vtxOff;   // [nMeshes+1] device
  const int64_t* elemOff;  // [nMeshes+1] device
  int64_t* outOff;         // [nMeshes+1] device: first output vertex of each mesh; [nMeshes] = D
  const uint32_t* blkV;    // mesh of vertex b*kSegBlock
  const uint32_t* blkI;    // mesh of index b*kSegBlock
  int32_t nMeshes;
  int32_t k;               // indices per element
};

// Mesh owning position pos, given the mesh of pos's block and the offsets (scaled by `scale`).
// The walk never passes the last mesh, whatever the offsets hold.
__device__ __forceinline__ uint32_t seg_mesh(int64_t pos, const int64_t* off, int64_t scale, const uint32_t* blk,
                                             int32_t nMeshes) {
  uint32_t m = __ldg(blk + (pos / kSegBlock));
  while ((int32_t)m + 1 < nMeshes && __ldg(off + m + 1) * scale <= pos) ++m;
  return m;
}

// ---------------------------------------------------------------------------------------------
// Sort items: K key words (word 0 most significant) plus the old vertex index.
//   S = 4, 12: array of structures, one 8- or 16-byte vector per item {k..., id}
//   S = 20:    array of structures, three 8-byte vectors per item {k0,k1}{k2,k3}{k4,id}
//   S = 8, 16: structure of arrays, an 8- or 16-byte key vector per item, then an id plane
//              starting at byte offset idoff (256-byte aligned)
//   S = 24, 32: structure of arrays, three 8-byte or two 16-byte vectors per key, then the id plane
template <int S>
struct Item {
  static constexpr int K = S / 4;
  uint32_t k[K];
  uint32_t id;
};

template <int S>
struct ItemIO;

template <>
struct ItemIO<4> {
  static __device__ __forceinline__ void load(const unsigned char* buf, int64_t, int64_t i, Item<4>& it) {
    uint2 v = reinterpret_cast<const uint2*>(buf)[i];
    it.k[0] = v.x; it.id = v.y;
  }
  static __device__ __forceinline__ void load_cs(const unsigned char* buf, int64_t, int64_t i, Item<4>& it) {
    uint2 v = __ldcs(reinterpret_cast<const uint2*>(buf) + i);
    it.k[0] = v.x; it.id = v.y;
  }
  static __device__ __forceinline__ void store(unsigned char* buf, int64_t, int64_t i, const Item<4>& it) {
    reinterpret_cast<uint2*>(buf)[i] = make_uint2(it.k[0], it.id);
  }
};

template <>
struct ItemIO<12> {
  static __device__ __forceinline__ void load(const unsigned char* buf, int64_t, int64_t i, Item<12>& it) {
    uint4 v = reinterpret_cast<const uint4*>(buf)[i];
    it.k[0] = v.x; it.k[1] = v.y; it.k[2] = v.z; it.id = v.w;
  }
  static __device__ __forceinline__ void load_cs(const unsigned char* buf, int64_t, int64_t i, Item<12>& it) {
    uint4 v = __ldcs(reinterpret_cast<const uint4*>(buf) + i);
    it.k[0] = v.x; it.k[1] = v.y; it.k[2] = v.z; it.id = v.w;
  }
  static __device__ __forceinline__ void store(unsigned char* buf, int64_t, int64_t i, const Item<12>& it) {
    reinterpret_cast<uint4*>(buf)[i] = make_uint4(it.k[0], it.k[1], it.k[2], it.id);
  }
};

template <>
struct ItemIO<8> {
  static __device__ __forceinline__ void load(const unsigned char* buf, int64_t idoff, int64_t i, Item<8>& it) {
    uint2 v = reinterpret_cast<const uint2*>(buf)[i];
    it.k[0] = v.x; it.k[1] = v.y;
    it.id = reinterpret_cast<const uint32_t*>(buf + idoff)[i];
  }
  static __device__ __forceinline__ void load_cs(const unsigned char* buf, int64_t idoff, int64_t i, Item<8>& it) {
    uint2 v = __ldcs(reinterpret_cast<const uint2*>(buf) + i);
    it.k[0] = v.x; it.k[1] = v.y;
    it.id = __ldcs(reinterpret_cast<const uint32_t*>(buf + idoff) + i);
  }
  static __device__ __forceinline__ void store(unsigned char* buf, int64_t idoff, int64_t i, const Item<8>& it) {
    reinterpret_cast<uint2*>(buf)[i] = make_uint2(it.k[0], it.k[1]);
    reinterpret_cast<uint32_t*>(buf + idoff)[i] = it.id;
  }
};

template <>
struct ItemIO<16> {
  static __device__ __forceinline__ void load(const unsigned char* buf, int64_t idoff, int64_t i, Item<16>& it) {
    uint4 v = reinterpret_cast<const uint4*>(buf)[i];
    it.k[0] = v.x; it.k[1] = v.y; it.k[2] = v.z; it.k[3] = v.w;
    it.id = reinterpret_cast<const uint32_t*>(buf + idoff)[i];
  }
  static __device__ __forceinline__ void load_cs(const unsigned char* buf, int64_t idoff, int64_t i, Item<16>& it) {
    uint4 v = __ldcs(reinterpret_cast<const uint4*>(buf) + i);
    it.k[0] = v.x; it.k[1] = v.y; it.k[2] = v.z; it.k[3] = v.w;
    it.id = __ldcs(reinterpret_cast<const uint32_t*>(buf + idoff) + i);
  }
  static __device__ __forceinline__ void store(unsigned char* buf, int64_t idoff, int64_t i, const Item<16>& it) {
    reinterpret_cast<uint4*>(buf)[i] = make_uint4(it.k[0], it.k[1], it.k[2], it.k[3]);
    reinterpret_cast<uint32_t*>(buf + idoff)[i] = it.id;
  }
};

template <>
struct ItemIO<20> {
  static __device__ __forceinline__ void load(const unsigned char* buf, int64_t, int64_t i, Item<20>& it) {
    const uint2* p = reinterpret_cast<const uint2*>(buf) + 3 * i;
    const uint2 a = p[0], b = p[1], c = p[2];
    it.k[0] = a.x; it.k[1] = a.y; it.k[2] = b.x; it.k[3] = b.y; it.k[4] = c.x; it.id = c.y;
  }
  static __device__ __forceinline__ void load_cs(const unsigned char* buf, int64_t, int64_t i, Item<20>& it) {
    const uint2* p = reinterpret_cast<const uint2*>(buf) + 3 * i;
    const uint2 a = __ldcs(p), b = __ldcs(p + 1), c = __ldcs(p + 2);
    it.k[0] = a.x; it.k[1] = a.y; it.k[2] = b.x; it.k[3] = b.y; it.k[4] = c.x; it.id = c.y;
  }
  static __device__ __forceinline__ void store(unsigned char* buf, int64_t, int64_t i, const Item<20>& it) {
    uint2* p = reinterpret_cast<uint2*>(buf) + 3 * i;
    p[0] = make_uint2(it.k[0], it.k[1]);
    p[1] = make_uint2(it.k[2], it.k[3]);
    p[2] = make_uint2(it.k[4], it.id);
  }
};

template <>
struct ItemIO<24> {
  static __device__ __forceinline__ void load(const unsigned char* buf, int64_t idoff, int64_t i, Item<24>& it) {
    const uint2* p = reinterpret_cast<const uint2*>(buf) + 3 * i;
    const uint2 a = p[0], b = p[1], c = p[2];
    it.k[0] = a.x; it.k[1] = a.y; it.k[2] = b.x; it.k[3] = b.y; it.k[4] = c.x; it.k[5] = c.y;
    it.id = reinterpret_cast<const uint32_t*>(buf + idoff)[i];
  }
  static __device__ __forceinline__ void load_cs(const unsigned char* buf, int64_t idoff, int64_t i, Item<24>& it) {
    const uint2* p = reinterpret_cast<const uint2*>(buf) + 3 * i;
    const uint2 a = __ldcs(p), b = __ldcs(p + 1), c = __ldcs(p + 2);
    it.k[0] = a.x; it.k[1] = a.y; it.k[2] = b.x; it.k[3] = b.y; it.k[4] = c.x; it.k[5] = c.y;
    it.id = __ldcs(reinterpret_cast<const uint32_t*>(buf + idoff) + i);
  }
  static __device__ __forceinline__ void store(unsigned char* buf, int64_t idoff, int64_t i, const Item<24>& it) {
    uint2* p = reinterpret_cast<uint2*>(buf) + 3 * i;
    p[0] = make_uint2(it.k[0], it.k[1]);
    p[1] = make_uint2(it.k[2], it.k[3]);
    p[2] = make_uint2(it.k[4], it.k[5]);
    reinterpret_cast<uint32_t*>(buf + idoff)[i] = it.id;
  }
};

template <>
struct ItemIO<32> {
  static __device__ __forceinline__ void load(const unsigned char* buf, int64_t idoff, int64_t i, Item<32>& it) {
    const uint4* p = reinterpret_cast<const uint4*>(buf) + 2 * i;
    const uint4 a = p[0], b = p[1];
    it.k[0] = a.x; it.k[1] = a.y; it.k[2] = a.z; it.k[3] = a.w;
    it.k[4] = b.x; it.k[5] = b.y; it.k[6] = b.z; it.k[7] = b.w;
    it.id = reinterpret_cast<const uint32_t*>(buf + idoff)[i];
  }
  static __device__ __forceinline__ void load_cs(const unsigned char* buf, int64_t idoff, int64_t i, Item<32>& it) {
    const uint4* p = reinterpret_cast<const uint4*>(buf) + 2 * i;
    const uint4 a = __ldcs(p), b = __ldcs(p + 1);
    it.k[0] = a.x; it.k[1] = a.y; it.k[2] = a.z; it.k[3] = a.w;
    it.k[4] = b.x; it.k[5] = b.y; it.k[6] = b.z; it.k[7] = b.w;
    it.id = __ldcs(reinterpret_cast<const uint32_t*>(buf + idoff) + i);
  }
  static __device__ __forceinline__ void store(unsigned char* buf, int64_t idoff, int64_t i, const Item<32>& it) {
    uint4* p = reinterpret_cast<uint4*>(buf) + 2 * i;
    p[0] = make_uint4(it.k[0], it.k[1], it.k[2], it.k[3]);
    p[1] = make_uint4(it.k[4], it.k[5], it.k[6], it.k[7]);
    reinterpret_cast<uint32_t*>(buf + idoff)[i] = it.id;
  }
};

// 48- and 64-byte keys: structure of arrays, three or four 16-byte vectors per key, then the id plane.
template <int S>
struct ItemIOWide {
  static_assert(S % 16 == 0 && S > 32, "wide key layouts");
  static constexpr int V = S / 16;
  static __device__ __forceinline__ void load(const unsigned char* buf, int64_t idoff, int64_t i, Item<S>& it) {
    const uint4* p = reinterpret_cast<const uint4*>(buf) + V * i;
#pragma unroll
    for (int h = 0; h < V; ++h) {
      const uint4 v = p[h];
      it.k[4 * h] = v.x; it.k[4 * h + 1] = v.y; it.k[4 * h + 2] = v.z; it.k[4 * h + 3] = v.w;
    }
    it.id = reinterpret_cast<const uint32_t*>(buf + idoff)[i];
  }
  static __device__ __forceinline__ void load_cs(const unsigned char* buf, int64_t idoff, int64_t i, Item<S>& it) {
    const uint4* p = reinterpret_cast<const uint4*>(buf) + V * i;
#pragma unroll
    for (int h = 0; h < V; ++h) {
      const uint4 v = __ldcs(p + h);
      it.k[4 * h] = v.x; it.k[4 * h + 1] = v.y; it.k[4 * h + 2] = v.z; it.k[4 * h + 3] = v.w;
    }
    it.id = __ldcs(reinterpret_cast<const uint32_t*>(buf + idoff) + i);
  }
  static __device__ __forceinline__ void store(unsigned char* buf, int64_t idoff, int64_t i, const Item<S>& it) {
    uint4* p = reinterpret_cast<uint4*>(buf) + V * i;
#pragma unroll
    for (int h = 0; h < V; ++h) p[h] = make_uint4(it.k[4 * h], it.k[4 * h + 1], it.k[4 * h + 2], it.k[4 * h + 3]);
    reinterpret_cast<uint32_t*>(buf + idoff)[i] = it.id;
  }
};
template <>
struct ItemIO<48> : ItemIOWide<48> {};
template <>
struct ItemIO<64> : ItemIOWide<64> {};

// Vertex key loads from the caller's vertex array (stride S, natural alignment).
// (streaming: the caller's vertex array is read once per call)
template <int S>
__device__ __forceinline__ void load_key(const void* vtx, int64_t i, uint32_t (&k)[S / 4]) {
  if constexpr (S == 4) {
    k[0] = __ldcs(reinterpret_cast<const uint32_t*>(vtx) + i);
  } else if constexpr (S == 8) {
    uint2 v = __ldcs(reinterpret_cast<const uint2*>(vtx) + i);
    k[0] = v.x; k[1] = v.y;
  } else if constexpr (S == 12) {
    const uint32_t* p = reinterpret_cast<const uint32_t*>(vtx) + i * 3;
    k[0] = __ldcs(p); k[1] = __ldcs(p + 1); k[2] = __ldcs(p + 2);
  } else if constexpr (S == 16) {
    uint4 v = __ldcs(reinterpret_cast<const uint4*>(vtx) + i);
    k[0] = v.x; k[1] = v.y; k[2] = v.z; k[3] = v.w;
  } else if constexpr (S == 24) {
    const uint2* p = reinterpret_cast<const uint2*>(vtx) + 3 * i;
    const uint2 a = __ldcs(p), b = __ldcs(p + 1), c = __ldcs(p + 2);
    k[0] = a.x; k[1] = a.y; k[2] = b.x; k[3] = b.y; k[4] = c.x; k[5] = c.y;
  } else if constexpr (S % 16 == 0) {  // 32, 48, 64 bytes: 16-byte vectors
    const uint4* p = reinterpret_cast<const uint4*>(vtx) + (S / 16) * i;
#pragma unroll
    for (int h = 0; h < S / 16; ++h) {
      const uint4 a = __ldcs(p + h);
      k[4 * h] = a.x; k[4 * h + 1] = a.y; k[4 * h + 2] = a.z; k[4 * h + 3] = a.w;
    }
  } else {
    const uint32_t* p = reinterpret_cast<const uint32_t*>(vtx) + i * (S / 4);
#pragma unroll
    for (int q = 0; q < S / 4; ++q) k[q] = __ldcs(p + q);
  }
}

// Vertex key load through the read-only cache, for random accesses (natural alignment).
template <int S>
__device__ __forceinline__ void load_key_ro(const void* vtx, uint32_t i, uint32_t (&k)[S / 4]) {
  if constexpr (S % 16 == 0) {
    const uint4* p = reinterpret_cast<const uint4*>(vtx) + (size_t)i * (S / 16);
#pragma unroll
    for (int h = 0; h < S / 16; ++h) {
      const uint4 v = __ldg(p + h);
      k[4 * h] = v.x; k[4 * h + 1] = v.y; k[4 * h + 2] = v.z; k[4 * h + 3] = v.w;
    }
  } else if constexpr (S == 8 || S == 24) {
    const uint2* p = reinterpret_cast<const uint2*>(vtx) + (size_t)i * (S / 8);
#pragma unroll
    for (int h = 0; h < S / 8; ++h) {
      const uint2 v = __ldg(p + h);
      k[2 * h] = v.x; k[2 * h + 1] = v.y;
    }
  } else {
    const uint32_t* p = reinterpret_cast<const uint32_t*>(vtx) + (size_t)i * (S / 4);
#pragma unroll
    for (int q = 0; q < S / 4; ++q) k[q] = __ldg(p + q);
  }
}

// (streaming: the caller's output vertex array is written once)
template <int S>
__device__ __forceinline__ void store_key(void* out, int64_t i, const uint32_t (&k)[S / 4]) {
  if constexpr (S == 4) {
    __stcs(reinterpret_cast<uint32_t*>(out) + i, k[0]);
  } else if constexpr (S == 8) {
    __stcs(reinterpret_cast<uint2*>(out) + i, make_uint2(k[0], k[1]));
  } else if constexpr (S == 12) {
    uint32_t* p = reinterpret_cast<uint32_t*>(out) + i * 3;
    __stcs(p, k[0]); __stcs(p + 1, k[1]); __stcs(p + 2, k[2]);
  } else if constexpr (S == 16) {
    __stcs(reinterpret_cast<uint4*>(out) + i, make_uint4(k[0], k[1], k[2], k[3]));
  } else if constexpr (S == 24) {
    uint2* p = reinterpret_cast<uint2*>(out) + 3 * i;
    __stcs(p, make_uint2(k[0], k[1])); __stcs(p + 1, make_uint2(k[2], k[3])); __stcs(p + 2, make_uint2(k[4], k[5]));
  } else if constexpr (S % 16 == 0) {  // 32, 48, 64 bytes
    uint4* p = reinterpret_cast<uint4*>(out) + (S / 16) * i;
#pragma unroll
    for (int h = 0; h < S / 16; ++h) __stcs(p + h, make_uint4(k[4 * h], k[4 * h + 1], k[4 * h + 2], k[4 * h + 3]));
  } else {
    uint32_t* p = reinterpret_cast<uint32_t*>(out) + i * (S / 4);
#pragma unroll
    for (int q = 0; q < S / 4; ++q) __stcs(p + q, k[q]);
  }
}

// L2 eviction-priority policies (createpolicy) and hinted 32-bit accesses.  oldToNew is written
// at random by the head scan and read at random by the remap right after; marking its lines
// evict-last while the item stream is marked evict-first keeps as much of it in L2 as fits.
__device__ __forceinline__ uint64_t l2_policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t l2_policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ void st_u32_hint(uint32_t* a, uint32_t v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.b32 [%0], %1, %2;" ::"l"(a), "r"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ uint32_t ld_u32_hint(const uint32_t* a, uint64_t pol) {
  uint32_t v;
  asm volatile("ld.global.nc.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(v) : "l"(a), "l"(pol));
  return v;
}

// Byte digit d of a key (d = 0 is the least significant byte of the least significant word).
template <int K>
__device__ __forceinline__ uint32_t key_digit(const uint32_t (&k)[K], int d) {
  const int w = K - 1 - (d >> 2);
  uint32_t word = k[0];
#pragma unroll
  for (int q = 1; q < K; ++q)
    if (q == w) word = k[q];
  return (word >> ((d & 3) * 8)) & 0xFFu;
}

// Word `w` (run time) of a key held in registers, and OR into it (select chains: a run-time index
// into a register array would move the array to local memory).
template <int K>
__host__ __device__ __forceinline__ uint32_t key_word(const uint32_t (&k)[K], int w) {
  uint32_t x = k[0];
#pragma unroll
  for (int q = 1; q < K; ++q)
    if (q == w) x = k[q];
  return x;
}
template <int K>
__host__ __device__ __forceinline__ void key_word_or(uint32_t (&k)[K], int w, uint32_t v) {
#pragma unroll
  for (int q = 0; q < K; ++q)
    if (q == w) k[q] |= v;
}

// Packs the varying bits of a key into its low bits (KeyPack runs, least significant first).
template <int K>
__host__ __device__ __forceinline__ void pack_key(uint32_t (&k)[K], const KeyPack& P) {
  uint32_t out[K];
#pragma unroll
  for (int q = 0; q < K; ++q) out[q] = 0;
  uint64_t acc = 0;
  uint32_t nacc = 0;
  int ow = K - 1;  // packed word being filled
  for (int r = 0; r < P.nruns; ++r) {
    const uint32_t len = P.len[r];
    const uint32_t v = (key_word<K>(k, P.word[r]) >> P.shift[r]) & (len >= 32 ? ~0u : (1u << len) - 1u);
    acc |= (uint64_t)v << nacc;
    nacc += len;
    if (nacc >= 32) {
      key_word_or<K>(out, ow, (uint32_t)acc);
      --ow;
      acc >>= 32;
      nacc -= 32;
    }
  }
  if (nacc) key_word_or<K>(out, ow, (uint32_t)acc);
#pragma unroll
  for (int q = 0; q < K; ++q) k[q] = out[q];
}

// pack_key for keys with at most one run of varying bits per word (KeyPack::simple): the words
// are visited in a fixed order with their run's shift and length, no per-run loop.
template <int K>
__host__ __device__ __forceinline__ void pack_key_simple(uint32_t (&k)[K], const KeyPack& P) {
  uint32_t out[K];
#pragma unroll
  for (int q = 0; q < K; ++q) out[q] = 0;
  uint64_t acc = 0;
  uint32_t nacc = 0;
  int ow = K - 1;
#pragma unroll
  for (int q = K - 1; q >= 0; --q) {
    const uint32_t len = P.wlen[q];
    const uint32_t v = (k[q] >> P.wshift[q]) & (len >= 32 ? ~0u : (1u << len) - 1u);
    acc |= (uint64_t)v << nacc;
    nacc += len;
    if (nacc >= 32) {
      key_word_or<K>(out, ow, (uint32_t)acc);
      --ow;
      acc >>= 32;
      nacc -= 32;
    }
  }
  if (nacc) key_word_or<K>(out, ow, (uint32_t)acc);
#pragma unroll
  for (int q = 0; q < K; ++q) k[q] = out[q];
}

// Bits [pos, pos + len) of a packed key (len <= 32).
template <int K>
__host__ __device__ __forceinline__ uint32_t packed_bits(const uint32_t (&k)[K], uint32_t pos, uint32_t len) {
  const int cw = K - 1 - (int)(pos >> 5), cb = pos & 31;
  uint32_t v = key_word<K>(k, cw) >> cb;
  if (cb + len > 32) v |= key_word<K>(k, cw - 1) << (32 - cb);
  return v & (len >= 32 ? ~0u : (1u << len) - 1u);
}

// Inverse of pack_key: every run back in place, the constant bits from kconst.
template <int K>
__host__ __device__ __forceinline__ void unpack_key(uint32_t (&k)[K], const KeyPack& P, const uint32_t* kconst) {
  uint32_t out[K];
#pragma unroll
  for (int q = 0; q < K; ++q) out[q] = kconst[q];
  for (int r = 0; r < P.nruns; ++r)
    key_word_or<K>(out, P.word[r], packed_bits<K>(k, P.pos[r], P.len[r]) << P.shift[r]);
#pragma unroll
  for (int q = 0; q < K; ++q) k[q] = out[q];
}

// Key word 0 (the mesh id in batched mode) of a packed key.
template <int K>
__host__ __device__ __forceinline__ uint32_t unpacked_word0(const uint32_t (&k)[K], const KeyPack& P, uint32_t kconst0) {
  uint32_t v = kconst0;
  for (int r = 0; r < P.nruns; ++r)
    if (P.word[r] == 0) v |= packed_bits<K>(k, P.pos[r], P.len[r]) << P.shift[r];
  return v;
}

// Programmatic dependent launch: wait until the previous kernel on the stream has completed and
// its writes are visible (returns at once for a kernel launched without the attribute), and let
// the next kernel be scheduled once every CTA of this one has started.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" :::); }

// ---------------------------------------------------------------------------------------------
// Memory-model helpers for decoupled look-back.
__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed(uint32_t* p, uint32_t v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void record_error(Control* c, uint32_t code) { atomicCAS(&c->err, 0u, code); }

// Block-uniform read of the error word (every thread of the CTA gets the same answer, so an
// early return never leaves a barrier half-populated).
__device__ __forceinline__ bool block_error(const Control* c) {
  __shared__ uint32_t s_err;
  if (threadIdx.x == 0) s_err = *(volatile const uint32_t*)&c->err;
  __syncthreads();
  const bool e = s_err != 0;
  __syncthreads();
  return e;
}

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Wait until *p is published; bounded.  Returns the status word, or on timeout records the error
// and returns a prefix of 0.  Failed polls back off
// briefly so that waiting threads leave issue slots to the warps doing useful work.
__device__ __forceinline__ uint32_t wait_status(const uint32_t* p, Control* c) {
  uint32_t s = ld_relaxed(p);
  uint32_t polls = 0;
  while (!lb_ready(s)) {
    ++polls;
    if ((polls & 255u) == 0 && (polls >= kSpinLimit || ld_relaxed(&c->err) != 0)) {
      record_error(c, kErrTimeout);
      return lb_pre(0);
    }
    __nanosleep(polls < 4 ? 32 : 128);
    s = ld_relaxed(p);
  }
  return s;
}

// Decoupled look-back over one counter per tile (status of tile q at lb[q * kLbPad]), done by one
// full warp: returns the exclusive
// prefix of tile `tile` (> 0) in every lane.  Each round inspects the 32*W nearest predecessors
// not yet accumulated (lane l: W consecutive ones), all loads in flight together, and stops at
// the nearest one carrying an inclusive prefix.  (The nearest prefix is usually within 32
// tiles: windows of 256 and 1024 measured slower, since every round waits for all of them.)
template <int W = 1>
__device__ __forceinline__ uint32_t warp_lookback(const uint32_t* lb, int64_t tile, Control* c) {
  const int lane = threadIdx.x & 31;
  uint32_t excl = 0;
  int64_t hi = tile - 1;  // newest predecessor not yet accumulated
  while (true) {
    uint32_t s[W];
#pragma unroll
    for (int i = 0; i < W; ++i) {
      const int64_t q = hi - (int64_t)lane * W - i;
      s[i] = q >= 0 ? ld_relaxed(lb + q * kLbPad) : lb_pre(0);  // before tile 0: prefix 0
    }
#pragma unroll
    for (int i = 0; i < W; ++i) {
      const int64_t q = hi - (int64_t)lane * W - i;
      if (q >= 0 && !lb_ready(s[i])) s[i] = wait_status(lb + q * kLbPad, c);
    }
    int stop = W;  // nearest predecessor of this lane carrying an inclusive prefix
#pragma unroll
    for (int i = W - 1; i >= 0; --i)
      if (lb_is_pre(s[i])) stop = i;
    uint32_t part = 0;
#pragma unroll
    for (int i = 0; i < W; ++i)
      if (i <= stop) part += lb_val(s[i]);
    const uint32_t pre_mask = __ballot_sync(0xffffffffu, stop < W);
    const int first = pre_mask ? __ffs(pre_mask) - 1 : 32;  // nearest lane with a prefix
    uint32_t v = lane <= first ? part : 0u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    excl += v;
    if (pre_mask != 0) break;
    hi -= 32 * W;
  }
  return excl;
}

// Warp-cooperative decoupled look-back for the DPW consecutive digits d0 .. d0+DPW-1 of tile
// `cur` on the tile-major status table (status of tile q, digit d at lb[q * 256 + d]).  Each
// load instruction of the warp covers 32/DPW predecessor tiles x DPW digits (contiguous words
// per tile), so DPW loads, all issued before any is used, cover the 32 nearest predecessors of
// every digit.  Per digit the lanes agree on the nearest inclusive prefix and sum the counts up
// to it; digits without a prefix in the window continue with the next 32 predecessors.
// Lanes 0 .. DPW-1 return the exclusive prefix of digit d0 + lane.
template <int DPW>
__device__ __forceinline__ uint32_t warp_lookback_tiles(const uint32_t* lb, uint32_t cur, int d0, Control* c) {
  constexpr int TPL = 32 / DPW;  // predecessor tiles per load instruction
  const int lane = threadIdx.x & 31;
  const int dl = lane % DPW, h = lane / DPW;
  uint32_t total = 0;
  bool found = false;
  for (int64_t top = (int64_t)cur;; top -= 32) {
    uint32_t v[DPW];
#pragma unroll
    for (int i = 0; i < DPW; ++i) {
      const int64_t q = top - 1 - (i * TPL + h);
      v[i] = q >= 0 ? ld_relaxed(lb + (size_t)q * kRadix + d0 + dl) : lb_pre(0);
    }
    int mypos = 64;  // nearest predecessor (0 = tile top-1) carrying an inclusive prefix
#pragma unroll
    for (int i = 0; i < DPW; ++i) {
      const int64_t q = top - 1 - (i * TPL + h);
      if (q >= 0 && !lb_ready(v[i])) v[i] = wait_status(lb + (size_t)q * kRadix + d0 + dl, c);
      if (lb_is_pre(v[i]) && mypos == 64) mypos = i * TPL + h;
    }
    int cut = mypos;
#pragma unroll
    for (int o = DPW; o < 32; o <<= 1) cut = min(cut, __shfl_xor_sync(0xffffffffu, cut, o));
    uint32_t sum = 0;
#pragma unroll
    for (int i = 0; i < DPW; ++i)
      if (i * TPL + h <= cut) sum += lb_val(v[i]);
#pragma unroll
    for (int o = DPW; o < 32; o <<= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (!found) total += sum;
    found = found || cut < 64;
    if (__all_sync(0xffffffffu, found)) break;
  }
  return total;
}

// Inclusive warp scan.
__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t n = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += n;
  }
  return v;
}

}  // namespace reindex
