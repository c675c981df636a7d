/*
 * reindex.h -- C ABI of the GB300 (sm_103a) mesh re-indexing library.
 *
 * Method: Wald, "GPGPU-Parallel Re-indexing of Triangle Meshes with Duplicate-Vertex and
 * Unused-Vertex Removal" (arXiv 2109.09812), Section 2.  Given a vertex array and an index
 * array of fixed-arity elements, the library produces a new vertex array without unused or
 * duplicate vertices and rewrites every index to point into it.
 *
 * Result definition (what every entry point computes, exactly):
 *   - A vertex is S = vtxStrideBytes raw bytes, viewed as K = S/4 little-endian uint32 words
 *     w[0..K-1].  Two vertices are equal iff all S bytes are equal (so +0.0 != -0.0 and NaNs
 *     compare by payload; padding bytes inside the stride take part).  Section 2 asks for
 *     "exact duplicates" and some total order without fixing either; this is the reading.
 *   - Vertices are ordered lexicographically by (w[0], w[1], ...), each word compared as an
 *     unsigned integer (raw-bit order: negative floats sort after non-negative ones).
 *   - out_vtx holds the distinct values of the vertices referenced by at least one index, in
 *     strictly ascending order; *out_nVtx is their number D.
 *   - out_idx[j] is the position in out_vtx of the value of vtx[idx[j]].
 *   This result is unique: it does not depend on any tie order inside the method.
 *
 * The pipeline (Sections 2.1-2.4, each step a CUDA kernel of this library):
 *   1. used-vertex flags scattered from the index buffer (Section 2.1, isUsed);
 *   2. stable compaction of the used vertices into (key, old index) items.  The paper instead
 *      overwrites each unused vertex with a used one (Section 2.1); both give the same result;
 *   3. LSD radix sort of the items by key, 8 bits per pass, onesweep style with decoupled
 *      look-back (Section 2.2, key-value sort); passes whose digit is constant are skipped;
 *   4. run-head flags where a key differs from its predecessor (Section 2.2, nodup);
 *   5. exclusive prefix sum of the flags giving new indices (Section 2.2, newIdx; the
 *      footnote there notes inclusive-minus-one equals exclusive);
 *   6. oldToNew scatter: oldToNew[orgID[j]] = newIdx[j] (Section 2.4, perm composed with
 *      newIdx);
 *   7. gather of the unique vertices (Section 2.3, newVtx);
 *   8. remap of every index: out_idx[j] = oldToNew[idx[j]] (Section 2.4).
 * For vertices of 16 bytes and more, steps 3-7 first run on the 64 most significant varying bits
 * of each key (an order-preserving prefix); a check that every used vertex equals the unique
 * vertex it was given proves that result exact, and only where it fails do steps 3-7 run again
 * on the whole keys.  Either way the result is the one defined above.
 *
 * Conventions shared by all entry points:
 *   - Pointers named vtx/idx/out_* are DEVICE pointers owned by the caller unless the entry
 *     point says "host".  The library never frees caller memory.
 *   - All calls are asynchronous on `stream` (0 = the legacy default stream) unless stated
 *     otherwise; they never synchronise it.  The returned status covers host-side argument
 *     checks, allocation and kernel launches only.
 *   - Device-detected errors (an index outside [0, nVtx), a look-back wait that ran out) are
 *     reported after the stream is synchronised in two ways: *out_nVtx holds the NEGATED
 *     status code (e.g. -REINDEX_ERR_INDEX_RANGE), and reindex_stream_status() returns it.
 *     When one occurs the contents of out_vtx and out_idx are unspecified.
 *   - Supported strides: vtxStrideBytes in {4, 8, 12, 16, 20, 24, 32, 48, 64} for single meshes
 *     (Section 3.5 expects other vertex formats to carry over directly: e.g. a position with a
 *     normal, 24 bytes, with a normal and texture coordinates, 32 bytes, and with a tangent and
 *     further attributes, 48 or 64 bytes); the batched entry point takes {4, 8, 12, 16}.  vtx and out_vtx must be aligned to the stride's natural
 *     vector type: 4 bytes for S = 4, 12 and 20, 8 bytes for S = 8 and 24, 16 bytes for
 *     S = 16, 32, 48 and 64.  idx and out_idx must be 4-byte aligned (16-byte alignment enables
 *     128-bit vector loads and stores).
 *   - nVtx <= 2^31 - 1 (INT32_MAX; the look-back status words carry 31-bit counts and the old
 *     vertex index travels as 32 bits) and nElem * idxPerElem <= 2^31 - 1 for int32 indices; the
 *     int64-index entry points (reindex_mesh64*) take up to 2^40 index entries, and
 *     reindex_mesh64 also meshes of up to 2^40 vertices (below).
 *   - out_idx may alias idx (the remap reads and writes the same slot in one thread).  No
 *     other output may overlap an input.
 *   - Thread safety: calls may be issued concurrently from several host threads on different
 *     streams; calls on one stream are ordered by that stream.
 */
#ifndef REINDEX_H
#define REINDEX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Opaque CUDA stream handle (binary-compatible with cudaStream_t / CUstream). */
typedef struct CUstream_st* reindex_stream_t;

typedef enum {
  REINDEX_OK = 0,
  REINDEX_ERR_INVALID_ARG = 1, /* bad pointer, size, alignment or workspace too small */
  REINDEX_ERR_UNSUPPORTED = 2, /* stride not supported, or sizes beyond the limits above */
  REINDEX_ERR_OOM = 3,         /* a library allocation failed */
  REINDEX_ERR_INDEX_RANGE = 4, /* some index < 0 or >= nVtx (device-detected) */
  REINDEX_ERR_TIMEOUT = 5,     /* a look-back wait exceeded its iteration limit (device-detected) */
  REINDEX_ERR_CUDA = 6,        /* a CUDA runtime call failed */
  REINDEX_ERR_INTERNAL = 7     /* a device-side consistency check failed (a library bug) */
} reindex_status;

/* Human-readable name of a status code.  Never returns NULL. */
const char* reindex_status_string(reindex_status s);

/* Bytes of device workspace reindex_mesh_ws needs for a mesh of this size (Section 3.6 notes
 * the method needs temporary memory comparable to the data: here two copies of the (key,
 * old index) items, one byte per item for radix digits, one uint32 per input vertex, a bit
 * per input vertex and small look-back and histogram tables).  Returns 0 for unsupported
 * arguments. */
size_t reindex_workspace_size(int64_t nVtx, int vtxStrideBytes, int64_t nElem, int idxPerElem);

/* Re-index one mesh (Sections 2.1-2.4).
 *   vtx         device, nVtx * vtxStrideBytes bytes (aligned as above)
 *   nVtx        number of input vertices (>= 0)
 *   idx         device int32[nElem * idxPerElem]; element e owns idx[e*idxPerElem ...]
 *   nElem       number of elements (>= 0); idxPerElem >= 1 (3 = triangles, 4 = quads/tets)
 *   out_vtx     device, room for min(nVtx, nElem*idxPerElem) * vtxStrideBytes bytes
 *   out_nVtx    device int64 scalar: D, or -status after a device-detected error
 *   out_idx     device int32[nElem * idxPerElem] (may alias idx)
 * Workspace comes from the device's stream-ordered memory pool (cudaMallocAsync on `stream`),
 * returned to the pool on the same stream.  nElem == 0 gives *out_nVtx = 0.  nVtx == 0 with
 * nElem > 0 returns REINDEX_ERR_INDEX_RANGE at once (every index is out of range). */
reindex_status reindex_mesh(const void* vtx, int64_t nVtx, int vtxStrideBytes,
                            const int32_t* idx, int64_t nElem, int idxPerElem,
                            void* out_vtx, int64_t* out_nVtx, int32_t* out_idx,
                            reindex_stream_t stream);

/* Same as reindex_mesh with a caller-supplied device workspace of wsBytes >=
 * reindex_workspace_size(...) bytes, 256-byte aligned.  Performs no allocation and no host
 * synchronisation, so it can be captured into a CUDA graph.  The workspace must not be used by
 * any other call until this one has finished on the device. */
reindex_status reindex_mesh_ws(const void* vtx, int64_t nVtx, int vtxStrideBytes,
                               const int32_t* idx, int64_t nElem, int idxPerElem,
                               void* out_vtx, int64_t* out_nVtx, int32_t* out_idx,
                               void* ws, size_t wsBytes, reindex_stream_t stream);

/* ---- int64 indices ----------------------------------------------------------------------------
 * reindex_mesh / reindex_mesh_ws for 8-byte indices: idx and out_idx are DEVICE int64 arrays of
 * nElem * idxPerElem entries (8-byte aligned; 16-byte alignment enables vector loads), which may
 * alias.  Everything else -- vertices, result, workspace layout, errors -- is as for the int32
 * entry points; the index arrays no longer cap the element count at 2^31 - 1 indices (up to 2^40
 * here); indices beyond nVtx, however large, and negative indices are REINDEX_ERR_INDEX_RANGE
 * (none is truncated to 32 bits).  Section 3.5 of the paper expects other formats to carry over;
 * int64 index buffers are the common one besides int32.
 * reindex_mesh64 takes meshes of more than 2^31 - 1 vertices too (up to 2^40): the vertex array is
 * re-indexed in ranges of 2^30 vertices, each range's unique vertices are concatenated and re-indexed
 * once more, and the two maps are composed for every index -- the same result as a single pass.
 * Such a call BLOCKS: it synchronises `stream` once per range, and allocates about 4 * nVtx bytes
 * besides a range's workspace.  The distinct used vertices must number at most 2^31 - 1, else
 * REINDEX_ERR_UNSUPPORTED; an index-range error is returned (and written into *out_nVtx as usual).
 * reindex_mesh64_ws keeps nVtx <= 2^31 - 1; reindex_workspace_size64 gives its workspace (0 for
 * unsupported sizes). */
size_t reindex_workspace_size64(int64_t nVtx, int vtxStrideBytes, int64_t nElem, int idxPerElem);
reindex_status reindex_mesh64(const void* vtx, int64_t nVtx, int vtxStrideBytes,
                              const int64_t* idx, int64_t nElem, int idxPerElem,
                              void* out_vtx, int64_t* out_nVtx, int64_t* out_idx,
                              reindex_stream_t stream);
reindex_status reindex_mesh64_ws(const void* vtx, int64_t nVtx, int vtxStrideBytes,
                                  const int64_t* idx, int64_t nElem, int idxPerElem,
                                  void* out_vtx, int64_t* out_nVtx, int64_t* out_idx,
                                  void* ws, size_t wsBytes, reindex_stream_t stream);

/* End-to-end variant on HOST buffers: copies vtx and idx to the device, runs the pipeline and
 * copies the D unique vertices, the indices and D back.  host_vtx / host_idx should be pinned
 * (page-locked) for full copy bandwidth; host_out_vtx needs room for min(nVtx, nElem *
 * idxPerElem) vertices.  Device buffers come from the stream-ordered pool.  BLOCKING: returns
 * after the results are in host memory; a device-detected error is returned as the status
 * and written (negated) to *host_out_nVtx. */
reindex_status reindex_mesh_host(const void* host_vtx, int64_t nVtx, int vtxStrideBytes,
                                 const int32_t* host_idx, int64_t nElem, int idxPerElem,
                                 void* host_out_vtx, int64_t* host_out_nVtx, int32_t* host_out_idx,
                                 reindex_stream_t stream);

/* Re-index one small mesh WITHOUT ALLOCATING ANYTHING.  The paper has no counterpart; this entry
 * point exists for callers that cannot allocate device memory when they call us: a program that
 * reserved its whole device-memory budget up front and accounts for every byte, a real-time
 * loop in which cudaMalloc/cudaFree would synchronise the device and stall its other streams, or
 * a plugin whose host application forbids allocations behind its back.
 *   Arguments, result and error reporting are those of reindex_mesh (inputs and outputs are
 *   still the caller's device buffers).
 *   Limit: nVtx <= REINDEX_NOALLOC_MAX_VTX (262,144 vertices, any number of elements) for
 *   vertices of up to 32 bytes; 48- and 64-byte vertices are taken while their workspace fits
 *   the scratch (every mesh of up to 188,949 or 146,472 vertices does).  A larger mesh returns
 *   REINDEX_ERR_UNSUPPORTED and nothing is launched.
 *   Scratch: one array of REINDEX_NOALLOC_SCRATCH_BYTES (20 MiB) of device memory inside the
 *   library, held on a device from the time the CUDA runtime loads the library's device code
 *   there until the process exits.  With lazy module loading (the CUDA default) that happens at
 *   the FIRST call on the device: that call reserves the 20 MiB (it can fail with
 *   REINDEX_ERR_CUDA if the device is full, and may synchronise the device) and looks up the
 *   array's device address (cudaGetSymbolAddress, with the device current), which later calls
 *   reuse.  So make one warm-up call per device -- nElem == 0 is enough, it launches one tiny
 *   kernel -- before committing the rest of the device-memory budget and before any stream
 *   capture on that device.
 *   All calls share the array.  Each call zeroes the parts that must start at zero, but two
 *   calls whose work overlaps on the GPU (e.g. on two streams with no ordering between them)
 *   race on it and corrupt each other's results: order them on one stream or with events.
 *   Keep per-launch timing (reindex_profile_enable) off: that facility allocates for itself. */
#define REINDEX_NOALLOC_SCRATCH_BYTES (20u << 20)
#define REINDEX_NOALLOC_MAX_VTX 262144
reindex_status reindex_mesh_noalloc(const void* vtx, int64_t nVtx, int vtxStrideBytes,
                                    const int32_t* idx, int64_t nElem, int idxPerElem,
                                    void* out_vtx, int64_t* out_nVtx, int32_t* out_idx,
                                    reindex_stream_t stream);

/* ---- batched: many independent meshes in one launch sequence ---------------------------------
 * Mesh m owns vertices [vtxOffsets[m], vtxOffsets[m+1]) of the concatenated vtx array and
 * elements [elemOffsets[m], elemOffsets[m+1]) of the concatenated idx array; its indices are
 * LOCAL to its own vertices (0 .. nVtx_m - 1).  vtxOffsets and elemOffsets are DEVICE int64 arrays
 * of nMeshes+1 entries, non-decreasing, starting at 0 and ending at nVtxTotal / nElemTotal (the
 * host passes the two totals so that no device value has to be read back).
 * Output: mesh m's unique vertices are out_vtx[out_vtxOffsets[m] .. out_vtxOffsets[m+1]) (a DEVICE
 * int64 array of nMeshes+1 entries written by the library; out_vtxOffsets[nMeshes] = total D, or
 * -status after a device-detected error), and mesh m's out_idx entries (same slots as its input
 * indices) are local to its own output range.  Each mesh's result is bitwise identical to
 * reindex_mesh on that mesh alone: duplicates are merged only inside a mesh.
 * vtxStrideBytes in {4, 8, 12, 16}; internally the mesh id is an extra key word.  Sizes as for
 * reindex_mesh over the totals.  out_idx may alias idx.  The workspace (reindex_meshes_workspace_size
 * bytes, 256-byte aligned) is caller-supplied; the call allocates nothing and never synchronises,
 * so the whole sequence can be captured into a CUDA graph and replayed.
 * Device-detected errors: INDEX_RANGE (a local index outside its mesh), INVALID_ARG (offsets
 * that are not non-decreasing from 0 to the totals). */
size_t reindex_meshes_workspace_size(int nMeshes, int64_t nVtxTotal, int vtxStrideBytes, int64_t nElemTotal,
                                     int idxPerElem);
reindex_status reindex_meshes(const void* vtx, const int64_t* vtxOffsets, int vtxStrideBytes,
                              const int32_t* idx, const int64_t* elemOffsets, int idxPerElem,
                              int nMeshes, int64_t nVtxTotal, int64_t nElemTotal,
                              void* out_vtx, int64_t* out_vtxOffsets, int32_t* out_idx,
                              void* ws, size_t wsBytes, reindex_stream_t stream);

/* ---- merging meshes (Section 3.2) ----------------------------------------------------------------
 * Same inputs as reindex_meshes (concatenated meshes, mesh-local indices, device offsets), but ONE
 * output mesh: the paper's merge -- concatenate the vertex arrays, offset each mesh's indices by
 * the number of vertices before it, then remove duplicate and unused vertices ACROSS meshes.
 * out_vtx / *out_nVtx / out_idx as for reindex_mesh over the concatenation (out_idx may alias
 * idx); workspace of reindex_merge_workspace_size bytes, 256-byte aligned; no allocation, no
 * synchronisation.  Device-detected errors: INDEX_RANGE (a local index outside its mesh),
 * INVALID_ARG (bad offsets). */
size_t reindex_merge_workspace_size(int nMeshes, int64_t nVtxTotal, int vtxStrideBytes, int64_t nElemTotal,
                                    int idxPerElem);
reindex_status reindex_merge_meshes(const void* vtx, const int64_t* vtxOffsets, int vtxStrideBytes,
                                    const int32_t* idx, const int64_t* elemOffsets, int idxPerElem,
                                    int nMeshes, int64_t nVtxTotal, int64_t nElemTotal,
                                    void* out_vtx, int64_t* out_nVtx, int32_t* out_idx,
                                    void* ws, size_t wsBytes, reindex_stream_t stream);

/* ---- subset of a mesh (Section 3.4) -------------------------------------------------------------
 * Keeps only the elements listed in elemList (device int32[nSel], each in [0, nElem); repeats
 * allowed, order kept) with the FULL vertex array, and removes the vertices they do not use and
 * the duplicates: out_idx (device int32[nSel * idxPerElem], must not alias idx) is the compact
 * subset mesh's index array, out_vtx its vertices (room for min(nVtx, nSel*idxPerElem)).
 * Workspace of reindex_submesh_workspace_size bytes.  Device-detected errors: INDEX_RANGE (a list
 * entry outside [0, nElem) or an index outside [0, nVtx)). */
size_t reindex_submesh_workspace_size(int64_t nVtx, int vtxStrideBytes, int64_t nSel, int idxPerElem);
reindex_status reindex_submesh(const void* vtx, int64_t nVtx, int vtxStrideBytes,
                               const int32_t* idx, int64_t nElem, int idxPerElem,
                               const int32_t* elemList, int64_t nSel,
                               void* out_vtx, int64_t* out_nVtx, int32_t* out_idx,
                               void* ws, size_t wsBytes, reindex_stream_t stream);

/* ---- serving: a request loop with continuous batching ------------------------------------------
 * A server owns one arena of device memory (the HBM budget) and a scheduler thread.  Clients
 * submit requests (device-resident meshes, which must stay valid and unchanged until the request
 * completes) at any time.  Whenever one of num_streams CUDA streams is free, the scheduler
 * coalesces the pending requests of the oldest request's stride/arity class, in arrival order,
 * into one reindex_meshes launch sequence, admitting only what fits the free part of the budget;
 * requests that arrive meanwhile join the next batch, and batches on different streams overlap.
 * Each result is identical to reindex_mesh on the request alone.  A batch whose device run fails
 * is split and its requests re-run one by one, so that only a faulty request fails.  Results
 * (pointers into the arena) stay valid until reindex_server_release. */
typedef struct reindex_server reindex_server;

typedef struct {
  size_t hbm_budget_bytes;  /* device memory for staging, outputs and workspaces (>= 1 MiB) */
  int max_batch_requests;   /* most requests per launch sequence (<= 0: 256) */
  int num_streams;          /* batches in flight at once (<= 0: 2) */
  int device;               /* CUDA device ordinal */
} reindex_server_config;

typedef struct {
  const void* vtx;          /* device, nVtx * vtxStrideBytes; vtxStrideBytes in {4, 8, 12, 16} */
  int64_t nVtx;
  int vtxStrideBytes;
  const int32_t* idx;       /* device, nElem * idxPerElem */
  int64_t nElem;
  int idxPerElem;
} reindex_request;

typedef struct {
  int64_t id;
  reindex_status status;    /* REINDEX_OK or this request's error */
  int64_t nVtxOut;          /* D */
  const void* out_vtx;      /* device, D * stride bytes (NULL after an error) */
  const int32_t* out_idx;   /* device, nElem * idxPerElem */
  double submit_us, start_us, done_us;  /* host steady-clock times: submitted, launched, finished */
} reindex_result;

typedef struct {
  int64_t requests_submitted, requests_started, requests_done, requests_failed, requests_rejected;
  int64_t batches, batches_split, arena_bytes_in_use, pending;
} reindex_server_stats;

/* Allocates the arena (cudaMalloc, once) and starts the scheduler thread. */
reindex_status reindex_server_create(const reindex_server_config* cfg, reindex_server** out);
/* Non-blocking.  REINDEX_ERR_OOM: the request could not fit the budget even alone. */
reindex_status reindex_server_submit(reindex_server* s, const reindex_request* req, int64_t* id_out);
/* Up to max_results finished requests (waiting up to wait_ms for the first); returns the count. */
int reindex_server_poll(reindex_server* s, reindex_result* out, int max_results, int wait_ms);
/* Returns a finished request's outputs to the arena. */
reindex_status reindex_server_release(reindex_server* s, int64_t id);
/* Waits until every submitted request has finished (REINDEX_ERR_TIMEOUT after timeout_ms). */
reindex_status reindex_server_drain(reindex_server* s, int timeout_ms);
reindex_status reindex_server_get_stats(reindex_server* s, reindex_server_stats* out);
/* Drops requests not yet started, waits for running batches, frees everything. */
void reindex_server_destroy(reindex_server* s);
/* Test hook for failure detection: while tile >= 0, the compaction kernel's tile `tile` (of 2048
 * vertices) never publishes its decoupled look-back status, so the bounded waits of the tiles
 * after it run out (about a second) and the call reports REINDEX_ERR_TIMEOUT through *out_nVtx
 * and reindex_stream_status, leaving the CUDA context usable.  -1 turns it off (the default). */
void reindex_debug_stall_tile(int64_t tile);

/* Host-only self-check of the server's arena allocator against a brute-force model; returns the
 * number of inconsistencies (0 = correct).  Needs no GPU. */
int reindex_debug_arena_check(uint64_t seed, int ops, size_t size);

/* Host-only test hook: the bit selection of the prefix sort for keys of K (1..16) 32-bit words,
 * given per word the OR of the word over the used vertices (kor) and of its complement (knand): a
 * bit varies iff it is set in both.  The prefix is the 64 most significant varying bits (at most
 * 16 runs of consecutive bits), word 0 most significant.  Writes the packing description (104
 * bytes: on, nbits, nruns, word[16], shift[16], len[16], pos[16] -- runs least significant first,
 * pos = the run's offset in the prefix --, simple, wshift[16], wlen[16], 4 bytes padding) to `out`
 * and returns the number of prefix bits, or -1 for bad arguments.  Needs no GPU. */
int reindex_debug_prefix_pack(const uint32_t* kor, const uint32_t* knand, int K, void* out, int outBytes);

/* Host-only test hook: the key packing arithmetic of the kernels (the same inline functions),
 * applied on the host to n keys of K (1..8, 12 or 16) words, row-major in `keys`, with a packing
 * description in the layout written by reindex_debug_prefix_pack.  mode 0: pack (general runs),
 * 1: pack (at most one run per word), 2: unpack packed keys, filling the constant bits from
 * kconst[K]; all three write n*K words to `out`.  mode 3: word 0 of each unpacked key (n words),
 * from kconst[0] and the runs of word 0.  Returns 0, or -1 for bad arguments.  Needs no GPU. */
int reindex_debug_pack_keys(const void* pack, int packBytes, int K, const uint32_t* kconst,
                            const uint32_t* keys, int64_t n, int mode, uint32_t* out);

/* Synchronises `stream`, then returns and clears this device's sticky device-side error: the
 * first INDEX_RANGE or TIMEOUT raised by any call on the current device since the last
 * reindex_stream_status() (REINDEX_OK if none).  A CUDA error from the synchronisation is
 * returned as REINDEX_ERR_CUDA. */
reindex_status reindex_stream_status(reindex_stream_t stream);

/* ---- autotuning ---------------------------------------------------------------------------------
 * The library has several kernel variants with identical results.  Each is a knob of a
 * comma-separated spec "name=value,...":
 *   sort    the radix pass: regs (register-tiled onesweep, 4096-item tiles), pipe (tiles pipelined
 *           through shared memory by the Tensor Memory Accelerator), tiles (precounted tile
 *           offsets), chunk (contiguous chunks of bulk-copied tiles), auto
 *   rank    digit matching inside a warp: ballot, match (match.any), vary (ballots on varying bits)
 *   hist    compaction histogram: uniform, peel, match;   grid: persist | tile
 *   swaves  CTAs of the "tiles" scatter: tile (one per tile), 1 or 4 (waves striding over tiles)
 *   chunk   chunk-sort tile shape: big, small, wide, deep;   cocc: max | 1 | 2 (CTAs per SM)
 *   cgrid   chunk-sort chunk count cap (0: none);   dbits: radix digit width, 6, 7 or 8 bits
 *   dedup   hash (remove duplicate vertices with a hash table before the sort, which then orders
 *           the distinct keys only; single meshes of 8-byte vertices and wider) | off
 *   dpub    on | off: with dedup=hash, representatives publish their item positions in the table
 *   pack    key packing: auto, on, off;   prefix: the 64-bit prefix sort for wide keys: auto, on, off
 * reindex_autotune times them on the caller's mesh with whole reindex_mesh_ws runs (coordinate
 * descent, median of `reps` runs each; BLOCKING: it synchronises `stream`) and keeps the fastest
 * for this device and stride, for every later call of this process; if the environment variable
 * REINDEX_TUNE_CACHE names a file, the choice is appended to it and read back by later processes.
 * out_idx must not alias idx.  desc (optional) receives the chosen configuration, every knob
 * named (under 300 characters), cut to descLen - 1 characters and NUL-terminated.  A spec given
 * to reindex_tuning_set may name any subset; unknown names and values are ignored. */
reindex_status reindex_autotune(const void* vtx, int64_t nVtx, int vtxStrideBytes,
                                const int32_t* idx, int64_t nElem, int idxPerElem,
                                void* out_vtx, int64_t* out_nVtx, int32_t* out_idx,
                                void* ws, size_t wsBytes, int reps, reindex_stream_t stream,
                                char* desc, int descLen);
/* The configuration in force for this device and stride (as above), or set one explicitly. */
reindex_status reindex_tuning_get(int vtxStrideBytes, char* desc, int descLen);
reindex_status reindex_tuning_set(int vtxStrideBytes, const char* spec);

/* ---- per-kernel timing (measurement support) ------------------------------------------------
 * While enabled, every pipeline kernel launch made by this process is bracketed by a pair of
 * CUDA events recorded on its stream.  reindex_profile_collect() synchronises those events and
 * returns one record per launch.  Off by default; not for use under stream capture. */
typedef struct {
  int kernel;      /* reindex_kernel_id */
  int digit;       /* radix digit position of a sort pass (0 = least significant byte), else -1 */
  int skipped;     /* 1 if a sort pass found its digit constant and moved no data */
  float ms;        /* event-measured duration */
  int item_bytes;  /* sort passes: bytes per item moved (key + old index), else 0 */
} reindex_profile_record;

typedef enum {
  REINDEX_K_CLEAR = 0,      /* zero the workspace tables */
  REINDEX_K_USED_FLAGS = 1, /* step 1 */
  REINDEX_K_COMPACT = 2,    /* step 2 (+ upfront digit histograms) */
  REINDEX_K_SORT_PLAN = 3,  /* digit offsets and pass skipping */
  REINDEX_K_ONESWEEP = 4,   /* step 3, one launch per digit */
  REINDEX_K_HEAD_SCAN = 5,  /* steps 4-7 fused */
  REINDEX_K_REMAP = 6,      /* step 8 */
  REINDEX_K_FINALIZE = 7,   /* error propagation */
  REINDEX_K_SEG_PREPARE = 8, /* batched: mesh lookup tables, offsets check */
  REINDEX_K_SEG_OFFSETS = 9, /* batched: per-mesh output offsets fix-up */
  REINDEX_K_TILE_COUNT = 10,   /* step 3, "tiles" variant: per-tile digit counts */
  REINDEX_K_TILE_OFFSETS = 11, /* step 3, "tiles" variant: tile offsets per digit */
  REINDEX_K_TILE_SCATTER = 12, /* step 3, "tiles" variant: the pass's data movement */
  REINDEX_K_KEY_MASKS = 13,    /* "tiles" variant: which key bits vary over the used vertices */
  REINDEX_K_PREFIX_GATE = 14,  /* prefix sort: skip the full-key sort unless two keys shared a prefix */
  REINDEX_K_PREFIX_CHECK = 15, /* prefix sort: every used vertex equals the unique vertex it was given */
  REINDEX_K_CHUNK_SCATTER = 16, /* step 3, "chunk" variant: the pass's data movement (its count and
                                   offset kernels report as TILE_COUNT and TILE_OFFSETS) */
  REINDEX_K_HASH_DEDUP = 17,   /* "hash" variant of steps 2-4: distinct keys by hash table before the
                                  sort (one representative per key is sorted; copies are tagged) */
  REINDEX_K_RESOLVE = 18,      /* "hash" variant: copies take their representative's new index */
  REINDEX_K_COUNT = 19
} reindex_kernel_id;

void reindex_profile_enable(int on);
/* Writes up to maxRecords records; returns the number of records pending (all of them are
 * consumed), or -1 on a CUDA error. */
int reindex_profile_collect(reindex_profile_record* out, int maxRecords);
const char* reindex_kernel_name(int kernel);

#ifdef __cplusplus
}
#endif

#endif /* REINDEX_H */
