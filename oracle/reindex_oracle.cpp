// Serial CPU oracle for mesh re-indexing with duplicate- and unused-vertex removal
// (Wald, "GPGPU-Parallel Re-indexing of Triangle Meshes with Duplicate-Vertex and
// Unused-Vertex Removal", arXiv 2109.09812).
//
// TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the benchmark's
// CPU-baseline leg load this library.  It shares no code, header, table or helper with
// the CUDA path, and the CUDA path never calls it.
//
// Conventions (the readings this oracle fixes):
//   * A vertex is S raw bytes (S a positive multiple of 4), viewed as K = S/4
//     little-endian uint32 words w[0..K-1].  Two vertices are equal iff all their bits are
//     equal (so +0.0 != -0.0 and NaNs compare by payload): Section 2 assumes "exact
//     duplicates" and some total order on vertices without fixing either.
//   * The order is lexicographic over the words, w[0] most significant, each word compared
//     as an unsigned integer.
//   * An index outside [0, nVtx) is an error (the paper does not say; no partial result).
//   * nElem == 0 gives zero output vertices (the paper's Step 1 would read triangle[0]).
//
// Three entry points:
//   oracle_reindex_sort   -- the plain definition of the result (unique, sorted used keys,
//                            each index replaced by the rank of its key), computed with one
//                            std::sort over (key, old index) pairs.
//   oracle_reindex_map    -- the serial std::map method of Section 1, numbering vertices in
//                            first-occurrence order; optionally relabelled to key order.
//   oracle_paper_steps    -- Steps 1-4 of Section 2 as the paper states them (overwrite the
//                            unused vertices, full key-value sort, nodup flags, inclusive scan
//                            minus one, newVtx scatter, perm, index update), exposing every
//                            intermediate array so that the worked example can be checked.
//
// Return codes: 0 ok, -1 invalid argument, -2 index out of range.

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <map>
#include <numeric>
#include <vector>

namespace {

constexpr int kOk = 0;
constexpr int kBadArg = -1;
constexpr int kIndexRange = -2;

// The K words of vertex i.
inline const uint32_t* key_of(const uint32_t* words, int K, int64_t i) { return words + i * (int64_t)K; }

// Lexicographic unsigned comparison, word 0 most significant.  Returns <0, 0, >0.
inline int compare_keys(const uint32_t* a, const uint32_t* b, int K) {
  for (int w = 0; w < K; ++w) {
    if (a[w] < b[w]) return -1;
    if (a[w] > b[w]) return 1;
  }
  return 0;
}

bool valid_args(const void* vtx, int64_t nVtx, int S, const int32_t* idx, int64_t M) {
  if (S <= 0 || S % 4 != 0) return false;
  if (nVtx < 0 || M < 0) return false;
  if (nVtx > 0 && vtx == nullptr) return false;
  if (M > 0 && idx == nullptr) return false;
  return true;
}

bool indices_in_range(const int32_t* idx, int64_t M, int64_t nVtx) {
  for (int64_t j = 0; j < M; ++j)
    if (idx[j] < 0 || (int64_t)idx[j] >= nVtx) return false;
  return true;
}

}  // namespace

extern "C" {

// Plain definition of the result (Sections 2.1-2.4 reach exactly this):
//   Used      = { idx[j] : 0 <= j < M }
//   out_vtx   = the distinct keys of the used vertices, strictly ascending; *out_nVtx = count
//   out_idx[j]= the position of key(idx[j]) in out_vtx
// out_vtx needs room for min(nVtx, M) vertices; out_idx for M entries.
int oracle_reindex_sort(const void* vtx, int64_t nVtx, int S, const int32_t* idx, int64_t M,
                        void* out_vtx, int64_t* out_nVtx, int32_t* out_idx) {
  if (!valid_args(vtx, nVtx, S, idx, M) || out_nVtx == nullptr) return kBadArg;
  if (!indices_in_range(idx, M, nVtx)) return kIndexRange;
  const int K = S / 4;
  const uint32_t* words = static_cast<const uint32_t*>(vtx);

  // The set of used vertex indices (Section 2.1, isUsed).
  std::vector<uint8_t> used(nVtx, 0);
  for (int64_t j = 0; j < M; ++j) used[idx[j]] = 1;

  // (key, old index) pairs of the used vertices, sorted by key, ties by index (Section 2.2).
  std::vector<int64_t> order;
  for (int64_t i = 0; i < nVtx; ++i)
    if (used[i]) order.push_back(i);
  std::sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
    int c = compare_keys(key_of(words, K, a), key_of(words, K, b), K);
    return c != 0 ? c < 0 : a < b;
  });

  // A new vertex starts wherever the key differs from its predecessor (Section 2.2, nodup);
  // its number is the count of earlier run starts (Section 2.2, newIdx); the run's key is
  // written once (Section 2.3, newVtx); every old index learns its new number (Section 2.4).
  std::vector<int32_t> old_to_new(nVtx, -1);
  uint32_t* outw = static_cast<uint32_t*>(out_vtx);
  int64_t D = 0;
  for (size_t p = 0; p < order.size(); ++p) {
    const int64_t i = order[p];
    const bool head = (p == 0) || compare_keys(key_of(words, K, i), key_of(words, K, order[p - 1]), K) != 0;
    if (head) {
      std::memcpy(outw + D * K, key_of(words, K, i), (size_t)S);
      ++D;
    }
    old_to_new[i] = (int32_t)(D - 1);
  }
  for (int64_t j = 0; j < M; ++j) out_idx[j] = old_to_new[idx[j]];
  *out_nVtx = D;
  return kOk;
}

// The serial method of Section 1: walk the elements in order, look each vertex up in a
// std::map keyed by its value, and append it to the new vertex array on first sight.
// With canonical == 0 the output keeps that first-occurrence numbering.  With canonical != 0
// the new vertices are relabelled in the map's (ascending key) order, which must reproduce
// oracle_reindex_sort exactly.
int oracle_reindex_map(const void* vtx, int64_t nVtx, int S, const int32_t* idx, int64_t M, int canonical,
                       void* out_vtx, int64_t* out_nVtx, int32_t* out_idx) {
  if (!valid_args(vtx, nVtx, S, idx, M) || out_nVtx == nullptr) return kBadArg;
  if (!indices_in_range(idx, M, nVtx)) return kIndexRange;
  const int K = S / 4;
  const uint32_t* words = static_cast<const uint32_t*>(vtx);
  uint32_t* outw = static_cast<uint32_t*>(out_vtx);

  // std::vector<uint32_t>::operator< is lexicographic with unsigned word compares.
  std::map<std::vector<uint32_t>, int32_t> already_inserted;
  int64_t n_new = 0;
  for (int64_t j = 0; j < M; ++j) {
    const uint32_t* k = key_of(words, K, idx[j]);
    std::vector<uint32_t> v(k, k + K);
    auto it = already_inserted.find(v);
    int32_t v_idx;
    if (it != already_inserted.end()) {
      v_idx = it->second;
    } else {
      v_idx = (int32_t)n_new;
      if (!canonical) std::memcpy(outw + n_new * K, k, (size_t)S);
      ++n_new;
      already_inserted.emplace(std::move(v), v_idx);
    }
    out_idx[j] = v_idx;
  }
  if (canonical) {
    std::vector<int32_t> rank(n_new, -1);
    int32_t r = 0;
    for (const auto& kv : already_inserted) {
      std::memcpy(outw + (int64_t)r * K, kv.first.data(), (size_t)S);
      rank[kv.second] = r++;
    }
    for (int64_t j = 0; j < M; ++j) out_idx[j] = rank[out_idx[j]];
  }
  *out_nVtx = n_new;
  return kOk;
}

// Steps 1-4 of Section 2, in the paper's order and notation.  Every array argument is
// optional output storage for one intermediate (nullptr skips the copy); all N-sized arrays
// hold nVtx entries:
//   isUsed[N]          Step 1: one flag per vertex, set for every index in any element
//   vtxAfterStep1[N*S] Step 1: vertex array with each unused vertex overwritten by the first
//                      element's first vertex
//   sortedOrgID[N]     Step 2: the identity array after the key-value sort (ties keep index
//                      order: a stable sort; the paper allows any tie order)
//   nodup[N]           Step 2: run-head flags over the sorted vertices
//   newIdxInclusive[N] Step 2: inclusive prefix sum over nodup
//   newIdx[N]          Step 2: the same minus one
//   newVtx[N*S]        Step 3: the scattered unique vertices (first *newN entries valid)
//   perm[N]            Step 4: perm[sortedOrgID[j]] = j
//   idxNew[M]          Step 4: idx(new)[i] = newIdx[perm[idx(old)[i]]]
// With M == 0 the paper's Step 1 is undefined; this returns *newN = 0 and touches nothing else.
int oracle_paper_steps(const void* vtx, int64_t nVtx, int S, const int32_t* idx, int64_t M,
                       uint8_t* isUsed, void* vtxAfterStep1, int32_t* sortedOrgID, uint8_t* nodup,
                       int32_t* newIdxInclusive, int32_t* newIdx, int32_t* perm, void* newVtx,
                       int64_t* newN, int32_t* idxNew) {
  if (!valid_args(vtx, nVtx, S, idx, M) || newN == nullptr) return kBadArg;
  if (!indices_in_range(idx, M, nVtx)) return kIndexRange;
  const int K = S / 4;
  const int64_t N = nVtx;
  if (M == 0) {
    *newN = 0;
    return kOk;
  }
  // Step 1: mark used vertices, then overwrite unused ones with vtx[idx[0]].
  std::vector<uint8_t> used(N, 0);
  for (int64_t j = 0; j < M; ++j) used[idx[j]] = 1;
  std::vector<uint32_t> v(static_cast<const uint32_t*>(vtx), static_cast<const uint32_t*>(vtx) + N * K);
  const int64_t first = idx[0];
  for (int64_t i = 0; i < N; ++i)
    if (!used[i])
      for (int w = 0; w < K; ++w) v[i * K + w] = v[first * K + w];

  // Step 2: orgID = identity; key-value sort with the vertex as key.
  std::vector<int32_t> orgID(N);
  std::iota(orgID.begin(), orgID.end(), 0);
  std::stable_sort(orgID.begin(), orgID.end(), [&](int32_t a, int32_t b) {
    return compare_keys(&v[(int64_t)a * K], &v[(int64_t)b * K], K) < 0;
  });
  std::vector<uint32_t> sorted(N * K);
  for (int64_t j = 0; j < N; ++j)
    for (int w = 0; w < K; ++w) sorted[j * K + w] = v[(int64_t)orgID[j] * K + w];
  //   nodup[i] = (i == 0) || vtx[i] != vtx[i-1]
  std::vector<uint8_t> nd(N);
  for (int64_t i = 0; i < N; ++i)
    nd[i] = (i == 0) || compare_keys(&sorted[i * K], &sorted[(i - 1) * K], K) != 0;
  //   newIdx = inclusive prefix sum of nodup, then minus one
  std::vector<int32_t> incl(N), ni(N);
  int64_t run = 0;
  for (int64_t i = 0; i < N; ++i) {
    run += nd[i];
    incl[i] = (int32_t)run;
    ni[i] = (int32_t)(run - 1);
  }
  // Step 3: newN = newIdx.back() + 1; newVtx[newIdx[i]] = vtx[i] where nodup[i].
  const int64_t nn = (int64_t)ni[N - 1] + 1;
  std::vector<uint32_t> nv(nn * K);
  for (int64_t i = 0; i < N; ++i)
    if (nd[i])
      for (int w = 0; w < K; ++w) nv[(int64_t)ni[i] * K + w] = sorted[i * K + w];
  // Step 4: perm[orgID[j]] = j; idx(new)[i] = newIdx[perm[idx(old)[i]]].
  std::vector<int32_t> pm(N);
  for (int64_t j = 0; j < N; ++j) pm[orgID[j]] = (int32_t)j;

  if (isUsed) std::memcpy(isUsed, used.data(), (size_t)N);
  if (vtxAfterStep1) std::memcpy(vtxAfterStep1, v.data(), (size_t)(N * S));
  if (sortedOrgID) std::memcpy(sortedOrgID, orgID.data(), (size_t)N * 4);
  if (nodup) std::memcpy(nodup, nd.data(), (size_t)N);
  if (newIdxInclusive) std::memcpy(newIdxInclusive, incl.data(), (size_t)N * 4);
  if (newIdx) std::memcpy(newIdx, ni.data(), (size_t)N * 4);
  if (perm) std::memcpy(perm, pm.data(), (size_t)N * 4);
  if (newVtx) std::memcpy(newVtx, nv.data(), (size_t)(nn * S));
  if (idxNew)
    for (int64_t j = 0; j < M; ++j) idxNew[j] = ni[pm[idx[j]]];
  *newN = nn;
  return kOk;
}

}  // extern "C"
