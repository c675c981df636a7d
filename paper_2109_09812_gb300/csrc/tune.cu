// Autotuner: picks, per device and vertex stride, the fastest of the library's kernel variants
// for the caller's own mesh, by timing whole reindex_mesh_ws runs with CUDA events.
//   knobs: radix-pass kernel (register-tiled onesweep, 4096-item tiles | TMA-pipelined through
//          shared memory, 2048-4096-item tiles | precounted tile offsets | contiguous chunks with
//          bulk-copied tiles), digit matching (8 ballots | match.any | ballots on varying bits),
//          histogram method (uniform check | peel | match.any), grid shape (persistent | one CTA
//          per tile), CTAs of the "tiles" scatter (one per tile | 1 or 4 waves striding over the
//          tiles), tile size and threads of the chunk sort (2048 or 4096 items, 256-1024 threads)
//          and its resident CTAs per SM (as many as fit | 1), its radix digit width (8, 7 or 6 bits),
//          duplicate removal before the sort (hash table, with or without published item positions),
//          key packing, prefix sort
// Coordinate descent: each knob in turn takes the value with the lowest median time while the
// others stay fixed.  The choice applies to every later call on the device and, if the
// environment variable REINDEX_TUNE_CACHE names a file, is appended to it so that a later
// process starts from it (lines "device name|SMs|stride|spec").
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "internal.h"
#include "reindex.h"

namespace reindex {

static std::string device_name(int dev) {
  cudaDeviceProp p;
  if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) return "unknown";
  std::string n = p.name;
  std::replace(n.begin(), n.end(), '|', '_');
  return n;
}

std::string tuning_from_cache(int dev, int sms, int S) {
  const char* path = std::getenv("REINDEX_TUNE_CACHE");
  if (!path) return "";
  std::ifstream f(path);
  std::string line, found;
  const std::string key = device_name(dev) + "|" + std::to_string(sms) + "|" + std::to_string(S) + "|";
  while (std::getline(f, line))
    if (line.compare(0, key.size(), key) == 0) found = line.substr(key.size());  // the last entry wins
  return found;
}

static void append_cache(int dev, int sms, int S, const std::string& spec) {
  const char* path = std::getenv("REINDEX_TUNE_CACHE");
  if (!path) return;
  static std::mutex mu;
  std::lock_guard<std::mutex> g(mu);
  std::ofstream f(path, std::ios::app);
  f << device_name(dev) << "|" << sms << "|" << S << "|" << spec << "\n";
}

}  // namespace reindex

using namespace reindex;

extern "C" {

reindex_status reindex_tuning_get(int vtxStrideBytes, char* desc, int descLen) {
  if (!desc || descLen < 1) return REINDEX_ERR_INVALID_ARG;
  const std::string d = describe_tuning(launch_cfg(vtxStrideBytes));
  std::snprintf(desc, (size_t)descLen, "%s", d.c_str());
  return REINDEX_OK;
}

reindex_status reindex_tuning_set(int vtxStrideBytes, const char* spec) {
  if (!spec) return REINDEX_ERR_INVALID_ARG;
  LaunchCfg c = launch_cfg(vtxStrideBytes);
  apply_tuning(c, spec);
  set_launch_cfg(vtxStrideBytes, c);
  return REINDEX_OK;
}

reindex_status reindex_autotune(const void* vtx, int64_t nVtx, int S, const int32_t* idx, int64_t nElem, int k,
                                void* out_vtx, int64_t* out_nVtx, int32_t* out_idx, void* ws, size_t wsBytes,
                                int reps, reindex_stream_t stream, char* desc, int descLen) {
  if (reps < 1) reps = 3;
  if (out_idx == idx) return REINDEX_ERR_INVALID_ARG;  // runs repeat: the input must survive
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return REINDEX_ERR_CUDA;
  auto timed = [&](float* ms) -> reindex_status {
    std::vector<float> t;
    for (int r = 0; r <= reps; ++r) {  // the first run warms up
      cudaEventRecord(e0, st);
      reindex_status rs = reindex_mesh_ws(vtx, nVtx, S, idx, nElem, k, out_vtx, out_nVtx, out_idx, ws, wsBytes, stream);
      if (rs != REINDEX_OK) return rs;
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess) return REINDEX_ERR_CUDA;
      float x = 0.f;
      cudaEventElapsedTime(&x, e0, e1);
      if (r) t.push_back(x);
    }
    std::sort(t.begin(), t.end());
    *ms = t[t.size() / 2];
    return REINDEX_OK;
  };
  const LaunchCfg start = launch_cfg(S);
  LaunchCfg best = start;
  float best_ms = 0.f;
  reindex_status rs = timed(&best_ms);
  const char* knobs[][5] = {{"sort=regs", "sort=pipe", "sort=tiles", "sort=chunk", nullptr},
                            {"rank=ballot", "rank=match", "rank=vary", nullptr, nullptr},
                            {"hist=uniform", "hist=peel", "hist=match", nullptr, nullptr},
                            {"grid=persist", "grid=tile", nullptr, nullptr, nullptr},
                            {"swaves=tile", "swaves=1", "swaves=4", nullptr, nullptr},
                            {"chunk=wide", "chunk=big", "chunk=small", "chunk=deep", nullptr},
                            {"cocc=max", "cocc=1", nullptr, nullptr, nullptr},
                            {"dbits=8", "dbits=7", "dbits=6", nullptr, nullptr},
                            {"dedup=off", "dedup=hash", nullptr, nullptr, nullptr},
                            {"dpub=on", "dpub=off", nullptr, nullptr, nullptr},
                            {"pack=auto", "pack=on", "pack=off", nullptr, nullptr},
                            {"prefix=auto", "prefix=on", "prefix=off", nullptr, nullptr}};
  for (int ki = 0; ki < 12; ++ki) {
    const auto& knob = knobs[ki];
    if (rs != REINDEX_OK) break;
    if (S >= kWideMin && ki < 3) continue;  // 24- and 32-byte keys: the tiles or chunk sort, vary ranking
    if (ki == 9 && !best.dedup) continue;   // publishing: a variant of the hash table only
    for (const char* v : knob) {
      if (!v) continue;
      LaunchCfg c = best;
      apply_tuning(c, v);
      if (describe_tuning(c) == describe_tuning(best)) continue;
      set_launch_cfg(S, c);
      float ms = 0.f;
      rs = timed(&ms);
      if (rs != REINDEX_OK) break;
      if (ms < best_ms) {
        best_ms = ms;
        best = c;
      }
    }
  }
  set_launch_cfg(S, rs == REINDEX_OK ? best : start);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rs != REINDEX_OK) return rs;
  int dev = 0;
  cudaGetDevice(&dev);
  append_cache(dev, best.sms, S, describe_tuning(best));
  if (desc && descLen > 0) std::snprintf(desc, (size_t)descLen, "%s", describe_tuning(best).c_str());
  return REINDEX_OK;
}

}  // extern "C"
