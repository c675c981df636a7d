// Device versions of the seeded mesh generators of synth.py (inputs only; no re-indexing
// arithmetic).  Every value is computed exactly as synth.py computes it: SplitMix64 hashes of
// (seed, tag, coordinates), float32 products and sums rounded one operation at a time
// (__fmul_rn / __fadd_rn / __fsub_rn never contract to FMA), and the same Feistel cycle-walking
// permutation of the vertex array.  The output is bit-identical to the host generator, which the
// GPU tests check; it lets a benchmark create hundreds of gigabytes of requests without the host.
//
// C ABI (device pointers, asynchronous on `stream`; returns 0, or a cudaError_t value):
//   synth_heightfield(vtx float32[N][3], idx int32[6*G*Gy], G, Gy, n_extra, seed, permute, stream)
//   synth_tets(vtx float32[N][4], idx int32[20*L^3], L, n_extra, seed, permute, stream)
// with N = soup vertices + n_extra, and
//   synth_attributes(in uint32[n][k_in], n, k_in, out uint32[n][k_out], k_out, seed, stream)
// which copies each vertex and appends k_out - k_in attribute words (synth.with_attributes).
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr uint64_t kTagNoise = 1, kTagExtra = 2, kTagPerm = 3, kTagJitter = 4, kTagField = 5, kTagAttr = 7;

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t hash_base(uint64_t seed, uint64_t tag) {
  return splitmix64(seed * 0x100000001B3ull + tag);
}
__device__ __forceinline__ uint64_t hmix(uint64_t h, int64_t c) { return splitmix64(h ^ (uint64_t)c); }

__device__ __forceinline__ float unit_float(uint64_t h) {
  return __fmul_rn((float)(uint32_t)(h >> 40), 1.0f / 16777216.0f);
}

// Four-round Feistel network on 2*hb-bit integers, then cycle walking into [0, n).
__device__ __forceinline__ uint64_t perm_dest(uint64_t x, uint64_t n, int hb, uint64_t seed) {
  const uint64_t mask = (1ull << hb) - 1ull;
  const uint64_t base = hash_base(seed, kTagPerm);
  do {
    uint64_t left = x >> hb, right = x & mask;
#pragma unroll
    for (int rnd = 0; rnd < 4; ++rnd) {
      const uint64_t f = hmix(hmix(base, rnd), (int64_t)right) & mask;
      const uint64_t nl = right;
      right = left ^ f;
      left = nl;
    }
    x = (left << hb) | right;
  } while (x >= n);
  return x;
}

__device__ __forceinline__ float lattice_value(uint64_t base, int64_t c0, int64_t c1, int64_t c2) {
  return __fsub_rn(__fmul_rn(unit_float(hmix(hmix(hmix(base, c0), c1), c2)), 2.0f), 1.0f);
}

// Four octaves of bilinear value noise (cell sizes 64/32/16/8, amplitudes 1, 1/2, 1/4, 1/8).
__device__ float noise2(int64_t a, int64_t b, uint64_t seed) {
  const uint64_t base = hash_base(seed, kTagNoise);
  float h = 0.0f;
#pragma unroll
  for (int octave = 0; octave < 4; ++octave) {
    const int64_t cs = 64 >> octave;
    const float amp = 1.0f / (float)(1 << octave);
    const int64_t ca = a / cs, cb = b / cs;
    const float inv = 1.0f / (float)cs;
    const float fa = __fmul_rn((float)(a % cs), inv), fb = __fmul_rn((float)(b % cs), inv);
    const uint64_t ob = hmix(base, octave);
    const float v00 = __fsub_rn(__fmul_rn(unit_float(hmix(hmix(ob, ca), cb)), 2.0f), 1.0f);
    const float v10 = __fsub_rn(__fmul_rn(unit_float(hmix(hmix(ob, ca + 1), cb)), 2.0f), 1.0f);
    const float v01 = __fsub_rn(__fmul_rn(unit_float(hmix(hmix(ob, ca), cb + 1)), 2.0f), 1.0f);
    const float v11 = __fsub_rn(__fmul_rn(unit_float(hmix(hmix(ob, ca + 1), cb + 1)), 2.0f), 1.0f);
    const float v0 = __fadd_rn(v00, __fmul_rn(__fsub_rn(v10, v00), fa));
    const float v1 = __fadd_rn(v01, __fmul_rn(__fsub_rn(v11, v01), fa));
    const float v = __fadd_rn(v0, __fmul_rn(__fsub_rn(v1, v0), fb));
    h = __fadd_rn(h, __fmul_rn(amp, v));
  }
  return h;
}

// One octave of trilinear value noise with cell size 16.
__device__ float noise3(int64_t a, int64_t b, int64_t c, uint64_t seed) {
  const uint64_t base = hash_base(seed, kTagField);
  const int64_t cs = 16;
  const int64_t ca = a / cs, cb = b / cs, cc = c / cs;
  const float inv = 1.0f / 16.0f;
  const float fa = __fmul_rn((float)(a % cs), inv), fb = __fmul_rn((float)(b % cs), inv),
              fc = __fmul_rn((float)(c % cs), inv);
  const float v000 = lattice_value(base, ca, cb, cc), v100 = lattice_value(base, ca + 1, cb, cc);
  const float v010 = lattice_value(base, ca, cb + 1, cc), v110 = lattice_value(base, ca + 1, cb + 1, cc);
  const float v001 = lattice_value(base, ca, cb, cc + 1), v101 = lattice_value(base, ca + 1, cb, cc + 1);
  const float v011 = lattice_value(base, ca, cb + 1, cc + 1), v111 = lattice_value(base, ca + 1, cb + 1, cc + 1);
  const float x00 = __fadd_rn(v000, __fmul_rn(__fsub_rn(v100, v000), fa));
  const float x10 = __fadd_rn(v010, __fmul_rn(__fsub_rn(v110, v010), fa));
  const float x01 = __fadd_rn(v001, __fmul_rn(__fsub_rn(v101, v001), fa));
  const float x11 = __fadd_rn(v011, __fmul_rn(__fsub_rn(v111, v011), fa));
  const float y0 = __fadd_rn(x00, __fmul_rn(__fsub_rn(x10, x00), fb));
  const float y1 = __fadd_rn(x01, __fmul_rn(__fsub_rn(x11, x01), fb));
  return __fadd_rn(y0, __fmul_rn(__fsub_rn(y1, y0), fc));
}

__device__ __forceinline__ int half_bits(uint64_t n) {
  int bits = n > 1 ? 64 - __clzll((long long)(n - 1)) : 1;
  if (bits < 2) bits = 2;
  bits += bits & 1;
  return bits / 2;
}

__global__ void k_heightfield(float* vtx, int32_t* idx, int64_t G, int64_t Gy, int64_t n_extra, uint64_t seed,
                              int permute) {
  const int64_t M = 6 * G * Gy, N = M + n_extra;
  const int hb = half_bits((uint64_t)N);
  const int da[6] = {0, 1, 1, 0, 1, 0}, db[6] = {0, 0, 1, 0, 1, 1};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t dst = permute ? (int64_t)perm_dest((uint64_t)i, (uint64_t)N, hb, seed) : i;
    float x, y, z;
    if (i < M) {
      const int64_t cell = i / 6, c = i % 6;
      const int64_t a = cell % G + da[c], b = cell / G + db[c];
      x = (float)a;
      y = (float)b;
      z = noise2(a, b, seed);
      idx[i] = (int32_t)dst;
    } else {
      const int64_t e = i - M;
      const uint64_t base = hash_base(seed, kTagExtra);
      x = __fmul_rn(unit_float(hmix(hmix(base, 0), e)), (float)G);
      y = __fmul_rn(unit_float(hmix(hmix(base, 1), e)), (float)Gy);
      z = __fsub_rn(__fmul_rn(unit_float(hmix(hmix(base, 2), e)), 4.0f), 2.0f);
    }
    vtx[3 * dst] = x;
    vtx[3 * dst + 1] = y;
    vtx[3 * dst + 2] = z;
  }
}

// Five-tetrahedron split of a cube (corner k = dx + 2*dy + 4*dz), by parity of i + j + k.
__constant__ int8_t c_tets[2][5][4] = {{{0, 1, 2, 4}, {3, 1, 2, 7}, {5, 1, 4, 7}, {6, 2, 4, 7}, {1, 2, 4, 7}},
                                       {{1, 0, 3, 5}, {2, 0, 3, 6}, {4, 0, 5, 6}, {7, 3, 5, 6}, {0, 3, 5, 6}}};

__global__ void k_tets(float4* vtx, int32_t* idx, int64_t L, int64_t n_extra, uint64_t seed, int permute) {
  const int64_t M = 20 * L * L * L, N = M + n_extra;
  const int hb = half_bits((uint64_t)N);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t dst = permute ? (int64_t)perm_dest((uint64_t)i, (uint64_t)N, hb, seed) : i;
    float4 v;
    if (i < M) {
      const int64_t t = i / 4, q = i % 4;
      const int64_t cell = t / 5, tt = t % 5;
      const int64_t I = cell % L, J = (cell / L) % L, K = cell / (L * L);
      const int corner = c_tets[(I + J + K) & 1][tt][q];
      const int64_t a = I + (corner & 1), b = J + ((corner >> 1) & 1), c = K + ((corner >> 2) & 1);
      const uint64_t jb = hash_base(seed, kTagJitter);
      v.x = __fadd_rn((float)a, __fsub_rn(__fmul_rn(unit_float(hmix(hmix(hmix(hmix(jb, 0), a), b), c)), 0.5f), 0.25f));
      v.y = __fadd_rn((float)b, __fsub_rn(__fmul_rn(unit_float(hmix(hmix(hmix(hmix(jb, 1), a), b), c)), 0.5f), 0.25f));
      v.z = __fadd_rn((float)c, __fsub_rn(__fmul_rn(unit_float(hmix(hmix(hmix(hmix(jb, 2), a), b), c)), 0.5f), 0.25f));
      v.w = noise3(a, b, c, seed);
      idx[i] = (int32_t)dst;
    } else {
      const int64_t e = i - M;
      const uint64_t base = hash_base(seed, kTagExtra);
      v.x = __fmul_rn(unit_float(hmix(hmix(base, 0), e)), (float)L);
      v.y = __fmul_rn(unit_float(hmix(hmix(base, 1), e)), (float)L);
      v.z = __fmul_rn(unit_float(hmix(hmix(base, 2), e)), (float)L);
      v.w = __fsub_rn(__fmul_rn(unit_float(hmix(hmix(base, 3), e)), 2.0f), 1.0f);
    }
    vtx[dst] = v;
  }
}

// Attribute q of vertex i: hash of (seed, kTagAttr, q, its key words); q < 3 maps to [-1, 1).
__global__ void k_attributes(const uint32_t* in, int64_t n, int k_in, uint32_t* out, int k_out, uint64_t seed) {
  const uint64_t base = hash_base(seed, kTagAttr);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t* v = in + i * k_in;
    uint32_t* o = out + i * k_out;
    for (int c = 0; c < k_in; ++c) o[c] = v[c];
    for (int q = 0; q < k_out - k_in; ++q) {
      uint64_t h = hmix(base, q);
      for (int c = 0; c < k_in; ++c) h = hmix(h, (int64_t)v[c]);
      float u = unit_float(h);
      if (q < 3) u = __fsub_rn(__fmul_rn(u, 2.0f), 1.0f);
      o[k_in + q] = __float_as_uint(u);
    }
  }
}

int grid_for(int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;
  return g < 1 ? 1 : (int)g;
}

}  // namespace

extern "C" int synth_heightfield(void* vtx, int32_t* idx, int64_t G, int64_t Gy, int64_t n_extra, uint64_t seed,
                                 int permute, cudaStream_t stream) {
  const int64_t N = 6 * G * Gy + n_extra;
  if (N == 0) return 0;
  k_heightfield<<<grid_for(N), 256, 0, stream>>>(static_cast<float*>(vtx), idx, G, Gy, n_extra, seed, permute);
  return (int)cudaGetLastError();
}

extern "C" int synth_tets(void* vtx, int32_t* idx, int64_t L, int64_t n_extra, uint64_t seed, int permute,
                          cudaStream_t stream) {
  const int64_t N = 20 * L * L * L + n_extra;
  if (N == 0) return 0;
  k_tets<<<grid_for(N), 256, 0, stream>>>(static_cast<float4*>(vtx), idx, L, n_extra, seed, permute);
  return (int)cudaGetLastError();
}

extern "C" int synth_attributes(const void* in, int64_t n, int k_in, void* out, int k_out, uint64_t seed,
                                cudaStream_t stream) {
  if (n == 0) return 0;
  if (k_in < 1 || k_out < k_in) return (int)cudaErrorInvalidValue;
  k_attributes<<<grid_for(n), 256, 0, stream>>>(static_cast<const uint32_t*>(in), n, k_in, static_cast<uint32_t*>(out),
                                                k_out, seed);
  return (int)cudaGetLastError();
}
