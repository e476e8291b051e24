// Device-side building blocks shared by the kernels of the library.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace spin {

// Random-word tags: the high nibble of counter word 3.
enum Tag : uint32_t {
  TAG_UPDATE = 0,     // Ising / EA Metropolis uniform, one word per (word-)site
  TAG_INIT = 1,       // Ising / EA hot start, one word per site
  TAG_COUPLING = 2,   // EA couplings, one word per (group, direction, site)
  TAG_PT = 3,         // replica exchange, one word per realisation
  TAG_HEIS = 4,       // Heisenberg update, one whole call per site
  TAG_HEIS_INIT = 5,  // Heisenberg hot start, one whole call per site
};

// Philox4x32-10 round keys for one seed: key + r * (0x9E3779B9, 0xBB67AE85).
// They are the same for every thread, so they travel in the kernel's
// parameter space instead of being recomputed per call.
struct RoundKeys {
  uint32_t k0[10];
  uint32_t k1[10];
};

inline RoundKeys make_round_keys(uint64_t seed) {
  RoundKeys rk;
  uint32_t k0 = (uint32_t)(seed & 0xffffffffu), k1 = (uint32_t)(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    rk.k0[r] = k0;
    rk.k1[r] = k1;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return rk;
}

// Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32->64
// multiplications whose halves are mixed with the other two counter words
// and the round key.
__device__ __forceinline__ uint4 philox(uint4 c, const RoundKeys &rk) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ rk.k0[r], lo1, hi0 ^ c.w ^ rk.k1[r], lo0);
  }
  return c;
}

__host__ __device__ __forceinline__ uint32_t ctr_w(uint32_t tag, uint32_t colour, uint32_t extra) {
  return (tag << 28) | (colour << 27) | extra;
}

__host__ __device__ __forceinline__ uint32_t lattice_id(uint32_t a, uint32_t rkey, uint32_t t) {
  return (a << 24) | (rkey << 12) | t;
}

__device__ __forceinline__ uint32_t word_of(const uint4 &v, uint32_t q) {
  return q == 0 ? v.x : q == 1 ? v.y : q == 2 ? v.z : v.w;
}

// 24-bit uniform in [0, 1), exact in float.
__device__ __forceinline__ float uniform24(uint32_t x) {
  return __uint2float_rn(x >> 8) * 5.9604644775390625e-8f;
}

// Geometry of one lattice of a handle.
struct Geom {
  int dim;
  int L;
  int64_t N;       // L^dim
  int n_real;
  int n_temps;
  int n_sets;
  int ea;          // realisation key is r >> 5
};

__host__ __device__ __forceinline__ uint32_t lattice_id_of(const Geom &g, int64_t lat) {
  const uint32_t r = (uint32_t)(lat % g.n_real);
  const uint32_t t = (uint32_t)((lat / g.n_real) % g.n_temps);
  const uint32_t a = (uint32_t)(lat / ((int64_t)g.n_real * g.n_temps));
  return lattice_id(a, g.ea ? (r >> 5) : r, t);
}

__host__ __device__ __forceinline__ int slot_of(const Geom &g, int64_t lat) {
  return (int)((lat / g.n_real) % g.n_temps);
}

// Warp-level sums.
__device__ __forceinline__ long long warp_sum(long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace spin
