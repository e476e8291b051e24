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
__device__ __forceinline__ uint64_t mul_wide(uint32_t a, uint32_t b) {
  uint64_t p;
  asm("mul.wide.u32 %0, %1, %2;" : "=l"(p) : "r"(a), "r"(b));
  return p;
}

__device__ __forceinline__ uint4 philox(uint4 c, const RoundKeys &rk) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = mul_wide(0xD2511F53u, c.x);
    const uint64_t p1 = mul_wide(0xCD9E8D57u, c.z);
    const uint32_t lo0 = (uint32_t)p0, hi0 = (uint32_t)(p0 >> 32);
    const uint32_t lo1 = (uint32_t)p1, hi1 = (uint32_t)(p1 >> 32);
    c = make_uint4(hi1 ^ c.y ^ rk.k0[r], lo1, hi0 ^ c.w ^ rk.k1[r], lo0);
  }
  return c;
}

// Philox4x32-10 for counters (x0, x1, x2, x3) of which only x1 changes from
// call to call (a thread re-drawing for the same sites at successive sweep
// numbers): the products and XORs of rounds 0 to 2 that do not involve x1
// are computed once, leaving 16 of the 20 multiplies per call.  Equal to
// philox() word for word.
struct PhiloxX1 {
  uint32_t a;    // hi(M1 x2) ^ k0[0]:             round-1 word 0 is a ^ x1
  uint32_t b;    // lo(M0 x0) ^ k1[1]:             round-2 word 2 is hi(M0 c1.x) ^ b
  uint32_t c2y;  // round-2 word 1
  uint32_t hz;   // hi(M0 c2.x) ^ k1[2]:           round-3 word 2 is hz ^ c2.w
  uint32_t c3w;  // round-3 word 3
};

__device__ __forceinline__ PhiloxX1 philox_x1_setup(uint32_t x0, uint32_t x2, uint32_t x3, const RoundKeys &rk) {
  const uint64_t p0 = mul_wide(0xD2511F53u, x0), p1 = mul_wide(0xCD9E8D57u, x2);
  PhiloxX1 q;
  q.a = (uint32_t)(p1 >> 32) ^ rk.k0[0];
  const uint32_t c1y = (uint32_t)p1, c1z = (uint32_t)(p0 >> 32) ^ x3 ^ rk.k1[0];
  q.b = (uint32_t)p0 ^ rk.k1[1];
  const uint64_t r1 = mul_wide(0xCD9E8D57u, c1z);
  const uint32_t c2x = (uint32_t)(r1 >> 32) ^ c1y ^ rk.k0[1];
  q.c2y = (uint32_t)r1;
  const uint64_t r2 = mul_wide(0xD2511F53u, c2x);
  q.hz = (uint32_t)(r2 >> 32) ^ rk.k1[2];
  q.c3w = (uint32_t)r2;
  return q;
}

__device__ __forceinline__ uint4 philox_x1(const PhiloxX1 &q, uint32_t x1, const RoundKeys &rk) {
  const uint64_t p0 = mul_wide(0xD2511F53u, q.a ^ x1);             // round 1, word 0 product
  const uint32_t c2z = (uint32_t)(p0 >> 32) ^ q.b, c2w = (uint32_t)p0;
  const uint64_t p1 = mul_wide(0xCD9E8D57u, c2z);                  // round 2, word 2 product
  uint4 c = make_uint4((uint32_t)(p1 >> 32) ^ q.c2y ^ rk.k0[2], (uint32_t)p1, q.hz ^ c2w, q.c3w);
#pragma unroll
  for (int r = 3; r < 10; ++r) {
    const uint64_t m0 = mul_wide(0xD2511F53u, c.x);
    const uint64_t m1 = mul_wide(0xCD9E8D57u, c.z);
    c = make_uint4((uint32_t)(m1 >> 32) ^ c.y ^ rk.k0[r], (uint32_t)m1, (uint32_t)(m0 >> 32) ^ c.w ^ rk.k1[r],
                   (uint32_t)m0);
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

// Unsigned 32-bit division by a run-time invariant divisor with one
// multiply-high (Granlund & Montgomery, PLDI 1994, round-up method):
// l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1,
// n / d = (t + ((n - t) >> min(l, 1))) >> max(l - 1, 0) with t = mulhi(m, n).
struct FastDiv {
  uint32_t d, m, s1, s2;
};

inline FastDiv make_fastdiv(uint32_t d) {
  FastDiv f;
  f.d = d;
  uint32_t l = 0;
  while ((1ull << l) < d) ++l;
  f.m = (uint32_t)(((1ull << 32) * ((1ull << l) - d)) / d + 1);
  f.s1 = l < 1 ? l : 1;
  f.s2 = l > 1 ? l - 1 : 0;
  return f;
}

__device__ __forceinline__ uint32_t fdiv(uint32_t n, const FastDiv &f) {
  const uint32_t t = __umulhi(f.m, n);
  return (t + ((n - t) >> f.s1)) >> f.s2;
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
  FastDiv fL;      // division by L
  FastDiv fHalfL;  // division by L / 2
  FastDiv fhalf;   // division by N / 2
  FastDiv fquads;  // division by (N / 2 + 3) / 4
  FastDiv freal;   // division by n_real
  FastDiv ftemps;  // division by n_temps
  FastDiv fgrp;    // division by the number of 32-realisation groups (at least 1)
  FastDiv fgrp2;   // division by the number of 64-realisation group pairs (at least 1)
};

// Colour (x + y + z) mod 2 of site i.
__device__ __forceinline__ uint32_t colour_of(const Geom &g, uint32_t i) {
  const uint32_t row = fdiv(i, g.fL);
  const uint32_t x = i - row * (uint32_t)g.L;
  if (g.dim == 3) {
    const uint32_t z = fdiv(row, g.fL);
    return (x + (row - z * (uint32_t)g.L) + z) & 1u;
  }
  return (x + row) & 1u;
}

// Site of colour index j (colour c): i = 2j + parity, with its coordinates.
struct Site {
  uint32_t i, x, y, z, rowbase;
};

__device__ __forceinline__ Site site_of(const Geom &g, uint32_t j, int colour) {
  Site s;
  const uint32_t i0 = 2u * j;
  const uint32_t row = fdiv(i0, g.fL);  // y + L z
  const uint32_t x0 = i0 - row * (uint32_t)g.L;
  if (g.dim == 3) {
    s.z = fdiv(row, g.fL);
    s.y = row - s.z * (uint32_t)g.L;
  } else {
    s.z = 0;
    s.y = row;
  }
  s.x = x0 + ((colour + s.y + s.z) & 1u);
  s.rowbase = i0 - x0;
  s.i = s.rowbase + s.x;
  return s;
}

// 32-bit versions for per-site kernels (lattice index < 2^32)
__device__ __forceinline__ uint32_t slot_of32(const Geom &g, uint32_t lat) {
  const uint32_t q = fdiv(lat, g.freal);
  return q - fdiv(q, g.ftemps) * (uint32_t)g.n_temps;
}

__device__ __forceinline__ uint32_t lattice_id32(const Geom &g, uint32_t lat) {
  const uint32_t q = fdiv(lat, g.freal);
  const uint32_t r = lat - q * (uint32_t)g.n_real;
  const uint32_t a = fdiv(q, g.ftemps);
  const uint32_t t = q - a * (uint32_t)g.n_temps;
  return lattice_id(a, g.ea ? (r >> 5) : r, t);
}

__host__ __device__ __forceinline__ uint32_t lattice_id_of(const Geom &g, int64_t lat) {
  const uint32_t r = (uint32_t)(lat % g.n_real);
  const uint32_t t = (uint32_t)((lat / g.n_real) % g.n_temps);
  const uint32_t a = (uint32_t)(lat / ((int64_t)g.n_real * g.n_temps));
  return lattice_id(a, g.ea ? (r >> 5) : r, t);
}

__host__ __device__ __forceinline__ int slot_of(const Geom &g, int64_t lat) {
  return (int)((lat / g.n_real) % g.n_temps);
}

// Programmatic dependent launch.  A kernel launched with launch_dependent()
// may start while the previous kernel of its stream is finishing: it calls
// griddep_wait() before touching memory, which returns once that kernel has
// completed and its writes are visible.  griddep_release() lets the next
// such kernel's CTAs be scheduled once every CTA of this grid has started
// (they wait in griddep_wait() until this grid is done).
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_release() { asm volatile("griddepcontrol.launch_dependents;"); }

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
