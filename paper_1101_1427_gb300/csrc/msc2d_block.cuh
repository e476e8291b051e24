// Bit-sliced Metropolis update of one block of the 2D coded ferromagnet
// (Sec. 5, synchronous multi-spin coding): the four words 4B .. 4B+3 of row
// y of one colour, i.e. 128 sites, given the acceptance masks of those four
// words for dE = 4 and dE = 8.  Shared by the per-phase kernel and the
// batched kernel.  A lattice is stored as [2 colours][L rows][L/64 words];
// in row y the colour-c sites are x = 2k + ((c + y) & 1), with
// k = 128 B + 4 l + q in bit l of word 4 B + q (bit set <=> s = -1).
#pragma once
#include "common.cuh"

namespace spin {

// kCount 1: adds to down the number of -1 spins among the block's sites
// after the update; kCount 2: also adds to anti their post-update number of
// antiparallel neighbours.
template <int kCount>
__device__ __forceinline__ void msc2d_block(uint32_t *wl, int L, int wpr, int bpr, int colour, int y, uint32_t B,
                                            const uint4 &m4, const uint4 &m8, long long &anti,
                                            long long &down) {
  const int yu = y == 0 ? L - 1 : y - 1, yd = y == L - 1 ? 0 : y + 1;
  const int oc = colour ^ 1;
  uint32_t *S = wl + ((int64_t)colour * L + y) * wpr + 4 * B;
  const uint32_t *O = wl + ((int64_t)oc * L + y) * wpr;
  const uint4 s = *reinterpret_cast<const uint4 *>(S);
  const uint4 o = *reinterpret_cast<const uint4 *>(O + 4 * B);
  const uint4 u = *reinterpret_cast<const uint4 *>(wl + ((int64_t)oc * L + yu) * wpr + 4 * B);
  const uint4 d = *reinterpret_cast<const uint4 *>(wl + ((int64_t)oc * L + yd) * wpr + 4 * B);
  const int p = (colour + y) & 1;
  // second horizontal neighbour: k - 1 (p = 0) or k + 1 (p = 1)
  uint32_t sh[4];
  if (p == 0) {
    const uint32_t Bp = B == 0 ? (uint32_t)bpr - 1 : B - 1;
    sh[0] = (o.w << 1) | (O[4 * Bp + 3] >> 31);
    sh[1] = o.x;
    sh[2] = o.y;
    sh[3] = o.z;
  } else {
    const uint32_t Bn = B == (uint32_t)bpr - 1 ? 0 : B + 1;
    sh[0] = o.y;
    sh[1] = o.z;
    sh[2] = o.w;
    sh[3] = (o.x >> 1) | (O[4 * Bn] << 31);
  }
  const uint32_t sv[4] = {s.x, s.y, s.z, s.w}, ov[4] = {o.x, o.y, o.z, o.w};
  const uint32_t uv[4] = {u.x, u.y, u.z, u.w}, dv[4] = {d.x, d.y, d.z, d.w};
  const uint32_t m4v[4] = {m4.x, m4.y, m4.z, m4.w}, m8v[4] = {m8.x, m8.y, m8.z, m8.w};
  uint32_t nv[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const uint32_t a0 = sv[q] ^ uv[q], a1 = sv[q] ^ dv[q], a2 = sv[q] ^ ov[q], a3 = sv[q] ^ sh[q];
    const uint32_t s1 = a0 ^ a1, c1 = a0 & a1, s2 = a2 ^ a3, c2 = a2 & a3;
    const uint32_t b0 = s1 ^ s2, c3 = s1 & s2;
    const uint32_t b1 = c1 ^ c2 ^ c3, b2 = (c1 & c2) | (c3 & (c1 ^ c2));
    // n antiparallel neighbours, dE = 8 - 4n
    const uint32_t ge2 = b2 | b1, eq1 = ~b2 & ~b1 & b0, eq0 = ~(b2 | b1 | b0);
    nv[q] = sv[q] ^ (ge2 | (eq1 & m4v[q]) | (eq0 & m8v[q]));
    if (kCount >= 1) down += __popc(nv[q]);
    if (kCount == 2)
      anti += __popc(nv[q] ^ uv[q]) + __popc(nv[q] ^ dv[q]) + __popc(nv[q] ^ ov[q]) + __popc(nv[q] ^ sh[q]);
  }
  *reinterpret_cast<uint4 *>(S) = make_uint4(nv[0], nv[1], nv[2], nv[3]);
}

}  // namespace spin
