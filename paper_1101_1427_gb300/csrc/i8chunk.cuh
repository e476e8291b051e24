// Metropolis update of one 8-site chunk of a 2D int8 (+-1) ferromagnet row
// (Eq. metropolis), shared by the tile and batched kernels.
#pragma once
#include "common.cuh"

namespace spin {

// One chunk of 8 sites (a row segment, int8 +-1) whose sites of the phase's
// colour sit at byte offsets p, p + 2, p + 4, p + 6: returns the chunk with
// those sites updated.  Only bytes of the other colour are read around
// them, and the phase never changes those.  kCount 1: adds the updated
// sites' number of -1 spins after the update to down; kCount 2: also their
// post-update number of antiparallel neighbours to anti.
template <int kCount>
__device__ __forceinline__ uint64_t ising_chunk(uint64_t C, uint64_t Uw, uint64_t Dw, uint64_t lb, uint64_t rb,
                                                const uint4 &r, int p, uint32_t thr4, uint32_t thr8,
                                                long long &anti, long long &down) {
  const uint64_t MASK = 0x0202020202020202ull;  // bit 1 of each byte: 1 for -1, 0 for +1
  const uint64_t Lw = (C << 8) | lb, Rw = (C >> 8) | (rb << 56);
  // per byte: twice the number of antiparallel neighbours
  const uint64_t A = ((C ^ Uw) & MASK) + ((C ^ Dw) & MASK) + ((C ^ Lw) & MASK) + ((C ^ Rw) & MASK);
  const uint64_t An = A >> (8 * p);
  const uint32_t lo = (uint32_t)An, hi = (uint32_t)(An >> 32);
  // dE <= 0 (at least two antiparallel neighbours): flip
  const uint32_t g_lo = ((lo | (lo >> 1)) >> 2) & 0x00010001u;
  const uint32_t g_hi = ((hi | (hi >> 1)) >> 2) & 0x00010001u;
  // one antiparallel neighbour: dE = 4; none: dE = 8
  const uint32_t q0 = (lo & 0x2u) ? thr4 : thr8, q1 = (lo & 0x20000u) ? thr4 : thr8;
  const uint32_t q2 = (hi & 0x2u) ? thr4 : thr8, q3 = (hi & 0x20000u) ? thr4 : thr8;
  const uint32_t f_lo = g_lo | (uint32_t)(r.x < q0) | ((uint32_t)(r.y < q1) << 16);
  const uint32_t f_hi = g_hi | (uint32_t)(r.z < q2) | ((uint32_t)(r.w < q3) << 16);
  if (kCount == 2) {
    const uint32_t n0 = (lo >> 1) & 7u, n1 = (lo >> 17) & 7u, n2 = (hi >> 1) & 7u, n3 = (hi >> 17) & 7u;
    anti += (long long)((f_lo & 1u) ? 4u - n0 : n0) + ((f_lo >> 16) ? 4u - n1 : n1) +
            ((f_hi & 1u) ? 4u - n2 : n2) + ((f_hi >> 16) ? 4u - n3 : n3);
  }
  if (kCount >= 1) {
    const uint64_t old_down = (C >> (8 * p)) & 0x0002000200020002ull;
    const uint64_t flips = ((uint64_t)f_hi << 33) | ((uint64_t)f_lo << 1);
    down += __popcll(old_down ^ flips);
  }
  return C ^ ((((uint64_t)(f_hi * 0xFEu) << 32) | (uint64_t)(f_lo * 0xFEu)) << (8 * p));
}

}  // namespace spin
