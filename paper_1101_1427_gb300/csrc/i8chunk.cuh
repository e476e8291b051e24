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
  // the four sites (bytes p, p+2, p+4, p+6) and each of their neighbours,
  // gathered into one 32-bit word apiece.  The horizontal neighbours of the
  // sites are the chunk's other-colour bytes O (right neighbours for p = 0,
  // left ones for p = 1) and the same bytes shifted by one site with the
  // byte beyond the chunk moved in (lb for p = 0, rb for p = 1); the count
  // below does not depend on which of the two is left and which is right.
  const uint32_t lo = (uint32_t)C, hi = (uint32_t)(C >> 32);
  const uint32_t sel = p ? 0x7531u : 0x6420u;
  const uint32_t S = __byte_perm(lo, hi, sel);
  const uint32_t O = __byte_perm(lo, hi, p ? 0x6420u : 0x7531u);
  const uint32_t E = __byte_perm(O, (uint32_t)(p ? rb : lb), p ? 0x4321u : 0x2104u);
  const uint32_t Un = __byte_perm((uint32_t)Uw, (uint32_t)(Uw >> 32), sel);
  const uint32_t Dn = __byte_perm((uint32_t)Dw, (uint32_t)(Dw >> 32), sel);
  // per site: 2n, n the number of antiparallel neighbours (bit 1 of a +-1
  // byte is set for -1, so (a ^ b) & 2 is 2 iff a != b); dE = 8 - 4n
  const uint32_t M = 0x02020202u;
  const uint32_t A = ((S ^ Un) & M) + ((S ^ Dn) & M) + ((S ^ O) & M) + ((S ^ E) & M);
  // n >= 2 (dE <= 0) flips; n = 1 flips iff r < thr4, n = 0 iff r < thr8
  uint32_t f = ((A | (A >> 1)) >> 2) & 0x01010101u;
  const uint32_t t0 = (A & 0x2u) ? thr4 : thr8, t1 = (A & 0x200u) ? thr4 : thr8;
  const uint32_t t2 = (A & 0x20000u) ? thr4 : thr8, t3 = (A & 0x2000000u) ? thr4 : thr8;
  f |= (r.x < t0 ? 0x1u : 0u) | (r.y < t1 ? 0x100u : 0u) | (r.z < t2 ? 0x10000u : 0u) |
       (r.w < t3 ? 0x1000000u : 0u);
  if (kCount >= 1) down += __popc(((S >> 1) & 0x01010101u) ^ f);
  if (kCount == 2) {
    const uint32_t n4 = (A >> 1) & 0x07070707u, m = f * 0xFFu;
    const uint32_t after = (n4 & ~m) | ((0x04040404u - n4) & m);  // a flip turns n into 4 - n
    anti += (long long)((after * 0x01010101u) >> 24);
  }
  // 0xFE (+1 <-> -1) in the bytes of the flipping sites, scattered back
  const uint32_t F = f * 0xFEu;
  const uint32_t flo = __byte_perm(F, 0u, p ? 0x1404u : 0x4140u);
  const uint32_t fhi = __byte_perm(F, 0u, p ? 0x3424u : 0x4342u);
  return C ^ (((uint64_t)fhi << 32) | flo);
}

// One chunk of 8 sites of a row of a 3D int8 (+-1) ferromagnet, as
// ising_chunk with two further neighbour words in z (Fw: plane z - 1, Bw:
// plane z + 1) and the one byte beyond the chunk the phase needs (the byte
// left of byte 0 for p = 0, right of byte 7 for p = 1).  n antiparallel
// neighbours of six, dE = 12 - 4n: n >= 3 flips; n = 2, 1, 0 flip iff
// r < thr4, thr8, thr12.
__device__ __forceinline__ uint64_t ising3d_chunk(uint64_t C, uint64_t Uw, uint64_t Dw, uint64_t Fw,
                                                  uint64_t Bw, uint32_t edge, const uint4 &r, int p,
                                                  uint32_t thr4, uint32_t thr8, uint32_t thr12) {
  const uint32_t lo = (uint32_t)C, hi = (uint32_t)(C >> 32);
  const uint32_t sel = p ? 0x7531u : 0x6420u;
  const uint32_t S = __byte_perm(lo, hi, sel);
  const uint32_t O = __byte_perm(lo, hi, p ? 0x6420u : 0x7531u);
  const uint32_t E = __byte_perm(O, edge, p ? 0x4321u : 0x2104u);
  const uint32_t Un = __byte_perm((uint32_t)Uw, (uint32_t)(Uw >> 32), sel);
  const uint32_t Dn = __byte_perm((uint32_t)Dw, (uint32_t)(Dw >> 32), sel);
  const uint32_t Fn = __byte_perm((uint32_t)Fw, (uint32_t)(Fw >> 32), sel);
  const uint32_t Bn = __byte_perm((uint32_t)Bw, (uint32_t)(Bw >> 32), sel);
  // per site 2n in 0..12 (six terms of 0 or 2 per byte, no carries)
  const uint32_t M = 0x02020202u;
  const uint32_t A = ((S ^ Un) & M) + ((S ^ Dn) & M) + ((S ^ Fn) & M) + ((S ^ Bn) & M) + ((S ^ O) & M) +
                     ((S ^ E) & M);
  // n >= 3 <=> 2n >= 6 <=> bit 3 set, or bits 2 and 1 both set
  uint32_t f = ((A >> 3) | ((A >> 2) & (A >> 1))) & 0x01010101u;
  // below that, 2n = 4 (bit 2) takes thr4, 2n = 2 (bit 1) thr8, 2n = 0 thr12
  const uint32_t t0 = (A & 0x4u) ? thr4 : ((A & 0x2u) ? thr8 : thr12);
  const uint32_t t1 = (A & 0x400u) ? thr4 : ((A & 0x200u) ? thr8 : thr12);
  const uint32_t t2 = (A & 0x40000u) ? thr4 : ((A & 0x20000u) ? thr8 : thr12);
  const uint32_t t3 = (A & 0x4000000u) ? thr4 : ((A & 0x2000000u) ? thr8 : thr12);
  f |= (r.x < t0 ? 0x1u : 0u) | (r.y < t1 ? 0x100u : 0u) | (r.z < t2 ? 0x10000u : 0u) |
       (r.w < t3 ? 0x1000000u : 0u);
  const uint32_t F = f * 0xFEu;
  const uint32_t flo = __byte_perm(F, 0u, p ? 0x1404u : 0x4140u);
  const uint32_t fhi = __byte_perm(F, 0u, p ? 0x3424u : 0x4342u);
  return C ^ (((uint64_t)fhi << 32) | flo);
}

}  // namespace spin
