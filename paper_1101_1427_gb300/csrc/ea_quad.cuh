// Vectorised update of one quad of EA word-sites (asynchronous multi-spin
// coding, 32 realisations per word) for L % 8 == 0.
//
// The four colour sites j = 4 j4 .. 4 j4 + 3 of a quad are the active words
// of the 8-word row segment x0 .. x0+7 (x0 = 8 (j4 mod L/8)): offsets p, p+2,
// p+4, p+6 with p = (colour + y + z) mod 2.  The segment and the segments
// above, below, in front and behind are read with 16-byte loads, so a warp
// reads whole cache lines instead of one word per 32 bytes.
//
// Quads are enumerated class by class: first the rows with y + z even, then
// those with y + z odd (`qk` below).  Inside a class p is the same for every
// quad, and with L^3/16 a multiple of 32 a warp never straddles two classes,
// so the parity is a template argument and all selects vanish.
#pragma once
#include "common.cuh"

namespace spin {

struct QuadPos {
  uint32_t i0;  // first word of the segment
  uint32_t x0, y, z;
  int cls;      // (y + z) mod 2
};

// qk in [0, L^3/8): class-ordered quad index -> segment position.
__device__ __forceinline__ QuadPos quad_pos(uint32_t qk, uint32_t L, const FastDiv &f_qpr,
                                           const FastDiv &f_halfL) {
  const uint32_t half_q = L * L * L / 16;
  QuadPos q;
  q.cls = qk >= half_q ? 1 : 0;
  const uint32_t k = qk - (uint32_t)q.cls * half_q;
  const uint32_t rr = fdiv(k, f_qpr);           // class row
  const uint32_t xq = k - rr * (L >> 3);        // segment within the row
  q.z = fdiv(rr, f_halfL);
  const uint32_t m = rr - q.z * (L >> 1);
  q.y = 2 * m + (((uint32_t)q.cls + q.z) & 1u);
  q.x0 = 8 * xq;
  q.i0 = (q.z * L + q.y) * L + q.x0;
  return q;
}

// 8 consecutive words with two 16-byte loads (generic addressing: the
// couplings may sit in shared memory, the spins in global memory).
__device__ __forceinline__ void ld8(const uint32_t *p, uint32_t (&w)[8]) {
  asm("ld.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]) : "l"(p));
  asm("ld.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(w[4]), "=r"(w[5]), "=r"(w[6]), "=r"(w[7]) : "l"(p + 4));
}

// P: parity of the active words.  kCount: add the post-update number of
// unsatisfied bonds of each site (bit-sliced, 3 planes) to the counter C.
template <int P, bool kCount, int K, typename AddFn>
__device__ __forceinline__ void ea_quad_update(uint32_t *__restrict__ s, const uint32_t *__restrict__ Jg,
                                               uint32_t N, uint32_t L, const QuadPos &q, uint4 r,
                                               uint32_t t4, uint32_t t8, uint32_t t12, uint32_t (&C)[K],
                                               AddFn add3) {
  const uint32_t LL = L * L;
  const uint32_t i0 = q.i0;
  const uint32_t x0 = q.x0;
  const uint32_t rb = i0 - x0;
  const uint32_t iyp = q.y == L - 1 ? i0 - (L - 1) * L : i0 + L;
  const uint32_t iym = q.y == 0 ? i0 + (L - 1) * L : i0 - L;
  const uint32_t izp = q.z == L - 1 ? i0 - (L - 1) * LL : i0 + LL;
  const uint32_t izm = q.z == 0 ? i0 + (L - 1) * LL : i0 - LL;
  uint32_t S[8], YP[8], YM[8], ZP[8], ZM[8], JX[8], JY[8], JYm[8], JZ[8], JZm[8];
  ld8(s + i0, S);
  ld8(s + iyp, YP);
  ld8(s + iym, YM);
  ld8(s + izp, ZP);
  ld8(s + izm, ZM);
  ld8(Jg + i0, JX);
  ld8(Jg + N + i0, JY);
  ld8(Jg + N + iym, JYm);
  ld8(Jg + 2 * N + i0, JZ);
  ld8(Jg + 2 * N + izm, JZm);
  // words just outside the segment: the left one (P == 0) or the right one (P == 1)
  uint32_t outS = 0, outJ = 0;
  if (P == 0) {
    const uint32_t xl = x0 == 0 ? rb + L - 1 : i0 - 1;
    outS = s[xl];
    outJ = Jg[xl];  // x-bond from the left word into word 0
  } else {
    outS = s[x0 + 8 == L ? rb : i0 + 8];
  }
  const uint32_t rw[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int o = P + 2 * k;
    const uint32_t Sv = S[o];
    const uint32_t xp = (o + 1 < 8) ? S[o + 1] : outS;
    const uint32_t xm = (o >= 1) ? S[o - 1] : outS;
    const uint32_t jxm = (o >= 1) ? JX[o - 1] : outJ;
    const uint32_t u0 = Sv ^ xp ^ JX[o];
    const uint32_t u1 = Sv ^ xm ^ jxm;
    const uint32_t u2 = Sv ^ YP[o] ^ JY[o];
    const uint32_t u3 = Sv ^ YM[o] ^ JYm[o];
    const uint32_t u4 = Sv ^ ZP[o] ^ JZ[o];
    const uint32_t u5 = Sv ^ ZM[o] ^ JZm[o];
    const uint32_t s1 = u0 ^ u1 ^ u2, c1 = (u0 & u1) | (u2 & (u0 ^ u1));
    const uint32_t s2 = u3 ^ u4 ^ u5, c2 = (u3 & u4) | (u5 & (u3 ^ u4));
    const uint32_t b0 = s1 ^ s2, c3 = s1 & s2;
    const uint32_t b1 = c1 ^ c2 ^ c3, b2 = (c1 & c2) | (c3 & (c1 ^ c2));
    const uint32_t rq = rw[k];
    const uint32_t R4 = rq < t4 ? ~0u : 0u, R8 = rq < t8 ? ~0u : 0u, R12 = rq < t12 ? ~0u : 0u;
    const uint32_t ge3 = b2 | (b1 & b0);
    const uint32_t eq2 = ~b2 & b1 & ~b0, eq1 = ~b2 & ~b1 & b0, eq0 = ~(b2 | b1 | b0);
    const uint32_t F = ge3 | (eq2 & R4) | (eq1 & R8) | (eq0 & R12);
    S[o] = Sv ^ F;
    if (kCount) {
      // a flip turns u unsatisfied bonds into 6 - u: bit 0 is unchanged
      const uint32_t v1 = (b2 & ~b1 & ~b0) | (~b2 & ~(b1 ^ b0));
      const uint32_t v2 = ~b2 & ~(b1 & b0);
      add3(C, b0, (F & v1) | (~F & b1), (F & v2) | (~F & b2));
    }
  }
  reinterpret_cast<uint4 *>(s + i0)[0] = make_uint4(S[0], S[1], S[2], S[3]);
  reinterpret_cast<uint4 *>(s + i0)[1] = make_uint4(S[4], S[5], S[6], S[7]);
}

}  // namespace spin
