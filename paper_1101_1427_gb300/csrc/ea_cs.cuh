// +-J EA glass, asynchronous multi-spin coding, colour-split storage.
//
// A word-lattice (one replica set, one realisation group of 32, one slot)
// stores its N = L^3 words as [colour][N/2]: site i of colour c sits at
// c N/2 + (i >> 1), i.e. at its colour index j = i >> 1.  Couplings of a
// group are stored as [direction][colour][N/2]: the bond (i, i + e_d) at
// d N + c(i) N/2 + (i >> 1).  During a colour phase the updated words, their
// six neighbours (all of the other colour) and the couplings are then
// contiguous across consecutive colour indices, so the lanes of a warp read
// whole cache lines.
#pragma once
#include "common.cuh"

namespace spin {

__host__ __device__ __forceinline__ uint32_t cs_word(uint32_t i, uint32_t colour, uint32_t half) {
  return colour * half + (i >> 1);
}

// Geometry of colour index j (colour c): site i and the linear indices of
// its six neighbours.
struct CsSite {
  uint32_t i, rb, xp, xm, yp, ym, zp, zm;  // rb: first site of the row
};

__device__ __forceinline__ CsSite cs_site(uint32_t j, int colour, uint32_t L, const FastDiv &fL) {
  const uint32_t LL = L * L;
  const uint32_t i0 = 2u * j;
  const uint32_t row = fdiv(i0, fL);
  const uint32_t x0 = i0 - row * L;
  const uint32_t z = fdiv(row, fL), y = row - z * L;
  const uint32_t x = x0 + ((colour + y + z) & 1u);
  const uint32_t rb = i0 - x0, i = rb + x;
  CsSite s;
  s.i = i;
  s.rb = rb;
  s.xp = rb + (x == L - 1 ? 0 : x + 1);
  s.xm = rb + (x == 0 ? L - 1 : x - 1);
  s.yp = y == L - 1 ? i - (L - 1) * L : i + L;
  s.ym = y == 0 ? i + (L - 1) * L : i - L;
  s.zp = z == L - 1 ? i - (L - 1) * LL : i + LL;
  s.zm = z == 0 ? i + (L - 1) * LL : i - LL;
  return s;
}

// Metropolis flip mask of one word-site from its six bond words
// u_k = s ^ s_nb ^ J (1 = unsatisfied) and the shared uniform r:
// dE = 12 - 4u per realisation; flip iff u >= 3 or r < thr(dE).  The
// thresholds decrease with dE (thr12 <= thr8 <= thr4).
// Also returns the bit-sliced count (b0, b1, b2) of u.
struct Flip {
  uint32_t F, b0, b1, b2;
};

__device__ __forceinline__ Flip ea_flip(uint32_t u0, uint32_t u1, uint32_t u2, uint32_t u3, uint32_t u4,
                                        uint32_t u5, uint32_t r, uint32_t t4, uint32_t t8, uint32_t t12) {
  const uint32_t s1 = u0 ^ u1 ^ u2, c1 = (u0 & u1) | (u2 & (u0 ^ u1));
  const uint32_t s2 = u3 ^ u4 ^ u5, c2 = (u3 & u4) | (u5 & (u3 ^ u4));
  Flip f;
  f.b0 = s1 ^ s2;
  const uint32_t c3 = s1 & s2;
  f.b1 = c1 ^ c2 ^ c3;
  f.b2 = (c1 & c2) | (c3 & (c1 ^ c2));
  // thr12 <= thr8 <= thr4, so the tests are nested: r < thr12 flips every
  // bit, else r < thr8 those with u >= 1, else r < thr4 those with u >= 2,
  // else those with u >= 3
  const uint32_t ge3 = f.b2 | (f.b1 & f.b0), ge2 = f.b2 | f.b1, ge1 = ge2 | f.b0;
  f.F = r < t12 ? ~0u : (r < t8 ? ge1 : (r < t4 ? ge2 : ge3));
  return f;
}

// Post-update number of unsatisfied bonds (bit-sliced): a flip turns u into
// 6 - u, whose bit 0 equals that of u.
__device__ __forceinline__ void ea_after(const Flip &f, uint32_t &a0, uint32_t &a1, uint32_t &a2) {
  const uint32_t v1 = (f.b2 & ~f.b1 & ~f.b0) | (~f.b2 & ~(f.b1 ^ f.b0));
  const uint32_t v2 = ~f.b2 & ~(f.b1 & f.b0);
  a0 = f.b0;
  a1 = (f.F & v1) | (~f.F & f.b1);
  a2 = (f.F & v2) | (~f.F & f.b2);
}

__device__ __forceinline__ uint4 ldv4(const uint32_t *p) {
  uint4 v;
  asm("ld.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
  return v;
}

// ---------------------------------------------------------------- 2D
// The square lattice (the paper's own Sec. 5 benchmark is 2D): four bonds,
// dE = 8 - 4u per realisation; flip iff u >= 2 or r < thr(dE).  Storage and
// couplings as in 3D with two directions ([2][colour][N/2] per group).

// Colour index j (colour c) of an L x L lattice: site i, row start and the
// linear indices of the four neighbours.
__device__ __forceinline__ CsSite cs_site2(uint32_t j, int colour, uint32_t L, const FastDiv &fL) {
  const uint32_t i0 = 2u * j;
  const uint32_t y = fdiv(i0, fL);
  const uint32_t x0 = i0 - y * L;
  const uint32_t x = x0 + ((colour + y) & 1u);
  const uint32_t rb = i0 - x0, i = rb + x;
  CsSite s;
  s.i = i;
  s.rb = rb;
  s.xp = rb + (x == L - 1 ? 0 : x + 1);
  s.xm = rb + (x == 0 ? L - 1 : x - 1);
  s.yp = y == L - 1 ? i - (L - 1) * L : i + L;
  s.ym = y == 0 ? i + (L - 1) * L : i - L;
  s.zp = s.zm = i;
  return s;
}

// Flip mask of one word-site from its four bond words (1 = unsatisfied)
// and the bit-sliced count (b0, b1, b2) of u in 0..4.
__device__ __forceinline__ Flip ea_flip2(uint32_t u0, uint32_t u1, uint32_t u2, uint32_t u3, uint32_t r,
                                         uint32_t t4, uint32_t t8) {
  const uint32_t s1 = u0 ^ u1, c1 = u0 & u1, s2 = u2 ^ u3, c2 = u2 & u3;
  Flip f;
  f.b0 = s1 ^ s2;
  const uint32_t c3 = s1 & s2;
  f.b1 = c1 ^ c2 ^ c3;
  f.b2 = c1 & c2;
  // nested tests as in ea_flip: r < thr8 flips every bit, else r < thr4
  // those with u >= 1, else those with u >= 2
  const uint32_t ge2 = f.b2 | f.b1, ge1 = ge2 | f.b0;
  f.F = r < t8 ? ~0u : (r < t4 ? ge1 : ge2);
  return f;
}

// Post-update count (bit-sliced): a flip turns u into 4 - u.
__device__ __forceinline__ void ea_after2(const Flip &f, uint32_t &a0, uint32_t &a1, uint32_t &a2) {
  const uint32_t v1 = ~f.b2 & (f.b1 ^ f.b0), v2 = ~(f.b2 | f.b1 | f.b0);
  a0 = f.b0;
  a1 = (f.F & v1) | (~f.F & f.b1);
  a2 = (f.F & v2) | (~f.F & f.b2);
}

// ---------------------------------------------------------------- quads
// When L % 8 == 0 the quad j0 = 4 j4 .. 4 j4 + 3 of one colour is four
// consecutive colour indices of one row, so each neighbour direction is one
// 16-byte load.  Its geometry and the coupling words of its bonds depend
// only on the realisation group, not on the replica set or slot: a thread
// that updates the quad in several word-lattices of one group computes them
// once (ea_quad_geom, ea_quad_couplings) and then updates each word-lattice
// (ea_quad_update).
struct EaQuadGeom {
  uint32_t j0;              // first colour index of the quad
  uint32_t jx;              // colour index of the other-colour word beyond the quad in x
  uint32_t yp, ym, zp, zm;  // first colour indices of the neighbour quads in y and z
  uint32_t p;               // x parity of the quad's sites
};

template <int kDim>
__device__ __forceinline__ EaQuadGeom ea_quad_geom(uint32_t j4, int colour, uint32_t L, const FastDiv &fL) {
  EaQuadGeom q;
  q.j0 = 4 * j4;
  const CsSite st = kDim == 3 ? cs_site(q.j0, colour, L, fL) : cs_site2(q.j0, colour, L, fL);
  q.p = st.i & 1u;
  const uint32_t jr = st.rb >> 1, LH = L >> 1;  // first colour index of the row, colour indices per row
  q.jx = q.p ? (q.j0 + 4 == jr + LH ? jr : q.j0 + 4) : (q.j0 == jr ? jr + LH - 1 : q.j0 - 1);
  q.yp = st.yp >> 1;
  q.ym = st.ym >> 1;
  q.zp = st.zp >> 1;
  q.zm = st.zm >> 1;
  return q;
}

// Coupling words of the bonds of the quad's four sites, per direction
// (x+, x-, y+, y-, z+, z-); the z entries are unused in 2D.
struct EaQuadJ {
  uint32_t xp[4], xm[4], yp[4], ym[4], zp[4], zm[4];
};

// J: the group's couplings, [kDim][colour][N/2].  A bond (i, i + e_d) is
// stored at site i, so the + bonds are the quad's own words and the - bonds
// those of the other-colour neighbour.
template <int kDim>
__device__ __forceinline__ EaQuadJ ea_quad_couplings(const uint32_t *__restrict__ J, const EaQuadGeom &q,
                                                     int colour, uint32_t N) {
  const uint32_t half = N >> 1;
  const uint32_t co = (uint32_t)colour * half, ot = ((uint32_t)colour ^ 1u) * half;
  const uint32_t *Jx = J, *Jy = J + N, *Jz = J + 2 * N;
  const uint4 JXo = ldv4(Jx + ot + q.j0);
  const uint32_t JXx = Jx[ot + q.jx];
  const uint4 JXs = ldv4(Jx + co + q.j0), JYs = ldv4(Jy + co + q.j0);
  const uint4 JYm = ldv4(Jy + ot + q.ym);
  const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
  const uint4 JZs = kDim == 3 ? ldv4(Jz + co + q.j0) : zero, JZm = kDim == 3 ? ldv4(Jz + ot + q.zm) : zero;
  const uint32_t jo_[4] = {JXo.x, JXo.y, JXo.z, JXo.w};
  EaQuadJ c;
  c.xp[0] = JXs.x, c.xp[1] = JXs.y, c.xp[2] = JXs.z, c.xp[3] = JXs.w;
  c.yp[0] = JYs.x, c.yp[1] = JYs.y, c.yp[2] = JYs.z, c.yp[3] = JYs.w;
  c.ym[0] = JYm.x, c.ym[1] = JYm.y, c.ym[2] = JYm.z, c.ym[3] = JYm.w;
  c.zp[0] = JZs.x, c.zp[1] = JZs.y, c.zp[2] = JZs.z, c.zp[3] = JZs.w;
  c.zm[0] = JZm.x, c.zm[1] = JZm.y, c.zm[2] = JZm.z, c.zm[3] = JZm.w;
#pragma unroll
  for (int k = 0; k < 4; ++k)
    // p = 0: the site's x - 1 neighbour is other-colour word k - 1; p = 1: word k
    c.xm[k] = q.p ? jo_[k] : (k ? jo_[k - 1] : JXx);
  return c;
}

// Metropolis update of the quad in one word-lattice w (colour-split) with
// shared uniforms r.x .. r.w of its four word-sites.  add(a0, a1, a2)
// receives the post-update count of each site when kCount.
template <int kDim, bool kCount, typename AddFn>
__device__ __forceinline__ void ea_quad_update(uint32_t *__restrict__ w, const EaQuadGeom &q, const EaQuadJ &c,
                                               int colour, uint32_t N, uint4 r, uint32_t t4, uint32_t t8,
                                               uint32_t t12, AddFn add) {
  const uint32_t half = N >> 1;
  uint32_t *own = w + (uint32_t)colour * half;
  const uint32_t *oth = w + ((uint32_t)colour ^ 1u) * half;
  const uint4 O = ldv4(oth + q.j0);
  const uint32_t Ox = oth[q.jx];
  const uint4 S = ldv4(own + q.j0);
  const uint4 YP = ldv4(oth + q.yp), YM = ldv4(oth + q.ym);
  const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
  const uint4 ZP = kDim == 3 ? ldv4(oth + q.zp) : zero, ZM = kDim == 3 ? ldv4(oth + q.zm) : zero;
  const uint32_t s_[4] = {S.x, S.y, S.z, S.w}, o_[4] = {O.x, O.y, O.z, O.w};
  const uint32_t yp_[4] = {YP.x, YP.y, YP.z, YP.w}, ym_[4] = {YM.x, YM.y, YM.z, YM.w};
  const uint32_t zp_[4] = {ZP.x, ZP.y, ZP.z, ZP.w}, zm_[4] = {ZM.x, ZM.y, ZM.z, ZM.w};
  const uint32_t rr[4] = {r.x, r.y, r.z, r.w};
  uint32_t nw[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    // p = 0: x-1 is the other colour at k-1, x+1 at k; p = 1: x-1 at k, x+1 at k+1
    const uint32_t xm = q.p ? o_[k] : (k ? o_[k - 1] : Ox);
    const uint32_t xp = q.p ? (k < 3 ? o_[k + 1] : Ox) : o_[k];
    const uint32_t s0 = s_[k];
    Flip f;
    if (kDim == 3)
      f = ea_flip(s0 ^ xp ^ c.xp[k], s0 ^ xm ^ c.xm[k], s0 ^ yp_[k] ^ c.yp[k], s0 ^ ym_[k] ^ c.ym[k],
                  s0 ^ zp_[k] ^ c.zp[k], s0 ^ zm_[k] ^ c.zm[k], rr[k], t4, t8, t12);
    else
      f = ea_flip2(s0 ^ xp ^ c.xp[k], s0 ^ xm ^ c.xm[k], s0 ^ yp_[k] ^ c.yp[k], s0 ^ ym_[k] ^ c.ym[k], rr[k], t4,
                   t8);
    nw[k] = s0 ^ f.F;
    if (kCount) {
      uint32_t a0, a1, a2;
      if (kDim == 3)
        ea_after(f, a0, a1, a2);
      else
        ea_after2(f, a0, a1, a2);
      add(a0, a1, a2);
    }
  }
  *reinterpret_cast<uint4 *>(own + q.j0) = make_uint4(nw[0], nw[1], nw[2], nw[3]);
}

// Update of the quad j = 4 j4 .. 4 j4 + 3 of colour `colour` in one
// word-lattice w (colour-split) with group couplings J (colour-split).
// Any even L: per-site neighbour indices.  add(a0, a1, a2) receives the
// post-update count of each site when kCount.
template <bool kCount, typename AddFn>
__device__ __forceinline__ void ea_cs_quad(uint32_t *__restrict__ w, const uint32_t *__restrict__ J,
                                           uint32_t j4, int colour, uint32_t L, uint32_t N,
                                           const FastDiv &fL, uint4 r, uint32_t t4, uint32_t t8,
                                           uint32_t t12, AddFn add) {
  const uint32_t half = N >> 1;
  const uint32_t oc = (uint32_t)colour ^ 1u;
  uint32_t *own = w + (uint32_t)colour * half;
  const uint32_t *oth = w + oc * half;
  const uint32_t *Jx = J, *Jy = J + N, *Jz = J + 2 * N;
  const uint32_t co = (uint32_t)colour * half, ot = oc * half;
  if ((L & 7u) == 0) {
    const EaQuadGeom q = ea_quad_geom<3>(j4, colour, L, fL);
    ea_quad_update<3, kCount>(w, q, ea_quad_couplings<3>(J, q, colour, N), colour, N, r, t4, t8, t12, add);
    return;
  }
  const uint32_t rr[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
  for (uint32_t k = 0; k < 4; ++k) {
    const uint32_t j = 4 * j4 + k;
    if (j >= half) break;
    const CsSite st = cs_site(j, colour, L, fL);
    const uint32_t S = own[j];
    const Flip f = ea_flip(S ^ oth[st.xp >> 1] ^ Jx[co + j], S ^ oth[st.xm >> 1] ^ Jx[ot + (st.xm >> 1)],
                           S ^ oth[st.yp >> 1] ^ Jy[co + j], S ^ oth[st.ym >> 1] ^ Jy[ot + (st.ym >> 1)],
                           S ^ oth[st.zp >> 1] ^ Jz[co + j], S ^ oth[st.zm >> 1] ^ Jz[ot + (st.zm >> 1)],
                           rr[k], t4, t8, t12);
    own[j] = S ^ f.F;
    if (kCount) {
      uint32_t a0, a1, a2;
      ea_after(f, a0, a1, a2);
      add(a0, a1, a2);
    }
  }
}

// Update of the quad j = 4 j4 .. 4 j4 + 3 of colour `colour` in one 2D
// word-lattice w with group couplings J ([2][colour][N/2]), as ea_cs_quad.
template <bool kCount, typename AddFn>
__device__ __forceinline__ void ea_cs_quad2(uint32_t *__restrict__ w, const uint32_t *__restrict__ J,
                                            uint32_t j4, int colour, uint32_t L, uint32_t N,
                                            const FastDiv &fL, uint4 r, uint32_t t4, uint32_t t8, AddFn add) {
  const uint32_t half = N >> 1;
  const uint32_t oc = (uint32_t)colour ^ 1u;
  uint32_t *own = w + (uint32_t)colour * half;
  const uint32_t *oth = w + oc * half;
  const uint32_t *Jx = J, *Jy = J + N;
  const uint32_t co = (uint32_t)colour * half, ot = oc * half;
  if ((L & 7u) == 0) {
    const EaQuadGeom q = ea_quad_geom<2>(j4, colour, L, fL);
    ea_quad_update<2, kCount>(w, q, ea_quad_couplings<2>(J, q, colour, N), colour, N, r, t4, t8, 0u, add);
    return;
  }
  const uint32_t rr[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
  for (uint32_t k = 0; k < 4; ++k) {
    const uint32_t j = 4 * j4 + k;
    if (j >= half) break;
    const CsSite st = cs_site2(j, colour, L, fL);
    const uint32_t S = own[j];
    const Flip f = ea_flip2(S ^ oth[st.xp >> 1] ^ Jx[co + j], S ^ oth[st.xm >> 1] ^ Jx[ot + (st.xm >> 1)],
                            S ^ oth[st.yp >> 1] ^ Jy[co + j], S ^ oth[st.ym >> 1] ^ Jy[ot + (st.ym >> 1)], rr[k],
                            t4, t8);
    own[j] = S ^ f.F;
    if (kCount) {
      uint32_t a0, a1, a2;
      ea_after2(f, a0, a1, a2);
      add(a0, a1, a2);
    }
  }
}

}  // namespace spin
