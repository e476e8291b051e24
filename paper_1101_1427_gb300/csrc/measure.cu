// Reductions (energy, magnetisation, overlap; Sec. 3.5 measurements by
// parallel reduction, double accumulation for continuous spins, Sec. 4)
// and the replica-exchange step (Eq. parallel_tempering, Sec. 6).
#include "bitslice.cuh"
#include "ea_cs.cuh"
#include "heis_reduce.cuh"
#include "internal.h"

namespace spin {

cudaError_t launch_measure_msc2d(spin_lattice *h, int64_t *E, int64_t *M);  // msc2d.cu

namespace {

__device__ __forceinline__ void add_ll(long long *p, long long v) {
  atomicAdd(reinterpret_cast<unsigned long long *>(p), (unsigned long long)v);
}

// ---------------------------------------------------------------- int8 lattices
// E = -sum_{i,d} J_{i,d} s_i s_{i+d}, M = sum_i s_i; integer sums, so the
// atomic accumulation order does not matter.
__global__ void measure_i8_kernel(const int8_t *__restrict__ s, const int8_t *__restrict__ J,
                                  Geom g, long long *__restrict__ E, long long *__restrict__ M) {
  griddep_wait();
  griddep_release();
  const int64_t lat = blockIdx.y;
  const int8_t *sl = s + lat * g.N;
  const int8_t *Jr = J ? J + (lat % g.n_real) * (int64_t)g.dim * g.N : nullptr;
  const int L = g.L;
  const int64_t LL = (int64_t)L * L;
  long long e = 0, m = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % L), y = (int)((i / L) % L), z = g.dim == 3 ? (int)(i / LL) : 0;
    const int si = sl[i];
    const int64_t ixp = i - x + (x == L - 1 ? 0 : x + 1);
    const int64_t iyp = y == L - 1 ? i - (int64_t)(L - 1) * L : i + L;
    int bonds = (Jr ? Jr[i] : 1) * sl[ixp] + (Jr ? Jr[g.N + i] : 1) * sl[iyp];
    if (g.dim == 3) {
      const int64_t izp = z == L - 1 ? i - (int64_t)(L - 1) * LL : i + LL;
      bonds += (Jr ? Jr[2 * g.N + i] : 1) * sl[izp];
    }
    e -= si * bonds;
    m += si;
  }
  e = warp_sum(e);
  m = warp_sum(m);
  if ((threadIdx.x & 31) == 0) {
    if (E) add_ll(&E[lat], e);
    if (M) add_ll(&M[lat], m);
  }
}

// 2D ferromagnet, L % 16 == 0: one thread per 16-byte row segment.  For +-1
// bytes bit 1 is set iff s = -1, so antiparallel bonds to the right and
// downward neighbours are popcounts of (a ^ b) & 0x02..; E = 2 n_anti - 2N,
// M = N - 2 n_down.
__global__ void measure2d_i8_kernel(const int8_t *__restrict__ s, int L, long long *__restrict__ E,
                                    long long *__restrict__ M) {
  griddep_wait();
  griddep_release();
  const int64_t lat = blockIdx.y;
  const int8_t *sl = s + lat * (int64_t)L * L;
  const uint32_t segs = (uint32_t)(L >> 4);
  const uint32_t total = segs * (uint32_t)L;
  const uint64_t B1 = 0x0202020202020202ull;
  long long anti = 0, down = 0;
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < total; k += gridDim.x * blockDim.x) {
    const uint32_t y = k / segs, sg = k - y * segs;
    const int8_t *row = sl + (int64_t)y * L;
    const int8_t *nrow = sl + (int64_t)(y == (uint32_t)L - 1 ? 0 : y + 1) * L;
    const uint4 c = *reinterpret_cast<const uint4 *>(row + 16 * sg);
    const uint4 d = *reinterpret_cast<const uint4 *>(nrow + 16 * sg);
    const uint64_t c0 = (uint64_t)c.x | ((uint64_t)c.y << 32), c1 = (uint64_t)c.z | ((uint64_t)c.w << 32);
    const uint64_t d0 = (uint64_t)d.x | ((uint64_t)d.y << 32), d1 = (uint64_t)d.z | ((uint64_t)d.w << 32);
    const uint64_t nb = (uint8_t)row[sg == segs - 1 ? 0 : 16 * sg + 16];
    const uint64_t r0 = (c0 >> 8) | (c1 << 56), r1 = (c1 >> 8) | (nb << 56);
    anti += __popcll((c0 ^ r0) & B1) + __popcll((c1 ^ r1) & B1) + __popcll((c0 ^ d0) & B1) +
            __popcll((c1 ^ d1) & B1);
    down += __popcll(c0 & B1) + __popcll(c1 & B1);
  }
  anti = warp_sum(anti);
  down = warp_sum(down);
  if ((threadIdx.x & 31) == 0) {
    if (E) add_ll(&E[lat], 2 * anti);
    if (M) add_ll(&M[lat], -2 * down);
  }
}

__global__ void add_per_lattice_kernel(long long *__restrict__ v, int64_t n, long long c) {
  griddep_wait();
  griddep_release();
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    v[k] += c;
}

// q_{t,r} = sum_i s_i^(0) s_i^(1) between sets 0 and 1.
__global__ void overlap_i8_kernel(const int8_t *__restrict__ s, Geom g, long long *__restrict__ Q) {
  griddep_wait();
  griddep_release();
  const int64_t tr = blockIdx.y;  // t * n_real + r
  const int64_t set_stride = (int64_t)g.n_temps * g.n_real * g.N;
  const int8_t *s0 = s + tr * g.N, *s1 = s0 + set_stride;
  long long q = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.N;
       i += (int64_t)gridDim.x * blockDim.x)
    q += s0[i] * s1[i];
  q = warp_sum(q);
  if ((threadIdx.x & 31) == 0) add_ll(&Q[tr], q);
}

// ---------------------------------------------------------------- EA, coded words
// Per word-lattice (a, g, t) and realisation bit b: the number of
// unsatisfied bonds, of down spins and (set 0 only) of spins that differ
// from set 1.  Each thread adds its words into bit-sliced vertical counters
// (plane k holds bit k of 32 per-realisation counts); the counters of a warp
// are added with shuffles, those of the warps through shared memory, and
// lane b of warp 0 finally reads count b out of the planes.
constexpr int kThr = 6;   // per-thread planes: at most 16 sites x 3 bonds = 48 < 64
constexpr int kWarp = 11; // per-warp planes: at most 32 x 48 = 1536 < 2048

// counter += one bit-plane of weight 2^w
template <int K>
__device__ __forceinline__ void vc_add(uint32_t (&C)[K], uint32_t v, int w) {
#pragma unroll
  for (int k = 0; k < K; ++k) {
    if (k < w) continue;
    const uint32_t c = C[k] & v;
    C[k] ^= v;
    v = c;
  }
}

// Sums the per-thread counters of the block; lane b of warp 0 gets count b.
__device__ long long vc_block_total(const uint32_t (&c)[kThr], uint32_t (*sm)[kWarp]) {
  uint32_t C[kWarp];
#pragma unroll
  for (int k = 0; k < kWarp; ++k) C[k] = k < kThr ? c[k] : 0u;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {  // bit-sliced ripple-carry adds across the warp
    uint32_t carry = 0;
#pragma unroll
    for (int k = 0; k < kWarp; ++k) {
      const uint32_t a = C[k], b = __shfl_xor_sync(0xffffffffu, C[k], o);
      C[k] = a ^ b ^ carry;
      carry = (a & b) | (carry & (a ^ b));
    }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < kWarp; ++k) sm[wid][k] = C[k];
  __syncthreads();
  long long tot = 0;
  if (wid == 0) {
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
#pragma unroll
      for (int k = 0; k < kWarp; ++k) tot += (long long)((sm[w][k] >> lane) & 1u) << k;
  }
  __syncthreads();
  return tot;
}

template <int kDim>
__global__ void __launch_bounds__(256) measure_msc_kernel(const uint32_t *__restrict__ w,
                                                          const uint32_t *__restrict__ J, Geom g,
                                                          long long *__restrict__ E,
                                                          long long *__restrict__ M,
                                                          long long *__restrict__ Q) {
  griddep_wait();
  griddep_release();
  __shared__ uint32_t sm[8][kWarp];
  const uint32_t G = (uint32_t)g.n_real / 32, T = (uint32_t)g.n_temps;
  const uint32_t wl = blockIdx.y;
  const uint32_t t = wl % T, grp = (wl / T) % G, a = wl / (T * G);
  const uint32_t L = (uint32_t)g.L, N = (uint32_t)g.N;
  const uint32_t *s = w + (size_t)wl * N;
  const uint32_t *Jg = J + (size_t)grp * kDim * N;
  const bool do_q = Q && a == 0 && g.n_sets >= 2;
  const uint32_t *s1 = s + (size_t)G * T * N;  // set 1, same (g, t)
  uint32_t CE[kThr] = {}, CM[kThr] = {}, CQ[kThr] = {};
  const uint32_t half = N / 2;
  // the bonds (i, i + e_d) of every site count each bond once
  if ((L & 7u) == 0) {
    // four consecutive colour indices of one row per step, 16-byte loads
    const uint32_t quads = half / 4, LH = L / 2;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < 2 * quads; q += gridDim.x * blockDim.x) {
      const int c = q >= quads ? 1 : 0;
      const uint32_t j0 = 4 * (q - (uint32_t)c * quads);
      const uint32_t co = (uint32_t)c * half, oc = (uint32_t)(c ^ 1) * half;
      const CsSite st = kDim == 3 ? cs_site(j0, c, L, g.fL) : cs_site2(j0, c, L, g.fL);
      const uint32_t p = st.i & 1u, jr = st.rb >> 1;
      const uint4 S = ldv4(s + co + j0), O = ldv4(s + oc + j0);
      // x + 1: the other colour at the same index (p = 0) or the next (p = 1)
      const uint32_t jx = j0 + 4 == jr + LH ? jr : j0 + 4;
      const uint32_t Ox = p ? s[oc + jx] : 0u;
      const uint4 YP = ldv4(s + oc + (st.yp >> 1));
      const uint4 ZP = kDim == 3 ? ldv4(s + oc + (st.zp >> 1)) : make_uint4(0, 0, 0, 0);
      const uint4 JX = ldv4(Jg + co + j0), JY = ldv4(Jg + N + co + j0);
      const uint4 JZ = kDim == 3 ? ldv4(Jg + 2 * N + co + j0) : make_uint4(0, 0, 0, 0);
      const uint4 S1 = do_q ? ldv4(s1 + co + j0) : make_uint4(0, 0, 0, 0);
      const uint32_t sv[4] = {S.x, S.y, S.z, S.w}, ov[4] = {O.x, O.y, O.z, O.w};
      const uint32_t yv[4] = {YP.x, YP.y, YP.z, YP.w}, zv[4] = {ZP.x, ZP.y, ZP.z, ZP.w};
      const uint32_t jxv[4] = {JX.x, JX.y, JX.z, JX.w}, jyv[4] = {JY.x, JY.y, JY.z, JY.w};
      const uint32_t jzv[4] = {JZ.x, JZ.y, JZ.z, JZ.w}, s1v[4] = {S1.x, S1.y, S1.z, S1.w};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const uint32_t xp = p ? (k < 3 ? ov[k + 1] : Ox) : ov[k];
        const uint32_t u0 = sv[k] ^ xp ^ jxv[k], u1 = sv[k] ^ yv[k] ^ jyv[k];
        const uint32_t u2 = kDim == 3 ? sv[k] ^ zv[k] ^ jzv[k] : 0u;
        vc_add(CE, u0 ^ u1 ^ u2, 0);
        vc_add(CE, (u0 & u1) | (u2 & (u0 ^ u1)), 1);
        if (M) vc_add(CM, sv[k], 0);
        if (do_q) vc_add(CQ, sv[k] ^ s1v[k], 0);
      }
    }
  } else
  // storage index k: colour c = k / half, colour index j = k % half
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
    const int c = k >= half ? 1 : 0;
    const uint32_t j = k - (uint32_t)c * half;
    const CsSite st = kDim == 3 ? cs_site(j, c, L, g.fL) : cs_site2(j, c, L, g.fL);
    const uint32_t oc = (uint32_t)(c ^ 1) * half;
    const uint32_t S = s[k];
    const uint32_t u0 = S ^ s[oc + (st.xp >> 1)] ^ Jg[k];
    const uint32_t u1 = S ^ s[oc + (st.yp >> 1)] ^ Jg[N + k];
    const uint32_t u2 = kDim == 3 ? S ^ s[oc + (st.zp >> 1)] ^ Jg[2 * N + k] : 0u;
    vc_add(CE, u0 ^ u1 ^ u2, 0);
    vc_add(CE, (u0 & u1) | (u2 & (u0 ^ u1)), 1);
    if (M) vc_add(CM, S, 0);
    if (do_q) vc_add(CQ, S ^ s1[k], 0);
  }
  const uint32_t lane = threadIdx.x & 31;
  const int64_t lat = ((int64_t)a * T + t) * g.n_real + 32 * grp + lane;
  // E = 2 unsat - kDim N, M = N - 2 down, Q = N - 2 diff: block 0 adds the constants
  const long long n0 = blockIdx.x == 0 ? (long long)N : 0;
  // one block per word-lattice stores its counts; several add them to
  // outputs the host has zeroed
  const bool direct = gridDim.x == 1;
  auto put = [direct](long long *p, long long v) {
    if (direct) *p = v;
    else add_ll(p, v);
  };
  const long long unsat = vc_block_total(CE, sm);
  if (threadIdx.x < 32 && E) put(&E[lat], 2 * unsat - kDim * n0);
  if (M) {
    const long long down = vc_block_total(CM, sm);
    if (threadIdx.x < 32) put(&M[lat], n0 - 2 * down);
  }
  if (do_q) {
    const long long diff = vc_block_total(CQ, sm);
    if (threadIdx.x < 32) put(&Q[(int64_t)t * g.n_real + 32 * grp + lane], n0 - 2 * diff);
  }
}


// The same counts when L % 8 == 0, counted with carry-save adders.  Each
// word-lattice gets one block of kRowThreads threads (small blocks, so that
// all of them are resident at once) or, for large lattices, several; a
// thread takes at most kRowItems quads of four consecutive colour indices of
// one row.  Per quad the four unsatisfied-bond sums (weight 1) and carries
// (weight 2) of E, and the four words of M and of Q (weight 1), go through
// carry-save adders into running planes of weight 1, 2, 4 (and 8 for E);
// only what carries out of those is rippled into the counter.  Then one
// butterfly per counter over the warp, and the warps of a word-lattice add
// their counts through shared memory.
constexpr int kRowThreads = 64;
constexpr int kRowItems = 16;
constexpr int kRP = 8;   // per-thread planes: at most 16 quads x 4 sites x 3 bonds = 192 < 256
constexpr int kRW = 13;  // per-warp planes: at most 32 x 192 = 6144 < 8192

// Running count of weight-1 words: planes o1, o2, o4 and the counter above.
struct CsaCount {
  uint32_t C[kRP];
  uint32_t o1, o2, o4;
  __device__ CsaCount() : o1(0), o2(0), o4(0) {
#pragma unroll
    for (int k = 0; k < kRP; ++k) C[k] = 0;
  }
  __device__ __forceinline__ void add4(uint32_t x0, uint32_t x1, uint32_t x2, uint32_t x3) {
    uint32_t t1, t2, f;
    csa(t1, o1, o1, x0, x1);
    csa(t2, o1, o1, x2, x3);
    csa(f, o2, o2, t1, t2);
    const uint32_t e = o4 & f;
    o4 ^= f;
    ripple_at<3>(C, e);
  }
  __device__ __forceinline__ void flush() {
    ripple_at<2>(C, o4);
    ripple_at<1>(C, o2);
    ripple_at<0>(C, o1);
    o1 = o2 = o4 = 0;
  }
};

// The same for four weight-1 words s and four weight-2 words c at a time.
struct CsaCount2 {
  uint32_t C[kRP];
  uint32_t o1, o2, o4, o8;
  __device__ CsaCount2() : o1(0), o2(0), o4(0), o8(0) {
#pragma unroll
    for (int k = 0; k < kRP; ++k) C[k] = 0;
  }
  __device__ __forceinline__ void add(const uint32_t (&sv)[4], const uint32_t (&cv)[4]) {
    uint32_t t1, t2, f1, f2, f3, e1, x;
    csa(t1, o1, o1, sv[0], sv[1]);
    csa(t2, o1, o1, sv[2], sv[3]);
    csa(f1, o2, o2, t1, t2);
    csa(f2, o2, o2, cv[0], cv[1]);
    csa(f3, o2, o2, cv[2], cv[3]);
    csa(e1, o4, o4, f1, f2);
    const uint32_t e2 = o4 & f3;
    o4 ^= f3;
    csa(x, o8, o8, e1, e2);
    ripple_at<4>(C, x);
  }
  __device__ __forceinline__ void flush() {
    ripple_at<3>(C, o8);
    ripple_at<2>(C, o4);
    ripple_at<1>(C, o2);
    ripple_at<0>(C, o1);
    o1 = o2 = o4 = o8 = 0;
  }
};

// Sum of the warp's counters; lane b returns the count of bit b.
__device__ __forceinline__ int warp_count(const uint32_t (&C)[kRP]) {
  uint32_t P[kRW];
#pragma unroll
  for (int k = 0; k < kRW; ++k) P[k] = k < kRP ? C[k] : 0u;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    uint32_t carry = 0;
#pragma unroll
    for (int k = 0; k < kRW; ++k) {
      const uint32_t a = P[k], b = __shfl_xor_sync(0xffffffffu, P[k], o);
      P[k] = a ^ b ^ carry;
      carry = (a & b) | (carry & (a ^ b));
    }
  }
  const int lane = threadIdx.x & 31;
  int cnt = 0;
#pragma unroll
  for (int k = 0; k < kRW; ++k) cnt += (int)((P[k] >> lane) & 1u) << k;
  return cnt;
}

// grid: (blocks per word-lattice, word-lattices), kRowThreads threads; the
// register bound lets 14 blocks share an SM.
template <int kDim>
__global__ void __launch_bounds__(kRowThreads, 14) measure_msc_rows_kernel(const uint32_t *__restrict__ w,
                                                               const uint32_t *__restrict__ J, Geom g,
                                                               long long *__restrict__ E,
                                                               long long *__restrict__ M,
                                                               long long *__restrict__ Q) {
  griddep_wait();
  griddep_release();
  constexpr int kWarps = kRowThreads / 32;
  __shared__ int cnt[3][kWarps][32];
  const uint32_t G = (uint32_t)g.n_real / 32, T = (uint32_t)g.n_temps;
  const uint32_t wl = blockIdx.y, lt = threadIdx.x;
  const uint32_t t = wl % T, grp = (wl / T) % G, a = wl / (T * G);
  const uint32_t L = (uint32_t)g.L, N = (uint32_t)g.N, half = N / 2, quads = half / 4, LH = L / 2;
  const uint32_t *s = w + (size_t)wl * N;
  const uint32_t *Jg = J + (size_t)grp * kDim * N;
  const bool do_q = Q && a == 0 && g.n_sets >= 2;
  const uint32_t *s1 = s + (size_t)G * T * N;  // set 1, same (g, t)
  CsaCount2 ce;
  CsaCount cm, cq;
  for (uint32_t q = blockIdx.x * kRowThreads + lt; q < 2 * quads; q += gridDim.x * kRowThreads) {
      const uint32_t c = q >= quads ? 1u : 0u;
      const uint32_t j0 = 4 * (q - c * quads);
      const uint32_t co = c * half, oc = (c ^ 1u) * half;
      const CsSite st = kDim == 3 ? cs_site(j0, (int)c, L, g.fL) : cs_site2(j0, (int)c, L, g.fL);
      const uint32_t p = st.i & 1u, jr = st.rb >> 1;
      const uint4 S = ldv4(s + co + j0), O = ldv4(s + oc + j0);
      // x + 1: the other colour at the same index (p = 0) or the next (p = 1)
      const uint32_t jx = j0 + 4 == jr + LH ? jr : j0 + 4;
      const uint32_t Ox = p ? s[oc + jx] : 0u;
      const uint4 YP = ldv4(s + oc + (st.yp >> 1));
      const uint4 ZP = kDim == 3 ? ldv4(s + oc + (st.zp >> 1)) : make_uint4(0, 0, 0, 0);
      const uint4 JX = ldv4(Jg + co + j0), JY = ldv4(Jg + N + co + j0);
      const uint4 JZ = kDim == 3 ? ldv4(Jg + 2 * N + co + j0) : make_uint4(0, 0, 0, 0);
      const uint32_t sv[4] = {S.x, S.y, S.z, S.w}, ov[4] = {O.x, O.y, O.z, O.w};
      const uint32_t yv[4] = {YP.x, YP.y, YP.z, YP.w}, zv[4] = {ZP.x, ZP.y, ZP.z, ZP.w};
      const uint32_t jxv[4] = {JX.x, JX.y, JX.z, JX.w}, jyv[4] = {JY.x, JY.y, JY.z, JY.w};
      const uint32_t jzv[4] = {JZ.x, JZ.y, JZ.z, JZ.w};
      // the bonds (i, i + e_d) of every site count each bond once
      uint32_t sum[4], car[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const uint32_t xp = p ? (k < 3 ? ov[k + 1] : Ox) : ov[k];
        const uint32_t u0 = sv[k] ^ xp ^ jxv[k], u1 = sv[k] ^ yv[k] ^ jyv[k];
        const uint32_t u2 = kDim == 3 ? sv[k] ^ zv[k] ^ jzv[k] : 0u;
        sum[k] = u0 ^ u1 ^ u2;
        car[k] = (u0 & u1) | (u2 & (u0 ^ u1));
      }
      ce.add(sum, car);
      if (M) cm.add4(sv[0], sv[1], sv[2], sv[3]);
      if (do_q) {
        const uint4 S1 = ldv4(s1 + co + j0);
        cq.add4(S.x ^ S1.x, S.y ^ S1.y, S.z ^ S1.z, S.w ^ S1.w);
      }
    }
  ce.flush();
  cm.flush();
  cq.flush();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  cnt[0][warp][lane] = warp_count(ce.C);
  if (M) cnt[1][warp][lane] = warp_count(cm.C);
  if (Q) cnt[2][warp][lane] = warp_count(cq.C);
  __syncthreads();
  if (warp != 0) return;
  // lane b of warp 0 adds the warps' counts of bit b
  long long e = 0, m = 0, d = 0;
#pragma unroll
  for (int k = 0; k < kWarps; ++k) {
    e += cnt[0][k][lane];
    if (M) m += cnt[1][k][lane];
    if (do_q) d += cnt[2][k][lane];
  }
  const int64_t lat = ((int64_t)a * T + t) * g.n_real + 32 * grp + lane;
  // E = 2 unsat - kDim N, M = N - 2 down, Q = N - 2 diff: part 0 adds the
  // constants; with one part per word-lattice the counts are stored
  const long long n0 = blockIdx.x == 0 ? (long long)N : 0;
  const bool direct = gridDim.x == 1;
  auto put = [direct](long long *ptr, long long v) {
    if (direct) *ptr = v;
    else add_ll(ptr, v);
  };
  if (E) put(&E[lat], 2 * e - kDim * n0);
  if (M) put(&M[lat], n0 - 2 * m);
  if (do_q) put(&Q[(int64_t)t * g.n_real + 32 * grp + lane], n0 - 2 * d);
}

// ---------------------------------------------------------------- Heisenberg
// Per-block partial sums in double, then a fixed-order second pass, so the
// result does not depend on scheduling.
constexpr int kHeisBlocks = 64;

__global__ void measure_heis_kernel(const float4 *__restrict__ s, Geom g,
                                    double *__restrict__ partial) {
  griddep_wait();
  griddep_release();
  const int64_t lat = blockIdx.y;
  heis_block_partials(s + lat * g.N, g.L, g.dim, g.N, blockIdx.x, gridDim.x,
                      partial + (lat * gridDim.x + blockIdx.x) * 4);
}

__global__ void finish_heis_kernel(const double *__restrict__ partial, int64_t n_lat, int nb,
                                   double *__restrict__ Ef, double *__restrict__ Mf) {
  griddep_wait();
  griddep_release();
  const int64_t lat = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (lat >= n_lat) return;
  heis_finish_lattice(partial, nb, lat, Ef, Mf);
}

// ---------------------------------------------------------------- replica exchange
// Thread per (set a, realisation r, pair t) of the step's parity.
// Delta = dbeta_t (E_{t+1} - E_t); accept iff Delta >= 0 or the PT word of
// (a, t, step, r) is below the tabulated threshold of exp(Delta).
__global__ void pt_decide_kernel(const long long *__restrict__ E, Geom g,
                                 const double *__restrict__ dbeta,
                                 const uint32_t *__restrict__ tab, const int32_t *__restrict__ off,
                                 const int32_t *__restrict__ len, RoundKeys rk, uint32_t step,
                                 uint8_t *__restrict__ decision, long long *__restrict__ accepted,
                                 int *__restrict__ labels) {
  griddep_wait();
  griddep_release();
  const int parity = (int)(step & 1u);
  const int n_pairs = (g.n_temps - parity) / 2;  // pairs (t, t+1), t = parity + 2k
  const int64_t total = (int64_t)g.n_sets * n_pairs * g.n_real;
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= total) return;
  const int r = (int)(k % g.n_real);
  const int pk = (int)((k / g.n_real) % n_pairs);
  const int a = (int)(k / ((int64_t)g.n_real * n_pairs));
  const int t = parity + 2 * pk;
  const int64_t lat0 = ((int64_t)a * g.n_temps + t) * g.n_real + r;
  const int64_t lat1 = lat0 + g.n_real;
  const long long dE = E[lat1] - E[lat0];
  const double db = dbeta[t];
  bool acc;
  if (db * (double)dE >= 0.0) {
    acc = true;
  } else {
    const long long m = (dE < 0 ? -dE : dE) / 4;
    const uint32_t thr = m < len[t] ? tab[off[t] + m] : 0u;
    const uint4 w = philox(make_uint4((uint32_t)r >> 2, step, lattice_id(a, 0, t), ctr_w(TAG_PT, 0, 0)), rk);
    acc = word_of(w, (uint32_t)r & 3u) < thr;
  }
  decision[lat0] = acc ? 1 : 0;
  if (labels && acc) {  // one thread per pair: no other thread touches these two
    const int l0 = labels[lat0];
    labels[lat0] = labels[lat1];
    labels[lat1] = l0;
  }
  if (!accepted) return;
  if ((g.n_real & 31) == 0) {
    // the 32 lanes of a warp share (a, t): one atomic per warp
    const uint32_t votes = __ballot_sync(0xffffffffu, acc);
    if ((threadIdx.x & 31) == 0 && votes) add_ll(&accepted[a * g.n_temps + t], __popc(votes));
  } else if (acc) {
    add_ll(&accepted[a * g.n_temps + t], 1);
  }
}

// Exchange of whole lattices (int8, or coded 2D lattices): 16 bytes per
// thread step when the lattice size is a multiple of 16 bytes (the spins
// buffer is 16-byte aligned, so every lattice then is), single bytes
// otherwise (e.g. 6^3 = 216-byte int8 lattices).
__global__ void pt_swap_bytes_kernel(uint8_t *__restrict__ s, const uint8_t *__restrict__ decision,
                                     Geom g, int parity, int64_t lat_bytes) {
  griddep_wait();
  griddep_release();
  const int64_t lat0 = blockIdx.y;
  const int t = (int)slot_of32(g, (uint32_t)lat0);
  if (((t - parity) & 1) || t + 1 >= g.n_temps || !decision[lat0]) return;
  uint8_t *b0 = s + lat0 * lat_bytes, *b1 = s + (lat0 + g.n_real) * lat_bytes;
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  if ((lat_bytes & 15) == 0) {
    uint4 *p0 = reinterpret_cast<uint4 *>(b0), *p1 = reinterpret_cast<uint4 *>(b1);
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < lat_bytes / 16; k += step) {
      const uint4 a = p0[k], b = p1[k];
      p0[k] = b;
      p1[k] = a;
    }
  } else {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < lat_bytes; k += step) {
      const uint8_t a = b0[k], b = b1[k];
      b0[k] = b;
      b1[k] = a;
    }
  }
}

// Bitwise exchange of coded EA words: per (a, g, pair) the accepted
// realisations form a mask A (one warp ballot over their decisions);
// x = (w_t ^ w_{t+1}) & A exchanges those bits, 16 bytes at a time (N is a
// multiple of 8 and every word-lattice starts 32-byte aligned).
__global__ void pt_swap_msc_kernel(uint32_t *__restrict__ w, const uint8_t *__restrict__ decision,
                                   Geom g, int parity) {
  griddep_wait();
  griddep_release();
  const int G = g.n_real / 32;
  const int64_t wl = blockIdx.y;  // (a, grp, t)
  const int t = (int)(wl % g.n_temps);
  if (((t - parity) & 1) || t + 1 >= g.n_temps) return;
  const int grp = (int)((wl / g.n_temps) % G);
  const int a = (int)(wl / ((int64_t)g.n_temps * G));
  const int64_t lat0 = ((int64_t)a * g.n_temps + t) * g.n_real + 32 * grp;
  const uint32_t mask = __ballot_sync(0xffffffffu, decision[lat0 + (threadIdx.x & 31)] != 0);
  if (!mask) return;
  uint4 *w0 = reinterpret_cast<uint4 *>(w + wl * g.N), *w1 = reinterpret_cast<uint4 *>(w + (wl + 1) * g.N);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.N / 4;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint4 a0 = w0[i], a1 = w1[i];
    const uint4 x = make_uint4((a0.x ^ a1.x) & mask, (a0.y ^ a1.y) & mask, (a0.z ^ a1.z) & mask,
                               (a0.w ^ a1.w) & mask);
    w0[i] = make_uint4(a0.x ^ x.x, a0.y ^ x.y, a0.z ^ x.z, a0.w ^ x.w);
    w1[i] = make_uint4(a1.x ^ x.x, a1.y ^ x.y, a1.z ^ x.z, a1.w ^ x.w);
  }
}

unsigned capped(int64_t n, unsigned cap) {
  unsigned g = grid_for(n, 256);
  return g > cap ? cap : g;
}

}  // namespace

cudaError_t launch_measure(spin_lattice *h, const void *J, int64_t *E, int64_t *M, int64_t *Q,
                           double *Ef, double *Mf) {
  const Geom &g = h->g;
  cudaStream_t st = h->stream;
  const int64_t nl = h->n_lat;
  if (h->d.model == SPIN_HEISENBERG) {
    if (!Ef && !Mf) return cudaSuccess;
    double *partial = (double *)h->d_scratch64;
    cudaError_t e = launch_dependent(measure_heis_kernel, dim3(kHeisBlocks, (unsigned)nl), dim3(256), 0, st,
                                     (const float4 *)h->spins, g, partial);
    if (e != cudaSuccess) return e;
    return launch_dependent(finish_heis_kernel, dim3(grid_for(nl, 128)), dim3(128), 0, st,
                            (const double *)partial, nl, kHeisBlocks, Ef, Mf);
  }
  if (h->d.layout == SPIN_MSC1 && h->d.model == SPIN_ISING) {
    if (Q) cudaMemsetAsync(Q, 0, sizeof(int64_t) * g.n_temps * g.n_real, st);
    return launch_measure_msc2d(h, E, M);
  }
  // EA coded words: blocks (or, with L % 8 == 0, parts of kRowThreads
  // threads) per word-lattice, at most 16 sites (quads) per thread; with one
  // per word-lattice the counts are stored, not added, and need no zeroing
  const bool rows = h->d.layout == SPIN_MSC1 && g.L % 8 == 0;
  const int64_t row_items = 2 * (g.N / 8);  // quads of both colours
  const unsigned gx = rows ? (unsigned)((row_items + kRowThreads * kRowItems - 1) / (kRowThreads * kRowItems))
                           : (unsigned)((g.N + 256 * 16 - 1) / (256 * 16));
  const bool coded_direct = h->d.layout == SPIN_MSC1 && gx == 1;
  if (!coded_direct) {
    if (E) cudaMemsetAsync(E, 0, sizeof(int64_t) * nl, st);
    if (M) cudaMemsetAsync(M, 0, sizeof(int64_t) * nl, st);
    if (Q) cudaMemsetAsync(Q, 0, sizeof(int64_t) * g.n_temps * g.n_real, st);
  }
  cudaError_t e = cudaSuccess;
  if (h->d.layout == SPIN_I8) {
    if ((E || M) && !J && g.dim == 2 && g.L % 16 == 0) {
      const int64_t segs = (int64_t)g.L * (g.L / 16);
      e = launch_dependent(measure2d_i8_kernel, dim3(capped(segs, 2048), (unsigned)nl), dim3(256), 0, st,
                           (const int8_t *)h->spins, g.L, (long long *)E, (long long *)M);
      if (e == cudaSuccess && E)
        e = launch_dependent(add_per_lattice_kernel, dim3(capped(nl, 4096)), dim3(256), 0, st, (long long *)E, nl,
                             -2 * (long long)g.N);
      if (e == cudaSuccess && M)
        e = launch_dependent(add_per_lattice_kernel, dim3(capped(nl, 4096)), dim3(256), 0, st, (long long *)M, nl,
                             (long long)g.N);
    } else if (E || M) {
      e = launch_dependent(measure_i8_kernel, dim3(capped(g.N, 1024), (unsigned)nl), dim3(256), 0, st,
                           (const int8_t *)h->spins, (const int8_t *)J, g, (long long *)E, (long long *)M);
    }
    if (e == cudaSuccess && Q && g.n_sets >= 2)
      e = launch_dependent(overlap_i8_kernel, dim3(capped(g.N, 1024), (unsigned)(g.n_temps * g.n_real)),
                           dim3(256), 0, st, (const int8_t *)h->spins, g, (long long *)Q);
    return e;
  }
  const int64_t n_wl = (int64_t)g.n_sets * (g.n_real / 32) * g.n_temps;
  if (rows)
    return launch_dependent(g.dim == 3 ? measure_msc_rows_kernel<3> : measure_msc_rows_kernel<2>,
                            dim3(gx, (unsigned)n_wl), dim3(kRowThreads), 0, st,
                            (const uint32_t *)h->spins, (const uint32_t *)J, g, (long long *)E, (long long *)M,
                            (g.n_sets >= 2) ? (long long *)Q : nullptr);
  return launch_dependent(g.dim == 3 ? measure_msc_kernel<3> : measure_msc_kernel<2>, dim3(gx, (unsigned)n_wl),
                          dim3(256), 0, st, (const uint32_t *)h->spins,
                          (const uint32_t *)J, g, (long long *)E, (long long *)M,
                          (g.n_sets >= 2) ? (long long *)Q : nullptr);
}

cudaError_t launch_pt_swap(spin_lattice *h, const void *J, int64_t *accepted, int32_t *labels,
                           const int64_t *energies) {
  const Geom &g = h->g;
  cudaStream_t st = h->stream;
  if (!energies) {
    cudaError_t e = launch_measure(h, J, h->d_energy, nullptr, nullptr, nullptr, nullptr);
    if (e != cudaSuccess) return e;
    energies = h->d_energy;
  }
  const uint32_t step = (uint32_t)h->pt_steps_done;
  const int parity = (int)(step & 1u);
  const int n_pairs = (g.n_temps - parity) / 2;
  uint8_t *decision = (uint8_t *)(h->d_energy + 2 * h->n_lat);
  if (n_pairs <= 0) return cudaSuccess;
  const int64_t total = (int64_t)g.n_sets * n_pairs * g.n_real;
  cudaError_t e = launch_dependent(pt_decide_kernel, dim3(grid_for(total, 256)), dim3(256), 0, st,
                                   (const long long *)energies, g, (const double *)h->d_pt_dbeta,
                                   (const uint32_t *)h->d_pt_thr, (const int32_t *)h->d_pt_off,
                                   (const int32_t *)h->d_pt_len, make_round_keys(h->d.seed), step, decision,
                                   (long long *)accepted, (int *)labels);
  if (e != cudaSuccess) return e;
  if (h->d.layout == SPIN_MSC1 && h->d.model == SPIN_EA) {
    const int64_t n_wl = (int64_t)g.n_sets * (g.n_real / 32) * g.n_temps;
    return launch_dependent(pt_swap_msc_kernel, dim3(capped(g.N / 4, 64), (unsigned)n_wl), dim3(256), 0, st,
                            (uint32_t *)h->spins, (const uint8_t *)decision, g, parity);
  } else {
    int64_t lat_bytes = g.N;  // int8
    if (h->d.layout == SPIN_MSC1) lat_bytes = g.N / 8;
    if (h->d.layout == SPIN_F32X4) lat_bytes = g.N * 16;
    const int64_t units = (lat_bytes & 15) == 0 ? lat_bytes / 16 : lat_bytes;
    return launch_dependent(pt_swap_bytes_kernel, dim3(capped(units, 1024), (unsigned)h->n_lat), dim3(256), 0, st,
                            (uint8_t *)h->spins, (const uint8_t *)decision, g, parity, lat_bytes);
  }
  return cudaGetLastError();
}

}  // namespace spin
