// +-J Edwards-Anderson glass in 3D with asynchronous multi-spin coding
// (Sec. 6): bit b of a 32-bit word is the spin of realisation 32 g + b at
// one site, bit set <=> s = -1; words [n_sets][groups][n_temps][L^3].
// Coupling words [groups][3][L^3], bit set <=> J = -1.  The 32 realisations
// of a word share one uniform per site and sweep (the paper's footnote to
// Sec. 6), so one Philox call serves four word-sites.
#include "ea_quad.cuh"
#include "internal.h"

namespace spin {
namespace {

__host__ __device__ inline int64_t word_lattice(const Geom &g, int a, int grp, int t) {
  return ((int64_t)a * (g.n_real / 32) + grp) * g.n_temps + t;
}

__global__ void init_msc_kernel(uint32_t *__restrict__ w, Geom g, RoundKeys rk) {
  const int G = g.n_real / 32;
  const int64_t quads = (g.N + 3) / 4;
  const int64_t n_wl = (int64_t)g.n_sets * G * g.n_temps;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n_wl * quads;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t wl = k / quads, q4 = k - wl * quads;
    const int t = (int)(wl % g.n_temps);
    const int grp = (int)((wl / g.n_temps) % G);
    const int a = (int)(wl / ((int64_t)g.n_temps * G));
    const uint4 r = philox(make_uint4((uint32_t)q4, 0u, lattice_id(a, grp, t), ctr_w(TAG_INIT, 0, 0)), rk);
    uint32_t *out = w + wl * g.N;
#pragma unroll
    for (uint32_t q = 0; q < 4; ++q)
      if (4 * q4 + q < g.N) out[4 * q4 + q] = word_of(r, q);
  }
}

__global__ void couplings_msc_kernel(uint32_t *__restrict__ J, Geom g, RoundKeys rk) {
  const int G = g.n_real / 32;
  const int64_t quads = (g.N + 3) / 4;
  const int64_t rows = (int64_t)G * 3;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < rows * quads;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t gd = k / quads, q4 = k - gd * quads;
    const int grp = (int)(gd / 3), d = (int)(gd % 3);
    const uint4 r = philox(make_uint4((uint32_t)q4, 0u, lattice_id(0, grp, 0),
                                      ctr_w(TAG_COUPLING, 0, (uint32_t)d)), rk);
    uint32_t *out = J + gd * g.N;
#pragma unroll
    for (uint32_t q = 0; q < 4; ++q)
      if (4 * q4 + q < g.N) out[4 * q4 + q] = word_of(r, q);
  }
}

// One colour phase over all word-lattices.  Per word-site: the six bond
// words u_k = s_i ^ s_j ^ J_ij have a 1 where the bond is unsatisfied; a
// bit-sliced adder gives the count u (0..6) per realisation; dE = 12 - 4u;
// the flip mask is (u >= 3) | (u == 2 & R4) | (u == 1 & R8) | (u == 0 & R12)
// with R_dE all ones iff the shared uniform r < thr(dE).
__global__ void __launch_bounds__(256) msc_phase_kernel(uint32_t *__restrict__ w,
                                                        const uint32_t *__restrict__ J, Geom g,
                                                        uint32_t total,
                                                        const uint32_t *__restrict__ thr,
                                                        RoundKeys rk, uint32_t sweep,
                                                        int colour) {
  const uint32_t L = (uint32_t)g.L, LL = L * L, N = (uint32_t)g.N, half = N / 2;
  const uint32_t quads = (half + 3) / 4;
  const uint32_t G = (uint32_t)g.n_real / 32, T = (uint32_t)g.n_temps;
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < total; k += gridDim.x * blockDim.x) {
    const uint32_t wl = fdiv(k, g.fquads), j4 = k - wl * quads;
    const uint32_t t = wl % T;
    const uint32_t grp = (wl / T) % G;
    const uint32_t a = wl / (T * G);
    uint32_t *s = w + (size_t)wl * N;
    const uint32_t *Jg = J + (size_t)grp * 3 * N;
    const uint4 r = philox(make_uint4(j4, sweep, lattice_id(a, grp, t),
                                      ctr_w(TAG_UPDATE, (uint32_t)colour, 0)), rk);
    const uint32_t t4 = __ldg(thr + 4 * t + 1), t8 = __ldg(thr + 4 * t + 2), t12 = __ldg(thr + 4 * t + 3);
#pragma unroll
    for (uint32_t q = 0; q < 4; ++q) {
      const uint32_t j = 4 * j4 + q;
      if (j >= half) break;
      const Site st = site_of(g, j, colour);
      const uint32_t i = st.i;
      const uint32_t ixp = st.rowbase + (st.x == L - 1 ? 0 : st.x + 1);
      const uint32_t ixm = st.rowbase + (st.x == 0 ? L - 1 : st.x - 1);
      const uint32_t iyp = st.y == L - 1 ? i - (L - 1) * L : i + L;
      const uint32_t iym = st.y == 0 ? i + (L - 1) * L : i - L;
      const uint32_t izp = st.z == L - 1 ? i - (L - 1) * LL : i + LL;
      const uint32_t izm = st.z == 0 ? i + (L - 1) * LL : i - LL;
      const uint32_t S = s[i];
      const uint32_t u0 = S ^ s[ixp] ^ Jg[i];
      const uint32_t u1 = S ^ s[ixm] ^ Jg[ixm];
      const uint32_t u2 = S ^ s[iyp] ^ Jg[N + i];
      const uint32_t u3 = S ^ s[iym] ^ Jg[N + iym];
      const uint32_t u4 = S ^ s[izp] ^ Jg[2 * N + i];
      const uint32_t u5 = S ^ s[izm] ^ Jg[2 * N + izm];
      // bit-sliced count of the six unsatisfied-bond indicators
      const uint32_t s1 = u0 ^ u1 ^ u2, c1 = (u0 & u1) | (u2 & (u0 ^ u1));
      const uint32_t s2 = u3 ^ u4 ^ u5, c2 = (u3 & u4) | (u5 & (u3 ^ u4));
      const uint32_t b0 = s1 ^ s2, c3 = s1 & s2;
      const uint32_t b1 = c1 ^ c2 ^ c3, b2 = (c1 & c2) | (c3 & (c1 ^ c2));
      const uint32_t rq = word_of(r, q);
      const uint32_t R4 = rq < t4 ? ~0u : 0u, R8 = rq < t8 ? ~0u : 0u, R12 = rq < t12 ? ~0u : 0u;
      const uint32_t ge3 = b2 | (b1 & b0);
      const uint32_t eq2 = ~b2 & b1 & ~b0, eq1 = ~b2 & ~b1 & b0, eq0 = ~(b2 | b1 | b0);
      const uint32_t flip = ge3 | (eq2 & R4) | (eq1 & R8) | (eq0 & R12);
      s[i] = S ^ flip;
    }
  }
}

// L % 8 == 0: one thread per quad (8-word row segment), quads enumerated
// class by class so that the active parity is uniform across a warp.
struct NoCount {
  template <int K>
  __device__ void operator()(uint32_t (&)[K], uint32_t, uint32_t, uint32_t) const {}
};

__global__ void __launch_bounds__(256) msc_phase_vec_kernel(uint32_t *__restrict__ w,
                                                            const uint32_t *__restrict__ J, Geom g,
                                                            uint32_t total,
                                                            const uint32_t *__restrict__ thr,
                                                            RoundKeys rk, uint32_t sweep,
                                                            int colour) {
  const uint32_t L = (uint32_t)g.L, N = (uint32_t)g.N, quads = N / 8;
  const uint32_t G = (uint32_t)g.n_real / 32, T = (uint32_t)g.n_temps;
  const uint32_t wctr = ctr_w(TAG_UPDATE, (uint32_t)colour, 0);
  uint32_t C[1] = {0};
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < total; k += gridDim.x * blockDim.x) {
    const uint32_t wl = fdiv(k, g.fquads), qk = k - wl * quads;
    const uint32_t t = wl % T, grp = (wl / T) % G, a = wl / (T * G);
    const QuadPos qp = quad_pos(qk, L, g.fqpr, g.fhalfL);
    const uint4 r = philox(make_uint4(qp.i0 >> 3, sweep, lattice_id(a, grp, t), wctr), rk);
    const uint32_t t4 = __ldg(thr + 4 * t + 1), t8 = __ldg(thr + 4 * t + 2), t12 = __ldg(thr + 4 * t + 3);
    uint32_t *s = w + (size_t)wl * N;
    const uint32_t *Jg = J + (size_t)grp * 3 * N;
    if ((colour + qp.cls) & 1)
      ea_quad_update<1, false>(s, Jg, N, L, qp, r, t4, t8, t12, C, NoCount());
    else
      ea_quad_update<0, false>(s, Jg, N, L, qp, r, t4, t8, t12, C, NoCount());
  }
}

// Shared-memory form for small lattices (3 N words of couplings fit): CTA
// (group, set, chunk of kTpc slots) stages the group's couplings once, then
// updates its word-lattices quad by quad.  Couplings are the same for every
// set and slot of a group, so they leave L2 once per CTA instead of once per
// word-lattice.
constexpr int kTpc = 8;

__global__ void __launch_bounds__(256) msc_phase_smem_kernel(uint32_t *__restrict__ w,
                                                             const uint32_t *__restrict__ J, Geom g,
                                                             const uint32_t *__restrict__ thr,
                                                             RoundKeys rk, uint32_t sweep,
                                                             int colour) {
  extern __shared__ __align__(16) uint32_t sJ[];
  const uint32_t L = (uint32_t)g.L, N = (uint32_t)g.N, quads = N / 8;
  const uint32_t G = (uint32_t)g.n_real / 32, T = (uint32_t)g.n_temps;
  const uint32_t chunks = (T + kTpc - 1) / kTpc;
  const uint32_t c = blockIdx.x % chunks, a = (blockIdx.x / chunks) % (uint32_t)g.n_sets;
  const uint32_t grp = blockIdx.x / (chunks * (uint32_t)g.n_sets);
  const uint32_t *Jg = J + (size_t)grp * 3 * N;
  for (uint32_t k = threadIdx.x; k < 3 * N / 4; k += blockDim.x)
    reinterpret_cast<uint4 *>(sJ)[k] = __ldg(reinterpret_cast<const uint4 *>(Jg) + k);
  __syncthreads();
  const uint32_t wctr = ctr_w(TAG_UPDATE, (uint32_t)colour, 0);
  uint32_t C[1] = {0};
  const uint32_t t0 = c * kTpc, t1 = min(T, t0 + kTpc);
  for (uint32_t t = t0; t < t1; ++t) {
    const uint32_t wl = (a * G + grp) * T + t;
    uint32_t *s = w + (size_t)wl * N;
    const uint32_t lid = lattice_id(a, grp, t);
    const uint32_t t4 = __ldg(thr + 4 * t + 1), t8 = __ldg(thr + 4 * t + 2), t12 = __ldg(thr + 4 * t + 3);
    for (uint32_t qk = threadIdx.x; qk < quads; qk += blockDim.x) {
      const QuadPos qp = quad_pos(qk, L, g.fqpr, g.fhalfL);
      const uint4 r = philox(make_uint4(qp.i0 >> 3, sweep, lid, wctr), rk);
      if ((colour + qp.cls) & 1)
        ea_quad_update<1, false>(s, sJ, N, L, qp, r, t4, t8, t12, C, NoCount());
      else
        ea_quad_update<0, false>(s, sJ, N, L, qp, r, t4, t8, t12, C, NoCount());
    }
  }
}

// words -> one int8 per spin, [n_sets][n_temps][n_real][N]
__global__ void unpack_msc_kernel(const uint32_t *__restrict__ w, int8_t *__restrict__ out, Geom g) {
  const int G = g.n_real / 32;
  const int64_t total = (int64_t)g.n_sets * G * g.n_temps * g.N;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t wl = k / g.N, i = k - wl * g.N;
    const int t = (int)(wl % g.n_temps);
    const int grp = (int)((wl / g.n_temps) % G);
    const int a = (int)(wl / ((int64_t)g.n_temps * G));
    const uint32_t v = w[k];
    for (int b = 0; b < 32; ++b) {
      const int64_t lat = ((int64_t)a * g.n_temps + t) * g.n_real + 32 * grp + b;
      out[lat * g.N + i] = ((v >> b) & 1u) ? (int8_t)-1 : (int8_t)1;
    }
  }
}

__global__ void pack_msc_kernel(const int8_t *__restrict__ in, uint32_t *__restrict__ w, Geom g) {
  const int G = g.n_real / 32;
  const int64_t total = (int64_t)g.n_sets * G * g.n_temps * g.N;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t wl = k / g.N, i = k - wl * g.N;
    const int t = (int)(wl % g.n_temps);
    const int grp = (int)((wl / g.n_temps) % G);
    const int a = (int)(wl / ((int64_t)g.n_temps * G));
    uint32_t v = 0;
    for (int b = 0; b < 32; ++b) {
      const int64_t lat = ((int64_t)a * g.n_temps + t) * g.n_real + 32 * grp + b;
      v |= (in[lat * g.N + i] < 0 ? 1u : 0u) << b;
    }
    w[k] = v;
  }
}

unsigned capped(int64_t n) {
  unsigned g = grid_for(n, 256);
  return g > (1u << 20) ? (1u << 20) : g;
}

}  // namespace

cudaError_t launch_init_msc(spin_lattice *h) {
  const Geom &g = h->g;
  const int64_t words = (int64_t)g.n_sets * (g.n_real / 32) * g.n_temps * g.N;
  if (!h->d.hot_start) return cudaMemsetAsync(h->spins, 0, (size_t)words * 4, h->stream);
  init_msc_kernel<<<capped(words / 4 + 1), 256, 0, h->stream>>>((uint32_t *)h->spins, g,
                                                                   make_round_keys(h->d.seed));
  return cudaGetLastError();
}

cudaError_t launch_couplings_msc(spin_lattice *h) {
  const Geom &g = h->g;
  couplings_msc_kernel<<<capped((int64_t)(g.n_real / 32) * 3 * g.N / 4 + 1), 256, 0, h->stream>>>(
      (uint32_t *)h->couplings, g, make_round_keys(h->d.seed));
  return cudaGetLastError();
}

cudaError_t launch_sweeps_msc_ea(spin_lattice *h, const uint32_t *J, int64_t n_sweeps) {
  const Geom &g = h->g;
  const RoundKeys rk = make_round_keys(h->d.seed);
  const int64_t n_wl = (int64_t)g.n_sets * (g.n_real / 32) * g.n_temps;
  const uint32_t work = (uint32_t)(n_wl * ((g.N / 2 + 3) / 4));
  for (int64_t k = 0; k < n_sweeps; ++k) {
    const uint32_t sweep = (uint32_t)(h->sweeps_done + k);
    for (int colour = 0; colour < 2; ++colour) {
      const size_t smem = (size_t)12 * g.N;  // 3 N coupling words
      if (g.L % 8 == 0 && smem <= 96 * 1024) {
        static bool attr = false;
        if (!attr) {
          cudaFuncSetAttribute(msc_phase_smem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
          attr = true;
        }
        const unsigned ctas = (unsigned)((g.n_real / 32) * g.n_sets * ((g.n_temps + kTpc - 1) / kTpc));
        msc_phase_smem_kernel<<<ctas, 256, smem, h->stream>>>((uint32_t *)h->spins, J, g, h->d_thr, rk,
                                                              sweep, colour);
      } else if (g.L % 8 == 0)
        msc_phase_vec_kernel<<<capped(work), 256, 0, h->stream>>>((uint32_t *)h->spins, J, g, work,
                                                                  h->d_thr, rk, sweep, colour);
      else
        msc_phase_kernel<<<capped(work), 256, 0, h->stream>>>((uint32_t *)h->spins, J, g, work,
                                                              h->d_thr, rk, sweep, colour);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_sweeps_msc2d(spin_lattice *h, int64_t n_sweeps);  // msc2d.cu

cudaError_t launch_sweeps_msc(spin_lattice *h, const uint32_t *J, int64_t n_sweeps) {
  if (h->d.model == SPIN_EA) return launch_sweeps_msc_ea(h, J, n_sweeps);
  return launch_sweeps_msc2d(h, n_sweeps);
}

cudaError_t launch_unpack_msc2d(spin_lattice *h, int8_t *out);      // msc2d.cu
cudaError_t launch_pack_msc2d(spin_lattice *h, const int8_t *in);   // msc2d.cu

cudaError_t launch_unpack_msc(spin_lattice *h, int8_t *out) {
  if (h->d.model != SPIN_EA) return launch_unpack_msc2d(h, out);
  const Geom &g = h->g;
  const int64_t words = (int64_t)g.n_sets * (g.n_real / 32) * g.n_temps * g.N;
  unpack_msc_kernel<<<capped(words), 256, 0, h->stream>>>((const uint32_t *)h->spins, out, g);
  return cudaGetLastError();
}

cudaError_t launch_pack_msc(spin_lattice *h, const int8_t *in) {
  if (h->d.model != SPIN_EA) return launch_pack_msc2d(h, in);
  const Geom &g = h->g;
  const int64_t words = (int64_t)g.n_sets * (g.n_real / 32) * g.n_temps * g.N;
  pack_msc_kernel<<<capped(words), 256, 0, h->stream>>>(in, (uint32_t *)h->spins, g);
  return cudaGetLastError();
}

}  // namespace spin
