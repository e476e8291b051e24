// +-J Edwards-Anderson glass in 3D (and on the square lattice of the
// paper's own Sec. 5 benchmark) with asynchronous multi-spin coding: bit b
// of a 32-bit word is the spin of realisation 32 g + b at one site, bit set
// <=> s = -1; word-lattices [n_sets][groups][n_temps], each stored
// colour-split (ea_cs.cuh).  Coupling words [groups][dim][colour][N/2], bit
// set <=> J = -1.  The 32 realisations of a word share one
// uniform per site and sweep (the paper's footnote to Sec. 5), so one Philox
// call serves four word-sites.
#include "ea_cs.cuh"
#include "internal.h"

namespace spin {
namespace {

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
    const uint32_t half = (uint32_t)(g.N / 2);
#pragma unroll
    for (uint32_t q = 0; q < 4; ++q) {
      const uint32_t i = (uint32_t)(4 * q4 + q);
      if (i < g.N) out[cs_word(i, colour_of(g, i), half)] = word_of(r, q);
    }
  }
}

__global__ void couplings_msc_kernel(uint32_t *__restrict__ J, Geom g, RoundKeys rk) {
  const int G = g.n_real / 32;
  const int64_t quads = (g.N + 3) / 4;
  const int64_t rows = (int64_t)G * g.dim;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < rows * quads;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t gd = k / quads, q4 = k - gd * quads;
    const int grp = (int)(gd / g.dim), d = (int)(gd % g.dim);
    const uint4 r = philox(make_uint4((uint32_t)q4, 0u, lattice_id(0, grp, 0),
                                      ctr_w(TAG_COUPLING, 0, (uint32_t)d)), rk);
    uint32_t *out = J + gd * g.N;
    const uint32_t half = (uint32_t)(g.N / 2);
#pragma unroll
    for (uint32_t q = 0; q < 4; ++q) {
      const uint32_t i = (uint32_t)(4 * q4 + q);
      if (i < g.N) out[cs_word(i, colour_of(g, i), half)] = word_of(r, q);
    }
  }
}

struct NoAdd {
  __device__ void operator()(uint32_t, uint32_t, uint32_t) const {}
};

// One quad update in kDim dimensions (the group's couplings start at J), any L.
template <int kDim>
__device__ __forceinline__ void ea_quad(uint32_t *w, const uint32_t *J, uint32_t j4, int colour, uint32_t L,
                                        uint32_t N, const FastDiv &fL, uint4 r, uint32_t t4, uint32_t t8,
                                        uint32_t t12) {
  if (kDim == 3)
    ea_cs_quad<false>(w, J, j4, colour, L, N, fL, r, t4, t8, t12, NoAdd());
  else
    ea_cs_quad2<false>(w, J, j4, colour, L, N, fL, r, t4, t8, NoAdd());
}

// Slots per thread of msc_phase_kernel: four when the updates can share the
// quad's geometry and couplings (L % 8 == 0), else one.
__host__ __device__ constexpr uint32_t ea_slots(bool row_quads) { return row_quads ? 4u : 1u; }

// One colour phase over all word-lattices.  Thread k takes one quad of
// colour sites (j4) in the word-lattices (a, grp, t) of kS consecutive
// slots t of one replica set a and group grp, one slot after the other.
// When L % 8 == 0 those updates share the quad's geometry and coupling
// words, read once (ea_cs.cuh); each word-lattice draws its own uniforms,
// so the mapping of updates to threads does not change the result.
// kPair (w = 64, Sec. 5: 64 spins per variable): groups 2q and 2q + 1 of
// one (set, slot) share their uniforms, keyed by q.  kRowQuads: L % 8 == 0
// (else every site takes its own neighbour indices).  ftb divides by the
// number of slot blocks ceil(n_temps / kS).  Register bounds: two CTAs per
// SM for the shared form (its coupling words stay live across the slots),
// three for the generic one.
template <int kDim, bool kPair, bool kRowQuads>
__global__ void __launch_bounds__(256, kRowQuads ? 2 : 3)
    msc_phase_kernel(uint32_t *__restrict__ w, const uint32_t *__restrict__ J, Geom g, uint32_t total,
                     FastDiv ftb, const uint32_t *__restrict__ thr, RoundKeys rk, uint32_t sweep, int colour) {
  griddep_wait();
  griddep_release();
  const uint32_t L = (uint32_t)g.L, N = (uint32_t)g.N, quads = (N / 2 + 3) / 4;
  constexpr uint32_t kS = ea_slots(kRowQuads);
  const uint32_t G = (uint32_t)g.n_real / 32, T = (uint32_t)g.n_temps, TB = (T + kS - 1) / kS;
  const uint32_t wctr = ctr_w(TAG_UPDATE, (uint32_t)colour, 0);
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < total; k += gridDim.x * blockDim.x) {
    const uint32_t sb = fdiv(k, g.fquads), j4 = k - sb * quads;
    const uint32_t st = fdiv(sb, ftb), tb = sb - st * TB;  // sb = (a G + grp) TB + tb
    const uint32_t a = fdiv(st, g.fgrp), grp = st - a * G;
    const uint32_t rkey = kPair ? grp >> 1 : grp;
    uint32_t *ws = w + (size_t)st * T * N;  // slot t of (a, grp) is word-lattice st T + t
    const uint32_t *Jg = J + (size_t)grp * kDim * N;
    const uint32_t t0 = tb * kS, t1 = t0 + kS < T ? t0 + kS : T;
    if (kRowQuads) {
      const EaQuadGeom q = ea_quad_geom<kDim>(j4, colour, L, g.fL);
      const EaQuadJ c = ea_quad_couplings<kDim>(Jg, q, colour, N);
#pragma unroll 1
      for (uint32_t t = t0; t < t1; ++t) {
        const uint4 r = philox(make_uint4(j4, sweep, lattice_id(a, rkey, t), wctr), rk);
        const uint32_t t4 = __ldg(thr + 4 * t + 1), t8 = __ldg(thr + 4 * t + 2);
        const uint32_t t12 = kDim == 3 ? __ldg(thr + 4 * t + 3) : 0u;
        ea_quad_update<kDim, false>(ws + (size_t)t * N, q, c, colour, N, r, t4, t8, t12, NoAdd());
      }
    } else {
      const uint32_t t = t0;  // kS = 1: the slot block is the slot
      const uint4 r = philox(make_uint4(j4, sweep, lattice_id(a, rkey, t), wctr), rk);
      const uint32_t t4 = __ldg(thr + 4 * t + 1), t8 = __ldg(thr + 4 * t + 2);
      const uint32_t t12 = kDim == 3 ? __ldg(thr + 4 * t + 3) : 0u;
      ea_quad<kDim>(ws + (size_t)t * N, Jg, j4, colour, L, N, g.fL, r, t4, t8, t12);
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
    const uint32_t v = w[wl * g.N + cs_word((uint32_t)i, colour_of(g, (uint32_t)i), (uint32_t)(g.N / 2))];
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
    w[wl * g.N + cs_word((uint32_t)i, colour_of(g, (uint32_t)i), (uint32_t)(g.N / 2))] = v;
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
  couplings_msc_kernel<<<capped((int64_t)(g.n_real / 32) * g.dim * g.N / 4 + 1), 256, 0, h->stream>>>(
      (uint32_t *)h->couplings, g, make_round_keys(h->d.seed));
  return cudaGetLastError();
}

cudaError_t launch_sweeps_msc_ea(spin_lattice *h, const uint32_t *J, int64_t n_sweeps) {
  const Geom &g = h->g;
  const RoundKeys rk = make_round_keys(h->d.seed);
  const bool pair = h->msc_width == 64;
  const bool row_quads = g.L % 8 == 0;
  const uint32_t TB = ((uint32_t)g.n_temps + ea_slots(row_quads) - 1) / ea_slots(row_quads);
  const uint32_t work = (uint32_t)g.n_sets * (uint32_t)(g.n_real / 32) * TB * (uint32_t)((g.N / 2 + 3) / 4);
  const FastDiv ftb = make_fastdiv(TB);
  using Kern = decltype(&msc_phase_kernel<3, false, true>);
  const Kern kerns[2][2][2] = {
      {{msc_phase_kernel<2, false, false>, msc_phase_kernel<2, false, true>},
       {msc_phase_kernel<2, true, false>, msc_phase_kernel<2, true, true>}},
      {{msc_phase_kernel<3, false, false>, msc_phase_kernel<3, false, true>},
       {msc_phase_kernel<3, true, false>, msc_phase_kernel<3, true, true>}}};
  const Kern kern = kerns[g.dim == 3][pair][row_quads];
  for (int64_t k = 0; k < n_sweeps; ++k) {
    const uint32_t sweep = (uint32_t)(h->sweeps_done + k);
    for (int colour = 0; colour < 2; ++colour) {
      const cudaError_t e = launch_dependent(kern, dim3(capped(work)), dim3(256), 0, h->stream,
                                             (uint32_t *)h->spins, J, g, work, ftb, (const uint32_t *)h->d_thr,
                                             rk, sweep, colour);
      if (e != cudaSuccess) return e;
    }
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
