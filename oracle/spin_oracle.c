/*
 * spin_oracle.c -- plain, serial CPU oracle for the checkerboard Metropolis
 * sweep, the measurements and the replica-exchange step of
 * M. Weigel, "Performance potential for simulating spin models on GPU"
 * (arXiv:1101.1427).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library may include,
 * link or call this file; only the tests, the package smoke check and the
 * benchmark's CPU-baseline leg use it.  It shares no code with the CUDA
 * path: its own Philox, its own threshold tables, its own loops.
 *
 * Everything is written for readability, not speed: one int8 per Ising
 * spin, three doubles per Heisenberg spin, one full Philox call per random
 * word that is used, sites visited in plain linear order.
 *
 * Conventions fixed here (the paper leaves them open; the CUDA path
 * implements the same conventions independently):
 *   - lattice: L^dim sites, x fastest, periodic boundaries, L even;
 *     site i <-> (x, y, z) with i = (z*L + y)*L + x.
 *   - colour c(i) = (x + y + z) mod 2; colour 0 is updated first
 *     (Sec. 3.2, the "even" sub-lattice).
 *   - j(i) = i >> 1 is the index of site i inside its colour sub-lattice.
 *   - a random word is word (idx & 3) of Philox4x32-10 applied to
 *       counter = (idx >> 2, sweep, lattice_id, tag << 28 | colour << 27 | extra)
 *       key     = (seed & 0xffffffff, seed >> 32).
 *   - Metropolis acceptance (Eq. metropolis) with the integer threshold
 *       thr(dE) = min(2^32 - 1, floor(exp(-beta*dE) * 2^32)):
 *       flip iff dE <= 0 or r < thr(dE).
 */
#define _DEFAULT_SOURCE
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* Random numbers: Philox4x32-10, from its published definition        */
/* (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as   */
/* 1, 2, 3", SC'11).  The paper only requires independent, reproducible */
/* per-thread streams whose result does not depend on thread order      */
/* (Sec. 3.3); a counter-based generator meets that by construction.    */
/* ------------------------------------------------------------------ */

enum {
  OR_TAG_UPDATE = 0,    /* Ising / EA Metropolis uniform, one word per site   */
  OR_TAG_INIT = 1,      /* Ising / EA hot start, one word per site            */
  OR_TAG_COUPLING = 2,  /* EA +-J couplings, one word per (group, dir, site)  */
  OR_TAG_PT = 3,        /* replica-exchange uniform, one word per realisation */
  OR_TAG_HEIS = 4,      /* Heisenberg update, one whole call per site         */
  OR_TAG_HEIS_INIT = 5  /* Heisenberg hot start, one whole call per site      */
};

void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                      uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;  /* round multipliers */
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;  /* Weyl key bumps    */
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += W0;
      k1 += W1;
    }
    uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* One whole Philox call for the counter layout above (word index w). */
static void or_call(uint64_t seed, uint32_t tag, uint32_t colour, uint32_t extra,
                    uint32_t lattice_id, uint32_t sweep, uint32_t x,
                    uint32_t out[4]) {
  uint32_t ctr[4] = {x, sweep, lattice_id, (tag << 28) | (colour << 27) | extra};
  uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  or_philox4x32_10(ctr, key, out);
}

/* The random word for index idx: word (idx & 3) of the call for idx >> 2. */
uint32_t or_draw(uint64_t seed, uint32_t tag, uint32_t colour, uint32_t extra,
                 uint32_t lattice_id, uint32_t sweep, uint32_t idx) {
  uint32_t out[4];
  or_call(seed, tag, colour, extra, lattice_id, sweep, idx >> 2, out);
  return out[idx & 3];
}

/* 24-bit uniform in [0,1): exactly representable in float and double. */
static double or_uniform(uint32_t x) { return (double)(x >> 8) * (1.0 / 16777216.0); }

/* Lattice identifiers: (replica set a, realisation key, temperature slot t).
 * The realisation key is the realisation r for Ising / Heisenberg lattices
 * and the group r >> 5 for EA lattices (the 32 realisations of a group
 * share one uniform per site, Sec. 5, asynchronous multi-spin coding). */
uint32_t or_lattice_id(uint32_t a, uint32_t rkey, uint32_t t) {
  return (a << 24) | (rkey << 12) | t;
}

/* ------------------------------------------------------------------ */
/* Acceptance thresholds (Eq. metropolis, Eq. parallel_tempering)      */
/* ------------------------------------------------------------------ */

/* floor(p * 2^32) capped at 2^32 - 1, for a probability p in [0, 1]. */
static uint32_t or_prob_to_threshold(double p) {
  double t = floor(p * 4294967296.0);
  if (t >= 4294967295.0) return 0xFFFFFFFFu;
  if (t <= 0.0) return 0u;
  return (uint32_t)t;
}

/* Metropolis threshold for an energy increase dE > 0 at inverse temperature
 * beta: P(r < thr) = thr / 2^32 ~ exp(-beta dE)  (Eq. metropolis). */
uint32_t or_metropolis_threshold(double beta, int dE) {
  return or_prob_to_threshold(exp(-beta * (double)dE));
}

/* Replica-exchange threshold for exponent -|dbeta| * 4m (Eq. parallel_tempering
 * with |Delta beta Delta E| = |dbeta| * 4m, energy differences being
 * multiples of 4 on these lattices). */
uint32_t or_pt_threshold(double abs_dbeta, int64_t m) {
  return or_prob_to_threshold(exp(-abs_dbeta * (double)(4 * m)));
}

/* ------------------------------------------------------------------ */
/* Lattice geometry                                                     */
/* ------------------------------------------------------------------ */

static int64_t or_nsites(int dim, int L) {
  int64_t n = 1;
  for (int d = 0; d < dim; ++d) n *= L;
  return n;
}

static void or_coords(int dim, int L, int64_t i, int c[3]) {
  c[0] = (int)(i % L);
  c[1] = dim > 1 ? (int)((i / L) % L) : 0;
  c[2] = dim > 2 ? (int)(i / ((int64_t)L * L)) : 0;
}

static int64_t or_index(int dim, int L, const int c[3]) {
  int64_t i = c[0];
  if (dim > 1) i += (int64_t)L * c[1];
  if (dim > 2) i += (int64_t)L * L * c[2];
  return i;
}

/* Neighbour of site i in direction d (0..dim-1), step +1 or -1, periodic. */
static int64_t or_neighbour(int dim, int L, int64_t i, int d, int step) {
  int c[3];
  or_coords(dim, L, i, c);
  c[d] = (c[d] + step + L) % L;
  return or_index(dim, L, c);
}

int or_colour(int dim, int L, int64_t i) {
  int c[3];
  or_coords(dim, L, i, c);
  return (c[0] + c[1] + c[2]) & 1;
}

/* ------------------------------------------------------------------ */
/* Ising ferromagnet / +-J Edwards-Anderson glass, one int8 per spin    */
/* ------------------------------------------------------------------ */

/* Hot start: s_i = -1 if bit `bit` of the INIT word of site i is set,
 * else +1.  Cold start (hot == 0): all +1. */
void or_ising_init(int dim, int L, int8_t *s, uint64_t seed, uint32_t lattice_id,
                   int bit, int hot) {
  int64_t n = or_nsites(dim, L);
  for (int64_t i = 0; i < n; ++i) {
    if (!hot) {
      s[i] = 1;
      continue;
    }
    uint32_t w = or_draw(seed, OR_TAG_INIT, 0, 0, lattice_id, 0, (uint32_t)i);
    s[i] = ((w >> bit) & 1u) ? -1 : 1;
  }
}

/* Bimodal couplings P(J) = (delta(J-1) + delta(J+1))/2 (Eq.
 * spinglass_hamiltonian).  J[d*N + i] is the coupling of the bond between
 * site i and its +d neighbour, for realisation r: bit (r & 31) of the
 * COUPLING word of (group r >> 5, direction d, site i); set means J = -1.
 * Couplings are quenched: the same for every replica set and slot. */
void or_ea_couplings(int dim, int L, int r, int8_t *J, uint64_t seed) {
  int64_t n = or_nsites(dim, L);
  uint32_t lid = or_lattice_id(0, (uint32_t)(r >> 5), 0);
  for (int d = 0; d < dim; ++d)
    for (int64_t i = 0; i < n; ++i) {
      uint32_t w = or_draw(seed, OR_TAG_COUPLING, 0, (uint32_t)d, lid, 0, (uint32_t)i);
      J[d * n + i] = ((w >> (r & 31)) & 1u) ? -1 : 1;
    }
}

/* Local field h_i = sum over neighbours of J_ij s_j (J == NULL: J = 1). */
static int or_local_field(int dim, int L, const int8_t *s, const int8_t *J,
                          int64_t i) {
  int64_t n = or_nsites(dim, L);
  int h = 0;
  for (int d = 0; d < dim; ++d) {
    int64_t up = or_neighbour(dim, L, i, d, +1);
    int64_t dn = or_neighbour(dim, L, i, d, -1);
    int j_up = J ? J[d * n + i] : 1;
    int j_dn = J ? J[d * n + dn] : 1;
    h += j_up * s[up] + j_dn * s[dn];
  }
  return h;
}

/* One checkerboard sweep (Sec. 3.2): all colour-0 sites, then all colour-1
 * sites; each site is updated with the Metropolis rule (Eq. metropolis),
 * dE = 2 s_i h_i, using its UPDATE word (colour c, index j = i >> 1).
 * Optional `flips` accumulates the number of accepted flips. */
void or_ising_sweep(int dim, int L, int8_t *s, const int8_t *J, double beta,
                    uint64_t seed, uint32_t lattice_id, uint32_t sweep,
                    int64_t *flips) {
  int64_t n = or_nsites(dim, L);
  uint32_t thr[4] = {0, 0, 0, 0};
  for (int m = 1; m <= dim; ++m) thr[m] = or_metropolis_threshold(beta, 4 * m);
  for (int colour = 0; colour < 2; ++colour) {
    for (int64_t i = 0; i < n; ++i) {
      if (or_colour(dim, L, i) != colour) continue;
      int h = or_local_field(dim, L, s, J, i);
      int dE = 2 * s[i] * h;
      int flip;
      if (dE <= 0) {
        flip = 1;
      } else {
        uint32_t r = or_draw(seed, OR_TAG_UPDATE, (uint32_t)colour, 0, lattice_id,
                             sweep, (uint32_t)(i >> 1));
        flip = r < thr[dE / 4];
      }
      if (flip) {
        s[i] = (int8_t)(-s[i]);
        if (flips) ++*flips;
      }
    }
  }
}

/* One colour phase of rows y0 .. y0 + rows - 1 (0 <= y0, y0 + rows <= L) of
 * a 2D L x L periodic ferromagnet held as a slab of rows + 2 rows of L
 * sites: slab row 0 holds a copy of row y0 - 1 and slab row rows + 1 a copy
 * of row y0 + rows (both mod L), rows 1 .. rows are the slab's own rows.
 * Every own site of the colour is updated as in or_ising_sweep: the colour
 * and the random word are those of its global index y L + x, so slabs that
 * exchange their boundary rows before every phase reproduce the unsplit
 * sweep.  The copies are only read. */
void or_ising_slab_phase(int L, int y0, int rows, int8_t *slab, double beta, uint64_t seed,
                         uint32_t lattice_id, uint32_t sweep, int colour, int64_t *flips) {
  uint32_t thr[3] = {0, 0, 0};
  for (int m = 1; m <= 2; ++m) thr[m] = or_metropolis_threshold(beta, 4 * m);
  for (int r = 1; r <= rows; ++r) {
    const int64_t y = y0 + r - 1;
    int8_t *row = slab + (int64_t)r * L;
    const int8_t *up = row - L, *dn = row + L;
    for (int x = 0; x < L; ++x) {
      if ((int)((x + y) & 1) != colour) continue;
      const int h = row[x == L - 1 ? 0 : x + 1] + row[x == 0 ? L - 1 : x - 1] + up[x] + dn[x];
      const int dE = 2 * row[x] * h;
      int flip;
      if (dE <= 0) {
        flip = 1;
      } else {
        const uint32_t rw = or_draw(seed, OR_TAG_UPDATE, (uint32_t)colour, 0, lattice_id, sweep,
                                    (uint32_t)((y * L + x) >> 1));
        flip = rw < thr[dE / 4];
      }
      if (flip) {
        row[x] = (int8_t)(-row[x]);
        if (flips) ++*flips;
      }
    }
  }
}

/* Double checkerboard order with multi-hit updates (Sec. 3.2 and 3.4; in
 * three dimensions, Sec. 3.6, the tiles are T x T x T cubes).  The lattice is
 * cut into tiles of edge T; tile (x / T, y / T[, z / T]) has the coarse
 * colour (x / T + y / T [+ z / T]) mod 2.  A compound move takes the tiles
 * of one coarse colour through k hits, each hit updating the fine colour-0
 * sites of those tiles (fine colour = the site's colour (x + y [+ z]) mod 2)
 * and then their fine colour-1 sites, and then treats the tiles of the other
 * coarse colour the same way.  Coarse colour 0 goes first; with `symmetric`,
 * odd compound moves (counted from the start of the chain) take coarse
 * colour 1 first, so the moves alternate A^k B^k and B^k A^k.  Hit h of
 * compound move m draws its words with sweep number m k + h, so every site
 * is updated k times per compound move and n_sweeps (a multiple of k) counts
 * those updates; first_sweep is a multiple of k.  T must divide L with L / T
 * even; any order within one fine-colour step is equivalent, since its
 * sites are not neighbours. */
void or_dcb_sweeps_dim(int dim, int L, int8_t *s, const int8_t *J, double beta, uint64_t seed,
                       uint32_t lattice_id, uint32_t first_sweep, int64_t n_sweeps, int T, int k,
                       int symmetric, int64_t *flips) {
  const int64_t n = or_nsites(dim, L);
  uint32_t thr[4] = {0, 0, 0, 0};
  for (int m = 1; m <= dim; ++m) thr[m] = or_metropolis_threshold(beta, 4 * m);
  for (int64_t mv = 0; mv < n_sweeps / k; ++mv) {
    const uint32_t M = first_sweep / (uint32_t)k + (uint32_t)mv;
    const int first = (symmetric && (M & 1u)) ? 1 : 0;
    for (int cc = 0; cc < 2; ++cc) {
      const int coarse = first ^ cc;
      for (int h = 0; h < k; ++h) {
        const uint32_t sweep = M * (uint32_t)k + (uint32_t)h;
        for (int colour = 0; colour < 2; ++colour) {
          for (int64_t i = 0; i < n; ++i) {
            const int x = (int)(i % L), y = (int)((i / L) % L), z = dim == 3 ? (int)(i / ((int64_t)L * L)) : 0;
            if (((x / T + y / T + z / T) & 1) != coarse) continue;
            if (or_colour(dim, L, i) != colour) continue;
            const int hf = or_local_field(dim, L, s, J, i);
            const int dE = 2 * s[i] * hf;
            int flip;
            if (dE <= 0) {
              flip = 1;
            } else {
              const uint32_t r = or_draw(seed, OR_TAG_UPDATE, (uint32_t)colour, 0, lattice_id, sweep,
                                         (uint32_t)(i >> 1));
              flip = r < thr[dE / 4];
            }
            if (flip) {
              s[i] = (int8_t)(-s[i]);
              if (flips) ++*flips;
            }
          }
        }
      }
    }
  }
}

/* The 2D form (kept for its callers). */
void or_dcb_sweeps(int L, int8_t *s, const int8_t *J, double beta, uint64_t seed,
                   uint32_t lattice_id, uint32_t first_sweep, int64_t n_sweeps, int T, int k,
                   int symmetric, int64_t *flips) {
  or_dcb_sweeps_dim(2, L, s, J, beta, seed, lattice_id, first_sweep, n_sweeps, T, k, symmetric, flips);
}

/* Energy E = -sum_<ij> J_ij s_i s_j (Eq. ising_hamiltonian with J = 1,
 * Eq. spinglass_hamiltonian otherwise), each bond counted once as (i, i+d). */
int64_t or_ising_energy(int dim, int L, const int8_t *s, const int8_t *J) {
  int64_t n = or_nsites(dim, L), e = 0;
  for (int64_t i = 0; i < n; ++i)
    for (int d = 0; d < dim; ++d) {
      int64_t up = or_neighbour(dim, L, i, d, +1);
      int jv = J ? J[d * n + i] : 1;
      e -= (int64_t)jv * s[i] * s[up];
    }
  return e;
}

int64_t or_ising_magnetisation(int dim, int L, const int8_t *s) {
  int64_t n = or_nsites(dim, L), m = 0;
  for (int64_t i = 0; i < n; ++i) m += s[i];
  return m;
}

/* Overlap q = sum_i s_i^(0) s_i^(1) of two replicas of one realisation. */
int64_t or_overlap(int dim, int L, const int8_t *s0, const int8_t *s1) {
  int64_t n = or_nsites(dim, L), q = 0;
  for (int64_t i = 0; i < n; ++i) q += s0[i] * s1[i];
  return q;
}

/* ------------------------------------------------------------------ */
/* Replica exchange (Eq. parallel_tempering)                           */
/* ------------------------------------------------------------------ */

/* One replica-exchange step for one realisation r of replica set a.
 * slots[t] is the configuration held at inverse temperature betas[t],
 * E[t] its energy.  Pairs (t, t+1) with t = pt_step (mod 2) are tried;
 * with Delta = (beta_{t+1} - beta_t) (E_{t+1} - E_t) the exchange is
 * accepted iff Delta >= 0 or r < thr, thr the threshold of exp(Delta).
 * The pairs of one step are disjoint, so their order does not matter.
 * On acceptance the two configurations and their energies are exchanged.
 * accepted[t] (optional) counts accepted exchanges of pair (t, t+1).
 * labels[t] (optional) names the configuration held at slot t; an accepted
 * exchange moves the two labels with their configurations (Sec. 6 on
 * exchanging configurations rather than temperatures: the labels let a
 * caller follow each configuration through the temperature slots). */
void or_pt_step(int dim, int L, int n_temps, int8_t **slots, int64_t *E,
                const double *betas, uint64_t seed, uint32_t set_a, uint32_t r,
                uint32_t pt_step, int64_t *accepted, int32_t *labels) {
  int64_t n = or_nsites(dim, L);
  for (int t = (int)(pt_step & 1u); t + 1 < n_temps; t += 2) {
    double dbeta = betas[t + 1] - betas[t];
    int64_t dE = E[t + 1] - E[t];
    int accept;
    if (dbeta * (double)dE >= 0.0) {
      accept = 1;
    } else {
      int64_t m = (dE < 0 ? -dE : dE) / 4;
      uint32_t rnd = or_draw(seed, OR_TAG_PT, 0, 0, or_lattice_id(set_a, 0, (uint32_t)t),
                             pt_step, r);
      accept = rnd < or_pt_threshold(fabs(dbeta), m);
    }
    if (accept) {
      for (int64_t i = 0; i < n; ++i) {
        int8_t tmp = slots[t][i];
        slots[t][i] = slots[t + 1][i];
        slots[t + 1][i] = tmp;
      }
      int64_t te = E[t];
      E[t] = E[t + 1];
      E[t + 1] = te;
      if (labels) {
        int32_t tl = labels[t];
        labels[t] = labels[t + 1];
        labels[t + 1] = tl;
      }
      if (accepted) accepted[t] += 1;
    }
  }
}

/* ------------------------------------------------------------------ */
/* Heisenberg model (Eq. On_hamiltonian, n = 3), double precision      */
/* ------------------------------------------------------------------ */

/* Uniformly distributed unit vector from two uniforms: z = 2u1 - 1,
 * phi = 2 pi u2 (Archimedes' z-phi construction; the paper asks only for a
 * uniformly drawn new direction, Sec. 4). */
static void or_unit_vector(double u1, double u2, double v[3]) {
  double z = 2.0 * u1 - 1.0;
  double phi = 6.283185307179586476925 * u2; /* 2 pi */
  double rho = sqrt(1.0 - z * z);
  v[0] = rho * cos(phi);
  v[1] = rho * sin(phi);
  v[2] = z;
}

/* Hot start: site i points along the unit vector of words 0, 1 of the
 * HEIS_INIT call with counter x = i. */
void or_heis_init(int dim, int L, double *s, uint64_t seed, uint32_t lattice_id) {
  int64_t n = or_nsites(dim, L);
  for (int64_t i = 0; i < n; ++i) {
    uint32_t w[4];
    or_call(seed, OR_TAG_HEIS_INIT, 0, 0, lattice_id, 0, (uint32_t)i, w);
    or_unit_vector(or_uniform(w[0]), or_uniform(w[1]), &s[3 * i]);
  }
}

/* One Metropolis update of Heisenberg site i (of colour `colour`): the site
 * proposes a new, uniformly drawn direction n (words 0, 1 of the HEIS call
 * with counter x = j = i >> 1, colour c, sweep number `sweep`) and accepts
 * it with the Metropolis rule using word 2: dE = -(n - s_i) . h_i, h_i the
 * sum of the neighbour spins; accept iff dE <= 0 or u3 < exp(-beta dE).
 * Returns |u3 - exp(-beta dE)|: how far the decision was from flipping. */
double or_heis_site(int dim, int L, double *s, int64_t i, int colour, double beta, uint64_t seed,
                    uint32_t lattice_id, uint32_t sweep) {
  double h[3] = {0.0, 0.0, 0.0};
  for (int d = 0; d < dim; ++d) {
    int64_t up = or_neighbour(dim, L, i, d, +1);
    int64_t dn = or_neighbour(dim, L, i, d, -1);
    for (int k = 0; k < 3; ++k) h[k] += s[3 * up + k] + s[3 * dn + k];
  }
  uint32_t w[4];
  or_call(seed, OR_TAG_HEIS, (uint32_t)colour, 0, lattice_id, sweep, (uint32_t)(i >> 1), w);
  double nv[3];
  or_unit_vector(or_uniform(w[0]), or_uniform(w[1]), nv);
  double u3 = or_uniform(w[2]);
  double dE = 0.0;
  for (int k = 0; k < 3; ++k) dE -= (nv[k] - s[3 * i + k]) * h[k];
  double boltz = exp(-beta * dE);
  if (dE <= 0.0 || u3 < boltz)
    for (int k = 0; k < 3; ++k) s[3 * i + k] = nv[k];
  return fabs(u3 - boltz);
}

/* One checkerboard sweep of the Heisenberg model (Sec. 4): every colour-0
 * site, then every colour-1 site, takes or_heis_site.  `margin` (optional)
 * receives the per-site distance of the decision from flipping. */
void or_heis_sweep(int dim, int L, double *s, double beta, uint64_t seed,
                   uint32_t lattice_id, uint32_t sweep, double *margin) {
  int64_t n = or_nsites(dim, L);
  for (int colour = 0; colour < 2; ++colour) {
    for (int64_t i = 0; i < n; ++i) {
      if (or_colour(dim, L, i) != colour) continue;
      const double mg = or_heis_site(dim, L, s, i, colour, beta, seed, lattice_id, sweep);
      if (margin) margin[i] = mg;
    }
  }
}

/* s_i <- s_i / |s_i| for every site. */
void or_heis_renormalise(int dim, int L, double *s) {
  int64_t n = or_nsites(dim, L);
  for (int64_t i = 0; i < n; ++i) {
    double r = sqrt(s[3 * i] * s[3 * i] + s[3 * i + 1] * s[3 * i + 1] +
                    s[3 * i + 2] * s[3 * i + 2]);
    for (int k = 0; k < 3; ++k) s[3 * i + k] /= r;
  }
}

/* The Heisenberg model in the double-checkerboard order with multi-hit
 * updates (Sec. 4 uses it for its GPU code): tiles, compound moves, hit
 * numbering and the symmetric variant exactly as in or_dcb_sweeps_dim, each
 * update being or_heis_site.  After a compound move the spins are
 * renormalised if the move passed a sweep count (1-based) that is a
 * multiple of renorm_every (> 0), the rule of the plain sweeps.  `margin`
 * (optional) receives per site the smallest distance of its decisions from
 * flipping over the whole call. */
void or_heis_dcb_sweeps(int dim, int L, double *s, double beta, uint64_t seed, uint32_t lattice_id,
                        uint32_t first_sweep, int64_t n_sweeps, int T, int k, int symmetric, int renorm_every,
                        double *margin) {
  const int64_t n = or_nsites(dim, L);
  if (margin)
    for (int64_t i = 0; i < n; ++i) margin[i] = 1e300;
  for (int64_t mv = 0; mv < n_sweeps / k; ++mv) {
    const uint32_t M = first_sweep / (uint32_t)k + (uint32_t)mv;
    const int first = (symmetric && (M & 1u)) ? 1 : 0;
    for (int cc = 0; cc < 2; ++cc) {
      const int coarse = first ^ cc;
      for (int h = 0; h < k; ++h) {
        const uint32_t sweep = M * (uint32_t)k + (uint32_t)h;
        for (int colour = 0; colour < 2; ++colour) {
          for (int64_t i = 0; i < n; ++i) {
            const int x = (int)(i % L), y = (int)((i / L) % L), z = dim == 3 ? (int)(i / ((int64_t)L * L)) : 0;
            if (((x / T + y / T + z / T) & 1) != coarse) continue;
            if (or_colour(dim, L, i) != colour) continue;
            const double mg = or_heis_site(dim, L, s, i, colour, beta, seed, lattice_id, sweep);
            if (margin && mg < margin[i]) margin[i] = mg;
          }
        }
      }
    }
    const uint64_t before = (uint64_t)M * (uint64_t)k, after = before + (uint64_t)k;
    if (renorm_every > 0 && after / (uint64_t)renorm_every > before / (uint64_t)renorm_every)
      or_heis_renormalise(dim, L, s);
  }
}

/* E = -sum_<ij> s_i . s_j, each bond once as (i, i+d); M = sum_i s_i. */
double or_heis_energy(int dim, int L, const double *s) {
  int64_t n = or_nsites(dim, L);
  double e = 0.0;
  for (int64_t i = 0; i < n; ++i)
    for (int d = 0; d < dim; ++d) {
      int64_t up = or_neighbour(dim, L, i, d, +1);
      e -= s[3 * i] * s[3 * up] + s[3 * i + 1] * s[3 * up + 1] + s[3 * i + 2] * s[3 * up + 2];
    }
  return e;
}

void or_heis_magnetisation(int dim, int L, const double *s, double m[3]) {
  int64_t n = or_nsites(dim, L);
  m[0] = m[1] = m[2] = 0.0;
  for (int64_t i = 0; i < n; ++i)
    for (int k = 0; k < 3; ++k) m[k] += s[3 * i + k];
}

/* ------------------------------------------------------------------ */
/* Drivers: several sweeps in a row, with per-sweep measurements        */
/* ------------------------------------------------------------------ */

/* n_sweeps sweeps with sweep indices first_sweep, first_sweep + 1, ...;
 * E[k], M[k] (optional) receive the energy and magnetisation after sweep k. */
void or_ising_run(int dim, int L, int8_t *s, const int8_t *J, double beta,
                  uint64_t seed, uint32_t lattice_id, uint32_t first_sweep,
                  int64_t n_sweeps, int64_t *E, int64_t *M, int64_t *flips) {
  for (int64_t k = 0; k < n_sweeps; ++k) {
    or_ising_sweep(dim, L, s, J, beta, seed, lattice_id, first_sweep + (uint32_t)k, flips);
    if (E) E[k] = or_ising_energy(dim, L, s, J);
    if (M) M[k] = or_ising_magnetisation(dim, L, s);
  }
}

/* Heisenberg run: after every sweep whose 1-based count is a multiple of
 * renorm_every (if > 0) all spins are renormalised to unit length. */
void or_heis_run(int dim, int L, double *s, double beta, uint64_t seed,
                 uint32_t lattice_id, uint32_t first_sweep, int64_t n_sweeps,
                 int renorm_every, double *E, double *M3) {
  for (int64_t k = 0; k < n_sweeps; ++k) {
    uint32_t sweep = first_sweep + (uint32_t)k;
    or_heis_sweep(dim, L, s, beta, seed, lattice_id, sweep, NULL);
    if (renorm_every > 0 && (sweep + 1u) % (uint32_t)renorm_every == 0u)
      or_heis_renormalise(dim, L, s);
    if (E) E[k] = or_heis_energy(dim, L, s);
    if (M3) or_heis_magnetisation(dim, L, s, &M3[3 * k]);
  }
}

/* Parallel-tempering run of one realisation r (Sec. 6): n_sets independent
 * replica sets, each with n_temps slots at betas[t]; spins is
 * [n_sets][n_temps][N].  Every sweep updates all lattices, then measures
 * E per (set, slot) and the overlap Q per slot between sets 0 and 1; when
 * pt_every divides the 1-based sweep count, every set performs one
 * exchange step (or_pt_step) with step counter pt_step, which then
 * advances.  rkey = r >> 5 for EA (group-shared update uniforms), r for
 * the ferromagnet.  E_series [n_sweeps][n_sets][n_temps] and Q_series
 * [n_sweeps][n_temps] hold the measurements taken before that sweep's
 * exchange step; accepted [n_sets][n_temps] counts accepted exchanges and
 * labels [n_sets][n_temps] (optional) follow the configurations as in
 * or_pt_step. */
void or_pt_run(int dim, int L, int n_temps, int n_sets, int8_t *spins, const int8_t *J,
               const double *betas, uint64_t seed, uint32_t r, uint32_t rkey,
               uint32_t first_sweep, int64_t n_sweeps, int pt_every,
               uint32_t *pt_step, int64_t *E_series, int64_t *Q_series,
               int64_t *accepted, int32_t *labels) {
  int64_t n = or_nsites(dim, L);
  int8_t **slots = (int8_t **)malloc(sizeof(int8_t *) * (size_t)n_temps);
  int64_t *E = (int64_t *)malloc(sizeof(int64_t) * (size_t)n_temps * (size_t)n_sets);
  for (int64_t k = 0; k < n_sweeps; ++k) {
    uint32_t sweep = first_sweep + (uint32_t)k;
    for (int a = 0; a < n_sets; ++a)
      for (int t = 0; t < n_temps; ++t) {
        int8_t *lat = spins + ((int64_t)a * n_temps + t) * n;
        or_ising_sweep(dim, L, lat, J, betas[t], seed,
                       or_lattice_id((uint32_t)a, rkey, (uint32_t)t), sweep, NULL);
        E[a * n_temps + t] = or_ising_energy(dim, L, lat, J);
      }
    if (E_series)
      for (int q = 0; q < n_sets * n_temps; ++q) E_series[k * n_sets * n_temps + q] = E[q];
    if (Q_series && n_sets >= 2)
      for (int t = 0; t < n_temps; ++t)
        Q_series[k * n_temps + t] =
            or_overlap(dim, L, spins + (int64_t)t * n, spins + ((int64_t)n_temps + t) * n);
    if (pt_every > 0 && (sweep + 1u) % (uint32_t)pt_every == 0u) {
      for (int a = 0; a < n_sets; ++a) {
        for (int t = 0; t < n_temps; ++t) slots[t] = spins + ((int64_t)a * n_temps + t) * n;
        or_pt_step(dim, L, n_temps, slots, &E[a * n_temps], betas, seed, (uint32_t)a, r,
                   *pt_step, accepted ? &accepted[a * n_temps] : NULL,
                   labels ? &labels[a * n_temps] : NULL);
      }
      *pt_step += 1u;
    }
  }
  free(E);
  free(slots);
}

/* ------------------------------------------------------------------ */
/* Light-cone evaluation for sampled checks of very large lattices     */
/* ------------------------------------------------------------------ */

/* The same checkerboard sweeps as or_ising_sweep (ferromagnet), restricted
 * to a W^dim window of a much larger L^dim lattice whose lowest corner is
 * at global coordinates origin[] (taken mod L).  win holds the window's
 * spins in the window's own row-major order.  At half-sweep k
 * (k = 0, 1, ...) only window sites at distance >= k + 1 from the window
 * boundary are updated, so after n sweeps the sites at distance >= 2n from
 * the boundary hold exactly the values the full-lattice sweeps would give.
 * Colours and random-number indices use the global coordinates. */
void or_ising_window_sweeps(int dim, int L, const int origin[3], int W, int8_t *win,
                            double beta, uint64_t seed, uint32_t lattice_id,
                            uint32_t first_sweep, int n_sweeps) {
  uint32_t thr[4] = {0, 0, 0, 0};
  for (int m = 1; m <= dim; ++m) thr[m] = or_metropolis_threshold(beta, 4 * m);
  int64_t nw = 1;
  for (int d = 0; d < dim; ++d) nw *= W;
  int8_t *next = (int8_t *)malloc((size_t)nw);
  for (int half = 0; half < 2 * n_sweeps; ++half) {
    int colour = half & 1;
    uint32_t sweep = first_sweep + (uint32_t)(half / 2);
    memcpy(next, win, (size_t)nw);
    for (int64_t p = 0; p < nw; ++p) {
      int wc[3] = {0, 0, 0}, gc[3] = {0, 0, 0};
      or_coords(dim, W, p, wc);
      int dist = W;
      for (int d = 0; d < dim; ++d) {
        int e = wc[d] < W - 1 - wc[d] ? wc[d] : W - 1 - wc[d];
        if (e < dist) dist = e;
        gc[d] = (origin[d] + wc[d]) % L;
      }
      if (dist < half + 1) continue;
      if (((gc[0] + gc[1] + gc[2]) & 1) != colour) continue;
      int h = 0;
      for (int d = 0; d < dim; ++d) {
        int c[3] = {wc[0], wc[1], wc[2]};
        c[d] += 1;
        h += win[or_index(dim, W, c)];
        c[d] -= 2;
        h += win[or_index(dim, W, c)];
      }
      int dE = 2 * win[p] * h;
      int flip = dE <= 0;
      if (!flip) {
        int64_t gi = or_index(dim, L, gc);
        uint32_t r = or_draw(seed, OR_TAG_UPDATE, (uint32_t)colour, 0, lattice_id, sweep,
                             (uint32_t)(gi >> 1));
        flip = r < thr[dE / 4];
      }
      if (flip) next[p] = (int8_t)(-win[p]);
    }
    memcpy(win, next, (size_t)nw);
  }
  free(next);
}

/* Hot-start values of arbitrary sites (global linear indices idx[]). */
void or_ising_init_sites(int64_t count, const int64_t *idx, int8_t *out, uint64_t seed,
                         uint32_t lattice_id, int bit) {
  for (int64_t k = 0; k < count; ++k) {
    uint32_t w = or_draw(seed, OR_TAG_INIT, 0, 0, lattice_id, 0, (uint32_t)idx[k]);
    out[k] = ((w >> bit) & 1u) ? -1 : 1;
  }
}
