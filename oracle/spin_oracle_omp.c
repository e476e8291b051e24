/*
 * spin_oracle_omp.c -- the oracle's checkerboard sweep of the 2D Ising
 * ferromagnet run on all host cores, for the CPU baseline of the benchmark.
 *
 * TEST INFRASTRUCTURE ONLY (like spin_oracle.c, whose conventions it keeps:
 * x fastest, periodic, colour (x + y) mod 2 with colour 0 first, integer
 * Metropolis thresholds, the UPDATE word of (seed, lattice_id, sweep,
 * colour, j = i >> 1)).  Sites of one colour have no neighbour of their own
 * colour (Sec. 3.2), so within one colour phase the rows can be updated in
 * any order and by any number of threads: OpenMP splits the rows of each
 * phase among the host cores.  The random words and thresholds come from the
 * serial oracle's own functions, so the result equals or_ising_sweep bit for
 * bit.  It is built into its own library so that the serial oracle needs no
 * OpenMP runtime.
 */
#include <stdint.h>

#include <omp.h>

uint32_t or_draw(uint64_t seed, uint32_t tag, uint32_t colour, uint32_t extra, uint32_t lattice_id,
                 uint32_t sweep, uint32_t idx);
uint32_t or_metropolis_threshold(double beta, int dE);

/* One colour phase of rows y0 .. y1 - 1 of an L x L periodic ferromagnet s
 * (the whole lattice is in memory; rows outside the range are read only). */
static int64_t phase_rows(int L, int8_t *s, int y0, int y1, const uint32_t thr[3], uint64_t seed,
                          uint32_t lattice_id, uint32_t sweep, int colour) {
  int64_t flips = 0;
  for (int y = y0; y < y1; ++y) {
    int8_t *row = s + (int64_t)y * L;
    const int8_t *up = s + (int64_t)(y == 0 ? L - 1 : y - 1) * L;
    const int8_t *dn = s + (int64_t)(y == L - 1 ? 0 : y + 1) * L;
    for (int x = (colour + y) & 1; x < L; x += 2) {
      const int h = row[x == L - 1 ? 0 : x + 1] + row[x == 0 ? L - 1 : x - 1] + up[x] + dn[x];
      const int dE = 2 * row[x] * h;
      int flip = dE <= 0;
      if (!flip) {
        const uint32_t r = or_draw(seed, 0u /* UPDATE */, (uint32_t)colour, 0u, lattice_id, sweep,
                                   (uint32_t)(((int64_t)y * L + x) >> 1));
        flip = r < thr[dE / 4];
      }
      if (flip) {
        row[x] = (int8_t)(-row[x]);
        ++flips;
      }
    }
  }
  return flips;
}

/* n_sweeps checkerboard sweeps (colour 0, then colour 1) with sweep numbers
 * first_sweep, first_sweep + 1, ...; rows of each phase are shared among
 * `threads` OpenMP threads (<= 0: the runtime's default).  Returns the
 * number of accepted flips; *threads_used receives the team size. */
int64_t or_omp_ising2d_sweeps(int L, int8_t *s, double beta, uint64_t seed, uint32_t lattice_id,
                              uint32_t first_sweep, int64_t n_sweeps, int threads, int *threads_used) {
  uint32_t thr[3] = {0u, or_metropolis_threshold(beta, 4), or_metropolis_threshold(beta, 8)};
  int64_t flips = 0;
  int used = 1;
  if (threads <= 0) threads = omp_get_max_threads();
  for (int64_t k = 0; k < n_sweeps; ++k) {
    for (int colour = 0; colour < 2; ++colour) {
#pragma omp parallel num_threads(threads) reduction(+ : flips)
      {
        const int nt = omp_get_num_threads(), id = omp_get_thread_num();
        if (id == 0) used = nt;
        const int y0 = (int)((int64_t)L * id / nt), y1 = (int)((int64_t)L * (id + 1) / nt);
        flips += phase_rows(L, s, y0, y1, thr, seed, lattice_id, first_sweep + (uint32_t)k, colour);
      }
    }
  }
  if (threads_used) *threads_used = used;
  return flips;
}

/* ------------------------------------------------------------------ */
/* Long oracle runs for the full-size parity tests                      */
/* ------------------------------------------------------------------ */

void or_ising_sweep(int dim, int L, int8_t *s, const int8_t *J, double beta, uint64_t seed,
                    uint32_t lattice_id, uint32_t sweep, int64_t *flips);
int64_t or_ising_energy(int dim, int L, const int8_t *s, const int8_t *J);
int64_t or_overlap(int dim, int L, const int8_t *s0, const int8_t *s1);
void or_pt_step(int dim, int L, int n_temps, int8_t **slots, int64_t *E, const double *betas, uint64_t seed,
                uint32_t set_a, uint32_t r, uint32_t pt_step, int64_t *accepted, int32_t *labels);
uint32_t or_lattice_id(uint32_t a, uint32_t rkey, uint32_t t);
double or_heis_site(int dim, int L, double *s, int64_t i, int colour, double beta, uint64_t seed,
                    uint32_t lattice_id, uint32_t sweep);
int or_colour(int dim, int L, int64_t i);
void or_heis_renormalise(int dim, int L, double *s);

/* or_pt_run of spin_oracle.c with the work of a sweep shared among threads:
 * the n_sets x n_temps lattices of a realisation are swept and measured
 * independently (different lattices, the same serial calls), so their
 * order does not matter; the overlaps and the exchange steps then run as
 * in the serial form.  Arguments and results as or_pt_run. */
void or_omp_pt_run(int dim, int L, int n_temps, int n_sets, int8_t *spins, const int8_t *J,
                   const double *betas, uint64_t seed, uint32_t r, uint32_t rkey, uint32_t first_sweep,
                   int64_t n_sweeps, int pt_every, uint32_t *pt_step, int64_t *E_series, int64_t *Q_series,
                   int64_t *accepted, int32_t *labels, int threads) {
  int64_t n = 1;
  for (int d = 0; d < dim; ++d) n *= L;
  const int n_lat = n_sets * n_temps;
  int8_t *slots[4096];
  int64_t E[2 * 4096];
  if (n_temps > 4096 || n_sets > 2) return;  /* sizes of the arrays above */
  if (threads <= 0) threads = omp_get_max_threads();
  for (int64_t k = 0; k < n_sweeps; ++k) {
    const uint32_t sweep = first_sweep + (uint32_t)k;
#pragma omp parallel for num_threads(threads) schedule(dynamic, 1)
    for (int q = 0; q < n_lat; ++q) {
      const int a = q / n_temps, t = q - a * n_temps;
      int8_t *lat = spins + (int64_t)q * n;
      or_ising_sweep(dim, L, lat, J, betas[t], seed, or_lattice_id((uint32_t)a, rkey, (uint32_t)t), sweep, 0);
      E[q] = or_ising_energy(dim, L, lat, J);
    }
    if (E_series)
      for (int q = 0; q < n_lat; ++q) E_series[k * n_lat + q] = E[q];
    if (Q_series && n_sets >= 2)
      for (int t = 0; t < n_temps; ++t)
        Q_series[k * n_temps + t] = or_overlap(dim, L, spins + (int64_t)t * n, spins + ((int64_t)n_temps + t) * n);
    if (pt_every > 0 && (sweep + 1u) % (uint32_t)pt_every == 0u) {
      for (int a = 0; a < n_sets; ++a) {
        for (int t = 0; t < n_temps; ++t) slots[t] = spins + ((int64_t)a * n_temps + t) * n;
        or_pt_step(dim, L, n_temps, slots, &E[a * n_temps], betas, seed, (uint32_t)a, r, *pt_step,
                   accepted ? &accepted[a * n_temps] : 0, labels ? &labels[a * n_temps] : 0);
      }
      *pt_step += 1u;
    }
  }
}

/* E = -sum_<ij> s_i . s_j (each bond once as (i, i + e_d)) and M = sum s_i
 * of a Heisenberg lattice, summed by threads (the order of the FP64 sums,
 * and so their last bits, depends on the thread count). */
static void heis_measure_omp(int dim, int L, const double *s, double *E, double *M3, int threads) {
  int64_t n = 1;
  for (int d = 0; d < dim; ++d) n *= L;
  double e = 0.0, mx = 0.0, my = 0.0, mz = 0.0;
#pragma omp parallel for num_threads(threads) reduction(+ : e, mx, my, mz) schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    const int64_t x = i % L, y = (i / L) % L, z = dim > 2 ? i / ((int64_t)L * L) : 0;
    const int64_t nb[3] = {i - x + (x + 1) % L, i + (((y + 1) % L) - y) * L,
                           dim > 2 ? i + (((z + 1) % L) - z) * (int64_t)L * L : i};
    for (int d = 0; d < dim; ++d)
      e -= s[3 * i] * s[3 * nb[d]] + s[3 * i + 1] * s[3 * nb[d] + 1] + s[3 * i + 2] * s[3 * nb[d] + 2];
    mx += s[3 * i];
    my += s[3 * i + 1];
    mz += s[3 * i + 2];
  }
  if (E) *E = e;
  if (M3) {
    M3[0] = mx;
    M3[1] = my;
    M3[2] = mz;
  }
}

/* or_heis_run of spin_oracle.c with the sites of each colour phase shared
 * among threads (each site is the serial or_heis_site call, so the lattice
 * equals the serial run bit for bit), renormalised after every sweep whose
 * 1-based count is a multiple of renorm_every, and measured (E[k], M3[3k..])
 * after every sweep whose 1-based count within the call is a multiple of
 * measure_every (row k = that count / measure_every - 1). */
void or_omp_heis_run(int dim, int L, double *s, double beta, uint64_t seed, uint32_t lattice_id,
                     uint32_t first_sweep, int64_t n_sweeps, int renorm_every, int measure_every, double *E,
                     double *M3, int threads) {
  int64_t n = 1;
  for (int d = 0; d < dim; ++d) n *= L;
  if (threads <= 0) threads = omp_get_max_threads();
  int64_t row = 0;
  for (int64_t k = 0; k < n_sweeps; ++k) {
    const uint32_t sweep = first_sweep + (uint32_t)k;
    for (int colour = 0; colour < 2; ++colour) {
#pragma omp parallel for num_threads(threads) schedule(static)
      for (int64_t i = 0; i < n; ++i)
        if (or_colour(dim, L, i) == colour) or_heis_site(dim, L, s, i, colour, beta, seed, lattice_id, sweep);
    }
    if (renorm_every > 0 && (sweep + 1u) % (uint32_t)renorm_every == 0u) or_heis_renormalise(dim, L, s);
    if (measure_every > 0 && (k + 1) % measure_every == 0) {
      heis_measure_omp(dim, L, s, E ? &E[row] : 0, M3 ? &M3[3 * row] : 0, threads);
      ++row;
    }
  }
}
