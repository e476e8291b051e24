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
