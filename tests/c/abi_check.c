/*
 * abi_check.c -- a plain C11 caller of the library, compiled with gcc
 * against include/spin.h and linked with libspin_gb300.so, so that the
 * header is exercised as a C user sees it (test infrastructure).
 *
 *   abi_check strerror
 *       prints "<code> <message>" for SPIN_OK .. SPIN_ETIMEOUT (no GPU needed).
 *   abi_check ising L n_sweeps seed beta
 *       2D Ising ferromagnet, int8 layout, one lattice, hot start:
 *       spin_init -> spin_sweep(n_sweeps) -> spin_measure, then prints
 *       "E <E>", "M <M>", "SWEEPS <count>" and "S <L*L characters + or ->".
 *   abi_check labels
 *       checks that spin_pt_swap leaves caller labels a permutation on a
 *       small EA handle and prints "LABELS ok" (or an error).
 * Exit status 0 on success, 1 on any library or CUDA error.
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cuda_runtime_api.h>

#include "spin.h"

static int fail(const char *what, int rc) {
  fprintf(stderr, "%s: %d (%s)\n", what, rc, spin_strerror(rc));
  return 1;
}

static int run_ising(int L, int64_t n_sweeps, uint64_t seed, double beta) {
  int8_t *spins = NULL;
  int64_t *dE = NULL, *dM = NULL;
  const size_t N = (size_t)L * (size_t)L;
  if (cudaMalloc((void **)&spins, N) != cudaSuccess || cudaMalloc((void **)&dE, 8) != cudaSuccess ||
      cudaMalloc((void **)&dM, 8) != cudaSuccess) {
    fprintf(stderr, "cudaMalloc failed\n");
    return 1;
  }
  spin_desc d;
  memset(&d, 0, sizeof d);
  d.model = SPIN_ISING;
  d.dim = 2;
  d.L = L;
  d.layout = SPIN_I8;
  d.n_real = 1;
  d.n_temps = 1;
  d.n_sets = 1;
  d.hot_start = 1;
  d.seed = seed;
  d.stream = NULL;
  spin_lattice *h = NULL;
  int rc = spin_init(&h, &d, spins, NULL);
  if (rc) return fail("spin_init", rc);
  rc = spin_sweep(h, NULL, &beta, n_sweeps, seed);
  if (rc) return fail("spin_sweep", rc);
  rc = spin_measure(h, NULL, dE, dM, NULL, NULL, NULL);
  if (rc) return fail("spin_measure", rc);
  rc = spin_sync(h);
  if (rc) return fail("spin_sync", rc);
  int64_t E = 0, M = 0;
  char *host = (char *)malloc(N + 1);
  if (!host || cudaMemcpy(&E, dE, 8, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(&M, dM, 8, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(host, spins, N, cudaMemcpyDeviceToHost) != cudaSuccess) {
    fprintf(stderr, "copy back failed\n");
    return 1;
  }
  for (size_t i = 0; i < N; ++i) host[i] = ((int8_t)host[i] > 0) ? '+' : '-';
  host[N] = 0;
  printf("E %lld\nM %lld\nSWEEPS %lld\nS %s\n", (long long)E, (long long)M,
         (long long)spin_sweeps_done(h), host);
  free(host);
  spin_destroy(h);
  cudaFree(spins);
  cudaFree(dE);
  cudaFree(dM);
  return 0;
}

static int run_labels(void) {
  const int L = 4, n_real = 32, n_temps = 4, n_sets = 2;
  const int n_lat = n_real * n_temps * n_sets;
  uint32_t *spins = NULL, *J = NULL;
  int32_t *dlab = NULL;
  const size_t words = (size_t)n_sets * n_temps * L * L * L;  /* one group of 32 */
  if (cudaMalloc((void **)&spins, 4 * words) != cudaSuccess ||
      cudaMalloc((void **)&J, 4 * (size_t)3 * L * L * L) != cudaSuccess ||
      cudaMalloc((void **)&dlab, 4 * (size_t)n_lat) != cudaSuccess) {
    fprintf(stderr, "cudaMalloc failed\n");
    return 1;
  }
  spin_desc d;
  memset(&d, 0, sizeof d);
  d.model = SPIN_EA;
  d.dim = 3;
  d.L = L;
  d.layout = SPIN_MSC1;
  d.n_real = n_real;
  d.n_temps = n_temps;
  d.n_sets = n_sets;
  d.hot_start = 1;
  d.seed = 5;
  spin_lattice *h = NULL;
  int rc = spin_init(&h, &d, spins, J);
  if (rc) return fail("spin_init", rc);
  int32_t lab[256];
  for (int k = 0; k < n_lat; ++k) lab[k] = (k / n_real) % n_temps;  /* the slot of lattice k */
  if (cudaMemcpy(dlab, lab, sizeof lab, cudaMemcpyHostToDevice) != cudaSuccess) return 1;
  const double betas[4] = {0.5, 0.6, 0.7, 0.8};
  for (int step = 0; step < 20; ++step) {
    rc = spin_sweep(h, J, betas, 1, 5);
    if (rc) return fail("spin_sweep", rc);
    rc = spin_pt_swap(h, J, betas, 5, NULL, dlab);
    if (rc) return fail("spin_pt_swap", rc);
  }
  rc = spin_sync(h);
  if (rc) return fail("spin_sync", rc);
  if (cudaMemcpy(lab, dlab, sizeof lab, cudaMemcpyDeviceToHost) != cudaSuccess) return 1;
  int moved = 0;
  for (int a = 0; a < n_sets; ++a)
    for (int r = 0; r < n_real; ++r) {
      int seen[4] = {0, 0, 0, 0};
      for (int t = 0; t < n_temps; ++t) {
        const int v = lab[(a * n_temps + t) * n_real + r];
        if (v < 0 || v >= n_temps || seen[v]++) {
          fprintf(stderr, "labels of (%d, %d) are not a permutation\n", a, r);
          return 1;
        }
        moved += v != t;
      }
    }
  printf("LABELS ok %d\n", moved);
  spin_destroy(h);
  cudaFree(spins);
  cudaFree(J);
  cudaFree(dlab);
  return 0;
}

int main(int argc, char **argv) {
  if (argc >= 2 && strcmp(argv[1], "strerror") == 0) {
    for (int code = SPIN_OK; code >= SPIN_ETIMEOUT; --code) printf("%d %s\n", code, spin_strerror(code));
    return 0;
  }
  if (argc == 6 && strcmp(argv[1], "ising") == 0)
    return run_ising(atoi(argv[2]), atoll(argv[3]), (uint64_t)strtoull(argv[4], NULL, 10), atof(argv[5]));
  if (argc == 2 && strcmp(argv[1], "labels") == 0) return run_labels();
  fprintf(stderr, "usage: abi_check strerror | ising L n_sweeps seed beta | labels\n");
  return 2;
}
