// Slab decomposition of one 2D int8 ferromagnet (multi-GPU design): a rank
// owns rows y0 .. y0 + rows - 1 of the L x L periodic lattice and holds them
// as [rows + 2][L] bytes, slab rows 0 and rows + 1 being copies of the rows
// above and below (exchanged by the caller before each colour phase).  The
// update of an own site is that of the checkerboard sweep (Sec. 3.2,
// Eq. metropolis) with its global colour and its global Philox counter, so
// any split reproduces the unsplit chain.
#include <math.h>

#include "i8chunk.cuh"
#include "internal.h"

namespace spin {
namespace {

__global__ void __launch_bounds__(256) slab_phase_kernel(int8_t *__restrict__ slab, int L, int y0, int rows,
                                                         uint32_t thr4, uint32_t thr8, RoundKeys rk,
                                                         uint32_t lid, uint32_t sweep, int colour) {
  const uint32_t chunks = (uint32_t)L >> 3;
  const uint32_t total = (uint32_t)rows * chunks;
  const uint32_t wctr = ctr_w(TAG_UPDATE, (uint32_t)colour, 0);
  long long unused_a = 0, unused_d = 0;
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < total; k += gridDim.x * blockDim.x) {
    const uint32_t rr = k / chunks, m = k - rr * chunks;
    const int r = (int)rr + 1;
    const uint32_t y = (uint32_t)y0 + rr;  // global row
    int8_t *row = slab + (int64_t)r * L;
    const uint64_t C = reinterpret_cast<const uint64_t *>(row)[m];
    const uint64_t U = reinterpret_cast<const uint64_t *>(row - L)[m];
    const uint64_t D = reinterpret_cast<const uint64_t *>(row + L)[m];
    const uint64_t lb = (uint8_t)row[m == 0 ? L - 1 : 8 * m - 1];
    const uint64_t rb = (uint8_t)row[m == chunks - 1 ? 0 : 8 * m + 8];
    const uint4 q = philox(make_uint4(y * chunks + m, sweep, lid, wctr), rk);
    reinterpret_cast<uint64_t *>(row)[m] =
        ising_chunk<0>(C, U, D, lb, rb, q, (colour + (int)y) & 1, thr4, thr8, unused_a, unused_d);
  }
}

// Partial sums of the slab's own rows: E over the bonds to the right and
// below of every own site (the row below the last own row is the lower
// ghost), so the partial energies of all slabs add up to E; M over own sites.
__global__ void slab_measure_kernel(const int8_t *__restrict__ slab, int L, int rows,
                                    unsigned long long *__restrict__ E, unsigned long long *__restrict__ M) {
  const int64_t total = (int64_t)rows * L;
  long long e = 0, m = 0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = k / L + 1, x = k - (r - 1) * L;
    const int8_t *row = slab + r * L;
    const int s = row[x];
    e -= s * (row[x == L - 1 ? 0 : x + 1] + row[x + L]);
    m += s;
  }
  e = warp_sum(e);
  m = warp_sum(m);
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(E, (unsigned long long)e);
    atomicAdd(M, (unsigned long long)m);
  }
}

uint32_t threshold(double beta, int dE) {
  const double t = floor(exp(-beta * (double)dE) * 4294967296.0);
  if (t >= 4294967295.0) return 0xFFFFFFFFu;
  return t <= 0.0 ? 0u : (uint32_t)t;
}

}  // namespace
}  // namespace spin

using namespace spin;

extern "C" int spin_slab_phase(int8_t *slab, int32_t L, int32_t y0, int32_t rows, double beta, uint64_t seed,
                               uint32_t lattice_id, uint32_t sweep, int32_t colour, void *stream) {
  if (!slab || L < 8 || (L & 7) || rows < 1 || y0 < 0 || (int64_t)y0 + rows > L || (colour & ~1) ||
      !isfinite(beta) || beta < 0.0 || (int64_t)(rows + 2) * L >= ((int64_t)1 << 31))
    return SPIN_EINVAL;
  if (((uintptr_t)slab & 7u) != 0) return SPIN_EALIGN;
  const int64_t total = (int64_t)rows * (L / 8);
  unsigned grid = grid_for(total, 256);
  if (grid > (1u << 20)) grid = 1u << 20;
  slab_phase_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(slab, L, y0, rows, threshold(beta, 4),
                                                            threshold(beta, 8), make_round_keys(seed),
                                                            lattice_id, sweep, colour);
  return cudaGetLastError() == cudaSuccess ? SPIN_OK : SPIN_ECUDA;
}

extern "C" int spin_slab_measure(const int8_t *slab, int32_t L, int32_t rows, int64_t *E, int64_t *M,
                                 void *stream) {
  if (!slab || !E || !M || L < 2 || rows < 1 || (int64_t)(rows + 2) * L >= ((int64_t)1 << 31))
    return SPIN_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemsetAsync(E, 0, sizeof(int64_t), st) != cudaSuccess ||
      cudaMemsetAsync(M, 0, sizeof(int64_t), st) != cudaSuccess)
    return SPIN_ECUDA;
  unsigned grid = grid_for((int64_t)rows * L, 256);
  if (grid > 4096u) grid = 4096u;
  slab_measure_kernel<<<grid, 256, 0, st>>>(slab, L, rows, (unsigned long long *)E, (unsigned long long *)M);
  return cudaGetLastError() == cudaSuccess ? SPIN_OK : SPIN_ECUDA;
}
