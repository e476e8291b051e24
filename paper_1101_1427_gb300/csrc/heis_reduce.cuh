// Heisenberg energy and magnetisation in FP64 (Sec. 4: double accumulation
// for continuous spins), shared by spin_measure and the allocation-free
// reduction so that the two give bit-identical sums.
//
// E = -sum_<ij> s_i . s_j with each bond counted once as (i, i + e_d), and
// M = sum_i s_i, over one lattice of L^dim float4 spins (x fastest, periodic).
// FP32 components are widened to double before every product; a thread sums
// its sites in grid-stride order, then warp, block and (in the finishing
// step) the block partials are added in a fixed order.
#pragma once
#include <stdint.h>

#include "common.cuh"

namespace spin {

// Block partials [E, Mx, My, Mz] of lattice `sl` (N = L^dim sites) from the
// blocks of one grid row: block b of nb visits sites b * blockDim.x + tid,
// then strides by nb * blockDim.x.  blockDim.x is a multiple of 32, <= 1024.
__device__ __forceinline__ void heis_block_partials(const float4 *__restrict__ sl, int L, int dim, int64_t N,
                                                    int b, int nb, double *__restrict__ out4) {
  const int64_t LL = (int64_t)L * L;
  double e = 0.0, mx = 0.0, my = 0.0, mz = 0.0;
  for (int64_t i = b * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)nb * blockDim.x) {
    const int x = (int)(i % L), y = (int)((i / L) % L), z = (int)(i / LL);
    const float4 a = sl[i];
    const float4 bx = sl[i - x + (x == L - 1 ? 0 : x + 1)];
    const float4 by = sl[y == L - 1 ? i - (int64_t)(L - 1) * L : i + L];
    const double ax = a.x, ay = a.y, az = a.z;
    if (dim == 3) {
      const float4 bz = sl[z == L - 1 ? i - (int64_t)(L - 1) * LL : i + LL];
      e -= ax * ((double)bx.x + (double)by.x + (double)bz.x) +
           ay * ((double)bx.y + (double)by.y + (double)bz.y) +
           az * ((double)bx.z + (double)by.z + (double)bz.z);
    } else {
      e -= ax * ((double)bx.x + (double)by.x) + ay * ((double)bx.y + (double)by.y) +
           az * ((double)bx.z + (double)by.z);
    }
    mx += ax;
    my += ay;
    mz += az;
  }
  __shared__ double red[4][32];
  e = warp_sum(e);
  mx = warp_sum(mx);
  my = warp_sum(my);
  mz = warp_sum(mz);
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    red[0][wid] = e;
    red[1][wid] = mx;
    red[2][wid] = my;
    red[3][wid] = mz;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double acc = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) acc += red[threadIdx.x][k];
    out4[threadIdx.x] = acc;
  }
}

// Adds the nb block partials of lattice `lat` (layout [lat][block][4]) in
// block order and stores E (Ef[lat]) and M (Mf[3 lat ..]); NULL skips.
__device__ __forceinline__ void heis_finish_lattice(const double *__restrict__ part, int nb, int64_t lat,
                                                    double *__restrict__ Ef, double *__restrict__ Mf) {
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int b = 0; b < nb; ++b)
    for (int c = 0; c < 4; ++c) acc[c] += part[(lat * nb + b) * 4 + c];
  if (Ef) Ef[lat] = acc[0];
  if (Mf) {
    Mf[3 * lat] = acc[1];
    Mf[3 * lat + 1] = acc[2];
    Mf[3 * lat + 2] = acc[3];
  }
}

}  // namespace spin
