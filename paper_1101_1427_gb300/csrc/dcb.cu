// Double checkerboard with multi-hit updates for the 2D and 3D int8
// ferromagnet (Sec. 3.2 and 3.4; Sec. 3.6 for three dimensions).  The lattice is cut into T x T tiles coloured like a
// checkerboard; one launch takes every tile of one coarse colour, loads it
// with a one-site halo (from tiles of the other colour, which this launch
// does not change) into shared memory, and gives it k hits there, each hit
// updating the fine colour-0 sites and then the fine colour-1 sites, before
// the tile goes back to global memory.  A compound move is one launch per
// coarse colour; hit h of compound move m draws its uniforms with sweep
// number m k + h, so every site takes k updates per compound move.
#include "i8chunk.cuh"
#include "internal.h"

namespace spin {
namespace {

// Shared tile: T + 2 rows (tile rows -1 .. T), each of T / 8 + 2 eight-byte
// words holding x = -8 .. T + 7 relative to the tile's first column, so
// that the halo bytes x = -1 and x = T sit in whole words read straight
// from the row above / below / beside.
template <int kT>
__global__ void __launch_bounds__(256) dcb_tile_kernel(int8_t *__restrict__ spins, int L, int coarse,
                                                       uint32_t sweep0, int k,
                                                       const uint32_t *__restrict__ thr, Geom g,
                                                       RoundKeys rk) {
  constexpr int kWords = kT / 8 + 2;  // words per shared row
  constexpr int kCpr = kT / 8;        // chunks per tile row
  constexpr int kChunks = kT * kCpr;  // chunks per tile
  // small tiles share a CTA of 256 threads (kTPT threads per tile)
  constexpr int kTPT = kChunks < 256 ? kChunks : 256;
  constexpr int kTiles = 256 / kTPT;
  constexpr int kTileWords = (kT + 2) * kWords;
  __shared__ __align__(16) uint64_t smem[kTiles * kTileWords];
  const int tsub = threadIdx.x / kTPT, tid = threadIdx.x - tsub * kTPT;
  uint64_t *sw = smem + tsub * kTileWords;
  const uint8_t *sb = reinterpret_cast<const uint8_t *>(sw);
  const int half = (L / kT) >> 1;
  const int t = blockIdx.x * kTiles + tsub;
  const bool active = t < (L / kT) * half;  // the last CTA may hold fewer tiles
  const int by = t / half, bx = 2 * (t % half) + ((by + coarse) & 1);
  const int64_t lat = blockIdx.y;
  int8_t *base = spins + lat * (int64_t)L * L;
  const int x0 = bx * kT, y0 = by * kT;
  if (active)
    for (int q = tid; q < kTileWords; q += kTPT) {
      const int ry = q / kWords - 1, rw = q % kWords - 1;
      const int gy = (y0 + ry + L) % L, gx = (x0 + 8 * rw + L) % L;  // L, x0 are multiples of 8
      sw[q] = *reinterpret_cast<const uint64_t *>(base + (int64_t)gy * L + gx);
    }
  __syncthreads();
  const uint32_t slot = slot_of32(g, (uint32_t)lat);
  const uint32_t thr4 = __ldg(thr + 4 * slot + 1), thr8 = __ldg(thr + 4 * slot + 2);
  const uint32_t lid = lattice_id32(g, (uint32_t)lat);
  const uint32_t row_chunks = (uint32_t)L >> 3;
  long long unused_a = 0, unused_d = 0;
  // a thread keeps the same kPer chunks for all hits, and only the sweep
  // word of their Philox counters changes: the rest of the first rounds is
  // computed once (PhiloxX1) where that fits in registers
  constexpr int kPer = kChunks / kTPT;
  constexpr bool kHoist = kPer <= 2;
  PhiloxX1 pre[kHoist ? kPer : 1][2];
  if (kHoist && active)
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
      const int q = tid + i * kTPT;
      const uint32_t gchunk = (uint32_t)(y0 + q / kCpr) * row_chunks + (uint32_t)(x0 >> 3) + (uint32_t)(q % kCpr);
#pragma unroll
      for (int c = 0; c < 2; ++c) pre[kHoist ? i : 0][c] = philox_x1_setup(gchunk, lid, ctr_w(TAG_UPDATE, (uint32_t)c, 0), rk);
    }
  for (int h = 0; h < k; ++h) {
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const uint32_t wctr = ctr_w(TAG_UPDATE, (uint32_t)c, 0);
      if (active)
#pragma unroll
        for (int i = 0; i < kPer; ++i) {
          const int q = tid + i * kTPT;
          const int ty = q / kCpr, m = q % kCpr;
          const int row = ty + 1, word = m + 1;
          const uint64_t C = sw[row * kWords + word];
          const uint64_t U = sw[(row - 1) * kWords + word], D = sw[(row + 1) * kWords + word];
          const uint64_t lb = sb[(row * kWords + word) * 8 - 1], rb = sb[(row * kWords + word) * 8 + 8];
          const int gy = y0 + ty;
          const uint32_t gchunk = (uint32_t)gy * row_chunks + (uint32_t)(x0 >> 3) + (uint32_t)m;
          const uint4 r = kHoist ? philox_x1(pre[kHoist ? i : 0][c], sweep0 + (uint32_t)h, rk)
                                 : philox(make_uint4(gchunk, sweep0 + (uint32_t)h, lid, wctr), rk);
          sw[row * kWords + word] =
              ising_chunk<0>(C, U, D, lb, rb, r, (c + gy) & 1, thr4, thr8, unused_a, unused_d);
        }
      __syncthreads();
    }
  }
  if (active)
    for (int q = tid; q < kChunks; q += kTPT) {
      const int ty = q / kCpr, m = q % kCpr;
      *reinterpret_cast<uint64_t *>(base + (int64_t)(y0 + ty) * L + x0 + 8 * m) = sw[(ty + 1) * kWords + m + 1];
    }
}

template <int kT>
cudaError_t launch_tiles(spin_lattice *h, int coarse, uint32_t sweep0) {
  constexpr int kChunks = kT * (kT / 8);
  constexpr int kTiles = kChunks < 256 ? 256 / kChunks : 1;
  const int B = h->g.L / kT;
  const int n_tiles = B * B / 2;
  dim3 grid((unsigned)((n_tiles + kTiles - 1) / kTiles), (unsigned)h->n_lat);
  dcb_tile_kernel<kT><<<grid, 256, 0, h->stream>>>((int8_t *)h->spins, h->g.L, coarse, sweep0, h->order_hits,
                                                    h->d_thr, h->g, make_round_keys(h->d.seed));
  return cudaGetLastError();
}

// ---------------------------------------------------------------- 3D
// The same order in three dimensions (Sec. 3.6: cubic tiles of edge T, coarse
// colour (x / T + y / T + z / T) mod 2).  Shared tile: (T + 2)^2 rows (z and
// y from -1 to T, z slowest), each of T / 8 + 2 eight-byte words holding
// x = -8 .. T + 7; only face neighbours are read, so the halo rows on the
// tile's edges (loaded along with the rest) are never used.  A chunk's
// active sites read only bytes of the other fine colour, which the current
// fine-colour step does not change, so chunks are updated in place.
template <int kT>
__global__ void __launch_bounds__(256) dcb3_tile_kernel(int8_t *__restrict__ spins, int L, int coarse,
                                                        uint32_t sweep0, int k,
                                                        const uint32_t *__restrict__ thr, Geom g,
                                                        RoundKeys rk) {
  constexpr int kWords = kT / 8 + 2;          // words per shared row
  constexpr int kSide = kT + 2;               // rows per shared plane
  constexpr int kTileWords = kSide * kSide * kWords;
  constexpr int kCpr = kT / 8;                // chunks per tile row
  constexpr int kChunks = kT * kT * kCpr;     // chunks per tile
  constexpr int kTPT = kChunks < 256 ? kChunks : 256;
  constexpr int kTiles = 256 / kTPT;
  constexpr int kPer = kChunks / kTPT;
  __shared__ __align__(16) uint64_t smem[kTiles * kTileWords];
  const int tsub = threadIdx.x / kTPT, tid = threadIdx.x - tsub * kTPT;
  uint64_t *sw = smem + tsub * kTileWords;
  const uint8_t *sb = reinterpret_cast<const uint8_t *>(sw);
  const int B = L / kT, half = B >> 1;
  const int64_t t = (int64_t)blockIdx.x * kTiles + tsub;
  const bool active = t < (int64_t)B * B * half;  // the last CTA may hold fewer tiles
  const int bxh = (int)(t % half);
  const int64_t rest = t / half;
  const int by = (int)(rest % B), bz = (int)(rest / B);
  const int bx = 2 * bxh + ((by + bz + coarse) & 1);
  const int64_t lat = blockIdx.y;
  int8_t *base = spins + lat * (int64_t)L * L * L;
  const int x0 = bx * kT, y0 = by * kT, z0 = bz * kT;
  if (active)
    for (int q = tid; q < kTileWords; q += kTPT) {
      const int row = q / kWords, rw = q % kWords - 1;
      const int ry = row % kSide - 1, rz = row / kSide - 1;
      const int gy = (y0 + ry + L) % L, gz = (z0 + rz + L) % L, gx = (x0 + 8 * rw + L) % L;
      sw[q] = *reinterpret_cast<const uint64_t *>(base + ((int64_t)gz * L + gy) * L + gx);
    }
  __syncthreads();
  const uint32_t slot = slot_of32(g, (uint32_t)lat);
  const uint32_t thr4 = __ldg(thr + 4 * slot + 1), thr8 = __ldg(thr + 4 * slot + 2),
                 thr12 = __ldg(thr + 4 * slot + 3);
  const uint32_t lid = lattice_id32(g, (uint32_t)lat);
  const uint32_t row_chunks = (uint32_t)L >> 3;
  // a thread keeps the same kPer chunks for all hits: the sweep-independent
  // part of the first Philox rounds is computed once (PhiloxX1)
  PhiloxX1 pre[kPer][2];
  if (active)
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
      const int q = tid + i * kTPT;
      const int m = q % kCpr, ty = (q / kCpr) % kT, tz = q / (kCpr * kT);
      const uint32_t gchunk =
          ((uint32_t)(z0 + tz) * (uint32_t)L + (uint32_t)(y0 + ty)) * row_chunks + (uint32_t)(x0 >> 3) + (uint32_t)m;
#pragma unroll
      for (int c = 0; c < 2; ++c) pre[i][c] = philox_x1_setup(gchunk, lid, ctr_w(TAG_UPDATE, (uint32_t)c, 0), rk);
    }
  for (int h = 0; h < k; ++h) {
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      if (active)
#pragma unroll
        for (int i = 0; i < kPer; ++i) {
          const int q = tid + i * kTPT;
          const int m = q % kCpr, ty = (q / kCpr) % kT, tz = q / (kCpr * kT);
          const int row = (tz + 1) * kSide + ty + 1, word = m + 1;
          const int at = row * kWords + word;
          const uint64_t C = sw[at];
          const uint64_t U = sw[at - kWords], D = sw[at + kWords];
          const uint64_t F = sw[at - kSide * kWords], Bk = sw[at + kSide * kWords];
          const int p = (c + y0 + ty + z0 + tz) & 1;
          const uint32_t edge = p ? sb[at * 8 + 8] : sb[at * 8 - 1];
          const uint4 r = philox_x1(pre[i][c], sweep0 + (uint32_t)h, rk);
          sw[at] = ising3d_chunk(C, U, D, F, Bk, edge, r, p, thr4, thr8, thr12);
        }
      __syncthreads();
    }
  }
  if (active)
    for (int q = tid; q < kChunks; q += kTPT) {
      const int m = q % kCpr, ty = (q / kCpr) % kT, tz = q / (kCpr * kT);
      *reinterpret_cast<uint64_t *>(base + ((int64_t)(z0 + tz) * L + (y0 + ty)) * L + x0 + 8 * m) =
          sw[((tz + 1) * kSide + ty + 1) * kWords + m + 1];
    }
}

template <int kT>
cudaError_t launch_tiles3(spin_lattice *h, int coarse, uint32_t sweep0) {
  constexpr int kChunks = kT * kT * (kT / 8);
  constexpr int kTiles = kChunks < 256 ? 256 / kChunks : 1;
  const int64_t B = h->g.L / kT;
  const int64_t n_tiles = B * B * B / 2;
  dim3 grid((unsigned)((n_tiles + kTiles - 1) / kTiles), (unsigned)h->n_lat);
  dcb3_tile_kernel<kT><<<grid, 256, 0, h->stream>>>((int8_t *)h->spins, h->g.L, coarse, sweep0, h->order_hits,
                                                     h->d_thr, h->g, make_round_keys(h->d.seed));
  return cudaGetLastError();
}

}  // namespace

bool dcb_supported(const spin_lattice *h, int tile) {
  if (h->n_lat > 65535) return false;
  if (h->d.model == SPIN_HEISENBERG)  // 2D, T x T tiles of float4 in shared memory
    return h->d.dim == 2 && (tile == 8 || tile == 16 || tile == 32) && h->g.L % tile == 0 &&
           ((h->g.L / tile) & 1) == 0;
  if (h->d.model != SPIN_ISING || h->d.layout != SPIN_I8) return false;
  if (h->d.dim == 2) {
    if (tile != 8 && tile != 16 && tile != 32 && tile != 64 && tile != 128) return false;
  } else if (h->d.dim == 3) {
    if (tile != 8 && tile != 16) return false;
  } else {
    return false;
  }
  return h->g.L % tile == 0 && ((h->g.L / tile) & 1) == 0;
}

// n_sweeps / k compound moves (the caller has checked that k divides both
// n_sweeps and the handle's sweep count).
cudaError_t launch_sweeps_dcb(spin_lattice *h, int64_t n_sweeps) {
  const int k = h->order_hits;
  for (int64_t mv = 0; mv < n_sweeps / k; ++mv) {
    const uint32_t M = (uint32_t)(h->sweeps_done / k + mv);
    const int first = (h->order == SPIN_ORDER_DCB_SYMMETRIC && (M & 1u)) ? 1 : 0;
    for (int cc = 0; cc < 2; ++cc) {
      const int coarse = first ^ cc;
      const uint32_t sweep0 = M * (uint32_t)k;
      cudaError_t e;
      if (h->d.model == SPIN_HEISENBERG) {
        e = launch_heis_dcb_tiles(h, coarse, sweep0);
      } else if (h->g.dim == 3) {
        e = h->order_tile == 8 ? launch_tiles3<8>(h, coarse, sweep0) : launch_tiles3<16>(h, coarse, sweep0);
      } else {
        switch (h->order_tile) {
          case 8: e = launch_tiles<8>(h, coarse, sweep0); break;
          case 16: e = launch_tiles<16>(h, coarse, sweep0); break;
          case 32: e = launch_tiles<32>(h, coarse, sweep0); break;
          case 64: e = launch_tiles<64>(h, coarse, sweep0); break;
          default: e = launch_tiles<128>(h, coarse, sweep0); break;
        }
      }
      if (e != cudaSuccess) return e;
    }
    // Heisenberg: renormalise after a compound move that passed a sweep
    // count (1-based) divisible by 100, the rule of the plain sweeps
    const uint64_t before = (uint64_t)M * (uint64_t)k, after = before + (uint64_t)k;
    if (h->d.model == SPIN_HEISENBERG && after / 100u > before / 100u) {
      const cudaError_t e = launch_heis_renorm(h);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

}  // namespace spin
