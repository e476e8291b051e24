// Heisenberg model (Eq. On_hamiltonian, n = 3) on the cubic lattice and, as
// in the paper's own study (Sec. 4), the square lattice, with FP32 unit
// vectors stored as float4 (x, y, z, 0): hot start, checkerboard Metropolis
// sweep with a uniformly drawn new direction (Sec. 4), renormalisation.
#include "heis_step.cuh"
#include "internal.h"

namespace spin {
namespace {

__global__ void heis_init_kernel(float4 *__restrict__ s, Geom g, int64_t n_lat, RoundKeys rk) {
  const int64_t total = n_lat * g.N;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t lat = k / g.N, i = k - lat * g.N;
    const uint4 w = philox(make_uint4((uint32_t)i, 0u, lattice_id_of(g, lat), ctr_w(TAG_HEIS_INIT, 0, 0)), rk);
    s[k] = unit_vector<false>(w.x, w.y);
  }
}

__global__ void heis_cold_kernel(float4 *__restrict__ s, int64_t total) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
       k += (int64_t)gridDim.x * blockDim.x)
    s[k] = make_float4(0.0f, 0.0f, 1.0f, 0.0f);
}

// One colour phase.  Thread per colour site j (site i = 2j + parity); one
// Philox call per site: words 0, 1 give the proposal, word 2 the acceptance
// uniform.  dE = -(n - s) . h with h the sum of the 2 kDim neighbour spins;
// accept iff dE <= 0 or u3 < exp(-beta dE).  beta (float) is read from
// word 0 of the slot's row of the threshold table.
template <bool kFast, int kDim>
__global__ void __launch_bounds__(256) heis_phase_kernel(float4 *__restrict__ s, Geom g,
                                                         uint32_t total,
                                                         const uint32_t *__restrict__ thr,
                                                         RoundKeys rk, uint32_t sweep,
                                                         int colour) {
  griddep_wait();
  griddep_release();
  const uint32_t L = (uint32_t)g.L, LL = L * L, N = (uint32_t)g.N, half = N / 2;
  const bool single = g.n_real == 1 && g.n_temps == 1 && g.n_sets == 1;
  const float beta0 = __uint_as_float(__ldg(thr)), bl0 = __uint_as_float(__ldg(thr + 1));
  const uint32_t wctr = ctr_w(TAG_HEIS, (uint32_t)colour, 0);
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < total; k += gridDim.x * blockDim.x) {
    uint32_t lat = 0, j = k, lid = 0;
    float beta = beta0, bl = bl0;
    if (!single) {
      lat = fdiv(k, g.fhalf);
      j = k - lat * half;
      lid = lattice_id32(g, lat);
      const uint32_t slot = slot_of32(g, lat);
      beta = __uint_as_float(__ldg(thr + 4 * slot));
      bl = __uint_as_float(__ldg(thr + 4 * slot + 1));
    }
    float4 *sl = s + (size_t)lat * N;
    const Site st = site_of(g, j, colour);
    const uint32_t i = st.i;
    const uint32_t ixp = st.rowbase + (st.x == L - 1 ? 0 : st.x + 1);
    const uint32_t ixm = st.rowbase + (st.x == 0 ? L - 1 : st.x - 1);
    const uint32_t iyp = st.y == L - 1 ? i - (L - 1) * L : i + L;
    const uint32_t iym = st.y == 0 ? i + (L - 1) * L : i - L;
    // (kDim is a compile-time constant: the 2D form drops the z terms)
    const uint32_t izp = kDim == 3 ? (st.z == L - 1 ? i - (L - 1) * LL : i + LL) : i;
    const uint32_t izm = kDim == 3 ? (st.z == 0 ? i + (L - 1) * LL : i - LL) : i;
    const float4 zero = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    const float4 a = sl[ixp], b = sl[ixm], c = sl[iyp], d = sl[iym], e = kDim == 3 ? sl[izp] : zero,
                 f = kDim == 3 ? sl[izm] : zero;
    const float4 si = sl[i];
    const uint4 w = philox(make_uint4(j, sweep, lid, wctr), rk);
    const float hx = kDim == 3 ? a.x + b.x + c.x + d.x + e.x + f.x : a.x + b.x + c.x + d.x;
    const float hy = kDim == 3 ? a.y + b.y + c.y + d.y + e.y + f.y : a.y + b.y + c.y + d.y;
    const float hz = kDim == 3 ? a.z + b.z + c.z + d.z + e.z + f.z : a.z + b.z + c.z + d.z;
    float4 n;
    if (heis_step<kFast>(si, hx, hy, hz, w, beta, bl, n)) sl[i] = n;
  }
}

// Colour-split working copy of the lattices for the long calls: per lattice
// [2 colours][L^(dim-1) rows][L/2], the site (x, row) of colour c at
// c N/2 + row L/2 + (x >> 1), i.e. at c N/2 + (i >> 1).  A warp's 32
// consecutive sites of one colour then read 32 consecutive float4 of the
// other colour for each neighbour direction instead of every other float4
// of two cache lines.
__global__ void heis_to_split_kernel(const float4 *__restrict__ s, float4 *__restrict__ S, Geom g, int64_t total) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t lat = k / g.N, i = k - lat * g.N;
    S[lat * g.N + (int64_t)colour_of(g, (uint32_t)i) * (g.N / 2) + (i >> 1)] = s[k];
  }
}

__global__ void heis_from_split_kernel(const float4 *__restrict__ S, float4 *__restrict__ s, Geom g, int64_t total) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t lat = k / g.N, i = k - lat * g.N;
    s[k] = S[lat * g.N + (int64_t)colour_of(g, (uint32_t)i) * (g.N / 2) + (i >> 1)];
  }
}

// One colour phase on the colour-split copy: thread per colour site j (the
// Philox index, j = row L/2 + kx); the neighbours x +- 1 are the other
// colour's entries kx and kx +- 1 of the same row (which one is x + 1
// depends on the row's parity p), y +- 1 and z +- 1 the entries kx of the
// neighbouring rows.  Same arithmetic as heis_phase_kernel, site for site.
template <bool kFast, int kDim>
__global__ void __launch_bounds__(256) heis_split_phase_kernel(float4 *__restrict__ S, Geom g, uint32_t total,
                                                               const uint32_t *__restrict__ thr, RoundKeys rk,
                                                               uint32_t sweep, int colour) {
  griddep_wait();
  griddep_release();
  const uint32_t L = (uint32_t)g.L, H = L >> 1, half = (uint32_t)(g.N / 2);
  const bool single = g.n_real == 1 && g.n_temps == 1 && g.n_sets == 1;
  const float beta0 = __uint_as_float(__ldg(thr)), bl0 = __uint_as_float(__ldg(thr + 1));
  const uint32_t wctr = ctr_w(TAG_HEIS, (uint32_t)colour, 0);
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < total; k += gridDim.x * blockDim.x) {
    uint32_t lat = 0, j = k, lid = 0;
    float beta = beta0, bl = bl0;
    if (!single) {
      lat = fdiv(k, g.fhalf);
      j = k - lat * half;
      lid = lattice_id32(g, lat);
      const uint32_t slot = slot_of32(g, lat);
      beta = __uint_as_float(__ldg(thr + 4 * slot));
      bl = __uint_as_float(__ldg(thr + 4 * slot + 1));
    }
    const uint32_t row = fdiv(j, g.fHalfL), kx = j - row * H;
    uint32_t y = row, z = 0;
    if (kDim == 3) {
      z = fdiv(row, g.fL);
      y = row - z * L;
    }
    const uint32_t p = (colour + y + z) & 1u;
    float4 *own = S + (size_t)lat * g.N + (colour ? half : 0) + j;
    const float4 *O = S + (size_t)lat * g.N + (colour ? 0 : half) + j;
    const int dr = p ? (kx == H - 1 ? 1 - (int)H : 1) : (kx == 0 ? (int)H - 1 : -1);
    const int dyp = y == L - 1 ? -(int)((L - 1) * H) : (int)H, dym = y == 0 ? (int)((L - 1) * H) : -(int)H;
    const float4 m = O[0], sh = O[dr];
    const float4 a = p ? sh : m, b = p ? m : sh;  // x + 1, x - 1
    const float4 c = O[dyp], d = O[dym];
    float hx, hy, hz;
    if (kDim == 3) {
      const int LH = (int)(L * H);
      const int dzp = z == L - 1 ? -(int)((L - 1) * L * H) : LH, dzm = z == 0 ? (int)((L - 1) * L * H) : -LH;
      const float4 e = O[dzp], f = O[dzm];
      hx = a.x + b.x + c.x + d.x + e.x + f.x;
      hy = a.y + b.y + c.y + d.y + e.y + f.y;
      hz = a.z + b.z + c.z + d.z + e.z + f.z;
    } else {
      hx = a.x + b.x + c.x + d.x;
      hy = a.y + b.y + c.y + d.y;
      hz = a.z + b.z + c.z + d.z;
    }
    const float4 si = *own;
    const uint4 w = philox(make_uint4(j, sweep, lid, wctr), rk);
    float4 n;
    if (heis_step<kFast>(si, hx, hy, hz, w, beta, bl, n)) *own = n;
  }
}

// Double checkerboard with multi-hit updates for the 2D model (Sec. 4 runs
// its GPU code this way; tiles and hits as Sec. 3.2, 3.4): one launch takes
// every T x T tile of one coarse colour into shared memory with a one-site
// halo (from tiles of the other colour, unchanged by this launch) and gives
// it k hits, each updating the fine colour-0 and then the fine colour-1
// sites; hit h of compound move m draws with sweep number m k + h.  Each
// update is the arithmetic of heis_phase_kernel, in the same order.
template <int kT, bool kFast>
__global__ void __launch_bounds__(256) heis_dcb2_kernel(float4 *__restrict__ s, Geom g, int coarse,
                                                        uint32_t sweep0, int k, const uint32_t *__restrict__ thr,
                                                        RoundKeys rk) {
  constexpr int kSide = kT + 2;
  constexpr int kTileV = kSide * kSide;   // float4 per shared tile
  constexpr int kPairs = kT * kT / 2;     // sites per fine colour per tile
  constexpr int kTPT = kPairs < 256 ? kPairs : 256;
  constexpr int kTiles = 256 / kTPT;
  constexpr int kPer = kPairs / kTPT;
  __shared__ float4 sm[kTiles * kTileV];
  const int tsub = threadIdx.x / kTPT, tid = threadIdx.x - tsub * kTPT;
  float4 *sw = sm + tsub * kTileV;
  const int L = g.L, B = L / kT, half = B >> 1;
  const int t = blockIdx.x * kTiles + tsub;
  const bool active = t < B * half;
  const int by = t / half, bx = 2 * (t % half) + ((by + coarse) & 1);
  const uint32_t lat = blockIdx.y;
  float4 *sl = s + (int64_t)lat * L * L;
  const int x0 = bx * kT, y0 = by * kT;
  if (active)
    for (int q = tid; q < kTileV; q += kTPT) {
      const int ry = q / kSide - 1, rx = q % kSide - 1;
      const int gy = (y0 + ry + L) % L, gx = (x0 + rx + L) % L;
      sw[q] = sl[(int64_t)gy * L + gx];
    }
  __syncthreads();
  const uint32_t slot = slot_of32(g, lat), lid = lattice_id32(g, lat);
  const float beta = __uint_as_float(__ldg(thr + 4 * slot)), bl = __uint_as_float(__ldg(thr + 4 * slot + 1));
  PhiloxX1 pre[kPer][2];
  if (active)
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
      const int q = tid + i * kTPT, ty = q / (kT / 2), xh = q % (kT / 2);
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int tx = 2 * xh + ((c + y0 + ty) & 1);
        const uint32_t j = (uint32_t)(((int64_t)(y0 + ty) * L + x0 + tx) >> 1);
        pre[i][c] = philox_x1_setup(j, lid, ctr_w(TAG_HEIS, (uint32_t)c, 0), rk);
      }
    }
  for (int h = 0; h < k; ++h) {
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      if (active)
#pragma unroll
        for (int i = 0; i < kPer; ++i) {
          const int q = tid + i * kTPT, ty = q / (kT / 2), xh = q % (kT / 2);
          const int tx = 2 * xh + ((c + y0 + ty) & 1);
          const int at = (ty + 1) * kSide + tx + 1;
          const float4 a = sw[at + 1], b = sw[at - 1], cc = sw[at + kSide], d = sw[at - kSide];
          const float4 si = sw[at];
          const uint4 w = philox_x1(pre[i][c], sweep0 + (uint32_t)h, rk);
          const float hx = a.x + b.x + cc.x + d.x;
          const float hy = a.y + b.y + cc.y + d.y;
          const float hz = a.z + b.z + cc.z + d.z;
          float4 n;
          if (heis_step<kFast>(si, hx, hy, hz, w, beta, bl, n)) sw[at] = n;
        }
      __syncthreads();
    }
  }
  if (active)
    for (int q = tid; q < kT * kT; q += kTPT) {
      const int ty = q / kT, tx = q % kT;
      sl[(int64_t)(y0 + ty) * L + x0 + tx] = sw[(ty + 1) * kSide + tx + 1];
    }
}

template <int kT>
cudaError_t launch_heis_tiles(spin_lattice *h, int coarse, uint32_t sweep0) {
  constexpr int kPairs = kT * kT / 2;
  constexpr int kTiles = kPairs < 256 ? 256 / kPairs : 1;
  const int B = h->g.L / kT;
  const int n_tiles = B * B / 2;
  dim3 grid((unsigned)((n_tiles + kTiles - 1) / kTiles), (unsigned)h->n_lat);
  const RoundKeys rk = make_round_keys(h->d.seed);
  if (h->variant == 2)
    heis_dcb2_kernel<kT, true><<<grid, 256, 0, h->stream>>>((float4 *)h->spins, h->g, coarse, sweep0,
                                                             h->order_hits, h->d_thr, rk);
  else
    heis_dcb2_kernel<kT, false><<<grid, 256, 0, h->stream>>>((float4 *)h->spins, h->g, coarse, sweep0,
                                                              h->order_hits, h->d_thr, rk);
  return cudaGetLastError();
}

// s <- s / |s| with IEEE sqrt and division.
__global__ void heis_renorm_kernel(float4 *__restrict__ s, int64_t total) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
       k += (int64_t)gridDim.x * blockDim.x) {
    float4 v = s[k];
    const float r = __fsqrt_rn(v.x * v.x + v.y * v.y + v.z * v.z);
    v.x = __fdiv_rn(v.x, r);
    v.y = __fdiv_rn(v.y, r);
    v.z = __fdiv_rn(v.z, r);
    s[k] = v;
  }
}

unsigned capped_grid(int64_t n) {
  unsigned g = grid_for(n, 256);
  return g > (1u << 20) ? (1u << 20) : g;
}

}  // namespace

cudaError_t launch_init_heis(spin_lattice *h) {
  const int64_t total = h->n_lat * h->g.N;
  if (h->d.hot_start)
    heis_init_kernel<<<capped_grid(total), 256, 0, h->stream>>>((float4 *)h->spins, h->g, h->n_lat,
                                                                  make_round_keys(h->d.seed));
  else
    heis_cold_kernel<<<capped_grid(total), 256, 0, h->stream>>>((float4 *)h->spins, total);
  return cudaGetLastError();
}

namespace {
// Calls of at least this many sweeps in the fast-math variant run on the
// colour-split copy (the two conversions cost about one sweep's memory
// traffic).  Measured on the L = 128 and 256 lattices: +6-7 % for the
// fast-math form, none for the full-accuracy form, which stays on the
// row-major kernel.
constexpr int64_t kSplitMinSweeps = 4;

cudaError_t sweeps_heis_split(spin_lattice *h, int64_t n_sweeps) {
  const int64_t total = h->n_lat * h->g.N;
  const size_t bytes = (size_t)total * 16;
  if (!h->d_pingpong || h->pingpong_bytes < bytes) {
    if (h->d_pingpong) cudaFree(h->d_pingpong);
    h->d_pingpong = nullptr;
    cudaError_t e = cudaMalloc(&h->d_pingpong, bytes);
    if (e != cudaSuccess) return e;
    h->pingpong_bytes = bytes;
  }
  float4 *S = (float4 *)h->d_pingpong;
  heis_to_split_kernel<<<capped_grid(total), 256, 0, h->stream>>>((const float4 *)h->spins, S, h->g, total);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const RoundKeys rk = make_round_keys(h->d.seed);
  const uint32_t half = (uint32_t)(total / 2);
  auto *kern = h->g.dim == 3 ? (h->variant == 2 ? heis_split_phase_kernel<true, 3> : heis_split_phase_kernel<false, 3>)
                             : (h->variant == 2 ? heis_split_phase_kernel<true, 2> : heis_split_phase_kernel<false, 2>);
  for (int64_t k = 0; k < n_sweeps; ++k) {
    const uint32_t sweep = (uint32_t)(h->sweeps_done + k);
    for (int colour = 0; colour < 2; ++colour) {
      e = launch_dependent(kern, dim3(capped_grid(half)), dim3(256), 0, h->stream, S, h->g, half, h->d_thr, rk,
                           sweep, colour);
      if (e != cudaSuccess) return e;
    }
    if ((sweep + 1u) % 100u == 0u) {  // renormalisation is site-wise: the layout does not matter
      heis_renorm_kernel<<<capped_grid(total), 256, 0, h->stream>>>(S, total);
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
  }
  heis_from_split_kernel<<<capped_grid(total), 256, 0, h->stream>>>(S, (float4 *)h->spins, h->g, total);
  return cudaGetLastError();
}


// Calls of at least this many sweeps of a 3D lattice that fits run resident
// in shared memory (heis_res.cu); the launch loads and stores the lattices
// once, about a quarter of one sweep's time at L = 128.
constexpr int64_t kResidentMinSweeps = 4;

// The resident sweeps, split at the renormalisation sweeps (every 100th,
// applied to the row-major lattices between two launches).
cudaError_t sweeps_heis_resident(spin_lattice *h, const HeisResPlan &plan, int64_t n_sweeps, int64_t &done) {
  done = 0;
  while (done < n_sweeps) {
    const int64_t s0 = h->sweeps_done + done;
    const int64_t to_renorm = 100 - s0 % 100;  // sweeps up to and including the next renormalised one
    const int64_t n = n_sweeps - done < to_renorm ? n_sweeps - done : to_renorm;
    cudaError_t e = launch_sweeps_heis_resident(h, plan, s0, n);
    if (e != cudaSuccess) return e;
    if (n == to_renorm) {
      heis_renorm_kernel<<<capped_grid(h->n_lat * h->g.N), 256, 0, h->stream>>>((float4 *)h->spins,
                                                                               h->n_lat * h->g.N);
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
    done += n;
  }
  return cudaSuccess;
}
}  // namespace

cudaError_t launch_sweeps_heis(spin_lattice *h, int64_t n_sweeps) {
  // Inside a stream capture only the per-phase kernels: they allocate
  // nothing, and a replayed graph must not meet the resident kernel's
  // published-phase counters already advanced by an earlier replay.
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(h->stream, &cs) != cudaSuccess) return cudaGetLastError();
  const bool capturing = cs != cudaStreamCaptureStatusNone;
  if (!capturing && n_sweeps >= kResidentMinSweeps) {
    const int v = h->variant == 2 ? 1 : 0;
    if (h->res_plan_state[v] == 0) h->res_plan_state[v] = heis_resident_plan(h, &h->res_plan[v]) ? 1 : -1;
    if (h->res_plan_state[v] == 1) {
      int64_t done = 0;
      cudaError_t e = sweeps_heis_resident(h, h->res_plan[v], n_sweeps, done);
      if (e != cudaErrorCooperativeLaunchTooLarge) return e;
      // The GPU cannot hold every CTA at once (its SMs shared with other
      // work): the refused launch ran nothing, and this handle takes the
      // other paths from here on, from the first sweep not yet done.
      cudaGetLastError();
      h->res_plan_state[v] = -1;
      h->sweeps_done += done;
      e = launch_sweeps_heis(h, n_sweeps - done);
      h->sweeps_done -= done;
      return e;
    }
  }
  if (!capturing && h->variant == 2 && n_sweeps >= kSplitMinSweeps && h->n_lat * h->g.N < ((int64_t)1 << 32))
    return sweeps_heis_split(h, n_sweeps);
  const RoundKeys rk = make_round_keys(h->d.seed);
  const uint32_t half = (uint32_t)(h->n_lat * (h->g.N / 2));
  for (int64_t k = 0; k < n_sweeps; ++k) {
    const uint32_t sweep = (uint32_t)(h->sweeps_done + k);
    for (int colour = 0; colour < 2; ++colour) {
      float4 *sp = (float4 *)h->spins;
      auto *k = h->g.dim == 3 ? (h->variant == 2 ? heis_phase_kernel<true, 3> : heis_phase_kernel<false, 3>)
                              : (h->variant == 2 ? heis_phase_kernel<true, 2> : heis_phase_kernel<false, 2>);
      const cudaError_t le = launch_dependent(k, dim3(capped_grid(half)), dim3(256), 0, h->stream, sp, h->g, half,
                                              h->d_thr, rk, sweep, colour);
      if (le != cudaSuccess) return le;
    }
    if ((sweep + 1u) % 100u == 0u)
      heis_renorm_kernel<<<capped_grid(h->n_lat * h->g.N), 256, 0, h->stream>>>(
          (float4 *)h->spins, h->n_lat * h->g.N);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// One double-checkerboard launch of the 2D model: the tiles of coarse
// colour `coarse` through the handle's hits, starting at sweep0.
cudaError_t launch_heis_dcb_tiles(spin_lattice *h, int coarse, uint32_t sweep0) {
  switch (h->order_tile) {
    case 8: return launch_heis_tiles<8>(h, coarse, sweep0);
    case 16: return launch_heis_tiles<16>(h, coarse, sweep0);
    default: return launch_heis_tiles<32>(h, coarse, sweep0);
  }
}

cudaError_t launch_heis_renorm(spin_lattice *h) {
  heis_renorm_kernel<<<capped_grid(h->n_lat * h->g.N), 256, 0, h->stream>>>((float4 *)h->spins,
                                                                           h->n_lat * h->g.N);
  return cudaGetLastError();
}

}  // namespace spin
