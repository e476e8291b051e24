// Ising ferromagnet and +-J EA glass with one int8 (+-1) per spin:
// initialisation, couplings and the checkerboard Metropolis sweep
// (Sec. 3.2, Eq. metropolis, Eq. spinglass_hamiltonian).
#include "i8chunk.cuh"
#include "internal.h"

namespace spin {
namespace {

// ---------------------------------------------------------------- init
// Hot start: s_i = -1 iff bit `bit` of the INIT word of site i is set, with
// bit = r & 31 for EA lattices (the group's word is shared by its 32
// realisations) and 0 otherwise.  One Philox call covers four sites.
__global__ void init_i8_kernel(int8_t *__restrict__ spins, Geom g, int64_t n_lat, RoundKeys rk) {
  const int64_t quads = (g.N + 3) / 4;
  const int64_t total = n_lat * quads;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t lat = k / quads, q4 = k - lat * quads;
    const uint32_t bit = g.ea ? (uint32_t)(lat % g.n_real) & 31u : 0u;
    const uint4 w = philox(make_uint4((uint32_t)q4, 0u, lattice_id_of(g, lat), ctr_w(TAG_INIT, 0, 0)), rk);
    int8_t *s = spins + lat * g.N;
#pragma unroll
    for (uint32_t q = 0; q < 4; ++q) {
      const int64_t i = 4 * q4 + q;
      if (i < g.N) s[i] = ((word_of(w, q) >> bit) & 1u) ? (int8_t)-1 : (int8_t)1;
    }
  }
}

// Bimodal couplings (Eq. spinglass_hamiltonian): J[r][d][i] = -1 iff bit
// r & 31 of the COUPLING word of (group r >> 5, direction d, site i) is set.
__global__ void couplings_i8_kernel(int8_t *__restrict__ J, Geom g, RoundKeys rk) {
  const int64_t quads = (g.N + 3) / 4;
  const int64_t total = (int64_t)g.n_real * g.dim * quads;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t rd = k / quads, q4 = k - rd * quads;
    const int r = (int)(rd / g.dim), d = (int)(rd % g.dim);
    const uint4 w = philox(make_uint4((uint32_t)q4, 0u, lattice_id(0, (uint32_t)r >> 5, 0),
                                      ctr_w(TAG_COUPLING, 0, (uint32_t)d)), rk);
    int8_t *out = J + rd * g.N;
#pragma unroll
    for (uint32_t q = 0; q < 4; ++q) {
      const int64_t i = 4 * q4 + q;
      if (i < g.N) out[i] = ((word_of(w, q) >> (r & 31)) & 1u) ? (int8_t)-1 : (int8_t)1;
    }
  }
}

// ---------------------------------------------------------------- 2D phase, L % 8 == 0
// One thread owns eight consecutive bytes of a row (x = 8m .. 8m+7): the
// four sites of the active colour among them draw their uniforms from one
// Philox call (their colour indices j = yL/2 + 4m + q share j >> 2); the
// update itself is ising_chunk (byte-wise neighbour counts, dE = 8 - 4n).
__global__ void __launch_bounds__(256) ising2d_phase_kernel(int8_t *__restrict__ spins, int L,
                                                            const uint32_t *__restrict__ thr,
                                                            Geom g, RoundKeys rk, uint32_t sweep,
                                                            int colour) {
  griddep_wait();
  griddep_release();
  const int chunks = L >> 3;
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int64_t lat = blockIdx.z;
  if (m >= chunks || y >= L) return;
  int8_t *base = spins + lat * (int64_t)L * L;
  const int yu = y == 0 ? L - 1 : y - 1, yd = y == L - 1 ? 0 : y + 1;
  const uint64_t *row = reinterpret_cast<const uint64_t *>(base + (int64_t)y * L);
  const uint64_t C = row[m];
  const uint64_t U = reinterpret_cast<const uint64_t *>(base + (int64_t)yu * L)[m];
  const uint64_t D = reinterpret_cast<const uint64_t *>(base + (int64_t)yd * L)[m];
  // only the byte beyond the chunk on the side the phase needs is read
  const int p = (colour + y) & 1;
  const int xe = p ? (m == chunks - 1 ? 0 : 8 * m + 8) : (m == 0 ? L - 1 : 8 * m - 1);
  const uint64_t lb = (uint8_t)base[(int64_t)y * L + xe], rb = lb;
  const uint32_t t = slot_of32(g, (uint32_t)lat);
  const uint32_t thr4 = __ldg(thr + 4 * t + 1), thr8 = __ldg(thr + 4 * t + 2);
  const uint32_t j4 = (uint32_t)y * (uint32_t)chunks + (uint32_t)m;
  const uint4 r = philox(make_uint4(j4, sweep, lattice_id32(g, (uint32_t)lat), ctr_w(TAG_UPDATE, colour, 0)), rk);
  long long unused_a = 0, unused_d = 0;
  reinterpret_cast<uint64_t *>(base + (int64_t)y * L)[m] =
      ising_chunk<0>(C, U, D, lb, rb, r, p, thr4, thr8, unused_a, unused_d);
}

// ---------------------------------------------------------------- 2D resident, small L
// Small lattices (L % 8 == 0, L <= kResidentMaxL): one CTA keeps a whole
// lattice in shared memory and runs every sweep of the call on it, the two
// colour phases separated by a CTA barrier, then writes it back.  Each
// chunk update is ising2d_phase_kernel's (same chunks, same Philox
// counters), so n sweeps give the lattice of 2n phase launches; lattices
// (replicas) map to CTAs, as the paper's tempering code maps replicas to
// thread blocks (Sec. 6).  Grid: one CTA per lattice; shared memory L^2
// bytes.  With E or M the kernel also measures after the sweeps s (0-based
// in the launch) with s + 1 = first + j * every, j = 0, 1, ...: row j of E
// and M (n_lat entries each) gets E = 2 anti - 2 N and M = N - 2 down of
// every lattice, the counts of antiparallel bonds (right and down of each
// site) and of down spins.
// Adds the CTA's counts of antiparallel bonds and down spins and stores
// E = 2 anti - bonds and M = sites - 2 down at E[at], M[at].
__device__ __forceinline__ void resident_put(int anti, int down, int (*red)[2], long long *E, long long *M,
                                             int64_t at, long long sites, long long bonds) {
  anti = __reduce_add_sync(0xffffffffu, anti);
  down = __reduce_add_sync(0xffffffffu, down);
  if ((threadIdx.x & 31) == 0) {
    red[threadIdx.x >> 5][0] = anti;
    red[threadIdx.x >> 5][1] = down;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    long long a = 0, d = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a += red[w][0], d += red[w][1];
    if (E) E[at] = 2 * a - bonds;
    if (M) M[at] = sites - 2 * d;
  }
  // the next measurement rewrites red only after the next sweep's barriers
}

// kPer: chunks per thread (total chunks <= 512 kPer).  A thread's chunks,
// their neighbour chunks and edge bytes, and (for kPer <= 2, where the
// registers allow) the part of each Philox call that does not depend on the
// sweep (PhiloxX1) are set up once per launch.
template <int kPer>
__global__ void __launch_bounds__(512) ising2d_resident_kernel(int8_t *__restrict__ spins, int L,
                                                               const uint32_t *__restrict__ thr, Geom g,
                                                               RoundKeys rk, uint32_t sweep0, int n_sweeps,
                                                               long long *__restrict__ E,
                                                               long long *__restrict__ M, int64_t n_lat,
                                                               int every, int first) {
  extern __shared__ __align__(16) uint8_t sl[];  // the lattice, row-major
  __shared__ int red[512 / 32][2];
  griddep_wait();
  griddep_release();
  const uint32_t lat = blockIdx.x;
  const int LL = L * L;
  int8_t *base = spins + (int64_t)lat * LL;
  for (int k = threadIdx.x; k < LL / 16; k += blockDim.x)
    reinterpret_cast<uint4 *>(sl)[k] = reinterpret_cast<const uint4 *>(base)[k];
  const int chunks = L >> 3, total = L * chunks;
  const uint32_t t = slot_of32(g, lat);
  const uint32_t thr4 = __ldg(thr + 4 * t + 1), thr8 = __ldg(thr + 4 * t + 2);
  const uint32_t lid = lattice_id32(g, lat);
  uint64_t *rows = reinterpret_cast<uint64_t *>(sl);
  constexpr bool kHoist = kPer <= 2;
  int ku[kPer], kd[kPer], kn[kPer], xe[kPer][2], py[kPer];  // kn: next chunk of the row
  PhiloxX1 pre[kPer][2];
#pragma unroll
  for (int i = 0; i < kPer; ++i) {
    const int k = threadIdx.x + i * blockDim.x;
    if (k >= total) break;
    const int y = k / chunks, m = k - y * chunks;
    const int yu = y == 0 ? L - 1 : y - 1, yd = y == L - 1 ? 0 : y + 1;
    ku[i] = yu * chunks + m;
    kd[i] = yd * chunks + m;
    kn[i] = y * chunks + (m == chunks - 1 ? 0 : m + 1);
    py[i] = y & 1;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      // only the byte beyond the chunk on the side the phase needs is read
      const int p = (c + y) & 1;
      xe[i][c] = y * L + (p ? (m == chunks - 1 ? 0 : 8 * m + 8) : (m == 0 ? L - 1 : 8 * m - 1));
      if (kHoist) pre[i][c] = philox_x1_setup((uint32_t)k, lid, ctr_w(TAG_UPDATE, (uint32_t)c, 0), rk);
    }
  }
  __syncthreads();
  for (int s = 0; s < n_sweeps; ++s) {
#pragma unroll
    for (int colour = 0; colour < 2; ++colour) {
#pragma unroll
      for (int i = 0; i < kPer; ++i) {
        const int k = threadIdx.x + i * blockDim.x;
        if (k >= total) break;
        const uint64_t C = rows[k], U = rows[ku[i]], D = rows[kd[i]];
        const uint64_t e = sl[xe[i][colour]];
        const uint4 r = kHoist ? philox_x1(pre[i][colour], sweep0 + (uint32_t)s, rk)
                               : philox(make_uint4((uint32_t)k, sweep0 + (uint32_t)s, lid,
                                                   ctr_w(TAG_UPDATE, (uint32_t)colour, 0)),
                                        rk);
        long long unused_a = 0, unused_d = 0;
        rows[k] = ising_chunk<0>(C, U, D, e, e, r, colour ^ py[i], thr4, thr8, unused_a, unused_d);
      }
      __syncthreads();
    }
    const int since = s + 1 - first;
    if ((E || M) && since >= 0 && since % every == 0) {
      // bit 1 of a +-1 byte is set for -1: (a ^ b) & 2 marks an antiparallel pair
      constexpr uint64_t kBit1 = 0x0202020202020202ull;
      int anti = 0, down = 0;
#pragma unroll
      for (int i = 0; i < kPer; ++i) {
        const int k = threadIdx.x + i * blockDim.x;
        if (k >= total) break;
        const uint64_t C = rows[k], D = rows[kd[i]], nx = rows[kn[i]];
        const uint64_t R = (C >> 8) | (nx << 56);  // right neighbours of the chunk's bytes
        anti += __popcll((C ^ R) & kBit1) + __popcll((C ^ D) & kBit1);
        down += __popcll(C & kBit1);
      }
      resident_put(anti, down, red, E, M, (int64_t)(since / every) * n_lat + lat, LL, 2 * (long long)LL);
    }
  }
  for (int k = threadIdx.x; k < LL / 16; k += blockDim.x)
    reinterpret_cast<uint4 *>(base)[k] = reinterpret_cast<const uint4 *>(sl)[k];
}

// The 3D form (L % 8 == 0, L <= kResident3MaxL, the cube in shared memory):
// chunk k = (z L + y) L / 8 + m is the chunk of ising3d_phase_kernel with the
// same Philox counter; its neighbours are the same chunk column's words in
// rows y -+ 1 and planes z -+ 1 and one edge byte (ising3d_chunk).  E counts
// the bonds to x + 1, y + 1 and z + 1 of every site (3 N bonds).
template <int kPer>
__global__ void __launch_bounds__(512) ising3d_resident_kernel(int8_t *__restrict__ spins, int L,
                                                               const uint32_t *__restrict__ thr, Geom g,
                                                               RoundKeys rk, uint32_t sweep0, int n_sweeps,
                                                               long long *__restrict__ E,
                                                               long long *__restrict__ M, int64_t n_lat,
                                                               int every, int first) {
  extern __shared__ __align__(16) uint8_t sl[];  // the cube, [z][y][x]
  __shared__ int red[512 / 32][2];
  griddep_wait();
  griddep_release();
  const uint32_t lat = blockIdx.x;
  const int LL = L * L, N = LL * L;
  int8_t *base = spins + (int64_t)lat * N;
  for (int k = threadIdx.x; k < N / 16; k += blockDim.x)
    reinterpret_cast<uint4 *>(sl)[k] = reinterpret_cast<const uint4 *>(base)[k];
  const int chunks = L >> 3, plane = L * chunks, total = L * plane;  // chunks per row, plane, cube
  const uint32_t t = slot_of32(g, lat);
  const uint32_t thr4 = __ldg(thr + 4 * t + 1), thr8 = __ldg(thr + 4 * t + 2), thr12 = __ldg(thr + 4 * t + 3);
  const uint32_t lid = lattice_id32(g, lat);
  uint64_t *w = reinterpret_cast<uint64_t *>(sl);
  // per chunk: rows y - 1, y + 1, planes z - 1, z + 1, the next chunk of the
  // row, the edge byte of each colour and the parity of y + z
  int ku[kPer], kd[kPer], kf[kPer], kb[kPer], kn[kPer], xe[kPer][2], pyz[kPer];
#pragma unroll
  for (int i = 0; i < kPer; ++i) {
    const int k = threadIdx.x + i * blockDim.x;
    if (k >= total) break;
    const int z = k / plane, r = k - z * plane, y = r / chunks, m = r - y * chunks;
    const int yu = y == 0 ? L - 1 : y - 1, yd = y == L - 1 ? 0 : y + 1;
    const int zf = z == 0 ? L - 1 : z - 1, zb = z == L - 1 ? 0 : z + 1;
    ku[i] = z * plane + yu * chunks + m;
    kd[i] = z * plane + yd * chunks + m;
    kf[i] = zf * plane + y * chunks + m;
    kb[i] = zb * plane + y * chunks + m;
    kn[i] = z * plane + y * chunks + (m == chunks - 1 ? 0 : m + 1);
    pyz[i] = (y + z) & 1;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      // only the byte beyond the chunk on the side the phase needs is read
      const int p = (c + y + z) & 1;
      xe[i][c] = z * LL + y * L + (p ? (m == chunks - 1 ? 0 : 8 * m + 8) : (m == 0 ? L - 1 : 8 * m - 1));
    }
  }
  __syncthreads();
  for (int s = 0; s < n_sweeps; ++s) {
#pragma unroll
    for (int colour = 0; colour < 2; ++colour) {
      const uint32_t wctr = ctr_w(TAG_UPDATE, (uint32_t)colour, 0);
#pragma unroll
      for (int i = 0; i < kPer; ++i) {
        const int k = threadIdx.x + i * blockDim.x;
        if (k >= total) break;
        const uint64_t C = w[k], U = w[ku[i]], D = w[kd[i]], F = w[kf[i]], Bk = w[kb[i]];
        const uint32_t edge = sl[xe[i][colour]];
        const uint4 r = philox(make_uint4((uint32_t)k, sweep0 + (uint32_t)s, lid, wctr), rk);
        w[k] = ising3d_chunk(C, U, D, F, Bk, edge, r, colour ^ pyz[i], thr4, thr8, thr12);
      }
      __syncthreads();
    }
    const int since = s + 1 - first;
    if ((E || M) && since >= 0 && since % every == 0) {
      constexpr uint64_t kBit1 = 0x0202020202020202ull;  // bit 1 of a +-1 byte: set for -1
      int anti = 0, down = 0;
#pragma unroll
      for (int i = 0; i < kPer; ++i) {
        const int k = threadIdx.x + i * blockDim.x;
        if (k >= total) break;
        const uint64_t C = w[k], R = (C >> 8) | (w[kn[i]] << 56);
        anti += __popcll((C ^ R) & kBit1) + __popcll((C ^ w[kd[i]]) & kBit1) + __popcll((C ^ w[kb[i]]) & kBit1);
        down += __popcll(C & kBit1);
      }
      resident_put(anti, down, red, E, M, (int64_t)(since / every) * n_lat + lat, N, 3 * (long long)N);
    }
  }
  for (int k = threadIdx.x; k < N / 16; k += blockDim.x)
    reinterpret_cast<uint4 *>(base)[k] = reinterpret_cast<const uint4 *>(sl)[k];
}

// ---------------------------------------------------------------- 3D phase, L % 8 == 0
// The 3D form of the 2D phase kernel: a thread owns the eight bytes
// x = 8m .. 8m+7 of row y in the planes z0 .. z0+zlen-1 and marches down z.
// The four active sites of a chunk have colour indices
// (z L^2 + y L + 8m) / 2 + q, q < 4, and share one Philox call
// (j4 = (z L^2 + y L) / 8 + m); the update is ising3d_chunk.  A site's
// neighbours are of the other colour, which the phase does not change, so
// the word of plane z - 1 kept from the previous step (before its update)
// serves as the lower neighbour and the word of plane z + 1 is loaded once
// for two steps.  A CTA takes blockDim.x chunks of blockDim.y rows; grid =
// (tiles of a plane, plane segments, lattices).
__global__ void __launch_bounds__(256) ising3d_phase_kernel(int8_t *__restrict__ spins, int L, int tiles_x,
                                                            int zlen, const uint32_t *__restrict__ thr, Geom g,
                                                            RoundKeys rk, uint32_t sweep, int colour) {
  griddep_wait();
  griddep_release();
  const int chunks = L >> 3;
  const int tile_y = blockIdx.x / tiles_x, tile_x = blockIdx.x - tile_y * tiles_x;
  const int m = tile_x * blockDim.x + threadIdx.x;
  const int y = tile_y * blockDim.y + threadIdx.y;
  const int z0 = blockIdx.y * zlen;
  const uint32_t lat = blockIdx.z;
  if (m >= chunks || y >= L || z0 >= L) return;
  const int z1 = min(z0 + zlen, L);
  const int64_t LL = (int64_t)L * L;
  int8_t *base = spins + (int64_t)lat * LL * L;
  uint64_t *col = reinterpret_cast<uint64_t *>(base + (int64_t)y * L) + m;  // word (z = 0, y, m)
  const int64_t zs = LL >> 3;                                               // words per plane
  const int64_t du = (int64_t)((y == 0 ? L - 1 : y - 1) - y) * (L >> 3);     // to row y - 1
  const int64_t dd = (int64_t)((y == L - 1 ? 0 : y + 1) - y) * (L >> 3);     // to row y + 1
  const uint32_t t = slot_of32(g, lat);
  const uint32_t thr4 = __ldg(thr + 4 * t + 1), thr8 = __ldg(thr + 4 * t + 2), thr12 = __ldg(thr + 4 * t + 3);
  const uint32_t lid = lattice_id32(g, lat), wctr = ctr_w(TAG_UPDATE, colour, 0);
  const int xl = m == 0 ? L - 1 : 8 * m - 1, xr = m == chunks - 1 ? 0 : 8 * m + 8;
  uint64_t F = col[(int64_t)(z0 == 0 ? L - 1 : z0 - 1) * zs];
  uint64_t *cz = col + (int64_t)z0 * zs;
  uint64_t C = *cz;
  // per step: the chunk moves one plane (zs words, L^2 bytes), its Philox
  // counter by L^2 / 8 and the active parity flips
  const uint8_t *row = reinterpret_cast<const uint8_t *>(base) + (int64_t)z0 * LL + (int64_t)y * L;
  uint32_t j4 = ((uint32_t)z0 * (uint32_t)L + (uint32_t)y) * (uint32_t)chunks + (uint32_t)m;
  const uint32_t dj = (uint32_t)L * (uint32_t)chunks;
  int p = (colour + y + z0) & 1;
  for (int z = z0; z < z1; ++z) {
    const uint64_t Bk = z == L - 1 ? col[0] : cz[zs];
    const uint64_t U = cz[du], D = cz[dd];
    const uint32_t edge = row[p ? xr : xl];
    const uint4 r = philox(make_uint4(j4, sweep, lid, wctr), rk);
    *cz = ising3d_chunk(C, U, D, F, Bk, edge, r, p, thr4, thr8, thr12);
    F = C;
    C = Bk;
    cz += zs;
    row += LL;
    j4 += dj;
    p ^= 1;
  }
}

// ---------------------------------------------------------------- generic phase
// Any even L, dim 2 or 3, ferromagnet (J == nullptr) or EA (J[r][d][i]).
// One thread takes four consecutive colour indices j = 4 j4 .. 4 j4 + 3 (one
// Philox call) and locates each site from its own coordinates.
__global__ void __launch_bounds__(256) phase_generic_kernel(int8_t *__restrict__ spins,
                                                            const int8_t *__restrict__ J,
                                                            const uint32_t *__restrict__ thr,
                                                            Geom g, uint32_t total, RoundKeys rk,
                                                            uint32_t sweep, int colour) {
  const uint32_t L = (uint32_t)g.L, LL = L * L, N = (uint32_t)g.N, half = N / 2;
  const uint32_t quads = (half + 3) / 4;
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < total; k += gridDim.x * blockDim.x) {
    const uint32_t lat = fdiv(k, g.fquads), j4 = k - lat * quads;
    int8_t *s = spins + (size_t)lat * N;
    const int8_t *Jr = J ? J + (size_t)(lat - fdiv(lat, g.freal) * (uint32_t)g.n_real) * g.dim * N : nullptr;
    const uint32_t t = slot_of32(g, lat);
    const uint4 r = philox(make_uint4(j4, sweep, lattice_id32(g, lat), ctr_w(TAG_UPDATE, colour, 0)), rk);
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
      int h;
      const int8_t sxp = s[ixp], sxm = s[ixm], syp = s[iyp], sym = s[iym];
      if (Jr) {
        h = Jr[i] * sxp + Jr[ixm] * sxm + Jr[N + i] * syp + Jr[N + iym] * sym;
      } else {
        h = sxp + sxm + syp + sym;
      }
      if (g.dim == 3) {
        const uint32_t izp = st.z == L - 1 ? i - (L - 1) * LL : i + LL;
        const uint32_t izm = st.z == 0 ? i + (L - 1) * LL : i - LL;
        if (Jr)
          h += Jr[2 * N + i] * s[izp] + Jr[2 * N + izm] * s[izm];
        else
          h += s[izp] + s[izm];
      }
      const int si = s[i];
      const int dE = 2 * si * h;
      const uint32_t rq = word_of(r, q);
      const bool flip = dE <= 0 || rq < __ldg(thr + 4 * t + (dE >> 2));
      if (flip) s[i] = (int8_t)(-si);
    }
  }
}

}  // namespace

cudaError_t launch_init_i8(spin_lattice *h) {
  if (!h->d.hot_start)
    return cudaMemsetAsync(h->spins, 1, (size_t)(h->n_lat * h->g.N), h->stream);
  const int64_t total = h->n_lat * ((h->g.N + 3) / 4);
  init_i8_kernel<<<grid_for(total, 256) > 65536u ? 65536u : grid_for(total, 256), 256, 0,
                   h->stream>>>((int8_t *)h->spins, h->g, h->n_lat, make_round_keys(h->d.seed));
  return cudaGetLastError();
}

cudaError_t launch_couplings_i8(spin_lattice *h) {
  const int64_t total = (int64_t)h->g.n_real * h->g.dim * ((h->g.N + 3) / 4);
  unsigned grid = grid_for(total, 256);
  if (grid > 65536u) grid = 65536u;
  couplings_i8_kernel<<<grid, 256, 0, h->stream>>>((int8_t *)h->couplings, h->g,
                                                    make_round_keys(h->d.seed));
  return cudaGetLastError();
}

cudaError_t launch_fused2d_i8(spin_lattice *h, int64_t n_sweeps);  // fused2d.cu
bool fused2d_supported(int L);                                     // fused2d.cu
cudaError_t launch_sweeps_i8_coded(spin_lattice *h, int64_t n_sweeps);  // msc2d.cu
bool coded_i8_supported(const spin_lattice *h);                         // msc2d.cu
// Calls of at least this many sweeps take the coded path (variant 4): the two
// transcoding passes cost about one sweep of HBM traffic, short calls take
// the fused pass instead.
constexpr int64_t kCodedMinSweeps = 4;

// Whole lattice in one CTA's shared memory: 16 KB at L = 128 in 2D, 13.5 KB
// at L = 24 in 3D (at most four chunks per thread, so that each thread's
// chunk geometry stays in registers).
bool resident_supported(int dim, int L) {
  return L % 8 == 0 && L >= 8 && L <= (dim == 2 ? kResidentMaxL : dim == 3 ? kResident3MaxL : 0);
}

cudaError_t launch_resident(spin_lattice *h, int64_t n_sweeps, int64_t *E, int64_t *M, int every, int first) {
  const Geom &g = h->g;
  const RoundKeys rk = make_round_keys(h->d.seed);
  const int64_t sites = g.N;
  const int chunks = (int)(sites / 8);
  const int threads = chunks < 512 ? (chunks + 31) / 32 * 32 : 512;
  using Kern = decltype(&ising2d_resident_kernel<1>);
  Kern kern;
  if (g.dim == 2)
    kern = chunks <= 512 ? ising2d_resident_kernel<1>
                         : (chunks <= 1024 ? ising2d_resident_kernel<2> : ising2d_resident_kernel<4>);
  else
    kern = chunks <= 512 ? ising3d_resident_kernel<1>
                         : (chunks <= 1024 ? ising3d_resident_kernel<2> : ising3d_resident_kernel<4>);
  // at most 4096 sweeps per launch, so that no launch runs for long; the
  // measurement rows continue from launch to launch
  for (int64_t done = 0; done < n_sweeps; done += 4096) {
    const int n = (int)(n_sweeps - done < 4096 ? n_sweeps - done : 4096);
    int64_t row = 0, f = first - done;  // f: first measured sweep, 1-based within this launch
    if (f < 1) {
      row = (done - first + every) / every;  // measurements before this launch
      f = first + row * every - done;
    }
    const cudaError_t e = launch_dependent(
        kern, dim3((unsigned)h->n_lat), dim3(threads), (size_t)sites, h->stream, (int8_t *)h->spins, g.L,
        (const uint32_t *)h->d_thr, g, rk, (uint32_t)(h->sweeps_done + done), n,
        (long long *)(E ? E + row * h->n_lat : nullptr), (long long *)(M ? M + row * h->n_lat : nullptr),
        h->n_lat, every, (int)f);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_sweeps_i8(spin_lattice *h, const int8_t *J, int64_t n_sweeps) {
  const Geom &g = h->g;
  const RoundKeys rk = make_round_keys(h->d.seed);
  const bool fast2d = g.dim == 2 && J == nullptr && (g.L % 8) == 0 && h->n_lat <= 65535;
  const bool fast3d = g.dim == 3 && J == nullptr && (g.L % 8) == 0 && h->n_lat <= 65535;
  if (fast2d && h->variant == 4 && coded_i8_supported(h) && n_sweeps >= kCodedMinSweeps)
    return launch_sweeps_i8_coded(h, n_sweeps);
  if (fast2d && (h->variant == 1 || h->variant == 4) && fused2d_supported(g.L)) return launch_fused2d_i8(h, n_sweeps);
  if ((fast2d || fast3d) && h->variant == 3 && resident_supported(g.dim, g.L))
    return launch_resident(h, n_sweeps, nullptr, nullptr, 1, 1);
  for (int64_t k = 0; k < n_sweeps; ++k) {
    const uint32_t sweep = (uint32_t)(h->sweeps_done + k);
    for (int colour = 0; colour < 2; ++colour) {
      if (fast2d) {
        const int chunks = g.L / 8;
        const int bx = chunks < 128 ? chunks : 128;
        const int by = 256 / bx;
        dim3 block(bx, by), grid((chunks + bx - 1) / bx, (g.L + by - 1) / by, (unsigned)h->n_lat);
        const cudaError_t e = launch_dependent(ising2d_phase_kernel, grid, block, 0, h->stream,
                                               (int8_t *)h->spins, g.L, (const uint32_t *)h->d_thr, g, rk,
                                               sweep, colour);
        if (e != cudaSuccess) return e;
      } else if (fast3d) {
        const int chunks = g.L / 8;
        const int bx = chunks < 64 ? chunks : 64;
        const int by = 256 / bx;
        const int tiles_x = (chunks + bx - 1) / bx, tiles_y = (g.L + by - 1) / by;
        const int zlen = g.L < 16 ? g.L : 16;
        dim3 block(bx, by), grid((unsigned)(tiles_x * tiles_y), (unsigned)((g.L + zlen - 1) / zlen),
                                 (unsigned)h->n_lat);
        const cudaError_t e = launch_dependent(ising3d_phase_kernel, grid, block, 0, h->stream,
                                               (int8_t *)h->spins, g.L, tiles_x, zlen, (const uint32_t *)h->d_thr,
                                               g, rk, sweep, colour);
        if (e != cudaSuccess) return e;
      } else {
        const uint32_t total = (uint32_t)(h->n_lat * ((g.N / 2 + 3) / 4));
        unsigned grid = grid_for(total, 256);
        if (grid > 1u << 20) grid = 1u << 20;
        phase_generic_kernel<<<grid, 256, 0, h->stream>>>((int8_t *)h->spins, J, h->d_thr, g,
                                                           total, rk, sweep, colour);
      }
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

}  // namespace spin
