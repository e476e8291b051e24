// Fused checkerboard sweep of the 2D Ising ferromagnet, int8 spins.
//
// A sweep (Sec. 3.2) updates all colour-0 sites from the old colour-1 sites
// and then all colour-1 sites from the new colour-0 sites.  Done in place it
// needs two passes over the lattice (~4 bytes of HBM traffic per flip, every
// 32-byte sector holding sites of both colours).  Here one pass reads the
// old lattice A and writes the new lattice B:
//
//   * a CTA owns a horizontal strip of rows [y0, y0 + H) across the whole
//     width; thread tid owns bytes [16 tid, 16 tid + 16) of every row and
//     streams down the strip keeping four rows in registers;
//   * at row step y it updates colour 0 of row y+1 (inputs: old rows y, y+1,
//     y+2, all still old in their colour-1 bytes), publishes that row to a
//     three-row shared-memory ring, waits at one barrier, then updates
//     colour 1 of row y (inputs: new colour-0 values of rows y-1, y, y+1;
//     the bytes across thread boundaries come from the ring) and stores
//     row y to B;
//   * rows y0-1 and y0 of colour 0 are recomputed by the strip itself.  The
//     random word of every site is a pure function of its counter, so the
//     recomputation equals what the neighbouring strip computes.
//
// The result is identical to the two in-place colour phases.
#include "i8chunk.cuh"
#include "internal.h"

namespace spin {
namespace {

// New value of one 8-byte chunk whose active colour sits on the bytes of
// parity p (the same for every thread of the CTA: it depends on the row and
// the colour only); lb/rb are the bytes left of byte 0 and right of byte 7.
__device__ __forceinline__ uint64_t update_chunk(uint64_t C, uint64_t U, uint64_t D, uint32_t lb,
                                                 uint32_t rb, int p, uint4 r, uint32_t thr4,
                                                 uint32_t thr8) {
  long long unused_a = 0, unused_d = 0;
  return ising_chunk<0>(C, U, D, lb, rb, r, p, thr4, thr8, unused_a, unused_d);
}

struct Row16 {
  uint64_t a, b;  // bytes 0..7 and 8..15 of the thread's segment
};

__device__ __forceinline__ Row16 ld_row(const int8_t *__restrict__ base, int64_t off) {
  const uint4 v = __ldcs(reinterpret_cast<const uint4 *>(base + off));
  Row16 r;
  r.a = (uint64_t)v.x | ((uint64_t)v.y << 32);
  r.b = (uint64_t)v.z | ((uint64_t)v.w << 32);
  return r;
}

// Colour update of one row segment (two chunks); lb/rb are the bytes just
// outside the segment.  j4 base = y * (L/8) + 2 tid.
__device__ __forceinline__ Row16 update_row(Row16 C, Row16 U, Row16 D, uint32_t lb, uint32_t rb,
                                            int colour, int y, uint32_t j4, uint32_t sweep,
                                            uint32_t lid, const RoundKeys &rk, uint32_t thr4,
                                            uint32_t thr8) {
  const int p = (colour + y) & 1;
  const uint32_t w = ctr_w(TAG_UPDATE, (uint32_t)colour, 0);
  const uint4 r0 = philox(make_uint4(j4, sweep, lid, w), rk);
  const uint4 r1 = philox(make_uint4(j4 + 1, sweep, lid, w), rk);
  Row16 out;
  out.a = update_chunk(C.a, U.a, D.a, lb, (uint32_t)(C.b & 0xffu), p, r0, thr4, thr8);
  out.b = update_chunk(C.b, U.b, D.b, (uint32_t)(C.a >> 56), rb, p, r1, thr4, thr8);
  return out;
}

__global__ void __launch_bounds__(1024, 1)
    fused2d_kernel(const int8_t *__restrict__ A, int8_t *__restrict__ B, int L, int H,
                   const uint32_t *__restrict__ thr, Geom g, RoundKeys rk, uint32_t sweep) {
  extern __shared__ __align__(16) uint8_t ring[];  // 3 rows x L bytes
  const int tid = threadIdx.x;
  const int64_t lat = blockIdx.y;
  const int y0 = blockIdx.x * H;
  if (y0 >= L) return;
  const int y1 = min(y0 + H, L);
  const int64_t LL = (int64_t)L * L;
  const int8_t *a = A + lat * LL;
  int8_t *b = B + lat * LL;
  const uint32_t t = slot_of32(g, (uint32_t)lat);
  const uint32_t thr4 = __ldg(thr + 4 * t + 1), thr8 = __ldg(thr + 4 * t + 2);
  const uint32_t lid = lattice_id32(g, (uint32_t)lat);
  const uint32_t cpr = (uint32_t)(L >> 3);  // chunks per row
  const int x0 = 16 * tid;
  const int xl = x0 == 0 ? L - 1 : x0 - 1;
  const int xr = x0 + 16 == L ? 0 : x0 + 16;
  auto wrap = [L](int y) { return y < 0 ? y + L : (y >= L ? y - L : y); };
  auto row_off = [&](int y) { return (int64_t)wrap(y) * L; };

  // Registers: R0 = row y-1 (colour 0 new), R1 = row y (colour 0 new,
  // colour 1 old), R2 = row y+1 (old), R3 = row y+2 (old).
  Row16 Rm2 = ld_row(a, row_off(y0 - 2) + x0);
  Row16 R0 = ld_row(a, row_off(y0 - 1) + x0);
  Row16 R1 = ld_row(a, row_off(y0) + x0);
  Row16 R2 = ld_row(a, row_off(y0 + 1) + x0);
  Row16 R3 = ld_row(a, row_off(y0 + 2) + x0);
  {
    // colour 0 of rows y0-1 and y0 (edge bytes are old values from A)
    const int ym = wrap(y0 - 1), yc = wrap(y0);
    const uint32_t lbm = (uint8_t)a[row_off(ym) + xl], rbm = (uint8_t)a[row_off(ym) + xr];
    const uint32_t lbc = (uint8_t)a[row_off(yc) + xl], rbc = (uint8_t)a[row_off(yc) + xr];
    const Row16 n0 = update_row(R0, Rm2, R1, lbm, rbm, 0, ym, (uint32_t)ym * cpr + 2 * tid, sweep,
                                lid, rk, thr4, thr8);
    const Row16 n1 = update_row(R1, R0, R2, lbc, rbc, 0, yc, (uint32_t)yc * cpr + 2 * tid, sweep,
                                lid, rk, thr4, thr8);
    R0 = n0;
    R1 = n1;
    // ring slots are indexed by the step (row - y0) mod 3, not by the
    // wrapped row, so consecutive rows never share a slot
    uint4 *slot = reinterpret_cast<uint4 *>(ring + x0);
    *slot = make_uint4((uint32_t)R1.a, (uint32_t)(R1.a >> 32), (uint32_t)R1.b, (uint32_t)(R1.b >> 32));
  }
  for (int y = y0; y < y1; ++y) {
    const int yn = wrap(y + 1);
    // prefetch row y+3 for the next step
    const Row16 R4 = ld_row(a, row_off(y + 3) + x0);
    // colour 0 of row y+1 (old neighbours; edge bytes from A)
    const uint32_t lbn = (uint8_t)a[(int64_t)yn * L + xl], rbn = (uint8_t)a[(int64_t)yn * L + xr];
    R2 = update_row(R2, R1, R3, lbn, rbn, 0, yn, (uint32_t)yn * cpr + 2 * tid, sweep, lid, rk,
                    thr4, thr8);
    *reinterpret_cast<uint4 *>(ring + (size_t)((y + 1 - y0) % 3) * L + x0) =
        make_uint4((uint32_t)R2.a, (uint32_t)(R2.a >> 32), (uint32_t)R2.b, (uint32_t)(R2.b >> 32));
    __syncthreads();
    // colour 1 of row y (new colour-0 neighbours; edge bytes from the ring)
    const int yc = wrap(y);
    const uint8_t *rr = ring + (size_t)((y - y0) % 3) * L;
    const uint32_t lbc = rr[xl], rbc = rr[xr];
    R1 = update_row(R1, R0, R2, lbc, rbc, 1, yc, (uint32_t)yc * cpr + 2 * tid, sweep, lid, rk,
                    thr4, thr8);
    __stcs(reinterpret_cast<uint4 *>(b + (int64_t)yc * L + x0),
           make_uint4((uint32_t)R1.a, (uint32_t)(R1.a >> 32), (uint32_t)R1.b, (uint32_t)(R1.b >> 32)));
    R0 = R1;
    R1 = R2;
    R2 = R3;
    R3 = R4;
  }
}

}  // namespace

// Requirements: L % 16 == 0 and 16 <= L <= 16384 (one thread per 16 bytes of a row).
bool fused2d_supported(int L) { return L % 16 == 0 && L >= 32 && L <= 16384; }

int fused2d_strip_height(int L, int n_lat) {
  int dev = 0, sms = 148, occ = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // a single wave of resident CTAs (one per SM for L = 16384, several of
  // the smaller CTAs of smaller lattices), rows split evenly over a
  // lattice's CTAs
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fused2d_kernel, L / 16, 3 * (size_t)L) != cudaSuccess ||
      occ < 1)
    occ = 1;
  int64_t ctas_per_lat = (int64_t)sms * occ / n_lat;
  if (ctas_per_lat < 1) ctas_per_lat = 1;
  int H = (int)((L + ctas_per_lat - 1) / ctas_per_lat);
  if (H < 8) H = 8;
  return H;
}

cudaError_t launch_fused2d_i8(spin_lattice *h, int64_t n_sweeps) {
  const int L = h->g.L;
  const size_t bytes = (size_t)h->n_lat * (size_t)h->g.N;
  if (!h->d_pingpong || h->pingpong_bytes < bytes) {
    if (h->d_pingpong) cudaFree(h->d_pingpong);
    h->d_pingpong = nullptr;
    cudaError_t e = cudaMalloc(&h->d_pingpong, bytes);
    if (e != cudaSuccess) return e;
    h->pingpong_bytes = bytes;
  }
  const int H = fused2d_strip_height(L, (int)h->n_lat);
  const int threads = L / 16;
  const size_t smem = 3 * (size_t)L;
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(fused2d_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 3 * 16384);
    attr_set = true;
  }
  dim3 grid((unsigned)((L + H - 1) / H), (unsigned)h->n_lat);
  const RoundKeys rk = make_round_keys(h->d.seed);
  int8_t *U = (int8_t *)h->spins, *S = (int8_t *)h->d_pingpong;
  // ping-pong so that the last sweep writes the caller's buffer
  const int8_t *src = U;
  int8_t *dst = S;
  if (n_sweeps & 1) {
    cudaError_t e = cudaMemcpyAsync(S, U, bytes, cudaMemcpyDeviceToDevice, h->stream);
    if (e != cudaSuccess) return e;
    src = S;
    dst = U;
  }
  for (int64_t k = 0; k < n_sweeps; ++k) {
    fused2d_kernel<<<grid, threads, smem, h->stream>>>(src, dst, L, H, h->d_thr, h->g, rk,
                                                       (uint32_t)(h->sweeps_done + k));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int8_t *tmp = dst;
    dst = const_cast<int8_t *>(src);
    src = tmp;
  }
  return cudaSuccess;
}

}  // namespace spin
