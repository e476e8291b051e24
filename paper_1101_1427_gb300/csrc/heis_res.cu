// Resident sweeps of the 3D Heisenberg model (Eq. On_hamiltonian, n = 3;
// the Metropolis update of Sec. 4) for lattices that fit, all together, in
// the shared memory of the GPU's SMs: L = 128 (2^21 float4 sites, 32 MiB) on
// 152 SMs of 227 KB, or a few lattices of L = 64.
//
// One persistent cooperative launch runs all sweeps of a call.  Each CTA owns
// a pencil of the lattice -- rows y0..y1-1 x z0..z1-1, every x -- and keeps
// both colours of it in shared memory (colour-split: [colour][row][L/2]) for
// the whole call.  Neighbours inside the pencil are read from shared memory;
// the rows on the pencil's faces are also published, after every update, to
// an exchange buffer in global memory ([lattice][colour][L^2 rows][L/2]),
// from which the neighbouring pencils read them.  Instead of one launch (and
// a grid-wide drain) per colour phase, each CTA waits only for its four
// neighbour pencils: a per-CTA counter of published phases, released once the
// CTA's face rows of a phase are written and polled (bounded in time) before
// the next phase.  Face sites are updated first in each phase so that the
// release comes early; the interior sites, whose neighbours are all in
// shared memory, cover the propagation of the neighbours' releases.
//
// Every site update is heis_step() of heis_step.cuh with the Philox counter
// of the other Heisenberg kernels (colour-site index, sweep, lattice id,
// colour), and h = (x+1) + (x-1) + (y+1) + (y-1) + (z+1) + (z-1) summed in
// that order, so a chain is the same bit for bit whichever kernel ran it.
#include "heis_step.cuh"
#include "internal.h"

namespace spin {
namespace {

constexpr int kResThreads = 1024;
constexpr int kResMaxRows = 128;  // rows per pencil (the row table is static shared memory)

struct ResArgs {
  float4 *s;             // row-major lattices [n_lat][N] (read at the start, written at the end)
  float4 *X;             // exchange buffer [n_lat][2][L^2][L/2]
  unsigned *flags;       // [grid]: phases published by each CTA, monotonic across launches
  int *err;              // handle error word (1: a wait timed out)
  const uint32_t *thr;   // per slot: beta (float bits), beta log2(e) (float bits)
  RoundKeys rk;
  Geom g;
  uint32_t Py, Pz;       // pencils per lattice along y and z (each >= 2, each pencil >= 2 rows)
  uint32_t sweep0, n_sweeps, base;
  uint32_t extra;        // phases a wait asks for beyond those published (0; > 0 only in tests of the timeout)
  uint64_t timeout_ns;
};

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_gpu(unsigned *p, unsigned v) {
  asm volatile("st.release.gpu.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// Load through a generic address (shared memory or global), bypassing L1 for
// global memory: the exchange buffer changes between phases.
__device__ __forceinline__ float4 ld_cg(const float4 *p) {
  float4 v;
  asm volatile("ld.cg.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Thread t owns column kx = t % kH and the local rows r0 + (kResThreads / kH) i
// of both colours.  Per local row the table holds the Philox index of its
// colour site 0 (global row * L/2), its face bits (1: y+1, 2: y-1, 4: z+1,
// 8: z-1 outside the pencil) | (y + z) parity << 8, and the exchange-buffer
// row offsets of its outside y and z neighbours.
template <bool kFast, int kH>
__global__ void __launch_bounds__(kResThreads, 1) heis_resident_kernel(ResArgs P) {
  extern __shared__ float4 sm[];
  __shared__ uint4 rinfo[kResMaxRows];
  __shared__ unsigned bcnt_s[2], nbwarps_s;
  __shared__ int abort_s;
  constexpr uint32_t kRowStep = kResThreads / kH;
  constexpr uint32_t L = 2 * kH, LL = L * L;
  const uint32_t per_lat = P.Py * P.Pz, lat = blockIdx.x / per_lat, pi = blockIdx.x - lat * per_lat;
  const uint32_t by = pi % P.Py, bz = pi / P.Py;
  const uint32_t y0 = by * L / P.Py, y1 = (by + 1) * L / P.Py, z0 = bz * L / P.Pz, z1 = (bz + 1) * L / P.Pz;
  const uint32_t ny = y1 - y0, nz = z1 - z0, nrows = ny * nz, nyH = ny * kH;
  float4 *sm0 = sm, *sm1 = sm + nrows * kH;
  float4 *sl = P.s + (size_t)lat * LL * L;
  float4 *Xl = P.X + (size_t)lat * LL * L;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool single = P.g.n_real == 1 && P.g.n_temps == 1 && P.g.n_sets == 1;
  const uint32_t lid = single ? 0u : lattice_id32(P.g, lat), slot = single ? 0u : slot_of32(P.g, lat);
  const float beta = __uint_as_float(__ldg(P.thr + 4 * slot)), bl = __uint_as_float(__ldg(P.thr + 4 * slot + 1));

  for (uint32_t lr = threadIdx.x; lr < nrows; lr += kResThreads) {
    const uint32_t yy = lr % ny, zz = lr / ny, y = y0 + yy, z = z0 + zz;
    uint32_t ext = 0, gy = 0, gz = 0;
    if (yy == ny - 1) {
      ext |= 1;
      gy = (z * L + (y == L - 1 ? 0 : y + 1)) * kH;
    }
    if (yy == 0) {
      ext |= 2;
      gy = (z * L + (y == 0 ? L - 1 : y - 1)) * kH;
    }
    if (zz == nz - 1) {
      ext |= 4;
      gz = ((z == L - 1 ? 0 : z + 1) * L + y) * kH;
    }
    if (zz == 0) {
      ext |= 8;
      gz = ((z == 0 ? L - 1 : z - 1) * L + y) * kH;
    }
    rinfo[lr] = make_uint4((z * L + y) * kH, ext | ((y + z) & 1u) << 8, gy, gz);
  }
  if (threadIdx.x == 0) {
    abort_s = 0;
    bcnt_s[0] = bcnt_s[1] = 0;
    nbwarps_s = 0;
  }
  // the pencil into shared memory; its face rows (both colours) into the exchange buffer
  for (uint32_t t = threadIdx.x; t < nrows * L; t += kResThreads) {
    const uint32_t lr = t / L, x = t - lr * L, yy = lr % ny, zz = lr / ny;
    const uint32_t y = y0 + yy, z = z0 + zz, row = z * L + y, c = (x + y + z) & 1u;
    const float4 v = sl[(size_t)row * L + x];
    (c ? sm1 : sm0)[lr * kH + (x >> 1)] = v;
    if (yy == 0 || yy == ny - 1 || zz == 0 || zz == nz - 1) __stcg(Xl + c * LL * kH + row * kH + (x >> 1), v);
  }
  __syncthreads();

  const uint32_t nbase = lat * per_lat;
  const uint32_t nbr[4] = {nbase + (by + 1) % P.Py + bz * P.Py, nbase + (by + P.Py - 1) % P.Py + bz * P.Py,
                           nbase + by + ((bz + 1) % P.Pz) * P.Py, nbase + by + ((bz + P.Pz - 1) % P.Pz) * P.Py};
  // Warp 0, lanes 0..3: wait until the four neighbours have published `need`
  // phases (bounded by the handle's timeout; gives up if another CTA failed).
  auto poll = [&](unsigned need) {
    need += P.extra;
    bool failed = false;
    if (lane < 4) {
      const unsigned *f = P.flags + (lane == 0 ? nbr[0] : lane == 1 ? nbr[1] : lane == 2 ? nbr[2] : nbr[3]);
      const uint64_t t0 = gtimer();
      while ((int)(ld_acquire_gpu(f) - need) < 0) {
        if (*(volatile int *)P.err) {
          failed = true;
          break;
        }
        if (gtimer() - t0 > P.timeout_ns) {
          atomicExch(P.err, 1);
          failed = true;
          break;
        }
      }
    }
    if (__any_sync(0xffffffffu, failed) && lane == 0) abort_s = 1;
    __syncwarp();
  };
  if (warp == 0) {
    if (lane == 0) {
      __threadfence();
      st_release_gpu(P.flags + blockIdx.x, P.base + 1);
    }
    __syncwarp();
    poll(P.base + 1);
  }

  const uint32_t kx = threadIdx.x % kH, r0 = threadIdx.x / kH;
  const uint32_t nsites = nrows > r0 ? (nrows - r0 + kRowStep - 1) / kRowStep : 0;
  uint32_t bmask = 0;  // this thread's face sites (the same for the whole warp: its lanes share rows)
  for (uint32_t i = 0; i < nsites; ++i) bmask |= (rinfo[r0 + kRowStep * i].y & 15u) ? 1u << i : 0u;
  const uint32_t imask = ((nsites >= 32) ? 0xffffffffu : ((1u << nsites) - 1u)) & ~bmask;
  if (lane == 0 && bmask) atomicAdd(&nbwarps_s, 1u);
  __syncthreads();
  const unsigned nbwarps = nbwarps_s;
  const int dxm = kx == 0 ? kH - 1 : -1, dxp = kx == kH - 1 ? 1 - (int)kH : 1;  // the other colour's x-1 / x+1

  const uint32_t nph = 2 * P.n_sweeps;
  for (uint32_t q = 0; q < nph; ++q) {
    if (abort_s) return;
    const uint32_t c = q & 1u, sweep = P.sweep0 + (q >> 1);
    if (threadIdx.x == 0) bcnt_s[c ^ 1u] = 0;  // the other counter is next used in phase q + 1
    const uint32_t wctr = ctr_w(TAG_HEIS, c, 0);
    float4 *own = c ? sm1 : sm0;
    const float4 *oth = c ? sm0 : sm1;
    const float4 *Xo = Xl + (1 - c) * LL * kH;
    float4 *Xw = Xl + c * LL * kH;
    // face sites: each neighbour row is the pencil's own (shared memory) or a
    // neighbour pencil's (exchange buffer); one generic load per neighbour
    for (uint32_t mk = bmask; mk; mk &= mk - 1) {
      const uint32_t lr = r0 + kRowStep * (__ffs(mk) - 1), idx = lr * kH + kx;
      const uint4 ri = rinfo[lr];
      const uint32_t ext = ri.y & 15u, p = (c + (ri.y >> 8)) & 1u;
      const float4 *o = oth + idx;
      const float4 m = o[0], sh = o[p ? dxp : dxm];  // x +- 1: sh is x + 1 if p, else x - 1
      const float4 *gy = Xo + ri.z + kx, *gz = Xo + ri.w + kx;
      // (the face bits are the same for the whole warp: no divergence)
      float4 cy, dy, ez, fz;
      if (ext & 1) cy = ld_cg(gy); else cy = o[kH];
      if (ext & 2) dy = ld_cg(gy); else dy = o[-kH];
      if (ext & 4) ez = ld_cg(gz); else ez = o[nyH];
      if (ext & 8) fz = ld_cg(gz); else fz = o[-(int)nyH];
      const float4 si = own[idx];
      const uint4 w = philox(make_uint4(ri.x + kx, sweep, lid, wctr), P.rk);
      // (x+1) + (x-1) first: the same sum in either order
      const float hx = m.x + sh.x + cy.x + dy.x + ez.x + fz.x;
      const float hy = m.y + sh.y + cy.y + dy.y + ez.y + fz.y;
      const float hz = m.z + sh.z + cy.z + dy.z + ez.z + fz.z;
      float4 n;
      if (heis_step<kFast>(si, hx, hy, hz, w, beta, bl, n)) {
        own[idx] = n;
        __stcg(Xw + ri.x + kx, n);
      }
    }
    if (bmask) {
      // this warp's face sites are written; the last such warp publishes the phase
      __syncwarp();
      if (lane == 0) {
        __threadfence_block();
        if (atomicAdd(&bcnt_s[c], 1u) == nbwarps - 1) {
          __threadfence();
          st_release_gpu(P.flags + blockIdx.x, P.base + 2 + q);
        }
      }
    }
    // interior sites: all six neighbours in shared memory at fixed offsets
    for (uint32_t mk = imask; mk; mk &= mk - 1) {
      const uint32_t lr = r0 + kRowStep * (__ffs(mk) - 1), idx = lr * kH + kx;
      const uint2 ri = make_uint2(rinfo[lr].x, rinfo[lr].y);
      const uint32_t p = (c + (ri.y >> 8)) & 1u;
      const float4 *o = oth + idx;
      const float4 m = o[0], sh = o[p ? dxp : dxm];
      const float4 cy = o[kH], dy = o[-kH], ez = o[nyH], fz = o[-(int)nyH];
      const float4 si = own[idx];
      const uint4 w = philox(make_uint4(ri.x + kx, sweep, lid, wctr), P.rk);
      const float hx = m.x + sh.x + cy.x + dy.x + ez.x + fz.x;
      const float hy = m.y + sh.y + cy.y + dy.y + ez.y + fz.y;
      const float hz = m.z + sh.z + cy.z + dy.z + ez.z + fz.z;
      float4 n;
      if (heis_step<kFast>(si, hx, hy, hz, w, beta, bl, n)) own[idx] = n;
    }
    if (nbwarps == 0 && threadIdx.x == 0) st_release_gpu(P.flags + blockIdx.x, P.base + 2 + q);
    if (warp == 0 && q + 1 < nph) poll(P.base + 2 + q);
    __syncthreads();
  }
  if (abort_s) return;
  for (uint32_t t = threadIdx.x; t < nrows * L; t += kResThreads) {
    const uint32_t lr = t / L, x = t - lr * L, yy = lr % ny, zz = lr / ny;
    const uint32_t y = y0 + yy, z = z0 + zz, c = (x + y + z) & 1u;
    sl[(size_t)(z * L + y) * L + x] = (c ? sm1 : sm0)[lr * kH + (x >> 1)];
  }
}

template <bool kFast, int kH>
const void *resident_kernel() {
  return (const void *)heis_resident_kernel<kFast, kH>;
}

const void *pick_kernel(int variant, int L) {
  const bool fast = variant == 2;
  if (L == 128) return fast ? resident_kernel<true, 64>() : resident_kernel<false, 64>();
  return fast ? resident_kernel<true, 32>() : resident_kernel<false, 32>();
}

// Shared memory the kernel's static arrays take (row table, counters).
constexpr size_t kResStaticSmem = sizeof(uint4) * kResMaxRows + 64;

}  // namespace

bool heis_resident_plan(const spin_lattice *h, HeisResPlan *plan) {
  if (h->g.dim != 3 || (h->g.L != 64 && h->g.L != 128) || h->n_lat < 1) return false;
  int dev = 0, sms = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return false;
  const int64_t L = h->g.L;
  if (h->n_lat > sms / 4) return false;
  const int64_t per_lat_max = sms / h->n_lat;
  // smallest largest pencil (then the fewest face rows): rows x L float4 of shared memory
  int64_t best_rows = 0, best_face = 0, best_py = 0, best_pz = 0;
  for (int64_t pz = 2; pz <= L / 2; ++pz)
    for (int64_t py = 2; py <= L / 2 && py * pz <= per_lat_max; ++py) {
      const int64_t ny = (L + py - 1) / py, nz = (L + pz - 1) / pz, rows = ny * nz, face = 2 * (ny + nz) - 4;
      if (rows > kResMaxRows || (size_t)rows * L * 16 + kResStaticSmem > (size_t)optin) continue;
      if (best_rows == 0 || rows < best_rows || (rows == best_rows && face < best_face)) {
        best_rows = rows;
        best_face = face;
        best_py = py;
        best_pz = pz;
      }
    }
  if (best_rows == 0) return false;
  plan->Py = (int)best_py;
  plan->Pz = (int)best_pz;
  plan->grid = (int)(h->n_lat * best_py * best_pz);
  plan->smem = (size_t)best_rows * L * 16;
  // the cooperative launch needs every CTA resident at once (one per SM)
  const void *k = pick_kernel(h->variant, (int)L);
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plan->smem) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, kResThreads, plan->smem) != cudaSuccess || occ < 1 ||
      plan->grid > occ * sms) {
    cudaGetLastError();
    return false;
  }
  return true;
}

cudaError_t launch_sweeps_heis_resident(spin_lattice *h, const HeisResPlan &plan, int64_t sweep0, int64_t n_sweeps) {
  const int64_t total = h->n_lat * h->g.N;
  const size_t bytes = (size_t)total * 16;
  if (!h->d_pingpong || h->pingpong_bytes < bytes) {
    if (h->d_pingpong) cudaFree(h->d_pingpong);
    h->d_pingpong = nullptr;
    cudaError_t e = cudaMalloc(&h->d_pingpong, bytes);
    if (e != cudaSuccess) return e;
    h->pingpong_bytes = bytes;
  }
  if (!h->d_res_flags || h->res_flags_n < plan.grid || h->res_base > 0x7fffffffu) {
    if (h->d_res_flags) cudaFree(h->d_res_flags);
    h->d_res_flags = nullptr;
    cudaError_t e = cudaMalloc(&h->d_res_flags, sizeof(unsigned) * plan.grid);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(h->d_res_flags, 0, sizeof(unsigned) * plan.grid, h->stream);
    if (e != cudaSuccess) return e;
    h->res_flags_n = plan.grid;
    h->res_base = 0;
  }
  ResArgs a;
  a.s = (float4 *)h->spins;
  a.X = (float4 *)h->d_pingpong;
  a.flags = h->d_res_flags;
  a.err = h->d_err;
  a.thr = h->d_thr;
  a.rk = make_round_keys(h->d.seed);
  a.g = h->g;
  a.Py = (uint32_t)plan.Py;
  a.Pz = (uint32_t)plan.Pz;
  a.sweep0 = (uint32_t)sweep0;
  a.n_sweeps = (uint32_t)n_sweeps;
  a.base = h->res_base;
  a.extra = (uint32_t)h->batch_fault_extra;
  a.timeout_ns = h->batch_timeout_ns ? h->batch_timeout_ns : 2000000000ull;
  h->res_base += 2u * (uint32_t)n_sweeps + 1u;
  void *args[] = {&a};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)plan.grid);
  cfg.blockDim = dim3(kResThreads);
  cfg.dynamicSmemBytes = plan.smem;
  cfg.stream = h->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;  // every CTA resident at once: the neighbour waits need it
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelExC(&cfg, pick_kernel(h->variant, h->g.L), args);
}

}  // namespace spin
