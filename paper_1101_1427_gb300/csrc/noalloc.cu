// Heisenberg energy and magnetisation for callers that cannot allocate
// device memory.
//
// The regular reduction (spin_measure) keeps its per-block partial sums in
// a workspace that spin_init allocates.  Some callers cannot get that far:
// code that runs inside a framework which owns the whole device-memory pool
// (a raw cudaMalloc there either fails or fragments the pool), and code
// that must not stall the device, since cudaFree and often cudaMalloc
// synchronise it.  This variant takes the spins and the outputs from the
// caller and keeps its partial sums in one fixed array compiled into the
// library (kMaxLattices lattices x 64 blocks x 4 doubles = 512 KiB per
// device, held from library load until process exit).
#include <mutex>

#include "internal.h"

namespace {

constexpr int kBlocks = 64;         // partial sums per lattice
constexpr int kMaxLattices = 256;   // capacity of the fixed scratch
constexpr int kMaxDevices = 64;

// Fixed scratch: [lattice][block][E, Mx, My, Mz].  Every call overwrites the
// entries it uses before reading them, so nothing has to start at zero.
static __device__ __align__(256) double g_partials[kMaxLattices * kBlocks * 4];

std::mutex g_setup_mutex;
double *g_partials_addr[kMaxDevices] = {};  // device address of g_partials, per device

// Same arithmetic and order as the reduction behind spin_measure: FP32
// products widened to double, per-thread double sums, warp and block sums,
// then a fixed-order pass over the block partials.
__global__ void heis_partials_kernel(const float4 *__restrict__ s, int L, double *__restrict__ part) {
  const int64_t lat = blockIdx.y;
  const int64_t N = (int64_t)L * L * L;
  const float4 *sl = s + lat * N;
  const int64_t LL = (int64_t)L * L;
  double e = 0.0, mx = 0.0, my = 0.0, mz = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % L), y = (int)((i / L) % L), z = (int)(i / LL);
    const float4 a = sl[i];
    const float4 bx = sl[i - x + (x == L - 1 ? 0 : x + 1)];
    const float4 by = sl[y == L - 1 ? i - (int64_t)(L - 1) * L : i + L];
    const float4 bz = sl[z == L - 1 ? i - (int64_t)(L - 1) * LL : i + LL];
    const double ax = a.x, ay = a.y, az = a.z;
    e -= ax * ((double)bx.x + (double)by.x + (double)bz.x) +
         ay * ((double)bx.y + (double)by.y + (double)bz.y) +
         az * ((double)bx.z + (double)by.z + (double)bz.z);
    mx += ax;
    my += ay;
    mz += az;
  }
  __shared__ double red[4][32];
  e = spin::warp_sum(e);
  mx = spin::warp_sum(mx);
  my = spin::warp_sum(my);
  mz = spin::warp_sum(mz);
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
    part[(lat * gridDim.x + blockIdx.x) * 4 + threadIdx.x] = acc;
  }
}

__global__ void heis_finish_kernel(const double *__restrict__ part, int64_t n_lat, double *__restrict__ Ef,
                                   double *__restrict__ Mf) {
  const int64_t lat = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (lat >= n_lat) return;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int b = 0; b < kBlocks; ++b)
    for (int c = 0; c < 4; ++c) acc[c] += part[(lat * kBlocks + b) * 4 + c];
  if (Ef) Ef[lat] = acc[0];
  if (Mf) {
    Mf[3 * lat] = acc[1];
    Mf[3 * lat + 1] = acc[2];
    Mf[3 * lat + 2] = acc[3];
  }
}

// Device address of the fixed scratch for the current device, looked up
// once per device (host code cannot use the symbol itself as a pointer).
int partials_for_current_device(double **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SPIN_ECUDA;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_partials_addr[dev]) {
    double *p = nullptr;
    if (cudaGetSymbolAddress((void **)&p, g_partials) != cudaSuccess || !p) return SPIN_ECUDA;
    g_partials_addr[dev] = p;
  }
  *out = g_partials_addr[dev];
  return SPIN_OK;
}

}  // namespace

extern "C" int spin_heis_measure_noalloc(const float *spins, int32_t L, int32_t n_lat, double *Ef,
                                         double *Mf, void *stream) {
  if (!spins || L < 4 || (L & 1) || n_lat < 1) return SPIN_EINVAL;
  if (n_lat > kMaxLattices) return SPIN_EINVAL;  // beyond the fixed scratch
  if ((int64_t)n_lat * L * L * L >= ((int64_t)1 << 31)) return SPIN_EINVAL;
  if (((uintptr_t)spins & 15u) != 0) return SPIN_EALIGN;
  if (!Ef && !Mf) return SPIN_OK;
  double *part = nullptr;
  const int rc = partials_for_current_device(&part);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  heis_partials_kernel<<<dim3(kBlocks, (unsigned)n_lat), 256, 0, st>>>((const float4 *)spins, L, part);
  heis_finish_kernel<<<(n_lat + 127) / 128, 128, 0, st>>>(part, n_lat, Ef, Mf);
  return cudaGetLastError() == cudaSuccess ? SPIN_OK : SPIN_ECUDA;
}
