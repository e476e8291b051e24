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

#include "heis_reduce.cuh"
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

// The arithmetic and order of the reduction behind spin_measure (one shared
// device function), so both give bit-identical sums.
__global__ void heis_partials_kernel(const float4 *__restrict__ s, int dim, int L, int64_t N,
                                     double *__restrict__ part) {
  const int64_t lat = blockIdx.y;
  spin::heis_block_partials(s + lat * N, L, dim, N, blockIdx.x, gridDim.x,
                            part + (lat * gridDim.x + blockIdx.x) * 4);
}

__global__ void heis_finish_kernel(const double *__restrict__ part, int64_t n_lat, double *__restrict__ Ef,
                                   double *__restrict__ Mf) {
  const int64_t lat = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (lat >= n_lat) return;
  spin::heis_finish_lattice(part, kBlocks, lat, Ef, Mf);
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

extern "C" int spin_heis_measure_noalloc(const float *spins, int32_t dim, int32_t L, int32_t n_lat, double *Ef,
                                         double *Mf, void *stream) {
  if (!spins || (dim != 2 && dim != 3) || L < 4 || (L & 1) || n_lat < 1) return SPIN_EINVAL;
  if (n_lat > kMaxLattices) return SPIN_EINVAL;  // beyond the fixed scratch
  // bound L on its own first, so that the products below cannot overflow
  if (L > (dim == 3 ? 1290 : 46340)) return SPIN_EINVAL;  // L^dim < 2^31
  const int64_t N = dim == 3 ? (int64_t)L * L * L : (int64_t)L * L;
  if ((int64_t)n_lat * N >= ((int64_t)1 << 31)) return SPIN_EINVAL;
  if (((uintptr_t)spins & 15u) != 0) return SPIN_EALIGN;
  if (!Ef && !Mf) return SPIN_OK;
  double *part = nullptr;
  const int rc = partials_for_current_device(&part);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  heis_partials_kernel<<<dim3(kBlocks, (unsigned)n_lat), 256, 0, st>>>((const float4 *)spins, dim, L, N, part);
  heis_finish_kernel<<<(n_lat + 127) / 128, 128, 0, st>>>(part, n_lat, Ef, Mf);
  return cudaGetLastError() == cudaSuccess ? SPIN_OK : SPIN_ECUDA;
}
