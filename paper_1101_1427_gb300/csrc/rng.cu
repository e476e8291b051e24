// Bulk random words with the library's counter layout (the in-kernel
// generator of every sweep, exposed for checks and for its throughput).
#include "internal.h"

namespace spin {
namespace {

__global__ void rng_fill_kernel(uint32_t *__restrict__ out, uint64_t count, RoundKeys rk,
                                uint32_t w, uint32_t lid, uint32_t sweep) {
  const uint64_t quads = (count + 3) / 4;
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < quads;
       k += (uint64_t)gridDim.x * blockDim.x) {
    const uint4 r = philox(make_uint4((uint32_t)k, sweep, lid, w), rk);
    if (4 * k + 3 < count) {
      reinterpret_cast<uint4 *>(out)[k] = r;
    } else {
      for (uint32_t q = 0; q < 4 && 4 * k + q < count; ++q) out[4 * k + q] = word_of(r, q);
    }
  }
}

// Throughput probe: thread k draws `calls` Philox calls (counter x = k + i *
// threads) and folds all words with XOR into out[k], so the generator is
// timed without the store traffic of a bulk fill.
__global__ void rng_probe_kernel(uint32_t *__restrict__ out, uint32_t threads, uint32_t calls,
                                 RoundKeys rk) {
  const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= threads) return;
  uint32_t acc0 = 0, acc1 = 0;
  uint32_t i = 0;
  for (; i + 1 < calls; i += 2) {  // two independent calls per iteration
    const uint4 a = philox(make_uint4(k + i * threads, 0u, 0u, 0u), rk);
    const uint4 b = philox(make_uint4(k + (i + 1) * threads, 0u, 0u, 0u), rk);
    acc0 ^= a.x ^ a.y ^ a.z ^ a.w;
    acc1 ^= b.x ^ b.y ^ b.z ^ b.w;
  }
  if (i < calls) {
    const uint4 a = philox(make_uint4(k + i * threads, 0u, 0u, 0u), rk);
    acc0 ^= a.x ^ a.y ^ a.z ^ a.w;
  }
  out[k] = acc0 ^ acc1;
}

}  // namespace

cudaError_t launch_rng_probe(uint64_t seed, uint32_t threads, uint32_t calls, uint32_t *out,
                             cudaStream_t s) {
  if (threads == 0) return cudaSuccess;
  rng_probe_kernel<<<(threads + 255) / 256, 256, 0, s>>>(out, threads, calls, make_round_keys(seed));
  return cudaGetLastError();
}

cudaError_t launch_rng_fill(uint64_t seed, uint32_t w, uint32_t lid, uint32_t sweep,
                            uint64_t count, uint32_t *out, cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const uint64_t quads = (count + 3) / 4;
  uint64_t grid = (quads + 255) / 256;
  const uint64_t cap = (uint64_t)sms * 8;
  if (grid > cap) grid = cap;
  rng_fill_kernel<<<(unsigned)grid, 256, 0, s>>>(out, count, make_round_keys(seed), w, lid, sweep);
  return cudaGetLastError();
}

}  // namespace spin
