// Bit-sliced counters: 32 counters side by side, bit b of plane k holding
// bit k of counter b.  Shared by the batched kernel and the measurement
// kernels of the coded EA glass.
#pragma once
#include <cstdint>

namespace spin {

// carry-save adder: (h, l) = 2h + l = a + b + c per bit
__device__ __forceinline__ void csa(uint32_t &h, uint32_t &l, uint32_t a, uint32_t b, uint32_t c) {
  const uint32_t u = a ^ b;
  h = (a & b) | (u & c);
  l = u ^ c;
}

// counter planes from level W up += x, a plane of weight 2^W (ripple carry)
template <int W, int K>
__device__ __forceinline__ void ripple_at(uint32_t (&C)[K], uint32_t x) {
#pragma unroll
  for (int k = W; k < K; ++k) {
    const uint32_t n = C[k] & x;
    C[k] ^= x;
    x = n;
  }
}

}  // namespace spin
