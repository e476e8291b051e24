// Instruction-throughput probe for the roofline of the sweeps: every thread
// runs eight independent chains of one operation (a wide multiply, a
// multiply-high, a three-input logic op, a three-input add, an FP32 fused
// multiply-add or a special-function reciprocal square root), and every CTA
// records the SM clock before and after its loop and the SM it ran on.  The
// CTAs of one SM do not progress evenly (the scheduler favours the oldest
// warps), so a rate is taken over the span of all CTAs of an SM.  The operations are the ones Philox and
// the spin updates are built from; the probe measures how many of them one
// SM completes per clock.
#include "internal.h"

namespace spin {
namespace {

template <int kOp>
__global__ void __launch_bounds__(256) pipe_probe_kernel(uint32_t iters, long long *__restrict__ clocks,
                                                        uint32_t *__restrict__ sink) {
  const uint32_t g = blockIdx.x * 256u + threadIdx.x;
  uint32_t x[8];
  uint64_t w[8];
  float f[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    x[c] = 8u * g + (uint32_t)c + 1u;
    w[c] = x[c];
    f[c] = 1.0f + (float)(8u * g + (uint32_t)c) * 0x1p-20f;
  }
  __syncthreads();
  const long long t0 = clock64();
  for (uint32_t it = 0; it < iters; ++it) {
    if (kOp == SPIN_PIPE_MUL_WIDE) {
#pragma unroll
      for (int c = 0; c < 8; ++c)
        asm volatile(
            "{\n\t.reg .u32 lo, hi;\n\tmov.b64 {lo, hi}, %0;\n\tmad.wide.u32 %0, lo, %1, %0;\n\t}"
            : "+l"(w[c])
            : "r"(0xD2511F53u));
    } else if (kOp == SPIN_PIPE_MAD_HI) {
#pragma unroll
      for (int c = 0; c < 8; ++c)
        asm volatile("mad.hi.u32 %0, %0, %1, %2;" : "+r"(x[c]) : "r"(0xCD9E8D57u), "r"(0x9E3779B9u));
    } else if (kOp == SPIN_PIPE_LOP3) {
      uint32_t y[8];
#pragma unroll
      for (int c = 0; c < 8; ++c)
        asm volatile("lop3.b32 %0, %1, %2, %3, 0x96;"
                     : "=r"(y[c])
                     : "r"(x[c]), "r"(x[(c + 1) & 7]), "r"(x[(c + 2) & 7]));
#pragma unroll
      for (int c = 0; c < 8; ++c) x[c] = y[c];
    } else if (kOp == SPIN_PIPE_IADD3) {
      uint32_t y[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) y[c] = x[c] + x[(c + 1) & 7] + x[(c + 2) & 7];
#pragma unroll
      for (int c = 0; c < 8; ++c) x[c] = y[c];
    } else if (kOp == SPIN_PIPE_FFMA) {
#pragma unroll
      for (int c = 0; c < 8; ++c) f[c] = __fmaf_rn(f[c], 0.999f, 0.001f);
    } else {
#pragma unroll
      for (int c = 0; c < 8; ++c) asm volatile("rsqrt.approx.ftz.f32 %0, %0;" : "+f"(f[c]));
    }
  }
  __syncthreads();
  const long long t1 = clock64();
  uint32_t s = 0;
  float sum = 0.0f;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    if (kOp == SPIN_PIPE_MUL_WIDE)
      s ^= (uint32_t)w[c] ^ (uint32_t)(w[c] >> 32);
    else if (kOp >= SPIN_PIPE_FFMA)
      sum = __fadd_rn(sum, f[c]);
    else
      s ^= x[c];
  }
  sink[g] = kOp >= SPIN_PIPE_FFMA ? __float_as_uint(sum) : s;
  if (threadIdx.x == 0) {
    uint32_t smid;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
    clocks[3 * blockIdx.x] = t0;
    clocks[3 * blockIdx.x + 1] = t1;
    clocks[3 * blockIdx.x + 2] = smid;
  }
}

template <int kOp>
int launch_op(int bpsm, int sms, uint32_t iters, long long *clocks, uint32_t *sink, cudaStream_t s) {
  int fit = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, pipe_probe_kernel<kOp>, 256, 0) != cudaSuccess)
    return SPIN_ECUDA;
  if (fit < bpsm) return SPIN_EINVAL;
  pipe_probe_kernel<kOp><<<(unsigned)(sms * bpsm), 256, 0, s>>>(iters, clocks, sink);
  return cudaGetLastError() == cudaSuccess ? SPIN_OK : SPIN_ECUDA;
}

}  // namespace

int launch_pipe_probe(int op, int bpsm, uint32_t iters, long long *clocks, uint32_t *sink, int *sms_out,
                      cudaStream_t s) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return SPIN_ECUDA;
  if (sms_out) *sms_out = sms;
  switch (op) {
    case SPIN_PIPE_MUL_WIDE: return launch_op<SPIN_PIPE_MUL_WIDE>(bpsm, sms, iters, clocks, sink, s);
    case SPIN_PIPE_MAD_HI: return launch_op<SPIN_PIPE_MAD_HI>(bpsm, sms, iters, clocks, sink, s);
    case SPIN_PIPE_LOP3: return launch_op<SPIN_PIPE_LOP3>(bpsm, sms, iters, clocks, sink, s);
    case SPIN_PIPE_IADD3: return launch_op<SPIN_PIPE_IADD3>(bpsm, sms, iters, clocks, sink, s);
    case SPIN_PIPE_FFMA: return launch_op<SPIN_PIPE_FFMA>(bpsm, sms, iters, clocks, sink, s);
    case SPIN_PIPE_MUFU_RSQ: return launch_op<SPIN_PIPE_MUFU_RSQ>(bpsm, sms, iters, clocks, sink, s);
    default: return SPIN_EINVAL;
  }
}

}  // namespace spin
