// The Metropolis step of one Heisenberg site (Sec. 4), shared by every
// Heisenberg sweep kernel so that a chain is the same bit for bit whichever
// kernel (per-phase, colour-split, double-checkerboard, resident) ran it.
#pragma once
#include "common.cuh"

namespace spin {

// Uniform unit vector from two uniforms: z = 2 u1 - 1, phi = 2 pi u2.
// sin/cos of 2 pi u2 are evaluated as sincospi(2 u2): 2 u2 is exact, so the
// argument reduction is exact too.  kFast selects the hardware
// approximations (the paper's "fast_math" mode, Sec. 4).
template <bool kFast>
__device__ __forceinline__ float4 unit_vector(uint32_t w1, uint32_t w2) {
  const float z = 2.0f * uniform24(w1) - 1.0f;
  const float rho = sqrtf(fmaxf(0.0f, 1.0f - z * z));
  float sn, cs;
  if (kFast) {
    __sincosf(6.28318530717958647692f * uniform24(w2), &sn, &cs);
  } else {
    sincospif(2.0f * uniform24(w2), &sn, &cs);
  }
  return make_float4(rho * cs, rho * sn, z, 0.0f);
}

// The Metropolis step of one site (Sec. 4) from its spin si, the sum h of
// its neighbours and its Philox call w: proposal n from words 0 and 1,
// acceptance from word 2, dE = -(n - si) . h; returns whether n is taken.
// kFast = false: the library's full-accuracy FP32 functions (sqrtf, sincospif,
// expf).  kFast = true, the paper's fast-math mode: rho = sqrt(1 - z^2) as
// s2 rsqrt(s2), sin and cos of phi = 2 pi u2 from the hardware sin and cos of
// phi - pi in [-pi, pi) (negated), and u3 < exp(-beta dE) tested as
// (w2 >> 8) < 2^(24 - beta log2(e) dE) with the hardware exp2 (beta_l2e =
// beta log2(e) from the host).  Every kernel of one variant calls this, so a
// chain does not depend on which kernel or call length ran it.
template <bool kFast>
__device__ __forceinline__ bool heis_step(const float4 &si, float hx, float hy, float hz, const uint4 &w,
                                          float beta, float beta_l2e, float4 &n) {
  if (!kFast) {
    n = unit_vector<false>(w.x, w.y);
    const float u3 = uniform24(w.z);
    const float dE = (si.x - n.x) * hx + (si.y - n.y) * hy + (si.z - n.z) * hz;
    return dE <= 0.0f || u3 < expf(-beta * dE);
  }
  const float z = fmaf(__uint2float_rn(w.x >> 8), 1.1920928955078125e-7f, -1.0f);  // 2 u1 - 1
  const float s2 = fmaf(-z, z, 1.0f);
  // the hardware approximations in their flush-to-zero forms: every input and
  // output here is 0 or a normal number (s2 >= 1e-30; xa = (k - 2^23) c with
  // c = fl(2 pi 2^-24), so |xa| is 0 or >= c, and the sine and cosine of such
  // angles are 0 or above 1e-8), so they equal the non-flushing forms and
  // skip their denormal handling
  float rs, sn, cs;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(rs) : "f"(fmaxf(s2, 1e-30f)));
  const float rho = s2 * rs;
  const float xa = fmaf(__uint2float_rn(w.y >> 8), 3.7450702663161573e-7f, -3.14159265358979f);
  asm("sin.approx.ftz.f32 %0, %1;" : "=f"(sn) : "f"(xa));
  asm("cos.approx.ftz.f32 %0, %1;" : "=f"(cs) : "f"(xa));
  n = make_float4(-rho * cs, -rho * sn, z, 0.0f);
  const float dE = (si.x - n.x) * hx + (si.y - n.y) * hy + (si.z - n.z) * hz;
  float p;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(p) : "f"(fmaf(-beta_l2e, dE, 24.0f)));
  return dE <= 0.0f || __uint2float_rn(w.z >> 8) < p;
}

}  // namespace spin
