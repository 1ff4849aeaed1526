// Device helpers shared by the kernels: digamma, exp(digamma), the
// per-element term of the variational bound, warp reductions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "nfhmm_kernels.h"

namespace nfhmm {

// psi(x) and w = exp(psi(x)) for x > 0, float.
// psi: recurrence psi(x) = psi(x + 1) - 1/x (Abramowitz & Stegun 6.3.5) up to
// x >= 6, then the asymptotic series psi(x) ~ ln x - 1/(2x) - sum_k
// B_2k / (2k x^2k) (A&S 6.3.18) through the x^-10 term.  w is formed as
// x' * exp(d - acc), where x' is the shifted argument, d = psi(x') - ln x'
// from the series and acc the recurrence sum, so no ln/exp round trip is
// needed for large x.  Returns NaN for x <= 0 or NaN.
__device__ __forceinline__ void digamma_exp(float x, float& psi, float& w) {
  if (!(x > 0.f)) {
    psi = __int_as_float(0x7fc00000);
    w = psi;
    return;
  }
  float acc = 0.f;
  // x > 0: the first step lands in [1, ...), five more reach x >= 6.
  // __frcp_rn: the correctly rounded reciprocal (same value as 1.f / x)
#pragma unroll 1
  for (int i = 0; i < 7 && x < 6.f; ++i) {
    acc += __frcp_rn(x);
    x += 1.f;
  }
  const float r = __frcp_rn(x);
  const float r2 = r * r;
  const float series =
      r2 * (1.f / 12.f -
            r2 * (1.f / 120.f - r2 * (1.f / 252.f - r2 * (1.f / 240.f - r2 * (1.f / 132.f)))));
  const float d = -0.5f * r - series;
  psi = logf(x) + d - acc;
  w = x * expf(d - acc);
}

__device__ __forceinline__ float digamma_f(float x) {
  float p, w;
  digamma_exp(x, p, w);
  return p;
}

// psi(x) in double for the per-frame terms of the bound (x >= 1 here).
// Same method as digamma_exp: recurrence to x >= 10, then A&S 6.3.18
// through the x^-14 term.
__device__ __forceinline__ double digamma_d(double x) {
  double acc = 0.0;
#pragma unroll 1
  for (int i = 0; i < 11 && x < 10.0; ++i) {
    acc += 1.0 / x;
    x += 1.0;
  }
  const double r = 1.0 / x;
  const double r2 = r * r;
  const double series =
      r2 * (1.0 / 12 -
            r2 * (1.0 / 120 -
                  r2 * (1.0 / 252 - r2 * (1.0 / 240 - r2 * (1.0 / 132 - r2 * (691.0 / 32760 - r2 / 12))))));
  return log(x) - 0.5 * r - series - acc;
}

// g(a) = lnGamma(a) - (a - 1) psi(a), the per-element part of the bound's
// entropy term, accumulated by the caller in double.  For a >= 4 the value
// is returned as (h(a), -a) with h(a) = g(a) + a evaluated by its
// asymptotic series (from Stirling's series for lnGamma and A&S 6.3.18):
//   h(a) = 1/2 ln a + 1/2 ln(2 pi) + 1/2 - 1/(3a) - 1/(12a^2) - 1/(90a^3)
//          + 1/(120a^4) + 1/(210a^5) - 1/(252a^6) - 1/(210a^7) + 1/(240a^8)
// so that the large, cancelling a ln a parts never meet in float.
__device__ __forceinline__ double bound_g_elem(float a) {
  if (a < 4.f) {
    return (double)(lgammaf(a) - (a - 1.f) * digamma_f(a));
  }
  const float r = __frcp_rn(a);
  const float poly =
      r * (-1.f / 3.f +
           r * (-1.f / 12.f +
                r * (-1.f / 90.f +
                     r * (1.f / 120.f +
                          r * (1.f / 210.f + r * (-1.f / 252.f + r * (-1.f / 210.f + r * (1.f / 240.f))))))));
  const float h = 0.5f * logf(a) + 1.4189385332046727f + poly;
  return (double)h - (double)a;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// tf32 split: hi = x rounded to tf32 (10 explicit mantissa bits, round to
// nearest with ties away from zero: cvt.rna.tf32.f32), lo = x - hi (exact in
// float) rounded again.  The tensor core reads only the tf32 bits of each
// operand, so hi*hi + hi*lo + lo*hi recovers ~22 bits of each product.
__device__ __forceinline__ float tf32_hi(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

}  // namespace nfhmm
