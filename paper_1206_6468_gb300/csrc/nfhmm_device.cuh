// Device helpers shared by the kernels: digamma, exp(digamma), the
// per-element term of the variational bound, warp reductions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "nfhmm_kernels.h"

namespace nfhmm {

// psi(x) and w = exp(psi(x)) for x > 0, float.
// psi: recurrence psi(x) = psi(x + 1) - 1/x (Abramowitz & Stegun 6.3.5) up to
// x >= 3 (the reciprocals summed as one fraction), then the asymptotic series
// psi(x) ~ ln x - 1/(2x) - sum_k B_2k / (2k x^2k) (A&S 6.3.18) through the
// x^-14 term (truncation below 1.1e-8 at x = 3).  w is formed as
// x' * exp(d - acc), where x' is the shifted argument, d = psi(x') - ln x'
// from the series and acc the recurrence sum, so no ln/exp round trip is
// needed for large x.  Returns NaN for x <= 0 or NaN.  (A float32 emulation
// over the accuracy test's arguments: 2.4e-7 in psi / (1 + |psi|) against
// 5.3e-7 with the shift to 6, as fewer recurrence steps are rounded.)
template <bool G, bool FAST = false>
__device__ __forceinline__ void digamma_impl(float x, float& psi, float& w, float& gsmall,
                                             float& gbig) {
  if (!(x > 0.f)) {
    psi = __int_as_float(0x7fc00000);
    w = psi;
    if (G) gsmall = gbig = psi;
    return;
  }
  const float a = x;
  // at most three steps reach x >= 3 (x > 0).  The recurrence sum
  // acc = sum_i 1/(x+i) is kept as one fraction num/den
  // (num' = num (x+i) + den, den' = den (x+i)), so the shift costs one
  // reciprocal instead of one per step; den is also the product
  // (x)(x+1)...(x+n-1) of the lnGamma shift.
  float num = 0.f, prod = 1.f;
  int n = 0;
#pragma unroll 1
  for (; n < 7 && x < 3.f; ++n) {
    num = fmaf(num, x, prod);
    prod *= x;
    x += 1.f;
  }
  // FAST: the hardware's approximate reciprocal (within 1 ulp; the shifted x
  // is >= 3 and prod >= 1 here, so neither is subnormal); otherwise the
  // correctly rounded one
  float rp_, rx_;
  if (FAST) {
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rp_) : "f"(prod));
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rx_) : "f"(x));
  } else {
    rp_ = __frcp_rn(prod);
    rx_ = __frcp_rn(x);
  }
  const float acc = n > 0 ? num * rp_ : 0.f;
  const float r = rx_;
  const float r2 = r * r;
  const float series =
      r2 * (1.f / 12.f -
            r2 * (1.f / 120.f -
                  r2 * (1.f / 252.f -
                        r2 * (1.f / 240.f -
                              r2 * (1.f / 132.f - r2 * (691.f / 32760.f - r2 * (1.f / 12.f)))))));
  const float d = -0.5f * r - series;
  // FAST: psi and w from the hardware log2/exp2 approximations (x >= 3 here,
  // d - acc in (-3, 0): within a few 1e-7 relative) and the approximate
  // reciprocals above -- the weights kernel of every sweep, so that forming
  // the bound does not change the state; the bound's own terms and every
  // other caller take the correctly rounded ones
  const float lx = FAST ? __logf(x) : logf(x);
  psi = lx + d - acc;
  w = x * (FAST ? __expf(d - acc) : expf(d - acc));
  if (G) {
    const float lxg = FAST ? logf(x) : lx;
    const float st =
        r * (1.f / 12.f -
             r2 * (1.f / 360.f -
                   r2 * (1.f / 1260.f -
                         r2 * (1.f / 1680.f - r2 * (1.f / 1188.f - r2 * (691.f / 360360.f))))));
    gsmall = ((float)n + 0.5f) * lxg + 0.91893853320467274f + st - logf(prod) -
             (a - 1.f) * (d - acc);
    gbig = -((float)n + a);
  }
}

__device__ __forceinline__ void digamma_exp(float x, float& psi, float& w) {
  float unused0, unused1;
  digamma_impl<false>(x, psi, w, unused0, unused1);
}
// the same with the hardware log2/exp2 approximations (the weights kernel)
__device__ __forceinline__ void digamma_exp_fast(float x, float& psi, float& w) {
  float unused0, unused1;
  digamma_impl<false, true>(x, psi, w, unused0, unused1);
}

// digamma_exp plus the bound's per-element term g(x) = lnGamma(x) - (x-1) psi(x)
// from the same shifted argument x' = x + n (n recurrence steps): with
// Stirling's series lnGamma(x') = (x' - 1/2) ln x' - x' + ln(2 pi)/2 + st(x'),
// st = 1/(12x') - 1/(360x'^3) + 1/(1260x'^5) - 1/(1680x'^7) + 1/(1188x'^9)
//      - 691/(360360x'^11), and lnGamma(x) = lnGamma(x') - ln(x (x+1) ... (x+n-1)),
//   g(x) = (n + 1/2) ln x' + ln(2 pi)/2 + st - ln(prod) - (x-1)(d - acc) - x'
// where d - acc is the series part of psi.  The large part -x' = -(x + n) is
// returned separately (gbig, exact in double) so that no float sum holds it.
__device__ __forceinline__ void digamma_exp_g(float x, float& psi, float& w, float& gsmall,
                                              float& gbig) {
  digamma_impl<true, true>(x, psi, w, gsmall, gbig);   // psi, w as digamma_exp_fast
}
// The two above for arguments >= 1 as a rule (alpha-hat of Eq. 6 is counts +
// gamma d-hat + 1, every term >= 0; the weights kernel): always two
// recurrence steps, x' = x + 2 >= 3, straight-line -- the recurrence sum and
// the lnGamma shift product in closed form,
//   acc = 1/x + 1/(x+1) = (2x + 1) / (x (x + 1)),   prod = x (x + 1),
// one approximate reciprocal for acc and one for the series at x', which is
// that of digamma_impl (FAST).  digamma_ge1_straight is the closed form alone,
// for callers that have checked 1 <= x < 2^60 themselves (from 2^60 on,
// x (x + 1) leaves float's range); digamma_ge1_fast sends other arguments
// (below 1, from 2^60 on, NaN, <= 0) to digamma_impl.  (A float32 emulation
// over the accuracy test's arguments, correctly rounded reciprocals, log and
// exp: 2.4e-7 in psi / (1 + |psi|), 3.2e-7 relative in w.)
template <bool G>
__device__ __forceinline__ void digamma_ge1_straight(float x, float& psi, float& w, float& gsmall,
                                                     float& gbig) {
  const float a = x;
  const float prod = fmaf(x, x, x);
  const float num = fmaf(2.f, x, 1.f);
  x += 2.f;
  float rp, r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rp) : "f"(prod));
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  const float acc = num * rp;
  const float r2 = r * r;
  const float series =
      r2 * (1.f / 12.f -
            r2 * (1.f / 120.f -
                  r2 * (1.f / 252.f -
                        r2 * (1.f / 240.f -
                              r2 * (1.f / 132.f - r2 * (691.f / 32760.f - r2 * (1.f / 12.f)))))));
  const float d = -0.5f * r - series;
  psi = __logf(x) + d - acc;
  w = x * __expf(d - acc);
  if (G) {
    const float st =
        r * (1.f / 12.f -
             r2 * (1.f / 360.f -
                   r2 * (1.f / 1260.f -
                         r2 * (1.f / 1680.f - r2 * (1.f / 1188.f - r2 * (691.f / 360360.f))))));
    gsmall = 2.5f * logf(x) + 0.91893853320467274f + st - logf(prod) - (a - 1.f) * (d - acc);
    gbig = -(2.f + a);
  }
}
template <bool G>
__device__ __forceinline__ void digamma_ge1_fast(float x, float& psi, float& w, float& gsmall,
                                                 float& gbig) {
  if (x >= 1.f && x < 0x1p60f)
    digamma_ge1_straight<G>(x, psi, w, gsmall, gbig);
  else
    digamma_impl<G, true>(x, psi, w, gsmall, gbig);
}
__device__ __forceinline__ void digamma_exp_fast_ge1(float x, float& psi, float& w) {
  float unused0, unused1;
  digamma_ge1_fast<false>(x, psi, w, unused0, unused1);
}
__device__ __forceinline__ void digamma_exp_g_ge1(float x, float& psi, float& w, float& gsmall,
                                                  float& gbig) {
  digamma_ge1_fast<true>(x, psi, w, gsmall, gbig);
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

// Programmatic dependent launch: wait for the grids this one depends on
// (no-op without such a dependency); let dependent grids be scheduled.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
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
