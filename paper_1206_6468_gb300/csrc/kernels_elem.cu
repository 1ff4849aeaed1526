// Elementwise and reduction kernels of the sweep:
//  * the weights kernel: Eq. 6 (alpha-hat), psi and w = exp(psi) (the
//    weights of Eq. 7), and Eq. 8 (phi-hat) as a warp-shuffle segmented
//    reduction over each dictionary's K consecutive elements;
//  * the bound reduction (FP64 accumulation);
//  * initialisation, validation, layout and separation helpers.
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>
#include <climits>
#include <type_traits>
#include <utility>

#include "nfhmm_device.cuh"
#include "nfhmm_kernels.h"

namespace nfhmm {

constexpr unsigned FULL = 0xffffffffu;

// ------------------------------------------------------------ weights (Eq. 6, 8)
// Per element: alpha-hat (Eq. 6), psi and w = exp(psi) (the weights of
// Eq. 7), written as float and as the contraction's operand format; per
// dictionary block (s, n): Eq. 8's sum of psi over its K consecutive
// elements, in a fixed order (deterministic, no atomics).  d-hat and
// phi-hat are S x Tstride x N.  With BOUND, the kernel also sums alpha-hat
// and the bound's element terms g(alpha) (Kahan-compensated in float per
// lane, then double) into fterm[t][h] for unit h of the frame.
//
// Units: WB consecutive blocks g = (s, n) of one frame t (WB*K consecutive
// elements).  Dictionaries of K <= 16 elements take the slab form below;
// larger ones this per-unit form, one warp per unit: each lane takes every
// 32nd element of the unit (coalesced loads and stores; the element table
// ktab[k] = (s, n) of element k in place of integer division), forms
// alpha-hat, psi and w, and parks psi in shared memory; then lane b sums the
// K values of the unit's block b in element order.  (Forms with four
// consecutive elements per lane and
// 16-byte vectors -- a warp per frame, or per segment of whole blocks --
// measured slower on GB300: fewer resident warps for the same work.)
constexpr int WB = 16;

template <int FMT, bool BOUND>
__device__ __forceinline__ void weights_elem(float alpha, float& psi, float& w, float& sa,
                                             float& ca, float& sg, float& cg, double& big) {
  if (BOUND) {
    float gs, gb;
    digamma_exp_g_ge1(alpha, psi, w, gs, gb);
    float y = alpha - ca, z = sa + y;
    ca = (z - sa) - y;
    sa = z;
    y = gs - cg;
    z = sg + y;
    cg = (z - sg) - y;
    sg = z;
    big += (double)gb;
  } else {
    digamma_exp_fast_ge1(alpha, psi, w);
  }
}

// WIDE: unit indices in 64 bits (frames x units per frame beyond 2^31)
template <int FMT, bool BOUND, bool WIDE>
__global__ void __launch_bounds__(256) k_weights(WeightsArgs a) {
  extern __shared__ float wsm[];
  griddep_wait();
  griddep_launch_dependents();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int NB = a.S * a.N;                 // blocks per frame
  const int NH = (NB + WB - 1) / WB;        // units per frame
  using U = typename std::conditional<WIDE, unsigned long long, unsigned>::type;
  const U u = (U)blockIdx.x * (blockDim.x >> 5) + warp;
  if (u >= (U)a.T * NH) return;             // whole warps
  const int t = (int)(u / (U)NH), h = (int)(u - (U)t * NH);
  const int UE = WB * a.K;
  const int k0 = h * UE, k1 = min(k0 + UE, a.M);
  const size_t SN = (size_t)a.Tstride * a.N;
  float* ps = wsm + warp * UE;
  const size_t row = (size_t)t * a.Mp;
  const size_t toff = (size_t)t * a.N;
  unsigned bad = 0;
  float chk = 0.f;
  float sa = 0.f, ca = 0.f, sg = 0.f, cg = 0.f;   // Kahan sums of alpha and g (small part)
  double big = 0.0;                                // sum of the exact large parts of g
  for (int k = k0 + lane; k < k1; k += 32) {
    const int2 e = a.ktab[k];
    const float alpha = a.counts[row + k] + a.gamma * a.dhat[(size_t)e.x * SN + toff + e.y] + 1.f;
    float psi, w;
    weights_elem<FMT, BOUND>(alpha, psi, w, sa, ca, sg, cg, big);
    chk = fmaf(0.f, psi + w, chk);   // stays 0 unless psi or w is NaN or infinite
    if (a.alpha) a.alpha[row + k] = alpha;
    a.w32[row + k] = w;
    if (FMT == WF_TF32X2) {
      const float hi = tf32_hi(w);
      reinterpret_cast<float*>(a.wop_hi)[row + k] = hi;
      reinterpret_cast<float*>(a.wop_lo)[row + k] = tf32_hi(w - hi);
    } else if (FMT == WF_BF16) {
      reinterpret_cast<__nv_bfloat16*>(a.wop_hi)[row + k] = __float2bfloat16_rn(w);
    }
    ps[k - k0] = psi;
  }
  __syncwarp();
  const int b = h * WB + lane;
  if (lane < WB && b < NB) {
    const float* pb = ps + lane * a.K;
    float x = 0.f;
    for (int j = 0; j < a.K; ++j) x += pb[j];
    const int2 e = a.ktab[b * a.K];
    a.phi[(size_t)e.x * SN + toff + e.y] = a.gamma * x;
  }
  if (!(chk == 0.f)) bad |= ERR_NONFINITE;
  bad = __reduce_or_sync(FULL, bad);
  if (bad && lane == 0) atomicOr(a.err, bad);
  if (BOUND) {
    const double s0 = warp_sum_d((double)sa - (double)ca);
    const double sgt = warp_sum_d(((double)sg - (double)cg) + big);
    if (lane == 0) {
      a.fterm[2 * (size_t)u] = s0;
      a.fterm[2 * (size_t)u + 1] = sgt;
    }
  }
}

// Slab form, for dictionaries of K <= 16 elements (a unit of at most 256
// elements, at most SLAB_EPL = 8 per lane): a warp walks `upw` consecutive
// units, frame after frame, with the next unit's counts and d-hat loads in
// flight while it forms the current one; the index arithmetic is done once
// per warp and the addresses once per unit.  Lane l takes elements l + 32 j
// of a unit, as above; lanes 2b and 2b + 1 load block b's d-hat value, and an
// element's value comes from lane 2 ((l + 32 j) / K) by one shuffle.  When
// every alpha-hat of the unit lies in [1, 2^60) -- always, for a valid state
// -- one warp vote sends the unit down the straight-line psi (no fallback
// branch, no NaN test: psi and w are finite there); otherwise the general
// psi with the NaN test (with BOUND, both forms also sum alpha-hat and the
// bound's element terms).  Eq. 8: lanes 2b and 2b + 1 sum the first
// ceil(K/2) and the last floor(K/2) of block b's psi values (shared memory,
// element order), and the two halves are added.  KT: K as a compile-time
// constant (1..16), or 0 for any K <= 16 at run time.
constexpr int SLAB_EPL = 8;
constexpr int SLAB_MAX_K = SLAB_EPL * 32 / WB;

template <int FMT, bool BOUND, int KT>
__global__ void __launch_bounds__(256, (BOUND || KT == 0) ? 2 : KT <= 10 ? 4 : 3)
    k_weights_slab(WeightsArgs a) {
  constexpr int EPL = KT > 0 ? (WB * KT + 31) / 32 : SLAB_EPL;
  extern __shared__ float wsm[];
  griddep_wait();
  griddep_launch_dependents();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int K = KT > 0 ? KT : a.K;
  const int N = a.N, NB = a.S * N, NH = (NB + WB - 1) / WB, UE = WB * K;
  const long long nunits = (long long)a.T * NH;
  const long long ub = ((long long)blockIdx.x * (blockDim.x >> 5) + warp) * a.upw;
  if (ub >= nunits) return;   // whole warps
  const int nu = (int)min((long long)a.upw, nunits - ub);
  int t = nunits < (1ll << 31) ? (int)((unsigned)ub / (unsigned)NH) : (int)(ub / NH);
  int h = (int)(ub - (long long)t * NH);
  const size_t SN = (size_t)a.Tstride * N;
  float* ps = wsm + warp * UE;
  // shuffle source of this lane's element j: lane 2 ((lane + 32 j) / K)
  int src[EPL];
#pragma unroll
  for (int j = 0; j < EPL; ++j)
    src[j] = KT > 0 ? 2 * ((lane + 32 * j) / KT)
                    : 2 * (int)(((unsigned)(lane + 32 * j) * a.kdiv) >> 16);
  const int hk = (K + 1) >> 1;
  const int jn = (lane & 1) ? K - hk : hk;   // psi values this lane sums
  const float* psb = ps + (lane >> 1) * K + ((lane & 1) ? hk : 0);
  float chk = 0.f;

  // counts and d-hat of unit (tu, hu); off: the d-hat (and phi-hat) offset of
  // this lane's block, -1 past the frame's last block
  auto load = [&](int tu, int hu, float* c, float& d, long long& off, int& nk, size_t& ro) {
    const int k0 = hu * UE;
    nk = min(UE, a.M - k0);
    ro = (size_t)tu * a.Mp + k0;
    const float* cp = a.counts + ro + lane;
#pragma unroll
    for (int j = 0; j < EPL; ++j) c[j] = lane + 32 * j < nk ? __ldg(cp + 32 * j) : 0.f;
    const int g = hu * WB + (lane >> 1);
    off = -1;
    d = 0.f;
    if (g < NB) {
      const int sg = (int)(((unsigned long long)g * a.ndiv) >> 32);
      off = (long long)sg * (long long)SN + (long long)tu * N + (g - sg * N);
      d = __ldg(a.dhat + off);
    }
  };
  auto process = [&](int tu, int hu, const float* c, float d, long long off, int nk, size_t ro) {
    float* pw = a.w32 + ro + lane;
    float* ph = FMT == WF_TF32X2 ? reinterpret_cast<float*>(a.wop_hi) + ro + lane : nullptr;
    float* pl = FMT == WF_TF32X2 ? reinterpret_cast<float*>(a.wop_lo) + ro + lane : nullptr;
    __nv_bfloat16* pb =
        FMT == WF_BF16 ? reinterpret_cast<__nv_bfloat16*>(a.wop_hi) + ro + lane : nullptr;
    float* pa = a.alpha ? a.alpha + ro + lane : nullptr;
    float al[EPL];
    unsigned span = 0u;   // largest bits(alpha) - bits(1): below bits(2^60) - bits(1) iff all in range
#pragma unroll
    for (int j = 0; j < EPL; ++j) {
      if (KT == 0 && 32 * j >= nk) break;   // warp-uniform
      const float dj = __shfl_sync(FULL, d, src[j]);
      al[j] = c[j] + a.gamma * dj + 1.f;
      span = max(span, __float_as_uint(al[j]) - 0x3f800000u);
    }
    const bool fast = __all_sync(FULL, span < 0x1e000000u);
    float sa = 0.f, ca = 0.f, sgk = 0.f, cg = 0.f;
    double big = 0.0;
#pragma unroll
    for (int j = 0; j < EPL; ++j) {
      if (KT == 0 && 32 * j >= nk) break;
      const int e = lane + 32 * j;
      if (e < nk) {
        float psi, w;
        if (fast) {
          float gs, gb;
          digamma_ge1_straight<BOUND>(al[j], psi, w, gs, gb);
          if (BOUND) {   // Kahan sums of alpha and of g's small part, as weights_elem
            float y = al[j] - ca, z = sa + y;
            ca = (z - sa) - y;
            sa = z;
            y = gs - cg;
            z = sgk + y;
            cg = (z - sgk) - y;
            sgk = z;
            big += (double)gb;
          }
        } else {
          weights_elem<FMT, BOUND>(al[j], psi, w, sa, ca, sgk, cg, big);
          chk = fmaf(0.f, psi + w, chk);   // stays 0 unless psi or w is NaN or infinite
        }
        if (pa) pa[32 * j] = al[j];
        pw[32 * j] = w;
        if (FMT == WF_TF32X2) {
          const float hi = tf32_hi(w);
          ph[32 * j] = hi;
          pl[32 * j] = tf32_hi(w - hi);
        } else if (FMT == WF_BF16) {
          pb[32 * j] = __float2bfloat16_rn(w);
        }
        ps[e] = psi;
      }
    }
    __syncwarp();
    float x = 0.f;
    if (off >= 0) {
      if (KT > 0) {
#pragma unroll
        for (int j = 0; j < (KT + 1) / 2; ++j)
          if (j < jn) x += psb[j];
      } else {
        for (int j = 0; j < jn; ++j) x += psb[j];
      }
    }
    x += __shfl_xor_sync(FULL, x, 1);
    if (off >= 0 && !(lane & 1)) a.phi[off] = a.gamma * x;
    if (BOUND) {
      const double s0 = warp_sum_d((double)sa - (double)ca);
      const double sgt = warp_sum_d(((double)sgk - (double)cg) + big);
      if (lane == 0) {
        const size_t u = (size_t)tu * NH + hu;
        a.fterm[2 * u] = s0;
        a.fterm[2 * u + 1] = sgt;
      }
    }
    __syncwarp();   // every lane's sums read before the next unit's psi
  };

  // two register sets: unit i in one while unit i + 1 loads into the other
  float c0[EPL], c1[EPL], d0, d1;
  long long o0, o1;
  int n0, n1;
  size_t r0, r1;
  load(t, h, c0, d0, o0, n0, r0);
  for (int i = 0;;) {
    int tn = t, hn = h + 1;
    if (hn == NH) {
      hn = 0;
      ++tn;
    }
    if (i + 1 < nu) load(tn, hn, c1, d1, o1, n1, r1);
    process(t, h, c0, d0, o0, n0, r0);
    if (++i >= nu) break;
    t = tn;
    h = hn;
    tn = t;
    hn = h + 1;
    if (hn == NH) {
      hn = 0;
      ++tn;
    }
    if (i + 1 < nu) load(tn, hn, c0, d0, o0, n0, r0);
    process(t, h, c1, d1, o1, n1, r1);
    if (++i >= nu) break;
    t = tn;
    h = hn;
  }
  unsigned bad = !(chk == 0.f) ? ERR_NONFINITE : 0u;
  bad = __reduce_or_sync(FULL, bad);
  if (bad && lane == 0) atomicOr(a.err, bad);
}

// the slab kernels with K fixed at compile time, by K - 1
template <int FMT, bool BOUND, int... KS>
static void (*slab_fixed_k(int K, std::integer_sequence<int, KS...>))(WeightsArgs) {
  void (*const tab[])(WeightsArgs) = {k_weights_slab<FMT, BOUND, KS + 1>...};
  return tab[K - 1];
}

int weights_units(int S, int N, int K, int T) {
  (void)K;
  (void)T;
  return (S * N + WB - 1) / WB;
}

__global__ void k_element_table(int M, int Mp, int K, int N, int2* ktab) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= Mp) return;
  if (k < M) {
    const int g = k / K, s = g / N, n = g - s * N;
    ktab[k] = make_int2(s, n);
  } else {
    ktab[k] = make_int2(0, 0);   // padding: a valid index, never used for a result
  }
}
void launch_element_table(int M, int Mp, int K, int N, int2* ktab, cudaStream_t st) {
  k_element_table<<<(Mp + 255) / 256, 256, 0, st>>>(M, Mp, K, N, ktab);
}

// multiprocessors of the current device (cached per device)
static int device_sms() {
  static int sms[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return 148;
  if (sms[dev] == 0) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    sms[dev] = v > 0 ? v : 148;
  }
  return sms[dev];
}

void launch_weights(const WeightsArgs& a_in, int fmt, cudaStream_t st) {
  WeightsArgs a = a_in;
  const bool b = a.fterm != nullptr;
  void (*k)(WeightsArgs) = nullptr;
  cudaLaunchConfig_t cfg = {};
  if (a.K <= SLAB_MAX_K) {
    // slab form: enough units per warp that the grid is about one wave of
    // 64 warps per multiprocessor (at least one unit, at most 16)
    const int warps = 8;
    const long long units = (long long)a.T * ((a.S * a.N + WB - 1) / WB);
    const long long wave = (long long)device_sms() * 64;
    a.upw = (int)std::max(1ll, std::min(16ll, (units + wave - 1) / wave));
    a.kdiv = (65536u + (unsigned)a.K - 1u) / (unsigned)a.K;
    a.ndiv = ((1ull << 32) + (unsigned long long)a.N - 1ull) / (unsigned long long)a.N;
    const auto ks = std::make_integer_sequence<int, SLAB_MAX_K>{};
    switch (fmt) {
      case WF_TF32X2:
        k = b ? slab_fixed_k<WF_TF32X2, true>(a.K, ks) : slab_fixed_k<WF_TF32X2, false>(a.K, ks);
        break;
      case WF_BF16:
        k = b ? slab_fixed_k<WF_BF16, true>(a.K, ks) : slab_fixed_k<WF_BF16, false>(a.K, ks);
        break;
      default:
        k = b ? k_weights_slab<WF_F32, true, 0> : k_weights_slab<WF_F32, false, 0>;
        break;
    }
    const long long nwarps = (units + a.upw - 1) / a.upw;
    cfg.gridDim = dim3((unsigned)((nwarps + warps - 1) / warps));
    cfg.blockDim = dim3(warps * 32);
    cfg.dynamicSmemBytes = (size_t)warps * WB * a.K * sizeof(float);
  } else {
    const int warps = 8;
    const long long units = (long long)a.T * ((a.S * a.N + WB - 1) / WB);
    const bool wide = units >= (1ll << 31);
    switch (fmt) {
      case WF_TF32X2:
        k = b ? (wide ? k_weights<WF_TF32X2, true, true> : k_weights<WF_TF32X2, true, false>)
              : (wide ? k_weights<WF_TF32X2, false, true> : k_weights<WF_TF32X2, false, false>);
        break;
      case WF_BF16:
        k = b ? (wide ? k_weights<WF_BF16, true, true> : k_weights<WF_BF16, true, false>)
              : (wide ? k_weights<WF_BF16, false, true> : k_weights<WF_BF16, false, false>);
        break;
      default:
        k = b ? (wide ? k_weights<WF_F32, true, true> : k_weights<WF_F32, true, false>)
              : (wide ? k_weights<WF_F32, false, true> : k_weights<WF_F32, false, false>);
        break;
    }
    cfg.gridDim = dim3((unsigned)((units + warps - 1) / warps));
    cfg.blockDim = dim3(warps * 32);
    cfg.dynamicSmemBytes = (size_t)warps * WB * a.K * sizeof(float);
  }
  if (a.T == 0) return;
  // a programmatic dependent of the previous kernel on the stream (ordinary
  // launch on the legacy default stream)
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  const bool legacy = st == nullptr || st == cudaStreamLegacy;
  cfg.attrs = legacy ? nullptr : attr;
  cfg.numAttrs = legacy ? 0 : 1;
  cudaLaunchKernelEx(&cfg, k, a);
}

// ------------------------------------------------------------------- fills
__global__ void k_fill_rows(float* buf, int T, int M, int ld, float value) {
  const size_t n = (size_t)T * ld;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(i % ld);
    buf[i] = k < M ? value : 0.f;
  }
}
void launch_fill_rows(float* buf, int T, int M, int ld, float value, cudaStream_t st) {
  const size_t n = (size_t)T * ld;
  int blocks = (int)((n + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  k_fill_rows<<<blocks, 256, 0, st>>>(buf, T, M, ld, value);
}
void launch_fill(float* buf, size_t n, float value, cudaStream_t st) {
  int blocks = (int)((n + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  k_fill_rows<<<blocks, 256, 0, st>>>(buf, 1, (int)n, (int)n, value);
}

// ---------------------------------------------------------------- row sums
__global__ void k_row_sums(const float* V, int T, int F, int Fp, double* v) {
  const int lane = threadIdx.x & 31;
  const int t = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (t >= T) return;
  double s = 0.0;
  for (int l = lane; l < F; l += 32) s += (double)V[(size_t)t * Fp + l];
  s = warp_sum_d(s);
  if (lane == 0) v[t] = s;
}
void launch_row_sums(const float* V, int T, int F, int Fp, double* v, cudaStream_t st) {
  k_row_sums<<<(T + 7) / 8, 256, 0, st>>>(V, T, F, Fp, v);
}

// -------------------------------------------------------------- validation
// One warp per row of W, A or pi (rows must be >= 0 and sum to 1 within 1e-4);
// grid-stride over V (finite, >= 0).
__global__ void k_validate(const float* V, int T, int F, int Fp, const float* W, int M,
                           const float* A, const float* pi, int S, int N, unsigned* err) {
  const int lane = threadIdx.x & 31;
  const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int nw = gridDim.x * (blockDim.x >> 5);
  unsigned bad = 0;
  const int rowsW = M, rowsA = S * N, rowsP = S;
  for (int r = gw; r < rowsW + rowsA + rowsP; r += nw) {
    const float* row;
    int len;
    if (r < rowsW) {
      row = W + (size_t)r * Fp;
      len = F;
    } else if (r < rowsW + rowsA) {
      row = A + (size_t)(r - rowsW) * N;
      len = N;
    } else {
      row = pi + (size_t)(r - rowsW - rowsA) * N;
      len = N;
    }
    double s = 0.0;
    unsigned b = 0;
    for (int i = lane; i < len; i += 32) {
      const float x = row[i];
      if (!(x >= 0.f) || !isfinite(x)) b = 1;
      s += (double)x;
    }
    s = warp_sum_d(s);
    b = __reduce_or_sync(FULL, b);
    if (b || fabs(s - 1.0) > 1e-4) bad = 1;
  }
  const size_t nv = (size_t)T * F;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nv;
       i += (size_t)gridDim.x * blockDim.x) {
    const float x = V[(i / F) * Fp + (i % F)];
    if (!(x >= 0.f) || !isfinite(x)) bad = 1;
  }
  bad = __reduce_or_sync(FULL, bad);
  if (bad && lane == 0) atomicOr(err, ERR_BAD_INPUT);
}
void launch_validate(const float* V, int T, int F, int Fp, const float* W, int M, const float* A,
                     const float* pi, int S, int N, unsigned* err, cudaStream_t st) {
  k_validate<<<256, 256, 0, st>>>(V, T, F, Fp, W, M, A, pi, S, N, err);
}

// --------------------------------------------------------------- transpose
__global__ void k_transpose(const float* in, int R, int Cc, int ldi, float* out, int ldo, int Rp,
                            int Cp) {
  __shared__ float tile[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    tile[i][threadIdx.x] = (r < R && c < Cc) ? in[(size_t)r * ldi + c] : 0.f;
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int c = c0 + i, r = r0 + threadIdx.x;
    if (c < Cp && r < Rp) out[(size_t)c * ldo + r] = tile[threadIdx.x][i];
  }
}
void launch_transpose(const float* in, int R, int Cc, int ldi, float* out, int ldo, int Rp, int Cp,
                      cudaStream_t st) {
  dim3 grid((Cp + 31) / 32, (Rp + 31) / 32);
  k_transpose<<<grid, dim3(32, 8), 0, st>>>(in, R, Cc, ldi, out, ldo, Rp, Cp);
}

// dst[r][l] = src[r][l] for l < F, 0 for F <= l < Fp: rows of F floats,
// packed, into rows of Fp (the frame store's padded layout).
__global__ void k_pad_rows(const float* src, int rows, int F, float* dst, int Fp) {
  const size_t n = (size_t)rows * Fp;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const size_t r = i / Fp;
    const int l = (int)(i - r * Fp);
    dst[i] = l < F ? src[r * F + l] : 0.f;
  }
}
void launch_pad_rows(const float* src, int rows, int F, float* dst, int Fp, cudaStream_t st) {
  const size_t n = (size_t)rows * Fp;
  const int blocks = (int)std::min<size_t>(8192, (n + 255) / 256);
  if (blocks > 0) k_pad_rows<<<blocks, 256, 0, st>>>(src, rows, F, dst, Fp);
}

// Column sums b_l = sum_k W[k][l] of the dictionary (Mp x Fp, padding zero):
// the reconstruction of the initial state, whose weights are all 1, is b_l in
// every frame.  32 columns per block (coalesced rows), eight groups of rows
// per column, each summed as an unevaluated float pair (hi + lo, error-free
// two-sums: FP64 arithmetic is a small fraction of FP32's rate on this GPU),
// the groups combined in shared memory and rounded once.
__device__ __forceinline__ void two_sum_acc_e(float& hi, float& lo, float x) {
  const float s = hi + x;
  const float bp = s - hi;
  lo += (hi - (s - bp)) + (x - bp);
  hi = s;
}
__global__ void __launch_bounds__(256) k_col_sums(const float* W, int M, int Fp, float* b) {
  __shared__ float part[2][8][32];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int l = blockIdx.x * 32 + tx;
  float hi = 0.f, lo = 0.f;
  if (l < Fp)
    for (int k = ty; k < M; k += 8) two_sum_acc_e(hi, lo, W[(size_t)k * Fp + l]);
  part[0][ty][tx] = hi;
  part[1][ty][tx] = lo;
  __syncthreads();
  if (ty == 0 && l < Fp) {
    float h = part[0][0][tx], o = part[1][0][tx];
    for (int g = 1; g < 8; ++g) {
      two_sum_acc_e(h, o, part[0][g][tx]);
      o += part[1][g][tx];
    }
    b[l] = (float)((double)h + (double)o);
  }
}
void launch_col_sums(const float* W, int M, int Fp, float* b, cudaStream_t st) {
  k_col_sums<<<(Fp + 31) / 32, 256, 0, st>>>(W, M, Fp, b);
}

// The initial state's ratio Q = V / Vhat with Vhat_tl = b_l (Eq. 7 at w = 1),
// for frames [0, T): float (out) or split into tf32 hi / lo; a frequency with
// energy but b_l <= 0 (or not finite) sets ERR_VHAT_ZERO and gives 0, as the
// contraction's ratio epilogue does.
__global__ void k_init_ratio(const float* V, const float* b, int T, int Fp, float* out,
                             float* hi, float* lo, unsigned* err) {
  const size_t n = (size_t)T * Fp;
  unsigned bad = 0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const float v = V[i], x = b[i % Fp];
    float q = 0.f;
    if (v > 0.f) {
      if (x > 0.f && isfinite(x))
        q = v / x;
      else
        bad |= ERR_VHAT_ZERO;
    }
    if (out) out[i] = q;
    if (hi) {
      const float h = tf32_hi(q);
      hi[i] = h;
      lo[i] = tf32_hi(q - h);
    }
  }
  bad = __reduce_or_sync(FULL, bad);
  if (bad && (threadIdx.x & 31) == 0) atomicOr(err, bad);
}
void launch_init_ratio(const float* V, const float* b, int T, int Fp, float* out, float* hi,
                       float* lo, unsigned* err, cudaStream_t st) {
  const size_t n = (size_t)T * Fp;
  const int blocks = (int)std::min<size_t>(4096, (n + 255) / 256);
  if (blocks > 0) k_init_ratio<<<blocks, 256, 0, st>>>(V, b, T, Fp, out, hi, lo, err);
}

__global__ void k_split_tf32(const float* in, float* hi, float* lo, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const float x = in[i];
    const float h = tf32_hi(x);
    hi[i] = h;
    lo[i] = tf32_hi(x - h);
  }
}
void launch_split_tf32(const float* in, float* hi, float* lo, size_t n, cudaStream_t st) {
  k_split_tf32<<<1024, 256, 0, st>>>(in, hi, lo, n);
}
__global__ void k_to_bf16(const float* in, __nv_bfloat16* out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    out[i] = __float2bfloat16_rn(in[i]);
}
void launch_to_bf16(const float* in, void* out, size_t n, cudaStream_t st) {
  k_to_bf16<<<1024, 256, 0, st>>>(in, reinterpret_cast<__nv_bfloat16*>(out), n);
}

// -------------------------------------------------------------------- bound
// Per frame t (one warp): FP64 accumulation of
//   sum_l V log Vhat (from the contraction's partials) - v_t psi(a0)
//   + konst - lnGamma(a0) + sum_k g(alpha_tk) + psi(a0) (a0 - M) - S gamma K psi(a0)
// with a0 = sum_k alpha_tk and g(a) = lnGamma(a) - (a - 1) psi(a).  The last
// term converts the forward-backward log normalisers, computed on phi-hat
// without its per-frame constant -gamma K psi(a0), back to Eq. 8's phi-hat.
__global__ void k_bound_frames(BoundArgs a) {
  const int lane = threadIdx.x & 31;
  const int t = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (t >= a.T) return;
  const float* row = a.alpha + (size_t)t * a.Mp;
  double s0 = 0.0, sg = 0.0;
  for (int k = lane; k < a.M; k += 32) {
    const float x = row[k];
    s0 += (double)x;
    sg += bound_g_elem(x);
  }
  s0 = warp_sum_d(s0);
  sg = warp_sum_d(sg);
  if (lane == 0) {
    double vl = 0.0;
    for (int j = 0; j < a.nbpart_used; ++j) vl += a.bpart[(size_t)t * a.nbpart + j];
    const double psi0 = digamma_d(s0);
    const double term = vl - a.v[t] * psi0 + a.konst - lgamma(s0) + sg + psi0 * (s0 - (double)a.M) -
                        (double)a.S * (double)a.gamma * (double)a.K * psi0;
    a.frame_terms[t] = term;
  }
}

// The same per-frame term from the weights kernel's per-frame sums
// (one thread per frame): no pass over the elements.
__global__ void k_bound_frames_fused(BoundArgs a) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a.T) return;
  double s0 = 0.0, sg = 0.0;
  for (int h = 0; h < a.funits; ++h) {
    s0 += a.fterm[2 * ((size_t)t * a.funits + h)];
    sg += a.fterm[2 * ((size_t)t * a.funits + h) + 1];
  }
  double vl = 0.0;
  for (int j = 0; j < a.nbpart_used; ++j) vl += a.bpart[(size_t)t * a.nbpart + j];
  const double psi0 = digamma_d(s0);
  a.frame_terms[t] = vl - a.v[t] * psi0 + a.konst - lgamma(s0) + sg + psi0 * (s0 - (double)a.M) -
                     (double)a.S * (double)a.gamma * (double)a.K * psi0;
}

// One block per job: the sum of its frames' terms and its chains' log
// normalisers.  A one-warp launch then sums the jobs into out[njobs].
__global__ void k_bound_final(BoundArgs a) {
  __shared__ double red[32];
  const int j = blockIdx.x;
  const int t0 = a.job_t0 ? a.job_t0[j] : 0;
  const int t1 = a.job_t0 ? a.job_t0[j + 1] : a.T;
  double s = 0.0;
  for (int t = t0 + threadIdx.x; t < t1; t += blockDim.x) s += a.frame_terms[t];
  s = warp_sum_d(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double r = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    r = warp_sum_d(r);
    if (threadIdx.x == 0) {
      for (int i = 0; i < a.S; ++i) r += a.logZ[(size_t)i * a.njobs + j];
      a.out[j] = r;
    }
  }
}

__global__ void k_bound_total(BoundArgs a) {
  double r = 0.0;
  for (int j = threadIdx.x; j < a.njobs; j += 32) r += a.out[j];
  r = warp_sum_d(r);
  if (threadIdx.x == 0) a.out[a.njobs] = r;
}

void launch_bound(const BoundArgs& a, cudaStream_t st, int* launches) {
  if (a.fterm)
    k_bound_frames_fused<<<(a.T + 127) / 128, 128, 0, st>>>(a);
  else
    k_bound_frames<<<(a.T + 7) / 8, 256, 0, st>>>(a);
  k_bound_final<<<a.njobs, 1024, 0, st>>>(a);
  k_bound_total<<<1, 32, 0, st>>>(a);
  if (launches) *launches += 3;
}

// -------------------------------------------------------------- separation
__global__ void k_sep_weights(const float* alpha, const double* v, int T, int M, int Mp, int mode,
                              float* wts) {
  const int lane = threadIdx.x & 31;
  const int t = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (t >= T) return;
  const float* row = alpha + (size_t)t * Mp;
  float* out = wts + (size_t)t * Mp;
  if (mode == 0) {
    double s = 0.0;
    for (int k = lane; k < M; k += 32) s += (double)row[k];
    s = warp_sum_d(s);
    const double scale = v[t] / s;
    for (int k = lane; k < Mp; k += 32) out[k] = k < M ? (float)(scale * (double)row[k]) : 0.f;
  } else {
    for (int k = lane; k < Mp; k += 32) {
      float p, w = 0.f;
      if (k < M) digamma_exp(row[k], p, w);
      out[k] = w;
    }
  }
}
void launch_sep_weights(const float* alpha, const double* v, int T, int M, int Mp, int mode,
                        float* wts, cudaStream_t st) {
  k_sep_weights<<<(T + 7) / 8, 256, 0, st>>>(alpha, v, T, M, Mp, mode, wts);
}

__global__ void k_sep_mask(const float* V, int Fp, float* out, int S, int T, int F) {
  const size_t n = (size_t)T * F;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const size_t t = i / F, l = i % F;
    const float vv = V[t * Fp + l];
    float den = 0.f;
    for (int s = 0; s < S; ++s) den += out[(size_t)s * n + i];
    for (int s = 0; s < S; ++s) {
      const float x = out[(size_t)s * n + i];
      out[(size_t)s * n + i] = den > 0.f ? vv * (x / den) : vv / (float)S;
    }
  }
}
void launch_sep_mask(const float* V, int Fp, float* out, int S, int T, int F, cudaStream_t st) {
  k_sep_mask<<<1024, 256, 0, st>>>(V, Fp, out, S, T, F);
}

// ----------------------------------------------------------------- digamma
// A stateless forward-backward has no context to carry its error word back
// to the caller: a set word turns its log normalisers into NaN.
__global__ void k_flag_errors(const unsigned* err, double* logZ, int n) {
  if (*err == 0u) return;
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    logZ[i] = __longlong_as_double(0x7ff8000000000000ll);
}

void launch_flag_errors(const unsigned* err, double* logZ, int n, cudaStream_t st) {
  k_flag_errors<<<1, 32, 0, st>>>(err, logZ, n);
}

__global__ void k_digamma(const float* x, float* psi, float* w, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    float p, e;
    digamma_exp(x[i], p, e);
    if (psi) psi[i] = p;
    if (w) w[i] = e;
  }
}
void launch_digamma(const float* x, float* psi, float* w, size_t n, cudaStream_t st) {
  k_digamma<<<512, 256, 0, st>>>(x, psi, w, n);
}

// ------------------------------------------------------ frame compaction
// One warp per destination frame: find its segment (binary search over the
// segment table), then copy the frame's V, counts, d-hat and v rows.
__global__ void k_move_frames(FrameMove m) {
  const int lane = threadIdx.x & 31;
  const int f = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (f >= m.frames) return;
  const int t = m.base + f;
  int lo = 0, hi = m.nseg - 1;
  while (lo < hi) {   // last segment with dst first frame <= t
    const int mid = (lo + hi + 1) >> 1;
    if (m.seg[3 * mid] <= t) lo = mid; else hi = mid - 1;
  }
  const int src = m.seg[3 * lo + 1] + (t - m.seg[3 * lo]);   // offset in the copy
  const float4* vs = reinterpret_cast<const float4*>(m.Vs + (size_t)src * m.Fp);
  float4* vd = reinterpret_cast<float4*>(m.V + (size_t)t * m.Fp);
  for (int i = lane; i < m.Fp / 4; i += 32) vd[i] = vs[i];
  const float4* cs = reinterpret_cast<const float4*>(m.cs + (size_t)src * m.Mp);
  float4* cd = reinterpret_cast<float4*>(m.c + (size_t)t * m.Mp);
  for (int i = lane; i < m.Mp / 4; i += 32) cd[i] = cs[i];
  for (int i = lane; i < m.SN; i += 32) {
    const int s = i / m.N, n = i - s * m.N;
    m.dhat[((size_t)s * m.Tc + t) * m.N + n] = m.ds[((size_t)s * m.Tc + src) * m.N + n];
  }
  if (lane == 0) m.v[t] = m.vs[src];
}
void launch_move_frames(const FrameMove& m, cudaStream_t st) {
  if (m.frames <= 0 || m.nseg <= 0) return;
  k_move_frames<<<(m.frames + 7) / 8, 256, 0, st>>>(m);
}

// --------------------------------------------------------- prior marginals
// dhat[s][t0] = pi_s, dhat[s][t] = dhat[s][t-1] A_s over each job's frames
// [t0, t1) (one block per (source, job)).  With a null job table there is one
// job, frames [t_begin, t_end).  T is the frame stride of dhat.
__global__ void k_prior_marginals(const float* A, const float* pi, int S, int N, int T,
                                  const int* job_t0, int njobs, int t_begin, int t_end,
                                  float* dhat) {
  extern __shared__ float sm[];
  float* As = sm;          // N*N
  float* d = sm + N * N;   // N
  const int s = blockIdx.x / njobs, jb = blockIdx.x - s * njobs;
  const int t0 = job_t0 ? job_t0[jb] : t_begin;
  const int t1 = job_t0 ? job_t0[jb + 1] : t_end;
  for (int i = threadIdx.x; i < N * N; i += blockDim.x) As[i] = A[(size_t)s * N * N + i];
  for (int i = threadIdx.x; i < N; i += blockDim.x) d[i] = pi[(size_t)s * N + i];
  __syncthreads();
  for (int t = t0; t < t1; ++t) {
    float nj = 0.f;
    const int j = threadIdx.x;
    if (j < N) {
      dhat[((size_t)s * T + t) * N + j] = d[j];
      for (int i = 0; i < N; ++i) nj += d[i] * As[i * N + j];
    }
    __syncthreads();
    if (j < N) d[j] = nj;
    __syncthreads();
  }
}
void launch_prior_marginals(const float* A, const float* pi, int S, int N, int T,
                            const int* job_t0, int njobs, int t_begin, int t_end, float* dhat,
                            cudaStream_t st) {
  if (!job_t0) njobs = 1;
  const int threads = ((N + 31) / 32) * 32;
  k_prior_marginals<<<S * njobs, threads, (N * N + N) * sizeof(float), st>>>(
      A, pi, S, N, T, job_t0, njobs, t_begin, t_end, dhat);
}

}  // namespace nfhmm
