// Exact inference in the original N-FHMM: the comparison system of Section 5
// (the model of Section 2.2's opening sentences).  Each frame t and joint
// state c = (d^(1), ..., d^(S)) has its own mixture weights theta_t(c) over
// the S*K elements c selects; one EM iteration is
//   E-step: l_t(c) = sum_f V_tf log Vhat_tc(f), Vhat_tc = sum_k theta_t(c)_k beta_ck
//           (batched tcgen05 contraction, one item per joint state), then
//           forward-backward over the N^S joint states (transitions prod_s A^(s),
//           applied one source at a time) -> posteriors gamma_t(c), log P(V | theta);
//   M-step: theta_t(c)_k <- theta_t(c)_k sum_f beta_ck(f) V_tf / Vhat_tc(f), normalised
//           (the second batched contraction and a row normalisation).
// The cost of an iteration grows as N^S (the paper's argument for variational
// inference); this implementation is the yardstick for that comparison.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>

#include <string>
#include <vector>

#include "../../include/nfhmm.h"
#include "nfhmm_device.cuh"
#include "nfhmm_kernels.h"
#include "nfhmm_tc.h"

using namespace nfhmm;

namespace {

int fail(int code, const std::string& m) {
  set_last_error(m);
  return code;
}

#define XCK(call)                                                                      \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return fail(e_ == cudaErrorMemoryAllocation ? NFHMM_ENOMEM : NFHMM_ECUDA,        \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                 \
  } while (0)

size_t rup(size_t x, size_t m) { return (x + m - 1) / m * m; }

struct Dev {
  int S, N, K, F, T, Tp, Fp, SK, SKp, NC, M, Mp;
};

// ------------------------------------------------------------------ kernels
// B1[c][f][k] = beta_{elem(c,k)}(f) and B2[c][k][f] = the same (zero outside
// k < S*K, f < F), as split-TF32 pairs or BF16.
template <bool BF>
__global__ void k_exact_build_b(Dev d, const float* WM /* Mp x Fp */, void* b1h, void* b1l,
                                void* b2h, void* b2l) {
  const size_t n = (size_t)d.NC * d.Fp * d.SKp;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n;
       idx += (size_t)gridDim.x * blockDim.x) {
    // idx enumerates B2 = [c][k][f]
    const int f = (int)(idx % d.Fp);
    const size_t ck = idx / d.Fp;
    const int k = (int)(ck % d.SKp), c = (int)(ck / d.SKp);
    float v = 0.f;
    if (k < d.SK && f < d.F) {
      const int s = k / d.K, j = k - s * d.K;
      int rest = c, stride = 1;
      for (int q = s + 1; q < d.S; ++q) stride *= d.N;
      const int ds = (rest / stride) % d.N;
      const int elem = (s * d.N + ds) * d.K + j;
      v = WM[(size_t)elem * d.Fp + f];
    }
    const size_t i1 = ((size_t)c * d.Fp + f) * d.SKp + k;   // B1[c][f][k]
    if (BF) {
      reinterpret_cast<__nv_bfloat16*>(b1h)[i1] = __float2bfloat16_rn(v);
      reinterpret_cast<__nv_bfloat16*>(b2h)[idx] = __float2bfloat16_rn(v);
    } else {
      const float h = tf32_hi(v), l = tf32_hi(v - h);
      reinterpret_cast<float*>(b1h)[i1] = h;
      reinterpret_cast<float*>(b1l)[i1] = l;
      reinterpret_cast<float*>(b2h)[idx] = h;
      reinterpret_cast<float*>(b2l)[idx] = l;
    }
  }
}

// theta rows (one warp per row c*Tp + t): init = uniform over the S*K
// elements; update = out / sum(out) (kept where the sum vanished).  Writes the
// float copy and the contraction operand.
template <bool BF, bool INIT>
__global__ void k_exact_theta(Dev d, float* th32, const float* out, void* thh, void* thl,
                              unsigned* err) {
  const int lane = threadIdx.x & 31;
  const size_t row = blockIdx.x * (size_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
  if (row >= (size_t)d.NC * d.Tp) return;
  const int t = (int)(row % d.Tp);
  const bool live = t < d.T;
  float v[2];
  float sum = 0.f;
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int k = lane + 32 * u;
    float x = 0.f;
    if (live && k < d.SK) x = INIT ? 1.f / (float)d.SK : out[row * d.SKp + k];
    v[u] = x;
    sum += x;
  }
  if (!INIT) {
    sum = warp_sum(sum);
    const bool ok = sum > 0.f && isfinite(sum);
    if (!isfinite(sum) && lane == 0) atomicOr(err, ERR_NONFINITE);
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int k = lane + 32 * u;
      if (k < d.SKp) v[u] = ok ? v[u] / sum : (live && k < d.SK ? th32[row * d.SKp + k] : 0.f);
    }
  }
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int k = lane + 32 * u;
    if (k >= d.SKp) continue;
    const size_t i = row * d.SKp + k;
    th32[i] = v[u];
    if (BF) {
      reinterpret_cast<__nv_bfloat16*>(thh)[i] = __float2bfloat16_rn(v[u]);
    } else {
      const float h = tf32_hi(v[u]);
      reinterpret_cast<float*>(thh)[i] = h;
      reinterpret_cast<float*>(thl)[i] = tf32_hi(v[u] - h);
    }
  }
}

// Per frame (one block): l_t(c) from the contraction's partials, its maximum
// m_t over joint states and the emissions e_t(c) = exp(l_t(c) - m_t).
__global__ void k_exact_emissions(Dev d, const double* bpart, int nbpart, float* e, double* m) {
  extern __shared__ double red[];
  const int t = blockIdx.x;
  double mx = -INFINITY;
  for (int c = threadIdx.x; c < d.NC; c += blockDim.x) {
    const double* bp = bpart + ((size_t)c * d.Tp + t) * nbpart;
    double l = 0.0;
    for (int j = 0; j < nbpart; ++j) l += bp[j];
    red[32 + c] = l;
    mx = fmax(mx, l);
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = -INFINITY;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = fmax(r, red[w]);
    red[0] = r;
    m[t] = r;
  }
  __syncthreads();
  const double mt = red[0];
  for (int c = threadIdx.x; c < d.NC; c += blockDim.x)
    e[(size_t)t * d.NC + c] = (float)exp(red[32 + c] - mt);
}

// Block-wide sum (every thread gets it); red: 33 floats of shared memory.
__device__ float block_sum(float v, float* red) {
  v = warp_sum(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    float r = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
    r = warp_sum(r);
    if (threadIdx.x == 0) red[32] = r;
  }
  __syncthreads();
  return red[32];
}

// Forward (block 0) and backward (block 1) recursions over the joint chain,
// serial in t; the joint transition is applied one source at a time (mode
// products), the last source's state varying fastest in c.  Each thread owns
// up to XC joint states.  A step is S mode products with one barrier each:
// the vector entering a step is rescaled by the sum of the previous one
// (its per-warp partial sums are published by the previous step's last
// barrier), the next frame's emissions are loaded while the step runs, and
// the stored vectors carry a per-frame scale that the posteriors' per-frame
// normalisation removes.  The forward sums give log P(V | theta).
constexpr int XC = 4;   // joint states per thread (N^S <= 4096, 1024 threads)
__global__ void __launch_bounds__(1024) k_exact_fb(Dev d, const float* A, const float* pi,
                                                   const float* e, float* fa, float* fb,
                                                   double* loglik, const double* m, float* scl,
                                                   unsigned* err) {
  extern __shared__ float sm[];
  const int NC = d.NC, N = d.N, S = d.S;
  const int nw = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* buf0 = sm;                       // NC
  float* buf1 = buf0 + NC;                // NC
  float* As = buf1 + NC;                  // S x N x N
  float* part = As + S * N * N;           // 2 x 32 per-warp partial sums
  const bool fwd = blockIdx.x == 0;
  for (int i = threadIdx.x; i < S * N * N; i += blockDim.x) As[i] = A[i];
  int cs[XC];
#pragma unroll
  for (int u = 0; u < XC; ++u) {
    const int c = threadIdx.x + u * blockDim.x;
    cs[u] = c < NC ? c : -1;
  }
  // S mode products from `in`; the last one's outputs go to `fin` through
  // `last` (value, state, slot); returns nothing, buffers alternate
  auto modes = [&](float* in, float* other, auto&& last) {
    int stride = 1;
    float* src = in;
    float* dst = other;
    for (int s = S - 1; s >= 0; --s) {
      const float* Am = As + s * N * N;
      const bool final_mode = s == 0;
#pragma unroll
      for (int u = 0; u < XC; ++u) {
        const int c = cs[u];
        if (c < 0) continue;
        const int ds = (c / stride) % N;
        const int base = c - ds * stride;
        float acc = 0.f;
        if (fwd) {
          for (int i = 0; i < N; ++i) acc = fmaf(src[base + i * stride], Am[i * N + ds], acc);
        } else {
          for (int j = 0; j < N; ++j) acc = fmaf(Am[ds * N + j], src[base + j * stride], acc);
        }
        if (final_mode) last(acc, c, u, dst);
        else dst[c] = acc;
      }
      if (!final_mode) {
        __syncthreads();
        float* tmp = src;
        src = dst;
        dst = tmp;
      }
      stride *= N;
    }
  };
  double lsum = 0.0;   // forward: log P(V | theta), summed after the loop
  float en[XC];
  float local = 0.f;
  if (fwd) {
    // a_0 = pi (.) e_0, unnormalised
#pragma unroll
    for (int u = 0; u < XC; ++u) {
      const int c = cs[u];
      if (c < 0) continue;
      float p = 1.f;
      int rest = c;
      for (int s = S - 1; s >= 0; --s) {
        p *= pi[s * N + rest % N];
        rest /= N;
      }
      const float v = p * e[c];
      buf0[c] = v;
      fa[c] = v;
      local += v;
    }
  } else {
    // b_{T-1} = 1; the vector entering the first step is e_{T-1} (.) b_{T-1}
#pragma unroll
    for (int u = 0; u < XC; ++u) {
      const int c = cs[u];
      if (c < 0) continue;
      fb[(size_t)(d.T - 1) * NC + c] = 1.f;
      buf0[c] = e[(size_t)(d.T - 1) * NC + c];
      local += 1.f;
    }
  }
  local = warp_sum(local);
  if (lane == 0) part[warp] = local;
#pragma unroll
  for (int u = 0; u < XC; ++u) {   // emissions of the first step
    const int c = cs[u];
    const int tn = fwd ? 1 : d.T - 2;
    en[u] = (c >= 0 && tn >= 0 && tn < d.T) ? e[(size_t)tn * NC + c] : 0.f;
  }
  __syncthreads();
  float* x = buf0;
  float* y = buf1;
  for (int q = 1; q < d.T; ++q) {
    const int t = fwd ? q : d.T - 1 - q;           // frame this step produces
    const float* pp = part + ((q - 1) & 1) * 32;   // the previous vector's partials
    float sprev = 0.f;
    for (int w = 0; w < nw; ++w) sprev += pp[w];
    if (!(sprev > 0.f) || !isfinite(sprev)) {
      if (threadIdx.x == 0) atomicOr(err, ERR_FB_ZERO);
      sprev = 1.f;
    }
    if (fwd && threadIdx.x == 0) scl[t - 1] = sprev;   // logs taken after the loop
    const float inv = 1.f / sprev;
    float eh[XC];
#pragma unroll
    for (int u = 0; u < XC; ++u) {
      eh[u] = en[u];
      // the next frame's emissions, loaded while this step runs
      const int c = cs[u];
      const int tn = fwd ? t + 1 : t - 1;
      en[u] = (c >= 0 && tn >= 0 && tn < d.T) ? e[(size_t)tn * NC + c] : 0.f;
    }
    float loc = 0.f;
    float* res = nullptr;
    modes(x, y, [&](float acc, int c, int u, float* dst) {
      float v;
      if (fwd) {
        v = acc * inv * eh[u];
        fa[(size_t)t * NC + c] = v;
        dst[c] = v;
        loc += v;
      } else {
        v = acc * inv;                            // b_t (scaled)
        fb[(size_t)t * NC + c] = v;
        dst[c] = v * eh[u];                       // e_t (.) b_t enters the next step
        loc += v;
      }
      res = dst;
    });
    loc = warp_sum(loc);
    if (lane == 0) part[(q & 1) * 32 + warp] = loc;
    __syncthreads();
    // the result sits in whichever buffer the last mode wrote
    if (S % 2 == 1) {
      float* tmp = x;
      x = y;
      y = tmp;
    }
    (void)res;
  }
  if (fwd) {
    if (threadIdx.x == 0) {
      const float* pp = part + (((d.T - 1) & 1) * 32);
      float sl = 0.f;
      for (int w = 0; w < nw; ++w) sl += pp[w];
      scl[d.T - 1] = sl;
    }
    __syncthreads();
    // log P(V | theta) = sum_t log(normaliser_t) + m_t, off the serial path
    for (int t = threadIdx.x; t < d.T; t += blockDim.x) lsum += log((double)scl[t]) + m[t];
    lsum = warp_sum_d(lsum);
    double* dred = reinterpret_cast<double*>(buf0);   // the vectors are no longer needed
    __syncthreads();
    if (lane == 0) dred[warp] = lsum;
    __syncthreads();
    if (threadIdx.x == 0) {
      double r = 0.0;
      for (int w = 0; w < nw; ++w) r += dred[w];
      *loglik = r;
    }
  }
}

// gamma_t(c) = fa_t(c) fb_t(c) / sum_c (one block per frame).
__global__ void k_exact_combine(Dev d, const float* fa, const float* fb, float* gamma,
                                unsigned* err) {
  __shared__ float red[33];
  const int t = blockIdx.x;
  float sum = 0.f;
  for (int c = threadIdx.x; c < d.NC; c += blockDim.x)
    sum += fa[(size_t)t * d.NC + c] * fb[(size_t)t * d.NC + c];
  sum = block_sum(sum, red);
  if (!(sum > 0.f) || !isfinite(sum)) {
    if (threadIdx.x == 0) atomicOr(err, ERR_FB_ZERO);
    sum = 1.f;
  }
  for (int c = threadIdx.x; c < d.NC; c += blockDim.x)
    gamma[(size_t)t * d.NC + c] = fa[(size_t)t * d.NC + c] * fb[(size_t)t * d.NC + c] / sum;
}

}  // namespace

struct nfhmm_exact {
  Dev d{};
  int precision = 0;
  cudaStream_t user = nullptr;
  float* V = nullptr;     // T x Fp
  float* WM = nullptr;    // Mp x Fp
  float* A = nullptr;     // S x N x N
  float* pi = nullptr;    // S x N
  float* th32 = nullptr;  // NC*Tp x SKp
  float* out = nullptr;   // NC*Tp x SKp
  double* bpart = nullptr;
  float* e = nullptr;     // T x NC
  double* m = nullptr;    // T
  float* fa = nullptr;    // T x NC
  float* fb = nullptr;    // T x NC
  float* gamma = nullptr; // T x NC
  double* loglik = nullptr;
  float* scl = nullptr;   // T forward normalisers
  unsigned* err = nullptr;
  double* h_ll = nullptr;
  unsigned* h_err = nullptr;
  ExactTc tc{};
  int iterations = 0;
  bool have_posteriors = false;
};

namespace {

void free_exact(nfhmm_exact* x) {
  if (!x) return;
  if (x->user) cudaStreamSynchronize(x->user);
  void* bufs[] = {x->V, x->WM, x->A, x->pi, x->th32, x->out, x->bpart, x->e, x->m,
                  x->fa, x->fb, x->gamma, x->loglik, x->err, x->scl};
  for (void* p : bufs)
    if (p) cudaFree(p);
  tc_exact_free(x->tc);
  if (x->h_ll) cudaFreeHost(x->h_ll);
  if (x->h_err) cudaFreeHost(x->h_err);
  delete x;
}

int exact_sync(nfhmm_exact* x) {
  XCK(cudaMemcpyAsync(x->h_err, x->err, 4, cudaMemcpyDeviceToHost, x->user));
  XCK(cudaStreamSynchronize(x->user));
  if (*x->h_err) {
    const unsigned e = *x->h_err;
    cudaMemsetAsync(x->err, 0, 4, x->user);
    cudaStreamSynchronize(x->user);
    if (e & ERR_TIMEOUT) return fail(NFHMM_ETIMEOUT, "a bounded device wait gave up");
    if (e & ERR_BAD_INPUT) return fail(NFHMM_EINVAL, "input validation failed");
    return fail(NFHMM_ENUMERIC, "reconstruction vanished where V > 0, or a normaliser vanished");
  }
  return NFHMM_OK;
}

}  // namespace

extern "C" {

int nfhmm_exact_create(nfhmm_exact** out, const nfhmm_dims* dp, const float* V, const float* W,
                       const float* A, const float* pi, int inputs_on_device, void* cuda_stream) {
  if (out) *out = nullptr;
  if (!out || !dp || !V || !W || !A || !pi) return fail(NFHMM_EINVAL, "NULL argument");
  const nfhmm_dims dd = *dp;
  if (dd.S < 1 || dd.N < 1 || dd.K < 1 || dd.F < 1 || dd.T < 1)
    return fail(NFHMM_EINVAL, "S, N, K, F, T must all be >= 1");
  if (dd.precision != NFHMM_FP32 && dd.precision != NFHMM_BF16)
    return fail(NFHMM_EINVAL, "precision must be NFHMM_FP32 or NFHMM_BF16");
  if (!tc_available()) return fail(NFHMM_EINVAL, "exact inference needs an sm_103 device");
  long long NC = 1;
  for (int s = 0; s < dd.S; ++s) NC *= dd.N;
  if (dd.S * dd.K > 64) return fail(NFHMM_EINVAL, "S*K must be <= 64");
  if (NC > 4096) return fail(NFHMM_EINVAL, "N^S must be <= 4096");
  nfhmm_exact* x = new nfhmm_exact();
  Dev& d = x->d;
  d.S = dd.S;
  d.N = dd.N;
  d.K = dd.K;
  d.F = dd.F;
  d.T = dd.T;
  d.Tp = (int)rup(dd.T, 128);
  d.Fp = (int)rup(dd.F, 32);
  d.SK = dd.S * dd.K;
  d.SKp = (int)rup(d.SK, 32);
  d.NC = (int)NC;
  d.M = dd.S * dd.N * dd.K;
  d.Mp = (int)rup(d.M, 32);
  x->precision = dd.precision;
  x->user = reinterpret_cast<cudaStream_t>(cuda_stream);
  const size_t rows = (size_t)d.NC * d.Tp;
  if (rows * d.Fp > (size_t)1 << 34 || rows / 128 > 65535) {
    free_exact(x);
    return fail(NFHMM_EINVAL, "N^S * T * F too large for exact inference on one GPU");
  }
  auto bail = [&](int rc) {
    free_exact(x);
    return rc;
  };
#define XMALLOC(ptr, bytes)                                                               \
  do {                                                                                  \
    cudaError_t e_ = cudaMalloc((void**)&(ptr), (bytes));                               \
    if (e_ != cudaSuccess)                                                              \
      return bail(fail(e_ == cudaErrorMemoryAllocation ? NFHMM_ENOMEM : NFHMM_ECUDA,      \
                       std::string("cudaMalloc: ") + cudaGetErrorString(e_)));          \
  } while (0)
  XMALLOC(x->V, (size_t)d.T * d.Fp * 4);
  XMALLOC(x->WM, (size_t)d.Mp * d.Fp * 4);
  XMALLOC(x->A, (size_t)d.S * d.N * d.N * 4);
  XMALLOC(x->pi, (size_t)d.S * d.N * 4);
  XMALLOC(x->th32, rows * d.SKp * 4);
  XMALLOC(x->out, rows * d.SKp * 4);
  x->tc.precision = dd.precision;
  x->tc.NC = d.NC;
  x->tc.T = d.T;
  x->tc.Tp = d.Tp;
  x->tc.SKp = d.SKp;
  x->tc.F = d.F;
  x->tc.Fp = d.Fp;
  if (tc_exact_plan(x->tc) != 0) return bail(fail(NFHMM_ECUDA, "tensor-core plan: " + tc_last_error()));
  XMALLOC(x->bpart, rows * x->tc.nbpart * 8);
  XMALLOC(x->e, (size_t)d.T * d.NC * 4);
  XMALLOC(x->m, (size_t)d.T * 8);
  XMALLOC(x->fa, (size_t)d.T * d.NC * 4);
  XMALLOC(x->fb, (size_t)d.T * d.NC * 4);
  XMALLOC(x->gamma, (size_t)d.T * d.NC * 4);
  XMALLOC(x->loglik, 8);
  XMALLOC(x->scl, (size_t)d.T * 4);
  XMALLOC(x->err, 4);
#undef XMALLOC
  if (cudaMallocHost(&x->h_ll, 8) != cudaSuccess || cudaMallocHost(&x->h_err, 4) != cudaSuccess)
    return bail(fail(NFHMM_ENOMEM, "pinned host staging"));
  x->tc.V = x->V;
  x->tc.th32 = x->th32;
  x->tc.out = x->out;
  x->tc.bpart = x->bpart;
  x->tc.err = x->err;
  cudaStream_t st = x->user;
  const cudaMemcpyKind kind = inputs_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDefault;
  int rc = NFHMM_OK;
  auto step = [&](cudaError_t e) {
    if (e != cudaSuccess && !rc) rc = fail(NFHMM_ECUDA, cudaGetErrorString(e));
  };
  step(cudaMemsetAsync(x->err, 0, 4, st));
  step(cudaMemsetAsync(x->V, 0, (size_t)d.T * d.Fp * 4, st));
  step(cudaMemsetAsync(x->WM, 0, (size_t)d.Mp * d.Fp * 4, st));
  step(cudaMemcpy2DAsync(x->V, (size_t)d.Fp * 4, V, (size_t)d.F * 4, (size_t)d.F * 4, d.T, kind, st));
  step(cudaMemcpy2DAsync(x->WM, (size_t)d.Fp * 4, W, (size_t)d.F * 4, (size_t)d.F * 4, d.M, kind, st));
  step(cudaMemcpyAsync(x->A, A, (size_t)d.S * d.N * d.N * 4, kind, st));
  step(cudaMemcpyAsync(x->pi, pi, (size_t)d.S * d.N * 4, kind, st));
  if (rc) return bail(rc);
  launch_validate(x->V, d.T, d.F, d.Fp, x->WM, d.M, x->A, x->pi, d.S, d.N, x->err, st);
  const bool bf = dd.precision == NFHMM_BF16;
  if (bf) {
    k_exact_build_b<true><<<2048, 256, 0, st>>>(d, x->WM, x->tc.b1_hi, x->tc.b1_lo, x->tc.b2_hi,
                                                x->tc.b2_lo);
    k_exact_theta<true, true><<<(unsigned)((rows + 7) / 8), 256, 0, st>>>(
        d, x->th32, x->out, x->tc.th_hi, x->tc.th_lo, x->err);
  } else {
    k_exact_build_b<false><<<2048, 256, 0, st>>>(d, x->WM, x->tc.b1_hi, x->tc.b1_lo, x->tc.b2_hi,
                                                 x->tc.b2_lo);
    k_exact_theta<false, true><<<(unsigned)((rows + 7) / 8), 256, 0, st>>>(
        d, x->th32, x->out, x->tc.th_hi, x->tc.th_lo, x->err);
  }
  step(cudaGetLastError());
  if (rc) return bail(rc);
  rc = exact_sync(x);
  if (rc) return bail(rc);
  *out = x;
  return NFHMM_OK;
}

int nfhmm_exact_iterate(nfhmm_exact* x, int n_iter, double* loglik_out) {
  if (!x) return fail(NFHMM_EINVAL, "NULL context");
  if (n_iter < 1) return fail(NFHMM_EINVAL, "n_iter must be >= 1");
  const Dev& d = x->d;
  cudaStream_t st = x->user;
  const size_t rows = (size_t)d.NC * d.Tp;
  const bool bf = x->precision == NFHMM_BF16;
  const size_t smem_fb = (size_t)(2 * d.NC + d.S * d.N * d.N + 64) * sizeof(float);
  const size_t smem_em = (size_t)(32 + d.NC) * sizeof(double);
  static bool attr_done = false;
  if (!attr_done) {
    XCK(cudaFuncSetAttribute(k_exact_fb, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    XCK(cudaFuncSetAttribute(k_exact_emissions, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             64 * 1024));
    attr_done = true;
  }
  for (int it = 0; it < n_iter; ++it) {
    // E-step
    if (tc_exact_gemm1(x->tc, st) < 0) return fail(NFHMM_ECUDA, "contraction: " + tc_last_error());
    k_exact_emissions<<<d.T, 256, smem_em, st>>>(d, x->bpart, x->tc.nbpart, x->e, x->m);
    const int fb_threads = d.NC >= 1024 ? 1024 : (int)rup(d.NC, 32);
    k_exact_fb<<<2, fb_threads, smem_fb, st>>>(d, x->A, x->pi, x->e, x->fa, x->fb, x->loglik,
                                               x->m, x->scl, x->err);
    k_exact_combine<<<d.T, 256, 0, st>>>(d, x->fa, x->fb, x->gamma, x->err);
    // M-step
    if (tc_exact_gemm2(x->tc, st) < 0) return fail(NFHMM_ECUDA, "contraction: " + tc_last_error());
    if (bf)
      k_exact_theta<true, false><<<(unsigned)((rows + 7) / 8), 256, 0, st>>>(
          d, x->th32, x->out, x->tc.th_hi, x->tc.th_lo, x->err);
    else
      k_exact_theta<false, false><<<(unsigned)((rows + 7) / 8), 256, 0, st>>>(
          d, x->th32, x->out, x->tc.th_hi, x->tc.th_lo, x->err);
    XCK(cudaGetLastError());
  }
  x->iterations += n_iter;
  x->have_posteriors = true;
  if (loglik_out) {
    XCK(cudaMemcpyAsync(x->h_ll, x->loglik, 8, cudaMemcpyDeviceToHost, st));
    const int rc = exact_sync(x);
    if (rc) return rc;
    *loglik_out = *x->h_ll;
  }
  return NFHMM_OK;
}

int nfhmm_exact_posteriors(nfhmm_exact* x, float* gamma, int on_device) {
  if (!x || !gamma) return fail(NFHMM_EINVAL, "NULL argument");
  if (!x->have_posteriors) return fail(NFHMM_ESTATE, "posteriors are defined after an iteration");
  XCK(cudaMemcpyAsync(gamma, x->gamma, (size_t)x->d.T * x->d.NC * 4,
                      on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDefault, x->user));
  if (!on_device) return exact_sync(x);
  return NFHMM_OK;
}

int nfhmm_exact_weights(nfhmm_exact* x, float* theta, int on_device) {
  if (!x || !theta) return fail(NFHMM_EINVAL, "NULL argument");
  const Dev& d = x->d;
  // theta_t(c)_k, T x N^S x S*K, from the item-major padded store
  for (int c = 0; c < d.NC; ++c)
    XCK(cudaMemcpy2DAsync(theta + (size_t)c * d.SK, (size_t)d.NC * d.SK * 4,
                          x->th32 + (size_t)c * d.Tp * d.SKp, (size_t)d.SKp * 4,
                          (size_t)d.SK * 4, d.T,
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDefault, x->user));
  if (!on_device) return exact_sync(x);
  return NFHMM_OK;
}

void nfhmm_exact_destroy(nfhmm_exact* x) { free_exact(x); }

}  // extern "C"
