// Forward-backward for the q(D^(s)) step of Section 3.2, parallel in time.
//
// With emissions e_t = exp(phi_t - max_n phi_t) and G_t = A diag(e_t), the
// forward row vector obeys a_t = a_{t-1} G_t and the backward column vector
// b_{t-1} = G_t b_t.  Frames are cut into C chunks of L; chunk c (frames
// t0..t1-1) has the transfer matrix P_c = G_t0 ... G_{t1-1}, so that
// a_{t1-1} = a_{t0-1} P_c and b_{t0-1} = P_c b_{t1-1}.  Three launches:
//   1. products: P_c for every chunk c >= 1 (N^3 per frame, all chunks in
//      parallel) and the forward vector at the end of chunk 0;
//   2. scan:     the forward and backward boundary vectors across chunks
//      (serial over C, N^2 per chunk) and log Z;
//   3. replay:   forward then backward inside each chunk from its boundary
//      vectors, giving d-hat_t = a_t b_t / sum_n a_tn b_tn.
// Every vector and matrix is rescaled as it goes; the logs of the scale
// factors and of the per-frame maxima are accumulated in double for log Z.
// Chunk length 1 <= L <= FB_MAX_L; states N <= FB_MAX_N.
#include <math.h>

#include "nfhmm_device.cuh"
#include "nfhmm_kernels.h"

namespace nfhmm {

namespace {
constexpr int FB_MAX_N = 64;
constexpr int FB_MAX_L = 128;
constexpr int P_THREADS = 256;
constexpr int R_THREADS = 64;

__host__ __device__ inline int round4(int n) { return (n + 3) & ~3; }

// Block-wide sum; `red` holds two slots per warp, alternating with `parity`.
__device__ __forceinline__ float block_sum(float x, float* red, int& parity) {
  const int nw = blockDim.x >> 5;
  x = warp_sum(x);
  float* r = red + parity * 32;
  if ((threadIdx.x & 31) == 0) r[threadIdx.x >> 5] = x;
  __syncthreads();
  float s = 0.f;
  for (int i = 0; i < nw; ++i) s += r[i];
  parity ^= 1;
  return s;
}
__device__ __forceinline__ float block_max(float x, float* red, int& parity) {
  const int nw = blockDim.x >> 5;
  x = warp_max(x);
  float* r = red + parity * 32;
  if ((threadIdx.x & 31) == 0) r[threadIdx.x >> 5] = x;
  __syncthreads();
  float s = r[0];
  for (int i = 1; i < nw; ++i) s = fmaxf(s, r[i]);
  parity ^= 1;
  return s;
}

// e[f*N + n] = exp(phi_{t0+f,n} - m_f) for the chunk's frames; returns
// (in thread 0) sum_f m_f in double.  One warp per frame.
__device__ double load_emissions(const float* phi_s, int N, int t0, int len, float* e,
                                 double* dred) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double msum = 0.0;
  for (int f = warp; f < len; f += nw) {
    const float* row = phi_s + (size_t)(t0 + f) * N;
    const float x0 = lane < N ? row[lane] : -INFINITY;
    const float x1 = lane + 32 < N ? row[lane + 32] : -INFINITY;
    const float m = warp_max(fmaxf(x0, x1));
    if (lane < N) e[f * N + lane] = expf(x0 - m);
    if (lane + 32 < N) e[f * N + lane + 32] = expf(x1 - m);
    msum += (double)m;
  }
  if (lane == 0) dred[warp] = msum;
  __syncthreads();
  double tot = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < nw; ++i) tot += dred[i];
  return tot;
}
}  // namespace

int fb_max_states() { return FB_MAX_N; }

int fb_default_chunk(int N, int T) {
  // ~sqrt(T) chunks of ~sqrt(T) frames balances the serial scan against the
  // serial replay; at least 16 frames per chunk.
  int L = (int)ceil(sqrt((double)T));
  if (L < 16) L = 16;
  if (L > 64) L = 64;
  if (L > T) L = T;
  (void)N;
  return L;
}

// --------------------------------------------------------------- 1. products
__global__ void __launch_bounds__(P_THREADS) k_fb_products(FBArgs a) {
  extern __shared__ float sm[];
  const int N = a.N, NP = round4(N), L = a.L;
  const int c = blockIdx.x, s = blockIdx.y;
  const int t0 = c * L;
  const int len = min(a.T, t0 + L) - t0;
  double* dred = reinterpret_cast<double*>(sm);  // 8 (first: 8-byte aligned)
  float* As = sm + 16;            // N x NP, A[i][j] at i*NP + j
  float* PT0 = As + N * NP;       // NP x NP, P^T: P[i][k] at k*NP + i
  float* PT1 = PT0 + NP * NP;
  float* e = PT1 + NP * NP;       // L x N
  float* red = e + L * N;         // 64

  const float* As_g = a.A + (size_t)s * N * N;
  for (int i = threadIdx.x; i < N * NP; i += blockDim.x) {
    const int r = i / NP, cc = i - r * NP;
    As[i] = cc < N ? As_g[r * N + cc] : 0.f;
  }
  const double msum = load_emissions(a.phi + (size_t)s * a.T * N, N, t0, len, e, dred);
  __syncthreads();
  int parity = 0;

  if (c == 0) {
    // forward vector over chunk 0, from pi
    const int j = threadIdx.x;
    float x = (j < N) ? a.pi[(size_t)s * N + j] * e[j] : 0.f;
    float* av = PT0;  // reuse
    double logacc = 0.0;
    float lam = block_sum(x, red, parity);
    if (!(lam > 0.f)) {
      if (threadIdx.x == 0) atomicOr(a.err, ERR_FB_ZERO);
      lam = 1.f;
    }
    x /= lam;
    logacc += log((double)lam);
    if (j < NP) av[j] = x;
    __syncthreads();
    for (int f = 1; f < len; ++f) {
      float y = 0.f;
      if (j < N) {
        for (int i = 0; i < N; ++i) y = fmaf(av[i], As[i * NP + j], y);
        y *= e[f * N + j];
      }
      lam = block_sum(y, red, parity);
      if (!(lam > 0.f)) {
        if (threadIdx.x == 0) atomicOr(a.err, ERR_FB_ZERO);
        lam = 1.f;
      }
      y /= lam;
      logacc += log((double)lam);
      if (j < N) av[j] = y;
      x = y;
      __syncthreads();
    }
    if (j < N) a.fwd[((size_t)s * a.C + 0) * N + j] = x;
    if (threadIdx.x == 0) a.fwdlog[(size_t)s * a.C + 0] = msum + logacc;
    return;
  }

  // chunk product P = G_t0 ... G_{t1-1}; thread (ti, tj) owns a 4 x 4 block
  const int NB = NP >> 2;
  const int ti = threadIdx.x / NB, tj = threadIdx.x - (threadIdx.x / NB) * NB;
  const bool act = threadIdx.x < NB * NB;
  float out[4][4];
  float lmax = 0.f;
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = 4 * ti + r, jj = 4 * tj + q;
      const float v = (act && i < N && jj < N) ? As[i * NP + jj] * e[jj] : 0.f;
      out[r][q] = v;
      lmax = fmaxf(lmax, v);
    }
  float* cur = PT0;
  float* nxt = PT1;
  if (act) {
#pragma unroll
    for (int q = 0; q < 4; ++q)
      *reinterpret_cast<float4*>(&cur[(4 * tj + q) * NP + 4 * ti]) =
          make_float4(out[0][q], out[1][q], out[2][q], out[3][q]);
  }
  float gmax = block_max(lmax, red, parity);  // includes the barrier publishing cur
  double logscale = 0.0;
  for (int f = 1; f < len; ++f) {
    if (!(gmax > 0.f) || !isfinite(gmax)) {
      if (threadIdx.x == 0) atomicOr(a.err, ERR_FB_ZERO);
      gmax = 1.f;
    }
    const float inv = 1.f / gmax;
    logscale += log((double)gmax);
    float acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[r][q] = 0.f;
    if (act) {
      for (int k = 0; k < N; ++k) {
        const float4 p = *reinterpret_cast<const float4*>(&cur[k * NP + 4 * ti]);
        const float4 b = *reinterpret_cast<const float4*>(&As[k * NP + 4 * tj]);
        const float pv[4] = {p.x, p.y, p.z, p.w};
        const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[r][q] = fmaf(pv[r], bv[q], acc[r][q]);
      }
    }
    lmax = 0.f;
    const float* ef = e + f * N;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int jj = 4 * tj + q;
      const float sc = (jj < N) ? ef[jj] * inv : 0.f;
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        out[r][q] = acc[r][q] * sc;
        lmax = fmaxf(lmax, out[r][q]);
      }
    }
    if (act) {
#pragma unroll
      for (int q = 0; q < 4; ++q)
        *reinterpret_cast<float4*>(&nxt[(4 * tj + q) * NP + 4 * ti]) =
            make_float4(out[0][q], out[1][q], out[2][q], out[3][q]);
    }
    float* tmp = cur;
    cur = nxt;
    nxt = tmp;
    gmax = block_max(lmax, red, parity);
  }
  if (!(gmax > 0.f) || !isfinite(gmax)) {
    if (threadIdx.x == 0) atomicOr(a.err, ERR_FB_ZERO);
    gmax = 1.f;
  }
  const float inv = 1.f / gmax;
  float* Pg = a.P + ((size_t)s * a.C + c) * N * N;
  if (act) {
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i = 4 * ti + r, jj = 4 * tj + q;
        if (i < N && jj < N) Pg[i * N + jj] = out[r][q] * inv;
      }
  }
  if (threadIdx.x == 0) a.Plog[(size_t)s * a.C + c] = msum + logscale + log((double)gmax);
}

// ------------------------------------------------------------------- 2. scan
// blockIdx.y == 0: forward boundaries and log Z; == 1: backward boundaries.
__global__ void __launch_bounds__(P_THREADS) k_fb_scan(FBArgs a) {
  extern __shared__ float sm[];
  const int N = a.N, C = a.C;
  const int s = blockIdx.x;
  const bool fwd = blockIdx.y == 0;
  float* P = sm;            // N x N
  float* v = P + N * N;     // N
  float* red = v + FB_MAX_N;
  const int per = (N * N + blockDim.x - 1) / blockDim.x;
  constexpr int MAXPER = (FB_MAX_N * FB_MAX_N + P_THREADS - 1) / P_THREADS;
  float reg[MAXPER];
  int parity = 0;
  const int j = threadIdx.x;
  const size_t base = (size_t)s * C;

  auto fetch = [&](int cc) {
    const float* src = a.P + (base + cc) * N * N;
#pragma unroll
    for (int q = 0; q < MAXPER; ++q) {
      const int idx = threadIdx.x + q * blockDim.x;
      if (q < per && idx < N * N) reg[q] = src[idx];
    }
  };
  auto publish = [&]() {
#pragma unroll
    for (int q = 0; q < MAXPER; ++q) {
      const int idx = threadIdx.x + q * blockDim.x;
      if (q < per && idx < N * N) P[idx] = reg[q];
    }
  };

  if (fwd) {
    double logacc = a.fwdlog[base];
    if (j < N) v[j] = a.fwd[base * N + j];
    if (C > 1) fetch(1);
    for (int cc = 1; cc < C; ++cc) {
      __syncthreads();  // previous step done with P and v
      publish();
      __syncthreads();
      if (cc + 1 < C) fetch(cc + 1);
      float y = 0.f;
      if (j < N)
        for (int i = 0; i < N; ++i) y = fmaf(v[i], P[i * N + j], y);
      float lam = block_sum(y, red, parity);
      if (!(lam > 0.f)) {
        if (threadIdx.x == 0) atomicOr(a.err, ERR_FB_ZERO);
        lam = 1.f;
      }
      y /= lam;
      logacc += a.Plog[base + cc] + log((double)lam);
      if (j < N) {
        v[j] = y;
        a.fwd[(base + cc) * N + j] = y;
      }
    }
    if (threadIdx.x == 0) a.logZ[s] = logacc;
  } else {
    if (j < N) {
      v[j] = 1.f;
      a.bwd[(base + C - 1) * N + j] = 1.f;
    }
    if (C > 1) fetch(C - 1);
    for (int cc = C - 1; cc >= 1; --cc) {
      __syncthreads();
      publish();
      __syncthreads();
      if (cc - 1 >= 1) fetch(cc - 1);
      float y = 0.f;
      if (j < N)
        for (int k = 0; k < N; ++k) y = fmaf(P[j * N + k], v[k], y);
      float lam = block_sum(y, red, parity);
      if (!(lam > 0.f)) {
        if (threadIdx.x == 0) atomicOr(a.err, ERR_FB_ZERO);
        lam = 1.f;
      }
      y /= lam;
      if (j < N) {
        v[j] = y;
        a.bwd[(base + cc - 1) * N + j] = y;
      }
    }
  }
}

// ----------------------------------------------------------------- 3. replay
__global__ void __launch_bounds__(R_THREADS) k_fb_replay(FBArgs a) {
  extern __shared__ float sm[];
  const int N = a.N, NP = round4(N), L = a.L;
  const int c = blockIdx.x, s = blockIdx.y;
  const int t0 = c * L;
  const int len = min(a.T, t0 + L) - t0;
  double* dred = reinterpret_cast<double*>(sm);  // 8 (first: 8-byte aligned)
  float* As = sm + 16;          // N x NP
  float* e = As + N * NP;       // L x N
  float* av = e + L * N;        // L x NP forward vectors
  float* bv = av + L * NP;      // NP
  float* red = bv + NP;         // 64
  const float* As_g = a.A + (size_t)s * N * N;
  for (int i = threadIdx.x; i < N * NP; i += blockDim.x) {
    const int r = i / NP, cc = i - r * NP;
    As[i] = cc < N ? As_g[r * N + cc] : 0.f;
  }
  (void)load_emissions(a.phi + (size_t)s * a.T * N, N, t0, len, e, dred);
  const int j = threadIdx.x;
  const size_t base = (size_t)s * a.C;
  if (c > 0 && j < N) bv[j] = a.fwd[(base + c - 1) * N + j];
  __syncthreads();
  int parity = 0;

  // forward inside the chunk
  float x;
  if (c == 0) {
    x = (j < N) ? a.pi[(size_t)s * N + j] * e[j] : 0.f;
  } else {
    x = 0.f;
    if (j < N) {
      for (int i = 0; i < N; ++i) x = fmaf(bv[i], As[i * NP + j], x);
      x *= e[j];
    }
  }
  float lam = block_sum(x, red, parity);
  if (!(lam > 0.f)) lam = 1.f;
  x /= lam;
  if (j < N) av[j] = x;
  __syncthreads();
  for (int f = 1; f < len; ++f) {
    float y = 0.f;
    if (j < N) {
      const float* ap = av + (f - 1) * NP;
      for (int i = 0; i < N; ++i) y = fmaf(ap[i], As[i * NP + j], y);
      y *= e[f * N + j];
    }
    lam = block_sum(y, red, parity);
    if (!(lam > 0.f)) lam = 1.f;
    if (j < N) av[f * NP + j] = y / lam;
    __syncthreads();
  }

  // backward inside the chunk, marginals
  float b = (j < N) ? a.bwd[(base + c) * N + j] : 0.f;
  float* dh = a.dhat + ((size_t)s * a.T + t0) * N;
  for (int f = len - 1; f >= 0; --f) {
    const float d = (j < N) ? av[f * NP + j] * b : 0.f;
    float z = block_sum(d, red, parity);
    if (!(z > 0.f)) {
      if (threadIdx.x == 0) atomicOr(a.err, ERR_FB_ZERO);
      z = 1.f;
    }
    if (j < N) dh[(size_t)f * N + j] = d / z;
    if (f > 0) {
      if (j < N) bv[j] = e[f * N + j] * b;
      __syncthreads();
      float y = 0.f;
      if (j < N)
        for (int k = 0; k < N; ++k) y = fmaf(As[j * NP + k], bv[k], y);
      lam = block_sum(y, red, parity);
      if (!(lam > 0.f)) lam = 1.f;
      b = y / lam;
    }
  }
}

static size_t smem_products(int N, int L) {
  const int NP = round4(N);
  return (size_t)(16 + N * NP + 2 * NP * NP + L * N + 64) * sizeof(float);
}
static size_t smem_scan(int N) { return (size_t)(N * N + FB_MAX_N + 64) * sizeof(float); }
static size_t smem_replay(int N, int L) {
  const int NP = round4(N);
  return (size_t)(16 + N * NP + L * N + L * NP + NP + 64) * sizeof(float);
}

size_t fb_scratch_bytes(int S, int N, int T, int L) {
  const int C = (T + L - 1) / L;
  size_t b = 0;
  b += (size_t)S * C * N * N * sizeof(float);     // P
  b = (b + 255) & ~(size_t)255;
  b += (size_t)S * C * sizeof(double);            // Plog
  b = (b + 255) & ~(size_t)255;
  b += (size_t)S * C * N * sizeof(float);         // fwd
  b = (b + 255) & ~(size_t)255;
  b += (size_t)S * C * sizeof(double);            // fwdlog
  b = (b + 255) & ~(size_t)255;
  b += (size_t)S * C * N * sizeof(float);         // bwd
  b = (b + 255) & ~(size_t)255;
  return b;
}

void fb_carve_scratch(FBArgs& a, void* base) {
  char* p = reinterpret_cast<char*>(base);
  const size_t S = a.S, C = a.C, N = a.N;
  auto take = [&](size_t bytes) {
    char* r = p;
    p += (bytes + 255) & ~(size_t)255;
    return r;
  };
  a.P = reinterpret_cast<float*>(take(S * C * N * N * sizeof(float)));
  a.Plog = reinterpret_cast<double*>(take(S * C * sizeof(double)));
  a.fwd = reinterpret_cast<float*>(take(S * C * N * sizeof(float)));
  a.fwdlog = reinterpret_cast<double*>(take(S * C * sizeof(double)));
  a.bwd = reinterpret_cast<float*>(take(S * C * N * sizeof(float)));
}

void launch_fb(const FBArgs& a, cudaStream_t st, int* launches) {
  static bool attr_done = false;
  if (!attr_done) {
    cudaFuncSetAttribute(k_fb_products, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem_products(FB_MAX_N, FB_MAX_L));
    cudaFuncSetAttribute(k_fb_replay, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem_replay(FB_MAX_N, FB_MAX_L));
    attr_done = true;
  }
  k_fb_products<<<dim3(a.C, a.S), P_THREADS, smem_products(a.N, a.L), st>>>(a);
  k_fb_scan<<<dim3(a.S, 2), P_THREADS, smem_scan(a.N), st>>>(a);
  k_fb_replay<<<dim3(a.C, a.S), R_THREADS, smem_replay(a.N, a.L), st>>>(a);
  if (launches) *launches += 3;
}

}  // namespace nfhmm
