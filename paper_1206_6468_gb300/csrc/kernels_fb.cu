// Forward-backward for the q(D^(s)) step of Section 3.2, parallel in time.
//
// With emissions e_t = exp(phi_t - max_n phi_t) and G_t = A diag(e_t), the
// forward row vector obeys a_t = a_{t-1} G_t (a_0 = pi diag(e_0)) and the
// backward column vector b_{t-1} = G_t b_t (b_{T-1} = 1).  Frames are cut
// into C chunks of L; chunk c covers frames t0..t1-1 and has the transfer
// matrix P_c = G_t0 ... G_{t1-1} (for c = 0 the first factor is diag(e_0)),
// so that a_{t1-1} = a_{t0-1} P_c (a_{L-1} = pi P_0) and b_{t0-1} = P_c b_{t1-1}.
// Three launches:
//   1. products: P_c of every chunk (N^3 per frame, all chunks in parallel);
//   2. scan:     forward and backward boundary vectors across chunks, one
//                warp per (source, direction), serial over C with the next
//                chunk matrices prefetched by cp.async; and log Z;
//   3. replay:   forward then backward inside each chunk from its boundary
//                vectors (one warp per chunk), giving
//                d-hat_t = a_t b_t / sum_n a_tn b_tn.
// Vectors and matrices are rescaled at every step.  The scale factors are
// kept in shared or global memory and their logs are summed in double after
// the serial loops, so no double-precision work sits on a serial path.
// Limits: chunk length 1 <= L <= FB_MAX_L, states N <= FB_MAX_N.
#include <math.h>

#include "nfhmm_device.cuh"
#include "nfhmm_kernels.h"

namespace nfhmm {

namespace {
constexpr int FB_MAX_N = 64;
constexpr int FB_MAX_L = 128;
constexpr int P_THREADS = 256;      // products
constexpr int R_WARPS_MAX = 4;      // replay: chunks per block (at most)
constexpr size_t SMEM_OPTIN = 227 * 1024;
constexpr int RING = 4;             // scan: prefetch depth


__host__ __device__ inline int round4(int n) { return (n + 3) & ~3; }

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

// Block-wide double sum (all threads get the result).
__device__ __forceinline__ double block_sum_d(double x, double* red) {
  const int nw = blockDim.x >> 5;
  x = warp_sum_d(x);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < nw; ++i) s += red[i];
  return s;
}

// e[f*N + n] = exp(phi_{t0+f,n} - m_f) for frames f of a chunk, one warp per
// frame starting at warp `w0` with stride `nw`; returns this warp's sum of m_f
// (double, valid in every lane).
__device__ double load_emissions(const float* phi_s, int N, int t0, int len, float* e, int w0,
                                 int nw) {
  const int lane = threadIdx.x & 31;
  double msum = 0.0;
  for (int f = w0; f < len; f += nw) {
    const float* row = phi_s + (size_t)(t0 + f) * N;
    const float x0 = lane < N ? row[lane] : -INFINITY;
    const float x1 = lane + 32 < N ? row[lane + 32] : -INFINITY;
    const float m = warp_max(fmaxf(x0, x1));
    if (lane < N) e[f * N + lane] = expf(x0 - m);
    if (lane + 32 < N) e[f * N + lane + 32] = expf(x1 - m);
    msum += (double)m;
  }
  return msum;
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}
}  // namespace

int fb_max_states() { return FB_MAX_N; }

int fb_default_chunk(int N, int T) {
  // chunk ~ sqrt(T): the serial scan (C = T/L steps) and the serial replay
  // (2L steps) then take about the same time.
  int L = (int)ceil(sqrt((double)T));
  if (L < 16) L = 16;
  if (L > 64) L = 64;
  if (L > T) L = T;
  (void)N;
  return L;
}

__host__ __device__ static inline int nn4(int N) { return round4(N * N); }

// --------------------------------------------------------------- 1. products
// Thread (ti, tj) owns a 4 x 4 block of P; P^T is kept in shared memory so
// that both operands of each k-step are float4 reads.  The matrix is scaled by
// its maximum after every step; the factors go to smem and their logs are
// summed at the end.  Writes P (row-major) and P^T, each at stride nn4(N).
__global__ void __launch_bounds__(P_THREADS) k_fb_products(FBArgs a) {
  extern __shared__ float sm[];
  const int N = a.N, NP = round4(N), L = a.L;
  const int c = blockIdx.x, s = blockIdx.y;
  const int t0 = c * L;
  const int len = min(a.T, t0 + L) - t0;
  double* dred = reinterpret_cast<double*>(sm);  // 8 doubles (first: aligned)
  float* As = sm + 16;            // N x NP, A[i][j] at i*NP + j
  float* PT0 = As + N * NP;       // NP x NP, P^T: P[i][k] at k*NP + i
  float* PT1 = PT0 + NP * NP;
  float* e = PT1 + NP * NP;       // L x N
  float* scl = e + L * N;         // L scale factors
  float* red = scl + FB_MAX_L;    // 64

  const float* As_g = a.A + (size_t)s * N * N;
  for (int i = threadIdx.x; i < N * NP; i += blockDim.x) {
    const int r = i / NP, cc = i - r * NP;
    As[i] = cc < N ? As_g[r * N + cc] : 0.f;
  }
  double msum = load_emissions(a.phi + (size_t)s * a.T * N, N, t0, len, e, threadIdx.x >> 5,
                               blockDim.x >> 5);
  __syncthreads();
  int parity = 0;

  const int NB = NP >> 2;
  const int ti = threadIdx.x / NB, tj = threadIdx.x - (threadIdx.x / NB) * NB;
  const bool act = threadIdx.x < NB * NB;
  float out[4][4];
  float lmax = 0.f;
  // first factor: A diag(e_t0), or diag(e_0) for the chunk that starts at pi
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = 4 * ti + r, jj = 4 * tj + q;
      float v = 0.f;
      if (act && i < N && jj < N) v = (c == 0) ? (i == jj ? e[jj] : 0.f) : As[i * NP + jj] * e[jj];
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
  float gmax = block_max(lmax, red, parity);  // barrier publishes cur
  for (int f = 1; f < len; ++f) {
    if (!(gmax > 0.f) || !isfinite(gmax)) {
      if (threadIdx.x == 0) atomicOr(a.err, ERR_FB_ZERO);
      gmax = 1.f;
    }
    if (threadIdx.x == 0) scl[f - 1] = gmax;
    const float inv = 1.f / gmax;
    float acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[r][q] = 0.f;
    if (act) {
#pragma unroll 4
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
  if (threadIdx.x == 0) scl[len - 1] = gmax;
  const float inv = 1.f / gmax;
  const size_t base = ((size_t)s * a.C + c) * nn4(N);
  float* Pg = a.P + base;
  float* PTg = a.PT + base;
  if (act) {
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i = 4 * ti + r, jj = 4 * tj + q;
        if (i < N && jj < N) {
          Pg[i * N + jj] = out[r][q] * inv;
          PTg[jj * N + i] = out[r][q] * inv;
        }
      }
  }
  __syncthreads();  // scl complete
  double lg = msum * ((threadIdx.x & 31) == 0 ? 1.0 : 0.0);
  for (int f = threadIdx.x; f < len; f += blockDim.x) lg += log((double)scl[f]);
  lg = block_sum_d(lg, dred);
  if (threadIdx.x == 0) a.Plog[(size_t)s * a.C + c] = lg;
}

// ------------------------------------------------------------------- 2. scan
// One warp per (source, direction).  Lane j holds states j and j + 32.
// blockIdx.y == 0: forward boundaries fwd[c] = normalised a at the end of
// chunk c (c = 0..C-1), log Z = sum_c (Plog_c + log lambda_c).
// blockIdx.y == 1: backward boundaries bwd[c] = normalised b at the end of
// chunk c (bwd[C-1] = 1).
__global__ void __launch_bounds__(32) k_fb_scan(FBArgs a) {
  extern __shared__ float sm[];
  const int N = a.N, C = a.C, NN = nn4(N);
  const int s = blockIdx.x;
  const bool fwd = blockIdx.y == 0;
  const int lane = threadIdx.x;
  float* ring = sm;                      // RING x NN
  float* v = ring + RING * NN;           // 64
  const size_t base = (size_t)s * C;
  const float* src = fwd ? a.P : a.PT;
  // chunk visited at step q: forward c = q (0..C-1), backward c = C-1-q (C-1..1)
  const int nsteps = fwd ? C : C - 1;
  auto chunk_of = [&](int q) { return fwd ? q : C - 1 - q; };
  auto prefetch = [&](int q) {
    if (q < nsteps) {
      const float* g = src + (base + chunk_of(q)) * NN;
      float* d = ring + (q % RING) * NN;
      for (int i = lane * 4; i < NN; i += 128) cp_async16(d + i, g + i);
    }
    cp_async_commit();
  };
#pragma unroll
  for (int q = 0; q < RING - 1; ++q) prefetch(q);

  // starting vector: pi (forward, into P_0) or ones (backward)
  float v0 = 0.f, v1 = 0.f;
  if (fwd) {
    if (lane < N) v0 = a.pi[(size_t)s * N + lane];
    if (lane + 32 < N) v1 = a.pi[(size_t)s * N + lane + 32];
  } else {
    if (lane < N) v0 = 1.f;
    if (lane + 32 < N) v1 = 1.f;
    if (lane < N) a.bwd[(base + C - 1) * N + lane] = 1.f;
    if (lane + 32 < N) a.bwd[(base + C - 1) * N + lane + 32] = 1.f;
  }
  v[lane] = v0;
  v[lane + 32] = v1;
  for (int q = 0; q < nsteps; ++q) {
    prefetch(q + RING - 1);
    cp_async_wait<RING - 1>();
    __syncwarp();
    const float* P = ring + (q % RING) * NN;
    // y_j = sum_i v_i P[i][j]  (P is P^T for the backward direction)
    float y0a = 0.f, y0b = 0.f, y1a = 0.f, y1b = 0.f;
    const int j0 = lane < N ? lane : 0, j1 = lane + 32 < N ? lane + 32 : 0;
    int i = 0;
    for (; i + 1 < N; i += 2) {
      const float va = v[i], vb = v[i + 1];
      y0a = fmaf(va, P[i * N + j0], y0a);
      y1a = fmaf(va, P[i * N + j1], y1a);
      y0b = fmaf(vb, P[(i + 1) * N + j0], y0b);
      y1b = fmaf(vb, P[(i + 1) * N + j1], y1b);
    }
    if (i < N) {
      const float va = v[i];
      y0a = fmaf(va, P[i * N + j0], y0a);
      y1a = fmaf(va, P[i * N + j1], y1a);
    }
    float y0 = lane < N ? y0a + y0b : 0.f;
    float y1 = lane + 32 < N ? y1a + y1b : 0.f;
    float lam = warp_sum(y0 + y1);
    if (!(lam > 0.f) || !isfinite(lam)) {
      if (lane == 0) atomicOr(a.err, ERR_FB_ZERO);
      lam = 1.f;
    }
    const float inv = 1.f / lam;
    y0 *= inv;
    y1 *= inv;
    __syncwarp();
    v[lane] = y0;
    v[lane + 32] = y1;
    const int c = chunk_of(q);
    if (fwd) {
      if (lane < N) a.fwd[(base + c) * N + lane] = y0;
      if (lane + 32 < N) a.fwd[(base + c) * N + lane + 32] = y1;
      if (lane == 0) a.lam[base + c] = lam;
    } else {
      if (lane < N) a.bwd[(base + c - 1) * N + lane] = y0;
      if (lane + 32 < N) a.bwd[(base + c - 1) * N + lane + 32] = y1;
    }
    __syncwarp();
  }
  cp_async_wait<0>();
  if (fwd) {
    __syncwarp();
    __threadfence_block();
    double lg = 0.0;
    for (int c = lane; c < C; c += 32) lg += a.Plog[base + c] + log((double)a.lam[base + c]);
    lg = warp_sum_d(lg);
    if (lane == 0) a.logZ[s] = lg;
  }
}

// ----------------------------------------------------------------- 3. replay
// One warp per chunk, blockDim/32 chunks per block sharing A and A^T in smem.
__global__ void __launch_bounds__(R_WARPS_MAX * 32) k_fb_replay(FBArgs a) {
  extern __shared__ float sm[];
  const int N = a.N, NP = round4(N), L = a.L;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int s = blockIdx.y;
  const int c = blockIdx.x * (blockDim.x >> 5) + warp;
  float* As = sm;                        // N x NP   A[i][j]
  float* AT = As + N * NP;               // N x NP   A[j][i] at j*NP + i
  float* wbase = AT + N * NP + warp * (2 * L * N + 64);
  float* e = wbase;                      // L x N
  float* av = e + L * N;                 // L x N forward vectors
  float* x = av + L * N;                 // 64
  const float* As_g = a.A + (size_t)s * N * N;
  for (int i = threadIdx.x; i < N * NP; i += blockDim.x) {
    const int r = i / NP, cc = i - r * NP;
    const float val = cc < N ? As_g[r * N + cc] : 0.f;
    As[i] = val;
    if (cc < N) AT[cc * NP + r] = val;
  }
  __syncthreads();
  if (c >= a.C) return;
  const int t0 = c * L;
  const int len = min(a.T, t0 + L) - t0;
  (void)load_emissions(a.phi + (size_t)s * a.T * N, N, t0, len, e, 0, 1);
  __syncwarp();
  const size_t base = (size_t)s * a.C;
  const bool h0 = lane < N, h1 = lane + 32 < N;
  const int j0 = h0 ? lane : 0, j1 = h1 ? lane + 32 : 0;

  // forward inside the chunk
  float y0, y1;
  if (c == 0) {
    y0 = h0 ? a.pi[(size_t)s * N + lane] * e[lane] : 0.f;
    y1 = h1 ? a.pi[(size_t)s * N + lane + 32] * e[lane + 32] : 0.f;
  } else {
    const float* prev = a.fwd + (base + c - 1) * N;
    x[lane] = h0 ? prev[lane] : 0.f;
    x[lane + 32] = h1 ? prev[lane + 32] : 0.f;
    __syncwarp();
    float p0 = 0.f, p1 = 0.f;
    for (int i = 0; i < N; ++i) {
      const float xi = x[i];
      p0 = fmaf(xi, As[i * NP + j0], p0);
      p1 = fmaf(xi, As[i * NP + j1], p1);
    }
    y0 = h0 ? p0 * e[lane] : 0.f;
    y1 = h1 ? p1 * e[lane + 32] : 0.f;
  }
  float lam = warp_sum(y0 + y1);
  float inv = lam > 0.f ? 1.f / lam : 1.f;
  if (h0) av[lane] = y0 * inv;
  if (h1) av[lane + 32] = y1 * inv;
  __syncwarp();
  for (int f = 1; f < len; ++f) {
    const float* ap = av + (f - 1) * N;
    float p0a = 0.f, p0b = 0.f, p1a = 0.f, p1b = 0.f;
    int i = 0;
    for (; i + 1 < N; i += 2) {
      const float xa = ap[i], xb = ap[i + 1];
      p0a = fmaf(xa, As[i * NP + j0], p0a);
      p1a = fmaf(xa, As[i * NP + j1], p1a);
      p0b = fmaf(xb, As[(i + 1) * NP + j0], p0b);
      p1b = fmaf(xb, As[(i + 1) * NP + j1], p1b);
    }
    if (i < N) {
      const float xa = ap[i];
      p0a = fmaf(xa, As[i * NP + j0], p0a);
      p1a = fmaf(xa, As[i * NP + j1], p1a);
    }
    y0 = h0 ? (p0a + p0b) * e[f * N + lane] : 0.f;
    y1 = h1 ? (p1a + p1b) * e[f * N + lane + 32] : 0.f;
    lam = warp_sum(y0 + y1);
    inv = lam > 0.f ? 1.f / lam : 1.f;
    if (h0) av[f * N + lane] = y0 * inv;
    if (h1) av[f * N + lane + 32] = y1 * inv;
    __syncwarp();
  }

  // backward inside the chunk and the marginals
  const float* bb = a.bwd + (base + c) * N;
  float b0 = h0 ? bb[lane] : 0.f, b1 = h1 ? bb[lane + 32] : 0.f;
  float* dh = a.dhat + ((size_t)s * a.T + t0) * N;
  unsigned bad = 0;
  for (int f = len - 1; f >= 0; --f) {
    const float d0 = h0 ? av[f * N + lane] * b0 : 0.f;
    const float d1 = h1 ? av[f * N + lane + 32] * b1 : 0.f;
    float z = warp_sum(d0 + d1);
    if (!(z > 0.f) || !isfinite(z)) {
      bad = 1;
      z = 1.f;
    }
    const float iz = 1.f / z;
    if (h0) dh[(size_t)f * N + lane] = d0 * iz;
    if (h1) dh[(size_t)f * N + lane + 32] = d1 * iz;
    if (f > 0) {
      __syncwarp();
      x[lane] = h0 ? e[f * N + lane] * b0 : 0.f;
      x[lane + 32] = h1 ? e[f * N + lane + 32] * b1 : 0.f;
      __syncwarp();
      float q0a = 0.f, q0b = 0.f, q1a = 0.f, q1b = 0.f;
      int k = 0;
      for (; k + 1 < N; k += 2) {
        const float xa = x[k], xb = x[k + 1];
        q0a = fmaf(AT[k * NP + j0], xa, q0a);
        q1a = fmaf(AT[k * NP + j1], xa, q1a);
        q0b = fmaf(AT[(k + 1) * NP + j0], xb, q0b);
        q1b = fmaf(AT[(k + 1) * NP + j1], xb, q1b);
      }
      if (k < N) {
        const float xa = x[k];
        q0a = fmaf(AT[k * NP + j0], xa, q0a);
        q1a = fmaf(AT[k * NP + j1], xa, q1a);
      }
      const float q0 = h0 ? q0a + q0b : 0.f, q1 = h1 ? q1a + q1b : 0.f;
      lam = warp_sum(q0 + q1);
      inv = lam > 0.f ? 1.f / lam : 1.f;
      b0 = q0 * inv;
      b1 = q1 * inv;
    }
  }
  if (bad && lane == 0) atomicOr(a.err, ERR_FB_ZERO);
}

static size_t smem_products(int N, int L) {
  const int NP = round4(N);
  (void)L;
  return (size_t)(16 + N * NP + 2 * NP * NP + FB_MAX_L * N + FB_MAX_L + 64) * sizeof(float);
}
static size_t smem_scan(int N) { return (size_t)(RING * nn4(N) + 64) * sizeof(float); }
static size_t smem_replay(int N, int L, int warps) {
  const int NP = round4(N);
  return (size_t)(2 * N * NP + warps * (2 * L * N + 64)) * sizeof(float);
}
static int replay_warps(int N, int L) {
  int w = R_WARPS_MAX;
  while (w > 1 && smem_replay(N, L, w) > SMEM_OPTIN) --w;
  return w;
}

size_t fb_scratch_bytes(int S, int N, int T, int L) {
  const int C = (T + L - 1) / L;
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  size_t b = 0;
  b += al((size_t)S * C * nn4(N) * sizeof(float));  // P
  b += al((size_t)S * C * nn4(N) * sizeof(float));  // P^T
  b += al((size_t)S * C * sizeof(double));          // Plog
  b += al((size_t)S * C * N * sizeof(float));       // fwd
  b += al((size_t)S * C * sizeof(float));           // lam
  b += al((size_t)S * C * N * sizeof(float));       // bwd
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
  a.P = reinterpret_cast<float*>(take(S * C * nn4((int)N) * sizeof(float)));
  a.PT = reinterpret_cast<float*>(take(S * C * nn4((int)N) * sizeof(float)));
  a.Plog = reinterpret_cast<double*>(take(S * C * sizeof(double)));
  a.fwd = reinterpret_cast<float*>(take(S * C * N * sizeof(float)));
  a.lam = reinterpret_cast<float*>(take(S * C * sizeof(float)));
  a.bwd = reinterpret_cast<float*>(take(S * C * N * sizeof(float)));
}

cudaError_t launch_fb(const FBArgs& a, cudaStream_t st, int* launches) {
  static cudaError_t attr = cudaErrorNotReady;
  if (attr == cudaErrorNotReady) {
    attr = cudaFuncSetAttribute(k_fb_products, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem_products(FB_MAX_N, FB_MAX_L));
    if (attr == cudaSuccess)
      attr = cudaFuncSetAttribute(k_fb_scan, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem_scan(FB_MAX_N));
    if (attr == cudaSuccess)
      attr = cudaFuncSetAttribute(k_fb_replay, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)SMEM_OPTIN);
  }
  if (attr != cudaSuccess) return attr;
  const int rw = replay_warps(a.N, a.L);
  k_fb_products<<<dim3(a.C, a.S), P_THREADS, smem_products(a.N, a.L), st>>>(a);
  k_fb_scan<<<dim3(a.S, 2), 32, smem_scan(a.N), st>>>(a);
  k_fb_replay<<<dim3((a.C + rw - 1) / rw, a.S), rw * 32, smem_replay(a.N, a.L, rw), st>>>(a);
  if (launches) *launches += 3;
  return cudaGetLastError();
}

}  // namespace nfhmm
