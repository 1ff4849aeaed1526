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
//   3. replay:   inside each chunk, a forward warp and a backward warp run
//                concurrently from the chunk's boundary vectors; then
//                d-hat_t = a_t b_t / sum_n a_tn b_tn.
// Vectors and matrices are rescaled at every step.  The scale factors are
// kept in shared or global memory and their logs are summed in double after
// the serial loops, so no double-precision work sits on a serial path.
// States are padded to NP = 8*ceil(N/8) with zero rows/columns in A, zero
// emissions and zero initial probability, so padded states never carry mass;
// every kernel is instantiated per NP and its loops unroll fully.
// Limits: chunk length 1 <= L <= FB_MAX_L, states N <= FB_MAX_N.
#include <math.h>

#include "nfhmm_device.cuh"
#include "nfhmm_kernels.h"

namespace nfhmm {

namespace {
constexpr int FB_MAX_N = 64;
constexpr int FB_MAX_L = 128;
constexpr int RING = 8;             // scan: prefetch depth
constexpr int R_CHUNKS_MAX = 4;     // replay: chunks per block (2 warps each)
constexpr size_t SMEM_OPTIN = 227 * 1024;

__host__ __device__ constexpr int pad8(int n) { return (n + 7) & ~7; }

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

// Emissions of frames [t0, t0 + len) of one source into e[f*NP + n] (padded
// states 0): the chunk's phi rows are contiguous in global memory and are
// first copied with coalesced loads by the whole block, then one warp per
// frame takes max and exp.  Returns the warp's sum of frame maxima (double,
// valid in every lane).
template <int NP>
__device__ double load_emissions(const float* phi_s, int N, int t0, int len, float* e) {
  const float* src = phi_s + (size_t)t0 * N;
  const int tot = len * N;
  for (int i = threadIdx.x; i < tot; i += blockDim.x) {
    const int f = i / N, n = i - f * N;
    e[f * NP + n] = src[i];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  double msum = 0.0;
  for (int f = threadIdx.x >> 5; f < len; f += blockDim.x >> 5) {
    float* row = e + f * NP;
    const float x0 = lane < N ? row[lane] : -INFINITY;
    const float x1 = lane + 32 < N ? row[lane + 32] : -INFINITY;
    const float m = warp_max(fmaxf(x0, x1));
    __syncwarp();
    if (lane < NP) row[lane] = lane < N ? expf(x0 - m) : 0.f;
    if (lane + 32 < NP) row[lane + 32] = lane + 32 < N ? expf(x1 - m) : 0.f;
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
  // The chunk products are the bulk of the work and run one chunk per block;
  // chunks of up to ~48 frames keep a paper-size job (S = 2, T = 3000) to
  // about one wave on 152 SMs while the serial scan stays ~T/48 steps long.
  int L = (int)ceil(sqrt((double)T)) - 6;
  if (L < 16) L = 16;
  if (L > 48) L = 48;
  if (L > T) L = T;
  (void)N;
  return L;
}

// P and P^T of one chunk are stored padded: NP x NP floats each.
static inline size_t mat_floats(int N) { return (size_t)pad8(N) * pad8(N); }

// --------------------------------------------------------------- 1. products
// Thread (ti, tj) owns rows 4ti..4ti+3 and columns TC*tj..TC*tj+TC-1 of P.
// Its TC columns of A stay in registers for the whole chunk; P^T is double
// buffered in shared memory (one float4 read per k).  The matrix is scaled by
// its maximum after every step.
template <int NP>
struct ProdCfg {
  static constexpr int TC = NP <= 40 ? 4 : 2;   // columns per thread
  static constexpr int NI = NP / 4, NJ = NP / TC;
  static constexpr int THREADS = ((NI * NJ + 31) / 32) * 32;
};

template <int NP>
__global__ void __launch_bounds__(ProdCfg<NP>::THREADS) k_fb_products(FBArgs a) {
  using Cfg = ProdCfg<NP>;
  constexpr int TC = Cfg::TC;
  extern __shared__ float sm[];
  const int N = a.N, L = a.L;
  const int c = blockIdx.x, s = blockIdx.y;
  const int t0 = c * L;
  const int len = min(a.T, t0 + L) - t0;
  double* dred = reinterpret_cast<double*>(sm);  // 32 doubles
  float* PT0 = sm + 64;                          // NP x NP, P[i][k] at k*NP + i
  float* PT1 = PT0 + NP * NP;
  float* e = PT1 + NP * NP;                      // L x NP
  float* scl = e + L * NP;                       // L
  float* red = scl + FB_MAX_L;                   // 64

  const int ti = threadIdx.x / Cfg::NJ, tj = threadIdx.x % Cfg::NJ;
  const bool act = threadIdx.x < Cfg::NI * Cfg::NJ;
  // this thread's columns of A, padded with zeros
  float Ar[NP][TC];
  const float* As_g = a.A + (size_t)s * N * N;
#pragma unroll
  for (int k = 0; k < NP; ++k)
#pragma unroll
    for (int q = 0; q < TC; ++q) {
      const int j = TC * tj + q;
      Ar[k][q] = (act && k < N && j < N) ? As_g[k * N + j] : 0.f;
    }
  double msum = load_emissions<NP>(a.phi + (size_t)s * a.T * N, N, t0, len, e);
  __syncthreads();
  int parity = 0;

  float out[4][TC];
  float lmax = 0.f;
  // first factor: A diag(e_t0), or diag(e_0) for the chunk that starts at pi
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int q = 0; q < TC; ++q) {
      const int i = 4 * ti + r, j = TC * tj + q;
      float v = 0.f;
      if (act) {
        if (c == 0) {
          v = (i == j) ? e[j] : 0.f;
        } else {
#pragma unroll
          for (int k = 0; k < NP; ++k)
            if (k == i) v = Ar[k][q] * e[j];
        }
      }
      out[r][q] = v;
      lmax = fmaxf(lmax, v);
    }
  float* cur = PT0;
  float* nxt = PT1;
  if (act) {
#pragma unroll
    for (int q = 0; q < TC; ++q)
      *reinterpret_cast<float4*>(&cur[(TC * tj + q) * NP + 4 * ti]) =
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
    float acc[4][TC];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int q = 0; q < TC; ++q) acc[r][q] = 0.f;
    if (act) {
#pragma unroll
      for (int k = 0; k < NP; ++k) {
        const float4 p = *reinterpret_cast<const float4*>(&cur[k * NP + 4 * ti]);
#pragma unroll
        for (int q = 0; q < TC; ++q) {
          acc[0][q] = fmaf(p.x, Ar[k][q], acc[0][q]);
          acc[1][q] = fmaf(p.y, Ar[k][q], acc[1][q]);
          acc[2][q] = fmaf(p.z, Ar[k][q], acc[2][q]);
          acc[3][q] = fmaf(p.w, Ar[k][q], acc[3][q]);
        }
      }
    }
    lmax = 0.f;
    const float* ef = e + f * NP;
#pragma unroll
    for (int q = 0; q < TC; ++q) {
      const float sc = act ? ef[TC * tj + q] * inv : 0.f;
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        out[r][q] = acc[r][q] * sc;
        lmax = fmaxf(lmax, out[r][q]);
      }
    }
    if (act) {
#pragma unroll
      for (int q = 0; q < TC; ++q)
        *reinterpret_cast<float4*>(&nxt[(TC * tj + q) * NP + 4 * ti]) =
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
  const size_t base = ((size_t)s * a.C + c) * NP * NP;
  float* Pg = a.P + base;
  float* PTg = a.PT + base;
  if (act) {
#pragma unroll
    for (int q = 0; q < TC; ++q) {
      const float4 v = make_float4(out[0][q] * inv, out[1][q] * inv, out[2][q] * inv,
                                   out[3][q] * inv);
      *reinterpret_cast<float4*>(&PTg[(TC * tj + q) * NP + 4 * ti]) = v;
#pragma unroll
      for (int r = 0; r < 4; ++r) Pg[(4 * ti + r) * NP + TC * tj + q] = out[r][q] * inv;
    }
  }
  __syncthreads();  // scl complete
  double lg = msum * ((threadIdx.x & 31) == 0 ? 1.0 : 0.0);
  for (int f = threadIdx.x; f < len; f += blockDim.x) lg += log((double)scl[f]);
  lg = block_sum_d(lg, dred);
  if (threadIdx.x == 0) a.Plog[(size_t)s * a.C + c] = lg;
}

// ------------------------------------------------------------------- 2. scan
// One warp per (source, direction); lane j holds states j and j + 32.
// blockIdx.y == 0: forward boundaries fwd[c] = normalised a at the end of
// chunk c (c = 0..C-1) and log Z = sum_c (Plog_c + log lambda_c).
// blockIdx.y == 1: backward boundaries bwd[c] = normalised b at the end of
// chunk c (bwd[C-1] = 1), from P^T.
template <int NP>
__global__ void __launch_bounds__(32) k_fb_scan(FBArgs a) {
  extern __shared__ float sm[];
  constexpr int NN = NP * NP;
  const int N = a.N, C = a.C;
  const int s = blockIdx.x;
  const bool fwd = blockIdx.y == 0;
  const int lane = threadIdx.x;
  float* ring = sm;                      // RING x NN
  float* v = ring + RING * NN;           // 64 (+ padding)
  const size_t base = (size_t)s * C;
  const float* src = fwd ? a.P : a.PT;
  const int nsteps = fwd ? C : C - 1;
  auto chunk_of = [&](int q) { return fwd ? q : C - 1 - q; };
  auto prefetch = [&](int q) {
    if (q < nsteps) {
      const float* g = src + (base + chunk_of(q)) * NN;
      float* d = ring + (q % RING) * NN;
#pragma unroll
      for (int i = lane * 4; i < NN; i += 128) cp_async16(d + i, g + i);
    }
    cp_async_commit();
  };
#pragma unroll
  for (int q = 0; q < RING - 1; ++q) prefetch(q);

  const bool h0 = lane < N, h1 = lane + 32 < N;
  float v0 = 0.f, v1 = 0.f;
  if (fwd) {
    if (h0) v0 = a.pi[(size_t)s * N + lane];
    if (h1) v1 = a.pi[(size_t)s * N + lane + 32];
  } else {
    v0 = h0 ? 1.f : 0.f;
    v1 = h1 ? 1.f : 0.f;
    if (h0) a.bwd[(base + C - 1) * N + lane] = 1.f;
    if (h1) a.bwd[(base + C - 1) * N + lane + 32] = 1.f;
  }
  v[lane] = v0;
  v[lane + 32] = v1;
  for (int q = 0; q < nsteps; ++q) {
    prefetch(q + RING - 1);
    cp_async_wait<RING - 1>();
    __syncwarp();
    const float* P = ring + (q % RING) * NN;
    // y_j = sum_i v_i P[i][j]  (P^T for the backward direction)
    float y0[4] = {0.f, 0.f, 0.f, 0.f}, y1[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int i = 0; i < NP; i += 4) {
      const float4 vv = *reinterpret_cast<const float4*>(&v[i]);
      const float vi[4] = {vv.x, vv.y, vv.z, vv.w};
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (lane < NP) y0[u] = fmaf(vi[u], P[(i + u) * NP + lane], y0[u]);
        if (lane + 32 < NP) y1[u] = fmaf(vi[u], P[(i + u) * NP + lane + 32], y1[u]);
      }
    }
    float r0 = (y0[0] + y0[1]) + (y0[2] + y0[3]);
    float r1 = (y1[0] + y1[1]) + (y1[2] + y1[3]);
    float lam = warp_sum(r0 + r1);
    if (!(lam > 0.f) || !isfinite(lam)) {
      if (lane == 0) atomicOr(a.err, ERR_FB_ZERO);
      lam = 1.f;
    }
    const float inv = 1.f / lam;
    r0 *= inv;
    r1 *= inv;
    __syncwarp();
    v[lane] = r0;
    v[lane + 32] = r1;
    const int c = chunk_of(q);
    if (fwd) {
      if (h0) a.fwd[(base + c) * N + lane] = r0;
      if (h1) a.fwd[(base + c) * N + lane + 32] = r1;
      if (lane == 0) a.lam[base + c] = lam;
    } else {
      if (h0) a.bwd[(base + c - 1) * N + lane] = r0;
      if (h1) a.bwd[(base + c - 1) * N + lane + 32] = r1;
    }
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
// Two warps per chunk: warp 2q runs the forward recursion of chunk q (A's
// columns j, j+32 in registers), warp 2q+1 the backward recursion (A's rows
// j, j+32 in registers), concurrently; then both combine a_t b_t into d-hat.
template <int NP>
__global__ void __launch_bounds__(R_CHUNKS_MAX * 64) k_fb_replay(FBArgs a) {
  extern __shared__ float sm[];
  const int N = a.N, L = a.L;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int chunks = blockDim.x >> 6;
  const int q = warp >> 1;
  const bool is_fwd = (warp & 1) == 0;
  const int s = blockIdx.y;
  const int c = blockIdx.x * chunks + q;
  const int per = 3 * L * NP + 128;
  float* e = sm + q * per;               // L x NP
  float* av = e + L * NP;                // L x NP forward vectors
  float* bv = av + L * NP;               // L x NP backward vectors
  float* x = bv + L * NP + (is_fwd ? 0 : 64);  // 64 per warp
  const bool live = c < a.C;
  const int t0 = c * L;
  const int len = live ? min(a.T, t0 + L) - t0 : 0;
  const float* Ag = a.A + (size_t)s * N * N;
  const bool h0 = lane < N, h1 = lane + 32 < N;
  // forward warp: A[k][j] for j = lane, lane + 32; backward warp: A[j][k]
  float A0[NP], A1[NP];
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    if (is_fwd) {
      A0[k] = (h0 && k < N) ? Ag[k * N + lane] : 0.f;
      A1[k] = (h1 && k < N) ? Ag[k * N + lane + 32] : 0.f;
    } else {
      A0[k] = (h0 && k < N) ? Ag[lane * N + k] : 0.f;
      A1[k] = (h1 && k < N) ? Ag[(lane + 32) * N + k] : 0.f;
    }
  }
  if (live) {
    // the chunk's two warps copy its phi rows (contiguous) with coalesced loads
    const float* src = a.phi + (size_t)s * a.T * N + (size_t)t0 * N;
    const int tot = len * N;
    for (int i = (int)threadIdx.x - q * 64; i < tot; i += 64) {
      const int f = i / N, n = i - f * N;
      e[f * NP + n] = src[i];
    }
  }
  __syncthreads();
  if (live) {
    for (int f = is_fwd ? 0 : 1; f < len; f += 2) {
      float* row = e + f * NP;
      const float x0 = h0 ? row[lane] : -INFINITY;
      const float x1 = h1 ? row[lane + 32] : -INFINITY;
      const float m = warp_max(fmaxf(x0, x1));
      __syncwarp();
      if (lane < NP) row[lane] = h0 ? expf(x0 - m) : 0.f;
      if (lane + 32 < NP) row[lane + 32] = h1 ? expf(x1 - m) : 0.f;
    }
  }
  __syncthreads();
  const size_t base = (size_t)s * a.C;
  if (live) {
    float* vec = is_fwd ? av : bv;
    float r0, r1;
    if (is_fwd) {
      if (c == 0) {
        r0 = h0 ? a.pi[(size_t)s * N + lane] * e[lane] : 0.f;
        r1 = h1 ? a.pi[(size_t)s * N + lane + 32] * e[lane + 32] : 0.f;
      } else {
        const float* prev = a.fwd + (base + c - 1) * N;
        x[lane] = h0 ? prev[lane] : 0.f;
        x[lane + 32] = h1 ? prev[lane + 32] : 0.f;
        __syncwarp();
        float p0 = 0.f, p1 = 0.f;
#pragma unroll
        for (int i = 0; i < NP; ++i) {
          p0 = fmaf(x[i], A0[i], p0);
          p1 = fmaf(x[i], A1[i], p1);
        }
        r0 = h0 ? p0 * e[lane] : 0.f;
        r1 = h1 ? p1 * e[lane + 32] : 0.f;
      }
    } else {
      const float* bb = a.bwd + (base + c) * N;
      r0 = h0 ? bb[lane] : 0.f;
      r1 = h1 ? bb[lane + 32] : 0.f;
    }
    // forward: vec[0] then f = 1..len-1; backward: vec[len-1] then f = len-2..0
    int f = is_fwd ? 0 : len - 1;
    float lam = warp_sum(r0 + r1);
    float inv = lam > 0.f ? 1.f / lam : 1.f;
    r0 *= inv;
    r1 *= inv;
    if (lane < NP) vec[f * NP + lane] = r0;
    if (lane + 32 < NP) vec[f * NP + lane + 32] = r1;
    for (int step = 1; step < len; ++step) {
      // forward: a_f = (a_{f-1} A) (.) e_f;  backward: b_{f-1} = A (e_f (.) b_f)
      const float* ef = e + f * NP;
      __syncwarp();
      if (is_fwd) {
        x[lane] = r0;
        x[lane + 32] = r1;
      } else {
        x[lane] = lane < NP ? r0 * ef[lane] : 0.f;
        x[lane + 32] = lane + 32 < NP ? r1 * ef[lane + 32] : 0.f;
      }
      __syncwarp();
      float p0[4] = {0.f, 0.f, 0.f, 0.f}, p1[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int i = 0; i < NP; i += 4) {
        const float4 xv = *reinterpret_cast<const float4*>(&x[i]);
        p0[0] = fmaf(xv.x, A0[i], p0[0]);
        p0[1] = fmaf(xv.y, A0[i + 1], p0[1]);
        p0[2] = fmaf(xv.z, A0[i + 2], p0[2]);
        p0[3] = fmaf(xv.w, A0[i + 3], p0[3]);
        p1[0] = fmaf(xv.x, A1[i], p1[0]);
        p1[1] = fmaf(xv.y, A1[i + 1], p1[1]);
        p1[2] = fmaf(xv.z, A1[i + 2], p1[2]);
        p1[3] = fmaf(xv.w, A1[i + 3], p1[3]);
      }
      f += is_fwd ? 1 : -1;
      float y0 = (p0[0] + p0[1]) + (p0[2] + p0[3]);
      float y1 = (p1[0] + p1[1]) + (p1[2] + p1[3]);
      if (is_fwd) {
        const float* en = e + f * NP;
        y0 = lane < NP ? y0 * en[lane] : 0.f;
        y1 = lane + 32 < NP ? y1 * en[lane + 32] : 0.f;
      }
      lam = warp_sum(y0 + y1);
      inv = lam > 0.f ? 1.f / lam : 1.f;
      r0 = y0 * inv;
      r1 = y1 * inv;
      if (lane < NP) vec[f * NP + lane] = r0;
      if (lane + 32 < NP) vec[f * NP + lane + 32] = r1;
    }
  }
  __syncthreads();
  if (live) {
    float* dh = a.dhat + ((size_t)s * a.T + t0) * N;
    unsigned bad = 0;
    for (int f = is_fwd ? 0 : 1; f < len; f += 2) {
      const float d0 = h0 ? av[f * NP + lane] * bv[f * NP + lane] : 0.f;
      const float d1 = h1 ? av[f * NP + lane + 32] * bv[f * NP + lane + 32] : 0.f;
      float z = warp_sum(d0 + d1);
      if (!(z > 0.f) || !isfinite(z)) {
        bad = 1;
        z = 1.f;
      }
      const float iz = 1.f / z;
      if (h0) dh[(size_t)f * N + lane] = d0 * iz;
      if (h1) dh[(size_t)f * N + lane + 32] = d1 * iz;
    }
    if (bad && lane == 0) atomicOr(a.err, ERR_FB_ZERO);
  }
}

// ------------------------------------------------------------------ launch
template <int NP>
static size_t smem_products() {
  return (size_t)(64 + 2 * NP * NP + FB_MAX_L * NP + FB_MAX_L + 64) * sizeof(float);
}
template <int NP>
static size_t smem_scan() {
  return (size_t)(RING * NP * NP + 128) * sizeof(float);
}
static size_t smem_replay_chunk(int NP, int L) { return (size_t)(3 * L * NP + 128) * sizeof(float); }
static int replay_chunks(int NP, int L) {
  int rc = R_CHUNKS_MAX;
  while (rc > 1 && rc * smem_replay_chunk(NP, L) > SMEM_OPTIN) --rc;
  return rc;
}

template <int NP>
static cudaError_t launch_np(const FBArgs& a, cudaStream_t st) {
  static cudaError_t attr = cudaErrorNotReady;
  if (attr == cudaErrorNotReady) {
    attr = cudaFuncSetAttribute(k_fb_products<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem_products<NP>());
    if (attr == cudaSuccess)
      attr = cudaFuncSetAttribute(k_fb_scan<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem_scan<NP>());
    if (attr == cudaSuccess)
      attr = cudaFuncSetAttribute(k_fb_replay<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)SMEM_OPTIN);
  }
  if (attr != cudaSuccess) return attr;
  const int rc = replay_chunks(NP, a.L);
  k_fb_products<NP><<<dim3(a.C, a.S), ProdCfg<NP>::THREADS, smem_products<NP>(), st>>>(a);
  k_fb_scan<NP><<<dim3(a.S, 2), 32, smem_scan<NP>(), st>>>(a);
  k_fb_replay<NP><<<dim3((a.C + rc - 1) / rc, a.S), rc * 64, rc * smem_replay_chunk(NP, a.L),
                    st>>>(a);
  return cudaGetLastError();
}

size_t fb_scratch_bytes(int S, int N, int T, int L) {
  const int C = (T + L - 1) / L;
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  size_t b = 0;
  b += al((size_t)S * C * mat_floats(N) * sizeof(float));  // P
  b += al((size_t)S * C * mat_floats(N) * sizeof(float));  // P^T
  b += al((size_t)S * C * sizeof(double));                 // Plog
  b += al((size_t)S * C * N * sizeof(float));              // fwd
  b += al((size_t)S * C * sizeof(float));                  // lam
  b += al((size_t)S * C * N * sizeof(float));              // bwd
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
  a.P = reinterpret_cast<float*>(take(S * C * mat_floats((int)N) * sizeof(float)));
  a.PT = reinterpret_cast<float*>(take(S * C * mat_floats((int)N) * sizeof(float)));
  a.Plog = reinterpret_cast<double*>(take(S * C * sizeof(double)));
  a.fwd = reinterpret_cast<float*>(take(S * C * N * sizeof(float)));
  a.lam = reinterpret_cast<float*>(take(S * C * sizeof(float)));
  a.bwd = reinterpret_cast<float*>(take(S * C * N * sizeof(float)));
}

cudaError_t launch_fb(const FBArgs& a, cudaStream_t st, int* launches) {
  if (launches) *launches += 3;
  switch (pad8(a.N)) {
    case 8: return launch_np<8>(a, st);
    case 16: return launch_np<16>(a, st);
    case 24: return launch_np<24>(a, st);
    case 32: return launch_np<32>(a, st);
    case 40: return launch_np<40>(a, st);
    case 48: return launch_np<48>(a, st);
    case 56: return launch_np<56>(a, st);
    case 64: return launch_np<64>(a, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace nfhmm
