// Forward-backward for the q(D^(s)) step of Section 3.2, in two forms: the
// scan, parallel in time (below), for a few long chains; and the sequential
// form (section 4 further down: one warp per chain and direction, frame by
// frame) for batches of many chains.
//
// With emissions e_t = exp(phi_t - max_n phi_t) and G_t = A diag(e_t), the
// forward row vector obeys a_t = a_{t-1} G_t (a_0 = pi diag(e_0)) and the
// backward column vector b_{t-1} = G_t b_t (b_{T-1} = 1).  Frames are cut
// into C chunks of L; chunk c covers frames t0..t1-1 and has the transfer
// matrix P_c = G_t0 ... G_{t1-1} (for c = 0 the first factor is diag(e_0)),
// so that a_{t1-1} = a_{t0-1} P_c (a_{L-1} = pi P_0) and b_{t0-1} = P_c b_{t1-1}.
// The scan, in three launches (five with groups of chunks, section 2'):
//   1. products: P_c of every chunk on the tensor cores.  Row i of P_c is
//      the forward recursion started from state i, so each row evolves on
//      its own: a 128-row tile holds the rows of floor(128/NP) chunks, one
//      TMEM lane per row, and every frame is one split-TF32 tcgen05.mma of
//      the tile by A followed by a thread-local epilogue (emission, per-row
//      rescaling, split back into the shared-memory operand).
//   2. scan:     forward and backward boundary vectors across chunks, one
//                warp per (source, direction), serial over C with the next
//                chunk matrices prefetched by cp.async; and log Z;
//   3. replay:   inside each chunk a forward warp and a backward warp run
//                concurrently from the chunk's boundary vectors; then
//                d-hat_t = a_t b_t / sum_n a_tn b_tn.
// In the serial loops a vector is rescaled by the sum computed one step
// earlier, so the warp reduction of a step overlaps the next step's
// arithmetic.  Scale factors are kept as exact (mantissa, exponent) products
// or in memory and turned into logs in double after the loops, so no
// double-precision work sits on a serial path.
// States are padded to NP = 8*ceil(N/8) with zero rows/columns in A, zero
// emissions and zero initial probability, so padded states never carry mass;
// every kernel is instantiated per NP and its loops unroll fully.
// Limits: chunk length 1 <= L <= FB_MAX_L, states N <= FB_MAX_N.
#include <float.h>
#include <limits.h>
#include <math.h>

#include "nfhmm_device.cuh"
#include "nfhmm_kernels.h"
#include "tc_ptx.cuh"

namespace nfhmm {

namespace {
constexpr int FB_MAX_N = 64;
constexpr int FB_MAX_L = 128;
// scan: prefetch depth (a step waits on a copy issued RING - 1 steps
// earlier), as deep as the shared memory allows
template <int NP>
struct ScanRing {
  static constexpr int R = NP <= 48 ? 16 : 8;
};
// the group replay (a group's few chunks per warp, up to 2 x S x groups
// one-warp blocks launched beside a contraction that holds most SMs) keeps a
// shallow ring, so that its blocks fit many to an SM
template <int NP>
struct ScanRingGroupReplay {
  static constexpr int R = 4;
};
constexpr int R_CHUNKS_MAX = 4;     // replay: chunks per block (2 warps each)
constexpr size_t SMEM_OPTIN = 227 * 1024;

__host__ __device__ constexpr int pad8(int n) { return (n + 7) & ~7; }

// Factor that brings a vector with sum (or maximum) x > 0 back towards 1:
// 1/x, or the exact power of two 2^100 when 1/x could overflow (x tiny or
// subnormal); 1 for x == 0 (an all-zero vector stays zero).
constexpr float BOOST = 0x1p100f;
__device__ __forceinline__ float renorm_factor(float x) {
  if (x >= 1e-30f) return 1.f / x;
  return x > 0.f ? BOOST : 1.f;
}
// The factor the vector was divided by: x, or 2^-100 after a boost.
__device__ __forceinline__ float removed_scale(float x) {
  if (x >= 1e-30f) return x;
  return x > 0.f ? 0x1p-100f : 1.f;
}

// Running product of positive scale factors as mantissa in [0.5, 1) and a
// power of two: exact apart from one rounding per factor.
struct ScaleAcc {
  float m = 1.f;
  int e = 0;
  __device__ __forceinline__ void mul(float s) {
    int ex;
    m = frexpf(m * s, &ex);
    e += ex;
  }
};

// 4-byte asynchronous copy (cp.async.ca): many in flight per thread, so a
// scattered gather into shared memory pays the global latency once
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}
// The row with the largest scale among n (mantissa m in [0.5, 1), or 0 for a
// row that vanished, and binary exponent e), or -1 if every row vanished.  A
// row's factor relative to it is then ldexpf(m / m_max, e - e_max), one
// rounding, and no double-precision work per row.
__device__ __forceinline__ int scale_argmax(const float* m, const int* e, int n) {
  int best = -1;
  float bk = -INFINITY;
  for (int i = 0; i < n; ++i) {
    if (m[i] > 0.f) {
      const float k = (float)e[i] + log2f(m[i]);
      if (k > bk) {
        bk = k;
        best = i;
      }
    }
  }
  return best;
}
constexpr double LN2 = 0.69314718055994530942;

struct ChunkInfo {
  int t0, len, chain;
  bool first;
};
// frames of global chunk c (null chain tables: one chain over all frames)
__device__ __forceinline__ ChunkInfo chunk_info(const FBArgs& a, int c) {
  ChunkInfo ci;
  const int j = a.chunk_chain ? a.chunk_chain[c] : 0;
  const int lc = c - (a.chain_c0 ? a.chain_c0[j] : 0);
  const int ct0 = a.chain_t0 ? a.chain_t0[j] : 0;
  const int clen = a.chain_len ? a.chain_len[j] : a.T;
  ci.chain = j;
  ci.first = lc == 0;
  ci.t0 = ct0 + lc * a.L;
  ci.len = min(a.L, clen - lc * a.L);
  return ci;
}
}  // namespace

int fb_max_states() { return FB_MAX_N; }

int fb_default_chunk(int N, int T) {
  // products and replay cost ~L serial frame steps, the two-level scan
  // ~2 sqrt(T/(2L)) chunk steps: chunks of ~0.3 sqrt(T) frames (8..64)
  // balance them (measured optimum 16 at T = 3000).
  int L = (int)lround(0.3 * sqrt((double)T));
  if (L < 8) L = 8;
  if (L > 64) L = 64;
  if (L > T) L = T;
  (void)N;
  return L;
}

static inline size_t mat_floats(int N) { return (size_t)pad8(N) * pad8(N); }

// ------------------------------------------------- 1. chain products (tensor cores)
// One 128-row tile of product rows advanced through a run of factors, one
// split-TF32 tcgen05.mma of the tile per factor.  Row i of a product of
// factors F_1 ... F_n is the forward recursion started from basis state i, so
// every row evolves on its own (one TMEM lane per row):
//   CHAIN_CHUNK: the rows of floor(128/NP) chunks; the factor of frame t is
//                G_t = A diag(e_t): B operand A (fixed), the emissions applied
//                to the product rows after each step;
//   CHAIN_GROUP: the rows of one group of chunks; the factors are its chunk
//                matrices, whose split operand images the chunk pass wrote,
//                brought in by bulk copies a few steps ahead.
// The B operand holds the factor's tf32 hi and lo parts stacked along N
// (rows [0, NOUT) and [NOUT, 2 NOUT) of each swizzle atom), so one MMA of
// N = 2 NOUT gives rows_hi*B_hi and rows_hi*B_lo, and a second (N = NOUT)
// adds rows_lo*B_hi to the cross terms: two MMAs per K step instead of three
// (the issue of tcgen05.mma by one thread, not the tensor core, bounds a
// step of these small tiles).
// Eight warps: warp w reads TMEM lanes 32(w%4).. (one row per thread) and
// half w/4 of the columns; the two halves of a row exchange their maxima
// through shared memory (a 64-thread named barrier).  Rows are rescaled by
// powers of two (exact), the removed exponents summed per row; at the end
// the rows of a chunk (group) are brought to the exponent of its largest row.
enum { CHAIN_CHUNK = 0, CHAIN_GROUP = 1 };
template <int NP>
struct ChainCfg {
  static constexpr int RCH = 128 / NP;              // chunks per tile (chunk pass)
  static constexpr int NOUT = (NP + 15) & ~15;      // MMA N (multiple of 16)
  static constexpr int HC = NOUT / 2;               // columns per epilogue half (multiple of 8)
  static constexpr int KSTEPS = NP / 8;             // tf32 MMA K = 8
  static constexpr int KATOMS = (NP + 31) / 32;     // 128-byte swizzle atoms along K
  static constexpr int ROWS_BYTES = KATOMS * 128 * 128;
  static constexpr int BATOM = 2 * NOUT * 128;      // one swizzle atom of B: hi rows, lo rows
  static constexpr int IMG_BYTES = KATOMS * BATOM;  // the stacked B operand of one factor
  static constexpr int RING = 4;                    // group pass: chunk images in flight
  static constexpr int TMEM_COLS = 2 * NOUT <= 32 ? 32 : 2 * NOUT <= 64 ? 64 : 128;
  // chunk pass: A staged with rows LDA floats apart, LDA / 4 odd, so that
  // 16-byte reads of 8 consecutive rows fall in distinct bank groups; NOUT
  // floats of slack after the last row for a thread's masked columns
  static constexpr int LDA = ((NP + 3) & ~3) + ((((NP + 3) & ~3) / 4) % 2 == 0 ? 4 : 0);
  static constexpr int A_FLOATS = NP * LDA + NOUT;
};
struct ChainMisc {
  double msum[16];       // chunk pass: summed frame maxima per chunk; group pass: [0] = chunk logs
  float pmax[2][128];    // row maxima of the two column halves
  int best[16];          // exponent of the largest row per chunk
  int clen[16];          // chunk pass: frames of each chunk of the tile
  uint64_t mma_bar;
  uint64_t full[ChainCfg<8>::RING];
  uint32_t tslot;
};

// byte offset of element (row r, k) in a K-major tile of 128-byte rows with
// 128-byte swizzle: 8-row groups 1024 bytes apart, 16-byte chunks XOR row%8
__device__ __forceinline__ uint32_t sw128_off(int r, int k, int atom_bytes) {
  const int atom = k >> 5, kk = k & 31;
  return atom * atom_bytes + (r >> 3) * 1024 + (r & 7) * 128 + ((((kk >> 2) ^ (r & 7))) << 4) +
         ((kk & 3) << 2);
}
__device__ __forceinline__ void named_bar(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}
__device__ __forceinline__ void tmem_ld8_nw(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7])
      : "r"(taddr));
}
// hi + lo += x, with hi + x formed exactly (Knuth's two-sum) and its rounding
// error carried in lo
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float x) {
  const float s = hi + x;
  const float bp = s - hi;
  const float err = (hi - (s - bp)) + (x - bp);
  hi = s;
  lo += err;
}
// exact power of two 2^k for -126 <= k <= 127
__device__ __forceinline__ float pow2f(int k) { return __int_as_float((127 + k) << 23); }

template <int NP, int MODE>
__global__ void __launch_bounds__(256, MODE == CHAIN_CHUNK ? 2 : 1) k_fb_chain(FBArgs a) {
  using namespace tc;
  using Cfg = ChainCfg<NP>;
  constexpr int NOUT = Cfg::NOUT, HC = Cfg::HC, RING = Cfg::RING;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint8_t* rows_hi = smem;
  uint8_t* rows_lo = rows_hi + Cfg::ROWS_BYTES;
  uint8_t* bbuf = rows_lo + Cfg::ROWS_BYTES;   // chunk pass: A split; group pass: image ring
  constexpr int BBUF = MODE == CHAIN_CHUNK ? Cfg::IMG_BYTES : RING * Cfg::IMG_BYTES;
  // chunk pass: RCH x L x NP emissions, RCH x L frame maxima, A (N x N)
  float* e = reinterpret_cast<float*>(bbuf + BBUF);
  const int ne = MODE == CHAIN_CHUNK ? Cfg::RCH * a.L * NP : 0;
  float* rmax = e + ne;
  float* As = rmax + (MODE == CHAIN_CHUNK ? ((Cfg::RCH * a.L + 3) & ~3) : 0);
  const int na = MODE == CHAIN_CHUNK ? Cfg::A_FLOATS : 0;
  ChainMisc* ms = reinterpret_cast<ChainMisc*>(As + na);

  const int N = a.N, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int quarter = warp & 3, half = warp >> 2;
  const int r = quarter * 32 + lane;           // tile row = TMEM lane
  const int j0 = half * HC;                    // first column of this thread
  const int s = blockIdx.y;
  const size_t cb = (size_t)s * a.C;

  // rows of this thread: chunk pass (chunk q of the tile, state i); group pass (state i)
  int q = 0, i = r, c = 0, c0 = 0, nst = 0;
  bool live = false, first = false;
  int len = 0, cbase = 0;
  if (MODE == CHAIN_CHUNK) {
    cbase = blockIdx.x * Cfg::RCH;
    q = r / NP;
    i = r - q * NP;
    c = cbase + q;
    const bool inchunk = q < Cfg::RCH && c < a.C;
    ChunkInfo ci = inchunk ? chunk_info(a, c) : ChunkInfo{0, 0, 0, false};
    live = inchunk && i < N;
    len = live ? ci.len : 0;
    first = ci.first;
    nst = a.L - 1;
  } else {
    const int g = blockIdx.x;
    c0 = a.grp_c0 ? a.grp_c0[g] : g * a.G;
    const int c1 = a.grp_c0 ? a.grp_c0[g + 1] : min((g + 1) * a.G, a.C);
    live = i < N;
    nst = c1 - c0 - 1;
  }

  if (tid == 0) {
    mbar_init(&ms->mma_bar, 1);
    if (MODE == CHAIN_GROUP)
      for (int u = 0; u < RING; ++u) mbar_init(&ms->full[u], 1);
    fence_barrier_init();
  }
  if (tid < 16) ms->best[tid] = INT_MIN;
  if (warp == 0) {
    tmem_alloc(&ms->tslot, Cfg::TMEM_COLS);
    tmem_relinquish();
  }
  const float* Ag = a.A + (size_t)s * N * N;
  if (MODE == CHAIN_CHUNK) {
    // A by asynchronous gathers: before the wait for the emissions' writer
    // when A is the caller's stable copy, else after it
    if (!a.inputs_stable) griddep_wait();
    for (int u = tid; u < N * N; u += 256) cp_async4(As + (u / N) * Cfg::LDA + u % N, Ag + u);
    cp_async_commit();
    if (tid < Cfg::RCH) ms->clen[tid] = cbase + tid < a.C ? chunk_info(a, cbase + tid).len : 0;
    cp_async_wait<0>();
    __syncthreads();
    // B operand: B[j][k] = A[k][j] (zero outside N x N), split into tf32 hi
    // (rows j) and lo (rows NOUT + j) of each swizzle atom; only the K < NP
    // columns the MMAs read
    for (int idx = tid; idx < NOUT * NP; idx += 256) {
      const int j = idx / NP, k = idx - j * NP;
      const float v = (j < N && k < N) ? As[k * Cfg::LDA + j] : 0.f;
      const float h = tf32_hi(v);
      *reinterpret_cast<float*>(bbuf + sw128_off(j, k, Cfg::BATOM)) = h;
      *reinterpret_cast<float*>(bbuf + sw128_off(j + NOUT, k, Cfg::BATOM)) = tf32_hi(v - h);
    }
    // the emissions, once the pass that wrote them (launched before this one
    // on the stream, as a programmatic dependency) has finished
    griddep_wait();
    for (int qq = 0; qq < Cfg::RCH; ++qq) {
      const int cc = cbase + qq;
      if (cc >= a.C) break;
      const ChunkInfo ci = chunk_info(a, cc);
      const float* src = a.phi + ((size_t)s * a.T + ci.t0) * N;
      float* eq = e + qq * a.L * NP;
      for (int u = tid; u < ci.len * N; u += 256) {
        const int f = u / N, n = u - f * N;
        cp_async4(eq + f * NP + n, src + u);
      }
    }
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    // e_t = exp(phi_t - max phi_t) for every frame of the tile: four
    // threads per frame (a quarter of the states each), the maxima kept per
    // frame and summed per chunk in double by one warp (fixed order)
    constexpr int QS = NP / 4;   // states per thread (NP is a multiple of 8)
    for (int base = warp * 8; base < Cfg::RCH * a.L; base += 64) {   // warp-uniform trips
      const int rho = base + (lane >> 2);
      const int qq = rho / a.L, f = rho - qq * a.L;
      // uniform across the row's 4 threads; every lane takes part in the shuffles
      const bool ok_row = rho < Cfg::RCH * a.L && f < ms->clen[qq];
      float* row = e + (ok_row ? rho : 0) * NP + (tid & 3) * QS;
      const int n0 = (tid & 3) * QS;
      float x[QS];
      float m = -INFINITY;
#pragma unroll
      for (int u = 0; u < QS; ++u) {
        x[u] = (ok_row && n0 + u < N) ? row[u] : -INFINITY;
        m = fmaxf(m, x[u]);
      }
      m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 1));
      m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 2));
      if (ok_row) {
#pragma unroll
        for (int u = 0; u < QS; ++u) row[u] = n0 + u < N ? expf(x[u] - m) : 0.f;
        if ((tid & 3) == 0) rmax[rho] = m;
      }
    }
    __syncthreads();
    for (int qq = warp; qq < Cfg::RCH; qq += 8) {
      // an unevaluated float pair (hi + lo, error-free sums): FP64 arithmetic
      // is a small fraction of FP32's rate on this GPU, and this sits on the
      // pass's critical path
      float hi = 0.f, lo = 0.f;
      for (int f = lane; f < ms->clen[qq]; f += 32) two_sum_acc(hi, lo, rmax[qq * a.L + f]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
        const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
        two_sum_acc(hi, lo, h2);
        lo += l2;
      }
      if (lane == 0) ms->msum[qq] = (double)hi + (double)lo;
    }
  } else {
    griddep_wait();    // the chunk pass's matrices, images and scales
    __syncthreads();   // barriers initialised
    if (tid == 0) {
      for (int u = 0; u < RING && u < nst; ++u) {
        mbar_expect_tx(&ms->full[u], Cfg::IMG_BYTES);
        bulk_g2s(bbuf + u * Cfg::IMG_BYTES, a.Pimg + (cb + c0 + 1 + u) * Cfg::IMG_BYTES,
                 Cfg::IMG_BYTES, &ms->full[u]);
      }
    }
    if (warp == 7) {   // the group's scale starts as the sum of its chunks' scales
      double lg = 0.0;
      for (int cc = c0 + lane; cc <= c0 + nst; cc += 32) lg += a.Plog[cb + cc];
      lg = warp_sum_d(lg);
      if (lane == 0) ms->msum[0] = lg;
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = ms->tslot;

  const float* eq = e + (MODE == CHAIN_CHUNK && q < Cfg::RCH ? q : 0) * a.L * NP;
  float cur[HC];
  int ex_row = 0;          // the row's true value = stored value * 2^ex_row
  bool zero_row = false;   // once zero, a row stays zero
  unsigned bad = 0;
  if (MODE == CHAIN_CHUNK) {
    // the chunk's first factor: row i of A diag(e_t0), or e_t0 on state i
    // when the chunk opens its job; row i of A by 16-byte reads
    const float* Ai = As + (live ? i : 0) * Cfg::LDA + j0;
#pragma unroll
    for (int jj = 0; jj < HC; jj += 4) {
      const float4 a4 = *reinterpret_cast<const float4*>(Ai + jj);
      const float av[4] = {a4.x, a4.y, a4.z, a4.w};
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int j = j0 + jj + u;
        float v = 0.f;
        if (live && j < N) v = first ? (j == i ? eq[j] : 0.f) : av[u] * eq[j];
        cur[jj + u] = v;
      }
    }
  } else {
    const float* Pr = a.P + (cb + c0) * NP * NP + (size_t)i * NP;
#pragma unroll
    for (int jj = 0; jj < HC; ++jj) {
      const int j = j0 + jj;
      cur[jj] = (live && j < NP) ? Pr[j] : 0.f;
    }
  }
  // rescale the row by a power of two that brings its maximum into [0.5, 1)
  // and write this thread's columns, split into tf32 hi/lo, into the
  // swizzled operand tile
  auto normalise_and_store = [&]() {
    float m4[4] = {0.f, 0.f, 0.f, 0.f};   // four independent chains
#pragma unroll
    for (int jj = 0; jj < HC; ++jj) m4[jj & 3] = fmaxf(m4[jj & 3], cur[jj]);
    float m = fmaxf(fmaxf(m4[0], m4[1]), fmaxf(m4[2], m4[3]));
    ms->pmax[half][r] = m;
    named_bar(1 + quarter, 64);
    m = fmaxf(m, ms->pmax[half ^ 1][r]);
    if (live) {
      // an all-zero row is legitimate (state i cannot start this chunk)
      if (!isfinite(m)) {
        bad = 1;
        m = 0.f;
      }
      if (m == 0.f) {
        zero_row = true;
      } else {
        int ex;
        if (m >= 0x1p-126f)
          ex = ((__float_as_int(m) >> 23) & 0xff) - 126;   // m = f 2^ex, f in [0.5, 1)
        else
          frexpf(m, &ex);
        const int k = -ex > 126 ? 126 : -ex;
        const float g = pow2f(k);
#pragma unroll
        for (int jj = 0; jj < HC; ++jj) cur[jj] *= g;
        ex_row -= k;
      }
    }
#pragma unroll
    for (int cc = 0; cc < HC / 4; ++cc) {
      if (j0 + 4 * cc < NP) {
        float h[4], l[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          h[u] = tf32_hi(cur[4 * cc + u]);
          l[u] = tf32_hi(cur[4 * cc + u] - h[u]);
        }
        const uint32_t off = sw128_off(r, j0 + 4 * cc, 128 * 128);
        *reinterpret_cast<float4*>(rows_hi + off) = make_float4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<float4*>(rows_lo + off) = make_float4(l[0], l[1], l[2], l[3]);
      }
    }
  };
  normalise_and_store();

  constexpr uint32_t ID2 = idesc<KIND_TF32X3>(128, 2 * NOUT);
  constexpr uint32_t ID1 = idesc<KIND_TF32X3>(128, NOUT);
  const uint32_t rh = smem_u32(rows_hi), rl = smem_u32(rows_lo);
  const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)j0;
  bool ok = true;
  int issued = MODE == CHAIN_GROUP ? min(RING, nst) : 0;   // group pass: images requested
  int consumed = 0;                                          // and waited for
  for (int f = 1; f <= nst; ++f) {
    bool okf = ok;
    uint32_t bh = smem_u32(bbuf);
    if (MODE == CHAIN_GROUP) {
      const int slot = (f - 1) % RING;
      bh = smem_u32(bbuf + slot * Cfg::IMG_BYTES);
      if (tid == 0) {
        if (!mbar_wait(&ms->full[slot], ((f - 1) / RING) & 1)) {
          okf = false;
          atomicOr(a.err, ERR_TIMEOUT);
        } else {
          consumed = f;
        }
      }
    }
    fence_proxy_async_smem();   // the operand rows written above, to the tensor core
    tc_fence_before();
    // every row written; and the decision to stop is the same in every thread
    if (__syncthreads_or(!okf)) {
      ok = false;
      break;
    }
    if (tid == 0) {
      tc_fence_after();
#pragma unroll
      for (int kk = 0; kk < Cfg::KSTEPS; ++kk) {
        const uint32_t ao = (kk >> 2) * (128 * 128) + (kk & 3) * 32;
        const uint32_t bo = (kk >> 2) * Cfg::BATOM + (kk & 3) * 32;
        // [main | cross] (+)= rows_hi [B_hi | B_lo];  cross += rows_lo B_hi
        mma<KIND_TF32X3>(tmem, sdesc(rh + ao), sdesc(bh + bo), ID2, kk > 0 ? 1u : 0u);
        mma<KIND_TF32X3>(tmem + NOUT, sdesc(rl + ao), sdesc(bh + bo), ID1, 1u);
      }
      mma_commit(&ms->mma_bar);
    }
    const bool done = mbar_wait(&ms->mma_bar, (f - 1) & 1);
    if (!done) {
      ok = false;   // the next step's barrier stops every thread
      if (lane == 0) atomicOr(a.err, ERR_TIMEOUT);
    }
    tc_fence_after();
    if (MODE == CHAIN_GROUP && tid == 0 && done && f + RING <= nst) {
      // the step's MMAs have completed: its slot takes the image RING steps ahead
      const int slot = (f - 1) % RING;
      mbar_expect_tx(&ms->full[slot], Cfg::IMG_BYTES);
      bulk_g2s(bbuf + slot * Cfg::IMG_BYTES, a.Pimg + (cb + c0 + f + RING) * Cfg::IMG_BYTES,
               Cfg::IMG_BYTES, &ms->full[slot]);
      issued = f + RING;
    }
    if (done) {
      // 8 columns of both accumulators at a time (bounded register use)
#pragma unroll
      for (int cc = 0; cc < HC / 8; ++cc) {
        uint32_t yr[8], xr[8];
        tmem_ld8_nw(taddr + 8 * cc, yr);
        tmem_ld8_nw(taddr + NOUT + 8 * cc, xr);
        tmem_wait_ld();
        if (MODE == CHAIN_CHUNK) {
          if (live && f < len) {
            const float* ef = eq + f * NP + j0 + 8 * cc;
#pragma unroll
            for (int h4 = 0; h4 < 8; h4 += 4) {
              const int jj = 8 * cc + h4;
              if (j0 + jj < NP) {
                const float4 e4 = *reinterpret_cast<const float4*>(ef + h4);
                const float ev[4] = {e4.x, e4.y, e4.z, e4.w};
#pragma unroll
                for (int u = 0; u < 4; ++u)
                  cur[jj + u] = (__uint_as_float(yr[h4 + u]) + __uint_as_float(xr[h4 + u])) * ev[u];
              } else {
                cur[jj] = cur[jj + 1] = cur[jj + 2] = cur[jj + 3] = 0.f;
              }
            }
          }
        } else if (live) {
#pragma unroll
          for (int u = 0; u < 8; ++u)
            cur[8 * cc + u] =
                j0 + 8 * cc + u < NP ? __uint_as_float(yr[u]) + __uint_as_float(xr[u]) : 0.f;
        }
      }
    }
    normalise_and_store();
  }
  griddep_launch_dependents();   // the next pass may start its launch and setup
  if (MODE == CHAIN_GROUP && tid == 0) {
    // every copy issued must have landed before the block may exit
    for (int f = consumed + 1; f <= issued; ++f)
      if (!mbar_wait(&ms->full[(f - 1) % RING], ((f - 1) / RING) & 1)) atomicOr(a.err, ERR_TIMEOUT);
  }
  if (bad) atomicOr(a.err, ERR_FB_ZERO);

  // common scale: the rows of a chunk (group) relative to its largest row
  if (half == 0 && live && !zero_row) atomicMax(&ms->best[MODE == CHAIN_CHUNK ? q : 0], ex_row);
  __syncthreads();
  const bool owner = MODE == CHAIN_CHUNK ? (q < Cfg::RCH && c < a.C && i < NP) : i < NP;
  if (owner) {
    // best == INT_MIN only if every row vanished (flagged by the scan)
    const int best = ms->best[MODE == CHAIN_CHUNK ? q : 0];
    const bool nz = live && !zero_row && best != INT_MIN;
    const float g = nz ? ldexpf(1.f, ex_row - best) : 0.f;
    const size_t base = (MODE == CHAIN_CHUNK ? cb + c : ((size_t)s * a.NG + blockIdx.x)) * NP * NP;
    float* Pg = (MODE == CHAIN_CHUNK ? a.P : a.Q) + base;
    float* PTg = (MODE == CHAIN_CHUNK ? a.PT : a.QT) + base;
    float v[HC];
#pragma unroll
    for (int jj = 0; jj < HC; ++jj) v[jj] = nz ? cur[jj] * g : 0.f;
#pragma unroll
    for (int jj = 0; jj < HC; jj += 4)
      if (j0 + jj < NP)
        *reinterpret_cast<float4*>(Pg + (size_t)i * NP + j0 + jj) =
            make_float4(v[jj], v[jj + 1], v[jj + 2], v[jj + 3]);
#pragma unroll
    for (int jj = 0; jj < HC; ++jj)
      if (j0 + jj < NP) PTg[(size_t)(j0 + jj) * NP + i] = v[jj];
    if (MODE == CHAIN_CHUNK && a.Pimg) {
      // the chunk matrix as the group pass's B operand: B[j][k = i] = P[i][j]
      uint8_t* img = a.Pimg + (cb + c) * Cfg::IMG_BYTES;
#pragma unroll
      for (int jj = 0; jj < HC; ++jj) {
        const float h = tf32_hi(v[jj]);
        *reinterpret_cast<float*>(img + sw128_off(j0 + jj, i, Cfg::BATOM)) = h;
        *reinterpret_cast<float*>(img + sw128_off(NOUT + j0 + jj, i, Cfg::BATOM)) =
            tf32_hi(v[jj] - h);
      }
    }
    if (i == 0 && half == 0) {
      const double lb = best != INT_MIN ? (double)best * LN2 : 0.0;
      if (MODE == CHAIN_CHUNK)
        a.Plog[cb + c] = ms->msum[q] + lb;
      else
        a.Qlog[(size_t)s * a.NG + blockIdx.x] = ms->msum[0] + lb;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, Cfg::TMEM_COLS);
  }
}

// --------------------------------------------- 1'. products on CUDA cores
// The same chunk matrices with FP32 FMAs: one thread per row of P_c (chunk
// q, basis state i), 128 threads holding the rows of floor(128/NP) chunks
// as in the tensor-core form.  A step is the row times A (read from shared
// memory, the same address in every lane: a broadcast) times the frame's
// emissions, then a rescale by the row's maximum: all thread-local, no
// barrier inside the frame loop.
template <int NP>
__global__ void __launch_bounds__(128) k_fb_products_simt(FBArgs a) {
  constexpr int RCH = 128 / NP;
  constexpr int XS = NP + 1;   // padded row stride: rows of neighbouring threads in different banks
  extern __shared__ double smd[];
  double* rhod = smd;                                      // 128
  double* msum = smd + 128;                                // RCH (<= 16)
  float* As = reinterpret_cast<float*>(smd + 128 + 16);    // NP x NP, A[k][j]
  float* xs = As + NP * NP;                                // 128 x XS current rows
  float* e = xs + 128 * XS + 3;                            // RCH x L x NP (16-byte aligned)
  e = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(e) + 15) & ~(uintptr_t)15);
  const int N = a.N, L = a.L, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int s = blockIdx.y;
  const int cbase = blockIdx.x * RCH;
  const float* Ag = a.A + (size_t)s * N * N;
  for (int idx = tid; idx < NP * NP; idx += 128) {
    const int k = idx / NP, j = idx - k * NP;
    if (k < N && j < N) cp_async4(As + idx, Ag + k * N + j);
    else As[idx] = 0.f;
  }
  for (int q = 0; q < RCH; ++q) {
    const int c = cbase + q;
    if (c >= a.C) break;
    const ChunkInfo ci = chunk_info(a, c);
    const float* src = a.phi + ((size_t)s * a.T + ci.t0) * N;
    float* eq = e + q * L * NP;
    for (int i = tid; i < ci.len * N; i += 128) {
      const int f = i / N, n = i - f * N;
      cp_async4(eq + f * NP + n, src + i);
    }
  }
  cp_async_commit();
  cp_async_wait<0>();
  __syncthreads();
  for (int q = 0; q < RCH; ++q) {
    const int c = cbase + q;
    if (c >= a.C) break;
    const int len = chunk_info(a, c).len;
    float* eq = e + q * L * NP;
    double ms = 0.0;
    for (int f = warp; f < len; f += 4) {
      float* row = eq + f * NP;
      const float x0 = lane < N ? row[lane] : -INFINITY;
      const float x1 = lane + 32 < N ? row[lane + 32] : -INFINITY;
      const float m = warp_max(fmaxf(x0, x1));
      __syncwarp();
      if (lane < NP) row[lane] = lane < N ? expf(x0 - m) : 0.f;
      if (lane + 32 < NP) row[lane + 32] = lane + 32 < N ? expf(x1 - m) : 0.f;
      ms += (double)m;
    }
    if (lane == 0) rhod[warp] = ms;
    __syncthreads();
    if (tid == 0) msum[q] = rhod[0] + rhod[1] + rhod[2] + rhod[3];
    __syncthreads();
  }
  const int q = tid / NP, i = tid - q * NP;
  const int c = cbase + q;
  const bool live = q < RCH && c < a.C && i < N;
  const ChunkInfo ci = (q < RCH && c < a.C) ? chunk_info(a, c) : ChunkInfo{0, 0, 0, false};
  const int len = live ? ci.len : 0;
  const float* eq = e + (q < RCH ? q : 0) * L * NP;
  float* xr = xs + tid * XS;   // this thread's row
  float y[NP];
  ScaleAcc sc;
  bool zero_row = false;
  unsigned bad = 0;
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    float v = 0.f;
    if (live && j < N) v = ci.first ? (j == i ? eq[j] : 0.f) : As[i * NP + j] * eq[j];
    y[j] = v;
  }
  // rescale y by its maximum into this thread's row in shared memory
  auto normalise_store = [&]() {
    float m = 0.f;
#pragma unroll
    for (int j = 0; j < NP; ++j) m = fmaxf(m, y[j]);
    if (!isfinite(m)) {
      bad = 1;
      m = 0.f;
    }
    if (m == 0.f) zero_row = true;
    const float g = renorm_factor(m);
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      y[j] *= g;
      xr[j] = y[j];
    }
    sc.mul(removed_scale(m));
  };
  if (live) normalise_store();
  for (int f = 1; f < len; ++f) {
#pragma unroll
    for (int j = 0; j < NP; ++j) y[j] = 0.f;
#pragma unroll 2
    for (int k = 0; k < NP; ++k) {
      const float xk = xr[k];
      const float* ak = As + k * NP;
#pragma unroll
      for (int j = 0; j < NP; j += 4) {
        const float4 a4 = *reinterpret_cast<const float4*>(ak + j);
        y[j] = fmaf(xk, a4.x, y[j]);
        y[j + 1] = fmaf(xk, a4.y, y[j + 1]);
        y[j + 2] = fmaf(xk, a4.z, y[j + 2]);
        y[j + 3] = fmaf(xk, a4.w, y[j + 3]);
      }
    }
    const float* ef = eq + f * NP;
#pragma unroll
    for (int j = 0; j < NP; j += 4) {
      const float4 e4 = *reinterpret_cast<const float4*>(ef + j);
      y[j] *= e4.x;
      y[j + 1] *= e4.y;
      y[j + 2] *= e4.z;
      y[j + 3] *= e4.w;
    }
    normalise_store();
  }
  if (bad) atomicOr(a.err, ERR_FB_ZERO);
  float* rm = reinterpret_cast<float*>(rhod);
  int* re = reinterpret_cast<int*>(rm + 128);
  rm[tid] = (live && !zero_row) ? sc.m : 0.f;
  re[tid] = sc.e;
  __syncthreads();
  if (q < RCH && c < a.C && i < NP) {
    // best < 0 only if every row of the chunk vanished (flagged by the scan)
    const int best = scale_argmax(rm + q * NP, re + q * NP, N);
    const float g = (live && best >= 0 && rm[tid] > 0.f)
                        ? ldexpf(rm[tid] / rm[q * NP + best], re[tid] - re[q * NP + best])
                        : 0.f;
    const size_t base = ((size_t)s * a.C + c) * NP * NP;
    float* Pg = a.P + base;
    float* PTg = a.PT + base;
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      const float v = live ? y[j] * g : 0.f;
      Pg[i * NP + j] = v;
      PTg[j * NP + i] = v;
    }
    if (i == 0)
      a.Plog[(size_t)s * a.C + c] =
          msum[q] + (best >= 0 ? (double)re[q * NP + best] * LN2 + log((double)rm[q * NP + best])
                               : 0.0);
  }
}

// ------------------------------------------------------------------- 2. scan
// One warp per (source, direction); lane j holds states j and j + 32.
// blockIdx.y == 0: forward boundaries fwd[c] = normalised a at the end of
// chunk c (c = 0..C-1) and log Z = sum_c (Plog_c + log lambda_c);
// y_j = sum_i v_i P[i][j] reads row j of P^T.
// blockIdx.y == 1: backward boundaries bwd[c] = normalised b at the end of
// chunk c (bwd[C-1] = 1); y_i = sum_j P[i][j] v_j reads row i of P.
// Matrices are staged with rows padded to NP + 4 floats (conflict-free
// float4 reads).  The vector is rescaled by the previous step's sum.
// MODE_CHAINS: one warp per (chain, direction) over the chain's units (the
// chunks, or the groups when called with the group arrays in place of the
// chunk arrays), as above.
// MODE_GROUP_REPLAY: one warp per (group, direction) over the group's chunks,
// started from the group-level boundary vectors (pi / ones at a chain's
// ends); writes the chunk boundary vectors only.
enum { MODE_CHAINS = 0, MODE_GROUP_REPLAY = 1 };
template <int NP, int MODE>
__global__ void __launch_bounds__(32) k_fb_scan(FBArgs a) {
  extern __shared__ float sm[];
  constexpr int RING = MODE == MODE_GROUP_REPLAY ? ScanRingGroupReplay<NP>::R : ScanRing<NP>::R;
  constexpr int LD = NP + 4;
  constexpr int NN = NP * LD;
  const int N = a.N, C = a.C;
  const bool fwd = blockIdx.y == 0;
  const int lane = threadIdx.x;
  griddep_wait();   // the matrices (and boundary vectors) of the previous pass
  if (MODE == MODE_GROUP_REPLAY) griddep_launch_dependents();
  float* ring = sm;                      // RING x NP x LD
  float* v = ring + RING * NN;           // 64
  int s, chain = 0, c0, c1;
  bool first = true, last = true;        // group replay: the group opens / closes its chain
  if (MODE == MODE_CHAINS) {
    s = blockIdx.x / a.nchains;
    chain = blockIdx.x - s * a.nchains;
    c0 = a.chain_c0 ? a.chain_c0[chain] : 0;
    c1 = a.chain_c0 ? a.chain_c0[chain + 1] : C;   // the chain's units [c0, c1)
  } else {
    s = blockIdx.x / a.NG;
    const int g = blockIdx.x - s * a.NG;
    c0 = a.grp_c0 ? a.grp_c0[g] : g * a.G;
    c1 = a.grp_c0 ? a.grp_c0[g + 1] : min((g + 1) * a.G, C);
    const int j = a.chunk_chain ? a.chunk_chain[c0] : 0;
    first = c0 == (a.chain_c0 ? a.chain_c0[j] : 0);
    last = c1 == (a.chain_c0 ? a.chain_c0[j + 1] : C);
    chain = g;   // for the start vectors below
  }
  const size_t base = (size_t)s * C;
  const float* src = fwd ? a.PT : a.P;
  const int nsteps = fwd ? c1 - c0 : c1 - c0 - 1;
  auto chunk_of = [&](int q) { return fwd ? c0 + q : c1 - 1 - q; };
  // this lane's 16-byte pieces of a matrix: source and padded destination offsets
  constexpr int CPL = (NP * NP / 4 + 31) / 32;   // 16-byte copies per lane per matrix
  int soff[CPL], doff[CPL];
#pragma unroll
  for (int m = 0; m < CPL; ++m) {
    const int i = (lane + 32 * m) * 4;
    soff[m] = i < NP * NP ? i : -1;
    doff[m] = (i / NP) * LD + (i % NP);
  }
  auto prefetch = [&](int q) {
    if (q < nsteps) {
      const float* g = src + (base + chunk_of(q)) * NP * NP;
      float* d = ring + (q % RING) * NN;
#pragma unroll
      for (int m = 0; m < CPL; ++m)
        if (soff[m] >= 0) cp_async16(d + doff[m], g + soff[m]);
    }
    cp_async_commit();
  };
#pragma unroll
  for (int q = 0; q < RING - 1; ++q) prefetch(q);

  const bool h0 = lane < N, h1 = lane + 32 < N;
  const int j0 = lane < NP ? lane : 0, j1 = lane + 32 < NP ? lane + 32 : 0;
  float r0 = 0.f, r1 = 0.f;
  if (fwd) {
    const float* st = (MODE == MODE_CHAINS || first)
                          ? a.pi + (size_t)s * N
                          : a.gfwd + ((size_t)s * a.NG + chain - 1) * N;
    if (h0) r0 = st[lane];
    if (h1) r1 = st[lane + 32];
  } else {
    if (MODE == MODE_CHAINS || last) {
      r0 = h0 ? 1.f : 0.f;
      r1 = h1 ? 1.f : 0.f;
    } else {
      const float* st = a.gbwd + ((size_t)s * a.NG + chain) * N;
      if (h0) r0 = st[lane];
      if (h1) r1 = st[lane + 32];
    }
    if (h0) a.bwd[(base + c1 - 1) * N + lane] = r0;
    if (h1) a.bwd[(base + c1 - 1) * N + lane + 32] = r1;
  }
  // u_prev: the previous step's output, not yet normalised; its sum (the
  // previous chunk's normaliser) is reduced while this step's products run.
  float u0 = r0, u1 = r1;
  auto emit = [&](int qq, float lam_q, float w0, float w1) {  // outputs of step qq
    const float il = renorm_factor(lam_q);
    const int c = chunk_of(qq);
    if (fwd) {
      if (h0) a.fwd[(base + c) * N + lane] = w0 * il;
      if (h1) a.fwd[(base + c) * N + lane + 32] = w1 * il;
      if (MODE == MODE_CHAINS && lane == 0) a.lam[base + c] = removed_scale(lam_q);
    } else {
      if (h0) a.bwd[(base + c - 1) * N + lane] = w0 * il;
      if (h1) a.bwd[(base + c - 1) * N + lane + 32] = w1 * il;
    }
  };
  // The step's serial chain runs u -> v (shared memory) -> products -> u; the
  // sum of u (this step's normaliser) is reduced beside the products, so no
  // branch stands between them (a vanishing or non-finite sum is flagged once
  // at the end), and the previous output is stored after the new one is formed.
  bool vanished = false;
  for (int q = 0; q < nsteps; ++q) {
    __syncwarp();   // every lane is past step q - 1's reads of v and of the slot refilled here
    v[lane] = u0;
    v[lane + 32] = u1;
    prefetch(q + RING - 1);
    cp_async_wait<RING - 1>();
    __syncwarp();
    float lam_prev = warp_sum(u0 + u1);
    const float* P = ring + (q % RING) * NN;
    float y0[4] = {0.f, 0.f, 0.f, 0.f}, y1[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int i = 0; i < NP; i += 4) {
      const float4 vv = *reinterpret_cast<const float4*>(&v[i]);
      const float4 p0 = *reinterpret_cast<const float4*>(&P[j0 * LD + i]);
      y0[0] = fmaf(vv.x, p0.x, y0[0]);
      y0[1] = fmaf(vv.y, p0.y, y0[1]);
      y0[2] = fmaf(vv.z, p0.z, y0[2]);
      y0[3] = fmaf(vv.w, p0.w, y0[3]);
      if (NP > 32) {
        const float4 p1 = *reinterpret_cast<const float4*>(&P[j1 * LD + i]);
        y1[0] = fmaf(vv.x, p1.x, y1[0]);
        y1[1] = fmaf(vv.y, p1.y, y1[1]);
        y1[2] = fmaf(vv.z, p1.z, y1[2]);
        y1[3] = fmaf(vv.w, p1.w, y1[3]);
      }
    }
    const bool bad_sum = q > 0 && !(lam_prev > 0.f && lam_prev <= FLT_MAX);
    vanished |= bad_sum;
    lam_prev = bad_sum ? 1.f : lam_prev;
    // the start vector (pi, or ones) enters unnormalised
    const float inv = q > 0 ? renorm_factor(lam_prev) : 1.f;
    const float w0 = u0, w1 = u1;
    u0 = h0 ? ((y0[0] + y0[1]) + (y0[2] + y0[3])) * inv : 0.f;
    u1 = h1 ? ((y1[0] + y1[1]) + (y1[2] + y1[3])) * inv : 0.f;
    if (q > 0) emit(q - 1, lam_prev, w0, w1);
  }
  if (vanished && lane == 0) atomicOr(a.err, ERR_FB_ZERO);
  if (MODE == MODE_CHAINS) griddep_launch_dependents();
  if (nsteps > 0) {
    float lam = warp_sum(u0 + u1);
    if (!(lam > 0.f) || !isfinite(lam)) {
      if (lane == 0) atomicOr(a.err, ERR_FB_ZERO);
      lam = 1.f;
    }
    emit(nsteps - 1, lam, u0, u1);
  }
  cp_async_wait<0>();
  if (MODE == MODE_CHAINS && fwd) {
    __syncwarp();
    __threadfence_block();
    double lg = 0.0;
    for (int c = c0 + lane; c < c1; c += 32) lg += a.Plog[base + c] + log((double)a.lam[base + c]);
    lg = warp_sum_d(lg);
    if (lane == 0) a.logZ[(size_t)s * a.nchains + chain] = lg;
  }
}

// ------------------------------------------------------ 2'. group products
// Q_g = P_c0 P_c0+1 ... P_c1-1 for each group of chunks, row by row: row i is
// the forward chain started from the basis vector e_i.  One block per group:
// warp w advances rows 2w and 2w+1 over the group's chunk matrices, staged
// once per step with cp.async and shared by all warps.  Each row is rescaled
// by the sum of its previous value, the removed factors kept per row; at the
// end the rows are brought to the common scale of the largest and written
// with the transpose and the group's log scale (plus its chunks' scales).
constexpr int GRING = 8;
template <int NP>
__global__ void __launch_bounds__(NP * 16) k_fb_group_products(FBArgs a) {
  constexpr int LD = NP + 4;
  constexpr int NN = NP * LD;
  constexpr int NT = NP * 16;                       // threads: NP/2 warps
  constexpr int CPT = (NP * NP / 4 + NT - 1) / NT;  // 16-byte copies per thread per matrix
  extern __shared__ float sm[];
  double* rl = reinterpret_cast<double*>(sm);       // NP row log scales
  float* ring = sm + 2 * NP;                        // GRING x NP x LD
  float* vbuf = ring + GRING * NN;                  // NP/2 warps x 2 rows x 64
  const int N = a.N, C = a.C;
  const int g = blockIdx.x, s = blockIdx.y;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int c0 = a.grp_c0 ? a.grp_c0[g] : g * a.G;
  const int c1 = a.grp_c0 ? a.grp_c0[g + 1] : min((g + 1) * a.G, C);
  const int nsteps = c1 - c0;
  const size_t cbase = (size_t)s * C;
  int soff[CPT], doff[CPT];
#pragma unroll
  for (int m = 0; m < CPT; ++m) {
    const int i = (tid + NT * m) * 4;
    soff[m] = i < NP * NP ? i : -1;
    doff[m] = (i / NP) * LD + (i % NP);
  }
  auto prefetch = [&](int q) {
    if (q < nsteps) {
      const float* gsrc = a.PT + (cbase + c0 + q) * NP * NP;
      float* d = ring + (q % GRING) * NN;
#pragma unroll
      for (int m = 0; m < CPT; ++m)
        if (soff[m] >= 0) cp_async16(d + doff[m], gsrc + soff[m]);
    }
    cp_async_commit();
  };
#pragma unroll
  for (int q = 0; q < GRING - 1; ++q) prefetch(q);

  const int ia = warp * 2, ib = ia + 1;
  const bool la = ia < N, lb = ib < N;
  const bool h0 = lane < N, h1 = lane + 32 < N;
  const int j0 = lane < NP ? lane : 0, j1 = lane + 32 < NP ? lane + 32 : 0;
  float ua0 = (la && lane == ia) ? 1.f : 0.f, ua1 = (la && lane + 32 == ia) ? 1.f : 0.f;
  float ub0 = (lb && lane == ib) ? 1.f : 0.f, ub1 = (lb && lane + 32 == ib) ? 1.f : 0.f;
  ScaleAcc sca, scb;
  float* va = vbuf + warp * 128;
  float* vb = va + 64;
  unsigned bad = 0;
  for (int q = 0; q < nsteps; ++q) {
    cp_async_wait<GRING - 2>();
    __syncthreads();              // matrix q landed; every warp is past step q - 1
    prefetch(q + GRING - 1);      // into the slot step q - 1 read
    va[lane] = ua0;
    va[lane + 32] = ua1;
    vb[lane] = ub0;
    vb[lane + 32] = ub1;
    __syncwarp();
    const float lama = warp_sum(ua0 + ua1), lamb = warp_sum(ub0 + ub1);
    if (q > 0) {
      if (!isfinite(lama) || !isfinite(lamb)) bad = 1;
      sca.mul(removed_scale(lama));
      scb.mul(removed_scale(lamb));
    }
    const float* P = ring + (q % GRING) * NN;
    float ya0[4] = {0.f, 0.f, 0.f, 0.f}, ya1[4] = {0.f, 0.f, 0.f, 0.f};
    float yb0[4] = {0.f, 0.f, 0.f, 0.f}, yb1[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int i = 0; i < NP; i += 4) {
      const float4 xa = *reinterpret_cast<const float4*>(&va[i]);
      const float4 xb = *reinterpret_cast<const float4*>(&vb[i]);
      const float4 p0 = *reinterpret_cast<const float4*>(&P[j0 * LD + i]);
      ya0[0] = fmaf(xa.x, p0.x, ya0[0]);
      ya0[1] = fmaf(xa.y, p0.y, ya0[1]);
      ya0[2] = fmaf(xa.z, p0.z, ya0[2]);
      ya0[3] = fmaf(xa.w, p0.w, ya0[3]);
      yb0[0] = fmaf(xb.x, p0.x, yb0[0]);
      yb0[1] = fmaf(xb.y, p0.y, yb0[1]);
      yb0[2] = fmaf(xb.z, p0.z, yb0[2]);
      yb0[3] = fmaf(xb.w, p0.w, yb0[3]);
      if (NP > 32) {
        const float4 p1 = *reinterpret_cast<const float4*>(&P[j1 * LD + i]);
        ya1[0] = fmaf(xa.x, p1.x, ya1[0]);
        ya1[1] = fmaf(xa.y, p1.y, ya1[1]);
        ya1[2] = fmaf(xa.z, p1.z, ya1[2]);
        ya1[3] = fmaf(xa.w, p1.w, ya1[3]);
        yb1[0] = fmaf(xb.x, p1.x, yb1[0]);
        yb1[1] = fmaf(xb.y, p1.y, yb1[1]);
        yb1[2] = fmaf(xb.z, p1.z, yb1[2]);
        yb1[3] = fmaf(xb.w, p1.w, yb1[3]);
      }
    }
    const float fa = q > 0 ? renorm_factor(lama) : 1.f;
    const float fb = q > 0 ? renorm_factor(lamb) : 1.f;
    ua0 = h0 ? ((ya0[0] + ya0[1]) + (ya0[2] + ya0[3])) * fa : 0.f;
    ua1 = h1 ? ((ya1[0] + ya1[1]) + (ya1[2] + ya1[3])) * fa : 0.f;
    ub0 = h0 ? ((yb0[0] + yb0[1]) + (yb0[2] + yb0[3])) * fb : 0.f;
    ub1 = h1 ? ((yb1[0] + yb1[1]) + (yb1[2] + yb1[3])) * fb : 0.f;
  }
  cp_async_wait<0>();
  // final normalisation of each row, then the common scale
  const float sa = warp_sum(ua0 + ua1), sb = warp_sum(ub0 + ub1);
  if (!isfinite(sa) || !isfinite(sb)) bad = 1;
  const float fa = renorm_factor(sa), fb = renorm_factor(sb);
  sca.mul(removed_scale(sa));
  scb.mul(removed_scale(sb));
  float* rm = reinterpret_cast<float*>(rl);
  int* re = reinterpret_cast<int*>(rm + NP);
  __shared__ int best_row;
  if (lane == 0) {
    rm[ia] = (la && sa > 0.f) ? sca.m : 0.f;
    re[ia] = sca.e;
    rm[ib] = (lb && sb > 0.f) ? scb.m : 0.f;
    re[ib] = scb.e;
  }
  __syncthreads();
  if (tid == 0) best_row = scale_argmax(rm, re, N);
  __syncthreads();
  const int best = best_row;
  const float ga = (best >= 0 && rm[ia] > 0.f)
                       ? ldexpf(rm[ia] / rm[best], re[ia] - re[best]) * fa : 0.f;
  const float gb = (best >= 0 && rm[ib] > 0.f)
                       ? ldexpf(rm[ib] / rm[best], re[ib] - re[best]) * fb : 0.f;
  const double rmax = best >= 0 ? (double)re[best] * LN2 + log((double)rm[best]) : -INFINITY;
  const size_t qb = ((size_t)s * a.NG + g) * NP * NP;
  if (lane < NP) {
    a.Q[qb + (size_t)ia * NP + lane] = ua0 * ga;
    a.Q[qb + (size_t)ib * NP + lane] = ub0 * gb;
    a.QT[qb + (size_t)lane * NP + ia] = ua0 * ga;
    a.QT[qb + (size_t)lane * NP + ib] = ub0 * gb;
  }
  if (lane + 32 < NP) {
    a.Q[qb + (size_t)ia * NP + lane + 32] = ua1 * ga;
    a.Q[qb + (size_t)ib * NP + lane + 32] = ub1 * gb;
    a.QT[qb + (size_t)(lane + 32) * NP + ia] = ua1 * ga;
    a.QT[qb + (size_t)(lane + 32) * NP + ib] = ub1 * gb;
  }
  if (warp == 0) {   // the group's scale: its chunks' scales (loaded in parallel) and rmax
    double lg = 0.0;
    for (int c = c0 + lane; c < c1; c += 32) lg += a.Plog[cbase + c];
    lg = warp_sum_d(lg);
    if (lane == 0) a.Qlog[(size_t)s * a.NG + g] = lg + (rmax > -INFINITY ? rmax : 0.0);
  }
  if (bad && lane == 0) atomicOr(a.err, ERR_FB_ZERO);
}

// ----------------------------------------------------------------- 3. replay
// Two warps per chunk: warp 2q runs the forward recursion of chunk q (A's
// columns j, j+32 in registers), warp 2q+1 the backward recursion (A's rows
// j, j+32 in registers), concurrently; then both combine a_t b_t into d-hat.
// Vectors are stored unnormalised and rescaled by the previous step's sum.
template <int NP>
__global__ void __launch_bounds__(R_CHUNKS_MAX * 64, NP <= 48 ? 2 : 1) k_fb_replay(FBArgs a) {
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
  const ChunkInfo ci = live ? chunk_info(a, c) : ChunkInfo{0, 0, 0, false};
  const int t0 = ci.t0;
  const int len = live ? ci.len : 0;
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
    // the chunk's two warps gather its phi rows (contiguous) with
    // asynchronous copies, all in flight together
    const float* src = a.phi + (size_t)s * a.T * N + (size_t)t0 * N;
    const int tot = len * N;
    for (int i = (int)threadIdx.x - q * 64; i < tot; i += 64) {
      const int f = i / N, n = i - f * N;
      cp_async4(e + f * NP + n, src + i);
    }
  }
  cp_async_commit();
  cp_async_wait<0>();
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
  griddep_wait();   // the boundary vectors of the scan (the setup above needs none)
  const size_t base = (size_t)s * a.C;
  if (live) {
    float* vec = is_fwd ? av : bv;
    float r0, r1;
    if (is_fwd) {
      if (ci.first) {
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
    const float inv = renorm_factor(warp_sum(r0 + r1));
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
      // the sum of the stored vector, used to rescale the next one
      const float sprev = warp_sum(r0 + r1);
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
      const float inv_prev = renorm_factor(sprev);
      r0 = y0 * inv_prev;
      r1 = y1 * inv_prev;
      if (lane < NP) vec[f * NP + lane] = r0;
      if (lane + 32 < NP) vec[f * NP + lane + 32] = r1;
    }
  }
  __syncthreads();
  // the sweep's next kernel (the weights, which waits for this one before it
  // reads d-hat) may start launching
  griddep_launch_dependents();
  // d-hat_t = a_t b_t / sum_n a_tn b_tn: the chunk's two warps take 16
  // frames at a time, four threads per frame (a quarter of the states each);
  // the stored vectors are only roughly normalised, so each is rescaled by
  // its sum first (the scales cancel in d-hat but keep the products in range)
  if (len > 0) {
    constexpr int QS = NP / 4;
    const int u = ((warp & 1) << 5) | lane;
    const int n0 = (u & 3) * QS;
    float* dh = a.dhat + ((size_t)s * a.T + t0) * N;
    unsigned bad = 0;
    for (int f0 = 0; f0 < len; f0 += 16) {   // uniform in both warps of the chunk
      const int f = f0 + (u >> 2);
      const bool ok = f < len;
      float av4[QS], bv4[QS];
      float sa = 0.f, sb = 0.f;
#pragma unroll
      for (int k = 0; k < QS; ++k) {
        const bool in = ok && n0 + k < N;
        av4[k] = in ? av[f * NP + n0 + k] : 0.f;
        bv4[k] = in ? bv[f * NP + n0 + k] : 0.f;
        sa += av4[k];
        sb += bv4[k];
      }
      sa += __shfl_xor_sync(0xffffffffu, sa, 1);
      sb += __shfl_xor_sync(0xffffffffu, sb, 1);
      sa += __shfl_xor_sync(0xffffffffu, sa, 2);
      sb += __shfl_xor_sync(0xffffffffu, sb, 2);
      const float fa = renorm_factor(sa), fb = renorm_factor(sb);
      float z = 0.f;
#pragma unroll
      for (int k = 0; k < QS; ++k) {
        av4[k] = (av4[k] * fa) * (bv4[k] * fb);
        z += av4[k];
      }
      z += __shfl_xor_sync(0xffffffffu, z, 1);
      z += __shfl_xor_sync(0xffffffffu, z, 2);
      if (ok) {
        if (!(z > 0.f) || !isfinite(z)) {
          bad = 1;
          z = 1.f;
        }
        const float iz = 1.f / z;
#pragma unroll
        for (int k = 0; k < QS; ++k)
          if (n0 + k < N) dh[(size_t)f * N + n0 + k] = av4[k] * iz;
      }
    }
    if (bad) atomicOr(a.err, ERR_FB_ZERO);
  }
}

// ------------------------------------------- 4. sequential form (many chains)
// One warp per (source, chain, direction) runs the recursion frame by frame:
// the forward warp a_t = (a_{t-1} A) diag(e_t) from a_0 = pi diag(e_0), the
// backward warp b_t = A diag(e_{t+1}) b_{t+1} from b_{T-1} = 1.  Lane n owns
// states n and n + 32; the chain's transition matrix sits in its registers as
// f32x2 pairs along the summed index ((A_in, A_i+1,n) for the forward warp,
// (A_ni, A_n,i+1) for the backward one), so that a 16-byte load of the
// previous vector from shared memory feeds two packed FMAs per state; all of
// a step's loads are issued before its FMAs.  Scaling: the vector stored at a
// step is the matrix product of the previous stored vector times 2^-k, k the
// exponent of that vector's largest entry (the maximum of non-negative floats
// is that of their bit patterns: one redux.sync, whose latency the next
// step's loads and FMAs hide), so stored vectors stay within one step's
// growth or shrinkage of [1, 2); the forward warp sums the applied exponents
// for log Z.  (A step that shrinks the vector below 2^-126 -- only possible
// when A has near-zero entries between the states holding the mass and the
// likely ones -- loses precision in that vector; the scan does not.)
// Emissions: a first pass (k_fb_seq_emit, one warp per frame, HBM-bound)
// writes every frame's e = exp(phi - max) (the hardware approximation) as a
// row of 68 floats, states n and n + 32 side by side at 2 (n % 32) + n / 32
// and the frame maximum at 64; the recursion warps copy those rows 32 frames
// at a time with cp.async one block ahead (lane r the block's r-th frame) and
// read one 8-byte pair per lane and step.  (Measured on the GB300: preparing
// the rows inside the recursion warps cost ~80 of a step's ~520 cycles.)  A
// block's stored vectors collect in shared memory and leave in one coalesced
// pass at the block's end, instead of two scattered stores per step.
// The forward vectors are written to d-hat, the backward ones to a scratch
// array, and a second kernel forms d-hat_t = a_t b_t / sum_n a_tn b_tn.
// Per frame this is 2 N^2 FMAs against the scan's N^3 for chunk products, but
// the latency is the chain's length in frame steps: the form for batches of
// many chains, run on a few SMs beside the contractions (blocks of `cpc`
// chains, two warps each).
constexpr int SEQ_ROW = 68;   // prepared emission row: 64 state positions, the maximum, padding
template <int NP>
struct SeqCfg {
  static constexpr bool TWO = NP > 32;   // two states per lane
  static constexpr int RS = SEQ_ROW;     // emission row stride (floats; 16-byte rows)
  static constexpr int BLK = 32;         // frames per emission block (one per lane)
  static constexpr int VEC = 64;         // floats per vector buffer
  static constexpr int OUT = BLK * NP;   // a block's stored vectors (rows of N floats)
  static constexpr int WARP_FLOATS = 2 * BLK * RS + 2 * VEC + OUT;
  static constexpr int MAX_THREADS = 256;   // registers: A and a step's loads
};

template <int NP>
static int seq_max_cpc() {
  using Cfg = SeqCfg<NP>;
  const int by_smem = (int)(SMEM_OPTIN / (2 * Cfg::WARP_FLOATS * sizeof(float)));
  const int by_threads = Cfg::MAX_THREADS / 64;
  return by_smem < by_threads ? by_smem : by_threads;
}

// One direction of one chain (the warp's whole job).
template <int NP, bool FWD>
__device__ __forceinline__ void seq_chain(const FBArgs& a, int s, int ch, float* eb, float* vb,
                                          float* ob, int lane) {
  using Cfg = SeqCfg<NP>;
  constexpr int RS = Cfg::RS, BLK = Cfg::BLK, VEC = Cfg::VEC;
  constexpr bool TWO = Cfg::TWO;
  const int N = a.N;
  const int j0 = lane, j1 = lane + 32;
  const bool h0 = j0 < N, h1 = TWO && j1 < N;
  const float* Ag = a.A + (size_t)s * N * N;
  auto A_of = [&](int i, int j) {   // the factor multiplying v_i in state j's sum
    return (i < N && j < N) ? (FWD ? Ag[i * N + j] : Ag[j * N + i]) : 0.f;
  };
  float2 P0[NP / 2], P1[TWO ? NP / 2 : 1];
#pragma unroll
  for (int i = 0; i < NP; i += 2) {
    P0[i / 2] = make_float2(A_of(i, j0), A_of(i + 1, j0));
    if (TWO) P1[i / 2] = make_float2(A_of(i, j1), A_of(i + 1, j1));
  }
  const float2 start = FWD ? make_float2(h0 ? a.pi[(size_t)s * N + j0] : 0.f,
                                         h1 ? a.pi[(size_t)s * N + j1] : 0.f)
                           : make_float2(h0 ? 1.f : 0.f, h1 ? 1.f : 0.f);
  const int t0 = a.chain_t0 ? a.chain_t0[ch] : 0;
  const int T = a.chain_len ? a.chain_len[ch] : a.T;
  float* out = (FWD ? a.dhat : a.beta) + ((size_t)s * a.T + t0) * N;   // the chain's first row
  const float* em = a.emis + ((size_t)s * a.T + t0) * SEQ_ROW;
  const int nblk = (T + BLK - 1) / BLK;
  // frame of row r of block b: forward b*BLK + r, backward T-1 - b*BLK - r
  auto issue = [&](int b) {
    const int t = FWD ? b * BLK + lane : T - 1 - b * BLK - lane;
    if (b < nblk && t >= 0 && t < T) {
      float* dst = eb + (b & 1) * BLK * RS + lane * RS;
      const float* src = em + (size_t)t * SEQ_ROW;
#pragma unroll
      for (int n = 0; n < SEQ_ROW; n += 4) cp_async16(dst + n, src + n);
    }
    cp_async_commit();
  };
  griddep_wait();   // the prepared emissions
  double msum = 0.0;   // forward: the frame maxima of the rows this lane copied
  int kexp = 0;        // forward: exponents removed by the scaling
  unsigned bad = 0;
  float2 z = make_float2(0.f, 0.f);
  unsigned mbprev = 0;   // bit pattern of the previous stored vector's largest entry
  issue(0);
  for (int b = 0; b < nblk; ++b) {
    issue(b + 1);
    cp_async_wait<1>();   // block b has landed
    __syncwarp();
    if (FWD) {
      const int t = b * BLK + lane;
      if (t < T) msum += (double)eb[(b & 1) * BLK * RS + lane * RS + 64];
    }
    const int nf = min(BLK, T - b * BLK);
    const float* erow = eb + (b & 1) * BLK * RS;
    for (int r = 0; r < nf; ++r, erow += RS) {
      const int q = b * BLK + r;   // step of this warp
      const float2 e2 = *reinterpret_cast<const float2*>(erow + 2 * lane);
      if (q == 0) {
        z = FWD ? __fmul2_rn(start, e2) : start;
      } else {
        // forward: (a_{t-1} A)_j;  backward: (A u_{t+1})_i with u = e (.) b
        const float* v = vb + ((q - 1) & 1) * VEC;
        float4 x[NP / 4];
#pragma unroll
        for (int i = 0; i < NP / 4; ++i) x[i] = *reinterpret_cast<const float4*>(v + 4 * i);
        float2 c0[4], c1[4];
#pragma unroll
        for (int k = 0; k < NP / 4; ++k) {
          const float2 lo = make_float2(x[k].x, x[k].y), hi = make_float2(x[k].z, x[k].w);
          const int u = (2 * k) & 3, w = (2 * k + 1) & 3;
          c0[u] = k < 2 ? __fmul2_rn(P0[2 * k], lo) : __ffma2_rn(P0[2 * k], lo, c0[u]);
          c0[w] = k < 2 ? __fmul2_rn(P0[2 * k + 1], hi) : __ffma2_rn(P0[2 * k + 1], hi, c0[w]);
          if (TWO) {
            c1[u] = k < 2 ? __fmul2_rn(P1[2 * k], lo) : __ffma2_rn(P1[2 * k], lo, c1[u]);
            c1[w] = k < 2 ? __fmul2_rn(P1[2 * k + 1], hi) : __ffma2_rn(P1[2 * k + 1], hi, c1[w]);
          }
        }
        const float2 s0 = __fadd2_rn(__fadd2_rn(c0[0], c0[1]), __fadd2_rn(c0[2], c0[3]));
        float2 y = make_float2(s0.x + s0.y, 0.f);
        if (TWO) {
          const float2 s1 = __fadd2_rn(__fadd2_rn(c1[0], c1[1]), __fadd2_rn(c1[2], c1[3]));
          y.y = s1.x + s1.y;
        }
        // the previous vector's scale 2^-k, decoded only now: the reduction
        // that produced its bit pattern ran during this step's loads and FMAs
        int k = mbprev < 0x00800000u ? -126 : (int)(mbprev >> 23) - 127;  // subnormal: one factor
        const bool okm = mbprev != 0u && mbprev < 0x7f000000u;   // else vanished or not finite
        bad |= okm ? 0u : 1u;
        k = okm ? k : 0;
        kexp += k;
        const float sc = pow2f(-k);
        y = __fmul2_rn(y, make_float2(sc, sc));
        z = FWD ? __fmul2_rn(y, e2) : y;
      }
      // the block's vectors in frame order, written out together below
      const int orow = FWD ? r : nf - 1 - r;
      if (h0) ob[orow * N + j0] = z.x;
      if (h1) ob[orow * N + j1] = z.y;
      const float2 u = FWD ? z : __fmul2_rn(z, e2);
      float* vn = vb + (q & 1) * VEC;
      vn[j0] = u.x;
      if (TWO) vn[j1] = u.y;
      // the next step's scale comes from this vector's largest entry
      mbprev = __reduce_max_sync(0xffffffffu, __float_as_uint(fmaxf(z.x, z.y)));
      __syncwarp();
    }
    // the block's nf rows, contiguous in memory (frames ascending), by
    // coalesced stores; the buffer is rewritten only after the next block's
    // opening __syncwarp
    float* dst = out + (size_t)(FWD ? b * BLK : T - b * BLK - nf) * N;
    const int cnt = nf * N;
    if ((N & 3) == 0 && (reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
      for (int i = lane; i < cnt / 4; i += 32)
        reinterpret_cast<float4*>(dst)[i] = reinterpret_cast<const float4*>(ob)[i];
    } else {
      for (int i = lane; i < cnt; i += 32) dst[i] = ob[i];
    }
  }
  cp_async_wait<0>();
  if (FWD) {
    // log Z = sum_t max_n phi_tn + ln 2 (exponents removed) + ln sum_n a_{T-1,n}
    const double mt = warp_sum_d(msum);
    const float sl = warp_sum(z.x + z.y);
    if (lane == 0)
      a.logZ[(size_t)s * a.nchains + ch] = T > 0 ? mt + LN2 * (double)kexp + log((double)sl) : 0.0;
  }
  if (bad && lane == 0) atomicOr(a.err, ERR_FB_ZERO);
}

template <int NP>
__global__ void __launch_bounds__(SeqCfg<NP>::MAX_THREADS) k_fb_seq(FBArgs a) {
  using Cfg = SeqCfg<NP>;
  extern __shared__ __align__(16) float sm[];
  if (!a.inputs_stable) griddep_wait();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = blockIdx.x * (blockDim.x >> 6) + (warp >> 1);
  if (g >= a.S * a.nchains) return;
  const int s = g / a.nchains, ch = g - s * a.nchains;
  float* eb = sm + warp * Cfg::WARP_FLOATS;   // two emission blocks
  float* vb = eb + 2 * Cfg::BLK * Cfg::RS;    // two vectors
  float* ob = vb + 2 * Cfg::VEC;              // a block's stored vectors
  if ((warp & 1) == 0)
    seq_chain<NP, true>(a, s, ch, eb, vb, ob, lane);
  else
    seq_chain<NP, false>(a, s, ch, eb, vb, ob, lane);
}


// The sequential form's emission rows: e = exp(phi - max_n phi) of every
// frame, states n and n + 32 at 2 (n % 32) + n / 32 (zeros past N), the
// maximum at 64.  One warp per frame, eight frames per warp, 64 frames of one
// chain per block; the row maximum by one redux.sync over order-preserving
// integer keys.
template <int NP>
__global__ void __launch_bounds__(256) k_fb_seq_emit(FBArgs a) {
  const int N = a.N;
  const int g = blockIdx.y;
  const int s = g / a.nchains, ch = g - s * a.nchains;
  const int t0 = a.chain_t0 ? a.chain_t0[ch] : 0;
  const int T = a.chain_len ? a.chain_len[ch] : a.T;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  griddep_wait();   // the log-emissions
  // the recursions may be scheduled now; they wait for this pass to finish
  griddep_launch_dependents();
  if ((int)blockIdx.x * 64 >= T) return;   // the whole block
  const bool h0 = lane < N, h1 = lane + 32 < N;
  for (int i = 0; i < 8; ++i) {   // uniform in the warp
    const int f = blockIdx.x * 64 + warp * 8 + i;
    if (f >= T) break;
    const size_t fr = (size_t)s * a.T + t0 + f;
    const float* x = a.phi + fr * N;
    const float x0 = h0 ? x[lane] : -INFINITY, x1 = h1 ? x[lane + 32] : -INFINITY;
    const unsigned u = __float_as_uint(fmaxf(x0, x1));
    const unsigned key = __reduce_max_sync(0xffffffffu, (u & 0x80000000u) ? ~u : (u | 0x80000000u));
    const float m = __uint_as_float((key & 0x80000000u) ? (key & 0x7fffffffu) : ~key);
    float* row = a.emis + fr * SEQ_ROW;
    *reinterpret_cast<float2*>(row + 2 * lane) =
        make_float2(h0 ? __expf(x0 - m) : 0.f, h1 ? __expf(x1 - m) : 0.f);
    if (lane == 0) row[64] = m;
  }
}

// d-hat_t = a_t b_t / sum_n a_tn b_tn for the sequential form: four threads
// per frame (a quarter of the states each), 64 frames of one chain per block;
// a_t is read from d-hat and overwritten.  The stored vectors have their
// largest entry in [1, 2), so the products stay in range.
template <int NP>
__global__ void __launch_bounds__(256) k_fb_seq_combine(FBArgs a) {
  constexpr int QS = NP / 4;
  const int N = a.N;
  const int g = blockIdx.y;
  const int s = g / a.nchains, ch = g - s * a.nchains;
  const int t0 = a.chain_t0 ? a.chain_t0[ch] : 0;
  const int T = a.chain_len ? a.chain_len[ch] : a.T;
  griddep_wait();
  if ((int)blockIdx.x * 64 >= T) return;   // the whole block
  const int f = blockIdx.x * 64 + (threadIdx.x >> 2);
  const int n0 = (threadIdx.x & 3) * QS;
  const bool ok = f < T;
  const size_t row = ((size_t)s * a.T + t0 + (ok ? f : 0)) * N;
  float p[QS];
  float z = 0.f;
#pragma unroll
  for (int k = 0; k < QS; ++k) {
    const bool in = ok && n0 + k < N;
    p[k] = in ? a.dhat[row + n0 + k] * a.beta[row + n0 + k] : 0.f;
    z += p[k];
  }
  z += __shfl_xor_sync(0xffffffffu, z, 1);
  z += __shfl_xor_sync(0xffffffffu, z, 2);
  if (ok) {
    if (!(z > 0.f) || !isfinite(z)) {
      atomicOr(a.err, ERR_FB_ZERO);
      z = 1.f;
    }
    const float iz = 1.f / z;
#pragma unroll
    for (int k = 0; k < QS; ++k)
      if (n0 + k < N) a.dhat[row + n0 + k] = p[k] * iz;
  }
}

// ------------------------------------------------------------------ launch
template <int NP>
static size_t smem_chain(int mode, int L) {
  using Cfg = ChainCfg<NP>;
  const size_t bb = mode == CHAIN_CHUNK ? Cfg::IMG_BYTES : Cfg::RING * Cfg::IMG_BYTES;
  const size_t ee = mode == CHAIN_CHUNK
                        ? ((size_t)Cfg::RCH * L * NP + ((Cfg::RCH * L + 3) & ~3) + Cfg::A_FLOATS) *
                              sizeof(float)
                        : 0;
  return 1024 + 2 * (size_t)Cfg::ROWS_BYTES + bb + ee + sizeof(ChainMisc);
}
template <int NP>
static size_t smem_products_simt(int L) {
  return (128 + 16) * sizeof(double) +
         (size_t)(NP * NP + 128 * (NP + 1) + 8 + (128 / NP) * L * NP) * sizeof(float);
}
template <int NP>
static size_t smem_group() {
  return (size_t)(2 * NP + GRING * NP * (NP + 4) + (NP / 2) * 128) * sizeof(float);
}
template <int NP, int MODE>
static size_t smem_scan() {
  const int ring = MODE == MODE_GROUP_REPLAY ? ScanRingGroupReplay<NP>::R : ScanRing<NP>::R;
  return (size_t)(ring * NP * (NP + 4) + 64) * sizeof(float);
}
static size_t smem_replay_chunk(int NP, int L) { return (size_t)(3 * L * NP + 128) * sizeof(float); }
// One chunk (two warps, <= 128 registers a thread, a few KB of shared memory)
// per block: such a block fits on an SM beside a persistent contraction CTA
// (which leaves ~11k registers and ~10-30 KB of shared memory), so the replay
// does not wait for the contraction's SMs; blocks of four chunks did.
static int replay_chunks(int NP, int L) {
  (void)NP;
  (void)L;
  return 1;
}

// Launch a pass that consumes the previous pass's results as a programmatic
// dependent of it: its blocks may be scheduled once every block of the
// previous pass has signalled (griddepcontrol.launch_dependents), run their
// independent setup, and wait (griddepcontrol.wait) before reading the
// previous results.  On the legacy default stream it is an ordinary launch.
static cudaError_t launch_dependent(void (*kernel)(FBArgs), dim3 grid, int block, size_t smem,
                                   cudaStream_t st, const FBArgs& a) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  const bool legacy = st == nullptr || st == cudaStreamLegacy;
  cfg.attrs = legacy ? nullptr : attr;
  cfg.numAttrs = legacy ? 0 : 1;
  return cudaLaunchKernelEx(&cfg, kernel, a);
}

template <int NP>
static cudaError_t launch_np(const FBArgs& a, cudaStream_t st) {
  static cudaError_t attr = cudaErrorNotReady;
  if (attr == cudaErrorNotReady) {
    attr = cudaFuncSetAttribute(k_fb_chain<NP, CHAIN_CHUNK>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem_chain<NP>(CHAIN_CHUNK, FB_MAX_L));
    if (attr == cudaSuccess)
      attr = cudaFuncSetAttribute(k_fb_chain<NP, CHAIN_GROUP>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem_chain<NP>(CHAIN_GROUP, 0));
    if (attr == cudaSuccess)
      attr = cudaFuncSetAttribute(k_fb_scan<NP, MODE_CHAINS>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem_scan<NP, MODE_CHAINS>());
    if (attr == cudaSuccess)
      attr = cudaFuncSetAttribute(k_fb_scan<NP, MODE_GROUP_REPLAY>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem_scan<NP, MODE_GROUP_REPLAY>());
    if (attr == cudaSuccess)
      attr = cudaFuncSetAttribute(k_fb_group_products<NP>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem_group<NP>());
    if (attr == cudaSuccess)
      attr = cudaFuncSetAttribute(k_fb_replay<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)SMEM_OPTIN);
    if (attr == cudaSuccess)
      attr = cudaFuncSetAttribute(k_fb_products_simt<NP>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem_products_simt<NP>(FB_MAX_L));
    if (attr == cudaSuccess)
      attr = cudaFuncSetAttribute(k_fb_seq<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)SMEM_OPTIN);
  }
  if (attr != cudaSuccess) return attr;
  if (a.seq > 0) {
    // the sequential form: recursions (a programmatic dependent of whatever
    // wrote the emissions), then d-hat
    const int cpc = a.seq < seq_max_cpc<NP>() ? a.seq : seq_max_cpc<NP>();
    const int chains = a.S * a.nchains;
    cudaError_t e = cudaSuccess;
    if (a.maxlen > 0)
      e = launch_dependent(k_fb_seq_emit<NP>, dim3((a.maxlen + 63) / 64, chains), 256, 0, st, a);
    // at least 120 KB of shared memory per block, so that no two blocks share
    // an SM: each warp keeps its sub-partition to itself (with up to four
    // chains per block, two), and the SMs the contractions leave free are
    // exactly the blocks' count
    size_t smem = (size_t)cpc * 2 * SeqCfg<NP>::WARP_FLOATS * sizeof(float);
    if (smem < 120 * 1024) smem = 120 * 1024;
    if (e == cudaSuccess)
      e = launch_dependent(k_fb_seq<NP>, dim3((chains + cpc - 1) / cpc), 64 * cpc, smem, st, a);
    if (e == cudaSuccess && a.maxlen > 0)
      e = launch_dependent(k_fb_seq_combine<NP>, dim3((a.maxlen + 63) / 64, chains), 256, 0, st,
                           a);
    const cudaError_t l = cudaGetLastError();
    return e != cudaSuccess ? e : l;
  }
  using Cfg = ChainCfg<NP>;
  const int rc = replay_chunks(NP, a.L);
  const bool tc = a.products == FB_PRODUCTS_TC;
  cudaError_t e = cudaSuccess;
  const dim3 pgrid((a.C + Cfg::RCH - 1) / Cfg::RCH, a.S);
  if (tc) {
    FBArgs p = a;   // the chunk pass writes the group pass's operand images
    if (a.G < 2) p.Pimg = nullptr;
    // a programmatic dependent of whatever wrote the emissions before it
    e = launch_dependent(k_fb_chain<NP, CHAIN_CHUNK>, pgrid, 256,
                         smem_chain<NP>(CHAIN_CHUNK, a.L), st, p);
  } else {
    k_fb_products_simt<NP><<<pgrid, 128, smem_products_simt<NP>(a.L), st>>>(a);
  }
  if (a.G >= 2) {
    // group products, the scan across groups (the chain scan over the group
    // arrays), then each group's chunk boundaries
    if (tc && e == cudaSuccess)
      e = launch_dependent(k_fb_chain<NP, CHAIN_GROUP>, dim3(a.NG, a.S), 256,
                           smem_chain<NP>(CHAIN_GROUP, 0), st, a);
    else
      k_fb_group_products<NP><<<dim3(a.NG, a.S), NP * 16, smem_group<NP>(), st>>>(a);
    FBArgs b = a;
    b.C = a.NG;
    b.chain_c0 = a.chain_g0;
    b.P = a.Q;
    b.PT = a.QT;
    b.Plog = a.Qlog;
    b.fwd = a.gfwd;
    b.bwd = a.gbwd;
    b.lam = a.glam;
    if (e == cudaSuccess)
      e = launch_dependent(k_fb_scan<NP, MODE_CHAINS>, dim3(a.S * a.nchains, 2), 32,
                           smem_scan<NP, MODE_CHAINS>(), st, b);
    if (e == cudaSuccess)
      e = launch_dependent(k_fb_scan<NP, MODE_GROUP_REPLAY>, dim3(a.S * a.NG, 2), 32,
                           smem_scan<NP, MODE_GROUP_REPLAY>(), st, a);
  } else {
    e = launch_dependent(k_fb_scan<NP, MODE_CHAINS>, dim3(a.S * a.nchains, 2), 32,
                         smem_scan<NP, MODE_CHAINS>(), st, a);
  }
  if (e == cudaSuccess)
    e = launch_dependent(k_fb_replay<NP>, dim3((a.C + rc - 1) / rc, a.S), rc * 64,
                         rc * smem_replay_chunk(NP, a.L), st, a);
  const cudaError_t l = cudaGetLastError();
  return e != cudaSuccess ? e : l;
}

int fb_chunk_count(const int* chain_len, int nchains, int L) {
  int C = 0;
  for (int j = 0; j < nchains; ++j) C += (chain_len[j] + L - 1) / L;
  return C;
}

size_t fb_scratch_bytes(int S, int N, int C, int NG) {
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  size_t b = 0;
  b += al((size_t)S * C * mat_floats(N) * sizeof(float));  // P
  b += al((size_t)S * C * mat_floats(N) * sizeof(float));  // P^T
  b += al((size_t)S * C * sizeof(double));                 // Plog
  b += al((size_t)S * C * N * sizeof(float));              // fwd
  b += al((size_t)S * C * sizeof(float));                  // lam
  b += al((size_t)S * C * N * sizeof(float));              // bwd
  b += al((size_t)S * NG * mat_floats(N) * sizeof(float)); // Q
  b += al((size_t)S * NG * mat_floats(N) * sizeof(float)); // Q^T
  b += al((size_t)S * NG * sizeof(double));                // Qlog
  b += al((size_t)S * NG * N * sizeof(float));             // gfwd
  b += al((size_t)S * NG * N * sizeof(float));             // gbwd
  b += al((size_t)S * NG * sizeof(float));                 // glam
  if (NG > 0) b += al((size_t)S * C * fb_image_bytes(N));  // chunk operand images
  return b;
}

size_t fb_image_bytes(int N) {
  const int NP = pad8(N), katoms = (NP + 31) / 32, nout = (NP + 15) & ~15;
  return 2 * (size_t)katoms * nout * 128;
}

void fb_carve_scratch(FBArgs& a, void* base) {
  char* p = reinterpret_cast<char*>(base);
  const size_t S = a.S, C = a.C, N = a.N, NG = a.NG;
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
  a.Q = reinterpret_cast<float*>(take(S * NG * mat_floats((int)N) * sizeof(float)));
  a.QT = reinterpret_cast<float*>(take(S * NG * mat_floats((int)N) * sizeof(float)));
  a.Qlog = reinterpret_cast<double*>(take(S * NG * sizeof(double)));
  a.gfwd = reinterpret_cast<float*>(take(S * NG * N * sizeof(float)));
  a.gbwd = reinterpret_cast<float*>(take(S * NG * N * sizeof(float)));
  a.glam = reinterpret_cast<float*>(take(S * NG * sizeof(float)));
  a.Pimg = NG > 0 ? reinterpret_cast<uint8_t*>(take(S * C * fb_image_bytes((int)N))) : nullptr;
}

int fb_default_group(int C) {
  // the grouped scan costs ~2G + C/G serial steps: G = sqrt(C/2); below
  // ~24 chunks a plain scan is as short
  if (C < 24) return 0;
  int G = (int)ceil(sqrt(0.5 * (double)C));
  return G < 2 ? 2 : G;
}

int fb_seq_max_cpc(int N) {
  switch (pad8(N)) {
    case 8: return seq_max_cpc<8>();
    case 16: return seq_max_cpc<16>();
    case 24: return seq_max_cpc<24>();
    case 32: return seq_max_cpc<32>();
    case 40: return seq_max_cpc<40>();
    case 48: return seq_max_cpc<48>();
    case 56: return seq_max_cpc<56>();
    case 64: return seq_max_cpc<64>();
    default: return 1;
  }
}

int fb_seq_blocks(int chains, int cpc, int N) {
  const int m = fb_seq_max_cpc(N);
  if (cpc > m) cpc = m;
  if (cpc < 1) cpc = 1;
  return (chains + cpc - 1) / cpc;
}

cudaError_t launch_fb(const FBArgs& a, cudaStream_t st, int* launches) {
  if (launches) *launches += a.seq > 0 ? (a.maxlen > 0 ? 3 : 1) : a.G >= 2 ? 5 : 3;
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
