// Tensor-core form of the two contractions of Eq. 7 on sm_103a:
//   reconstruction   Vhat[t][l] = sum_k w[t][k] beta[l][k]   -> Q = V / Vhat (+ bound partial)
//   back-projection  R[t][k]    = sum_l Q[t][l] beta[k][l]   -> counts = w * R
// Both are C[t][n] = sum_k A[t][k] B[n][k] with K contiguous in both operands.
//
// A persistent CTA per SM computes a sequence of 128 x BN output tiles; the
// accumulator lives in TMEM.  Warp 0 streams K-blocks of A and B into a ring
// of shared-memory stages with TMA (128-byte swizzle), warp 1 issues
// tcgen05.mma from one thread and frees each stage with tcgen05.commit, warps
// 2-9 copy a finished tile's accumulator out of TMEM with tcgen05.ld, release
// TMEM to the next tile's MMAs and apply the epilogue from registers.  Every
// mbarrier wait is bounded: a wait that gives up sets ERR_TIMEOUT in the error
// word and the CTA winds down (outstanding copies and MMAs are awaited, TMEM
// is freed) instead of hanging.
//
// FP32 mode ("split TF32"): each operand x is stored as hi = tf32(x) and
// lo = tf32(x - hi); each K-step issues hi*hi, hi*lo and lo*hi (~22
// significant bits per product).  BF16 mode: one pass over BF16 operands.
// The tensor core's FP32 accumulation does not round to nearest at every
// addition, so a long chain of additions into one accumulator drifts (a few
// 1e-6 relative after ~300 MMAs).  The accumulator is therefore split over
// all 512 TMEM columns: the hi*hi (or BF16) products of K-block kb go to
// accumulator kb % NMAIN, the small cross terms to one more accumulator, and
// the epilogue adds them in FP32 with round-to-nearest.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "nfhmm_device.cuh"
#include "nfhmm_kernels.h"
#include "nfhmm_tc.h"
#include "tc_ptx.cuh"

namespace nfhmm {

namespace {

using namespace tc;

constexpr int BM = 128;
constexpr int BN1 = 128;           // default reconstruction tile: columns = frequencies
constexpr int BN2 = 160;           // default back-projection tile: columns = elements
constexpr int BNX = 64;            // exact inference back-projection: the S*K elements of a joint state
constexpr int SMEM_BUDGET = 227 * 1024;   // per-block opt-in limit
constexpr int EPI_WARPS = 8;                    // two per TMEM lane quarter
constexpr int NUM_THREADS = 64 + EPI_WARPS * 32;  // TMA warp, MMA warp, epilogue
enum TcEpi { TEPI_RATIO = 0, TEPI_SCALE = 1 };

template <int KIND>
struct KindCfg;
template <>
struct KindCfg<KIND_TF32X3> {
  static constexpr int ES = 4;            // element bytes
  static constexpr int BK = 32;           // 128 bytes of K per stage row
  static constexpr int KSTEP = 8;         // K per MMA instruction
  static constexpr int NOPS = 2;          // hi and lo copies
};
template <>
struct KindCfg<KIND_BF16> {
  static constexpr int ES = 2;
  static constexpr int BK = 64;
  static constexpr int KSTEP = 16;
  static constexpr int NOPS = 1;
};

template <int KIND, int BN>
struct TileCfg {
  using K = KindCfg<KIND>;
  static constexpr int A_BYTES = BM * 128;          // one operand copy of A per stage
  static constexpr int B_BYTES = BN * 128;
  static constexpr int STAGE_BYTES = K::NOPS * (A_BYTES + B_BYTES);
  static constexpr int EXTRA = 1024 /*align*/ + 256 /*barriers*/;
  // staged epilogue operand: per epilogue thread (row, half) its BN/2 floats
  // of V or w, each segment padded by 16 bytes (conflict-free float4 reads)
  static constexpr int EPI_SEG = BN / 2 * 4 + 16;
  static constexpr int EPI_BYTES = 2 * BM * EPI_SEG;
  static constexpr int fit(int extra) {
    return (SMEM_BUDGET - EXTRA - extra) / STAGE_BYTES < 8
               ? (SMEM_BUDGET - EXTRA - extra) / STAGE_BYTES : 8;
  }
  // the deepest shared-memory ring that fits (at most 8 stages), without
  // and with the staged epilogue operand
  static constexpr int MAX_STAGES = fit(0);
  static constexpr int MAX_STAGES_EPI = fit(EPI_BYTES);
  static constexpr int smem(int stages, bool epi) {
    return stages * STAGE_BYTES + (epi ? EPI_BYTES : 0) + EXTRA;
  }
  static constexpr int TMEM_COLS = 512;
  static constexpr int NACC = 512 / BN;                          // accumulators of BN columns
  static constexpr int NMAIN = K::NOPS == 2 ? NACC - 1 : NACC;   // for hi*hi (or BF16) products
};

struct Maps {
  CUtensorMap a_hi, a_lo, b_hi, b_lo;
};

struct TcArgs {
  int rows, cols, kdim;           // T, output columns, K
  int row_off;                    // first row (one item: rows [row_off, row_off + rows))
  int nbpart;
  const float* V;                 // RATIO: T x ldv
  int ldv;
  const float* w;                 // SCALE: T x ldw (w in float)
  int ldw;
  float* out_f32;                 // RATIO: Q hi (tf32) or unused; SCALE: counts
  float* out_lo;                  // RATIO tf32: Q lo
  __nv_bfloat16* out_bf16;        // RATIO bf16: Q
  int ldo;
  double* bpart;                  // RATIO: bound partial per (row, column tile), may be null
  unsigned* err;
  // batched form: the rows are items of brows rows each (a multiple of BM),
  // of which the first bvalid are real; item b reads B rows from b * bstride
  // on, and V (RATIO) is shared by the items.  brows = 0: one item.
  int brows, bvalid, bstride;
  int stages;                     // depth of the shared-memory ring (2 .. MAX_STAGES)
  int prefetch;                   // K-blocks beyond the ring brought into L2 ahead (0: none)
  int epi_stage;                  // 1: the epilogue's V (or w) tile is copied into shared
                                  // memory before its accumulator is awaited
  // test hook, 0 in normal use: the MMA thread first waits this many
  // nanoseconds on a barrier nothing arrives on, so that the wait gives up
  // and the CTA takes its wind-down path (error word ERR_TIMEOUT)
  unsigned long long inject_wait_ns;
};

// ------------------------------------------------------------------ kernel
// Persistent: CTA b takes output tiles b, b + gridDim.x, ... (row-major over
// (row tile, column tile), so the CTAs in flight share A row tiles in L2).
// The stage ring runs on across tiles.  The epilogue warps copy a tile's
// summed accumulator out of TMEM into registers and release TMEM at once, so
// the MMA warp starts the next tile while they divide, take logs and store.
template <int KIND, int BN, int EPI>
__global__ void __launch_bounds__(NUM_THREADS, 1)
    k_tc_gemm(const __grid_constant__ Maps maps, const TcArgs p) {
  using K = KindCfg<KIND>;
  using Cfg = TileCfg<KIND, BN>;
  static_assert(Cfg::MAX_STAGES >= 2, "tile too large for a two-stage ring");
  static_assert(BN % 32 == 0 && BN <= 256, "the epilogue halves are multiples of 16 columns");
  const int STAGES = p.stages;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint8_t* epi_buf = smem + STAGES * Cfg::STAGE_BYTES;   // staged epilogue operand (if used)
  uint64_t* full =
      reinterpret_cast<uint64_t*>(epi_buf + (p.epi_stage ? Cfg::EPI_BYTES : 0));
  uint64_t* empty = full + STAGES;
  uint64_t* accum = empty + STAGES;        // MMA -> epilogue: a tile's accumulator is complete
  uint64_t* tmem_free = accum + 1;         // epilogue -> MMA: it has been read out
  uint64_t* drain = tmem_free + 1;         // the MMA thread's last commit (before TMEM is freed)
  uint64_t* never = drain + 1;             // test hook: a barrier nothing arrives on
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(never + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nkb = (p.kdim + K::BK - 1) / K::BK;
  const int ncol = (p.cols + BN - 1) / BN;
  const int ntiles = ncol * ((p.rows + BM - 1) / BM);

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accum, 1);
    mbar_init(tmem_free, EPI_WARPS);
    mbar_init(drain, 1);
    mbar_init(never, 1);
    *abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, Cfg::TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  auto stage_ptr = [&](int s, int which) {  // 0: A hi, 1: A lo, 2: B hi, 3: B lo
    uint8_t* base = smem + s * Cfg::STAGE_BYTES;
    if (which == 0) return base;
    if (which == 1) return base + Cfg::A_BYTES;
    return base + K::NOPS * Cfg::A_BYTES + (which - 2) * Cfg::B_BYTES;
  };
  auto give_up = [&]() {
    *abort_flag = 1;
    atomicOr(p.err, ERR_TIMEOUT);
  };

  if (warp == 0) {
    // ---------------- TMA producer
    if (lane == 0) {
      long long it = 0;   // K-blocks issued over all of this CTA's tiles
      int s = 0;          // its ring slot, it % STAGES
      uint32_t ph = 0;    // and (it / STAGES) & 1
      // the L2 prefetch runs `prefetch` K-blocks ahead of the loads, over the
      // same sequence of (tile, K-block)
      int ptile = blockIdx.x, pkb = 0;
      auto prefetch_next = [&]() {
        if (ptile >= ntiles) return;
        const int prow0 = p.row_off + (ptile / ncol) * BM, pcol0 = (ptile % ncol) * BN;
        const int pbcol0 = pcol0 + (p.brows ? prow0 / p.brows : 0) * p.bstride;
        tma_prefetch_l2_2d(&maps.a_hi, pkb * K::BK, prow0);
        tma_prefetch_l2_2d(&maps.b_hi, pkb * K::BK, pbcol0);
        if (K::NOPS == 2) {
          tma_prefetch_l2_2d(&maps.a_lo, pkb * K::BK, prow0);
          tma_prefetch_l2_2d(&maps.b_lo, pkb * K::BK, pbcol0);
        }
        if (++pkb == nkb) {
          pkb = 0;
          ptile += gridDim.x;
        }
      };
      for (int i = 0; i < p.prefetch; ++i) prefetch_next();
      for (int tile = blockIdx.x; tile < ntiles && !*abort_flag; tile += gridDim.x) {
        const int row0 = p.row_off + (tile / ncol) * BM, col0 = (tile % ncol) * BN;
        const int bitem = p.brows ? row0 / p.brows : 0;   // batch item of this row tile
        const int bcol0 = col0 + bitem * p.bstride;         // its first B row
        for (int kb = 0; kb < nkb; ++kb) {
          if (it >= STAGES && !mbar_wait(&empty[s], ph ^ 1u, abort_flag)) {
            give_up();
            break;
          }
          if (p.prefetch) prefetch_next();
          mbar_expect_tx(&full[s], Cfg::STAGE_BYTES);
          const int kx = kb * K::BK;
          tma_load_2d(stage_ptr(s, 0), &maps.a_hi, &full[s], kx, row0);
          tma_load_2d(stage_ptr(s, 2), &maps.b_hi, &full[s], kx, bcol0);
          if (K::NOPS == 2) {
            tma_load_2d(stage_ptr(s, 1), &maps.a_lo, &full[s], kx, row0);
            tma_load_2d(stage_ptr(s, 3), &maps.b_lo, &full[s], kx, bcol0);
          }
          ++it;
          if (++s == STAGES) {
            s = 0;
            ph ^= 1u;
          }
        }
        if (*abort_flag) break;
      }
      // every copy issued must have landed before the CTA may exit (the slot
      // of each of the last STAGES K-blocks has no later use)
      for (long long j = it - STAGES > 0 ? it - STAGES : 0; j < it; ++j) {
        if (!mbar_wait(&full[j % STAGES], (uint32_t)(j / STAGES) & 1)) atomicOr(p.err, ERR_TIMEOUT);
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer
    if (lane == 0) {
      constexpr uint32_t ID = idesc<KIND>(BM, BN);
      int s = 0;          // ring slot of the next K-block
      uint32_t ph = 0;    // and the phase its full barrier completes
      int j = 0;   // this CTA's tile count
      if (p.inject_wait_ns && !mbar_wait(never, 0, abort_flag, p.inject_wait_ns)) give_up();
      for (int tile = blockIdx.x; tile < ntiles && !*abort_flag; tile += gridDim.x, ++j) {
        // the previous tile's accumulator has been read out of TMEM
        if (j > 0 && !mbar_wait(tmem_free, (uint32_t)(j - 1) & 1, abort_flag)) {
          give_up();
          break;
        }
        tc_fence_after();
        bool ok = true;
        for (int kb = 0; kb < nkb; ++kb) {
          if (*abort_flag || !mbar_wait(&full[s], ph, abort_flag)) {
            give_up();
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a0 = smem_u32(stage_ptr(s, 0)), a1 = smem_u32(stage_ptr(s, 1));
          const uint32_t b0 = smem_u32(stage_ptr(s, 2)), b1 = smem_u32(stage_ptr(s, 3));
          const uint32_t d_main = tmem + (uint32_t)((kb % Cfg::NMAIN) * BN);
          const uint32_t d_cross = tmem + (uint32_t)(Cfg::NMAIN * BN);
#pragma unroll
          for (int kk = 0; kk < K::BK / K::KSTEP; ++kk) {
            const uint32_t off = kk * K::KSTEP * K::ES;  // bytes along K inside the swizzle atom
            mma<KIND>(d_main, sdesc(a0 + off), sdesc(b0 + off), ID,
                      (kb >= Cfg::NMAIN || kk > 0) ? 1u : 0u);
            if (K::NOPS == 2) {
              mma<KIND>(d_cross, sdesc(a0 + off), sdesc(b1 + off), ID, (kb > 0 || kk > 0) ? 1u : 0u);
              mma<KIND>(d_cross, sdesc(a1 + off), sdesc(b0 + off), ID, 1u);
            }
          }
          mma_commit(&empty[s]);
          if (++s == STAGES) {
            s = 0;
            ph ^= 1u;
          }
        }
        if (!ok) break;
        mma_commit(accum);  // fires once every MMA issued above has completed
      }
      // whatever happened above, no MMA of this thread may be in flight when TMEM is freed
      mma_commit(drain);
      if (!mbar_wait(drain, 0)) atomicOr(p.err, ERR_TIMEOUT);
    }
  } else {
    // ---------------- epilogue: warps 2..9.  Warp w reads TMEM lanes
    // 32*(w % 4) .. +31 (one output row per thread) and half (w - 2) / 4 of the
    // tile's columns.
    constexpr int HALF = BN / 2;        // a multiple of 16
    constexpr int NCH = HALF / 16;
    const int quarter = warp & 3;
    const int half = (warp - 2) >> 2;
    const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(half * HALF);
    const int nmain = nkb < Cfg::NMAIN ? nkb : Cfg::NMAIN;   // accumulators written
    // this thread's segment of the staged epilogue operand
    // (segments by half, then row: consecutive lanes 16 bytes apart mod 128)
    float* eseg = reinterpret_cast<float*>(epi_buf + (size_t)(half * BM + quarter * 32 + lane) *
                                                           Cfg::EPI_SEG);
    int j = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++j) {
      const int row0 = p.row_off + (tile / ncol) * BM, col0 = (tile % ncol) * BN;
      const int bitem = p.brows ? row0 / p.brows : 0;
      const int r = quarter * 32 + lane;
      const int t = row0 + r;
      const int tl = t - bitem * p.brows;               // row within its batch item
      const bool rv = p.brows ? tl < p.bvalid : t < p.row_off + p.rows;
      const int cbase = col0 + half * HALF;
      const float* erow = EPI == TEPI_RATIO ? p.V + (size_t)tl * p.ldv : p.w + (size_t)t * p.ldw;
      if (p.epi_stage) {
        // the tile's V (or w) for this thread's row and columns, copied while
        // the tile's MMAs run; the thread reads only what it copied itself
#pragma unroll
        for (int ch = 0; ch < NCH; ++ch) {
          const int c = cbase + 16 * ch;
          if (rv && c < p.cols) {
#pragma unroll
            for (int i = 0; i < 4; ++i) cp_async16_sm(eseg + 16 * ch + 4 * i, erow + c + 4 * i);
          }
        }
        cp_async_commit_group();
      }
      if (!mbar_wait(accum, (uint32_t)j & 1, abort_flag)) {
        give_up();
        break;
      }
      tc_fence_after();
      // the tile's accumulators, summed, into registers; then TMEM is free
      float acc[HALF];
#pragma unroll
      for (int i = 0; i < HALF; ++i) acc[i] = 0.f;
      // two accumulators' 16 columns in flight at a time (bounded registers)
#pragma unroll
      for (int ch = 0; ch < NCH; ++ch) {
#pragma unroll
        for (int a0 = 0; a0 < Cfg::NACC; a0 += 2) {
          uint32_t raw[2][16];
          bool use[2];
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const int a = a0 + u;
            use[u] = a < Cfg::NACC && (a == 0 || a < nmain || (K::NOPS == 2 && a == Cfg::NMAIN));
            if (use[u]) tmem_ld16_nw(taddr + (uint32_t)(a * BN + 16 * ch), raw[u]);
          }
          tmem_wait_ld();
#pragma unroll
          for (int u = 0; u < 2; ++u)
            if (use[u]) {
#pragma unroll
              for (int i = 0; i < 16; ++i) acc[16 * ch + i] += __uint_as_float(raw[u][i]);
            }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tmem_free);
      if (p.epi_stage) cp_async_wait_all();
      // the epilogue proper, from registers, beside the next tile's MMAs
      double part = 0.0;
      unsigned bad = 0;
#pragma unroll 1
      for (int ch = 0; ch < NCH; ++ch) {   // rolled: bounded register use
        const int c = cbase + 16 * ch;
        if (!rv || c >= p.cols) continue;   // cols is a multiple of 16
        float x16[16];                      // columns 16 ch .. of acc, by selects
#pragma unroll
        for (int cc = 0; cc < NCH; ++cc)
          if (cc == ch) {
#pragma unroll
            for (int i = 0; i < 16; ++i) x16[i] = acc[16 * cc + i];
          }
        // rows are padded to a multiple of 32 floats and c is a multiple of
        // 16, so the row segments are 64-byte aligned: 256-bit accesses, one
        // whole sector per thread
        float vv[16];
        if (p.epi_stage) {
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const float4 v4 = reinterpret_cast<const float4*>(eseg + 16 * ch)[i];
            vv[4 * i] = v4.x;
            vv[4 * i + 1] = v4.y;
            vv[4 * i + 2] = v4.z;
            vv[4 * i + 3] = v4.w;
          }
        } else {
          ld_global_v8(erow + c, vv);
          ld_global_v8(erow + c + 8, vv + 8);
        }
        if (EPI == TEPI_RATIO) {
          float* q = vv;     // Q = V / Vhat over V's registers, the bound terms over x16's
          float* vl = x16;
          // the bound's terms V log Vhat only on a sweep that forms them
          const bool want_l = p.bpart != nullptr;
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const float v = vv[i], x = x16[i];
            float qq = 0.f, l = 0.f;
            if (v > 0.f) {
              if (x > 0.f && isfinite(x)) {
                qq = v / x;
                if (want_l) l = v * logf(x);
              } else {
                bad |= ERR_VHAT_ZERO;
              }
            }
            q[i] = qq;
            vl[i] = l;
          }
          if (want_l) {
            // pairwise sum of the 16 terms in float, then into the double partial
#pragma unroll
            for (int w = 8; w > 0; w >>= 1)
#pragma unroll
              for (int i = 0; i < w; ++i) vl[i] += vl[i + w];
            part += (double)vl[0];
          }
          if (KIND == KIND_TF32X3) {
            float* hp = p.out_f32 + (size_t)t * p.ldo + c;
            float* lp = p.out_lo + (size_t)t * p.ldo + c;
#pragma unroll
            for (int i = 0; i < 2; ++i) {
              float h[8], l[8];
#pragma unroll
              for (int u = 0; u < 8; ++u) {
                h[u] = tf32_hi(q[8 * i + u]);
                l[u] = tf32_hi(q[8 * i + u] - h[u]);
              }
              st_global_v8(hp + 8 * i, h);
              st_global_v8(lp + 8 * i, l);
            }
          } else {
            uint32_t u[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
              const __nv_bfloat162 b2 = __floats2bfloat162_rn(q[2 * k], q[2 * k + 1]);
              u[k] = *reinterpret_cast<const uint32_t*>(&b2);
            }
            st_global_v8(static_cast<void*>(p.out_bf16 + (size_t)t * p.ldo + c), u);
          }
        } else {
          float* op = p.out_f32 + (size_t)t * p.ldo + c;
          float o[16];
#pragma unroll
          for (int i = 0; i < 16; ++i) o[i] = vv[i] * x16[i];
          st_global_v8(op, o);
          st_global_v8(op + 8, o + 8);
        }
      }
      if (EPI == TEPI_RATIO && p.bpart && rv)
        p.bpart[(size_t)t * p.nbpart + 2 * (tile % ncol) + half] = part;
      if (bad) atomicOr(p.err, bad);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, Cfg::TMEM_COLS);
  }
}

// ---------------------------------------------------------------- host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

thread_local std::string g_tc_err;

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

bool make_map(CUtensorMap* m, const void* base, int elem_bytes, int inner, int outer, int ld,
              int box_inner, int box_outer) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) {
    g_tc_err = "cuTensorMapEncodeTiled unavailable";
    return false;
  }
  const cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * elem_bytes};
  const cuuint32_t box[2] = {(cuuint32_t)box_inner, (cuuint32_t)box_outer};
  const cuuint32_t es[2] = {1, 1};
  const CUresult r = fn(m, elem_bytes == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                           : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                        2, const_cast<void*>(base), dims, strides, box, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    g_tc_err = "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")";
    return false;
  }
  return true;
}

constexpr int kMaxDevices = 64;

// Per device: the SM count, and whether a kernel's shared-memory opt-in has
// been made there (function attributes are per device).
int sm_count(int dev) {
  static int sms[kMaxDevices] = {};
  if (dev < 0 || dev >= kMaxDevices) return 1;
  if (sms[dev] == 0) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1)
      n = 1;
    sms[dev] = n;
  }
  return sms[dev];
}

template <int KIND, int BN, int EPI>
cudaError_t launch_gemm(const Maps& maps, TcArgs a, cudaStream_t st, int reserve = 0) {
  using Cfg = TileCfg<KIND, BN>;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  const int deepest = a.epi_stage ? Cfg::MAX_STAGES_EPI : Cfg::MAX_STAGES;
  if (deepest < 2) return cudaErrorInvalidValue;   // no room for a staged epilogue operand
  if (a.stages < 2 || a.stages > deepest) a.stages = deepest;
  static cudaError_t attr[kMaxDevices];
  static bool attr_set[kMaxDevices] = {};
  if (!attr_set[dev]) {
    attr[dev] = cudaFuncSetAttribute(k_tc_gemm<KIND, BN, EPI>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     SMEM_BUDGET);
    attr_set[dev] = true;
  }
  if (attr[dev] != cudaSuccess) return attr[dev];
  const int sms = sm_count(dev);
  const long long tiles = (long long)((a.cols + BN - 1) / BN) * ((a.rows + BM - 1) / BM);
  if (tiles == 0) return cudaSuccess;
  // persistent: one CTA per SM, less the SMs reserved (at most half of them)
  const int avail = sms - (reserve < sms / 2 ? reserve : sms / 2);
  const int grid = (int)(tiles < avail ? tiles : avail);
  k_tc_gemm<KIND, BN, EPI><<<grid, NUM_THREADS, Cfg::smem(a.stages, a.epi_stage != 0), st>>>(
      maps, a);
  return cudaGetLastError();
}

// The column tiles the tile-shape tuner may choose, per contraction and kind.
// FP32 (split TF32) keeps at least two accumulators for the hi*hi products
// (BN <= 160); BF16 may take wider tiles.
template <int EPI, int KIND>
cudaError_t launch_tile(int bn, const Maps& maps, const TcArgs& a, cudaStream_t st, int reserve) {
  switch (bn) {
    case 64: return launch_gemm<KIND, 64, EPI>(maps, a, st, reserve);
    case 96: return launch_gemm<KIND, 96, EPI>(maps, a, st, reserve);
    case 128: return launch_gemm<KIND, 128, EPI>(maps, a, st, reserve);
    case 160:
      if (EPI == TEPI_SCALE) return launch_gemm<KIND, 160, EPI>(maps, a, st, reserve);
      break;
    case 192:
      if (KIND == KIND_BF16) return launch_gemm<KIND, 192, EPI>(maps, a, st, reserve);
      break;
    default: break;
  }
  return cudaErrorInvalidValue;
}

template <int KIND>
int max_stages(int bn, bool epi) {
  switch (bn) {
    case 64: return epi ? TileCfg<KIND, 64>::MAX_STAGES_EPI : TileCfg<KIND, 64>::MAX_STAGES;
    case 96: return epi ? TileCfg<KIND, 96>::MAX_STAGES_EPI : TileCfg<KIND, 96>::MAX_STAGES;
    case 128: return epi ? TileCfg<KIND, 128>::MAX_STAGES_EPI : TileCfg<KIND, 128>::MAX_STAGES;
    case 160: return epi ? TileCfg<KIND, 160>::MAX_STAGES_EPI : TileCfg<KIND, 160>::MAX_STAGES;
    case 192: return epi ? TileCfg<KIND, 192>::MAX_STAGES_EPI : TileCfg<KIND, 192>::MAX_STAGES;
    default: return 0;
  }
}

}  // namespace

bool tc_available() {
  int dev = 0, major = 0, minor = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  return major == 10 && minor == 3 && encode_fn() != nullptr;
}

std::string tc_last_error() { return g_tc_err; }

// bound partials per frame: one per (column tile, epilogue half)
int tc_col_tiles_gemm1(int Fp) { return 2 * ((Fp + BN1 - 1) / BN1); }

static Maps* maps_of(TcPlan& p, int which) {
  return reinterpret_cast<Maps*>(&p.maps[which * 4][0]);
}

// The tile shapes the tuner chooses from: column tiles of each contraction
// (its output columns per 128-row tile) for each kind.
static const int kTilesF32[2][4] = {{64, 96, 128, 0}, {64, 96, 128, 160}};
static const int kTilesBF16[2][5] = {{64, 96, 128, 192, 0}, {64, 96, 128, 160, 192}};

int tc_tile_candidates(int precision, int which, int* out, int max_out) {
  int n = 0;
  const int* list = precision == 1 ? kTilesBF16[which] : kTilesF32[which];
  const int len = precision == 1 ? 5 : 4;
  for (int i = 0; i < len && n < max_out; ++i)
    if (list[i]) out[n++] = list[i];
  return n;
}

int tc_max_stages(int precision, int bn, bool epi) {
  return precision == 1 ? max_stages<KIND_BF16>(bn, epi) : max_stages<KIND_TF32X3>(bn, epi);
}

int tc_bpart_columns_max(int Fp) { return 2 * ((Fp + 63) / 64); }
int tc_bpart_used(const TcPlan& p) { return 2 * ((p.Fp + p.bn1 - 1) / p.bn1); }

// (Re)encode the B operands' tensor maps for the plan's column tiles.
static bool encode_b_maps(TcPlan& p) {
  const bool bf = p.precision == 1;
  const int es = bf ? 2 : 4;
  const int bk = bf ? KindCfg<KIND_BF16>::BK : KindCfg<KIND_TF32X3>::BK;
  Maps* m1 = maps_of(p, 0);
  Maps* m2 = maps_of(p, 1);
  bool ok = make_map(&m1->b_hi, p.bF_hi, es, p.Mp, p.Fp, p.Mp, bk, p.bn1) &&
            make_map(&m2->b_hi, p.bM_hi, es, p.Fp, p.Mp, p.Fp, bk, p.bn2);
  if (ok && !bf)
    ok = make_map(&m1->b_lo, p.bF_lo, es, p.Mp, p.Fp, p.Mp, bk, p.bn1) &&
         make_map(&m2->b_lo, p.bM_lo, es, p.Fp, p.Mp, p.Fp, bk, p.bn2);
  if (ok && bf) {  // unused lo maps: copies of hi (never read)
    m1->b_lo = m1->b_hi;
    m2->b_lo = m2->b_hi;
  }
  return ok;
}

int tc_set_tiles(TcPlan& p, int bn1, int bn2, int st1, int st2, int ep1, int ep2) {
  int c1[8], c2[8];
  const int n1 = tc_tile_candidates(p.precision, 0, c1, 8);
  const int n2 = tc_tile_candidates(p.precision, 1, c2, 8);
  bool ok1 = false, ok2 = false;
  for (int i = 0; i < n1; ++i) ok1 |= c1[i] == bn1;
  for (int i = 0; i < n2; ++i) ok2 |= c2[i] == bn2;
  if (!ok1 || !ok2) {
    g_tc_err = "column tile not among the tuner's shapes for this precision";
    return -1;
  }
  const int m1 = tc_max_stages(p.precision, bn1, ep1 != 0);
  const int m2 = tc_max_stages(p.precision, bn2, ep2 != 0);
  if (m1 < 2 || m2 < 2) {
    g_tc_err = "no room for a staged epilogue operand beside a two-stage ring at this tile";
    return -1;
  }
  if ((st1 != 0 && (st1 < 2 || st1 > m1)) || (st2 != 0 && (st2 < 2 || st2 > m2))) {
    g_tc_err = "ring depth must be 0 (deepest) or 2.." + std::to_string(m1) + " / " +
               std::to_string(m2);
    return -1;
  }
  const int o1 = p.bn1, o2 = p.bn2;
  p.bn1 = bn1;
  p.bn2 = bn2;
  if (!encode_b_maps(p)) {
    p.bn1 = o1;
    p.bn2 = o2;
    encode_b_maps(p);
    return -1;
  }
  p.st1 = st1;
  p.st2 = st2;
  p.ep1 = ep1 != 0;
  p.ep2 = ep2 != 0;
  return 0;
}

int tc_plan(TcPlan& p, int precision, int T, int M, int Mp, int F, int Fp, const float* V,
            const float* WM, const float* WF, const float* w32, float* Q, float* c, unsigned* err,
            cudaStream_t st) {
  (void)WM;
  (void)WF;
  (void)Q;
  (void)st;
  static_assert(sizeof(TcPlan::maps) >= 8 * sizeof(CUtensorMap), "tensor map storage");
  p.precision = precision;
  p.T = T;
  p.M = M;
  p.Mp = Mp;
  p.F = F;
  p.Fp = Fp;
  p.V = V;
  p.w32 = w32;
  p.c = c;
  p.err = err;
  const bool bf = precision == 1;
  p.w_format = bf ? WF_BF16 : WF_TF32X2;
  const int es = bf ? 2 : 4;
  const int bk = bf ? KindCfg<KIND_BF16>::BK : KindCfg<KIND_TF32X3>::BK;
  auto alloc = [&](void** ptr, size_t bytes) {
    cudaError_t e = cudaMalloc(ptr, bytes);
    if (e != cudaSuccess) {
      g_tc_err = std::string("cudaMalloc: ") + cudaGetErrorString(e);
      return false;
    }
    cudaMemset(*ptr, 0, bytes);
    return true;
  };
  const size_t tM = (size_t)T * Mp * es, tF = (size_t)T * Fp * es, MF = (size_t)Mp * Fp * es;
  if (!alloc(&p.w_hi, tM) || !alloc(&p.q_hi, tF) || !alloc(&p.bF_hi, MF) || !alloc(&p.bM_hi, MF))
    return -1;
  if (!bf && (!alloc(&p.w_lo, tM) || !alloc(&p.q_lo, tF) || !alloc(&p.bF_lo, MF) ||
              !alloc(&p.bM_lo, MF)))
    return -1;
  Maps* m1 = maps_of(p, 0);
  Maps* m2 = maps_of(p, 1);
  bool ok = make_map(&m1->a_hi, p.w_hi, es, Mp, T, Mp, bk, BM) &&
            make_map(&m2->a_hi, p.q_hi, es, Fp, T, Fp, bk, BM);
  if (ok && !bf)
    ok = make_map(&m1->a_lo, p.w_lo, es, Mp, T, Mp, bk, BM) &&
         make_map(&m2->a_lo, p.q_lo, es, Fp, T, Fp, bk, BM);
  if (!ok) return -1;
  if (bf) {  // unused lo maps: copies of hi (never read)
    m1->a_lo = m1->a_hi;
    m2->a_lo = m2->a_hi;
  }
  p.bn1 = BN1;
  p.bn2 = BN2;
  p.st1 = p.st2 = 0;
  if (!encode_b_maps(p)) return -1;
  p.bF_src = WF;
  p.bM_src = WM;
  return 0;
}

int tc_refresh_beta(TcPlan& p, cudaStream_t st) {
  const size_t n = (size_t)p.Mp * p.Fp;
  if (p.precision == 1) {
    launch_to_bf16(p.bF_src, p.bF_hi, n, st);
    launch_to_bf16(p.bM_src, p.bM_hi, n, st);
  } else {
    launch_split_tf32(p.bF_src, (float*)p.bF_hi, (float*)p.bF_lo, n, st);
    launch_split_tf32(p.bM_src, (float*)p.bM_hi, (float*)p.bM_lo, n, st);
  }
  return 2;
}

int tc_gemm1(TcPlan& p, int row_off, int rows, double* bpart, int reserve, cudaStream_t st) {
  TcArgs a{};
  a.inject_wait_ns = p.inject_wait_ns;   // one-shot test hook
  p.inject_wait_ns = 0;
  a.rows = rows;
  a.row_off = row_off;
  a.cols = p.Fp;
  a.kdim = p.Mp;
  a.nbpart = p.nbpart;
  a.V = p.V;
  a.ldv = p.Fp;
  a.ldo = p.Fp;
  a.bpart = bpart;
  a.err = p.err;
  cudaError_t e;
  a.stages = p.st1;
  a.prefetch = p.pf1;
  a.epi_stage = p.ep1;
  if (p.precision == 1) {
    a.out_bf16 = reinterpret_cast<__nv_bfloat16*>(p.q_hi);
    e = launch_tile<TEPI_RATIO, KIND_BF16>(p.bn1, *maps_of(p, 0), a, st, reserve);
  } else {
    a.out_f32 = reinterpret_cast<float*>(p.q_hi);
    a.out_lo = reinterpret_cast<float*>(p.q_lo);
    e = launch_tile<TEPI_RATIO, KIND_TF32X3>(p.bn1, *maps_of(p, 0), a, st, reserve);
  }
  if (e != cudaSuccess) {
    g_tc_err = cudaGetErrorString(e);
    return -1;
  }
  return 1;
}

int tc_gemm2(TcPlan& p, int row_off, int rows, int reserve, cudaStream_t st) {
  TcArgs a{};
  a.rows = rows;
  a.row_off = row_off;
  a.cols = p.Mp;
  a.kdim = p.Fp;
  a.w = p.w32;
  a.ldw = p.Mp;
  a.out_f32 = p.c;
  a.ldo = p.Mp;
  a.err = p.err;
  cudaError_t e;
  a.stages = p.st2;
  a.prefetch = p.pf2;
  a.epi_stage = p.ep2;
  if (p.precision == 1)
    e = launch_tile<TEPI_SCALE, KIND_BF16>(p.bn2, *maps_of(p, 1), a, st, reserve);
  else
    e = launch_tile<TEPI_SCALE, KIND_TF32X3>(p.bn2, *maps_of(p, 1), a, st, reserve);
  if (e != cudaSuccess) {
    g_tc_err = cudaGetErrorString(e);
    return -1;
  }
  return 1;
}

int tc_exact_plan(ExactTc& p) {
  const bool bf = p.precision == 1;
  p.w_format = bf ? WF_BF16 : WF_TF32X2;
  const int es = bf ? 2 : 4;
  const int bk = bf ? KindCfg<KIND_BF16>::BK : KindCfg<KIND_TF32X3>::BK;
  auto alloc = [&](void** ptr, size_t bytes) {
    cudaError_t e = cudaMalloc(ptr, bytes);
    if (e != cudaSuccess) {
      g_tc_err = std::string("cudaMalloc: ") + cudaGetErrorString(e);
      return false;
    }
    cudaMemset(*ptr, 0, bytes);
    return true;
  };
  const size_t rows = (size_t)p.NC * p.Tp;
  const size_t th = rows * p.SKp * es, q = rows * p.Fp * es, b = (size_t)p.NC * p.Fp * p.SKp * es;
  if (!alloc(&p.th_hi, th) || !alloc(&p.q_hi, q) || !alloc(&p.b1_hi, b) || !alloc(&p.b2_hi, b))
    return -1;
  if (!bf && (!alloc(&p.th_lo, th) || !alloc(&p.q_lo, q) || !alloc(&p.b1_lo, b) ||
              !alloc(&p.b2_lo, b)))
    return -1;
  if (rows > (size_t)INT32_MAX || (size_t)p.NC * p.Fp > (size_t)INT32_MAX) {
    g_tc_err = "exact inference: too many rows for one tensor map";
    return -1;
  }
  Maps* m1 = reinterpret_cast<Maps*>(&p.maps[0][0]);
  Maps* m2 = reinterpret_cast<Maps*>(&p.maps[4][0]);
  bool ok = make_map(&m1->a_hi, p.th_hi, es, p.SKp, (int)rows, p.SKp, bk, BM) &&
            make_map(&m1->b_hi, p.b1_hi, es, p.SKp, p.NC * p.Fp, p.SKp, bk, BN1) &&
            make_map(&m2->a_hi, p.q_hi, es, p.Fp, (int)rows, p.Fp, bk, BM) &&
            make_map(&m2->b_hi, p.b2_hi, es, p.Fp, p.NC * p.SKp, p.Fp, bk, BNX);
  if (ok && !bf)
    ok = make_map(&m1->a_lo, p.th_lo, es, p.SKp, (int)rows, p.SKp, bk, BM) &&
         make_map(&m1->b_lo, p.b1_lo, es, p.SKp, p.NC * p.Fp, p.SKp, bk, BN1) &&
         make_map(&m2->a_lo, p.q_lo, es, p.Fp, (int)rows, p.Fp, bk, BM) &&
         make_map(&m2->b_lo, p.b2_lo, es, p.Fp, p.NC * p.SKp, p.Fp, bk, BNX);
  if (!ok) return -1;
  if (bf) {
    m1->a_lo = m1->a_hi;
    m1->b_lo = m1->b_hi;
    m2->a_lo = m2->a_hi;
    m2->b_lo = m2->b_hi;
  }
  p.nbpart = tc_col_tiles_gemm1(p.Fp);
  return 0;
}

int tc_exact_gemm1(ExactTc& p, cudaStream_t st) {
  TcArgs a{};
  a.rows = p.NC * p.Tp;
  a.cols = p.Fp;
  a.kdim = p.SKp;
  a.nbpart = p.nbpart;
  a.V = p.V;
  a.ldv = p.Fp;
  a.ldo = p.Fp;
  a.bpart = p.bpart;
  a.err = p.err;
  a.brows = p.Tp;
  a.bvalid = p.T;
  a.bstride = p.Fp;
  const Maps& m = *reinterpret_cast<const Maps*>(&p.maps[0][0]);
  cudaError_t e;
  if (p.precision == 1) {
    a.out_bf16 = reinterpret_cast<__nv_bfloat16*>(p.q_hi);
    e = launch_gemm<KIND_BF16, BN1, TEPI_RATIO>(m, a, st);
  } else {
    a.out_f32 = reinterpret_cast<float*>(p.q_hi);
    a.out_lo = reinterpret_cast<float*>(p.q_lo);
    e = launch_gemm<KIND_TF32X3, BN1, TEPI_RATIO>(m, a, st);
  }
  if (e != cudaSuccess) {
    g_tc_err = cudaGetErrorString(e);
    return -1;
  }
  return 1;
}

int tc_exact_gemm2(ExactTc& p, cudaStream_t st) {
  TcArgs a{};
  a.rows = p.NC * p.Tp;
  a.cols = p.SKp;
  a.kdim = p.Fp;
  a.w = p.th32;
  a.ldw = p.SKp;
  a.out_f32 = p.out;
  a.ldo = p.SKp;
  a.err = p.err;
  a.brows = p.Tp;
  a.bvalid = p.T;
  a.bstride = p.SKp;
  const Maps& m = *reinterpret_cast<const Maps*>(&p.maps[4][0]);
  cudaError_t e;
  if (p.precision == 1)
    e = launch_gemm<KIND_BF16, BNX, TEPI_SCALE>(m, a, st);
  else
    e = launch_gemm<KIND_TF32X3, BNX, TEPI_SCALE>(m, a, st);
  if (e != cudaSuccess) {
    g_tc_err = cudaGetErrorString(e);
    return -1;
  }
  return 1;
}

void tc_exact_free(ExactTc& p) {
  void* bufs[] = {p.th_hi, p.th_lo, p.q_hi, p.q_lo, p.b1_hi, p.b1_lo, p.b2_hi, p.b2_lo};
  for (void* b : bufs)
    if (b) cudaFree(b);
  p.th_hi = p.th_lo = p.q_hi = p.q_lo = p.b1_hi = p.b1_lo = p.b2_hi = p.b2_lo = nullptr;
}

void tc_free(TcPlan& p) {
  void* bufs[] = {p.w_hi, p.w_lo, p.q_hi, p.q_lo, p.bF_hi, p.bF_lo, p.bM_hi, p.bM_lo};
  for (void* b : bufs)
    if (b) cudaFree(b);
  p.w_hi = p.w_lo = p.q_hi = p.q_lo = p.bF_hi = p.bF_lo = p.bM_hi = p.bM_lo = nullptr;
}

}  // namespace nfhmm
