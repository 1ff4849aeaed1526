// FP32 SIMT form of the two contractions of Eq. 7 (used for the initial
// state, for separation, and as the CUDA-core path):
//   reconstruction   Vhat[t][l] = sum_k w[t][k] beta[l][k]      (+ ratio epilogue)
//   back-projection  R[t][k]    = sum_l Q[t][l] beta[k][l]      (+ scale epilogue)
// Both are C[r][c] = sum_k A[r][k] B[c][k] with K contiguous in both operands.
// Tile 128 x 64 x 16, 256 threads, 8 x 4 outputs per thread, operands staged
// through shared memory (k-major) with a register prefetch of the next tile.
#include <math.h>

#include "nfhmm_device.cuh"
#include "nfhmm_kernels.h"

namespace nfhmm {

namespace {
constexpr int BM = 128, BN = 64, BK = 16;
}

int gemm_simt_col_tiles(int cols) { return (cols + BN - 1) / BN; }

template <int EPI>
__global__ void __launch_bounds__(256) k_gemm_simt(GemmArgs g) {
  __shared__ float As[BK][BM + 4];
  __shared__ float Bs[BK][BN + 4];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int row0 = blockIdx.y * BM, col0 = blockIdx.x * BN;

  // global -> register prefetch assignment
  const int ar = tid >> 1, ak = (tid & 1) * 8;  // A: 128 rows x 16 k, 8 per thread
  const int br = tid >> 2, bk = (tid & 3) * 4;  // B: 64 rows x 16 k, 4 per thread
  float ra[8], rb[4];
  auto load = [&](int k0) {
    const int r = row0 + ar;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int k = k0 + ak + i;
      ra[i] = (r < g.rows && k < g.kdim) ? g.A[(size_t)r * g.lda + k] : 0.f;
    }
    const int c = col0 + br;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int k = k0 + bk + i;
      rb[i] = (c < g.cols && k < g.kdim) ? g.B[(size_t)c * g.ldb + k] : 0.f;
    }
  };
  float acc[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;

  load(0);
  for (int k0 = 0; k0 < g.kdim; k0 += BK) {
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 8; ++i) As[ak + i][ar] = ra[i];
#pragma unroll
    for (int i = 0; i < 4; ++i) Bs[bk + i][br] = rb[i];
    __syncthreads();
    if (k0 + BK < g.kdim) load(k0 + BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[kk][ty * 8]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[kk][ty * 8 + 4]);
      const float4 b = *reinterpret_cast<const float4*>(&Bs[kk][tx * 4]);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
  }

  unsigned bad = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int r = row0 + ty * 8 + i;
    double part = 0.0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = col0 + tx * 4 + j;
      if (r < g.rows && c < g.cols) {
        const float x = acc[i][j];
        if (EPI == EPI_RATIO) {
          const float v = g.V[(size_t)r * g.ldv + c];
          float q = 0.f;
          if (v > 0.f) {
            if (x > 0.f && isfinite(x)) {
              q = v / x;
              if (g.bpart) part += (double)v * (double)logf(x);   // only when the bound is formed
            } else {
              bad |= ERR_VHAT_ZERO;
            }
          }
          g.out[(size_t)r * g.ldo + c] = q;
        } else if (EPI == EPI_SCALE) {
          g.out[(size_t)r * g.ldo + c] = g.w[(size_t)r * g.ldw + c] * x;
        } else {
          g.out[(size_t)r * g.ldo + c] = x;
        }
      }
    }
    if (EPI == EPI_RATIO && g.bpart) {
      // the 16 threads sharing this row are lanes with equal ty within a warp
#pragma unroll
      for (int o = 1; o < 16; o <<= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
      if (tx == 0 && r < g.rows) g.bpart[(size_t)r * g.nbpart + blockIdx.x] = part;
    }
  }
  if (EPI == EPI_RATIO) {
    bad = __reduce_or_sync(0xffffffffu, bad);
    if (bad && (tid & 31) == 0) atomicOr(g.err, bad);
  }
}

void launch_gemm_simt(const GemmArgs& g, int epi, cudaStream_t st) {
  dim3 grid((g.cols + BN - 1) / BN, (g.rows + BM - 1) / BM);
  switch (epi) {
    case EPI_RATIO: k_gemm_simt<EPI_RATIO><<<grid, 256, 0, st>>>(g); break;
    case EPI_SCALE: k_gemm_simt<EPI_SCALE><<<grid, 256, 0, st>>>(g); break;
    default: k_gemm_simt<EPI_STORE><<<grid, 256, 0, st>>>(g); break;
  }
}

}  // namespace nfhmm
