// Measured rate of this GPU's tcgen05 tensor cores: the denominator of the
// contractions' roofline.  Every SM issues back-to-back 128 x 256 MMAs from
// one K-block of operands in shared memory into one TMEM accumulator (the
// shape of the contraction kernels' MMAs at their widest), and the host times
// the launch with CUDA events.  The operands are zeros: the rate of an MMA
// does not depend on the values it multiplies.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/nfhmm.h"
#include "nfhmm_kernels.h"
#include "nfhmm_tc.h"
#include "tc_ptx.cuh"

namespace nfhmm {
namespace {

using namespace tc;

constexpr int RATE_BM = 128, RATE_BN = 256;
constexpr int RATE_A_BYTES = RATE_BM * 128, RATE_B_BYTES = RATE_BN * 128;
constexpr int RATE_SMEM_USED = RATE_A_BYTES + RATE_B_BYTES + 1024 + 64;
// asked for at launch: more than half of an SM's shared memory, so that
// exactly one block runs on each SM
constexpr int RATE_SMEM = 120 * 1024;
static_assert(RATE_SMEM >= RATE_SMEM_USED, "probe shared memory");
constexpr int RATE_MMAS_PER_REP = 4;   // 128 bytes of K per row, 32 bytes per instruction

template <int KIND>
__global__ void __launch_bounds__(128, 1) k_mma_rate(int reps, unsigned* err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint8_t* a = smem;
  uint8_t* b = smem + RATE_A_BYTES;
  uint64_t* done = reinterpret_cast<uint64_t*>(b + RATE_B_BYTES);
  uint32_t* slot = reinterpret_cast<uint32_t*>(done + 1);
  const int warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < (RATE_A_BYTES + RATE_B_BYTES) / 16; i += blockDim.x)
    reinterpret_cast<int4*>(smem)[i] = make_int4(0, 0, 0, 0);
  fence_proxy_async_smem();   // the zeros are read by the tensor cores (async proxy)
  if (threadIdx.x == 0) {
    mbar_init(done, 1);
    fence_barrier_init();
  }
  if (warp == 0) {
    tmem_alloc(slot, RATE_BN);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;
  if (threadIdx.x == 0) {
    constexpr uint32_t ID = idesc<KIND>(RATE_BM, RATE_BN);
    const uint32_t a0 = smem_u32(a), b0 = smem_u32(b);
    for (int r = 0; r < reps; ++r) {
#pragma unroll
      for (int kk = 0; kk < RATE_MMAS_PER_REP; ++kk)
        mma<KIND>(tmem, sdesc(a0 + 32 * kk), sdesc(b0 + 32 * kk), ID, (r > 0 || kk > 0) ? 1u : 0u);
    }
    mma_commit(done);
    if (!mbar_wait(done, 0)) atomicOr(err, ERR_TIMEOUT);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, RATE_BN);
  }
}

template <int KIND>
cudaError_t launch_rate(int grid, int reps, unsigned* err, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(k_mma_rate<KIND>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, RATE_SMEM);
  if (e != cudaSuccess) return e;
  k_mma_rate<KIND><<<grid, 128, RATE_SMEM, st>>>(reps, err);
  return cudaGetLastError();
}

}  // namespace
}  // namespace nfhmm

extern "C" {

int nfhmm_mma_rate(int precision, double* tflops_out, void* cuda_stream) {
  using namespace nfhmm;
  if (!tflops_out) {
    set_last_error("NULL argument");
    return NFHMM_EINVAL;
  }
  if (precision != NFHMM_FP32 && precision != NFHMM_BF16) {
    set_last_error("precision must be NFHMM_FP32 (tf32 MMAs) or NFHMM_BF16");
    return NFHMM_EINVAL;
  }
  if (!tc_available()) {
    set_last_error("the tensor-core rate needs an sm_103 device");
    return NFHMM_EINVAL;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  unsigned* err = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaMalloc(&err, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(unsigned), st);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  // about 1 ms per launch at the tensor peak (an instruction is 128 cycles)
  const int reps = 4000, timed = 5;
  auto launch = [&]() {
    return precision == NFHMM_FP32 ? launch_rate<KIND_TF32X3>(sms, reps, err, st)
                                   : launch_rate<KIND_BF16>(sms, reps, err, st);
  };
  if (e == cudaSuccess) e = launch();   // warm-up
  if (e == cudaSuccess) e = cudaEventRecord(e0, st);
  for (int i = 0; i < timed && e == cudaSuccess; ++i) e = launch();
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  unsigned h_err = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&h_err, err, sizeof(unsigned), cudaMemcpyDeviceToHost);
  if (err) cudaFree(err);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) {
    set_last_error(std::string("nfhmm_mma_rate: ") + cudaGetErrorString(e));
    return NFHMM_ECUDA;
  }
  if (h_err) {
    set_last_error("nfhmm_mma_rate: a bounded device wait gave up");
    return NFHMM_ETIMEOUT;
  }
  const double k = precision == NFHMM_FP32 ? 8.0 : 16.0;   // K per instruction
  const double macs = (double)sms * timed * reps * RATE_MMAS_PER_REP * RATE_BM * RATE_BN * k;
  *tflops_out = 2.0 * macs / (ms * 1e-3) / 1e12;
  return NFHMM_OK;
}

}  // extern "C"
