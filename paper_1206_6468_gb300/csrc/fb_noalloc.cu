// Forward-backward entry point that performs no device allocation.
//
// Some callers cannot allocate device memory when they call in: a process
// whose device memory is reserved up front by another allocator (a serving
// runtime with a fixed HBM budget, a host framework that owns every byte),
// or a latency-critical thread that must not hit cudaMalloc/cudaFree, which
// can block and synchronise the whole device.  For them this variant of
// nfhmm_forward_backward keeps its scratch (chunk matrices, boundary vectors,
// scale factors, error word) in one fixed array of device memory compiled
// into the library.  Every GPU that loads the library holds that array until
// the process exits; the caller still passes its own inputs and outputs.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/nfhmm.h"
#include "nfhmm_kernels.h"

namespace {

static __device__ __align__(256) unsigned char g_fb_scratch[NFHMM_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};  // device address of g_fb_scratch, per device

int fail(int code, const std::string& m) {
  nfhmm::set_last_error(m);
  return code;
}

// One-time set-up per device, with that device current: the host-side name
// g_fb_scratch is only a stand-in, so the device address is looked up here
// and handed to the kernels.
int scratch_address(int dev, void** out) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_fb_scratch);
    if (e != cudaSuccess)
      return fail(NFHMM_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return NFHMM_OK;
}

}  // namespace

extern "C" {

// Declared in include/nfhmm.h; a failure's message is what nfhmm_last_error
// returns on the calling thread.
int nfhmm_forward_backward_noalloc(int S, int N, int T, const float* phi, const float* A,
                                   const float* pi, float* dhat, double* logZ, int chunk_len,
                                   void* cuda_stream) {
  using namespace nfhmm;
  if (!phi || !A || !pi || !dhat || !logZ) return fail(NFHMM_EINVAL, "NULL argument");
  if (S < 1 || N < 1 || T < 1) return fail(NFHMM_EINVAL, "S, N, T must be >= 1");
  if (N > fb_max_states())
    return fail(NFHMM_EINVAL, "N must be <= " + std::to_string(fb_max_states()));
  FBArgs a{};
  a.S = S;
  a.N = N;
  a.T = T;
  a.L = chunk_len <= 0 ? fb_default_chunk(N, T) : chunk_len;
  if (a.L > 128) a.L = 128;
  if (a.L > T) a.L = T;
  a.C = (T + a.L - 1) / a.L;
  a.nchains = 1;   // one chain over all T frames (null chain tables)
  a.products = FB_PRODUCTS_TC;
  a.G = fb_default_group(a.C);
  a.NG = a.G >= 2 ? (a.C + a.G - 1) / a.G : 0;
  const size_t need = fb_scratch_bytes(S, N, a.C, a.NG) + 256;  // + error word
  if (need > (size_t)NFHMM_NOALLOC_SCRATCH_BYTES)
    return fail(NFHMM_EINVAL, "problem needs " + std::to_string(need) +
                                  " bytes of scratch; the fixed array holds " +
                                  std::to_string((size_t)NFHMM_NOALLOC_SCRATCH_BYTES));
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(NFHMM_ECUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(NFHMM_EINVAL, "device index out of range");
  void* base = nullptr;
  int rc = scratch_address(dev, &base);
  if (rc) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  a.phi = phi;
  a.A = A;
  a.pi = pi;
  a.dhat = dhat;
  a.logZ = logZ;
  fb_carve_scratch(a, base);
  a.err = reinterpret_cast<unsigned*>(reinterpret_cast<char*>(base) + need - 256);
  // the array keeps the previous call's contents: the error word must start at
  // zero; every other scratch word is written before it is read
  e = cudaMemsetAsync(a.err, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return fail(NFHMM_ECUDA, cudaGetErrorString(e));
  e = launch_fb(a, st, nullptr);
  if (e != cudaSuccess) return fail(NFHMM_ECUDA, cudaGetErrorString(e));
  // the error word stays in the shared array: a set word turns logZ into NaN
  launch_flag_errors(a.err, logZ, S, st);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(NFHMM_ECUDA, cudaGetErrorString(e));
  return NFHMM_OK;
}

}  // extern "C"
