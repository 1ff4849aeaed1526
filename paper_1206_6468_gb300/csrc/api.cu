// C ABI of the N-FHMM variational-inference library (see include/nfhmm.h).
// Host code: context and device buffers, stream ordering, the sweep loop,
// bound, separation, checkpoint and profiling.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <string>
#include <vector>

#include "../../include/nfhmm.h"
#include "nfhmm_kernels.h"
#include "nfhmm_tc.h"

using namespace nfhmm;

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

}  // namespace

void nfhmm::set_last_error(const std::string& msg) { g_last_error = msg; }

namespace {

#define CK(call)                                                                       \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) {                                                           \
      return fail(e_ == cudaErrorMemoryAllocation ? NFHMM_ENOMEM : NFHMM_ECUDA,        \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                 \
    }                                                                                  \
  } while (0)

size_t round_up(size_t x, size_t m) { return (x + m - 1) / m * m; }

struct StageEvents {
  std::vector<cudaEvent_t> begin, end;
  long long launches = 0;
  size_t device_bytes = 0;
};

}  // namespace

struct nfhmm_ctx {
  nfhmm_dims d{};
  int M = 0, Mp = 0, Fp = 0, NK = 0;
  cudaStream_t user = nullptr, s_main = nullptr, s_aux = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr, ev_fork = nullptr, ev_join = nullptr;
  // device buffers
  float* V = nullptr;       // T x Fp
  float* WM = nullptr;      // Mp x Fp   (beta by element: W[k][l])
  float* WF = nullptr;      // Fp x Mp   (beta by frequency)
  float* A = nullptr;       // S x N x N
  float* pi = nullptr;      // S x N
  float* alpha = nullptr;   // T x Mp
  float* w32 = nullptr;     // T x Mp
  float* c = nullptr;       // T x Mp
  float* Q = nullptr;       // T x Fp
  float* phi = nullptr;     // S x T x N
  float* dhat = nullptr;    // S x T x N
  float* wts = nullptr;     // T x Mp (separation weights)
  float* sep_tmp = nullptr; // S x T x F (host-output separation)
  double* v = nullptr;      // T
  double* bpart = nullptr;  // T x nbpart
  int nbpart = 0;
  double* frame_terms = nullptr;  // T
  double* logZ = nullptr;   // S
  double* bound_dev = nullptr;
  unsigned* err = nullptr;
  int2* ktab = nullptr;      // Mp element table
  void* fb_scratch = nullptr;
  FBArgs fb{};
  TcPlan tc{};
  bool use_tc = false;
  double konst = 0.0;
  // host staging (pinned)
  double* h_bound = nullptr;
  unsigned* h_err = nullptr;
  int sweeps_done = 0;
  bool have_alpha = false;
  bool inputs_ok = false;
  bool profiling = false;
  StageEvents stages[NFHMM_NUM_STAGES];
  long long launches = 0;
  size_t device_bytes = 0;
};

namespace {

void stage_begin(nfhmm_ctx* c, int stage, cudaStream_t st) {
  if (!c->profiling) return;
  cudaEvent_t e;
  cudaEventCreate(&e);
  cudaEventRecord(e, st);
  c->stages[stage].begin.push_back(e);
}
void stage_end(nfhmm_ctx* c, int stage, cudaStream_t st, int launches) {
  c->launches += launches;
  c->stages[stage].launches += launches;
  if (!c->profiling) return;
  cudaEvent_t e;
  cudaEventCreate(&e);
  cudaEventRecord(e, st);
  c->stages[stage].end.push_back(e);
}

void free_ctx(nfhmm_ctx* c) {
  if (!c) return;
  if (c->s_main) cudaStreamSynchronize(c->s_main);
  if (c->s_aux) cudaStreamSynchronize(c->s_aux);
  void* bufs[] = {c->V, c->WM, c->WF, c->A, c->pi, c->alpha, c->w32, c->c, c->Q, c->phi,
                  c->dhat, c->wts, c->sep_tmp, c->v, c->bpart, c->frame_terms, c->logZ,
                  c->bound_dev, c->err, c->ktab, c->fb_scratch};
  for (void* p : bufs)
    if (p) cudaFree(p);
  tc_free(c->tc);
  if (c->h_bound) cudaFreeHost(c->h_bound);
  if (c->h_err) cudaFreeHost(c->h_err);
  for (auto& s : c->stages) {
    for (auto e : s.begin) cudaEventDestroy(e);
    for (auto e : s.end) cudaEventDestroy(e);
  }
  cudaEvent_t evs[] = {c->ev_in, c->ev_out, c->ev_fork, c->ev_join};
  for (auto e : evs)
    if (e) cudaEventDestroy(e);
  if (c->s_main) cudaStreamDestroy(c->s_main);
  if (c->s_aux) cudaStreamDestroy(c->s_aux);
  delete c;
}

// Order the context's streams after the user's stream (entry) and the
// user's stream after the context's work (exit).
int enter(nfhmm_ctx* c) {
  CK(cudaEventRecord(c->ev_in, c->user));
  CK(cudaStreamWaitEvent(c->s_main, c->ev_in, 0));
  return NFHMM_OK;
}
int leave(nfhmm_ctx* c) {
  CK(cudaEventRecord(c->ev_out, c->s_main));
  CK(cudaStreamWaitEvent(c->user, c->ev_out, 0));
  CK(cudaGetLastError());
  return NFHMM_OK;
}

cudaError_t dmalloc(nfhmm_ctx* c, void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaSuccess) c->device_bytes += bytes;
  return e;
}

// Synchronise the context and turn the device error word into a code.
int sync_check(nfhmm_ctx* c) {
  CK(cudaMemcpyAsync(c->h_err, c->err, sizeof(unsigned), cudaMemcpyDeviceToHost, c->s_main));
  CK(cudaStreamSynchronize(c->s_main));
  const unsigned e = *c->h_err;
  if (e) {
    cudaMemsetAsync(c->err, 0, sizeof(unsigned), c->s_main);
    cudaStreamSynchronize(c->s_main);
    if (e & ERR_TIMEOUT)
      return fail(NFHMM_ETIMEOUT, "a bounded device wait gave up (tensor-core pipeline)");
    if (e & ERR_BAD_INPUT)
      return fail(NFHMM_EINVAL,
                  "input validation failed: V must be finite and >= 0; rows of W, A and pi "
                  "must be >= 0 and sum to 1 within 1e-4");
    if (e & ERR_VHAT_ZERO)
      return fail(NFHMM_ENUMERIC, "reconstruction Vhat vanished where V > 0");
    if (e & ERR_NONFINITE) return fail(NFHMM_ENUMERIC, "non-finite value in alpha-hat or psi");
    if (e & ERR_FB_ZERO)
      return fail(NFHMM_ENUMERIC, "forward-backward normaliser vanished or was not finite");
    return fail(NFHMM_ENUMERIC, "device error word set");
  }
  return NFHMM_OK;
}

// Reconstruction + ratio (GEMM1) and back-projection + counts (GEMM2) from
// the weights in w32 (and the operand copies of the tensor-core path).
int contract(nfhmm_ctx* c, bool want_bpart, bool init) {
  const nfhmm_dims& d = c->d;
  cudaStream_t st = c->s_main;
  if (c->use_tc && !init) {
    stage_begin(c, NFHMM_STAGE_GEMM1, st);
    const int n1 = tc_gemm1(c->tc, want_bpart ? c->bpart : nullptr, st);
    if (n1 < 0) return fail(NFHMM_ECUDA, "tensor-core contraction: " + tc_last_error());
    stage_end(c, NFHMM_STAGE_GEMM1, st, n1);
    stage_begin(c, NFHMM_STAGE_GEMM2, st);
    const int n2 = tc_gemm2(c->tc, st);
    if (n2 < 0) return fail(NFHMM_ECUDA, "tensor-core contraction: " + tc_last_error());
    stage_end(c, NFHMM_STAGE_GEMM2, st, n2);
    return NFHMM_OK;
  }
  const int stage1 = init ? NFHMM_STAGE_INIT : NFHMM_STAGE_GEMM1;
  const int stage2 = init ? NFHMM_STAGE_INIT : NFHMM_STAGE_GEMM2;
  GemmArgs g1{};
  g1.rows = d.T;
  g1.cols = c->Fp;
  g1.kdim = c->Mp;
  g1.A = c->w32;
  g1.lda = c->Mp;
  g1.B = c->WF;
  g1.ldb = c->Mp;
  g1.V = c->V;
  g1.ldv = c->Fp;
  g1.out = c->Q;
  g1.ldo = c->Fp;
  g1.bpart = want_bpart ? c->bpart : nullptr;
  g1.nbpart = c->nbpart;
  g1.err = c->err;
  stage_begin(c, stage1, st);
  launch_gemm_simt(g1, EPI_RATIO, st);
  stage_end(c, stage1, st, 1);
  GemmArgs g2{};
  g2.rows = d.T;
  g2.cols = c->Mp;
  g2.kdim = c->Fp;
  g2.A = c->Q;
  g2.lda = c->Fp;
  g2.B = c->WM;
  g2.ldb = c->Fp;
  g2.out = c->c;
  g2.ldo = c->Mp;
  g2.w = c->w32;
  g2.ldw = c->Mp;
  g2.err = c->err;
  stage_begin(c, stage2, st);
  launch_gemm_simt(g2, EPI_SCALE, st);
  stage_end(c, stage2, st, 1);
  return NFHMM_OK;
}

int one_sweep(nfhmm_ctx* c, bool want_bpart) {
  const nfhmm_dims& d = c->d;
  WeightsArgs wa{};
  wa.T = d.T;
  wa.M = c->M;
  wa.Mp = c->Mp;
  wa.S = d.S;
  wa.N = d.N;
  wa.K = d.K;
  wa.gamma = (float)d.gamma;
  wa.ktab = c->ktab;
  wa.counts = c->c;
  wa.dhat = c->dhat;
  wa.alpha = c->alpha;
  wa.w32 = c->w32;
  wa.phi = c->phi;
  wa.err = c->err;
  int fmt = WF_F32;
  if (c->use_tc) {
    fmt = c->tc.w_format;
    wa.wop_hi = c->tc.w_hi;
    wa.wop_lo = c->tc.w_lo;
  }
  stage_begin(c, NFHMM_STAGE_WEIGHTS, c->s_main);
  launch_weights(wa, fmt, c->s_main);
  stage_end(c, NFHMM_STAGE_WEIGHTS, c->s_main, 1);
  // forward-backward on the aux stream, concurrent with the contractions
  CK(cudaEventRecord(c->ev_fork, c->s_main));
  CK(cudaStreamWaitEvent(c->s_aux, c->ev_fork, 0));
  stage_begin(c, NFHMM_STAGE_FB, c->s_aux);
  int nfb = 0;
  CK(launch_fb(c->fb, c->s_aux, &nfb));
  stage_end(c, NFHMM_STAGE_FB, c->s_aux, nfb);
  int rc = contract(c, want_bpart, false);
  if (rc) return rc;
  CK(cudaEventRecord(c->ev_join, c->s_aux));
  CK(cudaStreamWaitEvent(c->s_main, c->ev_join, 0));
  return NFHMM_OK;
}

int compute_bound(nfhmm_ctx* c, double* out) {
  BoundArgs b{};
  b.T = c->d.T;
  b.M = c->M;
  b.Mp = c->Mp;
  b.S = c->d.S;
  b.K = c->d.K;
  b.gamma = (float)c->d.gamma;
  b.konst = c->konst;
  b.alpha = c->alpha;
  b.v = c->v;
  b.bpart = c->bpart;
  b.nbpart = c->nbpart;
  b.logZ = c->logZ;
  b.frame_terms = c->frame_terms;
  b.out = c->bound_dev;
  stage_begin(c, NFHMM_STAGE_BOUND, c->s_main);
  int n = 0;
  launch_bound(b, c->s_main, &n);
  stage_end(c, NFHMM_STAGE_BOUND, c->s_main, n);
  CK(cudaMemcpyAsync(c->h_bound, c->bound_dev, sizeof(double), cudaMemcpyDeviceToHost,
                     c->s_main));
  int rc = sync_check(c);
  if (rc) return rc;
  *out = *c->h_bound;
  return NFHMM_OK;
}

int copy_out(void* dst, const void* src, size_t bytes, int on_device, cudaStream_t st) {
  CK(cudaMemcpyAsync(dst, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDefault,
                     st));
  return NFHMM_OK;
}

// Copy (V, W, A, pi) into the context's buffers, validate them, refresh the
// operand copies of beta and set the initial state (z-hat from equal weights,
// d-hat from init_mode).  Synchronises once.
int load_and_init(nfhmm_ctx* c, const float* V, const float* W, const float* A, const float* pi,
                  int on_device) {
  const nfhmm_dims& d = c->d;
  const size_t T = d.T, Mp = c->Mp, Fp = c->Fp, S = d.S, N = d.N;
  int rc = enter(c);
  if (rc) return rc;
  cudaStream_t st = c->s_main;
  CK(cudaMemsetAsync(c->err, 0, 4, st));
  CK(cudaMemsetAsync(c->V, 0, T * Fp * 4, st));
  CK(cudaMemsetAsync(c->WM, 0, Mp * Fp * 4, st));
  CK(cudaMemsetAsync(c->c, 0, T * Mp * 4, st));
  CK(cudaMemsetAsync(c->alpha, 0, T * Mp * 4, st));
  CK(cudaMemsetAsync(c->bpart, 0, T * c->nbpart * 8, st));
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDefault;
  CK(cudaMemcpy2DAsync(c->V, Fp * 4, V, (size_t)d.F * 4, (size_t)d.F * 4, T, kind, st));
  CK(cudaMemcpy2DAsync(c->WM, Fp * 4, W, (size_t)d.F * 4, (size_t)d.F * 4, (size_t)c->M, kind,
                       st));
  CK(cudaMemcpyAsync(c->A, A, S * N * N * 4, kind, st));
  CK(cudaMemcpyAsync(c->pi, pi, S * N * 4, kind, st));
  stage_begin(c, NFHMM_STAGE_INIT, st);
  launch_validate(c->V, d.T, d.F, c->Fp, c->WM, c->M, c->A, c->pi, d.S, d.N, c->err, st);
  launch_transpose(c->WM, c->Mp, c->Fp, c->Fp, c->WF, c->Mp, c->Mp, c->Fp, st);
  launch_row_sums(c->V, d.T, d.F, c->Fp, c->v, st);
  launch_element_table(c->M, c->Mp, d.K, d.N, d.T, c->ktab, st);
  int n = 4;
  if (c->use_tc) n += tc_refresh_beta(c->tc, st);
  // initial state: equal weights (w = 1) through the FP32 contractions
  launch_fill_rows(c->w32, d.T, c->M, c->Mp, 1.f, st);
  n += 1;
  stage_end(c, NFHMM_STAGE_INIT, st, n);
  rc = contract(c, false, true);
  if (rc) return rc;
  stage_begin(c, NFHMM_STAGE_INIT, st);
  if (d.init_mode == NFHMM_INIT_UNIFORM) {
    launch_fill(c->dhat, S * T * N, 1.f / (float)d.N, st);
  } else {
    launch_prior_marginals(c->A, c->pi, d.S, d.N, d.T, c->dhat, st);
  }
  stage_end(c, NFHMM_STAGE_INIT, st, 1);
  rc = sync_check(c);
  if (rc) return rc;
  c->sweeps_done = 0;
  c->have_alpha = false;
  c->inputs_ok = true;
  return leave(c);
}

int need_inputs(nfhmm_ctx* c) {
  if (!c->inputs_ok)
    return fail(NFHMM_ESTATE, "the context's last nfhmm_vi_reinit failed; reinit it first");
  return NFHMM_OK;
}

}  // namespace

extern "C" {

const char* nfhmm_last_error(void) { return g_last_error.c_str(); }

int nfhmm_vi_init(nfhmm_ctx** out, const nfhmm_dims* dp, const float* V, const float* W,
                  const float* A, const float* pi, int inputs_on_device, void* cuda_stream) {
  if (out) *out = nullptr;
  if (!out || !dp || !V || !W || !A || !pi) return fail(NFHMM_EINVAL, "NULL argument");
  const nfhmm_dims d = *dp;
  if (d.S < 1 || d.N < 1 || d.K < 1 || d.F < 1 || d.T < 1)
    return fail(NFHMM_EINVAL, "S, N, K, F, T must all be >= 1");
  const long long M = (long long)d.S * d.N * d.K;
  if (M > (1 << 20) || d.F > (1 << 20) || d.T > (1 << 26))
    return fail(NFHMM_EINVAL, "sizes too large (M, F <= 2^20, T <= 2^26)");
  if (d.N > fb_max_states())
    return fail(NFHMM_EINVAL, "N must be <= " + std::to_string(fb_max_states()));
  if (!(d.gamma >= 0.0) || !isfinite(d.gamma)) return fail(NFHMM_EINVAL, "gamma must be >= 0");
  if (d.precision != NFHMM_FP32 && d.precision != NFHMM_BF16 && d.precision != NFHMM_FP32_SIMT)
    return fail(NFHMM_EINVAL, "precision must be NFHMM_FP32, NFHMM_BF16 or NFHMM_FP32_SIMT");
  if (d.init_mode != NFHMM_INIT_UNIFORM && d.init_mode != NFHMM_INIT_PRIOR)
    return fail(NFHMM_EINVAL, "init_mode must be NFHMM_INIT_UNIFORM or NFHMM_INIT_PRIOR");

  nfhmm_ctx* c = new nfhmm_ctx();
  c->d = d;
  c->M = (int)M;
  c->Mp = (int)round_up(M, 32);
  c->Fp = (int)round_up(d.F, 32);
  c->NK = d.N * d.K;
  c->user = reinterpret_cast<cudaStream_t>(cuda_stream);
  c->konst = lgamma((double)M + d.gamma * d.S * d.K) - (double)d.S * d.K * lgamma(1.0 + d.gamma);
  int rc = NFHMM_OK;
  auto bail = [&](int code) {
    free_ctx(c);
    return code;
  };
#define DMALLOC(ptr, bytes) CKI(dmalloc(c, (void**)&(ptr), (bytes)))
#define CKI(call)                                                                        \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) {                                                             \
      fail(e_ == cudaErrorMemoryAllocation ? NFHMM_ENOMEM : NFHMM_ECUDA,                 \
           std::string(#call) + ": " + cudaGetErrorString(e_));                          \
      return bail(e_ == cudaErrorMemoryAllocation ? NFHMM_ENOMEM : NFHMM_ECUDA);         \
    }                                                                                    \
  } while (0)
  CKI(cudaStreamCreateWithFlags(&c->s_main, cudaStreamNonBlocking));
  CKI(cudaStreamCreateWithFlags(&c->s_aux, cudaStreamNonBlocking));
  CKI(cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming));
  CKI(cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming));
  CKI(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
  CKI(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
  const size_t T = d.T, Mp = c->Mp, Fp = c->Fp, S = d.S, N = d.N;
  c->nbpart = gemm_simt_col_tiles(c->Fp);
  if (tc_col_tiles_gemm1(c->Fp) > c->nbpart) c->nbpart = tc_col_tiles_gemm1(c->Fp);
  DMALLOC(c->V, T * Fp * 4);
  DMALLOC(c->WM, Mp * Fp * 4);
  DMALLOC(c->WF, Fp * Mp * 4);
  DMALLOC(c->A, S * N * N * 4);
  DMALLOC(c->pi, S * N * 4);
  DMALLOC(c->alpha, T * Mp * 4);
  DMALLOC(c->w32, T * Mp * 4);
  DMALLOC(c->c, T * Mp * 4);
  DMALLOC(c->Q, T * Fp * 4);
  DMALLOC(c->phi, S * T * N * 4);
  DMALLOC(c->dhat, S * T * N * 4);
  DMALLOC(c->v, T * 8);
  DMALLOC(c->bpart, T * c->nbpart * 8);
  DMALLOC(c->frame_terms, T * 8);
  DMALLOC(c->logZ, S * 8);
  DMALLOC(c->bound_dev, 8);
  DMALLOC(c->err, 4);
  DMALLOC(c->ktab, Mp * sizeof(int2));
  CKI(cudaMallocHost(&c->h_bound, 8));
  CKI(cudaMallocHost(&c->h_err, 4));
  // forward-backward plan and scratch
  c->fb.S = d.S;
  c->fb.N = d.N;
  c->fb.T = d.T;
  c->fb.L = fb_default_chunk(d.N, d.T);
  c->fb.C = (d.T + c->fb.L - 1) / c->fb.L;
  DMALLOC(c->fb_scratch, fb_scratch_bytes(d.S, d.N, d.T, c->fb.L));
  fb_carve_scratch(c->fb, c->fb_scratch);
  c->fb.phi = c->phi;
  c->fb.A = c->A;
  c->fb.pi = c->pi;
  c->fb.dhat = c->dhat;
  c->fb.logZ = c->logZ;
  c->fb.err = c->err;

  // tensor-core plan (operand copies of beta, tensor maps)
  if (d.precision != NFHMM_FP32_SIMT) {
    if (!tc_available())
      return bail(fail(NFHMM_EINVAL, "tensor-core contractions need an sm_103 device"));
    rc = tc_plan(c->tc, d.precision, d.T, c->M, c->Mp, d.F, c->Fp, c->V, c->WM, c->WF, c->w32,
                 c->Q, c->c, c->err, c->s_main);
    if (rc != 0) return bail(fail(NFHMM_ECUDA, "tensor-core plan: " + tc_last_error()));
    c->tc.nbpart = c->nbpart;
    c->use_tc = true;
  }
  rc = load_and_init(c, V, W, A, pi, inputs_on_device);
  if (rc) return bail(rc);
  c->sweeps_done = 0;
  c->have_alpha = false;
  *out = c;
  g_last_error.clear();
  return NFHMM_OK;
#undef CKI
#undef DMALLOC
}

int nfhmm_vi_reinit(nfhmm_ctx* c, const float* V, const float* W, const float* A,
                    const float* pi, int inputs_on_device) {
  if (!c || !V || !W || !A || !pi) return fail(NFHMM_EINVAL, "NULL argument");
  c->inputs_ok = false;
  c->sweeps_done = 0;
  c->have_alpha = false;
  return load_and_init(c, V, W, A, pi, inputs_on_device);
}

int nfhmm_vi_sweep(nfhmm_ctx* c, int n_sweeps, double* bound_out) {
  if (!c) return fail(NFHMM_EINVAL, "NULL context");
  if (need_inputs(c)) return NFHMM_ESTATE;
  if (n_sweeps < 0) return fail(NFHMM_EINVAL, "n_sweeps must be >= 0");
  if (n_sweeps == 0 && bound_out && !c->have_alpha)
    return fail(NFHMM_ESTATE, "no sweep has run: the bound is defined after a sweep");
  int rc = enter(c);
  if (rc) return rc;
  for (int i = 0; i < n_sweeps; ++i) {
    rc = one_sweep(c, bound_out != nullptr && i == n_sweeps - 1);
    if (rc) return rc;
  }
  if (n_sweeps > 0) {
    c->sweeps_done += n_sweeps;
    c->have_alpha = true;
  }
  if (bound_out) {
    if (n_sweeps == 0) {
      rc = contract(c, true, false);
      if (rc) return rc;
    }
    rc = compute_bound(c, bound_out);
    if (rc) return rc;
  }
  return leave(c);
}

int nfhmm_bound(nfhmm_ctx* c, double* out) {
  if (!c || !out) return fail(NFHMM_EINVAL, "NULL argument");
  return nfhmm_vi_sweep(c, 0, out);
}

int nfhmm_separate(nfhmm_ctx* c, float* out, int masked, int weights, int out_on_device) {
  if (!c || !out) return fail(NFHMM_EINVAL, "NULL argument");
  if (need_inputs(c)) return NFHMM_ESTATE;
  if (!c->have_alpha) return fail(NFHMM_ESTATE, "separation needs at least one sweep");
  if (weights != NFHMM_SEP_MEAN && weights != NFHMM_SEP_EXPECTATION)
    return fail(NFHMM_EINVAL, "weights must be NFHMM_SEP_MEAN or NFHMM_SEP_EXPECTATION");
  const nfhmm_dims& d = c->d;
  const size_t T = d.T, F = d.F, S = d.S;
  int rc = enter(c);
  if (rc) return rc;
  cudaStream_t st = c->s_main;
  if (!c->wts) CK(cudaMalloc(&c->wts, T * c->Mp * 4));
  float* dst = out;
  if (!out_on_device) {
    if (!c->sep_tmp) CK(cudaMalloc(&c->sep_tmp, S * T * F * 4));
    dst = c->sep_tmp;
  }
  launch_sep_weights(c->alpha, c->v, d.T, c->M, c->Mp, weights, c->wts, st);
  c->launches += 1;
  for (int s = 0; s < d.S; ++s) {
    GemmArgs g{};
    g.rows = d.T;
    g.cols = d.F;
    g.kdim = c->NK;
    g.A = c->wts + (size_t)s * c->NK;
    g.lda = c->Mp;
    g.B = c->WF + (size_t)s * c->NK;
    g.ldb = c->Mp;
    g.out = dst + (size_t)s * T * F;
    g.ldo = d.F;
    g.err = c->err;
    launch_gemm_simt(g, EPI_STORE, st);
    c->launches += 1;
  }
  if (masked) {
    launch_sep_mask(c->V, c->Fp, dst, d.S, d.T, d.F, st);
    c->launches += 1;
  }
  if (!out_on_device) {
    CK(cudaMemcpyAsync(out, dst, S * T * F * 4, cudaMemcpyDefault, st));
    rc = sync_check(c);
    if (rc) return rc;
  }
  return leave(c);
}

int nfhmm_get_posteriors(nfhmm_ctx* c, float* dhat, int on_device) {
  if (!c || !dhat) return fail(NFHMM_EINVAL, "NULL argument");
  if (need_inputs(c)) return NFHMM_ESTATE;
  int rc = enter(c);
  if (rc) return rc;
  const size_t n = (size_t)c->d.S * c->d.T * c->d.N;
  rc = copy_out(dhat, c->dhat, n * 4, on_device, c->s_main);
  if (rc) return rc;
  if (!on_device) {
    rc = sync_check(c);
    if (rc) return rc;
  }
  return leave(c);
}

static int get_rows(nfhmm_ctx* c, float* dst, const float* src, int on_device) {
  int rc = enter(c);
  if (rc) return rc;
  CK(cudaMemcpy2DAsync(dst, (size_t)c->M * 4, src, (size_t)c->Mp * 4, (size_t)c->M * 4,
                       (size_t)c->d.T, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDefault,
                       c->s_main));
  if (!on_device) {
    rc = sync_check(c);
    if (rc) return rc;
  }
  return leave(c);
}

int nfhmm_get_weights(nfhmm_ctx* c, float* alpha, int on_device) {
  if (!c || !alpha) return fail(NFHMM_EINVAL, "NULL argument");
  if (need_inputs(c)) return NFHMM_ESTATE;
  if (!c->have_alpha) return fail(NFHMM_ESTATE, "alpha-hat is defined after a sweep");
  return get_rows(c, alpha, c->alpha, on_device);
}

int nfhmm_get_surrogate(nfhmm_ctx* c, float* phi, int on_device) {
  if (!c || !phi) return fail(NFHMM_EINVAL, "NULL argument");
  if (need_inputs(c)) return NFHMM_ESTATE;
  if (!c->have_alpha) return fail(NFHMM_ESTATE, "phi-hat is defined after a sweep");
  int rc = enter(c);
  if (rc) return rc;
  const size_t n = (size_t)c->d.S * c->d.T * c->d.N;
  rc = copy_out(phi, c->phi, n * 4, on_device, c->s_main);
  if (rc) return rc;
  if (!on_device) {
    rc = sync_check(c);
    if (rc) return rc;
  }
  return leave(c);
}

int nfhmm_get_state(nfhmm_ctx* c, float* counts, float* dhat, int* sweeps_done, int on_device) {
  if (!c || !counts || !dhat) return fail(NFHMM_EINVAL, "NULL argument");
  if (need_inputs(c)) return NFHMM_ESTATE;
  int rc = get_rows(c, counts, c->c, on_device);
  if (rc) return rc;
  rc = nfhmm_get_posteriors(c, dhat, on_device);
  if (rc) return rc;
  if (sweeps_done) *sweeps_done = c->sweeps_done;
  return NFHMM_OK;
}

int nfhmm_set_state(nfhmm_ctx* c, const float* counts, const float* dhat, int sweeps_done,
                    int on_device) {
  if (!c || !counts || !dhat) return fail(NFHMM_EINVAL, "NULL argument");
  if (sweeps_done < 0) return fail(NFHMM_EINVAL, "sweeps_done must be >= 0");
  if (need_inputs(c)) return NFHMM_ESTATE;
  int rc = enter(c);
  if (rc) return rc;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDefault;
  CK(cudaMemcpy2DAsync(c->c, (size_t)c->Mp * 4, counts, (size_t)c->M * 4, (size_t)c->M * 4,
                       (size_t)c->d.T, kind, c->s_main));
  const size_t n = (size_t)c->d.S * c->d.T * c->d.N;
  CK(cudaMemcpyAsync(c->dhat, dhat, n * 4, kind, c->s_main));
  if (!on_device) {
    rc = sync_check(c);
    if (rc) return rc;
  }
  c->sweeps_done = sweeps_done;
  c->have_alpha = false;
  return leave(c);
}

void nfhmm_destroy(nfhmm_ctx* c) { free_ctx(c); }

int nfhmm_forward_backward(int S, int N, int T, const float* phi, const float* A, const float* pi,
                           float* dhat, double* logZ, int chunk_len, void* cuda_stream) {
  if (!phi || !A || !pi || !dhat || !logZ) return fail(NFHMM_EINVAL, "NULL argument");
  if (S < 1 || N < 1 || T < 1) return fail(NFHMM_EINVAL, "S, N, T must be >= 1");
  if (N > fb_max_states())
    return fail(NFHMM_EINVAL, "N must be <= " + std::to_string(fb_max_states()));
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  FBArgs a{};
  a.S = S;
  a.N = N;
  a.T = T;
  a.L = chunk_len <= 0 ? fb_default_chunk(N, T) : chunk_len;
  if (a.L > 128) a.L = 128;
  if (a.L > T) a.L = T;
  a.C = (T + a.L - 1) / a.L;
  a.phi = phi;
  a.A = A;
  a.pi = pi;
  a.dhat = dhat;
  a.logZ = logZ;
  void* scratch = nullptr;
  const size_t bytes = fb_scratch_bytes(S, N, T, a.L) + 256;
  CK(cudaMallocAsync(&scratch, bytes, st));
  fb_carve_scratch(a, scratch);
  a.err = reinterpret_cast<unsigned*>(reinterpret_cast<char*>(scratch) + bytes - 256);
  CK(cudaMemsetAsync(a.err, 0, 4, st));
  const cudaError_t le = launch_fb(a, st, nullptr);
  CK(cudaFreeAsync(scratch, st));
  CK(le);
  return NFHMM_OK;
}

int nfhmm_digamma(const float* x, float* psi_out, float* w_out, size_t n, void* cuda_stream) {
  if (!x || (!psi_out && !w_out)) return fail(NFHMM_EINVAL, "NULL argument");
  if (n == 0) return NFHMM_OK;
  launch_digamma(x, psi_out, w_out, n, reinterpret_cast<cudaStream_t>(cuda_stream));
  CK(cudaGetLastError());
  return NFHMM_OK;
}

int nfhmm_profile_enable(nfhmm_ctx* c, int on) {
  if (!c) return fail(NFHMM_EINVAL, "NULL context");
  c->profiling = on != 0;
  return NFHMM_OK;
}

int nfhmm_profile_read(nfhmm_ctx* c, int stage, double* ms_total, long long* invocations,
                       long long* launches, int reset) {
  if (!c || stage < 0 || stage >= NFHMM_NUM_STAGES) return fail(NFHMM_EINVAL, "bad argument");
  CK(cudaStreamSynchronize(c->s_main));
  CK(cudaStreamSynchronize(c->s_aux));
  StageEvents& s = c->stages[stage];
  double tot = 0.0;
  const size_t n = s.begin.size() < s.end.size() ? s.begin.size() : s.end.size();
  for (size_t i = 0; i < n; ++i) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, s.begin[i], s.end[i]));
    tot += ms;
  }
  if (ms_total) *ms_total = tot;
  if (invocations) *invocations = (long long)n;
  if (launches) *launches = s.launches;
  if (reset) {
    for (auto e : s.begin) cudaEventDestroy(e);
    for (auto e : s.end) cudaEventDestroy(e);
    s.begin.clear();
    s.end.clear();
    s.launches = 0;
  }
  return NFHMM_OK;
}

long long nfhmm_kernel_launches(nfhmm_ctx* c) { return c ? c->launches : 0; }

int nfhmm_query(nfhmm_ctx* c, int key, long long* value) {
  if (!c || !value) return fail(NFHMM_EINVAL, "NULL argument");
  switch (key) {
    case NFHMM_Q_TENSOR_CORES: *value = c->use_tc ? 1 : 0; return NFHMM_OK;
    case NFHMM_Q_FB_CHUNK: *value = c->fb.L; return NFHMM_OK;
    case NFHMM_Q_SWEEPS_DONE: *value = c->sweeps_done; return NFHMM_OK;
    case NFHMM_Q_DEVICE_BYTES: *value = (long long)c->device_bytes; return NFHMM_OK;
    default: return fail(NFHMM_EINVAL, "unknown query key");
  }
}

}  // extern "C"
