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
  std::vector<cudaEvent_t> begin, end;   // launches made one by one
  long long launches = 0;
  double ms_acc = 0.0;                   // harvested from graph replays
  long long inv_acc = 0;
};

// A sweep captured as a CUDA graph.  With profiling on, the stage
// events are part of the graph (event record nodes) and are read after each
// replay, before the next one records them again.
struct SweepGraph {
  long long key = -1;
  cudaGraphExec_t exec = nullptr;
  int seen = 0;                          // runs made uncaptured with this key
  unsigned long long last_use = 0;
  long long launches = 0;                // kernels per replay
  long long stage_launches[NFHMM_NUM_STAGES] = {};
  struct Ev {
    int stage;
    cudaEvent_t begin, end;
  };
  std::vector<Ev> events;
  bool pending = false;                  // a replay whose events are unread
};

}  // namespace

struct Job {
  long long id;
  int t0, T, sweeps;
};

// A context is a batch of jobs sharing one model (W, A, pi): their frames lie
// back to back in [0, T_active) of a frame store of d.T frames.  nfhmm_vi_init
// makes a batch of one job holding all d.T frames.
struct nfhmm_ctx {
  nfhmm_dims d{};           // d.T = frame capacity
  int M = 0, Mp = 0, Fp = 0, NK = 0;
  int T_active = 0;         // frames held by the jobs
  int max_jobs = 1;
  std::vector<Job> jobs;
  long long next_id = 0;
  cudaStream_t user = nullptr, s_main = nullptr, s_aux = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr, ev_fork = nullptr, ev_join = nullptr;
  // device buffers (frame-indexed ones hold d.T frames)
  float* V = nullptr;       // T x Fp
  float* WM = nullptr;      // Mp x Fp   (beta by element: W[k][l])
  float* WF = nullptr;      // Fp x Mp   (beta by frequency)
  float* A = nullptr;       // S x N x N
  float* pi = nullptr;      // S x N
  float* alpha = nullptr;   // T x Mp
  float* w32 = nullptr;     // T x Mp
  float* c = nullptr;       // T x Mp
  float* Q = nullptr;       // T x Fp
  float* wcol = nullptr;    // Fp: column sums of W (the initial state's reconstruction)
  float* phi = nullptr;     // S x T x N
  float* dhat = nullptr;    // S x T x N
  float* wts = nullptr;     // T x Mp (separation weights)
  float* sep_tmp = nullptr; // S x T x F (host-output separation)
  double* v = nullptr;      // T
  double* bpart = nullptr;  // T x nbpart
  int nbpart = 0;
  double* frame_terms = nullptr;  // T
  double* fterm = nullptr;  // T x 2 per-frame sums for the bound (weights kernel)
  double* logZ = nullptr;   // S x max_jobs
  double* bound_dev = nullptr;    // max_jobs + 1
  unsigned* err = nullptr;
  int2* ktab = nullptr;      // Mp element table
  // job tables on the device: job_t0[max_jobs + 1] | chain_c0[max_jobs + 1] |
  // chain_len[max_jobs] | chunk_chain[Cmax]
  int* d_tab = nullptr;
  int* fb_seg = nullptr;     // 3 * max_jobs ints: segment table of a compaction
  int Cmax = 0;              // chunk capacity of the forward-backward scratch
  int NGmax = 0;             // group capacity
  bool group_auto = true;    // group size follows the chunk length
  void* fb_scratch = nullptr;
  FBArgs fb{};
  TcPlan tc{};
  bool use_tc = false;
  unsigned long long inject_wait_ns = 0;   // test hook for the next sweep (NFHMM_OPT_TEST_WAIT_TIMEOUT)
  double konst = 0.0;
  // host staging (pinned)
  double* h_bound = nullptr;  // max_jobs + 1
  unsigned* h_err = nullptr;
  int sweeps_done = 0;
  bool have_alpha = false;    // alpha-hat, phi-hat of a sweep over the current jobs
  bool bpart_ok = false;      // bound partials of the current alpha-hat
  bool fterm_ok = false;      // per-frame bound sums of the current alpha-hat
  bool bound_ok = false;      // h_bound holds the bound of the current state
  bool inputs_ok = false;
  bool profiling = false;
  int prof_stride = 1;        // events around every prof_stride-th sweep of a run
  bool prof_gate = true;      // this sweep's stages are timed
  // runs of sweeps captured as CUDA graphs, by launch configuration
  bool use_graphs = true;
  SweepGraph graphs[8];
  unsigned long long graph_clock = 0;
  SweepGraph* capturing = nullptr;
  StageEvents stages[NFHMM_NUM_STAGES];
  long long launches = 0;
  size_t device_bytes = 0;
};

namespace {

void stage_begin(nfhmm_ctx* c, int stage, cudaStream_t st) {
  if (!c->profiling || !c->prof_gate) return;
  cudaEvent_t e;
  cudaEventCreate(&e);
  if (c->capturing) {   // an event record node of the graph being captured
    cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
    c->capturing->events.push_back(SweepGraph::Ev{stage, e, nullptr});
    return;
  }
  cudaEventRecord(e, st);
  c->stages[stage].begin.push_back(e);
}
void stage_end(nfhmm_ctx* c, int stage, cudaStream_t st, int launches) {
  c->launches += launches;
  c->stages[stage].launches += launches;
  if (!c->profiling || !c->prof_gate) return;
  cudaEvent_t e;
  cudaEventCreate(&e);
  if (c->capturing) {
    cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
    auto& ev = c->capturing->events;
    for (auto it = ev.rbegin(); it != ev.rend(); ++it)
      if (it->stage == stage && !it->end) {
        it->end = e;
        break;
      }
    return;
  }
  cudaEventRecord(e, st);
  c->stages[stage].end.push_back(e);
}

// Add the stage times of a graph's last replay to the stage totals.
void harvest(nfhmm_ctx* c, SweepGraph& g) {
  if (!g.pending) return;
  g.pending = false;
  for (auto& ev : g.events) {
    if (!ev.end) continue;
    float ms = 0.f;
    if (cudaEventSynchronize(ev.end) == cudaSuccess &&
        cudaEventElapsedTime(&ms, ev.begin, ev.end) == cudaSuccess) {
      c->stages[ev.stage].ms_acc += ms;
      c->stages[ev.stage].inv_acc += 1;
    }
  }
}

void drop_graph(nfhmm_ctx* c, SweepGraph& g) {
  harvest(c, g);
  if (g.exec) cudaGraphExecDestroy(g.exec);
  for (auto& ev : g.events) {
    if (ev.begin) cudaEventDestroy(ev.begin);
    if (ev.end) cudaEventDestroy(ev.end);
  }
  g = SweepGraph();
}

void free_ctx(nfhmm_ctx* c) {
  if (!c) return;
  if (c->s_main) cudaStreamSynchronize(c->s_main);
  if (c->s_aux) cudaStreamSynchronize(c->s_aux);
  void* bufs[] = {c->V, c->WM, c->WF, c->A, c->pi, c->alpha, c->w32, c->c, c->Q, c->phi,
                  c->dhat, c->wts, c->sep_tmp, c->v, c->bpart, c->frame_terms, c->logZ,
                  c->bound_dev, c->err, c->ktab, c->fb_scratch, c->d_tab, c->fterm,
                  c->fb_seg, c->fb.beta, c->fb.emis, c->wcol};
  for (void* p : bufs)
    if (p) cudaFree(p);
  tc_free(c->tc);
  for (auto& g : c->graphs) drop_graph(c, g);
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
// the weights in w32 (and the operand copies of the tensor-core path), for
// frames [t0, t0 + rows); both forms take the row offset.  reserve: SMs the
// persistent tensor-core grids leave to a kernel running beside them.
int contract(nfhmm_ctx* c, bool want_bpart, bool init, int t0, int rows,
             cudaStream_t on = nullptr, int reserve = 0) {
  cudaStream_t st = on ? on : c->s_main;
  if (rows <= 0) return NFHMM_OK;
  // the sweep's contractions run on the tensor cores; so does the initial
  // state's back-projection (w = 1 on frames [t0, t0 + rows)) in split-TF32
  // mode, whose accuracy is FP32's (BF16 contexts form the initial state on
  // the CUDA cores in FP32)
  const bool tc = c->use_tc && (!init || c->tc.w_format == WF_TF32X2);
  if (init) {
    // every weight is 1, so the reconstruction is W's column sum b_l in every
    // frame: Q = V / b, in the form the back-projection reads; nothing runs
    // beside the initial state's contractions
    const size_t oF = (size_t)t0 * c->Fp;
    stage_begin(c, NFHMM_STAGE_INIT, st);
    launch_init_ratio(c->V + oF, c->wcol, rows, c->Fp, tc ? nullptr : c->Q + oF,
                      tc ? reinterpret_cast<float*>(c->tc.q_hi) + oF : nullptr,
                      tc ? reinterpret_cast<float*>(c->tc.q_lo) + oF : nullptr, c->err, st);
    stage_end(c, NFHMM_STAGE_INIT, st, 1);
    reserve = 0;
  }
  if (tc) {
    const int stage1 = init ? NFHMM_STAGE_INIT : NFHMM_STAGE_GEMM1;
    const int stage2 = init ? NFHMM_STAGE_INIT : NFHMM_STAGE_GEMM2;
    int n1 = 0;
    if (!init) {
      stage_begin(c, stage1, st);
      n1 = tc_gemm1(c->tc, t0, rows, want_bpart ? c->bpart : nullptr, reserve, st);
      if (n1 >= 0) stage_end(c, stage1, st, n1);
    }
    int n2 = -1;
    if (n1 >= 0) {
      stage_begin(c, stage2, st);
      n2 = tc_gemm2(c->tc, t0, rows, reserve, st);
      if (n2 >= 0) stage_end(c, stage2, st, n2);
    }
    if (n1 < 0 || n2 < 0) return fail(NFHMM_ECUDA, "tensor-core contraction: " + tc_last_error());
    return NFHMM_OK;
  }
  const int stage1 = init ? NFHMM_STAGE_INIT : NFHMM_STAGE_GEMM1;
  const int stage2 = init ? NFHMM_STAGE_INIT : NFHMM_STAGE_GEMM2;
  const size_t oM = (size_t)t0 * c->Mp, oF = (size_t)t0 * c->Fp;
  GemmArgs g1{};
  g1.rows = rows;
  g1.cols = c->Fp;
  g1.kdim = c->Mp;
  g1.A = c->w32 + oM;
  g1.lda = c->Mp;
  g1.B = c->WF;
  g1.ldb = c->Mp;
  g1.V = c->V + oF;
  g1.ldv = c->Fp;
  g1.out = c->Q + oF;
  g1.ldo = c->Fp;
  g1.bpart = want_bpart ? c->bpart + (size_t)t0 * c->nbpart : nullptr;
  g1.nbpart = c->nbpart;
  g1.err = c->err;
  if (!init) {
    stage_begin(c, stage1, st);
    launch_gemm_simt(g1, EPI_RATIO, st);
    stage_end(c, stage1, st, 1);
  }
  GemmArgs g2{};
  g2.rows = rows;
  g2.cols = c->Mp;
  g2.kdim = c->Fp;
  g2.A = c->Q + oF;
  g2.lda = c->Fp;
  g2.B = c->WM;
  g2.ldb = c->Fp;
  g2.out = c->c + oM;
  g2.ldo = c->Mp;
  g2.w = c->w32 + oM;
  g2.ldw = c->Mp;
  g2.err = c->err;
  stage_begin(c, stage2, st);
  launch_gemm_simt(g2, EPI_SCALE, st);
  stage_end(c, stage2, st, 1);
  return NFHMM_OK;
}

int one_sweep(nfhmm_ctx* c, bool want_bpart, bool keep_alpha) {
  // with the bound wanted, the weights kernel also forms its per-frame sums;
  // alpha-hat is stored only by the last sweep of a run (keep_alpha), the one
  // whose state the bound, the weights, the separation and checkpoints read
  const nfhmm_dims& d = c->d;
  if (c->T_active == 0) return NFHMM_OK;
  WeightsArgs wa{};
  wa.T = c->T_active;
  wa.M = c->M;
  wa.Mp = c->Mp;
  wa.S = d.S;
  wa.N = d.N;
  wa.K = d.K;
  wa.Tstride = d.T;
  wa.gamma = (float)d.gamma;
  wa.ktab = c->ktab;
  wa.counts = c->c;
  wa.dhat = c->dhat;
  wa.alpha = keep_alpha ? c->alpha : nullptr;
  wa.w32 = c->w32;
  wa.phi = c->phi;
  wa.fterm = want_bpart ? c->fterm : nullptr;
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
  // the contractions on the aux stream, concurrent with the forward-backward,
  // which follows the weights on the main stream: its first pass is then a
  // programmatic dependent of the weights kernel and sets up while it ends
  CK(cudaEventRecord(c->ev_fork, c->s_main));
  CK(cudaStreamWaitEvent(c->s_aux, c->ev_fork, 0));
  // the sequential forward-backward holds a few SMs for the whole sweep: the
  // persistent contractions size their grids to the others
  const int reserve = c->fb.seq > 0 ? fb_seq_blocks(d.S * c->fb.nchains, c->fb.seq, d.N) : 0;
  c->tc.inject_wait_ns = c->inject_wait_ns;   // the test hook, once
  c->inject_wait_ns = 0;
  int rc = contract(c, want_bpart, false, 0, c->T_active, c->s_aux, reserve);
  if (rc) return rc;
  stage_begin(c, NFHMM_STAGE_FB, c->s_main);
  int nfb = 0;
  CK(launch_fb(c->fb, c->s_main, &nfb));
  stage_end(c, NFHMM_STAGE_FB, c->s_main, nfb);
  CK(cudaEventRecord(c->ev_join, c->s_aux));
  CK(cudaStreamWaitEvent(c->s_main, c->ev_join, 0));
  return NFHMM_OK;
}

// Bound of every job and their sum into h_bound (synchronises).
int compute_bound(nfhmm_ctx* c) {
  const int nj = (int)c->jobs.size();
  if (nj == 0) {
    c->h_bound[0] = 0.0;
    c->bound_ok = true;
    return NFHMM_OK;
  }
  BoundArgs b{};
  b.T = c->T_active;
  b.M = c->M;
  b.Mp = c->Mp;
  b.S = c->d.S;
  b.K = c->d.K;
  b.njobs = nj;
  b.job_t0 = c->d_tab;
  b.gamma = (float)c->d.gamma;
  b.konst = c->konst;
  b.alpha = c->alpha;
  b.v = c->v;
  b.bpart = c->bpart;
  b.nbpart = c->nbpart;
  b.nbpart_used = c->use_tc ? tc_bpart_used(c->tc) : gemm_simt_col_tiles(c->Fp);
  b.fterm = c->fterm_ok ? c->fterm : nullptr;
  b.funits = weights_units(c->d.S, c->d.N, c->d.K, c->d.T);
  b.logZ = c->logZ;
  b.frame_terms = c->frame_terms;
  b.out = c->bound_dev;
  stage_begin(c, NFHMM_STAGE_BOUND, c->s_main);
  int n = 0;
  launch_bound(b, c->s_main, &n);
  stage_end(c, NFHMM_STAGE_BOUND, c->s_main, n);
  CK(cudaMemcpyAsync(c->h_bound, c->bound_dev, (nj + 1) * sizeof(double),
                     cudaMemcpyDeviceToHost, c->s_main));
  int rc = sync_check(c);
  if (rc) return rc;
  c->bound_ok = true;
  return NFHMM_OK;
}

// Copy the model (W, A, pi) into the context, validate it and refresh the
// layouts and operand copies derived from it.  Queued on s_main.
int load_model(nfhmm_ctx* c, const float* W, const float* A, const float* pi, int on_device) {
  const nfhmm_dims& d = c->d;
  const size_t Mp = c->Mp, Fp = c->Fp, S = d.S, N = d.N;
  cudaStream_t st = c->s_main;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDefault;
  CK(cudaMemsetAsync(c->WM, 0, Mp * Fp * 4, st));
  CK(cudaMemcpy2DAsync(c->WM, Fp * 4, W, (size_t)d.F * 4, (size_t)d.F * 4, (size_t)c->M, kind,
                       st));
  CK(cudaMemcpyAsync(c->A, A, S * N * N * 4, kind, st));
  CK(cudaMemcpyAsync(c->pi, pi, S * N * 4, kind, st));
  stage_begin(c, NFHMM_STAGE_INIT, st);
  launch_validate(c->V, 0, d.F, c->Fp, c->WM, c->M, c->A, c->pi, d.S, d.N, c->err, st);
  launch_transpose(c->WM, c->Mp, c->Fp, c->Fp, c->WF, c->Mp, c->Mp, c->Fp, st);
  launch_element_table(c->M, c->Mp, d.K, d.N, c->ktab, st);
  launch_col_sums(c->WM, c->M, c->Fp, c->wcol, st);
  int n = 4;
  if (c->use_tc) n += tc_refresh_beta(c->tc, st);
  stage_end(c, NFHMM_STAGE_INIT, st, n);
  return NFHMM_OK;
}

// Copy the spectrograms of n jobs (frames[j] rows from Vs[j]) into frames
// [t0, t0 + T) of the frame store, back to back, validate them and set those
// frames' initial state: z-hat from equal weights (w = 1 through the
// contractions: the tensor cores' in split-TF32 mode, the CUDA cores' FP32 ones
// otherwise) and d-hat from init_mode (the prior marginals restart at
// every job).  Queued on s_main.
int load_frames(nfhmm_ctx* c, int t0, int T, const float* const* Vs, int on_device,
                const int* frames, int n) {
  const nfhmm_dims& d = c->d;
  const size_t Mp = c->Mp, Fp = c->Fp, N = d.N;
  cudaStream_t st = c->s_main;
  if (T <= 0) return NFHMM_OK;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDefault;
  CK(cudaMemsetAsync(c->c + (size_t)t0 * Mp, 0, (size_t)T * Mp * 4, st));
  CK(cudaMemsetAsync(c->alpha + (size_t)t0 * Mp, 0, (size_t)T * Mp * 4, st));
  CK(cudaMemsetAsync(c->bpart + (size_t)t0 * c->nbpart, 0, (size_t)T * c->nbpart * 8, st));
  // the jobs' spectrograms, per run of jobs that follow each other in the
  // caller's memory: read in place by the padding kernel when the device can
  // address them (device memory, or mapped pinned host memory, read over the
  // host link); otherwise one contiguous copy (a copy of F-float rows into
  // the padded layout would move one short row at a time) staged packed in
  // the ratio buffer Q (free until the initial state's ratio below), then
  // padded into the frame store
  int pads = 0;
  for (int j = 0, t = t0; j < n;) {
    int k = j;
    size_t rows = (size_t)frames[j];
    while (k + 1 < n && Vs[k + 1] == Vs[k] + (size_t)frames[k] * d.F) rows += frames[++k];
    const float* direct = on_device ? Vs[j] : nullptr;
    if (!on_device) {
      cudaPointerAttributes pa{};
      if (cudaPointerGetAttributes(&pa, Vs[j]) == cudaSuccess && pa.type == cudaMemoryTypeHost &&
          pa.devicePointer)
        direct = static_cast<const float*>(pa.devicePointer);
      else
        cudaGetLastError();   // an unregistered host pointer is not an error here
    }
    if (direct) {
      launch_pad_rows(direct, (int)rows, d.F, c->V + (size_t)t * Fp, (int)Fp, st);
      ++pads;
    } else if (d.F == (int)Fp) {
      CK(cudaMemcpyAsync(c->V + (size_t)t * Fp, Vs[j], rows * Fp * 4, kind, st));
    } else {
      float* stage = c->Q + (size_t)t * Fp;
      CK(cudaMemcpyAsync(stage, Vs[j], rows * d.F * 4, kind, st));
      launch_pad_rows(stage, (int)rows, d.F, c->V + (size_t)t * Fp, (int)Fp, st);
      ++pads;
    }
    t += (int)rows;
    j = k + 1;
  }
  stage_begin(c, NFHMM_STAGE_INIT, st);
  launch_validate(c->V + (size_t)t0 * Fp, T, d.F, c->Fp, c->WM, c->M, c->A, c->pi, d.S, d.N,
                  c->err, st);
  launch_row_sums(c->V + (size_t)t0 * Fp, T, d.F, c->Fp, c->v + t0, st);
  launch_fill_rows(c->w32 + (size_t)t0 * Mp, T, c->M, c->Mp, 1.f, st);
  stage_end(c, NFHMM_STAGE_INIT, st, 3 + pads);
  int rc = contract(c, false, true, t0, T);
  if (rc) return rc;
  stage_begin(c, NFHMM_STAGE_INIT, st);
  int launches = 0;
  if (d.init_mode == NFHMM_INIT_UNIFORM) {
    for (int s = 0; s < d.S; ++s, ++launches)
      launch_fill(c->dhat + ((size_t)s * d.T + t0) * N, (size_t)T * N, 1.f / (float)d.N, st);
  } else {
    int t = t0;
    for (int j = 0; j < n; ++j, ++launches) {
      launch_prior_marginals(c->A, c->pi, d.S, d.N, d.T, nullptr, 1, t, t + frames[j], c->dhat,
                             st);
      t += frames[j];
    }
  }
  stage_end(c, NFHMM_STAGE_INIT, st, launches);
  return NFHMM_OK;
}

int fb_chunks(const nfhmm_ctx* c) {
  int C = 0;
  for (const Job& j : c->jobs) C += (j.T + c->fb.L - 1) / c->fb.L;
  return C;
}

// (Re)allocate the forward-backward scratch and the job tables for chunk
// length fb.L: room for every job set the frame store and job slots allow.
// Table layout (ints): job_t0[mj+1] | chain_c0[mj+1] | chain_len[mj] |
// chunk_chain[Cmax] | grp_c0[NGmax+1] | chain_g0[mj+1].
size_t tab_ints(const nfhmm_ctx* c) {
  return (size_t)3 * c->max_jobs + 2 + c->Cmax + c->NGmax + 1 + c->max_jobs + 1;
}

int groups_for(const nfhmm_ctx* c, int chunks) {
  return c->fb.G >= 2 ? (chunks + c->fb.G - 1) / c->fb.G : 0;
}

// (Re)allocate the forward-backward scratch and the job tables for chunk
// length fb.L and group size fb.G: room for every job set the frame store
// and job slots allow.
// The forward-backward form: 0 the scan over chunks, k >= 1 the sequential
// form with k chains per block (at most fb_seq_max_cpc); its backward-vector
// array (S x T x N floats) and emission rows (S x T x 68) are allocated on
// first use and kept.
int set_fb_mode(nfhmm_ctx* c, int cpc) {
  if (cpc > 0 && !c->fb.beta) {
    CK(dmalloc(c, (void**)&c->fb.beta, (size_t)c->d.S * c->d.T * c->d.N * sizeof(float)));
  }
  if (cpc > 0 && !c->fb.emis) {
    CK(dmalloc(c, (void**)&c->fb.emis, (size_t)c->d.S * c->d.T * 68 * sizeof(float)));
  }
  const int m = fb_seq_max_cpc(c->d.N);
  c->fb.seq = cpc <= 0 ? 0 : cpc < m ? cpc : m;
  return NFHMM_OK;
}

int ensure_fb_capacity(nfhmm_ctx* c) {
  const int need = (c->d.T + c->fb.L - 1) / c->fb.L + c->max_jobs;
  const int gneed = c->fb.G >= 2 ? need / c->fb.G + 1 + c->max_jobs : 0;
  if (c->fb_scratch && need <= c->Cmax && gneed <= c->NGmax) return NFHMM_OK;
  CK(cudaStreamSynchronize(c->s_main));
  CK(cudaStreamSynchronize(c->s_aux));
  // captured sweeps hold pointers into the buffers about to be replaced
  for (auto& g : c->graphs) drop_graph(c, g);
  if (c->fb_scratch) {
    cudaFree(c->fb_scratch);
    c->device_bytes -= fb_scratch_bytes(c->d.S, c->d.N, c->Cmax, c->NGmax);
    c->fb_scratch = nullptr;
  }
  if (c->d_tab) {
    cudaFree(c->d_tab);
    c->device_bytes -= tab_ints(c) * sizeof(int);
    c->d_tab = nullptr;
  }
  c->Cmax = need;
  c->NGmax = gneed;
  CK(dmalloc(c, &c->fb_scratch, fb_scratch_bytes(c->d.S, c->d.N, c->Cmax, c->NGmax)));
  CK(dmalloc(c, (void**)&c->d_tab, tab_ints(c) * sizeof(int)));
  c->fb.C = c->Cmax;
  c->fb.NG = c->NGmax;
  fb_carve_scratch(c->fb, c->fb_scratch);   // regions sized for Cmax chunks, NGmax groups
  const int mj = c->max_jobs;
  c->fb.chain_t0 = c->d_tab;
  c->fb.chain_c0 = c->d_tab + (mj + 1);
  c->fb.chain_len = c->d_tab + 2 * (mj + 1);
  c->fb.chunk_chain = c->d_tab + 3 * mj + 2;
  c->fb.grp_c0 = c->d_tab + 3 * mj + 2 + c->Cmax;
  c->fb.chain_g0 = c->fb.grp_c0 + c->NGmax + 1;
  c->fb.C = fb_chunks(c);
  c->fb.NG = 0;
  return NFHMM_OK;
}

// Upload the job tables for the current job list (queued on s_main; the
// host copy is staged by the runtime before the call returns).
int commit_jobs(nfhmm_ctx* c) {
  const int nj = (int)c->jobs.size(), mj = c->max_jobs;
  const int C = fb_chunks(c);
  std::vector<int> tab(tab_ints(c), 0);
  int* job_t0 = tab.data();
  int* chain_c0 = job_t0 + (mj + 1);
  int* chain_len = chain_c0 + (mj + 1);
  int* chunk_chain = chain_len + mj;
  int* grp_c0 = chunk_chain + c->Cmax;
  int* chain_g0 = grp_c0 + c->NGmax + 1;
  int cc = 0, ng = 0;
  for (int j = 0; j < nj; ++j) {
    job_t0[j] = c->jobs[j].t0;
    chain_c0[j] = cc;
    chain_g0[j] = ng;
    chain_len[j] = c->jobs[j].T;
    const int nc = (c->jobs[j].T + c->fb.L - 1) / c->fb.L;
    for (int q = 0; q < nc; ++q) chunk_chain[cc + q] = j;
    for (int k = 0; k < groups_for(c, nc); ++k) grp_c0[ng++] = cc + k * c->fb.G;
    cc += nc;
  }
  job_t0[nj] = c->T_active;
  chain_c0[nj] = cc;
  chain_g0[nj] = ng;
  if (c->NGmax > 0) grp_c0[ng] = cc;
  CK(cudaMemcpyAsync(c->d_tab, tab.data(), tab.size() * sizeof(int), cudaMemcpyHostToDevice,
                     c->s_main));
  c->fb.C = C;
  c->fb.NG = ng;
  c->fb.nchains = nj;
  int longest = 0;
  for (int j = 0; j < nj; ++j) longest = c->jobs[j].T > longest ? c->jobs[j].T : longest;
  c->fb.maxlen = longest;
  c->have_alpha = false;
  c->bpart_ok = false;
  c->fterm_ok = false;
  c->bound_ok = false;
  return NFHMM_OK;
}

// Append n jobs (frames[j] frames, spectrogram Vs[j]).  Validates
// (synchronises once); on failure nothing is added.
int add_jobs(nfhmm_ctx* c, int n, const int* frames, const float* const* Vs, int on_device,
             long long* ids) {
  long long total = 0;
  for (int j = 0; j < n; ++j) {
    if (frames[j] < 1) return fail(NFHMM_EINVAL, "every job needs at least one frame");
    total += frames[j];
  }
  if ((int)c->jobs.size() + n > c->max_jobs)
    return fail(NFHMM_EFULL, "the batch holds " + std::to_string(c->jobs.size()) + " of " +
                                 std::to_string(c->max_jobs) + " jobs");
  if (c->T_active + total > c->d.T)
    return fail(NFHMM_EFULL, "the batch has " + std::to_string(c->d.T - c->T_active) +
                                 " free frames; the jobs need " + std::to_string(total));
  int rc = enter(c);
  if (rc) return rc;
  const int t0 = c->T_active;
  rc = load_frames(c, t0, (int)total, Vs, on_device, frames, n);
  if (rc) return rc;
  rc = sync_check(c);
  if (rc) return rc;
  int t = t0;
  for (int j = 0; j < n; ++j) {
    const long long id = c->next_id++;
    c->jobs.push_back(Job{id, t, frames[j], 0});
    if (ids) ids[j] = id;
    t += frames[j];
  }
  c->T_active = t;
  rc = commit_jobs(c);
  if (rc) return rc;
  return leave(c);
}

// Remove the jobs whose flags are set and move the others down over the
// freed frames (their persistent state: V, counts, d-hat, v).  The frames
// from the first removed job on are copied to scratch buffers that the next
// sweep rewrites anyway (Q, alpha-hat, phi-hat, the bound's frame terms) and
// gathered back by one kernel.
int remove_jobs(nfhmm_ctx* c, const std::vector<char>& gone) {
  const nfhmm_dims& d = c->d;
  const size_t Mp = c->Mp, Fp = c->Fp, N = d.N, S = d.S, Tc = d.T;
  size_t first = 0;
  while (first < c->jobs.size() && !gone[first]) ++first;
  if (first == c->jobs.size()) return NFHMM_OK;
  const int base = c->jobs[first].t0, span = c->T_active - base;
  std::vector<int> seg;   // (destination first frame, source offset in the copy, frames)
  std::vector<Job> kept(c->jobs.begin(), c->jobs.begin() + first);
  int t = base;
  for (size_t j = first; j < c->jobs.size(); ++j) {
    if (gone[j]) continue;
    Job q = c->jobs[j];
    seg.push_back(t);
    seg.push_back(q.t0 - base);
    seg.push_back(q.T);
    q.t0 = t;
    t += q.T;
    kept.push_back(q);
  }
  int rc = enter(c);
  if (rc) return rc;
  cudaStream_t st = c->s_main;
  if (!seg.empty()) {
    const cudaMemcpyKind dd = cudaMemcpyDeviceToDevice;
    CK(cudaMemcpyAsync(c->Q, c->V + base * Fp, span * Fp * 4, dd, st));
    CK(cudaMemcpyAsync(c->alpha, c->c + base * Mp, span * Mp * 4, dd, st));
    CK(cudaMemcpy2DAsync(c->phi, Tc * N * 4, c->dhat + base * N, Tc * N * 4, span * N * 4, S, dd,
                         st));
    CK(cudaMemcpyAsync(c->frame_terms, c->v + base, span * 8, dd, st));
    // the segment table rides in the chunk-table region, rewritten below
    CK(cudaMemcpyAsync(c->fb_seg, seg.data(), seg.size() * sizeof(int), cudaMemcpyHostToDevice,
                       st));
    FrameMove m{};
    m.nseg = (int)seg.size() / 3;
    m.seg = c->fb_seg;
    m.frames = t - base;
    m.base = base;
    m.Tc = d.T;
    m.Fp = c->Fp;
    m.Mp = c->Mp;
    m.SN = d.S * d.N;
    m.N = d.N;
    m.S = d.S;
    m.V = c->V;
    m.Vs = c->Q;
    m.c = c->c;
    m.cs = c->alpha;
    m.dhat = c->dhat;
    m.ds = c->phi;
    m.v = c->v;
    m.vs = c->frame_terms;
    launch_move_frames(m, st);
    c->launches += 1;
  }
  c->jobs.swap(kept);
  c->T_active = t;
  rc = commit_jobs(c);
  if (rc) return rc;
  return leave(c);
}

int find_job(nfhmm_ctx* c, long long id) {
  for (size_t j = 0; j < c->jobs.size(); ++j)
    if (c->jobs[j].id == id) return (int)j;
  return -1;
}

// S slices of T_active frames (stride d.T frames) to or from a packed
// S x T_active x width array.
int copy_slices(nfhmm_ctx* c, void* dst, const void* src, int width, bool to_packed, int t0,
                int T, int on_device) {
  const size_t row = (size_t)T * width * 4, stride = (size_t)c->d.T * width * 4;
  const size_t off = (size_t)t0 * width * 4;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDefault;
  if (row == 0) return NFHMM_OK;
  if (to_packed)
    CK(cudaMemcpy2DAsync(dst, row, (const char*)src + off, stride, row, c->d.S, kind, c->s_main));
  else
    CK(cudaMemcpy2DAsync((char*)dst + off, stride, src, row, row, c->d.S, kind, c->s_main));
  return NFHMM_OK;
}

int need_inputs(nfhmm_ctx* c) {
  if (!c->inputs_ok)
    return fail(NFHMM_ESTATE, "the context's last nfhmm_vi_reinit failed; reinit it first");
  return NFHMM_OK;
}

}  // namespace

extern "C" {

const char* nfhmm_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"

namespace {

// Allocate a context for a frame store of d.T frames and max_jobs jobs and
// load the model; no jobs yet.  Synchronises once (model validation).
int create_ctx(nfhmm_ctx** out, const nfhmm_dims* dp, int max_jobs, const float* W,
               const float* A, const float* pi, int inputs_on_device, void* cuda_stream) {
  if (out) *out = nullptr;
  if (!out || !dp || !W || !A || !pi) return fail(NFHMM_EINVAL, "NULL argument");
  const nfhmm_dims d = *dp;
  if (d.S < 1 || d.N < 1 || d.K < 1 || d.F < 1 || d.T < 1)
    return fail(NFHMM_EINVAL, "S, N, K, F, T must all be >= 1");
  if (max_jobs < 1 || max_jobs > (1 << 20)) return fail(NFHMM_EINVAL, "max_jobs must be in [1, 2^20]");
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
  c->max_jobs = max_jobs;
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
  // bound partials per frame: room for the narrowest reconstruction tile
  c->nbpart = gemm_simt_col_tiles(c->Fp);
  if (tc_bpart_columns_max(c->Fp) > c->nbpart) c->nbpart = tc_bpart_columns_max(c->Fp);
  DMALLOC(c->V, T * Fp * 4);
  DMALLOC(c->WM, Mp * Fp * 4);
  DMALLOC(c->WF, Fp * Mp * 4);
  DMALLOC(c->A, S * N * N * 4);
  DMALLOC(c->pi, S * N * 4);
  DMALLOC(c->alpha, T * Mp * 4);
  DMALLOC(c->w32, T * Mp * 4);
  DMALLOC(c->c, T * Mp * 4);
  DMALLOC(c->Q, T * Fp * 4);
  DMALLOC(c->wcol, Fp * 4);
  DMALLOC(c->phi, S * T * N * 4);
  DMALLOC(c->dhat, S * T * N * 4);
  DMALLOC(c->v, T * 8);
  DMALLOC(c->bpart, T * c->nbpart * 8);
  DMALLOC(c->frame_terms, T * 8);
  DMALLOC(c->fterm, T * 16 * weights_units(d.S, d.N, d.K, d.T));
  DMALLOC(c->fb_seg, (size_t)3 * max_jobs * sizeof(int));
  DMALLOC(c->logZ, S * max_jobs * 8);
  DMALLOC(c->bound_dev, (max_jobs + 1) * 8);
  DMALLOC(c->err, 4);
  DMALLOC(c->ktab, Mp * sizeof(int2));
  CKI(cudaMallocHost(&c->h_bound, (max_jobs + 1) * 8));
  CKI(cudaMallocHost(&c->h_err, 4));
  // frames never written by a job are read by the tiles that straddle the
  // end of the jobs' frames: start them at zero
  CKI(cudaMemsetAsync(c->V, 0, T * Fp * 4, c->s_main));
  CKI(cudaMemsetAsync(c->w32, 0, T * Mp * 4, c->s_main));
  CKI(cudaMemsetAsync(c->err, 0, 4, c->s_main));
  // forward-backward plan, scratch and job tables
  c->fb.S = d.S;
  c->fb.N = d.N;
  c->fb.T = d.T;   // frame stride of phi-hat and d-hat
  // one job: the chain's latency sets the sweep (chunks of 0.3 sqrt(T) frames
  // and the two-level scan); batches: many chains run side by side and the
  // total work sets it (chunks of 32 frames, one-level scan)
  c->fb.L = max_jobs == 1 ? fb_default_chunk(d.N, d.T) : (d.T < 32 ? d.T : 32);
  c->fb.products = FB_PRODUCTS_TC;
  c->fb.inputs_stable = 1;   // the context's own copies of A and pi
  c->fb.G = max_jobs == 1 ? fb_default_group((d.T + c->fb.L - 1) / c->fb.L) : 0;
  c->group_auto = max_jobs == 1;
  c->fb.phi = c->phi;
  c->fb.A = c->A;
  c->fb.pi = c->pi;
  c->fb.dhat = c->dhat;
  c->fb.logZ = c->logZ;
  c->fb.err = c->err;
  rc = ensure_fb_capacity(c);
  if (rc) return bail(rc);

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
#undef CKI
#undef DMALLOC
  rc = enter(c);
  if (!rc) rc = load_model(c, W, A, pi, inputs_on_device);
  if (!rc) rc = commit_jobs(c);
  if (!rc) rc = sync_check(c);
  if (!rc) rc = leave(c);
  if (rc) return bail(rc);
  c->inputs_ok = true;
  *out = c;
  return NFHMM_OK;
}

// The launch configuration a captured run of `count` sweeps depends on;
// timed: its stages are bracketed by events (then slot alternates between two
// instances, so that one may still be in flight while the other is launched).
long long graph_key_of(const nfhmm_ctx* c, bool want_bpart, bool timed, int slot,
                       bool keep_alpha, int count) {
  long long k = c->T_active;
  k = k * 1000003 + c->fb.C;
  k = k * 1048583 + c->fb.nchains;
  k = k * 131 + c->fb.L;
  k = k * 4099 + c->fb.G;
  k = k * 1000033 + c->fb.NG;
  k = k * 3 + c->fb.products;
  k = k * 67 + c->fb.seq;
  k = k * 257 + c->tc.bn1;
  k = k * 257 + c->tc.bn2;
  k = k * 17 + c->tc.st1;
  k = k * 17 + c->tc.st2;
  k = k * 67 + c->tc.pf1;
  k = k * 67 + c->tc.pf2;
  k = k * 4 + c->tc.ep1 * 2 + c->tc.ep2;
  k = k * 2 + (want_bpart ? 1 : 0);
  k = k * 2 + (keep_alpha ? 1 : 0);
  k = k * 3 + (timed ? 1 + slot : 0);
  k = k * 17 + count;
  return k;
}

// n sweeps launched one by one; with profiling, the stages of sweep i are
// timed when (first + i) is a multiple of the profiling stride.
int sweeps_direct(nfhmm_ctx* c, int n, bool want_bpart, long long first = 0,
                  bool keep_alpha = true) {
  for (int i = 0; i < n; ++i) {
    c->prof_gate = (first + i) % c->prof_stride == 0;
    const int rc = one_sweep(c, want_bpart && i == n - 1, keep_alpha && i == n - 1);
    c->prof_gate = true;
    if (rc) return rc;
  }
  return NFHMM_OK;
}

// n sweeps (the last with the bound's terms if want_bpart), replayed from
// captured CUDA graphs once the same launch configuration has run uncaptured
// once, else launched one by one.  The run's last sweep (which keeps
// alpha-hat and may form the bound's terms) and, with profiling, every
// prof_stride-th sweep (stage events; two instances in turn, an instance's
// previous events read before it is launched again) replay one-sweep graphs;
// the plain sweeps between them replay graphs of up to kSweepsPerGraph sweeps,
// which saves the gap between graph launches (the sweeps themselves are the
// same kernels in the same order).
constexpr int kSweepsPerGraph = 8;
int run_graph(nfhmm_ctx* c, bool want_bpart, long long index, bool keep_alpha, int count);
int run_sweeps(nfhmm_ctx* c, int n, bool want_bpart) {
  // a sweep carrying the wait hook is launched directly (a graph would keep it)
  if (!c->use_graphs || c->T_active == 0 || n < 1 || c->inject_wait_ns)
    return sweeps_direct(c, n, want_bpart);
  auto plain = [&](int i) { return i < n - 1 && !(c->profiling && i % c->prof_stride == 0); };
  for (int i = 0; i < n;) {
    int m = 1;
    if (plain(i))
      while (m < kSweepsPerGraph && plain(i + m)) ++m;
    const int rc = run_graph(c, want_bpart && i == n - 1, i, i == n - 1, m);
    if (rc) return rc;
    i += m;
  }
  return NFHMM_OK;
}

int run_graph(nfhmm_ctx* c, bool want_bpart, long long index, bool keep_alpha, int count) {
  const bool timed = c->profiling && index % c->prof_stride == 0;
  const int slot = (int)((index / c->prof_stride) & 1);
  // the index the sweeps are captured with: one that gives them the same
  // gates (a run of plain sweeps is shorter than the profiling stride)
  const long long cap_index = timed || c->prof_stride == 1 ? 0 : 1;
  const long long key = graph_key_of(c, want_bpart, timed, slot, keep_alpha, count);
  SweepGraph* g = nullptr;
  for (auto& x : c->graphs)
    if (x.key == key) g = &x;
  if (!g) {   // reuse the least recently used slot
    g = &c->graphs[0];
    for (auto& x : c->graphs)
      if (x.last_use < g->last_use) g = &x;
    drop_graph(c, *g);
    g->key = key;
  }
  g->last_use = ++c->graph_clock;
  if (!g->exec) {
    if (g->seen++ == 0)   // first uncaptured
      return sweeps_direct(c, count, want_bpart, index, keep_alpha);
    const long long l0 = c->launches;
    long long s0[NFHMM_NUM_STAGES];
    for (int i = 0; i < NFHMM_NUM_STAGES; ++i) s0[i] = c->stages[i].launches;
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(c->s_main, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      c->use_graphs = false;
      return sweeps_direct(c, count, want_bpart, index, keep_alpha);
    }
    c->capturing = g;
    const int rc = sweeps_direct(c, count, want_bpart, cap_index, keep_alpha);
    c->capturing = nullptr;
    const cudaError_t e = cudaStreamEndCapture(c->s_main, &graph);
    const bool good = !rc && e == cudaSuccess && graph &&
                      cudaGraphInstantiate(&g->exec, graph, 0) == cudaSuccess;
    if (graph) cudaGraphDestroy(graph);
    g->launches = c->launches - l0;
    c->launches = l0;
    for (int i = 0; i < NFHMM_NUM_STAGES; ++i) {
      g->stage_launches[i] = c->stages[i].launches - s0[i];
      c->stages[i].launches = s0[i];
    }
    if (!good) {
      cudaGetLastError();
      drop_graph(c, *g);
      c->use_graphs = false;
      if (rc) return rc;
      // capture unavailable: launch directly
      return sweeps_direct(c, count, want_bpart, index, keep_alpha);
    }
  }
  harvest(c, *g);   // its events are about to be recorded again
  CK(cudaGraphLaunch(g->exec, c->s_main));
  c->launches += g->launches;
  for (int i = 0; i < NFHMM_NUM_STAGES; ++i) c->stages[i].launches += g->stage_launches[i];
  g->pending = c->profiling && !g->events.empty();
  return NFHMM_OK;
}

// Run n sweeps over every job; with want_bound, the last one also forms the
// bound's per-frame terms, and with finish the bounds of the final state go
// into h_bound (synchronises).
int sweep_impl(nfhmm_ctx* c, int n_sweeps, bool want_bound, bool finish = true) {
  if (n_sweeps == 0 && want_bound && !c->have_alpha)
    return fail(NFHMM_ESTATE, "no sweep has run over the current jobs: the bound is defined "
                              "after a sweep");
  if (n_sweeps == 0 && want_bound && c->bound_ok) return NFHMM_OK;
  int rc = enter(c);
  if (rc) return rc;
  rc = run_sweeps(c, n_sweeps, want_bound);
  if (rc) return rc;
  if (n_sweeps > 0) {
    c->sweeps_done += n_sweeps;
    for (Job& j : c->jobs) j.sweeps += n_sweeps;
    c->have_alpha = true;
    c->bpart_ok = want_bound;
    c->fterm_ok = want_bound;
    c->bound_ok = false;
  }
  if (want_bound && finish) {
    if (!c->bpart_ok) {
      rc = contract(c, true, false, 0, c->T_active);
      if (rc) return rc;
      c->bpart_ok = true;
    }
    rc = compute_bound(c);
    if (rc) return rc;
  }
  return leave(c);
}

}  // namespace

extern "C" {

int nfhmm_vi_init(nfhmm_ctx** out, const nfhmm_dims* dp, const float* V, const float* W,
                  const float* A, const float* pi, int inputs_on_device, void* cuda_stream) {
  if (out) *out = nullptr;
  if (!out || !dp || !V) return fail(NFHMM_EINVAL, "NULL argument");
  nfhmm_ctx* c = nullptr;
  int rc = create_ctx(&c, dp, 1, W, A, pi, inputs_on_device, cuda_stream);
  if (rc) return rc;
  const int T = dp->T;
  rc = add_jobs(c, 1, &T, &V, inputs_on_device, nullptr);
  if (rc) {
    free_ctx(c);
    return rc;
  }
  *out = c;
  g_last_error.clear();
  return NFHMM_OK;
}

int nfhmm_vi_init_batch(nfhmm_ctx** out, const nfhmm_dims* dp, int n_jobs, const int* job_frames,
                        const float* V, const float* W, const float* A, const float* pi,
                        int inputs_on_device, void* cuda_stream, long long* job_ids) {
  if (out) *out = nullptr;
  if (!out || !dp || !V || !job_frames) return fail(NFHMM_EINVAL, "NULL argument");
  if (n_jobs < 1) return fail(NFHMM_EINVAL, "n_jobs must be >= 1");
  long long total = 0;
  for (int j = 0; j < n_jobs; ++j) {
    if (job_frames[j] < 1) return fail(NFHMM_EINVAL, "every job needs at least one frame");
    total += job_frames[j];
  }
  if (total != dp->T) return fail(NFHMM_EINVAL, "d->T must equal the sum of job_frames");
  nfhmm_ctx* c = nullptr;
  int rc = create_ctx(&c, dp, n_jobs, W, A, pi, inputs_on_device, cuda_stream);
  if (rc) return rc;
  std::vector<const float*> Vs(n_jobs);
  for (int j = 0, t = 0; j < n_jobs; t += job_frames[j], ++j) Vs[j] = V + (size_t)t * dp->F;
  rc = add_jobs(c, n_jobs, job_frames, Vs.data(), inputs_on_device, job_ids);
  if (rc) {
    free_ctx(c);
    return rc;
  }
  *out = c;
  g_last_error.clear();
  return NFHMM_OK;
}

int nfhmm_batch_create(nfhmm_ctx** out, const nfhmm_dims* dp, int max_jobs, const float* W,
                       const float* A, const float* pi, int inputs_on_device, void* cuda_stream) {
  const int rc = create_ctx(out, dp, max_jobs, W, A, pi, inputs_on_device, cuda_stream);
  if (!rc) g_last_error.clear();
  return rc;
}

int nfhmm_batch_add(nfhmm_ctx* c, int T, const float* V, int on_device, long long* job_id) {
  if (!c || !V) return fail(NFHMM_EINVAL, "NULL argument");
  if (need_inputs(c)) return NFHMM_ESTATE;
  return add_jobs(c, 1, &T, &V, on_device, job_id);
}

int nfhmm_batch_add_many(nfhmm_ctx* c, int n, const int* T, const float* const* V, int on_device,
                         long long* job_ids) {
  if (!c || !T || !V || n < 0) return fail(NFHMM_EINVAL, "NULL argument or n < 0");
  if (need_inputs(c)) return NFHMM_ESTATE;
  for (int j = 0; j < n; ++j)
    if (!V[j]) return fail(NFHMM_EINVAL, "NULL spectrogram");
  if (n == 0) return NFHMM_OK;
  return add_jobs(c, n, T, V, on_device, job_ids);
}

int nfhmm_batch_remove(nfhmm_ctx* c, long long job_id) {
  return nfhmm_batch_remove_many(c, 1, &job_id);
}

int nfhmm_batch_remove_many(nfhmm_ctx* c, int n, const long long* job_ids) {
  if (!c || (n > 0 && !job_ids) || n < 0) return fail(NFHMM_EINVAL, "NULL argument or n < 0");
  std::vector<char> gone(c->jobs.size(), 0);
  for (int i = 0; i < n; ++i) {
    const int j = find_job(c, job_ids[i]);
    if (j < 0) return fail(NFHMM_EINVAL, "no job " + std::to_string(job_ids[i]) + " in the batch");
    gone[j] = 1;
  }
  return remove_jobs(c, gone);
}

int nfhmm_batch_info(nfhmm_ctx* c, int* n_jobs, int* frames_held, long long* ids, int* t0,
                     int* T, int* sweeps) {
  if (!c) return fail(NFHMM_EINVAL, "NULL context");
  if (n_jobs) *n_jobs = (int)c->jobs.size();
  if (frames_held) *frames_held = c->T_active;
  for (size_t j = 0; j < c->jobs.size(); ++j) {
    if (ids) ids[j] = c->jobs[j].id;
    if (t0) t0[j] = c->jobs[j].t0;
    if (T) T[j] = c->jobs[j].T;
    if (sweeps) sweeps[j] = c->jobs[j].sweeps;
  }
  return NFHMM_OK;
}

int nfhmm_job_bounds(nfhmm_ctx* c, double* bounds) {
  if (!c || !bounds) return fail(NFHMM_EINVAL, "NULL argument");
  if (need_inputs(c)) return NFHMM_ESTATE;
  const int rc = sweep_impl(c, 0, true);
  if (rc) return rc;
  for (size_t j = 0; j < c->jobs.size(); ++j) bounds[j] = c->h_bound[j];
  return NFHMM_OK;
}

int nfhmm_job_posteriors(nfhmm_ctx* c, long long job_id, float* dhat, int on_device) {
  if (!c || !dhat) return fail(NFHMM_EINVAL, "NULL argument");
  if (need_inputs(c)) return NFHMM_ESTATE;
  const int j = find_job(c, job_id);
  if (j < 0) return fail(NFHMM_EINVAL, "no job " + std::to_string(job_id) + " in the batch");
  int rc = enter(c);
  if (rc) return rc;
  rc = copy_slices(c, dhat, c->dhat, c->d.N, true, c->jobs[j].t0, c->jobs[j].T, on_device);
  if (rc) return rc;
  if (!on_device) {
    rc = sync_check(c);
    if (rc) return rc;
  }
  return leave(c);
}

int nfhmm_autotune(nfhmm_ctx* c, int reps, int* chunk_out, int* group_out, double* us_out) {
  using namespace nfhmm;
  if (!c) return fail(NFHMM_EINVAL, "NULL context");
  if (c->jobs.empty() || !c->have_alpha)
    return fail(NFHMM_ESTATE, "autotune times sweeps from the current state: run a sweep over "
                              "the current jobs first");
  if (reps <= 0) reps = 3;
  int longest = 0;
  for (const Job& j : c->jobs) longest = j.T > longest ? j.T : longest;
  const int oldL = c->fb.L, oldG = c->fb.G, old_seq = c->fb.seq;
  const bool old_auto = c->group_auto;
  const bool old_prof = c->profiling;
  int rc = enter(c);
  if (rc) return rc;
  // the bound of the current state is formed now (the trials overwrite the
  // weights it would be formed from later)
  if (!c->bound_ok) {
    if (!c->bpart_ok) {
      rc = contract(c, true, false, 0, c->T_active);
      if (rc) return rc;
      c->bpart_ok = true;
    }
    rc = compute_bound(c);
    if (rc) return rc;
  }
  CK(cudaStreamSynchronize(c->s_main));
  const nfhmm_dims& d = c->d;
  // a sweep reads only the counts and the posteriors (and the inputs); the
  // bound and the separation also read alpha-hat and the log normalisers.
  // Copies of those four are taken first: every trial starts from them and
  // they are put back at the end.
  void* live[4] = {c->c, c->dhat, c->alpha, c->logZ};
  const size_t bytes[4] = {(size_t)c->T_active * c->Mp * sizeof(float),
                           (size_t)d.S * d.T * d.N * sizeof(float),
                           (size_t)c->T_active * c->Mp * sizeof(float),
                           (size_t)d.S * c->max_jobs * sizeof(double)};
  void* saved[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto cleanup = [&]() {
    for (void* b : saved)
      if (b) cudaFree(b);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  };
  const bool f_alpha = c->have_alpha, f_bpart = c->bpart_ok, f_fterm = c->fterm_ok,
             f_bound = c->bound_ok;
  bool got = cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess;
  for (int i = 0; i < 4 && got; ++i) got = cudaMalloc(&saved[i], bytes[i]) == cudaSuccess;
  if (!got) {
    cleanup();
    cudaGetLastError();
    return fail(NFHMM_ENOMEM, "autotune: no room for a copy of the state");
  }
  auto copy_state = [&](bool save) -> cudaError_t {
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 4 && e == cudaSuccess; ++i)
      e = cudaMemcpyAsync(save ? saved[i] : live[i], save ? live[i] : saved[i], bytes[i],
                          cudaMemcpyDeviceToDevice, c->s_main);
    return e;
  };
  auto finish = [&](int code) {
    copy_state(false);
    cudaStreamSynchronize(c->s_main);
    cleanup();
    c->have_alpha = f_alpha;
    c->bpart_ok = f_bpart;
    c->fterm_ok = f_fterm;
    c->bound_ok = f_bound;
    c->profiling = old_prof;
    return code;
  };
  if (copy_state(true) != cudaSuccess) return finish(fail(NFHMM_ECUDA, "autotune: state copy"));
  c->profiling = false;
  // candidates: (chunk length, group size, 0) for the scan, then
  // (-, -, k) for the sequential form with k chains per block
  struct Cand {
    int L, G, seq;
  };
  std::vector<Cand> cands;
  const int cand_L[] = {8, 12, 16, 20, 24, 32, 48, 64};
  for (int L : cand_L) {
    if (L > longest && L != cand_L[0]) continue;
    const int G = fb_default_group((longest + L - 1) / L);
    cands.push_back({L, G, 0});
    if (G != 0) cands.push_back({L, 0, 0});   // and without groups
  }
  const int chains = c->d.S * (int)c->jobs.size(), mcpc = fb_seq_max_cpc(c->d.N);
  for (int k = 1; k <= mcpc; k *= 2) {
    if (k / 2 >= chains) break;   // one block already holds every chain
    cands.push_back({0, 0, k});
  }
  c->fb.seq = 0;
  int bestL = oldL, bestG = oldG, best_seq = old_seq;
  double best_us = 1e300;
  // two sweeps from the saved state capture the candidate's graph, then
  // `reps` sweeps are timed; rc: an error code, us: mean sweep time
  auto time_sweeps = [&](double* us) -> int {
    cudaError_t e = copy_state(false);
    int r = NFHMM_OK;
    if (e == cudaSuccess) r = run_sweeps(c, 2, false);
    if (e == cudaSuccess && !r) e = cudaEventRecord(e0, c->s_main);
    if (e == cudaSuccess && !r) r = run_sweeps(c, reps, false);
    if (e == cudaSuccess && !r) e = cudaEventRecord(e1, c->s_main);
    if (e == cudaSuccess && !r) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess && !r) e = cudaEventElapsedTime(&ms, e0, e1);
    if (r) return r;
    if (e != cudaSuccess) return fail(NFHMM_ECUDA, std::string("autotune: ") + cudaGetErrorString(e));
    *us = 1e3 * ms / reps;
    return NFHMM_OK;
  };
  for (const Cand& cd : cands) {
    {
      const int L = cd.seq ? c->fb.L : cd.L, G = cd.seq ? c->fb.G : cd.G;
      if (cd.seq) {
        // the sequential form (its scratch on first use; none: not a candidate)
        if (set_fb_mode(c, cd.seq) != NFHMM_OK) {
          cudaGetLastError();
          set_last_error("");
          continue;
        }
      } else {
        c->fb.L = L;
        c->fb.G = G;
        rc = ensure_fb_capacity(c);
        if (!rc) rc = commit_jobs(c);
        if (rc) return finish(rc);
      }
      double us = 0.0;
      rc = time_sweeps(&us);
      if (rc) return finish(rc);
      if (us < best_us) {
        best_us = us;
        bestL = L;
        bestG = G;
        best_seq = cd.seq;
      }
      set_fb_mode(c, 0);
    }
  }
  c->fb.L = bestL;
  c->fb.G = bestG;
  c->group_auto = false;
  rc = ensure_fb_capacity(c);
  if (!rc) rc = commit_jobs(c);
  if (!rc) rc = set_fb_mode(c, best_seq);
  if (rc) {
    c->fb.L = oldL;
    c->fb.G = oldG;
    c->group_auto = old_auto;
    set_fb_mode(c, old_seq);
    return finish(rc);
  }
  // the contractions' tile shapes beside the chosen form, one coordinate at
  // a time (column tile of each contraction, then each ring depth), starting
  // from the current shape, whose time under this form is measured first
  if (c->use_tc) {
    // shape: column tile, ring depth and staged epilogue operand of each
    // contraction, as {bn1, bn2, st1, st2, ep1, ep2}
    const int o[6] = {c->tc.bn1, c->tc.bn2, c->tc.st1, c->tc.st2, c->tc.ep1, c->tc.ep2};
    int b[6] = {o[0], o[1], o[2], o[3], o[4], o[5]};
    double t_best = 0.0;
    rc = time_sweeps(&t_best);
    const int order[6] = {0, 1, 4, 5, 2, 3};
    for (int oi = 0; oi < 6 && !rc; ++oi) {
      const int coord = order[oi];
      std::vector<int> vals;
      if (coord < 2) {
        int cand[8];
        const int n = tc_tile_candidates(c->tc.precision, coord, cand, 8);
        vals.assign(cand, cand + n);
      } else if (coord >= 4) {
        vals = {0, 1};
      } else {
        const int m = tc_max_stages(c->tc.precision, b[coord - 2], b[coord + 2] != 0);
        for (int st = 2; st < m; ++st) vals.push_back(st);   // m itself is depth 0
        vals.push_back(0);
      }
      for (int v : vals) {
        if (v == b[coord]) continue;
        int t[6] = {b[0], b[1], b[2], b[3], b[4], b[5]};
        t[coord] = v;
        // a new column tile or epilogue staging starts from the deepest ring it allows
        if (coord < 2) t[2 + coord] = 0;
        if (coord >= 4) t[coord - 2] = 0;
        if (tc_set_tiles(c->tc, t[0], t[1], t[2], t[3], t[4], t[5]) != 0) continue;
        double us = 0.0;
        rc = time_sweeps(&us);
        if (rc) break;
        if (us < t_best) {
          t_best = us;
          for (int i = 0; i < 6; ++i) b[i] = t[i];
        }
      }
    }
    // then the L2 prefetch distance of each contraction
    const int opf1 = c->tc.pf1, opf2 = c->tc.pf2;
    if (!rc && tc_set_tiles(c->tc, b[0], b[1], b[2], b[3], b[4], b[5]) != 0)
      rc = fail(NFHMM_ECUDA, "autotune: tile shape: " + tc_last_error());
    for (int which = 0; which < 2 && !rc; ++which) {
      int& pf = which == 0 ? c->tc.pf1 : c->tc.pf2;
      const int keep = pf;
      int best_pf = keep;
      const int dists[] = {0, 4, 8, 16};
      for (int d : dists) {
        if (d == keep) continue;
        pf = d;
        double us = 0.0;
        rc = time_sweeps(&us);
        if (rc) break;
        if (us < t_best) {
          t_best = us;
          best_pf = d;
        }
      }
      pf = best_pf;
    }
    if (rc) {
      c->tc.pf1 = opf1;
      c->tc.pf2 = opf2;
    }
    if (rc || tc_set_tiles(c->tc, b[0], b[1], b[2], b[3], b[4], b[5]) != 0) {
      tc_set_tiles(c->tc, o[0], o[1], o[2], o[3], o[4], o[5]);
      if (!rc) rc = fail(NFHMM_ECUDA, "autotune: tile shape: " + tc_last_error());
      return finish(rc);
    }
    best_us = t_best;
  }
  rc = finish(NFHMM_OK);
  if (rc) return rc;
  rc = sync_check(c);   // a trial's error word (none expected from a valid state)
  if (rc) return rc;
  if (chunk_out) *chunk_out = bestL;
  if (group_out) *group_out = bestG;
  if (us_out) *us_out = best_us;
  return leave(c);
}

int nfhmm_set_option(nfhmm_ctx* c, int key, long long value) {
  if (!c) return fail(NFHMM_EINVAL, "NULL context");
  switch (key) {
    case NFHMM_OPT_FB_CHUNK:
    case NFHMM_OPT_FB_GROUP: {
      if (key == NFHMM_OPT_FB_CHUNK && (value < 1 || value > 128))
        return fail(NFHMM_EINVAL, "chunk length must be in [1, 128]");
      if (key == NFHMM_OPT_FB_GROUP && (value < -1 || value == 1 || value > 4096))
        return fail(NFHMM_EINVAL, "group size must be -1 (automatic), 0 (none) or 2..4096");
      const int oldL = c->fb.L, oldG = c->fb.G;
      const bool old_auto = c->group_auto;
      if (key == NFHMM_OPT_FB_CHUNK) c->fb.L = (int)value;
      if (key == NFHMM_OPT_FB_GROUP) c->group_auto = value < 0;
      if (c->group_auto) {
        c->fb.G = fb_default_group((c->d.T + c->fb.L - 1) / c->fb.L);
      } else if (key == NFHMM_OPT_FB_GROUP) {
        c->fb.G = (int)value;
      }
      int rc = ensure_fb_capacity(c);
      if (rc) {
        c->fb.L = oldL;
        c->fb.G = oldG;
        c->group_auto = old_auto;
        return rc;
      }
      rc = enter(c);
      if (!rc) rc = commit_jobs(c);
      if (!rc) rc = leave(c);
      return rc;
    }
    case NFHMM_OPT_FB_PRODUCTS: {
      if (value != NFHMM_FB_PRODUCTS_SIMT && value != NFHMM_FB_PRODUCTS_TC)
        return fail(NFHMM_EINVAL, "products must be NFHMM_FB_PRODUCTS_SIMT or _TC");
      c->fb.products = value == NFHMM_FB_PRODUCTS_TC ? FB_PRODUCTS_TC : FB_PRODUCTS_SIMT;
      return NFHMM_OK;
    }
    case NFHMM_OPT_GRAPHS: {
      c->use_graphs = value != 0;
      return NFHMM_OK;
    }
    case NFHMM_OPT_FB_MODE: {
      if (value < 0 || value > 64)
        return fail(NFHMM_EINVAL, "forward-backward mode must be 0 (scan) or 1..64 (sequential)");
      return set_fb_mode(c, (int)value);
    }
    case NFHMM_OPT_TILE_GEMM1:
    case NFHMM_OPT_TILE_GEMM2:
    case NFHMM_OPT_TILE_STAGES1:
    case NFHMM_OPT_TILE_STAGES2:
    case NFHMM_OPT_TILE_EPI_STAGE1:
    case NFHMM_OPT_TILE_EPI_STAGE2: {
      if (!c->use_tc) return fail(NFHMM_EINVAL, "tile shapes apply to tensor-core contexts");
      if (value < 0 || value > 1024) return fail(NFHMM_EINVAL, "tile option out of range");
      int bn1 = c->tc.bn1, bn2 = c->tc.bn2, st1 = c->tc.st1, st2 = c->tc.st2;
      int ep1 = c->tc.ep1, ep2 = c->tc.ep2;
      if (key == NFHMM_OPT_TILE_GEMM1) bn1 = (int)value;
      if (key == NFHMM_OPT_TILE_GEMM2) bn2 = (int)value;
      if (key == NFHMM_OPT_TILE_STAGES1) st1 = (int)value;
      if (key == NFHMM_OPT_TILE_STAGES2) st2 = (int)value;
      if (key == NFHMM_OPT_TILE_EPI_STAGE1 || key == NFHMM_OPT_TILE_EPI_STAGE2) {
        if (value > 1) return fail(NFHMM_EINVAL, "epilogue staging is 0 or 1");
        (key == NFHMM_OPT_TILE_EPI_STAGE1 ? ep1 : ep2) = (int)value;
      }
      // a new column tile or staging keeps the depth only if it can hold it
      // (else the deepest); a depth asked for explicitly is validated as given
      if ((key == NFHMM_OPT_TILE_GEMM1 || key == NFHMM_OPT_TILE_EPI_STAGE1) &&
          st1 > tc_max_stages(c->tc.precision, bn1, ep1 != 0))
        st1 = 0;
      if ((key == NFHMM_OPT_TILE_GEMM2 || key == NFHMM_OPT_TILE_EPI_STAGE2) &&
          st2 > tc_max_stages(c->tc.precision, bn2, ep2 != 0))
        st2 = 0;
      int rc = enter(c);   // the plan's maps are read by launches already queued
      if (rc) return rc;
      CK(cudaStreamSynchronize(c->s_main));
      CK(cudaStreamSynchronize(c->s_aux));
      if (tc_set_tiles(c->tc, bn1, bn2, st1, st2, ep1, ep2) != 0)
        return fail(NFHMM_EINVAL, "tile shape: " + tc_last_error());
      c->bpart_ok = false;   // the bound's partials are counted per tile shape
      c->bound_ok = false;
      return leave(c);
    }
    case NFHMM_OPT_TILE_PREFETCH1:
    case NFHMM_OPT_TILE_PREFETCH2: {
      if (!c->use_tc) return fail(NFHMM_EINVAL, "tile options apply to tensor-core contexts");
      if (value < 0 || value > 64) return fail(NFHMM_EINVAL, "prefetch distance must be in [0, 64]");
      (key == NFHMM_OPT_TILE_PREFETCH1 ? c->tc.pf1 : c->tc.pf2) = (int)value;
      return NFHMM_OK;
    }
    case NFHMM_OPT_TEST_WAIT_TIMEOUT: {
      if (!c->use_tc) return fail(NFHMM_EINVAL, "the wait hook needs a tensor-core context");
      if (value < 0 || value > 1000000000)
        return fail(NFHMM_EINVAL, "wait hook must be 0 or 1..10^9 nanoseconds");
      c->inject_wait_ns = (unsigned long long)value;
      return NFHMM_OK;
    }
    case NFHMM_OPT_PROFILE_STRIDE: {
      if (value < 1 || value > 1000000) return fail(NFHMM_EINVAL, "profile stride must be >= 1");
      c->prof_stride = (int)value;
      return NFHMM_OK;
    }
    default: return fail(NFHMM_EINVAL, "unknown option key");
  }
}

int nfhmm_vi_reinit(nfhmm_ctx* c, const float* V, const float* W, const float* A,
                    const float* pi, int inputs_on_device) {
  if (!c || !V || !W || !A || !pi) return fail(NFHMM_EINVAL, "NULL argument");
  c->inputs_ok = false;
  c->sweeps_done = 0;
  c->have_alpha = false;
  c->bpart_ok = false;
  c->fterm_ok = false;
  c->bound_ok = false;
  std::vector<int> frames;
  for (Job& j : c->jobs) {
    j.sweeps = 0;
    frames.push_back(j.T);
  }
  int rc = enter(c);
  if (rc) return rc;
  CK(cudaMemsetAsync(c->err, 0, 4, c->s_main));
  rc = load_model(c, W, A, pi, inputs_on_device);
  if (rc) return rc;
  std::vector<const float*> Vs(frames.size());
  for (size_t j = 0, t = 0; j < frames.size(); t += frames[j], ++j) Vs[j] = V + t * c->d.F;
  rc = load_frames(c, 0, c->T_active, Vs.data(), inputs_on_device, frames.data(),
                   (int)frames.size());
  if (rc) return rc;
  rc = sync_check(c);
  if (rc) return rc;
  c->inputs_ok = true;
  return leave(c);
}

int nfhmm_vi_sweep(nfhmm_ctx* c, int n_sweeps, double* bound_out) {
  if (!c) return fail(NFHMM_EINVAL, "NULL context");
  if (need_inputs(c)) return NFHMM_ESTATE;
  if (n_sweeps < 0) return fail(NFHMM_EINVAL, "n_sweeps must be >= 0");
  const int rc = sweep_impl(c, n_sweeps, bound_out != nullptr);
  if (rc) return rc;
  if (bound_out) *bound_out = c->h_bound[c->jobs.size()];
  return NFHMM_OK;
}

int nfhmm_vi_sweep_async(nfhmm_ctx* c, int n_sweeps, int prepare_bound) {
  if (!c) return fail(NFHMM_EINVAL, "NULL context");
  if (need_inputs(c)) return NFHMM_ESTATE;
  if (n_sweeps < 1) return fail(NFHMM_EINVAL, "n_sweeps must be >= 1");
  return sweep_impl(c, n_sweeps, prepare_bound != 0, false);
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
  const size_t T = c->T_active, F = d.F, S = d.S;
  int rc = enter(c);
  if (rc) return rc;
  cudaStream_t st = c->s_main;
  if (!c->wts) CK(dmalloc(c, (void**)&c->wts, (size_t)d.T * c->Mp * 4));
  float* dst = out;
  if (!out_on_device) {
    if (!c->sep_tmp) CK(dmalloc(c, (void**)&c->sep_tmp, S * (size_t)d.T * F * 4));
    dst = c->sep_tmp;
  }
  launch_sep_weights(c->alpha, c->v, (int)T, c->M, c->Mp, weights, c->wts, st);
  c->launches += 1;
  for (int s = 0; s < d.S; ++s) {
    GemmArgs g{};
    g.rows = (int)T;
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
    launch_sep_mask(c->V, c->Fp, dst, d.S, (int)T, d.F, st);
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
  rc = copy_slices(c, dhat, c->dhat, c->d.N, true, 0, c->T_active, on_device);
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
  if (c->T_active > 0)
    CK(cudaMemcpy2DAsync(dst, (size_t)c->M * 4, src, (size_t)c->Mp * 4, (size_t)c->M * 4,
                         (size_t)c->T_active,
                         on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDefault, c->s_main));
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
  rc = copy_slices(c, phi, c->phi, c->d.N, true, 0, c->T_active, on_device);
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
  if (c->T_active > 0)
    CK(cudaMemcpy2DAsync(c->c, (size_t)c->Mp * 4, counts, (size_t)c->M * 4, (size_t)c->M * 4,
                         (size_t)c->T_active, kind, c->s_main));
  rc = copy_slices(c, c->dhat, dhat, c->d.N, false, 0, c->T_active, on_device);
  if (rc) return rc;
  if (!on_device) {
    rc = sync_check(c);
    if (rc) return rc;
  }
  c->sweeps_done = sweeps_done;
  for (Job& j : c->jobs) j.sweeps = sweeps_done;
  c->have_alpha = false;
  c->bpart_ok = false;
  c->fterm_ok = false;
  c->bound_ok = false;
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
  a.nchains = 1;   // one chain over all T frames (null chain tables)
  a.products = FB_PRODUCTS_TC;
  a.G = fb_default_group(a.C);
  a.NG = a.G >= 2 ? (a.C + a.G - 1) / a.G : 0;
  a.phi = phi;
  a.A = A;
  a.pi = pi;
  a.dhat = dhat;
  a.logZ = logZ;
  void* scratch = nullptr;
  const size_t bytes = fb_scratch_bytes(S, N, a.C, a.NG) + 256;
  CK(cudaMallocAsync(&scratch, bytes, st));
  fb_carve_scratch(a, scratch);
  a.err = reinterpret_cast<unsigned*>(reinterpret_cast<char*>(scratch) + bytes - 256);
  CK(cudaMemsetAsync(a.err, 0, 4, st));
  cudaError_t le = launch_fb(a, st, nullptr);
  if (le == cudaSuccess) {
    launch_flag_errors(a.err, logZ, S, st);   // a device-side failure: logZ NaN
    le = cudaGetLastError();
  }
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
  for (auto& g : c->graphs) harvest(c, g);
  StageEvents& s = c->stages[stage];
  double tot = s.ms_acc;
  const size_t n = s.begin.size() < s.end.size() ? s.begin.size() : s.end.size();
  for (size_t i = 0; i < n; ++i) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, s.begin[i], s.end[i]));
    tot += ms;
  }
  if (ms_total) *ms_total = tot;
  if (invocations) *invocations = (long long)n + s.inv_acc;
  if (launches) *launches = s.launches;
  if (reset) {
    for (auto e : s.begin) cudaEventDestroy(e);
    for (auto e : s.end) cudaEventDestroy(e);
    s.begin.clear();
    s.end.clear();
    s.launches = 0;
    s.ms_acc = 0.0;
    s.inv_acc = 0;
  }
  return NFHMM_OK;
}

long long nfhmm_kernel_launches(nfhmm_ctx* c) { return c ? c->launches : 0; }

int nfhmm_query(nfhmm_ctx* c, int key, long long* value) {
  if (!c || !value) return fail(NFHMM_EINVAL, "NULL argument");
  switch (key) {
    case NFHMM_Q_TENSOR_CORES: *value = c->use_tc ? 1 : 0; return NFHMM_OK;
    case NFHMM_Q_FB_CHUNK: *value = c->fb.L; return NFHMM_OK;
    case NFHMM_Q_FB_GROUP: *value = c->fb.G; return NFHMM_OK;
    case NFHMM_Q_FB_MODE: *value = c->fb.seq; return NFHMM_OK;
    case NFHMM_Q_TILE_GEMM1: *value = c->use_tc ? c->tc.bn1 : 0; return NFHMM_OK;
    case NFHMM_Q_TILE_GEMM2: *value = c->use_tc ? c->tc.bn2 : 0; return NFHMM_OK;
    case NFHMM_Q_TILE_STAGES1:
      *value = !c->use_tc ? 0
               : c->tc.st1 ? c->tc.st1
                           : tc_max_stages(c->tc.precision, c->tc.bn1, c->tc.ep1 != 0);
      return NFHMM_OK;
    case NFHMM_Q_TILE_PREFETCH1: *value = c->use_tc ? c->tc.pf1 : 0; return NFHMM_OK;
    case NFHMM_Q_TILE_EPI_STAGE1: *value = c->use_tc ? c->tc.ep1 : 0; return NFHMM_OK;
    case NFHMM_Q_TILE_EPI_STAGE2: *value = c->use_tc ? c->tc.ep2 : 0; return NFHMM_OK;
    case NFHMM_Q_TILE_PREFETCH2: *value = c->use_tc ? c->tc.pf2 : 0; return NFHMM_OK;
    case NFHMM_Q_TILE_STAGES2:
      *value = !c->use_tc ? 0
               : c->tc.st2 ? c->tc.st2
                           : tc_max_stages(c->tc.precision, c->tc.bn2, c->tc.ep2 != 0);
      return NFHMM_OK;
    case NFHMM_Q_SWEEPS_DONE: *value = c->sweeps_done; return NFHMM_OK;
    case NFHMM_Q_DEVICE_BYTES: *value = (long long)c->device_bytes; return NFHMM_OK;
    case NFHMM_Q_FRAME_CAPACITY: *value = c->d.T; return NFHMM_OK;
    case NFHMM_Q_MAX_JOBS: *value = c->max_jobs; return NFHMM_OK;
    default: return fail(NFHMM_EINVAL, "unknown query key");
  }
}

}  // extern "C"
