// Host-side launchers of the library's kernels (internal).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>

namespace nfhmm {

// Error word bits set by kernels (read by the host after a synchronise).
enum : unsigned {
  ERR_VHAT_ZERO = 1u,  // Vhat <= 0 (or not finite) where V > 0
  ERR_NONFINITE = 2u,  // NaN/Inf in a state array
  ERR_BAD_INPUT = 4u,  // input validation failed
  ERR_FB_ZERO = 8u,    // forward-backward normaliser vanished
  ERR_TIMEOUT = 16u,   // a bounded device wait gave up
};

// Records the calling thread's last error message (returned by nfhmm_last_error).
void set_last_error(const std::string& msg);

// Formats of the weight operand w = exp(psi(alpha)) written by the weights kernel.
enum WFormat { WF_F32 = 0, WF_TF32X2 = 1, WF_BF16 = 2 };

struct WeightsArgs {
  int T, M, Mp, S, N, K;
  int Tstride;          // frame stride of d-hat and phi-hat (S x Tstride x N)
  float gamma;
  const int2* ktab;     // Mp entries: (s, n) of element k ((0, 0) for padding)
  const float* counts;  // T x Mp
  const float* dhat;    // S x T x N
  float* alpha;         // T x Mp, or null: alpha-hat not stored (not the last sweep of a run)
  float* w32;           // T x Mp, w in float (always written)
  void* wop_hi;         // format-specific operand copies (may be null)
  void* wop_lo;
  float* phi;           // S x T x N (without the -gamma K psi(alpha_t0) constant)
  double* fterm;        // null, or T x weights_units(S, N, K, Tstride) x 2: per unit of the frame,
                        // (sum_k alpha_tk, sum_k g(alpha_tk)) for the bound
  unsigned* err;
  // set by launch_weights for the slab form: units per warp, and the
  // multipliers ceil(2^16 / K) and ceil(2^32 / N) of its exact divisions
  int upw;
  unsigned kdiv;
  unsigned long long ndiv;
};
void launch_weights(const WeightsArgs& a, int fmt, cudaStream_t st);
// units per frame of the weights kernel's bound sums (T: frame capacity)
int weights_units(int S, int N, int K, int T);
void launch_element_table(int M, int Mp, int K, int N, int2* ktab, cudaStream_t st);

// Fill buf[t*ld + k] = (k < M) ? value : 0 for t < T, k < ld.
void launch_fill_rows(float* buf, int T, int M, int ld, float value, cudaStream_t st);
void launch_fill(float* buf, size_t n, float value, cudaStream_t st);

// v[t] = sum_l V[t*Fp + l] in double.
void launch_row_sums(const float* V, int T, int F, int Fp, double* v, cudaStream_t st);

// Validation of V (T x Fp, first F columns), W (M x Fp), A (S*N rows of N), pi (S rows of N).
void launch_validate(const float* V, int T, int F, int Fp, const float* W, int M, const float* A,
                     const float* pi, int S, int N, unsigned* err, cudaStream_t st);

// out[c*ldo + r] = in[r*ldi + c] for r < R, c < Cc; zero elsewhere up to (Cp, Rp).
void launch_transpose(const float* in, int R, int Cc, int ldi, float* out, int ldo, int Rp, int Cp,
                      cudaStream_t st);

// Simple split copies used by the tensor-core path.
void launch_split_tf32(const float* in, float* hi, float* lo, size_t n, cudaStream_t st);
// rows of F floats, packed in src, into rows of Fp in dst (padding zero).
void launch_pad_rows(const float* src, int rows, int F, float* dst, int Fp, cudaStream_t st);
// b_l = sum_k W[k][l] (the initial state's reconstruction, every weight 1).
void launch_col_sums(const float* W, int M, int Fp, float* b, cudaStream_t st);
// Q = V / b_l on T frames (T x Fp), as float (out) and/or split tf32 hi / lo.
void launch_init_ratio(const float* V, const float* b, int T, int Fp, float* out, float* hi,
                       float* lo, unsigned* err, cudaStream_t st);

void launch_to_bf16(const float* in, void* out, size_t n, cudaStream_t st);

// SIMT FP32 contraction C[t][n] = sum_k A[t][k] B[n][k] with epilogues.
enum Epilogue { EPI_RATIO = 0, EPI_SCALE = 1, EPI_STORE = 2 };
struct GemmArgs {
  int rows, cols, kdim;
  const float* A; int lda;
  const float* B; int ldb;
  // EPI_RATIO: Q = V / C (0 where V == 0), bound partial V log C per (row, column tile)
  const float* V; int ldv;
  float* out; int ldo;           // Q (RATIO), counts (SCALE), output (STORE)
  const float* w; int ldw;       // SCALE: out = w * C
  double* bpart; int nbpart;     // RATIO: bpart[row * nbpart + column tile] (may be null)
  unsigned* err;
};
void launch_gemm_simt(const GemmArgs& g, int epi, cudaStream_t st);
int gemm_simt_col_tiles(int cols);

// Forward-backward, parallel in time over chunks of L frames.  The frames
// hold one or more independent chains (jobs) back to back; no chunk crosses
// a chain boundary and each chain's first chunk starts from pi.  With null
// chain tables there is one chain covering all T frames.
// how the chunk matrices are formed: FP32 FMAs on the CUDA cores (lowest
// latency per frame) or split-TF32 tcgen05 MMAs (a 128-row tile per step)
enum { FB_PRODUCTS_SIMT = 0, FB_PRODUCTS_TC = 1 };
struct FBArgs {
  int S, N, T, L, C;   // C = total chunks per source over all chains
  int products;        // FB_PRODUCTS_SIMT or FB_PRODUCTS_TC
  // 1: A and pi are the caller's own stable copies, so the first pass may read
  // them before its wait for the kernel that wrote the emissions (a sweep);
  // 0: every input may have been written by that kernel (stateless calls)
  int inputs_stable;
  int nchains;
  // seq > 0: the sequential form instead of the scan (one warp per chain and
  // direction, blocks of `seq` chains; the chunk geometry is then unused);
  // maxlen = frames of the longest chain; beta: S x T x N backward vectors;
  // emis: S x T x 68 prepared emission rows
  int seq, maxlen;
  float* beta;
  float* emis;
  const int* chain_c0;     // nchains + 1: first chunk of each chain (chain_c0[nchains] = C)
  const int* chain_t0;     // nchains: first frame of each chain
  const int* chain_len;    // nchains: frames of each chain
  const int* chunk_chain;  // C: chain of each chunk
  const float* phi;  // S x T x N
  const float* A;    // S x N x N row-stochastic
  const float* pi;   // S x N
  float* dhat;       // S x T x N
  double* logZ;      // S x nchains
  // scratch
  float* P;          // S x C x NP x NP   chunk matrices, row-major (NP = 8*ceil(N/8))
  float* PT;         // S x C x NP x NP   the same, transposed
  double* Plog;      // S x C            log of each chunk matrix's scale
  float* fwd;        // S x C x N        forward boundary vectors
  float* lam;        // S x C            forward scan normalisers
  float* bwd;        // S x C x N        backward boundary vectors
  // Groups of G consecutive chunks of a chain (G >= 2; 0 = no groups): the
  // scan across chunks becomes group products, a scan across groups and a
  // replay of each group's chunk boundaries.  Group g covers chunks
  // [grp_c0[g], grp_c0[g+1]); null tables: one chain, groups of G.
  int G, NG;
  const int* grp_c0;    // NG + 1
  const int* chain_g0;  // nchains + 1: first group of each chain
  float* Q;             // S x NG x NP x NP  group products (rows scaled to a common scale)
  float* QT;            // S x NG x NP x NP  the same, transposed
  double* Qlog;         // S x NG            log of each group product's scale
  float* gfwd;          // S x NG x N        forward vectors at group ends
  float* gbwd;          // S x NG x N        backward vectors at group ends
  float* glam;          // S x NG            group scan normalisers
  uint8_t* Pimg;        // S x C chunk matrices as split tf32 operand images (groups only)
  unsigned* err;
};
// chunks of L frames needed by chains of the given lengths
int fb_chunk_count(const int* chain_len, int nchains, int L);
size_t fb_scratch_bytes(int S, int N, int C, int NG);
size_t fb_image_bytes(int N);   // bytes of one chunk's operand image
void fb_carve_scratch(FBArgs& a, void* base);   // regions for a.C chunks and a.NG groups
int fb_default_chunk(int N, int T);
// group size for chains of about C chunks (0: no groups)
int fb_default_group(int C);
int fb_max_states();
// sequential form: the most chains a block can hold for N states, and the
// blocks a launch over `chains` (source, chain) pairs takes
int fb_seq_max_cpc(int N);
int fb_seq_blocks(int chains, int cpc, int N);
cudaError_t launch_fb(const FBArgs& a, cudaStream_t st, int* launches);

// Bound.
struct BoundArgs {
  int T, M, Mp, S, K;
  int njobs;
  const int* job_t0;       // njobs + 1 frame offsets (device)
  float gamma;
  double konst;            // lnGamma(M + gamma S K) - S K lnGamma(1 + gamma)
  const float* alpha;      // T x Mp
  const double* v;         // T
  const double* bpart; int nbpart;   // bpart: T x nbpart (row stride)
  int nbpart_used;         // partials per frame the contraction that formed them wrote
  const double* fterm;     // null, or T x funits x 2 per-unit sums from the weights kernel
  int funits;
  const double* logZ;      // S x njobs
  double* frame_terms;     // T
  double* out;             // njobs + 1: per-job bounds, then their sum
};
void launch_bound(const BoundArgs& a, cudaStream_t st, int* launches);

// Separation helpers.
void launch_sep_weights(const float* alpha, const double* v, int T, int M, int Mp, int mode,
                        float* wts, cudaStream_t st);
void launch_sep_mask(const float* V, int Fp, float* out, int S, int T, int F, cudaStream_t st);

// Stateless calls: every logZ[i], i < n, becomes NaN if the error word is set.
void launch_flag_errors(const unsigned* err, double* logZ, int n, cudaStream_t st);

// Digamma test entry.
void launch_digamma(const float* x, float* psi, float* w, size_t n, cudaStream_t st);

// Compaction of a batch's frame store: destination frames [base, base +
// frames) come from segments (dst first frame, source offset, length) of a
// copy of the old frames [base, ...) held in the *s buffers.
struct FrameMove {
  int nseg;
  const int* seg;   // 3 * nseg
  int frames, base, Tc, Fp, Mp, SN, N, S;
  float* V; const float* Vs;        // Fp per frame
  float* c; const float* cs;        // Mp per frame
  float* dhat; const float* ds;     // S x (Tc frames x N)
  double* v; const double* vs;
};
void launch_move_frames(const FrameMove& m, cudaStream_t st);

// Prior marginals dhat[s][t] = pi A^(t - t0(job)) restarted at every job
// (sequential in t, one block per (source, job)).  job_t0: njobs + 1 device
// offsets, or null for the single job [t_begin, t_end).  T: frame stride.
void launch_prior_marginals(const float* A, const float* pi, int S, int N, int T,
                            const int* job_t0, int njobs, int t_begin, int t_end, float* dhat,
                            cudaStream_t st);

}  // namespace nfhmm
