// Tensor-core (tcgen05 + TMEM + TMA) form of the two contractions (internal).
#pragma once

#include <cuda_runtime.h>

#include <string>

namespace nfhmm {

struct TcPlan {
  int precision = 0;   // NFHMM_FP32 (split TF32, three passes) or NFHMM_BF16
  int w_format = 0;    // WFormat the weights kernel must write
  int T = 0, M = 0, Mp = 0, F = 0, Fp = 0;
  // operand copies owned by the plan
  void* w_hi = nullptr;   // T x Mp  (tf32 hi as float, or bf16)
  void* w_lo = nullptr;   // T x Mp  (tf32 lo as float; null for bf16)
  void* q_hi = nullptr;   // T x Fp
  void* q_lo = nullptr;
  void* bF_hi = nullptr;  // Fp x Mp  (beta by frequency)
  void* bF_lo = nullptr;
  void* bM_hi = nullptr;  // Mp x Fp  (beta by element)
  void* bM_lo = nullptr;
  // borrowed from the context
  const float* bF_src = nullptr;  // beta by frequency (Fp x Mp), float
  const float* bM_src = nullptr;  // beta by element (Mp x Fp), float
  int nbpart = 0;                 // columns of the bound-partial array
  // tile shape: column tile of each contraction, and its shared-memory ring
  // depth (0: the deepest that fits); see tc_set_tiles
  int bn1 = 128, bn2 = 160, st1 = 0, st2 = 0;
  // L2 prefetch distance of each contraction's operand loads, in K-blocks (0: none)
  int pf1 = 0, pf2 = 0;
  // 1: the epilogue's V (or w) is staged in shared memory (ep1, ep2)
  int ep1 = 0, ep2 = 0;
  // test hook: the next tc_gemm1 launch makes its MMA thread wait this long on
  // a barrier nothing arrives on (see k_tc_gemm); cleared by that launch
  unsigned long long inject_wait_ns = 0;
  const float* V = nullptr;
  const float* w32 = nullptr;
  float* Q = nullptr;
  float* c = nullptr;
  unsigned* err = nullptr;
  // opaque tensor maps (CUtensorMap, 128 bytes each)
  alignas(64) unsigned char maps[8][128];
};

// Batched contractions of exact inference in the original N-FHMM: one item
// per joint state c, each with its own B rows (the S*K elements c selects):
//   gemm1: Vhat[c][t][f] = sum_k theta[c][t][k] beta_ck(f) -> Q = V / Vhat, log-lik partials
//   gemm2: out[c][t][k]  = theta[c][t][k] * sum_f Q[c][t][f] beta_ck(f)
struct ExactTc {
  int precision = 0, w_format = 0;
  int NC = 0, T = 0, Tp = 0, SKp = 0, F = 0, Fp = 0;
  void* th_hi = nullptr;  // NC*Tp x SKp  theta operand (tf32 hi as float, or bf16)
  void* th_lo = nullptr;
  void* q_hi = nullptr;   // NC*Tp x Fp   Q operand
  void* q_lo = nullptr;
  void* b1_hi = nullptr;  // NC*Fp x SKp  B1[c][f][k] = beta_ck(f)
  void* b1_lo = nullptr;
  void* b2_hi = nullptr;  // NC*SKp x Fp  B2[c][k][f] = beta_ck(f)
  void* b2_lo = nullptr;
  const float* V = nullptr;     // T x Fp (shared by the items)
  const float* th32 = nullptr;  // NC*Tp x SKp theta in float
  float* out = nullptr;         // NC*Tp x SKp
  double* bpart = nullptr;      // NC*Tp x nbpart
  int nbpart = 0;
  unsigned* err = nullptr;
  alignas(64) unsigned char maps[8][128];
};
int tc_exact_plan(ExactTc& p);   // allocates the operand arrays, builds the tensor maps
int tc_exact_gemm1(ExactTc& p, cudaStream_t st);
int tc_exact_gemm2(ExactTc& p, cudaStream_t st);
void tc_exact_free(ExactTc& p);

bool tc_available();
// Tile shapes: the column tiles the tuner may choose for contraction `which`
// (0 reconstruction, 1 back-projection) at a precision; the deepest ring for
// a column tile (with or without the staged epilogue operand); set a plan's
// shape (re-encodes its tensor maps; 0 on success, -1 with tc_last_error).
int tc_tile_candidates(int precision, int which, int* out, int max_out);
int tc_max_stages(int precision, int bn, bool epi_stage);
int tc_set_tiles(TcPlan& p, int bn1, int bn2, int st1, int st2, int ep1, int ep2);
// bound partials per frame: allocated for the narrowest tile, used by the plan's
int tc_bpart_columns_max(int Fp);
int tc_bpart_used(const TcPlan& p);
std::string tc_last_error();
int tc_col_tiles_gemm1(int Fp);
int tc_plan(TcPlan& p, int precision, int T, int M, int Mp, int F, int Fp, const float* V,
            const float* WM, const float* WF, const float* w32, float* Q, float* c,
            unsigned* err, cudaStream_t st);
// Refresh the operand copies of beta from WM/WF (returns launches).
int tc_refresh_beta(TcPlan& p, cudaStream_t st);
// frames [row_off, row_off + rows) of the plan's T (returns launches, or -1);
// reserve: SMs the persistent grid leaves free for a kernel running beside it
// (at most half of them)
int tc_gemm1(TcPlan& p, int row_off, int rows, double* bpart, int reserve, cudaStream_t st);
int tc_gemm2(TcPlan& p, int row_off, int rows, int reserve, cudaStream_t st);
void tc_free(TcPlan& p);

}  // namespace nfhmm
