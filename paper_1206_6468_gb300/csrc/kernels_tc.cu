// Tensor-core contractions: not yet enabled; the SIMT FP32 path runs.
#include "nfhmm_tc.h"

namespace nfhmm {

bool tc_available() { return false; }
std::string tc_last_error() { return "tensor-core path not built"; }
int tc_col_tiles_gemm1(int) { return 0; }
int tc_plan(TcPlan&, int, int, int, int, int, int, const float*, const float*, const float*,
            const float*, float*, float*, unsigned*, cudaStream_t) {
  return -1;
}
int tc_refresh_beta(TcPlan&, cudaStream_t) { return 0; }
int tc_gemm1(TcPlan&, double*, cudaStream_t) { return 0; }
int tc_gemm2(TcPlan&, cudaStream_t) { return 0; }
void tc_free(TcPlan&) {}

}  // namespace nfhmm
