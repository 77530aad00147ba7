// Tensor-core (tcgen05, TF32 with FP32 accumulation) path of the grouped GEMM.
#include "common.cuh"

namespace ttsg {

void gemm_tf32(const std::vector<GemmProblem>& probs, cudaStream_t st) {
  (void)probs;
  (void)st;
  if (g_dry_run) return;
  throw Error(TT_ERR_UNSUPPORTED, "TF32 tensor-core GEMM not built yet");
}

}  // namespace ttsg
