// Tensor-core (tcgen05, BF16 operands, FP32 accumulation) path of the
// per-species networks.  Placeholder until the kernels land.
#include "../../include/nnp.h"
#include "mlp.cuh"

namespace nnp {

int launch_mlp_tc(const Ws&, const MlpDims&, const MlpWeights&, const MlpBufs&, float,
                  cudaStream_t, int*, StageHook*) {
  return NNP_ERR_UNSUPPORTED;
}
int mlp_tc_prepare(const MlpDims&, const MlpWeights&, const MlpBufs&, int, const float*, float*,
                   void** state) {
  *state = nullptr;
  return NNP_ERR_UNSUPPORTED;
}
void mlp_tc_release(void*) {}

}  // namespace nnp
