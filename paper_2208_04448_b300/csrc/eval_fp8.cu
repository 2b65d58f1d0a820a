// Fused encode + MLP on tcgen05 tensor cores, TC_FP8 operands (mlp.cuh).
#include "eval_launch.cuh"

namespace nvdb {
nvdb_status launch_eval_fp8(const EvalBatch& b, int64_t ntiles, cudaStream_t s) {
  return launch_tc_shape<TC_FP8>(b, ntiles, "mlp_fp8", s);
}
}  // namespace nvdb
