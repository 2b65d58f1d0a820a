// Fused encode + MLP on tcgen05 tensor cores, TC_BF16X3 operands (mlp.cuh).
#include "eval_launch.cuh"

namespace nvdb {
nvdb_status launch_eval_bf16x3(const EvalBatch& b, int64_t ntiles, cudaStream_t s) {
  return launch_tc_shape<TC_BF16X3>(b, ntiles, "mlp_bf16x3", s);
}
}  // namespace nvdb
