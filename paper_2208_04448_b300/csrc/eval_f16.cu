// Fused encode + MLP on tcgen05 tensor cores, TC_FP16 operands (mlp.cuh).
#include "eval_launch.cuh"

namespace nvdb {
nvdb_status launch_eval_f16(const EvalBatch& b, int64_t ntiles, cudaStream_t s) {
  return launch_tc_shape<TC_FP16>(b, ntiles, "mlp_f16", s);
}
}  // namespace nvdb
