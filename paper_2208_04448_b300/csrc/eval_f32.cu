// Fused encode + MLP in plain FP32 on CUDA cores (mlp.cuh).
#include <algorithm>

#include "runtime.cuh"

namespace nvdb {
namespace {
template <int NIN, int W, bool MOE = false>
nvdb_status launch_f32(const EvalBatch& b, int64_t ntiles, cudaStream_t s) {
  if (!MOE && batch_moe(b)) return launch_f32<NIN, W, true>(b, ntiles, s);
  int occ = 0;
  const size_t smem = f32_smem_bytes<NIN, W>(b.it[0].net.layers, b.it[0].net.n_out);
  auto* kern = mlp_f32_kernel<NIN, W, MOE>;
  TRY(set_smem_limit((const void*)kern, smem));
  CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kTile, smem));
  const int64_t grid = std::min<int64_t>(ntiles, (int64_t)num_sms() * std::max(occ, 1));
  KLAUNCH(eval_name("mlp_f32", b.it[0].job.mode), s, kern<<<(unsigned)grid, kTile, smem, s>>>(b));
  CU(cudaGetLastError());
  return NVDB_OK;
}
}  // namespace

nvdb_status launch_eval_f32(const EvalBatch& b, int64_t ntiles, cudaStream_t s) {
  const NetView& nv = b.it[0].net;
  if (nv.n_in == 32 && nv.width == 32) return launch_f32<32, 32>(b, ntiles, s);
  if (nv.n_in == 32 && nv.width == 64) return launch_f32<32, 64>(b, ntiles, s);
  if (nv.n_in == 64 && nv.width == 32) return launch_f32<64, 32>(b, ntiles, s);
  if (nv.n_in == 64 && nv.width == 64) return launch_f32<64, 64>(b, ntiles, s);
  return fail(NVDB_ERR_UNSUPPORTED, "network shape n=%d w=%d", nv.n_in, nv.width);
}

}  // namespace nvdb
