// BF16 tensor-core training step (train_tc.cuh).
#include "runtime.cuh"
#include "train_tc.cuh"

namespace nvdb {
namespace {
template <int NIN, int W>
nvdb_status launch_t(const NetView& nv, const TrainJob& job, int grid, cudaStream_t s) {
  const size_t smem = TrainTcLayout<NIN, W>(nv.layers).total;
  if (smem > (size_t)kSmemPerSm - 1024) return fail(NVDB_ERR_UNSUPPORTED, "training tile needs %zu bytes of shared memory", smem);
  TRY(set_smem_limit((const void*)train_tc_kernel<NIN, W>, smem));
  KLAUNCH("train_tc_bf16", s, train_tc_kernel<NIN, W><<<grid, kTile, smem, s>>>(nv, job));
  CU(cudaGetLastError());
  return NVDB_OK;
}
}  // namespace

nvdb_status launch_train_tc(const NetView& nv, const TrainJob& job, int grid, cudaStream_t s) {
  if (nv.layers > kTrainTcMaxLayers) return fail(NVDB_ERR_UNSUPPORTED, "BF16 training: at most %d hidden layers", kTrainTcMaxLayers);
  if (nv.n_in == 32 && nv.width == 32) return launch_t<32, 32>(nv, job, grid, s);
  if (nv.n_in == 32 && nv.width == 64) return launch_t<32, 64>(nv, job, grid, s);
  if (nv.n_in == 64 && nv.width == 32) return launch_t<64, 32>(nv, job, grid, s);
  if (nv.n_in == 64 && nv.width == 64) return launch_t<64, 64>(nv, job, grid, s);
  return fail(NVDB_ERR_UNSUPPORTED, "network shape n=%d w=%d", nv.n_in, nv.width);
}
}  // namespace nvdb
