// BF16 tensor-core training step (train_tc.cuh).
#include "runtime.cuh"
#include "train_tc.cuh"

namespace nvdb {
namespace {
template <int NIN, int W, int NOUT>
nvdb_status launch_t(const NetView& nv, const TrainJob& job, const FusedAdam& fa, int grid, cudaStream_t s) {
  const size_t smem = TrainTcLayout<NIN, W, NOUT>(nv.layers).total;
  if (smem > (size_t)kSmemPerSm - 1024) return fail(NVDB_ERR_UNSUPPORTED, "training tile needs %zu bytes of shared memory", smem);
  auto* kern = train_tc_kernel<NIN, W, NOUT>;
  constexpr int T = TrainTcCfg<NIN, W>::T;
  TRY(set_smem_limit((const void*)kern, smem));
  if (!fa.sync) {
    KLAUNCH("train_tc_bf16", s, kern<<<grid, T, smem, s>>>(nv, job, fa));
    CU(cudaGetLastError());
    return NVDB_OK;
  }
  // the fused Adam tail waits on every CTA: a cooperative launch keeps them all resident
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(T);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  KLAUNCH("train_tc_bf16", s, CU(cudaLaunchKernelEx(&cfg, kern, nv, job, fa)));
  return NVDB_OK;
}

template <int NIN, int W>
nvdb_status launch_o(const NetView& nv, const TrainJob& job, const FusedAdam& fa, int grid, cudaStream_t s) {
  return nv.n_out == 3 ? launch_t<NIN, W, 3>(nv, job, fa, grid, s) : launch_t<NIN, W, 1>(nv, job, fa, grid, s);
}
}  // namespace

nvdb_status launch_train_tc(const NetView& nv, const TrainJob& job, int grid, cudaStream_t s, const FusedAdam* fa) {
  if (nv.layers > kTrainTcMaxLayers) return fail(NVDB_ERR_UNSUPPORTED, "BF16 training: at most %d hidden layers", kTrainTcMaxLayers);
  const FusedAdam none{};
  const FusedAdam& f = fa ? *fa : none;
  if (nv.n_in == 32 && nv.width == 32) return launch_o<32, 32>(nv, job, f, grid, s);
  if (nv.n_in == 32 && nv.width == 64) return launch_o<32, 64>(nv, job, f, grid, s);
  if (nv.n_in == 64 && nv.width == 32) return launch_o<64, 32>(nv, job, f, grid, s);
  if (nv.n_in == 64 && nv.width == 64) return launch_o<64, 64>(nv, job, f, grid, s);
  return fail(NVDB_ERR_UNSUPPORTED, "network shape n=%d w=%d", nv.n_in, nv.width);
}
}  // namespace nvdb
