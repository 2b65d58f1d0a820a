// Launchers of the fused encode + MLP kernels, instantiated once per precision in the
// eval_*.cu translation units.
#pragma once
#include <algorithm>

#include "mlp_tc2.cuh"
#include "runtime.cuh"

namespace nvdb {

template <int NIN, int W, int MODE, bool MOE = false, bool STAGE = false, bool SIN = false, bool TERN = false,
          int KM = 0>
nvdb_status launch_tc(const EvalBatch& b, int64_t ntiles, const char* base, cudaStream_t s) {
  if (!MOE && !TERN && batch_moe(b)) return launch_tc<NIN, W, MODE, true, false>(b, ntiles, base, s);
  const TcLayout<NIN, W, MODE> lay(b.it[0].net.layers, batch_wlo(b));
  auto* kern = mlp_tc_kernel<NIN, W, MODE, MOE, STAGE, SIN, TERN, KM>;
  TRY(set_smem_limit((const void*)kern, lay.total));
  // Residency from the kernel's own limits (the runtime's occupancy query reports 1 for
  // kernels that allocate tensor memory): registers, shared memory, and TMEM columns.
  cudaFuncAttributes fa;
  CU(cudaFuncGetAttributes(&fa, kern));
  const int regs = std::max(8, (fa.numRegs + 7) & ~7);
  const int by_regs = 65536 / (regs * kTile);
  const int by_smem = (int)(kSmemPerSm / (lay.total + 1024));
  int occ = std::min({by_regs, by_smem, TcCfg<NIN, W, MODE>::MAXC});
  if (occ < 1) return fail(NVDB_ERR_UNSUPPORTED, "tensor-core kernel does not fit on an SM");
  if (g_occ_override > 0) occ = std::min(occ, g_occ_override);
  const int64_t grid = std::min<int64_t>(ntiles, (int64_t)num_sms() * occ);
  KLAUNCH(eval_name(base, b.it[0].job.mode), s, kern<<<(unsigned)grid, kTile, lay.total, s>>>(b));
  CU(cudaGetLastError());
  return NVDB_OK;
}

template <int NIN, int W, int MODE>
nvdb_status launch_tc2(const EvalBatch& b, int64_t ntiles, const char* base, cudaStream_t s) {
  const Tc2Layout<NIN, W, MODE> lay(b.it[0].net.layers, batch_wlo(b));
  TRY(set_smem_limit((const void*)mlp_tc2_kernel<NIN, W, MODE>, lay.total));
  cudaFuncAttributes fa;
  CU(cudaFuncGetAttributes(&fa, mlp_tc2_kernel<NIN, W, MODE>));
  const int regs = std::max(8, (fa.numRegs + 7) & ~7);
  const int by_regs = 65536 / (regs * kTc2Threads);
  const int by_smem = (int)(kSmemPerSm / (lay.total + 1024));
  int occ = std::min({by_regs, by_smem, TcCfg<NIN, W, MODE>::MAXC});
  if (occ < 1) return fail(NVDB_ERR_UNSUPPORTED, "tensor-core kernel does not fit on an SM");
  if (g_occ_override > 0) occ = std::min(occ, g_occ_override);
  const int64_t grid = std::min<int64_t>(ntiles, (int64_t)num_sms() * occ);
  KLAUNCH(eval_name(base, b.it[0].job.mode), s,
          mlp_tc2_kernel<NIN, W, MODE><<<(unsigned)grid, kTc2Threads, lay.total, s>>>(b));
  CU(cudaGetLastError());
  return NVDB_OK;
}

// The default kernel in its lattice-only or list-only instantiation when every item of the
// batch has that kind of tiles (a decode stage, a query, a network evaluation).
template <int NIN, int W, int MODE>
nvdb_status launch_tc_km(const EvalBatch& b, int64_t ntiles, const char* base, cudaStream_t s) {
  int lists = 0;
  for (int i = 0; i < b.n; ++i) lists += b.it[i].job.mode == MODE_LIST;
  if (!batch_moe(b) && lists == b.n) return launch_tc<NIN, W, MODE, false, false, false, false, 2>(b, ntiles, base, s);
  if (!batch_moe(b) && lists == 0) return launch_tc<NIN, W, MODE, false, false, false, false, 1>(b, ntiles, base, s);
  return launch_tc<NIN, W, MODE>(b, ntiles, base, s);
}

template <int MODE>
nvdb_status launch_tc_shape(const EvalBatch& b, int64_t ntiles, const char* base, cudaStream_t s) {
  const NetView& nv = b.it[0].net;
  // variant 0: 128 threads per tile; 1: 256 threads, split epilogue (staged origins);
  // 2: 128 threads with staged origins.  Decomposed models take variant 0's expert passes.
  // sin networks (16-bit modes, no decomposition) take variant 0's SIN instantiation.
  const int v = batch_moe(b) ? 0 : tc_variant();
  if (nv.act && (MODE == TC_FP8 || batch_moe(b)))
    return fail(NVDB_ERR_UNSUPPORTED, "sin activation: FP8 and decomposed models evaluate at FP32");
  // the ternary level-1 classifier (three logits) takes the TERN instantiation of variant 0
#define NVDB_TC_SHAPE(A, B)                                                                       \
  if (nv.n_in == A && nv.width == B) {                                                            \
    if (nv.n_out == 3)                                                                            \
      return nv.act ? launch_tc<A, B, MODE, false, false, MODE != TC_FP8, true>(b, ntiles, base, s) \
                    : launch_tc<A, B, MODE, false, false, false, true>(b, ntiles, base, s);       \
    return nv.act ? launch_tc<A, B, MODE, false, false, MODE != TC_FP8>(b, ntiles, base, s)      \
         : v == 1 ? launch_tc2<A, B, MODE>(b, ntiles, base, s)                                    \
         : v == 2 ? launch_tc<A, B, MODE, false, true>(b, ntiles, base, s)                        \
                  : launch_tc_km<A, B, MODE>(b, ntiles, base, s);                                 \
  }
  NVDB_TC_SHAPE(32, 32)
  NVDB_TC_SHAPE(32, 64)
  NVDB_TC_SHAPE(64, 32)
  NVDB_TC_SHAPE(64, 64)
#undef NVDB_TC_SHAPE
  return fail(NVDB_ERR_UNSUPPORTED, "network shape n=%d w=%d", nv.n_in, nv.width);
}

}  // namespace nvdb
