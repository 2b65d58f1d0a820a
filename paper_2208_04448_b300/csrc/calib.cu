// FP8 scale calibration: the FP32 forward over seeded lattice points of a network's domain
// (calib_amax_kernel, mlp.cuh).
#include "runtime.cuh"

namespace nvdb {
nvdb_status launch_calib_amax(const NetView& nv, int lg, uint64_t seed, int n, uint32_t* amax, cudaStream_t s) {
  const unsigned blocks = blocks_for(n, 128);
  if (nv.n_in == 32 && nv.width == 32) KLAUNCH("calib_amax", s, calib_amax_kernel<32, 32><<<blocks, 128, 0, s>>>(nv, lg, seed, n, amax));
  else if (nv.n_in == 32 && nv.width == 64) KLAUNCH("calib_amax", s, calib_amax_kernel<32, 64><<<blocks, 128, 0, s>>>(nv, lg, seed, n, amax));
  else if (nv.n_in == 64 && nv.width == 32) KLAUNCH("calib_amax", s, calib_amax_kernel<64, 32><<<blocks, 128, 0, s>>>(nv, lg, seed, n, amax));
  else if (nv.n_in == 64 && nv.width == 64) KLAUNCH("calib_amax", s, calib_amax_kernel<64, 64><<<blocks, 128, 0, s>>>(nv, lg, seed, n, amax));
  else return fail(NVDB_ERR_UNSUPPORTED, "network shape n=%d w=%d", nv.n_in, nv.width);
  CU(cudaGetLastError());
  return NVDB_OK;
}
}  // namespace nvdb
