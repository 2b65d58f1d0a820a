// Key sort of the tree build (Section 3.1): CUB's radix sort of 63-bit canonical keys with
// their input indices.  Its temporary storage comes from the library's allocator.
#include <cub/cub.cuh>

#include "runtime.cuh"

namespace nvdb {
nvdb_status sort_keys(const uint64_t* k_in, uint64_t* k_out, const uint32_t* i_in, uint32_t* i_out, int n,
                      cudaStream_t s) {
  size_t tb = 0;
  CU(cub::DeviceRadixSort::SortPairs(nullptr, tb, k_in, k_out, i_in, i_out, n, 0, 63, s));
  uint8_t* tmp = nullptr;
  TRY(dalloc(&tmp, tb));
  const cudaError_t e = cub::DeviceRadixSort::SortPairs(tmp, tb, k_in, k_out, i_in, i_out, n, 0, 63, s);
  dfree(tmp);   // cudaFree waits for the sort to finish
  if (e != cudaSuccess) return fail(NVDB_ERR_CUDA, "radix sort: %s", cudaGetErrorString(e));
  return NVDB_OK;
}
}  // namespace nvdb
