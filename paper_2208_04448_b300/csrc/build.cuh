// VDB [Hash,5,4,3] tree build from sparse voxels (Section 3.1, Fig. 1).
// 63-bit canonical keys (level-2 key 27 bits | level-1 slot 15 | leaf slot 12 |
// voxel offset 9), a radix sort of the keys (CUB), head flags per level, scans
// of the head flags (the compaction scan), and mask words set with atomicOr
// (commutative, so the result is deterministic).
#pragma once
#include "common.cuh"

namespace nvdb {

__device__ __forceinline__ uint64_t canonical_key(int i, int j, int k) {
  const uint64_t l2 = ((uint64_t)(i >> 12) << 18) | ((uint64_t)(j >> 12) << 9) | (uint64_t)(k >> 12);
  const uint64_t l1 = (uint64_t)((((i >> 7) & 31) << 10) | (((j >> 7) & 31) << 5) | ((k >> 7) & 31));
  const uint64_t lf = (uint64_t)((((i >> 3) & 15) << 8) | (((j >> 3) & 15) << 4) | ((k >> 3) & 15));
  const uint64_t off = (uint64_t)(((i & 7) << 6) | ((j & 7) << 3) | (k & 7));
  return (l2 << 36) | (l1 << 21) | (lf << 9) | off;
}

constexpr int kCoordLimit = 1 << 21;

__global__ void build_keys_kernel(const int32_t* ijk, int64_t n, uint64_t* key, uint32_t* idx, uint32_t* status) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int i = ijk[3 * t], j = ijk[3 * t + 1], k = ijk[3 * t + 2];
  const bool ok = i >= 0 && j >= 0 && k >= 0 && i < kCoordLimit && j < kCoordLimit && k < kCoordLimit;
  if (!ok) set_status(status, ST_RANGE);
  key[t] = ok ? canonical_key(i, j, k) : 0;
  idx[t] = (uint32_t)t;
}

// Gather voxels into canonical order and flag the first voxel of every leaf,
// level-1 node and level-2 node.
__global__ void build_gather_kernel(const uint64_t* key, const uint32_t* idx, int64_t n, const int32_t* ijk_in,
                                    const float* val_in, int32_t* ijk, float* val, uint32_t* h0, uint32_t* h1,
                                    uint32_t* h2, uint32_t* status) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const uint32_t s = idx[t];
  ijk[3 * t] = ijk_in[3 * (int64_t)s];
  ijk[3 * t + 1] = ijk_in[3 * (int64_t)s + 1];
  ijk[3 * t + 2] = ijk_in[3 * (int64_t)s + 2];
  val[t] = val_in[s];
  const uint64_t k = key[t];
  const uint64_t p = t > 0 ? key[t - 1] : ~0ull;
  if (t > 0 && p == k) set_status(status, ST_DUP);
  h0[t] = (t == 0 || (p >> 9) != (k >> 9)) ? 1u : 0u;
  h1[t] = (t == 0 || (p >> 21) != (k >> 21)) ? 1u : 0u;
  h2[t] = (t == 0 || (p >> 36) != (k >> 36)) ? 1u : 0u;
}

// Node origins, first-voxel offsets, mask bits and the level-1 node of every leaf.  e* are the exclusive scans
// of the head flags, so the node index of voxel t is e[t] + h[t] - 1.
__global__ void build_fill_kernel(const int32_t* ijk, int64_t n, const uint32_t* h0, const uint32_t* h1,
                                  const uint32_t* h2, const int64_t* e0, const int64_t* e1, const int64_t* e2,
                                  int4* leaf_origin, int64_t* leaf_first, unsigned long long* leaf_mask,
                                  int4* l1_origin, unsigned long long* l1_mask, int4* l2_origin,
                                  unsigned long long* l2_mask, int64_t* leaf_node) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int i = ijk[3 * t], j = ijk[3 * t + 1], k = ijk[3 * t + 2];
  const int64_t leaf = e0[t] + h0[t] - 1, l1 = e1[t] + h1[t] - 1, l2 = e2[t] + h2[t] - 1;
  const int off = ((i & 7) << 6) | ((j & 7) << 3) | (k & 7);
  atomicOr(leaf_mask + leaf * 8 + (off >> 6), 1ull << (off & 63));
  if (h0[t]) {
    leaf_origin[leaf] = make_int4(i & ~7, j & ~7, k & ~7, 0);
    leaf_first[leaf] = t;
    leaf_node[leaf] = l1;
    const int s = (((i >> 3) & 15) << 8) | (((j >> 3) & 15) << 4) | ((k >> 3) & 15);
    atomicOr(l1_mask + l1 * 64 + (s >> 6), 1ull << (s & 63));
  }
  if (h1[t]) {
    l1_origin[l1] = make_int4(i & ~127, j & ~127, k & ~127, 0);
    const int s = (((i >> 7) & 31) << 10) | (((j >> 7) & 31) << 5) | ((k >> 7) & 31);
    atomicOr(l2_mask + l2 * 512 + (s >> 6), 1ull << (s & 63));
  }
  if (h2[t]) l2_origin[l2] = make_int4(i & ~4095, j & ~4095, k & ~4095, 0);
}

}  // namespace nvdb
