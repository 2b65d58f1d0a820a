// Random access on the explicit VDB [Hash,5,4,3] (Section 4.4's comparison samplers and the
// mCD metric of Section 4.1): a voxel's index in the grid's canonical value array by a
// top-down lookup (root key search, level-2 child bit, level-1 child bit, leaf active bit,
// each child's rank from per-word popcount prefixes), and point samplers of order 0
// (nearest voxel), 1 (trilinear) and 3 (Catmull-Rom tricubic) with the background for
// inactive voxels; zero crossings of a level set along voxel edges (isosurface points).
#pragma once
#include "common.cuh"

namespace nvdb {

struct GridView {
  int64_t n_l2;
  const uint64_t* l2_key;          // sorted level-2 keys
  const uint64_t* l2_mask;         // [n_l2][512]
  const uint32_t* l2_pre;          // [n_l2][512]
  const int64_t* l2_base;          // first level-1 node of each level-2 node
  const uint64_t* l1_mask;         // [n_l1][64]
  const uint32_t* l1_pre;          // [n_l1][64]
  const int64_t* l1_base;          // first leaf of each level-1 node
  const uint64_t* leaf_mask;       // [n_leaf][8]
  const int64_t* leaf_first;       // first voxel of each leaf
  const float* val;                // values, canonical order
  float background;
};

// Index of voxel (i, j, k) in the value array, or -1 if it is not active.
__device__ __forceinline__ int64_t grid_index(const GridView& g, int i, int j, int k) {
  if ((unsigned)i >= (1u << 21) || (unsigned)j >= (1u << 21) || (unsigned)k >= (1u << 21)) return -1;
  const uint64_t key = ((uint64_t)(i >> 12) << 18) | ((uint64_t)(j >> 12) << 9) | (uint64_t)(k >> 12);
  int64_t lo = 0, hi = g.n_l2;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (g.l2_key[mid] < key) lo = mid + 1; else hi = mid;
  }
  if (lo >= g.n_l2 || g.l2_key[lo] != key) return -1;
  const int s2 = (((i >> 7) & 31) << 10) | (((j >> 7) & 31) << 5) | ((k >> 7) & 31);
  const uint64_t w2 = g.l2_mask[lo * 512 + (s2 >> 6)];
  if (!((w2 >> (s2 & 63)) & 1ull)) return -1;
  const int64_t n1 = g.l2_base[lo] + g.l2_pre[lo * 512 + (s2 >> 6)] + __popcll(w2 & ((1ull << (s2 & 63)) - 1ull));
  const int s1 = (((i >> 3) & 15) << 8) | (((j >> 3) & 15) << 4) | ((k >> 3) & 15);
  const uint64_t w1 = g.l1_mask[n1 * 64 + (s1 >> 6)];
  if (!((w1 >> (s1 & 63)) & 1ull)) return -1;
  const int64_t leaf = g.l1_base[n1] + g.l1_pre[n1 * 64 + (s1 >> 6)] + __popcll(w1 & ((1ull << (s1 & 63)) - 1ull));
  const int v = ((i & 7) << 6) | ((j & 7) << 3) | (k & 7);
  const uint64_t* lw = g.leaf_mask + leaf * 8;
  if (!((lw[v >> 6] >> (v & 63)) & 1ull)) return -1;
  int64_t idx = g.leaf_first[leaf] + __popcll(lw[v >> 6] & ((1ull << (v & 63)) - 1ull));
  for (int q = 0; q < (v >> 6); ++q) idx += __popcll(lw[q]);
  return idx;
}

__device__ __forceinline__ float grid_value(const GridView& g, int i, int j, int k) {
  const int64_t idx = grid_index(g, i, j, k);
  return idx >= 0 ? g.val[idx] : g.background;
}

// Catmull-Rom weights of the four samples at offsets -1, 0, 1, 2 for fraction t in [0, 1).
__device__ __forceinline__ void catmull_rom(float t, float* w) {
  const float t2 = t * t, t3 = t2 * t;
  w[0] = 0.5f * (-t3 + 2.f * t2 - t);
  w[1] = 0.5f * (3.f * t3 - 5.f * t2 + 2.f);
  w[2] = 0.5f * (-3.f * t3 + 4.f * t2 + t);
  w[3] = 0.5f * (t3 - t2);
}

// order 0: the voxel nearest p (floor(p + 1/2)); 1: trilinear over the cell corners, corners
// summed in order c = 4a + 2b + d with weights (wx wy) wz; 3: Catmull-Rom over the 4^3
// samples around the cell, x-major, each weight wx[a] wy[b] wz[d].
__global__ void grid_sample_kernel(GridView g, const float* xyz, int64_t n, int order, float* out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const float px = xyz[3 * t], py = xyz[3 * t + 1], pz = xyz[3 * t + 2];
  if (order == 0) {
    out[t] = grid_value(g, (int)floorf(px + 0.5f), (int)floorf(py + 0.5f), (int)floorf(pz + 0.5f));
    return;
  }
  const int x0 = (int)floorf(px), y0 = (int)floorf(py), z0 = (int)floorf(pz);
  const float tx = px - (float)x0, ty = py - (float)y0, tz = pz - (float)z0;
  float acc = 0.f;
  if (order == 1) {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const float wx = ((c >> 2) & 1) ? tx : 1.f - tx;
      const float wy = ((c >> 1) & 1) ? ty : 1.f - ty;
      const float wz = (c & 1) ? tz : 1.f - tz;
      acc = acc + (wx * wy) * wz * grid_value(g, x0 + ((c >> 2) & 1), y0 + ((c >> 1) & 1), z0 + (c & 1));
    }
  } else {
    float wx[4], wy[4], wz[4];
    catmull_rom(tx, wx);
    catmull_rom(ty, wy);
    catmull_rom(tz, wz);
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b)
        for (int d = 0; d < 4; ++d)
          acc = acc + (wx[a] * wy[b]) * wz[d] * grid_value(g, x0 - 1 + a, y0 - 1 + b, z0 - 1 + d);
  }
  out[t] = acc;
}

// Zero crossings of a level set along the +x, +y, +z edges of every active voxel whose
// neighbour is active with the other sign (v < 0 versus v >= 0): the point
// v + t e_a, t = val(v) / (val(v) - val(v + e_a)).  Pass 1 counts per voxel, pass 2 emits
// at the scanned offsets (canonical voxel order, then axis order).
__global__ void iso_count_kernel(GridView g, const int32_t* ijk, int64_t n, uint32_t* counts) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int i = ijk[3 * t], j = ijk[3 * t + 1], k = ijk[3 * t + 2];
  const bool neg = g.val[t] < 0.f;
  uint32_t c = 0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int64_t q = grid_index(g, i + (a == 0), j + (a == 1), k + (a == 2));
    if (q >= 0 && (g.val[q] < 0.f) != neg) ++c;
  }
  counts[t] = c;
}

__global__ void iso_emit_kernel(GridView g, const int32_t* ijk, int64_t n, const int64_t* off, float* pts) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int i = ijk[3 * t], j = ijk[3 * t + 1], k = ijk[3 * t + 2];
  const float v0 = g.val[t];
  int64_t pos = off[t];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int64_t q = grid_index(g, i + (a == 0), j + (a == 1), k + (a == 2));
    if (q < 0 || (g.val[q] < 0.f) == (v0 < 0.f)) continue;
    const float s = v0 / (v0 - g.val[q]);
    pts[3 * pos] = (float)i + (a == 0 ? s : 0.f);
    pts[3 * pos + 1] = (float)j + (a == 1 ? s : 0.f);
    pts[3 * pos + 2] = (float)k + (a == 2 ? s : 0.f);
    ++pos;
  }
}

// Per-block sums of |x| in double, in index order (a deterministic reduction with its host
// side summing the blocks in order).
__global__ void abs_sum_kernel(const float* x, int64_t n, double* block_sums) {
  __shared__ double sh[256];
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) acc += fabs((double)x[i]);
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) block_sums[blockIdx.x] = sh[0];
}

}  // namespace nvdb
