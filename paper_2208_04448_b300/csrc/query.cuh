// Random access on [Hash,5,4,NN(3)] (Section 3.5, online random access):
// explicit top-down lookup of the 8 corners of the cell enclosing each point in
// the decoded topology (root -> level-2 child bit -> level-1 child bit -> leaf
// active bit), compaction of the active corners, regression of only those
// (the fused MLP kernels in list mode), trilinear blend with the background
// for inactive corners.
#pragma once
#include "common.cuh"

namespace nvdb {

// Topology of [Hash,5,4,NN(3)]: explicit masks plus per-word popcount prefixes
// (child index = base + prefix[word] + popc(bits below)).
struct TopoView {
  int64_t n_l2;
  const uint64_t* l2_key;        // sorted level-2 keys ((i>>12)<<18 | (j>>12)<<9 | (k>>12))
  const uint64_t* l2_mask;       // [n_l2][512]
  const uint32_t* l2_pre;        // [n_l2][512] exclusive popcount prefix within the node
  const int64_t* l2_base;        // [n_l2] index of the node's first level-1 child
  const uint32_t* l1_words;      // [n_l1][128] decoded child bits
  const uint32_t* l1_pre;        // [n_l1][128]
  const int64_t* l1_base;        // [n_l1] index of the node's first leaf
  const uint32_t* leaf_words;    // [n_leaf][16] decoded active bits
  const int4* items;             // ternary models: decoded leaf items, w = tile rank + 1 (0: leaf)
  const float* tval;             // ternary models: tile values (scaled), by tile rank
};

// Active state of voxel (i, j, k); `leaf` receives its leaf item when active.
__device__ __forceinline__ bool topo_active(const TopoView& tv, int i, int j, int k, int64_t& leaf_out) {
  if ((unsigned)i >= (1u << 21) || (unsigned)j >= (1u << 21) || (unsigned)k >= (1u << 21)) return false;
  const uint64_t key = ((uint64_t)(i >> 12) << 18) | ((uint64_t)(j >> 12) << 9) | (uint64_t)(k >> 12);
  int64_t lo = 0, hi = tv.n_l2;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (tv.l2_key[mid] < key) lo = mid + 1; else hi = mid;
  }
  if (lo >= tv.n_l2 || tv.l2_key[lo] != key) return false;
  const int s2 = (((i >> 7) & 31) << 10) | (((j >> 7) & 31) << 5) | ((k >> 7) & 31);
  const uint64_t w2 = tv.l2_mask[lo * 512 + (s2 >> 6)];
  if (!((w2 >> (s2 & 63)) & 1ull)) return false;
  const int64_t n1 = tv.l2_base[lo] + tv.l2_pre[lo * 512 + (s2 >> 6)] + __popcll(w2 & ((1ull << (s2 & 63)) - 1ull));
  const int s1 = (((i >> 3) & 15) << 8) | (((j >> 3) & 15) << 4) | ((k >> 3) & 15);
  const uint32_t w1 = tv.l1_words[n1 * 128 + (s1 >> 5)];
  if (!((w1 >> (s1 & 31)) & 1u)) return false;
  const int64_t leaf = tv.l1_base[n1] + tv.l1_pre[n1 * 128 + (s1 >> 5)] + __popc(w1 & ((1u << (s1 & 31)) - 1u));
  const int v = ((i & 7) << 6) | ((j & 7) << 3) | (k & 7);
  leaf_out = leaf;
  return (tv.leaf_words[leaf * 16 + (v >> 5)] >> (v & 31)) & 1u;
}

// Exclusive popcount prefix of each word within its node.
__global__ void word_prefix_kernel(const uint32_t* words, int wpi, int64_t n_items, uint32_t* pre) {
  const int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (it >= n_items) return;
  uint32_t c = 0;
  for (int w = 0; w < wpi; ++w) {
    pre[it * wpi + w] = c;
    c += __popc(words[it * wpi + w]);
  }
}

__global__ void word_prefix64_kernel(const uint64_t* words, int wpi, int64_t n_items, uint32_t* pre) {
  const int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (it >= n_items) return;
  uint32_t c = 0;
  for (int w = 0; w < wpi; ++w) {
    pre[it * wpi + w] = c;
    c += __popcll(words[it * wpi + w]);
  }
}

__global__ void l2_keys_kernel(const int4* l2_origin, int64_t n_l2, uint64_t* key) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_l2) return;
  const int4 o = l2_origin[t];
  key[t] = ((uint64_t)(o.x >> 12) << 18) | ((uint64_t)(o.y >> 12) << 9) | (uint64_t)(o.z >> 12);
}

// Corner c = 4a + 2b + d of cell floor(p) is floor(p) + (a, b, d).  qmask: active corners
// to regress; with tiles, qtile marks the active corners inside tiles and qtv[8t + c] holds
// their tile value.
__global__ void query_lookup_kernel(TopoView tv, const float* xyz, int64_t n, uint8_t* qmask, uint32_t* counts,
                                    uint8_t* active_out, uint8_t* qtile, float* qtv) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const float px = xyz[3 * t], py = xyz[3 * t + 1], pz = xyz[3 * t + 2];
  const int x0 = (int)floorf(px), y0 = (int)floorf(py), z0 = (int)floorf(pz);
  uint32_t m = 0, tm = 0;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    int64_t leaf = 0;
    if (topo_active(tv, x0 + ((c >> 2) & 1), y0 + ((c >> 1) & 1), z0 + (c & 1), leaf)) {
      m |= 1u << c;
      if (tv.items) {
        const int w = tv.items[leaf].w;
        if (w > 0) {
          tm |= 1u << c;
          qtv[8 * t + c] = tv.tval[w - 1];
        }
      }
    }
  }
  qmask[t] = (uint8_t)(m & ~tm);
  counts[t] = __popc(m & ~tm);
  if (qtile) qtile[t] = (uint8_t)tm;
  if (active_out) active_out[t] = (uint8_t)m;
}

__global__ void query_emit_kernel(const float* xyz, int64_t n, const uint8_t* qmask, const int64_t* off,
                                  int32_t* list) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const uint32_t m = qmask[t];
  if (!m) return;
  const int x0 = (int)floorf(xyz[3 * t]), y0 = (int)floorf(xyz[3 * t + 1]), z0 = (int)floorf(xyz[3 * t + 2]);
  int64_t pos = off[t];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    if ((m >> c) & 1u) {
      list[3 * pos] = x0 + ((c >> 2) & 1);
      list[3 * pos + 1] = y0 + ((c >> 1) & 1);
      list[3 * pos + 2] = z0 + (c & 1);
      ++pos;
    }
  }
}

__global__ void query_blend_kernel(const float* xyz, int64_t n, const uint8_t* qmask, const int64_t* off,
                                   const float* vals, float background, float* out, const uint8_t* qtile,
                                   const float* qtv) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const float px = xyz[3 * t], py = xyz[3 * t + 1], pz = xyz[3 * t + 2];
  const float tx = px - floorf(px), ty = py - floorf(py), tz = pz - floorf(pz);
  const uint32_t m = qmask[t], tm = qtile ? qtile[t] : 0u;
  int64_t pos = off[t];
  float acc = 0.f;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const float wx = ((c >> 2) & 1) ? tx : 1.f - tx;
    const float wy = ((c >> 1) & 1) ? ty : 1.f - ty;
    const float wz = (c & 1) ? tz : 1.f - tz;
    float v = background;
    if ((m >> c) & 1u) v = vals[pos++];
    else if ((tm >> c) & 1u) v = qtv[8 * t + c];
    acc = acc + (wx * wy) * wz * v;
  }
  out[t] = acc;
}

}  // namespace nvdb
