// Active tiles of level 1 (Section 3.1: a tile value stands for a constant 8^3 region) and
// their place in the codec (Section 3.3.1: the ternary level-1 classifier and the tile value
// regressor; Section 3.5: decoding and random access).
//
//  * build: a leaf whose 512 voxels are all active and whose values span at most the
//    tolerance becomes an active tile; the explicit grid keeps it expanded as its leaf, each
//    voxel carrying the tile value (FP32 midpoint of min and max);
//  * decode: ternary patches set a slot's class; the leaves of a decode are the slots of
//    class child leaf or active tile, in slot order, a tile's item flagged by w = tile rank
//    + 1 in its origin; tile items are all active and take the regressed tile value.
#pragma once
#include "common.cuh"
#include "compact.cuh"

namespace nvdb {

// One warp per leaf of the explicit grid.
__global__ void tile_prune_kernel(const unsigned long long* leaf_mask, const int64_t* leaf_first,
                                  const int4* leaf_origin, const int64_t* leaf_node, int64_t n_leaf, float tol,
                                  float* val, uint8_t* leaf_tile, unsigned long long* l1_tile_mask,
                                  unsigned long long* n_tiles) {
  const int64_t lf = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (lf >= n_leaf) return;
  const bool full = __all_sync(0xffffffffu, lane >= 8 || leaf_mask[lf * 8 + lane] == ~0ull);
  bool tile = false;
  float tv = 0.f;
  if (full) {
    const int64_t f = leaf_first[lf];
    float mn = val[f + lane], mx = mn;
    bool nan = mn != mn;
    for (int q = 1; q < 16; ++q) {
      const float v = val[f + lane + 32 * q];
      nan |= v != v;
      mn = fminf(mn, v);
      mx = fmaxf(mx, v);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
      mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    tile = mx - mn <= tol && !__any_sync(0xffffffffu, nan);   // a NaN value: no constant region
    tv = (mn + mx) * 0.5f;
    if (tile)
      for (int q = 0; q < 16; ++q) val[f + lane + 32 * q] = tv;
  }
  if (lane == 0) {
    leaf_tile[lf] = tile ? 1 : 0;
    if (tile) {
      const int4 o = leaf_origin[lf];
      const int s = (((o.x >> 3) & 15) << 8) | (((o.y >> 3) & 15) << 4) | ((o.z >> 3) & 15);
      atomicOr(l1_tile_mask + leaf_node[lf] * 64 + (s >> 6), 1ull << (s & 63));
      atomicAdd(n_tiles, 1ull);
    }
  }
}

// Ternary level-1 patches: entry e of item g sets slot e & 4095 to class e >> 12 in the
// child-or-tile words u (class <= 1) and the tile words t (class 1).  One warp per level-1
// node of any model of the batch.
__global__ void tern_patch_batch_kernel(uint32_t* u, uint32_t* t, int64_t n_items, const __grid_constant__ PatchBatch b) {
  const int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (g >= n_items) return;
  const int m = find_item(b.it, b.n, g);
  const uint32_t* off = b.it[m].off;
  if (!off) return;
  const int64_t local = g - b.it[m].start;
  for (uint32_t p = off[local] + lane; p < off[local + 1]; p += 32) {
    const uint32_t e = b.it[m].idx[p];
    const uint32_t s = e & 4095u, c = e >> 12, bit = 1u << (s & 31);
    uint32_t* uw = u + g * 128 + (s >> 5);
    uint32_t* tw = t + g * 128 + (s >> 5);
    if (c <= 1) atomicOr(uw, bit); else atomicAnd(uw, ~bit);
    if (c == 1) atomicOr(tw, bit); else atomicAnd(tw, ~bit);
  }
}

// Tile slots (t words) -> leaf-origin coordinates of the tiles, int32 [n][3], in canonical
// order (off: exclusive scan of the tile counts per node).  One warp per level-1 node.
__global__ void emit_tile_coords_kernel(const uint32_t* t, const int4* l1_origin, int64_t n_l1, const int64_t* off,
                                        int32_t* ijk, int64_t cap, uint32_t* status) {
  const int64_t node = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (node >= n_l1) return;
  const uint4 w = reinterpret_cast<const uint4*>(t + node * 128)[lane];
  const uint32_t ww[4] = {w.x, w.y, w.z, w.w};
  const int64_t cnt = __popc(w.x) + __popc(w.y) + __popc(w.z) + __popc(w.w);
  int64_t tot;
  int64_t pos = off[node] + warp_excl_scan(cnt, lane, tot);
  const int4 o = l1_origin[node];
  bool over = false;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    uint32_t b = ww[q];
    while (b) {
      const int bit = __ffs(b) - 1;
      b &= b - 1;
      const int s = (lane * 4 + q) * 32 + bit;
      if (pos < cap) {
        ijk[3 * pos] = o.x + 8 * (s >> 8);
        ijk[3 * pos + 1] = o.y + 8 * ((s >> 4) & 15);
        ijk[3 * pos + 2] = o.z + 8 * (s & 15);
      } else {
        over = true;
      }
      ++pos;
    }
  }
  if (over) set_status(status, ST_CORRUPT);
}

// Values of the tile items' voxels: item u with w = r + 1 covers out[off[u] .. +512).
__global__ void tile_fill_kernel(const int4* items, int64_t n_items, const int64_t* off, const float* tval,
                                 float* out, int64_t cap) {
  const int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (g >= n_items) return;
  const int w = items[g].w;
  if (w <= 0) return;
  const float v = tval[w - 1];
  const int64_t b = off[g];
  for (int k = lane; k < 512; k += 32)
    if (b + k < cap) out[b + k] = v;
}

// Ternary mismatches of level 1: predicted (u, t) against the truth (child mask including the
// tiles, tile mask); u is overwritten with the mismatch bits, counted per node.
__global__ void tern_mismatch_kernel(uint32_t* u, const uint32_t* t, const uint32_t* child, const uint32_t* tile,
                                     int64_t n_items, uint32_t* counts) {
  const int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (it >= n_items) return;
  uint32_t c = 0;
  for (int i = 0; i < 128; ++i) {
    const int64_t k = it * 128 + i;
    const uint32_t m = (u[k] ^ child[k]) | (t[k] ^ tile[k]);
    u[k] = m;
    c += __popc(m);
  }
  counts[it] = c;
}

// Mismatch bits -> ternary patch entries slot | true class << 12, CSR order.
__global__ void tern_emit_patches_kernel(const uint32_t* mis, const uint32_t* child, const uint32_t* tile,
                                         int64_t n_items, const int64_t* off, uint16_t* idx) {
  const int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (it >= n_items) return;
  int64_t pos = off[it];
  for (int i = 0; i < 128; ++i) {
    uint32_t b = mis[it * 128 + i];
    const uint32_t cw = child[it * 128 + i], tw = tile[it * 128 + i];
    while (b) {
      const int bit = __ffs(b) - 1;
      b &= b - 1;
      const uint32_t cls = (tw >> bit) & 1u ? 1u : ((cw >> bit) & 1u ? 0u : 2u);
      idx[pos++] = (uint16_t)(((uint32_t)(i * 32 + bit)) | (cls << 12));
    }
  }
}

// Level-0 candidate words of the grid's tile leaves set to all active (a tile is not
// classified, so it carries no level-0 patches).
__global__ void tile_words_full_kernel(uint32_t* words, const uint8_t* leaf_tile, int64_t n_leaf) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_leaf * 16 && leaf_tile[i >> 4]) words[i] = ~0u;
}

// Population flags of a pruned grid: leaves that are (want = 1) or are not (want = 0) tiles,
// and voxels of leaves that are not tiles (one warp per leaf).
__global__ void leaf_tile_flags_kernel(const uint8_t* leaf_tile, int64_t n_leaf, uint32_t want, uint32_t* flags) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_leaf) flags[i] = (uint32_t)(leaf_tile[i] ? 1u : 0u) == want ? 1u : 0u;
}

__global__ void voxel_nontile_flags_kernel(const uint8_t* leaf_tile, const int64_t* leaf_first, int64_t n_leaf,
                                           uint32_t* flags) {
  const int64_t lf = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (lf >= n_leaf) return;
  const uint32_t f = leaf_tile[lf] ? 0u : 1u;
  for (int64_t v = leaf_first[lf] + lane; v < leaf_first[lf + 1]; v += 32) flags[v] = f;
}

}  // namespace nvdb
