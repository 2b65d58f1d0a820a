// Stream compaction of classifier bitmasks into canonical lists (Section 3.5:
// child masks -> leaf list, active masks -> voxel list) and the patch
// correction of Section 3.3.2.  The decode uses single-pass scans with a decoupled
// look-back that apply the patches, count, scan and emit in one launch per level (end of
// this file); the build, the patch construction and the queries use a deterministic
// three-phase exclusive scan (block scans, one scan of the block sums, add-back).  Output
// order is the canonical bit order.
#pragma once
#include "common.cuh"

namespace nvdb {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 4;
constexpr int kScanBlock = kScanThreads * kScanItems;   // elements per scan block

__device__ __forceinline__ int64_t warp_excl_scan(int64_t v, int lane, int64_t& total) {
  int64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  total = __shfl_sync(0xffffffffu, x, 31);
  return x - v;
}

// Exclusive scan over the threads of a block (blockDim multiple of 32, <= 1024).
__device__ __forceinline__ int64_t block_excl_scan(int64_t v, int64_t* sh /* >= 33 */, int64_t& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int64_t wt;
  const int64_t ex = warp_excl_scan(v, lane, wt);
  if (lane == 31) sh[warp] = wt;
  __syncthreads();
  if (warp == 0) {
    const int64_t s = lane < nw ? sh[lane] : 0;
    int64_t t;
    const int64_t e = warp_excl_scan(s, lane, t);
    if (lane < nw) sh[lane] = e;
    if (lane == 0) sh[32] = t;
  }
  __syncthreads();
  const int64_t r = ex + sh[warp];
  total = sh[32];
  __syncthreads();
  return r;
}

// Phase 1: per-block exclusive scans of u32 counts; block totals to `sums`.
__global__ void scan_blocks_kernel(const uint32_t* in, int64_t n, int64_t* out, int64_t* sums) {
  __shared__ int64_t sh[33];
  const int64_t base = (int64_t)blockIdx.x * kScanBlock + (int64_t)threadIdx.x * kScanItems;
  uint32_t v[kScanItems];
  int64_t local = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = base + i < n ? in[base + i] : 0u;
    local += v[i];
  }
  int64_t tot;
  int64_t run = block_excl_scan(local, sh, tot);
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < n) out[base + i] = run;
    run += v[i];
  }
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// Phase 2: exclusive scan of the block totals by one block; grand total to out_total.
__global__ void scan_sums_kernel(int64_t* sums, int64_t nb, int64_t* out_total) {
  __shared__ int64_t sh[33];
  int64_t carry = 0;
  for (int64_t b0 = 0; b0 < nb; b0 += blockDim.x) {
    const int64_t i = b0 + threadIdx.x;
    const int64_t v = i < nb ? sums[i] : 0;
    int64_t tot;
    const int64_t e = block_excl_scan(v, sh, tot);
    if (i < nb) sums[i] = e + carry;
    carry += tot;
  }
  if (threadIdx.x == 0) *out_total = carry;
}

// Phase 3: add the block offsets.
__global__ void scan_add_kernel(int64_t* out, int64_t n, const int64_t* sums) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] += sums[i / kScanBlock];
}

// Validate an imported patch list: offsets off[0..items] start at 0, never decrease and
// end at n; every index is below `bound` (candidates per item).  Any violation sets
// ST_CORRUPT; the model is not returned then, so no decode reads the lists.
__global__ void check_patches_kernel(const uint32_t* off, int64_t items, const uint16_t* idx, int64_t n,
                                     uint32_t bound, uint32_t* status) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool bad = false;
  if (i < items) bad = off[i] > off[i + 1];
  if (i == 0) bad = bad || off[0] != 0u || (int64_t)off[items] != n;
  for (int64_t j = i; j < n; j += (int64_t)gridDim.x * blockDim.x) bad = bad || idx[j] >= bound;
  if (bad) set_status(status, ST_CORRUPT);
}

// Level-1 child words -> leaf origins in canonical order.  One warp per node,
// lane l owns words 4l..4l+3 (bits in slot order).  With tile words t (ternary level 1,
// toff their exclusive scan per node), a slot that is an active tile gets w = its tile rank
// + 1 in the emitted origin (0 for a child leaf).
__global__ void emit_leaves_kernel(const uint32_t* words, const int4* l1_origin, int64_t n_l1,
                                   const int64_t* off, int4* leaf_origin, int64_t cap, uint32_t* status,
                                   const uint32_t* t = nullptr, const int64_t* toff = nullptr) {
  const int64_t node = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (node >= n_l1) return;
  const uint4 w = reinterpret_cast<const uint4*>(words + node * 128)[lane];
  const uint32_t ww[4] = {w.x, w.y, w.z, w.w};
  uint32_t tt[4] = {0u, 0u, 0u, 0u};
  int64_t trank = 0;
  if (t) {
    const uint4 v = reinterpret_cast<const uint4*>(t + node * 128)[lane];
    tt[0] = v.x; tt[1] = v.y; tt[2] = v.z; tt[3] = v.w;
    int64_t ttot;
    trank = toff[node] + warp_excl_scan(__popc(v.x) + __popc(v.y) + __popc(v.z) + __popc(v.w), lane, ttot);
  }
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
      const int tw = (tt[q] >> bit) & 1u ? (int)(trank + __popc(tt[q] & ((1u << bit) - 1u))) + 1 : 0;
      if (pos < cap)
        leaf_origin[pos] = make_int4(o.x + 8 * (s >> 8), o.y + 8 * ((s >> 4) & 15), o.z + 8 * (s & 15), tw);
      else
        over = true;
      ++pos;
    }
    trank += __popc(tt[q]);
  }
  if (over) set_status(status, ST_CORRUPT);
}

// A level with no items whose model header expects some: the decode is inconsistent.
__global__ void flag_corrupt_kernel(uint32_t* status) { set_status(status, ST_CORRUPT); }

// XOR of two word arrays (prediction vs truth) -> mismatch words, counted per item.
__global__ void mismatch_count_kernel(uint32_t* pred, const uint32_t* truth, int wpi, int64_t n_items,
                                      uint32_t* counts) {
  const int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (it >= n_items) return;
  uint32_t c = 0;
  for (int i = 0; i < wpi; ++i) {
    const uint32_t m = pred[it * wpi + i] ^ truth[it * wpi + i];
    pred[it * wpi + i] = m;
    c += __popc(m);
  }
  counts[it] = c;
}

// Mismatch words -> patch indices (uint16 local candidate index), CSR order.
__global__ void emit_patches_kernel(const uint32_t* mis, int wpi, int64_t n_items, const int64_t* off,
                                    uint16_t* idx) {
  const int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (it >= n_items) return;
  int64_t pos = off[it];
  for (int i = 0; i < wpi; ++i) {
    uint32_t b = mis[it * wpi + i];
    while (b) {
      const int bit = __ffs(b) - 1;
      b &= b - 1;
      idx[pos++] = (uint16_t)(i * 32 + bit);
    }
  }
}

// Membership in one expert's support (Section 3.4: a subdomain plus its halo), box [lo, hi)
// in the level's units, of every element of a training population: net 0 the level-1
// slots (index node * 4096 + slot, the slot's leaf coordinates tested), net 1 the leaves
// (whole leaf inside; the box is leaf-aligned), net 2 the active voxels.
__global__ void support_flags_kernel(int net, const int4* l1_origin, const int4* leaf_origin, const int32_t* ijk,
                                     int64_t count, int4 lo, int4 hi, uint32_t* flags) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  int x, y, z, ext;
  if (net == 0) {
    const int4 o = l1_origin[i >> 12];
    const int sl = (int)(i & 4095);
    x = (o.x >> 3) + (sl >> 8); y = (o.y >> 3) + ((sl >> 4) & 15); z = (o.z >> 3) + (sl & 15); ext = 1;
  } else if (net == 1) {
    const int4 o = leaf_origin[i];
    x = o.x; y = o.y; z = o.z; ext = 8;
  } else {
    x = ijk[3 * i]; y = ijk[3 * i + 1]; z = ijk[3 * i + 2]; ext = 1;
  }
  flags[i] = x >= lo.x && y >= lo.y && z >= lo.z && x + ext <= hi.x && y + ext <= hi.y && z + ext <= hi.z ? 1u : 0u;
}

// Indices of the set flags, in index order (off: exclusive scan of the flags).
__global__ void compact_flags_kernel(const uint32_t* flags, const int64_t* off, int64_t count, uint32_t* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count && flags[i]) out[off[i]] = (uint32_t)i;
}

// ---------------------------------------------------------------- batched forms
// Per-model tables passed by value; item g of the concatenation belongs to the
// last model whose `start` is <= g.
constexpr int kMaxBatchC = 48;

template <class T>
__device__ __forceinline__ int find_item(const T* it, int n, int64_t g) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (it[mid].start <= g) lo = mid; else hi = mid - 1;
  }
  return lo;
}

struct L2Item {
  const uint64_t* mask;   // [n_l2][512] of this model
  const int4* origin;     // [n_l2]
  int64_t start;          // first level-2 node of this model in the concatenation
};
struct L2Batch {
  int n;
  L2Item it[kMaxBatchC];
};

struct PatchItem {
  const uint32_t* off;    // CSR offsets of this model's patch list (level 1 or level 0)
  const uint16_t* idx;
  int64_t start;          // first item (node / leaf) of this model in the concatenation
};
struct PatchBatch {
  int n;
  PatchItem it[kMaxBatchC];
};


}  // namespace nvdb

namespace nvdb {

// ---------------------------------------------------------------- single-pass scans
// Decoupled look-back (Merrill & Garland, "Single-pass parallel prefix scan with decoupled
// look-back", 2016): blocks take consecutive ids from a counter in the order they start, so
// every predecessor of a block is running or done; each block publishes its aggregate, then
// walks back over its predecessors' words until one holds an inclusive prefix, and publishes
// its own.  Word b of `state`: bits 62-63 the flag (1 aggregate, 2 inclusive prefix), bits
// 0-61 the value; word nblocks is the block counter.  The state is zeroed before each launch.
// Every wait is bounded (kWaitLimitNs): on expiry the block flags ST_TIMEOUT and publishes
// what it has, so no waiter behind it spins forever.
constexpr uint64_t kLbAgg = 1ull << 62, kLbInc = 2ull << 62, kLbVal = (1ull << 62) - 1;

__device__ __forceinline__ uint64_t lb_load(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void lb_store(uint64_t* p, uint64_t v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" :: "l"(p), "l"(v) : "memory");
}

// Thread 0 of block `bid`: the sum of all earlier blocks' aggregates.
__device__ int64_t lb_prefix(uint64_t* state, int64_t bid, int64_t agg, uint32_t* status) {
  if (bid == 0) {
    lb_store(state, kLbInc | (uint64_t)agg);
    return 0;
  }
  lb_store(state + bid, kLbAgg | (uint64_t)agg);
  int64_t prefix = 0;
  const uint64_t t0 = global_ns();
  for (int64_t p = bid - 1; p >= 0;) {
    const uint64_t w = lb_load(state + p);
    if ((w >> 62) == 0) {
      if (global_ns() - t0 > kWaitLimitNs) { set_status(status, ST_TIMEOUT); break; }
      continue;
    }
    prefix += (int64_t)(w & kLbVal);
    if ((w >> 62) == 2) break;
    --p;
  }
  lb_store(state + bid, kLbInc | (uint64_t)(prefix + agg));
  return prefix;
}

// Warp 0 of block `bid` (all 32 lanes): the same prefix, walking back over windows of 32
// predecessors at a time (one L2 round trip per window): the nearest inclusive prefix in the
// window ends the walk, the aggregates after it are summed; a window with a predecessor that
// has published nothing yet is read again.  Positions before block 0 count as an inclusive 0.
__device__ int64_t lb_prefix_warp(uint64_t* state, int64_t bid, int64_t agg, uint32_t* status, int lane) {
  if (bid == 0) {
    if (lane == 0) lb_store(state, kLbInc | (uint64_t)agg);
    return 0;
  }
  if (lane == 0) lb_store(state + bid, kLbAgg | (uint64_t)agg);
  int64_t prefix = 0;
  const uint64_t t0 = global_ns();
  for (int64_t end = bid;;) {
    const int64_t p = end - 32 + lane;
    const uint64_t w = p >= 0 ? lb_load(state + p) : kLbInc;
    const uint32_t flag = (uint32_t)(w >> 62);
    const uint32_t inc = __ballot_sync(0xffffffffu, flag == 2);
    const int last_inc = inc ? 31 - __clz(inc) : -1;
    if (__ballot_sync(0xffffffffu, flag == 0 && lane > last_inc)) {   // not all published yet
      if (global_ns() - t0 > kWaitLimitNs) {
        if (lane == 0) set_status(status, ST_TIMEOUT);
        break;
      }
      continue;
    }
    int64_t v = lane >= last_inc ? (int64_t)(w & kLbVal) : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    prefix += v;
    if (last_inc >= 0) break;
    end -= 32;
  }
  if (lane == 0) lb_store(state + bid, kLbInc | (uint64_t)(prefix + agg));
  return prefix;
}

__device__ __forceinline__ int64_t lb_block_id(uint64_t* state, int64_t nblocks, int64_t* sh) {
  if (threadIdx.x == 0) *sh = (int64_t)atomicAdd(reinterpret_cast<unsigned long long*>(state + nblocks), 1ull);
  __syncthreads();
  return *sh;
}

// Level-2 child counts with their scan, then the level-1 node origins: one block (512
// threads) per level-2 node of any model of the batch; off[node] = level-1 nodes before it
// (kept for the random-access lookup); the last block checks the total.
__global__ void l2_scan_batch_kernel(const __grid_constant__ L2Batch b, int64_t n_nodes, int64_t* off,
                                     int64_t expect, uint64_t* state, uint32_t* status, int4* l1_origin) {
  __shared__ int64_t sh[33];
  __shared__ int64_t sid, spre;
  const int64_t g = lb_block_id(state, n_nodes, &sid);
  const int m = find_item(b.it, b.n, g);
  const int64_t local = g - b.it[m].start;
  uint64_t w = b.it[m].mask[local * 512 + threadIdx.x];
  int64_t tot;
  const int64_t ex = block_excl_scan(__popcll(w), sh, tot);
  if (threadIdx.x == 0) {
    spre = lb_prefix(state, g, tot, status);
    off[g] = spre;
    if (g == n_nodes - 1 && spre + tot != expect) set_status(status, ST_CORRUPT);
  }
  __syncthreads();
  int64_t pos = spre + ex;
  const int4 o = b.it[m].origin[local];
  bool over = false;
  while (w) {
    const int bit = __ffsll((long long)w) - 1;
    w &= w - 1;
    const int sl = threadIdx.x * 64 + bit;
    if (pos < expect)
      l1_origin[pos] = make_int4(o.x + 128 * (sl >> 10), o.y + 128 * ((sl >> 5) & 31), o.z + 128 * (sl & 31), 0);
    else
      over = true;
    ++pos;
  }
  if (over) set_status(status, ST_CORRUPT);
}

// Patch application (XOR, Section 3.3.2) and set-bit counts of the items of a level with
// their scan: IPB items per block of 8 warps (IPB / 8 per warp); off[item] = set bits
// before it; the last block checks the total.  Items flagged as active tiles (tiles[g].w > 0)
// become all ones.  Once the block's offsets are known, EMIT writes its items' children in
// canonical order: kEmitLeaves the leaf origins of level-1 nodes (wpi 128), kEmitVoxels the
// voxel coordinates of leaves (wpi 16, the warp taking one 32-bit word at a time).
// Items per block of the decode's scans: level 1 has few items with much work each (one per
// warp); level 0 many small ones, where larger blocks keep the look-back chain short.
constexpr int kScanItemsL1 = 8, kScanItemsL0 = 32;
constexpr int kPatchScanItems = kScanItemsL1;
enum : int { kEmitNone = 0, kEmitLeaves = 1, kEmitVoxels = 2 };

template <int EMIT = kEmitNone, int IPB = kPatchScanItems>
__global__ void __launch_bounds__(256) patch_scan_batch_kernel(uint32_t* words, int wpi, int64_t n_items,
                                                              const __grid_constant__ PatchBatch b, int64_t* off,
                                                              int64_t expect, uint64_t* state, uint32_t* status,
                                                              const int4* tiles = nullptr,
                                                              const int4* origin = nullptr, void* out = nullptr) {
  static_assert(IPB % 8 == 0 && IPB <= 32, "items per block");
  __shared__ uint32_t sw[IPB][128];
  __shared__ uint32_t scnt[IPB];
  __shared__ int64_t soff[IPB];
  __shared__ int64_t sid, spre;
  const int64_t nblocks = (n_items + IPB - 1) / IPB;
  const int64_t bid = lb_block_id(state, nblocks, &sid);
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int q = 0; q < IPB / 8; ++q) {
    const int li = wib * (IPB / 8) + q;
    const int64_t g = bid * IPB + li;
    uint32_t c = 0;
    if (g < n_items) {
      const int m = find_item(b.it, b.n, g);
      const int64_t local = g - b.it[m].start;
      uint32_t* w = words + g * wpi;
      const bool full = tiles && tiles[g].w > 0;   // an active tile: every voxel, no patches
      for (int i = lane; i < wpi; i += 32) sw[li][i] = full ? ~0u : w[i];
      __syncwarp();
      const uint32_t* poff = b.it[m].off;
      if (poff && !full) {   // eight index loads in flight per lane, then their XORs
        const uint32_t p1 = poff[local + 1];
        for (uint32_t p0 = poff[local] + lane; p0 < p1; p0 += 32 * 8) {
          uint32_t bit[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) bit[j] = p0 + 32 * j < p1 ? (uint32_t)b.it[m].idx[p0 + 32 * j] : 0xFFFFFFFFu;
#pragma unroll
          for (int j = 0; j < 8; ++j)
            if (bit[j] != 0xFFFFFFFFu) atomicXor(&sw[li][bit[j] >> 5], 1u << (bit[j] & 31));
        }
      }
      __syncwarp();
      for (int i = lane; i < wpi; i += 32) {
        const uint32_t v = sw[li][i];
        w[i] = v;
        c += __popc(v);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
      __syncwarp();
    }
    if (lane == 0) scnt[li] = c;
  }
  __syncthreads();
  if (wib == 0) {
    int64_t tot;
    const int64_t ex = warp_excl_scan(lane < IPB ? scnt[lane] : 0u, lane, tot);
    const int64_t pre = lb_prefix_warp(state, bid, tot, status, lane);
    if (lane == 0) {
      spre = pre;
      if (bid == nblocks - 1 && pre + tot != expect) set_status(status, ST_CORRUPT);
    }
    __syncwarp();
    const int64_t g = bid * IPB + lane;
    if (lane < IPB) soff[lane] = spre + ex;
    if (lane < IPB && g < n_items) off[g] = spre + ex;
  }
  if constexpr (EMIT != kEmitNone) {
    __syncthreads();
    bool over = false;
    for (int q = 0; q < IPB / 8; ++q) {
      const int li = wib * (IPB / 8) + q;
      const int64_t g = bid * IPB + li;
      if (g >= n_items) break;
      const int4 o = origin[g];
      if constexpr (EMIT == kEmitLeaves) {   // lane l owns words 4l .. 4l+3 (bits in slot order)
        const uint32_t ww[4] = {sw[li][4 * lane], sw[li][4 * lane + 1], sw[li][4 * lane + 2], sw[li][4 * lane + 3]};
        int64_t tot;
        int64_t pos = soff[li] + warp_excl_scan(__popc(ww[0]) + __popc(ww[1]) + __popc(ww[2]) + __popc(ww[3]), lane, tot);
        int4* leaf_origin = static_cast<int4*>(out);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          uint32_t bb = ww[k];
          while (bb) {
            const int bit = __ffs(bb) - 1;
            bb &= bb - 1;
            const int sl = (lane * 4 + k) * 32 + bit;
            if (pos < expect)
              leaf_origin[pos] = make_int4(o.x + 8 * (sl >> 8), o.y + 8 * ((sl >> 4) & 15), o.z + 8 * (sl & 15), 0);
            else
              over = true;
            ++pos;
          }
        }
      } else {   // voxels: word k in turn, lane j taking bit j; the set lanes write consecutive ranks
        int32_t* ijk = static_cast<int32_t*>(out);
        int64_t pos = soff[li];
        for (int k = 0; k < 16; ++k) {
          const uint32_t wk = sw[li][k];
          if (wk == 0u) continue;
          if ((wk >> lane) & 1u) {
            const int v = k * 32 + lane;
            const int64_t p = pos + __popc(wk & ((1u << lane) - 1u));
            if (p < expect) {
              ijk[3 * p] = o.x + (v >> 6);
              ijk[3 * p + 1] = o.y + ((v >> 3) & 7);
              ijk[3 * p + 2] = o.z + (v & 7);
            } else {
              over = true;
            }
          }
          pos += __popc(wk);
        }
      }
    }
    if (over) set_status(status, EMIT == kEmitVoxels ? ST_CAPACITY : ST_CORRUPT);
  }
}

}  // namespace nvdb
