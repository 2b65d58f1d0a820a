// Fused encode + MLP forward kernels (Section 3.2.2 encoding, Section 3.3.1
// networks) over tiles of 128 coordinates, with the output stage fused:
// classifiers write one bit per candidate (logit > 0) with a warp ballot,
// regressors write the value.
//
//  * mlp_f32_kernel : plain FP32 on CUDA cores, one thread per coordinate,
//                     weights in shared memory, activations in registers.
//  * mlp_tc_kernel  : tcgen05 tensor cores (FP16 operands, or compensated
//                     BF16 hi+lo pairs).  Weights resident in shared memory
//                     (canonical no-swizzle K-major layout), the 128 x n
//                     encoding tile written straight into the MMA A operand,
//                     FP32 accumulators in TMEM, bias + ReLU + repack in the
//                     epilogue; the head stays FP32 on CUDA cores.
#pragma once
#include <type_traits>
#include <cuda_fp16.h>

#include "common.cuh"

namespace nvdb {

struct NetView {
  int n_in, width, layers;
  int n_out;                     // head outputs: 1, or 3 for the ternary level-1 classifier
  int act;                       // hidden activation: 0 ReLU, 1 sin(omega a)
  float omega;
  int wexact;                    // weights and biases are BF16 values: the BF16 lo tiles are zero
  const float* p32;              // flat FP32 parameters (W_0,b_0,...,W_{L-1},b_{L-1},w_h,b_h)
  const uint8_t* wpk;            // packed 16-bit weight tiles (see pack_weights_kernel)
  const uint32_t* q;             // Fourier matrix, [n_in/2][3]
};

enum EvalMode : int { MODE_L1 = 0, MODE_L0 = 1, MODE_LIST = 2 };

struct EvalJob {
  int mode;
  const int4* nodes;      // MODE_L1: level-1 node origins; MODE_L0: leaf origins
  const int32_t* ijk;     // MODE_LIST: voxel coordinates [n][3]
  int64_t n_items;        // nodes / leaves / coordinates
  int ox, oy, oz;         // encoding domain origin
  int shift;              // MODE_LIST: 3 for the level-1 classifier (leaf units), else 0
  uint32_t* words;        // MODE_L1/L0: candidate bits, word (tile*4 + warp); ternary level-1
                          // classifier: the child-or-tile bits (class <= 1)
  uint32_t* twords;       // ternary level-1 classifier, MODE_L1: the active-tile bits (class 1)
  float* out;             // MODE_LIST: outputs (three per row for the ternary classifier)
  float scale;            // MODE_LIST: output multiplier
  const int64_t* n_dev;   // MODE_LIST: if set, the list length is read from device memory (<= n_items)
  uint32_t* status;
};

__host__ __device__ inline int64_t job_tiles(int mode, int64_t n) {
  return mode == MODE_L1 ? n * 32 : mode == MODE_L0 ? n * 4 : (n + kTile - 1) / kTile;
}

// Level coordinates of row r of tile t.  Lattice modes enumerate the 16^3
// child slots of a level-1 node (leaf units) or the 8^3 voxels of a leaf in
// slot / offset order; list mode reads coordinates (ragged last tile: rows past
// the end repeat the last coordinate and are not written).
__device__ __forceinline__ bool job_coord(const EvalJob& j, int64_t t, int r, int& cx, int& cy, int& cz) {
  if (j.mode == MODE_L1) {
    const int4 o = __ldg(j.nodes + (t >> 5));
    const int s = ((int)(t & 31) << 7) | r;
    cx = ((o.x - j.ox) >> 3) + (s >> 8);
    cy = ((o.y - j.oy) >> 3) + ((s >> 4) & 15);
    cz = ((o.z - j.oz) >> 3) + (s & 15);
    return true;
  }
  if (j.mode == MODE_L0) {
    const int4 o = __ldg(j.nodes + (t >> 2));
    const int v = ((int)(t & 3) << 7) | r;
    cx = (o.x - j.ox) + (v >> 6);
    cy = (o.y - j.oy) + ((v >> 3) & 7);
    cz = (o.z - j.oz) + (v & 7);
    return true;
  }
  int64_t i = t * kTile + r;
  const bool ok = i < j.n_items;
  if (!ok) i = j.n_items - 1;
  cx = (__ldg(j.ijk + 3 * i) - j.ox) >> j.shift;
  cy = (__ldg(j.ijk + 3 * i + 1) - j.oy) >> j.shift;
  cz = (__ldg(j.ijk + 3 * i + 2) - j.oz) >> j.shift;
  return ok;
}

__device__ __forceinline__ void job_output(const EvalJob& j, int64_t t, int r, bool valid, float y) {
  if (j.mode == MODE_LIST) {
    if (valid) j.out[t * kTile + r] = y * j.scale;
  } else {
    const uint32_t b = __ballot_sync(0xffffffffu, y > 0.f);
    if ((r & 31) == 0) j.words[t * 4 + (r >> 5)] = b;
  }
}

// Class of three logits: the first maximum (ties go to the lower class).
__device__ __forceinline__ int class3(float y0, float y1, float y2) {
  int c = 0;
  float b = y0;
  if (y1 > b) { c = 1; b = y1; }
  if (y2 > b) c = 2;
  return c;
}

// Ternary output: list mode writes the three logits; lattice modes the child-or-tile bits
// (class <= 1) and the active-tile bits (class 1).
__device__ __forceinline__ void job_output3(const EvalJob& j, int64_t t, int r, bool valid, const float* y) {
  if (j.mode == MODE_LIST) {
    if (valid)
      for (int c = 0; c < 3; ++c) j.out[3 * (t * kTile + r) + c] = y[c] * j.scale;
  } else {
    const int c = class3(y[0], y[1], y[2]);
    const uint32_t u = __ballot_sync(0xffffffffu, c <= 1), tb = __ballot_sync(0xffffffffu, c == 1);
    if ((r & 31) == 0) {
      j.words[t * 4 + (r >> 5)] = u;
      j.twords[t * 4 + (r >> 5)] = tb;
    }
  }
}

// A batch of evaluations with the same network shape (e.g. the same level of
// many animation frames), passed by value as the kernel parameter.  Item m owns
// the global tiles [tile_start, tile_start + job_tiles(mode, n_items)); a
// persistent CTA restages the network only when it crosses into another item.
constexpr int kMaxBatch = 48;

// Sparse domain decomposition (Section 3.4, Eq. 3) of one model: expert k's network of the
// job's level is experts[k]; a row's output is sum_k G_k y_k / sum_k G_k over the kept
// experts whose clamped-tent gate G_k is non-zero there (at most two subdomains per axis).
// Coordinates are relative to the model's domain origin; the halo is a power of two >= 8.
struct MoeView {
  const NetView* experts;   // [n_exp] (device memory); nullptr: no decomposition
  const int* expert_of;     // [dims^3] expert of each grid subdomain (x-major), -1 = discarded
  const int4* origin;       // [n_exp] subdomain origins relative to the domain origin (voxels)
  int n_exp, dims, size, halo;   // size, halo in voxels
};

struct EvalItem {
  NetView net;
  EvalJob job;
  int64_t tile_start;
  MoeView moe;
};

// Gate of one axis at level coordinate `rel` for a subdomain starting at `a` (level units):
// min(clamp((rel - a + h + 1/2) / 2h), clamp((a + S + h - 1/2 - rel) / 2h)); exact for a
// power-of-two h.
__device__ __forceinline__ float moe_axis_gate(int rel, int a, int S, int h) {
  const float inv = 1.f / (float)(2 * h);
  const float up = fminf(fmaxf(((float)(rel - a + h) + 0.5f) * inv, 0.f), 1.f);
  const float dn = fminf(fmaxf(((float)(a + S + h - rel) - 0.5f) * inv, 0.f), 1.f);
  return fminf(up, dn);
}

// The smallest kept expert id > last whose gate is non-zero at level coordinates r (INT_MAX
// if none); `shift` = 3 for the level-1 classifier's leaf units.
__device__ __forceinline__ int moe_next(const MoeView& v, int shift, int rx, int ry, int rz, int last) {
  const int S = v.size >> shift, h = v.halo >> shift, n = v.dims;
  int base[3], nb[3];
  const int r[3] = {rx, ry, rz};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    base[d] = r[d] / S;
    const int off = r[d] - base[d] * S;
    nb[d] = off < h && base[d] > 0 ? -1 : (S - off <= h && base[d] + 1 < n ? 1 : 0);
  }
  int best = 0x7FFFFFFF;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int ix = base[0] + ((c >> 2) & 1) * nb[0], iy = base[1] + ((c >> 1) & 1) * nb[1], iz = base[2] + (c & 1) * nb[2];
    if (((c >> 2) & 1 && !nb[0]) || ((c >> 1) & 1 && !nb[1]) || (c & 1 && !nb[2])) continue;
    if (ix < 0 || iy < 0 || iz < 0 || ix >= n || iy >= n || iz >= n) continue;
    const int e = __ldg(v.expert_of + (ix * n + iy) * n + iz);
    if (e > last && e < best) best = e;
  }
  return best;
}

// Gate of expert e at level coordinates r (0 outside its support).
__device__ __forceinline__ float moe_gate(const MoeView& v, int shift, int rx, int ry, int rz, int e) {
  const int S = v.size >> shift, h = v.halo >> shift;
  const int4 o = __ldg(v.origin + e);
  return moe_axis_gate(rx, o.x >> shift, S, h) * moe_axis_gate(ry, o.y >> shift, S, h) *
         moe_axis_gate(rz, o.z >> shift, S, h);
}

struct EvalBatch {
  int n;
  EvalItem it[kMaxBatch];
};

__device__ __forceinline__ int batch_find(const EvalBatch& b, int64_t t) {
  int lo = 0, hi = b.n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (b.it[mid].tile_start <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Total tiles of a batch; a single item may take its length from device memory.
__device__ __forceinline__ int64_t batch_total(const EvalBatch& b, int64_t& n0) {
  const EvalJob& j0 = b.it[0].job;
  n0 = (b.n == 1 && j0.n_dev) ? *j0.n_dev : j0.n_items;
  if (b.n == 1) return job_tiles(j0.mode, n0);
  const EvalItem& last = b.it[b.n - 1];
  return last.tile_start + job_tiles(last.job.mode, last.job.n_items);
}

__host__ __device__ inline int64_t net_param_count(int nin, int w, int L, int nout = 1) {
  return (int64_t)w * nin + w + (int64_t)(L - 1) * (w * w + w) + (int64_t)nout * (w + 1);
}


// ============================================================== FP32 plain path

template <int K, int W>
__device__ __forceinline__ void dense_f32(const float* p, const float* h, float* a) {
  const float4* Wp = reinterpret_cast<const float4*>(p);
  const float* b = p + W * K;
#pragma unroll
  for (int o = 0; o < W; ++o) {
    float acc = b[o];
#pragma unroll
    for (int i = 0; i < K; i += 4) {
      const float4 w = Wp[(o * K + i) >> 2];
      acc = fmaf(w.x, h[i], acc);
      acc = fmaf(w.y, h[i + 1], acc);
      acc = fmaf(w.z, h[i + 2], acc);
      acc = fmaf(w.w, h[i + 3], acc);
    }
    a[o] = acc;
  }
}

// Encoding with FP32 sin/cos of the exact phase: angle = pi * (int32)Phi * 2^-31.
template <int NIN>
__device__ __forceinline__ void encode_f32(const uint32_t* sq, int cx, int cy, int cz, float* h) {
  constexpr int M = NIN / 2;
#pragma unroll
  for (int f = 0; f < M; ++f) {
    const uint32_t ph = ffm_phase(sq, f, cx, cy, cz);
    float s, c;
    sincospif((float)(int32_t)ph * 0x1p-31f, &s, &c);
    h[f] = c;
    h[M + f] = s;
  }
}

template <int NIN, int W>
__device__ __forceinline__ void forward_f32(const float* sp, const uint32_t* sq, int L, int act, float om, int nout,
                                            int cx, int cy, int cz, float* y) {
  constexpr int H = NIN > W ? NIN : W;
  float h[H], a[W];
  encode_f32<NIN>(sq, cx, cy, cz, h);
  const float* p = sp;
  dense_f32<NIN, W>(p, h, a);
  p += W * NIN + W;
  if (act) {
#pragma unroll
    for (int o = 0; o < W; ++o) h[o] = sinf(om * a[o]);
  } else {
#pragma unroll
    for (int o = 0; o < W; ++o) h[o] = fmaxf(a[o], 0.f);
  }
  for (int l = 1; l < L; ++l) {
    dense_f32<W, W>(p, h, a);
    p += W * W + W;
    if (act) {
#pragma unroll
      for (int o = 0; o < W; ++o) h[o] = sinf(om * a[o]);
    } else {
#pragma unroll
      for (int o = 0; o < W; ++o) h[o] = fmaxf(a[o], 0.f);
    }
  }
  // head: W_h [nout][W] then b_h [nout]
  for (int c = 0; c < nout; ++c) {
    float acc = p[nout * W + c];
#pragma unroll
    for (int i = 0; i < W; ++i) acc = fmaf(p[c * W + i], h[i], acc);
    y[c] = acc;
  }
}

template <int NIN, int W>
__host__ __device__ inline size_t f32_smem_bytes(int L, int nout = 3) {
  const int64_t P = net_param_count(NIN, W, L, nout);
  return (size_t)((P + 3) & ~3ll) * 4 + (size_t)(NIN / 2) * 3 * 4;
}

template <int NIN, int W, bool MOE = false>
__global__ void __launch_bounds__(kTile, 3) mlp_f32_kernel(const __grid_constant__ EvalBatch b) {
  extern __shared__ float4 smem_f4[];
  float* sp = reinterpret_cast<float*>(smem_f4);
  const int L = b.it[0].net.layers;
  const int nout = b.it[0].net.n_out;
  const int64_t P = net_param_count(NIN, W, L, nout);
  uint32_t* sq = reinterpret_cast<uint32_t*>(sp + ((P + 3) & ~3ll));
  int64_t n0;
  const int64_t ntiles = batch_total(b, n0);
  __shared__ int smin;
  const float* staged = nullptr;
  auto stage = [&](const NetView& net) {   // uniform across the CTA
    __syncthreads();
    for (int64_t i = threadIdx.x; i < P; i += blockDim.x) sp[i] = __ldg(net.p32 + i);
    for (int i = threadIdx.x; i < 3 * (NIN / 2); i += blockDim.x) sq[i] = __ldg(net.q + i);
    __syncthreads();
    staged = net.p32;
  };
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int m = batch_find(b, t);
    const MoeView& mv = b.it[m].moe;
    EvalJob job = b.it[m].job;
    if (b.n == 1) job.n_items = n0;
    const int64_t tl = t - b.it[m].tile_start;
    int cx, cy, cz;
    const bool valid = job_coord(job, tl, threadIdx.x, cx, cy, cz);
    const NetView& nv = b.it[m].net;
    float y;
    if (!MOE || !mv.experts) {
      if (staged != nv.p32) stage(nv);
      float yy[3];
      forward_f32<NIN, W>(sp, sq, L, nv.act, nv.omega, nout, cx, cy, cz, yy);
      if (nout == 3) {   // ternary level-1 classifier (Section 3.3.1)
        job_output3(job, tl, threadIdx.x, valid, yy);
        continue;
      }
      y = yy[0];
    } else {
      // decomposed model (Section 3.4): one pass per expert with a non-zero gate in the tile,
      // ascending expert order, y = sum_k G_k y_k / sum_k G_k
      const int shift = job.mode == MODE_L1 || job.shift == 3 ? 3 : 0;
      float acc = 0.f, gs = 0.f;
      for (int last = -1;;) {
        const int mine = moe_next(mv, shift, cx, cy, cz, last);
        if (threadIdx.x == 0) smin = 0x7FFFFFFF;
        __syncthreads();
        atomicMin(&smin, mine);
        __syncthreads();
        const int e = smin;
        __syncthreads();
        if (e == 0x7FFFFFFF) break;
        const NetView ev = mv.experts[e];
        if (staged != ev.p32) stage(ev);
        const int4 eo = __ldg(mv.origin + e);
        const float g = moe_gate(mv, shift, cx, cy, cz, e);
        float ye;
        forward_f32<NIN, W>(sp, sq, L, ev.act, ev.omega, 1, cx - (eo.x >> shift), cy - (eo.y >> shift), cz - (eo.z >> shift), &ye);
        acc = fmaf(g, ye, acc);
        gs += g;
        last = e;
      }
      y = acc / gs;
    }
    job_output(job, tl, threadIdx.x, valid, y);
  }
}

// ============================================================== tcgen05 tensor-core path
// Operand modes of kind::f16 (same tensor rate) and kind::f8f6f4:
//  TC_BF16X3: activations and weights carried as BF16 pairs v = hi + lo
//             (hi = bf16(v), lo = bf16(v - hi)); D = A_hi W_hi + A_lo W_hi + A_hi W_lo,
//             three MMAs per K step (two when the weights are BF16 values), error
//             ~2^-16 relative.
//  TC_FP16  : FP16 activations and weights, one MMA per K step.
//  TC_BF16  : BF16 operands.  The encoding and the inputs of every hidden layer but the
//             last are carried as hi + lo pairs (two MMA terms), the last hidden layer's
//             input as plain BF16 (one term); weights that are not BF16 values add the
//             A_hi W_lo term.  Rounding the earlier activations to 8 bits costs the most
//             accuracy, since every later layer amplifies it; the last layer's input
//             rounding alone stays well inside the 2e-2 band bar.
//  TC_FP8   : the first layer (on the encoding) as TC_FP16; the hidden layers with E4M3
//             activations and weights (kind::f8f6f4, K = 32 per MMA), one scale per
//             layer, applied in the FP32 epilogue: h = relu(alpha D + beta).
// Layout per CTA (one 128-row tile in flight):
//  * weights in shared memory, each layer a [W x (K+16)] tile in the canonical
//    no-swizzle K-major layout; column K holds the bias (FP16 tiles: its FP16 value, and
//    column K+1 the FP16 remainder b - fp16(b)), the other columns past K are zero;
//  * the bias: FP16 takes it through the MMA (A carries the constant 1 in columns K and
//    K+1: one more K step, no epilogue work); BF16 modes add the FP32 bias in the
//    epilogue (their hi + lo operands fill the tensor-memory columns a constant chunk
//    would need); FP8 folds it into the epilogue's beta;
//  * the A operand (16-bit activations) in tensor memory, two elements per 32-bit
//    column, written by each thread for its own row with tcgen05.st: hi at columns
//    [64, 96) (FP16: [64, 104) with the constant chunk), lo at [96, 128);
//  * the FP32 accumulator D in tensor memory columns [0, W).
enum TcMode : int { TC_BF16X3 = 0, TC_FP16 = 1, TC_BF16 = 2, TC_FP8 = 3 };

// FP16 encoding and first layer (TC_FP16, and TC_FP8's first layer).
template <int MODE>
struct Enc16 {
  static constexpr bool value = MODE == TC_FP16 || MODE == TC_FP8;
};

// BF16 modes: the A operand of hidden layer l (of L) is a hi + lo pair.
template <int MODE>
__host__ __device__ __forceinline__ bool comp_in(int l, int L) {
  return MODE == TC_BF16X3 || (MODE == TC_BF16 && l < L - 1);
}

// Transposed hidden-layer tiles W_l^T, l = 1..L-1: [W (in) x W (out)] BF16,
// canonical K-major over `out`; stored after the three forward tile copies.
__host__ __device__ inline int64_t wtile_t_elems(int w, int L) { return (int64_t)(L - 1) * w * w; }
// FP8 part of the packed weights, after the 16-bit tiles: the E4M3 tiles of layers
// 1..L-1 ([W x W], canonical 8-bit K-major), then floats alpha_l at [l] (l < kMaxLayers)
// and beta_l[W] at [kMaxLayers + l W] of the epilogue h = relu(alpha_l D + beta_l).
__host__ __device__ inline int64_t fp8_tile_bytes(int w, int L) { return (int64_t)(L - 1) * w * w; }
__host__ __device__ inline int64_t fp8_aux_bytes(int w, int L) {
  return ((int64_t)(kMaxLayers + L * w) * 4 + 15) & ~(int64_t)15;
}
__host__ __device__ inline int64_t wpk_fp8_off(int nin, int w, int L) {
  return (int64_t)w * (nin + 16) * 6 + (int64_t)(L - 1) * w * (w + 16) * 6 + wtile_t_elems(w, L) * 2;
}
// Bytes of the packed weights: [FP16 | BF16 hi | BF16 lo] tiles, BF16 W_l^T tiles, FP8 part.
__host__ __device__ inline int64_t wpk_bytes(int nin, int w, int L) {
  return wpk_fp8_off(nin, w, L) + fp8_tile_bytes(w, L) + fp8_aux_bytes(w, L);
}

__host__ __device__ inline int64_t wtile_elems(int nin, int w, int L) {
  return (int64_t)w * (nin + 16) + (int64_t)(L - 1) * w * (w + 16);
}

// Offset of layer l's weights in the flat FP32 parameters.
__host__ __device__ inline int64_t layer_offset(int nin, int w, int l) {
  return l == 0 ? 0 : (int64_t)w * nin + w + (int64_t)(l - 1) * (w * w + w);
}

template <int NIN, int W, int MODE>
struct TcCfg {
  static constexpr int M = NIN / 2;                         // frequencies
  static constexpr int K0 = NIN + 16, KH = W + 16;          // augmented widths of the packed tiles
  static constexpr uint32_t COLS = 128u;
  static constexpr uint32_t A_HI = 64u, A_LO = 96u;         // TMEM columns of the A operand(s)
  static constexpr int MAXC = (int)(512u / COLS);           // CTAs per SM that fit in TMEM
  static constexpr bool ENC16 = Enc16<MODE>::value;
  static constexpr bool WLO = MODE == TC_BF16X3 || MODE == TC_BF16;   // may read BF16 lo weight tiles
  static constexpr bool BIAS_MMA = MODE == TC_FP16;                    // bias through a constant-1 K step
};

constexpr size_t kSmemPerSmDev = 233472;

// Shared-memory layout of mlp_tc_kernel; `wlo`: the batch has a model whose weights are
// not BF16 values, so the BF16 modes also stage the lo weight tiles.
template <int NIN, int W, int MODE>
struct TcLayout {
  size_t w_bytes, t_off, p_off, b_off, wh_off, q_off, org_off, bar_off, obar_off, slot_off, min_off, total;
  int ncopy;
  __host__ __device__ TcLayout(int L, bool wlo) {
    using C = TcCfg<NIN, W, MODE>;
    ncopy = C::WLO && wlo ? 2 : 1;
    // one copy of the 16-bit tiles; FP8: the FP16 first-layer tile, the E4M3 tiles, alpha/beta
    w_bytes = MODE == TC_FP8 ? (size_t)W * C::K0 * 2 + fp8_tile_bytes(W, L) + fp8_aux_bytes(W, L)
                             : (size_t)wtile_elems(NIN, W, L) * 2;
    t_off = (ncopy * w_bytes + 15) & ~(size_t)15;
    p_off = t_off + (size_t)C::M * 64 * (C::ENC16 ? 4 : 8);   // T table [M][64]: half2 / float2
    b_off = p_off + (size_t)2 * 2 * C::M * 8;                // P tables, two buffers of [2][M] x 8 B
    wh_off = b_off + (size_t)L * W * 4;                      // FP32 biases [L][W]
    q_off = wh_off + (size_t)(3 * W + 4) * 4;                // head: W_h [<= 3][W], b_h [<= 3]
    org_off = (q_off + (size_t)C::M * 12 + 15) & ~(size_t)15;   // ring of four staged origins (int4)
    bar_off = org_off + 64;
    obar_off = bar_off + 8;
    slot_off = obar_off + 32;
    min_off = slot_off + 4;
    total = min_off + 4;
    // at most MAXC CTAs may be resident per SM (TMEM): make a (MAXC+1)-th not fit
    const size_t floor_bytes = kSmemPerSmDev / (C::MAXC + 1) - 1024 + 128;
    if (total < floor_bytes) total = floor_bytes;
  }
};

// Does any model of the batch need the BF16 lo weight tiles?  (A decomposed model's item
// carries the experts' common wexact flag in its NetView.)
__host__ __device__ inline bool batch_wlo(const EvalBatch& b) {
  for (int m = 0; m < b.n; ++m)
    if (!b.it[m].net.wexact) return true;
  return false;
}

// Does any model of the batch use a domain decomposition?
__host__ __device__ inline bool batch_moe(const EvalBatch& b) {
  for (int m = 0; m < b.n; ++m)
    if (b.it[m].moe.experts) return true;
  return false;
}

template <int MODE>
__device__ __forceinline__ void split_pair(float a, float b, uint32_t& hi, uint32_t& lo) {
  if (Enc16<MODE>::value) {
    hi = cvt_f16x2(a, b);
    lo = 0u;
  } else {
    hi = cvt_bf16x2(a, b);
    const float ha = __uint_as_float(hi << 16), hb = __uint_as_float(hi & 0xFFFF0000u);
    lo = cvt_bf16x2(a - ha, b - hb);
  }
}

// ReLU and pack two FP32 values into the next layer's 16-bit A operand; BF16 modes carry
// the rounding remainder in `lo` when `comp` (the next layer takes a hi + lo pair).
template <int MODE>
__device__ __forceinline__ void relu_pair(float a, float b, bool comp, uint32_t& hi, uint32_t& lo) {
  if (MODE == TC_FP16) {
    hi = cvt_relu_f16x2(a, b);
    lo = 0u;
  } else if (!comp) {
    hi = cvt_relu_bf16x2(a, b);
    lo = 0u;
  } else {
    split_pair<MODE>(fmaxf(a, 0.f), fmaxf(b, 0.f), hi, lo);
  }
}

// sin(omega a) networks (activation appendix): the pair converted without the ReLU.
template <int MODE>
__device__ __forceinline__ void sin_pair(float a, float b, bool comp, uint32_t& hi, uint32_t& lo) {
  if (MODE == TC_FP16) {
    hi = cvt_f16x2(a, b);
    lo = 0u;
  } else if (!comp) {
    hi = cvt_bf16x2(a, b);
    lo = 0u;
  } else {
    split_pair<MODE>(a, b, hi, lo);
  }
}

template <int NW>
__device__ __forceinline__ void tmem_st_cols(uint32_t taddr, const uint32_t* r) {
  static_assert(NW == 32 || NW == 16 || NW == 8 || NW == 4, "columns");
  if (NW == 32) tmem_st32(taddr, r);
  else if (NW == 16) tmem_st16(taddr, r);
  else if (NW == 8) tmem_st8(taddr, r);
  else tmem_st4(taddr, r);
}

// Write one row of the A operand: NK 16-bit values (NK/2 packed columns) at the hi
// columns, and their remainders at the lo columns when `comp`.
template <int NK>
__device__ __forceinline__ void store_a_row(uint32_t tlane, const uint32_t* hi, const uint32_t* lo, bool comp) {
  tmem_st_cols<NK / 2>(tlane + TcCfg<32, 32, TC_FP16>::A_HI, hi);
  if (comp) tmem_st_cols<NK / 2>(tlane + TcCfg<32, 32, TC_FP16>::A_LO, lo);
}

// FP16 constant chunk after NK activations: the pair (1, 1) that multiplies the bias and
// its remainder in the tile's columns K and K+1, then zeros.
template <int NK>
__device__ __forceinline__ void store_bias_chunk(uint32_t tlane) {
  const uint32_t cst[8] = {0x3C003C00u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
  tmem_st8(tlane + TcCfg<32, 32, TC_FP16>::A_HI + NK / 2, cst);
}

// Level-0 angle addition, per-tile factors: P[dxl][f] = e^{i Phi(o + (dx0 + dxl) e_x)} for
// the two x offsets of tile t of a leaf (origin o), as float2 (cos, sin) or, for FP16, as
// the half2 pairs (cos, cos) and (-sin, sin).  Thread tid < 2M writes entry tid.
template <int M, int MODE>
__device__ __forceinline__ void l0_factors(const EvalJob& job, const uint32_t* sq, int4 o, int64_t t, float2* sPb,
                                           int tid) {
  const int dxl = tid / M, f = tid % M;
  const uint32_t ph = sq[3 * f] * (uint32_t)(o.x - job.ox + 2 * (int)(t & 3) + dxl) +
                      sq[3 * f + 1] * (uint32_t)(o.y - job.oy) + sq[3 * f + 2] * (uint32_t)(o.z - job.oz);
  float sn, cs;
  sincospif((float)(int32_t)ph * 0x1p-31f, &sn, &cs);
  if (Enc16<MODE>::value) {
    const __half2 pc = __float2half2_rn(cs), ps = __floats2half2_rn(-sn, sn);
    reinterpret_cast<uint2*>(sPb)[tid] =
        make_uint2(*reinterpret_cast<const uint32_t*>(&pc), *reinterpret_cast<const uint32_t*>(&ps));
  } else {
    sPb[tid] = make_float2(cs, sn);
  }
}

// Stage network `net` into shared memory: weight tiles, biases, head, Fourier matrix and
// (level-0 lattice) the table T[f][dy*8+dz] = e^{i Phi(dy e_y + dz e_z)}.
template <int NIN, int W, int MODE, int NT = kTile, class Lay = TcLayout<NIN, W, MODE>>
__device__ __forceinline__ void tc_stage(const NetView& net, int mode, const Lay& lay, uint8_t* smem,
                                         bool table = true) {
  using C = TcCfg<NIN, W, MODE>;
  constexpr int M = C::M;
  const int L = net.layers, tid = threadIdx.x;
  float2* sT = reinterpret_cast<float2*>(smem + lay.t_off);
  __half2* sTh = reinterpret_cast<__half2*>(smem + lay.t_off);
  float* sb = reinterpret_cast<float*>(smem + lay.b_off);
  float* swh = reinterpret_cast<float*>(smem + lay.wh_off);
  uint32_t* sq = reinterpret_cast<uint32_t*>(smem + lay.q_off);
  const int64_t te = wtile_elems(NIN, W, L);
  uint4* dst = reinterpret_cast<uint4*>(smem);
  if (MODE == TC_FP8) {   // FP16 first-layer tile, then the FP8 part
    const size_t n0 = (size_t)W * C::K0 * 2 / 16, n1 = (size_t)(lay.w_bytes / 16) - n0;
    const uint4* s0 = reinterpret_cast<const uint4*>(net.wpk);
    const uint4* s1 = reinterpret_cast<const uint4*>(net.wpk + wpk_fp8_off(NIN, W, L));
    for (size_t i = tid; i < n0; i += NT) dst[i] = __ldg(s0 + i);
    for (size_t i = tid; i < n1; i += NT) dst[n0 + i] = __ldg(s1 + i);
  } else {
    const uint8_t* base = net.wpk + (MODE == TC_FP16 ? 0 : te * 2);
    const uint4* src = reinterpret_cast<const uint4*>(base);
    const size_t n16 = lay.ncopy * lay.w_bytes / 16;   // hi (or FP16) tiles, then the lo tiles
    for (size_t i = tid; i < n16; i += NT) dst[i] = __ldg(src + i);
  }
  for (int l = 0; l < L; ++l) {
    const int64_t bo = layer_offset(NIN, W, l) + (int64_t)W * (l == 0 ? NIN : W);
    for (int o = tid; o < W; o += NT) sb[l * W + o] = __ldg(net.p32 + bo + o);
  }
  // head W_h [n_out][W] then b_h [n_out]: the biases at swh[n_out W + c]
  const int nout = net.n_out;
  const int64_t hoff = net_param_count(NIN, W, L, nout) - (int64_t)nout * (W + 1);
  for (int o = tid; o < nout * (W + 1); o += NT) swh[o] = __ldg(net.p32 + hoff + o);
  for (int i = tid; i < 3 * M; i += NT) sq[i] = __ldg(net.q + i);
  __syncthreads();
  if (mode == MODE_L0 && table) {
    // entry (f, j) at [f / G][j][f % G], G = 4 (half2) or 2 (float2): one 16-byte load
    // gives a thread G consecutive frequencies of its (dy, dz)
    constexpr int G = C::ENC16 ? 4 : 2;
    for (int i = tid; i < M * 64; i += NT) {
      const int f = i >> 6, j = i & 63;
      const uint32_t ph = sq[3 * f + 1] * (uint32_t)(j >> 3) + sq[3 * f + 2] * (uint32_t)(j & 7);
      float sn, cs;
      sincospif((float)(int32_t)ph * 0x1p-31f, &sn, &cs);
      const int at = ((f / G) * 64 + j) * G + f % G;
      if (C::ENC16) sTh[at] = __floats2half2_rn(cs, sn);
      else sT[at] = make_float2(cs, sn);
    }
  }
  fence_proxy_async_smem();   // the weight tiles are read by the tensor core (async proxy)
}

// MOE: the batch holds decomposed models (Section 3.4); a separate instantiation, so the
// undecomposed kernel carries none of the expert passes.  STAGE: lattice tiles take their
// node / leaf origin from shared memory, filled by bulk copies two tiles ahead, instead of
// a load of their own (the decode-plan autotuner measures both).  KM: the batch's tiles
// are all lattice tiles (1) or all list tiles (2), so the kernel carries only that mode's
// code; 0: either, decided per tile.  List-only kernels load the next tile's coordinates
// during the current tile's first layer.
template <int NIN, int W, int MODE, bool MOE = false, bool STAGE = false, bool SIN = false, bool TERN = false,
          int KM = 0>
__global__ void __launch_bounds__(kTile, 4) mlp_tc_kernel(const __grid_constant__ EvalBatch b) {
  static_assert(W == 32 || W == 64, "width");
  static_assert(!SIN || (MODE != TC_FP8 && !MOE), "sin networks: 16-bit modes, no decomposition");
  static_assert(!TERN || !MOE, "the ternary classifier: no decomposition");
  const float om = SIN ? b.it[0].net.omega : 0.f;   // one activation per batch (same shapes)
  static_assert(NIN == 32 || NIN == 64, "encoding size");
  using C = TcCfg<NIN, W, MODE>;
  constexpr int M = C::M;
  extern __shared__ __align__(1024) uint8_t smem[];
  const int L = b.it[0].net.layers;
  const TcLayout<NIN, W, MODE> lay(L, batch_wlo(b));
  uint8_t* sw = smem;                              // hi (or FP16) weight tiles
  uint8_t* sw_lo = smem + lay.w_bytes;             // lo weight tiles (BF16 modes, inexact weights)
  float2* sT = reinterpret_cast<float2*>(smem + lay.t_off);      // BF16 modes: FP32 table
  __half2* sTh = reinterpret_cast<__half2*>(smem + lay.t_off);   // FP16: half table
  float2* sP = reinterpret_cast<float2*>(smem + lay.p_off);
  const float* sb = reinterpret_cast<const float*>(smem + lay.b_off);
  float* swh = reinterpret_cast<float*>(smem + lay.wh_off);
  uint32_t* sq = reinterpret_cast<uint32_t*>(smem + lay.q_off);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + lay.bar_off);
  int4* sorg = reinterpret_cast<int4*>(smem + lay.org_off);
  uint64_t* obar = reinterpret_cast<uint64_t*>(smem + lay.obar_off);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + lay.slot_off);
  const int tid = threadIdx.x, warp = tid >> 5;

  if (tid == 0) {
    mbar_init(bar, 1);
    for (int q = 0; q < 4; ++q) mbar_init(obar + q, 1);
  }
  if (warp == 0) tmem_alloc(tslot, C::COLS);
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *tslot;
  const uint32_t tlane = tbase + ((uint32_t)(warp * 32) << 16);
  const uint32_t idesc = C::ENC16 ? idesc_f16_f32(kTile, W) : idesc_bf16_f32(kTile, W);
  // FP8: E4M3 tiles and the per-layer epilogue constants, after the FP16 first-layer tile
  const uint32_t f8_tiles = (uint32_t)(W * C::K0 * 2);
  const float* f8_aux = reinterpret_cast<const float*>(smem + f8_tiles + fp8_tile_bytes(W, L));

  uint32_t phase = 0;
  bool failed = false;
  int64_t n0;
  const int64_t ntiles = batch_total(b, n0);
  int cur = -1;
  float bh = 0.f;
  bool wexact = false;
  int pbuf = 0;            // level-0 factor buffer of the current tile
  bool p_ready = false;    // its factors were computed during the previous tile
  // list-only kernels: the row's raw coordinates, loaded during the previous tile's first layer
  int pf_x = 0, pf_y = 0, pf_z = 0;
  bool pf_ok = false, pf_ready = false;
  const bool comp0 = comp_in<MODE>(0, L);
  // Lattice modes: the node / leaf origin each tile reads is staged into shared memory by a
  // bulk copy (the TMA unit) one tile ahead, alternating between two buffers, each with an
  // mbarrier; counters of copies issued / waited for per buffer keep the phases.
  // (decomposed models evaluate a tile once per expert, from __ldg origins, without either)
  const bool moe_batch = MOE && batch_moe(b);
  const bool lattice = STAGE && b.it[0].job.mode != MODE_LIST && !moe_batch;   // one mode per launch (a decode stage)
  auto origin_src = [&](int64_t g) -> const int4* {
    const int mm = batch_find(b, g);
    const int64_t tl = g - b.it[mm].tile_start;
    return b.it[mm].job.nodes + (b.it[mm].job.mode == MODE_L1 ? (tl >> 5) : (tl >> 2));
  };
  int* smin = reinterpret_cast<int*>(smem + lay.min_off);   // block-wide minimum (experts)
  const float* staged_p32 = nullptr;                          // the expert network staged
  // ring of four buffers, each copy issued two tiles ahead: the CTA's tile k (k-th of its
  // tiles) is in buffer k & 3 as that buffer's (k >> 2)-th copy, so its wait parity is
  // (k >> 2) & 1; `issued` / `waited` count tiles for the drain on exit
  int issued = 0, waited = 0;
  auto issue = [&](int kk) {   // the copy of this CTA's kk-th tile, if it exists
    const int64_t g = (int64_t)blockIdx.x + (int64_t)kk * gridDim.x;
    if (g >= ntiles) return;
    if (tid == 0) {
      mbar_arrive_expect_tx(obar + (kk & 3), 16);
      bulk_g2s(sorg + (kk & 3), origin_src(g), 16, obar + (kk & 3));
    }
    issued = kk + 1;
  };
  if (lattice) {
    issue(0);
    issue(1);
  }
  int k = 0;               // tiles done by this CTA
  // tiles strided over the CTAs (for decomposed models too: contiguous ranges measured
  // slower, the tiles of the halos, which take several expert passes, bunch up in a few CTAs)
  for (int64_t t0 = blockIdx.x; t0 < ntiles && !failed; t0 += gridDim.x, ++k) {
    const int m = batch_find(b, t0);
    const MoeView& mv = b.it[m].moe;
    const bool moe = MOE && mv.experts != nullptr;
    if (m != cur && !moe) {   // uniform across the CTA: restage the item's network
      __syncthreads();
      tc_stage<NIN, W, MODE>(b.it[m].net, b.it[m].job.mode, lay, smem);
      __syncthreads();
      bh = swh[TERN ? 3 * W : W];
      wexact = b.it[m].net.wexact != 0;
      staged_p32 = b.it[m].net.p32;
    }
    if (m != cur && moe) staged_p32 = nullptr;   // another model: its lattice table too
    cur = m;
    EvalJob job = b.it[m].job;
    if (b.n == 1) job.n_items = n0;
    if constexpr (KM == 2) job.mode = MODE_LIST;
    if constexpr (KM == 1) if (job.mode == MODE_LIST) __builtin_unreachable();
    const int64_t t = t0 - b.it[m].tile_start;
    // the next tile of this CTA, if it is a level-0 tile of the same item: its factors are
    // computed while this tile's first-layer MMAs run
    const int64_t end_m = m + 1 < b.n ? b.it[m + 1].tile_start : ntiles;
    const bool next_same = job.mode == MODE_L0 && t0 + gridDim.x < end_m && !moe_batch;
    const bool next_list = KM == 2 && t0 + gridDim.x < end_m && !moe_batch;
    const int64_t tn = t0 + gridDim.x - b.it[m].tile_start;
    const int cb = k & 3, nb = (k + 1) & 3;   // origin buffers of this tile and the next
    const uint32_t cpar = (uint32_t)(k >> 2) & 1u, npar = (uint32_t)((k + 1) >> 2) & 1u;
    if (lattice) issue(k + 2);   // two tiles ahead; its buffer held tile k - 2, consumed by now
    bool ok_enc = true;
    float2* sPc = sP + pbuf * 2 * M;
    bool valid = true;
    // Decomposed model: the row's level coordinates relative to the domain origin, then one
    // pass per expert with a non-zero gate somewhere in the tile, in ascending expert order
    // (the same order for every row), accumulating G_k y_k and G_k.
    const int shift = job.mode == MODE_L1 || job.shift == 3 ? 3 : 0;
    int rx = 0, ry = 0, rz = 0;
    if (moe) valid = job_coord(job, t, tid, rx, ry, rz);
    const int dox = job.ox, doy = job.oy, doz = job.oz;
    float macc = 0.f, mgs = 0.f, mg = 0.f, y = 0.f;
    float y3[3] = {0.f, 0.f, 0.f};   // the ternary classifier's logits
    for (int pass = 0, last = -1;; ++pass) {
    if (moe) {
      const int mine = moe_next(mv, shift, rx, ry, rz, last);
      if (tid == 0) *smin = 0x7FFFFFFF;
      __syncthreads();
      atomicMin(smin, mine);
      __syncthreads();
      const int e = *smin;
      __syncthreads();
      if (e == 0x7FFFFFFF) break;
      const NetView ev = mv.experts[e];
      if (ev.p32 != staged_p32) {   // uniform: restage (the level's lattice table is shared)
        tc_stage<NIN, W, MODE>(ev, job.mode, lay, smem, staged_p32 == nullptr);
        __syncthreads();
        bh = swh[W];
        wexact = ev.wexact != 0;
        staged_p32 = ev.p32;
      }
      const int4 eo = __ldg(mv.origin + e);
      job.ox = dox + eo.x; job.oy = doy + eo.y; job.oz = doz + eo.z;
      mg = moe_gate(mv, shift, rx, ry, rz, e);
      last = e;
    } else if (pass > 0) {
      break;
    }
    // ---- encoding -> A operand (layer 0) in TMEM.  Inside this kernel the features are
    // ordered (cos_0, sin_0, cos_1, sin_1, ...): packed column f holds frequency f; the
    // first-layer weight tile is packed with the matching column order.
    {
      uint32_t hi[NIN / 2], lo[NIN / 2];
      if (job.mode == MODE_L0) {
        // angle addition: e^{i Phi(v)} = e^{i Phi(origin + dx e_x)} * e^{i Phi(dy e_y + dz e_z)}
        if (!p_ready) {
          if (tid < 2 * M) {
            if (lattice) ok_enc = mbar_wait_bounded(obar + cb, cpar);
            l0_factors<M, MODE>(job, sq, lattice ? sorg[cb] : __ldg(job.nodes + (t >> 2)), t, sPc, tid);
          }
          __syncthreads();
        }
        const int j = tid & 63;
        if (C::ENC16) {
          // complex product in half2: (pc, pc) * (tc, ts) + (-ps, ps) * (ts, tc) = (cos, sin)
          const uint4* P4 = reinterpret_cast<const uint4*>(sPc) + (tid >> 6) * (M / 2);
          const uint4* T4 = reinterpret_cast<const uint4*>(sTh);
#pragma unroll
          for (int f4 = 0; f4 < M / 4; ++f4) {
            const uint4 tq = T4[f4 * 64 + j];
            const uint4 pa = P4[2 * f4], pb = P4[2 * f4 + 1];
            const uint32_t tw[4] = {tq.x, tq.y, tq.z, tq.w};
            const uint32_t pw[8] = {pa.x, pa.y, pa.z, pa.w, pb.x, pb.y, pb.z, pb.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const uint32_t qs = __byte_perm(tw[e], 0, 0x1032);
              const __half2 z = __hfma2(*reinterpret_cast<const __half2*>(&pw[2 * e + 1]),
                                        *reinterpret_cast<const __half2*>(&qs),
                                        __hmul2(*reinterpret_cast<const __half2*>(&pw[2 * e]),
                                                *reinterpret_cast<const __half2*>(&tw[e])));
              hi[4 * f4 + e] = *reinterpret_cast<const uint32_t*>(&z);
              lo[4 * f4 + e] = 0u;
            }
          }
        } else {
          const float4* P4 = reinterpret_cast<const float4*>(sPc) + (tid >> 6) * (M / 2);
          const float4* T4 = reinterpret_cast<const float4*>(sT);
#pragma unroll
          for (int f2 = 0; f2 < M / 2; ++f2) {
            const float4 tq = T4[f2 * 64 + j], pq = P4[f2];
            split_pair<MODE>(fmaf(pq.x, tq.x, -pq.y * tq.y), fmaf(pq.x, tq.y, pq.y * tq.x), hi[2 * f2], lo[2 * f2]);
            split_pair<MODE>(fmaf(pq.z, tq.z, -pq.w * tq.w), fmaf(pq.z, tq.w, pq.w * tq.z), hi[2 * f2 + 1],
                             lo[2 * f2 + 1]);
          }
        }
      } else {
        int cx, cy, cz;
        if (STAGE && job.mode == MODE_L1 && lattice) {   // the staged origin of this tile's level-1 node
          ok_enc = mbar_wait_bounded(obar + cb, cpar);
          const int4 o = sorg[cb];
          const int sl = ((int)(t & 31) << 7) | tid;
          cx = ((o.x - job.ox) >> 3) + (sl >> 8);
          cy = ((o.y - job.oy) >> 3) + ((sl >> 4) & 15);
          cz = ((o.z - job.oz) >> 3) + (sl & 15);
        } else if (KM == 2 && pf_ready) {   // as job_coord, from the coordinates loaded ahead
          cx = (pf_x - job.ox) >> job.shift;
          cy = (pf_y - job.oy) >> job.shift;
          cz = (pf_z - job.oz) >> job.shift;
          valid = pf_ok;
        } else {
          valid = job_coord(job, t, tid, cx, cy, cz);
        }
        // MUFU sin/cos of the exact phase mapped to [-pi, pi): absolute error ~4e-7,
        // below the 16-bit operand rounding of both modes
#pragma unroll
        for (int f = 0; f < M; ++f) {
          const uint32_t ph = ffm_phase(sq, f, cx, cy, cz);
          float sn, cs;
          __sincosf((float)(int32_t)ph * 1.4629180792671596e-09f, &sn, &cs);   // pi / 2^31
          split_pair<MODE>(cs, sn, hi[f], lo[f]);
        }
      }
      store_a_row<NIN>(tlane, hi, lo, comp0);
      if (C::BIAS_MMA) store_bias_chunk<NIN>(tlane);
    }
    if (lattice && (job.mode == MODE_L1 || !p_ready)) waited = k + 1;
    tmem_st_wait();
    tc_fence_before();
    if (__syncthreads_or(!ok_enc)) { failed = true; break; }
    for (int l = 0; l < L; ++l) {
      const int K = l == 0 ? NIN : W;                 // real columns; the tiles are K + 16 wide
      if (tid == 0 && MODE == TC_FP8 && l > 0) {   // E4M3 hidden layer: K = W, 32 per MMA
        tc_fence_after();
        const uint32_t b0 = smem_u32(sw) + f8_tiles + (uint32_t)((l - 1) * W * W);
        for (int ks = 0; ks < W / 32; ++ks)
          mma_f8kind_ts(tbase, tbase + C::A_HI + ks * 8, smem_desc(b0 + ks * 256, 128, W * 8), idesc, ks > 0 ? 1u : 0u);
        mma_commit(bar);
      } else if (tid == 0) {
        tc_fence_after();
        const uint32_t woff = l == 0 ? 0u : (uint32_t)(W * C::K0 + (l - 1) * W * C::KH) * 2u;
        const uint32_t sbo = (uint32_t)(K + 16) * 16u;
        // K step ks reads the tile 256 bytes further on: +16 in the descriptor's address
        // field (addresses stay below 2^18, so the 14-bit field does not carry)
        const uint64_t bd0 = smem_desc(smem_u32(sw) + woff, 128, sbo), bl0 = smem_desc(smem_u32(sw_lo) + woff, 128, sbo);
        const bool comp = comp_in<MODE>(l, L);
        auto issue_layer = [&](auto nks) {   // nks K steps, unrolled
#pragma unroll
          for (int ks = 0; ks < decltype(nks)::value; ++ks) {
            const uint64_t bd = bd0 + (uint64_t)(ks * 16);
            mma_f16kind_ts(tbase, tbase + C::A_HI + ks * 8, bd, idesc, ks > 0 ? 1u : 0u);
            if (C::WLO) {
              if (comp) mma_f16kind_ts(tbase, tbase + C::A_LO + ks * 8, bd, idesc, 1u);
              if (!wexact)   // A_hi * W_lo vanishes for BF16-exact weights
                mma_f16kind_ts(tbase, tbase + C::A_HI + ks * 8, bl0 + (uint64_t)(ks * 16), idesc, 1u);
            }
          }
        };
        if (l == 0) issue_layer(std::integral_constant<int, NIN / 16 + (C::BIAS_MMA ? 1 : 0)>{});
        else issue_layer(std::integral_constant<int, W / 16 + (C::BIAS_MMA ? 1 : 0)>{});
        mma_commit(bar);
      }
      bool ok = true;
      // the next tile's factors, into the other buffer, by the last 2M threads (warp 0 is
      // busy issuing the MMAs, so its share would outlast them)
      if (l == 0 && next_same && tid >= kTile - 2 * M) {
        if (lattice) ok = mbar_wait_bounded(obar + nb, npar);
        l0_factors<M, MODE>(job, sq, lattice ? sorg[nb] : __ldg(job.nodes + (tn >> 2)), tn, sP + (pbuf ^ 1) * 2 * M,
                            tid - (kTile - 2 * M));
      }
      if (l == 0 && next_same) waited = k + 2;
      if (KM == 2 && l == 0 && next_list) {   // the next tile's coordinates: used only at its encoding
        int64_t i = tn * kTile + tid;
        pf_ok = i < job.n_items;
        if (!pf_ok) i = job.n_items - 1;
        pf_x = __ldg(job.ijk + 3 * i);
        pf_y = __ldg(job.ijk + 3 * i + 1);
        pf_z = __ldg(job.ijk + 3 * i + 2);
      }
      ok = mbar_wait_bounded(bar, phase) && ok;
      phase ^= 1u;
      tc_fence_after();
      uint32_t accu[W];
      tmem_ld32_nowait(tlane, accu);
      if (W == 64) tmem_ld32_nowait(tlane + 32, accu + 32);
      tmem_ld_wait();
      if (MODE == TC_FP8) {   // h = relu(alpha D + beta): E4M3 input of the next layer, or the head's input
        const float al = f8_aux[l];
        const float2* be = reinterpret_cast<const float2*>(f8_aux + kMaxLayers + l * W);
#pragma unroll
        for (int c = 0; c < W / 2; ++c) {
          const float2 h = ffma2(make_float2(al, al), make_float2(__uint_as_float(accu[2 * c]), __uint_as_float(accu[2 * c + 1])),
                                 be[c]);
          accu[2 * c] = __float_as_uint(h.x);
          accu[2 * c + 1] = __float_as_uint(h.y);
        }
      } else if (!C::BIAS_MMA) {   // FP32 bias
        const float2* bl2 = reinterpret_cast<const float2*>(sb + l * W);
#pragma unroll
        for (int c = 0; c < W / 2; ++c) {   // 1 * D + b: one rounding, as an add
          const float2 h = ffma2(make_float2(1.f, 1.f), make_float2(__uint_as_float(accu[2 * c]), __uint_as_float(accu[2 * c + 1])),
                                 bl2[c]);
          accu[2 * c] = __float_as_uint(h.x);
          accu[2 * c + 1] = __float_as_uint(h.y);
        }
      }
      if constexpr (SIN) {   // h = sin(omega a), applied before the conversions below
#pragma unroll
        for (int c = 0; c < W; ++c) accu[c] = __float_as_uint(__sinf(om * __uint_as_float(accu[c])));
      }
      if (MODE == TC_FP8 && l < L - 1) {
        uint32_t q[W / 4];
#pragma unroll
        for (int c = 0; c < W / 4; ++c)
          q[c] = cvt_relu_e4m3x2(__uint_as_float(accu[4 * c]), __uint_as_float(accu[4 * c + 1])) |
                 (cvt_relu_e4m3x2(__uint_as_float(accu[4 * c + 2]), __uint_as_float(accu[4 * c + 3])) << 16);
        tmem_st_cols<W / 4>(tlane + C::A_HI, q);
        tmem_st_wait();
      } else if (l < L - 1) {
        const bool comp = comp_in<MODE>(l + 1, L);
        uint32_t hi[W / 2], lo[W / 2];
#pragma unroll
        for (int p = 0; p < W / 2; ++p) {
          if constexpr (SIN) sin_pair<MODE>(__uint_as_float(accu[2 * p]), __uint_as_float(accu[2 * p + 1]), comp, hi[p], lo[p]);
          else relu_pair<MODE>(__uint_as_float(accu[2 * p]), __uint_as_float(accu[2 * p + 1]), comp, hi[p], lo[p]);
        }
        store_a_row<W>(tlane, hi, lo, comp);
        if (C::BIAS_MMA && NIN != W) store_bias_chunk<W>(tlane);   // equal widths: still in place
        tmem_st_wait();
      } else {
        // FP32 head, two products per instruction.  The summation order is that of
        // mlp_tc2_kernel (each half of the columns in two pair accumulators, then the
        // halves added), so both variants give the same bits.  The ternary classifier
        // takes one such dot product per class.
#pragma unroll
        for (int cls = 0; cls < (TERN ? 3 : 1); ++cls) {
          const float4* swh4 = reinterpret_cast<const float4*>(swh + cls * W);
          float part[2];
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            float2 acc[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
#pragma unroll
            for (int c = h * (W / 8); c < (h + 1) * (W / 8); ++c) {
              const float4 wv = swh4[c];
              const float lo_ = SIN ? -3.4e38f : 0.f;   // sin outputs pass unclipped
              acc[0] = ffma2(make_float2(wv.x, wv.y),
                             make_float2(fmaxf(__uint_as_float(accu[4 * c]), lo_), fmaxf(__uint_as_float(accu[4 * c + 1]), lo_)), acc[0]);
              acc[1] = ffma2(make_float2(wv.z, wv.w),
                             make_float2(fmaxf(__uint_as_float(accu[4 * c + 2]), lo_), fmaxf(__uint_as_float(accu[4 * c + 3]), lo_)), acc[1]);
            }
            part[h] = (acc[0].x + acc[0].y) + (acc[1].x + acc[1].y);
          }
          if constexpr (TERN) y3[cls] = swh[3 * W + cls] + (part[0] + part[1]);
          else y = bh + (part[0] + part[1]);
        }
      }
      tc_fence_before();
      if (__syncthreads_or(!ok)) { failed = true; break; }   // all threads agree on a timeout
    }
    if (failed) break;
    if (moe) {
      macc = fmaf(mg, y, macc);
      mgs += mg;
    }
    }   // expert passes
    if (failed) break;
    if (moe) y = macc / mgs;
    if constexpr (TERN) job_output3(job, t, tid, valid, y3);
    else job_output(job, t, tid, valid, y);
    if (next_same) pbuf ^= 1;
    p_ready = next_same;
    pf_ready = next_list;
  }
  // copies still in flight (after a timeout): wait for them, bounded, before the shared
  // memory they write is released
  if (tid == 0 && lattice)
    for (; waited < issued && !failed; ++waited) failed = !mbar_wait_bounded(obar + (waited & 3), (uint32_t)(waited >> 2) & 1u);
  if (failed && tid == 0) set_status(b.it[0].job.status, ST_TIMEOUT);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tbase, C::COLS);
}

// FP32 master weights -> FP16 tiles, BF16 hi tiles and BF16 lo tiles in the
// canonical K-major layout: layer 0 [W x (n_in+16)], layers 1..L-1 [W x (W+16)];
// column K of a layer's tile is its bias (FP16 tiles: column K+1 the FP16 remainder of the
// bias), the other columns after it are zero.
static __global__ void pack_weights_kernel(const float* p32, uint8_t* wpk, int nin, int W, int L) {
  const int64_t total = wtile_elems(nin, W, L);
  const int64_t first = (int64_t)W * (nin + 16);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int l, K, o, i;
    size_t base;
    if (e < first) {
      l = 0; K = nin; o = (int)(e / (nin + 16)); i = (int)(e % (nin + 16)); base = 0;
    } else {
      const int64_t r = e - first;
      l = 1 + (int)(r / ((int64_t)W * (W + 16)));
      const int rr = (int)(r % ((int64_t)W * (W + 16)));
      K = W; o = rr / (W + 16); i = rr % (W + 16);
      base = (size_t)first * 2 + (size_t)(l - 1) * W * (W + 16) * 2;
    }
    const int64_t woff = l == 0 ? 0 : (int64_t)W * nin + W + (int64_t)(l - 1) * (W * W + W);
    // layer 0: packed column i holds feature (i even: cos_{i/2}, i odd: sin_{i/2}),
    // i.e. column i/2 or nin/2 + i/2 of W_0
    const int src = (l == 0 && i < K) ? ((i & 1) ? nin / 2 + (i >> 1) : (i >> 1)) : i;
    const float v = i < K ? p32[woff + (int64_t)o * K + src] : (i == K ? p32[woff + (int64_t)W * K + o] : 0.f);
    const size_t off = base + canon_off(o, i, K + 16);
    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
    if (i == K + 1) {   // FP16 tiles: the remainder of the bias, b - fp16(b)
      const float bv = p32[woff + (int64_t)W * K + o];
      *reinterpret_cast<__half*>(wpk + off) = __float2half_rn(bv - __half2float(__float2half_rn(bv)));
    } else {
      *reinterpret_cast<__half*>(wpk + off) = __float2half_rn(v);
    }
    *reinterpret_cast<__nv_bfloat16*>(wpk + total * 2 + off) = hi;
    *reinterpret_cast<__nv_bfloat16*>(wpk + total * 4 + off) = __float2bfloat16_rn(v - __bfloat162float(hi));
  }
}

// Largest ReLU output of every hidden layer of a network over n seeded lattice points of
// its domain (coordinates uniform in [0, 2^log2_extent) per axis, in the level's units),
// as float bits merged with atomicMax (the values are >= 0).  It calibrates the E4M3
// activation scales of TC_FP8 from the model alone, so an imported model gets the same.
template <int NIN, int W>
__global__ void calib_amax_kernel(NetView net, int log2_extent, uint64_t seed, int n, uint32_t* amax_bits) {
  constexpr int H = NIN > W ? NIN : W;
  __shared__ uint32_t sq[3 * (NIN / 2)];
  for (int i = threadIdx.x; i < 3 * (NIN / 2); i += blockDim.x) sq[i] = net.q[i];
  __syncthreads();
  const int L = net.layers;
  const uint32_t mask = (1u << log2_extent) - 1u;
  float lmax[kMaxLayers];   // the layer loop is not unrolled: this array lives in local memory
  for (int l = 0; l < kMaxLayers; ++l) lmax[l] = 0.f;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
    uint64_t z = seed + 0x9E3779B97F4A7C15ull * (uint64_t)(s + 1);   // SplitMix64 finaliser
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    float h[H], a[W];
    encode_f32<NIN>(sq, (int)(z & mask), (int)((z >> 21) & mask), (int)((z >> 42) & mask), h);
    const float* p = net.p32;
#pragma unroll 1
    for (int l = 0; l < L; ++l) {
      if (l == 0) {
        dense_f32<NIN, W>(p, h, a);
        p += W * NIN + W;
      } else {
        dense_f32<W, W>(p, h, a);
        p += W * W + W;
      }
#pragma unroll
      for (int o = 0; o < W; ++o) {
        h[o] = fmaxf(a[o], 0.f);
        lmax[l] = fmaxf(lmax[l], h[o]);
      }
    }
  }
  for (int l = 0; l < L; ++l) {
    float v = lmax[l];
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) atomicMax(amax_bits + l, __float_as_uint(v));
  }
}

// Headroom of the measured FP8 activation ranges over the calibration amax: the calibration
// points cover the whole domain, the decoded candidates sit near the surfaces, where a
// layer's outputs can exceed what the domain-wide sample saw.  E4M3 keeps the same relative
// precision over 2^14.8 of normal range, so the headroom costs nothing in the bulk.
constexpr float kFp8Headroom = 16.f;

// The FP8 part of the packed weights (fp8_tile_bytes, fp8_aux_bytes) for one network;
// one block of 256 threads.  Activation ranges: kFp8Headroom times the largest output of
// layer l that calib_amax_kernel measured (amax_bits, may be nullptr), capped by a bound that holds for
// every input since the encoding is bounded by 1 in absolute value:
//   a_0 = 1,  a_{l+1} <= max_o (sum_i |W_l[o][i]| a_l + |b_l[o]|)   (range of layer l's output);
// a tensor with bound a is stored as E4M3 of x / s, s = a / 448 (E4M3's largest finite
// value); layer l >= 1 stores E4M3 of W_l / s_w, s_w = max |W_l| / 448.  Epilogue constants:
//   l = 0 (FP16 layer): alpha = 1 / s_{a_1}, beta = b_0 / s_{a_1} (alpha = 1, beta = b_0 if L = 1);
//   0 < l < L-1: alpha = s_w s_{a_l} / s_{a_{l+1}}, beta = b_l / s_{a_{l+1}};
//   l = L-1 > 0: alpha = s_w s_{a_l}, beta = b_l (the FP32 input of the head).
static __global__ void pack_fp8_kernel(const float* p32, uint8_t* wpk, int nin, int W, int L, const uint32_t* amax_bits) {
  __shared__ float red_b[256], red_w[256];
  uint8_t* tiles = wpk + wpk_fp8_off(nin, W, L);
  float* aux = reinterpret_cast<float*>(tiles + fp8_tile_bytes(W, L));
  const int tid = threadIdx.x;
  float a_in = 1.f;
  int64_t woff = 0;
  for (int l = 0; l < L; ++l) {
    const int K = l == 0 ? nin : W;
    const float* Wl = p32 + woff;
    const float* bl = Wl + (int64_t)W * K;
    float rb = 0.f, wm = 0.f;
    for (int o = tid; o < W; o += blockDim.x) {
      float sum = 0.f;
      for (int i = 0; i < K; ++i) {
        const float w = fabsf(Wl[(int64_t)o * K + i]);
        sum += w;
        wm = fmaxf(wm, w);
      }
      rb = fmaxf(rb, sum * a_in + fabsf(bl[o]));
    }
    red_b[tid] = rb;
    red_w[tid] = wm;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
      if (tid < h) {
        red_b[tid] = fmaxf(red_b[tid], red_b[tid + h]);
        red_w[tid] = fmaxf(red_w[tid], red_w[tid + h]);
      }
      __syncthreads();
    }
    // the measured range (with headroom) where there is one, else the bound
    const float meas = amax_bits && l < L - 1 ? kFp8Headroom * __uint_as_float(amax_bits[l]) : 0.f;
    const float a_out = meas > 0.f ? fminf(meas, red_b[0]) : red_b[0] > 0.f ? red_b[0] : 1.f;
    const float s_in = a_in / 448.f, s_out = a_out / 448.f, s_w = red_w[0] > 0.f ? red_w[0] / 448.f : 1.f;
    float alpha, bscale;
    if (l == 0) {   // FP16 layer; its bias is added in the epilogue like the others
      alpha = L > 1 ? 1.f / s_out : 1.f;
      bscale = alpha;
    } else if (l < L - 1) {
      alpha = s_w * s_in / s_out;
      bscale = 1.f / s_out;
    } else {
      alpha = s_w * s_in;
      bscale = 1.f;
    }
    if (tid == 0) aux[l] = alpha;
    for (int o = tid; o < W; o += blockDim.x) aux[kMaxLayers + l * W + o] = bl[o] * bscale;
    if (l > 0) {
      uint8_t* tl = tiles + (int64_t)(l - 1) * W * W;
      for (int e = tid; e < W * W; e += blockDim.x) {
        const int o = e / W, i = e % W;
        tl[canon_off8(o, i, W)] = (uint8_t)(cvt_e4m3x2(Wl[(int64_t)o * W + i] / s_w, 0.f) & 0xFFu);
      }
    }
    __syncthreads();   // red_* are reused by the next layer
    a_in = a_out;
    woff += (int64_t)W * K + W;
  }
}

}  // namespace nvdb
