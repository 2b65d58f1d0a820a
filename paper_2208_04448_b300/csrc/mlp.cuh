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
#include <cuda_fp16.h>

#include "common.cuh"

namespace nvdb {

struct NetView {
  int n_in, width, layers;
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
  uint32_t* words;        // MODE_L1/L0: candidate bits, word (tile*4 + warp)
  float* out;             // MODE_LIST: outputs
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

__host__ __device__ inline int64_t net_param_count(int nin, int w, int L) {
  return (int64_t)w * nin + w + (int64_t)(L - 1) * (w * w + w) + w + 1;
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
__device__ __forceinline__ float forward_f32(const float* sp, const uint32_t* sq, int L, int cx, int cy, int cz) {
  constexpr int H = NIN > W ? NIN : W;
  float h[H], a[W];
  encode_f32<NIN>(sq, cx, cy, cz, h);
  const float* p = sp;
  dense_f32<NIN, W>(p, h, a);
  p += W * NIN + W;
#pragma unroll
  for (int o = 0; o < W; ++o) h[o] = fmaxf(a[o], 0.f);
  for (int l = 1; l < L; ++l) {
    dense_f32<W, W>(p, h, a);
    p += W * W + W;
#pragma unroll
    for (int o = 0; o < W; ++o) h[o] = fmaxf(a[o], 0.f);
  }
  float y = p[W];
#pragma unroll
  for (int i = 0; i < W; ++i) y = fmaf(p[i], h[i], y);
  return y;
}

template <int NIN, int W>
__host__ __device__ inline size_t f32_smem_bytes(int L) {
  const int64_t P = net_param_count(NIN, W, L);
  return (size_t)((P + 3) & ~3ll) * 4 + (size_t)(NIN / 2) * 3 * 4;
}

template <int NIN, int W>
__global__ void __launch_bounds__(kTile) mlp_f32_kernel(NetView net, EvalJob job) {
  extern __shared__ float4 smem_f4[];
  float* sp = reinterpret_cast<float*>(smem_f4);
  const int L = net.layers;
  const int64_t P = net_param_count(NIN, W, L);
  uint32_t* sq = reinterpret_cast<uint32_t*>(sp + ((P + 3) & ~3ll));
  for (int64_t i = threadIdx.x; i < P; i += blockDim.x) sp[i] = __ldg(net.p32 + i);
  for (int i = threadIdx.x; i < 3 * (NIN / 2); i += blockDim.x) sq[i] = __ldg(net.q + i);
  __syncthreads();
  if (job.n_dev) job.n_items = *job.n_dev;
  const int64_t ntiles = job_tiles(job.mode, job.n_items);
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    int cx, cy, cz;
    const bool valid = job_coord(job, t, threadIdx.x, cx, cy, cz);
    const float y = forward_f32<NIN, W>(sp, sq, L, cx, cy, cz);
    job_output(job, t, threadIdx.x, valid, y);
  }
}

// ============================================================== tcgen05 tensor-core path
// Two operand modes of kind::f16 (same tensor rate):
//  TC_BF16X3: activations and weights carried as BF16 pairs v = hi + lo
//             (hi = bf16(v), lo = bf16(v - hi)); D = A_hi W_hi + A_lo W_hi + A_hi W_lo,
//             three MMAs per K step, error ~2^-16 relative.
//  TC_FP16  : FP16 activations and weights, one MMA per K step.
enum TcMode : int { TC_BF16X3 = 0, TC_FP16 = 1 };

template <int MODE>
__device__ __forceinline__ void pack8(const float* v, uint4& hi, uint4& lo) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    if (MODE == TC_FP16) {
      __half2 x = __floats2half2_rn(v[2 * e], v[2 * e + 1]);
      h[e] = *reinterpret_cast<uint32_t*>(&x);
      l[e] = 0u;
    } else {
      __nv_bfloat162 x = __floats2bfloat162_rn(v[2 * e], v[2 * e + 1]);
      const float2 back = __bfloat1622float2(x);
      __nv_bfloat162 y = __floats2bfloat162_rn(v[2 * e] - back.x, v[2 * e + 1] - back.y);
      h[e] = *reinterpret_cast<uint32_t*>(&x);
      l[e] = *reinterpret_cast<uint32_t*>(&y);
    }
  }
  hi = make_uint4(h[0], h[1], h[2], h[3]);
  lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// Features of row r written into the A tile(s) (K = NIN): cos then sin.
template <int NIN, int MODE>
__device__ __forceinline__ void encode_tc_row(uint8_t* sa, uint8_t* sa_lo, int r, const uint32_t* sq, int cx, int cy,
                                              int cz) {
  constexpr int M = NIN / 2;
  float c[M], s[M];
#pragma unroll
  for (int f = 0; f < M; ++f) {
    const uint32_t ph = ffm_phase(sq, f, cx, cy, cz);
    if (MODE == TC_FP16)
      __sincosf((float)(int32_t)ph * 1.4629180792671596e-09f, &s[f], &c[f]);   // pi / 2^31
    else
      sincospif((float)(int32_t)ph * 0x1p-31f, &s[f], &c[f]);
  }
#pragma unroll
  for (int g = 0; g < M / 8; ++g) {
    uint4 hi, lo;
    pack8<MODE>(c + 8 * g, hi, lo);
    *reinterpret_cast<uint4*>(sa + canon_off(r, 8 * g, NIN)) = hi;
    if (MODE == TC_BF16X3) *reinterpret_cast<uint4*>(sa_lo + canon_off(r, 8 * g, NIN)) = lo;
    pack8<MODE>(s + 8 * g, hi, lo);
    *reinterpret_cast<uint4*>(sa + canon_off(r, M + 8 * g, NIN)) = hi;
    if (MODE == TC_BF16X3) *reinterpret_cast<uint4*>(sa_lo + canon_off(r, M + 8 * g, NIN)) = lo;
  }
}

constexpr uint32_t kTmemCols = 64;          // FP32 accumulator columns (width <= 64)
constexpr size_t kTcMinSmem = 33 * 1024;    // caps residency at 6 CTAs/SM -> 6 x 64 <= 512 TMEM columns

// Packed weight tiles per network: [FP16 tiles][BF16 hi tiles][BF16 lo tiles],
// each set = layer 0 [W x n_in] then layers 1..L-1 [W x W], canonical layout.
__host__ __device__ inline int64_t wtile_elems(int nin, int w, int L) { return (int64_t)w * nin + (int64_t)(L - 1) * w * w; }

template <int NIN, int W, int MODE>
struct TcLayout {
  static constexpr int KA = NIN > W ? NIN : W;
  static constexpr int NCOPY = MODE == TC_BF16X3 ? 2 : 1;
  size_t w_bytes, a_off, alo_off, b_off, wh_off, q_off, bar_off, slot_off, total;
  __host__ __device__ TcLayout(int L) {
    w_bytes = (size_t)wtile_elems(NIN, W, L) * 2;              // one copy
    a_off = ((NCOPY * w_bytes) + 127) & ~(size_t)127;
    alo_off = a_off + (size_t)kTile * KA * 2;
    b_off = a_off + (size_t)NCOPY * kTile * KA * 2;
    wh_off = b_off + (size_t)L * W * 4;
    q_off = wh_off + (size_t)(W + 4) * 4;
    bar_off = (q_off + (size_t)(NIN / 2) * 12 + 7) & ~(size_t)7;
    slot_off = bar_off + 8;
    total = slot_off + 8;
    if (total < kTcMinSmem) total = kTcMinSmem;
  }
};

template <int NIN, int W, int MODE>
__global__ void __launch_bounds__(kTile, 1) mlp_tc_kernel(NetView net, EvalJob job) {
  static_assert(W == 32 || W == 64, "width");
  static_assert(NIN == 32 || NIN == 64, "encoding size");
  extern __shared__ __align__(1024) uint8_t smem[];
  const int L = net.layers;
  const TcLayout<NIN, W, MODE> lay(L);
  uint8_t* sw = smem;                              // hi (or FP16) weights
  uint8_t* sw_lo = smem + lay.w_bytes;             // lo weights (BF16X3)
  uint8_t* sa = smem + lay.a_off;
  uint8_t* sa_lo = smem + lay.alo_off;
  float* sb = reinterpret_cast<float*>(smem + lay.b_off);
  float* swh = reinterpret_cast<float*>(smem + lay.wh_off);
  uint32_t* sq = reinterpret_cast<uint32_t*>(smem + lay.q_off);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + lay.bar_off);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + lay.slot_off);
  const int tid = threadIdx.x, warp = tid >> 5;

  // stage weight tiles, biases, head and Fourier matrix
  {
    const int64_t te = wtile_elems(NIN, W, L);
    const uint8_t* base = reinterpret_cast<const uint8_t*>(net.wpk) + (MODE == TC_FP16 ? 0 : te * 2);
    const uint4* src = reinterpret_cast<const uint4*>(base);
    uint4* dst = reinterpret_cast<uint4*>(sw);
    const size_t n16 = lay.NCOPY * lay.w_bytes / 16;
    for (size_t i = tid; i < n16; i += kTile) dst[i] = __ldg(src + i);
    for (int l = 0; l < L; ++l) {
      const int64_t off = l == 0 ? (int64_t)W * NIN : (int64_t)W * NIN + W + (int64_t)(l - 1) * (W * W + W) + W * W;
      for (int o = tid; o < W; o += kTile) sb[l * W + o] = __ldg(net.p32 + off + o);
    }
    const int64_t hoff = net_param_count(NIN, W, L) - W - 1;
    for (int o = tid; o <= W; o += kTile) swh[o] = __ldg(net.p32 + hoff + o);
    for (int i = tid; i < 3 * (NIN / 2); i += kTile) sq[i] = __ldg(net.q + i);
  }
  if (tid == 0) mbar_init(bar, 1);
  if (warp == 0) tmem_alloc(tslot, kTmemCols);
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *tslot;
  const uint32_t tlane = tbase + ((uint32_t)(warp * 32) << 16);
  const float bh = swh[W];
  const uint32_t idesc = MODE == TC_FP16 ? idesc_f16_f32(kTile, W) : idesc_bf16_f32(kTile, W);

  uint32_t phase = 0;
  bool failed = false;
  if (job.n_dev) job.n_items = *job.n_dev;
  const int64_t ntiles = job_tiles(job.mode, job.n_items);
  for (int64_t t = blockIdx.x; t < ntiles && !failed; t += gridDim.x) {
    int cx, cy, cz;
    const bool valid = job_coord(job, t, tid, cx, cy, cz);
    encode_tc_row<NIN, MODE>(sa, sa_lo, tid, sq, cx, cy, cz);
    fence_proxy_async_smem();
    __syncthreads();
    float y = 0.f;
    for (int l = 0; l < L; ++l) {
      const int K = l == 0 ? NIN : W;
      if (tid == 0) {
        tc_fence_after();
        const uint32_t woff = l == 0 ? 0u : (uint32_t)(W * NIN + (l - 1) * W * W) * 2u;
        const uint32_t a0 = smem_u32(sa), b0 = smem_u32(sw) + woff;
        for (int ks = 0; ks < K / 16; ++ks) {
          mma_f16kind(tbase, smem_desc(a0 + ks * 256, 128, K * 16), smem_desc(b0 + ks * 256, 128, K * 16), idesc,
                      ks > 0 ? 1u : 0u);
          if (MODE == TC_BF16X3) {
            const uint32_t al = smem_u32(sa_lo), bl = smem_u32(sw_lo) + woff;
            mma_f16kind(tbase, smem_desc(al + ks * 256, 128, K * 16), smem_desc(b0 + ks * 256, 128, K * 16), idesc, 1u);
            mma_f16kind(tbase, smem_desc(a0 + ks * 256, 128, K * 16), smem_desc(bl + ks * 256, 128, K * 16), idesc, 1u);
          }
        }
        mma_commit(bar);
      }
      const bool ok = mbar_wait_bounded(bar, phase);
      phase ^= 1u;
      if (__syncthreads_or(!ok)) { failed = true; break; }
      tc_fence_after();
      float acc[W];
      tmem_ld32(tlane, acc);
      if (W == 64) tmem_ld32(tlane + 32, acc + 32);
      const float* b = sb + l * W;
      if (l < L - 1) {
#pragma unroll
        for (int g = 0; g < W / 8; ++g) {
          float v[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) v[e] = fmaxf(acc[8 * g + e] + b[8 * g + e], 0.f);
          uint4 hi, lo;
          pack8<MODE>(v, hi, lo);
          *reinterpret_cast<uint4*>(sa + canon_off(tid, 8 * g, W)) = hi;
          if (MODE == TC_BF16X3) *reinterpret_cast<uint4*>(sa_lo + canon_off(tid, 8 * g, W)) = lo;
        }
      } else {
        y = bh;
#pragma unroll
        for (int c = 0; c < W; ++c) y = fmaf(swh[c], fmaxf(acc[c] + b[c], 0.f), y);
      }
      tc_fence_before();
      fence_proxy_async_smem();
      __syncthreads();
    }
    if (failed) break;
    job_output(job, t, tid, valid, y);
  }
  if (failed && tid == 0) set_status(job.status, ST_TIMEOUT);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tbase, kTmemCols);
}

// FP32 master weights -> FP16 tiles, BF16 hi tiles and BF16 lo tiles in the
// canonical K-major layout (layer 0: [W x n_in], layers 1..L-1: [W x W]).
__global__ void pack_weights_kernel(const float* p32, uint8_t* wpk, int nin, int W, int L) {
  const int64_t first = (int64_t)W * nin;
  const int64_t total = wtile_elems(nin, W, L);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    float v;
    size_t off;
    if (e < first) {
      const int o = (int)(e / nin), i = (int)(e % nin);
      v = p32[e];
      off = canon_off(o, i, nin);
    } else {
      const int64_t r = e - first;
      const int l = 1 + (int)(r / ((int64_t)W * W));
      const int rr = (int)(r % ((int64_t)W * W));
      const int o = rr / W, i = rr % W;
      v = p32[first + W + (int64_t)(l - 1) * (W * W + W) + rr];
      off = (size_t)first * 2 + (size_t)(l - 1) * W * W * 2 + canon_off(o, i, W);
    }
    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
    *reinterpret_cast<__half*>(wpk + off) = __float2half_rn(v);
    *reinterpret_cast<__nv_bfloat16*>(wpk + total * 2 + off) = hi;
    *reinterpret_cast<__nv_bfloat16*>(wpk + total * 4 + off) = __float2bfloat16_rn(v - __bfloat162float(hi));
  }
}

}  // namespace nvdb
