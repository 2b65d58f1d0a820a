// Sparse-field training (Section 3.2, Section 3.2.1): Philox-sampled batches,
// encode + forward with saved activations, hand-written backward of the mean
// BCE / MSE / L1 loss, deterministic per-CTA gradient partials, then a
// fixed-order reduction fused with the Adam update (Kingma & Ba; beta1 0.9,
// beta2 0.999, eps 1e-8, bias correction, exponentially decayed rate).
//
// FP32 on CUDA cores; one thread per sample row, 128 rows per tile.
// Shared memory holds the activations H_0..H_L and the backward deltas of the
// tile ([128][K+1] FP32 each, padded against bank conflicts); weights are read
// through L1 (broadcast loads).
#pragma once
#include "common.cuh"
#include "mlp.cuh"

namespace nvdb {

struct TrainJob {
  int net;                    // 0 level-1 classifier, 1 level-0 classifier, 2 regressor, 3 tile regressor
  int stream;                 // sample stream of the network: 3 expert + net (net without experts)
  int loss;                   // LOSS_*
  int step;                   // Adam step (1-based), keys the sample stream
  uint64_t seed;
  int64_t batch;              // samples per step
  int ox, oy, oz;             // encoding domain origin
  // explicit list (nvdb_mlp_grad) when ijk_list != nullptr
  const int32_t* ijk_list;
  const float* target_list;
  // population from the explicit grid
  const int4* l1_origin; const unsigned long long* l1_mask; int64_t n_l1;
  // active tiles (a pruned grid): the ternary level-1 label is 1 on a tile slot, 0 on a
  // child leaf, 2 elsewhere; the tile regressor (net 3) samples tile leaves (via pop) and
  // regresses the tile value at the slot's leaf-unit coordinate
  const unsigned long long* l1_tile_mask;
  const int4* leaf_origin; const unsigned long long* leaf_mask; int64_t n_leaf;
  const int32_t* ijk; const float* val; int64_t n;
  // a domain decomposition's expert samples a sub-population (Section 3.4): element i is
  // (pop[i >> pop_shift] << pop_shift) | (i & (2^pop_shift - 1)) of the population above,
  // pop_n << pop_shift elements (pop_shift = 9 for the level-0 classifier: lists of leaves)
  const uint32_t* pop; int64_t pop_n; int pop_shift;
  // subset resampling (Appendix E): every `resample` steps a subset of resample * batch
  // candidates is drawn (element i of interval r: Philox counter (i / 4, r, stream, 1), word
  // i % 4); each step draws its batch from the current subset.  0 = a fresh batch per step.
  int resample;
  // regressor population (Appendix C ablation): 0 the active voxels (sparse, the method),
  // 1 every voxel of the leaves (blocked), 2 every voxel of the domain's bounding box (dense,
  // log2 extent <= 10); inactive voxels take the target bg_target (the background)
  int sampling;
  const int64_t* leaf_first;  // blocked / dense: index of each leaf's first voxel
  int log2e, gx, gy, gz;      // dense: domain extent and origin
  float bg_target;
  float tscale;               // regressor target = val * tscale
  float* partial;             // [gridDim.x][P + 1]: gradient partials, then the loss sum
  uint32_t* status;           // ST_* bits (tensor-core kernel: a timed-out wait)
  int* step_dev;              // if set: the step is step_dev[0] (a graph replays fixed launches);
                              // block 0 copies it to step_dev[1] for the Adam kernel
};

// Read the step from device memory when the launch carries no fixed step.
__device__ __forceinline__ void take_step(TrainJob& job) {
  if (!job.step_dev) return;
  job.step = job.step_dev[0];
  if (blockIdx.x == 0 && threadIdx.x == 0) job.step_dev[1] = job.step;
}

// LOSS_LINEAR: the target is the caller's dL/dy per sample (a vector-Jacobian product,
// as an autograd backward needs): loss term t y, gradient t, no 1/batch factor.
// LOSS_CE: softmax cross-entropy of the ternary classifier's three logits (its only loss).
enum : int { LOSS_MSE = 0, LOSS_L1 = 1, LOSS_BCE = 2, LOSS_LINEAR = 3, LOSS_CE = 4 };

__device__ __forceinline__ int64_t train_population(const TrainJob& j) {
  if (j.pop) return j.pop_n << j.pop_shift;
  if (j.net == 2 && j.sampling == 1) return j.n_leaf * 512;
  if (j.net == 2 && j.sampling == 2) return (int64_t)1 << (3 * j.log2e);
  return j.net == 0 ? j.n_l1 * 4096 : j.net == 1 ? j.n_leaf * 512 : j.net == 3 ? j.n_leaf : j.n;
}

// Canonical key of the leaf holding voxel (i, j, k): level-2 key, level-1 slot, leaf slot.
__device__ __forceinline__ uint64_t leaf_key(int i, int j, int k) {
  const uint64_t l2 = ((uint64_t)(i >> 12) << 18) | ((uint64_t)(j >> 12) << 9) | (uint64_t)(k >> 12);
  const uint64_t l1 = (uint64_t)((((i >> 7) & 31) << 10) | (((j >> 7) & 31) << 5) | ((k >> 7) & 31));
  const uint64_t lf = (uint64_t)((((i >> 3) & 15) << 8) | (((j >> 3) & 15) << 4) | ((k >> 3) & 15));
  return (l2 << 27) | (l1 << 12) | lf;
}

// Value target of voxel `off` of leaf `leaf` (offset bit set: its value; else the background).
__device__ __forceinline__ float leaf_voxel_target(const TrainJob& j, int64_t leaf, int off) {
  const unsigned long long* w = j.leaf_mask + leaf * 8;
  if (!((w[off >> 6] >> (off & 63)) & 1ull)) return j.bg_target;
  int64_t vi = j.leaf_first[leaf];
  for (int q = 0; q < (off >> 6); ++q) vi += __popcll(w[q]);
  vi += __popcll(w[off >> 6] & ((1ull << (off & 63)) - 1ull));
  return j.val[vi] * j.tscale;
}

// Coordinates (level units) and target of sample s.
__device__ __forceinline__ void train_sample(const TrainJob& j, int64_t s, int& cx, int& cy, int& cz, float& tgt) {
  if (j.ijk_list) {
    const int sh = j.net == 0 || j.net == 3 ? 3 : 0;
    cx = (j.ijk_list[3 * s] - j.ox) >> sh;
    cy = (j.ijk_list[3 * s + 1] - j.oy) >> sh;
    cz = (j.ijk_list[3 * s + 2] - j.oz) >> sh;
    tgt = j.target_list[s];
    return;
  }
  const uint64_t npop = (uint64_t)train_population(j);
  uint64_t idx;
  if (j.resample > 0) {   // a position in the interval's subset, then that subset element
    const uint64_t pos = sample_index(j.seed, j.stream, j.step, (uint32_t)s, (uint64_t)j.resample * j.batch);
    const uint4 r = philox4x32_10(make_uint4((uint32_t)(pos >> 2), (uint32_t)((j.step - 1) / j.resample),
                                             (uint32_t)j.stream, 1u),
                                  make_uint2((uint32_t)j.seed, (uint32_t)(j.seed >> 32)));
    const uint32_t u = (pos & 3) == 0 ? r.x : (pos & 3) == 1 ? r.y : (pos & 3) == 2 ? r.z : r.w;
    idx = ((uint64_t)u * npop) >> 32;
  } else {
    idx = sample_index(j.seed, j.stream, j.step, (uint32_t)s, npop);
  }
  if (j.pop) idx = ((uint64_t)j.pop[idx >> j.pop_shift] << j.pop_shift) | (idx & ((1ull << j.pop_shift) - 1));
  if (j.net == 2 && j.sampling == 1) {   // blocked: every voxel of the leaves
    const int64_t leaf = (int64_t)(idx >> 9);
    const int off = (int)(idx & 511);
    const int4 o = j.leaf_origin[leaf];
    cx = (o.x - j.ox) + (off >> 6);
    cy = (o.y - j.oy) + ((off >> 3) & 7);
    cz = (o.z - j.oz) + (off & 7);
    tgt = leaf_voxel_target(j, leaf, off);
    return;
  }
  if (j.net == 2 && j.sampling == 2) {   // dense: every voxel of the domain's bounding box
    const int e = j.log2e;
    const int x = j.gx + (int)(idx >> (2 * e)), y = j.gy + (int)((idx >> e) & ((1u << e) - 1)),
              z = j.gz + (int)(idx & ((1u << e) - 1));
    cx = x - j.ox; cy = y - j.oy; cz = z - j.oz;
    const uint64_t key = leaf_key(x, y, z);
    int64_t lo = 0, hi = j.n_leaf;   // leaves are in canonical (key) order
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      const int4 o = j.leaf_origin[mid];
      if (leaf_key(o.x, o.y, o.z) < key) lo = mid + 1; else hi = mid;
    }
    const bool found = lo < j.n_leaf && leaf_key(j.leaf_origin[lo].x, j.leaf_origin[lo].y, j.leaf_origin[lo].z) == key;
    tgt = found ? leaf_voxel_target(j, lo, ((x & 7) << 6) | ((y & 7) << 3) | (z & 7)) : j.bg_target;
    return;
  }
  if (j.net == 0) {
    const int64_t node = (int64_t)(idx >> 12);
    const int slot = (int)(idx & 4095);
    const int4 o = j.l1_origin[node];
    cx = ((o.x - j.ox) >> 3) + (slot >> 8);
    cy = ((o.y - j.oy) >> 3) + ((slot >> 4) & 15);
    cz = ((o.z - j.oz) >> 3) + (slot & 15);
    const bool child = (j.l1_mask[node * 64 + (slot >> 6)] >> (slot & 63)) & 1ull;
    if (j.l1_tile_mask) {
      const bool tile = (j.l1_tile_mask[node * 64 + (slot >> 6)] >> (slot & 63)) & 1ull;
      tgt = tile ? 1.f : child ? 0.f : 2.f;
    } else {
      tgt = child ? 1.f : 0.f;
    }
  } else if (j.net == 3) {
    const int4 o = j.leaf_origin[idx];
    cx = (o.x - j.ox) >> 3;
    cy = (o.y - j.oy) >> 3;
    cz = (o.z - j.oz) >> 3;
    tgt = j.val[j.leaf_first[idx]] * j.tscale;
  } else if (j.net == 1) {
    const int64_t leaf = (int64_t)(idx >> 9);
    const int off = (int)(idx & 511);
    const int4 o = j.leaf_origin[leaf];
    cx = (o.x - j.ox) + (off >> 6);
    cy = (o.y - j.oy) + ((off >> 3) & 7);
    cz = (o.z - j.oz) + (off & 7);
    tgt = (float)((j.leaf_mask[leaf * 8 + (off >> 6)] >> (off & 63)) & 1ull);
  } else {
    cx = j.ijk[3 * idx] - j.ox;
    cy = j.ijk[3 * idx + 1] - j.oy;
    cz = j.ijk[3 * idx + 2] - j.oz;
    tgt = j.val[idx] * j.tscale;
  }
}

// Per-row loss and dL/dy of the batch mean.
__device__ __forceinline__ void row_loss(int kind, float y, float t, float inv_b, float& l, float& g) {
  if (kind == LOSS_BCE) {
    l = fmaxf(y, 0.f) - y * t + log1pf(expf(-fabsf(y)));
    g = (1.f / (1.f + expf(-y)) - t) * inv_b;
  } else if (kind == LOSS_MSE) {
    const float d = y - t;
    l = d * d;
    g = 2.f * d * inv_b;
  } else if (kind == LOSS_L1) {
    const float d = y - t;
    l = fabsf(d);
    g = (d > 0.f ? 1.f : d < 0.f ? -1.f : 0.f) * inv_b;
  } else {   // LOSS_LINEAR
    l = y * t;
    g = t;
  }
}

template <int NIN, int W, int NOUT = 1>
struct TrainSmem {
  static constexpr int KP = NIN + 1, WP = W + 1;
  __host__ __device__ static size_t bytes(int L) {
    return ((size_t)kTile * KP + (size_t)(L + 1) * kTile * WP + NOUT * kTile + 3 * (NIN / 2) + 64) * 4;
  }
};

__device__ __forceinline__ float act_f(int act, float om, float a) { return act ? sinf(om * a) : fmaxf(a, 0.f); }

// delta * act'(a): ReLU passes delta where a > 0; sin scales it by omega cos(omega a).
__device__ __forceinline__ float act_back(int act, float om, float a, float delta) {
  return act ? delta * (om * cosf(om * a)) : (a > 0.f ? delta : 0.f);
}

// dW[o][i] += sum_r D[r][o] H[r][i] for a [W x K] layer; thread t owns column
// i = t % K and the OPT output rows starting at (t / K) * OPT.  With act >= 0 the stored
// H holds pre-activations and the layer input is act(H); act < 0: H is the input itself.
template <int K, int W>
__device__ __forceinline__ void accum_dW(const float* D, int dstride, const float* H, int hstride, float* gW, int act,
                                         float om) {
  constexpr int OB = kTile / K, OPT = W / OB;
  const int i = threadIdx.x % K, o0 = (threadIdx.x / K) * OPT;
  float acc[OPT];
#pragma unroll
  for (int k = 0; k < OPT; ++k) acc[k] = 0.f;
  for (int r = 0; r < kTile; ++r) {
    const float hv = H[r * hstride + i];
    const float h = act < 0 ? hv : act_f(act, om, hv);
#pragma unroll
    for (int k = 0; k < OPT; ++k) acc[k] = fmaf(D[r * dstride + o0 + k], h, acc[k]);
  }
#pragma unroll
  for (int k = 0; k < OPT; ++k) gW[(o0 + k) * K + i] += acc[k];
}

// Class index of a ternary target: 0, 1 or 2, else -1 (a caller's target list may hold
// anything; sampled targets are always classes).
__device__ __forceinline__ int class_of(float t) { return t == 0.f ? 0 : t == 1.f ? 1 : t == 2.f ? 2 : -1; }

// Per-row softmax cross-entropy of three logits (Section 3.3.1, the ternary level-1
// classifier) and its gradient of the batch mean; t is the class (0, 1 or 2).
__device__ __forceinline__ void row_loss3(const float* y, int t, float inv_b, float& l, float* g) {
  const float mx = fmaxf(y[0], fmaxf(y[1], y[2]));
  const float e0 = expf(y[0] - mx), e1 = expf(y[1] - mx), e2 = expf(y[2] - mx);
  const float lse = mx + logf(e0 + e1 + e2);
  l = lse - (t == 0 ? y[0] : t == 1 ? y[1] : y[2]);
  const float inv = 1.f / (e0 + e1 + e2);
  g[0] = (e0 * inv - (t == 0 ? 1.f : 0.f)) * inv_b;
  g[1] = (e1 * inv - (t == 1 ? 1.f : 0.f)) * inv_b;
  g[2] = (e2 * inv - (t == 2 ? 1.f : 0.f)) * inv_b;
}

// FP32 training step on CUDA cores: forward with the pre-activations of every hidden layer
// kept in shared memory, head and loss, backward with per-CTA gradient partials summed in a
// fixed order.  NOUT = 3: the ternary level-1 classifier's softmax cross-entropy head.
template <int NIN, int W, int NOUT = 1>
__global__ void __launch_bounds__(kTile, 1) train_fwd_bwd_kernel(NetView net, TrainJob job) {
  extern __shared__ float4 smem_t4[];
  take_step(job);
  constexpr int M = NIN / 2, KP = NIN + 1, WP = W + 1;
  const int L = net.layers;
  const int act = net.act;
  const float om = net.omega;
  float* H0 = reinterpret_cast<float*>(smem_t4);            // [128][NIN+1] encoding
  float* Hl = H0 + kTile * KP;                               // A_1..A_L (pre-activations), then delta
  float* Dl = Hl + (size_t)L * kTile * WP;
  float* gsh = Dl + kTile * WP;                              // dL/dy per output and row [NOUT][128]
  uint32_t* sq = reinterpret_cast<uint32_t*>(gsh + NOUT * kTile);
  float* red = reinterpret_cast<float*>(sq + 3 * M);         // 32 floats for the loss reduction
  const int r = threadIdx.x;
  for (int i = r; i < 3 * M; i += kTile) sq[i] = net.q[i];
  __syncthreads();
  const float* p = net.p32;
  const int64_t P = net_param_count(NIN, W, L, NOUT);
  float* gpart = job.partial + (int64_t)blockIdx.x * (P + 1);
  for (int64_t e = r; e <= P; e += kTile) gpart[e] = 0.f;
  __syncthreads();
  const float inv_b = 1.f / (float)job.batch;
  float loss_acc = 0.f;
  const int64_t ntiles = (job.batch + kTile - 1) / kTile;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t s = t * kTile + r;
    const bool valid = s < job.batch;
    int cx = 0, cy = 0, cz = 0;
    float tgt = 0.f;
    if (valid) train_sample(job, s, cx, cy, cz, tgt);
    // ---- forward, saving pre-activations
    float h[NIN > W ? NIN : W], a[W];
    encode_f32<NIN>(sq, cx, cy, cz, h);
#pragma unroll
    for (int i = 0; i < NIN; ++i) H0[r * KP + i] = h[i];
    const float* pl = p;
    for (int l = 0; l < L; ++l) {
      if (l == 0) dense_f32<NIN, W>(pl, h, a); else dense_f32<W, W>(pl, h, a);
      pl += (l == 0 ? W * NIN : W * W) + W;
      float* Hs = Hl + (size_t)l * kTile * WP + r * WP;
#pragma unroll
      for (int o = 0; o < W; ++o) { h[o] = act_f(act, om, a[o]); Hs[o] = a[o]; }
    }
    const float* wh = pl;   // W_h [NOUT][W], then b_h [NOUT]
    float y[NOUT], g[NOUT], lr_;
#pragma unroll
    for (int c = 0; c < NOUT; ++c) {
      y[c] = wh[NOUT * W + c];
#pragma unroll
      for (int i = 0; i < W; ++i) y[c] = fmaf(wh[c * W + i], h[i], y[c]);
    }
    bool use = valid;
    if constexpr (NOUT == 3) {
      const int cls = class_of(tgt);
      if (valid && cls < 0) {   // not a class: the row is left out and the call fails
        if (job.status) set_status(job.status, ST_RANGE);
        use = false;
      }
      row_loss3(y, cls < 0 ? 0 : cls, inv_b, lr_, g);
    } else {
      row_loss(job.loss, y[0], tgt, inv_b, lr_, g[0]);
    }
    if (!use) {
      lr_ = 0.f;
#pragma unroll
      for (int c = 0; c < NOUT; ++c) g[c] = 0.f;
    }
    loss_acc += lr_;
#pragma unroll
    for (int c = 0; c < NOUT; ++c) gsh[c * kTile + r] = g[c];
    // delta_L = (sum_c g_c W_h[c]) * act'(a_L)
#pragma unroll
    for (int o = 0; o < W; ++o) {
      float d = g[0] * wh[o];
#pragma unroll
      for (int c = 1; c < NOUT; ++c) d = fmaf(g[c], wh[c * W + o], d);
      Dl[r * WP + o] = act_back(act, om, a[o], d);
    }
    __syncthreads();
    // ---- head gradients
    {
      const float* HL = Hl + (size_t)(L - 1) * kTile * WP;
      float* gwh = gpart + (P - (int64_t)NOUT * (W + 1));
      if (r < W) {
        for (int c = 0; c < NOUT; ++c) {
          float acc = 0.f;
          for (int rr = 0; rr < kTile; ++rr) acc = fmaf(gsh[c * kTile + rr], act_f(act, om, HL[rr * WP + r]), acc);
          gwh[c * W + r] += acc;
        }
      } else if (r == W) {
        for (int c = 0; c < NOUT; ++c) {
          float acc = 0.f;
          for (int rr = 0; rr < kTile; ++rr) acc += gsh[c * kTile + rr];
          gwh[NOUT * W + c] += acc;
        }
      }
    }
    // ---- hidden layers, top down
    for (int l = L - 1; l >= 0; --l) {
      const int64_t woff = l == 0 ? 0 : (int64_t)W * NIN + W + (int64_t)(l - 1) * (W * W + W);
      const int K = l == 0 ? NIN : W;
      const float* Hin = l == 0 ? H0 : Hl + (size_t)(l - 1) * kTile * WP;
      const int hs = l == 0 ? KP : WP;
      if (l == 0) accum_dW<NIN, W>(Dl, WP, Hin, hs, gpart + woff, -1, om);
      else accum_dW<W, W>(Dl, WP, Hin, hs, gpart + woff, act, om);
      if (r < W) {
        float acc = 0.f;
        for (int rr = 0; rr < kTile; ++rr) acc += Dl[rr * WP + r];
        gpart[woff + (int64_t)W * K + r] += acc;
      }
      __syncthreads();
      if (l > 0) {
        // delta_l = (W_l^T delta_{l+1}) * act'(a_l), own row only
        float d[W];
#pragma unroll
        for (int o = 0; o < W; ++o) d[o] = Dl[r * WP + o];
        const float* Wl = p + woff;
        const float* Hr = Hin + r * hs;
#pragma unroll 4
        for (int i = 0; i < W; ++i) {
          float acc = 0.f;
#pragma unroll
          for (int o = 0; o < W; ++o) acc = fmaf(__ldg(Wl + o * W + i), d[o], acc);
          Dl[r * WP + i] = act_back(act, om, Hr[i], acc);
        }
        __syncthreads();
      }
    }
  }
  // deterministic loss sum of this CTA
  float v = loss_acc;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((r & 31) == 0) red[r >> 5] = v;
  __syncthreads();
  if (r == 0) {
    float sum = 0.f;
    for (int w = 0; w < kTile / 32; ++w) sum += red[w];
    gpart[P] = sum;
  }
}


// Transposed BF16 hidden-layer tiles W_l^T (l >= 1) read by the tensor-core training step's
// delta propagation.
constexpr int kTrainTcMaxLayers = 4;

static __global__ void pack_weights_t_kernel(const float* p32, uint8_t* wpk, int nin, int W, int L) {
  const int64_t te = wtile_elems(nin, W, L);
  const int64_t total = wtile_t_elems(W, L);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int l = 1 + (int)(e / ((int64_t)W * W));
    const int rr = (int)(e % ((int64_t)W * W));
    const int o = rr / W, i = rr % W;   // W_l[o][i] -> row i, column o
    const int64_t woff = (int64_t)W * nin + W + (int64_t)(l - 1) * (W * W + W);
    *reinterpret_cast<__nv_bfloat16*>(wpk + te * 6 + (int64_t)(l - 1) * W * W * 2 + canon_off(i, o, W)) =
        __float2bfloat16_rn(p32[woff + (int64_t)o * W + i]);
  }
}

// Byte offsets, inside the packed buffer, of the BF16 copies of parameter e that the
// training kernel reads: `fo` in the BF16 forward tile (layer-0 columns interleaved
// as (cos_f, sin_f)), `to` in the transposed tile (hidden-layer weights only).
// Head parameters have neither (-1).
__device__ __forceinline__ void bf16_tile_offsets(int64_t e, int nin, int W, int L, int64_t& fo, int64_t& to) {
  const int64_t te = wtile_elems(nin, W, L);
  fo = -1;
  to = -1;
  int64_t base = 0, tbase = 0;
  for (int l = 0; l < L; ++l) {
    const int K = l == 0 ? nin : W;
    const int64_t sz = (int64_t)W * K + W;
    if (e < base + sz) {
      const int64_t r = e - base;
      if (r < (int64_t)W * K) {
        const int o = (int)(r / K), j = (int)(r % K);
        const int i = l == 0 ? (j < nin / 2 ? 2 * j : 2 * (j - nin / 2) + 1) : j;
        fo = te * 2 + tbase * 2 + canon_off(o, i, K + 16);
        if (l > 0) to = te * 6 + (int64_t)(l - 1) * W * W * 2 + canon_off(j, o, W);
      } else {
        fo = te * 2 + tbase * 2 + canon_off((int)(r - (int64_t)W * K), K, K + 16);
      }
      return;
    }
    base += sz;
    tbase += (int64_t)W * (K + 16);
  }
}

// What the reduction + Adam kernel needs to know about the tensor-core training kernel:
// the BF16 tiles it reads (refreshed with every update) and the order of its partials.
struct AdamAux {
  uint8_t* wpk;               // BF16 tiles to refresh after the update (nullptr: none)
  int tc_partials;            // partials are in the tensor-core order of partial_param()
  int nin, W, L;
};

// Order of the partials of the tensor-core training kernel: layer l's block (same offset
// and size as its parameters W_l, b_l) holds column i of the TMEM weight gradient at
// i*W + o, i in the kernel's feature order (layer 0 interleaved as (cos_f, sin_f)), the
// bias at K*W + o; head and loss entries keep their places.  Returns the parameter
// index stored in slot pe.
__device__ __forceinline__ int64_t partial_param(int64_t pe, int nin, int W, int L) {
  int64_t base = 0;
  for (int l = 0; l < L; ++l) {
    const int K = l == 0 ? nin : W;
    const int64_t sz = (int64_t)W * K + W;
    if (pe < base + sz) {
      const int64_t r = pe - base;
      const int i = (int)(r / W), o = (int)(r % W);
      if (i == K) return base + (int64_t)W * K + o;
      const int j = l == 0 ? ((i & 1) ? nin / 2 + (i >> 1) : (i >> 1)) : i;
      return base + (int64_t)o * K + j;
    }
    base += sz;
  }
  return pe;
}


// Sum the per-CTA partials in a fixed order, then Adam (or just write the gradient).
// Block = 32 slots x kRedGroups warps: warp q sums the partials of CTAs
// [q n / G, (q+1) n / G) in CTA order (coalesced over the 32 slots), then the G chunk
// sums are added in q order.
constexpr int kRedGroups = 8;

// Step-dependent inputs of the Adam kernel read from device memory (graph replay): the
// step from step_dev[1], lr_t = lr * decay^floor((step - 1) / interval), the loss slot
// loss_base[step - first_step]; block 0 advances step_dev[0] for the next step.
struct AdamSched {
  int* step_dev;              // nullptr: use the launch's step, lr_t and loss_out
  float lr, decay;
  int interval;
  float* loss_base;           // loss of step t at loss_base[t - first_step]
  int first_step;
};

// Learning rate of a step: lr * decay^floor((step - 1) / interval), constant if interval = 0.
__device__ __forceinline__ float sched_lr(const AdamSched& sc, int step) {
  return sc.interval > 0 ? sc.lr * powf(sc.decay, (float)((step - 1) / sc.interval)) : sc.lr;
}

// Sum of partial slot pe over the CTAs of group q, [q n / G, (q+1) n / G), in CTA order, with
// 16 loads in flight.  L2 loads (CG): the partials of other CTAs of the same launch.
template <bool CG>
__device__ __forceinline__ float group_sum(const float* partial, int nparts, int64_t P, int64_t pe, int q) {
  const int c0 = (int)((int64_t)q * nparts / kRedGroups), c1 = (int)((int64_t)(q + 1) * nparts / kRedGroups);
  float gq = 0.f;
  for (int cb = c0; cb < c1; cb += 16) {
    float v[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const float* a = partial + (int64_t)(cb + j) * (P + 1) + pe;
      v[j] = cb + j < c1 ? (CG ? __ldcg(a) : __ldcs(a)) : 0.f;
    }
#pragma unroll
    for (int j = 0; j < 16; ++j)
      if (cb + j < c1) gq += v[j];
  }
  return gq;
}

// Adam on the parameter held in partial slot pe, gradient g (or the loss, slot P).
__device__ __forceinline__ void adam_apply(int64_t pe, float g, int64_t P, float* params, float* m, float* v, int step,
                                           float lr_t, float* grad_out, float* loss_out, float loss_scale,
                                           const AdamAux& rp) {
  const int64_t e = rp.tc_partials ? partial_param(pe, rp.nin, rp.W, rp.L) : pe;
  if (e == P) {
    if (loss_out) *loss_out = g * loss_scale;
    return;
  }
  if (grad_out) grad_out[e] = g;
  if (params) {
    const float b1 = 0.9f, b2 = 0.999f;
    const float mm = b1 * m[e] + (1.f - b1) * g;
    const float vv = b2 * v[e] + (1.f - b2) * g * g;
    m[e] = mm;
    v[e] = vv;
    const float mhat = mm / (1.f - powf(b1, (float)step));
    const float vhat = vv / (1.f - powf(b2, (float)step));
    const float w = params[e] - lr_t * mhat / (sqrtf(vhat) + 1e-8f);
    params[e] = w;
    if (rp.wpk) {
      int64_t fo, to;
      bf16_tile_offsets(e, rp.nin, rp.W, rp.L, fo, to);
      const __nv_bfloat16 b = __float2bfloat16_rn(w);
      if (fo >= 0) *reinterpret_cast<__nv_bfloat16*>(rp.wpk + fo) = b;
      if (to >= 0) *reinterpret_cast<__nv_bfloat16*>(rp.wpk + to) = b;
    }
  }
}

static __global__ void __launch_bounds__(32 * kRedGroups) adam_reduce_kernel(
    const float* partial, int nparts, int64_t P, float* params, float* m, float* v, int step, float lr_t,
    float* grad_out, float* loss_out, float loss_scale, AdamAux rp, AdamSched sc) {
  __shared__ float red[kRedGroups][33];
  if (sc.step_dev) {
    step = sc.step_dev[1];
    lr_t = sched_lr(sc, step);
    loss_out = sc.loss_base + (step - sc.first_step);
    if (blockIdx.x == 0 && threadIdx.x == 0) sc.step_dev[0] = step + 1;
  }
  const int lane = threadIdx.x & 31, q = threadIdx.x >> 5;
  // one slot per lane (coalesced over the partials), mapped to its parameter
  const int64_t pe = (int64_t)blockIdx.x * 32 + lane;
  red[q][lane] = pe <= P ? group_sum<false>(partial, nparts, P, pe, q) : 0.f;
  __syncthreads();
  if (q != 0 || pe > P) return;
  float g = 0.f;
#pragma unroll
  for (int k = 0; k < kRedGroups; ++k) g += red[k][lane];
  adam_apply(pe, g, P, params, m, v, step, lr_t, grad_out, loss_out, loss_scale, rp);
}

// The Adam update fused into the tensor-core training step (one launch per step): after a
// grid-wide barrier every CTA reduces and updates a strided share of the partial slots, with
// the arithmetic of adam_reduce_kernel (same group sums, same order, same update).
struct FusedAdam {
  uint32_t* sync;           // [2] arrival count, generation (zero-initialised); nullptr: not fused
  float *params, *m, *v;
  AdamAux rp;
  AdamSched sc;             // sc.step_dev: step, rate and loss slot from device memory
  float lr_t, loss_scale;   // without step_dev
  float* loss_out;
};

// Grid-wide barrier of a cooperative launch (every CTA resident), bounded by kWaitLimitNs:
// false on expiry.  Each CTA's earlier global writes are visible to every CTA after it.
__device__ __forceinline__ bool grid_sync_bounded(uint32_t* sync) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    uint32_t gen;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(gen) : "l"(sync + 1) : "memory");
    bool ok = true;
    if (atomicAdd(sync, 1u) == gridDim.x - 1) {
      atomicExch(sync, 0u);
      __threadfence();
      asm volatile("st.release.gpu.global.u32 [%0], %1;" :: "l"(sync + 1), "r"(gen + 1u) : "memory");
    } else {
      const uint64_t t0 = global_ns();
      for (;;) {
        uint32_t g;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(g) : "l"(sync + 1) : "memory");
        if (g != gen) break;
        if (global_ns() - t0 > kWaitLimitNs) { ok = false; break; }
      }
    }
    __threadfence();
    s_ok = ok && !__ldg(&g_fail_waits);
  }
  __syncthreads();
  return s_ok != 0;
}

// The fused tail: barrier, then the slots pe = blockIdx.x * blockDim.x + tid, step
// gridDim.x * blockDim.x.  A CTA that met a failed wait still arrives; nobody updates then.
__device__ __forceinline__ void fused_adam_tail(const FusedAdam& fa, const float* partial, int64_t P, int step,
                                                uint32_t* status) {
  const bool ok = grid_sync_bounded(fa.sync);
  uint32_t st = 0;
  if (status) asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(st) : "l"(status) : "memory");
  if (!ok) {
    if (threadIdx.x == 0 && status) set_status(status, ST_TIMEOUT);
    return;
  }
  if (st & ST_TIMEOUT) return;   // a CTA's step failed: no update
  const float lr_t = fa.sc.step_dev ? sched_lr(fa.sc, step) : fa.lr_t;
  float* loss_out = fa.sc.step_dev ? fa.sc.loss_base + (step - fa.sc.first_step) : fa.loss_out;
  for (int64_t pe = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; pe <= P; pe += (int64_t)gridDim.x * blockDim.x) {
    float g = 0.f;
    for (int q = 0; q < kRedGroups; ++q) g += group_sum<true>(partial, gridDim.x, P, pe, q);
    adam_apply(pe, g, P, fa.params, fa.m, fa.v, step, lr_t, nullptr, loss_out, fa.loss_scale, fa.rp);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && fa.sc.step_dev) fa.sc.step_dev[0] = step + 1;
}

}  // namespace nvdb
