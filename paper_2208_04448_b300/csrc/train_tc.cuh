// Tensor-core training step (Section 3.2: the networks of Section 3.3 trained with
// Adam on sampled batches, Section 3.2.1): BF16 operands on tcgen05 with FP32
// accumulation; FP32 master weights, head, loss and Adam.  BF16 rather than FP16
// because the backward deltas carry the 1/batch factor of the mean loss and
// span many binades; BF16 has FP32's exponent range.
//
// One persistent CTA of 128 threads per SM works through 128-sample tiles:
//  * forward as in mlp_tc_kernel (A operand in TMEM, bias through a constant-1
//    column), each layer's BF16 input H_l also written to shared memory with
//    the samples contiguous (MN-major): the B operand of the weight gradient;
//  * head and loss in FP32; delta_{L-1} = g w_h [a_{L-1} > 0], g = dLoss/dy;
//  * for l = L-1 .. 0:  dW_l|db_l += delta_l^T [H_l | 1]  (M = 128 output rows,
//    W of them real, N = augmented input width, K = the tile's 128 samples),
//    accumulated in TMEM across all tiles of the CTA;
//    delta_{l-1} = (delta_l W_l) [H_l > 0]  (A = delta_l in TMEM, B = W_l^T);
//  * at the end the TMEM accumulators go, once, into the CTA's partial slot; with a
//    FusedAdam (cooperative launch) the CTAs then meet at a grid-wide barrier and each
//    sums and updates a share of the slots in CTA order (deterministic), otherwise
//    adam_reduce_kernel does that in a second launch.
#pragma once
#include "common.cuh"
#include "mlp.cuh"
#include "train.cuh"

namespace nvdb {

// Byte offset of element (mn, k) of a 16-bit MN-major no-swizzle operand: core
// matrices of 8 k-rows x 16 bytes (8 consecutive mn); MN groups of 8 at `sbo`
// bytes, K groups of 8 at `lbo` bytes.
__host__ __device__ __forceinline__ uint32_t mn_off(int mn, int k, uint32_t sbo, uint32_t lbo) {
  return (uint32_t)((mn & 7) * 2 + (k & 7) * 16) + (uint32_t)(mn >> 3) * sbo + (uint32_t)(k >> 3) * lbo;
}

template <int NIN, int W>
struct TrainTcCfg {
  static constexpr int M = NIN / 2;
  static constexpr int K0 = NIN + 16, KH = W + 16;         // augmented input widths
  static constexpr int KMAX = K0 > KH ? K0 : KH;
  // TMEM columns: D [0, W), forward A operand, delta A operand, dW accumulators
  static constexpr uint32_t D = 0, A_FWD = 64, A_DEL = 112, DW0 = 144, DW_STRIDE = KMAX;
  static constexpr uint32_t TCOLS = 512;
  static_assert(A_FWD + M + 8 <= A_DEL && A_DEL + W / 2 <= DW0, "TMEM map");
  static_assert(DW0 + kTrainTcMaxLayers * DW_STRIDE <= TCOLS, "TMEM map");
  static constexpr uint32_t DT_LBO = (kTile / 8) * 128;    // delta^T: K groups (8 samples) of 16 MN groups
  __host__ __device__ static constexpr uint32_t h_lbo(int K) { return (uint32_t)(K / 8) * 128u; }
};

template <int NIN, int W>
struct TrainTcLayout {
  using C = TrainTcCfg<NIN, W>;
  size_t wt_off, dt_off, h0_off, gh_off, wh_off, q_off, red_off, bar_off, slot_off, total;
  // H_l: [128 samples x augmented width] BF16, MN-major
  __host__ __device__ size_t hin_off(int l) const {
    return l == 0 ? h0_off : h0_off + (size_t)kTile * C::K0 * 2 + (size_t)(l - 1) * kTile * C::KH * 2;
  }
  __host__ __device__ TrainTcLayout(int L) {
    wt_off = (size_t)wtile_elems(NIN, W, L) * 2;            // forward tiles at 0
    dt_off = (wt_off + (size_t)wtile_t_elems(W, L) * 2 + 127) & ~(size_t)127;
    h0_off = dt_off + (size_t)kTile * kTile * 2;
    size_t o = hin_off(L);
    gh_off = o;
    o += (size_t)kTile * (W + 1) * 4;
    wh_off = o;
    o += (size_t)(W + 4) * 4;
    q_off = o;
    o += (size_t)C::M * 12;
    red_off = (o + 15) & ~(size_t)15;
    bar_off = red_off + 64;
    slot_off = bar_off + 8;
    total = slot_off + 8;
    // Slack after the MN-major operands: what an MMA reading them with the two
    // strides exchanged would reach stays inside the allocation.
    const size_t need_dt = dt_off + 64 * 1024, need_h = hin_off(L - 1) + 32 * 1024;
    if (total < need_dt) total = need_dt;
    if (total < need_h) total = need_h;
    // one CTA per SM (it allocates all 512 TMEM columns)
    const size_t floor_bytes = kSmemPerSmDev / 2 - 1024 + 128;
    if (total < floor_bytes) total = floor_bytes;
  }
};

template <int NIN, int W>
__global__ void __launch_bounds__(kTile, 1) train_tc_kernel(NetView net, TrainJob job, FusedAdam fa) {
  static_assert(W == 32 || W == 64, "width");
  take_step(job);
  static_assert(NIN == 32 || NIN == 64, "encoding size");
  using C = TrainTcCfg<NIN, W>;
  constexpr int M = C::M;
  extern __shared__ __align__(1024) uint8_t smem[];
  const int L = net.layers;
  const TrainTcLayout<NIN, W> lay(L);
  uint8_t* sdt = smem + lay.dt_off;
  float* sgh = reinterpret_cast<float*>(smem + lay.gh_off);
  float* swh = reinterpret_cast<float*>(smem + lay.wh_off);
  uint32_t* sq = reinterpret_cast<uint32_t*>(smem + lay.q_off);
  float* red = reinterpret_cast<float*>(smem + lay.red_off);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + lay.bar_off);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + lay.slot_off);
  const int tid = threadIdx.x, warp = tid >> 5, r = tid;
  const int64_t P = net_param_count(NIN, W, L);
  float* gpart = job.partial + (int64_t)blockIdx.x * (P + 1);

  // ---- stage: the BF16 forward and transposed tiles by bulk copies (TMA) completing on the
  // mbarrier's first phase; head and Fourier matrix by the threads; clear delta^T
  const int64_t te = wtile_elems(NIN, W, L);
  if (tid == 0) {
    const uint32_t fb = (uint32_t)(te * 2), tb = (uint32_t)(wtile_t_elems(W, L) * 2);
    mbar_init(bar, 1);
    mbar_arrive_expect_tx(bar, fb + tb);
    bulk_g2s(smem, net.wpk + te * 2, fb, bar);
    if (tb) bulk_g2s(smem + lay.wt_off, net.wpk + te * 6, tb, bar);
  }
  for (int i = tid; i <= W; i += kTile) swh[i] = __ldg(net.p32 + (P - W - 1) + i);
  for (int i = tid; i < 3 * M; i += kTile) sq[i] = __ldg(net.q + i);
  {
    uint4* z = reinterpret_cast<uint4*>(sdt);
    for (int i = tid; i < kTile * kTile * 2 / 16; i += kTile) z[i] = make_uint4(0u, 0u, 0u, 0u);
  }
  if (warp == 0) tmem_alloc(tslot, C::TCOLS);
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  uint32_t phase = 0;
  bool failed = !mbar_wait_bounded(bar, phase);   // the weight tiles have landed
  phase ^= 1u;
  failed = __syncthreads_or(failed) != 0;
  const uint32_t tbase = *tslot;
  const uint32_t tlane = tbase + ((uint32_t)(warp * 32) << 16);
  const float bh = swh[W];
  const float inv_b = 1.f / (float)job.batch;
  const uint32_t cst[8] = {0x3F80u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};   // BF16 1.0 then zeros
  float loss_acc = 0.f, gwh_acc = 0.f;   // thread c < W: dLoss/dw_h[c]; thread W: dLoss/db_h
  int ntile_done = 0;
  const int64_t ntiles = (job.batch + kTile - 1) / kTile;
  // sample of row r of tile t (coordinates and target); the next tile's is fetched while the
  // current tile's backward MMAs run, so its gathers overlap them
  int ncx = 0, ncy = 0, ncz = 0;
  float ntgt = 0.f;
  if ((int64_t)blockIdx.x < ntiles && (int64_t)blockIdx.x * kTile + r < job.batch)
    train_sample(job, (int64_t)blockIdx.x * kTile + r, ncx, ncy, ncz, ntgt);
  for (int64_t t = blockIdx.x; t < ntiles && !failed; t += gridDim.x, ++ntile_done) {
    const int64_t s = t * kTile + r;
    const bool valid = s < job.batch;
    const int cx = ncx, cy = ncy, cz = ncz;
    const float tgt = ntgt;
    // ---- encoding: A operand of layer 0 (TMEM) and H_0 (shared memory), features
    // interleaved (cos_0, sin_0, cos_1, ...) as in the packed first-layer tile
    {
      uint32_t h[M];
#pragma unroll
      for (int f = 0; f < M; ++f) {
        const uint32_t ph = ffm_phase(sq, f, cx, cy, cz);
        float sn, cs;
        __sincosf((float)(int32_t)ph * 1.4629180792671596e-09f, &sn, &cs);   // pi / 2^31
        h[f] = cvt_bf16x2(cs, sn);
      }
      tmem_st_cols<M>(tlane + C::A_FWD, h);
      tmem_st8(tlane + C::A_FWD + M, cst);
      uint8_t* h0 = smem + lay.hin_off(0);
#pragma unroll
      for (int c = 0; c < C::K0 / 8; ++c) {
        const uint4 v = c < NIN / 8 ? make_uint4(h[4 * c], h[4 * c + 1], h[4 * c + 2], h[4 * c + 3])
                                    : make_uint4(c == NIN / 8 ? 0x3F80u : 0u, 0u, 0u, 0u);
        *reinterpret_cast<uint4*>(h0 + mn_off(8 * c, r, 128u, C::h_lbo(C::K0))) = v;
      }
    }
    tmem_st_wait();
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    // ---- forward
    uint32_t accu[W];
    float y = 0.f;
    for (int l = 0; l < L; ++l) {
      const int K = l == 0 ? C::K0 : C::KH;
      if (tid == 0) {
        tc_fence_after();
        const uint32_t b0 = smem_u32(smem) + (l == 0 ? 0u : (uint32_t)(W * C::K0 + (l - 1) * W * C::KH) * 2u);
        for (int ks = 0; ks < K / 16; ++ks)
          mma_f16kind_ts(tbase + C::D, tbase + C::A_FWD + ks * 8, smem_desc(b0 + ks * 256, 128, K * 16),
                         idesc_bf16_f32(kTile, W), ks > 0 ? 1u : 0u);
        mma_commit(bar);
      }
      const bool ok = mbar_wait_bounded(bar, phase);
      phase ^= 1u;
      tc_fence_after();
      tmem_ld32_nowait(tlane + C::D, accu);
      if (W == 64) tmem_ld32_nowait(tlane + C::D + 32, accu + 32);
      tmem_ld_wait();
      if (l < L - 1) {
        uint32_t h[W / 2];
#pragma unroll
        for (int q = 0; q < W / 2; ++q)
          h[q] = cvt_bf16x2(fmaxf(__uint_as_float(accu[2 * q]), 0.f), fmaxf(__uint_as_float(accu[2 * q + 1]), 0.f));
        tmem_st_cols<W / 2>(tlane + C::A_FWD, h);
        tmem_st8(tlane + C::A_FWD + W / 2, cst);
        uint8_t* hn = smem + lay.hin_off(l + 1);
#pragma unroll
        for (int c = 0; c < C::KH / 8; ++c) {
          const uint4 v = c < W / 8 ? make_uint4(h[4 * c], h[4 * c + 1], h[4 * c + 2], h[4 * c + 3])
                                    : make_uint4(c == W / 8 ? 0x3F80u : 0u, 0u, 0u, 0u);
          *reinterpret_cast<uint4*>(hn + mn_off(8 * c, r, 128u, C::h_lbo(C::KH))) = v;
        }
        tmem_st_wait();
        fence_proxy_async_smem();
      } else {
        y = bh;
#pragma unroll
        for (int c = 0; c < W; ++c) y = fmaf(swh[c], fmaxf(__uint_as_float(accu[c]), 0.f), y);
      }
      tc_fence_before();
      if (__syncthreads_or(!ok)) { failed = true; break; }
    }
    if (failed) break;
    // ---- loss; head-gradient rows; delta_{L-1}
    float lrow, g;
    row_loss(job.loss, y, tgt, inv_b, lrow, g);
    if (!valid) { lrow = 0.f; g = 0.f; }
    loss_acc += lrow;
    {
      uint32_t d[W / 2];
#pragma unroll
      for (int q = 0; q < W / 2; ++q) {
        const float a0 = __uint_as_float(accu[2 * q]), a1 = __uint_as_float(accu[2 * q + 1]);
        sgh[r * (W + 1) + 2 * q] = g * fmaxf(a0, 0.f);
        sgh[r * (W + 1) + 2 * q + 1] = g * fmaxf(a1, 0.f);
        d[q] = cvt_bf16x2(a0 > 0.f ? g * swh[2 * q] : 0.f, a1 > 0.f ? g * swh[2 * q + 1] : 0.f);
      }
      sgh[r * (W + 1) + W] = g;
      tmem_st_cols<W / 2>(tlane + C::A_DEL, d);
#pragma unroll
      for (int c = 0; c < W / 8; ++c)
        *reinterpret_cast<uint4*>(sdt + mn_off(8 * c, r, 128u, C::DT_LBO)) = make_uint4(d[4 * c], d[4 * c + 1], d[4 * c + 2], d[4 * c + 3]);
      tmem_st_wait();
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    // ---- backward through the hidden layers
    for (int l = L - 1; l >= 0; --l) {
      const int K = l == 0 ? C::K0 : C::KH;
      if (tid == 0) {
        tc_fence_after();
        const uint32_t a0 = smem_u32(sdt), b0 = smem_u32(smem + lay.hin_off(l));
        const uint32_t hl = C::h_lbo(K);
        const uint32_t idw = idesc_bf16_f32(kTile, K) | (1u << 15) | (1u << 16);   // A, B MN-major
        for (int ks = 0; ks < kTile / 16; ++ks)
          mma_f16kind(tbase + C::DW0 + l * C::DW_STRIDE, smem_desc(a0 + ks * 2 * C::DT_LBO, C::DT_LBO, 128u),
                      smem_desc(b0 + ks * 2 * hl, hl, 128u), idw, (ntile_done > 0 || ks > 0) ? 1u : 0u);
        if (l > 0) {
          const uint32_t bt = smem_u32(smem + lay.wt_off) + (uint32_t)(l - 1) * W * W * 2u;
          for (int ks = 0; ks < W / 16; ++ks)
            mma_f16kind_ts(tbase + C::D, tbase + C::A_DEL + ks * 8, smem_desc(bt + ks * 256, 128, W * 16),
                           idesc_bf16_f32(kTile, W), ks > 0 ? 1u : 0u);
        }
        mma_commit(bar);
      }
      if (l == L - 1) {
        if (tid <= W) {   // fixed-order column sums of g h_L (and g), while the MMAs run
          float acc = 0.f;
          for (int rr = 0; rr < kTile; ++rr) acc += sgh[rr * (W + 1) + tid];
          gwh_acc += acc;
        }
        const int64_t sn = (t + gridDim.x) * kTile + r;   // the next tile's sample
        if (t + gridDim.x < ntiles && sn < job.batch) train_sample(job, sn, ncx, ncy, ncz, ntgt);
      }
      const bool ok = mbar_wait_bounded(bar, phase);
      phase ^= 1u;
      tc_fence_after();
      if (l > 0) {
        tmem_ld32_nowait(tlane + C::D, accu);
        if (W == 64) tmem_ld32_nowait(tlane + C::D + 32, accu + 32);
        tmem_ld_wait();
        const uint8_t* hl = smem + lay.hin_off(l);
        uint32_t d[W / 2];
#pragma unroll
        for (int c = 0; c < W / 8; ++c) {
          const uint4 hv = *reinterpret_cast<const uint4*>(hl + mn_off(8 * c, r, 128u, C::h_lbo(C::KH)));
          const uint32_t hw[4] = {hv.x, hv.y, hv.z, hv.w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int q = 4 * c + e;   // BF16 bits in [1, 0x7FFF] <=> H_l > 0
            d[q] = cvt_bf16x2(((hw[e] & 0xFFFFu) - 1u) < 0x7FFFu ? __uint_as_float(accu[2 * q]) : 0.f,
                              ((hw[e] >> 16) - 1u) < 0x7FFFu ? __uint_as_float(accu[2 * q + 1]) : 0.f);
          }
        }
        tmem_st_cols<W / 2>(tlane + C::A_DEL, d);
#pragma unroll
        for (int c = 0; c < W / 8; ++c)
          *reinterpret_cast<uint4*>(sdt + mn_off(8 * c, r, 128u, C::DT_LBO)) = make_uint4(d[4 * c], d[4 * c + 1], d[4 * c + 2], d[4 * c + 3]);
        tmem_st_wait();
        fence_proxy_async_smem();
      }
      tc_fence_before();
      if (__syncthreads_or(!ok)) { failed = true; break; }
    }
  }
  // ---- the TMEM gradient accumulators -> this CTA's partial slot, in the order of
  // partial_param(): column i of layer l's accumulator at i*W + o (coalesced over o)
  if (warp < W / 32) {
    const bool have = !failed && ntile_done > 0;
    if (have) tc_fence_after();
    const int o = tid;
    for (int l = 0; l < L; ++l) {
      const int K = l == 0 ? NIN : W;
      float* gl = gpart + (l == 0 ? 0 : (int64_t)W * NIN + W + (int64_t)(l - 1) * (W * W + W));
      for (int c0 = 0; c0 < K + 16; c0 += 16) {
        uint32_t v[16];
        if (have) {
          tmem_ld16_nowait(tlane + C::DW0 + l * C::DW_STRIDE + c0, v);
          tmem_ld_wait();
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j) v[j] = 0u;
        }
#pragma unroll
        for (int j = 0; j < 16; ++j)
          if (c0 + j <= K) gl[(int64_t)(c0 + j) * W + o] = __uint_as_float(v[j]);
      }
    }
  }
  if (tid < W) gpart[P - W - 1 + tid] = gwh_acc;
  else if (tid == W) gpart[P - 1] = gwh_acc;
  float v = loss_acc;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((tid & 31) == 0) red[warp] = v;
  __syncthreads();
  if (tid == 0) {
    float sum = 0.f;
    for (int w = 0; w < kTile / 32; ++w) sum += red[w];
    gpart[P] = sum;
    if (failed && job.status) set_status(job.status, ST_TIMEOUT);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tbase, C::TCOLS);
  if (fa.sync) fused_adam_tail(fa, job.partial, P, job.step, job.status);
}

}  // namespace nvdb
