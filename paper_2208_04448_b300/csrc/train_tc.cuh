// Tensor-core training step (Section 3.2: the networks of Section 3.3 trained with
// Adam on sampled batches, Section 3.2.1): BF16 operands on tcgen05 with FP32
// accumulation; FP32 master weights, head, loss and Adam.  BF16 rather than FP16
// because the backward deltas carry the 1/batch factor of the mean loss and
// span many binades; BF16 has FP32's exponent range.
//
// One persistent CTA per SM works through 128-sample tiles.  Row r of a tile lives in
// TMEM lane r; the four warps that share a lane quarter (warps q, q+4, ...) split each
// row's W columns into groups of 16, so a row's epilogue work is spread over W/16
// threads (W/16 x 128 threads per CTA):
//  * forward as in mlp_tc_kernel (A operand in TMEM, bias through a constant-1
//    column), each layer's BF16 input H_l also written to shared memory with
//    the samples contiguous (MN-major): the B operand of the weight gradient;
//  * head and loss in FP32 (the column groups' partial dot products summed in a fixed
//    order); one output (BCE / MSE / L1 / linear) or three (the ternary level-1
//    classifier's softmax cross-entropy); delta_{L-1} = (sum_c g_c w_h[c]) [a_{L-1} > 0];
//  * for l = L-1 .. 0:  dW_l|db_l += delta_l^T [H_l | 1]  (M = 128 output rows,
//    W of them real, N = augmented input width, K = the tile's 128 samples),
//    accumulated in TMEM across all tiles of the CTA, committed to its own mbarrier
//    so the next delta's epilogue does not wait for it;
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
  static constexpr int G = W / 16;                         // column groups per row
  static constexpr int T = kTile * G;                      // threads per CTA
  static constexpr int MF = M / G;                         // encoding frequencies per thread
  static_assert(MF % 4 == 0, "encoding split");
};

template <int NIN, int W, int NOUT>
struct TrainTcLayout {
  using C = TrainTcCfg<NIN, W>;
  static constexpr int GH = NOUT == 1 ? W + 1 : W + 3;     // row stride of the head-gradient rows
  static constexpr int NH = NOUT * (W + 1);                // head parameters
  static constexpr int NI = 4 * NH;                        // head-gradient sums: parameter x row quarter
  static_assert(NI <= 2 * (C::T - 32), "head-gradient items per thread (warp 0 takes none)");
  size_t wt_off, dt_off, h0_off, gh_off, wh_off, yp_off, smp_off, q_off, red_off, bar_off, slot_off, total;
  // H_l: [128 samples x augmented width] BF16, MN-major
  __host__ __device__ size_t hin_off(int l) const {
    return l == 0 ? h0_off : h0_off + (size_t)kTile * C::K0 * 2 + (size_t)(l - 1) * kTile * C::KH * 2;
  }
  __host__ __device__ TrainTcLayout(int L) {
    wt_off = (size_t)wtile_elems(NIN, W, L) * 2;            // forward tiles at 0
    dt_off = (wt_off + (size_t)wtile_t_elems(W, L) * 2 + 127) & ~(size_t)127;
    h0_off = dt_off + (size_t)kTile * kTile * 2;
    size_t o = hin_off(L);
    gh_off = o;                                             // per row: g h_L and g, or h_L and g_0..2
    o += (size_t)kTile * GH * 4;
    wh_off = o;                                             // w_h [NOUT][W], b_h [NOUT]
    o += (size_t)((NH + 3) & ~3) * 4;
    yp_off = o;                                             // head partials [G][NOUT][128]
    o += (size_t)C::G * NOUT * kTile * 4;
    smp_off = o;                                            // the tile's samples: (x, y, z, target bits)
    o += (size_t)kTile * 16;
    q_off = o;
    o += (size_t)C::M * 12;
    red_off = (o + 15) & ~(size_t)15;
    bar_off = red_off + (size_t)(C::T / 32) * 4;
    bar_off = (bar_off + 7) & ~(size_t)7;
    slot_off = bar_off + 16;                                // two mbarriers
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

// Store 8 packed BF16 pairs (16 columns of one row) as two 16-byte chunks of an MN-major
// operand: chunks c0 and c0 + 1 of row r.
__device__ __forceinline__ void store_mn16(uint8_t* base, int c0, int r, uint32_t lbo, const uint32_t* h) {
  *reinterpret_cast<uint4*>(base + mn_off(8 * c0, r, 128u, lbo)) = make_uint4(h[0], h[1], h[2], h[3]);
  *reinterpret_cast<uint4*>(base + mn_off(8 * c0 + 8, r, 128u, lbo)) = make_uint4(h[4], h[5], h[6], h[7]);
}

template <int NIN, int W, int NOUT>
__global__ void __launch_bounds__(TrainTcCfg<NIN, W>::T, 1) train_tc_kernel(NetView net, TrainJob job, FusedAdam fa) {
  static_assert(W == 32 || W == 64, "width");
  static_assert(NIN == 32 || NIN == 64, "encoding size");
  static_assert(NOUT == 1 || NOUT == 3, "outputs");
  take_step(job);
  using C = TrainTcCfg<NIN, W>;
  using Lay = TrainTcLayout<NIN, W, NOUT>;
  constexpr int M = C::M, G = C::G, T = C::T, MF = C::MF, GH = Lay::GH, NH = Lay::NH, NI = Lay::NI;
  extern __shared__ __align__(1024) uint8_t smem[];
  const int L = net.layers;
  const Lay lay(L);
  uint8_t* sdt = smem + lay.dt_off;
  float* sgh = reinterpret_cast<float*>(smem + lay.gh_off);
  float* swh = reinterpret_cast<float*>(smem + lay.wh_off);
  float* syp = reinterpret_cast<float*>(smem + lay.yp_off);
  int4* ssmp = reinterpret_cast<int4*>(smem + lay.smp_off);
  uint32_t* sq = reinterpret_cast<uint32_t*>(smem + lay.q_off);
  float* red = reinterpret_cast<float*>(smem + lay.red_off);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + lay.bar_off);   // staging, forward, delta
  uint64_t* bar_dw = bar + 1;                                          // weight-gradient MMAs
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + lay.slot_off);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int qw = warp & 3, cg = warp >> 2, r = qw * 32 + lane;   // lane quarter, column group, row
  const int64_t P = net_param_count(NIN, W, L, NOUT);
  float* gpart = job.partial + (int64_t)blockIdx.x * (P + 1);
  const int64_t ntiles = (job.batch + kTile - 1) / kTile;

  // ---- stage: the BF16 forward and transposed tiles by bulk copies (TMA) completing on the
  // mbarrier's first phase; head and Fourier matrix by the threads; clear delta^T; the
  // constant chunks (1, 0, ...) of every H_l, which the data never overwrites; the first
  // tile's samples
  const int64_t te = wtile_elems(NIN, W, L);
  if (tid == 0) {
    const uint32_t fb = (uint32_t)(te * 2), tb = (uint32_t)(wtile_t_elems(W, L) * 2);
    mbar_init(bar, 1);
    mbar_init(bar_dw, 1);
    mbar_arrive_expect_tx(bar, fb + tb);
    bulk_g2s(smem, net.wpk + te * 2, fb, bar);
    if (tb) bulk_g2s(smem + lay.wt_off, net.wpk + te * 6, tb, bar);
  }
  for (int i = tid; i < NH; i += T) swh[i] = __ldg(net.p32 + (P - NH) + i);
  for (int i = tid; i < 3 * M; i += T) sq[i] = __ldg(net.q + i);
  {
    uint4* z = reinterpret_cast<uint4*>(sdt);
    for (int i = tid; i < kTile * kTile * 2 / 16; i += T) z[i] = make_uint4(0u, 0u, 0u, 0u);
  }
  for (int l = 0; l < L; ++l) {
    const int K = l == 0 ? C::K0 : C::KH, n = l == 0 ? NIN : W;
    uint8_t* h = smem + lay.hin_off(l);
    for (int i = tid; i < 2 * kTile; i += T)
      *reinterpret_cast<uint4*>(h + mn_off(n + 8 * (i & 1), i >> 1, 128u, C::h_lbo(K))) =
          make_uint4((i & 1) ? 0u : 0x3F80u, 0u, 0u, 0u);
  }
  if (cg == G - 1) {
    int4 v = make_int4(0, 0, 0, 0);
    if ((int64_t)blockIdx.x < ntiles && (int64_t)blockIdx.x * kTile + r < job.batch) {
      float tg;
      train_sample(job, (int64_t)blockIdx.x * kTile + r, v.x, v.y, v.z, tg);
      v.w = __float_as_int(tg);
    }
    ssmp[r] = v;
  }
  if (warp == 0) tmem_alloc(tslot, C::TCOLS);
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  uint32_t phase = 0, phase_dw = 0;
  bool failed = !mbar_wait_bounded(bar, phase);   // the weight tiles have landed
  phase ^= 1u;
  failed = __syncthreads_or(failed) != 0;
  const uint32_t tbase = *tslot;
  const uint32_t tlane = tbase + ((uint32_t)(qw * 32) << 16);
  const float inv_b = 1.f / (float)job.batch;
  const uint32_t cst[8] = {0x3F80u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};   // BF16 1.0 then zeros
  float loss_acc = 0.f;
  // head-gradient sums of items tid - 32 and tid - 32 + (T - 32): warp 0, whose thread 0
  // issues the MMAs, takes none, nor the sample fetches (the last column group draws them)
  float gacc[2] = {0.f, 0.f};
  int ntile_done = 0;
  for (int64_t t = blockIdx.x; t < ntiles && !failed; t += gridDim.x, ++ntile_done) {
    const bool valid = t * kTile + r < job.batch;
    const int4 smp = ssmp[r];
    // ---- encoding: this thread's MF frequencies of the A operand of layer 0 (TMEM) and
    // of H_0 (shared memory), interleaved (cos_f, sin_f) as in the packed first-layer tile
    {
      uint32_t h[MF];
#pragma unroll
      for (int i = 0; i < MF; ++i) {
        const uint32_t ph = ffm_phase(sq, cg * MF + i, smp.x, smp.y, smp.z);
        float sn, cs;
        __sincosf((float)(int32_t)ph * 1.4629180792671596e-09f, &sn, &cs);   // pi / 2^31
        h[i] = cvt_bf16x2(cs, sn);
      }
      tmem_st_cols<MF>(tlane + C::A_FWD + cg * MF, h);
      if (cg == 0) tmem_st8(tlane + C::A_FWD + M, cst);
      uint8_t* h0 = smem + lay.hin_off(0);
#pragma unroll
      for (int c = 0; c < MF / 4; ++c)
        *reinterpret_cast<uint4*>(h0 + mn_off(8 * (cg * MF / 4 + c), r, 128u, C::h_lbo(C::K0))) =
            make_uint4(h[4 * c], h[4 * c + 1], h[4 * c + 2], h[4 * c + 3]);
    }
    tmem_st_wait();
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    // ---- forward: thread (row r, group cg) takes columns [16 cg, 16 cg + 16)
    uint32_t accu[16];
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
      tmem_ld16_nowait(tlane + C::D + cg * 16, accu);
      tmem_ld_wait();
      if (l < L - 1) {
        uint32_t h[8];
#pragma unroll
        for (int j = 0; j < 8; ++j)
          h[j] = cvt_bf16x2(fmaxf(__uint_as_float(accu[2 * j]), 0.f), fmaxf(__uint_as_float(accu[2 * j + 1]), 0.f));
        tmem_st8(tlane + C::A_FWD + cg * 8, h);
        if (cg == 0) tmem_st8(tlane + C::A_FWD + W / 2, cst);
        store_mn16(smem + lay.hin_off(l + 1), 2 * cg, r, C::h_lbo(C::KH), h);
        tmem_st_wait();
        fence_proxy_async_smem();
      } else {   // this group's share of the head dot products
#pragma unroll
        for (int o = 0; o < NOUT; ++o) {
          float yp = 0.f;
#pragma unroll
          for (int j = 0; j < 16; ++j) yp = fmaf(swh[o * W + cg * 16 + j], fmaxf(__uint_as_float(accu[j]), 0.f), yp);
          syp[(cg * NOUT + o) * kTile + r] = yp;
        }
      }
      tc_fence_before();
      if (__syncthreads_or(!ok)) { failed = true; break; }
    }
    if (failed) break;
    // ---- head (the groups' partials in group order), loss and dL/dy: every thread of the
    // row computes the same values; group 0 keeps the loss
    float y[NOUT], g[NOUT], lrow;
#pragma unroll
    for (int o = 0; o < NOUT; ++o) {
      y[o] = swh[NOUT * W + o];
#pragma unroll
      for (int gg = 0; gg < G; ++gg) y[o] += syp[(gg * NOUT + o) * kTile + r];
    }
    bool use = valid;
    if constexpr (NOUT == 3) {
      const int cls = class_of(__int_as_float(smp.w));
      if (valid && cls < 0) {   // not a class: the row is left out and the call fails
        if (cg == 0 && job.status) set_status(job.status, ST_RANGE);
        use = false;
      }
      row_loss3(y, cls < 0 ? 0 : cls, inv_b, lrow, g);
    } else {
      row_loss(job.loss, y[0], __int_as_float(smp.w), inv_b, lrow, g[0]);
    }
    if (!use) {
      lrow = 0.f;
#pragma unroll
      for (int o = 0; o < NOUT; ++o) g[o] = 0.f;
    }
    if (cg == 0) loss_acc += lrow;
    // ---- head-gradient rows and delta_{L-1} of this group's columns
    {
      uint32_t d[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        float dv[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int c = cg * 16 + 2 * j + e;
          const float a = __uint_as_float(accu[2 * j + e]);
          float s = g[0] * swh[c];
#pragma unroll
          for (int o = 1; o < NOUT; ++o) s = fmaf(g[o], swh[o * W + c], s);
          dv[e] = a > 0.f ? s : 0.f;
          sgh[r * GH + c] = NOUT == 1 ? g[0] * fmaxf(a, 0.f) : fmaxf(a, 0.f);
        }
        d[j] = cvt_bf16x2(dv[0], dv[1]);
      }
      if (cg == 0) {
#pragma unroll
        for (int o = 0; o < NOUT; ++o) sgh[r * GH + W + o] = g[o];
      }
      tmem_st8(tlane + C::A_DEL + cg * 8, d);
      store_mn16(sdt, 2 * cg, r, C::DT_LBO, d);
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
        if (l > 0) {   // delta first: the epilogue waits for it alone
          const uint32_t bt = smem_u32(smem + lay.wt_off) + (uint32_t)(l - 1) * W * W * 2u;
          for (int ks = 0; ks < W / 16; ++ks)
            mma_f16kind_ts(tbase + C::D, tbase + C::A_DEL + ks * 8, smem_desc(bt + ks * 256, 128, W * 16),
                           idesc_bf16_f32(kTile, W), ks > 0 ? 1u : 0u);
          mma_commit(bar);
        }
        const uint32_t a0 = smem_u32(sdt), b0 = smem_u32(smem + lay.hin_off(l));
        const uint32_t hl = C::h_lbo(K);
        const uint32_t idw = idesc_bf16_f32(kTile, K) | (1u << 15) | (1u << 16);   // A, B MN-major
        for (int ks = 0; ks < kTile / 16; ++ks)
          mma_f16kind(tbase + C::DW0 + l * C::DW_STRIDE, smem_desc(a0 + ks * 2 * C::DT_LBO, C::DT_LBO, 128u),
                      smem_desc(b0 + ks * 2 * hl, hl, 128u), idw, (ntile_done > 0 || ks > 0) ? 1u : 0u);
        mma_commit(bar_dw);
      }
      if (l == L - 1) {
        // fixed-order sums of the head-gradient rows over each row quarter, while the MMAs
        // run: item i = (quarter, output, column)
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          const int i = tid - 32 + k * (T - 32);
          if (warp > 0 && i < NI) {
            const int rq = i / NH, rem = i % NH, o = rem / (W + 1), c = rem % (W + 1);
            const float* rows = sgh + rq * 32 * GH;
            float acc = 0.f;
            if (NOUT == 1 || c == W) {
              for (int rr = 0; rr < 32; ++rr) acc += rows[rr * GH + (NOUT == 1 ? c : W + o)];
            } else {
              for (int rr = 0; rr < 32; ++rr) acc = fmaf(rows[rr * GH + W + o], rows[rr * GH + c], acc);
            }
            gacc[k] += acc;
          }
        }
        // the next tile's samples (this tile's were all read before the last barrier)
        if (cg == G - 1) {
          const int64_t sn = (t + gridDim.x) * kTile + r;
          if (t + gridDim.x < ntiles) {
            int4 v = make_int4(0, 0, 0, 0);
            if (sn < job.batch) {
              float tg;
              train_sample(job, sn, v.x, v.y, v.z, tg);
              v.w = __float_as_int(tg);
            }
            ssmp[r] = v;
          }
        }
      }
      bool ok = true;
      uint32_t d[8];
      if (l > 0) {
        ok = mbar_wait_bounded(bar, phase);
        phase ^= 1u;
        tc_fence_after();
        tmem_ld16_nowait(tlane + C::D + cg * 16, accu);
        tmem_ld_wait();
        const uint8_t* hl = smem + lay.hin_off(l);
        const uint4 h0 = *reinterpret_cast<const uint4*>(hl + mn_off(16 * cg, r, 128u, C::h_lbo(C::KH)));
        const uint4 h1 = *reinterpret_cast<const uint4*>(hl + mn_off(16 * cg + 8, r, 128u, C::h_lbo(C::KH)));
        const uint32_t hw[8] = {h0.x, h0.y, h0.z, h0.w, h1.x, h1.y, h1.z, h1.w};
#pragma unroll
        for (int j = 0; j < 8; ++j)   // BF16 bits in [1, 0x7FFF] <=> H_l > 0
          d[j] = cvt_bf16x2(((hw[j] & 0xFFFFu) - 1u) < 0x7FFFu ? __uint_as_float(accu[2 * j]) : 0.f,
                            ((hw[j] >> 16) - 1u) < 0x7FFFu ? __uint_as_float(accu[2 * j + 1]) : 0.f);
        tmem_st8(tlane + C::A_DEL + cg * 8, d);
      }
      ok = mbar_wait_bounded(bar_dw, phase_dw) && ok;   // the dW MMAs are done with delta^T and H_l
      phase_dw ^= 1u;
      if (l > 0) {
        store_mn16(sdt, 2 * cg, r, C::DT_LBO, d);
        tmem_st_wait();
        fence_proxy_async_smem();
      }
      tc_fence_before();
      if (__syncthreads_or(!ok)) { failed = true; break; }
    }
  }
  // ---- the TMEM gradient accumulators -> this CTA's partial slot, in the order of
  // partial_param(): column i of layer l's accumulator at i*W + o (coalesced over o); the
  // lane quarters that hold output rows split the 16-column chunks over their groups
  if (qw < W / 32) {
    const bool have = !failed && ntile_done > 0;
    if (have) tc_fence_after();
    const int o = qw * 32 + lane;
    for (int l = 0; l < L; ++l) {
      const int K = l == 0 ? NIN : W;
      float* gl = gpart + (l == 0 ? 0 : (int64_t)W * NIN + W + (int64_t)(l - 1) * (W * W + W));
      for (int c0 = cg * 16; c0 < K + 16; c0 += 2 * G * 16) {   // two 16-column loads in flight
        const int c1 = c0 + G * 16;
        uint32_t v[2][16];
        if (have) {
          tmem_ld16_nowait(tlane + C::DW0 + l * C::DW_STRIDE + c0, v[0]);
          if (c1 < K + 16) tmem_ld16_nowait(tlane + C::DW0 + l * C::DW_STRIDE + c1, v[1]);
          tmem_ld_wait();
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j) v[0][j] = v[1][j] = 0u;
        }
#pragma unroll
        for (int j = 0; j < 16; ++j)
          if (c0 + j <= K) gl[(int64_t)(c0 + j) * W + o] = __uint_as_float(v[0][j]);
        if (c1 < K + 16) {
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (c1 + j <= K) gl[(int64_t)(c1 + j) * W + o] = __uint_as_float(v[1][j]);
        }
      }
    }
  }
  // head gradient: the four row quarters summed in order
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 2; ++k)
    if (warp > 0 && tid - 32 + k * (T - 32) < NI) sgh[tid - 32 + k * (T - 32)] = gacc[k];
  __syncthreads();
  for (int j = tid; j < NH; j += T) {
    float v = 0.f;
#pragma unroll
    for (int rq = 0; rq < 4; ++rq) v += sgh[rq * NH + j];
    const int o = j / (W + 1), c = j % (W + 1);
    gpart[c < W ? P - NH + o * W + c : P - NOUT + o] = v;
  }
  float v = loss_acc;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (tid == 0) {
    float sum = 0.f;
    for (int w = 0; w < T / 32; ++w) sum += red[w];
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
