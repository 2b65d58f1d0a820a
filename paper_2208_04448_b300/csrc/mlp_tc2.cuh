// Split-epilogue variant of mlp_tc_kernel (same arithmetic, same outputs): 256 threads per
// 128-row tile.  Warp w reads tensor-memory lanes 32 (w & 3) .. 32 (w & 3) + 31 (its rows)
// and handles half h = w >> 2 of the columns: half of the encoding's frequencies, half of
// every layer's accumulator columns (load, bias, ReLU, repack, store back as the next A
// operand), half of the head's dot product.  Each thread's share of the epilogue that sits
// between two layers' MMAs is halved, and so is its register footprint, so four CTAs of
// 256 threads still fit an SM (TMEM: 4 x 128 columns).
//
// The lattice modes stage the node / leaf origin of the CTA's next tile into shared memory
// with a bulk copy (cp.async.bulk, the TMA unit) one tile ahead, completing on one of two
// mbarriers; the encoding waits for it with a bounded wait.
#pragma once
#include "mlp.cuh"

namespace nvdb {

constexpr int kTc2Threads = 256;

template <int NIN, int W, int MODE>
struct Tc2Layout {
  size_t w_bytes, t_off, p_off, b_off, wh_off, q_off, y_off, org_off, bar_off, obar_off, slot_off, total;
  int ncopy;
  __host__ __device__ Tc2Layout(int L, bool wlo) {
    using C = TcCfg<NIN, W, MODE>;
    ncopy = C::WLO && wlo ? 2 : 1;
    w_bytes = MODE == TC_FP8 ? (size_t)W * C::K0 * 2 + fp8_tile_bytes(W, L) + fp8_aux_bytes(W, L)
                             : (size_t)wtile_elems(NIN, W, L) * 2;
    t_off = (ncopy * w_bytes + 15) & ~(size_t)15;
    p_off = t_off + (size_t)C::M * 64 * (C::ENC16 ? 4 : 8);
    b_off = p_off + (size_t)2 * 2 * C::M * 8;
    wh_off = b_off + (size_t)L * W * 4;
    q_off = wh_off + (size_t)(W + 4) * 4;
    y_off = (q_off + (size_t)C::M * 12 + 15) & ~(size_t)15;   // head partials of half 1 [128]
    org_off = y_off + (size_t)kTile * 4;                       // two staged origins (int4)
    bar_off = org_off + 32;
    obar_off = bar_off + 8;
    slot_off = obar_off + 16;
    total = slot_off + 8;
    const size_t floor_bytes = kSmemPerSmDev / (C::MAXC + 1) - 1024 + 128;
    if (total < floor_bytes) total = floor_bytes;
  }
};

// Index of the origin a lattice tile reads (level-1 node or leaf of its item).
__device__ __forceinline__ int64_t tile_node(int mode, int64_t t) { return mode == MODE_L1 ? (t >> 5) : (t >> 2); }

template <int NIN, int W, int MODE>
__global__ void __launch_bounds__(kTc2Threads, 4) mlp_tc2_kernel(const __grid_constant__ EvalBatch b) {
  static_assert(W == 32 || W == 64, "width");
  static_assert(NIN == 32 || NIN == 64, "encoding size");
  using C = TcCfg<NIN, W, MODE>;
  constexpr int M = C::M;
  constexpr int MH = M / 2;          // frequencies per half
  constexpr int WH = W / 2;          // accumulator columns per half
  extern __shared__ __align__(1024) uint8_t smem[];
  const int L = b.it[0].net.layers;
  const Tc2Layout<NIN, W, MODE> lay(L, batch_wlo(b));
  uint8_t* sw = smem;
  uint8_t* sw_lo = smem + lay.w_bytes;
  float2* sT = reinterpret_cast<float2*>(smem + lay.t_off);
  __half2* sTh = reinterpret_cast<__half2*>(smem + lay.t_off);
  float2* sP = reinterpret_cast<float2*>(smem + lay.p_off);
  const float* sb = reinterpret_cast<const float*>(smem + lay.b_off);
  float* swh = reinterpret_cast<float*>(smem + lay.wh_off);
  uint32_t* sq = reinterpret_cast<uint32_t*>(smem + lay.q_off);
  float* sy = reinterpret_cast<float*>(smem + lay.y_off);
  int4* sorg = reinterpret_cast<int4*>(smem + lay.org_off);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + lay.bar_off);
  uint64_t* obar = reinterpret_cast<uint64_t*>(smem + lay.obar_off);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + lay.slot_off);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int half = warp >> 2, r = ((warp & 3) << 5) | lane;   // column half, tile row

  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_init(obar, 1);
    mbar_init(obar + 1, 1);
  }
  if (warp == 0) tmem_alloc(tslot, C::COLS);
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *tslot;
  const uint32_t tlane = tbase + ((uint32_t)((warp & 3) * 32) << 16);
  const uint32_t idesc = C::ENC16 ? idesc_f16_f32(kTile, W) : idesc_bf16_f32(kTile, W);
  const uint32_t f8_tiles = (uint32_t)(W * C::K0 * 2);
  const float* f8_aux = reinterpret_cast<const float*>(smem + f8_tiles + fp8_tile_bytes(W, L));

  int64_t n0;
  const int64_t ntiles = batch_total(b, n0);
  const bool lattice = b.it[0].job.mode != MODE_LIST;   // one mode per launch (a decode stage)
  // origin of global tile g: item, local tile, pointer
  auto origin_src = [&](int64_t g) -> const int4* {
    const int mm = batch_find(b, g);
    return b.it[mm].job.nodes + tile_node(b.it[mm].job.mode, g - b.it[mm].tile_start);
  };
  // bulk copies issued to / waited for on each origin buffer (scalars: no local memory)
  uint32_t iss0 = 0u, iss1 = 0u, con0 = 0u, con1 = 0u;
  if (lattice && tid == 0 && (int64_t)blockIdx.x < ntiles) {
    mbar_arrive_expect_tx(obar, 16);
    bulk_g2s(sorg, origin_src(blockIdx.x), 16, obar);
  }
  if (lattice && (int64_t)blockIdx.x < ntiles) iss0 = 1u;

  uint32_t phase = 0;
  bool failed = false;
  int cur = -1;
  float bh = 0.f;
  bool wexact = false;
  int pbuf = 0;
  bool p_ready = false;
  const bool comp0 = comp_in<MODE>(0, L);
  int k = 0;   // tiles done by this CTA
  for (int64_t t0 = blockIdx.x; t0 < ntiles && !failed; t0 += gridDim.x, ++k) {
    const int m = batch_find(b, t0);
    if (m != cur) {
      __syncthreads();
      tc_stage<NIN, W, MODE, kTc2Threads>(b.it[m].net, b.it[m].job.mode, lay, smem);
      __syncthreads();
      bh = swh[W];
      wexact = b.it[m].net.wexact != 0;
      cur = m;
    }
    EvalJob job = b.it[m].job;
    if (b.n == 1) job.n_items = n0;
    const int64_t t = t0 - b.it[m].tile_start;
    const int64_t end_m = m + 1 < b.n ? b.it[m + 1].tile_start : ntiles;
    const bool has_next = t0 + gridDim.x < ntiles;
    const bool next_same = job.mode == MODE_L0 && t0 + gridDim.x < end_m;
    const int64_t tn = t0 + gridDim.x - b.it[m].tile_start;
    const int cb = k & 1, nb = cb ^ 1;    // origin buffers of this tile and the next
    // the next tile's origin, one tile ahead (its buffer was read during the previous tile)
    if (lattice && has_next) {
      if (tid == 0) {
        mbar_arrive_expect_tx(obar + nb, 16);
        bulk_g2s(sorg + nb, origin_src(t0 + gridDim.x), 16, obar + nb);
      }
      if (nb) ++iss1; else ++iss0;
    }
    float2* sPc = sP + pbuf * 2 * M;
    bool ok_enc = true;
    bool valid = true;
    {
      uint32_t hi[MH], lo[MH];
      if (job.mode == MODE_L0) {
        if (!p_ready) {
          if (tid < 2 * M) {
            ok_enc = mbar_wait_bounded(obar + cb, (cb ? con1 : con0) & 1u);
            l0_factors<M, MODE>(job, sq, sorg[cb], t, sPc, tid);
          }
          __syncthreads();
        }
        const int j = r & 63;
        if (C::ENC16) {
          const uint4* P4 = reinterpret_cast<const uint4*>(sPc) + (r >> 6) * (M / 2);
          const uint4* T4 = reinterpret_cast<const uint4*>(sTh);
#pragma unroll
          for (int g = 0; g < MH / 4; ++g) {
            const int f4 = half * (MH / 4) + g;
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
              hi[4 * g + e] = *reinterpret_cast<const uint32_t*>(&z);
              lo[4 * g + e] = 0u;
            }
          }
        } else {
          const float4* P4 = reinterpret_cast<const float4*>(sPc) + (r >> 6) * (M / 2);
          const float4* T4 = reinterpret_cast<const float4*>(sT);
#pragma unroll
          for (int g = 0; g < MH / 2; ++g) {
            const int f2 = half * (MH / 2) + g;
            const float4 tq = T4[f2 * 64 + j], pq = P4[f2];
            split_pair<MODE>(fmaf(pq.x, tq.x, -pq.y * tq.y), fmaf(pq.x, tq.y, pq.y * tq.x), hi[2 * g], lo[2 * g]);
            split_pair<MODE>(fmaf(pq.z, tq.z, -pq.w * tq.w), fmaf(pq.z, tq.w, pq.w * tq.z), hi[2 * g + 1], lo[2 * g + 1]);
          }
        }
      } else {
        int cx, cy, cz;
        if (job.mode == MODE_L1) {   // the staged origin of this tile's level-1 node
          ok_enc = mbar_wait_bounded(obar + cb, (cb ? con1 : con0) & 1u);
          const int4 o = sorg[cb];
          const int sl = ((int)(t & 31) << 7) | r;
          cx = ((o.x - job.ox) >> 3) + (sl >> 8);
          cy = ((o.y - job.oy) >> 3) + ((sl >> 4) & 15);
          cz = ((o.z - job.oz) >> 3) + (sl & 15);
        } else {
          valid = job_coord(job, t, r, cx, cy, cz);
        }
#pragma unroll
        for (int g = 0; g < MH; ++g) {
          const uint32_t ph = ffm_phase(sq, half * MH + g, cx, cy, cz);
          float sn, cs;
          __sincosf((float)(int32_t)ph * 1.4629180792671596e-09f, &sn, &cs);   // pi / 2^31
          split_pair<MODE>(cs, sn, hi[g], lo[g]);
        }
      }
      tmem_st_cols<MH>(tlane + C::A_HI + half * MH, hi);
      if (comp0) tmem_st_cols<MH>(tlane + C::A_LO + half * MH, lo);
      if (C::BIAS_MMA && half == 1) store_bias_chunk<NIN>(tlane);
    }
    if (lattice && (job.mode == MODE_L1 || !p_ready)) {
      if (cb) ++con1; else ++con0;
    }
    tmem_st_wait();
    tc_fence_before();
    if (__syncthreads_or(!ok_enc)) { failed = true; break; }
    float ypart = 0.f;
    for (int l = 0; l < L; ++l) {
      const int K = l == 0 ? NIN : W;
      if (tid == 0 && MODE == TC_FP8 && l > 0) {
        tc_fence_after();
        const uint32_t b0 = smem_u32(sw) + f8_tiles + (uint32_t)((l - 1) * W * W);
        for (int ks = 0; ks < W / 32; ++ks)
          mma_f8kind_ts(tbase, tbase + C::A_HI + ks * 8, smem_desc(b0 + ks * 256, 128, W * 8), idesc, ks > 0 ? 1u : 0u);
        mma_commit(bar);
      } else if (tid == 0) {
        tc_fence_after();
        const uint32_t woff = l == 0 ? 0u : (uint32_t)(W * C::K0 + (l - 1) * W * C::KH) * 2u;
        const uint32_t b0 = smem_u32(sw) + woff, bl = smem_u32(sw_lo) + woff;
        const uint32_t sbo = (uint32_t)(K + 16) * 16u;
        const bool comp = comp_in<MODE>(l, L);
        for (int ks = 0; ks < K / 16 + (C::BIAS_MMA ? 1 : 0); ++ks) {
          const uint64_t bd = smem_desc(b0 + ks * 256, 128, sbo);
          mma_f16kind_ts(tbase, tbase + C::A_HI + ks * 8, bd, idesc, ks > 0 ? 1u : 0u);
          if (C::WLO) {
            if (comp) mma_f16kind_ts(tbase, tbase + C::A_LO + ks * 8, bd, idesc, 1u);
            if (!wexact)
              mma_f16kind_ts(tbase, tbase + C::A_HI + ks * 8, smem_desc(bl + ks * 256, 128, sbo), idesc, 1u);
          }
        }
        mma_commit(bar);
      }
      bool ok = true;
      if (l == 0 && next_same && tid < 2 * M) {   // the next tile's factors from its staged origin
        ok = mbar_wait_bounded(obar + nb, (nb ? con1 : con0) & 1u);
        l0_factors<M, MODE>(job, sq, sorg[nb], tn, sP + (pbuf ^ 1) * 2 * M, tid);
      }
      if (l == 0 && next_same) {
        if (nb) ++con1; else ++con0;
      }
      ok = mbar_wait_bounded(bar, phase) && ok;
      phase ^= 1u;
      tc_fence_after();
      uint32_t accu[WH];
      if (WH == 32) tmem_ld32_nowait(tlane + half * WH, accu);
      else tmem_ld16_nowait(tlane + half * WH, accu);
      tmem_ld_wait();
      if (MODE == TC_FP8) {
        const float al = f8_aux[l];
        const float2* be = reinterpret_cast<const float2*>(f8_aux + kMaxLayers + l * W + half * WH);
#pragma unroll
        for (int c = 0; c < WH / 2; ++c) {
          const float2 h = ffma2(make_float2(al, al), make_float2(__uint_as_float(accu[2 * c]), __uint_as_float(accu[2 * c + 1])),
                                 be[c]);
          accu[2 * c] = __float_as_uint(h.x);
          accu[2 * c + 1] = __float_as_uint(h.y);
        }
      } else if (!C::BIAS_MMA) {
        const float2* bl2 = reinterpret_cast<const float2*>(sb + l * W + half * WH);
#pragma unroll
        for (int c = 0; c < WH / 2; ++c) {   // 1 * D + b: one rounding, as an add
          const float2 h = ffma2(make_float2(1.f, 1.f), make_float2(__uint_as_float(accu[2 * c]), __uint_as_float(accu[2 * c + 1])),
                                 bl2[c]);
          accu[2 * c] = __float_as_uint(h.x);
          accu[2 * c + 1] = __float_as_uint(h.y);
        }
      }
      if (MODE == TC_FP8 && l < L - 1) {
        uint32_t q[WH / 4];
#pragma unroll
        for (int c = 0; c < WH / 4; ++c)
          q[c] = cvt_relu_e4m3x2(__uint_as_float(accu[4 * c]), __uint_as_float(accu[4 * c + 1])) |
                 (cvt_relu_e4m3x2(__uint_as_float(accu[4 * c + 2]), __uint_as_float(accu[4 * c + 3])) << 16);
        tmem_st_cols<WH / 4>(tlane + C::A_HI + half * (WH / 4), q);
        tmem_st_wait();
      } else if (l < L - 1) {
        const bool comp = comp_in<MODE>(l + 1, L);
        uint32_t hi[WH / 2], lo[WH / 2];
#pragma unroll
        for (int p = 0; p < WH / 2; ++p)
          relu_pair<MODE>(__uint_as_float(accu[2 * p]), __uint_as_float(accu[2 * p + 1]), comp, hi[p], lo[p]);
        tmem_st_cols<WH / 2>(tlane + C::A_HI + half * (WH / 2), hi);
        if (comp) tmem_st_cols<WH / 2>(tlane + C::A_LO + half * (WH / 2), lo);
        if (C::BIAS_MMA && NIN != W && half == 1) store_bias_chunk<W>(tlane);
        tmem_st_wait();
      } else {
        const float4* swh4 = reinterpret_cast<const float4*>(swh + half * WH);
        float2 acc[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
#pragma unroll
        for (int c = 0; c < WH / 4; ++c) {
          const float4 wv = swh4[c];
          acc[0] = ffma2(make_float2(wv.x, wv.y),
                         make_float2(fmaxf(__uint_as_float(accu[4 * c]), 0.f), fmaxf(__uint_as_float(accu[4 * c + 1]), 0.f)), acc[0]);
          acc[1] = ffma2(make_float2(wv.z, wv.w),
                         make_float2(fmaxf(__uint_as_float(accu[4 * c + 2]), 0.f), fmaxf(__uint_as_float(accu[4 * c + 3]), 0.f)), acc[1]);
        }
        ypart = (acc[0].x + acc[0].y) + (acc[1].x + acc[1].y);
        if (half == 1) sy[r] = ypart;
      }
      tc_fence_before();
      if (__syncthreads_or(!ok)) { failed = true; break; }
    }
    if (failed) break;
    if (half == 0) job_output(job, t, r, valid, bh + (ypart + sy[r]));
    if (next_same) pbuf ^= 1;
    p_ready = next_same;
  }
  // copies still in flight (a timed-out tile, or the last prefetch): wait for them, bounded,
  // before the shared memory they write is released
  if (tid == 0 && lattice) {
    for (; con0 < iss0 && !failed; ++con0) failed = !mbar_wait_bounded(obar, con0 & 1u);
    for (; con1 < iss1 && !failed; ++con1) failed = !mbar_wait_bounded(obar + 1, con1 & 1u);
  }
  if (failed && tid == 0) set_status(b.it[0].job.status, ST_TIMEOUT);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tbase, C::COLS);
}

}  // namespace nvdb
