// libnvdb: C ABI of the NeuralVDB hot path on B300 (sm_103a).  Host-side
// orchestration of the kernels in build.cuh (tree build), mlp.cuh (fused
// encode + MLP, FP32 and BF16 tcgen05), compact.cuh (threshold / patch /
// compaction), train.cuh (backward + Adam) and query.cuh (random access).
#include "nvdb.h"

#include <algorithm>
#include <atomic>
#include <map>
#include <memory>
#include <mutex>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "build.cuh"
#include "common.cuh"
#include "runtime.cuh"
#include "compact.cuh"
#include "mlp.cuh"
#include "query.cuh"
#include "render.cuh"
#include "sample.cuh"
#include "tiles.cuh"
#include "train.cuh"

using namespace nvdb;

namespace {
// ============================================================================ scan helper
struct Scan {
  int64_t* sums = nullptr;
  int64_t cap = 0;
  int64_t* total = nullptr;   // one device int64
  ~Scan() { dfree(sums); dfree(total); }
  nvdb_status reserve(int64_t n) {
    const int64_t nb = (n + kScanBlock - 1) / kScanBlock + 1;
    if (!total) TRY(dalloc(&total, 1));
    if (nb <= cap) return NVDB_OK;
    dfree(sums);
    TRY(dalloc(&sums, (size_t)nb));
    cap = nb;
    return NVDB_OK;
  }
  // out[i] = sum_{j<i} in[j]; *total = sum of all.
  nvdb_status run(const uint32_t* in, int64_t n, int64_t* out, cudaStream_t s) {
    TRY(reserve(n));
    if (n == 0) {
      CU(cudaMemsetAsync(total, 0, sizeof(int64_t), s));
      return NVDB_OK;
    }
    const int64_t nb = (n + kScanBlock - 1) / kScanBlock;
    KLAUNCH("scan_blocks", s, scan_blocks_kernel<<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, out, sums));
    KLAUNCH("scan_sums", s, scan_sums_kernel<<<1, 1024, 0, s>>>(sums, nb, total));
    KLAUNCH("scan_add", s, scan_add_kernel<<<blocks_for(n, 256), 256, 0, s>>>(out, n, sums));
    CU(cudaGetLastError());
    return NVDB_OK;
  }
};

__global__ void offsets_to_u32_kernel(const int64_t* off, const int64_t* total, int64_t n, uint32_t* out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) out[t] = (uint32_t)off[t];
  if (t == n) out[n] = (uint32_t)*total;
}

// ============================================================================ host init (SplitMix64)
constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ull;
constexpr uint64_t kNetStream = 0x632BE59BD9B4E019ull;
constexpr uint64_t kFfmStream = 0x8CB92BA72F3D8DD7ull;

uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
// Draw i of the SplitMix64 stream started at state s (Steele, Lea & Flood 2014).
double uniform01(uint64_t s, uint64_t i) { return (double)(mix64(s + (i + 1) * kGolden) >> 11) * (1.0 / 9007199254740992.0); }

// Xavier-uniform weights, zero biases; draw order W_0 (row-major), ..., W_{L-1}, then the
// head W_h [nout][w] row-major (bound sqrt(6 / (w + nout))).
std::vector<float> xavier_params(uint64_t seed, int net, int nin, int w, int L, int nout = 1) {
  const uint64_t s = seed + kNetStream * (uint64_t)(net + 1);
  std::vector<float> p((size_t)net_param_count(nin, w, L, nout), 0.f);
  uint64_t i = 0;
  size_t o = 0;
  for (int l = 0; l < L; ++l) {
    const int fan = l == 0 ? nin : w;
    const double a = std::sqrt(6.0 / (double)(fan + w));
    for (int r = 0; r < w; ++r)
      for (int c = 0; c < fan; ++c) p[o++] = (float)((2.0 * uniform01(s, i++) - 1.0) * a);
    o += w;   // bias = 0
  }
  const double a = std::sqrt(6.0 / (double)(w + nout));
  for (int c = 0; c < nout * w; ++c) p[o++] = (float)((2.0 * uniform01(s, i++) - 1.0) * a);
  return p;   // b_h = 0
}

// Fixed-point Fourier matrix q = rint(2^32 B / E) mod 2^32, B = sigma * N(0,1) (Box-Muller).
std::vector<uint32_t> ffm_increments(uint64_t seed, int level, int m, double sigma, double extent) {
  const uint64_t s = seed + kFfmStream * (uint64_t)(level + 1);
  std::vector<uint32_t> q((size_t)m * 3);
  for (int f = 0; f < m; ++f)
    for (int d = 0; d < 3; ++d) {
      const uint64_t i = (uint64_t)(3 * f + d);
      const double u1 = uniform01(s, 2 * i), u2 = uniform01(s, 2 * i + 1);
      const double z = std::sqrt(-2.0 * std::log(1.0 - u1)) * std::cos(2.0 * M_PI * u2);
      const double t = std::ldexp(sigma * z, 32) / extent;
      q[(size_t)3 * f + d] = (uint32_t)(int64_t)std::rint(t);
    }
  return q;
}
}  // namespace

// ============================================================================ handles
struct nvdb_grid {
  int grid_class = 0;
  float half_width = 0.f, background = 0.f;
  int64_t n = 0, n_leaf = 0, n_l1 = 0, n_l2 = 0;
  int32_t origin[3] = {0, 0, 0};
  int log2e = 7;
  int32_t* ijk = nullptr;
  float* val = nullptr;
  int4* leaf_origin = nullptr;
  int64_t* leaf_first = nullptr;
  unsigned long long* leaf_mask = nullptr;
  int4* l1_origin = nullptr;
  unsigned long long* l1_mask = nullptr;
  int4* l2_origin = nullptr;
  unsigned long long* l2_mask = nullptr;
  // active tiles of level 1 (tile pruning): per leaf 1 if it is a tile (kept expanded, its
  // voxels carrying the tile value), per level-1 node the active mask a_1
  int64_t n_tiles = 0;
  uint8_t* leaf_tile = nullptr;
  unsigned long long* l1_tile_mask = nullptr;
  // random-access structures of the explicit tree (built on first use by the samplers)
  uint64_t* l2_key = nullptr;
  uint32_t *l2_pre = nullptr, *l1_pre = nullptr;
  int64_t *l2_base = nullptr, *l1_base = nullptr;
  ~nvdb_grid() {
    dfree(ijk); dfree(val); dfree(leaf_origin); dfree(leaf_first); dfree(leaf_mask);
    dfree(l1_origin); dfree(l1_mask); dfree(l2_origin); dfree(l2_mask);
    dfree(leaf_tile); dfree(l1_tile_mask);
    dfree(l2_key); dfree(l2_pre); dfree(l1_pre); dfree(l2_base); dfree(l1_base);
  }
};

namespace {
struct DevNet {
  int n_in = 0, width = 0, layers = 0, n_out = 1;
  int64_t P = 0;
  float* p32 = nullptr;
  uint8_t* wpk = nullptr;   // [FP16 | BF16 hi | BF16 lo] weight tiles, then BF16 W_l^T tiles
  float* m = nullptr;
  float* v = nullptr;
  float* master = nullptr;  // BF16 training: the FP32 master weights before the final rounding
  bool bf16_exact = false;  // every weight and bias (not the head) is a BF16 value
  uint32_t* f8_amax = nullptr;  // calibrated activation ranges (float bits) per layer, FP8 scales
  ~DevNet() { dfree(p32); dfree(wpk); dfree(m); dfree(v); dfree(master); dfree(f8_amax); }
};

// Patch lists of one precision (Section 3.3.2), on the device only: CSR offsets per
// level-1 node / leaf and 16-bit candidate indices; n1, n0 = number of patches.
struct PatchSet {
  int prec = 0;
  int64_t n1 = 0, n0 = 0;
  uint32_t* d_l1_off = nullptr;
  uint32_t* d_l0_off = nullptr;
  uint16_t* d_l1_idx = nullptr;
  uint16_t* d_l0_idx = nullptr;
  void release() { dfree(d_l1_off); dfree(d_l0_off); dfree(d_l1_idx); dfree(d_l0_idx); }
};

// Device scratch of a top-down decode of one model or of several models whose
// levels are concatenated in model order.
struct DecodeScratch {
  int64_t cap2 = 0, cap1 = 0, capl = 0;
  int64_t* l2_off = nullptr;
  int4* l1_origin = nullptr;
  uint32_t* l1_words = nullptr;
  int64_t* l1_off = nullptr;
  int4* leaf_origin = nullptr;
  uint32_t* leaf_words = nullptr;
  int64_t* leaf_off = nullptr;
  // One zero-initialised block, cleared by a single memset per decode: word 0 holds the
  // status, then the single-pass scan states of level 2, level 1, level 0 and the level-1
  // tiles (one word per scan block plus the block counter).
  uint64_t* lb = nullptr;
  uint32_t* status = nullptr;
  // ternary level 1 (models with active tiles): tile words, their scan, the tiles' origins
  // and regressed values (concatenated per model, canonical order)
  int64_t capt = 0;
  uint32_t* t1_words = nullptr;
  int64_t* t1_off = nullptr;
  int32_t* tile_ijk = nullptr;
  float* tval = nullptr;
  static int64_t blocks1(int64_t n) { return (n + kScanItemsL1 - 1) / kScanItemsL1; }
  static int64_t blocks0(int64_t n) { return (n + kScanItemsL0 - 1) / kScanItemsL0; }
  static int64_t lb_words(int64_t n2, int64_t n1, int64_t nl) {
    return 1 + (n2 + 1) + 2 * (blocks1(n1) + 1) + (blocks0(nl) + 1);
  }
  uint64_t* lb2() { return lb + 1; }
  uint64_t* lb1() { return lb + 2 + cap2; }
  uint64_t* lb0() { return lb + 3 + cap2 + blocks1(cap1); }
  uint64_t* lbt() { return lb + 4 + cap2 + blocks1(cap1) + blocks0(capl); }
  nvdb_status reserve(int64_t n2, int64_t n1, int64_t nl) {
    if (lb && n2 <= cap2 && n1 <= cap1 && nl <= capl) return NVDB_OK;
    release();
    TRY(dalloc(&lb, (size_t)lb_words(n2, n1, nl)));
    status = reinterpret_cast<uint32_t*>(lb);
    TRY(dalloc(&l2_off, n2 + 1));
    TRY(dalloc(&l1_origin, n1 + 1)); TRY(dalloc(&l1_words, 128 * n1 + 4));
    TRY(dalloc(&l1_off, n1 + 1));
    TRY(dalloc(&leaf_origin, nl + 1)); TRY(dalloc(&leaf_words, 16 * nl + 4));
    TRY(dalloc(&leaf_off, nl + 1));
    cap2 = n2; cap1 = n1; capl = nl;
    return NVDB_OK;
  }
  // after reserve(): the tile arrays for n1 level-1 nodes and nt tiles
  nvdb_status reserve_tiles(int64_t nt) {
    if (t1_words && nt <= capt) return NVDB_OK;
    dfree(t1_words); dfree(t1_off); dfree(tile_ijk); dfree(tval);
    capt = 0;
    TRY(dalloc(&t1_words, 128 * cap1 + 4)); TRY(dalloc(&t1_off, cap1 + 1));
    TRY(dalloc(&tile_ijk, 3 * nt + 3)); TRY(dalloc(&tval, nt + 1));
    capt = nt;
    return NVDB_OK;
  }
  void release() {
    dfree(l2_off); dfree(l1_origin); dfree(l1_words); dfree(l1_off);
    dfree(leaf_origin); dfree(leaf_words); dfree(leaf_off); dfree(lb);
    dfree(t1_words); dfree(t1_off); dfree(tile_ijk); dfree(tval);
    status = nullptr;
    cap2 = cap1 = capl = capt = 0;
  }
  ~DecodeScratch() { release(); }
};

// Topology cache of [Hash,5,4,NN(3)] plus the per-batch query scratch.
struct QueryCache {
  bool ready = false;
  uint64_t* l2_key = nullptr;
  uint32_t* l2_pre = nullptr;
  uint32_t* l1_pre = nullptr;
  int64_t batch = 0;
  uint8_t* qmask = nullptr;
  uint32_t* counts = nullptr;
  int64_t* off = nullptr;
  int32_t* list = nullptr;
  float* vals = nullptr;
  uint8_t* qtile = nullptr;   // models with tiles: tile corners and their values
  float* qtv = nullptr;
  void release() {
    dfree(l2_key); dfree(l2_pre); dfree(l1_pre);
    dfree(qmask); dfree(counts); dfree(off); dfree(list); dfree(vals); dfree(qtile); dfree(qtv);
    ready = false;
    batch = 0;
  }
};
}  // namespace

struct nvdb_model {
  int grid_class = 0;
  float background = 0.f, half_width = 0.f;
  int32_t origin[3] = {0, 0, 0};
  int log2e = 7;
  int ffm[2] = {32, 32};
  int width[3] = {32, 32, 32}, layers[3] = {3, 3, 3};
  int64_t n_l2 = 0, n_l1 = 0, n_leaf = 0, n_active = 0;
  std::vector<uint32_t> q_host[2];
  uint32_t* q_dev[2] = {nullptr, nullptr};
  // Networks: expert e's network j (0 level-1 classifier, 1 level-0 classifier, 2 regressor)
  // is net[3e + j]; one expert unless the domain is decomposed (Section 3.4).  With active
  // tiles (a pruned source grid, one expert), net 0 is the ternary level-1 classifier and
  // net 3 the tile value regressor on the level-1 encoding (Section 3.3.1).
  int n_exp = 1;
  bool ternary = false;
  int tile_width = 0, tile_layers = 0;
  int64_t n_tiles = 0;
  int act = 0;              // hidden activation of every network: 0 ReLU, 1 sin(omega a)
  float omega = 1.f;
  std::unique_ptr<DevNet[]> net{new DevNet[3]};
  std::vector<std::vector<float>> losses = std::vector<std::vector<float>>(3);
  // Sparse domain decomposition: subdomain size (0 = none) and halo in voxels, grid of
  // dims^3 subdomains from the domain origin, expert of each (-1 discarded), expert origins
  // relative to the domain origin; per level, the experts' network views (device).
  int sub_size = 0, sub_halo = 0, sub_dims = 0;
  std::vector<int32_t> expert_of_host, exp_origin_host;
  int* expert_of = nullptr;
  int4* exp_origin = nullptr;
  NetView* exp_views[3] = {nullptr, nullptr, nullptr};
  std::vector<int32_t> l2_origin_host;
  std::vector<uint64_t> l2_mask_host;
  int4* l2_origin = nullptr;
  unsigned long long* l2_mask = nullptr;
  std::vector<PatchSet> patches;
  uint32_t* status = nullptr;
  DecodeScratch ds;
  QueryCache qc;
  Scan scan;
  float* partial = nullptr;
  int64_t partial_cap = 0;
  ~nvdb_model() {
    dfree(q_dev[0]); dfree(q_dev[1]); dfree(l2_origin); dfree(l2_mask); dfree(status); dfree(partial);
    dfree(expert_of); dfree(exp_origin);
    for (auto& v : exp_views) dfree(v);
    for (auto& p : patches) p.release();
    qc.release();
  }
  bool moe() const { return sub_size > 0; }
  int n_net() const { return 3 * n_exp + (ternary ? 1 : 0); }
  void set_experts(int n) {
    n_exp = n;
    net.reset(new DevNet[n_net()]);
    losses.assign(n_net(), {});
  }
  void set_ternary(bool t) {   // before the networks are allocated
    ternary = t;
    set_experts(n_exp);
  }
  bool tile_net(int k) const { return ternary && k == 3 * n_exp; }
  int net_level(int k) const { return k % 3 == 0 || tile_net(k) ? 1 : 0; }   // 1: level-1 encoding
  const PatchSet* patch_set(int prec) const {
    for (auto& p : patches)
      if (p.prec == prec) return &p;
    return nullptr;
  }
  float value_scale() const { return grid_class == 0 ? half_width : 1.f; }
};

// ============================================================================ kernel dispatch
namespace {
bool supported_shape(int nin, int w) { return (nin == 32 || nin == 64) && (w == 32 || w == 64); }

// View of network k (expert k / 3, level k % 3; or the tile value regressor).
NetView net_view(const nvdb_model* m, int k) {
  NetView v;
  v.n_in = m->net[k].n_in;
  v.width = m->net[k].width;
  v.layers = m->net[k].layers;
  v.n_out = m->net[k].n_out;
  v.act = m->act;
  v.omega = m->omega;
  v.p32 = m->net[k].p32;
  v.wpk = m->net[k].wpk;
  v.q = m->q_dev[m->net_level(k) ? 0 : 1];
  v.wexact = m->net[k].bf16_exact ? 1 : 0;
  return v;
}

// Level j's view for a decode item: the decomposition's experts when there is one (the
// item's NetView then carries expert 0's shape and the experts' common wexact flag).
MoeView moe_view(const nvdb_model* m, int j) {
  MoeView v{};
  if (!m->moe()) return v;
  v.experts = m->exp_views[j];
  v.expert_of = m->expert_of;
  v.origin = m->exp_origin;
  v.n_exp = m->n_exp;
  v.dims = m->sub_dims;
  v.size = m->sub_size;
  v.halo = m->sub_halo;
  return v;
}

// Device copies of the experts' views (after the networks' buffers or flags change).
nvdb_status upload_views(nvdb_model* m, cudaStream_t s) {
  if (!m->moe()) return NVDB_OK;
  for (int j = 0; j < 3; ++j) {
    std::vector<NetView> h(m->n_exp);
    for (int e = 0; e < m->n_exp; ++e) h[e] = net_view(m, 3 * e + j);
    if (!m->exp_views[j]) TRY(dalloc(&m->exp_views[j], (size_t)m->n_exp));
    CU(cudaMemcpyAsync(m->exp_views[j], h.data(), h.size() * sizeof(NetView), cudaMemcpyHostToDevice, s));
    CU(cudaStreamSynchronize(s));   // h is a stack vector
  }
  return NVDB_OK;
}

// Geometry of a decomposition on the device (grid and origins from the host copies).
nvdb_status upload_moe(nvdb_model* m, cudaStream_t s) {
  if (!m->moe()) return NVDB_OK;
  dfree(m->expert_of);
  dfree(m->exp_origin);
  TRY(dalloc(&m->expert_of, m->expert_of_host.size()));
  TRY(dalloc(&m->exp_origin, (size_t)m->n_exp));
  std::vector<int4> o(m->n_exp);
  for (int e = 0; e < m->n_exp; ++e)
    o[e] = make_int4(m->exp_origin_host[3 * e], m->exp_origin_host[3 * e + 1], m->exp_origin_host[3 * e + 2], 0);
  CU(cudaMemcpyAsync(m->expert_of, m->expert_of_host.data(), m->expert_of_host.size() * 4, cudaMemcpyHostToDevice, s));
  CU(cudaMemcpyAsync(m->exp_origin, o.data(), o.size() * sizeof(int4), cudaMemcpyHostToDevice, s));
  CU(cudaStreamSynchronize(s));
  return NVDB_OK;
}

// Precisions are 0 .. kNumPrecisions-1.
constexpr int kNumPrecisions = 5;
bool eval_prec_ok(int prec) {
  return prec == NVDB_FP32 || prec == NVDB_BF16 || prec == NVDB_FP16 || prec == NVDB_BF16X3 || prec == NVDB_FP8_E4M3;
}

nvdb_status launch_eval_prec(const EvalBatch& b, int64_t ntiles, nvdb_precision prec, cudaStream_t s) {
  switch (prec) {
    case NVDB_FP32: return launch_eval_f32(b, ntiles, s);
    case NVDB_BF16: return launch_eval_bf16(b, ntiles, s);
    case NVDB_BF16X3: return launch_eval_bf16x3(b, ntiles, s);
    case NVDB_FP16: return launch_eval_f16(b, ntiles, s);
    case NVDB_FP8_E4M3: return launch_eval_fp8(b, ntiles, s);
  }
  return fail(NVDB_ERR_UNSUPPORTED, "precision %d not implemented", (int)prec);
}

// Launch a batch whose items share one network shape; fills the tile offsets.
nvdb_status launch_batch(EvalBatch& b, nvdb_precision prec, cudaStream_t s) {
  int64_t tiles = 0;
  for (int m = 0; m < b.n; ++m) {
    b.it[m].tile_start = tiles;
    tiles += job_tiles(b.it[m].job.mode, b.it[m].job.n_items);
  }
  if (tiles == 0) return NVDB_OK;
  return launch_eval_prec(b, tiles, prec, s);
}

EvalItem eval_item(const nvdb_model* m, int k, EvalJob job) {
  EvalItem it{};
  it.net = net_view(m, k);
  it.moe = moe_view(m, k);
  for (int e = 1; e < m->n_exp && m->moe(); ++e)
    if (!m->net[3 * e + k].bf16_exact) it.net.wexact = 0;
  job.ox = m->origin[0];
  job.oy = m->origin[1];
  job.oz = m->origin[2];
  if (!job.status) job.status = m->status;
  it.job = job;
  return it;
}

nvdb_status launch_eval(const nvdb_model* m, int k, nvdb_precision prec, EvalJob job, cudaStream_t s) {
  EvalBatch b;
  b.n = 1;
  b.it[0] = eval_item(m, k, job);
  return launch_batch(b, prec, s);
}

template <int NIN, int W, int NOUT = 1>
nvdb_status launch_train_t(const NetView& nv, const TrainJob& job, int grid, cudaStream_t s) {
  if (NOUT == 1 && nv.n_out == 3) return launch_train_t<NIN, W, 3>(nv, job, grid, s);
  const size_t smem = TrainSmem<NIN, W, NOUT>::bytes(nv.layers);
  TRY(set_smem_limit((const void*)train_fwd_bwd_kernel<NIN, W, NOUT>, smem));
  KLAUNCH("train_fwd_bwd", s, train_fwd_bwd_kernel<NIN, W, NOUT><<<grid, kTile, smem, s>>>(nv, job));
  CU(cudaGetLastError());
  return NVDB_OK;
}

// Blocks of one training launch: one per 128-sample tile, at most one per SM (both
// kernels are persistent over tiles).
int train_grid(int64_t batch) { return (int)std::min<int64_t>((batch + kTile - 1) / kTile, num_sms()); }

bool train_prec_ok(int prec) { return prec == NVDB_FP32 || prec == NVDB_BF16; }

nvdb_status launch_train(const nvdb_model* m, int k, int prec, TrainJob job, int grid, cudaStream_t s,
                         const FusedAdam* fa = nullptr) {
  const NetView nv = net_view(m, k);
  const int e = k / 3;   // an expert normalises over its subdomain (Section 3.4)
  job.ox = m->origin[0] + (m->moe() ? m->exp_origin_host[3 * e] : 0);
  job.oy = m->origin[1] + (m->moe() ? m->exp_origin_host[3 * e + 1] : 0);
  job.oz = m->origin[2] + (m->moe() ? m->exp_origin_host[3 * e + 2] : 0);
  if (!job.status) job.status = m->status;
  if (prec == NVDB_BF16) {
    if ((nv.n_out != 1 && nv.n_out != 3) || nv.act != 0)
      return fail(NVDB_ERR_UNSUPPORTED, "BF16 training: ReLU networks only");
    return launch_train_tc(nv, job, grid, s, fa);
  } else if (prec == NVDB_FP32) {
    if (nv.n_in == 32 && nv.width == 32) return launch_train_t<32, 32>(nv, job, grid, s);
    if (nv.n_in == 32 && nv.width == 64) return launch_train_t<32, 64>(nv, job, grid, s);
    if (nv.n_in == 64 && nv.width == 32) return launch_train_t<64, 32>(nv, job, grid, s);
    if (nv.n_in == 64 && nv.width == 64) return launch_train_t<64, 64>(nv, job, grid, s);
  } else {
    return fail(NVDB_ERR_UNSUPPORTED, "training precision %d", prec);
  }
  return fail(NVDB_ERR_UNSUPPORTED, "network shape n=%d w=%d", nv.n_in, nv.width);
}

// Adam's view of the training step at precision `prec`; `refresh`: rewrite the BF16 tiles.
AdamAux adam_aux(const DevNet& d, int prec, bool refresh) {
  AdamAux a{};
  if (prec == NVDB_BF16) a = AdamAux{refresh ? d.wpk : nullptr, 1, d.n_in, d.width, d.layers};
  return a;
}

nvdb_status read_status(uint32_t* d_status, cudaStream_t s, uint32_t* out) {
  uint32_t h = 0;
  CU(cudaMemcpyAsync(&h, d_status, sizeof h, cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  *out = h;
  return NVDB_OK;
}

nvdb_status status_to_error(uint32_t st) {
  if (st & ST_TIMEOUT) return fail(NVDB_ERR_TIMEOUT, "a device-side wait timed out");
  if (st & ST_CAPACITY) return fail(NVDB_ERR_CAPACITY, "output capacity exceeded on the device");
  if (st & ST_CORRUPT) return fail(NVDB_ERR_CORRUPT, "decoded counts differ from the model header");
  return NVDB_OK;
}

// The tensor-core kernels' only device-side error is a timed-out wait; reading it costs
// one stream synchronisation, which the FP32 path (no waits) does not pay.
nvdb_status eval_status(const nvdb_model* m, nvdb_precision prec, cudaStream_t s) {
  if (prec == NVDB_FP32) return NVDB_OK;
  uint32_t hst = 0;
  TRY(read_status(m->status, s, &hst));
  return status_to_error(hst);
}

// Shape of network k: (encoding size, width, hidden layers, head outputs).
void net_shape(const nvdb_model* m, int k, int& nin, int& w, int& L, int& nout) {
  if (m->tile_net(k)) {
    nin = m->ffm[0]; w = m->tile_width; L = m->tile_layers; nout = 1;
    return;
  }
  const int j = k % 3;
  nin = j == 0 ? m->ffm[0] : m->ffm[1];
  w = m->width[j];
  L = m->layers[j];
  nout = j == 0 && m->ternary ? 3 : 1;
}

nvdb_status upload_net(nvdb_model* m, int k, const float* host_params, cudaStream_t s) {
  DevNet& d = m->net[k];
  net_shape(m, k, d.n_in, d.width, d.layers, d.n_out);
  d.P = net_param_count(d.n_in, d.width, d.layers, d.n_out);
  dfree(d.p32); dfree(d.wpk); dfree(d.m); dfree(d.v);
  TRY(dalloc(&d.p32, (size_t)d.P));
  TRY(dalloc(&d.wpk, (size_t)wpk_bytes(d.n_in, d.width, d.layers) + 64));
  if (host_params) CU(cudaMemcpyAsync(d.p32, host_params, d.P * 4, cudaMemcpyHostToDevice, s));
  return NVDB_OK;
}

__global__ void round_bf16_kernel(float* p, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = __bfloat162float(__float2bfloat16_rn(p[i]));
}

bool bf16_exact_layers(const float* p, int64_t n) {
  for (int64_t i = 0; i < n; ++i) {
    uint32_t u;
    std::memcpy(&u, p + i, 4);
    if (u & 0xFFFFu) return false;
  }
  return true;
}

nvdb_status pack_net(nvdb_model* m, int k, cudaStream_t s) {
  DevNet& d = m->net[k];
  KLAUNCH("pack_weights", s, pack_weights_kernel<<<64, 256, 0, s>>>(d.p32, d.wpk, d.n_in, d.width, d.layers));
  CU(cudaGetLastError());
  if (d.layers > 1) {
    KLAUNCH("pack_weights_t", s, pack_weights_t_kernel<<<16, 256, 0, s>>>(d.p32, d.wpk, d.n_in, d.width, d.layers));
    CU(cudaGetLastError());
  }
  if (m->act != 0) return NVDB_OK;   // FP8 tiles and scales: ReLU networks only
  // FP8 activation scales: calibrate on seeded points of the network's domain, then pack
  if (!d.f8_amax) TRY(dalloc(&d.f8_amax, kMaxLayers));
  CU(cudaMemsetAsync(d.f8_amax, 0, kMaxLayers * 4, s));
  const NetView nv = net_view(m, k);
  // calibration domain: the model's extent, or the subdomain's (rounded up to a power of two)
  int lgE = m->log2e;
  if (m->moe())
    for (lgE = 0; (1 << lgE) < m->sub_size; ++lgE) {
    }
  const int lg = m->net_level(k) ? lgE - 3 : lgE;   // level-1 networks work in leaf units
  constexpr int kCalibPoints = 1 << 12;   // one point per thread of 32 blocks
  TRY(launch_calib_amax(nv, lg, 0xF8CA11Bull, kCalibPoints, d.f8_amax, s));
  KLAUNCH("pack_fp8", s, pack_fp8_kernel<<<1, 256, 0, s>>>(d.p32, d.wpk, d.n_in, d.width, d.layers, d.f8_amax));
  CU(cudaGetLastError());
  return NVDB_OK;
}

nvdb_status check_model_shapes(const nvdb_model* m) {
  for (int k = 0; k < (m->ternary ? 4 : 3); ++k) {
    const int kk = k == 3 ? 3 * m->n_exp : k;
    int nin, w, L, nout;
    net_shape(m, kk, nin, w, L, nout);
    if (!supported_shape(nin, w))
      return fail(NVDB_ERR_UNSUPPORTED, "network %d: encoding size %d / width %d (supported: 32, 64)", k, nin, w);
    if (L < 1 || L > kMaxLayers)
      return fail(NVDB_ERR_UNSUPPORTED, "network %d: %d hidden layers (supported: 1..%d)", k, L, kMaxLayers);
  }
  if (m->act != 0 && m->act != 1) return fail(NVDB_ERR_UNSUPPORTED, "activation %d", m->act);
  return NVDB_OK;
}

// Sin networks evaluate in the 16-bit modes without a decomposition (FP8's scale folding
// assumes ReLU).
nvdb_status check_eval_prec(const nvdb_model* m, int k, nvdb_precision prec) {
  (void)k;
  if (prec == NVDB_FP32) return NVDB_OK;
  if (m->act != 0 && (prec == NVDB_FP8_E4M3 || m->moe()))
    return fail(NVDB_ERR_UNSUPPORTED, "sin activation: no FP8, no tensor-core decomposition");
  return NVDB_OK;
}
}  // namespace

// ============================================================================ build
extern "C" nvdb_status nvdb_build(const int32_t* d_ijk, const float* d_val, int64_t n, const nvdb_build_opts* opts,
                                  nvdb_stream stream, nvdb_grid** out) {
  const Range range("nvdb_build");
  if (!out || !opts || n < 0 || (n > 0 && (!d_ijk || !d_val))) return fail(NVDB_ERR_INVALID_ARG, "nvdb_build: bad arguments");
  if (opts->grid_class != 0 && opts->grid_class != 1) return fail(NVDB_ERR_INVALID_ARG, "grid_class must be 0 or 1");
  if (opts->grid_class == 0 && !(opts->half_width > 0.f)) return fail(NVDB_ERR_INVALID_ARG, "half_width must be > 0");
  if (n >= (int64_t)INT32_MAX) return fail(NVDB_ERR_UNSUPPORTED, "nvdb_build: n >= 2^31 - 1");
  if (opts->prune_tiles && !(opts->tile_tolerance >= 0.f))
    return fail(NVDB_ERR_INVALID_ARG, "nvdb_build: tile_tolerance must be >= 0");
  *out = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  auto* g = new nvdb_grid();
  g->grid_class = opts->grid_class;
  g->half_width = opts->grid_class == 0 ? opts->half_width : 0.f;
  g->background = opts->grid_class == 0 ? opts->half_width : 0.f;
  g->n = n;
  nvdb_status st = NVDB_OK;
  uint64_t *k0 = nullptr, *k1 = nullptr;
  uint32_t *i0 = nullptr, *i1 = nullptr, *h = nullptr, *status = nullptr;
  int64_t *e = nullptr, *leaf_node = nullptr;
  unsigned long long* ntile = nullptr;
  auto cleanup = [&]() {
    dfree(k0); dfree(k1); dfree(i0); dfree(i1); dfree(h); dfree(e); dfree(status); dfree(leaf_node); dfree(ntile);
  };
  auto run = [&]() -> nvdb_status {
    if (n == 0) return NVDB_OK;
    TRY(dalloc(&k0, n)); TRY(dalloc(&k1, n)); TRY(dalloc(&i0, n)); TRY(dalloc(&i1, n));
    TRY(dalloc(&h, 3 * (size_t)n)); TRY(dalloc(&e, 3 * (size_t)n)); TRY(dalloc(&status, 1));
    TRY(dalloc(&g->ijk, 3 * (size_t)n)); TRY(dalloc(&g->val, n));
    CU(cudaMemsetAsync(status, 0, 4, s));
    KLAUNCH("build_keys", s, build_keys_kernel<<<blocks_for(n, 256), 256, 0, s>>>(d_ijk, n, k0, i0, status));
    TRY(sort_keys(k0, k1, i0, i1, (int)n, s));
    KLAUNCH("build_gather", s, build_gather_kernel<<<blocks_for(n, 256), 256, 0, s>>>(k1, i1, n, d_ijk, d_val, g->ijk, g->val, h, h + n,
                                                            h + 2 * n, status));
    CU(cudaGetLastError());
    Scan sc;
    int64_t tot[3];
    for (int l = 0; l < 3; ++l) {
      TRY(sc.run(h + l * n, n, e + l * n, s));
      CU(cudaMemcpyAsync(&tot[l], sc.total, 8, cudaMemcpyDeviceToHost, s));
      CU(cudaStreamSynchronize(s));
    }
    uint32_t hst = 0;
    TRY(read_status(status, s, &hst));
    if (hst & ST_RANGE) return fail(NVDB_ERR_INVALID_ARG, "nvdb_build: coordinate outside [0, 2^21)");
    if (hst & ST_DUP) return fail(NVDB_ERR_DUPLICATE_VOXEL, "nvdb_build: duplicate voxel");
    g->n_leaf = tot[0];
    g->n_l1 = tot[1];
    g->n_l2 = tot[2];
    TRY(dalloc(&g->leaf_origin, g->n_leaf)); TRY(dalloc(&g->leaf_first, g->n_leaf + 1));
    TRY(dalloc(&g->leaf_mask, 8 * g->n_leaf)); TRY(dalloc(&g->l1_origin, g->n_l1));
    TRY(dalloc(&g->l1_mask, 64 * g->n_l1)); TRY(dalloc(&g->l2_origin, g->n_l2)); TRY(dalloc(&g->l2_mask, 512 * g->n_l2));
    CU(cudaMemsetAsync(g->leaf_mask, 0, 64 * g->n_leaf, s));
    CU(cudaMemsetAsync(g->l1_mask, 0, 512 * g->n_l1, s));
    CU(cudaMemsetAsync(g->l2_mask, 0, 4096 * g->n_l2, s));
    TRY(dalloc(&leaf_node, g->n_leaf));
    KLAUNCH("build_fill", s, build_fill_kernel<<<blocks_for(n, 256), 256, 0, s>>>(g->ijk, n, h, h + n, h + 2 * n, e, e + n, e + 2 * n,
                                                          g->leaf_origin, g->leaf_first, g->leaf_mask, g->l1_origin,
                                                          g->l1_mask, g->l2_origin, g->l2_mask, leaf_node));
    CU(cudaGetLastError());
    CU(cudaMemcpyAsync(g->leaf_first + g->n_leaf, &g->n, 8, cudaMemcpyHostToDevice, s));
    if (opts->prune_tiles) {   // active tiles of level 1 (Section 3.1)
      TRY(dalloc(&g->leaf_tile, g->n_leaf)); TRY(dalloc(&g->l1_tile_mask, 64 * g->n_l1)); TRY(dalloc(&ntile, 1));
      CU(cudaMemsetAsync(g->l1_tile_mask, 0, 512 * g->n_l1, s));
      CU(cudaMemsetAsync(ntile, 0, 8, s));
      KLAUNCH("tile_prune", s, tile_prune_kernel<<<blocks_for(g->n_leaf * 32, 256), 256, 0, s>>>(
                                   g->leaf_mask, g->leaf_first, g->leaf_origin, leaf_node, g->n_leaf,
                                   opts->tile_tolerance, g->val, g->leaf_tile, g->l1_tile_mask, ntile));
      unsigned long long nt = 0;
      CU(cudaMemcpyAsync(&nt, ntile, 8, cudaMemcpyDeviceToHost, s));
      CU(cudaStreamSynchronize(s));
      g->n_tiles = (int64_t)nt;
    }
    // encoding domain: level-1 aligned bounding box, power-of-two extent >= 128
    std::vector<int4> l1(g->n_l1);
    CU(cudaMemcpyAsync(l1.data(), g->l1_origin, g->n_l1 * sizeof(int4), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    int lo[3] = {INT32_MAX, INT32_MAX, INT32_MAX}, hi[3] = {0, 0, 0};
    for (auto& o : l1) {
      const int v[3] = {o.x, o.y, o.z};
      for (int d = 0; d < 3; ++d) { lo[d] = std::min(lo[d], v[d]); hi[d] = std::max(hi[d], v[d] + 128); }
    }
    int ext = 0;
    for (int d = 0; d < 3; ++d) { g->origin[d] = lo[d]; ext = std::max(ext, hi[d] - lo[d]); }
    g->log2e = 7;
    while ((1 << g->log2e) < ext) ++g->log2e;
    return NVDB_OK;
  };
  st = run();
  cleanup();
  if (st != NVDB_OK) { delete g; return st; }
  *out = g;
  return NVDB_OK;
}

extern "C" nvdb_status nvdb_grid_info(const nvdb_grid* g, nvdb_info* out) {
  if (!g || !out) return fail(NVDB_ERR_INVALID_ARG, "nvdb_grid_info: NULL");
  out->grid_class = g->grid_class;
  out->background = g->background;
  out->half_width = g->half_width;
  for (int d = 0; d < 3; ++d) out->origin[d] = g->origin[d];
  out->log2_extent = g->log2e;
  out->n_active = g->n;
  out->n_leaf = g->n_leaf;
  out->n_l1 = g->n_l1;
  out->n_l2 = g->n_l2;
  out->n_experts = 0;
  out->subdomain = 0;
  out->n_tiles = g->n_tiles;
  return NVDB_OK;
}

extern "C" nvdb_status nvdb_grid_tiles(const nvdb_grid* g, uint8_t* leaf_tile, uint64_t* l1_tile_mask,
                                       nvdb_stream stream) {
  if (!g) return fail(NVDB_ERR_INVALID_ARG, "nvdb_grid_tiles: NULL grid");
  cudaStream_t s = (cudaStream_t)stream;
  if (leaf_tile && g->n_leaf) {
    if (g->leaf_tile) CU(cudaMemcpyAsync(leaf_tile, g->leaf_tile, g->n_leaf, cudaMemcpyDeviceToHost, s));
    else std::memset(leaf_tile, 0, g->n_leaf);
  }
  if (l1_tile_mask && g->n_l1) {
    if (g->l1_tile_mask) CU(cudaMemcpyAsync(l1_tile_mask, g->l1_tile_mask, 512 * g->n_l1, cudaMemcpyDeviceToHost, s));
    else std::memset(l1_tile_mask, 0, 512 * g->n_l1);
  }
  CU(cudaStreamSynchronize(s));
  return NVDB_OK;
}

static nvdb_status copy_int4_to3(const int4* d, int64_t n, int32_t* host, cudaStream_t s) {
  std::vector<int4> t(n);
  if (n) CU(cudaMemcpyAsync(t.data(), d, n * sizeof(int4), cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  for (int64_t i = 0; i < n; ++i) { host[3 * i] = t[i].x; host[3 * i + 1] = t[i].y; host[3 * i + 2] = t[i].z; }
  return NVDB_OK;
}

extern "C" nvdb_status nvdb_grid_read(const nvdb_grid* g, int32_t* ijk, float* val, int32_t* leaf_origin,
                                      uint64_t* leaf_mask, int32_t* l1_origin, uint64_t* l1_mask, nvdb_stream stream) {
  if (!g) return fail(NVDB_ERR_INVALID_ARG, "nvdb_grid_read: NULL grid");
  cudaStream_t s = (cudaStream_t)stream;
  if (ijk && g->n) CU(cudaMemcpyAsync(ijk, g->ijk, 12 * g->n, cudaMemcpyDeviceToHost, s));
  if (val && g->n) CU(cudaMemcpyAsync(val, g->val, 4 * g->n, cudaMemcpyDeviceToHost, s));
  if (leaf_mask && g->n_leaf) CU(cudaMemcpyAsync(leaf_mask, g->leaf_mask, 64 * g->n_leaf, cudaMemcpyDeviceToHost, s));
  if (l1_mask && g->n_l1) CU(cudaMemcpyAsync(l1_mask, g->l1_mask, 512 * g->n_l1, cudaMemcpyDeviceToHost, s));
  if (leaf_origin) TRY(copy_int4_to3(g->leaf_origin, g->n_leaf, leaf_origin, s));
  if (l1_origin) TRY(copy_int4_to3(g->l1_origin, g->n_l1, l1_origin, s));
  CU(cudaStreamSynchronize(s));
  return NVDB_OK;
}

extern "C" nvdb_status nvdb_grid_free(nvdb_grid* g) {
  delete g;
  return NVDB_OK;
}

// ============================================================================ compress
extern "C" void nvdb_train_opts_default(nvdb_train_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof *o);
  o->seed = 1;
  for (int k = 0; k < 3; ++k) { o->width[k] = 32; o->layers[k] = 3; }
  o->ffm_sigma = 1.25f;
  o->steps = 200;
  o->batch = 4096;
  o->lr = 1e-3f;
  o->lr_decay = 0.975f;
  o->lr_interval = 100;
  o->loss = NVDB_LOSS_MSE;
  o->train_prec = NVDB_FP32;
  o->patch_precs = (1u << kNumPrecisions) - 1u;   // every precision
  o->stop_window = 50;
}

namespace {
nvdb_status ensure_partial(nvdb_model* m, int64_t count) {
  if (count <= m->partial_cap) return NVDB_OK;
  dfree(m->partial);
  TRY(dalloc(&m->partial, (size_t)count));
  m->partial_cap = count;
  return NVDB_OK;
}

// Training populations of one expert of a decomposed model (Section 3.4): per network, the
// indices of the candidates inside the expert's support (level-1 slots, leaves, voxels).
struct PopLists {
  uint32_t* list[4] = {nullptr, nullptr, nullptr, nullptr};
  int64_t n[4] = {0, 0, 0, 0};
  ~PopLists() { for (auto& l : list) dfree(l); }
};

// Indices of the set flags[0 .. count) into a new list (count of them in *total).
nvdb_status compact_list(const uint32_t* flags, int64_t count, uint32_t** list, int64_t* total, cudaStream_t s) {
  int64_t* off = nullptr;
  Scan sc;
  auto run = [&]() -> nvdb_status {
    TRY(dalloc(&off, (size_t)count + 1));
    TRY(sc.run(flags, count, off, s));
    CU(cudaMemcpyAsync(total, sc.total, 8, cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    TRY(dalloc(list, (size_t)*total + 1));
    if (count) KLAUNCH("compact_flags", s, compact_flags_kernel<<<blocks_for(count, 256), 256, 0, s>>>(flags, off, count, *list));
    CU(cudaGetLastError());
    CU(cudaStreamSynchronize(s));
    return NVDB_OK;
  };
  const nvdb_status st = run();
  dfree(off);
  return st;
}

// Training populations of a model with active tiles (Section 3.3.1): the level-0 networks
// train on the leaves that are not tiles (net 1: those leaves, net 2: their voxels), the
// tile value regressor on the tiles (net 3: the tile leaves).
nvdb_status tile_populations(const nvdb_grid* g, PopLists& pl, cudaStream_t s) {
  const Range range("tile populations");
  uint32_t* flags = nullptr;
  auto run = [&]() -> nvdb_status {
    TRY(dalloc(&flags, (size_t)std::max(g->n, g->n_leaf) + 1));
    KLAUNCH("leaf_tile_flags", s, leaf_tile_flags_kernel<<<blocks_for(g->n_leaf, 256), 256, 0, s>>>(g->leaf_tile, g->n_leaf, 0u, flags));
    TRY(compact_list(flags, g->n_leaf, &pl.list[1], &pl.n[1], s));
    KLAUNCH("leaf_tile_flags", s, leaf_tile_flags_kernel<<<blocks_for(g->n_leaf, 256), 256, 0, s>>>(g->leaf_tile, g->n_leaf, 1u, flags));
    TRY(compact_list(flags, g->n_leaf, &pl.list[3], &pl.n[3], s));
    KLAUNCH("voxel_nontile_flags", s, voxel_nontile_flags_kernel<<<blocks_for(g->n_leaf * 32, 256), 256, 0, s>>>(
                                          g->leaf_tile, g->leaf_first, g->n_leaf, flags));
    TRY(compact_list(flags, g->n, &pl.list[2], &pl.n[2], s));
    if (pl.n[1] == 0 || pl.n[2] == 0) return fail(NVDB_ERR_UNSUPPORTED, "every leaf is a tile: no level-0 networks to train");
    return NVDB_OK;
  };
  const nvdb_status st = run();
  dfree(flags);
  return st;
}

nvdb_status expert_populations(const nvdb_model* m, const nvdb_grid* g, int ex, PopLists& pl, cudaStream_t s) {
  const Range range("expert populations");
  for (int j = 0; j < 3; ++j) {
    const int64_t count = j == 0 ? g->n_l1 * 4096 : j == 1 ? g->n_leaf : g->n;
    const int sh = j == 0 ? 3 : 0;
    int lo[3], hi[3];
    for (int d = 0; d < 3; ++d) {
      const int a = g->origin[d] + m->exp_origin_host[3 * ex + d];
      lo[d] = (a >> sh) - (m->sub_halo >> sh);
      hi[d] = ((a + m->sub_size) >> sh) + (m->sub_halo >> sh);
    }
    uint32_t* flags = nullptr;
    int64_t* off = nullptr;
    Scan sc;
    auto run = [&]() -> nvdb_status {
      TRY(dalloc(&flags, (size_t)count + 1));
      TRY(dalloc(&off, (size_t)count + 1));
      if (count)
        KLAUNCH("support_flags", s, support_flags_kernel<<<blocks_for(count, 256), 256, 0, s>>>(
                                        j, g->l1_origin, g->leaf_origin, g->ijk, count, make_int4(lo[0], lo[1], lo[2], 0),
                                        make_int4(hi[0], hi[1], hi[2], 0), flags));
      TRY(sc.run(flags, count, off, s));
      int64_t total = 0;
      CU(cudaMemcpyAsync(&total, sc.total, 8, cudaMemcpyDeviceToHost, s));
      CU(cudaStreamSynchronize(s));
      if (total == 0) return fail(NVDB_ERR_INVALID_ARG, "expert %d has no training candidates for network %d", ex, j);
      TRY(dalloc(&pl.list[j], (size_t)total));
      KLAUNCH("compact_flags", s, compact_flags_kernel<<<blocks_for(count, 256), 256, 0, s>>>(flags, off, count, pl.list[j]));
      CU(cudaGetLastError());
      pl.n[j] = total;
      return NVDB_OK;
    };
    const nvdb_status st = run();
    CU(cudaStreamSynchronize(s));
    dfree(flags);
    dfree(off);
    TRY(st);
  }
  return NVDB_OK;
}

TrainJob grid_train_job(const nvdb_grid* g, int net, const nvdb_train_opts* o) {
  TrainJob j{};
  j.net = net;
  j.stream = net;
  j.loss = net >= 2 ? o->loss : LOSS_BCE;
  j.seed = o->seed;
  j.batch = o->batch;
  j.l1_origin = g->l1_origin; j.l1_mask = g->l1_mask; j.n_l1 = g->n_l1;
  j.l1_tile_mask = net == 0 && g->n_tiles > 0 ? g->l1_tile_mask : nullptr;
  j.leaf_origin = g->leaf_origin; j.leaf_mask = g->leaf_mask; j.n_leaf = g->n_leaf;
  j.ijk = g->ijk; j.val = g->val; j.n = g->n;
  j.tscale = g->grid_class == 0 ? 1.f / g->half_width : 1.f;
  j.resample = o->resample;
  j.sampling = net == 2 ? o->sampling : 0;
  j.leaf_first = g->leaf_first;
  j.log2e = g->log2e;
  j.gx = g->origin[0]; j.gy = g->origin[1]; j.gz = g->origin[2];
  j.bg_target = g->grid_class == 0 ? 1.f : 0.f;   // the background (+w for level sets), scaled
  return j;
}

// Classify every candidate of the grid at `prec`; mismatches with the explicit
// masks become the patch lists (Section 3.3.2).
nvdb_status make_patches(nvdb_model* m, const nvdb_grid* g, int prec, cudaStream_t s) {
  const Range range("patches");
  PatchSet ps;
  ps.prec = prec;
  for (int lev = 0; lev < 2; ++lev) {
    const int64_t items = lev == 0 ? g->n_l1 : g->n_leaf;
    const int wpi = lev == 0 ? 128 : 16;
    uint32_t *words = nullptr, *twords = nullptr, *counts = nullptr, *off32 = nullptr;
    int64_t* off = nullptr;
    uint16_t* idx = nullptr;
    auto run = [&]() -> nvdb_status {
      TRY(dalloc(&words, (size_t)items * wpi + 1));
      TRY(dalloc(&counts, items + 1));
      TRY(dalloc(&off, items + 1));
      TRY(dalloc(&off32, items + 1));
      EvalJob job{};
      job.mode = lev == 0 ? MODE_L1 : MODE_L0;
      job.nodes = lev == 0 ? g->l1_origin : g->leaf_origin;
      job.n_items = items;
      job.words = words;
      const bool tern1 = m->ternary && lev == 0;
      if (tern1) TRY(dalloc(&twords, (size_t)items * wpi + 1));
      job.twords = twords;
      TRY(launch_eval(m, lev == 0 ? 0 : 1, (nvdb_precision)prec, job, s));
      const uint32_t* truth = reinterpret_cast<const uint32_t*>(lev == 0 ? g->l1_mask : g->leaf_mask);
      if (m->ternary && lev == 1 && items)   // tiles are not classified: no level-0 patches
        KLAUNCH("tile_words_full", s, tile_words_full_kernel<<<blocks_for(items * 16, 256), 256, 0, s>>>(words, g->leaf_tile, items));
      if (tern1 && items)
        KLAUNCH("tern_mismatch", s, tern_mismatch_kernel<<<blocks_for(items, 128), 128, 0, s>>>(
                                        words, twords, truth, reinterpret_cast<const uint32_t*>(g->l1_tile_mask), items,
                                        counts));
      else if (items)
        KLAUNCH("mismatch_count", s, mismatch_count_kernel<<<blocks_for(items, 128), 128, 0, s>>>(words, truth, wpi, items, counts));
      TRY(m->scan.run(counts, items, off, s));
      KLAUNCH("offsets_to_u32", s, offsets_to_u32_kernel<<<blocks_for(items + 1, 256), 256, 0, s>>>(off, m->scan.total, items, off32));
      int64_t total = 0;
      CU(cudaMemcpyAsync(&total, m->scan.total, 8, cudaMemcpyDeviceToHost, s));
      CU(cudaStreamSynchronize(s));
      TRY(dalloc(&idx, (size_t)total + 1));
      if (tern1 && items)   // entries slot | true class << 12
        KLAUNCH("tern_emit_patches", s, tern_emit_patches_kernel<<<blocks_for(items, 128), 128, 0, s>>>(
                                            words, truth, reinterpret_cast<const uint32_t*>(g->l1_tile_mask), items, off, idx));
      else if (items)
        KLAUNCH("emit_patches", s, emit_patches_kernel<<<blocks_for(items, 128), 128, 0, s>>>(words, wpi, items, off, idx));
      CU(cudaGetLastError());
      // the set keeps the device lists
      (lev == 0 ? ps.d_l1_off : ps.d_l0_off) = off32;
      (lev == 0 ? ps.d_l1_idx : ps.d_l0_idx) = idx;
      (lev == 0 ? ps.n1 : ps.n0) = total;
      off32 = nullptr;
      idx = nullptr;
      return NVDB_OK;
    };
    const nvdb_status st = run();
    dfree(words); dfree(twords); dfree(counts); dfree(off); dfree(off32); dfree(idx);
    if (st != NVDB_OK) {
      ps.release();
      return st;
    }
  }
  for (auto& p : m->patches)
    if (p.prec == prec) { p.release(); p = ps; return NVDB_OK; }
  m->patches.push_back(ps);
  return NVDB_OK;
}
}  // namespace

extern "C" nvdb_status nvdb_compress(const nvdb_grid* g, const nvdb_train_opts* o, const nvdb_model* warm,
                                     nvdb_stream stream, nvdb_model** out) {
  const Range range("nvdb_compress");
  if (!g || !o || !out) return fail(NVDB_ERR_INVALID_ARG, "nvdb_compress: NULL argument");
  if (o->steps < 0 || o->batch <= 0 || !(o->lr >= 0.f) || o->lr_interval < 0)
    return fail(NVDB_ERR_INVALID_ARG, "nvdb_compress: bad steps/batch/lr");
  if (o->loss != NVDB_LOSS_MSE && o->loss != NVDB_LOSS_L1) return fail(NVDB_ERR_INVALID_ARG, "loss must be MSE or L1");
  if (o->patch_precs >> kNumPrecisions) return fail(NVDB_ERR_INVALID_ARG, "patch_precs: no precision %u", o->patch_precs);
  if (!train_prec_ok(o->train_prec)) return fail(NVDB_ERR_UNSUPPORTED, "training precision %d", o->train_prec);
  if (g->n == 0) return fail(NVDB_ERR_INVALID_ARG, "nvdb_compress: empty grid");
  if ((uint64_t)g->n_leaf * 512 >= (1ull << 32) || (uint64_t)g->n_l1 * 4096 >= (1ull << 32))
    return fail(NVDB_ERR_UNSUPPORTED, "candidate population >= 2^32");
  if (o->resample < 0 || (uint64_t)o->resample * (uint64_t)o->batch >= (1ull << 32))
    return fail(NVDB_ERR_INVALID_ARG, "resample x batch must be in [0, 2^32)");
  if (o->sampling < 0 || o->sampling > 2) return fail(NVDB_ERR_INVALID_ARG, "sampling must be 0, 1 or 2");
  if (o->sampling == 2 && (g->log2e > 10 || o->subdomain || (warm && warm->moe())))
    return fail(NVDB_ERR_UNSUPPORTED, "dense sampling: extent at most 1024 and no decomposition");
  const int sub = warm ? warm->sub_size : o->subdomain;
  const int halo = warm ? warm->sub_halo : (o->halo ? o->halo : 8);
  if (sub < 0 || sub % 512 || (sub && (halo < 8 || (halo & (halo - 1)) || 4 * halo > sub)))
    return fail(NVDB_ERR_INVALID_ARG, "subdomain must be a multiple of 512 and the halo a power of two in [8, subdomain/4]");
  const bool tern = g->n_tiles > 0;   // active tiles: ternary level 1 + tile value regressor
  if (warm && warm->ternary != tern) return fail(NVDB_ERR_INVALID_ARG, "warm start: the grids differ in active tiles");
  if (tern && (sub || o->sampling)) return fail(NVDB_ERR_UNSUPPORTED, "active tiles with a decomposition or ablation sampling");
  const int act = warm ? warm->act : o->activation;
  const float omega = warm ? warm->omega : (o->activation ? o->omega : 1.f);
  if (act != 0 && act != 1) return fail(NVDB_ERR_INVALID_ARG, "activation must be 0 (ReLU) or 1 (sin)");
  if (act == 1 && !(omega > 0.f)) return fail(NVDB_ERR_INVALID_ARG, "sin activation: omega must be > 0");
  if (act == 1 && o->train_prec != NVDB_FP32) return fail(NVDB_ERR_UNSUPPORTED, "sin activation: FP32 training only");
  if (act == 1 && ((o->patch_precs & (1u << NVDB_FP8_E4M3)) || (sub && (o->patch_precs & ~(1u << NVDB_FP32)))))
    return fail(NVDB_ERR_UNSUPPORTED, "sin activation: no FP8 patch set (and FP32 only with a decomposition)");
  *out = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  auto* m = new nvdb_model();
  const bool resume = o->resume != 0 && warm != nullptr;
  auto run = [&]() -> nvdb_status {
    m->grid_class = g->grid_class;
    m->background = g->background;
    m->half_width = g->half_width;
    for (int d = 0; d < 3; ++d) m->origin[d] = g->origin[d];
    m->log2e = g->log2e;
    m->n_l2 = g->n_l2; m->n_l1 = g->n_l1; m->n_leaf = g->n_leaf; m->n_active = g->n;
    m->act = act;
    m->omega = omega;
    m->n_tiles = g->n_tiles;
    if (warm) {
      m->ffm[0] = warm->ffm[0]; m->ffm[1] = warm->ffm[1];
      for (int k = 0; k < 3; ++k) { m->width[k] = warm->width[k]; m->layers[k] = warm->layers[k]; }
      m->tile_width = warm->tile_width;
      m->tile_layers = warm->tile_layers;
    } else {
      for (int k = 0; k < 3; ++k) { m->width[k] = o->width[k]; m->layers[k] = o->layers[k]; }
      m->ffm[0] = o->ffm_size[0] ? o->ffm_size[0] : o->width[0];
      m->ffm[1] = o->ffm_size[1] ? o->ffm_size[1] : std::max(o->width[1], o->width[2]);
      m->tile_width = o->tile_width ? o->tile_width : o->width[0];
      m->tile_layers = o->tile_layers ? o->tile_layers : o->layers[0];
    }
    if (tern) m->set_ternary(true);
    TRY(check_model_shapes(m));
    if (o->train_prec == NVDB_BF16)
      for (int k = 0; k < (tern ? 4 : 3); ++k) {
        int nin, w, L, nout;
        net_shape(m, k, nin, w, L, nout);
        if (L > kTrainTcMaxLayers)
          return fail(NVDB_ERR_UNSUPPORTED, "BF16 training: network %d has %d hidden layers (at most %d)", k, L,
                      kTrainTcMaxLayers);
      }
    TRY(dalloc(&m->status, 1));
    CU(cudaMemsetAsync(m->status, 0, 4, s));
    double E = std::ldexp(1.0, m->log2e);
    if (sub > 0) {   // sparse domain decomposition (Section 3.4): subdomains holding voxels
      m->sub_size = sub;
      m->sub_halo = halo;
      m->sub_dims = (int)((std::ldexp(1.0, m->log2e) + sub - 1) / sub);
      const int n = m->sub_dims;
      if ((int64_t)n * n * n > (1 << 24)) return fail(NVDB_ERR_UNSUPPORTED, "more than 2^24 subdomains");
      if (warm) {
        m->expert_of_host = warm->expert_of_host;
        m->exp_origin_host = warm->exp_origin_host;
        m->set_experts(warm->n_exp);
        if (g->origin[0] != warm->origin[0] || g->origin[1] != warm->origin[1] || g->origin[2] != warm->origin[2] ||
            g->log2e != warm->log2e)
          return fail(NVDB_ERR_INVALID_ARG, "warm start of a decomposed model: the grid's domain differs");
      } else {
        std::vector<int32_t> l1(3 * g->n_l1);
        TRY(copy_int4_to3(g->l1_origin, g->n_l1, l1.data(), s));   // a level-1 node lies in one subdomain
        std::vector<char> occ((size_t)n * n * n, 0);
        for (int64_t i = 0; i < g->n_l1; ++i) {
          const int ix = (l1[3 * i] - g->origin[0]) / sub, iy = (l1[3 * i + 1] - g->origin[1]) / sub,
                    iz = (l1[3 * i + 2] - g->origin[2]) / sub;
          occ[((size_t)ix * n + iy) * n + iz] = 1;
        }
        m->expert_of_host.assign((size_t)n * n * n, -1);
        int ne = 0;
        for (size_t c = 0; c < occ.size(); ++c)
          if (occ[c]) {
            m->expert_of_host[c] = ne++;
            m->exp_origin_host.push_back((int32_t)(c / ((size_t)n * n)) * sub);
            m->exp_origin_host.push_back((int32_t)((c / n) % n) * sub);
            m->exp_origin_host.push_back((int32_t)(c % n) * sub);
          }
        m->set_experts(ne);
      }
      TRY(upload_moe(m, s));
      E = sub;   // every expert normalises over its subdomain
    } else if (warm && warm->moe()) {
      return fail(NVDB_ERR_INVALID_ARG, "warm start: decomposition differs");
    }
    for (int lev = 0; lev < 2; ++lev) {
      m->q_host[lev] = warm ? warm->q_host[lev]
                            : ffm_increments(o->seed, lev == 0 ? 1 : 0, m->ffm[lev] / 2, (double)o->ffm_sigma,
                                             lev == 0 ? E / 8 : E);
      TRY(dalloc(&m->q_dev[lev], m->q_host[lev].size()));
      CU(cudaMemcpy(m->q_dev[lev], m->q_host[lev].data(), m->q_host[lev].size() * 4, cudaMemcpyHostToDevice));
    }
    for (int k = 0; k < m->n_net(); ++k) {
      if (warm) {
        TRY(upload_net(m, k, nullptr, s));
        const float* src = resume && warm->net[k].master ? warm->net[k].master : warm->net[k].p32;
        CU(cudaMemcpyAsync(m->net[k].p32, src, m->net[k].P * 4, cudaMemcpyDeviceToDevice, s));
        m->net[k].bf16_exact = warm->net[k].bf16_exact && o->steps == 0;
      } else {
        int nin, w, L, nout;
        net_shape(m, k, nin, w, L, nout);
        const std::vector<float> p = xavier_params(o->seed, k, nin, w, L, nout);
        TRY(upload_net(m, k, p.data(), s));
        CU(cudaStreamSynchronize(s));
      }
      TRY(dalloc(&m->net[k].m, m->net[k].P));
      TRY(dalloc(&m->net[k].v, m->net[k].P));
      if (resume) {   // Adam state and history of the interrupted run
        CU(cudaMemcpyAsync(m->net[k].m, warm->net[k].m, m->net[k].P * 4, cudaMemcpyDeviceToDevice, s));
        CU(cudaMemcpyAsync(m->net[k].v, warm->net[k].v, m->net[k].P * 4, cudaMemcpyDeviceToDevice, s));
        m->losses[k] = warm->losses[k];
      } else {
        CU(cudaMemsetAsync(m->net[k].m, 0, m->net[k].P * 4, s));
        CU(cudaMemsetAsync(m->net[k].v, 0, m->net[k].P * 4, s));
      }
    }
    // explicit upper tree (root + level-2 nodes) is kept as is (Section 3.3.1)
    TRY(dalloc(&m->l2_origin, g->n_l2));
    TRY(dalloc(&m->l2_mask, 512 * g->n_l2));
    CU(cudaMemcpyAsync(m->l2_origin, g->l2_origin, g->n_l2 * sizeof(int4), cudaMemcpyDeviceToDevice, s));
    CU(cudaMemcpyAsync(m->l2_mask, g->l2_mask, g->n_l2 * 4096, cudaMemcpyDeviceToDevice, s));
    m->l2_origin_host.resize(3 * g->n_l2);
    m->l2_mask_host.resize(512 * g->n_l2);
    TRY(copy_int4_to3(g->l2_origin, g->n_l2, m->l2_origin_host.data(), s));
    CU(cudaMemcpyAsync(m->l2_mask_host.data(), g->l2_mask, g->n_l2 * 4096, cudaMemcpyDeviceToHost, s));
    // training: each network for `steps` Adam steps.  The three networks share nothing
    // (parameters, Adam state, samples, partial sums, step counter and losses are per
    // network), so each trains on a stream of its own and their kernels overlap: a training
    // launch holds one CTA per SM, and the SMs its last, partial round of tiles leaves idle
    // take the next network's CTAs.  (The caller's stream may be the legacy default stream,
    // which cannot be captured.)  The step index lives in device memory, so one captured
    // chunk of steps replays as a CUDA graph.  Profiled runs launch every step and train the
    // networks one after another (per-kernel events would overlap otherwise).
    static const char* kTrainRange[4] = {"train level-1 classifier", "train level-0 classifier", "train regressor",
                                         "train tile regressor"};
    const int nk = tern ? 4 : 3;   // networks per expert
    // arithmetic of each network's training (every network, the ternary classifier included)
    auto tprec = [&](int) { return o->train_prec; };
    struct NetRun {
      cudaStream_t ts = nullptr;
      cudaEvent_t ev = nullptr;
      float* d_loss = nullptr;
      int* d_step = nullptr;
      uint32_t* d_sync = nullptr;   // grid barrier of the fused Adam step
      TrainJob job{};
      AdamSched sc{};
      cudaGraphExec_t exec = nullptr;
      int done = 0, ran = 0, chunk = 50;
      bool early = false, active = true;
    };
    const int grid = train_grid(o->batch);
    const bool profiled = prof::g_on.load();
    int64_t poff[5] = {0, 0, 0, 0, 0};
    for (int k = 0; k < nk; ++k) poff[k + 1] = poff[k] + (int64_t)grid * (m->net[k].P + 1);
    nvdb_status st = ensure_partial(m, poff[nk]);
    // a decomposed model trains expert after expert, each on the candidates of its support
    for (int ex = 0; ex < m->n_exp && st == NVDB_OK; ++ex) {
    PopLists pl;
    if (m->moe() && o->steps > 0) st = expert_populations(m, g, ex, pl, s);
    if (tern && o->steps > 0) st = tile_populations(g, pl, s);
    NetRun nr[4];
    for (int k = 0; k < nk && st == NVDB_OK; ++k) {
      NetRun& r = nr[k];
      if (cudaStreamCreateWithFlags(&r.ts, cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&r.ev, cudaEventDisableTiming) != cudaSuccess) {
        st = fail(NVDB_ERR_CUDA, "training stream");
        break;
      }
      if (cudaEventRecord(r.ev, s) != cudaSuccess || cudaStreamWaitEvent(r.ts, r.ev, 0) != cudaSuccess) {
        st = fail(NVDB_ERR_CUDA, "training stream order");
        break;
      }
      if ((st = dalloc(&r.d_loss, (size_t)std::max(1, o->steps))) != NVDB_OK) break;
      if ((st = dalloc(&r.d_step, 2)) != NVDB_OK) break;
      if ((st = dalloc(&r.d_sync, 2)) != NVDB_OK) break;
      if (cudaMemsetAsync(r.d_sync, 0, 8, r.ts) != cudaSuccess) {
        st = fail(NVDB_ERR_CUDA, "barrier words");
        break;
      }
      r.job = grid_train_job(g, k, o);
      r.job.stream = 3 * ex + k;
      if (m->moe() || (tern && k > 0)) {
        r.job.pop = pl.list[k];
        r.job.pop_n = pl.n[k];
        r.job.pop_shift = k == 1 ? 9 : 0;
      }
      r.job.partial = m->partial + poff[k];
      r.job.step_dev = r.d_step;
      if (tprec(k) == NVDB_BF16 && (st = pack_net(m, 3 * ex + k, r.ts)) != NVDB_OK) break;   // the BF16 tiles of step 1
      // the first step of this call: after the interrupted run's steps when resuming
      r.done = (int)m->losses[3 * ex + k].size();
      const int first = r.done + 1;
      if (cudaMemcpyAsync(r.d_step, &first, 4, cudaMemcpyHostToDevice, r.ts) != cudaSuccess ||
          cudaStreamSynchronize(r.ts) != cudaSuccess) {   // `first` is a stack value
        st = fail(NVDB_ERR_CUDA, "step counter");
        break;
      }
      r.sc = AdamSched{r.d_step, o->lr, o->lr_decay, o->lr_interval, r.d_loss, first};
      r.early = k < 3 && o->stop_loss[k] > 0.f && o->stop_window > 0;
      r.chunk = r.early ? o->stop_window : 50;
      r.active = o->steps > 0;
    }
    auto one_step = [&](int k) -> nvdb_status {
      NetRun& r = nr[k];
      DevNet& d = m->net[3 * ex + k];
      if (tprec(k) == NVDB_BF16 && fused_adam_enabled()) {   // gradient and Adam in one launch
        FusedAdam fa{};
        fa.sync = r.d_sync;
        fa.params = d.p32;
        fa.m = d.m;
        fa.v = d.v;
        fa.rp = adam_aux(d, NVDB_BF16, true);
        fa.sc = r.sc;
        fa.loss_scale = 1.f / (float)o->batch;
        return launch_train(m, 3 * ex + k, tprec(k), r.job, grid, r.ts, &fa);
      }
      TRY(launch_train(m, 3 * ex + k, tprec(k), r.job, grid, r.ts));
      KLAUNCH("adam_reduce", r.ts, adam_reduce_kernel<<<blocks_for(d.P + 1, 32), 32 * kRedGroups, 0, r.ts>>>(
                                       r.job.partial, grid, d.P, d.p32, d.m, d.v, 0, 0.f, nullptr, nullptr,
                                       1.f / (float)o->batch, adam_aux(d, tprec(k), true), r.sc));
      CU(cudaGetLastError());
      return NVDB_OK;
    };
    // one chunk of network k's steps: eager first, then captured once and replayed
    auto run_chunk = [&](int k) -> nvdb_status {
      NetRun& r = nr[k];
      const Range range(kTrainRange[k]);
      const int n = std::min(r.chunk, o->steps - r.ran);
      if (!r.exec && r.ran > 0 && n == r.chunk && !profiled) {
        cudaGraph_t gr = nullptr;
        if (cudaStreamBeginCapture(r.ts, cudaStreamCaptureModeRelaxed) != cudaSuccess)
          return fail(NVDB_ERR_CUDA, "training capture");
        nvdb_status cst = NVDB_OK;
        for (int i = 0; i < r.chunk && cst == NVDB_OK; ++i) cst = one_step(k);
        const cudaError_t e = cudaStreamEndCapture(r.ts, &gr);
        if (cst == NVDB_OK && e == cudaSuccess && cudaGraphInstantiate(&r.exec, gr, 0) != cudaSuccess) r.exec = nullptr;
        if (gr) cudaGraphDestroy(gr);
        TRY(cst);
        if (e != cudaSuccess || !r.exec) return fail(NVDB_ERR_CUDA, "training graph: %s", cudaGetErrorString(e));
      }
      if (r.exec && n == r.chunk) {
        if (cudaGraphLaunch(r.exec, r.ts) != cudaSuccess) return fail(NVDB_ERR_CUDA, "training graph launch");
      } else {
        for (int i = 0; i < n; ++i) TRY(one_step(k));
      }
      r.ran += n;
      if (r.ran >= o->steps) r.active = false;
      if (r.early && r.active && r.ran % o->stop_window == 0) {   // warm-start early stop (Section 3.6)
        std::vector<float> w(o->stop_window);
        cudaError_t e = cudaMemcpyAsync(w.data(), r.d_loss + (r.ran - o->stop_window), o->stop_window * 4,
                                        cudaMemcpyDeviceToHost, r.ts);
        if (e == cudaSuccess) e = cudaStreamSynchronize(r.ts);
        if (e != cudaSuccess) return fail(NVDB_ERR_CUDA, "loss readback: %s", cudaGetErrorString(e));
        double mean = 0.0;
        for (float v : w) mean += v;
        if (mean / o->stop_window < (double)o->stop_loss[k]) r.active = false;
      }
      return NVDB_OK;
    };
    // concurrent: chunks of the three networks interleaved; profiled: one network at a time
    for (int k0 = 0; k0 < (profiled ? nk : 1) && st == NVDB_OK; ++k0) {
      const int k1 = profiled ? k0 + 1 : nk;
      for (bool any = true; any && st == NVDB_OK;) {
        any = false;
        for (int k = profiled ? k0 : 0; k < k1 && st == NVDB_OK; ++k)
          if (nr[k].active) {
            st = run_chunk(k);
            any = true;
          }
      }
      // profiled: the next network starts when this one's kernels have run
      if (profiled && st == NVDB_OK && cudaStreamSynchronize(nr[k0].ts) != cudaSuccess)
        st = fail(NVDB_ERR_CUDA, "training stream");
    }
    for (int k = 0; k < nk; ++k) {
      NetRun& r = nr[k];
      if (r.exec) cudaGraphExecDestroy(r.exec);
      if (st == NVDB_OK) {
        m->losses[3 * ex + k].resize(r.done + r.ran);
        if (r.ran) {
          cudaError_t e = cudaMemcpyAsync(m->losses[3 * ex + k].data() + r.done, r.d_loss, r.ran * 4, cudaMemcpyDeviceToHost, r.ts);
          if (e == cudaSuccess) e = cudaStreamSynchronize(r.ts);
          if (e != cudaSuccess) st = fail(NVDB_ERR_CUDA, "loss readback: %s", cudaGetErrorString(e));
        }
      }
      if (r.ts) {   // the caller's stream continues after the training streams
        if (st == NVDB_OK && (cudaEventRecord(r.ev, r.ts) != cudaSuccess || cudaStreamWaitEvent(s, r.ev, 0) != cudaSuccess))
          st = fail(NVDB_ERR_CUDA, "training stream order");
        cudaStreamSynchronize(r.ts);
        cudaStreamDestroy(r.ts);
      }
      if (r.ev) cudaEventDestroy(r.ev);
      dfree(r.d_step);
      dfree(r.d_loss);
      dfree(r.d_sync);
    }
    }   // experts
    TRY(st);
    if (o->train_prec == NVDB_BF16)   // the BF16 step trained BF16 weights: store them as such
      for (int k = 0; k < m->n_net(); ++k) {
        if (tprec(m->tile_net(k) ? 3 : k % 3) != NVDB_BF16) continue;
        DevNet& d = m->net[k];
        const int64_t n = d.P - d.n_out * (d.width + 1);   // every weight and bias except the FP32 head
        TRY(dalloc(&d.master, d.P));        // kept for a resumed run
        CU(cudaMemcpyAsync(d.master, d.p32, d.P * 4, cudaMemcpyDeviceToDevice, s));
        KLAUNCH("round_bf16", s, round_bf16_kernel<<<blocks_for(n, 256), 256, 0, s>>>(d.p32, n));
        CU(cudaGetLastError());
        d.bf16_exact = true;
      }
    for (int k = 0; k < m->n_net(); ++k) TRY(pack_net(m, k, s));
    TRY(upload_views(m, s));
    uint32_t pp = o->patch_precs ? o->patch_precs : (1u << NVDB_FP32);
    for (int p = 0; p < kNumPrecisions; ++p)
      if (pp & (1u << p)) {
        TRY(make_patches(m, g, p, s));
      }
    uint32_t hst = 0;
    TRY(read_status(m->status, s, &hst));
    TRY(status_to_error(hst));
    return NVDB_OK;
  };
  const nvdb_status st = run();
  if (st != NVDB_OK) { delete m; return st; }
  *out = m;
  return NVDB_OK;
}

extern "C" nvdb_status nvdb_compress_sequence(const nvdb_grid* const* grids, int n_frames, const nvdb_train_opts* o,
                                              float refine_lr_scale, int32_t refine_steps, int32_t warm_steps,
                                              nvdb_stream stream, nvdb_model** out) {
  const Range range("nvdb_compress_sequence");
  if (!grids || n_frames <= 0 || !o || !out || refine_steps < 0 || warm_steps < 0 || !(refine_lr_scale > 0.f) ||
      o->stop_window <= 0)
    return fail(NVDB_ERR_INVALID_ARG, "nvdb_compress_sequence: bad arguments");
  for (int f = 0; f < n_frames; ++f)
    if (!grids[f]) return fail(NVDB_ERR_INVALID_ARG, "nvdb_compress_sequence: NULL grid %d", f);
  std::vector<nvdb_model*> ms(n_frames, nullptr);
  auto cleanup = [&]() { for (auto* m : ms) delete m; };
  nvdb_train_opts a = *o;
  for (int k = 0; k < 3; ++k) a.stop_loss[k] = 0.f;
  a.resume = 0;
  nvdb_status st = nvdb_compress(grids[0], &a, nullptr, stream, &ms[0]);   // frame 0, cold
  if (st == NVDB_OK && refine_steps > 0) {   // frame 0 refined at the lower rate
    nvdb_train_opts r = a;
    r.lr = a.lr * refine_lr_scale;
    r.steps = refine_steps;
    nvdb_model* refined = nullptr;
    st = nvdb_compress(grids[0], &r, ms[0], stream, &refined);
    if (st == NVDB_OK) {
      delete ms[0];
      ms[0] = refined;
    }
  }
  float target[3] = {0.f, 0.f, 0.f};
  if (st == NVDB_OK)
    for (int k = 0; k < 3; ++k) {   // frame 0's final loss (experts: their mean)
      double sum = 0.0;
      int64_t cnt = 0;
      for (int e = 0; e < ms[0]->n_exp; ++e) {
        const auto& l = ms[0]->losses[3 * e + k];
        for (size_t i = l.size() > (size_t)o->stop_window ? l.size() - o->stop_window : 0; i < l.size(); ++i, ++cnt) sum += l[i];
      }
      target[k] = cnt ? (float)(sum / cnt) : 0.f;
    }
  for (int f = 1; f < n_frames && st == NVDB_OK; ++f) {   // warm frames with the early stop
    nvdb_train_opts w = a;
    w.lr = a.lr * refine_lr_scale;
    w.steps = warm_steps;
    for (int k = 0; k < 3; ++k) w.stop_loss[k] = target[k];
    st = nvdb_compress(grids[f], &w, ms[f - 1], stream, &ms[f]);
  }
  if (st != NVDB_OK) {
    cleanup();
    return st;
  }
  for (int f = 0; f < n_frames; ++f) out[f] = ms[f];
  return NVDB_OK;
}

extern "C" nvdb_status nvdb_model_losses(const nvdb_model* m, int net, float* losses, int64_t cap, int64_t* count) {
  if (!m || net < 0 || net >= m->n_net() || (cap > 0 && !losses)) return fail(NVDB_ERR_INVALID_ARG, "nvdb_model_losses: bad arguments");
  const auto& l = m->losses[net];
  if (count) *count = (int64_t)l.size();
  for (int64_t i = 0; i < cap && i < (int64_t)l.size(); ++i) losses[i] = l[i];
  return NVDB_OK;
}

// ============================================================================ decompress
namespace {
bool same_shape(const nvdb_model* a, const nvdb_model* b) {
  if (a->ffm[0] != b->ffm[0] || a->ffm[1] != b->ffm[1]) return false;
  if (a->ternary != b->ternary || a->act != b->act || a->omega != b->omega) return false;
  if (a->ternary && (a->tile_width != b->tile_width || a->tile_layers != b->tile_layers)) return false;
  for (int k = 0; k < 3; ++k)
    if (a->width[k] != b->width[k] || a->layers[k] != b->layers[k]) return false;
  return true;
}

// Top-down decode (Section 3.5) of n <= kMaxBatch models with the same network
// shapes, in one launch per stage: level-1 origins from the level-2 child masks,
// level-1 classification + patches -> leaf origins, level-0 classification +
// patches -> voxel offsets; with an output, the voxels and their regressed
// values (concatenated per model, canonical order).  Levels of the models are
// concatenated in model order in `d`.
// A non-blocking stream of the library's own for device-to-host copies that overlap
// kernels of the caller's stream (one per device, created on first use).
nvdb_status copy_stream(cudaStream_t* out) {
  static std::mutex mu;
  static std::map<int, cudaStream_t> streams;
  int dev = 0;
  CU(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  auto it = streams.find(dev);
  if (it == streams.end()) {
    cudaStream_t cs = nullptr;
    CU(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    it = streams.emplace(dev, cs).first;
  }
  *out = it->second;
  return NVDB_OK;
}

// Host destination of a decode: the voxels are copied on the library's copy stream as soon
// as they are emitted (overlapping the regression), the values after the regression.
struct HostSink {
  int32_t* ijk;
  float* val;
  cudaStream_t copy;
  cudaEvent_t ev;
};

nvdb_status decode_batch(nvdb_model* const* ms, int n, nvdb_precision prec, DecodeScratch& d, int32_t* out_ijk,
                         float* out_val, cudaStream_t s, const HostSink* sink = nullptr) {
  std::vector<int64_t> s2(n + 1, 0), s1(n + 1, 0), sl(n + 1, 0), sa(n + 1, 0);
  for (int m = 0; m < n; ++m) {
    s2[m + 1] = s2[m] + ms[m]->n_l2;
    s1[m + 1] = s1[m] + ms[m]->n_l1;
    sl[m + 1] = sl[m] + ms[m]->n_leaf;
    sa[m + 1] = sa[m] + ms[m]->n_active;
  }
  const int64_t N2 = s2[n], N1 = s1[n], NL = sl[n], NA = sa[n];
  const bool tern = ms[0]->ternary;   // a batch holds models of one kind (same_shape)
  std::vector<int64_t> st(n + 1, 0);
  for (int m = 0; m < n; ++m) st[m + 1] = st[m] + ms[m]->n_tiles;
  const int64_t NT = st[n];
  TRY(d.reserve(N2, N1, NL));
  if (tern) TRY(d.reserve_tiles(NT));
  CU(cudaMemsetAsync(d.lb, 0, (size_t)DecodeScratch::lb_words(d.cap2, d.cap1, d.capl) * 8, s));
  std::vector<const PatchSet*> ps(n);
  for (int m = 0; m < n; ++m) ps[m] = ms[m]->patch_set(prec);
  if (N2) {
    L2Batch lb;
    lb.n = n;
    for (int m = 0; m < n; ++m)
      lb.it[m] = L2Item{reinterpret_cast<const uint64_t*>(ms[m]->l2_mask), ms[m]->l2_origin, s2[m]};
    KLAUNCH("l2_scan", s, l2_scan_batch_kernel<<<(unsigned)N2, 512, 0, s>>>(lb, N2, d.l2_off, N1, d.lb2(), d.status,
                                                                           d.l1_origin));
  }
  EvalBatch b;
  b.n = n;
  for (int m = 0; m < n; ++m) {
    EvalJob j{};
    j.mode = MODE_L1;
    j.nodes = d.l1_origin + s1[m];
    j.n_items = ms[m]->n_l1;
    j.words = d.l1_words + 128 * s1[m];
    j.twords = tern ? d.t1_words + 128 * s1[m] : nullptr;
    j.status = d.status;
    b.it[m] = eval_item(ms[m], 0, j);
  }
  {
    const Range range("decode: level-1 classification");
    TRY(launch_batch(b, prec, s));
  }
  PatchBatch pb;
  pb.n = n;
  for (int m = 0; m < n; ++m) pb.it[m] = PatchItem{ps[m]->d_l1_off, ps[m]->d_l1_idx, s1[m]};
  if (tern && N1) {   // ternary patches set each listed slot's class, then both masks are counted
    KLAUNCH("tern_patch", s, tern_patch_batch_kernel<<<blocks_for(N1 * 32, 256), 256, 0, s>>>(d.l1_words, d.t1_words, N1, pb));
    PatchBatch none = pb;
    for (int m = 0; m < n; ++m) none.it[m].off = nullptr;
    KLAUNCH("patch_scan_l1", s, patch_scan_batch_kernel<<<(unsigned)DecodeScratch::blocks1(N1), 256, 0, s>>>(
                                    d.l1_words, 128, N1, none, d.l1_off, NL, d.lb1(), d.status));
    KLAUNCH("tile_scan", s, patch_scan_batch_kernel<<<(unsigned)DecodeScratch::blocks1(N1), 256, 0, s>>>(
                                d.t1_words, 128, N1, none, d.t1_off, NT, d.lbt(), d.status));
    // the leaf items with their tile ranks (which need the tile scan), then the tiles
    KLAUNCH("emit_leaves", s, emit_leaves_kernel<<<blocks_for(N1 * 32, 256), 256, 0, s>>>(
                                  d.l1_words, d.l1_origin, N1, d.l1_off, d.leaf_origin, NL, d.status, d.t1_words,
                                  d.t1_off));
    if (NT)
      KLAUNCH("emit_tiles", s, emit_tile_coords_kernel<<<blocks_for(N1 * 32, 256), 256, 0, s>>>(
                                   d.t1_words, d.l1_origin, N1, d.t1_off, d.tile_ijk, NT, d.status));
  } else if (N1) {   // patches, counts, scan and the leaf origins in one launch
    KLAUNCH("patch_scan_l1", s, patch_scan_batch_kernel<kEmitLeaves><<<(unsigned)DecodeScratch::blocks1(N1), 256, 0, s>>>(
                                 d.l1_words, 128, N1, pb, d.l1_off, NL, d.lb1(), d.status, nullptr, d.l1_origin,
                                 d.leaf_origin));
  } else if (NL) {
    KLAUNCH("flag_corrupt", s, flag_corrupt_kernel<<<1, 1, 0, s>>>(d.status));   // leaves expected, no nodes
  }
  for (int m = 0; m < n; ++m) {
    EvalJob j{};
    j.mode = MODE_L0;
    j.nodes = d.leaf_origin + sl[m];
    j.n_items = ms[m]->n_leaf;
    j.words = d.leaf_words + 16 * sl[m];
    j.status = d.status;
    b.it[m] = eval_item(ms[m], 1, j);
  }
  {
    const Range range("decode: level-0 classification");
    TRY(launch_batch(b, prec, s));
  }
  for (int m = 0; m < n; ++m) pb.it[m] = PatchItem{ps[m]->d_l0_off, ps[m]->d_l0_idx, sl[m]};
  if (NL && out_ijk) {   // patches, counts, scan and the voxels in one launch
    KLAUNCH("patch_scan_l0", s, patch_scan_batch_kernel<kEmitVoxels, kScanItemsL0><<<(unsigned)DecodeScratch::blocks0(NL), 256, 0, s>>>(
                                 d.leaf_words, 16, NL, pb, d.leaf_off, NA, d.lb0(), d.status,
                                 tern ? d.leaf_origin : nullptr, d.leaf_origin, out_ijk));
  } else if (NL) {
    KLAUNCH("patch_scan_l0", s, patch_scan_batch_kernel<kEmitNone, kScanItemsL0><<<(unsigned)DecodeScratch::blocks0(NL), 256, 0, s>>>(
                                 d.leaf_words, 16, NL, pb, d.leaf_off, NA, d.lb0(), d.status,
                                 tern ? d.leaf_origin : nullptr));
  } else if (NA) {
    KLAUNCH("flag_corrupt", s, flag_corrupt_kernel<<<1, 1, 0, s>>>(d.status));   // voxels expected, no leaves
  }
  if (out_ijk) {
    if (sink && NA) {
      CU(cudaEventRecord(sink->ev, s));
      CU(cudaStreamWaitEvent(sink->copy, sink->ev, 0));
      CU(cudaMemcpyAsync(sink->ijk, out_ijk, (size_t)NA * 12, cudaMemcpyDeviceToHost, sink->copy));
    }
    for (int m = 0; m < n; ++m) {
      EvalJob j{};
      j.mode = MODE_LIST;
      j.ijk = out_ijk + 3 * sa[m];
      j.n_items = ms[m]->n_active;
      j.out = out_val + sa[m];
      j.scale = ms[m]->value_scale();
      j.status = d.status;
      b.it[m] = eval_item(ms[m], 2, j);
    }
    {
      const Range range("decode: regression");
      TRY(launch_batch(b, prec, s));
    }
  }
  if (tern && NT) {   // tile values (net 3 at the tile's leaf-unit coordinate), then the tiles' voxels
    for (int m = 0; m < n; ++m) {
      EvalJob j{};
      j.mode = MODE_LIST;
      j.ijk = d.tile_ijk + 3 * st[m];
      j.n_items = ms[m]->n_tiles;
      j.shift = 3;
      j.out = d.tval + st[m];
      j.scale = ms[m]->value_scale();
      j.status = d.status;
      b.it[m] = eval_item(ms[m], 3, j);
    }
    {
      const Range range("decode: tile values");
      TRY(launch_batch(b, prec, s));
    }
    if (out_val && NL)
      KLAUNCH("tile_fill", s, tile_fill_kernel<<<blocks_for(NL * 32, 256), 256, 0, s>>>(d.leaf_origin, NL, d.leaf_off,
                                                                                     d.tval, out_val, NA));
  }
  if (out_ijk) {
    if (sink && NA) {
      CU(cudaEventRecord(sink->ev, s));
      CU(cudaStreamWaitEvent(sink->copy, sink->ev, 0));
      CU(cudaMemcpyAsync(sink->val, out_val, (size_t)NA * 4, cudaMemcpyDeviceToHost, sink->copy));
    }
  }
  CU(cudaGetLastError());
  return NVDB_OK;
}

// Consecutive runs of models with the same shapes, at most kMaxBatch long.
std::vector<std::pair<int, int>> batch_runs(const nvdb_model* const* models, int n_models) {
  std::vector<std::pair<int, int>> runs;
  for (int i = 0; i < n_models;) {
    int j = i + 1;
    while (j < n_models && j - i < kMaxBatch && same_shape(models[i], models[j])) ++j;
    runs.emplace_back(i, j);
    i = j;
  }
  return runs;
}
}  // namespace

namespace {
nvdb_status decompress_impl(const nvdb_model* const* models, int n_models, nvdb_precision prec, int32_t* d_ijk,
                            float* d_val, int32_t* h_ijk, float* h_val, int64_t capacity, int64_t* counts,
                            nvdb_stream stream);
}

extern "C" nvdb_status nvdb_decompress(const nvdb_model* const* models, int n_models, nvdb_precision prec,
                                       int32_t* d_ijk, float* d_val, int64_t capacity, int64_t* counts,
                                       nvdb_stream stream) {
  const Range range("nvdb_decompress");
  return decompress_impl(models, n_models, prec, d_ijk, d_val, nullptr, nullptr, capacity, counts, stream);
}

extern "C" nvdb_status nvdb_decompress_host(const nvdb_model* const* models, int n_models, nvdb_precision prec,
                                            int32_t* d_ijk, float* d_val, int32_t* h_ijk, float* h_val,
                                            int64_t capacity, int64_t* counts, nvdb_stream stream) {
  const Range range("nvdb_decompress_host");
  if (d_ijk && (!h_ijk || !h_val)) return fail(NVDB_ERR_INVALID_ARG, "nvdb_decompress_host: NULL host buffer");
  return decompress_impl(models, n_models, prec, d_ijk, d_val, h_ijk, h_val, capacity, counts, stream);
}

namespace {
nvdb_status decompress_impl(const nvdb_model* const* models, int n_models, nvdb_precision prec, int32_t* d_ijk,
                            float* d_val, int32_t* h_ijk, float* h_val, int64_t capacity, int64_t* counts,
                            nvdb_stream stream) {
  if (!models || n_models < 0 || !counts || capacity < 0) return fail(NVDB_ERR_INVALID_ARG, "nvdb_decompress: bad arguments");
  if (d_ijk && !d_val) return fail(NVDB_ERR_INVALID_ARG, "nvdb_decompress: d_val is NULL");
  int64_t need = 0;
  for (int i = 0; i < n_models; ++i) {
    if (!models[i]) return fail(NVDB_ERR_INVALID_ARG, "nvdb_decompress: NULL model");
    counts[i] = models[i]->n_active;
    need += models[i]->n_active;
    if (!models[i]->patch_set(prec)) return fail(NVDB_ERR_UNSUPPORTED, "model %d has no patch set for precision %d", i, (int)prec);
    TRY(check_eval_prec(models[i], 1, prec));
  }
  if (!d_ijk) return NVDB_OK;
  if (need > capacity) return fail(NVDB_ERR_CAPACITY, "nvdb_decompress: need %lld voxels, capacity %lld", (long long)need, (long long)capacity);
  cudaStream_t s = (cudaStream_t)stream;
  nvdb_model* const* ms = const_cast<nvdb_model* const*>(models);
  int64_t base = 0;
  std::vector<DecodeScratch*> tmp;
  nvdb_status st = NVDB_OK;
  std::vector<uint32_t*> status_words;
  HostSink sink{};
  if (h_ijk) {
    TRY(copy_stream(&sink.copy));
    CU(cudaEventCreateWithFlags(&sink.ev, cudaEventDisableTiming));
  }
  for (const auto& r : batch_runs(models, n_models)) {
    const int n = r.second - r.first;
    DecodeScratch* d = &ms[r.first]->ds;
    if (n > 1) {
      tmp.push_back(new DecodeScratch());
      d = tmp.back();
    }
    sink.ijk = h_ijk + 3 * base;
    sink.val = h_val + base;
    st = decode_batch(ms + r.first, n, prec, *d, d_ijk + 3 * base, d_val + base, s, h_ijk ? &sink : nullptr);
    if (st != NVDB_OK) break;
    status_words.push_back(d->status);
    for (int m = r.first; m < r.second; ++m) base += ms[m]->n_active;
  }
  if (h_ijk) {   // the caller's stream continues after the copies
    const cudaError_t e1 = cudaEventRecord(sink.ev, sink.copy);
    const cudaError_t e2 = e1 == cudaSuccess ? cudaStreamWaitEvent(s, sink.ev, 0) : e1;
    if (st == NVDB_OK && e2 != cudaSuccess) st = fail(NVDB_ERR_CUDA, "copy stream: %s", cudaGetErrorString(e2));
  }
  for (uint32_t* sw : status_words) {
    if (st != NVDB_OK) break;
    uint32_t hst = 0;
    st = read_status(sw, s, &hst);
    if (st == NVDB_OK) st = status_to_error(hst);
  }
  if (!tmp.empty() || h_ijk) cudaStreamSynchronize(s);
  for (auto* d : tmp) delete d;
  if (h_ijk) cudaEventDestroy(sink.ev);
  return st;
}
}  // namespace

// ============================================================================ query
namespace {
constexpr int64_t kQueryBatch = 1 << 20;

nvdb_status build_query_cache(nvdb_model* m, cudaStream_t s) {
  QueryCache& q = m->qc;
  if (q.ready) return NVDB_OK;
  const PatchSet* ps = m->patch_set(NVDB_FP32);
  int prec = NVDB_FP32;
  if (!ps && !m->patches.empty()) { ps = &m->patches[0]; prec = ps->prec; }
  if (!ps) return fail(NVDB_ERR_UNSUPPORTED, "model has no patch set");
  nvdb_model* one[1] = {m};
  TRY(decode_batch(one, 1, (nvdb_precision)prec, m->ds, nullptr, nullptr, s));
  TRY(dalloc(&q.l2_key, m->n_l2 + 1)); TRY(dalloc(&q.l2_pre, 512 * m->n_l2 + 1));
  TRY(dalloc(&q.l1_pre, 128 * m->n_l1 + 1));
  if (m->n_l2) {
    KLAUNCH("l2_keys", s, l2_keys_kernel<<<blocks_for(m->n_l2, 128), 128, 0, s>>>(m->l2_origin, m->n_l2, q.l2_key));
    KLAUNCH("word_prefix64", s, word_prefix64_kernel<<<blocks_for(m->n_l2, 128), 128, 0, s>>>(reinterpret_cast<const uint64_t*>(m->l2_mask), 512,
                                                                  m->n_l2, q.l2_pre));
  }
  if (m->n_l1) KLAUNCH("word_prefix", s, word_prefix_kernel<<<blocks_for(m->n_l1, 128), 128, 0, s>>>(m->ds.l1_words, 128, m->n_l1, q.l1_pre));
  q.batch = kQueryBatch;
  TRY(dalloc(&q.qmask, q.batch)); TRY(dalloc(&q.counts, q.batch)); TRY(dalloc(&q.off, q.batch + 1));
  TRY(dalloc(&q.list, 3 * 8 * q.batch)); TRY(dalloc(&q.vals, 8 * q.batch));
  if (m->ternary) { TRY(dalloc(&q.qtile, q.batch)); TRY(dalloc(&q.qtv, 8 * q.batch)); }
  TRY(m->scan.reserve(q.batch));
  uint32_t hst = 0;
  TRY(read_status(m->ds.status, s, &hst));
  TRY(status_to_error(hst));
  q.ready = true;
  return NVDB_OK;
}

TopoView topo_view(const nvdb_model* m) {
  TopoView tv;
  tv.n_l2 = m->n_l2;
  tv.l2_key = m->qc.l2_key;
  tv.l2_mask = reinterpret_cast<const uint64_t*>(m->l2_mask);
  tv.l2_pre = m->qc.l2_pre;
  tv.l2_base = m->ds.l2_off;
  tv.l1_words = m->ds.l1_words;
  tv.l1_pre = m->qc.l1_pre;
  tv.l1_base = m->ds.l1_off;
  tv.leaf_words = m->ds.leaf_words;
  tv.items = m->ternary ? m->ds.leaf_origin : nullptr;
  tv.tval = m->ternary ? m->ds.tval : nullptr;
  return tv;
}
}  // namespace

extern "C" nvdb_status nvdb_query(const nvdb_model* cm, const float* d_xyz, int64_t n, nvdb_precision prec,
                                  float* d_out, uint8_t* d_active, nvdb_stream stream) {
  const Range range("nvdb_query");
  if (!cm || n < 0 || (n > 0 && (!d_xyz || !d_out))) return fail(NVDB_ERR_INVALID_ARG, "nvdb_query: bad arguments");
  if (!eval_prec_ok(prec)) return fail(NVDB_ERR_UNSUPPORTED, "precision %d", (int)prec);
  nvdb_model* m = const_cast<nvdb_model*>(cm);
  TRY(check_eval_prec(m, 2, prec));
  cudaStream_t s = (cudaStream_t)stream;
  TRY(build_query_cache(m, s));
  if (prec != NVDB_FP32) CU(cudaMemsetAsync(m->status, 0, 4, s));
  QueryCache& q = m->qc;
  const TopoView tv = topo_view(m);
  for (int64_t b0 = 0; b0 < n; b0 += q.batch) {
    const int64_t nb = std::min(q.batch, n - b0);
    const float* xyz = d_xyz + 3 * b0;
    KLAUNCH("query_lookup", s, query_lookup_kernel<<<blocks_for(nb, 256), 256, 0, s>>>(tv, xyz, nb, q.qmask, q.counts,
                                                             d_active ? d_active + b0 : nullptr, q.qtile, q.qtv));
    TRY(m->scan.run(q.counts, nb, q.off, s));
    KLAUNCH("query_emit", s, query_emit_kernel<<<blocks_for(nb, 256), 256, 0, s>>>(xyz, nb, q.qmask, q.off, q.list));
    EvalJob jr{};
    jr.mode = MODE_LIST;
    jr.ijk = q.list;
    jr.n_items = 8 * nb;
    jr.n_dev = m->scan.total;
    jr.out = q.vals;
    jr.scale = m->value_scale();
    TRY(launch_eval(m, 2, prec, jr, s));
    KLAUNCH("query_blend", s, query_blend_kernel<<<blocks_for(nb, 256), 256, 0, s>>>(xyz, nb, q.qmask, q.off, q.vals, m->background, d_out + b0,
                                                            q.qtile, q.qtv));
    CU(cudaGetLastError());
  }
  return eval_status(m, prec, s);
}

// ============================================================================ explicit-grid sampling, mCD
namespace {
__global__ void mask_count64_kernel(const unsigned long long* words, int wpi, int64_t n, uint32_t* counts) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  uint32_t c = 0;
  for (int w = 0; w < wpi; ++w) c += __popcll(words[t * wpi + w]);
  counts[t] = c;
}

// The grid's random-access view; the key, prefix and base arrays are built once per grid.
nvdb_status grid_view(nvdb_grid* g, cudaStream_t s, GridView* out) {
  if (!g->l2_key && g->n > 0) {
    Scan sc;
    uint32_t* cnt = nullptr;
    auto run = [&]() -> nvdb_status {
      TRY(dalloc(&g->l2_key, g->n_l2)); TRY(dalloc(&g->l2_pre, 512 * g->n_l2)); TRY(dalloc(&g->l2_base, g->n_l2 + 1));
      TRY(dalloc(&g->l1_pre, 64 * g->n_l1)); TRY(dalloc(&g->l1_base, g->n_l1 + 1));
      TRY(dalloc(&cnt, (size_t)std::max(g->n_l2, g->n_l1) + 1));
      KLAUNCH("l2_keys", s, l2_keys_kernel<<<blocks_for(g->n_l2, 128), 128, 0, s>>>(g->l2_origin, g->n_l2, g->l2_key));
      KLAUNCH("word_prefix64", s, word_prefix64_kernel<<<blocks_for(g->n_l2, 128), 128, 0, s>>>(
                                      reinterpret_cast<const uint64_t*>(g->l2_mask), 512, g->n_l2, g->l2_pre));
      KLAUNCH("mask_count", s, mask_count64_kernel<<<blocks_for(g->n_l2, 128), 128, 0, s>>>(g->l2_mask, 512, g->n_l2, cnt));
      TRY(sc.run(cnt, g->n_l2, g->l2_base, s));
      KLAUNCH("word_prefix64", s, word_prefix64_kernel<<<blocks_for(g->n_l1, 128), 128, 0, s>>>(
                                      reinterpret_cast<const uint64_t*>(g->l1_mask), 64, g->n_l1, g->l1_pre));
      KLAUNCH("mask_count", s, mask_count64_kernel<<<blocks_for(g->n_l1, 128), 128, 0, s>>>(g->l1_mask, 64, g->n_l1, cnt));
      TRY(sc.run(cnt, g->n_l1, g->l1_base, s));
      CU(cudaStreamSynchronize(s));
      return NVDB_OK;
    };
    const nvdb_status st = run();
    dfree(cnt);
    if (st != NVDB_OK) { dfree(g->l2_key); return st; }
  }
  GridView v;
  v.n_l2 = g->n_l2;
  v.l2_key = g->l2_key;
  v.l2_mask = reinterpret_cast<const uint64_t*>(g->l2_mask);
  v.l2_pre = g->l2_pre;
  v.l2_base = g->l2_base;
  v.l1_mask = reinterpret_cast<const uint64_t*>(g->l1_mask);
  v.l1_pre = g->l1_pre;
  v.l1_base = g->l1_base;
  v.leaf_mask = reinterpret_cast<const uint64_t*>(g->leaf_mask);
  v.leaf_first = g->leaf_first;
  v.val = g->val;
  v.background = g->background;
  *out = v;
  return NVDB_OK;
}

nvdb_status iso_points(nvdb_grid* g, cudaStream_t s, float** pts, int64_t* count) {
  *pts = nullptr;
  *count = 0;
  if (g->n == 0) return NVDB_OK;
  GridView v;
  TRY(grid_view(g, s, &v));
  uint32_t* cnt = nullptr;
  int64_t* off = nullptr;
  Scan sc;
  auto run = [&]() -> nvdb_status {
    TRY(dalloc(&cnt, g->n)); TRY(dalloc(&off, g->n));
    KLAUNCH("iso_count", s, iso_count_kernel<<<blocks_for(g->n, 256), 256, 0, s>>>(v, g->ijk, g->n, cnt));
    TRY(sc.run(cnt, g->n, off, s));
    CU(cudaMemcpyAsync(count, sc.total, 8, cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    TRY(dalloc(pts, 3 * (size_t)*count + 3));
    KLAUNCH("iso_emit", s, iso_emit_kernel<<<blocks_for(g->n, 256), 256, 0, s>>>(v, g->ijk, g->n, off, *pts));
    CU(cudaGetLastError());
    return NVDB_OK;
  };
  const nvdb_status st = run();
  cudaStreamSynchronize(s);
  dfree(cnt);
  dfree(off);
  if (st != NVDB_OK) dfree(*pts);
  return st;
}

// sum_i |out_i| over a device array, blocks reduced in order
nvdb_status abs_sum(const float* x, int64_t n, cudaStream_t s, double* out) {
  *out = 0.0;
  if (n == 0) return NVDB_OK;
  const int nb = (int)std::min<int64_t>(blocks_for(n, 256), 1024);
  double* bs = nullptr;
  TRY(dalloc(&bs, nb));
  std::vector<double> h(nb);
  KLAUNCH("abs_sum", s, abs_sum_kernel<<<nb, 256, 0, s>>>(x, n, bs));
  cudaError_t e = cudaMemcpyAsync(h.data(), bs, nb * 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  dfree(bs);
  if (e != cudaSuccess) return fail(NVDB_ERR_CUDA, "abs_sum: %s", cudaGetErrorString(e));
  for (double v : h) *out += v;
  return NVDB_OK;
}
}  // namespace

extern "C" nvdb_status nvdb_grid_sample(const nvdb_grid* cg, const float* d_xyz, int64_t n, int order, float* d_out,
                                        nvdb_stream stream) {
  if (!cg || n < 0 || (n > 0 && (!d_xyz || !d_out)) || (order != 0 && order != 1 && order != 3))
    return fail(NVDB_ERR_INVALID_ARG, "nvdb_grid_sample: bad arguments");
  if (n == 0) return NVDB_OK;
  nvdb_grid* g = const_cast<nvdb_grid*>(cg);
  cudaStream_t s = (cudaStream_t)stream;
  GridView v;
  TRY(grid_view(g, s, &v));
  KLAUNCH("grid_sample", s, grid_sample_kernel<<<blocks_for(n, 256), 256, 0, s>>>(v, d_xyz, n, order, d_out));
  CU(cudaGetLastError());
  return NVDB_OK;
}

extern "C" nvdb_status nvdb_grid_isosurface(const nvdb_grid* cg, float* d_pts, int64_t capacity, int64_t* count,
                                            nvdb_stream stream) {
  if (!cg || !count || capacity < 0) return fail(NVDB_ERR_INVALID_ARG, "nvdb_grid_isosurface: bad arguments");
  if (cg->grid_class != 0) return fail(NVDB_ERR_UNSUPPORTED, "nvdb_grid_isosurface: level sets only");
  cudaStream_t s = (cudaStream_t)stream;
  float* pts = nullptr;
  TRY(iso_points(const_cast<nvdb_grid*>(cg), s, &pts, count));
  nvdb_status st = NVDB_OK;
  if (d_pts && *count > capacity) st = fail(NVDB_ERR_CAPACITY, "nvdb_grid_isosurface: %lld points", (long long)*count);
  else if (d_pts && *count) {
    const cudaError_t e = cudaMemcpyAsync(d_pts, pts, (size_t)*count * 12, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) cudaStreamSynchronize(s);
    else st = fail(NVDB_ERR_CUDA, "isosurface copy: %s", cudaGetErrorString(e));
  }
  dfree(pts);
  return st;
}

extern "C" nvdb_status nvdb_mcd(const nvdb_grid* ref, const nvdb_grid* rec, double* mcd, nvdb_stream stream) {
  const Range range("nvdb_mcd");
  if (!ref || !rec || !mcd) return fail(NVDB_ERR_INVALID_ARG, "nvdb_mcd: bad arguments");
  if (ref->grid_class != 0 || rec->grid_class != 0) return fail(NVDB_ERR_UNSUPPORTED, "nvdb_mcd: level sets only");
  cudaStream_t s = (cudaStream_t)stream;
  nvdb_grid* g[2] = {const_cast<nvdb_grid*>(ref), const_cast<nvdb_grid*>(rec)};
  double part[2] = {0.0, 0.0};
  for (int a = 0; a < 2; ++a) {   // points of grid a's isosurface, sampled (trilinear) in the other grid
    float *pts = nullptr, *sdf = nullptr;
    int64_t n = 0;
    auto run = [&]() -> nvdb_status {
      TRY(iso_points(g[a], s, &pts, &n));
      if (n == 0) return fail(NVDB_ERR_INVALID_ARG, "nvdb_mcd: grid %d has no zero crossing", a);
      TRY(dalloc(&sdf, n));
      GridView v;
      TRY(grid_view(g[1 - a], s, &v));
      KLAUNCH("grid_sample", s, grid_sample_kernel<<<blocks_for(n, 256), 256, 0, s>>>(v, pts, n, 1, sdf));
      double sum = 0.0;
      TRY(abs_sum(sdf, n, s, &sum));
      part[a] = sum / (2.0 * (double)n);
      return NVDB_OK;
    };
    const nvdb_status st = run();
    cudaStreamSynchronize(s);
    dfree(pts);
    dfree(sdf);
    TRY(st);
  }
  *mcd = part[0] + part[1];
  return NVDB_OK;
}

// ============================================================================ ray marching
extern "C" nvdb_status nvdb_render(const nvdb_model* cm, const nvdb_camera* cam, nvdb_precision prec, float* d_image,
                                   nvdb_stream stream) {
  const Range range("nvdb_render");
  if (!cm || !cam || !d_image || cam->width <= 0 || cam->height <= 0 || !(cam->step > 0.f) || cam->max_steps < 0 ||
      !(cam->fov_deg > 0.f && cam->fov_deg < 180.f) || !(cam->sigma >= 0.f))
    return fail(NVDB_ERR_INVALID_ARG, "nvdb_render: bad arguments");
  if (!eval_prec_ok(prec)) return fail(NVDB_ERR_UNSUPPORTED, "precision %d", (int)prec);
  cudaStream_t s = (cudaStream_t)stream;
  // camera basis in FP64, film extent folded into right / up
  double f[3], r[3], u[3];
  double nf = 0.0;
  for (int a = 0; a < 3; ++a) { f[a] = (double)cam->target[a] - cam->eye[a]; nf += f[a] * f[a]; }
  if (!(nf > 0.0)) return fail(NVDB_ERR_INVALID_ARG, "nvdb_render: eye == target");
  for (auto& v : f) v /= std::sqrt(nf);
  r[0] = f[1] * cam->up[2] - f[2] * cam->up[1];
  r[1] = f[2] * cam->up[0] - f[0] * cam->up[2];
  r[2] = f[0] * cam->up[1] - f[1] * cam->up[0];
  const double nr = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
  if (!(nr > 1e-12)) return fail(NVDB_ERR_INVALID_ARG, "nvdb_render: up parallel to the view axis");
  for (auto& v : r) v /= nr;
  u[0] = r[1] * f[2] - r[2] * f[1];
  u[1] = r[2] * f[0] - r[0] * f[2];
  u[2] = r[0] * f[1] - r[1] * f[0];
  const double th = std::tan(cam->fov_deg * M_PI / 360.0), aspect = (double)cam->width / cam->height;
  RayCam c{};
  for (int a = 0; a < 3; ++a) {
    c.eye[a] = cam->eye[a];
    c.fwd[a] = (float)f[a];
    c.right[a] = (float)(r[a] * th * aspect);
    c.up[a] = (float)(u[a] * th);
    c.lo[a] = (float)cm->origin[a];
    c.hi[a] = (float)(cm->origin[a] + (1 << cm->log2e));
  }
  c.width = cam->width;
  c.height = cam->height;
  c.max_steps = cam->max_steps;
  c.step = cam->step;
  c.sigma = cam->sigma;
  const int64_t nray = (int64_t)cam->width * cam->height;
  KLAUNCH("ray_init", s, ray_init_kernel<<<blocks_for(nray, 256), 256, 0, s>>>(nray, d_image));
  const int ns = (int)std::max<int64_t>(1, std::min<int64_t>(cam->max_steps, (1 << 22) / std::max<int64_t>(nray, 1)));
  float *xyz = nullptr, *dens = nullptr;
  auto run = [&]() -> nvdb_status {
    TRY(dalloc(&xyz, (size_t)nray * ns * 3));
    TRY(dalloc(&dens, (size_t)nray * ns));
    for (int s0 = 0; s0 < cam->max_steps; s0 += ns) {
      const int k = std::min(ns, cam->max_steps - s0);
      KLAUNCH("ray_points", s, ray_points_kernel<<<blocks_for(nray * k, 256), 256, 0, s>>>(c, s0, k, xyz));
      TRY(nvdb_query(cm, xyz, nray * k, prec, dens, nullptr, stream));
      KLAUNCH("ray_accum", s, ray_accum_kernel<<<blocks_for(nray, 128), 128, 0, s>>>(c, k, dens, d_image));
      CU(cudaGetLastError());
    }
    CU(cudaStreamSynchronize(s));
    return NVDB_OK;
  };
  const nvdb_status st = run();
  cudaStreamSynchronize(s);
  dfree(xyz);
  dfree(dens);
  return st;
}

// ============================================================================ network-level calls
extern "C" nvdb_status nvdb_mlp_eval(const nvdb_model* m, int net, nvdb_precision prec, const int32_t* d_ijk,
                                     int64_t n, float* d_out, nvdb_stream stream) {
  if (!m || net < 0 || net >= m->n_net() || n < 0 || (n > 0 && (!d_ijk || !d_out)))
    return fail(NVDB_ERR_INVALID_ARG, "nvdb_mlp_eval: bad arguments");
  TRY(check_eval_prec(m, net, prec));
  EvalJob j{};
  j.mode = MODE_LIST;
  j.ijk = d_ijk;
  j.n_items = n;
  j.shift = m->net_level(net) ? 3 : 0;
  j.out = d_out;
  j.scale = 1.f;
  cudaStream_t s = (cudaStream_t)stream;
  if (prec != NVDB_FP32) CU(cudaMemsetAsync(m->status, 0, 4, s));
  TRY(launch_eval(m, net, prec, j, s));
  return eval_status(m, prec, s);
}

extern "C" int64_t nvdb_net_param_count(const nvdb_model* m, int net) {
  if (!m || net < 0 || net >= m->n_net()) return -1;
  return m->net[net].P;
}

extern "C" nvdb_status nvdb_mlp_grad(const nvdb_model* cm, int net, nvdb_precision prec, const int32_t* d_ijk,
                                     const float* d_target, int64_t n, int loss_kind, float* d_grad, float* loss,
                                     nvdb_stream stream) {
  if (!cm || net < 0 || net >= cm->n_net() || n <= 0 || !d_ijk || !d_target || !d_grad)
    return fail(NVDB_ERR_INVALID_ARG, "nvdb_mlp_grad: bad arguments");
  if (!train_prec_ok(prec)) return fail(NVDB_ERR_UNSUPPORTED, "nvdb_mlp_grad: precision %d", (int)prec);
  if (loss_kind < 0 || loss_kind > NVDB_LOSS_CE) return fail(NVDB_ERR_INVALID_ARG, "unknown loss %d", loss_kind);
  if (n >= (1ll << 31)) return fail(NVDB_ERR_UNSUPPORTED, "nvdb_mlp_grad: n >= 2^31");
  nvdb_model* m = const_cast<nvdb_model*>(cm);
  if ((m->net[net].n_out == 3) != (loss_kind == NVDB_LOSS_CE))
    return fail(NVDB_ERR_INVALID_ARG, "nvdb_mlp_grad: the ternary classifier takes NVDB_LOSS_CE, other networks not");
  cudaStream_t s = (cudaStream_t)stream;
  const DevNet& d = m->net[net];
  const int grid = train_grid(n);
  TRY(ensure_partial(m, (int64_t)grid * (d.P + 1)));
  CU(cudaMemsetAsync(m->status, 0, 4, s));   // this call's device-side errors only
  TrainJob j{};
  j.net = m->tile_net(net) ? 3 : net % 3;
  j.stream = net;
  j.loss = loss_kind;
  j.step = 1;
  j.batch = n;
  j.ijk_list = d_ijk;
  j.target_list = d_target;
  j.partial = m->partial;
  TRY(launch_train(m, net, prec, j, grid, s));
  float* d_loss = nullptr;
  TRY(dalloc(&d_loss, 1));
  KLAUNCH("adam_reduce", s, adam_reduce_kernel<<<blocks_for(d.P + 1, 32), 32 * kRedGroups, 0, s>>>(m->partial, grid, d.P, nullptr, nullptr, nullptr, 1, 0.f,
                                                              d_grad, d_loss, 1.f / (float)n, adam_aux(d, prec, false),
                                                              AdamSched{}));
  float h = 0.f;
  cudaError_t e = cudaMemcpyAsync(&h, d_loss, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  dfree(d_loss);
  if (e != cudaSuccess) return fail(NVDB_ERR_CUDA, "nvdb_mlp_grad: %s", cudaGetErrorString(e));
  if (prec == NVDB_BF16 || loss_kind == NVDB_LOSS_CE) {   // timed-out waits; targets that are not classes
    uint32_t hst = 0;
    TRY(read_status(m->status, s, &hst));
    if (hst & ST_RANGE) return fail(NVDB_ERR_INVALID_ARG, "nvdb_mlp_grad: a target is not a class (0, 1 or 2)");
    TRY(status_to_error(hst));
  }
  if (loss) *loss = h;
  return NVDB_OK;
}

// ============================================================================ fault injection (tests)
namespace {
// Floats of the allocation-free gradient's static scratch array (nvdb_mlp_grad_static).
constexpr int64_t kStaticGradFloats = 1 << 20;
// Test hook (nvdb_debug_inject, NVDB_INJECT_STATIC_LIMIT): use only this many floats of the
// array, so that the capacity check can be exercised with networks of supported shapes.
std::atomic<int64_t> g_static_limit{kStaticGradFloats};

// A kernel that waits on an mbarrier phase nothing completes, bounded by limit_ns.
__global__ void wait_selftest_kernel(int64_t limit_ns, uint32_t* status) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  const uint64_t t0 = global_ns();
  bool done = false;
  while (!done && global_ns() - t0 < (uint64_t)limit_ns) done = mbar_try_wait(&bar, 0);
  if (!done && threadIdx.x == 0) set_status(status, ST_TIMEOUT);
}
}  // namespace

extern "C" nvdb_status nvdb_debug_inject(int what, int64_t value) {
  if (what == NVDB_INJECT_WAIT_TIMEOUT) {
    const int v = value != 0 ? 1 : 0;
    for (FailWaitsSetter set : fail_waits_setters()) CU(set(v));
    return NVDB_OK;
  }
  if (what == NVDB_INJECT_STATIC_LIMIT) {
    if (value < 0 || value > kStaticGradFloats) return fail(NVDB_ERR_INVALID_ARG, "nvdb_debug_inject: static limit");
    g_static_limit.store(value > 0 ? value : kStaticGradFloats);
    return NVDB_OK;
  }
  if (what == NVDB_INJECT_FUSED_ADAM) {
    g_fused_override.store(value < 0 ? -1 : (value != 0 ? 1 : 0));
    return NVDB_OK;
  }
  if (what == NVDB_INJECT_ALLOC_BUDGET) {
    if (value < 0) return fail(NVDB_ERR_INVALID_ARG, "nvdb_debug_inject: negative budget");
    g_alloc_budget.store(value > 0 ? value : -1);
    return NVDB_OK;
  }
  return fail(NVDB_ERR_INVALID_ARG, "nvdb_debug_inject: unknown injection %d", what);
}

extern "C" nvdb_status nvdb_debug_wait_selftest(int64_t limit_ns) {
  if (limit_ns <= 0 || limit_ns > (int64_t)kWaitLimitNs) return fail(NVDB_ERR_INVALID_ARG, "limit_ns in (0, 1 s]");
  uint32_t* st = nullptr;
  TRY(dalloc(&st, 1));
  uint32_t h = 0;
  cudaError_t e = cudaMemset(st, 0, 4);
  if (e == cudaSuccess) {
    wait_selftest_kernel<<<1, 32>>>(limit_ns, st);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(&h, st, 4, cudaMemcpyDeviceToHost);
  dfree(st);
  if (e != cudaSuccess) return fail(NVDB_ERR_CUDA, "nvdb_debug_wait_selftest: %s", cudaGetErrorString(e));
  return status_to_error(h);
}

// ============================================================================ parameters (autograd)
extern "C" nvdb_status nvdb_net_params(const nvdb_model* m, int net, float* d_out, nvdb_stream stream) {
  if (!m || net < 0 || net >= m->n_net() || !d_out) return fail(NVDB_ERR_INVALID_ARG, "nvdb_net_params: bad arguments");
  const DevNet& d = m->net[net];
  CU(cudaMemcpyAsync(d_out, d.p32, d.P * 4, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  return NVDB_OK;
}

extern "C" nvdb_status nvdb_net_set_params(nvdb_model* m, int net, const float* d_in, nvdb_stream stream) {
  if (!m || net < 0 || net >= m->n_net() || !d_in) return fail(NVDB_ERR_INVALID_ARG, "nvdb_net_set_params: bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  DevNet& d = m->net[net];
  CU(cudaMemcpyAsync(d.p32, d_in, d.P * 4, cudaMemcpyDeviceToDevice, s));
  d.bf16_exact = false;
  TRY(pack_net(m, net, s));
  TRY(upload_views(m, s));
  // the patches and the decoded topology belonged to the old weights
  for (auto& p : m->patches) p.release();
  m->patches.clear();
  m->qc.release();
  return NVDB_OK;
}

extern "C" nvdb_status nvdb_model_repatch(nvdb_model* m, const nvdb_grid* g, uint32_t patch_precs, nvdb_stream stream) {
  if (!m || !g) return fail(NVDB_ERR_INVALID_ARG, "nvdb_model_repatch: NULL argument");
  if (patch_precs >> kNumPrecisions) return fail(NVDB_ERR_INVALID_ARG, "patch_precs: no precision %u", patch_precs);
  if (g->n_l1 != m->n_l1 || g->n_leaf != m->n_leaf || g->n != m->n_active || g->log2e != m->log2e ||
      g->origin[0] != m->origin[0] || g->origin[1] != m->origin[1] || g->origin[2] != m->origin[2])
    return fail(NVDB_ERR_INVALID_ARG, "nvdb_model_repatch: the grid is not the one the model encodes");
  if (g->n_tiles != m->n_tiles) return fail(NVDB_ERR_INVALID_ARG, "nvdb_model_repatch: the grid's tiles differ");
  for (int p = 0; p < kNumPrecisions; ++p)
    if (patch_precs & (1u << p)) TRY(check_eval_prec(m, 1, (nvdb_precision)p));
  cudaStream_t s = (cudaStream_t)stream;
  m->qc.release();
  CU(cudaMemsetAsync(m->status, 0, 4, s));
  for (int p = 0; p < kNumPrecisions; ++p)
    if (patch_precs & (1u << p)) TRY(make_patches(m, g, p, s));
  uint32_t hst = 0;
  TRY(read_status(m->status, s, &hst));
  return status_to_error(hst);
}

// ============================================================================ info / export / import
extern "C" nvdb_status nvdb_model_info(const nvdb_model* m, nvdb_info* out) {
  if (!m || !out) return fail(NVDB_ERR_INVALID_ARG, "nvdb_model_info: NULL");
  out->grid_class = m->grid_class;
  out->background = m->background;
  out->half_width = m->half_width;
  for (int d = 0; d < 3; ++d) out->origin[d] = m->origin[d];
  out->log2_extent = m->log2e;
  out->n_active = m->n_active;
  out->n_leaf = m->n_leaf;
  out->n_l1 = m->n_l1;
  out->n_l2 = m->n_l2;
  out->n_experts = m->n_exp;
  out->subdomain = m->sub_size;
  out->n_tiles = m->n_tiles;
  return NVDB_OK;
}

namespace {
struct BlobHeader {
  char magic[8];
  uint32_t version, grid_class;
  float background, half_width;
  int32_t origin[3], log2_extent, ffm_size[2], width[3], layers[3], n_patch_sets, reserved0;
  int64_t n_l2, n_l1, n_leaf, n_active;
  uint64_t reserved1[2];
};
static_assert(sizeof(BlobHeader) == 128, "blob header is 128 bytes");

// Version 3 extension, after the header: ternary level 1 with a tile value regressor, and the
// hidden activation.
struct BlobExt {
  int32_t flags;         // bit 0: ternary level-1 classifier + tile value regressor (net 3)
  int32_t activation;    // 0 ReLU, 1 sin
  float omega;
  int32_t tile_width, tile_layers, reserved;
  int64_t n_tiles;
};
static_assert(sizeof(BlobExt) == 32, "blob extension is 32 bytes");

struct Writer {
  std::vector<uint8_t> b;
  void put(const void* p, size_t n) {
    const uint8_t* c = static_cast<const uint8_t*>(p);
    b.insert(b.end(), c, c + n);
  }
  void pad() { b.resize((b.size() + 7) & ~(size_t)7, 0); }
};

struct Reader {
  const uint8_t* p;
  size_t n, o = 0;
  bool ok = true;
  const void* take(size_t bytes) {
    if (!ok || o + bytes > n) { ok = false; return nullptr; }
    const void* r = p + o;
    o += bytes;
    return r;
  }
  void pad() { o = (o + 7) & ~(size_t)7; }
};
}  // namespace

extern "C" nvdb_status nvdb_model_export(const nvdb_model* m, void* buf, size_t* bytes) {
  if (!m || !bytes) return fail(NVDB_ERR_INVALID_ARG, "nvdb_model_export: NULL");
  Writer w;
  BlobHeader h{};
  std::memcpy(h.magic, "NVDBMDL1", 8);
  const bool ext = m->ternary || m->act != 0;
  h.version = ext ? 3 : (m->moe() ? 2 : 1);   // 2: the domain decomposition; 3: the extension
  h.grid_class = (uint32_t)m->grid_class;
  h.background = m->background;
  h.half_width = m->half_width;
  for (int d = 0; d < 3; ++d) h.origin[d] = m->origin[d];
  h.log2_extent = m->log2e;
  h.ffm_size[0] = m->ffm[0];
  h.ffm_size[1] = m->ffm[1];
  for (int k = 0; k < 3; ++k) { h.width[k] = m->width[k]; h.layers[k] = m->layers[k]; }
  h.n_patch_sets = (int32_t)m->patches.size();
  h.n_l2 = m->n_l2; h.n_l1 = m->n_l1; h.n_leaf = m->n_leaf; h.n_active = m->n_active;
  if (m->moe()) {
    h.reserved0 = m->n_exp;
    h.reserved1[0] = (uint64_t)m->sub_size;
    h.reserved1[1] = (uint64_t)m->sub_halo;
  }
  w.put(&h, sizeof h);
  if (ext) {
    BlobExt e{};
    e.flags = m->ternary ? 1 : 0;
    e.activation = m->act;
    e.omega = m->omega;
    e.tile_width = m->ternary ? m->tile_width : 0;
    e.tile_layers = m->ternary ? m->tile_layers : 0;
    e.n_tiles = m->n_tiles;
    w.put(&e, sizeof e);
  }
  for (int lev = 0; lev < 2; ++lev) { w.put(m->q_host[lev].data(), m->q_host[lev].size() * 4); w.pad(); }
  CU(cudaDeviceSynchronize());
  for (int k = 0; k < m->n_net(); ++k) {
    std::vector<float> p(m->net[k].P);
    CU(cudaMemcpy(p.data(), m->net[k].p32, p.size() * 4, cudaMemcpyDeviceToHost));
    w.put(p.data(), p.size() * 4);
    w.pad();
  }
  if (m->moe()) {
    const int32_t dims[3] = {m->sub_dims, m->sub_dims, m->sub_dims};
    w.put(dims, sizeof dims); w.pad();
    w.put(m->expert_of_host.data(), m->expert_of_host.size() * 4); w.pad();
    w.put(m->exp_origin_host.data(), m->exp_origin_host.size() * 4); w.pad();
  }
  w.put(m->l2_origin_host.data(), m->l2_origin_host.size() * 4); w.pad();
  w.put(m->l2_mask_host.data(), m->l2_mask_host.size() * 8); w.pad();
  std::vector<const PatchSet*> sets;
  for (auto& p : m->patches) sets.push_back(&p);
  std::sort(sets.begin(), sets.end(), [](const PatchSet* a, const PatchSet* b) { return a->prec < b->prec; });
  for (const PatchSet* p : sets) {
    const int32_t hdr[2] = {p->prec, 0};
    w.put(hdr, 8);
    const int64_t nitem[2] = {m->n_l1, m->n_leaf}, npatch[2] = {p->n1, p->n0};
    const uint32_t* doff[2] = {p->d_l1_off, p->d_l0_off};
    const uint16_t* didx[2] = {p->d_l1_idx, p->d_l0_idx};
    for (int lev = 0; lev < 2; ++lev) {
      std::vector<uint32_t> off((size_t)nitem[lev] + 1);
      std::vector<uint16_t> idx((size_t)npatch[lev]);
      CU(cudaMemcpy(off.data(), doff[lev], off.size() * 4, cudaMemcpyDeviceToHost));
      if (!idx.empty()) CU(cudaMemcpy(idx.data(), didx[lev], idx.size() * 2, cudaMemcpyDeviceToHost));
      w.put(off.data(), off.size() * 4); w.pad();
      w.put(idx.data(), idx.size() * 2); w.pad();
    }
  }
  if (!buf) { *bytes = w.b.size(); return NVDB_OK; }
  if (*bytes < w.b.size()) { *bytes = w.b.size(); return fail(NVDB_ERR_CAPACITY, "nvdb_model_export: buffer too small"); }
  std::memcpy(buf, w.b.data(), w.b.size());
  *bytes = w.b.size();
  return NVDB_OK;
}

extern "C" nvdb_status nvdb_model_import(const void* buf, size_t bytes, nvdb_stream stream, nvdb_model** out) {
  if (!buf || !out) return fail(NVDB_ERR_INVALID_ARG, "nvdb_model_import: NULL");
  *out = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  Reader r{static_cast<const uint8_t*>(buf), bytes};
  const BlobHeader* h = static_cast<const BlobHeader*>(r.take(sizeof(BlobHeader)));
  if (!h || std::memcmp(h->magic, "NVDBMDL1", 8) != 0 || h->version < 1 || h->version > 3)
    return fail(NVDB_ERR_CORRUPT, "not an NVDBMDL1 blob");
  const bool moe = h->version == 2 || (h->version == 3 && h->reserved0 > 0);
  const BlobExt* ex = h->version == 3 ? static_cast<const BlobExt*>(r.take(sizeof(BlobExt))) : nullptr;
  if (h->version == 3 && (!ex || (ex->flags & ~1) || ex->activation < 0 || ex->activation > 1 ||
                          (ex->activation == 1 && !(ex->omega > 0.f)) || ex->n_tiles < 0 ||
                          ((ex->flags & 1) && (moe || ex->n_tiles == 0))))
    return fail(NVDB_ERR_CORRUPT, "bad blob extension");
  if (moe && (h->reserved0 < 1 || h->reserved0 > (1 << 20) || h->reserved1[0] == 0 || h->reserved1[0] % 512 ||
              h->reserved1[1] < 8 || (h->reserved1[1] & (h->reserved1[1] - 1)) || 4 * h->reserved1[1] > h->reserved1[0]))
    return fail(NVDB_ERR_CORRUPT, "bad decomposition header");
  if (h->n_l2 < 0 || h->n_l1 < 0 || h->n_leaf < 0 || h->n_active < 0 || h->n_patch_sets < 0 || h->n_patch_sets > kNumPrecisions ||
      h->grid_class > 1 || h->log2_extent < 0 || h->log2_extent > 21)
    return fail(NVDB_ERR_CORRUPT, "bad blob header");
  auto* m = new nvdb_model();
  auto run = [&]() -> nvdb_status {
    m->grid_class = (int)h->grid_class;
    m->background = h->background;
    m->half_width = h->half_width;
    for (int d = 0; d < 3; ++d) m->origin[d] = h->origin[d];
    m->log2e = h->log2_extent;
    m->ffm[0] = h->ffm_size[0];
    m->ffm[1] = h->ffm_size[1];
    for (int k = 0; k < 3; ++k) { m->width[k] = h->width[k]; m->layers[k] = h->layers[k]; }
    m->n_l2 = h->n_l2; m->n_l1 = h->n_l1; m->n_leaf = h->n_leaf; m->n_active = h->n_active;
    if (ex) {
      m->act = ex->activation;
      m->omega = ex->activation ? ex->omega : 1.f;
      m->n_tiles = ex->n_tiles;
      m->tile_width = ex->tile_width;
      m->tile_layers = ex->tile_layers;
      if (ex->flags & 1) m->set_ternary(true);
    }
    TRY(check_model_shapes(m));
    TRY(dalloc(&m->status, 1));
    CU(cudaMemsetAsync(m->status, 0, 4, s));
    for (int lev = 0; lev < 2; ++lev) {
      const size_t cnt = (size_t)(m->ffm[lev] / 2) * 3;
      const uint32_t* q = static_cast<const uint32_t*>(r.take(cnt * 4));
      r.pad();
      if (!q) return fail(NVDB_ERR_CORRUPT, "blob truncated (Fourier matrix)");
      m->q_host[lev].assign(q, q + cnt);
      TRY(dalloc(&m->q_dev[lev], cnt));
      CU(cudaMemcpy(m->q_dev[lev], q, cnt * 4, cudaMemcpyHostToDevice));
    }
    if (moe) {
      if (m->ternary) return fail(NVDB_ERR_CORRUPT, "tiles with a decomposition");
      m->set_experts((int)h->reserved0);
      m->sub_size = (int)h->reserved1[0];
      m->sub_halo = (int)h->reserved1[1];
    }
    for (int k = 0; k < m->n_net(); ++k) {
      int nin, w, L, nout;
      net_shape(m, k, nin, w, L, nout);
      const int64_t P = net_param_count(nin, w, L, nout);
      const float* p = static_cast<const float*>(r.take((size_t)P * 4));
      r.pad();
      if (!p) return fail(NVDB_ERR_CORRUPT, "blob truncated (network %d)", k);
      std::vector<float> tmp(p, p + P);
      TRY(upload_net(m, k, tmp.data(), s));
      m->net[k].bf16_exact = bf16_exact_layers(tmp.data(), P - (int64_t)nout * (w + 1));
      CU(cudaStreamSynchronize(s));
    }
    if (moe) {   // grid of subdomains and expert origins (Section 3.4)
      const int32_t* dims = static_cast<const int32_t*>(r.take(12));
      r.pad();
      if (!dims) return fail(NVDB_ERR_CORRUPT, "blob truncated (decomposition)");
      const int n = dims[0];
      const int64_t need = (int64_t)1 << (m->log2e);
      if (n < 1 || dims[1] != n || dims[2] != n || (int64_t)n * m->sub_size < need || (int64_t)(n - 1) * m->sub_size >= need)
        return fail(NVDB_ERR_CORRUPT, "bad subdomain grid");
      m->sub_dims = n;
      const int32_t* eo = static_cast<const int32_t*>(r.take((size_t)n * n * n * 4));
      r.pad();
      const int32_t* og = static_cast<const int32_t*>(r.take((size_t)m->n_exp * 12));
      r.pad();
      if (!eo || !og) return fail(NVDB_ERR_CORRUPT, "blob truncated (decomposition)");
      m->expert_of_host.assign(eo, eo + (size_t)n * n * n);
      m->exp_origin_host.assign(og, og + 3 * (size_t)m->n_exp);
      std::vector<int> seen(m->n_exp, 0);
      for (size_t c = 0; c < m->expert_of_host.size(); ++c) {   // every expert once, at its own subdomain
        const int e = m->expert_of_host[c];
        if (e < -1 || e >= m->n_exp) return fail(NVDB_ERR_CORRUPT, "bad expert id");
        if (e < 0) continue;
        const int32_t want[3] = {(int32_t)(c / ((size_t)n * n)) * m->sub_size, (int32_t)((c / n) % n) * m->sub_size,
                                 (int32_t)(c % n) * m->sub_size};
        if (seen[e]++ || std::memcmp(want, &m->exp_origin_host[3 * e], 12) != 0)
          return fail(NVDB_ERR_CORRUPT, "expert table inconsistent");
      }
      for (int e = 0; e < m->n_exp; ++e)
        if (!seen[e]) return fail(NVDB_ERR_CORRUPT, "expert %d has no subdomain", e);
      TRY(upload_moe(m, s));
    }
    for (int k = 0; k < m->n_net(); ++k) TRY(pack_net(m, k, s));
    TRY(upload_views(m, s));
    const int32_t* l2o = static_cast<const int32_t*>(r.take((size_t)m->n_l2 * 12));
    r.pad();
    const uint64_t* l2m = static_cast<const uint64_t*>(r.take((size_t)m->n_l2 * 4096));
    r.pad();
    if (!r.ok) return fail(NVDB_ERR_CORRUPT, "blob truncated (upper tree)");
    m->l2_origin_host.assign(l2o, l2o + 3 * m->n_l2);
    m->l2_mask_host.assign(l2m, l2m + 512 * m->n_l2);
    std::vector<int4> o4(m->n_l2);
    for (int64_t i = 0; i < m->n_l2; ++i) o4[i] = make_int4(l2o[3 * i], l2o[3 * i + 1], l2o[3 * i + 2], 0);
    TRY(dalloc(&m->l2_origin, m->n_l2));
    TRY(dalloc(&m->l2_mask, 512 * m->n_l2));
    if (m->n_l2) {
      CU(cudaMemcpy(m->l2_origin, o4.data(), m->n_l2 * sizeof(int4), cudaMemcpyHostToDevice));
      CU(cudaMemcpy(m->l2_mask, l2m, m->n_l2 * 4096, cudaMemcpyHostToDevice));
    }
    for (int i = 0; i < h->n_patch_sets; ++i) {
      const int32_t* ph = static_cast<const int32_t*>(r.take(8));
      if (!ph) return fail(NVDB_ERR_CORRUPT, "blob truncated (patch header)");
      PatchSet ps;
      ps.prec = ph[0];
      if (!eval_prec_ok(ps.prec) || m->patch_set((nvdb_precision)ps.prec) ||
          (m->act != 0 && (ps.prec == NVDB_FP8_E4M3 || (m->moe() && ps.prec != NVDB_FP32))))
        return fail(NVDB_ERR_CORRUPT, "patch set %d: bad or repeated precision %d", i, ps.prec);
      // both levels: offsets and indices straight from the blob to the device; the
      // offsets (monotone, from 0 to the patch count) and the index ranges are checked
      // on the device before the model is returned
      const int64_t nitem[2] = {m->n_l1, m->n_leaf};
      for (int lev = 0; lev < 2; ++lev) {
        const uint32_t* o = static_cast<const uint32_t*>(r.take((size_t)(nitem[lev] + 1) * 4));
        r.pad();
        const int64_t n = o ? o[nitem[lev]] : 0;
        const uint16_t* ix = o ? static_cast<const uint16_t*>(r.take((size_t)n * 2)) : nullptr;
        r.pad();
        if (!o || (!ix && n)) {
          ps.release();
          return fail(NVDB_ERR_CORRUPT, "blob truncated (patches)");
        }
        uint32_t*& doff = lev == 0 ? ps.d_l1_off : ps.d_l0_off;
        uint16_t*& didx = lev == 0 ? ps.d_l1_idx : ps.d_l0_idx;
        (lev == 0 ? ps.n1 : ps.n0) = n;
        nvdb_status ast = dalloc(&doff, (size_t)nitem[lev] + 1);
        if (ast == NVDB_OK) ast = dalloc(&didx, (size_t)n + 1);
        if (ast != NVDB_OK) { ps.release(); return ast; }
        if (cudaMemcpyAsync(doff, o, (nitem[lev] + 1) * 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            (n && cudaMemcpyAsync(didx, ix, n * 2, cudaMemcpyHostToDevice, s) != cudaSuccess)) {
          ps.release();
          return fail(NVDB_ERR_CUDA, "patch upload");
        }
        const int64_t work = std::max<int64_t>(nitem[lev] + 1, std::min<int64_t>(n, 1 << 22));
        // ternary level 1: entries slot | class << 12 with class <= 2
        const uint32_t lim = lev == 0 ? (m->ternary ? 3u * 4096u : 4096u) : 512u;
        KLAUNCH("check_patches", s, check_patches_kernel<<<blocks_for(work, 256), 256, 0, s>>>(
                                        doff, nitem[lev], didx, n, lim, m->status));
      }
      m->patches.push_back(ps);
    }
    uint32_t hst = 0;
    TRY(read_status(m->status, s, &hst));
    if (hst & ST_CORRUPT) return fail(NVDB_ERR_CORRUPT, "patch offsets or indices out of range");
    return status_to_error(hst);
  };
  const nvdb_status st = run();
  if (st != NVDB_OK) { delete m; return st; }
  *out = m;
  return NVDB_OK;
}

extern "C" nvdb_status nvdb_model_free(nvdb_model* m) {
  delete m;
  return NVDB_OK;
}

extern "C" const char* nvdb_last_error(void) { return g_err.c_str(); }

extern "C" void nvdb_profile_enable(int on) { prof::g_on.store(on != 0); }

extern "C" int64_t nvdb_launch_count(void) { return (int64_t)prof::g_launches.load(); }

extern "C" int nvdb_profile_read(char* names, int name_len, int64_t* launches, double* ms, int cap) {
  std::map<std::string, std::pair<int64_t, double>> agg;
  std::vector<prof::Rec> recs;
  {
    std::lock_guard<std::mutex> lk(prof::g_mu);
    recs.swap(prof::g_recs);
  }
  for (auto& r : recs) {
    float t = 0.f;
    cudaEventSynchronize(r.b);
    cudaEventElapsedTime(&t, r.a, r.b);
    auto& e = agg[r.name];
    e.first += 1;
    e.second += t;
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  int i = 0;
  for (auto& kv : agg) {
    if (i < cap) {
      if (names && name_len > 0) {
        std::strncpy(names + (size_t)i * name_len, kv.first.c_str(), name_len - 1);
        names[(size_t)i * name_len + name_len - 1] = 0;
      }
      if (launches) launches[i] = kv.second.first;
      if (ms) ms[i] = kv.second.second;
    }
    ++i;
  }
  return i;
}

// ============================================================================ allocation-free gradient
// nvdb_mlp_grad computes its per-CTA gradient partials in device memory that
// the model allocates with cudaMalloc on first use.  nvdb_mlp_grad_static is
// the same computation for callers that must not allocate: its partials and
// loss live in the file-scope array below (4 MiB, present on every device that
// loads this library for as long as the library stays loaded).
namespace {
static __device__ __align__(256) float g_grad_scratch[kStaticGradFloats];

template <int NIN, int W>
nvdb_status launch_train_static(const NetView& nv, const TrainJob& job, int grid, cudaStream_t s) {
  const size_t smem = TrainSmem<NIN, W>::bytes(nv.layers);
  TRY(set_smem_limit((const void*)train_fwd_bwd_kernel<NIN, W>, smem));
  KLAUNCH("train_fwd_bwd", s, train_fwd_bwd_kernel<NIN, W><<<grid, kTile, smem, s>>>(nv, job));
  CU(cudaGetLastError());
  return NVDB_OK;
}
}  // namespace

extern "C" nvdb_status nvdb_mlp_grad_static(const nvdb_model* m, int net, const int32_t* d_ijk, const float* d_target,
                                            int64_t n, int loss_kind, float* d_grad, float* loss, nvdb_stream stream) {
  if (!m || net < 0 || net >= m->n_net() || n <= 0 || !d_ijk || !d_target || !d_grad)
    return fail(NVDB_ERR_INVALID_ARG, "nvdb_mlp_grad_static: bad arguments");
  if (loss_kind < 0 || loss_kind > 3) return fail(NVDB_ERR_INVALID_ARG, "unknown loss %d", loss_kind);
  if (n >= (1ll << 31)) return fail(NVDB_ERR_UNSUPPORTED, "nvdb_mlp_grad_static: n >= 2^31");
  const DevNet& d = m->net[net];
  if (d.n_out != 1) return fail(NVDB_ERR_UNSUPPORTED, "nvdb_mlp_grad_static: networks with one output only");
  // one CTA needs P + 1 floats of partials, plus one float for the loss
  const int64_t limit = g_static_limit.load();
  if (d.P + 2 > limit)
    return fail(NVDB_ERR_CAPACITY, "nvdb_mlp_grad_static: network %d has %lld parameters; the static scratch "
                "holds %lld floats (at most %lld parameters)", net, (long long)d.P, (long long)limit,
                (long long)(limit - 2));
  // The array's device address, looked up on every call with the caller's device current:
  // the lookup allocates nothing, and an address cached across a device reset (which reloads
  // the module) could be stale.
  void* sym = nullptr;
  const cudaError_t se = cudaGetSymbolAddress(&sym, g_grad_scratch);
  if (se != cudaSuccess)
    return fail(NVDB_ERR_CUDA, "cudaGetSymbolAddress(static gradient scratch): %s", cudaGetErrorString(se));
  float* scratch = static_cast<float*>(sym);
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t fit = (limit - 1) / (d.P + 1);
  const int grid = (int)std::min<int64_t>(std::min<int64_t>((n + kTile - 1) / kTile, num_sms()), fit);
  float* loss_slot = scratch + (limit - 1);
  TrainJob j{};
  j.net = m->tile_net(net) ? 3 : net % 3;
  j.stream = net;
  j.loss = loss_kind;
  j.step = 1;
  j.batch = n;
  j.ijk_list = d_ijk;
  j.target_list = d_target;
  j.partial = scratch;   // every CTA zeroes its own slot before accumulating
  const int ex = net / 3;   // an expert's network works relative to its subdomain origin
  j.ox = m->origin[0] + (m->moe() ? m->exp_origin_host[3 * ex] : 0);
  j.oy = m->origin[1] + (m->moe() ? m->exp_origin_host[3 * ex + 1] : 0);
  j.oz = m->origin[2] + (m->moe() ? m->exp_origin_host[3 * ex + 2] : 0);
  const NetView nv = net_view(m, net);
  if (nv.n_in == 32 && nv.width == 32) TRY((launch_train_static<32, 32>(nv, j, grid, s)));
  else if (nv.n_in == 32 && nv.width == 64) TRY((launch_train_static<32, 64>(nv, j, grid, s)));
  else if (nv.n_in == 64 && nv.width == 32) TRY((launch_train_static<64, 32>(nv, j, grid, s)));
  else if (nv.n_in == 64 && nv.width == 64) TRY((launch_train_static<64, 64>(nv, j, grid, s)));
  else return fail(NVDB_ERR_UNSUPPORTED, "network shape n=%d w=%d", nv.n_in, nv.width);
  KLAUNCH("adam_reduce", s, adam_reduce_kernel<<<blocks_for(d.P + 1, 32), 32 * kRedGroups, 0, s>>>(
                                scratch, grid, d.P, nullptr, nullptr, nullptr, 1, 0.f, d_grad, loss_slot,
                                1.f / (float)n, AdamAux{}, AdamSched{}));
  CU(cudaGetLastError());
  float h = 0.f;
  CU(cudaMemcpyAsync(&h, loss_slot, sizeof h, cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  if (loss) *loss = h;
  return NVDB_OK;
}

// ============================================================================ decode plans (CUDA graphs)
struct nvdb_plan {
  std::vector<nvdb_model*> models;
  nvdb_precision prec = NVDB_FP32;
  int32_t* ijk = nullptr;
  float* val = nullptr;
  std::vector<std::pair<int, int>> runs;
  std::vector<DecodeScratch*> scratch;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int occ = 0, variant = 1;
  float best_ms = 0.f;
  ~nvdb_plan() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    for (auto* d : scratch) delete d;
  }
};

namespace {
nvdb_status plan_run(nvdb_plan* p, cudaStream_t s) {
  int64_t base = 0;
  for (size_t i = 0; i < p->runs.size(); ++i) {
    const auto& r = p->runs[i];
    TRY(decode_batch(p->models.data() + r.first, r.second - r.first, p->prec, *p->scratch[i], p->ijk + 3 * base,
                     p->val + base, s));
    for (int m = r.first; m < r.second; ++m) base += p->models[m]->n_active;
  }
  return NVDB_OK;
}
}  // namespace

extern "C" nvdb_status nvdb_decompress_plan(const nvdb_model* const* models, int n_models, nvdb_precision prec,
                                            int32_t* d_ijk, float* d_val, int64_t capacity, nvdb_stream stream,
                                            nvdb_plan** out) {
  if (!out || !models || n_models <= 0 || !d_ijk || !d_val) return fail(NVDB_ERR_INVALID_ARG, "nvdb_decompress_plan: bad arguments");
  *out = nullptr;
  int64_t need = 0;
  for (int i = 0; i < n_models; ++i) {
    if (!models[i]) return fail(NVDB_ERR_INVALID_ARG, "nvdb_decompress_plan: NULL model");
    if (!models[i]->patch_set(prec)) return fail(NVDB_ERR_UNSUPPORTED, "model %d has no patch set for precision %d", i, (int)prec);
    TRY(check_eval_prec(models[i], 1, prec));
    need += models[i]->n_active;
  }
  if (need > capacity) return fail(NVDB_ERR_CAPACITY, "nvdb_decompress_plan: need %lld voxels, capacity %lld", (long long)need, (long long)capacity);
  cudaStream_t s = (cudaStream_t)stream;
  auto* p = new nvdb_plan();
  p->models.assign(const_cast<nvdb_model* const*>(models), const_cast<nvdb_model* const*>(models) + n_models);
  p->prec = prec;
  p->ijk = d_ijk;
  p->val = d_val;
  p->runs = batch_runs(models, n_models);
  for (size_t i = 0; i < p->runs.size(); ++i) p->scratch.push_back(new DecodeScratch());
  const bool prof_on = prof::g_on.exchange(false);
  auto run = [&]() -> nvdb_status {
    // autotune: tensor-core CTAs per SM, timing the whole decode (events on the stream)
    cudaEvent_t a, b;
    CU(cudaEventCreate(&a));
    CU(cudaEventCreate(&b));
    // candidates: kernel variant (0: 128 threads per tile, 1: 256 threads, split epilogue)
    // x tensor-core CTAs per SM (0 = the kernel's own limit)
    float best = 1e30f;
    int best_occ = 0, best_var = 1;
    const int occs[] = {0, 2, 3};
    for (int v = 0; v < kTcVariants; ++v)
      for (int c : occs) {
        if (prec == NVDB_FP32 && (c != 0 || v != 0)) continue;
        g_occ_override = c;
        g_variant_override = v;
        nvdb_status st = plan_run(p, s);                   // warm-up (and sizes the scratch)
        if (st == NVDB_OK) {
          cudaEventRecord(a, s);
          st = plan_run(p, s);
          cudaEventRecord(b, s);
        }
        g_occ_override = 0;
        g_variant_override = -1;
        TRY(st);
        CU(cudaEventSynchronize(b));
        float ms = 0.f;
        CU(cudaEventElapsedTime(&ms, a, b));
        if (ms < best) { best = ms; best_occ = c; best_var = v; }
      }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    for (auto* d : p->scratch) {
      uint32_t hst = 0;
      TRY(read_status(d->status, s, &hst));
      TRY(status_to_error(hst));
    }
    p->occ = best_occ;
    p->variant = best_var;
    p->best_ms = best;
    // capture the tuned decode into a graph, on a stream of our own (the caller's may be
    // the legacy default stream, which cannot be captured); the stream is idle here
    cudaStream_t cs = nullptr;
    CU(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    g_occ_override = best_occ;
    g_variant_override = best_var;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
    nvdb_status st = e == cudaSuccess ? plan_run(p, cs) : fail(NVDB_ERR_CUDA, "stream capture: %s", cudaGetErrorString(e));
    cudaGraph_t g = nullptr;
    if (e == cudaSuccess) e = cudaStreamEndCapture(cs, &g);
    g_occ_override = 0;
    g_variant_override = -1;
    cudaStreamDestroy(cs);
    TRY(st);
    if (e != cudaSuccess) return fail(NVDB_ERR_CUDA, "stream capture: %s", cudaGetErrorString(e));
    p->graph = g;
    CU(cudaGraphInstantiate(&p->exec, p->graph, 0));
    return NVDB_OK;
  };
  const nvdb_status st = run();
  prof::g_on.store(prof_on);
  if (st != NVDB_OK) { delete p; return st; }
  *out = p;
  return NVDB_OK;
}

extern "C" nvdb_status nvdb_plan_launch(nvdb_plan* p, nvdb_stream stream) {
  if (!p || !p->exec) return fail(NVDB_ERR_INVALID_ARG, "nvdb_plan_launch: NULL plan");
  CU(cudaGraphLaunch(p->exec, (cudaStream_t)stream));
  return NVDB_OK;
}

extern "C" nvdb_status nvdb_plan_check(nvdb_plan* p, nvdb_stream stream) {
  if (!p) return fail(NVDB_ERR_INVALID_ARG, "nvdb_plan_check: NULL plan");
  for (auto* d : p->scratch) {
    uint32_t hst = 0;
    TRY(read_status(d->status, (cudaStream_t)stream, &hst));
    TRY(status_to_error(hst));
  }
  return NVDB_OK;
}

extern "C" nvdb_status nvdb_plan_info(const nvdb_plan* p, int* tc_ctas_per_sm, int* tc_variant, float* tuned_ms) {
  if (!p) return fail(NVDB_ERR_INVALID_ARG, "nvdb_plan_info: NULL plan");
  if (tc_ctas_per_sm) *tc_ctas_per_sm = p->occ;
  if (tc_variant) *tc_variant = p->variant;
  if (tuned_ms) *tuned_ms = p->best_ms;
  return NVDB_OK;
}

extern "C" nvdb_status nvdb_plan_free(nvdb_plan* p) {
  delete p;
  return NVDB_OK;
}
