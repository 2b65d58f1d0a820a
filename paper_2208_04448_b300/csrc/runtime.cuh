// Host-side runtime shared by the translation units of libnvdb: error reporting,
// the device allocator with its injectable budget, per-launch tracing, shared-memory
// limits, and the per-precision network launchers that live in their own units
// (eval_*.cu, train_tc.cu) so the kernels compile in parallel.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "nvdb.h"
#include "mlp.cuh"
#include "train.cuh"

#include <nvtx3/nvToolsExt.h>

namespace nvdb {

// ---------------------------------------------------------------- errors
inline thread_local std::string g_err;

inline nvdb_status fail(nvdb_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

#define CU(call)                                                                                   \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess) {                                                                       \
      if (e_ == cudaErrorMemoryAllocation) return ::nvdb::fail(NVDB_ERR_OUT_OF_MEMORY, "%s: out of memory", #call); \
      return ::nvdb::fail(NVDB_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_));                 \
    }                                                                                              \
  } while (0)

#define TRY(expr)                         \
  do {                                    \
    nvdb_status s_ = (expr);              \
    if (s_ != NVDB_OK) return s_;         \
  } while (0)

// ---------------------------------------------------------------- allocation
// Test hook (nvdb_debug_inject): a budget of bytes for later device allocations.
inline std::atomic<int64_t> g_alloc_budget{-1};   // -1: none

// Take `bytes` from the injected budget (if one is set), or fail.
inline nvdb_status take_budget(int64_t bytes) {
  for (int64_t b = g_alloc_budget.load(); b >= 0;) {
    if (b < bytes) return fail(NVDB_ERR_OUT_OF_MEMORY, "device allocation of %lld bytes over the injected budget", (long long)bytes);
    if (g_alloc_budget.compare_exchange_weak(b, b - bytes)) break;
  }
  return NVDB_OK;
}

template <class T>
nvdb_status dalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) return NVDB_OK;
  const int64_t bytes = (int64_t)(count * sizeof(T));
  TRY(take_budget(bytes));
  CU(cudaMalloc((void**)p, count * sizeof(T)));
  return NVDB_OK;
}

template <class T>
void dfree(T*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}

constexpr size_t kSmemPerSm = 233472;   // shared memory per SM on sm_103 (228 KiB)

inline int num_sms() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

// Raise a kernel's dynamic shared-memory limit on the current device, once per size: the
// attribute call costs host time comparable to a launch, so repeated launches skip it.
inline nvdb_status set_smem_limit(const void* kernel, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, size_t> done;
  int dev = 0;
  CU(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  size_t& have = done[{kernel, dev}];
  if (bytes <= have) return NVDB_OK;
  CU(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  have = bytes;
  return NVDB_OK;
}

inline unsigned blocks_for(int64_t n, int per) { return (unsigned)((n + per - 1) / per); }

// ---------------------------------------------------------------- tracing
// Optional CUDA events around every kernel launch (on the launching stream)
// and a running count of launches; read back with nvdb_profile_read.
namespace prof {
inline std::atomic<long long> g_launches{0};
inline std::atomic<bool> g_on{false};
struct Rec {
  std::string name;
  cudaEvent_t a, b;
};
inline std::mutex g_mu;
inline std::vector<Rec> g_recs;
struct Scope {
  cudaEvent_t a = nullptr, b = nullptr;
  const char* name;
  cudaStream_t s;
  Scope(const char* n, cudaStream_t st) : name(n), s(st) {
    g_launches.fetch_add(1);
    if (g_on.load() && cudaEventCreate(&a) == cudaSuccess) {
      cudaEventCreate(&b);
      cudaEventRecord(a, s);
    }
  }
  ~Scope() {
    if (!a) return;
    cudaEventRecord(b, s);
    std::lock_guard<std::mutex> lk(g_mu);
    g_recs.push_back({name, a, b});
  }
};
}  // namespace prof

#define KLAUNCH(name, stream, ...)        \
  do {                                    \
    ::nvdb::prof::Scope prof_scope_(name, stream); \
    __VA_ARGS__;                          \
  } while (0)

inline const char* eval_name(const char* base, int mode) {
  static const char* names[5][3] = {{"mlp_f32.L1", "mlp_f32.L0", "mlp_f32.list"},
                                    {"mlp_bf16x3.L1", "mlp_bf16x3.L0", "mlp_bf16x3.list"},
                                    {"mlp_f16.L1", "mlp_f16.L0", "mlp_f16.list"},
                                    {"mlp_bf16.L1", "mlp_bf16.L0", "mlp_bf16.list"},
                                    {"mlp_fp8.L1", "mlp_fp8.L0", "mlp_fp8.list"}};
  const int b = std::strcmp(base, "mlp_bf16x3") == 0 ? 1
                : std::strcmp(base, "mlp_f16") == 0  ? 2
                : std::strcmp(base, "mlp_bf16") == 0 ? 3
                : std::strcmp(base, "mlp_fp8") == 0  ? 4
                                                     : 0;
  return names[b][mode];
}

// NVTX range over a C-ABI call or one of its stages (visible in Nsight timelines).
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};

// ---------------------------------------------------------------- wait-failure hook
// Every translation unit holds its own copy of the device flag g_fail_waits (there is no
// device linking); each registers a setter here, and nvdb_debug_inject calls them all.
using FailWaitsSetter = cudaError_t (*)(int);
inline std::vector<FailWaitsSetter>& fail_waits_setters() {
  static std::vector<FailWaitsSetter> v;
  return v;
}
static cudaError_t set_fail_waits_here(int v) { return cudaMemcpyToSymbol(g_fail_waits, &v, sizeof v); }
struct FailWaitsHook {
  explicit FailWaitsHook(FailWaitsSetter f) { fail_waits_setters().push_back(f); }
};
static FailWaitsHook g_fail_waits_hook(&set_fail_waits_here);

// ---------------------------------------------------------------- per-precision launchers
// Tensor-core CTAs per SM chosen by the decode-plan autotuner (0: from the kernel's limits).
inline int g_occ_override = 0;
// Tensor-core kernel variant: 0 = mlp_tc_kernel (128 threads per tile), 1 = mlp_tc2_kernel
// (256 threads per tile, split epilogue, origins staged by bulk copies), 2 = mlp_tc_kernel
// with origins staged by bulk copies.  -1: the default (0), which the environment variable
// NVDB_TC_VARIANT may set; the decode-plan autotuner overrides it.
constexpr int kTcVariants = 3;
inline int g_variant_override = -1;
inline int tc_variant() {
  if (g_variant_override >= 0) return g_variant_override;
  static const int v = [] {
    const char* e = std::getenv("NVDB_TC_VARIANT");
    return e && e[0] >= '0' && e[0] < '0' + kTcVariants ? e[0] - '0' : 0;
  }();
  return v;
}

// One launch of the fused encode + MLP kernel over a batch of items of one network shape
// (eval_f32.cu, eval_f16.cu, eval_bf16.cu, eval_bf16x3.cu, eval_fp8.cu).
nvdb_status launch_eval_f32(const EvalBatch& b, int64_t ntiles, cudaStream_t s);
nvdb_status launch_eval_f16(const EvalBatch& b, int64_t ntiles, cudaStream_t s);
nvdb_status launch_eval_bf16(const EvalBatch& b, int64_t ntiles, cudaStream_t s);
nvdb_status launch_eval_bf16x3(const EvalBatch& b, int64_t ntiles, cudaStream_t s);
nvdb_status launch_eval_fp8(const EvalBatch& b, int64_t ntiles, cudaStream_t s);
// Largest ReLU output per hidden layer over seeded lattice points (FP8 scale calibration).
nvdb_status launch_calib_amax(const NetView& nv, int log2_extent, uint64_t seed, int n, uint32_t* amax_bits,
                              cudaStream_t s);
// Radix sort of (key, index) pairs by the 63 key bits (sort.cu).
nvdb_status sort_keys(const uint64_t* k_in, uint64_t* k_out, const uint32_t* i_in, uint32_t* i_out, int n,
                      cudaStream_t s);
// One BF16 tensor-core training launch (train_tc.cu); with `fa`, the Adam update fused into the
// same (cooperative) launch.
nvdb_status launch_train_tc(const NetView& nv, const TrainJob& job, int grid, cudaStream_t s,
                            const FusedAdam* fa = nullptr);

// The training step's Adam update fused into its launch: off by default (measured slower: the
// fused tail has fewer threads to hide the reduction's latency, and cooperative launches keep
// the three networks' steps from overlapping); NVDB_FUSED_ADAM=1 or nvdb_debug_inject
// (NVDB_INJECT_FUSED_ADAM) turns it on where the device supports cooperative launches.
inline std::atomic<int> g_fused_override{-1};
inline bool fused_adam_enabled() {
  static const bool env = [] {
    const char* e = std::getenv("NVDB_FUSED_ADAM");
    return e && e[0] == '1';
  }();
  const int o = g_fused_override.load();
  if (!(o >= 0 ? o != 0 : env)) return false;
  int coop = 0, dev = 0;
  return cudaGetDevice(&dev) == cudaSuccess &&
         cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) == cudaSuccess && coop != 0;
}

}  // namespace nvdb
