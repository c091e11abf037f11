// dc_api.cu -- status strings, per-thread error messages and the allocation
// hook of the Defrise-Clack library.
#include <atomic>
#include <cstdio>
#include <mutex>
#include <string>
#include <vector>

#include "dc_common.cuh"

namespace dc {

static thread_local std::string g_last_error;

// Host-side fault injection for tests: when >= 0, the allocation with this
// ordinal (counted from the moment it was set) fails with cudaErrorMemoryAllocation.
static std::atomic<long> g_fail_alloc_after{-1};
static std::atomic<unsigned long long> g_launches{0};

void count_launch(unsigned n) { g_launches.fetch_add(n); }

// ---------------------------------------------------------------- profiler
namespace {
struct ProfRec {
  int kid;
  cudaEvent_t a, b;
};
std::mutex g_prof_mu;
std::atomic<int> g_prof_on{0};
std::vector<ProfRec> g_prof_recs;
std::vector<cudaEvent_t> g_prof_pool;
double g_prof_ms[KID_COUNT];
unsigned long long g_prof_n[KID_COUNT];

cudaEvent_t pool_get() {
  if (!g_prof_pool.empty()) {
    cudaEvent_t e = g_prof_pool.back();
    g_prof_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}
}  // namespace

ProfScope::ProfScope(int kid, cudaStream_t s) : slot(-1), st(s) {
  if (!g_prof_on.load(std::memory_order_relaxed)) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  ProfRec r{kid, pool_get(), pool_get()};
  if (!r.a || !r.b) return;
  cudaEventRecord(r.a, s);
  slot = (int)g_prof_recs.size();
  g_prof_recs.push_back(r);
}

ProfScope::~ProfScope() {
  if (slot < 0) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  cudaEventRecord(g_prof_recs[slot].b, st);
}

void set_error(const std::string &msg) { g_last_error = msg; }

int fail(int code, const std::string &msg) {
  set_error(msg);
  return code;
}

int cuda_fail(cudaError_t e, const char *what) {
  std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" +
                  cudaGetErrorString(e) + ")";
  set_error(m);
  return (e == cudaErrorMemoryAllocation) ? DC_ERR_OOM : DC_ERR_CUDA;
}

cudaError_t dmalloc(void **p, size_t bytes) {
  long n = g_fail_alloc_after.load();
  if (n >= 0) {
    if (n == 0) {
      g_fail_alloc_after.store(-1);
      *p = nullptr;
      return cudaErrorMemoryAllocation;
    }
    g_fail_alloc_after.store(n - 1);
  }
  return cudaMalloc(p, bytes);
}

}  // namespace dc

extern "C" {

const char *dc_status_string(int status) {
  switch (status) {
    case DC_OK: return "DC_OK";
    case DC_ERR_ARG: return "DC_ERR_ARG: invalid argument";
    case DC_ERR_CUDA: return "DC_ERR_CUDA: CUDA call failed";
    case DC_ERR_OOM: return "DC_ERR_OOM: device allocation failed";
    case DC_ERR_TIMEOUT: return "DC_ERR_TIMEOUT: bounded device wait gave up";
    case DC_ERR_NONFINITE: return "DC_ERR_NONFINITE: NaN or infinite redundancy weight";
    case DC_ERR_UNSUPPORTED: return "DC_ERR_UNSUPPORTED: not supported by this build";
    default: return "unknown status";
  }
}

const char *dc_last_error(void) { return dc::g_last_error.c_str(); }

const char *dc_version(void) { return "dracogb 0.1 (sm_103a)"; }

unsigned long long dc_launch_count(void) { return dc::g_launches.load(); }

int dc_profile_enable(int on) { return dc::g_prof_on.exchange(on ? 1 : 0); }

int dc_profile_collect(double *ms, unsigned long long *launches, int n) {
  std::lock_guard<std::mutex> lk(dc::g_prof_mu);
  for (auto &r : dc::g_prof_recs) {
    if (cudaEventSynchronize(r.b) == cudaSuccess) {
      float t = 0.0f;
      if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
        dc::g_prof_ms[r.kid] += t;
        dc::g_prof_n[r.kid] += 1;
      }
    }
    dc::g_prof_pool.push_back(r.a);
    dc::g_prof_pool.push_back(r.b);
  }
  dc::g_prof_recs.clear();
  int k = n < dc::KID_COUNT ? n : (int)dc::KID_COUNT;
  for (int i = 0; i < k; ++i) {
    if (ms) ms[i] = dc::g_prof_ms[i];
    if (launches) launches[i] = dc::g_prof_n[i];
    dc::g_prof_ms[i] = 0.0;
    dc::g_prof_n[i] = 0;
  }
  return dc::KID_COUNT;
}

const char *dc_profile_kernel_name(int id) {
  static const char *names[] = {"k_prep", "k_linesum", "k_bp2d", "k_to_f16",
                                "k_reduce_gradW", "k_sino_in", "k_bp3d", "k_bp3d_adj",
                                "k_smooth", "k_adj_from_s", "k_filter_batched", "k_to_pairs"};
  return (id >= 0 && id < dc::KID_COUNT) ? names[id] : "";
}

// Test hook (not declared in the public header): make the n-th device
// allocation from now on fail; n < 0 disables the hook.
void dc_debug_fail_alloc_after(long n) { dc::g_fail_alloc_after.store(n); }

}  // extern "C"
