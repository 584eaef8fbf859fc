// Error reporting, scratch memory, and the host-only index entry points.
#include <atomic>
#include <cstdarg>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "device_common.cuh"
#include "internal.h"

namespace lj {

static thread_local char g_err[512] = "";

int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

int fail_cuda(cudaError_t e, const char* what) {
  return fail(e == cudaErrorMemoryAllocation ? LJ_E_NOMEM : LJ_E_CUDA, "%s: %s (%s)",
              what, cudaGetErrorName(e), cudaGetErrorString(e));
}

int current_device() {
  int d = 0;
  cudaGetDevice(&d);
  return d;
}

namespace {
std::mutex g_mu;
std::vector<cudaMemPool_t> g_pools;
std::vector<uint32_t*> g_err_words;
}  // namespace

static cudaMemPool_t pool_for(int dev) {
  std::lock_guard<std::mutex> lk(g_mu);
  if ((int)g_pools.size() <= dev) g_pools.resize(dev + 1, nullptr);
  if (!g_pools[dev]) {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p = nullptr;
    if (cudaMemPoolCreate(&p, &props) != cudaSuccess) return nullptr;
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &thr);
    g_pools[dev] = p;
  }
  return g_pools[dev];
}

cudaError_t scratch_alloc(void** p, size_t bytes, cudaStream_t s) {
  *p = nullptr;
  if (bytes == 0) bytes = 256;
  cudaMemPool_t pool = pool_for(current_device());
  if (!pool) return cudaErrorMemoryAllocation;
  return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

cudaError_t scratch_free(void* p, cudaStream_t s) {
  if (!p) return cudaSuccess;
  return cudaFreeAsync(p, s);
}

uint32_t* device_error_word(int dev) {
  std::lock_guard<std::mutex> lk(g_mu);
  if ((int)g_err_words.size() <= dev) g_err_words.resize(dev + 1, nullptr);
  if (!g_err_words[dev]) {
    uint32_t* p = nullptr;
    if (cudaMalloc(&p, 256) != cudaSuccess) return nullptr;
    if (cudaMemset(p, 0, 256) != cudaSuccess) return nullptr;
    g_err_words[dev] = p;
  }
  return g_err_words[dev];
}

int take_device_errors(int dev, cudaStream_t s) {
  uint32_t* w = device_error_word(dev);
  if (!w) return fail(LJ_E_NOMEM, "cannot allocate the device error word");
  uint32_t v = 0;
  LJ_CUDA(cudaMemcpyAsync(&v, w, sizeof(v), cudaMemcpyDeviceToHost, s));
  LJ_CUDA(cudaStreamSynchronize(s));
  if (v) {
    LJ_CUDA(cudaMemsetAsync(w, 0, sizeof(uint32_t), s));
    LJ_CUDA(cudaStreamSynchronize(s));
  }
  if (v & kErrLookbackTimeout)
    return fail(LJ_E_TIMEOUT, "a device-side look-back wait ran out (error word 0x%x)", v);
  if (v & kErrCapacity) return fail(LJ_E_CAPACITY, "output capacity exceeded on the device");
  return 0;
}

namespace {
std::atomic<bool> g_profile{false};
struct ProfRec {
  const char* name;
  cudaEvent_t a, b;
};
std::mutex g_prof_mu;
std::vector<ProfRec> g_prof;
}  // namespace

void set_profiling(bool on) { g_profile.store(on); }
bool profiling() { return g_profile.load(std::memory_order_relaxed); }

KernelTimer::KernelTimer(const char* name, cudaStream_t s) : name_(name), s_(s) {
  if (!profiling()) return;
  if (cudaEventCreate(&a_) != cudaSuccess || cudaEventCreate(&b_) != cudaSuccess) {
    if (a_) cudaEventDestroy(a_);
    a_ = b_ = nullptr;
    return;
  }
  cudaEventRecord(a_, s_);
}

KernelTimer::~KernelTimer() {
  if (!a_) return;
  cudaEventRecord(b_, s_);
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof.push_back({name_, a_, b_});
}

// Bound of one look-back wait (polls of a predecessor tile) and the test
// hook that makes such a wait run out (see lj_set_option).
namespace {
std::atomic<uint32_t> g_lookback_polls{kLookbackPolls};
std::atomic<uint32_t> g_fault_skip_tiles{0};
}  // namespace
uint32_t lookback_polls() { return g_lookback_polls.load(); }
uint32_t fault_skip_tiles() { return g_fault_skip_tiles.load(); }

}  // namespace lj

extern "C" {

int lj_set_option(const char* name, int64_t value) {
  using namespace lj;
  if (!name) return fail(LJ_E_INVAL, "lj_set_option: name is NULL");
  if (!strcmp(name, "single_pass_max")) {
    if (value < 0) return fail(LJ_E_INVAL, "single_pass_max must be >= 0");
    set_single_pass_max((uint64_t)value);
    return LJ_OK;
  }
  if (!strcmp(name, "key_levels")) {
    if (value < 0 || value > 2) return fail(LJ_E_INVAL, "key_levels must be 0, 1 or 2");
    set_key_levels((int)value);
    return LJ_OK;
  }
  if (!strcmp(name, "fused_max")) {
    if (value < 0 || value > (1ll << 22))
      return fail(LJ_E_INVAL, "fused_max must be in [0, 2^22]");
    set_fused_max((uint64_t)value);
    return LJ_OK;
  }
  if (!strcmp(name, "fused_groups")) {
    if (value < 0 || value > 1) return fail(LJ_E_INVAL, "fused_groups must be 0 or 1");
    set_fused_groups((int)value);
    return LJ_OK;
  }
  if (!strcmp(name, "profile")) {
    set_profiling(value != 0);
    return LJ_OK;
  }
  if (!strcmp(name, "probe_buckets")) {
    if (value < 0 || value > 2) return fail(LJ_E_INVAL, "probe_buckets must be 0, 1 or 2");
    set_probe_buckets((int)value);
    return LJ_OK;
  }
  if (!strcmp(name, "host_chunk")) {
    if (value < (1 << 16) || value >= (1ll << 32))
      return fail(LJ_E_INVAL, "host_chunk must be in [2^16, 2^32)");
    set_host_chunk((uint64_t)value);
    return LJ_OK;
  }
  if (!strcmp(name, "lookback_polls")) {
    if (value < 16 || value > (int64_t)kLookbackPolls)
      return fail(LJ_E_INVAL, "lookback_polls must be in [16, 2^20]");
    g_lookback_polls = (uint32_t)value;
    return LJ_OK;
  }
  if (!strcmp(name, "fault_skip_tiles")) {
    if (value < 0 || value > 1024) return fail(LJ_E_INVAL, "fault_skip_tiles must be in [0, 1024]");
    g_fault_skip_tiles = (uint32_t)value;
    return LJ_OK;
  }
  return fail(LJ_E_INVAL, "lj_set_option: unknown option '%s'", name);
}

int64_t lj_get_option(const char* name) {
  using namespace lj;
  if (name && !strcmp(name, "single_pass_max")) return (int64_t)get_single_pass_max();
  if (name && !strcmp(name, "key_levels")) return get_key_levels();
  if (name && !strcmp(name, "fused_max")) return (int64_t)get_fused_max();
  if (name && !strcmp(name, "fused_groups")) return get_fused_groups();
  if (name && !strcmp(name, "profile")) return profiling() ? 1 : 0;
  if (name && !strcmp(name, "host_chunk")) return (int64_t)get_host_chunk();
  if (name && !strcmp(name, "probe_buckets")) return get_probe_buckets();
  if (name && !strcmp(name, "lookback_polls")) return lookback_polls();
  if (name && !strcmp(name, "fault_skip_tiles")) return fault_skip_tiles();
  fail(LJ_E_INVAL, "lj_get_option: unknown option '%s'", name ? name : "(null)");
  return -1;
}

int lj_profile_report(char* buf, size_t len) {
  using namespace lj;
  std::vector<ProfRec> recs;
  {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    recs.swap(g_prof);
  }
  struct Agg {
    uint64_t n = 0;
    double total = 0, mn = 1e300, mx = 0;
  };
  std::map<std::string, Agg> agg;
  int rc = 0;
  for (auto& r : recs) {
    float ms = 0.f;
    if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      Agg& a = agg[r.name];
      a.n++;
      a.total += ms;
      a.mn = ms < a.mn ? ms : a.mn;
      a.mx = ms > a.mx ? ms : a.mx;
    } else {
      rc = LJ_E_CUDA;
    }
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  std::string out = "{";
  bool first = true;
  for (auto& kv : agg) {
    char tmp[256];
    snprintf(tmp, sizeof(tmp), "%s\"%s\": {\"launches\": %llu, \"total_ms\": %.6f, \"min_ms\": %.6f, \"max_ms\": %.6f}",
             first ? "" : ", ", kv.first.c_str(), (unsigned long long)kv.second.n, kv.second.total,
             kv.second.mn, kv.second.mx);
    out += tmp;
    first = false;
  }
  out += "}";
  if (rc) return fail(rc, "lj_profile_report: an event could not be read");
  if (!buf || len <= out.size()) return fail(LJ_E_INVAL, "lj_profile_report: buffer of %zu bytes too small (%zu needed)", len, out.size() + 1);
  memcpy(buf, out.c_str(), out.size() + 1);
  return (int)out.size();
}


const char* lj_last_error(void) { return lj::g_err; }

const char* lj_version(void) { return "ljoin-gb300 0.1 (sm_103a)"; }

void rmi_free(lj_index* index) {
  if (!index) return;
  lj::grmi_release(index);
  if (index->leaves && !index->leaves_block) cudaFree(index->leaves);
  if (index->levels) cudaFree(index->levels);
  delete index;   // the last index of a batch releases the batch's leaf records
}

int rmi_stats(const lj_index* index, lj_index_stats* out) {
  if (!index || !out) return lj::fail(LJ_E_INVAL, "rmi_stats: NULL argument");
  *out = index->stats;
  return LJ_OK;
}

int rmi_export(const lj_index* index, double* root_host, uint64_t* leaf_lo, double* leaf_ab,
               int64_t* leaf_err) {
  if (!index) return lj::fail(LJ_E_INVAL, "rmi_export: NULL index");
  const uint32_t L = index->L;
  if (root_host) {
    if (index->precision == LJ_FP64) {
      root_host[0] = index->root_f64[0];
      root_host[1] = index->root_f64[1];
    } else {
      root_host[0] = index->root_f32[0];
      root_host[1] = index->root_f32[1];
    }
  }
  if (!leaf_lo && !leaf_ab && !leaf_err) return LJ_OK;
  if (index->precision == LJ_FP64) {
    std::vector<lj::LeafF64> h(L);
    LJ_CUDA(cudaMemcpy(h.data(), index->leaves, sizeof(lj::LeafF64) * L, cudaMemcpyDeviceToHost));
    for (uint32_t l = 0; l < L; ++l) {
      if (leaf_lo) leaf_lo[l] = h[l].lo;
      if (leaf_ab) {
        leaf_ab[2 * l] = h[l].a;
        leaf_ab[2 * l + 1] = h[l].b;
      }
      if (leaf_err) {
        leaf_err[2 * l] = h[l].e_lo;
        leaf_err[2 * l + 1] = h[l].e_hi;
      }
    }
  } else {
    std::vector<lj::LeafF32> h(L);
    LJ_CUDA(cudaMemcpy(h.data(), index->leaves, sizeof(lj::LeafF32) * L, cudaMemcpyDeviceToHost));
    for (uint32_t l = 0; l < L; ++l) {
      if (leaf_lo) leaf_lo[l] = h[l].lo;
      if (leaf_ab) {
        leaf_ab[2 * l] = h[l].a;
        leaf_ab[2 * l + 1] = h[l].b;
      }
      if (leaf_err) {
        leaf_err[2 * l] = h[l].e_lo;
        leaf_err[2 * l + 1] = h[l].e_hi;
      }
    }
  }
  if (leaf_lo) leaf_lo[L] = index->n;
  return LJ_OK;
}

}  // extern "C"
