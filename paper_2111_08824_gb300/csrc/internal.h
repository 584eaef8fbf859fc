// Host-side internals shared by the translation units of the library.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <memory>
#include <string>

#include "../../include/ljoin.h"

namespace lj {
constexpr int kMaxLevels = 15;   // key levels of R: 4^16 > 2^32 - 1 positions
}  // namespace lj

struct lj_index {
  const uint64_t* R = nullptr;   // borrowed, sorted
  uint64_t n = 0;
  uint32_t L = 0;
  int precision = LJ_FP32;
  int device = 0;
  void* leaves = nullptr;        // L records (LeafF32 or LeafF64), device
  std::shared_ptr<void> leaves_block;   // owner of `leaves` (shared by a batch's indexes)
  double root_fit[2] = {0, 0};   // least-squares root (double)
  float root_f32[2] = {0, 0};    // deployed single-precision root
  double root_f64[2] = {0, 0};   // deployed double-precision root
  int unique = 1;
  int probe_order = -1;          // bucketed probe order: -1 follow the option, 0 off, 1 on
  lj_index_stats stats{};
  // gapped arrays (grmi_build): C slots of keys, C + 1 payloads (positions)
  uint64_t* gkeys = nullptr;
  uint32_t* gpos = nullptr;
  uint32_t gslots = 0;           // C
  uint32_t gscale = 0;           // 1 + gaps (gapped RMI)
  int gkind = 0;                 // 0: gapped RMI over R's keys, 1: learned hash over distinct
                                 // keys (RMI as the hash), 2: the same with a RadixSpline
  uint32_t* dfirst = nullptr;    // learned hash: first position of each distinct key, D + 1
  uint64_t* hrange = nullptr;    // learned hash: per slot, first | count << 32 of its entry
  uint64_t ndistinct = 0;        // learned hash: D
  uint64_t hbuckets = 0;         // learned hash: B
  // RadixSpline of the learned hash with a RadixSpline as the hash (gkind 2)
  uint64_t* rs_x = nullptr;      // spline keys
  uint32_t* rs_y = nullptr;      // spline positions
  double* rs_rcp = nullptr;      // 1 / (x_{i+1} - x_i)
  uint32_t* rs_table = nullptr;  // radix table, 2^rs_rbits + 1 entries
  uint32_t rs_S = 0, rs_shift = 0, rs_rbits = 0, rs_eps = 0;
  uint64_t rs_kmin = 0, rs_kmax = 0;
  lj_grmi_stats gstats{};
  // key levels of R (option "key_levels"): level k = 1 .. nlev holds
  // R[4^k i] (padded to whole 4-entry nodes) at levels + lev_off[k]
  uint64_t* levels = nullptr;
  uint32_t nlev = 0;
  int use_levels = 0;            // the pipeline's search descends the levels
  uint32_t lev_off[lj::kMaxLevels + 1] = {};
};

namespace lj {

// Thread-local error message; returns `code` for convenient `return fail(...)`.
int fail(int code, const char* fmt, ...);
int fail_cuda(cudaError_t e, const char* what);

#define LJ_CUDA(call)                                      \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return ::lj::fail_cuda(e_, #call); \
  } while (0)

// Stream-ordered scratch memory from a library-owned pool (one per device,
// release threshold = unlimited, so repeated calls reuse the same memory).
cudaError_t scratch_alloc(void** p, size_t bytes, cudaStream_t s);
cudaError_t scratch_free(void* p, cudaStream_t s);

// Sticky per-device error word that kernels OR bits into (kErr*).
uint32_t* device_error_word(int device);
// Read and clear the error word after `s` has been synchronised; maps bits to
// an LJ_E_* code (0 if clean).
int take_device_errors(int device, cudaStream_t s);

int current_device();

// Opt-in per-kernel timing (lj_set_option("profile", 1)): CUDA events are
// recorded around each launch on its own stream; lj_profile_report
// aggregates them.  Costs nothing when profiling is off.
class KernelTimer {
 public:
  KernelTimer(const char* name, cudaStream_t s);
  ~KernelTimer();
  KernelTimer(const KernelTimer&) = delete;
  KernelTimer& operator=(const KernelTimer&) = delete;

 private:
  const char* name_;
  cudaStream_t s_;
  cudaEvent_t a_ = nullptr, b_ = nullptr;
};
void set_profiling(bool on);
bool profiling();

// One join of a dynamically formed batch (serving): index (unique R), probe
// keys (device or page-locked host memory), output pairs and their room.
struct BatchJob {
  const lj_index* idx;
  const uint64_t* S;
  uint64_t m;
  lj_pair* out;
  uint64_t cap;
};

// Per-slot buffers of dynamic batches: descriptor tables on the device and
// their page-locked host staging (reused only after the slot's batch ends).
struct DynBatchBuffers {
  uint32_t max_jobs = 0;
  char* dev = nullptr;    // descriptors, then the two tile tables (one upload)
  char* host = nullptr;   // page-locked staging with the same layout
};
int dyn_batch_alloc(DynBatchBuffers& b, uint32_t max_jobs);
void dyn_batch_release(DynBatchBuffers& b);
// Scratch bytes a dynamic batch of these jobs needs (4 bytes per probe + tables).
size_t dyn_batch_scratch_bytes(const BatchJob* jobs, uint32_t k);
// Enqueue the batched search, scan and compaction of k jobs on s; writes each
// job's |J| to written_dev[k].  No allocation, no synchronisation.
int enqueue_dyn_batch(const BatchJob* jobs, uint32_t k, DynBatchBuffers& buf, char* scratch,
                      uint64_t* written_dev, cudaStream_t s);

// join_emit's direct or two-pass path on stream s (no synchronisation when
// total_host is NULL); total_dev receives |J|.
int probe_emit_impl(const lj_index* idx, const uint64_t* S, uint64_t m, const uint64_t* offsets,
                    lj_pair* pairs, uint64_t cap, uint64_t* total_dev, uint64_t* total_host,
                    uint32_t s_base, cudaStream_t s);

// Release the gapped arrays of an index (no-op without them).
void grmi_release(lj_index* idx);

// Probe keys per chunk of join_host.
void set_host_chunk(uint64_t v);
uint64_t get_host_chunk();

// Bucketed probe order in the count-scan-emit pipeline (0 off, 1 on).
void set_probe_buckets(int v);
int get_probe_buckets();

// Bound of one look-back wait (option "lookback_polls") and the test hook
// "fault_skip_tiles": single-pass launches skip that many leading tiles, whose
// states are then never published, so the waits of the next tiles run out.
uint32_t lookback_polls();
uint32_t fault_skip_tiles();

// Key levels built by rmi_build (option "key_levels": 0 never, 1 always,
// 2 for an R with duplicate keys).
void set_key_levels(int v);
int get_key_levels();
int build_key_levels(lj_index* idx, cudaStream_t s);

// Probe batches of at most this many keys take the single-pass kernel.
void set_fused_max(uint64_t v);
uint64_t get_fused_max();
void set_fused_groups(int v);
int get_fused_groups();
void set_single_pass_max(uint64_t v);
uint64_t get_single_pass_max();

}  // namespace lj
