// Batched joins: many independent (index, S) joins in three launches.
//
// The learned probe of Section 2.D (root -> leaf -> window -> bounded
// search) applied to k joins at once, each join writing its own pairs
// (Section 2.A semantics; the indexes must have a unique R, as in the
// single-join direct path).  A plan fixes the batch's shape and holds every
// buffer the run needs, so a run allocates nothing and never synchronises:
//   batch_search_kernel   persistent blocks pull (join, 256-probe tile) work
//                         items from one ticket counter, so thousands of
//                         uneven joins balance across the GPU; each probe's
//                         result is one 32-bit word, each block adds its match
//                         count to its join's compaction tile
//   tile_scan_kernel      exclusive scan of all compaction tiles' counts
//   batch_compact_kernel  every compaction tile of every join writes its
//                         join's pairs (offsets relative to the join's first
//                         tile), coalesced; the first tile of each join also
//                         writes the join's total
// A run can be captured once in a CUDA graph and replayed.
//
// rmi_autotune picks the leaf count L of an index by timing the probe path
// on a sample of S for L in {2^8, 2^10, ..., 2^22} (bounded by n); results
// are cached by (log2 n, skew bucket, precision), where the skew bucket is the
// position of R's median key within [R[0], R[n-1]] in eighths.
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "device_common.cuh"
#include "internal.h"
#include "probe_core.cuh"

struct lj_batch {
  int device = 0;
  uint32_t k = 0;
  int precision = LJ_FP32;
  int block = 128;                 // search block size (tile = 2 * block probes)
  int chunk = 4;                   // tiles per work item
  uint64_t search_tiles = 0, comp_tiles = 0, probes = 0;
  void* desc = nullptr;            // JoinDesc[k] (device)
  uint64_t* search_tile0 = nullptr;   // [k+1] first work item of each join (device)
  uint64_t* comp_tile0 = nullptr;     // [k+1] (device)
  char* ws = nullptr;              // header | comp counts | scan flags | scan states | prefix | words
  size_t zero_bytes = 0;           // bytes of ws cleared at each run
  unsigned long long* comp_counts = nullptr;
  uint64_t* prefix = nullptr;
  uint32_t* words = nullptr;
  uint64_t* written = nullptr;     // [k] (device)
  lj::TileState scan_st{};
  uint32_t scan_blocks = 0;
  unsigned search_grid = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
};

namespace lj {
namespace {

struct JoinDesc {
  const uint64_t* R;
  const void* leaves;
  const uint64_t* S;
  lj_pair* out;
  uint64_t m;
  uint64_t cap;
  uint64_t words_off;
  double a0, b0;
  uint32_t L, n, r32, pad;
};

__device__ __forceinline__ uint32_t find_join(const uint64_t* tile0, uint32_t k, uint64_t t) {
  // largest j with tile0[j] <= t (tile0[0] = 0, tile0[k] = total)
  uint32_t a = 0, b = k;
  while (b - a > 1) {
    const uint32_t mid = (a + b) >> 1;
    if (tile0[mid] <= t)
      a = mid;
    else
      b = mid;
  }
  return a;
}

template <class Model>
__device__ __forceinline__ Model model_of(const JoinDesc& d);
template <>
__device__ __forceinline__ ModelF32 model_of<ModelF32>(const JoinDesc& d) {
  return ModelF32::make((float)d.a0, (float)d.b0, d.L);
}
template <>
__device__ __forceinline__ ModelF64 model_of<ModelF64>(const JoinDesc& d) {
  return ModelF64::make(d.a0, d.b0, d.L);
}

// Work item = CHUNK consecutive tiles of 2*BLOCK probes of one join: one
// ticket, one join lookup and one count barrier per item.
template <class Model, int BLOCK, int CHUNK>
__global__ void __launch_bounds__(BLOCK) batch_search_kernel(const JoinDesc* __restrict__ desc,
                                                             const uint64_t* __restrict__ item0,
                                                             uint32_t k, uint64_t total_items,
                                                             const uint64_t* __restrict__ comp0,
                                                             unsigned long long* comp_counts,
                                                             uint32_t* __restrict__ words,
                                                             uint32_t* ticket) {
  constexpr uint64_t kItem = 2ull * BLOCK * CHUNK;
  static_assert(kCompactTile % kItem == 0, "a work item must lie in one compaction tile");
  __shared__ uint64_t s_item;
  __shared__ unsigned long long s_count[BLOCK / 32];
  while (true) {
    if (threadIdx.x == 0) s_item = atomicAdd(reinterpret_cast<unsigned long long*>(ticket), 1ull);
    __syncthreads();
    const uint64_t item = s_item;
    if (item >= total_items) return;
    const uint32_t j = find_join(item0, k, item);
    const JoinDesc d = desc[j];
    const uint64_t first = (item - item0[j]) * kItem;   // first probe of the item in join j
    ProbeParams<Model> P{};
    P.R = d.R;
    P.n = d.n;
    P.r32 = d.r32 != 0;
    P.leaves = (const typename Model::Leaf*)d.leaves;
    P.model = model_of<Model>(d);
    P.S = d.S;
    P.m = d.m;
    const bool vec = (reinterpret_cast<uintptr_t>(d.S) & 15) == 0;
    uint32_t* w = words + d.words_off;
    unsigned long long c = 0;
#pragma unroll 1
    for (int t = 0; t < CHUNK; ++t) {
      const uint64_t j0 = first + (uint64_t)t * 2 * BLOCK + 2 * threadIdx.x;
      if (__all_sync(0xffffffffu, j0 >= d.m)) break;   // warp-uniform: lookups run as a warp
      uint32_t r_idx[2], cnt[2];
      bool valid[2];
      if (vec)
        lookup_probes<Model, kUniqueCount, 1, true>(P, j0, 0, r_idx, cnt, valid);
      else
        lookup_probes<Model, kUniqueCount, 1, false>(P, j0, 0, r_idx, cnt, valid);
      const uint32_t w0 = cnt[0] ? r_idx[0] : kNoMatch, w1 = cnt[1] ? r_idx[1] : kNoMatch;
      if (valid[1]) {
        *reinterpret_cast<uint2*>(w + j0) = make_uint2(w0, w1);   // words_off % 4 == 0
      } else if (valid[0]) {
        w[j0] = w0;
      }
      c += (unsigned long long)cnt[0] + cnt[1];
    }
#pragma unroll
    for (int dd = 16; dd >= 1; dd >>= 1) c += __shfl_xor_sync(0xffffffffu, c, dd);
    if ((threadIdx.x & 31) == 0) s_count[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long tot = 0;
#pragma unroll
      for (int q = 0; q < BLOCK / 32; ++q) tot += s_count[q];
      if (tot) atomicAdd(comp_counts + comp0[j] + first / kCompactTile, tot);
    }
  }
}

// Work item of 2*BLOCK probes (the shape's CHUNK = 1), one block per item and
// no ticket: without the persistent loop the lookups fit in 32 registers, so
// 2048 threads are resident per SM (the persistent kernel needs 78-94
// registers).
template <class Model, int BLOCK>
__global__ void __launch_bounds__(BLOCK, 2048 / BLOCK)
    batch_item_kernel(const JoinDesc* __restrict__ desc, const uint64_t* __restrict__ item0,
                      uint32_t k, uint64_t total_items, const uint64_t* __restrict__ comp0,
                      unsigned long long* comp_counts, uint32_t* __restrict__ words) {
  constexpr uint64_t kItem = 2ull * BLOCK;
  static_assert(kCompactTile % kItem == 0, "a work item must lie in one compaction tile");
  __shared__ unsigned long long s_count[BLOCK / 32];
  const uint64_t item = blockIdx.x;
  if (item >= total_items) return;
  const uint32_t j = find_join(item0, k, item);
  const JoinDesc d = desc[j];
  const uint64_t first = (item - item0[j]) * kItem;   // first probe of the item in join j
  ProbeParams<Model> P{};
  P.R = d.R;
  P.n = d.n;
  P.r32 = d.r32 != 0;
  P.leaves = (const typename Model::Leaf*)d.leaves;
  P.model = model_of<Model>(d);
  P.S = d.S;
  P.m = d.m;
  uint32_t* w = words + d.words_off;
  const uint64_t j0 = first + 2 * threadIdx.x;
  unsigned long long c = 0;
  if (!__all_sync(0xffffffffu, j0 >= d.m)) {   // warp-uniform: lookups run as a warp
    uint32_t r_idx[2], cnt[2];
    bool valid[2];
    if ((reinterpret_cast<uintptr_t>(d.S) & 15) == 0)
      lookup_probes<Model, kUniqueCount, 1, true>(P, j0, 0, r_idx, cnt, valid);
    else
      lookup_probes<Model, kUniqueCount, 1, false>(P, j0, 0, r_idx, cnt, valid);
    const uint32_t w0 = cnt[0] ? r_idx[0] : kNoMatch, w1 = cnt[1] ? r_idx[1] : kNoMatch;
    if (valid[1]) {
      *reinterpret_cast<uint2*>(w + j0) = make_uint2(w0, w1);   // words_off % 4 == 0
    } else if (valid[0]) {
      w[j0] = w0;
    }
    c = (unsigned long long)cnt[0] + cnt[1];
  }
#pragma unroll
  for (int dd = 16; dd >= 1; dd >>= 1) c += __shfl_xor_sync(0xffffffffu, c, dd);
  if ((threadIdx.x & 31) == 0) s_count[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long tot = 0;
#pragma unroll
    for (int q = 0; q < BLOCK / 32; ++q) tot += s_count[q];
    if (tot) atomicAdd(comp_counts + comp0[j] + first / kCompactTile, tot);
  }
}

template <bool VEC>
__global__ void __launch_bounds__(kBlock) batch_compact_kernel(const JoinDesc* __restrict__ desc,
                                                               const uint64_t* __restrict__ comp0,
                                                               uint32_t k,
                                                               const uint64_t* __restrict__ prefix,
                                                               const uint32_t* __restrict__ words,
                                                               uint64_t* written, uint32_t* err) {
  __shared__ uint64_t s_warp[kWarps];
  __shared__ uint64_t s_stage[kCompactTile];
  __shared__ uint64_t s_count;
  const uint64_t tile = blockIdx.x;
  const uint32_t j = find_join(comp0, k, tile);
  const JoinDesc d = desc[j];
  const uint64_t first = comp0[j];
  const uint64_t local_tile = tile - first;
  const uint64_t join_base = prefix[first];
  const uint64_t out0 = prefix[tile] - join_base;   // first output position of this tile in join j
  if (local_tile == 0 && threadIdx.x == 0) {
    const uint64_t total = prefix[comp0[j + 1]] - join_base;
    written[j] = total;
    if (total > d.cap) atomicOr(err, kErrCapacity);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t base = local_tile * kCompactTile + (uint64_t)threadIdx.x * kScanItems;
  const uint32_t* in = words + d.words_off;
  uint32_t v[kScanItems];
  if (VEC && base + kScanItems <= d.m && ((d.words_off & 3) == 0)) {
#pragma unroll
    for (int q = 0; q < kScanItems / 4; ++q) {
      const uint4 u = __ldg(reinterpret_cast<const uint4*>(in + base) + q);
      v[4 * q] = u.x;
      v[4 * q + 1] = u.y;
      v[4 * q + 2] = u.z;
      v[4 * q + 3] = u.w;
    }
  } else {
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) v[i] = base + i < d.m ? __ldg(in + base + i) : kNoMatch;
  }
  uint64_t sum = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) sum += v[i] != kNoMatch ? 1u : 0u;
  const uint64_t inc = warp_inclusive_sum(sum, lane);
  if (lane == 31) s_warp[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    const uint64_t x = lane < kWarps ? s_warp[lane] : 0;
    const uint64_t xi = warp_inclusive_sum(x, lane);
    if (lane < kWarps) s_warp[lane] = xi - x;
  }
  __syncthreads();
  uint64_t local = s_warp[warp] + inc - sum;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i)
    if (v[i] != kNoMatch) {
      s_stage[local] = (uint64_t)v[i] | ((uint64_t)(uint32_t)(base + i) << 32);
      ++local;
    }
  if (threadIdx.x == kBlock - 1) s_count = local;
  __syncthreads();
  const uint64_t cnt = s_count;
  uint64_t* out = reinterpret_cast<uint64_t*>(d.out);
  for (uint64_t q = threadIdx.x; q < cnt; q += kBlock) {
    const uint64_t o = out0 + q;
    if (o < d.cap) out[o] = s_stage[q];
  }
}

// Persistent grid: as many blocks of the plan's search shape as fit at once.
template <class Model>
int blocks_per_sm(int block, int chunk) {
  int per_sm = 0;
#define LJ_OCC(BLK, CH)                                                                   \
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_search_kernel<Model, BLK, CH>, \
                                                BLK, 0)
  if (block == 256) {
    if (chunk == 8) LJ_OCC(256, 8); else if (chunk == 4) LJ_OCC(256, 4); else LJ_OCC(256, 1);
  } else {
    if (chunk == 8) LJ_OCC(128, 8); else if (chunk == 4) LJ_OCC(128, 4); else LJ_OCC(128, 1);
  }
#undef LJ_OCC
  return per_sm;
}

unsigned persistent_grid(const lj_batch* b) {
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
  const int per_sm = b->precision == LJ_FP64 ? blocks_per_sm<ModelF64>(b->block, b->chunk)
                                             : blocks_per_sm<ModelF32>(b->block, b->chunk);
  return (unsigned)std::max(1, sms * std::max(1, per_sm));
}

// Enqueue one run of a plan on `s` (no allocation, no synchronisation).
int enqueue_run(lj_batch* b, cudaStream_t s) {
  uint32_t* err = device_error_word(b->device);
  if (!err) return fail(LJ_E_NOMEM, "cannot allocate the device error word");
  LJ_CUDA(cudaMemsetAsync(b->ws, 0, b->zero_bytes, s));
  LJ_CUDA(cudaMemsetAsync(b->written, 0, (size_t)b->k * 8, s));   // joins with no probes
  if (b->comp_tiles == 0) return 0;
  uint32_t* ticket = (uint32_t*)(b->ws + 64);
  const JoinDesc* desc = (const JoinDesc*)b->desc;
  {
    KernelTimer kt("batch_search_kernel", s);
#define LJ_BS(MODEL, BLK, CH)                                                                  \
  batch_search_kernel<MODEL, BLK, CH><<<b->search_grid, BLK, 0, s>>>(                          \
      desc, b->search_tile0, b->k, b->search_tiles, b->comp_tile0, b->comp_counts, b->words,   \
      ticket)
#define LJ_BI(MODEL, BLK)                                                                      \
  batch_item_kernel<MODEL, BLK><<<(unsigned)b->search_tiles, BLK, 0, s>>>(                     \
      desc, b->search_tile0, b->k, b->search_tiles, b->comp_tile0, b->comp_counts, b->words)
#define LJ_BS_SHAPE(MODEL)                                         \
  if (b->block == 256) {                                           \
    if (b->chunk == 8) LJ_BS(MODEL, 256, 8);                       \
    else if (b->chunk == 4) LJ_BS(MODEL, 256, 4);                  \
    else LJ_BI(MODEL, 256);                                        \
  } else {                                                         \
    if (b->chunk == 8) LJ_BS(MODEL, 128, 8);                       \
    else if (b->chunk == 4) LJ_BS(MODEL, 128, 4);                  \
    else LJ_BI(MODEL, 128);                                        \
  }
    if (b->precision == LJ_FP64) {
      LJ_BS_SHAPE(ModelF64)
    } else {
      LJ_BS_SHAPE(ModelF32)
    }
#undef LJ_BS
#undef LJ_BI
#undef LJ_BS_SHAPE
  }
  LJ_CUDA(cudaGetLastError());
  {
    KernelTimer kt("tile_scan_kernel", s);
    uint64_t* total_ws = (uint64_t*)(b->ws + 128);
    tile_scan_kernel<<<b->scan_blocks, kBlock, 0, s>>>(b->comp_counts, (uint32_t)b->comp_tiles,
                                                      b->prefix, b->scan_st, b->scan_blocks,
                                                      total_ws, nullptr, nullptr, ~0ull, err);
  }
  LJ_CUDA(cudaGetLastError());
  {
    KernelTimer kt("batch_compact_kernel", s);
    batch_compact_kernel<true><<<(unsigned)b->comp_tiles, kBlock, 0, s>>>(
        desc, b->comp_tile0, b->k, b->prefix, b->words, b->written, err);
  }
  LJ_CUDA(cudaGetLastError());
  return 0;
}

// ------------------------------------------------------------- autotuner --

std::mutex g_tune_mu;
std::map<std::tuple<int, int, int>, uint32_t> g_tune_cache;

int skew_bucket(const uint64_t* R, uint64_t n, cudaStream_t s, int* out) {
  uint64_t h[3] = {0, 0, 0};
  if (n == 0) {
    *out = 0;
    return 0;
  }
  LJ_CUDA(cudaMemcpyAsync(&h[0], R, 8, cudaMemcpyDeviceToHost, s));
  LJ_CUDA(cudaMemcpyAsync(&h[1], R + n / 2, 8, cudaMemcpyDeviceToHost, s));
  LJ_CUDA(cudaMemcpyAsync(&h[2], R + n - 1, 8, cudaMemcpyDeviceToHost, s));
  LJ_CUDA(cudaStreamSynchronize(s));
  const double span = (double)(h[2] - h[0]);
  const double pos = span > 0 ? (double)(h[1] - h[0]) / span : 0.5;
  *out = std::min(7, std::max(0, (int)(pos * 8.0)));
  return 0;
}

}  // namespace

// ------------------------------------------------ dynamic batches (serving) --

namespace {
constexpr int kDynBlock = 128, kDynChunk = 8;
constexpr uint64_t kDynItem = 2ull * kDynBlock * kDynChunk;

struct DynLayout {
  uint64_t tiles = 0, items = 0;
  uint32_t scan_blocks = 0;
  size_t b_cnt = 0, b_flags = 0, b_states = 0, b_pre = 0, b_words = 0;
  size_t total() const { return 256 + b_cnt + b_flags + b_states + b_pre + b_words; }
};

DynLayout dyn_layout(const BatchJob* jobs, uint32_t k) {
  DynLayout L;
  uint64_t words = 0;
  for (uint32_t j = 0; j < k; ++j) {
    L.tiles += (jobs[j].m + kCompactTile - 1) / kCompactTile;
    L.items += (jobs[j].m + kDynItem - 1) / kDynItem;
    words += (jobs[j].m + 3) & ~3ull;
  }
  const uint64_t Tc = std::max<uint64_t>(1, L.tiles);
  L.scan_blocks = (uint32_t)((Tc + kTileScanSpan - 1) / kTileScanSpan);
  L.b_cnt = (Tc * 8 + 255) / 256 * 256;
  L.b_flags = ((size_t)L.scan_blocks * 4 + 255) / 256 * 256;
  L.b_states = ((size_t)L.scan_blocks * 16 + 255) / 256 * 256;
  L.b_pre = ((Tc + 1) * 8 + 255) / 256 * 256;
  L.b_words = std::max<uint64_t>(words, 4) * 4;
  return L;
}

unsigned dyn_grid(int dev, int precision) {
  static unsigned grid[2][64] = {};
  const int p = precision == LJ_FP64 ? 1 : 0;
  if (dev >= 0 && dev < 64 && grid[p][dev]) return grid[p][dev];
  int sms = 0, per_sm = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (p)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, batch_search_kernel<ModelF64, kDynBlock, kDynChunk>, kDynBlock, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, batch_search_kernel<ModelF32, kDynBlock, kDynChunk>, kDynBlock, 0);
  const unsigned g = (unsigned)std::max(1, sms * std::max(1, per_sm));
  if (dev >= 0 && dev < 64) grid[p][dev] = g;
  return g;
}
}  // namespace

static size_t dyn_table_bytes(uint32_t k) { return (size_t)k * sizeof(JoinDesc) + 2 * (size_t)(k + 1) * 8; }

int dyn_batch_alloc(DynBatchBuffers& b, uint32_t max_jobs) {
  b.max_jobs = max_jobs;
  LJ_CUDA(cudaMalloc(&b.dev, dyn_table_bytes(max_jobs)));
  LJ_CUDA(cudaMallocHost(&b.host, dyn_table_bytes(max_jobs)));
  return 0;
}

void dyn_batch_release(DynBatchBuffers& b) {
  if (b.dev) cudaFree(b.dev);
  if (b.host) cudaFreeHost(b.host);
  b = DynBatchBuffers{};
}

size_t dyn_batch_scratch_bytes(const BatchJob* jobs, uint32_t k) { return dyn_layout(jobs, k).total(); }

int enqueue_dyn_batch(const BatchJob* jobs, uint32_t k, DynBatchBuffers& buf, char* scratch,
                      uint64_t* written, cudaStream_t s) {
  if (k == 0) return 0;
  if (k > buf.max_jobs) return fail(LJ_E_INVAL, "dynamic batch of %u jobs > %u", k, buf.max_jobs);
  const int prec = jobs[0].idx->precision;
  const int dev = jobs[0].idx->device;
  // tables for k jobs, packed: descriptors | item0[k+1] | comp0[k+1]
  JoinDesc* hd = (JoinDesc*)buf.host;
  uint64_t* item0_host = (uint64_t*)(buf.host + (size_t)k * sizeof(JoinDesc));
  uint64_t* comp0_host = item0_host + (k + 1);
  const JoinDesc* desc = (const JoinDesc*)buf.dev;
  const uint64_t* item0_dev = (const uint64_t*)(buf.dev + (size_t)k * sizeof(JoinDesc));
  const uint64_t* comp0_dev = item0_dev + (k + 1);
  const DynLayout L = dyn_layout(jobs, k);
  uint64_t words = 0;
  item0_host[0] = comp0_host[0] = 0;
  for (uint32_t j = 0; j < k; ++j) {
    const lj_index* x = jobs[j].idx;
    if (!x->unique || x->precision != prec || x->gkeys)
      return fail(LJ_E_INVAL, "dynamic batch: job %u needs a unique R of the batch's precision "
                              "without gapped arrays", j);
    JoinDesc& d = hd[j];
    d.R = x->R;
    d.leaves = x->leaves;
    d.S = jobs[j].S;
    d.out = jobs[j].out;
    d.m = jobs[j].m;
    d.cap = jobs[j].cap;
    d.words_off = words;
    d.a0 = prec == LJ_FP64 ? x->root_f64[0] : (double)x->root_f32[0];
    d.b0 = prec == LJ_FP64 ? x->root_f64[1] : (double)x->root_f32[1];
    d.L = x->L;
    d.n = (uint32_t)x->n;
    d.r32 = (reinterpret_cast<uintptr_t>(x->R) & 31) == 0;
    d.pad = 0;
    words += (jobs[j].m + 3) & ~3ull;
    item0_host[j + 1] = item0_host[j] + (jobs[j].m + kDynItem - 1) / kDynItem;
    comp0_host[j + 1] = comp0_host[j] + (jobs[j].m + kCompactTile - 1) / kCompactTile;
  }
  LJ_CUDA(cudaMemcpyAsync(buf.dev, buf.host, dyn_table_bytes(k), cudaMemcpyHostToDevice, s));
  char* p = scratch + 256;
  unsigned long long* counts = (unsigned long long*)p;
  p += L.b_cnt;
  TileState st;
  st.ticket = (uint32_t*)(scratch + 192);
  st.flag = (uint32_t*)p;
  p += L.b_flags;
  const size_t zero = p - scratch;
  st.agg = (uint64_t*)p;
  st.incl = st.agg + L.scan_blocks;
  p += L.b_states;
  uint64_t* prefix = (uint64_t*)p;
  p += L.b_pre;
  uint32_t* wds = (uint32_t*)p;
  uint32_t* err = device_error_word(dev);
  if (!err) return fail(LJ_E_NOMEM, "cannot allocate the device error word");
  LJ_CUDA(cudaMemsetAsync(scratch, 0, zero, s));
  LJ_CUDA(cudaMemsetAsync(written, 0, (size_t)k * 8, s));
  if (L.tiles == 0) return 0;
  uint32_t* ticket = (uint32_t*)(scratch + 64);
  {
    KernelTimer kt("batch_search_kernel", s);
    if (prec == LJ_FP64)
      batch_search_kernel<ModelF64, kDynBlock, kDynChunk><<<dyn_grid(dev, prec), kDynBlock, 0, s>>>(
          desc, item0_dev, k, L.items, comp0_dev, counts, wds, ticket);
    else
      batch_search_kernel<ModelF32, kDynBlock, kDynChunk><<<dyn_grid(dev, prec), kDynBlock, 0, s>>>(
          desc, item0_dev, k, L.items, comp0_dev, counts, wds, ticket);
  }
  LJ_CUDA(cudaGetLastError());
  tile_scan_kernel<<<L.scan_blocks, kBlock, 0, s>>>(counts, (uint32_t)L.tiles, prefix, st,
                                                    L.scan_blocks, (uint64_t*)(scratch + 128),
                                                    nullptr, nullptr, ~0ull, err);
  LJ_CUDA(cudaGetLastError());
  {
    KernelTimer kt("batch_compact_kernel", s);
    batch_compact_kernel<true><<<(unsigned)L.tiles, kBlock, 0, s>>>(desc, comp0_dev, k, prefix,
                                                                    wds, written, err);
  }
  LJ_CUDA(cudaGetLastError());
  return 0;
}

}  // namespace lj

extern "C" {

int join_batch_plan(const lj_index* const* indexes, const uint64_t* const* S_dev,
                    const uint64_t* m, uint32_t k, lj_pair* const* pairs_dev,
                    const uint64_t* capacity, lj_stream_t stream, lj_batch** out) {
  using namespace lj;
  if (!out) return fail(LJ_E_INVAL, "join_batch_plan: out is NULL");
  *out = nullptr;
  if (k == 0 || !indexes || !S_dev || !m || !pairs_dev || !capacity)
    return fail(LJ_E_INVAL, "join_batch_plan: empty batch or NULL array");
  cudaStream_t s = (cudaStream_t)stream;
  const int dev = current_device();
  const int prec = indexes[0] ? indexes[0]->precision : LJ_FP32;
  std::vector<JoinDesc> h(k);
  std::vector<uint64_t> t0(k + 1), c0(k + 1);
  uint64_t words = 0;
  t0[0] = c0[0] = 0;
  for (uint32_t j = 0; j < k; ++j) {
    const lj_index* x = indexes[j];
    if (!x) return fail(LJ_E_INVAL, "join_batch_plan: index %u is NULL", j);
    if (!x->unique)
      return fail(LJ_E_NOTUNIQUE, "join_batch_plan: join %u: batched joins need an R without "
                                  "duplicate keys", j);
    if (x->gkeys)
      return fail(LJ_E_INVAL, "join_batch_plan: join %u: gapped indexes (grmi_build) are not "
                              "supported in batches", j);
    if (x->precision != prec)
      return fail(LJ_E_INVAL, "join_batch_plan: all indexes of a batch need one precision");
    if (x->device != dev) return fail(LJ_E_INVAL, "join_batch_plan: index %u on another device", j);
    if (m[j] >= (1ull << 32)) return fail(LJ_E_INVAL, "join_batch_plan: m[%u] >= 2^32", j);
    if (m[j] && !S_dev[j]) return fail(LJ_E_INVAL, "join_batch_plan: S[%u] is NULL", j);
    if (capacity[j] && !pairs_dev[j]) return fail(LJ_E_INVAL, "join_batch_plan: pairs[%u] is NULL", j);
    JoinDesc& d = h[j];
    d.R = x->R;
    d.leaves = x->leaves;
    d.S = S_dev[j];
    d.out = pairs_dev[j];
    d.m = m[j];
    d.cap = capacity[j];
    d.words_off = words;
    d.a0 = prec == LJ_FP64 ? x->root_f64[0] : (double)x->root_f32[0];
    d.b0 = prec == LJ_FP64 ? x->root_f64[1] : (double)x->root_f32[1];
    d.L = x->L;
    d.n = (uint32_t)x->n;
    d.r32 = (reinterpret_cast<uintptr_t>(x->R) & 31) == 0;
    d.pad = 0;
    words += (m[j] + 3) & ~3ull;   // keep every join's words 16-byte aligned
    t0[j + 1] = t0[j] + (m[j] + 1023) / 1024;   // work items of the default shape (128 x 2 x 4)
    c0[j + 1] = c0[j] + (m[j] + kCompactTile - 1) / kCompactTile;
  }
  lj_batch* b = new lj_batch();
  b->device = dev;
  b->k = k;
  b->precision = prec;
  b->search_tiles = t0[k];
  b->comp_tiles = c0[k];
  b->probes = words;
  auto bail = [&](int rc) {
    join_batch_free(b);
    return rc;
  };
  const uint64_t Tc = std::max<uint64_t>(1, b->comp_tiles);
  b->scan_blocks = (uint32_t)((Tc + kTileScanSpan - 1) / kTileScanSpan);
  const size_t b_cnt = (Tc * 8 + 255) / 256 * 256;
  const size_t b_flags = ((size_t)b->scan_blocks * 4 + 255) / 256 * 256;
  const size_t b_states = ((size_t)b->scan_blocks * 16 + 255) / 256 * 256;
  const size_t b_pre = ((Tc + 1) * 8 + 255) / 256 * 256;
  const size_t b_words = std::max<uint64_t>(words, 4) * 4;
  const size_t b_desc = ((size_t)k * sizeof(JoinDesc) + 255) / 256 * 256;
  const size_t b_t0 = ((size_t)(k + 1) * 8 + 255) / 256 * 256;
  const size_t b_written = ((size_t)k * 8 + 255) / 256 * 256;
  cudaError_t ce = cudaMalloc(&b->ws, 256 + b_cnt + b_flags + b_states + b_pre + b_words + b_desc +
                                          2 * b_t0 + b_written);
  if (ce != cudaSuccess) return bail(fail_cuda(ce, "join_batch_plan: scratch"));
  char* p = b->ws + 256;
  b->comp_counts = (unsigned long long*)p;
  p += b_cnt;
  b->scan_st.ticket = (uint32_t*)(b->ws + 192);
  b->scan_st.flag = (uint32_t*)p;
  p += b_flags;
  b->zero_bytes = p - b->ws;   // header, counts and scan flags
  b->scan_st.agg = (uint64_t*)p;
  b->scan_st.incl = b->scan_st.agg + b->scan_blocks;
  p += b_states;
  b->prefix = (uint64_t*)p;
  p += b_pre;
  b->words = (uint32_t*)p;
  p += b_words;
  b->desc = p;
  p += b_desc;
  b->search_tile0 = (uint64_t*)p;
  p += b_t0;
  b->comp_tile0 = (uint64_t*)p;
  p += b_t0;
  b->written = (uint64_t*)p;
  if ((ce = cudaMemcpyAsync(b->desc, h.data(), (size_t)k * sizeof(JoinDesc),
                            cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (ce = cudaMemcpyAsync(b->search_tile0, t0.data(), (k + 1) * 8, cudaMemcpyHostToDevice, s)) !=
          cudaSuccess ||
      (ce = cudaMemcpyAsync(b->comp_tile0, c0.data(), (k + 1) * 8, cudaMemcpyHostToDevice, s)) !=
          cudaSuccess ||
      (ce = cudaStreamSynchronize(s)) != cudaSuccess)
    return bail(fail_cuda(ce, "join_batch_plan: upload"));
  b->search_grid = persistent_grid(b);
  *out = b;
  return LJ_OK;
}

int join_batch_run(lj_batch* b, uint64_t* written_dev, uint64_t* written_host, lj_stream_t stream) {
  using namespace lj;
  if (!b) return fail(LJ_E_INVAL, "join_batch_run: plan is NULL");
  if (current_device() != b->device) return fail(LJ_E_INVAL, "join_batch_run: wrong device");
  cudaStream_t s = (cudaStream_t)stream;
  if (b->graph_exec) {
    LJ_CUDA(cudaGraphLaunch(b->graph_exec, s));
  } else if (int rc = enqueue_run(b, s)) {
    return rc;
  }
  if (written_dev)
    LJ_CUDA(cudaMemcpyAsync(written_dev, b->written, (size_t)b->k * 8, cudaMemcpyDeviceToDevice, s));
  if (written_host) {
    LJ_CUDA(cudaMemcpyAsync(written_host, b->written, (size_t)b->k * 8, cudaMemcpyDeviceToHost, s));
    LJ_CUDA(cudaStreamSynchronize(s));
    if (int rc = take_device_errors(b->device, s)) return rc;
  }
  return LJ_OK;
}

int join_batch_capture(lj_batch* b, lj_stream_t stream) {
  using namespace lj;
  if (!b) return fail(LJ_E_INVAL, "join_batch_capture: plan is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  if (!s) return fail(LJ_E_INVAL, "join_batch_capture: needs a non-default stream");
  if (!device_error_word(b->device)) return fail(LJ_E_NOMEM, "cannot allocate the error word");
  if (b->graph_exec) {
    cudaGraphExecDestroy(b->graph_exec);
    cudaGraphDestroy(b->graph);
    b->graph_exec = nullptr;
    b->graph = nullptr;
  }
  LJ_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  const bool prof = profiling();
  set_profiling(false);   // no timing events inside a graph
  int rc = enqueue_run(b, s);
  set_profiling(prof);
  cudaGraph_t g = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(s, &g);
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (ce != cudaSuccess) return fail_cuda(ce, "join_batch_capture: end capture");
  cudaGraphExec_t ex = nullptr;
  const cudaError_t ie = cudaGraphInstantiate(&ex, g, 0);
  if (ie != cudaSuccess) {
    cudaGraphDestroy(g);
    return fail_cuda(ie, "join_batch_capture: instantiate");
  }
  b->graph = g;
  b->graph_exec = ex;
  return LJ_OK;
}

int join_batch_set_shape(lj_batch* b, int block, int tiles_per_item) {
  using namespace lj;
  if (!b || (block != 128 && block != 256) ||
      (tiles_per_item != 1 && tiles_per_item != 4 && tiles_per_item != 8))
    return fail(LJ_E_INVAL, "join_batch_set_shape: block must be 128 or 256, tiles 1, 4 or 8");
  if (block == b->block && tiles_per_item == b->chunk) return LJ_OK;
  std::vector<JoinDesc> h(b->k);
  std::vector<uint64_t> t0(b->k + 1);
  LJ_CUDA(cudaMemcpy(h.data(), b->desc, (size_t)b->k * sizeof(JoinDesc), cudaMemcpyDeviceToHost));
  const uint64_t item = 2ull * block * tiles_per_item;
  t0[0] = 0;
  for (uint32_t j = 0; j < b->k; ++j) t0[j + 1] = t0[j] + (h[j].m + item - 1) / item;
  LJ_CUDA(cudaMemcpy(b->search_tile0, t0.data(), (b->k + 1) * 8, cudaMemcpyHostToDevice));
  b->search_tiles = t0[b->k];
  b->block = block;
  b->chunk = tiles_per_item;
  b->search_grid = persistent_grid(b);
  if (b->graph_exec) {   // the captured graph has the old shape
    cudaGraphExecDestroy(b->graph_exec);
    cudaGraphDestroy(b->graph);
    b->graph_exec = nullptr;
    b->graph = nullptr;
  }
  return LJ_OK;
}

int join_batch_autotune(lj_batch* b, lj_stream_t stream, int* best_block, int* best_tiles) {
  using namespace lj;
  if (!b) return fail(LJ_E_INVAL, "join_batch_autotune: plan is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  static const int shapes[][2] = {{128, 1}, {128, 4}, {128, 8}, {256, 1}, {256, 4}, {256, 8}};
  cudaEvent_t e0, e1;
  LJ_CUDA(cudaEventCreate(&e0));
  LJ_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  int bb = b->block, bt = b->chunk, rc = 0;
  for (const auto& sh : shapes) {
    if ((rc = join_batch_set_shape(b, sh[0], sh[1]))) break;
    if ((rc = enqueue_run(b, s))) break;   // warm-up
    cudaEventRecord(e0, s);
    if ((rc = enqueue_run(b, s))) break;
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) {
      best = ms;
      bb = sh[0];
      bt = sh[1];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  if ((rc = join_batch_set_shape(b, bb, bt))) return rc;
  if (best_block) *best_block = bb;
  if (best_tiles) *best_tiles = bt;
  return take_device_errors(b->device, s);
}

void join_batch_free(lj_batch* b) {
  if (!b) return;
  if (b->graph_exec) cudaGraphExecDestroy(b->graph_exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->ws) cudaFree(b->ws);
  delete b;
}

int join_batch(const lj_index* const* indexes, const uint64_t* const* S_dev, const uint64_t* m,
               uint32_t k, lj_pair* const* pairs_dev, const uint64_t* capacity,
               uint64_t* written_host, lj_stream_t stream) {
  lj_batch* b = nullptr;
  int rc = join_batch_plan(indexes, S_dev, m, k, pairs_dev, capacity, stream, &b);
  if (rc) return rc;
  rc = join_batch_run(b, nullptr, written_host, stream);
  if (!written_host) cudaStreamSynchronize((cudaStream_t)stream);
  join_batch_free(b);
  return rc;
}

int rmi_autotune(const uint64_t* R_dev, uint64_t n, const uint64_t* S_sample_dev, uint64_t m_sample,
                 int precision, lj_stream_t stream, uint32_t* best_leaves, double* best_ns_per_key) {
  using namespace lj;
  if (!best_leaves) return fail(LJ_E_INVAL, "rmi_autotune: best_leaves is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  int skew = 0;
  if (int rc = skew_bucket(R_dev, n, s, &skew)) return rc;
  const int lg = n ? (int)std::floor(std::log2((double)n)) : 0;
  const auto key = std::make_tuple(lg, skew, precision);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      *best_leaves = it->second;
      if (best_ns_per_key) *best_ns_per_key = -1.0;   // from the cache
      return LJ_OK;
    }
  }
  const uint64_t lmax = std::max<uint64_t>(256, std::min<uint64_t>(1u << 22, n / 2));
  uint32_t best = 256;
  double best_t = 1e300;
  lj_pair* pairs = nullptr;
  LJ_CUDA(scratch_alloc((void**)&pairs, std::max<uint64_t>(m_sample, 1) * 8, s));
  cudaEvent_t e0, e1;
  LJ_CUDA(cudaEventCreate(&e0));
  LJ_CUDA(cudaEventCreate(&e1));
  int rc = 0;
  for (uint64_t L = 256; L <= lmax && !rc; L *= 4) {
    lj_index* idx = nullptr;
    if ((rc = rmi_build(R_dev, n, (uint32_t)L, precision, stream, &idx))) break;
    float ms = 1e30f;
    for (int rep = 0; rep < 4 && !rc; ++rep) {
      cudaEventRecord(e0, s);
      if (idx->unique)
        rc = join_emit(idx, S_sample_dev, m_sample, nullptr, pairs, m_sample, nullptr, nullptr, stream);
      else
        rc = join_count(idx, S_sample_dev, m_sample, nullptr, nullptr, nullptr, stream);
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      if (rep > 0) ms = std::min(ms, t);   // first run warms up
    }
    rmi_free(idx);
    const double ns = m_sample ? ms * 1e6 / (double)m_sample : 0.0;
    if (!rc && ns < best_t) {
      best_t = ns;
      best = (uint32_t)L;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  scratch_free(pairs, s);
  cudaStreamSynchronize(s);
  if (rc) return rc;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = best;
  }
  *best_leaves = best;
  if (best_ns_per_key) *best_ns_per_key = best_t;
  return LJ_OK;
}

void rmi_autotune_clear(void) {
  std::lock_guard<std::mutex> lk(lj::g_tune_mu);
  lj::g_tune_cache.clear();
}

}  // extern "C"
