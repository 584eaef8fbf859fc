// Gapped layouts built by model-based insertion, and the choice among the
// lookup structures (Sabek and Kraska, "The Case for Learned In-Memory
// Joins"):
//   gapped RMI (Section 3.A, grmi_build): the RMI already fitted over R
//     places every tuple of R, in key order, into a gapped key array and a
//     gapped payload array, (1 + gaps) slots per key; a lookup starts at the
//     predicted slot and finishes with an exponential search (probe side:
//     gapped_search_kernel);
//   learned hash index (Section 3.C, lhash_build): the RMI as an
//     order-preserving hash into buckets of 4 slots, one entry per distinct
//     key of R whose payload gives its whole range of matches (probe side:
//     hash_search_kernel);
//   index_autotune: times the lookup structures on a probe sample and keeps
//     the fastest.
//
// Model-based insertion in key order puts key i at its predicted slot, or at
// the first slot after key i-1 if that one is later:
//     slot_i = max(pslot_i, slot_{i-1} + 1) = i + max_{j <= i} (pslot_j - j),
// an inclusive max-scan of d_j = pslot_j - j (the predicted slot comes from
// a GappedSlot or a HashSlot).  The build is three passes:
//   grmi_dmax_kernel     per tile of 2048 keys: max of d over the tile
//   grmi_prefix_kernel   exclusive max-scan of the tile maxima (one block)
//   grmi_fill_kernel     per tile: slots of its keys (block max-scan seeded
//                        with the tile prefix), then every slot the tile owns,
//                        (slot of the previous tile's last key, slot of its
//                        own last key], takes the key and position of the
//                        first key placed at or after it: gaps hold copies of
//                        the next key, so the key array stays sorted
//   grmi_tail_kernel     slots after the last key: 2^64-1 and the key count;
//                        pos[C] = the key count
// Each slot is written once, with coalesced stores.  The learned hash first
// extracts the distinct keys of R (run_count_kernel, a sum-scan,
// run_write_kernel) and places those.
#include <algorithm>
#include <climits>

#include "device_common.cuh"
#include "internal.h"

namespace lj {
namespace {

constexpr int kGThreads = 256;
constexpr int kGItems = 8;
constexpr int kGTile = kGThreads * kGItems;   // keys per tile

template <class Model, class Slot>
__device__ __forceinline__ int64_t key_pslot(const typename Model::Leaf* leaves, const Model& m,
                                             uint64_t x, const Slot& slot) {
  return (int64_t)slot.template at<Model>(Model::load_leaf(leaves, m.leaf(x)), x);
}

// The RadixSpline hash needs no leaf record (no RMI lookup).
template <class Model>
__device__ __forceinline__ int64_t key_pslot(const typename Model::Leaf*, const Model&,
                                             uint64_t x, const RsHashSlot& slot) {
  return (int64_t)slot.at(x);
}

__device__ __forceinline__ int64_t warp_max(int64_t v) {
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) v = max(v, (int64_t)__shfl_xor_sync(0xffffffffu, v, d));
  return v;
}

template <class Model, class Slot>
__global__ void __launch_bounds__(kGThreads)
    grmi_dmax_kernel(const uint64_t* __restrict__ R, uint64_t n, const typename Model::Leaf* leaves,
                     Model model, Slot scale, int64_t* __restrict__ tile_max) {
  __shared__ int64_t s_w[kGThreads / 32];
  const uint64_t i0 = (uint64_t)blockIdx.x * kGTile;
  int64_t mx = LLONG_MIN;
#pragma unroll 1
  for (int k = 0; k < kGItems; ++k) {
    const uint64_t i = i0 + (uint64_t)k * kGThreads + threadIdx.x;
    if (i < n) mx = max(mx, key_pslot(leaves, model, R[i], scale) - (int64_t)i);
  }
  mx = warp_max(mx);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t t = LLONG_MIN;
    for (int w = 0; w < kGThreads / 32; ++w) t = max(t, s_w[w]);
    tile_max[blockIdx.x] = t;
  }
}

// Exclusive scan (max, or sum when SUM) of `tiles` values in one block of
// 1024 threads (each thread a contiguous run of tiles); all[0] = the
// reduction of all.
template <bool SUM>
__global__ void __launch_bounds__(1024)
    grmi_prefix_kernel(const int64_t* __restrict__ tile_max, uint32_t tiles,
                       int64_t* __restrict__ tile_prefix, int64_t* __restrict__ all_max) {
  __shared__ int64_t s[1024];
  const int64_t id = SUM ? 0 : LLONG_MIN;
  auto op = [](int64_t a, int64_t b) { return SUM ? a + b : max(a, b); };
  const uint32_t per = (tiles + 1023) / 1024;
  const uint32_t b = threadIdx.x * per, e = min(tiles, b + per);
  int64_t mx = id;
  for (uint32_t t = b; t < e; ++t) mx = op(mx, tile_max[t]);
  s[threadIdx.x] = mx;
  __syncthreads();
  for (int d = 1; d < 1024; d <<= 1) {   // inclusive Hillis-Steele scan
    const int64_t v = threadIdx.x >= (unsigned)d ? s[threadIdx.x - d] : id;
    __syncthreads();
    s[threadIdx.x] = op(s[threadIdx.x], v);
    __syncthreads();
  }
  int64_t run = threadIdx.x ? s[threadIdx.x - 1] : id;
  for (uint32_t t = b; t < e; ++t) {
    tile_prefix[t] = run;
    run = op(run, tile_max[t]);
  }
  if (threadIdx.x == 1023) all_max[0] = s[1023];
}

// Distinct keys of the sorted R (learned hash index): per tile, the number of
// run starts (positions i with i == 0 or R[i] != R[i-1]) ...
__global__ void __launch_bounds__(kGThreads)
    run_count_kernel(const uint64_t* __restrict__ R, uint64_t n, int64_t* __restrict__ tile_cnt) {
  __shared__ int64_t s_w[kGThreads / 32];
  const uint64_t i0 = (uint64_t)blockIdx.x * kGTile;
  int64_t c = 0;
  for (int k = 0; k < kGItems; ++k) {
    const uint64_t i = i0 + (uint64_t)k * kGThreads + threadIdx.x;
    if (i < n && (i == 0 || R[i] != R[i - 1])) ++c;
  }
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) c += __shfl_xor_sync(0xffffffffu, c, d);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t t = 0;
    for (int w = 0; w < kGThreads / 32; ++w) t += s_w[w];
    tile_cnt[blockIdx.x] = t;
  }
}

// ... then each run start's key and position at its rank among the runs.
__global__ void __launch_bounds__(kGThreads)
    run_write_kernel(const uint64_t* __restrict__ R, uint64_t n,
                     const int64_t* __restrict__ tile_off, uint64_t* __restrict__ dkey,
                     uint32_t* __restrict__ dfirst) {
  __shared__ int64_t s_w[kGThreads / 32];
  const uint64_t i0 = (uint64_t)blockIdx.x * kGTile + (uint64_t)threadIdx.x * kGItems;
  bool f[kGItems];
  int64_t c = 0;
#pragma unroll
  for (int k = 0; k < kGItems; ++k) {
    const uint64_t i = i0 + k;
    f[k] = i < n && (i == 0 || R[i] != R[i - 1]);
    c += f[k];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t inc = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t v = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += v;
  }
  if (lane == 31) s_w[warp] = inc;
  __syncthreads();
  int64_t d = tile_off[blockIdx.x] + inc - c;
  for (int w = 0; w < warp; ++w) d += s_w[w];
#pragma unroll
  for (int k = 0; k < kGItems; ++k)
    if (f[k]) {
      dkey[d] = R[i0 + k];
      dfirst[d] = (uint32_t)(i0 + k);
      ++d;
    }
}

template <class Model, class Slot>
__global__ void __launch_bounds__(kGThreads)
    grmi_fill_kernel(const uint64_t* __restrict__ R, uint64_t n, const typename Model::Leaf* leaves,
                     Model model, Slot scale, const int64_t* __restrict__ tile_prefix,
                     uint64_t* __restrict__ gkeys, uint32_t* __restrict__ gpos,
                     unsigned long long* __restrict__ disp_stats) {
  __shared__ uint64_t s_key[kGTile];
  __shared__ uint32_t s_slot[kGTile];
  __shared__ int64_t s_w[kGThreads / 32];
  __shared__ unsigned long long s_sum[kGThreads / 32], s_max[kGThreads / 32];
  const uint64_t i0 = (uint64_t)blockIdx.x * kGTile;
  const uint32_t cnt = (uint32_t)(n - i0 < (uint64_t)kGTile ? n - i0 : (uint64_t)kGTile);
  for (uint32_t k = threadIdx.x; k < cnt; k += kGThreads) s_key[k] = R[i0 + k];
  __syncthreads();
  // this thread's kGItems consecutive keys: d = pslot - i and its running max
  const uint32_t k0 = threadIdx.x * kGItems;
  int64_t d[kGItems], ps[kGItems];
  int64_t mx = LLONG_MIN;
#pragma unroll
  for (int k = 0; k < kGItems; ++k) {
    ps[k] = 0;
    d[k] = LLONG_MIN;
    if (k0 + k < cnt) {
      ps[k] = key_pslot(leaves, model, s_key[k0 + k], scale);
      d[k] = ps[k] - (int64_t)(i0 + k0 + k);
    }
    mx = max(mx, d[k]);
  }
  // exclusive max-scan of the threads' maxima across the block
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t inc = mx;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t v = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc = max(inc, v);
  }
  if (lane == 31) s_w[warp] = inc;
  __syncthreads();
  int64_t run = tile_prefix[blockIdx.x];
  for (int w = 0; w < warp; ++w) run = max(run, s_w[w]);
  const int64_t excl_lane = __shfl_up_sync(0xffffffffu, inc, 1);
  if (lane > 0) run = max(run, excl_lane);
  unsigned long long dsum = 0, dmax = 0;
#pragma unroll
  for (int k = 0; k < kGItems; ++k)
    if (k0 + k < cnt) {
      run = max(run, d[k]);
      const int64_t slot = (int64_t)(i0 + k0 + k) + run;
      s_slot[k0 + k] = (uint32_t)slot;
      const unsigned long long disp = (unsigned long long)(slot - ps[k]);
      dsum += disp;
      dmax = max(dmax, disp);
    }
  // displacement statistics (sum and max over R's keys)
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
    dmax = max(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
  }
  if (lane == 0) {
    s_sum[warp] = dsum;
    s_max[warp] = dmax;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long a = 0, b = 0;
    for (int w = 0; w < kGThreads / 32; ++w) {
      a += s_sum[w];
      b = max(b, s_max[w]);
    }
    atomicAdd(disp_stats, a);
    atomicMax(disp_stats + 1, b);
  }
  // the slots this tile owns: (slot of key i0 - 1, slot of its last key]
  const int64_t prev = blockIdx.x == 0 ? -1 : (int64_t)(i0 - 1) + tile_prefix[blockIdx.x];
  const int64_t last = s_slot[cnt - 1];
  for (int64_t sl = prev + 1 + threadIdx.x; sl <= last; sl += kGThreads) {
    uint32_t a = 0, len = cnt;   // first key of the tile placed at or after sl
    while (len > 0) {
      const uint32_t half = len >> 1;
      if ((int64_t)s_slot[a + half] < sl) {
        a += half + 1;
        len -= half + 1;
      } else {
        len = half;
      }
    }
    gkeys[sl] = s_key[a];
    gpos[sl] = (uint32_t)(i0 + a);
  }
}

// Learned hash: every slot's range (first position | count << 32) from its
// payload (the distinct-key rank d): [first[d], first[d+1]); rank D: none.
__global__ void lhash_range_kernel(const uint32_t* __restrict__ gpos,
                                   const uint32_t* __restrict__ dfirst, uint64_t C, uint32_t D,
                                   uint64_t* __restrict__ hrange) {
  for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < C;
       s += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t d = gpos[s];
    const uint32_t a = dfirst[d];   // d <= D, dfirst[D] = n
    const uint32_t c = d < D ? dfirst[d + 1] - a : 0u;
    hrange[s] = ((uint64_t)c << 32) | a;
  }
}

__global__ void grmi_tail_kernel(uint64_t* __restrict__ gkeys, uint32_t* __restrict__ gpos,
                                 uint64_t from, uint64_t C, uint32_t n) {
  for (uint64_t s = from + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < C;
       s += (uint64_t)gridDim.x * blockDim.x) {
    gkeys[s] = ~0ull;
    gpos[s] = n;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) gpos[C] = n;
}

// ------------------------------------------------------------ RadixSpline --
//
// RadixSpline over R's distinct keys (Section 2.D), the hash of the
// RSHASH-INLJ learned hash index (Section 3.C).  CDF points: the distinct
// keys dk[d] with the position of their first copy dfirst[d].  Spline points
// are chosen greedily in one pass (the error corridor of Neumann and Michel,
// 2008, as RadixSpline does): from the last spline point b every further
// point q narrows a corridor of slopes to [q.y - eps, q.y + eps]; the first
// point whose own slope from b leaves the corridor makes the point before it
// a spline point.  Every CDF point then lies within eps positions of the line
// between its spline points.  One GPU thread runs the pass over a chunk of
// kRsChunk distinct keys (each chunk starts and ends with a spline point):
// a counting launch, a scan of the counts, a writing launch.  Slopes are
// compared exactly (128-bit cross products).  Then the radix table over the
// top bits of (key - k_0) of the spline points, and 1 / (x_{i+1} - x_i) for
// the interpolation.
constexpr uint64_t kRsChunk = 1024;

__device__ __forceinline__ bool slope_lt(__int128 a, __int128 b, __int128 c, __int128 d) {
  return a * d < c * b;   // a/b < c/d for b, d > 0
}

template <bool WRITE>
__global__ void rs_spline_kernel(const uint64_t* __restrict__ dk, const uint32_t* __restrict__ dy,
                                 uint64_t D, uint32_t eps, int64_t* __restrict__ cnt,
                                 const int64_t* __restrict__ off, uint64_t* __restrict__ sx,
                                 uint32_t* __restrict__ sy) {
  const uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t c0 = c * kRsChunk;
  if (c0 >= D) return;
  const uint64_t c1 = min(D, c0 + kRsChunk);
  uint64_t S = 0;
  const uint64_t o = WRITE ? (uint64_t)off[c] : 0;
  auto emit = [&](uint64_t d) {
    if (WRITE) {
      sx[o + S] = dk[d];
      sy[o + S] = dy[d];
    }
    ++S;
  };
  uint64_t base = c0;
  emit(base);
  __int128 up_dy = 0, up_dx = 1, lo_dy = 0, lo_dx = 1;
  bool open = false;
  for (uint64_t d = c0 + 1; d < c1; ++d) {
    const __int128 dx = (__int128)(dk[d] - dk[base]);
    const __int128 y = (__int128)dy[d] - (__int128)dy[base];
    if (!open) {
      up_dy = y + eps;
      up_dx = dx;
      lo_dy = y - eps;
      lo_dx = dx;
      open = true;
      continue;
    }
    if (slope_lt(up_dy, up_dx, y, dx) || slope_lt(y, dx, lo_dy, lo_dx)) {
      base = d - 1;   // d leaves the corridor: the point before it is a spline point
      emit(base);
      const __int128 dx2 = (__int128)(dk[d] - dk[base]);
      const __int128 y2 = (__int128)dy[d] - (__int128)dy[base];
      up_dy = y2 + eps;
      up_dx = dx2;
      lo_dy = y2 - eps;
      lo_dx = dx2;
      continue;
    }
    if (slope_lt(y + eps, dx, up_dy, up_dx)) {
      up_dy = y + eps;
      up_dx = dx;
    }
    if (slope_lt(lo_dy, lo_dx, y - eps, dx)) {
      lo_dy = y - eps;
      lo_dx = dx;
    }
  }
  if (c1 - 1 != base) emit(c1 - 1);
  if (!WRITE) cnt[c] = (int64_t)S;
}

// Radix table (table[b] = spline points with prefix below b, b = 0..T) and
// the reciprocal spline-segment widths.
__global__ void rs_table_kernel(const uint64_t* __restrict__ sx, uint32_t S, uint64_t kmin,
                                uint32_t shift, uint64_t T, uint32_t* __restrict__ table,
                                double* __restrict__ rcp) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < S;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t p = (sx[i] - kmin) >> shift;
    const int64_t pp = i ? (int64_t)((sx[i - 1] - kmin) >> shift) : -1;
    for (int64_t b = pp + 1; b <= (int64_t)p; ++b) table[b] = (uint32_t)i;
    if (i + 1 == S)
      for (uint64_t b = p + 1; b <= T; ++b) table[b] = S;
    rcp[i] = i + 1 < S ? 1.0 / (double)(sx[i + 1] - sx[i]) : 0.0;
  }
}

// Model-based insertion of the n sorted keys src[] into the index's gapped
// arrays, key i at max(slot(src[i]), slot of key i-1 + 1); payload = i.
template <class Model, class Slot>
int build_gapped(lj_index* idx, Model model, Slot scale, const uint64_t* src, uint64_t n,
                 uint64_t min_slots, cudaStream_t s) {
  const auto* leaves = (const typename Model::Leaf*)idx->leaves;
  const uint32_t tiles = (uint32_t)((n + kGTile - 1) / kGTile);
  char* ws = nullptr;
  const size_t b_tiles = ((size_t)std::max<uint32_t>(tiles, 1) * 8 + 255) / 256 * 256;
  LJ_CUDA(scratch_alloc((void**)&ws, 256 + 2 * b_tiles, s));
  int64_t* all_max = (int64_t*)ws;
  unsigned long long* stats = (unsigned long long*)(ws + 64);
  int64_t* tile_max = (int64_t*)(ws + 256);
  int64_t* tile_prefix = (int64_t*)(ws + 256 + b_tiles);
  int rc = 0;
  cudaError_t ce = cudaSuccess;
  int64_t h_max = 0;
  unsigned long long h_stats[2] = {0, 0};
  uint64_t C = 0;
  do {
    if ((ce = cudaMemsetAsync(ws, 0, 256, s)) != cudaSuccess) break;
    if (n > 0) {
      grmi_dmax_kernel<Model, Slot><<<tiles, kGThreads, 0, s>>>(src, n, leaves, model, scale, tile_max);
      grmi_prefix_kernel<false><<<1, 1024, 0, s>>>(tile_max, tiles, tile_prefix, all_max);
      if ((ce = cudaGetLastError()) != cudaSuccess) break;
      if ((ce = cudaMemcpyAsync(&h_max, all_max, 8, cudaMemcpyDeviceToHost, s)) != cudaSuccess) break;
      if ((ce = cudaStreamSynchronize(s)) != cudaSuccess) break;
    }
    const uint64_t last = n ? (uint64_t)((int64_t)(n - 1) + h_max) : 0;   // slot of the last key
    C = std::max<uint64_t>(n ? last + 1 : 0, min_slots);
    if (C >= 0xFFFFFFFFull) {
      rc = fail(LJ_E_INVAL, "grmi_build: %llu slots exceed the 32-bit slot range; use fewer gaps",
                (unsigned long long)C);
      break;
    }
    cudaFree(idx->gkeys);
    cudaFree(idx->gpos);
    idx->gkeys = nullptr;
    idx->gpos = nullptr;
    if ((ce = cudaMalloc(&idx->gkeys, std::max<uint64_t>(C, 1) * 8)) != cudaSuccess) break;
    if ((ce = cudaMalloc(&idx->gpos, (C + 1) * 4)) != cudaSuccess) break;
    if (n > 0)
      grmi_fill_kernel<Model, Slot><<<tiles, kGThreads, 0, s>>>(src, n, leaves, model, scale,
                                                                tile_prefix, idx->gkeys, idx->gpos,
                                                                stats);
    const uint64_t from = n ? last + 1 : 0;
    const uint64_t rest = C - from;
    const unsigned tb = (unsigned)std::min<uint64_t>(4096, std::max<uint64_t>(1, (rest + 255) / 256));
    grmi_tail_kernel<<<tb, 256, 0, s>>>(idx->gkeys, idx->gpos, from, C, (uint32_t)n);
    if ((ce = cudaGetLastError()) != cudaSuccess) break;
    if ((ce = cudaMemcpyAsync(h_stats, stats, 16, cudaMemcpyDeviceToHost, s)) != cudaSuccess) break;
    if ((ce = cudaStreamSynchronize(s)) != cudaSuccess) break;
  } while (0);
  scratch_free(ws, s);
  if (!rc && ce != cudaSuccess) rc = fail_cuda(ce, "grmi_build");
  if (rc) {
    grmi_release(idx);
    return rc;
  }
  idx->gslots = (uint32_t)C;
  idx->gstats.slots = C;
  idx->gstats.mean_disp = n ? (double)h_stats[0] / (double)n : 0.0;
  idx->gstats.max_disp = h_stats[1];
  return 0;
}

// Distinct keys of R: dkey[D] (scratch, caller frees) and the index's
// dfirst[D + 1] (dfirst[D] = n).
int distinct_keys(lj_index* idx, uint64_t** dkey_out, uint64_t* D_out, cudaStream_t s) {
  const uint64_t n = idx->n;
  const uint32_t tiles = (uint32_t)((n + kGTile - 1) / kGTile);
  const size_t b_tiles = ((size_t)std::max<uint32_t>(tiles, 1) * 8 + 255) / 256 * 256;
  char* ws = nullptr;
  LJ_CUDA(scratch_alloc((void**)&ws, 256 + 2 * b_tiles, s));
  int64_t* total = (int64_t*)ws;
  int64_t* tile_cnt = (int64_t*)(ws + 256);
  int64_t* tile_off = (int64_t*)(ws + 256 + b_tiles);
  int64_t D = 0;
  cudaError_t ce = cudaMemsetAsync(ws, 0, 256, s);
  if (ce == cudaSuccess && n > 0) {
    run_count_kernel<<<tiles, kGThreads, 0, s>>>(idx->R, n, tile_cnt);
    grmi_prefix_kernel<true><<<1, 1024, 0, s>>>(tile_cnt, tiles, tile_off, total);
    ce = cudaMemcpyAsync(&D, total, 8, cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
  }
  uint64_t* dkey = nullptr;
  if (ce == cudaSuccess) ce = scratch_alloc((void**)&dkey, std::max<int64_t>(D, 1) * 8, s);
  if (ce == cudaSuccess) ce = cudaMalloc(&idx->dfirst, (D + 1) * 4);
  if (ce == cudaSuccess && n > 0)
    run_write_kernel<<<tiles, kGThreads, 0, s>>>(idx->R, n, tile_off, dkey, idx->dfirst);
  const uint32_t n32 = (uint32_t)n;
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(idx->dfirst + D, &n32, 4, cudaMemcpyHostToDevice, s);
  if (ce == cudaSuccess) ce = cudaGetLastError();
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
  scratch_free(ws, s);
  if (ce != cudaSuccess) {
    if (dkey) scratch_free(dkey, s);
    return fail_cuda(ce, "lhash_build: distinct keys");
  }
  *dkey_out = dkey;
  *D_out = (uint64_t)D;
  return 0;
}

}  // namespace

void grmi_release(lj_index* idx) {
  if (idx->gkeys) cudaFree(idx->gkeys);
  if (idx->gpos) cudaFree(idx->gpos);
  if (idx->dfirst) cudaFree(idx->dfirst);
  if (idx->hrange) cudaFree(idx->hrange);
  idx->gkeys = nullptr;
  idx->gpos = nullptr;
  idx->dfirst = nullptr;
  idx->hrange = nullptr;
  if (idx->rs_x) cudaFree(idx->rs_x);
  if (idx->rs_y) cudaFree(idx->rs_y);
  if (idx->rs_rcp) cudaFree(idx->rs_rcp);
  if (idx->rs_table) cudaFree(idx->rs_table);
  idx->rs_x = nullptr;
  idx->rs_y = nullptr;
  idx->rs_rcp = nullptr;
  idx->rs_table = nullptr;
  idx->rs_S = idx->rs_shift = idx->rs_rbits = idx->rs_eps = 0;
  idx->rs_kmin = idx->rs_kmax = 0;
  idx->gslots = 0;
  idx->gscale = 0;
  idx->gkind = 0;
  idx->ndistinct = 0;
  idx->hbuckets = 0;
  idx->gstats = lj_grmi_stats{};
}

}  // namespace lj

extern "C" int grmi_build(lj_index* index, uint32_t gaps, lj_stream_t stream) {
  using namespace lj;
  if (!index) return fail(LJ_E_INVAL, "grmi_build: index is NULL");
  if (gaps > 16) return fail(LJ_E_INVAL, "grmi_build: gaps = %u must be at most 16", gaps);
  if (current_device() != index->device)
    return fail(LJ_E_INVAL, "grmi_build: index lives on device %d, current device is %d",
                index->device, current_device());
  if ((uint64_t)(1 + gaps) * index->n >= 0xFFFFFFFFull)
    return fail(LJ_E_INVAL, "grmi_build: (1 + gaps) * n = %llu slots exceed the 32-bit slot range",
                (unsigned long long)(1 + gaps) * index->n);
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return fail(LJ_E_CUDA, "grmi_build: cudaEventCreate failed");
  cudaEventRecord(e0, s);
  int rc;
  grmi_release(index);
  const GappedSlot slot{1 + gaps};
  const uint64_t min_slots = (uint64_t)(1 + gaps) * index->n;
  if (index->precision == LJ_FP64)
    rc = build_gapped(index, ModelF64::make(index->root_f64[0], index->root_f64[1], index->L), slot,
                      index->R, index->n, min_slots, s);
  else
    rc = build_gapped(index, ModelF32::make(index->root_f32[0], index->root_f32[1], index->L), slot,
                      index->R, index->n, min_slots, s);
  if (!rc) {
    index->gscale = 1 + gaps;
    index->gstats.gaps = gaps;
    index->gstats.kind = 0;
    index->gstats.distinct = 0;
  }
  cudaEventRecord(e1, s);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  if (int r2 = take_device_errors(index->device, s)) {
    grmi_release(index);
    return r2;
  }
  index->gstats.build_ms = ms;
  return LJ_OK;
}

extern "C" int lhash_build(lj_index* index, uint32_t spk, lj_stream_t stream) {
  using namespace lj;
  if (!index) return fail(LJ_E_INVAL, "lhash_build: index is NULL");
  if (spk < 1 || spk > 16) return fail(LJ_E_INVAL, "lhash_build: spk = %u must be in [1, 16]", spk);
  if (current_device() != index->device)
    return fail(LJ_E_INVAL, "lhash_build: index lives on device %d, current device is %d",
                index->device, current_device());
  if ((uint64_t)spk * index->n + 8 >= 0xFFFFFFFFull)
    return fail(LJ_E_INVAL, "lhash_build: spk * n exceeds the 32-bit slot range");
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return fail(LJ_E_CUDA, "lhash_build: cudaEventCreate failed");
  cudaEventRecord(e0, s);
  grmi_release(index);
  uint64_t* dkey = nullptr;
  uint64_t D = 0;
  int rc = distinct_keys(index, &dkey, &D, s);
  if (!rc) {
    const uint64_t B = std::max<uint64_t>(1, ((uint64_t)spk * D + 3) / 4);
    const HashSlot slot{B, index->n + 1};
    if (index->precision == LJ_FP64)
      rc = build_gapped(index, ModelF64::make(index->root_f64[0], index->root_f64[1], index->L), slot,
                        dkey, D, 4 * B, s);
    else
      rc = build_gapped(index, ModelF32::make(index->root_f32[0], index->root_f32[1], index->L), slot,
                        dkey, D, 4 * B, s);
    if (!rc) {   // per-slot ranges, so that a probe reads its matches with one load
      const uint64_t C = index->gslots;
      cudaError_t ce = cudaMalloc(&index->hrange, std::max<uint64_t>(C, 1) * 8);
      if (ce == cudaSuccess) {
        const unsigned g = (unsigned)std::min<uint64_t>(8192, std::max<uint64_t>(1, (C + 255) / 256));
        lhash_range_kernel<<<g, 256, 0, s>>>(index->gpos, index->dfirst, C, (uint32_t)D,
                                              index->hrange);
        ce = cudaGetLastError();
      }
      if (ce != cudaSuccess) rc = fail_cuda(ce, "lhash_build: slot ranges");
    }
    if (!rc) {
      index->gkind = 1;
      index->ndistinct = D;
      index->hbuckets = B;
      index->gstats.gaps = spk;
      index->gstats.kind = 1;
      index->gstats.distinct = D;
    }
  }
  if (dkey) scratch_free(dkey, s);
  cudaEventRecord(e1, s);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!rc) rc = take_device_errors(index->device, s);
  if (rc) {
    grmi_release(index);
    return rc;
  }
  index->gstats.build_ms = ms;
  return LJ_OK;
}

namespace lj {
namespace {

// The RadixSpline of the index's distinct keys (dkey[D], index->dfirst) into
// the index's rs_* arrays.
int build_radix_spline(lj_index* idx, const uint64_t* dkey, uint64_t D, uint32_t eps,
                       uint32_t rbits, cudaStream_t s) {
  const uint64_t chunks = std::max<uint64_t>(1, (D + kRsChunk - 1) / kRsChunk);
  const size_t b_c = (chunks * 8 + 255) / 256 * 256;
  char* ws = nullptr;
  LJ_CUDA(scratch_alloc((void**)&ws, 256 + 2 * b_c, s));
  int64_t* total = (int64_t*)ws;
  uint64_t* ends = (uint64_t*)(ws + 64);   // dkey[0], dkey[D-1]
  int64_t* cnt = (int64_t*)(ws + 256);
  int64_t* off = (int64_t*)(ws + 256 + b_c);
  int64_t S = 0;
  uint64_t hends[2] = {0, 0};
  cudaError_t ce = cudaMemsetAsync(ws, 0, 256, s);
  const unsigned g = (unsigned)((chunks + 127) / 128);
  if (ce == cudaSuccess && D > 0) {
    rs_spline_kernel<false><<<g, 128, 0, s>>>(dkey, idx->dfirst, D, eps, cnt, nullptr, nullptr,
                                              nullptr);
    grmi_prefix_kernel<true><<<1, 1024, 0, s>>>(cnt, (uint32_t)chunks, off, total);
    ce = cudaMemcpyAsync(ends, dkey, 8, cudaMemcpyDeviceToDevice, s);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(ends + 1, dkey + D - 1, 8, cudaMemcpyDeviceToDevice, s);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(&S, total, 8, cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(hends, ends, 16, cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
  }
  const uint64_t T = 1ull << rbits;
  uint32_t bl = 0;
  for (uint64_t v = hends[1] - hends[0]; v; v >>= 1) ++bl;
  const uint32_t shift = bl > rbits ? bl - rbits : 0;
  if (ce == cudaSuccess) ce = cudaMalloc(&idx->rs_x, std::max<int64_t>(S, 1) * 8);
  if (ce == cudaSuccess) ce = cudaMalloc(&idx->rs_y, std::max<int64_t>(S, 1) * 4);
  if (ce == cudaSuccess) ce = cudaMalloc(&idx->rs_rcp, std::max<int64_t>(S, 1) * 8);
  if (ce == cudaSuccess) ce = cudaMalloc(&idx->rs_table, (T + 1) * 4);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(idx->rs_table, 0, (T + 1) * 4, s);
  if (ce == cudaSuccess && D > 0) {
    rs_spline_kernel<true><<<g, 128, 0, s>>>(dkey, idx->dfirst, D, eps, nullptr, off, idx->rs_x,
                                             idx->rs_y);
    const unsigned gt = (unsigned)std::min<uint64_t>(4096, std::max<uint64_t>(1, (S + 255) / 256));
    rs_table_kernel<<<gt, 256, 0, s>>>(idx->rs_x, (uint32_t)S, hends[0], shift, T, idx->rs_table,
                                       idx->rs_rcp);
    ce = cudaGetLastError();
  }
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
  scratch_free(ws, s);
  if (ce != cudaSuccess) return fail_cuda(ce, "lhash_build_rs: RadixSpline");
  idx->rs_S = (uint32_t)S;
  idx->rs_shift = shift;
  idx->rs_rbits = rbits;
  idx->rs_eps = eps;
  idx->rs_kmin = hends[0];
  idx->rs_kmax = hends[1];
  return 0;
}

}  // namespace
}  // namespace lj

extern "C" int lhash_build_rs(lj_index* index, uint32_t spk, uint32_t eps, uint32_t radix_bits,
                              lj_stream_t stream) {
  using namespace lj;
  if (!index) return fail(LJ_E_INVAL, "lhash_build_rs: index is NULL");
  if (spk < 1 || spk > 16) return fail(LJ_E_INVAL, "lhash_build_rs: spk = %u must be in [1, 16]", spk);
  if (eps > (1u << 20)) return fail(LJ_E_INVAL, "lhash_build_rs: eps = %u above 2^20", eps);
  if (radix_bits < 1 || radix_bits > 24)
    return fail(LJ_E_INVAL, "lhash_build_rs: radix_bits = %u must be in [1, 24]", radix_bits);
  if (current_device() != index->device)
    return fail(LJ_E_INVAL, "lhash_build_rs: index lives on device %d, current device is %d",
                index->device, current_device());
  if ((uint64_t)spk * index->n + 8 >= 0xFFFFFFFFull)
    return fail(LJ_E_INVAL, "lhash_build_rs: spk * n exceeds the 32-bit slot range");
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return fail(LJ_E_CUDA, "lhash_build_rs: cudaEventCreate failed");
  cudaEventRecord(e0, s);
  grmi_release(index);
  uint64_t* dkey = nullptr;
  uint64_t D = 0;
  int rc = distinct_keys(index, &dkey, &D, s);
  if (!rc) rc = build_radix_spline(index, dkey, D, eps, radix_bits, s);
  if (!rc) {
    const uint64_t B = std::max<uint64_t>(1, ((uint64_t)spk * D + 3) / 4);
    const RsHashSlot slot{RsDev{index->rs_x, index->rs_y, index->rs_rcp, index->rs_table,
                                index->rs_kmin, index->rs_kmax, index->n, index->rs_S,
                                index->rs_shift},
                          B, index->n + 1};
    if (index->precision == LJ_FP64)
      rc = build_gapped(index, ModelF64::make(index->root_f64[0], index->root_f64[1], index->L),
                        slot, dkey, D, 4 * B, s);
    else
      rc = build_gapped(index, ModelF32::make(index->root_f32[0], index->root_f32[1], index->L),
                        slot, dkey, D, 4 * B, s);
    if (!rc) {   // per-slot ranges, as lhash_build
      const uint64_t C = index->gslots;
      cudaError_t ce = cudaMalloc(&index->hrange, std::max<uint64_t>(C, 1) * 8);
      if (ce == cudaSuccess) {
        const unsigned g = (unsigned)std::min<uint64_t>(8192, std::max<uint64_t>(1, (C + 255) / 256));
        lhash_range_kernel<<<g, 256, 0, s>>>(index->gpos, index->dfirst, C, (uint32_t)D,
                                              index->hrange);
        ce = cudaGetLastError();
      }
      if (ce != cudaSuccess) rc = fail_cuda(ce, "lhash_build_rs: slot ranges");
    }
    if (!rc) {
      index->gkind = kRsHash;
      index->ndistinct = D;
      index->hbuckets = B;
      index->gstats.gaps = spk;
      index->gstats.kind = 2;
      index->gstats.distinct = D;
    }
  }
  if (dkey) scratch_free(dkey, s);
  cudaEventRecord(e1, s);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!rc) rc = take_device_errors(index->device, s);
  if (rc) {
    grmi_release(index);
    return rc;
  }
  index->gstats.build_ms = ms;
  return LJ_OK;
}

extern "C" int rs_export(const lj_index* index, uint64_t* sx_host, uint32_t* sy_host,
                         uint32_t* table_host, uint32_t* shift_host, uint64_t* count_host) {
  using namespace lj;
  if (!index) return fail(LJ_E_INVAL, "rs_export: index is NULL");
  if (index->gkind != kRsHash || !index->rs_table)
    return fail(LJ_E_STATE, "rs_export: the index has no RadixSpline (lhash_build_rs)");
  if (count_host) *count_host = index->rs_S;
  if (shift_host) *shift_host = index->rs_shift;
  if (sx_host && index->rs_S)
    LJ_CUDA(cudaMemcpy(sx_host, index->rs_x, (size_t)index->rs_S * 8, cudaMemcpyDeviceToHost));
  if (sy_host && index->rs_S)
    LJ_CUDA(cudaMemcpy(sy_host, index->rs_y, (size_t)index->rs_S * 4, cudaMemcpyDeviceToHost));
  if (table_host)
    LJ_CUDA(cudaMemcpy(table_host, index->rs_table, ((1ull << index->rs_rbits) + 1) * 4,
                       cudaMemcpyDeviceToHost));
  return LJ_OK;
}

extern "C" int lhash_export_first(const lj_index* index, uint32_t* first_host) {
  using namespace lj;
  if (!index || !first_host) return fail(LJ_E_INVAL, "lhash_export_first: NULL argument");
  if ((index->gkind != 1 && index->gkind != 2) || !index->dfirst)
    return fail(LJ_E_STATE, "lhash_export_first: the index has no learned hash table");
  LJ_CUDA(cudaMemcpy(first_host, index->dfirst, (index->ndistinct + 1) * 4, cudaMemcpyDeviceToHost));
  return LJ_OK;
}

extern "C" int grmi_drop(lj_index* index) {
  if (!index) return lj::fail(LJ_E_INVAL, "grmi_drop: index is NULL");
  lj::grmi_release(index);
  return LJ_OK;
}

extern "C" int grmi_stats(const lj_index* index, lj_grmi_stats* out) {
  if (!index || !out) return lj::fail(LJ_E_INVAL, "grmi_stats: NULL argument");
  if (!index->gpos) return lj::fail(LJ_E_STATE, "grmi_stats: the index has no gapped arrays");
  *out = index->gstats;
  return LJ_OK;
}

extern "C" int grmi_export(const lj_index* index, uint64_t* keys_host, uint32_t* pos_host) {
  using namespace lj;
  if (!index) return fail(LJ_E_INVAL, "grmi_export: index is NULL");
  if (!index->gpos) return fail(LJ_E_STATE, "grmi_export: the index has no gapped arrays");
  const uint64_t C = index->gslots;
  if (keys_host && C) LJ_CUDA(cudaMemcpy(keys_host, index->gkeys, C * 8, cudaMemcpyDeviceToHost));
  if (pos_host) LJ_CUDA(cudaMemcpy(pos_host, index->gpos, (C + 1) * 4, cudaMemcpyDeviceToHost));
  return LJ_OK;
}

namespace lj {
int probe_count_impl(const lj_index* idx, const uint64_t* S, uint64_t m, uint32_t* counts,
                     uint64_t* offsets, uint32_t* first, uint64_t* total_dev, uint64_t* total_host,
                     cudaStream_t s);
}  // namespace lj

extern "C" int index_autotune(lj_index* index, const uint64_t* S_sample_dev, uint64_t m_sample,
                              lj_stream_t stream, int* choice, double* ns_per_key) {
  using namespace lj;
  if (!index || !choice) return fail(LJ_E_INVAL, "index_autotune: NULL argument");
  if (m_sample == 0 || !S_sample_dev) return fail(LJ_E_INVAL, "index_autotune: empty sample");
  if (m_sample >= (1ull << 32)) return fail(LJ_E_INVAL, "index_autotune: sample too large");
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  LJ_CUDA(cudaEventCreate(&e0));
  LJ_CUDA(cudaEventCreate(&e1));
  auto setup = [&](int c) -> int {
    index->probe_order = c == LJ_LOOKUP_RMI_BUCKETED ? 1 : c == LJ_LOOKUP_SORTMERGE ? 2 : 0;
    index->use_levels = 0;
    if (c == LJ_LOOKUP_RMI_LEVELS) {
      grmi_release(index);
      return build_key_levels(index, s);
    }
    if (c == LJ_LOOKUP_GRMI) return grmi_build(index, 4, stream);
    if (c == LJ_LOOKUP_LHASH) return lhash_build(index, 4, stream);
    if (c == LJ_LOOKUP_RSHASH) return lhash_build_rs(index, 4, 16, 18, stream);
    grmi_release(index);
    return 0;
  };
  double best = 1e300;
  int best_c = LJ_LOOKUP_RMI, rc = 0;
  for (int c = LJ_LOOKUP_RMI; c <= LJ_LOOKUP_RMI_LEVELS && !rc; ++c) {
    if ((rc = setup(c))) break;
    float ms = 1e30f;
    for (int rep = 0; rep < 4 && !rc; ++rep) {
      cudaEventRecord(e0, s);
      rc = probe_count_impl(index, S_sample_dev, m_sample, nullptr, nullptr, nullptr, nullptr,
                            nullptr, s);
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) rc = fail(LJ_E_CUDA, "index_autotune: sync");
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      if (rep > 0) ms = std::min(ms, t);   // the first run warms up
    }
    const double ns = (double)ms * 1e6 / (double)m_sample;
    if (ns_per_key) ns_per_key[c] = ns;
    if (!rc && ns < best) {
      best = ns;
      best_c = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!rc) rc = take_device_errors(index->device, s);
  if (!rc) rc = setup(best_c);
  if (!rc && !index->use_levels && index->levels) {   // levels not chosen: release them
    cudaStreamSynchronize(s);
    cudaFree(index->levels);
    index->levels = nullptr;
    index->nlev = 0;
  }
  if (rc) {
    grmi_release(index);
    index->probe_order = -1;
    return rc;
  }
  *choice = best_c;
  return LJ_OK;
}
