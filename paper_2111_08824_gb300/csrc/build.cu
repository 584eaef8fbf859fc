// rmi_build / rmi_build_batch: fit two-level linear RMIs over sorted
// relations on the device, k relations at a time.
//
// Section 2.D (Recursive Model Index): a root linear model routes a key to a
// leaf model; each leaf's linear model predicts the position; each leaf keeps
// the minimum and maximum error of its keys.  Fitting is least squares; the
// index is built once, before any join (Section 3.A).
//
// A batch of k relations is built as one segmented pass: every kernel below
// covers all relations (blocks or warps find their relation through prefix
// tables), and rmi_build is the batch of one.  Each relation's arithmetic is
// the same whatever the batch (same blocks of keys, same chunks of leaves,
// same fixed-order reductions), so an index built in a batch is bit for bit
// the index built alone.
//
// Steps (each one kernel over the whole batch):
//   check      R sorted non-decreasing; duplicates present (per relation).
//   A1 root    two passes over R in G blocks of `per` keys (G <= 2048 per
//              relation): means of (key, i*L/n), then the centred sums S_xy,
//              S_xx; a0 = S_xy / S_xx (>= 0), b0 = mean_y - a0 mean_x.
//   A2 bounds  leaf(R[i]) with the deployed root; the root is monotone, so
//              leaf l owns the range [lo_l, lo_{l+1}), found where
//              leaf(R[i-1]) != leaf(R[i]).
//   A3 fits    segmented least squares of (i - lo_l) on (R[i] - R[lo_l])
//              over the leaf ranges.  Leaves are cut into chunks of kChunk
//              keys (an exclusive scan over all leaves of the batch numbers
//              them), one warp per chunk, then one warp per leaf sums its
//              chunks: load balanced whatever the leaf and relation sizes.
//   A4 errors  err_i = (i - lo_l) - floor(a_l * (R[i] - R[lo_l]) + b_l)
//              with the deployed (possibly single-precision) parameters;
//              per-leaf min / max by warp reduction + integer atomics; then
//              the leaf records and per-relation window statistics.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <memory>
#include <vector>

#include "device_common.cuh"
#include "internal.h"

namespace lj {
namespace {

constexpr int kBlock = 256;
constexpr uint32_t kChunk = 2048;        // keys per chunk of a leaf (one warp)
constexpr uint64_t kKeyTile = 8192;      // keys per block of the check and bounds kernels
constexpr uint32_t kRootBlocks = 2048;   // most root partial blocks per relation
constexpr uint64_t kRootKeys = 8192;     // keys per root block below that

// One relation of a batch (device table).
struct RelDesc {
  const uint64_t* R;
  uint64_t n;
  uint64_t per;          // keys per root partial block
  uint32_t L;
  uint32_t leaf_base;    // first leaf of the relation in the batch's leaf numbering
  uint32_t G;            // root partial blocks
  uint32_t g_base;       // first root partial of the relation
  uint32_t t_base;       // first key tile of the relation
  uint32_t pad;
  void* leaves_out;      // the relation's leaf records
};

// Largest j in [0, k) with pre[j] <= v (pre[0] = 0, non-decreasing).
__device__ __forceinline__ uint32_t rel_of(const uint32_t* pre, uint32_t k, uint32_t v) {
  uint32_t a = 0, b = k;
  while (b - a > 1) {
    const uint32_t mid = (a + b) >> 1;
    if (pre[mid] <= v)
      a = mid;
    else
      b = mid;
  }
  return a;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) v = __dadd_rn(v, __shfl_xor_sync(0xffffffffu, v, d));
  return v;
}

// Block sum of two doubles in a fixed order; result valid in thread 0.
__device__ __forceinline__ void block_sum2(double& a, double& b) {
  __shared__ double sa[kBlock / 32], sb[kBlock / 32];
  a = warp_sum_d(a);
  b = warp_sum_d(b);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    sa[w] = a;
    sb[w] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double x = 0.0, y = 0.0;
    for (int i = 0; i < kBlock / 32; ++i) {
      x = __dadd_rn(x, sa[i]);
      y = __dadd_rn(y, sb[i]);
    }
    a = x;
    b = y;
  }
}

__device__ __forceinline__ double pos_scaled(uint64_t i, uint32_t L, uint64_t n) {
  return __ddiv_rn(__dmul_rn((double)i, (double)L), (double)n);
}

// Deployed root model of a relation from its least-squares fit (double).
template <class Model>
__device__ __forceinline__ Model root_model(const double2& f, uint32_t L);
template <>
__device__ __forceinline__ ModelF32 root_model<ModelF32>(const double2& f, uint32_t L) {
  return ModelF32::make(__double2float_rn(f.x), __double2float_rn(f.y), L);
}
template <>
__device__ __forceinline__ ModelF64 root_model<ModelF64>(const double2& f, uint32_t L) {
  return ModelF64::make(f.x, f.y, L);
}

// ------------------------------------------------------------------ checks --

// Block = key tile of one relation: pairs (i, i+1) with i in the tile.
// flags[2j] = unsorted, flags[2j+1] = has duplicates.
__global__ void check_sorted_kernel(const RelDesc* rel, const uint32_t* tpre, uint32_t k,
                                    uint32_t* flags) {
  const uint32_t j = rel_of(tpre, k, blockIdx.x);
  const RelDesc d = rel[j];
  const uint64_t s = (uint64_t)(blockIdx.x - d.t_base) * kKeyTile;
  const uint64_t e = min(d.n > 0 ? d.n - 1 : 0, s + kKeyTile);
  uint32_t unsorted = 0, dup = 0;
  for (uint64_t i = s + threadIdx.x; i < e; i += blockDim.x) {
    const uint64_t a = d.R[i], b = d.R[i + 1];
    unsorted |= a > b;
    dup |= a == b;
  }
  unsorted = __any_sync(0xffffffffu, unsorted);
  dup = __any_sync(0xffffffffu, dup);
  if ((threadIdx.x & 31) == 0) {
    if (unsorted) atomicOr(flags + 2 * j, 1u);
    if (dup) atomicOr(flags + 2 * j + 1, 1u);
  }
}

// --------------------------------------------------------------- A1: root --

// Root partial block b of a relation covers [b*per, min(n, (b+1)*per)).
__global__ void root_pass1_kernel(const RelDesc* rel, const uint32_t* gpre, uint32_t k,
                                  double2* part) {
  const uint32_t j = rel_of(gpre, k, blockIdx.x);
  const RelDesc d = rel[j];
  const uint64_t s = (uint64_t)(blockIdx.x - d.g_base) * d.per, e = min(d.n, s + d.per);
  double sx = 0.0, sy = 0.0;
  for (uint64_t i = s + threadIdx.x; i < e; i += kBlock) {
    sx = __dadd_rn(sx, (double)d.R[i]);
    sy = __dadd_rn(sy, pos_scaled(i, d.L, d.n));
  }
  block_sum2(sx, sy);
  if (threadIdx.x == 0) part[blockIdx.x] = make_double2(sx, sy);
}

// One block per relation: fixed-order sum of its partials; (mean_x, mean_y).
__global__ void root_mean_kernel(const RelDesc* rel, const double2* part, double2* mean) {
  const RelDesc d = rel[blockIdx.x];
  double sx = 0.0, sy = 0.0;
  for (uint32_t i = threadIdx.x; i < d.G; i += kBlock) {
    sx = __dadd_rn(sx, part[d.g_base + i].x);
    sy = __dadd_rn(sy, part[d.g_base + i].y);
  }
  block_sum2(sx, sy);
  if (threadIdx.x == 0)
    mean[blockIdx.x] = d.n ? make_double2(__ddiv_rn(sx, (double)d.n), __ddiv_rn(sy, (double)d.n))
                           : make_double2(0.0, 0.0);
}

__global__ void root_pass2_kernel(const RelDesc* rel, const uint32_t* gpre, uint32_t k,
                                  const double2* mean, double2* part) {
  const uint32_t j = rel_of(gpre, k, blockIdx.x);
  const RelDesc d = rel[j];
  const uint64_t s = (uint64_t)(blockIdx.x - d.g_base) * d.per, e = min(d.n, s + d.per);
  const double mx = mean[j].x, my = mean[j].y;
  double sxy = 0.0, sxx = 0.0;
  for (uint64_t i = s + threadIdx.x; i < e; i += kBlock) {
    const double dx = __dsub_rn((double)d.R[i], mx);
    const double dy = __dsub_rn(pos_scaled(i, d.L, d.n), my);
    sxy = __dadd_rn(sxy, __dmul_rn(dx, dy));
    sxx = __dadd_rn(sxx, __dmul_rn(dx, dx));
  }
  block_sum2(sxy, sxx);
  if (threadIdx.x == 0) part[blockIdx.x] = make_double2(sxy, sxx);
}

// One block per relation: root = (a0, b0) least squares, slope clamped >= 0.
__global__ void root_final_kernel(const RelDesc* rel, const double2* part, const double2* mean,
                                  double2* root) {
  const RelDesc d = rel[blockIdx.x];
  double sxy = 0.0, sxx = 0.0;
  for (uint32_t i = threadIdx.x; i < d.G; i += kBlock) {
    sxy = __dadd_rn(sxy, part[d.g_base + i].x);
    sxx = __dadd_rn(sxx, part[d.g_base + i].y);
  }
  block_sum2(sxy, sxx);
  if (threadIdx.x == 0) {
    if (d.n == 0) {
      root[blockIdx.x] = make_double2(0.0, 0.0);
      return;
    }
    double a = sxx > 0.0 ? __ddiv_rn(sxy, sxx) : 0.0;
    if (!(a > 0.0)) a = 0.0;
    root[blockIdx.x] =
        make_double2(a, __dsub_rn(mean[blockIdx.x].y, __dmul_rn(a, mean[blockIdx.x].x)));
  }
}

// -------------------------------------------------------- A2: leaf bounds --

// Relation of every leaf of the batch; an empty relation's leaf ranges are
// all empty (lo = 0).  The lo array of relation j (L_j + 1 entries) starts at
// lo[leaf_base_j + j].
__global__ void leaf_rel_kernel(const RelDesc* rel, const uint32_t* lpre, uint32_t k,
                                uint32_t GL, uint32_t* leaf_rel, uint32_t* lo) {
  for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < GL; g += gridDim.x * blockDim.x) {
    const uint32_t j = rel_of(lpre, k, g);
    leaf_rel[g] = j;
    if (rel[j].n == 0) {
      lo[g + j] = 0;
      if (g - rel[j].leaf_base + 1 == rel[j].L) lo[g + j + 1] = 0;
    }
  }
}

// Block = key tile of one relation: lo[l] = first position i with
// leaf(R[i]) >= l, for l = 0..L (lo[L] = n).
template <class Model>
__global__ void leaf_bounds_kernel(const RelDesc* rel, const uint32_t* tpre, uint32_t k,
                                   const double2* root, uint32_t* lo_all) {
  __shared__ Model s_model;
  const uint32_t j = rel_of(tpre, k, blockIdx.x);
  const RelDesc d = rel[j];
  if (threadIdx.x == 0) s_model = root_model<Model>(root[j], d.L);
  __syncthreads();
  const Model model = s_model;
  uint32_t* lo = lo_all + d.leaf_base + j;
  const uint64_t s = (uint64_t)(blockIdx.x - d.t_base) * kKeyTile, e = min(d.n, s + kKeyTile);
  for (uint64_t i = s + threadIdx.x; i < e; i += blockDim.x) {
    const int64_t li = model.leaf(d.R[i]);
    const int64_t lp = i > 0 ? (int64_t)model.leaf(d.R[i - 1]) : -1;
    for (int64_t l = lp + 1; l <= li; ++l) lo[l] = (uint32_t)i;
    if (i + 1 == d.n)
      for (int64_t l = li + 1; l <= (int64_t)d.L; ++l) lo[l] = (uint32_t)d.n;
  }
}

// cnt[g] = number of chunks of leaf g.
__global__ void chunk_count_kernel(const uint32_t* lo, const uint32_t* leaf_rel, uint32_t GL,
                                   uint32_t* cnt) {
  for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < GL; g += gridDim.x * blockDim.x) {
    const uint32_t q = g + leaf_rel[g];
    cnt[g] = (lo[q + 1] - lo[q] + kChunk - 1) / kChunk;
  }
}

// Exclusive scan of u32 (tile = 256 threads x 8 items) with decoupled
// look-back; out[count] = total.
__global__ void __launch_bounds__(kBlock) scan_u32_kernel(const uint32_t* in, uint32_t* out,
                                                          uint32_t count, TileState st,
                                                          uint32_t* err) {
  constexpr int kItems = 8;
  __shared__ uint32_t s_tile;
  __shared__ uint64_t s_warp[kBlock / 32];
  __shared__ uint64_t s_prefix;
  if (threadIdx.x == 0) s_tile = atomicAdd(st.ticket, 1u);
  __syncthreads();
  const uint32_t tile = s_tile;
  const uint64_t base = (uint64_t)tile * kBlock * kItems + (uint64_t)threadIdx.x * kItems;
  uint32_t v[kItems];
  uint64_t sum = 0;
#pragma unroll
  for (int q = 0; q < kItems; ++q) {
    v[q] = base + q < count ? in[base + q] : 0u;
    sum += v[q];
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint64_t incl = warp_inclusive_sum(sum, lane);
  if (lane == 31) s_warp[w] = incl;
  __syncthreads();
  if (w == 0) {
    uint64_t x = lane < kBlock / 32 ? s_warp[lane] : 0;
    const uint64_t xi = warp_inclusive_sum(x, lane);
    if (lane < kBlock / 32) s_warp[lane] = xi - x;
    const uint64_t agg = __shfl_sync(0xffffffffu, xi, 31);
    const uint64_t pre = lookback_warp(st, tile, agg, err);
    if (lane == 0) s_prefix = pre;
  }
  __syncthreads();
  uint64_t run = s_prefix + s_warp[w] + incl - sum;
#pragma unroll
  for (int q = 0; q < kItems; ++q) {
    if (base + q < count) out[base + q] = (uint32_t)run;
    if (base + q + 1 == count) out[count] = (uint32_t)(run + v[q]);
    run += v[q];
  }
}

// ---------------------------------------------------------- A3: leaf fits --

struct ChunkRange {
  uint32_t leaf, rel, lo, s, e;
};

// Chunk c of the batch: its leaf (the largest g with cstart[g] <= c), that
// leaf's relation and first position, and the chunk's positions [s, e).
__device__ __forceinline__ bool chunk_range(const uint32_t* cstart, const uint32_t* lo,
                                            const uint32_t* leaf_rel, uint32_t GL, uint32_t c,
                                            ChunkRange& r) {
  if (c >= cstart[GL]) return false;
  r.leaf = rel_of(cstart, GL, c);
  r.rel = leaf_rel[r.leaf];
  r.lo = lo[r.leaf + r.rel];
  const uint32_t hi = lo[r.leaf + r.rel + 1];
  r.s = r.lo + (c - cstart[r.leaf]) * kChunk;
  r.e = min(hi, r.s + kChunk);
  return true;
}

// Per chunk: (sum dx, sum dy), dx = R[i] - R[lo], dy = i - lo.
__global__ void leaf_pass1_kernel(const RelDesc* rel, const uint32_t* lo, const uint32_t* cstart,
                                  const uint32_t* leaf_rel, uint32_t GL, double2* part) {
  const uint32_t c = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  ChunkRange r;
  if (!chunk_range(cstart, lo, leaf_rel, GL, c, r)) return;
  const uint64_t* R = rel[r.rel].R;
  const uint64_t base = R[r.lo];
  double sx = 0.0, sy = 0.0;
  for (uint32_t i = r.s + lane; i < r.e; i += 32) {
    sx = __dadd_rn(sx, (double)(R[i] - base));
    sy = __dadd_rn(sy, (double)(i - r.lo));
  }
  sx = warp_sum_d(sx);
  sy = warp_sum_d(sy);
  if (lane == 0) part[c] = make_double2(sx, sy);
}

// Per leaf: means of dx and dy from its chunks (warp per leaf).
__global__ void leaf_mean_kernel(const uint32_t* lo, const uint32_t* cstart,
                                 const uint32_t* leaf_rel, uint32_t GL, const double2* part,
                                 double2* mean) {
  const uint32_t g = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (g >= GL) return;
  double sx = 0.0, sy = 0.0;
  for (uint32_t c = cstart[g] + lane; c < cstart[g + 1]; c += 32) {
    sx = __dadd_rn(sx, part[c].x);
    sy = __dadd_rn(sy, part[c].y);
  }
  sx = warp_sum_d(sx);
  sy = warp_sum_d(sy);
  if (lane == 0) {
    const uint32_t q = g + leaf_rel[g];
    const double kk = (double)(lo[q + 1] - lo[q]);
    mean[g] = kk > 0 ? make_double2(__ddiv_rn(sx, kk), __ddiv_rn(sy, kk)) : make_double2(0.0, 0.0);
  }
}

// Per chunk: centred (S_xy, S_xx).
__global__ void leaf_pass2_kernel(const RelDesc* rel, const uint32_t* lo, const uint32_t* cstart,
                                  const uint32_t* leaf_rel, uint32_t GL, const double2* mean,
                                  double2* part) {
  const uint32_t c = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  ChunkRange r;
  if (!chunk_range(cstart, lo, leaf_rel, GL, c, r)) return;
  const uint64_t* R = rel[r.rel].R;
  const uint64_t base = R[r.lo];
  const double mx = mean[r.leaf].x, my = mean[r.leaf].y;
  double sxy = 0.0, sxx = 0.0;
  for (uint32_t i = r.s + lane; i < r.e; i += 32) {
    const double dx = __dsub_rn((double)(R[i] - base), mx);
    const double dy = __dsub_rn((double)(i - r.lo), my);
    sxy = __dadd_rn(sxy, __dmul_rn(dx, dy));
    sxx = __dadd_rn(sxx, __dmul_rn(dx, dx));
  }
  sxy = warp_sum_d(sxy);
  sxx = warp_sum_d(sxx);
  if (lane == 0) part[c] = make_double2(sxy, sxx);
}

// Per leaf: slope / intercept (double), then initialise the error bounds.
__global__ void leaf_final_kernel(const uint32_t* lo, const uint32_t* cstart,
                                  const uint32_t* leaf_rel, uint32_t GL, const double2* part,
                                  const double2* mean, double2* fit, int32_t* elo, int32_t* ehi) {
  const uint32_t g = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (g >= GL) return;
  double sxy = 0.0, sxx = 0.0;
  for (uint32_t c = cstart[g] + lane; c < cstart[g + 1]; c += 32) {
    sxy = __dadd_rn(sxy, part[c].x);
    sxx = __dadd_rn(sxx, part[c].y);
  }
  sxy = warp_sum_d(sxy);
  sxx = warp_sum_d(sxx);
  if (lane == 0) {
    const uint32_t q = g + leaf_rel[g];
    double a = 0.0, b = 0.0;
    if (lo[q + 1] > lo[q]) {
      a = sxx > 0.0 ? __ddiv_rn(sxy, sxx) : 0.0;
      if (!(a > 0.0)) a = 0.0;
      b = __dsub_rn(mean[g].y, __dmul_rn(a, mean[g].x));
    }
    fit[g] = make_double2(a, b);
    elo[g] = INT32_MAX;
    ehi[g] = INT32_MIN;
  }
}

// ------------------------------------------------------------- A4: errors --

__device__ __forceinline__ int32_t sat32(int64_t v) {
  return v < INT32_MIN ? INT32_MIN : (v > INT32_MAX ? INT32_MAX : (int32_t)v);
}

template <class Model>
__global__ void leaf_err_kernel(const RelDesc* rel, const uint32_t* lo, const uint32_t* cstart,
                                const uint32_t* leaf_rel, uint32_t GL, const double2* fit,
                                int32_t* elo, int32_t* ehi) {
  const uint32_t c = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  ChunkRange r;
  if (!chunk_range(cstart, lo, leaf_rel, GL, c, r)) return;
  const uint64_t* R = rel[r.rel].R;
  const uint64_t base = R[r.lo];
  const double2 f = fit[r.leaf];
  int32_t mn = INT32_MAX, mx = INT32_MIN;
  for (uint32_t i = r.s + lane; i < r.e; i += 32) {
    const int64_t e = (int64_t)(i - r.lo) - Model::pred_fit(R[i], base, f.x, f.y);
    const int32_t e32 = sat32(e);
    mn = min(mn, e32);
    mx = max(mx, e32);
  }
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) {
    mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, d));
    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, d));
  }
  if (lane == 0) {
    atomicMin(elo + r.leaf, mn);
    atomicMax(ehi + r.leaf, mx);
  }
}

// Leaf records + per-relation statistics.  stats[4j + ...]: [0] sum
// size*width, [1] max width, [2] max size, [3] non-empty leaves.
template <class Model>
__global__ void leaf_records_kernel(const RelDesc* rel, const uint32_t* lo_all,
                                    const uint32_t* leaf_rel, uint32_t GL, const double2* fit,
                                    const int32_t* elo, const int32_t* ehi,
                                    unsigned long long* stats) {
  for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < GL; g += gridDim.x * blockDim.x) {
    const uint32_t j = leaf_rel[g];
    const RelDesc& d = rel[j];
    const uint32_t l = g - d.leaf_base;
    const uint32_t* lo = lo_all + d.leaf_base + j;
    typename Model::Leaf rec{};
    const uint32_t a = lo[l], b = lo[l + 1];
    rec.lo = a;
    rec.hi = b;
    rec.base_key = a < d.n ? d.R[a] : 0;
    const double2 f = fit[g];
    Model::set_params(rec, f.x, f.y);   // deployed parameters (float or double)
    unsigned long long* st = stats + 4 * (uint64_t)j;
    if (b > a) {
      rec.e_lo = elo[g];
      rec.e_hi = ehi[g];
      const int64_t w = (int64_t)rec.e_hi - (int64_t)rec.e_lo + 1;
      const int64_t sz = (int64_t)(b - a);
      const uint64_t width = (uint64_t)(w < sz ? w : sz);
      atomicAdd(st + 0, (unsigned long long)width * (b - a));
      atomicMax(st + 1, (unsigned long long)width);
      atomicMax(st + 2, (unsigned long long)(b - a));
      atomicAdd(st + 3, 1ull);
    } else {
      rec.e_lo = 0;
      rec.e_hi = 0;
    }
    reinterpret_cast<typename Model::Leaf*>(d.leaves_out)[l] = rec;
  }
}

unsigned grid_for(uint64_t work, int block, uint64_t cap = 152 * 32) {
  uint64_t g = (work + block - 1) / block;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (unsigned)g;
}

// Exclusive scan of `count` u32 into out[0..count] using the look-back kernel.
int scan_u32(const uint32_t* in, uint32_t* out, uint32_t count, cudaStream_t s) {
  const uint32_t tile = kBlock * 8;
  const uint32_t tiles = std::max<uint32_t>(1, (count + tile - 1) / tile);
  void* ws = nullptr;
  const size_t bytes = 256 + (size_t)tiles * (4 + 8 + 8);
  LJ_CUDA(scratch_alloc(&ws, bytes, s));
  LJ_CUDA(cudaMemsetAsync(ws, 0, 256 + (size_t)tiles * 4, s));
  TileState st;
  st.ticket = (uint32_t*)ws;
  st.flag = (uint32_t*)((char*)ws + 256);
  st.agg = (uint64_t*)((char*)ws + 256 + ((size_t)tiles * 4 + 15) / 16 * 16);
  st.incl = st.agg + tiles;
  uint32_t* err = device_error_word(current_device());
  scan_u32_kernel<<<tiles, kBlock, 0, s>>>(in, out, count, st, err);
  LJ_CUDA(cudaGetLastError());
  LJ_CUDA(scratch_free(ws, s));
  return 0;
}

size_t round256(size_t b) { return (b + 255) / 256 * 256; }

// Device work of a batch, once the host plan exists.  Returns an LJ code.
template <class Model>
int run_batch(const std::vector<RelDesc>& rd, const std::vector<uint32_t>& tpre,
              const std::vector<uint32_t>& gpre, const std::vector<uint32_t>& lpre,
              uint64_t tiles, uint64_t groot, uint64_t GL, uint64_t max_chunks, char* ws,
              cudaStream_t s, std::vector<uint32_t>& hflags, std::vector<double2>& hroot,
              std::vector<unsigned long long>& hstats) {
  const uint32_t k = (uint32_t)rd.size();
  const size_t b_rel = round256(sizeof(RelDesc) * k), b_pre = round256(4 * (size_t)(k + 1));
  const size_t b_flags = round256(8 * (size_t)k), b_root = round256(16 * (size_t)k);
  const size_t b_gpart = round256(16 * (size_t)groot), b_lo = round256(4 * (size_t)(GL + k));
  const size_t b_gl4 = round256(4 * (size_t)(GL + 1)), b_gl16 = round256(16 * (size_t)GL);
  const size_t b_part = round256(16 * (size_t)max_chunks);
  char* p = ws;
  auto take = [&](size_t b) {
    char* q = p;
    p += b;
    return q;
  };
  RelDesc* rel = (RelDesc*)take(b_rel);
  uint32_t* d_tpre = (uint32_t*)take(b_pre);
  uint32_t* d_gpre = (uint32_t*)take(b_pre);
  uint32_t* d_lpre = (uint32_t*)take(b_pre);
  uint32_t* flags = (uint32_t*)take(b_flags);
  double2* mean = (double2*)take(b_root);
  double2* root = (double2*)take(b_root);
  double2* gpart = (double2*)take(b_gpart);
  uint32_t* lo = (uint32_t*)take(b_lo);
  uint32_t* leaf_rel = (uint32_t*)take(b_gl4);
  uint32_t* cnt = (uint32_t*)take(b_gl4);
  uint32_t* cstart = (uint32_t*)take(b_gl4);
  int32_t* elo = (int32_t*)take(b_gl4);
  int32_t* ehi = (int32_t*)take(b_gl4);
  double2* lmean = (double2*)take(b_gl16);
  double2* fit = (double2*)take(b_gl16);
  double2* part = (double2*)take(b_part);
  unsigned long long* stats = (unsigned long long*)take(round256(32 * (size_t)k));

  // the tables are small: copies from pageable memory (staged by the driver)
  LJ_CUDA(cudaMemcpyAsync(rel, rd.data(), sizeof(RelDesc) * k, cudaMemcpyHostToDevice, s));
  LJ_CUDA(cudaMemcpyAsync(d_tpre, tpre.data(), 4 * (size_t)(k + 1), cudaMemcpyHostToDevice, s));
  LJ_CUDA(cudaMemcpyAsync(d_gpre, gpre.data(), 4 * (size_t)(k + 1), cudaMemcpyHostToDevice, s));
  LJ_CUDA(cudaMemcpyAsync(d_lpre, lpre.data(), 4 * (size_t)(k + 1), cudaMemcpyHostToDevice, s));
  LJ_CUDA(cudaMemsetAsync(flags, 0, b_flags, s));
  LJ_CUDA(cudaMemsetAsync(stats, 0, 32 * (size_t)k, s));

  // checks and root (A1)
  check_sorted_kernel<<<(unsigned)tiles, kBlock, 0, s>>>(rel, d_tpre, k, flags);
  root_pass1_kernel<<<(unsigned)groot, kBlock, 0, s>>>(rel, d_gpre, k, gpart);
  root_mean_kernel<<<k, kBlock, 0, s>>>(rel, gpart, mean);
  root_pass2_kernel<<<(unsigned)groot, kBlock, 0, s>>>(rel, d_gpre, k, mean, gpart);
  root_final_kernel<<<k, kBlock, 0, s>>>(rel, gpart, mean, root);
  LJ_CUDA(cudaGetLastError());
  LJ_CUDA(cudaMemcpyAsync(hflags.data(), flags, 8 * (size_t)k, cudaMemcpyDeviceToHost, s));
  LJ_CUDA(cudaMemcpyAsync(hroot.data(), root, 16 * (size_t)k, cudaMemcpyDeviceToHost, s));
  LJ_CUDA(cudaStreamSynchronize(s));
  for (uint32_t j = 0; j < k; ++j)
    if (hflags[2 * j])
      return fail(LJ_E_UNSORTED, "rmi_build: R (relation %u of the batch) is not sorted "
                                 "non-decreasing", j);

  // leaves (A2 - A4)
  const uint32_t gl = (uint32_t)GL;
  leaf_rel_kernel<<<grid_for(GL, kBlock), kBlock, 0, s>>>(rel, d_lpre, k, gl, leaf_rel, lo);
  leaf_bounds_kernel<Model><<<(unsigned)tiles, kBlock, 0, s>>>(rel, d_tpre, k, root, lo);
  chunk_count_kernel<<<grid_for(GL, kBlock), kBlock, 0, s>>>(lo, leaf_rel, gl, cnt);
  LJ_CUDA(cudaGetLastError());
  if (int rc = scan_u32(cnt, cstart, gl, s)) return rc;
  const unsigned warps_chunks = (unsigned)((max_chunks * 32 + kBlock - 1) / kBlock);
  const unsigned warps_leaves = (unsigned)((GL * 32 + kBlock - 1) / kBlock);
  leaf_pass1_kernel<<<warps_chunks, kBlock, 0, s>>>(rel, lo, cstart, leaf_rel, gl, part);
  leaf_mean_kernel<<<warps_leaves, kBlock, 0, s>>>(lo, cstart, leaf_rel, gl, part, lmean);
  leaf_pass2_kernel<<<warps_chunks, kBlock, 0, s>>>(rel, lo, cstart, leaf_rel, gl, lmean, part);
  leaf_final_kernel<<<warps_leaves, kBlock, 0, s>>>(lo, cstart, leaf_rel, gl, part, lmean, fit,
                                                    elo, ehi);
  leaf_err_kernel<Model><<<warps_chunks, kBlock, 0, s>>>(rel, lo, cstart, leaf_rel, gl, fit, elo,
                                                         ehi);
  leaf_records_kernel<Model><<<grid_for(GL, kBlock), kBlock, 0, s>>>(rel, lo, leaf_rel, gl, fit,
                                                                      elo, ehi, stats);
  LJ_CUDA(cudaGetLastError());
  LJ_CUDA(cudaMemcpyAsync(hstats.data(), stats, 32 * (size_t)k, cudaMemcpyDeviceToHost, s));
  return 0;
}

// Scratch bytes of run_batch.
size_t batch_scratch_bytes(uint32_t k, uint64_t groot, uint64_t GL, uint64_t max_chunks) {
  return round256(sizeof(RelDesc) * k) + 3 * round256(4 * (size_t)(k + 1)) +
         round256(8 * (size_t)k) + 2 * round256(16 * (size_t)k) + round256(16 * (size_t)groot) +
         round256(4 * (size_t)(GL + k)) + 5 * round256(4 * (size_t)(GL + 1)) +
         2 * round256(16 * (size_t)GL) + round256(16 * (size_t)max_chunks) +
         round256(32 * (size_t)k);
}

// Build the k indexes (idx[j] holds R, n, L, precision, device); fills the
// rest of each index.  Synchronises `s`.
template <class Model>
int build_batch(lj_index* const* idx, uint32_t k, cudaStream_t s, float* ms_out) {
  // host plan: prefix tables over the relations
  std::vector<RelDesc> rd(k);
  std::vector<uint32_t> tpre(k + 1), gpre(k + 1), lpre(k + 1);
  uint64_t tiles = 0, groot = 0, GL = 0, max_chunks = 1;
  const size_t rec = sizeof(typename Model::Leaf);
  std::vector<size_t> leaf_off(k);
  size_t leaf_bytes = 0;
  for (uint32_t j = 0; j < k; ++j) {
    RelDesc& d = rd[j];
    d = RelDesc{};
    d.R = idx[j]->R;
    d.n = idx[j]->n;
    d.L = idx[j]->L;
    d.G = (uint32_t)std::min<uint64_t>(kRootBlocks,
                                       std::max<uint64_t>(1, (d.n + kRootKeys - 1) / kRootKeys));
    d.per = d.n ? (d.n + d.G - 1) / d.G : 1;
    d.leaf_base = (uint32_t)GL;
    d.g_base = (uint32_t)groot;
    d.t_base = (uint32_t)tiles;
    tpre[j] = (uint32_t)tiles;
    gpre[j] = (uint32_t)groot;
    lpre[j] = (uint32_t)GL;
    tiles += std::max<uint64_t>(1, (d.n + kKeyTile - 1) / kKeyTile);
    groot += d.G;
    GL += d.L;
    max_chunks += d.n / kChunk + d.L;
    leaf_off[j] = leaf_bytes;
    leaf_bytes += round256(rec * d.L);
  }
  tpre[k] = (uint32_t)tiles;
  gpre[k] = (uint32_t)groot;
  lpre[k] = (uint32_t)GL;
  if (GL >= (1ull << 32) - 1 || max_chunks >= (1ull << 32) || tiles >= (1ull << 31))
    return fail(LJ_E_INVAL, "rmi_build_batch: the batch is too large (%llu leaves)",
                (unsigned long long)GL);

  // leaf records: one allocation shared by the batch's indexes
  void* block = nullptr;
  LJ_CUDA(cudaMalloc(&block, std::max<size_t>(leaf_bytes, 256)));
  std::shared_ptr<void> owner(block, [](void* q) { cudaFree(q); });
  for (uint32_t j = 0; j < k; ++j) rd[j].leaves_out = (char*)block + leaf_off[j];

  char* ws = nullptr;
  LJ_CUDA(scratch_alloc((void**)&ws, batch_scratch_bytes(k, groot, GL, max_chunks), s));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  LJ_CUDA(cudaEventCreate(&e0));
  LJ_CUDA(cudaEventCreate(&e1));
  cudaEventRecord(e0, s);
  std::vector<uint32_t> hflags(2 * (size_t)k);
  std::vector<double2> hroot(k);
  std::vector<unsigned long long> hstats(4 * (size_t)k);
  int rc = run_batch<Model>(rd, tpre, gpre, lpre, tiles, groot, GL, max_chunks, ws, s, hflags,
                            hroot, hstats);
  cudaEventRecord(e1, s);
  const cudaError_t ce = cudaStreamSynchronize(s);
  if (!rc && ce != cudaSuccess) rc = fail_cuda(ce, "rmi_build sync");
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  scratch_free(ws, s);
  if (rc) return rc;
  *ms_out = ms;
  for (uint32_t j = 0; j < k; ++j) {
    lj_index* x = idx[j];
    x->leaves = rd[j].leaves_out;
    x->leaves_block = owner;
    x->unique = hflags[2 * j + 1] ? 0 : 1;
    x->root_fit[0] = x->root_f64[0] = hroot[j].x;
    x->root_fit[1] = x->root_f64[1] = hroot[j].y;
    x->root_f32[0] = (float)hroot[j].x;
    x->root_f32[1] = (float)hroot[j].y;
    x->stats.root_a = x->precision == LJ_FP64 ? hroot[j].x : (double)x->root_f32[0];
    x->stats.root_b = x->precision == LJ_FP64 ? hroot[j].y : (double)x->root_f32[1];
    const uint64_t n = x->n;
    x->stats.mean_window = n ? (double)hstats[4 * j] / (double)n : 0.0;
    x->stats.max_window = (uint32_t)hstats[4 * j + 1];
    x->stats.max_leaf_size = (uint32_t)hstats[4 * j + 2];
    x->stats.nonempty_leaves = (uint32_t)hstats[4 * j + 3];
    x->stats.unique = x->unique;
  }
  return 0;
}

int check_build_args(const uint64_t* R, uint64_t n, uint32_t leaves, int precision,
                     const char* who) {
  if (n > 0 && !R) return fail(LJ_E_INVAL, "%s: R is NULL", who);
  if (n >= (1ull << 32))
    return fail(LJ_E_INVAL, "%s: n = %llu must be below 2^32", who, (unsigned long long)n);
  if (leaves < 1 || leaves > (1u << 24))
    return fail(LJ_E_INVAL, "%s: leaves = %u must be in [1, 2^24]", who, leaves);
  if (precision != LJ_FP32 && precision != LJ_FP64)
    return fail(LJ_E_INVAL, "%s: unknown precision %d", who, precision);
  return 0;
}

int build_many(const uint64_t* const* R, const uint64_t* n, const uint32_t* leaves, uint32_t k,
               int precision, cudaStream_t s, lj_index** out) {
  std::vector<lj_index*> idx(k, nullptr);
  const int dev = current_device();
  for (uint32_t j = 0; j < k; ++j) {
    lj_index* x = new lj_index();
    x->R = R[j];
    x->n = n[j];
    x->L = leaves[j];
    x->precision = precision;
    x->device = dev;
    x->stats.n = n[j];
    x->stats.leaves = leaves[j];
    x->stats.precision = precision;
    idx[j] = x;
  }
  float ms = 0.f;
  int rc = precision == LJ_FP64 ? build_batch<ModelF64>(idx.data(), k, s, &ms)
                                : build_batch<ModelF32>(idx.data(), k, s, &ms);
  if (!rc) rc = take_device_errors(dev, s);
  if (rc) {
    for (lj_index* x : idx) rmi_free(x);
    return rc;
  }
  for (uint32_t j = 0; j < k; ++j) {
    idx[j]->stats.build_ms = ms;
    out[j] = idx[j];
  }
  return LJ_OK;
}

}  // namespace
}  // namespace lj

namespace lj {

// Key levels of R for the descent search (search_levels): level k holds
// R[4^k i] for i < ceil(n / 4^k), padded with 2^64 - 1 to whole nodes of
// four entries (the probes never pass padding: they check positions).
namespace {
std::atomic<int> g_key_levels{2};

__global__ void key_level_kernel(const uint64_t* __restrict__ R, uint64_t n, uint32_t shift,
                                 uint64_t* __restrict__ out, uint64_t entries) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= entries) return;
  const uint64_t pos = i << shift;
  out[i] = pos < n ? __ldg(reinterpret_cast<const unsigned long long*>(R) + pos) : ~0ull;
}
}  // namespace

void set_key_levels(int v) { g_key_levels = v; }
int get_key_levels() { return g_key_levels; }

int build_key_levels(lj_index* idx, cudaStream_t s) {
  const uint64_t n = idx->n;
  idx->use_levels = 1;
  if (idx->levels || n <= 4) return 0;   // built already, or one node of R: no level above it
  uint64_t off[kMaxLevels + 1] = {};
  uint32_t nlev = 0;
  uint64_t total = 0;
  for (uint32_t k = 1; k <= (uint32_t)kMaxLevels; ++k) {
    const uint64_t Nk = (n + (1ull << (2 * k)) - 1) >> (2 * k);
    off[k] = total;
    total += (Nk + 3) & ~3ull;
    nlev = k;
    if (Nk <= 4) break;
  }
  uint64_t* lev = nullptr;
  LJ_CUDA(cudaMalloc((void**)&lev, total * 8));
  for (uint32_t k = 1; k <= nlev; ++k) {
    const uint64_t entries = (k < nlev ? off[k + 1] : total) - off[k];
    key_level_kernel<<<(unsigned)((entries + 255) / 256), 256, 0, s>>>(idx->R, n, 2 * k,
                                                                      lev + off[k], entries);
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    cudaFree(lev);
    return fail_cuda(e, "key_level_kernel");
  }
  idx->levels = lev;
  idx->nlev = nlev;
  for (int k = 0; k <= kMaxLevels; ++k) idx->lev_off[k] = (uint32_t)off[k];
  return 0;
}

}  // namespace lj

extern "C" int rmi_build(const uint64_t* R_dev, uint64_t n, uint32_t leaves, int precision,
                         lj_stream_t stream, lj_index** out) {
  using namespace lj;
  if (!out) return fail(LJ_E_INVAL, "rmi_build: out is NULL");
  *out = nullptr;
  if (int rc = check_build_args(R_dev, n, leaves, precision, "rmi_build")) return rc;
  if (int rc = build_many(&R_dev, &n, &leaves, 1, precision, (cudaStream_t)stream, out)) return rc;
  // key levels: measured faster for an R with duplicate keys (dup_seqh_50m:
  // search 24.4 -> 15.2 ms), slower for the unique lognormal and uniform
  // workloads, whose halving searches share pivots across a warp
  const int kl = get_key_levels();
  if (kl == 1 || (kl == 2 && !(*out)->unique)) {
    if (int rc = build_key_levels(*out, (cudaStream_t)stream)) {
      rmi_free(*out);
      *out = nullptr;
      return rc;
    }
  }
  return LJ_OK;
}

extern "C" int rmi_build_batch(const uint64_t* const* R_dev, const uint64_t* n,
                               const uint32_t* leaves, uint32_t k, int precision,
                               lj_stream_t stream, lj_index** out) {
  using namespace lj;
  if (k > 0 && (!out || !R_dev || !n || !leaves))
    return fail(LJ_E_INVAL, "rmi_build_batch: NULL argument");
  for (uint32_t j = 0; j < k; ++j) out[j] = nullptr;
  if (k == 0) return LJ_OK;
  if (k > (1u << 20)) return fail(LJ_E_INVAL, "rmi_build_batch: k = %u above 2^20", k);
  for (uint32_t j = 0; j < k; ++j)
    if (int rc = check_build_args(R_dev[j], n[j], leaves[j], precision, "rmi_build_batch"))
      return rc;
  return build_many(R_dev, n, leaves, k, precision, (cudaStream_t)stream, out);
}
