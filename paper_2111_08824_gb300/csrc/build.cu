// rmi_build: fit the two-level linear RMI over a sorted R on the device.
//
// Section 2.D (Recursive Model Index): a root linear model routes a key to a
// leaf model; each leaf's linear model predicts the position; each leaf keeps
// the minimum and maximum error of its keys.  Fitting is least squares; the
// index is built once, before any join (Section 3.A).
//
// Steps (each a kernel; every reduction has a fixed order, so a build is
// bit-for-bit reproducible for a given R and L):
//   A1 root fit    two passes over R: means of (key, i*L/n), then the
//                  centred sums S_xy and S_xx; a0 = S_xy / S_xx (>= 0).
//   A2 leaf bounds leaf(R[i]) with the probe's own arithmetic; the root is
//                  monotone, so leaf l owns the range [lo_l, lo_{l+1}),
//                  found where leaf(R[i-1]) != leaf(R[i]).
//   A3 leaf fits   segmented least squares of (i - lo_l) on (R[i] - R[lo_l])
//                  over the leaf ranges.  Leaves are cut into chunks of
//                  kChunk keys (an exclusive scan numbers them), one warp
//                  per chunk, then one warp per leaf sums its chunks: load
//                  balanced whatever the leaf sizes.
//   A4 errors      err_i = (i - lo_l) - floor(a_l * (R[i] - R[lo_l]) + b_l)
//                  with the deployed (possibly single-precision) parameters;
//                  per-leaf min / max by warp reduction + integer atomics.
#include <algorithm>
#include <cmath>
#include <vector>

#include "device_common.cuh"
#include "internal.h"

namespace lj {
namespace {

constexpr int kBlock = 256;
constexpr uint32_t kChunk = 2048;   // keys per chunk of a leaf (one warp)

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

// ------------------------------------------------------------------ checks --

__global__ void check_sorted_kernel(const uint64_t* R, uint64_t n, uint32_t* flags) {
  uint32_t unsorted = 0, dup = 0;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i + 1 < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t a = R[i], b = R[i + 1];
    unsorted |= a > b;
    dup |= a == b;
  }
  unsorted = __any_sync(0xffffffffu, unsorted);
  dup = __any_sync(0xffffffffu, dup);
  if ((threadIdx.x & 31) == 0) {
    if (unsorted) atomicOr(flags, 1u);
    if (dup) atomicOr(flags + 1, 1u);
  }
}

// --------------------------------------------------------------- A1: root --

// Block b covers [b*per, min(n, (b+1)*per)).
__global__ void root_pass1_kernel(const uint64_t* R, uint64_t n, uint32_t L, uint64_t per,
                                  double2* part) {
  const uint64_t s = blockIdx.x * per, e = min(n, s + per);
  double sx = 0.0, sy = 0.0;
  for (uint64_t i = s + threadIdx.x; i < e; i += kBlock) {
    sx = __dadd_rn(sx, (double)R[i]);
    sy = __dadd_rn(sy, pos_scaled(i, L, n));
  }
  block_sum2(sx, sy);
  if (threadIdx.x == 0) part[blockIdx.x] = make_double2(sx, sy);
}

// One block: fixed-order sum of the partials; out = (mean_x, mean_y).
__global__ void root_mean_kernel(const double2* part, int G, uint64_t n, double* out) {
  double sx = 0.0, sy = 0.0;
  for (int i = threadIdx.x; i < G; i += kBlock) {
    sx = __dadd_rn(sx, part[i].x);
    sy = __dadd_rn(sy, part[i].y);
  }
  block_sum2(sx, sy);
  if (threadIdx.x == 0) {
    out[0] = __ddiv_rn(sx, (double)n);
    out[1] = __ddiv_rn(sy, (double)n);
  }
}

__global__ void root_pass2_kernel(const uint64_t* R, uint64_t n, uint32_t L, uint64_t per,
                                  const double* mean, double2* part) {
  const uint64_t s = blockIdx.x * per, e = min(n, s + per);
  const double mx = mean[0], my = mean[1];
  double sxy = 0.0, sxx = 0.0;
  for (uint64_t i = s + threadIdx.x; i < e; i += kBlock) {
    const double dx = __dsub_rn((double)R[i], mx);
    const double dy = __dsub_rn(pos_scaled(i, L, n), my);
    sxy = __dadd_rn(sxy, __dmul_rn(dx, dy));
    sxx = __dadd_rn(sxx, __dmul_rn(dx, dx));
  }
  block_sum2(sxy, sxx);
  if (threadIdx.x == 0) part[blockIdx.x] = make_double2(sxy, sxx);
}

// out = (a0, b0) least squares, slope clamped >= 0.
__global__ void root_final_kernel(const double2* part, int G, const double* mean,
                                  double* out) {
  double sxy = 0.0, sxx = 0.0;
  for (int i = threadIdx.x; i < G; i += kBlock) {
    sxy = __dadd_rn(sxy, part[i].x);
    sxx = __dadd_rn(sxx, part[i].y);
  }
  block_sum2(sxy, sxx);
  if (threadIdx.x == 0) {
    double a = sxx > 0.0 ? __ddiv_rn(sxy, sxx) : 0.0;
    if (!(a > 0.0)) a = 0.0;
    out[0] = a;
    out[1] = __dsub_rn(mean[1], __dmul_rn(a, mean[0]));
  }
}

// -------------------------------------------------------- A2: leaf bounds --

// lo[l] = first position i with leaf(R[i]) >= l, for l = 0..L (lo[L] = n).
template <class Model>
__global__ void leaf_bounds_kernel(const uint64_t* R, uint64_t n, Model model, uint32_t* lo) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const int64_t li = model.leaf_exact(R[i]);
    const int64_t lp = i > 0 ? (int64_t)model.leaf_exact(R[i - 1]) : -1;
    for (int64_t l = lp + 1; l <= li; ++l) lo[l] = (uint32_t)i;
    if (i + 1 == n)
      for (int64_t l = li + 1; l <= (int64_t)model.L; ++l) lo[l] = (uint32_t)n;
  }
}

// cnt[l] = number of chunks of leaf l.
__global__ void chunk_count_kernel(const uint32_t* lo, uint32_t L, uint32_t* cnt) {
  for (uint32_t l = blockIdx.x * blockDim.x + threadIdx.x; l < L; l += gridDim.x * blockDim.x)
    cnt[l] = (lo[l + 1] - lo[l] + kChunk - 1) / kChunk;
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
  for (int k = 0; k < kItems; ++k) {
    v[k] = base + k < count ? in[base + k] : 0u;
    sum += v[k];
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
  for (int k = 0; k < kItems; ++k) {
    if (base + k < count) out[base + k] = (uint32_t)run;
    if (base + k + 1 == count) out[count] = (uint32_t)(run + v[k]);
    run += v[k];
  }
}

// ---------------------------------------------------------- A3: leaf fits --

// Leaf owning chunk c: the largest l with cstart[l] <= c.
__device__ __forceinline__ uint32_t chunk_leaf(const uint32_t* cstart, uint32_t L, uint32_t c) {
  uint32_t a = 0, b = L;   // cstart[0] = 0 <= c
  while (b - a > 1) {
    const uint32_t mid = (a + b) >> 1;
    if (cstart[mid] <= c)
      a = mid;
    else
      b = mid;
  }
  return a;
}

struct ChunkRange {
  uint32_t leaf, lo, s, e;
};

__device__ __forceinline__ bool chunk_range(const uint32_t* cstart, const uint32_t* lo,
                                            uint32_t L, uint32_t c, ChunkRange& r) {
  if (c >= cstart[L]) return false;
  r.leaf = chunk_leaf(cstart, L, c);
  r.lo = lo[r.leaf];
  const uint32_t hi = lo[r.leaf + 1];
  r.s = r.lo + (c - cstart[r.leaf]) * kChunk;
  r.e = min(hi, r.s + kChunk);
  return true;
}

// Per chunk: (sum dx, sum dy), dx = R[i] - R[lo], dy = i - lo.
__global__ void leaf_pass1_kernel(const uint64_t* R, const uint32_t* lo, const uint32_t* cstart,
                                  uint32_t L, double2* part) {
  const uint32_t c = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  ChunkRange r;
  if (!chunk_range(cstart, lo, L, c, r)) return;
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
__global__ void leaf_mean_kernel(const uint32_t* lo, const uint32_t* cstart, uint32_t L,
                                 const double2* part, double2* mean) {
  const uint32_t l = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (l >= L) return;
  double sx = 0.0, sy = 0.0;
  for (uint32_t c = cstart[l] + lane; c < cstart[l + 1]; c += 32) {
    sx = __dadd_rn(sx, part[c].x);
    sy = __dadd_rn(sy, part[c].y);
  }
  sx = warp_sum_d(sx);
  sy = warp_sum_d(sy);
  if (lane == 0) {
    const double k = (double)(lo[l + 1] - lo[l]);
    mean[l] = k > 0 ? make_double2(__ddiv_rn(sx, k), __ddiv_rn(sy, k)) : make_double2(0.0, 0.0);
  }
}

// Per chunk: centred (S_xy, S_xx).
__global__ void leaf_pass2_kernel(const uint64_t* R, const uint32_t* lo, const uint32_t* cstart,
                                  uint32_t L, const double2* mean, double2* part) {
  const uint32_t c = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  ChunkRange r;
  if (!chunk_range(cstart, lo, L, c, r)) return;
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
__global__ void leaf_final_kernel(const uint32_t* lo, const uint32_t* cstart, uint32_t L,
                                  const double2* part, const double2* mean, double2* fit,
                                  int32_t* elo, int32_t* ehi) {
  const uint32_t l = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (l >= L) return;
  double sxy = 0.0, sxx = 0.0;
  for (uint32_t c = cstart[l] + lane; c < cstart[l + 1]; c += 32) {
    sxy = __dadd_rn(sxy, part[c].x);
    sxx = __dadd_rn(sxx, part[c].y);
  }
  sxy = warp_sum_d(sxy);
  sxx = warp_sum_d(sxx);
  if (lane == 0) {
    double a = 0.0, b = 0.0;
    if (lo[l + 1] > lo[l]) {
      a = sxx > 0.0 ? __ddiv_rn(sxy, sxx) : 0.0;
      if (!(a > 0.0)) a = 0.0;
      b = __dsub_rn(mean[l].y, __dmul_rn(a, mean[l].x));
    }
    fit[l] = make_double2(a, b);
    elo[l] = INT32_MAX;
    ehi[l] = INT32_MIN;
  }
}

// ------------------------------------------------------------- A4: errors --

template <class Model>
struct Deployed;
template <>
struct Deployed<ModelF32> {
  __device__ __forceinline__ static int64_t pred(uint64_t x, uint64_t base, double2 f) {
    return ModelF32::pred_exact(x, base, f.x, f.y);
  }
};
template <>
struct Deployed<ModelF64> {
  __device__ __forceinline__ static int64_t pred(uint64_t x, uint64_t base, double2 f) {
    return ModelF64::pred_exact(x, base, f.x, f.y);
  }
};

__device__ __forceinline__ int32_t sat32(int64_t v) {
  return v < INT32_MIN ? INT32_MIN : (v > INT32_MAX ? INT32_MAX : (int32_t)v);
}

template <class Model>
__global__ void leaf_err_kernel(const uint64_t* R, const uint32_t* lo, const uint32_t* cstart,
                                uint32_t L, const double2* fit, int32_t* elo, int32_t* ehi) {
  const uint32_t c = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  ChunkRange r;
  if (!chunk_range(cstart, lo, L, c, r)) return;
  const uint64_t base = R[r.lo];
  const double2 f = fit[r.leaf];
  int32_t mn = INT32_MAX, mx = INT32_MIN;
  for (uint32_t i = r.s + lane; i < r.e; i += 32) {
    const int64_t e = (int64_t)(i - r.lo) - Deployed<Model>::pred(R[i], base, f);
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

// Leaf records + statistics.  stats: [0] sum size*width, [1] max width,
// [2] max size, [3] non-empty leaves.
template <class Model>
__global__ void leaf_records_kernel(const uint64_t* R, uint64_t n, const uint32_t* lo,
                                    uint32_t L, const double2* fit, const int32_t* elo,
                                    const int32_t* ehi, typename Model::Leaf* out,
                                    unsigned long long* stats) {
  for (uint32_t l = blockIdx.x * blockDim.x + threadIdx.x; l < L; l += gridDim.x * blockDim.x) {
    typename Model::Leaf rec{};
    const uint32_t a = lo[l], b = lo[l + 1];
    rec.lo = a;
    rec.hi = b;
    rec.base_key = a < n ? R[a] : 0;
    const double2 f = fit[l];
    Model::set_params(rec, f.x, f.y);   // deployed parameters (float or double)
    if (b > a) {
      rec.e_lo = elo[l];
      rec.e_hi = ehi[l];
      const int64_t w = (int64_t)rec.e_hi - (int64_t)rec.e_lo + 1;
      const int64_t sz = (int64_t)(b - a);
      const uint64_t width = (uint64_t)(w < sz ? w : sz);
      atomicAdd(stats + 0, (unsigned long long)width * (b - a));
      atomicMax(stats + 1, (unsigned long long)width);
      atomicMax(stats + 2, (unsigned long long)(b - a));
      atomicAdd(stats + 3, 1ull);
    } else {
      rec.e_lo = 0;
      rec.e_hi = 0;
    }
    out[l] = rec;
  }
}

int grid_for(uint64_t work, int block, int cap = 152 * 32) {
  uint64_t g = (work + block - 1) / block;
  if (g < 1) g = 1;
  if (g > (uint64_t)cap) g = cap;
  return (int)g;
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

template <class Model>
int build_leaves(lj_index* idx, Model model, cudaStream_t s, void* leaves_out) {
  const uint64_t n = idx->n;
  const uint32_t L = idx->L;
  const uint64_t* R = idx->R;
  // scratch: lo[L+1], cnt[L], cstart[L+1], mean[L], fit[L], elo[L], ehi[L],
  //          part[chunks], stats[4]
  const uint64_t max_chunks = n / kChunk + L + 1;
  const size_t b_lo = ((size_t)(L + 1) * 4 + 255) / 256 * 256;
  const size_t b_cnt = b_lo;
  const size_t b_dd = ((size_t)L * 16 + 255) / 256 * 256;
  const size_t b_i32 = ((size_t)L * 4 + 255) / 256 * 256;
  const size_t b_part = ((size_t)max_chunks * 16 + 255) / 256 * 256;
  const size_t total = b_lo + b_cnt + b_lo + 2 * b_dd + 2 * b_i32 + b_part + 256;
  char* ws = nullptr;
  LJ_CUDA(scratch_alloc((void**)&ws, total, s));
  uint32_t* lo = (uint32_t*)ws;
  uint32_t* cnt = (uint32_t*)(ws + b_lo);
  uint32_t* cstart = (uint32_t*)(ws + b_lo + b_cnt);
  double2* mean = (double2*)(ws + 2 * b_lo + b_cnt);
  double2* fit = (double2*)((char*)mean + b_dd);
  int32_t* elo = (int32_t*)((char*)fit + b_dd);
  int32_t* ehi = (int32_t*)((char*)elo + b_i32);
  double2* part = (double2*)((char*)ehi + b_i32);
  unsigned long long* stats = (unsigned long long*)((char*)part + b_part);
  LJ_CUDA(cudaMemsetAsync(stats, 0, 256, s));

  if (n == 0) {
    LJ_CUDA(cudaMemsetAsync(lo, 0, (size_t)(L + 1) * 4, s));
  } else {
    leaf_bounds_kernel<Model><<<grid_for(n, kBlock), kBlock, 0, s>>>(R, n, model, lo);
    LJ_CUDA(cudaGetLastError());
  }
  chunk_count_kernel<<<grid_for(L, kBlock), kBlock, 0, s>>>(lo, L, cnt);
  LJ_CUDA(cudaGetLastError());
  if (int rc = scan_u32(cnt, cstart, L, s)) return rc;

  const unsigned warps_chunks = (unsigned)((max_chunks * 32 + kBlock - 1) / kBlock);
  const unsigned warps_leaves = (unsigned)(((uint64_t)L * 32 + kBlock - 1) / kBlock);
  leaf_pass1_kernel<<<warps_chunks, kBlock, 0, s>>>(R, lo, cstart, L, part);
  leaf_mean_kernel<<<warps_leaves, kBlock, 0, s>>>(lo, cstart, L, part, mean);
  leaf_pass2_kernel<<<warps_chunks, kBlock, 0, s>>>(R, lo, cstart, L, mean, part);
  leaf_final_kernel<<<warps_leaves, kBlock, 0, s>>>(lo, cstart, L, part, mean, fit, elo, ehi);
  leaf_err_kernel<Model><<<warps_chunks, kBlock, 0, s>>>(R, lo, cstart, L, fit, elo, ehi);
  leaf_records_kernel<Model><<<grid_for(L, kBlock), kBlock, 0, s>>>(
      R, n, lo, L, fit, elo, ehi, (typename Model::Leaf*)leaves_out, stats);
  LJ_CUDA(cudaGetLastError());

  unsigned long long hstats[4];
  LJ_CUDA(cudaMemcpyAsync(hstats, stats, sizeof(hstats), cudaMemcpyDeviceToHost, s));
  LJ_CUDA(cudaStreamSynchronize(s));
  LJ_CUDA(scratch_free(ws, s));
  idx->stats.mean_window = n ? (double)hstats[0] / (double)n : 0.0;
  idx->stats.max_window = (uint32_t)hstats[1];
  idx->stats.max_leaf_size = (uint32_t)hstats[2];
  idx->stats.nonempty_leaves = (uint32_t)hstats[3];
  return 0;
}

}  // namespace
}  // namespace lj

extern "C" int rmi_build(const uint64_t* R_dev, uint64_t n, uint32_t leaves, int precision,
                         lj_stream_t stream, lj_index** out) {
  using namespace lj;
  if (!out) return fail(LJ_E_INVAL, "rmi_build: out is NULL");
  *out = nullptr;
  if (n > 0 && !R_dev) return fail(LJ_E_INVAL, "rmi_build: R is NULL");
  if (n >= (1ull << 32)) return fail(LJ_E_INVAL, "rmi_build: n = %llu must be below 2^32",
                                     (unsigned long long)n);
  if (leaves < 1 || leaves > (1u << 24))
    return fail(LJ_E_INVAL, "rmi_build: leaves = %u must be in [1, 2^24]", leaves);
  if (precision != LJ_FP32 && precision != LJ_FP64)
    return fail(LJ_E_INVAL, "rmi_build: unknown precision %d", precision);
  cudaStream_t s = (cudaStream_t)stream;

  lj_index* idx = new lj_index();
  idx->R = R_dev;
  idx->n = n;
  idx->L = leaves;
  idx->precision = precision;
  idx->device = current_device();
  idx->stats.n = n;
  idx->stats.leaves = leaves;
  idx->stats.precision = precision;

  auto bail = [&](int rc) {
    rmi_free(idx);
    return rc;
  };

  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return bail(fail(LJ_E_CUDA, "rmi_build: cudaEventCreate failed"));
  cudaEventRecord(e0, s);

  // scratch for checks and the root fit
  const int G = (int)std::min<uint64_t>(2048, std::max<uint64_t>(1, (n + 8191) / 8192));
  const uint64_t per = n ? (n + G - 1) / G : 1;
  char* ws = nullptr;
  cudaError_t ce = scratch_alloc((void**)&ws, 256 + (size_t)G * 16 * 2 + 256, s);
  if (ce != cudaSuccess) return bail(fail_cuda(ce, "rmi_build scratch"));
  uint32_t* flags = (uint32_t*)ws;           // [0] unsorted, [1] has duplicates
  double* mean = (double*)(ws + 64);         // 2
  double* root = (double*)(ws + 128);        // 2
  double2* part = (double2*)(ws + 256);
  int rc = 0;
  do {
    if ((ce = cudaMemsetAsync(ws, 0, 256, s)) != cudaSuccess) {
      rc = fail_cuda(ce, "memset");
      break;
    }
    if (n > 1) {
      check_sorted_kernel<<<grid_for(n, kBlock), kBlock, 0, s>>>(R_dev, n, flags);
    }
    if (n > 0) {
      root_pass1_kernel<<<G, kBlock, 0, s>>>(R_dev, n, leaves, per, part);
      root_mean_kernel<<<1, kBlock, 0, s>>>(part, G, n, mean);
      root_pass2_kernel<<<G, kBlock, 0, s>>>(R_dev, n, leaves, per, mean, part);
      root_final_kernel<<<1, kBlock, 0, s>>>(part, G, mean, root);
    }
    if ((ce = cudaGetLastError()) != cudaSuccess) {
      rc = fail_cuda(ce, "rmi_build root kernels");
      break;
    }
    uint32_t hflags[2] = {0, 0};
    double hroot[2] = {0, 0};
    cudaMemcpyAsync(hflags, flags, sizeof(hflags), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(hroot, root, sizeof(hroot), cudaMemcpyDeviceToHost, s);
    if ((ce = cudaStreamSynchronize(s)) != cudaSuccess) {
      rc = fail_cuda(ce, "rmi_build sync");
      break;
    }
    if (hflags[0]) {
      rc = fail(LJ_E_UNSORTED, "rmi_build: R is not sorted non-decreasing");
      break;
    }
    idx->unique = hflags[1] ? 0 : 1;
    if (n == 0) hroot[0] = hroot[1] = 0.0;
    idx->root_fit[0] = hroot[0];
    idx->root_fit[1] = hroot[1];
    idx->root_f64[0] = hroot[0];
    idx->root_f64[1] = hroot[1];
    idx->root_f32[0] = (float)hroot[0];
    idx->root_f32[1] = (float)hroot[1];

    const size_t rec = precision == LJ_FP64 ? sizeof(LeafF64) : sizeof(LeafF32);
    if ((ce = cudaMalloc(&idx->leaves, rec * leaves)) != cudaSuccess) {
      rc = fail_cuda(ce, "rmi_build leaf records");
      break;
    }
    if (precision == LJ_FP64) {
      const ModelF64 m = ModelF64::make(idx->root_f64[0], idx->root_f64[1], leaves);
      rc = build_leaves(idx, m, s, idx->leaves);
      idx->stats.root_a = m.a0;
      idx->stats.root_b = m.b0;
    } else {
      const ModelF32 m = ModelF32::make(idx->root_f32[0], idx->root_f32[1], leaves);
      rc = build_leaves(idx, m, s, idx->leaves);
      idx->stats.root_a = m.a0;
      idx->stats.root_b = m.b0;
    }
  } while (0);
  scratch_free(ws, s);
  cudaEventRecord(e1, s);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return bail(rc);
  if (int r2 = take_device_errors(idx->device, s)) return bail(r2);
  idx->stats.unique = idx->unique;
  idx->stats.build_ms = ms;
  *out = idx;
  return LJ_OK;
}
