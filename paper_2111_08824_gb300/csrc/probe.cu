// Probe side of RMI-INLJ: every key of S looks up the learned index of R.
//
// Section 2.A (indexed nested loop join) with the learned lookup of
// Section 2.D: root model -> leaf model -> predicted position -> binary
// search between the leaf's error bounds; Section 6.B: with duplicate keys
// every match in the range is returned.  Output pairs are written s-major,
// r-ascending.
//
// Kernels
//   probe_tile_kernel<Model, MODE, K, VEC>
//     One tile = 256 threads x K rounds x 2 probes (one 16-byte load of two
//     keys per thread and round).  Each thread keeps its 2K lookups in flight
//     together (their search loads interleave), then the tile scans its match
//     counts (warp shuffles + one warp over the per-round warp totals), takes
//     its global offset with a single-pass decoupled look-back and writes:
//       MODE kUniqueEmit   (r, j) pairs directly (single-pass join; R unique)
//       MODE kUniqueCount  counts / offsets, one search per probe (R unique)
//       MODE kDupCount     counts / offsets from a lower- and an upper-bound
//                          search (any R)
//   emit_kernel<Model>
//     Two-pass emit: recomputes each probe's lower bound, reads its offset,
//     and lets each warp write the contiguous output range of its 32 probes
//     with one coalesced 8-byte store per lane and step.
#include <algorithm>
#include <cstring>

#include "device_common.cuh"
#include "internal.h"

namespace lj {
namespace {

constexpr int kBlock = 256;
constexpr int kWarps = kBlock / 32;
enum { kUniqueEmit = 0, kUniqueCount = 1, kDupCount = 2 };

template <class Model>
struct ProbeParams {
  const uint64_t* R;
  const typename Model::Leaf* leaves;
  Model model;
  const uint64_t* S;
  uint64_t m;
  lj_pair* pairs;
  uint64_t capacity;
  uint32_t* counts;      // optional
  uint64_t* offsets;     // optional, m + 1
  uint64_t* total_out;   // optional, device
  uint64_t* total_ws;    // workspace copy of the total
  uint32_t s_base;       // added to s_idx (chunked host joins)
  TileState st;
  uint32_t* err;
  uint32_t num_tiles;
};

// Interleaved bounded searches over NP windows.  For each probe p with
// window [base, base+len): finds c = the last position whose key is < x
// (STRICT) or <= x (!STRICT), and returns res = c + 1 (so the lower bound,
// resp. the upper bound, of x) and cv = R[c] when res > window start.
template <int NP, bool STRICT>
__device__ __forceinline__ void search_last(const uint64_t* __restrict__ R,
                                            const uint64_t (&x)[NP], uint32_t (&base)[NP],
                                            uint32_t (&len)[NP], uint64_t (&cv)[NP]) {
  bool moved[NP];
  uint32_t start[NP];
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    moved[p] = false;
    start[p] = base[p];
    cv[p] = 0;
  }
  while (true) {
    bool any = false;
    uint64_t v[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p)
      if (len[p] > 1) {
        any = true;
        v[p] = ldg_key(R, base[p] + (len[p] >> 1));
      }
    if (!any) break;
#pragma unroll
    for (int p = 0; p < NP; ++p)
      if (len[p] > 1) {
        const uint32_t half = len[p] >> 1;
        const bool go = STRICT ? (v[p] < x[p]) : (v[p] <= x[p]);
        if (go) {
          base[p] += half;
          cv[p] = v[p];
          moved[p] = true;
        }
        len[p] -= half;
      }
  }
  uint64_t w[NP];
#pragma unroll
  for (int p = 0; p < NP; ++p)
    if (len[p] == 1 && !moved[p]) w[p] = ldg_key(R, base[p]);
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    if (len[p] == 0) {          // empty window
      base[p] = start[p];
    } else if (moved[p]) {
      base[p] += 1;
    } else {
      const bool go = STRICT ? (w[p] < x[p]) : (w[p] <= x[p]);
      if (go) {
        cv[p] = w[p];
        base[p] += 1;
      }
    }
    len[p] = start[p];   // keep the window start for the caller
  }
}

template <class Model, int MODE, int K, bool VEC>
__global__ void __launch_bounds__(kBlock) probe_tile_kernel(ProbeParams<Model> P) {
  constexpr int NP = 2 * K;
  static_assert(K * kWarps <= 32, "per-round warp totals must fit one warp");
  __shared__ uint32_t s_tile;
  __shared__ uint64_t s_wpre[K * kWarps];
  __shared__ uint64_t s_prefix;

  if (threadIdx.x == 0) s_tile = atomicAdd(P.st.ticket, 1u);
  __syncthreads();
  const uint32_t tile = s_tile;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t tile_base = (uint64_t)tile * (kBlock * NP);

  // ---- load keys: round k, thread t holds probes 2(k*256+t) + {0, 1}
  uint64_t x[NP];
  bool valid[NP];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const uint64_t j0 = tile_base + 2ull * (k * kBlock + threadIdx.x);
    if (VEC && j0 + 1 < P.m) {
      const ulonglong2 v = __ldg(reinterpret_cast<const ulonglong2*>(P.S + j0));
      x[2 * k] = v.x;
      x[2 * k + 1] = v.y;
      valid[2 * k] = valid[2 * k + 1] = true;
    } else {
      valid[2 * k] = j0 < P.m;
      valid[2 * k + 1] = j0 + 1 < P.m;
      x[2 * k] = valid[2 * k] ? __ldg(reinterpret_cast<const unsigned long long*>(P.S) + j0) : 0;
      x[2 * k + 1] =
          valid[2 * k + 1] ? __ldg(reinterpret_cast<const unsigned long long*>(P.S) + j0 + 1) : 0;
    }
  }

  // ---- predict: root -> leaf record -> window
  uint32_t base[NP], len[NP];
  {
    uint32_t leaf[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) leaf[p] = P.model.leaf(x[p]);
    typename Model::Leaf lf[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p)
      if (valid[p]) lf[p] = Model::load_leaf(P.leaves, leaf[p]);
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      uint32_t wl = 0, wh = 0;
      if (valid[p]) window<Model>(lf[p], x[p], wl, wh);
      base[p] = wl;
      len[p] = wh - wl;
    }
  }

  // ---- bounded search
  uint32_t r_idx[NP];
  uint32_t cnt[NP];
  if (MODE == kDupCount) {
    uint32_t wh[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) wh[p] = base[p] + len[p];
    uint64_t cv[NP];
    search_last<NP, true>(P.R, x, base, len, cv);   // base = lower bound
    uint32_t lb[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      lb[p] = base[p];
      len[p] = wh[p] - base[p];
    }
    search_last<NP, false>(P.R, x, base, len, cv);  // base = upper bound
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      cnt[p] = valid[p] ? base[p] - lb[p] : 0;
      r_idx[p] = lb[p];
    }
  } else {
    uint64_t cv[NP];
    search_last<NP, false>(P.R, x, base, len, cv);  // base = upper bound, len = start
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      const bool match = valid[p] && base[p] > len[p] && cv[p] == x[p];
      cnt[p] = match ? 1u : 0u;
      r_idx[p] = base[p] - 1;
    }
  }

  // ---- tile scan: per round a warp scan, then one warp over the K*8 totals
  uint64_t lane_excl[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const uint64_t s = (uint64_t)cnt[2 * k] + cnt[2 * k + 1];
    const uint64_t inc = warp_inclusive_sum(s, lane);
    lane_excl[k] = inc - s;
    if (lane == 31) s_wpre[k * kWarps + warp] = inc;
  }
  __syncthreads();
  if (warp == 0) {
    const uint64_t v = lane < K * kWarps ? s_wpre[lane] : 0;
    const uint64_t inc = warp_inclusive_sum(v, lane);
    if (lane < K * kWarps) s_wpre[lane] = inc - v;
    const uint64_t agg = __shfl_sync(0xffffffffu, inc, 31);
    const uint64_t pre = lookback_warp(P.st, tile, agg, P.err);
    if (lane == 0) {
      s_prefix = pre;
      if (tile + 1 == P.num_tiles) {
        const uint64_t total = pre + agg;
        *P.total_ws = total;
        if (P.total_out) *P.total_out = total;
        if (P.offsets) P.offsets[P.m] = total;
        if (MODE == kUniqueEmit && total > P.capacity) atomicOr(P.err, kErrCapacity);
      }
    }
  }
  __syncthreads();
  const uint64_t tile_prefix = s_prefix;

  // ---- outputs
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const uint64_t j0 = tile_base + 2ull * (k * kBlock + threadIdx.x);
    const uint64_t o0 = tile_prefix + s_wpre[k * kWarps + warp] + lane_excl[k];
    const uint64_t o1 = o0 + cnt[2 * k];
    if (MODE == kUniqueEmit) {
      if (cnt[2 * k] && o0 < P.capacity)
        P.pairs[o0] = lj_pair{r_idx[2 * k], (uint32_t)(j0 + P.s_base)};
      if (cnt[2 * k + 1] && o1 < P.capacity)
        P.pairs[o1] = lj_pair{r_idx[2 * k + 1], (uint32_t)(j0 + 1 + P.s_base)};
    } else {
      if (VEC && j0 + 1 < P.m) {
        if (P.offsets) *reinterpret_cast<ulonglong2*>(P.offsets + j0) = make_ulonglong2(o0, o1);
        if (P.counts) *reinterpret_cast<uint2*>(P.counts + j0) = make_uint2(cnt[2 * k], cnt[2 * k + 1]);
      } else {
        if (valid[2 * k]) {
          if (P.offsets) P.offsets[j0] = o0;
          if (P.counts) P.counts[j0] = cnt[2 * k];
        }
        if (valid[2 * k + 1]) {
          if (P.offsets) P.offsets[j0 + 1] = o1;
          if (P.counts) P.counts[j0 + 1] = cnt[2 * k + 1];
        }
      }
    }
  }
}

// Two-pass emit: warp w of block b handles probes [b*256 + 32w, +32).
template <class Model>
__global__ void __launch_bounds__(kBlock) emit_kernel(ProbeParams<Model> P) {
  __shared__ uint64_t s_off[kWarps][33];
  __shared__ uint32_t s_lb[kWarps][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t j = blockIdx.x * (uint64_t)kBlock + threadIdx.x;
  const uint64_t j_warp = j - lane;
  uint32_t lb = 0;
  uint64_t off = 0, end = 0;
  if (j < P.m) {
    const uint64_t key = __ldg(reinterpret_cast<const unsigned long long*>(P.S) + j);
    const typename Model::Leaf lf = Model::load_leaf(P.leaves, P.model.leaf(key));
    uint32_t wl, wh;
    window<Model>(lf, key, wl, wh);
    uint64_t xk[1] = {key};
    uint32_t b[1] = {wl}, l[1] = {wh - wl};
    uint64_t cv[1];
    search_last<1, true>(P.R, xk, b, l, cv);
    lb = b[0];
    off = P.offsets[j];
    end = P.offsets[j + 1];
  }
  // last valid lane's end closes the warp's range
  const uint64_t rem = P.m > j_warp ? P.m - 1 - j_warp : 0;
  const uint64_t last = rem < 31 ? rem : 31;
  s_off[warp][lane] = off;
  s_lb[warp][lane] = lb;
  const uint64_t warp_end = __shfl_sync(0xffffffffu, end, (int)last);
  if (lane == 0) s_off[warp][32] = warp_end;
  __syncwarp();
  if (j_warp >= P.m) return;
  const uint64_t warp_start = s_off[warp][0];
  if (lane == 0 && warp_end > P.capacity) atomicOr(P.err, kErrCapacity);
  const uint64_t stop = min(warp_end, P.capacity);
  int p = 0;
  for (uint64_t q = warp_start + lane; q < stop; q += 32) {
    while (p < (int)last && s_off[warp][p + 1] <= q) ++p;
    P.pairs[q] = lj_pair{s_lb[warp][p] + (uint32_t)(q - s_off[warp][p]),
                         (uint32_t)(j_warp + p + P.s_base)};
  }
}

constexpr int kRounds = 4;   // probes per thread = 2 * kRounds
constexpr uint64_t kTileProbes = (uint64_t)kBlock * 2 * kRounds;

struct Workspace {
  void* mem = nullptr;
  TileState st{};
  uint64_t* total = nullptr;
  uint32_t tiles = 0;
};

int ws_acquire(Workspace& w, uint64_t m, cudaStream_t s) {
  w.tiles = (uint32_t)std::max<uint64_t>(1, (m + kTileProbes - 1) / kTileProbes);
  const size_t flags = ((size_t)w.tiles * 4 + 255) / 256 * 256;
  const size_t bytes = 256 + flags + (size_t)w.tiles * 16;
  LJ_CUDA(scratch_alloc(&w.mem, bytes, s));
  char* b = (char*)w.mem;
  LJ_CUDA(cudaMemsetAsync(b, 0, 256 + flags, s));
  w.st.ticket = (uint32_t*)b;
  w.total = (uint64_t*)(b + 64);
  w.st.flag = (uint32_t*)(b + 256);
  w.st.agg = (uint64_t*)(b + 256 + flags);
  w.st.incl = w.st.agg + w.tiles;
  return 0;
}

template <class Model>
int launch_probe(const lj_index* idx, Model model, int mode, const uint64_t* S, uint64_t m,
                 lj_pair* pairs, uint64_t cap, uint32_t* counts, uint64_t* offsets,
                 uint64_t* total_dev, uint64_t* total_host, uint32_t s_base, cudaStream_t s) {
  Workspace w;
  if (int rc = ws_acquire(w, m, s)) return rc;
  ProbeParams<Model> P;
  P.R = idx->R;
  P.leaves = (const typename Model::Leaf*)idx->leaves;
  P.model = model;
  P.S = S;
  P.m = m;
  P.pairs = pairs;
  P.capacity = cap;
  P.counts = counts;
  P.offsets = offsets;
  P.total_out = total_dev;
  P.total_ws = w.total;
  P.s_base = s_base;
  P.st = w.st;
  P.err = device_error_word(idx->device);
  P.num_tiles = w.tiles;
  if (!P.err) return fail(LJ_E_NOMEM, "cannot allocate the device error word");
  const bool vec = (reinterpret_cast<uintptr_t>(S) & 15) == 0 &&
                   (!offsets || (reinterpret_cast<uintptr_t>(offsets) & 15) == 0) &&
                   (!counts || (reinterpret_cast<uintptr_t>(counts) & 7) == 0);
  const dim3 grid(w.tiles), block(kBlock);
#define LJ_LAUNCH(MODE)                                                            \
  (vec ? probe_tile_kernel<Model, MODE, kRounds, true><<<grid, block, 0, s>>>(P)  \
       : probe_tile_kernel<Model, MODE, kRounds, false><<<grid, block, 0, s>>>(P))
  if (mode == kUniqueEmit)
    LJ_LAUNCH(kUniqueEmit);
  else if (mode == kUniqueCount)
    LJ_LAUNCH(kUniqueCount);
  else
    LJ_LAUNCH(kDupCount);
#undef LJ_LAUNCH
  LJ_CUDA(cudaGetLastError());
  if (total_host) LJ_CUDA(cudaMemcpyAsync(total_host, w.total, 8, cudaMemcpyDeviceToHost, s));
  LJ_CUDA(scratch_free(w.mem, s));
  if (total_host) {
    LJ_CUDA(cudaStreamSynchronize(s));
    if (int rc = take_device_errors(idx->device, s)) return rc;
  }
  return 0;
}

template <class Model>
int launch_emit(const lj_index* idx, Model model, const uint64_t* S, uint64_t m,
                const uint64_t* offsets, lj_pair* pairs, uint64_t cap, uint32_t s_base,
                cudaStream_t s) {
  ProbeParams<Model> P{};
  P.R = idx->R;
  P.leaves = (const typename Model::Leaf*)idx->leaves;
  P.model = model;
  P.S = S;
  P.m = m;
  P.pairs = pairs;
  P.capacity = cap;
  P.offsets = const_cast<uint64_t*>(offsets);
  P.s_base = s_base;
  P.err = device_error_word(idx->device);
  if (!P.err) return fail(LJ_E_NOMEM, "cannot allocate the device error word");
  const uint64_t blocks = (m + kBlock - 1) / kBlock;
  emit_kernel<Model><<<(unsigned)blocks, kBlock, 0, s>>>(P);
  LJ_CUDA(cudaGetLastError());
  return 0;
}

ModelF32 f32_model(const lj_index* idx) {
  return ModelF32{idx->root_f32[0], idx->root_f32[1], idx->L};
}
ModelF64 f64_model(const lj_index* idx) {
  return ModelF64{idx->root_f64[0], idx->root_f64[1], idx->L};
}

int check_common(const lj_index* idx, const uint64_t* S, uint64_t m, const char* who) {
  if (!idx) return fail(LJ_E_INVAL, "%s: index is NULL", who);
  if (m >= (1ull << 32)) return fail(LJ_E_INVAL, "%s: m must be below 2^32", who);
  if (m > 0 && !S) return fail(LJ_E_INVAL, "%s: S is NULL", who);
  if (current_device() != idx->device)
    return fail(LJ_E_INVAL, "%s: index lives on device %d, current device is %d", who,
                idx->device, current_device());
  return 0;
}

}  // namespace

// Shared with the chunked host join (same translation unit family).
int probe_count_impl(const lj_index* idx, const uint64_t* S, uint64_t m, uint32_t* counts,
                     uint64_t* offsets, uint64_t* total_dev, uint64_t* total_host,
                     cudaStream_t s) {
  const int mode = idx->unique ? kUniqueCount : kDupCount;
  if (idx->precision == LJ_FP64)
    return launch_probe(idx, f64_model(idx), mode, S, m, nullptr, 0, counts, offsets, total_dev,
                        total_host, 0, s);
  return launch_probe(idx, f32_model(idx), mode, S, m, nullptr, 0, counts, offsets, total_dev,
                      total_host, 0, s);
}

int probe_emit_impl(const lj_index* idx, const uint64_t* S, uint64_t m, const uint64_t* offsets,
                    lj_pair* pairs, uint64_t cap, uint64_t* total_dev, uint64_t* total_host,
                    uint32_t s_base, cudaStream_t s) {
  if (!offsets) {
    if (idx->precision == LJ_FP64)
      return launch_probe(idx, f64_model(idx), kUniqueEmit, S, m, pairs, cap, nullptr, nullptr,
                          total_dev, total_host, s_base, s);
    return launch_probe(idx, f32_model(idx), kUniqueEmit, S, m, pairs, cap, nullptr, nullptr,
                        total_dev, total_host, s_base, s);
  }
  int rc = idx->precision == LJ_FP64
               ? launch_emit(idx, f64_model(idx), S, m, offsets, pairs, cap, s_base, s)
               : launch_emit(idx, f32_model(idx), S, m, offsets, pairs, cap, s_base, s);
  if (rc) return rc;
  if (total_dev) LJ_CUDA(cudaMemcpyAsync(total_dev, offsets + m, 8, cudaMemcpyDeviceToDevice, s));
  if (total_host) {
    LJ_CUDA(cudaMemcpyAsync(total_host, offsets + m, 8, cudaMemcpyDeviceToHost, s));
    LJ_CUDA(cudaStreamSynchronize(s));
    if (int r2 = take_device_errors(idx->device, s)) return r2;
  }
  return 0;
}

}  // namespace lj

extern "C" int join_count(const lj_index* idx, const uint64_t* S_dev, uint64_t m,
                          uint32_t* counts_dev, uint64_t* offsets_dev, uint64_t* total_host,
                          lj_stream_t stream) {
  using namespace lj;
  if (int rc = check_common(idx, S_dev, m, "join_count")) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if (m == 0) {
    if (offsets_dev) LJ_CUDA(cudaMemsetAsync(offsets_dev, 0, 8, s));
    if (total_host) {
      *total_host = 0;
      LJ_CUDA(cudaStreamSynchronize(s));
    }
    return LJ_OK;
  }
  return probe_count_impl(idx, S_dev, m, counts_dev, offsets_dev, nullptr, total_host, s);
}

extern "C" int join_emit(const lj_index* idx, const uint64_t* S_dev, uint64_t m,
                         const uint64_t* offsets_dev, lj_pair* pairs_dev, uint64_t capacity,
                         uint64_t* written_dev, uint64_t* written_host, lj_stream_t stream) {
  using namespace lj;
  if (int rc = check_common(idx, S_dev, m, "join_emit")) return rc;
  if (capacity > 0 && !pairs_dev) return fail(LJ_E_INVAL, "join_emit: pairs is NULL");
  if (!offsets_dev && !idx->unique)
    return fail(LJ_E_NOTUNIQUE,
                "join_emit: the single-pass path needs an R without duplicate keys; "
                "call join_count first and pass its offsets");
  cudaStream_t s = (cudaStream_t)stream;
  if (m == 0) {
    if (written_dev) LJ_CUDA(cudaMemsetAsync(written_dev, 0, 8, s));
    if (written_host) {
      *written_host = 0;
      LJ_CUDA(cudaStreamSynchronize(s));
    }
    return LJ_OK;
  }
  int rc = probe_emit_impl(idx, S_dev, m, offsets_dev, pairs_dev, capacity, written_dev,
                           written_host, 0, s);
  if (rc) return rc;
  if (written_host && *written_host > capacity)
    return fail(LJ_E_CAPACITY, "join_emit: %llu pairs do not fit the capacity of %llu",
                (unsigned long long)*written_host, (unsigned long long)capacity);
  return LJ_OK;
}
