// Probe side of RMI-INLJ: every key of S looks up the learned index of R.
//
// Section 2.A (indexed nested loop join) with the learned lookup of
// Section 2.D: root model -> leaf model -> predicted position -> binary
// search between the leaf's error bounds; Section 6.B: with duplicate keys
// every match in the range is returned.  Output pairs are written s-major,
// r-ascending.
//
// Execution paths, chosen by the size of the probe batch:
//   fused (join_emit against a unique R, m <= fused_max, default 2^21):
//     probe_fused_kernel: one cooperative launch of resident blocks;
//     lookups, a grid-wide barrier, block prefixes from group sums, pairs.
//   single pass (m <= single_pass_max, default 0, i.e. on request only):
//     probe_single_pass_kernel<Model, MODE, K, VEC>: block tiles of 256
//     threads x K rounds x 2 probes; lookups, block scan, decoupled look-back
//     and writes in one launch.
//   count-scan-emit pipeline (larger batches):
//     probe_search_kernel: lookups only, one 32-bit word per probe (first
//       match or "none" for a unique R, the match count otherwise); no scan
//       and no barrier, so a warp never waits for a slower one.
//       Each warp also adds its probes' match count to its tile's count.
//     tile_scan_kernel: exclusive scan of the per-tile counts.
//     compact_kernel: every tile scans its words, stages its output in shared
//       memory and writes it with coalesced stores (pairs, or offsets and
//       counts); tiles know their offsets up front, so none waits.
//   Measured on the 100M x 400M lognormal workload, the single-pass kernel
//   spent almost half its time waiting in the look-back for tiles whose
//   searches were slower; the pipeline's extra 8 bytes per probe of
//   streaming traffic cost far less.
//   gapped_search_kernel: the search kernel with the lookup of a gapped RMI
//     (Section 3.A: exponential search from the predicted slot in the gapped
//     key array, position read from the payload array); an index with
//     gapped arrays always takes the pipeline.
//   expand_kernel: pairs of the ranges located by join_locate (first match
//     and offsets per probe); no second search.
//   emit_kernel<Model>: two-pass emit from join_count's offsets; recomputes
//     each probe's lower bound and lets each warp write the contiguous
//     output range of its 32 probes with coalesced 8-byte stores.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <mutex>

#include "device_common.cuh"
#include "internal.h"
#include "probe_core.cuh"

namespace lj {
namespace {

// Probe batches up to this size take the single-pass kernel (one launch).
// Default 0: with the L2 flushed, 2^14 .. 2^22 probes took 24-100 us through
// the pipeline against 28-170 us in the single-pass kernel, whose blocks of
// 2048 probes leave most SMs idle on small batches and wait in the
// look-back on large ones.
std::atomic<uint64_t> g_single_pass_max{0};

// Unique-R batches up to this size take the fused cooperative kernel
// (option "fused_max"); fused_groups = 1 searches their windows on 4-key
// groups (option "fused_groups").  Measured with the L2 flushed (uniform
// 1M-key R, L = 4096, fp64 model): 2^14 probes 17.4 -> 16.5 us, 2^18
// 23.3 -> 19.1 us, 2^20 40.6 -> 37.0 us, 2^21 71.3 -> 61.5 us against the
// pipeline; bisection instead of the 4-key groups: 2^20 40.1 us.
std::atomic<uint64_t> g_fused_max{1ull << 21};
std::atomic<int> g_fused_groups{1};
constexpr uint32_t kFusedMaxPerBlock = 4096;   // probes (words in shared memory) per block

// Bucketed probe order in the pipeline (option "probe_buckets"; off by
// default: it pays where probes spread over an R larger than L2, and costs
// where they concentrate on a few hot regions).
std::atomic<int> g_probe_buckets{0};

// Writes of one round: pairs (kUniqueEmit) or counts / offsets.
template <class Model, int MODE, bool VEC>
__device__ __forceinline__ void write_round(const ProbeParams<Model>& P, uint64_t j0,
                                            uint64_t o0, uint32_t c0, uint32_t c1, uint32_t r0,
                                            uint32_t r1, bool v0, bool v1) {
  const uint64_t o1 = o0 + c0;
  if (MODE == kUniqueEmit) {
    if (c0 && o0 < P.capacity) P.pairs[o0] = lj_pair{r0, (uint32_t)(j0 + P.s_base)};
    if (c1 && o1 < P.capacity) P.pairs[o1] = lj_pair{r1, (uint32_t)(j0 + 1 + P.s_base)};
  } else if (VEC && v1) {
    if (P.offsets) *reinterpret_cast<ulonglong2*>(P.offsets + j0) = make_ulonglong2(o0, o1);
    if (P.counts) *reinterpret_cast<uint2*>(P.counts + j0) = make_uint2(c0, c1);
    if (P.first) *reinterpret_cast<uint2*>(P.first + j0) = make_uint2(r0, r1);
  } else {
    if (v0) {
      if (P.offsets) P.offsets[j0] = o0;
      if (P.counts) P.counts[j0] = c0;
      if (P.first) P.first[j0] = r0;
    }
    if (v1) {
      if (P.offsets) P.offsets[j0 + 1] = o1;
      if (P.counts) P.counts[j0 + 1] = c1;
      if (P.first) P.first[j0 + 1] = r1;
    }
  }
}

template <class Model, int MODE>
__device__ __forceinline__ void last_tile_total(const ProbeParams<Model>& P, uint64_t total) {
  *P.total_ws = total;
  if (P.total_out) *P.total_out = total;
  if (P.offsets) P.offsets[P.m] = total;
  if (MODE == kUniqueEmit && total > P.capacity) atomicOr(P.err, kErrCapacity);
}


// Single-pass kernel (small probe batches): block tiles of 256 threads x K
// rounds x 2 probes; the block scans its counts, warp 0 takes the tile's
// offset by look-back, then the block writes pairs or offsets directly.
template <class Model, int MODE, int K, bool VEC>
__global__ void __launch_bounds__(kBlock, LJ_MINB) probe_single_pass_kernel(ProbeParams<Model> P) {
  static_assert(K * kWarps <= 32, "per-round warp totals must fit one warp");
  __shared__ uint32_t s_tile;
  __shared__ uint64_t s_wpre[K * kWarps];
  __shared__ uint64_t s_prefix;
  if (threadIdx.x == 0) s_tile = atomicAdd(P.st.ticket, 1u) + P.tile_skip;
  __syncthreads();
  const uint32_t tile = s_tile;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t tile_base = (uint64_t)tile * (kBlock * 2 * K);
  uint32_t r_idx[2 * K], cnt[2 * K];
  bool valid[2 * K];
  lookup_probes<Model, MODE, K, VEC>(P, tile_base + 2ull * threadIdx.x, kBlock, r_idx, cnt, valid);
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
      if (tile + 1 == P.num_tiles) last_tile_total<Model, MODE>(P, pre + agg);
    }
  }
  __syncthreads();
  const uint64_t tile_prefix = s_prefix;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const uint64_t j0 = tile_base + 2ull * (k * kBlock + threadIdx.x);
    write_round<Model, MODE, VEC>(P, j0, tile_prefix + s_wpre[k * kWarps + warp] + lane_excl[k],
                                  cnt[2 * k], cnt[2 * k + 1], r_idx[2 * k], r_idx[2 * k + 1],
                                  valid[2 * k], valid[2 * k + 1]);
  }
}

// Fused kernel for small batches against a unique R (join_emit's direct
// path, m <= fused_max): one cooperative launch of resident blocks.  Block b
// owns the contiguous probes [b * per_block, (b + 1) * per_block):
//   1. lookups, two probes per thread and round, one word per probe kept in
//      shared memory (first match or kNoMatch);
//   2. the block's match count goes to bcount[b] and to the sum of its group
//      of 32 blocks; then a grid-wide barrier (bounded wait);
//   3. exclusive prefix of block b = the sums of the groups before its group
//      + the counts of the blocks before it in its group (two warp loads);
//   4. the block writes its pairs in probe order, 256 words per step (warp
//      ballots, one block scan of 8 warp totals), coalesced 8-byte stores.
// Compared with the pipeline this saves a launch, the per-probe words'
// round trip through memory and the compaction's prefix sums; compared with
// the single-pass kernel no block waits for a predecessor's lookups: the
// barrier is passed once, when every block has counted.
constexpr int kFusedBlock = 256;
constexpr uint32_t kFusedGroup = 32;   // blocks per group sum

struct FusedState {
  uint32_t* arrive;              // barrier counter, zeroed before the launch
  unsigned long long* gsum;      // per group of kFusedGroup blocks, zeroed
  uint32_t* bcount;              // per block (written before the barrier)
  uint32_t polls;                // bound of the barrier wait (polls)
};

template <class Model, bool VEC, int SEARCH>
__global__ void __launch_bounds__(kFusedBlock, LJ_FMINB)
    probe_fused_kernel(ProbeParams<Model> P, FusedState F, uint32_t per_block) {
  extern __shared__ uint32_t s_word[];   // per_block words
  __shared__ uint32_t s_wsum[kFusedBlock / 32];
  __shared__ unsigned long long s_prefix;
  if (blockIdx.x < P.tile_skip) return;   // fault-injection hook (0): such blocks never arrive
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t b0 = (uint64_t)blockIdx.x * per_block;
  const uint32_t nb = b0 < P.m ? (uint32_t)(P.m - b0 < per_block ? P.m - b0 : per_block) : 0u;
  uint32_t c = 0;
#pragma unroll 1
  for (uint32_t o = 2 * threadIdx.x; o < nb; o += 2 * kFusedBlock) {
    uint32_t r_idx[2], cnt[2];
    bool valid[2];
    lookup_probes<Model, kUniqueCount, 1, VEC, SEARCH>(P, b0 + o, 0, r_idx, cnt, valid);
    s_word[o] = cnt[0] ? r_idx[0] : kNoMatch;
    if (o + 1 < nb) s_word[o + 1] = cnt[1] ? r_idx[1] : kNoMatch;
    c += cnt[0] + cnt[1];   // probe o + 1 >= nb only at the end of S: cnt[1] = 0
  }
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) c += __shfl_xor_sync(0xffffffffu, c, d);
  if (lane == 0) s_wsum[warp] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t tot = 0;
#pragma unroll
    for (int w = 0; w < kFusedBlock / 32; ++w) tot += s_wsum[w];
    F.bcount[blockIdx.x] = tot;
    if (tot) atomicAdd(F.gsum + blockIdx.x / kFusedGroup, (unsigned long long)tot);
    __threadfence();
    atomicAdd(F.arrive, 1u);
    // every block is resident (cooperative launch), so the wait ends; it is
    // still bounded, and a timeout is reported as an error
    uint32_t polls = 0;
    while (ld_acquire_u32(F.arrive) < gridDim.x) {
      if (++polls > F.polls) {
        atomicOr(P.err, kErrLookbackTimeout);
        break;
      }
      __nanosleep(64);
    }
  }
  __syncthreads();
  if (warp == 0) {
    const uint32_t g = blockIdx.x / kFusedGroup, g0 = g * kFusedGroup;
    unsigned long long pre = 0;
    for (uint32_t q = lane; q < g; q += 32) pre += __ldcg(F.gsum + q);
    if (g0 + lane < blockIdx.x) pre += __ldcg(F.bcount + g0 + lane);
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) pre += __shfl_xor_sync(0xffffffffu, pre, d);
    if (lane == 0) {
      s_prefix = pre;
      if (blockIdx.x + 1 == gridDim.x) last_tile_total<Model, kUniqueEmit>(P, pre + __ldcg(F.bcount + blockIdx.x));
    }
  }
  __syncthreads();
  unsigned long long run = s_prefix;
  const unsigned below = (1u << lane) - 1u;
#pragma unroll 1
  for (uint32_t o = 0; o < nb; o += kFusedBlock) {
    const uint32_t i = o + threadIdx.x;
    const uint32_t w = i < nb ? s_word[i] : kNoMatch;
    const unsigned bal = __ballot_sync(0xffffffffu, w != kNoMatch);
    if (lane == 0) s_wsum[warp] = __popc(bal);
    __syncthreads();
    uint32_t woff = 0, tot = 0;
#pragma unroll
    for (int q = 0; q < kFusedBlock / 32; ++q) {
      const uint32_t t = s_wsum[q];
      woff += q < warp ? t : 0u;
      tot += t;
    }
    if (w != kNoMatch) {
      const unsigned long long pos = run + woff + __popc(bal & below);
      if (pos < P.capacity) P.pairs[pos] = lj_pair{w, (uint32_t)(b0 + i + P.s_base)};
    }
    run += tot;
    __syncthreads();   // s_wsum is rewritten by the next step
  }
}

// Two-pass emit: warp w of block b handles probes [b*256 + 32w, +32).
template <class Model, int GAP>
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
    uint64_t xk[1] = {key};
    if constexpr (GAP == 3) {                       // RadixSpline hash: no leaf record
      uint32_t q[1] = {gapped_start<Model, kRsHash>(P, typename Model::Leaf{}, key)};
      uint64_t v[1];
      gallop_first<1, false>(P.gkeys, P.gslots, xk, q, v);
      lb = __ldg(P.dfirst + __ldg(P.gpos + q[0]));  // the distinct-key rank's first position
    } else if constexpr (GAP != 0) {
      const typename Model::Leaf lf = Model::load_leaf(P.leaves, P.model.leaf(key));
      uint32_t q[1] = {gapped_start<Model, GAP == 2 ? kRmiHash : kGappedRmi>(P, lf, key)};
      uint64_t v[1];
      gallop_first<1, false>(P.gkeys, P.gslots, xk, q, v);
      lb = __ldg(P.gpos + q[0]);                    // GAP 2: the distinct-key rank
      if (GAP == 2) lb = __ldg(P.dfirst + lb);      // (rank D: dfirst[D] = n, unused)
    } else {
      const typename Model::Leaf lf = Model::load_leaf(P.leaves, P.model.leaf(key));
      uint32_t wl, wh;
      window<Model>(lf, key, wl, wh);
      uint32_t b[1] = {wl}, l[1] = {wh - wl};
      uint64_t cv[1];
      search_last<1, true>(P.R, xk, b, l, cv);
      lb = b[0];
    }
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

// Expansion of located ranges (join_expand): warp w of block b handles
// probes [b*256 + 32w, +32) like emit_kernel, with each probe's first match
// read from `first` instead of searched again.  The warp's output range is
// written in aligned groups of 4 pairs (one 32-byte store per lane), with
// 32-bit offsets relative to the warp's first pair; a lane walks forward
// through the warp's probes as its positions grow.
__device__ __forceinline__ void st_pairs4(lj_pair* p, const uint32_t (&r)[4], const uint32_t (&j)[4]) {
  const unsigned long long a = ((unsigned long long)j[0] << 32) | r[0];
  const unsigned long long b = ((unsigned long long)j[1] << 32) | r[1];
  const unsigned long long c = ((unsigned long long)j[2] << 32) | r[2];
  const unsigned long long d = ((unsigned long long)j[3] << 32) | r[3];
  asm volatile("st.global.v4.u64 [%0], {%1, %2, %3, %4};" ::"l"(p), "l"(a), "l"(b), "l"(c), "l"(d)
               : "memory");
}

__global__ void __launch_bounds__(kBlock)
    expand_kernel(const uint32_t* __restrict__ first, const uint64_t* __restrict__ offsets,
                  uint64_t m, lj_pair* __restrict__ pairs, uint64_t capacity, uint32_t s_base,
                  uint32_t* err) {
  __shared__ uint64_t s_off[kWarps][33];
  __shared__ uint32_t s_rel[kWarps][33];
  __shared__ uint32_t s_lb[kWarps][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t j = blockIdx.x * (uint64_t)kBlock + threadIdx.x;
  const uint64_t j_warp = j - lane;
  uint32_t lb = 0;
  uint64_t off = 0, end = 0;
  if (j < m) {
    off = offsets[j];
    end = offsets[j + 1];
    if (end > off) lb = first[j];
  }
  const uint64_t rem = m > j_warp ? m - 1 - j_warp : 0;
  const int last = rem < 31 ? (int)rem : 31;
  s_off[warp][lane] = off;
  s_lb[warp][lane] = lb;
  const uint64_t warp_end = __shfl_sync(0xffffffffu, end, last);
  if (lane == 0) s_off[warp][32] = warp_end;
  __syncwarp();
  if (j_warp >= m) return;
  const uint64_t warp_start = s_off[warp][0];
  if (lane == 0 && warp_end > capacity) atomicOr(err, kErrCapacity);
  const uint64_t stop = min(warp_end, capacity);
  if (stop <= warp_start) return;
  const uint32_t sj = (uint32_t)(j_warp + s_base);
  if (stop - warp_start >= (1ull << 31) ||
      (reinterpret_cast<uintptr_t>(pairs) & 31) != 0) {   // huge ranges or an unaligned output:
                                                           // 64-bit positions, one pair at a time
    int p = 0;
    for (uint64_t q = warp_start + lane; q < stop; q += 32) {
      while (p < last && s_off[warp][p + 1] <= q) ++p;
      pairs[q] = lj_pair{s_lb[warp][p] + (uint32_t)(q - s_off[warp][p]), sj + p};
    }
    return;
  }
  // positions relative to warp_start (32-bit); probes past `last` start at the end
  s_rel[warp][lane] = lane <= last ? (uint32_t)(s_off[warp][lane] - warp_start)
                                   : (uint32_t)(warp_end - warp_start);
  if (lane == 0) s_rel[warp][32] = (uint32_t)(warp_end - warp_start);
  __syncwarp();
  const uint32_t total = (uint32_t)(stop - warp_start);
  const uint32_t head = (uint32_t)((4 - (warp_start & 3)) & 3);   // pairs before the first aligned group
  lj_pair* out = pairs + warp_start;
  int p = 0;
  if ((uint32_t)lane < head && (uint32_t)lane < total) {
    const uint32_t t = lane;
    while (p < last && s_rel[warp][p + 1] <= t) ++p;
    out[t] = lj_pair{s_lb[warp][p] + (t - s_rel[warp][p]), sj + p};
  }
  p = 0;
  for (uint32_t t0 = head + 4u * lane; t0 < total; t0 += 128u) {
    uint32_t r[4], jj[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint32_t t = t0 + k;
      while (p < last && s_rel[warp][p + 1] <= t) ++p;
      r[k] = s_lb[warp][p] + (t - s_rel[warp][p]);
      jj[k] = sj + p;
    }
    if (t0 + 4 <= total) {
      st_pairs4(out + t0, r, jj);
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (t0 + k < total) out[t0 + k] = lj_pair{r[k], jj[k]};
    }
  }
}

// Search kernel of the count-scan-emit pipeline: block b looks up the CHUNK
// consecutive tiles of 2*kSearchBlock probes starting at probe
// b * CHUNK * 2 * kSearchBlock, two probes per thread and tile, and writes one
// 32-bit word per probe, with no scan, so a warp never waits for a slower one
// until the end of its block's chunk:
//   kUniqueCount  out[j] = first matching position, or kNoMatch
//   kDupCount     out[j] = number of matches
// At the end of the chunk the block adds its probes' match count to the
// count of their compaction tile (a chunk never straddles two): one barrier
// and one atomic per chunk (per-warp atomics contended badly).
template <class Model, int MODE, int CHUNK, bool VEC, int GAP, int SEARCH = kSearchHalve>
__device__ __forceinline__ void search_chunk(const ProbeParams<Model>& P, uint32_t* __restrict__ out,
                                             unsigned long long* __restrict__ tile_counts) {
  constexpr uint64_t kChunkProbes = 2ull * kSearchBlock * CHUNK;
  static_assert((256ull * kSmallScanItems) % kChunkProbes == 0,
                "a chunk must lie in one compaction tile");
  __shared__ unsigned long long s_count[kSearchBlock / 32];
  const uint64_t first = blockIdx.x * kChunkProbes;
  unsigned long long c = 0;
#pragma unroll 1
  for (int t = 0; t < CHUNK; ++t) {
    const uint64_t j0 = first + (uint64_t)t * 2 * kSearchBlock + 2 * threadIdx.x;
    if (__all_sync(0xffffffffu, j0 >= P.m)) break;   // warp-uniform: lookups run as a warp
    uint32_t r_idx[2], cnt[2];
    bool valid[2];
    if constexpr (GAP != 0)
      lookup_gapped<Model, MODE, VEC, GAP - 1>(P, j0, r_idx, cnt, valid);
    else
      lookup_probes<Model, MODE, 1, VEC, SEARCH>(P, j0, 0, r_idx, cnt, valid);
    uint32_t w0, w1;
    if (MODE == kDupCount) {
      w0 = cnt[0];
      w1 = cnt[1];
    } else {
      w0 = cnt[0] ? r_idx[0] : kNoMatch;
      w1 = cnt[1] ? r_idx[1] : kNoMatch;
    }
    if (VEC && valid[1]) {
      st_stream_u32x2(out + j0, w0, w1);
    } else {
      if (valid[0]) out[j0] = w0;
      if (valid[1]) out[j0 + 1] = w1;
    }
    if (P.first) {   // join_locate: where each probe's matches start
      if (VEC && valid[1]) {
        st_stream_u32x2(P.first + j0, r_idx[0], r_idx[1]);
      } else {
        if (valid[0]) P.first[j0] = r_idx[0];
        if (valid[1]) P.first[j0 + 1] = r_idx[1];
      }
    }
    c += (unsigned long long)cnt[0] + cnt[1];
  }
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) c += __shfl_xor_sync(0xffffffffu, c, d);
  if ((threadIdx.x & 31) == 0) s_count[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long tot = 0;
#pragma unroll
    for (int w = 0; w < kSearchBlock / 32; ++w) tot += s_count[w];
    if (tot) atomicAdd(tile_counts + (first >> P.tile_shift), tot);
  }
}

template <class Model, int MODE, int CHUNK, bool VEC>
__global__ void __launch_bounds__(kSearchBlock, LJ_SMINB)
    probe_search_kernel(ProbeParams<Model> P, uint32_t* __restrict__ out,
                        unsigned long long* __restrict__ tile_counts) {
  search_chunk<Model, MODE, CHUNK, VEC, 0>(P, out, tile_counts);
}

// The same with the bounded search as a descent of R's key levels
// (search_levels), for an index that has them.
template <class Model, int MODE, int CHUNK, bool VEC>
__global__ void __launch_bounds__(kSearchBlock, LJ_LMINB)
    levels_search_kernel(ProbeParams<Model> P, uint32_t* __restrict__ out,
                         unsigned long long* __restrict__ tile_counts) {
  search_chunk<Model, MODE, CHUNK, VEC, 0, kSearchLevels>(P, out, tile_counts);
}

// The same with the GRMI lookup (Section 3.A): exponential search in the
// gapped key array from the predicted slot.
template <class Model, int MODE, int CHUNK, bool VEC>
__global__ void __launch_bounds__(kSearchBlock, LJ_SMINB)
    gapped_search_kernel(ProbeParams<Model> P, uint32_t* __restrict__ out,
                         unsigned long long* __restrict__ tile_counts) {
  search_chunk<Model, MODE, CHUNK, VEC, 1>(P, out, tile_counts);
}

// The same with the learned hash index (Section 3.C): search from the first
// slot of the probe's bucket; the entry gives the whole range of matches.
template <class Model, int MODE, int CHUNK, bool VEC>
__global__ void __launch_bounds__(kSearchBlock, LJ_SMINB)
    hash_search_kernel(ProbeParams<Model> P, uint32_t* __restrict__ out,
                       unsigned long long* __restrict__ tile_counts) {
  search_chunk<Model, MODE, CHUNK, VEC, 2>(P, out, tile_counts);
}

// The same with the RadixSpline as the hash (the paper's RSHASH-INLJ).
template <class Model, int MODE, int CHUNK, bool VEC>
__global__ void __launch_bounds__(kSearchBlock, LJ_SMINB)
    rs_hash_search_kernel(ProbeParams<Model> P, uint32_t* __restrict__ out,
                          unsigned long long* __restrict__ tile_counts) {
  search_chunk<Model, MODE, CHUNK, VEC, 3>(P, out, tile_counts);
}

// ---------------------------------------------------------------------------
// Bucketed probe order (option "probe_buckets"): the probes of each chunk of
// 2^22 are first grouped by the region of R their predicted position falls
// in (2^14 buckets per chunk), then looked up bucket by bucket, so that the
// lanes of a warp and the warps of an SM search nearby parts of R (shared
// L1/L2 lines, TLB entries and DRAM pages).  The results go back to the
// probes' own positions, so everything after the search is unchanged.
//   bucket_count_kernel    bucket sizes (warp-aggregated atomics)
//   tile_scan_kernel       bucket start positions (the scan of tile counts)
//   bucket_scatter_kernel  (key, probe index) into bucket order
//   bucketed_search_kernel lookups in bucket order, words written back to
//                          the probes' positions
//   tile_count_kernel      match count per compaction tile, from the words
constexpr int kBucketChunkLog2 = 22;
constexpr int kBucketsLog2 = 14;
constexpr uint32_t kBucketsPerChunk = 1u << kBucketsLog2;

template <class Model>
__device__ __forceinline__ uint32_t bucket_of(const ProbeParams<Model>& P, uint64_t x, uint64_t j,
                                              uint32_t shift) {
  const typename Model::Leaf lf = Model::load_leaf(P.leaves, P.model.leaf(x));
  const int64_t lo = lf.lo, hi = lf.hi;
  int64_t p = lo + Model::pred(lf, x);
  p = p < lo ? lo : (p > hi ? hi : p);   // p <= n, and n >> shift < kBucketsPerChunk
  return (uint32_t)(j >> kBucketChunkLog2) * kBucketsPerChunk + (uint32_t)((uint64_t)p >> shift);
}

// Adds 1 to ctr[key] for every active lane, one atomic per distinct key of
// the warp; returns the lane's own position among the increments.
__device__ __forceinline__ unsigned long long warp_add_one(unsigned long long* ctr, uint32_t key,
                                                           bool active) {
  const unsigned mask = __ballot_sync(0xffffffffu, active);
  if (!active) return 0;
  const unsigned grp = __match_any_sync(mask, key);
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(grp) - 1;
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(ctr + key, (unsigned long long)__popc(grp));
  base = __shfl_sync(grp, base, leader);
  return base + __popc(grp & ((1u << lane) - 1u));
}

// Bucket sizes: each probe's bucket is kept in bkey for the scatter pass;
// one reduction (no returned value) per distinct bucket of a warp.
template <class Model>
__global__ void __launch_bounds__(kSearchBlock)
    bucket_count_kernel(ProbeParams<Model> P, uint32_t shift, unsigned long long* __restrict__ ctr,
                        uint32_t* __restrict__ bkey) {
  const uint64_t j0 = ((uint64_t)blockIdx.x * kSearchBlock + threadIdx.x) * 2;
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    const uint64_t j = j0 + p;
    const bool valid = j < P.m;
    const uint64_t x = valid ? __ldg(reinterpret_cast<const unsigned long long*>(P.S) + j) : 0;
    const uint32_t key = valid ? bucket_of(P, x, j, shift) : 0u;
    const unsigned mask = __ballot_sync(0xffffffffu, valid);
    if (valid) {
      bkey[j] = key;
      const unsigned grp = __match_any_sync(mask, key);
      if ((int)(threadIdx.x & 31) == __ffs(grp) - 1)
        atomicAdd(ctr + key, (unsigned long long)__popc(grp));
    }
  }
}

// Probes into bucket order: (key, probe index) at the bucket's next free slot.
__global__ void __launch_bounds__(kSearchBlock)
    bucket_scatter_kernel(const uint64_t* __restrict__ S, uint64_t m,
                          const uint32_t* __restrict__ bkey, unsigned long long* __restrict__ cursor,
                          uint64_t* __restrict__ bx, uint32_t* __restrict__ bj) {
  const uint64_t j0 = ((uint64_t)blockIdx.x * kSearchBlock + threadIdx.x) * 2;
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    const uint64_t j = j0 + p;
    const bool valid = j < m;
    const uint32_t key = valid ? bkey[j] : 0u;
    const unsigned long long at = warp_add_one(cursor, key, valid);
    if (valid) {
      bx[at] = __ldg(reinterpret_cast<const unsigned long long*>(S) + j);
      bj[at] = (uint32_t)j;
    }
  }
}

constexpr uint32_t kSortMergeMax = 1024;   // largest bucket sorted and merged in shared memory

// LARGE_ONLY (sort-merge order): only the entries of buckets too large for
// sortmerge_kernel are looked up here; the others are skipped.
template <class Model, int MODE, bool LARGE_ONLY = false>
__global__ void __launch_bounds__(kSearchBlock, LJ_SMINB)
    bucketed_search_kernel(ProbeParams<Model> P, const uint64_t* __restrict__ bx,
                           const uint32_t* __restrict__ bj, uint32_t* __restrict__ out,
                           const uint32_t* __restrict__ bkey = nullptr,
                           const uint64_t* __restrict__ bend = nullptr) {
  const uint64_t i0 = ((uint64_t)blockIdx.x * kSearchBlock + threadIdx.x) * 2;
  uint64_t x[2];
  uint32_t j[2];
  bool valid[2];
  if (i0 + 1 < P.m) {
    const ulonglong2 v = ldg_stream_u64x2(bx + i0);
    const uint2 w = __ldg(reinterpret_cast<const uint2*>(bj + i0));
    x[0] = v.x;
    x[1] = v.y;
    j[0] = w.x;
    j[1] = w.y;
    valid[0] = valid[1] = true;
  } else {
    valid[0] = i0 < P.m;
    valid[1] = false;
    x[0] = valid[0] ? bx[i0] : 0;
    j[0] = valid[0] ? bj[i0] : 0;
    x[1] = 0;
    j[1] = 0;
  }
  if (LARGE_ONLY) {
#pragma unroll
    for (int p = 0; p < 2; ++p)
      if (valid[p]) {
        const uint32_t b = bkey[j[p]];
        const uint64_t size = bend[b] - (b ? bend[b - 1] : 0);
        valid[p] = size > kSortMergeMax;
      }
    if (__all_sync(0xffffffffu, !valid[0] && !valid[1])) return;   // warp-uniform
  }
  uint32_t r_idx[2], cnt[2];
  lookup_keys<Model, MODE, 2>(P, x, valid, r_idx, cnt);
#pragma unroll
  for (int p = 0; p < 2; ++p)
    if (valid[p]) {
      out[j[p]] = MODE == kDupCount ? cnt[p] : (cnt[p] ? r_idx[p] : kNoMatch);
      if (P.first) P.first[j[p]] = r_idx[p];
    }
}

// Learned sort-merge order (Section 4, option "probe_buckets" = 2): block b
// takes bucket b (a range of R's predicted positions within one chunk of
// probes), sorts its keys in shared memory with a bitonic network, finds the
// part of R the bucket spans from the lower bound of its smallest key to the
// upper bound of its largest, and merges: each sorted key's lower (and upper)
// bound is searched inside that part only.  Buckets larger than
// kSortMergeMax are left to bucketed_search_kernel<..., true>.
constexpr int kSortMergeBlock = 256;

template <class Model, int MODE>
__global__ void __launch_bounds__(kSortMergeBlock)
    sortmerge_kernel(ProbeParams<Model> P, const uint64_t* __restrict__ bend,
                     const uint64_t* __restrict__ bx, const uint32_t* __restrict__ bj,
                     uint32_t* __restrict__ out) {
  __shared__ uint64_t s_key[kSortMergeMax];
  __shared__ uint32_t s_idx[kSortMergeMax];
  __shared__ uint32_t s_lo, s_hi;
  const uint32_t b = blockIdx.x;
  const uint64_t start = b ? bend[b - 1] : 0;
  const uint64_t k = bend[b] - start;
  if (k == 0 || k > kSortMergeMax) return;
  uint32_t N = 2;
  while (N < k) N <<= 1;
  for (uint32_t i = threadIdx.x; i < N; i += kSortMergeBlock) {   // padding sorts last,
    s_key[i] = i < k ? bx[start + i] : ~0ull;                      // even after keys 2^64-1
    s_idx[i] = i < k ? bj[start + i] : ~0u;
  }
  __syncthreads();
  for (uint32_t size = 2; size <= N; size <<= 1) {   // bitonic sort by (key, probe), ascending
    for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
      for (uint32_t i = threadIdx.x; i < N / 2; i += kSortMergeBlock) {
        const uint32_t lo = 2 * i - (i & (stride - 1));
        const uint32_t hi = lo + stride;
        const bool up = (lo & size) == 0;
        const uint64_t a = s_key[lo], c = s_key[hi];
        const bool greater = a > c || (a == c && s_idx[lo] > s_idx[hi]);
        if (greater == up) {
          s_key[lo] = c;
          s_key[hi] = a;
          const uint32_t t = s_idx[lo];
          s_idx[lo] = s_idx[hi];
          s_idx[hi] = t;
        }
      }
      __syncthreads();
    }
  }
  if (threadIdx.x < 2) {   // the part of R the bucket spans
    const uint64_t x = threadIdx.x == 0 ? s_key[0] : s_key[k - 1];
    const typename Model::Leaf lf = Model::load_leaf(P.leaves, P.model.leaf(x));
    uint32_t wl, wh;
    window<Model>(lf, x, wl, wh);
    uint64_t xk[1] = {x};
    uint32_t base[1] = {wl}, len[1] = {wh - wl};
    uint64_t cv[1];
    if (threadIdx.x == 0) {
      search_last<1, true>(P.R, xk, base, len, cv);   // lower bound of the smallest key
      s_lo = base[0];
    } else {
      search_last<1, false>(P.R, xk, base, len, cv);  // upper bound of the largest key
      s_hi = base[0];
    }
  }
  __syncthreads();
  const uint32_t lo = s_lo, hi = s_hi;
  auto key_at = [&](uint32_t q) -> uint64_t {
    return __ldg(reinterpret_cast<const unsigned long long*>(P.R) + q);
  };
  for (uint32_t i = threadIdx.x; i < k; i += kSortMergeBlock) {
    const uint64_t x = s_key[i];
    uint32_t a = lo, len = hi - lo;   // lower bound in [lo, hi)
    while (len > 0) {
      const uint32_t half = len >> 1;
      if (key_at(a + half) < x) {
        a += half + 1;
        len -= half + 1;
      } else {
        len = half;
      }
    }
    uint32_t c = 0;
    if (MODE == kDupCount) {
      uint32_t u = a, ulen = hi - a;   // upper bound in [a, hi)
      while (ulen > 0) {
        const uint32_t half = ulen >> 1;
        if (key_at(u + half) <= x) {
          u += half + 1;
          ulen -= half + 1;
        } else {
          ulen = half;
        }
      }
      c = u - a;
    } else {
      c = (a < hi && key_at(a) == x) ? 1u : 0u;
    }
    const uint32_t j = s_idx[i];
    out[j] = MODE == kDupCount ? c : (c ? a : kNoMatch);
    if (P.first) P.first[j] = a;
  }
}

// Matches per compaction tile (`tile` words), one block per tile.
template <int MODE>
__global__ void __launch_bounds__(kBlock)
    tile_count_kernel(const uint32_t* __restrict__ words, uint64_t m,
                      unsigned long long* __restrict__ tile_counts, uint32_t tile) {
  __shared__ unsigned long long s_w[kWarps];
  const uint64_t base = (uint64_t)blockIdx.x * tile;
  unsigned long long c = 0;
#pragma unroll 4
  for (uint32_t i = threadIdx.x; i < tile; i += kBlock) {
    const uint64_t q = base + i;
    if (q < m) {
      const uint32_t w = words[q];
      c += MODE == kDupCount ? w : (w != kNoMatch ? 1u : 0u);
    }
  }
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) c += __shfl_xor_sync(0xffffffffu, c, d);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int w = 0; w < kWarps; ++w) t += s_w[w];
    tile_counts[blockIdx.x] = t;
  }
}

// Compaction kernel of the pipeline: tiles of 256 threads x 16 words
// (kCompactTile probes; 256 x 4 for small batches).  Each tile already knows its first output position
// (tile_scan_kernel), so tiles never wait for one another: load the words,
// scan them in the block, stage the output in shared memory and write it
// with coalesced stores:
//   kScanPairs     (r_idx, s_idx) pairs of the matching probes
//   kScanOffsets   offsets[j] (u64, exclusive) and optionally counts[j]
// (FROM_COUNTS: the word is a match count; else a position or kNoMatch).
struct ScanParams {
  const uint32_t* in;
  uint64_t m;
  uint32_t s_base;
  lj_pair* pairs;
  uint64_t capacity;
  uint64_t* offsets;
  uint32_t* counts;       // kScanOffsets from matches: optional 0/1 counts
  const uint64_t* tile_prefix;
  // direct prefixes (small batches, no tile_scan_kernel): each tile sums the
  // counts of the tiles before it; the last tile publishes the total
  const unsigned long long* tile_counts;   // non-null: direct mode
  uint32_t tiles;
  uint64_t* total_ws;
  uint64_t* total_out;    // optional
  uint64_t* offsets_end;  // optional: offsets[m]
  uint32_t* err;
};

// Batches of at most this many compaction tiles take the direct prefixes.
constexpr uint32_t kDirectPrefixTiles = 1024;

template <int MODE, bool FROM_COUNTS, bool VEC, int ITEMS>
__global__ void __launch_bounds__(kBlock) compact_kernel(ScanParams P) {
  constexpr uint64_t kTile = (uint64_t)kBlock * ITEMS;
  __shared__ uint64_t s_warp[kWarps];
  __shared__ uint64_t s_stage[kTile];   // 32 KB for tiles of 4096
  __shared__ uint64_t s_count;
  const uint32_t tile = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t tile_base = (uint64_t)tile * kTile;
  const uint64_t base = tile_base + (uint64_t)threadIdx.x * ITEMS;
  uint64_t prefix;
  if (P.tile_counts) {
    __shared__ unsigned long long s_red[kWarps];
    unsigned long long part = 0;
    for (uint32_t u = threadIdx.x; u < tile; u += kBlock) part += __ldg(P.tile_counts + u);
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) part += __shfl_xor_sync(0xffffffffu, part, d);
    if (lane == 0) s_red[warp] = part;
    __syncthreads();
    prefix = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) prefix += s_red[w];
    if (tile + 1 == P.tiles && threadIdx.x == 0) {
      const uint64_t total = prefix + __ldg(P.tile_counts + tile);
      *P.total_ws = total;
      if (P.total_out) *P.total_out = total;
      if (P.offsets_end) *P.offsets_end = total;
      if (MODE == kScanPairs && total > P.capacity) atomicOr(P.err, kErrCapacity);
    }
  } else {
    prefix = P.tile_prefix[tile];
  }
  uint32_t v[ITEMS];
  if (VEC && base + ITEMS <= P.m) {
#pragma unroll
    for (int q = 0; q < ITEMS / 4; ++q) {
      const uint4 u = ldg_stream_u32x4(P.in + base + 4 * q);
      v[4 * q] = u.x;
      v[4 * q + 1] = u.y;
      v[4 * q + 2] = u.z;
      v[4 * q + 3] = u.w;
    }
  } else {
#pragma unroll
    for (int i = 0; i < ITEMS; ++i)
      v[i] = base + i < P.m ? __ldg(P.in + base + i) : (FROM_COUNTS ? 0u : kNoMatch);
  }
  uint64_t sum = 0;
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) sum += FROM_COUNTS ? v[i] : (v[i] != kNoMatch ? 1u : 0u);
  const uint64_t inc = warp_inclusive_sum(sum, lane);
  if (lane == 31) s_warp[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    const uint64_t x = lane < kWarps ? s_warp[lane] : 0;
    const uint64_t xi = warp_inclusive_sum(x, lane);
    if (lane < kWarps) s_warp[lane] = xi - x;
  }
  __syncthreads();
  uint64_t local = s_warp[warp] + inc - sum;   // tile offset of this thread's first item
  if (MODE == kScanPairs) {
#pragma unroll
    for (int i = 0; i < ITEMS; ++i)
      if (v[i] != kNoMatch) {
        s_stage[local] = (uint64_t)v[i] | ((uint64_t)(uint32_t)(base + i + P.s_base) << 32);
        ++local;
      }
    if (threadIdx.x == kBlock - 1) s_count = local;   // the tile's number of pairs
    __syncthreads();
    const uint64_t cnt = s_count;
    uint64_t* out = reinterpret_cast<uint64_t*>(P.pairs);
    for (uint64_t q = threadIdx.x; q < cnt; q += kBlock) {
      const uint64_t o = prefix + q;
      if (o < P.capacity) st_stream_u64(out + o, s_stage[q]);
    }
  } else {
    const uint32_t first = threadIdx.x * ITEMS;
    if (P.offsets) {
#pragma unroll
      for (int i = 0; i < ITEMS; ++i) {
        s_stage[first + i] = prefix + local;
        local += FROM_COUNTS ? v[i] : (v[i] != kNoMatch ? 1u : 0u);
      }
    }
    if (!FROM_COUNTS && P.counts && base < P.m) {
      if (VEC && base + ITEMS <= P.m) {
#pragma unroll
        for (int q = 0; q < ITEMS / 4; ++q)
          reinterpret_cast<uint4*>(P.counts + base)[q] =
              make_uint4(v[4 * q] != kNoMatch, v[4 * q + 1] != kNoMatch, v[4 * q + 2] != kNoMatch,
                         v[4 * q + 3] != kNoMatch);
      } else {
        for (int i = 0; i < ITEMS; ++i)
          if (base + i < P.m) P.counts[base + i] = v[i] != kNoMatch;
      }
    }
    if (P.offsets) {
      __syncthreads();
      const uint64_t len = P.m - tile_base < kTile ? P.m - tile_base : kTile;
      for (uint64_t q = threadIdx.x; q < len; q += kBlock) P.offsets[tile_base + q] = s_stage[q];
    }
  }
}

struct Workspace {
  void* mem = nullptr;
  TileState st{};
  uint64_t* total = nullptr;
  uint32_t* words = nullptr;   // one 32-bit word per probe (search output)
  uint32_t tiles = 0;
};

// Scratch: header (ticket, total) + tile states for `tiles` tiles + optional
// per-probe words.  The header and the flags are zeroed on the stream.
int ws_acquire(Workspace& w, uint32_t tiles, uint64_t words, cudaStream_t s) {
  w.tiles = std::max<uint32_t>(1, tiles);
  const size_t flags = ((size_t)w.tiles * 4 + 255) / 256 * 256;
  const size_t states = ((size_t)w.tiles * 16 + 255) / 256 * 256;
  const size_t bytes = 256 + flags + states + words * 4;
  LJ_CUDA(scratch_alloc(&w.mem, bytes, s));
  char* b = (char*)w.mem;
  LJ_CUDA(cudaMemsetAsync(b, 0, 256 + flags, s));
  w.st.ticket = (uint32_t*)b;
  w.total = (uint64_t*)(b + 64);
  w.st.flag = (uint32_t*)(b + 256);
  w.st.agg = (uint64_t*)(b + 256 + flags);
  w.st.incl = w.st.agg + w.tiles;
  w.st.polls = lookback_polls();
  w.words = words ? (uint32_t*)(b + 256 + flags + states) : nullptr;
  return 0;
}

// Parameters of a probe launch; err = the word its kernels OR errors into
// (the per-device error word unless the caller passes another).
template <class Model>
ProbeParams<Model> make_params(const lj_index* idx, Model model, const uint64_t* S, uint64_t m,
                               uint32_t s_base, uint32_t* err) {
  ProbeParams<Model> P{};
  P.R = idx->R;
  P.n = (uint32_t)idx->n;
  P.r32 = (reinterpret_cast<uintptr_t>(idx->R) & 31) == 0;
  P.leaves = (const typename Model::Leaf*)idx->leaves;
  P.model = model;
  P.S = S;
  P.m = m;
  P.s_base = s_base;
  P.err = err;
  P.gkeys = idx->gkeys;
  P.gpos = idx->gpos;
  P.gslots = idx->gslots;
  P.gscale = idx->gscale;
  P.dfirst = idx->dfirst;
  P.hrange = idx->hrange;
  P.ndistinct = (uint32_t)idx->ndistinct;
  P.hB = idx->hbuckets;
  P.hn1 = idx->n + 1;
  P.rs = RsDev{idx->rs_x, idx->rs_y, idx->rs_rcp, idx->rs_table, idx->rs_kmin, idx->rs_kmax,
               idx->n, idx->rs_S, idx->rs_shift};
  P.levels = idx->use_levels ? idx->levels : nullptr;
  P.nlev = idx->nlev;
  for (int k = 0; k <= kMaxLevels; ++k) P.lev_off[k] = idx->lev_off[k];
  return P;
}

inline bool aligned(const void* p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

// Single-pass path: one kernel does lookup + scan + write.
template <class Model>
int launch_single_pass(const lj_index* idx, Model model, int mode, const uint64_t* S, uint64_t m,
                       lj_pair* pairs, uint64_t cap, uint32_t* counts, uint64_t* offsets,
                       uint32_t* first, uint64_t* total_dev, uint64_t* total_host,
                       uint32_t s_base, cudaStream_t s) {
  constexpr uint64_t tile = (uint64_t)kBlock * 2 * kRounds;
  Workspace w;
  if (int rc = ws_acquire(w, (uint32_t)((m + tile - 1) / tile), 0, s)) return rc;
  ProbeParams<Model> P = make_params(idx, model, S, m, s_base, device_error_word(idx->device));
  if (!P.err) return fail(LJ_E_NOMEM, "cannot allocate the device error word");
  P.pairs = pairs;
  P.capacity = cap;
  P.counts = counts;
  P.offsets = offsets;
  P.first = first;
  P.total_out = total_dev;
  P.total_ws = w.total;
  P.st = w.st;
  P.num_tiles = w.tiles;
  P.tile_skip = std::min(fault_skip_tiles(), w.tiles - 1);
  const unsigned grid = w.tiles - P.tile_skip;
  const bool vec = aligned(S, 16) && (!offsets || aligned(offsets, 16)) &&
                   (!counts || aligned(counts, 8)) && (!first || aligned(first, 8));
  KernelTimer kt("probe_single_pass_kernel", s);
#define LJ_LAUNCH(MODE)                                                                  \
  (vec ? probe_single_pass_kernel<Model, MODE, kRounds, true><<<grid, kBlock, 0, s>>>(P) \
       : probe_single_pass_kernel<Model, MODE, kRounds, false><<<grid, kBlock, 0, s>>>(P))
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

// Search step of the pipeline in bucketed probe order: bucket sizes, bucket
// starts, scatter into bucket order, lookups, per-tile match counts.
template <class Model>
int launch_bucketed(const lj_index* idx, const ProbeParams<Model>& P, bool dup, uint32_t* words,
                    unsigned long long* tile_counts, uint32_t tiles, bool sortmerge,
                    cudaStream_t s) {
  const uint64_t m = P.m;
  const uint64_t chunks = (m + (1ull << kBucketChunkLog2) - 1) >> kBucketChunkLog2;
  const uint64_t nb = chunks * kBucketsPerChunk;
  uint32_t shift = 0;
  while ((idx->n >> shift) >= kBucketsPerChunk) ++shift;
  const uint32_t sb = (uint32_t)((nb + kTileScanSpan - 1) / kTileScanSpan);
  const size_t b_ctr = (nb * 8 + 255) / 256 * 256;
  const size_t b_flags = ((size_t)sb * 4 + 255) / 256 * 256;
  const size_t b_states = ((size_t)sb * 16 + 255) / 256 * 256;
  const size_t b_cur = ((nb + 1) * 8 + 255) / 256 * 256;
  const size_t b_x = (m * 8 + 255) / 256 * 256;
  const size_t b_j = (m * 4 + 255) / 256 * 256;
  char* ws = nullptr;
  LJ_CUDA(scratch_alloc((void**)&ws, 256 + b_ctr + b_flags + b_states + b_cur + b_x + 2 * b_j, s));
  LJ_CUDA(cudaMemsetAsync(ws, 0, 256 + b_ctr + b_flags, s));
  unsigned long long* ctr = (unsigned long long*)(ws + 256);
  TileState st;
  st.ticket = (uint32_t*)ws;
  st.flag = (uint32_t*)(ws + 256 + b_ctr);
  st.agg = (uint64_t*)(ws + 256 + b_ctr + b_flags);
  st.incl = st.agg + sb;
  st.polls = lookback_polls();
  uint64_t* cursor = (uint64_t*)(ws + 256 + b_ctr + b_flags + b_states);
  uint64_t* bx = (uint64_t*)(ws + 256 + b_ctr + b_flags + b_states + b_cur);
  uint32_t* bj = (uint32_t*)(ws + 256 + b_ctr + b_flags + b_states + b_cur + b_x);
  uint32_t* bkey = (uint32_t*)(ws + 256 + b_ctr + b_flags + b_states + b_cur + b_x + b_j);
  const unsigned grid = (unsigned)((m + 2 * kSearchBlock - 1) / (2 * kSearchBlock));
  {
    KernelTimer kt("bucket_count_kernel", s);
    bucket_count_kernel<Model><<<grid, kSearchBlock, 0, s>>>(P, shift, ctr, bkey);
  }
  {
    KernelTimer kt("bucket_scan_kernel", s);
    tile_scan_kernel<<<sb, kBlock, 0, s>>>(ctr, (uint32_t)nb, cursor, st, sb, (uint64_t*)(ws + 64),
                                           nullptr, nullptr, ~0ull, P.err);
  }
  {
    KernelTimer kt("bucket_scatter_kernel", s);
    bucket_scatter_kernel<<<grid, kSearchBlock, 0, s>>>(P.S, m, bkey, (unsigned long long*)cursor,
                                                         bx, bj);
  }
  if (sortmerge) {
    {
      KernelTimer kt("sortmerge_kernel", s);
      if (dup)
        sortmerge_kernel<Model, kDupCount>
            <<<(unsigned)nb, kSortMergeBlock, 0, s>>>(P, cursor, bx, bj, words);
      else
        sortmerge_kernel<Model, kUniqueCount>
            <<<(unsigned)nb, kSortMergeBlock, 0, s>>>(P, cursor, bx, bj, words);
    }
    KernelTimer kt("bucketed_search_kernel", s);   // buckets too large to sort in shared memory
    if (dup)
      bucketed_search_kernel<Model, kDupCount, true>
          <<<grid, kSearchBlock, 0, s>>>(P, bx, bj, words, bkey, cursor);
    else
      bucketed_search_kernel<Model, kUniqueCount, true>
          <<<grid, kSearchBlock, 0, s>>>(P, bx, bj, words, bkey, cursor);
  } else {
    KernelTimer kt("bucketed_search_kernel", s);
    if (dup)
      bucketed_search_kernel<Model, kDupCount><<<grid, kSearchBlock, 0, s>>>(P, bx, bj, words);
    else
      bucketed_search_kernel<Model, kUniqueCount><<<grid, kSearchBlock, 0, s>>>(P, bx, bj, words);
  }
  {
    KernelTimer kt("tile_count_kernel", s);
    if (dup)
      tile_count_kernel<kDupCount><<<tiles, kBlock, 0, s>>>(words, m, tile_counts, 1u << P.tile_shift);
    else
      tile_count_kernel<kUniqueCount><<<tiles, kBlock, 0, s>>>(words, m, tile_counts, 1u << P.tile_shift);
  }
  LJ_CUDA(cudaGetLastError());
  LJ_CUDA(scratch_free(ws, s));
  return 0;
}

// Fused path (join_emit, unique R, m <= fused_max): one cooperative launch
// of probe_fused_kernel over at most as many blocks as can be resident.
template <class Model, bool VEC, int SEARCH>
int launch_fused_as(const lj_index* idx, ProbeParams<Model> P, uint64_t* total_host,
                    cudaStream_t s) {
  const uint64_t m = P.m;
  static std::atomic<int> per_sm_cache{0};
  int per_sm = per_sm_cache.load();
  if (per_sm == 0) {
    LJ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, probe_fused_kernel<Model, VEC, SEARCH>, kFusedBlock, kFusedMaxPerBlock * 4));
    if (per_sm <= 0) return fail(LJ_E_CUDA, "probe_fused_kernel: no resident block fits an SM");
    per_sm_cache = per_sm;
  }
  int sms = 0;
  LJ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, idx->device));
  const uint64_t cap_blocks = (uint64_t)per_sm * (uint64_t)sms;
  uint64_t grid = std::min<uint64_t>(cap_blocks, (m + 2 * kFusedBlock - 1) / (2 * kFusedBlock));
  // probes per block: even (pairs of keys are read with one 16-byte load)
  uint32_t per_block = (uint32_t)(((m + grid - 1) / grid + 1) & ~1ull);
  if (per_block > kFusedMaxPerBlock) return 1;   // more than the resident blocks hold: the pipeline
  grid = (m + per_block - 1) / per_block;   // no empty block
  // scratch: barrier counter | total | group sums (zeroed) | block counts
  const size_t b_gsum = ((grid / kFusedGroup + 1) * 8 + 255) / 256 * 256;
  const size_t b_cnt = (grid * 4 + 255) / 256 * 256;
  char* ws = nullptr;
  LJ_CUDA(scratch_alloc((void**)&ws, 256 + b_gsum + b_cnt, s));
  LJ_CUDA(cudaMemsetAsync(ws, 0, 256 + b_gsum, s));
  FusedState F;
  F.arrive = (uint32_t*)ws;
  F.gsum = (unsigned long long*)(ws + 256);
  F.bcount = (uint32_t*)(ws + 256 + b_gsum);
  F.polls = lookback_polls();
  P.total_ws = (uint64_t*)(ws + 64);
  P.tile_skip = std::min<uint32_t>(fault_skip_tiles(), (uint32_t)grid - 1);
  void* args[] = {&P, &F, &per_block};
  cudaError_t e;
  {
    KernelTimer kt("probe_fused_kernel", s);
    e = cudaLaunchCooperativeKernel((const void*)probe_fused_kernel<Model, VEC, SEARCH>,
                                    dim3((unsigned)grid), dim3(kFusedBlock), args,
                                    (size_t)per_block * 4, s);
  }
  if (e != cudaSuccess) {
    scratch_free(ws, s);
    return fail_cuda(e, "probe_fused_kernel: cooperative launch");
  }
  if (total_host) LJ_CUDA(cudaMemcpyAsync(total_host, P.total_ws, 8, cudaMemcpyDeviceToHost, s));
  LJ_CUDA(scratch_free(ws, s));
  if (total_host) {
    LJ_CUDA(cudaStreamSynchronize(s));
    if (int r2 = take_device_errors(idx->device, s)) return r2;
  }
  return 0;
}

template <class Model>
int launch_fused(const lj_index* idx, Model model, const uint64_t* S, uint64_t m, lj_pair* pairs,
                 uint64_t cap, uint64_t* total_dev, uint64_t* total_host, uint32_t s_base,
                 cudaStream_t s) {
  ProbeParams<Model> P = make_params(idx, model, S, m, s_base, device_error_word(idx->device));
  if (!P.err) return fail(LJ_E_NOMEM, "cannot allocate the device error word");
  P.pairs = pairs;
  P.capacity = cap;
  P.total_out = total_dev;
  const bool vec = aligned(S, 16);
  if (P.levels)
    return vec ? launch_fused_as<Model, true, kSearchLevels>(idx, P, total_host, s)
               : launch_fused_as<Model, false, kSearchLevels>(idx, P, total_host, s);
  if (g_fused_groups.load() != 0)
    return vec ? launch_fused_as<Model, true, kSearchGroups>(idx, P, total_host, s)
               : launch_fused_as<Model, false, kSearchGroups>(idx, P, total_host, s);
  return vec ? launch_fused_as<Model, true, kSearchHalve>(idx, P, total_host, s)
             : launch_fused_as<Model, false, kSearchHalve>(idx, P, total_host, s);
}

// Count-scan-emit path: search kernel (per-probe words + per-tile counts)
// -> tile_scan_kernel (tile prefixes, total) -> compact_kernel.
template <class Model>
int launch_pipeline(const lj_index* idx, Model model, int mode, const uint64_t* S, uint64_t m,
                    lj_pair* pairs, uint64_t cap, uint32_t* counts, uint64_t* offsets,
                    uint32_t* first, uint64_t* total_dev, uint64_t* total_host, uint32_t s_base,
                    cudaStream_t s) {
  const bool dup = mode == kDupCount;
  // duplicates: the search writes counts, into the caller's buffer if given
  const bool words_in_counts = dup && counts && aligned(counts, 16);
  // small batches: tiles of 1024 probes (more blocks for the compaction)
  const bool small = m <= kSmallBatch;
  const uint32_t tile_shift = small ? 10 : 12;
  static_assert(kCompactTile == 4096 && 256 * kSmallScanItems == 1024, "tile sizes");
  const uint32_t tiles = (uint32_t)std::max<uint64_t>(1, (m + (1ull << tile_shift) - 1) >> tile_shift);
  const size_t b_cnt = ((size_t)tiles * 8 + 255) / 256 * 256;
  const size_t b_pre = ((size_t)(tiles + 1) * 8 + 255) / 256 * 256;
  const size_t b_words = words_in_counts ? 0 : ((m + 3) & ~3ull) * 4;
  const uint32_t scan_blocks = (tiles + kTileScanSpan - 1) / kTileScanSpan;
  const size_t b_flags = ((size_t)scan_blocks * 4 + 255) / 256 * 256;
  const size_t b_states = ((size_t)scan_blocks * 16 + 255) / 256 * 256;
  // layout: header | tile counts | scan flags | (zeroed so far) scan states |
  //         tile prefixes | words
  char* ws = nullptr;
  LJ_CUDA(scratch_alloc((void**)&ws, 256 + b_cnt + b_flags + b_states + b_pre + b_words, s));
  LJ_CUDA(cudaMemsetAsync(ws, 0, 256 + b_cnt + b_flags, s));
  uint64_t* total_ws = (uint64_t*)(ws + 64);
  unsigned long long* tile_counts = (unsigned long long*)(ws + 256);
  TileState st;
  st.ticket = (uint32_t*)(ws + 128);
  st.flag = (uint32_t*)(ws + 256 + b_cnt);
  st.agg = (uint64_t*)(ws + 256 + b_cnt + b_flags);
  st.incl = st.agg + scan_blocks;
  st.polls = lookback_polls();
  uint64_t* tile_prefix = (uint64_t*)(ws + 256 + b_cnt + b_flags + b_states);
  uint32_t* words = words_in_counts ? counts : (uint32_t*)(ws + 256 + b_cnt + b_flags + b_states + b_pre);

  ProbeParams<Model> P = make_params(idx, model, S, m, s_base, device_error_word(idx->device));
  if (!P.err) return fail(LJ_E_NOMEM, "cannot allocate the device error word");
  P.first = first;
  P.tile_shift = tile_shift;
  const bool vec = aligned(S, 16) && (!first || aligned(first, 8));
  constexpr uint64_t kChunkProbes = 2ull * kSearchBlock * kSearchChunk;
  const unsigned grid = (unsigned)std::max<uint64_t>(1, (m + kChunkProbes - 1) / kChunkProbes);
  const int order = idx->probe_order >= 0 ? idx->probe_order : g_probe_buckets.load();
  if (order != 0 && !P.gkeys) {
    if (int rc = launch_bucketed(idx, P, dup, words, tile_counts, tiles, order == 2, s)) {
      scratch_free(ws, s);
      return rc;
    }
  } else {
    KernelTimer kt(!P.gkeys                  ? (P.levels ? "levels_search_kernel" : "probe_search_kernel")
                   : idx->gkind == kRmiHash ? "hash_search_kernel"
                   : idx->gkind == kRsHash  ? "rs_hash_search_kernel"
                                            : "gapped_search_kernel", s);
#define LJ_SEARCH(KERNEL, MODE)                                                              \
  (vec ? KERNEL<Model, MODE, kSearchChunk, true><<<grid, kSearchBlock, 0, s>>>(P, words, tile_counts) \
       : KERNEL<Model, MODE, kSearchChunk, false><<<grid, kSearchBlock, 0, s>>>(P, words, tile_counts))
    if (P.gkeys && idx->gkind == kRmiHash) {
      if (dup)
        LJ_SEARCH(hash_search_kernel, kDupCount);
      else
        LJ_SEARCH(hash_search_kernel, kUniqueCount);
    } else if (P.gkeys && idx->gkind == kRsHash) {
      if (dup)
        LJ_SEARCH(rs_hash_search_kernel, kDupCount);
      else
        LJ_SEARCH(rs_hash_search_kernel, kUniqueCount);
    } else if (P.gkeys) {
      if (dup)
        LJ_SEARCH(gapped_search_kernel, kDupCount);
      else
        LJ_SEARCH(gapped_search_kernel, kUniqueCount);
    } else if (P.levels) {
      if (dup)
        LJ_SEARCH(levels_search_kernel, kDupCount);
      else
        LJ_SEARCH(levels_search_kernel, kUniqueCount);
    } else {
      if (dup)
        LJ_SEARCH(probe_search_kernel, kDupCount);
      else
        LJ_SEARCH(probe_search_kernel, kUniqueCount);
    }
#undef LJ_SEARCH
  }
  LJ_CUDA(cudaGetLastError());
  const bool need_compact = mode == kUniqueEmit || offsets || (!dup && counts);
  // small batches: the compaction tiles sum their predecessors' counts
  // themselves (one launch less); larger ones scan the tile counts first
  const bool direct = need_compact && tiles <= kDirectPrefixTiles;
  if (!direct) {
    KernelTimer kt("tile_scan_kernel", s);
    tile_scan_kernel<<<scan_blocks, kBlock, 0, s>>>(tile_counts, tiles, tile_prefix, st,
                                                   scan_blocks, total_ws, total_dev,
                                                   offsets ? offsets + m : nullptr,
                                                   mode == kUniqueEmit ? cap : ~0ull, P.err);
  }
  LJ_CUDA(cudaGetLastError());

  ScanParams Q{};
  if (direct) {
    Q.tile_counts = tile_counts;
    Q.tiles = tiles;
    Q.total_ws = total_ws;
    Q.total_out = total_dev;
    Q.offsets_end = offsets ? offsets + m : nullptr;
    Q.err = P.err;
  }
  Q.in = words;
  Q.m = m;
  Q.s_base = s_base;
  Q.pairs = pairs;
  Q.capacity = cap;
  Q.offsets = offsets;
  Q.counts = dup ? nullptr : counts;
  Q.tile_prefix = tile_prefix;
  const bool qvec = aligned(words, 16) && (!Q.counts || aligned(Q.counts, 16));
  if (need_compact) {
    KernelTimer kt("compact_kernel", s);
#define LJ_COMPACT(ITEMS)                                                                  \
  do {                                                                                     \
    if (mode == kUniqueEmit)                                                               \
      qvec ? compact_kernel<kScanPairs, false, true, ITEMS><<<tiles, kBlock, 0, s>>>(Q)    \
           : compact_kernel<kScanPairs, false, false, ITEMS><<<tiles, kBlock, 0, s>>>(Q);  \
    else if (dup)                                                                          \
      qvec ? compact_kernel<kScanOffsets, true, true, ITEMS><<<tiles, kBlock, 0, s>>>(Q)   \
           : compact_kernel<kScanOffsets, true, false, ITEMS><<<tiles, kBlock, 0, s>>>(Q); \
    else                                                                                   \
      qvec ? compact_kernel<kScanOffsets, false, true, ITEMS><<<tiles, kBlock, 0, s>>>(Q)  \
           : compact_kernel<kScanOffsets, false, false, ITEMS><<<tiles, kBlock, 0, s>>>(Q); \
  } while (0)
    if (small)
      LJ_COMPACT(kSmallScanItems);
    else
      LJ_COMPACT(kScanItems);
#undef LJ_COMPACT
  }
  LJ_CUDA(cudaGetLastError());
  if (dup && counts && !words_in_counts)
    LJ_CUDA(cudaMemcpyAsync(counts, words, m * 4, cudaMemcpyDeviceToDevice, s));
  if (total_host) LJ_CUDA(cudaMemcpyAsync(total_host, total_ws, 8, cudaMemcpyDeviceToHost, s));
  LJ_CUDA(scratch_free(ws, s));
  if (total_host) {
    LJ_CUDA(cudaStreamSynchronize(s));
    if (int rc = take_device_errors(idx->device, s)) return rc;
  }
  return 0;
}

template <class Model>
int launch_probe(const lj_index* idx, Model model, int mode, const uint64_t* S, uint64_t m,
                 lj_pair* pairs, uint64_t cap, uint32_t* counts, uint64_t* offsets,
                 uint32_t* first, uint64_t* total_dev, uint64_t* total_host, uint32_t s_base,
                 cudaStream_t s) {
  if (m <= g_single_pass_max.load() && !idx->gkeys)   // the GRMI lookup runs in the pipeline only
    return launch_single_pass(idx, model, mode, S, m, pairs, cap, counts, offsets, first,
                              total_dev, total_host, s_base, s);
  const int order = idx->probe_order >= 0 ? idx->probe_order : g_probe_buckets.load();
  if (mode == kUniqueEmit && m <= g_fused_max.load() && !idx->gkeys && order == 0) {
    const int rc = launch_fused(idx, model, S, m, pairs, cap, total_dev, total_host, s_base, s);
    if (rc <= 0) return rc;   // rc > 0: the batch does not fit the resident blocks
  }
  return launch_pipeline(idx, model, mode, S, m, pairs, cap, counts, offsets, first, total_dev,
                         total_host, s_base, s);
}

template <class Model>
int launch_emit(const lj_index* idx, Model model, const uint64_t* S, uint64_t m,
                const uint64_t* offsets, lj_pair* pairs, uint64_t cap, uint32_t s_base,
                cudaStream_t s) {
  ProbeParams<Model> P = make_params(idx, model, S, m, s_base, device_error_word(idx->device));
  if (!P.err) return fail(LJ_E_NOMEM, "cannot allocate the device error word");
  P.pairs = pairs;
  P.capacity = cap;
  P.offsets = const_cast<uint64_t*>(offsets);
  const uint64_t blocks = (m + kBlock - 1) / kBlock;
  {
    KernelTimer kt("emit_kernel", s);
    if (P.gkeys && idx->gkind == kRsHash)
      emit_kernel<Model, 3><<<(unsigned)blocks, kBlock, 0, s>>>(P);
    else if (P.gkeys && idx->gkind == kRmiHash)
      emit_kernel<Model, 2><<<(unsigned)blocks, kBlock, 0, s>>>(P);
    else if (P.gkeys)
      emit_kernel<Model, 1><<<(unsigned)blocks, kBlock, 0, s>>>(P);
    else
      emit_kernel<Model, 0><<<(unsigned)blocks, kBlock, 0, s>>>(P);
  }
  LJ_CUDA(cudaGetLastError());
  return 0;
}

ModelF32 f32_model(const lj_index* idx) {
  return ModelF32::make(idx->root_f32[0], idx->root_f32[1], idx->L);
}
ModelF64 f64_model(const lj_index* idx) {
  return ModelF64::make(idx->root_f64[0], idx->root_f64[1], idx->L);
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

// Shared with the chunked host join.
int probe_count_impl(const lj_index* idx, const uint64_t* S, uint64_t m, uint32_t* counts,
                     uint64_t* offsets, uint32_t* first, uint64_t* total_dev, uint64_t* total_host,
                     cudaStream_t s) {
  const int mode = idx->unique ? kUniqueCount : kDupCount;
  if (idx->precision == LJ_FP64)
    return launch_probe(idx, f64_model(idx), mode, S, m, nullptr, 0, counts, offsets, first,
                        total_dev, total_host, 0, s);
  return launch_probe(idx, f32_model(idx), mode, S, m, nullptr, 0, counts, offsets, first,
                      total_dev, total_host, 0, s);
}

int probe_emit_impl(const lj_index* idx, const uint64_t* S, uint64_t m, const uint64_t* offsets,
                    lj_pair* pairs, uint64_t cap, uint64_t* total_dev, uint64_t* total_host,
                    uint32_t s_base, cudaStream_t s) {
  if (!offsets) {
    if (idx->precision == LJ_FP64)
      return launch_probe(idx, f64_model(idx), kUniqueEmit, S, m, pairs, cap, nullptr, nullptr,
                          nullptr, total_dev, total_host, s_base, s);
    return launch_probe(idx, f32_model(idx), kUniqueEmit, S, m, pairs, cap, nullptr, nullptr,
                        nullptr, total_dev, total_host, s_base, s);
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

// Pairs of located ranges (join_expand, and join_host with duplicates).
int probe_expand_impl(const uint32_t* first, const uint64_t* offsets, uint64_t m, lj_pair* pairs,
                      uint64_t cap, uint32_t s_base, cudaStream_t s) {
  uint32_t* err = device_error_word(current_device());
  if (!err) return fail(LJ_E_NOMEM, "cannot allocate the device error word");
  const uint64_t blocks = (m + kBlock - 1) / kBlock;
  {
    KernelTimer kt("expand_kernel", s);
    expand_kernel<<<(unsigned)blocks, kBlock, 0, s>>>(first, offsets, m, pairs, cap, s_base, err);
  }
  LJ_CUDA(cudaGetLastError());
  return 0;
}

void set_probe_buckets(int v) { g_probe_buckets = v; }
int get_probe_buckets() { return g_probe_buckets; }
void set_fused_max(uint64_t v) { g_fused_max = v; }
uint64_t get_fused_max() { return g_fused_max; }
void set_fused_groups(int v) { g_fused_groups = v; }
int get_fused_groups() { return g_fused_groups; }
void set_single_pass_max(uint64_t v) { g_single_pass_max = v; }
uint64_t get_single_pass_max() { return g_single_pass_max; }

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
  return probe_count_impl(idx, S_dev, m, counts_dev, offsets_dev, nullptr, nullptr, total_host, s);
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

extern "C" int join_locate(const lj_index* idx, const uint64_t* S_dev, uint64_t m,
                           uint32_t* first_dev, uint32_t* counts_dev, uint64_t* offsets_dev,
                           uint64_t* total_host, lj_stream_t stream) {
  using namespace lj;
  if (int rc = check_common(idx, S_dev, m, "join_locate")) return rc;
  if (m > 0 && !first_dev) return fail(LJ_E_INVAL, "join_locate: first is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  if (m == 0) {
    if (offsets_dev) LJ_CUDA(cudaMemsetAsync(offsets_dev, 0, 8, s));
    if (total_host) {
      *total_host = 0;
      LJ_CUDA(cudaStreamSynchronize(s));
    }
    return LJ_OK;
  }
  return probe_count_impl(idx, S_dev, m, counts_dev, offsets_dev, first_dev, nullptr, total_host,
                          s);
}

extern "C" int join_expand(const uint32_t* first_dev, const uint64_t* offsets_dev, uint64_t m,
                           lj_pair* pairs_dev, uint64_t capacity, uint64_t* written_dev,
                           uint64_t* written_host, lj_stream_t stream) {
  using namespace lj;
  if (m >= (1ull << 32)) return fail(LJ_E_INVAL, "join_expand: m must be below 2^32");
  if (!offsets_dev) return fail(LJ_E_INVAL, "join_expand: offsets is NULL");
  if (m > 0 && !first_dev) return fail(LJ_E_INVAL, "join_expand: first is NULL");
  if (capacity > 0 && !pairs_dev) return fail(LJ_E_INVAL, "join_expand: pairs is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  if (m > 0)
    if (int rc = probe_expand_impl(first_dev, offsets_dev, m, pairs_dev, capacity, 0, s)) return rc;
  if (written_dev) LJ_CUDA(cudaMemcpyAsync(written_dev, offsets_dev + m, 8, cudaMemcpyDeviceToDevice, s));
  if (written_host) {
    LJ_CUDA(cudaMemcpyAsync(written_host, offsets_dev + m, 8, cudaMemcpyDeviceToHost, s));
    LJ_CUDA(cudaStreamSynchronize(s));
    if (int rc = take_device_errors(current_device(), s)) return rc;
    if (*written_host > capacity)
      return fail(LJ_E_CAPACITY, "join_expand: %llu pairs do not fit the capacity of %llu",
                  (unsigned long long)*written_host, (unsigned long long)capacity);
  }
  return LJ_OK;
}

// ---------------------------------------------------------------------------
// join_count_noalloc: join_count for callers that must not allocate.
//
// The single-pass count kernel needs scratch memory for its tile states (a
// ticket, one flag and two 64-bit values per tile, the total and an error
// word).  Here that scratch is one file-scope device array of fixed size, so
// the call allocates nothing: no cudaMalloc / cudaFree, no memory pool, no
// library allocator.  Its size fixes the largest batch: kNoAllocMaxProbes.
// Every call on a device shares the array and leaves its last contents in
// it; the ticket, the flags and the error word are cleared at the start of
// each call, on the caller's stream.
namespace lj {
namespace {
constexpr uint64_t kNoAllocMaxProbes = 1ull << 25;   // 33,554,432 probes per call
constexpr uint64_t kNoAllocTile = (uint64_t)kBlock * 2 * kRounds;
constexpr uint32_t kNoAllocTiles = (uint32_t)((kNoAllocMaxProbes + kNoAllocTile - 1) / kNoAllocTile);
constexpr size_t kNoAllocFlagBytes = ((size_t)kNoAllocTiles * 4 + 255) / 256 * 256;
constexpr size_t kNoAllocBytes = 256 + kNoAllocFlagBytes + (size_t)kNoAllocTiles * 16;

// header: [0] ticket (u32), [64] total (u64), [128] error word (u32,
// sticky: an asynchronous call's error stays until a synchronising call
// reports and clears it); then the tile flags, then the aggregates and the
// inclusive prefixes.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[64] = {};

// Device address of the array on the current device.  The host-side name of
// a __device__ variable is not a device address, so it is looked up once per
// device with cudaGetSymbolAddress while that device is current.
int noalloc_scratch(int dev, unsigned char** out) {
  if (dev < 0 || dev >= 64) return fail(LJ_E_INVAL, "join_count_noalloc: device %d unsupported", dev);
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return fail_cuda(e, "join_count_noalloc: cudaGetSymbolAddress");
    g_noalloc_ptr[dev] = p;
  }
  *out = (unsigned char*)g_noalloc_ptr[dev];
  return 0;
}

template <class Model>
int noalloc_count(const lj_index* idx, Model model, const uint64_t* S, uint64_t m,
                  uint32_t* counts, uint64_t* offsets, uint64_t* total_host, cudaStream_t s) {
  unsigned char* b = nullptr;
  if (int rc = noalloc_scratch(idx->device, &b)) return rc;
  const uint32_t tiles = (uint32_t)std::max<uint64_t>(1, (m + kNoAllocTile - 1) / kNoAllocTile);
  // clear the ticket and the flags of this call's tiles (not the error word)
  LJ_CUDA(cudaMemsetAsync(b, 0, 128, s));
  LJ_CUDA(cudaMemsetAsync(b + 256, 0, ((size_t)tiles * 4 + 255) / 256 * 256, s));
  uint32_t* err = (uint32_t*)(b + 128);
  ProbeParams<Model> P = make_params(idx, model, S, m, 0, err);
  P.counts = counts;
  P.offsets = offsets;
  P.total_ws = (uint64_t*)(b + 64);
  P.st.ticket = (uint32_t*)b;
  P.st.flag = (uint32_t*)(b + 256);
  P.st.agg = (uint64_t*)(b + 256 + kNoAllocFlagBytes);
  P.st.incl = P.st.agg + kNoAllocTiles;
  P.st.polls = lookback_polls();
  P.num_tiles = tiles;
  P.tile_skip = std::min(fault_skip_tiles(), tiles - 1);
  const unsigned grid = tiles - P.tile_skip;
  const bool vec = aligned(S, 16) && (!offsets || aligned(offsets, 16)) && (!counts || aligned(counts, 8));
  if (idx->unique)
    vec ? probe_single_pass_kernel<Model, kUniqueCount, kRounds, true><<<grid, kBlock, 0, s>>>(P)
        : probe_single_pass_kernel<Model, kUniqueCount, kRounds, false><<<grid, kBlock, 0, s>>>(P);
  else
    vec ? probe_single_pass_kernel<Model, kDupCount, kRounds, true><<<grid, kBlock, 0, s>>>(P)
        : probe_single_pass_kernel<Model, kDupCount, kRounds, false><<<grid, kBlock, 0, s>>>(P);
  LJ_CUDA(cudaGetLastError());
  if (total_host) {
    uint32_t e = 0;
    LJ_CUDA(cudaMemcpyAsync(total_host, P.total_ws, 8, cudaMemcpyDeviceToHost, s));
    LJ_CUDA(cudaMemcpyAsync(&e, err, 4, cudaMemcpyDeviceToHost, s));
    LJ_CUDA(cudaStreamSynchronize(s));
    if (e) {
      LJ_CUDA(cudaMemsetAsync(err, 0, 4, s));
      LJ_CUDA(cudaStreamSynchronize(s));
      if (e & kErrLookbackTimeout)
        return fail(LJ_E_TIMEOUT, "join_count_noalloc: a device-side look-back wait ran out "
                                  "(in this call or an earlier one without total_host)");
      return fail(LJ_E_CUDA, "join_count_noalloc: device error bits 0x%x", e);
    }
  }
  return 0;
}
}  // namespace
}  // namespace lj

extern "C" int join_count_noalloc(const lj_index* idx, const uint64_t* S_dev, uint64_t m,
                                  uint32_t* counts_dev, uint64_t* offsets_dev,
                                  uint64_t* total_host, lj_stream_t stream) {
  using namespace lj;
  if (int rc = check_common(idx, S_dev, m, "join_count_noalloc")) return rc;
  if (idx->gkeys)
    return fail(LJ_E_INVAL, "join_count_noalloc: a gapped index (grmi_build) is not supported; "
                            "use join_count or grmi_drop");
  if (m > kNoAllocMaxProbes)
    return fail(LJ_E_INVAL,
                "join_count_noalloc: m = %llu exceeds the limit of %llu probes per call set by "
                "its fixed scratch array; split the batch or use join_count",
                (unsigned long long)m, (unsigned long long)kNoAllocMaxProbes);
  cudaStream_t s = (cudaStream_t)stream;
  if (m == 0) {
    if (offsets_dev) LJ_CUDA(cudaMemsetAsync(offsets_dev, 0, 8, s));
    if (total_host) {
      *total_host = 0;
      LJ_CUDA(cudaStreamSynchronize(s));
    }
    return LJ_OK;
  }
  if (idx->precision == LJ_FP64)
    return noalloc_count(idx, f64_model(idx), S_dev, m, counts_dev, offsets_dev, total_host, s);
  return noalloc_count(idx, f32_model(idx), S_dev, m, counts_dev, offsets_dev, total_host, s);
}
