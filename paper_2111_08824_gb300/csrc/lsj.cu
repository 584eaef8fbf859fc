// Learned sort-merge join (L-SJ, Section 4 of Sabek and Kraska, "The Case
// for Learned In-Memory Joins") of two unsorted relations on the GPU.
//
//   model      (Section 4.B, model building) per relation, a sample of up
//              to kSample keys at evenly spaced positions, sorted in shared
//              memory by one block; the CDF model is the piecewise-linear
//              function through every kKnotGap-th key of the sorted sample
//              (the empirical CDF of the sample, smoothed).
//              part(x) = min(P - 1, floor(p(x) * P / s)), p(x) the spline's
//              position of x in the sample (a real number, monotone), s the
//              sample size, P the number of partitions (one per kPartKeys
//              keys on average).
//   partition  (Section 4.B, range partitioning) each key's partition
//              (histogram with warp-aggregated atomics), a scan, and a
//              scatter of (key, position) into partition order.  The model
//              is monotone, so the partitions are key ranges in order.
//   sort       (Section 4.C) every partition sorted on its own, by (key,
//              position): one block per partition; in shared memory (up to
//              kSortCap entries) the partition is split once more, into
//              buckets by the top bits of its keys' offsets from its smallest
//              key, and each entry is placed by its rank inside its bucket
//              (a bitonic network when a bucket is crowded); larger
//              partitions, e.g. many copies of one key, take a bitonic
//              network in global memory.  After this the relation is
//              globally sorted.
//   join       (Section 4.D, chunked join) R's sorted partitions are cut
//              into chunks of at most kJoinChunk keys; S's model, queried
//              with a chunk's first and last key, gives the overlapping
//              partitions of S; each S key of them is looked up in the chunk
//              (staged in shared memory): a count pass, a scan of the counts
//              per chunk, a write pass.
// Output: the pairs (i, j) with R[i] == S[j], i and j positions in the
// relations as given, grouped by R chunk, then in S's sorted order, then in
// R's sorted order (deterministic).
//
// Differences from the paper's CPU design: the sample is evenly spaced and
// at most 16,384 keys (one block sorts it in shared memory); the partitions
// are sized for a thread block's shared memory rather than for TLB entries;
// inside a partition the keys are split further (the paper's idea of
// sub-partitioning before sorting, taken one level down: by key offset
// rather than by the model) and ranked in shared memory, with a bitonic
// network in shared memory (not AVX registers) only for crowded buckets; no
// software write-combine buffers (the scatter goes through L2).
#include <algorithm>
#include <vector>

#include "device_common.cuh"
#include "internal.h"

namespace lj {
namespace {

constexpr uint32_t kSample = 16384;      // largest sample per relation
constexpr uint32_t kPartKeys = 2048;     // keys per partition on average
constexpr uint32_t kSortCap = 8192;      // largest partition sorted in shared memory
constexpr uint32_t kJoinChunk = 4096;    // R keys per join work item
constexpr int kLBlock = 256;

__device__ __forceinline__ bool kv_less(uint64_t ka, uint32_t va, uint64_t kb, uint32_t vb) {
  return ka < kb || (ka == kb && va < vb);
}

// Ascending sort of (k[i], v[i]), i < cnt, by (key, value): a bitonic
// network whose merges begin with the mirrored comparison, so every
// comparison sends the smaller entry to the lower index and the virtual
// entries past cnt (+infinity) never move.  Called by the whole block.
__device__ void bitonic_kv(uint64_t* k, uint32_t* v, uint32_t cnt) {
  uint32_t N = 1;
  while (N < cnt) N <<= 1;
  for (uint32_t size = 2; size <= N; size <<= 1) {
    const uint32_t half = size >> 1;
    for (uint32_t i = threadIdx.x; i < N / 2; i += blockDim.x) {
      const uint32_t blk = i / half, off = i % half;
      const uint32_t lo = blk * size + off, hi = blk * size + size - 1 - off;
      if (hi < cnt && kv_less(k[hi], v[hi], k[lo], v[lo])) {
        const uint64_t tk = k[lo];
        k[lo] = k[hi];
        k[hi] = tk;
        const uint32_t tv = v[lo];
        v[lo] = v[hi];
        v[hi] = tv;
      }
    }
    __syncthreads();
    for (uint32_t stride = half >> 1; stride > 0; stride >>= 1) {
      for (uint32_t i = threadIdx.x; i < N / 2; i += blockDim.x) {
        const uint32_t lo = 2 * stride * (i / stride) + (i % stride), hi = lo + stride;
        if (hi < cnt && kv_less(k[hi], v[hi], k[lo], v[lo])) {
          const uint64_t tk = k[lo];
          k[lo] = k[hi];
          k[hi] = tk;
          const uint32_t tv = v[lo];
          v[lo] = v[hi];
          v[hi] = tv;
        }
      }
      __syncthreads();
    }
  }
}

// Evenly spaced sample of s keys (position floor((2t + 1) n / (2s))),
// sorted in shared memory by one block.
__global__ void __launch_bounds__(1024) lsj_sample_kernel(const uint64_t* __restrict__ X,
                                                          uint64_t n, uint32_t s,
                                                          uint64_t* __restrict__ out) {
  extern __shared__ uint64_t sk[];
  uint32_t* sv = reinterpret_cast<uint32_t*>(sk + kSample);
  for (uint32_t t = threadIdx.x; t < s; t += blockDim.x) {
    sk[t] = X[((2 * (uint64_t)t + 1) * n) / (2 * (uint64_t)s)];
    sv[t] = t;
  }
  __syncthreads();
  bitonic_kv(sk, sv, s);
  for (uint32_t t = threadIdx.x; t < s; t += blockDim.x) out[t] = sk[t];
}

// CDF model of a relation (Section 4.B): the piecewise-linear function
// through every kKnotGap-th key of its sorted sample (knot k = sample[k G],
// the last knot the largest sample key), i.e. the sample's empirical CDF
// smoothed over kKnotGap sample gaps.  Unlike the clamped prediction of a
// model with separately fitted pieces it is continuous, so no partition
// collects the keys of a gap between two pieces.
struct Spline {
  const uint64_t* knot;   // K + 1 knot keys, non-decreasing
  const uint32_t* table;  // radix table: 2^kRadixBits + 1 entries
  uint32_t K;             // segments
  uint32_t s;             // sample size (positions 0 .. s - 1)
  uint32_t shift;         // prefix of x = (x - knot[0]) >> shift
};
constexpr uint32_t kKnotGap = 32;
constexpr uint32_t kRadixBits = 12;

__device__ __forceinline__ uint32_t knot_pos(const Spline& m, uint32_t k) {
  return min(k * kKnotGap, m.s - 1);
}

// Partition of key x: its position in the sample by the spline (a real
// number in [0, s - 1]), scaled to the P partitions.  Monotone in x (the
// interpolation within a segment is, and segments meet at the knots), so
// the partitions are key ranges in key order.
__device__ __forceinline__ uint32_t part_of(const Spline& m, uint64_t x, uint32_t P) {
  const uint64_t* kn = m.knot;
  if (x <= __ldg(reinterpret_cast<const unsigned long long*>(kn))) return 0;
  if (x >= __ldg(reinterpret_cast<const unsigned long long*>(kn) + m.K)) return P - 1;
  // last knot <= x: the knots with x's prefix (table) and the one before them
  const uint32_t b = (uint32_t)((x - __ldg(reinterpret_cast<const unsigned long long*>(kn))) >> m.shift);
  const uint32_t t0 = __ldg(m.table + b), t1 = __ldg(m.table + b + 1);
  uint32_t lo = t0 ? t0 - 1 : 0, len = min(t1, m.K) - lo;
  while (len > 1) {
    const uint32_t h = len >> 1;
    if (__ldg(reinterpret_cast<const unsigned long long*>(kn) + lo + h) <= x) lo += h;
    len -= h;
  }
  const uint64_t k0 = __ldg(reinterpret_cast<const unsigned long long*>(kn) + lo);
  const uint64_t k1 = __ldg(reinterpret_cast<const unsigned long long*>(kn) + lo + 1);
  const float y0 = (float)knot_pos(m, lo), y1 = (float)knot_pos(m, lo + 1);
  const float f = __fdiv_rn(__ull2float_rn(x - k0), __ull2float_rn(k1 - k0));   // in [0, 1]
  const float q = __fmul_rn(__fmaf_rn(y1 - y0, f, y0), (float)P / (float)m.s);
  return q < (float)P ? (uint32_t)q : P - 1;
}

// Knots of the spline from the sorted sample, and the radix table over their
// prefixes: table[b] = the number of knots whose prefix is below b, for
// b = 0 .. 2^kRadixBits (knot k fills the entries after its predecessor's
// prefix up to its own).  One block.
__global__ void lsj_knots_kernel(const uint64_t* __restrict__ sample, uint32_t s, uint32_t K,
                                 uint32_t shift, uint64_t* __restrict__ knot,
                                 uint32_t* __restrict__ table) {
  for (uint32_t k = threadIdx.x; k <= K; k += blockDim.x) knot[k] = sample[min(k * kKnotGap, s - 1)];
  __syncthreads();
  const uint64_t k0 = knot[0];
  constexpr uint32_t T = 1u << kRadixBits;
  for (uint32_t k = threadIdx.x; k <= K; k += blockDim.x) {
    const int64_t p = (int64_t)((knot[k] - k0) >> shift);   // < T
    const int64_t q = k ? (int64_t)((knot[k - 1] - k0) >> shift) : -1;
    for (int64_t b = q + 1; b <= p; ++b) table[b] = k;
    if (k == K)
      for (uint32_t b = (uint32_t)p + 1; b <= T; ++b) table[b] = K + 1;
  }
}

// Partition of every key and the partition sizes.
__global__ void __launch_bounds__(kLBlock)
    lsj_hist_kernel(const uint64_t* __restrict__ X, uint64_t n, Spline m, uint32_t P,
                    uint32_t* __restrict__ pid, unsigned long long* __restrict__ cnt) {
  const uint64_t i = (uint64_t)blockIdx.x * kLBlock + threadIdx.x;
  const bool valid = i < n;
  const uint32_t p =
      valid ? part_of(m, __ldg(reinterpret_cast<const unsigned long long*>(X) + i), P) : 0;
  const unsigned mask = __ballot_sync(0xffffffffu, valid);
  if (valid) {
    pid[i] = p;
    const unsigned grp = __match_any_sync(mask, p);
    if ((int)(threadIdx.x & 31) == __ffs(grp) - 1) atomicAdd(cnt + p, (unsigned long long)__popc(grp));
  }
}

// Exclusive scan of cnt[0..P) into off[0..P] (off[P] = total), one block.
__global__ void __launch_bounds__(1024) lsj_scan_kernel(const unsigned long long* __restrict__ cnt,
                                                        uint32_t P, uint64_t* __restrict__ off) {
  __shared__ uint64_t s[1024];
  const uint32_t per = (P + 1023) / 1024;
  const uint32_t b = threadIdx.x * per, e = min(P, b + per);
  uint64_t sum = 0;
  for (uint32_t t = b; t < e; ++t) sum += cnt[t];
  s[threadIdx.x] = sum;
  __syncthreads();
  for (uint32_t d = 1; d < 1024; d <<= 1) {
    const uint64_t v = threadIdx.x >= d ? s[threadIdx.x - d] : 0;
    __syncthreads();
    s[threadIdx.x] += v;
    __syncthreads();
  }
  uint64_t run = threadIdx.x ? s[threadIdx.x - 1] : 0;
  for (uint32_t t = b; t < e; ++t) {
    off[t] = run;
    run += cnt[t];
  }
  if (threadIdx.x == 1023) off[P] = s[1023];
}

// (key, position) into its partition's next free slot, as one 16-byte
// record (one scattered store per key instead of two).
__global__ void __launch_bounds__(kLBlock)
    lsj_scatter_kernel(const uint64_t* __restrict__ X, uint64_t n, const uint32_t* __restrict__ pid,
                       const uint64_t* __restrict__ off, unsigned long long* __restrict__ cursor,
                       ulonglong2* __restrict__ rec) {
  const uint64_t i = (uint64_t)blockIdx.x * kLBlock + threadIdx.x;
  const bool valid = i < n;
  const uint32_t p = valid ? pid[i] : 0;
  const unsigned mask = __ballot_sync(0xffffffffu, valid);
  if (!valid) return;
  const unsigned grp = __match_any_sync(mask, p);
  const int lane = threadIdx.x & 31, leader = __ffs(grp) - 1;
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(cursor + p, (unsigned long long)__popc(grp));
  base = __shfl_sync(grp, base, leader);
  const uint64_t at = off[p] + base + __popc(grp & ((1u << lane) - 1u));
  rec[at] = make_ulonglong2(X[i], i);   // one 16-byte store per key
}

// One block per partition: sort it by (key, position).  Launched twice:
// CAP = kSortSmall for the partitions of at most kSortSmall entries (48 KB of
// shared memory, four blocks per SM), CAP = kSortCap for the larger ones
// (and, above kSortCap, a bitonic network in global memory).  In shared
// memory the partition is bucketed by the top bits of (key - its smallest
// key), about 8 entries per bucket, and every entry's rank inside its bucket
// by (key, position) -- the pairs are all distinct -- gives its final place
// directly: a handful of barriers instead of the O(log^2) stages of a
// bitonic network.  A partition with a bucket above kRankMax entries (many
// equal or clustered keys) goes through the bitonic network instead.
constexpr uint32_t kSortSmall = 4096;
#ifndef LJ_SORT_THREADS
#define LJ_SORT_THREADS 512    // threads of the first sort launch: 512 x 3 blocks per SM
#endif                         // (1.63 ms per 100M keys; 1024 x 2 blocks: 2.33 ms)
#ifndef LJ_SORT_MINB
#define LJ_SORT_MINB 3
#endif
constexpr uint32_t kSortThreads = LJ_SORT_THREADS;
constexpr uint32_t kRankMax = 64;

__device__ __forceinline__ uint32_t bitlen64(uint64_t v) { return v ? 64u - __clzll(v) : 0u; }

// Sort of one partition [a, a + n) in shared memory (2 <= n <= CAP), by the
// whole block.  ITEMS > 0: each thread keeps its ITEMS entries (t,
// t + blockDim.x, ...) in registers, so the partition is read from global
// memory once.
template <uint32_t CAP, int ITEMS>
__device__ void sort_partition(const ulonglong2* __restrict__ rec, uint64_t* __restrict__ keys,
                               uint32_t* __restrict__ pos, uint64_t a, uint32_t n, uint64_t* sk,
                               uint32_t* sv,
                               uint32_t* s_cur, uint32_t* s_start, uint64_t* s_min,
                               uint64_t* s_max, uint32_t* s_big) {
  constexpr uint32_t kBuckets = CAP / 8;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int kR = ITEMS > 0 ? ITEMS : 1;
  uint64_t rk[kR];
  uint32_t rv[kR];
  // smallest and largest key
  uint64_t lo = ~0ull, hi = 0;
  if (ITEMS > 0) {
#pragma unroll
    for (int i = 0; i < kR; ++i) {
      const uint32_t t = threadIdx.x + i * blockDim.x;
      const ulonglong2 e = t < n ? rec[a + t] : make_ulonglong2(0, 0);
      rk[i] = e.x;
      rv[i] = (uint32_t)e.y;
      if (t < n) {
        lo = rk[i] < lo ? rk[i] : lo;
        hi = rk[i] > hi ? rk[i] : hi;
      }
    }
  } else {
    for (uint32_t t = threadIdx.x; t < n; t += blockDim.x) {
      const uint64_t x = rec[a + t].x;
      lo = x < lo ? x : lo;
      hi = x > hi ? x : hi;
    }
  }
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) {
    const uint64_t l2 = __shfl_xor_sync(0xffffffffu, (unsigned long long)lo, d);
    const uint64_t h2 = __shfl_xor_sync(0xffffffffu, (unsigned long long)hi, d);
    lo = l2 < lo ? l2 : lo;
    hi = h2 > hi ? h2 : hi;
  }
  if (lane == 0) {
    s_min[warp] = lo;
    s_max[warp] = hi;
  }
  const uint32_t nbits = min(31u - __clz(max(n / 8, 1u)) + 1u, 31u - __clz(kBuckets));
  const uint32_t nb = 1u << nbits;   // buckets: about 4 to 8 entries each, at most kBuckets
  for (uint32_t t = threadIdx.x; t < nb; t += blockDim.x) s_cur[t] = 0;
  if (threadIdx.x == 0) *s_big = 0;
  __syncthreads();
  lo = s_min[0];
  hi = s_max[0];
  for (uint32_t w = 1; w < blockDim.x / 32; ++w) {
    lo = s_min[w] < lo ? s_min[w] : lo;
    hi = s_max[w] > hi ? s_max[w] : hi;
  }
  const uint32_t rb = bitlen64(hi - lo);
  const uint32_t shift = rb > nbits ? rb - nbits : 0u;   // (hi - lo) >> shift < nb
  if (ITEMS > 0) {
#pragma unroll
    for (int i = 0; i < kR; ++i)
      if (threadIdx.x + i * blockDim.x < n) atomicAdd(&s_cur[(uint32_t)((rk[i] - lo) >> shift)], 1u);
  } else {
    for (uint32_t t = threadIdx.x; t < n; t += blockDim.x)
      atomicAdd(&s_cur[(uint32_t)((rec[a + t].x - lo) >> shift)], 1u);
  }
  __syncthreads();
  // bucket starts (exclusive scan by warp 0) and the largest bucket
  if (warp == 0) {
    uint32_t run = 0, big = 0;
    for (uint32_t c0 = 0; c0 < nb; c0 += 32) {
      const uint32_t v = c0 + lane < nb ? s_cur[c0 + lane] : 0u;
      big = v > big ? v : big;
      uint32_t inc = v;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += u;
      }
      if (c0 + lane < nb) s_start[c0 + lane] = run + inc - v;
      run += __shfl_sync(0xffffffffu, inc, 31);
    }
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) big = max(big, __shfl_xor_sync(0xffffffffu, big, d));
    if (lane == 0) {
      s_start[nb] = run;
      *s_big = big > kRankMax ? 1u : 0u;
    }
  }
  __syncthreads();
  if (*s_big) {   // a crowded bucket: the bitonic network on the whole partition
    if (ITEMS > 0) {
#pragma unroll
      for (int i = 0; i < kR; ++i) {
        const uint32_t t = threadIdx.x + i * blockDim.x;
        if (t < n) {
          sk[t] = rk[i];
          sv[t] = rv[i];
        }
      }
    } else {
      for (uint32_t t = threadIdx.x; t < n; t += blockDim.x) {
        const ulonglong2 e = rec[a + t];
        sk[t] = e.x;
        sv[t] = (uint32_t)e.y;
      }
    }
    __syncthreads();
    bitonic_kv(sk, sv, n);
    for (uint32_t t = threadIdx.x; t < n; t += blockDim.x) {
      keys[a + t] = sk[t];
      pos[a + t] = sv[t];
    }
    __syncthreads();   // shared memory is reused by the block's next partition
    return;
  }
  // scatter into bucket order (any order inside a bucket)
  for (uint32_t t = threadIdx.x; t < nb; t += blockDim.x) s_cur[t] = s_start[t];
  __syncthreads();
  if (ITEMS > 0) {
#pragma unroll
    for (int i = 0; i < kR; ++i)
      if (threadIdx.x + i * blockDim.x < n) {
        const uint32_t q = atomicAdd(&s_cur[(uint32_t)((rk[i] - lo) >> shift)], 1u);
        sk[q] = rk[i];
        sv[q] = rv[i];
      }
  } else {
    for (uint32_t t = threadIdx.x; t < n; t += blockDim.x) {
      const ulonglong2 e = rec[a + t];
      const uint32_t q = atomicAdd(&s_cur[(uint32_t)((e.x - lo) >> shift)], 1u);
      sk[q] = e.x;
      sv[q] = (uint32_t)e.y;
    }
  }
  __syncthreads();
  // final place of each entry: its bucket's start + its rank in the bucket
  for (uint32_t q = threadIdx.x; q < n; q += blockDim.x) {
    const uint64_t x = sk[q];
    const uint32_t v = sv[q];
    const uint32_t bk = (uint32_t)((x - lo) >> shift);
    const uint32_t s0 = s_start[bk], s1 = s_start[bk + 1];
    uint32_t r = 0;
    for (uint32_t j = s0; j < s1; ++j) r += kv_less(sk[j], sv[j], x, v) ? 1u : 0u;
    keys[a + s0 + r] = x;
    pos[a + s0 + r] = v;
  }
  __syncthreads();   // shared memory is reused by the block's next partition
}

// First sort launch, one block per partition: partitions of at most
// kSortSmall entries are sorted here (48 KB of shared memory, entries kept in
// registers); larger ones are appended to `big` for lsj_sort_big_kernel.
__global__ void __launch_bounds__(kSortThreads, LJ_SORT_MINB)
    lsj_sort_kernel(const ulonglong2* __restrict__ rec, uint64_t* __restrict__ keys,
                    uint32_t* __restrict__ pos, const uint64_t* __restrict__ off,
                    uint32_t* __restrict__ big) {
  extern __shared__ uint64_t sk[];
  uint32_t* sv = reinterpret_cast<uint32_t*>(sk + kSortSmall);
  __shared__ uint32_t s_cur[kSortSmall / 8];
  __shared__ uint32_t s_start[kSortSmall / 8 + 1];
  __shared__ uint64_t s_min[32], s_max[32];
  __shared__ uint32_t s_big;
  const uint64_t a = off[blockIdx.x], b = off[blockIdx.x + 1];
  const uint64_t cnt = b - a;
  if (cnt <= 1) {   // nothing to sort; a lone record is copied out
    if (cnt == 1 && threadIdx.x == 0) {
      const ulonglong2 e = rec[a];
      keys[a] = e.x;
      pos[a] = (uint32_t)e.y;
    }
    return;
  }
  if (cnt > kSortSmall) {
    if (threadIdx.x == 0) big[1 + atomicAdd(big, 1u)] = blockIdx.x;   // big[0] = count
    return;
  }
  sort_partition<kSortSmall, kSortSmall / kSortThreads>(rec, keys, pos, a, (uint32_t)cnt, sk, sv,
                                                        s_cur, s_start, s_min, s_max, &s_big);
}

// Second sort launch: the partitions listed in `big` (more than kSortSmall
// entries), a few blocks striding over the list; up to kSortCap entries in
// shared memory, larger ones (e.g. many copies of one key) through a bitonic
// network in global memory.
__global__ void __launch_bounds__(512)
    lsj_sort_big_kernel(const ulonglong2* __restrict__ rec, uint64_t* __restrict__ keys,
                        uint32_t* __restrict__ pos, const uint64_t* __restrict__ off,
                        const uint32_t* __restrict__ big) {
  extern __shared__ uint64_t sk[];
  uint32_t* sv = reinterpret_cast<uint32_t*>(sk + kSortCap);
  __shared__ uint32_t s_cur[kSortCap / 8];
  __shared__ uint32_t s_start[kSortCap / 8 + 1];
  __shared__ uint64_t s_min[16], s_max[16];
  __shared__ uint32_t s_big;
  const uint32_t count = big[0];
  for (uint32_t i = blockIdx.x; i < count; i += gridDim.x) {
    const uint32_t part = big[1 + i];
    const uint64_t a = off[part], cnt = off[part + 1] - a;
    if (cnt > kSortCap) {   // large partition: a bitonic network in global memory
      for (uint64_t t = threadIdx.x; t < cnt; t += blockDim.x) {
        const ulonglong2 e = rec[a + t];
        keys[a + t] = e.x;
        pos[a + t] = (uint32_t)e.y;
      }
      __syncthreads();
      bitonic_kv(keys + a, pos + a, (uint32_t)cnt);
      __syncthreads();
    } else {
      sort_partition<kSortCap, 0>(rec, keys, pos, a, (uint32_t)cnt, sk, sv, s_cur, s_start, s_min,
                                  s_max, &s_big);
    }
  }
}

// Join work item: R's sorted positions [ra, ra + len) (len <= kJoinChunk, in
// one partition) and the overlapping range [sa, sb) of S's sorted keys.
struct JoinItem {
  uint64_t ra, sa, sb;
  uint32_t len, pad;
};

// Items of R's partitions (chunks of kJoinChunk keys) with their S ranges.
__global__ void lsj_items_kernel(const uint64_t* __restrict__ rkeys, const uint64_t* __restrict__ roff,
                                 uint32_t PR, const uint64_t* __restrict__ item0, Spline ms,
                                 uint32_t PS, const uint64_t* __restrict__ soff,
                                 JoinItem* __restrict__ items) {
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < PR; p += gridDim.x * blockDim.x) {
    const uint64_t a = roff[p], b = roff[p + 1];
    uint64_t it = item0[p];
    for (uint64_t c = a; c < b; c += kJoinChunk, ++it) {
      const uint64_t e = min(b, c + kJoinChunk);
      JoinItem J;
      J.ra = c;
      J.len = (uint32_t)(e - c);
      J.pad = 0;
      const uint32_t f = part_of(ms, rkeys[c], PS);
      const uint32_t l = part_of(ms, rkeys[e - 1], PS);
      J.sa = soff[f];
      J.sb = soff[l + 1];
      items[it] = J;
    }
  }
}

// Count pass (WRITE = false: per-item match counts) and write pass (WRITE:
// the pairs at the item's offset).  Block per item; the item's R keys are
// staged in shared memory and every S key of the range is bounded in them.
template <bool WRITE>
__global__ void __launch_bounds__(kLBlock)
    lsj_join_kernel(const JoinItem* __restrict__ items, const uint64_t* __restrict__ rkeys,
                    const uint32_t* __restrict__ rpos, const uint64_t* __restrict__ skeys,
                    const uint32_t* __restrict__ spos, unsigned long long* __restrict__ count,
                    const uint64_t* __restrict__ ioff, lj_pair* __restrict__ pairs,
                    uint64_t capacity) {
  __shared__ uint64_t sr[kJoinChunk];
  __shared__ uint32_t sw[kLBlock / 32];
  __shared__ uint64_t s_run;
  const JoinItem J = items[blockIdx.x];
  for (uint32_t t = threadIdx.x; t < J.len; t += kLBlock) sr[t] = rkeys[J.ra + t];
  if (threadIdx.x == 0) s_run = WRITE ? ioff[blockIdx.x] : 0;
  __syncthreads();
  const uint64_t lo_key = sr[0], hi_key = sr[J.len - 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long total = 0;
  for (uint64_t base = J.sa; base < J.sb; base += kLBlock) {
    const uint64_t q = base + threadIdx.x;
    uint32_t lb = 0, c = 0;
    if (q < J.sb) {
      const uint64_t x = skeys[q];
      if (x >= lo_key && x <= hi_key) {
        uint32_t a = 0, len = J.len;   // lower bound of x in the chunk
        while (len > 0) {
          const uint32_t h = len >> 1;
          if (sr[a + h] < x) {
            a += h + 1;
            len -= h + 1;
          } else {
            len = h;
          }
        }
        uint32_t u = a;
        len = J.len - a;               // upper bound
        while (len > 0) {
          const uint32_t h = len >> 1;
          if (sr[u + h] <= x) {
            u += h + 1;
            len -= h + 1;
          } else {
            len = h;
          }
        }
        lb = a;
        c = u - a;
      }
    }
    if (!WRITE) {
      total += c;
      continue;
    }
    // block exclusive scan of c: the round's output positions
    uint32_t inc = c;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t v = __shfl_up_sync(0xffffffffu, inc, d);
      if (lane >= d) inc += v;
    }
    if (lane == 31) sw[warp] = inc;
    __syncthreads();
    uint64_t at = s_run + inc - c;
    uint32_t round = 0;
    for (int w = 0; w < kLBlock / 32; ++w) {
      if (w < warp) at += sw[w];
      round += sw[w];
    }
    if (c) {
      const uint32_t sj = spos[q];
      for (uint32_t t = 0; t < c; ++t)
        if (at + t < capacity) pairs[at + t] = lj_pair{rpos[J.ra + lb + t], sj};
    }
    __syncthreads();
    if (threadIdx.x == 0) s_run += round;
    __syncthreads();
  }
  if (!WRITE) {
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) total += __shfl_xor_sync(0xffffffffu, total, d);
    __shared__ unsigned long long s_tot[kLBlock / 32];
    if (lane == 0) s_tot[warp] = total;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long t = 0;
      for (int w = 0; w < kLBlock / 32; ++w) t += s_tot[w];
      count[blockIdx.x] = t;
    }
  }
}

unsigned blocks_for(uint64_t work, unsigned block) {
  return (unsigned)std::max<uint64_t>(1, (work + block - 1) / block);
}

// One relation, partitioned and sorted: keys/pos in sorted order, off[P+1]
// partition starts, and the model that partitioned it.
struct Sorted {
  uint64_t* knot = nullptr;   // the spline's knots (kSample / kKnotGap + 1 at most)
  uint32_t* table = nullptr;  // its radix table, after the knots
  uint32_t K = 0, shift = 0;
  uint32_t s = 0, P = 1;
  uint64_t* keys = nullptr;
  uint32_t* pos = nullptr;
  uint64_t* off = nullptr;
};

int sort_relation(const uint64_t* X, uint64_t n, Sorted& out, cudaStream_t s,
                  uint64_t* sample_buf, uint32_t* pid, unsigned long long* cnt,
                  unsigned long long* cursor, uint32_t* big, ulonglong2* rec) {
  out.s = (uint32_t)std::min<uint64_t>(n, kSample);
  out.P = (uint32_t)std::max<uint64_t>(1, (n + kPartKeys - 1) / kPartKeys);
  // model: sorted sample, knots of its spline
  const size_t smem = (size_t)kSample * 12;
  lsj_sample_kernel<<<1, 1024, smem, s>>>(X, n, out.s, sample_buf);
  LJ_CUDA(cudaGetLastError());
  out.K = std::max<uint32_t>(1, (out.s - 1 + kKnotGap - 1) / kKnotGap);
  // the radix table's shift needs the key range of the knots: the sample's
  // smallest and largest keys, read back (one small copy, synchronising)
  uint64_t ends[2];
  LJ_CUDA(cudaMemcpyAsync(&ends[0], sample_buf, 8, cudaMemcpyDeviceToHost, s));
  LJ_CUDA(cudaMemcpyAsync(&ends[1], sample_buf + out.s - 1, 8, cudaMemcpyDeviceToHost, s));
  LJ_CUDA(cudaStreamSynchronize(s));
  uint32_t bits = 0;
  for (uint64_t r = ends[1] - ends[0]; r; r >>= 1) ++bits;
  out.shift = bits > kRadixBits ? bits - kRadixBits : 0;
  out.table = (uint32_t*)(out.knot + kSample / kKnotGap + 2);
  lsj_knots_kernel<<<1, 256, 0, s>>>(sample_buf, out.s, out.K, out.shift, out.knot, out.table);
  LJ_CUDA(cudaGetLastError());
  const Spline m{out.knot, out.table, out.K, out.s, out.shift};
  LJ_CUDA(cudaMemsetAsync(cnt, 0, (size_t)out.P * 8, s));
  LJ_CUDA(cudaMemsetAsync(cursor, 0, (size_t)out.P * 8, s));
  {
    KernelTimer kt("lsj_hist_kernel", s);
    lsj_hist_kernel<<<blocks_for(n, kLBlock), kLBlock, 0, s>>>(X, n, m, out.P, pid, cnt);
  }
  lsj_scan_kernel<<<1, 1024, 0, s>>>(cnt, out.P, out.off);
  {
    KernelTimer kt("lsj_scatter_kernel", s);
    lsj_scatter_kernel<<<blocks_for(n, kLBlock), kLBlock, 0, s>>>(X, n, pid, out.off, cursor,
                                                                  rec);
  }
  LJ_CUDA(cudaMemsetAsync(big, 0, 4, s));
  {
    KernelTimer kt("lsj_sort_kernel", s);
    lsj_sort_kernel<<<out.P, kSortThreads, (size_t)kSortSmall * 12, s>>>(rec, out.keys, out.pos,
                                                                        out.off, big);
  }
  {
    KernelTimer kt("lsj_sort_big_kernel", s);
    lsj_sort_big_kernel<<<std::min<uint32_t>(out.P, 304), 512, (size_t)kSortCap * 12, s>>>(
        rec, out.keys, out.pos, out.off, big);
  }
  LJ_CUDA(cudaGetLastError());
  return 0;
}

size_t round256(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace
}  // namespace lj

extern "C" int lsj_join(const uint64_t* R_dev, uint64_t n, const uint64_t* S_dev, uint64_t m,
                        lj_pair* pairs_dev, uint64_t capacity, uint64_t* written_host,
                        lj_stream_t stream) {
  using namespace lj;
  if (n >= (1ull << 32) || m >= (1ull << 32))
    return fail(LJ_E_INVAL, "lsj_join: n and m must be below 2^32");
  if ((n && !R_dev) || (m && !S_dev)) return fail(LJ_E_INVAL, "lsj_join: R or S is NULL");
  if (capacity > 0 && !pairs_dev) return fail(LJ_E_INVAL, "lsj_join: pairs is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  if (n == 0 || m == 0) {
    if (written_host) {
      *written_host = 0;
      LJ_CUDA(cudaStreamSynchronize(s));
    }
    return LJ_OK;
  }
  // shared memory above 48 KB for the two sorting kernels (on the current device)
  LJ_CUDA(cudaFuncSetAttribute(lsj_sample_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)(kSample * 12)));
  LJ_CUDA(cudaFuncSetAttribute(lsj_sort_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)(kSortSmall * 12)));
  LJ_CUDA(cudaFuncSetAttribute(lsj_sort_big_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)(kSortCap * 12)));
  Sorted R, S;
  const uint64_t nm = std::max(n, m);
  const uint32_t Pmax = (uint32_t)((nm + kPartKeys - 1) / kPartKeys) + 1;
  // scratch: sample, pid, counts, cursors, offsets x2, sorted keys/pos x2
  const size_t b_sample = round256((size_t)kSample * 8);
  const size_t b_pid = round256(nm * 4);
  const size_t b_cnt = round256((size_t)Pmax * 8);
  const size_t b_big = round256(((size_t)Pmax + 1) * 4);
  const size_t b_knot =
      round256(((size_t)kSample / kKnotGap + 2) * 8 + (((size_t)1 << kRadixBits) + 1) * 4);
  const size_t b_rec = round256(nm * 16);
  const size_t total = b_sample + b_pid + 2 * b_cnt + b_big + 2 * b_knot + b_rec +
                       2 * round256(((size_t)Pmax + 1) * 8) +
                       round256(n * 8) + round256(n * 4) + round256(m * 8) + round256(m * 4);
  char* ws = nullptr;
  LJ_CUDA(scratch_alloc((void**)&ws, total, s));
  char* p = ws;
  auto take = [&](size_t b) {
    char* q = p;
    p += b;
    return q;
  };
  uint64_t* sample = (uint64_t*)take(b_sample);
  uint32_t* pid = (uint32_t*)take(b_pid);
  unsigned long long* cnt = (unsigned long long*)take(b_cnt);
  unsigned long long* cursor = (unsigned long long*)take(b_cnt);
  uint32_t* big = (uint32_t*)take(b_big);   // [0] count, then partition ids
  R.knot = (uint64_t*)take(b_knot);
  S.knot = (uint64_t*)take(b_knot);
  ulonglong2* rec = (ulonglong2*)take(b_rec);   // partitioned (key, position) records
  R.off = (uint64_t*)take(round256(((size_t)Pmax + 1) * 8));
  S.off = (uint64_t*)take(round256(((size_t)Pmax + 1) * 8));
  R.keys = (uint64_t*)take(round256(n * 8));
  R.pos = (uint32_t*)take(round256(n * 4));
  S.keys = (uint64_t*)take(round256(m * 8));
  S.pos = (uint32_t*)take(round256(m * 4));
  int rc = 0;
  JoinItem* items = nullptr;
  char* ws2 = nullptr;
  do {
    // S first (its model is queried by the join), then R; the sample buffer
    // is reused, so each model's knots are taken (copied) before the
    // next relation's sample is drawn
    if ((rc = sort_relation(S_dev, m, S, s, sample, pid, cnt, cursor, big, rec))) break;
    if ((rc = sort_relation(R_dev, n, R, s, sample, pid, cnt, cursor, big, rec))) break;
    // join items: chunks of R's partitions
    std::vector<uint64_t> roff(R.P + 1);
    cudaError_t ce = cudaMemcpyAsync(roff.data(), R.off, (R.P + 1) * 8, cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess) {
      rc = fail_cuda(ce, "lsj_join: partition offsets");
      break;
    }
    std::vector<uint64_t> item0(R.P + 1, 0);
    for (uint32_t q = 0; q < R.P; ++q)
      item0[q + 1] = item0[q] + (roff[q + 1] - roff[q] + kJoinChunk - 1) / kJoinChunk;
    const uint64_t nitems = item0[R.P];
    if (nitems >= (1ull << 31)) {
      rc = fail(LJ_E_INVAL, "lsj_join: too many join items");
      break;
    }
    const size_t b_items = round256(std::max<uint64_t>(nitems, 1) * sizeof(JoinItem));
    const size_t b_i0 = round256(((size_t)R.P + 1) * 8);
    const size_t b_ic = round256(std::max<uint64_t>(nitems, 1) * 8);
    const size_t b_io = round256((std::max<uint64_t>(nitems, 1) + 1) * 8);
    if ((ce = scratch_alloc((void**)&ws2, b_items + b_i0 + b_ic + b_io, s)) != cudaSuccess) {
      rc = fail_cuda(ce, "lsj_join: item scratch");
      break;
    }
    items = (JoinItem*)ws2;
    uint64_t* d_item0 = (uint64_t*)(ws2 + b_items);
    unsigned long long* icnt = (unsigned long long*)(ws2 + b_items + b_i0);
    uint64_t* ioff = (uint64_t*)(ws2 + b_items + b_i0 + b_ic);
    ce = cudaMemcpyAsync(d_item0, item0.data(), (R.P + 1) * 8, cudaMemcpyHostToDevice, s);
    if (ce != cudaSuccess) {
      rc = fail_cuda(ce, "lsj_join: item table");
      break;
    }
    const Spline ms{S.knot, S.table, S.K, S.s, S.shift};
    {
      KernelTimer kt("lsj_items_kernel", s);
      lsj_items_kernel<<<blocks_for(R.P, 256), 256, 0, s>>>(R.keys, R.off, R.P, d_item0, ms,
                                                            S.P, S.off, items);
    }
    {
      KernelTimer kt("lsj_join_count_kernel", s);
      lsj_join_kernel<false><<<(unsigned)nitems, kLBlock, 0, s>>>(items, R.keys, R.pos, S.keys,
                                                                  S.pos, icnt, nullptr, nullptr, 0);
    }
    lsj_scan_kernel<<<1, 1024, 0, s>>>(icnt, (uint32_t)nitems, ioff);
    {
      KernelTimer kt("lsj_join_write_kernel", s);
      lsj_join_kernel<true><<<(unsigned)nitems, kLBlock, 0, s>>>(items, R.keys, R.pos, S.keys,
                                                                 S.pos, nullptr, ioff, pairs_dev,
                                                                 capacity);
    }
    if ((ce = cudaGetLastError()) != cudaSuccess) {
      rc = fail_cuda(ce, "lsj_join kernels");
      break;
    }
    uint64_t written = 0;
    ce = cudaMemcpyAsync(&written, ioff + nitems, 8, cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess) {
      rc = fail_cuda(ce, "lsj_join: total");
      break;
    }
    if (written_host) *written_host = written;
    if (written > capacity)
      rc = fail(LJ_E_CAPACITY, "lsj_join: %llu pairs do not fit the capacity of %llu",
                (unsigned long long)written, (unsigned long long)capacity);
  } while (0);
  if (ws2) scratch_free(ws2, s);
  scratch_free(ws, s);
  cudaStreamSynchronize(s);
  if (!rc) rc = take_device_errors(current_device(), s);
  return rc;
}
