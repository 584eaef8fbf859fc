// Device-side building blocks of the learned indexed nested loop join.
//
// The two-level linear RMI (Section 2.D of Sabek and Kraska, "The Case for
// Learned In-Memory Joins"): a root linear model selects one of L leaf
// models; the leaf's linear model predicts a position; the leaf's min/max
// error bounds delimit the last-mile search.  The same inline functions are
// used when the index is built (to measure the error bounds) and when it is
// probed, so both evaluate the models bit for bit identically: one
// correctly rounded conversion of the key, one fused multiply-add, a floor.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace lj {

constexpr float kPredClampF = 1099511627776.0f;   // 2^40
constexpr double kPredClampD = 1099511627776.0;

// Error word bits (sticky, per device).
constexpr uint32_t kErrLookbackTimeout = 1u;
constexpr uint32_t kErrCapacity = 2u;

// --------------------------------------------------------------- records --

// Leaf record, single-precision model: 32 bytes = one DRAM sector.
struct __align__(16) LeafF32 {
  uint64_t base_key;   // R[lo]
  uint32_t lo, hi;     // positions [lo, hi) owned by the leaf
  float a, b;          // pred = lo + floor(fmaf(a, x - base_key, b))
  int32_t e_lo, e_hi;  // min / max of (i - pred(R[i])) over the leaf
};
static_assert(sizeof(LeafF32) == 32, "LeafF32 must be one sector");

// Leaf record, double-precision model: 48 bytes.
struct __align__(16) LeafF64 {
  uint64_t base_key;
  uint32_t lo, hi;
  double a, b;
  int32_t e_lo, e_hi;
  uint64_t pad;
};
static_assert(sizeof(LeafF64) == 48, "LeafF64 layout");

// ----------------------------------------------------------------- models --

struct ModelF32 {
  using Leaf = LeafF32;
  float a0, b0;
  uint32_t L;

  __device__ __forceinline__ uint32_t leaf(uint64_t x) const {
    float v = floorf(__fmaf_rn(a0, __ull2float_rn(x), b0));
    if (!(v >= 0.0f)) return 0u;
    const uint32_t lm1 = L - 1u;                 // L <= 2^24: exact in float
    return v >= (float)lm1 ? lm1 : (uint32_t)v;
  }
  __device__ __forceinline__ static int64_t pred(uint64_t x, uint64_t base, float a,
                                                 float b) {
    float d = x >= base ? __ull2float_rn(x - base) : -__ull2float_rn(base - x);
    float v = floorf(__fmaf_rn(a, d, b));
    v = fminf(fmaxf(v, -kPredClampF), kPredClampF);
    return (int64_t)v;
  }
  // one 32-byte load (the record is one aligned sector)
  __device__ __forceinline__ static Leaf load_leaf(const Leaf* leaves, uint32_t l) {
    unsigned long long w0, w1, w2, w3;
    asm("ld.global.nc.v4.u64 {%0, %1, %2, %3}, [%4];"
        : "=l"(w0), "=l"(w1), "=l"(w2), "=l"(w3)
        : "l"(leaves + l));
    Leaf r;
    r.base_key = w0;
    r.lo = (uint32_t)w1;
    r.hi = (uint32_t)(w1 >> 32);
    r.a = __uint_as_float((uint32_t)w2);
    r.b = __uint_as_float((uint32_t)(w2 >> 32));
    r.e_lo = (int32_t)(uint32_t)w3;
    r.e_hi = (int32_t)(uint32_t)(w3 >> 32);
    return r;
  }
  __device__ __forceinline__ static int64_t pred(const Leaf& lf, uint64_t x) {
    return pred(x, lf.base_key, lf.a, lf.b);
  }
};

struct ModelF64 {
  using Leaf = LeafF64;
  double a0, b0;
  uint32_t L;

  __device__ __forceinline__ uint32_t leaf(uint64_t x) const {
    double v = floor(__fma_rn(a0, __ull2double_rn(x), b0));
    if (!(v >= 0.0)) return 0u;
    const uint32_t lm1 = L - 1u;
    return v >= (double)lm1 ? lm1 : (uint32_t)v;
  }
  __device__ __forceinline__ static int64_t pred(uint64_t x, uint64_t base, double a,
                                                 double b) {
    double d = x >= base ? __ull2double_rn(x - base) : -__ull2double_rn(base - x);
    double v = floor(__fma_rn(a, d, b));
    v = fmin(fmax(v, -kPredClampD), kPredClampD);
    return (int64_t)v;
  }
  __device__ __forceinline__ static Leaf load_leaf(const Leaf* leaves, uint32_t l) {
    const uint4* p = reinterpret_cast<const uint4*>(leaves + l);
    uint4 u0 = __ldg(p), u1 = __ldg(p + 1), u2 = __ldg(p + 2);
    Leaf r;
    r.base_key = (uint64_t)u0.x | ((uint64_t)u0.y << 32);
    r.lo = u0.z;
    r.hi = u0.w;
    r.a = __hiloint2double((int)u1.y, (int)u1.x);
    r.b = __hiloint2double((int)u1.w, (int)u1.z);
    r.e_lo = (int32_t)u2.x;
    r.e_hi = (int32_t)u2.y;
    r.pad = 0;
    return r;
  }
  __device__ __forceinline__ static int64_t pred(const Leaf& lf, uint64_t x) {
    return pred(x, lf.base_key, lf.a, lf.b);
  }
};

// Search window [wl, wh) of key x in leaf lf: the lower and the upper bound
// of x in R both lie in it (monotone models; the leaf owns [lo, hi)).
// pred_pos (optional) receives the predicted position clamped to [wl, wh).
template <class Model>
__device__ __forceinline__ void window(const typename Model::Leaf& lf, uint64_t x,
                                       uint32_t& wl, uint32_t& wh, uint32_t* pred_pos = nullptr) {
  const int64_t lo = lf.lo, hi = lf.hi;
  const int64_t p = lo + Model::pred(lf, x);
  int64_t a = p + lf.e_lo, b = p + (int64_t)lf.e_hi + 1;
  a = a < lo ? lo : (a > hi ? hi : a);
  b = b < lo ? lo : (b > hi ? hi : b);
  wl = (uint32_t)a;
  wh = (uint32_t)b;
  if (pred_pos) *pred_pos = (uint32_t)(p < a ? a : (p >= b ? (b > a ? b - 1 : a) : p));
}

// Predicted slot of key x in the gapped arrays of a GRMI (Section 3.A):
// (1 + gaps) times the leaf's predicted position clamped to the leaf's
// positions [lo, hi].  The build places R's keys and the probes start their
// searches with this one function, so both sides agree bit for bit.  It is
// monotone in x: the root and the leaf models are, and leaf ranges follow
// each other.
template <class Model>
__device__ __forceinline__ uint64_t clamped_pos(const typename Model::Leaf& lf, uint64_t x) {
  const int64_t lo = lf.lo, hi = lf.hi;
  int64_t p = lo + Model::pred(lf, x);
  p = p < lo ? lo : (p > hi ? hi : p);
  return (uint64_t)p;
}

template <class Model>
__device__ __forceinline__ uint64_t gapped_pslot(const typename Model::Leaf& lf, uint64_t x,
                                                 uint32_t scale) {
  return clamped_pos<Model>(lf, x) * scale;
}

// Slot functions of the two gapped layouts built by model-based insertion:
//   GappedSlot  GRMI (Section 3.A): (1 + gaps) slots per key of R
//   HashSlot    learned hash index (Section 3.C): the model as an
//               order-preserving hash into B buckets of 4 slots,
//               h(x) = p(x) * B / (n + 1), first slot 4 h(x)
struct GappedSlot {
  uint32_t scale;
  template <class Model>
  __device__ __forceinline__ uint64_t at(const typename Model::Leaf& lf, uint64_t x) const {
    return clamped_pos<Model>(lf, x) * scale;
  }
};
struct HashSlot {
  uint64_t B;    // buckets
  uint64_t n1;   // n + 1
  template <class Model>
  __device__ __forceinline__ uint64_t at(const typename Model::Leaf& lf, uint64_t x) const {
    return 4 * (clamped_pos<Model>(lf, x) * B / n1);
  }
};

__device__ __forceinline__ uint64_t ldg_key(const uint64_t* R, uint32_t i) {
  return __ldg(reinterpret_cast<const unsigned long long*>(R) + i);
}

// Streaming accesses (S and per-probe results, read or written once).
__device__ __forceinline__ ulonglong2 ldg_stream_u64x2(const uint64_t* p) {
  return __ldg(reinterpret_cast<const ulonglong2*>(p));
}
__device__ __forceinline__ void st_stream_u32x2(uint32_t* p, uint32_t a, uint32_t b) {
  *reinterpret_cast<uint2*>(p) = make_uint2(a, b);
}
__device__ __forceinline__ uint4 ldg_stream_u32x4(const uint32_t* p) {
  return __ldg(reinterpret_cast<const uint4*>(p));
}
__device__ __forceinline__ void st_stream_u64(uint64_t* p, uint64_t v) {
  *p = v;
}

// Four consecutive keys R[g .. g+3] with one 32-byte load (R + g 32-byte aligned).
__device__ __forceinline__ void ldg_key4(const uint64_t* R, uint32_t g, uint64_t (&k)[4]) {
  unsigned long long a, b, c, d;
  asm("ld.global.nc.v4.u64 {%0, %1, %2, %3}, [%4];"
      : "=l"(a), "=l"(b), "=l"(c), "=l"(d)
      : "l"(R + g));
  k[0] = a;
  k[1] = b;
  k[2] = c;
  k[3] = d;
}

// ------------------------------------------------------------ warp / block --

__device__ __forceinline__ uint64_t shfl_up64(uint64_t v, int d) {
  return __shfl_up_sync(0xffffffffu, (unsigned long long)v, d);
}

// Inclusive prefix sum over the warp.
__device__ __forceinline__ uint64_t warp_inclusive_sum(uint64_t v, int lane) {
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    uint64_t t = shfl_up64(v, d);
    if (lane >= d) v += t;
  }
  return v;
}

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_u64(uint64_t* p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// ------------------------------------------- single-pass decoupled look-back --
//
// Merrill and Garland, "Single-pass Parallel Prefix Scan with Decoupled
// Look-back" (2016).  Tile t publishes its aggregate, then walks back over
// its predecessors' published states until it meets an inclusive prefix.
// Tiles take their ids from an atomic ticket, so every predecessor of a
// running tile has already started and the walk finishes; the wait is still
// bounded (st.polls polls of a predecessor, by default kLookbackPolls; the
// option "lookback_polls" lowers it) and, if it ever runs out, the tile
// records kErrLookbackTimeout and continues with a zero prefix.

enum : uint32_t { kTileEmpty = 0, kTileAggregate = 1, kTilePrefix = 2 };

constexpr uint32_t kLookbackPolls = 1u << 20;   // default bound of one look-back wait

struct TileState {
  uint32_t* flag;     // [tiles], zeroed before the launch
  uint64_t* agg;      // [tiles]
  uint64_t* incl;     // [tiles]
  uint32_t* ticket;   // 1 counter, zeroed before the launch
  uint32_t polls = kLookbackPolls;   // polls of one predecessor before giving up
};

// Called by all 32 lanes of one warp.  Returns the exclusive prefix of tile t.
__device__ __forceinline__ uint64_t lookback_warp(const TileState& st, uint32_t t,
                                                  uint64_t aggregate, uint32_t* err) {
  const int lane = threadIdx.x & 31;
  if (t == 0) {
    if (lane == 0) {
      st_relaxed_u64(st.incl, aggregate);
      st_release_u32(st.flag, kTilePrefix);
    }
    return 0;
  }
  if (lane == 0) {
    st_relaxed_u64(st.agg + t, aggregate);
    st_release_u32(st.flag + t, kTileAggregate);
  }
  uint64_t exclusive = 0;
  int64_t window_end = (int64_t)t - 1;   // highest predecessor not yet folded in
  uint32_t polls = 0;
  bool timed_out = false;
  while (true) {
    const int64_t pt = window_end - lane;
    uint32_t f = kTilePrefix;   // before tile 0: an inclusive prefix of zero
    if (pt >= 0) {
      f = ld_acquire_u32(st.flag + pt);
      while (f == kTileEmpty) {
        if (++polls > st.polls) {
          timed_out = true;
          break;
        }
        __nanosleep(32);
        f = ld_acquire_u32(st.flag + pt);
      }
    }
    if (__any_sync(0xffffffffu, timed_out)) {
      if (lane == 0) atomicOr(err, kErrLookbackTimeout);
      return 0;
    }
    uint64_t v = 0;
    if (pt >= 0) v = (f == kTilePrefix) ? ld_relaxed_u64(st.incl + pt) : ld_relaxed_u64(st.agg + pt);
    const uint32_t prefix_mask = __ballot_sync(0xffffffffu, f == kTilePrefix);
    if (prefix_mask) {
      const int first = __ffs(prefix_mask) - 1;   // nearest predecessor with a prefix
      uint64_t mine = lane <= first ? v : 0;
#pragma unroll
      for (int d = 16; d >= 1; d >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, d);
      exclusive += mine;
      break;
    }
    uint64_t sum = v;
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, d);
    exclusive += sum;
    window_end -= 32;
  }
  if (lane == 0) {
    st_relaxed_u64(st.incl + t, exclusive + aggregate);
    st_release_u32(st.flag + t, kTilePrefix);
  }
  return exclusive;
}

}  // namespace lj
