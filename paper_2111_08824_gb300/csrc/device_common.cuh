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


// Kinds of gapped lookup structure (lj_index::gkind): gapped RMI (Section
// 3.A), learned hash with the RMI as the hash, learned hash with a
// RadixSpline as the hash (Section 3.C).
enum { kGappedRmi = 0, kRmiHash = 1, kRsHash = 2 };

// Error word bits (sticky, per device).
constexpr uint32_t kErrLookbackTimeout = 1u;
constexpr uint32_t kErrCapacity = 2u;

// --------------------------------------------------------------- records --

// ------------------------------------------------------ floor + convert --
//
// floor of a model output converted to an integer in one instruction
// (cvt.rmi: round toward minus infinity; NaN gives 0, out-of-range values
// saturate).  The clamps that follow are integer operations, so a model
// evaluation issues no separate floor or min/max in floating point (on GB300
// the FP64 pipe is narrow: the double-precision model then needs three FP64
// instructions per evaluation: the key conversion, the fma and this one).
__device__ __forceinline__ int64_t floor_to_i64(double v) {
  long long r;
  asm("cvt.rmi.s64.f64 %0, %1;" : "=l"(r) : "d"(v));
  return r;
}
__device__ __forceinline__ int64_t floor_to_i64(float v) {
  long long r;
  asm("cvt.rmi.s64.f32 %0, %1;" : "=l"(r) : "f"(v));
  return r;
}
__device__ __forceinline__ int32_t floor_to_i32(float v) {
  int r;
  asm("cvt.rmi.s32.f32 %0, %1;" : "=r"(r) : "f"(v));
  return r;
}

constexpr int64_t kPredClamp = 1ll << 40;   // predictions are clamped to [-2^40, 2^40]

__device__ __forceinline__ int64_t clamp_pred(int64_t v) {
  return v < -kPredClamp ? -kPredClamp : (v > kPredClamp ? kPredClamp : v);
}

// ---------------------------------------------------------------- records --

// Leaf record, single-precision model: 32 bytes = one DRAM sector.
struct __align__(32) LeafF32 {
  uint64_t base_key;   // R[lo]
  uint32_t lo, hi;     // positions [lo, hi) owned by the leaf
  float a, b;          // pred = lo + floor(fmaf(a, x - base_key, b))
  int32_t e_lo, e_hi;  // min / max of (i - pred(R[i])) over the leaf
};
static_assert(sizeof(LeafF32) == 32, "LeafF32 must be one sector");

// Leaf record, double-precision model: 64 bytes = two aligned sectors, read
// with two 32-byte loads.
struct __align__(32) LeafF64 {
  uint64_t base_key;
  uint32_t lo, hi;
  double a, b;
  int32_t e_lo, e_hi;
  uint64_t pad[3];
};
static_assert(sizeof(LeafF64) == 64, "LeafF64 layout");

// ----------------------------------------------------------------- models --
//
// Root:  leaf(x) = clamp(floor(fma(a0, X, b0)), 0, L-1), X = x rounded to the
//        model precision.
// Leaf:  pred(x) = clamp(floor(fma(a, D, b)), -2^40, 2^40), D = x - base_key
//        as a signed value rounded to the model precision.
// The index build and the lookups evaluate these same functions.

struct ModelF32 {
  using Leaf = LeafF32;
  float a0, b0;
  uint32_t L;

  static __host__ __device__ ModelF32 make(float a0, float b0, uint32_t L) {
    return ModelF32{a0, b0, L};
  }
  __device__ __forceinline__ uint32_t leaf(uint64_t x) const {
    const int32_t v = floor_to_i32(__fmaf_rn(a0, __ull2float_rn(x), b0));
    return v <= 0 ? 0u : ((uint32_t)v >= L - 1u ? L - 1u : (uint32_t)v);
  }
  __device__ __forceinline__ static int64_t pred(uint64_t x, uint64_t base, float a,
                                                 float b) {
    const float d = x >= base ? __ull2float_rn(x - base) : -__ull2float_rn(base - x);
    return clamp_pred(floor_to_i64(__fmaf_rn(a, d, b)));
  }
  __device__ __forceinline__ static void set_params(Leaf& r, double a, double b) {
    r.a = (float)a;
    r.b = (float)b;
  }
  // deployed parameters of a double-precision fit
  __device__ __forceinline__ static int64_t pred_fit(uint64_t x, uint64_t base, double a,
                                                     double b) {
    return pred(x, base, (float)a, (float)b);
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

  static __host__ __device__ ModelF64 make(double a0, double b0, uint32_t L) {
    return ModelF64{a0, b0, L};
  }
  __device__ __forceinline__ uint32_t leaf(uint64_t x) const {
    const int64_t v = floor_to_i64(__fma_rn(a0, __ull2double_rn(x), b0));
    return v <= 0 ? 0u : (v >= (int64_t)L - 1 ? L - 1u : (uint32_t)v);
  }
  __device__ __forceinline__ static int64_t pred(uint64_t x, uint64_t base, double a,
                                                 double b) {
    const double d = x >= base ? __ull2double_rn(x - base) : -__ull2double_rn(base - x);
    return clamp_pred(floor_to_i64(__fma_rn(a, d, b)));
  }
  __device__ __forceinline__ static void set_params(Leaf& r, double a, double b) {
    r.a = a;
    r.b = b;
  }
  __device__ __forceinline__ static int64_t pred_fit(uint64_t x, uint64_t base, double a,
                                                     double b) {
    return pred(x, base, a, b);
  }
  // two 32-byte loads (the record is two aligned sectors)
  __device__ __forceinline__ static Leaf load_leaf(const Leaf* leaves, uint32_t l) {
    unsigned long long w0, w1, w2, w3, w4, w5, w6, w7;
    asm("ld.global.nc.v4.u64 {%0, %1, %2, %3}, [%4];"
        : "=l"(w0), "=l"(w1), "=l"(w2), "=l"(w3)
        : "l"(leaves + l));
    asm("ld.global.nc.v4.u64 {%0, %1, %2, %3}, [%4];"
        : "=l"(w4), "=l"(w5), "=l"(w6), "=l"(w7)
        : "l"(reinterpret_cast<const char*>(leaves + l) + 32));
    Leaf r;
    r.base_key = w0;
    r.lo = (uint32_t)w1;
    r.hi = (uint32_t)(w1 >> 32);
    r.a = __longlong_as_double((long long)w2);
    r.b = __longlong_as_double((long long)w3);
    r.e_lo = (int32_t)(uint32_t)w4;
    r.e_hi = (int32_t)(uint32_t)(w4 >> 32);
    r.pad[0] = w5;
    r.pad[1] = w6;
    r.pad[2] = w7;
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

// RadixSpline (Section 2.D) as used by the learned hash index (Section 3.C):
// spline points (sx[i], sy[i]) over the CDF of R's distinct keys, a radix
// table over the top bits of (key - sx[0]) of the spline points, and the
// interpolated position of a key.  rcp[i] = 1 / (sx[i+1] - sx[i]) in double
// only seeds the exact integer division.
struct RsDev {
  const uint64_t* sx;
  const uint32_t* sy;
  const double* rcp;
  const uint32_t* table;   // 2^rbits + 1 entries: spline points with prefix below b
  uint64_t kmin, kmax;     // sx[0], sx[S-1]
  uint64_t n;              // |R|: the prediction above the largest key
  uint32_t S;              // spline points
  uint32_t shift;          // prefix = (x - kmin) >> shift
};

// floor(num / den) for num = a * b (a < 2^64, b < 2^32) and a < den: a
// double-precision estimate corrected by exact 128-bit products.
__device__ __forceinline__ uint64_t muldiv_floor(uint64_t a, uint32_t b, uint64_t den, double rcp) {
  const unsigned __int128 num = (unsigned __int128)a * b;
  const double est = ((double)(uint64_t)(num >> 64) * 18446744073709551616.0 +
                      (double)(uint64_t)num) * rcp;
  uint64_t q = est > 0.0 ? (uint64_t)est : 0;
  if ((unsigned __int128)q * den > num) --q;                       // estimate one too high
  else if ((unsigned __int128)(q + 1) * den <= num) ++q;           // or one too low
  return q;
}

// Interpolated position of x: 0 below the smallest key, n above the largest,
// else y_i + floor((x - x_i)(y_{i+1} - y_i) / (x_{i+1} - x_i)) between the
// spline points around x (found through the radix table).
__device__ __forceinline__ uint64_t rs_predict(const RsDev& rs, uint64_t x) {
  if (rs.S == 0 || x < rs.kmin) return 0;
  if (x > rs.kmax) return rs.n;
  const uint32_t b = (uint32_t)((x - rs.kmin) >> rs.shift);
  uint32_t lo = __ldg(rs.table + b), len = __ldg(rs.table + b + 1) - lo;
  // count the spline points <= x among those with x's prefix
  while (len > 0) {
    const uint32_t half = len >> 1;
    if (__ldg(reinterpret_cast<const unsigned long long*>(rs.sx) + lo + half) <= x) {
      lo += half + 1;
      len -= half + 1;
    } else {
      len = half;
    }
  }
  const uint32_t i = lo - 1;   // the last spline point <= x (exists: sx[0] = kmin <= x)
  const uint64_t x0 = __ldg(reinterpret_cast<const unsigned long long*>(rs.sx) + i);
  const uint32_t y0 = __ldg(rs.sy + i);
  if (x == x0 || i + 1 == rs.S) return y0;
  const uint64_t x1 = __ldg(reinterpret_cast<const unsigned long long*>(rs.sx) + i + 1);
  const uint32_t y1 = __ldg(rs.sy + i + 1);
  return y0 + muldiv_floor(x - x0, y1 - y0, x1 - x0, __ldg(rs.rcp + i));
}

// Learned hash with the RadixSpline as the hash: first slot 4 h(x),
// h(x) = pred(x) * B / (n + 1).
struct RsHashSlot {
  RsDev rs;
  uint64_t B, n1;
  __device__ __forceinline__ uint64_t at(uint64_t x) const { return 4 * (rs_predict(rs, x) * B / n1); }
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
