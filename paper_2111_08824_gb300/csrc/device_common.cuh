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

// ------------------------------------------- conversions without FP64 --
//
// On GB300 the FP64 pipe runs at a small fraction of the FP32 rate, and
// conversions between 64-bit integers and floating point run on it too.
// The probe kernels therefore convert with integer instructions; the results
// are the correctly rounded values the conversion instructions would give.

// x * 2^e as a float, for a 24-bit significand m in [2^23, 2^24] (2^24: the
// carry of a rounding, folded into the exponent) and -149 < e + 23 < 128.
__device__ __forceinline__ float f32_from_sig(uint32_t m, int e) {
  return __uint_as_float(((uint32_t)(e + 149) << 23) + m);
}

// uint64 -> float, round to nearest even (as __ull2float_rn).
__device__ __forceinline__ float u64_to_f32_rn(uint64_t x) {
  if (x == 0) return 0.0f;
  const int lz = __clzll(x);
  const uint64_t y = x << lz;                       // leading one at bit 63
  uint32_t m = (uint32_t)(y >> 40);                 // 24-bit significand
  const uint64_t rest = y & ((1ull << 40) - 1);     // the 40 bits below it
  const uint64_t half = 1ull << 39;
  m += (rest > half || (rest == half && (m & 1u))) ? 1u : 0u;
  return f32_from_sig(m, 40 - lz);
}

// uint64 -> float, rounded toward zero; `val` receives the integer value of
// the result (x - val < 2^-23 x).
__device__ __forceinline__ float u64_to_f32_rz(uint64_t x, uint64_t& val) {
  if (x == 0) {
    val = 0;
    return 0.0f;
  }
  const int lz = __clzll(x);
  const uint32_t m = (uint32_t)((x << lz) >> 40);
  const int e = 40 - lz;
  val = e >= 0 ? (uint64_t)m << e : (uint64_t)(m >> -e);
  return f32_from_sig(m, e);
}

// uint64 as an unevaluated sum hi + lo of two floats, |x - hi - lo| < 2^-46 x.
__device__ __forceinline__ void u64_to_ff(uint64_t x, float& hi, float& lo) {
  uint64_t v, w;
  hi = u64_to_f32_rz(x, v);
  lo = u64_to_f32_rz(x - v, w);
}

// An integral float with |v| <= 2^40 (or +-0) as int64 (as a float -> int64
// conversion would give).
__device__ __forceinline__ int64_t f32_integral_to_i64(float v) {
  const uint32_t b = __float_as_uint(v);
  const uint32_t ef = (b >> 23) & 0xFFu;
  if (ef == 0) return 0;
  const int e = (int)ef - 150;                      // v = m * 2^e
  const uint64_t m = (uint64_t)((b & 0x7FFFFFu) | 0x800000u);
  const uint64_t mag = e >= 0 ? m << e : m >> -e;
  return (b >> 31) ? -(int64_t)mag : (int64_t)mag;
}

// floor(fma(a, D, b)) of the double-precision model, exactly, from float
// parts: a ~ ah + al, D ~ Dh + Dl, b ~ bh + bl (each pair within 2^-45 of
// the double it stands for).  The product and the sum are carried as an
// unevaluated float sum (exact product error by fmaf, TwoSum), whose error is
// below 2^-21 while |ah*Dh|, |bh| < 2^20.  Returns false (no answer) outside
// that range and when the value lies within 2^-20 of an integer: there the
// floor of the double-precision fma must be computed in double.  Explicit
// _rn intrinsics keep the compiler from contracting the error terms.
__device__ __forceinline__ bool ff_floor_fma(float ah, float al, float Dh, float Dl, float bh,
                                             float bl, int64_t& out) {
  constexpr float kLimit = 1048576.0f;               // 2^20
  constexpr float kMargin = 9.5367431640625e-07f;    // 2^-20
  const float p = __fmul_rn(ah, Dh);
  if (!(fabsf(p) < kLimit && fabsf(bh) < kLimit)) return false;
  const float pe = __fmaf_rn(ah, Dh, -p);            // ah*Dh - p, exact
  const float cross = __fmaf_rn(ah, Dl, __fmul_rn(al, Dh));
  const float s = __fadd_rn(p, bh);                  // TwoSum: s + se == p + bh
  const float bb = __fsub_rn(s, p);
  const float se = __fadd_rn(__fsub_rn(p, __fsub_rn(s, bb)), __fsub_rn(bh, bb));
  const float t = __fadd_rn(__fadd_rn(__fadd_rn(pe, cross), bl), se);
  const float k1 = floorf(s);
  const float u = __fsub_rn(s, k1);                  // TwoSum: u + ue == s - k1
  const float bv = __fsub_rn(u, s);
  const float ue = __fadd_rn(__fsub_rn(s, __fsub_rn(u, bv)), __fsub_rn(-k1, bv));
  const float f = __fadd_rn(u, __fadd_rn(ue, t));    // value - k1
  const float k2 = floorf(f);
  const float frac = __fsub_rn(f, k2);
  if (!(frac >= kMargin && frac <= 1.0f - kMargin)) return false;
  out = f32_integral_to_i64(k1) + f32_integral_to_i64(k2);
  return true;
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

// Leaf record, double-precision model: 64 bytes = two sectors.  The first
// holds what a lookup needs besides the bounds: the key base, the positions
// and the parameters as float pairs (ah + al ~ a, bh + bl ~ b) for the
// single-precision evaluation of the double-precision model; the second the
// error bounds and the parameters in double (for values near an integer).
struct __align__(32) LeafF64 {
  uint64_t base_key;
  uint32_t lo, hi;
  float ah, al, bh, bl;
  int32_t e_lo, e_hi;
  double a, b;
  uint64_t pad;
};
static_assert(sizeof(LeafF64) == 64, "LeafF64 layout");

// ----------------------------------------------------------------- models --
//
// leaf()/pred() are the lookups' evaluation (no FP64 instruction in the
// common case); leaf_exact()/pred_exact() evaluate the same formulas with the
// conversion and fma instructions of the model's precision and are used by
// the index build.  The two give identical integers for every input.

struct ModelF32 {
  using Leaf = LeafF32;
  float a0, b0;
  uint32_t L;
  float lm1f;          // L - 1 (exact: L <= 2^24)

  static __host__ __device__ ModelF32 make(float a0, float b0, uint32_t L) {
    return ModelF32{a0, b0, L, (float)(L - 1u)};
  }

  __device__ __forceinline__ uint32_t leaf(uint64_t x) const {
    const float v = floorf(__fmaf_rn(a0, u64_to_f32_rn(x), b0));
    if (!(v >= 0.0f)) return 0u;
    if (v >= lm1f) return L - 1u;
    return (uint32_t)f32_integral_to_i64(v);
  }
  __device__ __forceinline__ uint32_t leaf_exact(uint64_t x) const {
    float v = floorf(__fmaf_rn(a0, __ull2float_rn(x), b0));
    if (!(v >= 0.0f)) return 0u;
    const uint32_t lm1 = L - 1u;
    return v >= (float)lm1 ? lm1 : (uint32_t)v;
  }
  __device__ __forceinline__ static int64_t pred(uint64_t x, uint64_t base, float a,
                                                 float b) {
    const float d = x >= base ? u64_to_f32_rn(x - base) : -u64_to_f32_rn(base - x);
    float v = floorf(__fmaf_rn(a, d, b));
    v = fminf(fmaxf(v, -kPredClampF), kPredClampF);
    return f32_integral_to_i64(v);
  }
  __device__ __forceinline__ static int64_t pred_exact(uint64_t x, uint64_t base, double a,
                                                       double b) {
    const float d = x >= base ? __ull2float_rn(x - base) : -__ull2float_rn(base - x);
    float v = floorf(__fmaf_rn((float)a, d, (float)b));
    v = fminf(fmaxf(v, -kPredClampF), kPredClampF);
    return (int64_t)v;
  }
  __device__ __forceinline__ static void set_params(Leaf& r, double a, double b) {
    r.a = (float)a;
    r.b = (float)b;
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
  float a0h, a0l, b0h, b0l;   // a0 ~ a0h + a0l, b0 ~ b0h + b0l

  static __host__ __device__ ModelF64 make(double a0, double b0, uint32_t L) {
    const float ah = (float)a0, bh = (float)b0;
    return ModelF64{a0, b0, L, ah, (float)(a0 - (double)ah), bh, (float)(b0 - (double)bh)};
  }

  __device__ __forceinline__ uint32_t leaf(uint64_t x) const {
    float xh, xl;
    u64_to_ff(x, xh, xl);
    int64_t f;
    if (ff_floor_fma(a0h, a0l, xh, xl, b0h, b0l, f))
      return f < 0 ? 0u : (f >= (int64_t)L - 1 ? L - 1u : (uint32_t)f);
    return leaf_exact(x);
  }
  __device__ __forceinline__ uint32_t leaf_exact(uint64_t x) const {
    double v = floor(__fma_rn(a0, __ull2double_rn(x), b0));
    if (!(v >= 0.0)) return 0u;
    const uint32_t lm1 = L - 1u;
    return v >= (double)lm1 ? lm1 : (uint32_t)v;
  }
  __device__ __forceinline__ static int64_t pred_exact(uint64_t x, uint64_t base, double a,
                                                       double b) {
    double d = x >= base ? __ull2double_rn(x - base) : -__ull2double_rn(base - x);
    double v = floor(__fma_rn(a, d, b));
    v = fmin(fmax(v, -kPredClampD), kPredClampD);
    return (int64_t)v;
  }
  __device__ __forceinline__ static void set_params(Leaf& r, double a, double b) {
    r.a = a;
    r.b = b;
    r.ah = (float)a;
    r.al = (float)(a - (double)r.ah);
    r.bh = (float)b;
    r.bl = (float)(b - (double)r.bh);
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
    r.ah = __uint_as_float((uint32_t)w2);
    r.al = __uint_as_float((uint32_t)(w2 >> 32));
    r.bh = __uint_as_float((uint32_t)w3);
    r.bl = __uint_as_float((uint32_t)(w3 >> 32));
    r.e_lo = (int32_t)(uint32_t)w4;
    r.e_hi = (int32_t)(uint32_t)(w4 >> 32);
    r.a = __longlong_as_double((long long)w5);
    r.b = __longlong_as_double((long long)w6);
    r.pad = w7;
    return r;
  }
  __device__ __forceinline__ static int64_t pred(const Leaf& lf, uint64_t x) {
    const bool neg = x < lf.base_key;
    const uint64_t d = neg ? lf.base_key - x : x - lf.base_key;
    float Dh, Dl;
    u64_to_ff(d, Dh, Dl);
    if (neg) {
      Dh = -Dh;
      Dl = -Dl;
    }
    int64_t f;
    if (ff_floor_fma(lf.ah, lf.al, Dh, Dl, lf.bh, lf.bl, f)) return f;   // |f| < 2^21
    return pred_exact(x, lf.base_key, lf.a, lf.b);
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
