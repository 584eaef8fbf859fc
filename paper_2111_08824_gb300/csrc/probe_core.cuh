// Device code shared by the probe paths (single join, batched joins):
// tunables, probe parameters, the interleaved bounded search of the learned
// lookup (Section 2.D of Sabek and Kraska, "The Case for Learned In-Memory
// Joins": root -> leaf -> predicted position -> binary search between the
// leaf's error bounds) and the scan of per-tile match counts.
#pragma once

#include <cstdint>

#include "device_common.cuh"
#include "internal.h"

namespace lj {
namespace {   // internal linkage: each translation unit keeps its own copy

constexpr int kBlock = 256;
constexpr int kWarps = kBlock / 32;
enum { kUniqueEmit = 0, kUniqueCount = 1, kDupCount = 2 };

template <class Model>
struct ProbeParams {
  const uint64_t* R;
  uint32_t n;            // |R|
  bool r32;              // R is 32-byte aligned (4-key sector loads allowed)
  const typename Model::Leaf* leaves;
  Model model;
  const uint64_t* S;
  uint64_t m;
  lj_pair* pairs;
  uint64_t capacity;
  uint32_t* counts;      // optional
  uint32_t* first;       // optional: first matching position per probe (join_locate)
  uint64_t* offsets;     // optional, m + 1
  uint64_t* total_out;   // optional, device
  uint64_t* total_ws;    // workspace copy of the total
  uint32_t s_base;       // added to s_idx (chunked host joins)
  TileState st;
  uint32_t* err;
  uint32_t num_tiles;
  uint32_t tile_skip;     // single-pass kernel: tile ids start here (fault-injection hook; 0)
  uint32_t tile_shift;    // pipeline: log2 of the probes per compaction tile
  // gapped arrays of a GRMI (Section 3.A); gkeys == nullptr: plain RMI lookup
  const uint64_t* gkeys;
  const uint32_t* gpos;   // gslots + 1 payloads (positions in R)
  uint32_t gslots;        // C
  uint32_t gscale;        // 1 + gaps
  // learned hash index (Section 3.C): payload = distinct-key rank d,
  // matches of d = [dfirst[d], dfirst[d+1])
  const uint32_t* dfirst;
  const uint64_t* hrange; // per slot: first | count << 32 of the slot's entry (count 0: none)
  uint32_t ndistinct;     // D
  uint64_t hB;            // buckets
  uint64_t hn1;           // n + 1
  RsDev rs;               // RadixSpline of the learned hash over it (kind kRsHash)
  // key levels of R (search_levels): level k >= 1 holds R[4^k i] at
  // levels + lev_off[k]; nlev levels (0: none)
  const uint64_t* levels;
  uint32_t nlev;
  uint32_t lev_off[kMaxLevels + 1];
};

// Tunables (fixed at compile time; the defaults are the measured best).
#ifndef LJ_ROUNDS
#define LJ_ROUNDS 4        // probe rounds per thread (2 probes each)
#endif
#ifndef LJ_MINB
#define LJ_MINB 1          // min resident blocks per SM requested from ptxas
#endif
#ifndef LJ_SCHUNK
#define LJ_SCHUNK 1        // search kernel: tiles of 2*LJ_SBLOCK probes per block (1 measured best)
#endif
#ifndef LJ_SBLOCK
#define LJ_SBLOCK 128      // search kernel: threads per block
#endif
#ifndef LJ_SMINB
#define LJ_SMINB 16        // search kernel: 16 blocks of 128 threads per SM (32 registers,
                           // full occupancy): measured 9% faster than the unconstrained build
#endif
#ifndef LJ_LMINB
#define LJ_LMINB 10        // key-level search kernel: 10 blocks of 128 threads per SM (51
                           // registers: measured best against 12 and 16 on dup_seqh_50m)
#endif
#ifndef LJ_FMINB
#define LJ_FMINB 4         // fused small-batch kernel: 4 blocks of 256 threads per SM (64
                           // registers; fewer registers spill its lookup loop)
#endif
#ifndef LJ_GROUP4
#define LJ_GROUP4 true     // duplicates: halving over aligned 4-key groups + one 32-byte load
                           // (measured 11% faster on the duplicate workload, whose search
                           // is DRAM-bound; 7% slower on unique lognormal keys, where the
                           // bisection stays in use)
#endif
constexpr int kRounds = LJ_ROUNDS;
constexpr int kSearchChunk = LJ_SCHUNK;
constexpr int kSearchBlock = LJ_SBLOCK;
constexpr uint32_t kNoMatch = 0xFFFFFFFFu;
enum { kScanPairs = 0, kScanOffsets = 1 };
constexpr int kScanItems = 16;
constexpr uint64_t kCompactTile = 256ull * kScanItems;   // probes per compaction tile (large batches)
constexpr int kSmallScanItems = 4;                       // small batches: tiles of 1024 probes
constexpr uint64_t kSmallBatch = 1ull << 22;             // batches up to this size use them

// Interleaved bounded searches over NP windows.  For each probe p with
// window [base, base+len): finds c = the last position whose key is < x
// (STRICT) or <= x (!STRICT), and returns res = c + 1 (so the lower bound,
// resp. the upper bound, of x) and cv = R[c] when res > window start.
// Branch-free halving, the NP searches' loads issued together each round.
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

// Bounded search on 4-key groups (same contract as search_last; R 32-byte
// aligned): the window is widened to whole aligned groups of 4 keys, the
// halving runs over the groups' first keys, and the last group is read with
// one 32-byte load (one sector) instead of two more halving steps.  The
// widening is exact: every key left of the window is below x's lower bound
// and every key right of it above its upper bound.  Keys at or past n count
// as +infinity.
template <int NP, bool STRICT>
__device__ __forceinline__ void search_last_g4(const uint64_t* __restrict__ R, uint32_t n,
                                               const uint64_t (&x)[NP], uint32_t (&base)[NP],
                                               uint32_t (&len)[NP], uint64_t (&cv)[NP]) {
  uint32_t start[NP], g[NP], cnt[NP];
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    start[p] = base[p];
    cv[p] = 0;
    g[p] = base[p] >> 2;
    cnt[p] = len[p] ? ((base[p] + len[p] + 3) >> 2) - g[p] : 0;
  }
  while (true) {   // last group whose first key passes
    bool any = false;
    uint64_t v[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p)
      if (cnt[p] > 1) {
        any = true;
        v[p] = ldg_key(R, (g[p] + (cnt[p] >> 1)) << 2);
      }
    if (!any) break;
#pragma unroll
    for (int p = 0; p < NP; ++p)
      if (cnt[p] > 1) {
        const uint32_t half = cnt[p] >> 1;
        if (STRICT ? (v[p] < x[p]) : (v[p] <= x[p])) g[p] += half;
        cnt[p] -= half;
      }
  }
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    uint32_t res = start[p];
    if (cnt[p]) {
      const uint32_t q = g[p] << 2;
      uint64_t k[4];
      if (q + 4 <= n) {
        ldg_key4(R, q, k);
      } else {
#pragma unroll
        for (int i = 0; i < 4; ++i) k[i] = q + i < n ? ldg_key(R, q + i) : ~0ull;
      }
      uint32_t c = 0;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const bool go = (q + i < n) && (STRICT ? (k[i] < x[p]) : (k[i] <= x[p]));
        if (go) {
          c = i + 1;
          cv[p] = k[i];
        }
      }
      res = q + c;
      if (res < start[p]) res = start[p];   // nothing passed inside the window
    }
    base[p] = res;
    len[p] = start[p];
  }
}

// Bounded search by descending the key levels of R, a static 4-ary tree of
// fence keys over the sorted keys: level 0 is R itself, level k holds
// R[4^k i], so node b of level k (entries 4b .. 4b + 3, one 32-byte load)
// splits the block of positions [b 4^(k+1), (b + 1) 4^(k+1)) into its four
// children.  Same contract as search_last: the wanted position (the first
// key >= x when STRICT, > x otherwise) lies in [base, base + len].  The
// descent starts at the lowest level whose block holds both the position
// before the window and the window's last position (so the last passing key
// is in that block), takes in each node the last child whose first key
// passes, and ends with one sector of R: about log4 of the window's width
// plus one loads, against log2 for halving.  Entries at positions >= n
// never pass.  lev_off[k] = offset of level k in `lev`.
template <int NP, bool STRICT, class P_>
__device__ __forceinline__ void search_levels(const P_& P, const uint64_t (&x)[NP],
                                              uint32_t (&base)[NP], uint32_t (&len)[NP],
                                              uint64_t (&cv)[NP]) {
  const uint32_t n = P.n;
  uint32_t start[NP], blk[NP];
  int lvl[NP];
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    start[p] = base[p];
    cv[p] = 0;
    lvl[p] = -1;   // done
    blk[p] = 0;
    if (len[p] > 0) {
      const uint32_t lo = base[p] ? base[p] - 1 : 0, hi = base[p] + len[p] - 1;
      const uint32_t d = lo ^ hi;
      lvl[p] = d ? (31 - __clz(d)) >> 1 : 0;
      blk[p] = (uint32_t)((uint64_t)hi >> (2 * lvl[p] + 2));
    }
  }
  while (true) {
    bool any = false;
    uint64_t k[NP][4];
#pragma unroll
    for (int p = 0; p < NP; ++p)
      if (lvl[p] >= 0) {
        any = true;
        const uint64_t e = 4ull * blk[p];   // first entry of the node in its level
        if (lvl[p] > 0) {
          ldg_key4(P.levels + P.lev_off[lvl[p]], (uint32_t)e, k[p]);   // levels are padded
        } else if (P.r32 && e + 4 <= n) {
          ldg_key4(P.R, (uint32_t)e, k[p]);
        } else {
#pragma unroll
          for (int c = 0; c < 4; ++c) k[p][c] = e + c < n ? ldg_key(P.R, (uint32_t)(e + c)) : 0;
        }
      }
    if (!any) break;
#pragma unroll
    for (int p = 0; p < NP; ++p)
      if (lvl[p] >= 0) {
        const uint64_t pos0 = (uint64_t)blk[p] << (2 * lvl[p] + 2);   // position of entry 0
        const uint64_t step = 1ull << (2 * lvl[p]);
        uint32_t t = 0;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const bool pass = pos0 + c * step < n && (STRICT ? k[p][c] < x[p] : k[p][c] <= x[p]);
          t += pass ? 1u : 0u;
        }
        if (lvl[p] == 0) {
          base[p] = (uint32_t)pos0 + t;
          cv[p] = t == 1 ? k[p][0] : t == 2 ? k[p][1] : t == 3 ? k[p][2] : t == 4 ? k[p][3] : 0;
          lvl[p] = -1;
        } else if (t == 0) {   // nothing in the block passes (its start is position 0)
          base[p] = (uint32_t)pos0;
          lvl[p] = -1;
        } else {
          blk[p] = 4 * blk[p] + t - 1;
          --lvl[p];
        }
      }
  }
#pragma unroll
  for (int p = 0; p < NP; ++p) len[p] = start[p];
}

// Exponential search of a GRMI (Section 3.A), NP probes interleaved: for
// each probe p the first slot s >= pos[p] of the sorted gapped key array K
// (C slots) with K[s] >= x[p] (STRICT: K[s] > x[p]), or C.  Keys at pos,
// pos+1, pos+3, pos+7, ... until one passes, then a binary search in the
// last stretch.  pos[p] receives s and val[p] = K[s] (when s < C).  No key
// that passes lies before the predicted slot, so the search only moves to
// later slots.
template <int NP, bool STRICT>
__device__ __forceinline__ void gallop_first(const uint64_t* __restrict__ K, uint32_t C,
                                             const uint64_t (&x)[NP], uint32_t (&pos)[NP],
                                             uint64_t (&val)[NP]) {
  uint32_t lo[NP], hi[NP], off[NP];
  bool open[NP];
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    lo[p] = pos[p];
    hi[p] = C;
    off[p] = 0;
    open[p] = pos[p] < C;
    val[p] = 0;
  }
  while (true) {   // exponential phase
    bool any = false;
    uint32_t t[NP];
    uint64_t v[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p)
      if (open[p]) {
        const uint64_t tt = (uint64_t)pos[p] + off[p];
        if (tt >= C) {
          open[p] = false;
        } else {
          t[p] = (uint32_t)tt;
          v[p] = ldg_key(K, t[p]);
          any = true;
        }
      }
    if (!any) break;
#pragma unroll
    for (int p = 0; p < NP; ++p)
      if (open[p]) {
        const bool pass = STRICT ? v[p] > x[p] : v[p] >= x[p];
        if (pass) {
          hi[p] = t[p];
          val[p] = v[p];
          open[p] = false;
        } else {
          lo[p] = t[p] + 1;
          off[p] = 2 * off[p] + 1;
        }
      }
  }
  uint32_t len[NP];
#pragma unroll
  for (int p = 0; p < NP; ++p) len[p] = hi[p] - lo[p];
  while (true) {   // binary search in [lo, hi)
    bool any = false;
    uint64_t v[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p)
      if (len[p] > 0) {
        any = true;
        v[p] = ldg_key(K, lo[p] + (len[p] >> 1));
      }
    if (!any) break;
#pragma unroll
    for (int p = 0; p < NP; ++p)
      if (len[p] > 0) {
        const uint32_t half = len[p] >> 1;
        const bool pass = STRICT ? v[p] > x[p] : v[p] >= x[p];
        if (pass) {
          val[p] = v[p];
          len[p] = half;
        } else {
          lo[p] += half + 1;
          len[p] -= half + 1;
        }
      }
  }
#pragma unroll
  for (int p = 0; p < NP; ++p) pos[p] = lo[p];
}

// Predicted slot of x, at most C: the gapped RMI's, or the first slot of
// x's bucket in the learned hash table (RMI or RadixSpline as the hash).
// The leaf record is not used by the RadixSpline hash.
template <class Model, int KIND = kGappedRmi>
__device__ __forceinline__ uint32_t gapped_start(const ProbeParams<Model>& P,
                                                 const typename Model::Leaf& lf, uint64_t x) {
  const uint64_t q = KIND == kRsHash    ? RsHashSlot{P.rs, P.hB, P.hn1}.at(x)
                     : KIND == kRmiHash ? HashSlot{P.hB, P.hn1}.template at<Model>(lf, x)
                                        : gapped_pslot<Model>(lf, x, P.gscale);
  return q < P.gslots ? (uint32_t)q : P.gslots;
}

// GRMI lookups of the two probes j0, j0 + 1 (Section 3.A): root -> leaf ->
// predicted slot -> exponential search for the first slot holding a key
// >= x; its payload is the lower bound of x in R.  With duplicates a second
// search from there finds the first key > x, and cnt is the difference of
// the two payloads.
template <class Model, int MODE, bool VEC, int KIND = kGappedRmi>
__device__ __forceinline__ void lookup_gapped(const ProbeParams<Model>& P, uint64_t j0,
                                              uint32_t (&r_idx)[2], uint32_t (&cnt)[2],
                                              bool (&valid)[2]) {
  uint64_t x[2];
  if (VEC && j0 + 1 < P.m) {
    const ulonglong2 v = ldg_stream_u64x2(P.S + j0);
    x[0] = v.x;
    x[1] = v.y;
    valid[0] = valid[1] = true;
  } else {
    valid[0] = j0 < P.m;
    valid[1] = j0 + 1 < P.m;
    x[0] = valid[0] ? __ldg(reinterpret_cast<const unsigned long long*>(P.S) + j0) : 0;
    x[1] = valid[1] ? __ldg(reinterpret_cast<const unsigned long long*>(P.S) + j0 + 1) : 0;
  }
  uint32_t pos[2];
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    pos[p] = P.gslots;
    if (valid[p]) {
      if (KIND == kRsHash)   // the RadixSpline needs no leaf record
        pos[p] = gapped_start<Model, KIND>(P, typename Model::Leaf{}, x[p]);
      else
        pos[p] = gapped_start<Model, KIND>(P, Model::load_leaf(P.leaves, P.model.leaf(x[p])), x[p]);
    }
  }
  uint64_t val[2];
  gallop_first<2, false>(P.gkeys, P.gslots, x, pos, val);
  bool hit[2];
#pragma unroll
  for (int p = 0; p < 2; ++p) hit[p] = valid[p] && pos[p] < P.gslots && val[p] == x[p];
  if (KIND != kGappedRmi) {
    // one 8-byte load gives the slot's whole range of matches (the copies
    // after the last key carry count 0: no match)
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      const uint64_t rg = hit[p] ? __ldg(reinterpret_cast<const unsigned long long*>(P.hrange) + pos[p])
                                 : 0ull;
      const uint32_t c = (uint32_t)(rg >> 32);
      cnt[p] = MODE == kDupCount ? c : (c ? 1u : 0u);
      r_idx[p] = (uint32_t)rg;
    }
  } else if (MODE == kDupCount) {
    uint32_t ub[2] = {hit[0] ? pos[0] : P.gslots, hit[1] ? pos[1] : P.gslots};
    uint64_t v2[2];
    gallop_first<2, true>(P.gkeys, P.gslots, x, ub, v2);
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      const uint32_t a = hit[p] ? __ldg(P.gpos + pos[p]) : 0u;
      const uint32_t b = hit[p] ? __ldg(P.gpos + ub[p]) : 0u;
      cnt[p] = b - a;
      r_idx[p] = a;
    }
  } else {
    // slots after R's last key hold 2^64-1 with payload n: a probe 2^64-1
    // that is not in R lands there, so a match also needs a payload below n
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      const uint32_t r = hit[p] ? __ldg(P.gpos + pos[p]) : P.n;
      cnt[p] = r < P.n ? 1u : 0u;
      r_idx[p] = r;
    }
  }
}

// Lookups of NP keys already loaded (x, valid): root -> leaf record ->
// window, then the interleaved bounded searches; cnt = number of matches,
// r_idx = first matching position (when cnt > 0).  SEARCH selects the
// bounded search: kSearchHalve (halving; duplicates on 4-key groups when
// LJ_GROUP4), kSearchGroups (halving over 4-key groups for unique keys too:
// about two dependent loads fewer on small windows), kSearchLevels (descent
// of the key levels, when the index has them).
enum { kSearchHalve = 0, kSearchGroups = 1, kSearchLevels = 2 };
template <class Model, int MODE, int NP, int SEARCH = kSearchHalve>
__device__ __forceinline__ void lookup_keys(const ProbeParams<Model>& P, const uint64_t (&x)[NP],
                                            const bool (&valid)[NP], uint32_t (&r_idx)[NP],
                                            uint32_t (&cnt)[NP]) {
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
  if (MODE == kDupCount) {
    uint32_t wh[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) wh[p] = base[p] + len[p];
    uint64_t cv[NP];
    if (SEARCH == kSearchLevels)
      search_levels<NP, true>(P, x, base, len, cv);            // base = lower bound
    else if (LJ_GROUP4 && P.r32)
      search_last_g4<NP, true>(P.R, P.n, x, base, len, cv);   // base = lower bound
    else
      search_last<NP, true>(P.R, x, base, len, cv);            // base = lower bound
    uint32_t lb[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      lb[p] = base[p];
      len[p] = wh[p] - base[p];
    }
    if (SEARCH == kSearchLevels)
      search_levels<NP, false>(P, x, base, len, cv);           // base = upper bound
    else if (LJ_GROUP4 && P.r32)
      search_last_g4<NP, false>(P.R, P.n, x, base, len, cv);  // base = upper bound
    else
      search_last<NP, false>(P.R, x, base, len, cv);           // base = upper bound
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      cnt[p] = valid[p] ? base[p] - lb[p] : 0;
      r_idx[p] = lb[p];
    }
  } else {
    uint64_t cv[NP];
    if (SEARCH == kSearchLevels)
      search_levels<NP, false>(P, x, base, len, cv);          // base = upper bound, len = start
    else if (SEARCH == kSearchGroups && P.r32)
      search_last_g4<NP, false>(P.R, P.n, x, base, len, cv);  // base = upper bound, len = start
    else
      search_last<NP, false>(P.R, x, base, len, cv);          // base = upper bound, len = start
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      const bool match = valid[p] && base[p] > len[p] && cv[p] == x[p];
      cnt[p] = match ? 1u : 0u;
      r_idx[p] = base[p] - 1;
    }
  }
}

// Lookups of 2K probes per thread: round k covers probes
// j0 = first + 2*stride*k + {0, 1} (one 16-byte load of two keys).  Root ->
// leaf record -> window, then the interleaved bounded searches.  cnt is the
// number of matches, r_idx the first matching position (when cnt > 0).
template <class Model, int MODE, int K, bool VEC, int SEARCH = kSearchHalve>
__device__ __forceinline__ void lookup_probes(const ProbeParams<Model>& P, uint64_t first,
                                              uint32_t stride, uint32_t (&r_idx)[2 * K],
                                              uint32_t (&cnt)[2 * K], bool (&valid)[2 * K]) {
  constexpr int NP = 2 * K;
  uint64_t x[NP];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const uint64_t j0 = first + 2ull * stride * k;
    if (VEC && j0 + 1 < P.m) {
      const ulonglong2 v = ldg_stream_u64x2(P.S + j0);
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
  lookup_keys<Model, MODE, NP, SEARCH>(P, x, valid, r_idx, cnt);
}

// Exclusive scan of the per-tile counts: blocks of 256 threads x 16 counts
// with a decoupled look-back between blocks (a few hundred at most).
// prefix[t] = first output position of tile t, prefix[tiles] = |J|; the last
// block also publishes the total.
constexpr int kTileScanItems = 16;
constexpr uint32_t kTileScanSpan = kBlock * kTileScanItems;

__global__ void __launch_bounds__(kBlock) tile_scan_kernel(const unsigned long long* counts,
                                                           uint32_t tiles, uint64_t* prefix,
                                                           TileState st, uint32_t blocks,
                                                           uint64_t* total_ws, uint64_t* total_out,
                                                           uint64_t* offsets_end, uint64_t capacity,
                                                           uint32_t* err) {
  __shared__ uint32_t s_blk;
  __shared__ uint64_t s_warp[kWarps];
  __shared__ uint64_t s_prefix;
  if (threadIdx.x == 0) s_blk = atomicAdd(st.ticket, 1u);
  __syncthreads();
  const uint32_t blk = s_blk;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint64_t base = (uint64_t)blk * kTileScanSpan + (uint64_t)threadIdx.x * kTileScanItems;
  uint64_t v[kTileScanItems];
  uint64_t sum = 0;
#pragma unroll
  for (int i = 0; i < kTileScanItems; ++i) {
    v[i] = base + i < tiles ? counts[base + i] : 0;
    sum += v[i];
  }
  const uint64_t inc = warp_inclusive_sum(sum, lane);
  if (lane == 31) s_warp[w] = inc;
  __syncthreads();
  if (w == 0) {
    const uint64_t x = lane < kWarps ? s_warp[lane] : 0;
    const uint64_t xi = warp_inclusive_sum(x, lane);
    if (lane < kWarps) s_warp[lane] = xi - x;
    const uint64_t agg = __shfl_sync(0xffffffffu, xi, 31);
    const uint64_t pre = lookback_warp(st, blk, agg, err);
    if (lane == 0) {
      s_prefix = pre;
      if (blk + 1 == blocks) {
        const uint64_t total = pre + agg;
        prefix[tiles] = total;
        *total_ws = total;
        if (total_out) *total_out = total;
        if (offsets_end) *offsets_end = total;
        if (total > capacity) atomicOr(err, kErrCapacity);
      }
    }
  }
  __syncthreads();
  uint64_t run = s_prefix + s_warp[w] + inc - sum;
#pragma unroll
  for (int i = 0; i < kTileScanItems; ++i) {
    if (base + i < tiles) prefix[base + i] = run;
    run += v[i];
  }
}

}  // namespace
}  // namespace lj
