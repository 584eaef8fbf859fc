/*
 * CPU oracle for the learned indexed nested loop join (RMI-INLJ).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path links,
 * loads or calls this file; only the tests, the package's smoke check and
 * the benchmark's CPU baseline do.  It shares no code, header, table or
 * constant with the CUDA implementation.
 *
 * Plain, slow and written to be checked by eye against the paper
 * ("The Case for Learned In-Memory Joins", Sabek and Kraska):
 *
 *  1. lj_oracle_join_ranges / lj_oracle_join_pairs: the join result itself.
 *     Section 2.A defines the indexed nested loop join: for every tuple s of
 *     S, fetch the tuples of R with the same join key.  Section 6.B (the
 *     duplicates experiment) returns every match, so the result is the set
 *       J(R, S) = { (i, j) : R[i] == S[j] }.
 *     Computed by a sort-merge equi-join (sort S by (key, j), merge with the
 *     sorted R).  Because R is sorted, the matches of one probe j form one
 *     contiguous range [lo_j, hi_j) of R's positions.
 *
 *  2. lj_oracle_rmi_fit / lj_oracle_rmi_lookup: the two-level linear
 *     Recursive Model Index of Section 2.D ("Recursive Model Index"): a root
 *     linear model picks a leaf model, the leaf's linear model predicts a
 *     position, each leaf keeps the minimum and maximum error of its keys and
 *     a lookup binary-searches between those bounds.  The paper gives no
 *     formulas; the readings taken here are:
 *       root:  leaf(x) = clamp(floor(a0 * X + b0), 0, L-1), X = x rounded to
 *              the model's precision, (a0, b0) the least-squares line of
 *              i * L / n on R[i] (fit in double precision);
 *       leaf l owns the contiguous positions [lo_l, hi_l) of the keys the
 *              root sends to it; base key k_l = R[lo_l];
 *       leaf:  pred(x) = lo_l + floor(a_l * D + b_l), D = x - k_l as a signed
 *              quantity rounded to the model's precision, (a_l, b_l) the
 *              least-squares line of (i - lo_l) on (R[i] - k_l) over the
 *              leaf's keys (fit in double precision, slope kept >= 0);
 *       a*X+b is one fused multiply-add in the model's precision (fmaf for
 *              the single-precision model, fma for the double one);
 *       errors: err_i = i - pred(R[i]); e_lo = min, e_hi = max over the leaf;
 *       window: [clamp(pred+e_lo), clamp(pred+e_hi+1)] within [lo_l, hi_l].
 *
 * Compile with -ffp-contract=off so that no a*b+c outside the explicit
 * fma/fmaf calls is fused (the results must not depend on the host CPU).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- join -- */

typedef struct {
  uint64_t key;
  uint64_t j;
} probe_t;

static int cmp_probe(const void* a, const void* b) {
  const probe_t* x = (const probe_t*)a;
  const probe_t* y = (const probe_t*)b;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  if (x->j != y->j) return x->j < y->j ? -1 : 1;
  return 0;
}

/* 1 if R is sorted non-decreasing, else 0. */
int lj_oracle_is_sorted(const uint64_t* R, uint64_t n) {
  for (uint64_t i = 1; i < n; ++i)
    if (R[i - 1] > R[i]) return 0;
  return 1;
}

/*
 * For every probe j, the range [lo[j], hi[j]) of positions i with
 * R[i] == S[j] (lo[j] == hi[j] when S[j] has no match; the value is then
 * the number of keys of R below S[j]).  Returns |J| = sum (hi - lo), -1 if R
 * is not sorted, -2 if memory runs out.
 */
int64_t lj_oracle_join_ranges(const uint64_t* R, uint64_t n, const uint64_t* S,
                              uint64_t m, uint64_t* lo, uint64_t* hi) {
  if (!lj_oracle_is_sorted(R, n)) return -1;
  if (m == 0) return 0;
  probe_t* P = (probe_t*)malloc(sizeof(probe_t) * m);
  if (!P) return -2;
  for (uint64_t j = 0; j < m; ++j) {
    P[j].key = S[j];
    P[j].j = j;
  }
  qsort(P, m, sizeof(probe_t), cmp_probe);

  int64_t total = 0;
  uint64_t i = 0; /* first position of R whose key is >= the current probe key */
  uint64_t k = 0;
  while (k < m) {
    uint64_t key = P[k].key;
    while (i < n && R[i] < key) ++i;
    uint64_t a = i, b = i;
    while (b < n && R[b] == key) ++b;
    /* every probe carrying this key gets the whole run [a, b) */
    while (k < m && P[k].key == key) {
      lo[P[k].j] = a;
      hi[P[k].j] = b;
      total += (int64_t)(b - a);
      ++k;
    }
  }
  free(P);
  return total;
}

/*
 * The join as (r_idx, s_idx) pairs in canonical order: s_idx ascending,
 * r_idx ascending within one probe.  pairs holds 2*cap uint32 values
 * (r, s interleaved).  Returns |J| (which may exceed cap: only the first cap
 * pairs are written), -1 if R is not sorted, -2 if memory runs out.
 */
int64_t lj_oracle_join_pairs(const uint64_t* R, uint64_t n, const uint64_t* S,
                             uint64_t m, uint32_t* pairs, uint64_t cap) {
  if (m == 0) return lj_oracle_is_sorted(R, n) ? 0 : -1;
  uint64_t* lo = (uint64_t*)malloc(sizeof(uint64_t) * m);
  uint64_t* hi = (uint64_t*)malloc(sizeof(uint64_t) * m);
  if (!lo || !hi) {
    free(lo);
    free(hi);
    return -2;
  }
  int64_t total = lj_oracle_join_ranges(R, n, S, m, lo, hi);
  if (total >= 0) {
    uint64_t q = 0;
    for (uint64_t j = 0; j < m && q < cap; ++j)
      for (uint64_t r = lo[j]; r < hi[j] && q < cap; ++r, ++q) {
        pairs[2 * q] = (uint32_t)r;
        pairs[2 * q + 1] = (uint32_t)j;
      }
  }
  free(lo);
  free(hi);
  return total;
}

/* ----------------------------------------------------------------- RMI -- */

/* Least-squares line y = a*x + b by centred two-pass sums (double). */
static void lsq_fit(const double* x, const double* y, uint64_t k, double* a,
                    double* b) {
  if (k == 0) {
    *a = 0.0;
    *b = 0.0;
    return;
  }
  double sx = 0.0, sy = 0.0;
  for (uint64_t t = 0; t < k; ++t) {
    sx += x[t];
    sy += y[t];
  }
  double mx = sx / (double)k, my = sy / (double)k;
  double sxy = 0.0, sxx = 0.0;
  for (uint64_t t = 0; t < k; ++t) {
    double dx = x[t] - mx, dy = y[t] - my;
    sxy += dx * dy;
    sxx += dx * dx;
  }
  double slope = sxx > 0.0 ? sxy / sxx : 0.0;
  if (!(slope > 0.0)) slope = 0.0; /* sorted keys: the slope is never negative */
  *a = slope;
  *b = my - slope * mx;
}

/* Deployed parameter: rounded to float for the single-precision model. */
static double deploy(double v, int fp64) { return fp64 ? v : (double)(float)v; }

/* floor of the model output clamped to [-2^40, 2^40], as an integer. */
static int64_t clamp_floor(double v) {
  v = floor(v);
  if (v < -1099511627776.0) v = -1099511627776.0;
  if (v > 1099511627776.0) v = 1099511627776.0;
  return (int64_t)v;
}

/* Root model: which leaf serves key x. */
static uint32_t root_leaf(uint64_t x, double a0, double b0, uint32_t L, int fp64) {
  double v;
  if (fp64)
    v = fma(a0, (double)x, b0);
  else
    v = (double)fmaf((float)a0, (float)x, (float)b0);
  v = floor(v);
  if (!(v >= 0.0)) return 0; /* also catches NaN */
  if (v >= (double)(L - 1)) return L - 1;
  return (uint32_t)v;
}

/* Leaf model: predicted offset of key x from the leaf's first position. */
static int64_t leaf_pred(uint64_t x, uint64_t base, double a, double b, int fp64) {
  double v;
  if (fp64) {
    double d = x >= base ? (double)(x - base) : -(double)(base - x);
    v = fma(a, d, b);
  } else {
    float d = x >= base ? (float)(x - base) : -(float)(base - x);
    v = (double)fmaf((float)a, d, (float)b);
  }
  return clamp_floor(v);
}

/*
 * Fit the two-level RMI over sorted R (n keys) with L leaves.
 *   root_fit[2]  = (a0, b0) least-squares fit (double)
 *   root_dep[2]  = deployed (a0, b0) (float-rounded for fp64 == 0)
 *   leaf_lo[L+1] = first position of each leaf; leaf_lo[L] = n
 *   leaf_fit[2L] = per-leaf (a, b) least-squares fit (double)
 *   leaf_dep[2L] = deployed per-leaf (a, b)
 *   err[2L]      = per-leaf (e_lo, e_hi); (0, 0) for an empty leaf
 * Returns 0, -1 if R is not sorted or L == 0, -2 if memory runs out.
 */
int lj_oracle_rmi_fit(const uint64_t* R, uint64_t n, uint32_t L, int fp64,
                      double* root_fit, double* root_dep, uint64_t* leaf_lo,
                      double* leaf_fit, double* leaf_dep, int64_t* err) {
  if (L == 0 || !lj_oracle_is_sorted(R, n)) return -1;
  double* x = (double*)malloc(sizeof(double) * (n ? n : 1));
  double* y = (double*)malloc(sizeof(double) * (n ? n : 1));
  if (!x || !y) {
    free(x);
    free(y);
    return -2;
  }
  /* root: least squares of the scaled position i*L/n on the key */
  for (uint64_t i = 0; i < n; ++i) {
    x[i] = (double)R[i];
    y[i] = (double)i * (double)L / (double)n;
  }
  lsq_fit(x, y, n, &root_fit[0], &root_fit[1]);
  root_dep[0] = deploy(root_fit[0], fp64);
  root_dep[1] = deploy(root_fit[1], fp64);

  /* leaf of every key; the root is monotone, so each leaf is one range */
  for (uint32_t l = 0; l <= L; ++l) leaf_lo[l] = n;
  for (uint64_t i = n; i-- > 0;) {
    uint32_t l = root_leaf(R[i], root_dep[0], root_dep[1], L, fp64);
    leaf_lo[l] = i;
  }
  for (uint32_t l = L; l-- > 0;)
    if (leaf_lo[l] > leaf_lo[l + 1]) leaf_lo[l] = leaf_lo[l + 1];

  /* leaves: least squares of (i - lo) on (R[i] - base), then the errors */
  for (uint32_t l = 0; l < L; ++l) {
    uint64_t lo = leaf_lo[l], hi = leaf_lo[l + 1];
    double a = 0.0, b = 0.0;
    if (hi > lo) {
      uint64_t base = R[lo];
      for (uint64_t i = lo; i < hi; ++i) {
        x[i - lo] = (double)(R[i] - base);
        y[i - lo] = (double)(i - lo);
      }
      lsq_fit(x, y, hi - lo, &a, &b);
    }
    leaf_fit[2 * l] = a;
    leaf_fit[2 * l + 1] = b;
    leaf_dep[2 * l] = deploy(a, fp64);
    leaf_dep[2 * l + 1] = deploy(b, fp64);
    int64_t elo = 0, ehi = 0;
    for (uint64_t i = lo; i < hi; ++i) {
      int64_t e = (int64_t)(i - lo) -
                  leaf_pred(R[i], R[lo], leaf_dep[2 * l], leaf_dep[2 * l + 1], fp64);
      if (i == lo || e < elo) elo = e;
      if (i == lo || e > ehi) ehi = e;
    }
    err[2 * l] = elo;
    err[2 * l + 1] = ehi;
  }
  free(x);
  free(y);
  return 0;
}

/*
 * Learned lookup of key x through a fitted RMI (Section 2.D): root picks the
 * leaf, the leaf predicts a position, and a binary search between the error
 * bounds finds the first position whose key is >= x (lower bound) and the
 * first whose key is > x (upper bound).  Writes [lb, ub) and the searched
 * window [w_lo, w_hi); returns the leaf.
 */
uint32_t lj_oracle_rmi_lookup(const uint64_t* R, uint64_t n, uint32_t L, int fp64,
                              const double* root_dep, const uint64_t* leaf_lo,
                              const double* leaf_dep, const int64_t* err,
                              uint64_t x, uint64_t* lb, uint64_t* ub,
                              uint64_t* w_lo, uint64_t* w_hi) {
  uint32_t l = root_leaf(x, root_dep[0], root_dep[1], L, fp64);
  int64_t lo = (int64_t)leaf_lo[l], hi = (int64_t)leaf_lo[l + 1];
  int64_t wl = lo, wh = lo;
  if (hi > lo) {
    int64_t p = lo + leaf_pred(x, R[lo], leaf_dep[2 * l], leaf_dep[2 * l + 1], fp64);
    wl = p + err[2 * l];
    wh = p + err[2 * l + 1] + 1;
    if (wl < lo) wl = lo;
    if (wl > hi) wl = hi;
    if (wh < lo) wh = lo;
    if (wh > hi) wh = hi;
  }
  /* binary search for the lower bound inside [wl, wh) */
  int64_t a = wl, b = wh;
  while (a < b) {
    int64_t mid = a + (b - a) / 2;
    if (R[mid] < x)
      a = mid + 1;
    else
      b = mid;
  }
  *lb = (uint64_t)a;
  /* and for the upper bound */
  b = wh;
  while (a < b) {
    int64_t mid = a + (b - a) / 2;
    if (R[mid] <= x)
      a = mid + 1;
    else
      b = mid;
  }
  *ub = (uint64_t)a;
  *w_lo = (uint64_t)wl;
  *w_hi = (uint64_t)wh;
  (void)n;
  return l;
}

/* ------------------------------------------------- gapped RMI (3.A) ---- */
/*
 * Gapped RMI (Section 3.A): a typical RMI fitted over R
 * places every tuple of R, in key order, by model-based insertion into two
 * gapped arrays, one of keys and one of payloads; a lookup predicts a slot
 * with the same RMI and finishes with an exponential search.  The payload of
 * a key is its position in the sorted R (the join's r_idx).  Readings (the
 * paper gives no formulas):
 *   slots:     (1 + gaps) per key of R; the predicted slot of key x is
 *              (1 + gaps) * p(x), p(x) the RMI's predicted position (root ->
 *              leaf -> leaf model, the arithmetic of rmi_fit/rmi_lookup)
 *              clamped to the leaf's positions [lo_l, hi_l];
 *   insertion: keys in sorted order; a key takes its predicted slot when that
 *              slot comes after the slot of the previous key, else the first
 *              slot after it; the arrays have C = max((1 + gaps) * n,
 *              last slot + 1) slots;
 *   gaps:      a gap holds a copy of the next filled slot's key and payload
 *              (slots after the last key hold 2^64-1 and n), so the key array
 *              is sorted and a search needs no bitmap; pos[C] = n;
 *   lookup:    no key >= x is ever placed before x's predicted slot q (the
 *              model is monotone and insertion only moves keys to later
 *              slots), so the search runs from q to later slots: keys at
 *              q, q+1, q+3, q+7, ... until one is >= x, then a binary search
 *              in the last gap of that sequence.  The first slot with a key
 *              >= x holds, as payload, the position of the first key of R
 *              that is >= x (the lower bound); the first slot with a key > x
 *              gives the upper bound.
 */

/* Predicted slot of key x (before clamping to C). */
uint64_t lj_oracle_grmi_pslot(const uint64_t* R, uint32_t L, int fp64, const double* root_dep,
                              const uint64_t* leaf_lo, const double* leaf_dep, uint32_t gaps,
                              uint64_t x) {
  uint32_t l = root_leaf(x, root_dep[0], root_dep[1], L, fp64);
  int64_t lo = (int64_t)leaf_lo[l], hi = (int64_t)leaf_lo[l + 1];
  int64_t p = lo;
  if (hi > lo) p = lo + leaf_pred(x, R[lo], leaf_dep[2 * l], leaf_dep[2 * l + 1], fp64);
  if (p < lo) p = lo;
  if (p > hi) p = hi;
  return (uint64_t)p * (uint64_t)(1 + gaps);
}

/*
 * Model-based insertion of the n keys of sorted R.  Returns C, the number of
 * slots (with keys == NULL only C is computed); fills keys[C] and pos[C + 1]
 * when cap >= C and, if slot_of_key is not NULL, the slot of every key.
 * Returns -1 if R is not sorted, -2 if memory runs out, -3 if cap < C.
 */
int64_t lj_oracle_grmi_build(const uint64_t* R, uint64_t n, uint32_t L, int fp64,
                             const double* root_dep, const uint64_t* leaf_lo,
                             const double* leaf_dep, uint32_t gaps, uint64_t* keys,
                             uint32_t* pos, uint64_t cap, uint64_t* slot_of_key) {
  if (!lj_oracle_is_sorted(R, n)) return -1;
  uint64_t* slot = (uint64_t*)malloc(sizeof(uint64_t) * (n ? n : 1));
  if (!slot) return -2;
  /* insert in key order: predicted slot, or the first slot after the previous key */
  for (uint64_t i = 0; i < n; ++i) {
    uint64_t s = lj_oracle_grmi_pslot(R, L, fp64, root_dep, leaf_lo, leaf_dep, gaps, R[i]);
    if (i > 0 && s <= slot[i - 1]) s = slot[i - 1] + 1;
    slot[i] = s;
  }
  uint64_t C = (uint64_t)(1 + gaps) * n;
  if (n > 0 && slot[n - 1] + 1 > C) C = slot[n - 1] + 1;
  if (keys) {
    if (cap < C) {
      free(slot);
      return -3;
    }
    /* from the end: every slot takes the next filled slot's key and payload */
    uint64_t next_key = UINT64_MAX;
    uint32_t next_pos = (uint32_t)n;
    uint64_t i = n;
    for (uint64_t s = C; s-- > 0;) {
      if (i > 0 && slot[i - 1] == s) {
        --i;
        next_key = R[i];
        next_pos = (uint32_t)i;
      }
      keys[s] = next_key;
      pos[s] = next_pos;
    }
    pos[C] = (uint32_t)n;
  }
  if (slot_of_key) memcpy(slot_of_key, slot, sizeof(uint64_t) * n);
  free(slot);
  return (int64_t)C;
}

/* First slot at or after q whose key is >= x (strict: > x), or C. */
static uint64_t grmi_first(const uint64_t* keys, uint64_t C, uint64_t x, uint64_t q, int strict,
                           uint64_t* loads) {
  if (q >= C) return C;
  uint64_t lo = q, hi = C, off = 0;
  for (;;) { /* exponential phase: q, q+1, q+3, q+7, ... */
    uint64_t t = q + off;
    if (t >= C) break;
    ++*loads;
    if (strict ? keys[t] > x : keys[t] >= x) {
      hi = t;
      break;
    }
    lo = t + 1;
    off = 2 * off + 1;
  }
  while (lo < hi) { /* binary search in [lo, hi) */
    uint64_t mid = lo + (hi - lo) / 2;
    ++*loads;
    if (strict ? keys[mid] > x : keys[mid] >= x)
      hi = mid;
    else
      lo = mid + 1;
  }
  return lo;
}

/*
 * Join of S against a GRMI: for every probe j, [lo[j], hi[j]) = positions of
 * R with key S[j] (payloads of the first slots >= and > S[j]); loads[j]
 * (optional) = keys read by the two searches.  Returns |J|.
 */
int64_t lj_oracle_grmi_join_ranges(const uint64_t* R, uint32_t L, int fp64,
                                   const double* root_dep, const uint64_t* leaf_lo,
                                   const double* leaf_dep, uint32_t gaps, const uint64_t* keys,
                                   const uint32_t* pos, uint64_t C, const uint64_t* S,
                                   uint64_t m, uint64_t* lo, uint64_t* hi, uint64_t* loads) {
  int64_t total = 0;
  for (uint64_t j = 0; j < m; ++j) {
    uint64_t q = lj_oracle_grmi_pslot(R, L, fp64, root_dep, leaf_lo, leaf_dep, gaps, S[j]);
    uint64_t nl = 0;
    uint64_t lb = grmi_first(keys, C, S[j], q, 0, &nl);
    uint64_t ub = lb;
    if (lb < C && keys[lb] == S[j]) ub = grmi_first(keys, C, S[j], lb, 1, &nl);
    lo[j] = pos[lb];
    hi[j] = pos[ub];
    if (loads) loads[j] = nl;
    total += (int64_t)(hi[j] - lo[j]);
  }
  return total;
}

/* -------------------------------------------- learned hash index (3.C) -- */
/*
 * Learned hash index (Section 3.C): the CDF model serves as an
 * order-preserving hash function into a hash table; lookups hash the probe
 * key and look in the table, with no search over R.  Readings (the paper
 * uses a RadixSpline and gives no formulas; any monotone CDF model serves,
 * so the RMI of rmi_fit is used):
 *   entries:   one per distinct key of R, payload = its rank d among the
 *              distinct keys; first[d] = position of its first copy in R,
 *              first[D] = n, so its matches are [first[d], first[d+1]);
 *   table:     B = max(1, ceil(spk * D / 4)) buckets of 4 slots (spk = slots
 *              per distinct key, the inverse of the load factor);
 *   hash:      h(x) = p(x) * B / (n + 1) (integer division), p(x) the RMI's
 *              predicted position clamped to its leaf's positions [lo, hi];
 *   insertion: distinct keys in key order into the first free slot at or
 *              after slot 4 h(x) (linear probing; as h is monotone, keys stay
 *              in order, so the slot is max(4 h(x), previous slot + 1));
 *              C = max(4B, last slot + 1) slots; a free slot holds a copy of
 *              the next filled slot (after the last: 2^64-1 and D);
 *   lookup:    slots from 4 h(x) on, one by one, until a key >= x; a hit
 *              when it equals x and its payload is below D.
 */
static uint64_t lhash_h(const uint64_t* R, uint64_t n, uint32_t L, int fp64,
                        const double* root_dep, const uint64_t* leaf_lo, const double* leaf_dep,
                        uint64_t B, uint64_t x) {
  uint64_t p = lj_oracle_grmi_pslot(R, L, fp64, root_dep, leaf_lo, leaf_dep, 0, x);
  return p * B / (n + 1);
}

/*
 * Build: returns C (with keys == NULL, only C, D and B); fills keys[C],
 * pos[C + 1], first[D + 1], *D_out and *B_out.  -1: R not sorted, -2: out of
 * memory, -3: cap < C.
 */
int64_t lj_oracle_lhash_build(const uint64_t* R, uint64_t n, uint32_t L, int fp64,
                              const double* root_dep, const uint64_t* leaf_lo,
                              const double* leaf_dep, uint32_t spk, uint64_t* keys, uint32_t* pos,
                              uint64_t cap, uint32_t* first, uint64_t* D_out, uint64_t* B_out) {
  if (!lj_oracle_is_sorted(R, n)) return -1;
  uint64_t D = 0;
  for (uint64_t i = 0; i < n; ++i)
    if (i == 0 || R[i] != R[i - 1]) ++D;
  uint64_t B = (spk * D + 3) / 4;
  if (B == 0) B = 1;
  uint64_t* slot = (uint64_t*)malloc(sizeof(uint64_t) * (D ? D : 1));
  uint64_t* dkey = (uint64_t*)malloc(sizeof(uint64_t) * (D ? D : 1));
  if (!slot || !dkey) {
    free(slot);
    free(dkey);
    return -2;
  }
  uint64_t d = 0;
  for (uint64_t i = 0; i < n; ++i) {
    if (i > 0 && R[i] == R[i - 1]) continue;
    dkey[d] = R[i];
    if (first) first[d] = (uint32_t)i;
    uint64_t s = 4 * lhash_h(R, n, L, fp64, root_dep, leaf_lo, leaf_dep, B, R[i]);
    if (d > 0 && s <= slot[d - 1]) s = slot[d - 1] + 1;   /* linear probing */
    slot[d] = s;
    ++d;
  }
  if (first) first[D] = (uint32_t)n;
  uint64_t C = 4 * B;
  if (D > 0 && slot[D - 1] + 1 > C) C = slot[D - 1] + 1;
  if (keys) {
    if (cap < C) {
      free(slot);
      free(dkey);
      return -3;
    }
    uint64_t next_key = UINT64_MAX;
    uint32_t next_pos = (uint32_t)D;
    uint64_t k = D;
    for (uint64_t s = C; s-- > 0;) {
      if (k > 0 && slot[k - 1] == s) {
        --k;
        next_key = dkey[k];
        next_pos = (uint32_t)k;
      }
      keys[s] = next_key;
      pos[s] = next_pos;
    }
    pos[C] = (uint32_t)D;
  }
  if (D_out) *D_out = D;
  if (B_out) *B_out = B;
  free(slot);
  free(dkey);
  return (int64_t)C;
}

/* Join through the learned hash index: [lo[j], hi[j]) per probe, loads[j] =
 * table slots read; returns |J|. */
int64_t lj_oracle_lhash_join_ranges(const uint64_t* R, uint64_t n, uint32_t L, int fp64,
                                    const double* root_dep, const uint64_t* leaf_lo,
                                    const double* leaf_dep, uint64_t B, const uint64_t* keys,
                                    const uint32_t* pos, uint64_t C, const uint32_t* first,
                                    uint64_t D, const uint64_t* S, uint64_t m, uint64_t* lo,
                                    uint64_t* hi, uint64_t* loads) {
  int64_t total = 0;
  for (uint64_t j = 0; j < m; ++j) {
    uint64_t s = 4 * lhash_h(R, n, L, fp64, root_dep, leaf_lo, leaf_dep, B, S[j]);
    uint64_t nl = 0;
    while (s < C) {
      ++nl;
      if (keys[s] >= S[j]) break;
      ++s;
    }
    lo[j] = hi[j] = 0;
    if (s < C && keys[s] == S[j] && pos[s] < D) {
      lo[j] = first[pos[s]];
      hi[j] = first[pos[s] + 1];
    } else {
      /* no match: the lower bound of S[j] in R (for an empty range) */
      uint64_t a = 0, b = n;
      while (a < b) {
        uint64_t mid = a + (b - a) / 2;
        if (R[mid] < S[j]) a = mid + 1; else b = mid;
      }
      lo[j] = hi[j] = a;
    }
    if (loads) loads[j] = nl;
    total += (int64_t)(hi[j] - lo[j]);
  }
  return total;
}

/* ---------------------------------------------------------- RadixSpline -- */
/*
 * RadixSpline (Section 2.D; Kipf et al., "RadixSpline: a single-pass learned
 * index", aiDM 2020), the model of the learned hash INLJ variant (Section
 * 3.C uses a RadixSpline as the hash function).  Built bottom-up in one pass
 * over the sorted keys:
 *   CDF points  the distinct keys k_d with the position of their first copy
 *               in R, (k_d, first_d), d = 0..D-1;
 *   spline      points chosen greedily (the error corridor of Neumann and
 *               Michel, "Smooth interpolating histograms with error
 *               guarantees", 2008): from the last spline point b, every
 *               later CDF point q narrows a corridor of slopes to the window
 *               [q.y - eps, q.y + eps]; the first point whose own slope from b
 *               leaves the corridor makes the point before it a spline point,
 *               which restarts the corridor.  Every CDF point then lies
 *               within eps positions of the straight line between the spline
 *               points around it.  The pass restarts at every `chunk`-th
 *               CDF point (a spline point; chunk = 0: one pass over all);
 *   radix table over the r most significant bits of (key - k_0) of the
 *               spline points: table[b] = number of spline points whose
 *               prefix is below b, b = 0..2^r, shift = max(0, bitlen(k_max -
 *               k_0) - r);
 *   prediction  for k_0 <= x <= k_max: the spline points (x_i, y_i) <= x <
 *               (x_{i+1}, y_{i+1}) around x (prefix of x -> table -> binary
 *               search), pred = y_i + floor((x - x_i)(y_{i+1} - y_i) /
 *               (x_{i+1} - x_i)); below k_0: 0; above k_max: n.
 * The slope comparisons and the interpolation are exact integer arithmetic.
 */

/* a/b < c/d for b, d > 0 */
static int slope_lt(__int128 a, __int128 b, __int128 c, __int128 d) { return a * d < c * b; }

/* Spline points of the distinct keys dk[0..D) with positions dy[0..D):
 * writes up to cap points to sx/sy (if non-NULL) and returns their count. */
static uint64_t rs_spline(const uint64_t* dk, const uint64_t* dy, uint64_t D, uint32_t eps,
                          uint64_t chunk, uint64_t* sx, uint32_t* sy, uint64_t cap) {
  uint64_t S = 0;
#define RS_EMIT(d)                                         \
  do {                                                     \
    if (sx && S < cap) {                                   \
      sx[S] = dk[d];                                       \
      sy[S] = (uint32_t)dy[d];                             \
    }                                                      \
    ++S;                                                   \
  } while (0)
  if (chunk == 0) chunk = D ? D : 1;
  for (uint64_t c0 = 0; c0 < D; c0 += chunk) {
    const uint64_t c1 = c0 + chunk < D ? c0 + chunk : D;
    uint64_t base = c0;                 /* last spline point */
    RS_EMIT(base);
    __int128 up_dy = 0, up_dx = 1, lo_dy = 0, lo_dx = 1;   /* corridor: slopes lo <= s <= up */
    int open = 0;                       /* corridor started (a point after base seen) */
    for (uint64_t d = c0 + 1; d < c1; ++d) {
      const __int128 dx = (__int128)(dk[d] - dk[base]);
      const __int128 y = (__int128)dy[d] - (__int128)dy[base];
      if (!open) {
        up_dy = y + eps;
        up_dx = dx;
        lo_dy = y - eps;
        lo_dx = dx;
        open = 1;
        continue;
      }
      if (slope_lt(up_dy, up_dx, y, dx) || slope_lt(y, dx, lo_dy, lo_dx)) {
        /* d leaves the corridor: the point before it becomes a spline point */
        base = d - 1;
        RS_EMIT(base);
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
    if (c1 - 1 != base) RS_EMIT(c1 - 1);
  }
#undef RS_EMIT
  return S;
}

/* bit length of v (0 for 0) */
static uint32_t bitlen64(uint64_t v) {
  uint32_t b = 0;
  while (v) {
    ++b;
    v >>= 1;
  }
  return b;
}

/*
 * Build the RadixSpline of sorted R.  Returns S (the number of spline
 * points); sx/sy (S entries) and table (2^rbits + 1 entries) are written when
 * non-NULL and S <= cap; *shift_out receives the prefix shift.  -1: R not
 * sorted, -2: out of memory, -3: cap < S.
 */
int64_t lj_oracle_rs_build(const uint64_t* R, uint64_t n, uint32_t eps, uint64_t chunk,
                           uint32_t rbits, uint64_t* sx, uint32_t* sy, uint64_t cap,
                           uint32_t* table, uint32_t* shift_out) {
  if (!lj_oracle_is_sorted(R, n)) return -1;
  uint64_t D = 0;
  for (uint64_t i = 0; i < n; ++i)
    if (i == 0 || R[i] != R[i - 1]) ++D;
  uint64_t* dk = (uint64_t*)malloc(sizeof(uint64_t) * (D ? D : 1));
  uint64_t* dy = (uint64_t*)malloc(sizeof(uint64_t) * (D ? D : 1));
  if (!dk || !dy) {
    free(dk);
    free(dy);
    return -2;
  }
  uint64_t d = 0;
  for (uint64_t i = 0; i < n; ++i)
    if (i == 0 || R[i] != R[i - 1]) {
      dk[d] = R[i];
      dy[d] = i;
      ++d;
    }
  const uint64_t S = rs_spline(dk, dy, D, eps, chunk, NULL, NULL, 0);
  if (sx) {
    if (cap < S) {
      free(dk);
      free(dy);
      return -3;
    }
    rs_spline(dk, dy, D, eps, chunk, sx, sy, cap);
  }
  const uint32_t bl = D ? bitlen64(dk[D - 1] - dk[0]) : 0;
  const uint32_t shift = bl > rbits ? bl - rbits : 0;
  if (shift_out) *shift_out = shift;
  if (table && sx) {
    const uint64_t T = 1ull << rbits;
    for (uint64_t b = 0; b <= T; ++b) {
      uint64_t c = 0;   /* spline points with prefix below b */
      while (c < S && ((sx[c] - dk[0]) >> shift) < b) ++c;
      table[b] = (uint32_t)c;
    }
  }
  free(dk);
  free(dy);
  return (int64_t)S;
}

/* Position predicted for x (see above); binary search over all spline points. */
uint64_t lj_oracle_rs_predict(const uint64_t* sx, const uint32_t* sy, uint64_t S, uint64_t n,
                              uint64_t x) {
  if (S == 0 || x < sx[0]) return 0;
  if (x > sx[S - 1]) return n;
  uint64_t a = 0, b = S;   /* last i with sx[i] <= x */
  while (b - a > 1) {
    const uint64_t mid = a + (b - a) / 2;
    if (sx[mid] <= x)
      a = mid;
    else
      b = mid;
  }
  if (sx[a] == x || a + 1 == S) return sy[a];
  const unsigned __int128 num = (unsigned __int128)(x - sx[a]) * (uint64_t)(sy[a + 1] - sy[a]);
  return sy[a] + (uint64_t)(num / (sx[a + 1] - sx[a]));
}

/* Learned hash index with a RadixSpline as the hash (RSHASH-INLJ):
 * h(x) = pred(x) * B / (n + 1); otherwise as lj_oracle_lhash_build. */
int64_t lj_oracle_rs_lhash_build(const uint64_t* R, uint64_t n, const uint64_t* sx,
                                 const uint32_t* sy, uint64_t S, uint32_t spk, uint64_t* keys,
                                 uint32_t* pos, uint64_t cap, uint32_t* first, uint64_t* D_out,
                                 uint64_t* B_out) {
  if (!lj_oracle_is_sorted(R, n)) return -1;
  uint64_t D = 0;
  for (uint64_t i = 0; i < n; ++i)
    if (i == 0 || R[i] != R[i - 1]) ++D;
  uint64_t B = (spk * D + 3) / 4;
  if (B == 0) B = 1;
  uint64_t* slot = (uint64_t*)malloc(sizeof(uint64_t) * (D ? D : 1));
  uint64_t* dkey = (uint64_t*)malloc(sizeof(uint64_t) * (D ? D : 1));
  if (!slot || !dkey) {
    free(slot);
    free(dkey);
    return -2;
  }
  uint64_t d = 0;
  for (uint64_t i = 0; i < n; ++i) {
    if (i > 0 && R[i] == R[i - 1]) continue;
    dkey[d] = R[i];
    if (first) first[d] = (uint32_t)i;
    uint64_t s = 4 * (lj_oracle_rs_predict(sx, sy, S, n, R[i]) * B / (n + 1));
    if (d > 0 && s <= slot[d - 1]) s = slot[d - 1] + 1;   /* linear probing */
    slot[d] = s;
    ++d;
  }
  if (first) first[D] = (uint32_t)n;
  uint64_t C = 4 * B;
  if (D > 0 && slot[D - 1] + 1 > C) C = slot[D - 1] + 1;
  if (keys) {
    if (cap < C) {
      free(slot);
      free(dkey);
      return -3;
    }
    uint64_t next_key = UINT64_MAX;
    uint32_t next_pos = (uint32_t)D;
    uint64_t k = D;
    for (uint64_t s = C; s-- > 0;) {
      if (k > 0 && slot[k - 1] == s) {
        --k;
        next_key = dkey[k];
        next_pos = (uint32_t)k;
      }
      keys[s] = next_key;
      pos[s] = next_pos;
    }
    pos[C] = (uint32_t)D;
  }
  if (D_out) *D_out = D;
  if (B_out) *B_out = B;
  free(slot);
  free(dkey);
  return (int64_t)C;
}

/* Join through the RadixSpline hash index: [lo[j], hi[j]) per probe. */
int64_t lj_oracle_rs_lhash_join_ranges(const uint64_t* R, uint64_t n, const uint64_t* sx,
                                       const uint32_t* sy, uint64_t S, uint64_t B,
                                       const uint64_t* keys, const uint32_t* pos, uint64_t C,
                                       const uint32_t* first, uint64_t D, const uint64_t* Sq,
                                       uint64_t m, uint64_t* lo, uint64_t* hi) {
  int64_t total = 0;
  for (uint64_t j = 0; j < m; ++j) {
    uint64_t s = 4 * (lj_oracle_rs_predict(sx, sy, S, n, Sq[j]) * B / (n + 1));
    while (s < C && keys[s] < Sq[j]) ++s;
    if (s < C && keys[s] == Sq[j] && pos[s] < D) {
      lo[j] = first[pos[s]];
      hi[j] = first[pos[s] + 1];
    } else {
      uint64_t a = 0, b = n;
      while (a < b) {
        uint64_t mid = a + (b - a) / 2;
        if (R[mid] < Sq[j]) a = mid + 1; else b = mid;
      }
      lo[j] = hi[j] = a;
    }
    total += (int64_t)(hi[j] - lo[j]);
  }
  return total;
}

/* pred[j] = lj_oracle_rs_predict(..., X[j]) for j < m. */
void lj_oracle_rs_predict_many(const uint64_t* sx, const uint32_t* sy, uint64_t S, uint64_t n,
                               const uint64_t* X, uint64_t m, uint64_t* pred) {
  for (uint64_t j = 0; j < m; ++j) pred[j] = lj_oracle_rs_predict(sx, sy, S, n, X[j]);
}
