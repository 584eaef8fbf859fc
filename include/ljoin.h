/*
 * ljoin.h -- C ABI of the GB300 learned indexed nested loop join (RMI-INLJ).
 *
 * Method: Sabek and Kraska, "The Case for Learned In-Memory Joins".
 *   Section 2.A  indexed nested loop join: R carries an index on the join
 *                key; every tuple s of S fetches the R tuples with equal key.
 *   Section 2.D  two-level linear Recursive Model Index (RMI): a root linear
 *                model picks a leaf model, the leaf's linear model predicts
 *                a position, per-leaf min/max error bounds delimit a binary
 *                search.
 *   Section 3    RMI-INLJ: index R with an RMI, probe it with every s;
 *                3.A gapped RMI (grmi_build), 3.B buffered probing (the
 *                bucketed probe order), 3.C learned hash index
 *                (lhash_build).
 *   Section 4    learned sort-merge join (the sort-merge probe order).
 *   Section 6.A  the index is built before the join; its build time is not
 *                part of the join (Section 3.A).
 *   Section 6.B  duplicate keys: a range scan between the error bounds
 *                returns every match (1-to-m and n-to-m joins).
 *
 * Result of a join: J(R, S) = { (i, j) : R[i] == S[j] } as (r_idx, s_idx)
 * pairs, r_idx a position in the sorted R as passed, s_idx a position in S.
 * The library writes them s-major, r-ascending (deterministic).
 *
 * Conventions (all entry points):
 *   - Return 0 (LJ_OK) or a negative LJ_E_* code; lj_last_error() then gives
 *     a thread-local message.  No entry point aborts or exits the process.
 *   - Pointers named *_dev are CUDA device pointers (or managed memory) on
 *     the current device; *_host are host pointers.  Keys are uint64.
 *   - R is BORROWED by the index: device memory, sorted non-decreasing, left
 *     unchanged and alive until rmi_free.  S and every output buffer belong
 *     to the caller.
 *   - n = |R| and m = |S| are below 2^32 (indices are uint32); pair totals
 *     and offsets are uint64.
 *   - Work is ordered on `stream` (NULL = the legacy default stream) and is
 *     asynchronous, except where the call fills a *_host result: such a call
 *     synchronises `stream` before returning.
 *   - Empty R or empty S are valid and give zero pairs.
 *   - Device code never traps: a bounded wait that runs out or a capacity
 *     overflow sets an error word that the next synchronising call reports.
 */
#ifndef LJOIN_H
#define LJOIN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

struct CUstream_st;                     /* cudaStream_t == struct CUstream_st* */
typedef struct CUstream_st* lj_stream_t;

enum {
  LJ_OK = 0,
  LJ_E_INVAL = -1,      /* bad argument (NULL pointer, size out of range) */
  LJ_E_NOMEM = -2,      /* device or host allocation failed */
  LJ_E_CUDA = -3,       /* a CUDA runtime call failed (message has details) */
  LJ_E_UNSORTED = -4,   /* R is not sorted non-decreasing */
  LJ_E_CAPACITY = -5,   /* output buffer smaller than the join result */
  LJ_E_TIMEOUT = -6,    /* a bounded device wait or a host wait ran out */
  LJ_E_BUDGET = -7,     /* request larger than the server's memory budget */
  LJ_E_NOTUNIQUE = -8,  /* direct path (no offsets) asked for on an R with duplicates */
  LJ_E_STATE = -9       /* object used in a state that does not allow it */
};

enum { LJ_FP32 = 0, LJ_FP64 = 1 };     /* precision of the model evaluation */

typedef struct lj_index lj_index;       /* opaque, owned by the library */

typedef struct {
  uint32_t r_idx;
  uint32_t s_idx;
} lj_pair;                              /* 8 bytes, array of structs */

typedef struct {
  uint64_t n;               /* |R| */
  uint32_t leaves;          /* L */
  int32_t precision;        /* LJ_FP32 | LJ_FP64 */
  int32_t unique;           /* 1 if no key of R repeats */
  uint32_t nonempty_leaves;
  uint32_t max_leaf_size;
  uint32_t max_window;      /* max over leaves of min(e_hi - e_lo + 1, size) */
  double mean_window;       /* key-weighted mean of that width */
  double root_a, root_b;    /* deployed root parameters (widened) */
  double build_ms;          /* device time of the build, CUDA events */
} lj_index_stats;

/* ------------------------------------------------------------- index ---- */

/*
 * rmi_build -- fit a two-level linear RMI over the sorted R (Section 2.D).
 *   R_dev      n sorted keys (device, borrowed for the index's lifetime)
 *   leaves     L, number of leaf models, 1 .. 2^24
 *   precision  LJ_FP32: models evaluated in single precision (fused
 *              multiply-add), fits in double; LJ_FP64: double throughout.
 *              Error bounds are always measured with the deployed arithmetic,
 *              so the join is exact at either precision.
 *   out        receives the index; free with rmi_free.
 * Root: leaf(x) = clamp(floor(a0*X + b0), 0, L-1), (a0, b0) the least-squares
 * line of i*L/n on R[i].  Leaf l owns positions [lo_l, hi_l); with base key
 * k_l = R[lo_l]: pred(x) = lo_l + floor(a_l*(x - k_l) + b_l), (a_l, b_l) the
 * least-squares line of (i - lo_l) on (R[i] - k_l), slope >= 0; e_lo/e_hi the
 * min/max of i - pred(R[i]) over the leaf.
 * Synchronises `stream`.  Errors: LJ_E_INVAL, LJ_E_UNSORTED, LJ_E_NOMEM,
 * LJ_E_CUDA.
 */
int rmi_build(const uint64_t* R_dev, uint64_t n, uint32_t leaves, int precision,
              lj_stream_t stream, lj_index** out);

/*
 * rmi_build_batch -- fit k RMIs at once (Section 2.D, as rmi_build), one
 * segmented pass over all relations: every build kernel covers the whole
 * batch (root sums per relation, leaf bounds, chunked leaf fits and error
 * bounds over all leaves of all relations), a dozen launches in all instead
 * of a dozen per relation.  Each relation's arithmetic is the one rmi_build
 * uses, so out[j] is bit for bit the index rmi_build(R_dev[j], n[j],
 * leaves[j], precision) gives.
 *   R_dev[k], n[k], leaves[k]   as rmi_build, per relation (borrowed)
 *   precision                   one precision for the batch
 *   out[k]                      receives the indexes; free each with
 *                               rmi_free (their leaf records share one
 *                               allocation, released with the last index)
 * stats.build_ms of each index is the time of the whole batch.  Synchronises.
 * Errors: those of rmi_build (for any relation); no index is returned then.
 */
int rmi_build_batch(const uint64_t* const* R_dev, const uint64_t* n, const uint32_t* leaves,
                    uint32_t k, int precision, lj_stream_t stream, lj_index** out);

/* Release an index (its device memory; R itself is not touched). NULL is ok. */
void rmi_free(lj_index* index);

/* Summary statistics of a built index.  Host-only, no device work. */
int rmi_stats(const lj_index* index, lj_index_stats* out);

/*
 * rmi_export -- copy the index to host memory for inspection.
 *   root_host   2 doubles: deployed (a0, b0), widened to double
 *   leaf_lo     L+1 uint64: first position of each leaf, leaf_lo[L] = n
 *   leaf_ab     2L doubles: deployed (a_l, b_l) per leaf, widened
 *   leaf_err    2L int64: (e_lo, e_hi) per leaf
 * Any pointer may be NULL.  Synchronises.  Section 2.D, as rmi_build.
 */
int rmi_export(const lj_index* index, double* root_host, uint64_t* leaf_lo,
               double* leaf_ab, int64_t* leaf_err);

/* -------------------------------------------------------- gapped RMI ---- */

/* Statistics of an index's gapped arrays (grmi_build or lhash_build). */
typedef struct {
  uint64_t slots;           /* C: length of the gapped key array */
  uint32_t gaps;            /* grmi_build: gaps per key; lhash_build: slots per distinct key */
  uint32_t kind;            /* 0: gapped RMI (grmi_build), 1: learned hash (lhash_build) */
  double mean_disp;         /* mean of (slot - predicted slot) over the placed keys */
  uint64_t max_disp;        /* largest such displacement */
  double build_ms;          /* device time of the build, CUDA events */
  uint64_t distinct;        /* lhash_build: number of distinct keys of R (else 0) */
} lj_grmi_stats;

/*
 * grmi_build -- Gapped RMI (Section 3.A): model-based insertion of every key
 * of R, in key order, into a gapped key array and a gapped payload array
 * attached to `index` (payload = the key's position in R).
 *   index   built by rmi_build; its model predicts the slots
 *   gaps    gaps per key, 0 .. 16 (the paper's default is 4): the arrays
 *           have C = max((1 + gaps) * n, last slot + 1) slots, C < 2^32 - 1
 * Predicted slot of key x: (1 + gaps) * p(x), p(x) the RMI's predicted
 * position clamped to its leaf's positions [lo_l, hi_l].  A key takes its
 * predicted slot, or the first slot after the previous key's if that is
 * later.  A gap holds a copy of the next key and its payload (after the last
 * key: 2^64-1 and n), so the key array is sorted and no bitmap is needed.
 * From then on join_count, join_emit and join_host on this index look keys
 * up by exponential search from the predicted slot (keys at q, q+1, q+3,
 * q+7, ... then a binary search); results are identical to the plain RMI's.
 * The batched path and join_count_noalloc reject a gapped index
 * (LJ_E_INVAL); the serving path runs each request to such a relation alone,
 * with join_emit's kernels.  Rebuilding replaces the arrays.  Not safe while a join on
 * the index is in flight.  Synchronises `stream`.
 * Errors: LJ_E_INVAL (NULL index, gaps > 16, C too large), LJ_E_NOMEM,
 * LJ_E_CUDA.
 */
int grmi_build(lj_index* index, uint32_t gaps, lj_stream_t stream);

/*
 * lhash_build -- learned hash index (Section 3.C): the RMI serves as an
 * order-preserving hash function into a table of 4-slot buckets, one entry
 * per distinct key of R, attached to `index` (replacing gapped arrays it
 * may have).
 *   spk    slots per distinct key, 1 .. 16 (the inverse load factor; the
 *          paper's hash baselines use 4): B = max(1, ceil(spk * D / 4))
 *          buckets for D distinct keys
 * Hash of key x: h(x) = p(x) * B / (n + 1) (integer division), p(x) the
 * RMI's predicted position clamped to its leaf's positions.  Distinct keys
 * take, in key order, the first free slot at or after slot 4 h(x) (linear
 * probing; the hash is monotone, so the table stays sorted and a free slot
 * holds a copy of the next entry).  An entry's payload is the rank d of its
 * key among the distinct keys; first[d] is the position of its first copy in
 * R, first[D] = n, and its matches are R's positions [first[d], first[d+1]);
 * each slot also stores that range (8 bytes), so a hit reads it with one load.
 * Lookups hash the probe and search forward from its bucket (exponential
 * steps, then a binary search); duplicates need no second search.  Joins on
 * the index then behave as after grmi_build (same results, same paths).
 * Synchronises.  Errors: LJ_E_INVAL (NULL index, spk out of range, too many
 * slots), LJ_E_NOMEM, LJ_E_CUDA.
 */
int lhash_build(lj_index* index, uint32_t spk, lj_stream_t stream);

/*
 * lhash_build_rs -- the learned hash index of lhash_build with a RadixSpline
 * (Section 2.D) as the hash function instead of the RMI: the paper's
 * RSHASH-INLJ (Section 3.C; Section 6.A picks a RadixSpline for it).
 *   spk         slots per distinct key, 1 .. 16 (as lhash_build)
 *   eps         error bound of the spline, in positions (0 .. 2^20)
 *   radix_bits  bits of the radix table, 1 .. 24 (2^radix_bits + 1 entries)
 * The RadixSpline is fitted to the CDF of R's distinct keys (each at the
 * position of its first copy): spline points are chosen greedily in one pass
 * so that every CDF point lies within eps positions of the line between the
 * spline points around it (the pass restarts every 1024 distinct keys: one
 * GPU thread per run; each run starts and ends with a spline point); the
 * radix table indexes the spline points by the top radix_bits bits of
 * (key - smallest key).  Prediction of x: 0 below the smallest key, n above
 * the largest, else y_i + floor((x - x_i)(y_{i+1} - y_i) / (x_{i+1} - x_i))
 * for the spline points around x (exact integer arithmetic); the hash is
 * h(x) = pred(x) * B / (n + 1), and the table and its lookups are those of
 * lhash_build.  The RMI of `index` is not used by its joins.  Synchronises.
 * Errors: LJ_E_INVAL, LJ_E_NOMEM, LJ_E_CUDA.
 */
int lhash_build_rs(lj_index* index, uint32_t spk, uint32_t eps, uint32_t radix_bits,
                   lj_stream_t stream);

/*
 * rs_export -- the RadixSpline of an lhash_build_rs index into host memory:
 * sx_host[count] keys and sy_host[count] positions of the spline points,
 * table_host[2^radix_bits + 1] (spline points with prefix below b), the
 * prefix shift and the count.  Any pointer may be NULL.  LJ_E_STATE without
 * a RadixSpline.  Synchronises.
 */
int rs_export(const lj_index* index, uint64_t* sx_host, uint32_t* sy_host, uint32_t* table_host,
              uint32_t* shift_host, uint64_t* count_host);

/* first[D + 1] of a learned hash index (lhash_build, lhash_build_rs) into
 * host memory; LJ_E_STATE without one.  Synchronises. */
int lhash_export_first(const lj_index* index, uint32_t* first_host);

/* Release the gapped arrays (grmi_build or lhash_build); joins go back to
 * the RMI's bounded search. */
int grmi_drop(lj_index* index);

/* Lookup structures index_autotune chooses from. */
enum {
  LJ_LOOKUP_RMI = 0,            /* bounded search in R, probes in S order */
  LJ_LOOKUP_RMI_BUCKETED = 1,   /* bounded search in R, bucketed probe order */
  LJ_LOOKUP_GRMI = 2,           /* gapped RMI, 4 gaps per key (grmi_build) */
  LJ_LOOKUP_LHASH = 3,          /* learned hash index, 4 slots per key (lhash_build) */
  LJ_LOOKUP_SORTMERGE = 4,      /* bounded search in R, learned sort-merge order (Section 4) */
  LJ_LOOKUP_RSHASH = 5,         /* learned hash with a RadixSpline as the hash, 4 slots per key,
                                   eps 16, 18 radix bits (lhash_build_rs) */
  LJ_LOOKUP_RMI_LEVELS = 6      /* bounded search in R as a descent of R's key levels
                                   (option "key_levels"), probes in S order */
};

/*
 * index_autotune -- choose the lookup structure for joins on `index`: builds
 * each of LJ_LOOKUP_* in turn, times the count pass of the join on the
 * sample S_sample_dev (m_sample probes, device; a uniform sample of the
 * probes to come, ideally at least 2^22 of them) with CUDA events (best of
 * three after a warm-up), and leaves the fastest in place: its gapped arrays
 * if any, and the index's own probe order (which overrides the process-wide
 * "probe_buckets" option for this index).  The RMI itself is unchanged, so
 * results are the same whatever the choice (Sections 2.D, 3.A, 3.B, 3.C).
 *   choice       receives LJ_LOOKUP_*
 *   ns_per_key   optional: receives the seven timings (ns per probe, by LJ_LOOKUP_*)
 * Synchronises.  Errors: those of grmi_build, lhash_build and join_count.
 */
int index_autotune(lj_index* index, const uint64_t* S_sample_dev, uint64_t m_sample,
                   lj_stream_t stream, int* choice, double* ns_per_key);

/* Statistics of the gapped arrays; LJ_E_STATE if the index has none. */
int grmi_stats(const lj_index* index, lj_grmi_stats* out);

/*
 * grmi_export -- copy the gapped arrays to host memory.
 *   keys_host  C uint64 (grmi_stats().slots), may be NULL
 *   pos_host   C + 1 uint32 (pos_host[C] = n), may be NULL
 * Synchronises.  LJ_E_STATE if the index has no gapped arrays.
 */
int grmi_export(const lj_index* index, uint64_t* keys_host, uint32_t* pos_host);

/* ------------------------------------------------------------- join ----- */

/*
 * join_count -- number of matches of every probe, and their offsets
 * (Section 2.A probe of every s; Section 6.B all duplicates).
 *   S_dev        m probe keys (device)
 *   counts_dev   optional, m uint32: c_j = |{ i : R[i] == S[j] }|
 *   offsets_dev  optional, m+1 uint64: exclusive prefix sum of c,
 *                offsets[m] = |J|
 *   total_host   optional: |J|; if given the call synchronises.
 * Learned lookup (root, leaf, bounded lower/upper-bound search) and a scan:
 * one kernel with a decoupled look-back for batches up to "single_pass_max"
 * keys (lj_set_option), else a search kernel followed by a streaming scan.
 * Errors: LJ_E_INVAL, LJ_E_NOMEM, LJ_E_CUDA, LJ_E_TIMEOUT.
 */
int join_count(const lj_index* index, const uint64_t* S_dev, uint64_t m,
               uint32_t* counts_dev, uint64_t* offsets_dev, uint64_t* total_host,
               lj_stream_t stream);

/*
 * join_count_noalloc -- join_count without any memory allocation.
 *   The paper has no counterpart: this entry point exists for callers that
 *   cannot allocate device memory at call time -- for example a real-time
 *   serving loop whose latency budget forbids cudaMalloc and its implicit
 *   device synchronisation, code running under another allocator that owns
 *   all device memory, or a host that pre-plans every allocation up front.
 *   Same arguments, results and errors as join_count, but the scratch memory
 *   of its kernel (tile states of the single-pass scan, total, error word)
 *   is a fixed array of about 320 KiB compiled into the library, which every
 *   GPU that loads the library keeps until the process exits.  The call
 *   itself allocates nothing: no cudaMalloc, no cudaFree, no memory pool.
 *   Limits and rules:
 *     - m must be at most 2^25 (33,554,432) probes, else LJ_E_INVAL;
 *     - the first call on a device looks up the array's device address
 *       (once per device); make that first call before any stream capture;
 *     - every call on a device shares the one array: calls whose kernels can
 *       overlap on the GPU (different streams without ordering, several host
 *       threads) race and give wrong results; order them on one stream.
 *   The array keeps the last call's contents; each call clears what must
 *   start at zero (ticket, tile flags) on `stream`.  Errors of the kernel
 *   (a look-back wait that ran out) go to an error word in the array: a call
 *   with total_host reports them (LJ_E_TIMEOUT) and clears the word; the
 *   error of a call without total_host stays there until the next call on the
 *   device that passes total_host.
 */
int join_count_noalloc(const lj_index* index, const uint64_t* S_dev, uint64_t m,
                       uint32_t* counts_dev, uint64_t* offsets_dev, uint64_t* total_host,
                       lj_stream_t stream);

/*
 * join_emit -- write the join pairs (Section 2.A; Section 6.B).
 *   offsets_dev   m+1 offsets from join_count (two-pass path), or NULL for
 *                 the direct path, which needs an index whose R has no
 *                 duplicate key (else LJ_E_NOTUNIQUE): for batches up to
 *                 "fused_max" keys one cooperative kernel (lookups, a
 *                 grid-wide barrier, block prefixes, pairs); for larger ones
 *                 a search kernel, a scan of per-tile counts and a kernel
 *                 that writes the pairs (or, for batches up to
 *                 "single_pass_max" keys, the single-pass look-back kernel).
 *   pairs_dev     capacity pairs; pairs beyond capacity are not written.
 *   written_dev   optional device uint64: |J| (stream-ordered, no sync)
 *   written_host  optional host uint64: |J|; if given the call synchronises
 *                 and returns LJ_E_CAPACITY when |J| > capacity.
 * Errors: LJ_E_INVAL, LJ_E_NOTUNIQUE, LJ_E_NOMEM, LJ_E_CUDA, LJ_E_CAPACITY,
 * LJ_E_TIMEOUT.
 */
int join_emit(const lj_index* index, const uint64_t* S_dev, uint64_t m,
              const uint64_t* offsets_dev, lj_pair* pairs_dev, uint64_t capacity,
              uint64_t* written_dev, uint64_t* written_host, lj_stream_t stream);

/*
 * join_locate -- join_count that also records where each probe's matches
 * start (Section 2.A; Section 6.B: the matches of a key are one contiguous
 * run of the sorted R, so a probe's result is the range
 * [first[j], first[j] + counts[j]) of R's positions).
 *   first_dev    m uint32 (required): position of the first key of R equal to
 *                S[j]; unspecified when S[j] has no match
 *   counts_dev, offsets_dev, total_host   as join_count
 * With join_expand this is a two-pass join whose second pass searches
 * nothing.  Errors: as join_count.
 */
int join_locate(const lj_index* index, const uint64_t* S_dev, uint64_t m, uint32_t* first_dev,
                uint32_t* counts_dev, uint64_t* offsets_dev, uint64_t* total_host,
                lj_stream_t stream);

/*
 * join_expand -- write the pairs of located ranges: for every probe j the
 * pairs (first[j] + t, j), t < offsets[j+1] - offsets[j], at positions
 * offsets[j] + t (s-major, r-ascending: the order join_emit writes).
 *   first_dev    m uint32 from join_locate
 *   offsets_dev  m+1 uint64 from join_locate
 *   pairs_dev, capacity, written_dev, written_host   as join_emit
 * Streams first and offsets once and writes the pairs with coalesced stores;
 * needs neither the index nor S.  Errors: LJ_E_INVAL, LJ_E_CUDA,
 * LJ_E_CAPACITY.
 */
int join_expand(const uint32_t* first_dev, const uint64_t* offsets_dev, uint64_t m,
                lj_pair* pairs_dev, uint64_t capacity, uint64_t* written_dev,
                uint64_t* written_host, lj_stream_t stream);

/*
 * join_host -- the whole join from host buffers: copies S (host, ideally
 * pinned) to the device in chunks, runs the lookup on each chunk while the
 * next one is in flight, and copies the pairs back into pairs_host
 * (capacity pairs).  s_idx values are positions in the whole S.  Per chunk:
 * the direct path when R is unique, else join_locate + join_expand, with the
 * pairs of one chunk copied out while the next is looked up.  Page-locked S
 * is read in place by the kernels.  The lookup structure, probe order and
 * options of the index apply.  Synchronises.  Errors: as join_emit.
 */
int join_host(const lj_index* index, const uint64_t* S_host, uint64_t m,
              lj_pair* pairs_host, uint64_t capacity, uint64_t* written_host,
              lj_stream_t stream);

/* ------------------------------------------------ learned sort-merge ---- */

/*
 * lsj_join -- learned sort-merge join (L-SJ, Section 4) of two UNSORTED
 * relations: J = { (i, j) : R[i] == S[j] }, i and j positions in R and S as
 * given (no index, no sorted input).
 *   model      per relation, a CDF model built from an evenly spaced sample
 *              of at most 16,384 keys, sorted on the device: the
 *              piecewise-linear function through every 32nd sample key,
 *              looked up through a radix table (Section 4.B);
 *   partition  both relations range-partitioned with their model into
 *              partitions of about 2048 keys (histogram, scan, scatter of
 *              one 16-byte (key, position) record per key);
 *   sort       each partition sorted on its own by (key, position) in
 *              shared memory: split into buckets by the top bits of the key
 *              offsets, each entry placed by its rank in its bucket (Section
 *              4.C); the relations are then sorted;
 *   join       R's partitions in chunks of up to 4096 keys, each merged with
 *              the partitions of S its first and last keys map to under S's
 *              model (Section 4.D).
 *   pairs_dev, capacity   output (device); pairs beyond capacity are not written
 *   written_host          |J| (optional)
 * Pairs are grouped by R chunk (R's key order), then in S's (key, position)
 * order, then R's; the same for the same input.  Work memory: about 36
 * bytes per key of R and S, plus 16 bytes per key of the larger relation
 * (stream-ordered pool).  Synchronises.
 * Errors: LJ_E_INVAL, LJ_E_NOMEM, LJ_E_CUDA, LJ_E_CAPACITY.
 */
int lsj_join(const uint64_t* R_dev, uint64_t n, const uint64_t* S_dev, uint64_t m,
             lj_pair* pairs_dev, uint64_t capacity, uint64_t* written_host, lj_stream_t stream);

/* ----------------------------------------------------------- batches ---- */

typedef struct lj_batch lj_batch;      /* opaque batch plan, owned by the library */

/*
 * join_batch_plan -- prepare k independent joins (Section 2.A / 2.D probe of
 * S_j against index_j, each into its own pairs buffer) to run together.
 *   indexes[k]   built indexes; R must be unique in each (else
 *                LJ_E_NOTUNIQUE) and all must share one precision
 *   S_dev[k], m[k]                 probe keys of each join (device)
 *   pairs_dev[k], capacity[k]      output of each join (device); pairs beyond
 *                                  a join's capacity are not written
 * The plan copies the descriptors to the device and allocates all scratch
 * (4 bytes per probe of the batch plus small tables) up front; it borrows
 * every pointer, which must stay valid while the plan is used.  Synchronises.
 * Errors: LJ_E_INVAL, LJ_E_NOTUNIQUE, LJ_E_NOMEM, LJ_E_CUDA.
 */
int join_batch_plan(const lj_index* const* indexes, const uint64_t* const* S_dev,
                    const uint64_t* m, uint32_t k, lj_pair* const* pairs_dev,
                    const uint64_t* capacity, lj_stream_t stream, lj_batch** out);

/*
 * join_batch_run -- run every join of a plan: one persistent search launch
 * that balances all joins' tiles over the GPU, one scan, one compaction;
 * asynchronous, allocation-free.  Outputs:
 *   written_dev   optional device array of k uint64: each join's |J|
 *   written_host  optional host array of k uint64; if given the call
 *                 synchronises and reports LJ_E_CAPACITY if a join overflowed.
 * A plan's runs must not overlap on the GPU (they share the plan's scratch).
 */
int join_batch_run(lj_batch* plan, uint64_t* written_dev, uint64_t* written_host,
                   lj_stream_t stream);

/*
 * join_batch_capture -- record one run of the plan as a CUDA graph on
 * `stream` (a non-default stream); later join_batch_run calls launch the
 * graph instead of the individual operations.  Errors: LJ_E_INVAL, LJ_E_CUDA.
 */
int join_batch_capture(lj_batch* plan, lj_stream_t stream);

/*
 * join_batch_set_shape -- work-item shape of the batched search: `block`
 * threads per block (128 or 256, two probes per thread and tile) and
 * `tiles_per_item` consecutive tiles of one join per work item (1, 4 or 8).
 * Default 128 x 4 (1024 probes per item).  Drops a captured graph.
 * Synchronises.  Errors: LJ_E_INVAL, LJ_E_CUDA.
 */
int join_batch_set_shape(lj_batch* plan, int block, int tiles_per_item);

/*
 * join_batch_autotune -- time one run of the plan for each work-item shape
 * (128 or 256 threads x 1, 4 or 8 tiles) and keep the fastest; the chosen
 * shape is returned in best_block / best_tiles (nullable).  The runs write
 * the joins' outputs.  Synchronises.  Errors: as join_batch_run.
 */
int join_batch_autotune(lj_batch* plan, lj_stream_t stream, int* best_block, int* best_tiles);

/* Release a plan (its scratch and graph).  NULL is ok. */
void join_batch_free(lj_batch* plan);

/* join_batch -- plan + run + free in one call (the one-shot form).  written_host
 * (k uint64, nullable) receives each join's |J|.  Synchronises. */
int join_batch(const lj_index* const* indexes, const uint64_t* const* S_dev, const uint64_t* m,
               uint32_t k, lj_pair* const* pairs_dev, const uint64_t* capacity,
               uint64_t* written_host, lj_stream_t stream);

/*
 * rmi_autotune -- choose the leaf count L for an index over R (the paper tunes
 * its RMIs with an optimiser, Section 6.A; this is the library's own tuner):
 * builds the index for L = 2^8, 2^10, ... up to min(2^22, n/2), times the probe
 * path on the sample S_sample_dev (m_sample keys, device) and returns the L
 * with the least time per key (best_ns_per_key: that time, or -1 when the
 * answer came from the cache).  Answers are cached per (floor(log2 n), skew
 * bucket of R, precision); rmi_autotune_clear empties the cache.
 * Synchronises.  Errors: those of rmi_build / join_emit.
 */
int rmi_autotune(const uint64_t* R_dev, uint64_t n, const uint64_t* S_sample_dev,
                 uint64_t m_sample, int precision, lj_stream_t stream, uint32_t* best_leaves,
                 double* best_ns_per_key);
void rmi_autotune_clear(void);

/* ----------------------------------------------------------- serving ---- */

typedef struct lj_server lj_server;    /* opaque request server */
typedef uint64_t lj_ticket;            /* one submitted request */

typedef struct {
  uint64_t hbm_budget_bytes;   /* device memory requests may hold at once */
  uint32_t streams;            /* in-flight batches (slots), 1..16 */
  uint32_t max_batch;          /* requests per batch, 1..65536 */
} lj_server_cfg;

typedef struct {
  int32_t status;              /* 0, or the request's LJ_E_* error */
  uint64_t pairs;              /* |J| of the request */
  const lj_pair* pairs_dev;    /* server-owned result until join_release */
  double latency_us;           /* submit -> completion seen by the server */
  double queue_us;             /* submit -> launch */
} lj_result;

typedef struct {
  uint64_t submitted, completed, rejected, keys, batches;
  double mean_batch;           /* requests per launched batch */
  uint64_t mem_in_use, mem_peak;
  double p50_us, p99_us, mean_us, max_us;
  double span_s;               /* first submit -> last completion */
  double keys_per_s;           /* probe keys completed / span */
  uint64_t resident;           /* bytes of the registered relations (keys + leaf records),
                                  part of mem_in_use */
} lj_server_stats;

/*
 * Serving: resident learned indexes answer probe requests with continuous
 * batching.  Each request is one join (Section 2.A probe of its keys against
 * a resident relation's index, Section 2.D), answered exactly as join_emit
 * would answer it alone.  The budget covers the registered relations (their
 * keys, leaf records and any gapped or hash arrays, charged when added) and
 * the requests in flight.  A scheduler thread admits pending requests first
 * come, first served, when an in-flight slot is free and the memory they
 * need (12 bytes per probe: 8 for pairs, 4 for search words) fits what the
 * budget has left; every admitted group runs as one batched launch on its
 * slot's stream -- a group of one request, and every request to a relation
 * with gapped or hash arrays (which always runs alone), with join_emit's own
 * kernels -- so batches admitted while others run overlap on the device.
 *
 * join_server_create   start a server on the current device.
 * join_server_add_relation  register a built index (unique R, one precision
 *                      for all relations; borrowed; gapped or hash arrays
 *                      allowed, not to be rebuilt or dropped while
 *                      registered); returns its id.  LJ_E_BUDGET if its keys,
 *                      leaf records and arrays do not fit the budget left.
 * join_submit          queue a request: m probe keys at S (device or
 *                      page-locked host memory, valid until the request
 *                      completes).  Returns at once.  LJ_E_BUDGET if the
 *                      request alone exceeds what the relations leave of the
 *                      budget.
 * join_wait            wait (timeout_us < 0: forever) for a request;
 *                      LJ_E_TIMEOUT if it is not done in time.
 * join_fetch           copy a completed request's pairs to dst_dev
 *                      (stream-ordered on `stream`; a later join_release
 *                      frees the pairs only after that copy).
 * join_release         drop a completed request and free its pairs.
 * join_server_stats    counters and latency percentiles (reset: clear them).
 * join_server_destroy  finish queued work, stop the scheduler, free all.
 */
int join_server_create(const lj_server_cfg* cfg, lj_server** out);
int join_server_add_relation(lj_server* server, const lj_index* index, uint32_t* rel_id);
int join_submit(lj_server* server, uint32_t rel_id, const uint64_t* S, uint64_t m,
                lj_ticket* ticket);
int join_wait(lj_server* server, lj_ticket ticket, int64_t timeout_us, lj_result* result);
int join_fetch(lj_server* server, lj_ticket ticket, lj_pair* dst_dev, uint64_t capacity,
               lj_stream_t stream);
int join_release(lj_server* server, lj_ticket ticket);
int join_server_stats(lj_server* server, lj_server_stats* out, int reset);
void join_server_destroy(lj_server* server);

/* ------------------------------------------------------ diagnostics ----- */

/*
 * lj_set_option / lj_get_option -- process-wide tuning knobs (atomic: a call
 * in flight uses the value it read when it started).
 *   "single_pass_max"  probe batches of at most this many keys use the
 *                      single-pass kernel (lookup + scan + write in one
 *                      launch); larger ones use the count-scan-emit pipeline
 *                      (search kernel, then a streaming scan).  Default 0: the
 *                      pipeline measured faster at every batch size from
 *                      2^14 to 2^22 keys.  Both paths give identical results.
 *   "key_levels"       1: rmi_build also stores R's key levels,
 *                      a static 4-ary tree of fence keys (level k holds
 *                      R[4^k i]; about n/3 keys, 8 bytes each), and the
 *                      pipeline's and the fused kernel's bounded searches
 *                      descend it (one 32-byte node per level, about
 *                      log4(window) + 1 loads) instead of halving the window
 *                      (log2).  2 (default): only for an R with duplicate
 *                      keys (measured faster there; on unique keys halving
 *                      shares more of its pivots across a warp).  0: never.
 *                      Applies to indexes built afterwards (index_autotune
 *                      also tries the descent, LJ_LOOKUP_RMI_LEVELS);
 *                      results are the same either way.
 *   "fused_max"        join_emit's direct path (unique R) runs batches of
 *                      at most this many keys in one cooperative kernel of
 *                      resident blocks (0 .. 2^22; default 2^21; a batch
 *                      that does not fit the resident blocks takes the
 *                      pipeline).  Same results as the pipeline.
 *   "fused_groups"     1 (default): that kernel searches the error window by
 *                      halving over aligned 4-key groups and reads the last
 *                      group with one 32-byte load; 0: plain bisection.
 *   "host_chunk"       probe keys per chunk of join_host (2^16 .. 2^32-1;
 *                      default 2^25).
 *   "probe_buckets"    1: the pipeline first groups the probes of every
 *                      chunk of 2^22 by the region of R their predicted
 *                      position falls in (2^14 regions), looks them up in that
 *                      order and writes the results back to the probes' own
 *                      positions (same results, more locality in R; pays
 *                      when probes spread over an R larger than L2).
 *                      2: learned sort-merge order (Section 4): the same
 *                      buckets, each sorted in shared memory and merged with
 *                      the part of R it spans (buckets above 1024 probes
 *                      are searched probe by probe).
 *                      0 (default): probes in S order.  Gapped indexes
 *                      ignore it.
 *   "lookback_polls"   bound of one decoupled look-back wait of the probe
 *                      kernels: polls of a predecessor tile's state before the
 *                      tile gives up, records LJ_E_TIMEOUT in the error word
 *                      and goes on (16 .. 2^20; default 2^20).
 *   "fault_skip_tiles" fault injection for tests (0 .. 1024; default 0): the
 *                      single-pass kernel (single_pass_max, join_count_noalloc)
 *                      skips this many leading tiles, which then never publish
 *                      their state, so the look-back waits of the next tiles
 *                      run out and the call reports LJ_E_TIMEOUT (no device
 *                      trap; the context stays usable); likewise the fused
 *                      kernel (fused_max) skips this many leading blocks,
 *                      which never reach its grid-wide barrier.  Results of
 *                      such a call are unspecified.
 *   "profile"          1: record CUDA events around every kernel the library
 *                      launches (on the launch's stream); lj_profile_report
 *                      returns the per-kernel totals.  0 (default): off.
 * lj_set_option returns LJ_OK or LJ_E_INVAL (unknown name, bad value);
 * lj_get_option returns the value, or -1 for an unknown name.
 */
int lj_set_option(const char* name, int64_t value);
int64_t lj_get_option(const char* name);

/*
 * lj_profile_report -- per-kernel timings recorded since the last report
 * (with the "profile" option on), as JSON
 *   {"<kernel>": {"launches": N, "total_ms": T, "min_ms": a, "max_ms": b}, ...}
 * written NUL-terminated into buf (len bytes).  Waits for the recorded events;
 * clears the records.  Returns the string length, or LJ_E_INVAL if buf is too
 * small (the records are then lost), LJ_E_CUDA if an event failed.
 */
int lj_profile_report(char* buf, size_t len);

/* Thread-local message describing the last error of this thread. */
const char* lj_last_error(void);

/* Library version string. */
const char* lj_version(void);

#ifdef __cplusplus
}
#endif
#endif /* LJOIN_H */
