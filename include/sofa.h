/*
 * sofa.h -- C ABI of a single-GPU (sm_103a) implementation of SOFA's exact
 * Euclidean k-NN search over z-normalised data series (Schaefer, Brand,
 * Leser, Peng, Palpanas: "Fast and Exact Similarity Search in less than a
 * Blink of an Eye").
 *
 * The hot path has two halves:
 *   1. SFA summarisation (Sec. IV "SFA", Alg. 1 MCB, Alg. 2 SFA Transform):
 *      z-normalise, project on the variance-selected Fourier values, quantise
 *      with learned per-value bins into uint8 words.
 *   2. GEMINI query answering (Sec. II-A, Sec. IV "Exact Similarity Search"):
 *      per-query lower bounds (Eq. 1 with Eq. dist_i) over leaf blocks, tiles and
 *      series of a key-sorted flat layout, pruning against the best-so-far,
 *      exact refinement of survivors and top-k.
 *
 * Conventions for every call:
 *   - Return 0 (SOFA_OK) on success or a negative SOFA_ERR_* code; handle
 *     constructors return NULL on error.  The message of the last error of the
 *     calling thread is available from sofa_last_error().
 *   - `stream` is a CUDA stream (cudaStream_t); NULL means the legacy default
 *     stream.  Device work is enqueued on it in order.
 *   - Arrays are row-major, without padding, unless stated otherwise.
 *   - Arguments are validated before any device work is enqueued; an invalid
 *     argument changes nothing.
 *   - A handle belongs to the device that was current when it was built or
 *     loaded.  Every call that launches device work for a handle (query,
 *     lower bounds, training, autotuning, the dense contraction) returns
 *     SOFA_ERR_INVALID_ARG when another device is current.
 *   - There is no CPU fallback: every step runs in this library's CUDA kernels.
 *   - Testing hook: when the environment variable SOFA_TEST_MEM_CAP holds a
 *     byte count, every device allocation of the library larger than it fails
 *     as if the device were full (calls return SOFA_ERR_OOM, constructors
 *     NULL), so the out-of-memory paths can be tested without exhausting a GPU.
 */
#ifndef SOFA_H_
#define SOFA_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sofa_index* sofa_handle;   /* opaque; owns every index buffer */
typedef struct CUstream_st* sofa_stream;  /* same type as cudaStream_t       */

enum {
  SOFA_OK = 0,
  SOFA_ERR_INVALID_ARG = -1,  /* bad size, null pointer, unsupported option     */
  SOFA_ERR_OOM = -2,          /* device allocation failed; handle unchanged     */
  SOFA_ERR_CUDA = -3,         /* a CUDA call failed; see sofa_last_error()      */
  SOFA_ERR_TIMEOUT = -4,      /* a bounded device wait ran out                  */
  SOFA_ERR_NOT_TRAINED = -5,  /* learned seeding asked for before training      */
  SOFA_ERR_TIE_OVERFLOW = -6, /* more near-tied results than the kept list holds */
  SOFA_ERR_INTERNAL = -7      /* a device-side consistency check failed: a
                                 candidate position out of range was skipped,
                                 so the answers of that call are not valid      */
};

/* Limits. */
#define SOFA_MAX_WORD 32      /* l <= 32 word values                            */
#define SOFA_MAX_K 64         /* k <= 64 neighbours per query                   */
#define SOFA_MAX_WINDOW 96    /* entries of a k-NN window (sofa_query_window)   */

/* Build options (sofa_build uses the defaults: every field zero). */
typedef struct {
  float sample_ratio;   /* Alg. 1 sampling ratio r in (0,1]; 0 -> 0.1.  Every
                           ceil(1/r - 1e-9)-th series from row 0 is sampled.   */
  int32_t binning;      /* 0 equi-depth (default), 1 equi-width (Sec. IV MCB)  */
  int32_t select;       /* 0 highest variance (Sec. IV feature selection),
                           1 first values (classical low-pass SFA)              */
  int32_t pool_coeffs;  /* candidate coefficients k <= pool; 0 = all k <= n/2  */
  int32_t leaf_tiles;   /* tiles of 256 series per leaf block (<= 256); 0 -> 64 */
  int32_t precision;    /* 0: FP32 series only; 1: also an int8 copy of every
                           canonical series with its scale and quantisation
                           error norm, and int8 codes of its selected Fourier
                           values (the refinement filters); 2: as 1, plus an
                           FP16 copy of every canonical series, which the
                           dense tensor-core contraction then reads (FP16
                           operands instead of TF32).  When n % 8 != 0 the
                           FP16 rows could not be TMA-addressed, so no FP16
                           copy is made and 2 acts as 1 (TF32 operands)     */
  /* Optional user-supplied summarisation (host pointers), replacing Alg. 1:
     user_sel: value ids in the candidate order (k ascending, real before
     imaginary, Nyquist imaginary part excluded), word values first;
     user_beta: l x (alphabet+1) fp32 breakpoints with -inf / +inf ends.    */
  const int32_t* user_sel;
  int32_t user_nsel;    /* number of ids in user_sel, l <= user_nsel <= 2l     */
  const float* user_beta;
} sofa_build_opts;

/* Index construction (Sec. IV "SOFA index": sample -> learn SFA -> transform
 * all series -> index).  1 <= N < 2^31.  data: N x n fp32 series, host or device memory,
 * read during the call only and never retained.  l: word length (1..32, at
 * most the number of candidate values); alphabet: 2..256 symbols.
 * The call synchronises `stream` before returning.  Returns NULL on error. */
sofa_handle sofa_build(const float* data, int64_t N, int32_t n, int32_t l, int32_t alphabet);
sofa_handle sofa_build_ex(const float* data, int64_t N, int32_t n, int32_t l, int32_t alphabet,
                          const sofa_build_opts* opts, sofa_stream stream);

/* Incremental insert (Sec. IV "Structure": the index takes new series, which
 * the paper's tree routes to the leaf of their word).  N_add new series of the
 * index's length n (data: N_add x n fp32, host or device memory, read during
 * the call only) are z-normalised and summarised with the index's learned
 * summary (Alg. 2; the selection and bins are not relearned), and merged by
 * layout key into the appended region: a second key-sorted run after the
 * build's, with its own tiles and leaf blocks.  New series get the row ids
 * N, N+1, ... in data order (N the size before the call).  Later queries,
 * lower bounds, the dense contraction and sofa_save cover every row; the seed
 * searches both runs by key.  A trained proposal network keeps its classes
 * (blocks of the positions it was trained on); its seed stays an upper bound,
 * so answers stay exact.  While the rows are merged the old and the grown
 * arrays are held together: SOFA_ERR_OOM, returned before any change, means
 * the device lacks that room.  N + N_add < 2^31.  The call synchronises
 * `stream`; N_add = 0 is a no-op. */
int sofa_insert(sofa_handle h, const float* data, int64_t N_add, sofa_stream stream);

/* Exact k-NN (Sec. II NN problem; k-NN as in Sec. V Table III) of Q queries.
 * queries: Q x n fp32 (raw, z-normalised inside); idx: Q x k int64 original
 * row ids; dist: Q x k fp32 z-normalised Euclidean distances (not squared),
 * ascending; distances within 1e-6 relative of a run's first are ordered by
 * ascending id.  Each pointer may be host or device memory: device buffers
 * must stay valid until `stream` reaches the end of the call; with host
 * buffers the call copies through the stream and synchronises it.
 * 1 <= k <= min(SOFA_MAX_K, N).  Q = 0 is a no-op.  Returns the status code. */
int sofa_query(sofa_handle h, const float* queries, int64_t Q, int32_t k,
               int64_t* idx, float* dist, sofa_stream stream);

/* k-NN windows for merging the answers of several indexes over disjoint row
 * ranges (series sharding: each shard searched exactly on its own, the
 * k-NN of the union merged from per-shard windows; Sec. II NN problem and the
 * k-NN extension of Sec. V Table III, with the tie rule of sofa_query).  For
 * each query: every series of this index whose distance d satisfies
 * d <= D_k + 1e-6 D_k, D_k its k-th smallest distance in this index -- the
 * only rows that can take one of the first k places of the tie rule in the
 * union, whose k-th distance is at most D_k.  ids: Q x cap int64 original
 * row ids of this index; d2: Q x cap FP64 squared distances (the
 * left-to-right FP64 sum of squared differences of the canonical series, the
 * precision in which the tie rule is decided); both ascending by (distance,
 * id) and padded with -1 / +inf; counts: Q int32 window sizes.  A window of
 * more than cap rows is cut to cap and flagged SOFA_ERR_TIE_OVERFLOW in the
 * status word (sofa_query_status).  k <= cap <= SOFA_MAX_WINDOW.  Pointers
 * may be host or device memory (same rules as sofa_query). */
int sofa_query_window(sofa_handle h, const float* queries, int64_t Q, int32_t k, int32_t cap,
                      int64_t* ids, double* d2, int32_t* counts, sofa_stream stream);

/* Mixed workload: queries of different lengths against several indexes in
 * one call.  Query i (packed at float offset q_offsets[i] of `queries`, length
 * q_len[i]) goes to the handle whose series length equals q_len[i]; its
 * q_k[i] results are written at element offset out_offsets[i] of idx / dist.
 * All arrays may be host or device memory (same rules as sofa_query). */
int sofa_query_multi(const sofa_handle* hs, int32_t nh, const float* queries,
                     const int64_t* q_offsets, const int32_t* q_len, const int32_t* q_k,
                     int64_t Q, int64_t* idx, float* dist, const int64_t* out_offsets,
                     sofa_stream stream);

/* Learned seeding (not in the paper): a 2l -> 256 -> 256 -> C GELU network
 * trained on (query SFA values -> block of the exact nearest neighbour)
 * pairs that the exact search itself labels; C blocks of ceil(N/C) consecutive
 * key-sorted series.  It only seeds the best-so-far distance; pruning and
 * refinement stay exact, so answers never depend on it. */
typedef struct {
  int64_t n_train;      /* training queries (generated on the device)          */
  int32_t n_classes;    /* C, <= 8192; 0 -> 4096                               */
  int32_t epochs;       /* 0 -> 4                                              */
  int32_t batch;        /* 0 -> 4096                                           */
  float lr;             /* Adam learning rate; 0 -> 1e-3                       */
  uint64_t seed;        /* generator seed for queries and initial weights      */
  const float* train_queries; /* optional n_train x n fp32 (host or device);
                                 NULL -> half perturbed members, half fresh
                                 random walks, from `seed`                      */
  int32_t top_m;        /* blocks probed when seeding; 0 -> 4                  */
} sofa_train_opts;
int sofa_train_proposal(sofa_handle h, const sofa_train_opts* opts, sofa_stream stream);

/* Loss and parameter gradients of the proposal network on one batch, for
 * checking the training kernels (not in the paper).  Network din -> hidden
 * -> hidden -> classes with exact-erf GELU; params and grads are flat FP32 in
 * the order W1 [din x hidden], b1, W2 [hidden x hidden], b2,
 * W3 [hidden x classes], b3; x is B x din FP32, y B int32 labels; loss is
 * the mean softmax cross-entropy (host).  Arithmetic: BF16 operands on
 * tensor cores, FP32 accumulation.  params/x/y/grads: host or device. */
int sofa_mlp_grad(int32_t din, int32_t hidden, int32_t classes, const float* params, const float* x,
                  const int32_t* y, int32_t B, float* grads, float* loss, sofa_stream stream);

/* Seed mode of later sofa_query calls: 0 plain approximate search (best leaf,
 * best tile), 1 learned proposal (needs sofa_train_proposal). */
int sofa_set_seed_mode(sofa_handle h, int32_t mode);

/* Run-time tuning knobs (any value keeps answers exact). */
typedef struct {
  int32_t group;        /* queries per scan work unit (1..64); 0 -> 64         */
  int32_t cand_cap;     /* candidate slots reserved per query (the excess goes
                           to a shared pool); 0 -> 65536                       */
  int32_t seed_count;   /* series refined by the seed; 0 -> 128 (>= k used)    */
  int32_t seed_window;  /* key-sorted series bounded by the seed (power of two
                           <= 4096); 0 -> 4096                                  */
  int32_t bound_precision; /* series-bound arithmetic: 0 FP32, 1 FP16x2 with a
                              derived rounding margin on the threshold          */
  int64_t pool_cap;     /* entries of the shared candidate pool; 0 -> sized for
                           the batch (at most 2^29).  A full pool is never an
                           error: the queries concerned are scanned again.      */
  int32_t refine_filter; /* 1: before its FP32 distance, a candidate is bounded
                            from its int8 copy (triangle inequality with the
                            stored quantisation error); 2: first from int8
                            codes of its selected Fourier values (Eq. (1) on
                            those values, triangle inequality with the stored
                            margin), then as 1.  Both need precision 1         */
  int32_t use_graph;    /* 1: each batch shape is run once eagerly and recorded
                           as a CUDA graph, later batches of that shape replay
                           it (inputs and outputs staged through fixed buffers;
                           a batch whose candidate pool ran full is recomputed
                           eagerly).  Ignored while profiling is on.            */
  int64_t cand_budget;  /* candidate-region entries one overflow pass may use
                           (queries beyond it wait for a later pass); 0 ->
                           2^30                                                 */
  int32_t dense;        /* 0: a batch whose leaf bounds pass more than half of
                           the (query, leaf block) pairs is bounded by the
                           dense tensor-core contraction instead of the series
                           scan (needs n % 4 == 0 and k <= 16); 1: never;
                           2: always when supported                            */
  int32_t approximate;  /* 1: answer from the seed alone -- the approximate
                           search (key window, and the proposal network's
                           blocks in learned mode) without the pruning scan;
                           answers are real distances re-scored in FP64 and
                           ordered by the tie rule, but not necessarily the
                           exact k-NN.  0: exact (default)                     */
  int32_t series_bound; /* series-level bound of the scan, after the leaf and
                           tile envelope checks: 0 the SFA word bound (Eq. 1
                           with Eq. dist_i, default); 1 Eq. (1) on all the
                           selected values from their int8 codes, one tcgen05
                           contraction per (work unit, tile) with a derived
                           FP16 rounding margin (needs precision >= 1).  Both
                           are lower bounds of the distance: answers do not
                           change                                               */
  int32_t tile_checks;  /* with series_bound = 1: 0 (default) every tile of a
                           leaf block that passed the leaf check is bounded on
                           the tensor cores for every query of its unit; 1 the
                           tiles are first checked against each query's SFA
                           symbol envelope (Eq. 1 with Eq. dist_i), and a tile
                           no query passes is not loaded.  Both are exact; the
                           per-series bound is tighter than a tile envelope, so
                           the checks pay only where whole tiles fail them.
                           Ignored with series_bound = 0 (the word scan always
                           checks its tiles)                                    */
} sofa_tuning;
int sofa_set_tuning(sofa_handle h, const sofa_tuning* t);

/* Autotuner: times candidate tunings (unit size, seed window and count, the
 * refinement filter when the index has its int8 copy, the series bound when
 * it has its value codes) on Q sample queries (device memory) at this k,
 * keeps the fastest and, when that uses the tensor-core bound, times it once
 * more with tile_checks flipped; applies the winner to the handle.  Every
 * candidate returns the same exact answers.  cache_path (may be NULL): a
 * text file of earlier choices, one line per (device, N, n, l, k bucket,
 * Q bucket, filter, tensor-core bound available, seed mode) key; a hit
 * applies the stored choice without timing, a miss appends the new one.
 * chosen (may be NULL) receives it. */
int sofa_autotune(sofa_handle h, const float* queries, int64_t Q, int32_t k, const char* cache_path,
                  sofa_tuning* chosen, sofa_stream stream);

/* Status word of the last sofa_query on this handle (after the caller has
 * synchronised the stream): 0 or a negative SOFA_ERR_* code. */
int sofa_query_status(sofa_handle h);

/* Counters accumulated by sofa_query since the last reset. */
typedef struct {
  int64_t queries;
  int64_t leaf_pairs;       /* (query, leaf block) pairs passing the leaf bound  */
  int64_t tile_pairs;       /* (query, tile) pairs whose series were bounded     */
  int64_t candidates;       /* series whose bound did not prune them             */
  int64_t refined;          /* series whose exact distance was computed          */
  int64_t overflow_passes;  /* extra scan passes after a full candidate buffer   */
  int64_t n_leaves;         /* leaf blocks in the index                          */
  int64_t n_tiles;          /* tiles in the index                                */
  int64_t filtered;         /* candidates read from the int8 copy only           */
  int64_t graph_replays;    /* query batches answered by replaying a CUDA graph  */
  int64_t graphs_recorded;  /* CUDA graphs recorded                              */
  double seed_dist_sum;     /* sum over queries of the seed's k-th distance      */
  double final_dist_sum;    /* sum over queries of the answer's k-th distance    */
  int64_t value_filtered;   /* candidates dropped by the value-code bound
                               (refine_filter 2)                                */
  int64_t dense_pairs;      /* (query slot, series) pairs of the dense
                               contraction (query slots x series per launch)   */
  int64_t dense_passes;     /* batch passes bounded by the dense contraction    */
} sofa_stats_t;
int sofa_stats(sofa_handle h, sofa_stats_t* out, int32_t reset);

/* Per-phase device time of sofa_query calls made while profiling is on,
 * from CUDA events recorded on the call's stream around each phase: index
 * 0 query transform, 1 seed, 2 routing, 3 series scan, 4 refinement,
 * 5 final re-score, 6 proposal network inference, 7 grouping of the
 * candidate pool.  launches[i] counts this library's kernel launches per
 * phase (counted whether or not profiling is on); scan_tile_loads counts the
 * (work unit, tile) pairs whose words the scan read. */
typedef struct {
  double ms[8];
  int64_t launches[8];
  int64_t scan_tile_loads;
  int64_t scan_tile_checks;
} sofa_profile_t;
int sofa_set_profiling(sofa_handle h, int32_t on);
int sofa_profile(sofa_handle h, sofa_profile_t* out, int32_t reset);

/* Index description. */
typedef struct {
  int64_t N;
  int32_t n, l, alphabet, nsel, word_bytes, nyquist_first, leaf_tiles;
  int64_t n_leaves, n_tiles;
  double delta_data, delta_query;  /* projection error margins in use          */
  int64_t device_bytes;            /* bytes of device memory the index holds   */
  int64_t proposal_classes;        /* trained proposal network: classes (0: none) */
  int64_t proposal_train;          /* training pairs                           */
  double proposal_loss;            /* mean cross-entropy of the last epoch     */
  double proposal_top1, proposal_topm;  /* held-out hit rate of the block of the
                                           exact nearest neighbour (top-1, top-m) */
  int64_t appended;                /* rows added by sofa_insert since the build */
} sofa_info_t;
int sofa_info(sofa_handle h, sofa_info_t* out);

/* Learned summarisation: sel (nsel value ids, word values first), var (nsel
 * FP64 sample variances), beta (l x (alphabet+1) fp32).  Host pointers; any may
 * be NULL. */
int sofa_export_summary(sofa_handle h, int32_t* sel, double* var, float* beta);

/* Words in ORIGINAL row order (N x l uint8, host) and the layout permutation
 * perm[p] = original row id at key-sorted position p (N uint32, host). */
int sofa_export_words(sofa_handle h, uint8_t* words);
int sofa_export_perm(sofa_handle h, uint32_t* perm);

/* The scan's squared lower bounds (Eq. 1 with Eq. dist_i, widened by the
 * error margins) of Q queries against every series, in ORIGINAL row order:
 * out is Q x N fp32, device memory; queries Q x n fp32 device memory. */
int sofa_lower_bounds(sofa_handle h, const float* queries, int64_t Q, float* out, sofa_stream stream);

/* Allocation-free variant of sofa_lower_bounds (the paper has no counterpart).
 * For callers that cannot have the library allocate device memory during the
 * call (a memory budget already spent, an allocator owned by the caller, a
 * thread that must not take allocation locks, or a loop that cannot absorb an
 * allocation's implicit synchronisation): its work space is a fixed 16 MiB
 * array in the library's device image, held by every GPU that loads the
 * library until the process exits.  Same arguments and output as
 * sofa_lower_bounds (device or managed pointers); Q <= 2^22 / (n + 2 *
 * word_bytes) queries per call, larger Q is rejected with SOFA_ERR_INVALID_ARG
 * before any work, and so is a call made while a device other than the
 * index's is current.  It calls no cudaMalloc or cudaFree.  The first call on a device looks
 * up the work space's device address (cudaGetSymbolAddress) and should happen
 * before any stream capture.  All calls share the one work space: calls whose
 * device work overlaps (different streams, or host threads) race and must be
 * serialised by the caller.  Nothing in it needs clearing between calls. */
int sofa_lower_bounds_noalloc(sofa_handle h, const float* queries, int64_t Q, float* out, sofa_stream stream);

/* Index persistence (the paper builds its index once per dataset, Sec. V
 * "Index creation"; this saves that work across processes).  sofa_save
 * writes every array of the index -- summary, bins, bound tables, key-sorted
 * words and series, permutation, envelopes, the optional precision copies
 * and a trained proposal network -- to `path` (overwritten; removed again on
 * failure).  sofa_load recreates a handle on the current device from such a
 * file (NULL on error, see sofa_last_error); run-time tuning starts at its
 * defaults.  The file is specific to this library version and byte order. */
int sofa_save(sofa_handle h, const char* path);
sofa_handle sofa_load(const char* path, sofa_stream stream);

/* Approximate squared distances of the dense tensor-core contraction (a test
 * and inspection aid; the paper has no counterpart).  For every query q (raw,
 * z-normalised here) and every series at sorted position p (see
 * sofa_export_perm): out[q * N + p] = ||q||^2 + ||x_p||^2 - 2 q.x_p from TF32
 * operands (FP16 when the index holds an FP16 copy, precision 2) with FP32
 * accumulation on the tensor cores.  *margin (may be NULL)
 * receives the bound M >= |out - d^2| that the query path's dense form relies
 * on.  queries (Q x n) and out (Q x N) are device memory; 1 <= Q <= 8192,
 * Q * N <= 2^31, n % 4 == 0.  Returns 0 or a negative SOFA_ERR_* code. */
int sofa_dense_sqdist(sofa_handle h, const float* queries, int64_t Q, float* out, float* margin,
                      sofa_stream stream);

/* Lower bounds of the tensor-core series bound (series_bound = 1; a test and
 * inspection aid, the paper has no counterpart): for every query q (raw,
 * z-normalised here) and every series x, out[q * N + id] (original row ids)
 * = max(sqrt(max(e~ - M', 0)) - r_x, 0)^2 <= ||q - v_x||_w^2 <= ED^2, e~ the
 * tensor-core value of ||q~ - y_x||_w^2 (Eq. 1 on the selected values, y_x the
 * value codes, r_x their margin).  *margin (may be NULL) receives M'.  queries
 * (Q x n) and out (Q x N) are device memory; 1 <= Q, Q * N <= 2^31; needs an
 * index with the value codes (precision >= 1). */
int sofa_value_bounds(sofa_handle h, const float* queries, int64_t Q, float* out, float* margin,
                      sofa_stream stream);

/* The bounded device wait every tensor-core kernel uses (a test aid; the
 * paper has no counterpart): one warp waits on a barrier that nothing ever
 * completes; the wait gives up after limit_ms (1..2000) and the kernel returns
 * normally.  Returns SOFA_ERR_TIMEOUT when the wait ran out as intended, and
 * the context stays usable. */
int sofa_wait_selftest(int32_t limit_ms, sofa_stream stream);

/* Canonical z-normalisation of R rows (Sec. II Def. z-ED) as the index uses
 * it: device pointers, R x n fp32 in and out. */
int sofa_znorm(const float* x, int64_t R, int32_t n, float* z, sofa_stream stream);

void sofa_free(sofa_handle h);
const char* sofa_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SOFA_H_ */
