// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <utility>
#include <vector>

#include "../../include/sofa.h"

namespace sofa {

constexpr int TILE = 256;          // series per tile (one scan CTA pass)
constexpr int MAX_ALPHA = 256;
constexpr int KCAP = 96;           // kept-list capacity per query (>= SOFA_MAX_K + near ties)
constexpr int MAX_GROUP = 64;      // queries per scan work unit
constexpr int NB_MAX = 64;         // projection columns (2l <= 64)
constexpr int SEED_MAX = 4096;     // largest seed window

void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
// True for device or managed memory (host memory, or an unknown pointer: false).
bool is_device_ptr(const void* p);
// Every device allocation of the library.  For testing the out-of-memory
// paths without exhausting a GPU: when the environment variable
// SOFA_TEST_MEM_CAP holds a byte count, any single allocation larger than it
// fails with cudaErrorMemoryAllocation, as if the device were full.
cudaError_t dev_malloc(void** p, size_t bytes);
// SOFA_ERR_INVALID_ARG unless the calling thread's current device is the one
// the index was built or loaded on: its buffers and the kernels launched for
// it must be on the same GPU.
struct Index;
int check_device(const Index* ix);

#define SOFA_CUDA(call)                                                               \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess)                                                            \
      return ::sofa::fail(e_ == cudaErrorMemoryAllocation ? SOFA_ERR_OOM : SOFA_ERR_CUDA, \
                          std::string(#call) + ": " + cudaGetErrorString(e_));        \
  } while (0)

// Bumped whenever any scratch buffer is reallocated: recorded graphs that
// captured older addresses are then discarded.
extern unsigned long long g_buf_generation;

// Device buffers that grow on demand and are reused across calls.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  int ensure(size_t want);
  void release();
  template <class T> T* as() const { return reinterpret_cast<T*>(p); }
};

struct QueryScratch {
  DevBuf zq;        // Q x n canonical query series
  DevBuf qv;        // Q x NB projected values
  DevBuf qn;        // Q squared norms of the canonical queries (dense path)
  DevBuf zqh;       // Q x n FP16 canonical queries (dense path with FP16 operands)
  DevBuf llb;       // Q x L leaf lower bounds (half units)
  DevBuf thr;       // Q prune thresholds (half units, fp32)
  DevBuf list_d;    // Q x KCAP kept squared distances (fp32)
  DevBuf list_p;    // Q x KCAP kept sorted positions
  DevBuf list_n;    // Q kept counts
  DevBuf leaf_cnt;  // L + 1
  DevBuf leaf_off;  // L + 1
  DevBuf leaf_q;    // routed (query, leaf) pairs grouped by leaf
  DevBuf leaf_cursor;  // L fill cursors
  DevBuf unit_off;  // L + 1
  DevBuf units;     // int4 work units
  DevBuf cand_p;    // Q x cap candidate positions
  DevBuf cand_lb;   // Q x cap candidate bounds
  DevBuf cand_n;    // Q candidate counts
  DevBuf qflag;     // 2 x Q per-query flags (overflow), double-buffered
  DevBuf qslot;     // Q candidate-buffer slots of overflowed queries
  DevBuf qsel;      // Q flags: queries scanned in an overflow pass
  DevBuf pool_q, pool_p, pool_lb;   // shared candidate pool (slot, position, bound)
  DevBuf pool_sp, pool_slb;         // the pool grouped by slot
  DevBuf qpool_cnt, qpool_off, qcursor, choff, chunk_q, qof;
  DevBuf chunk_d;   // refined chunk kept lists
  DevBuf chunk_p;
  DevBuf chunk_n;
  DevBuf counters;  // misc device counters (int64)
  DevBuf graph_in, graph_out;  // fixed input / output of recorded query graphs
  int* h_pinned = nullptr;      // pinned host words for small read-backs
  DevBuf stage_in;  // staging for host queries
  DevBuf stage_out;
  DevBuf pinned_dummy;
};

struct Mlp;  // proposal network (mlp.cu)

// Phase timing with CUDA events on the launching stream, and an NVTX range
// per phase ("sofa.<phase>", pushed on the calling host thread) so that
// profilers can attribute kernels to phases.  NVTX ranges cost nothing
// unless a tool is attached.
constexpr int NPHASE = 8;
struct Prof {
  bool on = false;
  std::vector<cudaEvent_t> pool;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> open;
  double ms[NPHASE] = {0};
  long long launches[NPHASE] = {0};
  int nvtx_depth = 0;           // ranges pushed by begin() and not yet popped
  cudaEvent_t get();
  void begin(int phase, cudaStream_t st, int kernels = 1);
  void end(cudaStream_t st);
  void unwind(int depth);       // pop ranges left open by an early error return
  void collect();  // after the stream has been synchronised
  void release();
};

// Pushes an NVTX range for its scope; on exit also closes phase ranges that
// an early error return left open.
struct NvtxScope {
  Prof& prof;
  int depth;
  NvtxScope(Prof& p, const char* name);
  ~NvtxScope();
};

struct Index {
  int64_t N = 0;
  // Rows [0, Ns) are the build's key-sorted run; rows [Ns, N) were added by
  // sofa_insert and form a second key-sorted run (the appended region).
  int64_t Ns = 0;
  int n = 0, l = 0, alpha = 0, LW = 16, nsel = 0, NB = 16, bps = 8;
  int nyq_first = 0;
  int leaf_tiles = 64;
  int64_t T = 0, L = 0;
  int precision = 0;
  double delta_d = 0, delta_q = 0, vmax = 0;
  int device = 0;
  // summary
  int32_t* sel = nullptr;      // [nsel] value ids (device)
  int32_t* sel_k = nullptr;    // [nsel]
  int32_t* sel_part = nullptr; // [nsel]
  double* var = nullptr;       // [nsel] selected variances
  float* basis = nullptr;      // [n][NB] projection basis
  float* beta = nullptr;       // [LW][alpha+1]
  float2* edge = nullptr;      // [LW][256] widened (lo, hi) per symbol
  float2* ch = nullptr;        // [LW][256] (centre, half-width) per symbol
  __half2* ch16 = nullptr;     // [LW][256] (centre, -half-width) for the FP16 bound
  float outer = 0.f;           // magnitude bound of every value interval
  // layout
  uint8_t* words = nullptr;    // [N][LW] key-sorted
  float* Z = nullptr;          // [N][n] key-sorted canonical series
  int8_t* Z8 = nullptr;        // [N][n] int8 copy (refinement filter), optional
  float* s8 = nullptr;         // [N] its scales
  float* e8 = nullptr;         // [N] its residual norms (rounded up)
  int8_t* VC = nullptr;        // [N][NB] int8 codes of the selected Fourier values (value filter), optional
  float2* vsr = nullptr;       // [N] (scale, margin) of the value codes
  float* vw = nullptr;         // [NB] Eq. (1) weight of each basis column (0 for unused columns)
  float* xn = nullptr;         // [N] ||x||^2 of each canonical series (dense path)
  __half* Zh = nullptr;        // [N][n] FP16 copy of the canonical series (dense path, precision 2)
  __half* VH = nullptr;        // [N][NB] the value codes as FP16 (tensor-core series bound), with VC
  uint4* VK = nullptr;         // [N] 8 FP16 folded constants of the tensor-core test (alpha, beta, phi split)
  float tc_margin = 0.f;       // M': rounding margin of the tensor-core series bound
  bool graph_probe = false;    // the eager batch before a graph recording reads the routed totals back
  bool graph_dense = false;    // that batch's first pass took the dense contraction (the recording does too)
  bool last_dense = false;     // the last eager batch's first pass took the dense contraction
  float tc_amax = 0.f;         // A: the tensor-core test clamps sqrt(2 T) to A (it prunes nothing above)
  int64_t tc_bytes = 0;        // device bytes of VH and VK
  uint32_t* perm = nullptr;    // [N] sorted position -> original row
  uint64_t* keys = nullptr;    // [N] sorted layout keys
  uint8_t* keyorder = nullptr; // [64] key bit order (dim << 3 | bit)
  int keybits = 0;
  uint8_t* tenv = nullptr;     // [T][2][LW] tile envelopes (lo row, hi row)
  uint8_t* lenv = nullptr;     // [L][2][LW] leaf envelopes
  int64_t device_bytes = 0;
  // query state
  QueryScratch qs;
  int group = 64, cand_cap = 65536, seed_count = 128, seed_window = 4096;
  int seed_mode = 0;
  int bound_precision = 0;     // 0 FP32 series bounds, 1 FP16x2 series bounds
  int64_t pool_cap = 0;        // shared candidate pool entries (0: automatic)
  int refine_filter = 0;       // 1: int8 filter before the FP32 distance
  int use_graph = 0;           // 1: replay recorded CUDA graphs of query batches
  int64_t cand_budget = (int64_t)1 << 30;  // candidate-region entries of one overflow pass
  int approximate = 0;         // 1: answers from the seed alone
  int dense_mode = 0;          // 0: dense contraction when the leaf bound prunes little, 1: never, 2: always
  int tile_checks = 0;         // series_bound 1: per-tile envelope checks before the tensor-core bound
  int series_bound = 0;        // 0: SFA word bound (k_scan); 1: value codes on the tensor cores (k_vscan)
  struct GraphEntry {
    int64_t key[16];
    unsigned long long gen;
    cudaGraphExec_t exec;
    bool failed;
  };
  std::vector<GraphEntry> graphs;
  cudaStream_t gstream = nullptr;
  cudaEvent_t gev[2] = {nullptr, nullptr};
  int status = 0;
  int64_t stats[8] = {0};
  Mlp* mlp = nullptr;
  Prof prof;
};

// ---------------------------------------------------------------- helpers
__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Canonical z-normalisation statistics of one row, the left-to-right FP64
// sums of Sec. II Def. z-ED (explicit IEEE intrinsics: nothing is fused).
__device__ inline void znorm_stats_seq(const float* row, int n, int stride, double& mu, double& inv) {
  double s = 0.0;
  for (int t = 0; t < n; ++t) s = __dadd_rn(s, (double)row[t * stride]);
  mu = __ddiv_rn(s, (double)n);
  double ss = 0.0;
  for (int t = 0; t < n; ++t) {
    double d = __dsub_rn((double)row[t * stride], mu);
    ss = __dadd_rn(ss, __dmul_rn(d, d));
  }
  double sigma = __dsqrt_rn(__ddiv_rn(ss, (double)n));
  inv = (sigma == 0.0) ? 0.0 : __ddiv_rn(1.0, sigma);
}

__device__ inline float znorm_value(float x, double mu, double inv) {
  return __double2float_rn(__dmul_rn(__dsub_rn((double)x, mu), inv));
}

// Launch helpers implemented in the .cu files.
int build_index(Index* ix, const float* data_dev, const sofa_build_opts& o, cudaStream_t st);
// Dense path (tensor-core contraction of a whole batch against every series).
struct DenseArgs {
  const float* zq;             // Q x n canonical queries of the batch
  int Q, k, cap;
  int64_t pool_cap;
  float f_prune;
  const int* qsel;             // queries of this pass (nullptr: all)
  const int* qslot;            // their candidate slots (nullptr: identity)
  float* thr;                  // per-query thresholds, half units
  uint32_t* cand_p;
  float* cand_lb;
  int* cand_n;
  int* pool_n;
  int* pool_q;
  uint32_t* pool_p;
  float* pool_lb;
  int* qpool_cnt;
  float* dump;                 // non-null: write every d~^2 (Q x N) instead of emitting
  unsigned long long* counters;
  int* status;
  DevBuf* qn_buf;
};
bool dense_supported(const Index* ix, int k);
int launch_dense(Index* ix, const DenseArgs& a, cudaStream_t st);
int launch_row_norms(const float* Z, int64_t N, int n, float* xn, cudaStream_t st);
int insert_rows(Index* ix, const float* x_dev, int64_t A, cudaStream_t st);
float dense_margin_of(const Index* ix);

// Tensor-core series bound (vscan.cu).
struct VscanArgs {
  const int4* units;
  const int* n_units;          // device: number of units
  const int* leaf_q;
  const float* qv;
  const float* thr;
  int cap;
  const int* qslot;
  uint32_t* cand_p;
  float* cand_lb;
  int* cand_n;
  int64_t pool_cap;
  int* pool_n;
  int* pool_q;
  uint32_t* pool_p;
  float* pool_lb;
  int* qpool_cnt;
  float* dump;                 // non-null: every pair's bound (Q x N, original order) instead of emitting
  int64_t dumpQ;
  unsigned long long* counters;
  int* status;
};
int make_tc_codes(Index* ix, cudaStream_t st);
void release_tc_codes(Index* ix);
bool vscan_supported(const Index* ix);
int launch_vscan(Index* ix, const VscanArgs& a, cudaStream_t st);
double tc_margin(const Index* ix);
double tc_amax(const Index* ix);

void destroy_index(Index* ix);
int mlp_save(const Index* ix, void* file);   // FILE*; 0 or an error code
int mlp_load(Index* ix, void* file, cudaStream_t st);

// With qk (device, Q ints) each query has its own k <= k, and its results go
// to idx / dist at element offset qo[i] (device, Q int64); otherwise query i's
// k results go to offset i * k.
int run_query(Index* ix, const float* q_dev, int64_t Q, int k, int64_t* idx_dev, float* dist_dev,
              cudaStream_t st, const int* qk = nullptr, const int64_t* qo = nullptr);
int run_query_window(Index* ix, const float* q_dev, int64_t Q, int k, int cap, int64_t* wid, double* wd2, int* wcnt,
                     cudaStream_t st);
int launch_qprep(Index* ix, const float* q_dev, int64_t Q, float* zq, float* qv, cudaStream_t st);
int launch_lower_bounds(Index* ix, const float* qv, int64_t Q, float* out, cudaStream_t st);
int launch_znorm(const float* x, int64_t R, int n, float* z, cudaStream_t st);
int mlp_train(Index* ix, const sofa_train_opts& o, cudaStream_t st);
int mlp_seed(Index* ix, const float* qv, int64_t Q, int k, cudaStream_t st);
void mlp_free(Mlp* m);
const int32_t* mlp_topm(Index* ix, int* m, int64_t* block);
void mlp_report(Index* ix, double* loss, double* top1, double* topm, int64_t* classes, int64_t* n_train);

}  // namespace sofa

// The opaque handle type of the C ABI is the index itself.
struct sofa_index : public sofa::Index {};
