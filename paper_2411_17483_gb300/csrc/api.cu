// C ABI entry points: argument checks, handle lifetime, host/device buffers.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "sofa_internal.cuh"

namespace sofa {

static thread_local std::string g_err;

void set_error(const std::string& msg) { g_err = msg; }

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

unsigned long long g_buf_generation = 0;

int DevBuf::ensure(size_t want) {
  if (want <= bytes && p) return 0;
  ++g_buf_generation;
  if (p) cudaFree(p);
  p = nullptr;
  bytes = 0;
  size_t grow = want + want / 4 + 256;
  cudaError_t e = dev_malloc(&p, grow);
  if (e != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
    return fail(SOFA_ERR_OOM, "scratch allocation of " + std::to_string(grow) + " bytes failed");
  }
  bytes = grow;
  return 0;
}

void DevBuf::release() {
  if (p) cudaFree(p);
  p = nullptr;
  bytes = 0;
}

cudaEvent_t Prof::get() {
  if (!pool.empty()) {
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

static const char* const kPhaseName[NPHASE] = {"sofa.qprep", "sofa.seed",  "sofa.route",    "sofa.scan",
                                                 "sofa.refine", "sofa.final", "sofa.proposal", "sofa.pool"};

void Prof::begin(int phase, cudaStream_t st, int kernels) {
  launches[phase] += kernels;
  nvtxRangePushA(kPhaseName[phase]);
  ++nvtx_depth;
  if (!on) return;
  cudaEvent_t a = get(), b = get();
  cudaEventRecord(a, st);
  open.push_back({phase, {a, b}});
}

void Prof::end(cudaStream_t st) {
  if (nvtx_depth > 0) {
    nvtxRangePop();
    --nvtx_depth;
  }
  if (!on || open.empty()) return;
  cudaEventRecord(open.back().second.second, st);
}

void Prof::unwind(int depth) {
  while (nvtx_depth > depth) {
    nvtxRangePop();
    --nvtx_depth;
  }
}

NvtxScope::NvtxScope(Prof& p, const char* name) : prof(p), depth(p.nvtx_depth) {
  nvtxRangePushA(name);
  ++prof.nvtx_depth;
}

NvtxScope::~NvtxScope() { prof.unwind(depth); }

void Prof::collect() {
  for (auto& o : open) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, o.second.first, o.second.second) == cudaSuccess) ms[o.first] += t;
    else cudaGetLastError();
    pool.push_back(o.second.first);
    pool.push_back(o.second.second);
  }
  open.clear();
}

void Prof::release() {
  collect();
  for (cudaEvent_t e : pool) cudaEventDestroy(e);
  pool.clear();
}

cudaError_t dev_malloc(void** p, size_t bytes) {
  if (const char* cap = std::getenv("SOFA_TEST_MEM_CAP")) {
    char* end = nullptr;
    const unsigned long long c = std::strtoull(cap, &end, 10);
    if (end != cap && bytes > c) {
      *p = nullptr;
      return cudaErrorMemoryAllocation;
    }
  }
  return cudaMalloc(p, bytes);
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int check_device(const Index* ix) {
  int dev = -1;
  SOFA_CUDA(cudaGetDevice(&dev));
  if (dev != ix->device)
    return fail(SOFA_ERR_INVALID_ARG, "the current device (" + std::to_string(dev) + ") is not the index's device (" +
                                          std::to_string(ix->device) + "): make that device current first");
  return 0;
}

static int num_candidates_host(int n, int pool) {
  int K = (pool <= 0) ? n / 2 : std::min(pool, n / 2);
  return 2 * K - ((n % 2 == 0 && 2 * K == n) ? 1 : 0);
}

void destroy_index(Index* ix) {
  if (!ix) return;
  void* ptrs[] = {ix->sel, ix->sel_k, ix->sel_part, ix->var, ix->basis, ix->beta, ix->edge, ix->ch, ix->ch16,
                  ix->words, ix->Z, ix->Z8, ix->s8, ix->e8, ix->VC, ix->vsr, ix->vw, ix->xn, ix->Zh, ix->VH, ix->VK, ix->perm, ix->keys, ix->keyorder, ix->tenv, ix->lenv};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  DevBuf* bufs[] = {&ix->qs.zq, &ix->qs.qv, &ix->qs.qn, &ix->qs.zqh, &ix->qs.llb, &ix->qs.thr, &ix->qs.list_d, &ix->qs.list_p,
                    &ix->qs.list_n, &ix->qs.leaf_cnt, &ix->qs.leaf_off, &ix->qs.leaf_q, &ix->qs.leaf_cursor,
                    &ix->qs.unit_off, &ix->qs.units, &ix->qs.cand_p, &ix->qs.cand_lb, &ix->qs.cand_n,
                    &ix->qs.qflag, &ix->qs.qslot, &ix->qs.qsel, &ix->qs.chunk_d, &ix->qs.chunk_p, &ix->qs.chunk_n, &ix->qs.pool_q, &ix->qs.pool_p, &ix->qs.pool_lb,
                    &ix->qs.pool_sp, &ix->qs.pool_slb, &ix->qs.qpool_cnt, &ix->qs.qpool_off, &ix->qs.qcursor,
                    &ix->qs.choff, &ix->qs.chunk_q, &ix->qs.qof, &ix->qs.counters, &ix->qs.stage_in, &ix->qs.stage_out, &ix->qs.graph_in, &ix->qs.graph_out, &ix->qs.pinned_dummy};
  for (DevBuf* b : bufs) b->release();
  if (ix->mlp) mlp_free(ix->mlp);
  ix->prof.release();
  for (auto& g : ix->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  ix->graphs.clear();
  if (ix->gstream) cudaStreamDestroy(ix->gstream);
  for (cudaEvent_t e : ix->gev)
    if (e) cudaEventDestroy(e);
  if (ix->qs.h_pinned) cudaFreeHost(ix->qs.h_pinned);
  delete static_cast<sofa_index*>(ix);
}

}  // namespace sofa

using namespace sofa;

extern "C" {

const char* sofa_last_error(void) { return g_err.c_str(); }

sofa_handle sofa_build_ex(const float* data, int64_t N, int32_t n, int32_t l, int32_t alphabet,
                          const sofa_build_opts* opts, sofa_stream stream) {
  g_err.clear();
  sofa_build_opts o;
  std::memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  auto bad = [](const std::string& m) -> sofa_handle {
    set_error(m);
    return nullptr;
  };
  if (!data) return bad("data is NULL");
  if (N < 1 || N >= ((int64_t)1 << 31)) return bad("N must lie in [1, 2^31)");
  if (n < 4 || n > 1024) return bad("series length n must lie in [4, 1024]");
  const int ncand = num_candidates_host(n, o.pool_coeffs);
  if (l < 1 || l > SOFA_MAX_WORD || l > ncand) return bad("word length l must lie in [1, min(32, candidate values)]");
  if (alphabet < 2 || alphabet > 256) return bad("alphabet must lie in [2, 256]");
  if (o.sample_ratio < 0.f || o.sample_ratio > 1.f) return bad("sample_ratio must lie in [0, 1]");
  if (o.binning < 0 || o.binning > 1) return bad("binning must be 0 or 1");
  if (o.select < 0 || o.select > 1) return bad("select must be 0 or 1");
  if (o.precision < 0 || o.precision > 2) return bad("precision must be 0, 1 or 2");
  if (o.leaf_tiles < 0 || o.leaf_tiles > 256) return bad("leaf_tiles must lie in [0, 256]");
  if (o.user_sel) {
    if (o.user_nsel < l || o.user_nsel > 2 * l) return bad("user_nsel must lie in [l, 2l]");
    for (int i = 0; i < o.user_nsel; ++i)
      if (o.user_sel[i] < 0 || o.user_sel[i] >= ncand) return bad("user_sel id out of range");
    if (!o.user_beta) return bad("user_sel needs user_beta");
  }
  sofa_index* ix = new (std::nothrow) sofa_index();
  if (!ix) return bad("host allocation failed");
  ix->N = N;
  ix->n = n;
  ix->l = l;
  ix->alpha = alphabet;
  ix->LW = l <= 16 ? 16 : 32;
  ix->NB = 2 * ix->LW;
  ix->bps = 1;
  while ((1 << ix->bps) < alphabet) ++ix->bps;
  ix->leaf_tiles = o.leaf_tiles > 0 ? o.leaf_tiles : 64;
  ix->precision = o.precision;
  cudaGetDevice(&ix->device);
  cudaStream_t st = (cudaStream_t)stream;
  const float* x = data;
  float* owned = nullptr;
  if (!is_device_ptr(data)) {
    cudaError_t e = dev_malloc((void**)&owned, (size_t)N * n * sizeof(float));
    if (e != cudaSuccess) {
      cudaGetLastError();
      destroy_index(ix);
      return bad("device allocation for the input copy failed");
    }
    e = cudaMemcpyAsync(owned, data, (size_t)N * n * sizeof(float), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) {
      cudaFree(owned);
      destroy_index(ix);
      return bad(std::string("input copy failed: ") + cudaGetErrorString(e));
    }
    x = owned;
  }
  int rc = 0;
  {
    NvtxScope range(ix->prof, "sofa_build");
    rc = build_index(ix, x, o, st);
  }
  if (owned) {
    cudaStreamSynchronize(st);
    cudaFree(owned);
  }
  if (rc) {
    std::string m = g_err;
    cudaStreamSynchronize(st);
    destroy_index(ix);
    set_error(m);
    return nullptr;
  }
  return ix;
}

sofa_handle sofa_build(const float* data, int64_t N, int32_t n, int32_t l, int32_t alphabet) {
  return sofa_build_ex(data, N, n, l, alphabet, nullptr, nullptr);
}

int sofa_insert(sofa_handle h, const float* data, int64_t N_add, sofa_stream stream) {
  g_err.clear();
  if (!h) return fail(SOFA_ERR_INVALID_ARG, "handle is NULL");
  if (N_add < 0) return fail(SOFA_ERR_INVALID_ARG, "N_add must be >= 0");
  if (N_add == 0) return 0;
  if (!data) return fail(SOFA_ERR_INVALID_ARG, "data is NULL");
  if (h->N + N_add >= ((int64_t)1 << 31)) return fail(SOFA_ERR_INVALID_ARG, "N + N_add must stay below 2^31");
  if (int rc = check_device(h)) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  SOFA_CUDA(cudaStreamSynchronize(st));
  // the query scratch is regrown on demand: release it to make room for the
  // grown index
  Index* ix = h;
  DevBuf* bufs[] = {&ix->qs.zq, &ix->qs.qv, &ix->qs.qn, &ix->qs.zqh, &ix->qs.llb, &ix->qs.thr, &ix->qs.list_d,
                    &ix->qs.list_p, &ix->qs.list_n, &ix->qs.leaf_cnt, &ix->qs.leaf_off, &ix->qs.leaf_q,
                    &ix->qs.leaf_cursor, &ix->qs.unit_off, &ix->qs.units, &ix->qs.cand_p, &ix->qs.cand_lb,
                    &ix->qs.cand_n, &ix->qs.qflag, &ix->qs.qslot, &ix->qs.qsel, &ix->qs.chunk_d, &ix->qs.chunk_p,
                    &ix->qs.chunk_n, &ix->qs.pool_q, &ix->qs.pool_p, &ix->qs.pool_lb, &ix->qs.pool_sp,
                    &ix->qs.pool_slb, &ix->qs.qpool_cnt, &ix->qs.qpool_off, &ix->qs.qcursor, &ix->qs.choff,
                    &ix->qs.chunk_q, &ix->qs.qof, &ix->qs.stage_in, &ix->qs.stage_out, &ix->qs.graph_in,
                    &ix->qs.graph_out};
  for (DevBuf* b : bufs) b->release();
  ++g_buf_generation;
  const float* x = data;
  float* owned = nullptr;
  if (!is_device_ptr(data)) {
    cudaError_t e = dev_malloc((void**)&owned, (size_t)N_add * h->n * sizeof(float));
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(SOFA_ERR_OOM, "device allocation for the input copy failed; the index is unchanged");
    }
    e = cudaMemcpyAsync(owned, data, (size_t)N_add * h->n * sizeof(float), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) {
      cudaFree(owned);
      return fail(SOFA_ERR_CUDA, std::string("input copy failed: ") + cudaGetErrorString(e));
    }
    x = owned;
  }
  int rc = 0;
  {
    NvtxScope range(ix->prof, "sofa_insert");
    rc = insert_rows(h, x, N_add, st);
  }
  if (owned) {
    cudaStreamSynchronize(st);
    cudaFree(owned);
  }
  return rc;
}

int sofa_query(sofa_handle h, const float* queries, int64_t Q, int32_t k, int64_t* idx, float* dist,
               sofa_stream stream) {
  g_err.clear();
  if (!h) return fail(SOFA_ERR_INVALID_ARG, "handle is NULL");
  if (Q < 0) return fail(SOFA_ERR_INVALID_ARG, "Q must be >= 0");
  if (k < 1 || k > SOFA_MAX_K || k > h->N) return fail(SOFA_ERR_INVALID_ARG, "k must lie in [1, min(64, N)]");
  if (Q == 0) return 0;
  if (!queries || !idx || !dist) return fail(SOFA_ERR_INVALID_ARG, "null pointer argument");
  if (Q > ((int64_t)1 << 31) / std::max(1, h->n)) return fail(SOFA_ERR_INVALID_ARG, "Q too large");
  if (int rc = check_device(h)) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  Index* ix = h;
  const bool qd = is_device_ptr(queries), id = is_device_ptr(idx), dd = is_device_ptr(dist);
  const float* qdev = queries;
  int64_t* idev = idx;
  float* ddev = dist;
  if (!qd) {
    if (int rc = ix->qs.stage_in.ensure((size_t)Q * ix->n * sizeof(float))) return rc;
    SOFA_CUDA(cudaMemcpyAsync(ix->qs.stage_in.p, queries, (size_t)Q * ix->n * sizeof(float), cudaMemcpyHostToDevice, st));
    qdev = ix->qs.stage_in.as<float>();
  }
  if (!id || !dd) {
    if (int rc = ix->qs.stage_out.ensure((size_t)Q * k * (sizeof(int64_t) + sizeof(float)))) return rc;
    if (!id) idev = ix->qs.stage_out.as<int64_t>();
    if (!dd) ddev = reinterpret_cast<float*>(ix->qs.stage_out.as<int64_t>() + Q * k);
  }
  int rc = run_query(ix, qdev, Q, k, idev, ddev, st);
  if (rc) return rc;
  if (!id) SOFA_CUDA(cudaMemcpyAsync(idx, idev, (size_t)Q * k * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  if (!dd) SOFA_CUDA(cudaMemcpyAsync(dist, ddev, (size_t)Q * k * sizeof(float), cudaMemcpyDeviceToHost, st));
  if (!qd || !id || !dd) SOFA_CUDA(cudaStreamSynchronize(st));
  return 0;
}

int sofa_query_window(sofa_handle h, const float* queries, int64_t Q, int32_t k, int32_t cap, int64_t* ids,
                      double* d2, int32_t* counts, sofa_stream stream) {
  g_err.clear();
  if (!h) return fail(SOFA_ERR_INVALID_ARG, "handle is NULL");
  if (Q < 0) return fail(SOFA_ERR_INVALID_ARG, "Q must be >= 0");
  if (k < 1 || k > SOFA_MAX_K || k > h->N) return fail(SOFA_ERR_INVALID_ARG, "k must lie in [1, min(64, N)]");
  if (cap < k || cap > SOFA_MAX_WINDOW) return fail(SOFA_ERR_INVALID_ARG, "cap must lie in [k, SOFA_MAX_WINDOW]");
  if (Q == 0) return 0;
  if (!queries || !ids || !d2 || !counts) return fail(SOFA_ERR_INVALID_ARG, "null pointer argument");
  if (Q > ((int64_t)1 << 31) / std::max(1, h->n)) return fail(SOFA_ERR_INVALID_ARG, "Q too large");
  if (int rc = check_device(h)) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  Index* ix = h;
  const bool qd = is_device_ptr(queries);
  const bool od = is_device_ptr(ids) && is_device_ptr(d2) && is_device_ptr(counts);
  const float* qdev = queries;
  int64_t* idev = ids;
  double* ddev = d2;
  int32_t* cdev = counts;
  const size_t nw = (size_t)Q * cap;
  if (!qd) {
    if (int rc = ix->qs.stage_in.ensure((size_t)Q * ix->n * sizeof(float))) return rc;
    SOFA_CUDA(cudaMemcpyAsync(ix->qs.stage_in.p, queries, (size_t)Q * ix->n * sizeof(float), cudaMemcpyHostToDevice, st));
    qdev = ix->qs.stage_in.as<float>();
  }
  if (!od) {
    if (int rc = ix->qs.stage_out.ensure(nw * (sizeof(int64_t) + sizeof(double)) + (size_t)Q * sizeof(int32_t)))
      return rc;
    idev = ix->qs.stage_out.as<int64_t>();
    ddev = reinterpret_cast<double*>(idev + nw);
    cdev = reinterpret_cast<int32_t*>(ddev + nw);
  }
  if (int rc = run_query_window(ix, qdev, Q, k, cap, idev, ddev, cdev, st)) return rc;
  if (!od) {
    SOFA_CUDA(cudaMemcpyAsync(ids, idev, nw * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    SOFA_CUDA(cudaMemcpyAsync(d2, ddev, nw * sizeof(double), cudaMemcpyDeviceToHost, st));
    SOFA_CUDA(cudaMemcpyAsync(counts, cdev, (size_t)Q * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  }
  if (!qd || !od) SOFA_CUDA(cudaStreamSynchronize(st));
  return 0;
}

int sofa_query_status(sofa_handle h) {
  if (!h) return fail(SOFA_ERR_INVALID_ARG, "handle is NULL");
  if (!h->qs.counters.p) return 0;
  int s = 0;
  SOFA_CUDA(cudaMemcpy(&s, h->qs.counters.as<unsigned long long>() + 8, sizeof(int), cudaMemcpyDeviceToHost));
  return s;
}

int sofa_stats(sofa_handle h, sofa_stats_t* out, int32_t reset) {
  if (!h || !out) return fail(SOFA_ERR_INVALID_ARG, "null argument");
  unsigned long long c[16] = {0};
  if (h->qs.counters.p) SOFA_CUDA(cudaMemcpy(c, h->qs.counters.p, sizeof(c), cudaMemcpyDeviceToHost));
  out->queries = h->stats[0];
  out->leaf_pairs = (int64_t)c[0];
  out->tile_pairs = (int64_t)c[1];
  out->candidates = (int64_t)c[2];
  out->refined = (int64_t)c[3];
  out->overflow_passes = h->stats[5];
  out->filtered = (int64_t)c[12];
  out->graph_replays = h->stats[6];
  out->graphs_recorded = h->stats[7];
  out->seed_dist_sum = (double)c[6] * 1e-6;
  out->final_dist_sum = (double)c[7] * 1e-6;
  out->value_filtered = (int64_t)c[13];
  out->dense_pairs = (int64_t)c[11];
  out->dense_passes = h->stats[1];
  out->n_leaves = h->L;
  out->n_tiles = h->T;
  if (reset) {
    if (h->qs.counters.p) {
      SOFA_CUDA(cudaMemset(h->qs.counters.p, 0, 4 * sizeof(unsigned long long)));
      SOFA_CUDA(cudaMemset(h->qs.counters.as<unsigned long long>() + 6, 0, 2 * sizeof(unsigned long long)));
      SOFA_CUDA(cudaMemset(h->qs.counters.as<unsigned long long>() + 11, 0, 3 * sizeof(unsigned long long)));
    }
    h->stats[0] = 0;
    h->stats[1] = 0;
    h->stats[5] = 0;
    h->stats[6] = 0;
  }
  return 0;
}

int sofa_set_tuning(sofa_handle h, const sofa_tuning* t) {
  if (!h || !t) return fail(SOFA_ERR_INVALID_ARG, "null argument");
  if (t->group < 0 || t->group > MAX_GROUP) return fail(SOFA_ERR_INVALID_ARG, "group must lie in [0, 64]");
  if (t->cand_cap < 0) return fail(SOFA_ERR_INVALID_ARG, "cand_cap must be >= 0");
  if (t->seed_count < 0 || t->seed_count > TILE) return fail(SOFA_ERR_INVALID_ARG, "seed_count must lie in [0, 256]");
  if (t->seed_window < 0 || t->seed_window > SEED_MAX || (t->seed_window & (t->seed_window - 1)))
    return fail(SOFA_ERR_INVALID_ARG, "seed_window must be 0 or a power of two <= 4096");
  if (t->bound_precision < 0 || t->bound_precision > 1) return fail(SOFA_ERR_INVALID_ARG, "bound_precision must be 0 or 1");
  if (t->pool_cap < 0 || t->pool_cap > ((int64_t)1 << 30)) return fail(SOFA_ERR_INVALID_ARG, "pool_cap must lie in [0, 2^30]");
  if (t->refine_filter < 0 || t->refine_filter > 2) return fail(SOFA_ERR_INVALID_ARG, "refine_filter must be 0, 1 or 2");
  if (t->refine_filter >= 1 && (!h->Z8 || !h->VC))
    return fail(SOFA_ERR_INVALID_ARG, "refine_filter needs an index built with precision 1");
  if (t->cand_budget < 0) return fail(SOFA_ERR_INVALID_ARG, "cand_budget must be >= 0");
  if (t->dense < 0 || t->dense > 2) return fail(SOFA_ERR_INVALID_ARG, "dense must be 0, 1 or 2");
  if (t->approximate < 0 || t->approximate > 1) return fail(SOFA_ERR_INVALID_ARG, "approximate must be 0 or 1");
  if (t->use_graph < 0 || t->use_graph > 1) return fail(SOFA_ERR_INVALID_ARG, "use_graph must be 0 or 1");
  if (t->series_bound < 0 || t->series_bound > 1) return fail(SOFA_ERR_INVALID_ARG, "series_bound must be 0 or 1");
  if (t->series_bound == 1 && !vscan_supported(h))
    return fail(SOFA_ERR_INVALID_ARG, "series_bound 1 needs an index built with precision >= 1");
  if (t->tile_checks < 0 || t->tile_checks > 1) return fail(SOFA_ERR_INVALID_ARG, "tile_checks must be 0 or 1");
  h->group = t->group ? t->group : 64;
  h->cand_cap = t->cand_cap ? t->cand_cap : 65536;
  h->seed_count = t->seed_count ? t->seed_count : 128;
  h->seed_window = t->seed_window ? t->seed_window : 4096;
  h->bound_precision = t->bound_precision;
  h->pool_cap = t->pool_cap;
  h->refine_filter = t->refine_filter;
  h->use_graph = t->use_graph;
  h->cand_budget = t->cand_budget ? t->cand_budget : ((int64_t)1 << 30);
  h->dense_mode = t->dense;
  h->approximate = t->approximate;
  h->series_bound = t->series_bound;
  h->tile_checks = t->tile_checks;
  return 0;
}

int sofa_info(sofa_handle h, sofa_info_t* out) {
  if (!h || !out) return fail(SOFA_ERR_INVALID_ARG, "null argument");
  out->N = h->N;
  out->n = h->n;
  out->l = h->l;
  out->alphabet = h->alpha;
  out->nsel = h->nsel;
  out->word_bytes = h->LW;
  out->nyquist_first = h->nyq_first;
  out->leaf_tiles = h->leaf_tiles;
  out->n_leaves = h->L;
  out->n_tiles = h->T;
  out->delta_data = h->delta_d;
  out->delta_query = h->delta_q;
  out->device_bytes = h->device_bytes;
  out->appended = h->N - h->Ns;
  mlp_report(h, &out->proposal_loss, &out->proposal_top1, &out->proposal_topm, &out->proposal_classes,
             &out->proposal_train);
  return 0;
}

int sofa_export_summary(sofa_handle h, int32_t* sel, double* var, float* beta) {
  if (!h) return fail(SOFA_ERR_INVALID_ARG, "handle is NULL");
  if (sel) SOFA_CUDA(cudaMemcpy(sel, h->sel, h->nsel * sizeof(int32_t), cudaMemcpyDeviceToHost));
  if (var) SOFA_CUDA(cudaMemcpy(var, h->var, h->nsel * sizeof(double), cudaMemcpyDeviceToHost));
  if (beta) SOFA_CUDA(cudaMemcpy(beta, h->beta, (size_t)h->l * (h->alpha + 1) * sizeof(float), cudaMemcpyDeviceToHost));
  return 0;
}

int sofa_export_perm(sofa_handle h, uint32_t* perm) {
  if (!h || !perm) return fail(SOFA_ERR_INVALID_ARG, "null argument");
  SOFA_CUDA(cudaMemcpy(perm, h->perm, (size_t)h->N * sizeof(uint32_t), cudaMemcpyDeviceToHost));
  return 0;
}

int sofa_export_words(sofa_handle h, uint8_t* words) {
  if (!h || !words) return fail(SOFA_ERR_INVALID_ARG, "null argument");
  std::vector<uint8_t> w((size_t)h->N * h->LW);
  std::vector<uint32_t> perm((size_t)h->N);
  SOFA_CUDA(cudaMemcpy(w.data(), h->words, w.size(), cudaMemcpyDeviceToHost));
  SOFA_CUDA(cudaMemcpy(perm.data(), h->perm, perm.size() * sizeof(uint32_t), cudaMemcpyDeviceToHost));
  for (int64_t p = 0; p < h->N; ++p)
    std::memcpy(words + (size_t)perm[p] * h->l, w.data() + (size_t)p * h->LW, h->l);
  return 0;
}

int sofa_lower_bounds(sofa_handle h, const float* queries, int64_t Q, float* out, sofa_stream stream) {
  if (!h || !queries || !out) return fail(SOFA_ERR_INVALID_ARG, "null argument");
  if (Q <= 0) return Q == 0 ? 0 : fail(SOFA_ERR_INVALID_ARG, "Q must be >= 0");
  if (!is_device_ptr(queries) || !is_device_ptr(out)) return fail(SOFA_ERR_INVALID_ARG, "device pointers required");
  if (int rc = check_device(h)) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  if (int rc = h->qs.zq.ensure((size_t)Q * h->n * sizeof(float))) return rc;
  if (int rc = h->qs.qv.ensure((size_t)Q * h->NB * sizeof(float))) return rc;
  if (int rc = launch_qprep(h, queries, Q, h->qs.zq.as<float>(), h->qs.qv.as<float>(), st)) return rc;
  return launch_lower_bounds(h, h->qs.qv.as<float>(), Q, out, st);
}

int sofa_znorm(const float* x, int64_t R, int32_t n, float* z, sofa_stream stream) {
  if (!x || !z || R < 0 || n < 1 || n > 1024) return fail(SOFA_ERR_INVALID_ARG, "bad argument");
  if (!is_device_ptr(x) || !is_device_ptr(z)) return fail(SOFA_ERR_INVALID_ARG, "device pointers required");
  return launch_znorm(x, R, n, z, (cudaStream_t)stream);
}

int sofa_set_profiling(sofa_handle h, int32_t on) {
  if (!h) return fail(SOFA_ERR_INVALID_ARG, "handle is NULL");
  h->prof.on = on != 0;
  return 0;
}

int sofa_profile(sofa_handle h, sofa_profile_t* out, int32_t reset) {
  if (!h || !out) return fail(SOFA_ERR_INVALID_ARG, "null argument");
  SOFA_CUDA(cudaDeviceSynchronize());
  h->prof.collect();
  for (int i = 0; i < 8; ++i) {
    out->ms[i] = h->prof.ms[i];
    out->launches[i] = h->prof.launches[i];
  }
  unsigned long long c[8] = {0};
  if (h->qs.counters.p) SOFA_CUDA(cudaMemcpy(c, h->qs.counters.p, sizeof(c), cudaMemcpyDeviceToHost));
  out->scan_tile_loads = (int64_t)c[4];
  out->scan_tile_checks = (int64_t)c[5];
  if (reset) {
    for (int i = 0; i < 8; ++i) {
      h->prof.ms[i] = 0;
      h->prof.launches[i] = 0;
    }
    if (h->qs.counters.p) SOFA_CUDA(cudaMemset(h->qs.counters.as<unsigned long long>() + 4, 0, 2 * sizeof(unsigned long long)));
  }
  return 0;
}

void sofa_free(sofa_handle h) {
  if (!h) return;
  cudaDeviceSynchronize();
  destroy_index(h);
}

}  // extern "C"
