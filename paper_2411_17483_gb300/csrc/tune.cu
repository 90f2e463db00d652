// Autotuner: picks the run-time tuning of an index by timing candidate
// settings on a sample of queries.  Every setting returns the same exact
// answers, so the choice only affects speed.  Choices can be cached in a text
// file, one line per (device, N, n, l, k bucket, Q bucket) key.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "sofa_internal.cuh"

namespace sofa {

static std::string tune_key(const Index* ix, int k, int64_t Q) {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp prop;
  std::memset(&prop, 0, sizeof(prop));
  cudaGetDeviceProperties(&prop, dev);
  int kb = k <= 1 ? 1 : k <= 8 ? 8 : 64;
  int64_t qb = Q <= 256 ? 256 : Q <= 4096 ? 4096 : 65536;
  std::ostringstream s;
  s << prop.name << "|N=" << ix->N << "|n=" << ix->n << "|l=" << ix->l << "|k<=" << kb << "|Q<=" << qb
    << "|filter=" << (ix->Z8 ? 1 : 0) << "|tc=" << (vscan_supported(ix) ? 1 : 0) << "|learned=" << ix->seed_mode;
  std::string key = s.str();
  for (char& c : key)
    if (c == ' ') c = '_';
  return key;
}

// A cached line holds the timed knobs; the others keep the current values.
static bool cache_lookup(const char* path, const std::string& key, const sofa_tuning& cur, sofa_tuning* t) {
  if (!path) return false;
  std::ifstream in(path);
  std::string line;
  while (std::getline(in, line)) {
    std::istringstream ls(line);
    std::string k;
    sofa_tuning c = cur;
    long long pool = 0;
    if (ls >> k >> c.group >> c.cand_cap >> c.seed_count >> c.seed_window >> c.bound_precision >> pool >>
        c.refine_filter) {
      c.pool_cap = pool;
      int sb = 0, tc = 0;
      if (ls >> sb) c.series_bound = sb;  // absent in lines written before this knob
      if (ls >> tc) c.tile_checks = tc;   // likewise
      if (k == key) {
        *t = c;
        return true;
      }
    }
  }
  return false;
}

static void cache_store(const char* path, const std::string& key, const sofa_tuning& c) {
  if (!path) return;
  std::ofstream out(path, std::ios::app);
  out << key << " " << c.group << " " << c.cand_cap << " " << c.seed_count << " " << c.seed_window << " "
      << c.bound_precision << " " << (long long)c.pool_cap << " " << c.refine_filter << " " << c.series_bound
      << " " << c.tile_checks << "\n";
}

static void apply(Index* ix, const sofa_tuning& t) {
  ix->group = t.group;
  ix->cand_cap = t.cand_cap;
  ix->seed_count = t.seed_count;
  ix->seed_window = t.seed_window;
  ix->bound_precision = t.bound_precision;
  ix->pool_cap = t.pool_cap;
  ix->refine_filter = t.refine_filter;
  ix->use_graph = t.use_graph;
  ix->cand_budget = t.cand_budget ? t.cand_budget : ((int64_t)1 << 30);
  ix->dense_mode = t.dense;
  ix->approximate = t.approximate;
  ix->series_bound = t.series_bound == 1 && vscan_supported(ix) ? 1 : 0;
  ix->tile_checks = t.tile_checks;
}

}  // namespace sofa

using namespace sofa;

extern "C" int sofa_autotune(sofa_handle h, const float* queries, int64_t Q, int32_t k, const char* cache_path,
                             sofa_tuning* chosen, sofa_stream stream) {
  if (!h || !queries || Q < 1 || k < 1 || k > SOFA_MAX_K || k > h->N)
    return fail(SOFA_ERR_INVALID_ARG, "bad autotune argument");
  if (!is_device_ptr(queries)) return fail(SOFA_ERR_INVALID_ARG, "autotune queries must be device memory");
  if (int rc = check_device(h)) return rc;
  Index* ix = h;
  cudaStream_t st = (cudaStream_t)stream;
  const std::string key = tune_key(ix, k, Q);
  sofa_tuning cur;
  std::memset(&cur, 0, sizeof(cur));
  cur.group = ix->group;
  cur.cand_cap = ix->cand_cap;
  cur.seed_count = ix->seed_count;
  cur.seed_window = ix->seed_window;
  cur.bound_precision = ix->bound_precision;
  cur.pool_cap = ix->pool_cap;
  cur.refine_filter = ix->refine_filter;
  cur.use_graph = ix->use_graph;
  cur.cand_budget = ix->cand_budget;
  cur.dense = ix->dense_mode;
  cur.approximate = ix->approximate;
  cur.series_bound = ix->series_bound;
  cur.tile_checks = ix->tile_checks;
  sofa_tuning best = cur;
  if (cache_lookup(cache_path, key, cur, &best)) {
    apply(ix, best);
    if (chosen) *chosen = best;
    return 0;
  }
  // candidate grid (all exact); the current setting is the first candidate
  std::vector<sofa_tuning> cands;
  cands.push_back(cur);
  const int groups[] = {32, 64};
  const int windows[] = {1024, 4096};
  const int counts[] = {64, 128, 256};
  const int max_bound = vscan_supported(ix) ? 1 : 0;
  for (int g : groups)
    for (int w : windows)
      for (int c : counts)
        for (int f = 0; f <= ((ix->Z8 && ix->VC) ? 2 : 0); ++f)
          for (int sb = 0; sb <= max_bound; ++sb) {
            sofa_tuning t = cur;
            t.group = g;
            t.seed_window = w;
            t.seed_count = c;
            t.refine_filter = f;
            t.bound_precision = 0;
            t.series_bound = sb;
            t.tile_checks = 0;
            cands.push_back(t);
          }
  DevBuf outi, outd;
  if (int rc = outi.ensure((size_t)Q * k * sizeof(int64_t))) return rc;
  if (int rc = outd.ensure((size_t)Q * k * sizeof(float))) return rc;
  cudaEvent_t e0, e1;
  SOFA_CUDA(cudaEventCreate(&e0));
  SOFA_CUDA(cudaEventCreate(&e1));
  float best_ms = 1e30f;
  int rc = 0;
  // one warm-up and the better of two timed runs of a candidate
  auto time_one = [&](const sofa_tuning& t, float* ms_out) {
    apply(ix, t);
    int r = run_query(ix, queries, Q, k, outi.as<int64_t>(), outd.as<float>(), st);  // warm-up
    float ms_min = 1e30f;
    for (int rep = 0; rep < 2 && !r; ++rep) {
      cudaEventRecord(e0, st);
      r = run_query(ix, queries, Q, k, outi.as<int64_t>(), outd.as<float>(), st);
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess) r = fail(SOFA_ERR_CUDA, "autotune timing failed");
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      ms_min = std::min(ms_min, ms);
    }
    *ms_out = ms_min;
    return r;
  };
  for (const sofa_tuning& t : cands) {
    float ms = 0;
    if ((rc = time_one(t, &ms))) break;
    if (ms < best_ms) {
      best_ms = ms;
      best = t;
    }
  }
  // second stage: the winner with the tensor-core bound, with and without
  // the per-tile envelope checks
  if (!rc && best.series_bound == 1) {
    sofa_tuning t = best;
    t.tile_checks = 1 - best.tile_checks;
    float ms = 0;
    rc = time_one(t, &ms);
    if (!rc && ms < best_ms) {
      best_ms = ms;
      best = t;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  outi.release();
  outd.release();
  if (rc) {
    apply(ix, cur);
    return rc;
  }
  apply(ix, best);
  cache_store(cache_path, key, best);
  if (chosen) *chosen = best;
  return 0;
}
