// Mixed workload: queries of different lengths and k over several indexes.
// The queries of each index form one batch through that index's pipeline,
// each query with its own k (the batch's largest k sizes its buffers), and
// every query's results go straight to its output offset.
#include <algorithm>
#include <map>
#include <string>
#include <vector>

#include "sofa_internal.cuh"

namespace sofa {

// One CTA per gathered row (R < 2^31 rows on gridDim.x).
__global__ void k_gather_rows(const float* __restrict__ src, const int64_t* __restrict__ offs,
                              const int32_t* __restrict__ sel, int64_t R, int n, float* __restrict__ dst) {
  const int64_t r = blockIdx.x;
  if (r >= R) return;
  const float* s = src + offs[sel[r]];
  for (int t = threadIdx.x; t < n; t += blockDim.x) dst[r * n + t] = s[t];
}

static bool dev_ptr(const void* p) { return is_device_ptr(p); }

template <class T>
static int to_host(const T* p, int64_t count, std::vector<T>& out) {
  out.resize((size_t)count);
  if (count == 0) return 0;
  if (dev_ptr(p)) SOFA_CUDA(cudaMemcpy(out.data(), p, (size_t)count * sizeof(T), cudaMemcpyDeviceToHost));
  else std::copy(p, p + count, out.begin());
  return 0;
}

struct DevVec {
  void* p = nullptr;
  ~DevVec() {
    if (p) cudaFree(p);
  }
};

}  // namespace sofa

using namespace sofa;

extern "C" int sofa_query_multi(const sofa_handle* hs, int32_t nh, const float* queries, const int64_t* q_offsets,
                                const int32_t* q_len, const int32_t* q_k, int64_t Q, int64_t* idx, float* dist,
                                const int64_t* out_offsets, sofa_stream stream) {
  if (Q < 0 || nh < 1 || !hs) return fail(SOFA_ERR_INVALID_ARG, "bad handle list or Q");
  if (Q == 0) return 0;
  if (!queries || !q_offsets || !q_len || !q_k || !idx || !dist || !out_offsets)
    return fail(SOFA_ERR_INVALID_ARG, "null pointer argument");
  for (int j = 0; j < nh; ++j)
    if (hs[j])
      if (int rc = check_device(hs[j])) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<int64_t> off, oo;
  std::vector<int32_t> len, kk;
  if (int rc = to_host(q_offsets, Q, off)) return rc;
  if (int rc = to_host(q_len, Q, len)) return rc;
  if (int rc = to_host(q_k, Q, kk)) return rc;
  if (int rc = to_host(out_offsets, Q, oo)) return rc;
  int64_t qfloats = 0, outs = 0;
  // one group per index: its queries, each with its own k, in one pipeline
  std::map<int, std::vector<int32_t>> groups;
  for (int64_t i = 0; i < Q; ++i) {
    int h = -1;
    for (int j = 0; j < nh; ++j)
      if (hs[j] && hs[j]->n == len[i]) {
        h = j;
        break;
      }
    if (h < 0) return fail(SOFA_ERR_INVALID_ARG, "query " + std::to_string(i) + ": no index of its length");
    if (kk[i] < 1 || kk[i] > SOFA_MAX_K || kk[i] > hs[h]->N) return fail(SOFA_ERR_INVALID_ARG, "bad k");
    if (off[i] < 0 || oo[i] < 0) return fail(SOFA_ERR_INVALID_ARG, "negative offset");
    qfloats = std::max(qfloats, off[i] + len[i]);
    outs = std::max(outs, oo[i] + kk[i]);
    groups[h].push_back((int32_t)i);
  }
  // device copies of the packed queries, offsets and outputs when given host memory
  DevVec dq, doff, dsel, dgq, didx, ddist, dgk, dgo;
  const float* qdev = queries;
  if (!dev_ptr(queries)) {
    SOFA_CUDA(dev_malloc(&dq.p, qfloats * sizeof(float)));
    SOFA_CUDA(cudaMemcpyAsync(dq.p, queries, qfloats * sizeof(float), cudaMemcpyHostToDevice, st));
    qdev = (const float*)dq.p;
  }
  const bool host_out = !dev_ptr(idx) || !dev_ptr(dist);
  int64_t* idev = idx;
  float* ddev = dist;
  if (host_out) {
    SOFA_CUDA(dev_malloc(&didx.p, outs * sizeof(int64_t)));
    SOFA_CUDA(dev_malloc(&ddist.p, outs * sizeof(float)));
    idev = (int64_t*)didx.p;
    ddev = (float*)ddist.p;
  }
  SOFA_CUDA(dev_malloc(&doff.p, Q * sizeof(int64_t)));
  SOFA_CUDA(cudaMemcpyAsync(doff.p, off.data(), Q * sizeof(int64_t), cudaMemcpyHostToDevice, st));
  int64_t maxRow = 0;
  for (auto& g : groups) maxRow = std::max<int64_t>(maxRow, (int64_t)g.second.size() * hs[g.first]->n);
  // per group, in group order: the queries' ids, their k and their output offsets
  std::vector<int32_t> allsel, allk;
  std::vector<int64_t> allo;
  allsel.reserve(Q);
  allk.reserve(Q);
  allo.reserve(Q);
  for (auto& g : groups)
    for (int32_t i : g.second) {
      allsel.push_back(i);
      allk.push_back(kk[i]);
      allo.push_back(oo[i]);
    }
  SOFA_CUDA(dev_malloc(&dsel.p, Q * sizeof(int32_t)));
  SOFA_CUDA(dev_malloc(&dgk.p, Q * sizeof(int32_t)));
  SOFA_CUDA(dev_malloc(&dgo.p, Q * sizeof(int64_t)));
  SOFA_CUDA(dev_malloc(&dgq.p, maxRow * sizeof(float)));
  SOFA_CUDA(cudaMemcpyAsync(dsel.p, allsel.data(), Q * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  SOFA_CUDA(cudaMemcpyAsync(dgk.p, allk.data(), Q * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  SOFA_CUDA(cudaMemcpyAsync(dgo.p, allo.data(), Q * sizeof(int64_t), cudaMemcpyHostToDevice, st));
  int64_t base = 0;
  for (auto& g : groups) {
    Index* ix = hs[g.first];
    const int64_t R = (int64_t)g.second.size();
    int kmax = 1;
    for (int32_t i : g.second) kmax = std::max(kmax, kk[i]);
    const int32_t* sel = (const int32_t*)dsel.p + base;
    k_gather_rows<<<(unsigned)R, 256, 0, st>>>(qdev, (const int64_t*)doff.p, sel, R, ix->n, (float*)dgq.p);
    SOFA_CUDA(cudaGetLastError());
    if (int rc = run_query(ix, (const float*)dgq.p, R, kmax, idev, ddev, st, (const int*)dgk.p + base,
                           (const int64_t*)dgo.p + base))
      return rc;
    base += R;
  }
  if (host_out) {
    // copy back only the slots this call wrote (outs covers all of them)
    std::vector<int64_t> hi((size_t)outs);
    std::vector<float> hd((size_t)outs);
    SOFA_CUDA(cudaMemcpyAsync(hi.data(), idev, outs * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    SOFA_CUDA(cudaMemcpyAsync(hd.data(), ddev, outs * sizeof(float), cudaMemcpyDeviceToHost, st));
    SOFA_CUDA(cudaStreamSynchronize(st));
    for (int64_t i = 0; i < Q; ++i)
      for (int j = 0; j < kk[i]; ++j) {
        idx[oo[i] + j] = hi[oo[i] + j];
        dist[oo[i] + j] = hd[oo[i] + j];
      }
  }
  SOFA_CUDA(cudaStreamSynchronize(st));
  return 0;
}
