// Mixed workload: queries of different lengths and k over several indexes.
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

__global__ void k_scatter_out(const int64_t* __restrict__ gi, const float* __restrict__ gd, int64_t R, int k,
                              const int32_t* __restrict__ sel, const int64_t* __restrict__ out_off,
                              int64_t* __restrict__ idx, float* __restrict__ dist) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= R * k) return;
  int64_t r = e / k;
  int j = (int)(e - r * k);
  int64_t o = out_off[sel[r]] + j;
  idx[o] = gi[e];
  dist[o] = gd[e];
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
  std::map<std::pair<int, int>, std::vector<int32_t>> groups;
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
    groups[{h, kk[i]}].push_back((int32_t)i);
  }
  // device copies of the packed queries, offsets and outputs when given host memory
  DevVec dq, doff, doo, dsel, dgi, dgd, dgq, didx, ddist;
  const float* qdev = queries;
  if (!dev_ptr(queries)) {
    SOFA_CUDA(cudaMalloc(&dq.p, qfloats * sizeof(float)));
    SOFA_CUDA(cudaMemcpyAsync(dq.p, queries, qfloats * sizeof(float), cudaMemcpyHostToDevice, st));
    qdev = (const float*)dq.p;
  }
  const bool host_out = !dev_ptr(idx) || !dev_ptr(dist);
  int64_t* idev = idx;
  float* ddev = dist;
  if (host_out) {
    SOFA_CUDA(cudaMalloc(&didx.p, outs * sizeof(int64_t)));
    SOFA_CUDA(cudaMalloc(&ddist.p, outs * sizeof(float)));
    idev = (int64_t*)didx.p;
    ddev = (float*)ddist.p;
  }
  SOFA_CUDA(cudaMalloc(&doff.p, Q * sizeof(int64_t)));
  SOFA_CUDA(cudaMalloc(&doo.p, Q * sizeof(int64_t)));
  SOFA_CUDA(cudaMemcpyAsync(doff.p, off.data(), Q * sizeof(int64_t), cudaMemcpyHostToDevice, st));
  SOFA_CUDA(cudaMemcpyAsync(doo.p, oo.data(), Q * sizeof(int64_t), cudaMemcpyHostToDevice, st));
  int64_t maxR = 0, maxRow = 0;
  for (auto& g : groups) {
    maxR = std::max<int64_t>(maxR, (int64_t)g.second.size());
    maxRow = std::max<int64_t>(maxRow, (int64_t)g.second.size() * hs[g.first.first]->n);
  }
  SOFA_CUDA(cudaMalloc(&dsel.p, Q * sizeof(int32_t)));
  SOFA_CUDA(cudaMalloc(&dgq.p, maxRow * sizeof(float)));
  SOFA_CUDA(cudaMalloc(&dgi.p, maxR * SOFA_MAX_K * sizeof(int64_t)));
  SOFA_CUDA(cudaMalloc(&dgd.p, maxR * SOFA_MAX_K * sizeof(float)));
  std::vector<int32_t> allsel;
  allsel.reserve(Q);
  for (auto& g : groups) allsel.insert(allsel.end(), g.second.begin(), g.second.end());
  SOFA_CUDA(cudaMemcpyAsync(dsel.p, allsel.data(), Q * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  int64_t base = 0;
  for (auto& g : groups) {
    Index* ix = hs[g.first.first];
    const int k = g.first.second;
    const int64_t R = (int64_t)g.second.size();
    const int32_t* sel = (const int32_t*)dsel.p + base;
    k_gather_rows<<<(unsigned)R, 256, 0, st>>>(qdev, (const int64_t*)doff.p, sel, R, ix->n, (float*)dgq.p);
    SOFA_CUDA(cudaGetLastError());
    if (int rc = run_query(ix, (const float*)dgq.p, R, k, (int64_t*)dgi.p, (float*)dgd.p, st)) return rc;
    k_scatter_out<<<(unsigned)ceil_div(R * k, 256), 256, 0, st>>>((const int64_t*)dgi.p, (const float*)dgd.p, R, k,
                                                                   sel, (const int64_t*)doo.p, idev, ddev);
    SOFA_CUDA(cudaGetLastError());
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
