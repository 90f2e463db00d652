// GEMINI exact k-NN query kernels (Sec. II-A; Sec. IV "Exact Similarity
// Search", "SOFA LBD calculation"): leaf / tile / series SFA lower bounds
// against the best-so-far, exact refinement of survivors and top-k.
//
// Bounds are kept in "half units": acc = sum_j c_j m_j^2 with c_j = 1, or 1/2
// for a Nyquist value (always word position 0), so that LB^2 = 2 acc matches
// Eq. 1's weights (2 for 0<k<n/2, 1 for k=n/2).  m_j is Eq. dist_i against
// the symbol interval widened by the projection error margins.
#include <cfloat>
#include <algorithm>
#include <vector>
#include <cmath>

#include "sofa_internal.cuh"
#include "bounds.cuh"

namespace sofa {



constexpr int LEARN_CAP = 2048;  // learned-seed candidates kept beside the key window
constexpr int SEED_TL = 512;     // tiles of a predicted block examined per pass

struct QueryParams {
  int64_t N, T, L;
  int64_t Ns;     // rows of the build's key-sorted run; [Ns, N) is the appended run
  int n, NB, leaf_tiles, k, cap, group, seed_count, seed_window;
  float f_prune;  // threshold = d2_kth * f_prune / 2 (half units)
  float f_keep;   // kept list: d2 <= d2_kth * f_keep
  // per-query k of a mixed batch (nullptr: every query has k), and the
  // element offset of each query's k results in idx / dist
  const int* qk;
  const int64_t* qo;
};

// k of query q of the batch (k is the batch's largest, which sizes every
// buffer and, in the dense contraction, sets a threshold that is valid for
// every smaller k).
__device__ __forceinline__ int kq(const QueryParams& P, int64_t q) { return P.qk ? P.qk[q] : P.k; }

// Series bound from a word: m_j = max(|q_j - c_j| - h_j, 0) with (c, h) the
// symbol's widened interval as centre / half-width.
template <int LW, bool NYQ>
__device__ __forceinline__ float word_bound(const float* c, const float* h, const float* q) {
  float acc = 0.f;
#pragma unroll
  for (int j = 0; j < LW; ++j) {
    float m = fmaxf(fabsf(q[j] - c[j]) - h[j], 0.f);
    float mm = (NYQ && j == 0) ? 0.5f * m : m;
    acc = fmaf(mm, m, acc);
  }
  return acc;
}

template <int LW>
__device__ __forceinline__ void load_word_bounds(const uint8_t* __restrict__ words, int64_t p, bool valid,
                                                 const float2* __restrict__ ch, float* c, float* h) {
  uint32_t w32[LW / 4];
  if (valid) {
    const uint4* w = reinterpret_cast<const uint4*>(words + p * LW);
#pragma unroll
    for (int i = 0; i < LW / 16; ++i) {
      uint4 v = __ldg(w + i);
      w32[4 * i] = v.x;
      w32[4 * i + 1] = v.y;
      w32[4 * i + 2] = v.z;
      w32[4 * i + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int i = 0; i < LW / 4; ++i) w32[i] = 0u;
  }
#pragma unroll
  for (int j = 0; j < LW; ++j) {
    float2 v = ch[j * MAX_ALPHA + ((w32[j >> 2] >> (8 * (j & 3))) & 0xFFu)];
    c[j] = v.x;
    h[j] = v.y;
  }
}

// FP32 squared distance of series p computed by a group of 4 lanes (sub =
// lane & 3); every lane of the warp must call it (the group reduction uses
// shuffles), inactive groups pass active = false.
__device__ __forceinline__ float group4_sqdist(const float* __restrict__ zq, const float* __restrict__ Z, int64_t p,
                                               int n, int sub, bool active) {
  float acc = 0.f;
  if (active) {
    const float* row = Z + p * n;
    if ((n & 3) == 0) {
      const float4* r4 = reinterpret_cast<const float4*>(row);
      const float4* q4 = reinterpret_cast<const float4*>(zq);
#pragma unroll 16
      for (int i = sub; i < n / 4; i += 4) {
        float4 x = __ldg(r4 + i);
        float4 y = q4[i];
        float d0 = y.x - x.x, d1 = y.y - x.y, d2 = y.z - x.z, d3 = y.w - x.w;
        acc = fmaf(d0, d0, acc);
        acc = fmaf(d1, d1, acc);
        acc = fmaf(d2, d2, acc);
        acc = fmaf(d3, d3, acc);
      }
    } else {
      for (int t = sub; t < n; t += 4) {
        float d = zq[t] - __ldg(row + t);
        acc = fmaf(d, d, acc);
      }
    }
  }
  acc += __shfl_xor_sync(0xFFFFFFFFu, acc, 1);
  acc += __shfl_xor_sync(0xFFFFFFFFu, acc, 2);
  return acc;
}

// FP32 squared distance between the canonical query and the int8 copy of
// series p, by one thread (a 256-value row is 16 consecutive 16-byte loads).
// The copy's values s * v_t are exact reals and fmaf(-s, v, q) rounds once.
__device__ __forceinline__ float thread_sqdist8(const float* __restrict__ zq, const int8_t* __restrict__ Z8, float sc,
                                                int64_t p, int n) {
  const int8_t* row = Z8 + p * n;
  float a0 = 0.f, a1 = 0.f;
  if ((n & 15) == 0) {
    const uint4* r4 = reinterpret_cast<const uint4*>(row);
    for (int i = 0; i < n / 16; ++i) {
      const uint4 w = __ldg(r4 + i);
      const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
      for (int b = 0; b < 4; ++b)
#pragma unroll
        for (int j = 0; j < 4; j += 2) {
          const float v0 = (float)((int)(ws[b] << (24 - 8 * j)) >> 24);
          const float v1 = (float)((int)(ws[b] << (16 - 8 * j)) >> 24);
          const float d0 = fmaf(-sc, v0, zq[16 * i + 4 * b + j]);
          const float d1 = fmaf(-sc, v1, zq[16 * i + 4 * b + j + 1]);
          a0 = fmaf(d0, d0, a0);
          a1 = fmaf(d1, d1, a1);
        }
    }
  } else {
    for (int t = 0; t < n; ++t) {
      const float d = fmaf(-sc, (float)row[t], zq[t]);
      a0 = fmaf(d, d, a0);
    }
  }
  return a0 + a1;
}

// Bitonic sort of `len` (power of two) 64-bit keys in shared memory by the
// whole block.
__device__ inline void block_bitonic(unsigned long long* key, int len) {
  for (int size = 2; size <= len; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      __syncthreads();
      for (int i = threadIdx.x; i < len / 2; i += blockDim.x) {
        int lo = 2 * i - (i & (stride - 1));
        int hi = lo + stride;
        bool up = ((lo & size) == 0);
        unsigned long long a = key[lo], b = key[hi];
        if ((a > b) == up) {
          key[lo] = b;
          key[hi] = a;
        }
      }
    }
  }
  __syncthreads();
}

// The kk smallest of key[0, len) in ascending order in key[0, kp), kp = kk
// rounded up to a power of two; returns the number of leading entries it
// sorted (kp, or len when it sorted them all).  len is a power of two.  Each
// warp sorts its len / 8 keys (warp-synchronous bitonic sort), then three
// tournament levels keep the kp smallest of two sorted runs: with A and B
// ascending, C_i = min(A_i, B_{kp-1-i}) rises then falls and holds exactly
// the kp smallest of A and B, so a bitonic merge sorts it.  A run shorter
// than kp falls back to the full block sort.  All threads of the block call
// it with the keys in place; the rest of key[] is left unordered.
__device__ int block_topk(unsigned long long* key, int len, int kk) {
  int kp = 1;
  while (kp < kk) kp <<= 1;
  const int chunk = len >> 3;
  if (blockDim.x != 256 || len < 256 || chunk < kp) {
    block_bitonic(key, len);
    return len;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  unsigned long long* run = key + warp * chunk;
  for (int size = 2; size <= chunk; size <<= 1)
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      __syncwarp();
      for (int i = lane; i < (chunk >> 1); i += 32) {
        const int lo = 2 * i - (i & (stride - 1)), hi = lo + stride;
        const bool up = (lo & size) == 0;
        const unsigned long long a = run[lo], b = run[hi];
        if ((a > b) == up) {
          run[lo] = b;
          run[hi] = a;
        }
      }
    }
  for (int step = 1; step < 8; step <<= 1) {
    const int npair = 4 / step;
    __syncthreads();
    for (int e = threadIdx.x; e < npair * kp; e += blockDim.x) {
      const int pr = e / kp, i = e - pr * kp;
      unsigned long long* A = key + (2 * pr * step) * chunk;
      const unsigned long long b = key[(2 * pr * step + step) * chunk + kp - 1 - i];
      if (b < A[i]) A[i] = b;
    }
    for (int stride = kp >> 1; stride > 0; stride >>= 1) {
      __syncthreads();
      for (int e = threadIdx.x; e < npair * (kp >> 1); e += blockDim.x) {
        const int pr = e / (kp >> 1), i = e - pr * (kp >> 1);
        unsigned long long* A = key + (2 * pr * step) * chunk;
        const int lo = 2 * i - (i & (stride - 1)), hi = lo + stride;
        const unsigned long long a = A[lo], b = A[hi];
        if (a > b) {
          A[lo] = b;
          A[hi] = a;
        }
      }
    }
  }
  __syncthreads();
  return kp;
}

__device__ __forceinline__ unsigned long long pack_key(float v, uint32_t p) {
  return ((unsigned long long)__float_as_uint(v) << 32) | p;  // v >= 0: bit order = value order
}

// Write the kept list of a query from `len` sorted (d2, pos) keys: the first
// k entries and every later one within the tie window of the k-th.  Sets the
// prune threshold.  Returns false when entries inside the window were dropped.
__device__ inline bool emit_list(const unsigned long long* key, int len, const QueryParams& P, int64_t q,
                                 float* list_d, uint32_t* list_p, int* list_n, float* thr) {
  __shared__ int s_cnt;
  const int K = kq(P, q);
  const float dk = __uint_as_float((uint32_t)(key[K - 1] >> 32));
  const float lim = __fmul_ru(dk, P.f_keep);
  if (threadIdx.x == 0) s_cnt = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < len; i += blockDim.x) {
    float d = __uint_as_float((uint32_t)(key[i] >> 32));
    if (i < K || d <= lim) atomicMax(&s_cnt, i + 1);
  }
  __syncthreads();
  const int cnt = s_cnt;
  const int keep = cnt < KCAP ? cnt : KCAP;
  for (int i = threadIdx.x; i < keep; i += blockDim.x) {
    list_d[q * KCAP + i] = __uint_as_float((uint32_t)(key[i] >> 32));
    list_p[q * KCAP + i] = (uint32_t)key[i];
  }
  if (threadIdx.x == 0) {
    list_n[q] = keep;
    thr[q] = __fmul_ru(__fmul_ru(dk, P.f_prune), 0.5f);
  }
  __syncthreads();
  return cnt <= KCAP;
}

// ------------------------------------------------------------------------
// Leaf bounds of every (query, leaf block) pair -> llb, the routing input
// (Eq. 1 with Eq. dist_i against each leaf block's symbol envelope): the
// bound of env_bound, term for term.  A CTA takes 256 leaf blocks and 64
// queries.  Each leaf block's LW intervals [edge(lo).lo, edge(hi).hi] are
// formed once; then a warp bounds its 32 leaf blocks (lanes) against one
// query at a time: the query's values are broadcast, the intervals are read
// value-major (no bank conflicts), the stores are coalesced.
constexpr int LB_LEAVES = 256, LB_QUERIES = 64;
template <int LW, bool NYQ>
__global__ void __launch_bounds__(256) k_leaf_bounds(int64_t Q, int64_t L, int NBq, const float* __restrict__ qv,
                                                     const uint8_t* __restrict__ lenv,
                                                     const float2* __restrict__ edge, float* __restrict__ llb) {
  extern __shared__ float2 s_lint[];  // [LW][LB_LEAVES]
  __shared__ float s_qv[LB_QUERIES][LW];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t b0 = (int64_t)blockIdx.x * LB_LEAVES, q0 = (int64_t)blockIdx.y * LB_QUERIES;
  const int nb = (int)(L - b0 < LB_LEAVES ? L - b0 : LB_LEAVES);
  const int nq = (int)(Q - q0 < LB_QUERIES ? Q - q0 : LB_QUERIES);
  if (tid < nb) {
    const uint32_t* e32 = reinterpret_cast<const uint32_t*>(lenv + (b0 + tid) * 2 * LW);
#pragma unroll
    for (int w = 0; w < LW / 4; ++w) {
      const uint32_t lo = e32[w], hi = e32[LW / 4 + w];
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int j = 4 * w + b;
        s_lint[j * LB_LEAVES + tid] = make_float2(edge[j * MAX_ALPHA + ((lo >> (8 * b)) & 0xFFu)].x,
                                                  edge[j * MAX_ALPHA + ((hi >> (8 * b)) & 0xFFu)].y);
      }
    }
  }
  for (int e = tid; e < nq * LW; e += blockDim.x) {
    const int g = e / LW, j = e - g * LW;
    s_qv[g][j] = qv[(q0 + g) * NBq + j];
  }
  __syncthreads();
  const int leaf = warp * 32 + lane;
  if (warp * 32 >= nb) return;  // no barrier follows
  const int lf = leaf < nb ? leaf : 0;
  for (int g = 0; g < nq; ++g) {
    float acc = 0.f;
#pragma unroll
    for (int j = 0; j < LW; ++j) {
      const float2 iv = s_lint[j * LB_LEAVES + lf];
      const float qj = s_qv[g][j];
      const float m = fmaxf(fmaxf(iv.x - qj, qj - iv.y), 0.f);
      const float mm = (NYQ && j == 0) ? 0.5f * m : m;
      acc = fmaf(mm, m, acc);
    }
    if (leaf < nb) llb[(q0 + g) * L + b0 + leaf] = acc;
  }
}

// ------------------------------------------------------------------------
// Seed (plain approximate search, Sec. IV "Exact Similarity Search": the
// series nearest the query's own word in the key order, and the proposal
// network's blocks, give the first best-so-far).  One CTA per query (the
// leaf bounds, the routing input, come from k_leaf_bounds): (2) the query's
// key and its insertion point in each key-sorted run; (3) the key window's
// series bounds, the seed_count smallest refined in FP32; (4) kept list and
// prune threshold.
template <int LW, bool NYQ>
__global__ void __launch_bounds__(256) k_seed(QueryParams P, const float* __restrict__ qv,
                                              const float* __restrict__ zq,
                                              const uint8_t* __restrict__ tenv, const uint8_t* __restrict__ words,
                                              const float* __restrict__ Z, const float2* __restrict__ edge,
                                              const float2* __restrict__ ch, const float* __restrict__ beta,
                                              int alpha, int l, const uint64_t* __restrict__ keys,
                                              const uint8_t* __restrict__ keyorder, int keybits,
                                              float* __restrict__ list_d,
                                              uint32_t* __restrict__ list_p, int* __restrict__ list_n,
                                              float* __restrict__ thr, int* __restrict__ status,
                                              unsigned long long* __restrict__ counters,
                                              const int32_t* __restrict__ topm, int top_m, int64_t block) {
  extern __shared__ float4 ssm[];
  float* szq = reinterpret_cast<float*>(ssm);            // n
  __shared__ float sq[LW];
  __shared__ unsigned long long skey[SEED_MAX];
  const int64_t q = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid < LW) sq[tid] = qv[q * P.NB + tid];
  for (int t = tid; t < P.n; t += blockDim.x) szq[t] = zq[q * P.n + t];
  __syncthreads();


  // (2) approximate search: the query's own SFA word and layout key, and the
  // key-sorted position where it would be inserted (the flat layout's analogue
  // of descending the tree to the leaf of the query's word)
  __shared__ uint8_t qsym[LW];
  __shared__ uint64_t s_qkey;
  __shared__ int64_t s_lo, s_hi;
  __shared__ int s_less;
  if (tid < LW) {
    int c = 0;
    if (tid < l) {
      const float* bj = beta + (int64_t)tid * (alpha + 1);
      for (int step = 128; step > 0; step >>= 1)
        if (c + step <= alpha - 1 && bj[c + step] <= sq[tid]) c += step;
    }
    qsym[tid] = (uint8_t)c;
  }
  __syncthreads();
  if (tid == 0) {
    uint64_t key = 0;
    for (int t = 0; t < keybits; ++t) {
      const int d = keyorder[t] >> 3, bb = keyorder[t] & 7;
      key |= (uint64_t)((qsym[d] >> bb) & 1u) << (63 - t);
    }
    s_qkey = key;
  }
  // The layout holds one or two key-sorted runs: the build's [0, Ns) and the
  // rows added since, [Ns, N).  In each, a 256-ary search finds the first
  // position a whose key is >= the query's key.  Invariant: keys[p] < qkey for
  // p < lo, keys[p] >= qkey for p >= hi.  Each round probes lo + span*t/256;
  // the probes below the key form a prefix of m, so a lies in
  // [probe m-1 + 1, probe m]; lo grows by >= 1 or hi becomes lo.
  int64_t ins[2] = {0, P.Ns};
  for (int run = 0; run < 2; ++run) {
    const int64_t r_lo = run == 0 ? 0 : P.Ns, r_hi = run == 0 ? P.Ns : P.N;
    if (r_hi <= r_lo) continue;
    if (tid == 0) {
      s_lo = r_lo;
      s_hi = r_hi;
    }
    __syncthreads();
    for (int it = 0; it < 64; ++it) {
      const int64_t lo = s_lo, hi = s_hi;
      if (hi <= lo) break;
      const int64_t span = hi - lo;
      if (tid == 0) s_less = 0;
      __syncthreads();
      const int64_t pos = lo + (span * tid) / 256;
      if (keys[pos] < s_qkey) atomicAdd(&s_less, 1);
      __syncthreads();
      if (tid == 0) {
        const int m = s_less;
        if (m == 0) {
          s_hi = lo;
        } else {
          s_lo = lo + (span * (m - 1)) / 256 + 1;
          if (m < 256) s_hi = lo + (span * m) / 256;
        }
      }
      __syncthreads();
    }
    ins[run] = s_lo;
    __syncthreads();
  }
  // the key window: W consecutive positions around each insertion point, at
  // most half of them in the appended run while the build's run has room
  const int64_t W = P.N < P.seed_window ? P.N : P.seed_window;
  const int64_t na = P.Ns, nb = P.N - P.Ns;
  int64_t Wb = nb < W / 2 ? nb : W / 2;
  const int64_t Wa = na < W - Wb ? na : W - Wb;
  if (Wa + Wb < W) Wb = nb < W - Wa ? nb : W - Wa;
  int64_t p0a = ins[0] - Wa / 2;
  if (p0a > na - Wa) p0a = na - Wa;
  if (p0a < 0) p0a = 0;
  int64_t p0b = ins[1] - Wb / 2;
  if (p0b > P.N - Wb) p0b = P.N - Wb;
  if (p0b < P.Ns) p0b = P.Ns;

  // (3) series bounds of the key window; its seed_count smallest are the
  // approximate answer's candidates
  for (int i = tid; i < P.seed_window; i += blockDim.x) {
    const int64_t p = i < Wa ? p0a + i : p0b + (i - Wa);
    const bool valid = i < Wa + Wb;
    float c[LW], h[LW];
    load_word_bounds<LW>(words, p, valid, ch, c, h);
    skey[i] = valid ? pack_key(word_bound<LW, NYQ>(c, h, sq), (uint32_t)p) : ~0ull;
  }
  const int Kq = kq(P, q);
  int cnt = P.seed_count > Kq ? P.seed_count : Kq;
  if (cnt > W) cnt = (int)W;
  // only the window's cnt smallest bounds are used below
  block_topk(skey, P.seed_window, cnt);
  // learned seeding: every series of the proposal network's top-m blocks whose
  // bound beats the window's cnt-th joins the candidates (up to LEARN_CAP)
  __shared__ int s_nl2;
  if (tid == 0) s_nl2 = 0;
  __syncthreads();
  if (topm) {
    const float tau = __uint_as_float((uint32_t)(skey[cnt - 1] >> 32));
    __shared__ int s_tl[SEED_TL];
    __shared__ int s_nt;
    for (int i = 0; i < top_m; ++i) {
      const int64_t b = topm[q * top_m + i];
      const int64_t lo = b * block;
      const int64_t hi = (b + 1) * block < P.N ? (b + 1) * block : P.N;
      for (int64_t tb = lo / TILE; tb * TILE < hi; tb += SEED_TL) {
        // tiles of the block whose envelope bound is below the cut-off
        if (tid == 0) s_nt = 0;
        __syncthreads();
        for (int j = tid; j < SEED_TL; j += blockDim.x) {
          const int64_t t = tb + j;
          if (t * TILE < hi && t < P.T && env_bound<LW, NYQ>(tenv + t * 2 * LW, sq, edge) < tau)
            s_tl[atomicAdd(&s_nt, 1)] = (int)(t - tb);
        }
        __syncthreads();
        const int nt2 = s_nt;
        // surviving tiles four at a time: the words of all four are loaded
        // before any bound, so their global-memory latencies overlap
        for (int j0 = 0; j0 < nt2; j0 += 4) {
          uint4 wv[4][LW / 16];
          int64_t pp[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            pp[u] = j0 + u < nt2 ? (tb + s_tl[j0 + u]) * TILE + tid : -1;
            const bool ok = pp[u] >= lo && pp[u] < hi;
            const uint4* wp = reinterpret_cast<const uint4*>(words + (ok ? pp[u] : 0) * LW);
#pragma unroll
            for (int i4 = 0; i4 < LW / 16; ++i4) wv[u][i4] = ok ? __ldg(wp + i4) : make_uint4(0u, 0u, 0u, 0u);
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            if (!(pp[u] >= lo && pp[u] < hi)) continue;
            const uint32_t* w32 = reinterpret_cast<const uint32_t*>(wv[u]);
            float c[LW], h[LW];
#pragma unroll
            for (int j = 0; j < LW; ++j) {
              const float2 v = ch[j * MAX_ALPHA + ((w32[j >> 2] >> (8 * (j & 3))) & 0xFFu)];
              c[j] = v.x;
              h[j] = v.y;
            }
            const float a = word_bound<LW, NYQ>(c, h, sq);
            if (a < tau) {
              const int slot = atomicAdd(&s_nl2, 1);
              if (slot < LEARN_CAP) skey[cnt + slot] = pack_key(a, (uint32_t)pp[u]);
            }
          }
        }
        __syncthreads();
      }
    }
  }
  __syncthreads();
  int len = cnt + (s_nl2 < LEARN_CAP ? s_nl2 : LEARN_CAP);
  int sorted_n = len;  // the leading entries in ascending order
  if (len > cnt) {
    int pw2 = 1;
    while (pw2 < len) pw2 <<= 1;
    for (int i = len + tid; i < pw2; i += blockDim.x) skey[i] = ~0ull;
    // the cnt smallest, with room for repeats of window entries
    const int sn = block_topk(skey, pw2, 2 * cnt < pw2 ? 2 * cnt : pw2);
    sorted_n = sn < len ? sn : len;
  }
  __shared__ int s_avail;
  if (tid == 0) {  // a learned block may overlap the key window: drop repeats
    int u = 0;
    for (int i = 0; i < sorted_n && u < cnt; ++i) {
      if (skey[i] == ~0ull) break;
      if (u == 0 || skey[i] != skey[u - 1]) skey[u++] = skey[i];
    }
    s_avail = u;
  }
  __syncthreads();
  if (cnt > s_avail) cnt = s_avail;
  __shared__ float sd[TILE];
  __shared__ uint32_t sp[TILE];
  for (int base = 0; base < cnt; base += 64) {  // same 4-lane FP32 sum as the refinement
    const int i = base + warp * 8 + (lane >> 2);
    const bool active = i < cnt;
    const uint32_t p = active ? (uint32_t)skey[i] : 0u;
    const float d2 = group4_sqdist(szq, Z, p, P.n, lane & 3, active);
    if (active && (lane & 3) == 0) {
      sd[i] = d2;
      sp[i] = p;
    }
  }
  __syncthreads();
  // (4) sort the refined entries by (d2, pos) and emit the kept list
  for (int i = tid; i < TILE; i += blockDim.x) skey[i] = i < cnt ? pack_key(sd[i], sp[i]) : ~0ull;
  block_bitonic(skey, TILE);
  if (!emit_list(skey, cnt, P, q, list_d, list_p, list_n, thr) && tid == 0) atomicExch(status, SOFA_ERR_TIE_OVERFLOW);
  if (tid == 0)
    atomicAdd(counters + 6, (unsigned long long)(1e6 * sqrt((double)__uint_as_float((uint32_t)(skey[Kq - 1] >> 32)))));
}

// ------------------------------------------------------------------------
// Routing: every (query, leaf block) whose leaf bound does not exceed the
// query's threshold goes to that leaf's query list (only queries with
// qsel[q] != 0 when qsel is given).  Count pass, then fill pass.
__global__ void k_route_count(int64_t Q, int64_t L, const float* __restrict__ llb, const float* __restrict__ thr,
                              const int* __restrict__ qsel, int* __restrict__ leaf_cnt,
                              unsigned long long* __restrict__ counters) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool take = false;
  if (e < Q * L) {
    int64_t q = e / L, b = e - q * L;
    take = (!qsel || qsel[q]) && llb[e] <= thr[q];
    if (take) atomicAdd(leaf_cnt + b, 1);
  }
  unsigned m = __ballot_sync(0xFFFFFFFFu, take);
  if ((threadIdx.x & 31) == 0 && m) atomicAdd(counters + 0, (unsigned long long)__popc(m));
}

// Exclusive scans over leaves of the routed counts and of the unit counts
// ceil(cnt / group); totals land at index L.  One CTA of 1024 threads.
__global__ void __launch_bounds__(1024) k_leaf_scan(int64_t L, int group, const int* __restrict__ leaf_cnt,
                                                    int* __restrict__ leaf_off, int* __restrict__ unit_off,
                                                    int* __restrict__ leaf_cursor) {
  __shared__ long long s1[1024], s2[1024];
  const int tid = threadIdx.x;
  const int64_t per = (L + 1023) / 1024;
  const int64_t b0 = tid * per, b1 = min(L, b0 + per);
  long long a = 0, u = 0;
  for (int64_t b = b0; b < b1; ++b) {
    a += leaf_cnt[b];
    u += (leaf_cnt[b] + group - 1) / group;
  }
  s1[tid] = a;
  s2[tid] = u;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    long long x1 = tid >= o ? s1[tid - o] : 0, x2 = tid >= o ? s2[tid - o] : 0;
    __syncthreads();
    s1[tid] += x1;
    s2[tid] += x2;
    __syncthreads();
  }
  long long ra = s1[tid] - a, ru = s2[tid] - u;
  for (int64_t b = b0; b < b1; ++b) {
    leaf_off[b] = (int)ra;
    unit_off[b] = (int)ru;
    leaf_cursor[b] = 0;
    ra += leaf_cnt[b];
    ru += (leaf_cnt[b] + group - 1) / group;
  }
  if (tid == 1023) {
    leaf_off[L] = (int)s1[1023];
    unit_off[L] = (int)s2[1023];
  }
}

__global__ void k_route_fill(int64_t Q, int64_t L, const float* __restrict__ llb, const float* __restrict__ thr,
                             const int* __restrict__ qsel, const int* __restrict__ leaf_off,
                             int* __restrict__ leaf_cursor, int* __restrict__ leaf_q) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= Q * L) return;
  int64_t q = e / L, b = e - q * L;
  if ((!qsel || qsel[q]) && llb[e] <= thr[q]) {
    int pos = atomicAdd(leaf_cursor + b, 1);
    leaf_q[leaf_off[b] + pos] = (int)q;
  }
}

// Work units (leaf, first list entry, count <= group).
__global__ void k_units(int64_t L, int group, const int* __restrict__ leaf_cnt, const int* __restrict__ leaf_off,
                        const int* __restrict__ unit_off, int4* __restrict__ units) {
  int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= L) return;
  int c = leaf_cnt[b], u0 = unit_off[b];
  for (int i = 0, u = 0; i < c; i += group, ++u)
    units[u0 + u] = make_int4((int)b, leaf_off[b] + i, min(group, c - i), 0);
}

// ------------------------------------------------------------------------
// The series scan (Alg. 3's bound, batched).  A persistent CTA takes work
// units (leaf block, up to 64 queries).  First every (tile, query) envelope
// check of the unit is done in one parallel pass into a per-tile query mask.
// Then each thread walks the tiles with a non-empty mask on its own series
// (no barriers): it reads the word once, gathers its symbol intervals from
// shared memory once, and evaluates the bound for every query of the mask in
// chunks of 8 values; after each chunk a warp vote abandons the query when
// the partial sum already exceeds the threshold for all 32 series (Alg. 3's
// chunked early abandoning).  Survivors are appended to the query's candidate
// buffer with warp-aggregated atomics.
constexpr int MAX_LEAF_TILES = 256;
template <int LW, bool NYQ, bool H16>
__global__ void __launch_bounds__(256) k_scan(QueryParams P, const int4* __restrict__ units,
                                              const int* __restrict__ n_units_ptr, const int* __restrict__ leaf_q,
                                              const float* __restrict__ qv, const float* __restrict__ thr,
                                              const uint8_t* __restrict__ tenv, const uint8_t* __restrict__ words,
                                              const float2* __restrict__ edge, const float2* __restrict__ ch,
                                              const __half2* __restrict__ ch16, float f16, float inv_f16,
                                              const int* __restrict__ qslot, uint32_t* __restrict__ cand_p,
                                              float* __restrict__ cand_lb, int* __restrict__ cand_n,
                                              int64_t pool_cap, int* __restrict__ pool_n, int* __restrict__ pool_q,
                                              uint32_t* __restrict__ pool_p, float* __restrict__ pool_lb,
                                              int* __restrict__ qpool_cnt, unsigned long long* __restrict__ counters) {
  extern __shared__ float2 tabs[];
  float2* sch = tabs;                                                   // LW x 256 (tile checks, FP32 bounds)
  __half2* sch16 = reinterpret_cast<__half2*>(tabs + LW * MAX_ALPHA);   // LW x 256 (FP16 bounds)
  // per-tile lists of the unit's queries that passed the tile envelope
  // (leaf_tiles x MAX_GROUP bytes after the tables)
  uint8_t* sql = reinterpret_cast<uint8_t*>(tabs + LW * MAX_ALPHA) + (H16 ? LW * MAX_ALPHA * sizeof(__half2) : 0);
  __shared__ uint16_t s_off[MAX_LEAF_TILES + 1];
  __shared__ __align__(16) float sq[MAX_GROUP][LW];
  __shared__ __align__(16) __half2 sq16[MAX_GROUP][LW / 2];
  __shared__ float sT[MAX_GROUP];
  __shared__ float sTs[MAX_GROUP];  // thresholds in the unit's scaled units (FP32 path)
  __shared__ float s_a, s_inva2;
  __shared__ int sslot[MAX_GROUP];
  __shared__ unsigned long long smask[MAX_LEAF_TILES];
  const int tid = threadIdx.x, lane = tid & 31;
  for (int e = tid; e < LW * MAX_ALPHA; e += blockDim.x) {
    sch[e] = ch[e];
    if (H16) sch16[e] = ch16[e];
  }
  unsigned long long n_tile_pairs = 0, n_cand = 0, n_loads = 0, n_checks = 0;
  const int n_units = *n_units_ptr;
  for (int u = blockIdx.x; u < n_units; u += gridDim.x) {
    __syncthreads();
    const int4 un = units[u];
    const int64_t b = un.x;
    const int cnt = un.z;
    const int64_t t0 = b * P.leaf_tiles;
    const int nt = (int)((P.T - t0) < P.leaf_tiles ? (P.T - t0) : P.leaf_tiles);
    for (int e = tid; e < cnt * LW; e += blockDim.x) {
      int g = e / LW, j = e - g * LW;
      int qq = leaf_q[un.y + g];
      sq[g][j] = qv[(int64_t)qq * P.NB + j];
      if (H16 && (j & 1) == 0)
        sq16[g][j >> 1] = __floats2half2_rn(qv[(int64_t)qq * P.NB + j], qv[(int64_t)qq * P.NB + j + 1]);
      if (j == 0) {
        sslot[g] = qslot ? qslot[qq] : qq;
        sT[g] = thr[qq];
      }
    }
    for (int t = tid; t < nt; t += blockDim.x) smask[t] = 0ull;
    __syncthreads();
    if (!H16) {
      // Scale a = 1/M with M^2 >= 2.5 max T: each value's term is computed as
      // u = sat(|q - c| a - h a), clipping m at M; a clipped term alone exceeds
      // every threshold of the unit, so clipping never keeps a series that the
      // exact bound prunes (nor prunes one it keeps).
      if (tid == 0) {
        float tmax = 0.f;
        for (int g = 0; g < cnt; ++g) tmax = fmaxf(tmax, sT[g]);
        float a = __frcp_rd(__fsqrt_ru(__fmul_ru(2.5f, tmax)));
        a = fminf(fmaxf(a, 0x1p-20f), 0x1p20f);
        s_a = a;
        s_inva2 = __frcp_rd(__fmul_ru(a, a));
      }
      __syncthreads();
      for (int g = tid; g < cnt; g += blockDim.x) sTs[g] = __fmul_ru(__fmul_ru(sT[g], s_a), s_a);
      __syncthreads();
    }
    // all envelope checks of the unit
    for (int e = tid; e < nt * cnt; e += blockDim.x) {
      const int t = e / cnt, g = e - t * cnt;
      float a = env_bound_ch<LW, NYQ>(tenv + (t0 + t) * 2 * LW, sq[g], sch);
      if (a <= sT[g]) atomicOr(&smask[t], 1ull << g);
    }
    n_checks += (tid == 0) ? (unsigned long long)nt : 0ull;
    __syncthreads();
    // compact each tile's mask into a list of query indices once per unit, so
    // the threads walk the list instead of each scanning the mask bits
    if (tid < 32) {  // exclusive scan of the per-tile counts by one warp
      int run = 0;
      for (int base = 0; base < nt; base += 32) {
        const int t = base + lane;
        const int c = t < nt ? __popcll(smask[t]) : 0;
        int x = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(0xFFFFFFFFu, x, o);
          if (lane >= o) x += y;
        }
        if (t < nt) s_off[t] = (uint16_t)(run + x - c);
        run += __shfl_sync(0xFFFFFFFFu, x, 31);
      }
      if (lane == 0) s_off[nt] = (uint16_t)run;
    }
    __syncthreads();
    for (int t = tid; t < nt; t += blockDim.x) {
      unsigned long long m = smask[t];
      int o = s_off[t];
      while (m) {
        sql[o++] = (uint8_t)(__ffsll((long long)m) - 1);
        m &= m - 1;
      }
    }
    __syncthreads();
    for (int t = 0; t < nt; ++t) {
      const int o0 = s_off[t], o1 = s_off[t + 1];
      if (o0 == o1) continue;
      if (tid == 0) {
        n_tile_pairs += (unsigned long long)(o1 - o0);
        n_loads += 1;
      }
      const int64_t p = (t0 + t) * TILE + tid;
      const bool valid = p < P.N;
      [[maybe_unused]] const float acc0 = valid ? 0.f : __int_as_float(0x7f800000);  // +inf: never live
      float c[H16 ? 1 : LW], h[H16 ? 1 : LW];
      __half2 c2[H16 ? LW / 2 : 1], nh2[H16 ? LW / 2 : 1];
      if constexpr (H16) {
        // gather (c, -h) of each value, then pair values 2i, 2i+1 per register
        uint32_t w32[LW / 4];
        if (valid) {
          const uint4* wp = reinterpret_cast<const uint4*>(words + p * LW);
#pragma unroll
          for (int i = 0; i < LW / 16; ++i) {
            uint4 v = __ldg(wp + i);
            w32[4 * i] = v.x;
            w32[4 * i + 1] = v.y;
            w32[4 * i + 2] = v.z;
            w32[4 * i + 3] = v.w;
          }
        } else {
#pragma unroll
          for (int i = 0; i < LW / 4; ++i) w32[i] = 0u;
        }
#pragma unroll
        for (int i = 0; i < LW / 2; ++i) {
          const int j0 = 2 * i, j1 = 2 * i + 1;
          const __half2 v0 = sch16[j0 * MAX_ALPHA + ((w32[j0 >> 2] >> (8 * (j0 & 3))) & 0xFFu)];
          const __half2 v1 = sch16[j1 * MAX_ALPHA + ((w32[j1 >> 2] >> (8 * (j1 & 3))) & 0xFFu)];
          c2[i] = __lows2half2(v0, v1);
          nh2[i] = __highs2half2(v0, v1);
        }
      } else {
        load_word_bounds<LW>(words, p, valid, sch, c, h);
        const float a = s_a;
#pragma unroll
        for (int j = 0; j < LW; ++j) h[j] = __fmul_ru(h[j], a);  // h a, rounded up
      }
      for (int oi = o0; oi < o1; ++oi) {
        const int g = sql[oi];
        const float T = H16 ? sT[g] * f16 : sTs[g];
        bool live = valid;
        float acc;
        if constexpr (H16) {
          // m = relu(|q - c| - h) by one fused multiply-add with relu, then
          // m^2 accumulated in two half lanes (even / odd values)
          const __half2* qg = sq16[g];
          const __half2 one2 = __floats2half2_rn(1.f, 1.f);
          __half2 a2 = __floats2half2_rn(0.f, 0.f);
#pragma unroll
          for (int stage = 0; stage < 8; ++stage) {
            const int i0 = stage == 0 ? 0 : (2 << (stage - 1));
            const int i1 = 2 << stage;
            if (i0 >= LW / 2) break;
            if (!__any_sync(0xFFFFFFFFu, live)) break;
#pragma unroll
            for (int i = i0; i < i1 && i < LW / 2; ++i) {
              const __half2 d = __habs2(__hsub2(qg[i], c2[i]));
              const __half2 mv = __hfma2_relu(d, one2, nh2[i]);
              const __half2 mm = (NYQ && i == 0) ? __hmul2(mv, __floats2half2_rn(0.5f, 1.f)) : mv;
              a2 = __hfma2(mm, mv, a2);
            }
            const float2 af = __half22float2(a2);
            live = live && (af.x + af.y) <= T;
          }
          const float2 af = __half22float2(a2);
          acc = __fmul_rd(af.x + af.y, inv_f16);  // deflated: a lower bound in exact units
        } else {
          const float4* qg4 = reinterpret_cast<const float4*>(sq[g]);
          const float a = s_a;
          // u = sat(|q - c| a - h a) (one FADD, one FFMA.SAT), one running sum
          // s.  Every term is >= 0, so s never decreases and "s <= T" is the
          // lane's whole liveness (lanes past N start at +inf): the warp votes
          // on it after every 4 of the first 16 values (about 10 of 16 are
          // evaluated on average at 100M x 256), then after 24 and 32, and a
          // warp with no live lane goes straight to the next query.
          float s = acc0;
          bool warp_dead = false;
#pragma unroll
          for (int stage = 0; stage < 6; ++stage) {
            const int j0 = stage < 4 ? 4 * stage : 16 + 8 * (stage - 4);
            const int j1 = stage < 4 ? j0 + 4 : j0 + 8;
            if (j0 >= LW) break;
            if (stage > 0 && !__any_sync(0xFFFFFFFFu, s <= T)) {
              warp_dead = true;
              break;
            }
#pragma unroll
            for (int j = j0; j < j1 && j < LW; j += 4) {
              const float4 q4 = qg4[j >> 2];
              const float u0 = __saturatef(fmaf(fabsf(q4.x - c[j]), a, -h[j]));
              const float u1 = __saturatef(fmaf(fabsf(q4.y - c[j + 1]), a, -h[j + 1]));
              const float u2 = __saturatef(fmaf(fabsf(q4.z - c[j + 2]), a, -h[j + 2]));
              const float u3 = __saturatef(fmaf(fabsf(q4.w - c[j + 3]), a, -h[j + 3]));
              s = fmaf((NYQ && j == 0) ? 0.5f * u0 : u0, u0, s);
              s = fmaf(u1, u1, s);
              s = fmaf(u2, u2, s);
              s = fmaf(u3, u3, s);
            }
          }
          if (warp_dead) continue;  // warp-uniform: no lane left for this query
          live = s <= T;
          acc = __fmul_rd(s, s_inva2);  // back to half units, rounded down
        }
        const unsigned hit = __ballot_sync(0xFFFFFFFFu, live);
        if (hit) {
          const int qs = sslot[g];
          const int npop = __popc(hit);
          int base = 0, pbase = 0;
          if (lane == 0) base = atomicAdd(cand_n + qs, npop);
          base = __shfl_sync(0xFFFFFFFFu, base, 0);
          // slots beyond the query's region go to the shared pool
          const int over0 = base > P.cap ? base : P.cap;
          const int nover = base + npop - over0;
          if (lane == 0 && nover > 0) {
            // the counter grows only while the pool has room, so however
            // many candidates are refused it stays below pool_cap + 32 x
            // (warps in flight) and cannot wrap
            pbase = *reinterpret_cast<volatile int*>(pool_n) < pool_cap ? atomicAdd(pool_n, nover) : (int)pool_cap;
            const int64_t room = pool_cap - pbase;
            const int written = room <= 0 ? 0 : (room < nover ? (int)room : nover);
            if (written > 0) atomicAdd(qpool_cnt + qs, written);
          }
          pbase = __shfl_sync(0xFFFFFFFFu, pbase, 0);
          if (live) {
            const int slot = base + __popc(hit & ((1u << lane) - 1u));
            if (slot < P.cap) {
              cand_p[(int64_t)qs * P.cap + slot] = (uint32_t)p;
              cand_lb[(int64_t)qs * P.cap + slot] = acc;
            } else {
              const int64_t pi = (int64_t)pbase + (slot - over0);
              if (pi < pool_cap) {
                pool_q[pi] = qs;
                pool_p[pi] = (uint32_t)p;
                pool_lb[pi] = acc;
              }
            }
          }
          if (lane == 0) n_cand += __popc(hit);
        }
      }
    }
  }
  if (n_tile_pairs) atomicAdd(counters + 1, n_tile_pairs);
  if (n_cand) atomicAdd(counters + 2, n_cand);
  if (n_loads) atomicAdd(counters + 4, n_loads);
  if (n_checks) atomicAdd(counters + 5, n_checks);
}

// ------------------------------------------------------------------------
// Candidate store: each query slot has a region of P.cap entries; the excess
// of a pass goes to a shared pool of (slot, position, bound) triples.  After
// the scan one CTA plans the refinement: per slot, r = min(count, cap) region
// entries plus pool_cnt pool entries, cut into chunks of RSORT; exclusive
// scans give each slot its pool segment and its first chunk, and the chunk
// total goes to the device (the refinement is persistent and reads it), and
// the word after it, the refinement's chunk cursor, is zeroed.
constexpr int RSORT = 4096;
constexpr uint16_t VDROP = 0xFFFFu;  // ordered slot of a candidate the value codes dropped (RSORT <= 0xFFFF)
__global__ void __launch_bounds__(1024) k_chunk_plan(int64_t slots, int cap, const int* __restrict__ cand_n,
                                                     const int* __restrict__ qpool_cnt, int* __restrict__ qpool_off,
                                                     int* __restrict__ qcursor, int* __restrict__ choff,
                                                     int* __restrict__ n_chunks) {
  __shared__ long long s1[1024], s2[1024];
  const int tid = threadIdx.x;
  const int64_t per = (slots + 1023) / 1024;
  const int64_t a0 = tid * per, a1 = a0 + per < slots ? a0 + per : slots;
  long long pc = 0, nc = 0;
  for (int64_t q = a0; q < a1; ++q) {
    const int r = cand_n[q] < cap ? cand_n[q] : cap;
    pc += qpool_cnt[q];
    nc += (r + qpool_cnt[q] + RSORT - 1) / RSORT;
  }
  s1[tid] = pc;
  s2[tid] = nc;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    const long long x1 = tid >= o ? s1[tid - o] : 0, x2 = tid >= o ? s2[tid - o] : 0;
    __syncthreads();
    s1[tid] += x1;
    s2[tid] += x2;
    __syncthreads();
  }
  long long rp = s1[tid] - pc, rc = s2[tid] - nc;
  for (int64_t q = a0; q < a1; ++q) {
    const int r = cand_n[q] < cap ? cand_n[q] : cap;
    qpool_off[q] = (int)rp;
    choff[q] = (int)rc;
    qcursor[q] = 0;
    rp += qpool_cnt[q];
    rc += (r + qpool_cnt[q] + RSORT - 1) / RSORT;
  }
  if (tid == 1023) {
    n_chunks[0] = (int)s2[1023];
    n_chunks[1] = 0;
  }
}

// Counting-sort scatter of the pool into per-slot segments (grid-stride).
__global__ void k_pool_scatter(const int* __restrict__ pool_n, int64_t pool_cap, const int* __restrict__ pool_q,
                               const uint32_t* __restrict__ pool_p, const float* __restrict__ pool_lb,
                               const int* __restrict__ qpool_off, int* __restrict__ qcursor,
                               uint32_t* __restrict__ sp, float* __restrict__ slb) {
  const int64_t n = *pool_n < pool_cap ? *pool_n : pool_cap;
  const int lane = threadIdx.x & 31;
  // the scan wrote each query's entries in runs: lanes with the same query
  // share one atomic (warp-uniform loop bounds keep every lane in the vote)
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x; i0 < n; i0 += stride) {
    const int64_t i = i0 + threadIdx.x;
    const bool ok = i < n;
    const int q = ok ? pool_q[i] : -1;
    const unsigned grp = __match_any_sync(0xFFFFFFFFu, q);
    const int leader = __ffs(grp) - 1;
    int base = 0;
    if (ok && lane == leader) base = atomicAdd(qcursor + q, __popc(grp));
    base = __shfl_sync(0xFFFFFFFFu, base, leader);
    if (ok) {
      const int pos = base + __popc(grp & ((1u << lane) - 1u));
      sp[qpool_off[q] + pos] = pool_p[i];
      slb[qpool_off[q] + pos] = pool_lb[i];
    }
  }
}

// Chunk list: chunk_q[choff[s] + c] = s for every chunk c of slot s.
__global__ void k_chunk_fill(int64_t slots, int cap, const int* __restrict__ cand_n, const int* __restrict__ qpool_cnt,
                             const int* __restrict__ choff, int* __restrict__ chunk_q) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= slots) return;
  const int r = cand_n[q] < cap ? cand_n[q] : cap;
  const int nch = (r + qpool_cnt[q] + RSORT - 1) / RSORT;
  for (int c = 0; c < nch; ++c) chunk_q[choff[q] + c] = (int)q;
}

// ------------------------------------------------------------------------
// Refinement (GEMINI's exact distance for the survivors of the bound, Sec.
// II-A, visited in ascending bound order as in Sec. IV "Exact Similarity
// Search").  Every chunk of RSORT candidates of a query gets its own CTA:
// the chunk is sorted by bound; rounds of 64 candidates (8 warps x 8 groups of
// 4 lanes) get their FP32 distance; entries inside the chunk's tie window go to
// a chunk-local kept list.  The query's threshold lives in global memory: a
// chunk whose list holds k entries publishes k-th * f_prune / 2 with atomicMin
// (a real k-th distance of k distinct series, hence a valid bound), and each
// round reads the current value, so all chunks of a query tighten together.
// The first candidate whose bound exceeds the threshold ends the chunk.
constexpr int RROUND = 64;  // candidates refined per round: 8 warps x 8 groups of 4 lanes
template <int FILTER>  // 0: FP32 only; 1: int8 rows first; 2: value codes, then int8 rows
__global__ void __launch_bounds__(256, FILTER ? 4 : 5) k_refine(QueryParams P, const int* __restrict__ n_chunks_ptr,
                                                const int* __restrict__ chunk_q, const int* __restrict__ choff,
                                                const int* __restrict__ qof, const float* __restrict__ zq,
                                                const float* __restrict__ Z, const uint32_t* __restrict__ cand_p,
                                                const float* __restrict__ cand_lb, const int* __restrict__ cand_n,
                                                const int* __restrict__ qpool_cnt, const int* __restrict__ qpool_off,
                                                const uint32_t* __restrict__ sp, const float* __restrict__ slb,
                                                float* __restrict__ thr, float* __restrict__ chunk_d,
                                                uint32_t* __restrict__ chunk_p, int* __restrict__ chunk_n,
                                                const int8_t* __restrict__ Z8, const float* __restrict__ s8,
                                                const float* __restrict__ e8, float one_minus_g,
                                                const float* __restrict__ qv, const int8_t* __restrict__ VC,
                                                const float2* __restrict__ vsr, const float* __restrict__ vw,
                                                float one_minus_gv, int* __restrict__ next_chunk,
                                                unsigned long long* __restrict__ counters, int* __restrict__ status) {
  extern __shared__ float4 rsm[];
  float* szq = reinterpret_cast<float*>(rsm);  // n
  __shared__ unsigned long long skey[RSORT];
  __shared__ float sld[KCAP];
  __shared__ uint32_t slp[KCAP];
  __shared__ float acc_d[RROUND];
  __shared__ uint32_t acc_p[RROUND];
  __shared__ int s_nacc, s_nl, s_lost, s_nsurv, s_stop0;  // s_stop0: thread 0 only
  __shared__ int s_ch;
  __shared__ float s_lim, s_T0;
  __shared__ uint32_t surv[FILTER ? 256 : 1];
  __shared__ uint32_t s1[FILTER == 2 ? 256 : 1];      // survivors of the value-code bound
  __shared__ float sqv[FILTER == 2 ? NB_MAX : 1];     // the query's selected values
  __shared__ float sw[FILTER == 2 ? NB_MAX : 1];      // their Eq. (1) weights
  __shared__ int s_n1;
  constexpr int NBK = 32;  // bound buckets of a chunk
  __shared__ int bcnt[NBK + 1], bcur[NBK + 1];
  __shared__ uint16_t ord[RSORT];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  unsigned long long refined = 0, filtered = 0, vfiltered = 0;
  const int n_chunks = *n_chunks_ptr;
  // chunks differ widely in work (early stop, pool share), so each CTA takes
  // its next chunk from a cursor instead of a fixed stride
  for (;;) {
  __syncthreads();
  if (tid == 0) s_ch = atomicAdd(next_chunk, 1);
  __syncthreads();
  const int ch = s_ch;
  if (ch >= n_chunks) break;
  const int slot_q = chunk_q[ch];
  const int c = ch - choff[slot_q];
  const int64_t q = qof ? qof[slot_q] : slot_q;
  const int K = kq(P, q);
  const int r = cand_n[slot_q] < P.cap ? cand_n[slot_q] : P.cap;
  const int total = r + qpool_cnt[slot_q];
  const int c0 = c * RSORT;
  const int cc = total - c0 < RSORT ? total - c0 : RSORT;
  for (int t = tid; t < P.n; t += blockDim.x) szq[t] = zq[q * P.n + t];
  if constexpr (FILTER == 2)
    for (int t = tid; t < P.NB; t += blockDim.x) {
      sqv[t] = qv[q * P.NB + t];
      sw[t] = vw[t];
    }
  volatile float* vthr = thr;
  if (tid == 0) {
    s_nl = 0;
    s_lost = 0;
    s_lim = INFINITY;
    s_nacc = 0;
    s_T0 = vthr[q];
  }
  for (int i = tid; i <= NBK; i += blockDim.x) bcnt[i] = 0;
  __syncthreads();
  // coarse ascending-bound order by a counting sort into NBK buckets of width
  // T0 / NBK (T0 = the threshold now); bounds above T0 can never pass and are
  // dropped, so no full sort is needed for the early stop below
  const float T0 = s_T0;
  const float bscale = T0 > 0.f ? (float)NBK / T0 : 0.f;
  for (int i = tid; i < cc; i += blockDim.x) {
    const int e = c0 + i;
    unsigned long long kk;
    if (e < r) kk = pack_key(cand_lb[(int64_t)slot_q * P.cap + e], cand_p[(int64_t)slot_q * P.cap + e]);
    else kk = pack_key(slb[qpool_off[slot_q] + (e - r)], sp[qpool_off[slot_q] + (e - r)]);
    if ((uint32_t)kk >= P.N) {  // consistency check: record it; the NaN key below drops the entry
      atomicExch(status, SOFA_ERR_INTERNAL);
      kk = ~0ull;
    }
    skey[i] = kk;
    const float lb = __uint_as_float((uint32_t)(kk >> 32));
    const int b = lb <= T0 ? min(NBK - 1, (int)(lb * bscale)) : NBK;
    atomicAdd(&bcnt[b], 1);
  }
  __syncthreads();
  if (tid == 0) {
    int acc = 0;
    for (int b = 0; b <= NBK; ++b) {
      const int c_ = bcnt[b];
      bcnt[b] = acc;  // bucket start
      bcur[b] = acc;
      acc += c_;
    }
  }
  __syncthreads();
  for (int i = tid; i < cc; i += blockDim.x) {
    const float lb = __uint_as_float((uint32_t)(skey[i] >> 32));
    const int b = lb <= T0 ? min(NBK - 1, (int)(lb * bscale)) : NBK;
    if (b < NBK) ord[atomicAdd(&bcur[b], 1)] = (uint16_t)i;
  }
  __syncthreads();
  const int nlive = bcnt[NBK];  // candidates with bound <= T0, bucket-ordered in ord
  // a lower bound of every bound at ordered positions >= j: the edge of the
  // bucket below the one holding j (the bucket index was rounded, so a bound
  // may sit a hair under its own bucket's edge, never under the previous one's)
  auto edge_of = [&](int j) {
    int b = 0;
    while (b + 1 < NBK && bcnt[b + 1] <= j) ++b;
    return b > 0 ? (float)(b - 1) / bscale : 0.f;
  };
  // thread 0: merge the accepted distances of a round into the chunk's kept
  // list, tighten its window and publish the query's threshold
  auto merge_round = [&]() {
    int nl = s_nl;
    float lim = s_lim;
    const int na = s_nacc;
    for (int w = 0; w < na; ++w) {
      const float d = acc_d[w];
      const uint32_t pp = acc_p[w];
      if (!(d <= lim)) continue;
      int j = nl - 1;  // insertion by (d2, pos)
      while (j >= 0 && (sld[j] > d || (sld[j] == d && slp[j] > pp))) {
        if (j + 1 < KCAP) {
          sld[j + 1] = sld[j];
          slp[j + 1] = slp[j];
        }
        --j;
      }
      if (j + 1 < KCAP) {
        sld[j + 1] = d;
        slp[j + 1] = pp;
      }
      if (nl < KCAP) ++nl;
      else s_lost = 1;
      if (nl >= K) {
        lim = __fmul_ru(sld[K - 1], P.f_keep);
        while (nl > K && sld[nl - 1] > lim) --nl;  // drop entries that left the window
      }
    }
    s_nacc = 0;
    s_nl = nl;
    s_lim = lim;
    if (nl >= K) {
      const float t = __fmul_ru(__fmul_ru(sld[K - 1], P.f_prune), 0.5f);
      atomicMin(reinterpret_cast<int*>(thr) + q, __float_as_int(t));  // t >= 0: int order = float order
    }
  };
  if constexpr (FILTER == 2) {
    // value-code pass over the whole chunk before the rounds (many candidates
    // per thread, so their gathers overlap instead of one per round and
    // barrier): Eq. (1) on the selected values from their int8 codes,
    // ||q~ - s c||_w - r <= ||q - v||_w <= d(q, x), against the threshold at
    // this point (any threshold at or above the final one is valid); a
    // dropped candidate's ordered slot is marked VDROP
    const float Tv = vthr[q];
#pragma unroll 2
    for (int j = tid; j < nlive; j += blockDim.x) {
      const int i = ord[j];
      const unsigned long long kk = skey[i];
      if (__uint_as_float((uint32_t)(kk >> 32)) > Tv) continue;  // left to the rounds' own check
      const uint32_t p = (uint32_t)kk;
      const float2 sr = __ldg(vsr + p);
      const uint4* cp = reinterpret_cast<const uint4*>(VC + (int64_t)p * P.NB);
      float a0 = 0.f, a1 = 0.f;
      for (int u = 0; u < P.NB / 16; ++u) {
        const uint4 w4 = __ldg(cp + u);
        const uint32_t ws[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
          for (int e = 0; e < 4; e += 2) {
            const int t0 = 16 * u + 4 * b + e;
            const float c0 = (float)((int)(ws[b] << (24 - 8 * e)) >> 24);
            const float c1 = (float)((int)(ws[b] << (16 - 8 * e)) >> 24);
            const float d0 = fmaf(-sr.x, c0, sqv[t0]), d1 = fmaf(-sr.x, c1, sqv[t0 + 1]);
            a0 = fmaf(d0 * sw[t0], d0, a0);          // weight 0, 1 or 2: exact products
            a1 = fmaf(d1 * sw[t0 + 1], d1, a1);
          }
      }
      const float lbv = __fsub_rd(__fsqrt_rd(__fmul_rd(a0 + a1, one_minus_gv)), sr.y);
      if (lbv > 0.f && __fmul_rd(lbv, lbv) > 2.0f * Tv) {
        ++vfiltered;
        ord[j] = VDROP;
      }
    }
    __syncthreads();
  }
  if constexpr (FILTER != 0) {
    // rounds of 256 candidates, one per thread: the int8 bound
    // d(q, x) >= d(q, s v) - e (2 T is the squared distance bound, T in half
    // units); only survivors get the FP32 distance, by groups of 4 lanes
    for (int base = 0; base < nlive; base += 256) {
      const float T = vthr[q];
      // thread 0's verdict (every later bucket starts above T) is kept in a
      // word only thread 0 touches and joined by __syncthreads_or at the end
      // of the round: no shared flag that the next round could overwrite
      // while a warp still reads it
      if (tid == 0) {
        s_nsurv = 0;
        s_n1 = 0;
        s_stop0 = edge_of(base) > T;
      }
      __syncthreads();
      // candidates of this round entering the int8 stage: the value-code
      // survivors (compacted into s1), or the round's ordered candidates
      int n1 = nlive - base < 256 ? nlive - base : 256;
      if constexpr (FILTER == 2) {
        // the round's candidates that the value-code pass kept
        const int j = base + tid;
        const int i = j < nlive ? ord[j] : VDROP;
        if (i != VDROP && __uint_as_float((uint32_t)(skey[i] >> 32)) <= T)
          s1[atomicAdd(&s_n1, 1)] = (uint32_t)skey[i];
        __syncthreads();
        n1 = s_n1;
      }
      if ((P.n & 15) == 0) {
        // 16 lanes per candidate row: lane `sub` reads 16-byte pieces sub,
        // sub + 16, ... of the int8 row and the matching float4s of the query
        const int half = lane >> 4, sub = lane & 15;
        const int n16 = P.n >> 4;
        const float4* zq4 = reinterpret_cast<const float4*>(szq);
        // four candidates per half-warp at a time: all their loads are issued
        // before any reduction, and the query float4s are shared by the four
        for (int it = 0; it < 16; it += 4) {
          if (FILTER == 2 && it * 16 >= n1) break;  // n1 is the same for the whole block
          bool act[4];
          uint32_t pp[4];
          float sc[4], a0[4], a1[4];
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            if constexpr (FILTER == 2) {
              // compacted survivors, spread over all half-warps first
              const int jj = (it + k) * 16 + warp * 2 + half;
              act[k] = jj < n1;
              pp[k] = act[k] ? s1[jj] : 0u;
            } else {
              const int j = base + warp * 32 + (it + k) * 2 + half;
              const int i = j < nlive ? ord[j] : 0;
              act[k] = j < nlive && __uint_as_float((uint32_t)(skey[i] >> 32)) <= T;
              pp[k] = act[k] ? (uint32_t)skey[i] : 0u;
            }
            sc[k] = act[k] ? __ldg(s8 + pp[k]) : 0.f;
            a0[k] = 0.f;
            a1[k] = 0.f;
          }
          for (int u = sub; u < n16; u += 16) {
            uint4 w[4];
#pragma unroll
            for (int k = 0; k < 4; ++k)
              w[k] = act[k] ? __ldg(reinterpret_cast<const uint4*>(Z8 + (int64_t)pp[k] * P.n) + u)
                            : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
            for (int b = 0; b < 4; ++b) {
              const float4 qv4 = zq4[4 * u + b];
#pragma unroll
              for (int k = 0; k < 4; ++k) {
                const uint32_t ws = b == 0 ? w[k].x : b == 1 ? w[k].y : b == 2 ? w[k].z : w[k].w;
                const float v0 = (float)((int)(ws << 24) >> 24), v1 = (float)((int)(ws << 16) >> 24);
                const float v2 = (float)((int)(ws << 8) >> 24), v3 = (float)((int)ws >> 24);
                const float d0 = fmaf(-sc[k], v0, qv4.x), d1 = fmaf(-sc[k], v1, qv4.y);
                const float d2 = fmaf(-sc[k], v2, qv4.z), d3 = fmaf(-sc[k], v3, qv4.w);
                a0[k] = fmaf(d0, d0, a0[k]);
                a1[k] = fmaf(d1, d1, a1[k]);
                a0[k] = fmaf(d2, d2, a0[k]);
                a1[k] = fmaf(d3, d3, a1[k]);
              }
            }
          }
          float e2[4];
#pragma unroll
          for (int k = 0; k < 4; ++k) e2[k] = a0[k] + a1[k];
#pragma unroll
          for (int o = 8; o > 0; o >>= 1)
#pragma unroll
            for (int k = 0; k < 4; ++k) e2[k] += __shfl_xor_sync(0xFFFFFFFFu, e2[k], o);
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            if (act[k] && sub == 0) {
              const float lbd = __fsub_rd(__fsqrt_rd(__fmul_rd(e2[k], one_minus_g)), __ldg(e8 + pp[k]));
              if (lbd > 0.f && __fmul_rd(lbd, lbd) > 2.0f * T) ++filtered;
              else surv[atomicAdd(&s_nsurv, 1)] = pp[k];
            }
          }
        }
      } else {
        bool act;
        uint32_t p = 0u;
        if constexpr (FILTER == 2) {
          act = tid < n1;
          if (act) p = s1[tid];
        } else {
          const int j = base + tid;
          const int i = j < nlive ? ord[j] : 0;
          act = j < nlive && __uint_as_float((uint32_t)(skey[i] >> 32)) <= T;
          if (act) p = (uint32_t)skey[i];
        }
        if (act) {
          const float e2 = thread_sqdist8(szq, Z8, s8[p], p, P.n);
          const float lbd = __fsub_rd(__fsqrt_rd(__fmul_rd(e2, one_minus_g)), e8[p]);
          if (lbd > 0.f && __fmul_rd(lbd, lbd) > 2.0f * T) ++filtered;
          else surv[atomicAdd(&s_nsurv, 1)] = p;
        }
      }
      __syncthreads();
      const int ns = s_nsurv;
      for (int sb = 0; sb < ns; sb += RROUND) {
        const int j = sb + warp * 8 + (lane >> 2);
        const bool active = j < ns;
        const uint32_t p = active ? surv[j] : 0u;
        const float d2 = group4_sqdist(szq, Z, p, P.n, lane & 3, active);
        if ((lane & 3) == 0 && active) {
          ++refined;
          if (d2 <= s_lim) {
            const int a2 = atomicAdd(&s_nacc, 1);
            acc_d[a2] = d2;
            acc_p[a2] = p;
          }
        }
        __syncthreads();
        if (tid == 0) merge_round();
        __syncthreads();
      }
      if (__syncthreads_or(tid == 0 && s_stop0)) break;
    }
  } else {
    for (int base = 0; base < nlive; base += RROUND) {
      const int slot = warp * 8 + (lane >> 2);
      const int j = base + slot;
      const float T = vthr[q];
      bool active = false;
      uint32_t p = 0xFFFFFFFFu;
      if (j < nlive) {
        const int i = ord[j];
        const float lb = __uint_as_float((uint32_t)(skey[i] >> 32));
        active = lb <= T;
        if (active) p = (uint32_t)skey[i];
      }
      const bool stop_after = tid == 0 && edge_of(base) > T;  // every later bucket starts above T
      const float d2 = group4_sqdist(szq, Z, p, P.n, lane & 3, active);
      if ((lane & 3) == 0 && active) {
        ++refined;
        if (d2 <= s_lim) {  // a candidate for the local kept list
          const int a2 = atomicAdd(&s_nacc, 1);
          acc_d[a2] = d2;
          acc_p[a2] = p;
        }
      }
      __syncthreads();
      if (tid == 0) merge_round();
      if (__syncthreads_or(stop_after)) break;  // barrier and block-wide verdict in one
    }
  }
  const int nl = s_nl;
  float* od = chunk_d + (int64_t)ch * KCAP;
  uint32_t* op = chunk_p + (int64_t)ch * KCAP;
  for (int i = tid; i < nl; i += blockDim.x) {
    od[i] = sld[i];
    op[i] = slp[i];
  }
  if (tid == 0) {
    chunk_n[ch] = nl;
    if (s_lost) atomicExch(status, SOFA_ERR_TIE_OVERFLOW);
  }
  }
  if ((lane & 3) == 0 && refined) atomicAdd(counters + 3, refined);
  if (FILTER && filtered) atomicAdd(counters + 12, filtered);
  if (FILTER == 2 && vfiltered) atomicAdd(counters + 13, vfiltered);
}

// Merge of a query's kept list with the lists of its refined chunks: drop
// duplicates (an overflow pass may meet a series again) and entries outside
// the window of the current threshold, sort by (d2, pos), emit the new kept
// list and its threshold, and flag the query when its buffer overflowed.
constexpr int MSORT = 4096;
__global__ void __launch_bounds__(256) k_merge(QueryParams P, const int* __restrict__ qsel,
                                               const int* __restrict__ qslot, const int* __restrict__ cand_n,
                                               const int* __restrict__ qpool_cnt, const int* __restrict__ choff,
                                               const float* __restrict__ chunk_d, const uint32_t* __restrict__ chunk_p,
                                               const int* __restrict__ chunk_n, float* __restrict__ list_d,
                                               uint32_t* __restrict__ list_p, int* __restrict__ list_n,
                                               float* __restrict__ thr, int* __restrict__ qflag_out,
                                               int* __restrict__ n_overflow, int* __restrict__ status) {
  __shared__ unsigned long long skey[MSORT];
  __shared__ int s_cnt;
  const int64_t q = blockIdx.x;
  if (qsel && !qsel[q]) return;
  const int tid = threadIdx.x;
  const int K = kq(P, q);
  const int64_t slot_q = qslot ? qslot[q] : q;
  const int all = cand_n[slot_q];
  if (all == 0) return;
  const int rq = all < P.cap ? all : P.cap;
  const int stored = rq + qpool_cnt[slot_q];
  const int nch = (stored + RSORT - 1) / RSORT;
  const int c_first = choff[slot_q];
  // The window limit: D_k f_keep, D_k the k-th smallest distance among the
  // kept list and this pass's chunk lists.  Three upper bounds of D_k: the
  // threshold (a k-th distance of k real entries, times f_prune / 2), the kept
  // list's own k-th, and the k-th smallest over the chunk lists.  The last is
  // found exactly by bisection on the fp32 bit pattern (distances are >= 0,
  // so bit order is value order), counting with a binary search in each
  // chunk's sorted list; a series occurs at most once among one pass's chunks.
  // The entries under the smallest bound number at most about 2k, so none is
  // lost however many chunks the query has.
  __shared__ unsigned s_count;
  __shared__ int s_total;
  if (tid == 0) s_total = 0;
  __syncthreads();
  for (int c = c_first + tid; c < c_first + nch; c += blockDim.x) atomicAdd(&s_total, chunk_n[c]);
  __syncthreads();
  float lim_c = INFINITY;
  if (s_total >= K) {
    uint32_t lo = 0u, hi = 0x7F800000u;  // count(<= hi) >= k holds for hi = +inf
    while (lo < hi) {
      const uint32_t mid = lo + ((hi - lo) >> 1);
      const float x = __uint_as_float(mid);
      if (tid == 0) s_count = 0;
      __syncthreads();
      unsigned cnt = 0;
      for (int c = c_first + tid; c < c_first + nch; c += blockDim.x) {
        const float* cd = chunk_d + (int64_t)c * KCAP;
        int a = 0, b = chunk_n[c];  // first index with cd > x
        while (a < b) {
          const int m = (a + b) >> 1;
          if (cd[m] <= x) a = m + 1;
          else b = m;
        }
        cnt += (unsigned)a;
      }
      if (cnt) atomicAdd(&s_count, cnt);
      __syncthreads();
      if (s_count >= (unsigned)K) hi = mid;
      else lo = mid + 1;
      __syncthreads();
    }
    lim_c = __uint_as_float(hi);
  }
  const int nl = list_n[q];
  const float lim_k = nl >= K ? list_d[q * KCAP + K - 1] : INFINITY;
  const float lim = fminf(__fmul_ru(__fdiv_ru(__fmul_ru(thr[q], 2.0f), P.f_prune), P.f_keep),
                          __fmul_ru(fminf(lim_c, lim_k), P.f_keep));
  if (tid == 0) s_cnt = 0;
  __syncthreads();
  for (int i = tid; i < nl; i += blockDim.x) {
    const float d = list_d[q * KCAP + i];
    if (i < K || d <= lim) {
      const int a = atomicAdd(&s_cnt, 1);
      if (a < MSORT) skey[a] = pack_key(d, list_p[q * KCAP + i]);
    }
  }
  for (int c = c_first; c < c_first + nch; ++c) {
    const int m = chunk_n[c];
    const float* cd = chunk_d + (int64_t)c * KCAP;
    const uint32_t* cp = chunk_p + (int64_t)c * KCAP;
    for (int i = tid; i < m; i += blockDim.x) {
      if (cd[i] <= lim) {
        const int a = atomicAdd(&s_cnt, 1);
        if (a < MSORT) skey[a] = pack_key(cd[i], cp[i]);
      }
    }
  }
  __syncthreads();
  int len = s_cnt;
  if (len > MSORT) {
    len = MSORT;
    if (tid == 0) atomicExch(status, SOFA_ERR_TIE_OVERFLOW);
  }
  int pw = 1;
  while (pw < len) pw <<= 1;
  for (int i = len + tid; i < pw; i += blockDim.x) skey[i] = ~0ull;
  block_bitonic(skey, pw);
  // equal keys are the same (d2, pos): keep the first of each run
  __shared__ int s_u;
  if (tid == 0) {
    int u = 0;
    for (int i = 0; i < len; ++i)
      if (i == 0 || skey[i] != skey[u - 1]) skey[u++] = skey[i];
    s_u = u;
  }
  __syncthreads();
  if (!emit_list(skey, s_u, P, q, list_d, list_p, list_n, thr) && tid == 0) atomicExch(status, SOFA_ERR_TIE_OVERFLOW);
  if (tid == 0 && stored < all) {  // the pool ran out: scan this query again
    qflag_out[q] = 1;
    atomicAdd(n_overflow, 1);
  }
}

// ------------------------------------------------------------------------
// Final answer: FP64 re-score of every kept entry (the left-to-right FP64 sum
// of squared differences of the canonical series), order by (distance, id),
// then each run of distances within 1e-6 relative of the run's first is
// ordered by ascending id; the first k are written out.
__global__ void __launch_bounds__(128) k_final(QueryParams P, const float* __restrict__ zq,
                                               const float* __restrict__ Z, const uint32_t* __restrict__ perm,
                                               const uint32_t* __restrict__ list_p, const int* __restrict__ list_n,
                                               int64_t* __restrict__ idx, float* __restrict__ dist,
                                               unsigned long long* __restrict__ counters, int* __restrict__ status) {
  extern __shared__ float dsm[];
  float* szq = dsm;
  __shared__ double sd[128];
  __shared__ uint32_t sid[128];
  const int64_t q = blockIdx.x;
  const int tid = threadIdx.x;
  const int nl = list_n[q];
  for (int t = tid; t < P.n; t += blockDim.x) szq[t] = zq[q * P.n + t];
  __syncthreads();
  double d = INFINITY;
  uint32_t id = 0xFFFFFFFFu;
  const uint32_t p = tid < nl ? list_p[q * KCAP + tid] : 0u;
  if (tid < nl && p >= P.N) atomicExch(status, SOFA_ERR_INTERNAL);  // consistency check: skip the row
  if (tid < nl && p < P.N) {
    const float* row = Z + (int64_t)p * P.n;
    double acc = 0.0;
    for (int t = 0; t < P.n; ++t) {
      double df = __dsub_rn((double)szq[t], (double)row[t]);
      acc = __dadd_rn(acc, __dmul_rn(df, df));
    }
    d = __dsqrt_rn(acc);
    id = perm[p];
  }
  sd[tid] = d;
  sid[tid] = id;
  // sort the list's slots only (the next power of two; the rest hold +inf)
  int pw = 2;
  while (pw < nl) pw <<= 1;
  for (int size = 2; size <= pw; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      __syncthreads();
      if (tid < (pw >> 1)) {
        int lo = 2 * tid - (tid & (stride - 1));
        int hi = lo + stride;
        bool up = ((lo & size) == 0);
        bool gt = sd[lo] > sd[hi] || (sd[lo] == sd[hi] && sid[lo] > sid[hi]);
        if (gt == up) {
          double td = sd[lo];
          sd[lo] = sd[hi];
          sd[hi] = td;
          uint32_t ti = sid[lo];
          sid[lo] = sid[hi];
          sid[hi] = ti;
        }
      }
    }
  }
  __syncthreads();
  const int K = kq(P, q);
  if (tid == 0) {
    int i = 0;
    while (i < nl && i < K) {
      const double d0 = sd[i];
      const double lim = __dadd_rn(d0, __dmul_rn(1e-6, d0));
      int j = i;
      while (j + 1 < nl && sd[j + 1] <= lim) ++j;
      for (int a = i + 1; a <= j; ++a) {  // insertion sort of the run by id
        double vd = sd[a];
        uint32_t vi = sid[a];
        int b = a - 1;
        while (b >= i && sid[b] > vi) {
          sd[b + 1] = sd[b];
          sid[b + 1] = sid[b];
          --b;
        }
        sd[b + 1] = vd;
        sid[b + 1] = vi;
      }
      i = j + 1;
    }
  }
  __syncthreads();
  if (tid == 0 && nl >= K) atomicAdd(counters + 7, (unsigned long long)(1e6 * sd[K - 1]));
  const int64_t o = P.qo ? P.qo[q] : q * P.k;
  if (tid < K) {
    idx[o + tid] = tid < nl ? (int64_t)sid[tid] : -1;
    dist[o + tid] = tid < nl ? (float)sd[tid] : INFINITY;
  }
}

// A query's k-NN window for a merge across shards: its kept list re-scored
// with the oracle's FP64 left-to-right sum of squared differences, sorted by
// (distance, id), and cut to the rows whose distance d satisfies
// d <= D_k + 1e-6 D_k (D_k the k-th smallest): every row that can take one of
// the first k places of the tie rule in any union of shards (the global k-th
// distance is at most this shard's).  The kept list holds that window (it
// keeps every entry within the tie window of the k-th, with margin).
// Outputs: ids (original row ids), d2 (FP64 squared distances), -1 / +inf
// beyond the window; cnt the window size (at most cap: a larger window is
// cut and flagged with SOFA_ERR_TIE_OVERFLOW).
__global__ void __launch_bounds__(128) k_window(QueryParams P, const float* __restrict__ zq,
                                                const float* __restrict__ Z, const uint32_t* __restrict__ perm,
                                                const uint32_t* __restrict__ list_p, const int* __restrict__ list_n,
                                                int cap, int64_t* __restrict__ ids, double* __restrict__ d2,
                                                int* __restrict__ cnt, int* __restrict__ status) {
  extern __shared__ float dsm[];
  float* szq = dsm;
  __shared__ double sd[128], sq2[128];
  __shared__ uint32_t sid[128];
  __shared__ int s_cnt;
  const int64_t q = blockIdx.x;
  const int tid = threadIdx.x;
  const int nl = list_n[q];
  for (int t = tid; t < P.n; t += blockDim.x) szq[t] = zq[q * P.n + t];
  if (tid == 0) s_cnt = 0;
  __syncthreads();
  double d = INFINITY, a2 = INFINITY;
  uint32_t id = 0xFFFFFFFFu;
  const uint32_t p = tid < nl ? list_p[q * KCAP + tid] : 0u;
  if (tid < nl && p >= P.N) atomicExch(status, SOFA_ERR_INTERNAL);  // consistency check: skip the row
  if (tid < nl && p < P.N) {
    const float* row = Z + (int64_t)p * P.n;
    double acc = 0.0;
    for (int t = 0; t < P.n; ++t) {
      double df = __dsub_rn((double)szq[t], (double)row[t]);
      acc = __dadd_rn(acc, __dmul_rn(df, df));
    }
    a2 = acc;
    d = __dsqrt_rn(acc);
    id = perm[p];
  }
  sd[tid] = d;
  sq2[tid] = a2;
  sid[tid] = id;
  for (int size = 2; size <= 128; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      __syncthreads();
      if (tid < 64) {
        int lo = 2 * tid - (tid & (stride - 1));
        int hi = lo + stride;
        bool up = ((lo & size) == 0);
        bool gt = sd[lo] > sd[hi] || (sd[lo] == sd[hi] && sid[lo] > sid[hi]);
        if (gt == up) {
          double td = sd[lo];
          sd[lo] = sd[hi];
          sd[hi] = td;
          td = sq2[lo];
          sq2[lo] = sq2[hi];
          sq2[hi] = td;
          uint32_t ti = sid[lo];
          sid[lo] = sid[hi];
          sid[hi] = ti;
        }
      }
    }
  }
  __syncthreads();
  const int K = kq(P, q);
  const int kk = K < nl ? K : nl;
  const double dk = kk > 0 ? sd[kk - 1] : INFINITY;
  const double lim = __dadd_rn(dk, __dmul_rn(1e-6, dk));
  if (tid < nl && sid[tid] != 0xFFFFFFFFu && (tid < kk || sd[tid] <= lim)) atomicMax(&s_cnt, tid + 1);
  __syncthreads();
  const int w = s_cnt;
  if (tid == 0 && w > cap) atomicExch(status, SOFA_ERR_TIE_OVERFLOW);
  if (tid < cap) {
    const bool in = tid < w;
    ids[q * cap + tid] = in ? (int64_t)sid[tid] : -1;
    d2[q * cap + tid] = in ? sq2[tid] : INFINITY;
  }
  if (tid == 0) cnt[q] = w < cap ? w : cap;
}

// ========================================================================
// Host driver of one sofa_query call.
// ========================================================================
#define TRYQ(x)          \
  do {                   \
    int rc_ = (x);       \
    if (rc_) return rc_; \
  } while (0)

static QueryParams make_params(const Index* ix, int k) {
  QueryParams P;
  P.N = ix->N;
  P.Ns = ix->Ns;
  P.T = ix->T;
  P.L = ix->L;
  P.n = ix->n;
  P.NB = ix->NB;
  P.leaf_tiles = ix->leaf_tiles;
  P.k = k;
  P.qk = nullptr;
  P.qo = nullptr;
  P.cap = ix->cand_cap;
  P.group = ix->group;
  P.seed_count = ix->seed_count;
  P.seed_window = ix->seed_window;
  // Rounding-error factors (u = 2^-24): the FP32 bound sum over LW values has
  // relative error <= (LW+3)u; the FP32 distance <= (n+3)u/(1-(n+3)u).  A
  // series is pruned only when its bound proves it farther than the k-th kept
  // distance widened by the 1e-6 tie window; the kept list holds every entry
  // that may fall inside that window.
  const double u = std::ldexp(1.0, -24);
  const double g_lb = (ix->LW + 3) * u;
  const double g_ed = (ix->n + 3) * u / (1.0 - (ix->n + 3) * u);
  const double tie = (1.0 + 1e-6) * (1.0 + 1e-6);
  P.f_prune = std::nextafter((float)(tie * (1.0 + g_lb) / (1.0 - g_ed) * (1.0 + 4 * u)), 2.0f);
  P.f_keep = std::nextafter((float)(tie * (1.0 + g_ed) / (1.0 - g_ed) * (1.0 + 4 * u)), 2.0f);
  return P;
}

// One batch of queries.  With `capturing` the sequence is being recorded into
// a CUDA graph: every buffer has been sized by an earlier eager call, the
// routed-list sizes are upper bounds instead of read-back totals, and only the
// first scan pass is recorded (a full pool is detected after the replay).
// Where a batch's answers go: the k-NN (idx, dist), or, with wid set, each
// query's window (ids, FP64 squared distances, count; wcap entries per query).
struct WindowOut {
  int64_t* wid = nullptr;
  double* wd2 = nullptr;
  int* wcnt = nullptr;
  int wcap = 0;
};

template <int LW, bool NYQ>
static int final_launch(Index* ix, const QueryParams& P, int64_t Q, const float* zq, int64_t* idx, float* dist,
                        const WindowOut& wo, unsigned long long* counters, int* status, cudaStream_t st) {
  QueryScratch& s = ix->qs;
  const size_t nsm = (size_t)ix->n * sizeof(float);
  ix->prof.begin(5, st);
  if (wo.wid)
    k_window<<<(unsigned)Q, 128, nsm, st>>>(P, zq, ix->Z, ix->perm, s.list_p.as<uint32_t>(), s.list_n.as<int>(),
                                            wo.wcap, wo.wid, wo.wd2, wo.wcnt, status);
  else
    k_final<<<(unsigned)Q, 128, nsm, st>>>(P, zq, ix->Z, ix->perm, s.list_p.as<uint32_t>(), s.list_n.as<int>(), idx,
                                           dist, counters, status);
  ix->prof.end(st);
  SOFA_CUDA(cudaGetLastError());
  return 0;
}

template <int LW, bool NYQ>
static int query_batch(Index* ix, const float* qdev, int64_t Q, int k, int64_t* idx, float* dist,
                       cudaStream_t st, bool capturing = false, const WindowOut& wo = WindowOut(),
                       const int* qk = nullptr, const int64_t* qo = nullptr) {
  QueryScratch& s = ix->qs;
  const int n = ix->n, NB = ix->NB;
  const int64_t L = ix->L;
  QueryParams P = make_params(ix, k);
  P.qk = qk;
  P.qo = qo;
  TRYQ(s.zq.ensure(Q * n * sizeof(float)));
  TRYQ(s.qv.ensure(Q * NB * sizeof(float)));
  TRYQ(s.llb.ensure(Q * L * sizeof(float)));
  TRYQ(s.thr.ensure(Q * sizeof(float)));
  TRYQ(s.list_d.ensure(Q * KCAP * sizeof(float)));
  TRYQ(s.list_p.ensure(Q * KCAP * sizeof(uint32_t)));
  TRYQ(s.list_n.ensure(Q * sizeof(int)));
  TRYQ(s.leaf_cnt.ensure((L + 1) * sizeof(int)));
  TRYQ(s.leaf_off.ensure((L + 1) * sizeof(int)));
  TRYQ(s.unit_off.ensure((L + 1) * sizeof(int)));
  TRYQ(s.leaf_cursor.ensure((L + 1) * sizeof(int)));
  TRYQ(s.cand_n.ensure(Q * sizeof(int)));
  TRYQ(s.qflag.ensure(2 * Q * sizeof(int)));
  TRYQ(s.counters.ensure(16 * sizeof(unsigned long long)));

  float* zq = s.zq.as<float>();
  float* qv = s.qv.as<float>();
  float* llb = s.llb.as<float>();
  float* thr = s.thr.as<float>();
  int* status = reinterpret_cast<int*>(s.counters.as<unsigned long long>() + 8);
  int* n_overflow = status + 1;
  int* n_units = status + 2;
  unsigned long long* counters = s.counters.as<unsigned long long>();

  ix->prof.begin(0, st);
  TRYQ(launch_qprep(ix, qdev, Q, zq, qv, st));
  ix->prof.end(st);
  const size_t nsm = (size_t)n * sizeof(float);
  const int32_t* topm = nullptr;
  int top_m = 0;
  int64_t block = 0;
  if (ix->seed_mode == 1) {
    ix->prof.begin(6, st, 6);
    TRYQ(mlp_seed(ix, qv, Q, k, st));
    ix->prof.end(st);
    topm = mlp_topm(ix, &top_m, &block);
  }
  ix->prof.begin(1, st, 2);
  {
    const size_t lsm = (size_t)LW * LB_LEAVES * sizeof(float2);
    SOFA_CUDA(cudaFuncSetAttribute(k_leaf_bounds<LW, NYQ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lsm));
    const dim3 lg((unsigned)ceil_div(L, LB_LEAVES), (unsigned)ceil_div(Q, LB_QUERIES));
    k_leaf_bounds<LW, NYQ><<<lg, 256, lsm, st>>>(Q, L, NB, qv, ix->lenv, ix->edge, llb);
  }
  k_seed<LW, NYQ><<<(unsigned)Q, 256, nsm, st>>>(P, qv, zq, ix->tenv, ix->words, ix->Z, ix->edge, ix->ch,
                                                  ix->beta, ix->alpha, ix->l, ix->keys, ix->keyorder, ix->keybits,
                                                  s.list_d.as<float>(), s.list_p.as<uint32_t>(),
                                                  s.list_n.as<int>(), thr, status, counters, topm, top_m, block);
  ix->prof.end(st);
  SOFA_CUDA(cudaGetLastError());
  if (ix->approximate)  // the approximate search's answer: the seed's kept list, re-scored
    return final_launch<LW, NYQ>(ix, P, Q, zq, idx, dist, wo, counters, status, st);

  // series-bound arithmetic: FP32, or FP16x2 with the derived factor
  // f16 = 1 + (LW/2 + 5) u16 (u16 = 2^-11) on the threshold
  const bool h16 = ix->bound_precision == 1;
  const float f16 = std::nextafter((float)(1.0 + (LW / 2 + 5) * std::ldexp(1.0, -11)), 2.0f);
  const float inv_f16 = std::nextafter(1.0f / f16, 0.0f);
  auto scan_fn = h16 ? k_scan<LW, NYQ, true> : k_scan<LW, NYQ, false>;
  // series-level bound: the SFA word bound, or Eq. (1) on the value codes on
  // the tensor cores (same candidate store, same refinement)
  const bool use_tc = ix->series_bound == 1 && vscan_supported(ix);
  // symbol tables, then the per-tile query lists (leaf_tiles x MAX_GROUP bytes)
  const size_t scan_smem = (size_t)LW * MAX_ALPHA * (sizeof(float2) + (h16 ? sizeof(__half2) : 0)) +
                           (size_t)ix->leaf_tiles * MAX_GROUP;
  SOFA_CUDA(cudaFuncSetAttribute(scan_fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)scan_smem));
  int nb = 0;  // persistent grid: resident CTAs
  {
    int per_sm = 0, sms = 0, dev = 0;
    SOFA_CUDA(cudaGetDevice(&dev));
    SOFA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    SOFA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, scan_fn, 256, scan_smem));
    nb = sms * (per_sm > 0 ? per_sm : 1);
  }

  int* qsel = nullptr;     // queries scanned in this pass (all in the first)
  int* qslot = nullptr;    // their candidate-buffer slots (identity in the first)
  int* qflag_out = s.qflag.as<int>();
  if (!s.h_pinned) SOFA_CUDA(cudaMallocHost((void**)&s.h_pinned, 4 * sizeof(int)));
  int* h_over = s.h_pinned;
  std::vector<int> hflag, hslot, deferred;
  const int max_passes = 64 + 8 * (int)std::min<int64_t>(Q, 1 << 20);
  // graph-eligible batches size the routed lists by their upper bounds
  const bool upper = ix->use_graph && Q * L <= ((int64_t)1 << 28);
  if (upper) {
    TRYQ(s.leaf_q.ensure(((size_t)Q * L + 1) * sizeof(int)));
    TRYQ(s.units.ensure(((size_t)(Q * L / P.group + L) + 1) * sizeof(int4)));
  }
  int rc = 0;
  int64_t slots = Q;
  int* qof = nullptr;  // slot -> query (identity in the first pass)
  // shared candidate pool: sized for the batch, at most 2^29 entries
  const int64_t pool_cap =
      ix->pool_cap > 0 ? ix->pool_cap
                       : std::min<int64_t>((int64_t)1 << 29, std::max<int64_t>((int64_t)1 << 20, Q * std::min<int64_t>(ix->N, 65536)));
  TRYQ(s.pool_q.ensure((size_t)pool_cap * sizeof(int)));
  TRYQ(s.pool_p.ensure((size_t)pool_cap * sizeof(uint32_t)));
  TRYQ(s.pool_lb.ensure((size_t)pool_cap * sizeof(float)));
  TRYQ(s.pool_sp.ensure((size_t)pool_cap * sizeof(uint32_t)));
  TRYQ(s.pool_slb.ensure((size_t)pool_cap * sizeof(float)));
  int* pool_n = status + 3;  // pool appends (stops growing once the pool is full)
  int* n_chunks = status + 4;  // and status + 5: the refinement's chunk cursor
  // persistent refinement grid: resident CTAs of the instantiation that runs
  // (with the value-code stage the static and dynamic shared memory may pass
  // 48 KB, so the dynamic part is declared)
  const int rlevel = (ix->refine_filter && ix->Z8) ? (ix->refine_filter == 2 && ix->VC ? 2 : 1) : 0;
  auto refine_fn = rlevel == 2 ? k_refine<2> : rlevel == 1 ? k_refine<1> : k_refine<0>;
  SOFA_CUDA(cudaFuncSetAttribute(refine_fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)nsm));
  int refine_blocks = 0;
  {
    int per_sm = 0, sms = 0, dev = 0;
    SOFA_CUDA(cudaGetDevice(&dev));
    SOFA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    SOFA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, refine_fn, 256, nsm));
    refine_blocks = sms * (per_sm > 0 ? per_sm : 1);
  }
  for (int pass = 0;; ++pass) {
    TRYQ(s.cand_p.ensure((size_t)slots * P.cap * sizeof(uint32_t)));
    TRYQ(s.cand_lb.ensure((size_t)slots * P.cap * sizeof(float)));
    TRYQ(s.qpool_cnt.ensure((size_t)(slots + 1) * sizeof(int)));
    TRYQ(s.qpool_off.ensure((size_t)(slots + 1) * sizeof(int)));
    TRYQ(s.qcursor.ensure((size_t)(slots + 1) * sizeof(int)));
    TRYQ(s.choff.ensure((size_t)(slots + 1) * sizeof(int)));
    const int64_t max_chunks = ceil_div(slots * (int64_t)P.cap, RSORT) + slots + ceil_div(pool_cap, RSORT);
    TRYQ(s.chunk_q.ensure((size_t)max_chunks * sizeof(int)));
    TRYQ(s.chunk_d.ensure((size_t)max_chunks * KCAP * sizeof(float)));
    TRYQ(s.chunk_p.ensure((size_t)max_chunks * KCAP * sizeof(uint32_t)));
    TRYQ(s.chunk_n.ensure((size_t)max_chunks * sizeof(int)));
    SOFA_CUDA(cudaMemsetAsync(s.qpool_cnt.p, 0, (slots + 1) * sizeof(int), st));
    SOFA_CUDA(cudaMemsetAsync(pool_n, 0, sizeof(int), st));
    SOFA_CUDA(cudaMemsetAsync(s.leaf_cnt.p, 0, (L + 1) * sizeof(int), st));
    SOFA_CUDA(cudaMemsetAsync(s.cand_n.p, 0, Q * sizeof(int), st));
    SOFA_CUDA(cudaMemsetAsync(qflag_out, 0, Q * sizeof(int), st));
    SOFA_CUDA(cudaMemsetAsync(n_overflow, 0, sizeof(int), st));
    const int64_t pairs = Q * L;
    const unsigned rb = (unsigned)ceil_div(pairs, 256);
    ix->prof.begin(2, st, 2);
    k_route_count<<<rb, 256, 0, st>>>(Q, L, llb, thr, qsel, s.leaf_cnt.as<int>(), counters);
    int* cursor = s.leaf_cursor.as<int>();
    k_leaf_scan<<<1, 1024, 0, st>>>(L, P.group, s.leaf_cnt.as<int>(), s.leaf_off.as<int>(), s.unit_off.as<int>(),
                                     cursor);
    ix->prof.end(st);
    SOFA_CUDA(cudaGetLastError());
    // sizes of the routed list and the unit list are only known on the device:
    // read the two totals back (one small copy per pass)
    // When the leaf bounds pass more than half of the (query, leaf block)
    // pairs, the series bounds would prune little: the batch is bounded by the
    // dense tensor-core contraction instead (same candidate store).
    // A graph's recording takes the decision its shape's eager batch made
    // (that batch reads the totals back even with upper-bound buffers).
    bool dense = false;
    if (capturing && pass == 0) {
      dense = ix->graph_dense;
    } else if (!(upper && pass == 0) || ix->graph_probe) {
      if (capturing) return fail(SOFA_ERR_CUDA, "capture needs upper-bound buffers");
      int* tot = h_over + 2;
      SOFA_CUDA(cudaMemcpyAsync(&tot[0], s.leaf_off.as<int>() + L, sizeof(int), cudaMemcpyDeviceToHost, st));
      SOFA_CUDA(cudaMemcpyAsync(&tot[1], s.unit_off.as<int>() + L, sizeof(int), cudaMemcpyDeviceToHost, st));
      SOFA_CUDA(cudaStreamSynchronize(st));
      const int64_t active = pass == 0 ? Q : slots;
      dense = ix->dense_mode != 1 && dense_supported(ix, k) &&
              (ix->dense_mode == 2 || 2 * (int64_t)tot[0] > active * L);
      if (!dense) {
        TRYQ(s.leaf_q.ensure(((size_t)tot[0] + 1) * sizeof(int)));
        TRYQ(s.units.ensure(((size_t)tot[1] + 1) * sizeof(int4)));
      }
    }
    if (pass == 0 && !capturing) ix->last_dense = dense;
    if (dense) {
      // the FP16 query copy (FP16 operands only), the query norms, the contraction
      ix->prof.begin(3, st, ix->Zh ? 3 : 2);
      DenseArgs A;
      A.zq = zq;
      A.Q = (int)Q;
      A.k = k;
      A.cap = P.cap;
      A.pool_cap = pool_cap;
      A.f_prune = P.f_prune;
      A.qsel = qsel;
      A.qslot = qslot;
      A.thr = thr;
      A.cand_p = s.cand_p.as<uint32_t>();
      A.cand_lb = s.cand_lb.as<float>();
      A.cand_n = s.cand_n.as<int>();
      A.pool_n = pool_n;
      A.pool_q = s.pool_q.as<int>();
      A.pool_p = s.pool_p.as<uint32_t>();
      A.pool_lb = s.pool_lb.as<float>();
      A.qpool_cnt = s.qpool_cnt.as<int>();
      A.dump = nullptr;
      A.counters = counters;
      A.status = status;
      A.qn_buf = &s.qn;
      TRYQ(launch_dense(ix, A, st));
      ix->prof.end(st);
      ix->stats[1] += 1;
    } else {
      ix->prof.begin(2, st, 2);
      k_route_fill<<<rb, 256, 0, st>>>(Q, L, llb, thr, qsel, s.leaf_off.as<int>(), cursor, s.leaf_q.as<int>());
      k_units<<<(unsigned)ceil_div(L, 256), 256, 0, st>>>(L, P.group, s.leaf_cnt.as<int>(), s.leaf_off.as<int>(),
                                                           s.unit_off.as<int>(), s.units.as<int4>());
      SOFA_CUDA(cudaMemcpyAsync(n_units, s.unit_off.as<int>() + L, sizeof(int), cudaMemcpyDeviceToDevice, st));
      ix->prof.end(st);
      ix->prof.begin(3, st);
      if (use_tc) {  // Eq. (1) on the value codes, one tcgen05 contraction per (unit, tile)
        VscanArgs V;
        V.units = s.units.as<int4>();
        V.n_units = n_units;
        V.leaf_q = s.leaf_q.as<int>();
        V.qv = qv;
        V.thr = thr;
        V.cap = P.cap;
        V.qslot = qslot;
        V.cand_p = s.cand_p.as<uint32_t>();
        V.cand_lb = s.cand_lb.as<float>();
        V.cand_n = s.cand_n.as<int>();
        V.pool_cap = pool_cap;
        V.pool_n = pool_n;
        V.pool_q = s.pool_q.as<int>();
        V.pool_p = s.pool_p.as<uint32_t>();
        V.pool_lb = s.pool_lb.as<float>();
        V.qpool_cnt = s.qpool_cnt.as<int>();
        V.dump = nullptr;
        V.dumpQ = 0;
        V.counters = counters;
        V.status = status;
        TRYQ(launch_vscan(ix, V, st));
      } else {
        scan_fn<<<nb, 256, scan_smem, st>>>(P, s.units.as<int4>(), n_units, s.leaf_q.as<int>(), qv, thr,
                                             ix->tenv, ix->words, ix->edge, ix->ch, ix->ch16, f16, inv_f16, qslot,
                                             s.cand_p.as<uint32_t>(), s.cand_lb.as<float>(), s.cand_n.as<int>(),
                                             pool_cap, pool_n, s.pool_q.as<int>(), s.pool_p.as<uint32_t>(),
                                             s.pool_lb.as<float>(), s.qpool_cnt.as<int>(), counters);
      }
      ix->prof.end(st);
    }
    SOFA_CUDA(cudaGetLastError());
    ix->prof.begin(7, st, 3);
    k_chunk_plan<<<1, 1024, 0, st>>>(slots, P.cap, s.cand_n.as<int>(), s.qpool_cnt.as<int>(), s.qpool_off.as<int>(),
                                      s.qcursor.as<int>(), s.choff.as<int>(), n_chunks);
    k_pool_scatter<<<nb, 256, 0, st>>>(pool_n, pool_cap, s.pool_q.as<int>(), s.pool_p.as<uint32_t>(),
                                       s.pool_lb.as<float>(), s.qpool_off.as<int>(), s.qcursor.as<int>(),
                                       s.pool_sp.as<uint32_t>(), s.pool_slb.as<float>());
    k_chunk_fill<<<(unsigned)ceil_div(slots, 256), 256, 0, st>>>(slots, P.cap, s.cand_n.as<int>(),
                                                                  s.qpool_cnt.as<int>(), s.choff.as<int>(),
                                                                  s.chunk_q.as<int>());
    ix->prof.end(st);
    ix->prof.begin(4, st, 2);
    const float one_minus_g = std::nextafter((float)(1.0 - (n + 4) * std::ldexp(1.0, -24) / (1.0 - (n + 4) * std::ldexp(1.0, -24))), 0.0f);
    const float one_minus_gv = std::nextafter((float)(1.0 - (NB + 4) * std::ldexp(1.0, -24) / (1.0 - (NB + 4) * std::ldexp(1.0, -24))), 0.0f);
    refine_fn<<<refine_blocks, 256, nsm, st>>>(P, n_chunks, s.chunk_q.as<int>(), s.choff.as<int>(), qof, zq, ix->Z,
                                             s.cand_p.as<uint32_t>(), s.cand_lb.as<float>(), s.cand_n.as<int>(),
                                             s.qpool_cnt.as<int>(), s.qpool_off.as<int>(), s.pool_sp.as<uint32_t>(),
                                             s.pool_slb.as<float>(), thr, s.chunk_d.as<float>(),
                                             s.chunk_p.as<uint32_t>(), s.chunk_n.as<int>(), ix->Z8, ix->s8, ix->e8,
                                             one_minus_g, qv, ix->VC, ix->vsr, ix->vw, one_minus_gv,
                                             n_chunks + 1, counters, status);
    SOFA_CUDA(cudaGetLastError());
    k_merge<<<(unsigned)Q, 256, 0, st>>>(P, qsel, qslot, s.cand_n.as<int>(), s.qpool_cnt.as<int>(), s.choff.as<int>(),
                                         s.chunk_d.as<float>(), s.chunk_p.as<uint32_t>(), s.chunk_n.as<int>(),
                                         s.list_d.as<float>(), s.list_p.as<uint32_t>(), s.list_n.as<int>(), thr,
                                         qflag_out, n_overflow, status);
    ix->prof.end(st);
    SOFA_CUDA(cudaGetLastError());
    if (capturing) break;  // a full pool is detected after the replay
    SOFA_CUDA(cudaMemcpyAsync(h_over, n_overflow, sizeof(int), cudaMemcpyDeviceToHost, st));
    SOFA_CUDA(cudaStreamSynchronize(st));
    if (*h_over == 0 && deferred.empty()) break;
    ix->stats[5] += 1;
    if (pass >= max_passes) {
      rc = fail(SOFA_ERR_TIMEOUT, "candidate overflow passes did not converge");
      break;
    }
    // Next pass: the queries that overflowed, against their tightened
    // thresholds, with an 8x larger candidate region (so a query stops
    // overflowing at the latest when its region holds every series), plus the
    // queries deferred by an earlier pass.  A pass takes only as many queries
    // as fit the region budget at the new size; the rest wait, keeping the
    // kept lists and thresholds they have.
    hflag.assign(Q, 0);
    if (*h_over > 0) {
      SOFA_CUDA(cudaMemcpy(hflag.data(), qflag_out, Q * sizeof(int), cudaMemcpyDeviceToHost));
      P.cap = (int)std::min<int64_t>((int64_t)P.cap * 8, std::max<int64_t>(ix->N, 1));
    }
    for (int i : deferred) hflag[i] = 1;
    deferred.clear();
    const int64_t take_max = std::max<int64_t>(1, ix->cand_budget / P.cap);
    hslot.assign(Q, 0);
    std::vector<int> hsel(Q, 0);
    int64_t m = 0;
    for (int64_t i = 0; i < Q; ++i) {
      if (!hflag[i]) continue;
      if (m < take_max) {
        hsel[i] = 1;
        hslot[i] = (int)m++;
      } else {
        deferred.push_back((int)i);
      }
    }
    slots = m;
    TRYQ(s.qslot.ensure(Q * sizeof(int)));
    SOFA_CUDA(cudaMemcpy(s.qslot.p, hslot.data(), Q * sizeof(int), cudaMemcpyHostToDevice));
    qslot = s.qslot.as<int>();
    TRYQ(s.qsel.ensure(Q * sizeof(int)));
    SOFA_CUDA(cudaMemcpy(s.qsel.p, hsel.data(), Q * sizeof(int), cudaMemcpyHostToDevice));
    qsel = s.qsel.as<int>();
    std::vector<int> hqof((size_t)std::max<int64_t>(m, 1));
    for (int64_t i = 0; i < Q; ++i)
      if (hsel[i]) hqof[hslot[i]] = (int)i;
    TRYQ(s.qof.ensure((size_t)std::max<int64_t>(m, 1) * sizeof(int)));
    SOFA_CUDA(cudaMemcpy(s.qof.p, hqof.data(), hqof.size() * sizeof(int), cudaMemcpyHostToDevice));
    qof = s.qof.as<int>();
    qflag_out = (qflag_out == s.qflag.as<int>()) ? s.qflag.as<int>() + Q : s.qflag.as<int>();
  }
  if (rc) return rc;
  return final_launch<LW, NYQ>(ix, P, Q, zq, idx, dist, wo, counters, status, st);
}

static int dispatch_batch(Index* ix, const float* qp, int64_t qb, int k, int64_t* ip, float* dp, cudaStream_t st,
                          bool capturing, const WindowOut& wo = WindowOut(), const int* qk = nullptr,
                          const int64_t* qo = nullptr) {
  if (ix->LW == 16)
    return ix->nyq_first ? query_batch<16, true>(ix, qp, qb, k, ip, dp, st, capturing, wo, qk, qo)
                         : query_batch<16, false>(ix, qp, qb, k, ip, dp, st, capturing, wo, qk, qo);
  return ix->nyq_first ? query_batch<32, true>(ix, qp, qb, k, ip, dp, st, capturing, wo, qk, qo)
                       : query_batch<32, false>(ix, qp, qb, k, ip, dp, st, capturing, wo, qk, qo);
}

// A batch through a recorded CUDA graph.  The first batch of a shape runs
// eagerly (sizing every buffer and producing its answers) and is then recorded
// from fixed staging buffers; later batches copy their queries in, replay the
// graph and copy the answers out.  If a replay's candidate pool ran full, the
// batch is recomputed eagerly, so answers are always exact.
static int graph_batch(Index* ix, const float* qp, int64_t qb, int k, int64_t* ip, float* dp, cudaStream_t st) {
  QueryScratch& s = ix->qs;
  if (!ix->gstream) {
    SOFA_CUDA(cudaStreamCreateWithFlags(&ix->gstream, cudaStreamNonBlocking));
    SOFA_CUDA(cudaEventCreateWithFlags(&ix->gev[0], cudaEventDisableTiming));
    SOFA_CUDA(cudaEventCreateWithFlags(&ix->gev[1], cudaEventDisableTiming));
  }
  const int64_t key[16] = {qb, k, ix->bound_precision, ix->refine_filter, ix->seed_mode, ix->group, ix->cand_cap,
                           ix->seed_count, ix->seed_window, ix->pool_cap, ix->LW, ix->nyq_first, ix->approximate,
                           ix->dense_mode, ix->cand_budget, ix->series_bound | (ix->tile_checks << 1)};
  Index::GraphEntry* e = nullptr;
  for (auto& g : ix->graphs)
    if (std::equal(key, key + 16, g.key)) e = &g;
  if (e && !e->failed && e->gen != g_buf_generation) {  // buffers moved since the recording
    cudaGraphExecDestroy(e->exec);
    e->exec = nullptr;
    e = nullptr;
    ix->graphs.erase(std::remove_if(ix->graphs.begin(), ix->graphs.end(),
                                    [&](const Index::GraphEntry& g) { return std::equal(key, key + 16, g.key); }),
                     ix->graphs.end());
  }
  if (e && e->failed) return dispatch_batch(ix, qp, qb, k, ip, dp, st, false);
  if (!e) {
    TRYQ(s.graph_in.ensure((size_t)qb * ix->n * sizeof(float)));
    TRYQ(s.graph_out.ensure((size_t)qb * k * (sizeof(int64_t) + sizeof(float))));
    ix->graph_probe = true;  // the eager batch decides dense or scan for the recording
    const int rc0 = dispatch_batch(ix, qp, qb, k, ip, dp, st, false);  // sizes every buffer; the answers
    ix->graph_probe = false;
    TRYQ(rc0);
    ix->graph_dense = ix->last_dense;
    SOFA_CUDA(cudaStreamSynchronize(st));
    const unsigned long long gen0 = g_buf_generation;
    Index::GraphEntry ne;
    std::copy(key, key + 16, ne.key);
    ne.exec = nullptr;
    ne.failed = true;
    const bool prof_on = ix->prof.on;
    ix->prof.on = false;
    cudaGraph_t graph = nullptr;
    int rc = 0;
    if (cudaStreamBeginCapture(ix->gstream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      int64_t* gi = s.graph_out.as<int64_t>();
      float* gd = reinterpret_cast<float*>(gi + qb * k);
      rc = dispatch_batch(ix, s.graph_in.as<float>(), qb, k, gi, gd, ix->gstream, true);
      cudaError_t ec = cudaStreamEndCapture(ix->gstream, &graph);
      if (!rc && ec == cudaSuccess && graph && g_buf_generation == gen0 &&
          cudaGraphInstantiate(&ne.exec, graph, 0) == cudaSuccess)
        ne.failed = false;
    }
    cudaGetLastError();  // a refused recording only disables the graph for this shape
    if (graph) cudaGraphDestroy(graph);
    ix->prof.on = prof_on;
    ne.gen = g_buf_generation;
    if (!ne.failed) ix->stats[7] += 1;
    ix->graphs.push_back(ne);
    (void)rc;
    return 0;
  }
  SOFA_CUDA(cudaEventRecord(ix->gev[0], st));
  SOFA_CUDA(cudaStreamWaitEvent(ix->gstream, ix->gev[0], 0));
  SOFA_CUDA(cudaMemcpyAsync(s.graph_in.p, qp, (size_t)qb * ix->n * sizeof(float), cudaMemcpyDeviceToDevice,
                            ix->gstream));
  SOFA_CUDA(cudaGraphLaunch(e->exec, ix->gstream));
  ix->stats[6] += 1;
  int* status = reinterpret_cast<int*>(s.counters.as<unsigned long long>() + 8);
  SOFA_CUDA(cudaMemcpyAsync(s.h_pinned, status + 1, sizeof(int), cudaMemcpyDeviceToHost, ix->gstream));
  SOFA_CUDA(cudaStreamSynchronize(ix->gstream));
  if (*s.h_pinned > 0) return dispatch_batch(ix, qp, qb, k, ip, dp, st, false);  // pool ran full
  int64_t* gi = s.graph_out.as<int64_t>();
  float* gd = reinterpret_cast<float*>(gi + qb * k);
  SOFA_CUDA(cudaMemcpyAsync(ip, gi, (size_t)qb * k * sizeof(int64_t), cudaMemcpyDeviceToDevice, ix->gstream));
  SOFA_CUDA(cudaMemcpyAsync(dp, gd, (size_t)qb * k * sizeof(float), cudaMemcpyDeviceToDevice, ix->gstream));
  SOFA_CUDA(cudaEventRecord(ix->gev[1], ix->gstream));
  SOFA_CUDA(cudaStreamWaitEvent(st, ix->gev[1], 0));
  return 0;
}

int run_query(Index* ix, const float* q, int64_t Q, int k, int64_t* idx, float* dist, cudaStream_t st,
              const int* qk, const int64_t* qo) {
  NvtxScope range(ix->prof, "sofa_query");
  QueryScratch& s = ix->qs;
  const bool fresh = s.counters.p == nullptr;
  TRYQ(s.counters.ensure(16 * sizeof(unsigned long long)));
  if (fresh) SOFA_CUDA(cudaMemsetAsync(s.counters.p, 0, 16 * sizeof(unsigned long long), st));
  int* status = reinterpret_cast<int*>(s.counters.as<unsigned long long>() + 8);
  SOFA_CUDA(cudaMemsetAsync(status, 0, sizeof(int), st));
  const int64_t QB = 8192;
  for (int64_t q0 = 0; q0 < Q; q0 += QB) {
    const int64_t qb = std::min(QB, Q - q0);
    const float* qp = q + q0 * ix->n;
    if (qk) {  // mixed k: each query's results at its own offset (absolute); eager batches
      TRYQ(dispatch_batch(ix, qp, qb, k, idx, dist, st, false, WindowOut(), qk + q0, qo + q0));
      continue;
    }
    int64_t* ip = idx + q0 * k;
    float* dp = dist + q0 * k;
    const bool graph = ix->use_graph && !ix->prof.on && qb * ix->L <= ((int64_t)1 << 28);
    int rc = graph ? graph_batch(ix, qp, qb, k, ip, dp, st) : dispatch_batch(ix, qp, qb, k, ip, dp, st, false);
    if (rc) return rc;
  }
  ix->stats[0] += Q;
  return 0;
}

// The k-NN windows of Q queries (sofa_query_window), batch by batch, eagerly.
int run_query_window(Index* ix, const float* q, int64_t Q, int k, int cap, int64_t* wid, double* wd2, int* wcnt,
                     cudaStream_t st) {
  NvtxScope range(ix->prof, "sofa_query_window");
  QueryScratch& s = ix->qs;
  const bool fresh = s.counters.p == nullptr;
  TRYQ(s.counters.ensure(16 * sizeof(unsigned long long)));
  if (fresh) SOFA_CUDA(cudaMemsetAsync(s.counters.p, 0, 16 * sizeof(unsigned long long), st));
  int* status = reinterpret_cast<int*>(s.counters.as<unsigned long long>() + 8);
  SOFA_CUDA(cudaMemsetAsync(status, 0, sizeof(int), st));
  const int64_t QB = 8192;
  for (int64_t q0 = 0; q0 < Q; q0 += QB) {
    const int64_t qb = std::min(QB, Q - q0);
    WindowOut wo;
    wo.wid = wid + q0 * cap;
    wo.wd2 = wd2 + q0 * cap;
    wo.wcnt = wcnt + q0;
    wo.wcap = cap;
    TRYQ(dispatch_batch(ix, q + q0 * ix->n, qb, k, nullptr, nullptr, st, false, wo));
  }
  ix->stats[0] += Q;
  return 0;
}

// Scan bounds of Q queries against every series (testing aid): out[q][perm[p]].
template <int LW, bool NYQ>
__global__ void k_all_bounds(int64_t Q, int64_t N, int NB, const float* __restrict__ qv,
                             const uint8_t* __restrict__ words, const uint32_t* __restrict__ perm,
                             const float2* __restrict__ ch, float* __restrict__ out) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t q = blockIdx.y;
  if (p >= N) return;
  float qq[LW];
#pragma unroll
  for (int j = 0; j < LW; ++j) qq[j] = qv[q * NB + j];
  float c[LW], h[LW];
  load_word_bounds<LW>(words, p, true, ch, c, h);
  out[q * N + perm[p]] = 2.0f * word_bound<LW, NYQ>(c, h, qq);
}

int launch_lower_bounds(Index* ix, const float* qv, int64_t Q, float* out, cudaStream_t st) {
  // queries go on gridDim.y, at most 65535 per launch
  for (int64_t q0 = 0; q0 < Q; q0 += 65535) {
    const int64_t qc = std::min<int64_t>(65535, Q - q0);
    const float* qvc = qv + q0 * ix->NB;
    float* oc = out + q0 * ix->N;
    dim3 g((unsigned)ceil_div(ix->N, 256), (unsigned)qc);
    if (ix->LW == 16) {
      if (ix->nyq_first) k_all_bounds<16, true><<<g, 256, 0, st>>>(qc, ix->N, ix->NB, qvc, ix->words, ix->perm, ix->ch, oc);
      else k_all_bounds<16, false><<<g, 256, 0, st>>>(qc, ix->N, ix->NB, qvc, ix->words, ix->perm, ix->ch, oc);
    } else {
      if (ix->nyq_first) k_all_bounds<32, true><<<g, 256, 0, st>>>(qc, ix->N, ix->NB, qvc, ix->words, ix->perm, ix->ch, oc);
      else k_all_bounds<32, false><<<g, 256, 0, st>>>(qc, ix->N, ix->NB, qvc, ix->words, ix->perm, ix->ch, oc);
    }
    SOFA_CUDA(cudaGetLastError());
  }
  return 0;
}

}  // namespace sofa
