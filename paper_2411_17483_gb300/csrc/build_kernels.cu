// Index construction kernels: SFA summarisation (Alg. 1 MCB, Alg. 2 SFA
// Transform) and the flat key-sorted layout that replaces the MESSI tree.
#include <cub/device/device_radix_sort.cuh>

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <vector>

#include "sofa_internal.cuh"

namespace sofa {

constexpr int ROWS = 32;       // rows per CTA in the row kernels
constexpr int WTHREADS = 256;  // threads per CTA of the row kernels (all stage; per-row work as stated)

// Stage rows first..first+ROWS-1 (global rows row*stride) of a row-major
// matrix by every thread of the CTA, 16-byte loads when n % 4 == 0, into the
// padded layout: row r at r*(n+1), so that a thread walking its own row hits
// its own banks.
__device__ inline void stage_rows_vec(const float* __restrict__ x, int64_t first, int64_t R, int n, float* sm,
                                      int64_t stride = 1) {
  const int nr = (int)(R - first < ROWS ? R - first : ROWS);
  if ((n & 3) == 0) {
    const int n4 = n >> 2;
    const float4* x4 = reinterpret_cast<const float4*>(x);
    for (int e = threadIdx.x; e < nr * n4; e += blockDim.x) {
      const int r = e / n4, c = e - r * n4;
      const float4 v = __ldg(x4 + (first + r) * stride * n4 + c);
      float* d = sm + r * (n + 1) + 4 * c;
      d[0] = v.x;
      d[1] = v.y;
      d[2] = v.z;
      d[3] = v.w;
    }
  } else {
    for (int e = threadIdx.x; e < nr * n; e += blockDim.x) {
      const int r = e / n, t = e - r * n;
      sm[r * (n + 1) + t] = x[(first + r) * stride * (int64_t)n + t];
    }
  }
  __syncthreads();
}

// ------------------------------------------------------------------------
// Canonical z-normalisation and projection of rows onto NB basis columns.
// x row r of the launch is global row r*stride.  With NORMALIZE the input is
// raw and is z-normalised (Sec. II Def. z-ED); otherwise it is already
// canonical.  Outputs (each optional): z (R x n), v (R x NB or NB x R when
// vt), stats (mu, 1/sigma).
template <bool NORMALIZE>
__global__ void k_rows_project(const float* __restrict__ x, int64_t R, int n, int64_t stride,
                               const float* __restrict__ basis, int bstride, int NB, float* __restrict__ z,
                               float* __restrict__ v, int vt, double2* __restrict__ stats) {
  extern __shared__ float sm[];
  const int64_t first = (int64_t)blockIdx.x * ROWS;
  stage_rows_vec(x, first, R, n, sm, stride);  // every thread of the CTA stages
  const int r = threadIdx.x;
  const int64_t row = first + r;
  if (r >= ROWS || row >= R) return;        // one thread per row from here
  const float* my = sm + r * (n + 1);
  double mu = 0.0, inv = 1.0;
  if (NORMALIZE) znorm_stats_seq(my, n, 1, mu, inv);
  if (stats) stats[row] = make_double2(mu, inv);
  float acc[NB_MAX];
#pragma unroll
  for (int j = 0; j < NB_MAX; ++j) acc[j] = 0.f;
  for (int t = 0; t < n; ++t) {
    float zt = NORMALIZE ? znorm_value(my[t], mu, inv) : my[t];
    if (z) z[row * n + t] = zt;
    if (v) {
      const float* b = basis + (int64_t)t * bstride;
#pragma unroll
      for (int j = 0; j < NB_MAX; ++j)
        if (j < NB) acc[j] = fmaf(zt, __ldg(b + j), acc[j]);
    }
  }
  if (v) {
#pragma unroll
    for (int j = 0; j < NB_MAX; ++j)
      if (j < NB) {
        if (vt) v[(int64_t)j * R + row] = acc[j];
        else v[row * NB + j] = acc[j];
      }
  }
}

// Query transform (Alg. 2 on queries, keeping the values), RQ query rows per
// CTA of 256 threads (RQ a power of two <= 32, chosen per batch so that
// there are at least two CTAs per SM).  Lane r of warp 0 takes row r's
// canonical FP64 statistics (the same left-to-right sums as every
// z-normalisation here: a dependent chain of about 2n FP64 additions, on all
// RQ lanes at once); all threads then write the z-values; for the projection
// warp w takes rows w, w+8, w+16, w+24 (those below RQ) and lane c the basis
// columns c and c+32, each a sequence of one FMA per t in ascending t (the
// thread-per-row kernel's sequence, so the values are the same bit for bit),
// the basis loads shared by the warp's rows.
template <int RQ>
__global__ void __launch_bounds__(256) k_qprep(const float* __restrict__ x, int64_t R, int n,
                                               const float* __restrict__ basis, int NB, float* __restrict__ z,
                                               float* __restrict__ v) {
  static_assert(RQ >= 1 && RQ <= 32 && (RQ & (RQ - 1)) == 0, "RQ: a power of two <= 32 (one warp's lanes)");
  constexpr int RPW = (RQ + 7) / 8;  // rows per warp in the projection
  extern __shared__ float sm[];      // RQ x (n + 1): the rows, then their z-values in place
  __shared__ double s_mu[RQ], s_inv[RQ];
  const int64_t first = (int64_t)blockIdx.x * RQ;
  const int nr = (int)(R - first < RQ ? R - first : RQ);
  for (int e = threadIdx.x; e < RQ * n; e += blockDim.x) {
    const int r = e / n, t = e - r * n;
    sm[r * (n + 1) + t] = r < nr ? x[(first + r) * n + t] : 0.f;
  }
  __syncthreads();
  if (threadIdx.x < nr) {
    double mu, inv;
    znorm_stats_seq(sm + threadIdx.x * (n + 1), n, 1, mu, inv);
    s_mu[threadIdx.x] = mu;
    s_inv[threadIdx.x] = inv;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nr * n; e += blockDim.x) {
    const int r = e / n, t = e - r * n;
    const float zt = znorm_value(sm[r * (n + 1) + t], s_mu[r], s_inv[r]);
    sm[r * (n + 1) + t] = zt;
    z[(first + r) * n + t] = zt;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp >= RQ) return;  // no rows for this warp (RQ < 8); no barrier follows
  const int c0 = lane, c1 = lane + 32;
  float acc[RPW][2];
#pragma unroll
  for (int i = 0; i < RPW; ++i) acc[i][0] = acc[i][1] = 0.f;
  for (int t = 0; t < n; ++t) {
    const float b0 = c0 < NB ? __ldg(basis + (int64_t)t * NB + c0) : 0.f;
    const float b1 = c1 < NB ? __ldg(basis + (int64_t)t * NB + c1) : 0.f;
#pragma unroll
    for (int i = 0; i < RPW; ++i) {
      const float zt = sm[(warp + 8 * i) * (n + 1) + t];
      acc[i][0] = fmaf(zt, b0, acc[i][0]);
      acc[i][1] = fmaf(zt, b1, acc[i][1]);
    }
  }
#pragma unroll
  for (int i = 0; i < RPW; ++i) {
    const int r = warp + 8 * i;
    if (r < nr) {
      if (c0 < NB) v[(first + r) * NB + c0] = acc[i][0];
      if (c1 < NB) v[(first + r) * NB + c1] = acc[i][1];
    }
  }
}

template <int RQ>
static int launch_qprep_rq(Index* ix, const float* q, int64_t Q, float* zq, float* qv, cudaStream_t st) {
  const size_t smem = (size_t)RQ * (ix->n + 1) * sizeof(float);
  SOFA_CUDA(cudaFuncSetAttribute(k_qprep<RQ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_qprep<RQ><<<(unsigned)ceil_div(Q, RQ), 256, smem, st>>>(q, Q, ix->n, ix->basis, ix->NB, zq, qv);
  SOFA_CUDA(cudaGetLastError());
  return 0;
}

// ------------------------------------------------------------------------
// SFA words of every series (Alg. 2): z-normalise, project on the l word
// columns in FP32, quantise by counting breakpoints <= value (half-open bins
// [beta(a-1), beta(a))), then form the 64-bit layout key from the symbol bits
// in the order given by keyorder (dim << 3 | bit).  A CTA of WTHREADS
// threads takes ROWS rows: all threads stage them; one thread per row runs
// the canonical FP64 statistics (a sequential chain); all threads write the
// z-values in place; thread (r, g) projects row r on columns g*CPT..+CPT, one
// FMA per t in ascending t for each column (so every value is the same FP32
// sequence as a thread-per-row projection); one thread per row packs the
// word and its key.
template <int LW>
__global__ void __launch_bounds__(WTHREADS) k_words(const float* __restrict__ x, int64_t N, int n,
                                                    const float* __restrict__ basis, int NB,
                                                    const float* __restrict__ beta, int alpha, int l,
                                                    const uint8_t* __restrict__ keyorder, int keybits,
                                                    uint8_t* __restrict__ words, uint64_t* __restrict__ keys,
                                                    uint32_t* __restrict__ ids, double2* __restrict__ stats) {
  constexpr int GPR = WTHREADS / ROWS;  // threads per row in the projection (8)
  constexpr int CPT = LW / GPR;         // columns per thread (2 or 4)
  extern __shared__ float sm[];
  float* sbeta = sm;                                  // LW x (alpha+1)
  float* srows = sm + LW * (alpha + 1);               // ROWS x (n+1)
  uint8_t* ssym = reinterpret_cast<uint8_t*>(srows + ROWS * (n + 1));  // ROWS x LW
  __shared__ double s_mu[ROWS], s_inv[ROWS];
  for (int e = threadIdx.x; e < LW * (alpha + 1); e += blockDim.x) sbeta[e] = beta[e];
  const int64_t first = (int64_t)blockIdx.x * ROWS;
  const int nr = (int)(N - first < ROWS ? N - first : ROWS);
  stage_rows_vec(x, first, N, n, srows);
  const int tid = threadIdx.x;
  if (tid < nr) {
    double mu, inv;
    znorm_stats_seq(srows + tid * (n + 1), n, 1, mu, inv);
    s_mu[tid] = mu;
    s_inv[tid] = inv;
    stats[first + tid] = make_double2(mu, inv);
  }
  __syncthreads();
  for (int e = tid; e < nr * n; e += blockDim.x) {
    const int r = e / n, t = e - r * n;
    srows[r * (n + 1) + t] = znorm_value(srows[r * (n + 1) + t], s_mu[r], s_inv[r]);
  }
  __syncthreads();
  const int r = tid / GPR, g = tid - r * GPR;
  if (r < nr) {
    const float* my = srows + r * (n + 1);
    float acc[CPT];
#pragma unroll
    for (int c = 0; c < CPT; ++c) acc[c] = 0.f;
    const float* bcol = basis + g * CPT;
    for (int t = 0; t < n; ++t) {
      const float zt = my[t];
#pragma unroll
      for (int c = 0; c < CPT; ++c) acc[c] = fmaf(zt, __ldg(bcol + (int64_t)t * NB + c), acc[c]);
    }
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
      const int j = g * CPT + c;
      int sym = 0;
      if (j < l) {
        const float* bj = sbeta + j * (alpha + 1);
        for (int step = 128; step > 0; step >>= 1)
          if (sym + step <= alpha - 1 && bj[sym + step] <= acc[c]) sym += step;
      }
      ssym[r * LW + j] = (uint8_t)sym;
    }
  }
  __syncthreads();
  if (tid >= nr) return;
  const int64_t row = first + tid;
  uint32_t packed[LW / 4];
#pragma unroll
  for (int q = 0; q < LW / 4; ++q)
    packed[q] = (uint32_t)ssym[tid * LW + 4 * q] | ((uint32_t)ssym[tid * LW + 4 * q + 1] << 8) |
                ((uint32_t)ssym[tid * LW + 4 * q + 2] << 16) | ((uint32_t)ssym[tid * LW + 4 * q + 3] << 24);
  uint4* wo = reinterpret_cast<uint4*>(words + row * LW);
#pragma unroll
  for (int q = 0; q < LW / 16; ++q)
    wo[q] = make_uint4(packed[4 * q], packed[4 * q + 1], packed[4 * q + 2], packed[4 * q + 3]);
  uint64_t key = 0;
  for (int t = 0; t < keybits; ++t) {
    int d = keyorder[t] >> 3, b = keyorder[t] & 7;
    uint32_t word = packed[d >> 2];
    uint64_t bit = (word >> ((d & 3) * 8 + b)) & 1u;
    key |= bit << (63 - t);
  }
  keys[row] = key;
  ids[row] = (uint32_t)row;
}

// ------------------------------------------------------------------------
// Per-value mean / variance of every candidate Fourier value over the sample
// (Alg. 1 steps 1-2): V = Zs[S x n] * Bf[n x ncand] as a register-tiled FP32
// GEMM whose epilogue accumulates sum(v) and sum(v^2) in FP64 per column.
// Row blocks are assigned to CTAs statically (blockIdx.x + i*gridDim.x), so
// the FP64 partials are deterministic.
constexpr int GM = 64, GN = 64, GK = 32;
__global__ void __launch_bounds__(256) k_dft_var(const float* __restrict__ Zs, int64_t S, int n,
                                                 const float* __restrict__ Bf, int ncand,
                                                 double2* __restrict__ partial) {
  __shared__ float As[GK][GM + 4];
  __shared__ float Bs[GK][GN + 4];
  __shared__ double red_s[16][GN];
  __shared__ double red_q[16][GN];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int col0 = blockIdx.y * GN;
  double cs[4] = {0, 0, 0, 0}, cq[4] = {0, 0, 0, 0};
  for (int64_t rb = blockIdx.x; rb * GM < S; rb += gridDim.x) {
    const int64_t row0 = rb * GM;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    for (int k0 = 0; k0 < n; k0 += GK) {
      for (int e = threadIdx.x; e < GM * GK; e += 256) {
        int r = e / GK, kk = e % GK;
        int64_t gr = row0 + r;
        int gk = k0 + kk;
        As[kk][r] = (gr < S && gk < n) ? Zs[gr * n + gk] : 0.f;
      }
      for (int e = threadIdx.x; e < GK * GN; e += 256) {
        int kk = e / GN, c = e % GN;
        int gk = k0 + kk, gc = col0 + c;
        Bs[kk][c] = (gk < n && gc < ncand) ? Bf[(int64_t)gk * ncand + gc] : 0.f;
      }
      __syncthreads();
#pragma unroll 8
      for (int kk = 0; kk < GK; ++kk) {
        float a[4], b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
        for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
      }
      __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (row0 + ty * 4 + i < S) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          double vv = (double)acc[i][j];
          cs[j] += vv;
          cq[j] += vv * vv;
        }
      }
    }
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    red_s[ty][tx * 4 + j] = cs[j];
    red_q[ty][tx * 4 + j] = cq[j];
  }
  __syncthreads();
  if (threadIdx.x < GN) {
    double s = 0, q = 0;
    for (int i = 0; i < 16; ++i) {
      s += red_s[i][threadIdx.x];
      q += red_q[i][threadIdx.x];
    }
    int gc = col0 + threadIdx.x;
    if (gc < ncand) partial[(int64_t)blockIdx.x * ncand + gc] = make_double2(s, q);
  }
}

__global__ void k_var_reduce(const double2* __restrict__ partial, int nparts, int ncand, int64_t S,
                             double* __restrict__ var) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncand) return;
  double s = 0, q = 0;
  for (int p = 0; p < nparts; ++p) {
    double2 v = partial[(int64_t)p * ncand + c];
    s += v.x;
    q += v.y;
  }
  double mean = s / (double)S;
  double v = q / (double)S - mean * mean;
  var[c] = v > 0 ? v : 0.0;
}

// ------------------------------------------------------------------------
// Candidate value c -> (coefficient k, part): k = c/2 + 1, part = c & 1
// (k ascending, real before imaginary; a Nyquist imaginary part, when the pool
// reaches n/2 with n even, would be the last id and is not a candidate).
__host__ __device__ inline int num_candidates(int n, int pool) {
  int K = (pool <= 0) ? n / 2 : min(pool, n / 2);
  return 2 * K - ((n % 2 == 0 && 2 * K == n) ? 1 : 0);
}

// Variance-based selection (Sec. IV "Novel Feature Selection", Alg. 1 step 2):
// rank = number of candidates with larger variance (ties: smaller id first).
// The top m = min(2l, ncand) are kept; the first l form the word, with a
// selected Nyquist value moved to word position 0.  mode 1 keeps the first ids.
__global__ void k_select(const double* __restrict__ var, int ncand, int n, int l, int mode,
                         int32_t* __restrict__ sel, int32_t* __restrict__ sel_k, int32_t* __restrict__ sel_part,
                         double* __restrict__ var_sel, int32_t* __restrict__ nyq_first) {
  __shared__ int order[1024];
  const int m = min(2 * l, ncand);
  for (int c = threadIdx.x; c < ncand; c += blockDim.x) {
    int rank = c;
    if (mode == 0) {
      rank = 0;
      double vc = var[c];
      for (int d = 0; d < ncand; ++d) {
        double vd = var[d];
        rank += (vd > vc) || (vd == vc && d < c);
      }
    }
    if (rank < m) order[rank] = c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int word[SOFA_MAX_WORD];
    int lw = min(l, m);
    int nyq = -1;
    for (int j = 0; j < lw; ++j)
      if (n % 2 == 0 && 2 * (order[j] / 2 + 1) == n) nyq = j;
    int w = 0;
    if (nyq >= 0) word[w++] = order[nyq];
    for (int j = 0; j < lw; ++j)
      if (j != nyq) word[w++] = order[j];
    for (int j = 0; j < m; ++j) {
      int c = j < lw ? word[j] : order[j];
      sel[j] = c;
      sel_k[j] = c / 2 + 1;
      sel_part[j] = c & 1;
      var_sel[j] = var[c];
    }
    *nyq_first = nyq >= 0 ? 1 : 0;
  }
}

// Selected (k, part) of the user's ids plus their variances.
__global__ void k_user_sel(const int32_t* __restrict__ sel, int m, int n, const double* __restrict__ var,
                           int32_t* __restrict__ sel_k, int32_t* __restrict__ sel_part,
                           double* __restrict__ var_sel, int32_t* __restrict__ nyq_first, int l) {
  if (threadIdx.x != 0) return;
  int nyq = 0;
  for (int j = 0; j < m; ++j) {
    int c = sel[j];
    sel_k[j] = c / 2 + 1;
    sel_part[j] = c & 1;
    var_sel[j] = var[c];
    if (j == 0 && l > 0 && n % 2 == 0 && 2 * (c / 2 + 1) == n) nyq = 1;
  }
  *nyq_first = nyq;
}

// Orthonormal real DFT basis column of value (k, part) at sample t:
// n^{-1/2} cos(2 pi m/n) for the real part, -n^{-1/2} sin(2 pi m/n) for the
// imaginary part, m = k t mod n (Alg. 1/2 step 1, Eq. 1 normalisation).
__device__ inline float basis_value(int n, int k, int part, int t) {
  int64_t m = ((int64_t)k * t) % n;
  double s, c;
  sincospi(2.0 * (double)m / (double)n, &s, &c);
  double sc = rsqrt((double)n);
  return (float)((part == 0 ? c : -s) * sc);
}

// Full candidate basis Bf[n][ncand] for the variance pass.
__global__ void k_basis_full(int n, int ncand, float* __restrict__ Bf) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * ncand) return;
  int t = (int)(e / ncand), c = (int)(e % ncand);
  Bf[e] = basis_value(n, c / 2 + 1, c & 1, t);
}

// Projection basis [n][NB]: columns [0, LW) are the word values (zero beyond
// l), columns [LW, NB) the remaining selected values (zero beyond nsel).
__global__ void k_basis_sel(int n, int NB, int LW, int l, int nsel, const int32_t* __restrict__ sel_k,
                            const int32_t* __restrict__ sel_part, float* __restrict__ B) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * NB) return;
  int t = (int)(e / NB), col = (int)(e % NB);
  int j = col < LW ? (col < l ? col : -1) : (l + col - LW < nsel ? l + col - LW : -1);
  B[e] = j < 0 ? 0.f : basis_value(n, sel_k[j], sel_part[j], t);
}

// Greedy key bit order: repeatedly take the next most significant symbol bit
// of the word value with the largest var_j / 4^{bits already taken} (each bit
// halves that value's interval, quartering its squared width).
__global__ void k_keyorder(const double* __restrict__ var_sel, int l, int bps, uint8_t* __restrict__ order,
                           int32_t* __restrict__ nbits) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int taken[SOFA_MAX_WORD];
  for (int j = 0; j < l; ++j) taken[j] = 0;
  int total = min(64, l * bps);
  for (int t = 0; t < total; ++t) {
    int best = -1;
    double bv = -1.0;
    for (int j = 0; j < l; ++j) {
      if (taken[j] >= bps) continue;
      double v = ldexp(var_sel[j], -2 * taken[j]);
      if (v > bv) {
        bv = v;
        best = j;
      }
    }
    order[t] = (uint8_t)((best << 3) | (bps - 1 - taken[best]));
    taken[best]++;
  }
  *nbits = total;
}

// MCB breakpoints from the sorted sample values of word value j
// (Alg. 1 step 3): equi-depth beta(a) = sorted[floor(a S / alpha)], equi-width
// beta(a) = min + a (max - min) / alpha (FP64), beta(0) = -inf, beta(alpha) = +inf.
__global__ void k_bins(const float* __restrict__ sorted, int64_t S, int l, int alpha, int binning,
                       float* __restrict__ beta) {
  int j = blockIdx.x;
  const float* v = sorted + (int64_t)j * S;
  for (int a = threadIdx.x; a <= alpha; a += blockDim.x) {
    float b;
    if (a == 0) b = -INFINITY;
    else if (a == alpha) b = INFINITY;
    else if (binning == 0) b = v[((int64_t)a * S) / alpha];
    else {
      double lo = v[0], hi = v[S - 1];
      b = (float)(lo + (double)a * (hi - lo) / (double)alpha);
    }
    beta[(int64_t)j * (alpha + 1) + a] = b;
  }
}

// Per-symbol bound tables.  edge[j][s] = [beta_j(s) - delta, beta_j(s+1) + delta]
// rounded outward, with the open outer ends replaced by -/+ (vmax + delta)
// (no z-normalised value exceeds vmax = sqrt(n) in magnitude).  ch[j][s] is
// the same interval as (centre, half-width), the half-width rounded up and
// widened by eps_abs to absorb the rounding of |q - centre|.  Unused dims and
// symbols get an interval that never contributes.
// ch16[j][s] holds the same interval for the FP16 bound as (centre, -half
// width) in half precision: the centre rounded to nearest, the half-width
// widened by 4 u16 outer (rounding of the centre, of the query value and of
// q - c, u16 = 2^-11) and rounded up.
__global__ void k_tables(const float* __restrict__ beta, int l, int LW, int alpha, float delta, float outer,
                         float eps_abs, float2* __restrict__ edge, float2* __restrict__ ch,
                         __half2* __restrict__ ch16) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= LW * MAX_ALPHA) return;
  int j = e / MAX_ALPHA, s = e % MAX_ALPHA;
  const float BIG = 1e30f;
  if (j >= l || s >= alpha) {
    edge[e] = make_float2(-BIG, BIG);
    ch[e] = make_float2(0.f, BIG);
    ch16[e] = __halves2half2(__float2half_rn(0.f), __float2half_rn(-60000.f));
    return;
  }
  const float* bj = beta + (int64_t)j * (alpha + 1);
  float lo = (s == 0) ? -outer : __fsub_rd(bj[s], delta);
  float hi = (s == alpha - 1) ? outer : __fadd_ru(bj[s + 1], delta);
  lo = fmaxf(lo, -outer);
  hi = fminf(hi, outer);
  if (hi < lo) hi = lo;
  edge[e] = make_float2(lo, hi);
  float c = 0.5f * (lo + hi);
  float h = fmaxf(__fsub_ru(c, lo), __fsub_ru(hi, c));
  ch[e] = make_float2(c, __fadd_ru(h, eps_abs));
  const __half c16 = __float2half_rn(c);
  const float cerr = fabsf(__half2float(c16) - c);
  const float u16 = 1.0f / 2048.0f;
  const float h16 = __fadd_ru(__fadd_ru(h, cerr), 4.0f * u16 * outer);
  __half hh = __float2half_ru(h16);
  ch16[e] = __halves2half2(c16, __hneg(hh));
}

// Key-sorted layout: Z[p] = canonical z-normalisation of data row perm[p]
// (from the stored mu, 1/sigma), words[p] = words of that row.  Warp per row.
template <int LW>
__global__ void k_layout(const float* __restrict__ x, int64_t N, int n, const uint32_t* __restrict__ perm,
                         const double2* __restrict__ stats, const uint8_t* __restrict__ words_in,
                         float* __restrict__ Z, uint8_t* __restrict__ words_out) {
  int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (p >= N) return;
  uint32_t o = perm[p];
  double2 st = stats[o];
  const float* src = x + (int64_t)o * n;
  float* dst = Z + p * n;
  for (int t = lane; t < n; t += 32) dst[t] = znorm_value(src[t], st.x, st.y);
  if (lane < LW / 16)
    reinterpret_cast<uint4*>(words_out + p * LW)[lane] =
        reinterpret_cast<const uint4*>(words_in + (int64_t)o * LW)[lane];
}

// Int8 copy of every key-sorted canonical series for the refinement filter:
// scale s = max|z| / 127 (1 for the zero series), v_t = rint(z_t / s) in
// [-127, 127] (any integer code is valid: the residual is of the codes
// chosen), and an upper bound e of the residual norm ||z - s v||.  Each
// residual d_t = fma(-s, v_t, z_t) is rounded once (|d~ - d| <= u |d|, u =
// 2^-24), and the FP32 sum of the m = ceil(n / 32) + 5 terms a lane and the
// warp's tree add has relative error <= (m + 1) u (non-negative terms), so
// ||z - s v||^2 <= e~^2 (1 + u)^2 (1 + (m + 1) u)^... <= e~^2 (1 + (m + 4) 2^-23):
// e = sqrt_ru(e~^2 (1 + (m + 4) 2^-23)) with a 1e-6 relative cushion.  Warp
// per series.
__global__ void k_quant8(const float* __restrict__ Z, int64_t N, int n, int8_t* __restrict__ Z8,
                         float* __restrict__ scale, float* __restrict__ err) {
  const int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (p >= N) return;
  const float* z = Z + p * n;
  float mx = 0.f;
  for (int t = lane; t < n; t += 32) mx = fmaxf(mx, fabsf(z[t]));
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
  const float sc = mx > 0.f ? mx / 127.0f : 1.0f;
  const float inv = 1.0f / sc;
  float e2 = 0.f;
  for (int t = lane; t < n; t += 32) {
    float v = rintf(z[t] * inv);
    v = fminf(fmaxf(v, -127.f), 127.f);
    Z8[p * n + t] = (int8_t)v;
    const float d = fmaf(-sc, v, z[t]);
    e2 = fmaf(d, d, e2);
  }
  for (int o = 16; o > 0; o >>= 1) e2 += __shfl_xor_sync(0xFFFFFFFFu, e2, o);
  if (lane == 0) {
    scale[p] = sc;
    const float m = (float)((n + 31) / 32 + 5);
    const float cush = __fadd_ru(1.0f, __fmul_ru(m + 4.0f, 0x1p-23f));
    err[p] = __fadd_ru(__fmul_ru(__fsqrt_ru(__fmul_ru(e2, cush)), 1.000001f), 1e-30f);
  }
}

// Eq. (1) weight of each projection column: 2 for a value of coefficient
// 0 < k < n/2 (it stands for itself and its conjugate), 1 for the Nyquist
// value, 0 for an unused column.  Columns [0, LW) hold the word values
// (0..l-1), columns [LW, NB) the remaining selected values (l..nsel-1).
__global__ void k_vweights(int n, int NB, int LW, int l, int nsel, const int32_t* __restrict__ sel_k,
                           float* __restrict__ vw) {
  const int col = threadIdx.x;
  if (col >= NB) return;
  const int j = col < LW ? (col < l ? col : -1) : (l + col - LW < nsel ? l + col - LW : -1);
  vw[col] = j < 0 ? 0.f : (2 * sel_k[j] == n ? 1.f : 2.f);
}

// Value codes for the refinement's first filter.  Each canonical series'
// NB selected Fourier values v~ (the FP32 projection of the word kernel, so
// |v~ - v| <= delta_d per value) become int8 codes c with one scale s per
// series; y = s c is an exact real vector.  The stored margin is
//   r = ||v~ - y||_w (FP64, rounded up) + sqrt(W) (delta_d + delta_q),
// W = sum of the weights, so that for the exact values v of the series and q
// of a query (computed as q~):  ||q - v||_w >= ||q~ - y||_w - r  by the
// triangle inequality in the weighted norm, and Eq. (1) restricted to the
// selected values gives ||q - v||_w <= ED.  A CTA of WTHREADS threads takes
// ROWS rows (staged by all threads); thread (r, g) projects row r on columns
// g*CPT..+CPT in ascending t (one FMA per t and column), the row's maximum
// and squared residual are reduced over its GPR threads.
template <int NBT>
__global__ void __launch_bounds__(WTHREADS) k_quantv(const float* __restrict__ Z, int64_t N, int n,
                                                     const float* __restrict__ basis, const float* __restrict__ vw,
                                                     float dmargin, int8_t* __restrict__ vc,
                                                     float2* __restrict__ vsr) {
  constexpr int GPR = WTHREADS / ROWS;  // 8 threads per row
  constexpr int CPT = NBT / GPR;        // 4 or 8 columns per thread
  extern __shared__ float sm[];
  const int64_t first = (int64_t)blockIdx.x * ROWS;
  const int nr = (int)(N - first < ROWS ? N - first : ROWS);
  stage_rows_vec(Z, first, N, n, sm);
  const int tid = threadIdx.x, r = tid / GPR, g = tid - r * GPR;
  const bool active = r < nr;
  float acc[CPT];
#pragma unroll
  for (int c = 0; c < CPT; ++c) acc[c] = 0.f;
  if (active) {
    const float* my = sm + r * (n + 1);
    const float* bcol = basis + g * CPT;
    for (int t = 0; t < n; ++t) {
      const float zt = my[t];
#pragma unroll
      for (int c = 0; c < CPT; ++c) acc[c] = fmaf(zt, __ldg(bcol + (int64_t)t * NBT + c), acc[c]);
    }
  }
  float mx = 0.f;
#pragma unroll
  for (int c = 0; c < CPT; ++c) mx = fmaxf(mx, fabsf(acc[c]));
  // the GPR threads of a row are consecutive lanes of one warp
#pragma unroll
  for (int o = 1; o < GPR; o <<= 1) mx = fmaxf(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
  const float sc = mx > 0.f ? mx / 127.0f : 1.0f;
  double e2 = 0.0;
  uint32_t packed[CPT / 4];
#pragma unroll
  for (int c4 = 0; c4 < CPT / 4; ++c4) {
    uint32_t w = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int c = 4 * c4 + b, j = g * CPT + c;
      const float code = fminf(fmaxf(rintf(acc[c] / sc), -127.f), 127.f);
      const double d = (double)acc[c] - (double)sc * (double)code;
      e2 += (double)__ldg(vw + j) * d * d;
      w |= ((uint32_t)(int)code & 0xFFu) << (8 * b);
    }
    packed[c4] = w;
  }
#pragma unroll
  for (int o = 1; o < GPR; o <<= 1) e2 += __shfl_xor_sync(0xFFFFFFFFu, e2, o);
  if (!active) return;
  const int64_t row = first + r;
  uint32_t* o4 = reinterpret_cast<uint32_t*>(vc + row * NBT + g * CPT);
#pragma unroll
  for (int c4 = 0; c4 < CPT / 4; ++c4) o4[c4] = packed[c4];
  if (g == 0) vsr[row] = make_float2(sc, __double2float_ru(sqrt(e2) * (1.0 + 1e-6) + (double)dmargin + 1e-30));
}

// FP16 copy (round to nearest) of count fp32 values, 4 per thread.
__global__ void k_to_half(const float* __restrict__ src, int64_t count, __half* __restrict__ dst) {
  const int64_t i0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
  for (int64_t i = i0; i < i0 + 4 && i < count; ++i) dst[i] = __float2half_rn(src[i]);
}

// Symbol envelope (per word value min and max symbol) of each tile of 256
// consecutive key-sorted series, using byte-wise SIMD min / max.
template <int LW>
__global__ void __launch_bounds__(TILE) k_tile_env(const uint8_t* __restrict__ words, int64_t N,
                                                   uint8_t* __restrict__ tenv) {
  constexpr int NW = LW / 4;
  __shared__ uint32_t slo[8][NW], shi[8][NW];
  const int64_t p = (int64_t)blockIdx.x * TILE + threadIdx.x;
  uint32_t lo[NW], hi[NW];
  const uint32_t* w = reinterpret_cast<const uint32_t*>(words + p * LW);
#pragma unroll
  for (int q = 0; q < NW; ++q) {
    uint32_t v = p < N ? w[q] : 0u;
    lo[q] = p < N ? v : 0xFFFFFFFFu;
    hi[q] = v;
  }
#pragma unroll
  for (int q = 0; q < NW; ++q)
    for (int o = 16; o > 0; o >>= 1) {
      lo[q] = __vminu4(lo[q], __shfl_xor_sync(0xFFFFFFFFu, lo[q], o));
      hi[q] = __vmaxu4(hi[q], __shfl_xor_sync(0xFFFFFFFFu, hi[q], o));
    }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < NW; ++q) {
      slo[warp][q] = lo[q];
      shi[warp][q] = hi[q];
    }
  __syncthreads();
  if (threadIdx.x < NW) {
    uint32_t a = 0xFFFFFFFFu, b = 0u;
    for (int i = 0; i < 8; ++i) {
      a = __vminu4(a, slo[i][threadIdx.x]);
      b = __vmaxu4(b, shi[i][threadIdx.x]);
    }
    uint32_t* out = reinterpret_cast<uint32_t*>(tenv + (int64_t)blockIdx.x * 2 * LW);
    out[threadIdx.x] = a;
    out[NW + threadIdx.x] = b;
  }
}

// Leaf-block envelope = byte-wise min / max over its tiles.
__global__ void k_leaf_env(const uint8_t* __restrict__ tenv, int64_t T, int LW, int leaf_tiles, int64_t L,
                           uint8_t* __restrict__ lenv) {
  const int NW = LW / 4;
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= L * NW) return;
  int64_t b = e / NW;
  int q = (int)(e % NW);
  uint32_t a = 0xFFFFFFFFu, h = 0u;
  for (int64_t t = b * leaf_tiles; t < ((b + 1) * leaf_tiles < T ? (b + 1) * leaf_tiles : T); ++t) {
    const uint32_t* te = reinterpret_cast<const uint32_t*>(tenv + t * 2 * LW);
    a = __vminu4(a, te[q]);
    h = __vmaxu4(h, te[NW + q]);
  }
  uint32_t* out = reinterpret_cast<uint32_t*>(lenv + b * 2 * LW);
  out[q] = a;
  out[NW + q] = h;
}

__global__ void k_iota(uint32_t* v, int64_t N) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) v[i] = (uint32_t)i;
}

// ========================================================================
// Host orchestration of sofa_build (Sec. IV "SOFA index" workflow).
// ========================================================================
template <class T>
static int dalloc(T** p, int64_t count, int64_t* acct) {
  *p = nullptr;
  if (count <= 0) count = 1;
  cudaError_t e = dev_malloc((void**)p, (size_t)count * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(SOFA_ERR_OOM, std::string("cudaMalloc of ") + std::to_string(count * sizeof(T)) +
                                  " bytes failed: " + cudaGetErrorString(e));
  }
  if (acct) *acct += count * (int64_t)sizeof(T);
  return 0;
}

struct Tmp {  // frees every temporary on scope exit
  std::vector<void*> ptrs;
  ~Tmp() {
    for (void* p : ptrs) cudaFree(p);
  }
  template <class T>
  int get(T** p, int64_t count) {
    int rc = dalloc(p, count, nullptr);
    if (!rc) ptrs.push_back(*p);
    return rc;
  }
};

#define TRY(x)           \
  do {                   \
    int rc_ = (x);       \
    if (rc_) return rc_; \
  } while (0)

int launch_znorm(const float* x, int64_t R, int n, float* z, cudaStream_t st) {
  if (R <= 0) return 0;
  size_t smem = (size_t)ROWS * (n + 1) * sizeof(float);
  SOFA_CUDA(cudaFuncSetAttribute(k_rows_project<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_rows_project<true><<<(unsigned)ceil_div(R, ROWS), WTHREADS, smem, st>>>(x, R, n, 1, nullptr, 0, 0, z, nullptr, 0,
                                                                         nullptr);
  SOFA_CUDA(cudaGetLastError());
  return 0;
}

int launch_qprep(Index* ix, const float* q, int64_t Q, float* zq, float* qv, cudaStream_t st) {
  if (Q <= 0) return 0;
  // rows per CTA: the largest power of two <= 32 that still gives two CTAs
  // per SM (the FP64 chain of a row is the floor; more CTAs spread the rest)
  int dev = 0, sms = 0;
  SOFA_CUDA(cudaGetDevice(&dev));
  SOFA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int64_t per = Q / (2 * (int64_t)(sms > 0 ? sms : 1));
  if (per >= 32) return launch_qprep_rq<32>(ix, q, Q, zq, qv, st);
  if (per >= 16) return launch_qprep_rq<16>(ix, q, Q, zq, qv, st);
  if (per >= 8) return launch_qprep_rq<8>(ix, q, Q, zq, qv, st);
  if (per >= 4) return launch_qprep_rq<4>(ix, q, Q, zq, qv, st);
  if (per >= 2) return launch_qprep_rq<2>(ix, q, Q, zq, qv, st);
  return launch_qprep_rq<1>(ix, q, Q, zq, qv, st);
}

int build_index(Index* ix, const float* x, const sofa_build_opts& o, cudaStream_t st) {
  const int64_t N = ix->N;
  const int n = ix->n, l = ix->l, alpha = ix->alpha, LW = ix->LW, NB = ix->NB;
  Tmp tmp;
  int64_t* acct = &ix->device_bytes;
  const float ratio = o.sample_ratio > 0 ? o.sample_ratio : 0.1f;
  const int stride = (int)std::max(1.0, std::ceil(1.0 / (double)ratio - 1e-9));
  const int64_t S = ceil_div(N, stride);
  const int ncand = num_candidates(n, o.pool_coeffs);
  const size_t row_smem = (size_t)ROWS * (n + 1) * sizeof(float);
  SOFA_CUDA(cudaFuncSetAttribute(k_rows_project<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)row_smem));
  SOFA_CUDA(cudaFuncSetAttribute(k_rows_project<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)row_smem));

  // ---- Alg. 1 step 1: sample, z-normalise, DFT variance of every candidate value
  float* Zs;
  TRY(tmp.get(&Zs, S * n));
  k_rows_project<true><<<(unsigned)ceil_div(S, ROWS), WTHREADS, row_smem, st>>>(x, S, n, stride, nullptr, 0, 0, Zs,
                                                                             nullptr, 0, nullptr);
  SOFA_CUDA(cudaGetLastError());
  float* Bf;
  TRY(tmp.get(&Bf, (int64_t)n * ncand));
  k_basis_full<<<(unsigned)ceil_div((int64_t)n * ncand, 256), 256, 0, st>>>(n, ncand, Bf);
  const int nparts = (int)std::min<int64_t>(ceil_div(S, GM), 608);
  double2* partial;
  TRY(tmp.get(&partial, (int64_t)nparts * ncand));
  dim3 g(nparts, (unsigned)ceil_div(ncand, GN));
  k_dft_var<<<g, 256, 0, st>>>(Zs, S, n, Bf, ncand, partial);
  double* var_all;
  TRY(tmp.get(&var_all, ncand));
  k_var_reduce<<<(unsigned)ceil_div(ncand, 128), 128, 0, st>>>(partial, nparts, ncand, S, var_all);
  SOFA_CUDA(cudaGetLastError());

  // ---- Alg. 1 step 2: selection
  const int m = o.user_sel ? o.user_nsel : std::min(2 * l, ncand);
  ix->nsel = m;
  TRY(dalloc(&ix->sel, m, acct));
  TRY(dalloc(&ix->sel_k, m, acct));
  TRY(dalloc(&ix->sel_part, m, acct));
  TRY(dalloc(&ix->var, m, acct));
  int32_t* d_nyq;
  TRY(tmp.get(&d_nyq, 1));
  if (o.user_sel) {
    SOFA_CUDA(cudaMemcpyAsync(ix->sel, o.user_sel, m * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    k_user_sel<<<1, 32, 0, st>>>(ix->sel, m, n, var_all, ix->sel_k, ix->sel_part, ix->var, d_nyq, l);
  } else {
    k_select<<<1, 256, 0, st>>>(var_all, ncand, n, l, o.select, ix->sel, ix->sel_k, ix->sel_part, ix->var, d_nyq);
  }
  SOFA_CUDA(cudaGetLastError());
  int32_t h_nyq = 0;
  SOFA_CUDA(cudaMemcpyAsync(&h_nyq, d_nyq, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  SOFA_CUDA(cudaStreamSynchronize(st));
  ix->nyq_first = h_nyq;

  // ---- projection basis [n][NB]
  TRY(dalloc(&ix->basis, (int64_t)n * NB, acct));
  k_basis_sel<<<(unsigned)ceil_div((int64_t)n * NB, 256), 256, 0, st>>>(n, NB, LW, l, m, ix->sel_k, ix->sel_part,
                                                                         ix->basis);
  SOFA_CUDA(cudaGetLastError());

  // ---- Alg. 1 step 3: bins from the sample's word values
  TRY(dalloc(&ix->beta, (int64_t)LW * (alpha + 1), acct));
  SOFA_CUDA(cudaMemsetAsync(ix->beta, 0, (size_t)LW * (alpha + 1) * sizeof(float), st));
  if (o.user_beta) {
    SOFA_CUDA(cudaMemcpyAsync(ix->beta, o.user_beta, (size_t)l * (alpha + 1) * sizeof(float),
                              cudaMemcpyHostToDevice, st));
  } else {
    float *vals, *sorted;
    TRY(tmp.get(&vals, S * l));
    TRY(tmp.get(&sorted, S * l));
    k_rows_project<false><<<(unsigned)ceil_div(S, ROWS), WTHREADS, row_smem, st>>>(Zs, S, n, 1, ix->basis, NB, l,
                                                                                nullptr, vals, 1, nullptr);
    SOFA_CUDA(cudaGetLastError());
    size_t tb = 0;
    SOFA_CUDA(cub::DeviceRadixSort::SortKeys(nullptr, tb, vals, sorted, (int)S, 0, 32, st));
    void* tstore;
    TRY(tmp.get((char**)&tstore, (int64_t)tb));
    for (int j = 0; j < l; ++j)
      SOFA_CUDA(cub::DeviceRadixSort::SortKeys(tstore, tb, vals + (int64_t)j * S, sorted + (int64_t)j * S, (int)S,
                                               0, 32, st));
    k_bins<<<l, 256, 0, st>>>(sorted, S, l, alpha, o.binning, ix->beta);
    SOFA_CUDA(cudaGetLastError());
  }

  // ---- margins and bound tables
  const double u = std::ldexp(1.0, -24);
  ix->vmax = std::sqrt((double)n) * (1.0 + 1e-4);
  ix->delta_d = (double)(n + 2) * u * std::sqrt((double)n) * 1.02;
  ix->delta_q = ix->delta_d;
  const float delta = (float)((ix->delta_d + ix->delta_q) * 1.0001);
  const float outer = (float)(ix->vmax + ix->delta_d + ix->delta_q);
  const float eps_abs = (float)(4.0 * u * (outer + 1.0));
  TRY(dalloc(&ix->edge, (int64_t)LW * MAX_ALPHA, acct));
  TRY(dalloc(&ix->ch, (int64_t)LW * MAX_ALPHA, acct));
  TRY(dalloc(&ix->ch16, (int64_t)LW * MAX_ALPHA, acct));
  k_tables<<<(unsigned)ceil_div(LW * MAX_ALPHA, 256), 256, 0, st>>>(ix->beta, l, LW, alpha, delta, outer, eps_abs,
                                                                     ix->edge, ix->ch, ix->ch16);
  ix->outer = outer;
  SOFA_CUDA(cudaGetLastError());

  // ---- key bit order
  int32_t* d_nbits;
  TRY(dalloc(&ix->keyorder, 64, acct));
  uint8_t* keyorder = ix->keyorder;
  TRY(tmp.get(&d_nbits, 1));
  k_keyorder<<<1, 32, 0, st>>>(ix->var, l, ix->bps, keyorder, d_nbits);
  int32_t keybits = 0;
  SOFA_CUDA(cudaMemcpyAsync(&keybits, d_nbits, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  SOFA_CUDA(cudaStreamSynchronize(st));
  ix->keybits = keybits;
  // the sample is no longer needed: release it before the full pass
  cudaFree(Zs);
  tmp.ptrs.erase(std::find(tmp.ptrs.begin(), tmp.ptrs.end(), (void*)Zs));

  // ---- Alg. 2 over every series: words and layout keys
  uint8_t* words0;
  uint64_t* keys0;
  uint32_t* ids0;
  double2* stats;
  TRY(tmp.get(&words0, N * LW));
  TRY(tmp.get(&keys0, N));
  TRY(dalloc(&ix->keys, N, acct));
  uint64_t* keys1 = ix->keys;
  TRY(tmp.get(&ids0, N));
  TRY(tmp.get(&stats, N));
  const size_t wsmem = row_smem + (size_t)LW * (alpha + 1) * sizeof(float) + (size_t)ROWS * LW;
  if (LW == 16) {
    SOFA_CUDA(cudaFuncSetAttribute(k_words<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wsmem));
    k_words<16><<<(unsigned)ceil_div(N, ROWS), WTHREADS, wsmem, st>>>(x, N, n, ix->basis, NB, ix->beta, alpha, l,
                                                                       keyorder, keybits, words0, keys0, ids0, stats);
  } else {
    SOFA_CUDA(cudaFuncSetAttribute(k_words<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wsmem));
    k_words<32><<<(unsigned)ceil_div(N, ROWS), WTHREADS, wsmem, st>>>(x, N, n, ix->basis, NB, ix->beta, alpha, l,
                                                                       keyorder, keybits, words0, keys0, ids0, stats);
  }
  SOFA_CUDA(cudaGetLastError());

  // ---- key sort -> permutation
  TRY(dalloc(&ix->perm, N, acct));
  {
    size_t tb = 0;
    int end_bit = 64, begin_bit = 64 - std::min(64, (int)keybits);
    SOFA_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, tb, keys0, keys1, ids0, ix->perm, N, begin_bit, end_bit, st));
    char* tstore;
    TRY(tmp.get(&tstore, (int64_t)tb));
    SOFA_CUDA(cub::DeviceRadixSort::SortPairs(tstore, tb, keys0, keys1, ids0, ix->perm, N, begin_bit, end_bit, st));
  }

  // ---- layout: canonical series and words in key order
  TRY(dalloc(&ix->Z, N * n, acct));
  TRY(dalloc(&ix->words, N * LW, acct));
  {
    int64_t threads = N * 32;
    unsigned blocks = (unsigned)ceil_div(threads, 256);
    if (LW == 16)
      k_layout<16><<<blocks, 256, 0, st>>>(x, N, n, ix->perm, stats, words0, ix->Z, ix->words);
    else
      k_layout<32><<<blocks, 256, 0, st>>>(x, N, n, ix->perm, stats, words0, ix->Z, ix->words);
    SOFA_CUDA(cudaGetLastError());
  }

  // ---- int8 copy for the refinement filter (optional)
  if (o.precision >= 1) {
    TRY(dalloc(&ix->Z8, N * n, acct));
    TRY(dalloc(&ix->s8, N, acct));
    TRY(dalloc(&ix->e8, N, acct));
    k_quant8<<<(unsigned)ceil_div(N * 32, 256), 256, 0, st>>>(ix->Z, N, n, ix->Z8, ix->s8, ix->e8);
    SOFA_CUDA(cudaGetLastError());
    // value codes (the refinement's first filter), in key order
    TRY(dalloc(&ix->VC, N * NB, acct));
    TRY(dalloc(&ix->vsr, N, acct));
    TRY(dalloc(&ix->vw, NB, acct));
    k_vweights<<<1, NB_MAX, 0, st>>>(n, NB, LW, l, ix->nsel, ix->sel_k, ix->vw);
    SOFA_CUDA(cudaGetLastError());
    // sqrt(W) (delta_d + delta_q) with W <= 2 nsel, rounded up
    const float dmargin = std::nextafter(
        (float)(std::sqrt(2.0 * ix->nsel) * (ix->delta_d + ix->delta_q) * 1.0001), INFINITY);
    const size_t vsmem = (size_t)ROWS * (n + 1) * sizeof(float);
    if (NB == 32) {
      SOFA_CUDA(cudaFuncSetAttribute(k_quantv<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vsmem));
      k_quantv<32><<<(unsigned)ceil_div(N, ROWS), WTHREADS, vsmem, st>>>(ix->Z, N, n, ix->basis, ix->vw, dmargin,
                                                                     ix->VC, ix->vsr);
    } else {
      SOFA_CUDA(cudaFuncSetAttribute(k_quantv<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vsmem));
      k_quantv<64><<<(unsigned)ceil_div(N, ROWS), WTHREADS, vsmem, st>>>(ix->Z, N, n, ix->basis, ix->vw, dmargin,
                                                                     ix->VC, ix->vsr);
    }
    SOFA_CUDA(cudaGetLastError());
  }

  // ---- FP16 copy of the canonical series (dense path with FP16 operands);
  // its rows are TMA-addressed, so their stride must be a multiple of 16 bytes
  if (o.precision == 2 && n % 8 == 0) {
    TRY(dalloc(&ix->Zh, N * n, acct));
    k_to_half<<<(unsigned)ceil_div(N * n, 1024), 256, 0, st>>>(ix->Z, N * n, ix->Zh);
    SOFA_CUDA(cudaGetLastError());
  }

  // ---- squared norms of the canonical series (dense path)
  TRY(dalloc(&ix->xn, N, acct));
  TRY(launch_row_norms(ix->Z, N, n, ix->xn, st));

  // ---- envelopes
  ix->T = ceil_div(N, TILE);
  ix->L = ceil_div(ix->T, ix->leaf_tiles);
  TRY(dalloc(&ix->tenv, ix->T * 2 * LW, acct));
  TRY(dalloc(&ix->lenv, ix->L * 2 * LW, acct));
  if (LW == 16)
    k_tile_env<16><<<(unsigned)ix->T, TILE, 0, st>>>(ix->words, N, ix->tenv);
  else
    k_tile_env<32><<<(unsigned)ix->T, TILE, 0, st>>>(ix->words, N, ix->tenv);
  k_leaf_env<<<(unsigned)ceil_div(ix->L * (LW / 4), 256), 256, 0, st>>>(ix->tenv, ix->T, LW, ix->leaf_tiles, ix->L,
                                                                         ix->lenv);
  SOFA_CUDA(cudaGetLastError());
  // FP16 value codes and constants of the tensor-core series bound
  TRY(make_tc_codes(ix, st));
  SOFA_CUDA(cudaStreamSynchronize(st));
  ix->Ns = N;
  return 0;
}

// ========================================================================
// Incremental insert (Sec. IV "Structure": the index takes new series; the
// paper's tree inserts each into the leaf of its word and splits full
// leaves).  Here the new series are summarised with the index's learned
// summary (Alg. 2, no relearning of selection or bins), then merged by layout
// key into the appended region [Ns, N): a second key-sorted run after the
// build's.  Both runs are cut into tiles and leaf blocks like the build's
// layout, so the scan, the routing and the refinement cover every row
// unchanged, and the seed searches each run by key.
// ========================================================================

// Rows j = 0..R-1 of dst (row_bytes each): row src_idx[j] of the sequence
// "rows [0, n_old) of old, then rows of fresh".  Warp per row, 4-byte words
// when the row size allows.
__global__ void k_gather_rows2(const uint8_t* __restrict__ old, int64_t n_old, const uint8_t* __restrict__ fresh,
                               const uint32_t* __restrict__ src_idx, int64_t R, int row_bytes,
                               uint8_t* __restrict__ dst) {
  const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (j >= R) return;
  const int64_t s = src_idx[j];
  const uint8_t* src = s < n_old ? old + s * row_bytes : fresh + (s - n_old) * row_bytes;
  uint8_t* d = dst + j * row_bytes;
  if ((row_bytes & 3) == 0) {
    const uint32_t* s4 = reinterpret_cast<const uint32_t*>(src);
    uint32_t* d4 = reinterpret_cast<uint32_t*>(d);
    for (int i = lane; i < row_bytes / 4; i += 32) d4[i] = s4[i];
  } else {
    for (int i = lane; i < row_bytes; i += 32) d[i] = src[i];
  }
}

// Original row ids of an inserted batch: base + batch row.
__global__ void k_ids_from(uint32_t* __restrict__ ids, int64_t A, int64_t base) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < A) ids[i] = (uint32_t)(base + i);
}

// One per-row array of the index and its grown replacement: rows [0, Ns)
// copied, rows [Ns, N_old + A) gathered by src_idx from the old appended
// region (indices < N_old - Ns) and the batch rows `fresh`.
struct Grow {
  void** arr;
  int row_bytes;
  const void* fresh;
  uint8_t* nw;
};

static void launch_grow(const Grow& g, int64_t N_old, int64_t Ns, int64_t A, const uint32_t* src_idx,
                        cudaStream_t st) {
  const uint8_t* od = static_cast<const uint8_t*>(*g.arr);
  const int64_t rb = g.row_bytes;
  if (Ns > 0) cudaMemcpyAsync(g.nw, od, (size_t)(Ns * rb), cudaMemcpyDeviceToDevice, st);
  const int64_t R = N_old - Ns + A;
  k_gather_rows2<<<(unsigned)ceil_div(R * 32, 256), 256, 0, st>>>(od + Ns * rb, N_old - Ns,
                                                                   static_cast<const uint8_t*>(g.fresh), src_idx, R,
                                                                   g.row_bytes, g.nw + Ns * rb);
}

int insert_rows(Index* ix, const float* x, int64_t A, cudaStream_t st) {
  const int64_t N_old = ix->N, Ns = ix->Ns, R_old = N_old - Ns, N_new = N_old + A;
  const int n = ix->n, l = ix->l, alpha = ix->alpha, LW = ix->LW, NB = ix->NB;
  Tmp tmp;
  int64_t* acct = &ix->device_bytes;
  const size_t row_smem = (size_t)ROWS * (n + 1) * sizeof(float);

  // ---- Alg. 2 on the batch with the index's summary: words, keys, statistics
  uint8_t* words_b;
  uint64_t* keys_b;
  uint32_t* rows_b;
  double2* stats;
  TRY(tmp.get(&words_b, A * LW));
  TRY(tmp.get(&keys_b, A));
  TRY(tmp.get(&rows_b, A));
  TRY(tmp.get(&stats, A));
  const size_t wsmem = row_smem + (size_t)LW * (alpha + 1) * sizeof(float) + (size_t)ROWS * LW;
  if (LW == 16) {
    SOFA_CUDA(cudaFuncSetAttribute(k_words<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wsmem));
    k_words<16><<<(unsigned)ceil_div(A, ROWS), WTHREADS, wsmem, st>>>(x, A, n, ix->basis, NB, ix->beta, alpha, l,
                                                                   ix->keyorder, ix->keybits, words_b, keys_b,
                                                                   rows_b, stats);
  } else {
    SOFA_CUDA(cudaFuncSetAttribute(k_words<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wsmem));
    k_words<32><<<(unsigned)ceil_div(A, ROWS), WTHREADS, wsmem, st>>>(x, A, n, ix->basis, NB, ix->beta, alpha, l,
                                                                   ix->keyorder, ix->keybits, words_b, keys_b,
                                                                   rows_b, stats);
  }
  SOFA_CUDA(cudaGetLastError());

  // ---- the batch's per-row arrays in batch order (rows_b is the identity)
  float* Zb;
  uint8_t* Wb;
  TRY(tmp.get(&Zb, A * n));
  TRY(tmp.get(&Wb, A * LW));
  if (LW == 16)
    k_layout<16><<<(unsigned)ceil_div(A * 32, 256), 256, 0, st>>>(x, A, n, rows_b, stats, words_b, Zb, Wb);
  else
    k_layout<32><<<(unsigned)ceil_div(A * 32, 256), 256, 0, st>>>(x, A, n, rows_b, stats, words_b, Zb, Wb);
  SOFA_CUDA(cudaGetLastError());
  int8_t *Z8b = nullptr, *VCb = nullptr;
  float *s8b = nullptr, *e8b = nullptr, *xnb = nullptr;
  float2* vsrb = nullptr;
  __half* Zhb = nullptr;
  if (ix->Z8) {
    TRY(tmp.get(&Z8b, A * n));
    TRY(tmp.get(&s8b, A));
    TRY(tmp.get(&e8b, A));
    k_quant8<<<(unsigned)ceil_div(A * 32, 256), 256, 0, st>>>(Zb, A, n, Z8b, s8b, e8b);
    SOFA_CUDA(cudaGetLastError());
  }
  if (ix->VC) {
    TRY(tmp.get(&VCb, A * NB));
    TRY(tmp.get(&vsrb, A));
    const float dmargin = std::nextafter(
        (float)(std::sqrt(2.0 * ix->nsel) * (ix->delta_d + ix->delta_q) * 1.0001), INFINITY);
    if (NB == 32) {
      SOFA_CUDA(cudaFuncSetAttribute(k_quantv<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)row_smem));
      k_quantv<32><<<(unsigned)ceil_div(A, ROWS), WTHREADS, row_smem, st>>>(Zb, A, n, ix->basis, ix->vw, dmargin, VCb,
                                                                        vsrb);
    } else {
      SOFA_CUDA(cudaFuncSetAttribute(k_quantv<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)row_smem));
      k_quantv<64><<<(unsigned)ceil_div(A, ROWS), WTHREADS, row_smem, st>>>(Zb, A, n, ix->basis, ix->vw, dmargin, VCb,
                                                                        vsrb);
    }
    SOFA_CUDA(cudaGetLastError());
  }
  if (ix->Zh) {
    TRY(tmp.get(&Zhb, A * n));
    k_to_half<<<(unsigned)ceil_div(A * n, 1024), 256, 0, st>>>(Zb, A * n, Zhb);
    SOFA_CUDA(cudaGetLastError());
  }
  TRY(tmp.get(&xnb, A));
  TRY(launch_row_norms(Zb, A, n, xnb, st));
  uint32_t* idb;
  TRY(tmp.get(&idb, A));
  k_ids_from<<<(unsigned)ceil_div(A, 256), 256, 0, st>>>(idb, A, N_old);
  SOFA_CUDA(cudaGetLastError());

  // ---- merge the appended region's keys with the batch's: one key sort of
  // both, carrying each row's source index (region rows first, then batch)
  const int64_t R = R_old + A;
  uint64_t *kin, *kout;
  uint32_t *vin, *vout;
  TRY(tmp.get(&kin, R));
  TRY(tmp.get(&kout, R));
  TRY(tmp.get(&vin, R));
  TRY(tmp.get(&vout, R));
  if (R_old > 0)
    SOFA_CUDA(cudaMemcpyAsync(kin, ix->keys + Ns, (size_t)R_old * sizeof(uint64_t), cudaMemcpyDeviceToDevice, st));
  SOFA_CUDA(cudaMemcpyAsync(kin + R_old, keys_b, (size_t)A * sizeof(uint64_t), cudaMemcpyDeviceToDevice, st));
  k_iota<<<(unsigned)ceil_div(R, 256), 256, 0, st>>>(vin, R);
  SOFA_CUDA(cudaGetLastError());
  {
    size_t tb = 0;
    const int begin_bit = 64 - std::min(64, ix->keybits);
    SOFA_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, tb, kin, kout, vin, vout, R, begin_bit, 64, st));
    char* tstore;
    TRY(tmp.get(&tstore, (int64_t)tb));
    SOFA_CUDA(cub::DeviceRadixSort::SortPairs(tstore, tb, kin, kout, vin, vout, R, begin_bit, 64, st));
  }

  // ---- every per-row array grows by A rows, its region merged in key order.
  // All grown arrays (and the new envelopes) are allocated before any is
  // written, and the old ones are freed only once every copy is done: an
  // allocation failure leaves the index as it was.
  std::vector<Grow> grows = {{(void**)&ix->Z, n * (int)sizeof(float), Zb, nullptr},
                             {(void**)&ix->words, LW, Wb, nullptr},
                             {(void**)&ix->perm, (int)sizeof(uint32_t), idb, nullptr},
                             {(void**)&ix->keys, (int)sizeof(uint64_t), keys_b, nullptr},
                             {(void**)&ix->xn, (int)sizeof(float), xnb, nullptr}};
  if (ix->Z8) {
    grows.push_back({(void**)&ix->Z8, n, Z8b, nullptr});
    grows.push_back({(void**)&ix->s8, (int)sizeof(float), s8b, nullptr});
    grows.push_back({(void**)&ix->e8, (int)sizeof(float), e8b, nullptr});
  }
  if (ix->VC) {
    grows.push_back({(void**)&ix->VC, NB, VCb, nullptr});
    grows.push_back({(void**)&ix->vsr, (int)sizeof(float2), vsrb, nullptr});
  }
  if (ix->Zh) grows.push_back({(void**)&ix->Zh, n * (int)sizeof(__half), Zhb, nullptr});
  const int64_t T = ceil_div(N_new, TILE), L = ceil_div(T, ix->leaf_tiles);
  uint8_t *tenv = nullptr, *lenv = nullptr;
  auto release_new = [&]() {
    for (Grow& g : grows)
      if (g.nw) cudaFree(g.nw);
    if (tenv) cudaFree(tenv);
    if (lenv) cudaFree(lenv);
  };
  int rc = 0;
  for (Grow& g : grows) {
    rc = dalloc(&g.nw, N_new * (int64_t)g.row_bytes, nullptr);
    if (rc) break;
  }
  if (!rc) rc = dalloc(&tenv, T * 2 * LW, nullptr);
  if (!rc) rc = dalloc(&lenv, L * 2 * LW, nullptr);
  if (rc) {
    release_new();
    return fail(SOFA_ERR_OOM, "sofa_insert: no room on the device for the grown index (the old and the grown "
                              "arrays are held together while the rows are merged); the index is unchanged");
  }
  for (const Grow& g : grows) launch_grow(g, N_old, Ns, A, vout, st);
  uint8_t* words_new = nullptr;
  for (const Grow& g : grows)
    if (g.arr == (void**)&ix->words) words_new = g.nw;
  if (LW == 16)
    k_tile_env<16><<<(unsigned)T, TILE, 0, st>>>(words_new, N_new, tenv);
  else
    k_tile_env<32><<<(unsigned)T, TILE, 0, st>>>(words_new, N_new, tenv);
  k_leaf_env<<<(unsigned)ceil_div(L * (LW / 4), 256), 256, 0, st>>>(tenv, T, LW, ix->leaf_tiles, L, lenv);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    release_new();
    return fail(SOFA_ERR_CUDA, std::string("sofa_insert: ") + cudaGetErrorString(e));
  }
  // commit: the grown arrays replace the old ones
  for (Grow& g : grows) {
    cudaFree(*g.arr);
    *g.arr = g.nw;
    g.nw = nullptr;
    *acct += A * (int64_t)g.row_bytes;
  }
  cudaFree(ix->tenv);
  cudaFree(ix->lenv);
  *acct += (T - ix->T) * 2 * LW + (L - ix->L) * 2 * LW;
  ix->tenv = tenv;
  ix->lenv = lenv;
  ix->N = N_new;
  ix->T = T;
  ix->L = L;
  ++g_buf_generation;  // recorded query graphs hold the old array addresses
  // the tensor-core codes of the grown layout (derived from the value codes;
  // if they cannot be allocated the index stays usable with the word bound)
  if (ix->VC && make_tc_codes(ix, st) != 0) {
    release_tc_codes(ix);
    if (ix->series_bound == 1) ix->series_bound = 0;
  }
  SOFA_CUDA(cudaStreamSynchronize(st));
  return 0;
}

}  // namespace sofa
