// Proposal network for seeding the best-so-far distance (not in the paper).
//
// A 2l -> 256 -> 256 -> C network with exact-erf GELU hidden layers and a
// softmax over C blocks of consecutive key-sorted series.  It is trained on
// (query SFA values -> block of the exact nearest neighbour) pairs that the
// exact search labels, in BF16 on tensor cores with FP32 master weights and
// Adam.  At query time its top-m blocks add seed candidates; the exact scan
// still decides every answer, so the answers never depend on it.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <new>
#include <string>
#include <vector>

#include "sofa_internal.cuh"

namespace sofa {

typedef __nv_bfloat16 bf16;

// ------------------------------------------------------------------------
// Philox-4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11):
// ten rounds of two 32x32->64 multiplies with key bumps by the Weyl constants.
__host__ __device__ inline void philox4x32_10(uint32_t ctr[4], uint32_t k0, uint32_t k1, uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)M0 * c0, p1 = (uint64_t)M1 * c2;
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    c0 = hi1 ^ c1 ^ k0;
    c1 = lo1;
    c2 = hi0 ^ c3 ^ k1;
    c3 = lo0;
    k0 += W0;
    k1 += W1;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

// Uniform in (0, 1) from 32 random bits.
__device__ inline double u01(uint32_t x) { return ((double)x + 0.5) * (1.0 / 4294967296.0); }

// Two standard normals (Box-Muller, FP64) from stream (seed, a, b).
__device__ inline void normal2(uint64_t seed, uint32_t a, uint32_t b, double& z0, double& z1) {
  uint32_t ctr[4] = {a, b, 0x51ED2701u, 0u}, out[4];
  philox4x32_10(ctr, (uint32_t)seed, (uint32_t)(seed >> 32), out);
  const double r = sqrt(-2.0 * log(u01(out[0])));
  double s, c;
  sincospi(2.0 * u01(out[1]), &s, &c);
  z0 = r * c;
  z1 = r * s;
}

// ------------------------------------------------------------------------
// BF16 tensor-core GEMM C[M x N] = A[M x K] B[K x N], FP32 accumulate, with
// mma.sync m16n8k16.  A is row-major (A[m*lda+k]) or, with AT, stored
// transposed (A[k*lda+m]); B is row-major (B[k*ldb+n]) or, with BT, stored
// transposed (B[n*ldb+k]).  Tiles of 128 x 128 x 32 in shared memory with
// k contiguous (row stride 40 bf16: conflict-free fragment loads); 8 warps,
// each 64 x 32.  Epilogues: plain FP32 store, bias add, or bias + GELU
// storing the pre-activation (FP32) and the activation (BF16).
enum { EPI_F32 = 0, EPI_BIAS_F32 = 1, EPI_BIAS_GELU = 2 };
constexpr int GBM = 128, GBN = 128, GBK = 32, GPAD = 8;

__device__ inline float gelu_f(float a) { return 0.5f * a * (1.0f + erff(a * 0.70710678118654752f)); }
__device__ inline float gelu_grad_f(float a) {
  return 0.5f * (1.0f + erff(a * 0.70710678118654752f)) + a * expf(-0.5f * a * a) * 0.39894228040143268f;
}

template <bool AT, bool BT, int EPI>
__global__ void __launch_bounds__(256) k_gemm(int M, int N, int K, const bf16* __restrict__ A, int lda,
                                              const bf16* __restrict__ B, int ldb, float* __restrict__ C, int ldc,
                                              const float* __restrict__ bias, bf16* __restrict__ H, int ldh) {
  __shared__ __align__(16) bf16 As[GBM][GBK + GPAD];
  __shared__ __align__(16) bf16 Bs[GBN][GBK + GPAD];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp >> 2, wn = warp & 3;
  const int m0 = blockIdx.y * GBM, n0 = blockIdx.x * GBN;
  const int g = lane >> 2, t = lane & 3;
  float acc[4][4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;
  const bf16 zero = __float2bfloat16(0.f);
  for (int k0 = 0; k0 < K; k0 += GBK) {
    for (int e = tid; e < GBM * GBK; e += 256) {
      int m, k;
      if (AT) {
        m = e % GBM;
        k = e / GBM;
      } else {
        k = e % GBK;
        m = e / GBK;
      }
      const int gm = m0 + m, gk = k0 + k;
      As[m][k] = (gm < M && gk < K) ? (AT ? A[(int64_t)gk * lda + gm] : A[(int64_t)gm * lda + gk]) : zero;
    }
    for (int e = tid; e < GBN * GBK; e += 256) {
      int nn, k;
      if (BT) {
        k = e % GBK;
        nn = e / GBK;
      } else {
        nn = e % GBN;
        k = e / GBN;
      }
      const int gn = n0 + nn, gk = k0 + k;
      Bs[nn][k] = (gn < N && gk < K) ? (BT ? B[(int64_t)gn * ldb + gk] : B[(int64_t)gk * ldb + gn]) : zero;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GBK; kk += 16) {
      uint32_t af[4][4], bfr[4][2];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int r0 = wm * 64 + i * 16;
        af[i][0] = *reinterpret_cast<const uint32_t*>(&As[r0 + g][kk + 2 * t]);
        af[i][1] = *reinterpret_cast<const uint32_t*>(&As[r0 + g + 8][kk + 2 * t]);
        af[i][2] = *reinterpret_cast<const uint32_t*>(&As[r0 + g][kk + 2 * t + 8]);
        af[i][3] = *reinterpret_cast<const uint32_t*>(&As[r0 + g + 8][kk + 2 * t + 8]);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c0 = wn * 32 + j * 8;
        bfr[j][0] = *reinterpret_cast<const uint32_t*>(&Bs[c0 + g][kk + 2 * t]);
        bfr[j][1] = *reinterpret_cast<const uint32_t*>(&Bs[c0 + g][kk + 2 * t + 8]);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
          asm volatile(
              "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
              "{%0,%1,%2,%3};\n"
              : "+f"(acc[i][j][0]), "+f"(acc[i][j][1]), "+f"(acc[i][j][2]), "+f"(acc[i][j][3])
              : "r"(af[i][0]), "r"(af[i][1]), "r"(af[i][2]), "r"(af[i][3]), "r"(bfr[j][0]), "r"(bfr[j][1]));
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int row = m0 + wm * 64 + i * 16 + g + (r >= 2 ? 8 : 0);
        const int col = n0 + wn * 32 + j * 8 + 2 * t + (r & 1);
        if (row >= M || col >= N) continue;
        float v = acc[i][j][r];
        if (EPI != EPI_F32) v += bias[col];
        C[(int64_t)row * ldc + col] = v;
        if (EPI == EPI_BIAS_GELU) H[(int64_t)row * ldh + col] = __float2bfloat16(gelu_f(v));
      }
}

template <bool AT, bool BT, int EPI>
static int gemm(int M, int N, int K, const bf16* A, int lda, const bf16* B, int ldb, float* C, int ldc,
                const float* bias, bf16* H, int ldh, cudaStream_t st) {
  if (M <= 0 || N <= 0) return 0;
  dim3 grid((unsigned)ceil_div(N, GBN), (unsigned)ceil_div(M, GBM));
  k_gemm<AT, BT, EPI><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, H, ldh);
  SOFA_CUDA(cudaGetLastError());
  return 0;
}

// ------------------------------------------------------------------------
// Elementwise kernels.

// Network input: the query's selected values (word values in columns [0, l),
// the others in [LW, LW + nsel - l)) divided by their sample standard
// deviation; padded to din columns with zeros.  Output BF16 [R x din].
__global__ void k_mlp_input(const float* __restrict__ qv, int64_t R, int NB, int LW, int l, int nsel,
                            const double* __restrict__ var, int din, bf16* __restrict__ X) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= R * din) return;
  int64_t r = e / din;
  int j = (int)(e - r * din);
  float v = 0.f;
  if (j < nsel) {
    const int col = j < l ? j : LW + (j - l);
    const double sd = sqrt(var[j]);
    v = sd > 0 ? (float)((double)qv[r * NB + col] / sd) : 0.f;
  }
  X[e] = __float2bfloat16(v);
}

__global__ void k_f32_to_bf16(const float* __restrict__ a, int64_t n, bf16* __restrict__ b) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = __float2bfloat16(a[i]);
}

// Softmax cross-entropy of one row per CTA: loss_sum += -log p_y;
// dz = (softmax - onehot) / B, written FP32 and BF16.
__global__ void __launch_bounds__(256) k_softmax_xent(const float* __restrict__ logits, int C,
                                                      const int32_t* __restrict__ y, int B,
                                                      float* __restrict__ dz, bf16* __restrict__ dzb,
                                                      float* __restrict__ loss_sum) {
  __shared__ float red[8];
  const int64_t r = blockIdx.x;
  const float* z = logits + r * C;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float mx = -INFINITY;
  for (int c = tid; c < C; c += 256) mx = fmaxf(mx, z[c]);
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
  if (lane == 0) red[warp] = mx;
  __syncthreads();
  mx = red[0];
  for (int i = 1; i < 8; ++i) mx = fmaxf(mx, red[i]);
  __syncthreads();
  float s = 0.f;
  for (int c = tid; c < C; c += 256) s += expf(z[c] - mx);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
  if (lane == 0) red[warp] = s;
  __syncthreads();
  s = 0.f;
  for (int i = 0; i < 8; ++i) s += red[i];
  const int yr = y[r];
  const float inv = 1.f / s, invB = 1.f / (float)B;
  for (int c = tid; c < C; c += 256) {
    const float p = expf(z[c] - mx) * inv;
    const float d = (p - (c == yr ? 1.f : 0.f)) * invB;
    dz[r * C + c] = d;
    dzb[r * C + c] = __float2bfloat16(d);
  }
  if (tid == 0) atomicAdd(loss_sum, -(z[yr] - mx - logf(s)));
}

// da = dh * GELU'(a), FP32 and BF16.
__global__ void k_gelu_bwd(const float* __restrict__ dh, const float* __restrict__ a, int64_t n,
                           float* __restrict__ da, bf16* __restrict__ dab) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float v = dh[i] * gelu_grad_f(a[i]);
  da[i] = v;
  dab[i] = __float2bfloat16(v);
}

// out[c] = sum over rows of X[r][c] (bias gradients), FP32 in row order.
__global__ void k_colsum(const float* __restrict__ X, int rows, int cols, float* __restrict__ out) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  float s = 0.f;
  for (int r = 0; r < rows; ++r) s += X[(int64_t)r * cols + c];
  out[c] = s;
}

// Adam (Kingma & Ba) with bias correction, t counted from 1.
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ gr, float* __restrict__ m,
                       float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float c1, float c2) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float g = gr[i];
  const float mi = b1 * m[i] + (1.f - b1) * g;
  const float vi = b2 * v[i] + (1.f - b2) * g * g;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// Xavier-uniform weights U(-a, a), a = sqrt(6 / (fan_in + fan_out)); zero biases.
__global__ void k_init_uniform(float* __restrict__ w, int64_t n, float a, uint64_t seed, uint32_t stream) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t ctr[4] = {(uint32_t)i, (uint32_t)(i >> 32), stream, 0x1A17u}, out[4];
  philox4x32_10(ctr, (uint32_t)seed, (uint32_t)(seed >> 32), out);
  w[i] = (float)((2.0 * u01(out[0]) - 1.0) * a);
}

// Training queries: rows [0, n_fresh) are fresh random walks (FP64 cumsum of
// N(0,1)), the rest are index members (canonical series of a uniformly drawn
// sorted position) plus N(0, 0.1^2) per point.  Thread per row.
__global__ void k_gen_queries(int64_t R, int64_t n_fresh, int n, int64_t N, const float* __restrict__ Z,
                              uint64_t seed, float* __restrict__ out) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  float* o = out + r * n;
  if (r < n_fresh) {
    double acc = 0.0;
    for (int t = 0; t < n; t += 2) {
      double z0, z1;
      normal2(seed, (uint32_t)r, (uint32_t)(t + ((uint64_t)(r >> 32) << 20)), z0, z1);
      acc += z0;
      o[t] = (float)acc;
      if (t + 1 < n) {
        acc += z1;
        o[t + 1] = (float)acc;
      }
    }
  } else {
    uint32_t ctr[4] = {(uint32_t)r, (uint32_t)(r >> 32), 0x9E37u, 7u}, rnd[4];
    philox4x32_10(ctr, (uint32_t)(seed ^ 0xABCDEFu), (uint32_t)(seed >> 32), rnd);
    const int64_t p = (int64_t)((((uint64_t)rnd[0] << 32) | rnd[1]) % (uint64_t)N);
    const float* src = Z + p * n;
    for (int t = 0; t < n; t += 2) {
      double z0, z1;
      normal2(seed + 1, (uint32_t)r, (uint32_t)(t + ((uint64_t)(r >> 32) << 20)), z0, z1);
      o[t] = (float)((double)src[t] + 0.1 * z0);
      if (t + 1 < n) o[t + 1] = (float)((double)src[t + 1] + 0.1 * z1);
    }
  }
}

__global__ void k_invperm(const uint32_t* __restrict__ perm, int64_t N, uint32_t* __restrict__ pos_of) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < N) pos_of[perm[p]] = (uint32_t)p;
}

__global__ void k_labels(const int64_t* __restrict__ idx, int64_t R, const uint32_t* __restrict__ pos_of,
                         int64_t block, int C, int32_t* __restrict__ y) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  int64_t c = (int64_t)pos_of[idx[r]] / block;
  y[r] = (int32_t)(c < C ? c : C - 1);
}

// Top-m logits of each row (ties: lower class first), CTA per row.
__global__ void __launch_bounds__(256) k_topm(const float* __restrict__ logits, int C, int m,
                                              int32_t* __restrict__ out) {
  __shared__ unsigned long long red[8];
  __shared__ int chosen[16];
  const int64_t r = blockIdx.x;
  const float* z = logits + r * C;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = 0; i < m; ++i) {
    unsigned long long best = 0ull;
    for (int c = tid; c < C; c += 256) {
      bool taken = false;
      for (int j = 0; j < i; ++j) taken |= (chosen[j] == c);
      if (taken) continue;
      // order-preserving map of the float to uint32, larger logit -> larger key
      uint32_t b = __float_as_uint(z[c]);
      b = (b & 0x80000000u) ? ~b : (b | 0x80000000u);
      const unsigned long long key = ((unsigned long long)b << 32) | (uint32_t)(0xFFFFFFFFu - (uint32_t)c);
      best = key > best ? key : best;
    }
    for (int o = 16; o > 0; o >>= 1) {
      unsigned long long v = __shfl_xor_sync(0xFFFFFFFFu, best, o);
      best = v > best ? v : best;
    }
    if (lane == 0) red[warp] = best;
    __syncthreads();
    if (tid == 0) {
      unsigned long long v = red[0];
      for (int w = 1; w < 8; ++w) v = red[w] > v ? red[w] : v;
      chosen[i] = (int)(0xFFFFFFFFu - (uint32_t)v);
      out[r * m + i] = chosen[i];
    }
    __syncthreads();
  }
}

__global__ void k_count_hits(const int32_t* __restrict__ topm, int m, const int32_t* __restrict__ y, int64_t R,
                             unsigned long long* __restrict__ hits) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  if (topm[r * m] == y[r]) atomicAdd(hits, 1ull);
  bool any = false;
  for (int i = 0; i < m; ++i) any |= topm[r * m + i] == y[r];
  if (any) atomicAdd(hits + 1, 1ull);
}

// ========================================================================
// Network state, forward and backward passes.
// ========================================================================
struct Mlp {
  int din = 32, H = 256, C = 4096, top_m = 4;
  int64_t block = 0;  // key-sorted series per class block
  bool trained = false;
  int64_t o_W1 = 0, o_b1 = 0, o_W2 = 0, o_b2 = 0, o_W3 = 0, o_b3 = 0, total = 0;
  float *P = nullptr, *G = nullptr, *Mo = nullptr, *Ve = nullptr;
  bf16* Pb = nullptr;
  int64_t step = 0;
  double train_loss = 0, val_top1 = 0, val_topm = 0;
  int64_t n_train = 0;
  DevBuf a1, h1, a2, h2, logits, dz, dzb, dh, da, dab, xb, topm, misc;

  void layout() {
    o_W1 = 0;
    o_b1 = o_W1 + (int64_t)din * H;
    o_W2 = o_b1 + H;
    o_b2 = o_W2 + (int64_t)H * H;
    o_W3 = o_b2 + H;
    o_b3 = o_W3 + (int64_t)H * C;
    total = o_b3 + C;
  }
  int alloc() {
    layout();
    float** fs[] = {&P, &G, &Mo, &Ve};
    for (float** f : fs) {
      if (dev_malloc((void**)f, total * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        return fail(SOFA_ERR_OOM, "proposal network allocation failed");
      }
      cudaMemset(*f, 0, total * sizeof(float));
    }
    if (dev_malloc((void**)&Pb, total * sizeof(bf16)) != cudaSuccess) {
      cudaGetLastError();
      return fail(SOFA_ERR_OOM, "proposal network allocation failed");
    }
    return 0;
  }
  void release() {
    float* fs[] = {P, G, Mo, Ve};
    for (float* f : fs)
      if (f) cudaFree(f);
    if (Pb) cudaFree(Pb);
    P = G = Mo = Ve = nullptr;
    Pb = nullptr;
    DevBuf* bs[] = {&a1, &h1, &a2, &h2, &logits, &dz, &dzb, &dh, &da, &dab, &xb, &topm, &misc};
    for (DevBuf* b : bs) b->release();
  }
  int ensure_rows(int64_t R) {
    int rc = 0;
    rc |= a1.ensure(R * H * sizeof(float));
    rc |= h1.ensure(R * H * sizeof(bf16));
    rc |= a2.ensure(R * H * sizeof(float));
    rc |= h2.ensure(R * H * sizeof(bf16));
    rc |= logits.ensure(R * C * sizeof(float));
    return rc ? SOFA_ERR_OOM : 0;
  }
  int ensure_train(int64_t B) {
    int rc = ensure_rows(B);
    rc |= dz.ensure(B * C * sizeof(float));
    rc |= dzb.ensure(B * C * sizeof(bf16));
    rc |= dh.ensure(B * H * sizeof(float));
    rc |= da.ensure(B * H * sizeof(float));
    rc |= dab.ensure(B * H * sizeof(bf16));
    rc |= misc.ensure(64);
    return rc ? SOFA_ERR_OOM : 0;
  }
  int sync_bf16(cudaStream_t st) {
    k_f32_to_bf16<<<(unsigned)ceil_div(total, 256), 256, 0, st>>>(P, total, Pb);
    SOFA_CUDA(cudaGetLastError());
    return 0;
  }
  // logits = f(X), X: BF16 [R x din]
  int forward(const bf16* X, int64_t R, cudaStream_t st) {
    const int r = (int)R;
    if (int rc = gemm<false, false, EPI_BIAS_GELU>(r, H, din, X, din, Pb + o_W1, H, a1.as<float>(), H, P + o_b1,
                                                   h1.as<bf16>(), H, st))
      return rc;
    if (int rc = gemm<false, false, EPI_BIAS_GELU>(r, H, H, h1.as<bf16>(), H, Pb + o_W2, H, a2.as<float>(), H,
                                                   P + o_b2, h2.as<bf16>(), H, st))
      return rc;
    return gemm<false, false, EPI_BIAS_F32>(r, C, H, h2.as<bf16>(), H, Pb + o_W3, C, logits.as<float>(), C,
                                            P + o_b3, nullptr, 0, st);
  }
  // gradients of the mean softmax cross-entropy into G; loss sum into *loss
  int backward(const bf16* X, const int32_t* y, int B, float* loss, cudaStream_t st) {
    k_softmax_xent<<<B, 256, 0, st>>>(logits.as<float>(), C, y, B, dz.as<float>(), dzb.as<bf16>(), loss);
    SOFA_CUDA(cudaGetLastError());
    const int64_t bh = (int64_t)B * H;
    const unsigned ge = (unsigned)ceil_div(bh, 256);
    if (int rc = gemm<true, false, EPI_F32>(H, C, B, h2.as<bf16>(), H, dzb.as<bf16>(), C, G + o_W3, C, nullptr,
                                            nullptr, 0, st))
      return rc;
    k_colsum<<<(unsigned)ceil_div(C, 256), 256, 0, st>>>(dz.as<float>(), B, C, G + o_b3);
    if (int rc = gemm<false, true, EPI_F32>(B, H, C, dzb.as<bf16>(), C, Pb + o_W3, C, dh.as<float>(), H, nullptr,
                                            nullptr, 0, st))
      return rc;
    k_gelu_bwd<<<ge, 256, 0, st>>>(dh.as<float>(), a2.as<float>(), bh, da.as<float>(), dab.as<bf16>());
    if (int rc = gemm<true, false, EPI_F32>(H, H, B, h1.as<bf16>(), H, dab.as<bf16>(), H, G + o_W2, H, nullptr,
                                            nullptr, 0, st))
      return rc;
    k_colsum<<<(unsigned)ceil_div(H, 256), 256, 0, st>>>(da.as<float>(), B, H, G + o_b2);
    if (int rc = gemm<false, true, EPI_F32>(B, H, H, dab.as<bf16>(), H, Pb + o_W2, H, dh.as<float>(), H, nullptr,
                                            nullptr, 0, st))
      return rc;
    k_gelu_bwd<<<ge, 256, 0, st>>>(dh.as<float>(), a1.as<float>(), bh, da.as<float>(), dab.as<bf16>());
    if (int rc = gemm<true, false, EPI_F32>(din, H, B, X, din, dab.as<bf16>(), H, G + o_W1, H, nullptr, nullptr, 0,
                                            st))
      return rc;
    k_colsum<<<(unsigned)ceil_div(H, 256), 256, 0, st>>>(da.as<float>(), B, H, G + o_b1);
    SOFA_CUDA(cudaGetLastError());
    return 0;
  }
};

void mlp_free(Mlp* m) {
  if (!m) return;
  m->release();
  delete m;
}

#define TRYM(x)          \
  do {                   \
    int rc_ = (x);       \
    if (rc_) return rc_; \
  } while (0)

// Inputs (standardised selected values) of R raw queries, via the index's
// own query transform.
static int mlp_inputs(Index* ix, Mlp* m, const float* q, int64_t R, bf16* X, cudaStream_t st) {
  const int64_t QB = 8192;
  for (int64_t r0 = 0; r0 < R; r0 += QB) {
    const int64_t rb = std::min(QB, R - r0);
    TRYM(ix->qs.zq.ensure(rb * ix->n * sizeof(float)));
    TRYM(ix->qs.qv.ensure(rb * ix->NB * sizeof(float)));
    TRYM(launch_qprep(ix, q + r0 * ix->n, rb, ix->qs.zq.as<float>(), ix->qs.qv.as<float>(), st));
    k_mlp_input<<<(unsigned)ceil_div(rb * m->din, 256), 256, 0, st>>>(ix->qs.qv.as<float>(), rb, ix->NB, ix->LW,
                                                                       ix->l, ix->nsel, ix->var, m->din,
                                                                       X + r0 * m->din);
    SOFA_CUDA(cudaGetLastError());
  }
  return 0;
}

int mlp_train(Index* ix, const sofa_train_opts& o, cudaStream_t st) {
  Mlp* m = ix->mlp;
  if (!m) {
    m = new Mlp();
    ix->mlp = m;
  } else {
    m->release();
  }
  m->C = o.n_classes > 0 ? o.n_classes : 4096;
  m->top_m = o.top_m > 0 ? o.top_m : 4;
  m->din = 32;
  m->trained = false;
  m->block = ceil_div(ix->N, m->C);
  TRYM(m->alloc());
  const int64_t R = o.n_train > 0 ? o.n_train : (1 << 20);
  const int epochs = o.epochs > 0 ? o.epochs : 4;
  const int B = o.batch > 0 ? o.batch : 4096;
  const float lr = o.lr > 0 ? o.lr : 1e-3f;
  const uint64_t seed = o.seed;
  m->n_train = R;
  // training queries
  DevBuf qbuf, xbuf, ybuf, ibuf, dbuf, posbuf;
  TRYM(qbuf.ensure((size_t)R * ix->n * sizeof(float)));
  float* qd = qbuf.as<float>();
  if (o.train_queries) {
    SOFA_CUDA(cudaMemcpyAsync(qd, o.train_queries, (size_t)R * ix->n * sizeof(float), cudaMemcpyDefault, st));
  } else {
    k_gen_queries<<<(unsigned)ceil_div(R, 128), 128, 0, st>>>(R, R / 2, ix->n, ix->N, ix->Z, seed, qd);
    SOFA_CUDA(cudaGetLastError());
  }
  // labels: block of the exact nearest neighbour (the exact search itself)
  TRYM(ibuf.ensure((size_t)R * sizeof(int64_t)));
  TRYM(dbuf.ensure((size_t)R * sizeof(float)));
  TRYM(ybuf.ensure((size_t)R * sizeof(int32_t)));
  TRYM(posbuf.ensure((size_t)ix->N * sizeof(uint32_t)));
  const int saved_mode = ix->seed_mode;
  ix->seed_mode = 0;
  TRYM(run_query(ix, qd, R, 1, ibuf.as<int64_t>(), dbuf.as<float>(), st));
  ix->seed_mode = saved_mode;
  k_invperm<<<(unsigned)ceil_div(ix->N, 256), 256, 0, st>>>(ix->perm, ix->N, posbuf.as<uint32_t>());
  k_labels<<<(unsigned)ceil_div(R, 256), 256, 0, st>>>(ibuf.as<int64_t>(), R, posbuf.as<uint32_t>(), m->block, m->C,
                                                       ybuf.as<int32_t>());
  SOFA_CUDA(cudaGetLastError());
  // inputs
  TRYM(xbuf.ensure((size_t)R * m->din * sizeof(bf16)));
  TRYM(mlp_inputs(ix, m, qd, R, xbuf.as<bf16>(), st));
  qbuf.release();
  // Xavier-uniform initial weights
  const float aw1 = std::sqrt(6.0f / (m->din + m->H)), aw2 = std::sqrt(6.0f / (2 * m->H)),
              aw3 = std::sqrt(6.0f / (m->H + m->C));
  k_init_uniform<<<(unsigned)ceil_div((int64_t)m->din * m->H, 256), 256, 0, st>>>(m->P + m->o_W1,
                                                                                   (int64_t)m->din * m->H, aw1, seed, 1);
  k_init_uniform<<<(unsigned)ceil_div((int64_t)m->H * m->H, 256), 256, 0, st>>>(m->P + m->o_W2, (int64_t)m->H * m->H,
                                                                                 aw2, seed, 2);
  k_init_uniform<<<(unsigned)ceil_div((int64_t)m->H * m->C, 256), 256, 0, st>>>(m->P + m->o_W3, (int64_t)m->H * m->C,
                                                                                 aw3, seed, 3);
  SOFA_CUDA(cudaGetLastError());
  // held-out split: the last 1/20 of the pairs
  const int64_t R_val = std::max<int64_t>(1, R / 20);
  const int64_t R_tr = std::max<int64_t>(1, R - R_val);
  TRYM(m->ensure_train(B));
  float* dloss = m->misc.as<float>();
  double loss_last = 0;
  for (int ep = 0; ep < epochs; ++ep) {
    SOFA_CUDA(cudaMemsetAsync(dloss, 0, sizeof(float), st));
    int64_t seen = 0;
    for (int64_t b0 = 0; b0 + 1 <= R_tr; b0 += B) {
      const int bsz = (int)std::min<int64_t>(B, R_tr - b0);
      const bf16* X = xbuf.as<bf16>() + b0 * m->din;
      TRYM(m->sync_bf16(st));
      TRYM(m->forward(X, bsz, st));
      TRYM(m->backward(X, ybuf.as<int32_t>() + b0, bsz, dloss, st));
      m->step += 1;
      const float c1 = 1.f - std::pow(0.9f, (float)m->step), c2 = 1.f - std::pow(0.999f, (float)m->step);
      k_adam<<<(unsigned)ceil_div(m->total, 256), 256, 0, st>>>(m->P, m->G, m->Mo, m->Ve, m->total, lr, 0.9f, 0.999f,
                                                                 1e-8f, c1, c2);
      SOFA_CUDA(cudaGetLastError());
      seen += bsz;
    }
    float hl = 0;
    SOFA_CUDA(cudaMemcpyAsync(&hl, dloss, sizeof(float), cudaMemcpyDeviceToHost, st));
    SOFA_CUDA(cudaStreamSynchronize(st));
    loss_last = seen ? hl / (double)seen : 0.0;
  }
  m->train_loss = loss_last;
  // held-out accuracy of the block prediction (top-1 and top-m)
  TRYM(m->sync_bf16(st));
  TRYM(m->topm.ensure((size_t)R_val * m->top_m * sizeof(int32_t)));
  unsigned long long* hits = reinterpret_cast<unsigned long long*>(m->misc.as<char>() + 16);
  SOFA_CUDA(cudaMemsetAsync(hits, 0, 2 * sizeof(unsigned long long), st));
  for (int64_t r0 = R - R_val; r0 < R; r0 += B) {
    const int bsz = (int)std::min<int64_t>(B, R - r0);
    TRYM(m->forward(xbuf.as<bf16>() + r0 * m->din, bsz, st));
    k_topm<<<bsz, 256, 0, st>>>(m->logits.as<float>(), m->C, m->top_m, m->topm.as<int32_t>());
    k_count_hits<<<(unsigned)ceil_div(bsz, 256), 256, 0, st>>>(m->topm.as<int32_t>(), m->top_m,
                                                                ybuf.as<int32_t>() + r0, bsz, hits);
    SOFA_CUDA(cudaGetLastError());
  }
  unsigned long long hh[2];
  SOFA_CUDA(cudaMemcpyAsync(hh, hits, sizeof(hh), cudaMemcpyDeviceToHost, st));
  SOFA_CUDA(cudaStreamSynchronize(st));
  m->val_top1 = (double)hh[0] / (double)R_val;
  m->val_topm = (double)hh[1] / (double)R_val;
  m->trained = true;
  return 0;
}

// Top-m predicted blocks of Q queries (given their projected values qv).
int mlp_seed(Index* ix, const float* qv, int64_t Q, int k, cudaStream_t st) {
  (void)k;
  Mlp* m = ix->mlp;
  if (!m || !m->trained) return fail(SOFA_ERR_NOT_TRAINED, "proposal network not trained");
  TRYM(m->xb.ensure((size_t)Q * m->din * sizeof(bf16)));
  TRYM(m->topm.ensure((size_t)Q * m->top_m * sizeof(int32_t)));
  TRYM(m->ensure_rows(Q));
  k_mlp_input<<<(unsigned)ceil_div(Q * m->din, 256), 256, 0, st>>>(qv, Q, ix->NB, ix->LW, ix->l, ix->nsel, ix->var,
                                                                    m->din, m->xb.as<bf16>());
  SOFA_CUDA(cudaGetLastError());
  TRYM(m->forward(m->xb.as<bf16>(), Q, st));
  k_topm<<<(unsigned)Q, 256, 0, st>>>(m->logits.as<float>(), m->C, m->top_m, m->topm.as<int32_t>());
  SOFA_CUDA(cudaGetLastError());
  return 0;
}

const int32_t* mlp_topm(Index* ix, int* m, int64_t* block) {
  if (!ix->mlp || !ix->mlp->trained) return nullptr;
  *m = ix->mlp->top_m;
  *block = ix->mlp->block;
  return ix->mlp->topm.as<int32_t>();
}

// Proposal network in an index file: shape, state and statistics, then the
// FP32 master weights (the BF16 copy is derived again on loading).
int mlp_save(const Index* ix, void* file) {
  FILE* f = static_cast<FILE*>(file);
  const Mlp* m = ix->mlp;
  const int64_t hdr[8] = {m->din, m->H, m->C, m->top_m, m->block, m->trained ? 1 : 0, m->n_train, m->total};
  const double stats[3] = {m->train_loss, m->val_top1, m->val_topm};
  std::vector<float> w((size_t)m->total);
  if (m->total) SOFA_CUDA(cudaMemcpy(w.data(), m->P, (size_t)m->total * sizeof(float), cudaMemcpyDeviceToHost));
  if (fwrite(hdr, sizeof(hdr), 1, f) != 1 || fwrite(stats, sizeof(stats), 1, f) != 1 ||
      fwrite(w.data(), sizeof(float), w.size(), f) != w.size())
    return fail(SOFA_ERR_INVALID_ARG, "write failed");
  return 0;
}

int mlp_load(Index* ix, void* file, cudaStream_t st) {
  FILE* f = static_cast<FILE*>(file);
  int64_t hdr[8];
  double stats[3];
  if (fread(hdr, sizeof(hdr), 1, f) != 1 || fread(stats, sizeof(stats), 1, f) != 1)
    return fail(SOFA_ERR_INVALID_ARG, "truncated index file (proposal network)");
  if (hdr[0] != 32 || hdr[1] < 1 || hdr[1] > 4096 || hdr[2] < 1 || hdr[2] > (1 << 20) || hdr[3] < 1 ||
      hdr[3] > 16 || hdr[3] > hdr[2] || hdr[4] < 1)
    return fail(SOFA_ERR_INVALID_ARG, "index file: inconsistent proposal network header");
  Mlp* m = new (std::nothrow) Mlp();
  if (!m) return fail(SOFA_ERR_OOM, "host allocation failed");
  m->din = (int)hdr[0];
  m->H = (int)hdr[1];
  m->C = (int)hdr[2];
  m->top_m = (int)hdr[3];
  m->block = hdr[4];
  m->n_train = hdr[6];
  m->train_loss = stats[0];
  m->val_top1 = stats[1];
  m->val_topm = stats[2];
  ix->mlp = m;  // freed with the index on any error below
  TRYM(m->alloc());
  if (m->total != hdr[7]) return fail(SOFA_ERR_INVALID_ARG, "index file: proposal network size mismatch");
  std::vector<float> w((size_t)m->total);
  if (fread(w.data(), sizeof(float), w.size(), f) != w.size())
    return fail(SOFA_ERR_INVALID_ARG, "truncated index file (proposal network)");
  SOFA_CUDA(cudaMemcpy(m->P, w.data(), w.size() * sizeof(float), cudaMemcpyHostToDevice));
  TRYM(m->sync_bf16(st));
  SOFA_CUDA(cudaStreamSynchronize(st));
  m->trained = hdr[5] != 0;
  return 0;
}

void mlp_report(Index* ix, double* loss, double* top1, double* topm, int64_t* classes, int64_t* n_train) {
  Mlp* m = ix->mlp;
  *loss = m && m->trained ? m->train_loss : 0;
  *top1 = m && m->trained ? m->val_top1 : 0;
  *topm = m && m->trained ? m->val_topm : 0;
  *classes = m && m->trained ? m->C : 0;
  *n_train = m && m->trained ? m->n_train : 0;
}

}  // namespace sofa

using namespace sofa;

extern "C" int sofa_train_proposal(sofa_handle h, const sofa_train_opts* o, sofa_stream stream) {
  if (!h || !o) return fail(SOFA_ERR_INVALID_ARG, "null argument");
  if (o->n_train < 0 || o->n_classes < 0 || o->n_classes > 8192 || o->epochs < 0 || o->batch < 0 ||
      o->top_m < 0 || o->top_m > 8 || o->lr < 0)
    return fail(SOFA_ERR_INVALID_ARG, "bad training options");
  if (o->n_classes > 0 && o->n_classes > h->N) return fail(SOFA_ERR_INVALID_ARG, "more classes than series");
  if (o->n_classes == 0 && h->N < 4096) return fail(SOFA_ERR_INVALID_ARG, "n_classes must be set when N < 4096");
  if (int rc = check_device(h)) return rc;
  return mlp_train(h, *o, (cudaStream_t)stream);
}

extern "C" int sofa_set_seed_mode(sofa_handle h, int32_t mode) {
  if (!h) return fail(SOFA_ERR_INVALID_ARG, "handle is NULL");
  if (mode == 0) {
    h->seed_mode = 0;
    return 0;
  }
  if (mode == 1) {
    if (!h->mlp || !h->mlp->trained) return fail(SOFA_ERR_NOT_TRAINED, "learned seeding needs sofa_train_proposal first");
    h->seed_mode = 1;
    return 0;
  }
  return fail(SOFA_ERR_INVALID_ARG, "seed mode must be 0 or 1");
}

// Loss and gradients of the proposal network on one batch (see sofa.h).
extern "C" int sofa_mlp_grad(int32_t din, int32_t hidden, int32_t classes, const float* params, const float* x,
                             const int32_t* y, int32_t B, float* grads, float* loss, sofa_stream stream) {
  if (din < 1 || din > 64 || hidden < 1 || hidden > 1024 || classes < 2 || classes > 8192 || B < 1 || !params || !x ||
      !y || !grads || !loss)
    return fail(SOFA_ERR_INVALID_ARG, "bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  Mlp m;
  m.din = din;
  m.H = hidden;
  m.C = classes;
  int rc = m.alloc();
  if (!rc) rc = m.ensure_train(B);
  DevBuf xb;
  if (!rc) rc = xb.ensure((size_t)B * din * sizeof(bf16));
  if (!rc) {
    cudaMemcpyAsync(m.P, params, m.total * sizeof(float), cudaMemcpyDefault, st);
    k_f32_to_bf16<<<(unsigned)ceil_div((int64_t)B * din, 256), 256, 0, st>>>(x, (int64_t)B * din, xb.as<bf16>());
    cudaMemsetAsync(m.misc.p, 0, sizeof(float), st);
    rc = m.sync_bf16(st);
  }
  if (!rc) rc = m.forward(xb.as<bf16>(), B, st);
  if (!rc) rc = m.backward(xb.as<bf16>(), y, B, m.misc.as<float>(), st);
  if (!rc) {
    cudaMemcpyAsync(grads, m.G, m.total * sizeof(float), cudaMemcpyDefault, st);
    float l = 0;
    cudaMemcpyAsync(&l, m.misc.p, sizeof(float), cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) rc = fail(SOFA_ERR_CUDA, "stream failed");
    *loss = l / (float)B;
  }
  xb.release();
  m.release();
  return rc;
}
