// Dense form of the query for batches whose lower bounds prune (almost)
// nothing.  GEMINI's refinement computes exact distances of the survivors of
// the bound (Sec. II-A); when the bound passes every series -- high-frequency
// data whose selected Fourier values carry little of the energy -- the
// survivors are the whole collection, and the distances of a batch are one
// dense contraction: d^2(q, x) = ||q||^2 + ||x||^2 - 2 q.x.
//
// The contraction runs on the tensor cores (tcgen05, kind::tf32) straight
// from the fp32 canonical series: operands are staged by TMA into 128-byte
// swizzled shared-memory tiles, the accumulator lives in tensor memory.  A CTA
// holds 128 queries (the MMA's M, one TMEM lane each) and walks a chunk of
// tiles of 256 series (N, the TMEM columns), K in blocks of 32 values.  Its
// epilogue turns each accumulator column into an approximate squared distance
// and emits every series whose lower bound (d~^2 - M) / 2 may still reach the
// query's answer into the same candidate store the series scan fills, so the
// exact refinement, merge and final re-score are unchanged.  M bounds
// |d~^2 - d^2| (TF32 operands, FP32 accumulation; derived on the host).  Each
// thread keeps the k smallest d~^2 it has seen, which tightens the emission
// threshold as the chunk proceeds and is published to the query's threshold.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cmath>
#include <cstring>

#include "sofa_internal.cuh"
#include "tc_ptx.cuh"

namespace sofa {

constexpr int DM = 128;                  // queries per CTA: MMA M, TMEM lanes
constexpr int DN = 256;                  // series per tile: MMA N, TMEM columns
constexpr int DK = 32;                   // fp32 values per k-block: one 128-byte swizzled row (64 for fp16)
constexpr int DSTAGES = 4;               // TMA pipeline depth
constexpr int A_BYTES = DM * DK * 4;     // 16 KB
constexpr int B_BYTES = DN * DK * 4;     // 32 KB
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int DENSE_SMEM = DSTAGES * STAGE_BYTES + 1024;  // + alignment slack
constexpr int DKMAX = 16;                // largest k of the dense path

// Instruction descriptor of tcgen05.mma kind::tf32 / kind::f16: D fp32
// (bits 4-5 = 1), A and B tf32 (bits 7-9, 10-12 = 2) or f16 (= 0), both
// K-major (bits 15, 16 = 0), N >> 3 in bits 17-22, M >> 4 in bits 24-28.
template <bool F16>
__host__ __device__ constexpr uint32_t dense_idesc() {
  return (1u << 4) | ((F16 ? 0u : 2u) << 7) | ((F16 ? 0u : 2u) << 10) | ((uint32_t)(DN >> 3) << 17) |
         ((uint32_t)(DM >> 4) << 24);
}

struct DenseParams {
  int64_t N;           // series
  int Q;               // queries of the batch
  int n;               // values per series
  int k;               // neighbours
  int cap;             // candidate region per query slot
  int64_t pool_cap;    // shared pool entries
  int64_t tiles_per_cta;
  float margin;        // M >= |d~^2 - d^2|
  float f_half;        // f_prune / 2: threshold of a real k-th squared distance
};


// One MMA of K = 32 bytes of each operand row (8 tf32 or 16 f16 values).
template <bool F16>
__device__ __forceinline__ void mma_dense(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  if constexpr (F16)
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(dense_idesc<true>()), "r"(accumulate));
  else
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(dense_idesc<false>()), "r"(accumulate));
}


// ||x||^2 of every canonical series: FP64 sum (lane-strided partial sums,
// then a warp reduction), rounded to fp32.
__global__ void k_row_norms(const float* __restrict__ Z, int64_t N, int n, float* __restrict__ out) {
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= N) return;
  double s = 0.0;
  for (int t = lane; t < n; t += 32) {
    const double z = Z[row * n + t];
    s += z * z;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
  if (lane == 0) out[row] = (float)s;
}

// The k smallest approximate squared distances seen by a thread (ascending);
// KD = 1 for k = 1, else DKMAX.
template <int KD>
__device__ __forceinline__ void topk_insert(float* top, float x) {
#pragma unroll
  for (int i = 0; i < KD; ++i) {
    const float lo = fminf(top[i], x);
    x = fmaxf(top[i], x);
    top[i] = lo;
  }
}

template <int KD>
__device__ __forceinline__ float topk_kth(const float* top, int k) {
  float v = top[0];
#pragma unroll
  for (int i = 1; i < KD; ++i)
    if (i == k - 1) v = top[i];
  return v;
}


// Warp-specialised CTA of 6 warps: warp 0 issues the TMA loads, warp 1 the
// MMAs (and owns the tensor memory: two 256-column accumulators, so the
// epilogue of one series tile overlaps the MMAs of the next), warps 2-5 run
// the epilogue, each on its quarter of the TMEM lanes (lane quadrant = warp
// index mod 4).  Barriers: full / empty per pipeline stage (TMA -> MMA ->
// TMA), tfull / tempty per accumulator (MMA -> epilogue -> MMA).  Every wait
// is bounded; a timed-out wait stops all roles and sets the status.
constexpr int DWARPS = 6;
constexpr int DTHREADS = 32 * DWARPS;
constexpr int DACC = 2;

template <int KD, bool F16>
__global__ void __launch_bounds__(DTHREADS, 1) k_dense(const __grid_constant__ CUtensorMap tmQ,
                                                       const __grid_constant__ CUtensorMap tmX, DenseParams D,
                                                       const float* __restrict__ qn, const float* __restrict__ xn,
                                                       const int* __restrict__ qsel, const int* __restrict__ qslot,
                                                       float* __restrict__ thr, uint32_t* __restrict__ cand_p,
                                                       float* __restrict__ cand_lb, int* __restrict__ cand_n,
                                                       int* __restrict__ pool_n,
                                                       int* __restrict__ pool_q, uint32_t* __restrict__ pool_p,
                                                       float* __restrict__ pool_lb, int* __restrict__ qpool_cnt,
                                                       float* __restrict__ dump,
                                                       unsigned long long* __restrict__ counters,
                                                       int* __restrict__ status) {
  extern __shared__ uint8_t dsm_raw[];
  __shared__ __align__(8) uint64_t full[DSTAGES], empty[DSTAGES], tfull[DACC], tempty[DACC], drain;
  __shared__ __align__(16) float s_x[4][DN];  // per epilogue warp: ||x||^2 of the tile's series
  __shared__ float s_v[4][32][32];             // per epilogue warp: 32 accumulator columns x 32 lanes
  __shared__ uint32_t s_tmem;
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t n_tiles = (D.N + DN - 1) / DN;
  const int64_t t_begin = (int64_t)blockIdx.y * D.tiles_per_cta;
  const int64_t t_end = t_begin + D.tiles_per_cta < n_tiles ? t_begin + D.tiles_per_cta : n_tiles;
  if (t_begin >= t_end) return;  // the whole CTA, before any barrier or allocation
  const uint32_t raw = smem_u32(dsm_raw);
  uint8_t* stages = dsm_raw + (((raw + 1023u) & ~1023u) - raw);  // 1024-byte swizzle atoms
  const int q0 = blockIdx.x * DM;
  constexpr int DKE = F16 ? 2 * DK : DK;  // values per k-block (one 128-byte row)
  const int kblocks = (D.n + DKE - 1) / DKE;
  const int64_t ntiles = t_end - t_begin;
  const int64_t total = ntiles * kblocks;
  volatile int* vfail = &s_fail;

  if (warp == 1) tmem_alloc(&s_tmem, DN * DACC);
  if (tid == 0) {
    for (int s = 0; s < DSTAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < DACC; ++a) {
      mbar_init(&tfull[a], 1);
      mbar_init(&tempty[a], 4 * 32);  // every epilogue thread
    }
    mbar_init(&drain, 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;

  // epilogue threads: one query each (its TMEM lane)
  const bool epi = warp >= 2;
  const int er = 32 * (warp & 3) + lane;
  const int q = q0 + er;
  const bool qa = epi && q < D.Q && (!qsel || qsel[q]);
  const int nq_active = __syncthreads_count(qa);

  if (warp == 0) {
    if (lane == 0) {  // TMA producer
      for (int64_t idx = 0; idx < total; ++idx) {
        const int s = (int)(idx % DSTAGES);
        if (idx >= DSTAGES && !mbar_wait(&empty[s], (uint32_t)((idx / DSTAGES - 1) & 1))) {
          *vfail = 1;
          break;
        }
        if (*vfail) break;
        const int64_t tile = t_begin + idx / kblocks;
        const int kb = (int)(idx % kblocks);
        uint8_t* a = stages + s * STAGE_BYTES;
        mbar_expect_tx(&full[s], STAGE_BYTES);
        tma_load_2d(a, &tmQ, kb * DKE, q0, &full[s]);
        tma_load_2d(a + A_BYTES, &tmX, kb * DKE, (int)(tile * DN), &full[s]);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer
      for (int64_t ti = 0; ti < ntiles && !*vfail; ++ti) {
        const int acc = (int)(ti & 1);
        if (ti >= DACC && !mbar_wait(&tempty[acc], (uint32_t)((ti / DACC - 1) & 1))) {
          *vfail = 1;
          break;
        }
        tc_fence_after();
        const uint32_t dcol = tmem + (uint32_t)(acc * DN);
        bool ok = true;
        for (int kb = 0; kb < kblocks; ++kb) {
          const int64_t idx = ti * kblocks + kb;
          const int s = (int)(idx % DSTAGES);
          if (!mbar_wait(&full[s], (uint32_t)((idx / DSTAGES) & 1))) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = smem_u32(stages + s * STAGE_BYTES);
          const uint64_t ad = sw128_desc(sa), bd = sw128_desc(sa + A_BYTES);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)  // 32 bytes of K per MMA: 8 tf32 or 16 f16 values
            mma_dense<F16>(dcol, ad + (uint64_t)(2 * kk), bd + (uint64_t)(2 * kk), (kb | kk) != 0 ? 1u : 0u);
          mma_commit(&empty[s]);
        }
        if (!ok) {
          *vfail = 1;
          break;
        }
        mma_commit(&tfull[acc]);
      }
    }
  } else {
    // epilogue.  Per 32 columns: d~^2 = ||q||^2 + ||x||^2 - 2 q.x of each
    // (one FADD, one FFMA) and their minimum; the lower bound is monotone in
    // d~^2, so the columns are visited one by one only when the minimum
    // passes the threshold (rare once the threshold is tight).
    float* xs = s_x[warp - 2];      // this warp's copy of the tile's ||x||^2 (+inf past N)
    float* vs = &s_v[warp - 2][0][0];  // [column][lane] spill of the accumulator for the slow path
    const int qs = qa ? (qslot ? qslot[q] : q) : 0;
    const float qnr = qa ? qn[q] : INFINITY;  // inactive lanes: every d~^2 is +inf
    volatile float* vthr = thr;
    float T = qa ? vthr[q] : -1.f;  // emission threshold, half units
    float top[KD];
#pragma unroll
    for (int i = 0; i < KD; ++i) top[i] = INFINITY;
    unsigned long long emitted = 0;
    const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
    // ||x||^2 of the next tile, prefetched a tile ahead.  The addresses are
    // clamped and the +inf past N is applied where the values are used, so
    // nothing waits for the loads before then.
    float xr[DN / 32];
    uint32_t xok = 0u;  // bit j: xr[j] is a series of the index
#pragma unroll
    for (int j = 0; j < DN / 32; ++j) {
      const int64_t sx = t_begin * DN + lane + 32 * j;
      xr[j] = __ldg(xn + (sx < D.N ? sx : (int64_t)0));
      xok |= (sx < D.N ? 1u : 0u) << j;
    }
    for (int64_t ti = 0; ti < ntiles; ++ti) {
      const int acc = (int)(ti & 1);
      const float Tg = vthr[qa ? q : 0];  // in flight during the wait below (used by active lanes only)
      // warp-uniform: the TMEM loads below are warp-collective
      if (!__all_sync(0xFFFFFFFFu, mbar_wait(&tfull[acc], (uint32_t)((ti / DACC) & 1)))) {
        *vfail = 1;
        break;
      }
      tc_fence_after();
      const int64_t s0 = (t_begin + ti) * DN;
      __syncwarp();
#pragma unroll
      for (int j = 0; j < DN / 32; ++j) xs[lane + 32 * j] = ((xok >> j) & 1u) ? xr[j] : INFINITY;
      __syncwarp();
      if (ti + 1 < ntiles) {
        xok = 0u;
#pragma unroll
        for (int j = 0; j < DN / 32; ++j) {
          const int64_t sx = s0 + DN + lane + 32 * j;
          xr[j] = __ldg(xn + (sx < D.N ? sx : (int64_t)0));
          xok |= (sx < D.N ? 1u : 0u) << j;
        }
      }
      if (qa) T = fminf(T, Tg);
      const float T_in = T;
#pragma unroll 1
      for (int c0 = 0; c0 < DN; c0 += 32) {
        float v[32];
        tmem_ld32(tmem + lane_base + (uint32_t)(acc * DN + c0), v);  // warp-collective
        const float4* x4 = reinterpret_cast<const float4*>(xs + c0);
        if (dump) {
#pragma unroll
          for (int i = 0; i < 32; i += 4) {
            const float4 xv = x4[i >> 2];
            const float xq[4] = {xv.x, xv.y, xv.z, xv.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const int64_t sidx = s0 + c0 + i + e;
              if (qa && sidx < D.N) dump[(int64_t)q * D.N + sidx] = fmaf(-2.f, v[i + e], qnr + xq[e]);
            }
          }
          continue;
        }
        float m = INFINITY;
#pragma unroll
        for (int i = 0; i < 32; i += 4) {
          const float4 xv = x4[i >> 2];
          m = fminf(m, fminf(fminf(fmaf(-2.f, v[i], qnr + xv.x), fmaf(-2.f, v[i + 1], qnr + xv.y)),
                             fminf(fmaf(-2.f, v[i + 2], qnr + xv.z), fmaf(-2.f, v[i + 3], qnr + xv.w))));
        }
        const bool pass = __fmul_rd(__fsub_rd(m, D.margin), 0.5f) <= T;
        if (!__any_sync(0xFFFFFFFFu, pass)) continue;
        // slow path: the accumulator columns through shared memory, one by one
#pragma unroll
        for (int i = 0; i < 32; ++i) vs[i * 32 + lane] = v[i];
        __syncwarp();
        if (pass) {
#pragma unroll 1
          for (int i = 0; i < 32; ++i) {
            const float d2 = fmaf(-2.f, vs[i * 32 + lane], qnr + xs[c0 + i]);  // the value the minimum took
            const float lb = __fmul_rd(__fsub_rd(d2, D.margin), 0.5f);       // lower bound, half units
            if (lb > T) continue;
            const int64_t sidx = s0 + c0 + i;  // < N: columns past N carry +inf
            ++emitted;
            const int slot = atomicAdd(cand_n + qs, 1);
            if (slot < D.cap) {
              cand_p[(int64_t)qs * D.cap + slot] = (uint32_t)sidx;
              cand_lb[(int64_t)qs * D.cap + slot] = fmaxf(lb, 0.f);
            } else {
              // the pool counter grows only while the pool has room (it cannot wrap)
              const int pb = *reinterpret_cast<volatile int*>(pool_n) < D.pool_cap ? atomicAdd(pool_n, 1)
                                                                                    : (int)D.pool_cap;
              if (pb < D.pool_cap) {
                pool_q[pb] = qs;
                pool_p[pb] = (uint32_t)sidx;
                pool_lb[pb] = fmaxf(lb, 0.f);
                atomicAdd(qpool_cnt + qs, 1);
              }
            }
            if (d2 < top[KD - 1]) {
              topk_insert<KD>(top, d2);
              const float kth = topk_kth<KD>(top, D.k);
              // k series with d^2 <= d~^2 + M each: a valid threshold
              if (kth < INFINITY) T = fminf(T, __fmul_ru(__fadd_ru(kth, D.margin), D.f_half));
            }
          }
        }
        __syncwarp();
      }
      tc_fence_before();
      mbar_arrive(&tempty[acc]);  // the accumulator is free for the MMA warp
      if (qa && T < T_in) atomicMin(reinterpret_cast<int*>(thr) + q, __float_as_int(T));  // T >= 0
      if (__any_sync(0xFFFFFFFFu, *vfail != 0)) break;
    }
    if (emitted) atomicAdd(counters + 2, emitted);
  }
  // drain: after a timed-out wait, the MMAs and the copies already issued
  // finish (bounded) before the tensor memory is freed and the CTA exits
  __syncthreads();
  if (*vfail) {
    if (warp == 1 && lane == 0) {
      mma_commit(&drain);
      mbar_wait(&drain, 0u);
    }
    if (warp == 0 && lane == 0)
      for (int64_t idx = total > DSTAGES ? total - DSTAGES : 0; idx < total; ++idx)
        mbar_wait(&full[idx % DSTAGES], (uint32_t)((idx / DSTAGES) & 1));
  }
  __syncthreads();
  if (tid == 0) {
    if (*vfail) atomicExch(status, SOFA_ERR_TIMEOUT);
    const int64_t s_hi = t_end * DN < D.N ? t_end * DN : D.N;
    atomicAdd(counters + 11, (unsigned long long)nq_active * (unsigned long long)(s_hi - t_begin * DN));
  }
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, DN * DACC);
  }
}

// The bounded wait itself (a test aid): one warp waits on an mbarrier that
// nothing ever arrives on; the wait gives up after limit_ns and the kernel
// returns normally with SOFA_ERR_TIMEOUT in *status.  Nothing is in flight
// when it gives up (no copy, no MMA, no tensor memory).
__global__ void k_wait_probe(unsigned long long limit_ns, int* __restrict__ status) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const bool ok = mbar_wait(&bar, 0u, limit_ns);
  if (threadIdx.x == 0) *status = ok ? 0 : SOFA_ERR_TIMEOUT;
}

// ------------------------------------------------------------------------
// host side

#define TRYD(x)          \
  do {                   \
    int rc_ = (x);       \
    if (rc_) return rc_; \
  } while (0)

using EncodeTiled = PFN_cuTensorMapEncodeTiled_v12000;

static EncodeTiled encode_fn() {
  static EncodeTiled fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult qr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &qr) ==
            cudaSuccess &&
        qr == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(p);
    cudaGetLastError();
  }
  return fn;
}

int make_tensor_map_2d(CUtensorMap* m, const void* base, int64_t rows, int cols, int elem_bytes, int box_cols,
                       int box_rows, int swizzle_bytes) {
  EncodeTiled fn = encode_fn();
  if (!fn) return fail(SOFA_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)cols * (cuuint64_t)elem_bytes};
  cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  const CUtensorMapDataType dt = elem_bytes == 2 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                 : elem_bytes == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                                   : CU_TENSOR_MAP_DATA_TYPE_UINT8;
  const CUtensorMapSwizzle sw = swizzle_bytes == 128 ? CU_TENSOR_MAP_SWIZZLE_128B
                                : swizzle_bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B
                                : swizzle_bytes == 32 ? CU_TENSOR_MAP_SWIZZLE_32B
                                                      : CU_TENSOR_MAP_SWIZZLE_NONE;
  CUresult r = fn(m, dt, 2, const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(SOFA_ERR_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
  return 0;
}

// 2-d map of a row-major matrix (rows x n) of fp32 or fp16 values, boxes of
// one 128-byte row (32 fp32 or 64 fp16 values) x box_rows, 128-byte swizzle;
// elements outside the matrix read as zero.
static int make_map(CUtensorMap* m, const void* base, int64_t rows, int n, int box_rows, bool f16) {
  EncodeTiled fn = encode_fn();
  if (!fn) return fail(SOFA_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
  const size_t es_bytes = f16 ? 2 : 4;
  cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)n * es_bytes};
  cuuint32_t box[2] = {(cuuint32_t)(128 / es_bytes), (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = fn(m, f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                  const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(SOFA_ERR_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
  return 0;
}

// FP16 operands when the index holds the FP16 copy of its series.
static bool dense_f16(const Index* ix) { return ix->Zh != nullptr; }

bool dense_supported(const Index* ix, int k) {
  // row strides must be multiples of 16 bytes
  return ix->xn && ix->n % (dense_f16(ix) ? 8 : 4) == 0 && k <= DKMAX && ix->N < ((int64_t)1 << 31) - 2 * DN &&
         encode_fn() != nullptr;
}

// |d~^2 - d^2| for canonical series (||x||^2 <= n (1 + 4u)), n' = n (1 + 4u):
// * TF32 operands: relative error < 2^-10 each (truncated or rounded), so
//   |q.x~ - q.x| <= n' (2^-9 + 2^-20 + n 2^-22 (1 + 2^-9));
// * FP16 operands (round to nearest): relative error <= 2^-11 each plus at
//   most 2^-25 absolute for subnormals, so
//   |q.x~ - q.x| <= n' (2^-10 + 2^-22 + 2^-24 + n 2^-22 (1 + 2^-10));
// where n 2^-22 covers an FP32 accumulation whose additions may lose up to 2
// bits against IEEE.  Twice that for -2 q.x, plus the fp32 roundings of
// ||x||^2 and ||q||^2 and of the two fp32 operations forming d~^2 (8.2 u n');
// 1 % on top.
static float dense_margin(int n, bool f16) {
  const double u = std::ldexp(1.0, -24);
  const double np = n * (1.0 + 4 * u);
  const double dot =
      f16 ? np * (std::ldexp(1.0, -10) + std::ldexp(1.0, -22) + std::ldexp(1.0, -24) +
                  n * std::ldexp(1.0, -22) * (1.0 + std::ldexp(1.0, -10)))
          : np * (std::ldexp(1.0, -9) + std::ldexp(1.0, -20) + n * std::ldexp(1.0, -22) * (1.0 + std::ldexp(1.0, -9)));
  return std::nextafter((float)((2.0 * dot + 8.2 * u * np) * 1.01), INFINITY);
}

float dense_margin_of(const Index* ix) { return dense_margin(ix->n, dense_f16(ix)); }

// FP16 copy (round to nearest) of the batch's canonical queries.
__global__ void k_queries_half(const float* __restrict__ zq, int64_t count, __half* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) out[i] = __float2half_rn(zq[i]);
}

// ||q||^2 of each canonical query (FP64 sum rounded to fp32).
__global__ void k_qnorms(const float* __restrict__ zq, int Q, int n, float* __restrict__ out) {
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= Q) return;
  double s = 0.0;
  for (int t = lane; t < n; t += 32) {
    const double z = zq[row * n + t];
    s += z * z;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
  if (lane == 0) out[row] = (float)s;
}

int launch_row_norms(const float* Z, int64_t N, int n, float* xn, cudaStream_t st) {
  if (N <= 0) return 0;
  k_row_norms<<<(unsigned)ceil_div(N * 32, 256), 256, 0, st>>>(Z, N, n, xn);
  SOFA_CUDA(cudaGetLastError());
  return 0;
}

template <int KD, bool F16>
static int launch_dense_t(const CUtensorMap& tq, const CUtensorMap& tx, const DenseParams& D, dim3 grid,
                          const float* qn, const Index* ix, const DenseArgs& A, cudaStream_t st) {
  SOFA_CUDA(cudaFuncSetAttribute(k_dense<KD, F16>, cudaFuncAttributeMaxDynamicSharedMemorySize, DENSE_SMEM));
  k_dense<KD, F16><<<grid, DTHREADS, DENSE_SMEM, st>>>(tq, tx, D, qn, ix->xn, A.qsel, A.qslot, A.thr, A.cand_p,
                                                      A.cand_lb, A.cand_n, A.pool_n, A.pool_q, A.pool_p, A.pool_lb,
                                                      A.qpool_cnt, A.dump, A.counters, A.status);
  SOFA_CUDA(cudaGetLastError());
  return 0;
}

int launch_dense(Index* ix, const DenseArgs& A, cudaStream_t st) {
  const bool f16 = dense_f16(ix);
  CUtensorMap tq, tx;
  if (f16) {
    TRYD(ix->qs.zqh.ensure((size_t)A.Q * ix->n * sizeof(__half)));
    const int64_t cnt = (int64_t)A.Q * ix->n;
    k_queries_half<<<(unsigned)ceil_div(cnt, 256), 256, 0, st>>>(A.zq, cnt, ix->qs.zqh.as<__half>());
    SOFA_CUDA(cudaGetLastError());
    TRYD(make_map(&tq, ix->qs.zqh.p, A.Q, ix->n, DM, true));
    TRYD(make_map(&tx, ix->Zh, ix->N, ix->n, DN, true));
  } else {
    TRYD(make_map(&tq, A.zq, A.Q, ix->n, DM, false));
    TRYD(make_map(&tx, ix->Z, ix->N, ix->n, DN, false));
  }
  TRYD(A.qn_buf->ensure((size_t)A.Q * sizeof(float)));
  float* qn = A.qn_buf->as<float>();
  k_qnorms<<<(unsigned)ceil_div((int64_t)A.Q * 32, 256), 256, 0, st>>>(A.zq, A.Q, ix->n, qn);
  SOFA_CUDA(cudaGetLastError());
  int sms = 0, dev = 0;
  SOFA_CUDA(cudaGetDevice(&dev));
  SOFA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int gx = (int)ceil_div(A.Q, DM);
  const int64_t n_tiles = ceil_div(ix->N, DN);
  // about two waves of one CTA per SM; the query blocks of a chunk are
  // adjacent in launch order, so its series tiles are read once from HBM
  const int64_t chunks = std::max<int64_t>(1, std::min<int64_t>(n_tiles, (2 * sms + gx - 1) / gx));
  DenseParams D;
  D.N = ix->N;
  D.Q = A.Q;
  D.n = ix->n;
  D.k = A.k;
  D.cap = A.cap;
  D.pool_cap = A.pool_cap;
  D.tiles_per_cta = ceil_div(n_tiles, chunks);
  D.margin = dense_margin(ix->n, f16);
  D.f_half = std::nextafter(A.f_prune * 0.5f, INFINITY);
  const dim3 grid((unsigned)gx, (unsigned)ceil_div(n_tiles, D.tiles_per_cta));
  if (A.k == 1) return f16 ? launch_dense_t<1, true>(tq, tx, D, grid, qn, ix, A, st)
                           : launch_dense_t<1, false>(tq, tx, D, grid, qn, ix, A, st);
  return f16 ? launch_dense_t<DKMAX, true>(tq, tx, D, grid, qn, ix, A, st)
             : launch_dense_t<DKMAX, false>(tq, tx, D, grid, qn, ix, A, st);
}

}  // namespace sofa

using namespace sofa;

extern "C" int sofa_wait_selftest(int32_t limit_ms, sofa_stream stream) {
  if (limit_ms < 1 || limit_ms > 2000) return fail(SOFA_ERR_INVALID_ARG, "limit_ms must lie in [1, 2000]");
  cudaStream_t st = (cudaStream_t)stream;
  int* d = nullptr;
  SOFA_CUDA(dev_malloc((void**)&d, sizeof(int)));
  int h = 0;
  k_wait_probe<<<1, 32, 0, st>>>((unsigned long long)limit_ms * 1000000ull, d);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(d);
  if (e != cudaSuccess) return fail(SOFA_ERR_CUDA, std::string("wait self-test: ") + cudaGetErrorString(e));
  if (h == SOFA_ERR_TIMEOUT) return fail(SOFA_ERR_TIMEOUT, "the bounded wait ran out, as the self-test intends");
  return h;
}

extern "C" int sofa_dense_sqdist(sofa_handle h, const float* queries, int64_t Q, float* out, float* margin,
                                 sofa_stream stream) {
  if (!h || !queries || !out) return fail(SOFA_ERR_INVALID_ARG, "null argument");
  if (Q < 1 || Q > 8192) return fail(SOFA_ERR_INVALID_ARG, "Q must lie in [1, 8192]");
  if (Q * h->N > ((int64_t)1 << 31)) return fail(SOFA_ERR_INVALID_ARG, "Q * N must be <= 2^31");
  if (!dense_supported(h, 1))
    return fail(SOFA_ERR_INVALID_ARG, "the dense contraction needs n % 4 == 0 (n % 8 == 0 with FP16 operands)");
  if (!is_device_ptr(queries) || !is_device_ptr(out))
    return fail(SOFA_ERR_INVALID_ARG, "queries and out must be device memory");
  if (int rc = check_device(h)) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  QueryScratch& s = h->qs;
  TRYD(s.zq.ensure((size_t)Q * h->n * sizeof(float)));
  TRYD(s.qv.ensure((size_t)Q * h->NB * sizeof(float)));
  TRYD(s.thr.ensure((size_t)Q * sizeof(float)));
  TRYD(s.counters.ensure(16 * sizeof(unsigned long long)));
  TRYD(launch_qprep(h, queries, Q, s.zq.as<float>(), s.qv.as<float>(), st));
  SOFA_CUDA(cudaMemsetAsync(s.thr.p, 0x7F, (size_t)Q * sizeof(float), st));  // huge thresholds
  DenseArgs A;
  std::memset(&A, 0, sizeof(A));
  A.zq = s.zq.as<float>();
  A.Q = (int)Q;
  A.k = 1;
  A.cap = 1;
  A.f_prune = 1.f;
  A.thr = s.thr.as<float>();
  A.dump = out;
  A.counters = s.counters.as<unsigned long long>();
  A.status = reinterpret_cast<int*>(s.counters.as<unsigned long long>() + 8);
  A.qn_buf = &s.qn;
  TRYD(launch_dense(h, A, st));
  if (margin) *margin = dense_margin(h->n, dense_f16(h));
  return 0;
}
