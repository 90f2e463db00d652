// Series bound on the tensor cores: Eq. (1) restricted to the NB selected
// Fourier values (Sec. IV "SFA", Eq. 1; the lower bound GEMINI prunes with,
// Sec. II-A), evaluated from int8 value codes for every (series, query) pair
// of a work unit's surviving tiles as one tcgen05 contraction per tile.
//
// Each series x of the index holds its selected values v as int8 codes c with
// one scale s (y = s c, exact) and a margin r >= ||v - y||_w + (projection
// error), see k_quantv.  For a query with computed values q~:
//   ||q~ - y||_w^2 = ||q~||_w^2 + s^2 ||c||_w^2 - 2 s (w o q~) . c,
// and ||q - v||_w >= ||q~ - y||_w - r, ||q - v||_w <= ED (Parseval).  The
// dot products (w o q~) . c of a tile's 256 series (rows, M) and a unit's up
// to 64 queries (columns, N) are one MMA of K = NB on the tensor cores: the
// codes are exact in FP16 (|c| <= 127), the query operand w o q~ is rounded to
// FP16, the accumulation is FP32.  A derived margin M' bounds every error of
// that contraction and of the epilogue's FP32 arithmetic (tc_margin below),
// so a pair is pruned only when
//   sqrt(max(e~ - M', 0)) - r > sqrt(2 T)      (T: the query's threshold),
// which implies ED > sqrt(2 T): no series that can reach the first k places
// is pruned.  Leaf blocks and tiles are still pruned by their SFA symbol
// envelopes first, exactly as in the word scan.
#include <cuda.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "bounds.cuh"
#include "sofa_internal.cuh"
#include "tc_ptx.cuh"

namespace sofa {

constexpr int VS_WARPS = 10;             // 8 epilogue warps, 1 TMA producer, 1 MMA issuer
constexpr int VS_THREADS = 32 * VS_WARPS;
constexpr int VS_EPI = 256;              // epilogue threads: one series of the tile each
constexpr int VS_N = 64;                 // queries per MMA (the work unit's capacity)
constexpr int VS_TMEM = 256;             // two accumulators of 2 halves x 64 columns
constexpr int MAX_LEAF_TILES_VS = 256;

template <int NB>
struct VsCfg {
  static constexpr int ROWB = NB * 2;             // bytes of one operand row (64 or 128)
  static constexpr int ATILE = TILE * ROWB;       // codes of one tile (16 KB or 32 KB)
  static constexpr int BTILE = VS_N * ROWB;       // query operand of one unit (4 KB or 8 KB)
  static constexpr int KTILE = TILE * 16;         // folded constants of one tile: 8 FP16 per series
  static constexpr int STAGE = ATILE + KTILE;     // one pipeline stage (multiple of 1024 bytes)
  // staging area of a unit (the queries' SFA values, value-major; up to 64
  // tile envelopes; the intervals of 16 tiles), reused during its tiles as
  // the candidate list (10 bytes an entry)
  static constexpr int SQ_BYTES = VS_N * (NB / 2) * 4;
  static constexpr int ENV_BYTES = 64 * NB;
  static constexpr int IVL_BYTES = 16 * (NB / 2) * 8;
  static constexpr int UNION = SQ_BYTES + ENV_BYTES + IVL_BYTES;
  static constexpr int SC = (UNION / 10 & ~31) < 1024 ? (UNION / 10 & ~31) : 1024;
  static constexpr int STAGES = NB == 32 ? 3 : 2; // TMA pipeline depth (two CTAs per SM at NB = 32)
  static constexpr int MIN_CTAS = NB == 32 ? 2 : 1;
  static constexpr int KSTEPS = NB / 16;          // MMAs of K = 16 per half
};

// Instruction descriptor of tcgen05.mma kind::f16: D fp32 (bits 4-5 = 1), A
// and B f16 (bits 7-9, 10-12 = 0), both K-major, N = 64 (bits 17-22: N >> 3),
// M = 128 (bits 24-28: M >> 4).
__host__ __device__ constexpr uint32_t vscan_idesc() {
  return (1u << 4) | ((uint32_t)(VS_N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

template <int NB>
__device__ __forceinline__ uint64_t vs_desc(uint32_t saddr) {
  if constexpr (NB == 32) return sw64_desc(saddr);
  else return sw128_desc(saddr);
}

// Physical 16-byte chunk of logical chunk c in row r of a K-major operand
// tile with the TMA swizzle of its row size (address bits [4, 4+b) are
// XORed with bits [7, 7+b): b = 2 for 64-byte rows, 3 for 128-byte rows).
template <int NB>
__device__ __forceinline__ int vs_chunk(int r, int c) {
  if constexpr (NB == 32) return c ^ ((r >> 1) & 3);
  else return c ^ (r & 7);
}

__device__ __forceinline__ void mma_f16_n64(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(vscan_idesc()), "r"(accumulate));
}

// One accumulator column of this thread's TMEM lane (load and wait).
__device__ __forceinline__ float tmem_ld1(uint32_t taddr) {
  uint32_t r;
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r)
      : "r"(taddr)
      : "memory");
  return __uint_as_float(r);
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// ------------------------------------------------------------------------
// The folded test.  With D = (w o q~) . c (the MMA over the codes), the pair
// survives iff  -2 s D - 2 r a - c_q <= -S'  (a = sqrt(2 T) of the query,
// c_q = a^2 - ||q~||_w^2, S' = s^2 ||c||_w^2 - r^2 - M'), i.e. after dividing
// by -2 s < 0:
//   y = D + alpha a + beta c_q + phi >= 0,  alpha = r / s, beta = 1 / (2 s),
//   phi = -S' / (2 s).
// The three rank-one terms are one more K = 16 step of the same MMA: the
// series side holds (alpha_h, alpha_h, alpha_l, beta_h, beta_h, beta_l,
// phi_h, phi_l) and the query side (a_h, a_l, a_h, c_h, c_l, c_h, 1, 1),
// each value split into an FP16 high part and an FP16 remainder, so that the
// three products of each term carry its value to about 2^-21 (the low x low
// product is dropped); the K step's other 8 columns are zero on the query
// side.  The epilogue's test is then the sign of y: no per-pair arithmetic.
// A series whose constants do not fit FP16 (scale s near 0) gets
// (0, 0, 0, 0, 0, 0, FP16_MAX, FP16_MAX): y > 0 for every live query, so it
// always survives (and its emitted bound is 0).
constexpr float VK_LIMIT = 30000.f;  // |alpha|, |beta|, |phi| below this fit FP16 with their remainders
constexpr float VK_ALWAYS = 65504.f; // FP16 max: the always-survive constant
constexpr float VK_UNUSED_C = -60000.f;  // c of a query slot past the unit's queries: y < 0

// FP16 high part and remainder of v (v - h is exact in FP32)
__device__ __forceinline__ void split_f16(float v, __half& h, __half& l) {
  h = __float2half_rn(v);
  l = __float2half_rn(v - __half2float(h));
}

// Derived per-series arrays of the tensor-core bound, from the value codes:
// VH[p] = the codes as FP16 (exact); VK[p] = the folded constants above, with
// S = s^2 ||c||_w^2 (FP64, rounded down) and S' = S - r^2 - M' rounded down.
__global__ void k_vcodes_tc(const int8_t* __restrict__ VC, const float2* __restrict__ vsr,
                            const float* __restrict__ vw, int64_t N, int NB, float Mp, __half* __restrict__ VH,
                            uint4* __restrict__ VK) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  double cw = 0.0;
  for (int j = 0; j < NB; ++j) {
    const int c = VC[p * NB + j];
    VH[p * NB + j] = __int2half_rn(c);
    cw += (double)vw[j] * (double)(c * c);
  }
  const float2 sr = vsr[p];
  const double S = (double)sr.x * (double)sr.x * cw;
  const float r2 = __fmul_ru(sr.y, sr.y);
  const float Sp = __fsub_rd(__fsub_rd(__double2float_rd(S), r2), Mp);
  __align__(16) __half h[8];
  bool always = true;
  if (sr.x > 0.f) {
    const float al = __fdiv_rn(sr.y, sr.x), be = __fdiv_rn(0.5f, sr.x), ph = -__fmul_rn(Sp, be);
    always = !(al >= 0.f && al < VK_LIMIT && be >= 0.25f && be < VK_LIMIT && fabsf(ph) < VK_LIMIT);
    if (!always) {
      split_f16(al, h[0], h[2]);
      h[1] = h[0];
      split_f16(be, h[3], h[5]);
      h[4] = h[3];
      split_f16(ph, h[6], h[7]);
    }
  }
  if (always) {
    for (int i = 0; i < 6; ++i) h[i] = __float2half_rn(0.f);
    h[6] = h[7] = __float2half_rn(VK_ALWAYS);
  }
  VK[p] = *reinterpret_cast<const uint4*>(h);
}

// The margin M' >= the error of the folded test, in squared-distance units
// (multiply an error of y by 2 s).  With R = sqrt(n) (1 + 2^-20) + sqrt(W)
// (delta_d + delta_q) >= ||q~||_w, ||v~||_w (Parseval; W <= 2 nsel),
// Y = 1.04 R >= ||y||_w (||v~ - y||_w <= sqrt(W) s / 2, s = max|v~| / 127),
// r <= Y, a <= A = 2.1 R + 1 (larger thresholds are clamped to A, which
// prunes nothing either: sqrt(e) - r <= R + Y < A) and |c_q| <= C =
// max(A^2, R^2):
//  * query operand rounded to FP16: |fl(b) - b| <= 2^-11 |b| (+2^-25 below the
//    normal range), so |2 s (fl(b) - b) . c| <= 2 (2^-11 + 2^-24) Y R
//    + 2 s 127 NB 2^-25;
//  * FP32 accumulation of the NB + 16 products of the MMA, at most 2 ulps
//    (2^-22) of the sum of their magnitudes per product: those magnitudes
//    sum (times 2 s) to at most 2 Y R + 2 Y A + C + 2 Y^2;
//  * the split constants: alpha a to 2^-19 Y A + 2^-23 (Y + 8 A), beta c_q to
//    2^-19 C + 2^-24, phi to 2^-20 (2 Y^2 + 1) + 2^-21 (divisions, products
//    and splits correctly rounded; remainders below the FP16 normal range
//    lose at most 2^-25; s <= 8);
//  * ||q~||_w^2 summed in FP32 over NB terms, S' and c_q:
//    (64 + NB + 1) 2^-24 R^2.
double tc_margin(const Index* ix) {
  const double n = ix->n, W = 2.0 * ix->nsel, NB = ix->NB;
  const double R = std::sqrt(n) * (1.0 + std::ldexp(1.0, -20)) + std::sqrt(W) * (ix->delta_d + ix->delta_q);
  const double Y = 1.04 * R, A = tc_amax(ix), C = std::max(A * A, R * R);
  const double m_tc = 2.0 * (std::ldexp(1.0, -11) + std::ldexp(1.0, -24)) * Y * R +
                      2.0 * (R / 127.0) * 127.0 * NB * std::ldexp(1.0, -25);
  const double m_acc = (NB + 16.0) * std::ldexp(1.0, -22) * (2.0 * Y * R + 2.0 * Y * A + C + 2.0 * Y * Y) *
                       (1.0 + std::ldexp(1.0, -10));
  const double m_split = std::ldexp(1.0, -19) * Y * A + std::ldexp(1.0, -23) * (Y + 8.0 * A) +
                         std::ldexp(1.0, -19) * C + std::ldexp(1.0, -24) +
                         std::ldexp(1.0, -20) * (2.0 * Y * Y + 1.0) + std::ldexp(1.0, -21);
  const double m_ep = (64.0 + NB + 1) * std::ldexp(1.0, -24) * R * R;
  return (m_tc + m_acc + m_split + m_ep) * 1.01;
}

// Threshold clamp A = 2.1 R + 1 (R as in tc_margin).
double tc_amax(const Index* ix) {
  const double n = ix->n, W = 2.0 * ix->nsel;
  const double R = std::sqrt(n) * (1.0 + std::ldexp(1.0, -20)) + std::sqrt(W) * (ix->delta_d + ix->delta_q);
  return 2.1 * R + 1.0;
}

// The folded test needs C = max(A^2, R^2) and |D| <= 127 sqrt(W) R to stay
// well inside FP16 (c_q) and below the always-survive offset 2 FP16_MAX.
static bool tc_fits(const Index* ix) {
  const double n = ix->n, W = 2.0 * ix->nsel;
  const double R = std::sqrt(n) * (1.0 + std::ldexp(1.0, -20)) + std::sqrt(W) * (ix->delta_d + ix->delta_q);
  const double A = tc_amax(ix);
  return std::max(A * A, R * R) < 30000.0 && 127.0 * std::sqrt(W) * R * 1.01 < 2.0 * 65504.0 - 1.0;
}

int make_tc_codes(Index* ix, cudaStream_t st) {
  if (!ix->VC || !ix->vsr || !ix->vw) return 0;
  release_tc_codes(ix);
  if (!tc_fits(ix)) return 0;  // the folded test's constants would not fit FP16: no tensor-core bound
  const size_t hb = (size_t)ix->N * ix->NB * sizeof(__half), xb = (size_t)ix->N * sizeof(uint4);
  if (dev_malloc((void**)&ix->VH, hb) != cudaSuccess || dev_malloc((void**)&ix->VK, xb) != cudaSuccess) {
    cudaGetLastError();
    release_tc_codes(ix);
    return fail(SOFA_ERR_OOM, "allocation of the tensor-core value codes failed");
  }
  ix->tc_bytes = (int64_t)(hb + xb);
  ix->device_bytes += ix->tc_bytes;
  ix->tc_margin = (float)tc_margin(ix);
  ix->tc_amax = (float)tc_amax(ix);
  k_vcodes_tc<<<(unsigned)ceil_div(ix->N, 256), 256, 0, st>>>(ix->VC, ix->vsr, ix->vw, ix->N, ix->NB,
                                                               ix->tc_margin, ix->VH, ix->VK);
  SOFA_CUDA(cudaGetLastError());
  return 0;
}

void release_tc_codes(Index* ix) {
  if (ix->VH) cudaFree(ix->VH);
  if (ix->VK) cudaFree(ix->VK);
  ix->VH = nullptr;
  ix->VK = nullptr;
  ix->device_bytes -= ix->tc_bytes;
  ix->tc_bytes = 0;
}

// ------------------------------------------------------------------------
// The tensor-core series scan.  A persistent CTA takes work units (leaf
// block, up to 64 queries).  All warps first stage the unit: the queries'
// SFA values (for the tile envelope checks), their FP16 operand w o q~ in the
// swizzled layout the MMA reads, their folded-test operand (a, c_q split) and
// a = min(sqrt(2 T) rounded up, A); then the tile envelope checks give each
// tile its mask of live queries (as in the word scan) and a list of live
// tiles.  Then: warp 8 streams the live tiles' FP16 codes and folded
// constants by TMA into a ring of stages; warp 9 issues per tile 2 halves x
// (NB/16 + 1) MMAs (M = 128 series, N = 64 queries, K = 16) into one of two
// TMEM accumulators; warps 0-7 (thread i = series i of the tile) read the
// accumulator rows, take the maximum of y over the columns (three-input max,
// no other arithmetic), and only where some y >= 0 walk the surviving
// columns, computing each survivor's lower bound and appending it to the
// unit's candidate list in shared memory; at the end of the unit the list
// goes to the candidate store with one global reservation per query.  Every wait is bounded; a
// wait that runs out stops all roles, lets issued copies and MMAs finish,
// and sets SOFA_ERR_TIMEOUT.  With `dump` the kernel instead writes every
// pair's lower bound (Q x N, original order) and emits nothing.

// No-swizzle K-major shared-memory descriptor: core matrices of 8 rows x 16
// bytes, `lbo` bytes apart along K and `sbo` bytes apart along M (or N),
// descriptor version 1, layout type 0.
__device__ __forceinline__ uint64_t nosw_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

__device__ __forceinline__ float fmax3(float a, float b, float c) {
  float d;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}

// 2 x 32 consecutive fp32 columns of this thread's TMEM lane, one wait.
__device__ __forceinline__ void tmem_ld32x2(uint32_t t0, uint32_t t1, float* v) {
  uint32_t r[64];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%64];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, "
      "%45, %46, %47, %48, %49, %50, %51, %52, %53, %54, %55, %56, %57, %58, %59, %60, %61, %62, %63}, [%65];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]),
        "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]),
        "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]),
        "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]),
        "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
      : "r"(t0), "r"(t1)
      : "memory");
#pragma unroll
  for (int i = 0; i < 64; ++i) v[i] = __uint_as_float(r[i]);
}

// The squared lower bound of a pair from its folded-test value y, the
// query's a and the series' constants (k).  Algebra: with the true s and r,
// (a + r)^2 - 2 s y = ||q~||_w^2 + S - 2 s D - M' - (the test's errors) <=
// ||q~ - y||_w^2 = e, since M' covers those errors.  Here s and r come from
// the split constants (s^ = 1 / (2 beta~), r^ = alpha~ s^, each within
// 2^-18 relative (+2^-25 s absolute) of the true values); mu covers that and
// the FP32 rounding of (a + r^)^2 - 2 s^ y, and r is rounded up before the
// square root's difference, so the result is <= (sqrt(e) - r)^2 when
// sqrt(e) >= r, and 0 otherwise.  A series with the always-survive
// constants (beta~ = 0) gets 0.
__device__ __forceinline__ float folded_lb2(float y, float a, uint4 k) {
  const __half2 k0 = *reinterpret_cast<const __half2*>(&k.x);  // (alpha_h, alpha_h)
  const __half2 k1 = *reinterpret_cast<const __half2*>(&k.y);  // (alpha_l, beta_h)
  const __half2 k2 = *reinterpret_cast<const __half2*>(&k.z);  // (beta_h, beta_l)
  const float be = __half2float(__low2half(k2)) + __half2float(__high2half(k2));  // exact in FP32
  if (!(be > 0.f)) return 0.f;
  const float al = __half2float(__low2half(k0)) + __half2float(__low2half(k1));
  const float s_ = __fdiv_rn(0.5f, be);
  const float r_ = al * s_;
  const float ar = a + r_;
  const float A2 = ar * ar;
  const float Y2 = 2.0f * s_ * y;
  const float mu = __fmul_ru(__fadd_ru(__fadd_ru(A2, fabsf(Y2)), 1.0f), 0x1.0p-15f);
  const float el = __fsub_rd(__fsub_rd(A2, Y2), mu);
  const float r_up = __fadd_ru(__fmul_ru(r_, 1.0f + 0x1.0p-17f), 0x1.0p-24f);
  const float m = fmaxf(__fsub_rd(__fsqrt_rd(fmaxf(el, 0.f)), r_up), 0.f);
  return __fmul_rd(m, m);
}

template <int NB, bool NYQ>
__global__ void __launch_bounds__(VS_THREADS, VsCfg<NB>::MIN_CTAS)
    k_vscan(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmK, int64_t N, int64_t T,
            int n_leaf_tiles, int NBq, const int4* __restrict__ units, const int* __restrict__ n_units_ptr,
            const int* __restrict__ leaf_q, const float* __restrict__ qv, const float* __restrict__ thr,
            const uint8_t* __restrict__ tenv, const float2* __restrict__ ch, const uint4* __restrict__ VK,
            const float* __restrict__ vw, float amax, int tile_checks, int cap, const int* __restrict__ qslot,
            uint32_t* __restrict__ cand_p, float* __restrict__ cand_lb, int* __restrict__ cand_n, int64_t pool_cap,
            int* __restrict__ pool_n, int* __restrict__ pool_q, uint32_t* __restrict__ pool_p,
            float* __restrict__ pool_lb, int* __restrict__ qpool_cnt, float* __restrict__ dump, int64_t dumpQ,
            const uint32_t* __restrict__ perm, unsigned long long* __restrict__ counters, int* __restrict__ status) {
  constexpr int LW = NB / 2;
  using C = VsCfg<NB>;
  extern __shared__ __align__(16) uint8_t vsm[];
  float2* sch = reinterpret_cast<float2*>(vsm);  // LW x 256 (tile checks)
  const uint32_t raw = smem_u32(vsm);
  const uint32_t tab_end = raw + (uint32_t)(LW * MAX_ALPHA * sizeof(float2));
  // [tables | pad to 1024 | folded-test operand of the unit: 64 x 16 B, then
  // 1 KB of zeros | stages (1024-byte aligned swizzle atoms) | code operand]
  uint8_t* sBK = vsm + (((tab_end + 1023u) & ~1023u) - raw);
  uint8_t* stages = sBK + 2048;
  uint8_t* sB = stages + C::STAGES * C::STAGE;  // the unit's code operand (swizzled)
  __shared__ __align__(8) uint64_t full[C::STAGES], empty[C::STAGES], tfull[4], tempty[4], drain;
  __shared__ uint16_t s_off[MAX_LEAF_TILES_VS + 1];
  __shared__ uint16_t stl[MAX_LEAF_TILES_VS];
  // staging: sqT (the queries' SFA values, value-major), s_env (64 tile
  // envelopes) and s_ivl (the intervals of 16 tiles); during the tiles: the
  // candidate list (positions, bounds, query slot << 10 | rank in its query)
  __shared__ __align__(16) uint8_t s_union[C::UNION];
  float(*sqT)[VS_N] = reinterpret_cast<float(*)[VS_N]>(s_union);
  uint8_t* s_env = s_union + C::SQ_BYTES;
  float2* s_ivl = reinterpret_cast<float2*>(s_union + C::SQ_BYTES + C::ENV_BYTES);
  uint32_t* s_cp = reinterpret_cast<uint32_t*>(s_union);
  float* s_cl = reinterpret_cast<float*>(s_union + 4 * C::SC);
  uint16_t* s_cgr = reinterpret_cast<uint16_t*>(s_union + 8 * C::SC);
  __shared__ int s_qn[VS_N], s_qbase[VS_N], s_qpbase[VS_N];
  __shared__ int s_cn, s_clim;
  __shared__ float sT[VS_N], sA[VS_N];
  __shared__ int sslot[VS_N], sqid[VS_N];
  __shared__ unsigned long long smask[MAX_LEAF_TILES_VS];
  __shared__ uint32_t s_tmem;
  __shared__ int s_fail, s_ntl;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  volatile int* vfail = &s_fail;
  for (int e = tid; e < LW * MAX_ALPHA; e += blockDim.x) sch[e] = ch[e];
  // the zero half (K columns 8-15) of the folded-test operand, written once
  for (int e = tid; e < 1024 / 16; e += blockDim.x) reinterpret_cast<uint4*>(sBK + 1024)[e] = make_uint4(0, 0, 0, 0);
  if (warp == 9) tmem_alloc(&s_tmem, VS_TMEM);
  if (tid == 0) {
    for (int s = 0; s < C::STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    // one pair of barriers per (accumulator, 128-series half): each half is
    // read by its own four epilogue warps
    for (int a = 0; a < 4; ++a) {
      mbar_init(&tfull[a], 1);
      mbar_init(&tempty[a], VS_EPI / 2);
    }
    mbar_init(&drain, 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  unsigned long long n_tile_pairs = 0, n_cand = 0, n_loads = 0, n_checks = 0;
  long long gi = 0;  // running index of this CTA's live tiles (the same in every role)
  const int n_units = *n_units_ptr;
  for (int u = blockIdx.x; u < n_units; u += gridDim.x) {
    __syncthreads();
    if (*vfail) break;  // read after the barrier: the same verdict in every thread
    const int4 un = units[u];
    const int64_t b = un.x;
    const int cnt = un.z;
    const int64_t t0 = b * n_leaf_tiles;
    const int nt = (int)((T - t0) < n_leaf_tiles ? (T - t0) : n_leaf_tiles);
    // ---- stage the unit's queries: CH threads per query slot, 8 values each
    // (two 16-byte loads after the query's id); the FP16 operand w o q~ in
    // the swizzled layout, the SFA values for the envelope checks, ||q~||_w^2
    // (FP32, partial sums over the CH threads; its rounding is part of M'),
    // and the folded-test operand (a_h, a_l, a_h, c_h, c_l, c_h, 1, 1) with
    // a = min(sqrt(2 T) rounded up, A) and c_q = a^2 - ||q~||_w^2 rounded up;
    // a slot past the unit's queries gets a = 0, c = -60000 and -1's, which
    // make y negative for every series
    constexpr int CH = NB / 8;  // 16-byte chunks of an operand row
    if (tid < VS_N) s_qn[tid] = 0;
    if (tid == 0) {
      s_cn = 0;
      s_clim = C::SC;
    }
    for (int e = tid; e < VS_N * CH; e += blockDim.x) {  // whole warps: VS_N * CH is a multiple of 32
      const int g = e / CH, c = e - g * CH;
      float v[8];
      float T_ = 0.f;
      int qq = 0, qs = 0;
      if (g < cnt) {
        qq = leaf_q[un.y + g];
        const float4* src = reinterpret_cast<const float4*>(qv + (int64_t)qq * NBq + 8 * c);
        const float4 v0 = src[0], v1 = src[1];
        v[0] = v0.x, v[1] = v0.y, v[2] = v0.z, v[3] = v0.w, v[4] = v1.x, v[5] = v1.y, v[6] = v1.z, v[7] = v1.w;
        if (c == 0) {
          T_ = dump ? 0.f : thr[qq];
          qs = qslot ? qslot[qq] : qq;
        }
      } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = 0.f;
      }
      __align__(16) __half hv[8];
      float part = 0.f;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const float wv = __ldg(vw + 8 * c + i) * v[i];
        hv[i] = __float2half_rn(wv);
        part = fmaf(wv, v[i], part);
      }
      *reinterpret_cast<uint4*>(sB + g * C::ROWB + vs_chunk<NB>(g, c) * 16) = *reinterpret_cast<const uint4*>(hv);
      if (8 * c < LW) {
#pragma unroll
        for (int i = 0; i < 8; ++i) sqT[8 * c + i][g] = v[i];
      }
#pragma unroll
      for (int o = 1; o < CH; o <<= 1) part += __shfl_xor_sync(0xFFFFFFFFu, part, o);
      if (c == 0) {
        __align__(16) __half hk[8];
        if (g < cnt) {
          const float a = fminf(__fsqrt_ru(__fmul_ru(2.0f, T_)), amax);
          const float cq = __fsub_ru(__fmul_ru(a, a), part);
          sA[g] = a;
          sT[g] = T_;
          sqid[g] = qq;
          sslot[g] = qs;
          split_f16(a, hk[0], hk[1]);
          hk[2] = hk[0];
          split_f16(cq, hk[3], hk[4]);
          hk[5] = hk[3];
          hk[6] = hk[7] = __float2half_rn(1.0f);
        } else {
          hk[0] = hk[1] = hk[2] = hk[4] = __float2half_rn(0.f);
          hk[3] = hk[5] = __float2half_rn(VK_UNUSED_C);
          hk[6] = hk[7] = __float2half_rn(-1.0f);
          sA[g] = 0.f;
        }
        *reinterpret_cast<uint4*>(sBK + 16 * g) = *reinterpret_cast<const uint4*>(hk);
      }
    }
    for (int t = tid; t < nt; t += blockDim.x) smask[t] = 0ull;
    fence_proxy_async();  // the operands' generic stores, before the MMAs read them
    // ---- tile envelope checks (with tile_checks; otherwise, and when
    // dumping, every tile is live for every query of the unit).  The envelopes of
    // up to 64 tiles are staged by one coalesced pass; then, 16 tiles at a
    // time, each tile's LW intervals [c(lo) - h(lo), c(hi) + h(hi)] (rounded
    // outward) are formed once, and a warp checks one tile against 32 query
    // slots (lane = slot; interval reads are broadcasts, the values are
    // stored value-major): the bound of env_bound_ch, term for term.
    if (dump || !tile_checks) {
      __syncthreads();
      const unsigned long long all = cnt >= 64 ? ~0ull : ((1ull << cnt) - 1ull);
      for (int t = tid; t < nt; t += blockDim.x) smask[t] = all;
    } else {
      const int npass = (cnt + 31) >> 5;
      for (int tb0 = 0; tb0 < nt; tb0 += 64) {
        const int nc = nt - tb0 < 64 ? nt - tb0 : 64;
        constexpr int EV = 2 * LW / 16;  // 16-byte pieces of one tile's envelope
        const uint4* src = reinterpret_cast<const uint4*>(tenv + (t0 + tb0) * 2 * LW);
        for (int e = tid; e < nc * EV; e += blockDim.x) reinterpret_cast<uint4*>(s_env)[e] = src[e];
        __syncthreads();
        for (int cb = 0; cb < nc; cb += 16) {
          const int nk = nc - cb < 16 ? nc - cb : 16;
          for (int e = tid; e < nk * LW; e += blockDim.x) {
            const int t = e / LW, j = e - t * LW;
            const uint8_t* env = s_env + (cb + t) * 2 * LW;
            const float2 vl = sch[j * MAX_ALPHA + env[j]], vh = sch[j * MAX_ALPHA + env[LW + j]];
            s_ivl[e] = make_float2(__fsub_rd(vl.x, vl.y), __fadd_ru(vh.x, vh.y));
          }
          __syncthreads();
          for (int w = warp; w < nk * npass; w += VS_WARPS) {
            const int t = w / npass, g0 = (w - t * npass) << 5, g = g0 + lane;
            const int gg = g < cnt ? g : 0;
            float acc = 0.f;
#pragma unroll
            for (int j = 0; j < LW; ++j) {
              const float2 iv = s_ivl[t * LW + j];
              const float qj = sqT[j][gg];
              const float m = fmaxf(fmaxf(iv.x - qj, qj - iv.y), 0.f);
              const float mm = (NYQ && j == 0) ? 0.5f * m : m;
              acc = fmaf(mm, m, acc);
            }
            const unsigned live = __ballot_sync(0xFFFFFFFFu, g < cnt && acc <= sT[gg]);
            if (lane == 0 && live) atomicOr(&smask[tb0 + cb + t], (unsigned long long)live << g0);
          }
          __syncthreads();
        }
      }
      n_checks += (tid == 0) ? (unsigned long long)nt : 0ull;
    }
    __syncthreads();
    if (tid < 32) {  // exclusive scan of the per-tile counts; the live tiles in order
      int run = 0, nl = 0;
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
        const unsigned live = __ballot_sync(0xFFFFFFFFu, c > 0);
        if (c > 0) stl[nl + __popc(live & ((1u << lane) - 1u))] = (uint16_t)t;
        nl += __popc(live);
      }
      if (lane == 0) {
        s_off[nt] = (uint16_t)run;
        s_ntl = nl;
      }
    }
    __syncthreads();
    const int ntl = s_ntl;
    if (warp == 8) {
      if (lane == 0) {  // TMA producer: codes and folded constants of each live tile
        for (int i = 0; i < ntl; ++i) {
          const long long g_ = gi + i;
          const int s = (int)(g_ % C::STAGES);
          if (g_ >= C::STAGES && !mbar_wait(&empty[s], (uint32_t)(((g_ / C::STAGES) - 1) & 1))) {
            *vfail = 1;
            break;
          }
          if (*vfail) break;
          const int row = (int)((t0 + stl[i]) * TILE);
          mbar_expect_tx(&full[s], C::ATILE + C::KTILE);
          tma_load_2d(stages + s * C::STAGE, &tmA, 0, row, &full[s]);
          tma_load_2d(stages + s * C::STAGE + C::ATILE, &tmK, 0, row, &full[s]);
        }
      }
    } else if (warp == 9) {
      if (lane == 0) {  // MMA issuer
        const uint32_t sb = smem_u32(sB), sbk = smem_u32(sBK);
        for (int i = 0; i < ntl; ++i) {
          const long long g_ = gi + i;
          const int s = (int)(g_ % C::STAGES), acc = (int)(g_ & 1);
          if (!mbar_wait(&full[s], (uint32_t)((g_ / C::STAGES) & 1))) {
            *vfail = 1;
            break;
          }
          const uint32_t sa = smem_u32(stages + s * C::STAGE), sk = sa + C::ATILE;
          bool ok = true;
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            // this half of the accumulator is free once its four warps released it
            if (g_ >= 2 && !mbar_wait(&tempty[acc * 2 + h], (uint32_t)(((g_ >> 1) - 1) & 1))) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t d = tmem + (uint32_t)(acc * 128 + h * 64);
#pragma unroll
            for (int kk = 0; kk < C::KSTEPS; ++kk)
              mma_f16_n64(d, vs_desc<NB>(sa + h * 128 * C::ROWB) + 2 * kk, vs_desc<NB>(sb) + 2 * kk, kk > 0 ? 1u : 0u);
            // the folded constants: the series side's K columns 8-15 repeat
            // columns 0-7 (LBO 0; the query side is zero there)
            mma_f16_n64(d, nosw_desc(sk + h * 128 * 16, 0, 128), nosw_desc(sbk, 1024, 128), 1u);
            mma_commit(&tfull[acc * 2 + h]);
          }
          if (!ok) {
            *vfail = 1;
            break;
          }
          mma_commit(&empty[s]);
        }
      }
    } else {
      // epilogue: thread tid = series tid of the tile; TMEM lanes of its warp's
      // quadrant, columns of its half
      const int half = warp >> 2;
      const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
      for (int i = 0; i < ntl; ++i) {
        const long long g_ = gi + i;
        const int acc = (int)(g_ & 1);
        const int t = stl[i];
        const int o0 = s_off[t], o1 = s_off[t + 1];
        const int64_t p = (t0 + t) * TILE + tid;
        const bool valid = p < N;
        // the series' folded constants (for the bounds of its survivors; the
        // tile's TMA copy brought the line into L2), loaded before the wait.
        // The address is clamped rather than the value selected, so nothing
        // waits for the load before a survivor needs it (a lane past N is
        // never a survivor).
        const uint4 kx = __ldg(VK + (valid ? p : (int64_t)0));
        if (!__all_sync(0xFFFFFFFFu, mbar_wait(&tfull[acc * 2 + half], (uint32_t)((g_ >> 1) & 1)))) {
          *vfail = 1;
          break;
        }
        tc_fence_after();
        const uint32_t tb = tmem + lane_base + (uint32_t)(acc * 128 + half * 64);
        if (tid == 0) {
          n_tile_pairs += (unsigned long long)(o1 - o0);
          n_loads += 1;
        }
        const unsigned long long tmask = smask[t];
        if (dump) {  // every live pair's bound, 32 columns at a time
#pragma unroll 1
          for (int h32 = 0; h32 < 2; ++h32) {
            float w[32];
            tmem_ld32(tb + (uint32_t)(32 * h32), w);  // warp-collective
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              const int g = 32 * h32 + j;
              if (((tmask >> g) & 1ull) && valid) dump[(int64_t)sqid[g] * N + perm[p]] = folded_lb2(w[j], sA[g], kx);
            }
          }
        }
        float mx[2];  // the lane's maximum of y over each 32 columns
        {
          float v[64];
          tmem_ld32x2(tb, tb + 32u, v);  // warp-collective
#pragma unroll
          for (int h32 = 0; h32 < 2; ++h32) {
            const float* w = v + 32 * h32;
            float c0 = fmax3(w[0], w[1], w[2]), c1 = fmax3(w[3], w[4], w[5]);
            float c2 = fmax3(w[6], w[7], w[8]), c3 = fmax3(w[9], w[10], w[11]);
            c0 = fmax3(c0, w[12], w[13]);
            c1 = fmax3(c1, w[14], w[15]);
            c2 = fmax3(c2, w[16], w[17]);
            c3 = fmax3(c3, w[18], w[19]);
            c0 = fmax3(c0, w[20], w[21]);
            c1 = fmax3(c1, w[22], w[23]);
            c2 = fmax3(c2, w[24], w[25]);
            c3 = fmax3(c3, w[26], w[27]);
            c0 = fmax3(c0, w[28], w[29]);
            c1 = fmax3(c1, w[30], w[31]);
            mx[h32] = fmax3(c0, c1, fmaxf(c2, c3));
          }
        }
        // a series survives a query iff its y >= 0: a lane whose maxima are
        // negative is done with the tile
#pragma unroll
        for (int h32 = 0; h32 < 2; ++h32) {
          const uint32_t m = (uint32_t)(tmask >> (32 * h32));
          const bool maybe = !dump && valid && m != 0u && mx[h32] >= 0.f;
          if (!__any_sync(0xFFFFFFFFu, maybe)) continue;
          // rare: this lane's surviving columns of the half (its 32 columns
          // reloaded), then a walk over the columns where some lane survives
          uint32_t mine = 0u;
          {
            float w[32];
            tmem_ld32(tb + (uint32_t)(32 * h32), w);  // warp-collective
            if (maybe) {
#pragma unroll
              for (int j = 0; j < 32; ++j) mine |= (w[j] >= 0.f ? 1u : 0u) << j;
              mine &= m;
            }
          }
          uint32_t any = __reduce_or_sync(0xFFFFFFFFu, mine);
          while (any) {
            const int j = __ffs(any) - 1;
            any &= any - 1u;
            const int g = 32 * h32 + j;
            const bool live = (mine >> j) & 1u;
            const unsigned hit = __ballot_sync(0xFFFFFFFFu, live);
            const float yg = tmem_ld1(tb + (uint32_t)g);  // warp-collective
            // the pair's lower bound in half units, rounded down
            const float acc_lb = live ? __fmul_rd(folded_lb2(yg, sA[g], kx), 0.5f) : 0.f;
            const int npop = __popc(hit);
            const int rank = __popc(hit & ((1u << lane) - 1u));
            // into the unit's candidate list (shared-memory atomics only);
            // a column that does not fit goes straight to the global store
            int lb0 = 0, rb0 = -1;
            if (lane == 0) {
              lb0 = atomicAdd(&s_cn, npop);
              if (lb0 + npop <= C::SC) rb0 = atomicAdd(&s_qn[g], npop);
              else atomicMin(&s_clim, lb0);
            }
            lb0 = __shfl_sync(0xFFFFFFFFu, lb0, 0);
            rb0 = __shfl_sync(0xFFFFFFFFu, rb0, 0);
            if (rb0 >= 0) {
              if (live) {
                s_cp[lb0 + rank] = (uint32_t)p;
                s_cl[lb0 + rank] = acc_lb;
                s_cgr[lb0 + rank] = (uint16_t)((g << 10) | (rb0 + rank));
              }
            } else {
              const int qs = sslot[g];
              int base = 0, pbase = 0;
              if (lane == 0) base = atomicAdd(cand_n + qs, npop);
              base = __shfl_sync(0xFFFFFFFFu, base, 0);
              const int over0 = base > cap ? base : cap;
              const int nover = base + npop - over0;
              if (lane == 0 && nover > 0) {
                // the pool counter grows only while the pool has room (it cannot wrap)
                pbase = *reinterpret_cast<volatile int*>(pool_n) < pool_cap ? atomicAdd(pool_n, nover) : (int)pool_cap;
                const int64_t room = pool_cap - pbase;
                const int written = room <= 0 ? 0 : (room < nover ? (int)room : nover);
                if (written > 0) atomicAdd(qpool_cnt + qs, written);
              }
              pbase = __shfl_sync(0xFFFFFFFFu, pbase, 0);
              if (live) {
                const int slot = base + rank;
                if (slot < cap) {
                  cand_p[(int64_t)qs * cap + slot] = (uint32_t)p;
                  cand_lb[(int64_t)qs * cap + slot] = acc_lb;
                } else {
                  const int64_t pi = (int64_t)pbase + (slot - over0);
                  if (pi < pool_cap) {
                    pool_q[pi] = qs;
                    pool_p[pi] = (uint32_t)p;
                    pool_lb[pi] = acc_lb;
                  }
                }
              }
            }
            if (lane == 0) n_cand += (unsigned long long)npop;
          }
        }
        tc_fence_before();
        mbar_arrive(&tempty[acc * 2 + half]);  // this half of the accumulator is free for the MMA warp
      }
      // flush the unit's candidate list: one global reservation per query
      // (and one pool reservation per query that overflows its slots), then
      // every entry to its slot; the epilogue warps only (named barrier 1)
      asm volatile("bar.sync 1, %0;" ::"n"(VS_EPI) : "memory");
      if (tid < VS_N) {
        const int cnt_g = s_qn[tid];
        int base = 0, pbase = 0;
        if (cnt_g > 0) {
          const int qs = sslot[tid];
          base = atomicAdd(cand_n + qs, cnt_g);
          const int over0 = base > cap ? base : cap;
          const int nover = base + cnt_g - over0;
          if (nover > 0) {
            pbase = *reinterpret_cast<volatile int*>(pool_n) < pool_cap ? atomicAdd(pool_n, nover) : (int)pool_cap;
            const int64_t room = pool_cap - pbase;
            const int written = room <= 0 ? 0 : (room < nover ? (int)room : nover);
            if (written > 0) atomicAdd(qpool_cnt + qs, written);
          }
        }
        s_qbase[tid] = base;
        s_qpbase[tid] = pbase;
      }
      asm volatile("bar.sync 1, %0;" ::"n"(VS_EPI) : "memory");
      // entries below the first reservation that did not fit are all written
      const int ncl = s_cn < s_clim ? s_cn : s_clim;
      for (int i = tid; i < ncl; i += VS_EPI) {
        const int g = s_cgr[i] >> 10, slot = s_qbase[g] + (s_cgr[i] & 1023);
        const int qs = sslot[g];
        if (slot < cap) {
          cand_p[(int64_t)qs * cap + slot] = s_cp[i];
          cand_lb[(int64_t)qs * cap + slot] = s_cl[i];
        } else {
          const int over0 = s_qbase[g] > cap ? s_qbase[g] : cap;
          const int64_t pi = (int64_t)s_qpbase[g] + (slot - over0);
          if (pi < pool_cap) {
            pool_q[pi] = qs;
            pool_p[pi] = s_cp[i];
            pool_lb[pi] = s_cl[i];
          }
        }
      }
    }
    gi += ntl;
  }
  // drain: the MMA warp's issued MMAs and the producer's issued copies finish
  // before the tensor memory is freed and the CTA exits (they always have on
  // the normal path; after a timed-out wait this waits for them, bounded)
  __syncthreads();
  if (warp == 9 && lane == 0) {
    mma_commit(&drain);
    if (!mbar_wait(&drain, 0u)) *vfail = 1;
  }
  if (warp == 8 && lane == 0 && *vfail) {
    for (long long g_ = gi > C::STAGES ? gi - C::STAGES : 0; g_ < gi; ++g_)
      mbar_wait(&full[g_ % C::STAGES], (uint32_t)((g_ / C::STAGES) & 1));
  }
  __syncthreads();
  if (warp == 9) {
    tc_fence_after();
    tmem_dealloc(tmem, VS_TMEM);
  }
  if (tid == 0 && *vfail) atomicExch(status, SOFA_ERR_TIMEOUT);
  if (n_tile_pairs) atomicAdd(counters + 1, n_tile_pairs);
  if (n_cand) atomicAdd(counters + 2, n_cand);
  if (n_loads) atomicAdd(counters + 4, n_loads);
  if (n_checks) atomicAdd(counters + 5, n_checks);
}

// ------------------------------------------------------------------------
// host side

static size_t vscan_smem(const Index* ix) {
  const int LW = ix->LW;
  const size_t tab = (size_t)LW * MAX_ALPHA * sizeof(float2);
  const size_t stage = ix->NB == 32 ? (size_t)VsCfg<32>::STAGES * VsCfg<32>::STAGE + VsCfg<32>::BTILE
                                    : (size_t)VsCfg<64>::STAGES * VsCfg<64>::STAGE + VsCfg<64>::BTILE;
  return tab + 1024 + stage + 2048;  // + the folded-test operand (1 KB) and its zero half (1 KB)
}

bool vscan_supported(const Index* ix) {
  return ix->VH && ix->VK && (ix->NB == 32 || ix->NB == 64) && ix->leaf_tiles <= MAX_LEAF_TILES_VS &&
         ix->group <= VS_N;
}

template <int NB, bool NYQ>
static int launch_vscan_t(Index* ix, const VscanArgs& A, cudaStream_t st) {
  CUtensorMap tm, tk;
  if (int rc = make_tensor_map_2d(&tm, ix->VH, ix->N, NB, 2, NB, TILE, NB == 32 ? 64 : 128)) return rc;
  if (int rc = make_tensor_map_2d(&tk, ix->VK, ix->N, 8, 2, 8, TILE, 0)) return rc;  // 16-byte rows, no swizzle
  const size_t smem = vscan_smem(ix);
  auto fn = k_vscan<NB, NYQ>;
  SOFA_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  // all of the SM's unified memory as shared memory, so that two CTAs fit
  SOFA_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared));
  int sms = 0, dev = 0, smem_sm = 0, regs_sm = 0;
  SOFA_CUDA(cudaGetDevice(&dev));
  SOFA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  SOFA_CUDA(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
  SOFA_CUDA(cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev));
  cudaFuncAttributes fa;
  SOFA_CUDA(cudaFuncGetAttributes(&fa, fn));
  // resident CTAs per SM from the kernel's own resources: shared memory
  // (dynamic + static + the 1 KB the system reserves per CTA), registers
  // (allocated per warp in units of 256), and the tensor memory (each CTA
  // holds VS_TMEM of the SM's 512 columns for its lifetime)
  const int64_t smem_cta = (int64_t)smem + fa.sharedSizeBytes + 1024;
  const int64_t regs_cta = (int64_t)VS_WARPS * (((int64_t)fa.numRegs * 32 + 255) / 256 * 256);
  int per_sm = (int)std::min<int64_t>(smem_sm / smem_cta, regs_sm / std::max<int64_t>(1, regs_cta));
  per_sm = std::max(1, std::min(per_sm, 512 / VS_TMEM));
  const int grid = sms * per_sm;
  fn<<<grid, VS_THREADS, smem, st>>>(tm, tk, ix->N, ix->T, ix->leaf_tiles, ix->NB, A.units, A.n_units, A.leaf_q,
                                     A.qv, A.thr, ix->tenv, ix->ch, ix->VK, ix->vw, ix->tc_amax, ix->tile_checks,
                                     A.cap, A.qslot,
                                     A.cand_p, A.cand_lb,
                                     A.cand_n, A.pool_cap, A.pool_n, A.pool_q, A.pool_p, A.pool_lb, A.qpool_cnt,
                                     A.dump, A.dumpQ, ix->perm, A.counters, A.status);
  SOFA_CUDA(cudaGetLastError());
  return 0;
}

int launch_vscan(Index* ix, const VscanArgs& A, cudaStream_t st) {
  if (!vscan_supported(ix)) return fail(SOFA_ERR_INVALID_ARG, "the tensor-core bound needs the value codes");
  if (ix->NB == 32)
    return ix->nyq_first ? launch_vscan_t<32, true>(ix, A, st) : launch_vscan_t<32, false>(ix, A, st);
  return ix->nyq_first ? launch_vscan_t<64, true>(ix, A, st) : launch_vscan_t<64, false>(ix, A, st);
}

}  // namespace sofa

using namespace sofa;

// Every pair's tensor-core lower bound (see sofa.h): the scan kernel in its
// dump mode over units that pair every leaf block with every query (all
// tiles live, no envelope checks).
extern "C" int sofa_value_bounds(sofa_handle h, const float* queries, int64_t Q, float* out, float* margin,
                                 sofa_stream stream) {
  if (!h || !queries || !out) return fail(SOFA_ERR_INVALID_ARG, "null argument");
  if (Q < 1 || Q * h->N > ((int64_t)1 << 31)) return fail(SOFA_ERR_INVALID_ARG, "need 1 <= Q and Q * N <= 2^31");
  if (!vscan_supported(h)) return fail(SOFA_ERR_INVALID_ARG, "the tensor-core bound needs an index with precision >= 1");
  if (!is_device_ptr(queries) || !is_device_ptr(out))
    return fail(SOFA_ERR_INVALID_ARG, "queries and out must be device memory");
  if (int rc = check_device(h)) return rc;
  Index* ix = h;
  cudaStream_t st = (cudaStream_t)stream;
  QueryScratch& s = ix->qs;
  if (int rc = s.zq.ensure((size_t)Q * ix->n * sizeof(float))) return rc;
  if (int rc = s.qv.ensure((size_t)Q * ix->NB * sizeof(float))) return rc;
  if (int rc = s.counters.ensure(16 * sizeof(unsigned long long))) return rc;
  if (int rc = launch_qprep(ix, queries, Q, s.zq.as<float>(), s.qv.as<float>(), st)) return rc;
  std::vector<int4> units;
  std::vector<int> lq((size_t)ix->L * Q);
  for (int64_t b = 0; b < ix->L; ++b) {
    for (int64_t i = 0; i < Q; ++i) lq[(size_t)(b * Q + i)] = (int)i;
    for (int64_t g0 = 0; g0 < Q; g0 += VS_N)
      units.push_back(make_int4((int)b, (int)(b * Q + g0), (int)std::min<int64_t>(VS_N, Q - g0), 0));
  }
  DevBuf du, dl, dn;
  if (int rc = du.ensure(units.size() * sizeof(int4))) return rc;
  if (int rc = dl.ensure(lq.size() * sizeof(int))) return rc;
  if (int rc = dn.ensure(sizeof(int))) return rc;
  const int nu = (int)units.size();
  SOFA_CUDA(cudaMemcpyAsync(du.p, units.data(), units.size() * sizeof(int4), cudaMemcpyHostToDevice, st));
  SOFA_CUDA(cudaMemcpyAsync(dl.p, lq.data(), lq.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  SOFA_CUDA(cudaMemcpyAsync(dn.p, &nu, sizeof(int), cudaMemcpyHostToDevice, st));
  VscanArgs V;
  std::memset(&V, 0, sizeof(V));
  V.units = du.as<int4>();
  V.n_units = dn.as<int>();
  V.leaf_q = dl.as<int>();
  V.qv = s.qv.as<float>();
  V.cap = 1;
  V.dump = out;
  V.dumpQ = Q;
  V.counters = s.counters.as<unsigned long long>();
  V.status = reinterpret_cast<int*>(s.counters.as<unsigned long long>() + 8);
  int rc = launch_vscan(ix, V, st);
  if (!rc) rc = cudaStreamSynchronize(st) == cudaSuccess ? 0 : fail(SOFA_ERR_CUDA, "sofa_value_bounds failed");
  du.release();
  dl.release();
  dn.release();
  if (margin) *margin = ix->tc_margin;
  return rc;
}
