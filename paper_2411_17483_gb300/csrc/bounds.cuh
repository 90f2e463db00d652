// SFA envelope bounds (leaf blocks and tiles of the flat layout), shared by
// the series scans.  Bounds are in half units: acc = sum_j c_j m_j^2 with
// c_j = 1, or 1/2 for a Nyquist value (always word position 0), so that
// LB^2 = 2 acc matches Eq. 1's weights; m_j is Eq. dist_i against the symbol
// interval widened by the projection error margins.
#pragma once

#include "sofa_internal.cuh"

namespace sofa {

// Envelope bound (leaf block or tile): per value j the interval spanned by
// symbols lo_j..hi_j, i.e. [edge(lo_j).lo, edge(hi_j).hi].
template <int LW, bool NYQ>
__device__ __forceinline__ float env_bound(const uint8_t* __restrict__ env, const float* q,
                                           const float2* __restrict__ edge) {
  const uint32_t* e32 = reinterpret_cast<const uint32_t*>(env);
  float acc = 0.f;
#pragma unroll
  for (int w = 0; w < LW / 4; ++w) {
    uint32_t lo = e32[w], hi = e32[LW / 4 + w];
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int j = 4 * w + b;
      float elo = edge[j * MAX_ALPHA + ((lo >> (8 * b)) & 0xFFu)].x;
      float ehi = edge[j * MAX_ALPHA + ((hi >> (8 * b)) & 0xFFu)].y;
      float m = fmaxf(fmaxf(elo - q[j], q[j] - ehi), 0.f);
      float mm = (NYQ && j == 0) ? 0.5f * m : m;
      acc = fmaf(mm, m, acc);
    }
  }
  return acc;
}

// Envelope bound from the (centre, half-width) table: the interval of
// symbols lo_j..hi_j is contained in [c(lo) - h(lo), c(hi) + h(hi)], both ends
// rounded outward (a hair looser than the edge table, never tighter).
template <int LW, bool NYQ>
__device__ __forceinline__ float env_bound_ch(const uint8_t* __restrict__ env, const float* q,
                                              const float2* __restrict__ chs) {
  const uint32_t* e32 = reinterpret_cast<const uint32_t*>(env);
  float acc = 0.f;
#pragma unroll
  for (int w = 0; w < LW / 4; ++w) {
    uint32_t lo = e32[w], hi = e32[LW / 4 + w];
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int j = 4 * w + b;
      const float2 vl = chs[j * MAX_ALPHA + ((lo >> (8 * b)) & 0xFFu)];
      const float2 vh = chs[j * MAX_ALPHA + ((hi >> (8 * b)) & 0xFFu)];
      const float elo = __fsub_rd(vl.x, vl.y), ehi = __fadd_ru(vh.x, vh.y);
      float m = fmaxf(fmaxf(elo - q[j], q[j] - ehi), 0.f);
      float mm = (NYQ && j == 0) ? 0.5f * m : m;
      acc = fmaf(mm, m, acc);
    }
  }
  return acc;
}

}  // namespace sofa
