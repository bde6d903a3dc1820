// Shared pieces of the fused multiply-divide update of one MM half step
// (Section 3.1, Eqs. (3.3)-(3.4)): shared-memory tile strides and the store
// of a new factor value into the operand plane(s) the next product streams.
//
// Tile space: rows m of a tile are rows of W (left update, p rows) or
// columns of H (right update, n columns); columns k are the r factor ranks.
// In both cases the update of entry (m, k) is
//     new[m,k] = old[m,k] * num[m,k] / (sum_l old[m,l] G[l,k] + eps)
// where num is the V-streaming product (V H^T or (W^T V)^T) and G the r x r
// Gram matrix of the *other* factor (H H^T or W^T W): the paper's
// V_n W_n W_n^t (resp. V^t V W_n) grouped through the Gram matrix.
// Multiplication and division are IEEE round-to-nearest (no fast math).
#pragma once

#include "nmf_internal.cuh"

namespace nmf {

// Row stride of the epilogue's shared tile Ns (numerator, then new factor):
// 16-byte aligned rows for vector access.
template <int RPAD> __host__ __device__ constexpr int epi_ldn() { return RPAD + 4; }

__device__ __forceinline__ void store_plane(const EpiArgs& e, int k, int64_t m, float v) {
  const int64_t off = (int64_t)k * e.ldop + m;
  if (e.plane == kPlaneF32) {
    static_cast<float*>(e.op_hi)[off] = v;
  } else if (e.plane == kPlaneTF32) {
    static_cast<float*>(e.op_hi)[off] = round_tf32(v);
  } else {
    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
    static_cast<__nv_bfloat16*>(e.op_hi)[off] = hi;
    if (e.plane == kPlaneBF16x2) {
      const float rem = __fsub_rn(v, __bfloat162float(hi));
      static_cast<__nv_bfloat16*>(e.op_lo)[off] = __float2bfloat16_rn(rem);
    }
  }
}

// Entries (k, m0 .. m0+n8-1) of the [k][m]-ordered outputs of an update --
// the operand plane(s) and, for a column-major factor (H), the factor itself
// -- from v[0 .. n8-1]: one 16-byte store per plane (two for float32 planes)
// when all 8 entries exist and the address is aligned, else element stores.
__device__ __forceinline__ void store_col8(const EpiArgs& e, int k, int64_t m0, int n8,
                                           const float* v) {
  const bool full = n8 == 8;
  auto aligned = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
  if (e.layout != kFactorRowMajor) {
    float* f = e.F + (int64_t)k * e.ldf + m0;
    if (full && aligned(f)) {
      reinterpret_cast<float4*>(f)[0] = make_float4(v[0], v[1], v[2], v[3]);
      reinterpret_cast<float4*>(f)[1] = make_float4(v[4], v[5], v[6], v[7]);
    } else {
      for (int t = 0; t < n8; ++t) f[t] = v[t];
    }
  }
  const int64_t off = (int64_t)k * e.ldop + m0;
  if (e.plane == kPlaneF32 || e.plane == kPlaneTF32) {
    float w[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) w[t] = e.plane == kPlaneTF32 ? round_tf32(v[t]) : v[t];
    float* p = static_cast<float*>(e.op_hi) + off;
    if (full && aligned(p)) {
      reinterpret_cast<float4*>(p)[0] = make_float4(w[0], w[1], w[2], w[3]);
      reinterpret_cast<float4*>(p)[1] = make_float4(w[4], w[5], w[6], w[7]);
    } else {
      for (int t = 0; t < n8; ++t) p[t] = w[t];
    }
  } else {
    __align__(16) __nv_bfloat16 hi[8];
    __align__(16) __nv_bfloat16 lo[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      hi[t] = __float2bfloat16_rn(v[t]);
      lo[t] = __float2bfloat16_rn(__fsub_rn(v[t], __bfloat162float(hi[t])));
    }
    __nv_bfloat16* ph = static_cast<__nv_bfloat16*>(e.op_hi) + off;
    __nv_bfloat16* pl = e.plane == kPlaneBF16x2 ? static_cast<__nv_bfloat16*>(e.op_lo) + off
                                                : nullptr;
    if (full && aligned(ph) && (!pl || aligned(pl))) {
      *reinterpret_cast<uint4*>(ph) = *reinterpret_cast<const uint4*>(hi);
      if (pl) *reinterpret_cast<uint4*>(pl) = *reinterpret_cast<const uint4*>(lo);
    } else {
      for (int t = 0; t < n8; ++t) {
        ph[t] = hi[t];
        if (pl) pl[t] = lo[t];
      }
    }
  }
}

}  // namespace nmf
