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

// Row strides of the epilogue's shared tiles: Ns (numerator, then new
// factor) keeps 16-byte aligned rows for the Gram's vector loads; Os (old
// factor) uses an odd stride so that column reads are bank-conflict free.
template <int RPAD> __host__ __device__ constexpr int epi_ldn() { return RPAD + 4; }
template <int RPAD> __host__ __device__ constexpr int epi_ldo() { return RPAD + 1; }

// Shared-memory floats needed by mu_epilogue for an R x RPAD slice.
template <int RPAD>
__host__ __device__ constexpr int epi_smem_floats(int R) {
  return R * epi_ldn<RPAD>() + R * epi_ldo<RPAD>() + RPAD * RPAD;
}

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

}  // namespace nmf
