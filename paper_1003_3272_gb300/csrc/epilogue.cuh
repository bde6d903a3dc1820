// Fused multiply-divide epilogue of one MM half step (Section 3.1,
// Eqs. (3.3)-(3.4)), run by the block that owns a finished output tile.
//
// Tile space: rows m of the tile are rows of W (left update, p rows) or
// columns of H (right update, n columns); columns k are the r factor ranks.
// In both cases the update of entry (m, k) is
//     new[m,k] = old[m,k] * num[m,k] / (sum_l old[m,l] G[l,k] + eps)
// where num is the V-streaming product (V H^T or (W^T V)^T) and G the r x r
// Gram matrix of the *other* factor (H H^T or W^T W).  The denominator is
// the paper's V_n W_n W_n^t (resp. V^t V W_n) grouped through the Gram
// matrix.  Multiplication and division are IEEE round-to-nearest (no fast
// math), matching (old * num) / den.
//
// The block then writes the new factor (user storage and the operand
// plane(s) the next product streams) and the tile's partial Gram matrix
// sum_m new[m,:]^T new[m,:], summed over m in a fixed order.
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

// Multiply-divide update of an R-row slice of a tile whose first row is
// global row `row0` (rows beyond e.M are ignored).
// Ns: [R][RPAD+4] holds the final numerator slice on entry and the new
//     factor slice on exit.
// Os: [R][RPAD+1] scratch for the old factor slice.
// Gs: [RPAD][RPAD] scratch, filled here from e.G (the other factor's Gram,
//     read through L2: it may have been written earlier in the same launch).
// P : r x r destination of the slice's partial Gram of the new factor.
// Both products in here -- the denominators old . G and the partial Gram
// new^T new -- are register-blocked so that each thread keeps 16-32
// independent accumulators (the block has few warps to hide latency with).
// All NT threads of the block must call it.
template <int RPAD, int NT>
__device__ void mu_epilogue(float* Ns, float* Os, float* Gs, int R, int64_t row0, float* P,
                            const EpiArgs& e) {
  constexpr int LDN = epi_ldn<RPAD>();
  constexpr int LDO = epi_ldo<RPAD>();
  const int tid = threadIdx.x;
  const int r = e.r;
  const int64_t M = e.M;
  const int rows = (int)((M - row0) < R ? (M - row0 > 0 ? M - row0 : 0) : R);

  // Loads are issued eight at a time before any use, so a thread waits for
  // one memory round trip per eight values instead of one per value.
  for (int b = tid; b < RPAD * RPAD; b += 8 * NT) {
    float v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int i = b + j * NT;
      const int l = i / RPAD, k = i % RPAD;
      v[j] = (i < RPAD * RPAD && l < r && k < r) ? __ldcg(e.G + l * r + k) : 0.f;
    }
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if (b + j * NT < RPAD * RPAD) Gs[b + j * NT] = v[j];
  }
  if (e.layout == kFactorRowMajor) {
    for (int b = tid; b < R * RPAD; b += 8 * NT) {
      float v[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int i = b + j * NT;
        const int m = i / RPAD, k = i % RPAD;
        v[j] = (i < R * RPAD && m < rows && k < r) ? e.F[(row0 + m) * r + k] : 0.f;
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int i = b + j * NT;
        if (i < R * RPAD) Os[(i / RPAD) * LDO + (i % RPAD)] = v[j];
      }
    }
  } else {
    for (int b = tid; b < R * RPAD; b += 8 * NT) {
      float v[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int i = b + j * NT;
        const int k = i / R, m = i % R;
        v[j] = (i < R * RPAD && m < rows && k < r) ? e.F[(int64_t)k * e.ldf + row0 + m] : 0.f;
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int i = b + j * NT;
        if (i < R * RPAD) Os[(i % R) * LDO + (i / R)] = v[j];
      }
    }
  }
  __syncthreads();

  // ---- den = old . G + eps; new = old * num / den ---------------------------
  // Thread (kg, mg): ranks kg*8 .. kg*8+7, rows mg, mg + MG, ... (4 at a time).
  {
    constexpr int KG = RPAD / 8;
    constexpr int MG = NT / KG;
    const int kg = tid % KG, mg = tid / KG;
    for (int mb = mg; mb < R && tid < KG * MG; mb += 4 * MG) {
      float acc[4][8];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
      int mrow[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) mrow[i] = min(mb + i * MG, R - 1);
#pragma unroll 2
      for (int l = 0; l < r; ++l) {
        const float4 g0 = *reinterpret_cast<const float4*>(&Gs[l * RPAD + kg * 8]);
        const float4 g1 = *reinterpret_cast<const float4*>(&Gs[l * RPAD + kg * 8 + 4]);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float o = Os[mrow[i] * LDO + l];
          acc[i][0] = fmaf(o, g0.x, acc[i][0]); acc[i][1] = fmaf(o, g0.y, acc[i][1]);
          acc[i][2] = fmaf(o, g0.z, acc[i][2]); acc[i][3] = fmaf(o, g0.w, acc[i][3]);
          acc[i][4] = fmaf(o, g1.x, acc[i][4]); acc[i][5] = fmaf(o, g1.y, acc[i][5]);
          acc[i][6] = fmaf(o, g1.z, acc[i][6]); acc[i][7] = fmaf(o, g1.w, acc[i][7]);
        }
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int m = mb + i * MG;
        if (m >= R) continue;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int k = kg * 8 + j;
          float v = 0.f;
          if (m < rows && k < r) {
            const float d = __fadd_rn(acc[i][j], e.eps);
            v = __fdiv_rn(__fmul_rn(Os[m * LDO + k], Ns[m * LDN + k]), d);
          }
          Ns[m * LDN + k] = v;
        }
      }
    }
  }
  __syncthreads();

  // Write the new factor and its operand plane(s).
  if (e.layout == kFactorRowMajor) {
    for (int i = tid; i < rows * r; i += NT) {
      const int m = i / r, k = i % r;
      e.F[(row0 + m) * r + k] = Ns[m * LDN + k];
    }
  } else {
    for (int i = tid; i < rows * r; i += NT) {
      const int k = i / rows, m = i % rows;
      e.F[(int64_t)k * e.ldf + row0 + m] = Ns[m * LDN + k];
    }
  }
  for (int i = tid; i < rows * r; i += NT) {
    const int k = i / rows, m = i % rows;
    store_plane(e, k, row0 + m, Ns[m * LDN + k]);
  }

  // ---- partial Gram of the new slice: P = new^T new (rows >= `rows` are 0) --
  // 4 x 4 blocks (kb <= lb) of the r x r result, one or more per thread,
  // rows summed in order 0..R-1.
  {
    constexpr int NB = RPAD / 4;
    const int nbr = (r + 3) / 4;
    const int npairs = nbr * (nbr + 1) / 2;
    for (int it = tid; it < npairs; it += NT) {
      int kb = 0, rem = it;
      while (rem >= nbr - kb) { rem -= nbr - kb; ++kb; }
      const int lb = kb + rem;
      float acc[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
#pragma unroll 4
      for (int m = 0; m < R; ++m) {
        const float4 a = *reinterpret_cast<const float4*>(&Ns[m * LDN + kb * 4]);
        const float4 b = *reinterpret_cast<const float4*>(&Ns[m * LDN + lb * 4]);
        const float av[4] = {a.x, a.y, a.z, a.w};
        const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
      }
      (void)NB;
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int k = kb * 4 + i, l = lb * 4 + j;
          if (k < r && l < r) {
            P[k * r + l] = acc[i][j];
            P[l * r + k] = acc[i][j];
          }
        }
    }
  }
}

}  // namespace nmf
