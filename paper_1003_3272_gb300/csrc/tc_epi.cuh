// Helper-warp work of the tensor-core half step (k_stream_tc.cu).
//
// While warps 0-1 stream V through the tensor cores, warps 2-7 (192 "helper"
// threads, synchronised among themselves with named barrier 1) do all the
// work of the multiply-divide update that does not depend on this launch's
// product:
//   * the r x r Gram matrix G of the *other* factor Q (W^T W for the H update,
//     H H^T for the W update): each block sums an even share of Q's rows
//     (float32 within 128-row windows, float64 across them), then each block
//     adds up a share of the r^2 entries over all blocks' partials in float64
//     in a fixed order (two grid-wide publication points);
//   * for each output tile, the old rows of the factor being updated and the
//     denominators  den[m,k] = sum_l old[m,l] G[l,k]  (the paper's V_n W_n
//     W_n^t, resp. V^t V W_n, grouped through G; Section 3.1).
// After the product lands, the helpers put the denominators into shared
// memory and the whole block, while it sums the cluster's partial tiles,
// forms  new[m,k] = old[m,k] * num[m,k] / (den[m,k] + eps),  then writes the
// factor and its operand plane(s).
#pragma once

#include <cooperative_groups.h>

#include <type_traits>

#include "epilogue.cuh"
#include "tc_ptx.cuh"

namespace nmf {
namespace tcepi {

constexpr int kHelpers = 192;     // warps 2-7
constexpr int kHelperBase = 64;   // first helper thread
constexpr int kRmax = 64;         // rows of a tile slice (cluster size >= 2)
constexpr int kQsRows = 32;       // staging rows

template <int RPAD> __host__ __device__ constexpr int ldq() { return RPAD + 4; }
template <int RPAD> __host__ __device__ constexpr int ldo() { return RPAD + 1; }

// Floats of the helpers' dedicated shared memory: staging Qs and old rows Os.
// (The denominators stay in the helpers' registers until the stream ends.)
template <int RPAD>
__host__ __device__ constexpr int dedicated_floats() {
  return kQsRows * ldq<RPAD>() + kRmax * ldo<RPAD>();
}

// Denominators of one helper thread: ranks kg*8 .. kg*8+7 of up to 8 rows
// mg, mg + MG, ... of the slice (thread h: kg = h % KG, mg = h / KG).
template <int RPAD, int NH = kHelpers>
struct DenTile {
  static constexpr int KG = RPAD / 8;
  static constexpr int MG = NH / KG;
  static constexpr int NA = (kRmax + 4 * MG - 1) / (4 * MG);   // passes of 4 rows
  float d[NA][4][8];
  // Threads that hold no denominators call this at the end of their own
  // work, so that the registers are not live across it.
  __device__ __forceinline__ void clear() {
#pragma unroll
    for (int a = 0; a < NA; ++a)
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) d[a][i][j] = 0.f;
  }
};

// Denominators for ranks above 64: one 8 x 8 block per helper thread, rows
// mg*8 .. mg*8+7 and ranks kg*8 .. kg*8+7 (thread h: kg = h % KG, mg = h / KG),
// so that each rank of G read from shared memory feeds 8 rows.
template <int RPAD, int NH = kHelpers>
struct DenTile8 {
  static constexpr int KG = RPAD / 8;
  static constexpr int MG = kRmax / 8;
  static_assert(KG * MG <= NH, "one 8 x 8 block per helper");
  float d[8][8];
  __device__ __forceinline__ void clear() {
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) d[i][j] = 0.f;
  }
};

template <int RPAD, int NH = kHelpers>
using DenFor = typename std::conditional<(RPAD > 64), DenTile8<RPAD, NH>, DenTile<RPAD, NH>>::type;

// new = (old * num) / (den + eps) for 8 entries at once: the quick
// correctly rounded divisions first (independent, so they overlap), then the
// IEEE division for any entry outside the quick form's range.
template <int N = 8>
__device__ __forceinline__ void update8(const float* old, const float* num, const float* den,
                                        float eps, float* v) {
  float x[N], d[N];
  bool slow = false;
#pragma unroll
  for (int j = 0; j < N; ++j) {
    x[j] = __fmul_rn(old[j], num[j]);
    d[j] = __fadd_rn(den[j], eps);
    slow |= !div_rn_quick_ok(x[j], d[j]);
    v[j] = div_rn_quick(x[j], d[j]);
  }
  if (slow) {
#pragma unroll
    for (int j = 0; j < N; ++j)
      if (!div_rn_quick_ok(x[j], d[j])) v[j] = __fdiv_rn(x[j], d[j]);
  }
}

template <int NH = kHelpers>
__device__ __forceinline__ void helper_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(NH) : "memory");
}

// The helpers' denominators into Ds[m][k] (stride ldd = RPAD + 4), once
// the stream is over (the ring's shared memory is free then).
template <int RPAD> __host__ __device__ constexpr int ldd();
template <int RPAD, int NH = kHelpers>
__device__ void den_to_smem(const DenTile<RPAD, NH>& den, float* Ds, int R, int h) {
  constexpr int KG = DenTile<RPAD, NH>::KG;
  constexpr int MG = DenTile<RPAD, NH>::MG;
  constexpr int NA = DenTile<RPAD, NH>::NA;
  constexpr int LD = ldd<RPAD>();
  if (h < 0 || h >= KG * MG) return;
  const int kg = h % KG, mg = h / KG;
#pragma unroll
  for (int a = 0; a < NA; ++a)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int m = mg + (4 * a + i) * MG;
      if (m < R) {
        *reinterpret_cast<float4*>(&Ds[m * LD + kg * 8]) =
            make_float4(den.d[a][i][0], den.d[a][i][1], den.d[a][i][2], den.d[a][i][3]);
        *reinterpret_cast<float4*>(&Ds[m * LD + kg * 8 + 4]) =
            make_float4(den.d[a][i][4], den.d[a][i][5], den.d[a][i][6], den.d[a][i][7]);
      }
    }
}
template <int RPAD, int NH = kHelpers>
__device__ void den_to_smem(const DenTile8<RPAD, NH>& den, float* Ds, int R, int h) {
  constexpr int KG = DenTile8<RPAD, NH>::KG;
  constexpr int MG = DenTile8<RPAD, NH>::MG;
  constexpr int LD = ldd<RPAD>();
  if (h < 0 || h >= KG * MG) return;
  const int kg = h % KG, mg = h / KG;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int m = mg * 8 + i;
    if (m < R) {
      *reinterpret_cast<float4*>(&Ds[m * LD + kg * 8]) =
          make_float4(den.d[i][0], den.d[i][1], den.d[i][2], den.d[i][3]);
      *reinterpret_cast<float4*>(&Ds[m * LD + kg * 8 + 4]) =
          make_float4(den.d[i][4], den.d[i][5], den.d[i][6], den.d[i][7]);
    }
  }
}

// The cluster reduction fused with pass 1 of the update: each thread sums
// four ranks of one row over the S partial tiles (rank order), and at once
// forms new = (old * num) / (den + eps) from Os and Ds, writing the new
// values to Ns (for pass 2) and, for a row-major factor (W), to the factor.
template <int S, int RPAD, int NT>
__device__ void cluster_update_s(const float* Acc, float* Ns, const float* Os, const float* Ds,
                                 const EpiArgs& e, int q, int64_t row0, int rows) {
  constexpr int R = 128 / S;
  constexpr int NQ = RPAD / 4;
  constexpr int TOT = R * NQ;
  constexpr int J = (TOT + NT - 1) / NT;
  constexpr int JC = (8 / S) < 1 ? 1 : (8 / S);   // at most 8 loads in flight
  constexpr int LDA = RPAD + 4;
  constexpr int LN = epi_ldn<RPAD>();
  constexpr int LO = ldo<RPAD>();
  constexpr int LD = ldd<RPAD>();
  const int r = e.r;
#pragma unroll 1
  for (int j0 = 0; j0 < J; j0 += JC) {
    float4 v[JC][S];
#pragma unroll
    for (int j = 0; j < JC; ++j) {
      const int i = threadIdx.x + (j0 + j) * NT;
      if (j0 + j < J && i < TOT) {
        const int m = i / NQ, k4 = (i - m * NQ) * 4;
        const float* mine = &Acc[(q * R + m) * LDA + k4];
        const uint32_t sa = ptx::smem_u32(mine);
        // this block's own partial from its shared memory, the peers' over
        // distributed shared memory
#pragma unroll
        for (int s = 0; s < S; ++s)
          v[j][s] = s == q ? *reinterpret_cast<const float4*>(mine)
                           : ptx::ld_dsmem_v4(ptx::mapa(sa, (uint32_t)s));
      }
    }
#pragma unroll
    for (int j = 0; j < JC; ++j) {
      const int i = threadIdx.x + (j0 + j) * NT;
      if (j0 + j < J && i < TOT) {
        const int m = i / NQ, k4 = (i - m * NQ) * 4;
        float4 sum = v[j][0];
#pragma unroll
        for (int s = 1; s < S; ++s) {
          sum.x += v[j][s].x; sum.y += v[j][s].y; sum.z += v[j][s].z; sum.w += v[j][s].w;
        }
        const float nu[4] = {sum.x, sum.y, sum.z, sum.w};
        float o[4], nv[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) o[t] = Os[m * LO + k4 + t];
        const float4 dn = *reinterpret_cast<const float4*>(&Ds[m * LD + k4]);
        const float dv[4] = {dn.x, dn.y, dn.z, dn.w};
        update8<4>(o, nu, dv, e.eps, nv);
#pragma unroll
        for (int t = 0; t < 4; ++t)
          if (k4 + t >= r) nv[t] = 0.f;
        *reinterpret_cast<float4*>(&Ns[m * LN + k4]) = make_float4(nv[0], nv[1], nv[2], nv[3]);
        if (e.layout == kFactorRowMajor && m < rows) {
#pragma unroll
          for (int t = 0; t < 4; ++t)
            if (k4 + t < r) e.F[(row0 + m) * r + k4 + t] = nv[t];
        }
      }
    }
  }
}

template <int RPAD, int NT>
__device__ void cluster_update(int S, const float* Acc, float* Ns, const float* Os,
                               const float* Ds, const EpiArgs& e, int q, int64_t row0,
                               int rows) {
  if (S == 2) cluster_update_s<2, RPAD, NT>(Acc, Ns, Os, Ds, e, q, row0, rows);
  else if (S == 4) cluster_update_s<4, RPAD, NT>(Acc, Ns, Os, Ds, e, q, row0, rows);
  else cluster_update_s<8, RPAD, NT>(Acc, Ns, Os, Ds, e, q, row0, rows);
}

// Pass 2 of an update: the [k][m]-ordered outputs (planes, and H itself) of
// the slice's new values Ns[m][k], 8 consecutive rows per thread and step.
template <int RPAD, int NT>
__device__ void store_cols(const float* Ns, const EpiArgs& e, int64_t row0, int rows) {
  constexpr int LN = epi_ldn<RPAD>();
  const int ng = (rows + 7) >> 3;
  for (int i = threadIdx.x; i < e.r * ng; i += NT) {
    const int k = i / ng, m0 = (i - k * ng) * 8;
    const int n8 = min(8, rows - m0);
    float v[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) v[t] = t < n8 ? Ns[(m0 + t) * LN + k] : 0.f;
    store_col8(e, k, row0 + m0, n8, v);
  }
}

// Values of rows [m0, m0 + nrows) (nrows <= kQsRows) of a factor, in the
// order they land in Qs[row][k] (zero for k >= r and rows beyond nrows):
// each thread owns up to SV values and issues all their loads at once.
// layout 0: F[m * ldf + k];  layout 1: F[k * ldf + m].
template <int RPAD, int NH = kHelpers>
struct RowStage {
  static constexpr int N = kQsRows * RPAD;
  static constexpr int SV = (N + NH - 1) / NH;
  float v[SV];
  __device__ __forceinline__ void load(const float* F, int layout, int64_t ldf, int r,
                                       int64_t m0, int nrows, int h) {
#pragma unroll
    for (int j = 0; j < SV; ++j) {
      const int i = h + j * NH;
      int row, k;
      if (layout == 0) { row = i / RPAD; k = i % RPAD; }
      else             { k = i / kQsRows; row = i % kQsRows; }
      v[j] = (i < N && row < nrows && k < r)
                 ? (layout == 0 ? F[(m0 + row) * ldf + k] : F[(int64_t)k * ldf + m0 + row])
                 : 0.f;
    }
  }
  __device__ __forceinline__ void store(float* Qs, int layout, int h) const {
    constexpr int LQ = ldq<RPAD>();
#pragma unroll
    for (int j = 0; j < SV; ++j) {
      const int i = h + j * NH;
      if (i < N) {
        int row, k;
        if (layout == 0) { row = i / RPAD; k = i % RPAD; }
        else             { k = i / kQsRows; row = i % kQsRows; }
        Qs[row * LQ + k] = v[j];
      }
    }
  }
};

// Partial Gram of rows [q0, q1) of Q, written to gpart (r x r doubles, both
// triangles): float32 sums over windows of 128 rows, float64 across
// windows.  Each thread owns one 4 x 4 block (kb <= lb) per pass over the
// rows (passes until every block is done); rows are staged 32 at a time,
// the next 32 loaded into registers while the current ones are multiplied.
template <int RPAD, int NH = kHelpers>
__device__ void gram_rows4(float* Qs, const float* Q, int layout, int64_t ldq_g, int64_t q0,
                           int64_t q1, int r, double* gpart, int h) {
  constexpr int LQ = ldq<RPAD>();
  const int nbr = (r + 3) / 4;
  const int npairs = nbr * (nbr + 1) / 2;
  for (int pb = 0; pb < npairs; pb += NH) {
    const int it = pb + h;
    const bool mine = it < npairs;
    int kb = 0, rem = mine ? it : 0;
    while (rem >= nbr - kb) { rem -= nbr - kb; ++kb; }
    const int lb = kb + rem;
    float acc[4][4];
    double tot[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) { acc[i][j] = 0.f; tot[i][j] = 0.0; }
    RowStage<RPAD, NH> st;
    if (q0 < q1) st.load(Q, layout, ldq_g, r, q0, (int)min((int64_t)kQsRows, q1 - q0), h);
    int in_window = 0;
    for (int64_t s0 = q0; s0 < q1; s0 += kQsRows) {
      helper_sync<NH>();          // previous rows consumed
      st.store(Qs, layout, h);
      helper_sync<NH>();
      const int64_t s1 = s0 + kQsRows;
      if (s1 < q1) st.load(Q, layout, ldq_g, r, s1, (int)min((int64_t)kQsRows, q1 - s1), h);
      if (mine) {
#pragma unroll 4
        for (int m = 0; m < kQsRows; ++m) {
          const float4 a = *reinterpret_cast<const float4*>(&Qs[m * LQ + kb * 4]);
          const float4 b = *reinterpret_cast<const float4*>(&Qs[m * LQ + lb * 4]);
          const float av[4] = {a.x, a.y, a.z, a.w};
          const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
      }
      in_window += kQsRows;
      if (in_window == 128 || s1 >= q1) {   // fold the window into float64
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) { tot[i][j] += (double)acc[i][j]; acc[i][j] = 0.f; }
        in_window = 0;
      }
    }
    if (mine) {
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int k = kb * 4 + i, l = lb * 4 + j;
          if (k < r && l < r) {
            gpart[k * r + l] = tot[i][j];
            gpart[l * r + k] = tot[i][j];
          }
        }
    }
    helper_sync<NH>();            // Qs free for the next pass
  }
}

// The same partial Gram with one 8 x 8 block per thread (kb <= lb) in a
// single pass, for ranks whose 4 x 4 blocks would need several passes: four
// 16-byte loads per 64 FMAs.  The float64 window sums accumulate in the
// thread's own entries of gpart (read-modify-write by that thread only), so
// they take no registers.  Needs (ceil(r/8) (ceil(r/8) + 1) / 2) <= NH.
template <int RPAD, int NH = kHelpers>
__device__ void gram_rows8(float* Qs, const float* Q, int layout, int64_t ldq_g, int64_t q0,
                           int64_t q1, int r, double* gpart, int h) {
  constexpr int LQ = ldq<RPAD>();
  const int nb = (r + 7) / 8;
  const int npairs = nb * (nb + 1) / 2;
  const bool mine = h < npairs;
  int kb = 0, rem = mine ? h : 0;
  while (rem >= nb - kb) { rem -= nb - kb; ++kb; }
  const int lb = kb + rem;
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
  bool first = true;
  RowStage<RPAD, NH> st;
  if (q0 < q1) st.load(Q, layout, ldq_g, r, q0, (int)min((int64_t)kQsRows, q1 - q0), h);
  int in_window = 0;
  for (int64_t s0 = q0; s0 < q1; s0 += kQsRows) {
    helper_sync<NH>();          // previous rows consumed
    st.store(Qs, layout, h);
    helper_sync<NH>();
    const int64_t s1 = s0 + kQsRows;
    if (s1 < q1) st.load(Q, layout, ldq_g, r, s1, (int)min((int64_t)kQsRows, q1 - s1), h);
    if (mine) {
#pragma unroll 2
      for (int m = 0; m < kQsRows; ++m) {
        const float4 a0 = *reinterpret_cast<const float4*>(&Qs[m * LQ + kb * 8]);
        const float4 a1 = *reinterpret_cast<const float4*>(&Qs[m * LQ + kb * 8 + 4]);
        const float4 b0 = *reinterpret_cast<const float4*>(&Qs[m * LQ + lb * 8]);
        const float4 b1 = *reinterpret_cast<const float4*>(&Qs[m * LQ + lb * 8 + 4]);
        const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
      }
    }
    in_window += kQsRows;
    if (in_window == 128 || s1 >= q1) {   // fold the window into float64
      if (mine) {
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int k = kb * 8 + i, l = lb * 8 + j;
            if (k < r && l < r) {
              double* g = gpart + k * r + l;
              *g = first ? (double)acc[i][j] : *g + (double)acc[i][j];
            }
            acc[i][j] = 0.f;
          }
      }
      first = false;
      in_window = 0;
    }
  }
  if (mine) {
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int k = kb * 8 + i, l = lb * 8 + j;
        if (k < r && l < r) {
          if (first) gpart[k * r + l] = 0.0;           // no rows in this share
          if (kb != lb) gpart[l * r + k] = gpart[k * r + l];
        }
      }
  }
  helper_sync<NH>();            // Qs free
}

template <int RPAD, int NH = kHelpers>
__device__ void gram_rows(float* Qs, const float* Q, int layout, int64_t ldq_g, int64_t q0,
                          int64_t q1, int r, double* gpart, int h) {
  const int nb = (r + 7) / 8;
  if (RPAD > 64 && nb * (nb + 1) / 2 <= NH)
    gram_rows8<RPAD, NH>(Qs, Q, layout, ldq_g, q0, q1, r, gpart, h);
  else
    gram_rows4<RPAD, NH>(Qs, Q, layout, ldq_g, q0, q1, r, gpart, h);
}

// Float64 sum, in a fixed order, of the `nparts` partials of entries
// [e0, e1), nb entries at a time: the helpers form ng groups per entry (ng
// the largest power of two <= min(NH / nb, nparts)); group g adds partials
// g, g + ng, g + 2 ng, ... (16 loads in flight), and the ng group sums are
// added pairwise in a fixed tree (log2 ng rounds).  Writes G64 (r x r) and
// the zero-padded float32 copy Gpad.  `scratch` holds NH doubles (shared).
template <int RPAD, int NH = kHelpers>
__device__ void gram_reduce_slice(const double* gpart, int nparts, int r, int e0, int e1,
                                  double* G64, float* Gpad, double* scratch, int h) {
  const int rr = r * r;
  const int ne = e1 - e0;
  if (ne <= 0) return;
  for (int eb = e0; eb < e1; eb += NH) {
    const int nb = min(NH, e1 - eb);
    const int cap = min(NH / nb, nparts);
    int ng = 1;
    while (2 * ng <= cap) ng *= 2;
    const int g = h / nb, e = eb + h % nb;
    if (g < ng) {
      double s = 0.0;
      for (int t0 = g; t0 < nparts; t0 += 16 * ng) {
        double v[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int t = t0 + j * ng;
          v[j] = t < nparts ? __ldcg(gpart + (int64_t)t * rr + e) : 0.0;
        }
#pragma unroll
        for (int j = 0; j < 16; ++j)
          if (t0 + j * ng < nparts) s += v[j];
      }
      scratch[g * nb + (h % nb)] = s;
    }
    helper_sync<NH>();
    for (int w = ng / 2; w >= 1; w >>= 1) {
      if (g < w) scratch[g * nb + (h % nb)] += scratch[(g + w) * nb + (h % nb)];
      helper_sync<NH>();
    }
    if (h < nb) {
      const double tot = scratch[h];
      G64[eb + h] = tot;
      Gpad[((eb + h) / r) * RPAD + ((eb + h) % r)] = (float)tot;
    }
    helper_sync<NH>();
  }
}

// Old rows of the slice into Os (issued early: they do not depend on G).
template <int RPAD, int NH = kHelpers>
__device__ void load_old(float* Os, const EpiArgs& e, int R, int64_t row0, int rows, int h) {
  constexpr int LO = ldo<RPAD>();
  constexpr int NV = 16;   // loads in flight per thread per batch
  const int r = e.r;
  for (int b0 = 0; b0 < R * RPAD; b0 += NV * NH) {
    float v[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      const int i = b0 + h + j * NH;
      int m, k;
      if (e.layout == kFactorRowMajor) { m = i / RPAD; k = i % RPAD; }
      else                             { k = i / R;    m = i % R; }
      v[j] = (i < R * RPAD && m < rows && k < r)
                 ? (e.layout == kFactorRowMajor ? e.F[(row0 + m) * r + k]
                                                : e.F[(int64_t)k * e.ldf + row0 + m])
                 : 0.f;
    }
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      const int i = b0 + h + j * NH;
      if (i < R * RPAD) {
        int m, k;
        if (e.layout == kFactorRowMajor) { m = i / RPAD; k = i % RPAD; }
        else                             { k = i / R;    m = i % R; }
        Os[m * LO + k] = v[j];
      }
    }
  }
}

// den = old . G for the slice into the helper's registers (Os already
// loaded; rows beyond the slice's valid rows and ranks beyond r are zero).  G rows are staged
// 32 at a time through Qs from the padded float32 copy; the next 32 are in
// flight while the current ones are used.
template <int RPAD, int NH = kHelpers>
__device__ void compute_den(float* Qs, const float* Os, DenTile<RPAD, NH>& den, const float* Gpad,
                            int r, int R, int h) {
  constexpr int LQ = ldq<RPAD>();
  constexpr int LO = ldo<RPAD>();
  constexpr int NG = kQsRows * RPAD;
  constexpr int GV = (NG + NH - 1) / NH;
  constexpr int KG = RPAD / 8;
  constexpr int MG = NH / KG;
  constexpr int NA = DenTile<RPAD, NH>::NA;
  const int kg = h % KG, mg = h / KG;
  const bool active = h < KG * MG;
  auto& acc = den.d;    // rows mg + (4a + i) MG of the slice
#pragma unroll
  for (int a = 0; a < NA; ++a)
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[a][i][j] = 0.f;
  float gv[GV];
  auto gload = [&](int l0) {
#pragma unroll
    for (int j = 0; j < GV; ++j) {
      const int i = h + j * NH;
      gv[j] = (i < NG && l0 + i / RPAD < r) ? __ldcg(Gpad + l0 * RPAD + i) : 0.f;
    }
  };
  gload(0);
  for (int l0 = 0; l0 < r; l0 += kQsRows) {
    helper_sync<NH>();   // previous G rows consumed (and Os complete on entry)
#pragma unroll
    for (int j = 0; j < GV; ++j) {
      const int i = h + j * NH;
      if (i < NG) Qs[(i / RPAD) * LQ + (i % RPAD)] = gv[j];
    }
    helper_sync<NH>();
    if (l0 + kQsRows < r) gload(l0 + kQsRows);
    const int nl = min(kQsRows, r - l0);
    if (active) {
#pragma unroll
      for (int a = 0; a < NA; ++a) {
        if (mg + 4 * a * MG >= R) break;
        int mrow[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) mrow[i] = min(mg + (4 * a + i) * MG, R - 1);
#pragma unroll 2
        for (int l = 0; l < nl; ++l) {
          const float4 g0 = *reinterpret_cast<const float4*>(&Qs[l * LQ + kg * 8]);
          const float4 g1 = *reinterpret_cast<const float4*>(&Qs[l * LQ + kg * 8 + 4]);
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const float o = Os[mrow[i] * LO + l0 + l];
            acc[a][i][0] = fmaf(o, g0.x, acc[a][i][0]); acc[a][i][1] = fmaf(o, g0.y, acc[a][i][1]);
            acc[a][i][2] = fmaf(o, g0.z, acc[a][i][2]); acc[a][i][3] = fmaf(o, g0.w, acc[a][i][3]);
            acc[a][i][4] = fmaf(o, g1.x, acc[a][i][4]); acc[a][i][5] = fmaf(o, g1.y, acc[a][i][5]);
            acc[a][i][6] = fmaf(o, g1.z, acc[a][i][6]); acc[a][i][7] = fmaf(o, g1.w, acc[a][i][7]);
          }
        }
      }
    }
  }
}

// compute_den for DenTile8 (ranks above 64).
template <int RPAD, int NH = kHelpers>
__device__ void compute_den(float* Qs, const float* Os, DenTile8<RPAD, NH>& den,
                            const float* Gpad, int r, int R, int h) {
  constexpr int LQ = ldq<RPAD>();
  constexpr int LO = ldo<RPAD>();
  constexpr int NG = kQsRows * RPAD;
  constexpr int GV = (NG + NH - 1) / NH;
  constexpr int KG = DenTile8<RPAD, NH>::KG;
  constexpr int MG = DenTile8<RPAD, NH>::MG;
  const int kg = h % KG, mg = h / KG;
  const bool active = h < KG * MG && mg * 8 < R;
  auto& acc = den.d;
  den.clear();
  int mrow[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) mrow[i] = min(mg * 8 + i, R - 1);
  float gv[GV];
  auto gload = [&](int l0) {
#pragma unroll
    for (int j = 0; j < GV; ++j) {
      const int i = h + j * NH;
      gv[j] = (i < NG && l0 + i / RPAD < r) ? __ldcg(Gpad + l0 * RPAD + i) : 0.f;
    }
  };
  gload(0);
  for (int l0 = 0; l0 < r; l0 += kQsRows) {
    helper_sync<NH>();   // previous G rows consumed (and Os complete on entry)
#pragma unroll
    for (int j = 0; j < GV; ++j) {
      const int i = h + j * NH;
      if (i < NG) Qs[(i / RPAD) * LQ + (i % RPAD)] = gv[j];
    }
    helper_sync<NH>();
    if (l0 + kQsRows < r) gload(l0 + kQsRows);
    const int nl = min(kQsRows, r - l0);
    if (active) {
#pragma unroll 2
      for (int l = 0; l < nl; ++l) {
        const float4 g0 = *reinterpret_cast<const float4*>(&Qs[l * LQ + kg * 8]);
        const float4 g1 = *reinterpret_cast<const float4*>(&Qs[l * LQ + kg * 8 + 4]);
        const float gw[8] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w};
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const float o = Os[mrow[i] * LO + l0 + l];
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(o, gw[j], acc[i][j]);
        }
      }
    }
  }
}

// Variant for kernels with shared memory to spare: den into Ds[m][k]
// (stride RPAD + 4), one pass of up to 4 x 8 values per thread at a time
// (G re-staged per pass), so no denominators live in registers.
template <int RPAD> __host__ __device__ constexpr int ldd() { return RPAD + 4; }

template <int RPAD, int NH>
__device__ void compute_den_smem(float* Qs, const float* Os, float* Ds, const float* Gpad,
                                 int r, int R, int h) {
  constexpr int LQ = ldq<RPAD>();
  constexpr int LO = ldo<RPAD>();
  constexpr int LD = ldd<RPAD>();
  constexpr int NG = kQsRows * RPAD;
  constexpr int GV = 16;
  constexpr int KG = RPAD / 8;
  constexpr int MG = NH / KG;
  const int kg = h % KG, mg = h / KG;
  const bool active = h < KG * MG;
  for (int mb = mg; mb - mg < R; mb += 4 * MG) {
    float acc[4][8];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
    int mrow[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) mrow[i] = min(mb + i * MG, R - 1);
    for (int l0 = 0; l0 < r; l0 += kQsRows) {
      helper_sync<NH>();   // Os complete / previous G rows consumed
      for (int b = h; b < NG; b += GV * NH) {
        float gv[GV];
#pragma unroll
        for (int j = 0; j < GV; ++j) {
          const int i = b + j * NH;
          gv[j] = (i < NG && l0 + i / RPAD < r) ? __ldcg(Gpad + l0 * RPAD + i) : 0.f;
        }
#pragma unroll
        for (int j = 0; j < GV; ++j) {
          const int i = b + j * NH;
          if (i < NG) Qs[(i / RPAD) * LQ + (i % RPAD)] = gv[j];
        }
      }
      helper_sync<NH>();
      const int nl = min(kQsRows, r - l0);
      if (active && mb < R) {
#pragma unroll 2
        for (int l = 0; l < nl; ++l) {
          const float4 g0 = *reinterpret_cast<const float4*>(&Qs[l * LQ + kg * 8]);
          const float4 g1 = *reinterpret_cast<const float4*>(&Qs[l * LQ + kg * 8 + 4]);
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const float o = Os[mrow[i] * LO + l0 + l];
            acc[i][0] = fmaf(o, g0.x, acc[i][0]); acc[i][1] = fmaf(o, g0.y, acc[i][1]);
            acc[i][2] = fmaf(o, g0.z, acc[i][2]); acc[i][3] = fmaf(o, g0.w, acc[i][3]);
            acc[i][4] = fmaf(o, g1.x, acc[i][4]); acc[i][5] = fmaf(o, g1.y, acc[i][5]);
            acc[i][6] = fmaf(o, g1.z, acc[i][6]); acc[i][7] = fmaf(o, g1.w, acc[i][7]);
          }
        }
      }
    }
    if (active) {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int m = mb + i * MG;
        if (m < R) {
          *reinterpret_cast<float4*>(&Ds[m * LD + kg * 8]) =
              make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
          *reinterpret_cast<float4*>(&Ds[m * LD + kg * 8 + 4]) =
              make_float4(acc[i][4], acc[i][5], acc[i][6], acc[i][7]);
        }
      }
    }
  }
}

// finish() with the denominators in Ds: every thread of the block takes part
// in both passes; pass 1 works on 8 consecutive ranks of a row at a time.
template <int RPAD, int NT>
__device__ void finish_smem(float* Ns, const float* Os, const float* Ds, const EpiArgs& e,
                            int R, int64_t row0, int rows) {
  constexpr int LN = epi_ldn<RPAD>();
  constexpr int LO = ldo<RPAD>();
  constexpr int LD = ldd<RPAD>();
  constexpr int KG = RPAD / 4;
  const int r = e.r;
  for (int i = threadIdx.x; i < rows * KG; i += NT) {
    const int m = i / KG, k0 = (i - m * KG) * 4;
    if (k0 >= r) continue;
    float o[4], nu[4], v[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      o[j] = Os[m * LO + k0 + j];
      nu[j] = Ns[m * LN + k0 + j];
    }
    const float4 dn = *reinterpret_cast<const float4*>(&Ds[m * LD + k0]);
    const float dv[4] = {dn.x, dn.y, dn.z, dn.w};
    update8<4>(o, nu, dv, e.eps, v);
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (k0 + j >= r) v[j] = 0.f;
    *reinterpret_cast<float4*>(&Ns[m * LN + k0]) = make_float4(v[0], v[1], v[2], v[3]);
    if (e.layout == kFactorRowMajor) {
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (k0 + j < r) e.F[(row0 + m) * r + k0 + j] = v[j];
    }
  }
  __syncthreads();
  store_cols<RPAD, NT>(Ns, e, row0, rows);
  (void)R;
}

}  // namespace tcepi
}  // namespace nmf
