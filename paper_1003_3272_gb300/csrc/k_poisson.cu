// Poisson variant of the MM NMF iteration (Section 3.1, closing paragraph):
// maximise L = sum_ij [v_ij ln b_ij - b_ij], b = W H, by the simultaneous
// square-root update the paper prints after it,
//     w_ik <- w_ik sqrt( (sum_j v_ij h_kj / b_ij) / (sum_j h_kj) )
//     h_kj <- h_kj sqrt( (sum_i v_ij w_ik / b_ij) / (sum_i w_ik) )
// with b, the sums and both right-hand sides from the factors of the same
// iteration.  eps guards the two divisions (v / (b + eps), num / (den + eps));
// a term with v_ij = 0 is zero.
//
// One iteration is four launches on the float32 FMA pipes:
//   k_pois_sums    the r row sums of H and column sums of W (float64, a
//                  fixed-order tree per rank);
//   k_pois_pass<0> per 64-row panel of V and a segment of its 64-column
//                  tiles: b = W_I H_J (K = r), q = v / (b + eps), and the
//                  numerator of W, q H_J^T (K = 64), summed over the
//                  segment's tiles in float32 and written out in float64;
//   k_pois_pass<1> the same per 64-column panel and a segment of its row
//                  tiles, with the numerator of H, W_I^T q;
//   k_pois_update  both factors in place from the segment partials (summed
//                  in segment order), the sums and the old factors.
// Both passes read V once each (float32, row-major, as the caller holds it);
// b is formed twice (once per pass), so an iteration is 8pnr flops.  The
// loglikelihood L is one more launch (k_pois_loglik).  Every sum runs in a
// fixed order: the result is deterministic.
#include <cstdint>
#include <climits>

#include "nmf_internal.cuh"

namespace nmf {
namespace {

constexpr int kPT = 64;          // tile edge (rows and columns of V)
constexpr int kPThreads = 256;   // 16 x 16 threads, a 4 x 4 sub-tile each
constexpr int kPMaxRank = 64;
static_assert(kPMaxRank <= 64, "stage_w gives each rank one of 64 lanes");
constexpr int kLW = kPT + 4;     // row stride of Wt and Qs (16-byte rows)

// Shared memory of a pass block: Wt[r][kLW] (W_I transposed), Hs[r][64]
// (H_J), Qs[64][kLW] (q of the tile, row-major).
__host__ __device__ inline int pois_floats(int r) { return r * kLW + r * kPT + kPT * kLW; }

// Block 2k + which: the row sum of H's rank k (which = 0, the denominator
// of the W update) or the column sum of W's rank k (which = 1, of the H
// update), in float64 (strided per thread, then a fixed tree).
__global__ void k_pois_sums(const float* __restrict__ W, const float* __restrict__ H,
                            int64_t p, int64_t n, int r, double* __restrict__ sums) {
  __shared__ double red[kPThreads];
  const int k = blockIdx.x >> 1, which = blockIdx.x & 1;
  double s = 0.0;
  if (which == 0) {
    for (int64_t j = threadIdx.x; j < n; j += kPThreads) s += (double)H[(int64_t)k * n + j];
  } else {
    for (int64_t i = threadIdx.x; i < p; i += kPThreads) s += (double)W[i * r + k];
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = kPThreads / 2; w >= 1; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) sums[which * r + k] = red[0];
}

// Loads a 64 x 64 tile of V (rows i0.., columns j0..) for the thread's 4 x 4
// sub-tile: rows i0 + 4 ty + a, columns j0 + 4 tx + c; zero outside V.
__device__ __forceinline__ void load_v(const float* __restrict__ V, int64_t ldv, int64_t p,
                                       int64_t n, int64_t i0, int64_t j0, int ty, int tx,
                                       bool vec, float (&v)[4][4]) {
  const int64_t jc = j0 + 4 * tx;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int64_t i = i0 + 4 * ty + a;
    if (i < p && vec && jc + 3 < n) {
      const float4 x = __ldcs(reinterpret_cast<const float4*>(V + i * ldv + jc));
      v[a][0] = x.x; v[a][1] = x.y; v[a][2] = x.z; v[a][3] = x.w;
    } else {
#pragma unroll
      for (int c = 0; c < 4; ++c)
        v[a][c] = (i < p && jc + c < n) ? __ldcs(V + i * ldv + jc + c) : 0.f;
    }
  }
}

// Stages W rows [i0, i0 + 64) as Wt[k][i] and H columns [j0, j0 + 64) as
// Hs[k][j], zero outside the factors.  W: thread t reads rank t % 64 of row
// t / 64 (+4 per pass), so a warp reads along a row of W and writes down a
// column of Wt (stride kLW words: four-way bank conflicts); no division by
// the runtime rank.  H: along rows on both sides.
__device__ __forceinline__ void stage_w(const float* __restrict__ W, int64_t p, int r,
                                        int64_t i0, float* Wt) {
  const int k = threadIdx.x & 63;
  if (k >= r) return;
  for (int i = threadIdx.x >> 6; i < kPT; i += kPThreads / 64)
    Wt[k * kLW + i] = i0 + i < p ? W[(i0 + i) * r + k] : 0.f;
}
__device__ __forceinline__ void stage_h(const float* __restrict__ H, int64_t n, int r,
                                        int64_t j0, float* Hs) {
  for (int idx = threadIdx.x; idx < r * kPT; idx += kPThreads) {
    const int k = idx / kPT, j = idx - k * kPT;
    Hs[idx] = j0 + j < n ? H[(int64_t)k * n + j0 + j] : 0.f;
  }
}

// The next tile's streamed factor block, held in registers while the
// current tile's GEMM2 runs (its loads then overlap the arithmetic):
// MODE 0 H_J (r x 64; element tid + 256 m), MODE 1 W_I (64 x r; rank
// tid % 64 of rows tid / 64 + 4 m, as stage_w).  Zero outside the factors.
template <int MODE>
struct NextBlock {
  float x[16];
  __device__ __forceinline__ void load(const float* __restrict__ W, const float* __restrict__ H,
                                       int64_t p, int64_t n, int r, int64_t i0, int64_t j0) {
    if (MODE == 0) {
#pragma unroll
      for (int m = 0; m < 16; ++m) {
        const int idx = threadIdx.x + kPThreads * m;
        const int k = idx >> 6, j = idx & 63;
        x[m] = (k < r && j0 + j < n) ? H[(int64_t)k * n + j0 + j] : 0.f;
      }
    } else {
      const int k = threadIdx.x & 63;
#pragma unroll
      for (int m = 0; m < 16; ++m) {
        const int i = (threadIdx.x >> 6) + 4 * m;
        x[m] = (k < r && i0 + i < p) ? W[(i0 + i) * r + k] : 0.f;
      }
    }
  }
  __device__ __forceinline__ void store(int r, float* Wt, float* Hs) const {
    if (MODE == 0) {
#pragma unroll
      for (int m = 0; m < 16; ++m) {
        const int idx = threadIdx.x + kPThreads * m;
        if (idx < r * kPT) Hs[idx] = x[m];
      }
    } else {
      const int k = threadIdx.x & 63;
      if (k < r) {
#pragma unroll
        for (int m = 0; m < 16; ++m) Wt[k * kLW + (threadIdx.x >> 6) + 4 * m] = x[m];
      }
    }
  }
};

// Knuth's two-sum: s + e = a + b exactly (round to nearest).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// MODE 0: block = (row panel I, segment of column tiles); numerator of W.
// MODE 1: block = (column panel J, segment of row tiles); numerator of H.
// part: MODE 0 [seg][p][r], MODE 1 [seg][n][r] (float64).  Ranks above 64
// are not served (pois_supported).
//
// Per tile: GEMM1 b = W_I H_J (thread: rows 4 ty .. 4 ty + 3, columns
// 4 tx .. 4 tx + 3, K = r), q into Qs, then GEMM2 over the tile's 64 entries
// of K, four at a time so that every operand load is 16 bytes:
//   MODE 0: acc[x][y] += sum_u q[g + 16 x][j + u] h[4 c + y][j + u]
//           (rows g + 16 x: consecutive lanes on consecutive rows of Qs)
//   MODE 1: acc[x][y] += sum_u q[i + u][4 g + x] w[i + u][4 c + y]
// with g = tid % 16 and c = tid / 16 (ranks 4 c .. 4 c + 3 < r4).
template <int MODE>
__global__ void __launch_bounds__(kPThreads)
k_pois_pass(const float* __restrict__ V, int64_t ldv, const float* __restrict__ W,
            const float* __restrict__ H, int64_t p, int64_t n, int r, float eps, int segs,
            double* __restrict__ part) {
  extern __shared__ float sm[];
  float* Wt = sm;
  float* Hs = sm + r * kLW;
  float* Qs = Hs + r * kPT;
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  const int panel = blockIdx.x / segs, seg = blockIdx.x - panel * segs;
  const int64_t panel0 = (int64_t)panel * kPT;
  const int64_t other = MODE == 0 ? n : p;              // extent streamed
  const int ntiles = (int)((other + kPT - 1) / kPT);
  const int t0 = (int)((int64_t)seg * ntiles / segs);
  const int t1 = (int)((int64_t)(seg + 1) * ntiles / segs);
  const bool vec = (ldv % 4 == 0) && (reinterpret_cast<uintptr_t>(V) % 16 == 0);
  const int r4 = (r + 3) & ~3;
  const int g = tid & 15, c = tid >> 4;
  const bool item = 4 * c < r4;
  // ranks of this thread's GEMM2 item, clamped into the staged rows (the
  // products of ranks r .. r4-1 are formed and discarded)
  int ky[4];
#pragma unroll
  for (int y = 0; y < 4; ++y) ky[y] = min(4 * c + y, r - 1);

  // the panel's resident factor block
  if (MODE == 0) stage_w(W, p, r, panel0, Wt);
  else stage_h(H, n, r, panel0, Hs);

  // the segment's running sums (float32 over its tiles)
  float tot[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) tot[a][b] = 0.f;

  NextBlock<MODE> nb;
  if (t0 < t1)
    nb.load(W, H, p, n, r, MODE == 0 ? panel0 : (int64_t)t0 * kPT,
            MODE == 0 ? (int64_t)t0 * kPT : panel0);
  for (int t = t0; t < t1; ++t) {
    const int64_t o0 = (int64_t)t * kPT;
    const int64_t i0 = MODE == 0 ? panel0 : o0;
    const int64_t j0 = MODE == 0 ? o0 : panel0;
    float v[4][4];
    load_v(V, ldv, p, n, i0, j0, ty, tx, vec, v);
    __syncthreads();   // the previous tile's operands are consumed
    nb.store(r, Wt, Hs);
    __syncthreads();

    // GEMM1: b = W_I H_J for rows 4 ty.., columns 4 tx..
    float b[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int e = 0; e < 4; ++e) b[a][e] = 0.f;
#pragma unroll 4
    for (int k = 0; k < r; ++k) {
      const float4 w4 = *reinterpret_cast<const float4*>(&Wt[k * kLW + 4 * ty]);
      const float4 h4 = *reinterpret_cast<const float4*>(&Hs[k * kPT + 4 * tx]);
      const float wv[4] = {w4.x, w4.y, w4.z, w4.w};
      const float hv[4] = {h4.x, h4.y, h4.z, h4.w};
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int e = 0; e < 4; ++e) b[a][e] = fmaf(wv[a], hv[e], b[a][e]);
    }
    // q = v / (b + eps), zero where v is zero; row-major into Qs.  q only
    // weights the sums of the numerators, so the fast division serves: within
    // two ulps for divisors in [2^-126, 2^126] (the default eps = 1e-10 keeps
    // b + eps above the lower end).
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      float q[4];
#pragma unroll
      for (int e = 0; e < 4; ++e)
        q[e] = v[a][e] == 0.f ? 0.f : __fdividef(v[a][e], __fadd_rn(b[a][e], eps));
      *reinterpret_cast<float4*>(&Qs[(4 * ty + a) * kLW + 4 * tx]) =
          make_float4(q[0], q[1], q[2], q[3]);
    }
    __syncthreads();
    if (t + 1 < t1) {
      const int64_t o1 = o0 + kPT;
      nb.load(W, H, p, n, r, MODE == 0 ? panel0 : o1, MODE == 0 ? o1 : panel0);
    }

    if (item) {
      float acc[4][4];
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] = 0.f;
#pragma unroll 2
      for (int kk = 0; kk < kPT; kk += 4) {
        float qa[4][4], fa[4][4];
        if (MODE == 0) {
#pragma unroll
          for (int x = 0; x < 4; ++x) {
            const float4 q4 = *reinterpret_cast<const float4*>(&Qs[(g + 16 * x) * kLW + kk]);
            qa[x][0] = q4.x; qa[x][1] = q4.y; qa[x][2] = q4.z; qa[x][3] = q4.w;
          }
#pragma unroll
          for (int y = 0; y < 4; ++y) {
            const float4 f4 = *reinterpret_cast<const float4*>(&Hs[ky[y] * kPT + kk]);
            fa[y][0] = f4.x; fa[y][1] = f4.y; fa[y][2] = f4.z; fa[y][3] = f4.w;
          }
        } else {
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const float4 q4 = *reinterpret_cast<const float4*>(&Qs[(kk + u) * kLW + 4 * g]);
            qa[0][u] = q4.x; qa[1][u] = q4.y; qa[2][u] = q4.z; qa[3][u] = q4.w;
          }
#pragma unroll
          for (int y = 0; y < 4; ++y) {
            const float4 f4 = *reinterpret_cast<const float4*>(&Wt[ky[y] * kLW + kk]);
            fa[y][0] = f4.x; fa[y][1] = f4.y; fa[y][2] = f4.z; fa[y][3] = f4.w;
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int y = 0; y < 4; ++y) acc[x][y] = fmaf(qa[x][u], fa[y][u], acc[x][y]);
      }
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) tot[x][y] = __fadd_rn(tot[x][y], acc[x][y]);
    }
  }

  if (item) {
    const int64_t extent = MODE == 0 ? p : n;
    double* dst = part + (int64_t)seg * extent * r;
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      const int64_t m = panel0 + (MODE == 0 ? g + 16 * x : 4 * g + x);
      if (m >= extent) continue;
#pragma unroll
      for (int y = 0; y < 4; ++y) {
        const int k = 4 * c + y;
        if (k < r) dst[m * r + k] = (double)tot[x][y];
      }
    }
  }
}

// Both factors in place: W entries (idx < p r) and H entries (the rest).
// The numerator's segment partials are summed in float64 (fixed order); the
// ratio to the denominator, its square root and the product with the old
// entry are IEEE float32 operations (a few units of 2^-24 in all; float64
// division and square root are slow on this part and buy nothing here).
__global__ void k_pois_update(float* __restrict__ W, float* __restrict__ H, int64_t p,
                              int64_t n, int r, float eps, const double* __restrict__ partW,
                              int segW, const double* __restrict__ partH, int segH,
                              const double* __restrict__ sums) {
  const int64_t nw = p * r, total = nw + (int64_t)r * n;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    if (idx < nw) {
      const int64_t i = idx / r;
      const int k = (int)(idx - i * r);
      double num = 0.0;
      for (int s = 0; s < segW; ++s) num += partW[((int64_t)s * p + i) * r + k];
      const float ratio = __fdiv_rn((float)num, (float)(sums[k] + (double)eps));
      W[idx] = __fmul_rn(W[idx], __fsqrt_rn(ratio));
    } else {
      const int64_t h = idx - nw;
      const int k = (int)(h / n);
      const int64_t j = h - (int64_t)k * n;
      double num = 0.0;
      for (int s = 0; s < segH; ++s) num += partH[((int64_t)s * n + j) * r + k];
      const float ratio = __fdiv_rn((float)num, (float)(sums[r + k] + (double)eps));
      H[h] = __fmul_rn(H[h], __fsqrt_rn(ratio));
    }
  }
}

// Float-float arithmetic: an unevaluated pair hi + lo of float32 values
// (about 48 significant bits), on the float32 pipes.  x += (yh + yl), the
// result renormalised (Dekker 1971).
__device__ __forceinline__ void ff_add(float& xh, float& xl, float yh, float yl) {
  float s, e;
  two_sum(xh, yh, s, e);
  e = __fadd_rn(e, __fadd_rn(xl, yl));
  xh = __fadd_rn(s, e);
  xl = __fsub_rn(e, __fsub_rn(xh, s));
}

// ln 2 in three parts, the high part with 16 significant bits (Cody and
// Waite 1980): e * kLn2Hi is exact for every float32 exponent e, and
// kLn2Hi + kLn2Lo + kLn2Lo2 is ln 2 to about 2^-70.
constexpr float kLn2Hi = 0.693145751953125f;
constexpr float kLn2Lo = 1.428606765330187e-06f;
constexpr float kLn2Lo2 = 5.497923018708371e-14f;
constexpr int kLnTab = 256;   // ln(1 + k / 256), k = 0 .. 256

// ln(bh + bl) for a normalised float-float pair with bh a positive normal
// float32, as a float-float pair within about 2^-48 of |ln b| (2^-43 at the
// largest exponents), by the
// table-driven reduction of Tang (1990, ACM TOMS 16): bh = 2^e m with m in
// [1, 2); c = 1 + k / 256 the table point nearest m, so that
//   ln b = e ln 2 + ln c + ln(1 + r) + ln(1 + bl / bh),  r = (m - c) / c,
// |r| <= 2^-9; ln(1 + r) = r - r^2 / 2 + r^3 / 3 - r^4 / 4 + r^5 / 5 (the
// next term is below 2^-56), r and r^2 carried as float-float, the rest in
// float32; ln(1 + bl / bh) = bl / bh to within 2^-49.  tab holds
// ln(1 + k / 256) as float-float pairs.
__device__ __forceinline__ void ln_ff(float bh, float bl, const float2* tab, float& lh,
                                      float& ll) {
  const uint32_t u = __float_as_uint(bh);
  const float ex = (float)((int)(u >> 23) - 127);
  const float m = __uint_as_float((u & 0x007FFFFFu) | 0x3F800000u);
  const int k = __float2int_rn(__fmul_rn(__fsub_rn(m, 1.f), (float)kLnTab));
  const float c = __fadd_rn(1.f, __fmul_rn((float)k, 1.f / (float)kLnTab));   // exact
  const float d = __fsub_rn(m, c);                                             // exact
  const float rc = __fdiv_rn(1.f, c);
  const float rh = __fmul_rn(d, rc);
  const float rl = __fmul_rn(__fmaf_rn(-rh, c, d), rc);   // the exact remainder / c
  const float sq = __fmul_rn(rh, rh);
  const float sqe = __fmaf_rn(rh, rh, -sq);
  const float tail = __fmul_rn(__fmul_rn(sq, rh),
                               __fmaf_rn(rh, __fmaf_rn(rh, 0.2f, -0.25f), 1.f / 3.f));
  const float eh = __fmul_rn(ex, kLn2Lo);
  const float ehe = __fadd_rn(__fmaf_rn(ex, kLn2Lo, -eh), __fmul_rn(ex, kLn2Lo2));
  const float2 t = tab[k];
  // the large parts in float-float, the small ones summed in float32
  float sh = __fmul_rn(ex, kLn2Hi), sl = 0.f;   // exact
  ff_add(sh, sl, t.x, 0.f);
  ff_add(sh, sl, eh, 0.f);
  ff_add(sh, sl, rh, 0.f);
  ff_add(sh, sl, __fmul_rn(-0.5f, sq), 0.f);
  float small = __fadd_rn(__fadd_rn(t.y, ehe), __fadd_rn(rl, __fmul_rn(-0.5f, sqe)));
  small = __fadd_rn(small, __fadd_rn(__fmul_rn(-rh, rl), tail));
  small = __fadd_rn(small, __fdiv_rn(bl, bh));
  ff_add(sh, sl, small, 0.f);
  lh = sh;
  ll = sl;
}

// L = sum_ij [v_ij ln b_ij - b_ij], 0 ln 0 = 0, over 64 x 64 tiles (block b
// takes tiles b, b + grid, ...; the grid is fixed, so the order is too).
// b_ij = sum_k w_ik h_kj as an unevaluated float32 pair hi + lo by the
// compensated dot product of Ogita, Rump and Oishi (2005, "Dot2": exact
// products by FMA, Knuth's two-sum on the running sum), within a few units
// of 2^-48 relative of the exact sum; ln b by ln_ff; each thread keeps
// sum v ln b and sum b as float-float pairs, and the thread and block
// partials are added in float64 in a fixed order.  The float32 pipes carry
// the per-entry work (the float64 pipe is narrow on this part); entries whose
// b is not a positive normal float32 take a float64 logarithm instead.
constexpr int kLBlocks = 2 * 152;
__global__ void __launch_bounds__(kPThreads)
k_pois_loglik(const float* __restrict__ V, int64_t ldv, const float* __restrict__ W,
              const float* __restrict__ H, int64_t p, int64_t n, int r,
              double* __restrict__ partials, unsigned int* done, double* __restrict__ out) {
  extern __shared__ float sm[];
  float* Wt = sm;
  float* Hs = sm + r * kLW;
  __shared__ double red[kPThreads];
  __shared__ float2 lntab[kLnTab + 1];
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  for (int k = tid; k <= kLnTab; k += kPThreads) {
    const double x = log1p((double)k / kLnTab);
    const float hi = (float)x;
    lntab[k] = make_float2(hi, (float)(x - (double)hi));
  }
  const int64_t tp = (p + kPT - 1) / kPT, tn = (n + kPT - 1) / kPT;
  const bool vec = (ldv % 4 == 0) && (reinterpret_cast<uintptr_t>(V) % 16 == 0);
  // sum v ln b and sum b as float-float pairs; entries whose b is not a
  // positive normal float32 (zero, tiny) take the float64 path
  float vh = 0.f, vl = 0.f, bsh = 0.f, bsl = 0.f;
  double s = 0.0;
  for (int64_t t = blockIdx.x; t < tp * tn; t += gridDim.x) {
    const int64_t i0 = (t / tn) * kPT, j0 = (t % tn) * kPT;
    float v[4][4];
    load_v(V, ldv, p, n, i0, j0, ty, tx, vec, v);
    __syncthreads();
    stage_w(W, p, r, i0, Wt);
    stage_h(H, n, r, j0, Hs);
    __syncthreads();
    float hi[4][4], lo[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int e = 0; e < 4; ++e) hi[a][e] = lo[a][e] = 0.f;
    for (int k = 0; k < r; ++k) {
      const float4 w4 = *reinterpret_cast<const float4*>(&Wt[k * kLW + 4 * ty]);
      const float4 h4 = *reinterpret_cast<const float4*>(&Hs[k * kPT + 4 * tx]);
      const float wv[4] = {w4.x, w4.y, w4.z, w4.w};
      const float hv[4] = {h4.x, h4.y, h4.z, h4.w};
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const float pr = __fmul_rn(wv[a], hv[e]);
          const float pe = fmaf(wv[a], hv[e], -pr);          // exact product error
          float sum, se;
          two_sum(hi[a][e], pr, sum, se);
          hi[a][e] = sum;
          lo[a][e] = __fadd_rn(lo[a][e], __fadd_rn(pe, se));
        }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        if (i0 + 4 * ty + a >= p || j0 + 4 * tx + e >= n) continue;
        float bh, bl;
        two_sum(hi[a][e], lo[a][e], bh, bl);
        ff_add(bsh, bsl, bh, bl);
        const float x = v[a][e];
        if (x == 0.f) continue;
        if (bh >= 1.17549435e-38f && bh <= 3.4e38f) {
          float lh, ll;
          ln_ff(bh, bl, lntab, lh, ll);
          const float ph = __fmul_rn(x, lh);
          const float pe = __fmaf_rn(x, lh, -ph);
          ff_add(vh, vl, ph, __fmaf_rn(x, ll, pe));
        } else {
          s += (double)x * log((double)bh + (double)bl);
        }
      }
  }
  s += ((double)vh + (double)vl) - ((double)bsh + (double)bsl);
  red[tid] = s;
  __syncthreads();
  for (int w = kPThreads / 2; w >= 1; w >>= 1) {
    if (tid < w) red[tid] += red[tid + w];
    __syncthreads();
  }
  // the grid's last block adds the block partials in index order (fixed:
  // deterministic) and re-arms the counter
  __shared__ bool last;
  if (tid == 0) {
    partials[blockIdx.x] = red[0];
    __threadfence();
    last = atomicAdd(done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double t = 0.0;
  for (unsigned i = tid; i < gridDim.x; i += kPThreads) t += __ldcg(&partials[i]);
  __syncthreads();
  red[tid] = t;
  __syncthreads();
  for (int w = kPThreads / 2; w >= 1; w >>= 1) {
    if (tid < w) red[tid] += red[tid + w];
    __syncthreads();
  }
  if (tid == 0) {
    *out = red[0];
    *done = 0u;
  }
}

}  // namespace

bool pois_supported(int r) { return r >= 1 && r <= kPMaxRank; }

static size_t pois_smem_bytes(int r) { return (size_t)pois_floats(r) * sizeof(float); }

PoisPlan pois_plan(int64_t p, int64_t n, int r, int sms) {
  PoisPlan pl;
  pl.smem = (int)pois_smem_bytes(r);
  const int64_t tp = (p + kPT - 1) / kPT, tn = (n + kPT - 1) / kPT;
  // Resident blocks of a pass (both instances have the same footprint).
  int per_sm = 0;
  if (cudaFuncSetAttribute(k_pois_pass<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           pl.smem) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pois_pass<0>, kPThreads,
                                                    (size_t)pl.smem) != cudaSuccess)
    per_sm = 1;
  (void)cudaGetLastError();
  const int64_t slots = (int64_t)sms * (per_sm < 1 ? 1 : per_sm);
  // Segments per panel: the block count comes in waves of `slots`, and a
  // block's time is its tiles plus about one tile of staging and partial
  // writing; take the split with the least waves x (tiles + 1), at most 64.
  auto segs = [&](int64_t panels, int64_t tiles) {
    int64_t best = 1, best_cost = INT64_MAX;
    const int64_t smax = tiles < 64 ? tiles : 64;
    for (int64_t s = 1; s <= smax; ++s) {
      const int64_t waves = (panels * s + slots - 1) / slots;
      const int64_t cost = waves * ((tiles + s - 1) / s + 1);
      if (cost < best_cost) { best_cost = cost; best = s; }
    }
    return (int)best;
  };
  pl.segW = segs(tp, tn);
  pl.segH = segs(tn, tp);
  pl.gridW = (int)(tp * pl.segW);
  pl.gridH = (int)(tn * pl.segH);
  return pl;
}

// Block partials plus the arrival counter of the last-block sum.
int pois_loglik_parts() { return kLBlocks + 1; }

cudaError_t pois_iteration(const PoisPlan& pl, const float* V, int64_t ldv, float* W, float* H,
                           int64_t p, int64_t n, int r, float eps, double* sums, double* partW,
                           double* partH, cudaStream_t st) {
  cudaError_t e;
  e = cudaFuncSetAttribute(k_pois_pass<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, pl.smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_pois_pass<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, pl.smem);
  if (e != cudaSuccess) return e;
  k_pois_sums<<<2 * r, kPThreads, 0, st>>>(W, H, p, n, r, sums);
  k_pois_pass<0><<<pl.gridW, kPThreads, pl.smem, st>>>(V, ldv, W, H, p, n, r, eps, pl.segW,
                                                        partW);
  k_pois_pass<1><<<pl.gridH, kPThreads, pl.smem, st>>>(V, ldv, W, H, p, n, r, eps, pl.segH,
                                                        partH);
  const int64_t total = p * r + (int64_t)r * n;
  int64_t blocks = (total + kPThreads - 1) / kPThreads;
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_pois_update<<<(unsigned)blocks, kPThreads, 0, st>>>(W, H, p, n, r, eps, partW, pl.segW,
                                                         partH, pl.segH, sums);
  return cudaGetLastError();
}

cudaError_t pois_loglik(const float* V, int64_t ldv, const float* W, const float* H, int64_t p,
                        int64_t n, int r, double* partials, double* out, cudaStream_t st) {
  const int smem = (r * kLW + r * kPT) * (int)sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(k_pois_loglik, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       smem);
  if (e != cudaSuccess) return e;
  unsigned int* done = reinterpret_cast<unsigned int*>(partials + kLBlocks);
  k_pois_loglik<<<kLBlocks, kPThreads, smem, st>>>(V, ldv, W, H, p, n, r, partials, done, out);
  return cudaGetLastError();
}

}  // namespace nmf
