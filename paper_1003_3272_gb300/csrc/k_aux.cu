// Auxiliary kernels of the MM NMF path: Algorithm 1's seeded start, the
// operand copies of V, the Gram matrices of the factors and the Frobenius
// objective (Eq. (3.1)).
#include "nmf_internal.cuh"

namespace nmf {
namespace {

// ---------------------------------------------------------------------------
// Algorithm 1's start: iid uniform(0,1) draws.  Counter-based SplitMix64
// (Steele, Lea & Flood 2014): word i of stream s under `seed` is
//   mix64(mix64(seed + (s+1) G) + (i+1) G),  G = 0x9E3779B97F4A7C15,
// and the open-interval uniform is ((word >> 41) + 1/2) * 2^-23, exact in
// float32 and strictly inside (0, 1).
// ---------------------------------------------------------------------------
__host__ __device__ inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ull;

__global__ void k_seed_uniform(float* dst, int64_t count, uint64_t key) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t w = mix64(key + (uint64_t)(i + 1) * kGolden);
    dst[i] = ((float)(uint32_t)(w >> 41) + 0.5f) * 0x1p-23f;
  }
}

// ---------------------------------------------------------------------------
// Operand copies of V.
// ---------------------------------------------------------------------------
__global__ void k_copy_pad(const float* __restrict__ src, int64_t rows, int64_t cols,
                           int64_t lds, float* __restrict__ dst, int64_t ldd, int tf32) {
  const int64_t total = rows * ldd;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / ldd, c = i % ldd;
    const float v = c < cols ? src[r * lds + c] : 0.f;
    dst[i] = tf32 ? round_tf32(v) : v;
  }
}

// dst (cols x ldd) = src (rows x cols)^T, zero in columns rows..ldd-1.
__global__ void k_transpose_pad(const float* __restrict__ src, int64_t rows, int64_t cols,
                                int64_t lds, float* __restrict__ dst, int64_t ldd, int tf32) {
  __shared__ float t[32][33];
  const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int64_t r = r0 + y, c = c0 + threadIdx.x;
    t[y][threadIdx.x] = (r < rows && c < cols) ? src[r * lds + c] : 0.f;
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int64_t c = c0 + y, r = r0 + threadIdx.x;  // dst row c, column r
    if (c < cols && r < ldd) {
      const float v = t[threadIdx.x][y];
      dst[c * ldd + r] = tf32 ? round_tf32(v) : v;
    }
  }
}

// hi = bf16(v), lo = bf16(v - hi); optional transpose; zero padding.
__global__ void k_split_bf16(const float* __restrict__ src, int64_t rows, int64_t cols,
                             int64_t lds, int transpose, __nv_bfloat16* __restrict__ hi,
                             __nv_bfloat16* __restrict__ lo, int64_t ldd) {
  __shared__ float t[32][33];
  const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int64_t r = r0 + y, c = c0 + threadIdx.x;
    t[y][threadIdx.x] = (r < rows && c < cols) ? src[r * lds + c] : 0.f;
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    int64_t orow, ocol;
    float v;
    if (transpose) { orow = c0 + y; ocol = r0 + threadIdx.x; v = t[threadIdx.x][y];
                     if (orow >= cols) continue; }
    else           { orow = r0 + y; ocol = c0 + threadIdx.x; v = t[y][threadIdx.x];
                     if (orow >= rows) continue; }
    if (ocol >= ldd) continue;
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    hi[orow * ldd + ocol] = h;
    if (lo) lo[orow * ldd + ocol] = __float2bfloat16_rn(__fsub_rn(v, __bfloat162float(h)));
  }
}

// Tile-blocked operand copy of V for the tensor-core products.  The output
// is the M x K matrix (V itself, or V^T when `transpose`) cut into blocks of
// 128 rows x KBE columns (KBE = 64 bf16 or 32 tf32 = 128 bytes); block
// (mt, kb) is stored contiguously (row pitch 128 bytes) at block index
// mt * nkb + kb, so one tile's K range is a single contiguous stream.
// mode 0: bf16 hi (and lo = bf16(v - hi) when lo != null); mode 1: tf32;
// mode 2: float32 as is.
// Entries outside M x K are never written (the buffer starts zeroed).
__global__ void k_operand_blocked(const float* __restrict__ src, int64_t rows, int64_t cols,
                                  int64_t lds, int transpose, int mode, void* __restrict__ hi,
                                  void* __restrict__ lo, int64_t nkb, int kbe) {
  __shared__ float t[32][33];
  const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int64_t r = r0 + y, c = c0 + threadIdx.x;
    t[y][threadIdx.x] = (r < rows && c < cols) ? src[r * lds + c] : 0.f;
  }
  __syncthreads();
  const int64_t M = transpose ? cols : rows, K = transpose ? rows : cols;
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    int64_t m, k;
    float v;
    if (transpose) { m = c0 + y; k = r0 + threadIdx.x; v = t[threadIdx.x][y]; }
    else           { m = r0 + y; k = c0 + threadIdx.x; v = t[y][threadIdx.x]; }
    if (m >= M || k >= K) continue;
    const int64_t off = (((m >> 7) * nkb + k / kbe) * 128 + (m & 127)) * kbe + (k % kbe);
    if (mode == 1) {
      static_cast<float*>(hi)[off] = round_tf32(v);
    } else if (mode == 2) {
      static_cast<float*>(hi)[off] = v;
    } else {
      const __nv_bfloat16 h = __float2bfloat16_rn(v);
      static_cast<__nv_bfloat16*>(hi)[off] = h;
      if (lo)
        static_cast<__nv_bfloat16*>(lo)[off] =
            __float2bfloat16_rn(__fsub_rn(v, __bfloat162float(h)));
    }
  }
}

// Operand plane(s) [k][m] of a factor: W (row-major p x r, plane = W^T) or
// H (r x n, plane = H itself), in the precision of the streaming product.
__global__ void k_factor_planes(const float* __restrict__ F, int layout, int64_t M,
                                int64_t ldf, int r, void* op_hi, void* op_lo, int64_t ldop,
                                int plane) {
  const int64_t total = (int64_t)r * M;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(i / M);
    const int64_t m = i % M;
    const float v = layout == kFactorRowMajor ? F[m * r + k] : F[(int64_t)k * ldf + m];
    const int64_t off = (int64_t)k * ldop + m;
    if (plane == kPlaneF32) {
      static_cast<float*>(op_hi)[off] = v;
    } else if (plane == kPlaneTF32) {
      static_cast<float*>(op_hi)[off] = round_tf32(v);
    } else {
      const __nv_bfloat16 h = __float2bfloat16_rn(v);
      static_cast<__nv_bfloat16*>(op_hi)[off] = h;
      if (plane == kPlaneBF16x2)
        static_cast<__nv_bfloat16*>(op_lo)[off] =
            __float2bfloat16_rn(__fsub_rn(v, __bfloat162float(h)));
    }
  }
}

__global__ void k_validate(const float* __restrict__ V, int64_t rows, int64_t cols,
                           int* flag) {
  const int64_t total = rows * cols;
  int bad = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float v = V[i];
    bad |= !(v >= 0.f) || isinf(v);  // catches NaN, negatives, +inf
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1);
}

// ---------------------------------------------------------------------------
// Gram matrices.  Partial sums over tiles of 128 rows of the factor (rows of
// W, columns of H) in float32, then the cross-tile sum in float64 in tile
// order.
// ---------------------------------------------------------------------------
constexpr int kGramBM = 128;

__global__ void k_gram_tiles(const float* __restrict__ F, int layout, int64_t M, int64_t ldf,
                             int r, float* __restrict__ part) {
  extern __shared__ float Ts[];  // [kGramBM][r + 1]
  const int LD = r + 1;
  const int64_t m0 = (int64_t)blockIdx.x * kGramBM;
  const int rows = (int)min((int64_t)kGramBM, M - m0);
  for (int i = threadIdx.x; i < kGramBM * r; i += blockDim.x) {
    int m, k;
    if (layout == kFactorRowMajor) { m = i / r; k = i % r; }
    else                           { k = i / kGramBM; m = i % kGramBM; }
    float v = 0.f;
    if (m < rows) v = layout == kFactorRowMajor ? F[(m0 + m) * r + k] : F[(int64_t)k * ldf + m0 + m];
    Ts[m * LD + k] = v;
  }
  __syncthreads();
  float* P = part + (int64_t)blockIdx.x * r * r;
  const int npairs = r * (r + 1) / 2;
  for (int it = threadIdx.x; it < npairs; it += blockDim.x) {
    int k = 0, rem = it;
    while (rem >= r - k) { rem -= r - k; ++k; }
    const int l = k + rem;
    float s = 0.f;
    for (int m = 0; m < rows; ++m) s = fmaf(Ts[m * LD + k], Ts[m * LD + l], s);
    P[k * r + l] = s;
    P[l * r + k] = s;
  }
}

// One warp per Gram entry: lane t sums tiles t, t+32, ... in float64, then a
// fixed shuffle tree combines the lanes (deterministic order).
__global__ void k_gram_reduce(const float* __restrict__ part, int tiles, int r,
                              float* __restrict__ G32, double* __restrict__ G64) {
  const int rr = r * r;
  const int e = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (e >= rr) return;
  double s = 0.0;
  for (int t = lane; t < tiles; t += 32) s += (double)__ldcg(part + (int64_t)t * rr + e);
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) {
    G64[e] = s;
    G32[e] = (float)s;
  }
}

// ---------------------------------------------------------------------------
// Objective f = ||V - W H||_F^2 (Eq. (3.1)), direct residual.
// Each (i, j) entry of W H is a rank-r dot product accumulated in two float32
// FMA chains (even and odd k), combined by an error-free TwoSum into an
// unevaluated pair hi + lo; the residual is (v - hi) - lo.  Squares are
// summed pairwise per thread (32 entries per tile), then in float64 across
// tiles, then across threads and blocks in a fixed order.
// Tile: 64 rows x 128 columns of V; 256 threads; thread (ty, tx) owns rows
// ty + 8a (a < 8) and columns tx + 32b (b < 4).
// ---------------------------------------------------------------------------
constexpr int kObjBM = 64, kObjBN = 128, kObjThreads = 256, kObjBlocks = 1216;

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& err) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__global__ void __launch_bounds__(kObjThreads)
k_objective(const float* __restrict__ V, int64_t ldv, const float* __restrict__ W,
            const float* __restrict__ H, int64_t p, int64_t n, int r,
            double* __restrict__ partials) {
  extern __shared__ float sm[];
  const int rp = (r + 1) & ~1;               // even
  float* Ws = sm;                            // [kObjBM][rp + 1]
  float* Hs = sm + kObjBM * (rp + 1);        // [rp][kObjBN]
  const int LW = rp + 1;
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  const int64_t tiles_m = ceil_div(p, kObjBM), tiles_n = ceil_div(n, kObjBN);
  const int64_t ntiles = tiles_m * tiles_n;
  double acc64 = 0.0;

  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t i0 = (t / tiles_n) * kObjBM, j0 = (t % tiles_n) * kObjBN;
    __syncthreads();
    for (int q = tid; q < kObjBM * rp; q += kObjThreads) {
      const int m = q / rp, k = q % rp;
      Ws[m * LW + k] = (i0 + m < p && k < r) ? W[(i0 + m) * r + k] : 0.f;
    }
    for (int q = tid; q < rp * kObjBN; q += kObjThreads) {
      const int k = q / kObjBN, c = q % kObjBN;
      Hs[k * kObjBN + c] = (j0 + c < n && k < r) ? H[(int64_t)k * n + j0 + c] : 0.f;
    }
    float v[8][4];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int64_t i = i0 + ty + 8 * a, j = j0 + tx + 32 * b;
        v[a][b] = (i < p && j < n) ? __ldcs(V + i * ldv + j) : 0.f;
      }
    __syncthreads();
    float s0[8][4], s1[8][4];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) { s0[a][b] = 0.f; s1[a][b] = 0.f; }
    for (int k = 0; k < rp; k += 2) {
      float h0[4], h1[4], w0[8], w1[8];
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        h0[b] = Hs[k * kObjBN + tx + 32 * b];
        h1[b] = Hs[(k + 1) * kObjBN + tx + 32 * b];
      }
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        w0[a] = Ws[(ty + 8 * a) * LW + k];
        w1[a] = Ws[(ty + 8 * a) * LW + k + 1];
      }
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          s0[a][b] = fmaf(w0[a], h0[b], s0[a][b]);
          s1[a][b] = fmaf(w1[a], h1[b], s1[a][b]);
        }
    }
    float sq[32];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        float hi, lo;
        two_sum(s0[a][b], s1[a][b], hi, lo);
        const float d = __fsub_rn(__fsub_rn(v[a][b], hi), lo);
        sq[a * 4 + b] = __fmul_rn(d, d);  // zero for padded entries (v = hi = lo = 0)
      }
#pragma unroll
    for (int w = 16; w >= 1; w >>= 1)
#pragma unroll
      for (int q = 0; q < w; ++q) sq[q] = __fadd_rn(sq[q], sq[q + w]);
    acc64 += (double)sq[0];
  }

  // Block reduction in float64, fixed order.
  __shared__ double red[kObjThreads];
  red[tid] = acc64;
  __syncthreads();
  for (int w = kObjThreads / 2; w >= 1; w >>= 1) {
    if (tid < w) red[tid] += red[tid + w];
    __syncthreads();
  }
  if (tid == 0) partials[blockIdx.x] = red[0];
}

__global__ void k_sum_partials(const double* __restrict__ partials, int nparts,
                               double* __restrict__ out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < nparts; i += 256) s += partials[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w >= 1; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

inline unsigned grid_for(int64_t total, int threads, unsigned cap = 152u * 16u) {
  const int64_t g = ceil_div(total, threads);
  return (unsigned)(g < 1 ? 1 : (g > cap ? cap : g));
}

}  // namespace

cudaError_t launch_seed_uniform(float* dst, int64_t count, uint64_t seed, uint64_t stream_id,
                                cudaStream_t st) {
  const uint64_t key = mix64(seed + (stream_id + 1) * kGolden);
  k_seed_uniform<<<grid_for(count, 256), 256, 0, st>>>(dst, count, key);
  return cudaGetLastError();
}

cudaError_t launch_copy_pad(const float* src, int64_t rows, int64_t cols, int64_t lds,
                            float* dst, int64_t ldd, bool tf32, cudaStream_t st) {
  k_copy_pad<<<grid_for(rows * ldd, 256), 256, 0, st>>>(src, rows, cols, lds, dst, ldd,
                                                          tf32 ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_transpose_pad(const float* src, int64_t rows, int64_t cols, int64_t lds,
                                 float* dst, int64_t ldd, bool tf32, cudaStream_t st) {
  // dst columns run over src rows 0..ldd-1 (zero beyond rows)
  dim3 grid((unsigned)ceil_div(cols, 32), (unsigned)ceil_div(ldd, 32));
  k_transpose_pad<<<grid, dim3(32, 8), 0, st>>>(src, rows, cols, lds, dst, ldd, tf32 ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_split_bf16(const float* src, int64_t rows, int64_t cols, int64_t lds,
                              bool transpose, __nv_bfloat16* hi, __nv_bfloat16* lo,
                              int64_t ldd, cudaStream_t st) {
  // grid covers the padded output extent
  const int64_t gr = transpose ? ldd : rows;
  const int64_t gc = transpose ? cols : ldd;
  dim3 grid((unsigned)ceil_div(gc, 32), (unsigned)ceil_div(gr, 32));
  k_split_bf16<<<grid, dim3(32, 8), 0, st>>>(src, rows, cols, lds, transpose ? 1 : 0, hi, lo,
                                              ldd);
  return cudaGetLastError();
}

cudaError_t launch_operand_blocked(const float* src, int64_t rows, int64_t cols, int64_t lds,
                                   bool transpose, int mode, void* hi, void* lo, int64_t nkb,
                                   int kbe, cudaStream_t st) {
  dim3 grid((unsigned)ceil_div(cols, 32), (unsigned)ceil_div(rows, 32));
  k_operand_blocked<<<grid, dim3(32, 8), 0, st>>>(src, rows, cols, lds, transpose ? 1 : 0, mode,
                                                   hi, lo, nkb, kbe);
  return cudaGetLastError();
}

cudaError_t launch_factor_planes(const float* F, int layout, int64_t M, int64_t ldf, int r,
                                 void* op_hi, void* op_lo, int64_t ldop, int plane,
                                 cudaStream_t st) {
  k_factor_planes<<<grid_for((int64_t)r * M, 256), 256, 0, st>>>(F, layout, M, ldf, r, op_hi,
                                                                   op_lo, ldop, plane);
  return cudaGetLastError();
}

cudaError_t launch_validate(const float* V, int64_t rows, int64_t cols, int* flag,
                            cudaStream_t st) {
  k_validate<<<grid_for(rows * cols, 256), 256, 0, st>>>(V, rows, cols, flag);
  return cudaGetLastError();
}

cudaError_t launch_gram_tiles(const float* F, int layout, int64_t M, int64_t ldf, int r,
                              float* gram_part, int block_m, cudaStream_t st) {
  (void)block_m;
  const size_t smem = (size_t)kGramBM * (r + 1) * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(k_gram_tiles, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_gram_tiles<<<(unsigned)ceil_div(M, kGramBM), 256, smem, st>>>(F, layout, M, ldf, r,
                                                                    gram_part);
  return cudaGetLastError();
}

cudaError_t launch_gram_reduce(const float* gram_part, int tiles, int r, float* G32,
                               double* G64, cudaStream_t st) {
  const int rr = r * r;
  k_gram_reduce<<<(unsigned)ceil_div(rr, 8), 256, 0, st>>>(gram_part, tiles, r, G32, G64);
  return cudaGetLastError();
}

int objective_parts() { return kObjBlocks; }

cudaError_t launch_objective(const float* V, int64_t ldv, const float* W, const float* H,
                             int64_t p, int64_t n, int r, double* partials, int nparts,
                             double* f_dev, cudaStream_t st) {
  const int rp = (r + 1) & ~1;
  const size_t smem = ((size_t)kObjBM * (rp + 1) + (size_t)rp * kObjBN) * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(k_objective, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_objective<<<nparts, kObjThreads, smem, st>>>(V, ldv, W, H, p, n, r, partials);
  k_sum_partials<<<1, 256, 0, st>>>(partials, nparts, f_dev);
  return cudaGetLastError();
}

}  // namespace nmf
