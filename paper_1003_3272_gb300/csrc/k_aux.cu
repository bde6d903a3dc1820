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
// Tile-blocked operand copy of V for the tensor-core products.  The output
// is the M x K matrix (V itself, or V^T when `transpose`) cut into blocks of
// 128 rows x KBE columns (KBE = 64 bf16 or 32 tf32 = 128 bytes); block
// (mt, kb) is stored contiguously (row pitch 128 bytes) at block index
// mt * nkb + kb, so one tile's K range is a single contiguous stream.
// mode 0: bf16 hi (and lo = bf16(v - hi) when lo != null); mode 1: tf32;
// mode 2: float32 as is.  Entries of a block outside M x K are written as 0.
//
// One CTA writes one output block: 16-byte loads of V (coalesced rows), and
// 4 consecutive K values per thread stored as one 8-byte (bf16) or 16-byte
// (float32) store, so each warp writes 256 or 512 contiguous bytes.  The
// transposed copy goes through a [KBE][128] shared-memory tile.
constexpr int kObThreads = 256;
constexpr int kObLd = 129;

__device__ __forceinline__ float4 load4(const float* s, int64_t idx, int64_t lim, bool vec) {
  // V[idx .. idx+3] with entries at or past `lim` (the row's end) read as 0
  if (vec && idx + 3 < lim) return __ldcs(reinterpret_cast<const float4*>(s + idx));
  float4 v;
  v.x = idx < lim ? __ldcs(s + idx) : 0.f;
  v.y = idx + 1 < lim ? __ldcs(s + idx + 1) : 0.f;
  v.z = idx + 2 < lim ? __ldcs(s + idx + 2) : 0.f;
  v.w = idx + 3 < lim ? __ldcs(s + idx + 3) : 0.f;
  return v;
}

__device__ __forceinline__ void store4(void* hi, void* lo, int64_t off, int mode, float4 v) {
  if (mode == 2) {
    *reinterpret_cast<float4*>(static_cast<float*>(hi) + off) = v;
  } else if (mode == 1) {
    *reinterpret_cast<float4*>(static_cast<float*>(hi) + off) =
        make_float4(round_tf32(v.x), round_tf32(v.y), round_tf32(v.z), round_tf32(v.w));
  } else {
    const float x[4] = {v.x, v.y, v.z, v.w};
    __nv_bfloat16 h[4], l[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      h[i] = __float2bfloat16_rn(x[i]);
      l[i] = __float2bfloat16_rn(__fsub_rn(x[i], __bfloat162float(h[i])));
    }
    *reinterpret_cast<uint2*>(static_cast<__nv_bfloat16*>(hi) + off) =
        *reinterpret_cast<const uint2*>(h);
    if (lo)
      *reinterpret_cast<uint2*>(static_cast<__nv_bfloat16*>(lo) + off) =
          *reinterpret_cast<const uint2*>(l);
  }
}

__global__ void __launch_bounds__(kObThreads)
k_operand_blocked(const float* __restrict__ src, int64_t rows, int64_t cols, int64_t lds,
                  int transpose, int mode, void* __restrict__ hi, void* __restrict__ lo,
                  int64_t nkb, int kbe, int vec) {
  __shared__ float T[64 * kObLd];   // transposed copy: T[k][m]
  const int64_t blk = blockIdx.x;
  const int64_t mt = blk / nkb, kb = blk % nkb;
  const int64_t m0 = mt * 128, k0 = kb * kbe;
  const int64_t M = transpose ? cols : rows, K = transpose ? rows : cols;
  const int kq = kbe / 4;                 // 4-value groups per output row
  const int nq = 128 * kq;
  const int64_t base = blk * 128 * (int64_t)kbe;
  if (transpose) {
    // source rows k0 .. k0+kbe-1 (K index), columns m0 .. m0+127 (M index)
    for (int q = threadIdx.x; q < kbe * 32; q += kObThreads) {
      const int kk = q >> 5, mq = (q & 31) * 4;
      const int64_t k = k0 + kk;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (k < K) v = load4(src + k * lds, m0 + mq, M, vec != 0);
      float* t = &T[kk * kObLd + mq];
      t[0] = v.x; t[1] = v.y; t[2] = v.z; t[3] = v.w;
    }
    __syncthreads();
#pragma unroll 4
    for (int q = threadIdx.x; q < nq; q += kObThreads) {
      const int mm = q / kq, kk = (q % kq) * 4;
      float4 v;
      v.x = T[(kk + 0) * kObLd + mm];
      v.y = T[(kk + 1) * kObLd + mm];
      v.z = T[(kk + 2) * kObLd + mm];
      v.w = T[(kk + 3) * kObLd + mm];
      store4(hi, lo, base + (int64_t)mm * kbe + kk, mode, v);
    }
  } else {
#pragma unroll 4
    for (int q = threadIdx.x; q < nq; q += kObThreads) {
      const int mm = q / kq, kk = (q % kq) * 4;
      const int64_t m = m0 + mm;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (m < M) v = load4(src + m * lds, k0 + kk, K, vec != 0);
      store4(hi, lo, base + (int64_t)mm * kbe + kk, mode, v);
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
// ty + 8a (a < 8) and columns 4 tx + b (b < 4): 16-byte loads of V and H,
// and per pair of ranks two 16-byte H loads and eight 8-byte W loads
// (broadcast within the warp) for 64 FMAs.
// ---------------------------------------------------------------------------
constexpr int kObjBM = 64, kObjBN = 128, kObjThreads = 256, kObjBlocks = 1216;

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& err) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Sums block partials into *out once every block of the grid has written
// its own: the block whose arrival on `done` is the last one adds them in
// index order (a fixed order: deterministic) and re-arms the counter.
__device__ __forceinline__ void last_block_sum(double part, double* __restrict__ partials,
                                               unsigned int* done, double* __restrict__ out) {
  __shared__ bool last;
  __shared__ double red2[kObjThreads];
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = part;
    __threadfence();
    last = atomicAdd(done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double s = 0.0;
  for (unsigned i = threadIdx.x; i < gridDim.x; i += kObjThreads) s += __ldcg(&partials[i]);
  red2[threadIdx.x] = s;
  __syncthreads();
  for (int w = kObjThreads / 2; w >= 1; w >>= 1) {
    if ((int)threadIdx.x < w) red2[threadIdx.x] += red2[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    *out = red2[0];
    *done = 0u;
  }
}

__global__ void __launch_bounds__(kObjThreads)
k_objective(const float* __restrict__ V, int64_t ldv, const float* __restrict__ W,
            const float* __restrict__ H, int64_t p, int64_t n, int r,
            double* __restrict__ partials, unsigned int* done, double* __restrict__ out) {
  extern __shared__ float sm[];
  const int rp = (r + 1) & ~1;               // even
  const int LW = rp;                         // W row stride (even: 8-byte loads)
  float* Ws = sm;                            // [kObjBM][rp]
  float* Hs = sm + kObjBM * rp;              // [rp][kObjBN]
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  const int64_t tiles_m = ceil_div(p, kObjBM), tiles_n = ceil_div(n, kObjBN);
  const int64_t ntiles = tiles_m * tiles_n;
  const bool vec_v = (ldv % 4 == 0) && (reinterpret_cast<uintptr_t>(V) % 16 == 0);
  const bool vec_h = (n % 4 == 0) && (reinterpret_cast<uintptr_t>(H) % 16 == 0);
  double acc64 = 0.0;

  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t i0 = (t / tiles_n) * kObjBM, j0 = (t % tiles_n) * kObjBN;
    __syncthreads();
    for (int q = tid; q < kObjBM * rp; q += kObjThreads) {
      const int m = q / rp, k = q % rp;
      Ws[m * LW + k] = (i0 + m < p && k < r) ? W[(i0 + m) * r + k] : 0.f;
    }
    for (int q = tid; q < rp * (kObjBN / 4); q += kObjThreads) {
      const int k = q / (kObjBN / 4), c = (q % (kObjBN / 4)) * 4;
      const int64_t j = j0 + c;
      float4 h = make_float4(0.f, 0.f, 0.f, 0.f);
      if (k < r) {
        const float* src = H + (int64_t)k * n + j;
        if (vec_h && j + 3 < n) {
          h = *reinterpret_cast<const float4*>(src);
        } else {
          h.x = j < n ? src[0] : 0.f;
          h.y = j + 1 < n ? src[1] : 0.f;
          h.z = j + 2 < n ? src[2] : 0.f;
          h.w = j + 3 < n ? src[3] : 0.f;
        }
      }
      *reinterpret_cast<float4*>(&Hs[k * kObjBN + c]) = h;
    }
    float v[8][4];
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const int64_t i = i0 + ty + 8 * a, j = j0 + 4 * tx;
      float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
      if (i < p) {
        const float* src = V + i * ldv + j;
        if (vec_v && j + 3 < n) {
          x = __ldcs(reinterpret_cast<const float4*>(src));
        } else {
          x.x = j < n ? __ldcs(src) : 0.f;
          x.y = j + 1 < n ? __ldcs(src + 1) : 0.f;
          x.z = j + 2 < n ? __ldcs(src + 2) : 0.f;
          x.w = j + 3 < n ? __ldcs(src + 3) : 0.f;
        }
      }
      v[a][0] = x.x; v[a][1] = x.y; v[a][2] = x.z; v[a][3] = x.w;
    }
    __syncthreads();
    float s0[8][4], s1[8][4];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) { s0[a][b] = 0.f; s1[a][b] = 0.f; }
    for (int k = 0; k < rp; k += 2) {
      const float4 h0 = *reinterpret_cast<const float4*>(&Hs[k * kObjBN + 4 * tx]);
      const float4 h1 = *reinterpret_cast<const float4*>(&Hs[(k + 1) * kObjBN + 4 * tx]);
      const float h0v[4] = {h0.x, h0.y, h0.z, h0.w};
      const float h1v[4] = {h1.x, h1.y, h1.z, h1.w};
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        const float2 w = *reinterpret_cast<const float2*>(&Ws[(ty + 8 * a) * LW + k]);
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          s0[a][b] = fmaf(w.x, h0v[b], s0[a][b]);
          s1[a][b] = fmaf(w.y, h1v[b], s1[a][b]);
        }
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

  // Block reduction in float64, fixed order; the grid's last block adds the
  // partials.
  __shared__ double red[kObjThreads];
  red[tid] = acc64;
  __syncthreads();
  for (int w = kObjThreads / 2; w >= 1; w >>= 1) {
    if (tid < w) red[tid] += red[tid + w];
    __syncthreads();
  }
  last_block_sum(red[0], partials, done, out);
}

// Section 3's stopping rule, |f_k - f_{k-1}| / (|f_{k-1}| + 1) < tol, taken
// in float64 with the same operations as the host-side loop (nmf_run), so
// both stop after the same iteration.
__global__ void k_run_init(RunState* s, const double* __restrict__ f_dev, int max_iters,
                           double tol) {
  const double f = *f_dev;
  s->f_prev = f;
  s->f = f;
  s->tol = tol;
  s->done = 0;
  s->checks = 0;
  s->stop = 0;
  s->max_iters = max_iters;
}

__global__ void k_run_test(RunState* s, const double* __restrict__ f_dev, int iters,
                           cudaGraphConditionalHandle loop) {
  const double f = *f_dev, fp = s->f_prev;
  s->done += iters;
  s->checks += 1;
  s->f = f;
  const bool conv = s->tol > 0.0 && fabs(f - fp) / (fabs(fp) + 1.0) < s->tol;
  if (conv) s->stop = 1;
  else s->f_prev = f;
  const bool more = !conv && s->max_iters - s->done >= iters;
  cudaGraphSetConditional(loop, more ? 1u : 0u);
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

cudaError_t launch_operand_blocked(const float* src, int64_t rows, int64_t cols, int64_t lds,
                                   bool transpose, int mode, void* hi, void* lo, int64_t nkb,
                                   int kbe, cudaStream_t st) {
  if (kbe % 4 != 0 || kbe > 64) return cudaErrorInvalidValue;
  const int64_t M = transpose ? cols : rows;
  const int64_t blocks = ceil_div(M, 128) * nkb;
  if (blocks <= 0) return cudaSuccess;
  if (blocks > INT32_MAX) return cudaErrorInvalidValue;
  const int vec = (lds % 4 == 0 && reinterpret_cast<uintptr_t>(src) % 16 == 0) ? 1 : 0;
  k_operand_blocked<<<(unsigned)blocks, kObThreads, 0, st>>>(src, rows, cols, lds,
                                                            transpose ? 1 : 0, mode, hi, lo, nkb,
                                                            kbe, vec);
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

cudaError_t launch_run_init(RunState* s, const double* f_dev, int max_iters, double tol,
                            cudaStream_t st) {
  k_run_init<<<1, 1, 0, st>>>(s, f_dev, max_iters, tol);
  return cudaGetLastError();
}

cudaError_t launch_run_test(RunState* s, const double* f_dev, int iters,
                            cudaGraphConditionalHandle loop, cudaStream_t st) {
  k_run_test<<<1, 1, 0, st>>>(s, f_dev, iters, loop);
  return cudaGetLastError();
}

// Partials plus the arrival counter of the last-block sum (zeroed at
// allocation, re-armed by every launch).
int objective_parts() { return kObjBlocks + 1; }

cudaError_t launch_objective(const float* V, int64_t ldv, const float* W, const float* H,
                             int64_t p, int64_t n, int r, double* partials, int nparts,
                             double* f_dev, cudaStream_t st) {
  const int rp = (r + 1) & ~1;
  const size_t smem = ((size_t)kObjBM * rp + (size_t)rp * kObjBN) * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(k_objective, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  // one block per tile up to kObjBlocks; the counter sits after the partials
  const int64_t tiles = ceil_div(p, kObjBM) * ceil_div(n, kObjBN);
  const int grid = (int)(tiles < kObjBlocks ? (tiles < 1 ? 1 : tiles) : kObjBlocks);
  if (nparts < kObjBlocks + 1) return cudaErrorInvalidValue;
  unsigned int* done = reinterpret_cast<unsigned int*>(partials + kObjBlocks);
  k_objective<<<grid, kObjThreads, smem, st>>>(V, ldv, W, H, p, n, r, partials, done, f_dev);
  return cudaGetLastError();
}

}  // namespace nmf

// ---------------------------------------------------------------------------
// Self-check of div_rn against the IEEE division: case i < 2^23 * nx sweeps
// every significand of d in [1, 2) against nx significands of x (drawn from
// the counter generator, with exponents spread over the quick range); the
// remaining cases draw both operands at random (x = 0 included).
// ---------------------------------------------------------------------------
namespace nmf {
namespace {

__global__ void k_selfcheck_div(uint64_t key, int64_t count, int nx,
                                unsigned long long* mismatches, unsigned long long* quick) {
  unsigned long long bad = 0, fast = 0;
  const int64_t sweep = (int64_t)nx << 23;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t bx, bd;
    if (i < sweep) {
      const uint64_t w = mix64(key + (uint64_t)(i >> 23) * kGolden);
      const uint32_t ex = 64u + (uint32_t)(w % 127u);          // 2^-63 .. 2^63
      bx = (ex << 23) | (uint32_t)((w >> 20) & 0x7fffffu);
      const uint32_t ed = 64u + (uint32_t)((w >> 50) % 127u);
      bd = (ed << 23) | (uint32_t)(i & 0x7fffff);
    } else {
      const uint64_t w = mix64(key + (uint64_t)(i + 1) * kGolden);
      bx = (uint32_t)(1u + (w % 253u)) << 23 | (uint32_t)((w >> 8) & 0x7fffffu);
      bd = (uint32_t)(1u + ((w >> 32) % 253u)) << 23 | (uint32_t)((w >> 40) & 0x7fffffu);
      if ((w & 0xffu) == 0u) bx = 0u;
    }
    const float x = __uint_as_float(bx), d = __uint_as_float(bd);
    const float a = div_rn(x, d), b = __fdiv_rn(x, d);
    if (__float_as_uint(a) != __float_as_uint(b)) ++bad;
    if (div_rn_quick_ok(x, d)) ++fast;
  }
  if (bad) atomicAdd(mismatches, bad);
  atomicAdd(quick, fast);
}

}  // namespace
}  // namespace nmf

extern "C" nmf_status nmf_selfcheck_div(int64_t count, uint64_t seed, uint64_t* mismatches,
                                        uint64_t* quick) {
  using namespace nmf;
  if (count < 0 || !mismatches || !quick) {
    record_error("nmf_selfcheck_div: count must be >= 0 and the outputs non-null");
    return NMF_EINVAL;
  }
  unsigned long long* d = nullptr;
  cudaError_t e = cudaMalloc(&d, 2 * sizeof(unsigned long long));
  if (e != cudaSuccess) { record_error("nmf_selfcheck_div: cudaMalloc failed"); return NMF_ENOMEM; }
  unsigned long long h[2] = {0, 0};
  e = cudaMemset(d, 0, sizeof(h));
  const int nx = 64;
  if (e == cudaSuccess) {
    k_selfcheck_div<<<1216, 256>>>(mix64(seed), count, nx, d, d + 1);
    count_launches(1);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) {
    record_error(cudaGetErrorString(e));
    return NMF_ECUDA;
  }
  *mismatches = h[0];
  *quick = h[1];
  return NMF_OK;
}

