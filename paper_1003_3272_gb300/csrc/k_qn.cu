// Vector kernels of the quasi-Newton acceleration of the MM map (the scheme
// the paper names in Section 4; Zhou, Alexander & Lange): the secant pair of
// an iteration, the float64 inner products of the secant memory, and the
// quasi-Newton point F(x_n) + V c with its sign check.  The state x stacks W
// (p x r) and H (r x n), N = (p + n) r entries.  Fixed reduction orders: the
// results are deterministic.
#include "nmf_internal.cuh"

namespace nmf {
namespace {

constexpr int kQThreads = 256;

// u = x1 - x0, v = x2 - x1 (float32, as the iterates are).
__global__ void k_qn_secant(float* __restrict__ u, float* __restrict__ v,
                            const float* __restrict__ x0, const float* __restrict__ x1,
                            const float* __restrict__ x2, int64_t N) {
  for (int64_t i = (int64_t)blockIdx.x * kQThreads + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * kQThreads) {
    const float a = x1[i];
    u[i] = __fsub_rn(a, x0[i]);
    v[i] = __fsub_rn(x2[i], a);
  }
}

// Block (chunk c, pair d): the chunk's share of <a_d, b_d> in float64 (exact
// products of the float32 entries; per-thread sums in index order, then a
// fixed tree) into part[d * chunks + c].
__global__ void k_qn_dot_parts(const float* const* __restrict__ a, const float* const* __restrict__ b,
                               int64_t N, int64_t chunk, double* __restrict__ part) {
  __shared__ double red[kQThreads];
  const int d = blockIdx.y, c = blockIdx.x;
  const float* x = a[d];
  const float* y = b[d];
  const int64_t i0 = (int64_t)c * chunk;
  const int64_t i1 = min(N, i0 + chunk);
  double s = 0.0;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += kQThreads) s += (double)x[i] * (double)y[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = kQThreads / 2; w >= 1; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[(int64_t)d * gridDim.x + c] = red[0];
}

// out[d] = sum over chunks of part[d][.] in chunk order.
__global__ void k_qn_dot_sum(const double* __restrict__ part, int chunks, int ndots,
                             double* __restrict__ out) {
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= ndots) return;
  double s = 0.0;
  for (int c = 0; c < chunks; ++c) s += part[(int64_t)d * chunks + c];
  out[d] = s;
}

// x = x1 + sum_j coef[j] V_j in float64, rounded once to float32, written to
// W (entries [0, nw)) and H (the rest); *neg = 1 if an entry is negative or
// not finite (NaN fails the x >= 0 test), so such a point is never taken.
__global__ void k_qn_combine(float* __restrict__ W, float* __restrict__ H, int64_t nw, int64_t N,
                             const float* __restrict__ x1, const float* const* __restrict__ Vj,
                             const double* __restrict__ coef, int m, int* __restrict__ neg) {
  for (int64_t i = (int64_t)blockIdx.x * kQThreads + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * kQThreads) {
    double x = (double)x1[i];
    for (int j = 0; j < m; ++j) x = fma(coef[j], (double)Vj[j][i], x);
    const float xf = (float)x;
    if (!(xf >= 0.f) || isinf(xf)) atomicExch(neg, 1);
    if (i < nw) W[i] = xf;
    else H[i - nw] = xf;
  }
}

inline unsigned grid_n(int64_t N) {
  const int64_t g = (N + kQThreads - 1) / kQThreads;
  return (unsigned)(g < 1 ? 1 : (g > 152 * 8 ? 152 * 8 : g));
}

}  // namespace

int qn_dot_chunks(int64_t N) {
  const int64_t c = (N + 16383) / 16384;   // 16K entries per block
  return (int)(c < 1 ? 1 : (c > 1024 ? 1024 : c));
}

cudaError_t qn_secant(float* u, float* v, const float* x0, const float* x1, const float* x2,
                      int64_t N, cudaStream_t st) {
  k_qn_secant<<<grid_n(N), kQThreads, 0, st>>>(u, v, x0, x1, x2, N);
  return cudaGetLastError();
}

cudaError_t qn_dots(const float* const* a, const float* const* b, int ndots, int64_t N,
                    double* part, double* out, cudaStream_t st) {
  if (ndots <= 0) return cudaSuccess;
  const int chunks = qn_dot_chunks(N);
  const int64_t chunk = (N + chunks - 1) / chunks;
  k_qn_dot_parts<<<dim3((unsigned)chunks, (unsigned)ndots), kQThreads, 0, st>>>(a, b, N, chunk,
                                                                                 part);
  k_qn_dot_sum<<<(ndots + 63) / 64, 64, 0, st>>>(part, chunks, ndots, out);
  return cudaGetLastError();
}

cudaError_t qn_combine(float* W, float* H, int64_t nw, int64_t N, const float* x1,
                       const float* const* Vj, const double* coef, int m, int* neg,
                       cudaStream_t st) {
  k_qn_combine<<<grid_n(N), kQThreads, 0, st>>>(W, H, nw, N, x1, Vj, coef, m, neg);
  return cudaGetLastError();
}

}  // namespace nmf
