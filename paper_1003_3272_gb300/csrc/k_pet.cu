// Penalised PET reconstruction by MM (Section 3.2, Algorithm 2): kernels and
// the C ABI of include/pet.h.
//
// One iteration of Algorithm 2 for K images at once (one per penalty
// constant mu_k; they share E, y and the neighbourhood system):
//
//   k_pet_forward   a warp per line i, one block per SM, u staged in shared
//                   memory: s_ki = sum_j e_ij u_kj with
//                   u_kj = lambda_kj / sigma_j (sigma_j = sum_i e_ij, so
//                   this is the projection through the unit-column-sum E of
//                   Algorithm 2's first step), then r_ki = y_i / s_ki
//                   (0 when y_i = 0).  E is read once for all K images.
//   k_pet_back      a block per (128-column block, segment of lines): warp w
//                   sums e_ij r_ki over lines w, w + 8, ... of the segment
//                   (16-byte loads of E, four lines in flight), the eight
//                   warps' sums are added in warp order and stored as the
//                   segment's partial; the block that finishes a column
//                   block last (arrival counter) adds the segments' partials
//                   in segment order in float64 and applies the update:
//                     c_j = lambda_j t_j / sigma_j        (t_j = sum_i e_ij r_i)
//                     b_j = mu (|N_j| lambda_j + sum_{k in N_j} lambda_k) - 1
//                     a_j = -2 mu |N_j|
//                     lambda_j <- positive root of a x^2 + b x + c = 0
//                   in float64, the root taken as 2c / (-b + sqrt(b^2 - 4ac))
//                   when b <= 0 (the paper's (-b - sqrt(.)) / (2a) cancels
//                   there; the two are the same root) and in the paper's
//                   form when b > 0; mu = 0 gives the EM update c_j.
//
// The new intensities go to the other of two buffers (neighbours are read
// from the old one), so an iteration has no read-after-write hazard; the
// context copies back when an odd number of iterations ends in the work
// buffer.  Every sum runs in a fixed order: the results do not depend on
// scheduling.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "nmf_internal.cuh"
#include "pet.h"

using namespace nmf;

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kColBlock = 128;      // columns per back-projection block (32 lanes x 4)
constexpr int kRowChunk = 1024;     // lines of ratios staged per pass of the back projection
constexpr int kFwdThreads = 512;    // forward projection: one block per SM
constexpr int kFwdRows = 4;         // lines a forward warp carries per pass
constexpr int kFwdSmem = 96 * 1024; // shared memory for the staged u chunk
constexpr int kMaxImages = 8;
constexpr int kObjBlocks = 304;     // objective: fixed grid (2 x 152), fixed order

thread_local std::string g_pet_error = "no error";

void pet_set_err(std::string* dst, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_pet_error = buf;
  record_error(buf);
  if (dst) *dst = buf;
}

// ---------------------------------------------------------------------------
// set-up kernels
// ---------------------------------------------------------------------------

// sigma_j = sum_i e_ij in float64 (lines in order); flags: 1 = an entry of E
// is negative or not finite, 8 = a column sums to zero.
__global__ void k_pet_colsum(const float* __restrict__ E, int64_t d, int64_t p,
                             double* __restrict__ sigma, int* __restrict__ flag) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < p;
       j += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    bool bad = false;
    for (int64_t i = 0; i < d; ++i) {
      const float e = E[i * p + j];
      bad |= !(e >= 0.f) || isinf(e);
      s += (double)e;
    }
    sigma[j] = s;
    if (bad) atomicOr(flag, 1);
    if (!(s > 0.0)) atomicOr(flag, 8);
  }
}

// flags: 2 = a count is negative or not finite, 4 = a starting intensity is.
__global__ void k_pet_check(const float* __restrict__ v, int64_t n, int bit,
                            int* __restrict__ flag) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float x = v[i];
    if (!(x >= 0.f) || isinf(x)) atomicOr(flag, bit);
  }
}

// Optionally lambda = 1 (Algorithm 2's start); u = lambda / sigma (float32).
__global__ void k_pet_start(float* __restrict__ lam, float* __restrict__ u,
                            const double* __restrict__ sigma, int64_t p, int nimg, int ones) {
  const int64_t n = (int64_t)nimg * p;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x) {
    if (ones) lam[q] = 1.0f;
    u[q] = (float)((double)lam[q] / sigma[q % p]);
  }
}

// ---------------------------------------------------------------------------
// the iteration
// ---------------------------------------------------------------------------

template <int K>
__device__ __forceinline__ void warp_sum(float (&a)[K]) {
#pragma unroll
  for (int k = 0; k < K; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a[k] += __shfl_xor_sync(0xffffffffu, a[k], o);
}

// Forward projection and ratios.  One block of kFwdThreads per SM
// (persistent); the grid's warps take the lines round-robin (warp g: lines
// g, g + G, ..., G = the grid's warps), at most kFwdRows per warp per pass.
// The scaled intensities u are staged in shared memory a column chunk at a
// time (all K images; one chunk covers the row when it fits), so E is the
// only operand streamed from memory and u is read from L2 once per block
// and chunk instead of once per line.  Lane l reads columns 4l + 128 t of a
// chunk (VEC: 16-byte loads; p a multiple of 4 and E 16-byte aligned) or
// l + 32 t (element loads), eight loads in flight; the lanes' partial sums
// are added by a fixed butterfly and the chunks in order, so the result
// does not depend on the grid.
template <int K, bool VEC>
__global__ void __launch_bounds__(kFwdThreads)
k_pet_forward(const float* __restrict__ E, int64_t d, int64_t p, const float* __restrict__ u,
              const float* __restrict__ y, float* __restrict__ r, int cw) {
  extern __shared__ __align__(16) float us[];   // [K][cw]
  const int lane = threadIdx.x & 31;
  constexpr int W = kFwdThreads / 32;
  const int64_t G = (int64_t)gridDim.x * W;
  const int64_t g = (int64_t)blockIdx.x * W + (threadIdx.x >> 5);
  for (int64_t pass = 0; pass * G * kFwdRows < d; ++pass) {
    const int64_t first = pass * G * kFwdRows + g;   // lines first + G t, t < kFwdRows
    float acc[kFwdRows][K];
#pragma unroll
    for (int t = 0; t < kFwdRows; ++t)
#pragma unroll
      for (int k = 0; k < K; ++k) acc[t][k] = 0.f;
    for (int64_t c0 = 0; c0 < p; c0 += cw) {
      const int w = (int)min((int64_t)cw, p - c0);
      __syncthreads();   // the previous chunk is consumed
      if (VEC) {
        for (int q = threadIdx.x; q < K * (cw / 4); q += kFwdThreads) {
          const int k = q / (cw / 4), c = 4 * (q % (cw / 4));
          *reinterpret_cast<float4*>(us + (int64_t)k * cw + c) =
              c < w ? __ldg(reinterpret_cast<const float4*>(u + (int64_t)k * p + c0 + c))
                    : make_float4(0.f, 0.f, 0.f, 0.f);
        }
      } else {
        for (int q = threadIdx.x; q < K * cw; q += kFwdThreads) {
          const int k = q / cw, c = q % cw;
          us[(int64_t)k * cw + c] = c < w ? __ldg(u + (int64_t)k * p + c0 + c) : 0.f;
        }
      }
      __syncthreads();
      // the warp's lines together: each staged value of u serves all of them
      bool live[kFwdRows];
      const float* e[kFwdRows];
#pragma unroll
      for (int t = 0; t < kFwdRows; ++t) {
        live[t] = first + G * t < d;
        e[t] = E + (live[t] ? first + G * t : 0) * p + c0;
      }
      if (VEC) {
        // U column steps of all the warp's lines loaded before any is used:
        // up to U * kFwdRows 16-byte loads in flight per lane
        constexpr int U = K <= 2 ? 4 : (K <= 4 ? 2 : 1);
        for (int c = 4 * lane; c < w; c += 128 * U) {
          float4 ev[U][kFwdRows];
#pragma unroll
          for (int v = 0; v < U; ++v)
#pragma unroll
            for (int t = 0; t < kFwdRows; ++t)
              ev[v][t] = (live[t] && c + 128 * v < w)
                             ? __ldcs(reinterpret_cast<const float4*>(e[t] + c + 128 * v))
                             : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
          for (int v = 0; v < U; ++v) {
            if (c + 128 * v >= w) continue;
#pragma unroll
            for (int k = 0; k < K; ++k) {
              const float4 uv = *reinterpret_cast<const float4*>(us + (int64_t)k * cw + c + 128 * v);
#pragma unroll
              for (int t = 0; t < kFwdRows; ++t) {
                acc[t][k] = fmaf(ev[v][t].x, uv.x, acc[t][k]);
                acc[t][k] = fmaf(ev[v][t].y, uv.y, acc[t][k]);
                acc[t][k] = fmaf(ev[v][t].z, uv.z, acc[t][k]);
                acc[t][k] = fmaf(ev[v][t].w, uv.w, acc[t][k]);
              }
            }
          }
        }
      } else {
#pragma unroll 2
        for (int c = lane; c < w; c += 32) {
          float ev[kFwdRows];
#pragma unroll
          for (int t = 0; t < kFwdRows; ++t) ev[t] = live[t] ? __ldcs(e[t] + c) : 0.f;
#pragma unroll
          for (int k = 0; k < K; ++k) {
            const float uv = us[(int64_t)k * cw + c];
#pragma unroll
            for (int t = 0; t < kFwdRows; ++t) acc[t][k] = fmaf(ev[t], uv, acc[t][k]);
          }
        }
      }
    }
#pragma unroll
    for (int t = 0; t < kFwdRows; ++t) {
      const int64_t i = first + G * t;
      if (i < d) {   // warp-uniform
#pragma unroll
        for (int k = 0; k < K; ++k)
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) acc[t][k] += __shfl_xor_sync(0xffffffffu, acc[t][k], o);
        if (lane == 0) {
          const float yi = y[i];
#pragma unroll
          for (int k = 0; k < K; ++k)
            r[(int64_t)k * d + i] = yi > 0.f ? __fdiv_rn(yi, acc[t][k]) : 0.f;
        }
      }
    }
  }
}

struct BackArgs {
  const float* E;
  int64_t d, p;
  const float* r;          // K x d
  float* part;             // nseg x K x p
  unsigned* ctr;           // ncb arrival counters (0 between launches)
  int ncb, nseg;
  const double* sigma;     // p
  const int* nbr_ptr;      // p + 1
  const int* nbr_idx;
  const float* lam_in;     // K x p (old)
  float* lam_out;          // K x p (new)
  float* u;                // K x p: new lambda / sigma
  double mu[kMaxImages];
};

// Positive root of a x^2 + b x + c = 0 (a <= 0, c >= 0) as described above.
__device__ __forceinline__ double positive_root(double a, double b, double c) {
  const double disc = sqrt(fma(b, b, -4.0 * a * c));
  if (b <= 0.0) {
    const double den = disc - b;
    return den > 0.0 ? (2.0 * c) / den : 0.0;
  }
  return (-b - disc) / (2.0 * a);
}

template <int K, bool VEC>
__global__ void __launch_bounds__(kThreads)
k_pet_back(const BackArgs a) {
  __shared__ float red[kWarps][K][kColBlock];
  __shared__ __align__(16) float rs[K][kRowChunk];
  __shared__ int s_last;
  const int cb = blockIdx.x % a.ncb;
  const int seg = blockIdx.x / a.ncb;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t j0 = (int64_t)cb * kColBlock + 4 * lane;
  const int64_t i0 = (int64_t)seg * a.d / a.nseg;
  const int64_t i1 = (int64_t)(seg + 1) * a.d / a.nseg;

  float acc[K][4];
#pragma unroll
  for (int k = 0; k < K; ++k)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[k][c] = 0.f;

  auto load4 = [&](int64_t i) -> float4 {
    const float* e = a.E + i * a.p + j0;
    if (VEC) {
      return j0 < a.p ? __ldg(reinterpret_cast<const float4*>(e)) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    float4 v;
    v.x = j0 < a.p ? __ldg(e) : 0.f;
    v.y = j0 + 1 < a.p ? __ldg(e + 1) : 0.f;
    v.z = j0 + 2 < a.p ? __ldg(e + 2) : 0.f;
    v.w = j0 + 3 < a.p ? __ldg(e + 3) : 0.f;
    return v;
  };
  // Lines in chunks of kRowChunk: the chunk's ratios are staged in shared
  // memory (zero past the segment), warp w takes the line quads w, w + 8, ...
  // of the chunk, so one 16-byte shared load gives a quad's four ratios.
  for (int64_t c0 = i0; c0 < i1; c0 += kRowChunk) {
    const int rows = (int)min((int64_t)kRowChunk, i1 - c0);
    __syncthreads();
    for (int q = threadIdx.x; q < K * kRowChunk; q += kThreads) {
      const int k = q / kRowChunk, t = q % kRowChunk;
      rs[k][t] = t < rows ? __ldg(a.r + (int64_t)k * a.d + c0 + t) : 0.f;
    }
    __syncthreads();
    const int quads = (rows + 3) / 4;
    // QB quads of the warp loaded before any is used: 4 QB 16-byte loads in
    // flight per lane
    constexpr int QB = K <= 4 ? 4 : 2;
    for (int qd = warp; qd < quads; qd += kWarps * QB) {
      float4 ev[QB][4];
#pragma unroll
      for (int b = 0; b < QB; ++b)
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int row = 4 * (qd + b * kWarps) + t;
          ev[b][t] = row < rows ? load4(c0 + row) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
      for (int b = 0; b < QB; ++b) {
        const int t0 = 4 * (qd + b * kWarps);
        if (t0 >= rows) continue;
#pragma unroll
        for (int k = 0; k < K; ++k) {
          const float4 rv = *reinterpret_cast<const float4*>(&rs[k][t0]);
          const float rr[4] = {rv.x, rv.y, rv.z, rv.w};
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            acc[k][0] = fmaf(ev[b][t].x, rr[t], acc[k][0]);
            acc[k][1] = fmaf(ev[b][t].y, rr[t], acc[k][1]);
            acc[k][2] = fmaf(ev[b][t].z, rr[t], acc[k][2]);
            acc[k][3] = fmaf(ev[b][t].w, rr[t], acc[k][3]);
          }
        }
      }
    }
  }

#pragma unroll
  for (int k = 0; k < K; ++k)
#pragma unroll
    for (int c = 0; c < 4; ++c) red[warp][k][4 * lane + c] = acc[k][c];
  __syncthreads();
  // the warps' sums in warp order -> this segment's partial
  for (int q = threadIdx.x; q < K * kColBlock; q += kThreads) {
    const int k = q / kColBlock, c = q % kColBlock;
    const int64_t j = (int64_t)cb * kColBlock + c;
    float s = red[0][k][c];
#pragma unroll
    for (int w = 1; w < kWarps; ++w) s += red[w][k][c];
    if (j < a.p) a.part[((int64_t)seg * K + k) * a.p + j] = s;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&a.ctr[cb], 1u) == (unsigned)(a.nseg - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();

  // The last block of this column block: segments in order, then the root.
  for (int q = threadIdx.x; q < K * kColBlock; q += kThreads) {
    const int k = q / kColBlock;
    const int64_t j = (int64_t)cb * kColBlock + q % kColBlock;
    if (j >= a.p) continue;
    double t = 0.0;
    for (int s = 0; s < a.nseg; ++s) t += (double)__ldcg(a.part + ((int64_t)s * K + k) * a.p + j);
    const float* lam = a.lam_in + (int64_t)k * a.p;
    const double lj = (double)lam[j];
    const double sj = a.sigma[j];
    const double c = lj * t / sj;
    const int q0 = a.nbr_ptr[j], q1 = a.nbr_ptr[j + 1];
    double nsum = 0.0;
    for (int qq = q0; qq < q1; ++qq) nsum += (double)lam[a.nbr_idx[qq]];
    const double nj = (double)(q1 - q0);
    const double mu = a.mu[k];
    const double aa = -2.0 * mu * nj;
    const double bb = mu * (nj * lj + nsum) - 1.0;
    const double x = positive_root(aa, bb, c);
    a.lam_out[(int64_t)k * a.p + j] = (float)x;
    a.u[(int64_t)k * a.p + j] = (float)(x / sj);
  }
  if (threadIdx.x == 0) a.ctr[cb] = 0u;   // re-armed for the next launch
}

// ---------------------------------------------------------------------------
// the objective (float64)
// ---------------------------------------------------------------------------

// w_kj = lambda_kj / sigma_j in float64.
__global__ void k_pet_scaled(const float* __restrict__ lam, const double* __restrict__ sigma,
                             int64_t p, int nimg, double* __restrict__ w) {
  const int64_t n = (int64_t)nimg * p;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x)
    w[q] = (double)lam[q] / sigma[q % p];
}

// Per block: sum over its lines (warp w of block b takes lines
// b * kWarps + w + t * gridDim.x * kWarps) of y_i ln s_ki - s_ki, s_ki =
// sum_j e_ij w_kj in float64; lines with y_i = 0 give -s_ki.  Block partial
// out[b][k], warps added in order.
template <int K>
__global__ void __launch_bounds__(kThreads)
k_pet_loglik(const float* __restrict__ E, const float* __restrict__ y, int64_t d, int64_t p,
             const double* __restrict__ w, double* __restrict__ out) {
  __shared__ double part[kWarps][K];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double L[K];
#pragma unroll
  for (int k = 0; k < K; ++k) L[k] = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kWarps + warp; i < d; i += (int64_t)gridDim.x * kWarps) {
    double s[K];
#pragma unroll
    for (int k = 0; k < K; ++k) s[k] = 0.0;
    for (int64_t j = lane; j < p; j += 32) {
      const double e = (double)E[i * p + j];
#pragma unroll
      for (int k = 0; k < K; ++k) s[k] = fma(e, w[(int64_t)k * p + j], s[k]);
    }
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s[k] += __shfl_xor_sync(0xffffffffu, s[k], o);
    const double yi = (double)y[i];
#pragma unroll
    for (int k = 0; k < K; ++k) L[k] += (yi > 0.0 ? yi * log(s[k]) : 0.0) - s[k];
  }
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) part[warp][k] = L[k];
  __syncthreads();
  if (threadIdx.x < K) {
    double t = 0.0;
    for (int q = 0; q < kWarps; ++q) t += part[q][threadIdx.x];
    out[(int64_t)blockIdx.x * K + threadIdx.x] = t;
  }
}

// Per block: sum over its pixels j of (lambda_kj - lambda_kl)^2 for the
// neighbours l > j (each pair once).  Block partial out[b][k].
template <int K>
__global__ void __launch_bounds__(kThreads)
k_pet_penalty(const float* __restrict__ lam, int64_t p, const int* __restrict__ ptr,
              const int* __restrict__ idx, double* __restrict__ out) {
  __shared__ double part[kThreads][K];
  double P[K];
#pragma unroll
  for (int k = 0; k < K; ++k) P[k] = 0.0;
  for (int64_t j = (int64_t)blockIdx.x * kThreads + threadIdx.x; j < p;
       j += (int64_t)gridDim.x * kThreads) {
    for (int q = ptr[j]; q < ptr[j + 1]; ++q) {
      const int l = idx[q];
      if (l <= j) continue;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const double dl = (double)lam[(int64_t)k * p + j] - (double)lam[(int64_t)k * p + l];
        P[k] = fma(dl, dl, P[k]);
      }
    }
  }
#pragma unroll
  for (int k = 0; k < K; ++k) part[threadIdx.x][k] = P[k];
  __syncthreads();
  if (threadIdx.x < K) {
    double t = 0.0;
    for (int q = 0; q < kThreads; ++q) t += part[q][threadIdx.x];
    out[(int64_t)blockIdx.x * K + threadIdx.x] = t;
  }
}

// f_k = sum_b Lpart[b][k] - mu_k / 2 sum_b Ppart[b][k] (blocks in order).
__global__ void k_pet_obj_finish(const double* __restrict__ Lp, int nbL,
                                 const double* __restrict__ Pp, int nbP, int K,
                                 const double* __restrict__ mu, double* __restrict__ f) {
  const int k = threadIdx.x;
  if (k >= K) return;
  double L = 0.0, P = 0.0;
  for (int b = 0; b < nbL; ++b) L += Lp[(int64_t)b * K + k];
  for (int b = 0; b < nbP; ++b) P += Pp[(int64_t)b * K + k];
  f[k] = L - 0.5 * mu[k] * P;
}

// ---------------------------------------------------------------------------
// dispatch over the image count and the load width
// ---------------------------------------------------------------------------

template <int K>
cudaError_t launch_iter_k(bool vec, int fgrid, int cw, int bgrid, const float* E, int64_t d,
                          int64_t p,
                          const float* u, const float* y, float* r, const BackArgs& ba,
                          cudaStream_t st, cudaEvent_t* ev) {
  if (ev) cudaEventRecord(ev[0], st);
  const size_t sm = (size_t)K * cw * sizeof(float);
  if (vec) k_pet_forward<K, true><<<fgrid, kFwdThreads, sm, st>>>(E, d, p, u, y, r, cw);
  else k_pet_forward<K, false><<<fgrid, kFwdThreads, sm, st>>>(E, d, p, u, y, r, cw);
  if (ev) cudaEventRecord(ev[1], st);
  if (vec) k_pet_back<K, true><<<bgrid, kThreads, 0, st>>>(ba);
  else k_pet_back<K, false><<<bgrid, kThreads, 0, st>>>(ba);
  if (ev) cudaEventRecord(ev[2], st);
  return cudaGetLastError();
}

template <int K>
cudaError_t launch_obj_k(const float* E, const float* y, int64_t d, int64_t p, const double* w,
                         double* Lp, const float* lam, const int* ptr, const int* idx, double* Pp,
                         int pgrid, cudaStream_t st) {
  k_pet_loglik<K><<<kObjBlocks, kThreads, 0, st>>>(E, y, d, p, w, Lp);
  k_pet_penalty<K><<<pgrid, kThreads, 0, st>>>(lam, p, ptr, idx, Pp);
  return cudaGetLastError();
}

// Lets the forward projection for K images use kFwdSmem of dynamic shared
// memory and returns the back projection's resident blocks per SM.
template <int K>
void prepare_k(bool vec, int* b) {
  if (vec) {
    cudaFuncSetAttribute(k_pet_forward<K, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         kFwdSmem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(b, k_pet_back<K, true>, kThreads, 0);
  } else {
    cudaFuncSetAttribute(k_pet_forward<K, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         kFwdSmem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(b, k_pet_back<K, false>, kThreads, 0);
  }
}

void pet_prepare(int K, bool vec, int* b) {
  switch (K) {
    case 1: prepare_k<1>(vec, b); break;
    case 2: prepare_k<2>(vec, b); break;
    case 3: prepare_k<3>(vec, b); break;
    case 4: prepare_k<4>(vec, b); break;
    case 5: prepare_k<5>(vec, b); break;
    case 6: prepare_k<6>(vec, b); break;
    case 7: prepare_k<7>(vec, b); break;
    default: prepare_k<8>(vec, b); break;
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------

struct pet_ctx {
  int64_t d = 0, p = 0;
  int K = 1;
  const float* E = nullptr;
  const float* y = nullptr;
  float* lam_user = nullptr;
  cudaStream_t st = nullptr;
  bool vec = false;
  int fgrid = 0, cw = 0, ncb = 0, nseg = 0;
  double mu[kMaxImages] = {0};
  // device workspaces
  double* sigma = nullptr;
  float* lam_work = nullptr;
  float* u = nullptr;
  float* r = nullptr;
  float* part = nullptr;
  unsigned* ctr = nullptr;
  int* nbr_ptr = nullptr;
  int* nbr_idx = nullptr;
  double* mu_dev = nullptr;
  double* w64 = nullptr;
  double* Lp = nullptr;
  double* Pp = nullptr;
  int pgrid = 0;
  double* f_dev = nullptr;
  double* f_host = nullptr;   // pinned
  int* flag = nullptr;
  bool cur_is_work = false;   // the current intensities live in lam_work
  std::string err;
  // CUDA-event timing by kind (0 forward, 1 back, 2 objective)
  bool prof = false;
  double prof_ms[3] = {0, 0, 0};
  int64_t prof_n[3] = {0, 0, 0};
  std::vector<cudaEvent_t> ev_pool;
  struct Open { int iters; cudaEvent_t e[3]; };
  std::vector<Open> open_iters;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> open_obj;
};

namespace {

#define PET_CK(call, what)                                                          \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess) {                                                        \
      pet_set_err(c ? &c->err : nullptr, "%s: %s", what, cudaGetErrorString(e_));   \
      return NMF_ECUDA;                                                             \
    }                                                                               \
  } while (0)

void free_ctx(pet_ctx* c) {
  if (!c) return;
  void* bufs[] = {c->sigma, c->lam_work, c->u, c->r, c->part, c->ctr, c->nbr_ptr, c->nbr_idx,
                  c->mu_dev, c->w64, c->Lp, c->Pp, c->f_dev, c->flag};
  for (void* b : bufs)
    if (b) cudaFree(b);
  if (c->f_host) cudaFreeHost(c->f_host);
  for (auto e : c->ev_pool) cudaEventDestroy(e);
  for (auto& o : c->open_iters)
    for (auto e : o.e) cudaEventDestroy(e);
  for (auto& o : c->open_obj) {
    cudaEventDestroy(o.first);
    cudaEventDestroy(o.second);
  }
  (void)cudaGetLastError();
  delete c;
}

cudaEvent_t take_event(pet_ctx* c) {
  if (!c->ev_pool.empty()) {
    cudaEvent_t e = c->ev_pool.back();
    c->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

void prof_collect(pet_ctx* c) {
  for (auto& o : c->open_iters) {
    float a = 0.f, b = 0.f;
    if (cudaEventElapsedTime(&a, o.e[0], o.e[1]) == cudaSuccess &&
        cudaEventElapsedTime(&b, o.e[1], o.e[2]) == cudaSuccess) {
      c->prof_ms[0] += a;
      c->prof_ms[1] += b;
      c->prof_n[0] += 1;
      c->prof_n[1] += 1;
    }
    for (auto e : o.e) c->ev_pool.push_back(e);
  }
  c->open_iters.clear();
  for (auto& o : c->open_obj) {
    float a = 0.f;
    if (cudaEventElapsedTime(&a, o.first, o.second) == cudaSuccess) {
      c->prof_ms[2] += a;
      c->prof_n[2] += 1;
    }
    c->ev_pool.push_back(o.first);
    c->ev_pool.push_back(o.second);
  }
  c->open_obj.clear();
  (void)cudaGetLastError();
}

cudaError_t launch_iteration(pet_ctx* c) {
  BackArgs ba;
  ba.E = c->E;
  ba.d = c->d;
  ba.p = c->p;
  ba.r = c->r;
  ba.part = c->part;
  ba.ctr = c->ctr;
  ba.ncb = c->ncb;
  ba.nseg = c->nseg;
  ba.sigma = c->sigma;
  ba.nbr_ptr = c->nbr_ptr;
  ba.nbr_idx = c->nbr_idx;
  ba.lam_in = c->cur_is_work ? c->lam_work : c->lam_user;
  ba.lam_out = c->cur_is_work ? c->lam_user : c->lam_work;
  ba.u = c->u;
  for (int k = 0; k < kMaxImages; ++k) ba.mu[k] = c->mu[k];
  const int bgrid = c->ncb * c->nseg;
  cudaEvent_t* ev = nullptr;
  pet_ctx::Open o{};
  if (c->prof) {
    o.iters = 1;
    for (auto& e : o.e) e = take_event(c);
    if (o.e[0] && o.e[1] && o.e[2]) ev = o.e;
  }
  cudaError_t e;
  switch (c->K) {
#define PET_K(KK)                                                                         \
  case KK:                                                                                \
    e = launch_iter_k<KK>(c->vec, c->fgrid, c->cw, bgrid, c->E, c->d, c->p, c->u, c->y, c->r, ba, \
                          c->st, ev);                                                     \
    break;
    PET_K(1) PET_K(2) PET_K(3) PET_K(4) PET_K(5) PET_K(6) PET_K(7) PET_K(8)
#undef PET_K
    default: e = cudaErrorInvalidValue;
  }
  if (ev) c->open_iters.push_back(o);
  count_launches(2);
  c->cur_is_work = !c->cur_is_work;
  return e;
}

nmf_status finish_in_user_buffer(pet_ctx* c) {
  if (!c->cur_is_work) return NMF_OK;
  PET_CK(cudaMemcpyAsync(c->lam_user, c->lam_work, (size_t)c->K * c->p * sizeof(float),
                         cudaMemcpyDeviceToDevice, c->st), "copy lambda");
  c->cur_is_work = false;
  return NMF_OK;
}

nmf_status objective_async(pet_ctx* c) {
  cudaEvent_t a = nullptr, b = nullptr;
  if (c->prof) {
    a = take_event(c);
    b = take_event(c);
    if (a && b) cudaEventRecord(a, c->st);
  }
  const int64_t n = (int64_t)c->K * c->p;
  const unsigned g = (unsigned)std::min<int64_t>((n + kThreads - 1) / kThreads, 152 * 8);
  k_pet_scaled<<<g, kThreads, 0, c->st>>>(c->lam_user, c->sigma, c->p, c->K, c->w64);
  cudaError_t e;
  switch (c->K) {
#define PET_K(KK)                                                                          \
  case KK:                                                                                 \
    e = launch_obj_k<KK>(c->E, c->y, c->d, c->p, c->w64, c->Lp, c->lam_user, c->nbr_ptr,    \
                         c->nbr_idx, c->Pp, c->pgrid, c->st);                              \
    break;
    PET_K(1) PET_K(2) PET_K(3) PET_K(4) PET_K(5) PET_K(6) PET_K(7) PET_K(8)
#undef PET_K
    default: e = cudaErrorInvalidValue;
  }
  if (e == cudaSuccess) {
    k_pet_obj_finish<<<1, 32, 0, c->st>>>(c->Lp, kObjBlocks, c->Pp, c->pgrid, c->K, c->mu_dev,
                                          c->f_dev);
    e = cudaGetLastError();
  }
  if (a && b) {
    cudaEventRecord(b, c->st);
    c->open_obj.push_back({a, b});
  }
  count_launches(5);
  if (e != cudaSuccess) {
    pet_set_err(&c->err, "objective launch: %s", cudaGetErrorString(e));
    return NMF_ECUDA;
  }
  return NMF_OK;
}

}  // namespace

extern "C" {

nmf_status pet_init(int64_t d, int64_t p, const float* E, const float* y, const int32_t* nbr_ptr,
                    const int32_t* nbr_idx, int32_t nimg, const double* mu, float* lambda,
                    int32_t init_ones, void* stream, pet_ctx** out) {
  pet_ctx* c = nullptr;
  if (out) *out = nullptr;
  if (!out || !E || !y || !nbr_ptr || !mu || !lambda) {
    pet_set_err(nullptr, "pet_init: null argument");
    return NMF_EINVAL;
  }
  if (d < 1 || p < 1 || p > (int64_t)INT32_MAX) {
    pet_set_err(nullptr, "pet_init: need d >= 1 and 1 <= p < 2^31");
    return NMF_EINVAL;
  }
  if (nimg < 1 || nimg > kMaxImages) {
    pet_set_err(nullptr, "pet_init: nimg must be 1..%d", kMaxImages);
    return NMF_EINVAL;
  }
  for (int k = 0; k < nimg; ++k)
    if (!(mu[k] >= 0.0) || std::isinf(mu[k])) {
      pet_set_err(nullptr, "pet_init: mu[%d] must be finite and >= 0", k);
      return NMF_EINVAL;
    }
  // the neighbourhood system: CSR shape, range, no self pairs, symmetry
  if (nbr_ptr[0] != 0) {
    pet_set_err(nullptr, "pet_init: nbr_ptr[0] must be 0");
    return NMF_EINVAL;
  }
  for (int64_t j = 0; j < p; ++j)
    if (nbr_ptr[j + 1] < nbr_ptr[j]) {
      pet_set_err(nullptr, "pet_init: nbr_ptr must be nondecreasing");
      return NMF_EINVAL;
    }
  const int64_t nnz = nbr_ptr[p];
  if (nnz > 0 && !nbr_idx) {
    pet_set_err(nullptr, "pet_init: nbr_idx is NULL");
    return NMF_EINVAL;
  }
  for (int64_t j = 0; j < p; ++j)
    for (int q = nbr_ptr[j]; q < nbr_ptr[j + 1]; ++q) {
      const int k = nbr_idx[q];
      if (k < 0 || k >= p || k == j) {
        pet_set_err(nullptr, "pet_init: neighbour %d of pixel %lld out of range or itself", k,
                    (long long)j);
        return NMF_EINVAL;
      }
      bool back = false;
      for (int qq = nbr_ptr[k]; qq < nbr_ptr[k + 1] && !back; ++qq) back = nbr_idx[qq] == j;
      if (!back) {
        pet_set_err(nullptr, "pet_init: the neighbourhood system is not symmetric (%lld -> %d)",
                    (long long)j, k);
        return NMF_EINVAL;
      }
    }

  c = new (std::nothrow) pet_ctx;
  if (!c) {
    pet_set_err(nullptr, "pet_init: host allocation failed");
    return NMF_ENOMEM;
  }
  c->d = d;
  c->p = p;
  c->K = nimg;
  c->E = E;
  c->y = y;
  c->lam_user = lambda;
  c->st = static_cast<cudaStream_t>(stream);
  for (int k = 0; k < nimg; ++k) c->mu[k] = mu[k];
  c->vec = (p % 4 == 0) && (reinterpret_cast<uintptr_t>(E) % 16 == 0);
  // The forward projection is a persistent grid of one block per SM with u
  // staged in chunks of cw columns (a multiple of 128, all images within
  // kFwdSmem); the back projection has as many line segments per column
  // block as fit in one wave of its resident blocks, so that it ends in no
  // partial wave.
  int dev = 0, sms = 152, occ_b = 4;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  pet_prepare(nimg, c->vec, &occ_b);
  (void)cudaGetLastError();
  c->cw = (int)std::min<int64_t>(round_up(p, 128), (kFwdSmem / 4 / nimg) / 128 * 128);
  c->fgrid = (int)std::max<int64_t>(
      1, std::min<int64_t>(sms, (d + kFwdThreads / 32 - 1) / (kFwdThreads / 32)));
  c->ncb = (int)((p + kColBlock - 1) / kColBlock);
  const int64_t wave = (int64_t)sms * std::max(occ_b, 1);
  c->nseg = (int)std::max<int64_t>(1, std::min<int64_t>(d, wave / c->ncb));
  c->pgrid = (int)std::min<int64_t>((p + kThreads - 1) / kThreads, kObjBlocks);

  auto dalloc = [&](void** ptr, size_t bytes) -> bool {
    if (cudaMalloc(ptr, bytes) != cudaSuccess) {
      (void)cudaGetLastError();
      pet_set_err(nullptr, "pet_init: cudaMalloc of %zu bytes failed", bytes);
      return false;
    }
    return true;
  };
  const size_t Kp = (size_t)nimg * p;
  if (!dalloc((void**)&c->sigma, p * sizeof(double)) ||
      !dalloc((void**)&c->lam_work, Kp * sizeof(float)) ||
      !dalloc((void**)&c->u, Kp * sizeof(float)) ||
      !dalloc((void**)&c->r, (size_t)nimg * d * sizeof(float)) ||
      !dalloc((void**)&c->part, (size_t)c->nseg * Kp * sizeof(float)) ||
      !dalloc((void**)&c->ctr, c->ncb * sizeof(unsigned)) ||
      !dalloc((void**)&c->nbr_ptr, (p + 1) * sizeof(int)) ||
      !dalloc((void**)&c->nbr_idx, std::max<int64_t>(nnz, 1) * sizeof(int)) ||
      !dalloc((void**)&c->mu_dev, kMaxImages * sizeof(double)) ||
      !dalloc((void**)&c->w64, Kp * sizeof(double)) ||
      !dalloc((void**)&c->Lp, (size_t)kObjBlocks * nimg * sizeof(double)) ||
      !dalloc((void**)&c->Pp, (size_t)kObjBlocks * nimg * sizeof(double)) ||
      !dalloc((void**)&c->f_dev, kMaxImages * sizeof(double)) ||
      !dalloc((void**)&c->flag, sizeof(int))) {
    free_ctx(c);
    return NMF_ENOMEM;
  }
  if (cudaMallocHost((void**)&c->f_host, kMaxImages * sizeof(double) + sizeof(int)) !=
      cudaSuccess) {
    (void)cudaGetLastError();
    free_ctx(c);
    pet_set_err(nullptr, "pet_init: pinned allocation failed");
    return NMF_ENOMEM;
  }
  auto fail = [&](const char* what, cudaError_t e) {
    pet_set_err(nullptr, "pet_init: %s: %s", what, cudaGetErrorString(e));
    free_ctx(c);
    return NMF_ECUDA;
  };
  cudaError_t e;
  if ((e = cudaMemcpyAsync(c->nbr_ptr, nbr_ptr, (p + 1) * sizeof(int), cudaMemcpyHostToDevice,
                           c->st)) != cudaSuccess)
    return fail("copy nbr_ptr", e);
  if (nnz > 0 && (e = cudaMemcpyAsync(c->nbr_idx, nbr_idx, nnz * sizeof(int),
                                      cudaMemcpyHostToDevice, c->st)) != cudaSuccess)
    return fail("copy nbr_idx", e);
  double mu_pad[kMaxImages] = {0};
  for (int k = 0; k < nimg; ++k) mu_pad[k] = mu[k];
  if ((e = cudaMemcpyAsync(c->mu_dev, mu_pad, sizeof mu_pad, cudaMemcpyHostToDevice, c->st)) !=
      cudaSuccess)
    return fail("copy mu", e);
  if ((e = cudaMemsetAsync(c->ctr, 0, c->ncb * sizeof(unsigned), c->st)) != cudaSuccess ||
      (e = cudaMemsetAsync(c->flag, 0, sizeof(int), c->st)) != cudaSuccess)
    return fail("memset", e);
  const unsigned cg = (unsigned)std::min<int64_t>((p + kThreads - 1) / kThreads, 152 * 8);
  k_pet_colsum<<<cg, kThreads, 0, c->st>>>(E, d, p, c->sigma, c->flag);
  const unsigned yg = (unsigned)std::min<int64_t>((d + kThreads - 1) / kThreads, 152 * 8);
  k_pet_check<<<yg, kThreads, 0, c->st>>>(y, d, 2, c->flag);
  int launches = 2;
  if (!init_ones) {
    const unsigned lg = (unsigned)std::min<int64_t>((Kp + kThreads - 1) / kThreads, 152 * 8);
    k_pet_check<<<lg, kThreads, 0, c->st>>>(lambda, (int64_t)Kp, 4, c->flag);
    ++launches;
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return fail("check launch", e);
  int* hflag = reinterpret_cast<int*>(c->f_host + kMaxImages);
  if ((e = cudaMemcpyAsync(hflag, c->flag, sizeof(int), cudaMemcpyDeviceToHost, c->st)) !=
          cudaSuccess ||
      (e = cudaStreamSynchronize(c->st)) != cudaSuccess)
    return fail("checks", e);
  count_launches(launches);
  if (*hflag) {
    const int f = *hflag;
    pet_set_err(nullptr, "pet_init: %s%s%s%s", (f & 1) ? "E has a negative or non-finite entry; " : "",
                (f & 8) ? "a column of E sums to zero (a pixel no line sees); " : "",
                (f & 2) ? "y has a negative or non-finite entry; " : "",
                (f & 4) ? "the starting lambda has a negative or non-finite entry" : "");
    free_ctx(c);
    return (f & 7) ? NMF_ENONFINITE : NMF_EINVAL;
  }
  const unsigned sg = (unsigned)std::min<int64_t>((Kp + kThreads - 1) / kThreads, 152 * 8);
  k_pet_start<<<sg, kThreads, 0, c->st>>>(lambda, c->u, c->sigma, p, nimg, init_ones ? 1 : 0);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail("start", e);
  count_launches(1);
  *out = c;
  return NMF_OK;
}

nmf_status pet_step(pet_ctx* c, int iters) {
  if (!c || iters < 0) {
    pet_set_err(c ? &c->err : nullptr, "pet_step: null context or iters < 0");
    return NMF_EINVAL;
  }
  for (int it = 0; it < iters; ++it) PET_CK(launch_iteration(c), "iteration launch");
  return finish_in_user_buffer(c);
}

nmf_status pet_restart(pet_ctx* c) {
  if (!c) {
    pet_set_err(nullptr, "pet_restart: ctx is NULL");
    return NMF_EINVAL;
  }
  const int64_t Kp = (int64_t)c->K * c->p;
  const unsigned sg = (unsigned)std::min<int64_t>((Kp + kThreads - 1) / kThreads, 152 * 8);
  k_pet_start<<<sg, kThreads, 0, c->st>>>(c->lam_user, c->u, c->sigma, c->p, c->K, 1);
  PET_CK(cudaGetLastError(), "restart");
  count_launches(1);
  c->cur_is_work = false;
  return NMF_OK;
}

nmf_status pet_objective(pet_ctx* c, double* f_out) {
  if (!c || !f_out) {
    pet_set_err(c ? &c->err : nullptr, "pet_objective: null argument");
    return NMF_EINVAL;
  }
  nmf_status s = objective_async(c);
  if (s != NMF_OK) return s;
  PET_CK(cudaMemcpyAsync(c->f_host, c->f_dev, c->K * sizeof(double), cudaMemcpyDeviceToHost,
                         c->st), "copy f");
  PET_CK(cudaStreamSynchronize(c->st), "sync");
  for (int k = 0; k < c->K; ++k) f_out[k] = c->f_host[k];
  return NMF_OK;
}

nmf_status pet_run(pet_ctx* c, int max_iters, double tol, int check_every, int* iters_done,
                   double* f_out) {
  if (!c || max_iters < 0 || check_every < 1 || !(tol >= 0.0)) {
    pet_set_err(c ? &c->err : nullptr, "pet_run: bad argument");
    return NMF_EINVAL;
  }
  double prev[kMaxImages], cur[kMaxImages];
  nmf_status s = pet_objective(c, prev);
  if (s != NMF_OK) return s;
  int done = 0;
  while (done < max_iters) {
    const int k = std::min(check_every, max_iters - done);
    if ((s = pet_step(c, k)) != NMF_OK) return s;
    done += k;
    if ((s = pet_objective(c, cur)) != NMF_OK) return s;
    bool all = true;
    for (int q = 0; q < c->K; ++q)
      all &= std::fabs(cur[q] - prev[q]) / (std::fabs(prev[q]) + 1.0) < tol;
    for (int q = 0; q < c->K; ++q) prev[q] = cur[q];
    if (all) break;
  }
  if (iters_done) *iters_done = done;
  if (f_out)
    for (int q = 0; q < c->K; ++q) f_out[q] = prev[q];
  return NMF_OK;
}

nmf_status pet_profile_enable(pet_ctx* c, int on) {
  if (!c) {
    pet_set_err(nullptr, "pet_profile_enable: ctx is NULL");
    return NMF_EINVAL;
  }
  if (on) {
    PET_CK(cudaStreamSynchronize(c->st), "sync");
    prof_collect(c);
    for (int k = 0; k < 3; ++k) {
      c->prof_ms[k] = 0;
      c->prof_n[k] = 0;
    }
  }
  c->prof = on != 0;
  return NMF_OK;
}

nmf_status pet_profile_read(pet_ctx* c, int kind, double* ms, int64_t* count) {
  if (!c || kind < 0 || kind > 2) {
    pet_set_err(c ? &c->err : nullptr, "pet_profile_read: bad kind");
    return NMF_EINVAL;
  }
  PET_CK(cudaStreamSynchronize(c->st), "sync");
  prof_collect(c);
  if (ms) *ms = c->prof_ms[kind];
  if (count) *count = c->prof_n[kind];
  return NMF_OK;
}

void pet_destroy(pet_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->st);
  free_ctx(c);
}

const char* pet_last_error(const pet_ctx* c) {
  return c ? c->err.c_str() : g_pet_error.c_str();
}

}  // extern "C"
