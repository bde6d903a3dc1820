// Algorithm 1 with Section 3's stopping rule for a small Gaussian problem,
// every iteration in ONE persistent launch (the multiplicative updates
// Eqs. (3.3)-(3.4), the objective Eq. (3.1)).  For a V that is launch-bound
// rather than HBM-bound (the CBCL faces matrix of Table 2 is 361 x 2429):
// each block keeps, for the whole run, a column slice of V (for the H
// update) and the transpose of a row slice of V (for the W update) in
// shared memory; the factors live in global memory (and in L2).
//
// One half step of block b (the H update; the W update is the same with the
// roles of the factors and slices exchanged):
//   1. the whole other factor Y = W (p x r) into shared memory as Ys[K][RP]
//      (asynchronous 16-byte copies of a padded [K][RP] copy of each factor
//      that the kernel keeps beside W and H), the block's own old columns O
//      of H;
//   2. the Gram W^T W as the sum, in block order, of the partial Grams that
//      every block left for its own rows of W (upper triangle, float32);
//   3. the numerators (W^T V)[k][j] for the block's columns j as one small
//      contraction Ys^T X over K = p in float32 (each thread a 4 x 4 tile of
//      one K segment; the segments summed by a fixed xor tree within a warp,
//      then warp by warp in order);
//   4. den = O G + eps and new = O * num / den (IEEE division), written to H
//      and to the padded copy, and the partial Gram of the block's new
//      columns for the next half step;
//   5. when the half step ends a round, the block's part of
//      ||V - W H||_F^2 over its slice (compensated float32 dot products,
//      float64 sums) into its partial slot;
//   6. a grid-wide barrier (a counter with bounded waits).
// After each round every block sums the objective partials in block order,
// so all blocks take the same stopping decision.
#include <algorithm>

#include "nmf_internal.cuh"

namespace nmf {
namespace {

constexpr int kRT = 512;                 // threads per block
constexpr int kRW = kRT / 32;            // warps per block
constexpr int kMaxTasks = 32;            // 4 x 4 numerator tiles of a half step
constexpr long long kBarCycles = 2000000000LL;   // a grid barrier waits at most ~1 s

struct ResArgs {
  const float* V;
  float* W;
  float* H;
  float* Wp;              // p x RP, rows 16-byte aligned, columns >= r zero
  float* Hp;              // n x RP (H transposed), the same layout
  float* gpW;             // [grid][E] partial Grams of W over each block's rows
  float* gpH;             // [grid][E] partial Grams of H over each block's columns
  int p, n, r, E;         // E = r (r + 1) / 2 entries of an upper triangle
  float eps;
  int h_first;
  int max_iters, check_every;
  double tol;
  const double* f0;       // objective at the start
  double* fpart;          // [grid] objective partials of a round
  unsigned long long* bar;   // barrier counter, zero at launch
  int* err;
  RunState* out;
  int ldc, ldr;           // strides of the column slice [p][ldc] and row slice [n][ldr]
  int mnm;                // largest own slice (rows or columns) of any block
};

template <int RP>
struct ResSmem {
  // float offsets into the dynamic shared memory
  int xc, xr, ys, o, on, num, gr, sg, red, total, ldn;
  __host__ __device__ ResSmem(int p, int n, int ldc, int ldr, int mnm) {
    const int mnm4 = (mnm + 3) & ~3;
    ldn = mnm4;
    xc = 0;
    xr = xc + p * ldc;
    ys = xr + n * ldr;
    o = ys + (p > n ? p : n) * RP;
    on = o + mnm4 * RP;
    num = on + mnm4 * RP;        // NUM[k][m], RP x mnm4
    gr = num + RP * mnm4;        // the Gram, RP x RP (zero beyond r)
    sg = gr + RP * RP;           // chunk sums of the partial Grams (<= kRT)
    red = sg + kRT;
    total = red + kRW * kMaxTasks * 16;
  }
};

__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& e) {
  // Knuth's TwoSum: s + e == a + b exactly
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Grid-wide barrier number `idx` (0, 1, 2, ...): every block adds one to the
// counter and waits, at most kBarCycles, until all gridDim.x blocks of this
// barrier have arrived.  Returns false (and sets the error word) on expiry.
__device__ bool grid_barrier(unsigned long long* bar, unsigned long long idx, int* err,
                             int* s_ok) {
  __syncthreads();
  if (threadIdx.x == 0) {
    // release: this block's writes (ordered before by the block barrier)
    // are visible to whoever acquires the counter
    asm volatile("red.release.gpu.global.add.u64 [%0], 1;" ::"l"(bar) : "memory");
    const unsigned long long target = (idx + 1) * (unsigned long long)gridDim.x;
    const long long t0 = clock64();
    int ok = 1;
    while (ld_acquire_u64(bar) < target) {
      if (clock64() - t0 > kBarCycles) {
        ok = 0;
        atomicExch(err, 3);
        break;
      }
    }
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

// NUM[k][m] = sum over K of Ys[K][k] * X[K][m] (k < RP, m < 4 gx): the
// tasks are the 4 x 4 tiles (k block a4, m block g); thread t takes task
// t % ntp and the K segment t / ntp; the segments are summed by an xor tree
// over the lanes of a warp that share a task, then warp by warp in order.
template <int RP>
__device__ void contract_num(const float* X, int ldx, int gx, const float* Ys, int K,
                             float* Red, float* NUM, int ldn) {
  const int ntask = (RP / 4) * gx;
  int ntp = 1;
  while (ntp < ntask) ntp <<= 1;
  const int t = threadIdx.x, task = t % ntp, s = t / ntp, nseg = kRT / ntp;
  const int k0 = (int)((int64_t)s * K / nseg), k1 = (int)((int64_t)(s + 1) * K / nseg);
  float acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[u][c] = 0.f;
  if (task < ntask) {
    const int a4 = task / gx, g = task - a4 * gx;
    const float* yb = Ys + 4 * a4;
    const float* xb = X + 4 * g;
    for (int q = k0; q < k1; ++q) {
      const float4 y = *reinterpret_cast<const float4*>(yb + q * RP);
      const float4 z = *reinterpret_cast<const float4*>(xb + q * ldx);
      const float yv[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        acc[u][0] = fmaf(yv[u], z.x, acc[u][0]);
        acc[u][1] = fmaf(yv[u], z.y, acc[u][1]);
        acc[u][2] = fmaf(yv[u], z.z, acc[u][2]);
        acc[u][3] = fmaf(yv[u], z.w, acc[u][3]);
      }
    }
  }
  for (int d = ntp; d < 32; d <<= 1)
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[u][c] += __shfl_xor_sync(0xffffffffu, acc[u][c], d);
  const int lane = t & 31, warp = t >> 5;
  if (lane < ntp && task < ntask) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
      *reinterpret_cast<float4*>(&Red[((warp * kMaxTasks + task) * 4 + u) * 4]) =
          make_float4(acc[u][0], acc[u][1], acc[u][2], acc[u][3]);
  }
  __syncthreads();
  for (int o = t; o < ntask * 16; o += kRT) {
    const int tk = o >> 4, e = o & 15;
    float sum = Red[tk * 16 + e];
    for (int w = 1; w < kRW; ++w) sum += Red[(w * kMaxTasks + tk) * 16 + e];
    const int a4 = tk / gx, g = tk - a4 * gx;
    NUM[(4 * a4 + (e >> 2)) * ldn + 4 * g + (e & 3)] = sum;
  }
  __syncthreads();
}

// Upper-triangle entry e of an r x r matrix (row-major over k <= l).
__device__ __forceinline__ void tri_index(int e, int r, int& k, int& l) {
  k = 0;
  while (e >= r - k) { e -= r - k; ++k; }
  l = k + e;
}

// The Gram of the other factor from the grid's partials gp[G][E], in block
// order: thread t < E * nch sums the blocks of chunk t / E (chunks of
// consecutive blocks, in order) into Sg; gram_finish adds the chunks in
// order and fills GR (both triangles).
__device__ __forceinline__ int gram_chunks(int E) {
  const int c = kRT / E;
  return c < 1 ? 1 : c;
}
__device__ void gram_partial_sums(const float* gp, int E, float* Sg) {
  const int G = gridDim.x, nch = gram_chunks(E), t = threadIdx.x;
  if (t < E * nch) {
    const int e = t % E, c = t / E;
    const int b0 = (int)((int64_t)c * G / nch), b1 = (int)((int64_t)(c + 1) * G / nch);
    float sum = 0.f;
    for (int b = b0; b < b1; ++b) sum += __ldcg(gp + (int64_t)b * E + e);
    Sg[c * E + e] = sum;
  }
}
template <int RP>
__device__ void gram_finish(const float* Sg, int E, int r, float* GR) {
  const int nch = gram_chunks(E), t = threadIdx.x;
  if (t < E) {
    float sum = Sg[t];
    for (int c = 1; c < nch; ++c) sum += Sg[c * E + t];
    int k, l;
    tri_index(t, r, k, l);
    GR[k * RP + l] = sum;
    GR[l * RP + k] = sum;
  }
}

// The partial Gram of a slice of factor values val(m, k) (m < nm, k < r),
// upper triangle, into gp[blockIdx.x][E]: float32 sums over m in order.
template <typename Fn>
__device__ void gram_partial(Fn val, int nm, int r, int E, float* gp) {
  for (int e = threadIdx.x; e < E; e += kRT) {
    int k, l;
    tri_index(e, r, k, l);
    float sum = 0.f;
    for (int m = 0; m < nm; ++m) sum = fmaf(val(m, k), val(m, l), sum);
    gp[(int64_t)blockIdx.x * E + e] = sum;
  }
}

__device__ __forceinline__ void cp_async16(float* dst, const float* src) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// Step 1 of a half step: the other factor's padded copy ([K][RP], 16-byte
// rows) into Ys by asynchronous 16-byte copies (all in flight at once, no
// registers), the block's own old values into O.  The caller waits for the
// copies (cp_async_wait_all) and synchronises.
template <int RP, bool HU>
__device__ void load_operands(const ResArgs& a, float* Ys, float* O, float* On, int g0,
                              int nm) {
  const int t = threadIdx.x;
  const int r = a.r;
  const float* src = HU ? a.Wp : a.Hp;
  const int nv = (HU ? a.p : a.n) * (RP / 4);
  for (int e = t; e < nv; e += kRT) cp_async16(Ys + 4 * e, src + 4 * e);
  for (int e = t; e < nm * RP; e += kRT) {
    const int m = e / RP, k = e - m * RP;
    float v = 0.f;
    if (k < r) v = HU ? __ldcg(a.H + (int64_t)k * a.n + g0 + m) : __ldcg(a.W + (int64_t)(g0 + m) * r + k);
    O[e] = v;
    On[e] = 0.f;
  }
}

// One half step of this block.  HU = true: the H update over the block's
// columns [j0, j0 + nm) (K = p, Y = W); false: the W update over its rows
// [i0, i0 + nm) (K = n, Y = H).  `check`: also the objective partial.
template <int RP, bool HU>
__device__ void half_step(const ResArgs& a, float* sm, const ResSmem<RP>& L, int g0, int nm,
                          bool check) {
  const int t = threadIdx.x;
  const int r = a.r;
  const int K = HU ? a.p : a.n;
  const float* X = sm + (HU ? L.xc : L.xr);
  const int ldx = HU ? a.ldc : a.ldr;
  float* Ys = sm + L.ys;
  float* O = sm + L.o;
  float* On = sm + L.on;
  float* NUM = sm + L.num;
  float* GR = sm + L.gr;
  float* Sg = sm + L.sg;
  load_operands<RP, HU>(a, Ys, O, On, g0, nm);   // copies still in flight
  gram_partial_sums(HU ? a.gpW : a.gpH, a.E, Sg);
  cp_async_wait_all();
  __syncthreads();
  gram_finish<RP>(Sg, a.E, r, GR);
  // numerators (their own barriers also order GR)
  const int gx = (nm + 3) / 4;
  contract_num<RP>(X, ldx, gx, Ys, K, sm + L.red, NUM, L.ldn);
  // den = O G + eps, new = O * num / den
  for (int e = t; e < nm * r; e += kRT) {
    const int m = e / r, k = e - m * r;
    float den = 0.f;
    for (int l = 0; l < r; ++l) den = fmaf(O[m * RP + l], GR[l * RP + k], den);
    const float num = NUM[k * L.ldn + m];
    const float v = div_rn(__fmul_rn(O[m * RP + k], num), __fadd_rn(den, a.eps));
    On[m * RP + k] = v;
    if (HU) {
      a.H[(int64_t)k * a.n + g0 + m] = v;
      a.Hp[(int64_t)(g0 + m) * RP + k] = v;
    } else {
      a.W[(int64_t)(g0 + m) * r + k] = v;
      a.Wp[(int64_t)(g0 + m) * RP + k] = v;
    }
  }
  __syncthreads();
  // the partial Gram of this block's new values, for the other half step
  gram_partial([&](int m, int k) { return On[m * RP + k]; }, nm, r, a.E, HU ? a.gpH : a.gpW);
  if (!check) return;
  // 4. this slice's part of ||V - W H||^2: entries (K index q, own index m)
  double acc = 0.0;
  const int tot = K * nm;
  if (nm > 0) {
    const int dq = kRT / nm, dm = kRT - dq * nm;
    int q = t / nm, m = t - q * nm;
    for (int e = t; e < tot; e += kRT) {
      const float* y = Ys + q * RP;
      const float* o = On + m * RP;
      float s0 = 0.f, s1 = 0.f;
#pragma unroll
      for (int k = 0; k < RP; k += 2) {
        s0 = fmaf(y[k], o[k], s0);
        s1 = fmaf(y[k + 1], o[k + 1], s1);
      }
      float hi, lo;
      two_sum_f(s0, s1, hi, lo);
      const float d = __fsub_rn(__fsub_rn(X[q * ldx + m], hi), lo);
      acc += (double)__fmul_rn(d, d);
      q += dq;
      m += dm;
      if (m >= nm) { m -= nm; ++q; }
    }
  }
  for (int d = 16; d >= 1; d >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, d);
  double* dred = reinterpret_cast<double*>(sm + L.red);   // the contraction is done with Red
  if ((t & 31) == 0) dred[t >> 5] = acc;
  __syncthreads();
  if (t == 0) {
    double s = dred[0];
    for (int w = 1; w < kRW; ++w) s += dred[w];
    a.fpart[blockIdx.x] = s;
  }
}

template <int RP>
__global__ void __launch_bounds__(kRT, 1) k_resident(const ResArgs a) {
  extern __shared__ __align__(16) float sm[];
  __shared__ int s_ok;
  __shared__ double s_f;
  const ResSmem<RP> L(a.p, a.n, a.ldc, a.ldr, a.mnm);
  const int t = threadIdx.x, b = blockIdx.x, G = gridDim.x;
  const int j0 = (int)((int64_t)b * a.n / G), j1 = (int)((int64_t)(b + 1) * a.n / G);
  const int i0 = (int)((int64_t)b * a.p / G), i1 = (int)((int64_t)(b + 1) * a.p / G);
  const int nc = j1 - j0, nr = i1 - i0;
  // V's slices, once: Xc[i][jj] = V[i][j0 + jj], Xr[j][ii] = V[i0 + ii][j]
  float* Xc = sm + L.xc;
  float* Xr = sm + L.xr;
  for (int e = t; e < a.p * a.ldc; e += kRT) {
    const int i = e / a.ldc, jj = e - i * a.ldc;
    Xc[e] = jj < nc ? __ldg(a.V + (int64_t)i * a.n + j0 + jj) : 0.f;
  }
  for (int ii = 0; ii < a.ldr; ++ii)
    for (int j = t; j < a.n; j += kRT)
      Xr[j * a.ldr + ii] = ii < nr ? __ldg(a.V + (int64_t)(i0 + ii) * a.n + j) : 0.f;
  for (int e = t; e < (a.p > a.n ? a.p : a.n) * RP; e += kRT) sm[L.ys + e] = 0.f;
  for (int e = t; e < RP * RP; e += kRT) sm[L.gr + e] = 0.f;
  // partial Grams of this block's rows of the starting W and columns of H
  gram_partial([&](int m, int k) { return a.W[(int64_t)(i0 + m) * a.r + k]; }, nr, a.r, a.E,
               a.gpW);
  gram_partial([&](int m, int k) { return a.H[(int64_t)k * a.n + j0 + m]; }, nc, a.r, a.E,
               a.gpH);
  // the padded copies of this block's slices of the starting factors
  for (int e = t; e < nr * RP; e += kRT) {
    const int m = e / RP, k = e - m * RP;
    a.Wp[(int64_t)(i0 + m) * RP + k] = k < a.r ? a.W[(int64_t)(i0 + m) * a.r + k] : 0.f;
  }
  for (int e = t; e < nc * RP; e += kRT) {
    const int m = e / RP, k = e - m * RP;
    a.Hp[(int64_t)(j0 + m) * RP + k] = k < a.r ? a.H[(int64_t)k * a.n + j0 + m] : 0.f;
  }
  unsigned long long nbar = 0;
  bool ok = grid_barrier(a.bar, nbar++, a.err, &s_ok);

  double f_prev = *a.f0, f = f_prev;
  int done = 0, checks = 0, stop = 0;
  while (ok) {
    int it;
    bool full;
    if (a.max_iters - done >= a.check_every) { it = a.check_every; full = true; }
    else if (done < a.max_iters) { it = a.max_iters - done; full = false; }
    else break;
    for (int s = 0; s < it && ok; ++s) {
      const bool chk = s == it - 1;
      if (a.h_first) {
        half_step<RP, true>(a, sm, L, j0, nc, false);
        ok = grid_barrier(a.bar, nbar++, a.err, &s_ok);
        if (!ok) break;
        half_step<RP, false>(a, sm, L, i0, nr, chk);
      } else {
        half_step<RP, false>(a, sm, L, i0, nr, false);
        ok = grid_barrier(a.bar, nbar++, a.err, &s_ok);
        if (!ok) break;
        half_step<RP, true>(a, sm, L, j0, nc, chk);
      }
      ok = grid_barrier(a.bar, nbar++, a.err, &s_ok);
    }
    if (!ok) break;
    done += it;
    if (t == 0) {
      double sum = __ldcg(a.fpart);
      for (int q = 1; q < G; ++q) sum += __ldcg(a.fpart + q);
      s_f = sum;
    }
    __syncthreads();
    f = s_f;
    if (!full) break;
    ++checks;
    const bool conv = a.tol > 0.0 && fabs(f - f_prev) / (fabs(f_prev) + 1.0) < a.tol;
    if (conv) { stop = 1; break; }
    f_prev = f;
  }
  if (b == 0 && t == 0) {
    a.out->f_prev = f_prev;
    a.out->f = f;
    a.out->tol = a.tol;
    a.out->done = done;
    a.out->checks = checks;
    a.out->stop = stop;
    a.out->max_iters = a.max_iters;
  }
}

int rpad4(int r) { return (r + 3) & ~3; }

template <int RP>
size_t smem_bytes(int p, int n, int G) {
  const int mc = (n + G - 1) / G, mr = (p + G - 1) / G;
  const int ldc = (mc + 3) & ~3, ldr = (mr + 3) & ~3;
  const ResSmem<RP> L(p, n, ldc, ldr, mc > mr ? mc : mr);
  return (size_t)L.total * sizeof(float);
}

size_t smem_for(int p, int n, int r, int G) {
  switch (rpad4(r)) {
    case 4: return smem_bytes<4>(p, n, G);
    case 8: return smem_bytes<8>(p, n, G);
    case 12: return smem_bytes<12>(p, n, G);
    default: return smem_bytes<16>(p, n, G);
  }
}

const void* kernel_for(int r) {
  switch (rpad4(r)) {
    case 4: return (const void*)k_resident<4>;
    case 8: return (const void*)k_resident<8>;
    case 12: return (const void*)k_resident<12>;
    default: return (const void*)k_resident<16>;
  }
}

}  // namespace

bool resident_supported(int64_t p, int64_t n, int r, int sms, size_t smem_optin) {
  if (r < 1 || r > kResidentMaxRank || p < 1 || n < 1 || sms < 1) return false;
  if (p > (1 << 20) || n > (1 << 20)) return false;
  // 4 x 4 numerator tiles of the larger own slice
  const int64_t mnm = std::max((n + sms - 1) / sms, (p + sms - 1) / sms);
  if ((mnm + 3) / 4 * (rpad4(r) / 4) > kMaxTasks) return false;
  return smem_for((int)p, (int)n, r, sms) + 1024 <= smem_optin;
}

size_t resident_workspace_floats(int64_t p, int64_t n, int r, int sms) {
  return (size_t)(p + n) * rpad4(r) + 2 * (size_t)sms * (size_t)(r * (r + 1) / 2);
}

cudaError_t launch_resident(const float* V, float* W, float* H, int64_t p, int64_t n, int r,
                            float eps, bool h_first, int max_iters, int check_every, double tol,
                            const double* f0, float* work, double* fpart,
                            unsigned long long* bar, int* err, RunState* out, int sms,
                            cudaStream_t st) {
  const int G = sms;
  const int mc = (int)((n + G - 1) / G), mr = (int)((p + G - 1) / G);
  ResArgs a{};
  a.V = V;
  a.W = W;
  a.H = H;
  a.Wp = work;
  a.Hp = work + (size_t)p * rpad4(r);
  a.E = r * (r + 1) / 2;
  a.gpW = a.Hp + (size_t)n * rpad4(r);
  a.gpH = a.gpW + (size_t)G * a.E;
  a.p = (int)p;
  a.n = (int)n;
  a.r = r;
  a.eps = eps;
  a.h_first = h_first ? 1 : 0;
  a.max_iters = max_iters;
  a.check_every = check_every;
  a.tol = tol;
  a.f0 = f0;
  a.fpart = fpart;
  a.bar = bar;
  a.err = err;
  a.out = out;
  a.ldc = (mc + 3) & ~3;
  a.ldr = (mr + 3) & ~3;
  a.mnm = mc > mr ? mc : mr;
  const size_t smem = smem_for((int)p, (int)n, r, G);
  const void* kern = kernel_for(r);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kRT, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
  e = cudaMemsetAsync(bar, 0, kResidentBarWords * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  void* args[] = {&a};
  return cudaLaunchCooperativeKernel(kern, dim3((unsigned)G), dim3(kRT), args, smem, st);
}

}  // namespace nmf
