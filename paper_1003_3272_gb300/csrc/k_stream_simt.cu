// Plain float32 form of the two V-streaming products (NMF_FP32).
//
// Both products of an MM iteration (Section 3.1: the numerators V H^T of
// Eq. (3.3) and W^T V of Eq. (3.4)) have the same shape once the data is
// laid out so that the contraction index is contiguous:
//     D[M x r] = X[M x K] . Y[r x K]^T
//   left update : X = V   (p x n),  Y = H     (r x n),   D = V H^T
//   right update: X = V^T (n x p),  Y = W^T   (r x p),   D = (W^T V)^T
// This kernel computes D with float32 FMAs on the SM cores.  A block owns a
// BM-row tile of X and one K-range (split-K).  X and Y k-blocks are staged
// through shared memory by cp.async (3-stage ring); each thread keeps a
// TM x TR register tile of D.  The block that finishes a tile last sums the
// split partials in split order (deterministic) and runs the fused
// multiply-divide epilogue (epilogue.cuh).
#include "epilogue.cuh"

namespace nmf {
namespace {

constexpr int kBK = 32;           // k-block depth (floats)
constexpr int kLDS = kBK + 4;     // smem row stride (floats): conflict-free LDS.128
constexpr int kStages = 3;
constexpr int kThreads = 128;     // 16 row groups x 8 rank groups

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int src_bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem),
               "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

struct SimtParams {
  const float* X; int64_t ldx;
  const float* Y; int64_t ldy;
  int64_t M, K; int r;
  SplitArgs sp;
  EpiArgs ep;
};

// TM rows x TR ranks per thread; BM = 16 * TM rows, RPAD = 8 * TR ranks.
template <int TM, int TR>
__global__ void __launch_bounds__(kThreads)
k_stream_simt(const SimtParams a) {
  constexpr int BM = 16 * TM;
  constexpr int RPAD = 8 * TR;
  extern __shared__ __align__(16) float smem[];
  float* Xs = smem;                                  // [kStages][BM][kLDS]
  float* Ys = smem + kStages * BM * kLDS;            // [kStages][RPAD][kLDS]
  __shared__ int s_last;

  const int tid = threadIdx.x;
  const int cg = tid & 7, rg = tid >> 3;
  const int tile = blockIdx.x, split = blockIdx.y;
  const int64_t m0 = (int64_t)tile * BM;
  const int64_t kb = (int64_t)split * a.sp.kchunk;
  const int64_t ke = min(a.K, kb + a.sp.kchunk);
  const int nch = kb < ke ? (int)ceil_div(ke - kb, kBK) : 0;

  auto load_stage = [&](int s, int ch) {
    const int64_t k0 = kb + (int64_t)ch * kBK;
    float* xs = Xs + s * BM * kLDS;
    float* ys = Ys + s * RPAD * kLDS;
    for (int q = tid; q < BM * (kBK / 4); q += kThreads) {
      const int row = q >> 3, kq = q & 7;
      const int64_t gk = k0 + kq * 4;
      const bool ok = (m0 + row < a.M) && (gk < ke);
      const float* src = ok ? a.X + (m0 + row) * a.ldx + gk : a.X;
      cp_async16(xs + row * kLDS + kq * 4, src, ok ? 16 : 0);
    }
    for (int q = tid; q < RPAD * (kBK / 4); q += kThreads) {
      const int row = q >> 3, kq = q & 7;
      const int64_t gk = k0 + kq * 4;
      const bool ok = (row < a.r) && (gk < ke);
      const float* src = ok ? a.Y + (int64_t)row * a.ldy + gk : a.Y;
      cp_async16(ys + row * kLDS + kq * 4, src, ok ? 16 : 0);
    }
  };

  float acc[TM][TR];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int t = 0; t < TR; ++t) acc[i][t] = 0.f;

#pragma unroll
  for (int s = 0; s < kStages - 1; ++s) {
    if (s < nch) load_stage(s, s);
    cp_async_commit();
  }
  for (int ch = 0; ch < nch; ++ch) {
    cp_async_wait<kStages - 2>();
    __syncthreads();
    {
      const int nxt = ch + kStages - 1;
      if (nxt < nch) load_stage(nxt % kStages, nxt);
      cp_async_commit();
    }
    const float* xs = Xs + (ch % kStages) * BM * kLDS;
    const float* ys = Ys + (ch % kStages) * RPAD * kLDS;
#pragma unroll 2
    for (int kq = 0; kq < kBK / 4; ++kq) {
      float4 xv[TM], yv[TR];
#pragma unroll
      for (int i = 0; i < TM; ++i)
        xv[i] = *reinterpret_cast<const float4*>(xs + (rg + 16 * i) * kLDS + kq * 4);
#pragma unroll
      for (int t = 0; t < TR; ++t)
        yv[t] = *reinterpret_cast<const float4*>(ys + (cg + 8 * t) * kLDS + kq * 4);
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int t = 0; t < TR; ++t) {
          acc[i][t] = fmaf(xv[i].x, yv[t].x, acc[i][t]);
          acc[i][t] = fmaf(xv[i].y, yv[t].y, acc[i][t]);
          acc[i][t] = fmaf(xv[i].z, yv[t].z, acc[i][t]);
          acc[i][t] = fmaf(xv[i].w, yv[t].w, acc[i][t]);
        }
    }
  }
  cp_async_wait<0>();
  __syncthreads();

  // Reuse the staging buffers for the epilogue tiles.
  constexpr int LD = epi_ldn<RPAD>();
  float* Ns = smem;
  float* Os = Ns + BM * LD;
  float* Gs = Os + BM * epi_ldo<RPAD>();

  if (a.sp.splits == 1) {
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int t = 0; t < TR; ++t) Ns[(rg + 16 * i) * LD + cg + 8 * t] = acc[i][t];
  } else {
    float* part = a.sp.part + ((int64_t)tile * a.sp.splits + split) * BM * RPAD;
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int t = 0; t < TR; ++t) part[(rg + 16 * i) * RPAD + cg + 8 * t] = acc[i][t];
    __threadfence();
    __syncthreads();
    if (tid == 0) {
      const unsigned prev = atomicAdd(&a.sp.counters[tile], 1u);
      s_last = (prev == (unsigned)a.sp.splits - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // Sum the partials of this tile in split order 0..splits-1.
    const float* base = a.sp.part + (int64_t)tile * a.sp.splits * BM * RPAD;
    for (int i = tid; i < BM * RPAD; i += kThreads) {
      float s = 0.f;
      for (int sp = 0; sp < a.sp.splits; ++sp) s += __ldcg(base + (int64_t)sp * BM * RPAD + i);
      Ns[(i / RPAD) * LD + (i % RPAD)] = s;
    }
    if (tid == 0) a.sp.counters[tile] = 0u;  // ready for the next launch
  }
  __syncthreads();
  mu_epilogue<RPAD, kThreads>(Ns, Os, Gs, BM, m0, a.ep.gram_part + (int64_t)tile * a.r * a.r,
                              a.ep);
}

template <int TM, int TR>
cudaError_t launch_t(const SimtParams& p, cudaStream_t st) {
  constexpr int BM = 16 * TM, RPAD = 8 * TR;
  const size_t stage = (size_t)kStages * (BM + RPAD) * kLDS * sizeof(float);
  const size_t epi = (size_t)epi_smem_floats<RPAD>(BM) * sizeof(float);
  const size_t smem = stage > epi ? stage : epi;
  auto kern = k_stream_simt<TM, TR>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)ceil_div(p.M, BM), (unsigned)p.sp.splits);
  kern<<<grid, kThreads, smem, st>>>(p);
  return cudaGetLastError();
}

}  // namespace

int simt_block_m(int r) { return (r <= 64) ? 128 : 64; }

cudaError_t launch_stream_simt(const float* X, int64_t ldx, const float* Y, int64_t ldy,
                               int64_t M, int64_t K, int r, const SplitArgs& sp,
                               const EpiArgs& ep, cudaStream_t st) {
  SimtParams p{X, ldx, Y, ldy, M, K, r, sp, ep};
  const int tr = (int)ceil_div(r, 8);
  if (r <= 64) {
    switch (tr) {
      case 1: return launch_t<8, 1>(p, st);
      case 2: return launch_t<8, 2>(p, st);
      case 3: return launch_t<8, 3>(p, st);
      case 4: return launch_t<8, 4>(p, st);
      case 5: return launch_t<8, 5>(p, st);
      case 6: return launch_t<8, 6>(p, st);
      case 7: return launch_t<8, 7>(p, st);
      case 8: return launch_t<8, 8>(p, st);
    }
  } else {
    switch (tr) {
      case 9: return launch_t<4, 9>(p, st);
      case 10: return launch_t<4, 10>(p, st);
      case 11: return launch_t<4, 11>(p, st);
      case 12: return launch_t<4, 12>(p, st);
      case 13: return launch_t<4, 13>(p, st);
      case 14: return launch_t<4, 14>(p, st);
      case 15: return launch_t<4, 15>(p, st);
      case 16: return launch_t<4, 16>(p, st);
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace nmf
