// Plain float32 form (NMF_FP32) of the two V-streaming products of an MM
// iteration (Section 3.1: the numerators V H^T of Eq. (3.3) and W^T V of
// Eq. (3.4)), with the multiply-divide update fused behind them.
//
// Same frame as the tensor-core kernel (k_stream_tc.cu): a persistent grid of
// thread-block clusters, each cluster owning one 128-row tile of X at a time
// and splitting its K range over its S blocks; V is streamed by TMA from the
// tile-blocked float32 copy into a 128-byte-swizzled shared-memory ring;
// after the stream the cluster sums its partial tiles over distributed
// shared memory and the helper warps (tc_epi.cuh), which formed the other
// factor's Gram and the denominators during the stream, finish the update.
// The difference: the product is accumulated with float32 FMAs on the SM
// cores by eight compute warps (thread tile 4 rows x TR ranks, RPAD = 8 TR;
// for TR <= 4, 8 rows in two groups that split each stage's K, their partial
// tiles added in a fixed order), reading the swizzled stages with
// bank-conflict-free 16-byte loads.
//
// Warps: 0 = TMA producer (one lane); 1-8 = compute; 9-11 = helpers.
#include <cooperative_groups.h>

#include "epilogue.cuh"
#include "tc.cuh"
#include "tc_epi.cuh"
#include "tc_ptx.cuh"

namespace cg = cooperative_groups;

namespace nmf {
namespace {

constexpr int kThreads = 384;
constexpr int kCompute0 = 32;      // first compute thread
constexpr int kHelper0 = 288;      // first helper thread
constexpr int kNH = 96;            // helper threads (warps 9-11)
constexpr int kBM = 128;
constexpr int kKB = 32;            // float32 values of K per stage (128 bytes)
constexpr uint64_t kWaitLimitNs = 1500ull * 1000 * 1000;
constexpr uint64_t kWaitLimitCycles = 3000ull * 1000 * 1000;
constexpr int kSmemMax = 227 * 1024;

struct F32Params {
  int64_t M, K;
  int r;
  int S, tiles, nclusters;
  int64_t kper;
  int nkbt;
  EpiArgs ep;
  const float* Q;
  int q_layout;
  int64_t ldq, QM;
  double* gpart;
  float* Gpad;
  double* G64;
  unsigned long long* ctr;
  unsigned long long unit;   // every launch adds 2 * unit (see k_stream_tc.cu)
  unsigned long long skew;
  int old_first;             // see k_stream_tc.cu
  int* err;
};

template <int RPAD>
struct F32Shape {
  static constexpr int TR = RPAD / 8;
  static constexpr int X_BYTES = kBM * 128;
  static constexpr int Y_BYTES = RPAD * 128;
  static constexpr int STAGE = X_BYTES + Y_BYTES;
  static constexpr int LDA = RPAD + 4;
  static constexpr int ACC = kBM * LDA * 4;
  static constexpr int NSB = tcepi::kRmax * epi_ldn<RPAD>() * 4;
  // helpers' region: staging Qs, old rows Os, denominators Ds
  static constexpr int DED =
      (tcepi::dedicated_floats<RPAD>() + tcepi::kRmax * tcepi::ldd<RPAD>()) * 4;
  static constexpr int STAGES_RAW = (kSmemMax - DED - 2048) / STAGE;
  static constexpr int STAGES = STAGES_RAW > 8 ? 8 : STAGES_RAW;
  static constexpr int RING = STAGES * STAGE;
  static constexpr int MAIN = RING > ACC + NSB ? RING : ACC + NSB;
  static constexpr int SMEM = MAIN + DED + 1024;
  static_assert(STAGES >= 2, "pipeline needs two stages");
  static_assert(Y_BYTES % 1024 == 0, "stage slots stay 1024-byte aligned");
};

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ bool wait_counter(const unsigned long long* ctr,
                                             unsigned long long target) {
  const uint64_t t0 = ptx::globaltimer();
  while (ld_acquire(ctr) < target) {
    if (ptx::globaltimer() - t0 > kWaitLimitNs) return false;
  }
  return true;
}

// Counter protocol of the tensor-core kernel: each launch adds 2 * unit, so
// the launch's base is the multiple of 2 * unit below the value a block reads
// after griddepcontrol.wait and before its own first add.
__device__ __forceinline__ unsigned long long launch_base(const unsigned long long* ctr,
                                                          unsigned long long unit) {
  const unsigned long long v = ld_acquire(ctr);
  return v - v % (2ull * unit);
}
__device__ __forceinline__ unsigned long long phase_add(int grid, unsigned long long unit) {
  return blockIdx.x == 0 ? 1ull + unit - (unsigned long long)grid : 1ull;
}

template <int RPAD>
__global__ void __launch_bounds__(kThreads, 1)
k_stream_f32(const __grid_constant__ CUtensorMap tx, const __grid_constant__ CUtensorMap ty,
             const F32Params a) {
  using Sh = F32Shape<RPAD>;
  constexpr int STAGES = Sh::STAGES;
  constexpr int TR = Sh::TR;
  constexpr int LDA = Sh::LDA;
  constexpr int LDN = epi_ldn<RPAD>();

  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[STAGES];
  __shared__ __align__(8) uint64_t empty_bar[STAGES];
  __shared__ int s_abort;

  cg::cluster_group cluster = cg::this_cluster();
  const int S = a.S;
  const int q = (int)cluster.block_rank();
  const int cid = blockIdx.x / S;
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const uint32_t sbase = ptx::smem_u32(smem);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool compute = threadIdx.x >= kCompute0 && threadIdx.x < kHelper0;
  const bool helper = threadIdx.x >= kHelper0;
  const int h = threadIdx.x - kHelper0;

  float* Qs = reinterpret_cast<float*>(smem + Sh::MAIN);
  float* Os = Qs + tcepi::kQsRows * tcepi::ldq<RPAD>();
  float* Ds = Os + tcepi::kRmax * tcepi::ldo<RPAD>();

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      ptx::mbar_init(ptx::smem_u32(&full_bar[s]), 1);
      ptx::mbar_init(ptx::smem_u32(&empty_bar[s]), 8);   // one arrival per compute warp
    }
    s_abort = 0;
    ptx::fence_mbar_init();
    ptx::tma_prefetch(&tx);
    ptx::tma_prefetch(&ty);
  }
  __syncthreads();

  const int64_t kbeg = (int64_t)q * a.kper;
  const int64_t kend = min(a.K, kbeg + a.kper);
  const int nkb = kbeg < kend ? (int)ceil_div(kend - kbeg, kKB) : 0;
  const int R = kBM / S;

  // ---- helpers, prologue: first tile's old rows, the other factor's Gram --
  if (helper) {
    const int G = gridDim.x;
    ptx::pdl_wait();
    const unsigned long long base = h == 0 ? launch_base(a.ctr, a.unit) + a.skew : 0ull;
    // The first tile's old rows: before the Gram when the launch streams
    // long (they are then off the critical path), else while the other
    // blocks arrive at the Gram's first grid-wide step.
    auto first_old = [&]() {
      if (cid < a.tiles) {
        const int64_t row0 = (int64_t)cid * kBM + (int64_t)q * R;
        const int rows = (int)max((int64_t)0, min((int64_t)R, a.M - row0));
        tcepi::load_old<RPAD, kNH>(Os, a.ep, R, row0, rows, h);
      }
    };
    if (a.old_first) first_old();
    const int64_t q0 = (int64_t)blockIdx.x * a.QM / G;
    const int64_t q1 = (int64_t)(blockIdx.x + 1) * a.QM / G;
    tcepi::gram_rows<RPAD, kNH>(Qs, a.Q, a.q_layout, a.ldq, q0, q1, a.r,
                           a.gpart + (int64_t)blockIdx.x * a.r * a.r, h);
    __threadfence();
    tcepi::helper_sync<kNH>();
    if (h == 0) atomicAdd(a.ctr, phase_add(G, a.unit));
    if (!a.old_first) first_old();   // while the other blocks arrive
    if (h == 0 && !wait_counter(a.ctr, base + a.unit)) atomicExch(&s_abort, 1);
    tcepi::helper_sync<kNH>();
    if (!*(volatile int*)&s_abort) {
      const int rr = a.r * a.r;
      const int e0 = (int)((int64_t)blockIdx.x * rr / G);
      const int e1 = (int)((int64_t)(blockIdx.x + 1) * rr / G);
      tcepi::gram_reduce_slice<RPAD, kNH>(a.gpart, G, a.r, e0, e1, a.G64, a.Gpad,
                                     reinterpret_cast<double*>(Qs), h);
    }
    __threadfence();
    tcepi::helper_sync<kNH>();
    if (h == 0) atomicAdd(a.ctr, phase_add(G, a.unit));
    if (h == 0 && !wait_counter(a.ctr, base + 2ull * a.unit)) atomicExch(&s_abort, 1);
    tcepi::helper_sync<kNH>();
  }

  // compute thread layout: RT rows x TR ranks per thread.  RT = 8 (TR <= 4):
  // two groups of four warps split each stage's K (16-byte chunks 0-3 and
  // 4-7), rows rg + 16 i; RT = 4: one group, rows rg + 32 i.  Ranks cgi + 8 t.
  // (The 8-row tile halves the X loads per FMA; above TR = 4 its registers
  // cost more than that saves.)
  constexpr int RT = TR <= 4 ? 8 : 4;
  constexpr int NKG = RT / 4;                 // K groups
  constexpr int TPG = 256 / NKG;              // threads per group
  constexpr int RS = 128 / RT;                // row stride
  constexpr int CPG = 8 / NKG;                // 16-byte K chunks per group and stage
  const int c = threadIdx.x - kCompute0;
  const int kgrp = NKG == 2 ? ((c >> 7) & 1) : 0;
  const int rg = (((c % TPG) >> 5) << 2) + (c & 3);   // 0 .. RS-1
  const int cgi = (c & 31) >> 2;                      // 0..7

  int it = 0;
  int kb_base = 0;
  for (int tile = cid; tile < a.tiles; tile += a.nclusters, ++it) {
    const int64_t m0 = (int64_t)tile * kBM;
    const int64_t row0 = m0 + (int64_t)q * R;
    const int rows = (int)max((int64_t)0, min((int64_t)R, a.M - row0));
    const int nkb_run = *(volatile int*)&s_abort ? 0 : nkb;
    float acc[RT][TR];
#pragma unroll
    for (int i = 0; i < RT; ++i)
#pragma unroll
      for (int t = 0; t < TR; ++t) acc[i][t] = 0.f;

    if (warp == 0 && lane == 0) {
      // ---------------- TMA producer ----------------
      int issued = 0, pre = 0;
      if (it == 0) {
        pre = nkb_run < STAGES ? nkb_run : STAGES;
        for (int kb = 0; kb < pre; ++kb) {
          const uint32_t fb = ptx::smem_u32(&full_bar[kb]);
          ptx::mbar_expect_tx(fb, Sh::STAGE);
          ptx::tma_load_3d(sbase + kb * Sh::STAGE, &tx, 0, 0,
                           (int32_t)((int64_t)tile * a.nkbt + kbeg / kKB + kb), fb);
        }
        ptx::pdl_wait();
        ptx::pdl_launch_dependents();
        for (int kb = 0; kb < pre; ++kb)
          ptx::tma_load_2d(sbase + kb * Sh::STAGE + Sh::X_BYTES, &ty,
                           (int32_t)(kbeg + (int64_t)kb * kKB), 0,
                           ptx::smem_u32(&full_bar[kb]));
        issued = pre;
      }
      for (int kb = pre; kb < nkb_run; ++kb) {
        const int g = kb_base + kb;
        const int s = g % STAGES;
        const uint32_t ph = (uint32_t)(g / STAGES) & 1u;
        if (!ptx::mbar_wait(ptx::smem_u32(&empty_bar[s]), ph ^ 1u, kWaitLimitCycles)) {
          atomicExch(&s_abort, 1);
          break;
        }
        if (*(volatile int*)&s_abort) break;
        const uint32_t fb = ptx::smem_u32(&full_bar[s]);
        ptx::mbar_expect_tx(fb, Sh::STAGE);
        ptx::tma_load_3d(sbase + s * Sh::STAGE, &tx, 0, 0,
                         (int32_t)((int64_t)tile * a.nkbt + kbeg / kKB + kb), fb);
        ptx::tma_load_2d(sbase + s * Sh::STAGE + Sh::X_BYTES, &ty,
                         (int32_t)(kbeg + (int64_t)kb * kKB), 0, fb);
        issued = kb + 1;
      }
      for (int kb = issued - 1; kb >= 0 && kb >= issued - STAGES; --kb) {
        const int g = kb_base + kb;
        if (!ptx::mbar_wait(ptx::smem_u32(&full_bar[g % STAGES]), (uint32_t)(g / STAGES) & 1u,
                            kWaitLimitCycles))
          atomicExch(&s_abort, 1);
      }
    } else if (compute) {
      // ---------------- float32 FMA mainloop ----------------
      for (int kb = 0; kb < nkb_run; ++kb) {
        const int g = kb_base + kb;
        const int s = g % STAGES;
        const uint32_t ph = (uint32_t)(g / STAGES) & 1u;
        if (!ptx::mbar_wait(ptx::smem_u32(&full_bar[s]), ph, kWaitLimitCycles)) {
          atomicExch(&s_abort, 1);
          break;
        }
        // 128-byte swizzle: 16-byte chunk c4 of row m sits at chunk c4 ^ (m & 7);
        // every row this thread reads has the same (m & 7), so one XOR per
        // chunk places all its loads (immediate row offsets).
        const uint8_t* xb = smem + s * Sh::STAGE + rg * 128;
        const uint8_t* yb = smem + s * Sh::STAGE + Sh::X_BYTES + cgi * 128;
#pragma unroll
        for (int cc = 0; cc < CPG; ++cc) {
          const int c4 = kgrp * CPG + cc;
          const int xo = (c4 ^ (rg & 7)) << 4;
          const int yo = (c4 ^ cgi) << 4;
          float4 xv[RT], yv[TR];
#pragma unroll
          for (int i = 0; i < RT; ++i)
            xv[i] = *reinterpret_cast<const float4*>(xb + i * (RS * 128) + xo);
#pragma unroll
          for (int t = 0; t < TR; ++t)
            yv[t] = *reinterpret_cast<const float4*>(yb + t * (8 * 128) + yo);
#pragma unroll
          for (int i = 0; i < RT; ++i)
#pragma unroll
            for (int t = 0; t < TR; ++t) {
              acc[i][t] = fmaf(xv[i].x, yv[t].x, acc[i][t]);
              acc[i][t] = fmaf(xv[i].y, yv[t].y, acc[i][t]);
              acc[i][t] = fmaf(xv[i].z, yv[t].z, acc[i][t]);
              acc[i][t] = fmaf(xv[i].w, yv[t].w, acc[i][t]);
            }
        }
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive(ptx::smem_u32(&empty_bar[s]));
      }
    } else if (helper && !*(volatile int*)&s_abort) {
      if (it > 0) tcepi::load_old<RPAD, kNH>(Os, a.ep, R, row0, rows, h);
      tcepi::compute_den_smem<RPAD, kNH>(Qs, Os, Ds, a.Gpad, a.r, R, h);
    }
    __syncwarp();
    kb_base += nkb_run;
    if (it == 0) ptx::pdl_wait();
    __syncthreads();   // every stage consumed and landed; the ring is free
    const bool abort = *(volatile int*)&s_abort != 0;

    float* Acc = reinterpret_cast<float*>(smem);
    float* Ns = reinterpret_cast<float*>(smem + Sh::ACC);
    // the K groups' partial sums: group 1 stores, group 0 adds (fixed order)
    if (compute && !abort && kgrp == NKG - 1) {
#pragma unroll
      for (int i = 0; i < RT; ++i)
#pragma unroll
        for (int t = 0; t < TR; ++t) Acc[(rg + RS * i) * LDA + cgi + 8 * t] = acc[i][t];
    }
    if (NKG == 2) {
      if (compute) asm volatile("bar.sync 2, 256;" ::: "memory");   // the compute warps
      if (compute && !abort && kgrp == 0) {
#pragma unroll
        for (int i = 0; i < RT; ++i)
#pragma unroll
          for (int t = 0; t < TR; ++t) {
            float* p = &Acc[(rg + RS * i) * LDA + cgi + 8 * t];
            *p = acc[i][t] + *p;
          }
      }
    }
    cluster.sync();   // every block's partial tile is in its shared memory
    if (!abort) {
      // rows [q R, (q+1) R) of the tile: the S partial tiles summed in rank order
      for (int i = threadIdx.x; i < R * (RPAD / 4); i += kThreads) {
        const int m = i / (RPAD / 4), k4 = (i % (RPAD / 4)) * 4;
        const float4* mine = reinterpret_cast<const float4*>(&Acc[(q * R + m) * LDA + k4]);
        float4 v[8];
#pragma unroll
        for (int s = 0; s < 8; ++s)
          if (s < S) v[s] = *cluster.map_shared_rank(mine, s);
        float4 sum = v[0];
#pragma unroll
        for (int s = 1; s < 8; ++s)
          if (s < S) { sum.x += v[s].x; sum.y += v[s].y; sum.z += v[s].z; sum.w += v[s].w; }
        *reinterpret_cast<float4*>(&Ns[m * LDN + k4]) = sum;
      }
    }
    cluster.sync();   // peers are done reading this block's tile
    if (!*(volatile int*)&s_abort)
      tcepi::finish_smem<RPAD, kThreads>(Ns, Os, Ds, a.ep, R, row0, rows);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
  }
  if (*(volatile int*)&s_abort && threadIdx.x == 0) atomicExch(a.err, (int)NMF_ETIMEOUT);
}

template <int RPAD>
void* f32_ptr() { return reinterpret_cast<void*>(k_stream_f32<RPAD>); }

}  // namespace

bool f32_kernel_for(int rpad, void** fn, int* smem, int* threads) {
  *threads = kThreads;
  switch (rpad) {
#define NMF_F32(R) case R: *fn = f32_ptr<R>(); *smem = F32Shape<R>::SMEM; return true;
    NMF_F32(8) NMF_F32(16) NMF_F32(24) NMF_F32(32) NMF_F32(40) NMF_F32(48) NMF_F32(56)
    NMF_F32(64) NMF_F32(72) NMF_F32(80) NMF_F32(88) NMF_F32(96) NMF_F32(104) NMF_F32(112)
    NMF_F32(120) NMF_F32(128)
#undef NMF_F32
  }
  return false;
}

// The float32 kernel shares the tensor-core kernel's parameter meaning; this
// packs a TcParams-equivalent launch for it.
cudaError_t f32_launch(const TcPlan& pl, const EpiArgs& ep, const TcGram& gr, int* err,
                       cudaStream_t st) {
  F32Params prm;
  prm.M = pl.M; prm.K = pl.K; prm.r = pl.r;
  prm.S = pl.S; prm.tiles = pl.tiles; prm.nclusters = pl.nclusters; prm.kper = pl.kchunk;
  prm.nkbt = pl.nkbt;
  prm.ep = ep;
  prm.Q = gr.Q; prm.q_layout = gr.q_layout; prm.ldq = gr.ldq; prm.QM = gr.QM;
  prm.gpart = gr.gpart; prm.Gpad = gr.Gpad; prm.G64 = gr.G64;
  prm.ctr = gr.ctr; prm.unit = gr.unit; prm.skew = gr.skew;
  prm.old_first = gr.old_first;
  prm.err = err;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)pl.grid, 1, 1);
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.dynamicSmemBytes = (size_t)pl.smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)pl.S;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  void* args[] = {(void*)&pl.x_hi, (void*)&pl.y_hi, (void*)&prm};
  cudaError_t e = cudaLaunchKernelExC(&cfg, pl.fn, args);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace nmf
