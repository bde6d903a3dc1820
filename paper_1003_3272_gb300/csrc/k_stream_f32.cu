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
// cores by eight compute warps (thread tile 8 rows x TR ranks, TR <= 8; the
// warps form NKG groups that split each stage's K, their partial tiles added
// in a fixed order, see F32Shape), reading the swizzled stages with
// bank-conflict-free 16-byte loads.
//
// Warps: 0 = TMA producer (one lane); 1-3 = helpers; 4-11 = compute (two
// warpgroups, which take registers from warpgroup 0 by setmaxnreg).
#include <cooperative_groups.h>

#include <type_traits>

#include "epilogue.cuh"
#include "tc.cuh"
#include "tc_epi.cuh"
#include "tc_ptx.cuh"

namespace cg = cooperative_groups;

namespace nmf {
namespace {

constexpr int kThreads = 384;
constexpr int kHelper0 = 32;       // first helper thread (warps 1-3)
constexpr int kNH = 96;            // helper threads
constexpr int kCompute0 = 128;     // first compute thread (warps 4-11)
// registers a thread after the split (setmaxnreg); the kernel is built with
// kRegsLaunch (= 65536 / 384, rounded down to a multiple of 8)
constexpr int kRegsLaunch = 168;
constexpr int kRegsWG0 = 136;
constexpr int kRegsCompute = 184;
static_assert(128 * kRegsWG0 + 256 * kRegsCompute == kThreads * kRegsLaunch,
              "the register split must add up to the launch's registers");
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

// Compute-thread tile: every compute thread accumulates 8 rows x TR ranks;
// the 8 warps form NKG groups that split each stage's K (group g takes the
// stage's 16-byte K chunks [g 8 / NKG, (g + 1) 8 / NKG)), so TR = RPAD NKG /
// 16.  NKG is chosen so that TR is close to 8: each value a thread reads
// from shared memory then feeds TR (X) or 8 (Y) FMAs, which keeps the FMA
// pipe ahead of the shared-memory bandwidth (one 128-byte wavefront per
// clock, four per 16-byte load).
template <int RPAD>
__host__ __device__ constexpr int f32_groups() {
  return RPAD <= 16 ? 8 : RPAD <= 32 ? 4 : RPAD <= 64 ? 2 : 1;
}

template <int RPAD>
struct F32Shape {
  static constexpr int NKG = f32_groups<RPAD>();
  static constexpr int TR = RPAD * NKG / 16;
  static_assert(TR * 16 == RPAD * NKG && TR >= 1 && TR <= 8, "rank padding of the FP32 tile");
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
  // after the stream: the K groups' partial tiles, then the cluster sums Ns
  static constexpr int MAIN = RING > NKG * ACC + NSB ? RING : NKG * ACC + NSB;
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
  const bool helper = threadIdx.x >= kHelper0 && threadIdx.x < kCompute0;
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

  // compute thread layout (see F32Shape): thread (group kgrp, row group rg,
  // rank group cgi) accumulates rows rg + 16 i (i < 8) and ranks cgi + GR t
  // (t < TR), GR = 16 / NKG rank groups.  Within each quarter warp the eight
  // lanes read one X row (a broadcast) or consecutive rows, and distinct
  // ranks, so the swizzled 16-byte loads are free of bank conflicts.
  constexpr int NKG = Sh::NKG;
  constexpr int GR = 16 / NKG;                // rank groups
  constexpr int TPG = 256 / NKG;              // threads per K group
  constexpr int CPG = 8 / NKG;                // 16-byte K chunks per group and stage
  const int c = threadIdx.x - kCompute0;
  const int kgrp = c / TPG;
  const int wg = (c % TPG) >> 5;
  int rg, cgi;
  if (GR >= 8) {
    cgi = (lane & 7) + 8 * (wg % (GR >= 8 ? GR / 8 : 1));
    rg = (lane >> 3) + 4 * (wg / (GR >= 8 ? GR / 8 : 1));
  } else {
    cgi = lane % GR;
    rg = lane / GR + (32 / GR) * wg;
  }

  // Register split (setmaxnreg): warpgroup 0 (the producer warp and the
  // helpers) runs with kRegsWG0 registers a thread, the two compute
  // warpgroups with kRegsCompute; the launch's 384 x 168 registers cover
  // exactly 128 x kRegsWG0 + 256 x kRegsCompute (the host launches only
  // when the kernel was built with 168).  Each side then runs its own copy
  // of the tile loop, so each copy is compiled within its own budget.
  auto tiles_loop = [&](auto role) {
    constexpr bool kComp = decltype(role)::value;
    int it = 0;
    int kb_base = 0;
    for (int tile = cid; tile < a.tiles; tile += a.nclusters, ++it) {
      const int64_t m0 = (int64_t)tile * kBM;
      const int64_t row0 = m0 + (int64_t)q * R;
      const int rows = (int)max((int64_t)0, min((int64_t)R, a.M - row0));
      const int nkb_run = *(volatile int*)&s_abort ? 0 : nkb;
      float acc[kComp ? 8 : 1][kComp ? TR : 1];
      if constexpr (kComp) {
        // ---------------- float32 FMA mainloop ----------------
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int t = 0; t < TR; ++t) acc[i][t] = 0.f;
        for (int kb = 0; kb < nkb_run; ++kb) {
          const int g = kb_base + kb;
          const int s = g % STAGES;
          const uint32_t ph = (uint32_t)(g / STAGES) & 1u;
          if (!ptx::mbar_wait(ptx::smem_u32(&full_bar[s]), ph, kWaitLimitCycles)) {
            atomicExch(&s_abort, 1);
            break;
          }
          // 128-byte swizzle: 16-byte chunk c4 of row m sits at chunk c4 ^ (m & 7);
          // the rows this thread reads share (m & 7), its ranks cgi + GR t too
          // when GR >= 8 (else the XOR is taken per rank).
          const uint8_t* xb = smem + s * Sh::STAGE + rg * 128;
          const uint8_t* yb = smem + s * Sh::STAGE + Sh::X_BYTES;
#pragma unroll 1
          for (int cc = 0; cc < CPG; ++cc) {
            const int c4 = kgrp * CPG + cc;
            const int xo = (c4 ^ (rg & 7)) << 4;
            float4 xv[8], yv[TR];
#pragma unroll
            for (int i = 0; i < 8; ++i)
              xv[i] = *reinterpret_cast<const float4*>(xb + i * (16 * 128) + xo);
#pragma unroll
            for (int t = 0; t < TR; ++t) {
              const int rk = cgi + GR * t;
              yv[t] = *reinterpret_cast<const float4*>(yb + rk * 128 + ((c4 ^ (rk & 7)) << 4));
            }
            // one K value at a time over the whole tile: consecutive FMAs
            // update different accumulators (no dependent chains); each
            // accumulator still adds its K values in increasing order
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
              for (int t = 0; t < TR; ++t) acc[i][t] = fmaf(xv[i].x, yv[t].x, acc[i][t]);
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
              for (int t = 0; t < TR; ++t) acc[i][t] = fmaf(xv[i].y, yv[t].y, acc[i][t]);
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
              for (int t = 0; t < TR; ++t) acc[i][t] = fmaf(xv[i].z, yv[t].z, acc[i][t]);
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
              for (int t = 0; t < TR; ++t) acc[i][t] = fmaf(xv[i].w, yv[t].w, acc[i][t]);
          }
          __syncwarp();
          if (lane == 0) ptx::mbar_arrive(ptx::smem_u32(&empty_bar[s]));
        }
      } else if (warp == 0 && lane == 0) {
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
          if (!ptx::mbar_wait(ptx::smem_u32(&full_bar[g % STAGES]),
                              (uint32_t)(g / STAGES) & 1u, kWaitLimitCycles))
            atomicExch(&s_abort, 1);
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
      float* Ns = reinterpret_cast<float*>(smem + NKG * Sh::ACC);
      if constexpr (kComp) {
        // each K group's partial tile into its own slot, then the slots
        // added in group order into slot 0 (fixed order)
        if (!abort) {
          float* mine = Acc + kgrp * (Sh::ACC / 4);
#pragma unroll
          for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int t = 0; t < TR; ++t) mine[(rg + 16 * i) * LDA + cgi + GR * t] = acc[i][t];
        }
        if (NKG > 1) {
          asm volatile("bar.sync 2, 256;" ::: "memory");   // the compute warps
          if (!abort) {
            for (int q4 = c; q4 < kBM * (RPAD / 4); q4 += 256) {
              const int m = q4 / (RPAD / 4), k4 = 4 * (q4 % (RPAD / 4));
              float4 v = *reinterpret_cast<const float4*>(&Acc[m * LDA + k4]);
#pragma unroll
              for (int g = 1; g < NKG; ++g) {
                const float4 w =
                    *reinterpret_cast<const float4*>(&Acc[g * (Sh::ACC / 4) + m * LDA + k4]);
                v.x += w.x; v.y += w.y; v.z += w.z; v.w += w.w;
              }
              *reinterpret_cast<float4*>(&Acc[m * LDA + k4]) = v;
            }
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
  };
  if (warp < 4) {
    ptx::setmaxnreg_dec<kRegsWG0>();
    tiles_loop(std::integral_constant<bool, false>{});
  } else {
    ptx::setmaxnreg_inc<kRegsCompute>();
    tiles_loop(std::integral_constant<bool, true>{});
  }
  if (*(volatile int*)&s_abort && threadIdx.x == 0) atomicExch(a.err, (int)NMF_ETIMEOUT);
}

template <int RPAD>
void* f32_ptr() { return reinterpret_cast<void*>(k_stream_f32<RPAD>); }

}  // namespace

// The kernel's register split (setmaxnreg) is sized for a build with
// kRegsLaunch registers a thread: with any other count the compute
// warpgroups' increase could wait forever, so such a build is not launched.
bool f32_regs_ok(void* fn) {
  cudaFuncAttributes at;
  if (cudaFuncGetAttributes(&at, fn) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  return at.numRegs == kRegsLaunch;
}

bool f32_kernel_for(int rpad, void** fn, int* smem, int* threads) {
  *threads = kThreads;
  switch (rpad) {
#define NMF_F32(R) case R: *fn = f32_ptr<R>(); *smem = F32Shape<R>::SMEM; return true;
    NMF_F32(8) NMF_F32(16) NMF_F32(24) NMF_F32(32) NMF_F32(40) NMF_F32(48) NMF_F32(56)
    NMF_F32(64) NMF_F32(80) NMF_F32(96) NMF_F32(112) NMF_F32(128)
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
