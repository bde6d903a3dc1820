// Tensor-core (tcgen05) form of the two V-streaming products of an MM
// iteration (Section 3.1: the numerators V H^T of Eq. (3.3) and W^T V of
// Eq. (3.4)), for the TF32, split-BF16x3 and BF16 precisions, with the Gram
// of the other factor and the multiply-divide update fused into the same
// launch: one launch per half step.
//
// Both products are D[M x r] = X[M x K] . Y[r x K]^T with X and Y K-major:
// the H update has X = V^T (M = n, K = p) and Y = W^T, the W update X = V
// (M = p, K = n) and Y = H.  X is read from a tile-blocked copy (blocks of
// 128 rows x 128 bytes of K stored contiguously), Y from the factor's
// operand plane.
//
// Work decomposition.  A thread-block cluster of S blocks (S = 2, 4, 8) owns
// one 128-row tile of X at a time and splits its K range evenly; the grid is
// persistent (at most the co-resident number of clusters) and a cluster
// walks the tiles g, g + G, g + 2G, ...  Per block (256 threads):
//   warp 0, one lane : TMA producer.  A stage holds 128 (or 64) bytes of K of
//                      the X tile (128 rows) and of the Y tile (RPAD rows),
//                      swizzled to the stage width.
//   warp 1, one lane : MMA issuer, tcgen05.mma M=128, N=RPAD, 32 bytes of K
//                      per instruction, float32 accumulators in tensor
//                      memory; BF16x3 issues hi*hi + hi*lo + lo*hi.
//   warps 2-7        : helpers (tc_epi.cuh).  Prologue: the Gram of the
//                      other factor (per-block partials, grid-wide counter,
//                      fixed-order float64 reduction, counter).  During the
//                      stream: the old rows of this block's slice and the
//                      denominators old . G.
//   after the stream : accumulators to shared memory; the cluster sums its S
//                      partial tiles over distributed shared memory in rank
//                      order (deterministic), each block taking 128/S rows;
//                      then the update (IEEE multiply and divide) and the new
//                      factor's operand planes.
// Every wait is bounded: on a timeout the block records NMF_ETIMEOUT in the
// error word, lets its copies and MMAs drain, frees its tensor memory and
// returns.
#include <cooperative_groups.h>

#include <algorithm>
#include <cstdio>
#include <mutex>

#include "epilogue.cuh"
#include "tc.cuh"
#include "tc_epi.cuh"
#include "tc_ptx.cuh"

namespace cg = cooperative_groups;

namespace nmf {
namespace {

constexpr int kThreads = 256;   // 8 warps; warps 0-3 own the 128 TMEM lanes
constexpr int kBM = 128;
constexpr uint64_t kWaitLimitNs = 1500ull * 1000 * 1000;      // 1.5 s (global timer)
constexpr uint64_t kWaitLimitCycles = 3000ull * 1000 * 1000;  // ~1.5 s at 2 GHz
constexpr int kSmemMax = 227 * 1024;

struct TcParams {
  int64_t M, K;
  int r;
  int S;                 // cluster size = K-splits per tile (>= 2)
  int tiles;
  int nclusters;
  int64_t kper;          // K per split (multiple of the k-block)
  int nkbt;              // k-blocks per tile row (blocked X layout)
  int nacc;              // accumulators for the main products (k-block kb -> kb % nacc)
  int tmem_cols;         // tensor-memory columns allocated
  EpiArgs ep;            // the factor being updated and its planes
  // the other factor Q, whose Gram the helpers form in the prologue
  const float* Q;
  int q_layout;          // 0: Q[m * ldq + k] (W);  1: Q[k * ldq + m] (H)
  int64_t ldq;
  int64_t QM;            // rows of Q (p for W, n for H)
  double* gpart;         // [grid][r][r] per-block partial Grams (workspace)
  float* Gpad;           // [RPAD][RPAD] float32 Gram, zero padded
  double* G64;           // [r][r] float64 Gram
  unsigned long long* ctr;     // grid-wide publication counter (monotone)
  unsigned long long unit;     // every launch adds 2 * unit to it (unit >= grid)
  unsigned long long skew;     // added to the wait targets (0; test hook)
  int old_first;               // 1: the first tile's old rows before the Gram
  int* err;              // device error word
};

template <int PREC>
struct PrecTraits;
template <> struct PrecTraits<NMF_TF32>   { static constexpr int XPL = 1, FMT = 2; };
template <> struct PrecTraits<NMF_BF16X3> { static constexpr int XPL = 2, FMT = 1; };
template <> struct PrecTraits<NMF_BF16>   { static constexpr int XPL = 1, FMT = 1; };

// Bytes of K per stage: 128 (one block of the blocked copy), or 64 for split
// BF16x3 at ranks above 64, whose 128-byte stages (4 planes) would leave
// room for only two in shared memory; 64-byte stages (64-byte swizzle) give
// five.
template <int PREC, int RPAD>
__host__ __device__ constexpr int stage_kbytes() {
  return (PREC == NMF_BF16X3 && RPAD >= 80) ? 64 : 128;
}

// Sub-blocks of K per stage: single-plane forms (TF32, BF16) up to rank 64
// carry two 128-byte k-blocks per stage, so that a stage moves as many bytes
// as a split-BF16x3 stage (the per-stage cost of the pipeline is then paid
// half as often).
template <int PREC, int RPAD>
__host__ __device__ constexpr int stage_subs() {
  return (PREC != NMF_BF16X3 && RPAD <= 64) ? 2 : 1;
}

template <int PREC, int RPAD>
struct TcShape {
  static constexpr int XPL = PrecTraits<PREC>::XPL;
  static constexpr int KBY = stage_kbytes<PREC, RPAD>();
  static constexpr int NSUB = stage_subs<PREC, RPAD>();
  static constexpr int KB = KBY / (PREC == NMF_TF32 ? 4 : 2);   // K elements per sub-block
  static constexpr int X_BYTES = kBM * KBY;       // one plane of X: 128 rows x KBY
  static constexpr int Y_BYTES = RPAD * KBY;      // one plane of Y
  static constexpr int SUB = XPL * (X_BYTES + Y_BYTES);   // one sub-block: X planes, Y planes
  static constexpr int STAGE = NSUB * SUB;
  static constexpr int LDA = RPAD + 4;            // accumulator tile row stride (floats)
  static constexpr int ACC = kBM * LDA * 4;       // partial accumulator tile
  static constexpr int NSB = tcepi::kRmax * epi_ldn<RPAD>() * 4;   // reduced slice
  static constexpr int DED = tcepi::dedicated_floats<RPAD>() * 4;  // helpers' region
  static constexpr int STAGES_RAW = (kSmemMax - DED - 2048) / STAGE;
  static constexpr int STAGES = STAGES_RAW > 8 ? 8 : STAGES_RAW;
  static constexpr int RING = STAGES * STAGE;
  static constexpr int DSB = tcepi::kRmax * tcepi::ldd<RPAD>() * 4;  // denominators
  // Acc, Ns and Ds reuse the ring after the stream
  static constexpr int MAIN = RING > ACC + NSB + DSB ? RING : ACC + NSB + DSB;
  static constexpr int SMEM = MAIN + DED + 1024;   // + alignment slack
  // Tensor-memory column stride of one accumulator; the block allocates up
  // to 512 columns (it is alone on its SM: its shared memory exceeds half
  // of the SM's).
  static constexpr int CS = RPAD <= 32 ? 32 : (RPAD <= 64 ? 64 : 128);
  static_assert(STAGES >= 2, "pipeline needs two stages");
};

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// One helper thread waits (bounded) for the counter; false on timeout.
__device__ __forceinline__ bool wait_counter(const unsigned long long* ctr,
                                             unsigned long long target) {
  const uint64_t t0 = ptx::globaltimer();
  while (ld_acquire(ctr) < target) {
    if (ptx::globaltimer() - t0 > kWaitLimitNs) return false;
  }
  return true;
}

// The grid-wide counter carries no host-tracked state, so that a CUDA graph
// can replay the launch: every launch adds exactly 2 * unit (block 0 adds
// 1 + unit - grid in each of the two phases, every other block 1), launch
// bases are therefore multiples of 2 * unit, and a block reads its launch's
// base after the previous launch has completed (griddepcontrol.wait) and
// before its own first add, when the counter lies in [base, base + unit).
__device__ __forceinline__ unsigned long long launch_base(const unsigned long long* ctr,
                                                          unsigned long long unit) {
  const unsigned long long v = ld_acquire(ctr);
  return v - v % (2ull * unit);
}
__device__ __forceinline__ unsigned long long phase_add(int grid, unsigned long long unit) {
  return blockIdx.x == 0 ? 1ull + unit - (unsigned long long)grid : 1ull;
}

template <int PREC, int RPAD>
__global__ void __launch_bounds__(kThreads, 1)
k_stream_tc(const __grid_constant__ CUtensorMap tx_hi, const __grid_constant__ CUtensorMap tx_lo,
            const __grid_constant__ CUtensorMap ty_hi, const __grid_constant__ CUtensorMap ty_lo,
            const TcParams a) {
  using Sh = TcShape<PREC, RPAD>;
  constexpr int STAGES = Sh::STAGES;
  constexpr int KB = Sh::KB;
  constexpr int NSUB = Sh::NSUB;
  constexpr int KPB = 128 / Sh::KBY;   // sub-blocks per block of the blocked copy
  constexpr bool X3 = PREC == NMF_BF16X3;
  constexpr uint32_t IDESC = ptx::idesc(PrecTraits<PREC>::FMT, kBM, RPAD);
  constexpr int LDA = Sh::LDA;
  constexpr int LDN = epi_ldn<RPAD>();

  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[STAGES];
  __shared__ __align__(8) uint64_t empty_bar[STAGES];
  __shared__ __align__(8) uint64_t acc_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int s_abort;

  cg::cluster_group cluster = cg::this_cluster();
  const int S = a.S;
  const int q = (int)cluster.block_rank();
  const int cid = blockIdx.x / S;          // cluster index
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const uint32_t sbase = ptx::smem_u32(smem);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool helper = threadIdx.x >= tcepi::kHelperBase;
  const int h = threadIdx.x - tcepi::kHelperBase;

  // helpers' dedicated region: Qs | Os; denominators in the helpers' registers
  float* Qs = reinterpret_cast<float*>(smem + Sh::MAIN);
  float* Os = Qs + tcepi::kQsRows * tcepi::ldq<RPAD>();
  tcepi::DenFor<RPAD> den;

  auto x_addr = [&](int s, int plane, int sub = 0) {
    return sbase + s * Sh::STAGE + sub * Sh::SUB + plane * Sh::X_BYTES;
  };
  auto sdesc = [](uint32_t addr) {
    return Sh::KBY == 128 ? ptx::sdesc_sw128(addr) : ptx::sdesc_sw64(addr);
  };
  auto y_addr = [&](int s, int plane, int sub = 0) {
    return sbase + s * Sh::STAGE + sub * Sh::SUB + Sh::XPL * Sh::X_BYTES + plane * Sh::Y_BYTES;
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      ptx::mbar_init(ptx::smem_u32(&full_bar[s]), 1);
      ptx::mbar_init(ptx::smem_u32(&empty_bar[s]), 1);
    }
    ptx::mbar_init(ptx::smem_u32(&acc_bar), 1);
    s_abort = 0;
    ptx::fence_mbar_init();
    ptx::tma_prefetch(&tx_hi);
    ptx::tma_prefetch(&ty_hi);
    if (X3) { ptx::tma_prefetch(&tx_lo); ptx::tma_prefetch(&ty_lo); }
  }
  if (warp == 1) {
    ptx::tmem_alloc(ptx::smem_u32(&tmem_slot), (uint32_t)a.tmem_cols);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = tmem_slot;

  // K range of this block (same for every tile).
  const int64_t kbeg = (int64_t)q * a.kper;
  const int64_t kend = min(a.K, kbeg + a.kper);
  const int nkb = kbeg < kend ? (int)ceil_div(kend - kbeg, (int64_t)KB * NSUB) : 0;   // stages
  const int R = kBM / S;

  // ---- helpers, prologue: old rows of the first tile, then the Gram of the
  // other factor (partials over an even share of its rows, grid barrier,
  // this block's share of the entries, grid barrier) ------------------------
  if (helper) {
    const int G = gridDim.x;
    ptx::pdl_wait();   // the factors of the previous half step are final
    const unsigned long long base = h == 0 ? launch_base(a.ctr, a.unit) + a.skew : 0ull;
    // The first tile's old rows: before the Gram when the launch streams
    // long (they are then off the critical path), else while the other
    // blocks arrive at the Gram's first grid-wide step.
    auto first_old = [&]() {
      if (cid < a.tiles) {
        const int64_t row0 = (int64_t)cid * kBM + (int64_t)q * R;
        const int rows = (int)max((int64_t)0, min((int64_t)R, a.M - row0));
        tcepi::load_old<RPAD>(Os, a.ep, R, row0, rows, h);
      }
    };
    if (a.old_first) first_old();
    const int64_t q0 = (int64_t)blockIdx.x * a.QM / G;
    const int64_t q1 = (int64_t)(blockIdx.x + 1) * a.QM / G;
    tcepi::gram_rows<RPAD>(Qs, a.Q, a.q_layout, a.ldq, q0, q1, a.r,
                           a.gpart + (int64_t)blockIdx.x * a.r * a.r, h);
    __threadfence();
    tcepi::helper_sync();
    if (h == 0) atomicAdd(a.ctr, phase_add(G, a.unit));
    if (!a.old_first) first_old();   // while the other blocks arrive
    if (h == 0 && !wait_counter(a.ctr, base + a.unit)) atomicExch(&s_abort, 1);
    tcepi::helper_sync();
    if (!*(volatile int*)&s_abort) {
      const int rr = a.r * a.r;
      const int e0 = (int)((int64_t)blockIdx.x * rr / G);
      const int e1 = (int)((int64_t)(blockIdx.x + 1) * rr / G);
      tcepi::gram_reduce_slice<RPAD>(a.gpart, G, a.r, e0, e1, a.G64, a.Gpad,
                                     reinterpret_cast<double*>(Qs), h);
    }
    __threadfence();
    tcepi::helper_sync();
    if (h == 0) atomicAdd(a.ctr, phase_add(G, a.unit));
    if (h == 0 && !wait_counter(a.ctr, base + 2ull * a.unit)) atomicExch(&s_abort, 1);
    tcepi::helper_sync();
  }

  int it = 0;        // tiles processed by this block
  int kb_base = 0;   // k-blocks processed by this block (ring position)
  for (int tile = cid; tile < a.tiles; tile += a.nclusters, ++it) {
    const int64_t m0 = (int64_t)tile * kBM;
    const int64_t row0 = m0 + (int64_t)q * R;
    const int rows = (int)max((int64_t)0, min((int64_t)R, a.M - row0));
    const int nkb_run = *(volatile int*)&s_abort ? 0 : nkb;
    if (warp == 0 && lane == 0) {
      // ---------------- TMA producer ----------------
      // First tile: the X halves of the first stages go out before waiting
      // for the previous launch (V never changes); the Y halves (the factor
      // the previous launch wrote) after.
      int issued = 0;
      int pre = 0;
      if (it == 0) {
        pre = nkb_run < STAGES ? nkb_run : STAGES;
        for (int kb = 0; kb < pre; ++kb) {
          const uint32_t fb = ptx::smem_u32(&full_bar[kb]);
          ptx::mbar_expect_tx(fb, Sh::STAGE);
#pragma unroll
          for (int sub = 0; sub < NSUB; ++sub) {
            const int64_t hk = kbeg / KB + (int64_t)kb * NSUB + sub;
            const int32_t xb = (int32_t)((int64_t)tile * a.nkbt + hk / KPB);
            const int32_t xk = (int32_t)(hk % KPB) * KB;
            ptx::tma_load_3d(x_addr(kb, 0, sub), &tx_hi, xk, 0, xb, fb);
            if (X3) ptx::tma_load_3d(x_addr(kb, 1, sub), &tx_lo, xk, 0, xb, fb);
          }
        }
        ptx::pdl_wait();
        // Our own predecessor is complete: the next half step may now be
        // scheduled (its blocks take SMs as ours leave and prefetch V, which
        // no tensor-core launch writes, before they wait for us).
        ptx::pdl_launch_dependents();
        for (int kb = 0; kb < pre; ++kb) {
          const uint32_t fb = ptx::smem_u32(&full_bar[kb]);
#pragma unroll
          for (int sub = 0; sub < NSUB; ++sub) {
            const int32_t kc = (int32_t)(kbeg + ((int64_t)kb * NSUB + sub) * KB);
            ptx::tma_load_2d(y_addr(kb, 0, sub), &ty_hi, kc, 0, fb);
            if (X3) ptx::tma_load_2d(y_addr(kb, 1, sub), &ty_lo, kc, 0, fb);
          }
        }
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
#pragma unroll
        for (int sub = 0; sub < NSUB; ++sub) {
          // X block (tile, k-block) of the tile-blocked copy (or its half)
          const int64_t hk = kbeg / KB + (int64_t)kb * NSUB + sub;
          const int32_t kc = (int32_t)(hk * KB);
          const int32_t xb = (int32_t)((int64_t)tile * a.nkbt + hk / KPB);
          const int32_t xk = (int32_t)(hk % KPB) * KB;
          ptx::tma_load_3d(x_addr(s, 0, sub), &tx_hi, xk, 0, xb, fb);
          if (X3) ptx::tma_load_3d(x_addr(s, 1, sub), &tx_lo, xk, 0, xb, fb);
          ptx::tma_load_2d(y_addr(s, 0, sub), &ty_hi, kc, 0, fb);
          if (X3) ptx::tma_load_2d(y_addr(s, 1, sub), &ty_lo, kc, 0, fb);
        }
        issued = kb + 1;
      }
      // Drain: the last load issued into each stage must have landed.
      for (int kb = issued - 1; kb >= 0 && kb >= issued - STAGES; --kb) {
        const int g = kb_base + kb;
        if (!ptx::mbar_wait(ptx::smem_u32(&full_bar[g % STAGES]), (uint32_t)(g / STAGES) & 1u,
                            kWaitLimitCycles))
          atomicExch(&s_abort, 1);
      }
    } else if (warp == 1 && lane == 0) {
      // ---------------- MMA issuer ----------------
      // The tensor core's float32 accumulation is not round-to-nearest, so
      // its error grows with the number of additions into one accumulator.
      // The main products (hi x hi) rotate over nacc accumulators, k-block kb
      // into kb % nacc, and the small split-BF16 cross terms (2^-8 of the
      // main term) go to one accumulator of their own; the epilogue sums them
      // with IEEE adds.
      const uint32_t tcross = tmem + (uint32_t)(a.nacc * Sh::CS);
      int ai = 0;
      for (int kb = 0; kb < nkb_run; ++kb) {
        const int g = kb_base + kb;
        const int s = g % STAGES;
        const uint32_t ph = (uint32_t)(g / STAGES) & 1u;
        if (!ptx::mbar_wait(ptx::smem_u32(&full_bar[s]), ph, kWaitLimitCycles)) {
          atomicExch(&s_abort, 1);
          break;
        }
        if (*(volatile int*)&s_abort) break;
        ptx::tc_fence_after();
#pragma unroll
        for (int sub = 0; sub < NSUB; ++sub)
#pragma unroll
        for (int kk = 0; kk < Sh::KBY / 32; ++kk) {
          const uint64_t ah = sdesc(x_addr(s, 0, sub) + kk * 32);
          const uint64_t bh = sdesc(y_addr(s, 0, sub) + kk * 32);
          const uint32_t tacc = tmem + (uint32_t)(ai * Sh::CS);
          const uint32_t acc = (kb >= a.nacc || sub != 0 || kk != 0) ? 1u : 0u;
          if (PREC == NMF_TF32) {
            ptx::mma_tf32(tacc, ah, bh, IDESC, acc);
          } else {
            ptx::mma_bf16(tacc, ah, bh, IDESC, acc);
            if (X3) {
              const uint64_t al = sdesc(x_addr(s, 1, sub) + kk * 32);
              const uint64_t bl = sdesc(y_addr(s, 1, sub) + kk * 32);
              ptx::mma_bf16(tcross, ah, bl, IDESC, (kb | sub | kk) != 0);
              ptx::mma_bf16(tcross, al, bh, IDESC, 1);
            }
          }
        }
        ptx::mma_commit(ptx::smem_u32(&empty_bar[s]));
        if (++ai == a.nacc) ai = 0;
      }
      // Always signal: also covers MMAs still in flight on the abort path.
      ptx::mma_commit(ptx::smem_u32(&acc_bar));
    } else if (helper && !*(volatile int*)&s_abort) {
      // ---------------- helpers: old rows and denominators of this slice ----
      if (it > 0) {
        tcepi::load_old<RPAD>(Os, a.ep, R, row0, rows, h);   // first tile: in the prologue
      }
      tcepi::compute_den<RPAD>(Qs, Os, den, a.Gpad, a.r, R, h);
    }
    __syncwarp();
    kb_base += nkb_run;

    // ---------------- accumulator -> shared memory ----------------
    if (it == 0) ptx::pdl_wait();   // results of the previous launch are final
    const bool acc_ok = ptx::mbar_wait(ptx::smem_u32(&acc_bar), (uint32_t)it & 1u, kWaitLimitCycles);
    ptx::tc_fence_after();
    if (!acc_ok) atomicExch(&s_abort, 1);
    __syncthreads();
    const bool abort = *(volatile int*)&s_abort != 0;

    float* Acc = reinterpret_cast<float*>(smem);                  // [128][LDA] (ring region)
    float* Ns = reinterpret_cast<float*>(smem + Sh::ACC);         // [R][LDN]
    const int row = warp * 32 + lane;  // TMEM lane == tile row
    if (!abort && warp < 4) {
      const int used = nkb_run < a.nacc ? nkb_run : a.nacc;   // accumulators written
      const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll
      for (int c = 0; c < RPAD / 16; ++c) {
        float v[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = 0.f;
        // Fixed order: the main accumulators 0 .. used-1, then the cross
        // terms, loaded two at a time.
        const int nload = used + ((X3 && used > 0) ? 1 : 0);
        for (int ac = 0; ac < nload; ac += 2) {
          // load index i < used: main accumulator i; i == used: cross terms
          // (allocated only for X3); an odd tail re-loads a0 and skips it
          const bool two = ac + 1 < nload;
          const int a0 = ac < used ? ac : a.nacc;
          const int a1 = two ? (ac + 1 < used ? ac + 1 : a.nacc) : a0;
          float t0[16], t1[16];
          ptx::tmem_ld16x2(tl + (uint32_t)(a0 * Sh::CS + c * 16),
                           tl + (uint32_t)(a1 * Sh::CS + c * 16), t0, t1);
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            v[j] = __fadd_rn(v[j], t0[j]);
            if (two) v[j] = __fadd_rn(v[j], t1[j]);
          }
        }
#pragma unroll
        for (int j = 0; j < 16; j += 4)
          *reinterpret_cast<float4*>(&Acc[row * LDA + c * 16 + j]) =
              make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
      }
    }
    float* Ds = reinterpret_cast<float*>(smem + Sh::ACC + Sh::NSB);   // [R][RPAD + 4]
    if (!abort && helper) tcepi::den_to_smem<RPAD>(den, Ds, R, h);
    ptx::tc_fence_before();
    // Cluster barriers are executed the same number of times by every block
    // of a cluster, aborted or not, so no block can wait on a peer forever.
    cluster.sync();   // every block's partial tile (and its Ds) is in shared memory
    if (!abort) {
      // rows [q R, (q+1) R) of the tile: the S partial tiles summed in rank
      // order, and the update of each entry from old, num and den
      tcepi::cluster_update<RPAD, kThreads>(S, Acc, Ns, Os, Ds, a.ep, q, row0, rows);
    }
    __syncthreads();  // Ns is complete
    if (!abort) tcepi::store_cols<RPAD, kThreads>(Ns, a.ep, row0, rows);
    cluster.sync();   // peers are done reading this block's tile
    // The next tile's copies overwrite this shared memory through the async proxy.
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
  }

  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 1) ptx::tmem_dealloc(tmem, (uint32_t)a.tmem_cols);
  if (*(volatile int*)&s_abort && threadIdx.x == 0) atomicExch(a.err, (int)NMF_ETIMEOUT);
}

// ---------------------------------------------------------------------------
// Host side: tensor maps, work plan and launch.
// ---------------------------------------------------------------------------
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                 const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                 const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                 CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled get_encode() {
  static EncodeTiled fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(p);
    (void)cudaGetLastError();
  });
  return fn;
}

// 2-D K-major map: inner dimension K (elements), outer `rows`, row pitch
// ld elements; box = kbytes (128 or 64) bytes of K x box_rows rows, swizzle
// of the same width, zero fill outside the tensor.
bool make_map(CUtensorMap* map, const void* base, bool bf16, int64_t K, int64_t rows, int64_t ld,
              int box_rows, std::string* err, int kbytes = 128) {
  EncodeTiled enc = get_encode();
  if (!enc) { if (err) *err = "cuTensorMapEncodeTiled unavailable"; return false; }
  const int esz = bf16 ? 2 : 4;
  cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * esz)};
  cuuint32_t box[2] = {(cuuint32_t)(kbytes / esz), (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                   2, const_cast<void*>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE,
                   kbytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    if (err) *err = "cuTensorMapEncodeTiled failed (code " + std::to_string((int)r) + ")";
    return false;
  }
  return true;
}

// 3-D map over a tile-blocked copy: blocks of 128 rows x 128 bytes stored
// contiguously, `nblocks` of them; box = one block (kbytes = 128) or its
// left or right half (kbytes = 64, 64-byte swizzle).
bool make_map_blocked(CUtensorMap* map, const void* base, bool bf16, int64_t nblocks,
                      std::string* err, int kbytes = 128) {
  EncodeTiled enc = get_encode();
  if (!enc) { if (err) *err = "cuTensorMapEncodeTiled unavailable"; return false; }
  const int esz = bf16 ? 2 : 4;
  const int kbe = 128 / esz;
  cuuint64_t dims[3] = {(cuuint64_t)kbe, 128, (cuuint64_t)nblocks};
  cuuint64_t strides[2] = {128, 128 * 128};
  cuuint32_t box[3] = {(cuuint32_t)(kbytes / esz), 128, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                   3, const_cast<void*>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE,
                   kbytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    if (err) *err = "cuTensorMapEncodeTiled (blocked) failed (code " + std::to_string((int)r) + ")";
    return false;
  }
  return true;
}

template <int PREC, int RPAD>
void* kernel_ptr() {
  return reinterpret_cast<void*>(k_stream_tc<PREC, RPAD>);
}
template <int PREC, int RPAD>
int smem_bytes() {
  return TcShape<PREC, RPAD>::SMEM;
}

template <int PREC>
bool kernel_info(int rpad, void** fn, int* smem) {
  switch (rpad) {
#define NMF_CASE(R) case R: *fn = kernel_ptr<PREC, R>(); *smem = smem_bytes<PREC, R>(); return true;
    NMF_CASE(16) NMF_CASE(32) NMF_CASE(48) NMF_CASE(64)
    NMF_CASE(80) NMF_CASE(96) NMF_CASE(112) NMF_CASE(128)
#undef NMF_CASE
  }
  return false;
}

bool kernel_for(int prec, int rpad, void** fn, int* smem) {
  switch (prec) {
    case NMF_TF32: return kernel_info<NMF_TF32>(rpad, fn, smem);
    case NMF_BF16X3: return kernel_info<NMF_BF16X3>(rpad, fn, smem);
    case NMF_BF16: return kernel_info<NMF_BF16>(rpad, fn, smem);
  }
  return false;
}

cudaError_t prepare_kernel(void* fn, int smem) {
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  return cudaSuccess;
}

int max_clusters(void* fn, int smem, int threads, int S, int sms) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)((sms / S) * S), 1, 1);
  cfg.blockDim = dim3((unsigned)threads, 1, 1);
  cfg.dynamicSmemBytes = (size_t)smem;
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeClusterDimension;
  attr.val.clusterDim.x = (unsigned)S;
  attr.val.clusterDim.y = 1;
  attr.val.clusterDim.z = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, fn, &cfg) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  return n;
}

}  // namespace

nmf_status tc_plan(int prec, const void* X_hi, const void* X_lo, int64_t ldx, const void* Y_hi,
                   const void* Y_lo, int64_t ldy, int64_t M, int64_t K, int r, int sms,
                   int user_split, TcPlan* plan, std::string* err) {
  TcPlan& pl = *plan;
  pl.prec = prec;
  // float32 FMA path: ranks padded to 8 (16 above 64); tensor cores: N granularity 16
  pl.rpad = prec == NMF_FP32 ? rank_pad_f32(r) : rank_pad16(r);
  pl.block_m = kBM;
  // K elements per pipeline stage: 128 bytes, or 64 for split BF16x3 at
  // ranks above 64 (see stage_kbytes)
  const int kbytes = (prec == NMF_BF16X3 && pl.rpad >= 80) ? 64 : 128;
  const int esz = (prec == NMF_TF32 || prec == NMF_FP32) ? 4 : 2;
  // sub-blocks per stage (see stage_subs)
  const int nsub = (prec == NMF_TF32 || prec == NMF_BF16) && pl.rpad <= 64 ? 2 : 1;
  pl.kblock = nsub * kbytes / esz;   // K elements per pipeline stage
  pl.M = M; pl.K = K; pl.r = r;
  pl.tiles = (int)ceil_div(M, kBM);
  if (M > INT32_MAX || K > INT32_MAX) { if (err) *err = "size exceeds TMA coordinates"; return NMF_EINVAL; }
  void* fn = nullptr;
  int smem = 0, threads = kThreads;
  const bool have = prec == NMF_FP32 ? f32_kernel_for(pl.rpad, &fn, &smem, &threads)
                                     : kernel_for(prec, pl.rpad, &fn, &smem);
  if (!have) { if (err) *err = "no kernel for this rank"; return NMF_EINVAL; }
  if (prec == NMF_FP32 && !f32_regs_ok(fn)) {
    if (err) *err = "the float32 kernel was not built with the register count its warpgroup split needs";
    return NMF_ECUDA;
  }
  pl.threads = threads;
  if (prepare_kernel(fn, smem) != cudaSuccess) {
    (void)cudaGetLastError();
    if (err) *err = "cannot configure the tensor-core kernel's shared memory";
    return NMF_ECUDA;
  }
  pl.smem = smem;
  const int64_t nkb = ceil_div(K, pl.kblock);
  // Choose the cluster size S by a time model: a block's share of a tile,
  // ceil(nkb / S) stages at its share of HBM bandwidth (or, for the float32
  // form, at about half its FMA rate), plus the tile epilogue (cluster
  // reduction and update, a few microseconds growing with the rank), times
  // the rounds of tiles; ties go to the most blocks at work.
  const int xpl = prec == NMF_BF16X3 ? 2 : 1;
  double stage_us = 128.0 * kbytes * xpl * nsub / 44000.0;   // ~6.7 TB/s over 152 SMs
  if (prec == NMF_FP32)
    stage_us = std::max(stage_us, 128.0 * pl.kblock * pl.rpad / (128.0 * 1900.0 * 0.5));
  const double epi_us = 3.0 + pl.rpad / 16.0;
  int bestS = 0, bestG = 0;
  double best_cost = 1e300;
  int want = user_split;
  if (want > 0) {
    if (want != 1 && want != 2 && want != 4 && want != 8) {
      if (err) *err = "split_k must be 1, 2, 4 or 8 for tensor-core precisions";
      return NMF_EINVAL;
    }
    while (want > 2 && nkb < (int64_t)want) want /= 2;   // at most one split per k-block
  }
  if (want == 1) want = 2;   // a slice of at most 64 rows per block: clusters of >= 2
  for (int S = 2; S <= 8; S *= 2) {
    if (want > 0 && S != want) continue;
    if (S > 2 && nkb < (int64_t)S) continue;
    const int maxc = max_clusters(fn, smem, threads, S, sms);
    if (maxc < 1) continue;
    const int G = maxc < pl.tiles ? maxc : pl.tiles;
    const int rounds = (int)ceil_div(pl.tiles, G);
    const double cost = (double)rounds * ((double)ceil_div(nkb, S) * stage_us + epi_us);
    if (cost < best_cost - 1e-9 || (cost < best_cost + 1e-9 && G * S > bestG * bestS)) {
      best_cost = cost;
      bestS = S;
      bestG = G;
    }
  }
  if (bestS == 0) {
    if (err) *err = user_split > 0 ? "split_k must be 1, 2, 4 or 8 for tensor-core precisions "
                                     "(and at most the number of k-blocks)"
                                   : "no co-resident cluster configuration";
    return user_split > 0 ? NMF_EINVAL : NMF_EUNSUPPORTED;
  }
  pl.S = bestS;
  pl.nclusters = bestG;
  pl.splits = bestS;
  pl.kchunk = ceil_div(nkb, bestS) * pl.kblock;
  pl.grid = bestG * bestS;
  pl.fn = fn;
  // Accumulators: enough that no main accumulator takes more than about 256
  // additions (4 MMAs per k-block), at most 8 and within 512 columns.
  if (prec != NMF_FP32) {
    const int cs = pl.rpad <= 32 ? 32 : (pl.rpad <= 64 ? 64 : 128);
    const int cross = prec == NMF_BF16X3 ? 1 : 0;
    const int amax = (512 / cs - cross) < 8 ? 512 / cs - cross : 8;
    const int64_t adds = (pl.kchunk / pl.kblock) * nsub * (kbytes / 32);   // MMAs per stage
    int na = (int)ceil_div(adds, 256);
    pl.nacc = na < 1 ? 1 : (na > amax ? amax : na);
    int cols = 32;
    while (cols < (pl.nacc + cross) * cs) cols *= 2;
    pl.tmem_cols = cols;
  }
  const bool bf = prec == NMF_BF16X3 || prec == NMF_BF16;
  (void)ldx;
  // blocks of the blocked copy (128 bytes of K each) per tile row
  pl.nkbt = (int)ceil_div(K, (int64_t)(128 / esz));
  const int64_t nblocks = (int64_t)pl.tiles * pl.nkbt;
  if (!make_map_blocked(&pl.x_hi, X_hi, bf, nblocks, err, kbytes)) return NMF_ECUDA;
  if (!make_map(&pl.y_hi, Y_hi, bf, K, r, ldy, pl.rpad, err, kbytes)) return NMF_ECUDA;
  if (prec == NMF_BF16X3) {
    if (!make_map_blocked(&pl.x_lo, X_lo, bf, nblocks, err, kbytes)) return NMF_ECUDA;
    if (!make_map(&pl.y_lo, Y_lo, bf, K, r, ldy, pl.rpad, err, kbytes)) return NMF_ECUDA;
  } else {
    pl.x_lo = pl.x_hi;
    pl.y_lo = pl.y_hi;
  }
  return NMF_OK;
}

cudaError_t tc_launch(const TcPlan& pl, const EpiArgs& ep, const TcGram& gr, int* err,
                      cudaStream_t st) {
  if (pl.prec == NMF_FP32) return f32_launch(pl, ep, gr, err, st);
  TcParams prm;
  prm.M = pl.M; prm.K = pl.K; prm.r = pl.r;
  prm.S = pl.S; prm.tiles = pl.tiles; prm.nclusters = pl.nclusters; prm.kper = pl.kchunk;
  prm.nkbt = pl.nkbt;
  prm.nacc = pl.nacc;
  prm.tmem_cols = pl.tmem_cols;
  prm.ep = ep;
  prm.Q = gr.Q; prm.q_layout = gr.q_layout; prm.ldq = gr.ldq; prm.QM = gr.QM;
  prm.gpart = gr.gpart;
  prm.Gpad = gr.Gpad; prm.G64 = gr.G64;
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
  // Programmatic dependent launch: this grid may start while the previous
  // kernel in the stream drains; it waits (griddepcontrol.wait) before using
  // that kernel's results.
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  void* args[] = {(void*)&pl.x_hi, (void*)&pl.x_lo, (void*)&pl.y_hi, (void*)&pl.y_lo,
                  (void*)&prm};
  cudaError_t e = cudaLaunchKernelExC(&cfg, pl.fn, args);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace nmf
