// Poisson variant (Section 3.1, closing paragraph) on the tensor cores:
// the split-BF16x3 form (NMF_BF16X3) of the two passes of k_poisson.cu.
//
// The update needs, at every entry of V, the ratio q = v / (b + eps) with
// b = W H from the same iteration, and then the numerators q H^T (for W) and
// W^T q (for H).  Pass 0 takes a 128-row panel I of V and a segment of its
// 64-column tiles J; per tile
//     MMA1   b[i][j]  = sum_k W[i][k] H[k][j]           M = 128, N = 64, K = r
//     epilogue  q[i][j] = v[i][j] / (b[i][j] + eps)    (0 where v = 0), split
//               into bf16 hi + lo and stored to tensor memory as the A
//               operand of
//     MMA2   N_W[i][k] += sum_j q[i][j] H[k][j]          M = 128, N = r, K = 64
// with N_W in tensor memory for the whole segment.  Pass 1 is the same with
// the roles of the factors swapped (128-column panel J, 64-row tiles I,
// b^T = H^T W^T, q^T, N_H += q^T W).  Every product is split BF16x3
// (hi hi + hi lo + lo hi): per K step, one MMA of A_hi against B's hi and lo
// planes stacked along N (N = 128, resp. 2 RP) and one of A_lo against B_hi
// (N = 64, resp. RP) into the first half, so that the result is the sum of
// the two halves of the accumulator.  V
// is read once per pass, as float32, from a tile-blocked copy made once when
// the plan is created: [128-row panel][32-column block][128][32], zero
// outside V, so that every TMA box is one contiguous piece of HBM (16 KB for
// pass 0, 8 KB for pass 1) and ragged shapes need no special case.  Each
// segment's numerator goes out as float32 partials [seg][rows][r].
//
// Both A operands live in tensor memory: the panel's factor rows (MMA1's A,
// the same for every tile of the segment, copied there once) and q (MMA2's
// A, written by the epilogue with tcgen05.st, double-buffered).  Shared
// memory carries only V and the other factor's tiles.
//
// Warps: 0 copies V, 1 issues the MMAs, 2 copies the panel's factor rows
// and B1, 3 copies B2 (one lane each), 4-11 epilogue (warp w: TMEM lanes
// 32 (w % 4) .., tile columns 32 ((w - 4) / 4) ..).  Rings, each released as
// soon as its reader is done with it: V (three stages; freed when the
// epilogue has read the tile into registers), B1 (the other factor's 64 rows
// for MMA1, three stages; freed when MMA1 completes) and B2 (the other
// factor's plane for MMA2, two stages; freed when MMA2 completes); q
// double-buffered in tensor memory.  An M = 128 BF16 MMA costs the tensor
// pipe about 45 cycles at N = 64 and 64 at N = 128, and the one thread that
// issues them competes for issue slots with the epilogue warps of its
// sub-partition: the stacked form issues 16 instructions per tile instead of
// 24.  MMA1 of the next tile is issued as soon as the epilogue has read b,
// before MMA2 of the current one.  Every wait is bounded: on expiry the block records
// NMF_ETIMEOUT, stops, waits (bounded) for its copies and MMAs and frees
// tensor memory.
//
// k_pois_finish then updates both factors from the partials (the float32
// form's update, fused), and from the new factors writes the operand planes
// and the denominators (row sums of H, column sums of W) the next
// iteration's passes and update read.
#include <cuda.h>

#include <algorithm>
#include <climits>
#include <cstdint>
#include <mutex>
#include <new>
#include <string>

#include "nmf_internal.cuh"
#include "tc_ptx_ta.cuh"

namespace nmf {
namespace {

constexpr int kEC = 32;               // tile columns per epilogue thread
constexpr int kNG = 64 / kEC;         // column groups
constexpr int kEpi = 4 * kNG * 32;    // epilogue threads (warps 4 ..): 4 lane quarters x kNG
constexpr int kPT = 128 + kEpi;       // threads: four single-lane roles + the epilogue
constexpr int kPM = 128;              // rows of a tile (tcgen05 M, TMEM lanes)
constexpr int kPN = 64;               // columns of a tile (MMA1 N, MMA2 K)
constexpr int kPlaneK = 64;           // bf16 elements per row of the K-major factor planes
constexpr int kNV = 3;                // V stages
constexpr int kNB1 = 3;               // B1 stages
constexpr int kNB2 = 2;               // B2 stages
constexpr uint64_t kWait = 3000ull * 1000 * 1000;   // ~1.5 s at 2 GHz

// Tensor memory (512 columns of 32 bits x 128 lanes):
//   [0, 128)    b: Ahi Bhi + Alo Bhi in [0, 64), Ahi Blo in [64, 128)
//   [128, 256)  q, two buffers: 32 columns of bf16 pairs hi, then 32 lo
//   [256, 320)  the panel's factor rows: 32 columns hi, 32 lo
//   [320, 320 + 2 RP)  the numerator, in the same two halves
constexpr int kColB = 0, kColQ = 128, kColA = 256, kColAcc = 320, kTCols = 512;

// Shared memory (bytes), every tile 1024-byte aligned:
//   A1 hi, lo     128 rows x 128 B each (staging for tensor memory)    32 KB
//   V  (3)        pass 0 two boxes 128 x 32 floats, pass 1 four
//                 boxes 64 x 32 floats                           3 x   32 KB
//   B1 hi, lo (3) 64 rows x 128 B each                           3 x   16 KB
//   B2 hi, lo (2) RP rows x 128 B each                           2 x 2 RP x 128 B
template <int RP>
struct PShape {
  static constexpr int A1 = 2 * kPM * 128;
  static constexpr int VT = kPM * kPN * 4;
  static constexpr int B1 = 2 * kPN * 128;
  static constexpr int B2 = 2 * RP * 128;
  static constexpr int OFF_V = A1;
  static constexpr int OFF_B1 = OFF_V + kNV * VT;
  static constexpr int OFF_B2 = OFF_B1 + kNB1 * B1;
  static constexpr int SMEM = OFF_B2 + kNB2 * B2 + 1024;
  static_assert(kColAcc + 2 * RP <= kTCols, "tensor memory columns");
  static_assert(SMEM <= 232448, "shared memory per block");
  static_assert(B2 % 1024 == 0, "B2 stages stay 1024-byte aligned");
};

// The tensor maps of one pass (see pois_tc_create).
struct PMaps {
  CUtensorMap a1_hi, a1_lo;   // the panel's factor rows: box 64 bf16 x 128 rows
  CUtensorMap b1_hi, b1_lo;   // the tile's rows of the other factor: box 64 x 64
  CUtensorMap v;              // blocked V {32, 128, blocks}: box 32 x 128 x 1 (pass 0)
                              // or 32 x 64 x 1 (pass 1)
  CUtensorMap b2_hi, b2_lo;   // the other factor's plane [rank][m]: box 64 x RP
};

struct PParams {
  int64_t rows;              // extent of the panel dimension (p for pass 0, n for pass 1)
  int r;
  float eps;
  int segs;                  // segments per panel
  int64_t tiles;             // tiles of kPN per panel
  int64_t nkb;               // 32-column blocks per 128-row panel of the blocked V
  float* part;               // [seg][rows][r]
  int* err;
  int test_extra_tx;         // added to the first V stage's byte count (tests)
};

// Two floats to their bf16 hi parts (packed) and lo parts (packed).
__device__ __forceinline__ void bf16_split2(float x0, float x1, uint32_t& hi, uint32_t& lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
  const __nv_bfloat162 l = __floats2bfloat162_rn(__fsub_rn(x0, __low2float(h)),
                                                 __fsub_rn(x1, __high2float(h)));
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

// kEC consecutive float32 columns of this warp's 32 lanes, loaded; kEC / 2
// columns stored at each of two addresses.
__device__ __forceinline__ void ld_cols(uint32_t ta, float* v) {
  if constexpr (kEC == 32) ptx::tmem_ld16x2(ta, ta + 16, v, v + 16);
  else ptx::tmem_ld16(ta, v);
}
__device__ __forceinline__ void st_cols(uint32_t ta, const uint32_t* a, uint32_t tb,
                                        const uint32_t* b) {
  if constexpr (kEC == 32) ptx::tmem_st16x2(ta, a, tb, b);
  else ptx::tmem_st8x2(ta, a, tb, b);
}

template <int PASS, int RP>
__global__ void __launch_bounds__(kPT, 1)
k_pois_tc(const __grid_constant__ PMaps mp, const PParams a) {
  using Sh = PShape<RP>;
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t a1_bar;          // A1 landed in shared memory
  __shared__ __align__(8) uint64_t a1_tmem;         // A1 stored to tensor memory
  __shared__ __align__(8) uint64_t v_full[kNV];
  __shared__ __align__(8) uint64_t v_empty[kNV];    // the epilogue read the V tile
  __shared__ __align__(8) uint64_t b1_full[kNB1];
  __shared__ __align__(8) uint64_t b1_empty[kNB1];  // MMA1 complete
  __shared__ __align__(8) uint64_t b2_full[kNB2];
  __shared__ __align__(8) uint64_t b2_empty[kNB2];  // MMA2 complete
  __shared__ __align__(8) uint64_t bfull;           // b ready in TMEM (MMA1 -> epilogue)
  __shared__ __align__(8) uint64_t bempty;          // b read (epilogue -> MMA1)
  __shared__ __align__(8) uint64_t qfull[2];        // q stored (epilogue -> MMA2)
  __shared__ __align__(8) uint64_t qempty[2];       // q read by MMA2 (MMA2 -> epilogue)
  __shared__ __align__(8) uint64_t done_bar;        // every MMA of this block complete
  __shared__ uint32_t tmem_slot;
  __shared__ int s_abort;

  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const uint32_t sbase = ptx::smem_u32(smem);
  const uint32_t a1_addr = sbase;
  auto v_addr = [&](int s) { return sbase + Sh::OFF_V + s * Sh::VT; };
  auto b1_addr = [&](int s) { return sbase + Sh::OFF_B1 + s * Sh::B1; };
  auto b2_addr = [&](int s) { return sbase + Sh::OFF_B2 + s * Sh::B2; };
  auto bar = [](uint64_t& b) { return ptx::smem_u32(&b); };
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t panel = blockIdx.x / a.segs;
  const int seg = blockIdx.x % a.segs;
  const int64_t t0 = (int64_t)seg * a.tiles / a.segs;
  const int64_t t1 = (int64_t)(seg + 1) * a.tiles / a.segs;
  const int nt = (int)(t1 - t0);

  if (threadIdx.x == 0) {
    ptx::mbar_init(bar(a1_bar), 1);
    ptx::mbar_init(bar(a1_tmem), kEpi);
    for (int s = 0; s < kNV; ++s) {
      ptx::mbar_init(bar(v_full[s]), 1);
      ptx::mbar_init(bar(v_empty[s]), kEpi);
    }
    for (int s = 0; s < kNB1; ++s) {
      ptx::mbar_init(bar(b1_full[s]), 1);
      ptx::mbar_init(bar(b1_empty[s]), 1);
    }
    for (int s = 0; s < kNB2; ++s) {
      ptx::mbar_init(bar(b2_full[s]), 1);
      ptx::mbar_init(bar(b2_empty[s]), 1);
    }
    ptx::mbar_init(bar(bfull), 1);
    ptx::mbar_init(bar(bempty), kEpi);
    for (int s = 0; s < 2; ++s) {
      ptx::mbar_init(bar(qfull[s]), kEpi);
      ptx::mbar_init(bar(qempty[s]), 1);
    }
    ptx::mbar_init(bar(done_bar), 1);
    s_abort = 0;
    ptx::fence_mbar_init();
  }
  if (warp == 1) {
    ptx::tmem_alloc(ptx::smem_u32(&tmem_slot), kTCols);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = tmem_slot;
  // Pass 1 reads nothing pass 0 writes, so pass 0 lets it be scheduled at
  // once: its blocks take the SMs pass 0 leaves idle, then those pass 0's
  // blocks free (see the end of the kernel for the other half of this).
  if (PASS == 0 && threadIdx.x == 0) ptx::pdl_launch_dependents();
  // copies started by this thread (its ring's tiles), for the drain at the end
  int issued = 0;
  bool a1_issued = false;

  if (warp == 0 && lane == 0) {
    // ---------------- V copies ----------------
    for (int t = 0; t < nt; ++t) {
      const int s = t % kNV;
      const uint32_t ph = (uint32_t)(t / kNV) & 1u;
      if (!ptx::mbar_wait(bar(v_empty[s]), ph ^ 1u, kWait)) {
        atomicExch(&s_abort, 1);
        break;
      }
      if (*(volatile int*)&s_abort) break;
      const int64_t c0 = (t0 + t) * kPN;   // first column (pass 0) / row (pass 1) of the tile
      const uint32_t vb = v_addr(s);
      const uint32_t fb = bar(v_full[s]);
      ptx::mbar_expect_tx(fb, Sh::VT + (t == 0 ? a.test_extra_tx : 0));
      if (PASS == 0) {
        // V rows panel*128 .., columns c0 .. c0+63: blocks 2 (c0 / 64) + h
        // of the panel, whole
        for (int h = 0; h < 2; ++h)
          ptx::tma_load_3d(vb + h * (kPM * 128), &mp.v, 0, 0,
                           (int32_t)(panel * a.nkb + 2 * (t0 + t) + h), fb);
      } else {
        // V rows c0 .. c0+63, columns panel*128 ..: rows c0 % 128 .. of
        // blocks 4 panel + h of row panel c0 / 128
        for (int h = 0; h < 4; ++h)
          ptx::tma_load_3d(vb + h * (kPN * 128), &mp.v, 0, (int32_t)(c0 % kPM),
                           (int32_t)((c0 / kPM) * a.nkb + 4 * panel + h), fb);
      }
      issued = t + 1;
    }
  } else if (warp == 2 && lane == 0) {
    // ---------------- the panel's factor rows, then B1 copies ----------------
    {
      const uint32_t fb = bar(a1_bar);
      ptx::mbar_expect_tx(fb, Sh::A1);
      ptx::tma_load_2d(a1_addr, &mp.a1_hi, 0, (int32_t)(panel * kPM), fb);
      ptx::tma_load_2d(a1_addr + kPM * 128, &mp.a1_lo, 0, (int32_t)(panel * kPM), fb);
      a1_issued = true;
    }
    for (int t = 0; t < nt; ++t) {
      const int s = t % kNB1;
      const uint32_t ph = (uint32_t)(t / kNB1) & 1u;
      if (!ptx::mbar_wait(bar(b1_empty[s]), ph ^ 1u, kWait)) {
        atomicExch(&s_abort, 1);
        break;
      }
      if (*(volatile int*)&s_abort) break;
      const int32_t c0 = (int32_t)((t0 + t) * kPN);
      ptx::mbar_expect_tx(bar(b1_full[s]), Sh::B1);
      ptx::tma_load_2d(b1_addr(s), &mp.b1_hi, 0, c0, bar(b1_full[s]));
      ptx::tma_load_2d(b1_addr(s) + kPN * 128, &mp.b1_lo, 0, c0, bar(b1_full[s]));
      issued = t + 1;
    }
  } else if (warp == 3 && lane == 0) {
    // ---------------- B2 copies ----------------
    for (int t = 0; t < nt; ++t) {
      const int s = t % kNB2;
      const uint32_t ph = (uint32_t)(t / kNB2) & 1u;
      if (!ptx::mbar_wait(bar(b2_empty[s]), ph ^ 1u, kWait)) {
        atomicExch(&s_abort, 1);
        break;
      }
      if (*(volatile int*)&s_abort) break;
      const int32_t c0 = (int32_t)((t0 + t) * kPN);
      ptx::mbar_expect_tx(bar(b2_full[s]), Sh::B2);
      ptx::tma_load_2d(b2_addr(s), &mp.b2_hi, c0, 0, bar(b2_full[s]));
      ptx::tma_load_2d(b2_addr(s) + RP * 128, &mp.b2_lo, c0, 0, bar(b2_full[s]));
      issued = t + 1;
    }
  }
  else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer ----------------
    // MMA1 of tile t + 1 goes out as soon as the epilogue has read b of
    // tile t, before MMA2 of tile t, which needs the epilogue's q of tile t.
    // Each K step is two instructions: A_hi against B's hi and lo planes
    // stacked along N, then A_lo against B_hi.  Both A operands come from
    // tensor memory.
    constexpr uint32_t ID1W = ptx::idesc(1, kPM, 2 * kPN), ID1N = ptx::idesc(1, kPM, kPN);
    constexpr uint32_t ID2W = ptx::idesc(1, kPM, 2 * RP), ID2N = ptx::idesc(1, kPM, RP);
    bool ok = ptx::mbar_wait(bar(a1_tmem), 0, kWait);
    ptx::tc_fence_after();
    const uint32_t a1_hi = tmem + (uint32_t)kColA;
    auto mma1 = [&](int t) -> bool {
      const int s1 = t % kNB1;
      if (!ptx::mbar_wait(bar(b1_full[s1]), (uint32_t)(t / kNB1) & 1u, kWait) ||
          !ptx::mbar_wait(bar(bempty), ((uint32_t)t & 1u) ^ 1u, kWait))
        return false;
      ptx::tc_fence_after();
      const uint64_t db = ptx::sdesc_sw128(b1_addr(s1));   // hi rows, then lo rows
      const uint32_t tb = tmem + (uint32_t)kColB;
      // +32 bytes along K per step: +2 in the descriptor's address field
#pragma unroll
      for (int kk = 0; kk < RP / 16; ++kk)
        ptx::mma2w_ta(tb, a1_hi + 8 * kk, a1_hi + 32 + 8 * kk, db + 2 * kk, ID1W, ID1N,
                      kk > 0 ? 1u : 0u);
      ptx::mma_commit(bar(bfull));
      ptx::mma_commit(bar(b1_empty[s1]));
      return true;
    };
    auto mma2 = [&](int t) -> bool {
      const int u = t & 1, s2 = t % kNB2;
      if (!ptx::mbar_wait(bar(qfull[u]), (uint32_t)(t >> 1) & 1u, kWait) ||
          !ptx::mbar_wait(bar(b2_full[s2]), (uint32_t)(t / kNB2) & 1u, kWait))
        return false;
      ptx::tc_fence_after();
      const uint64_t dh = ptx::sdesc_sw128(b2_addr(s2));   // hi rows, then lo rows
      const uint32_t qa = tmem + (uint32_t)(kColQ + 64 * u);
      const uint32_t td = tmem + (uint32_t)kColAcc;
#pragma unroll
      for (int kk = 0; kk < kPN / 16; ++kk)
        ptx::mma2w_ta(td, qa + 8 * kk, qa + 32 + 8 * kk, dh + 2 * kk, ID2W, ID2N,
                      (t > 0 || kk > 0) ? 1u : 0u);
      ptx::mma_commit(bar(qempty[u]));       // the q buffer may be rewritten
      ptx::mma_commit(bar(b2_empty[s2]));    // the B2 stage may be refilled
      return true;
    };
    if (nt > 0) ok = ok && mma1(0);
    for (int t = 0; ok && t < nt; ++t) {
      if (t + 1 < nt) ok = mma1(t + 1);
      if (ok) ok = mma2(t);
    }
    if (!ok) atomicExch(&s_abort, 1);
    // Always signal: covers MMAs still in flight on the abort path.
    ptx::mma_commit(bar(done_bar));
  }
  else if (warp >= 4) {
    // ---------------- epilogue warps ----
    // warp w: TMEM lanes (tile rows) 32 (w % 4) .., tile columns kEC cg ..
    const int quarter = warp & 3;
    const int cg = (warp - 4) >> 2;
    const int row = quarter * 32 + lane;
    const uint32_t tl = (uint32_t)(quarter * 32) << 16;
    // the panel's factor rows to tensor memory: this thread's kEC K-entries
    // of its row (16-byte chunks kEC / 8 cg .. of the swizzled row)
    bool ok = ptx::mbar_wait(bar(a1_bar), 0, kWait);
    ok = __all_sync(0xffffffffu, ok);
    if (ok) {
      uint32_t hi[kEC / 2], lo[kEC / 2];
#pragma unroll
      for (int c = 0; c < kEC / 8; ++c) {
        const int pos = (((kEC / 8) * cg + c) ^ (row & 7)) << 4;
        const uint4 x = *reinterpret_cast<const uint4*>(smem + row * 128 + pos);
        const uint4 y = *reinterpret_cast<const uint4*>(smem + kPM * 128 + row * 128 + pos);
        hi[4 * c] = x.x; hi[4 * c + 1] = x.y; hi[4 * c + 2] = x.z; hi[4 * c + 3] = x.w;
        lo[4 * c] = y.x; lo[4 * c + 1] = y.y; lo[4 * c + 2] = y.z; lo[4 * c + 3] = y.w;
      }
      st_cols(tmem + tl + (uint32_t)(kColA + (kEC / 2) * cg), hi,
              tmem + tl + (uint32_t)(kColA + 32 + (kEC / 2) * cg), lo);
      ptx::tc_fence_before();
      ptx::mbar_arrive(bar(a1_tmem));
    }
    for (int t = 0; t < nt && ok; ++t) {
      const int sv = t % kNV;
      const int s = t & 1;
      const uint32_t ph = (uint32_t)(t >> 1) & 1u;
      // the V tile landed (TMA) and MMA1 of this tile is complete
      ok = ptx::mbar_wait(bar(v_full[sv]), (uint32_t)(t / kNV) & 1u, kWait) &&
           ptx::mbar_wait(bar(bfull), (uint32_t)t & 1u, kWait);
      ok = __all_sync(0xffffffffu, ok);   // tensor-memory accesses are warp-collective
      if (!ok) break;
      ptx::tc_fence_after();
      float b[kEC], bl[kEC];
      ld_cols(tmem + tl + (uint32_t)(kColB + kEC * cg), b);
      ld_cols(tmem + tl + (uint32_t)(kColB + kPN + kEC * cg), bl);
      ptx::tc_fence_before();
      ptx::mbar_arrive(bar(bempty));
#pragma unroll
      for (int e = 0; e < kEC; ++e) b[e] = __fadd_rn(b[e], bl[e]);
      // v at this thread's kEC entries: pass 0 row `row` of the 128 x 64
      // tile, columns kEC cg .. (box of 32 columns kEC cg / 32); pass 1
      // column `row` of the 64 x 128 tile, rows kEC cg .. (box row / 32)
      const uint8_t* vb = smem + Sh::OFF_V + sv * Sh::VT;
      float v[kEC];
      if (PASS == 0) {
        const int c0 = kEC * cg;
        const uint8_t* bx = vb + (c0 >> 5) * (kPM * 128) + row * 128;
#pragma unroll
        for (int c = 0; c < kEC / 4; ++c) {
          const float4 x = *reinterpret_cast<const float4*>(
              bx + (((((c0 & 31) >> 2) + c) ^ (row & 7)) << 4));
          v[4 * c] = x.x;
          v[4 * c + 1] = x.y;
          v[4 * c + 2] = x.z;
          v[4 * c + 3] = x.w;
        }
      } else {
        const int jj = row & 31;
        const uint8_t* bx = vb + (row >> 5) * (kPN * 128) + ((jj & 3) << 2);
#pragma unroll
        for (int ii = 0; ii < kEC; ++ii) {
          const int i = kEC * cg + ii;
          v[ii] = *reinterpret_cast<const float*>(bx + i * 128 + (((jj >> 2) ^ (i & 7)) << 4));
        }
      }
      ptx::mbar_arrive(bar(v_empty[sv]));   // the V stage may be refilled
      // q = v / (b + eps), 0 where v = 0; hi + lo bf16, packed in pairs
      uint32_t qh[kEC / 2], ql[kEC / 2];
#pragma unroll
      for (int e = 0; e < kEC / 2; ++e) {
        const float x0 = v[2 * e], x1 = v[2 * e + 1];
        const float q0 = x0 > 0.f ? __fdividef(x0, __fadd_rn(b[2 * e], a.eps)) : 0.f;
        const float q1 = x1 > 0.f ? __fdividef(x1, __fadd_rn(b[2 * e + 1], a.eps)) : 0.f;
        bf16_split2(q0, q1, qh[e], ql[e]);
      }
      // MMA2 of tile t - 2 has read this q buffer
      ok = ptx::mbar_wait(bar(qempty[s]), ph ^ 1u, kWait);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) break;
      ptx::tc_fence_after();
      st_cols(tmem + tl + (uint32_t)(kColQ + 64 * s + (kEC / 2) * cg), qh,
              tmem + tl + (uint32_t)(kColQ + 64 * s + 32 + (kEC / 2) * cg), ql);
      ptx::tc_fence_before();
      ptx::mbar_arrive(bar(qfull[s]));
    }
    if (!ok) atomicExch(&s_abort, 1);
    // ---- the segment's numerator: the accumulators in order ----
    bool fin = ptx::mbar_wait(bar(done_bar), 0, kWait);
    fin = __all_sync(0xffffffffu, fin) && ok;
    if (!fin) atomicExch(&s_abort, 1);
    ptx::tc_fence_after();
    // warp-uniform: tensor-memory loads are collective
    const bool rd = __all_sync(0xffffffffu, fin && !*(volatile int*)&s_abort);
    const int64_t m = panel * kPM + row;
    float* dst = a.part + ((int64_t)seg * a.rows + m) * a.r;
#pragma unroll
    for (int c = 0; c < RP / 16; ++c) {
      if (c % kNG != cg) continue;   // the column groups split the rank chunks
      float sum[16];
#pragma unroll
      for (int e = 0; e < 16; ++e) sum[e] = 0.f;
      if (rd && nt > 0) {
        float x[16];
        ptx::tmem_ld16x2(tmem + tl + (uint32_t)(kColAcc + 16 * c),
                         tmem + tl + (uint32_t)(kColAcc + RP + 16 * c), sum, x);
#pragma unroll
        for (int e = 0; e < 16; ++e) sum[e] = __fadd_rn(sum[e], x[e]);
      }
      if (m < a.rows && rd) {
#pragma unroll
        for (int e = 0; e < 16; ++e)
          if (16 * c + e < a.r) dst[16 * c + e] = sum[e];
      }
    }
  }
  __syncwarp();
  // Teardown: every MMA of this block has completed and every copy it
  // started has landed (on the abort path the readers may have left before
  // the last stages arrived) before tensor memory is freed and the block
  // exits.
  if (threadIdx.x == 32 && !ptx::mbar_wait(bar(done_bar), 0, kWait)) atomicExch(&s_abort, 1);
  if (threadIdx.x == 0 || threadIdx.x == 64 || threadIdx.x == 96) {
    bool landed = threadIdx.x != 64 || !a1_issued || ptx::mbar_wait(bar(a1_bar), 0, kWait);
    const int nst = threadIdx.x == 0 ? kNV : (threadIdx.x == 64 ? kNB1 : kNB2);
    uint64_t* full = threadIdx.x == 0 ? v_full : (threadIdx.x == 64 ? b1_full : b2_full);
    for (int t = issued > nst ? issued - nst : 0; t < issued; ++t)
      landed = ptx::mbar_wait(bar(full[t % nst]), (uint32_t)(t / nst) & 1u, kWait) && landed;
    if (!landed) atomicExch(&s_abort, 1);
  }
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 1) ptx::tmem_dealloc(tmem, kTCols);
  if (*(volatile int*)&s_abort && threadIdx.x == 0) atomicExch(a.err, (int)NMF_ETIMEOUT);
  // Pass 1 completes only after pass 0 has: the update launched after it
  // reads both passes' partials.  (A no-op when not launched as a
  // programmatic dependent.)
  if (PASS == 1 && threadIdx.x == 0) ptx::pdl_wait();
}

// Factor planes for both passes, bf16 hi + lo each (entries of rank >= r and
// rows past the factor stay zero from the allocation):
//   Wb [p][64]   rows of W, K-major (pass 0's A1, pass 1's B1)
//   Wt [RP][ldp] W^T (pass 1's B2)
//   Hb [n][64]   columns of H, K-major (pass 1's A1, pass 0's B1)
//   Hp [RP][ldn] H itself (pass 0's B2)
struct Planes {
  __nv_bfloat16 *wb[2], *wt[2], *hb[2], *hp[2];
};

struct FParams {
  float* W;
  float* H;
  int64_t p, n;
  int r;
  float eps;
  int update;                 // 0: the planes and denominators of W, H as they are
  const float* partW;         // [segW][p][r]
  int segW;
  const float* partH;         // [segH][n][r]
  int segH;
  double* sums;               // 2r: row sums of H, then column sums of W
  const int* err;             // set: a pass gave up, the factors stay as they are
  int64_t ldp, ldn, wblocks;
  Planes pl;
  float2* psum;               // [block][64] per-block sums, compensated (sum, correction)
  unsigned* counter;          // last-block counter (zero between launches)
};

// Kahan's compensated summation (Kahan 1965) in float32: the pair (s, c)
// carries the running sum and the part of it that rounding dropped.
__device__ __forceinline__ void kahan_add(float& s, float& c, float x) {
  const float y = __fsub_rn(x, c);
  const float t = __fadd_rn(s, y);
  c = __fsub_rn(__fsub_rn(t, s), y);
  s = t;
}

// One block per 64 rows of W (blocks 0 .. wblocks-1) or 64 columns of H
// (the rest).  The slice is staged in shared memory; with `update`, each
// entry becomes x sqrt(num / (den + eps)), num the segment partials summed in
// segment order, den this iteration's denominator (float32 sum, ratio,
// square root and product, as in the float32 form).  Then the new slice
// goes to both of its operand planes (coalesced bf16-pair stores; rank
// entries r .. 63 of the K-major planes as zeros) and its per-rank sums
// (compensated float32, in order) to psum; the last block to finish sums
// those in block order into the denominators of the next iteration and
// rearms the counter (every block has read the old denominators before it
// counts itself).  No float64 arithmetic per entry: that pipe is narrow on
// this part, and the compensated sums carry about twice float32's digits.
constexpr int kPlT = 64;
constexpr int kFT = 512;    // threads of k_pois_finish: a few entries each
constexpr int kFS = kFT / kPlT;   // interleaved runs of the last block's sums
__global__ void __launch_bounds__(kFT) k_pois_finish(const FParams f) {
  __shared__ float tile[kPlT][kPlT + 1];
  __shared__ float den[kPlT];
  __shared__ float2 red[kFS][kPlT];
  __shared__ bool s_last;
  const int tid = threadIdx.x;
  const int r = f.r;
  const bool upd = f.update != 0 && !(f.err != nullptr && *(volatile const int*)f.err != 0);
  const bool wblock = (int64_t)blockIdx.x < f.wblocks;
  if (upd && tid < r) den[tid] = (float)(f.sums[wblock ? tid : r + tid] + (double)f.eps);
  __syncthreads();
  uint32_t h, l;
  if (wblock) {
    const int64_t i0 = (int64_t)blockIdx.x * kPlT;
    const int rows = (int)(f.p - i0 < kPlT ? f.p - i0 : kPlT);
    // rows i0 .. of W are contiguous, and so are their partials
    const float* pw = f.partW + i0 * r;
#pragma unroll 4
    for (int e = tid; e < rows * r; e += kFT) {
      const int ii = e / r, k = e - ii * r;
      float w = f.W[i0 * r + e];
      if (upd) {
        float num = __ldg(pw + e);
        for (int s = 1; s < f.segW; ++s) num = __fadd_rn(num, __ldg(pw + (int64_t)s * f.p * r + e));
        w = __fmul_rn(w, __fsqrt_rn(__fdiv_rn(num, den[k])));
        f.W[i0 * r + e] = w;
      }
      tile[ii][k] = w;
    }
    __syncthreads();
    if (tid < r) {
      float s = 0.f, c = 0.f;
      for (int ii = 0; ii < rows; ++ii) kahan_add(s, c, tile[ii][tid]);
      f.psum[(int64_t)blockIdx.x * kPlT + tid] = make_float2(s, c);
    }
    // Wb: row i, rank pairs (k, k + 1)
    for (int e = tid; e < rows * 32; e += kFT) {
      const int ii = e >> 5, k = 2 * (e & 31);
      bf16_split2(k < r ? tile[ii][k] : 0.f, k + 1 < r ? tile[ii][k + 1] : 0.f, h, l);
      const int64_t at = ((i0 + ii) * kPlaneK + k) >> 1;
      reinterpret_cast<uint32_t*>(f.pl.wb[0])[at] = h;
      reinterpret_cast<uint32_t*>(f.pl.wb[1])[at] = l;
    }
    // Wt: row k, entry pairs (i, i + 1); i0 and ldp are even, and a pair
    // reaching past p writes a zero into the row's padding (ldp > p then)
    for (int e = tid; e < r * 32; e += kFT) {
      const int k = e >> 5, ii = 2 * (e & 31);
      if (ii >= rows) continue;
      bf16_split2(tile[ii][k], ii + 1 < rows ? tile[ii + 1][k] : 0.f, h, l);
      const int64_t at = ((int64_t)k * f.ldp + i0 + ii) >> 1;
      reinterpret_cast<uint32_t*>(f.pl.wt[0])[at] = h;
      reinterpret_cast<uint32_t*>(f.pl.wt[1])[at] = l;
    }
  } else {
    const int64_t j0 = ((int64_t)blockIdx.x - f.wblocks) * kPlT;
    const int cols = (int)(f.n - j0 < kPlT ? f.n - j0 : kPlT);
    for (int e = tid; e < r * kPlT; e += kFT) {
      const int k = e >> 6, jj = e & 63;
      if (jj < cols) tile[k][jj] = f.H[(int64_t)k * f.n + j0 + jj];
    }
    __syncthreads();
    if (upd) {
      // the partials of columns j0 .. are contiguous ([j][k])
      const float* ph = f.partH + j0 * r;
#pragma unroll 4
      for (int e = tid; e < cols * r; e += kFT) {
        const int jj = e / r, k = e - jj * r;
        float num = __ldg(ph + e);
        for (int s = 1; s < f.segH; ++s) num = __fadd_rn(num, __ldg(ph + (int64_t)s * f.n * r + e));
        tile[k][jj] = __fmul_rn(tile[k][jj], __fsqrt_rn(__fdiv_rn(num, den[k])));
      }
      __syncthreads();
      for (int e = tid; e < r * kPlT; e += kFT) {
        const int k = e >> 6, jj = e & 63;
        if (jj < cols) f.H[(int64_t)k * f.n + j0 + jj] = tile[k][jj];
      }
    }
    if (tid < r) {
      float s = 0.f, c = 0.f;
      for (int jj = 0; jj < cols; ++jj) kahan_add(s, c, tile[tid][jj]);
      f.psum[(int64_t)blockIdx.x * kPlT + tid] = make_float2(s, c);
    }
    // Hp: row k, entry pairs (j, j + 1)
    for (int e = tid; e < r * 32; e += kFT) {
      const int k = e >> 5, jj = 2 * (e & 31);
      if (jj >= cols) continue;
      bf16_split2(tile[k][jj], jj + 1 < cols ? tile[k][jj + 1] : 0.f, h, l);
      const int64_t at = ((int64_t)k * f.ldn + j0 + jj) >> 1;
      reinterpret_cast<uint32_t*>(f.pl.hp[0])[at] = h;
      reinterpret_cast<uint32_t*>(f.pl.hp[1])[at] = l;
    }
    // Hb: row j, rank pairs (k, k + 1)
    for (int e = tid; e < cols * 32; e += kFT) {
      const int jj = e >> 5, k = 2 * (e & 31);
      bf16_split2(k < r ? tile[k][jj] : 0.f, k + 1 < r ? tile[k + 1][jj] : 0.f, h, l);
      const int64_t at = ((j0 + jj) * kPlaneK + k) >> 1;
      reinterpret_cast<uint32_t*>(f.pl.hb[0])[at] = h;
      reinterpret_cast<uint32_t*>(f.pl.hb[1])[at] = l;
    }
  }
  // the last block sums the per-block partials: kFS interleaved compensated
  // runs per rank, then those runs in order
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = atomicAdd(f.counter, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const int k = tid & 63, sl = tid >> 6;
  for (int side = 0; side < 2; ++side) {
    // side 0: row sums of H (blocks wblocks ..), side 1: column sums of W
    const int64_t b0 = side ? 0 : f.wblocks, b1 = side ? f.wblocks : (int64_t)gridDim.x;
    float s = 0.f, c = 0.f;
    if (k < r) {
      for (int64_t b = b0 + sl; b < b1; b += kFS) {
        const float2 x = __ldcg(f.psum + b * kPlT + k);
        kahan_add(s, c, -x.y);   // a pair (s, c) stands for s - c
        kahan_add(s, c, x.x);
      }
    }
    red[sl][k] = make_float2(s, c);
    __syncthreads();
    if (tid < r) {
      float ts = 0.f, tc = 0.f;
      for (int q = 0; q < kFS; ++q) {
        kahan_add(ts, tc, -red[q][tid].y);
        kahan_add(ts, tc, red[q][tid].x);
      }
      f.sums[side ? r + tid : tid] = (double)ts - (double)tc;
    }
    __syncthreads();
  }
  if (tid == 0) *f.counter = 0u;
}

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                 const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                 const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                 CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder() {
  static EncodeTiled fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(ptr);
    (void)cudaGetLastError();
  });
  return fn;
}

// A bf16 plane as a 2-D tensor: `inner` elements per row (row pitch `pitch`
// elements), `rows` rows; box = 64 elements (128 bytes) x box_rows rows,
// 128-byte swizzle, zero outside.
bool map_plane(CUtensorMap* m, const void* base, int64_t inner, int64_t rows, int64_t pitch,
               int box_rows) {
  EncodeTiled enc = encoder();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(pitch * 2)};
  cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box,
             es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

// The blocked V as a 3-D tensor {32 floats, 128 rows, blocks}: one box is
// box_rows rows of one block (contiguous), 128-byte swizzle.
bool map_v(CUtensorMap* m, const float* vb, int64_t blocks, int box_rows) {
  EncodeTiled enc = encoder();
  if (!enc) return false;
  cuuint64_t dims[3] = {32, (cuuint64_t)kPM, (cuuint64_t)blocks};
  cuuint64_t strides[2] = {32 * sizeof(float), (cuuint64_t)kPM * 32 * sizeof(float)};
  cuuint32_t box[3] = {32, (cuuint32_t)box_rows, 1};
  cuuint32_t es[3] = {1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(vb), dims, strides, box,
             es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

template <int PASS, int RP>
void* pois_fn() { return reinterpret_cast<void*>(k_pois_tc<PASS, RP>); }

void* kernel_for(int pass, int rp) {
  switch (rp) {
    case 16: return pass ? pois_fn<1, 16>() : pois_fn<0, 16>();
    case 32: return pass ? pois_fn<1, 32>() : pois_fn<0, 32>();
    case 48: return pass ? pois_fn<1, 48>() : pois_fn<0, 48>();
    case 64: return pass ? pois_fn<1, 64>() : pois_fn<0, 64>();
  }
  return nullptr;
}

int smem_for(int rp) {
  switch (rp) {
    case 16: return PShape<16>::SMEM;
    case 32: return PShape<32>::SMEM;
    case 48: return PShape<48>::SMEM;
    default: return PShape<64>::SMEM;
  }
}

size_t al256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

struct PoisTc {
  int64_t p = 0, n = 0, ldp = 0, ldn = 0;
  int r = 0, rp = 16;
  int segs[2] = {1, 1};
  int64_t tiles[2] = {0, 0};
  int smem = 0;
  int sms = 0;
  bool overlap = false;        // pass 1 as a programmatic dependent of pass 0
  void* fn[2] = {nullptr, nullptr};
  PMaps maps[2];
  Planes planes{};
  float* vb = nullptr;         // tile-blocked copy of V: [panel][block][128][32]
  int64_t nkb = 0;             // 32-column blocks per panel (a multiple of 4)
  float* part[2] = {nullptr, nullptr};   // numerator partials of W, H
  double* sums = nullptr;      // 2r denominators
  float2* psum = nullptr;      // per-block denominator partials (k_pois_finish)
  unsigned* counter = nullptr; // its last-block counter (zero between launches)
  int64_t fblocks[2] = {0, 0}; // k_pois_finish blocks over W, over H
  void* buf = nullptr;         // one allocation for all of the above
};

bool pois_tc_supported(int64_t p, int64_t n, int r) {
  return r >= 1 && r <= 64 && p >= 1 && n >= 1 && p <= INT32_MAX && n <= INT32_MAX;
}

void pois_tc_destroy(PoisTc* t) {
  if (!t) return;
  if (t->buf) cudaFree(t->buf);
  (void)cudaGetLastError();
  delete t;
}

PoisTc* pois_tc_create(const float* V, int64_t p, int64_t n, int r, int sms, cudaStream_t st,
                       std::string* err) {
  if (!pois_tc_supported(p, n, r)) {
    if (err) *err = "the tensor-core Poisson form needs 1 <= r <= 64";
    return nullptr;
  }
  PoisTc* t = new (std::nothrow) PoisTc;
  if (!t) return nullptr;
  t->p = p; t->n = n; t->r = r;
  t->rp = (int)round_up(r, 16);
  t->ldp = round_up(p, 8);
  t->ldn = round_up(n, 8);
  // pass 0: panels of 128 rows of V (p), tiles of 64 columns (n)
  // pass 1: panels of 128 columns of V (n), tiles of 64 rows (p)
  const int64_t panels[2] = {ceil_div(p, (int64_t)kPM), ceil_div(n, (int64_t)kPM)};
  t->tiles[0] = ceil_div(n, (int64_t)kPN);
  t->tiles[1] = ceil_div(p, (int64_t)kPN);
  for (int ps = 0; ps < 2; ++ps) {
    // segments per panel: the most that keep every block in one wave (one
    // block per SM), at most the panel's tiles
    int64_t sg = sms / panels[ps];
    if (sg < 1) sg = 1;
    if (sg > t->tiles[ps]) sg = t->tiles[ps];
    t->segs[ps] = (int)sg;
  }
  // The passes overlap only while pass 0 is one wave (every block resident
  // from the start): pass 1's blocks wait at their end for pass 0, so they
  // must never hold SMs that pass 0's later blocks need.
  t->sms = sms;
  t->overlap = panels[0] * t->segs[0] <= sms;
  t->fblocks[0] = ceil_div(p, (int64_t)kPlT);
  t->fblocks[1] = ceil_div(n, (int64_t)kPlT);
  // the blocked V: every 128-column panel of pass 1 is four whole blocks
  t->nkb = 4 * ceil_div(n, (int64_t)kPM);
  const int64_t vblocks = panels[0] * t->nkb;
  const size_t b_vb = al256((size_t)vblocks * kPM * 32 * sizeof(float));
  const size_t e_wb = (size_t)p * kPlaneK, e_wt = (size_t)t->rp * t->ldp;
  const size_t e_hb = (size_t)n * kPlaneK, e_hp = (size_t)t->rp * t->ldn;
  const size_t b_planes = al256(2 * (e_wb + e_wt + e_hb + e_hp) * sizeof(__nv_bfloat16));
  const size_t b_pw = al256((size_t)t->segs[0] * p * r * sizeof(float));
  const size_t b_ph = al256((size_t)t->segs[1] * n * r * sizeof(float));
  const size_t b_sums = al256(2 * (size_t)r * sizeof(double));
  const size_t b_psum = al256((size_t)(t->fblocks[0] + t->fblocks[1]) * kPlT * sizeof(float2));
  const size_t total = b_vb + b_planes + b_pw + b_ph + b_sums + b_psum + 256;
  // the copy kernel writes every entry of the blocked V, padding included;
  // the rest starts at zero (plane padding, counter)
  if (cudaMalloc(&t->buf, total) != cudaSuccess ||
      cudaMemsetAsync(static_cast<uint8_t*>(t->buf) + b_vb, 0, total - b_vb, st) != cudaSuccess) {
    (void)cudaGetLastError();
    if (err) *err = "cudaMalloc of the Poisson tensor-core workspace failed";
    pois_tc_destroy(t);
    return nullptr;
  }
  uint8_t* at = static_cast<uint8_t*>(t->buf);
  t->vb = reinterpret_cast<float*>(at);
  at += b_vb;
  __nv_bfloat16* b = reinterpret_cast<__nv_bfloat16*>(at);
  for (int h = 0; h < 2; ++h) {
    t->planes.wb[h] = b; b += e_wb;
    t->planes.wt[h] = b; b += e_wt;
    t->planes.hb[h] = b; b += e_hb;
    t->planes.hp[h] = b; b += e_hp;
  }
  at += b_planes;
  t->part[0] = reinterpret_cast<float*>(at);
  at += b_pw;
  t->part[1] = reinterpret_cast<float*>(at);
  at += b_ph;
  t->sums = reinterpret_cast<double*>(at);
  at += b_sums;
  t->psum = reinterpret_cast<float2*>(at);
  at += b_psum;
  t->counter = reinterpret_cast<unsigned*>(at);
  if (launch_operand_blocked(V, p, n, n, false, 2, t->vb, nullptr, t->nkb, 32, st) !=
      cudaSuccess) {
    (void)cudaGetLastError();
    if (err) *err = "cannot launch the blocked copy of V";
    pois_tc_destroy(t);
    return nullptr;
  }
  const Planes& pl = t->planes;
  bool ok = true;
  PMaps& m0 = t->maps[0];
  ok = ok && map_plane(&m0.a1_hi, pl.wb[0], kPlaneK, p, kPlaneK, kPM) &&
       map_plane(&m0.a1_lo, pl.wb[1], kPlaneK, p, kPlaneK, kPM) &&
       map_plane(&m0.b1_hi, pl.hb[0], kPlaneK, n, kPlaneK, kPN) &&
       map_plane(&m0.b1_lo, pl.hb[1], kPlaneK, n, kPlaneK, kPN) &&
       map_v(&m0.v, t->vb, vblocks, kPM) &&
       map_plane(&m0.b2_hi, pl.hp[0], n, t->rp, t->ldn, t->rp) &&
       map_plane(&m0.b2_lo, pl.hp[1], n, t->rp, t->ldn, t->rp);
  PMaps& m1 = t->maps[1];
  ok = ok && map_plane(&m1.a1_hi, pl.hb[0], kPlaneK, n, kPlaneK, kPM) &&
       map_plane(&m1.a1_lo, pl.hb[1], kPlaneK, n, kPlaneK, kPM) &&
       map_plane(&m1.b1_hi, pl.wb[0], kPlaneK, p, kPlaneK, kPN) &&
       map_plane(&m1.b1_lo, pl.wb[1], kPlaneK, p, kPlaneK, kPN) &&
       map_v(&m1.v, t->vb, vblocks, kPN) &&
       map_plane(&m1.b2_hi, pl.wt[0], p, t->rp, t->ldp, t->rp) &&
       map_plane(&m1.b2_lo, pl.wt[1], p, t->rp, t->ldp, t->rp);
  t->smem = smem_for(t->rp);
  for (int ps = 0; ps < 2 && ok; ++ps) {
    t->fn[ps] = kernel_for(ps, t->rp);
    ok = t->fn[ps] && cudaFuncSetAttribute(t->fn[ps], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           t->smem) == cudaSuccess;
  }
  if (!ok) {
    (void)cudaGetLastError();
    if (err) *err = "cannot set up the tensor-core Poisson passes (tensor maps or shared memory)";
    pois_tc_destroy(t);
    return nullptr;
  }
  return t;
}

namespace {
cudaError_t launch_finish(PoisTc* t, float* W, float* H, float eps, int update, const int* err,
                          cudaStream_t st) {
  FParams f;
  f.W = W;
  f.H = H;
  f.p = t->p;
  f.n = t->n;
  f.r = t->r;
  f.eps = eps;
  f.update = update;
  f.partW = t->part[0];
  f.segW = t->segs[0];
  f.partH = t->part[1];
  f.segH = t->segs[1];
  f.sums = t->sums;
  f.err = err;
  f.ldp = t->ldp;
  f.ldn = t->ldn;
  f.wblocks = t->fblocks[0];
  f.pl = t->planes;
  f.psum = t->psum;
  f.counter = t->counter;
  k_pois_finish<<<(unsigned)(t->fblocks[0] + t->fblocks[1]), kFT, 0, st>>>(f);
  return cudaGetLastError();
}
}  // namespace

cudaError_t pois_tc_prepare(PoisTc* t, const float* W, const float* H, cudaStream_t st) {
  // update = 0: the kernel only reads the factors
  return launch_finish(t, const_cast<float*>(W), const_cast<float*>(H), 0.f, 0, nullptr, st);
}

cudaError_t pois_tc_iteration(PoisTc* t, float* W, float* H, float eps, int* err,
                              int test_extra_tx, cudaStream_t st) {
  for (int ps = 0; ps < 2; ++ps) {
    PParams prm;
    prm.rows = ps == 0 ? t->p : t->n;
    prm.r = t->r;
    prm.eps = eps;
    prm.segs = t->segs[ps];
    prm.tiles = t->tiles[ps];
    prm.nkb = t->nkb;
    prm.part = t->part[ps];
    prm.err = err;
    prm.test_extra_tx = ps == 0 ? test_extra_tx : 0;
    const unsigned grid = (unsigned)(ceil_div(prm.rows, (int64_t)kPM) * prm.segs);
    void* args[] = {(void*)&t->maps[ps], (void*)&prm};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid, 1, 1);
    cfg.blockDim = dim3(kPT, 1, 1);
    cfg.dynamicSmemBytes = (size_t)t->smem;
    cfg.stream = st;
    // pass 1 as a programmatic dependent of pass 0 (the passes overlap)
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = ps == 1 && t->overlap ? 1 : 0;
    const cudaError_t e = cudaLaunchKernelExC(&cfg, t->fn[ps], args);
    if (e != cudaSuccess) return e;
  }
  return launch_finish(t, W, H, eps, 1, err, st);
}

}  // namespace nmf
