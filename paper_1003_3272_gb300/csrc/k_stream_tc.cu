// Tensor-core (tcgen05) form of the two V-streaming products of an MM
// iteration (Section 3.1: the numerators V H^T of Eq. (3.3) and W^T V of
// Eq. (3.4)), for the TF32, split-BF16x3 and BF16 precisions.
//
// Both products are D[M x r] = X[M x K] . Y[r x K]^T with X and Y K-major
// (see k_stream_simt.cu for the operand roles).  A block owns a 128-row tile
// of X and one K-range (split-K):
//   warp 0, one lane : TMA producer.  Each pipeline stage holds 128 bytes of
//                      K (64 bf16 or 32 tf32 values) of the X tile (128 rows)
//                      and of the Y tile (RPAD rows), 128-byte swizzled.
//   warp 1, one lane : MMA issuer.  tcgen05.mma M=128, N=RPAD, K=32 bytes
//                      per instruction into a float32 accumulator in tensor
//                      memory; BF16x3 issues hi*hi + hi*lo + lo*hi.
//   all 4 warps      : read the accumulator (warp w owns TMEM lanes 32w..),
//                      then the split-K reduction (last block of a tile, in
//                      split order) and the fused multiply-divide epilogue.
// Every wait is bounded: on a timeout the block records NMF_ETIMEOUT in the
// error word, lets its copies and MMAs drain, frees its tensor memory and
// returns.
#include <cstdio>
#include <mutex>

#include "epilogue.cuh"
#include "tc.cuh"
#include "tc_ptx.cuh"

namespace nmf {
namespace {

constexpr int kThreads = 128;
constexpr int kBM = 128;
constexpr uint64_t kWaitLimitNs = 1500ull * 1000 * 1000;  // 1.5 s
constexpr int kSmemBudget = 200 * 1024;

struct TcParams {
  int64_t M, K;
  int r;
  int splits;
  int64_t kchunk;
  float* part;           // [tiles][splits][RPAD][128] partial numerators
  unsigned* counters;    // [tiles]
  EpiArgs ep;
  int* err;              // device error word (NMF_ETIMEOUT on a timeout)
};

template <int PREC>
struct PrecTraits;
template <> struct PrecTraits<NMF_TF32>   { static constexpr int XPL = 1, KB = 32, FMT = 2; };
template <> struct PrecTraits<NMF_BF16X3> { static constexpr int XPL = 2, KB = 64, FMT = 1; };
template <> struct PrecTraits<NMF_BF16>   { static constexpr int XPL = 1, KB = 64, FMT = 1; };

template <int PREC, int RPAD>
struct TcShape {
  static constexpr int XPL = PrecTraits<PREC>::XPL;
  static constexpr int X_BYTES = kBM * 128;       // one plane of X: 128 rows x 128 B
  static constexpr int Y_BYTES = RPAD * 128;      // one plane of Y
  static constexpr int STAGE = XPL * (X_BYTES + Y_BYTES);
  static constexpr int EPI = epi_smem_floats<kBM, RPAD>() * 4;
  static constexpr int STAGES_RAW = kSmemBudget / STAGE;
  static constexpr int STAGES = STAGES_RAW > 8 ? 8 : (STAGES_RAW < 2 ? 2 : STAGES_RAW);
  static constexpr int MAIN = STAGES * STAGE;
  static constexpr int SMEM = (MAIN > EPI ? MAIN : EPI) + 1024;   // + alignment slack
  static constexpr int TMEM_COLS = RPAD <= 32 ? 32 : (RPAD <= 64 ? 64 : 128);
};

template <int PREC, int RPAD>
__global__ void __launch_bounds__(kThreads, 1)
k_stream_tc(const __grid_constant__ CUtensorMap tx_hi, const __grid_constant__ CUtensorMap tx_lo,
            const __grid_constant__ CUtensorMap ty_hi, const __grid_constant__ CUtensorMap ty_lo,
            const TcParams a) {
  using S = TcShape<PREC, RPAD>;
  constexpr int STAGES = S::STAGES;
  constexpr int KB = PrecTraits<PREC>::KB;
  constexpr bool X3 = PREC == NMF_BF16X3;
  constexpr uint32_t IDESC = ptx::idesc(PrecTraits<PREC>::FMT, kBM, RPAD);

  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[STAGES];
  __shared__ __align__(8) uint64_t empty_bar[STAGES];
  __shared__ __align__(8) uint64_t acc_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int s_abort;
  __shared__ int s_last;

  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const uint32_t sbase = ptx::smem_u32(smem);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tile = blockIdx.x, split = blockIdx.y;
  const int64_t m0 = (int64_t)tile * kBM;
  const int64_t kbeg = (int64_t)split * a.kchunk;
  const int64_t kend = min(a.K, kbeg + a.kchunk);
  const int nkb = kbeg < kend ? (int)ceil_div(kend - kbeg, KB) : 0;

  // stage s: [X_hi | X_lo | Y_hi | Y_lo]
  auto x_addr = [&](int s, int plane) { return sbase + s * S::STAGE + plane * S::X_BYTES; };
  auto y_addr = [&](int s, int plane) {
    return sbase + s * S::STAGE + S::XPL * S::X_BYTES + plane * S::Y_BYTES;
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
    ptx::tmem_alloc(ptx::smem_u32(&tmem_slot), S::TMEM_COLS);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer ----------------
    int issued = 0;
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % STAGES;
      const uint32_t ph = (uint32_t)(kb / STAGES) & 1u;
      if (!ptx::mbar_wait(ptx::smem_u32(&empty_bar[s]), ph ^ 1u, kWaitLimitNs)) {
        atomicExch(&s_abort, 1);
        break;
      }
      if (*(volatile int*)&s_abort) break;
      const uint32_t fb = ptx::smem_u32(&full_bar[s]);
      ptx::mbar_expect_tx(fb, S::STAGE);
      const int32_t kc = (int32_t)(kbeg + (int64_t)kb * KB);
      ptx::tma_load_2d(x_addr(s, 0), &tx_hi, kc, (int32_t)m0, fb);
      if (X3) ptx::tma_load_2d(x_addr(s, 1), &tx_lo, kc, (int32_t)m0, fb);
      ptx::tma_load_2d(y_addr(s, 0), &ty_hi, kc, 0, fb);
      if (X3) ptx::tma_load_2d(y_addr(s, 1), &ty_lo, kc, 0, fb);
      issued = kb + 1;
    }
    // Drain: the last load issued into each stage must have landed before
    // this block may exit (normal path: already consumed, returns at once).
    for (int kb = issued - 1; kb >= 0 && kb >= issued - STAGES; --kb) {
      const int s = kb % STAGES;
      const uint32_t ph = (uint32_t)(kb / STAGES) & 1u;
      if (!ptx::mbar_wait(ptx::smem_u32(&full_bar[s]), ph, kWaitLimitNs)) atomicExch(&s_abort, 1);
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer ----------------
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % STAGES;
      const uint32_t ph = (uint32_t)(kb / STAGES) & 1u;
      if (!ptx::mbar_wait(ptx::smem_u32(&full_bar[s]), ph, kWaitLimitNs)) {
        atomicExch(&s_abort, 1);
        break;
      }
      if (*(volatile int*)&s_abort) break;
      ptx::tc_fence_after();
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const uint64_t ah = ptx::sdesc_sw128(x_addr(s, 0) + kk * 32);
        const uint64_t bh = ptx::sdesc_sw128(y_addr(s, 0) + kk * 32);
        const uint32_t acc = (kb | kk) != 0;
        if (PREC == NMF_TF32) {
          ptx::mma_tf32(tmem, ah, bh, IDESC, acc);
        } else {
          ptx::mma_bf16(tmem, ah, bh, IDESC, acc);
          if (X3) {
            const uint64_t al = ptx::sdesc_sw128(x_addr(s, 1) + kk * 32);
            const uint64_t bl = ptx::sdesc_sw128(y_addr(s, 1) + kk * 32);
            ptx::mma_bf16(tmem, ah, bl, IDESC, 1);
            ptx::mma_bf16(tmem, al, bh, IDESC, 1);
          }
        }
      }
      ptx::mma_commit(ptx::smem_u32(&empty_bar[s]));
    }
    // Always signal: also covers MMAs still in flight on the abort path.
    ptx::mma_commit(ptx::smem_u32(&acc_bar));
  }
  __syncwarp();

  // ---------------- accumulator -> registers ----------------
  const bool acc_ok = ptx::mbar_wait(ptx::smem_u32(&acc_bar), 0, kWaitLimitNs);
  ptx::tc_fence_after();
  if (!acc_ok) atomicExch(&s_abort, 1);
  __syncthreads();
  const bool abort = *(volatile int*)&s_abort != 0;

  constexpr int LD = RPAD + 1;
  float* Ns = reinterpret_cast<float*>(smem);
  float* Os = Ns + kBM * LD;
  float* Gs = Os + kBM * LD;
  const int row = warp * 32 + lane;  // TMEM lane == tile row
  if (!abort) {
    float* part = a.part + ((int64_t)tile * a.splits + split) * RPAD * kBM;
#pragma unroll
    for (int c = 0; c < RPAD / 16; ++c) {
      float v[16];
      ptx::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c * 16), v);
      if (a.splits == 1) {
#pragma unroll
        for (int j = 0; j < 16; ++j) Ns[row * LD + c * 16 + j] = v[j];
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) part[(c * 16 + j) * kBM + row] = v[j];
      }
    }
  }
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 1) ptx::tmem_dealloc(tmem, S::TMEM_COLS);
  if (abort) {
    if (threadIdx.x == 0) atomicExch(a.err, (int)NMF_ETIMEOUT);
    return;
  }

  if (a.splits > 1) {
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      const unsigned prev = atomicAdd(&a.counters[tile], 1u);
      s_last = (prev == (unsigned)a.splits - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const float* base = a.part + (int64_t)tile * a.splits * RPAD * kBM;
    for (int i = threadIdx.x; i < RPAD * kBM; i += kThreads) {
      float sum = 0.f;
      for (int sp = 0; sp < a.splits; ++sp) sum += __ldcg(base + (int64_t)sp * RPAD * kBM + i);
      Ns[(i % kBM) * LD + (i / kBM)] = sum;
    }
    if (threadIdx.x == 0) a.counters[tile] = 0u;
  }
  __syncthreads();
  mu_epilogue<kBM, RPAD, kThreads>(Ns, Os, Gs, m0, tile, a.ep);
}

// ---------------------------------------------------------------------------
// Host side: tensor maps and launch.
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
// ld elements; box = 128 bytes of K x box_rows rows, 128-byte swizzle,
// zero fill outside the tensor.
bool make_map(CUtensorMap* map, const void* base, bool bf16, int64_t K, int64_t rows, int64_t ld,
              int box_rows, std::string* err) {
  EncodeTiled enc = get_encode();
  if (!enc) { if (err) *err = "cuTensorMapEncodeTiled unavailable"; return false; }
  const int esz = bf16 ? 2 : 4;
  cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * esz)};
  cuuint32_t box[2] = {(cuuint32_t)(128 / esz), (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                   2, const_cast<void*>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    if (err) *err = "cuTensorMapEncodeTiled failed (code " + std::to_string((int)r) + ")";
    return false;
  }
  return true;
}

template <int PREC, int RPAD>
cudaError_t launch_t(const TcPlan& pl, const TcParams& prm, cudaStream_t st) {
  using S = TcShape<PREC, RPAD>;
  auto kern = k_stream_tc<PREC, RPAD>;
  static bool attr_done = false;
  if (!attr_done) {
    cudaError_t e =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM);
    if (e != cudaSuccess) return e;
    attr_done = true;
  }
  dim3 grid((unsigned)pl.tiles, (unsigned)pl.splits);
  kern<<<grid, kThreads, S::SMEM, st>>>(pl.x_hi, pl.x_lo, pl.y_hi, pl.y_lo, prm);
  return cudaGetLastError();
}

template <int PREC>
cudaError_t launch_prec(const TcPlan& pl, const TcParams& prm, cudaStream_t st) {
  switch (pl.rpad) {
    case 16: return launch_t<PREC, 16>(pl, prm, st);
    case 32: return launch_t<PREC, 32>(pl, prm, st);
    case 48: return launch_t<PREC, 48>(pl, prm, st);
    case 64: return launch_t<PREC, 64>(pl, prm, st);
    case 80: return launch_t<PREC, 80>(pl, prm, st);
    case 96: return launch_t<PREC, 96>(pl, prm, st);
    case 112: return launch_t<PREC, 112>(pl, prm, st);
    case 128: return launch_t<PREC, 128>(pl, prm, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

nmf_status tc_plan(int prec, const void* X_hi, const void* X_lo, int64_t ldx, const void* Y_hi,
                   const void* Y_lo, int64_t ldy, int64_t M, int64_t K, int r, int sms,
                   int user_split, TcPlan* plan, std::string* err) {
  TcPlan& pl = *plan;
  pl.prec = prec;
  pl.rpad = rank_pad16(r);
  pl.block_m = kBM;
  pl.kblock = (prec == NMF_TF32) ? 32 : 64;
  pl.M = M; pl.K = K; pl.r = r;
  pl.tiles = (int)ceil_div(M, kBM);
  const int64_t nkb = ceil_div(K, pl.kblock);
  int splits;
  if (user_split > 0) {
    splits = user_split;
  } else {
    // About 4 waves of one block per SM, at least 4 k-blocks per split.
    splits = (int)ceil_div((int64_t)sms * 4, pl.tiles);
    const int64_t max_by_k = ceil_div(nkb, 4);
    if (splits > max_by_k) splits = (int)max_by_k;
    if (splits < 1) splits = 1;
  }
  pl.kchunk = ceil_div(nkb, splits) * pl.kblock;
  pl.splits = (int)ceil_div(K, pl.kchunk);
  const bool bf = prec != NMF_TF32;
  if (M > INT32_MAX || K > INT32_MAX) { if (err) *err = "size exceeds TMA coordinates"; return NMF_EINVAL; }
  if (!make_map(&pl.x_hi, X_hi, bf, K, M, ldx, kBM, err)) return NMF_ECUDA;
  if (!make_map(&pl.y_hi, Y_hi, bf, K, r, ldy, pl.rpad, err)) return NMF_ECUDA;
  if (prec == NMF_BF16X3) {
    if (!make_map(&pl.x_lo, X_lo, bf, K, M, ldx, kBM, err)) return NMF_ECUDA;
    if (!make_map(&pl.y_lo, Y_lo, bf, K, r, ldy, pl.rpad, err)) return NMF_ECUDA;
  } else {
    pl.x_lo = pl.x_hi;
    pl.y_lo = pl.y_hi;
  }
  return NMF_OK;
}

cudaError_t tc_launch(const TcPlan& pl, const SplitArgs& sp, const EpiArgs& ep, int* err,
                      cudaStream_t st) {
  TcParams prm{pl.M, pl.K, pl.r, sp.splits, sp.kchunk, sp.part, sp.counters, ep, err};
  switch (pl.prec) {
    case NMF_TF32: return launch_prec<NMF_TF32>(pl, prm, st);
    case NMF_BF16X3: return launch_prec<NMF_BF16X3>(pl, prm, st);
    case NMF_BF16: return launch_prec<NMF_BF16>(pl, prm, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace nmf
