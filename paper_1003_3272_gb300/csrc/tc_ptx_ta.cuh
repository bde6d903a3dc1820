// Inline-PTX building blocks for kernels whose MMA A operand lives in
// tensor memory (tcgen05.st, tcgen05.mma with [a-tmem]); the rest of the
// tcgen05 / TMA / mbarrier helpers are in tc_ptx.cuh.
#pragma once

#include "tc_ptx.cuh"

namespace nmf {
namespace ptx {

// 32 lanes x 32 bits, 16 consecutive columns per thread, from registers, at
// two addresses; the wait makes both stores complete in this thread's view
// (a tcgen05 fence and a thread synchronisation then publish them to the
// MMA-issuing thread).
__device__ __forceinline__ void tmem_st16x2(uint32_t ta, const uint32_t* a, uint32_t tb,
                                            const uint32_t* b) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
      "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(ta),
      "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(a[6]), "r"(a[7]),
      "r"(a[8]), "r"(a[9]), "r"(a[10]), "r"(a[11]), "r"(a[12]), "r"(a[13]), "r"(a[14]),
      "r"(a[15])
      : "memory");
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
      "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(tb),
      "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(b[4]), "r"(b[5]), "r"(b[6]), "r"(b[7]),
      "r"(b[8]), "r"(b[9]), "r"(b[10]), "r"(b[11]), "r"(b[12]), "r"(b[13]), "r"(b[14]),
      "r"(b[15])
      : "memory");
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}
// The same with 8 columns per thread.
__device__ __forceinline__ void tmem_st8x2(uint32_t ta, const uint32_t* a, uint32_t tb,
                                           const uint32_t* b) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(ta),
               "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(a[6]),
               "r"(a[7])
               : "memory");
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(tb),
               "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(b[4]), "r"(b[5]), "r"(b[6]),
               "r"(b[7])
               : "memory");
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}
// D (tensor memory) += A (tensor memory: row m in lane m, two bf16 per
// 32-bit column along K) x B (shared memory descriptor), kind::f16.
__device__ __forceinline__ void mma_bf16_ta(uint32_t tmem_d, uint32_t tmem_a, uint64_t b,
                                            uint32_t id, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(tmem_d),
      "r"(tmem_a), "l"(b), "r"(id), "r"(accumulate)
      : "memory");
}

// One K step of a split-BF16x3 product with A in tensor memory: D (+)=
// Ahi Bhi, then D += Ahi Blo and D += Alo Bhi, in one block so that the
// issuing thread spends four instructions on the three MMAs.
__device__ __forceinline__ void mma3_ta(uint32_t d, uint32_t a_hi, uint32_t a_lo, uint64_t b_hi,
                                        uint64_t b_lo, uint32_t id, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p, t;\n\t"
      "setp.ne.b32 p, %6, 0;\n\t"
      "setp.eq.b32 t, %6, %6;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %3, %5, p;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %4, %5, t;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%2], %3, %5, t;\n\t}" ::"r"(d),
      "r"(a_hi), "r"(a_lo), "l"(b_hi), "l"(b_lo), "r"(id), "r"(accumulate)
      : "memory");
}

// One K step of a split-BF16x3 product with A in tensor memory and B's hi
// and lo planes stacked along N in shared memory (rows [0, N) hi, [N, 2N) lo,
// one descriptor): D[:, 0:2N] (+)= Ahi [Bhi; Blo] (id_wide: N' = 2N), then
// D[:, 0:N] += Alo Bhi (id_narrow: N' = N).  The product is then
// D[:, 0:N] + D[:, N:2N]; two instructions instead of three, the wide one at
// a better tensor rate.
__device__ __forceinline__ void mma2w_ta(uint32_t d, uint32_t a_hi, uint32_t a_lo, uint64_t b,
                                         uint32_t id_wide, uint32_t id_narrow,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p, t;\n\t"
      "setp.ne.b32 p, %5, 0;\n\t"
      "setp.eq.b32 t, %5, %5;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %3, %4, p;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%2], %3, %6, t;\n\t}" ::"r"(d),
      "r"(a_hi), "r"(a_lo), "l"(b), "r"(id_wide), "r"(accumulate), "r"(id_narrow)
      : "memory");
}

}  // namespace ptx
}  // namespace nmf
