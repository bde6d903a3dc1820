// Batched form of the MM NMF path (placeholder until the grouped persistent
// kernel lands): the entry points exist and report NMF_EUNSUPPORTED.
#include "nmf_internal.cuh"

extern "C" {

nmf_status nmf_batched_init(int, const nmf_config*, const float* const*, float* const*,
                            float* const*, void*, nmf_batch** out) {
  if (out) *out = nullptr;
  return NMF_EUNSUPPORTED;
}
nmf_status nmf_batched_step(nmf_batch*, int) { return NMF_EUNSUPPORTED; }
nmf_status nmf_batched_objective(nmf_batch*, double*) { return NMF_EUNSUPPORTED; }
void nmf_batched_destroy(nmf_batch*) {}

}  // extern "C"
