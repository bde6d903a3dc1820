// nmf_gram_noalloc: the Gram matrix of one factor without any allocation.
//
// Some callers of this library cannot call cudaMalloc: a host program whose
// device memory is handed out entirely by another allocator (a framework's
// caching allocator or a fixed arena sized at start-up), where a foreign
// cudaMalloc either fails or steals memory the arena counts on, and code on
// a latency-critical path, where cudaMalloc may synchronise the device.  For
// them this entry point computes F^T F (or F F^T) with the same two kernels
// the library uses for the starting Grams, but its scratch space is the
// file-scope device array below instead of a context workspace.
//
// The array's name is a host-side stand-in in host code, not a device
// address, so its device address is looked up once per device with
// cudaGetSymbolAddress (on the first call made with that device current)
// and then passed to the kernels.  Only a successful lookup is kept: after a
// failed one the next call tries again.  With CUDA's lazy module loading the
// library's device code, and the array with it, may be loaded on a device
// only at that first lookup, which can then allocate and synchronise inside
// the driver; so the first call per device belongs off the latency-critical
// path (at start-up, before any stream capture).  From then on the device
// holds the array until the process exits.  All calls share it and it keeps the
// last call's contents; the kernels overwrite every entry they later read,
// so nothing needs clearing.  Calls that overlap on the GPU (different
// streams, or different host threads) race on the array and must not be
// issued concurrently.
#include <cstdio>
#include <mutex>

#include "nmf_internal.cuh"

namespace {

// 2^21 floats = 8 MiB of scratch per device.
constexpr size_t kScratchFloats = size_t(1) << 21;
static __device__ __align__(256) float g_scratch[kScratchFloats];

constexpr int kMaxDevices = 64;
float* g_scratch_ptr[kMaxDevices];   // device address per device, once found
std::mutex g_setup_mu;

char* msg_buf() {
  static thread_local char buf[256];
  return buf;
}
nmf_status fail(nmf_status s, const char* what) {
  nmf::record_error(what);
  return s;
}

}  // namespace

extern "C" {

nmf_status nmf_gram_noalloc(const float* F, int32_t layout, int64_t M, int64_t ldf, int32_t r,
                            double* G_out, void* stream) {
  using namespace nmf;
  if (!F || !G_out) {
    return fail(NMF_EINVAL, "nmf_gram_noalloc: F and G_out must be non-NULL");
  }
  if (r < 1 || r > kMaxRank || M < 1 || (layout != 0 && layout != 1)) {
    return fail(NMF_EINVAL, "nmf_gram_noalloc: need 1 <= r <= 128, M >= 1, layout 0 or 1");
  }
  if ((layout == 0 && ldf != r) || (layout == 1 && ldf < M)) {
    return fail(NMF_EINVAL, "nmf_gram_noalloc: ldf must be r (layout 0) or >= M (layout 1)");
  }
  const int64_t tiles = ceil_div(M, 128);
  const int64_t need = tiles * r * r + (int64_t)r * r;
  if (need > (int64_t)kScratchFloats) {
    snprintf(msg_buf(), 256,
             "nmf_gram_noalloc: the problem needs %lld floats of scratch "
             "(ceil(M/128)*r*r + r*r) but the static scratch holds %lld",
             (long long)need, (long long)kScratchFloats);
    return fail(NMF_EINVAL, msg_buf());
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    snprintf(msg_buf(), 256, "nmf_gram_noalloc: cudaGetDevice: %s", cudaGetErrorString(e));
    return fail(NMF_ECUDA, msg_buf());
  }
  if (dev < 0 || dev >= kMaxDevices) {
    return fail(NMF_EUNSUPPORTED, "nmf_gram_noalloc: device ordinal beyond 63");
  }
  float* part = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_ptr[dev]) {
      float* p = nullptr;
      e = cudaGetSymbolAddress((void**)&p, g_scratch);
      if (e != cudaSuccess || !p) {
        snprintf(msg_buf(), 256, "nmf_gram_noalloc: cudaGetSymbolAddress: %s",
                 cudaGetErrorString(e));
        return fail(NMF_ECUDA, msg_buf());
      }
      g_scratch_ptr[dev] = p;
    }
    part = g_scratch_ptr[dev];
  }
  float* G32 = part + tiles * r * r;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if ((e = launch_gram_tiles(F, layout == 0 ? kFactorRowMajor : kFactorColMajor, M, ldf, r, part,
                             128, st)) != cudaSuccess ||
      (e = launch_gram_reduce(part, (int)tiles, r, G32, G_out, st)) != cudaSuccess) {
    snprintf(msg_buf(), 256, "nmf_gram_noalloc: launch: %s", cudaGetErrorString(e));
    return fail(NMF_ECUDA, msg_buf());
  }
  count_launches(2);
  return NMF_OK;
}

}  // extern "C"
