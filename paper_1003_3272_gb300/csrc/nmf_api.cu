// C ABI of the MM NMF library: contexts, workspaces, validation and the
// per-iteration launch sequence.  See include/nmf.h for the contract.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "nmf_internal.cuh"
#include "tc.cuh"

using namespace nmf;

namespace {

thread_local std::string g_last_error = "no error";
std::atomic<uint64_t> g_launches{0};

inline void launched(int k) { g_launches.fetch_add((uint64_t)k, std::memory_order_relaxed); }

void set_err(std::string* dst, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  if (dst) *dst = buf;
}

}  // namespace

namespace nmf {
void record_error(const char* msg) { g_last_error = msg; }
void count_launches(int k) { launched(k); }
}  // namespace nmf

// One V-streaming product followed by its fused epilogue: which operands,
// which factor, which workspace.
struct HalfPlan {
  // X operand (M x K, K contiguous) in the precision's format
  const void* X_hi = nullptr;
  const void* X_lo = nullptr;
  int64_t ldx = 0;
  // Y operand: plane of the other factor (r x K)
  const void* Y_hi = nullptr;
  const void* Y_lo = nullptr;
  int64_t ldy = 0;
  int64_t M = 0, K = 0;
  int splits = 1;
  int64_t kchunk = 0;
  int tiles = 0;
  EpiArgs ep{};
  float* G32_out = nullptr;   // Gram of the updated factor (output of the reduce)
  double* G64_out = nullptr;
  int own = 0;                // factor this half updates: 0 = W, 1 = H
  TcPlan tc{};                // tcgen05 launch plan (tensor-core precisions)
};

struct nmf_ctx {
  nmf_config cfg{};
  const float* V = nullptr;
  float* W = nullptr;
  float* H = nullptr;
  cudaStream_t st = nullptr;
  int64_t p = 0, n = 0;
  int r = 0;
  int sms = 0;
  std::string err = "no error";
  std::vector<void*> allocs;

  // operand copies of V: Xw (p x ld_n) streams the left update, Xh (n x ld_p)
  // the right update; *_hi / *_lo for the bf16 forms, f32 otherwise.
  const void* Xw_hi = nullptr; const void* Xw_lo = nullptr;
  const void* Xh_hi = nullptr; const void* Xh_lo = nullptr;
  int64_t ld_n = 0, ld_p = 0;
  // factor planes: Wop = W^T (r x ld_p), Hop = H (r x ld_n)
  void* Wop_hi = nullptr; void* Wop_lo = nullptr;
  void* Hop_hi = nullptr; void* Hop_lo = nullptr;
  int plane = kPlaneF32;
  int rpad = 0;
  // Grams
  float* GW32 = nullptr; double* GW64 = nullptr;
  float* GH32 = nullptr; double* GH64 = nullptr;
  // per-factor partial Grams ([count][r][r]) left by the last producer of
  // that factor; the matching Gram is their float64 sum.
  float* gpart[2] = {nullptr, nullptr};   // [0] W, [1] H
  int gcount[2] = {0, 0};
  unsigned long long* gctr = nullptr;     // grid-wide counter of the streaming launches
  unsigned long long gunit = 0;           // each launch adds 2 x gunit (>= every grid)
  unsigned long long gctr_skew = 0;       // test hook: added to the next launch's target
  float* GWpad = nullptr; float* GHpad = nullptr;   // rpad x rpad Grams (tensor-core form)
  double* tc_gpart = nullptr;             // tensor-core prologue partials (one per block)
  // objective
  double* obj_parts = nullptr;
  double* f_dev = nullptr;
  double* f_host = nullptr;   // pinned
  int* flag = nullptr;
  int* err_dev = nullptr;     // device error word written by bounded waits
  int* err_host = nullptr;    // pinned
  HalfPlan half[2];           // [0] right update (H), [1] left update (W)
  // CUDA-event timing by kind (nmf_profile_*)
  bool prof = false;
  bool in_step = false;       // inside nmf_step (tensor-core launches timed as a group)
  bool capturing = false;     // recording the convergence graph: no events, no test skew
  // Poisson model: plan and workspaces (k_poisson.cu)
  bool pois = false;
  PoisPlan pplan{};
  double* psums = nullptr;        // 2r: row sums of H, column sums of W
  double* ppartW = nullptr;       // segW x p x r
  double* ppartH = nullptr;       // segH x n x r
  double* pobj_parts = nullptr;   // loglikelihood partials
  PoisTc* ptc = nullptr;          // NMF_BF16X3: the tensor-core passes (k_pois_tc.cu)
  bool ptc_expire = false;        // nmf_test_expire_next_wait on the tensor-core passes
  // nmf_qn_run: the quasi-Newton workspace, made on first use for memory q
  int qn_q = 0;
  float* qn_x[3] = {nullptr, nullptr, nullptr};   // x_n, F(x_n), F(F(x_n))
  float* qn_u = nullptr;              // q x N secant differences u
  float* qn_v = nullptr;              // q x N secant differences v
  double* qn_part = nullptr;          // 3q x chunks inner-product partials
  double* qn_dot = nullptr;           // 3q inner products
  double* qn_coef = nullptr;          // q coefficients
  const float** qn_ptr = nullptr;     // device: 3q + 3q + q operand pointers
  int* qn_neg = nullptr;              // sign flag of the quasi-Newton point
  double* qn_hdot = nullptr;          // pinned mirrors: 3q dots, then q coefficients
  const float** qn_hptr = nullptr;    // pinned: 7q pointers
  int* qn_hneg = nullptr;             // pinned
  // nmf_converge: the run's device state and the graph of its loop, built
  // for one check interval and kept until another is asked for
  RunState* run_dev = nullptr;
  RunState* run_host = nullptr;   // pinned
  cudaStream_t cap_st = nullptr;  // private stream the loop body is captured on
  // nmf_converge_resident: padded factor copies, objective partials, barrier
  float* res_work = nullptr;
  double* res_fpart = nullptr;
  unsigned long long* res_bar = nullptr;
  cudaGraphExec_t conv_exec = nullptr;
  int conv_k = 0;
  std::vector<cudaEvent_t> ev_pool;
  struct Open { int kind; int launches; cudaEvent_t a, b; };
  std::vector<Open> ev_open;
  double prof_ms[4] = {0, 0, 0, 0};
  int64_t prof_n[4] = {0, 0, 0, 0};
};

namespace {

nmf_status cuda_fail(nmf_ctx* c, cudaError_t e, const char* what) {
  set_err(c ? &c->err : nullptr, "%s: %s", what, cudaGetErrorString(e));
  return NMF_ECUDA;
}

#define CK(call, what)                                    \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, what); \
  } while (0)

nmf_status dalloc(nmf_ctx* c, void** p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    set_err(&c->err, "cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
    return NMF_ENOMEM;
  }
  c->allocs.push_back(*p);
  e = cudaMemsetAsync(*p, 0, bytes, c->st);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemsetAsync");
  return NMF_OK;
}

cudaEvent_t take_event(nmf_ctx* c) {
  if (!c->ev_pool.empty()) {
    cudaEvent_t e = c->ev_pool.back();
    c->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) { (void)cudaGetLastError(); return nullptr; }
  return e;
}

// Brackets one region of work of `kind` with events when profiling is on.
// `launches` kernels of that kind run inside the bracket (their mean
// duration is total time / launches).
struct ProfScope {
  nmf_ctx* c;
  int kind;
  int launches;
  cudaEvent_t a = nullptr, b = nullptr;
  ProfScope(nmf_ctx* c_, int k, int n = 1) : c(c_), kind(k), launches(n) {
    if (!c->prof || c->capturing || n <= 0) return;
    a = take_event(c);
    b = take_event(c);
    if (a && b) cudaEventRecord(a, c->st);
  }
  ~ProfScope() {
    if (!c->prof || !a || !b) return;
    cudaEventRecord(b, c->st);
    c->ev_open.push_back({kind, launches, a, b});
  }
};

void prof_collect(nmf_ctx* c) {
  for (auto& it : c->ev_open) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, it.a, it.b) == cudaSuccess) {
      c->prof_ms[it.kind] += ms;
      c->prof_n[it.kind] += it.launches;
    }
    c->ev_pool.push_back(it.a);
    c->ev_pool.push_back(it.b);
  }
  (void)cudaGetLastError();
  c->ev_open.clear();
}

nmf_status validate_cfg(const nmf_config* cfg) {
  if (!cfg) { set_err(nullptr, "cfg is NULL"); return NMF_EINVAL; }
  if (cfg->p < 1 || cfg->n < 1) { set_err(nullptr, "p and n must be >= 1"); return NMF_EINVAL; }
  if (cfg->r < 1 || cfg->r > kMaxRank) {
    set_err(nullptr, "rank r=%d outside 1..%d", cfg->r, kMaxRank);
    return NMF_EINVAL;
  }
  if (cfg->r > cfg->p || cfg->r > cfg->n) {
    set_err(nullptr, "rank r=%d exceeds min(p, n)", cfg->r);
    return NMF_EINVAL;
  }
  if (!(cfg->eps >= 0.f) || isinf(cfg->eps)) { set_err(nullptr, "eps must be finite and >= 0"); return NMF_EINVAL; }
  if (cfg->prec < NMF_FP32 || cfg->prec > NMF_BF16) { set_err(nullptr, "unknown precision"); return NMF_EINVAL; }
  if (cfg->order != NMF_ORDER_H_FIRST && cfg->order != NMF_ORDER_W_FIRST) {
    set_err(nullptr, "unknown order");
    return NMF_EINVAL;
  }
  if (cfg->split_k < 0) { set_err(nullptr, "split_k must be >= 0"); return NMF_EINVAL; }
  if (cfg->model != NMF_MODEL_GAUSSIAN && cfg->model != NMF_MODEL_POISSON) {
    set_err(nullptr, "unknown model");
    return NMF_EINVAL;
  }
  if (cfg->model == NMF_MODEL_POISSON &&
      ((cfg->prec != NMF_FP32 && cfg->prec != NMF_BF16X3) || !pois_supported(cfg->r))) {
    set_err(nullptr, "the Poisson model is served in NMF_FP32 and NMF_BF16X3 for ranks 1..64");
    return NMF_EUNSUPPORTED;
  }
  if (cfg->p > (int64_t)1 << 31 || cfg->n > (int64_t)1 << 31) {
    set_err(nullptr, "p and n must be <= 2^31");
    return NMF_EINVAL;
  }
  return NMF_OK;
}

// Operand copies of V, Algorithm 1's seeded start (optional), the factor
// planes and the starting Gram matrices.  No allocation.
nmf_status prepare(nmf_ctx* c, bool seed_factors, uint64_t seed) {
  const int64_t p = c->p, n = c->n;
  const int r = c->r;
  cudaStream_t st = c->st;
  ProfScope ps(c, 3);
  if (c->pois) {
    if (seed_factors) {
      CK(launch_seed_uniform(c->W, p * r, seed, 1, st), "seed W");
      CK(launch_seed_uniform(c->H, (int64_t)r * n, seed, 2, st), "seed H");
      launched(2);
    }
    if (c->ptc) {
      CK(pois_tc_prepare(c->ptc, c->W, c->H, st), "Poisson factor planes");
      launched(1);
    }
    return NMF_OK;
  }
  {
    // tile-blocked copies: Xw = V (p x n), Xh = V^T (n x p)
    const int mode = c->plane == kPlaneTF32 ? 1 : (c->plane == kPlaneF32 ? 2 : 0);
    const int kbe = mode == 0 ? 64 : 32;
    CK(launch_operand_blocked(c->V, p, n, n, false, mode, (void*)c->Xw_hi, (void*)c->Xw_lo,
                              ceil_div(n, kbe), kbe, st), "operand V");
    CK(launch_operand_blocked(c->V, p, n, n, true, mode, (void*)c->Xh_hi, (void*)c->Xh_lo,
                              ceil_div(p, kbe), kbe, st), "operand V^T");
    launched(2);
  }
  if (seed_factors) {
    CK(launch_seed_uniform(c->W, p * r, seed, 1, st), "seed W");
    CK(launch_seed_uniform(c->H, (int64_t)r * n, seed, 2, st), "seed H");
    launched(2);
  }
  CK(launch_factor_planes(c->W, kFactorRowMajor, p, r, r, c->Wop_hi, c->Wop_lo, c->ld_p,
                          c->plane, st), "W planes");
  CK(launch_factor_planes(c->H, kFactorColMajor, n, n, r, c->Hop_hi, c->Hop_lo, c->ld_n,
                          c->plane, st), "H planes");
  CK(launch_gram_tiles(c->W, kFactorRowMajor, p, r, r, c->gpart[0], 128, st), "gram W");
  c->gcount[0] = (int)ceil_div(p, 128);
  CK(launch_gram_reduce(c->gpart[0], c->gcount[0], r, c->GW32, c->GW64, st), "gram W reduce");
  CK(launch_gram_tiles(c->H, kFactorColMajor, n, n, r, c->gpart[1], 128, st), "gram H");
  c->gcount[1] = (int)ceil_div(n, 128);
  CK(launch_gram_reduce(c->gpart[1], c->gcount[1], r, c->GH32, c->GH64, st), "gram H reduce");
  launched(6);
  return NMF_OK;
}

// The objective value, the error word and the run state (both models).
nmf_status alloc_common(nmf_ctx* c) {
  nmf_status s;
  if ((s = dalloc(c, (void**)&c->f_dev, 8)) != NMF_OK) return s;
  if ((s = dalloc(c, (void**)&c->err_dev, sizeof(int))) != NMF_OK) return s;
  CK(cudaMallocHost((void**)&c->f_host, 8), "cudaMallocHost");
  CK(cudaMallocHost((void**)&c->err_host, sizeof(int)), "cudaMallocHost");
  if ((s = dalloc(c, (void**)&c->run_dev, sizeof(RunState))) != NMF_OK) return s;
  CK(cudaMallocHost((void**)&c->run_host, sizeof(RunState)), "cudaMallocHost");
  return NMF_OK;
}

// Poisson model: V is read as the caller holds it (no operand copies).
nmf_status build_poisson(nmf_ctx* c) {
  const int64_t p = c->p, n = c->n;
  const int r = c->r;
  nmf_status s;
  c->pois = true;
  if (c->cfg.prec == NMF_BF16X3) {
    // the tensor-core form holds its own workspace (blocked V, planes,
    // partials, denominators)
    std::string why;
    c->ptc = pois_tc_create(c->V, p, n, r, c->sms, c->st, &why);
    if (!c->ptc) {
      (void)cudaGetLastError();
      set_err(&c->err, "%s", why.empty() ? "out of host memory" : why.c_str());
      return why.empty() || why.compare(0, 10, "cudaMalloc") == 0 ? NMF_ENOMEM : NMF_ECUDA;
    }
    launched(1);   // the blocked copy of V
  } else {
    c->pplan = pois_plan(p, n, r, c->sms);
    if ((s = dalloc(c, (void**)&c->psums, 2 * (size_t)r * 8)) != NMF_OK) return s;
    if ((s = dalloc(c, (void**)&c->ppartW, (size_t)c->pplan.segW * p * r * 8)) != NMF_OK) return s;
    if ((s = dalloc(c, (void**)&c->ppartH, (size_t)c->pplan.segH * n * r * 8)) != NMF_OK) return s;
  }
  if ((s = dalloc(c, (void**)&c->pobj_parts, (size_t)pois_loglik_parts() * 8)) != NMF_OK) return s;
  if ((s = alloc_common(c)) != NMF_OK) return s;
  return prepare(c, c->cfg.init_from_seed != 0, c->cfg.seed);
}

nmf_status build_ctx(nmf_ctx* c) {
  const int64_t p = c->p, n = c->n;
  const int r = c->r;
  const nmf_precision prec = c->cfg.prec;
  cudaStream_t st = c->st;
  int dev = 0;
  CK(cudaGetDevice(&dev), "cudaGetDevice");
  CK(cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev), "attr");
  {
    int major = 0, minor = 0;
    CK(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev), "attr");
    CK(cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev), "attr");
    if (major != 10 || minor != 3) {
      set_err(&c->err, "the streaming kernels need an sm_103 GPU (found sm_%d%d)", major, minor);
      return NMF_EUNSUPPORTED;
    }
  }
  nmf_status s;
  // Validation of V (optional): one pass.
  if (c->cfg.validate) {
    if ((s = dalloc(c, (void**)&c->flag, sizeof(int))) != NMF_OK) return s;
    CK(launch_validate(c->V, p, n, c->flag, st), "validate");
    launched(1);
    int h = 0;
    CK(cudaMemcpyAsync(&h, c->flag, sizeof(int), cudaMemcpyDeviceToHost, st), "memcpy");
    CK(cudaStreamSynchronize(st), "sync");
    if (h) {
      set_err(&c->err, "V holds a negative or non-finite entry");
      return NMF_ENONFINITE;
    }
  }
  if (c->cfg.model == NMF_MODEL_POISSON) return build_poisson(c);
  // Operand copies of V.
  const bool bf = (prec == NMF_BF16X3 || prec == NMF_BF16);
  const int elem = bf ? 2 : 4;
  const int64_t align_el = 16 / elem;          // 16-byte rows (cp.async / TMA)
  c->ld_n = round_up(n, align_el);
  c->ld_p = round_up(p, align_el);
  c->plane = (prec == NMF_BF16X3) ? kPlaneBF16x2
             : (prec == NMF_BF16) ? kPlaneBF16 : (prec == NMF_TF32 ? kPlaneTF32 : kPlaneF32);
  c->rpad = prec == NMF_FP32 ? rank_pad_f32(r) : rank_pad16(r);
  {
    // tile-blocked copies (128 rows x 128 bytes per block), zero padded
    const int kbe = bf ? 64 : 32;
    const size_t bw = (size_t)ceil_div(p, 128) * ceil_div(n, kbe) * 128 * 128;  // bytes
    const size_t bh = (size_t)ceil_div(n, 128) * ceil_div(p, kbe) * 128 * 128;
    void *a = nullptr, *b = nullptr, *ta = nullptr, *tb = nullptr;
    if ((s = dalloc(c, &a, bw)) != NMF_OK) return s;
    if ((s = dalloc(c, &ta, bh)) != NMF_OK) return s;
    if (prec == NMF_BF16X3) {
      if ((s = dalloc(c, &b, bw)) != NMF_OK) return s;
      if ((s = dalloc(c, &tb, bh)) != NMF_OK) return s;
    }
    c->Xw_hi = a; c->Xw_lo = b; c->Xh_hi = ta; c->Xh_lo = tb;
  }
  // Factor planes (rpad rows; rows >= r stay zero).
  {
    const size_t wbytes = (size_t)c->rpad * c->ld_p * elem;
    const size_t hbytes = (size_t)c->rpad * c->ld_n * elem;
    if ((s = dalloc(c, &c->Wop_hi, wbytes)) != NMF_OK) return s;
    if ((s = dalloc(c, &c->Hop_hi, hbytes)) != NMF_OK) return s;
    if (c->plane == kPlaneBF16x2) {
      if ((s = dalloc(c, &c->Wop_lo, wbytes)) != NMF_OK) return s;
      if ((s = dalloc(c, &c->Hop_lo, hbytes)) != NMF_OK) return s;
    }
  }
  // Grams.
  const size_t rr = (size_t)r * r;
  if ((s = dalloc(c, (void**)&c->GW32, rr * 4)) != NMF_OK) return s;
  if ((s = dalloc(c, (void**)&c->GH32, rr * 4)) != NMF_OK) return s;
  if ((s = dalloc(c, (void**)&c->GW64, rr * 8)) != NMF_OK) return s;
  if ((s = dalloc(c, (void**)&c->GH64, rr * 8)) != NMF_OK) return s;

  // Half-step plans.  [0]: right update (H) streams X = V^T (n x p) against
  // Y = W^T; [1]: left update (W) streams X = V (p x n) against Y = H.
  HalfPlan& hh = c->half[0];
  HalfPlan& hw = c->half[1];
  hh.X_hi = c->Xh_hi; hh.X_lo = c->Xh_lo; hh.ldx = c->ld_p;
  hh.Y_hi = c->Wop_hi; hh.Y_lo = c->Wop_lo; hh.ldy = c->ld_p;
  hh.M = n; hh.K = p;
  hw.X_hi = c->Xw_hi; hw.X_lo = c->Xw_lo; hw.ldx = c->ld_n;
  hw.Y_hi = c->Hop_hi; hw.Y_lo = c->Hop_lo; hw.ldy = c->ld_n;
  hw.M = p; hw.K = n;

  hh.ep.F = c->H; hh.ep.ldf = n; hh.ep.layout = kFactorColMajor; hh.ep.M = n;
  hh.ep.op_hi = c->Hop_hi; hh.ep.op_lo = c->Hop_lo; hh.ep.ldop = c->ld_n;
  hh.G32_out = c->GH32; hh.G64_out = c->GH64; hh.own = 1;
  hw.ep.F = c->W; hw.ep.ldf = r; hw.ep.layout = kFactorRowMajor; hw.ep.M = p;
  hw.ep.op_hi = c->Wop_hi; hw.ep.op_lo = c->Wop_lo; hw.ep.ldop = c->ld_p;
  hw.G32_out = c->GW32; hw.G64_out = c->GW64; hw.own = 0;

  const size_t gtiles[2] = {(size_t)ceil_div(p, 128), (size_t)ceil_div(n, 128)};
  for (HalfPlan* h : {&hh, &hw}) {
    h->ep.r = r;
    h->ep.eps = c->cfg.eps;
    h->ep.plane = c->plane;
    s = tc_plan(c->cfg.prec, h->X_hi, h->X_lo, h->ldx, h->Y_hi, h->Y_lo, h->ldy, h->M, h->K, r,
                c->sms, c->cfg.split_k, &h->tc, &c->err);
    if (s != NMF_OK) return s;
    h->tiles = h->tc.tiles;
    h->splits = h->tc.splits;
    h->kchunk = h->tc.kchunk;
  }
  // partial Grams of the starting factors (and of nmf_read_gram): per 128 rows
  for (int f = 0; f < 2; ++f)
    if ((s = dalloc(c, (void**)&c->gpart[f], gtiles[f] * rr * 4)) != NMF_OK) return s;
  if ((s = dalloc(c, (void**)&c->gctr, sizeof(unsigned long long))) != NMF_OK) return s;
  c->gunit = (unsigned long long)(hh.tc.grid > hw.tc.grid ? hh.tc.grid : hw.tc.grid);
  {
    const size_t rp2 = (size_t)c->rpad * c->rpad;
    if ((s = dalloc(c, (void**)&c->GWpad, rp2 * 4)) != NMF_OK) return s;
    if ((s = dalloc(c, (void**)&c->GHpad, rp2 * 4)) != NMF_OK) return s;
    const size_t grid = (size_t)(hh.tc.grid > hw.tc.grid ? hh.tc.grid : hw.tc.grid);
    if ((s = dalloc(c, (void**)&c->tc_gpart, grid * rr * 8)) != NMF_OK) return s;
  }
  if ((s = dalloc(c, (void**)&c->obj_parts, objective_parts() * 8)) != NMF_OK) return s;
  if ((s = alloc_common(c)) != NMF_OK) return s;
  return prepare(c, c->cfg.init_from_seed != 0, c->cfg.seed);
}

void free_ctx(nmf_ctx* c) {
  if (!c) return;
  if (c->st == nullptr || cudaStreamSynchronize(c->st) != cudaSuccess) (void)cudaDeviceSynchronize();
  for (void* p : c->allocs) cudaFree(p);
  pois_tc_destroy(c->ptc);
  if (c->f_host) cudaFreeHost(c->f_host);
  if (c->err_host) cudaFreeHost(c->err_host);
  if (c->run_host) cudaFreeHost(c->run_host);
  if (c->qn_hdot) cudaFreeHost(c->qn_hdot);
  if (c->qn_hptr) cudaFreeHost((void*)c->qn_hptr);
  if (c->qn_hneg) cudaFreeHost(c->qn_hneg);
  if (c->conv_exec) cudaGraphExecDestroy(c->conv_exec);
  if (c->cap_st) cudaStreamDestroy(c->cap_st);
  for (auto& it : c->ev_open) { cudaEventDestroy(it.a); cudaEventDestroy(it.b); }
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  (void)cudaGetLastError();
  delete c;
}

// Reads the device error word (synchronises).  A bounded device-side wait
// that ran out reports NMF_ETIMEOUT here; the word is then cleared.
nmf_status check_device_error(nmf_ctx* c) {
  CK(cudaMemcpyAsync(c->err_host, c->err_dev, sizeof(int), cudaMemcpyDeviceToHost, c->st),
     "memcpy err");
  CK(cudaStreamSynchronize(c->st), "sync");
  if (*c->err_host != 0) {
    const int code = *c->err_host;
    CK(cudaMemsetAsync(c->err_dev, 0, sizeof(int), c->st), "memset err");
    set_err(&c->err, "a bounded device wait expired (code %d); results are invalid", code);
    return NMF_ETIMEOUT;
  }
  return NMF_OK;
}

nmf_status run_half(nmf_ctx* c, int which) {
  HalfPlan& h = c->half[which];
  const int own = h.own, other = 1 - h.own;
  (void)own;
  {
    // The launch forms the other factor's Gram itself (prologue), then
    // streams V and updates this factor.
    TcGram g;
    g.Q = other == 0 ? c->W : c->H;
    g.q_layout = other == 0 ? 0 : 1;
    g.ldq = other == 0 ? c->r : c->n;
    g.QM = other == 0 ? c->p : c->n;
    g.gpart = c->tc_gpart;
    g.Gpad = other == 0 ? c->GWpad : c->GHpad;
    g.G64 = other == 0 ? c->GW64 : c->GH64;
    g.ctr = c->gctr;
    g.unit = c->gunit;
    // long streams (V of 2^24 entries and more) hide the old rows' loads
    // behind the Gram; short launches overlap them with its first grid step
    g.old_first = c->p * c->n >= (int64_t)1 << 24 ? 1 : 0;
    g.skew = 0;
    if (!c->capturing) {   // skew: only from nmf_test_expire_next_wait
      g.skew = c->gctr_skew;
      c->gctr_skew = 0;
    }
    // timed per nmf_step (events between launches would break the
    // programmatic dependent launch chain); a lone half step times itself
    ProfScope ps(c, 0, c->in_step ? 0 : 1);
    CK(tc_launch(h.tc, h.ep, g, c->err_dev, c->st), "stream (tensor)");
    if (!c->capturing) launched(1);   // graph replays are counted by nmf_converge
  }
  return NMF_OK;
}

// One full iteration of the context's model.
nmf_status run_iteration(nmf_ctx* c) {
  if (c->ptc) {
    // the test hook acts on one directly launched iteration, never on a
    // captured graph
    const int extra = c->ptc_expire && !c->capturing ? 16 : 0;
    if (extra) c->ptc_expire = false;
    CK(pois_tc_iteration(c->ptc, c->W, c->H, c->cfg.eps, c->err_dev, extra, c->st),
       "Poisson iteration (tensor)");
    if (!c->capturing) launched(3);
    return NMF_OK;
  }
  if (c->pois) {
    CK(pois_iteration(c->pplan, c->V, c->n, c->W, c->H, c->p, c->n, c->r, c->cfg.eps, c->psums,
                      c->ppartW, c->ppartH, c->st), "Poisson iteration");
    if (!c->capturing) launched(4);
    return NMF_OK;
  }
  const int first = c->cfg.order == NMF_ORDER_H_FIRST ? 0 : 1;
  nmf_status s = run_half(c, first);
  if (s == NMF_OK) s = run_half(c, 1 - first);
  return s;
}

// The model's objective into f_dev (asynchronous): ||V - WH||_F^2 or L.
cudaError_t launch_model_objective(nmf_ctx* c) {
  if (c->pois)
    return pois_loglik(c->V, c->n, c->W, c->H, c->p, c->n, c->r, c->pobj_parts, c->f_dev, c->st);
  return launch_objective(c->V, c->n, c->W, c->H, c->p, c->n, c->r, c->obj_parts,
                          objective_parts(), c->f_dev, c->st);
}

// Float64 Gram of factor f (0 = W, 1 = H), formed afresh from the factor.
nmf_status reduce_gram(nmf_ctx* c, int f) {
  const int64_t M = f == 0 ? c->p : c->n;
  CK(launch_gram_tiles(f == 0 ? c->W : c->H, f == 0 ? kFactorRowMajor : kFactorColMajor, M,
                       f == 0 ? c->r : c->n, c->r, c->gpart[f], 128, c->st), "gram tiles");
  c->gcount[f] = (int)ceil_div(M, 128);
  CK(launch_gram_reduce(c->gpart[f], c->gcount[f], c->r, f == 0 ? c->GW32 : c->GH32,
                        f == 0 ? c->GW64 : c->GH64, c->st), "gram reduce");
  launched(2);
  return NMF_OK;
}

}  // namespace

extern "C" {

nmf_status nmf_config_default(nmf_config* cfg, int64_t p, int64_t n, int32_t r) {
  if (!cfg) { set_err(nullptr, "cfg is NULL"); return NMF_EINVAL; }
  std::memset(cfg, 0, sizeof *cfg);
  cfg->p = p; cfg->n = n; cfg->r = r;
  cfg->eps = 1e-10f;
  cfg->prec = NMF_FP32;
  cfg->order = NMF_ORDER_H_FIRST;
  return NMF_OK;
}

nmf_status nmf_init(const nmf_config* cfg, const float* V, float* W, float* H, void* stream,
                    nmf_ctx** out) {
  if (!out) { set_err(nullptr, "out is NULL"); return NMF_EINVAL; }
  *out = nullptr;
  nmf_status s = validate_cfg(cfg);
  if (s != NMF_OK) return s;
  if (!V || !W || !H) { set_err(nullptr, "V, W and H must be non-NULL"); return NMF_EINVAL; }
  nmf_ctx* c = new (std::nothrow) nmf_ctx;
  if (!c) { set_err(nullptr, "host allocation failed"); return NMF_ENOMEM; }
  c->cfg = *cfg;
  c->V = V; c->W = W; c->H = H;
  c->st = static_cast<cudaStream_t>(stream);
  c->p = cfg->p; c->n = cfg->n; c->r = cfg->r;
  s = build_ctx(c);
  if (s != NMF_OK) {
    std::string why = c->err;
    free_ctx(c);
    g_last_error = why;
    return s;
  }
  *out = c;
  return NMF_OK;
}

nmf_status nmf_half_step(nmf_ctx* c, int which) {
  if (!c) { set_err(nullptr, "ctx is NULL"); return NMF_EINVAL; }
  if (which != 0 && which != 1) { set_err(&c->err, "which must be 0 (H) or 1 (W)"); return NMF_EINVAL; }
  if (c->pois) { set_err(&c->err, "the Poisson update is simultaneous: no half steps"); return NMF_EUNSUPPORTED; }
  return run_half(c, which);
}

nmf_status nmf_step(nmf_ctx* c, int iters) {
  if (!c) { set_err(nullptr, "ctx is NULL"); return NMF_EINVAL; }
  if (iters < 0) { set_err(&c->err, "iters must be >= 0"); return NMF_EINVAL; }
  // The streaming launches chain by programmatic dependent launch: one
  // bracket (for the Poisson model, one unit per iteration).
  ProfScope ps(c, 0, c->pois ? iters : 2 * iters);
  c->in_step = true;
  nmf_status s = NMF_OK;
  for (int it = 0; it < iters && s == NMF_OK; ++it) s = run_iteration(c);
  c->in_step = false;
  return s;
}

nmf_status nmf_objective(nmf_ctx* c, double* f_out) {
  if (!c || !f_out) { set_err(c ? &c->err : nullptr, "ctx and f_out must be non-NULL"); return NMF_EINVAL; }
  {
    ProfScope ps(c, 2);
    CK(launch_model_objective(c), "objective");
    launched(1);
  }
  CK(cudaMemcpyAsync(c->f_host, c->f_dev, 8, cudaMemcpyDeviceToHost, c->st), "memcpy f");
  nmf_status s = check_device_error(c);
  if (s != NMF_OK) return s;
  *f_out = *c->f_host;
  return NMF_OK;
}

nmf_status nmf_run(nmf_ctx* c, int max_iters, double tol, int check_every, int* iters_done,
                   double* f_out) {
  if (!c) { set_err(nullptr, "ctx is NULL"); return NMF_EINVAL; }
  if (max_iters < 0 || check_every < 1 || !(tol >= 0.0)) {
    set_err(&c->err, "need max_iters >= 0, check_every >= 1, tol >= 0");
    return NMF_EINVAL;
  }
  double f_prev = 0.0, f = 0.0;
  nmf_status s = nmf_objective(c, &f_prev);
  if (s != NMF_OK) return s;
  f = f_prev;
  int done = 0;
  while (done < max_iters) {
    const int k = (max_iters - done) < check_every ? (max_iters - done) : check_every;
    if ((s = nmf_step(c, k)) != NMF_OK) return s;
    done += k;
    if ((s = nmf_objective(c, &f)) != NMF_OK) return s;
    // Section 3's rule: |f_k - f_{k-1}| / (|f_{k-1}| + 1) < tol
    if (tol > 0.0 && std::fabs(f - f_prev) / (std::fabs(f_prev) + 1.0) < tol) break;
    f_prev = f;
  }
  if (iters_done) *iters_done = done;
  if (f_out) *f_out = f;
  return NMF_OK;
}

}  // extern "C"

namespace {

// The loop of nmf_converge as one CUDA graph: a while-node whose body runs
// k iterations (2k streaming launches), the objective and the stopping
// test; the test kernel sets the node's condition, so the whole run to
// convergence is one graph launch with no host round trip.
nmf_status build_conv_graph(nmf_ctx* c, int k) {
  if (c->conv_exec && c->conv_k == k) return NMF_OK;
  if (c->conv_exec) { cudaGraphExecDestroy(c->conv_exec); c->conv_exec = nullptr; }
  if (!c->cap_st) CK(cudaStreamCreateWithFlags(&c->cap_st, cudaStreamNonBlocking), "stream");
  cudaGraph_t g = nullptr;
  CK(cudaGraphCreate(&g, 0), "graph create");
  cudaGraphConditionalHandle loop;
  cudaError_t e = cudaGraphConditionalHandleCreate(&loop, g, 1, cudaGraphCondAssignDefault);
  cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};   // the rest zero
  np.conditional.handle = loop;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node = nullptr;
  if (e == cudaSuccess) e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
  cudaGraph_t body = e == cudaSuccess ? np.conditional.phGraph_out[0] : nullptr;
  if (e == cudaSuccess)
    e = cudaStreamBeginCaptureToGraph(c->cap_st, body, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeRelaxed);
  nmf_status s = NMF_OK;
  if (e == cudaSuccess) {
    cudaStream_t user = c->st;
    c->st = c->cap_st;
    c->capturing = true;
    for (int it = 0; it < k && s == NMF_OK; ++it) s = run_iteration(c);
    cudaError_t le = cudaSuccess;
    if (s == NMF_OK) le = launch_model_objective(c);
    if (s == NMF_OK && le == cudaSuccess) le = launch_run_test(c->run_dev, c->f_dev, k, loop, c->st);
    c->capturing = false;
    c->st = user;
    cudaGraph_t out = nullptr;
    e = cudaStreamEndCapture(c->cap_st, &out);
    if (e == cudaSuccess) e = le;
  }
  if (e == cudaSuccess && s == NMF_OK) e = cudaGraphInstantiate(&c->conv_exec, g, 0);
  cudaGraphDestroy(g);
  if (s != NMF_OK) return s;
  if (e != cudaSuccess) {
    c->conv_exec = nullptr;
    return cuda_fail(c, e, "convergence graph");
  }
  c->conv_k = k;
  return NMF_OK;
}

}  // namespace

extern "C" {

nmf_status nmf_converge(nmf_ctx* c, int max_iters, double tol, int check_every,
                        int* iters_done, double* f_out) {
  if (!c) { set_err(nullptr, "ctx is NULL"); return NMF_EINVAL; }
  if (max_iters < 0 || check_every < 1 || !(tol >= 0.0)) {
    set_err(&c->err, "need max_iters >= 0, check_every >= 1, tol >= 0");
    return NMF_EINVAL;
  }
  nmf_status s = NMF_OK;
  const bool loop = max_iters >= check_every;
  if (loop && (s = build_conv_graph(c, check_every)) != NMF_OK) return s;
  {
    ProfScope ps(c, 2);
    CK(launch_model_objective(c), "objective");
    launched(1);
  }
  CK(launch_run_init(c->run_dev, c->f_dev, max_iters, tol, c->st), "run init");
  launched(1);
  if (loop) CK(cudaGraphLaunch(c->conv_exec, c->st), "graph launch");
  CK(cudaMemcpyAsync(c->run_host, c->run_dev, sizeof(RunState), cudaMemcpyDeviceToHost, c->st),
     "memcpy run state");
  if ((s = check_device_error(c)) != NMF_OK) return s;
  const RunState r = *c->run_host;
  // kernels the graph ran: two (Poisson: four) per iteration, two per test
  launched((c->ptc ? 3 : c->pois ? 4 : 2) * r.done + 2 * r.checks);
  int done = r.done;
  double f = r.f;
  if (!r.stop && done < max_iters) {
    // the remaining iterations, fewer than check_every, and the final objective
    if ((s = nmf_step(c, max_iters - done)) != NMF_OK) return s;
    done = max_iters;
    if ((s = nmf_objective(c, &f)) != NMF_OK) return s;
  }
  if (iters_done) *iters_done = done;
  if (f_out) *f_out = f;
  return NMF_OK;
}

}  // extern "C"

namespace {
nmf_status refresh_planes(nmf_ctx* c);
}  // namespace

extern "C" {

nmf_status nmf_converge_resident(nmf_ctx* c, int max_iters, double tol, int check_every,
                                 int* iters_done, double* f_out) {
  if (!c) { set_err(nullptr, "ctx is NULL"); return NMF_EINVAL; }
  if (max_iters < 0 || check_every < 1 || !(tol >= 0.0)) {
    set_err(&c->err, "need max_iters >= 0, check_every >= 1, tol >= 0");
    return NMF_EINVAL;
  }
  if (c->pois || c->cfg.prec != NMF_FP32) {
    set_err(&c->err, "the resident form runs the Gaussian model in NMF_FP32");
    return NMF_EUNSUPPORTED;
  }
  int dev = 0, optin = 0;
  CK(cudaGetDevice(&dev), "cudaGetDevice");
  CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev), "attribute");
  if (!resident_supported(c->p, c->n, c->r, c->sms, (size_t)optin)) {
    set_err(&c->err, "the resident form needs r <= %d and V's slices and a factor within one "
                     "block's shared memory (p = %lld, n = %lld, r = %d)",
            kResidentMaxRank, (long long)c->p, (long long)c->n, c->r);
    return NMF_EUNSUPPORTED;
  }
  nmf_status s = NMF_OK;
  if (!c->res_work) {
    if ((s = dalloc(c, (void**)&c->res_work,
                    resident_workspace_floats(c->p, c->n, c->r, c->sms) * sizeof(float))) != NMF_OK ||
        (s = dalloc(c, (void**)&c->res_fpart, sizeof(double) * (size_t)c->sms)) != NMF_OK ||
        (s = dalloc(c, (void**)&c->res_bar,
                    kResidentBarWords * sizeof(unsigned long long))) != NMF_OK)
      return s;
  }
  CK(launch_model_objective(c), "objective");
  CK(launch_resident(c->V, c->W, c->H, c->p, c->n, c->r, c->cfg.eps,
                     c->cfg.order == NMF_ORDER_H_FIRST, max_iters, check_every, tol, c->f_dev,
                     c->res_work, c->res_fpart, c->res_bar, c->err_dev, c->run_dev, c->sms,
                     c->st), "resident launch");
  launched(2);
  CK(cudaMemcpyAsync(c->run_host, c->run_dev, sizeof(RunState), cudaMemcpyDeviceToHost, c->st),
     "memcpy run state");
  if ((s = check_device_error(c)) != NMF_OK) return s;
  const RunState r = *c->run_host;
  // the streaming forms' operand planes and Grams from the new factors
  if ((s = refresh_planes(c)) != NMF_OK || (s = reduce_gram(c, 0)) != NMF_OK ||
      (s = reduce_gram(c, 1)) != NMF_OK)
    return s;
  if (iters_done) *iters_done = r.done;
  if (f_out) *f_out = r.f;
  return NMF_OK;
}

}  // extern "C"

namespace {

// The factor operand planes from the factors as they are now (after the
// quasi-Newton loop wrote W and H itself).
nmf_status refresh_planes(nmf_ctx* c) {
  if (c->ptc) {
    CK(pois_tc_prepare(c->ptc, c->W, c->H, c->st), "Poisson factor planes");
    launched(1);
    return NMF_OK;
  }
  if (c->pois) return NMF_OK;
  CK(launch_factor_planes(c->W, kFactorRowMajor, c->p, c->r, c->r, c->Wop_hi, c->Wop_lo,
                          c->ld_p, c->plane, c->st), "W planes");
  CK(launch_factor_planes(c->H, kFactorColMajor, c->n, c->n, c->r, c->Hop_hi, c->Hop_lo,
                          c->ld_n, c->plane, c->st), "H planes");
  launched(2);
  return NMF_OK;
}

// x <- (W, H) and (W, H) <- x, x stacking W (p r entries) then H.
nmf_status save_state(nmf_ctx* c, float* x) {
  const size_t nw = (size_t)c->p * c->r, nh = (size_t)c->r * c->n;
  CK(cudaMemcpyAsync(x, c->W, nw * 4, cudaMemcpyDeviceToDevice, c->st), "copy W");
  CK(cudaMemcpyAsync(x + nw, c->H, nh * 4, cudaMemcpyDeviceToDevice, c->st), "copy H");
  return NMF_OK;
}
nmf_status load_state(nmf_ctx* c, const float* x) {
  const size_t nw = (size_t)c->p * c->r, nh = (size_t)c->r * c->n;
  CK(cudaMemcpyAsync(c->W, x, nw * 4, cudaMemcpyDeviceToDevice, c->st), "copy W");
  CK(cudaMemcpyAsync(c->H, x + nw, nh * 4, cudaMemcpyDeviceToDevice, c->st), "copy H");
  return refresh_planes(c);
}

nmf_status qn_workspace(nmf_ctx* c, int q) {
  if (c->qn_q >= q) return NMF_OK;
  if (c->qn_q != 0) {
    set_err(&c->err, "the quasi-Newton workspace of a context is sized by its first call "
            "(q <= %d)", c->qn_q);
    return NMF_EINVAL;
  }
  const int64_t N = (c->p + c->n) * (int64_t)c->r;
  nmf_status s;
  for (int i = 0; i < 3; ++i)
    if ((s = dalloc(c, (void**)&c->qn_x[i], (size_t)N * 4)) != NMF_OK) return s;
  if ((s = dalloc(c, (void**)&c->qn_u, (size_t)q * N * 4)) != NMF_OK) return s;
  if ((s = dalloc(c, (void**)&c->qn_v, (size_t)q * N * 4)) != NMF_OK) return s;
  if ((s = dalloc(c, (void**)&c->qn_part, (size_t)3 * q * qn_dot_chunks(N) * 8)) != NMF_OK) return s;
  if ((s = dalloc(c, (void**)&c->qn_dot, (size_t)3 * q * 8)) != NMF_OK) return s;
  if ((s = dalloc(c, (void**)&c->qn_coef, (size_t)q * 8)) != NMF_OK) return s;
  if ((s = dalloc(c, (void**)&c->qn_ptr, (size_t)7 * q * sizeof(void*))) != NMF_OK) return s;
  if ((s = dalloc(c, (void**)&c->qn_neg, sizeof(int))) != NMF_OK) return s;
  CK(cudaMallocHost((void**)&c->qn_hdot, (size_t)4 * q * 8), "cudaMallocHost");
  CK(cudaMallocHost((void**)&c->qn_hptr, (size_t)7 * q * sizeof(void*)), "cudaMallocHost");
  CK(cudaMallocHost((void**)&c->qn_hneg, sizeof(int)), "cudaMallocHost");
  c->qn_q = q;
  return NMF_OK;
}

// Solves A c = b (m x m, row-major, float64) by Gaussian elimination with
// partial pivoting; false if a pivot is below 1e-13 of A's largest entry.
bool solve_small(std::vector<double> A, std::vector<double> b, int m, std::vector<double>* x) {
  double amax = 0.0;
  for (double v : A) amax = std::max(amax, std::fabs(v));
  if (!(amax > 0.0) || !std::isfinite(amax)) return false;
  for (int k = 0; k < m; ++k) {
    int piv = k;
    for (int i = k + 1; i < m; ++i)
      if (std::fabs(A[i * m + k]) > std::fabs(A[piv * m + k])) piv = i;
    if (!(std::fabs(A[piv * m + k]) > 1e-13 * amax)) return false;
    if (piv != k) {
      for (int j = 0; j < m; ++j) std::swap(A[k * m + j], A[piv * m + j]);
      std::swap(b[k], b[piv]);
    }
    for (int i = k + 1; i < m; ++i) {
      const double f = A[i * m + k] / A[k * m + k];
      for (int j = k; j < m; ++j) A[i * m + j] -= f * A[k * m + j];
      b[i] -= f * b[k];
    }
  }
  x->assign(m, 0.0);
  for (int i = m - 1; i >= 0; --i) {
    double t = b[i];
    for (int j = i + 1; j < m; ++j) t -= A[i * m + j] * (*x)[j];
    (*x)[i] = t / A[i * m + i];
    if (!std::isfinite((*x)[i])) return false;
  }
  return true;
}

}  // namespace

extern "C" {

nmf_status nmf_qn_run(nmf_ctx* c, int q, int max_iters, double tol, int* iters_done,
                      double* f_out, int* qn_taken) {
  if (!c) { set_err(nullptr, "ctx is NULL"); return NMF_EINVAL; }
  if (q < 1 || q > 32 || max_iters < 0 || !(tol >= 0.0)) {
    set_err(&c->err, "need 1 <= q <= 32, max_iters >= 0, tol >= 0");
    return NMF_EINVAL;
  }
  nmf_status s = qn_workspace(c, q);
  if (s != NMF_OK) return s;
  const int64_t nw = (int64_t)c->p * c->r;
  const int64_t N = nw + (int64_t)c->r * c->n;
  const double sign = c->pois ? -1.0 : 1.0;   // the quantity minimised
  float* X0 = c->qn_x[0];
  float* X1 = c->qn_x[1];
  float* X2 = c->qn_x[2];
  std::vector<double> UU((size_t)q * q, 0.0), UV((size_t)q * q, 0.0);
  double f = 0.0;
  if ((s = nmf_objective(c, &f)) != NMF_OK) return s;
  double g = sign * f;
  int done = 0, taken = 0;
  for (int it = 0; it < max_iters; ++it) {
    // the secant pair of this iterate: x_n, F(x_n), F(F(x_n))
    if ((s = save_state(c, X0)) != NMF_OK) return s;
    if ((s = nmf_step(c, 1)) != NMF_OK) return s;
    if ((s = save_state(c, X1)) != NMF_OK) return s;
    if ((s = nmf_step(c, 1)) != NMF_OK) return s;
    if ((s = save_state(c, X2)) != NMF_OK) return s;
    const int slot = it % q;
    float* us = c->qn_u + (int64_t)slot * N;
    float* vs = c->qn_v + (int64_t)slot * N;
    CK(qn_secant(us, vs, X0, X1, X2, N, c->st), "secant");
    launched(1);
    // inner products of the new pair with the memory (oldest first)
    const int m = it + 1 < q ? it + 1 : q;
    std::vector<int> act(m);
    for (int a = 0; a < m; ++a) act[a] = (it - m + 1 + a) % q;
    const float** hp = c->qn_hptr;
    for (int a = 0; a < m; ++a) {
      const float* uj = c->qn_u + (int64_t)act[a] * N;
      const float* vj = c->qn_v + (int64_t)act[a] * N;
      hp[3 * a + 0] = uj; hp[3 * q + 3 * a + 0] = us;   // <u_j, u_new>
      hp[3 * a + 1] = uj; hp[3 * q + 3 * a + 1] = vs;   // <u_j, v_new>
      hp[3 * a + 2] = us; hp[3 * q + 3 * a + 2] = vj;   // <u_new, v_j>
    }
    CK(cudaMemcpyAsync(c->qn_ptr, hp, (size_t)6 * q * sizeof(void*), cudaMemcpyHostToDevice,
                       c->st), "copy pointers");
    CK(qn_dots(c->qn_ptr, c->qn_ptr + 3 * q, 3 * m, N, c->qn_part, c->qn_dot, c->st), "dots");
    launched(2);
    CK(cudaMemcpyAsync(c->qn_hdot, c->qn_dot, (size_t)3 * m * 8, cudaMemcpyDeviceToHost, c->st),
       "copy dots");
    double f2 = 0.0;   // synchronises: the dots are in qn_hdot too
    if ((s = nmf_objective(c, &f2)) != NMF_OK) return s;
    const double g2 = sign * f2;
    for (int a = 0; a < m; ++a) {
      const int j = act[a];
      UU[(size_t)j * q + slot] = UU[(size_t)slot * q + j] = c->qn_hdot[3 * a + 0];
      UV[(size_t)j * q + slot] = c->qn_hdot[3 * a + 1];
      UV[(size_t)slot * q + j] = c->qn_hdot[3 * a + 2];
    }
    // (U^T U - U^T V) coef = U^T u_new over the active pairs
    std::vector<double> A((size_t)m * m), rhs(m), coef;
    for (int a = 0; a < m; ++a) {
      for (int b = 0; b < m; ++b)
        A[(size_t)a * m + b] = UU[(size_t)act[a] * q + act[b]] - UV[(size_t)act[a] * q + act[b]];
      rhs[a] = UU[(size_t)act[a] * q + slot];
    }
    double gnew = g2;
    if (solve_small(A, rhs, m, &coef)) {
      for (int a = 0; a < m; ++a) c->qn_hdot[3 * q + a] = coef[a];
      const float** hv = c->qn_hptr + 6 * q;
      for (int a = 0; a < m; ++a) hv[a] = c->qn_v + (int64_t)act[a] * N;
      *c->qn_hneg = 0;
      CK(cudaMemcpyAsync(c->qn_coef, c->qn_hdot + 3 * q, (size_t)m * 8, cudaMemcpyHostToDevice,
                         c->st), "copy coefficients");
      CK(cudaMemcpyAsync(c->qn_ptr + 6 * q, hv, (size_t)m * sizeof(void*),
                         cudaMemcpyHostToDevice, c->st), "copy pointers");
      CK(cudaMemsetAsync(c->qn_neg, 0, sizeof(int), c->st), "memset");
      CK(qn_combine(c->W, c->H, nw, N, X1, c->qn_ptr + 6 * q, c->qn_coef, m, c->qn_neg, c->st),
         "combine");
      launched(1);
      CK(cudaMemcpyAsync(c->qn_hneg, c->qn_neg, sizeof(int), cudaMemcpyDeviceToHost, c->st),
         "copy flag");
      CK(cudaStreamSynchronize(c->st), "sync");
      bool take = false;
      if (*c->qn_hneg == 0) {
        if ((s = refresh_planes(c)) != NMF_OK) return s;
        double fq = 0.0;
        if ((s = nmf_objective(c, &fq)) != NMF_OK) return s;
        if (sign * fq <= g2) { take = true; gnew = sign * fq; }
      }
      if (take) ++taken;
      else if ((s = load_state(c, X2)) != NMF_OK) return s;
    }
    ++done;
    const double gprev = g;
    g = gnew;
    if (tol > 0.0 && std::fabs(g - gprev) / (std::fabs(gprev) + 1.0) < tol) break;
  }
  if (iters_done) *iters_done = done;
  if (f_out) *f_out = sign * g;
  if (qn_taken) *qn_taken = taken;
  return check_device_error(c);
}

nmf_status nmf_read_gram(nmf_ctx* c, int which, double* out) {

  if (!c || !out || (which != 0 && which != 1)) {
    set_err(c ? &c->err : nullptr, "bad argument to nmf_read_gram");
    return NMF_EINVAL;
  }
  if (c->pois) { set_err(&c->err, "the Poisson model forms no Gram matrices"); return NMF_EUNSUPPORTED; }
  nmf_status s = reduce_gram(c, which);
  if (s != NMF_OK) return s;
  CK(cudaMemcpyAsync(out, which == 0 ? c->GW64 : c->GH64, (size_t)c->r * c->r * 8,
                     cudaMemcpyDeviceToHost, c->st), "memcpy gram");
  return check_device_error(c);
}

void nmf_destroy(nmf_ctx* c) { free_ctx(c); }

static bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) { (void)cudaGetLastError(); return false; }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

nmf_status nmf_solve(const nmf_config* cfg, const float* V, float* W, float* H, int iters,
                     double* f_out, void* stream) {
  nmf_status s = validate_cfg(cfg);
  if (s != NMF_OK) return s;
  if (!V || !W || !H || iters < 0) { set_err(nullptr, "bad argument to nmf_solve"); return NMF_EINVAL; }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t p = cfg->p, n = cfg->n, r = cfg->r;
  const size_t vb = (size_t)p * n * 4, wb = (size_t)p * r * 4, hb = (size_t)r * n * 4;
  const bool dv = is_device_ptr(V), dw = is_device_ptr(W), dh = is_device_ptr(H);
  float *Vd = const_cast<float*>(V), *Wd = W, *Hd = H;
  std::vector<void*> tmp;
  auto cleanup = [&]() { for (void* q : tmp) cudaFree(q); };
  auto fail = [&](cudaError_t e, const char* what) {
    set_err(nullptr, "%s: %s", what, cudaGetErrorString(e));
    cudaStreamSynchronize(st);
    cleanup();
    return NMF_ECUDA;
  };
  cudaError_t e;
  if (!dv) { if ((e = cudaMalloc((void**)&Vd, vb)) != cudaSuccess) return fail(e, "cudaMalloc V"); tmp.push_back(Vd);
             if ((e = cudaMemcpyAsync(Vd, V, vb, cudaMemcpyHostToDevice, st)) != cudaSuccess) return fail(e, "H2D V"); }
  if (!dw) { if ((e = cudaMalloc((void**)&Wd, wb)) != cudaSuccess) return fail(e, "cudaMalloc W"); tmp.push_back(Wd);
             if ((e = cudaMemcpyAsync(Wd, W, wb, cudaMemcpyHostToDevice, st)) != cudaSuccess) return fail(e, "H2D W"); }
  if (!dh) { if ((e = cudaMalloc((void**)&Hd, hb)) != cudaSuccess) return fail(e, "cudaMalloc H"); tmp.push_back(Hd);
             if ((e = cudaMemcpyAsync(Hd, H, hb, cudaMemcpyHostToDevice, st)) != cudaSuccess) return fail(e, "H2D H"); }
  nmf_ctx* c = nullptr;
  s = nmf_init(cfg, Vd, Wd, Hd, stream, &c);
  if (s == NMF_OK) s = nmf_step(c, iters);
  if (s == NMF_OK && f_out) s = nmf_objective(c, f_out);
  if (s == NMF_OK) {
    if (!dw && (e = cudaMemcpyAsync(W, Wd, wb, cudaMemcpyDeviceToHost, st)) != cudaSuccess) { nmf_destroy(c); return fail(e, "D2H W"); }
    if (!dh && (e = cudaMemcpyAsync(H, Hd, hb, cudaMemcpyDeviceToHost, st)) != cudaSuccess) { nmf_destroy(c); return fail(e, "D2H H"); }
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) { nmf_destroy(c); return fail(e, "sync"); }
  }
  std::string why = c ? c->err : g_last_error;
  if (c) nmf_destroy(c);
  cleanup();
  if (s != NMF_OK) g_last_error = why;
  return s;
}

nmf_status nmf_test_expire_next_wait(nmf_ctx* c) {
  if (!c) { set_err(nullptr, "ctx is NULL"); return NMF_EINVAL; }
  if (c->ptc) {
    c->ptc_expire = true;
    return NMF_OK;
  }
  if (c->pois) { set_err(&c->err, "the NMF_FP32 Poisson kernels have no bounded waits"); return NMF_EUNSUPPORTED; }
  c->gctr_skew = 1ull << 40;   // a counter value no launch reaches
  return NMF_OK;
}

nmf_status nmf_restart(nmf_ctx* c, uint64_t seed) {
  if (!c) { set_err(nullptr, "ctx is NULL"); return NMF_EINVAL; }
  return prepare(c, true, seed);
}

uint64_t nmf_kernel_launches(void) { return g_launches.load(); }

nmf_status nmf_profile_enable(nmf_ctx* c, int on) {
  if (!c) { set_err(nullptr, "ctx is NULL"); return NMF_EINVAL; }
  if (on) {
    CK(cudaStreamSynchronize(c->st), "sync");
    prof_collect(c);
    for (int k = 0; k < 4; ++k) { c->prof_ms[k] = 0; c->prof_n[k] = 0; }
  }
  c->prof = on != 0;
  return NMF_OK;
}

nmf_status nmf_profile_read(nmf_ctx* c, int kind, double* ms, int64_t* count) {
  if (!c || kind < 0 || kind > 3) { set_err(c ? &c->err : nullptr, "bad profile kind"); return NMF_EINVAL; }
  CK(cudaStreamSynchronize(c->st), "sync");
  prof_collect(c);
  if (ms) *ms = c->prof_ms[kind];
  if (count) *count = c->prof_n[kind];
  return NMF_OK;
}

const char* nmf_status_str(nmf_status s) {
  switch (s) {
    case NMF_OK: return "NMF_OK";
    case NMF_EINVAL: return "NMF_EINVAL: invalid argument";
    case NMF_ENOMEM: return "NMF_ENOMEM: out of memory";
    case NMF_ECUDA: return "NMF_ECUDA: CUDA error";
    case NMF_ETIMEOUT: return "NMF_ETIMEOUT: bounded device wait expired";
    case NMF_ENONFINITE: return "NMF_ENONFINITE: V has a negative or non-finite entry";
    case NMF_EUNSUPPORTED: return "NMF_EUNSUPPORTED: not supported by this build/device";
  }
  return "unknown nmf_status";
}

const char* nmf_last_error(const nmf_ctx* c) { return c ? c->err.c_str() : g_last_error.c_str(); }

const char* nmf_version(void) { return "nmf-gb300 0.1 (sm_103a)"; }

}  // extern "C"
