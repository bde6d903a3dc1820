// tcgen05 (5th-generation tensor core) form of the V-streaming products:
// plan (tensor maps, tiling, split-K) and launch.  Implemented in k_stream_tc.cu.
#pragma once

#include <cuda.h>
#include <string>

#include "nmf_internal.cuh"

namespace nmf {

struct TcPlan {
  int prec = 0;          // nmf_precision
  int block_m = 128;     // rows of X per output tile (tcgen05 M)
  int rpad = 16;         // accumulator columns (tcgen05 N), multiple of 16
  int tiles = 0;
  int splits = 1;
  int64_t kchunk = 0;    // K per split, multiple of the k-block
  int kblock = 64;       // K elements per pipeline stage
  int64_t M = 0, K = 0;
  int r = 0;
  int grid = 0;
  int smem = 0;
  int S = 1;             // cluster size (K-splits per tile)
  int threads = 256;     // block size of the kernel instance
  int nkbt = 0;          // k-blocks per tile row of the blocked X copy
  int nclusters = 0;     // persistent clusters
  int nacc = 1;          // tensor-memory accumulators the main products rotate over
  int tmem_cols = 32;    // tensor-memory columns the kernel allocates
  void* fn = nullptr;    // kernel instance
  CUtensorMap x_hi, x_lo, y_hi, y_lo;
};

// The other factor Q, whose Gram the launch forms itself (prologue), and
// the grid-wide counter that orders the prologue's two phases.
struct TcGram {
  const float* Q;                // W (p x r, layout 0) or H (r x n, layout 1)
  int q_layout;
  int64_t ldq;
  int64_t QM;                    // rows of Q
  double* gpart;                 // workspace, grid * r * r doubles
  float* Gpad;                   // out: rpad x rpad float32 (zero padded)
  double* G64;                   // out: r x r float64
  unsigned long long* ctr;       // monotone counter, starts at 0
  unsigned long long unit;       // every launch adds 2 x unit; unit >= grid of every
                                 // launch on this counter (fixed for its lifetime)
  unsigned long long skew;       // added to the wait targets: 0 (test hook)
  int old_first;                 // 1: load the first tile's old rows before the Gram
                                 // (long launches), 0: during its first grid-wide step
};

nmf_status tc_plan(int prec, const void* X_hi, const void* X_lo, int64_t ldx, const void* Y_hi,
                   const void* Y_lo, int64_t ldy, int64_t M, int64_t K, int r, int sms,
                   int user_split, TcPlan* plan, std::string* err);

cudaError_t tc_launch(const TcPlan& plan, const EpiArgs& ep, const TcGram& gram, int* err,
                      cudaStream_t st);

// The float32 FMA form of the same half step (k_stream_f32.cu).
bool f32_kernel_for(int rpad, void** fn, int* smem, int* threads);
bool f32_regs_ok(void* fn);   // built with the register count its split assumes
cudaError_t f32_launch(const TcPlan& plan, const EpiArgs& ep, const TcGram& gram, int* err,
                       cudaStream_t st);

}  // namespace nmf
