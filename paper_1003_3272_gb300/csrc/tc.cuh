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
  int nkbt = 0;          // k-blocks per tile row of the blocked X copy
  int nclusters = 0;     // persistent clusters
  void* fn = nullptr;    // kernel instance
  CUtensorMap x_hi, x_lo, y_hi, y_lo;
};

// The other factor's Gram, reduced inside the launch from per-slice partials.
struct TcGram {
  const float* gin;              // partials [gin_count][r][r]
  int gin_count;
  float* G32;                    // r x r, float32 (used by the epilogue)
  double* G64;                   // r x r, float64
  unsigned long long* ctr;       // grid-wide publication counter
  unsigned long long target;     // counter value once every block published
};

// X_hi / X_lo: tile-blocked operand copies (blocks of 128 rows x 128 bytes,
// block (tile, kb) at index tile * ceil(K / kblock) + kb); Y: K-major planes
// with row pitch ldy.
nmf_status tc_plan(int prec, const void* X_hi, const void* X_lo, int64_t ldx, const void* Y_hi,
                   const void* Y_lo, int64_t ldy, int64_t M, int64_t K, int r, int sms,
                   int user_split, TcPlan* plan, std::string* err);

cudaError_t tc_launch(const TcPlan& plan, const EpiArgs& ep, const TcGram& gram, int* err,
                      cudaStream_t st);

}  // namespace nmf
