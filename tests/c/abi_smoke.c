/* A C99 program that uses libnmf.so through include/nmf.h alone: seeded
 * start, ten MM iterations of a small problem in the split-BF16x3 form, the
 * objective before and after (the MM descent property, Section 3.1), the
 * error path of a bad argument, then cleanup; then a tiny penalised PET
 * reconstruction through include/pet.h (Section 3.2: the penalised
 * loglikelihood rises).  Exit status 0 on success. */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime_api.h>

#include "nmf.h"
#include "pet.h"

#define CHECK(x)                                                        \
  do {                                                                  \
    if (!(x)) {                                                         \
      fprintf(stderr, "check failed at line %d: %s\n", __LINE__, #x);   \
      return 1;                                                         \
    }                                                                   \
  } while (0)

int main(void) {
  const int64_t p = 300, n = 500;
  const int32_t r = 12;
  float *hV = (float*)malloc(sizeof(float) * p * n);
  CHECK(hV != NULL);
  for (int64_t i = 0; i < p * n; ++i) hV[i] = (float)((i * 2654435761u) % 1000u) / 1000.0f;
  float *V = NULL, *W = NULL, *H = NULL;
  CHECK(cudaMalloc((void**)&V, sizeof(float) * p * n) == cudaSuccess);
  CHECK(cudaMalloc((void**)&W, sizeof(float) * p * r) == cudaSuccess);
  CHECK(cudaMalloc((void**)&H, sizeof(float) * r * n) == cudaSuccess);
  CHECK(cudaMemcpy(V, hV, sizeof(float) * p * n, cudaMemcpyHostToDevice) == cudaSuccess);

  nmf_config cfg;
  CHECK(nmf_config_default(&cfg, p, n, r) == NMF_OK);
  cfg.prec = NMF_BF16X3;
  cfg.seed = 7;
  cfg.init_from_seed = 1;              /* W, H iid uniform(0,1) from the seed */
  nmf_ctx* ctx = NULL;
  CHECK(nmf_init(&cfg, V, W, H, NULL, &ctx) == NMF_OK && ctx != NULL);

  double f0 = 0.0, f1 = 0.0;
  CHECK(nmf_objective(ctx, &f0) == NMF_OK);
  CHECK(nmf_step(ctx, 10) == NMF_OK);
  CHECK(nmf_objective(ctx, &f1) == NMF_OK);
  printf("f0 = %.9g  f10 = %.9g\n", f0, f1);
  CHECK(isfinite(f0) && isfinite(f1) && f1 > 0.0 && f1 < f0);

  /* errors come back as codes, with a reason */
  CHECK(nmf_step(NULL, 1) == NMF_EINVAL);
  CHECK(nmf_last_error(NULL)[0] != '\0');

  nmf_destroy(ctx);
  cudaFree(V);
  cudaFree(W);
  cudaFree(H);
  free(hV);

  /* PET: 4 lines through 3 pixels in a row, neighbours 0-1-2 */
  {
    const float hE[12] = {1.0f, 0.5f, 0.0f, 0.0f, 1.0f, 1.0f, 0.3f, 0.3f, 0.3f, 1.0f, 0.0f, 2.0f};
    const float hy[4] = {4.0f, 7.0f, 2.0f, 0.0f};
    const int32_t ptr[4] = {0, 1, 3, 4}, idx[4] = {1, 0, 2, 1};
    const double mu[2] = {0.0, 0.1};
    float *E = NULL, *y = NULL, *lam = NULL;
    CHECK(cudaMalloc((void**)&E, sizeof hE) == cudaSuccess);
    CHECK(cudaMalloc((void**)&y, sizeof hy) == cudaSuccess);
    CHECK(cudaMalloc((void**)&lam, 2 * 3 * sizeof(float)) == cudaSuccess);
    CHECK(cudaMemcpy(E, hE, sizeof hE, cudaMemcpyHostToDevice) == cudaSuccess);
    CHECK(cudaMemcpy(y, hy, sizeof hy, cudaMemcpyHostToDevice) == cudaSuccess);
    pet_ctx* pc = NULL;
    CHECK(pet_init(4, 3, E, y, ptr, idx, 2, mu, lam, 1, NULL, &pc) == NMF_OK && pc != NULL);
    double g0[2], g1[2];
    CHECK(pet_objective(pc, g0) == NMF_OK);
    CHECK(pet_step(pc, 20) == NMF_OK);
    CHECK(pet_objective(pc, g1) == NMF_OK);
    printf("pet f0 = %.9g %.9g  f20 = %.9g %.9g\n", g0[0], g0[1], g1[0], g1[1]);
    CHECK(g1[0] > g0[0] && g1[1] > g0[1]);
    CHECK(pet_step(NULL, 1) == NMF_EINVAL && pet_last_error(NULL)[0] != '\0');
    pet_destroy(pc);
    cudaFree(E);
    cudaFree(y);
    cudaFree(lam);
  }
  printf("ok %s\n", nmf_version());
  return 0;
}
