/* A C99 program that uses libnmf.so through include/nmf.h alone: seeded
 * start, ten MM iterations of a small problem in the split-BF16x3 form, the
 * objective before and after (the MM descent property, Section 3.1), the
 * error path of a bad argument, then cleanup.  Exit status 0 on success. */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime_api.h>

#include "nmf.h"

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
  printf("ok %s\n", nmf_version());
  return 0;
}
