/*
 * A plain C client of libsrt (no Python): builds the plan of the 32^3
 * geometry, runs the forward (Algorithm 1) and the matched adjoint
 * (Algorithm 2) on device buffers, checks the adjoint identity
 * <A f, g> = <f, A^T g> with the library's FP64 device dots, runs the same
 * forward through pipelined host-buffer calls and checks it bitwise against
 * the device result, and checks two error codes.  Prints "OK" and exits 0
 * on success.  Built and run by tests/test_gpu_c_client.py.
 */
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "srt.h"

#define CK(x)                                                               \
  do {                                                                      \
    int s_ = (x);                                                           \
    if (s_) {                                                               \
      fprintf(stderr, "%s failed: %s\n", #x, srt_error_string(s_));         \
      return 1;                                                             \
    }                                                                       \
  } while (0)
#define CC(x)                                                               \
  do {                                                                      \
    cudaError_t e_ = (x);                                                   \
    if (e_ != cudaSuccess) {                                                \
      fprintf(stderr, "%s failed: %s\n", #x, cudaGetErrorString(e_));      \
      return 1;                                                             \
    }                                                                       \
  } while (0)

/* seeded uniform values in [-1, 1) (64-bit LCG, top 24 bits) */
static void fill(float* v, size_t n, uint64_t seed) {
  uint64_t s = seed * 6364136223846793005ull + 1442695040888963407ull;
  for (size_t i = 0; i < n; ++i) {
    s = s * 6364136223846793005ull + 1442695040888963407ull;
    v[i] = (float)((double)(s >> 40) / (double)(1u << 23) - 1.0);
  }
}

static int dot(const float* a, const float* b, int64_t n, void* ws, size_t wsb, double* dd,
               double* out) {
  CK(srt_dot_f64(a, b, n, dd, ws, wsb, NULL));
  CC(cudaMemcpy(out, dd, sizeof(double), cudaMemcpyDeviceToHost));
  return 0;
}

int main(void) {
  srt_geometry g;
  CK(srt_geometry_default(&g, 32, 32, 0.5, 0.5, 12.0, 64, 32, 96));
  srt_plan_t plan = NULL;
  CK(srt_plan(&g, NULL, &plan));
  srt_plan_info_t info;
  CK(srt_plan_info(plan, &info));
  const size_t nf = (size_t)g.ms * g.ms * g.mz, np = (size_t)g.n_phi * g.n_zs * g.n_ell;

  float *hf, *hg, *hp_dev, *hp_pipe;
  CC(cudaMallocHost((void**)&hf, nf * 4));
  CC(cudaMallocHost((void**)&hg, np * 4));
  CC(cudaMallocHost((void**)&hp_dev, np * 4));
  CC(cudaMallocHost((void**)&hp_pipe, np * 4));
  fill(hf, nf, 1);
  fill(hg, np, 2);

  float *f, *gp, *af, *atg;
  CC(cudaMalloc((void**)&f, nf * 4));
  CC(cudaMalloc((void**)&gp, np * 4));
  CC(cudaMalloc((void**)&af, np * 4));
  CC(cudaMalloc((void**)&atg, nf * 4));
  CC(cudaMemcpy(f, hf, nf * 4, cudaMemcpyHostToDevice));
  CC(cudaMemcpy(gp, hg, np * 4, cudaMemcpyHostToDevice));
  size_t wsb = 0;
  CK(srt_workspace_bytes(plan, 1, &wsb));
  void* ws;
  CC(cudaMalloc(&ws, wsb));
  CK(srt_forward(plan, f, af, 1, ws, wsb, NULL));
  CK(srt_adjoint(plan, gp, atg, 1, ws, wsb, NULL));

  const size_t dwsb = srt_dot_workspace_bytes();
  void* dws;
  double* dd;
  CC(cudaMalloc(&dws, dwsb));
  CC(cudaMalloc((void**)&dd, sizeof(double)));
  double lhs, rhs, naf, ng;
  if (dot(af, gp, (int64_t)np, dws, dwsb, dd, &lhs) || dot(f, atg, (int64_t)nf, dws, dwsb, dd, &rhs) ||
      dot(af, af, (int64_t)np, dws, dwsb, dd, &naf) || dot(gp, gp, (int64_t)np, dws, dwsb, dd, &ng))
    return 1;
  const double rel = fabs(lhs - rhs) / sqrt(naf * ng);
  printf("nnz1 %lld nnz2 %lld adjoint identity %.3e\n", (long long)info.nnz1,
         (long long)info.nnz2, rel);
  if (!(rel <= 1e-6) || !(naf > 0)) {
    fprintf(stderr, "adjoint identity %.3e\n", rel);
    return 1;
  }

  /* the same forward through pipelined host-buffer calls: bitwise equal */
  CC(cudaMemcpy(hp_dev, af, np * 4, cudaMemcpyDeviceToHost));
  srt_pipe_t pipe = NULL;
  CK(srt_pipe_create(plan, 1, 2, &pipe));
  int64_t t0 = -1, t1 = -1;
  CK(srt_pipe_submit(pipe, 0, hf, hp_pipe, &t0));
  CK(srt_pipe_submit(pipe, 0, hf, hp_pipe, &t1));
  CK(srt_pipe_wait(pipe, t1, 60.0));
  CK(srt_pipe_wait(pipe, t0, 60.0));
  if (t0 != 0 || t1 != 1 || memcmp(hp_dev, hp_pipe, np * 4) != 0) {
    fprintf(stderr, "pipelined forward differs from the device forward\n");
    return 1;
  }
  CK(srt_pipe_destroy(pipe));

  /* errors come back as codes */
  if (srt_forward(NULL, f, af, 1, ws, wsb, NULL) != SRT_ERR_ARG) return 1;
  if (srt_forward(plan, f, af, 1, ws, 16, NULL) != SRT_ERR_WORKSPACE) return 1;

  cudaFree(dd);
  cudaFree(dws);
  cudaFree(ws);
  cudaFree(f);
  cudaFree(gp);
  cudaFree(af);
  cudaFree(atg);
  cudaFreeHost(hf);
  cudaFreeHost(hg);
  cudaFreeHost(hp_dev);
  cudaFreeHost(hp_pipe);
  CK(srt_plan_destroy(plan));
  printf("OK\n");
  return 0;
}
