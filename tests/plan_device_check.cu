// A plan used with another device current is refused before any work.
// Built with nvcc against the library's internal header (for the plan's
// device field) and linked to libsrt.so by tests/test_gpu_device_check.py.
// It builds a small plan on the current GPU, then marks the plan as made on
// device index (current + 1), which is not current: every call that would
// launch work must return SRT_ERR_ARG without launching anything.  It then
// restores the field and checks that the same calls succeed.  Prints "OK".
#include <cstdio>
#include <vector>

#include "common.cuh"

#define EXPECT(cond)                                         \
  do {                                                       \
    if (!(cond)) {                                           \
      std::fprintf(stderr, "failed: %s (line %d)\n", #cond, __LINE__); \
      return 1;                                              \
    }                                                        \
  } while (0)

int main() {
  srt_geometry g;
  EXPECT(srt_geometry_default(&g, 8, 6, 0.5, 0.5, 6.0, 8, 6, 16) == SRT_OK);
  srt_plan_t plan = nullptr;
  EXPECT(srt_plan(&g, nullptr, &plan) == SRT_OK);
  const size_t nf = 8 * 8 * 6, np = 8 * 6 * 16;
  size_t wsb = 0, hwsb = 0;
  EXPECT(srt_workspace_bytes(plan, 1, &wsb) == SRT_OK);
  EXPECT(srt_host_workspace_bytes(plan, 1, &hwsb) == SRT_OK);
  float *f = nullptr, *p = nullptr;
  void *ws = nullptr, *hws = nullptr;
  EXPECT(cudaMalloc(&f, nf * 4) == cudaSuccess && cudaMalloc(&p, np * 4) == cudaSuccess);
  EXPECT(cudaMalloc(&ws, wsb) == cudaSuccess && cudaMalloc(&hws, hwsb) == cudaSuccess);
  EXPECT(cudaMemset(f, 0, nf * 4) == cudaSuccess && cudaMemset(p, 0, np * 4) == cudaSuccess);
  std::vector<float> fh(nf, 1.0f), ph(np, 0.0f);
  srt_pipe_t pipe = nullptr;
  EXPECT(srt_pipe_create(plan, 1, 2, &pipe) == SRT_OK);

  const int dev = plan->device;
  plan->device = dev + 1;  // a device index that is not the current one
  EXPECT(srt_forward(plan, f, p, 1, ws, wsb, nullptr) == SRT_ERR_ARG);
  EXPECT(srt_adjoint(plan, p, f, 1, ws, wsb, nullptr) == SRT_ERR_ARG);
  EXPECT(srt_forward_host(plan, fh.data(), ph.data(), 1, hws, hwsb, nullptr) == SRT_ERR_ARG);
  EXPECT(srt_adjoint_host(plan, ph.data(), fh.data(), 1, hws, hwsb, nullptr) == SRT_ERR_ARG);
  EXPECT(srt_forward_noalloc(plan, f, p, 1, nullptr) == SRT_ERR_ARG);
  EXPECT(srt_adjoint_noalloc(plan, p, f, 1, nullptr) == SRT_ERR_ARG);
  srt_pipe_t pipe2 = nullptr;
  EXPECT(srt_pipe_create(plan, 1, 2, &pipe2) == SRT_ERR_ARG && pipe2 == nullptr);
  int64_t ticket = -1;
  EXPECT(srt_pipe_submit(pipe, 0, fh.data(), ph.data(), &ticket) == SRT_ERR_ARG);
  EXPECT(cudaDeviceSynchronize() == cudaSuccess);

  plan->device = dev;
  EXPECT(srt_forward(plan, f, p, 1, ws, wsb, nullptr) == SRT_OK);
  EXPECT(srt_adjoint(plan, p, f, 1, ws, wsb, nullptr) == SRT_OK);
  EXPECT(srt_forward_host(plan, fh.data(), ph.data(), 1, hws, hwsb, nullptr) == SRT_OK);
  EXPECT(srt_pipe_submit(pipe, 0, fh.data(), ph.data(), &ticket) == SRT_OK && ticket == 0);
  EXPECT(srt_pipe_wait(pipe, ticket, 30.0) == SRT_OK);
  EXPECT(cudaDeviceSynchronize() == cudaSuccess);
  srt_pipe_destroy(pipe);
  srt_plan_destroy(plan);
  cudaFree(f);
  cudaFree(p);
  cudaFree(ws);
  cudaFree(hws);
  std::printf("OK\n");
  return 0;
}
