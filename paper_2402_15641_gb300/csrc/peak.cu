// Measurement helper with no counterpart in the paper: the FP32 FMA rate the
// CUDA cores sustain on this GPU, the arithmetic roof of the sparse products.
// Each thread runs 16 independent FMA chains (enough to cover the FMA
// latency), on 8 blocks of 256 threads per SM.
#include "common.cuh"

namespace {

__device__ float g_fma_sink;

__global__ void __launch_bounds__(256) k_fma_peak(int iters, float a, float b) {
  float x[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) x[i] = threadIdx.x * 1e-3f + i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 16; ++i) x[i] = fmaf(x[i], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < 16; ++i) s += x[i];
  if (s == -1.0f) g_fma_sink = s;  // never true: keeps the chains live
}

}  // namespace

extern "C" int srt_fp32_fma_peak(int32_t iters, double* tflops, void* stream) {
  if (!tflops || iters <= 0) return SRT_ERR_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  SRT_CUDA_TRY(cudaGetDevice(&dev));
  SRT_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * 8, threads = 256;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  SRT_CUDA_TRY(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return SRT_ERR_CUDA;
  }
  k_fma_peak<<<blocks, threads, 0, st>>>(iters, 0.999f, 0.001f);  // warm-up
  cudaEventRecord(e0, st);
  k_fma_peak<<<blocks, threads, 0, st>>>(iters, 0.999f, 0.001f);
  cudaEventRecord(e1, st);
  cudaError_t err = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
  if (err == cudaSuccess) err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess || ms <= 0.f) return SRT_ERR_CUDA;
  const double flop = 2.0 * blocks * threads * (double)iters * 16.0;
  *tflops = flop / (ms * 1e-3) / 1e12;
  return SRT_OK;
}
