// Device-memory helpers for the plan-building code (not used on the
// forward/adjoint path, which allocates nothing).
#pragma once

#include "common.cuh"

// cudaMalloc of n elements; adds the bytes to *bytes when given.
template <class T>
inline int srt_dmalloc(T** p, int64_t n, int64_t* bytes) {
  *p = nullptr;
  if (n <= 0) n = 1;
  cudaError_t e = cudaMalloc((void**)p, (size_t)n * sizeof(T));
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return SRT_ERR_OOM;
  }
  if (e != cudaSuccess) return SRT_ERR_CUDA;
  if (bytes) *bytes += n * (int64_t)sizeof(T);
  return SRT_OK;
}

// Temporaries released on every exit path of a build step.
struct SrtTmp {
  void* p[16] = {};
  int n = 0;
  SrtTmp() = default;
  SrtTmp(const SrtTmp&) = delete;
  SrtTmp& operator=(const SrtTmp&) = delete;
  ~SrtTmp() {
    for (int i = 0; i < n; ++i) cudaFree(p[i]);
  }
  template <class T>
  int get(T** out, int64_t count) {
    if (n >= 16) return SRT_ERR_ARG;
    int s = srt_dmalloc(out, count, nullptr);
    if (s == SRT_OK) p[n++] = *out;
    return s;
  }
};

// Exclusive scan of n int32 counts into out[0..n]; *total gets the exact sum.
int srt_scan_counts(const int32_t* counts, int32_t* out, int64_t n, long long* dtotal,
                    int64_t* total, cudaStream_t st);

// Deterministic CSR transpose of a rows x cols pattern: output rows list
// their entries by increasing source row; values/payloads (each optional)
// are copied bitwise.  Output arrays are allocated by the caller.
int srt_csr_transpose(int rows, int cols, int64_t nnz, const int32_t* rowptr, const int32_t* col,
                      const float* v32, const uint16_t* v16, const double* v64,
                      const int32_t* pay, int32_t* trowptr, int32_t* tcol, float* t32,
                      uint16_t* t16, double* t64, int32_t* tpay, cudaStream_t st);
