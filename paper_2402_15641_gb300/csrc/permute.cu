// Reshapes between the stages of Algorithms 1 and 2 of the paper, and the
// FP64 inner product used for adjoint-identity checks.
//
// The reshapes are batched 2-D transposes through a padded shared-memory
// tile: out[b*obs + c*old + r] = in[b*ibs + r*ild + c].
#include "common.cuh"

namespace {

constexpr int TILE = 32;

__global__ void __launch_bounds__(256) k_transpose(const float* __restrict__ in, int64_t ild,
                                                   int64_t ibs, float* __restrict__ out,
                                                   int64_t old, int64_t obs, int rows, int cols) {
  __shared__ float tile[TILE][TILE + 1];
  in += blockIdx.z * ibs;
  out += blockIdx.z * obs;
  const int c0 = blockIdx.x * TILE, r0 = blockIdx.y * TILE;
  const int tx = threadIdx.x, ty = threadIdx.y;
#pragma unroll
  for (int i = ty; i < TILE; i += 8) {
    const int r = r0 + i, c = c0 + tx;
    if (r < rows && c < cols) tile[i][tx] = in[(int64_t)r * ild + c];
  }
  __syncthreads();
#pragma unroll
  for (int i = ty; i < TILE; i += 8) {
    const int c = c0 + i, r = r0 + tx;
    if (r < rows && c < cols) out[(int64_t)c * old + r] = tile[tx][i];
  }
}

// Partial FP64 sums, one per block, in a fixed order.
__global__ void __launch_bounds__(256) k_dot_partial(const float* __restrict__ a,
                                                     const float* __restrict__ b, int64_t n,
                                                     double* __restrict__ part) {
  __shared__ double ws[8];
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    s = fma((double)a[i], (double)b[i], s);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += ws[w];
    part[blockIdx.x] = t;
  }
}

__global__ void k_dot_final(const double* __restrict__ part, int n, double* __restrict__ out) {
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < n; ++i) t += part[i];
    *out = t;
  }
}

}  // namespace

int srt_transpose(const float* in, int64_t ild, int64_t ibs, float* out, int64_t old, int64_t obs,
                  int rows, int cols, int batch, cudaStream_t st) {
  dim3 block(TILE, 8);
  dim3 grid((cols + TILE - 1) / TILE, (rows + TILE - 1) / TILE, batch);
  if (grid.y > 65535 || grid.z > 65535) return SRT_ERR_ARG;
  k_transpose<<<grid, block, 0, st>>>(in, ild, ibs, out, old, obs, rows, cols);
  SRT_CUDA_TRY(cudaGetLastError());
  return SRT_OK;
}

int srt_dot(const float* a, const float* b, int64_t n, double* out, double* partials,
            cudaStream_t st) {
  k_dot_partial<<<SRT_DOT_BLOCKS, 256, 0, st>>>(a, b, n, partials);
  SRT_CUDA_TRY(cudaGetLastError());
  k_dot_final<<<1, 32, 0, st>>>(partials, SRT_DOT_BLOCKS, out);
  SRT_CUDA_TRY(cudaGetLastError());
  return SRT_OK;
}
