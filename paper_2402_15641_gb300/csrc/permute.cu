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

// 64 x 64 tiles with 16-byte global accesses on both sides: each of the 256
// threads moves 16 elements, so a block keeps 16 KB of loads in flight.
// Requires rows, cols, ild, old, ibs, obs multiples of 4 and 16-byte aligned
// bases.  Shared tile padded to 65 columns (at most 2-way bank conflicts).
constexpr int VT = 64;
__global__ void __launch_bounds__(256) k_transpose_v4(const float* __restrict__ in, int64_t ild,
                                                      int64_t ibs, float* __restrict__ out,
                                                      int64_t old, int64_t obs, int rows,
                                                      int cols) {
  __shared__ float tile[VT][VT + 1];
  in += blockIdx.z * ibs;
  out += blockIdx.z * obs;
  const int c0 = blockIdx.x * VT, r0 = blockIdx.y * VT;
  const int t = threadIdx.x;
  const int q = t & 15, rr = t >> 4;  // float4 column within a row, row within 16
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int i = rr + 16 * k;  // tile row
    const int r = r0 + i, c = c0 + 4 * q;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (r < rows && c < cols) v = __ldg(reinterpret_cast<const float4*>(in + (int64_t)r * ild + c));
    tile[i][4 * q] = v.x;
    tile[i][4 * q + 1] = v.y;
    tile[i][4 * q + 2] = v.z;
    tile[i][4 * q + 3] = v.w;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int j = rr + 16 * k;  // tile column = output row
    const int c = c0 + j, r = r0 + 4 * q;
    if (c < cols && r < rows) {
      const float4 v = make_float4(tile[4 * q][j], tile[4 * q + 1][j], tile[4 * q + 2][j],
                                   tile[4 * q + 3][j]);
      *reinterpret_cast<float4*>(out + (int64_t)c * old + r) = v;
    }
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
  const bool v4 = rows % 4 == 0 && cols % 4 == 0 && ild % 4 == 0 && old % 4 == 0 && ibs % 4 == 0 &&
                  obs % 4 == 0 && (uintptr_t)in % 16 == 0 && (uintptr_t)out % 16 == 0;
  if (v4) {
    dim3 grid((cols + VT - 1) / VT, (rows + VT - 1) / VT, batch);
    if (grid.y > 65535 || grid.z > 65535) return SRT_ERR_ARG;
    k_transpose_v4<<<grid, 256, 0, st>>>(in, ild, ibs, out, old, obs, rows, cols);
    SRT_CUDA_TRY(cudaGetLastError());
    return SRT_OK;
  }
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
