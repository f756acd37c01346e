// Sparse-times-dense products of Algorithm 1 (A1 F, A2 Y) and Algorithm 2
// (A2^T Y, A1^T F') of the paper, in gather form: every output row is owned by
// one warp, so no atomics are used and results are deterministic.
//
// y[b][r][n] = sum_{e in row r} A[e] * x[b][col[e]][n],  n < ncols.
// Lanes own consecutive dense columns (float4 when rows are 16-byte aligned);
// a row's (column, value) pairs are loaded 32 at a time and broadcast with
// warp shuffles.  Entries are FP32 or BF16; accumulation is FP32.
#include "common.cuh"

namespace {

constexpr unsigned FULL = 0xffffffffu;

template <typename V>
__device__ __forceinline__ float wval(V v);
template <>
__device__ __forceinline__ float wval<float>(float v) {
  return v;
}
template <>
__device__ __forceinline__ float wval<uint16_t>(uint16_t v) {
  return srt_bf16_to_f32(v);
}

// Vector path: each lane owns 4 consecutive columns of each 128-column chunk;
// a warp covers CH chunks.  Requires ncols, ldx, ldy multiples of 4 and
// 16-byte aligned bases.
// Block-to-rows order.  Rows come in G groups of R rows (r = g*R + i).  With
// G > 0 a block owns a tile of TG groups x 8/TG consecutive i, and
// consecutive blocks take the same chunk of i in consecutive group tiles
// (chunk-major): all groups advance through i together, so the dense rows
// gathered by concurrently running blocks stay within a narrow band of the
// operand (L2 reuse), while a block's 8 warps gather overlapping rows (L1
// reuse).  With G = 0 blocks take consecutive rows.
__device__ __forceinline__ int block_row(int G, int R, int TG) {
  const int w = threadIdx.x >> 5;
  if (G <= 0) return blockIdx.x * (blockDim.x >> 5) + w;
  const int TI = 8 / TG;
  const int chunks = (R + TI - 1) / TI, tiles = (G + TG - 1) / TG;
  const int bid = blockIdx.x;
  const int c = bid / tiles, t = bid - c * tiles;
  if (c >= chunks) return -1;
  const int g = t * TG + w / TI, i = c * TI + w % TI;
  return (g < G && i < R) ? g * R + i : -1;
}

template <typename V, int CH>
__global__ void __launch_bounds__(256) k_spmm_vec(int rows, const int32_t* __restrict__ rowptr,
                                                  const int32_t* __restrict__ col,
                                                  const V* __restrict__ val,
                                                  const float* __restrict__ x, int64_t ldx,
                                                  int64_t bsx, float* __restrict__ y, int64_t ldy,
                                                  int64_t bsy, int ncols, int G, int R, int TG) {
  const int lane = threadIdx.x & 31;
  const int row = block_row(G, R, TG);
  if (row < 0 || row >= rows) return;
  x += blockIdx.z * bsx;
  y += blockIdx.z * bsy;
  const int n0 = blockIdx.y * (128 * CH) + lane * 4;
  float4 acc[CH];
#pragma unroll
  for (int q = 0; q < CH; ++q) acc[q] = make_float4(0.f, 0.f, 0.f, 0.f);
  const int e0 = rowptr[row], e1 = rowptr[row + 1];
  for (int eb = e0; eb < e1; eb += 32) {
    int c = 0;
    float v = 0.f;
    if (eb + lane < e1) {
      c = col[eb + lane];
      v = wval<V>(val[eb + lane]);
    }
    const int cnt = min(32, e1 - eb);
    for (int i = 0; i < cnt; ++i) {
      const int ci = __shfl_sync(FULL, c, i);
      const float vi = __shfl_sync(FULL, v, i);
      const float* xr = x + (int64_t)ci * ldx;
#pragma unroll
      for (int q = 0; q < CH; ++q) {
        const int n = n0 + q * 128;
        if (n < ncols) {
          const float4 xv = __ldg(reinterpret_cast<const float4*>(xr + n));
          acc[q].x = fmaf(vi, xv.x, acc[q].x);
          acc[q].y = fmaf(vi, xv.y, acc[q].y);
          acc[q].z = fmaf(vi, xv.z, acc[q].z);
          acc[q].w = fmaf(vi, xv.w, acc[q].w);
        }
      }
    }
  }
  float* yr = y + (int64_t)row * ldy;
#pragma unroll
  for (int q = 0; q < CH; ++q) {
    const int n = n0 + q * 128;
    if (n < ncols) *reinterpret_cast<float4*>(yr + n) = acc[q];
  }
}

// Scalar path for any ncols / strides: lane owns columns lane + 32 i.
template <typename V, int PER>
__global__ void __launch_bounds__(256) k_spmm_scalar(int rows, const int32_t* __restrict__ rowptr,
                                                     const int32_t* __restrict__ col,
                                                     const V* __restrict__ val,
                                                     const float* __restrict__ x, int64_t ldx,
                                                     int64_t bsx, float* __restrict__ y,
                                                     int64_t ldy, int64_t bsy, int ncols) {
  const int lane = threadIdx.x & 31;
  const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (row >= rows) return;
  x += blockIdx.z * bsx;
  y += blockIdx.z * bsy;
  const int n0 = blockIdx.y * (32 * PER) + lane;
  float acc[PER];
#pragma unroll
  for (int q = 0; q < PER; ++q) acc[q] = 0.f;
  const int e0 = rowptr[row], e1 = rowptr[row + 1];
  for (int eb = e0; eb < e1; eb += 32) {
    int c = 0;
    float v = 0.f;
    if (eb + lane < e1) {
      c = col[eb + lane];
      v = wval<V>(val[eb + lane]);
    }
    const int cnt = min(32, e1 - eb);
    for (int i = 0; i < cnt; ++i) {
      const int ci = __shfl_sync(FULL, c, i);
      const float vi = __shfl_sync(FULL, v, i);
      const float* xr = x + (int64_t)ci * ldx;
#pragma unroll
      for (int q = 0; q < PER; ++q) {
        const int n = n0 + q * 32;
        if (n < ncols) acc[q] = fmaf(vi, __ldg(xr + n), acc[q]);
      }
    }
  }
  float* yr = y + (int64_t)row * ldy;
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int n = n0 + q * 32;
    if (n < ncols) yr[n] = acc[q];
  }
}

template <typename V>
int launch(const SrtCsr& A, const V* val, const float* x, int64_t ldx, int64_t bsx, float* y,
           int64_t ldy, int64_t bsy, int ncols, int batch, int G, int R, int TG, cudaStream_t st) {
  const int rows_per_block = 8;
  dim3 block(256);
  const bool vec = (ncols % 4 == 0) && (ldx % 4 == 0) && (ldy % 4 == 0) && (bsx % 4 == 0) &&
                   (bsy % 4 == 0) && ((uintptr_t)x % 16 == 0) && ((uintptr_t)y % 16 == 0);
  if (G > 0 && (int64_t)G * R != A.rows) G = 0;
  if (TG != 1 && TG != 2 && TG != 4 && TG != 8) TG = 1;
  const int gx = G > 0 ? ((G + TG - 1) / TG) * ((R + 8 / TG - 1) / (8 / TG))
                       : (A.rows + rows_per_block - 1) / rows_per_block;
  if (vec) {
    const int chunks = (ncols + 127) / 128;
    if (chunks >= 4) {
      dim3 grid(gx, (ncols + 511) / 512, batch);
      k_spmm_vec<V, 4><<<grid, block, 0, st>>>(A.rows, A.rowptr, A.col, val, x, ldx, bsx, y, ldy,
                                               bsy, ncols, G, R, TG);
    } else if (chunks == 3) {
      dim3 grid(gx, 1, batch);
      k_spmm_vec<V, 3><<<grid, block, 0, st>>>(A.rows, A.rowptr, A.col, val, x, ldx, bsx, y, ldy,
                                               bsy, ncols, G, R, TG);
    } else if (chunks == 2) {
      dim3 grid(gx, 1, batch);
      k_spmm_vec<V, 2><<<grid, block, 0, st>>>(A.rows, A.rowptr, A.col, val, x, ldx, bsx, y, ldy,
                                               bsy, ncols, G, R, TG);
    } else {
      dim3 grid(gx, 1, batch);
      k_spmm_vec<V, 1><<<grid, block, 0, st>>>(A.rows, A.rowptr, A.col, val, x, ldx, bsx, y, ldy,
                                               bsy, ncols, G, R, TG);
    }
  } else {
    dim3 grid((A.rows + rows_per_block - 1) / rows_per_block, (ncols + 127) / 128, batch);
    k_spmm_scalar<V, 4><<<grid, block, 0, st>>>(A.rows, A.rowptr, A.col, val, x, ldx, bsx, y, ldy,
                                                bsy, ncols);
  }
  SRT_CUDA_TRY(cudaGetLastError());
  return SRT_OK;
}


}  // namespace

int srt_spmm(const SrtCsr& A, int wdt, const float* x, int64_t ldx, int64_t bsx, float* y,
             int64_t ldy, int64_t bsy, int ncols, int batch, cudaStream_t st, int G, int R,
             int TG) {
  if (wdt == SRT_BF16)
    return launch<uint16_t>(A, A.v16, x, ldx, bsx, y, ldy, bsy, ncols, batch, G, R, TG, st);
  return launch<float>(A, A.v32, x, ldx, bsx, y, ldy, bsy, ncols, batch, G, R, TG, st);
}

