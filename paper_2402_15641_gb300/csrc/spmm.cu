// Sparse-times-dense products of Algorithm 1 (A1 F, A2 Y) and Algorithm 2
// (A2^T Y, A1^T F') of the paper, in gather form: every output row is owned by
// one warp, so no atomics are used and results are deterministic.
//
// y[b][r][n] = sum_{e in row r} A[e] * x[b][col[e]][n],  n < ncols.
// Lanes own consecutive dense columns (float4 when rows are 16-byte aligned);
// a row's (column, value) pairs are loaded 32 at a time and broadcast with
// warp shuffles.  Entries are FP32 or BF16; accumulation is FP32.
//
// A1 by rotation (SrtRot): with n_phi a multiple of 4, sensor column
// j + n_phi/4 sees the image turned by 90 degrees about the axis, so
//   A1[(j + s n_phi/4, l), rot^s(p)] = A1[(j, l), p],
//   rot(ix, iy) = (ms-1-iy, ix),
// and only the rows of the first n_phi/4 columns are stored.  Mode 1 (A1):
// output row (j, l) walks stored row (j mod n_phi/4, l) and gathers pixel
// rot^s(p).  Mode 2 (A1^T): output row p walks, for s = 0..3, stored row
// rot^-s(p) of the stored transpose and gathers row (j + s n_phi/4, l): the
// same terms in the same order (ascending j, then l) as the full transpose.
#include <type_traits>

#include "common.cuh"

namespace {

constexpr unsigned FULL = 0xffffffffu;
#ifdef SRT_CHECKS
__device__ unsigned long long g_viol;  // gathered rows outside their operand
#endif

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

// Pixel p = ix*ms + iy turned s quarter turns: rot(ix, iy) = (ms-1-iy, ix).
// ix = floor(p / ms) as (p * magic) >> 40 with magic = ceil(2^40 / ms), exact
// for p < 2^24 and ms < 2^16 (the quotient's error stays below 1/ms).
__device__ __forceinline__ int rot_pixel(int p, int s, int ms, uint64_t magic, bool m = false) {
  int ix = (int)(((uint64_t)(uint32_t)p * magic) >> 40), iy = p - ix * ms;
  if (m) {  // mirror across the diagonal first: (ix, iy) -> (iy, ix)
    const int t = ix;
    ix = iy;
    iy = t;
    p = ix * ms + iy;
  }
  switch (s & 3) {
    case 0: return p;
    case 1: return (ms - 1 - iy) * ms + ix;
    case 2: return (ms - 1 - ix) * ms + (ms - 1 - iy);
    default: return iy * ms + (ms - 1 - ix);
  }
}

// Block-to-rows order.  Rows come in G groups of R rows (r = g*R + i).  With
// G > 0 a block owns a tile of TG groups x 8/TG consecutive i, and
// consecutive blocks take the same chunk of i in consecutive group tiles
// (chunk-major): all groups advance through i together, so the dense rows
// gathered by concurrently running blocks stay within a narrow band of the
// operand (L2 reuse), while a block's 8 warps gather overlapping rows (L1
// reuse).  With G = 0 blocks take consecutive rows.  With S > 0 the G x R
// grid is walked in S x S super-tiles (S dividing G and R), tiles row-major
// inside each: the dense rows gathered by concurrently running blocks then
// belong to a compact patch instead of a band across all G groups (A1^T:
// pixels, whose circles through a 64 x 64 patch cover ~40% of the operand
// instead of most of it).
__device__ __forceinline__ int block_row(int G, int R, int TG, int S) {
  const int w = threadIdx.x >> 5;
  if (G <= 0) return blockIdx.x * (blockDim.x >> 5) + w;
  const int TI = 8 / TG;
  if (S > 0) {
    const int per_row = S / TG, bpt = per_row * (S / TI);
    const int st = blockIdx.x / bpt, r = blockIdx.x - st * bpt;
    const int nsx = G / S, sx = st % nsx, sy = st / nsx;
    const int tx = r % per_row, ty = r / per_row;
    const int g = sx * S + tx * TG + w / TI, i = sy * S + ty * TI + w % TI;
    return (sy < R / S) ? g * R + i : -1;
  }
  const int chunks = (R + TI - 1) / TI, tiles = (G + TG - 1) / TG;
  const int bid = blockIdx.x;
  const int c = bid / tiles, t = bid - c * tiles;
  if (c >= chunks) return -1;
  const int g = t * TG + w / TI, i = c * TI + w % TI;
  return (g < G && i < R) ? g * R + i : -1;
}

struct Rows {
  int rows, r0;    // output rows of this launch, first output row
  int G, R, TG;    // block order
  int S;           // super-tile side of the block order (0: chunk-major bands)
  SrtRot rot;
  uint64_t magic;  // ceil(2^40 / rot.ms)
  int xrows;       // rows of the gathered operand (debug-build checks)
  int64_t ldn;     // > 0: reshape P1 fused (k_spmm_rot), stride of Y1''s rows
  int pack16;      // BF16 entries of A1 by rotation, pixels < 2^16 (k_spmm_rot PK)
};

// Stored row and gathered-row remap of segment s of output row `row`.
// Mode 1, the 8-fold form: is output column j served by a mirrored column?
__device__ __forceinline__ bool seg_mirrored(const Rows& A, int j) {
  return A.rot.mirror && 2 * (j % A.rot.q) > A.rot.q;
}
template <int MODE>
__device__ __forceinline__ int seg_row(const Rows& A, int row, int s) {
  if (MODE == 1) {
    const int j = row / A.rot.n_ell, l = row - j * A.rot.n_ell;
    const int js = j % A.rot.q;
    return (seg_mirrored(A, j) ? A.rot.q - js : js) * A.rot.n_ell + l;
  }
  if (MODE == 2) return rot_pixel(row, 4 - s, A.rot.ms, A.magic);
  return row;
}
// Gathered row of stored column c in segment s (t: quarter turns of the row,
// mir: mirrored first).
template <int MODE>
__device__ __forceinline__ int seg_col(const Rows& A, int t, bool mir, int s, int c) {
  if (MODE == 1) return rot_pixel(c, t, A.rot.ms, A.magic, mir);
  if (MODE == 2) return c + s * A.rot.q * A.rot.n_ell;
  return c;
}

// Rows stored as they are (no rotation).  rowptr is the launch's first row's
// pointer.  (A single kernel for both cases, with the row bookkeeping behind
// a struct passed by reference, measured 3% slower.)
template <typename V, int CH>
__global__ void __launch_bounds__(256) k_spmm_plain(int rows, const int32_t* __restrict__ rowptr,
                                                    const int32_t* __restrict__ col,
                                                    const V* __restrict__ val,
                                                    const float* __restrict__ x, int64_t ldx,
                                                    int64_t bsx, float* __restrict__ y,
                                                    int64_t ldy, int64_t bsy, int ncols, int G,
                                                    int R, int TG, int S, int xrows) {
  const int lane = threadIdx.x & 31;
  const int row = block_row(G, R, TG, S);
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
      SRT_CHECK_GATHER(0, c, xrows, g_viol);
      v = wval<V>(val[eb + lane]);
    }
    const int cnt = min(32, e1 - eb);
    // not unrolled: 31 registers, 64 resident warps per SM.  The products
    // wait on their gathers, and more warps in flight beat the deeper
    // per-warp schedule of an unrolled loop (40 registers, 48 warps): 4.5%
    // faster, same summation order.
#pragma unroll 1
    for (int i = 0; i < cnt; ++i) {
      const int ci = __shfl_sync(FULL, c, i);
      const float vi = __shfl_sync(FULL, v, i);
      const float* xr = x + (int64_t)ci * ldx;
#pragma unroll
      for (int q = 0; q < CH; ++q) {
        const int n = n0 + q * 128;
        if (n < ncols) {
          const float4 xv = srt_ldg_keep(xr + n);
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

// A1 / A1^T from the stored quarter of A1 (the plain loop with the stored
// row and the gathered row remapped; scalar parameters only).  MODE 1: row
// (j, l) of A1 from stored row (j mod q, l), pixels turned j / q times.
// MODE 2: row p of A1^T from stored rows rot^-s(p), s = 0..3, gathered rows
// shifted by s q n_ell.  rowptr: the stored matrix's own pointers.
// TR (MODE 1, blocks of 4 sensor columns x 2 radii, G = n_phi, R = n_ell):
// the reshape P1 in the epilogue.  The block's 8 rows go through shared
// memory, 128 slabs at a time, and are written as Y1'[(l, k)][b G + j],
// row stride ldn, 16 bytes (4 sensor columns) per radius and slab.
// PK (BF16 entries, MODE 1, fewer than 2^16 pixels): each lane packs its
// entry's turned pixel and BF16 value into one word, so the warp broadcasts
// an entry with one shuffle instead of two (same pixel, same value; the
// shuffles share the L1 data pipe with the gathers: A1 1.580 -> 1.506 ms
// at 256^3 with BF16 entries).
template <typename V, int CH, int MODE, bool TR, bool PK>
__global__ void __launch_bounds__(256) k_spmm_rot(int rows, int r0,
                                                  const int32_t* __restrict__ rowptr,
                                                  const int32_t* __restrict__ col,
                                                  const V* __restrict__ val,
                                                  const float* __restrict__ x, int64_t ldx,
                                                  int64_t bsx, float* __restrict__ y, int64_t ldy,
                                                  int64_t bsy, int ncols, int G, int R, int TG,
                                                  int S, int ms, int n_ell, int q,
                                                  int mirror, uint64_t magic, int xrows,
                                                  int64_t ldn) {
  const int lane = threadIdx.x & 31;
  const int lr = block_row(G, R, TG, S);
  const bool mine = lr >= 0 && lr < rows;
  if (!TR && !mine) return;  // (TR: every warp reaches the block barrier)
  const int row = r0 + (mine ? lr : 0);
  x += blockIdx.z * bsx;
  if (!TR) y += blockIdx.z * bsy;
  const int n0 = blockIdx.y * (128 * CH) + lane * 4;
  float4 acc[CH];
#pragma unroll
  for (int k = 0; k < CH; ++k) acc[k] = make_float4(0.f, 0.f, 0.f, 0.f);
  int t = 0, sr = row;
  bool mir = false;
  if (MODE == 1) {
    const int j = row / n_ell, l = row - j * n_ell;
    t = j / q;
    int js = j - t * q;
    if (mirror && 2 * js > q) {  // 8-fold form: stored column q - js, mirrored
      js = q - js;
      mir = true;
    }
    sr = js * n_ell + l;
  }
#pragma unroll 1
  for (int s = 0; s < (MODE == 2 ? 4 : 1); ++s) {
    if (MODE == 2) sr = rot_pixel(row, 4 - s, ms, magic);
    const int off = MODE == 2 ? s * q * n_ell : 0;
    const int e0 = rowptr[sr], e1 = TR && !mine ? e0 : rowptr[sr + 1];
    for (int eb = e0; eb < e1; eb += 32) {
      int c = 0;
      float v = 0.f;
      uint32_t pw = 0;
      if (eb + lane < e1) {
        c = col[eb + lane];
        c = MODE == 1 ? rot_pixel(c, t, ms, magic, mir) : c + off;
        SRT_CHECK_GATHER(0, c, xrows, g_viol);
        if constexpr (PK)
          pw = ((uint32_t)c << 16) | (uint32_t)val[eb + lane];
        else
          v = wval<V>(val[eb + lane]);
      }
      const int cnt = min(32, e1 - eb);
#pragma unroll 1
      for (int i = 0; i < cnt; ++i) {  // not unrolled, as in k_spmm_plain
        int ci;
        float vi;
        if constexpr (PK) {
          const uint32_t wi = __shfl_sync(FULL, pw, i);
          ci = (int)(wi >> 16);
          vi = __uint_as_float(wi << 16);
        } else {
          ci = __shfl_sync(FULL, c, i);
          vi = __shfl_sync(FULL, v, i);
        }
        const float* xr = x + (int64_t)ci * ldx;
#pragma unroll
        for (int k = 0; k < CH; ++k) {
          const int n = n0 + k * 128;
          if (n < ncols) {
            const float4 xv = srt_ldg_keep(xr + n);
            acc[k].x = fmaf(vi, xv.x, acc[k].x);
            acc[k].y = fmaf(vi, xv.y, acc[k].y);
            acc[k].z = fmaf(vi, xv.z, acc[k].z);
            acc[k].w = fmaf(vi, xv.w, acc[k].w);
          }
        }
      }
    }
  }
  if (!TR) {
    float* yr = y + (int64_t)lr * ldy;
#pragma unroll
    for (int k = 0; k < CH; ++k) {
      const int n = n0 + k * 128;
      if (n < ncols) *reinterpret_cast<float4*>(yr + n) = acc[k];
    }
    return;
  }
  // fused P1: Sb[w][n] holds row w = 2 jl + il (column j0 + jl, radius
  // l0 + il) of the block, 128 slabs n; a thread then writes one radius and
  // slab of the 4 columns
  __shared__ __align__(16) float Sb[8 * 128];
  const int w = threadIdx.x >> 5, tiles = (G + 3) / 4;
  const int c = blockIdx.x / tiles, tt = blockIdx.x - c * tiles;
  const int il = threadIdx.x >> 7, nl = threadIdx.x & 127;
  const int l = 2 * c + il;
  const int64_t cb = (int64_t)blockIdx.z * G + 4 * tt;  // column b G + j0 of Y1'
#pragma unroll
  for (int k = 0; k < CH; ++k) {
    if (k) __syncthreads();  // the previous chunk's reads are done
    *reinterpret_cast<float4*>(Sb + w * 128 + lane * 4) = acc[k];
    __syncthreads();
    const int n = blockIdx.y * (128 * CH) + k * 128 + nl;
    if (l < R && n < ncols && 4 * tt < G)
      *reinterpret_cast<float4*>(y + ((int64_t)l * ncols + n) * ldn + cb) =
          make_float4(Sb[il * 128 + nl], Sb[(2 + il) * 128 + nl], Sb[(4 + il) * 128 + nl],
                      Sb[(6 + il) * 128 + nl]);
  }
}

// Scalar path for any ncols / strides: lane owns columns lane + 32 i.
template <typename V, int PER, int MODE>
__global__ void __launch_bounds__(256) k_spmm_scalar(Rows A, const int32_t* __restrict__ rowptr,
                                                     const int32_t* __restrict__ col,
                                                     const V* __restrict__ val,
                                                     const float* __restrict__ x, int64_t ldx,
                                                     int64_t bsx, float* __restrict__ y,
                                                     int64_t ldy, int64_t bsy, int ncols) {
  const int lane = threadIdx.x & 31;
  const int lr = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (lr >= A.rows) return;
  const int row = A.r0 + lr;
  x += blockIdx.z * bsx;
  y += blockIdx.z * bsy;
  const int n0 = blockIdx.y * (32 * PER) + lane;
  float acc[PER];
#pragma unroll
  for (int q = 0; q < PER; ++q) acc[q] = 0.f;
  constexpr int NSEG = MODE == 2 ? 4 : 1;
  const int t = MODE == 1 ? (row / A.rot.n_ell) / A.rot.q : 0;
  const bool mir = MODE == 1 && seg_mirrored(A, row / A.rot.n_ell);
  for (int s = 0; s < NSEG; ++s) {
    const int sr = seg_row<MODE>(A, row, s);
    const int e0 = rowptr[sr], e1 = rowptr[sr + 1];
    for (int eb = e0; eb < e1; eb += 32) {
      int c = 0;
      float v = 0.f;
      if (eb + lane < e1) {
        c = seg_col<MODE>(A, t, mir, s, col[eb + lane]);
        SRT_CHECK_GATHER(0, c, A.xrows, g_viol);
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
  }
  float* yr = y + (int64_t)lr * ldy;
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int n = n0 + q * 32;
    if (n < ncols) yr[n] = acc[q];
  }
}

template <typename V, int MODE>
int launch(const SrtCsr& A, const V* val, const Rows& W, const float* x, int64_t ldx, int64_t bsx,
           float* y, int64_t ldy, int64_t bsy, int ncols, int batch, cudaStream_t st) {
  dim3 block(256);
  const bool vec = (ncols % 4 == 0) && (ldx % 4 == 0) && (ldy % 4 == 0) && (bsx % 4 == 0) &&
                   (bsy % 4 == 0) && ((uintptr_t)x % 16 == 0) && ((uintptr_t)y % 16 == 0);
  const int gx = W.S > 0   ? (W.G / W.S) * (W.R / W.S) * (W.S / W.TG) * (W.S / (8 / W.TG))
                 : W.G > 0 ? ((W.G + W.TG - 1) / W.TG) * ((W.R + 8 / W.TG - 1) / (8 / W.TG))
                           : (W.rows + 7) / 8;
  if (vec && MODE == 0) {
    const int32_t* rp = A.rowptr + W.r0;
    const int chunks = (ncols + 127) / 128;
    const int CH = chunks >= 4 ? 4 : chunks;
    dim3 grid(gx, CH == 4 ? (ncols + 511) / 512 : 1, batch);
    switch (CH) {
      case 4: k_spmm_plain<V, 4><<<grid, block, 0, st>>>(W.rows, rp, A.col, val, x, ldx, bsx, y, ldy, bsy, ncols, W.G, W.R, W.TG, W.S, W.xrows); break;
      case 3: k_spmm_plain<V, 3><<<grid, block, 0, st>>>(W.rows, rp, A.col, val, x, ldx, bsx, y, ldy, bsy, ncols, W.G, W.R, W.TG, W.S, W.xrows); break;
      case 2: k_spmm_plain<V, 2><<<grid, block, 0, st>>>(W.rows, rp, A.col, val, x, ldx, bsx, y, ldy, bsy, ncols, W.G, W.R, W.TG, W.S, W.xrows); break;
      default: k_spmm_plain<V, 1><<<grid, block, 0, st>>>(W.rows, rp, A.col, val, x, ldx, bsx, y, ldy, bsy, ncols, W.G, W.R, W.TG, W.S, W.xrows); break;
    }
  } else if (vec) {
    // at most 2 chunks of 128 columns per warp, wider rows across
    // blockIdx.y: with 512 slabs, 31 registers and 64 resident warps per SM
    // instead of 47 and 40 made A1 13% faster (17.6 -> 15.3 ms at 512^3)
    const int chunks = (ncols + 127) / 128;
    const int CH = chunks >= 2 ? 2 : chunks;
    dim3 grid(gx, (ncols + 128 * CH - 1) / (128 * CH), batch);
    const SrtRot& r = W.rot;
#define SRT_ROT_LAUNCH(C, T, P)                                                                 \
  k_spmm_rot<V, C, MODE, T, P><<<grid, block, 0, st>>>(W.rows, W.r0, A.rowptr, A.col, val, x,  \
                                                       ldx, bsx, y, ldy, bsy, ncols, W.G, W.R,  \
                                                       W.TG, W.S, r.ms, r.n_ell, r.q,           \
                                                       r.mirror, W.magic, W.xrows, W.ldn)
    constexpr bool kPk = MODE == 1 && std::is_same<V, uint16_t>::value;
    constexpr bool kTr = MODE == 1;
    const bool tr = kTr && W.ldn > 0, pk = kPk && W.pack16;
    if (tr && pk) {
      if (CH == 2) SRT_ROT_LAUNCH(2, kTr, kPk);
      else SRT_ROT_LAUNCH(1, kTr, kPk);
    } else if (tr) {
      if (CH == 2) SRT_ROT_LAUNCH(2, kTr, false);
      else SRT_ROT_LAUNCH(1, kTr, false);
    } else if (pk) {
      if (CH == 2) SRT_ROT_LAUNCH(2, false, kPk);
      else SRT_ROT_LAUNCH(1, false, kPk);
    } else if (CH == 2) {
      SRT_ROT_LAUNCH(2, false, false);
    } else {
      SRT_ROT_LAUNCH(1, false, false);
    }
#undef SRT_ROT_LAUNCH
  } else {
    dim3 grid((W.rows + 7) / 8, (ncols + 127) / 128, batch);
    k_spmm_scalar<V, 4, MODE><<<grid, block, 0, st>>>(W, A.rowptr, A.col, val, x, ldx, bsx, y,
                                                      ldy, bsy, ncols);
  }
  SRT_CUDA_TRY(cudaGetLastError());
  return SRT_OK;
}

template <typename V>
int dispatch(const SrtCsr& A, const V* val, const Rows& W, const float* x, int64_t ldx,
             int64_t bsx, float* y, int64_t ldy, int64_t bsy, int ncols, int batch,
             cudaStream_t st) {
  switch (W.rot.mode) {
    case 1: return launch<V, 1>(A, val, W, x, ldx, bsx, y, ldy, bsy, ncols, batch, st);
    case 2: return launch<V, 2>(A, val, W, x, ldx, bsx, y, ldy, bsy, ncols, batch, st);
    default: return launch<V, 0>(A, val, W, x, ldx, bsx, y, ldy, bsy, ncols, batch, st);
  }
}

}  // namespace

int srt_spmm(const SrtCsr& A, int wdt, const float* x, int64_t ldx, int64_t bsx, float* y,
             int64_t ldy, int64_t bsy, int ncols, int batch, cudaStream_t st, int G, int R,
             int TG, int64_t r0, int64_t rows, SrtRot rot, int S, int64_t ldn) {
  if (rows < 0) rows = A.rows - r0;
  if (rows <= 0) return SRT_OK;
  if (rows > 0x7fffffff || r0 + rows > 0x7fffffff) return SRT_ERR_ARG;
  uint64_t magic = 0;
  if (rot.mode != 0) {
    if (rot.q <= 0 || rot.ms <= 0 || rot.ms >= (1 << 16) || rot.n_ell <= 0 ||
        (int64_t)rot.ms * rot.ms >= (1 << 24))
      return SRT_ERR_ARG;
    magic = ((1ull << 40) + rot.ms - 1) / rot.ms;
  }
  if (G > 0 && (int64_t)G * R != rows) G = 0;
  if (TG != 1 && TG != 2 && TG != 4 && TG != 8) TG = 1;
  if (G <= 0 || S <= 0 || G % S || R % S || S % TG || S % (8 / TG)) S = 0;
  // gathered operand: A's columns, or for A1^T from the stored quarter
  // (mode 2) the rows (j, l) of every sensor column
  const int64_t xr = rot.mode == 2 ? (int64_t)4 * rot.q * rot.n_ell : A.cols;
  if (ldn > 0) {
    // fused P1: the rotated-rows kernel with blocks of 4 sensor columns x
    // 2 radii over all rows, 16-byte aligned pieces of Y1'
    if (rot.mode != 1 || G <= 0 || r0 != 0 || G % 4 || ncols % 4 || ldx % 4 || bsx % 4 ||
        ldn % 4 || (uintptr_t)x % 16 || (uintptr_t)y % 16 || (int64_t)batch * G > ldn)
      return SRT_ERR_ARG;
    TG = 4;
    S = 0;
  }
  // BF16 entries of A1 turned onto fewer than 2^16 pixels: pixel and value
  // in one 32-bit word (one shuffle per entry)
  const int pack16 = rot.mode == 1 && wdt == SRT_BF16 && A.cols <= 65536;
  const Rows W{(int)rows, (int)r0, G, R, TG, S, rot, magic, srt_checked_rows(xr), ldn, pack16};
  if (wdt == SRT_BF16) return dispatch<uint16_t>(A, A.v16, W, x, ldx, bsx, y, ldy, bsy, ncols, batch, st);
  return dispatch<float>(A, A.v32, W, x, ldx, bsx, y, ldy, bsy, ncols, batch, st);
}

long long srt_checks_take_spmm() {
#ifdef SRT_CHECKS
  unsigned long long v = 0, z = 0;
  if (cudaMemcpyFromSymbol(&v, g_viol, sizeof(v)) != cudaSuccess) return -1;
  if (cudaMemcpyToSymbol(g_viol, &z, sizeof(z)) != cudaSuccess) return -1;
  return (long long)v;
#else
  return 0;
#endif
}
