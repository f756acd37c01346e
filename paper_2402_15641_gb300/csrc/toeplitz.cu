// Second product of Algorithms 1 and 2 through the Toeplitz structure of A2.
//
// When the sensor rings are spaced like the slabs (ring spacing dz, any
// number n_zs of rings, any offset), ring h sits at slab h + s plus a fixed
// fraction eps of a slab (offset of the ring range = s dz + eps), and the
// semicircle of ring h and radius l_m meets cell (radius bin l, slab k)
// exactly as the semicircle of ring h+1 meets cell (l, k+1):
//   A2[(h,m),(l,k)] = T[m, d = k - h - s, l],
// so all of A2 (and A2^T) is held by the master tensor T: a few "taps"
// (l, d, weight) per radius m instead of one row per (ring, radius).  T is
// assembled once for one ring at eps over the D = mz + n_zs - 1 slab offsets
// d = q - (n_zs - 1) - s, q < D, that some (ring, slab) pair takes.
//
// The taps are stored twice, grouped so that the entries of any output row
// form ONE contiguous range, which the product kernel then walks exactly like
// a CSR row (coalesced batch of 32 entries, shuffle broadcast, float4
// gathers of dense rows):
//   forward  (rows (h, m) of A2):   sub-rows (m, q), each listing l
//     ascending; row (h, m) is sub-rows q = n_zs-1-h .. n_zs-2-h+mz, i.e.
//     every slab k = h + q - (n_zs-1) of the volume.  Entry key = l | q << 16;
//     gathered row l*mz + k.
//   adjoint (rows (l, k) of A2^T):  sub-rows (l, e = D - 1 - q), each listing
//     m ascending; row (l, k) is sub-rows e = mz-1-k .. mz-2-k+n_zs, i.e.
//     rings h = k + e - (mz-1) = 0 .. n_zs-1 in ascending order.  Entry key =
//     m | e << 16; gathered row h*n_ell + m.
// With the rings at the slab centres (n_zs = mz, s = eps = 0), D = 2 mz - 1.
// The adjoint visits its entries in the same order as the CSR form of A2^T
// (ascending (h, m)), the forward by ascending (d, l).  Every output row is
// owned by one warp: no atomics.
#include <algorithm>
#include <cstdlib>
#include <vector>

#include "common.cuh"
#include "devutil.cuh"

namespace {

constexpr unsigned FULL = 0xffffffffu;
#ifdef SRT_CHECKS
__device__ unsigned long long g_viol;  // gathered rows outside their operand
#endif

template <typename V>
__device__ __forceinline__ float tap_w(V v);
template <>
__device__ __forceinline__ float tap_w<float>(float v) {
  return v;
}
template <>
__device__ __forceinline__ float tap_w<uint16_t>(uint16_t v) {
  return srt_bf16_to_f32(v);
}

struct TapArgs {
  const int32_t* rowptr;  // sub-row pointers
  const int32_t* key;     // packed (index, offset) per tap
  int mz, n_zs, n_ell, r0;  // r0: first output row of this launch
  int rows, G, R, TG;     // rows of this launch; block order (G groups of R, TG per block)
  int xrows;              // rows of the gathered operand (debug-build checks)
};

// Block-to-row order as in spmm.cu: with G > 0 a block owns TG groups x 8/TG
// consecutive rows, blocks chunk-major; with G = 0 consecutive rows.
__device__ __forceinline__ int tap_row(int G, int R, int TG) {
  const int w = threadIdx.x >> 5;
  if (G <= 0) return blockIdx.x * (blockDim.x >> 5) + w;
  const int TI = 8 / TG;
  const int chunks = (R + TI - 1) / TI, tiles = (G + TG - 1) / TG;
  const int c = blockIdx.x / tiles, t = blockIdx.x - c * tiles;
  if (c >= chunks) return -1;
  const int g = t * TG + w / TI, i = c * TI + w % TI;
  return (g < G && i < R) ? g * R + i : -1;
}

// ADJ = false: y[(h,m)][n] = sum T[m,d,l] x[l*mz + h + d][n]      (A2 Y1')
// ADJ = true:  y[(l,k)][n] = sum T[m,k-h,l] x[h*n_ell + m][n]     (A2^T P')
// Lanes own 4 consecutive dense columns of each 128-column chunk.
template <typename V, int CH, bool ADJ>
__global__ void __launch_bounds__(256) k_taps(TapArgs A, const V* __restrict__ val,
                                              const float* __restrict__ x, int64_t ldx,
                                              float* __restrict__ y, int64_t ldy, int ncols) {
  const int lane = threadIdx.x & 31;
  const int lr = tap_row(A.G, A.R, A.TG);
  if (lr < 0 || lr >= A.rows) return;
  const int row = A.r0 + lr;
  const int mz = A.mz, nz = A.n_zs, D = mz + nz - 1;
  int a, b;  // (h, m) forward, (l, k) adjoint
  if (ADJ) {
    a = row / mz;
    b = row - a * mz;
  } else {
    a = row / A.n_ell;
    b = row - a * A.n_ell;
  }
  // forward: sub-rows m*D + (nz-1-h) .. +mz; adjoint: l*D + (mz-1-k) .. +nz
  const int64_t s0 = ADJ ? (int64_t)a * D + (mz - 1 - b) : (int64_t)b * D + (nz - 1 - a);
  const int e0 = A.rowptr[s0], e1 = A.rowptr[s0 + (ADJ ? nz : mz)];
  const int n0 = blockIdx.y * (128 * CH) + lane * 4;
  float4 acc[CH];
#pragma unroll
  for (int q = 0; q < CH; ++q) acc[q] = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int eb = e0; eb < e1; eb += 32) {
    int c = 0;
    float v = 0.f;
    if (eb + lane < e1) {
      const int kk = A.key[eb + lane];
      const int lo = kk & 0xffff, off = kk >> 16;
      // forward: off = q, gathered row l*mz + h + q - (nz-1)
      // adjoint: off = e, h = k + e - (mz-1), gathered row h*n_ell + m
      c = ADJ ? (b + off - (mz - 1)) * A.n_ell + lo : lo * mz + a + off - (nz - 1);
      SRT_CHECK_GATHER(0, c, A.xrows, g_viol);
      v = tap_w<V>(val[eb + lane]);
    }
    const int cnt = min(32, e1 - eb);
    // not unrolled: 31 registers and 64 resident warps per SM against 48
    // registers / 40 warps for the compiler's unroll; the product waits on
    // its gathers, and more warps win (A2, A2^T 4.7% faster, same order)
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
  float* yr = y + (int64_t)lr * ldy;
#pragma unroll
  for (int q = 0; q < CH; ++q) {
    const int n = n0 + q * 128;
    if (n < ncols) *reinterpret_cast<float4*>(yr + n) = acc[q];
  }
}

// The same for any dense width and strides: lane owns columns lane + 32 i.
template <typename V, int PER, bool ADJ>
__global__ void __launch_bounds__(256) k_taps_scalar(TapArgs A, const V* __restrict__ val,
                                                     const float* __restrict__ x, int64_t ldx,
                                                     float* __restrict__ y, int64_t ldy,
                                                     int ncols) {
  const int lane = threadIdx.x & 31;
  const int lr = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (lr >= A.rows) return;
  const int row = A.r0 + lr;
  const int mz = A.mz, nz = A.n_zs, D = mz + nz - 1;
  const int a = ADJ ? row / mz : row / A.n_ell;
  const int b = ADJ ? row - a * mz : row - a * A.n_ell;
  const int64_t s0 = ADJ ? (int64_t)a * D + (mz - 1 - b) : (int64_t)b * D + (nz - 1 - a);
  const int e0 = A.rowptr[s0], e1 = A.rowptr[s0 + (ADJ ? nz : mz)];
  const int n0 = blockIdx.y * (32 * PER) + lane;
  float acc[PER];
#pragma unroll
  for (int q = 0; q < PER; ++q) acc[q] = 0.f;
  for (int eb = e0; eb < e1; eb += 32) {
    int c = 0;
    float v = 0.f;
    if (eb + lane < e1) {
      const int kk = A.key[eb + lane];
      const int lo = kk & 0xffff, off = kk >> 16;
      c = ADJ ? (b + off - (mz - 1)) * A.n_ell + lo : lo * mz + a + off - (nz - 1);
      SRT_CHECK_GATHER(0, c, A.xrows, g_viol);
      v = tap_w<V>(val[eb + lane]);
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
  float* yr = y + (int64_t)lr * ldy;
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int n = n0 + q * 32;
    if (n < ncols) yr[n] = acc[q];
  }
}

template <typename V, bool ADJ>
int launch(const TapArgs& A, const V* val, const float* x, int64_t ldx, float* y, int64_t ldy,
           int ncols, cudaStream_t st) {
  const bool vec = ncols % 4 == 0 && ldx % 4 == 0 && ldy % 4 == 0 && (uintptr_t)x % 16 == 0 &&
                   (uintptr_t)y % 16 == 0;
  if (!vec) {
    dim3 grid((unsigned)(((int64_t)A.rows + 7) / 8), (ncols + 127) / 128, 1);
    k_taps_scalar<V, 4, ADJ><<<grid, 256, 0, st>>>(A, val, x, ldx, y, ldy, ncols);
    SRT_CUDA_TRY(cudaGetLastError());
    return SRT_OK;
  }
  const int TI = 8 / A.TG;
  const int64_t gx = A.G > 0 ? (int64_t)((A.R + TI - 1) / TI) * ((A.G + A.TG - 1) / A.TG)
                             : ((int64_t)A.rows + 7) / 8;
  if (gx > 0x7fffffff) return SRT_ERR_ARG;
  const int chunks = (ncols + 127) / 128;
  const int CH = chunks >= 4 ? 4 : chunks;
  dim3 grid((unsigned)gx, (ncols + 128 * CH - 1) / (128 * CH), 1);
  switch (CH) {
    case 4: k_taps<V, 4, ADJ><<<grid, 256, 0, st>>>(A, val, x, ldx, y, ldy, ncols); break;
    case 3: k_taps<V, 3, ADJ><<<grid, 256, 0, st>>>(A, val, x, ldx, y, ldy, ncols); break;
    case 2: k_taps<V, 2, ADJ><<<grid, 256, 0, st>>>(A, val, x, ldx, y, ldy, ncols); break;
    default: k_taps<V, 1, ADJ><<<grid, 256, 0, st>>>(A, val, x, ldx, y, ldy, ncols); break;
  }
  SRT_CUDA_TRY(cudaGetLastError());
  return SRT_OK;
}

// Upload one grouped tap list (host vectors) into t.
int upload(const std::vector<int32_t>& rp, const std::vector<int32_t>& key,
           const std::vector<float>& w32, const std::vector<uint16_t>& w16, SrtTaps* t,
           int64_t* bytes) {
  t->nsub = (int64_t)rp.size() - 1;
  t->nent = (int64_t)key.size();
  SRT_TRY(srt_dmalloc(&t->rowptr, (int64_t)rp.size(), bytes));
  SRT_TRY(srt_dmalloc(&t->key, t->nent, bytes));
  SRT_CUDA_TRY(cudaMemcpy(t->rowptr, rp.data(), rp.size() * 4, cudaMemcpyHostToDevice));
  if (t->nent)
    SRT_CUDA_TRY(cudaMemcpy(t->key, key.data(), key.size() * 4, cudaMemcpyHostToDevice));
  if (!w32.empty()) {
    SRT_TRY(srt_dmalloc(&t->w32, t->nent, bytes));
    SRT_CUDA_TRY(cudaMemcpy(t->w32, w32.data(), w32.size() * 4, cudaMemcpyHostToDevice));
  }
  if (!w16.empty()) {
    SRT_TRY(srt_dmalloc(&t->w16, t->nent, bytes));
    SRT_CUDA_TRY(cudaMemcpy(t->w16, w16.data(), w16.size() * 2, cudaMemcpyHostToDevice));
  }
  return SRT_OK;
}

}  // namespace

void srt_taps_free(SrtTaps* t) {
  cudaFree(t->rowptr);
  cudaFree(t->key);
  cudaFree(t->w32);
  cudaFree(t->w16);
  *t = SrtTaps();
}

// T: rows m < n_ell, columns l*D + q (D = mz + n_zs - 1), ascending.
int srt_build_taps(srt_plan_s* plan, const SrtCsr& T, int64_t* nnz2, int64_t* bytes) {
  const srt_geometry& g = plan->g;
  const int mz = g.mz, nz = g.n_zs, n_ell = g.n_ell, D = mz + nz - 1;
  if (T.rows != n_ell || n_ell > 0xffff || D > 0x7fff) return SRT_ERR_ARG;
  const int64_t nt = T.nnz;
  std::vector<int32_t> rp(n_ell + 1), col(nt);
  std::vector<float> v32(T.v32 ? nt : 0);
  std::vector<uint16_t> v16(T.v16 ? nt : 0);
  SRT_CUDA_TRY(cudaMemcpy(rp.data(), T.rowptr, rp.size() * 4, cudaMemcpyDeviceToHost));
  if (nt) {
    SRT_CUDA_TRY(cudaMemcpy(col.data(), T.col, nt * 4, cudaMemcpyDeviceToHost));
    if (T.v32) SRT_CUDA_TRY(cudaMemcpy(v32.data(), T.v32, nt * 4, cudaMemcpyDeviceToHost));
    if (T.v16) SRT_CUDA_TRY(cudaMemcpy(v16.data(), T.v16, nt * 2, cudaMemcpyDeviceToHost));
  }
  // entries of A2: the tap in column q serves the rings h < nz whose slab
  // k = h + u, u = q - (nz - 1), lies in the volume
  int64_t n2 = 0;
  for (int64_t e = 0; e < nt; ++e) {
    const int u = col[e] % D - (nz - 1);
    const int h0 = std::max(0, -u), h1 = std::min(nz - 1, mz - 1 - u);
    n2 += h1 >= h0 ? h1 - h0 + 1 : 0;
  }
  *nnz2 = n2;
  // counting sorts, stable in T's (m, l, q) order
  const int64_t nsub = (int64_t)n_ell * D;
  std::vector<int32_t> fp(nsub + 1, 0), ap(nsub + 1, 0);
  for (int m = 0; m < n_ell; ++m)
    for (int e = rp[m]; e < rp[m + 1]; ++e) {
      const int l = col[e] / D, q = col[e] % D;
      ++fp[(int64_t)m * D + q + 1];
      ++ap[(int64_t)l * D + (D - 1 - q) + 1];
    }
  for (int64_t i = 0; i < nsub; ++i) {
    fp[i + 1] += fp[i];
    ap[i + 1] += ap[i];
  }
  std::vector<int32_t> fk(nt), ak(nt);
  std::vector<int32_t> fpos(fp.begin(), fp.end() - 1), apos(ap.begin(), ap.end() - 1);
  std::vector<float> f32(v32.size()), a32(v32.size());
  std::vector<uint16_t> f16(v16.size()), a16(v16.size());
  for (int m = 0; m < n_ell; ++m)
    for (int e = rp[m]; e < rp[m + 1]; ++e) {
      const int l = col[e] / D, q = col[e] % D, ee = D - 1 - q;
      const int64_t i = fpos[(int64_t)m * D + q]++, j = apos[(int64_t)l * D + ee]++;
      fk[i] = l | (q << 16);
      ak[j] = m | (ee << 16);
      if (!v32.empty()) f32[i] = a32[j] = v32[e];
      if (!v16.empty()) f16[i] = a16[j] = v16[e];
    }
  SRT_TRY(upload(fp, fk, f32, f16, &plan->tf, bytes));
  SRT_TRY(upload(ap, ak, a32, a16, &plan->ta, bytes));
  if (!(plan->g.flags & SRT_ROWWISE)) {
    SRT_TRY(srt_build_tiles(plan, rp, col, v32, v16, bytes));
    plan->tiles = 1;
  }
  return SRT_OK;
}

int srt_taps_apply(const srt_plan_s* plan, bool adjoint, int64_t r0, int64_t rows, int G, int R,
                   int TG, const float* x, int64_t ldx, float* y, int64_t ldy, int ncols,
                   cudaStream_t st) {
  const srt_geometry& g = plan->g;
  const SrtTaps& t = adjoint ? plan->ta : plan->tf;
  if (!t.rowptr || rows <= 0 || ncols <= 0) return SRT_ERR_ARG;
  if (G > 0 && (int64_t)G * R != rows) G = 0;
  if (TG != 1 && TG != 2 && TG != 4 && TG != 8) TG = 1;
  TapArgs A{t.rowptr, t.key, g.mz, g.n_zs, g.n_ell, (int)r0, (int)rows, G, R, TG,
            srt_checked_rows(adjoint ? (int64_t)g.n_zs * g.n_ell : (int64_t)g.n_ell * g.mz)};
  if (g.weight_dtype == SRT_BF16) {
    if (!t.w16) return SRT_ERR_ARG;
    return adjoint ? launch<uint16_t, true>(A, t.w16, x, ldx, y, ldy, ncols, st)
                   : launch<uint16_t, false>(A, t.w16, x, ldx, y, ldy, ncols, st);
  }
  if (!t.w32) return SRT_ERR_ARG;
  return adjoint ? launch<float, true>(A, t.w32, x, ldx, y, ldy, ncols, st)
                 : launch<float, false>(A, t.w32, x, ldx, y, ldy, ncols, st);
}

long long srt_checks_take_taps() {
#ifdef SRT_CHECKS
  unsigned long long v = 0, z = 0;
  if (cudaMemcpyFromSymbol(&v, g_viol, sizeof(v)) != cudaSuccess) return -1;
  if (cudaMemcpyToSymbol(g_viol, &z, sizeof(z)) != cudaSuccess) return -1;
  return (long long)v;
#else
  return 0;
#endif
}
