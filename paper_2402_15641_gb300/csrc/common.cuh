// Internal declarations shared by the CUDA translation units of libsrt.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <vector>

#include "srt.h"

#define SRT_PI 3.14159265358979323846264338327950288

// Debug builds (-DSRT_CHECKS, build.py's checked library): every product
// kernel checks each gathered row index base + off against its operand's row
// count n before the access.  An index outside [0, n) is counted in the
// translation unit's violation counter and replaced by row 0 (off = -base),
// so a bad index is reported (srt_checks_read, and the call's status)
// without touching memory outside the operand.  Release builds compile the
// check away.
#ifdef SRT_CHECKS
#define SRT_CHECK_GATHER(base, off, n, counter)                                            \
  do {                                                                                     \
    if ((unsigned long long)((long long)(base) + (long long)(off)) >=                      \
        (unsigned long long)(n)) {                                                         \
      atomicAdd(&(counter), 1ull);                                                         \
      (off) = -(base);                                                                     \
    }                                                                                      \
  } while (0)
#else
#define SRT_CHECK_GATHER(base, off, n, counter) \
  do {                                          \
  } while (0)
#endif

// Violations counted by each translation unit's kernels since the last
// call, then reset (0 in release builds), and the row cap of srt_checks_cap.
long long srt_checks_take_spmm();
long long srt_checks_take_taps();
long long srt_checks_take_tiles();
long long srt_checks_take_a1tiles();
int srt_checks_rowcap();
// The operand row count a launch checks against: n, or the test cap if lower.
inline int srt_checked_rows(int64_t n) {
  const int cap = srt_checks_rowcap();
  return (cap > 0 && cap < n) ? cap : (int)(n > 0x7fffffff ? 0x7fffffff : n);
}

// Return SRT_ERR_CUDA from the enclosing function when a runtime call fails.
#define SRT_CUDA_TRY(expr)                         \
  do {                                             \
    cudaError_t e_ = (expr);                       \
    if (e_ != cudaSuccess) return SRT_ERR_CUDA;    \
  } while (0)

#define SRT_TRY(expr)                 \
  do {                                \
    int s_ = (expr);                  \
    if (s_ != SRT_OK) return s_;      \
  } while (0)

// One sparse operator in CSR form.  Entries are stored either as FP32 (v32)
// or as BF16 bit patterns (v16); v64 holds the FP64 lengths when the plan was
// built with SRT_KEEP_F64.
struct SrtCsr {
  int32_t rows = 0, cols = 0;
  int64_t nnz = 0;
  int32_t* rowptr = nullptr;  // rows + 1
  int32_t* col = nullptr;     // nnz
  float* v32 = nullptr;       // nnz (SRT_FP32)
  uint16_t* v16 = nullptr;    // nnz (SRT_BF16)
  double* v64 = nullptr;      // nnz (SRT_KEEP_F64)
};

// Toeplitz form of A2 (toeplitz.cu), used when the rings are spaced like the
// slabs (ring h at slab h + s plus a fixed fraction): A2[(h,m),(l,k)] =
// T[m, k - h - s, l] over D = mz + n_zs - 1 offsets, column q of T at
// offset q - (n_zs - 1) - s.  Taps grouped in sub-rows so that every output
// row of A2 (forward) or A2^T (adjoint) is one contiguous range: forward
// sub-rows (m, q) listing l, key l | q << 16; adjoint sub-rows
// (l, D - 1 - q) listing m, key m | (D - 1 - q) << 16.
struct SrtTaps {
  int64_t nsub = 0, nent = 0;
  int32_t* rowptr = nullptr;  // nsub + 1
  int32_t* key = nullptr;     // nent
  float* w32 = nullptr;       // nent (SRT_FP32)
  uint16_t* w16 = nullptr;    // nent (SRT_BF16)
};

// The same operator as records of 2 x 2 output-row tiles (tiles.cu): per
// radius pair, one record per gathered row of a tile, holding the row's
// offset and four weights, sorted by key (the gathered row's slab or ring
// offset from the tile) with the first record of each key in ptr.
struct SrtTiles {
  int pairs = 0, nkeys = 0, key0 = 0;
  bool desc = false;       // blocks issued from the last radius pair down
  int64_t nrec = 0;
  int32_t* ptr = nullptr;  // pairs * (nkeys + 1)
  int32_t* off = nullptr;  // nrec
  float* w32 = nullptr;    // 4 * nrec (SRT_FP32)
  uint16_t* w16 = nullptr; // 4 * nrec (SRT_BF16)
};

// A1^T as records of 2 x 2 pixel tiles (a1tiles.cu): key = (j << 16 | l),
// four weights per record, two lists per tile (aptr[2t] .. aptr[2t+1]: read
// by every symmetry pass; .. aptr[2t+2]: by the unmirrored passes only).
struct SrtA1Tiles {
  int ntx = 0;
  int64_t na = 0;
  int32_t* aptr = nullptr;  // 2 * ntx^2 + 1
  int32_t* akey = nullptr;  // na
  float* aw32 = nullptr;    // 4 * na (SRT_FP32)
  uint16_t* aw16 = nullptr; // 4 * na (SRT_BF16)
};

struct SrtHostPool;  // copy streams and events of host-buffer calls (api.cu)

struct srt_plan_s {
  srt_geometry g;
  int device = 0;
  SrtCsr a1, a2, a1t, a2t;  // A1 = A^{1,2}, A2 = A^{3,4} and their transposes
  int a1_rot = 0;           // 1: a1, a1t hold the first n_phi/4 sensor columns (4-fold
                            // rotation); 2: the first n_phi/8 + 1 (rotation and mirror)
  SrtA1Tiles a1tl;          // A1^T tile records (a1tiles.cu)
  int a1tiles = 0;          // apply A1^T from a1tl
  int64_t nnz1 = 0;         // entries of the full A1
  int toeplitz = 0;         // second product through the Toeplitz taps below
  SrtTaps tf, ta;           // forward / adjoint taps of A2 (a2, a2t then hold no arrays)
  SrtTiles tlf, tla;        // forward / adjoint 2 x 2 tile records (from the same taps)
  int tiles = 0;            // apply A2, A2^T from tlf / tla (else from tf / ta)
  SrtCsr tm;                // master tensor T (rows m, columns l*(2mz-1) + d + mz - 1)
  int64_t dropped1 = 0, dropped2 = 0;
  int64_t bytes = 0;
  // per-stage timing (srt_plan_set_timing)
  int timing = 0;
  cudaEvent_t ev[2][5] = {};
  int have_times[2] = {0, 0};
  SrtHostPool* host_pool = nullptr;  // created by srt_plan, reused by every host call
};

// ------------------------------------------------------------- assembly
// Builds a1, a2, a1t, a2t of the plan (device kernels on `stream`).
int srt_assemble(srt_plan_s* plan, cudaStream_t stream);
void srt_csr_free(SrtCsr* m);

// Build plan->tf / plan->ta from the master tensor T (rows m, columns
// l*(2 mz - 1) + d + mz - 1); *nnz2 = number of entries of the A2 they stand for.
int srt_build_taps(srt_plan_s* plan, const SrtCsr& T, int64_t* nnz2, int64_t* bytes);
void srt_taps_free(SrtTaps* t);
// Build plan->tlf / plan->tla from T on the host (rows m, columns l*D + q,
// D = mz + n_zs - 1; FP32 or BF16 values, whichever is non-empty).
int srt_build_tiles(srt_plan_s* plan, const std::vector<int32_t>& rp,
                    const std::vector<int32_t>& col, const std::vector<float>& v32,
                    const std::vector<uint16_t>& v16, int64_t* bytes);
void srt_tiles_free(SrtTiles* t);
// Expand the master tensor into CSR A2 (and A2^T when a2t is given), for export.
int srt_expand_a2(const srt_plan_s* plan, SrtCsr* a2, SrtCsr* a2t, cudaStream_t stream);

// ------------------------------------------------------------- operators
// Rows [r0, r0 + rows) of A2 (adjoint = false; rows (h, m)) or A2^T
// (adjoint = true; rows (l, k)) through the taps: y[r - r0][n] = sum over the
// row's taps of w * x[gathered row][n], n < ncols.  Blocks visit the rows as
// srt_spmm does with (G, R, TG).
int srt_taps_apply(const srt_plan_s* plan, bool adjoint, int64_t r0, int64_t rows, int G, int R,
                   int TG, const float* x, int64_t ldx, float* y, int64_t ldy, int ncols,
                   cudaStream_t stream);

// A2 (adjoint = false: ring rows [c0, c1), y at ring c0's first row) or A2^T
// (adjoint = true: slabs [c0, c1) = [0, mz)) from the 2 x 2 tile records,
// blocks of TG coordinate pairs x 8/TG radius pairs.  With ldn > 0 the
// reshape that follows is fused (blocks of 4 x 2 pairs): the forward writes
// y[n ldn + h n_ell + m] for every ring h in [c0, c1) (y at ring 0), the
// adjoint y[n ldn + l mz + k]; ldy is then unused.
int srt_tiles_apply(const srt_plan_s* plan, bool adjoint, int c0, int c1, int TG, const float* x,
                    int64_t ldx, float* y, int64_t ldy, int ncols, cudaStream_t stream,
                    int64_t ldn = 0);

// A1^T tile records from the plan's stored A1 (CSR on the device).
int srt_build_a1tiles(srt_plan_s* plan, int64_t* bytes);
void srt_a1tiles_free(SrtA1Tiles* t);
// A1^T from the tile records: 2 x 2 pixel tiles of pixel rows 2 g0 .. 2 g1 - 1,
// y at pixel row 2 g0; batch items b at x + b bsx, y + b bsy.
int srt_a1tiles_apply(const srt_plan_s* plan, int g0, int g1, const float* x, int64_t ldx,
                      int64_t bsx, float* y, int64_t ldy, int64_t bsy, int ncols, int batch,
                      cudaStream_t stream);

// Output rows of A1 / A1^T served from the stored quarter of A1 (spmm.cu):
// mode 1 = A1 rows (j, l) from stored rows (j mod q, l), pixels turned (with
// mirror: column s q + t from stored column q - t for t > q/2, pixels
// mirrored across the diagonal first);
// mode 2 = A1^T rows (pixels) from 4 stored rows of the stored transpose.
struct SrtRot {
  int mode = 0;           // 0: rows are stored as they are
  int ms = 0, n_ell = 0;  // pixel grid edge, radius bins
  int q = 0;              // n_phi / 4
  int mirror = 0;         // mode 1 only: the 8-fold form (stored columns 0 .. q/2)
};

// y[b][r - r0][n] = sum_e A[r, col[e]] * x[b][col[e]][n] for output rows
// r0 <= r < r0 + rows (rows < 0: to A's end) and n < ncols.  With G > 0 the
// launch's rows (G groups of R) are visited chunk-major across groups, a
// block owning TG groups (1, 2, 4 or 8) x 8/TG consecutive rows of each.
// With S > 0 (dividing G and R) the blocks walk S x S super-tiles of the
// G x R row grid instead of chunk-major bands.  ldn > 0 (A1 with rot.mode
// 1, G = n_phi, R = n_ell, ncols = mz, batch items b): y is Y1', the
// output of the reshape P1, y[(l ncols + k) ldn + b G + j] for row (j, l).
int srt_spmm(const SrtCsr& A, int weight_dtype, const float* x, int64_t ldx, int64_t bsx, float* y,
             int64_t ldy, int64_t bsy, int ncols, int batch, cudaStream_t stream, int G = 0,
             int R = 0, int TG = 1, int64_t r0 = 0, int64_t rows = -1, SrtRot rot = SrtRot(),
             int S = 0, int64_t ldn = 0);

// out[b*obs + c*old + r] = in[b*ibs + r*ild + c] for r < rows, c < cols.
int srt_transpose(const float* in, int64_t ild, int64_t ibs, float* out, int64_t old, int64_t obs,
                  int rows, int cols, int batch, cudaStream_t stream);

int srt_dot(const float* a, const float* b, int64_t n, double* out, double* partials,
            cudaStream_t stream);
constexpr int SRT_DOT_BLOCKS = 608;  // 152 SMs x 4

// --------------------------------------------------- FP64 device helpers
// Angle in [0, pi] whose cosine is u/r, clamped at the ends.  The sine side
// is formed as sqrt((r-u)(r+u)) so tangency keeps full precision.
__host__ __device__ inline double srt_acos_r(double u, double r) {
  if (u >= r) return 0.0;
  if (u <= -r) return SRT_PI;
  return atan2(sqrt((r - u) * (r + u)), u);
}

// Angle in [-pi/2, pi/2] whose sine is u/r, clamped at the ends.
__host__ __device__ inline double srt_asin_r(double u, double r) {
  if (u >= r) return 0.5 * SRT_PI;
  if (u <= -r) return -0.5 * SRT_PI;
  return atan2(u, sqrt((r - u) * (r + u)));
}

__host__ __device__ inline double srt_overlap3(double a0, double a1, double b0, double b1, double c0,
                                               double c1) {
  double lo = fmax(a0, fmax(b0, c0));
  double hi = fmin(a1, fmin(b1, c1));
  return hi > lo ? hi - lo : 0.0;
}

// Exact length of the circle (cx, cy, r) inside the box [x0,x1] x [y0,y1].
// On each quarter of the circle cos and sin are monotone, so the angles whose
// x coordinate lies in [x0, x1] form one interval there, and likewise for y;
// the arc measure is the sum over the quarters of the triple overlap.
__host__ __device__ inline double srt_arc_in_rect(double cx, double cy, double r, double x0,
                                                  double x1, double y0, double y1) {
  const double hp = 0.5 * SRT_PI;
  double a1 = srt_acos_r(x1 - cx, r), a0 = srt_acos_r(x0 - cx, r);  // x in box: [a1, a0] up
  double s0 = srt_asin_r(y0 - cy, r), s1 = srt_asin_r(y1 - cy, r);  // y in box: [s0, s1] right
  double t = srt_overlap3(0.0, hp, a1, a0, s0, s1);
  t += srt_overlap3(hp, SRT_PI, a1, a0, SRT_PI - s1, SRT_PI - s0);
  t += srt_overlap3(-SRT_PI, -hp, -a0, -a1, -SRT_PI - s1, -SRT_PI - s0);
  t += srt_overlap3(-hp, 0.0, -a0, -a1, s0, s1);
  return r * t;
}

// Length of the circle (cx, cy, r) inside the box (the return value) and its
// first moment int y ds there (*my), from the same quarter intervals: on an
// interval [t0, t1] of y = cy + r sin t, the moment is r cy (t1 - t0) +
// r^2 (cos t0 - cos t1), the last factor taken as 2 sin(tm) sin(dt/2).
__host__ __device__ inline double srt_arc_in_rect_m(double cx, double cy, double r, double x0,
                                                    double x1, double y0, double y1, double* my) {
  const double hp = 0.5 * SRT_PI;
  const double a1 = srt_acos_r(x1 - cx, r), a0 = srt_acos_r(x0 - cx, r);
  const double s0 = srt_asin_r(y0 - cy, r), s1 = srt_asin_r(y1 - cy, r);
  const double lo[4] = {fmax(0.0, fmax(a1, s0)), fmax(hp, fmax(a1, SRT_PI - s1)),
                        fmax(-SRT_PI, fmax(-a0, -SRT_PI - s1)), fmax(-hp, fmax(-a0, s0))};
  const double hi[4] = {fmin(hp, fmin(a0, s1)), fmin(SRT_PI, fmin(a0, SRT_PI - s0)),
                        fmin(-hp, fmin(-a1, -SRT_PI - s0)), fmin(0.0, fmin(-a1, s1))};
  double t = 0.0, m = 0.0;
  for (int i = 0; i < 4; ++i) {
    if (hi[i] > lo[i]) {
      const double dt = hi[i] - lo[i];
      t += dt;
      m += r * cy * dt + 2.0 * r * r * sin(0.5 * (lo[i] + hi[i])) * sin(0.5 * dt);
    }
  }
  *my = m;
  return r * t;
}

// int (1 + bx x)(1 + by y) ds along the circle (cx, cy, r) inside the box
// [x0, x1] x [y0, y1], in coordinates centred on a node of the piecewise-
// linear voxels (so x, y and the result stay small).  On each quarter
// interval [t0, t1] = tm -/+ h, with x = X0 + r C (cos s - 1) - r S sin s and
// y = Y0 + r S (cos s - 1) + r C sin s (C = cos tm, S = sin tm, (X0, Y0) the
// interval's midpoint, s in [-h, h]):
//   int ds    = 2 h r
//   int x ds  = r (2 h X0 + r C Ic)
//   int y ds  = r (2 h Y0 + r S Ic)
//   int xy ds = r (2 h X0 Y0 + r (X0 S + Y0 C) Ic + r^2 C S Id)
// with Ic = int (cos s - 1) ds = 2 (sin h - h) and Id = int (cos s - 1)^2 -
// sin^2 s ds = 2 h + sin 2h - 4 sin h over [-h, h] (odd terms vanish),
// taken from their Taylor series for h < 0.05, where the closed forms
// cancel (truncation below 1e-12 relative).
__host__ __device__ inline double srt_arc_bilinear(double cx, double cy, double r, double x0,
                                                   double x1, double y0, double y1, double bx,
                                                   double by) {
  const double hp = 0.5 * SRT_PI;
  const double a1 = srt_acos_r(x1 - cx, r), a0 = srt_acos_r(x0 - cx, r);
  const double s0 = srt_asin_r(y0 - cy, r), s1 = srt_asin_r(y1 - cy, r);
  const double lo[4] = {fmax(0.0, fmax(a1, s0)), fmax(hp, fmax(a1, SRT_PI - s1)),
                        fmax(-SRT_PI, fmax(-a0, -SRT_PI - s1)), fmax(-hp, fmax(-a0, s0))};
  const double hi[4] = {fmin(hp, fmin(a0, s1)), fmin(SRT_PI, fmin(a0, SRT_PI - s0)),
                        fmin(-hp, fmin(-a1, -SRT_PI - s0)), fmin(0.0, fmin(-a1, s1))};
  double acc = 0.0;
  for (int i = 0; i < 4; ++i) {
    if (!(hi[i] > lo[i])) continue;
    const double tm = 0.5 * (lo[i] + hi[i]), h = 0.5 * (hi[i] - lo[i]);
    const double C = cos(tm), S = sin(tm);
    const double X0 = cx + r * C, Y0 = cy + r * S;
    double ic, id;
    if (h < 0.05) {
      const double h2 = h * h, h3 = h2 * h;
      ic = h3 * (-1.0 / 3.0 + h2 * (1.0 / 60.0 - h2 / 2520.0));
      id = h3 * (-2.0 / 3.0 + h2 * (7.0 / 30.0 - h2 * 31.0 / 1260.0));
    } else {
      ic = 2.0 * (sin(h) - h);
      id = 2.0 * h + sin(2.0 * h) - 4.0 * sin(h);
    }
    const double L = 2.0 * h;
    const double mx = L * X0 + r * C * ic, my = L * Y0 + r * S * ic;
    const double mxy = L * X0 * Y0 + r * (X0 * S + Y0 * C) * ic + r * r * C * S * id;
    acc += r * (L + bx * mx + by * my + bx * by * mxy);
  }
  return acc;
}

// Round an FP64 value to BF16 (round to nearest, ties to even) in one step,
// from the FP64 bit pattern: keep 7 fraction bits, round on the other 45.
// Values below the BF16 normal range flush to signed zero (entries here are
// lengths far above it).
__host__ __device__ inline uint16_t srt_f64_to_bf16(double x) {
#ifdef __CUDA_ARCH__
  uint64_t b = (uint64_t)__double_as_longlong(x);
#else
  uint64_t b;
  memcpy(&b, &x, 8);
#endif
  uint64_t sign = b >> 63;
  uint64_t mag = b & 0x7FFFFFFFFFFFFFFFull;
  int e = (int)(mag >> 52) - 1023 + 127;
  if (mag == 0 || e <= 0) return (uint16_t)(sign << 15);
  if (e >= 255) return (uint16_t)((sign << 15) | 0x7F80u);
  uint64_t frac = mag & ((1ull << 52) - 1);
  uint64_t q = ((uint64_t)e << 7) | (frac >> 45);
  uint64_t rem = frac & ((1ull << 45) - 1);
  const uint64_t half = 1ull << 44;
  if (rem > half || (rem == half && (q & 1))) q += 1;  // a carry moves into the exponent
  return (uint16_t)((sign << 15) | q);
}

// 16-byte read-only gather of a dense row with the L1 evict-last hint: the
// rows gathered by a block's 8 warps overlap, and keeping them in L1 ahead
// of streaming data made the products 0.2-2.4% faster (same values).
__device__ __forceinline__ float4 srt_ldg_keep(const float* p) {
  float4 r;
  asm volatile("ld.global.nc.L1::evict_last.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
               : "l"(p));
  return r;
}

// The L2 lines holding bytes [b, e), requested by a warp's 32 lanes at once
// (one line each per round): a list of sparse records read in order then
// costs one L2-miss latency instead of one per line.
__device__ __forceinline__ void srt_prefetch_l2(const void* b, const void* e) {
  const uintptr_t lo = reinterpret_cast<uintptr_t>(b) & ~(uintptr_t)127;
  const uintptr_t hi = reinterpret_cast<uintptr_t>(e);
  for (uintptr_t p = lo + (threadIdx.x & 31) * 128; p < hi; p += 32 * 128)
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

__device__ __forceinline__ float srt_bf16_to_f32(uint16_t v) {
  return __uint_as_float(((uint32_t)v) << 16);
}
