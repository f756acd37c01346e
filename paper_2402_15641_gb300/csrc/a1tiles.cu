// Transposed first product of Algorithm 2 (A1^T F1) from register tiles of
// output rows, with A1 stored for a fundamental set of sensor columns of the
// aperture's symmetry group.
//
// Tiles.  A gather-per-FMA product is bound by the L1 data pipe (one dense
// row fetched per entry).  A circle crossing a pixel usually crosses its
// neighbour too, so a warp owns a 2 x 2 tile of pixels (rows of A1^T) and
// walks the union of its rows' gathered rows: one record per gathered row,
// with four weights (zero where a pixel does not use it).  At 256^3 a record
// serves 2.0 entries on average.  (The same idea for A1 itself, 4
// consecutive radii of one column per warp, measured slower than the
// row-per-warp CSR kernel: there the 8 warps of a block already share their
// gathered pixels through L1, and the tiles lose that sharing.)
//
// Symmetry (Sec. 2's columns are equispaced around the axis).  Let
// rot(ix, iy) = (ms-1-iy, ix) (a quarter turn of the pixel grid) and
// D(ix, iy) = (iy, ix) (the mirror across the diagonal).  With q = n_phi/4,
// phi0 = 0 and the whole aperture, the quarter turn takes sensor column j to
// j + q and the mirror takes column t to q - t, and both map circles to
// circles, so for g = rot^s D^m
//   A1[(C_g(j), l), P_g(p)] = A1[(j, l), p],  C_g(j) = s q + (m ? q - j : j),
// P_g = rot^s after D^m.  Mode 2 (8-fold) stores the columns j = 0 .. q/2:
// column J = s q + t is stored column t (m = 0) for t <= q/2 and q - t
// (m = 1) otherwise.  Columns 0 and q/2 are fixed by a mirror, so in the
// transpose they count once per quarter turn, not twice: their records sit
// apart (list B) and only the unmirrored passes read them.  Mode 1 (4-fold)
// stores j < q; mode 0 stores every column.
//
// A1^T tile T: for each group element g, the stored tile Q = P_g^-1(T) (rot
// and D map aligned 2 x 2 tiles to aligned 2 x 2 tiles when ms is even),
// whose records (j, l), sorted by (list, j, l), gather row (C_g(j), l) of F1
// into the output pixel P_g(q_sigma) of T: a fixed permutation of the
// tile's four slots per g.  With every column stored (one pass) each pixel
// sums its entries in the CSR order of A1^T, ascending (j, l).  Every output
// row is one warp's FP32 sum: no atomics, deterministic.
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "devutil.cuh"

namespace {

#ifdef SRT_CHECKS
__device__ unsigned long long g_viol;  // gathered rows outside their operand
#endif

// Records per group of the main loop; two groups alternate, as in tiles.cu.
constexpr int kH = 3;

template <typename W>
__device__ __forceinline__ void rec_w(const W* p, float w[4]);
template <>
__device__ __forceinline__ void rec_w<float4>(const float4* p, float w[4]) {
  const float4 v = __ldg(p);
  w[0] = v.x;
  w[1] = v.y;
  w[2] = v.z;
  w[3] = v.w;
}
template <>
__device__ __forceinline__ void rec_w<uint2>(const uint2* p, float w[4]) {
  const uint2 v = __ldg(p);  // four BF16 weights, w[0] in the low half of .x
  w[0] = __uint_as_float(v.x << 16);
  w[1] = __uint_as_float(v.x & 0xffff0000u);
  w[2] = __uint_as_float(v.y << 16);
  w[3] = __uint_as_float(v.y & 0xffff0000u);
}

__device__ __forceinline__ void fma4(float2 (&a)[2], float w, const float4& xv) {
  const float2 ww = make_float2(w, w);
  a[0] = __ffma2_rn(ww, make_float2(xv.x, xv.y), a[0]);
  a[1] = __ffma2_rn(ww, make_float2(xv.z, xv.w), a[1]);
}

// Slot (dx*2 + dy) of the stored tile's pixel -> slot of its image under
// g = rot^s D^m (rot: (dx, dy) -> (1-dy, dx); D: (dx, dy) -> (dy, dx)).
__host__ __device__ constexpr int sym_slot(int s, int m, int sg) {
  int dx = sg >> 1, dy = sg & 1;
  if (m) {
    const int t = dx;
    dx = dy;
    dy = t;
  }
  for (int k = 0; k < (s & 3); ++k) {
    const int t = dx;
    dx = 1 - dy;
    dy = t;
  }
  return dx * 2 + dy;
}

struct A1Args {
  const int32_t* ptr;  // record ranges (see the kernels)
  const int32_t* key;  // (j << 16 | l)
  int mode, q, ms, n_phi, n_ell, ntx;
  int G, R, TG, S;     // block order
  int g0, g1;          // tile rows [g0, g1) (pixel rows 2 g0 .. 2 g1 - 1)
  int xrows;           // rows of the gathered operand (debug-build checks)
};


// Warp -> (group, index) as in spmm.cu's block_row: G groups of R, a block
// owning TG groups x 8/TG consecutive indices, chunk-major, or S x S
// super-tiles (S > 0).
__device__ __forceinline__ bool warp_tile(const A1Args& A, int* g, int* i) {
  const int w = threadIdx.x >> 5;
  const int TI = 8 / A.TG;
  if (A.S > 0) {
    const int per_row = A.S / A.TG, bpt = per_row * (A.S / TI);
    const int st = blockIdx.x / bpt, r = blockIdx.x - st * bpt;
    const int nsx = (A.G + A.S - 1) / A.S, sx = st % nsx, sy = st / nsx;
    const int tx = r % per_row, ty = r / per_row;
    *g = sx * A.S + tx * A.TG + w / TI;
    *i = sy * A.S + ty * TI + w % TI;
  } else {
    const int tiles = (A.G + A.TG - 1) / A.TG;
    const int c = blockIdx.x / tiles, t = blockIdx.x - c * tiles;
    *g = t * A.TG + w / TI;
    *i = c * TI + w % TI;
  }
  return *g < A.G && *i < A.R;
}

// ----------------------------------------------------------------- A1^T
// One group element's pass over the stored tile's records: list A
// (ptr[2t] .. ptr[2t+1]) always, list B (.. ptr[2t+2]) for unmirrored g.
template <typename W, int CH, int PS, int PM>
__device__ __forceinline__ void a1t_pass(const A1Args& A, const W* __restrict__ wt, int ta,
                                         int tb, const float* x0, int ldx, const bool (&in)[CH],
                                         float2 (&acc)[4][CH][2]) {
  int qa = ta, qb = tb;
#pragma unroll
  for (int k = 0; k < PS; ++k) {  // rot^-1 on tiles: (a, b) -> (b, ntx-1-a)
    const int t = qa;
    qa = qb;
    qb = A.ntx - 1 - t;
  }
  if (PM) {
    const int t = qa;
    qa = qb;
    qb = t;
  }
  const int64_t t2 = 2 * ((int64_t)qa * A.ntx + qb);
  const int e0 = A.ptr[t2], e1 = A.ptr[t2 + (PM ? 1 : 2)];
  // The stored tile's records are read by its 8 images' warps, far apart in
  // the launch, so they are mostly fetched from DRAM: request the pass's
  // lines at once rather than one miss per line as the walk reaches them
  // (A1^T 1.407 -> 1.374 ms at 256^3; the next pass's lines instead: 1.391,
  // every pass's at the kernel's start: 1.415).
  if (e1 > e0) {
    srt_prefetch_l2(A.key + e0, A.key + e1);
    srt_prefetch_l2(wt + e0, wt + e1);
  }
  const int base = PM ? (PS + 1) * A.q : PS * A.q;
  auto row_of = [&](int k) {  // gathered row (C_g(j), l)
    const int j = k >> 16, l = k & 0xffff;
    int J = PM ? base - j : base + j;
    if (J >= A.n_phi) J -= A.n_phi;
    int row = J * A.n_ell + l;
    SRT_CHECK_GATHER(0, row, A.xrows, g_viol);
    return row;
  };
  constexpr int H = kH;
  int oA[H], oB[H];
  float wA[H][4], wB[H][4];
  float4 vA[H][CH], vB[H][CH];
  // group of records eb .. eb + H - 1: gathered rows, then weights
  auto load = [&](int eb, int (&o)[H], float (&w)[H][4], float4 (&v)[H][CH]) {
#pragma unroll
    for (int u = 0; u < H; ++u) o[u] = row_of(__ldg(A.key + eb + u));
#pragma unroll
    for (int u = 0; u < H; ++u) {
      const float* xr = x0 + (int64_t)o[u] * ldx;
#pragma unroll
      for (int c = 0; c < CH; ++c)
        if (in[c]) v[u][c] = srt_ldg_keep(xr + c * 128);
    }
#pragma unroll
    for (int u = 0; u < H; ++u) rec_w<W>(wt + eb + u, w[u]);
  };
  auto comp = [&](float (&w)[H][4], float4 (&v)[H][CH]) {
#pragma unroll
    for (int u = 0; u < H; ++u)
#pragma unroll
      for (int c = 0; c < CH; ++c)
        if (in[c]) {
#pragma unroll
          for (int sg = 0; sg < 4; ++sg) fma4(acc[sym_slot(PS, PM, sg)][c], w[u][sg], v[u][c]);
        }
  };
  int e = e0;
  const int groups = (e1 - e0) / H;
  if (groups >= 2) {  // two groups alternate: one's gathers fly while the other computes
    load(e, oA, wA, vA);
    int gi = 1;
#pragma unroll 1
    for (; gi + 1 < groups; gi += 2) {
      load(e + gi * H, oB, wB, vB);
      comp(wA, vA);
      load(e + (gi + 1) * H, oA, wA, vA);
      comp(wB, vB);
    }
    if (gi < groups) {
      load(e + gi * H, oB, wB, vB);
      comp(wA, vA);
      comp(wB, vB);
    } else {
      comp(wA, vA);
    }
    e += groups * H;
  }
#pragma unroll 1
  for (; e < e1; ++e) {
    const float* xr = x0 + (int64_t)row_of(__ldg(A.key + e)) * ldx;
    float w[4];
    rec_w<W>(wt + e, w);
#pragma unroll
    for (int c = 0; c < CH; ++c)
      if (in[c]) {
        const float4 xv = srt_ldg_keep(xr + c * 128);
#pragma unroll
        for (int sg = 0; sg < 4; ++sg) fma4(acc[sym_slot(PS, PM, sg)][c], w[sg], xv);
      }
  }
}

// f[b][p][k] = sum_(J,l) A1[(J, l), p] F1[b][(J, l)][k] for the 2 x 2 pixel
// tile (ta, tb) with ta in [g0, g1); y points at pixel row 2 g0.
template <typename W, int CH>
__global__ void __launch_bounds__(256) k_a1t_tile(A1Args A, const W* __restrict__ wt,
                                                  const float* __restrict__ x, int ldx,
                                                  int64_t bsx, float* __restrict__ y, int ldy,
                                                  int64_t bsy, int ncols) {
  const int lane = threadIdx.x & 31;
  int ga, tb;
  if (!warp_tile(A, &ga, &tb)) return;
  const int ta = A.g0 + ga;
  const int n0 = blockIdx.y * (128 * CH) + lane * 4;
  const float* x0 = x + blockIdx.z * bsx + n0;
  bool in[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) in[c] = n0 + c * 128 < ncols;
  float2 acc[4][CH][2];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int c = 0; c < CH; ++c) acc[i][c][0] = acc[i][c][1] = make_float2(0.f, 0.f);
  a1t_pass<W, CH, 0, 0>(A, wt, ta, tb, x0, ldx, in, acc);
  if (A.mode == 2) a1t_pass<W, CH, 0, 1>(A, wt, ta, tb, x0, ldx, in, acc);
  if (A.mode) {
    a1t_pass<W, CH, 1, 0>(A, wt, ta, tb, x0, ldx, in, acc);
    if (A.mode == 2) a1t_pass<W, CH, 1, 1>(A, wt, ta, tb, x0, ldx, in, acc);
    a1t_pass<W, CH, 2, 0>(A, wt, ta, tb, x0, ldx, in, acc);
    if (A.mode == 2) a1t_pass<W, CH, 2, 1>(A, wt, ta, tb, x0, ldx, in, acc);
    a1t_pass<W, CH, 3, 0>(A, wt, ta, tb, x0, ldx, in, acc);
    if (A.mode == 2) a1t_pass<W, CH, 3, 1>(A, wt, ta, tb, x0, ldx, in, acc);
  }
  float* y0 = y + blockIdx.z * bsy;
#pragma unroll
  for (int sg = 0; sg < 4; ++sg) {
    const int ix = 2 * ga + (sg >> 1), iy = 2 * tb + (sg & 1);  // ix relative to row 2 g0
    float* yr = y0 + ((int64_t)ix * A.ms + iy) * ldy;
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      const int n = n0 + c * 128;
      if (n < ncols)
        *reinterpret_cast<float4*>(yr + n) =
            make_float4(acc[sg][c][0].x, acc[sg][c][0].y, acc[sg][c][1].x, acc[sg][c][1].y);
    }
  }
}

// ------------------------------------------------------------ records
struct TEnt {
  int64_t key;  // list << 40 | j << 16 | l
  int32_t slot;
  int64_t src;
};

template <typename T>
int upload(const std::vector<T>& h, T** d, int64_t* bytes) {
  SRT_TRY(srt_dmalloc(d, (int64_t)h.size(), bytes));
  if (!h.empty())
    SRT_CUDA_TRY(cudaMemcpy(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
  return SRT_OK;
}

}  // namespace

void srt_a1tiles_free(SrtA1Tiles* t) {
  cudaFree(t->aptr);
  cudaFree(t->akey);
  cudaFree(t->aw32);
  cudaFree(t->aw16);
  *t = SrtA1Tiles();
}

int srt_build_a1tiles(srt_plan_s* plan, int64_t* bytes) {
  const srt_geometry& g = plan->g;
  const SrtCsr& a = plan->a1;
  const int ms = g.ms, ne = g.n_ell, q = g.n_phi / 4;
  const int mode = plan->a1_rot;
  if (ms % 2 || ms >= (1 << 15) || ne >= (1 << 16)) return SRT_ERR_ARG;
  const int64_t ns = a.nnz;
  std::vector<int32_t> rp(a.rows + 1), cl(ns);
  std::vector<float> v32(a.v32 ? ns : 0);
  std::vector<uint16_t> v16(a.v16 ? ns : 0);
  SRT_CUDA_TRY(cudaMemcpy(rp.data(), a.rowptr, rp.size() * 4, cudaMemcpyDeviceToHost));
  if (ns) {
    SRT_CUDA_TRY(cudaMemcpy(cl.data(), a.col, ns * 4, cudaMemcpyDeviceToHost));
    if (a.v32) SRT_CUDA_TRY(cudaMemcpy(v32.data(), a.v32, ns * 4, cudaMemcpyDeviceToHost));
    if (a.v16) SRT_CUDA_TRY(cudaMemcpy(v16.data(), a.v16, ns * 2, cudaMemcpyDeviceToHost));
  }
  SrtA1Tiles& t = plan->a1tl;
  t.ntx = ms / 2;
  // A1^T: per 2 x 2 pixel tile, records (j, l) sorted by (list, j, l); list
  // B holds the mirror-fixed stored columns 0 and q/2 of the 8-fold form
  {
    const int64_t ntiles = (int64_t)t.ntx * t.ntx;
    std::vector<int64_t> cnt(ntiles + 1, 0);
    for (int64_t row = 0; row < a.rows; ++row)
      for (int64_t e = rp[row]; e < rp[row + 1]; ++e) {
        const int ix = cl[e] / ms, iy = cl[e] % ms;
        ++cnt[(int64_t)(ix / 2) * t.ntx + iy / 2 + 1];
      }
    for (int64_t i = 0; i < ntiles; ++i) cnt[i + 1] += cnt[i];
    std::vector<TEnt> ent(ns);
    std::vector<int64_t> at(cnt.begin(), cnt.end() - 1);
    for (int64_t row = 0; row < a.rows; ++row) {
      const int j = (int)(row / ne), l = (int)(row % ne);
      const int64_t list = (mode == 2 && (j == 0 || 2 * j == q)) ? 1 : 0;
      for (int64_t e = rp[row]; e < rp[row + 1]; ++e) {
        const int ix = cl[e] / ms, iy = cl[e] % ms;
        const int64_t tt = (int64_t)(ix / 2) * t.ntx + iy / 2;
        ent[at[tt]++] = TEnt{list << 40 | (int64_t)j << 16 | l, (ix & 1) * 2 + (iy & 1), e};
      }
    }
    std::vector<int32_t> ptr(2 * ntiles + 1), key;
    std::vector<float> w32;
    std::vector<uint16_t> w16;
    for (int64_t tt = 0; tt < ntiles; ++tt) {
      auto b0 = ent.begin() + cnt[tt], b1 = ent.begin() + cnt[tt + 1];
      std::stable_sort(b0, b1, [](const TEnt& x, const TEnt& y) { return x.key < y.key; });
      ptr[2 * tt] = (int32_t)key.size();
      ptr[2 * tt + 1] = -1;
      for (auto b = b0; b != b1;) {
        if ((b->key >> 40) && ptr[2 * tt + 1] < 0) ptr[2 * tt + 1] = (int32_t)key.size();
        float f[4] = {0.f, 0.f, 0.f, 0.f};
        uint16_t h[4] = {0, 0, 0, 0};
        auto c = b;
        for (; c != b1 && c->key == b->key; ++c) {
          if (!v32.empty()) f[c->slot] = v32[c->src];
          if (!v16.empty()) h[c->slot] = v16[c->src];
        }
        key.push_back((int32_t)(b->key & 0xffffffffll));
        if (!v32.empty()) w32.insert(w32.end(), f, f + 4);
        if (!v16.empty()) w16.insert(w16.end(), h, h + 4);
        b = c;
      }
      if (ptr[2 * tt + 1] < 0) ptr[2 * tt + 1] = (int32_t)key.size();
    }
    ptr.back() = (int32_t)key.size();
    if (key.size() >= ((size_t)1 << 31)) return SRT_ERR_GEOMETRY;
    t.na = (int64_t)key.size();
    SRT_TRY(upload(ptr, &t.aptr, bytes));
    SRT_TRY(upload(key, &t.akey, bytes));
    if (!w32.empty()) SRT_TRY(upload(w32, &t.aw32, bytes));
    if (!w16.empty()) SRT_TRY(upload(w16, &t.aw16, bytes));
  }
  return SRT_OK;
}

namespace {

template <typename W>
int launch_a1t(const A1Args& A, const W* w, const float* x, int64_t ldx, int64_t bsx, float* y,
               int64_t ldy, int64_t bsy, int ncols, int batch, cudaStream_t st) {
  const int TI = 8 / A.TG;
  int64_t gx;
  if (A.S > 0) {
    gx = (int64_t)((A.G + A.S - 1) / A.S) * ((A.R + A.S - 1) / A.S) * (A.S / A.TG) * (A.S / TI);
  } else {
    gx = (int64_t)((A.R + TI - 1) / TI) * ((A.G + A.TG - 1) / A.TG);
  }
  if (gx > 0x7fffffff || batch > 65535) return SRT_ERR_ARG;
  const int CH = ncols > 128 ? 2 : 1;
  dim3 grid((unsigned)gx, (ncols + 128 * CH - 1) / (128 * CH), batch);
  if (CH == 2)
    k_a1t_tile<W, 2><<<grid, 256, 0, st>>>(A, w, x, (int)ldx, bsx, y, (int)ldy, bsy, ncols);
  else
    k_a1t_tile<W, 1><<<grid, 256, 0, st>>>(A, w, x, (int)ldx, bsx, y, (int)ldy, bsy, ncols);
  SRT_CUDA_TRY(cudaGetLastError());
  return SRT_OK;
}

}  // namespace

int srt_a1tiles_apply(const srt_plan_s* plan, int g0, int g1, const float* x, int64_t ldx,
                      int64_t bsx, float* y, int64_t ldy, int64_t bsy, int ncols, int batch,
                      cudaStream_t st) {
  const srt_geometry& g = plan->g;
  const SrtA1Tiles& t = plan->a1tl;
  if (!t.aptr || ncols <= 0 || batch <= 0) return SRT_ERR_ARG;
  // float4 gathers and stores of 16-byte aligned rows
  if (ncols % 4 || ldx % 4 || ldy % 4 || bsx % 4 || bsy % 4 || (uintptr_t)x % 16 ||
      (uintptr_t)y % 16 || ldx > 0x7fffffff || ldy > 0x7fffffff)
    return SRT_ERR_ARG;
  if (g0 < 0 || g1 > t.ntx || g1 <= g0) return SRT_ERR_ARG;
  A1Args A{};
  A.ptr = t.aptr;
  A.key = t.akey;
  A.mode = plan->a1_rot;
  A.q = g.n_phi / 4;
  A.ms = g.ms;
  A.n_phi = g.n_phi;
  A.n_ell = g.n_ell;
  A.ntx = t.ntx;
  A.xrows = srt_checked_rows((int64_t)g.n_phi * g.n_ell);
  // tiles (ta, tb), ta in [g0, g1): blocks of 4 x 2 tiles (8 x 4 pixels)
  // walked in 16 x 16 tile (32 x 32 pixel) super-tiles where they fit, so
  // the rows gathered at any time belong to a compact patch (1.457 ms at
  // 256^3, against 1.483 with 32 x 32 tiles and 1.469 with none)
  A.g0 = g0;
  A.g1 = g1;
  A.G = g1 - g0;
  A.R = t.ntx;
  A.TG = 4;
  A.S = (A.G % 16 == 0 && A.R % 16 == 0) ? 16 : 0;
  if (g.weight_dtype == SRT_BF16) {
    const uint2* w = reinterpret_cast<const uint2*>(t.aw16);
    if (!w) return SRT_ERR_ARG;
    return launch_a1t<uint2>(A, w, x, ldx, bsx, y, ldy, bsy, ncols, batch, st);
  }
  const float4* w = reinterpret_cast<const float4*>(t.aw32);
  if (!w) return SRT_ERR_ARG;
  return launch_a1t<float4>(A, w, x, ldx, bsx, y, ldy, bsy, ncols, batch, st);
}

long long srt_checks_take_a1tiles() {
#ifdef SRT_CHECKS
  unsigned long long v = 0, z = 0;
  if (cudaMemcpyFromSymbol(&v, g_viol, sizeof(v)) != cudaSuccess) return -1;
  if (cudaMemcpyToSymbol(g_viol, &z, sizeof(z)) != cudaSuccess) return -1;
  return (long long)v;
#else
  return 0;
#endif
}
