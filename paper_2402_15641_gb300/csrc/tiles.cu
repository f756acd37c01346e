// Second product of Algorithms 1 and 2 (A2 Y1' and A2^T P') from 2 x 2
// register tiles of output rows.
//
// With the rings spaced like the slabs, A2[(h,m),(l,k)] = T[m, k - h - s, l]
// (Toeplitz in z, see toeplitz.cu).  A product that gives each output row its
// own warp reads one gathered dense row per entry, and each gathered operand
// feeds one FMA: the L1 data pipe, not the FMA pipe, then bounds the
// product.  Neighbouring rows share gathered rows: the semicircles of two
// consecutive radii about one ring cross many of the same (slab, radius-bin)
// cells, and so do the semicircles of one radius about two neighbouring
// rings, shifted by one slab.  Here a warp owns a 2 x 2 tile of output rows
//   forward: rings (c, c+1) x radii (2p, 2p+1)      rows (h, m) of A2
//   adjoint: slabs (c, c+1) x radius bins (2p, 2p+1) rows (l, k) of A2^T
// and walks the union of the four rows' gathered rows: one record per
// gathered row, holding the four weights (zero where a row does not use it)
// and the row's offset.  Each gathered operand then feeds four FMAs.  At
// 256^3 a record serves 1.88 entries on average in the forward and 2.0 in
// the adjoint (counted from T's taps), so the gathered bytes per FMA fall
// by that factor.
//
// Thanks to the Toeplitz structure the records depend only on the radius
// pair and on the gathered row's position relative to the tile (key):
//   forward: key delta = k - c (slab offset from the tile's first ring), the
//     record of (delta, l) holds w[i][j] = T[2p+j, q, l] with
//     q = delta - i + (n_zs - 1) - the column of T at offset k - (c+i) - s;
//     gathered row l*mz + c + delta.
//   adjoint: key gamma = h - c (ring offset from the tile's first slab), the
//     record of (gamma, m) holds w[i][j] = T[m, q, 2p+j] with
//     q = i - gamma + (n_zs - 1); gathered row (c + gamma)*n_ell + m.
// Records of one radius pair are sorted by (key, l) resp. (key, m), with a
// pointer per key, so the tile's gathered rows inside the volume (forward:
// 0 <= c + delta < mz; adjoint: 0 <= c + gamma < n_zs) are one contiguous
// range.  Each output row therefore sums its entries in the order of the
// taps kernel: ascending (offset, l) in the forward, ascending (h, m) (the
// CSR order of A2^T) in the adjoint; the padded zero weights add +0.
//
// The reshape that follows each product in Algorithms 1 and 2 (P2 after A2,
// P1^-1 after A2^T) can be folded into the product's epilogue (TR): the
// block's 8 x 4 tile of output rows x its dense columns is staged in shared
// memory and written in the layout the next step reads, column by column:
//   forward: p[n][h][m] (n = b n_phi + j), 4 consecutive radii per store;
//   adjoint: F1[n][l][k], 8 consecutive slabs per store (a 32-byte sector).
// The sums are the same, so the two forms agree bitwise.
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "devutil.cuh"

namespace {

#ifdef SRT_CHECKS
__device__ unsigned long long g_viol;  // gathered rows outside their operand
#endif

struct TileArgs {
  const int32_t* ptr;  // [pairs][nkeys + 1]: first record of each key
  const int32_t* off;  // [records]: gathered-row offset
  int nkeys, key0;     // key index = key + key0
  int E;               // keys of one tile: [-c, E - 1 - c]
  int c0, c1;          // tile coordinate range (forward: rings, adjoint: slabs)
  int n_ell, mz;
  int G, R, TG;        // block order: G coordinate pairs x R radius pairs
  int desc;            // radius chunks issued from the last one down
  int xrows;           // rows of the gathered operand (debug-build checks)
  int64_t ldn;         // fused reshape: stride of the output's columns n
};

template <typename W>
__device__ __forceinline__ void tile_w(const W* p, float w[4]);
template <>
__device__ __forceinline__ void tile_w<float4>(const float4* p, float w[4]) {
  const float4 v = __ldg(p);
  w[0] = v.x;
  w[1] = v.y;
  w[2] = v.z;
  w[3] = v.w;
}
template <>
__device__ __forceinline__ void tile_w<uint2>(const uint2* p, float w[4]) {
  const uint2 v = __ldg(p);  // four BF16 weights, w[0] in the low half of .x
  w[0] = __uint_as_float(v.x << 16);
  w[1] = __uint_as_float(v.x & 0xffff0000u);
  w[2] = __uint_as_float(v.y << 16);
  w[3] = __uint_as_float(v.y & 0xffff0000u);
}

// Radius chunk ch and coordinate tile t of this block.  Blocks are issued
// radius-chunk-major (all coordinate pairs advance through the radius
// chunks together, so the rows gathered at any time stay in L2), from the
// end of the radius range whose chunks hold more records: the last blocks
// to start are then the light ones, and the SMs finish together.
__device__ __forceinline__ void block_chunk(const TileArgs& A, int TG, int* ch, int* t) {
  const int TI = 8 / TG;
  const int tiles = (A.G + TG - 1) / TG;
  const int c = blockIdx.x / tiles;
  *t = blockIdx.x - c * tiles;
  *ch = A.desc ? (A.R + TI - 1) / TI - 1 - c : c;
}

// Tile of this warp: a block owns TG coordinate pairs x 8/TG radius pairs.
__device__ __forceinline__ bool tile_of(const TileArgs& A, int* g, int* r) {
  const int w = threadIdx.x >> 5;
  const int TI = 8 / A.TG;
  int ch, t;
  block_chunk(A, A.TG, &ch, &t);
  *g = t * A.TG + w / TI;
  *r = ch * TI + w % TI;
  return *g < A.G && *r < A.R;
}

// acc (two float2: columns n..n+3) += w * xv, as two packed FP32 FMAs (each
// lane of a packed FMA rounds exactly as fmaf does)
__device__ __forceinline__ void fma4(float2 (&a)[2], float w, const float4& xv) {
  const float2 ww = make_float2(w, w);
  a[0] = __ffma2_rn(ww, make_float2(xv.x, xv.y), a[0]);
  a[1] = __ffma2_rn(ww, make_float2(xv.z, xv.w), a[1]);
}

// Records per group of the main loop.  The product waits on its gathers (L2
// latency), so a warp alternates two groups: it requests the next group's
// gathered rows before the FMAs of the current one, and its gathers stay in
// flight while it computes.  At 128 registers and 16 warps per SM, groups
// of three were fastest at 256^3 (A2 2.09 ms, A2^T 1.94 ms; a single group
// of six whose FMAs wait for all its gathers: 2.24 / 2.06 ms; two groups
// of two or of four: 3.20 / 3.29 and 3.60 / 4.20 ms; one record at a time,
// 60 registers and 32 warps: 2.77 / 2.59 ms).
constexpr int kTileH = 3;

// Lanes own 4 consecutive dense columns of each of CH 128-column chunks.
// TR: the block's outputs go through shared memory to the reshaped layout
// (blocks of TG = 4 coordinate pairs x 2 radius pairs only).
template <typename W, bool ADJ, int CH, bool TR>
__global__ void __launch_bounds__(256) k_tile22(TileArgs A, const W* __restrict__ wt,
                                                const float* __restrict__ x, int ldx,
                                                float* __restrict__ y, int64_t ldy, int ncols) {
  const int lane = threadIdx.x & 31;
  int g, r;
  const bool mine = tile_of(A, &g, &r);
  if (!TR && !mine) return;  // (TR: every warp reaches the block barrier)
  const int c = A.c0 + 2 * g;
  const int n0 = blockIdx.y * (128 * CH) + lane * 4;
  bool in[CH];
#pragma unroll
  for (int q = 0; q < CH; ++q) in[q] = n0 + q * 128 < ncols;
  float2 acc[4][CH][2];
#pragma unroll
  for (int s = 0; s < 4; ++s)
#pragma unroll
    for (int q = 0; q < CH; ++q) acc[s][q][0] = acc[s][q][1] = make_float2(0.f, 0.f);
  if (mine) {
    const int32_t* pp = A.ptr + (int64_t)r * (A.nkeys + 1) + (A.key0 - c);
    const int e0 = pp[0], e1 = pp[A.E];
    const int64_t xb = ADJ ? (int64_t)c * A.n_ell : (int64_t)c;
    const float* x0 = x + xb * ldx + n0;
    constexpr int H = kTileH;
    int oA[H], oB[H];
    float wA[H][4], wB[H][4];
    float4 vA[H][CH], vB[H][CH];
    // group of records eb .. eb + H - 1: offsets, gathered rows, weights
    auto load = [&](int eb, int (&o)[H], float (&w)[H][4], float4 (&v)[H][CH]) {
#pragma unroll
      for (int u = 0; u < H; ++u) {
        o[u] = __ldg(A.off + eb + u);
        SRT_CHECK_GATHER(xb, o[u], A.xrows, g_viol);
      }
#pragma unroll
      for (int u = 0; u < H; ++u) {
        const float* xr = x0 + (int64_t)o[u] * ldx;
#pragma unroll
        for (int q = 0; q < CH; ++q)
          if (in[q]) v[u][q] = srt_ldg_keep(xr + q * 128);
      }
#pragma unroll
      for (int u = 0; u < H; ++u) tile_w<W>(wt + eb + u, w[u]);
    };
    // its FMAs, record by record (the rows' summation order)
    auto comp = [&](float (&w)[H][4], float4 (&v)[H][CH]) {
#pragma unroll
      for (int u = 0; u < H; ++u)
#pragma unroll
        for (int q = 0; q < CH; ++q)
          if (in[q]) {
#pragma unroll
            for (int s = 0; s < 4; ++s) fma4(acc[s][q], w[u][s], v[u][q]);
          }
    };
    int e = e0;
    const int groups = (e1 - e0) / H;
    if (groups >= 2) {
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
      int o = __ldg(A.off + e);
      SRT_CHECK_GATHER(xb, o, A.xrows, g_viol);
      float w[4];
      tile_w<W>(wt + e, w);
      const float* xr = x0 + (int64_t)o * ldx;
#pragma unroll
      for (int q = 0; q < CH; ++q)
        if (in[q]) {
          const float4 xv = srt_ldg_keep(xr + q * 128);
#pragma unroll
          for (int s = 0; s < 4; ++s) fma4(acc[s][q], w[s], xv);
        }
    }
  }
  if (!TR) {
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const int i = s >> 1, j = s & 1;
      if (c + i >= A.c1 || 2 * r + j >= A.n_ell) continue;
      const int64_t row = ADJ ? (int64_t)(2 * r + j) * A.mz + c + i
                              : (int64_t)(c - A.c0 + i) * A.n_ell + 2 * r + j;
      float* yr = y + row * ldy;
#pragma unroll
      for (int q = 0; q < CH; ++q) {
        const int n = n0 + q * 128;
        if (n < ncols)
          *reinterpret_cast<float4*>(yr + n) =
              make_float4(acc[s][q][0].x, acc[s][q][0].y, acc[s][q][1].x, acc[s][q][1].y);
      }
    }
    return;
  }
  // fused reshape, 64 columns at a time (8 KB of shared memory, so that the
  // L1 left for the gathers barely shrinks): S[cl][rl][n], cl = the block's
  // coordinate 0..7 (ring or slab), rl = its radius 0..3 (radius or bin)
  __shared__ __align__(16) float S[8 * 4 * 64];
  const int w = threadIdx.x >> 5;
  int ch, t;
  block_chunk(A, 4, &ch, &t);
  const int cb = A.c0 + 8 * t, rb = 4 * ch;  // the block's first coordinate and radius
#pragma unroll
  for (int pass = 0; pass < 2 * CH; ++pass) {
    const int q = pass >> 1, half = pass & 1;
    if (pass) __syncthreads();  // the previous pass's reads are done
    if ((lane >> 4) == half) {
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const int cl = 2 * (w >> 1) + (s >> 1), rl = 2 * (w & 1) + (s & 1);
        *reinterpret_cast<float4*>(S + (cl * 4 + rl) * 64 + (lane & 15) * 4) =
            make_float4(acc[s][q][0].x, acc[s][q][0].y, acc[s][q][1].x, acc[s][q][1].y);
      }
    }
    __syncthreads();
    const int nb0 = blockIdx.y * (128 * CH) + q * 128 + half * 64;
    if (!ADJ) {
      // p[n][h][m]: per (ring, column) the 4 radii rb .. rb + 3
#pragma unroll
      for (int it = threadIdx.x; it < 8 * 64; it += 256) {
        const int cl = it >> 6, nl = it & 63, n = nb0 + nl, h = cb + cl;
        if (h >= A.c1 || n >= ncols) continue;
        const int64_t o = (int64_t)n * A.ldn + (int64_t)h * A.n_ell + rb;
        const float* sp = S + cl * 4 * 64 + nl;
        if (rb + 3 < A.n_ell && (o & 3) == 0) {
          *reinterpret_cast<float4*>(y + o) = make_float4(sp[0], sp[64], sp[128], sp[192]);
        } else {
          for (int k = 0; k < 4 && rb + k < A.n_ell; ++k) y[o + k] = sp[k * 64];
        }
      }
    } else {
      // F1[n][l][k]: per (radius bin, column) the 8 slabs cb .. cb + 7
      const int rl = threadIdx.x >> 6, nl = threadIdx.x & 63, n = nb0 + nl, l = rb + rl;
      if (l < A.n_ell && n < ncols) {
        const int64_t o = (int64_t)n * A.ldn + (int64_t)l * A.mz + cb;
        const float* sp = S + rl * 64 + nl;
        if (cb + 7 < A.c1 && (o & 3) == 0) {
          *reinterpret_cast<float4*>(y + o) =
              make_float4(sp[0], sp[256], sp[512], sp[768]);
          *reinterpret_cast<float4*>(y + o + 4) =
              make_float4(sp[1024], sp[1280], sp[1536], sp[1792]);
        } else {
          for (int k = 0; k < 8 && cb + k < A.c1; ++k) y[o + k] = sp[k * 256];
        }
      }
    }
  }
}

template <typename W, bool ADJ>
int launch(const TileArgs& A, const W* w, const float* x, int ldx, float* y, int64_t ldy,
           int ncols, cudaStream_t st) {
  const int TI = 8 / A.TG;
  const int64_t gx = (int64_t)((A.R + TI - 1) / TI) * ((A.G + A.TG - 1) / A.TG);
  if (gx > 0x7fffffff) return SRT_ERR_ARG;
  const int CH = ncols > 128 ? 2 : 1;
  dim3 grid((unsigned)gx, (ncols + 128 * CH - 1) / (128 * CH), 1);
  if (A.ldn > 0) {
    if (CH == 2)
      k_tile22<W, ADJ, 2, true><<<grid, 256, 0, st>>>(A, w, x, ldx, y, ldy, ncols);
    else
      k_tile22<W, ADJ, 1, true><<<grid, 256, 0, st>>>(A, w, x, ldx, y, ldy, ncols);
  } else if (CH == 2) {
    k_tile22<W, ADJ, 2, false><<<grid, 256, 0, st>>>(A, w, x, ldx, y, ldy, ncols);
  } else {
    k_tile22<W, ADJ, 1, false><<<grid, 256, 0, st>>>(A, w, x, ldx, y, ldy, ncols);
  }
  SRT_CUDA_TRY(cudaGetLastError());
  return SRT_OK;
}

// One direction's records from T (host arrays: rows m, columns l*D + q).
// For each radius pair, entries (key index, l or m, slot i*2 + j, weight)
// are sorted by (key index, l or m) and merged into records.
struct Ent {
  int64_t key;   // key index * n_ell + (l or m)
  int32_t slot;  // i * 2 + j
  int64_t src;   // index of the tap in T
};

int build_dir(const srt_plan_s* plan, bool adj, const std::vector<int32_t>& rp,
              const std::vector<int32_t>& col, const std::vector<float>& v32,
              const std::vector<uint16_t>& v16, SrtTiles* t, int64_t* bytes) {
  const srt_geometry& g = plan->g;
  const int mz = g.mz, nz = g.n_zs, n_ell = g.n_ell, D = mz + nz - 1;
  const int pairs = (n_ell + 1) / 2, nkeys = mz + nz;
  const int key0 = adj ? mz - 1 : nz - 1;
  // taps of T (index, row m) by radius pair: forward pairs of rows m,
  // adjoint pairs of radius bins l
  std::vector<std::vector<std::pair<int64_t, int>>> by(pairs);
  for (int m = 0; m < n_ell; ++m)
    for (int e = rp[m]; e < rp[m + 1]; ++e) by[(adj ? col[e] / D : m) / 2].push_back({e, m});
  std::vector<int32_t> ptr((int64_t)pairs * (nkeys + 1)), off;
  std::vector<float> w32;
  std::vector<uint16_t> w16;
  std::vector<Ent> ent;
  for (int p = 0; p < pairs; ++p) {
    ent.clear();
    for (const auto& em : by[p]) {
      const int64_t e = em.first;
      const int m = em.second;
      const int l = col[e] / D, q = col[e] % D;
      const int j = (adj ? l : m) & 1;
      for (int i = 0; i < 2; ++i) {
        // forward: delta = q - (nz - 1) + i; adjoint: gamma = i + nz - 1 - q
        const int key = adj ? i + nz - 1 - q : q - (nz - 1) + i;
        const int ki = key + key0;
        ent.push_back(Ent{(int64_t)ki * n_ell + (adj ? m : l), i * 2 + j, e});
      }
    }
    std::stable_sort(ent.begin(), ent.end(),
                     [](const Ent& a, const Ent& b) { return a.key < b.key; });
    int32_t* pk = ptr.data() + (int64_t)p * (nkeys + 1);
    int next_key = 0;
    for (size_t a = 0; a < ent.size();) {
      const int ki = (int)(ent[a].key / n_ell), idx = (int)(ent[a].key % n_ell);
      while (next_key <= ki) pk[next_key++] = (int32_t)off.size();
      const int key = ki - key0;
      off.push_back(adj ? key * n_ell + idx : idx * mz + key);
      float f[4] = {0.f, 0.f, 0.f, 0.f};
      uint16_t h[4] = {0, 0, 0, 0};
      size_t b = a;
      for (; b < ent.size() && ent[b].key == ent[a].key; ++b) {
        if (!v32.empty()) f[ent[b].slot] = v32[ent[b].src];
        if (!v16.empty()) h[ent[b].slot] = v16[ent[b].src];
      }
      if (!v32.empty()) w32.insert(w32.end(), f, f + 4);
      if (!v16.empty()) w16.insert(w16.end(), h, h + 4);
      a = b;
    }
    while (next_key <= nkeys) pk[next_key++] = (int32_t)off.size();
  }
  if (off.size() >= ((size_t)1 << 31)) return SRT_ERR_GEOMETRY;
  // Issue order: the heavier end of the radius range first (a tile's time
  // follows its record count; the forward's records grow with the radius
  // until the semicircle reaches the largest ring-to-slab offset, the
  // adjoint's fall from the first radius bins on).  Compared over the first
  // and last eighth of the radius pairs.
  {
    const int e = std::max(1, pairs / 8);
    int64_t lo = 0, hi = 0;
    for (int p = 0; p < e; ++p) {
      lo += ptr[(int64_t)p * (nkeys + 1) + nkeys] - ptr[(int64_t)p * (nkeys + 1)];
      const int q = pairs - 1 - p;
      hi += ptr[(int64_t)q * (nkeys + 1) + nkeys] - ptr[(int64_t)q * (nkeys + 1)];
    }
    t->desc = hi > lo;
  }
  t->pairs = pairs;
  t->nkeys = nkeys;
  t->key0 = key0;
  t->nrec = (int64_t)off.size();
  SRT_TRY(srt_dmalloc(&t->ptr, (int64_t)ptr.size(), bytes));
  SRT_TRY(srt_dmalloc(&t->off, t->nrec, bytes));
  SRT_CUDA_TRY(cudaMemcpy(t->ptr, ptr.data(), ptr.size() * 4, cudaMemcpyHostToDevice));
  if (t->nrec) SRT_CUDA_TRY(cudaMemcpy(t->off, off.data(), off.size() * 4, cudaMemcpyHostToDevice));
  if (!w32.empty()) {
    SRT_TRY(srt_dmalloc(&t->w32, 4 * t->nrec, bytes));
    SRT_CUDA_TRY(cudaMemcpy(t->w32, w32.data(), w32.size() * 4, cudaMemcpyHostToDevice));
  }
  if (!w16.empty()) {
    SRT_TRY(srt_dmalloc(&t->w16, 4 * t->nrec, bytes));
    SRT_CUDA_TRY(cudaMemcpy(t->w16, w16.data(), w16.size() * 2, cudaMemcpyHostToDevice));
  }
  return SRT_OK;
}

}  // namespace

void srt_tiles_free(SrtTiles* t) {
  cudaFree(t->ptr);
  cudaFree(t->off);
  cudaFree(t->w32);
  cudaFree(t->w16);
  *t = SrtTiles();
}

int srt_build_tiles(srt_plan_s* plan, const std::vector<int32_t>& rp,
                    const std::vector<int32_t>& col, const std::vector<float>& v32,
                    const std::vector<uint16_t>& v16, int64_t* bytes) {
  SRT_TRY(build_dir(plan, false, rp, col, v32, v16, &plan->tlf, bytes));
  SRT_TRY(build_dir(plan, true, rp, col, v32, v16, &plan->tla, bytes));
  return SRT_OK;
}

int srt_tiles_apply(const srt_plan_s* plan, bool adjoint, int c0, int c1, int TG, const float* x,
                    int64_t ldx, float* y, int64_t ldy, int ncols, cudaStream_t st, int64_t ldn) {
  const srt_geometry& g = plan->g;
  const SrtTiles& t = adjoint ? plan->tla : plan->tlf;
  // float4 gathers and stores: 16-byte aligned rows of whole float4s
  if (!t.ptr || c1 <= c0 || ncols <= 0 || ncols % 4 || ldx % 4 || (ldn <= 0 && ldy % 4) ||
      (uintptr_t)x % 16 || (uintptr_t)y % 16 || ldx > 0x7fffffff || ldn < 0)
    return SRT_ERR_ARG;
  if (TG != 1 && TG != 2 && TG != 4 && TG != 8) TG = 4;
  if (ldn > 0) TG = 4;  // the fused reshape stages blocks of 8 x 4 output rows
  TileArgs A{t.ptr, t.off, t.nkeys, t.key0, adjoint ? g.n_zs : g.mz, c0, c1, g.n_ell, g.mz,
             (c1 - c0 + 1) / 2, t.pairs, TG, t.desc ? 1 : 0,
             srt_checked_rows(adjoint ? (int64_t)g.n_zs * g.n_ell : (int64_t)g.n_ell * g.mz),
             ldn};
  if (g.weight_dtype == SRT_BF16) {
    if (!t.w16) return SRT_ERR_ARG;
    const uint2* w = reinterpret_cast<const uint2*>(t.w16);
    return adjoint ? launch<uint2, true>(A, w, x, (int)ldx, y, ldy, ncols, st)
                   : launch<uint2, false>(A, w, x, (int)ldx, y, ldy, ncols, st);
  }
  if (!t.w32) return SRT_ERR_ARG;
  const float4* w = reinterpret_cast<const float4*>(t.w32);
  return adjoint ? launch<float4, true>(A, w, x, (int)ldx, y, ldy, ncols, st)
                 : launch<float4, false>(A, w, x, (int)ldx, y, ldy, ncols, st);
}

long long srt_checks_take_tiles() {
#ifdef SRT_CHECKS
  unsigned long long v = 0, z = 0;
  if (cudaMemcpyFromSymbol(&v, g_viol, sizeof(v)) != cudaSuccess) return -1;
  if (cudaMemcpyToSymbol(g_viol, &z, sizeof(z)) != cudaSuccess) return -1;
  return (long long)v;
#else
  return 0;
#endif
}
