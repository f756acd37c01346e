// Assembly of the two circular-Radon-transform matrices (Sec. 3.1 of the
// paper) and of their transposes for the matched adjoint (Sec. 3.2).
//
// A1 = A^{1,2}: row r = j*n_ell + l is the circle of sensor column j
//   (centre (R cos phi_j, R sin phi_j)) with bin-centre radius rho_l; column
//   p = ix*ms + iy is a pixel; the entry is the exact arc length of the circle
//   inside the pixel (in-plane CRT, measure rho da, Sec. 2).
// A2 = A^{3,4}: row r = h*n_ell + m is the semicircle of ring h (centre
//   (z_h, 0) in the (z, rho) half plane) with radius l_m; column c = l*mz + k
//   is the cell slab k x radius bin l; the entry is the exact arc length of
//   the semicircle inside the cell (vertical CRT, measure l dt, Sec. 2).
//   Every cell has rho >= ell_lo > 0, so the full circle's lower half never
//   meets a cell and the full-circle arc length equals the semicircle's.
//   With SRT_RHO_LINEAR the intermediate is piecewise linear in rho (the basis
//   remark of Sec. 3.1): column c = l*mz + k is node l's hat on slab k and the
//   entry is the hat integrated along the semicircle there (hat_weight); A1 is
//   unchanged (its circles sit at the nodes).
//
// Lengths are computed in FP64 (srt_arc_in_rect), rounded once to the stored
// type.  Rows are enumerated strip by strip (pixel columns for A1, radius bins
// for A2): in each strip the circle's two branches cover a range of the other
// index, widened by one cell each side, and every candidate's exact length is
// computed; lengths <= 1e-12 x spacing are dropped (tangent touches).  The
// count pass and the fill pass run the same enumeration, so they agree.
#include <string.h>

#include <vector>

#include "common.cuh"
#include "devutil.cuh"

namespace {

constexpr unsigned FULL = 0xffffffffu;

struct GeomDev {
  int ms, mz, n_phi, n_zs, n_ell;
  int nj;       // sensor columns whose A1 rows are assembled (the first nj of n_phi)
  int jfirst, ntot;  // column j sits at angle phi0 + 2 pi (jfirst + j) / ntot
  int rho_lin;  // A2 columns are hats of the radius nodes (else bins)
  int vox_lin;  // A1 columns are bilinear hats of the voxel centres (else pixels)
  double dxy, dz, radius, phi0, zs_lo, zs_hi, ell_lo, ell_hi;
  double hx, hz, dl, thr1, thr2;
};

GeomDev make_geom(const srt_geometry& g) {
  GeomDev G;
  G.ms = g.ms;
  G.mz = g.mz;
  G.n_phi = g.n_phi;
  G.nj = g.n_phi;
  G.jfirst = g.n_phi_total > 0 ? g.phi_first : 0;
  G.ntot = g.n_phi_total > 0 ? g.n_phi_total : g.n_phi;
  G.rho_lin = (g.flags & SRT_RHO_LINEAR) ? 1 : 0;
  G.vox_lin = (g.flags & SRT_VOXEL_LINEAR) ? 1 : 0;
  G.n_zs = g.n_zs;
  G.n_ell = g.n_ell;
  G.dxy = g.dxy;
  G.dz = g.dz;
  G.radius = g.radius;
  G.phi0 = g.phi0;
  G.zs_lo = g.zs_lo;
  G.zs_hi = g.zs_hi;
  G.ell_lo = g.ell_lo;
  G.ell_hi = g.ell_hi;
  G.hx = 0.5 * g.ms * g.dxy;
  G.hz = 0.5 * g.mz * g.dz;
  G.dl = (g.ell_hi - g.ell_lo) / g.n_ell;
  G.thr1 = 1e-12 * g.dxy;
  G.thr2 = 1e-12 * fmin(g.dz, G.dl);
  return G;
}

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// Pixel/slab index range [lo, hi] covering the coordinate interval [a, b]
// (origin at -half, spacing d), widened by one each side and clamped.
__device__ __forceinline__ void cover(double a, double b, double half, double d, int n, int& lo,
                                      int& hi) {
  lo = clampi((int)floor((a + half) / d) - 1, 0, n - 1);
  hi = clampi((int)floor((b + half) / d) + 1, 0, n - 1);
}

// Piecewise-linear intermediate: the hat of radius node l (linear between
// the nodes rho_i = ell_lo + (i + 1/2) dl, constant from ell_lo to rho_0 and
// from rho_{n-1} to ell_hi) integrated along the (z, rho) semicircle of centre
// (zc, 0) and radius r inside the slab [c0, c1].  On [rho_a, rho_b] = [rho_{l-1},
// rho_l] the hat is (rho - rho_a)/dl, so its integral is (M - rho_a L)/dl with L
// the arc length and M = int rho ds there; likewise (rho_b L - M)/dl above.
__device__ double hat_weight(const GeomDev& G, double zc, double r, int l, double c0, double c1) {
  const double rl = G.ell_lo + (l + 0.5) * G.dl;
  double w = 0.0, m = 0.0;
  if (l == 0) {
    w += srt_arc_in_rect(zc, 0.0, r, c0, c1, G.ell_lo, rl);
  } else {
    const double ra = G.ell_lo + (l - 0.5) * G.dl;
    const double len = srt_arc_in_rect_m(zc, 0.0, r, c0, c1, ra, rl, &m);
    w += (m - ra * len) / G.dl;
  }
  if (l == G.n_ell - 1) {
    w += srt_arc_in_rect(zc, 0.0, r, c0, c1, rl, G.ell_hi);
  } else {
    const double rb = G.ell_lo + (l + 1.5) * G.dl;
    const double len = srt_arc_in_rect_m(zc, 0.0, r, c0, c1, rl, rb, &m);
    w += (rb * len - m) / G.dl;
  }
  return w;
}

// Piecewise-linear voxels: node (i, k) at the voxel centre (x_i, y_k) has the
// basis (1 + bx (x - x_i))(1 + by (y - y_k)) on each of the four boxes of its
// support, bx = 1/dxy below the node and -1/dxy above it; at the volume's
// edge the outer half voxel holds the edge node's value (basis 1, bx = 0).
// The weight is the basis integrated along the circle (centre (cx, cy),
// radius r) over those boxes, in coordinates centred on the node.
__device__ double node_weight(const GeomDev& G, double cx, double cy, double r, int i, int k) {
  const double d = G.dxy;
  const double xn = -G.hx + (i + 0.5) * d, yn = -G.hx + (k + 0.5) * d;
  const double cxr = cx - xn, cyr = cy - yn;
  double w = 0.0;
  for (int p = 0; p < 2; ++p) {
    const bool edge_x = p == 0 ? i == 0 : i == G.ms - 1;
    const double xa = p == 0 ? (edge_x ? -0.5 * d : -d) : 0.0;
    const double xb = p == 0 ? 0.0 : (edge_x ? 0.5 * d : d);
    const double bx = edge_x ? 0.0 : (p == 0 ? 1.0 / d : -1.0 / d);
    for (int q = 0; q < 2; ++q) {
      const bool edge_y = q == 0 ? k == 0 : k == G.ms - 1;
      const double ya = q == 0 ? (edge_y ? -0.5 * d : -d) : 0.0;
      const double yb = q == 0 ? 0.0 : (edge_y ? 0.5 * d : d);
      const double by = edge_y ? 0.0 : (q == 0 ? 1.0 / d : -1.0 / d);
      w += srt_arc_bilinear(cxr, cyr, r, xa, xb, ya, yb, bx, by);
    }
  }
  return w;
}

// Enumerate one strip.  The strip spans [s0, s1] along the strip axis; the
// circle (centre (cu, cv) in (strip axis, cross axis), radius r) has two
// branches over it.  For every candidate cross index q (ascending) the exact
// length inside the cell is computed; f(q, w) is called for w > thr.
// Returns the number of kept entries; *drop counts 0 < w <= thr.
template <bool A1, class F>
__device__ int strip_enum(const GeomDev& G, double cu, double cv, double r, int s, int& drop, F f) {
  double s0, s1, half, d;
  int n;
  if (A1 && !G.vox_lin) {  // strip = pixel column ix, cross axis = y
    s0 = -G.hx + s * G.dxy;
    s1 = -G.hx + (s + 1) * G.dxy;
    half = G.hx;
    d = G.dxy;
    n = G.ms;
  } else if (A1) {  // strip = support of node column i (half a voxel at the edges)
    s0 = s == 0 ? -G.hx : -G.hx + (s - 0.5) * G.dxy;
    s1 = s == G.ms - 1 ? G.hx : -G.hx + (s + 1.5) * G.dxy;
    half = G.hx;
    d = G.dxy;
    n = G.ms;
  } else if (!G.rho_lin) {  // strip = radius bin l, cross axis = z
    s0 = G.ell_lo + s * G.dl;
    s1 = G.ell_lo + (s + 1) * G.dl;
    half = G.hz;
    d = G.dz;
    n = G.mz;
  } else {  // strip = support of node l's hat
    s0 = s == 0 ? G.ell_lo : G.ell_lo + (s - 0.5) * G.dl;
    s1 = s == G.n_ell - 1 ? G.ell_hi : G.ell_lo + (s + 1.5) * G.dl;
    half = G.hz;
    d = G.dz;
    n = G.mz;
  }
  const double u0 = s0 - cu, u1 = s1 - cu;
  const double umin = (u0 <= 0.0 && u1 >= 0.0) ? 0.0 : fmin(fabs(u0), fabs(u1));
  const double umax = fmax(fabs(u0), fabs(u1));
  if (umin >= r) return 0;
  const double thi = sqrt((r - umin) * (r + umin));
  const double tlo = umax >= r ? 0.0 : sqrt((r - umax) * (r + umax));
  int a0, a1, b0, b1;
  cover(cv - thi, cv - tlo, half, d, n, a0, a1);
  cover(cv + tlo, cv + thi, half, d, n, b0, b1);
  if (A1 && G.vox_lin) {  // node supports reach a voxel further down
    a0 = a0 > 0 ? a0 - 1 : 0;
    b0 = b0 > 0 ? b0 - 1 : 0;
  }
  if (b0 <= a1) b0 = a1 + 1;  // union, ascending
  const double thr = A1 ? G.thr1 : G.thr2;
  int kept = 0;
  for (int pass = 0; pass < 2; ++pass) {
    const int q0 = pass ? b0 : a0, q1 = pass ? b1 : a1;
    for (int q = q0; q <= q1; ++q) {
      const double c0 = -half + q * d, c1 = -half + (q + 1) * d;
      double w;
      if (A1 && G.vox_lin)
        w = node_weight(G, cu, cv, r, s, q);
      else if (A1)
        w = srt_arc_in_rect(cu, cv, r, s0, s1, c0, c1);
      else if (!G.rho_lin)  // (z, rho) plane: x = z, y = rho
        w = srt_arc_in_rect(cv, cu, r, c0, c1, s0, s1);
      else
        w = hat_weight(G, cv, r, s, c0, c1);
      if (w > thr) {
        f(q, w, kept);
        ++kept;
      } else if (w > 0.0) {
        ++drop;
      }
    }
  }
  return kept;
}

// One warp per row.  pass 0: counts[row] = entries, drops summed into *dropped.
// pass 1: write (column, FP64 length) at rowptr[row] in ascending column order.
template <bool A1>
__global__ void __launch_bounds__(256) k_assemble(GeomDev G, int rows, int pass,
                                                  int32_t* __restrict__ counts,
                                                  const int32_t* __restrict__ rowptr,
                                                  int32_t* __restrict__ col,
                                                  double* __restrict__ val,
                                                  unsigned long long* __restrict__ dropped) {
  const int lane = threadIdx.x & 31;
  const int row = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  if (row >= rows) return;  // warp-uniform
  double cu, cv, r;
  const int nstrips = A1 ? G.ms : G.n_ell;
  if (A1) {
    const int j = row / G.n_ell, l = row % G.n_ell;
    const double phi = G.phi0 + 2.0 * SRT_PI * (G.jfirst + j) / G.ntot;
    cu = G.radius * cos(phi);  // x of the sensor column (strip axis)
    cv = G.radius * sin(phi);  // y
    r = G.ell_lo + (l + 0.5) * G.dl;
  } else {
    const int h = row / G.n_ell, m = row % G.n_ell;
    cu = 0.0;                                                   // rho of the centre
    cv = G.zs_lo + (h + 0.5) * (G.zs_hi - G.zs_lo) / G.n_zs;    // z of the centre
    r = G.ell_lo + (m + 0.5) * G.dl;
  }
  const int64_t base = pass ? rowptr[row] : 0;
  const int64_t end = pass ? rowptr[row + 1] : 0;
  const int stride = A1 ? G.ms : G.mz;
  int total = 0, drop = 0, dummy = 0;
  // One emitter for the count and the fill, so both run the same code.
  bool write = false;
  int64_t at = 0;
  int strip = 0;
  auto emit = [&](int q, double w, int i) {
    if (write && at + i < end) {
      col[at + i] = strip * stride + q;
      val[at + i] = w;
    }
  };
  for (int s0 = 0; s0 < nstrips; s0 += 32) {
    strip = s0 + lane;
    int cnt = 0;
    write = false;
    if (strip < nstrips) cnt = strip_enum<A1>(G, cu, cv, r, strip, pass ? dummy : drop, emit);
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(FULL, incl, o);
      if (lane >= o) incl += v;
    }
    if (pass && cnt > 0) {
      at = base + total + (incl - cnt);
      write = true;
      strip_enum<A1>(G, cu, cv, r, strip, dummy, emit);
    }
    total += __shfl_sync(FULL, incl, 31);
  }
  if (!pass) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) drop += __shfl_xor_sync(FULL, drop, o);
    if (lane == 0) {
      counts[row] = total;
      if (drop) atomicAdd(dropped, (unsigned long long)drop);
    }
  }
}

// Expand the master tensor T (one ring over D = mz + n_zs - 1 slab offsets:
// rows m, columns l*D + q) into A2's rows (h, m): entry (l, k) with slab
// k = h + q - (n_zs - 1) when 0 <= k < mz.  One warp per row; order and
// values are kept, so A2 holds T's entries bitwise.
__global__ void __launch_bounds__(256) k_expand_toeplitz(int mz, int n_zs, int n_ell, int rows,
                                                         int pass,
                                                         const int32_t* __restrict__ tptr,
                                                         const int32_t* __restrict__ tcol,
                                                         const float* __restrict__ t32,
                                                         const uint16_t* __restrict__ t16,
                                                         const double* __restrict__ t64,
                                                         int32_t* __restrict__ counts,
                                                         const int32_t* __restrict__ rowptr,
                                                         int32_t* __restrict__ col,
                                                         float* __restrict__ v32,
                                                         uint16_t* __restrict__ v16,
                                                         double* __restrict__ v64) {
  const int lane = threadIdx.x & 31;
  const int row = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  if (row >= rows) return;
  const int h = row / n_ell, m = row % n_ell;
  const int D = mz + n_zs - 1;
  const int e0 = tptr[m], e1 = tptr[m + 1];
  int total = 0;
  const int64_t base = pass ? rowptr[row] : 0;
  for (int eb = e0; eb < e1; eb += 32) {
    const int e = eb + lane;
    bool keep = false;
    int c = 0;
    if (e < e1) {
      const int cc = tcol[e];
      const int l = cc / D, k = h + (cc % D) - (n_zs - 1);
      keep = k >= 0 && k < mz;
      c = l * mz + k;
    }
    const unsigned bal = __ballot_sync(FULL, keep);
    if (pass && keep) {
      const int64_t at = base + total + __popc(bal & ((1u << lane) - 1));
      col[at] = c;
      if (v32) v32[at] = t32[e];
      if (v16) v16[at] = t16[e];
      if (v64) v64[at] = t64[e];
    }
    total += __popc(bal);
  }
  if (!pass && lane == 0) counts[row] = total;
}

// Exclusive scan of n int32 counts into out[0..n] (out[n] = total) with a
// 64-bit running sum; *total receives the exact 64-bit total.  One block.
__global__ void __launch_bounds__(1024) k_scan(const int32_t* __restrict__ in,
                                               int32_t* __restrict__ out, int64_t n,
                                               long long* __restrict__ total) {
  constexpr int ITEMS = 8;
  __shared__ long long warp_sum[32];
  __shared__ long long carry;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < n; base += 1024 * ITEMS) {
    long long v[ITEMS];
    long long s = 0;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      const int64_t idx = base + (int64_t)tid * ITEMS + i;
      v[i] = idx < n ? in[idx] : 0;
      s += v[i];
    }
    long long incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long t = __shfl_up_sync(FULL, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) warp_sum[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      long long w = warp_sum[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const long long t = __shfl_up_sync(FULL, w, o);
        if (lane >= o) w += t;
      }
      warp_sum[lane] = w;  // inclusive over warps
    }
    __syncthreads();
    long long run = carry + (wid ? warp_sum[wid - 1] : 0) + incl - s;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      const int64_t idx = base + (int64_t)tid * ITEMS + i;
      if (idx < n) out[idx] = (int32_t)run;
      run += v[i];
    }
    __syncthreads();
    if (tid == 0) carry += warp_sum[31];
    __syncthreads();
  }
  if (tid == 0) {
    out[n] = (int32_t)carry;
    *total = carry;
  }
}

__global__ void k_round(const double* __restrict__ v64, int64_t n, float* __restrict__ v32,
                        uint16_t* __restrict__ v16) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double w = v64[i];
    if (v32) v32[i] = __double2float_rn(w);
    if (v16) v16[i] = srt_f64_to_bf16(w);
  }
}

// ---- transpose: rows are grouped in blocks of rb consecutive rows ----------
// cnt[b][c] = entries of block b in column c.
__global__ void k_block_count(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                              int rows, int rb, int cols, int32_t* __restrict__ cnt) {
  const int b = blockIdx.x;
  const int ra = b * rb, rz = min(rows, ra + rb);
  if (ra >= rz) return;
  const int64_t e0 = rowptr[ra], e1 = rowptr[rz];
  int32_t* c = cnt + (int64_t)b * cols;
  for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) atomicAdd(&c[col[e]], 1);
}

// Per column: exclusive prefix over blocks (in place) and the column total.
__global__ void k_col_prefix(int32_t* __restrict__ cnt, int nblocks, int cols,
                             int32_t* __restrict__ tot) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  int32_t run = 0;
  for (int b = 0; b < nblocks; ++b) {
    const int64_t i = (int64_t)b * cols + c;
    const int32_t v = cnt[i];
    cnt[i] = run;
    run += v;
  }
  tot[c] = run;
}

// Scatter block b's rows in row order: each row's columns are distinct, so a
// row's entries are written concurrently; rows follow each other after a
// barrier.  Output rows come out sorted by source row; values and payloads
// are copied bitwise.
__global__ void k_block_fill(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                             const float* __restrict__ v32, const uint16_t* __restrict__ v16,
                             const double* __restrict__ v64, const int32_t* __restrict__ pay,
                             int rows, int rb, int cols, const int32_t* __restrict__ tptr,
                             int32_t* __restrict__ cur, int32_t* __restrict__ tcol,
                             float* __restrict__ t32, uint16_t* __restrict__ t16,
                             double* __restrict__ t64, int32_t* __restrict__ tpay) {
  const int b = blockIdx.x;
  int32_t* c = cur + (int64_t)b * cols;
  const int rz = min(rows, (b + 1) * rb);
  for (int r = b * rb; r < rz; ++r) {
    const int32_t e0 = rowptr[r], e1 = rowptr[r + 1];
    for (int32_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
      const int32_t k = col[e];
      const int64_t pos = (int64_t)tptr[k] + c[k];
      c[k] += 1;
      tcol[pos] = r;
      if (t32) t32[pos] = v32[e];
      if (t16) t16[pos] = v16[e];
      if (t64) t64[pos] = v64[e];
      if (tpay) tpay[pos] = pay[e];
    }
    __syncthreads();
  }
}

}  // namespace

int srt_scan_counts(const int32_t* counts, int32_t* out, int64_t n, long long* dtotal,
                    int64_t* total, cudaStream_t st) {
  k_scan<<<1, 1024, 0, st>>>(counts, out, n, dtotal);
  SRT_CUDA_TRY(cudaGetLastError());
  long long t = 0;
  SRT_CUDA_TRY(cudaMemcpyAsync(&t, dtotal, sizeof(t), cudaMemcpyDeviceToHost, st));
  SRT_CUDA_TRY(cudaStreamSynchronize(st));
  *total = t;
  return SRT_OK;
}

int srt_csr_transpose(int rows, int cols, int64_t nnz, const int32_t* rowptr, const int32_t* col,
                      const float* v32, const uint16_t* v16, const double* v64,
                      const int32_t* pay, int32_t* trowptr, int32_t* tcol, float* t32,
                      uint16_t* t16, double* t64, int32_t* tpay, cudaStream_t st) {
  const int nb = rows < 256 ? (rows > 0 ? rows : 1) : 256;
  const int rb = (rows + nb - 1) / nb;
  SrtTmp tmp;
  int32_t *cnt, *tot;
  long long* dtot;
  SRT_TRY(tmp.get(&cnt, (int64_t)nb * cols));
  SRT_TRY(tmp.get(&tot, cols));
  SRT_TRY(tmp.get(&dtot, 1));
  SRT_CUDA_TRY(cudaMemsetAsync(cnt, 0, (size_t)nb * cols * sizeof(int32_t), st));
  k_block_count<<<nb, 512, 0, st>>>(rowptr, col, rows, rb, cols, cnt);
  SRT_CUDA_TRY(cudaGetLastError());
  k_col_prefix<<<(cols + 255) / 256, 256, 0, st>>>(cnt, nb, cols, tot);
  SRT_CUDA_TRY(cudaGetLastError());
  int64_t got = 0;
  SRT_TRY(srt_scan_counts(tot, trowptr, cols, dtot, &got, st));
  if (got != nnz) return SRT_ERR_CUDA;
  k_block_fill<<<nb, 512, 0, st>>>(rowptr, col, v32, v16, v64, pay, rows, rb, cols, trowptr, cnt,
                                   tcol, t32, t16, t64, tpay);
  SRT_CUDA_TRY(cudaGetLastError());
  SRT_CUDA_TRY(cudaStreamSynchronize(st));
  return SRT_OK;
}

namespace {

// Assemble one operator (A1 if a1, else A2) into m, FP64 lengths rounded to
// the plan's type; the FP64 lengths stay in m->v64 for the caller to keep or free.
template <bool A1>
int assemble_one(const GeomDev& G, int wdt, SrtCsr* m, int64_t* dropped, int64_t* bytes,
                 cudaStream_t st) {
  const int rows = A1 ? G.nj * G.n_ell : G.n_zs * G.n_ell;
  const int cols = A1 ? G.ms * G.ms : G.n_ell * G.mz;
  m->rows = rows;
  m->cols = cols;
  SrtTmp tmp;
  int32_t* counts;
  long long* dtot;
  unsigned long long* ddrop;
  SRT_TRY(tmp.get(&counts, rows));
  SRT_TRY(tmp.get(&dtot, 1));
  SRT_TRY(tmp.get(&ddrop, 1));
  SRT_CUDA_TRY(cudaMemsetAsync(ddrop, 0, sizeof(unsigned long long), st));
  SRT_TRY(srt_dmalloc(&m->rowptr, (int64_t)rows + 1, bytes));
  const int threads = 256;
  const int blocks = (int)(((int64_t)rows * 32 + threads - 1) / threads);
  k_assemble<A1><<<blocks, threads, 0, st>>>(G, rows, 0, counts, nullptr, nullptr, nullptr, ddrop);
  SRT_CUDA_TRY(cudaGetLastError());
  int64_t nnz = 0;
  SRT_TRY(srt_scan_counts(counts, m->rowptr, rows, dtot, &nnz, st));
  if (nnz >= ((int64_t)1 << 31)) return SRT_ERR_GEOMETRY;
  m->nnz = nnz;
  unsigned long long dr = 0;
  SRT_CUDA_TRY(cudaMemcpyAsync(&dr, ddrop, sizeof(dr), cudaMemcpyDeviceToHost, st));
  SRT_TRY(srt_dmalloc(&m->col, nnz, bytes));
  SRT_TRY(srt_dmalloc(&m->v64, nnz, nullptr));
  k_assemble<A1><<<blocks, threads, 0, st>>>(G, rows, 1, nullptr, m->rowptr, m->col, m->v64,
                                             nullptr);
  SRT_CUDA_TRY(cudaGetLastError());
  if (wdt == SRT_BF16)
    SRT_TRY(srt_dmalloc(&m->v16, nnz, bytes));
  else
    SRT_TRY(srt_dmalloc(&m->v32, nnz, bytes));
  k_round<<<1216, 256, 0, st>>>(m->v64, nnz, m->v32, m->v16);
  SRT_CUDA_TRY(cudaGetLastError());
  SRT_CUDA_TRY(cudaStreamSynchronize(st));
  *dropped = (int64_t)dr;
  return SRT_OK;
}

// t = transpose of a: rows sorted by source row, values bit-identical.
int transpose_csr(const SrtCsr& a, SrtCsr* t, int64_t* bytes, cudaStream_t st) {
  t->rows = a.cols;
  t->cols = a.rows;
  t->nnz = a.nnz;
  SRT_TRY(srt_dmalloc(&t->rowptr, (int64_t)a.cols + 1, bytes));
  SRT_TRY(srt_dmalloc(&t->col, a.nnz, bytes));
  if (a.v32) SRT_TRY(srt_dmalloc(&t->v32, a.nnz, bytes));
  if (a.v16) SRT_TRY(srt_dmalloc(&t->v16, a.nnz, bytes));
  if (a.v64) SRT_TRY(srt_dmalloc(&t->v64, a.nnz, bytes));
  return srt_csr_transpose(a.rows, a.cols, a.nnz, a.rowptr, a.col, a.v32, a.v16, a.v64, nullptr,
                           t->rowptr, t->col, t->v32, t->v16, t->v64, nullptr, st);
}

}  // namespace

void srt_csr_free(SrtCsr* m) {
  cudaFree(m->rowptr);
  cudaFree(m->col);
  cudaFree(m->v32);
  cudaFree(m->v16);
  cudaFree(m->v64);
  *m = SrtCsr();
}

// The rings are spaced like the slabs (ring spacing = dz to rounding), so A2
// is Toeplitz in the slab offset whatever the number of rings and their
// offset from the slab centres.
static bool toeplitz_applies(const srt_geometry& g) {
  const double spacing = (g.zs_hi - g.zs_lo) / g.n_zs;
  return fabs(spacing - g.dz) <= 1e-12 * g.dz && !(g.flags & SRT_CSR_ONLY) &&
         g.n_ell <= 0xffff && (int64_t)g.mz + g.n_zs - 1 <= 0x7fff;
}

static int expand_toeplitz(const SrtCsr& T, const srt_geometry& g, SrtCsr* a2, int64_t* bytes,
                           cudaStream_t st) {
  const int rows = g.n_zs * g.n_ell;
  a2->rows = rows;
  a2->cols = g.n_ell * g.mz;
  SrtTmp tmp;
  int32_t* counts;
  long long* dtot;
  SRT_TRY(tmp.get(&counts, rows));
  SRT_TRY(tmp.get(&dtot, 1));
  SRT_TRY(srt_dmalloc(&a2->rowptr, (int64_t)rows + 1, bytes));
  const int blocks = (int)(((int64_t)rows * 32 + 255) / 256);
  k_expand_toeplitz<<<blocks, 256, 0, st>>>(g.mz, g.n_zs, g.n_ell, rows, 0, T.rowptr, T.col,
                                            T.v32, T.v16, T.v64, counts, nullptr, nullptr,
                                            nullptr, nullptr, nullptr);
  SRT_CUDA_TRY(cudaGetLastError());
  int64_t nnz = 0;
  SRT_TRY(srt_scan_counts(counts, a2->rowptr, rows, dtot, &nnz, st));
  if (nnz >= ((int64_t)1 << 31)) return SRT_ERR_GEOMETRY;
  a2->nnz = nnz;
  SRT_TRY(srt_dmalloc(&a2->col, nnz, bytes));
  if (T.v32) SRT_TRY(srt_dmalloc(&a2->v32, nnz, bytes));
  if (T.v16) SRT_TRY(srt_dmalloc(&a2->v16, nnz, bytes));
  if (T.v64) SRT_TRY(srt_dmalloc(&a2->v64, nnz, nullptr));
  k_expand_toeplitz<<<blocks, 256, 0, st>>>(g.mz, g.n_zs, g.n_ell, rows, 1, T.rowptr, T.col,
                                            T.v32, T.v16, T.v64, nullptr, a2->rowptr, a2->col,
                                            a2->v32, a2->v16, a2->v64);
  SRT_CUDA_TRY(cudaGetLastError());
  SRT_CUDA_TRY(cudaStreamSynchronize(st));
  return SRT_OK;
}

int srt_assemble(srt_plan_s* plan, cudaStream_t st) {
  const GeomDev G = make_geom(plan->g);
  const bool keep = (plan->g.flags & SRT_KEEP_F64) != 0;
  const int wdt = plan->g.weight_dtype;
  // A1 by rotation: with n_phi a multiple of 4, column j + n_phi/4 sees the
  // pixel grid turned by 90 degrees about the axis, so the rows of the first
  // n_phi/4 columns determine all of A1 (and A1^T)
  // (and the mirror across the diagonal takes column t to n_phi/4 - t, so
  // with n_phi a multiple of 8 and phi0 = 0 the first n_phi/8 + 1 do).
  // The 8-fold form is applied by the tile kernels only (a1tiles.cu).
  const srt_geometry& g0 = plan->g;
  const int fl = g0.flags;
  const bool full_circle =
      g0.n_phi_total <= 0 || (g0.n_phi_total == g0.n_phi && g0.phi_first == 0);
  const bool tiles = g0.ms % 2 == 0 && g0.ms < 4096 && g0.mz % 4 == 0 && g0.n_phi < 32768 &&
                     g0.n_ell < 65536 && !(fl & SRT_ROWWISE);
  GeomDev G1 = G;
  if (!(fl & SRT_A1_FULL) && full_circle && g0.n_phi % 4 == 0 && g0.ms < 4096) {
    if (tiles && g0.n_phi % 8 == 0 && g0.phi0 == 0.0 && !(fl & SRT_A1_ROTATION)) {
      G1.nj = g0.n_phi / 8 + 1;
      plan->a1_rot = 2;
    } else {
      G1.nj = g0.n_phi / 4;
      plan->a1_rot = 1;
    }
  }
  SRT_TRY(assemble_one<true>(G1, wdt, &plan->a1, &plan->dropped1, &plan->bytes, st));
  if (plan->a1_rot == 2) {
    // columns 0 and n_phi/8 have 4 images, the others 8
    const int ne = g0.n_ell, half = g0.n_phi / 8;
    std::vector<int32_t> rp(plan->a1.rows + 1);
    SRT_CUDA_TRY(cudaMemcpy(rp.data(), plan->a1.rowptr, rp.size() * 4, cudaMemcpyDeviceToHost));
    int64_t n = 0;
    for (int j = 0; j <= half; ++j)
      n += (int64_t)(rp[(j + 1) * ne] - rp[j * ne]) * ((j == 0 || j == half) ? 4 : 8);
    plan->nnz1 = n;
    plan->dropped1 *= 8;  // an upper bound: the drops are not counted per column
  } else {
    const int64_t copies = plan->a1_rot ? 4 : 1;
    plan->nnz1 = plan->a1.nnz * copies;
    plan->dropped1 *= copies;
  }
  if (tiles) {
    SRT_TRY(srt_build_a1tiles(plan, &plan->bytes));
    plan->a1tiles = 1;
  }
  if (toeplitz_applies(plan->g)) {
    // master tensor: one ring over D = mz + n_zs - 1 slabs, slab q at offset
    // d = q + dmin from it, dmin = -(n_zs - 1) - s, where the ring range
    // starts s dz + eps above the volume's bottom (s the nearest integer);
    // the ring sits eps above its slab's centre, as every ring does.  A2 and
    // A2^T are applied from its taps and never stored as matrices.
    const int D = G.mz + G.n_zs - 1;
    const double delta = G.zs_lo + G.hz;
    const double sh = nearbyint(delta / G.dz), eps = delta - sh * G.dz;
    const double dmin = -(G.n_zs - 1) - sh;
    const double zr = eps - dmin * G.dz - 0.5 * D * G.dz + 0.5 * G.dz;
    GeomDev GT = G;
    GT.mz = D;
    GT.n_zs = 1;
    GT.zs_lo = zr - 0.5 * G.dz;
    GT.zs_hi = zr + 0.5 * G.dz;
    GT.hz = 0.5 * GT.mz * GT.dz;
    SRT_TRY(assemble_one<false>(GT, wdt, &plan->tm, &plan->dropped2, &plan->bytes, st));
    int64_t nnz2 = 0;
    SRT_TRY(srt_build_taps(plan, plan->tm, &nnz2, &plan->bytes));
    const srt_geometry& g = plan->g;
    plan->a2.rows = plan->a2t.cols = g.n_zs * g.n_ell;
    plan->a2.cols = plan->a2t.rows = g.n_ell * g.mz;
    plan->a2.nnz = plan->a2t.nnz = nnz2;
    plan->toeplitz = 1;
    if (!keep) {
      cudaFree(plan->tm.v64);
      plan->tm.v64 = nullptr;
    } else {
      plan->bytes += plan->tm.nnz * (int64_t)sizeof(double);
    }
  } else {
    SRT_TRY(assemble_one<false>(G, wdt, &plan->a2, &plan->dropped2, &plan->bytes, st));
  }
  if (!keep) {  // FP64 lengths are only needed for export: drop before transposing
    cudaFree(plan->a1.v64);
    cudaFree(plan->a2.v64);
    plan->a1.v64 = plan->a2.v64 = nullptr;
  } else {
    plan->bytes += (plan->a1.nnz + (plan->toeplitz ? 0 : plan->a2.nnz)) * (int64_t)sizeof(double);
  }
  // (the 8-fold form's A1^T runs from the tile records only)
  if (plan->a1_rot != 2) SRT_TRY(transpose_csr(plan->a1, &plan->a1t, &plan->bytes, st));
  if (!plan->toeplitz) SRT_TRY(transpose_csr(plan->a2, &plan->a2t, &plan->bytes, st));
  return SRT_OK;
}

int srt_expand_a2(const srt_plan_s* plan, SrtCsr* a2, SrtCsr* a2t, cudaStream_t st) {
  if (!plan->toeplitz) return SRT_ERR_ARG;
  SRT_TRY(expand_toeplitz(plan->tm, plan->g, a2, nullptr, st));
  if (a2t) SRT_TRY(transpose_csr(*a2, a2t, nullptr, st));
  return SRT_OK;
}
