/*
 * FP64 CPU oracle for the discrete spherical Radon transform (SRT) with a
 * cylindrical aperture.  TEST INFRASTRUCTURE ONLY: it is called by tests/,
 * by __graft_entry__.smoke() and by bench.py's CPU-baseline leg, never by the
 * product path.  It shares no code, header or table with the CUDA library.
 *
 * What it computes (Sec. 2 and Sec. 3.1 of the paper):
 *   The SRT of f over the shell of radius l centred at sensor r is
 *     int_0^pi int_0^2pi f(r + l(sin t cos a, sin t sin a, cos t)) l^2 sin t da dt
 *   (Sec. 2, spherical parametrisation), rewritten as an outer integral over
 *   t with measure l dt of an in-plane circle integral at radius l sin t with
 *   measure (l sin t) da (Sec. 2, "bringing a copy of l outside").
 *   The paper discretises f with piecewise-constant voxels and represents the
 *   two circular transforms by exact-arc-length matrices on a shared radius
 *   grid {l_l} (Sec. 3.1, Algorithm 1).  The intermediate f^{1,2} therefore
 *   lives on (z-slab k, radius bin l) cells and is constant on each cell,
 *   taking the value of the in-plane circle integral at the bin centre rho_l.
 *
 *   This oracle evaluates that discrete operator shell by shell, WITHOUT
 *   forming either matrix and without the two-stage product:
 *     p[j,h,m] = sum over t-segments s of  l_m |s|  *  rho_{l(s)} *
 *                sum over a-segments q of |q| * f(pixel(q), slab(s))
 *   where the t-breakpoints are the crossings of the semicircle
 *   (z_h + l_m cos t, l_m sin t) with slab planes and radius-bin edges, and
 *   the a-breakpoints are the crossings of the circle s_j + rho (cos a, sin a)
 *   with the pixel grid lines.  Every segment is assigned to the cell holding
 *   its midpoint (boundary ties have measure zero).
 *
 * Readings of the paper used here (its text is silent on them):
 *   - radii grid shared by rho and l, cell centred: l_l = lo + (l+1/2) dl;
 *   - radius bins [lo + l dl, lo + (l+1) dl]; parts of a semicircle outside
 *     [lo, hi] carry no weight (the in-plane integral vanishes below lo and
 *     the aperture is truncated above hi);
 *   - sensors phi_j = phi0 + 2 pi j / n_phi, ring heights at cell centres of
 *     [zs_lo, zs_hi]; voxel centres (i - (M-1)/2) * spacing (box centred at 0);
 *   - arc lengths in mm, no normalisation.
 *
 * Piecewise-linear intermediate (rho_linear = 1; the paper notes that the
 * algorithms carry over to other bases, naming piecewise-linear ones): f^{1,2}
 * is interpolated linearly in rho between the bin centres rho_l (the nodes),
 * held constant from lo to rho_0 and from rho_{n-1} to hi, still piecewise
 * constant in z.  The t-breakpoints are then the crossings with the radii
 * lo, rho_0, ..., rho_{n-1}, hi, and a segment between nodes rho_l and
 * rho_{l+1} gives node l the weight int (rho_{l+1} - rho) ds / dl and node l+1
 * the weight int (rho - rho_l) ds / dl, with int ds = l_m dt and
 * int rho ds = l_m^2 (cos t0 - cos t1) along the semicircle rho = l_m sin t.
 *
 * Piecewise-linear voxels (voxel_linear = 1; the same remark of the paper):
 * in every slab, f is the bilinear interpolation in (x, y) of its values at
 * the voxel centres (the nodes x_i = -hx + (i + 1/2) dxy), held constant in
 * x beyond the first and the last node column (the outer half voxel on each
 * side of the volume), likewise in y, and still constant along z within a
 * slab.  Node i's basis along x is (x - x_{i-1})/dxy on [x_{i-1}, x_i] and
 * (x_{i+1} - x)/dxy on [x_i, x_{i+1}], replaced by 1 on [-hx, x_0] for i = 0
 * and on [x_{ms-1}, hx] for i = ms - 1; the in-plane weight of node
 * (ix, iy) is the product of its x and y bases integrated along the circle.
 * The circle walk then also breaks at the node lines x = x_i, y = y_i, so
 * that every arc lies in one piece of the bases, and gives each of the (up
 * to) four nodes of that piece the integral of its basis product over the
 * arc, in closed form:
 *   int_{a0}^{a1} (px + qx cos a)(py + qy sin a) rho da.
 *
 * Layouts: f[ix][iy][iz] (z fastest), p[j][h][m].  All arithmetic is FP64.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846264338327950288

typedef struct {
  int32_t ms, mz;        /* voxels: ms x ms x mz                          */
  double dxy, dz;        /* voxel spacing, mm                              */
  double radius;         /* cylinder radius R, mm                          */
  int32_t n_phi;         /* sensor columns                                 */
  double phi0;           /* angle of column 0, rad                         */
  int32_t n_zs;          /* sensor rings                                   */
  double zs_lo, zs_hi;   /* ring heights are cell centres of [lo, hi]      */
  int32_t n_ell;         /* radius bins shared by rho and l                */
  double ell_lo, ell_hi; /* radius grid range                              */
  int32_t rho_linear;    /* 1: f^{1,2} piecewise linear in rho (see above) */
  int32_t voxel_linear;  /* 1: f bilinear in (x, y) between voxel centres   */
} orc_geom;

/* ---------------------------------------------------------------- helpers */

static int cmp_double(const void* a, const void* b) {
  double x = *(const double*)a, y = *(const double*)b;
  return (x > y) - (x < y);
}

static double wrap_2pi(double a) { return a < 0.0 ? a + 2.0 * ORC_PI : a; }

static double half_x(const orc_geom* g) { return 0.5 * g->ms * g->dxy; }
static double half_z(const orc_geom* g) { return 0.5 * g->mz * g->dz; }
static double dell(const orc_geom* g) { return (g->ell_hi - g->ell_lo) / g->n_ell; }
static double ell_centre(const orc_geom* g, int l) { return g->ell_lo + (l + 0.5) * dell(g); }
static double ring_z(const orc_geom* g, int h) {
  return g->zs_lo + (h + 0.5) * (g->zs_hi - g->zs_lo) / g->n_zs;
}
static double sensor_x(const orc_geom* g, int j) {
  return g->radius * cos(g->phi0 + 2.0 * ORC_PI * j / g->n_phi);
}
static double sensor_y(const orc_geom* g, int j) {
  return g->radius * sin(g->phi0 + 2.0 * ORC_PI * j / g->n_phi);
}

/* Work buffers of one thread: t-breakpoints, a-breakpoints and two cached
 * in-plane circles (a piecewise-linear segment needs two radii at once). */
typedef struct {
  double* tb;      /* t-breakpoints                  */
  double* ab;      /* a-breakpoints                  */
  int* cpix[2];    /* cached circle: pixel index     */
  double* clen[2]; /* cached circle: arc length      */
  int cn[2];       /* cached circle: segment count   */
  int cl[2];       /* cached circle: radius index, -1 */
} orc_ws;

/* Sizes of one in-plane circle walk: breakpoints (two per grid line met),
 * and the (pixel or node, weight) entries it writes (one per arc, or up to
 * four per arc with the piecewise-linear voxels, whose walk also breaks at
 * the node lines). */
static int walk_breaks(const orc_geom* g) {
  return g->voxel_linear ? 8 * g->ms + 8 : 4 * (g->ms + 1) + 4;
}
static int walk_entries(const orc_geom* g) {
  return g->voxel_linear ? 4 * walk_breaks(g) : walk_breaks(g);
}

static int ws_init(orc_ws* w, const orc_geom* g) {
  int nt = 2 * (g->mz + 1) + 2 * (g->n_ell + 2) + 4;
  int na = walk_breaks(g), ne = walk_entries(g);
  w->tb = (double*)malloc(sizeof(double) * nt);
  w->ab = (double*)malloc(sizeof(double) * na);
  int ok = w->tb && w->ab;
  for (int c = 0; c < 2; ++c) {
    w->cpix[c] = (int*)malloc(sizeof(int) * ne);
    w->clen[c] = (double*)malloc(sizeof(double) * ne);
    w->cn[c] = 0;
    w->cl[c] = -1;
    ok = ok && w->cpix[c] && w->clen[c];
  }
  return ok ? 0 : -1;
}

static void ws_free(orc_ws* w) {
  free(w->tb);
  free(w->ab);
  for (int c = 0; c < 2; ++c) {
    free(w->cpix[c]);
    free(w->clen[c]);
  }
}

/* ------------------------------------------------- in-plane circle walk
 * Circle centre (sx, sy), radius rho, in the (x, y) plane of the pixel grid.
 * Breakpoints: every angle where the circle meets a grid line x = const or
 * y = const, including a line it only touches (|u| = rho): the point of
 * contact splits the arc around it, so that no arc's midpoint lies on a grid
 * line.  Each arc between consecutive breakpoints then lies in one pixel
 * (the one holding its midpoint).  Output: (pixel ix*ms+iy, arc length)
 * for arcs inside the grid.  Returns the number of arcs written.          */
static int circle_walk_hat(const orc_geom* g, double sx, double sy, double rho, double* ab,
                           int* pix, double* len);

static int circle_walk(const orc_geom* g, double sx, double sy, double rho, double* ab,
                       int* pix, double* len) {
  if (g->voxel_linear) return circle_walk_hat(g, sx, sy, rho, ab, pix, len);
  const double hx = half_x(g);
  int n = 0;
  for (int i = 0; i <= g->ms; ++i) {
    double u = -hx + i * g->dxy - sx; /* x-line offset from centre */
    if (fabs(u) <= rho) {
      double v = sqrt((rho - u) * (rho + u));
      ab[n++] = wrap_2pi(atan2(v, u));
      ab[n++] = wrap_2pi(atan2(-v, u));
    }
  }
  for (int i = 0; i <= g->ms; ++i) {
    double u = -hx + i * g->dxy - sy; /* y-line offset from centre */
    if (fabs(u) <= rho) {
      double v = sqrt((rho - u) * (rho + u));
      ab[n++] = wrap_2pi(atan2(u, v));
      ab[n++] = wrap_2pi(atan2(u, -v));
    }
  }
  qsort(ab, n, sizeof(double), cmp_double);
  int out = 0;
  int nseg = n > 0 ? n : 1;
  for (int s = 0; s < nseg; ++s) {
    double a0, a1;
    if (n == 0) {
      a0 = 0.0;
      a1 = 2.0 * ORC_PI;
    } else {
      a0 = ab[s];
      a1 = (s + 1 < n) ? ab[s + 1] : ab[0] + 2.0 * ORC_PI;
    }
    if (!(a1 > a0)) continue;
    double am = 0.5 * (a0 + a1);
    double x = sx + rho * cos(am), y = sy + rho * sin(am);
    int ix = (int)floor((x + hx) / g->dxy);
    int iy = (int)floor((y + hx) / g->dxy);
    if (ix < 0 || ix >= g->ms || iy < 0 || iy >= g->ms) continue;
    pix[out] = ix * g->ms + iy;
    len[out] = rho * (a1 - a0);
    ++out;
  }
  return out;
}

/* One axis of the piecewise-linear voxels at coordinate u (x or y): the
 * nodes whose basis is non-zero there (1 or 2) and each basis as
 * a + b u.  Node centres -hx + (i + 1/2) d. */
static int axis_pieces(const orc_geom* g, double u, int* node, double* a, double* b) {
  const double hx = half_x(g), d = g->dxy;
  const double s = (u + hx) / d - 0.5; /* node coordinate: node i at s = i */
  if (s <= 0.0 || g->ms == 1) {
    node[0] = 0;
    a[0] = 1.0;
    b[0] = 0.0;
    return 1;
  }
  if (s >= g->ms - 1) {
    node[0] = g->ms - 1;
    a[0] = 1.0;
    b[0] = 0.0;
    return 1;
  }
  int i = (int)floor(s);
  if (i > g->ms - 2) i = g->ms - 2;
  const double x0 = -hx + (i + 0.5) * d, x1 = x0 + d;
  node[0] = i; /* (x1 - u) / d */
  a[0] = x1 / d;
  b[0] = -1.0 / d;
  node[1] = i + 1; /* (u - x0) / d */
  a[1] = -x0 / d;
  b[1] = 1.0 / d;
  return 2;
}

/* Circle walk of the piecewise-linear voxels: breakpoints at the pixel
 * lines and the node lines; on each arc [a0, a1] the bases are
 * ax + bx x and ay + by y with x = sx + rho cos a, y = sy + rho sin a, so
 * node (i, k) gets rho * int (px + qx cos a)(py + qy sin a) da with
 * px = ax + bx sx, qx = bx rho (likewise y), whose terms integrate to
 *   px py (a1 - a0) + px qy (cos a0 - cos a1) + qx py (sin a1 - sin a0)
 *   + qx qy (sin^2 a1 - sin^2 a0) / 2
 * (the differences taken as products of sines and cosines of the half sum
 * and half difference).  Arcs outside the volume carry no weight. */
static int circle_walk_hat(const orc_geom* g, double sx, double sy, double rho, double* ab,
                           int* pix, double* len) {
  const double hx = half_x(g), hd = 0.5 * g->dxy;
  int n = 0;
  for (int i = 0; i <= 2 * g->ms; ++i) {
    double u = -hx + i * hd - sx; /* pixel line (i even) or node line (i odd) */
    if (fabs(u) <= rho) {
      double v = sqrt((rho - u) * (rho + u));
      ab[n++] = wrap_2pi(atan2(v, u));
      ab[n++] = wrap_2pi(atan2(-v, u));
    }
  }
  for (int i = 0; i <= 2 * g->ms; ++i) {
    double u = -hx + i * hd - sy;
    if (fabs(u) <= rho) {
      double v = sqrt((rho - u) * (rho + u));
      ab[n++] = wrap_2pi(atan2(u, v));
      ab[n++] = wrap_2pi(atan2(u, -v));
    }
  }
  qsort(ab, n, sizeof(double), cmp_double);
  int out = 0;
  int nseg = n > 0 ? n : 1;
  for (int s = 0; s < nseg; ++s) {
    double a0, a1;
    if (n == 0) {
      a0 = 0.0;
      a1 = 2.0 * ORC_PI;
    } else {
      a0 = ab[s];
      a1 = (s + 1 < n) ? ab[s + 1] : ab[0] + 2.0 * ORC_PI;
    }
    if (!(a1 > a0)) continue;
    const double am = 0.5 * (a0 + a1), ah = 0.5 * (a1 - a0);
    const double x = sx + rho * cos(am), y = sy + rho * sin(am);
    if (!(x > -hx && x < hx && y > -hx && y < hx)) continue;
    int nx[2], ny[2];
    double ax[2], bx[2], ay[2], by[2];
    const int cx = axis_pieces(g, x, nx, ax, bx), cy = axis_pieces(g, y, ny, ay, by);
    const double dcos = 2.0 * sin(am) * sin(ah);         /* cos a0 - cos a1 */
    const double dsin = 2.0 * cos(am) * sin(ah);         /* sin a1 - sin a0 */
    const double dsq = 0.5 * sin(2.0 * am) * sin(2.0 * ah); /* (sin^2 a1 - sin^2 a0) / 2 */
    for (int p = 0; p < cx; ++p)
      for (int q = 0; q < cy; ++q) {
        const double px = ax[p] + bx[p] * sx, qx = bx[p] * rho;
        const double py = ay[q] + by[q] * sy, qy = by[q] * rho;
        pix[out] = nx[p] * g->ms + ny[q];
        len[out] = rho * (px * py * (a1 - a0) + px * qy * dcos + qx * py * dsin + qx * qy * dsq);
        ++out;
      }
  }
  return out;
}

/* ------------------------------------------------------- shell walk
 * Shell (j, h, m): sensor (s_j, z_h), radius l_m.  The outer variable t runs
 * over [0, pi]; the point (z, rho) = (z_h + l_m cos t, l_m sin t) moves on a
 * semicircle of the (z, rho) half plane.  For every t-segment inside a
 * (slab k, radius bin l) cell, the in-plane circle of radius rho_l about s_j
 * is walked through slab k.  emit(ctx, voxel, weight) receives every
 * elementary contribution; voxel = (ix*ms + iy)*mz + k.                  */
typedef void (*emit_fn)(void* ctx, long voxel, double weight);

static int circle_walk(const orc_geom* g, double sx, double sy, double rho, double* ab,
                       int* pix, double* len);

/* t-breakpoints of the semicircle (z_h + l cos t, l sin t): slab planes and
 * the radii that bound the intermediate's pieces (bin edges, or for the
 * piecewise-linear intermediate lo, the bin centres and hi).  Sorted. */
static int shell_breaks(const orc_geom* g, double ell, double zc, double* tb) {
  const double hz = half_z(g), dl = dell(g);
  int n = 0;
  tb[n++] = 0.0;
  tb[n++] = ORC_PI;
  for (int k = 0; k <= g->mz; ++k) {
    double u = -hz + k * g->dz - zc; /* slab plane offset */
    if (fabs(u) < ell) tb[n++] = atan2(sqrt((ell - u) * (ell + u)), u);
  }
  const int nr = g->rho_linear ? g->n_ell + 2 : g->n_ell + 1;
  for (int i = 0; i < nr; ++i) {
    double rb; /* radius-bin edge, or lo / node / hi */
    if (!g->rho_linear) rb = g->ell_lo + i * dl;
    else rb = i == 0 ? g->ell_lo : (i == nr - 1 ? g->ell_hi : ell_centre(g, i - 1));
    if (rb > 0.0 && rb < ell) {
      double a = atan2(rb, sqrt((ell - rb) * (ell + rb)));
      tb[n++] = a;
      tb[n++] = ORC_PI - a;
    }
  }
  qsort(tb, n, sizeof(double), cmp_double);
  return n;
}

/* Weights of the t-segment [t0, t1] of the semicircle of radius ell on the
 * intermediate's radius pieces: up to two (radius index, weight) pairs.
 * Returns how many (0 when the segment lies outside [lo, hi]). */
static int segment_weights(const orc_geom* g, double ell, double t0, double t1, int* idx,
                           double* wt) {
  const double dl = dell(g);
  const double tm = 0.5 * (t0 + t1);
  const double L = ell * (t1 - t0); /* arc length in the (z, rho) plane */
  /* The piece is chosen by the middle of the segment's rho range, not by rho
   * at its middle t: the radius grid meets the semicircle at its top (where
   * ell is itself a node, rho = ell only at t = pi/2), and a segment ending
   * or centred there has rho(tm) = ell, on the node, although it lies below. */
  const double s0 = sin(t0), s1 = sin(t1);
  const double smax = (t0 < 0.5 * ORC_PI && t1 > 0.5 * ORC_PI) ? 1.0 : fmax(s0, s1);
  const double rho = 0.5 * ell * (fmin(s0, s1) + smax);
  if (!g->rho_linear) {
    int l = (int)floor((rho - g->ell_lo) / dl);
    if (l < 0 || l >= g->n_ell) return 0;
    idx[0] = l;
    wt[0] = L;
    return 1;
  }
  if (rho <= g->ell_lo || rho >= g->ell_hi) return 0;
  const double u = (rho - ell_centre(g, 0)) / dl;
  if (u < 0.0 || g->n_ell == 1) { /* below the first node: constant */
    idx[0] = 0;
    wt[0] = L;
    return 1;
  }
  if (u >= g->n_ell - 1) { /* above the last node: constant */
    idx[0] = g->n_ell - 1;
    wt[0] = L;
    return 1;
  }
  int l = (int)floor(u);
  if (l > g->n_ell - 2) l = g->n_ell - 2;
  /* int rho ds = ell^2 (cos t0 - cos t1), written without cancellation */
  const double M = 2.0 * ell * ell * sin(tm) * sin(0.5 * (t1 - t0));
  idx[0] = l;
  wt[0] = (ell_centre(g, l + 1) * L - M) / dl;
  idx[1] = l + 1;
  wt[1] = (M - ell_centre(g, l) * L) / dl;
  return 2;
}

/* In-plane circle of sensor (sx, sy) at the centre radius of bin l, from the
 * two-slot cache (slot `avoid` is kept for the other radius of a segment). */
static int cached_circle(const orc_geom* g, orc_ws* w, double sx, double sy, int l, int avoid) {
  for (int c = 0; c < 2; ++c)
    if (w->cl[c] == l) return c;
  int c = avoid == 0 ? 1 : 0;
  w->cn[c] = circle_walk(g, sx, sy, ell_centre(g, l), w->ab, w->cpix[c], w->clen[c]);
  w->cl[c] = l;
  return c;
}

static void shell_walk_k(const orc_geom* g, orc_ws* w, int j, int h, int m, int k_lo, int k_hi,
                         emit_fn emit, void* ctx) {
  const double hz = half_z(g);
  const double ell = ell_centre(g, m), zc = ring_z(g, h);
  const double sx = sensor_x(g, j), sy = sensor_y(g, j);
  double* tb = w->tb;
  const int n = shell_breaks(g, ell, zc, tb);
  w->cl[0] = w->cl[1] = -1;
  for (int s = 0; s + 1 < n; ++s) {
    double t0 = tb[s], t1 = tb[s + 1];
    if (!(t1 > t0)) continue;
    double tm = 0.5 * (t0 + t1);
    double z = zc + ell * cos(tm);
    int k = (int)floor((z + hz) / g->dz);
    if (k < k_lo || k >= k_hi) continue;
    int idx[2];
    double wt[2];
    const int nw = segment_weights(g, ell, t0, t1, idx, wt);
    int used = -1;
    for (int i = 0; i < nw; ++i) {
      const int c = cached_circle(g, w, sx, sy, idx[i], used);
      used = c;
      for (int q = 0; q < w->cn[c]; ++q)
        emit(ctx, (long)w->cpix[c][q] * g->mz + k, wt[i] * w->clen[c][q]);
    }
  }
}

static void shell_walk(const orc_geom* g, orc_ws* w, int j, int h, int m, emit_fn emit,
                       void* ctx) {
  shell_walk_k(g, w, j, h, m, 0, g->mz, emit, ctx);
}

/* ------------------------------------------------------- callbacks */
typedef struct {
  const double* f;
  double acc;
} fwd_ctx;
static void emit_fwd(void* c, long v, double wgt) {
  fwd_ctx* x = (fwd_ctx*)c;
  x->acc += wgt * x->f[v];
}

typedef struct {
  double* out;
  double gval;
} adj_ctx;
static void emit_adj(void* c, long v, double wgt) {
  adj_ctx* x = (adj_ctx*)c;
  x->out[v] += wgt * x->gval;
}

typedef struct {
  long* vox;
  double* wgt;
  int n, cap, overflow;
} list_ctx;
static void emit_list(void* c, long v, double wgt) {
  list_ctx* x = (list_ctx*)c;
  if (x->n < x->cap) {
    x->vox[x->n] = v;
    x->wgt[x->n] = wgt;
    x->n++;
  } else {
    x->overflow = 1;
  }
}

static int check_geom(const orc_geom* g) {
  if (!g || g->ms <= 0 || g->mz <= 0 || g->n_phi <= 0 || g->n_zs <= 0 || g->n_ell <= 0) return -1;
  if (!(g->dxy > 0) || !(g->dz > 0) || !(g->radius > 0) || !(g->ell_hi > g->ell_lo)) return -1;
  if (!(g->ell_lo > 0)) return -1;
  if (!(g->zs_hi > g->zs_lo)) return -1;
  return 0;
}

static void set_threads(int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
}

/* ====================================================== exported API */

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Forward on a list of shells: shells[3*i .. 3*i+2] = (j, h, m). */
int orc_forward_shells(const orc_geom* g, const double* f, const int32_t* shells, long n,
                       double* out, int nthreads) {
  if (check_geom(g)) return -1;
  set_threads(nthreads);
  int err = 0;
#pragma omp parallel
  {
    orc_ws w;
    if (ws_init(&w, g)) {
#pragma omp atomic write
      err = -2;
    } else {
#pragma omp for schedule(dynamic, 8)
      for (long i = 0; i < n; ++i) {
        fwd_ctx c = {f, 0.0};
        shell_walk(g, &w, shells[3 * i], shells[3 * i + 1], shells[3 * i + 2], emit_fwd, &c);
        out[i] = c.acc;
      }
    }
    ws_free(&w);
  }
  return err;
}

/* Full forward: p[j][h][m]. */
int orc_forward(const orc_geom* g, const double* f, double* p, int nthreads) {
  if (check_geom(g)) return -1;
  long ns = (long)g->n_phi * g->n_zs * g->n_ell;
  int32_t* sh = (int32_t*)malloc(sizeof(int32_t) * 3 * ns);
  if (!sh) return -2;
  long i = 0;
  for (int j = 0; j < g->n_phi; ++j)
    for (int h = 0; h < g->n_zs; ++h)
      for (int m = 0; m < g->n_ell; ++m) {
        sh[3 * i] = j;
        sh[3 * i + 1] = h;
        sh[3 * i + 2] = m;
        ++i;
      }
  int r = orc_forward_shells(g, f, sh, ns, p, nthreads);
  free(sh);
  return r;
}

/* Full adjoint: f'[ix][iy][iz] = sum over shells of weight * p[shell].
 * Uses the same shell walk (and hence the same weights) as the forward, with
 * one FP64 accumulation buffer per thread summed in thread order.        */
int orc_adjoint(const orc_geom* g, const double* p, double* f, int nthreads) {
  if (check_geom(g)) return -1;
  set_threads(nthreads);
  long nv = (long)g->ms * g->ms * g->mz;
  long ns = (long)g->n_phi * g->n_zs * g->n_ell;
  int nt = orc_num_threads();
  double* buf = (double*)calloc((size_t)nt * nv, sizeof(double));
  if (!buf) return -2;
  int err = 0;
#pragma omp parallel
  {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    orc_ws w;
    if (ws_init(&w, g)) {
#pragma omp atomic write
      err = -2;
    } else {
      adj_ctx c = {buf + (size_t)tid * nv, 0.0};
#pragma omp for schedule(dynamic, 8)
      for (long s = 0; s < ns; ++s) {
        int j = (int)(s / ((long)g->n_zs * g->n_ell));
        int h = (int)((s / g->n_ell) % g->n_zs);
        int m = (int)(s % g->n_ell);
        c.gval = p[s];
        if (c.gval != 0.0) shell_walk(g, &w, j, h, m, emit_adj, &c);
      }
    }
    ws_free(&w);
  }
  for (long v = 0; v < nv; ++v) {
    double a = 0.0;
    for (int t = 0; t < nt; ++t) a += buf[(size_t)t * nv + v];
    f[v] = a;
  }
  free(buf);
  return err;
}

/* Adjoint restricted to a list of shells: f[voxel] += sum_i vals[i] *
 * weight(shell_i, voxel).  Each thread owns a range of slabs and walks every
 * listed shell, keeping only its own slabs, so the sums are deterministic and
 * no per-thread volume copies are needed.  f must be zeroed by the caller. */
int orc_adjoint_shells(const orc_geom* g, const int32_t* shells, const double* vals, long n,
                       double* f, int nthreads) {
  if (check_geom(g)) return -1;
  set_threads(nthreads);
  int err = 0;
#pragma omp parallel
  {
    int nt = 1, tid = 0;
#ifdef _OPENMP
    nt = omp_get_num_threads();
    tid = omp_get_thread_num();
#endif
    int k_lo = (int)((long)g->mz * tid / nt), k_hi = (int)((long)g->mz * (tid + 1) / nt);
    orc_ws w;
    if (ws_init(&w, g)) {
#pragma omp atomic write
      err = -2;
    } else if (k_hi > k_lo) {
      adj_ctx c = {f, 0.0};
      for (long i = 0; i < n; ++i) {
        c.gval = vals[i];
        if (c.gval != 0.0)
          shell_walk_k(g, &w, shells[3 * i], shells[3 * i + 1], shells[3 * i + 2], k_lo, k_hi,
                       emit_adj, &c);
      }
    }
    ws_free(&w);
  }
  return err;
}

/* Elementary contributions of one shell: (voxel, weight) pairs as emitted by
 * the walk (a voxel may appear several times).  Returns the count, or -3 if
 * cap was too small.                                                       */
long orc_shell_contrib(const orc_geom* g, int j, int h, int m, long* vox, double* wgt, long cap) {
  if (check_geom(g)) return -1;
  orc_ws w;
  if (ws_init(&w, g)) return -2;
  list_ctx c = {vox, wgt, 0, (int)cap, 0};
  shell_walk(g, &w, j, h, m, emit_list, &c);
  ws_free(&w);
  return c.overflow ? -3 : c.n;
}

/* In-plane circle of sensor column j at bin-centre radius rho_l: arcs per
 * pixel, in walk order (a pixel may appear twice); with the piecewise-linear
 * voxels, the basis integrals per node (a node appears once per arc of its
 * support).                                                               */
int orc_circle_arcs(const orc_geom* g, int j, int l, int32_t* pix, double* len, int cap) {
  if (check_geom(g)) return -1;
  int na = walk_breaks(g), ne = walk_entries(g);
  if (cap < ne) return -3;
  double* ab = (double*)malloc(sizeof(double) * na);
  if (!ab) return -2;
  int* p = (int*)malloc(sizeof(int) * ne);
  int n = circle_walk(g, sensor_x(g, j), sensor_y(g, j), ell_centre(g, l), ab, p, len);
  for (int i = 0; i < n; ++i) pix[i] = p[i];
  free(p);
  free(ab);
  return n;
}

/* (z, rho)-plane semicircle of ring h at shell radius l_m: arc length per
 * (slab k, radius bin l) cell, one entry per t-segment, cell = l*mz + k.  */
int orc_semicircle_arcs(const orc_geom* g, int h, int m, int32_t* cell, double* len, int cap) {
  if (check_geom(g)) return -1;
  const double hz = half_z(g);
  const double ell = ell_centre(g, m), zc = ring_z(g, h);
  int nt = 2 * (g->mz + 1) + 2 * (g->n_ell + 2) + 4;
  double* tb = (double*)malloc(sizeof(double) * nt);
  if (!tb) return -2;
  const int n = shell_breaks(g, ell, zc, tb);
  int out = 0;
  for (int s = 0; s + 1 < n; ++s) {
    double t0 = tb[s], t1 = tb[s + 1];
    if (!(t1 > t0)) continue;
    double tm = 0.5 * (t0 + t1);
    int k = (int)floor((zc + ell * cos(tm) + hz) / g->dz);
    if (k < 0 || k >= g->mz) continue;
    int idx[2];
    double wt[2];
    const int nw = segment_weights(g, ell, t0, t1, idx, wt);
    for (int i = 0; i < nw; ++i) {
      if (out >= cap) {
        free(tb);
        return -3;
      }
      cell[out] = idx[i] * g->mz + k;
      len[out] = wt[i];
      ++out;
    }
  }
  free(tb);
  return out;
}

/* --------------------------------------------- per-voxel weight path
 * Arc length of the circle (cx, cy, r) inside the box [x0,x1] x [y0,y1]:
 * breakpoints where the circle meets the four box lines, midpoint test.    */
static double arc_in_box_m(double cx, double cy, double r, double x0, double x1, double y0,
                           double y1, double* moment);

static double arc_in_box(double cx, double cy, double r, double x0, double x1, double y0,
                         double y1) {
  return arc_in_box_m(cx, cy, r, x0, x1, y0, y1, NULL);
}

/* The same, and *moment = int y ds over those arcs (y = cy + r sin a, so
 * int y ds = r cy (a1 - a0) + r^2 (cos a0 - cos a1) per arc). */
static double arc_in_box_m(double cx, double cy, double r, double x0, double x1, double y0,
                           double y1, double* moment) {
  double ab[8];
  int n = 0;
  double xs[2] = {x0, x1}, ys[2] = {y0, y1};
  /* A line the circle touches (|u| = r) also gives a breakpoint, at the
   * point of contact: otherwise the midpoint of the arc around that point
   * would lie on the line and fail the open-box test below. */
  for (int i = 0; i < 2; ++i) {
    double u = xs[i] - cx;
    if (fabs(u) <= r) {
      double v = sqrt((r - u) * (r + u));
      ab[n++] = wrap_2pi(atan2(v, u));
      ab[n++] = wrap_2pi(atan2(-v, u));
    }
    u = ys[i] - cy;
    if (fabs(u) <= r) {
      double v = sqrt((r - u) * (r + u));
      ab[n++] = wrap_2pi(atan2(u, v));
      ab[n++] = wrap_2pi(atan2(u, -v));
    }
  }
  qsort(ab, n, sizeof(double), cmp_double);
  double acc = 0.0, mom = 0.0;
  int nseg = n > 0 ? n : 1;
  for (int s = 0; s < nseg; ++s) {
    double a0, a1;
    if (n == 0) {
      a0 = 0.0;
      a1 = 2.0 * ORC_PI;
    } else {
      a0 = ab[s];
      a1 = (s + 1 < n) ? ab[s + 1] : ab[0] + 2.0 * ORC_PI;
    }
    if (!(a1 > a0)) continue;
    double am = 0.5 * (a0 + a1);
    double x = cx + r * cos(am), y = cy + r * sin(am);
    if (x > x0 && x < x1 && y > y0 && y < y1) {
      acc += r * (a1 - a0);
      mom += r * cy * (a1 - a0) + 2.0 * r * r * sin(am) * sin(0.5 * (a1 - a0));
    }
  }
  if (moment) *moment = mom;
  return acc;
}

double orc_arc_in_box(double cx, double cy, double r, double x0, double x1, double y0, double y1) {
  return arc_in_box(cx, cy, r, x0, x1, y0, y1);
}

/* Length and moments of the circle (cx, cy, r) inside the box, from the same
 * breakpoints and midpoint test as arc_in_box: m[0] = int ds, m[1] = int x ds,
 * m[2] = int y ds, m[3] = int x y ds, with, per arc [a0, a1],
 *   int x ds  = r cx (a1 - a0) + r^2 (sin a1 - sin a0),
 *   int y ds  = r cy (a1 - a0) + r^2 (cos a0 - cos a1),
 *   int xy ds = r cx cy (a1 - a0) + r^2 cx (cos a0 - cos a1)
 *               + r^2 cy (sin a1 - sin a0) + r^3 (sin^2 a1 - sin^2 a0) / 2. */
static void arc_moments_in_box(double cx, double cy, double r, double x0, double x1, double y0,
                               double y1, double* m) {
  double ab[8];
  int n = 0;
  double xs[2] = {x0, x1}, ys[2] = {y0, y1};
  for (int i = 0; i < 2; ++i) {
    double u = xs[i] - cx;
    if (fabs(u) <= r) {
      double v = sqrt((r - u) * (r + u));
      ab[n++] = wrap_2pi(atan2(v, u));
      ab[n++] = wrap_2pi(atan2(-v, u));
    }
    u = ys[i] - cy;
    if (fabs(u) <= r) {
      double v = sqrt((r - u) * (r + u));
      ab[n++] = wrap_2pi(atan2(u, v));
      ab[n++] = wrap_2pi(atan2(u, -v));
    }
  }
  qsort(ab, n, sizeof(double), cmp_double);
  m[0] = m[1] = m[2] = m[3] = 0.0;
  int nseg = n > 0 ? n : 1;
  for (int s = 0; s < nseg; ++s) {
    double a0, a1;
    if (n == 0) {
      a0 = 0.0;
      a1 = 2.0 * ORC_PI;
    } else {
      a0 = ab[s];
      a1 = (s + 1 < n) ? ab[s + 1] : ab[0] + 2.0 * ORC_PI;
    }
    if (!(a1 > a0)) continue;
    const double am = 0.5 * (a0 + a1), ah = 0.5 * (a1 - a0);
    const double x = cx + r * cos(am), y = cy + r * sin(am);
    if (!(x > x0 && x < x1 && y > y0 && y < y1)) continue;
    const double dcos = 2.0 * sin(am) * sin(ah), dsin = 2.0 * cos(am) * sin(ah);
    const double dsq = 0.5 * sin(2.0 * am) * sin(2.0 * ah);
    m[0] += r * (a1 - a0);
    m[1] += r * cx * (a1 - a0) + r * r * dsin;
    m[2] += r * cy * (a1 - a0) + r * r * dcos;
    m[3] += r * cx * cy * (a1 - a0) + r * r * (cx * dcos + cy * dsin) + r * r * r * dsq;
  }
}

/* One side of node i's basis along an axis: the interval [u0, u1] and the
 * basis a + b u on it (side 0: below the node, side 1: above).  Returns 0
 * where the side is empty. */
static int node_side(const orc_geom* g, int i, int side, double* u0, double* u1, double* a,
                     double* b) {
  const double hx = half_x(g), d = g->dxy, xc = -hx + (i + 0.5) * d;
  if (side == 0) {
    if (i == 0) { /* margin: constant 1 from the volume's edge */
      *u0 = -hx;
      *u1 = xc;
      *a = 1.0;
      *b = 0.0;
    } else { /* (u - x_{i-1}) / d */
      *u0 = xc - d;
      *u1 = xc;
      *a = -(xc - d) / d;
      *b = 1.0 / d;
    }
  } else {
    if (i == g->ms - 1) {
      *u0 = xc;
      *u1 = hx;
      *a = 1.0;
      *b = 0.0;
    } else { /* (x_{i+1} - u) / d */
      *u0 = xc;
      *u1 = xc + d;
      *a = (xc + d) / d;
      *b = -1.0 / d;
    }
  }
  return *u1 > *u0;
}

/* In-plane weight of node (ix, iy) on the circle (sx, sy, rho), piecewise-
 * linear voxels: over the four boxes of its support (sides of x times sides
 * of y), int (ax + bx x)(ay + by y) ds = ax ay L + ax by My + bx ay Mx
 * + bx by Mxy from the box moments. */
static double node_plane_weight(const orc_geom* g, double sx, double sy, double rho, int ix,
                                int iy) {
  double acc = 0.0;
  for (int p = 0; p < 2; ++p) {
    double x0, x1, ax, bx;
    if (!node_side(g, ix, p, &x0, &x1, &ax, &bx)) continue;
    for (int q = 0; q < 2; ++q) {
      double y0, y1, ay, by, m[4];
      if (!node_side(g, iy, q, &y0, &y1, &ay, &by)) continue;
      arc_moments_in_box(sx, sy, rho, x0, x1, y0, y1, m);
      acc += ax * ay * m[0] + ax * by * m[2] + bx * ay * m[1] + bx * by * m[3];
    }
  }
  return acc;
}

/* Weight of the intermediate's value at (slab k, radius l) in the (z, rho)
 * semicircle (centre (zc, 0), radius ell): piecewise constant, the arc in the
 * cell [z0, z0 + dz] x [bin l]; piecewise linear, the hat of node rho_l
 * integrated along the arc in the slab (pieces [rho_{l-1}, rho_l] and
 * [rho_l, rho_{l+1}], constant pieces [lo, rho_0] and [rho_{n-1}, hi]). */
static double semicircle_weight(const orc_geom* g, double zc, double ell, double z0, int l) {
  const double dl = dell(g);
  if (!g->rho_linear) {
    double rb0 = g->ell_lo + l * dl;
    return arc_in_box(zc, 0.0, ell, z0, z0 + g->dz, rb0, rb0 + dl);
  }
  const double rl = ell_centre(g, l);
  double acc = 0.0, L, M;
  if (l == 0) {
    acc += arc_in_box(zc, 0.0, ell, z0, z0 + g->dz, g->ell_lo, rl);
  } else {
    const double ra = ell_centre(g, l - 1);
    L = arc_in_box_m(zc, 0.0, ell, z0, z0 + g->dz, ra, rl, &M);
    acc += (M - ra * L) / dl;
  }
  if (l == g->n_ell - 1) {
    acc += arc_in_box(zc, 0.0, ell, z0, z0 + g->dz, rl, g->ell_hi);
  } else {
    const double rb = ell_centre(g, l + 1);
    L = arc_in_box_m(zc, 0.0, ell, z0, z0 + g->dz, rl, rb, &M);
    acc += (rb * L - M) / dl;
  }
  return acc;
}

/* Weight of voxel (ix, iy, k) in shell (j, h, m):
 *   sum over radius indices l of [weight of (k, l) in the (z,rho) semicircle]
 *                              x [arc of the in-plane circle rho_l in pixel]. */
static double point_weight(const orc_geom* g, int j, int h, int m, int ix, int iy, int k) {
  const double hx = half_x(g), hz = half_z(g), dl = dell(g);
  const double sx = sensor_x(g, j), sy = sensor_y(g, j);
  const double ell = ell_centre(g, m), zc = ring_z(g, h);
  /* the pixel, or with the piecewise-linear voxels the node's support (the
   * pixel widened by half a voxel on each side inside the volume) */
  double px0 = -hx + ix * g->dxy, py0 = -hx + iy * g->dxy;
  double px1 = px0 + g->dxy, py1 = py0 + g->dxy;
  if (g->voxel_linear) {
    px0 = fmax(-hx, px0 - 0.5 * g->dxy);
    px1 = fmin(hx, px1 + 0.5 * g->dxy);
    py0 = fmax(-hx, py0 - 0.5 * g->dxy);
    py1 = fmin(hx, py1 + 0.5 * g->dxy);
  }
  const double z0 = -hz + k * g->dz;
  /* in-plane distance range from the sensor to the box: only bins whose
   * centre radius lies in it (plus one bin of margin) can meet the box */
  double cx = fmax(px0 - sx, fmax(0.0, sx - px1));
  double cy = fmax(py0 - sy, fmax(0.0, sy - py1));
  double fx = fmax(fabs(px0 - sx), fabs(px1 - sx));
  double fy = fmax(fabs(py0 - sy), fabs(py1 - sy));
  int l0 = (int)floor((sqrt(cx * cx + cy * cy) - g->ell_lo) / dl) - 1;
  int l1 = (int)floor((sqrt(fx * fx + fy * fy) - g->ell_lo) / dl) + 1;
  if (l0 < 0) l0 = 0;
  if (l1 > g->n_ell - 1) l1 = g->n_ell - 1;
  double acc = 0.0;
  for (int l = l0; l <= l1; ++l) {
    double rho = ell_centre(g, l);
    double a1 = g->voxel_linear ? node_plane_weight(g, sx, sy, rho, ix, iy)
                                : arc_in_box(sx, sy, rho, px0, px1, py0, py1);
    if (a1 == 0.0) continue;
    acc += a1 * semicircle_weight(g, zc, ell, z0, l);
  }
  return acc;
}

double orc_point_weight(const orc_geom* g, int j, int h, int m, int ix, int iy, int k) {
  if (check_geom(g)) return -1.0;
  return point_weight(g, j, h, m, ix, iy, k);
}

/* Adjoint at a list of voxels: voxels[3*i..] = (ix, iy, k).
 * out[i] = sum over all shells of point_weight * p[shell].  Only shells whose
 * radius range can reach the voxel box are visited.                        */
int orc_adjoint_voxels(const orc_geom* g, const double* p, const int32_t* voxels, long n,
                       double* out, int nthreads) {
  if (check_geom(g)) return -1;
  set_threads(nthreads);
  const double hx = half_x(g), hz = half_z(g), dl = dell(g);
#pragma omp parallel for schedule(dynamic, 1)
  for (long i = 0; i < n; ++i) {
    int ix = voxels[3 * i], iy = voxels[3 * i + 1], k = voxels[3 * i + 2];
    /* the voxel's box, or the node's support (piecewise-linear voxels) */
    double bx0 = -hx + ix * g->dxy, by0 = -hx + iy * g->dxy, bz0 = -hz + k * g->dz;
    double bx1 = bx0 + g->dxy, by1 = by0 + g->dxy;
    if (g->voxel_linear) {
      bx0 = fmax(-hx, bx0 - 0.5 * g->dxy);
      bx1 = fmin(hx, bx1 + 0.5 * g->dxy);
      by0 = fmax(-hx, by0 - 0.5 * g->dxy);
      by1 = fmin(hx, by1 + 0.5 * g->dxy);
    }
    double acc = 0.0;
    for (int j = 0; j < g->n_phi; ++j) {
      double sx = sensor_x(g, j), sy = sensor_y(g, j);
      for (int h = 0; h < g->n_zs; ++h) {
        double zc = ring_z(g, h);
        /* distance range from the sensor point to the voxel box */
        double cx = fmax(bx0 - sx, fmax(0.0, sx - bx1));
        double cy = fmax(by0 - sy, fmax(0.0, sy - by1));
        double cz = fmax(bz0 - zc, fmax(0.0, zc - (bz0 + g->dz)));
        double dmin = sqrt(cx * cx + cy * cy + cz * cz);
        double fx = fmax(fabs(bx0 - sx), fabs(bx1 - sx));
        double fy = fmax(fabs(by0 - sy), fabs(by1 - sy));
        double fz = fmax(fabs(bz0 - zc), fabs(bz0 + g->dz - zc));
        double dmax = sqrt(fx * fx + fy * fy + fz * fz);
        int m0 = (int)floor((dmin - g->ell_lo) / dl) - 1;
        int m1 = (int)floor((dmax - g->ell_lo) / dl) + 1;
        if (m0 < 0) m0 = 0;
        if (m1 > g->n_ell - 1) m1 = g->n_ell - 1;
        for (int m = m0; m <= m1; ++m) {
          double gv = p[((long)j * g->n_zs + h) * g->n_ell + m];
          if (gv == 0.0) continue;
          acc += gv * point_weight(g, j, h, m, ix, iy, k);
        }
      }
    }
    out[i] = acc;
  }
  return 0;
}
