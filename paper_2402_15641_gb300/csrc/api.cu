// C ABI of libsrt (declared in include/srt.h): plan management, the forward
// transform (Algorithm 1 of the paper) and the matched adjoint (Algorithm 2).
//
// Forward, batch B, on every sensor column at once:
//   SpMM1  Y1[b][(j,l)][k]  = A1 F_b                 (A1: Sec. 3.1, Alg. 1)
//   P1     Y1'[(l,k)][b][j] <- Y1[b][j][(l,k)]       (Alg. 1 reshape)
//   SpMM2  P'[(h,m)][b][j]  = A2 Y1'                 (one A2 for all columns,
//                                                      so (b, j) are the dense
//                                                      columns of one product)
//   P2     p[b][j][(h,m)]   <- P'[(h,m)][b][j]       (Alg. 1 final reshape)
// Adjoint (Alg. 2): P2^-1, A2^T, P1^-1, A1^T with the transposed matrices.
#include <math.h>
#include <algorithm>
#include <chrono>
#include <mutex>
#include <new>
#include <thread>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"

namespace {

inline cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

inline int64_t align256(int64_t b) { return (b + 255) & ~(int64_t)255; }

// Elements of one intermediate buffer: the larger of Y1 (= Y1') and P'.
int64_t buf_elems(const srt_geometry& g, int batch) {
  const int64_t nb = (int64_t)batch * g.n_phi;
  const int64_t zmax = g.mz > g.n_zs ? g.mz : g.n_zs;
  return nb * g.n_ell * zmax;
}

int check_geometry(const srt_geometry& g) {
  if (g.ms <= 0 || g.mz <= 0 || g.n_phi <= 0 || g.n_zs <= 0 || g.n_ell <= 0) return SRT_ERR_GEOMETRY;
  if (!(g.dxy > 0) || !(g.dz > 0) || !(g.radius > 0)) return SRT_ERR_GEOMETRY;
  if (!(g.ell_lo > 0) || !(g.ell_hi > g.ell_lo) || !(g.zs_hi > g.zs_lo)) return SRT_ERR_GEOMETRY;
  if (!isfinite(g.phi0) || !isfinite(g.ell_hi) || !isfinite(g.zs_lo) || !isfinite(g.zs_hi))
    return SRT_ERR_GEOMETRY;
  if (!(g.radius > g.ms * g.dxy / sqrt(2.0))) return SRT_ERR_GEOMETRY;  // sensors outside
  if (g.weight_dtype != SRT_FP32 && g.weight_dtype != SRT_BF16) return SRT_ERR_GEOMETRY;
  if (g.n_phi_total < 0 || (g.n_phi_total > 0 && (g.phi_first < 0 ||
                                                  (int64_t)g.phi_first + g.n_phi > g.n_phi_total)))
    return SRT_ERR_GEOMETRY;
  // index ranges used in int32 arithmetic by the kernels
  const int64_t pix = (int64_t)g.ms * g.ms, cells = (int64_t)g.n_ell * g.mz;
  const int64_t r1 = (int64_t)g.n_phi * g.n_ell, r2 = (int64_t)g.n_zs * g.n_ell;
  const int64_t lim = ((int64_t)1 << 31) - 1;
  if (pix > lim || cells > lim || r1 > lim || r2 > lim) return SRT_ERR_GEOMETRY;
  return SRT_OK;
}

void free_plan(srt_plan_s* p);

inline void mark(srt_plan_s* p, int dir, int i, cudaStream_t st) {
  if (p->timing) cudaEventRecord(p->ev[dir][i], st);
}

int check_ws(srt_plan_s* p, int batch, const void* ws, size_t ws_bytes) {
  if (!ws || ((uintptr_t)ws & 255)) return SRT_ERR_WORKSPACE;
  if ((int64_t)ws_bytes < 2 * align256(buf_elems(p->g, batch) * 4)) return SRT_ERR_WORKSPACE;
  return SRT_OK;
}

// NVTX range over a scope (host-side: marks when each stage is enqueued, and
// lets a profiler select launches by stage name).  Header-only NVTX3: a no-op
// unless a tool is attached.
struct NvRange {
  explicit NvRange(const char* name) { nvtxRangePushA(name); }
  ~NvRange() { nvtxRangePop(); }
  NvRange(const NvRange&) = delete;
  NvRange& operator=(const NvRange&) = delete;
};

// Destination of a host-buffer call: the result is copied to `host` in
// chunks on the copy stream `cs` as the chunks are produced on the compute
// stream, so the copies overlap the rest of the transform.
constexpr int kHostChunks = 4;
struct HostSink {
  float* host = nullptr;
  cudaStream_t cs = nullptr;
  int chunks = kHostChunks;  // 1: the whole result in one copy after the transform
  cudaEvent_t ev[kHostChunks] = {};
  cudaEvent_t t0 = nullptr;  // when set, recorded on cs before the first copy
};

}  // namespace

// Copy streams (with their chunk events) of host-buffer calls, kept on the
// plan: a call takes an idle set, or creates one when every set is in use by
// a concurrent call, and returns it when it has synchronised, so a sequence
// of calls creates no stream or event after the first.
struct SrtHostPool {
  struct Set {
    cudaStream_t cs = nullptr;
    cudaEvent_t ev[kHostChunks] = {};
  };
  std::mutex mu;
  std::vector<Set> idle;
};

namespace {

void host_set_destroy(SrtHostPool::Set& s) {
  for (cudaEvent_t& e : s.ev)
    if (e) cudaEventDestroy(e);
  if (s.cs) cudaStreamDestroy(s.cs);
  s = SrtHostPool::Set();
}

int host_set_take(srt_plan_s* p, SrtHostPool::Set* out) {
  {
    std::lock_guard<std::mutex> lk(p->host_pool->mu);
    if (!p->host_pool->idle.empty()) {
      *out = p->host_pool->idle.back();
      p->host_pool->idle.pop_back();
      return SRT_OK;
    }
  }
  SrtHostPool::Set s;
  bool ok = cudaStreamCreateWithFlags(&s.cs, cudaStreamNonBlocking) == cudaSuccess;
  for (cudaEvent_t& e : s.ev)
    if (ok) ok = cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    host_set_destroy(s);
    return SRT_ERR_CUDA;
  }
  *out = s;
  return SRT_OK;
}

void host_set_give(srt_plan_s* p, SrtHostPool::Set& s) {
  std::lock_guard<std::mutex> lk(p->host_pool->mu);
  p->host_pool->idle.push_back(s);
}

void free_plan(srt_plan_s* p) {
  if (!p) return;
  srt_csr_free(&p->a1);
  srt_csr_free(&p->a2);
  srt_csr_free(&p->a1t);
  srt_csr_free(&p->a2t);
  srt_taps_free(&p->tf);
  srt_taps_free(&p->ta);
  srt_tiles_free(&p->tlf);
  srt_tiles_free(&p->tla);
  srt_a1tiles_free(&p->a1tl);
  srt_csr_free(&p->tm);
  for (int d = 0; d < 2; ++d)
    for (int i = 0; i < 5; ++i)
      if (p->ev[d][i]) cudaEventDestroy(p->ev[d][i]);
  if (p->host_pool) {
    for (SrtHostPool::Set& s : p->host_pool->idle) host_set_destroy(s);
    delete p->host_pool;
  }
  delete p;
}

// How the A1 products reach the rows the plan did not store (SrtRot).
SrtRot a1_rot(const srt_plan_s* p, int mode) {
  SrtRot r;
  if (p->a1_rot) {
    r.mode = mode;
    r.ms = p->g.ms;
    r.n_ell = p->g.n_ell;
    r.q = p->g.n_phi / 4;
    r.mirror = p->a1_rot == 2 ? 1 : 0;
  }
  return r;
}

// Copy `height` rows of `width_elems` floats, `pitch_elems` apart, from the
// device to the host on the sink's copy stream once the compute stream has
// reached this point.
int sink_copy(HostSink* hs, int chunk, cudaStream_t st, float* host, const float* dev,
              int64_t width_elems, int64_t pitch_elems, int64_t height) {
  SRT_CUDA_TRY(cudaEventRecord(hs->ev[chunk], st));
  SRT_CUDA_TRY(cudaStreamWaitEvent(hs->cs, hs->ev[chunk], 0));
  if (chunk == 0 && hs->t0) SRT_CUDA_TRY(cudaEventRecord(hs->t0, hs->cs));
  SRT_CUDA_TRY(cudaMemcpy2DAsync(host, pitch_elems * 4, dev, pitch_elems * 4, width_elems * 4,
                                 height, cudaMemcpyDeviceToHost, hs->cs));
  return SRT_OK;
}

// Forward (Algorithm 1).  With a sink, the second product and the final
// reshape run in kHostChunks ring ranges and each range of p is copied to
// the host while the next one is computed (no per-stage timing then).
// With SRT_FUSE_RESHAPES the tile products write their output in the layout
// of the step after the reshape (P2 in the forward, P1^-1 in the adjoint),
// and so does the A1 product stored by rotation (P1: blocks of 4 sensor
// columns x 2 radii, 16-byte pieces of 4 columns).
bool fused_reshapes(const srt_plan_s* p, int64_t nb) {
  return p->tiles && nb % 4 == 0 && (p->g.flags & SRT_FUSE_RESHAPES);
}
bool fused_p1(const srt_plan_s* p) {
  return p->a1_rot && p->g.n_phi % 4 == 0 && p->g.mz % 4 == 0 &&
         (p->g.flags & SRT_FUSE_RESHAPES);
}

int run_forward(srt_plan_s* p, const float* f, float* out, int B, float* w0, float* w1,
                cudaStream_t st, HostSink* hs = nullptr) {
  const srt_geometry& g = p->g;
  const int64_t pix = (int64_t)g.ms * g.ms, r1 = (int64_t)g.n_phi * g.n_ell;
  const int64_t c1 = (int64_t)g.n_ell * g.mz, r2 = (int64_t)g.n_zs * g.n_ell;
  const int64_t nb = (int64_t)B * g.n_phi;  // dense width of the second stage
  NvRange all("srt forward (Algorithm 1)");
  if (!hs) mark(p, 0, 0, st);
  // Y1[b][j][l][k] = A1 F_b (CRT in the first plane, all slabs at once)
  // rows (j, l) visited radius-chunk-major across sensor columns (L2 reuse of F)
  {
    NvRange r(fused_p1(p) ? "A1 product + reshape P1" : "A1 product");
    // CSR rows, a warp per row: the 8 warps of a block take 8 consecutive
    // radii of one column, whose circles cross the same pixels, and share
    // those gathers in L1 (46% hits).  4-radius register tiles
    // (srt_a1tiles_apply) fetch each pixel once per tile instead, but lose
    // that sharing (13% L1 hits) and measured slower (1.74-1.97 against
    // 1.56 ms at 256^3).
    if (fused_p1(p))  // writing Y1' (the reshape P1's output) itself
      SRT_TRY(srt_spmm(p->a1, g.weight_dtype, f, g.mz, pix * g.mz, w1, 0, 0, g.mz, B, st,
                       g.n_phi, g.n_ell, 4, 0, r1, a1_rot(p, 1), 0, nb));
    else
      SRT_TRY(srt_spmm(p->a1, g.weight_dtype, f, g.mz, pix * g.mz, w0, g.mz, r1 * g.mz, g.mz,
                       B, st, g.n_phi, g.n_ell, 1, 0, r1, a1_rot(p, 1)));
  }
  if (!hs) mark(p, 0, 1, st);
  if (!fused_p1(p)) {
    NvRange r("reshape P1");
    SRT_TRY(srt_transpose(w0, c1, (int64_t)g.n_phi * c1, w1, nb, g.n_phi, g.n_phi, (int)c1, B, st));
  }
  if (!hs) mark(p, 0, 2, st);
  // rows (h, m) visited radius-chunk-major across rings: blocks running at
  // the same time gather a narrow band of Y1' rows, which stays in L2.  A
  // block owns 4 rings x 2 radii: neighbouring rings gather shifted copies
  // of the same cells (A2 is Toeplitz in z), so its warps share L1 lines.
  const int nc = hs ? (g.n_zs < hs->chunks ? g.n_zs : hs->chunks) : 1;
  for (int c = 0; c < nc; ++c) {
    const int h0 = (int)((int64_t)g.n_zs * c / nc), h1 = (int)((int64_t)g.n_zs * (c + 1) / nc);
    const int64_t ra = (int64_t)h0 * g.n_ell, rn = (int64_t)(h1 - h0) * g.n_ell;
    NvRange r("A2 product + reshape P2");
    if (fused_reshapes(p, nb)) {  // A2 tiles writing p[b][j][h][m] directly
      SRT_TRY(srt_tiles_apply(p, false, h0, h1, 4, w1, nb, out, 0, (int)nb, st, r2));
      if (!hs) mark(p, 0, 3, st);
      if (hs) SRT_TRY(sink_copy(hs, c, st, hs->host + ra, out + ra, rn, r2, (int64_t)B * g.n_phi));
      continue;
    }
    if (p->tiles && nb % 4 == 0)  // A2 from 2 x 2 tiles of the master tensor's taps
      SRT_TRY(srt_tiles_apply(p, false, h0, h1, 4, w1, nb, w0 + ra * nb, nb, (int)nb, st));
    else if (p->toeplitz)  // A2 from the taps of the master tensor, a warp per row
      SRT_TRY(srt_taps_apply(p, false, ra, rn, h1 - h0, g.n_ell, 4, w1, nb, w0 + ra * nb, nb,
                             (int)nb, st));
    else
      SRT_TRY(srt_spmm(p->a2, g.weight_dtype, w1, nb, 0, w0 + ra * nb, nb, 0, (int)nb, 1, st,
                       h1 - h0, g.n_ell, 4, ra, rn));
    if (!hs) mark(p, 0, 3, st);
    SRT_TRY(srt_transpose(w0 + ra * nb, nb, g.n_phi, out + ra, r2, (int64_t)g.n_phi * r2,
                          (int)rn, g.n_phi, B, st));
    if (hs) SRT_TRY(sink_copy(hs, c, st, hs->host + ra, out + ra, rn, r2, (int64_t)B * g.n_phi));
  }
  if (!hs) {
    mark(p, 0, 4, st);
    if (p->timing) p->have_times[0] = 1;
  }
  return SRT_OK;
}

// Adjoint (Algorithm 2).  With a sink, the last product (A1^T) runs in
// kHostChunks ranges of pixel columns ix and each range of f is copied to the
// host while the next one is computed (no per-stage timing then).
int run_adjoint(srt_plan_s* p, const float* in, float* f, int B, float* w0, float* w1,
                cudaStream_t st, HostSink* hs = nullptr) {
  const srt_geometry& g = p->g;
  const int64_t pix = (int64_t)g.ms * g.ms, r1 = (int64_t)g.n_phi * g.n_ell;
  const int64_t c1 = (int64_t)g.n_ell * g.mz, r2 = (int64_t)g.n_zs * g.n_ell;
  const int64_t nb = (int64_t)B * g.n_phi;
  NvRange all("srt adjoint (Algorithm 2)");
  if (!hs) mark(p, 1, 0, st);
  {
    NvRange r("reshape P2^-1");
    SRT_TRY(srt_transpose(in, r2, (int64_t)g.n_phi * r2, w0, nb, g.n_phi, g.n_phi, (int)r2, B, st));
  }
  if (!hs) mark(p, 1, 1, st);
  const bool fused = fused_reshapes(p, nb);
  {
    NvRange r(fused ? "A2^T product + reshape P1^-1" : "A2^T product");
    if (fused)  // A2^T tiles writing F1[b][j][l][k] directly
      SRT_TRY(srt_tiles_apply(p, true, 0, g.mz, 4, w0, nb, w1, 0, (int)nb, st, c1));
    else if (p->tiles && nb % 4 == 0)  // A2^T from 2 x 2 tiles of the master tensor's taps
      SRT_TRY(srt_tiles_apply(p, true, 0, g.mz, 4, w0, nb, w1, nb, (int)nb, st));
    else if (p->toeplitz)  // A2^T from the taps of the master tensor, a warp per row
      SRT_TRY(srt_taps_apply(p, true, 0, c1, 0, 0, 1, w0, nb, w1, nb, (int)nb, st));
    else
      SRT_TRY(srt_spmm(p->a2t, g.weight_dtype, w0, nb, 0, w1, nb, 0, (int)nb, 1, st));
  }
  if (!hs) mark(p, 1, 2, st);
  if (!fused) {
    NvRange r("reshape P1^-1");
    SRT_TRY(srt_transpose(w1, nb, g.n_phi, w0, c1, (int64_t)g.n_phi * c1, (int)c1, g.n_phi, B, st));
  }
  const float* f1 = fused ? w1 : w0;  // F1[b][j][l][k], input of A1^T
  if (!hs) mark(p, 1, 3, st);
  // rows (pixels) in blocks of 4 x 2 pixels: a circle crossing a compact
  // tile touches more of its pixels than of a line of 8, so warps share L1;
  // blocks walk 64 x 64 pixel super-tiles (where the grid divides), so the
  // rows gathered at any time stay within what L2 holds (2% faster at 256^3)
  // (tiles: 2 x 2 pixel tiles, chunks of whole tile rows)
  const int span = p->a1tiles ? g.ms / 2 : g.ms;
  const int nc = hs ? (span < hs->chunks ? span : hs->chunks) : 1;
  for (int c = 0; c < nc; ++c) {
    const int t0 = (int)((int64_t)span * c / nc), t1 = (int)((int64_t)span * (c + 1) / nc);
    const int x0 = p->a1tiles ? 2 * t0 : t0, x1 = p->a1tiles ? 2 * t1 : t1;
    const int64_t ra = (int64_t)x0 * g.ms, rn = (int64_t)(x1 - x0) * g.ms;
    NvRange r("A1^T product");
    if (p->a1tiles)
      SRT_TRY(srt_a1tiles_apply(p, t0, t1, f1, g.mz, r1 * g.mz, f + ra * g.mz, g.mz,
                                pix * g.mz, g.mz, B, st));
    else
      SRT_TRY(srt_spmm(p->a1t, g.weight_dtype, f1, g.mz, r1 * g.mz, f + ra * g.mz, g.mz,
                       pix * g.mz, g.mz, B, st, x1 - x0, g.ms, 4, ra, rn, a1_rot(p, 2), 64));
    if (hs) SRT_TRY(sink_copy(hs, c, st, hs->host + ra * g.mz, f + ra * g.mz, rn * g.mz, pix * g.mz, B));
  }
  if (hs) return SRT_OK;
  mark(p, 1, 4, st);
  if (p->timing) p->have_times[1] = 1;
  return SRT_OK;
}

// Debug builds (-DSRT_CHECKS): bad gathered rows counted by the kernels and
// not yet reported by srt_checks_read, and the test cap on operand rows.
long long g_checks_total = 0;
int g_checks_cap = 0;

long long checks_take_all() {
  long long n = 0;
  for (long long v : {srt_checks_take_spmm(), srt_checks_take_taps(), srt_checks_take_tiles(),
                      srt_checks_take_a1tiles()}) {
    if (v < 0) return -1;
    n += v;
  }
  return n;
}

// After a call in a debug build: wait for it and report a failed check.
int checks_after(int status, cudaStream_t st) {
#ifdef SRT_CHECKS
  if (status != SRT_OK) return status;
  if (cudaStreamSynchronize(st) != cudaSuccess) return SRT_ERR_CUDA;
  const long long n = checks_take_all();
  if (n < 0) return SRT_ERR_CUDA;
  g_checks_total += n;
  return n ? SRT_ERR_CUDA : SRT_OK;
#else
  (void)st;
  return status;
#endif
}

// The plan's matrices live on the device it was built on: a call made with
// another device current would launch there with pointers into the plan's
// device memory, so it is refused before any work.
int check_device(const srt_plan_s* plan) {
  int dev = -1;
  SRT_CUDA_TRY(cudaGetDevice(&dev));
  return dev == plan->device ? SRT_OK : SRT_ERR_ARG;
}

int common_checks(srt_plan_t plan, const void* a, const void* b, int32_t batch) {
  if (!plan || !a || !b || batch <= 0) return SRT_ERR_ARG;
  if (((uintptr_t)a & 15) || ((uintptr_t)b & 15)) return SRT_ERR_ARG;
  return check_device(plan);
}

}  // namespace

int srt_checks_rowcap() { return g_checks_cap; }

extern "C" {

int srt_geometry_default(srt_geometry* g, int32_t ms, int32_t mz, double dxy, double dz,
                         double radius, int32_t n_phi, int32_t n_zs, int32_t n_ell) {
  if (!g) return SRT_ERR_ARG;
  const double h = mz * dz, rxy = ms * dxy / sqrt(2.0);
  g->ms = ms;
  g->mz = mz;
  g->dxy = dxy;
  g->dz = dz;
  g->radius = radius;
  g->n_phi = n_phi;
  g->phi0 = 0.0;
  g->n_zs = n_zs;
  g->zs_lo = -0.5 * h;
  g->zs_hi = 0.5 * h;
  g->n_ell = n_ell;
  g->ell_lo = radius - rxy;
  g->ell_hi = radius + rxy;
  g->weight_dtype = SRT_FP32;
  g->flags = 0;
  g->n_phi_total = 0;
  g->phi_first = 0;
  return SRT_OK;
}

int srt_plan(const srt_geometry* g, void* stream, srt_plan_t* out) {
  if (!out) return SRT_ERR_ARG;
  *out = nullptr;
  if (!g) return SRT_ERR_ARG;
  SRT_TRY(check_geometry(*g));
  srt_plan_s* p = new (std::nothrow) srt_plan_s();
  if (!p) return SRT_ERR_OOM;
  p->host_pool = new (std::nothrow) SrtHostPool();
  if (!p->host_pool) {
    delete p;
    return SRT_ERR_OOM;
  }
  p->g = *g;
  if (cudaGetDevice(&p->device) != cudaSuccess) {
    free_plan(p);
    return SRT_ERR_CUDA;
  }
  int s = srt_assemble(p, S(stream));
  if (s != SRT_OK) {
    cudaStreamSynchronize(S(stream));
    cudaGetLastError();
    free_plan(p);
    return s;
  }
  *out = p;
  return SRT_OK;
}

int srt_plan_info(srt_plan_t p, srt_plan_info_t* o) {
  if (!p || !o) return SRT_ERR_ARG;
  o->rows1 = (int64_t)p->g.n_phi * p->g.n_ell;
  o->cols1 = p->a1.cols;
  o->nnz1 = p->nnz1;
  o->rows2 = p->a2.rows;
  o->cols2 = p->a2.cols;
  o->nnz2 = p->a2.nnz;
  o->dropped1 = p->dropped1;
  o->dropped2 = p->dropped2;
  o->device_bytes = p->bytes;
  o->weight_dtype = p->g.weight_dtype;
  o->a2_taps = p->toeplitz;
  o->n_taps = p->toeplitz ? p->tm.nnz : 0;
  o->a1_rot = p->a1_rot;
  o->tile_order = (p->tiles && p->tlf.desc ? 1 : 0) | (p->tiles && p->tla.desc ? 2 : 0);
  o->tile_records[0] = p->tiles ? p->tlf.nrec : 0;
  o->tile_records[1] = p->tiles ? p->tla.nrec : 0;
  o->tile_records[2] = p->a1tiles ? p->a1tl.na : 0;
  return SRT_OK;
}

int srt_workspace_bytes(srt_plan_t p, int32_t batch, size_t* bytes) {
  if (!p || !bytes || batch <= 0) return SRT_ERR_ARG;
  *bytes = (size_t)(2 * align256(buf_elems(p->g, batch) * 4));
  return SRT_OK;
}

int srt_forward(srt_plan_t p, const float* f, float* out, int32_t batch, void* ws,
                size_t ws_bytes, void* stream) {
  SRT_TRY(common_checks(p, f, out, batch));
  SRT_TRY(check_ws(p, batch, ws, ws_bytes));
  float* w0 = (float*)ws;
  float* w1 = w0 + align256(buf_elems(p->g, batch) * 4) / 4;
  return checks_after(run_forward(p, f, out, batch, w0, w1, S(stream)), S(stream));
}

int srt_adjoint(srt_plan_t p, const float* in, float* f, int32_t batch, void* ws,
                size_t ws_bytes, void* stream) {
  SRT_TRY(common_checks(p, in, f, batch));
  SRT_TRY(check_ws(p, batch, ws, ws_bytes));
  float* w0 = (float*)ws;
  float* w1 = w0 + align256(buf_elems(p->g, batch) * 4) / 4;
  return checks_after(run_adjoint(p, in, f, batch, w0, w1, S(stream)), S(stream));
}

int srt_host_workspace_bytes(srt_plan_t p, int32_t batch, size_t* bytes) {
  if (!p || !bytes || batch <= 0) return SRT_ERR_ARG;
  const srt_geometry& g = p->g;
  const int64_t nf = (int64_t)batch * g.ms * g.ms * g.mz;
  const int64_t np = (int64_t)batch * g.n_phi * g.n_zs * g.n_ell;
  *bytes = (size_t)(align256(nf * 4) + align256(np * 4) + 2 * align256(buf_elems(g, batch) * 4));
  return SRT_OK;
}

static int host_call(srt_plan_t p, int dir, const float* in_h, float* out_h, int32_t batch,
                     void* ws, size_t ws_bytes, void* stream) {
  if (!p || !in_h || !out_h || batch <= 0) return SRT_ERR_ARG;
  SRT_TRY(check_device(p));
  size_t need = 0;
  srt_host_workspace_bytes(p, batch, &need);
  if (!ws || ((uintptr_t)ws & 255) || ws_bytes < need) return SRT_ERR_WORKSPACE;
  const srt_geometry& g = p->g;
  const int64_t nf = (int64_t)batch * g.ms * g.ms * g.mz;
  const int64_t np = (int64_t)batch * g.n_phi * g.n_zs * g.n_ell;
  float* df = (float*)ws;
  float* dp = df + align256(nf * 4) / 4;
  float* w0 = dp + align256(np * 4) / 4;
  float* w1 = w0 + align256(buf_elems(g, batch) * 4) / 4;
  cudaStream_t st = S(stream);
  // results go back in chunks on a copy stream taken from the plan's pool,
  // overlapping the rest of the transform
  SrtHostPool::Set cp;
  SRT_TRY(host_set_take(p, &cp));
  HostSink hs;
  hs.host = out_h;
  hs.cs = cp.cs;
  for (int i = 0; i < kHostChunks; ++i) hs.ev[i] = cp.ev[i];
  int s = SRT_OK;
  {
    if (dir == 0) {
      s = cudaMemcpyAsync(df, in_h, nf * 4, cudaMemcpyHostToDevice, st) == cudaSuccess
              ? run_forward(p, df, dp, batch, w0, w1, st, &hs)
              : SRT_ERR_CUDA;
    } else {
      s = cudaMemcpyAsync(dp, in_h, np * 4, cudaMemcpyHostToDevice, st) == cudaSuccess
              ? run_adjoint(p, dp, df, batch, w0, w1, st, &hs)
              : SRT_ERR_CUDA;
    }
  }
  // wait for both streams whatever happened; the copy stream goes back to
  // the pool only when it finished cleanly
  const bool ok_st = cudaStreamSynchronize(st) == cudaSuccess;
  const bool ok_cs = cudaStreamSynchronize(cp.cs) == cudaSuccess;
  if ((!ok_st || !ok_cs) && s == SRT_OK) s = SRT_ERR_CUDA;
  if (ok_cs) host_set_give(p, cp);
  else host_set_destroy(cp);
  return checks_after(s, st);
}

int srt_forward_host(srt_plan_t p, const float* f_host, float* p_host, int32_t batch, void* ws,
                     size_t ws_bytes, void* stream) {
  return host_call(p, 0, f_host, p_host, batch, ws, ws_bytes, stream);
}

int srt_adjoint_host(srt_plan_t p, const float* p_host, float* f_host, int32_t batch, void* ws,
                     size_t ws_bytes, void* stream) {
  return host_call(p, 1, p_host, f_host, batch, ws, ws_bytes, stream);
}

// ------------------------------------------------------------ pipelines
// Host-buffer calls with several in flight: 2-4 slots of device input and
// output buffers, one stream each for input copies, computation and result
// copies.  Call i copies its input into slot i % slots while earlier calls
// compute, and its result goes back while later calls compute, so
// a sequence of calls costs about the larger of the copy and the compute
// time per call instead of their sum.  The compute stream runs the calls in
// submission order, sharing one pair of intermediate buffers.
}  // extern "C"

struct srt_pipe_s {
  // events of one call: input copy (h0, h1), transform (c0, c1), result copy
  // (d0, d1); d1 marks the call complete.  Kept for the last kRing calls.
  static constexpr int kRing = 8;
  struct Call {
    cudaEvent_t h0 = nullptr, h1 = nullptr, c0 = nullptr, c1 = nullptr, d0 = nullptr,
                d1 = nullptr;
  };
  static constexpr int kMaxSlots = 4;
  srt_plan_s* plan = nullptr;
  int batch = 0;
  int slots = 2;
  void* mem = nullptr;
  float* in[kMaxSlots] = {};
  float* out[kMaxSlots] = {};
  float* w0 = nullptr;
  float* w1 = nullptr;
  cudaStream_t cs = nullptr, h2d = nullptr, d2h = nullptr;
  Call call[kRing];
  cudaEvent_t chunk[kHostChunks] = {};
  int64_t next = 0;       // tickets issued
  int64_t done_upto = -1; // every call up to this ticket has completed
};

namespace {

void pipe_free(srt_pipe_s* q) {
  if (!q) return;
  if (q->cs) cudaStreamSynchronize(q->cs);
  if (q->h2d) cudaStreamSynchronize(q->h2d);
  if (q->d2h) cudaStreamSynchronize(q->d2h);
  for (auto& c : q->call)
    for (cudaEvent_t e : {c.h0, c.h1, c.c0, c.c1, c.d0, c.d1})
      if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : q->chunk)
    if (e) cudaEventDestroy(e);
  if (q->cs) cudaStreamDestroy(q->cs);
  if (q->h2d) cudaStreamDestroy(q->h2d);
  if (q->d2h) cudaStreamDestroy(q->d2h);
  cudaFree(q->mem);
  delete q;
}

}  // namespace

extern "C" {

int srt_pipe_create(srt_plan_t p, int32_t batch, int32_t slots, srt_pipe_t* out) {
  if (!out) return SRT_ERR_ARG;
  *out = nullptr;
  if (!p || batch <= 0 || slots < 2 || slots > srt_pipe_s::kMaxSlots) return SRT_ERR_ARG;
  SRT_TRY(check_device(p));
  const srt_geometry& g = p->g;
  const int64_t nf = (int64_t)batch * g.ms * g.ms * g.mz;
  const int64_t np = (int64_t)batch * g.n_phi * g.n_zs * g.n_ell;
  const int64_t io = align256((nf > np ? nf : np) * 4), buf = align256(buf_elems(g, batch) * 4);
  srt_pipe_s* q = new (std::nothrow) srt_pipe_s();
  if (!q) return SRT_ERR_OOM;
  q->plan = p;
  q->batch = batch;
  q->slots = slots;
  cudaError_t e = cudaMalloc(&q->mem, (size_t)(2 * slots * io + 2 * buf));
  if (e != cudaSuccess) {
    cudaGetLastError();
    q->mem = nullptr;
    pipe_free(q);
    return e == cudaErrorMemoryAllocation ? SRT_ERR_OOM : SRT_ERR_CUDA;
  }
  char* m = (char*)q->mem;
  for (int s = 0; s < slots; ++s) {
    q->in[s] = (float*)(m + (2 * s) * io);
    q->out[s] = (float*)(m + (2 * s + 1) * io);
  }
  q->w0 = (float*)(m + 2 * slots * io);
  q->w1 = (float*)(m + 2 * slots * io + buf);
  bool ok = cudaStreamCreateWithFlags(&q->cs, cudaStreamNonBlocking) == cudaSuccess &&
            cudaStreamCreateWithFlags(&q->h2d, cudaStreamNonBlocking) == cudaSuccess &&
            cudaStreamCreateWithFlags(&q->d2h, cudaStreamNonBlocking) == cudaSuccess;
  for (auto& c : q->call)
    for (cudaEvent_t* ev : {&c.h0, &c.h1, &c.c0, &c.c1, &c.d0, &c.d1})
      if (ok) ok = cudaEventCreate(ev) == cudaSuccess;
  for (cudaEvent_t& ev : q->chunk)
    if (ok) ok = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    pipe_free(q);
    return SRT_ERR_CUDA;
  }
  *out = q;
  return SRT_OK;
}

int srt_pipe_submit(srt_pipe_t q, int32_t direction, const float* in_host, float* out_host,
                    int64_t* ticket) {
  if (!q || !in_host || !out_host || (direction != 0 && direction != 1)) return SRT_ERR_ARG;
  SRT_TRY(check_device(q->plan));
  const srt_geometry& g = q->plan->g;
  const int64_t nf = (int64_t)q->batch * g.ms * g.ms * g.mz;
  const int64_t np = (int64_t)q->batch * g.n_phi * g.n_zs * g.n_ell;
  const int64_t t = q->next;
  const int s = (int)(t % q->slots);
  srt_pipe_s::Call& c = q->call[t % srt_pipe_s::kRing];
  if (t >= q->slots) {
    // the slot's input is free once call t - slots has consumed it, and its
    // output once that call's result has reached the host
    const srt_pipe_s::Call& pc = q->call[(t - q->slots) % srt_pipe_s::kRing];
    SRT_CUDA_TRY(cudaStreamWaitEvent(q->h2d, pc.c1, 0));
    SRT_CUDA_TRY(cudaStreamWaitEvent(q->cs, pc.d1, 0));
  }
  SRT_CUDA_TRY(cudaEventRecord(c.h0, q->h2d));
  SRT_CUDA_TRY(cudaMemcpyAsync(q->in[s], in_host, (direction ? np : nf) * 4,
                               cudaMemcpyHostToDevice, q->h2d));
  SRT_CUDA_TRY(cudaEventRecord(c.h1, q->h2d));
  SRT_CUDA_TRY(cudaStreamWaitEvent(q->cs, c.h1, 0));
  SRT_CUDA_TRY(cudaEventRecord(c.c0, q->cs));
  // one result copy after the transform: the next call's computation hides
  // it, and the unchunked products keep their full launch width
  HostSink hs;
  hs.host = out_host;
  hs.cs = q->d2h;
  hs.chunks = 1;
  hs.t0 = c.d0;
  for (int k = 0; k < kHostChunks; ++k) hs.ev[k] = q->chunk[k];
  if (direction == 0)
    SRT_TRY(run_forward(q->plan, q->in[s], q->out[s], q->batch, q->w0, q->w1, q->cs, &hs));
  else
    SRT_TRY(run_adjoint(q->plan, q->in[s], q->out[s], q->batch, q->w0, q->w1, q->cs, &hs));
  SRT_CUDA_TRY(cudaEventRecord(c.c1, q->cs));
  SRT_CUDA_TRY(cudaEventRecord(c.d1, q->d2h));
  if (ticket) *ticket = t;
  ++q->next;
  return SRT_OK;
}

int srt_pipe_stage_times(srt_pipe_t q, int64_t ticket, float* ms) {
  constexpr int R = srt_pipe_s::kRing;
  if (!q || !ms || ticket < 0 || ticket >= q->next) return SRT_ERR_ARG;
  if (ticket < q->next - R) return SRT_ERR_NOT_READY;  // its events were reused
  const srt_pipe_s::Call& c = q->call[ticket % R];
  const cudaError_t e = cudaEventQuery(c.d1);
  if (e == cudaErrorNotReady) return SRT_ERR_NOT_READY;
  if (e != cudaSuccess) return SRT_ERR_CUDA;
  SRT_CUDA_TRY(cudaEventElapsedTime(&ms[0], c.h0, c.h1));
  SRT_CUDA_TRY(cudaEventElapsedTime(&ms[1], c.c0, c.c1));
  SRT_CUDA_TRY(cudaEventElapsedTime(&ms[2], c.d0, c.d1));
  // idle time of the compute stream before this call: from the end of the
  // previous call's transform (0 for the first call)
  ms[3] = 0.0f;
  if (ticket > 0 && ticket - 1 >= q->next - R)
    SRT_CUDA_TRY(cudaEventElapsedTime(&ms[3], q->call[(ticket - 1) % R].c1, c.c0));
  return SRT_OK;
}

int srt_pipe_wait(srt_pipe_t q, int64_t ticket, double timeout_s) {
  constexpr int R = srt_pipe_s::kRing;
  if (!q || ticket < 0 || ticket >= q->next) return SRT_ERR_ARG;
  if (ticket <= q->done_upto) return SRT_OK;
  // the result copies run in submission order on one stream: an older call
  // whose events were reused is complete once the oldest kept call is
  const int64_t t = ticket < q->next - R ? q->next - R : ticket;
  const cudaEvent_t ev = q->call[t % R].d1;
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    const cudaError_t e = cudaEventQuery(ev);
    if (e == cudaSuccess) {
      if (t > q->done_upto) q->done_upto = t;
      return SRT_OK;
    }
    if (e != cudaErrorNotReady) return SRT_ERR_CUDA;
    const double dt = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (timeout_s >= 0 && dt > timeout_s) return SRT_ERR_TIMEOUT;
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

int srt_pipe_destroy(srt_pipe_t q) {
  pipe_free(q);
  return SRT_OK;
}

size_t srt_dot_workspace_bytes(void) { return (size_t)SRT_DOT_BLOCKS * sizeof(double); }

int srt_dot_f64(const float* a, const float* b, int64_t n, double* out, void* ws, size_t ws_bytes,
                void* stream) {
  if (!a || !b || !out || n < 0) return SRT_ERR_ARG;
  if (!ws || ((uintptr_t)ws & 7) || ws_bytes < srt_dot_workspace_bytes()) return SRT_ERR_WORKSPACE;
  return srt_dot(a, b, n, out, (double*)ws, S(stream));
}

namespace {

int export_csr(const SrtCsr* m, int32_t* rowptr, int32_t* col, float* val32, double* val64) {
  if (val64 && !m->v64) return SRT_ERR_ARG;
  SRT_CUDA_TRY(cudaMemcpy(rowptr, m->rowptr, ((size_t)m->rows + 1) * 4, cudaMemcpyDeviceToHost));
  SRT_CUDA_TRY(cudaMemcpy(col, m->col, (size_t)m->nnz * 4, cudaMemcpyDeviceToHost));
  if (val64) SRT_CUDA_TRY(cudaMemcpy(val64, m->v64, (size_t)m->nnz * 8, cudaMemcpyDeviceToHost));
  if (val32) {
    if (m->v32) {
      SRT_CUDA_TRY(cudaMemcpy(val32, m->v32, (size_t)m->nnz * 4, cudaMemcpyDeviceToHost));
    } else {
      uint16_t* tmp = new (std::nothrow) uint16_t[m->nnz > 0 ? m->nnz : 1];
      if (!tmp) return SRT_ERR_OOM;
      cudaError_t e = cudaMemcpy(tmp, m->v16, (size_t)m->nnz * 2, cudaMemcpyDeviceToHost);
      if (e == cudaSuccess)
        for (int64_t i = 0; i < m->nnz; ++i) {
          const uint32_t u = ((uint32_t)tmp[i]) << 16;
          memcpy(&val32[i], &u, 4);
        }
      delete[] tmp;
      if (e != cudaSuccess) return SRT_ERR_CUDA;
    }
  }
  return SRT_OK;
}

// Full A1 (transpose = false) or A1^T from the stored quarter of A1: row
// (j, l) is stored row (j mod q, l) with its pixels turned j / q quarter
// turns, columns sorted; the transpose is formed on the host by a stable
// counting sort (rows by increasing source row, as on the device).
int export_a1_rot(const srt_plan_s* p, bool transpose, int32_t* rowptr, int32_t* col,
                  float* val32, double* val64) {
  const SrtCsr& m = p->a1;
  const srt_geometry& g = p->g;
  if (val64 && !m.v64) return SRT_ERR_ARG;
  const int q = g.n_phi / 4, ms = g.ms, ne = g.n_ell, mode = p->a1_rot;
  const int64_t ns = m.nnz, rows = (int64_t)g.n_phi * ne, pix = (int64_t)ms * ms;
  std::vector<int32_t> rp(m.rows + 1), cl(ns);
  std::vector<float> v(ns);
  std::vector<double> v64(val64 ? ns : 0);
  SRT_CUDA_TRY(cudaMemcpy(rp.data(), m.rowptr, rp.size() * 4, cudaMemcpyDeviceToHost));
  if (ns) {
    SRT_CUDA_TRY(cudaMemcpy(cl.data(), m.col, ns * 4, cudaMemcpyDeviceToHost));
    if (m.v32) {
      SRT_CUDA_TRY(cudaMemcpy(v.data(), m.v32, ns * 4, cudaMemcpyDeviceToHost));
    } else {
      std::vector<uint16_t> h(ns);
      SRT_CUDA_TRY(cudaMemcpy(h.data(), m.v16, ns * 2, cudaMemcpyDeviceToHost));
      for (int64_t i = 0; i < ns; ++i) {
        const uint32_t u = ((uint32_t)h[i]) << 16;
        memcpy(&v[i], &u, 4);
      }
    }
    if (val64) SRT_CUDA_TRY(cudaMemcpy(v64.data(), m.v64, ns * 8, cudaMemcpyDeviceToHost));
  }
  // pixel pp under s quarter turns after the diagonal mirror when m
  auto turn = [ms](int pp, int s, int m) {
    int ix = pp / ms, iy = pp - ix * ms;
    if (m) std::swap(ix, iy);
    switch (s & 3) {
      case 0: return ix * ms + iy;
      case 1: return (ms - 1 - iy) * ms + ix;
      case 2: return (ms - 1 - ix) * ms + (ms - 1 - iy);
      default: return iy * ms + (ms - 1 - ix);
    }
  };
  // full A1, rows sorted by column
  std::vector<int32_t> frp(rows + 1), fcl(8 * ns);
  std::vector<float> fv(8 * ns);
  std::vector<double> f64(val64 ? 8 * ns : 0);
  std::vector<std::pair<int32_t, int64_t>> tmp;
  int64_t at = 0;
  for (int64_t r = 0; r < rows; ++r) {
    frp[r] = (int32_t)at;
    const int jj = (int)(r / ne), l = (int)(r % ne), s = jj / q;
    int j = jj % q, m = 0;
    if (mode == 2 && 2 * j > q) {  // column s q + t is stored column q - t, mirrored
      j = q - j;
      m = 1;
    }
    const int64_t sr = (int64_t)j * ne + l;
    tmp.clear();
    for (int64_t e = rp[sr]; e < rp[sr + 1]; ++e) tmp.emplace_back(turn(cl[e], s, m), e);
    std::sort(tmp.begin(), tmp.end());
    for (auto& t : tmp) {
      fcl[at] = t.first;
      fv[at] = v[t.second];
      if (val64) f64[at] = v64[t.second];
      ++at;
    }
  }
  frp[rows] = (int32_t)at;
  if (!transpose) {
    memcpy(rowptr, frp.data(), frp.size() * 4);
    memcpy(col, fcl.data(), at * 4);
    if (val32) memcpy(val32, fv.data(), at * 4);
    if (val64) memcpy(val64, f64.data(), at * 8);
    return SRT_OK;
  }
  std::vector<int64_t> cnt(pix + 1, 0);
  for (int64_t e = 0; e < at; ++e) ++cnt[fcl[e] + 1];
  for (int64_t i = 0; i < pix; ++i) cnt[i + 1] += cnt[i];
  for (int64_t i = 0; i <= pix; ++i) rowptr[i] = (int32_t)cnt[i];
  for (int64_t r = 0; r < rows; ++r)
    for (int64_t e = frp[r]; e < frp[r + 1]; ++e) {
      const int64_t d = cnt[fcl[e]]++;
      col[d] = (int32_t)r;
      if (val32) val32[d] = fv[e];
      if (val64) val64[d] = f64[e];
    }
  return SRT_OK;
}

}  // namespace

int srt_plan_export(srt_plan_t p, int32_t which, int32_t* rowptr, int32_t* col, float* val32,
                    double* val64) {
  if (!p || !rowptr || !col) return SRT_ERR_ARG;
  if (which < 1 || which > 4) return SRT_ERR_ARG;
  if ((which == 1 || which == 3) && p->a1_rot)
    return export_a1_rot(p, which == 3, rowptr, col, val32, val64);
  if (which == 1 || which == 3 || !p->toeplitz)
    return export_csr(which == 1 ? &p->a1 : which == 2 ? &p->a2 : which == 3 ? &p->a1t : &p->a2t,
                      rowptr, col, val32, val64);
  // A2 / A2^T of a plan that keeps only the Toeplitz taps: expand the master
  // tensor into temporary CSR matrices
  if (val64 && !p->tm.v64) return SRT_ERR_ARG;
  SrtCsr a2, a2t;
  int s = srt_expand_a2(p, &a2, which == 4 ? &a2t : nullptr, nullptr);
  if (s == SRT_OK) s = export_csr(which == 2 ? &a2 : &a2t, rowptr, col, val32, val64);
  srt_csr_free(&a2);
  srt_csr_free(&a2t);
  return s;
}

int srt_plan_set_timing(srt_plan_t p, int32_t enable) {
  if (!p) return SRT_ERR_ARG;
  if (enable && !p->ev[0][0]) {
    for (int d = 0; d < 2; ++d)
      for (int i = 0; i < 5; ++i) SRT_CUDA_TRY(cudaEventCreate(&p->ev[d][i]));
  }
  p->timing = enable ? 1 : 0;
  p->have_times[0] = p->have_times[1] = 0;
  return SRT_OK;
}

int srt_stage_times(srt_plan_t p, int32_t dir, float* ms, int32_t n) {
  if (!p || !ms || dir < 0 || dir > 1 || n < 4) return SRT_ERR_ARG;
  if (!p->have_times[dir]) return SRT_ERR_NOT_READY;
  SRT_CUDA_TRY(cudaEventSynchronize(p->ev[dir][4]));
  for (int i = 0; i < 4; ++i) SRT_CUDA_TRY(cudaEventElapsedTime(&ms[i], p->ev[dir][i], p->ev[dir][i + 1]));
  return SRT_OK;
}

int srt_launches_per_call(srt_plan_t p, int32_t dir, int32_t batch) {
  if (!p || batch <= 0 || dir < 0 || dir > 1) return 0;
  return 4 - (fused_reshapes(p, (int64_t)batch * p->g.n_phi) ? 1 : 0) -
         (dir == 0 && fused_p1(p) ? 1 : 0);
}

int srt_plan_destroy(srt_plan_t p) {
  free_plan(p);
  return SRT_OK;
}

int srt_checks_read(int64_t* violations) {
#ifdef SRT_CHECKS
  if (!violations) return SRT_ERR_ARG;
  if (cudaDeviceSynchronize() != cudaSuccess) return SRT_ERR_CUDA;
  const long long n = checks_take_all();
  if (n < 0) return SRT_ERR_CUDA;
  *violations = g_checks_total + n;
  g_checks_total = 0;
  return SRT_OK;
#else
  (void)violations;
  return SRT_ERR_ARG;
#endif
}

int srt_checks_cap(int32_t rows) {
#ifdef SRT_CHECKS
  if (rows < 0) return SRT_ERR_ARG;
  g_checks_cap = rows;
  return SRT_OK;
#else
  (void)rows;
  return SRT_ERR_ARG;
#endif
}

const char* srt_error_string(int code) {
  switch (code) {
    case SRT_OK: return "success";
    case SRT_ERR_ARG: return "invalid argument";
    case SRT_ERR_GEOMETRY: return "invalid geometry or operator too large";
    case SRT_ERR_OOM: return "out of device memory";
    case SRT_ERR_CUDA: return "CUDA runtime error";
    case SRT_ERR_WORKSPACE: return "workspace missing, too small or misaligned";
    case SRT_ERR_TIMEOUT: return "wait timed out";
    case SRT_ERR_NOT_READY: return "no timed call recorded";
    default: return "unknown status";
  }
}

}  // extern "C"
