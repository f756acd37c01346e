/*
 * srt.h -- C ABI of the GB300 (sm_103a) discrete spherical Radon transform
 * for a cylindrical sensor aperture.
 *
 * The transform follows the paper "An Efficient Implementation of the
 * Spherical Radon Transform with Cylindrical Apertures" (Lozenski, Cam,
 * Anastasio, Villa):
 *   - Sec. 2: the SRT over a shell centred on the cylinder factors into an
 *     in-plane circular Radon transform (CRT^{1,2}, radius l sin t, measure
 *     (l sin t) da) followed by a CRT^{3,4} in the (z, rho) half plane
 *     (semicircle centred (r3, 0), radius l, measure l dt);
 *   - Sec. 3.1: piecewise-constant voxels, both CRTs as sparse matrices with
 *     exact arc-length entries on a radius grid {l_l} shared by rho and l;
 *     Algorithm 1 (forward) = A1 F, reshape, A2 Y, reshape;
 *   - Sec. 3.2: Algorithm 2 (adjoint) = A2^T, reshape, A1^T: the matched
 *     adjoint, the exact transpose of the forward.
 *
 * All compute runs in hand-written CUDA kernels on the device that was current
 * when the plan was made.  There is no CPU fallback.  Every call returns an
 * srt_status; nothing throws across the ABI.  Calls that take a stream are
 * asynchronous on it (0 = legacy default stream).
 */
#ifndef SRT_H
#define SRT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
enum srt_status {
  SRT_OK = 0,
  SRT_ERR_ARG = 1,       /* null pointer, non-positive size, bad enum        */
  SRT_ERR_GEOMETRY = 2,  /* invalid geometry or operator too large (int32)   */
  SRT_ERR_OOM = 3,       /* device allocation failed during srt_plan          */
  SRT_ERR_CUDA = 4,      /* a CUDA runtime call or launch failed              */
  SRT_ERR_WORKSPACE = 5, /* workspace missing, too small or misaligned        */
  SRT_ERR_TIMEOUT = 6,   /* host-side wait exceeded its deadline              */
  SRT_ERR_NOT_READY = 7  /* timing data requested before any timed call       */
};

/* Storage type of the matrix entries; accumulation is always FP32. */
enum srt_weight_dtype { SRT_FP32 = 0, SRT_BF16 = 1 };

/* Plan flags. */
#define SRT_KEEP_F64 0x1 /* keep FP64 copies of A1/A2 entries for srt_plan_export */
#define SRT_CSR_ONLY 0x2 /* store A2, A2^T as CSR even when the taps would serve   */
/* SRT_A1_ROTATION: use the quarter turns only (n_phi % 4 == 0, ms < 4096):
 * store A1 and A1^T for the first n_phi/4 sensor columns; column j + n_phi/4
 * sees the pixel grid turned by 90 degrees, A1[(j + n_phi/4, l), rot(p)] =
 * A1[(j, l), p] with rot(ix, iy) = (ms-1-iy, ix).  The 8-fold form adds the
 * mirror across the diagonal (ix, iy) -> (iy, ix), which takes column t to
 * n_phi/4 - t (see SRT_A1_FULL for when each form applies). */
#define SRT_A1_ROTATION 0x8
/* SRT_RHO_LINEAR: the intermediate f^{1,2} is piecewise linear in rho instead
 * of constant on the radius bins (Sec. 3.1 notes the method carries over to
 * other bases): linear between the nodes rho_i = ell_lo + (i + 1/2) d,
 * constant from ell_lo to rho_0 and from rho_{n_ell-1} to ell_hi, zero
 * outside [ell_lo, ell_hi].  A1 is unchanged (it samples f^{1,2} at the
 * nodes); A2's entry (l, k) becomes node l's hat integrated along the
 * semicircle inside slab k, so A2 holds more entries (1.49x at 256^3). */
#define SRT_RHO_LINEAR 0x10
/* SRT_ROWWISE: apply every product with one warp per output row (CSR rows,
 * or A2's taps) instead of register tiles of output rows (the default).  A
 * row then sums its entries in ascending column order: with A1 stored for
 * every column the tiled and the row-wise forms agree bitwise (up to the
 * sign of zero sums); with the symmetric forms the order differs. */
#define SRT_ROWWISE 0x20
/* SRT_A1_FULL: store A1 and A1^T for every sensor column.  By default the
 * plan stores A1 for a fundamental set of columns of the aperture's
 * symmetry (srt_plan_info_t.a1_rot): the first n_phi/8 + 1 columns under
 * quarter turns and the mirror across the diagonal (n_phi % 8 == 0,
 * phi0 = 0, the whole aperture, ms even, mz % 4 == 0), else the first
 * n_phi/4 under quarter turns (n_phi % 4 == 0, the whole aperture), else
 * every column. */
#define SRT_A1_FULL 0x40
/* SRT_FUSE_RESHAPES: fold the reshapes P1, P2 (forward) and P1^-1 (adjoint)
 * into the products before them.  When A2 and A2^T are applied from
 * register tiles (srt_plan_info_t.tile_records[0] > 0) and the dense width
 * batch * n_phi is a multiple of 4, those products write their output
 * straight into the reshaped layout (p[b][j][h][m]; F1[b][j][l][k]); when
 * A1 is stored for a fundamental set of columns (srt_plan_info_t.a1_rot >
 * 0) and n_phi and mz are multiples of 4, the A1 product writes Y1' (rows
 * (l, k), columns b * n_phi + j) itself.  A forward call then makes 2 or 3
 * kernel launches instead of 4, an adjoint 3 (srt_launches_per_call); the
 * results are bitwise the same.  Off by default: the reshaped layouts take
 * each dense column as a separate 16- or 32-byte piece, which costs the
 * products more than the separate reshape kernels (which run at HBM speed)
 * cost. */
#define SRT_FUSE_RESHAPES 0x80
/* SRT_VOXEL_LINEAR: the volume is piecewise linear in x and y instead of
 * constant on the voxels (Sec. 3.1 notes the method carries over to other
 * bases): in every slab, f is the bilinear interpolation of its values at
 * the voxel centres, held constant across the outer half voxel at each side
 * of the volume, and still constant along z within a slab.  A1's entry
 * ((j, l), node (ix, iy)) becomes the node's basis integrated along the
 * circle; A1 holds more entries (each node's support is 2 x 2 voxels), the
 * layouts and every kernel stay the same, and f is read and written as the
 * node values. */
#define SRT_VOXEL_LINEAR 0x100
/* When the rings are spaced like the slabs ((zs_hi - zs_lo) / n_zs = dz, any
 * n_zs, any offset; e.g. n_zs = mz over the volume height), ring h sits at
 * slab h + s plus a fixed fraction of a slab, A2[(h,m),(l,k)] = T[m, k-h-s, l]
 * for a master tensor T, and the plan applies A2 and A2^T from T's taps
 * without storing them (srt_plan_info_t.a2_taps = 1), unless SRT_CSR_ONLY is
 * set (or mz + n_zs - 1 > 32767). */

/*
 * Geometry (Sec. 3.1, Algorithm 1 inputs).  Lengths in mm, angles in rad.
 *   Volume: ms x ms x mz voxels of size dxy x dxy x dz, voxel centres at
 *     ((i - (ms-1)/2) dxy, (j - (ms-1)/2) dxy, (k - (mz-1)/2) dz).
 *   Sensor columns: (radius cos phi_j, radius sin phi_j), phi_j = phi0 +
 *     2 pi j / n_phi, j < n_phi.  Requires radius > ms*dxy/sqrt(2).
 *   A block of the columns of a larger aperture (n_phi_total > 0): the plan
 *     holds columns phi_first .. phi_first + n_phi - 1 of n_phi_total
 *     equispaced columns, phi_j = phi0 + 2 pi (phi_first + j) / n_phi_total,
 *     computed exactly as the full aperture's plan computes those columns,
 *     so its forward is bitwise the full forward's rows of those columns and
 *     its adjoint is their share of the full adjoint (one A2 serves every
 *     column, Sec. 2).  Requires 0 <= phi_first, phi_first + n_phi <=
 *     n_phi_total; n_phi_total = 0 means the whole aperture (n_phi columns).
 *     SRT_A1_ROTATION needs the whole aperture and is ignored otherwise.
 *   Sensor rings: z_h = zs_lo + (h + 1/2)(zs_hi - zs_lo)/n_zs, h < n_zs.
 *   Radius grid shared by the in-plane radius rho and the shell radius l:
 *     bins [ell_lo + i d, ell_lo + (i+1) d], d = (ell_hi - ell_lo)/n_ell,
 *     centres l_i = ell_lo + (i + 1/2) d; requires 0 < ell_lo < ell_hi.
 *   weight_dtype: SRT_FP32 or SRT_BF16 (entries rounded once from FP64,
 *     round-to-nearest-even; the adjoint uses the identical rounded values).
 */
typedef struct srt_geometry {
  int32_t ms, mz;
  double dxy, dz;
  double radius;
  int32_t n_phi;
  double phi0;
  int32_t n_zs;
  double zs_lo, zs_hi;
  int32_t n_ell;
  double ell_lo, ell_hi;
  int32_t weight_dtype;
  int32_t flags;
  int32_t n_phi_total;  /* 0, or the aperture's column count when this plan holds a block */
  int32_t phi_first;    /* first column of the block (0 for the whole aperture) */
} srt_geometry;

typedef struct srt_plan_s* srt_plan_t;

/* Sizes of an assembled plan. */
typedef struct srt_plan_info_t {
  int64_t rows1, cols1, nnz1; /* A1 = A^{1,2}: (n_phi n_ell) x ms^2            */
  int64_t rows2, cols2, nnz2; /* A2 = A^{3,4}: (n_zs n_ell) x (n_ell mz)       */
  int64_t dropped1, dropped2; /* entries with 0 < length <= 1e-12 spacing     */
  int64_t device_bytes;       /* device memory owned by the plan              */
  int32_t weight_dtype;
  int32_t a2_taps;            /* 1: A2, A2^T applied from Toeplitz taps       */
  int64_t n_taps;             /* taps of the master tensor T (0 for CSR A2)   */
  int32_t a1_rot;             /* 1: only the first n_phi/4 columns of A1 are  */
                              /*    stored, the rest follow by quarter turns; */
                              /* 2: the first n_phi/8 + 1, by quarter turns   */
                              /*    and the diagonal mirror; 0: every column  */
  int32_t tile_order;         /* bit 0: A2's register tiles are issued from   */
                              /* the last radius pair down, bit 1: A2^T's     */
                              /* (the end of the radius range whose tiles     */
                              /* hold more records goes first); 0 otherwise   */
  int64_t tile_records[3];    /* records of the register-tile products: A2,   */
                              /* A2^T (2 x 2 row tiles) and A1^T (2 x 2 pixel */
                              /* tiles); 0 where that product runs row-wise   */
} srt_plan_info_t;

/*
 * Fill *g with the default readings: rings at the cell centres of the volume
 * height [-mz dz/2, mz dz/2], radius grid [R - r, R + r] with r = ms dxy /
 * sqrt(2) (the in-plane half diagonal), phi0 = 0, FP32 weights, no flags,
 * the whole aperture (n_phi_total = phi_first = 0).
 * Returns SRT_ERR_ARG for a null g.
 */
int srt_geometry_default(srt_geometry* g, int32_t ms, int32_t mz, double dxy, double dz,
                         double radius, int32_t n_phi, int32_t n_zs, int32_t n_ell);

/*
 * Build a plan on the current device (Sec. 3.1): assemble A1 and A2 from
 * exact FP64 arc lengths, then the transposes A1^T, A2^T used by the adjoint
 * (Sec. 3.2), all by device kernels on `stream`.  Synchronises the stream
 * before returning.  The plan owns its device memory and is immutable: it may
 * be used concurrently from several streams with distinct workspaces.
 * Errors: SRT_ERR_ARG (null), SRT_ERR_GEOMETRY (invalid geometry, nnz >=
 * 2^31), SRT_ERR_OOM, SRT_ERR_CUDA.  On error *out is set to NULL.
 */
int srt_plan(const srt_geometry* g, void* stream, srt_plan_t* out);

/* Sizes of a plan.  Errors: SRT_ERR_ARG. */
int srt_plan_info(srt_plan_t plan, srt_plan_info_t* out);

/*
 * Device workspace, in bytes, that srt_forward / srt_adjoint need for `batch`
 * volumes (intermediates of Algorithm 1/2).  Errors: SRT_ERR_ARG.
 */
int srt_workspace_bytes(srt_plan_t plan, int32_t batch, size_t* bytes);

/*
 * Forward transform, Algorithm 1 on every sensor column at once:
 *   f: device, float[batch][ms][ms][mz]        (read only, z fastest)
 *   p: device, float[batch][n_phi][n_zs][n_ell] (overwritten, never accumulated)
 *   workspace: device, >= srt_workspace_bytes(batch), 256-byte aligned; the
 *   caller owns it; concurrent calls need distinct workspaces.
 * f, p must be 16-byte aligned.  Asynchronous on `stream`.  The device that
 * was current when the plan was made must be current.
 * Errors: SRT_ERR_ARG (also: another device current), SRT_ERR_WORKSPACE,
 * SRT_ERR_CUDA (launch failure).
 */
int srt_forward(srt_plan_t plan, const float* f, float* p, int32_t batch, void* workspace,
                size_t workspace_bytes, void* stream);

/*
 * Matched adjoint, Algorithm 2 (A2^T then A1^T, gather form, no atomics):
 *   p: device, float[batch][n_phi][n_zs][n_ell] (read only)
 *   f: device, float[batch][ms][ms][mz]         (overwritten)
 * Same workspace, alignment and error rules as srt_forward.
 */
int srt_adjoint(srt_plan_t plan, const float* p, float* f, int32_t batch, void* workspace,
                size_t workspace_bytes, void* stream);

/*
 * End-to-end variants on HOST buffers (same layouts as above; pinned memory
 * gives full copy speed).  The call copies the input to the device, runs the
 * transform in `workspace` and copies the result back, then synchronises.
 * The result is copied back in four chunks on a copy stream the call creates,
 * each as soon as the transform has produced it (the forward's second product
 * and reshape, and the adjoint's A1^T product, run in four row ranges), so
 * most of the device-to-host copy overlaps the computation; results are
 * bitwise those of srt_forward / srt_adjoint.  These calls record no
 * per-stage timing.  `workspace` must hold srt_host_workspace_bytes(batch)
 * bytes of device memory (device copies of input and output plus the
 * transform workspace).  The copy stream and its events come from a pool on
 * the plan, created at a call's first use and reused by later calls (a call
 * that overlaps another on the same plan takes a second set).
 * Errors: as srt_forward.
 */
int srt_host_workspace_bytes(srt_plan_t plan, int32_t batch, size_t* bytes);
int srt_forward_host(srt_plan_t plan, const float* f_host, float* p_host, int32_t batch,
                     void* workspace, size_t workspace_bytes, void* stream);
int srt_adjoint_host(srt_plan_t plan, const float* p_host, float* f_host, int32_t batch,
                     void* workspace, size_t workspace_bytes, void* stream);

/*
 * Pipelined host-buffer calls: a sequence of forward and adjoint calls on
 * HOST buffers with up to `slots` (2-4) in flight, so that a call's input
 * copy overlaps earlier calls' computation and its result copy (one copy,
 * after the transform) overlaps later calls'.  Results are bitwise those of srt_forward_host /
 * srt_adjoint_host.  (The paper has no counterpart; this is the serving-side
 * form of the host-buffer calls.)
 *   srt_pipe_create: device buffers for `slots` calls of `batch` volumes
 *     (an input and an output buffer per slot, each the larger of f and p,
 *     plus one transform workspace) and three streams of its own (input
 *     copies, computation, result copies).  More slots give a slow copy
 *     more time to finish before its call's transform is due.  Errors:
 *     SRT_ERR_ARG (slots outside 2-4, or another device current than the
 *     plan's), SRT_ERR_OOM, SRT_ERR_CUDA; on error *pipe is set to NULL.
 *   srt_pipe_submit: enqueue one call (direction 0 = forward, f_host ->
 *     p_host; 1 = adjoint, p_host -> f_host) and return without waiting;
 *     *ticket (may be NULL) numbers the calls 0, 1, 2, ...  Call i uses slot
 *     i % slots and starts its input copy once call i - slots has consumed
 *     that slot's input.  in_host and out_host must stay allocated and unchanged
 *     (out_host unread) until srt_pipe_wait(ticket) has returned SRT_OK;
 *     pinned memory gives full copy speed.  The calls run in submission
 *     order.  Errors: SRT_ERR_ARG (null pipe or buffer, bad direction,
 *     another device current than the plan's), SRT_ERR_CUDA.
 *   srt_pipe_wait: block until call `ticket`'s result is in its host buffer
 *     (polling, at most timeout_s seconds; a negative timeout waits without
 *     limit).  Errors: SRT_ERR_ARG (unknown ticket), SRT_ERR_TIMEOUT,
 *     SRT_ERR_CUDA (a failure in this or an earlier call of the pipe).
 *   srt_pipe_stage_times: for a finished call among the last 8 submitted,
 *     ms[0..3] = input copy,
 *     transform and result copy durations, and the idle time of the compute
 *     stream between the previous call's transform and this one's (0 for
 *     the first call), in milliseconds from CUDA events.  Errors:
 *     SRT_ERR_ARG, SRT_ERR_NOT_READY (not finished, or older than the last 8).
 *   srt_pipe_destroy: wait for every call, then free the pipe (NULL is a
 *     no-op).  Not thread safe: one host thread drives a pipe.
 */
typedef struct srt_pipe_s* srt_pipe_t;
int srt_pipe_create(srt_plan_t plan, int32_t batch, int32_t slots, srt_pipe_t* pipe);
int srt_pipe_submit(srt_pipe_t pipe, int32_t direction, const float* in_host, float* out_host,
                    int64_t* ticket);
int srt_pipe_wait(srt_pipe_t pipe, int64_t ticket, double timeout_s);
int srt_pipe_stage_times(srt_pipe_t pipe, int64_t ticket, float* ms);
int srt_pipe_destroy(srt_pipe_t pipe);

/*
 * Forward transform that allocates nothing, for callers that cannot hand the
 * library a device workspace: programs whose device memory is owned by another
 * allocator that forbids direct cudaMalloc/cudaFree, code running in callbacks
 * or plug-ins that may not allocate, and latency-critical loops that cannot
 * afford an allocation.  (The paper has no counterpart; this is an interface
 * convenience.)  Same inputs, output and layouts as srt_forward; instead of a
 * caller workspace it uses a scratch array of SRT_NOALLOC_WORKSPACE_BYTES that
 * the library keeps in device memory on every GPU that loads it, until the
 * process exits.
 *   - Returns SRT_ERR_WORKSPACE when srt_workspace_bytes(plan, batch) exceeds
 *     SRT_NOALLOC_WORKSPACE_BYTES (use srt_forward then), SRT_ERR_ARG when the
 *     plan was made on a different device than the current one.
 *   - The first call on a device looks up the scratch array's device address
 *     (a runtime call, cudaGetSymbolAddress); make that first call before any
 *     stream capture begins.  The address is kept for the life of the
 *     process: calls after cudaDeviceReset on that device are not supported
 *     (the reset unloads the library's device code and may move the array).
 *   - All calls on a device share the scratch, which keeps the last call's
 *     contents (no element needs to start at zero).  Calls whose work overlaps
 *     on the GPU race on it: order them on one stream.
 */
#define SRT_NOALLOC_WORKSPACE_BYTES (32u << 20)
int srt_forward_noalloc(srt_plan_t plan, const float* f, float* p, int32_t batch, void* stream);
/* The matched adjoint (as srt_adjoint) on the same scratch, with the same
 * limits, errors and ordering rule. */
int srt_adjoint_noalloc(srt_plan_t plan, const float* p, float* f, int32_t batch, void* stream);

/*
 * Debug builds (the library compiled with -DSRT_CHECKS; the package's
 * build.build_checked() makes one): every product kernel checks each
 * gathered row index against the row count of the operand it reads, before
 * the access.  An index outside the operand is counted and replaced by row 0,
 * so it is reported without a fault; srt_forward / srt_adjoint and the
 * host-buffer calls (and the no-alloc calls, which run them) then
 * synchronise their stream and return SRT_ERR_CUDA if a check failed during
 * the call (pipelined calls are reported by srt_checks_read only).
 *   srt_checks_read: *violations = indices found outside their operand since
 *     the last read (synchronises the device), then resets the count.
 *   srt_checks_cap: count every operand as having at most `rows` rows (0: no
 *     cap), so that a test can make in-range indices trip the check without
 *     any access outside an operand.
 * Release builds compile the checks away; both calls return SRT_ERR_ARG there.
 */
int srt_checks_read(int64_t* violations);
int srt_checks_cap(int32_t rows);

/*
 * FP64 inner product on the device: *out = sum_i (double)a[i] * (double)b[i],
 * summed in a fixed order (deterministic).  a, b: device float[n]; out:
 * device double[1]; workspace: device, >= srt_dot_workspace_bytes() bytes.
 * Used for adjoint-identity checks <A f, g> = <f, A^T g>.
 * Errors: SRT_ERR_ARG, SRT_ERR_WORKSPACE, SRT_ERR_CUDA.
 */
size_t srt_dot_workspace_bytes(void);
int srt_dot_f64(const float* a, const float* b, int64_t n, double* out, void* workspace,
                size_t workspace_bytes, void* stream);

/*
 * Copy an assembled operator to HOST memory, for inspection and tests.
 *   which: 1 = A1, 2 = A2, 3 = A1^T, 4 = A2^T.
 *   rowptr: int32[rows+1]; col: int32[nnz]; val32: float[nnz] (the stored
 *   entries widened to FP32; may be NULL); val64: double[nnz] (the FP64
 *   entries before rounding; requires SRT_KEEP_F64; may be NULL).
 *   Rows are sorted by column index.  Synchronous.
 * Errors: SRT_ERR_ARG (bad which, null rowptr/col, val64 without the flag),
 * SRT_ERR_CUDA.
 */
int srt_plan_export(srt_plan_t plan, int32_t which, int32_t* rowptr, int32_t* col, float* val32,
                    double* val64);

/*
 * Per-stage timing with CUDA events recorded on the launch stream.
 * srt_plan_set_timing(plan, 1) makes every later srt_forward / srt_adjoint
 * record events around each kernel stage; srt_stage_times(plan, dir, ms, n)
 * then returns, for the LAST call in direction dir (0 forward, 1 adjoint), the
 * elapsed milliseconds of its stages in launch order (n >= 4: first SpMM,
 * permute, second SpMM, permute) after synchronising on the last event.
 * With the fused reshapes (SRT_FUSE_RESHAPES) a fused permute's stage
 * reads 0 and its time is part of the product before it (A1 for P1, A2 for
 * P2, A2^T for P1^-1).
 * Not for use with stream capture.  Errors: SRT_ERR_ARG, SRT_ERR_NOT_READY.
 */
int srt_plan_set_timing(srt_plan_t plan, int32_t enable);
int srt_stage_times(srt_plan_t plan, int32_t dir, float* ms, int32_t n);

/* Number of kernel launches one srt_forward (dir 0) or srt_adjoint (dir 1)
 * call on `batch` volumes makes: 4 (two products, two reshapes), fewer with
 * SRT_FUSE_RESHAPES.  0 for a null plan, batch <= 0 or another dir. */
int srt_launches_per_call(srt_plan_t plan, int32_t dir, int32_t batch);

/*
 * Measurement helper (no counterpart in the paper): the FP32 FMA rate the
 * CUDA cores of the current GPU sustain, in TFLOP/s, from a kernel of
 * independent FMA chains (8 blocks of 256 threads per SM, 16 chains per
 * thread, iters FMAs per chain) timed with CUDA events on `stream` after one
 * warm-up launch.  Synchronous.  This is the arithmetic roof of the sparse
 * products (Sec. 3.1 products run on the CUDA cores, not tensor cores).
 * Errors: SRT_ERR_ARG (null tflops, iters <= 0), SRT_ERR_CUDA.
 */
int srt_fp32_fma_peak(int32_t iters, double* tflops, void* stream);

/* Release the plan's device memory.  NULL is accepted.  Not stream-ordered:
 * the caller must ensure no work using the plan is still in flight. */
int srt_plan_destroy(srt_plan_t plan);

/* Static description of a status code. */
const char* srt_error_string(int code);

#ifdef __cplusplus
}
#endif

#endif /* SRT_H */
