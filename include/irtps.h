/*
 * irtps.h — C ABI of the GB300 IRT-PS library (Iterative Ray Tracing
 * Photometric Stereo; Khadka, Remagnino, Argyriou, arXiv:1811.02357).
 *
 * One context holds one object: an H x W pixel grid seen orthographically along
 * -z, K distant white lights, C colour channels (1 or 3) and a known
 * environment.  All device memory is allocated and owned by the context; every
 * caller buffer is only read or written during the call that receives it.
 *
 * Geometry and units.  Pixel (i, j), row i in [0, H), column j in [0, W),
 * linear index p = i*W + j, pixel pitch h = 1/W (object width 1); the depth
 * H_ij is in the same unit; +z points to the viewer; a normal is
 * n ~ (-dH/dx, -dH/dy, 1) with y increasing with i.  The surface is meshed
 * with vertices at the pixel centres, two triangles per cell.  The environment
 * is a C x EH x EW latitude-longitude map over the full sphere: rows cover
 * theta = acos(w_z) in [0, pi], columns phi = atan2(w_y, w_x) in [0, 2 pi).
 *
 * Array layouts (all row-major, float32 unless noted):
 *   lights   K x 3 unit vectors, z > 0                    (Eq. 3, matrix L)
 *   env      C x EH x EW
 *   images   K x C x H x W (float32 or float16)           (stage 0 input A)
 *   depth    H x W
 *   normals  H x W x 4: nx, ny, nz, mean albedo           (Eq. 4 output)
 *   albedo   C x H x W
 *   indirect K x C x H x W: Lbar, the mean incident radiance of the
 *            reverted trace (irradiance = pi * Lbar); the subtracted image is
 *            rho * Lbar                                   (Eq. 7, E^r_t)
 *
 * Status.  Every call returns IRTPS_OK (0) or a negative code; the message of
 * the last failure is available from irtps_last_error.  A CUDA failure
 * (IRTPS_ECUDA) leaves the context unusable except for irtps_destroy.
 * Contexts are not thread-safe: use one context per host thread.
 */
#ifndef IRTPS_H
#define IRTPS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define IRTPS_OK 0
#define IRTPS_EINVAL (-1)    /* bad argument or size outside the supported range */
#define IRTPS_ENOMEM (-2)    /* device or pinned host allocation failed */
#define IRTPS_ECUDA (-3)     /* a CUDA runtime call or kernel launch failed */
#define IRTPS_ENOTREADY (-4) /* irtps_iterate / irtps_solve_normals before irtps_set_images */
#define IRTPS_ETIMEOUT (-5)  /* a bounded device loop gave up (step budget exhausted) */
#define IRTPS_ENUMERIC (-6)  /* non-finite values, or the depth solve did not converge */

#define IRTPS_F32 0
#define IRTPS_F16 1

#define IRTPS_MAX_LIGHTS 64

typedef struct irtps_ctx irtps_ctx;

/* Tunables.  Fill with irtps_default_options, then override. */
typedef struct irtps_options {
  int shadow_rays;    /* 1: light visibility at every hit by a shadow ray (default 1) */
  float tau_lo;       /* a row k of pixel p takes part in the normal solve iff     */
  float tau_hi;       /* tau_lo < mean_c I(p,k,c) < tau_hi (0.02, 0.98)             */
  double cond_max;    /* masked 3x3 solves with 1-norm condition above this: invalid pixel (1e8) */
  float nz_min;       /* n_z clamp of the slopes -n_x/n_z, -n_y/n_z (0.05) */
  double cg_tol;      /* depth solve: stop at FP64 |b - A x| / |b| <= cg_tol (1e-9) */
  int cg_max_iter;    /* depth solve iteration cap (50000) */
  int cg_check_every; /* FP64 true-residual refresh and convergence test period (10) */
  double stop_tol;    /* irtps_iterate stops early when D_H < stop_tol; 0 = never (0) */
  int precond;        /* depth solve: 0 Jacobi-preconditioned CG, 1 multigrid-preconditioned CG,
                         2 direct: unit-weight solves of grids up to 1024 x 1024 by the cosine
                         transform that diagonalises the grid Laplacian (four FP64 transform
                         products, then the same FP64 residual check against cg_tol); weighted
                         (irls) solves, larger grids and batches use multigrid (2) */
  int use_graph;      /* 1: irtps_iterate captures one iteration as a CUDA graph and replays it (0);
                         per-stage times are then not measured (reported as 0) */
  int sampling;       /* trace sampling (0):
                         0 per light: spp paths for every (pixel, light), counter light field k;
                         1 light-shared: spp paths per pixel serve all K lights (counter light
                           field 0; at each hit one shadow ray per light facing the hit normal);
                           the same expectation with about K times fewer path segments */
  int irls_iters;     /* integration by the Huber M-estimator: reweighting steps after the
                         least-squares solve (0 = least squares only) (0) */
  float irls_delta;   /* Huber threshold on the edge slope residual (H_b - H_a)/h - mean slope (0.05) */
  int early_escape;   /* before a trace, bound every pixel's horizon in eight octants of azimuth
                         from the max pyramid (a fixed scan of nodes around the pixel per level);
                         a rising primary ray above it skips its march after the triangle test of
                         its first cell (results unchanged, bit for bit).  0 off, 1 on, 2 where it
                         pays: per-light sampling, at least 16 samples per item, and H W K >= 2^18
                         work items (a smaller object cannot fill the GPU; in a batch any size) (2) */
  int fill_holes;     /* 1: the single-sample variant of Sec. IV (per-light sampling only): a (pixel,
                         light) none of whose samples hit the surface with its first segment has no
                         environment value (a hole); after every trace of the IRT loop (irtps_iterate,
                         irtps_trace) Lbar at the holes is replaced by a non-uniform interpolation
                         of the known pixels of the same light and channel (pull-push normalised
                         convolution: confidence-weighted 2x2 means up a pyramid to 1 x 1, then
                         confidence blends with the 2x linear upsampling of the coarser level back
                         down; known pixels keep their values, a light without known pixels keeps
                         its traced values) (0) */
  int ps_tensor;      /* subtract + PS (Eq. 4) of a single context: 0 the contraction on the FP32
                         pipes (1, 2 or 4 pixels a thread, vector loads; pinv(L) I, or (L^T L)^-1 L^T I
                         when L^T L is well conditioned); 1 on the tensor cores (tcgen05, 128 pixels a
                         tile, BF16 hi + lo split of I and pinv(L), FP32 accumulation:
                         I_hi P_hi + I_lo P_hi + I_hi P_lo).  Row masks and masked pixels are decided
                         and solved identically in both (FP32 masks; masked 3x3 systems in FP32 when
                         well conditioned, else double-float sums with an FP64 inverse and condition
                         number).  Batches use the FP32 form (0) */
} irtps_options;

/* Counters of the last irtps_iterate / irtps_trace / irtps_integrate call. */
typedef struct irtps_stats {
  unsigned long long primary_segments; /* primary rays: pixels * K * spp per trace */
  unsigned long long segments;         /* all traced segments incl. bounces and shadow rays */
  unsigned long long walk_overflows;   /* marches that hit their step budget (expected 0) */
  int cg_iterations;                   /* CG iterations of the last depth solve */
  double cg_rel_residual;              /* FP64 |b - A x| / |b| at its end */
  double dH_max;                       /* D_H of the last iteration: max |dH| / range(H) */
  double dH_rms;                       /* RMS of H_{t+1} - H_t */
  int iterations_done;                 /* IRT iterations completed by the last irtps_iterate */
  unsigned long long node_visits;      /* pyramid nodes and cells examined by the marches */
  unsigned long long tri_tests;        /* ray / triangle tests */
  double trace_ms;                     /* device time of the trace kernel(s), CUDA events */
  double ps_ms;                        /* device time of the subtract + PS kernel(s) */
  double depth_ms;                     /* device time of the depth solve(s) incl. host checks */
  unsigned long long launches;         /* kernels launched since irtps_create (cumulative) */
  unsigned long long draws;            /* sampled directions (primary and bounce segments) */
  double fill_ms;                      /* device time of the hole interpolation (fill_holes) */
} irtps_stats;

/* Defaults listed beside each field of irtps_options. */
void irtps_default_options(irtps_options *opt);

/* Create a context for an H x W object (H, W >= 2; H*W*K < 2^31), K lights
 * (3 <= K <= 64, at least three non-coplanar: Eq. 4 needs (L^T L)^-1), C in {1, 3},
 * environment EH x EW (>= 1).  lights, env: host pointers, copied.  opt may be
 * NULL (defaults).  (L^T L)^-1 L^T is formed on the host in FP64 (Eq. 4). */
int irtps_create(irtps_ctx **out, int H, int W, int K, int C, const float *lights, const float *env, int EH,
                 int EW, const irtps_options *opt);

/* Run all later work on `stream` (a cudaStream_t, e.g. torch's current stream);
 * NULL restores the context's own stream.  The caller keeps the stream alive. */
int irtps_set_stream(irtps_ctx *ctx, void *stream);

/* Stage 0 / stage 1 (Sec. IV): take the K input images (dtype IRTPS_F32 or
 * IRTPS_F16; host pointer if on_device == 0, else a device pointer readable on
 * the context stream) and run iteration 0: classic PS (Eq. 4; pixels with masked
 * rows solved from their valid rows) and integration of the normals into the surface H_0.
 * Resets the IRT iteration index to 0. */
int irtps_set_images(irtps_ctx *ctx, const void *images, int dtype, int on_device);

/* IRT iterations (Sec. IV, stages 4-5 and the loop): n_iter times
 *   build the min/max pyramid of H_t; trace Lbar_t over (H_t, n_t, rho_t) with
 *   spp samples per (pixel, light) (per pixel with light-shared sampling) and
 *   bounces in 1..3 (the paper's r1..r3);
 *   I = A0 - rho_t * Lbar_t (subtracted from the ORIGINAL images); PS -> n, rho;
 *   integrate -> H_{t+1} (least squares, or the Huber M-estimator with
 *   irls_iters > 0); D_H = max|H_{t+1} - H_t| / range(H_{t+1}).
 * Random draws: Philox4x32-10, key {seed_lo ^ object, seed_hi}, counter
 * {pixel, sample, light<<8 | bounce<<4 | 0, t} (light field 0 with light-shared
 * sampling); t advances by one per iteration.
 * out_dH (nullable host pointer) receives D_H of the last iteration. */
int irtps_iterate(irtps_ctx *ctx, int n_iter, int spp, int bounces, uint64_t seed, double *out_dH);

/* Single stages over the current state, for staged use and testing. */
/* Trace only: Lbar over the current (depth, normals, albedo) with iteration
 * field `iteration` and stream tag `stream_tag` (0 for the IRT loop, 1 for the
 * forward render) in the Philox counter; result in the context's indirect buffer. */
int irtps_trace(irtps_ctx *ctx, int spp, int bounces, uint64_t seed, uint32_t iteration, uint32_t stream_tag);
/* Subtract + PS: images minus albedo * indirect, then Eq. 4 per pixel. */
int irtps_solve_normals(irtps_ctx *ctx);
/* Integrate the current normals into the depth (the CG solves warm-start from the current depth;
 * the direct solve of precond = 2 needs no start). */
int irtps_integrate(irtps_ctx *ctx);

/* Trace a list of pixels only (host arrays): out_lbar K x C x n_pix;
 * out_rec (nullable) n_pix x K x spp x bounces x 2 int32 per segment:
 * {hit pixel | -1 escape | -2 not reached, shadow visibility 1 | 0 | -1 not cast};
 * with light-shared sampling n_pix x spp x bounces x (1 + K):
 * {hit pixel | -1 | -2, then the visibility of each light 1 | 0 | -1 not cast | -2}. */
int irtps_trace_pixels(irtps_ctx *ctx, const int32_t *pixels, int n_pix, int spp, int bounces, uint64_t seed,
                       uint32_t iteration, uint32_t stream_tag, float *out_lbar, int32_t *out_rec);

/* Replace the current estimate (host arrays): depth H x W, normals H x W x 3
 * (unit), albedo C x H x W.  Any of them may be NULL to keep the current one. */
int irtps_set_state(irtps_ctx *ctx, const float *depth, const float *normals, const float *albedo);
/* Replace the indirect buffer (host, K x C x H x W). */
int irtps_set_indirect(irtps_ctx *ctx, const float *indirect);

/* Synthetic stage-0 images of the current state taken as ground truth
 * (test-input generation): A0 = rho max(0, n.l) V + rho Lbar_gt + sigma z with
 * Lbar_gt traced with stream tag 1 and iteration 0xFFFFFFFF (left in the
 * indirect buffer), z ~ N(0,1) from Philox.  out: K x C x H x W float32, host
 * or device (on_device). */
int irtps_render(irtps_ctx *ctx, int spp, int bounces, uint64_t seed, float sigma, float *out, int on_device);

/* Copies of the state (host pointer if on_device == 0, else device). */
int irtps_get_normals(irtps_ctx *ctx, float *out, int on_device);   /* H x W x 4 */
int irtps_get_albedo(irtps_ctx *ctx, float *out, int on_device);    /* C x H x W */
int irtps_get_depth(irtps_ctx *ctx, float *out, int on_device);     /* H x W, mean 0 */
int irtps_get_indirect(irtps_ctx *ctx, float *out, int on_device);  /* K x C x H x W */
int irtps_get_valid(irtps_ctx *ctx, uint8_t *out, int on_device);   /* H x W, 1 = normal solved */
/* K x H x W, 1 = hole of the last whole-field trace (contexts created with
 * fill_holes only; IRTPS_EINVAL otherwise). */
int irtps_get_holes(irtps_ctx *ctx, uint8_t *out, int on_device);
int irtps_get_stats(irtps_ctx *ctx, irtps_stats *out);

/* Geometry probes for the parity tests.  Host arrays.
 * irtps_probe_dirs: cosine-weighted directions (Eq. 7 sampling) for n unit
 * normals (n x 3) and raw Philox words x0, x1 -> out n x 3.
 * irtps_probe_rays: closest hit of n grid-space rays (n x 6: origin, direction;
 * vertex (i, j) at (j, i, depth)) with the current depth's mesh -> t (NaN on a
 * miss) and triangle index 2*(cell_row*(W-1) + cell_col) + {0, 1} (-1). */
int irtps_probe_dirs(int n, const float *normals, const uint32_t *x0, const uint32_t *x1, float *out);
int irtps_probe_rays(irtps_ctx *ctx, int n, const float *rays, float *out_t, int32_t *out_tri);

/* The hole interpolation of fill_holes on caller data (Sec. IV: the missing
 * pixels of single-sample environment images filled by a non-uniform
 * interpolation), for staged use and testing.  Host arrays:
 *   values : K x C x H x W float, in place; known pixels keep their values,
 *            holes get the interpolation (their input values are ignored); an
 *            image (k) without known pixels is left unchanged
 *   holes  : K x H x W uint8, nonzero = missing
 * C in {1, 3}, K, H, W >= 1, K*C*H*W < 2^31.  Allocates its device buffers for
 * the call and returns after the result is copied back.  IRTPS_EINVAL on bad
 * arguments, IRTPS_ENOMEM / IRTPS_ECUDA on CUDA failures. */
int irtps_interpolate_holes(float *values, const uint8_t *holes, int K, int C, int H, int W);

/* Depth integration without any device allocation.  The paper has no
 * counterpart: this entry exists for callers that cannot allocate device memory
 * when they need the surface (a host framework that owns the whole device pool
 * through its own allocator, or a latency-critical loop that cannot accept the
 * device-wide synchronisation of cudaMalloc / cudaFree).  It always runs the
 * unweighted least-squares solve by Jacobi-preconditioned CG (FP32 vectors, the
 * FP64 residual refreshed every 10 iterations), whatever the options of any
 * context, so its surface agrees with irtps_integrate (which by default solves
 * directly by the cosine transform) to within the solver tolerance, not bit for
 * bit.  Its working vectors live in one file-scope device array that holds at
 * most 512 x 512 = 262144 pixels (about 11 MB, kept by every GPU that loads the
 * library until the process exits).
 *   normals : device, H x W x 4 float (nx, ny, nz, unused), read only
 *   depth   : device, H x W float; in: warm start, out: the surface, mean 0
 *   nz_min, tol, max_iter: as irtps_options.nz_min, cg_tol, cg_max_iter
 *   stream  : cudaStream_t to run on (NULL: the legacy default stream); the call
 *             returns after the work on it has finished
 * Returns IRTPS_EINVAL for H or W < 2, H*W > 262144 or bad tolerances,
 * IRTPS_ENUMERIC if the residual stays above tol, IRTPS_ETIMEOUT if a grid
 * barrier gave up, IRTPS_ECUDA on a CUDA failure (after waiting for the work it
 * had queued).  The first call on a device looks up the array's device address
 * and keeps it for the life of the process (make that first call before any
 * stream capture; a cudaDeviceReset invalidates the kept address, so the entry
 * point is not for use across device resets).  All calls share the array: calls
 * that overlap on the GPU race and must not be issued. */
int irtps_integrate_noalloc(const float *normals, int H, int W, float nz_min, double tol, int max_iter, float *depth,
                            void *stream);

const char *irtps_last_error(const irtps_ctx *ctx);
void irtps_destroy(irtps_ctx *ctx);

/* Object index of a context: the `object` term of its Philox key
 * {seed_lo ^ object, seed_hi} (0 after irtps_create). */
int irtps_set_object(irtps_ctx *ctx, uint32_t object);

/* Scheduling tunables of a context's trace, chosen by irtps_autotune or set
 * directly.  Neither changes any result bit: work items are traced one per lane
 * in sample order whatever the grid, and the pyramid skip lands in the cell the
 * plain walk reaches whatever the number of levels.
 *   blocks_per_sm : resident 128-thread blocks per SM of the persistent trace
 *                   grid (1 .. occupancy limit; 0 = the occupancy limit)
 *   mip_cut       : top levels of the min/max pyramid the march leaves out
 *                   (0 = full depth; clamped so that two levels remain) */
int irtps_set_tuning(irtps_ctx *ctx, int blocks_per_sm, int mip_cut);
int irtps_get_tuning(irtps_ctx *ctx, int *blocks_per_sm, int *mip_cut);
/* Pixels per thread of the FP32 subtract + PS kernel (Eq. 4; ps_tensor = 0):
 * 1, 2 or 4 consecutive pixels, one vector load per plane row for all of them
 * (0 = the default, 2).  A grid whose pixel count is not a multiple of the width
 * runs one pixel per thread.  No result bit depends on it. */
int irtps_set_ps_tuning(irtps_ctx *ctx, int pixels_per_thread);
int irtps_get_ps_tuning(irtps_ctx *ctx, int *pixels_per_thread); /* the width in use */
/* Time the trace of the current state with spp_probe samples for each candidate
 * (blocks_per_sm, mip_cut) and keep the fastest; right after irtps_set_images
 * (iteration 0) it also times the PS widths 1, 2, 4 by re-running classic PS,
 * which rewrites the normals and albedo the context already holds, bit for bit.
 * Writes the indirect buffer (re-trace before using it).  out_ms (nullable)
 * receives the best trace time. */
int irtps_autotune(irtps_ctx *ctx, int spp_probe, int bounces, uint64_t seed, double *out_ms);

/* ---- Batches: many objects, one launch per IRT stage ----
 * A batch runs the IRT loop of n_obj contexts together: per iteration one
 * batched pyramid launch per level, ONE persistent trace launch whose lanes take
 * (object, light, pixel) work items from a shared queue (objects of larger
 * per-item cost first), one PS launch, one cooperative depth-solve launch in
 * which each object's solve runs on its own team of blocks, and one D_H launch.
 * Objects may differ in H, W, K, spp, bounces and options; all must have the
 * same C, image dtype, sampling option and irls_iters (robust integration runs
 * the same number of reweighting steps for every object; irls_delta may differ),
 * and none may have fill_holes (hole interpolation runs per context).  Every object's results are bit-identical to its own
 * irtps_iterate in the trace and the normal solve; the depth solve differs from
 * it only by the summation order of its reductions (team size), within cg_tol.
 *
 * The batch keeps pointers to the caller's contexts, which must outlive it and
 * must not be used concurrently with a batch call.  irtps_batch_create sets the
 * object index of context i to i (irtps_set_object).  n_obj in 1..64. */
typedef struct irtps_batch irtps_batch;
int irtps_batch_create(irtps_batch **out, irtps_ctx *const *objs, int n_obj, int use_graph);
/* Run the batch's work on `stream` (a cudaStream_t); NULL restores its own
 * stream.  The batch orders itself after the work queued on every object's
 * stream and every object's stream after the batch's work. */
int irtps_batch_set_stream(irtps_batch *b, void *stream);
/* Stage 0 / iteration 0 of every object, batched: copy images[i] (K_i x C x H_i
 * x W_i, dtype IRTPS_F32 or IRTPS_F16, host pointers if on_device == 0, else
 * device pointers readable on the batch stream) into object i, then classic PS
 * (Eq. 4) and integration for all objects, as irtps_set_images does for one.
 * Results equal irtps_set_images' up to the summation order of the solve. */
int irtps_batch_set_images(irtps_batch *b, const void *const *images, int dtype, int on_device);
/* n_iter IRT iterations of every object (each context must have images set):
 * spp[i], bounces[i] for object i (host arrays of n_obj; bounces in 1..3); seed
 * as in irtps_iterate.  Object i's iteration index advances by n_iter.
 * out_dH (nullable, host, n_obj) receives each object's D_H of the last
 * iteration.  With use_graph, one iteration is captured as a CUDA graph and
 * replayed (re-captured when spp, bounces or seed change). */
int irtps_batch_iterate(irtps_batch *b, int n_iter, const int *spp, const int *bounces, uint64_t seed, double *out_dH);
/* Sums over the objects of the last irtps_batch_iterate (cg_iterations: the
 * largest of the last solves, cg_rel_residual: the largest, dH_max: the largest). */
int irtps_batch_get_stats(irtps_batch *b, irtps_stats *out);
/* Trace grid of the batch, as irtps_set_tuning (mip_cut applies to every object). */
int irtps_batch_set_tuning(irtps_batch *b, int blocks_per_sm, int mip_cut);
int irtps_batch_get_tuning(irtps_batch *b, int *blocks_per_sm, int *mip_cut);
/* As irtps_autotune for the batched trace launch (writes every object's indirect buffer). */
int irtps_batch_autotune(irtps_batch *b, const int *spp_probe, const int *bounces, uint64_t seed, double *out_ms);
const char *irtps_batch_last_error(const irtps_batch *b);
void irtps_batch_destroy(irtps_batch *b);

#ifdef __cplusplus
}
#endif

#endif /* IRTPS_H */
