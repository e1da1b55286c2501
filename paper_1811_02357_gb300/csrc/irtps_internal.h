// Internal state of one IRT-PS context and the launchers behind the C ABI.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/irtps.h"
#include "geom.cuh"

namespace irtps {

constexpr int kMaxLights = 64;

// Control block of the cooperative depth-solve loop (see poisson.cu).
struct CGCtl {
  unsigned count, gen;  // grid-barrier state
  int err;              // a barrier poll ran out
  int iters;            // iterations of the last solve
  double rel;           // FP64 |b - A x| / |b| (start, then at the end)
  double bnorm;         // |b|; 0 for a flat right-hand side
};

// Accumulated over the depth solves of one call (read once at its end).
struct CGAcc {
  unsigned long long iters;  // all iterations
  double rel_last;           // relative residual of the last solve
  int err;                   // some barrier timed out
  int bad;                   // some solve ended above tolerance or non-finite
  int last_iters;            // iterations of the last solve
  int pad;
};

// Device-side results of one call, read by the host once at its end.
struct DevStats {
  unsigned long long counts[8];  // {unused, segments, walk overflows, node visits, triangle tests, draws,
                                 //  tensor-core PS waits that ran out}
  CGAcc cg;
  double dh_max, dh_rms;         // D_H of the last iteration
};
constexpr int kCounters = 7;  // used slots of DevStats::counts

// Per-object trace descriptor: the current surface and state estimates, the
// environment, the lights and the output of one object.
struct ObjTrace {
  Field f;
  const float4 *nrm;      // H*W (nx, ny, nz, mean albedo)
  const float *albedo;    // C*H*W
  const float *env;       // C*EH*EW
  const float *lights;    // K*3, unit, z > 0
  float *out;             // K*C*n_pix
  uint2 key;              // Philox key {seed_lo ^ object, seed_hi}
  int EH, EW, K, spp, bounces, n_pix, shadow;
  float eps, Wf;          // ray-origin lift; W (grid units per world unit in x and y)
  unsigned item_begin;    // first work item of the object (batched launches)
  uint32_t iter0;         // added to the launch's iteration field
  float *part;            // light-shared sampling: partial sums, n_chunks x n_pix x K x C, then n_chunks x n_pix x C
  int n_chunks, chunk;    // light-shared sampling: sample chunks per pixel and samples per chunk
  const float *hz;        // horizon bounds, 8 octants x H W (null: no early escape)
  uint8_t *hole;          // per-light sampling: K x n_pix, 1 where no sample's first segment hit (null: none)
  int hz_stride;          // H W
};


// Pyramid levels the march uses when the top `cut` levels are left out (at least two remain).
inline int march_levels(int levels, int cut) {
  const int keep = levels < 2 ? levels : 2;
  return levels - cut > keep ? levels - cut : keep;
}

// Levels of the hole-interpolation pyramid: level 0 is the image (h[0] x w[0]),
// each next one halves both sides (rounded up) down to 1 x 1; level l >= 1 starts
// off[l] pixels into the per-image scratch of `total` pixels.
constexpr int kMaxFillLevels = 32;
struct FillPyramid {
  int n = 0;
  int h[kMaxFillLevels] = {0}, w[kMaxFillLevels] = {0};
  size_t off[kMaxFillLevels] = {0};
  size_t total = 0;
};

struct Ctx {
  int H = 0, W = 0, K = 0, C = 0, EH = 0, EW = 0;
  uint32_t obj = 0;
  irtps_options opt{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  bool have_images = false;
  uint32_t t = 0;                 // IRT iteration index of the next irtps_iterate step
  float eps = 0.0f;               // ray-origin lift, 1e-3 of a pixel pitch
  std::string err;

  // host copies
  std::vector<float> h_lights;    // K*3
  std::vector<float> h_pinv;      // 3*K, (L^T L)^-1 L^T rounded to float
  float h_minv[6] = {0};         // (L^T L)^-1 rounded to float: m00 m01 m02 m11 m12 m22
  int normal_eq = 0;              // 1: PS of fully valid pixels as (L^T L)^-1 (L^T I) (cond(L^T L) <= 16)
  float *d_lights = nullptr;      // K*3 on the device (read at trace hits)
  float *horizon = nullptr;       // early escape: horizon bounds of every pixel, 8 x H x W (option)
  float *shared_part = nullptr;   // light-shared trace: partial sums of its sample chunks
  uint8_t *holes = nullptr;       // fill_holes: K x H x W, 1 where the last trace saw no surface point
  float *fill_v = nullptr, *fill_w = nullptr;  // fill_holes: pyramid levels >= 1, K C and K per pixel
  FillPyramid fill_py;
  // spectral depth solve (precond = 2): DCT-II matrices H x H and W x W, path-Laplacian
  // eigenvalues, one H x W work array (FP64)
  double *sp_ch = nullptr, *sp_cw = nullptr, *sp_mu = nullptr, *sp_nu = nullptr, *sp_t = nullptr;
  size_t shared_cap = 0;          // floats in shared_part

  // device buffers (owned)
  float *env = nullptr;           // C*EH*EW
  void *images = nullptr;         // K*C*H*W, float or half
  int images_dtype = IRTPS_F32;
  float *lbar = nullptr;          // K*C*H*W
  float *depth = nullptr;         // H*W
  float *depth_prev = nullptr;    // H*W
  float4 *nrm = nullptr;          // H*W
  float *albedo = nullptr;        // C*H*W
  uint8_t *valid = nullptr;       // H*W, 1 = normal solved
  int *ps_pix = nullptr;          // PS: pixels with masked rows (H*W capacity), their row masks and
  unsigned long long *ps_mask = nullptr;  // right-hand sides (9 floats each), count
  float *ps_rhs = nullptr;
  unsigned *ps_count = nullptr;
  float *pmin = nullptr, *pmax = nullptr;  // pyramid, all levels
  int levels = 0;
  int trace_blocks = 0;           // resident blocks of the persistent trace grid (0: one lane per item)
  int mip_cut = 0;                // top pyramid levels the march leaves out (tuning; results do not change)
  int ps_vec = 2;                 // pixels per thread of the PS kernel, 1, 2 or 4 (tuning; results do not change)
  int sms = 0, trace_per_sm_max = 0;  // SM count; resident trace blocks per SM at full occupancy
  int off[kMaxLevels] = {0}, lw[kMaxLevels] = {0}, lh[kMaxLevels] = {0};
  // depth solve
  double *cg_x = nullptr, *cg_b = nullptr;
  float *cg_r = nullptr, *cg_z = nullptr, *cg_p = nullptr, *cg_ap = nullptr;
  double *part = nullptr;         // reduction partials: kPartSlots slots of part_stride doubles
  int part_stride = 0, cg_blocks = 0;
  double *h_part = nullptr;       // pinned host mirror of one partial slot
  void *cg_ctl = nullptr;         // device control block of the cooperative CG loop
  // multigrid hierarchy of the depth solve (levels of 2x2 aggregates, pooled arrays)
  int mg_levels = 0;
  int mg_h[kMaxLevels] = {0}, mg_w[kMaxLevels] = {0}, mg_off[kMaxLevels] = {0};
  float *mg_x0 = nullptr, *mg_x1 = nullptr, *mg_b = nullptr, *mg_wh = nullptr, *mg_wv = nullptr;
  float *mg_wh_unit = nullptr, *mg_wv_unit = nullptr;  // unit-weight hierarchy (restored after IRLS)
  int mg_total = 0;               // points of all levels
  DevStats *dstats = nullptr;     // device counters of the current call
  unsigned *next_item = nullptr;  // work-item counter of the trace launch
  uint32_t *iter_dev = nullptr;   // IRT iteration index read by replayed graphs
  cudaGraphExec_t graph = nullptr;  // one captured IRT iteration
  int graph_spp = 0, graph_bounces = 0;
  uint64_t graph_seed = 0;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  std::vector<cudaEvent_t> tev;   // start/stop event pairs of the timed stages of one call
  std::vector<int> tev_stage;     // stage of each pair (trace, PS, depth)
  int tev_used = 0;
  irtps_stats stats{};

  Field field() const {
    Field f;
    f.depth = depth;
    f.pmax = pmax;
    f.H = H;
    f.W = W;
    f.Wc = W - 1;
    f.Hc = H - 1;
    f.levels = march_levels(levels, mip_cut);
    f.top_off = off[levels - 1];
    for (int l = 0; l < kMaxLevels; ++l) {
      f.off[l] = off[l];
      f.lw[l] = lw[l];
    }
    return f;
  }
};

constexpr int kPartSlots = 12;

}  // namespace irtps

struct irtps_ctx {
  irtps::Ctx c;
};

namespace irtps {

// Pyramid of one object in a batched build.
struct PyrObj {
  const float *depth;
  float *prev;  // when set, level 0 also copies depth here (D_H reference)
  float *pmin, *pmax;
  int H, W, levels;
  int off[kMaxLevels], lw[kMaxLevels], lh[kMaxLevels];
  int blk[kMaxLevels];  // first block of the object in the launch of each level
  float *hz;            // horizon bounds (null: none)
  int hz_blk;           // first block of the object in the batched horizon launch
};
constexpr int kPyrThreads = 256;

// trace.cu
cudaError_t build_pyramid(Ctx &c);
// Early escape: option 1 always; option 2 where it was measured to pay: per-light
// sampling with at least kEarlyEscapeMinSpp samples per item (fewer do not pay for the
// bounds), on a grid whose work items fill the GPU - at least kEarlyEscapeMinItems
// in a single-object trace (with fewer the launch waits on its longest items, which
// the per-ray test only lengthens), any size in a batch (whose queue fills it).
constexpr int kEarlyEscapeMinSpp = 16;
constexpr long long kEarlyEscapeMinItems = 1ll << 18;
// whether some trace of the context may use the bounds (option 1, or option 2 with per-light sampling)
inline bool early_escape_possible(const Ctx &c) {
  return c.horizon && (c.opt.early_escape == 1 || (c.opt.early_escape == 2 && c.opt.sampling == 0));
}
inline bool early_escape_on(const Ctx &c, int spp, bool batched = false) {
  if (!c.horizon || c.opt.early_escape == 0) return false;
  if (c.opt.early_escape == 1) return true;
  return c.opt.sampling == 0 && spp >= kEarlyEscapeMinSpp &&
         (batched || (long long)c.H * c.W * c.K >= kEarlyEscapeMinItems);
}
cudaError_t launch_horizon(Ctx &c, int spp);  // horizon bounds of the current surface (after the pyramid)
void fill_pyr_obj(const Ctx &c, PyrObj &o);
cudaError_t build_pyramid_batch(cudaStream_t s, const PyrObj *d_objs, int n, int levels, const int *blocks);
cudaError_t launch_horizon_batch(cudaStream_t s, const PyrObj *d_objs, int n, int blocks);
cudaError_t launch_trace(Ctx &c, const int32_t *pixels, int n_pix, int spp, int bounces, uint64_t seed,
                         uint32_t iter, uint32_t stream, float *out, int32_t *rec, bool iter_from_device = false,
                         bool mark_holes = false);
// hole interpolation (holes.cu): pyramid of an H x W image; fill the holes (K x H x W, nonzero = hole)
// of a K x C x H x W device stack in place, scratch v_scr K C py.total and w_scr K py.total floats
FillPyramid fill_pyramid(int H, int W);
// spectral depth solve (spectral.cu): grids up to kSpectralMaxSide on both sides
constexpr int kSpectralMaxSide = 1024;
bool spectral_fits(int H, int W);
cudaError_t spectral_setup(Ctx &c);                                 // matrices and work array
cudaError_t launch_spectral(Ctx &c, const double *b, double *x);   // x = A^+ b, unit weights
// whether a context's unit-weight solves are direct (option precond = 2 on a grid the transform covers)
inline bool direct_solve(const Ctx &c) { return c.opt.precond == 2 && c.sp_t != nullptr; }
// pass descriptors of the direct solve (one 16 x 16 output tile per block)
struct DctFwd {
  int M, N, K, L;
  const double *A;
  int lda;
  const double *B;
  int ldb;
  double *D;
  int ldd, dro, dco;
  const double *mu, *nu;
  int tiles_n, blk_begin;  // tiles along N; first block of the object in a batched launch
};
struct DctInv {
  int M, N, K1, K2, M2, N2, L;
  const double *A1, *A2;
  int lda1, lda2;
  const double *B1, *B2;
  int ldb1, ldb2;
  double *D;
  int ldd;
  int tiles_n, blk_begin;
};
// the direct solves of a batch's objects: six pass tables (four forward, two inverse) in one device block
struct SpectralBatch {
  int n = 0;          // objects with direct solves
  int blocks[6] = {0};
  void *table = nullptr;  // owned
};
cudaError_t spectral_batch_setup(const std::vector<Ctx *> &objs, SpectralBatch &sb);
cudaError_t launch_spectral_batch(cudaStream_t s, const SpectralBatch &sb);
cudaError_t launch_interpolate_holes(cudaStream_t s, float *values, const uint8_t *holes, int K, int C,
                                     const FillPyramid &py, float *v_scr, float *w_scr, int sms, int &launches);
cudaError_t launch_next_iter(Ctx &c);  // iter_dev += 1 (end of a captured iteration)
cudaError_t launch_next_iter(cudaStream_t s, uint32_t *iter_dev);
cudaError_t launch_render(Ctx &c, uint64_t seed, float sigma, const float *lbar, float *out);
// resident blocks of the (batched) trace kernel, per-light or light-shared, 0 if unknown
int trace_grid_limit(int C, int n_obj = 0, bool shared = false);
void fill_obj_trace(const Ctx &c, ObjTrace &o);  // descriptor of a context's object (no sampling fields)
size_t shared_scratch_floats(const Ctx &c, int n_pix, int spp);  // light-shared chunk partials needed
cudaError_t launch_trace_batch(cudaStream_t s, int C, bool shared, const ObjTrace *d_objs, int n_obj,
                               unsigned n_items, unsigned long long *counts, unsigned *next_item,
                               const uint32_t *iter_dev, uint32_t iter, int grid_limit);
// light-shared sampling: sample chunks per pixel (fixed by the sizes), scratch, batched zero / reduce
struct SharedSplit {
  int n_chunks, chunk;  // as in ObjTrace
};
SharedSplit shared_split(int n_pix, int spp);
cudaError_t ensure_shared_scratch(Ctx &c, size_t need, bool &grown);
struct ReduceObj {
  float *part;     // n_chunks x n_pix x kc light partial sums, then n_chunks x n_pix x C environment sums
  float *out;      // kc x n_pix (Lbar)
  int n_chunks, n_pix, kc, C;
  double inv_spp;
  int blk_begin, nblk;
};
cudaError_t launch_parts_batch(cudaStream_t s, bool zero, const ReduceObj *d_objs, int n, int blocks);
cudaError_t launch_probe_dirs(cudaStream_t s, int n, const float *normals, const uint32_t *x0, const uint32_t *x1,
                              float *out);
cudaError_t launch_probe_rays(Ctx &c, int n, const float *rays, float *t_out, int32_t *tri_out, int *overflow);
// ps.cu
// pixels per thread the PS kernel takes: the tuned width when the pixel count is a multiple of it, else 1
inline int ps_vec_for(const Ctx &c) { return (c.H * c.W) % c.ps_vec == 0 ? c.ps_vec : 1; }
cudaError_t launch_ps(Ctx &c, bool zero_indirect);
size_t ps_args_bytes();
void ps_fill_args(const Ctx &c, bool zero_indirect, int blk_begin, void *dst);
cudaError_t launch_ps_batch(cudaStream_t s, int C, int dtype, const void *d_args, int n, int blocks);
// poisson.cu
cudaError_t solve_depth_async(Ctx &c);  // enqueue one depth solve (results accumulate in dstats->cg)
cudaError_t depth_change_async(Ctx &c);  // enqueue D_H of depth against depth_prev into dstats
int solve_depth(Ctx &c);                 // one solve, waited for (IRTPS_OK or an error code, message in c.err)
int cg_grid_limit();  // co-resident blocks available to the cooperative solve
// batched solves: one job per object, teams of blocks in one launch per step
size_t cg_job_bytes();
void cg_fill_job(Ctx &c, int nblk, int blk_begin, DevStats *ds, void *dst);
int cg_batch_grid_limit();
cudaError_t solve_depth_batch_async(cudaStream_t s, const void *d_jobs, int n, int blocks, int irls_iters,
                                    int max_levels, const SpectralBatch &sb);
cudaError_t depth_change_batch_async(cudaStream_t s, const void *d_jobs, int n, int blocks);
cudaError_t zero_depth_batch_async(cudaStream_t s, const void *d_jobs, int n, int blocks);
void mg_layout(int H, int W, int *levels, int *h, int *w, int *off, int *total);
void mg_weights(int levels, const int *h, const int *w, const int *off, float *wh, float *wv);

}  // namespace irtps
