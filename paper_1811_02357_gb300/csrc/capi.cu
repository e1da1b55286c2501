// C ABI of the IRT-PS library: context life cycle, buffers, and the stage
// sequence of one IRT iteration (Sec. IV): pyramid -> trace -> subtract + PS ->
// integration -> D_H.  Declarations and argument contracts: include/irtps.h.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "irtps_internal.h"

using irtps::Ctx;

namespace {

int fail(Ctx &c, int code, const std::string &msg) {
  c.err = msg;
  return code;
}

int cuda_fail(Ctx &c, cudaError_t e, const char *what) {
  c.err = std::string(what) + ": " + cudaGetErrorString(e);
  return IRTPS_ECUDA;
}

#define CK(call, what)                                     \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, what);  \
  } while (0)

template <typename T>
int dalloc(Ctx &c, T **p, size_t n, const char *what) {
  cudaError_t e = cudaMalloc((void **)p, n * sizeof(T) > 0 ? n * sizeof(T) : 16);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(c, e == cudaErrorMemoryAllocation ? IRTPS_ENOMEM : IRTPS_ECUDA,
                std::string("allocation of ") + what + ": " + cudaGetErrorString(e));
  }
  return IRTPS_OK;
}

void release(Ctx &c) {
  void *bufs[] = {c.env, c.d_lights, c.horizon, c.shared_part, c.images, c.lbar, c.depth, c.depth_prev, c.nrm, c.albedo, c.valid, c.pmin, c.pmax,
                  c.cg_x, c.cg_b, c.cg_r, c.cg_z, c.cg_p, c.cg_ap, c.part, c.dstats, c.next_item, c.cg_ctl,
                  c.mg_x0, c.mg_x1, c.mg_b, c.mg_wh, c.mg_wv, c.mg_wh_unit, c.mg_wv_unit, c.iter_dev, c.holes,
                  c.fill_v, c.fill_w, c.sp_ch, c.sp_cw, c.sp_mu, c.sp_nu, c.sp_t, c.ps_pix, c.ps_mask,
                  c.ps_rhs, c.ps_count};
  for (void *b : bufs)
    if (b) cudaFree(b);
  if (c.h_part) cudaFreeHost(c.h_part);
  for (cudaEvent_t ev : c.ev)
    if (ev) cudaEventDestroy(ev);
  for (cudaEvent_t ev : c.tev)
    if (ev) cudaEventDestroy(ev);
  if (c.graph) cudaGraphExecDestroy(c.graph);
  if (c.own_stream && c.stream) cudaStreamDestroy(c.stream);
}

// Copy to or from a caller buffer on the context stream; host copies complete before return.
int copy_out(Ctx &c, void *dst, const void *src, size_t bytes, int on_device) {
  CK(cudaMemcpyAsync(dst, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c.stream),
     "copy out");
  if (!on_device) CK(cudaStreamSynchronize(c.stream), "copy out");
  return IRTPS_OK;
}

int copy_in(Ctx &c, void *dst, const void *src, size_t bytes, int on_device) {
  CK(cudaMemcpyAsync(dst, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c.stream),
     "copy in");
  if (!on_device) CK(cudaStreamSynchronize(c.stream), "copy in");
  return IRTPS_OK;
}

// ---- per-call bookkeeping: device statistics cleared at the start, read once at the end ----
enum Stage { ST_TRACE = 0, ST_PS = 1, ST_DEPTH = 2, ST_FILL = 3 };

int begin_call(Ctx &c) {
  CK(cudaMemsetAsync(c.dstats, 0, sizeof(irtps::DevStats), c.stream), "statistics reset");
  c.stats.trace_ms = c.stats.ps_ms = c.stats.depth_ms = c.stats.fill_ms = 0.0;
  c.stats.node_visits = c.stats.tri_tests = c.stats.draws = 0;
  c.stats.segments = c.stats.walk_overflows = c.stats.primary_segments = 0;
  c.tev_used = 0;
  return IRTPS_OK;
}

// CUDA events around one stage on the context stream (pairs, summed at the end of the call).
int stage_mark(Ctx &c, int stage, bool start) {
  const int need = c.tev_used + 1;
  while ((int)c.tev.size() < 2 * need) {
    cudaEvent_t e;
    CK(cudaEventCreate(&e), "timing events");
    c.tev.push_back(e);
  }
  if (start) {
    c.tev_stage.resize(need);
    c.tev_stage[c.tev_used] = stage;
    CK(cudaEventRecord(c.tev[2 * c.tev_used], c.stream), "timing");
  } else {
    CK(cudaEventRecord(c.tev[2 * c.tev_used + 1], c.stream), "timing");
    ++c.tev_used;
  }
  return IRTPS_OK;
}

#define STAGE(stage, start)                        \
  do {                                             \
    int rc_ = stage_mark(c, stage, start);         \
    if (rc_) return rc_;                           \
  } while (0)

// Wait for the call's work, read the device statistics and turn failures into codes.
int end_call(Ctx &c, bool had_solve) {
  irtps::DevStats h;
  CK(cudaMemcpyAsync(&h, c.dstats, sizeof(h), cudaMemcpyDeviceToHost, c.stream), "statistics");
  CK(cudaStreamSynchronize(c.stream), "call");
  for (int i = 0; i < c.tev_used; ++i) {
    float ms = 0.0f;
    CK(cudaEventElapsedTime(&ms, c.tev[2 * i], c.tev[2 * i + 1]), "timing");
    double *const dst[] = {&c.stats.trace_ms, &c.stats.ps_ms, &c.stats.depth_ms, &c.stats.fill_ms};
    *dst[c.tev_stage[i]] += ms;
  }
  c.stats.segments = h.counts[1];
  c.stats.walk_overflows = h.counts[2];
  c.stats.node_visits = h.counts[3];
  c.stats.tri_tests = h.counts[4];
  c.stats.draws = h.counts[5];
  c.stats.dH_max = h.dh_max;
  c.stats.dH_rms = h.dh_rms;
  if (had_solve) {
    c.stats.cg_iterations = h.cg.last_iters;
    c.stats.cg_rel_residual = h.cg.rel_last;
  }
  if (h.counts[2]) return fail(c, IRTPS_ETIMEOUT, "trace: a heightfield march exhausted its step budget");
  if (h.counts[6]) return fail(c, IRTPS_ETIMEOUT, "ps: a tensor-core product did not complete in time");
  if (had_solve && h.cg.err) return fail(c, IRTPS_ETIMEOUT, "depth solve: a grid barrier timed out");
  if (had_solve && h.cg.bad)
    return fail(c, IRTPS_ENUMERIC, "depth solve: relative residual " + std::to_string(h.cg.rel_last) +
                                       " above cg_tol or not finite (" + std::to_string(h.cg.last_iters) +
                                       " iterations)");
  return IRTPS_OK;
}

// fill: the whole field's trace of the IRT loop with fill_holes on marks the holes
// and replaces Lbar there by the interpolation of the known pixels.
int trace_into(Ctx &c, const int32_t *pixels, int n_pix, int spp, int bounces, uint64_t seed, uint32_t iter,
               uint32_t stream_tag, float *out, int32_t *rec, bool iter_from_device = false, bool fill = false) {
  fill = fill && c.opt.fill_holes && !pixels && out == c.lbar;
  CK(irtps::build_pyramid(c), "pyramid build");
  if (!iter_from_device) STAGE(ST_TRACE, true);
  CK(irtps::launch_horizon(c, spp), "horizon bounds");
  CK(irtps::launch_trace(c, pixels, n_pix, spp, bounces, seed, iter, stream_tag, out, rec, iter_from_device, fill),
     "trace launch");
  if (!iter_from_device) STAGE(ST_TRACE, false);
  if (fill) {
    int launches = 0;
    if (!iter_from_device) STAGE(ST_FILL, true);
    CK(irtps::launch_interpolate_holes(c.stream, c.lbar, c.holes, c.K, c.C, c.fill_py, c.fill_v, c.fill_w, c.sms,
                                       launches),
       "hole interpolation");
    if (!iter_from_device) STAGE(ST_FILL, false);
    c.stats.launches += launches;
  }
  c.stats.primary_segments += (unsigned long long)n_pix * (c.opt.sampling == 1 ? 1 : c.K) * spp;
  return IRTPS_OK;
}

bool trace_args_ok(Ctx &c, int spp, int bounces) {
  if (spp < 1 || bounces < 1 || bounces > 3) {
    c.err = "spp must be >= 1 and bounces in 1..3";
    return false;
  }
  return true;
}

// Light-shared traces keep per-chunk partial sums; size them before any capture.
int prepare_trace(Ctx &c, int n_pix, int spp) {
  if (c.opt.sampling != 1) return IRTPS_OK;
  bool grown = false;
  const cudaError_t e = irtps::ensure_shared_scratch(c, irtps::shared_scratch_floats(c, n_pix, spp), grown);
  if (e != cudaSuccess)
    return fail(c, e == cudaErrorMemoryAllocation ? IRTPS_ENOMEM : IRTPS_ECUDA,
                std::string("light-shared partial sums: ") + cudaGetErrorString(e));
  return IRTPS_OK;
}

int run_ps(Ctx &c, bool zero_indirect) {
  STAGE(ST_PS, true);
  CK(irtps::launch_ps(c, zero_indirect), "ps launch");
  STAGE(ST_PS, false);
  return IRTPS_OK;
}

int run_depth(Ctx &c) {
  STAGE(ST_DEPTH, true);
  CK(irtps::solve_depth_async(c), "depth solve launch");
  STAGE(ST_DEPTH, false);
  return IRTPS_OK;
}

int iteration_zero(Ctx &c) {
  int rc = run_ps(c, true);
  if (rc) return rc;
  CK(cudaMemsetAsync(c.depth, 0, sizeof(float) * c.H * c.W, c.stream), "depth reset");
  return run_depth(c);
}

// One IRT iteration enqueued on the context stream.  With `captured`, the trace
// reads the iteration index from iter_dev and the iteration ends by advancing it,
// so that a captured copy can be replayed for every iteration; stage timing events
// are then left out.
int enqueue_iteration(Ctx &c, int spp, int bounces, uint64_t seed, bool captured) {
  int rc;
  CK(cudaMemcpyAsync(c.depth_prev, c.depth, sizeof(float) * c.H * c.W, cudaMemcpyDeviceToDevice, c.stream),
     "iterate");
  if ((rc = trace_into(c, nullptr, c.H * c.W, spp, bounces, seed, c.t, 0u, c.lbar, nullptr, captured, true)))
    return rc;
  if (captured) {
    CK(irtps::launch_ps(c, false), "ps launch");
    CK(irtps::solve_depth_async(c), "depth solve launch");
  } else {
    if ((rc = run_ps(c, false))) return rc;
    if ((rc = run_depth(c))) return rc;
  }
  CK(irtps::depth_change_async(c), "depth change");
  if (captured) CK(irtps::launch_next_iter(c), "iteration counter");
  return IRTPS_OK;
}

// Capture one iteration as a CUDA graph (again when spp, bounces or seed change).
int capture_iteration(Ctx &c, int spp, int bounces, uint64_t seed) {
  if (c.graph && c.graph_spp == spp && c.graph_bounces == bounces && c.graph_seed == seed) return IRTPS_OK;
  if (c.graph) {
    cudaGraphExecDestroy(c.graph);
    c.graph = nullptr;
  }
  CK(cudaStreamBeginCapture(c.stream, cudaStreamCaptureModeThreadLocal), "graph capture");
  const unsigned long long launches = c.stats.launches;
  int rc = enqueue_iteration(c, spp, bounces, seed, true);
  c.stats.launches = launches;
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(c.stream, &g);
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "graph capture");
  const cudaError_t e2 = cudaGraphInstantiate(&c.graph, g, 0);
  cudaGraphDestroy(g);
  if (e2 != cudaSuccess) {
    c.graph = nullptr;
    return cuda_fail(c, e2, "graph instantiate");
  }
  c.graph_spp = spp;
  c.graph_bounces = bounces;
  c.graph_seed = seed;
  return IRTPS_OK;
}

}  // namespace

extern "C" {

void irtps_default_options(irtps_options *opt) {
  if (!opt) return;
  opt->shadow_rays = 1;
  opt->tau_lo = 0.02f;
  opt->tau_hi = 0.98f;
  opt->cond_max = 1e8;
  opt->nz_min = 0.05f;
  opt->cg_tol = 1e-9;
  opt->cg_max_iter = 50000;
  opt->cg_check_every = 10;
  opt->stop_tol = 0.0;
  opt->precond = 2;
  opt->use_graph = 0;
  opt->sampling = 0;
  opt->irls_iters = 0;
  opt->irls_delta = 0.05f;
  opt->early_escape = 2;
  opt->fill_holes = 0;
  opt->ps_tensor = 0;
}

int irtps_create(irtps_ctx **out, int H, int W, int K, int C, const float *lights, const float *env, int EH,
                 int EW, const irtps_options *opt) {
  if (!out) return IRTPS_EINVAL;
  *out = nullptr;
  irtps_ctx *x = new (std::nothrow) irtps_ctx;
  if (!x) return IRTPS_ENOMEM;
  Ctx &c = x->c;
  auto bail = [&](int rc) {
    // keep the context so that the caller can read the message; it is still destroyable
    *out = x;
    return rc;
  };
  if (H < 2 || W < 2 || K < 3 || K > irtps::kMaxLights || (C != 1 && C != 3) || EH < 1 || EW < 1 || !lights ||
      !env)
    return bail(fail(c, IRTPS_EINVAL, "create: need H, W >= 2, 3 <= K <= 64, C in {1,3}, EH, EW >= 1, lights, env"));
  if ((long long)H * W * K >= (1LL << 31) || (long long)(W - 1) * (H - 1) * 2 >= (1LL << 31))
    return bail(fail(c, IRTPS_EINVAL, "create: H*W*K must stay below 2^31"));
  c.H = H;
  c.W = W;
  c.K = K;
  c.C = C;
  c.EH = EH;
  c.EW = EW;
  if (opt)
    c.opt = *opt;
  else
    irtps_default_options(&c.opt);
  if (c.opt.precond < 0 || c.opt.precond > 2)
    return bail(fail(c, IRTPS_EINVAL, "create: precond must be 0 (Jacobi), 1 (multigrid) or 2 (spectral)"));
  if (c.opt.sampling != 0 && c.opt.sampling != 1)
    return bail(fail(c, IRTPS_EINVAL, "create: sampling must be 0 (per light) or 1 (light-shared)"));
  if (c.opt.irls_iters < 0 || c.opt.irls_iters > 100 || !(c.opt.irls_delta > 0.0f))
    return bail(fail(c, IRTPS_EINVAL, "create: irls_iters in 0..100 and irls_delta > 0"));
  if (c.opt.early_escape < 0 || c.opt.early_escape > 2)
    return bail(fail(c, IRTPS_EINVAL, "create: early_escape must be 0, 1 or 2"));
  if (c.opt.fill_holes != 0 && c.opt.fill_holes != 1)
    return bail(fail(c, IRTPS_EINVAL, "create: fill_holes must be 0 or 1"));
  if (c.opt.fill_holes && c.opt.sampling != 0)
    return bail(fail(c, IRTPS_EINVAL, "create: fill_holes needs per-light sampling (sampling = 0)"));
  if (c.opt.ps_tensor != 0 && c.opt.ps_tensor != 1)
    return bail(fail(c, IRTPS_EINVAL, "create: ps_tensor must be 0 or 1"));
  c.eps = (float)1e-3 / (float)W;  // same expression as the oracle's lift
  // lights and pinv(L) = (L^T L)^-1 L^T in FP64 (Eq. 4)
  c.h_lights.assign(lights, lights + 3 * K);
  double M[3][3] = {{0}};
  for (int k = 0; k < K; ++k) {
    const double l[3] = {lights[3 * k], lights[3 * k + 1], lights[3 * k + 2]};
    if (!std::isfinite(l[0]) || !std::isfinite(l[1]) || !std::isfinite(l[2]))
      return bail(fail(c, IRTPS_EINVAL, "create: non-finite light direction"));
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) M[a][b] += l[a] * l[b];
  }
  const double A[3][3] = {{M[1][1] * M[2][2] - M[1][2] * M[2][1], M[0][2] * M[2][1] - M[0][1] * M[2][2],
                           M[0][1] * M[1][2] - M[0][2] * M[1][1]},
                          {M[1][2] * M[2][0] - M[1][0] * M[2][2], M[0][0] * M[2][2] - M[0][2] * M[2][0],
                           M[0][2] * M[1][0] - M[0][0] * M[1][2]},
                          {M[1][0] * M[2][1] - M[1][1] * M[2][0], M[0][1] * M[2][0] - M[0][0] * M[2][1],
                           M[0][0] * M[1][1] - M[0][1] * M[1][0]}};
  const double det = M[0][0] * A[0][0] + M[0][1] * A[1][0] + M[0][2] * A[2][0];
  double trace = M[0][0] + M[1][1] + M[2][2];
  if (!(std::fabs(det) > 1e-12 * trace * trace * trace))
    return bail(fail(c, IRTPS_EINVAL, "create: the lights are coplanar (L^T L is singular)"));
  c.h_pinv.resize(3 * K);
  for (int a = 0; a < 3; ++a)
    for (int k = 0; k < K; ++k) {
      double v = 0.0;
      for (int b = 0; b < 3; ++b) v += A[a][b] / det * lights[3 * k + b];
      c.h_pinv[a * K + k] = (float)v;
    }
  {  // (L^T L)^-1 and its 1-norm condition number: a well-conditioned system lets PS sum
     // R = L^T I alone and apply the inverse once per pixel (pinv(L) I = (L^T L)^-1 L^T I)
    double nm = 0.0, ni = 0.0;
    for (int a = 0; a < 3; ++a) {
      double rm = 0.0, ri = 0.0;
      for (int b = 0; b < 3; ++b) {
        rm += std::fabs(M[a][b]);
        ri += std::fabs(A[a][b] / det);
      }
      nm = std::max(nm, rm);
      ni = std::max(ni, ri);
    }
    const int idx[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
    for (int i = 0; i < 6; ++i) c.h_minv[i] = (float)(A[idx[i][0]][idx[i][1]] / det);
    c.normal_eq = nm * ni <= 16.0 ? 1 : 0;
  }
  // pyramid geometry
  int w = W - 1, h = H - 1, total = 0, l = 0;
  while (true) {
    if (l >= irtps::kMaxLevels) return bail(fail(c, IRTPS_EINVAL, "create: grid too large for the pyramid"));
    c.off[l] = total;
    c.lw[l] = w;
    c.lh[l] = h;
    total += w * h;
    ++l;
    if (w == 1 && h == 1) break;
    w = (w + 1) / 2;
    h = (h + 1) / 2;
  }
  c.levels = l;
  // buffers
  const size_t P = (size_t)H * W;
  int rc;
  cudaError_t e = cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) return bail(cuda_fail(c, e, "create: stream"));
  c.own_stream = true;
  for (int i = 0; i < 2; ++i) {
    e = cudaEventCreate(&c.ev[i]);
    if (e != cudaSuccess) return bail(cuda_fail(c, e, "create: events"));
  }
  c.cg_blocks = (int)std::min<size_t>((P + 255) / 256, (size_t)irtps::cg_grid_limit());
  c.trace_blocks = irtps::trace_grid_limit(C, 0, c.opt.sampling == 1);
  {
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&c.sms, cudaDevAttrMultiProcessorCount, dev);
    c.trace_per_sm_max = c.sms > 0 ? c.trace_blocks / c.sms : 0;
  }
  c.part_stride = c.cg_blocks;
  if ((rc = dalloc(c, &c.env, (size_t)C * EH * EW, "environment")) ||
      (rc = dalloc(c, &c.d_lights, (size_t)K * 3, "lights")) ||
      (c.opt.early_escape && H <= 16384 && W <= 16384 &&
       (rc = dalloc(c, &c.horizon, (size_t)8 * P, "horizon bounds"))) ||
      (rc = dalloc(c, (float **)&c.images, (size_t)K * C * P, "images")) ||
      (rc = dalloc(c, &c.lbar, (size_t)K * C * P, "indirect")) || (rc = dalloc(c, &c.depth, P, "depth")) ||
      (rc = dalloc(c, &c.depth_prev, P, "depth")) || (rc = dalloc(c, &c.nrm, P, "normals")) ||
      (rc = dalloc(c, &c.albedo, (size_t)C * P, "albedo")) || (rc = dalloc(c, &c.valid, P, "valid")) ||
      (rc = dalloc(c, &c.ps_pix, P, "masked-pixel list")) || (rc = dalloc(c, &c.ps_mask, P, "masked-pixel list")) ||
      (rc = dalloc(c, &c.ps_rhs, (size_t)9 * P, "masked-pixel list")) ||
      (rc = dalloc(c, &c.ps_count, 1, "masked-pixel list")) ||
      (rc = dalloc(c, &c.pmin, (size_t)total, "pyramid")) || (rc = dalloc(c, &c.pmax, (size_t)total, "pyramid")) ||
      (rc = dalloc(c, &c.cg_x, P, "cg")) || (rc = dalloc(c, &c.cg_b, P, "cg")) ||
      (rc = dalloc(c, &c.cg_r, P, "cg")) || (rc = dalloc(c, &c.cg_z, P, "cg")) ||
      (rc = dalloc(c, &c.cg_p, 2 * P, "cg")) || (rc = dalloc(c, &c.cg_ap, 2 * P, "cg")) ||
      (rc = dalloc(c, &c.part, (size_t)irtps::kPartSlots * c.part_stride, "partials")) ||
      (rc = dalloc(c, &c.dstats, 1, "statistics")) || (rc = dalloc(c, &c.next_item, 1, "work counter")) ||
      (rc = dalloc(c, &c.iter_dev, 1, "iteration counter")) ||
      (rc = dalloc(c, (irtps::CGCtl **)&c.cg_ctl, 1, "solver control")))
    return bail(rc);
  if (c.opt.precond == 2 && irtps::spectral_fits(H, W)) {
    e = irtps::spectral_setup(c);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return bail(fail(c, e == cudaErrorMemoryAllocation ? IRTPS_ENOMEM : IRTPS_ECUDA,
                       std::string("create: spectral solve: ") + cudaGetErrorString(e)));
    }
  }
  if (c.opt.fill_holes) {  // hole mask and the interpolation pyramid above level 0
    c.fill_py = irtps::fill_pyramid(H, W);
    if ((rc = dalloc(c, &c.holes, (size_t)K * P, "hole mask")) ||
        (rc = dalloc(c, &c.fill_v, (size_t)K * C * c.fill_py.total, "hole interpolation")) ||
        (rc = dalloc(c, &c.fill_w, (size_t)K * c.fill_py.total, "hole interpolation")))
      return bail(rc);
  }
  {  // multigrid hierarchy: layout and Galerkin weights built on the host once
    int total = 0;
    irtps::mg_layout(H, W, &c.mg_levels, c.mg_h, c.mg_w, c.mg_off, &total);
    std::vector<float> wh((size_t)total), wv((size_t)total);
    irtps::mg_weights(c.mg_levels, c.mg_h, c.mg_w, c.mg_off, wh.data(), wv.data());
    c.mg_total = total;
    if ((rc = dalloc(c, &c.mg_x0, (size_t)total, "multigrid")) || (rc = dalloc(c, &c.mg_x1, (size_t)total, "multigrid")) ||
        (rc = dalloc(c, &c.mg_b, (size_t)total, "multigrid")) || (rc = dalloc(c, &c.mg_wh, (size_t)total, "multigrid")) ||
        (rc = dalloc(c, &c.mg_wv, (size_t)total, "multigrid")))
      return bail(rc);
    e = cudaMemcpy(c.mg_wh, wh.data(), sizeof(float) * total, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c.mg_wv, wv.data(), sizeof(float) * total, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && c.opt.irls_iters > 0) {  // a pristine copy to restore after the weighted solves
      if ((rc = dalloc(c, &c.mg_wh_unit, (size_t)total, "multigrid")) ||
          (rc = dalloc(c, &c.mg_wv_unit, (size_t)total, "multigrid")))
        return bail(rc);
      e = cudaMemcpy(c.mg_wh_unit, wh.data(), sizeof(float) * total, cudaMemcpyHostToDevice);
      if (e == cudaSuccess) e = cudaMemcpy(c.mg_wv_unit, wv.data(), sizeof(float) * total, cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) return bail(cuda_fail(c, e, "create: multigrid weights"));
  }
  e = cudaMallocHost((void **)&c.h_part, sizeof(double) * c.part_stride);
  if (e != cudaSuccess) return bail(cuda_fail(c, e, "create: pinned partials"));
  e = cudaMemcpyAsync(c.env, env, sizeof(float) * C * EH * EW, cudaMemcpyHostToDevice, c.stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c.d_lights, c.h_lights.data(), sizeof(float) * K * 3, cudaMemcpyHostToDevice, c.stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c.lbar, 0, sizeof(float) * K * C * P, c.stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c.depth, 0, sizeof(float) * P, c.stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c.albedo, 0, sizeof(float) * C * P, c.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
  if (e != cudaSuccess) return bail(cuda_fail(c, e, "create: upload"));
  *out = x;
  return IRTPS_OK;
}

int irtps_set_stream(irtps_ctx *ctx, void *stream) {
  if (!ctx) return IRTPS_EINVAL;
  Ctx &c = ctx->c;
  if (c.own_stream && c.stream) {
    CK(cudaStreamSynchronize(c.stream), "set stream");
    CK(cudaStreamDestroy(c.stream), "set stream");
    c.own_stream = false;
  }
  if (stream) {
    c.stream = (cudaStream_t)stream;
  } else {
    CK(cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking), "set stream");
    c.own_stream = true;
  }
  return IRTPS_OK;
}

int irtps_set_images(irtps_ctx *ctx, const void *images, int dtype, int on_device) {
  if (!ctx) return IRTPS_EINVAL;
  Ctx &c = ctx->c;
  if (!images || (dtype != IRTPS_F32 && dtype != IRTPS_F16))
    return fail(c, IRTPS_EINVAL, "set_images: need images and dtype IRTPS_F32 or IRTPS_F16");
  const size_t n = (size_t)c.K * c.C * c.H * c.W;
  c.images_dtype = dtype;
  int rc = copy_in(c, c.images, images, n * (dtype == IRTPS_F16 ? 2 : 4), on_device);
  if (rc) return rc;
  c.have_images = true;
  c.t = 0;
  if ((rc = begin_call(c)) || (rc = iteration_zero(c))) return rc;
  return end_call(c, true);
}

int irtps_iterate(irtps_ctx *ctx, int n_iter, int spp, int bounces, uint64_t seed, double *out_dH) {
  if (!ctx) return IRTPS_EINVAL;
  Ctx &c = ctx->c;
  if (!c.have_images) return fail(c, IRTPS_ENOTREADY, "iterate: call irtps_set_images first");
  if (n_iter < 0 || !trace_args_ok(c, spp, bounces)) return fail(c, IRTPS_EINVAL, c.err.empty() ? "iterate" : c.err);
  c.stats.iterations_done = 0;
  int rc = prepare_trace(c, c.H * c.W, spp);
  if (rc || (rc = begin_call(c))) return rc;
  if (c.opt.use_graph && n_iter > 0) {
    if ((rc = capture_iteration(c, spp, bounces, seed))) return rc;
    CK(cudaMemcpyAsync(c.iter_dev, &c.t, sizeof(uint32_t), cudaMemcpyHostToDevice, c.stream), "iteration counter");
  }
  // One iteration is enqueued without host round trips; the host waits once at
  // the end (and after each iteration only when early stopping is requested).
  for (int it = 0; it < n_iter; ++it) {
    if (c.opt.use_graph) {
      CK(cudaGraphLaunch(c.graph, c.stream), "graph launch");
      c.stats.primary_segments += (unsigned long long)c.H * c.W * (c.opt.sampling == 1 ? 1 : c.K) * spp;
    } else if ((rc = enqueue_iteration(c, spp, bounces, seed, false))) {
      return rc;
    }
    ++c.t;
    c.stats.iterations_done = it + 1;
    if (c.opt.stop_tol > 0.0) {
      double dh = 0.0;
      CK(cudaMemcpyAsync(&dh, &c.dstats->dh_max, sizeof(double), cudaMemcpyDeviceToHost, c.stream), "D_H");
      CK(cudaStreamSynchronize(c.stream), "D_H");
      if (dh < c.opt.stop_tol) break;
    }
  }
  rc = end_call(c, c.stats.iterations_done > 0);
  if (out_dH) *out_dH = c.stats.dH_max;
  return rc;
}

int irtps_trace(irtps_ctx *ctx, int spp, int bounces, uint64_t seed, uint32_t iteration, uint32_t stream_tag) {
  if (!ctx) return IRTPS_EINVAL;
  Ctx &c = ctx->c;
  if (!trace_args_ok(c, spp, bounces) || stream_tag > 15) return fail(c, IRTPS_EINVAL, "trace: bad arguments");
  int rc = prepare_trace(c, c.H * c.W, spp);
  if (rc) return rc;
  rc = begin_call(c);
  if (rc || (rc = trace_into(c, nullptr, c.H * c.W, spp, bounces, seed, iteration, stream_tag, c.lbar, nullptr,
                             false, true)))
    return rc;
  return end_call(c, false);
}

int irtps_solve_normals(irtps_ctx *ctx) {
  if (!ctx) return IRTPS_EINVAL;
  Ctx &c = ctx->c;
  if (!c.have_images) return fail(c, IRTPS_ENOTREADY, "solve_normals: call irtps_set_images first");
  int rc = begin_call(c);
  if (rc || (rc = run_ps(c, false))) return rc;
  return end_call(c, false);
}

int irtps_integrate(irtps_ctx *ctx) {
  if (!ctx) return IRTPS_EINVAL;
  Ctx &c = ctx->c;
  int rc = begin_call(c);
  if (rc || (rc = run_depth(c))) return rc;
  return end_call(c, true);
}

int irtps_trace_pixels(irtps_ctx *ctx, const int32_t *pixels, int n_pix, int spp, int bounces, uint64_t seed,
                       uint32_t iteration, uint32_t stream_tag, float *out_lbar, int32_t *out_rec) {
  if (!ctx) return IRTPS_EINVAL;
  Ctx &c = ctx->c;
  if (!pixels || n_pix < 1 || !out_lbar || !trace_args_ok(c, spp, bounces) || stream_tag > 15)
    return fail(c, IRTPS_EINVAL, "trace_pixels: bad arguments");
  const int P = c.H * c.W;
  for (int i = 0; i < n_pix; ++i)
    if (pixels[i] < 0 || pixels[i] >= P) return fail(c, IRTPS_EINVAL, "trace_pixels: pixel index out of range");
  const size_t nrec = !out_rec ? 0
                     : (c.opt.sampling == 1 ? (size_t)n_pix * spp * bounces * (1 + c.K)
                                            : (size_t)n_pix * c.K * spp * bounces * 2);
  int32_t *d_pix = nullptr, *d_rec = nullptr;
  float *d_out = nullptr;
  int rc = prepare_trace(c, n_pix, spp);
  if (rc) return rc;
  if ((rc = dalloc(c, &d_pix, n_pix, "pixel list")) || (rc = dalloc(c, &d_out, (size_t)c.K * c.C * n_pix, "out")) ||
      (out_rec && (rc = dalloc(c, &d_rec, nrec, "records")))) {
    cudaFree(d_pix);
    cudaFree(d_out);
    return rc;
  }
  cudaError_t e = cudaMemcpyAsync(d_pix, pixels, sizeof(int32_t) * n_pix, cudaMemcpyHostToDevice, c.stream);
  if (e == cudaSuccess) {
    rc = begin_call(c);
    if (rc == IRTPS_OK) rc = trace_into(c, d_pix, n_pix, spp, bounces, seed, iteration, stream_tag, d_out, d_rec);
    if (rc == IRTPS_OK) rc = end_call(c, false);
    if (rc == IRTPS_OK) {
      e = cudaMemcpyAsync(out_lbar, d_out, sizeof(float) * c.K * c.C * n_pix, cudaMemcpyDeviceToHost, c.stream);
      if (e == cudaSuccess && out_rec)
        e = cudaMemcpyAsync(out_rec, d_rec, sizeof(int32_t) * nrec, cudaMemcpyDeviceToHost, c.stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
    }
  }
  cudaFree(d_pix);
  cudaFree(d_out);
  if (d_rec) cudaFree(d_rec);
  if (e != cudaSuccess) return cuda_fail(c, e, "trace_pixels");
  return rc;
}

int irtps_set_state(irtps_ctx *ctx, const float *depth, const float *normals, const float *albedo) {
  if (!ctx) return IRTPS_EINVAL;
  Ctx &c = ctx->c;
  const size_t P = (size_t)c.H * c.W;
  if (depth) {
    int rc = copy_in(c, c.depth, depth, sizeof(float) * P, 0);
    if (rc) return rc;
  }
  if (albedo) {
    int rc = copy_in(c, c.albedo, albedo, sizeof(float) * c.C * P, 0);
    if (rc) return rc;
  }
  if (normals || albedo) {
    // pack (n, mean albedo) on the host from the given or current arrays
    std::vector<float> n4(4 * P), rho((size_t)c.C * P), cur(4 * P);
    if (!normals) CK(cudaMemcpy(cur.data(), c.nrm, sizeof(float) * 4 * P, cudaMemcpyDeviceToHost), "set_state");
    if (albedo)
      std::memcpy(rho.data(), albedo, sizeof(float) * c.C * P);
    else
      CK(cudaMemcpy(rho.data(), c.albedo, sizeof(float) * c.C * P, cudaMemcpyDeviceToHost), "set_state");
    for (size_t p = 0; p < P; ++p) {
      for (int a = 0; a < 3; ++a) n4[4 * p + a] = normals ? normals[3 * p + a] : cur[4 * p + a];
      float s = 0.0f;
      for (int ch = 0; ch < c.C; ++ch) s += rho[ch * P + p];
      n4[4 * p + 3] = s / (float)c.C;
    }
    int rc = copy_in(c, c.nrm, n4.data(), sizeof(float) * 4 * P, 0);
    if (rc) return rc;
    CK(cudaMemsetAsync(c.valid, 1, P, c.stream), "set_state");
  }
  return IRTPS_OK;
}

int irtps_set_indirect(irtps_ctx *ctx, const float *indirect) {
  if (!ctx) return IRTPS_EINVAL;
  Ctx &c = ctx->c;
  if (!indirect) return fail(c, IRTPS_EINVAL, "set_indirect: NULL");
  return copy_in(c, c.lbar, indirect, sizeof(float) * c.K * c.C * c.H * c.W, 0);
}

int irtps_render(irtps_ctx *ctx, int spp, int bounces, uint64_t seed, float sigma, float *out, int on_device) {
  if (!ctx) return IRTPS_EINVAL;
  Ctx &c = ctx->c;
  if (!out || !trace_args_ok(c, spp, bounces) || !(sigma >= 0.0f)) return fail(c, IRTPS_EINVAL, "render: bad arguments");
  // the synthetic images take the per-light trace whatever the context's sampling
  const int sampling = c.opt.sampling;
  c.opt.sampling = 0;
  int rc = begin_call(c);
  if (rc == IRTPS_OK) rc = trace_into(c, nullptr, c.H * c.W, spp, bounces, seed, 0xFFFFFFFFu, 1u, c.lbar, nullptr);
  if (rc == IRTPS_OK) rc = end_call(c, false);
  c.opt.sampling = sampling;
  if (rc) return rc;
  const size_t n = (size_t)c.K * c.C * c.H * c.W;
  float *dst = out;
  float *tmp = nullptr;
  if (!on_device) {
    if ((rc = dalloc(c, &tmp, n, "render output"))) return rc;
    dst = tmp;
  }
  cudaError_t e = irtps::launch_render(c, seed, sigma, c.lbar, dst);
  if (e == cudaSuccess && !on_device) {
    e = cudaMemcpyAsync(out, tmp, sizeof(float) * n, cudaMemcpyDeviceToHost, c.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
  }
  if (tmp) cudaFree(tmp);
  if (e != cudaSuccess) return cuda_fail(c, e, "render");
  return IRTPS_OK;
}

int irtps_get_normals(irtps_ctx *ctx, float *out, int on_device) {
  if (!ctx || !out) return IRTPS_EINVAL;
  Ctx &c = ctx->c;
  return copy_out(c, out, c.nrm, sizeof(float) * 4 * c.H * c.W, on_device);
}
int irtps_get_albedo(irtps_ctx *ctx, float *out, int on_device) {
  if (!ctx || !out) return IRTPS_EINVAL;
  Ctx &c = ctx->c;
  return copy_out(c, out, c.albedo, sizeof(float) * c.C * c.H * c.W, on_device);
}
int irtps_get_depth(irtps_ctx *ctx, float *out, int on_device) {
  if (!ctx || !out) return IRTPS_EINVAL;
  Ctx &c = ctx->c;
  return copy_out(c, out, c.depth, sizeof(float) * c.H * c.W, on_device);
}
int irtps_get_indirect(irtps_ctx *ctx, float *out, int on_device) {
  if (!ctx || !out) return IRTPS_EINVAL;
  Ctx &c = ctx->c;
  return copy_out(c, out, c.lbar, sizeof(float) * c.K * c.C * c.H * c.W, on_device);
}
int irtps_get_valid(irtps_ctx *ctx, uint8_t *out, int on_device) {
  if (!ctx || !out) return IRTPS_EINVAL;
  Ctx &c = ctx->c;
  return copy_out(c, out, c.valid, (size_t)c.H * c.W, on_device);
}
int irtps_get_holes(irtps_ctx *ctx, uint8_t *out, int on_device) {
  if (!ctx || !out) return IRTPS_EINVAL;
  Ctx &c = ctx->c;
  if (!c.holes) return fail(c, IRTPS_EINVAL, "get_holes: the context was created without fill_holes");
  return copy_out(c, out, c.holes, (size_t)c.K * c.H * c.W, on_device);
}

int irtps_interpolate_holes(float *values, const uint8_t *holes, int K, int C, int H, int W) {
  if (!values || !holes || K < 1 || (C != 1 && C != 3) || H < 1 || W < 1) return IRTPS_EINVAL;
  if ((long long)K * C * H * W >= (1LL << 31)) return IRTPS_EINVAL;
  const irtps::FillPyramid py = irtps::fill_pyramid(H, W);
  const size_t P = (size_t)H * W;
  int sms = 0, dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  float *dv = nullptr, *sv = nullptr, *sw = nullptr;
  uint8_t *dh = nullptr;
  cudaError_t e = cudaMalloc(&dv, sizeof(float) * K * C * P);
  if (e == cudaSuccess) e = cudaMalloc(&dh, (size_t)K * P);
  if (e == cudaSuccess) e = cudaMalloc(&sv, sizeof(float) * (K * C * py.total + 1));
  if (e == cudaSuccess) e = cudaMalloc(&sw, sizeof(float) * (K * py.total + 1));
  if (e == cudaSuccess) e = cudaMemcpy(dv, values, sizeof(float) * K * C * P, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dh, holes, (size_t)K * P, cudaMemcpyHostToDevice);
  int launches = 0;
  if (e == cudaSuccess) e = irtps::launch_interpolate_holes(nullptr, dv, dh, K, C, py, sv, sw, sms, launches);
  if (e == cudaSuccess) e = cudaMemcpy(values, dv, sizeof(float) * K * C * P, cudaMemcpyDeviceToHost);
  const bool oom = e == cudaErrorMemoryAllocation;
  if (e != cudaSuccess) cudaGetLastError();
  cudaFree(dv);
  cudaFree(dh);
  cudaFree(sv);
  cudaFree(sw);
  return e == cudaSuccess ? IRTPS_OK : (oom ? IRTPS_ENOMEM : IRTPS_ECUDA);
}

int irtps_get_stats(irtps_ctx *ctx, irtps_stats *out) {
  if (!ctx || !out) return IRTPS_EINVAL;
  *out = ctx->c.stats;
  return IRTPS_OK;
}

int irtps_probe_dirs(int n, const float *normals, const uint32_t *x0, const uint32_t *x1, float *out) {
  if (n < 1 || !normals || !x0 || !x1 || !out) return IRTPS_EINVAL;
  float *dn = nullptr, *dout = nullptr;
  uint32_t *d0 = nullptr, *d1 = nullptr;
  cudaError_t e = cudaMalloc(&dn, sizeof(float) * 3 * n);
  if (e == cudaSuccess) e = cudaMalloc(&dout, sizeof(float) * 3 * n);
  if (e == cudaSuccess) e = cudaMalloc(&d0, sizeof(uint32_t) * n);
  if (e == cudaSuccess) e = cudaMalloc(&d1, sizeof(uint32_t) * n);
  if (e == cudaSuccess) e = cudaMemcpy(dn, normals, sizeof(float) * 3 * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d0, x0, sizeof(uint32_t) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d1, x1, sizeof(uint32_t) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = irtps::launch_probe_dirs(nullptr, n, dn, d0, d1, dout);
  if (e == cudaSuccess) e = cudaMemcpy(out, dout, sizeof(float) * 3 * n, cudaMemcpyDeviceToHost);
  cudaFree(dn);
  cudaFree(dout);
  cudaFree(d0);
  cudaFree(d1);
  return e == cudaSuccess ? IRTPS_OK : IRTPS_ECUDA;
}

int irtps_probe_rays(irtps_ctx *ctx, int n, const float *rays, float *out_t, int32_t *out_tri) {
  if (!ctx) return IRTPS_EINVAL;
  Ctx &c = ctx->c;
  if (n < 1 || !rays || !out_t || !out_tri) return fail(c, IRTPS_EINVAL, "probe_rays: bad arguments");
  CK(irtps::build_pyramid(c), "pyramid build");
  float *dr = nullptr, *dt = nullptr;
  int32_t *dtri = nullptr;
  int *dov = nullptr;
  int rc;
  if ((rc = dalloc(c, &dr, (size_t)6 * n, "rays")) || (rc = dalloc(c, &dt, (size_t)n, "t")) ||
      (rc = dalloc(c, &dtri, (size_t)n, "tri")) || (rc = dalloc(c, &dov, 1, "flag"))) {
    cudaFree(dr);
    cudaFree(dt);
    cudaFree(dtri);
    return rc;
  }
  int ov = 0;
  cudaError_t e = cudaMemcpyAsync(dr, rays, sizeof(float) * 6 * n, cudaMemcpyHostToDevice, c.stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(dov, 0, sizeof(int), c.stream);
  if (e == cudaSuccess) e = irtps::launch_probe_rays(c, n, dr, dt, dtri, dov);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out_t, dt, sizeof(float) * n, cudaMemcpyDeviceToHost, c.stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out_tri, dtri, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, c.stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&ov, dov, sizeof(int), cudaMemcpyDeviceToHost, c.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
  cudaFree(dr);
  cudaFree(dt);
  cudaFree(dtri);
  cudaFree(dov);
  if (e != cudaSuccess) return cuda_fail(c, e, "probe_rays");
  if (ov) return fail(c, IRTPS_ETIMEOUT, "probe_rays: a march exhausted its step budget");
  return IRTPS_OK;
}

int irtps_set_object(irtps_ctx *ctx, uint32_t object) {
  if (!ctx) return IRTPS_EINVAL;
  if (ctx->c.graph) {  // a captured iteration holds the old key
    cudaGraphExecDestroy(ctx->c.graph);
    ctx->c.graph = nullptr;
  }
  ctx->c.obj = object;
  return IRTPS_OK;
}

int irtps_set_tuning(irtps_ctx *ctx, int blocks_per_sm, int mip_cut) {
  if (!ctx) return IRTPS_EINVAL;
  Ctx &c = ctx->c;
  if (blocks_per_sm < 0 || blocks_per_sm > c.trace_per_sm_max || mip_cut < 0 || mip_cut >= irtps::kMaxLevels)
    return fail(c, IRTPS_EINVAL, "tuning: blocks_per_sm in 0.." + std::to_string(c.trace_per_sm_max) +
                                     ", mip_cut in 0..15");
  c.trace_blocks = (blocks_per_sm == 0 ? c.trace_per_sm_max : blocks_per_sm) * c.sms;
  c.mip_cut = mip_cut;
  if (c.graph) {
    cudaGraphExecDestroy(c.graph);
    c.graph = nullptr;
  }
  return IRTPS_OK;
}

int irtps_get_tuning(irtps_ctx *ctx, int *blocks_per_sm, int *mip_cut) {
  if (!ctx) return IRTPS_EINVAL;
  Ctx &c = ctx->c;
  if (blocks_per_sm) *blocks_per_sm = c.sms > 0 ? c.trace_blocks / c.sms : 0;
  if (mip_cut) *mip_cut = c.mip_cut;
  return IRTPS_OK;
}

int irtps_set_ps_tuning(irtps_ctx *ctx, int pixels_per_thread) {
  if (!ctx) return IRTPS_EINVAL;
  Ctx &c = ctx->c;
  if (pixels_per_thread != 0 && pixels_per_thread != 1 && pixels_per_thread != 2 && pixels_per_thread != 4)
    return fail(c, IRTPS_EINVAL, "ps tuning: pixels_per_thread must be 0, 1, 2 or 4");
  c.ps_vec = pixels_per_thread == 0 ? 2 : pixels_per_thread;
  if (c.graph) {
    cudaGraphExecDestroy(c.graph);
    c.graph = nullptr;
  }
  return IRTPS_OK;
}

int irtps_get_ps_tuning(irtps_ctx *ctx, int *pixels_per_thread) {
  if (!ctx) return IRTPS_EINVAL;
  if (pixels_per_thread) *pixels_per_thread = irtps::ps_vec_for(ctx->c);
  return IRTPS_OK;
}

int irtps_autotune(irtps_ctx *ctx, int spp_probe, int bounces, uint64_t seed, double *out_ms) {
  if (!ctx) return IRTPS_EINVAL;
  Ctx &c = ctx->c;
  if (!trace_args_ok(c, spp_probe, bounces)) return fail(c, IRTPS_EINVAL, "autotune: bad arguments");
  const int mx = c.trace_per_sm_max;
  std::vector<int> per_sm;
  for (int v : {mx, mx - 1, mx - 2, (mx + 1) / 2})
    if (v >= 1 && std::find(per_sm.begin(), per_sm.end(), v) == per_sm.end()) per_sm.push_back(v);
  std::vector<int> cuts;
  for (int v = 0; v <= 3 && v < c.levels - 1; ++v) cuts.push_back(v);
  int rc = begin_call(c);
  if (rc) return rc;
  double best = INFINITY;
  int best_ps = c.trace_blocks / (c.sms > 0 ? c.sms : 1), best_cut = c.mip_cut;
  for (int cut : cuts)
    for (int ps : per_sm) {
      c.trace_blocks = ps * c.sms;
      c.mip_cut = cut;
      if ((rc = prepare_trace(c, c.H * c.W, spp_probe))) break;
      for (int rep = 0; rep < 2; ++rep) {  // the first run warms the caches; the second is timed
        c.tev_used = 0;
        if ((rc = trace_into(c, nullptr, c.H * c.W, spp_probe, bounces, seed, c.t, 0u, c.lbar, nullptr))) break;
      }
      if (rc) break;
      float ms = 0.0f;
      CK(cudaEventSynchronize(c.tev[1]), "autotune");
      CK(cudaEventElapsedTime(&ms, c.tev[0], c.tev[1]), "autotune");
      if (ms < best) {
        best = ms;
        best_ps = ps;
        best_cut = cut;
      }
    }
  c.trace_blocks = best_ps * c.sms;
  c.mip_cut = best_cut;
  // PS pixels per thread: timed at iteration 0 only, where the probe (classic PS from the
  // images) writes the state the context already holds, bit for bit
  if (!rc && c.have_images && c.t == 0 && !c.opt.ps_tensor) {
    float best_v_ms = INFINITY;
    int best_v = c.ps_vec;
    for (int v : {1, 2, 4}) {
      if ((c.H * c.W) % v) continue;
      c.ps_vec = v;
      for (int rep = 0; rep < 2 && !rc; ++rep) {
        c.tev_used = 0;
        rc = run_ps(c, true);
      }
      if (rc) break;
      float ms = 0.0f;
      CK(cudaEventSynchronize(c.tev[1]), "autotune");
      CK(cudaEventElapsedTime(&ms, c.tev[0], c.tev[1]), "autotune");
      if (ms < best_v_ms) {
        best_v_ms = ms;
        best_v = v;
      }
    }
    c.ps_vec = best_v;
  }
  c.tev_used = 0;
  if (c.graph) {
    cudaGraphExecDestroy(c.graph);
    c.graph = nullptr;
  }
  if (rc) return rc;
  rc = end_call(c, false);
  if (out_ms) *out_ms = best;
  return rc;
}

const char *irtps_last_error(const irtps_ctx *ctx) { return ctx ? ctx->c.err.c_str() : "null context"; }

void irtps_destroy(irtps_ctx *ctx) {
  if (!ctx) return;
  if (ctx->c.stream) cudaStreamSynchronize(ctx->c.stream);
  release(ctx->c);
  delete ctx;
}

}  // extern "C"
