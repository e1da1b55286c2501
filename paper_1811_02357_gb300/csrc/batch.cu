// Batches of objects: the IRT loop (Sec. IV) of many contexts with one launch
// per stage.  Each stage's kernel takes a table of per-object descriptors and
// maps its blocks (pyramid, PS, depth solve) or its work items (trace) onto the
// objects, so that the whole batch costs the launches of one object and small
// objects fill the GPU together.  Declarations and contracts: include/irtps.h.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "irtps_internal.h"

using irtps::Ctx;

constexpr int kMaxBatch = 64;

struct irtps_batch {
  std::vector<irtps_ctx *> objs;
  int n = 0, C = 0;
  bool shared = false;  // light-shared sampling (every object's option)
  int irls_iters = 0;   // robust-integration reweighting steps (every object's option)
  int mg_levels = 0;    // most multigrid levels of an object
  int use_graph = 0;
  cudaStream_t stream = nullptr;      // where the batch's work runs
  cudaStream_t own_stream = nullptr;
  std::string err;
  int sms = 0, trace_per_sm_max = 0, trace_per_sm = 0, mip_cut = 0;
  // device tables (owned)
  irtps::ObjTrace *d_trace = nullptr;
  void *d_ps = nullptr;    // PS descriptors (iterations: Lbar subtracted)
  void *d_ps0 = nullptr;   // PS descriptors of iteration 0 (classic PS: Lbar taken as 0)
  void *d_jobs = nullptr;  // depth-solve jobs
  irtps::SpectralBatch spectral;  // the direct solves of the objects that take them
  irtps::PyrObj *d_pyr = nullptr;
  irtps::ReduceObj *d_reduce = nullptr;  // light-shared: partial-sum buffers of the objects
  int reduce_blocks = 0;
  irtps::DevStats *d_stats = nullptr;  // per object (solver, D_H); [n]: trace counters
  unsigned *next_item = nullptr;
  uint32_t *iter_dev = nullptr;
  // launch geometry
  int pyr_levels = 0;
  std::vector<int> pyr_blocks;
  int hz_blocks = 0;  // batched horizon launch (early escape)
  int ps_blocks = 0, cg_blocks = 0;
  unsigned n_items = 0;
  unsigned long long primary_per_iter = 0;
  // captured iteration
  cudaGraphExec_t graph = nullptr;
  std::vector<int> g_spp, g_bounces;
  uint64_t g_seed = 0;
  int g_grid = -1, g_cut = -1;
  // timing
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> tev;
  std::vector<int> tev_stage;
  int tev_used = 0;
  irtps_stats stats{};
  std::vector<irtps::DevStats> h_stats;
};

namespace {

enum Stage { ST_TRACE = 0, ST_PS = 1, ST_DEPTH = 2 };

int bfail(irtps_batch &b, int code, const std::string &msg) {
  b.err = msg;
  return code;
}

int bcuda(irtps_batch &b, cudaError_t e, const char *what) {
  b.err = std::string(what) + ": " + cudaGetErrorString(e);
  return IRTPS_ECUDA;
}

#define BCK(call, what)                                   \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return bcuda(b, e_, what);     \
  } while (0)

void release(irtps_batch &b) {
  void *bufs[] = {b.d_trace,  b.d_ps,    b.d_ps0,     b.d_jobs,  b.d_pyr, b.d_reduce,
                  b.d_stats, b.next_item, b.iter_dev, b.spectral.table};
  for (void *p : bufs)
    if (p) cudaFree(p);
  if (b.graph) cudaGraphExecDestroy(b.graph);
  if (b.fork) cudaEventDestroy(b.fork);
  for (cudaEvent_t e : b.tev)
    if (e) cudaEventDestroy(e);
  if (b.own_stream) cudaStreamDestroy(b.own_stream);
}

int stage_mark(irtps_batch &b, int stage, bool start) {
  const int need = b.tev_used + 1;
  while ((int)b.tev.size() < 2 * need) {
    cudaEvent_t e;
    BCK(cudaEventCreate(&e), "timing events");
    b.tev.push_back(e);
  }
  if (start) {
    b.tev_stage.resize(need);
    b.tev_stage[b.tev_used] = stage;
    BCK(cudaEventRecord(b.tev[2 * b.tev_used], b.stream), "timing");
  } else {
    BCK(cudaEventRecord(b.tev[2 * b.tev_used + 1], b.stream), "timing");
    ++b.tev_used;
  }
  return IRTPS_OK;
}

#define BSTAGE(stage, start)                   \
  do {                                         \
    if (timed) {                               \
      int rc_ = stage_mark(b, stage, start);   \
      if (rc_) return rc_;                     \
    }                                          \
  } while (0)

int trace_grid(const irtps_batch &b) { return b.trace_per_sm * b.sms; }

// Kernels the robust-integration steps add to each batched solve.
int irls_kernels(const irtps_batch &b) {
  return b.irls_iters > 0 ? b.irls_iters * (1 + (b.mg_levels - 1) + 7) + 1 : 0;
}

// Kernels of the least-squares solve: seven, plus the six transform passes when some object solves directly.
int solve_kernels(const irtps_batch &b) { return 7 + (b.spectral.n > 0 ? 6 : 0); }

// Trace descriptors for this call: objects of larger per-item cost first, so
// that the cheap items of the last claims fill the tail of the launch.
int upload_trace(irtps_batch &b, const int *spp, const int *bounces, uint64_t seed) {
  std::vector<int> order(b.n);
  for (int i = 0; i < b.n; ++i) order[i] = i;
  auto cost = [&](int i) -> long long {  // samples x bounces of one work item (x K when shared)
    const Ctx &c = b.objs[i]->c;
    if (!b.shared) return (long long)spp[i] * bounces[i];
    return (long long)irtps::shared_split(c.H * c.W, spp[i]).chunk * bounces[i] * c.K;
  };
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost(x) > cost(y); });
  std::vector<irtps::ObjTrace> h(b.n);
  std::vector<irtps::ReduceObj> red(b.shared ? b.n : 0);
  unsigned begin = 0;
  unsigned long long primary = 0, items = 0;
  int rblk = 0;
  bool grown = false;
  for (int r = 0; r < b.n; ++r) {
    const int i = order[r];
    Ctx &c = b.objs[i]->c;
    const int P = c.H * c.W;
    irtps::ObjTrace &o = h[r];
    irtps::fill_obj_trace(c, o);
    o.f.levels = irtps::march_levels(c.levels, b.mip_cut);
    o.spp = spp[i];
    if (!irtps::early_escape_on(c, spp[i], true)) o.hz = nullptr;  // bounds computed, not used
    o.bounces = bounces[i];
    o.key = make_uint2((uint32_t)seed ^ c.obj, (uint32_t)(seed >> 32));
    o.out = c.lbar;
    o.item_begin = begin;
    o.iter0 = c.t;
    unsigned long long n_it = (unsigned long long)P * c.K;
    if (b.shared) {  // (chunk, pixel) items; partial sums in the object's scratch
      const irtps::SharedSplit sp = irtps::shared_split(P, spp[i]);
      o.n_chunks = sp.n_chunks;
      o.chunk = sp.chunk;
      bool g = false;
      BCK(irtps::ensure_shared_scratch(c, (size_t)o.n_chunks * (c.K + 1) * c.C * P, g), "light-shared partial sums");
      grown = grown || g;
      o.part = c.shared_part;
      n_it = (unsigned long long)P * o.n_chunks;
      irtps::ReduceObj &q = red[r];
      q.part = c.shared_part;
      q.out = c.lbar;
      q.n_chunks = o.n_chunks;
      q.n_pix = P;
      q.kc = c.K * c.C;
      q.C = c.C;
      q.inv_spp = 1.0 / (double)spp[i];
      q.blk_begin = rblk;
      q.nblk = (int)std::min<long long>(4096, std::max<long long>(1, ((long long)P * q.kc + 2047) / 2048));
      rblk += q.nblk;
    }
    begin += (unsigned)n_it;
    items += n_it;
    primary += (unsigned long long)P * (b.shared ? 1 : c.K) * spp[i];
  }
  if (grown && b.graph) {  // a captured iteration holds the old buffers
    cudaGraphExecDestroy(b.graph);
    b.graph = nullptr;
  }
  // claims run past the last item by at most one per lane: keep the counter far from wrapping
  if (items > (1ull << 32) - (1ull << 24))
    return bfail(b, IRTPS_EINVAL, "batch: too many work items (objects x lights x pixels >= 2^32 - 2^24)");
  b.n_items = begin;
  b.primary_per_iter = primary;
  BCK(cudaMemcpyAsync(b.d_trace, h.data(), sizeof(irtps::ObjTrace) * b.n, cudaMemcpyHostToDevice, b.stream),
      "trace descriptors");
  if (b.shared) {
    BCK(cudaMemcpyAsync(b.d_reduce, red.data(), sizeof(irtps::ReduceObj) * b.n, cudaMemcpyHostToDevice, b.stream),
        "partial-sum descriptors");
    if (rblk != b.reduce_blocks && b.graph) {
      cudaGraphExecDestroy(b.graph);
      b.graph = nullptr;
    }
    b.reduce_blocks = rblk;
  }
  return IRTPS_OK;
}

int enqueue_trace(irtps_batch &b, uint32_t iter, bool captured, bool timed) {
  BSTAGE(ST_TRACE, true);
  BCK(irtps::build_pyramid_batch(b.stream, b.d_pyr, b.n, b.pyr_levels, b.pyr_blocks.data()), "pyramid launch");
  BCK(irtps::launch_horizon_batch(b.stream, b.d_pyr, b.n, b.hz_blocks), "horizon bounds");
  if (b.shared) BCK(irtps::launch_parts_batch(b.stream, true, b.d_reduce, b.n, b.reduce_blocks), "partial sums");
  BCK(irtps::launch_trace_batch(b.stream, b.C, b.shared, b.d_trace, b.n, b.n_items, b.d_stats[b.n].counts,
                                b.next_item, captured ? b.iter_dev : nullptr, iter, trace_grid(b)),
      "trace launch");
  if (b.shared) BCK(irtps::launch_parts_batch(b.stream, false, b.d_reduce, b.n, b.reduce_blocks), "partial sums");
  BSTAGE(ST_TRACE, false);
  return IRTPS_OK;
}

// One IRT iteration of every object on the batch stream.
int enqueue_iteration(irtps_batch &b, uint32_t iter, bool captured) {
  const bool timed = !captured;
  int rc = enqueue_trace(b, iter, captured, timed);
  if (rc) return rc;
  BSTAGE(ST_PS, true);
  BCK(irtps::launch_ps_batch(b.stream, b.C, b.objs[0]->c.images_dtype, b.d_ps, b.n, b.ps_blocks), "ps launch");
  BSTAGE(ST_PS, false);
  BSTAGE(ST_DEPTH, true);
  BCK(irtps::solve_depth_batch_async(b.stream, b.d_jobs, b.n, b.cg_blocks, b.irls_iters, b.mg_levels, b.spectral), "depth solve launch");
  BSTAGE(ST_DEPTH, false);
  BCK(irtps::depth_change_batch_async(b.stream, b.d_jobs, b.n, b.cg_blocks), "depth change launch");
  if (captured) BCK(irtps::launch_next_iter(b.stream, b.iter_dev), "iteration counter");
  return IRTPS_OK;
}

int capture(irtps_batch &b, const int *spp, const int *bounces, uint64_t seed) {
  const bool same = b.graph && b.g_seed == seed && b.g_grid == trace_grid(b) && b.g_cut == b.mip_cut &&
                    std::equal(b.g_spp.begin(), b.g_spp.end(), spp) &&
                    std::equal(b.g_bounces.begin(), b.g_bounces.end(), bounces);
  if (same) return IRTPS_OK;
  if (b.graph) {
    cudaGraphExecDestroy(b.graph);
    b.graph = nullptr;
  }
  BCK(cudaStreamBeginCapture(b.stream, cudaStreamCaptureModeThreadLocal), "graph capture");
  const int rc = enqueue_iteration(b, 0u, true);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(b.stream, &g);
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return bcuda(b, e, "graph capture");
  const cudaError_t e2 = cudaGraphInstantiate(&b.graph, g, 0);
  cudaGraphDestroy(g);
  if (e2 != cudaSuccess) {
    b.graph = nullptr;
    return bcuda(b, e2, "graph instantiate");
  }
  b.g_spp.assign(spp, spp + b.n);
  b.g_bounces.assign(bounces, bounces + b.n);
  b.g_seed = seed;
  b.g_grid = trace_grid(b);
  b.g_cut = b.mip_cut;
  return IRTPS_OK;
}

// The batch stream waits for the work queued on every object's stream.
int fork_in(irtps_batch &b) {
  for (irtps_ctx *x : b.objs) {
    BCK(cudaEventRecord(b.fork, x->c.stream), "fork");
    BCK(cudaStreamWaitEvent(b.stream, b.fork, 0), "fork");
  }
  return IRTPS_OK;
}

int begin_call(irtps_batch &b) {
  int rc = fork_in(b);
  if (rc) return rc;
  BCK(cudaMemsetAsync(b.d_stats, 0, sizeof(irtps::DevStats) * (b.n + 1), b.stream), "statistics reset");
  BCK(cudaMemsetAsync(b.iter_dev, 0, sizeof(uint32_t), b.stream), "iteration counter");
  b.tev_used = 0;
  b.stats.trace_ms = b.stats.ps_ms = b.stats.depth_ms = 0.0;
  return IRTPS_OK;
}

// Wait for the call, read the statistics once, turn failures into codes.
int end_call(irtps_batch &b, bool had_solve, int n_iter, double *out_dH) {
  b.h_stats.resize(b.n + 1);
  BCK(cudaMemcpyAsync(b.h_stats.data(), b.d_stats, sizeof(irtps::DevStats) * (b.n + 1), cudaMemcpyDeviceToHost,
                      b.stream),
      "statistics");
  BCK(cudaStreamSynchronize(b.stream), "batch call");
  for (int i = 0; i < b.tev_used; ++i) {
    float ms = 0.0f;
    BCK(cudaEventElapsedTime(&ms, b.tev[2 * i], b.tev[2 * i + 1]), "timing");
    double *dst = b.tev_stage[i] == ST_TRACE ? &b.stats.trace_ms
                                             : (b.tev_stage[i] == ST_PS ? &b.stats.ps_ms : &b.stats.depth_ms);
    *dst += ms;
  }
  const irtps::DevStats &tr = b.h_stats[b.n];
  irtps_stats &s = b.stats;
  s.segments = tr.counts[1];
  s.walk_overflows = tr.counts[2];
  s.node_visits = tr.counts[3];
  s.tri_tests = tr.counts[4];
  s.draws = tr.counts[5];
  s.primary_segments = b.primary_per_iter * (unsigned long long)n_iter;
  s.iterations_done = had_solve ? n_iter : 0;
  s.cg_iterations = 0;
  s.cg_rel_residual = 0.0;
  s.dH_max = s.dH_rms = 0.0;
  int bad = -1, timeout = -1;
  for (int i = 0; i < b.n; ++i) {
    const irtps::DevStats &d = b.h_stats[i];
    if (!had_solve) break;
    s.cg_iterations = std::max(s.cg_iterations, d.cg.last_iters);
    s.cg_rel_residual = std::max(s.cg_rel_residual, d.cg.rel_last);
    s.dH_max = std::max(s.dH_max, d.dh_max);
    s.dH_rms = std::max(s.dH_rms, d.dh_rms);
    if (out_dH) out_dH[i] = d.dh_max;
    if (d.cg.err && timeout < 0) timeout = i;
    if (d.cg.bad && bad < 0) bad = i;
  }
  if (tr.counts[2]) return bfail(b, IRTPS_ETIMEOUT, "trace: a heightfield march exhausted its step budget");
  if (timeout >= 0)
    return bfail(b, IRTPS_ETIMEOUT, "depth solve of object " + std::to_string(timeout) + ": a barrier timed out");
  if (bad >= 0)
    return bfail(b, IRTPS_ENUMERIC, "depth solve of object " + std::to_string(bad) + ": relative residual " +
                                        std::to_string(b.h_stats[bad].cg.rel_last) + " above cg_tol or not finite");
  return IRTPS_OK;
}

// Objects' streams wait for the batch's work (later per-object calls see its results).
int join_out(irtps_batch &b) {
  BCK(cudaEventRecord(b.fork, b.stream), "join");
  for (irtps_ctx *x : b.objs) BCK(cudaStreamWaitEvent(x->c.stream, b.fork, 0), "join");
  return IRTPS_OK;
}

bool args_ok(irtps_batch &b, const int *spp, const int *bounces) {
  if (!spp || !bounces) {
    b.err = "spp and bounces arrays are required";
    return false;
  }
  for (int i = 0; i < b.n; ++i)
    if (spp[i] < 1 || bounces[i] < 1 || bounces[i] > 3) {
      b.err = "object " + std::to_string(i) + ": spp must be >= 1 and bounces in 1..3";
      return false;
    }
  return true;
}

int ready(irtps_batch &b) {
  const int dtype = b.objs[0]->c.images_dtype;
  for (int i = 0; i < b.n; ++i) {
    const Ctx &c = b.objs[i]->c;
    if (!c.have_images) return bfail(b, IRTPS_ENOTREADY, "object " + std::to_string(i) + ": no images set");
    if (c.images_dtype != dtype) return bfail(b, IRTPS_EINVAL, "objects differ in image dtype");
  }
  return IRTPS_OK;
}

int set_grid(irtps_batch &b, int per_sm, int cut) {
  if (per_sm < 0 || per_sm > b.trace_per_sm_max || cut < 0 || cut >= irtps::kMaxLevels)
    return bfail(b, IRTPS_EINVAL, "tuning: blocks_per_sm in 0.." + std::to_string(b.trace_per_sm_max) +
                                      ", mip_cut in 0..15");
  b.trace_per_sm = per_sm == 0 ? b.trace_per_sm_max : per_sm;
  b.mip_cut = cut;
  return IRTPS_OK;
}

}  // namespace

extern "C" {

int irtps_batch_create(irtps_batch **out, irtps_ctx *const *objs, int n_obj, int use_graph) {
  if (!out) return IRTPS_EINVAL;
  *out = nullptr;
  if (!objs || n_obj < 1 || n_obj > kMaxBatch) return IRTPS_EINVAL;
  for (int i = 0; i < n_obj; ++i)
    if (!objs[i]) return IRTPS_EINVAL;
  for (int i = 0; i < n_obj; ++i)
    for (int j = 0; j < i; ++j)
      if (objs[i] == objs[j]) return IRTPS_EINVAL;
  irtps_batch *x = new (std::nothrow) irtps_batch;
  if (!x) return IRTPS_ENOMEM;
  irtps_batch &b = *x;
  auto bail = [&](int rc) {
    release(b);
    delete x;
    return rc;
  };
  b.objs.assign(objs, objs + n_obj);
  b.n = n_obj;
  b.C = objs[0]->c.C;
  b.use_graph = use_graph ? 1 : 0;
  b.shared = objs[0]->c.opt.sampling == 1;
  b.irls_iters = objs[0]->c.opt.irls_iters;
  for (int i = 0; i < n_obj; ++i) {
    if (objs[i]->c.C != b.C || (objs[i]->c.opt.sampling == 1) != b.shared ||
        objs[i]->c.opt.irls_iters != b.irls_iters || objs[i]->c.opt.fill_holes)
      return bail(IRTPS_EINVAL);
    b.mg_levels = std::max(b.mg_levels, objs[i]->c.mg_levels);
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&b.sms, cudaDevAttrMultiProcessorCount, dev) !=
                                               cudaSuccess)
    return bail(IRTPS_ECUDA);
  const int limit = irtps::trace_grid_limit(b.C, n_obj, b.shared);
  b.trace_per_sm_max = b.sms > 0 ? limit / b.sms : 0;
  if (b.trace_per_sm_max < 1) return bail(IRTPS_ECUDA);
  b.trace_per_sm = b.trace_per_sm_max;
  if (cudaStreamCreateWithFlags(&b.own_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b.fork, cudaEventDisableTiming) != cudaSuccess)
    return bail(IRTPS_ECUDA);
  b.stream = b.own_stream;

  // pyramid: per level, each object's block range (none beyond its levels)
  std::vector<irtps::PyrObj> pyr(n_obj);
  for (int i = 0; i < n_obj; ++i) {
    irtps::fill_pyr_obj(objs[i]->c, pyr[i]);
    if (!irtps::early_escape_possible(objs[i]->c)) pyr[i].hz = nullptr;  // no trace of it would read them
    b.pyr_levels = std::max(b.pyr_levels, objs[i]->c.levels);
  }
  for (int i = 0; i < n_obj; ++i) {  // horizon bounds: 128 pixels per block for objects that keep them
    pyr[i].hz_blk = b.hz_blocks;
    if (pyr[i].hz) b.hz_blocks += (objs[i]->c.H * objs[i]->c.W + 127) / 128;
  }
  b.pyr_blocks.assign(b.pyr_levels, 0);
  for (int l = 0; l < b.pyr_levels; ++l)
    for (int i = 0; i < n_obj; ++i) {
      pyr[i].blk[l] = b.pyr_blocks[l];
      if (l < pyr[i].levels)
        b.pyr_blocks[l] += (pyr[i].lw[l] * pyr[i].lh[l] + irtps::kPyrThreads - 1) / irtps::kPyrThreads;
    }
  // PS: ceil(P / 256) blocks per object
  const size_t ps_bytes = irtps::ps_args_bytes();
  std::vector<unsigned char> ps(ps_bytes * n_obj), ps0(ps_bytes * n_obj);
  for (int i = 0; i < n_obj; ++i) {
    const Ctx &c = objs[i]->c;
    irtps::ps_fill_args(c, false, b.ps_blocks, ps.data() + ps_bytes * i);
    irtps::ps_fill_args(c, true, b.ps_blocks, ps0.data() + ps_bytes * i);
    b.ps_blocks += (c.H * c.W + 255) / 256;
  }
  // depth solves: every object gets a team, the co-resident grid shared in
  // proportion to the pixel counts (at most the object's own solve grid)
  const int budget = irtps::cg_batch_grid_limit();
  if (budget < n_obj) return bail(IRTPS_ECUDA);
  double total_p = 0.0;
  for (int i = 0; i < n_obj; ++i) total_p += (double)objs[i]->c.H * objs[i]->c.W;
  const size_t job_bytes = irtps::cg_job_bytes();
  std::vector<unsigned char> jobs(job_bytes * n_obj);
  b.cg_blocks = 0;
  std::vector<int> nblk(n_obj);
  for (int i = 0; i < n_obj; ++i) {
    const Ctx &c = objs[i]->c;
    const int share = 1 + (int)std::floor((double)(budget - n_obj) * ((double)c.H * c.W) / total_p);
    nblk[i] = std::max(1, std::min(share, c.cg_blocks));
  }
  if ((cudaMalloc((void **)&b.d_stats, sizeof(irtps::DevStats) * (n_obj + 1)) != cudaSuccess) ||
      (cudaMalloc((void **)&b.d_trace, sizeof(irtps::ObjTrace) * n_obj) != cudaSuccess) ||
      (cudaMalloc(&b.d_ps, ps_bytes * n_obj) != cudaSuccess) ||
      (cudaMalloc(&b.d_ps0, ps_bytes * n_obj) != cudaSuccess) || (cudaMalloc(&b.d_jobs, job_bytes * n_obj) != cudaSuccess) ||
      (cudaMalloc((void **)&b.d_pyr, sizeof(irtps::PyrObj) * n_obj) != cudaSuccess) ||
      (cudaMalloc((void **)&b.d_reduce, sizeof(irtps::ReduceObj) * n_obj) != cudaSuccess) ||
      (cudaMalloc((void **)&b.next_item, sizeof(unsigned)) != cudaSuccess) ||
      (cudaMalloc((void **)&b.iter_dev, sizeof(uint32_t)) != cudaSuccess)) {
    cudaGetLastError();
    return bail(IRTPS_ENOMEM);
  }
  for (int i = 0; i < n_obj; ++i) {
    irtps::cg_fill_job(objs[i]->c, nblk[i], b.cg_blocks, b.d_stats + i, jobs.data() + job_bytes * i);
    b.cg_blocks += nblk[i];
  }
  {
    std::vector<Ctx *> cs;
    for (int i = 0; i < n_obj; ++i) cs.push_back(&objs[i]->c);
    if (irtps::spectral_batch_setup(cs, b.spectral) != cudaSuccess) {
      cudaGetLastError();
      return bail(IRTPS_ENOMEM);
    }
  }
  if (cudaMemcpy(b.d_pyr, pyr.data(), sizeof(irtps::PyrObj) * n_obj, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b.d_ps, ps.data(), ps_bytes * n_obj, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b.d_ps0, ps0.data(), ps_bytes * n_obj, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b.d_jobs, jobs.data(), job_bytes * n_obj, cudaMemcpyHostToDevice) != cudaSuccess)
    return bail(IRTPS_ECUDA);
  for (int i = 0; i < n_obj; ++i) irtps_set_object(objs[i], (uint32_t)i);
  *out = x;
  return IRTPS_OK;
}

int irtps_batch_set_images(irtps_batch *x, const void *const *images, int dtype, int on_device) {
  if (!x) return IRTPS_EINVAL;
  irtps_batch &b = *x;
  if (!images || (dtype != IRTPS_F32 && dtype != IRTPS_F16))
    return bfail(b, IRTPS_EINVAL, "set_images: need n_obj image pointers and dtype IRTPS_F32 or IRTPS_F16");
  for (int i = 0; i < b.n; ++i)
    if (!images[i]) return bfail(b, IRTPS_EINVAL, "set_images: image pointer " + std::to_string(i) + " is NULL");
  int rc = begin_call(b);
  if (rc) return rc;
  for (int i = 0; i < b.n; ++i) {
    Ctx &c = b.objs[i]->c;
    const size_t bytes = (size_t)c.K * c.C * c.H * c.W * (dtype == IRTPS_F16 ? 2 : 4);
    BCK(cudaMemcpyAsync(c.images, images[i], bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                        b.stream),
        "set_images: copy");
    c.images_dtype = dtype;
    c.have_images = true;
    c.t = 0;
  }
  // iteration 0 of every object: classic PS, then integration from a flat start
  const bool timed = true;
  BSTAGE(ST_PS, true);
  BCK(irtps::launch_ps_batch(b.stream, b.C, dtype, b.d_ps0, b.n, b.ps_blocks), "ps launch");
  BSTAGE(ST_PS, false);
  BSTAGE(ST_DEPTH, true);
  BCK(irtps::zero_depth_batch_async(b.stream, b.d_jobs, b.n, b.cg_blocks), "depth reset");
  BCK(irtps::solve_depth_batch_async(b.stream, b.d_jobs, b.n, b.cg_blocks, b.irls_iters, b.mg_levels, b.spectral), "depth solve launch");
  BSTAGE(ST_DEPTH, false);
  b.primary_per_iter = 0;
  rc = end_call(b, true, 0, nullptr);
  b.stats.iterations_done = 0;
  b.stats.launches += 1 + 1 + solve_kernels(b) + irls_kernels(b);
  const int rj = join_out(b);
  return rc ? rc : rj;
}

int irtps_batch_iterate(irtps_batch *x, int n_iter, const int *spp, const int *bounces, uint64_t seed,
                        double *out_dH) {
  if (!x) return IRTPS_EINVAL;
  irtps_batch &b = *x;
  if (n_iter < 0) return bfail(b, IRTPS_EINVAL, "n_iter must be >= 0");
  if (!args_ok(b, spp, bounces)) return IRTPS_EINVAL;
  int rc = ready(b);
  if (rc) return rc;
  if (n_iter == 0) return IRTPS_OK;
  if ((rc = begin_call(b))) return rc;
  if ((rc = upload_trace(b, spp, bounces, seed))) return rc;
  if (b.use_graph) {
    if ((rc = capture(b, spp, bounces, seed))) return rc;
    for (int it = 0; it < n_iter; ++it) BCK(cudaGraphLaunch(b.graph, b.stream), "graph launch");
  } else {
    for (int it = 0; it < n_iter; ++it)
      if ((rc = enqueue_iteration(b, (uint32_t)it, false))) return rc;
  }
  rc = end_call(b, true, n_iter, out_dH);
  {  // kernels per iteration: pyramid levels, trace, PS, the solve's, two of D_H (+ counter)
    int k = 1 + 1 + solve_kernels(b) + 2 + (b.use_graph ? 1 : 0) + (b.shared ? 2 : 0) + (b.hz_blocks > 0 ? 1 : 0) +
            irls_kernels(b);
    for (int l = 0; l < b.pyr_levels; ++l) k += b.pyr_blocks[l] > 0 ? 1 : 0;
    b.stats.launches += (unsigned long long)k * n_iter;
  }
  for (irtps_ctx *o : b.objs) o->c.t += (uint32_t)n_iter;
  const int rj = join_out(b);
  return rc ? rc : rj;
}

int irtps_batch_set_stream(irtps_batch *b, void *stream) {
  if (!b) return IRTPS_EINVAL;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return bcuda(*b, cudaGetLastError(), "set_stream");
  b->stream = stream ? (cudaStream_t)stream : b->own_stream;
  if (b->graph) {  // captured on the old stream: capture again
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  return IRTPS_OK;
}

int irtps_batch_get_stats(irtps_batch *b, irtps_stats *out) {
  if (!b || !out) return IRTPS_EINVAL;
  *out = b->stats;
  return IRTPS_OK;
}

int irtps_batch_set_tuning(irtps_batch *b, int blocks_per_sm, int mip_cut) {
  if (!b) return IRTPS_EINVAL;
  return set_grid(*b, blocks_per_sm, mip_cut);
}

int irtps_batch_get_tuning(irtps_batch *b, int *blocks_per_sm, int *mip_cut) {
  if (!b) return IRTPS_EINVAL;
  if (blocks_per_sm) *blocks_per_sm = b->trace_per_sm;
  if (mip_cut) *mip_cut = b->mip_cut;
  return IRTPS_OK;
}

int irtps_batch_autotune(irtps_batch *x, const int *spp_probe, const int *bounces, uint64_t seed, double *out_ms) {
  if (!x) return IRTPS_EINVAL;
  irtps_batch &b = *x;
  if (!args_ok(b, spp_probe, bounces)) return IRTPS_EINVAL;
  int rc = ready(b);
  if (rc) return rc;
  int max_levels = 0;
  for (irtps_ctx *o : b.objs) max_levels = std::max(max_levels, o->c.levels);
  std::vector<int> per_sm;
  for (int v : {b.trace_per_sm_max, b.trace_per_sm_max - 1, b.trace_per_sm_max - 2, (b.trace_per_sm_max + 1) / 2})
    if (v >= 1 && std::find(per_sm.begin(), per_sm.end(), v) == per_sm.end()) per_sm.push_back(v);
  std::vector<int> cuts;
  for (int v = 0; v <= 3 && v < max_levels - 1; ++v) cuts.push_back(v);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  BCK(cudaEventCreate(&e0), "autotune");
  BCK(cudaEventCreate(&e1), "autotune");
  double best = INFINITY;
  int best_ps = b.trace_per_sm, best_cut = b.mip_cut;
  rc = fork_in(b);
  for (int cut : cuts) {
    for (int ps : per_sm) {
      if (rc) break;
      b.trace_per_sm = ps;
      b.mip_cut = cut;
      if ((rc = upload_trace(b, spp_probe, bounces, seed))) break;
      float ms = 0.0f;
      for (int rep = 0; rep < 2 && !rc; ++rep) {  // the first run warms the caches; the second is timed
        cudaEventRecord(e0, b.stream);
        rc = enqueue_trace(b, 0u, false, false);
        cudaEventRecord(e1, b.stream);
      }
      if (rc) break;
      const cudaError_t e = cudaEventSynchronize(e1);
      if (e != cudaSuccess) {
        rc = bcuda(b, e, "autotune");
        break;
      }
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) {
        best = ms;
        best_ps = ps;
        best_cut = cut;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b.trace_per_sm = best_ps;
  b.mip_cut = best_cut;
  if (rc) return rc;
  if (out_ms) *out_ms = best;
  return join_out(b);
}

const char *irtps_batch_last_error(const irtps_batch *b) { return b ? b->err.c_str() : "null batch"; }

void irtps_batch_destroy(irtps_batch *b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  release(*b);
  delete b;
}

}  // extern "C"
