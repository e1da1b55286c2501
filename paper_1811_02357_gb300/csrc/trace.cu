// Reverted Monte-Carlo trace (Sec. IV, Eq. 5-7): min/max pyramid build, the
// trace kernel (per light or light-shared, single object or batched), the
// stage-0 forward render, and geometry probes used by the parity tests.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <cuda_fp16.h>

#include "geom.cuh"
#include "irtps_internal.h"

namespace irtps {

// ---------------------------------------------------------------------------
// Min / max pyramid.  Level 0: one node per cell, over its 4 vertex heights.
// Level l: one node per 2x2 block of level l-1 nodes (clipped at the border).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pyramid_leaf_node(const float *__restrict__ depth, int W, int Wc, int i,
                                                  float *__restrict__ pmin, float *__restrict__ pmax) {
  const int cy = i / Wc, cx = i - cy * Wc;
  const float *r = depth + (size_t)cy * W + cx;
  const float a = r[0], b = r[1], c = r[W], d = r[W + 1];
  pmin[i] = fminf(fminf(a, b), fminf(c, d));
  pmax[i] = fmaxf(fmaxf(a, b), fmaxf(c, d));
}

__device__ __forceinline__ void pyramid_up_node(const float *__restrict__ cmin, const float *__restrict__ cmax,
                                                int cw, int ch, int w, int i, float *__restrict__ pmin,
                                                float *__restrict__ pmax) {
  const int y = i / w, x = i - y * w;
  float lo = __int_as_float(0x7f800000), hi = -lo;
  for (int dy = 0; dy < 2; ++dy) {
    const int yy = 2 * y + dy;
    if (yy >= ch) break;
    for (int dx = 0; dx < 2; ++dx) {
      const int xx = 2 * x + dx;
      if (xx >= cw) break;
      lo = fminf(lo, cmin[yy * cw + xx]);
      hi = fmaxf(hi, cmax[yy * cw + xx]);
    }
  }
  pmin[i] = lo;
  pmax[i] = hi;
}

__global__ void k_pyramid_leaf(const float *__restrict__ depth, int H, int W, float *__restrict__ pmin,
                               float *__restrict__ pmax) {
  const int Wc = W - 1, Hc = H - 1;
  const int n = Wc * Hc;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    pyramid_leaf_node(depth, W, Wc, i, pmin, pmax);
}

__global__ void k_pyramid_up(const float *__restrict__ cmin, const float *__restrict__ cmax, int cw, int ch,
                             float *__restrict__ pmin, float *__restrict__ pmax, int w, int h) {
  const int n = w * h;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    pyramid_up_node(cmin, cmax, cw, ch, w, i, pmin, pmax);
}

// Batched pyramid level l over many objects: object o owns the blocks
// [blk[l] of o, blk[l] of o + 1) of the launch (none once its levels run out).
__global__ void k_pyramid_b(const PyrObj *__restrict__ objs, int n, int l) {
  __shared__ int s_o;
  if (threadIdx.x == 0) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (objs[mid].blk[l] <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
    }
    s_o = lo;
  }
  __syncthreads();
  const PyrObj &o = objs[s_o];
  if (l >= o.levels) return;
  const int i = ((int)blockIdx.x - o.blk[l]) * blockDim.x + threadIdx.x;
  if (i >= o.lw[l] * o.lh[l]) return;
  if (l == 0) {
    const int W = o.W, Wc = W - 1;
    pyramid_leaf_node(o.depth, W, Wc, i, o.pmin, o.pmax);
    if (o.prev) {  // each cell saves its lower-left vertex; the last row and column their others
      const int cy = i / Wc, cx = i - cy * Wc;
      const size_t v = (size_t)cy * W + cx;
      o.prev[v] = o.depth[v];
      const bool last_x = cx == Wc - 1, last_y = cy == o.H - 2;
      if (last_x) o.prev[v + 1] = o.depth[v + 1];
      if (last_y) o.prev[v + W] = o.depth[v + W];
      if (last_x && last_y) o.prev[v + W + 1] = o.depth[v + W + 1];
    }
  } else
    pyramid_up_node(o.pmin + o.off[l - 1], o.pmax + o.off[l - 1], o.lw[l - 1], o.lh[l - 1], o.lw[l], i,
                    o.pmin + o.off[l], o.pmax + o.off[l]);
}

void fill_pyr_obj(const Ctx &c, PyrObj &o) {
  o.hz = c.horizon;
  o.hz_blk = 0;
  o.depth = c.depth;
  o.prev = c.depth_prev;
  o.pmin = c.pmin;
  o.pmax = c.pmax;
  o.H = c.H;
  o.W = c.W;
  o.levels = c.levels;
  for (int l = 0; l < kMaxLevels; ++l) {
    o.off[l] = c.off[l];
    o.lw[l] = c.lw[l];
    o.lh[l] = c.lh[l];
    o.blk[l] = 0;
  }
}

// One launch per level; blocks[l] = total blocks of level l (objects' ranges set in d_objs).
cudaError_t build_pyramid_batch(cudaStream_t s, const PyrObj *d_objs, int n, int levels, const int *blocks) {
  for (int l = 0; l < levels; ++l)
    if (blocks[l] > 0) k_pyramid_b<<<blocks[l], kPyrThreads, 0, s>>>(d_objs, n, l);
  return cudaGetLastError();
}

cudaError_t build_pyramid(Ctx &c) {
  const int Wc = c.W - 1, Hc = c.H - 1;
  const int threads = 256;
  int blocks = (Wc * Hc + threads - 1) / threads;
  blocks = blocks < 1 ? 1 : (blocks > 4096 ? 4096 : blocks);
  k_pyramid_leaf<<<blocks, threads, 0, c.stream>>>(c.depth, c.H, c.W, c.pmin, c.pmax);
  c.stats.launches += c.levels;
  for (int l = 1; l < c.levels; ++l) {
    const int n = c.lw[l] * c.lh[l];
    int b = (n + threads - 1) / threads;
    b = b > 4096 ? 4096 : b;
    k_pyramid_up<<<b, threads, 0, c.stream>>>(c.pmin + c.off[l - 1], c.pmax + c.off[l - 1], c.lw[l - 1],
                                               c.lh[l - 1], c.pmin + c.off[l], c.pmax + c.off[l], c.lw[l],
                                               c.lh[l]);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Horizon bounds (see octant_of in geom.cuh): one thread per pixel, all eight
// octants at once, a fixed scan of the max pyramid.  At level l the thread looks
// at the nodes within kHorizonRing nodes of p's own node, except those lying
// wholly inside the window of level l - 1 (covered by finer nodes); the windows
// are nested and the top level covers the grid, so every cell is covered by
// some scanned node, and cells touching p (tested exactly by the march) only at
// level 0, where they are left out.  A node bounds the cells it must cover - its
// part outside the finer window - by (node max - H_p) / d, d the least distance
// from p to that part (to a node's part beyond the window's left edge, at least
// that edge's distance from p, and so on).  The bound is not tight (far cells are
// judged by their coarse nodes) but costs a fixed number of nodes per level.
// FP32 with every rounding directed toward a larger bound.
// ---------------------------------------------------------------------------
#ifndef IRTPS_HORIZON_RING
#define IRTPS_HORIZON_RING 4
#endif
constexpr int kHorizonRing = IRTPS_HORIZON_RING;  // >= 2: nodes touching p stay inside the finer window
static_assert(kHorizonRing >= 2, "a node touching p must lie inside the finer window");

__device__ __forceinline__ void horizon_pixel(const float *__restrict__ depth, const float *__restrict__ pmax,
                                              const int *off, const int *lw, int H, int W, int levels, int p,
                                              float *__restrict__ hz) {
  const int P = H * W, Wc = W - 1, Hc = H - 1;
  const int pi = p / W, pj = p - pi * W;
  const float zp = __ldg(depth + p);
  float best[8];
#pragma unroll
  for (int o = 0; o < 8; ++o) best[o] = -INFINITY;
  bool none = false;                        // a node touching p outside the finer window: no bound
  int ix0 = 0, ix1 = 0, iy0 = 0, iy1 = 0;   // cells of the previous level's window (empty at level 0)
  const int ci = min(pi, Hc - 1), cj = min(pj, Wc - 1);  // a cell at vertex p
  for (int l = 0; l < levels && !none; ++l) {
    const int nw = lw[l], nh = ((Hc - 1) >> l) + 1;
    const int cx = cj >> l, cy = ci >> l;
    const int x_lo = max(cx - kHorizonRing, 0), x_hi = min(cx + kHorizonRing, nw - 1);
    const int y_lo = max(cy - kHorizonRing, 0), y_hi = min(cy + kHorizonRing, nh - 1);
    for (int ny = y_lo; ny <= y_hi && !none; ++ny) {
      const int Y0 = ny << l, Y1 = min(Y0 + (1 << l), Hc);
      const int b1 = Y0 - pi, b2 = Y1 - pi;
      const int dy = max(max(b1, -b2), 0);
      const bool y_in = Y0 >= iy0 && Y1 <= iy1;
      for (int nx = x_lo; nx <= x_hi; ++nx) {
        const int X0 = nx << l, X1 = min(X0 + (1 << l), Wc);
        if (y_in && X0 >= ix0 && X1 <= ix1) continue;  // covered by the finer levels
        const int a1 = X0 - pj, a2 = X1 - pj;
        const int dx = max(max(a1, -a2), 0);
        if (dx == 0 && dy == 0 && l == 0) continue;  // a cell touching p
        // squared distance to the node's part outside the finer window
        int d2i = dx * dx + dy * dy;
        if (l > 0) {
          const int big = 1 << 30;
          int hx = big, vy = big;  // across its columns beyond the window, its rows beyond the window
          if (X0 < ix0) hx = min(hx, max(dx, pj - ix0));
          if (X1 > ix1) hx = min(hx, max(dx, ix1 - pj));
          if (Y0 < iy0) vy = min(vy, max(dy, pi - iy0));
          if (Y1 > iy1) vy = min(vy, max(dy, iy1 - pi));
          d2i = min(hx < big ? hx * hx + dy * dy : big, vy < big ? dx * dx + vy * vy : big);
        }
        if (d2i == 0) {
          none = true;
          break;
        }
        bool meets[8], any = false;
#pragma unroll
        for (int o = 0; o < 8; ++o) {
          meets[o] = wedge_meets(o, a1, a2, b1, b2);
          any = any || meets[o];
        }
        if (!any) continue;
        const float nmax = __ldg(pmax + off[l] + ny * nw + nx);
        // (nmax - zp) / distance, every rounding toward a larger bound
        const float num = __fsub_ru(nmax, zp);
        const float dist = num >= 0.0f ? __fsqrt_rd((float)d2i) : __fsqrt_ru((float)d2i);  // d2i < 2^24: exact
        const float bnd = __fdiv_ru(num, dist);
#pragma unroll
        for (int o = 0; o < 8; ++o)
          if (meets[o]) best[o] = fmaxf(best[o], bnd);
      }
    }
    ix0 = x_lo << l;
    ix1 = min((x_hi + 1) << l, Wc);
    iy0 = y_lo << l;
    iy1 = min((y_hi + 1) << l, Hc);
  }
#pragma unroll
  for (int o = 0; o < 8; ++o) hz[(size_t)o * P + p] = none ? INFINITY : best[o];
}

// levels: of the full pyramid (its top node covers the grid), whatever the march uses.
__global__ void k_horizon(const Field f, int levels, float *__restrict__ hz) {
  __shared__ int s_off[kMaxLevels], s_lw[kMaxLevels];
  if (threadIdx.x < kMaxLevels) {
    s_off[threadIdx.x] = f.off[threadIdx.x];
    s_lw[threadIdx.x] = f.lw[threadIdx.x];
  }
  __syncthreads();
  const int P = f.H * f.W;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x)
    horizon_pixel(f.depth, f.pmax, s_off, s_lw, f.H, f.W, levels, p, hz);
}

// Batched: object o owns blocks [hz_blk of o, hz_blk of o + 1) (128 pixels each).
__global__ void k_horizon_b(const PyrObj *__restrict__ objs, int n) {
  __shared__ int s_o;
  if (threadIdx.x == 0) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (objs[mid].hz_blk <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
    }
    s_o = lo;
  }
  __syncthreads();
  const PyrObj &o = objs[s_o];
  if (!o.hz) return;
  const int p = ((int)blockIdx.x - o.hz_blk) * blockDim.x + threadIdx.x;
  if (p < o.H * o.W) horizon_pixel(o.depth, o.pmax, o.off, o.lw, o.H, o.W, o.levels, p, o.hz);
}

cudaError_t launch_horizon(Ctx &c, int spp) {
  if (!early_escape_on(c, spp)) return cudaSuccess;
  const int P = c.H * c.W;
  k_horizon<<<(P + 127) / 128, 128, 0, c.stream>>>(c.field(), c.levels, c.horizon);
  ++c.stats.launches;
  return cudaGetLastError();
}

cudaError_t launch_horizon_batch(cudaStream_t s, const PyrObj *d_objs, int n, int blocks) {
  if (blocks > 0) k_horizon_b<<<blocks, 128, 0, s>>>(d_objs, n);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Environment: bilinear lookup in a C x EH x EW latitude-longitude map over the
// full sphere (theta = acos(w_z) down the rows, phi = atan2(w_y, w_x) across,
// texel centres at half-integers, wrap in phi, clamp in theta).
// ---------------------------------------------------------------------------
template <int C>
__device__ __forceinline__ void env_lookup(const float *__restrict__ env, int EH, int EW, F3 w, float *out) {
  const float inv = rsqrtf(w.x * w.x + w.y * w.y + w.z * w.z);
  const float z = fminf(1.0f, fmaxf(-1.0f, w.z * inv));
  const float theta = acosf(z);
  float phi = atan2f(w.y, w.x);
  if (phi < 0.0f) phi += 6.28318530717958647692f;
  const float row = theta * ((float)EH * 0.318309886183790671538f) - 0.5f;
  const float col = phi * ((float)EW * 0.159154943091895335769f) - 0.5f;
  const float r0 = floorf(row), c0 = floorf(col);
  const float fr = row - r0, fc = col - c0;
  const int ra = min(EH - 1, max(0, (int)r0));
  const int rb = min(EH - 1, max(0, (int)r0 + 1));
  int ca = (int)c0 % EW;
  if (ca < 0) ca += EW;
  const int cb = ca + 1 == EW ? 0 : ca + 1;
#pragma unroll
  for (int c = 0; c < C; ++c) {
    const float *m = env + (size_t)c * EH * EW;
    const float top = (1.0f - fc) * __ldg(m + ra * EW + ca) + fc * __ldg(m + ra * EW + cb);
    const float bot = (1.0f - fc) * __ldg(m + rb * EW + ca) + fc * __ldg(m + rb * EW + cb);
    out[c] = (1.0f - fr) * top + fr * bot;
  }
}

// ---------------------------------------------------------------------------
// The trace.  A work item (light k, pixel p) runs its spp sample paths in
// order in one lane, Kahan-summing their radiance in FP32.  Sample path: bounce
// b = 1..B draws Philox4x32-10 at counter {p, s, (k<<8)|(b<<4)|stream, iteration}
// with key {seed_lo ^ obj, seed_hi}, samples a cosine direction about the
// current normal estimate at the origin, and marches the heightfield.  Escape:
// add T * Env(w), stop.  Hit at q (nearest vertex): add
// T * rho_q * max(0, n_q . l_k) * V_k(q) (V from a shadow ray, cast when
// n_q . l_k > 0), then T <- T * rho_q and continue from q lifted by eps.
// Lbar(k, c, p) = sum / spp: mean incident radiance (irradiance / pi).
//
// Execution: every lane is a small state machine (set up a segment -> march ->
// resolve).  March steps of all lanes run in a loop that the warp leaves only
// when at most half of its live lanes are still marching; the finished lanes
// then resolve and set up their next segments together.  Lanes therefore stay
// busy although path lengths differ widely, while each lane's own sequence of
// operations - and so every result bit - is that of a plain sequential trace.
// ---------------------------------------------------------------------------
// One trace launch: a single object (`one`) or a batch of objects whose work
// items follow one another in descriptor order.
struct TraceArgs {
  ObjTrace one;
  const ObjTrace *objs;        // batched launch: n_obj descriptors in device memory
  int n_obj;
  unsigned n_items;            // all work items of the launch
  const int32_t *pixels;       // optional pixel list (single object)
  int32_t *rec;                // optional records (single object): per light n_pix*K*spp*B*2,
                               // light-shared n_pix*spp*B*(1+K)
  unsigned long long *counts;  // {unused, segments, walk overflows, node visits, triangle tests, draws}
  unsigned *next_item;         // work-item counter, zero before the launch
  const uint32_t *iter_dev;    // when set, the iteration field is read here (graph replays)
  uint32_t iter, stream;
};

#ifndef IRTPS_TRACE_MINB
#define IRTPS_TRACE_MINB 9
#endif
#ifndef IRTPS_TRACE_MINB_BATCH
#define IRTPS_TRACE_MINB_BATCH 8
#endif
#ifndef IRTPS_TRACE_MINB_SHARED
#define IRTPS_TRACE_MINB_SHARED 9
#endif
#ifndef IRTPS_MARCH_KEEP
#define IRTPS_MARCH_KEEP 2
#endif
#ifndef IRTPS_LEAF_BATCH
#define IRTPS_LEAF_BATCH 4
#endif
constexpr int kTraceThreads = 128;
// leave the march loop when marching lanes <= live lanes / kMarchKeep
constexpr int kMarchKeep = IRTPS_MARCH_KEEP;
// run leaf steps once kLeafBatch * (lanes waiting for one) >= lanes doing node steps
constexpr int kLeafBatch = IRTPS_LEAF_BATCH;
enum : int { PH_SETUP = 0, PH_MARCH = 1, PH_RESOLVE = 2, PH_DONE = 3 };

// Dynamic shared memory of a trace launch over n objects: level tables and item ranges.
static size_t trace_smem_bytes(int n) { return (size_t)n * sizeof(LevelTable) + (size_t)(n + 1) * sizeof(unsigned); }

template <int C, bool BATCH, bool SHARED>
__global__ void __launch_bounds__(kTraceThreads,
                                  BATCH ? IRTPS_TRACE_MINB_BATCH : (SHARED ? IRTPS_TRACE_MINB_SHARED : IRTPS_TRACE_MINB))
    k_trace(const __grid_constant__ TraceArgs a) {
  extern __shared__ __align__(16) unsigned char trace_smem[];
  LevelTable *lts = reinterpret_cast<LevelTable *>(trace_smem);
  const int n_obj = BATCH ? a.n_obj : 1;
  unsigned *s_begin = reinterpret_cast<unsigned *>(lts + n_obj);
  if constexpr (BATCH) {
    for (int i = threadIdx.x; i < n_obj * kMaxLevels; i += blockDim.x) {
      const int o = i / kMaxLevels, l = i - o * kMaxLevels;
      lts[o].ol[l] = make_int2(a.objs[o].f.off[l], a.objs[o].f.lw[l]);
    }
    for (int o = threadIdx.x; o < n_obj; o += blockDim.x) {
      set_height_bounds(a.objs[o].f, lts + o);
      s_begin[o] = a.objs[o].item_begin;
    }
    __syncthreads();
  } else {
    load_levels(a.one.f, lts);
  }
  // Work items.  Per-light sampling: (object, light k, pixel), within an object
  // item = k * n_pix + ip, all spp samples of (p, k).  Light-shared sampling:
  // (chunk j, pixel), item = j * n_pix + ip, samples [j * chunk, (j + 1) * chunk)
  // of pixel p for all lights.  Each lane starts with the item of its global
  // index and, when done, takes the next unclaimed item from a counter (claimed a
  // warp at a time), so that no lane idles while items remain.  An item is
  // always traced by one lane, samples in order.
  const unsigned n_items = a.n_items;
  unsigned item = blockIdx.x * blockDim.x + threadIdx.x;
  const ObjTrace *ob = &a.one;
  const LevelTable *lt = lts;
  // the item's indices and the path's bounce state, used at set-up and resolve only, in shared-memory
  // columns (one per lane) like the path's sums below: the registers go to the march
  __shared__ int s_item[9][kTraceThreads];
  int &k = s_item[0][threadIdx.x], &ip = s_item[1][threadIdx.x], &p = s_item[2][threadIdx.x];
  int &j = s_item[3][threadIdx.x], &s_end = s_item[4][threadIdx.x];
  k = ip = p = j = s_end = 0;
  auto take = [&](unsigned it) -> int {  // returns the item's first sample
    item = it;
    if constexpr (BATCH) {
      int lo = 0, hi = n_obj - 1;  // last object whose range starts at or before it
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (s_begin[mid] <= it) lo = mid; else hi = mid - 1;
      }
      ob = a.objs + lo;
      lt = lts + lo;
      it -= s_begin[lo];
    }
    const int q = (int)(it / (unsigned)ob->n_pix);
    ip = (int)it - q * ob->n_pix;
    p = a.pixels ? a.pixels[ip] : ip;
    if constexpr (SHARED) {
      j = q;
      s_end = min(ob->spp, (j + 1) * ob->chunk);
      return j * ob->chunk;
    } else {
      k = q;
      return 0;
    }
  };
  const bool alive = item < n_items;
  int &s = s_item[5][threadIdx.x];
  s = alive ? take(item) : 0;
  // the pixel's own vertex, lifted: origin of every primary ray of this lane
  auto pixel_origin = [&]() -> F3 {
    const int W = ob->f.W;
    const int pi = p / W, pj = p - pi * W;
    return F3{(float)pj, (float)pi, radd(__ldg(ob->f.depth + p), ob->eps)};
  };
  auto light_k = [&](int kk) -> F3 {
    const float *l = ob->lights + 3 * kk;
    return F3{__ldg(l), __ldg(l + 1), __ldg(l + 2)};
  };
  auto budget0 = [&]() -> int { return 8 * (ob->f.Wc + ob->f.Hc + 8) * (ob->f.levels + 1); };
  const uint32_t iter_base = a.iter_dev ? *a.iter_dev : a.iter;

  int phase = alive ? PH_SETUP : PH_DONE;
  int &b = s_item[6][threadIdx.x], &qp = s_item[7][threadIdx.x], &ks = s_item[8][threadIdx.x];
  b = 1;
  qp = 0;
  ks = 0;
  int budget = alive ? budget0() : 0;
  bool shadow = false;
  float cosv = 0.0f;
  // the path's throughput and radiance (touched once per segment) and the item's Kahan sums over
  // samples (once per sample) in shared memory, one column per lane: the registers they free keep
  // the march's state out of local memory
  __shared__ float s_path[4][3][kTraceThreads];
  auto thr = [&](int c) -> float & { return s_path[0][c][threadIdx.x]; };
  auto acc = [&](int c) -> float & { return s_path[1][c][threadIdx.x]; };
  auto sum = [&](int c) -> float & { return s_path[2][c][threadIdx.x]; };
  auto comp = [&](int c) -> float & { return s_path[3][c][threadIdx.x]; };
#pragma unroll
  for (int c = 0; c < C; ++c) {
    thr(c) = 1.0f;
    acc(c) = sum(c) = comp(c) = 0.0f;
  }
  Walker m;
  bool at_leaf = false;
  bool seen = false;  // per-light item: some sample's first segment hit the surface
  Work w;
  uint32_t segs = 0;
  int overflow = 0;

  // records: per light {hit, visibility} per bounce; light-shared {hit, V_0 .. V_{K-1}} per bounce
  auto rec_slot = [&](int bb) -> int32_t * {
    if constexpr (SHARED)
      return a.rec + (((size_t)ip * ob->spp + s) * ob->bounces + (bb - 1)) * (1 + ob->K);
    else
      return a.rec + ((((size_t)ip * ob->K + k) * ob->spp + s) * ob->bounces + (bb - 1)) * 2;
  };
  auto rec_width = [&]() -> int { return SHARED ? 1 + ob->K : 2; };
  auto albedo_at = [&](int c, int q) -> float {
    return __ldg(ob->albedo + (size_t)c * ob->f.H * ob->f.W + q);
  };
  // light-shared: the direct term of light kk at the current hit, into the item's
  // partial sums (K x C contiguous per item, so a lane's updates stay in one or two lines)
  auto add_direct = [&](int kk) {
    float *d = ob->part + ((size_t)j * ob->n_pix + ip) * ob->K * C + kk * C;
#pragma unroll
    for (int c = 0; c < C; ++c) d[c] += thr(c) * albedo_at(c, qp) * cosv;
  };
  auto end_sample = [&]() {
#pragma unroll
    for (int c = 0; c < C; ++c) {  // Kahan summation over samples
      const float y = acc(c) - comp(c);
      const float t = sum(c) + y;
      comp(c) = (t - sum(c)) - y;
      sum(c) = t;
      acc(c) = 0.0f;
      thr(c) = 1.0f;
    }
    ++s;
    b = 1;
    budget = budget0();
    phase = PH_SETUP;
  };
  // after a hit at pixel q (qp) the next bounce starts from the lifted hit point,
  // which the walker keeps as its origin m.o until the next set-up
  auto continue_path = [&](int q) {
#pragma unroll
    for (int c = 0; c < C; ++c) thr(c) *= albedo_at(c, q);
    if (b < ob->bounces) {
      ++b;
      phase = PH_SETUP;
    } else {
      end_sample();
    }
  };
  // light-shared: the next light from ks on that faces the hit normal gets its
  // shadow ray (or, without shadow rays, its direct term); then the path goes on
  auto next_light = [&]() {
    const float4 m4 = __ldg(ob->nrm + qp);
    const F3 nq = {m4.x, m4.y, m4.z};
    while (ks < ob->K) {
      const F3 l = light_k(ks);
      if (f3dot(nq, l) > 0.0f) {
        cosv = fmaxf(0.0f, nq.x * l.x + nq.y * l.y + nq.z * l.z);
        if (ob->shadow) {
          walker_init(m, m.o, F3{rmul(l.x, ob->Wf), rmul(l.y, ob->Wf), l.z}, true, lt->zmax_margin);
          shadow = true;
          ++segs;
          budget = budget0();
          phase = PH_MARCH;
          return;
        }
        if (a.rec) rec_slot(b)[1 + ks] = 1;
        add_direct(ks);
      }
      ++ks;
    }
    shadow = false;
    continue_path(qp);
  };

  while (true) {
    // ---- finished items: store the result and claim the next item ----
    const bool item_done = phase == PH_SETUP && s >= (SHARED ? s_end : ob->spp);
    const unsigned need = __ballot_sync(0xffffffffu, item_done);
    if (need) {
      if (item_done) {
        if constexpr (SHARED) {
          // the environment part, common to every light, in the item's own C sums
          // (after all chunks' light sums); the reduction adds it to each light
          float *e = ob->part + ((size_t)ob->n_chunks * ob->n_pix * ob->K + (size_t)j * ob->n_pix + ip) * C;
#pragma unroll
          for (int c = 0; c < C; ++c) e[c] = sum(c);
        } else {
          const float inv = 1.0f / (float)ob->spp;
#pragma unroll
          for (int c = 0; c < C; ++c) ob->out[((size_t)k * C + c) * ob->n_pix + ip] = sum(c) * inv;
          if (ob->hole) ob->hole[(size_t)k * ob->n_pix + ip] = seen ? 0 : 1;
          seen = false;
        }
#pragma unroll
        for (int c = 0; c < C; ++c) sum(c) = comp(c) = 0.0f;
      }
      const int lane = threadIdx.x & 31;
      const int leader = __ffs(need) - 1;
      unsigned base = 0;
      // the counter counts claims beyond the lanes' start items (one per thread of the grid)
      if (lane == leader) base = atomicAdd(a.next_item, (unsigned)__popc(need)) + gridDim.x * blockDim.x;
      base = __shfl_sync(0xffffffffu, base, leader);
      if (item_done) {
        const unsigned mine = base + (unsigned)__popc(need & ((1u << lane) - 1u));
        if (mine < n_items) {
          s = take(mine);
          b = 1;
          budget = budget0();
        } else {
          phase = PH_DONE;
        }
      }
    }
    // ---- set up the next primary or bounce segment ----
    if (phase == PH_SETUP) {
      if (a.rec && b == 1) {
        int32_t *r = rec_slot(1);
        const int n = rec_width() * ob->bounces;
        for (int i = 0; i < n; ++i) r[i] = -2;
      }
      const uint32_t lf = SHARED ? 0u : (uint32_t)k;
      const uint4 x = philox4x32_10(
          make_uint4((uint32_t)p, (uint32_t)s, (lf << 8) | ((uint32_t)b << 4) | a.stream, ob->iter0 + iter_base),
          ob->key);
      // bounce 1 leaves the pixel's own vertex about its normal; later bounces the
      // previous hit point (m.o) about the hit pixel's normal
      const F3 org = b == 1 ? pixel_origin() : m.o;
      const float4 n4 = __ldg(ob->nrm + (b == 1 ? p : qp));
      const F3 dw = cosine_dir(F3{n4.x, n4.y, n4.z}, x.x, x.y);
      const F3 dg = {rmul(dw.x, ob->Wf), rmul(dw.y, ob->Wf), dw.z};
      walker_init(m, org, dg, false, lt->zmax_margin);
      shadow = false;
      ++segs;
      ++w.draws;
      phase = PH_MARCH;
      // early escape: a rising primary ray steeper than the pixel's horizon in its octant
      // misses everything beyond its first cell; that cell gets its own triangle test
      if (b == 1 && ob->hz && dg.z > 0.0f && dg.x != 0.0f && dg.y != 0.0f) {
        const float slope = dg.z / sqrtf(dg.x * dg.x + dg.y * dg.y);
        const float hz = __ldg(ob->hz + (size_t)octant_of(dg.x, dg.y) * ob->hz_stride + p);
        if (slope > hz + 1e-5f * fabsf(hz) + 1e-7f) {
          if ((unsigned)m.cx >= (unsigned)ob->f.Wc || (unsigned)m.cy >= (unsigned)ob->f.Hc) {
            phase = PH_RESOLVE;  // leaves the grid at once
          } else {
            test_cell(ob->f, m.cy, m.cx, m.o, m.d, m.bt, m.btri, w);
            if (m.btri < 0) phase = PH_RESOLVE;
            else m.bt = __int_as_float(0x7f800000), m.btri = -1;  // a hit there: the plain march decides
          }
        }
      }
    }
    const unsigned live = __ballot_sync(0xffffffffu, phase != PH_DONE);  // no lane finishes inside the march loop
    if (live == 0u) break;
    // ---- march while enough of the live lanes are marching; node steps every
    // iteration, leaf steps once enough marching lanes wait for one ----
    while (true) {
      if (phase == PH_MARCH && !at_leaf) {
        if (walker_node_step(m, ob->f, *lt, w, at_leaf)) phase = PH_RESOLVE;
      }
      const unsigned leaf = __ballot_sync(0xffffffffu, phase == PH_MARCH && at_leaf);
      const unsigned node = __ballot_sync(0xffffffffu, phase == PH_MARCH && !at_leaf);
      if (leaf != 0u && kLeafBatch * __popc(leaf) >= __popc(node)) {
        if (phase == PH_MARCH && at_leaf) {
          at_leaf = false;
          if (walker_leaf_step(m, ob->f, w)) phase = PH_RESOLVE;
        }
      }
      if (phase == PH_MARCH && --budget < 0) {
        overflow = 1;
        at_leaf = false;
        phase = PH_RESOLVE;
      }
      const unsigned marching = __ballot_sync(0xffffffffu, phase == PH_MARCH);
      if (marching == 0u || kMarchKeep * __popc(marching) <= __popc(live)) break;
    }
    // ---- resolve finished segments ----
    if (phase == PH_RESOLVE) {
      if (shadow) {
        const int vis = m.btri >= 0 ? 0 : 1;
        if constexpr (SHARED) {
          if (a.rec) rec_slot(b)[1 + ks] = vis;
          if (vis) add_direct(ks);
          ++ks;
          next_light();
        } else {
          if (a.rec) rec_slot(b)[1] = vis;
          if (vis) {
#pragma unroll
            for (int c = 0; c < C; ++c) acc(c) = fmaf(thr(c) * albedo_at(c, qp), cosv, acc(c));
          }
          continue_path(qp);
        }
      } else if (m.btri < 0) {
        // escaped: environment radiance along the (world) direction
        const F3 dw = {m.d.x / ob->Wf, m.d.y / ob->Wf, m.d.z};
        float e[C];
        env_lookup<C>(ob->env, ob->EH, ob->EW, dw, e);
#pragma unroll
        for (int c = 0; c < C; ++c) acc(c) = fmaf(thr(c), e[c], acc(c));
        if (a.rec) {
          int32_t *r = rec_slot(b);
          const int n = rec_width();
          for (int i = 0; i < n; ++i) r[i] = -1;
        }
        end_sample();
      } else {
        const int W = ob->f.W, H = ob->f.H;
        const float t = m.bt;
        if (b == 1) seen = true;
        const F3 q = {radd(m.o.x, rmul(t, m.d.x)), radd(m.o.y, rmul(t, m.d.y)), radd(m.o.z, rmul(t, m.d.z))};
        qp = nearest_index(q.y, H) * W + nearest_index(q.x, W);
        const F3 o2 = {q.x, q.y, radd(q.z, ob->eps)};
        if (a.rec) {
          int32_t *r = rec_slot(b);
          r[0] = qp;
          const int n = rec_width();
          for (int i = 1; i < n; ++i) r[i] = -1;
        }
        if constexpr (SHARED) {
          m.o = o2;  // origin of the shadow rays and of the next bounce
          ks = 0;
          next_light();
        } else {
          const float4 m4 = __ldg(ob->nrm + qp);
          const F3 nq = {m4.x, m4.y, m4.z};
          const F3 l = light_k(k);
          if (f3dot(nq, l) > 0.0f) {
            cosv = fmaxf(0.0f, nq.x * l.x + nq.y * l.y + nq.z * l.z);
            if (ob->shadow) {
              walker_init(m, o2, F3{rmul(l.x, ob->Wf), rmul(l.y, ob->Wf), l.z}, true, lt->zmax_margin);
              shadow = true;
              ++segs;
              phase = PH_MARCH;
            } else {
              if (a.rec) rec_slot(b)[1] = 1;
#pragma unroll
              for (int c = 0; c < C; ++c) acc(c) = fmaf(thr(c) * albedo_at(c, qp), cosv, acc(c));
              m.o = o2;
              continue_path(qp);
            }
          } else {
            m.o = o2;
            continue_path(qp);
          }
        }
      }
    }
  }
  // counters: warp sums, one atomic per warp and counter
  unsigned long long sg = segs, ov = (unsigned)overflow, nv = w.nodes, tt = w.tris, dr = w.draws;
  for (int o = 16; o > 0; o >>= 1) {
    sg += __shfl_down_sync(0xffffffffu, sg, o);
    ov += __shfl_down_sync(0xffffffffu, ov, o);
    nv += __shfl_down_sync(0xffffffffu, nv, o);
    tt += __shfl_down_sync(0xffffffffu, tt, o);
    dr += __shfl_down_sync(0xffffffffu, dr, o);
  }
  if ((threadIdx.x & 31) == 0 && a.counts) {
    if (sg) atomicAdd(a.counts + 1, sg);
    if (ov) atomicAdd(a.counts + 2, ov);
    if (nv) atomicAdd(a.counts + 3, nv);
    if (tt) atomicAdd(a.counts + 4, tt);
    if (dr) atomicAdd(a.counts + 5, dr);
  }
}

// Light-shared traces: Lbar(k, c, p) = (sum over the sample chunks of the partial
// sums, n_chunks x n_pix x KC with KC = K C, in chunk order, FP64) / spp.
__global__ void k_reduce_chunks(const float *__restrict__ part, int n_chunks, int n_pix, int kc, int C,
                                double inv_spp, float *__restrict__ out) {
  const size_t n = (size_t)n_pix * kc;
  const float *env = part + (size_t)n_chunks * n;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const size_t ip = i / kc, e = i - ip * kc;
    const size_t ie = ip * C + e % C;
    double v = 0.0;
    for (int jj = 0; jj < n_chunks; ++jj) {
      v += (double)part[(size_t)jj * n + i];
      v += (double)env[(size_t)jj * n_pix * C + ie];
    }
    out[e * n_pix + ip] = (float)(v * inv_spp);
  }
}

// The descriptor of a context's object (no output or sampling fields set).
void fill_obj_trace(const Ctx &c, ObjTrace &o) {
  o.f = c.field();
  o.nrm = c.nrm;
  o.albedo = c.albedo;
  o.env = c.env;
  o.lights = c.d_lights;
  o.out = nullptr;
  o.key = make_uint2(0u, 0u);
  o.EH = c.EH;
  o.EW = c.EW;
  o.K = c.K;
  o.spp = 0;
  o.bounces = 0;
  o.n_pix = c.H * c.W;
  o.shadow = c.opt.shadow_rays;
  o.eps = c.eps;
  o.Wf = (float)c.W;
  o.item_begin = 0;
  o.iter0 = 0;
  o.part = nullptr;
  o.n_chunks = 1;
  o.chunk = 0;
  o.hz = c.horizon;
  o.hz_stride = c.H * c.W;
  o.hole = nullptr;
}

__global__ void k_next_iter(uint32_t *iter) { *iter += 1u; }

cudaError_t launch_next_iter(Ctx &c) {
  ++c.stats.launches;
  return launch_next_iter(c.stream, c.iter_dev);
}

cudaError_t launch_next_iter(cudaStream_t s, uint32_t *iter_dev) {
  k_next_iter<<<1, 1, 0, s>>>(iter_dev);
  return cudaGetLastError();
}

// Light-shared sampling splits each pixel's samples into chunks, one work item
// each: about 2^22 items (a few tens per lane of a full persistent grid), with at
// least 16 samples per chunk.  Short items keep the lanes' loads even up to the
// last item (a launch ends when its slowest lane does, and the cost of a pixel's
// samples varies several-fold across a field), while every chunk costs a K x C
// block of partial sums (cleared, updated, reduced), which few samples would not
// pay for.  The split depends on the sizes only, never on the grid, so that the
// summation order - and every result bit - is the same for any tuning.
#ifndef IRTPS_SHARED_ITEMS_LOG2
#define IRTPS_SHARED_ITEMS_LOG2 22
#endif
#ifndef IRTPS_SHARED_MIN_CHUNK
#define IRTPS_SHARED_MIN_CHUNK 16
#endif
constexpr long long kSharedItems = 1ll << IRTPS_SHARED_ITEMS_LOG2;
constexpr int kSharedMinChunk = IRTPS_SHARED_MIN_CHUNK;

SharedSplit shared_split(int n_pix, int spp) {
  long long n = (kSharedItems + n_pix - 1) / n_pix;
  const long long most = spp / kSharedMinChunk > 1 ? spp / kSharedMinChunk : 1;
  n = n < 1 ? 1 : (n > most ? most : n);
  SharedSplit r;
  r.chunk = (int)((spp + n - 1) / n);
  r.n_chunks = (spp + r.chunk - 1) / r.chunk;
  return r;
}

size_t shared_scratch_floats(const Ctx &c, int n_pix, int spp) {
  return (size_t)shared_split(n_pix, spp).n_chunks * (c.K + 1) * c.C * n_pix;
}

cudaError_t launch_trace(Ctx &c, const int32_t *pixels, int n_pix, int spp, int bounces, uint64_t seed,
                         uint32_t iter, uint32_t stream, float *out, int32_t *rec, bool iter_from_device,
                         bool mark_holes) {
  const bool shared = c.opt.sampling == 1;
  TraceArgs a;
  fill_obj_trace(c, a.one);
  a.one.n_pix = n_pix;
  a.one.spp = spp;
  a.one.bounces = bounces;
  a.one.key = make_uint2((uint32_t)seed ^ c.obj, (uint32_t)(seed >> 32));
  a.one.out = out;
  a.one.hole = mark_holes && !shared && !pixels ? c.holes : nullptr;
  if (!early_escape_on(c, spp)) a.one.hz = nullptr;
  a.objs = nullptr;
  a.n_obj = 1;
  a.pixels = pixels;
  a.rec = rec;
  a.counts = c.dstats->counts;
  a.next_item = c.next_item;
  a.iter_dev = iter_from_device ? c.iter_dev : nullptr;
  a.iter = iter;
  a.stream = stream;
  long long n = (long long)n_pix * c.K;
  if (shared) {
    const SharedSplit sp = shared_split(n_pix, spp);
    a.one.n_chunks = sp.n_chunks;
    a.one.chunk = sp.chunk;
    const size_t lights = (size_t)a.one.n_chunks * c.K * c.C * n_pix;  // updated in place: cleared first
    if (lights + (size_t)a.one.n_chunks * c.C * n_pix > c.shared_cap) return cudaErrorInvalidValue;  // not prepared
    a.one.part = c.shared_part;
    if (cudaMemsetAsync(a.one.part, 0, sizeof(float) * lights, c.stream) != cudaSuccess) return cudaGetLastError();
    n = (long long)n_pix * a.one.n_chunks;
  }
  a.n_items = (unsigned)n;
  const int threads = kTraceThreads;
  if (cudaMemsetAsync(a.next_item, 0, sizeof(unsigned), c.stream) != cudaSuccess) return cudaGetLastError();
  ++c.stats.launches;
  // a persistent grid: as many blocks as stay resident, each lane claiming items until none remain
  long long blocks = (n + threads - 1) / threads;
  if (c.trace_blocks > 0 && blocks > c.trace_blocks) blocks = c.trace_blocks;
  const size_t smem = trace_smem_bytes(1);
  if (shared) {
    if (c.C == 1)
      k_trace<1, false, true><<<(unsigned)blocks, threads, smem, c.stream>>>(a);
    else
      k_trace<3, false, true><<<(unsigned)blocks, threads, smem, c.stream>>>(a);
    const size_t m = (size_t)c.K * c.C * n_pix;
    const unsigned rb = (unsigned)std::min<size_t>((m + 255) / 256, 8192);
    k_reduce_chunks<<<rb, 256, 0, c.stream>>>(a.one.part, a.one.n_chunks, n_pix, c.K * c.C, c.C, 1.0 / (double)spp,
                                              out);
    ++c.stats.launches;
  } else {
    if (c.C == 1)
      k_trace<1, false, false><<<(unsigned)blocks, threads, smem, c.stream>>>(a);
    else
      k_trace<3, false, false><<<(unsigned)blocks, threads, smem, c.stream>>>(a);
  }
  return cudaGetLastError();
}

// Batched trace: one persistent launch over the work items of n objects (all of
// C channels, all with the same sampling); descriptors in device memory, items in
// descriptor order.
cudaError_t launch_trace_batch(cudaStream_t s, int C, bool shared, const ObjTrace *d_objs, int n_obj,
                               unsigned n_items, unsigned long long *counts, unsigned *next_item,
                               const uint32_t *iter_dev, uint32_t iter, int grid_limit) {
  TraceArgs a;
  std::memset(&a, 0, sizeof(a));
  a.objs = d_objs;
  a.n_obj = n_obj;
  a.n_items = n_items;
  a.pixels = nullptr;
  a.rec = nullptr;
  a.counts = counts;
  a.next_item = next_item;
  a.iter_dev = iter_dev;
  a.iter = iter;
  a.stream = 0u;
  const int threads = kTraceThreads;
  if (cudaMemsetAsync(next_item, 0, sizeof(unsigned), s) != cudaSuccess) return cudaGetLastError();
  long long blocks = ((long long)n_items + threads - 1) / threads;
  if (grid_limit > 0 && blocks > grid_limit) blocks = grid_limit;
  if (blocks < 1) blocks = 1;
  const size_t smem = trace_smem_bytes(n_obj);
  if (shared) {
    if (C == 1)
      k_trace<1, true, true><<<(unsigned)blocks, threads, smem, s>>>(a);
    else
      k_trace<3, true, true><<<(unsigned)blocks, threads, smem, s>>>(a);
  } else {
    if (C == 1)
      k_trace<1, true, false><<<(unsigned)blocks, threads, smem, s>>>(a);
    else
      k_trace<3, true, false><<<(unsigned)blocks, threads, smem, s>>>(a);
  }
  return cudaGetLastError();
}

// Light-shared partial sums of a batch: ZERO clears every object's buffer before
// the trace; otherwise each object's chunks are reduced into its Lbar (as
// k_reduce_chunks).  Object o owns blocks [blk_begin, blk_begin + nblk).
template <bool ZERO>
__global__ void k_parts_b(const ReduceObj *__restrict__ objs, int n) {
  __shared__ int s_o;
  if (threadIdx.x == 0) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (objs[mid].blk_begin <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
    }
    s_o = lo;
  }
  __syncthreads();
  const ReduceObj &o = objs[s_o];
  const size_t m = (size_t)o.n_pix * o.kc;
  const size_t start = (size_t)((int)blockIdx.x - o.blk_begin) * blockDim.x + threadIdx.x;
  const size_t step = (size_t)o.nblk * blockDim.x;
  if (ZERO) {
    const size_t all = m * o.n_chunks;
    for (size_t i = start; i < all; i += step) o.part[i] = 0.0f;
  } else {
    for (size_t i = start; i < m; i += step) {
      double v = 0.0;
      const size_t ip = i / o.kc, e = i - ip * o.kc;
      const size_t ie = ip * o.C + e % o.C;
      const float *env = o.part + (size_t)o.n_chunks * m;
      for (int jj = 0; jj < o.n_chunks; ++jj) {
        v += (double)o.part[(size_t)jj * m + i];
        v += (double)env[(size_t)jj * o.n_pix * o.C + ie];
      }
      o.out[e * o.n_pix + ip] = (float)(v * o.inv_spp);
    }
  }
}

cudaError_t launch_parts_batch(cudaStream_t s, bool zero, const ReduceObj *d_objs, int n, int blocks) {
  if (zero)
    k_parts_b<true><<<blocks, 256, 0, s>>>(d_objs, n);
  else
    k_parts_b<false><<<blocks, 256, 0, s>>>(d_objs, n);
  return cudaGetLastError();
}

cudaError_t ensure_shared_scratch(Ctx &c, size_t need, bool &grown) {
  grown = false;
  if (need <= c.shared_cap) return cudaSuccess;
  cudaError_t e = cudaStreamSynchronize(c.stream);
  if (e != cudaSuccess) return e;
  if (c.graph) {  // a captured iteration holds the old buffer
    cudaGraphExecDestroy(c.graph);
    c.graph = nullptr;
  }
  if (c.shared_part) cudaFree(c.shared_part);
  c.shared_part = nullptr;
  c.shared_cap = 0;
  e = cudaMalloc((void **)&c.shared_part, sizeof(float) * need);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e;
  }
  c.shared_cap = need;
  grown = true;
  return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Stage-0 forward render of a ground-truth state (synthetic input images):
// A0(k, c, p) = rho * max(0, n . l_k) * V_k(p) + rho * Lbar_gt(k, c, p) + sigma * z,
// V_k(p) from a shadow ray at the pixel's own vertex (cast when n . l_k > 0),
// z standard normal by Box-Muller on Philox counter {p, 0, (k<<8)|(c<<4)|2, ~0}.
// ---------------------------------------------------------------------------
template <int C>
__global__ void k_render(const ObjTrace a, const float *__restrict__ lbar, float sigma, float *__restrict__ out) {
  __shared__ LevelTable lt;
  load_levels(a.f, &lt);
  const int P = a.f.H * a.f.W;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= P * a.K) return;
  const int k = idx / P, p = idx - k * P;
  const int pi = p / a.f.W, pj = p - pi * a.f.W;
  const float4 n4 = a.nrm[p];
  const F3 n = {n4.x, n4.y, n4.z};
  const F3 l = {a.lights[3 * k], a.lights[3 * k + 1], a.lights[3 * k + 2]};
  float cosv = 0.0f;
  if (f3dot(n, l) > 0.0f) {
    int vis = 1;
    if (a.shadow) {
      const F3 o = {(float)pj, (float)pi, radd(a.f.depth[p], a.eps)};
      const F3 lg = {rmul(l.x, a.Wf), rmul(l.y, a.Wf), l.z};
      float t;
      int tri;
      int budget = 8 * (a.f.Wc + a.f.Hc + 8) * (a.f.levels + 1);
      Work w;
      vis = march(a.f, lt, o, lg, true, t, tri, budget, w) ? 0 : 1;
    }
    if (vis) cosv = fmaxf(0.0f, n.x * l.x + n.y * l.y + n.z * l.z);
  }
#pragma unroll
  for (int c = 0; c < C; ++c) {
    const uint4 x = philox4x32_10(make_uint4((uint32_t)p, 0u, ((uint32_t)k << 8) | ((uint32_t)c << 4) | 2u,
                                             0xFFFFFFFFu), a.key);
    const float u1 = (float)((x.x >> 8) + 1u) * 5.9604644775390625e-08f;
    const float u2 = (float)(x.y >> 8) * 5.9604644775390625e-08f;
    const float z = sqrtf(-2.0f * logf(u1)) * cosf(6.28318530717958647692f * u2);
    const float rho = a.albedo[(size_t)c * P + p];
    const size_t o = ((size_t)k * C + c) * P + p;
    out[o] = rho * cosv + rho * lbar[o] + sigma * z;
  }
}

// Resident blocks of the trace kernel for C channels (the persistent grid size);
// n_obj > 0: the batched kernel over n_obj objects; shared: the light-shared kernel,
// else the per-light one.
template <typename F>
static int grid_of(F kernel, size_t smem, int sms) {
  int per = 0;
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, kTraceThreads, smem) != cudaSuccess) return 0;
  return per * sms;
}

int trace_grid_limit(int C, int n_obj, bool shared) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  const size_t smem = trace_smem_bytes(n_obj > 0 ? n_obj : 1);
  if (shared) {
    if (n_obj > 0)
      return C == 1 ? grid_of(k_trace<1, true, true>, smem, sms) : grid_of(k_trace<3, true, true>, smem, sms);
    return C == 1 ? grid_of(k_trace<1, false, true>, smem, sms) : grid_of(k_trace<3, false, true>, smem, sms);
  }
  if (n_obj > 0)
    return C == 1 ? grid_of(k_trace<1, true, false>, smem, sms) : grid_of(k_trace<3, true, false>, smem, sms);
  return C == 1 ? grid_of(k_trace<1, false, false>, smem, sms) : grid_of(k_trace<3, false, false>, smem, sms);
}

cudaError_t launch_render(Ctx &c, uint64_t seed, float sigma, const float *lbar, float *out) {
  ObjTrace a;
  fill_obj_trace(c, a);
  a.key = make_uint2((uint32_t)seed ^ c.obj, (uint32_t)(seed >> 32));
  const long long n = (long long)c.H * c.W * c.K;
  const int threads = 128;
  const unsigned blocks = (unsigned)((n + threads - 1) / threads);
  ++c.stats.launches;
  if (c.C == 1)
    k_render<1><<<blocks, threads, 0, c.stream>>>(a, lbar, sigma, out);
  else
    k_render<3><<<blocks, threads, 0, c.stream>>>(a, lbar, sigma, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Geometry probes (parity tests): sampled directions and ray / mesh hits.
// ---------------------------------------------------------------------------
__global__ void k_probe_dirs(int n, const float *__restrict__ normals, const uint32_t *__restrict__ x0,
                             const uint32_t *__restrict__ x1, float *__restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const F3 nn = {normals[3 * i], normals[3 * i + 1], normals[3 * i + 2]};
  const F3 d = cosine_dir(nn, x0[i], x1[i]);
  out[3 * i] = d.x;
  out[3 * i + 1] = d.y;
  out[3 * i + 2] = d.z;
}

__global__ void k_probe_rays(const Field f, int n, const float *__restrict__ rays, float *__restrict__ t_out,
                             int32_t *__restrict__ tri_out, int *__restrict__ overflow) {
  __shared__ LevelTable lt;
  load_levels(f, &lt);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const F3 o = {rays[6 * i], rays[6 * i + 1], rays[6 * i + 2]};
  const F3 d = {rays[6 * i + 3], rays[6 * i + 4], rays[6 * i + 5]};
  float t;
  int tri;
  int budget = 8 * (f.Wc + f.Hc + 8) * (f.levels + 1);
  Work w;
  const bool hit = march(f, lt, o, d, false, t, tri, budget, w);
  t_out[i] = hit ? t : __int_as_float(0x7fc00000);
  tri_out[i] = hit ? tri : -1;
  if (budget < 0) atomicAdd(overflow, 1);
}

cudaError_t launch_probe_dirs(cudaStream_t s, int n, const float *normals, const uint32_t *x0, const uint32_t *x1,
                              float *out) {
  k_probe_dirs<<<(n + 127) / 128, 128, 0, s>>>(n, normals, x0, x1, out);
  return cudaGetLastError();
}

cudaError_t launch_probe_rays(Ctx &c, int n, const float *rays, float *t_out, int32_t *tri_out, int *overflow) {
  k_probe_rays<<<(n + 127) / 128, 128, 0, c.stream>>>(c.field(), n, rays, t_out, tri_out, overflow);
  return cudaGetLastError();
}

}  // namespace irtps
