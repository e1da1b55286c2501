// Integration of the normals into the surface (Sec. IV, stage 1: "integrating
// over the obtained normals a 3D surface H_t is obtained") and the convergence
// measure D_H = H_{t+1} - H_t of the loop.
//
// The surface minimises sum over grid edges (H_b - H_a - g_e)^2 with trapezoidal
// edge targets g = h (p_a + p_b) / 2 (rows) and h (q_a + q_b) / 2 (columns), slopes
// p = -n_x / max(n_z, nz_min), q = -n_y / max(n_z, nz_min); mean(H) = 0.  Its normal
// equations L H = D^T g use the Neumann 5-point graph Laplacian L.
//
// Solver: Jacobi-preconditioned CG (M = diag(degree)) in FP32 for the search
// direction, residual and preconditioned residual, with the iterate x and the
// right-hand side b in FP64; every cg_check_every iterations the residual is
// replaced by the FP64 true residual b - A x (iterative refinement) and tested
// against cg_tol.  Reductions are two-stage and deterministic: each block writes
// one partial, and every consumer block sums all partials in the same order.
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "irtps_internal.h"

namespace irtps {

enum Slot { S_BB = 0, S_PAP = 1, S_RZ0 = 2, S_RZ1 = 3, S_RR = 4, S_SUMX = 5, S_DMAX = 6, S_DSQ = 7, S_HMAX = 8,
            S_HMIN = 9, S_RZREF = 10 };
static_assert(S_RZREF < kPartSlots, "partial slots");

#ifndef IRTPS_CG_THREADS
#define IRTPS_CG_THREADS 256
#endif
#ifndef IRTPS_CG_BLOCKS_PER_SM
#define IRTPS_CG_BLOCKS_PER_SM 2
#endif
// batched solves: smaller teams (a share of the grid per object) gain from more co-resident blocks
#ifndef IRTPS_CG_BATCH_BLOCKS_PER_SM
#define IRTPS_CG_BATCH_BLOCKS_PER_SM 4
#endif
#ifndef IRTPS_CG_BATCH_MINB
#define IRTPS_CG_BATCH_MINB 4
#endif
constexpr int kThreads = IRTPS_CG_THREADS;
#ifndef IRTPS_BARRIER_SLEEP_NS
#define IRTPS_BARRIER_SLEEP_NS 64
#endif
constexpr unsigned kBarrierSleepNs = IRTPS_BARRIER_SLEEP_NS;  // back-off between barrier polls

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}

// Block-wide sum (or max); the result is valid in thread 0.
template <bool MAX>
__device__ __forceinline__ double block_reduce(double v, double *sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  v = MAX ? warp_max(v) : warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  if (wid == 0) {
    const double ident = MAX ? -INFINITY : 0.0;
    v = lane < (int)(blockDim.x >> 5) ? sh[lane] : ident;
    v = MAX ? warp_max(v) : warp_sum(v);
  }
  return v;
}

// Sum of n partials, identical in every block (fixed order); all threads get it.
__device__ __forceinline__ double total(const double *part, int n, double *sh) {
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = 0.0;
    for (int i = threadIdx.x; i < n; i += 32) v += part[i];
    v = warp_sum(v);
    if (threadIdx.x == 0) sh[32] = v;
  }
  __syncthreads();
  return sh[32];
}

template <typename T>
__device__ __forceinline__ T lap_at(const T *v, int i, int j, int H, int W) {
  const size_t p = (size_t)i * W + j;
  const T c = v[p];
  T s = 0;
  int deg = 0;
  if (j > 0) { s += v[p - 1]; ++deg; }
  if (j < W - 1) { s += v[p + 1]; ++deg; }
  if (i > 0) { s += v[p - W]; ++deg; }
  if (i < H - 1) { s += v[p + W]; ++deg; }
  return (T)deg * c - s;
}

__device__ __forceinline__ int degree(int i, int j, int H, int W) {
  return (j > 0) + (j < W - 1) + (i > 0) + (i < H - 1);
}

// The weighted graph Laplacian (IRLS solves): sum over the edges of p of
// w_e (v_p - v_neighbour); wh[p] weighs edge p - p+1, wv[p] edge p - p+W.
template <typename T>
__device__ __forceinline__ T lap_weighted(const T *v, const float *wh, const float *wv, int i, int j, int H, int W) {
  const size_t p = (size_t)i * W + j;
  const T c = v[p];
  T s = 0, d = 0;
  if (j > 0) { const T w = (T)wh[p - 1]; s = fma(w, v[p - 1], s); d += w; }
  if (j < W - 1) { const T w = (T)wh[p]; s = fma(w, v[p + 1], s); d += w; }
  if (i > 0) { const T w = (T)wv[p - W]; s = fma(w, v[p - W], s); d += w; }
  if (i < H - 1) { const T w = (T)wv[p]; s = fma(w, v[p + W], s); d += w; }
  return d * c - s;
}

__device__ __forceinline__ float weighted_degree(const float *wh, const float *wv, int p, int i, int j, int H, int W) {
  float d = 0.0f;
  if (j > 0) d += wh[p - 1];
  if (j < W - 1) d += wh[p];
  if (i > 0) d += wv[p - W];
  if (i < H - 1) d += wv[p];
  return d;
}

// The blocks that work on one solve: all of a plain launch, or the range of a
// batched launch that belongs to one object (bid = block index within it).
struct Team {
  int bid, nblk;
};
__device__ __forceinline__ Team whole_grid() { return Team{(int)blockIdx.x, (int)gridDim.x}; }

struct CG {
  int H, W, P;
  double h;
  float nz_min;
  const float4 *nrm;
  float *depth;
  double *x, *b;
  float *r, *z, *p, *ap;  // p: two buffers of P; ap: A p, then the FP32 correction
  double *part;
  int stride, nblk;
  const float *wh, *wv;   // edge weights of the weighted (IRLS) solves, level 0 of the multigrid pool
};

__device__ __forceinline__ void slopes(const float4 *nrm, size_t p, float nz_min, double &sp, double &sq) {
  const float4 n = nrm[p];
  const double nz = fmax((double)n.z, (double)nz_min);
  sp = -(double)n.x / nz;
  sq = -(double)n.y / nz;
}

// b = D^T g (FP64; weighted: D^T W g) and |b|^2 partials.
template <bool WEIGHTED>
__device__ __forceinline__ void rhs_body(const CG &g, Team t) {
  __shared__ double sh[33];
  double bb = 0.0;
  auto wt = [&](const float *w, int e, double x) -> double { return WEIGHTED ? (double)w[e] * x : x; };
  for (int p = t.bid * blockDim.x + threadIdx.x; p < g.P; p += t.nblk * blockDim.x) {
    const int i = p / g.W, j = p - i * g.W;
    double pc, qc, pn, qn;
    slopes(g.nrm, p, g.nz_min, pc, qc);
    double v = 0.0;
    if (j > 0) { slopes(g.nrm, p - 1, g.nz_min, pn, qn); v += wt(g.wh, p - 1, g.h * (pn + pc) * 0.5); }
    if (j < g.W - 1) { slopes(g.nrm, p + 1, g.nz_min, pn, qn); v -= wt(g.wh, p, g.h * (pc + pn) * 0.5); }
    if (i > 0) { slopes(g.nrm, p - g.W, g.nz_min, pn, qn); v += wt(g.wv, p - g.W, g.h * (qn + qc) * 0.5); }
    if (i < g.H - 1) { slopes(g.nrm, p + g.W, g.nz_min, pn, qn); v -= wt(g.wv, p, g.h * (qc + qn) * 0.5); }
    g.b[p] = v;
    bb += v * v;
  }
  bb = block_reduce<false>(bb, sh);
  if (threadIdx.x == 0) g.part[S_BB * g.stride + t.bid] = bb;
}

__device__ __forceinline__ void load_x_body(const CG &g, Team t) {
  for (int p = t.bid * blockDim.x + threadIdx.x; p < g.P; p += t.nblk * blockDim.x) g.x[p] = (double)g.depth[p];
}

// True residual r = b - A x in FP64 (stored FP32), z = r / deg, partials of r.z and |r|^2 (FP64).
template <bool WEIGHTED>
__device__ __forceinline__ void residual_body(const CG &g, int rz_slot, Team t) {
  __shared__ double sh[33];
  double rz = 0.0, rr = 0.0;
  for (int p = t.bid * blockDim.x + threadIdx.x; p < g.P; p += t.nblk * blockDim.x) {
    const int i = p / g.W, j = p - i * g.W;
    const double ax = WEIGHTED ? lap_weighted<double>(g.x, g.wh, g.wv, i, j, g.H, g.W)
                               : lap_at<double>(g.x, i, j, g.H, g.W);
    const double res = g.b[p] - ax;
    const float rf = (float)res;
    const float zf = rf / (WEIGHTED ? weighted_degree(g.wh, g.wv, p, i, j, g.H, g.W) : (float)degree(i, j, g.H, g.W));
    g.r[p] = rf;
    g.z[p] = zf;
    rz += (double)rf * (double)zf;
    rr += res * res;
  }
  rz = block_reduce<false>(rz, sh);
  if (threadIdx.x == 0) {
    g.part[rz_slot * g.stride + t.bid] = rz;
    g.part[S_RZREF * g.stride + t.bid] = rz;
  }
  rr = block_reduce<false>(rr, sh);
  if (threadIdx.x == 0) g.part[S_RR * g.stride + t.bid] = rr;
}

// Barrier of the nblk blocks of a team in a cooperative launch (all blocks
// co-resident).  Thread 0 of each block arrives on a counter; the last one resets it and advances the
// generation word the others poll.  Every poll loop is bounded: on running out it
// raises the error flag, and all blocks leave the solve at the next check.
__device__ __forceinline__ void grid_barrier(unsigned *count, volatile unsigned *gen, int *err, int nblk) {
  __syncthreads();
  if (threadIdx.x == 0 && !*(volatile int *)err) {  // after a failure every barrier is a no-op
    const unsigned g0 = *gen;
    __threadfence();
    if (atomicAdd(count, 1u) == (unsigned)nblk - 1u) {
      *count = 0u;
      __threadfence();
      atomicAdd((unsigned *)gen, 1u);
    } else {
      unsigned long long polls = 0;
      while (*gen == g0) {
        if (++polls > (1ull << 24)) {
          atomicExch(err, 1);
          break;
        }
        if (kBarrierSleepNs > 0) __nanosleep(kBarrierSleepNs);
      }
    }
    __threadfence();
  }
  __syncthreads();
}

// Block-wide FP32 sum; the result is valid in thread 0.
__device__ __forceinline__ float block_sum_f(float v, float *shf) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) shf[wid] = v;
  __syncthreads();
  if (wid == 0) {
    v = lane < (int)(blockDim.x >> 5) ? shf[lane] : 0.0f;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  }
  return v;
}

// Pixel coordinates of a grid-stride loop, advanced without divisions.
struct Stride {
  int p, i, j, dp, di, dj;
  __device__ __forceinline__ Stride(int W, Team t) {
    p = t.bid * blockDim.x + threadIdx.x;
    i = p / W;
    j = p - i * W;
    dp = t.nblk * blockDim.x;
    di = dp / W;
    dj = dp - di * W;
  }
  __device__ __forceinline__ void next(int W) {
    p += dp;
    i += di;
    j += dj;
    if (j >= W) {
      j -= W;
      ++i;
    }
  }
};

__device__ __forceinline__ float inv_degree(int i, int j, int H, int W) {
  const int d = (j > 0) + (j < W - 1) + (i > 0) + (i < H - 1);
  return d == 4 ? 0.25f : (d == 3 ? (1.0f / 3.0f) : (d == 2 ? 0.5f : 1.0f));
}

// ---------------------------------------------------------------------------
// Multigrid V-cycle preconditioner (option precond = 1).  Levels coarsen the
// pixel grid by 2x2 aggregation; the operator of each coarse level is the
// Galerkin product R A P of the finer one with piecewise-constant P and R = P^T,
// which is again a weighted 5-point graph Laplacian: its edge weight between two
// aggregates is the sum of the fine weights crossing between them (weights are
// built once on the host).  Smoother: two weighted-Jacobi sweeps before and after
// the coarse correction (symmetric, so the V-cycle is an admissible CG
// preconditioner).  The fine levels are swept by the whole grid between grid
// barriers; levels of at most kMgBlockPoints points are handled by block 0
// alone, the coarsest (<= 16 points) by repeated sweeps and a mean projection.
// ---------------------------------------------------------------------------
constexpr int kMgMaxLevels = 16;
constexpr int kMgBlockPoints = 4096;
// Scale of the coarse-grid correction.  Piecewise-constant aggregation
// under-corrects the smooth error components; scaling the correction by 1.5
// (a scalar, so the V-cycle stays symmetric) cut the warm 512x512 solve from 90
// to 30 iterations.  Above about 1.7 the preconditioner lost definiteness on some
// grids.  The weighted (IRLS) solves keep the plain correction.
#ifndef IRTPS_MG_CSCALE
#define IRTPS_MG_CSCALE 1.5f
#endif

struct MG {
  int levels, grid_levels;
  int H[kMgMaxLevels], W[kMgMaxLevels], off[kMgMaxLevels];
  float *x0, *x1, *b;  // pooled per level at off[l]
  const float *wh;     // weight of edge (i, j)-(i, j+1), pooled, H*W slots per level
  const float *wv;     // weight of edge (i, j)-(i+1, j)
  float omega, cscale;
};

__device__ __forceinline__ float mg_diag(const MG &m, int l, int i, int j) {
  const int H = m.H[l], W = m.W[l], o = m.off[l];
  const int p = i * W + j;
  float d = 0.0f;
  if (j > 0) d += m.wh[o + p - 1];
  if (j < W - 1) d += m.wh[o + p];
  if (i > 0) d += m.wv[o + p - W];
  if (i < H - 1) d += m.wv[o + p];
  return d;
}

__device__ __forceinline__ float mg_ax(const MG &m, int l, const float *x, int i, int j, float xc, float &d) {
  const int H = m.H[l], W = m.W[l], o = m.off[l];
  const int p = i * W + j;
  float s = 0.0f;
  d = 0.0f;
  if (j > 0) { const float w = m.wh[o + p - 1]; s = fmaf(w, x[o + p - 1], s); d += w; }
  if (j < W - 1) { const float w = m.wh[o + p]; s = fmaf(w, x[o + p + 1], s); d += w; }
  if (i > 0) { const float w = m.wv[o + p - W]; s = fmaf(w, x[o + p - W], s); d += w; }
  if (i < H - 1) { const float w = m.wv[o + p]; s = fmaf(w, x[o + p + W], s); d += w; }
  return fmaf(d, xc, -s);
}

// The same with the coarse correction of level l+1 added to x on the fly.
__device__ __forceinline__ float mg_xc(const MG &m, int l, const float *x, int i, int j) {
  const int Wc = m.W[l + 1];
  return x[m.off[l] + i * m.W[l] + j] + m.cscale * m.x1[m.off[l + 1] + (i >> 1) * Wc + (j >> 1)];
}

__device__ __forceinline__ float mg_ax_corr(const MG &m, int l, const float *x, int i, int j, float &d, float &xcen) {
  const int H = m.H[l], W = m.W[l], o = m.off[l];
  const int p = i * W + j;
  float s = 0.0f;
  d = 0.0f;
  if (j > 0) { const float w = m.wh[o + p - 1]; s = fmaf(w, mg_xc(m, l, x, i, j - 1), s); d += w; }
  if (j < W - 1) { const float w = m.wh[o + p]; s = fmaf(w, mg_xc(m, l, x, i, j + 1), s); d += w; }
  if (i > 0) { const float w = m.wv[o + p - W]; s = fmaf(w, mg_xc(m, l, x, i - 1, j), s); d += w; }
  if (i < H - 1) { const float w = m.wv[o + p]; s = fmaf(w, mg_xc(m, l, x, i + 1, j), s); d += w; }
  xcen = mg_xc(m, l, x, i, j);
  return fmaf(d, xcen, -s);
}

// Iterate the points of level l: the whole grid (grid levels) or block 0 alone.
#define MG_FOR(l, pt)                                                                              \
  for (int pt = (l < m.grid_levels ? t.bid * (int)blockDim.x : 0) + threadIdx.x,                 \
           pt##_n = m.H[l] * m.W[l], pt##_s = (l < m.grid_levels ? t.nblk : 1) * blockDim.x;   \
       pt < pt##_n; pt += pt##_s)

// Synchronise after a step on level l: a grid barrier on grid levels, the block on block levels.
__device__ __forceinline__ void mg_sync(const MG &m, int l, CGCtl *ctl, Team t) {
  if (l < m.grid_levels) grid_barrier(&ctl->count, &ctl->gen, &ctl->err, t.nblk);
  else __syncthreads();
}

// z = V(r): level-0 right-hand side r (length P), result in x1 of level 0.
// Called by all blocks; on return all of z is visible to all blocks.
__device__ void mg_vcycle(const MG &m, const float *r, CGCtl *ctl, Team t) {
  const float om = m.omega;
  const int L = m.levels;
  // ---- down ----
  for (int l = 0; l < L - 1; ++l) {
    const bool active = l < m.grid_levels || t.bid == 0;
    const float *b = l == 0 ? r : m.b + m.off[l];
    const int W = m.W[l], o = m.off[l];
    if (active) {
      MG_FOR(l, pt) {  // first sweep from zero: x = omega b / d
        const int i = pt / W, j = pt - i * W;
        m.x0[o + pt] = om * b[pt] / mg_diag(m, l, i, j);
      }
    }
    if (l < m.grid_levels) mg_sync(m, l, ctl, t); else if (active) __syncthreads();
    if (active) {
      MG_FOR(l, pt) {  // second sweep
        const int i = pt / W, j = pt - i * W;
        float d;
        const float ax = mg_ax(m, l, m.x0, i, j, m.x0[o + pt], d);
        m.x1[o + pt] = m.x0[o + pt] + om * (b[pt] - ax) / d;
      }
    }
    if (l < m.grid_levels) mg_sync(m, l, ctl, t); else if (active) __syncthreads();
    // residual, summed over each 2x2 aggregate into the next level's right-hand side
    const int lc = l + 1;
    const bool active_c = lc < m.grid_levels || t.bid == 0;
    if (active && active_c) {
      const int Wc = m.W[lc], Hf = m.H[l];
      MG_FOR(lc, pt) {
        const int I = pt / Wc, J = pt - I * Wc;
        float sum = 0.0f;
        for (int di = 0; di < 2; ++di) {
          const int i = 2 * I + di;
          if (i >= Hf) break;
          for (int dj = 0; dj < 2; ++dj) {
            const int j = 2 * J + dj;
            if (j >= W) break;
            float d;
            const float ax = mg_ax(m, l, m.x1, i, j, m.x1[o + i * W + j], d);
            sum += b[i * W + j] - ax;
          }
        }
        m.b[m.off[lc] + pt] = sum;
      }
    }
    if (l < m.grid_levels) mg_sync(m, l, ctl, t); else if (active) __syncthreads();
  }
  // ---- coarsest: sweeps and a mean projection (block 0) ----
  if (t.bid == 0) {
    const int l = L - 1, W = m.W[l], o = m.off[l], n = m.H[l] * m.W[l];
    const float *b = L == 1 ? r : m.b + o;
    for (int q = threadIdx.x; q < n; q += blockDim.x) m.x1[o + q] = 0.0f;
    __syncthreads();
    for (int sweep = 0; sweep < 64; ++sweep) {
      float v = 0.0f;
      if (threadIdx.x < n) {
        const int i = threadIdx.x / W, j = threadIdx.x - i * W;
        float d;
        const float ax = mg_ax(m, l, m.x1, i, j, m.x1[o + threadIdx.x], d);
        v = d > 0.0f ? m.x1[o + threadIdx.x] + om * (b[threadIdx.x] - ax) / d : 0.0f;
      }
      __syncthreads();
      if (threadIdx.x < n) m.x1[o + threadIdx.x] = v;
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      float mean = 0.0f;
      for (int q = 0; q < n; ++q) mean += m.x1[o + q];
      mean /= (float)n;
      for (int q = 0; q < n; ++q) m.x1[o + q] -= mean;
    }
    __syncthreads();
  }
  // ---- up ----
  for (int l = L - 2; l >= 0; --l) {
    const bool active = l < m.grid_levels || t.bid == 0;
    const float *b = l == 0 ? r : m.b + m.off[l];
    const int W = m.W[l], o = m.off[l];
    // the coarse level's result must be visible before it is interpolated
    if (l + 1 == m.grid_levels || l + 1 == L - 1) {
      if (l < m.grid_levels) grid_barrier(&ctl->count, &ctl->gen, &ctl->err, t.nblk);
      else if (active) __syncthreads();
    }
    if (active) {
      MG_FOR(l, pt) {  // first sweep on x + P x_coarse
        const int i = pt / W, j = pt - i * W;
        float d, xcen;
        const float ax = mg_ax_corr(m, l, m.x1, i, j, d, xcen);
        m.x0[o + pt] = xcen + om * (b[pt] - ax) / d;
      }
    }
    if (l < m.grid_levels) mg_sync(m, l, ctl, t); else if (active) __syncthreads();
    if (active) {
      MG_FOR(l, pt) {  // second sweep
        const int i = pt / W, j = pt - i * W;
        float d;
        const float ax = mg_ax(m, l, m.x0, i, j, m.x0[o + pt], d);
        m.x1[o + pt] = m.x0[o + pt] + om * (b[pt] - ax) / d;
      }
    }
    if (l < m.grid_levels) mg_sync(m, l, ctl, t); else if (active) __syncthreads();
  }
  if (m.grid_levels == 0) grid_barrier(&ctl->count, &ctl->gen, &ctl->err, t.nblk);  // z was written by block 0 alone
}
#undef MG_FOR

// The whole PCG loop in one cooperative launch (PRE 0: Jacobi, M = diag(degree);
// PRE 1: the multigrid V-cycle above).  The iterate is x = x64 + e: the FP64 part
// changes only at a refresh, the FP32 correction e collects alpha * p in between.
// Per iteration:
//  A: beta = rz_{it-1}/rz_{it-2}; p_it = z + beta p_{it-1} (also at the 4
//     neighbours, recomputed locally); Ap; partial p.Ap       -- barrier --
//  B: alpha = rz_{it-1}/p.Ap; e += alpha p; r -= alpha Ap; z = M^-1 r;
//     partial r.z                                             -- barrier --
// Every `check` iterations, or as soon as r.z has fallen below 1e-10 of its
// value at the last refresh (the FP32 recursion has converged and further steps
// would follow rounding noise: the direction is then frozen to 0), x64 += e,
// e = 0, and the residual is recomputed in FP64 (r = b - A x64) and tested
// against tol (iterative refinement).  Dot products are FP32 within a block and
// FP64 across blocks; every block sums the same partials in the same order and
// so takes the same decisions.
template <int PRE, bool WEIGHTED>
__device__ __forceinline__ void cg_loop_body(const CG &g, CGCtl *ctl, CGAcc *acc, double tol, int max_iter, int check,
                                             const MG &mg, Team t) {
  __shared__ double sh[33];
  __shared__ float shf[33];
  __shared__ float s_ab[2];
  __shared__ int s_frozen;
  double best = INFINITY;
  int stall = 0, it = 0;
  double rel = ctl->rel;
  const double bnorm = ctl->bnorm;
  if (!(bnorm > 0.0) || !isfinite(bnorm)) rel = 0.0;  // flat (or broken) right-hand side: nothing to solve
  float *e = g.ap + g.P;  // correction accumulator (second half of the Ap buffer)
  float *z = PRE == 1 ? mg.x1 : g.z;  // preconditioned residual (level 0 of the hierarchy for PRE 1)
  for (Stride q(g.W, t); q.p < g.P; q.next(g.W)) e[q.p] = 0.0f;
  // z = M^-1 r and the partial sums of r.z into `slot` (and the refresh reference)
  auto precondition = [&](int slot, bool refresh) {
    if (PRE == 1) {
      grid_barrier(&ctl->count, &ctl->gen, &ctl->err, t.nblk);  // r complete
      mg_vcycle(mg, g.r, ctl, t);
    }
    float rz = 0.0f;
    for (Stride q(g.W, t); q.p < g.P; q.next(g.W)) {
      const float rf = g.r[q.p];
      float zf;
      if (PRE == 1) {
        zf = z[q.p];
      } else {
        zf = WEIGHTED ? rf / weighted_degree(g.wh, g.wv, q.p, q.i, q.j, g.H, g.W)
                      : rf * inv_degree(q.i, q.j, g.H, g.W);
        z[q.p] = zf;
      }
      rz = fmaf(rf, zf, rz);
    }
    rz = block_sum_f(rz, shf);
    if (threadIdx.x == 0) {
      g.part[slot * g.stride + t.bid] = (double)rz;
      if (refresh) g.part[S_RZREF * g.stride + t.bid] = (double)rz;
    }
  };
  if (PRE == 1 && rel > tol) {  // the residual kernel left r; z and r.z come from the V-cycle
    precondition(S_RZ0, true);
    grid_barrier(&ctl->count, &ctl->gen, &ctl->err, t.nblk);
  }
  while (rel > tol && it < max_iter && !*(volatile int *)&ctl->err) {
    ++it;
    // ---- A ----
    const double num = total(g.part + (S_RZ0 + ((it - 1) & 1)) * g.stride, g.nblk, sh);
    const double ref = total(g.part + S_RZREF * g.stride, g.nblk, sh);
    const double den = it > 1 ? total(g.part + (S_RZ0 + (it & 1)) * g.stride, g.nblk, sh) : 0.0;
    if (threadIdx.x == 0) {
      const bool frozen = !(num > 1e-10 * ref);
      s_frozen = frozen;
      s_ab[1] = (it > 1 && !frozen && den > 0.0) ? (float)(num / den) : 0.0f;
    }
    __syncthreads();
    const bool frozen = s_frozen;
    const float beta = s_ab[1];
    const bool first = it == 1;
    const float *pold = g.p + (size_t)((it - 1) & 1) * g.P;
    float *pnew = g.p + (size_t)(it & 1) * g.P;
    auto dir = [&](int r) { return frozen ? 0.0f : (first ? z[r] : fmaf(beta, pold[r], z[r])); };
    float pap = 0.0f;
    for (Stride q(g.W, t); q.p < g.P; q.next(g.W)) {
      const int p = q.p;
      const float pc = dir(p);
      float s = 0.0f, deg = 0.0f;
      if (WEIGHTED) {
        if (q.j > 0) { const float w = g.wh[p - 1]; s = fmaf(w, dir(p - 1), s); deg += w; }
        if (q.j < g.W - 1) { const float w = g.wh[p]; s = fmaf(w, dir(p + 1), s); deg += w; }
        if (q.i > 0) { const float w = g.wv[p - g.W]; s = fmaf(w, dir(p - g.W), s); deg += w; }
        if (q.i < g.H - 1) { const float w = g.wv[p]; s = fmaf(w, dir(p + g.W), s); deg += w; }
      } else {
        if (q.j > 0) { s += dir(p - 1); deg += 1.0f; }
        if (q.j < g.W - 1) { s += dir(p + 1); deg += 1.0f; }
        if (q.i > 0) { s += dir(p - g.W); deg += 1.0f; }
        if (q.i < g.H - 1) { s += dir(p + g.W); deg += 1.0f; }
      }
      const float apv = fmaf(deg, pc, -s);
      pnew[p] = pc;
      g.ap[p] = apv;
      pap = fmaf(pc, apv, pap);
    }
    pap = block_sum_f(pap, shf);
    if (threadIdx.x == 0) g.part[S_PAP * g.stride + t.bid] = (double)pap;
    grid_barrier(&ctl->count, &ctl->gen, &ctl->err, t.nblk);
    if (*(volatile int *)&ctl->err) break;
    // ---- B ----
    const double dpap = total(g.part + S_PAP * g.stride, g.nblk, sh);
    if (threadIdx.x == 0) s_ab[0] = (dpap > 0.0 && isfinite(dpap)) ? (float)(num / dpap) : 0.0f;
    __syncthreads();
    const float af = s_ab[0];
    for (Stride q(g.W, t); q.p < g.P; q.next(g.W)) {
      const int p = q.p;
      e[p] = fmaf(af, pnew[p], e[p]);
      g.r[p] = fmaf(-af, g.ap[p], g.r[p]);
    }
    precondition(S_RZ0 + (it & 1), false);
    grid_barrier(&ctl->count, &ctl->gen, &ctl->err, t.nblk);
    if (*(volatile int *)&ctl->err) break;
    // ---- refresh from FP64 ----
    if (it % check == 0 || frozen) {
      for (Stride q(g.W, t); q.p < g.P; q.next(g.W)) {
        g.x[q.p] += (double)e[q.p];
        e[q.p] = 0.0f;
      }
      grid_barrier(&ctl->count, &ctl->gen, &ctl->err, t.nblk);
      if (*(volatile int *)&ctl->err) break;
      double rr = 0.0;
      for (Stride q(g.W, t); q.p < g.P; q.next(g.W)) {
        const double ax = WEIGHTED ? lap_weighted<double>(g.x, g.wh, g.wv, q.i, q.j, g.H, g.W)
                                   : lap_at<double>(g.x, q.i, q.j, g.H, g.W);
        const double res = g.b[q.p] - ax;
        g.r[q.p] = (float)res;
        rr += res * res;
      }
      rr = block_reduce<false>(rr, sh);
      if (threadIdx.x == 0) g.part[S_RR * g.stride + t.bid] = rr;
      precondition(S_RZ0 + (it & 1), true);
      grid_barrier(&ctl->count, &ctl->gen, &ctl->err, t.nblk);
      if (*(volatile int *)&ctl->err) break;
      rel = sqrt(total(g.part + S_RR * g.stride, g.nblk, sh)) / bnorm;
      if (!isfinite(rel)) break;
      if (rel < 0.95 * best) {
        best = rel;
        stall = it;
      } else if (it - stall >= 1000) {
        break;  // no 5% gain in 1000 iterations: the FP64 residual is at its rounding floor
      }
    }
  }
  // fold in a correction collected since the last refresh (none when the loop ended on a refresh)
  for (Stride q(g.W, t); q.p < g.P; q.next(g.W)) g.x[q.p] += (double)e[q.p];
  if (t.bid == 0 && threadIdx.x == 0) {
    ctl->iters = it;
    ctl->rel = rel;
    if (acc) {
      acc->iters += it;
      acc->last_iters = it;
      acc->rel_last = rel;
      if (*(volatile int *)&ctl->err) acc->err = 1;
      if (!isfinite(bnorm) || !isfinite(rel) || rel > tol) acc->bad = 1;
    }
  }
}

template <int PRE, bool WEIGHTED = false>
__global__ void __launch_bounds__(kThreads) k_cg_loop(const CG g, CGCtl *ctl, CGAcc *acc, double tol, int max_iter,
                                                      int check, const MG mg) {
  cg_loop_body<PRE, WEIGHTED>(g, ctl, acc, tol, max_iter, check, mg, whole_grid());
}

// Start of a solve: |b| and the warm start's relative residual from the partials,
// barrier state reset (one warp).
__device__ __forceinline__ void cg_start_body(const CG &g, CGCtl *ctl) {
  double bb = 0.0, rr = 0.0;
  for (int i = threadIdx.x; i < g.nblk; i += 32) {
    bb += g.part[S_BB * g.stride + i];
    rr += g.part[S_RR * g.stride + i];
  }
  bb = warp_sum(bb);
  rr = warp_sum(rr);
  if (threadIdx.x == 0) {
    ctl->count = 0u;
    ctl->gen = 0u;
    ctl->err = 0;
    ctl->iters = 0;
    ctl->bnorm = sqrt(bb);
    ctl->rel = bb > 0.0 ? sqrt(rr) / sqrt(bb) : 0.0;
  }
}

__device__ __forceinline__ void sum_x_body(const CG &g, Team t) {
  __shared__ double sh[33];
  double s = 0.0;
  for (int p = t.bid * blockDim.x + threadIdx.x; p < g.P; p += t.nblk * blockDim.x) s += g.x[p];
  s = block_reduce<false>(s, sh);
  if (threadIdx.x == 0) g.part[S_SUMX * g.stride + t.bid] = s;
}

__device__ __forceinline__ void store_depth_body(const CG &g, const CGCtl *ctl, Team t) {
  __shared__ double sh[33];
  const double mean = total(g.part + S_SUMX * g.stride, g.nblk, sh) / (double)g.P;
  const bool flat = !(ctl->bnorm > 0.0);  // zero slopes everywhere: the surface is the plane H = 0
  for (int p = t.bid * blockDim.x + threadIdx.x; p < g.P; p += t.nblk * blockDim.x)
    g.depth[p] = flat ? 0.0f : (float)(g.x[p] - mean);
}

__global__ void __launch_bounds__(kThreads) k_zero_depth(const CG g) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < g.P; p += gridDim.x * blockDim.x) g.depth[p] = 0.0f;
}

// D_H partials: max |H_new - H_old|, sum (H_new - H_old)^2, max H_new, -min H_new.
__device__ __forceinline__ void depth_change_body(const CG &g, const float *old, Team t) {
  __shared__ double sh[33];
  double dmax = 0.0, dsq = 0.0, hmax = -INFINITY, hmin = -INFINITY;
  for (int p = t.bid * blockDim.x + threadIdx.x; p < g.P; p += t.nblk * blockDim.x) {
    const double a = g.depth[p], d = a - (double)old[p];
    dmax = fmax(dmax, fabs(d));
    dsq += d * d;
    hmax = fmax(hmax, a);
    hmin = fmax(hmin, -a);
  }
  dmax = block_reduce<true>(dmax, sh);
  if (threadIdx.x == 0) g.part[S_DMAX * g.stride + t.bid] = dmax;
  dsq = block_reduce<false>(dsq, sh);
  if (threadIdx.x == 0) g.part[S_DSQ * g.stride + t.bid] = dsq;
  hmax = block_reduce<true>(hmax, sh);
  if (threadIdx.x == 0) g.part[S_HMAX * g.stride + t.bid] = hmax;
  hmin = block_reduce<true>(hmin, sh);
  if (threadIdx.x == 0) g.part[S_HMIN * g.stride + t.bid] = hmin;
}

// Plain (one solve per launch) forms of the solver's kernels.
template <bool WEIGHTED = false>
__global__ void __launch_bounds__(kThreads) k_rhs(const CG g) { rhs_body<WEIGHTED>(g, whole_grid()); }
__global__ void __launch_bounds__(kThreads) k_load_x(const CG g) { load_x_body(g, whole_grid()); }
template <bool WEIGHTED = false>
__global__ void __launch_bounds__(kThreads) k_residual(const CG g, int rz_slot) {
  residual_body<WEIGHTED>(g, rz_slot, whole_grid());
}
__global__ void k_cg_start(const CG g, CGCtl *ctl) { cg_start_body(g, ctl); }
__global__ void __launch_bounds__(kThreads) k_sum_x(const CG g) { sum_x_body(g, whole_grid()); }
__global__ void __launch_bounds__(kThreads) k_store_depth(const CG g, const CGCtl *ctl) {
  store_depth_body(g, ctl, whole_grid());
}
__global__ void __launch_bounds__(kThreads) k_depth_change(const CG g, const float *old) {
  depth_change_body(g, old, whole_grid());
}

// Blocks of the cooperative solve: all must be co-resident; two per SM keep the
// barrier's arrival counter short.
int cg_grid_limit() {
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
  const void *fns[] = {(const void *)k_cg_loop<0, false>, (const void *)k_cg_loop<1, false>,
                       (const void *)k_cg_loop<0, true>, (const void *)k_cg_loop<1, true>};
  per = 1 << 30;
  for (const void *fn : fns) {
    int q = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&q, fn, kThreads, 0) != cudaSuccess) return 1;
    per = per < q ? per : q;
  }
  per = per < IRTPS_CG_BLOCKS_PER_SM ? per : IRTPS_CG_BLOCKS_PER_SM;
  return per * sms > 0 ? per * sms : 1;
}

static MG make_mg(const Ctx &c) {
  MG m{};
  m.levels = c.mg_levels;
  m.grid_levels = 0;
  for (int l = 0; l < c.mg_levels; ++l) {
    m.H[l] = c.mg_h[l];
    m.W[l] = c.mg_w[l];
    m.off[l] = c.mg_off[l];
    if (c.mg_h[l] * c.mg_w[l] > kMgBlockPoints) m.grid_levels = l + 1;
  }
  m.x0 = c.mg_x0;
  m.x1 = c.mg_x1;
  m.b = c.mg_b;
  m.wh = c.mg_wh;
  m.wv = c.mg_wv;
  m.omega = 0.8f;
  m.cscale = IRTPS_MG_CSCALE;
  return m;
}

// Levels and Galerkin edge weights of the multigrid hierarchy (host, once per context).
void mg_layout(int H, int W, int *levels, int *h, int *w, int *off, int *total) {
  int l = 0, o = 0;
  h[0] = H;
  w[0] = W;
  while (true) {
    off[l] = o;
    o += h[l] * w[l];
    if (h[l] * w[l] <= 16 || l + 1 >= kMgMaxLevels) break;
    h[l + 1] = (h[l] + 1) / 2;
    w[l + 1] = (w[l] + 1) / 2;
    ++l;
  }
  *levels = l + 1;
  *total = o;
}

void mg_weights(int levels, const int *h, const int *w, const int *off, float *wh, float *wv) {
  for (int i = 0; i < h[0]; ++i)
    for (int j = 0; j < w[0]; ++j) {
      wh[off[0] + i * w[0] + j] = j < w[0] - 1 ? 1.0f : 0.0f;
      wv[off[0] + i * w[0] + j] = i < h[0] - 1 ? 1.0f : 0.0f;
    }
  for (int l = 0; l + 1 < levels; ++l) {
    const int Hf = h[l], Wf = w[l], Hc = h[l + 1], Wc = w[l + 1];
    const float *fh = wh + off[l], *fv = wv + off[l];
    float *ch = wh + off[l + 1], *cv = wv + off[l + 1];
    for (int I = 0; I < Hc; ++I)
      for (int J = 0; J < Wc; ++J) {
        float sh = 0.0f, sv = 0.0f;
        if (2 * J + 2 < Wf)
          for (int i = 2 * I; i < 2 * I + 2 && i < Hf; ++i) sh += fh[i * Wf + 2 * J + 1];
        if (2 * I + 2 < Hf)
          for (int j = 2 * J; j < 2 * J + 2 && j < Wf; ++j) sv += fv[(2 * I + 1) * Wf + j];
        ch[I * Wc + J] = sh;
        cv[I * Wc + J] = sv;
      }
  }
}

static CG make_cg(Ctx &c) {
  CG g;
  g.H = c.H;
  g.W = c.W;
  g.P = c.H * c.W;
  g.h = 1.0 / (double)c.W;
  g.nz_min = c.opt.nz_min;
  g.nrm = c.nrm;
  g.depth = c.depth;
  g.x = c.cg_x;
  g.b = c.cg_b;
  g.r = c.cg_r;
  g.z = c.cg_z;
  g.p = c.cg_p;
  g.ap = c.cg_ap;
  g.part = c.part;
  g.stride = c.part_stride;
  g.nblk = c.cg_blocks;
  g.wh = c.mg_wh;
  g.wv = c.mg_wv;
  return g;
}

#define LAUNCH_CHECK()                      \
  do {                                      \
    cudaError_t e_ = cudaGetLastError();    \
    if (e_ != cudaSuccess) return e_;       \
  } while (0)

// D_H of the last iteration into the device statistics (one warp).
__device__ __forceinline__ void dh_final_body(const CG &g, DevStats *ds) {
  double dmax = 0.0, dsq = 0.0, hmax = -INFINITY, hmin = -INFINITY;
  for (int i = threadIdx.x; i < g.nblk; i += 32) {
    dmax = fmax(dmax, g.part[S_DMAX * g.stride + i]);
    dsq += g.part[S_DSQ * g.stride + i];
    hmax = fmax(hmax, g.part[S_HMAX * g.stride + i]);
    hmin = fmax(hmin, g.part[S_HMIN * g.stride + i]);
  }
  dmax = warp_max(dmax);
  dsq = warp_sum(dsq);
  hmax = warp_max(hmax);
  hmin = warp_max(hmin);
  if (threadIdx.x == 0) {
    const double range = hmax + hmin;  // max H - min H
    ds->dh_max = range > 0.0 ? dmax / range : 0.0;
    ds->dh_rms = sqrt(dsq / (double)g.P);
  }
}
__global__ void k_dh_final(const CG g, DevStats *ds) { dh_final_body(g, ds); }

// IRLS weights of the Huber M-estimator from the current iterate x: for every
// edge the slope residual u = (x_b - x_a) / h - (s_a + s_b) / 2 (FP64) gives
// w = 1 if |u| <= delta, else delta / |u|; written as the level-0 edge weights of
// the multigrid pool (zero on the last column / row, as the unit weights).
__device__ __forceinline__ void irls_weights_body(const CG &g, float *wh, float *wv, double delta, Team t) {
  for (int p = t.bid * blockDim.x + threadIdx.x; p < g.P; p += t.nblk * blockDim.x) {
    const int i = p / g.W, j = p - i * g.W;
    double pc, qc, pn, qn;
    slopes(g.nrm, p, g.nz_min, pc, qc);
    float a = 0.0f, b = 0.0f;
    if (j < g.W - 1) {
      slopes(g.nrm, p + 1, g.nz_min, pn, qn);
      const double u = fabs((g.x[p + 1] - g.x[p]) / g.h - (pc + pn) * 0.5);
      a = u <= delta ? 1.0f : (float)(delta / u);
    }
    if (i < g.H - 1) {
      slopes(g.nrm, p + g.W, g.nz_min, pn, qn);
      const double u = fabs((g.x[p + g.W] - g.x[p]) / g.h - (qc + qn) * 0.5);
      b = u <= delta ? 1.0f : (float)(delta / u);
    }
    wh[p] = a;
    wv[p] = b;
  }
}

// Galerkin weights of level l+1 from level l (2x2 aggregates): the sum of the fine
// edge weights crossing between two aggregates (the host's construction, on the device).
__device__ __forceinline__ void mg_coarsen_body(const MG &m, int l, float *wh, float *wv, Team t) {
  const int Hf = m.H[l], Wf = m.W[l], Hc = m.H[l + 1], Wc = m.W[l + 1];
  const float *fh = wh + m.off[l], *fv = wv + m.off[l];
  float *ch = wh + m.off[l + 1], *cv = wv + m.off[l + 1];
  for (int q = t.bid * blockDim.x + threadIdx.x; q < Hc * Wc; q += t.nblk * blockDim.x) {
    const int I = q / Wc, J = q - I * Wc;
    float sh = 0.0f, sv = 0.0f;
    if (2 * J + 2 < Wf)
      for (int i = 2 * I; i < 2 * I + 2 && i < Hf; ++i) sh += fh[i * Wf + 2 * J + 1];
    if (2 * I + 2 < Hf)
      for (int j = 2 * J; j < 2 * J + 2 && j < Wf; ++j) sv += fv[(2 * I + 1) * Wf + j];
    ch[q] = sh;
    cv[q] = sv;
  }
}

__global__ void __launch_bounds__(kThreads) k_irls_weights(const CG g, float *wh, float *wv, double delta) {
  irls_weights_body(g, wh, wv, delta, whole_grid());
}
__global__ void __launch_bounds__(kThreads) k_mg_coarsen(const MG m, int l, float *wh, float *wv) {
  mg_coarsen_body(m, l, wh, wv, whole_grid());
}

// A direct (spectral) solve counts as one iteration; its FP64 residual is checked
// against the tolerance like the last one of a PCG loop.
__global__ void k_direct_done(const CGCtl *ctl, CGAcc *acc, double tol) {
  const double rel = ctl->rel;
  acc->iters += 1;
  acc->last_iters = 1;
  acc->rel_last = rel;
  if (!isfinite(ctl->bnorm) || !isfinite(rel) || rel > tol) acc->bad = 1;
}

// One depth solve, enqueued without host round trips: right-hand side, warm
// start, residual, |b| on the device, the cooperative PCG loop, mean removal.
// Unit-weight solves with precond = 2 take the direct cosine-transform solve
// instead of the loop, then the same residual check and mean removal.
template <bool WEIGHTED>
static cudaError_t solve_once(Ctx &c) {
  const CG g = make_cg(c);
  const int nb = c.cg_blocks;
  CGCtl *ctl = (CGCtl *)c.cg_ctl;
  CGAcc *acc = &c.dstats->cg;
  k_rhs<WEIGHTED><<<nb, kThreads, 0, c.stream>>>(g);
  if (!WEIGHTED && c.opt.precond == 2 && c.sp_t) {
    LAUNCH_CHECK();
    cudaError_t e = launch_spectral(c, c.cg_b, c.cg_x);
    if (e != cudaSuccess) return e;
    k_residual<false><<<nb, kThreads, 0, c.stream>>>(g, S_RZ0);
    k_cg_start<<<1, 32, 0, c.stream>>>(g, ctl);
    k_direct_done<<<1, 1, 0, c.stream>>>(ctl, acc, c.opt.cg_tol);
    k_sum_x<<<nb, kThreads, 0, c.stream>>>(g);
    k_store_depth<<<nb, kThreads, 0, c.stream>>>(g, ctl);
    c.stats.launches += 6;
    LAUNCH_CHECK();
    return cudaSuccess;
  }
  k_load_x<<<nb, kThreads, 0, c.stream>>>(g);
  k_residual<WEIGHTED><<<nb, kThreads, 0, c.stream>>>(g, S_RZ0);
  k_cg_start<<<1, 32, 0, c.stream>>>(g, ctl);
  LAUNCH_CHECK();
  int m = c.opt.cg_check_every > 0 ? c.opt.cg_check_every : 10;
  double tol = c.opt.cg_tol;
  int max_iter = c.opt.cg_max_iter;
  MG mg = make_mg(c);
  if (WEIGHTED) mg.cscale = 1.0f;
  void *args[] = {(void *)&g, (void *)&ctl, (void *)&acc, (void *)&tol, (void *)&max_iter, (void *)&m, (void *)&mg};
  // multigrid for precond 1, and for the solves the spectral form does not cover
  const void *fn = c.opt.precond != 0 ? (const void *)k_cg_loop<1, WEIGHTED> : (const void *)k_cg_loop<0, WEIGHTED>;
  cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3(nb), dim3(kThreads), args, 0, c.stream);
  if (e != cudaSuccess) return e;
  k_sum_x<<<nb, kThreads, 0, c.stream>>>(g);
  k_store_depth<<<nb, kThreads, 0, c.stream>>>(g, ctl);
  c.stats.launches += 7;
  LAUNCH_CHECK();
  return cudaSuccess;
}

// The least-squares solve, then (option irls_iters) the Huber M-estimator by
// IRLS: weights from the last surface, Galerkin hierarchy rebuilt, weighted solve
// warm-started from it; the unit weights are put back at the end.
cudaError_t solve_depth_async(Ctx &c) {
  cudaError_t e = solve_once<false>(c);
  if (e != cudaSuccess || c.opt.irls_iters <= 0) return e;
  const CG g = make_cg(c);
  const MG mg = make_mg(c);
  const int nb = c.cg_blocks;
  for (int it = 0; it < c.opt.irls_iters; ++it) {
    k_irls_weights<<<nb, kThreads, 0, c.stream>>>(g, c.mg_wh, c.mg_wv, (double)c.opt.irls_delta);
    for (int l = 0; l + 1 < mg.levels; ++l) {
      const int n = mg.H[l + 1] * mg.W[l + 1];
      k_mg_coarsen<<<(n + kThreads - 1) / kThreads, kThreads, 0, c.stream>>>(mg, l, c.mg_wh, c.mg_wv);
    }
    c.stats.launches += mg.levels;
    LAUNCH_CHECK();
    if ((e = solve_once<true>(c)) != cudaSuccess) return e;
  }
  const size_t bytes = sizeof(float) * (size_t)c.mg_total;
  e = cudaMemcpyAsync(c.mg_wh, c.mg_wh_unit, bytes, cudaMemcpyDeviceToDevice, c.stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c.mg_wv, c.mg_wv_unit, bytes, cudaMemcpyDeviceToDevice, c.stream);
  return e;
}

int solve_depth(Ctx &c) {
  const cudaError_t e = solve_depth_async(c);
  if (e != cudaSuccess) {
    c.err = std::string("depth solve: ") + cudaGetErrorString(e);
    return IRTPS_ECUDA;
  }
  return IRTPS_OK;
}

cudaError_t depth_change_async(Ctx &c) {
  const CG g = make_cg(c);
  k_depth_change<<<c.cg_blocks, kThreads, 0, c.stream>>>(g, c.depth_prev);
  k_dh_final<<<1, 32, 0, c.stream>>>(g, c.dstats);
  c.stats.launches += 2;
  LAUNCH_CHECK();
  return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Batched depth solves: the solves of many objects in one launch per step.
// The blocks of a batched launch are split into contiguous teams, one per
// object (job o owns blocks [blk_begin(o), blk_begin(o + 1))); each team runs
// the plain solver on its object with barriers of its own, so objects of any
// size proceed independently within one co-resident cooperative grid.
// ---------------------------------------------------------------------------
struct CGJob {
  CG g;            // g.nblk: the team's block count
  MG mg;
  CGCtl *ctl;
  DevStats *ds;    // the object's statistics (solver accumulators, D_H)
  const float *old;  // previous surface (D_H)
  double tol;
  int max_iter, check, pre;
  int direct;      // unit-weight solves by the cosine transform (their passes run before the loop)
  int blk_begin;
  // robust integration (IRLS): the object's writable level-0.. weights, their unit copy, threshold
  float *wh, *wv;
  const float *wh_unit, *wv_unit;
  int mg_total;
  float irls_delta;
};

// Copy the job of this block's team into shared memory and run body(job, team)
// (PLAIN: with the unscaled coarse-grid correction of the weighted solves).
template <bool PLAIN = false, typename F>
__device__ __forceinline__ void for_team(const CGJob *__restrict__ jobs, int n, F &&body) {
  __shared__ CGJob sj;
  __shared__ int s_bid;
  if (threadIdx.x == 0) {
    int lo = 0, hi = n - 1;  // last job whose range starts at or before this block
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (jobs[mid].blk_begin <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
    }
    sj = jobs[lo];
    if (PLAIN) sj.mg.cscale = 1.0f;
    s_bid = (int)blockIdx.x - jobs[lo].blk_begin;
  }
  __syncthreads();
  body(sj, Team{s_bid, sj.g.nblk});
}

template <bool WEIGHTED>
__global__ void __launch_bounds__(kThreads) k_rhs_b(const CGJob *jobs, int n) {
  for_team(jobs, n, [](const CGJob &j, Team t) { rhs_body<WEIGHTED>(j.g, t); });
}
// the warm start of the iterative solves (a direct solve has its x already)
template <bool WEIGHTED>
__global__ void __launch_bounds__(kThreads) k_load_x_b(const CGJob *jobs, int n) {
  for_team(jobs, n, [](const CGJob &j, Team t) {
    if (WEIGHTED || !j.direct) load_x_body(j.g, t);
  });
}
template <bool WEIGHTED>
__global__ void __launch_bounds__(kThreads) k_residual_b(const CGJob *jobs, int n) {
  for_team(jobs, n, [](const CGJob &j, Team t) { residual_body<WEIGHTED>(j.g, S_RZ0, t); });
}
// one warp per job
__global__ void k_cg_start_b(const CGJob *jobs) { cg_start_body(jobs[blockIdx.x].g, jobs[blockIdx.x].ctl); }
template <bool WEIGHTED>
__global__ void __launch_bounds__(kThreads, IRTPS_CG_BATCH_MINB) k_cg_loop_b(const CGJob *jobs, int n) {
  for_team<WEIGHTED>(jobs, n, [](const CGJob &j, Team t) {
    if (!WEIGHTED && j.direct) {  // solved directly: one iteration, its FP64 residual checked
      if (t.bid == 0 && threadIdx.x == 0) {
        const double rel = j.ctl->rel;
        CGAcc *acc = &j.ds->cg;
        acc->iters += 1;
        acc->last_iters = 1;
        acc->rel_last = rel;
        if (!isfinite(j.ctl->bnorm) || !isfinite(rel) || rel > j.tol) acc->bad = 1;
      }
      return;
    }
    if (j.pre == 1)
      cg_loop_body<1, WEIGHTED>(j.g, j.ctl, &j.ds->cg, j.tol, j.max_iter, j.check, j.mg, t);
    else
      cg_loop_body<0, WEIGHTED>(j.g, j.ctl, &j.ds->cg, j.tol, j.max_iter, j.check, j.mg, t);
  });
}
__global__ void __launch_bounds__(kThreads) k_sum_x_b(const CGJob *jobs, int n) {
  for_team(jobs, n, [](const CGJob &j, Team t) { sum_x_body(j.g, t); });
}
__global__ void __launch_bounds__(kThreads) k_store_depth_b(const CGJob *jobs, int n) {
  for_team(jobs, n, [](const CGJob &j, Team t) { store_depth_body(j.g, j.ctl, t); });
}
__global__ void __launch_bounds__(kThreads) k_depth_change_b(const CGJob *jobs, int n) {
  for_team(jobs, n, [](const CGJob &j, Team t) { depth_change_body(j.g, j.old, t); });
}
__global__ void k_dh_final_b(const CGJob *jobs) { dh_final_body(jobs[blockIdx.x].g, jobs[blockIdx.x].ds); }
__global__ void __launch_bounds__(kThreads) k_irls_weights_b(const CGJob *jobs, int n) {
  for_team(jobs, n, [](const CGJob &j, Team t) { irls_weights_body(j.g, j.wh, j.wv, (double)j.irls_delta, t); });
}
__global__ void __launch_bounds__(kThreads) k_mg_coarsen_b(const CGJob *jobs, int n, int l) {
  for_team(jobs, n, [l](const CGJob &j, Team t) {
    if (l + 1 < j.mg.levels) mg_coarsen_body(j.mg, l, j.wh, j.wv, t);
  });
}
__global__ void __launch_bounds__(kThreads) k_unit_weights_b(const CGJob *jobs, int n) {
  for_team(jobs, n, [](const CGJob &j, Team t) {
    for (int q = t.bid * blockDim.x + threadIdx.x; q < j.mg_total; q += t.nblk * blockDim.x) {
      j.wh[q] = j.wh_unit[q];
      j.wv[q] = j.wv_unit[q];
    }
  });
}
__global__ void __launch_bounds__(kThreads) k_zero_depth_b(const CGJob *jobs, int n) {
  for_team(jobs, n, [](const CGJob &j, Team t) {
    for (int p = t.bid * blockDim.x + threadIdx.x; p < j.g.P; p += t.nblk * blockDim.x) j.g.depth[p] = 0.0f;
  });
}

size_t cg_job_bytes() { return sizeof(CGJob); }

// Co-resident blocks of the batched solve loop (at most IRTPS_CG_BATCH_BLOCKS_PER_SM per SM).
int cg_batch_grid_limit() {
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  int per_w = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_cg_loop_b<false>, kThreads, 0) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_w, k_cg_loop_b<true>, kThreads, 0) != cudaSuccess) return 0;
  per = per < per_w ? per : per_w;
  per = per < IRTPS_CG_BATCH_BLOCKS_PER_SM ? per : IRTPS_CG_BATCH_BLOCKS_PER_SM;
  return per * sms;
}

void cg_fill_job(Ctx &c, int nblk, int blk_begin, DevStats *ds, void *dst) {
  CGJob j{};
  j.g = make_cg(c);
  j.g.nblk = nblk;
  j.mg = make_mg(c);
  if (nblk == 1) j.mg.grid_levels = 0;  // a one-block team sweeps every level alone
  j.ctl = (CGCtl *)c.cg_ctl;
  j.ds = ds;
  j.old = c.depth_prev;
  j.tol = c.opt.cg_tol;
  j.max_iter = c.opt.cg_max_iter;
  j.check = c.opt.cg_check_every > 0 ? c.opt.cg_check_every : 10;
  j.pre = c.opt.precond != 0 ? 1 : 0;  // iterative solves: multigrid for precond 1 and 2
  j.direct = direct_solve(c) ? 1 : 0;
  j.blk_begin = blk_begin;
  j.wh = c.mg_wh;
  j.wv = c.mg_wv;
  j.wh_unit = c.mg_wh_unit;
  j.wv_unit = c.mg_wv_unit;
  j.mg_total = c.mg_total;
  j.irls_delta = c.opt.irls_delta;
  std::memcpy(dst, &j, sizeof(j));
}

template <bool WEIGHTED>
static cudaError_t solve_batch_once(cudaStream_t s, const CGJob *jobs, int n, int blocks, const SpectralBatch &sb) {
  k_rhs_b<WEIGHTED><<<blocks, kThreads, 0, s>>>(jobs, n);
  if (!WEIGHTED) {
    LAUNCH_CHECK();
    cudaError_t e = launch_spectral_batch(s, sb);
    if (e != cudaSuccess) return e;
  }
  k_load_x_b<WEIGHTED><<<blocks, kThreads, 0, s>>>(jobs, n);
  k_residual_b<WEIGHTED><<<blocks, kThreads, 0, s>>>(jobs, n);
  k_cg_start_b<<<n, 32, 0, s>>>(jobs);
  LAUNCH_CHECK();
  void *args[] = {(void *)&jobs, (void *)&n};
  cudaError_t e =
      cudaLaunchCooperativeKernel((const void *)k_cg_loop_b<WEIGHTED>, dim3(blocks), dim3(kThreads), args, 0, s);
  if (e != cudaSuccess) return e;
  k_sum_x_b<<<blocks, kThreads, 0, s>>>(jobs, n);
  k_store_depth_b<<<blocks, kThreads, 0, s>>>(jobs, n);
  LAUNCH_CHECK();
  return cudaSuccess;
}

// The batched solves; with irls_iters > 0 (the same for every object) each is
// followed by that many reweighting steps of the Huber M-estimator, as in the
// single-object solve, and the unit weights are put back at the end.
cudaError_t solve_depth_batch_async(cudaStream_t s, const void *d_jobs, int n, int blocks, int irls_iters,
                                    int max_levels, const SpectralBatch &sb) {
  const CGJob *jobs = (const CGJob *)d_jobs;
  cudaError_t e = solve_batch_once<false>(s, jobs, n, blocks, sb);
  if (e != cudaSuccess || irls_iters <= 0) return e;
  for (int it = 0; it < irls_iters; ++it) {
    k_irls_weights_b<<<blocks, kThreads, 0, s>>>(jobs, n);
    for (int l = 0; l + 1 < max_levels; ++l) k_mg_coarsen_b<<<blocks, kThreads, 0, s>>>(jobs, n, l);
    LAUNCH_CHECK();
    if ((e = solve_batch_once<true>(s, jobs, n, blocks, sb)) != cudaSuccess) return e;
  }
  k_unit_weights_b<<<blocks, kThreads, 0, s>>>(jobs, n);
  LAUNCH_CHECK();
  return cudaSuccess;
}

cudaError_t zero_depth_batch_async(cudaStream_t s, const void *d_jobs, int n, int blocks) {
  k_zero_depth_b<<<blocks, kThreads, 0, s>>>((const CGJob *)d_jobs, n);
  return cudaGetLastError();
}

cudaError_t depth_change_batch_async(cudaStream_t s, const void *d_jobs, int n, int blocks) {
  const CGJob *jobs = (const CGJob *)d_jobs;
  k_depth_change_b<<<blocks, kThreads, 0, s>>>(jobs, n);
  k_dh_final_b<<<n, 32, 0, s>>>(jobs);
  LAUNCH_CHECK();
  return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Allocation-free depth solve.  Some callers cannot allocate device memory at
// the moment they need a result: a host framework may own the whole device
// pool through its own allocator, or a latency-critical loop may not accept the
// device-wide synchronisation of cudaMalloc / cudaFree.  For them the solver's
// working vectors live in one file-scope device array, sized for at most
// kNoAllocMaxPixels pixels, that every GPU loading this library holds until the
// process exits.  Every call shares it, so calls that overlap on the GPU race.
// ---------------------------------------------------------------------------
constexpr int kNoAllocMaxPixels = 512 * 512;
constexpr int kNoAllocMaxBlocks = 2048;
constexpr size_t kNaX = 0;                                              // x: doubles
constexpr size_t kNaB = kNaX + 8ull * kNoAllocMaxPixels;               // b: doubles
constexpr size_t kNaR = kNaB + 8ull * kNoAllocMaxPixels;               // r: floats
constexpr size_t kNaZ = kNaR + 4ull * kNoAllocMaxPixels;               // z: floats
constexpr size_t kNaP = kNaZ + 4ull * kNoAllocMaxPixels;               // p: 2 x floats
constexpr size_t kNaAp = kNaP + 8ull * kNoAllocMaxPixels;              // Ap and correction: 2 x floats
constexpr size_t kNaPart = kNaAp + 8ull * kNoAllocMaxPixels;           // partials: doubles
constexpr size_t kNaCtl = kNaPart + 8ull * kPartSlots * kNoAllocMaxBlocks;
constexpr size_t kNaBytes = kNaCtl + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

// Device address of the scratch array on the current device: looked up once per
// device (the first call on a device does it) and cached for the life of the
// process; a cudaDeviceReset unloads the module, after which the cached address
// is no longer valid (the entry point is not for use across device resets).
static unsigned char *noalloc_base() {
  static std::mutex mu;
  static unsigned char *base[64] = {nullptr};
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!base[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) return nullptr;
    base[dev] = (unsigned char *)p;
  }
  return base[dev];
}

}  // namespace irtps

extern "C" int irtps_integrate_noalloc(const float *normals, int H, int W, float nz_min, double tol, int max_iter,
                                       float *depth, void *stream) {
  using namespace irtps;
  if (!normals || !depth || H < 2 || W < 2 || (long long)H * W > kNoAllocMaxPixels || !(nz_min > 0.0f) ||
      !(tol > 0.0) || max_iter < 0)
    return IRTPS_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char *base = noalloc_base();
  if (!base) return IRTPS_ECUDA;
  const int P = H * W;
  int nb = std::min((P + kThreads - 1) / kThreads, cg_grid_limit());
  nb = std::max(1, std::min(nb, kNoAllocMaxBlocks));
  CG g;
  g.H = H;
  g.W = W;
  g.P = P;
  g.h = 1.0 / (double)W;
  g.nz_min = nz_min;
  g.nrm = reinterpret_cast<const float4 *>(normals);
  g.depth = depth;
  g.x = reinterpret_cast<double *>(base + kNaX);
  g.b = reinterpret_cast<double *>(base + kNaB);
  g.r = reinterpret_cast<float *>(base + kNaR);
  g.z = reinterpret_cast<float *>(base + kNaZ);
  g.p = reinterpret_cast<float *>(base + kNaP);
  g.ap = reinterpret_cast<float *>(base + kNaAp);
  g.part = reinterpret_cast<double *>(base + kNaPart);
  g.stride = kNoAllocMaxBlocks;
  g.nblk = nb;
  g.wh = g.wv = nullptr;
  CGCtl *ctl = reinterpret_cast<CGCtl *>(base + kNaCtl);

  // a failure after the first launch waits for the queued kernels, so that none of
  // them still works on the shared array when the call returns
  auto failed = [s]() {
    cudaStreamSynchronize(s);
    return IRTPS_ECUDA;
  };
  k_rhs<false><<<nb, kThreads, 0, s>>>(g);
  k_load_x<<<nb, kThreads, 0, s>>>(g);
  k_residual<false><<<nb, kThreads, 0, s>>>(g, S_RZ0);
  k_cg_start<<<1, 32, 0, s>>>(g, ctl);  // also clears the barrier state left by the previous call
  if (cudaGetLastError() != cudaSuccess) return failed();
  int m = 10;
  const MG none{};
  CGAcc *acc = nullptr;
  void *args[] = {(void *)&g, (void *)&ctl, (void *)&acc, (void *)&tol, (void *)&max_iter, (void *)&m, (void *)&none};
  if (cudaLaunchCooperativeKernel((const void *)k_cg_loop<0, false>, dim3(nb), dim3(kThreads), args, 0, s) !=
      cudaSuccess)
    return failed();
  k_sum_x<<<nb, kThreads, 0, s>>>(g);
  k_store_depth<<<nb, kThreads, 0, s>>>(g, ctl);
  if (cudaGetLastError() != cudaSuccess) return failed();
  CGCtl h;
  if (cudaMemcpyAsync(&h, ctl, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess) return failed();
  if (cudaStreamSynchronize(s) != cudaSuccess) return IRTPS_ECUDA;
  if (h.err) return IRTPS_ETIMEOUT;
  if (!std::isfinite(h.bnorm)) return IRTPS_ENUMERIC;
  return (std::isfinite(h.rel) && h.rel <= tol) ? IRTPS_OK : IRTPS_ENUMERIC;
}


