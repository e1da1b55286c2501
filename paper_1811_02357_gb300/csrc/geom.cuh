// Device geometry of the reverted Monte-Carlo trace: random numbers, cosine
// sampling, ray / triangle tests and the max-pyramid heightfield march.
//
// Every operation whose result decides an integer (hit or miss, hit triangle,
// hit pixel, shadow visibility) is written with explicitly rounded FP32
// intrinsics (__fmul_rn, __fadd_rn, ...), which the compiler never fuses, so
// that the decision is a fixed function of the FP32 inputs.
//
// Coordinates: "grid" space, vertex (i, j) at (x, y, z) = (j, i, depth[i*W+j]);
// a world direction (dx, dy, dz) maps to (W dx, W dy, dz) (pixel pitch 1/W).
// Cell (cy, cx) holds triangles T0 = {(cy,cx), (cy,cx+1), (cy+1,cx+1)} and
// T1 = {(cy,cx), (cy+1,cx+1), (cy+1,cx)} with index 2*(cy*(W-1)+cx) + {0,1}.
#pragma once

#include <cstdint>
#include <math.h>
#include <cuda_runtime.h>

namespace irtps {

constexpr int kMaxLevels = 16;

__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float radd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float rsub(float a, float b) { return __fsub_rn(a, b); }

struct F3 {
  float x, y, z;
};

__device__ __forceinline__ F3 f3sub(F3 a, F3 b) { return {rsub(a.x, b.x), rsub(a.y, b.y), rsub(a.z, b.z)}; }
__device__ __forceinline__ F3 f3cross(F3 a, F3 b) {
  return {rsub(rmul(a.y, b.z), rmul(a.z, b.y)), rsub(rmul(a.z, b.x), rmul(a.x, b.z)),
          rsub(rmul(a.x, b.y), rmul(a.y, b.x))};
}
__device__ __forceinline__ float f3dot(F3 a, F3 b) {
  return radd(radd(rmul(a.x, b.x), rmul(a.y, b.y)), rmul(a.z, b.z));
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// 24-bit uniform in [0, 1), exact in FP32.
__device__ __forceinline__ float u24(uint32_t x) { return __uint2float_rn(x >> 8) * 5.9604644775390625e-08f; }

// cos(2 pi u), sin(2 pi u) for a 24-bit u: quadrant reduction (exact) and Taylor
// polynomials on [0, pi/4], every step rounded to FP32 on its own.
__device__ __forceinline__ void sincos_turn(float u, float &c, float &s) {
  const float v = rmul(u, 4.0f);
  const int q = (int)v;
  const float f = rsub(v, (float)q);
  const bool swap = f > 0.5f;
  const float g = swap ? rsub(1.0f, f) : f;
  const float x = rmul(g, (float)M_PI_2);
  const float x2 = rmul(x, x);
  float ps = 1.0f / 362880.0f;
  ps = rmul(ps, x2);
  ps = radd(-(1.0f / 5040.0f), ps);
  ps = rmul(ps, x2);
  ps = radd(1.0f / 120.0f, ps);
  ps = rmul(ps, x2);
  ps = radd(-(1.0f / 6.0f), ps);
  ps = rmul(ps, x2);
  ps = radd(1.0f, ps);
  const float sx = rmul(x, ps);
  float pc = -(1.0f / 3628800.0f);
  pc = rmul(pc, x2);
  pc = radd(1.0f / 40320.0f, pc);
  pc = rmul(pc, x2);
  pc = radd(-(1.0f / 720.0f), pc);
  pc = rmul(pc, x2);
  pc = radd(1.0f / 24.0f, pc);
  pc = rmul(pc, x2);
  pc = radd(-0.5f, pc);
  pc = rmul(pc, x2);
  const float cx = radd(1.0f, pc);
  const float st = swap ? cx : sx;
  const float ct = swap ? sx : cx;
  switch (q & 3) {
    case 0: c = ct; s = st; break;
    case 1: c = -st; s = ct; break;
    case 2: c = -ct; s = -st; break;
    default: c = st; s = -ct; break;
  }
}

// Cosine-weighted direction about the unit normal n (Malley's method) in the
// orthonormal basis of Duff et al., "Building an Orthonormal Basis, Revisited".
__device__ __forceinline__ F3 cosine_dir(F3 n, uint32_t x0, uint32_t x1) {
  const float u1 = u24(x0), u2 = u24(x1);
  const float r = __fsqrt_rn(u1);
  float c, s;
  sincos_turn(u2, c, s);
  const float lx = rmul(r, c), ly = rmul(r, s);
  const float lz = __fsqrt_rn(rsub(1.0f, u1));
  const float sign = copysignf(1.0f, n.z);
  const float a = __fdiv_rn(-1.0f, radd(sign, n.z));
  const float b = rmul(rmul(n.x, n.y), a);
  const F3 b1 = {radd(1.0f, rmul(rmul(rmul(sign, n.x), n.x), a)), rmul(sign, b), rmul(-sign, n.x)};
  const F3 b2 = {b, radd(sign, rmul(rmul(n.y, n.y), a)), -n.y};
  return {radd(radd(rmul(lx, b1.x), rmul(ly, b2.x)), rmul(lz, n.x)),
          radd(radd(rmul(lx, b1.y), rmul(ly, b2.y)), rmul(lz, n.y)),
          radd(radd(rmul(lx, b1.z), rmul(ly, b2.z)), rmul(lz, n.z))};
}

// Moeller-Trumbore, two-sided, closed barycentric bounds, hit iff t > 0.
__device__ __forceinline__ bool tri_hit(F3 o, F3 d, F3 v0, F3 v1, F3 v2, float &t_out) {
  const F3 e1 = f3sub(v1, v0);
  const F3 e2 = f3sub(v2, v0);
  const F3 pv = f3cross(d, e2);
  const float det = f3dot(e1, pv);
  if (det == 0.0f) return false;
  const float inv = __frcp_rn(det);
  const F3 tv = f3sub(o, v0);
  const float u = rmul(f3dot(tv, pv), inv);
  if (u < 0.0f || u > 1.0f) return false;
  const F3 qv = f3cross(tv, e1);
  const float v = rmul(f3dot(d, qv), inv);
  if (v < 0.0f || radd(u, v) > 1.0f) return false;
  const float t = rmul(f3dot(e2, qv), inv);
  if (!(t > 0.0f)) return false;
  t_out = t;
  return true;
}

// Heightfield + max pyramid as the march sees it.  The level table (offsets and
// row widths) lives in shared memory, filled by each block before use, so that
// a lane-dependent level index does not force it into local memory.
struct Field {
  const float *depth;       // H*W
  const float *pmax;        // all levels, level l at off[l], row-major lw[l] wide
  int H, W, Wc, Hc;         // Wc = W-1, Hc = H-1 cells
  int levels;               // levels the march uses (the top one may hold several nodes)
  int top_off;              // offset of the single node of the full pyramid (the surface maximum)
  int off[kMaxLevels];
  int lw[kMaxLevels];
};

struct LevelTable {
  int2 ol[kMaxLevels];  // per level: offset of its nodes in the pyramid arrays, row width
  float zmax_margin;    // (max height) + 1e-4: above it a rising ray can hit nothing
  float dz;             // node-skip margin on heights, 1e-5 (1 + |max height|)
};

// Height bounds of a surface from its top pyramid node.
__device__ __forceinline__ void set_height_bounds(const Field &f, LevelTable *t) {
  const float zmax = __ldg(f.pmax + f.top_off);
  t->zmax_margin = zmax + 1e-4f;
  t->dz = 1e-5f * (1.0f + fabsf(zmax));
}

// Copy the level table of f into shared memory and derive the height bounds from
// the top pyramid node (whole block; ends with a barrier).
__device__ __forceinline__ void load_levels(const Field &f, LevelTable *t) {
  if (threadIdx.x < kMaxLevels) t->ol[threadIdx.x] = make_int2(f.off[threadIdx.x], f.lw[threadIdx.x]);
  if (threadIdx.x == 0) set_height_bounds(f, t);
  __syncthreads();
}

// Work counters of one thread (pyramid nodes / cells examined, triangle tests, sampled directions).
struct Work {
  uint32_t nodes = 0, tris = 0, draws = 0;
};

#ifndef IRTPS_CLIMB
#define IRTPS_CLIMB 1
#endif
constexpr int kClimb = IRTPS_CLIMB;     // levels climbed after passing over a node
constexpr float kHitMargin = 1e-4f;   // entry beyond best hit by this: stop
constexpr float kCorner = 1e-5f;      // near-vertex crossing: test both side cells

// Both triangles of cell (cy, cx).  This is the Moeller-Trumbore test above
// written out for the cell's vertices, whose x and y are consecutive integers:
// every product with an edge component of 0 or 1 is exact, so dropping it leaves
// each remaining rounding, and hence every result bit, unchanged.  The
// rejections are evaluated as one predicate per triangle (straight-line code).
__device__ __forceinline__ void test_cell(const Field &f, int cy, int cx, F3 o, F3 d, float &bt, int &btri, Work &w) {
  w.tris += 2;
  const float *r0 = f.depth + (size_t)cy * f.W + cx;
  const float h00 = __ldg(r0), h01 = __ldg(r0 + 1), h10 = __ldg(r0 + f.W), h11 = __ldg(r0 + f.W + 1);
  const int base = 2 * (cy * f.Wc + cx);
  // shared by both triangles: v0 = (cx, cy, h00), tv = o - v0
  const F3 tv = {rsub(o.x, (float)cx), rsub(o.y, (float)cy), rsub(o.z, h00)};
  const float e11 = rsub(h11, h00);  // z of v11 - v0 (edge to the far corner)
  // T0 = (v00, v01, v11): e1 = (1, 0, h01 - h00), e2 = (1, 1, h11 - h00)
  float t0;
  bool hit0;
  {
    const float e1z = rsub(h01, h00);
    const F3 pv = {rsub(rmul(d.y, e11), d.z), rsub(d.z, rmul(d.x, e11)), rsub(d.x, d.y)};
    const float det = radd(pv.x, rmul(e1z, pv.z));
    const float inv = __frcp_rn(det);
    const float u = rmul(f3dot(tv, pv), inv);
    const F3 qv = {rmul(tv.y, e1z), rsub(tv.z, rmul(tv.x, e1z)), -tv.y};
    const float v = rmul(f3dot(d, qv), inv);
    t0 = rmul(radd(radd(qv.x, qv.y), rmul(e11, qv.z)), inv);
    hit0 = det != 0.0f && u >= 0.0f && u <= 1.0f && v >= 0.0f && radd(u, v) <= 1.0f && t0 > 0.0f;
  }
  // T1 = (v00, v11, v10): e1 = (1, 1, h11 - h00), e2 = (0, 1, h10 - h00)
  float t1;
  bool hit1;
  {
    const float e2z = rsub(h10, h00);
    const F3 pv = {rsub(rmul(d.y, e2z), d.z), -rmul(d.x, e2z), d.x};
    const float det = radd(radd(pv.x, pv.y), rmul(e11, pv.z));
    const float inv = __frcp_rn(det);
    const float u = rmul(f3dot(tv, pv), inv);
    const F3 qv = {rsub(rmul(tv.y, e11), tv.z), rsub(tv.z, rmul(tv.x, e11)), rsub(tv.x, tv.y)};
    const float v = rmul(f3dot(d, qv), inv);
    t1 = rmul(radd(qv.y, rmul(e2z, qv.z)), inv);
    hit1 = det != 0.0f && u >= 0.0f && u <= 1.0f && v >= 0.0f && radd(u, v) <= 1.0f && t1 > 0.0f;
  }
  if (hit0 && (btri < 0 || t0 < bt || (t0 == bt && base < btri))) {
    bt = t0;
    btri = base;
  }
  if (hit1 && (btri < 0 || t1 < bt || (t1 == bt && base + 1 < btri))) {
    bt = t1;
    btri = base + 1;
  }
}

// Cell index along one axis at which a cell walk stands when the other axis is
// crossed at parameter t: the first index c (from `cur`, moving by `s`, inside
// [lo, hi)) whose own exit parameter e(c) = (edge(c) - o) * inv is >= t, plus one
// step when e(c) == t (the walk then steps diagonally).  e(c) is monotone in c
// and differs from the exact crossing only by rounding (far below one cell), so
// the floor of the crossing coordinate is the answer or its neighbour: one probe
// on each side settles it.
__device__ __forceinline__ int cell_at(float o, float d, float inv, int s, int cur, int lo, int hi, float t) {
  const int cmin = s > 0 ? cur : lo;
  const int cmax = s > 0 ? hi - 1 : cur;
  int c = (int)floorf(radd(o, rmul(t, d)));
  c = min(max(c, cmin), cmax);
  // exit parameter of cell c along the direction of travel: edge c+1 (s > 0) or c (s < 0)
  const int up = s > 0 ? 1 : 0;
  const float e_c = rmul(rsub((float)(c + up), o), inv);
  const float e_back = rmul(rsub((float)(c + up - s), o), inv);  // e of the cell behind c
  if (c != (s > 0 ? cmin : cmax) && e_back >= t) {
    c -= s;
  } else if (c != (s > 0 ? cmax : cmin) && e_c < t) {
    c += s;
  }
  if (rmul(rsub((float)(c + up), o), inv) == t) c += s;
  return c;
}

// Incremental heightfield march.  The leaf steps are those of a plain 2D cell
// walk (exit parameter (X - o) * (1/d), ties stepping diagonally, both side cells
// tested at a near-vertex crossing); whole pyramid nodes that the ray passes
// above (by the margin dz) are skipped, landing in the exact cell the plain walk
// would reach.  The start cell holds the origin, on the side the ray moves toward
// when the origin is on a grid line; a ray running exactly along a grid line
// walks the cells on both sides (up to four walks).  `any` stops at the first hit.
struct Walker {
  F3 o, d;
  float ix, iy;
  int cx, cy, lv;
  float t_entry;
  float t_stop;  // the walk ends once a cell's entry lies beyond it: past the best hit (plus a margin),
                 // or, rising, above every vertex (plus a margin)
  float bt;
  int btri;
  int flags;  // bit 0: any-hit; bits 1, 2: a second walk in x, in y; bits 3-4: current walk index;
              // bits 5-6, 7-8: sign of d.x, of d.y, plus one
};

__device__ __forceinline__ int walker_sx(const Walker &m) { return ((m.flags >> 5) & 3) - 1; }
__device__ __forceinline__ int walker_sy(const Walker &m) { return ((m.flags >> 7) & 3) - 1; }

// Start cell of walk `wi`: the cell holding the origin, on the side the ray moves
// toward when the origin is on a grid line, shifted back by one column / row for
// the second walk of a ray that runs exactly along that grid line.
__device__ __forceinline__ void walker_begin_walk(Walker &m, int wi) {
  int cx = (int)floorf(m.o.x), cy = (int)floorf(m.o.y);
  if ((float)cx == m.o.x && m.d.x < 0.0f) --cx;
  if ((float)cy == m.o.y && m.d.y < 0.0f) --cy;
  const int nx = (m.flags & 2) ? 2 : 1;
  m.cx = cx - (wi % nx);
  m.cy = cy - (wi / nx);
  m.lv = 0;
  m.t_entry = 0.0f;
  m.flags = (m.flags & ~(3 << 3)) | (wi << 3);
}

// zmax_margin: the surface's maximum height plus its margin (LevelTable::zmax_margin).
__device__ __forceinline__ void walker_init(Walker &m, F3 o, F3 d, bool any, float zmax_margin) {
  m.o = o;
  m.d = d;
  m.ix = __frcp_rn(d.x);
  m.iy = __frcp_rn(d.y);
  const bool on_x = floorf(o.x) == o.x, on_y = floorf(o.y) == o.y;
  const int sx = d.x > 0.0f ? 1 : (d.x < 0.0f ? -1 : 0);
  const int sy = d.y > 0.0f ? 1 : (d.y < 0.0f ? -1 : 0);
  m.flags = (any ? 1 : 0) | ((on_x && d.x == 0.0f) ? 2 : 0) | ((on_y && d.y == 0.0f) ? 4 : 0) | ((sx + 1) << 5) |
            ((sy + 1) << 7);
  m.bt = __int_as_float(0x7f800000);
  m.btri = -1;
  // a rising ray is above every vertex (by the margin) beyond this parameter; any rounding of it
  // only moves the end of the walk within the margin, where no triangle can be hit
  m.t_stop = d.z > 0.0f ? (zmax_margin - o.z) / d.z : __int_as_float(0x7f800000);
  walker_begin_walk(m, 0);
}

// The march advances in two kinds of steps.  A node step examines the pyramid
// node at the current level: it passes over it (skip), descends a level, or -
// at level 0, when the ray is not above the cell - leaves the walker waiting for
// a leaf step, which tests the cell's triangles and takes the plain walk's step
// to the next cell.  Keeping the two apart lets a warp run the expensive leaf
// step for many lanes at once.

// Bookkeeping at the start of every step: ends the current walk (and the march,
// or moves to the next walk of a grid-line ray).  Returns true when the march is over.
__device__ __forceinline__ bool walker_finish_walk(Walker &m) {
  if ((m.flags & 1) && m.btri >= 0) return true;
  const int wi = ((m.flags >> 3) & 3) + 1;
  const int walks = ((m.flags & 2) ? 2 : 1) * ((m.flags & 4) ? 2 : 1);
  if (wi < walks) {
    walker_begin_walk(m, wi);
    return false;
  }
  return true;
}

__device__ __forceinline__ bool walker_walk_over(const Walker &m, const Field &f) {
  return (unsigned)m.cx >= (unsigned)f.Wc || (unsigned)m.cy >= (unsigned)f.Hc || m.t_entry > m.t_stop;
}

// Node step.  Returns true when the march is over; sets at_leaf when the walker
// waits for a leaf step.  A skip leaves the node across the axis whose exit comes
// first (both on a tie); the cell on the other axis at that parameter comes from one
// cell_at on the selected axis, so that lanes skipping across x and across y run the
// same instructions.  The walk's end has one call site.
__device__ __forceinline__ bool walker_node_step(Walker &m, const Field &f, const LevelTable &lt, Work &w,
                                                 bool &at_leaf) {
  const float inf = __int_as_float(0x7f800000);
  bool over = walker_walk_over(m, f);
  if (!over) {
    const int sx = walker_sx(m), sy = walker_sy(m);
    const int lv = m.lv;
    const int nx = m.cx >> lv, ny = m.cy >> lv;
    const int X0 = nx << lv, Y0 = ny << lv;
    const int X1 = min(X0 + (1 << lv), f.Wc), Y1 = min(Y0 + (1 << lv), f.Hc);
    const int2 ol = lt.ol[lv];
    const float nmax = __ldg(f.pmax + ol.x + ny * ol.y + nx);
    ++w.nodes;
    const float tX = sx != 0 ? rmul(rsub((float)(sx > 0 ? X1 : X0), m.o.x), m.ix) : inf;
    const float tY = sy != 0 ? rmul(rsub((float)(sy > 0 ? Y1 : Y0), m.o.y), m.iy) : inf;
    const float t_exit = fminf(tX, tY);
    // lowest height of the ray over the node: at entry when rising, else at exit
    const float zlow = fmaf(m.d.z >= 0.0f ? m.t_entry : t_exit, m.d.z, m.o.z);
    if (zlow > nmax + lt.dz) {
      if (t_exit == inf) {
        over = true;  // vertical ray above everything below it
      } else {
        // crossed axes: x alone (tX < tY), y alone (tY < tX), or both (a tie)
        const bool cross_x = !(tY < tX), cross_y = !(tX < tY);
        const float te = (cross_y && !cross_x) ? tY : tX;
        const bool y_alone = cross_y && !cross_x;
        const int s_o = y_alone ? sx : sy;  // the axis not crossed, when one is crossed alone
        if (cross_x != cross_y && s_o != 0) {
          const int c = cell_at(y_alone ? m.o.x : m.o.y, y_alone ? m.d.x : m.d.y, y_alone ? m.ix : m.iy, s_o,
                                y_alone ? m.cx : m.cy, y_alone ? X0 : Y0, y_alone ? X1 : Y1, te);
          if (y_alone) m.cx = c; else m.cy = c;
        }
        if (cross_x) m.cx = sx > 0 ? X1 : X0 - 1;
        if (cross_y) m.cy = sy > 0 ? Y1 : Y0 - 1;
        m.t_entry = te;
        m.lv = min(lv + kClimb, f.levels - 1);
      }
    } else if (lv > 0) {
      m.lv = lv - 1;
    } else {
      at_leaf = true;
    }
  }
  return over ? walker_finish_walk(m) : false;
}

// Leaf step: both triangles of the current cell (and, at a near-vertex
// crossing, of the two cells beside the vertex), then the plain walk's step.
// Returns true when the march is over.
__device__ __forceinline__ bool walker_leaf_step(Walker &m, const Field &f, Work &w) {
  const float inf = __int_as_float(0x7f800000);
  const int sx = walker_sx(m), sy = walker_sy(m);
  test_cell(f, m.cy, m.cx, m.o, m.d, m.bt, m.btri, w);
  const float tx =
      sx > 0 ? rmul(rsub((float)(m.cx + 1), m.o.x), m.ix) : (sx < 0 ? rmul(rsub((float)m.cx, m.o.x), m.ix) : inf);
  const float ty =
      sy > 0 ? rmul(rsub((float)(m.cy + 1), m.o.y), m.iy) : (sy < 0 ? rmul(rsub((float)m.cy, m.o.y), m.iy) : inf);
  if (tx != inf && ty != inf && fabsf(rsub(tx, ty)) <= rmul(kCorner, fmaxf(tx, ty))) {
    if (m.cx + sx >= 0 && m.cx + sx < f.Wc) test_cell(f, m.cy, m.cx + sx, m.o, m.d, m.bt, m.btri, w);
    if (m.cy + sy >= 0 && m.cy + sy < f.Hc) test_cell(f, m.cy + sy, m.cx, m.o, m.d, m.bt, m.btri, w);
  }
  if (m.btri >= 0) {
    if (m.flags & 1) return true;
    m.t_stop = fminf(m.t_stop, radd(m.bt, kHitMargin));  // later cells may only hold closer hits
  }
  if (tx == inf && ty == inf) return walker_finish_walk(m);
  if (tx < ty) {
    m.cx += sx;
    m.t_entry = tx;
  } else if (ty < tx) {
    m.cy += sy;
    m.t_entry = ty;
  } else {
    m.cx += sx;
    m.cy += sy;
    m.t_entry = tx;
  }
  return false;
}

// One step of either kind.  Returns true when the march is over.
__device__ __forceinline__ bool walker_step(Walker &m, const Field &f, const LevelTable &lt, Work &w) {
  bool at_leaf = false;
  if (walker_node_step(m, f, lt, w, at_leaf)) return true;
  return at_leaf ? walker_leaf_step(m, f, w) : false;
}

// Blocking march (probes, render): steps until done or until `budget` steps are used.
__device__ __forceinline__ bool march(const Field &f, const LevelTable &lt, F3 o, F3 d, bool any, float &t, int &tri,
                                     int &budget, Work &w) {
  Walker m;
  walker_init(m, o, d, any, lt.zmax_margin);
  while (!walker_step(m, f, lt, w)) {
    if (--budget < 0) break;
  }
  t = m.bt;
  tri = m.btri;
  return m.btri >= 0;
}

// ---------------------------------------------------------------------------
// Early escape of primary rays.  For every pixel vertex p and each of the eight
// octants of azimuth (signs of the grid direction's x and y, and whether |y|
// exceeds |x|; the diagonals belong to both neighbours), hz bounds from above
// the slope (height per grid unit) under which the terrain is seen from p:
//   hz = max over cells c meeting the closed octant wedge at p, c not touching p,
//        of (max height of c - H_p) / (distance from p to c).
// A rising ray leaving p's lifted vertex with slope above hz is at every cell c of
// the wedge above c's highest vertex (its height there is at least
// H_p + dist * slope), so it can hit nothing beyond the cell it starts in.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int octant_of(float gx, float gy) {
  return (gx < 0.0f ? 1 : 0) | (gy < 0.0f ? 2 : 0) | (fabsf(gy) > fabsf(gx) ? 4 : 0);
}

// Whether the rectangle [a1, a2] x [b1, b2] (relative to p) meets the closed wedge of octant o.
__device__ __forceinline__ bool wedge_meets(int o, int a1, int a2, int b1, int b2) {
  int A1 = a1, A2 = a2, B1 = b1, B2 = b2;
  if (o & 1) { A1 = -a2; A2 = -a1; }
  if (o & 2) { B1 = -b2; B2 = -b1; }
  if (o & 4) {
    int t = A1; A1 = B1; B1 = t;
    t = A2; A2 = B2; B2 = t;
  }
  return A2 >= 0 && B2 >= 0 && max(B1, 0) <= A2;
}

// Nearest vertex index of a hit coordinate, ties to the lower index.
__device__ __forceinline__ int nearest_index(float q, int n) {
  const int v = (int)ceilf(rsub(q, 0.5f));
  return min(n - 1, max(0, v));
}

}  // namespace irtps
