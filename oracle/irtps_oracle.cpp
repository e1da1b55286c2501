// IRT-PS oracle: reverted Monte-Carlo trace, forward render and their helpers.
//
// TEST INFRASTRUCTURE ONLY.  This is a plain, slow, CPU restatement of what
// the IRT-PS hot path computes, written from the paper (Khadka, Remagnino,
// Argyriou, "Object 3D Reconstruction based on Photometric Stereo and Inverted
// Rendering", arXiv:1811.02357).  Only the test-suite, the smoke check and the
// benchmark's CPU-baseline leg may load it; the CUDA library never does, and
// this file shares no code with it.
//
// Precision.  Radiance is accumulated in FP64 (plain sums, sample order
// ascending, bounce order ascending).  The geometry of every ray (sampled
// direction, triangle tests, hit point) is a template on the scalar type T:
// T = double is the FP64 reference; T = float takes each integer decision
// (hit / miss, hit triangle, hit pixel, shadow visibility) in single
// precision with every operation rounded on its own, which is the precision
// the GPU kernel decides in.  Build with -ffp-contract=off so that no product
// is fused into a sum.
//
// Coordinates.  The heightfield has H rows and W columns of samples at the
// pixel centres; pixel pitch h = 1/W in x and y, heights in the same unit.
// Geometry is done in "grid" coordinates: vertex (i, j) sits at
// (x, y, z) = (j, i, depth[i*W + j]), so a world direction (dx, dy, dz) maps to
// (W*dx, W*dy, dz).  Cell (cy, cx) is split on the diagonal into
// T0 = {(cy,cx), (cy,cx+1), (cy+1,cx+1)} and T1 = {(cy,cx), (cy+1,cx+1), (cy+1,cx)};
// triangle index = 2*(cy*(W-1) + cx) + {0,1}.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// ---------------------------------------------------------------------------
// Philox4x32-10, from Salmon, Moraes, Dror and Shaw, "Parallel Random Numbers:
// As Easy as 1, 2, 3" (SC'11): ten rounds of two 32x32->64 multiplies with the
// key bumped by the Weyl constants between rounds.
// ---------------------------------------------------------------------------
void philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c1 ^ k0;
    const uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

// 24-bit uniform in [0, 1): exact in both float and double.
template <class T>
T uniform24(uint32_t x) {
  return (T)(x >> 8) * (T)(1.0 / 16777216.0);
}

// Counter layout of one random draw: {pixel, sample, (light<<8)|(bounce<<4)|stream, iteration}.
void draw(uint32_t pixel, uint32_t sample, uint32_t light, uint32_t bounce, uint32_t stream,
          uint32_t iter, const uint32_t key[2], uint32_t out[4]) {
  const uint32_t ctr[4] = {pixel, sample, (light << 8) | (bounce << 4) | stream, iter};
  philox4x32_10(ctr, key, out);
}

// ---------------------------------------------------------------------------
// cos(2*pi*u), sin(2*pi*u).
// double: the C library.  float: quadrant reduction (exact for a 24-bit u) and
// Taylor polynomials of sin and cos about 0 on [0, pi/4], each operation rounded
// to float, so that a second implementation following the same steps returns
// the same bits.
// ---------------------------------------------------------------------------
template <class T>
void sincos_turn(T u, T &c, T &s);

template <>
void sincos_turn<double>(double u, double &c, double &s) {
  const double phi = 2.0 * M_PI * u;
  c = std::cos(phi);
  s = std::sin(phi);
}

template <>
void sincos_turn<float>(float u, float &c, float &s) {
  const float v = u * 4.0f;             // exact: power-of-two scale
  const int q = (int)v;                 // quadrant, v >= 0
  const float f = v - (float)q;         // exact, in [0, 1)
  const bool swap = f > 0.5f;
  const float g = swap ? (1.0f - f) : f;  // exact, in [0, 0.5]
  const float x = g * (float)M_PI_2;    // angle in [0, pi/4]
  const float x2 = x * x;
  // sin x = x (1 - x^2/3! + x^4/5! - x^6/7! + x^8/9!)
  float ps = 1.0f / 362880.0f;           // 1/9!
  ps = ps * x2;
  ps = -(1.0f / 5040.0f) + ps;           // -1/7!
  ps = ps * x2;
  ps = 1.0f / 120.0f + ps;               // 1/5!
  ps = ps * x2;
  ps = -(1.0f / 6.0f) + ps;              // -1/3!
  ps = ps * x2;
  ps = 1.0f + ps;
  const float sx = x * ps;
  // cos x = 1 - x^2/2! + x^4/4! - x^6/6! + x^8/8! - x^10/10!
  float pc = -(1.0f / 3628800.0f);       // -1/10!
  pc = pc * x2;
  pc = 1.0f / 40320.0f + pc;             // 1/8!
  pc = pc * x2;
  pc = -(1.0f / 720.0f) + pc;            // -1/6!
  pc = pc * x2;
  pc = 1.0f / 24.0f + pc;                // 1/4!
  pc = pc * x2;
  pc = -0.5f + pc;                      // -1/2!
  pc = pc * x2;
  const float cx = 1.0f + pc;
  // angle within the quadrant: theta = g*pi/2 (swap: theta = pi/2 - x)
  const float st = swap ? cx : sx;
  const float ct = swap ? sx : cx;
  switch (q & 3) {
    case 0: c = ct;  s = st;  break;
    case 1: c = -st; s = ct;  break;
    case 2: c = -ct; s = -st; break;
    default: c = st; s = -ct; break;
  }
}

template <class T>
struct V3 {
  T x, y, z;
};

template <class T>
inline V3<T> sub(const V3<T> &a, const V3<T> &b) {
  return {a.x - b.x, a.y - b.y, a.z - b.z};
}
template <class T>
inline V3<T> cross(const V3<T> &a, const V3<T> &b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
template <class T>
inline T dot(const V3<T> &a, const V3<T> &b) {
  return a.x * b.x + a.y * b.y + a.z * b.z;
}

// Orthonormal basis (b1, b2) completing the unit vector n, after Duff et al.,
// "Building an Orthonormal Basis, Revisited" (JCGT 2017).
template <class T>
void onb(const V3<T> &n, V3<T> &b1, V3<T> &b2) {
  const T sign = std::copysign((T)1, n.z);
  const T a = (T)(-1) / (sign + n.z);
  const T b = n.x * n.y * a;
  b1 = {(T)1 + sign * n.x * n.x * a, sign * b, -sign * n.x};
  b2 = {b, sign + n.y * n.y * a, -n.y};
}

// Cosine-weighted direction about n (Malley's method: a uniform point on the
// unit disc lifted to the hemisphere), pdf = cos(theta)/pi.
template <class T>
V3<T> cosine_dir(const V3<T> &n, uint32_t x0, uint32_t x1) {
  const T u1 = uniform24<T>(x0);
  const T u2 = uniform24<T>(x1);
  const T r = std::sqrt(u1);
  T c, s;
  sincos_turn<T>(u2, c, s);
  const T lx = r * c;
  const T ly = r * s;
  const T lz = std::sqrt((T)1 - u1);
  V3<T> b1, b2;
  onb<T>(n, b1, b2);
  return {lx * b1.x + ly * b2.x + lz * n.x,
          lx * b1.y + ly * b2.y + lz * n.y,
          lx * b1.z + ly * b2.z + lz * n.z};
}

// Moeller-Trumbore ray/triangle test ("Fast, Minimum Storage Ray/Triangle
// Intersection", 1997), two-sided, closed barycentric bounds, hit iff t > 0.
template <class T>
bool tri_hit(const V3<T> &o, const V3<T> &d, const V3<T> &v0, const V3<T> &v1,
             const V3<T> &v2, T &t_out) {
  const V3<T> e1 = sub(v1, v0);
  const V3<T> e2 = sub(v2, v0);
  const V3<T> pv = cross(d, e2);
  const T det = dot(e1, pv);
  if (det == (T)0) return false;
  const T inv = (T)1 / det;
  const V3<T> tv = sub(o, v0);
  const T u = dot(tv, pv) * inv;
  if (u < (T)0 || u > (T)1) return false;
  const V3<T> qv = cross(tv, e1);
  const T v = dot(d, qv) * inv;
  if (v < (T)0 || u + v > (T)1) return false;
  const T t = dot(e2, qv) * inv;
  if (!(t > (T)0)) return false;
  t_out = t;
  return true;
}

struct Field {
  int H, W;
  const float *depth;  // H*W
  float zmax;          // max over all heights
};

template <class T>
inline V3<T> vertex(const Field &f, int i, int j) {
  return {(T)j, (T)i, (T)f.depth[(size_t)i * f.W + j]};
}

template <class T>
struct Hit {
  bool hit;
  T t;
  long tri;
};

// Test both triangles of cell (cy, cx); keep the closest hit, ties to the lower index.
template <class T>
inline void test_cell(const Field &f, int cy, int cx, const V3<T> &o, const V3<T> &d, Hit<T> &best) {
  const V3<T> a = vertex<T>(f, cy, cx);
  const V3<T> b = vertex<T>(f, cy, cx + 1);
  const V3<T> c = vertex<T>(f, cy + 1, cx + 1);
  const V3<T> e = vertex<T>(f, cy + 1, cx);
  const long base = 2L * ((long)cy * (f.W - 1) + cx);
  T t;
  if (tri_hit<T>(o, d, a, b, c, t)) {
    if (!best.hit || t < best.t || (t == best.t && base < best.tri)) best = {true, t, base};
  }
  if (tri_hit<T>(o, d, a, c, e, t)) {
    if (!best.hit || t < best.t || (t == best.t && base + 1 < best.tri)) best = {true, t, base + 1};
  }
}

// Reference intersector: every triangle of the mesh.
template <class T>
Hit<T> brute_force(const Field &f, const V3<T> &o, const V3<T> &d) {
  Hit<T> best{false, std::numeric_limits<T>::infinity(), -1};
  for (int cy = 0; cy + 1 < f.H; ++cy)
    for (int cx = 0; cx + 1 < f.W; ++cx) test_cell<T>(f, cy, cx, o, d, best);
  return best;
}

// Plain 2D walk over the cells the ray's xy-projection crosses (Amanatides and
// Woo, "A Fast Voxel Traversal Algorithm", 1987), starting in cell (cx, cy).
// The parameter at which the ray reaches grid line X is (X - o.x) * (1 / d.x),
// the reciprocal rounded once.  Cells are visited in order of entry parameter;
// when a crossing passes within a rounding margin of a grid vertex, the two
// cells beside the vertex are tested as well, so that a hit at (or rounding-near)
// the vertex is seen whichever way the crossing rounds.  The walk stops once the
// next entry lies beyond the best hit (plus a margin), when an upward ray is above
// every vertex, or when it leaves the mesh.
template <class T>
void walk(const Field &f, const V3<T> &o, const V3<T> &d, int cx, int cy, Hit<T> &best) {
  const T inf = std::numeric_limits<T>::infinity();
  const T margin = sizeof(T) == 4 ? (T)1e-4 : (T)1e-9;
  const T corner = sizeof(T) == 4 ? (T)1e-5 : (T)1e-12;
  const int Wc = f.W - 1, Hc = f.H - 1;
  const int sx = d.x > (T)0 ? 1 : (d.x < (T)0 ? -1 : 0);
  const int sy = d.y > (T)0 ? 1 : (d.y < (T)0 ? -1 : 0);
  const T ix = (T)1 / d.x, iy = (T)1 / d.y;
  T t_entry = 0;
  const int max_steps = 2 * (Wc + Hc) + 8;
  for (int step = 0; step < max_steps; ++step) {
    if (cx < 0 || cy < 0 || cx >= Wc || cy >= Hc) break;
    if (best.hit && t_entry > best.t + margin) break;
    if (d.z > (T)0 && o.z + t_entry * d.z > (T)f.zmax + margin) break;
    test_cell<T>(f, cy, cx, o, d, best);
    const T tx = sx > 0 ? ((T)(cx + 1) - o.x) * ix : (sx < 0 ? ((T)cx - o.x) * ix : inf);
    const T ty = sy > 0 ? ((T)(cy + 1) - o.y) * iy : (sy < 0 ? ((T)cy - o.y) * iy : inf);
    if (tx == inf && ty == inf) break;
    if (tx != inf && ty != inf && std::fabs(tx - ty) <= corner * std::max(tx, ty)) {
      if (cx + sx >= 0 && cx + sx < Wc) test_cell<T>(f, cy, cx + sx, o, d, best);
      if (cy + sy >= 0 && cy + sy < Hc) test_cell<T>(f, cy + sy, cx, o, d, best);
    }
    if (tx < ty) {
      cx += sx;
      t_entry = tx;
    } else if (ty < tx) {
      cy += sy;
      t_entry = ty;
    } else {
      cx += sx;
      cy += sy;
      t_entry = tx;
    }
  }
}

// Closest hit along the ray.  The start cell holds the origin, taking the cell
// on the side the ray moves toward when the origin lies on a grid line.  A ray
// that runs exactly along a grid line (zero x or y direction from an integer
// coordinate) touches the cells on both sides of it, so both are walked.
template <class T>
Hit<T> march(const Field &f, const V3<T> &o, const V3<T> &d) {
  Hit<T> best{false, std::numeric_limits<T>::infinity(), -1};
  if (f.W < 2 || f.H < 2) return best;
  int cx = (int)std::floor(o.x);
  int cy = (int)std::floor(o.y);
  const bool on_x = (T)cx == o.x, on_y = (T)cy == o.y;
  if (on_x && d.x < (T)0) --cx;
  if (on_y && d.y < (T)0) --cy;
  const int nx = (on_x && d.x == (T)0) ? 2 : 1;
  const int ny = (on_y && d.y == (T)0) ? 2 : 1;
  for (int a = 0; a < ny; ++a)
    for (int b = 0; b < nx; ++b) walk<T>(f, o, d, cx - b, cy - a, best);
  return best;
}

// Bilinear lookup of a C x EH x EW latitude-longitude map over the full sphere:
// theta = acos(w_z) over rows, phi = atan2(w_y, w_x) in [0, 2pi) over columns,
// texel centres at half-integers, wrap in phi, clamp in theta.
double env_lookup(const float *env, int EH, int EW, int c, double wx, double wy, double wz) {
  const double norm = std::sqrt(wx * wx + wy * wy + wz * wz);
  const double z = std::min(1.0, std::max(-1.0, wz / norm));
  const double theta = std::acos(z);
  double phi = std::atan2(wy, wx);
  if (phi < 0) phi += 2.0 * M_PI;
  const double row = theta / M_PI * EH - 0.5;
  const double col = phi / (2.0 * M_PI) * EW - 0.5;
  const double r0 = std::floor(row), c0 = std::floor(col);
  const double fr = row - r0, fc = col - c0;
  const int ra = std::min(EH - 1, std::max(0, (int)r0));
  const int rb = std::min(EH - 1, std::max(0, (int)r0 + 1));
  int ca = (int)c0 % EW;
  if (ca < 0) ca += EW;
  const int cb = (ca + 1) % EW;
  const float *m = env + (size_t)c * EH * EW;
  const double top = (1.0 - fc) * m[(size_t)ra * EW + ca] + fc * m[(size_t)ra * EW + cb];
  const double bot = (1.0 - fc) * m[(size_t)rb * EW + ca] + fc * m[(size_t)rb * EW + cb];
  return (1.0 - fr) * top + fr * bot;
}

struct Scene {
  int H, W, C, K;
  const float *depth;   // H*W
  const float *nrm;     // H*W*4 : nx, ny, nz, mean albedo
  const float *albedo;  // C*H*W
  const float *lights;  // K*3, unit, world
  const float *env;     // C*EH*EW
  int EH, EW;
  int shadow_rays;
  Field field;
};

// Nearest vertex to a hit point (grid coordinates), ties to the lower index.
template <class T>
inline int nearest_index(T q, int n) {
  int v = (int)std::ceil(q - (T)0.5);
  return std::min(n - 1, std::max(0, v));
}

// Hit point o + t d of a march (grid coordinates) and the pixel whose shading the
// path reads there: the mesh vertex nearest in x-y, ties to the lower index.
template <class T>
inline V3<T> hit_point(const V3<T> &o, const V3<T> &d, T t) {
  return {o.x + t * d.x, o.y + t * d.y, o.z + t * d.z};
}
template <class T>
inline size_t hit_pixel(const V3<T> &q, int H, int W) {
  return (size_t)nearest_index<T>(q.y, H) * W + nearest_index<T>(q.x, W);
}

template <class T>
inline T eps_lift(int W) {
  return (T)1e-3 / (T)W;
}

// Shadow ray from o toward light k: true when the light is visible.
template <class T>
bool visible(const Scene &sc, const V3<T> &o, int k) {
  const V3<T> dl = {(T)sc.lights[3 * k + 0] * (T)sc.W, (T)sc.lights[3 * k + 1] * (T)sc.W,
                    (T)sc.lights[3 * k + 2]};
  return !march<T>(sc.field, o, dl).hit;
}

struct Counts {
  uint64_t primary = 0, segments = 0;
};

// One sample path of the reverted trace for (pixel p, light k, sample s):
// adds the path's radiance to acc[0..C) (in units of incident radiance).
// Bounce b = 1..B: sample a cosine direction about the current normal estimate,
// march; on escape add T*Env(w) and stop; on a hit at q add
// T * rho_q * max(0, n_q . l_k) * V_k(q), then T <- T * rho_q and continue from q.
template <class T>
void trace_path(const Scene &sc, int p, int k, int s, int B, uint32_t iter, uint32_t stream,
                const uint32_t key[2], double *acc, int32_t *rec, Counts &cnt) {
  const int W = sc.W, H = sc.H;
  const T eps = eps_lift<T>(W);
  const int pi = p / W, pj = p % W;
  V3<T> o = {(T)pj, (T)pi, (T)sc.depth[p] + eps};
  V3<T> n = {(T)sc.nrm[4 * (size_t)p + 0], (T)sc.nrm[4 * (size_t)p + 1], (T)sc.nrm[4 * (size_t)p + 2]};
  double thr[3] = {1.0, 1.0, 1.0};
  const float *l = sc.lights + 3 * k;
  const V3<T> lf = {(T)l[0], (T)l[1], (T)l[2]};
  for (int b = 1; b <= B; ++b) {
    uint32_t x[4];
    draw((uint32_t)p, (uint32_t)s, (uint32_t)k, (uint32_t)b, stream, iter, key, x);
    const V3<T> dw = cosine_dir<T>(n, x[0], x[1]);
    const V3<T> dg = {dw.x * (T)W, dw.y * (T)W, dw.z};
    cnt.segments++;
    if (b == 1) cnt.primary++;
    const Hit<T> h = march<T>(sc.field, o, dg);
    if (!h.hit) {
      for (int c = 0; c < sc.C; ++c)
        acc[c] += thr[c] * env_lookup(sc.env, sc.EH, sc.EW, c, (double)dw.x, (double)dw.y, (double)dw.z);
      if (rec) {
        rec[2 * (b - 1)] = -1;
        rec[2 * (b - 1) + 1] = -1;
      }
      return;
    }
    const V3<T> q = hit_point<T>(o, dg, h.t);
    const size_t qp = hit_pixel<T>(q, H, W);
    const V3<T> nq = {(T)sc.nrm[4 * qp + 0], (T)sc.nrm[4 * qp + 1], (T)sc.nrm[4 * qp + 2]};
    const V3<T> o2 = {q.x, q.y, q.z + eps};
    int vis = -1;
    if (dot(nq, lf) > (T)0) {
      vis = 1;
      if (sc.shadow_rays) {
        cnt.segments++;
        vis = visible<T>(sc, o2, k) ? 1 : 0;
      }
      const double cosd = std::max(0.0, (double)sc.nrm[4 * qp + 0] * l[0] +
                                            (double)sc.nrm[4 * qp + 1] * l[1] +
                                            (double)sc.nrm[4 * qp + 2] * l[2]);
      for (int c = 0; c < sc.C; ++c)
        acc[c] += thr[c] * (double)sc.albedo[(size_t)c * H * W + qp] * cosd * (double)vis;
    }
    if (rec) {
      rec[2 * (b - 1)] = (int32_t)qp;
      rec[2 * (b - 1) + 1] = vis;
    }
    for (int c = 0; c < sc.C; ++c) thr[c] *= (double)sc.albedo[(size_t)c * H * W + qp];
    o = o2;
    n = nq;
  }
}

template <class T>
void trace_pixels(const Scene &sc, const int32_t *pixels, int n_pix, int spp, int B, uint32_t iter,
                  uint32_t stream, const uint32_t key[2], double *out_lbar, int32_t *out_rec,
                  uint64_t *out_counts, int n_threads) {
  const int K = sc.K, C = sc.C;
  uint64_t prim = 0, segs = 0;
#ifdef _OPENMP
  if (n_threads <= 0) n_threads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads) reduction(+ : prim, segs)
#endif
  for (int ip = 0; ip < n_pix; ++ip) {
    const int p = pixels ? pixels[ip] : ip;
    Counts cnt;
    for (int k = 0; k < K; ++k) {
      double sum[3] = {0.0, 0.0, 0.0};
      for (int s = 0; s < spp; ++s) {
        double acc[3] = {0.0, 0.0, 0.0};
        int32_t *rec = nullptr;
        if (out_rec) {
          rec = out_rec + ((((size_t)ip * K + k) * spp + s) * B) * 2;
          for (int b = 0; b < 2 * B; ++b) rec[b] = -2;
        }
        trace_path<T>(sc, p, k, s, B, iter, stream, key, acc, rec, cnt);
        for (int c = 0; c < C; ++c) sum[c] += acc[c];
      }
      for (int c = 0; c < C; ++c) out_lbar[((size_t)k * C + c) * n_pix + ip] = sum[c] / (double)spp;
    }
    prim += cnt.primary;
    segs += cnt.segments;
  }
  if (out_counts) {
    out_counts[0] = prim;
    out_counts[1] = segs;
  }
}

// Light-shared sampling: one sample path per (pixel p, sample s) serves all K
// lights.  The directions are drawn with light field 0 of the counter, so the
// path of sample s is the one light 0 takes in the per-light trace.  On escape
// T*Env(w) is added for every light; on a hit at q, every light k with
// n_q . l_k > 0 gets T * rho_q * (n_q . l_k) * V_k(q) (one shadow ray per such
// light); then T <- T * rho_q and the path continues.  acc is K x 3.
// rec (nullable) holds B entries of 1 + K ints: {hit pixel | -1, V_0 .. V_{K-1}}.
template <class T>
void trace_path_shared(const Scene &sc, int p, int s, int B, uint32_t iter, uint32_t stream,
                       const uint32_t key[2], double *acc, int32_t *rec, Counts &cnt) {
  const int W = sc.W, H = sc.H, K = sc.K;
  const T eps = eps_lift<T>(W);
  const int pi = p / W, pj = p % W;
  V3<T> o = {(T)pj, (T)pi, (T)sc.depth[p] + eps};
  V3<T> n = {(T)sc.nrm[4 * (size_t)p + 0], (T)sc.nrm[4 * (size_t)p + 1], (T)sc.nrm[4 * (size_t)p + 2]};
  double thr[3] = {1.0, 1.0, 1.0};
  for (int b = 1; b <= B; ++b) {
    int32_t *r = rec ? rec + (size_t)(b - 1) * (1 + K) : nullptr;
    uint32_t x[4];
    draw((uint32_t)p, (uint32_t)s, 0u, (uint32_t)b, stream, iter, key, x);
    const V3<T> dw = cosine_dir<T>(n, x[0], x[1]);
    const V3<T> dg = {dw.x * (T)W, dw.y * (T)W, dw.z};
    cnt.segments++;
    if (b == 1) cnt.primary++;
    const Hit<T> h = march<T>(sc.field, o, dg);
    if (!h.hit) {
      for (int k = 0; k < K; ++k)
        for (int c = 0; c < sc.C; ++c)
          acc[3 * k + c] +=
              thr[c] * env_lookup(sc.env, sc.EH, sc.EW, c, (double)dw.x, (double)dw.y, (double)dw.z);
      if (r)
        for (int k = 0; k <= K; ++k) r[k] = -1;
      return;
    }
    const V3<T> q = hit_point<T>(o, dg, h.t);
    const size_t qp = hit_pixel<T>(q, H, W);
    const V3<T> nq = {(T)sc.nrm[4 * qp + 0], (T)sc.nrm[4 * qp + 1], (T)sc.nrm[4 * qp + 2]};
    const V3<T> o2 = {q.x, q.y, q.z + eps};
    if (r) r[0] = (int32_t)qp;
    for (int k = 0; k < K; ++k) {
      const float *l = sc.lights + 3 * k;
      const V3<T> lf = {(T)l[0], (T)l[1], (T)l[2]};
      int vis = -1;
      if (dot(nq, lf) > (T)0) {
        vis = 1;
        if (sc.shadow_rays) {
          cnt.segments++;
          vis = visible<T>(sc, o2, k) ? 1 : 0;
        }
        const double cosd = std::max(0.0, (double)sc.nrm[4 * qp + 0] * l[0] + (double)sc.nrm[4 * qp + 1] * l[1] +
                                              (double)sc.nrm[4 * qp + 2] * l[2]);
        for (int c = 0; c < sc.C; ++c)
          acc[3 * k + c] += thr[c] * (double)sc.albedo[(size_t)c * H * W + qp] * cosd * (double)vis;
      }
      if (r) r[1 + k] = vis;
    }
    for (int c = 0; c < sc.C; ++c) thr[c] *= (double)sc.albedo[(size_t)c * H * W + qp];
    o = o2;
    n = nq;
  }
}

template <class T>
void trace_pixels_shared(const Scene &sc, const int32_t *pixels, int n_pix, int spp, int B, uint32_t iter,
                         uint32_t stream, const uint32_t key[2], double *out_lbar, int32_t *out_rec,
                         uint64_t *out_counts, int n_threads) {
  const int K = sc.K, C = sc.C;
  uint64_t prim = 0, segs = 0;
#ifdef _OPENMP
  if (n_threads <= 0) n_threads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads) reduction(+ : prim, segs)
#endif
  for (int ip = 0; ip < n_pix; ++ip) {
    const int p = pixels ? pixels[ip] : ip;
    Counts cnt;
    std::vector<double> sum((size_t)3 * K, 0.0), acc((size_t)3 * K);
    for (int s = 0; s < spp; ++s) {
      std::fill(acc.begin(), acc.end(), 0.0);
      int32_t *rec = nullptr;
      if (out_rec) {
        rec = out_rec + ((size_t)ip * spp + s) * B * (1 + K);
        for (int i = 0; i < B * (1 + K); ++i) rec[i] = -2;
      }
      trace_path_shared<T>(sc, p, s, B, iter, stream, key, acc.data(), rec, cnt);
      for (int i = 0; i < 3 * K; ++i) sum[i] += acc[i];
    }
    for (int k = 0; k < K; ++k)
      for (int c = 0; c < C; ++c) out_lbar[((size_t)k * C + c) * n_pix + ip] = sum[3 * k + c] / (double)spp;
    prim += cnt.primary;
    segs += cnt.segments;
  }
  if (out_counts) {
    out_counts[0] = prim;
    out_counts[1] = segs;
  }
}

Scene make_scene(int H, int W, int C, int K, const float *depth, const float *nrm, const float *albedo,
                 const float *lights, const float *env, int EH, int EW, int shadow_rays) {
  Scene sc{H, W, C, K, depth, nrm, albedo, lights, env, EH, EW, shadow_rays, {H, W, depth, 0.0f}};
  float zmax = -std::numeric_limits<float>::infinity();
  for (size_t i = 0; i < (size_t)H * W; ++i) zmax = std::max(zmax, depth[i]);
  sc.field.zmax = zmax;
  return sc;
}

}  // namespace

extern "C" {

// Known-answer access to the generator.
void oracle_philox4x32_10(const uint32_t *ctr, const uint32_t *key, uint32_t *out) {
  philox4x32_10(ctr, key, out);
}

// n directions for (normal[i], x0[i], x1[i]); fp32 != 0 selects single precision.
void oracle_cosine_dirs(int n, const double *normals, const uint32_t *x0, const uint32_t *x1, int fp32,
                        double *out) {
  for (int i = 0; i < n; ++i) {
    if (fp32) {
      const V3<float> nn = {(float)normals[3 * i], (float)normals[3 * i + 1], (float)normals[3 * i + 2]};
      const V3<float> d = cosine_dir<float>(nn, x0[i], x1[i]);
      out[3 * i] = d.x;
      out[3 * i + 1] = d.y;
      out[3 * i + 2] = d.z;
    } else {
      const V3<double> nn = {normals[3 * i], normals[3 * i + 1], normals[3 * i + 2]};
      const V3<double> d = cosine_dir<double>(nn, x0[i], x1[i]);
      out[3 * i] = d.x;
      out[3 * i + 1] = d.y;
      out[3 * i + 2] = d.z;
    }
  }
}

// Basis vectors b1, b2 for n normals (FP64).
void oracle_onb(int n, const double *normals, double *b1, double *b2) {
  for (int i = 0; i < n; ++i) {
    V3<double> a, b;
    onb<double>({normals[3 * i], normals[3 * i + 1], normals[3 * i + 2]}, a, b);
    b1[3 * i] = a.x;
    b1[3 * i + 1] = a.y;
    b1[3 * i + 2] = a.z;
    b2[3 * i] = b.x;
    b2[3 * i + 1] = b.y;
    b2[3 * i + 2] = b.z;
  }
}

// cos(2 pi u), sin(2 pi u) for n 24-bit uniforms given as their integer numerators m (u = m / 2^24).
void oracle_sincos_turn(int n, const uint32_t *m, int fp32, double *c, double *s) {
  for (int i = 0; i < n; ++i) {
    if (fp32) {
      float cf, sf;
      sincos_turn<float>((float)m[i] * (1.0f / 16777216.0f), cf, sf);
      c[i] = cf;
      s[i] = sf;
    } else {
      sincos_turn<double>((double)m[i] / 16777216.0, c[i], s[i]);
    }
  }
}

// One Moeller-Trumbore test per row: o, d, v0, v1, v2 (3 doubles each, rounded to
// float first when fp32 != 0).  out_t = t, or NaN on a miss.
void oracle_tri_hit(int n, const double *rows, int fp32, double *out_t) {
  for (int i = 0; i < n; ++i) {
    const double *r = rows + 15 * i;
    if (fp32) {
      V3<float> v[5];
      for (int a = 0; a < 5; ++a) v[a] = {(float)r[3 * a], (float)r[3 * a + 1], (float)r[3 * a + 2]};
      float t;
      out_t[i] = tri_hit<float>(v[0], v[1], v[2], v[3], v[4], t) ? (double)t : NAN;
    } else {
      V3<double> v[5];
      for (int a = 0; a < 5; ++a) v[a] = {r[3 * a], r[3 * a + 1], r[3 * a + 2]};
      double t;
      out_t[i] = tri_hit<double>(v[0], v[1], v[2], v[3], v[4], t) ? t : NAN;
    }
  }
}

// Intersect n rays (origin, direction in grid coordinates; 6 doubles each) with the
// meshed heightfield.  brute != 0 tests every triangle, else walks the cells.
// out_t = t or NaN; out_tri = triangle index or -1.
void oracle_intersect(int H, int W, const float *depth, int n, const double *rays, int fp32, int brute,
                      double *out_t, int64_t *out_tri) {
  Field f{H, W, depth, -std::numeric_limits<float>::infinity()};
  for (size_t i = 0; i < (size_t)H * W; ++i) f.zmax = std::max(f.zmax, depth[i]);
  for (int i = 0; i < n; ++i) {
    const double *r = rays + 6 * i;
    if (fp32) {
      const V3<float> o = {(float)r[0], (float)r[1], (float)r[2]};
      const V3<float> d = {(float)r[3], (float)r[4], (float)r[5]};
      const Hit<float> h = brute ? brute_force<float>(f, o, d) : march<float>(f, o, d);
      out_t[i] = h.hit ? (double)h.t : NAN;
      out_tri[i] = h.hit ? h.tri : -1;
    } else {
      const V3<double> o = {r[0], r[1], r[2]};
      const V3<double> d = {r[3], r[4], r[5]};
      const Hit<double> h = brute ? brute_force<double>(f, o, d) : march<double>(f, o, d);
      out_t[i] = h.hit ? h.t : NAN;
      out_tri[i] = h.hit ? h.tri : -1;
    }
  }
}

// Hit pixel of n rays (origin, direction in grid coordinates; 6 doubles each)
// as the trace takes it: the march's closest hit, its point o + t d and the
// nearest mesh vertex (ties to the lower index); -1 when the ray escapes.
void oracle_hit_pixels(int H, int W, const float *depth, int n, const double *rays, int fp32, int64_t *out) {
  Field f{H, W, depth, -std::numeric_limits<float>::infinity()};
  for (size_t i = 0; i < (size_t)H * W; ++i) f.zmax = std::max(f.zmax, depth[i]);
  for (int i = 0; i < n; ++i) {
    const double *r = rays + 6 * i;
    if (fp32) {
      const V3<float> o = {(float)r[0], (float)r[1], (float)r[2]};
      const V3<float> d = {(float)r[3], (float)r[4], (float)r[5]};
      const Hit<float> h = march<float>(f, o, d);
      out[i] = h.hit ? (int64_t)hit_pixel<float>(hit_point<float>(o, d, h.t), H, W) : -1;
    } else {
      const V3<double> o = {r[0], r[1], r[2]};
      const V3<double> d = {r[3], r[4], r[5]};
      const Hit<double> h = march<double>(f, o, d);
      out[i] = h.hit ? (int64_t)hit_pixel<double>(hit_point<double>(o, d, h.t), H, W) : -1;
    }
  }
}

// Environment lookup for n world directions (3 doubles each), channel c.
void oracle_env_lookup(const float *env, int EH, int EW, int c, int n, const double *dirs, double *out) {
  for (int i = 0; i < n; ++i) out[i] = env_lookup(env, EH, EW, c, dirs[3 * i], dirs[3 * i + 1], dirs[3 * i + 2]);
}

// Mean incident radiance Lbar(k, c, pixel) of the reverted trace over the current
// estimate (depth, normals, albedo), for the listed pixels (NULL: all H*W).
//   out_lbar  : K*C*n_pix doubles, [k][c][ip]
//   out_rec   : optional, n_pix*K*spp*B*2 int32, per segment {hit pixel or -1 escape or
//               -2 not reached, shadow visibility 1/0 or -1 not cast}
//   out_counts: optional, {primary segments, all segments incl. shadow rays}
// Random draws: Philox4x32-10 with key {seed_lo ^ obj, seed_hi} and counter
// {pixel, sample, (k<<8)|(b<<4)|stream, iter}.
int oracle_trace(int H, int W, int C, int K, const float *depth, const float *nrm, const float *albedo,
                 const float *lights, const float *env, int EH, int EW, const int32_t *pixels, int n_pix,
                 int spp, int bounces, uint64_t seed, uint32_t obj, uint32_t iter, uint32_t stream,
                 int shadow_rays, int fp32, int n_threads, double *out_lbar, int32_t *out_rec,
                 uint64_t *out_counts) {
  if (H < 2 || W < 2 || C < 1 || C > 3 || K < 1 || spp < 1 || bounces < 1 || bounces > 3) return -1;
  const Scene sc = make_scene(H, W, C, K, depth, nrm, albedo, lights, env, EH, EW, shadow_rays);
  const uint32_t key[2] = {(uint32_t)seed ^ obj, (uint32_t)(seed >> 32)};
  if (!pixels) n_pix = H * W;
  if (fp32)
    trace_pixels<float>(sc, pixels, n_pix, spp, bounces, iter, stream, key, out_lbar, out_rec, out_counts,
                        n_threads);
  else
    trace_pixels<double>(sc, pixels, n_pix, spp, bounces, iter, stream, key, out_lbar, out_rec, out_counts,
                         n_threads);
  return 0;
}

// The light-shared trace (same arguments as oracle_trace): out_lbar K x C x n_pix;
// out_rec optional n_pix x spp x bounces x (1 + K): {hit pixel | -1 escape | -2 not
// reached, then V_k: 1 visible, 0 blocked, -1 not cast, -2 not reached}.
int oracle_trace_shared(int H, int W, int C, int K, const float *depth, const float *nrm, const float *albedo,
                        const float *lights, const float *env, int EH, int EW, const int32_t *pixels, int n_pix,
                        int spp, int bounces, uint64_t seed, uint32_t obj, uint32_t iter, uint32_t stream,
                        int shadow_rays, int fp32, int n_threads, double *out_lbar, int32_t *out_rec,
                        uint64_t *out_counts) {
  if (H < 2 || W < 2 || C < 1 || C > 3 || K < 1 || spp < 1 || bounces < 1 || bounces > 3) return -1;
  const Scene sc = make_scene(H, W, C, K, depth, nrm, albedo, lights, env, EH, EW, shadow_rays);
  const uint32_t key[2] = {(uint32_t)seed ^ obj, (uint32_t)(seed >> 32)};
  if (!pixels) n_pix = H * W;
  if (fp32)
    trace_pixels_shared<float>(sc, pixels, n_pix, spp, bounces, iter, stream, key, out_lbar, out_rec, out_counts,
                               n_threads);
  else
    trace_pixels_shared<double>(sc, pixels, n_pix, spp, bounces, iter, stream, key, out_lbar, out_rec,
                                out_counts, n_threads);
  return 0;
}

// Shadow visibility V_k(p) of every pixel's own vertex toward every light:
// out[k*H*W + p] = 1 visible, 0 blocked, -1 not cast (n_p . l_k <= 0).
int oracle_pixel_visibility(int H, int W, int K, const float *depth, const float *nrm, const float *lights,
                            int fp32, int32_t *out) {
  if (H < 2 || W < 2 || K < 1) return -1;
  const Scene sc = make_scene(H, W, 1, K, depth, nrm, nullptr, lights, nullptr, 0, 0, 1);
  for (int k = 0; k < K; ++k) {
    for (int p = 0; p < H * W; ++p) {
      const int pi = p / W, pj = p % W;
      int32_t v;
      if (fp32) {
        const V3<float> n = {sc.nrm[4 * p], sc.nrm[4 * p + 1], sc.nrm[4 * p + 2]};
        const V3<float> l = {lights[3 * k], lights[3 * k + 1], lights[3 * k + 2]};
        const V3<float> o = {(float)pj, (float)pi, depth[p] + eps_lift<float>(W)};
        v = dot(n, l) > 0.0f ? (visible<float>(sc, o, k) ? 1 : 0) : -1;
      } else {
        const V3<double> n = {sc.nrm[4 * p], sc.nrm[4 * p + 1], sc.nrm[4 * p + 2]};
        const V3<double> l = {lights[3 * k], lights[3 * k + 1], lights[3 * k + 2]};
        const V3<double> o = {(double)pj, (double)pi, (double)depth[p] + eps_lift<double>(W)};
        v = dot(n, l) > 0.0 ? (visible<double>(sc, o, k) ? 1 : 0) : -1;
      }
      out[(size_t)k * H * W + p] = v;
    }
  }
  return 0;
}

// Standard normal deviates of the image noise, Box-Muller on Philox with
// counter {pixel, 0, (k<<8)|(c<<4)|2, 0xFFFFFFFF}: out[(k*C + c)*H*W + p].
void oracle_noise(int H, int W, int C, int K, uint64_t seed, uint32_t obj, double *out) {
  const uint32_t key[2] = {(uint32_t)seed ^ obj, (uint32_t)(seed >> 32)};
  for (int k = 0; k < K; ++k)
    for (int c = 0; c < C; ++c)
      for (int p = 0; p < H * W; ++p) {
        uint32_t x[4];
        draw((uint32_t)p, 0u, (uint32_t)k, (uint32_t)c, 2u, 0xFFFFFFFFu, key, x);
        const double u1 = (double)((x[0] >> 8) + 1u) / 16777216.0;  // (0, 1]
        const double u2 = (double)(x[1] >> 8) / 16777216.0;
        out[((size_t)k * C + c) * H * W + p] = std::sqrt(-2.0 * std::log(u1)) * std::cos(2.0 * M_PI * u2);
      }
}

}  // extern "C"
