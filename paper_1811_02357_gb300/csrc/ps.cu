// Image correction and photometric stereo (Sec. III Eq. 3-4; Sec. IV stage 5).
//
// Per pixel p: I(k, c) = A0(k, c, p) - rho_t(c, p) * Lbar(k, c, p); row k is valid
// iff tau_lo < mean_c I(k, c) < tau_hi (decided in FP32, each operation rounded
// on its own).  All rows valid: G_c = pinv(L) I_c with pinv(L) = (L^T L)^-1 L^T
// (Eq. 4), summed as pinv(L) I, or - when L^T L is well conditioned (1-norm
// condition number at most 16, decided on the host in FP64) - as (L^T L)^-1 (L^T I),
// the same product associated the other way, which needs only the one running
// sum L^T I that masked pixels need anyway.  Otherwise the normal equations
// (L_v^T L_v) G_c = L_v^T I_v,c over the valid rows; fewer than 3 rows or a 1-norm
// condition number above cond_max marks the pixel invalid.
// n = normalize(sum_c G_c), rho_c = |G_c|; invalid pixels get n = (0, 0, 1), rho = 0.
//
// The contraction pinv(L) [3 x K] x I [K x C*P] streams K*C values per pixel for
// 6*K*C flops: far below the tensor-core ridge, so it runs on the FP32 pipes
// with coalesced [k][c][p] loads and the pixel's state written once.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "irtps_internal.h"

namespace irtps {

struct PSArgs {
  const void *images;
  const float *lbar;
  float *albedo;        // in: rho_t, out: rho_{t+1}
  float4 *nrm;
  uint8_t *valid;
  int P, K;
  float tau_lo, tau_hi;
  double cond_max;
  int zero_indirect;    // 1: Lbar taken as 0 (iteration 0, classic PS)
  float pinv[3][kMaxLights];
  float light[kMaxLights][3];
  float minv[6];        // (L^T L)^-1: m00 m01 m02 m11 m12 m22
  int normal_eq;        // 1: fully valid pixels as (L^T L)^-1 (L^T I)
  int blk_begin;        // first block of the object in a batched launch
};

template <typename TI>
__device__ __forceinline__ float load_img(const TI *p);
template <>
__device__ __forceinline__ float load_img<float>(const float *p) { return __ldg(p); }
template <>
__device__ __forceinline__ float load_img<__half>(const __half *p) { return __half2float(__ldg(p)); }

// Row k of pixel p: I(k, c) = A0 - rho_c Lbar (each operation rounded on its own)
// and its validity (tau_lo < mean_c I < tau_hi), accumulated into R = L_v^T I over
// the valid rows (the right-hand side of the masked normal equations) and, unless
// the normal-equation form (NE) serves fully valid pixels, into G = pinv(L) I over
// all rows; both in FP32.
template <int C, bool NE>
__device__ __forceinline__ void ps_row(const PSArgs &a, int k, const float *rho, const float *a0, const float *lb,
                                       float (&G)[3][C], float (&R)[3][C], unsigned long long &valid) {
  float I[C];
#pragma unroll
  for (int c = 0; c < C; ++c) I[c] = __fsub_rn(a0[c], __fmul_rn(rho[c], lb[c]));
  float chat = I[0];
  if (C == 3) chat = __fdiv_rn(__fadd_rn(__fadd_rn(I[0], I[1]), I[2]), 3.0f);
  const bool ok = chat > a.tau_lo && chat < a.tau_hi;
  if (ok) valid |= 1ull << k;
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const float l = ok ? a.light[k][r] : 0.0f;
#pragma unroll
    for (int c = 0; c < C; ++c) {
      if (!NE) G[r][c] = fmaf(a.pinv[r][k], I[c], G[r][c]);
      R[r][c] = fmaf(l, I[c], R[r][c]);
    }
  }
}

// G = (L^T L)^-1 R for a fully valid pixel in the normal-equation form.
template <int C>
__device__ __forceinline__ void ps_apply_minv(const PSArgs &a, const float (&R)[3][C], float (&G)[3][C]) {
  const float *m = a.minv;
#pragma unroll
  for (int c = 0; c < C; ++c) {
    const float r0 = R[0][c], r1 = R[1][c], r2 = R[2][c];
    G[0][c] = fmaf(m[0], r0, fmaf(m[1], r1, m[2] * r2));
    G[1][c] = fmaf(m[1], r0, fmaf(m[3], r1, m[4] * r2));
    G[2][c] = fmaf(m[2], r0, fmaf(m[4], r1, m[5] * r2));
  }
}

// Normal and albedo of pixel p from G (Eq. 4 and the text after it): n = normalize(sum_c G_c),
// rho_c = |G_c|; a pixel whose solve failed (ok false) or whose sum vanishes is invalid.
template <int C>
__device__ __forceinline__ void ps_store(const PSArgs &a, int p, const float (&G)[3][C], bool ok) {
  const size_t P = (size_t)a.P;
  float sx = 0.0f, sy = 0.0f, sz = 0.0f;
#pragma unroll
  for (int c = 0; c < C; ++c) {
    sx += G[0][c];
    sy += G[1][c];
    sz += G[2][c];
  }
  const float norm = sqrtf(sx * sx + sy * sy + sz * sz);
  if (!(norm > 0.0f) || !isfinite(norm)) ok = false;
  float4 out = make_float4(0.0f, 0.0f, 1.0f, 0.0f);
  float rsum = 0.0f;
  float rout[C];
#pragma unroll
  for (int c = 0; c < C; ++c) {
    rout[c] = ok ? sqrtf(G[0][c] * G[0][c] + G[1][c] * G[1][c] + G[2][c] * G[2][c]) : 0.0f;
    rsum += rout[c];
  }
  if (ok) {
    const float inv = 1.0f / norm;
    out = make_float4(sx * inv, sy * inv, sz * inv, rsum * (1.0f / (float)C));
  }
  a.nrm[p] = out;
#pragma unroll
  for (int c = 0; c < C; ++c) a.albedo[c * P + p] = rout[c];
  a.valid[p] = ok ? 1 : 0;
}

// A pixel with masked rows: the normal equations (L_v^T L_v) G_c = L_v^T I_v,c over the
// valid rows, R = L_v^T I the FP32 sum of ps_row.  A well-conditioned system (FP32
// condition number at most kRefineCond, the common case) is solved in FP32.  Otherwise
// the matrix is summed from the lights in double-float arithmetic and its inverse (by the
// adjugate) and 1-norm condition number are formed in FP64; fewer than 3 rows, a singular
// or ill-conditioned system (condition above cond_max): ok = false; and R, whose FP32
// rounding the condition number would amplify, is summed again in double-float from the
// pixel's valid rows (read again).
constexpr double kRefineCond = 16.0;
enum : int { PS_SOLVED = 0, PS_INVALID = 1, PS_NEED_FP64 = 2 };

// The FP32 part: fewer than 3 rows -> PS_INVALID; a system whose FP32 condition number
// is at most kRefineCond -> solved (PS_SOLVED); anything else -> PS_NEED_FP64.
template <int C>
__device__ __forceinline__ int ps_masked_fp32(const PSArgs &a, const float (&R)[3][C], float (&G)[3][C],
                                              unsigned long long valid) {
  if (__popcll(valid) < 3) return PS_INVALID;
  {  // the common case in FP32: a system whose FP32 condition number is at most kRefineCond is
     // certainly below cond_max in FP64 too (FP32 rounding moves it by far less than the gap),
     // so its validity is decided as in FP64, and FP32 solves it within the normal tolerance
    float m00 = 0, m01 = 0, m02 = 0, m11 = 0, m12 = 0, m22 = 0;
    for (int k = 0; k < a.K; ++k) {
      if (!((valid >> k) & 1ull)) continue;
      const float lx = a.light[k][0], ly = a.light[k][1], lz = a.light[k][2];
      m00 = fmaf(lx, lx, m00);
      m01 = fmaf(lx, ly, m01);
      m02 = fmaf(lx, lz, m02);
      m11 = fmaf(ly, ly, m11);
      m12 = fmaf(ly, lz, m12);
      m22 = fmaf(lz, lz, m22);
    }
    const float a00 = m11 * m22 - m12 * m12, a01 = m02 * m12 - m01 * m22, a02 = m01 * m12 - m02 * m11;
    const float a11 = m00 * m22 - m02 * m02, a12 = m01 * m02 - m00 * m12, a22 = m00 * m11 - m01 * m01;
    const float det = m00 * a00 + m01 * a01 + m02 * a02;
    const float nm = fmaxf(fabsf(m00) + fabsf(m01) + fabsf(m02),
                           fmaxf(fabsf(m01) + fabsf(m11) + fabsf(m12), fabsf(m02) + fabsf(m12) + fabsf(m22)));
    const float na = fmaxf(fabsf(a00) + fabsf(a01) + fabsf(a02),
                           fmaxf(fabsf(a01) + fabsf(a11) + fabsf(a12), fabsf(a02) + fabsf(a12) + fabsf(a22)));
    // cond = nm * |M^-1|_1 = nm * na / |det|; the test also keeps det away from zero; with a
    // cond_max below kRefineCond only systems well inside it take this path
    const float thr = (float)fmin(kRefineCond, 0.5 * a.cond_max);
    if (det > 0.0f && isfinite(det) && nm * na <= thr * det) {
      const float id = 1.0f / det;
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const float r0 = R[0][c], r1 = R[1][c], r2 = R[2][c];
        G[0][c] = (a00 * r0 + a01 * r1 + a02 * r2) * id;
        G[1][c] = (a01 * r0 + a11 * r1 + a12 * r2) * id;
        G[2][c] = (a02 * r0 + a12 * r1 + a22 * r2) * id;
      }
      return PS_SOLVED;
    }
  }
  return PS_NEED_FP64;
}

// The part that FP32 passed on (ps_masked_fp32): the matrix L_v^T L_v and the right-hand side
// in double-float arithmetic, the inverse (by the adjugate) and the 1-norm condition number in
// FP64; singular or above cond_max: false.  Above kRefineCond the right-hand side is summed again
// from the pixel's valid rows (read again), since the condition number would amplify the FP32
// rounding of the streaming pass's sum.  GB300's FP64 pipe is narrow, so the sums, which are
// most of the work, run on the FP32 pipes as double-float values (hi + lo, about 48 bits), built
// from error-free transformations: Knuth's two-sum and the fused-multiply-add two-product.
// Every operation is rounded on its own (the _rn intrinsics keep the compiler from fusing or
// reordering them), so the per-thread uses of these helpers give the same bits everywhere.
struct DF {
  float hi, lo;
};
__device__ __forceinline__ DF df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return DF{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ DF df_fast_two_sum(float a, float b) {  // needs |a| >= |b| (or a = 0)
  const float s = __fadd_rn(a, b);
  return DF{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ DF df_add(DF x, DF y) {
  const DF s = df_two_sum(x.hi, y.hi);
  const DF t = df_two_sum(x.lo, y.lo);
  const DF u = df_fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
  return df_fast_two_sum(u.hi, __fadd_rn(u.lo, t.lo));
}
// x * b exactly as hi + lo (two-product)
__device__ __forceinline__ DF df_prod(float x, float b) {
  const float p = __fmul_rn(x, b);
  return DF{p, __fmaf_rn(x, b, -p)};
}
__device__ __forceinline__ DF df_mul_f(DF x, float b) {
  const DF p = df_prod(x.hi, b);
  return df_fast_two_sum(p.hi, __fmaf_rn(x.lo, b, p.lo));
}
__device__ __forceinline__ double df_to_double(DF x) { return (double)x.hi + (double)x.lo; }

// Entry (u, v) of L_v^T L_v, over the valid rows in light order (each product exact).
__device__ __forceinline__ double ps_m_df(const PSArgs &a, unsigned long long valid, int u, int v) {
  DF s = {0.0f, 0.0f};
  for (int k = 0; k < a.K; ++k)
    if ((valid >> k) & 1ull) s = df_add(s, df_prod(a.light[k][u], a.light[k][v]));
  return df_to_double(s);
}
// the six entries m00 m01 m02 m11 m12 m22
__device__ __constant__ const int kMu[6] = {0, 0, 0, 1, 1, 2};
__device__ __constant__ const int kMv[6] = {0, 1, 2, 1, 2, 2};

// Inverse (m00 m01 m02 m11 m12 m22 layout) and 1-norm condition number; false when the
// system is singular or above cond_max.
__device__ __forceinline__ bool ps_inv64(const PSArgs &a, const double (&M)[6], double (&I)[6], double &cond) {
  const double M00 = M[0], M01 = M[1], M02 = M[2], M11 = M[3], M12 = M[4], M22 = M[5];
  const double A00 = M11 * M22 - M12 * M12, A01 = M02 * M12 - M01 * M22, A02 = M01 * M12 - M02 * M11;
  const double A11 = M00 * M22 - M02 * M02, A12 = M01 * M02 - M00 * M12, A22 = M00 * M11 - M01 * M01;
  const double det = M00 * A00 + M01 * A01 + M02 * A02;
  if (!(det != 0.0) || !isfinite(det)) return false;
  const double id = 1.0 / det;
  I[0] = A00 * id;
  I[1] = A01 * id;
  I[2] = A02 * id;
  I[3] = A11 * id;
  I[4] = A12 * id;
  I[5] = A22 * id;
  const double nM = fmax(fabs(M00) + fabs(M01) + fabs(M02),
                         fmax(fabs(M01) + fabs(M11) + fabs(M12), fabs(M02) + fabs(M12) + fabs(M22)));
  const double nI = fmax(fabs(I[0]) + fabs(I[1]) + fabs(I[2]),
                         fmax(fabs(I[1]) + fabs(I[3]) + fabs(I[4]), fabs(I[2]) + fabs(I[4]) + fabs(I[5])));
  cond = nM * nI;
  return cond <= a.cond_max;
}

template <int C, typename TI>
__device__ __forceinline__ bool ps_masked_fp64(const PSArgs &a, int p, const float (&R)[3][C], float (&G)[3][C],
                                               unsigned long long valid) {
  double M[6], I[6], cond;
#pragma unroll
  for (int e = 0; e < 6; ++e) M[e] = ps_m_df(a, valid, kMu[e], kMv[e]);
  if (!ps_inv64(a, M, I, cond)) return false;
  double Rd[3][C];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < C; ++c) Rd[r][c] = R[r][c];
  if (cond > kRefineCond) {  // ill-conditioned: the right-hand side again, in double-float
    const TI *img = reinterpret_cast<const TI *>(a.images);
    const size_t P = (size_t)a.P;
    float rho[C];
#pragma unroll
    for (int c = 0; c < C; ++c) rho[c] = a.zero_indirect ? 0.0f : a.albedo[c * P + p];
    DF Rf[3][C];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < C; ++c) Rf[r][c] = DF{0.0f, 0.0f};
    for (int k = 0; k < a.K; ++k) {
      if (!((valid >> k) & 1ull)) continue;
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const size_t o = ((size_t)k * C + c) * P + p;
        const float a0 = load_img<TI>(img + o);
        const float lb = a.zero_indirect ? 0.0f : __ldg(a.lbar + o);
        // I = a0 - rho lb: rho lb = q.hi + q.lo exactly, then two exact-error subtractions
        const DF q = df_prod(rho[c], lb);
        const DF d = df_two_sum(a0, -q.hi);
        const DF iv = df_two_sum(d.hi, __fsub_rn(d.lo, q.lo));
#pragma unroll
        for (int r = 0; r < 3; ++r) Rf[r][c] = df_add(Rf[r][c], df_mul_f(iv, a.light[k][r]));
      }
    }
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < C; ++c) Rd[r][c] = df_to_double(Rf[r][c]);
  }
#pragma unroll
  for (int c = 0; c < C; ++c) {
    G[0][c] = (float)(I[0] * Rd[0][c] + I[1] * Rd[1][c] + I[2] * Rd[2][c]);
    G[1][c] = (float)(I[1] * Rd[0][c] + I[3] * Rd[1][c] + I[4] * Rd[2][c]);
    G[2][c] = (float)(I[2] * Rd[0][c] + I[4] * Rd[1][c] + I[5] * Rd[2][c]);
  }
  return true;
}

template <int C, typename TI>
__device__ __forceinline__ bool ps_masked_solve(const PSArgs &a, int p, const float (&R)[3][C], float (&G)[3][C],
                                                unsigned long long valid) {
  const int st = ps_masked_fp32<C>(a, R, G, valid);
  if (st != PS_NEED_FP64) return st == PS_SOLVED;
  return ps_masked_fp64<C, TI>(a, p, R, G, valid);
}

// The rest of pixel p once every row is in: the masked solve when some row is masked
// (else G as summed, or from R in the normal-equation form), then the stored normal,
// albedo and validity.
template <int C, typename TI, bool NE>
__device__ __forceinline__ void ps_finish(const PSArgs &a, int p, const float (&R)[3][C], float (&G)[3][C],
                                          unsigned long long valid) {
  const unsigned long long all = a.K == 64 ? ~0ull : ((1ull << a.K) - 1ull);
  bool ok = true;
  if (valid != all) ok = ps_masked_solve<C, TI>(a, p, R, G, valid);
  else if (NE) ps_apply_minv<C>(a, R, G);
  ps_store<C>(a, p, G, ok);
}

template <int C, typename TI, bool NE>
__device__ __forceinline__ void ps_pixel_t(const PSArgs &a, int p) {
  const TI *img = reinterpret_cast<const TI *>(a.images);
  const size_t P = (size_t)a.P;
  float rho[C];
#pragma unroll
  for (int c = 0; c < C; ++c) rho[c] = a.zero_indirect ? 0.0f : a.albedo[c * P + p];
  float G[3][C], R[3][C];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < C; ++c) G[r][c] = R[r][c] = 0.0f;
  unsigned long long valid = 0;
  for (int k = 0; k < a.K; ++k) {
    float a0[C], lb[C];
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const size_t o = ((size_t)k * C + c) * P + p;
      a0[c] = load_img<TI>(img + o);
      lb[c] = a.zero_indirect ? 0.0f : __ldg(a.lbar + o);
    }
    ps_row<C, NE>(a, k, rho, a0, lb, G, R, valid);
  }
  ps_finish<C, TI, NE>(a, p, R, G, valid);
}

template <int C, typename TI>
__device__ __forceinline__ void ps_pixel(const PSArgs &a, int p) {
  if (a.normal_eq)
    ps_pixel_t<C, TI, true>(a, p);
  else
    ps_pixel_t<C, TI, false>(a, p);
}

// The single-object form in two kernels, so that the common path stays small (few
// registers, many resident threads, several pixels' loads in flight per thread):
//   k_ps_fast: V consecutive pixels per thread (P a multiple of V, so that every
//     plane row is 4V-byte aligned; one vector load per plane row for all V), the
//     FP32 contraction and row masks; a pixel with every row valid is stored, and so
//     is a masked one whose system FP32 settles (ps_masked_fp32); the rest go to a
//     list with their row masks and right-hand sides;
//   k_ps_masked: the rest of the listed pixels' solves (ps_masked_fp64).
// Per pixel the arithmetic is that of ps_pixel, so both forms give the same bits.

template <typename TI, int V>
struct VecLoad;
template <>
struct VecLoad<float, 1> {
  static __device__ __forceinline__ void get(const float *p, float (&v)[1]) { v[0] = __ldg(p); }
};
template <>
struct VecLoad<float, 2> {
  static __device__ __forceinline__ void get(const float *p, float (&v)[2]) {
    const float2 x = __ldg(reinterpret_cast<const float2 *>(p));
    v[0] = x.x;
    v[1] = x.y;
  }
};
template <>
struct VecLoad<float, 4> {
  static __device__ __forceinline__ void get(const float *p, float (&v)[4]) {
    const float4 x = __ldg(reinterpret_cast<const float4 *>(p));
    v[0] = x.x;
    v[1] = x.y;
    v[2] = x.z;
    v[3] = x.w;
  }
};
template <>
struct VecLoad<__half, 1> {
  static __device__ __forceinline__ void get(const __half *p, float (&v)[1]) { v[0] = __half2float(__ldg(p)); }
};
template <>
struct VecLoad<__half, 2> {
  static __device__ __forceinline__ void get(const __half *p, float (&v)[2]) {
    const float2 x = __half22float2(__ldg(reinterpret_cast<const __half2 *>(p)));
    v[0] = x.x;
    v[1] = x.y;
  }
};
template <>
struct VecLoad<__half, 4> {
  static __device__ __forceinline__ void get(const __half *p, float (&v)[4]) {
    const uint2 x = __ldg(reinterpret_cast<const uint2 *>(p));
    const float2 lo = __half22float2(*reinterpret_cast<const __half2 *>(&x.x));
    const float2 hi = __half22float2(*reinterpret_cast<const __half2 *>(&x.y));
    v[0] = lo.x;
    v[1] = lo.y;
    v[2] = hi.x;
    v[3] = hi.y;
  }
};

struct PSList {
  int *pix;                  // masked pixels
  unsigned long long *mask;  // their row masks
  float *rhs;                // their right-hand sides R = L_v^T I, 9 floats each (3 x C used)
  unsigned *count;           // entries (zero before the launch)
};

#ifndef IRTPS_PS_MINB
#define IRTPS_PS_MINB 4
#endif
#ifndef IRTPS_PS_KUNROLL
#define IRTPS_PS_KUNROLL 4
#endif
// resident blocks per SM asked of the normal-equation form (its state fits 64 registers at V <= 2)
constexpr int kPsMinBlocks = IRTPS_PS_MINB;
// lights per unrolled step of the streaming loop, over all V pixels of a thread
constexpr int kPsKUnroll = IRTPS_PS_KUNROLL;

template <int C, typename TI, int V, bool NE>
__global__ void __launch_bounds__(256, (NE && V < 4) ? kPsMinBlocks : 2) k_ps_fast(const PSArgs a, const PSList L) {
  const int p = (blockIdx.x * blockDim.x + threadIdx.x) * V;
  const bool in = p < a.P;
  const TI *img = reinterpret_cast<const TI *>(a.images);
  const size_t P = (size_t)a.P;
  float rho[V][C];
  float G[V][3][C], R[V][3][C];
  unsigned long long valid[V];
#pragma unroll
  for (int j = 0; j < V; ++j) {
    valid[j] = 0;
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < C; ++c) G[j][r][c] = R[j][r][c] = 0.0f;
  }
  if (in) {
#pragma unroll
    for (int c = 0; c < C; ++c) {
      float v[V];
#pragma unroll
      for (int j = 0; j < V; ++j) v[j] = 0.0f;
      if (!a.zero_indirect) VecLoad<float, V>::get(a.albedo + c * P + p, v);
#pragma unroll
      for (int j = 0; j < V; ++j) rho[j][c] = v[j];
    }
#pragma unroll(kPsKUnroll / V > 0 ? kPsKUnroll / V : 1)
    for (int k = 0; k < a.K; ++k) {
      float a0[C][V], lb[C][V];
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const size_t o = ((size_t)k * C + c) * P + p;
        VecLoad<TI, V>::get(img + o, a0[c]);
        if (a.zero_indirect) {
#pragma unroll
          for (int j = 0; j < V; ++j) lb[c][j] = 0.0f;
        } else {
          VecLoad<float, V>::get(a.lbar + o, lb[c]);
        }
      }
#pragma unroll
      for (int j = 0; j < V; ++j) {
        float x0[C], x1[C];
#pragma unroll
        for (int c = 0; c < C; ++c) {
          x0[c] = a0[c][j];
          x1[c] = lb[c][j];
        }
        ps_row<C, NE>(a, k, rho[j], x0, x1, G[j], R[j], valid[j]);
      }
    }
  }
  const unsigned long long all = a.K == 64 ? ~0ull : ((1ull << a.K) - 1ull);
#pragma unroll
  for (int j = 0; j < V; ++j) {
    bool masked = false;
    if (in) {
      if (valid[j] == all) {
        if (NE) ps_apply_minv<C>(a, R[j], G[j]);
        ps_store<C>(a, p + j, G[j], true);
      } else {
        const int st = ps_masked_fp32<C>(a, R[j], G[j], valid[j]);
        if (st != PS_NEED_FP64) ps_store<C>(a, p + j, G[j], st == PS_SOLVED);
        masked = st == PS_NEED_FP64;
      }
    }
    // pixels left for the list kernel, appended with one atomic per warp
    const unsigned mm = __ballot_sync(0xffffffffu, masked);
    if (mm) {
      const int lane = threadIdx.x & 31, leader = __ffs(mm) - 1;
      unsigned base = 0;
      if (lane == leader) base = atomicAdd(L.count, (unsigned)__popc(mm));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (masked) {
        const unsigned i = base + __popc(mm & ((1u << lane) - 1u));
        L.pix[i] = p + j;
        L.mask[i] = valid[j];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
          for (int c = 0; c < C; ++c) L.rhs[(size_t)i * 9 + r * C + c] = R[j][r][c];
      }
    }
  }
}

// The listed pixels, one per thread (the FP64 pipe is narrow: a pixel's FP64 work stays in
// one lane), a grid-stride loop over the list.
template <int C, typename TI>
__global__ void __launch_bounds__(128) k_ps_masked(const PSArgs a, const PSList L) {
  const unsigned n = *L.count;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int p = L.pix[i];
    float R[3][C], G[3][C] = {};
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < C; ++c) R[r][c] = L.rhs[(size_t)i * 9 + r * C + c];
    const bool ok = ps_masked_fp64<C, TI>(a, p, R, G, L.mask[i]);
    ps_store<C>(a, p, G, ok);
  }
}

// Batched: the blocks of object o are [objs[o].blk_begin, objs[o + 1].blk_begin).
template <int C, typename TI>
__global__ void __launch_bounds__(256) k_ps_b(const PSArgs *__restrict__ objs, int n) {
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
  const PSArgs &a = objs[s_o];
  const int p = ((int)blockIdx.x - a.blk_begin) * blockDim.x + threadIdx.x;
  if (p < a.P) ps_pixel<C, TI>(a, p);
}

// ---------------------------------------------------------------------------
// Tensor-core form of the contraction (option ps_tensor = 1).  A tile of 128
// pixels is one [128 x KCp] x [KCp x 16] product on tcgen05: row p holds the
// corrected values I(p, kk), kk = k C + c (the image layout's own plane index),
// and column n = r C + c of the right operand holds pinv(L)[r][k] where the
// channels agree (zero elsewhere), so that the accumulator row p is
// G(p)[r][c] = sum_k pinv[r][k] I(p, k, c) (Eq. 4).  Split precision: I and
// pinv are each a BF16 pair hi + lo (hi = bf16(x), lo = bf16(x - hi)); the chain
// I_hi P_hi + I_lo P_hi + I_hi P_lo accumulates in FP32 in tensor memory (the
// dropped I_lo P_lo is below 2^-16 of the product).  Row masks are decided in
// FP32 from I exactly as in k_ps_fast, and masked pixels take the same masked solve.
//
// Shared-memory operands use the canonical K-major layout without swizzle:
// 8-row x 16-byte core matrices, the 16 core matrices of one 8-wide K column
// of the 128 rows contiguous (stride 128 B between row groups), 2 KB between K
// columns; segment hi, then lo.  One thread issues the MMAs; their completion
// arrives on an mbarrier that all threads wait on (bounded), then each warp reads
// its 32 accumulator rows from tensor memory.
// ---------------------------------------------------------------------------
constexpr int kTcRows = 128;                 // M: pixels per tile, one per thread
constexpr int kTcN = 16;                     // N: outputs (r, c), 3 C used
constexpr int kTcSlack = 0;                  // spare shared memory after the operands
constexpr long long kTcWaitPolls = 1ll << 22;  // bound of the MMA-completion wait

// K*C padded: a multiple of 16 (the MMA's K) and of the fill chunk (24 for C = 3, 8 for C = 1).
__host__ __device__ inline int tc_kcp(int K, int C) {
  const int q = C == 3 ? 48 : 16;
  return (K * C + q - 1) / q * q;
}
inline size_t tc_smem_bytes(int K, int C) {
  const int kcp = tc_kcp(K, C);
  return (size_t)512 * kcp + (size_t)64 * kcp + kTcSlack + 64;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start, leading (K-direction) and stride (row-group) byte offsets.
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B (both K-major), N = 16, M = 128.
constexpr uint32_t kTcIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTcN >> 3) << 17) |
                              ((uint32_t)(kTcRows >> 4) << 24);

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(kTcIdesc), "r"(acc));
}

__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity) {
  for (long long i = 0; i < kTcWaitPolls; ++i) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t *>(&v);
}

// x -> (hi, lo) in BF16, hi = bf16(x), lo = bf16(x - hi)
__device__ __forceinline__ void split_bf16(float x, float &hi, float &lo) {
  hi = __bfloat162float(__float2bfloat16_rn(x));
  lo = __bfloat162float(__float2bfloat16_rn(x - hi));
}

template <int C, typename TI>
__global__ void __launch_bounds__(kTcRows) k_ps_tc(const PSArgs a, unsigned long long *err) {
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  const int kc = a.K * C, kcp = tc_kcp(a.K, C), ncol = kcp / 8;
  unsigned char *As = tc_smem;                            // 2 segments x ncol x 2 KB
  unsigned char *Bs = tc_smem + (size_t)512 * kcp;        // 2 segments x ncol x 256 B
  uint64_t *mbar = reinterpret_cast<uint64_t *>(Bs + (size_t)64 * kcp + kTcSlack);
  uint32_t *s_tmem = reinterpret_cast<uint32_t *>(mbar + 1);
  int *s_fail = reinterpret_cast<int *>(mbar + 2);
  const int tid = threadIdx.x, warp = tid >> 5;

  // operands: zero A (its padding columns stay zero); B = pinv(L) per channel, hi and lo
  for (int i = tid; i < 128 * kcp / 4; i += kTcRows) reinterpret_cast<uint32_t *>(As)[i] = 0u;
  for (int i = tid; i < 2 * ncol * kTcN; i += kTcRows) {
    const int seg = i / (ncol * kTcN), rem = i - seg * ncol * kTcN, q = rem / kTcN, n = rem - q * kTcN;
    float v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int kk = 8 * q + e;
      float x = 0.0f;
      if (kk < kc && n < 3 * C && (n % C) == (kk % C)) x = a.pinv[n / C][kk / C];
      float hi, lo;
      split_bf16(x, hi, lo);
      v[e] = seg == 0 ? hi : lo;
    }
    uint4 w = make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]), pack_bf16(v[6], v[7]));
    *reinterpret_cast<uint4 *>(Bs + (size_t)(seg * ncol + q) * 256 + (n >> 3) * 128 + (n & 7) * 16) = w;
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *s_fail = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(smem_u32(s_tmem))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *s_tmem;

  const TI *img = reinterpret_cast<const TI *>(a.images);
  const size_t P = (size_t)a.P;
  const int n_tiles = (a.P + kTcRows - 1) / kTcRows;
  constexpr int CH = C == 3 ? 24 : 8;  // values per fill step: whole lights and whole core columns
  uint32_t phase = 0;
  for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int p = tile * kTcRows + tid;
    const bool in = p < a.P;
    float rho[C];
#pragma unroll
    for (int c = 0; c < C; ++c) rho[c] = (in && !a.zero_indirect) ? a.albedo[c * P + p] : 0.0f;
    unsigned long long valid = 0;
    float R[3][C];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < C; ++c) R[r][c] = 0.0f;
    unsigned char *row = As + (tid >> 3) * 128 + (tid & 7) * 16;
    for (int q0 = 0; q0 < kcp; q0 += CH) {
      float I[CH];
#pragma unroll
      for (int e = 0; e < CH; ++e) {
        const int kk = q0 + e;
        float a0 = 0.0f, lb = 0.0f;
        if (in && kk < kc) {
          a0 = load_img<TI>(img + (size_t)kk * P + p);
          if (!a.zero_indirect) lb = __ldg(a.lbar + (size_t)kk * P + p);
        }
        I[e] = __fsub_rn(a0, __fmul_rn(rho[e % C], lb));
      }
      // row masks in FP32 and the masked system's right-hand side, as in ps_row
#pragma unroll
      for (int e = 0; e < CH; e += C) {
        const int k = (q0 + e) / C;
        float chat = I[e];
        if (C == 3) chat = __fdiv_rn(__fadd_rn(__fadd_rn(I[e], I[e + 1]), I[e + 2]), 3.0f);
        const bool ok = q0 + e < kc && chat > a.tau_lo && chat < a.tau_hi;
        if (ok) valid |= 1ull << k;
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          const float l = ok ? a.light[k][r] : 0.0f;
#pragma unroll
          for (int c = 0; c < C; ++c) R[r][c] = fmaf(l, I[e + c], R[r][c]);
        }
      }
#pragma unroll
      for (int g = 0; g < CH / 8; ++g) {
        float hi[8], lo[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) split_bf16(I[8 * g + e], hi[e], lo[e]);
        const int q = q0 / 8 + g;
        *reinterpret_cast<uint4 *>(row + (size_t)q * 2048) =
            make_uint4(pack_bf16(hi[0], hi[1]), pack_bf16(hi[2], hi[3]), pack_bf16(hi[4], hi[5]),
                       pack_bf16(hi[6], hi[7]));
        *reinterpret_cast<uint4 *>(row + (size_t)(ncol + q) * 2048) =
            make_uint4(pack_bf16(lo[0], lo[1]), pack_bf16(lo[2], lo[3]), pack_bf16(lo[4], lo[5]),
                       pack_bf16(lo[6], lo[7]));
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = smem_u32(As), b0 = smem_u32(Bs);
      for (int j = 0; j < kcp / 16; ++j) {
        const uint64_t ah = umma_desc(a0 + (uint32_t)(2 * j) * 2048u, 2048u, 128u);
        const uint64_t al = umma_desc(a0 + (uint32_t)(ncol + 2 * j) * 2048u, 2048u, 128u);
        const uint64_t bh = umma_desc(b0 + (uint32_t)(2 * j) * 256u, 256u, 128u);
        const uint64_t bl = umma_desc(b0 + (uint32_t)(ncol + 2 * j) * 256u, 256u, 128u);
        umma_bf16(tmem, ah, bh, j > 0 ? 1u : 0u);
        umma_bf16(tmem, al, bh, 1u);
        umma_bf16(tmem, ah, bl, 1u);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(mbar))
                   : "memory");
    }
    const bool done = mbar_wait(smem_u32(mbar), phase);
    phase ^= 1u;
    if (!done) *s_fail = 1;
    __syncthreads();
    if (*s_fail) break;  // every thread leaves; the tensor memory is freed below
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    uint32_t d[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(d[0]), "=r"(d[1]), "=r"(d[2]), "=r"(d[3]), "=r"(d[4]), "=r"(d[5]), "=r"(d[6]), "=r"(d[7]),
          "=r"(d[8]), "=r"(d[9]), "=r"(d[10]), "=r"(d[11]), "=r"(d[12]), "=r"(d[13]), "=r"(d[14]), "=r"(d[15])
        : "r"(tmem + ((uint32_t)(warp * 32) << 16)));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    if (in) {
      float G[3][C];
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < C; ++c) G[r][c] = __uint_as_float(d[r * C + c]);
      ps_finish<C, TI, false>(a, p, R, G, valid);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
  }
  if (tid == 0 && *s_fail) atomicAdd(err, 1ull);
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(tmem) : "memory");
}

static void fill_ps_args(const Ctx &c, bool zero_indirect, PSArgs &a) {
  a.images = c.images;
  a.lbar = c.lbar;
  a.albedo = c.albedo;
  a.nrm = c.nrm;
  a.valid = c.valid;
  a.P = c.H * c.W;
  a.K = c.K;
  a.tau_lo = c.opt.tau_lo;
  a.tau_hi = c.opt.tau_hi;
  a.cond_max = c.opt.cond_max;
  a.zero_indirect = zero_indirect ? 1 : 0;
  for (int k = 0; k < c.K; ++k) {
    for (int r = 0; r < 3; ++r) {
      a.pinv[r][k] = c.h_pinv[r * c.K + k];
      a.light[k][r] = c.h_lights[3 * k + r];
    }
  }
  for (int i = 0; i < 6; ++i) a.minv[i] = c.h_minv[i];
  a.normal_eq = c.normal_eq;
  a.blk_begin = 0;
}

size_t ps_args_bytes() { return sizeof(PSArgs); }

void ps_fill_args(const Ctx &c, bool zero_indirect, int blk_begin, void *dst) {
  PSArgs a;
  fill_ps_args(c, zero_indirect, a);
  a.blk_begin = blk_begin;
  std::memcpy(dst, &a, sizeof(a));
}

cudaError_t launch_ps_batch(cudaStream_t s, int C, int dtype, const void *d_args, int n, int blocks) {
  const PSArgs *a = (const PSArgs *)d_args;
  if (C == 1) {
    if (dtype == IRTPS_F16)
      k_ps_b<1, __half><<<blocks, 256, 0, s>>>(a, n);
    else
      k_ps_b<1, float><<<blocks, 256, 0, s>>>(a, n);
  } else {
    if (dtype == IRTPS_F16)
      k_ps_b<3, __half><<<blocks, 256, 0, s>>>(a, n);
    else
      k_ps_b<3, float><<<blocks, 256, 0, s>>>(a, n);
  }
  return cudaGetLastError();
}

template <int C, typename TI>
static cudaError_t launch_ps_tc_t(Ctx &c, const PSArgs &a) {
  const size_t smem = tc_smem_bytes(c.K, C);
  cudaError_t e = cudaFuncSetAttribute(k_ps_tc<C, TI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // CTAs per SM from the shared-memory fit (the operands are most of a CTA's footprint; the
  // occupancy query answered one for this kernel).  The CTAs never wait on one another, and 4 of
  // them hold 128 of an SM's 512 tensor-memory columns, so any grid size is safe.
  e = cudaFuncSetAttribute(k_ps_tc<C, TI>, cudaFuncAttributePreferredSharedMemoryCarveout,
                           (int)cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  int dev = 0, smem_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) != cudaSuccess)
    return e;
  const int fit = std::max(1, std::min(4, smem_sm / (int)(smem + 1024)));
  const int tiles = (a.P + kTcRows - 1) / kTcRows;
  int blocks = fit * (c.sms > 0 ? c.sms : 1);
  if (blocks > tiles) blocks = tiles;
  k_ps_tc<C, TI><<<blocks, kTcRows, smem, c.stream>>>(a, c.dstats->counts + 6);
  return cudaGetLastError();
}

template <int C, typename TI, bool NE>
static void launch_ps_fast(Ctx &c, const PSArgs &a, const PSList &L, int v, unsigned blocks) {
  if (v == 4)
    k_ps_fast<C, TI, 4, NE><<<blocks, 256, 0, c.stream>>>(a, L);
  else if (v == 2)
    k_ps_fast<C, TI, 2, NE><<<blocks, 256, 0, c.stream>>>(a, L);
  else
    k_ps_fast<C, TI, 1, NE><<<blocks, 256, 0, c.stream>>>(a, L);
}

template <int C, typename TI>
static cudaError_t launch_ps_split(Ctx &c, const PSArgs &a) {
  const PSList L{c.ps_pix, c.ps_mask, c.ps_rhs, c.ps_count};
  cudaError_t e = cudaMemsetAsync(c.ps_count, 0, sizeof(unsigned), c.stream);
  if (e != cudaSuccess) return e;
  const int v = ps_vec_for(c);
  const int n = (a.P + v - 1) / v;
  const unsigned blocks = (unsigned)((n + 255) / 256);
  if (a.normal_eq)
    launch_ps_fast<C, TI, true>(c, a, L, v, blocks);
  else
    launch_ps_fast<C, TI, false>(c, a, L, v, blocks);
  // the listed pixels (few: ill-conditioned masked systems), a grid-stride loop over the list
  const int cap = 4 * (c.sms > 0 ? c.sms : 1);
  const unsigned mblocks = (unsigned)std::min<long long>(cap, ((long long)a.P + 127) / 128);
  k_ps_masked<C, TI><<<mblocks, 128, 0, c.stream>>>(a, L);
  return cudaGetLastError();
}

cudaError_t launch_ps(Ctx &c, bool zero_indirect) {
  PSArgs a;
  fill_ps_args(c, zero_indirect, a);
  if (c.opt.ps_tensor) {
    ++c.stats.launches;
    if (c.C == 1)
      return c.images_dtype == IRTPS_F16 ? launch_ps_tc_t<1, __half>(c, a) : launch_ps_tc_t<1, float>(c, a);
    return c.images_dtype == IRTPS_F16 ? launch_ps_tc_t<3, __half>(c, a) : launch_ps_tc_t<3, float>(c, a);
  }
  c.stats.launches += 2;
  if (c.C == 1)
    return c.images_dtype == IRTPS_F16 ? launch_ps_split<1, __half>(c, a) : launch_ps_split<1, float>(c, a);
  return c.images_dtype == IRTPS_F16 ? launch_ps_split<3, __half>(c, a) : launch_ps_split<3, float>(c, a);
}

}  // namespace irtps
