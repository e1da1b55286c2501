// Non-uniform interpolation of the holes of single-sample environment images
// (Sec. IV: with one sample per pixel some pixels get no environment value and
// are filled from their neighbours; the paper names a non-uniform interpolation
// without giving it).  Pull-push normalised convolution:
//
//   pull  level l -> l+1: a coarse pixel sums the confidences S of its (up to 4)
//         children and takes their confidence-weighted mean value; its own
//         confidence is min(S, 1).  Level 0: confidence 1 at known pixels, 0 at holes.
//   push  level l+1 -> l, from the 1 x 1 level down: v <- w v + (1 - w) u, with w
//         the pixel's confidence and u the 2x linear upsampling of the finished
//         coarser level (fine centre i at coarse coordinate i/2 - 1/4: taps
//         (i/2 - 1, i/2) with weights (1/4, 3/4) for even i, ((i-1)/2, (i+1)/2) with
//         (3/4, 1/4) for odd i, clamped at the border).
//
// Level 0 is the caller's K x C x H x W image stack itself: the pull reads it, the
// last push writes the holes only, so known pixels keep their bits; images without
// a known pixel (confidence 0 at the top) stay as they are.  Every pass is one
// grid-stride launch over all K images of one level, HBM-bound at level 0 (the
// stack is read once by the first pull and the holes written once by the last
// push) and L2-resident above it (the coarser levels together hold a third of a
// level-0 image stack).  FP32 throughout.
#include <algorithm>
#include <cstdint>

#include "irtps_internal.h"

namespace irtps {

FillPyramid fill_pyramid(int H, int W) {
  FillPyramid py;
  py.n = 1;
  py.h[0] = H;
  py.w[0] = W;
  py.off[0] = 0;
  size_t total = 0;
  while (py.h[py.n - 1] > 1 || py.w[py.n - 1] > 1) {
    const int l = py.n++;
    py.h[l] = (py.h[l - 1] + 1) / 2;
    py.w[l] = (py.w[l - 1] + 1) / 2;
    py.off[l] = total;
    total += (size_t)py.h[l] * py.w[l];
  }
  py.total = total;
  return py;
}

namespace {

constexpr int kFillThreads = 256;

unsigned fill_blocks(size_t n, int sms) {
  const size_t want = (n + kFillThreads - 1) / kFillThreads;
  const size_t cap = (size_t)(sms > 0 ? sms : 152) * 8;
  return (unsigned)std::max<size_t>(1, std::min(want, cap));
}

// level l (h x w; values v, confidences cw, or the hole mask at level 0) -> level
// l+1 (h2 x w2).  Children summed in the order (0,0), (1,0), (0,1), (1,1).
template <int C>
__global__ void k_pull(const float *__restrict__ v, const float *__restrict__ cw, const uint8_t *__restrict__ holes,
                       int K, int h, int w, float *__restrict__ v2, float *__restrict__ cw2, int h2, int w2) {
  const size_t P = (size_t)h * w, P2 = (size_t)h2 * w2, n = (size_t)K * P2;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(t / P2);
    const int q = (int)(t - (size_t)k * P2);
    const int I = q / w2, J = q - I * w2;
    float s = 0.0f, sv[C];
#pragma unroll
    for (int c = 0; c < C; ++c) sv[c] = 0.0f;
#pragma unroll
    for (int dj = 0; dj < 2; ++dj)
#pragma unroll
      for (int di = 0; di < 2; ++di) {
        const int i = 2 * I + di, j = 2 * J + dj;
        if (i >= h || j >= w) continue;
        const size_t e = (size_t)i * w + j;
        const float a = holes ? (holes[(size_t)k * P + e] ? 0.0f : 1.0f) : cw[(size_t)k * P + e];
        if (a == 0.0f) continue;
        s += a;
#pragma unroll
        for (int c = 0; c < C; ++c) sv[c] = fmaf(a, v[((size_t)k * C + c) * P + e], sv[c]);
      }
#pragma unroll
    for (int c = 0; c < C; ++c) v2[((size_t)k * C + c) * P2 + q] = s > 0.0f ? sv[c] / s : 0.0f;
    cw2[(size_t)k * P2 + q] = fminf(s, 1.0f);
  }
}

__device__ __forceinline__ void up_taps(int i, int n2, int &lo, int &hi, float &wlo) {
  const bool even = (i & 1) == 0;
  lo = even ? (i >> 1) - 1 : (i - 1) >> 1;
  hi = lo + 1;
  wlo = even ? 0.25f : 0.75f;
  lo = min(max(lo, 0), n2 - 1);
  hi = min(max(hi, 0), n2 - 1);
}

// level l+1 (h2 x w2, finished values u) -> level l (h x w).  Above level 0 the
// level's values v are blended in place with confidences cw; at level 0 (holes
// set) only the holes are written, and only in images whose top confidence top[k]
// is above 0.
template <int C>
__global__ void k_push(const float *__restrict__ u, int h2, int w2, float *__restrict__ v,
                       const float *__restrict__ cw, const uint8_t *__restrict__ holes,
                       const float *__restrict__ top, int K, int h, int w) {
  const size_t P = (size_t)h * w, P2 = (size_t)h2 * w2, n = (size_t)K * P;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(t / P);
    const int e = (int)(t - (size_t)k * P);
    float a = 0.0f;
    if (holes) {
      if (!holes[t] || top[k] == 0.0f) continue;
    } else {
      a = cw[t];
    }
    const int i = e / w, j = e - i * w;
    int y0, y1, x0, x1;
    float a0, b0;
    up_taps(i, h2, y0, y1, a0);
    up_taps(j, w2, x0, x1, b0);
    const float a1 = 1.0f - a0, b1 = 1.0f - b0;
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const float *uc = u + ((size_t)k * C + c) * P2;
      const float up = a0 * (b0 * uc[(size_t)y0 * w2 + x0] + b1 * uc[(size_t)y0 * w2 + x1]) +
                       a1 * (b0 * uc[(size_t)y1 * w2 + x0] + b1 * uc[(size_t)y1 * w2 + x1]);
      float *vc = v + ((size_t)k * C + c) * P + e;
      *vc = holes ? up : a * *vc + (1.0f - a) * up;
    }
  }
}

template <int C>
cudaError_t interpolate_c(cudaStream_t s, float *values, const uint8_t *holes, int K, const FillPyramid &py,
                          float *v_scr, float *w_scr, int sms, int &launches) {
  auto lv = [&](int l) -> float * { return l == 0 ? values : v_scr + (size_t)K * C * py.off[l]; };
  auto lw = [&](int l) -> float * { return l == 0 ? nullptr : w_scr + (size_t)K * py.off[l]; };
  for (int l = 0; l + 1 < py.n; ++l) {
    const size_t n = (size_t)K * py.h[l + 1] * py.w[l + 1];
    k_pull<C><<<fill_blocks(n, sms), kFillThreads, 0, s>>>(lv(l), lw(l), l == 0 ? holes : nullptr, K, py.h[l],
                                                          py.w[l], lv(l + 1), lw(l + 1), py.h[l + 1], py.w[l + 1]);
    ++launches;
  }
  const float *top = lw(py.n - 1);
  for (int l = py.n - 2; l >= 0; --l) {
    const size_t n = (size_t)K * py.h[l] * py.w[l];
    k_push<C><<<fill_blocks(n, sms), kFillThreads, 0, s>>>(lv(l + 1), py.h[l + 1], py.w[l + 1], lv(l), lw(l),
                                                          l == 0 ? holes : nullptr, top, K, py.h[l], py.w[l]);
    ++launches;
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_interpolate_holes(cudaStream_t s, float *values, const uint8_t *holes, int K, int C,
                                     const FillPyramid &py, float *v_scr, float *w_scr, int sms, int &launches) {
  if (py.n < 2) return cudaSuccess;  // a 1 x 1 image: a hole has no neighbour to take a value from
  return C == 1 ? interpolate_c<1>(s, values, holes, K, py, v_scr, w_scr, sms, launches)
                : interpolate_c<3>(s, values, holes, K, py, v_scr, w_scr, sms, launches);
}

}  // namespace irtps
