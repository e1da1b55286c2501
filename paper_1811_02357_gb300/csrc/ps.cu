// Image correction and photometric stereo (Sec. III Eq. 3-4; Sec. IV stage 5).
//
// Per pixel p: I(k, c) = A0(k, c, p) - rho_t(c, p) * Lbar(k, c, p); row k is valid
// iff tau_lo < mean_c I(k, c) < tau_hi (decided in FP32, each operation rounded
// on its own).  All rows valid: G_c = pinv(L) I_c with pinv(L) = (L^T L)^-1 L^T
// (Eq. 4).  Otherwise the FP64 normal equations (L_v^T L_v) G_c = L_v^T I_v,c over
// the valid rows; fewer than 3 rows or a 1-norm condition number above cond_max
// marks the pixel invalid.  n = normalize(sum_c G_c), rho_c = |G_c|; invalid
// pixels get n = (0, 0, 1), rho = 0.
//
// The contraction pinv(L) [3 x K] x I [K x C*P] streams K*C values per pixel for
// 6*K*C flops: far below the tensor-core ridge, so it runs on the FP32 pipes
// with coalesced [k][c][p] loads and the pixel's state written once.
#include <cstdint>
#include <cstring>
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
  int blk_begin;        // first block of the object in a batched launch
};

template <typename TI>
__device__ __forceinline__ float load_img(const TI *p);
template <>
__device__ __forceinline__ float load_img<float>(const float *p) { return __ldg(p); }
template <>
__device__ __forceinline__ float load_img<__half>(const __half *p) { return __half2float(__ldg(p)); }

template <int C, typename TI>
__device__ __forceinline__ void ps_pixel(const PSArgs &a, int p) {
  const TI *img = reinterpret_cast<const TI *>(a.images);
  const size_t P = (size_t)a.P;
  float rho[C];
#pragma unroll
  for (int c = 0; c < C; ++c) rho[c] = a.zero_indirect ? 0.0f : a.albedo[c * P + p];
  float G[3][C];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < C; ++c) G[r][c] = 0.0f;
  unsigned long long valid = 0;
  for (int k = 0; k < a.K; ++k) {
    float I[C];
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const size_t o = ((size_t)k * C + c) * P + p;
      const float a0 = load_img<TI>(img + o);
      const float lb = a.zero_indirect ? 0.0f : __ldg(a.lbar + o);
      I[c] = __fsub_rn(a0, __fmul_rn(rho[c], lb));
    }
    float chat = I[0];
    if (C == 3) chat = __fdiv_rn(__fadd_rn(__fadd_rn(I[0], I[1]), I[2]), 3.0f);
    if (chat > a.tau_lo && chat < a.tau_hi) valid |= 1ull << k;
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < C; ++c) G[r][c] = fmaf(a.pinv[r][k], I[c], G[r][c]);
  }
  const unsigned long long all = a.K == 64 ? ~0ull : ((1ull << a.K) - 1ull);
  bool ok = true;
  if (valid != all) {
    // masked pixel: FP64 normal equations over the valid rows
    if (__popcll(valid) < 3) {
      ok = false;
    } else {
      double M00 = 0, M01 = 0, M02 = 0, M11 = 0, M12 = 0, M22 = 0;
      double R[3][C];
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < C; ++c) R[r][c] = 0.0;
      for (int k = 0; k < a.K; ++k) {
        if (!((valid >> k) & 1ull)) continue;
        const double lx = a.light[k][0], ly = a.light[k][1], lz = a.light[k][2];
        M00 += lx * lx;
        M01 += lx * ly;
        M02 += lx * lz;
        M11 += ly * ly;
        M12 += ly * lz;
        M22 += lz * lz;
#pragma unroll
        for (int c = 0; c < C; ++c) {
          const size_t o = ((size_t)k * C + c) * P + p;
          const double lb = a.zero_indirect ? 0.0 : (double)__ldg(a.lbar + o);
          const double Iv = (double)load_img<TI>(img + o) - (double)rho[c] * lb;
          R[0][c] += lx * Iv;
          R[1][c] += ly * Iv;
          R[2][c] += lz * Iv;
        }
      }
      // inverse by the adjugate; 1-norm condition number
      const double A00 = M11 * M22 - M12 * M12, A01 = M02 * M12 - M01 * M22, A02 = M01 * M12 - M02 * M11;
      const double A11 = M00 * M22 - M02 * M02, A12 = M01 * M02 - M00 * M12, A22 = M00 * M11 - M01 * M01;
      const double det = M00 * A00 + M01 * A01 + M02 * A02;
      if (!(det != 0.0) || !isfinite(det)) {
        ok = false;
      } else {
        const double id = 1.0 / det;
        const double i00 = A00 * id, i01 = A01 * id, i02 = A02 * id, i11 = A11 * id, i12 = A12 * id, i22 = A22 * id;
        const double nM = fmax(fabs(M00) + fabs(M01) + fabs(M02),
                               fmax(fabs(M01) + fabs(M11) + fabs(M12), fabs(M02) + fabs(M12) + fabs(M22)));
        const double nI = fmax(fabs(i00) + fabs(i01) + fabs(i02),
                               fmax(fabs(i01) + fabs(i11) + fabs(i12), fabs(i02) + fabs(i12) + fabs(i22)));
        const double cond = nM * nI;
        if (!(cond <= a.cond_max)) {
          ok = false;
        } else {
#pragma unroll
          for (int c = 0; c < C; ++c) {
            G[0][c] = (float)(i00 * R[0][c] + i01 * R[1][c] + i02 * R[2][c]);
            G[1][c] = (float)(i01 * R[0][c] + i11 * R[1][c] + i12 * R[2][c]);
            G[2][c] = (float)(i02 * R[0][c] + i12 * R[1][c] + i22 * R[2][c]);
          }
        }
      }
    }
  }
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

template <int C, typename TI>
__global__ void __launch_bounds__(256) k_ps(const PSArgs a) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < a.P) ps_pixel<C, TI>(a, p);
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

cudaError_t launch_ps(Ctx &c, bool zero_indirect) {
  PSArgs a;
  fill_ps_args(c, zero_indirect, a);
  const int threads = 256;
  const unsigned blocks = (unsigned)((a.P + threads - 1) / threads);
  ++c.stats.launches;
  if (c.C == 1) {
    if (c.images_dtype == IRTPS_F16)
      k_ps<1, __half><<<blocks, threads, 0, c.stream>>>(a);
    else
      k_ps<1, float><<<blocks, threads, 0, c.stream>>>(a);
  } else {
    if (c.images_dtype == IRTPS_F16)
      k_ps<3, __half><<<blocks, threads, 0, c.stream>>>(a);
    else
      k_ps<3, float><<<blocks, threads, 0, c.stream>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace irtps
