// Direct depth solve by the cosine transform (option precond = 2).  With unit
// edge weights the normal equations of the integration are A x = b with A the
// graph Laplacian of the H x W grid (Neumann boundary), the sum of the path
// Laplacians of the rows and of the columns.  The orthonormal DCT-II vectors
// diagonalise a path Laplacian of n nodes: C[k][i] = s_k cos(pi k (2i+1) / 2n),
// s_0 = sqrt(1/n), s_k = sqrt(2/n), eigenvalue 4 sin^2(pi k / 2n).  So
//
//     x = C_H^T [ (C_H B C_W^T) ./ (mu_l + nu_k) ] C_W,   the (0, 0) term dropped,
//
// B and x the H x W arrays of b and x, which is the mean-zero least-squares
// surface.  Four dense products of FP64 matrices (an H x H or W x W transform
// against the H x W data): 4 H W (H + W) multiply-adds, done by one tiled FP64
// kernel; the division by the eigenvalues is fused into the second product.
// GB300's FP64 rate bounds it (about 0.85 ms at 512 x 512), far below the
// barrier-bound multigrid PCG it replaces for unit weights at these sizes.
#include <cmath>
#include <cstdint>
#include <vector>

#include "irtps_internal.h"

namespace irtps {

namespace {

constexpr int kTile = 32;      // output tile (rows and columns)
constexpr int kTileK = 32;     // depth of one shared-memory stage
constexpr int kGemmThreads = 256;

// D = op(A) op(B), M x N, inner dimension K; op(A)(m, k) = TA ? A[k lda + m] : A[m lda + k],
// op(B)(k, n) = TB ? B[n ldb + k] : B[k ldb + n].  SCALE: D(m, n) /= mu[m] + nu[n], D(0, 0) = 0.
template <bool TA, bool TB, bool SCALE>
__global__ void __launch_bounds__(kGemmThreads) k_dgemm(int M, int N, int K, const double *__restrict__ A, int lda,
                                                         const double *__restrict__ B, int ldb,
                                                         double *__restrict__ D, int ldd,
                                                         const double *__restrict__ mu,
                                                         const double *__restrict__ nu) {
  __shared__ double As[kTileK][kTile + 1];
  __shared__ double Bs[kTileK][kTile + 1];
  const int m0 = blockIdx.y * kTile, n0 = blockIdx.x * kTile;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;  // 2 x 2 outputs per thread
  double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
  for (int k0 = 0; k0 < K; k0 += kTileK) {
#pragma unroll
    for (int r = 0; r < (kTile * kTileK) / kGemmThreads; ++r) {
      const int e = threadIdx.x + r * kGemmThreads;
      // A tile: the contiguous index of the source runs fastest across the threads
      int mm, kk;
      if (TA) { kk = e / kTile; mm = e - kk * kTile; } else { mm = e / kTileK; kk = e - mm * kTileK; }
      const int gm = m0 + mm, gk = k0 + kk;
      As[kk][mm] = (gm < M && gk < K) ? (TA ? A[(size_t)gk * lda + gm] : A[(size_t)gm * lda + gk]) : 0.0;
      int nn;
      if (TB) { nn = e / kTileK; kk = e - nn * kTileK; } else { kk = e / kTile; nn = e - kk * kTile; }
      const int gn = n0 + nn, gk2 = k0 + kk;
      Bs[kk][nn] = (gn < N && gk2 < K) ? (TB ? B[(size_t)gn * ldb + gk2] : B[(size_t)gk2 * ldb + gn]) : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < kTileK; ++kk) {
      const double a0 = As[kk][2 * ty], a1 = As[kk][2 * ty + 1];
      const double b0 = Bs[kk][2 * tx], b1 = Bs[kk][2 * tx + 1];
      acc[0][0] = fma(a0, b0, acc[0][0]);
      acc[0][1] = fma(a0, b1, acc[0][1]);
      acc[1][0] = fma(a1, b0, acc[1][0]);
      acc[1][1] = fma(a1, b1, acc[1][1]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int m = m0 + 2 * ty + a, n = n0 + 2 * tx + b;
      if (m >= M || n >= N) continue;
      double v = acc[a][b];
      if (SCALE) v = (m == 0 && n == 0) ? 0.0 : v / (mu[m] + nu[n]);
      D[(size_t)m * ldd + n] = v;
    }
}

template <bool TA, bool TB, bool SCALE>
void gemm(cudaStream_t s, int M, int N, int K, const double *A, int lda, const double *B, int ldb, double *D,
          int ldd, const double *mu = nullptr, const double *nu = nullptr) {
  const dim3 grid((N + kTile - 1) / kTile, (M + kTile - 1) / kTile);
  k_dgemm<TA, TB, SCALE><<<grid, kGemmThreads, 0, s>>>(M, N, K, A, lda, B, ldb, D, ldd, mu, nu);
}

void dct_matrix(int n, double *c) {
  const double pi = 3.14159265358979323846;
  for (int k = 0; k < n; ++k) {
    const double s = k == 0 ? std::sqrt(1.0 / n) : std::sqrt(2.0 / n);
    for (int i = 0; i < n; ++i) c[(size_t)k * n + i] = s * std::cos(pi * k * (2.0 * i + 1.0) / (2.0 * n));
  }
}

void dct_eigenvalues(int n, double *lam) {
  const double pi = 3.14159265358979323846;
  for (int k = 0; k < n; ++k) {
    const double s = std::sin(pi * k / (2.0 * n));
    lam[k] = 4.0 * s * s;
  }
}

}  // namespace

bool spectral_fits(int H, int W) { return H <= kSpectralMaxSide && W <= kSpectralMaxSide; }

cudaError_t spectral_setup(Ctx &c) {
  const int H = c.H, W = c.W;
  std::vector<double> ch((size_t)H * H), cw((size_t)W * W), mu(H), nu(W);
  dct_matrix(H, ch.data());
  dct_matrix(W, cw.data());
  dct_eigenvalues(H, mu.data());
  dct_eigenvalues(W, nu.data());
  cudaError_t e = cudaMalloc((void **)&c.sp_ch, sizeof(double) * ch.size());
  if (e == cudaSuccess) e = cudaMalloc((void **)&c.sp_cw, sizeof(double) * cw.size());
  if (e == cudaSuccess) e = cudaMalloc((void **)&c.sp_mu, sizeof(double) * H);
  if (e == cudaSuccess) e = cudaMalloc((void **)&c.sp_nu, sizeof(double) * W);
  if (e == cudaSuccess) e = cudaMalloc((void **)&c.sp_t, sizeof(double) * (size_t)H * W);
  if (e == cudaSuccess) e = cudaMemcpy(c.sp_ch, ch.data(), sizeof(double) * ch.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(c.sp_cw, cw.data(), sizeof(double) * cw.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(c.sp_mu, mu.data(), sizeof(double) * H, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(c.sp_nu, nu.data(), sizeof(double) * W, cudaMemcpyHostToDevice);
  return e;
}

// x = A^+ b for the unit-weight grid Laplacian (b, x: H x W, FP64 device arrays).
cudaError_t launch_spectral(Ctx &c, const double *b, double *x) {
  const int H = c.H, W = c.W;
  double *t = c.sp_t;
  gemm<false, false, false>(c.stream, H, W, H, c.sp_ch, H, b, W, t, W);                    // C_H B
  gemm<false, true, true>(c.stream, H, W, W, t, W, c.sp_cw, W, x, W, c.sp_mu, c.sp_nu);  // (.) C_W^T ./ lambda
  gemm<true, false, false>(c.stream, H, W, H, c.sp_ch, H, x, W, t, W);                     // C_H^T (.)
  gemm<false, false, false>(c.stream, H, W, W, t, W, c.sp_cw, W, x, W);                    // (.) C_W
  c.stats.launches += 4;
  return cudaGetLastError();
}

}  // namespace irtps
