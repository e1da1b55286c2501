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
// against the H x W data): 2 H W (H + W) multiply-adds, done by one tiled FP64
// kernel; the division by the eigenvalues is fused into the second product.
// GB300's FP64 rate bounds it (about 1 ms at 512 x 512, 7 ms at 1024 x 1024),
// below the barrier-bound multigrid PCG it replaces for unit weights up to 1024.
#include <cmath>
#include <cstdint>
#include <vector>

#include "irtps_internal.h"

namespace irtps {

namespace {

// 16 x 16 output tiles, one output per thread: GB300's FP64 rate (about two
// multiply-adds per clock per SM) is far below what shared memory feeds, so the
// small tile costs nothing and spreads a 512 x 512 product over 1024 blocks
// (about 7 per SM) instead of leaving whole SMs idle or doubly loaded.
constexpr int kTile = 16;      // output tile (rows and columns) and depth of one shared-memory stage
constexpr int kGemmThreads = kTile * kTile;

// D = op(A) op(B), M x N, inner dimension K; op(A)(m, k) = TA ? A[k lda + m] : A[m lda + k],
// op(B)(k, n) = TB ? B[n ldb + k] : B[k ldb + n].  SCALE: D(m, n) /= mu[m] + nu[n], D(0, 0) = 0.
template <bool TA, bool TB, bool SCALE>
__global__ void __launch_bounds__(kGemmThreads) k_dgemm(int M, int N, int K, const double *__restrict__ A, int lda,
                                                         const double *__restrict__ B, int ldb,
                                                         double *__restrict__ D, int ldd,
                                                         const double *__restrict__ mu,
                                                         const double *__restrict__ nu) {
  __shared__ double As[kTile][kTile + 1];  // [k][m]
  __shared__ double Bs[kTile][kTile + 1];  // [k][n]
  const int m0 = blockIdx.y * kTile, n0 = blockIdx.x * kTile;
  const int tx = threadIdx.x % kTile, ty = threadIdx.x / kTile;
  double acc = 0.0;
  for (int k0 = 0; k0 < K; k0 += kTile) {
    // the contiguous index of each source runs fastest across the threads
    {
      const int mm = TA ? tx : ty, kk = TA ? ty : tx;
      const int gm = m0 + mm, gk = k0 + kk;
      As[kk][mm] = (gm < M && gk < K) ? (TA ? A[(size_t)gk * lda + gm] : A[(size_t)gm * lda + gk]) : 0.0;
    }
    {
      const int nn = TB ? ty : tx, kk = TB ? tx : ty;
      const int gn = n0 + nn, gk = k0 + kk;
      Bs[kk][nn] = (gn < N && gk < K) ? (TB ? B[(size_t)gn * ldb + gk] : B[(size_t)gk * ldb + gn]) : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kTile; ++kk) acc = fma(As[kk][ty], Bs[kk][tx], acc);
    __syncthreads();
  }
  const int m = m0 + ty, n = n0 + tx;
  if (m < M && n < N) {
    double v = acc;
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
