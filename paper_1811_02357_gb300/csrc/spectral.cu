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
// surface.  Each transform is halved by the symmetry C[k][n-1-i] = (-1)^k C[k][i]:
// the even frequencies are the products of the half matrix E[r][i] = C[2r][i]
// with the folded sums x_i + x_{n-1-i}, the odd ones of O[r][i] = C[2r+1][i] with
// the differences x_i - x_{n-1-i}; back, a = E^T (even) and b = O^T (odd) give
// x_i = a + b and x_{n-1-i} = a - b.  The folds and unfolds happen in the loads and
// stores of the tiled FP64 kernels; the division by the eigenvalues is fused into
// the second forward pass.  About H W (H + W) multiply-adds in all, bound by
// GB300's FP64 rate, below the barrier-bound multigrid PCG it replaces for unit
// weights up to 1024 on a side.
#include <cmath>
#include <cstdint>
#include <vector>

#include "irtps_internal.h"

namespace irtps {

namespace {

// 16 x 16 output tiles, one output per thread: GB300's FP64 rate (about two
// multiply-adds per clock per SM) is far below what shared memory feeds, so the
// small tile costs nothing and spreads a 256 x 512 half product over 512 blocks
// (between 3 and 4 per SM) instead of leaving whole SMs idle or doubly loaded.
constexpr int kTile = 16;      // output tile (rows and columns) and depth of one shared-memory stage
constexpr int kGemmThreads = kTile * kTile;

// Forward half-transform: D(m + dro, n + dco) = sum_k A'(m, k) B'(k, n), K terms, where
// A'(m, k) = A[m lda + k] (FA = 0) or A[m lda + k] + FA A[m lda + L-1-k] (the fold of a row of
// length L; the middle element of an odd row alone), and B'(k, n) = B[n ldb + k] (TB) or the same
// fold along B's rows (FB).  SCALE divides by mu[m + dro] + nu[n + dco] and drops the (0, 0) term.
template <int FA, int FB, bool TB, bool SCALE>
__global__ void __launch_bounds__(kGemmThreads) k_dct_fwd(int M, int N, int K, int L, const double *__restrict__ A,
                                                           int lda, const double *__restrict__ B, int ldb,
                                                           double *__restrict__ D, int ldd, int dro, int dco,
                                                           const double *__restrict__ mu,
                                                           const double *__restrict__ nu) {
  __shared__ double As[kTile][kTile + 1];  // [k][m]
  __shared__ double Bs[kTile][kTile + 1];  // [k][n]
  const int m0 = blockIdx.y * kTile, n0 = blockIdx.x * kTile;
  const int tx = threadIdx.x % kTile, ty = threadIdx.x / kTile;
  double acc = 0.0;
  for (int k0 = 0; k0 < K; k0 += kTile) {
    {  // A tile, k fastest across the threads (rows of A are contiguous)
      const int gm = m0 + ty, gk = k0 + tx;
      double a = 0.0;
      if (gm < M && gk < K) {
        a = A[(size_t)gm * lda + gk];
        if (FA != 0 && L - 1 - gk != gk) a += FA * A[(size_t)gm * lda + (L - 1 - gk)];
      }
      As[tx][ty] = a;
    }
    {
      const int nn = TB ? ty : tx, kk = TB ? tx : ty;
      const int gn = n0 + nn, gk = k0 + kk;
      double b = 0.0;
      if (gn < N && gk < K) {
        if (TB) {
          b = B[(size_t)gn * ldb + gk];
        } else {
          b = B[(size_t)gk * ldb + gn];
          if (FB != 0 && L - 1 - gk != gk) b += FB * B[(size_t)(L - 1 - gk) * ldb + gn];
        }
      }
      Bs[kk][nn] = b;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kTile; ++kk) acc = fma(As[kk][ty], Bs[kk][tx], acc);
    __syncthreads();
  }
  const int m = m0 + ty, n = n0 + tx;
  if (m < M && n < N) {
    double v = acc;
    const int gm = m + dro, gn = n + dco;
    if (SCALE) v = (gm == 0 && gn == 0) ? 0.0 : v / (mu[gm] + nu[gn]);
    D[(size_t)gm * ldd + gn] = v;
  }
}

// Inverse half-transforms, paired: a = sum_k A1(m, k) B1(k, n) over K1 terms (even
// frequencies), b = sum_k A2(m, k) B2(k, n) over K2 terms for m < M2, n < N2 (odd
// frequencies; 0 elsewhere), A(m, k) = TA ? A[k lda + m] : A[m lda + k], B(k, n) = B[k ldb + n].
// ROWS: the output index m is a row i < ceil(L/2): D[i] = a + b, D[L-1-i] = a - b;
// else n is a column j < ceil(L/2): D[., j] = a + b, D[., L-1-j] = a - b.
template <bool TA, bool ROWS>
__global__ void __launch_bounds__(kGemmThreads) k_dct_inv(int M, int N, int K1, int K2, int M2, int N2, int L,
                                                           const double *__restrict__ A1, const double *__restrict__ A2,
                                                           int lda1, int lda2, const double *__restrict__ B1,
                                                           const double *__restrict__ B2, int ldb1, int ldb2,
                                                           double *__restrict__ D, int ldd) {
  __shared__ double As1[kTile][kTile + 1], As2[kTile][kTile + 1];  // [k][m]
  __shared__ double Bs1[kTile][kTile + 1], Bs2[kTile][kTile + 1];  // [k][n]
  const int m0 = blockIdx.y * kTile, n0 = blockIdx.x * kTile;
  const int tx = threadIdx.x % kTile, ty = threadIdx.x / kTile;
  const int K = K1 > K2 ? K1 : K2;
  double a = 0.0, b = 0.0;
  for (int k0 = 0; k0 < K; k0 += kTile) {
    {
      const int mm = TA ? tx : ty, kk = TA ? ty : tx;
      const int gm = m0 + mm, gk = k0 + kk;
      const size_t i1 = TA ? (size_t)gk * lda1 + gm : (size_t)gm * lda1 + gk;
      const size_t i2 = TA ? (size_t)gk * lda2 + gm : (size_t)gm * lda2 + gk;
      As1[kk][mm] = (gm < M && gk < K1) ? A1[i1] : 0.0;
      As2[kk][mm] = (gm < M2 && gk < K2) ? A2[i2] : 0.0;
    }
    {
      const int gn = n0 + tx, gk = k0 + ty;
      Bs1[ty][tx] = (gn < N && gk < K1) ? B1[(size_t)gk * ldb1 + gn] : 0.0;
      Bs2[ty][tx] = (gn < N2 && gk < K2) ? B2[(size_t)gk * ldb2 + gn] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kTile; ++kk) {
      a = fma(As1[kk][ty], Bs1[kk][tx], a);
      b = fma(As2[kk][ty], Bs2[kk][tx], b);
    }
    __syncthreads();
  }
  const int m = m0 + ty, n = n0 + tx;
  if (m >= M || n >= N) return;
  if (ROWS) {
    D[(size_t)m * ldd + n] = a + b;
    if (L - 1 - m != m) D[(size_t)(L - 1 - m) * ldd + n] = a - b;
  } else {
    D[(size_t)m * ldd + n] = a + b;
    if (L - 1 - n != n) D[(size_t)m * ldd + (L - 1 - n)] = a - b;
  }
}

dim3 grid_of(int M, int N) { return dim3((N + kTile - 1) / kTile, (M + kTile - 1) / kTile); }

// E (even frequencies, ceil(n/2) x ceil(n/2)) then O (odd, floor(n/2) x floor(n/2)) of the
// orthonormal DCT-II of length n: E[r][i] = C[2r][i], O[r][i] = C[2r+1][i] on the first
// half of the samples, C[k][i] = s_k cos(pi k (2i+1) / 2n).
void dct_halves(int n, double *eo) {
  const double pi = 3.14159265358979323846;
  const int he = (n + 1) / 2, ho = n / 2;
  auto c = [&](int k, int i) {
    const double s = k == 0 ? std::sqrt(1.0 / n) : std::sqrt(2.0 / n);
    return s * std::cos(pi * k * (2.0 * i + 1.0) / (2.0 * n));
  };
  for (int r = 0; r < he; ++r)
    for (int i = 0; i < he; ++i) eo[(size_t)r * he + i] = c(2 * r, i);
  double *o = eo + (size_t)he * he;
  for (int r = 0; r < ho; ++r)
    for (int i = 0; i < ho; ++i) o[(size_t)r * ho + i] = c(2 * r + 1, i);
}

// Path-Laplacian eigenvalues 4 sin^2(pi k / 2n) in the spectral order of the halves:
// even k first, then odd k.
void dct_eigenvalues(int n, double *lam) {
  const double pi = 3.14159265358979323846;
  const int he = (n + 1) / 2;
  for (int k = 0; k < n; ++k) {
    const double s = std::sin(pi * k / (2.0 * n));
    lam[(k & 1) ? he + k / 2 : k / 2] = 4.0 * s * s;
  }
}

}  // namespace

bool spectral_fits(int H, int W) { return H <= kSpectralMaxSide && W <= kSpectralMaxSide; }

cudaError_t spectral_setup(Ctx &c) {
  const int H = c.H, W = c.W;
  auto halves = [](int n) { return (size_t)((n + 1) / 2) * ((n + 1) / 2) + (size_t)(n / 2) * (n / 2); };
  std::vector<double> ch(halves(H)), cw(halves(W)), mu(H), nu(W);
  dct_halves(H, ch.data());
  dct_halves(W, cw.data());
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

// x = A^+ b for the unit-weight grid Laplacian (b, x: H x W, FP64 device arrays).  The spectral
// array between the passes holds the even frequencies of each axis before the odd ones.
cudaError_t launch_spectral(Ctx &c, const double *b, double *x) {
  const int H = c.H, W = c.W;
  const int heH = (H + 1) / 2, hoH = H / 2, heW = (W + 1) / 2, hoW = W / 2;
  const double *EH = c.sp_ch, *OH = c.sp_ch + (size_t)heH * heH;
  const double *EW = c.sp_cw, *OW = c.sp_cw + (size_t)heW * heW;
  double *t = c.sp_t;
  cudaStream_t s = c.stream;
  // columns: t = C_H b (even rows from the row sums, odd rows from the differences)
  k_dct_fwd<0, 1, false, false><<<grid_of(heH, W), kGemmThreads, 0, s>>>(heH, W, heH, H, EH, heH, b, W, t, W, 0,
                                                                        0, nullptr, nullptr);
  k_dct_fwd<0, -1, false, false><<<grid_of(hoH, W), kGemmThreads, 0, s>>>(hoH, W, hoH, H, OH, hoH, b, W, t, W,
                                                                         heH, 0, nullptr, nullptr);
  // rows: x = (t C_W^T) ./ (mu + nu), the (0, 0) term dropped
  k_dct_fwd<1, 0, true, true><<<grid_of(H, heW), kGemmThreads, 0, s>>>(H, heW, heW, W, t, W, EW, heW, x, W, 0, 0,
                                                                      c.sp_mu, c.sp_nu);
  k_dct_fwd<-1, 0, true, true><<<grid_of(H, hoW), kGemmThreads, 0, s>>>(H, hoW, hoW, W, t, W, OW, hoW, x, W, 0,
                                                                       heW, c.sp_mu, c.sp_nu);
  // columns back: t = C_H^T x
  k_dct_inv<true, true><<<grid_of(heH, W), kGemmThreads, 0, s>>>(heH, W, heH, hoH, hoH, W, H, EH, OH, heH, hoH, x,
                                                                 x + (size_t)heH * W, W, W, t, W);
  // rows back: x = t C_W
  k_dct_inv<false, false><<<grid_of(H, heW), kGemmThreads, 0, s>>>(H, heW, heW, hoW, H, hoW, W, t, t + heW, W, W,
                                                                   EW, OW, heW, hoW, x, W);
  c.stats.launches += 6;
  return cudaGetLastError();
}

}  // namespace irtps
