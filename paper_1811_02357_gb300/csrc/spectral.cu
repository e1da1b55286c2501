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
// One 16 x 16 output tile at (m0, n0) per block.
template <int FA, int FB, bool TB, bool SCALE>
__device__ __forceinline__ void dct_fwd_tile(const DctFwd &p, int m0, int n0) {
  __shared__ double As[kTile][kTile + 1];  // [k][m]
  __shared__ double Bs[kTile][kTile + 1];  // [k][n]
  const int M = p.M, N = p.N, K = p.K, L = p.L, lda = p.lda, ldb = p.ldb;
  const double *__restrict__ A = p.A;
  const double *__restrict__ B = p.B;
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
    const int gm = m + p.dro, gn = n + p.dco;
    if (SCALE) v = (gm == 0 && gn == 0) ? 0.0 : v / (p.mu[gm] + p.nu[gn]);
    p.D[(size_t)gm * p.ldd + gn] = v;
  }
}

// Inverse half-transforms, paired: a = sum_k A1(m, k) B1(k, n) over K1 terms (even
// frequencies), b = sum_k A2(m, k) B2(k, n) over K2 terms for m < M2, n < N2 (odd
// frequencies; 0 elsewhere), A(m, k) = TA ? A[k lda + m] : A[m lda + k], B(k, n) = B[k ldb + n].
// ROWS: the output index m is a row i < ceil(L/2): D[i] = a + b, D[L-1-i] = a - b;
// else n is a column j < ceil(L/2): D[., j] = a + b, D[., L-1-j] = a - b.
template <bool TA, bool ROWS>
__device__ __forceinline__ void dct_inv_tile(const DctInv &p, int m0, int n0) {
  __shared__ double As1[kTile][kTile + 1], As2[kTile][kTile + 1];  // [k][m]
  __shared__ double Bs1[kTile][kTile + 1], Bs2[kTile][kTile + 1];  // [k][n]
  const int M = p.M, N = p.N, K1 = p.K1, K2 = p.K2, M2 = p.M2, N2 = p.N2, L = p.L;
  const int tx = threadIdx.x % kTile, ty = threadIdx.x / kTile;
  const int K = K1 > K2 ? K1 : K2;
  double a = 0.0, b = 0.0;
  for (int k0 = 0; k0 < K; k0 += kTile) {
    {
      const int mm = TA ? tx : ty, kk = TA ? ty : tx;
      const int gm = m0 + mm, gk = k0 + kk;
      const size_t i1 = TA ? (size_t)gk * p.lda1 + gm : (size_t)gm * p.lda1 + gk;
      const size_t i2 = TA ? (size_t)gk * p.lda2 + gm : (size_t)gm * p.lda2 + gk;
      As1[kk][mm] = (gm < M && gk < K1) ? p.A1[i1] : 0.0;
      As2[kk][mm] = (gm < M2 && gk < K2) ? p.A2[i2] : 0.0;
    }
    {
      const int gn = n0 + tx, gk = k0 + ty;
      Bs1[ty][tx] = (gn < N && gk < K1) ? p.B1[(size_t)gk * p.ldb1 + gn] : 0.0;
      Bs2[ty][tx] = (gn < N2 && gk < K2) ? p.B2[(size_t)gk * p.ldb2 + gn] : 0.0;
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
  double *D = p.D;
  const int ldd = p.ldd;
  if (ROWS) {
    D[(size_t)m * ldd + n] = a + b;
    if (L - 1 - m != m) D[(size_t)(L - 1 - m) * ldd + n] = a - b;
  } else {
    D[(size_t)m * ldd + n] = a + b;
    if (L - 1 - n != n) D[(size_t)m * ldd + (L - 1 - n)] = a - b;
  }
}

// Single object: blockIdx (x, y) = tile (column, row).
template <int FA, int FB, bool TB, bool SCALE>
__global__ void __launch_bounds__(kGemmThreads) k_dct_fwd(const DctFwd p) {
  dct_fwd_tile<FA, FB, TB, SCALE>(p, blockIdx.y * kTile, blockIdx.x * kTile);
}
template <bool TA, bool ROWS>
__global__ void __launch_bounds__(kGemmThreads) k_dct_inv(const DctInv p) {
  dct_inv_tile<TA, ROWS>(p, blockIdx.y * kTile, blockIdx.x * kTile);
}

// Batched: the tiles of every object's pass in one launch; object o owns blocks
// [blk_begin of o, blk_begin of o + 1), its tiles in row-major order.
template <typename D>
__device__ __forceinline__ int dct_object(const D *__restrict__ ps, int n, int &tile) {
  __shared__ int s_o;
  if (threadIdx.x == 0) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (ps[mid].blk_begin <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
    }
    s_o = lo;
  }
  __syncthreads();
  tile = (int)blockIdx.x - ps[s_o].blk_begin;
  return s_o;
}
template <int FA, int FB, bool TB, bool SCALE>
__global__ void __launch_bounds__(kGemmThreads) k_dct_fwd_b(const DctFwd *__restrict__ ps, int n) {
  int tile;
  const DctFwd &p = ps[dct_object(ps, n, tile)];
  dct_fwd_tile<FA, FB, TB, SCALE>(p, tile / p.tiles_n * kTile, tile % p.tiles_n * kTile);
}
template <bool TA, bool ROWS>
__global__ void __launch_bounds__(kGemmThreads) k_dct_inv_b(const DctInv *__restrict__ ps, int n) {
  int tile;
  const DctInv &p = ps[dct_object(ps, n, tile)];
  dct_inv_tile<TA, ROWS>(p, tile / p.tiles_n * kTile, tile % p.tiles_n * kTile);
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

// The six passes of x = A^+ b for the unit-weight grid Laplacian of a context (b, x:
// H x W, FP64 device arrays).  The spectral array between the passes holds the even
// frequencies of each axis before the odd ones.
static void spectral_passes(const Ctx &c, const double *b, double *x, DctFwd f[4], DctInv v[2]) {
  const int H = c.H, W = c.W;
  const int heH = (H + 1) / 2, hoH = H / 2, heW = (W + 1) / 2, hoW = W / 2;
  const double *EH = c.sp_ch, *OH = c.sp_ch + (size_t)heH * heH;
  const double *EW = c.sp_cw, *OW = c.sp_cw + (size_t)heW * heW;
  double *t = c.sp_t;
  // columns: t = C_H b (even rows from the row sums, odd rows from the differences)
  f[0] = DctFwd{heH, W, heH, H, EH, heH, b, W, t, W, 0, 0, nullptr, nullptr, 0, 0};
  f[1] = DctFwd{hoH, W, hoH, H, OH, hoH, b, W, t, W, heH, 0, nullptr, nullptr, 0, 0};
  // rows: x = (t C_W^T) ./ (mu + nu), the (0, 0) term dropped
  f[2] = DctFwd{H, heW, heW, W, t, W, EW, heW, x, W, 0, 0, c.sp_mu, c.sp_nu, 0, 0};
  f[3] = DctFwd{H, hoW, hoW, W, t, W, OW, hoW, x, W, 0, heW, c.sp_mu, c.sp_nu, 0, 0};
  // columns back: t = C_H^T x
  v[0] = DctInv{heH, W, heH, hoH, hoH, W, H, EH, OH, heH, hoH, x, x + (size_t)heH * W, W, W, t, W, 0, 0};
  // rows back: x = t C_W
  v[1] = DctInv{H, heW, heW, hoW, H, hoW, W, t, t + heW, W, W, EW, OW, heW, hoW, x, W, 0, 0};
  for (int i = 0; i < 4; ++i) f[i].tiles_n = (f[i].N + kTile - 1) / kTile;
  for (int i = 0; i < 2; ++i) v[i].tiles_n = (v[i].N + kTile - 1) / kTile;
}

cudaError_t launch_spectral(Ctx &c, const double *b, double *x) {
  DctFwd f[4];
  DctInv v[2];
  spectral_passes(c, b, x, f, v);
  cudaStream_t s = c.stream;
  k_dct_fwd<0, 1, false, false><<<grid_of(f[0].M, f[0].N), kGemmThreads, 0, s>>>(f[0]);
  k_dct_fwd<0, -1, false, false><<<grid_of(f[1].M, f[1].N), kGemmThreads, 0, s>>>(f[1]);
  k_dct_fwd<1, 0, true, true><<<grid_of(f[2].M, f[2].N), kGemmThreads, 0, s>>>(f[2]);
  k_dct_fwd<-1, 0, true, true><<<grid_of(f[3].M, f[3].N), kGemmThreads, 0, s>>>(f[3]);
  k_dct_inv<true, true><<<grid_of(v[0].M, v[0].N), kGemmThreads, 0, s>>>(v[0]);
  k_dct_inv<false, false><<<grid_of(v[1].M, v[1].N), kGemmThreads, 0, s>>>(v[1]);
  c.stats.launches += 6;
  return cudaGetLastError();
}

// Batched direct solves: one launch per pass over the objects whose unit-weight
// solves are direct; each object's pass descriptors point at its own arrays.
cudaError_t spectral_batch_setup(const std::vector<Ctx *> &objs, SpectralBatch &sb) {
  sb.n = 0;
  std::vector<DctFwd> f[4];
  std::vector<DctInv> v[2];
  for (int i = 0; i < 4; ++i) sb.blocks[i] = 0;
  sb.blocks[4] = sb.blocks[5] = 0;
  for (Ctx *c : objs) {
    if (!direct_solve(*c)) continue;
    DctFwd ff[4];
    DctInv vv[2];
    spectral_passes(*c, c->cg_b, c->cg_x, ff, vv);
    for (int i = 0; i < 4; ++i) {
      ff[i].blk_begin = sb.blocks[i];
      sb.blocks[i] += ((ff[i].M + kTile - 1) / kTile) * ff[i].tiles_n;
      f[i].push_back(ff[i]);
    }
    for (int i = 0; i < 2; ++i) {
      vv[i].blk_begin = sb.blocks[4 + i];
      sb.blocks[4 + i] += ((vv[i].M + kTile - 1) / kTile) * vv[i].tiles_n;
      v[i].push_back(vv[i]);
    }
    ++sb.n;
  }
  if (sb.n == 0) return cudaSuccess;
  const size_t fb = sizeof(DctFwd) * sb.n, vb = sizeof(DctInv) * sb.n;
  cudaError_t e = cudaMalloc(&sb.table, 4 * fb + 2 * vb);
  if (e != cudaSuccess) return e;
  unsigned char *t = (unsigned char *)sb.table;
  for (int i = 0; i < 4 && e == cudaSuccess; ++i) e = cudaMemcpy(t + i * fb, f[i].data(), fb, cudaMemcpyHostToDevice);
  for (int i = 0; i < 2 && e == cudaSuccess; ++i)
    e = cudaMemcpy(t + 4 * fb + i * vb, v[i].data(), vb, cudaMemcpyHostToDevice);
  return e;
}

cudaError_t launch_spectral_batch(cudaStream_t s, const SpectralBatch &sb) {
  if (sb.n == 0) return cudaSuccess;
  const DctFwd *f = (const DctFwd *)sb.table;
  const DctInv *v = (const DctInv *)(f + 4 * sb.n);
  const int n = sb.n;
  k_dct_fwd_b<0, 1, false, false><<<sb.blocks[0], kGemmThreads, 0, s>>>(f, n);
  k_dct_fwd_b<0, -1, false, false><<<sb.blocks[1], kGemmThreads, 0, s>>>(f + n, n);
  k_dct_fwd_b<1, 0, true, true><<<sb.blocks[2], kGemmThreads, 0, s>>>(f + 2 * n, n);
  k_dct_fwd_b<-1, 0, true, true><<<sb.blocks[3], kGemmThreads, 0, s>>>(f + 3 * n, n);
  k_dct_inv_b<true, true><<<sb.blocks[4], kGemmThreads, 0, s>>>(v, n);
  k_dct_inv_b<false, false><<<sb.blocks[5], kGemmThreads, 0, s>>>(v + n, n);
  return cudaGetLastError();
}

}  // namespace irtps
