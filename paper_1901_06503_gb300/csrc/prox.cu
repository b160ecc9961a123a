// prox.cu -- the proximal map of the gradient regulariser R(h) = 1/2 |grad h|^2
// (the regulariser of the paper's experiments, Sec. 5, inside the FB step of
// Sec. 3.2), discretised as R(h) = 1/2 <D h, D h> / dx^2 with D the forward
// differences between neighbouring cells of the box and none across its faces:
//
//   prox_{s lambda R}(f) = (I + a D^T D)^{-1} f,   a = s lambda / dx^2.
//
// D^T D is the cell-centred Laplacian with zero-flux faces; the orthonormal
// DCT-II C (C[k][i] = w_k cos(pi k (2i+1) / 2n)) diagonalises it along every
// axis with eigenvalues mu_k = 4 sin^2(pi k / 2n).  So the prox is
// C^T diag(1 / (1 + a (mu_kx + mu_ky + mu_kz))) C f, six passes of "multiply
// every line along one axis by an n x n matrix" with the division fused into
// the third.  Each pass is a dense contraction of n^4 multiply-adds done by a
// register-blocked FFMA (DFMA) tile kernel: the transforms need the full
// precision of the problem, which the bf16/tf32 tensor-core kinds do not give.
#include <math.h>
#include <string.h>

#include <vector>

#include "internal.cuh"

namespace ffpat {
namespace {

constexpr int BM = 64, BN = 64, BK = 16, kThreads = 256;

// out[o][k][j] = sum_i M[k][i] in[o][i][j] over the lines of one axis of the
// n^3 volume viewed as [outer][n][inner] (x: inner 1, y: inner n, z: inner
// n^2).  scale (z pass only): divide by 1 + a (mu[kx] + mu[ky] + mu[kz]).
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_axis_apply(const T* __restrict__ in, T* __restrict__ out, const T* __restrict__ M, int n,
             size_t inner, const double* __restrict__ mu, double a, int scale) {
  __shared__ T As[BK][BM];
  __shared__ T Bs[BK][BN];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int row0 = blockIdx.y * BM;
  const size_t col0 = (size_t)blockIdx.x * BN;
  const size_t ncol = (size_t)n * n;
  const size_t line = (size_t)n * inner;
  T acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = T(0);

  for (int i0 = 0; i0 < n; i0 += BK) {
    for (int e = tid; e < BM * BK; e += kThreads) {
      const int r = e / BK, kk = e % BK;
      const int k = row0 + r, i = i0 + kk;
      As[kk][r] = (k < n && i < n) ? M[(size_t)k * n + i] : T(0);
    }
    if (inner == 1) {
      // x lines are contiguous: neighbouring threads take neighbouring i
      for (int e = tid; e < BN * BK; e += kThreads) {
        const int kk = e % BK, cc = e / BK;
        const size_t col = col0 + cc;
        const int i = i0 + kk;
        Bs[kk][cc] = (col < ncol && i < n) ? in[col * n + i] : T(0);
      }
    } else {
      // y and z lines: neighbouring columns are contiguous
      for (int e = tid; e < BN * BK; e += kThreads) {
        const int cc = e % BN, kk = e / BN;
        const size_t col = col0 + cc;
        const int i = i0 + kk;
        Bs[kk][cc] = (col < ncol && i < n)
                         ? in[(col / inner) * line + (size_t)i * inner + col % inner]
                         : T(0);
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T av[4], bv[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) av[r] = As[kk][ty * 4 + r];
#pragma unroll
      for (int c = 0; c < 4; ++c) bv[c] = Bs[kk][tx * 4 + c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] += av[r] * bv[c];
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int k = row0 + ty * 4 + r;
    if (k >= n) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const size_t col = col0 + tx * 4 + c;
      if (col >= ncol) continue;
      T v = acc[r][c];
      if (scale) {
        const double den = 1.0 + a * (mu[col % n] + mu[col / n] + mu[k]);
        v = (T)((double)v / den);
      }
      out[(col / inner) * line + (size_t)k * inner + col % inner] = v;
    }
  }
}

template <typename T>
int apply_axis(const Plan& pl, const T* in, T* out, const T* M, int axis, double a, bool scale,
               cudaStream_t st) {
  const int n = pl.n;
  const size_t inner = axis == 0 ? 1 : (axis == 1 ? (size_t)n : (size_t)n * n);
  const dim3 grid((unsigned)(((size_t)n * n + BN - 1) / BN), (unsigned)((n + BM - 1) / BM));
  k_axis_apply<T><<<grid, kThreads, 0, st>>>(in, out, M, n, inner, pl.dct_mu, a, scale ? 1 : 0);
  count_launch();
  return check_launch("prox: axis transform");
}

template <typename T>
int prox_t(const Plan& pl, double a, const T* in, T* out, T* s0, T* s1, cudaStream_t st) {
  const T* C = (const T*)pl.dct;
  const T* Ct = C + (size_t)pl.n * pl.n;
  int rc = apply_axis<T>(pl, in, s0, C, 0, a, false, st);
  if (rc == FFPAT_OK) rc = apply_axis<T>(pl, s0, s1, C, 1, a, false, st);
  if (rc == FFPAT_OK) rc = apply_axis<T>(pl, s1, s0, C, 2, a, true, st);
  if (rc == FFPAT_OK) rc = apply_axis<T>(pl, s0, s1, Ct, 2, a, false, st);
  if (rc == FFPAT_OK) rc = apply_axis<T>(pl, s1, s0, Ct, 1, a, false, st);
  if (rc == FFPAT_OK) rc = apply_axis<T>(pl, s0, out, Ct, 0, a, false, st);
  return rc;
}

}  // namespace

size_t dct_bytes(int n, size_t esize) {
  return 2 * (size_t)n * n * esize + (size_t)n * sizeof(double);
}

int upload_dct(const Plan& pl, cudaStream_t st) {
  const int n = pl.n;
  std::vector<double> C((size_t)n * n), mu(n);
  for (int k = 0; k < n; ++k) {
    const double w = k == 0 ? sqrt(1.0 / n) : sqrt(2.0 / n);
    for (int i = 0; i < n; ++i) {
      // angle pi m / (2n) with m = k (2i + 1) reduced mod 4n: exact argument
      const long long m = ((long long)k * (2 * i + 1)) % (4LL * n);
      C[(size_t)k * n + i] = w * cos(M_PI * (double)m / (2.0 * n));
    }
    const double sn = sin(M_PI * k / (2.0 * n));
    mu[k] = 4.0 * sn * sn;
  }
  std::vector<unsigned char> buf(dct_bytes(n, pl.esize));
  const size_t nn = (size_t)n * n;
  for (size_t e = 0; e < nn; ++e) {
    const size_t k = e / n, i = e % n;
    const double c = C[e], ct = C[i * n + k];  // (C^T)[k][i] = C[i][k]
    if (pl.esize == 8) {
      ((double*)buf.data())[e] = c;
      ((double*)buf.data())[nn + e] = ct;
    } else {
      ((float*)buf.data())[e] = (float)c;
      ((float*)buf.data())[nn + e] = (float)ct;
    }
  }
  memcpy(buf.data() + 2 * nn * pl.esize, mu.data(), (size_t)n * sizeof(double));
  if (cudaMemcpyAsync(pl.dct, buf.data(), buf.size(), cudaMemcpyHostToDevice, st) != cudaSuccess)
    return check_launch("prox: table upload");
  // the host buffer dies at return
  if (cudaStreamSynchronize(st) != cudaSuccess) return check_launch("prox: table upload");
  return FFPAT_OK;
}

int launch_prox_grad(const Plan& pl, double a, const void* in, void* out, void* s0, void* s1,
                     cudaStream_t st) {
  if (pl.esize == 8)
    return prox_t<double>(pl, a, (const double*)in, (double*)out, (double*)s0, (double*)s1, st);
  return prox_t<float>(pl, a, (const float*)in, (float*)out, (float*)s0, (float*)s1, st);
}

}  // namespace ffpat
