// stencil.cu -- leapfrog time steps of the variable-sound-speed wave equation
// p_tt = c^2 Delta p (Sec. 2.1, eq. (1)-(2)) on the N^3 cell-centred grid.
//
// One launch advances the whole volume by one time step.  A CTA owns a 32 x 8
// column tile of the (x, y) plane and streams a range of z planes through it
// (2.5D blocking): the plane at z is staged in shared memory with a two-point
// halo in x and y, and each thread keeps its own column's z-neighbours
// z-2 .. z+3 in registers, so every value of p^n is read from HBM once per
// step (halo re-reads hit L2).  The c^2 factor is fused in as the per-point
// coefficient kap = (c dt / dx)^2 / 12 multiplying L = 12 L4, the integer-
// weight fourth-order Laplacian:
//   L = sum_axes (-u[-2] + 16 u[-1] - 30 u[0] + 16 u[+1] - u[+2]).
// Ghost values outside the box are zero.
//
// Two time-update forms:
//   three-term   p^{n+1} = 2 p^n - p^{n-1} + kap L p^n  (p^{n+1} overwrites
//                p^{n-1} in place): FP64 16+16 B, FP32 8+8 B per point-step;
//   increment    d^{n+1} = d^n + kap L p^n, p^{n+1} = p^n + d^{n+1} with a
//                Kahan carry e (FP32): 16 B read + 12 B written per point-step.
// Both start from p^0 = h, p^1 = p^0 + kap L p^0 / 2 (zero initial velocity).
#include "internal.cuh"

namespace ffpat {
namespace {

constexpr int BX = 32;
constexpr int BY = 8;

template <typename T>
struct Tile {
  T s[BY + 4][BX + 4];
};

template <typename T>
__device__ __forceinline__ T load_col(const T* __restrict__ p, size_t pl, size_t col, int z, int n,
                                      bool in) {
  return (in && z >= 0 && z < n) ? __ldg(p + (size_t)z * pl + col) : T(0);
}

// Stage plane z of p into the tile: the caller's own value plus the halo.
template <typename T>
__device__ __forceinline__ void fill_plane(Tile<T>& t, const T* __restrict__ p, int n, int z,
                                           int x0, int y0, int tx, int ty, T centre) {
  t.s[ty + 2][tx + 2] = centre;
  const T* pz = p + (size_t)z * n * n;
  const int x = x0 + tx;
  if (ty < 2) {
    const int ya = y0 - 2 + ty;
    const int yb = y0 + BY + ty;
    t.s[ty][tx + 2] = (x < n && ya >= 0) ? __ldg(pz + (size_t)ya * n + x) : T(0);
    t.s[BY + 2 + ty][tx + 2] = (x < n && yb < n) ? __ldg(pz + (size_t)yb * n + x) : T(0);
  }
  if (tx < 2) {
    const int y = y0 + ty;
    const int xa = x0 - 2 + tx;
    const int xb = x0 + BX + tx;
    t.s[ty + 2][tx] = (y < n && xa >= 0) ? __ldg(pz + (size_t)y * n + xa) : T(0);
    t.s[ty + 2][BX + 2 + tx] = (y < n && xb < n) ? __ldg(pz + (size_t)y * n + xb) : T(0);
  }
}

// L = 12 L4 at the thread's point.
__device__ __forceinline__ double lap12(const Tile<double>& t, int tx, int ty, double m2, double m1,
                                        double c, double p1, double p2) {
  // plain sums: FP64 has the precision and GB300 has few FP64 units
  double s1 = t.s[ty + 2][tx + 1] + t.s[ty + 2][tx + 3];
  s1 += t.s[ty + 1][tx + 2];
  s1 += t.s[ty + 3][tx + 2];
  s1 += m1;
  s1 += p1;
  double s2 = fma(90.0, c, t.s[ty + 2][tx]);
  s2 += t.s[ty + 2][tx + 4];
  s2 += t.s[ty][tx + 2];
  s2 += t.s[ty + 4][tx + 2];
  s2 += m2;
  s2 += p2;
  return fma(16.0, s1, -s2);
}

__device__ __forceinline__ float lap12(const Tile<float>& t, int tx, int ty, float m2, float m1,
                                       float c, float p1, float p2) {
  // difference form: neighbours minus centre first, so that the rounding is
  // relative to the (small) differences and not to the field value itself
  float d1 = (t.s[ty + 2][tx + 1] - c) + (t.s[ty + 2][tx + 3] - c);
  d1 += (t.s[ty + 1][tx + 2] - c) + (t.s[ty + 3][tx + 2] - c);
  d1 += (m1 - c) + (p1 - c);
  float d2 = (t.s[ty + 2][tx] - c) + (t.s[ty + 2][tx + 4] - c);
  d2 += (t.s[ty][tx + 2] - c) + (t.s[ty + 4][tx + 2] - c);
  d2 += (m2 - c) + (p2 - c);
  return fmaf(16.0f, d1, -d2);
}

// three-term update p^{n+1} = 2 p^n - p^{n-1} + kap L
__device__ __forceinline__ double update3(double c, double pm, double k, double L) {
  return fma(k, L, fma(2.0, c, -pm));
}
__device__ __forceinline__ float update3(float c, float pm, float k, float L) {
  return c + fmaf(k, L, c - pm);
}

template <typename T, bool START>
__global__ void __launch_bounds__(BX* BY)
    k_step3(const T* __restrict__ p, const T* qin, T* qout, const T* __restrict__ kap,
            T* __restrict__ copy0, int n, int zc) {
  __shared__ Tile<T> t;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int x0 = blockIdx.x * BX, y0 = blockIdx.y * BY;
  const int x = x0 + tx, y = y0 + ty;
  const int z0 = blockIdx.z * zc;
  const int z1 = min(n, z0 + zc);
  const bool in = (x < n) && (y < n);
  const size_t pl = (size_t)n * n;
  const size_t col = in ? (size_t)y * n + x : 0;

  T m2 = load_col(p, pl, col, z0 - 2, n, in);
  T m1 = load_col(p, pl, col, z0 - 1, n, in);
  T c0 = load_col(p, pl, col, z0, n, in);
  T p1 = load_col(p, pl, col, z0 + 1, n, in);
  T p2 = load_col(p, pl, col, z0 + 2, n, in);
  for (int z = z0; z < z1; ++z) {
    const size_t i = (size_t)z * pl + col;
    const T p3 = load_col(p, pl, col, z + 3, n, in);
    const T k = in ? __ldg(kap + i) : T(0);
    const T pm = (!START && in) ? qin[i] : T(0);
    fill_plane(t, p, n, z, x0, y0, tx, ty, c0);
    __syncthreads();
    if (in) {
      const T L = lap12(t, tx, ty, m2, m1, c0, p1, p2);
      if (START) {
        qout[i] = c0 + T(0.5) * k * L;
        if (copy0) copy0[i] = c0;
      } else {
        qout[i] = update3(c0, pm, k, L);
      }
    }
    __syncthreads();
    m2 = m1;
    m1 = c0;
    c0 = p1;
    p1 = p2;
    p2 = p3;
  }
}

template <bool START>
__global__ void __launch_bounds__(BX* BY)
    k_step_inc(const float* __restrict__ p, float* __restrict__ pout, float* __restrict__ d,
               float* __restrict__ e, const float* __restrict__ kap, int n, int zc) {
  __shared__ Tile<float> t;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int x0 = blockIdx.x * BX, y0 = blockIdx.y * BY;
  const int x = x0 + tx, y = y0 + ty;
  const int z0 = blockIdx.z * zc;
  const int z1 = min(n, z0 + zc);
  const bool in = (x < n) && (y < n);
  const size_t pl = (size_t)n * n;
  const size_t col = in ? (size_t)y * n + x : 0;

  float m2 = load_col(p, pl, col, z0 - 2, n, in);
  float m1 = load_col(p, pl, col, z0 - 1, n, in);
  float c0 = load_col(p, pl, col, z0, n, in);
  float p1 = load_col(p, pl, col, z0 + 1, n, in);
  float p2 = load_col(p, pl, col, z0 + 2, n, in);
  for (int z = z0; z < z1; ++z) {
    const size_t i = (size_t)z * pl + col;
    const float p3 = load_col(p, pl, col, z + 3, n, in);
    const float k = in ? __ldg(kap + i) : 0.0f;
    const float dold = (!START && in) ? d[i] : 0.0f;
    const float eold = (!START && in) ? e[i] : 0.0f;
    fill_plane(t, p, n, z, x0, y0, tx, ty, c0);
    __syncthreads();
    if (in) {
      const float L = lap12(t, tx, ty, m2, m1, c0, p1, p2);
      const float dn = START ? 0.5f * k * L : fmaf(k, L, dold);
      // Kahan-compensated p^{n+1} = p^n + d^{n+1}
      const float yv = dn - eold;
      const float tv = c0 + yv;
      const float en = (tv - c0) - yv;
      pout[i] = tv;
      d[i] = dn;
      e[i] = en;
    }
    __syncthreads();
    m2 = m1;
    m1 = c0;
    c0 = p1;
    p1 = p2;
    p2 = p3;
  }
}

// acc += w * u * L(p): the kappa-derivative terms of the differentiated
// leapfrog (u holds kappa/12 times the adjoint state, so that, with L = 12 L4,
// the sum over steps is the c-gradient up to the factor 2/c).
template <typename T>
__global__ void __launch_bounds__(BX* BY)
    k_lap_accum(T* __restrict__ acc, const T* __restrict__ u, const T* __restrict__ p, T w, int n,
                int zc) {
  __shared__ Tile<T> t;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int x0 = blockIdx.x * BX, y0 = blockIdx.y * BY;
  const int x = x0 + tx, y = y0 + ty;
  const int z0 = blockIdx.z * zc;
  const int z1 = min(n, z0 + zc);
  const bool in = (x < n) && (y < n);
  const size_t pl = (size_t)n * n;
  const size_t col = in ? (size_t)y * n + x : 0;
  T m2 = load_col(p, pl, col, z0 - 2, n, in);
  T m1 = load_col(p, pl, col, z0 - 1, n, in);
  T c0 = load_col(p, pl, col, z0, n, in);
  T p1 = load_col(p, pl, col, z0 + 1, n, in);
  T p2 = load_col(p, pl, col, z0 + 2, n, in);
  for (int z = z0; z < z1; ++z) {
    const size_t i = (size_t)z * pl + col;
    const T p3 = load_col(p, pl, col, z + 3, n, in);
    fill_plane(t, p, n, z, x0, y0, tx, ty, c0);
    __syncthreads();
    if (in) acc[i] += w * __ldg(u + i) * lap12(t, tx, ty, m2, m1, c0, p1, p2);
    __syncthreads();
    m2 = m1;
    m1 = c0;
    c0 = p1;
    p1 = p2;
    p2 = p3;
  }
}

dim3 step_grid(int n, int* zc) {
  const int gx = (n + BX - 1) / BX, gy = (n + BY - 1) / BY;
  const int target = 8 * kNumSMs;  // 8 CTAs of 256 threads fill an SM
  int zsplit = (target + gx * gy - 1) / (gx * gy);
  int zmax = n / 4 > 0 ? n / 4 : 1;
  if (zsplit > zmax) zsplit = zmax;
  if (zsplit < 1) zsplit = 1;
  *zc = (n + zsplit - 1) / zsplit;
  zsplit = (n + *zc - 1) / *zc;
  return dim3(gx, gy, zsplit);
}

}  // namespace

int launch_lap_accum(const Plan& pl, void* acc, const void* u, const void* p, double w,
                     cudaStream_t st) {
  // FP32 on TMA-aligned arrays: the single-step TMA kernel's accumulation form
  // (p through its plane ring with the halo, mu and acc as halo-free tiles)
  const void* ptrs[3] = {acc, u, p};
  if (pl.prec != FFPAT_FP64 && (w == 1.0 || w == 0.5) && tma_supported(pl, ptrs, 3)) {
    const void* q[2] = {u, acc};
    return launch_step_tma(pl, 2, w == 0.5, p, q, acc, nullptr, nullptr, st);
  }
  int zc;
  const dim3 grid = step_grid(pl.n, &zc);
  const dim3 block(BX, BY);
  if (pl.prec == FFPAT_FP64)
    k_lap_accum<double><<<grid, block, 0, st>>>((double*)acc, (const double*)u, (const double*)p, w,
                                                pl.n, zc);
  else
    k_lap_accum<float><<<grid, block, 0, st>>>((float*)acc, (const float*)u, (const float*)p,
                                               (float)w, pl.n, zc);
  count_launch();
  return check_launch(__func__);
}

int launch_step3(const Plan& pl, const void* p, const void* qin, void* qout, bool start,
                 void* copy_p0, cudaStream_t st) {
  int zc;
  const dim3 grid = step_grid(pl.n, &zc);
  const dim3 block(BX, BY);
  if (pl.prec == FFPAT_FP64) {
    if (start)
      k_step3<double, true><<<grid, block, 0, st>>>((const double*)p, nullptr, (double*)qout,
                                                   (const double*)pl.kap, (double*)copy_p0, pl.n, zc);
    else
      k_step3<double, false><<<grid, block, 0, st>>>((const double*)p, (const double*)qin,
                                                    (double*)qout, (const double*)pl.kap, nullptr,
                                                    pl.n, zc);
  } else {
    if (start)
      k_step3<float, true><<<grid, block, 0, st>>>((const float*)p, nullptr, (float*)qout,
                                                  (const float*)pl.kap, (float*)copy_p0, pl.n, zc);
    else
      k_step3<float, false><<<grid, block, 0, st>>>((const float*)p, (const float*)qin,
                                                   (float*)qout, (const float*)pl.kap, nullptr,
                                                   pl.n, zc);
  }
  count_launch();
  return check_launch(__func__);
}

int launch_step_inc(const Plan& pl, const void* pin, void* pout, void* d, void* e, bool start,
                    cudaStream_t st) {
  int zc;
  const dim3 grid = step_grid(pl.n, &zc);
  const dim3 block(BX, BY);
  if (start)
    k_step_inc<true><<<grid, block, 0, st>>>((const float*)pin, (float*)pout, (float*)d, (float*)e,
                                             (const float*)pl.kap, pl.n, zc);
  else
    k_step_inc<false><<<grid, block, 0, st>>>((const float*)pin, (float*)pout, (float*)d,
                                              (float*)e, (const float*)pl.kap, pl.n, zc);
  count_launch();
  return check_launch(__func__);
}

}  // namespace ffpat
