// xray.cu -- the X-ray transform P of eq. (4) in every horizontal plane, its
// exact transpose P^T (the discrete backprojection X^* of Sec. 3.1) and the
// ramp preconditioner Lambda of Sec. 3.1.
//
// P (ray-driven, no atomics): one thread per detector xi_k of one (theta_j,
// z_l) row; it walks the ray samples s_m that can touch the grid and
// accumulates the zero-extended bilinear samples in order, reading the plane
// through the read-only cache.  For FP64 problems the sample arithmetic is
// done in round-to-nearest multiply/add with no contraction, in the same
// order as the plain definition, so that indices and weights are reproducible
// bit for bit.
//
// P^T (voxel-driven gather, no atomics): one thread per voxel.  For every
// angle the samples whose bilinear footprint covers the voxel lie within
// sqrt(2) grid units of it in the rotated (xi, s) frame, i.e. at most 3 x 3
// candidates; each contributes hat(dx) hat(dy) times its row value, which is
// exactly the bilinear weight P gives that voxel.  Deterministic: fixed order.
//
// Lambda: one CTA per detector row, the row staged in shared memory, the odd
// taps t_d = -1/(2 pi^2 d^2 dxi) and t_0 = 1/(8 dxi) applied as a linear
// (non-circular) convolution.
#include "internal.cuh"

namespace ffpat {
namespace {

constexpr double kPi = 3.14159265358979323846;

// FP64 ray sample (theta, k, m): lower-left corner and fractions.  Same
// operations, same order as the plain definition; no fused multiply-add.
__device__ __forceinline__ void sample64(double cs, double sn, int k, int m, int ns, double dx,
                                         double half, int& i0, int& j0, double& fx, double& fy) {
  const double xi = __dadd_rn(-1.0, __dmul_rn((double)k + 0.5, dx));
  const double s = __dmul_rn(((double)m + 0.5) - (double)(ns / 2), dx);
  const double x = __dsub_rn(__dmul_rn(xi, cs), __dmul_rn(s, sn));
  const double y = __dadd_rn(__dmul_rn(xi, sn), __dmul_rn(s, cs));
  const double gx = __dsub_rn(__dmul_rn(__dadd_rn(x, 1.0), half), 0.5);
  const double gy = __dsub_rn(__dmul_rn(__dadd_rn(y, 1.0), half), 0.5);
  const double flx = floor(gx), fly = floor(gy);
  i0 = (int)flx;
  j0 = (int)fly;
  fx = __dsub_rn(gx, flx);
  fy = __dsub_rn(gy, fly);
}

template <typename T>
__device__ __forceinline__ T pix(const T* __restrict__ sl, int n, int iy, int ix) {
  return (ix >= 0 && iy >= 0 && ix < n && iy < n) ? __ldg(sl + (size_t)iy * n + ix) : T(0);
}

// Range [mlo, mhi) of ray samples that can touch the grid (conservative).
__device__ __forceinline__ void ray_range(float cs, float sn, int k, int n, int ns, int& mlo,
                                          int& mhi) {
  const float cN = 0.5f * (float)(n - 1);
  const float u = (float)k + 0.5f - 0.5f * (float)n;
  float vlo = -1e30f, vhi = 1e30f;
  // x = cN + u cs - v sn must lie in (-1, n)
  const float ax = cN + u * cs;
  if (fabsf(sn) > 1e-6f) {
    float a = (ax + 1.0f) / sn, b = (ax - (float)n) / sn;
    vlo = fmaxf(vlo, fminf(a, b));
    vhi = fminf(vhi, fmaxf(a, b));
  } else if (!(ax > -1.5f && ax < (float)n + 0.5f)) {
    vlo = 1.0f;
    vhi = -1.0f;
  }
  // y = cN + u sn + v cs must lie in (-1, n)
  const float ay = cN + u * sn;
  if (fabsf(cs) > 1e-6f) {
    float a = (-1.0f - ay) / cs, b = ((float)n - ay) / cs;
    vlo = fmaxf(vlo, fminf(a, b));
    vhi = fminf(vhi, fmaxf(a, b));
  } else if (!(ay > -1.5f && ay < (float)n + 0.5f)) {
    vlo = 1.0f;
    vhi = -1.0f;
  }
  if (!(vlo <= vhi)) {
    mlo = 0;
    mhi = 0;
    return;
  }
  const float off = 0.5f * (float)ns - 0.5f;
  mlo = max(0, (int)floorf(vlo + off) - 2);
  mhi = min(ns, (int)ceilf(vhi + off) + 3);
  if (mhi < mlo) mhi = mlo;
}

template <typename T>
__global__ void __launch_bounds__(128)
    k_project(const T* __restrict__ p, T* __restrict__ g, const T* __restrict__ sub,
              const double* __restrict__ tab, const float* __restrict__ tabf,
              const int32_t* __restrict__ tabi, int n, int nth, int ns) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int l = blockIdx.y;
  const int j = blockIdx.z;
  const T* __restrict__ sl = p + (size_t)l * n * n;
  const float csf = tabf[j], snf = tabf[nth + j];
  int mlo = 0, mhi = 0;
  if (k < n) ray_range(csf, snf, k, n, ns, mlo, mhi);
  T acc = T(0);
  if constexpr (sizeof(T) == 8) {
    const double cs = tab[j], sn = tab[nth + j];
    const double dx = 2.0 / n, half = n / 2.0;
    for (int m = mlo; m < mhi; ++m) {
      int i0, j0;
      double fx, fy;
      sample64(cs, sn, k, m, ns, dx, half, i0, j0, fx, fy);
      const double ofx = __dsub_rn(1.0, fx), ofy = __dsub_rn(1.0, fy);
      double b = __dmul_rn(__dmul_rn(ofx, ofy), pix(sl, n, j0, i0));
      b = __dadd_rn(b, __dmul_rn(__dmul_rn(fx, ofy), pix(sl, n, j0, i0 + 1)));
      b = __dadd_rn(b, __dmul_rn(__dmul_rn(ofx, fy), pix(sl, n, j0 + 1, i0)));
      b = __dadd_rn(b, __dmul_rn(__dmul_rn(fx, fy), pix(sl, n, j0 + 1, i0 + 1)));
      acc = __dadd_rn(acc, b);
    }
    if (k < n) {
      double out = __dmul_rn(dx, acc);
      const size_t o = ((size_t)j * n + l) * n + k;
      if (sub) out = out - sub[o];
      g[o] = out;
    }
  } else {
    // fixed point, scale 2^31 grid units: the coordinates of the samples of one
    // ray advance by exact integer steps, so fx, fy carry ~1e-9 absolute error
    // at any grid size (a float coordinate near 384 would carry 3e-5)
    const long long CS = tabi[j], SN = tabi[nth + j];
    const long long u2 = 2LL * k + 1 - n, v2 = 2LL * mlo + 1 - ns;
    const long long c2 = (long long)(n - 1) << 30;
    long long GX = c2 + u2 * CS - v2 * SN;
    long long GY = c2 + u2 * SN + v2 * CS;
    const long long dGX = -2 * SN, dGY = 2 * CS;
    constexpr float kInv = 4.656612873077392578125e-10f;  // 2^-31
    for (int m = mlo; m < mhi; ++m) {
      const int i0 = (int)(GX >> 31), j0 = (int)(GY >> 31);
      const float fx = (float)(unsigned)(GX & 0x7fffffffLL) * kInv;
      const float fy = (float)(unsigned)(GY & 0x7fffffffLL) * kInv;
      GX += dGX;
      GY += dGY;
      const float v00 = pix(sl, n, j0, i0), v10 = pix(sl, n, j0, i0 + 1);
      const float v01 = pix(sl, n, j0 + 1, i0), v11 = pix(sl, n, j0 + 1, i0 + 1);
      const float r0 = fmaf(fx, v10 - v00, v00);
      const float r1 = fmaf(fx, v11 - v01, v01);
      acc += fmaf(fy, r1 - r0, r0);
    }
    if (k < n) {
      float out = (2.0f / (float)n) * acc;
      const size_t o = ((size_t)j * n + l) * n + k;
      if (sub) out = out - sub[o];
      g[o] = out;
    }
  }
}

template <typename T>
__device__ __forceinline__ T hat(T a) {
  const T v = T(1) - (a < T(0) ? -a : a);
  return v > T(0) ? v : T(0);
}

template <typename T>
__global__ void __launch_bounds__(256)
    k_backproject(const T* __restrict__ g, T* __restrict__ h, const T* __restrict__ scale,
                  const double* __restrict__ tab, const float* __restrict__ tabf,
                  const int32_t* __restrict__ tabi, int n, int nth, int ns) {
  const int ix = blockIdx.x * 32 + threadIdx.x;
  const int iy = blockIdx.y * 8 + threadIdx.y;
  const int l = blockIdx.z;
  if (ix >= n || iy >= n) return;
  constexpr float R = 1.41521f;  // sqrt(2) plus a margin; the hat weights vanish beyond it
  T acc = T(0);
  if constexpr (sizeof(T) == 8) {
    const double cN = 0.5 * (n - 1);
    const double X = ix - cN, Y = iy - cN;
    const double koff = 0.5 * n - 0.5, moff = 0.5 * ns - 0.5;
    for (int j = 0; j < nth; ++j) {
      const double cs = tab[j], sn = tab[nth + j];
      const double kk = X * cs + Y * sn + koff;  // detector index of the voxel
      const double mm = Y * cs - X * sn + moff;  // ray sample index of the voxel
      const int klo = max(0, (int)ceil(kk - R)), khi = min(n - 1, (int)floor(kk + R));
      const int mlo = max(0, (int)ceil(mm - R)), mhi = min(ns - 1, (int)floor(mm + R));
      const double* __restrict__ row = g + ((size_t)j * n + l) * n;
      for (int k = klo; k <= khi; ++k) {
        const double du = k - kk;
        double wsum = 0.0;
        for (int m = mlo; m <= mhi; ++m) {
          const double dv = m - mm;
          wsum += hat(du * cs - dv * sn) * hat(du * sn + dv * cs);
        }
        acc += wsum * __ldg(row + k);
      }
    }
  } else {
    // voxel position in the rotated frame in fixed point (scale 2^31) so
    // that the offsets du, dv to the candidate samples are exact to ~1e-9
    const long long X2 = 2LL * ix - (n - 1), Y2 = 2LL * iy - (n - 1);
    const long long koff = (long long)(n - 1) << 30, moff = (long long)(ns - 1) << 30;
    constexpr float kInv = 4.656612873077392578125e-10f;  // 2^-31
    for (int j = 0; j < nth; ++j) {
      const long long CS = tabi[j], SN = tabi[nth + j];
      const float cs = tabf[j], sn = tabf[nth + j];
      const long long KK = X2 * CS + Y2 * SN + koff;
      const long long MM = Y2 * CS - X2 * SN + moff;
      const float kkf = (float)KK * kInv, mmf = (float)MM * kInv;
      const int klo = max(0, (int)ceilf(kkf - R)), khi = min(n - 1, (int)floorf(kkf + R));
      const int mlo = max(0, (int)ceilf(mmf - R)), mhi = min(ns - 1, (int)floorf(mmf + R));
      const float* __restrict__ row = g + ((size_t)j * n + l) * n;
      for (int k = klo; k <= khi; ++k) {
        const float du = (float)(((long long)k << 31) - KK) * kInv;
        float wsum = 0.0f;
        for (int m = mlo; m <= mhi; ++m) {
          const float dv = (float)(((long long)m << 31) - MM) * kInv;
          wsum += hat(du * cs - dv * sn) * hat(du * sn + dv * cs);
        }
        acc += wsum * __ldg(row + k);
      }
    }
  }
  const size_t o = ((size_t)l * n + iy) * n + ix;
  T out = (T(2) / T(n)) * acc;
  if (scale) out *= scale[o];
  h[o] = out;
}

template <typename T>
__global__ void __launch_bounds__(128)
    k_ramp(const T* __restrict__ r, T* __restrict__ out, int n) {
  extern __shared__ unsigned char smem_raw[];
  T* row = reinterpret_cast<T*>(smem_raw);
  T* tap = row + n;  // tap[d] for d < n (odd d nonzero)
  const size_t base = (size_t)blockIdx.x * n;
  const double dxi = 2.0 / n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    row[i] = r[base + i];
    double t;
    if (i == 0)
      t = 1.0 / (8.0 * dxi);
    else if (i % 2 == 0)
      t = 0.0;
    else
      t = -1.0 / (2.0 * kPi * kPi * (double)i * (double)i * dxi);
    tap[i] = (T)t;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    T acc = tap[0] * row[k];
    for (int d = 1; d < n; d += 2) {
      T a = T(0);
      if (k - d >= 0) a += row[k - d];
      if (k + d < n) a += row[k + d];
      acc += tap[d] * a;
    }
    out[base + k] = acc;
  }
}

__global__ void k_debug_samples(int count, const int32_t* __restrict__ jkm, int32_t* __restrict__ ij,
                                double* __restrict__ f, const double* __restrict__ tab, int n,
                                int nth, int ns) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count) return;
  const int j = jkm[3 * t], k = jkm[3 * t + 1], m = jkm[3 * t + 2];
  if (j < 0 || j >= nth) return;
  int i0, j0;
  double fx, fy;
  sample64(tab[j], tab[nth + j], k, m, ns, 2.0 / n, n / 2.0, i0, j0, fx, fy);
  ij[2 * t] = i0;
  ij[2 * t + 1] = j0;
  f[2 * t] = fx;
  f[2 * t + 1] = fy;
}

}  // namespace

int launch_project(const Plan& pl, const void* p, void* g, const void* sub, cudaStream_t st) {
  const dim3 block(128);
  const dim3 grid((pl.n + 127) / 128, pl.n, pl.nth);
  if (pl.prec == FFPAT_FP64)
    k_project<double><<<grid, block, 0, st>>>((const double*)p, (double*)g, (const double*)sub,
                                              pl.tab, pl.tabf, pl.tabi, pl.n, pl.nth, pl.ns);
  else
    k_project<float><<<grid, block, 0, st>>>((const float*)p, (float*)g, (const float*)sub, pl.tab,
                                             pl.tabf, pl.tabi, pl.n, pl.nth, pl.ns);
  count_launch();
  return check_launch(__func__);
}

int launch_backproject(const Plan& pl, const void* g, void* h, const void* scale, cudaStream_t st) {
  const dim3 block(32, 8);
  const dim3 grid((pl.n + 31) / 32, (pl.n + 7) / 8, pl.n);
  if (pl.prec == FFPAT_FP64)
    k_backproject<double><<<grid, block, 0, st>>>((const double*)g, (double*)h,
                                                  (const double*)scale, pl.tab, pl.tabf,
                                                  pl.tabi, pl.n, pl.nth, pl.ns);
  else
    k_backproject<float><<<grid, block, 0, st>>>((const float*)g, (float*)h, (const float*)scale,
                                                 pl.tab, pl.tabf, pl.tabi, pl.n, pl.nth, pl.ns);
  count_launch();
  return check_launch(__func__);
}

int launch_ramp(const Plan& pl, const void* r, void* out, cudaStream_t st) {
  const unsigned rows = (unsigned)(pl.nth * pl.n);
  const size_t smem = 2 * (size_t)pl.n * pl.esize;
  if (pl.prec == FFPAT_FP64)
    k_ramp<double><<<rows, 128, smem, st>>>((const double*)r, (double*)out, pl.n);
  else
    k_ramp<float><<<rows, 128, smem, st>>>((const float*)r, (float*)out, pl.n);
  count_launch();
  return check_launch(__func__);
}

int launch_debug_samples(const Plan& pl, int count, const int32_t* jkm, int32_t* ij, double* f,
                         cudaStream_t st) {
  if (count <= 0) return FFPAT_OK;
  k_debug_samples<<<(count + 127) / 128, 128, 0, st>>>(count, jkm, ij, f, pl.tab, pl.n, pl.nth,
                                                      pl.ns);
  count_launch();
  return check_launch(__func__);
}

}  // namespace ffpat
