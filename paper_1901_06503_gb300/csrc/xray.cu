// xray.cu -- the X-ray transform P of eq. (4) in every horizontal plane, its
// exact transpose P^T (the discrete backprojection X^* of Sec. 3.1) and the
// ramp preconditioner Lambda of Sec. 3.1.
//
// Geometry: the planes have n cells per axis of physical size dx = 2 / nimg
// (nimg = n on the box [-1, 1]^3; n = nimg + 2 pad on a padded wave grid,
// which then spans [-L, L], L = n / nimg); n detectors and Ns = 2 ceil(n /
// sqrt 2) ray samples, both spaced dx.  The index geometry depends on n only;
// dx enters as the sample length and the detector spacing of Lambda.
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
// P stages the plane in shared memory when it fits (N <= 220 in FP32).
//
// Lambda: one CTA per detector row, the row staged in shared memory, the odd
// taps t_d = -1/(2 pi^2 d^2 dxi) and t_0 = 1/(8 dxi) applied as a linear
// (non-circular) convolution.
#include <limits.h>
#include <math.h>
#include <stdlib.h>

#include <mutex>
#include <vector>

#include "internal.cuh"

namespace ffpat {
namespace {

constexpr double kPi = 3.14159265358979323846;

// FP64 ray sample (theta, k, m): lower-left corner and fractions.  Same
// operations, same order as the plain definition; no fused multiply-add.  The
// plane spans [-L, L] in cells of size dx = 2 / nimg (L = n / nimg: 1 on the
// box, larger on a padded wave grid); half = nimg / 2.
__device__ __forceinline__ void sample64(double cs, double sn, int k, int m, int ns, double dx,
                                         double half, double L, int& i0, int& j0, double& fx,
                                         double& fy) {
  const double xi = __dadd_rn(-L, __dmul_rn((double)k + 0.5, dx));
  const double s = __dmul_rn(((double)m + 0.5) - (double)(ns / 2), dx);
  const double x = __dsub_rn(__dmul_rn(xi, cs), __dmul_rn(s, sn));
  const double y = __dadd_rn(__dmul_rn(xi, sn), __dmul_rn(s, cs));
  const double gx = __dsub_rn(__dmul_rn(__dadd_rn(x, L), half), 0.5);
  const double gy = __dsub_rn(__dmul_rn(__dadd_rn(y, L), half), 0.5);
  const double flx = floor(gx), fly = floor(gy);
  i0 = (int)flx;
  j0 = (int)fly;
  fx = __dsub_rn(gx, flx);
  fy = __dsub_rn(gy, fly);
}

// fraction (bits 0..30 of a scale-2^31 fixed-point value) as a float in
// [0, 1): the top 23 fraction bits become the mantissa of a number in [1, 2)
// (integer and logic ops only; no int-to-float conversion)
__device__ __forceinline__ float frac31(long long v) {
  const unsigned f = (unsigned)v & 0x7fffffffu;
  return __uint_as_float(0x3f800000u | (f >> 8)) - 1.0f;
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
  mlo = max(0, (int)floorf(vlo + off) - 1);
  mhi = min(ns, (int)ceilf(vhi + off) + 2);
  if (mhi < mlo) mhi = mlo;
}

// Plane value at (row iy, column ix); `tr`: the plane is stored transposed
// (column-major), so element (iy, ix) sits at ix * n + iy.
template <typename T>
__device__ __forceinline__ T pix2(const T* __restrict__ sl, int n, int iy, int ix, bool tr) {
  return (ix >= 0 && iy >= 0 && ix < n && iy < n)
             ? __ldg(sl + (tr ? (size_t)ix * n + iy : (size_t)iy * n + ix))
             : T(0);
}

// P from global memory (planes too large for shared memory).  The threads of
// a block are neighbouring detectors of one angle: at a given sample index
// they sit one cell apart along (cos, sin).  For steep angles (|sin| > |cos|)
// that is mostly along y, so their loads would touch one row each; given the
// transposed planes `pt` the block reads those instead and the same loads run
// along memory.  Same values, weights and summation order either way.
template <typename T>
__global__ void __launch_bounds__(128)
    k_project(const T* __restrict__ p, const T* __restrict__ pt, T* __restrict__ g,
              const T* __restrict__ sub, const T* __restrict__ mask,
              const double* __restrict__ tab, const float* __restrict__ tabf,
              const int32_t* __restrict__ tabi, int n, int nth, int ns, int nimg) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int l = blockIdx.y;
  const int j = blockIdx.z;
  const float csf = tabf[j], snf = tabf[nth + j];
  const bool tr = pt != nullptr && fabsf(snf) > fabsf(csf);
  const T* __restrict__ sl = (tr ? pt : p) + (size_t)l * n * n;
  int mlo = 0, mhi = 0;
  if (k < n) ray_range(csf, snf, k, n, ns, mlo, mhi);
  T acc = T(0);
  if constexpr (sizeof(T) == 8) {
    const double cs = tab[j], sn = tab[nth + j];
    const double dx = 2.0 / nimg, half = nimg / 2.0, L = (double)n / nimg;
    for (int m = mlo; m < mhi; ++m) {
      int i0, j0;
      double fx, fy;
      sample64(cs, sn, k, m, ns, dx, half, L, i0, j0, fx, fy);
      const double ofx = __dsub_rn(1.0, fx), ofy = __dsub_rn(1.0, fy);
      double b = __dmul_rn(__dmul_rn(ofx, ofy), pix2(sl, n, j0, i0, tr));
      b = __dadd_rn(b, __dmul_rn(__dmul_rn(fx, ofy), pix2(sl, n, j0, i0 + 1, tr)));
      b = __dadd_rn(b, __dmul_rn(__dmul_rn(ofx, fy), pix2(sl, n, j0 + 1, i0, tr)));
      b = __dadd_rn(b, __dmul_rn(__dmul_rn(fx, fy), pix2(sl, n, j0 + 1, i0 + 1, tr)));
      acc = __dadd_rn(acc, b);
    }
    if (k < n) {
      double out = __dmul_rn(dx, acc);
      const size_t o = ((size_t)j * n + l) * n + k;
      if (sub) out = out - sub[o];
      if (mask) out = out * mask[o];
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
    for (int m = mlo; m < mhi; ++m) {
      const int i0 = (int)(GX >> 31), j0 = (int)(GY >> 31);
      const float fx = frac31(GX), fy = frac31(GY);
      GX += dGX;
      GY += dGY;
      const float v00 = pix2(sl, n, j0, i0, tr), v10 = pix2(sl, n, j0, i0 + 1, tr);
      const float v01 = pix2(sl, n, j0 + 1, i0, tr), v11 = pix2(sl, n, j0 + 1, i0 + 1, tr);
      const float r0 = fmaf(fx, v10 - v00, v00);
      const float r1 = fmaf(fx, v11 - v01, v01);
      acc += fmaf(fy, r1 - r0, r0);
    }
    if (k < n) {
      float out = (2.0f / (float)nimg) * acc;
      const size_t o = ((size_t)j * n + l) * n + k;
      if (sub) out = out - sub[o];
      if (mask) out = out * mask[o];
      g[o] = out;
    }
  }
}

// P with the whole plane staged in shared memory behind a zero border of
// kPad points, so the bilinear corner loads need no bounds tests (used when
// the padded plane fits; one CTA per (plane, group of angles), threads over
// (angle, detector) pairs).  Same per-sample arithmetic as k_project.
constexpr int kPad = 3;
constexpr int kProjThreads = 1024;  // threads of the whole-plane kernel (8 angles x N rays)

// row pitch of the staged plane: at least n + 2 kPad, and 1 mod 32 so that the
// 32 rays of a warp, which cross the plane along one direction, fall on
// different shared-memory banks when they run along y
__host__ __device__ inline int plane_pitch(int n) {
  const int w = n + 2 * kPad;
  return w + ((33 - w % 32) % 32);
}

template <typename T>
__global__ void __launch_bounds__(kProjThreads)
    k_project_smem(const T* __restrict__ p, T* __restrict__ g, const T* __restrict__ sub,
                   const T* __restrict__ mask, const double* __restrict__ tab,
                   const float* __restrict__ tabf, const int32_t* __restrict__ tabi, int n,
                   int nth, int ns, int nimg, int group) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* s = reinterpret_cast<T*>(smem_raw);
  const int W = plane_pitch(n);  // row pitch; rows = n + 2 kPad
  const int l = blockIdx.x;
  const int ja = blockIdx.y * group, jb = min(nth, ja + group);
  const T* __restrict__ sl = p + (size_t)l * n * n;
  const int H = n + 2 * kPad;
  for (int yy = threadIdx.x / 32; yy < H; yy += blockDim.x / 32) {
    const int y = yy - kPad;
    for (int xx = threadIdx.x % 32; xx < W; xx += 32) {
      const int x = xx - kPad;
      s[yy * W + xx] = (x >= 0 && y >= 0 && x < n && y < n) ? __ldg(sl + (size_t)y * n + x) : T(0);
    }
  }
  __syncthreads();
  // corner (i0, j0) of the padded plane, clamped so that no load leaves it
  auto at = [&](int j0, int i0) -> int {
    const int jj = min(max(j0 + kPad, 0), H - 2), ii = min(max(i0 + kPad, 0), H - 2);
    return jj * W + ii;
  };
  const int work = (jb - ja) * n;
  for (int w = threadIdx.x; w < work; w += blockDim.x) {
    const int j = ja + w / n, k = w % n;
    int mlo, mhi;
    ray_range(tabf[j], tabf[nth + j], k, n, ns, mlo, mhi);
    T acc = T(0);
    if constexpr (sizeof(T) == 8) {
      const double cs = tab[j], sn = tab[nth + j];
      const double dx = 2.0 / nimg, half = nimg / 2.0, L = (double)n / nimg;
      for (int m = mlo; m < mhi; ++m) {
        int i0, j0;
        double fx, fy;
        sample64(cs, sn, k, m, ns, dx, half, L, i0, j0, fx, fy);
        const int o = at(j0, i0);
        const double ofx = __dsub_rn(1.0, fx), ofy = __dsub_rn(1.0, fy);
        double b = __dmul_rn(__dmul_rn(ofx, ofy), s[o]);
        b = __dadd_rn(b, __dmul_rn(__dmul_rn(fx, ofy), s[o + 1]));
        b = __dadd_rn(b, __dmul_rn(__dmul_rn(ofx, fy), s[o + W]));
        b = __dadd_rn(b, __dmul_rn(__dmul_rn(fx, fy), s[o + W + 1]));
        acc = __dadd_rn(acc, b);
      }
      double out = __dmul_rn(dx, acc);
      const size_t oo = ((size_t)j * n + l) * n + k;
      if (sub) out = out - sub[oo];
      if (mask) out = out * mask[oo];
      g[oo] = out;
    } else {
      const long long CS = tabi[j], SN = tabi[nth + j];
      const long long u2 = 2LL * k + 1 - n, v2 = 2LL * mlo + 1 - ns;
      const long long c2 = (long long)(n - 1) << 30;
      long long GX = c2 + u2 * CS - v2 * SN;
      long long GY = c2 + u2 * SN + v2 * CS;
      const long long dGX = -2 * SN, dGY = 2 * CS;
      for (int m = mlo; m < mhi; ++m) {
        const int i0 = (int)(GX >> 31), j0 = (int)(GY >> 31);
        const float fx = frac31(GX), fy = frac31(GY);
        GX += dGX;
        GY += dGY;
        const int o = at(j0, i0);
        const float v00 = s[o], v10 = s[o + 1], v01 = s[o + W], v11 = s[o + W + 1];
        const float r0 = fmaf(fx, v10 - v00, v00);
        const float r1 = fmaf(fx, v11 - v01, v01);
        acc += fmaf(fy, r1 - r0, r0);
      }
      float out = (2.0f / (float)nimg) * acc;
      const size_t oo = ((size_t)j * n + l) * n + k;
      if (sub) out = out - sub[oo];
      if (mask) out = out * mask[oo];
      g[oo] = out;
    }
  }
}

// FP32 P for planes too large for shared memory, band by band.  A CTA owns
// one plane and a group of angles whose rays all run the same way in y (cos
// >= 0, or cos < 0): it stages the plane in bands of bh rows (plus the zero
// border) and visits the bands in the order its rays cross them, so every ray
// still adds its samples in increasing m, the order of k_project.  Between
// bands each ray's next sample, end of range and running sum live in shared
// memory.  A sample belongs to the band of its lower row j0 (the first and
// last bands take the rows beyond), whose buffer also holds row j0 + 1.
__global__ void __launch_bounds__(1024)
    k_project_band(const float* __restrict__ p, float* __restrict__ g,
                   const float* __restrict__ sub, const float* __restrict__ mask,
                   const float* __restrict__ tabf, const int32_t* __restrict__ tabi, int n,
                   int nth, int ns, int nimg, int group, int jsplit, int bh, int nb) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int W = plane_pitch(n);
  const int HB = bh + 2 * kPad;  // rows of the band buffer
  float* s = reinterpret_cast<float*>(smem_raw);
  float* racc = s + (size_t)HB * W;
  int* rm = reinterpret_cast<int*>(racc + (size_t)group * n);  // next sample of each ray
  int* rend = rm + (size_t)group * n;                          // end of its sample range
  // angle groups vary fastest, so the CTAs resident together read the same
  // planes and the plane traffic hits L2
  const int l = blockIdx.y;
  const int g1 = (jsplit + group - 1) / group;
  int ja, jb;
  if ((int)blockIdx.x < g1) {
    ja = blockIdx.x * group;
    jb = min(jsplit, ja + group);
  } else {
    ja = jsplit + (blockIdx.x - g1) * group;
    jb = min(nth, ja + group);
  }
  const bool asc = ja < jsplit;
  const float* __restrict__ sl = p + (size_t)l * n * n;
  const int work = (jb - ja) * n;
  for (int w = threadIdx.x; w < work; w += blockDim.x) {
    const int j = ja + w / n, k = w % n;
    int mlo, mhi;
    ray_range(tabf[j], tabf[nth + j], k, n, ns, mlo, mhi);
    racc[w] = 0.0f;
    rm[w] = mlo;
    rend[w] = mhi;
  }
  for (int bi = 0; bi < nb; ++bi) {
    const int b = asc ? bi : nb - 1 - bi;
    const int y_lo = b * bh;  // first row of the band
    __syncthreads();
    for (int yy = threadIdx.x / 32; yy < HB; yy += blockDim.x / 32) {
      const int y = y_lo - kPad + yy;
      for (int xx = threadIdx.x % 32; xx < W; xx += 32) {
        const int x = xx - kPad;
        s[yy * W + xx] =
            (x >= 0 && y >= 0 && x < n && y < n) ? __ldg(sl + (size_t)y * n + x) : 0.0f;
      }
    }
    __syncthreads();
    // rows j0 of this band (the first and last bands take everything beyond)
    const int jlo = b == 0 ? INT_MIN : y_lo;
    const int jhi = b == nb - 1 ? INT_MAX : y_lo + bh;
    for (int w = threadIdx.x; w < work; w += blockDim.x) {
      const int j = ja + w / n, k = w % n;
      int m = rm[w];
      const int mhi = rend[w];
      if (m >= mhi) continue;
      float acc = racc[w];
      const long long CS = tabi[j], SN = tabi[nth + j];
      const long long u2 = 2LL * k + 1 - n, v2 = 2LL * m + 1 - ns;
      const long long c2 = (long long)(n - 1) << 30;
      long long GX = c2 + u2 * CS - v2 * SN;
      long long GY = c2 + u2 * SN + v2 * CS;
      const long long dGX = -2 * SN, dGY = 2 * CS;
      for (; m < mhi; ++m) {
        const int i0 = (int)(GX >> 31), j0 = (int)(GY >> 31);
        if (j0 < jlo || j0 >= jhi) break;
        const float fx = frac31(GX), fy = frac31(GY);
        GX += dGX;
        GY += dGY;
        // buffer offset of corner (i0, j0), clamped into the buffer
        const int jj = min(max(j0 - y_lo + kPad, 0), HB - 2);
        const int ii = min(max(i0 + kPad, 0), n + 2 * kPad - 2);
        const int o = jj * W + ii;
        const float v00 = s[o], v10 = s[o + 1], v01 = s[o + W], v11 = s[o + W + 1];
        const float r0 = fmaf(fx, v10 - v00, v00);
        const float r1 = fmaf(fx, v11 - v01, v01);
        acc += fmaf(fy, r1 - r0, r0);
      }
      racc[w] = acc;
      rm[w] = m;
    }
  }
  __syncthreads();
  for (int w = threadIdx.x; w < work; w += blockDim.x) {
    const int j = ja + w / n, k = w % n;
    const size_t oo = ((size_t)j * n + l) * n + k;
    float out = (2.0f / (float)nimg) * racc[w];
    if (sub) out = out - sub[oo];
    if (mask) out = out * mask[oo];
    g[oo] = out;
  }
}

// FP32 P by angle classes (even N, even n_angles = 2h), the forward
// counterpart of k_backproject_quad.  The bilinear samples of theta's
// lattice serve four angles: (1) theta's ray k is the sum over its samples m
// ("row" k); (2) theta + 90 deg's ray k' is the sum of "column" m = k' + koff
// (koff = (Ns - N)/2) over the lattice points k = -koff .. N + koff - 1 (its
// samples m' = (N + Ns)/2 - 1 - k); (3) pi - theta's ray k sums the mirror
// image x -> N-1-x of theta's row k (its sample m' is theta's Ns-1-m', so
// only the order of the terms differs); (4) pi/2 - theta's ray k' sums that
// mirror image's column k' + koff, by (2) applied to the pair (pi/2 - theta,
// pi - theta).  So the lattice spans Ns x Ns points, both indices shifted to
// 0 .. Ns-1 (kidx = k + koff): rows kidx in [koff, koff + N) and columns m in
// [koff, koff + N) are rays.  The mirror image of a sample uses the same
// corner row, fractions and weights, read at the mirrored columns.  Classes
// j = 0 and 2j = h have only the pair (1), (2).
// A CTA takes one plane and one class (several classes, one after the
// other, when the plane fits one band and is staged once).  Warp (kg, mg)
// owns the tiles of 32 lattice rows (lane = row) x 16 samples whose k-tile
// is kg mod KG and m-tile mg mod MG; tiles whose samples miss the plane (or the band) are skipped, and tiles
// whose samples all lie on it take a path without per-sample tests.  A lane's
// running sum over a tile is its row's partial sum; the column partials of an
// m-tile accumulate per lane over the warp's k-tiles, then one transposed
// butterfly over the lanes gives the 16 column sums.  The owner adds both to
// its partial sums in shared memory (rows per m-group, columns per k-group),
// and the groups are summed at the end.  The plane is staged band by band
// (one band when it fits) behind a zero border of 4 points, with rows of a
// pitch = 16 mod 32 words: the 32 lanes of a load lie along theta (direct
// image) or along its mirror, and this pitch keeps both near two wavefronts
// per load.  A sample belongs to the band of its lower corner row j0, the
// first and last bands taking the rows beyond.  Fixed order everywhere:
// deterministic, no atomics.
constexpr int kQuadMaxWarps = 16;
constexpr int kQPad = 4;  // zero border of the staged plane (keeps rows 16-byte aligned)

__host__ __device__ inline int quad_pitch(int n) {
  const int w = n + 2 * kQPad;
  return w + ((48 - w % 32) % 32);
}

constexpr int kQuadTM = 16;  // samples of a lattice tile (its rows: the 32 lanes)

// kQuadTM samples of one lattice row per lane (the lanes: 32 consecutive rows),
// both images; CHECK: skip the samples that do not exist or miss the plane
// or band (else every sample is known to touch it)
template <bool CHECK>
__device__ __forceinline__ void quad_tile(const float* __restrict__ sb, int W, int n,
                                          long long GX, long long GY, long long dGX,
                                          long long dGY, bool kin, int mlim, int jmin,
                                          unsigned jspan, float (&cv)[kQuadTM],
                                          float (&cm)[kQuadTM], float& rt, float& rm) {
  const int nm1 = n - 1;
#pragma unroll
  for (int i = 0; i < kQuadTM; ++i) {
    const int i0 = (int)(GX >> 32), j0 = (int)(GY >> 32);
    const unsigned lx = (unsigned)GX, ly = (unsigned)GY;
    GX += dGX;
    GY += dGY;
    if (!CHECK ||
        (kin && i < mlim && (unsigned)(j0 - jmin) <= jspan && (unsigned)(i0 + 1) <= (unsigned)n)) {
      const float fx = __uint_as_float(0x3f800000u | (lx >> 9)) - 1.0f;
      const float fy = __uint_as_float(0x3f800000u | (ly >> 9)) - 1.0f;
      const float* q = sb + j0 * W;
      const float v00 = q[i0], v10 = q[i0 + 1], v01 = q[i0 + W], v11 = q[i0 + W + 1];
      const int im = nm1 - i0;  // the mirror column N - 1 - i0
      const float a0 = q[im], b0 = q[im - 1], a1 = q[im + W], b1 = q[im + W - 1];
      const float r0 = fmaf(fx, v10 - v00, v00), r1 = fmaf(fx, v11 - v01, v01);
      const float q0 = fmaf(fx, b0 - a0, a0), q1 = fmaf(fx, b1 - a1, a1);
      const float v = fmaf(fy, r1 - r0, r0), vm = fmaf(fy, q1 - q0, q0);
      rt += v;
      rm += vm;
      cv[i] += v;
      cm[i] += vm;
    }
  }
}

__global__ void __launch_bounds__(kQuadMaxWarps * 32, 1)
    k_project_quad(const float* __restrict__ p, float* __restrict__ g,
                   const float* __restrict__ sub, const float* __restrict__ mask,
                   const int32_t* __restrict__ tabi, int n, int nth, int ns, int nimg, int tiles,
                   int kg_n, int mg_n, int bh, int nb, int cpb) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int W = quad_pitch(n);
  const int HB = bh + 2 * kQPad;  // rows of the band buffer
  const int TW = tiles * 32;      // lattice rows (and samples) rounded up to tiles
  float* s = reinterpret_cast<float*>(smem_raw);
  float* rowp = s + (size_t)HB * W;             // [mg][2][TW]: row sums of both images
  float* colp = rowp + (size_t)mg_n * 2 * TW;   // [kg][2][TW]: column sums of both images
  const int hh = nth / 2;
  const int ncls = nth / 4 + 1;
  const int l = blockIdx.y;  // plane
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nthreads = blockDim.x, nwarps = nthreads / 32;
  const int kg = warp % kg_n, mg = warp / kg_n;
  const float* __restrict__ sl = p + (size_t)l * n * n;
  const int koff = (ns - n) / 2;

  // stage rows y_lo - 4 .. y_lo + bh + 3 of the plane (zero outside it)
  auto stage = [&](int y_lo) {
    if ((n & 3) == 0 && ((uintptr_t)p & 15) == 0) {
      // rows of W / 4 float4: column 4q .. 4q+3 holds the plane's 4q-4 .. 4q-1
      const int W4 = W / 4, n4 = n / 4;
      for (int yy = warp; yy < HB; yy += nwarps) {
        const int y = y_lo - kQPad + yy;
        float4* dst = reinterpret_cast<float4*>(s + (size_t)yy * W);
        if (y >= 0 && y < n) {
          const float4* src = reinterpret_cast<const float4*>(sl + (size_t)y * n);
          for (int q = lane; q < W4; q += 32)
            dst[q] = (q >= 1 && q <= n4) ? __ldg(src + q - 1) : make_float4(0.f, 0.f, 0.f, 0.f);
        } else {
          for (int q = lane; q < W4; q += 32) dst[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
    } else {
      for (int yy = warp; yy < HB; yy += nwarps) {
        const int y = y_lo - kQPad + yy;
        for (int xx = lane; xx < W; xx += 32) {
          const int x = xx - kQPad;
          s[yy * W + xx] =
              (x >= 0 && y >= 0 && x < n && y < n) ? __ldg(sl + (size_t)y * n + x) : 0.0f;
        }
      }
    }
  };
  if (nb == 1) stage(0);  // one band: staged once for all classes of the CTA

  const int c1 = min(ncls, (int)(blockIdx.x + 1) * cpb);
  for (int j = blockIdx.x * cpb; j < c1; ++j) {  // angle class: theta_j in [0, 45] degrees
    const bool four = j != 0 && 2 * j != hh;
    __syncthreads();  // the previous class's sums are read
    for (int i = tid; i < (mg_n + kg_n) * 2 * TW; i += nthreads) rowp[i] = 0.0f;
    // fixed-point coordinates at twice the scale of the other FP32 kernels
    // (2^32 per cell): the corner index is the high word and the fraction the
    // low word, the same corners and fraction bits as frac31 of the 2^31 form.
    // cos, sin >= 0: x grows along the rows and falls along the samples, y
    // grows along both, so a tile's extremes sit at known corners
    const long long CS = 2LL * tabi[j], SN = 2LL * tabi[nth + j];
    const long long c2 = (long long)(n - 1) << 31;
    const long long dGX = -2 * SN, dGY = 2 * CS;
    for (int b = 0; b < nb; ++b) {
      const int y_lo = b * bh;
      if (nb > 1) {
        __syncthreads();  // the previous band's readers are done
        stage(y_lo);
      }
      __syncthreads();
      // corner rows whose samples can be nonzero and belong to this band
      const int jmin = b == 0 ? -1 : y_lo;
      const int jmax = b == nb - 1 ? n - 1 : min(y_lo + bh, n) - 1;
      const unsigned jspan = (unsigned)(jmax - jmin);
      const float* sb = s + (kQPad - y_lo) * W + kQPad;  // element (row j0, column i0)
      const int mtiles = (ns + kQuadTM - 1) / kQuadTM;
      for (int mt = mg; mt < mtiles; mt += mg_n) {
        const int m0 = mt * kQuadTM;
        const long long v2 = 2LL * m0 + 1 - ns, vb = v2 + 2 * (kQuadTM - 1);
        const long long xa = c2 - vb * SN, xb = c2 - v2 * SN;  // x at the low / high samples
        const long long ya = c2 + v2 * CS, yb = c2 + vb * CS;  // y at them
        const int mlim = ns - m0;  // samples m0 + i with i < mlim exist
        float cv[kQuadTM], cm[kQuadTM];
#pragma unroll
        for (int i = 0; i < kQuadTM; ++i) cv[i] = cm[i] = 0.0f;
        bool any = false;
        for (int kt = kg; kt < tiles; kt += kg_n) {
          const int r0i = kt * 32;  // first lattice row of the tile
          const long long ua = 2LL * (r0i - koff) + 1 - n, ub = ua + 62;
          const long long xlo = (xa + ua * CS) >> 32, xhi = (xb + ub * CS) >> 32;
          const long long ylo = (ya + ua * SN) >> 32, yhi = (yb + ub * SN) >> 32;
          // no sample of the tile touches the plane within this band
          if (xhi < -1 || xlo > n - 1 || yhi < jmin || ylo > jmax) continue;
          any = true;
          const int kidx = r0i + lane;
          const long long u2 = ua + 2 * lane;
          const long long GX = c2 + u2 * CS - v2 * SN;
          const long long GY = c2 + u2 * SN + v2 * CS;
          float rt = 0.0f, rm = 0.0f;
          if (xlo >= -1 && xhi <= n - 1 && ylo >= jmin && yhi <= jmax && r0i + 31 < ns &&
              mlim >= kQuadTM)
            quad_tile<false>(sb, W, n, GX, GY, dGX, dGY, true, kQuadTM, jmin, jspan, cv, cm, rt,
                             rm);
          else
            quad_tile<true>(sb, W, n, GX, GY, dGX, dGY, kidx < ns, mlim, jmin, jspan, cv, cm, rt,
                            rm);
          float* rp = rowp + (size_t)mg * 2 * TW + kidx;
          rp[0] += rt;
          rp[TW] += rm;
        }
        if (!any) continue;
        // column sums over the 32 lanes: fold the lane groups above the tile
        // length, then a transposed butterfly over the kQuadTM lanes of each
        // group leaves the sum of sample t mod kQuadTM in lane t
#pragma unroll
        for (int sh = 16; sh >= kQuadTM; sh >>= 1) {
#pragma unroll
          for (int i = 0; i < kQuadTM; ++i) {
            cv[i] += __shfl_xor_sync(0xffffffffu, cv[i], sh);
            cm[i] += __shfl_xor_sync(0xffffffffu, cm[i], sh);
          }
        }
#pragma unroll
        for (int sh = kQuadTM / 2; sh >= 1; sh >>= 1) {
          const bool up = (lane & sh) != 0;
#pragma unroll
          for (int i = 0; i < sh; ++i) {
            const float sv = up ? cv[i] : cv[i + sh], kv = up ? cv[i + sh] : cv[i];
            const float sm = up ? cm[i] : cm[i + sh], km = up ? cm[i + sh] : cm[i];
            cv[i] = kv + __shfl_xor_sync(0xffffffffu, sv, sh);
            cm[i] = km + __shfl_xor_sync(0xffffffffu, sm, sh);
          }
        }
        if (lane < kQuadTM) {
          float* cp = colp + (size_t)kg * 2 * TW + m0 + lane;
          cp[0] += cv[0];
          cp[TW] += cm[0];
        }
      }
    }
    __syncthreads();
    const float scale = 2.0f / (float)nimg;
    const int nout = four ? 4 : 2;
    for (int w = tid; w < nout * n; w += nthreads) {
      const int which = w / n, kk = w % n;
      // row sums of theta and pi - theta; column sums of theta + 90 and pi/2 - theta
      const bool row = which == 0 || which == 2;
      const float* src = (row ? rowp : colp) + (which >= 2 ? TW : 0) + koff + kk;
      const int groups = row ? mg_n : kg_n;
      float acc = 0.0f;
      for (int q = 0; q < groups; ++q) acc += src[(size_t)q * 2 * TW];
      const int ang = which == 0 ? j : which == 1 ? j + hh : which == 2 ? nth - j : hh - j;
      const size_t oo = ((size_t)ang * n + l) * n + kk;
      float out = scale * acc;
      if (sub) out = out - sub[oo];
      if (mask) out = out * mask[oo];
      g[oo] = out;
    }
  }
}

// P^T, voxel-driven gather (deterministic, no atomics).  For each angle the
// voxel's position in the rotated frame, kk (detector units) and mm (sample
// units), is split into integer and fractional parts; the samples that can
// reach the voxel are the 3 x 3 candidates k = kb .. kb + 2, m = mb .. mb + 2
// around it (|k - kk|, |m - mm| < sqrt 2).  Each contributes hat(a) hat(b) of
// its offset (a, b) in the grid frame, the bilinear weight P gives the voxel;
// a and b step by (cos, sin) and (-sin, cos) between candidates.
template <typename T>
__device__ __forceinline__ T hat1(T a) {
  const T v = T(1) - fabs(a);
  return v > T(0) ? v : T(0);
}

// FP32 hat: 1 - |a| <= 1 always, so clamping to [0, 1] is max(0, .); one
// saturating add on the FMA pipe instead of an add and a min/max on the ALU
__device__ __forceinline__ float hat1f(float a) { return __saturatef(1.0f - fabsf(a)); }
template <>
__device__ __forceinline__ float hat1<float>(float a) {
  return hat1f(a);
}

constexpr int kAngleChunk = 1024;

template <typename T>
__global__ void __launch_bounds__(256)
    k_backproject2(const T* __restrict__ g, T* __restrict__ h, const T* __restrict__ scale,
                   const double* __restrict__ tab, const float* __restrict__ tabf,
                   const int32_t* __restrict__ tabi, int n, int nth, int ns, int nimg, T mult) {
  __shared__ T s_cs[kAngleChunk], s_sn[kAngleChunk];
  __shared__ int s_CS[kAngleChunk], s_SN[kAngleChunk];
  const int ix = blockIdx.x * 32 + threadIdx.x;
  const int iy = blockIdx.y * 8 + threadIdx.y;
  const int l = blockIdx.z;
  const int tid = threadIdx.y * 32 + threadIdx.x;
  const bool in = ix < n && iy < n;
  T acc = T(0);
  for (int ja = 0; ja < nth; ja += kAngleChunk) {
    const int jn = min(kAngleChunk, nth - ja);
    __syncthreads();
    for (int t = tid; t < jn; t += 256) {
      if constexpr (sizeof(T) == 8) {
        s_cs[t] = tab[ja + t];
        s_sn[t] = tab[nth + ja + t];
      } else {
        s_cs[t] = tabf[ja + t];
        s_sn[t] = tabf[nth + ja + t];
      }
      s_CS[t] = tabi[ja + t];
      s_SN[t] = tabi[nth + ja + t];
    }
    __syncthreads();
    if (!in) continue;
    for (int t = 0; t < jn; ++t) {
      const T cs = s_cs[t], sn = s_sn[t];
      int KI, MI;
      T fk, fm;
      if constexpr (sizeof(T) == 8) {
        const double X = ix - 0.5 * (n - 1), Y = iy - 0.5 * (n - 1);
        const double kk = fma(X, cs, Y * sn) + 0.5 * (n - 1);
        const double mm = fma(Y, cs, -X * sn) + 0.5 * (ns - 1);
        const double fkk = floor(kk), fmm = floor(mm);
        KI = (int)fkk;
        MI = (int)fmm;
        fk = kk - fkk;
        fm = mm - fmm;
      } else {
        // fixed point, scale 2^31: exact integer parts, fractions to ~1e-9
        const int X2 = 2 * ix - (n - 1), Y2 = 2 * iy - (n - 1);
        const int CS = s_CS[t], SN = s_SN[t];
        const long long KK = (long long)X2 * CS + (long long)Y2 * SN + ((long long)(n - 1) << 30);
        const long long MM = (long long)Y2 * CS - (long long)X2 * SN + ((long long)(ns - 1) << 30);
        KI = (int)(KK >> 31);
        MI = (int)(MM >> 31);
        fk = frac31(KK);
        fm = frac31(MM);
      }
      const int hk = fk >= T(0.5) ? 1 : 0, hm = fm >= T(0.5) ? 1 : 0;
      const int kb = KI - 1 + hk, mb = MI - 1 + hm;
      const T du0 = T(hk - 1) - fk, dv0 = T(hm - 1) - fm;  // offsets of candidate (kb, mb)
      const T a0 = du0 * cs - dv0 * sn, b0 = du0 * sn + dv0 * cs;
      const bool m0 = mb >= 0 && mb < ns, m1 = mb + 1 >= 0 && mb + 1 < ns,
                 m2 = mb + 2 >= 0 && mb + 2 < ns;
      const T* __restrict__ row = g + ((size_t)(ja + t) * n + l) * n;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const int k = kb + i;
        if (k < 0 || k >= n) continue;
        const T ai = a0 + T(i) * cs, bi = b0 + T(i) * sn;
        T w = T(0);
        if (m0) w += hat1(ai) * hat1(bi);
        if (m1) w += hat1(ai - sn) * hat1(bi + cs);
        if (m2) w += hat1(ai - T(2) * sn) * hat1(bi + T(2) * cs);
        acc += w * __ldg(row + k);
      }
    }
  }
  if (!in) return;
  const size_t o = ((size_t)l * n + iy) * n + ix;
  T out = (T(2) / T(nimg)) * acc;
  if (scale) out *= scale[o];
  if (mult != T(1)) out *= mult;
  h[o] = out;
}

// FP32 P^T with the angles paired as theta_j and theta_j + 90 degrees (even
// n_angles, even N).  With equal detector and sample spacing the rays of
// theta + 90 degrees sample exactly the points of theta's lattice: detector
// k' = m - (Ns - N)/2 and sample m' = (N + Ns)/2 - 1 - k of the rotated angle
// is the point (k, m) of theta, in the fixed-point coordinates of P as well
// (the tables hold cos(theta + 90) = -sin(theta), sin(theta + 90) = cos(theta)
// to the rounding of the angle itself).  So the 3 x 3 candidate weights w_ij
// that a voxel gets from theta's samples serve both angles: theta's detector
// kb + i takes the row sum over valid samples, the rotated angle's detector
// k'(mb + j) the column sum.  Half the weight evaluations of k_backproject2.
__global__ void __launch_bounds__(256)
    k_backproject_pair(const float* __restrict__ g, float* __restrict__ h,
                       const float* __restrict__ scale, const float* __restrict__ tabf,
                       const int32_t* __restrict__ tabi, int n, int nth, int ns, int nimg,
                       float mult) {
  __shared__ float s_cs[kAngleChunk], s_sn[kAngleChunk];
  __shared__ int s_CS[kAngleChunk], s_SN[kAngleChunk];
  const int ix = blockIdx.x * 32 + threadIdx.x;
  const int iy = blockIdx.y * 8 + threadIdx.y;
  const int l = blockIdx.z;
  const int tid = threadIdx.y * 32 + threadIdx.x;
  const bool in = ix < n && iy < n;
  const int half = nth / 2;
  const int koff = (ns - n) / 2;       // k' = m - koff
  const int mrot = (n + ns) / 2 - 1;   // m' = mrot - k
  const int X2 = 2 * ix - (n - 1), Y2 = 2 * iy - (n - 1);
  float acc = 0.0f;
  for (int ja = 0; ja < half; ja += kAngleChunk) {
    const int jn = min(kAngleChunk, half - ja);
    __syncthreads();
    for (int t = tid; t < jn; t += 256) {
      s_cs[t] = tabf[ja + t];
      s_sn[t] = tabf[nth + ja + t];
      s_CS[t] = tabi[ja + t];
      s_SN[t] = tabi[nth + ja + t];
    }
    __syncthreads();
    if (!in) continue;
    for (int t = 0; t < jn; ++t) {
      const float cs = s_cs[t], sn = s_sn[t];
      const int CS = s_CS[t], SN = s_SN[t];
      const long long KK = (long long)X2 * CS + (long long)Y2 * SN + ((long long)(n - 1) << 30);
      const long long MM = (long long)Y2 * CS - (long long)X2 * SN + ((long long)(ns - 1) << 30);
      const int KI = (int)(KK >> 31), MI = (int)(MM >> 31);
      const float fk = frac31(KK), fm = frac31(MM);
      const int hk = fk >= 0.5f ? 1 : 0, hm = fm >= 0.5f ? 1 : 0;
      const int kb = KI - 1 + hk, mb = MI - 1 + hm;
      const float du0 = (float)(hk - 1) - fk, dv0 = (float)(hm - 1) - fm;
      const float a0 = du0 * cs - dv0 * sn, b0 = du0 * sn + dv0 * cs;
      // validity of theta's samples mb + jj and of the rotated angle's
      // samples (its m' = mrot - k) as 0/1 factors
      float mv[3], mv2[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        mv[q] = (unsigned)(mb + q) < (unsigned)ns ? 1.0f : 0.0f;
        mv2[q] = (unsigned)(mrot - (kb + q)) < (unsigned)ns ? 1.0f : 0.0f;
      }
      float r[3] = {0.0f, 0.0f, 0.0f}, cc[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int jj = 0; jj < 3; ++jj) {
          const float a = a0 + (float)i * cs - (float)jj * sn;
          const float b = b0 + (float)i * sn + (float)jj * cs;
          const float w = hat1f(a) * hat1f(b);
          r[i] = fmaf(w, mv[jj], r[i]);
          cc[jj] = fmaf(w, mv2[i], cc[jj]);
        }
      const float* __restrict__ row = g + ((size_t)(ja + t) * n + l) * n;
      const float* __restrict__ row2 = g + ((size_t)(ja + t + half) * n + l) * n;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const int k = kb + i;
        if ((unsigned)k < (unsigned)n) acc = fmaf(r[i], __ldg(row + k), acc);
      }
#pragma unroll
      for (int jj = 0; jj < 3; ++jj) {
        const int k2 = mb + jj - koff;
        if ((unsigned)k2 < (unsigned)n) acc = fmaf(cc[jj], __ldg(row2 + k2), acc);
      }
    }
  }
  if (!in) return;
  const size_t o = ((size_t)l * n + iy) * n + ix;
  float out = (2.0f / (float)nimg) * acc;
  if (scale) out *= scale[o];
  if (mult != 1.0f) out *= mult;
  h[o] = out;
}

// The 3 x 3 candidate weights of one voxel for angle theta (fixed-point
// frame KK, MM), reduced to row sums over theta's valid samples (r) and
// column sums over the rotated angle's valid samples (c), with the first
// candidate detector kb and sample mb (see k_backproject_pair).
struct Sums3 {
  float r[3], c[3];
  int kb, mb;
};

// IN: the voxel lies within (N - 6) / 2 grid units of the plane's centre,
// where every candidate detector and sample of every angle exists (its
// rotated coordinates stay within (N - 5) / 2), so no validity factors.
template <bool IN>
__device__ __forceinline__ Sums3 candidate_sums(long long KK, long long MM, float cs, float sn,
                                                int ns, int mrot) {
  Sums3 o;
  const int KI = (int)(KK >> 31), MI = (int)(MM >> 31);
  const float fk = frac31(KK), fm = frac31(MM);
  const int hk = fk >= 0.5f ? 1 : 0, hm = fm >= 0.5f ? 1 : 0;
  o.kb = KI - 1 + hk;
  o.mb = MI - 1 + hm;
  const float du0 = (float)(hk - 1) - fk, dv0 = (float)(hm - 1) - fm;
  const float a0 = du0 * cs - dv0 * sn, b0 = du0 * sn + dv0 * cs;
  float mv[3], mv2[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    if (!IN) {
      mv[q] = (unsigned)(o.mb + q) < (unsigned)ns ? 1.0f : 0.0f;
      mv2[q] = (unsigned)(mrot - (o.kb + q)) < (unsigned)ns ? 1.0f : 0.0f;
    }
    o.r[q] = 0.0f;
    o.c[q] = 0.0f;
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int jj = 0; jj < 3; ++jj) {
      const float a = a0 + (float)i * cs - (float)jj * sn;
      const float b = b0 + (float)i * sn + (float)jj * cs;
      const float w = hat1f(a) * hat1f(b);
      if (IN) {
        o.r[i] += w;
        o.c[jj] += w;
      } else {
        o.r[i] = fmaf(w, mv[jj], o.r[i]);
        o.c[jj] = fmaf(w, mv2[i], o.c[jj]);
      }
    }
  return o;
}

// acc += sum_i r_i row[kb + i] + sum_j c_j row2[mb + j - koff] (valid detectors)
template <bool IN>
__device__ __forceinline__ float apply_sums(const Sums3& s, const float* __restrict__ row,
                                            const float* __restrict__ row2, int n, int koff,
                                            float acc) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const int k = s.kb + i;
    if (IN || (unsigned)k < (unsigned)n) acc = fmaf(s.r[i], __ldg(row + k), acc);
  }
#pragma unroll
  for (int jj = 0; jj < 3; ++jj) {
    const int k2 = s.mb + jj - koff;
    if (IN || (unsigned)k2 < (unsigned)n) acc = fmaf(s.c[jj], __ldg(row2 + k2), acc);
  }
  return acc;
}

// The angle classes of k_backproject_quad for one voxel pair (u, u').
template <bool IN>
__device__ __forceinline__ void bp_quad_classes(const float* __restrict__ gl, size_t rows, int n,
                                                int nth, int ns, int hh, int nclass, int koff,
                                                int mrot, long long X2, long long Y2,
                                                long long ck, long long cm, bool in, int tid,
                                                const float* __restrict__ tabf,
                                                const int32_t* __restrict__ tabi, float* s_cs,
                                                float* s_sn, int* s_CS, int* s_SN, float& acc_u,
                                                float& acc_m) {
  for (int ja = 0; ja < nclass; ja += kAngleChunk) {
    const int jn = min(kAngleChunk, nclass - ja);
    __syncthreads();
    for (int t = tid; t < jn; t += 256) {
      s_cs[t] = tabf[ja + t];
      s_sn[t] = tabf[nth + ja + t];
      s_CS[t] = tabi[ja + t];
      s_SN[t] = tabi[nth + ja + t];
    }
    __syncthreads();
    if (!in) continue;
    for (int t = 0; t < jn; ++t) {
      const int j = ja + t;
      const float cs = s_cs[t], sn = s_sn[t];
      const long long CS = s_CS[t], SN = s_SN[t];
      const long long A = X2 * CS, B = Y2 * SN, C = Y2 * CS, D = X2 * SN;
      const Sums3 su = candidate_sums<IN>(A + B + ck, C - D + cm, cs, sn, ns, mrot);
      const Sums3 sm = candidate_sums<IN>(-A + B + ck, C + D + cm, cs, sn, ns, mrot);
      const float* __restrict__ r0 = gl + (size_t)j * rows;         // theta_j
      const float* __restrict__ r1 = gl + (size_t)(j + hh) * rows;  // theta_j + 90
      acc_u = apply_sums<IN>(su, r0, r1, n, koff, acc_u);
      acc_m = apply_sums<IN>(sm, r0, r1, n, koff, acc_m);
      if (j != 0 && 2 * j != hh) {
        const float* __restrict__ r2 = gl + (size_t)(nth - j) * rows;  // pi - theta_j
        const float* __restrict__ r3 = gl + (size_t)(hh - j) * rows;   // pi/2 - theta_j
        acc_m = apply_sums<IN>(su, r2, r3, n, koff, acc_m);
        acc_u = apply_sums<IN>(sm, r2, r3, n, koff, acc_u);
      }
    }
  }
}

// FP32 P^T using two exact symmetries of the sample lattices (even N, even
// n_angles = 2h).  (1) theta + 90 deg samples theta's lattice points (see
// k_backproject_pair).  (2) pi - theta samples the mirror image x -> N-1-x of
// theta's lattice with the sample index reversed (m -> Ns-1-m), which keeps
// the detector index and the row sums; so the weight sums a voxel u gets at
// theta are those its mirror u' gets at pi - theta, and (through (1) for the
// pair pi/2 - theta, pi - theta) at pi/2 - theta with the same column sums and
// detectors.  A thread owns u and u': for each angle class j = 1 .. h/2 with
// 2j != h it evaluates the weights of u and u' at theta_j once and applies
// each set to four angles {j, j + h, 2h - j, h - j}; j = 0 and j = h/2 (0 and
// 45 degrees) have only the pair (j, j + h).  A quarter of the weight
// evaluations of k_backproject2.  In fixed point the mirror frame is exact
// (KK' = -X2 CS + Y2 SN + c, MM' = Y2 CS + X2 SN + c); the tables of
// pi - theta and pi/2 - theta agree with -cos, sin and sin, cos of theta to the
// rounding of the angles themselves.
__global__ void __launch_bounds__(256)
    k_backproject_quad(const float* __restrict__ g, float* __restrict__ h,
                       const float* __restrict__ scale, const float* __restrict__ tabf,
                       const int32_t* __restrict__ tabi, int n, int nth, int ns, int nimg,
                       float mult) {
  __shared__ float s_cs[kAngleChunk], s_sn[kAngleChunk];
  __shared__ int s_CS[kAngleChunk], s_SN[kAngleChunk];
  const int ix = blockIdx.x * 32 + threadIdx.x;  // voxel u; its mirror is n - 1 - ix
  const int iy = blockIdx.y * 8 + threadIdx.y;
  const int l = blockIdx.z;
  const int tid = threadIdx.y * 32 + threadIdx.x;
  const int nh = n / 2;
  const bool in = ix < nh && iy < n;
  const int hh = nth / 2;
  const int nclass = hh / 2 + 1;        // classes j = 0 .. hh/2
  const int koff = (ns - n) / 2;
  const int mrot = (n + ns) / 2 - 1;
  const long long X2 = 2 * ix - (n - 1), Y2 = 2 * iy - (n - 1);
  const long long ck = (long long)(n - 1) << 30, cm = (long long)(ns - 1) << 30;
  const size_t rows = (size_t)n * n;    // stride between the angles' data
  const float* __restrict__ gl = g + (size_t)l * n;
  // the CTA's voxels (and their mirrors) all within (N - 6) / 2 of the centre:
  // the loop without validity tests
  const float cc = 0.5f * (float)(n - 1);
  const float x0 = (float)(blockIdx.x * 32), x1 = (float)min((int)blockIdx.x * 32 + 31, nh - 1);
  const float y0 = (float)(blockIdx.y * 8), y1 = (float)min((int)blockIdx.y * 8 + 7, n - 1);
  const float dxm = fmaxf(fabsf(x0 - cc), fabsf(x1 - cc)), dym = fmaxf(fabsf(y0 - cc), fabsf(y1 - cc));
  const float rin = 0.5f * (float)(n - 6);
  const bool inner = n > 6 && dxm * dxm + dym * dym <= rin * rin;
  float acc_u = 0.0f, acc_m = 0.0f;
  if (inner)
    bp_quad_classes<true>(gl, rows, n, nth, ns, hh, nclass, koff, mrot, X2, Y2, ck, cm, in, tid,
                          tabf, tabi, s_cs, s_sn, s_CS, s_SN, acc_u, acc_m);
  else
    bp_quad_classes<false>(gl, rows, n, nth, ns, hh, nclass, koff, mrot, X2, Y2, ck, cm, in, tid,
                           tabf, tabi, s_cs, s_sn, s_CS, s_SN, acc_u, acc_m);
  if (!in) return;
  const float f = 2.0f / (float)nimg;
  const size_t ou = ((size_t)l * n + iy) * n + ix;
  const size_t om = ((size_t)l * n + iy) * n + (n - 1 - ix);
  float out_u = f * acc_u, out_m = f * acc_m;
  if (scale) {
    out_u *= scale[ou];
    out_m *= scale[om];
  }
  if (mult != 1.0f) {
    out_u *= mult;
    out_m *= mult;
  }
  h[ou] = out_u;
  h[om] = out_m;
}

// Lambda on rows of n detectors.  A CTA computes the taps once (FP64, then
// rounded to T) and walks rows; each row sits in shared memory between n
// zeros on either side, so out-of-range neighbours read as zero (the same
// sums, term for term, as testing the range).
template <typename T>
__global__ void __launch_bounds__(128)
    k_ramp(const T* __restrict__ r, T* __restrict__ out, const T* __restrict__ mask, int n,
           int nimg, int rows) {
  extern __shared__ unsigned char smem_raw[];
  T* tap = reinterpret_cast<T*>(smem_raw);  // tap[d] for d < n (odd d nonzero)
  T* row = tap + n;                         // zeros, the row, zeros: 3n
  const double dxi = 2.0 / nimg;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double t;
    if (i == 0)
      t = 1.0 / (8.0 * dxi);
    else if (i % 2 == 0)
      t = 0.0;
    else
      t = -1.0 / (2.0 * kPi * kPi * (double)i * (double)i * dxi);
    tap[i] = (T)t;
    row[i] = T(0);
    row[2 * n + i] = T(0);
  }
  const T* rc = row + n;
  for (int rw = blockIdx.x; rw < rows; rw += gridDim.x) {
    const size_t base = (size_t)rw * n;
    __syncthreads();  // the previous row is read (and the taps and zeros written)
    for (int i = threadIdx.x; i < n; i += blockDim.x) row[n + i] = r[base + i];
    __syncthreads();
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
      T acc = tap[0] * rc[k];
      for (int d = 1; d < n; d += 2) acc += tap[d] * (rc[k - d] + rc[k + d]);
      if (mask) acc = acc * mask[base + k];
      out[base + k] = acc;
    }
  }
}

// out[l][x][y] = in[l][y][x] for every plane l (32 x 32 tiles through shared memory)
template <typename T>
__global__ void __launch_bounds__(256) k_transpose_planes(const T* __restrict__ in,
                                                          T* __restrict__ out, int n) {
  __shared__ T t[32][33];
  const size_t off = (size_t)blockIdx.z * n * n;
  const int x0 = blockIdx.x * 32, y0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int y = y0 + r, x = x0 + threadIdx.x;
    if (x < n && y < n) t[r][threadIdx.x] = in[off + (size_t)y * n + x];
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int x = x0 + r, y = y0 + threadIdx.x;
    if (x < n && y < n) out[off + (size_t)x * n + y] = t[threadIdx.x][r];
  }
}

__global__ void k_debug_samples(int count, const int32_t* __restrict__ jkm, int32_t* __restrict__ ij,
                                double* __restrict__ f, const double* __restrict__ tab, int n,
                                int nth, int ns, int nimg) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count) return;
  const int j = jkm[3 * t], k = jkm[3 * t + 1], m = jkm[3 * t + 2];
  if (j < 0 || j >= nth) return;
  int i0, j0;
  double fx, fy;
  sample64(tab[j], tab[nth + j], k, m, ns, 2.0 / nimg, nimg / 2.0, (double)n / nimg, i0, j0, fx,
           fy);
  ij[2 * t] = i0;
  ij[2 * t + 1] = j0;
  f[2 * t] = fx;
  f[2 * t + 1] = fy;
}

}  // namespace

static size_t project_smem_bytes(const Plan& pl) {
  return (size_t)plane_pitch(pl.n) * (pl.n + 2 * kPad) * pl.esize;
}

// FFPAT_BACKPROJECT_QUAD=0 turns the four-angle transpose off (a comparison knob)
static bool backproject_quad_off() {
  static const bool off = [] {
    const char* e = getenv("FFPAT_BACKPROJECT_QUAD");
    return e && e[0] == '0';
  }();
  return off;
}

// FFPAT_BACKPROJECT_PAIR=0 turns both multi-angle transposes off: the per-angle gather runs
static bool backproject_pair_off() {
  static const bool off = [] {
    const char* e = getenv("FFPAT_BACKPROJECT_PAIR");
    return e && e[0] == '0';
  }();
  return off;
}

// FFPAT_PROJECT_BAND=0 turns the banded projection off (a comparison knob)
static bool project_band_off() {
  static const bool off = [] {
    const char* e = getenv("FFPAT_PROJECT_BAND");
    return e && e[0] == '0';
  }();
  return off;
}

// The banded projection's shape: a group of angles whose per-ray state (sum
// and sample range) takes <= 48 KB, and bands of bh >= 16 rows, so that one
// CTA stays within ~110 KB of shared memory (two per SM).  False if the whole
// plane fits (the one-pass kernel) or no such band fits (global memory).
static bool band_plan(const Plan& pl, int* group, int* bh, int* nb, size_t* sm) {
  // FP64 projections are bound by the FP64 pipes, not by loads: measured on
  // GB300 the banded kernel gains nothing there (656 ms either way at 384^3, 180
  // angles) and loses at 256^3, so FP64 keeps the global-memory kernel
  if (pl.esize != 4 || project_smem_bytes(pl) <= 200 * 1024 || project_band_off()) return false;
  const int W = plane_pitch(pl.n);
  int gr = 8;
  while (gr > 1 && (size_t)gr * pl.n * (pl.esize + 8) > 48 * 1024) gr /= 2;
  const size_t state = (size_t)gr * pl.n * (pl.esize + 8);
  const size_t budget = 110 * 1024;
  const long long rows =
      state < budget ? (long long)((budget - state) / ((size_t)W * pl.esize)) - 2 * kPad : 0;
  if (rows < 16) return false;
  *group = gr;
  *nb = (int)((pl.n + rows - 1) / rows);
  *bh = (pl.n + *nb - 1) / *nb;
  *sm = (size_t)(*bh + 2 * kPad) * W * pl.esize + state;
  return true;
}

// FFPAT_PROJECT_QUAD=0 turns the angle-class projection off (a comparison knob)
static bool project_quad_off() {
  static const bool off = [] {
    const char* e = getenv("FFPAT_PROJECT_QUAD");
    return e && e[0] == '0';
  }();
  return off;
}

// Shape of the angle-class projection (FP32, even N, even angle count): a
// lattice of `tiles` x `tiles` tiles of 32 x 32, warps kg x mg, and the plane
// in nb bands of bh rows.  When the plane fits with the partial sums in half
// the shared memory of an SM, one band and 2 x 4 warps (two CTAs per SM);
// else 4 x 4 warps and bands as tall as the rest of 220 KB allows.
constexpr size_t kQuadSmem = 220 * 1024;

static bool quad_plan(const Plan& pl, int* tiles, int* kg, int* mg, int* bh, int* nb,
                      size_t* sm, int* cpb) {
  if (pl.esize != 4 || pl.n % 2 != 0 || pl.nth % 2 != 0 || project_quad_off()) return false;
  const int T = (pl.ns + 31) / 32;
  const size_t W = (size_t)quad_pitch(pl.n);
  auto state = [&](int g1, int g2) { return (size_t)(g1 + g2) * 2 * T * 32 * 4; };
  int KG = 2, MG = 4, rows_b = pl.n, nbands = 1;
  size_t need = (size_t)(pl.n + 2 * kQPad) * W * 4 + state(KG, MG);
  if (need > 110 * 1024) {
    KG = 4;
    MG = 4;
    const size_t st = state(KG, MG);
    need = (size_t)(pl.n + 2 * kQPad) * W * 4 + st;
    if (need > kQuadSmem) {
      const long long rows = st < kQuadSmem ? (long long)((kQuadSmem - st) / (W * 4)) - 2 * kQPad : 0;
      if (rows < 16) return false;
      nbands = (int)((pl.n + rows - 1) / rows);
      rows_b = (pl.n + nbands - 1) / nbands;
      need = (size_t)(rows_b + 2 * kQPad) * W * 4 + st;
    }
  }
  *tiles = T;
  *kg = KG;
  *mg = MG;
  *bh = rows_b;
  *nb = nbands;
  *sm = need;
  // one band: several classes per CTA share the staged plane, as long as the
  // grid keeps about four CTAs per SM
  const int ncls = pl.nth / 4 + 1;
  int c = 1;
  if (nbands == 1)
    while (c < ncls && (long long)((ncls + 2 * c - 1) / (2 * c)) * pl.n >= 4LL * kNumSMs) c *= 2;
  *cpb = c;
  return true;
}

size_t project_scratch_bytes(const Plan& pl) {
  int group, bh, nb, tl, kg, mg, cpb;
  size_t sm;
  if (quad_plan(pl, &tl, &kg, &mg, &bh, &nb, &sm, &cpb) || project_smem_bytes(pl) <= 200 * 1024 ||
      band_plan(pl, &group, &bh, &nb, &sm))
    return 0;
  return (size_t)pl.n * pl.n * pl.n * pl.esize;
}

int launch_project(const Plan& pl, const void* p, void* g, const void* sub, cudaStream_t st,
                   const void* mask, void* scratch) {
  {
    // FP32, even N and angle count: one weight evaluation per four angles
    int tl, kg, mg, bh, nb, cpb;
    size_t sm;
    if (quad_plan(pl, &tl, &kg, &mg, &bh, &nb, &sm, &cpb)) {
      static std::once_flag once;
      static cudaError_t attr = cudaSuccess;
      std::call_once(once, [] {
        attr = cudaFuncSetAttribute(k_project_quad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)kQuadSmem);
      });
      if (attr != cudaSuccess) {
        cudaGetLastError();
        return report(FFPAT_ECUDA, "k_project_quad: %zu bytes of shared memory refused", sm);
      }
      const dim3 grid((pl.nth / 4 + cpb) / cpb, pl.n);
      k_project_quad<<<grid, kg * mg * 32, sm, st>>>((const float*)p, (float*)g,
                                                     (const float*)sub, (const float*)mask,
                                                     pl.tabi, pl.n, pl.nth, pl.ns, pl.nimg, tl,
                                                     kg, mg, bh, nb, cpb);
      count_launch();
      return check_launch("k_project_quad");
    }
  }
  const size_t smem = project_smem_bytes(pl);
  if (smem <= 200 * 1024) {
    // one CTA per (plane, group of 8 angles); the padded plane is read once per CTA
    const int group = 8;
    const dim3 grid(pl.n, (pl.nth + group - 1) / group);
    if (pl.prec == FFPAT_FP64) {
      static bool attr = false;
      if (!attr) {
        cudaFuncSetAttribute(k_project_smem<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             200 * 1024);
        attr = true;
      }
      k_project_smem<double><<<grid, kProjThreads, smem, st>>>((const double*)p, (double*)g,
                                                      (const double*)sub, (const double*)mask,
                                                      pl.tab, pl.tabf, pl.tabi, pl.n, pl.nth,
                                                      pl.ns, pl.nimg, group);
    } else {
      static bool attr = false;
      if (!attr) {
        cudaFuncSetAttribute(k_project_smem<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             200 * 1024);
        attr = true;
      }
      k_project_smem<float><<<grid, kProjThreads, smem, st>>>((const float*)p, (float*)g, (const float*)sub,
                                                     (const float*)mask, pl.tab, pl.tabf, pl.tabi,
                                                     pl.n, pl.nth, pl.ns, pl.nimg, group);
    }
    count_launch();
    return check_launch(__func__);
  }
  // FP32 planes too large for shared memory: band by band ...
  int group, bh, nb;
  size_t sm;
  if (band_plan(pl, &group, &bh, &nb, &sm)) {
    // angles with cos >= 0 first (the table is in increasing theta)
    int jsplit = 0;
    for (int j = 0; j < pl.nth; ++j)
      if (cos((M_PI * j) / pl.nth) >= 0.0) jsplit = j + 1;
    const int groups = (jsplit + group - 1) / group + (pl.nth - jsplit + group - 1) / group;
    const dim3 grid(groups, pl.n);
    cudaFuncSetAttribute(k_project_band, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_project_band<<<grid, 1024, sm, st>>>((const float*)p, (float*)g, (const float*)sub,
                                          (const float*)mask, pl.tabf, pl.tabi, pl.n, pl.nth,
                                          pl.ns, pl.nimg, group, jsplit, bh, nb);
    count_launch();
    return check_launch("k_project_band");
  }
  // ... else from global memory; with scratch, the steep angles read a
  // transposed copy of the volume
  if (scratch) {
    const dim3 tg((pl.n + 31) / 32, (pl.n + 31) / 32, pl.n);
    if (pl.prec == FFPAT_FP64)
      k_transpose_planes<double><<<tg, dim3(32, 8), 0, st>>>((const double*)p, (double*)scratch,
                                                            pl.n);
    else
      k_transpose_planes<float><<<tg, dim3(32, 8), 0, st>>>((const float*)p, (float*)scratch,
                                                           pl.n);
    count_launch();
    if (check_launch("transpose planes") != FFPAT_OK) return FFPAT_ECUDA;
  }
  const dim3 block(128);
  const dim3 grid((pl.n + 127) / 128, pl.n, pl.nth);
  if (pl.prec == FFPAT_FP64)
    k_project<double><<<grid, block, 0, st>>>((const double*)p, (const double*)scratch, (double*)g,
                                              (const double*)sub, (const double*)mask, pl.tab,
                                              pl.tabf, pl.tabi, pl.n, pl.nth, pl.ns, pl.nimg);
  else
    k_project<float><<<grid, block, 0, st>>>((const float*)p, (const float*)scratch, (float*)g,
                                             (const float*)sub, (const float*)mask, pl.tab,
                                             pl.tabf, pl.tabi, pl.n, pl.nth, pl.ns, pl.nimg);
  count_launch();
  return check_launch(__func__);
}

int launch_backproject(const Plan& pl, const void* g, void* h, const void* scale, cudaStream_t st,
                       double mult) {
  const dim3 block(32, 8);
  const dim3 grid((pl.n + 31) / 32, (pl.n + 7) / 8, pl.n);
  if (pl.prec != FFPAT_FP64 && pl.nth % 2 == 0 && pl.n % 2 == 0 && !backproject_quad_off() &&
      !backproject_pair_off()) {
    const dim3 gq((pl.n / 2 + 31) / 32, (pl.n + 7) / 8, pl.n);
    k_backproject_quad<<<gq, block, 0, st>>>((const float*)g, (float*)h, (const float*)scale,
                                             pl.tabf, pl.tabi, pl.n, pl.nth, pl.ns, pl.nimg,
                                             (float)mult);
    count_launch();
    return check_launch("k_backproject_quad");
  }
  if (pl.prec != FFPAT_FP64 && pl.nth % 2 == 0 && pl.n % 2 == 0 && !backproject_pair_off()) {
    k_backproject_pair<<<grid, block, 0, st>>>((const float*)g, (float*)h, (const float*)scale,
                                               pl.tabf, pl.tabi, pl.n, pl.nth, pl.ns, pl.nimg,
                                               (float)mult);
    count_launch();
    return check_launch("k_backproject_pair");
  }
  if (pl.prec == FFPAT_FP64)
    k_backproject2<double><<<grid, block, 0, st>>>((const double*)g, (double*)h,
                                                  (const double*)scale, pl.tab, pl.tabf,
                                                  pl.tabi, pl.n, pl.nth, pl.ns, pl.nimg, mult);
  else
    k_backproject2<float><<<grid, block, 0, st>>>((const float*)g, (float*)h, (const float*)scale,
                                                 pl.tab, pl.tabf, pl.tabi, pl.n, pl.nth, pl.ns,
                                                 pl.nimg, (float)mult);
  count_launch();
  return check_launch(__func__);
}

int launch_ramp(const Plan& pl, const void* r, void* out, cudaStream_t st, const void* mask) {
  const int rows = pl.nth * pl.n;
  const size_t smem = 4 * (size_t)pl.n * pl.esize;
  // eight 128-thread CTAs per SM walk the rows
  const unsigned grid = (unsigned)(rows < 8 * kNumSMs ? rows : 8 * kNumSMs);
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [] {
    attr = cudaFuncSetAttribute(k_ramp<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                200 * 1024);
    if (attr == cudaSuccess)
      attr = cudaFuncSetAttribute(k_ramp<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  200 * 1024);
  });
  if (attr != cudaSuccess || smem > 200 * 1024) {
    cudaGetLastError();
    return report(FFPAT_ECUDA, "k_ramp: %zu bytes of shared memory refused", smem);
  }
  if (pl.prec == FFPAT_FP64)
    k_ramp<double><<<grid, 128, smem, st>>>((const double*)r, (double*)out, (const double*)mask,
                                            pl.n, pl.nimg, rows);
  else
    k_ramp<float><<<grid, 128, smem, st>>>((const float*)r, (float*)out, (const float*)mask, pl.n,
                                           pl.nimg, rows);
  count_launch();
  return check_launch(__func__);
}

int launch_debug_samples(const Plan& pl, int count, const int32_t* jkm, int32_t* ij, double* f,
                         cudaStream_t st) {
  if (count <= 0) return FFPAT_OK;
  k_debug_samples<<<(count + 127) / 128, 128, 0, st>>>(count, jkm, ij, f, pl.tab, pl.n, pl.nth,
                                                      pl.ns, pl.nimg);
  count_launch();
  return check_launch(__func__);
}

}  // namespace ffpat
