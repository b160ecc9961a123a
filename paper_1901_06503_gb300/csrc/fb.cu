// fb.cu -- setup of the wave coefficients, elementwise passes and the fused
// forward-backward update of Algorithm 8 (Sec. 3.2), with deterministic FP64
// reductions.
//
// Every reduction runs on a fixed grid of kReduceBlocks CTAs with a grid-
// stride loop; each CTA reduces its FP64 partial in a fixed shuffle tree and
// writes it to `partials`; a single-CTA pass then sums the partials in a fixed
// order.  Results are therefore bit-reproducible from run to run.
#include <math.h>

#include "internal.cuh"

namespace ffpat {
namespace {

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sm[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sm[w] = v;
  __syncthreads();
  double t = 0.0;
  if (w == 0) {
    t = lane < (int)(blockDim.x >> 5) ? sm[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  }
  return t;
}

__device__ __forceinline__ double block_max(double v) {
  __shared__ double sm[32];
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sm[w] = v;
  __syncthreads();
  double t = -INFINITY;
  if (w == 0) {
    t = lane < (int)(blockDim.x >> 5) ? sm[lane] : -INFINITY;
    for (int o = 16; o > 0; o >>= 1) t = fmax(t, __shfl_down_sync(0xffffffffu, t, o));
  }
  return t;
}

// sum `nq` rows of kReduceBlocks partials (fixed order) into dst[0..nq)
__global__ void __launch_bounds__(kReduceThreads)
    k_finalize(const double* __restrict__ partials, int nq, double* __restrict__ dst) {
  for (int q = 0; q < nq; ++q) {
    double acc = 0.0;
    for (int i = threadIdx.x; i < kReduceBlocks; i += blockDim.x) acc += partials[q * kReduceBlocks + i];
    acc = block_sum(acc);
    if (threadIdx.x == 0) dst[q] = acc;
  }
}

// max c, -min c, count of invalid entries (not finite or <= 0)
template <typename T>
__global__ void __launch_bounds__(kReduceThreads)
    k_speed_stats(const T* __restrict__ c, size_t len, double* __restrict__ partials) {
  // the element loop runs in the input's own type (max and min of floats are
  // exact in float, and the count is an integer): FP32 input stays off the
  // FP64 pipe; only the per-thread results go through the FP64 block reductions
  T mxt = T(-INFINITY), mnt = T(INFINITY);
  unsigned nbad = 0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < len;
       i += (size_t)gridDim.x * blockDim.x) {
    const T v = c[i];
    if (!(v > T(0)) || !isfinite(v)) ++nbad;
    mxt = fmax(mxt, v);
    mnt = fmin(mnt, v);
  }
  const double mx = block_max((double)mxt);
  const double nmn = block_max(-(double)mnt);
  const double bad = block_sum((double)nbad);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = mx;
    partials[kReduceBlocks + blockIdx.x] = nmn;
    partials[2 * kReduceBlocks + blockIdx.x] = bad;
  }
}

__global__ void __launch_bounds__(kReduceThreads)
    k_speed_final(const double* __restrict__ partials, double* __restrict__ dst) {
  double mx = -INFINITY, nmn = -INFINITY, bad = 0.0;
  for (int i = threadIdx.x; i < kReduceBlocks; i += blockDim.x) {
    mx = fmax(mx, partials[i]);
    nmn = fmax(nmn, partials[kReduceBlocks + i]);
    bad += partials[2 * kReduceBlocks + i];
  }
  mx = block_max(mx);
  nmn = block_max(nmn);
  bad = block_sum(bad);
  if (threadIdx.x == 0) {
    dst[0] = mx;
    dst[1] = -nmn;
    dst[2] = bad;
  }
}

// kap = (c dt / dx)^2 / 12 in FP64, with dt / dx and 1/12 folded into one
// factor q = (dt / dx)^2 / 12 computed on the host (multiplications only)
template <typename T>
__global__ void k_kappa(const T* __restrict__ c, T* __restrict__ kap, size_t len, double q) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < len;
       i += (size_t)gridDim.x * blockDim.x) {
    const double cv = (double)c[i];
    kap[i] = (T)(cv * cv * q);
  }
}

template <typename T>
__global__ void k_kscale(const T* __restrict__ a, T* __restrict__ out, const T* __restrict__ kap,
                         size_t len, bool mul) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < len;
       i += (size_t)gridDim.x * blockDim.x)
    out[i] = mul ? a[i] * kap[i] : a[i] / kap[i];
}

// to_wave: the wave grid (nw^3) gets the box (n^3) in its central cells and
// zero elsewhere; else the box gets the central cells of the wave grid
template <typename T>
__global__ void k_box_copy(const T* __restrict__ src, T* __restrict__ dst, int n, int nw, int pad,
                           bool to_wave) {
  const int m = to_wave ? nw : n;
  const size_t len = (size_t)m * m * m;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < len;
       i += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % m);
    const size_t t = i / m;
    const int y = (int)(t % m);
    const int z = (int)(t / m);
    if (to_wave) {
      const int bx = x - pad, by = y - pad, bz = z - pad;
      const bool in = bx >= 0 && by >= 0 && bz >= 0 && bx < n && by < n && bz < n;
      dst[i] = in ? src[((size_t)bz * n + by) * n + bx] : T(0);
    } else {
      dst[i] = src[((size_t)(z + pad) * nw + (y + pad)) * nw + (x + pad)];
    }
  }
}

template <typename T>
__global__ void k_scale_dev(const T* __restrict__ a, T* __restrict__ out, size_t len,
                            const double* __restrict__ sq) {
  const double s = 1.0 / sqrt(sq[0]);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < len;
       i += (size_t)gridDim.x * blockDim.x)
    out[i] = (T)((double)a[i] * s);
}

// partials rows: 0 = sum a b, 1 = sum b b
template <typename T>
__global__ void __launch_bounds__(kReduceThreads)
    k_dots(const T* __restrict__ a, const T* __restrict__ b, size_t len,
           double* __restrict__ partials) {
  double ab = 0.0, bb = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < len;
       i += (size_t)gridDim.x * blockDim.x) {
    const double x = (double)a[i], y = (double)b[i];
    ab = fma(x, y, ab);
    bb = fma(y, y, bb);
  }
  ab = block_sum(ab);
  bb = block_sum(bb);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = ab;
    partials[kReduceBlocks + blockIdx.x] = bb;
  }
}

// Algorithm 8, second line, with R = ||.||_1 + indicator(>= 0):
// grad = w / kap (the last division of W^T = K^-1 W K), h+ = max(h - s grad - s lambda, 0).
// partial rows: 0 = sum |h|, 1 = sum h^2, 2 = sum (h+ - h)^2, 3 = sum h+^2
template <typename T>
__global__ void __launch_bounds__(kReduceThreads)
    k_fb_update(T* __restrict__ h, const T* __restrict__ w, const T* __restrict__ kap, size_t len,
                double step, const double* __restrict__ step_dev, double lambda,
                const T* __restrict__ support, double* __restrict__ partials) {
  double l1 = 0.0, hh = 0.0, dd = 0.0, nn = 0.0;
  if (step_dev) step = *step_dev;
  const T s = (T)step, sl = (T)(step * lambda);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < len;
       i += (size_t)gridDim.x * blockDim.x) {
    const T hv = h[i];
    const T grad = w[i] / kap[i];
    const T f = (hv - s * grad) - sl;
    T hn = f > T(0) ? f : T(0);
    if (support) hn = hn * support[i];
    h[i] = hn;
    const double hd = (double)hv, nd = (double)hn, df = nd - hd;
    l1 += fabs(hd);
    hh = fma(hd, hd, hh);
    dd = fma(df, df, dd);
    nn = fma(nd, nd, nn);
  }
  l1 = block_sum(l1);
  hh = block_sum(hh);
  dd = block_sum(dd);
  nn = block_sum(nn);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = l1;
    partials[kReduceBlocks + blockIdx.x] = hh;
    partials[2 * kReduceBlocks + blockIdx.x] = dd;
    partials[3 * kReduceBlocks + blockIdx.x] = nn;
  }
}

// gradient-regulariser FB step, part 1: x = h - s w / kap (the argument of
// the prox; the same arithmetic as k_fb_update before its shrinkage)
template <typename T>
__global__ void k_prox_prep(const T* __restrict__ h, const T* __restrict__ w,
                            const T* __restrict__ kap, T* __restrict__ x, size_t len, double step,
                            const double* __restrict__ step_dev) {
  if (step_dev) step = *step_dev;
  const T s = (T)step;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < len;
       i += (size_t)gridDim.x * blockDim.x)
    x[i] = h[i] - s * (w[i] / kap[i]);
}

// part 2, after the prox wrote hn: the FP64 partials of R(h) = 1/2 <D h, D h>
// / dx^2 (forward differences inside the box), ||h||^2, ||hn - h||^2, ||hn||^2
// in the rows k_fb_update uses for |h|_1, ||h||^2, ...
template <typename T>
__global__ void __launch_bounds__(kReduceThreads)
    k_prox_finish(const T* __restrict__ h, const T* __restrict__ hn, int n, double half_inv_dx2,
                  double* __restrict__ partials) {
  const size_t nn = (size_t)n * n, len = nn * n;
  double rr = 0.0, hh = 0.0, dd = 0.0, qq = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < len;
       i += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % n), y = (int)((i / n) % n), z = (int)(i / nn);
    const double u = (double)h[i], v = (double)hn[i], df = v - u;
    if (x + 1 < n) { const double e = (double)h[i + 1] - u; rr = fma(e, e, rr); }
    if (y + 1 < n) { const double e = (double)h[i + n] - u; rr = fma(e, e, rr); }
    if (z + 1 < n) { const double e = (double)h[i + nn] - u; rr = fma(e, e, rr); }
    hh = fma(u, u, hh);
    dd = fma(df, df, dd);
    qq = fma(v, v, qq);
  }
  rr = block_sum(rr);
  hh = block_sum(hh);
  dd = block_sum(dd);
  qq = block_sum(qq);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = rr * half_inv_dx2;
    partials[kReduceBlocks + blockIdx.x] = hh;
    partials[2 * kReduceBlocks + blockIdx.x] = dd;
    partials[3 * kReduceBlocks + blockIdx.x] = qq;
  }
}

// dst = 1 / sqrt(src): the step 1 / L from the last power-iteration norm,
// the same arithmetic as the host's 1.0 / sqrt(.)
__global__ void k_inv_sqrt(const double* __restrict__ src, double* __restrict__ dst) {
  if (threadIdx.x == 0 && blockIdx.x == 0) dst[0] = 1.0 / sqrt(src[0]);
}

// Algorithm 9 residual: x = kap (w - g) (the input of W^T = K^-1 W K) and
// the FP64 partial of sum (w - g)^2 (rows 0 and 1 both get it)
template <typename T>
__global__ void __launch_bounds__(kReduceThreads)
    k_resid_kap(const T* __restrict__ w, const T* __restrict__ g, const T* __restrict__ kap,
                T* __restrict__ x, size_t len, double* __restrict__ partials) {
  double rr = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < len;
       i += (size_t)gridDim.x * blockDim.x) {
    const T r = w[i] - g[i];
    x[i] = kap[i] * r;
    rr = fma((double)r, (double)r, rr);
  }
  rr = block_sum(rr);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = rr;
    partials[kReduceBlocks + blockIdx.x] = rr;
  }
}

// out = (a - b) / kap   (last step of the transposed recurrence, back from kap-scaled form)
template <typename T>
__global__ void k_sub_div(const T* __restrict__ a, const T* __restrict__ b, const T* __restrict__ kap,
                          T* __restrict__ out, size_t len) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < len;
       i += (size_t)gridDim.x * blockDim.x)
    out[i] = (a[i] - b[i]) / kap[i];
}

// out = s * a / c
template <typename T>
__global__ void k_scale_div(const T* __restrict__ a, const T* __restrict__ c, T s,
                            T* __restrict__ out, size_t len) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < len;
       i += (size_t)gridDim.x * blockDim.x)
    out[i] = s * a[i] / c[i];
}

// counter-based pseudo-random start vector (splitmix64 + Box-Muller)
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

template <typename T>
__global__ void k_hash_fill(T* __restrict__ out, size_t len, uint64_t seed) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < len;
       i += (size_t)gridDim.x * blockDim.x) {
    const uint64_t a = splitmix64(seed ^ (2 * i)), b = splitmix64(seed ^ (2 * i + 1));
    const double u1 = ((a >> 11) + 1) * (1.0 / 9007199254740993.0);
    const double u2 = (b >> 11) * (1.0 / 9007199254740992.0);
    out[i] = (T)(sqrt(-2.0 * log(u1)) * cospi(2.0 * u2));
  }
}


unsigned ew_blocks(size_t len) {
  size_t b = (len + 255) / 256;
  const size_t cap = 16 * kNumSMs;
  return (unsigned)(b < 1 ? 1 : (b > cap ? cap : b));
}

}  // namespace

int launch_speed_stats(const Plan& pl, const void* c, double* out3, cudaStream_t st) {
  if (pl.prec == FFPAT_FP64)
    k_speed_stats<double><<<kReduceBlocks, kReduceThreads, 0, st>>>((const double*)c, pl.n3, pl.partials);
  else
    k_speed_stats<float><<<kReduceBlocks, kReduceThreads, 0, st>>>((const float*)c, pl.n3, pl.partials);
  k_speed_final<<<1, kReduceThreads, 0, st>>>(pl.partials, out3);
  count_launch(2);
  return check_launch(__func__);
}

int launch_kappa(const Plan& pl, const void* c, cudaStream_t st) {
  const unsigned nb = ew_blocks(pl.n3);
  const double r = pl.dt / pl.dx;
  const double q = r * r / 12.0;
  if (pl.prec == FFPAT_FP64)
    k_kappa<double><<<nb, 256, 0, st>>>((const double*)c, (double*)pl.kap, pl.n3, q);
  else
    k_kappa<float><<<nb, 256, 0, st>>>((const float*)c, (float*)pl.kap, pl.n3, q);
  count_launch();
  return check_launch(__func__);
}

int launch_kscale(const Plan& pl, const void* a, void* out, bool mul, cudaStream_t st) {
  const unsigned nb = ew_blocks(pl.n3);
  if (pl.prec == FFPAT_FP64)
    k_kscale<double><<<nb, 256, 0, st>>>((const double*)a, (double*)out, (const double*)pl.kap, pl.n3, mul);
  else
    k_kscale<float><<<nb, 256, 0, st>>>((const float*)a, (float*)out, (const float*)pl.kap, pl.n3, mul);
  count_launch();
  return check_launch(__func__);
}

static int box_copy(const Plan& pl, const void* src, void* dst, bool to_wave, cudaStream_t st) {
  const unsigned nb = ew_blocks(to_wave ? pl.nw3 : pl.n3);
  if (pl.prec == FFPAT_FP64)
    k_box_copy<double><<<nb, 256, 0, st>>>((const double*)src, (double*)dst, pl.n, pl.nw, pl.pad,
                                           to_wave);
  else
    k_box_copy<float><<<nb, 256, 0, st>>>((const float*)src, (float*)dst, pl.n, pl.nw, pl.pad,
                                          to_wave);
  count_launch();
  return check_launch(__func__);
}

int launch_embed(const Plan& pl, const void* box, void* wave, cudaStream_t st) {
  return box_copy(pl, box, wave, true, st);
}

int launch_restrict(const Plan& pl, const void* wave, void* box, cudaStream_t st) {
  return box_copy(pl, wave, box, false, st);
}

int launch_scale_dev(const Plan& pl, size_t len, const void* a, void* out, const double* s,
                     cudaStream_t st) {
  const unsigned nb = ew_blocks(len);
  if (pl.prec == FFPAT_FP64)
    k_scale_dev<double><<<nb, 256, 0, st>>>((const double*)a, (double*)out, len, s);
  else
    k_scale_dev<float><<<nb, 256, 0, st>>>((const float*)a, (float*)out, len, s);
  count_launch();
  return check_launch(__func__);
}

int launch_dot(const Plan& pl, size_t len, const void* a, const void* b, double* result,
               cudaStream_t st) {
  if (pl.prec == FFPAT_FP64)
    k_dots<double><<<kReduceBlocks, kReduceThreads, 0, st>>>((const double*)a, (const double*)b, len, pl.partials);
  else
    k_dots<float><<<kReduceBlocks, kReduceThreads, 0, st>>>((const float*)a, (const float*)b, len, pl.partials);
  k_finalize<<<1, kReduceThreads, 0, st>>>(pl.partials, 2, result);
  count_launch(2);
  return check_launch(__func__);
}

int launch_fb_update(const Plan& pl, void* h, const void* w, double step, double lambda,
                     double* dst, cudaStream_t st, const double* step_dev, const void* support) {
  if (pl.prec == FFPAT_FP64)
    k_fb_update<double><<<kReduceBlocks, kReduceThreads, 0, st>>>(
        (double*)h, (const double*)w, (const double*)pl.kap, pl.n3, step, step_dev, lambda,
        (const double*)support, pl.partials);
  else
    k_fb_update<float><<<kReduceBlocks, kReduceThreads, 0, st>>>(
        (float*)h, (const float*)w, (const float*)pl.kap, pl.n3, step, step_dev, lambda,
        (const float*)support, pl.partials);
  k_finalize<<<1, kReduceThreads, 0, st>>>(pl.partials, 4, dst);
  count_launch(2);
  return check_launch(__func__);
}

int launch_prox_prep(const Plan& pl, const void* h, const void* w, double step, void* x,
                     cudaStream_t st, const double* step_dev) {
  const unsigned nb = ew_blocks(pl.n3);
  if (pl.prec == FFPAT_FP64)
    k_prox_prep<double><<<nb, 256, 0, st>>>((const double*)h, (const double*)w,
                                            (const double*)pl.kap, (double*)x, pl.n3, step, step_dev);
  else
    k_prox_prep<float><<<nb, 256, 0, st>>>((const float*)h, (const float*)w, (const float*)pl.kap,
                                           (float*)x, pl.n3, step, step_dev);
  count_launch();
  return check_launch(__func__);
}

int launch_prox_finish(const Plan& pl, void* h, const void* hn, double* dst, cudaStream_t st) {
  const double q = 0.5 / (pl.dx * pl.dx);
  if (pl.prec == FFPAT_FP64)
    k_prox_finish<double><<<kReduceBlocks, kReduceThreads, 0, st>>>(
        (const double*)h, (const double*)hn, pl.n, q, pl.partials);
  else
    k_prox_finish<float><<<kReduceBlocks, kReduceThreads, 0, st>>>(
        (const float*)h, (const float*)hn, pl.n, q, pl.partials);
  k_finalize<<<1, kReduceThreads, 0, st>>>(pl.partials, 4, dst);
  count_launch(2);
  if (check_launch(__func__) != FFPAT_OK) return FFPAT_ECUDA;
  if (cudaMemcpyAsync(h, hn, pl.n3 * pl.esize, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return check_launch("prox: copy of the iterate");
  return FFPAT_OK;
}

int launch_resid_kap(const Plan& pl, const void* w, const void* g, void* x, double* dst,
                     cudaStream_t st) {
  if (pl.prec == FFPAT_FP64)
    k_resid_kap<double><<<kReduceBlocks, kReduceThreads, 0, st>>>(
        (const double*)w, (const double*)g, (const double*)pl.kap, (double*)x, pl.n3, pl.partials);
  else
    k_resid_kap<float><<<kReduceBlocks, kReduceThreads, 0, st>>>(
        (const float*)w, (const float*)g, (const float*)pl.kap, (float*)x, pl.n3, pl.partials);
  k_finalize<<<1, kReduceThreads, 0, st>>>(pl.partials, 2, dst);
  count_launch(2);
  return check_launch(__func__);
}

int launch_sub_div(const Plan& pl, const void* a, const void* b, void* out, cudaStream_t st) {
  const unsigned nb = ew_blocks(pl.n3);
  if (pl.prec == FFPAT_FP64)
    k_sub_div<double><<<nb, 256, 0, st>>>((const double*)a, (const double*)b,
                                          (const double*)pl.kap, (double*)out, pl.n3);
  else
    k_sub_div<float><<<nb, 256, 0, st>>>((const float*)a, (const float*)b, (const float*)pl.kap,
                                         (float*)out, pl.n3);
  count_launch();
  return check_launch(__func__);
}

int launch_scale_div(const Plan& pl, const void* a, const void* c, double s, void* out,
                     cudaStream_t st) {
  const unsigned nb = ew_blocks(pl.n3);
  if (pl.prec == FFPAT_FP64)
    k_scale_div<double><<<nb, 256, 0, st>>>((const double*)a, (const double*)c, s, (double*)out,
                                            pl.n3);
  else
    k_scale_div<float><<<nb, 256, 0, st>>>((const float*)a, (const float*)c, (float)s,
                                           (float*)out, pl.n3);
  count_launch();
  return check_launch(__func__);
}

int launch_inv_sqrt(const double* src, double* dst, cudaStream_t st) {
  k_inv_sqrt<<<1, 32, 0, st>>>(src, dst);
  count_launch();
  return check_launch(__func__);
}

int launch_hash_fill(const Plan& pl, void* out, uint64_t seed, cudaStream_t st) {
  const unsigned nb = ew_blocks(pl.n3);
  if (pl.prec == FFPAT_FP64)
    k_hash_fill<double><<<nb, 256, 0, st>>>((double*)out, pl.n3, seed);
  else
    k_hash_fill<float><<<nb, 256, 0, st>>>((float*)out, pl.n3, seed);
  count_launch();
  return check_launch(__func__);
}

}  // namespace ffpat
