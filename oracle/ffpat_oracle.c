/*
 * ffpat_oracle.c -- plain FP64 CPU oracle for one-step full-field photoacoustic
 * reconstruction (Haltmeier, Zangerl, Nuster, Nguyen, "Photoacoustic image
 * reconstruction from full field data in heterogeneous media", 2019).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls
 * this file: only the tests, the smoke check and the benchmark's CPU baseline
 * do.  It shares no code, header or table with the CUDA library.
 *
 * Every function is the plain definition, written out as slow loops in double
 * precision (compile with -ffp-contract=off so that no multiply-add is fused).
 *
 * Discretisation (readings of the paper, which uses a k-space solver and
 * Matlab's radon for its own 2D experiments):
 *   grid      N^3 cell-centred points on [-1,1]^3, x_i = -1 + (i + 1/2) dx,
 *             dx = 2/N, layout [z][y][x] with x fastest;
 *   Laplacian L4 u = sum over the three axes of
 *             (-u[-2] + 16 u[-1] - 30 u[0] + 16 u[+1] - u[+2]) / 12,
 *             with zero ghost values outside the box (the 1/dx^2 is folded
 *             into kappa);
 *   time      Nt = ceil(T c_max / (cfl dx) (1 - 1e-12)), dt = T / Nt,
 *             kappa = (c dt / dx)^2.
 *
 * Parity status: every function below is pinned by tests/test_oracle_pins.py
 * (closed forms, spectral closed form of the time stepping, exact polynomial
 * reproduction, energy conservation, dense transposes, FBP identity, KKT).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define FFO_PI 3.14159265358979323846

static size_t at3(int n, int z, int y, int x) { return ((size_t)z * n + y) * n + x; }

/* value of u at (z,y,x), zero outside the box (homogeneous Dirichlet ghosts) */
static double ghost(const double *u, int n, int z, int y, int x) {
  if (x < 0 || y < 0 || z < 0 || x >= n || y >= n || z >= n) return 0.0;
  return u[at3(n, z, y, x)];
}

/* one axis of the fourth-order central second difference (times 12) */
static double d2_axis(double um2, double um1, double u0, double up1, double up2) {
  return -um2 + 16.0 * um1 - 30.0 * u0 + 16.0 * up1 - up2;
}

/* L4 u at one point: the discrete Laplacian of the wave equation (Sec. 2.1,
 * eq. (1)), fourth order in space, dimensionless */
static double lap4_at(const double *u, int n, int z, int y, int x) {
  double u0 = u[at3(n, z, y, x)];
  double ax = d2_axis(ghost(u, n, z, y, x - 2), ghost(u, n, z, y, x - 1), u0,
                      ghost(u, n, z, y, x + 1), ghost(u, n, z, y, x + 2));
  double ay = d2_axis(ghost(u, n, z, y - 2, x), ghost(u, n, z, y - 1, x), u0,
                      ghost(u, n, z, y + 1, x), ghost(u, n, z, y + 2, x));
  double az = d2_axis(ghost(u, n, z - 2, y, x), ghost(u, n, z - 1, y, x), u0,
                      ghost(u, n, z + 1, y, x), ghost(u, n, z + 2, y, x));
  return (ax + ay + az) / 12.0;
}

static void lap4(const double *u, int n, double *out) {
  int z;
#pragma omp parallel for schedule(static)
  for (z = 0; z < n; ++z)
    for (int y = 0; y < n; ++y)
      for (int x = 0; x < n; ++x) out[at3(n, z, y, x)] = lap4_at(u, n, z, y, x);
}

int ffo_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void ffo_set_num_threads(int k) {
#ifdef _OPENMP
  if (k > 0) omp_set_num_threads(k);
#else
  (void)k;
#endif
}

/* ---------------------------------------------------------------- setup -- */

/* Number of leapfrog steps for final time T (wave model, Sec. 2.1): the
 * smallest Nt with T/Nt <= cfl dx / c_max; the factor (1 - 1e-12) keeps a
 * ratio that is an integer up to round-off from gaining a step. */
int ffo_time_steps(int n, double T, double cfl, double cmax, double *dt_out) {
  double dx = 2.0 / n;
  double x = T * cmax / (cfl * dx);
  int nt = (int)ceil(x * (1.0 - 1e-12));
  if (nt < 1) nt = 1;
  if (dt_out) *dt_out = T / nt;
  return nt;
}

/* kappa = (c dt / dx)^2 for every grid point (c^2 scaling of eq. (1)) */
void ffo_kappa(int n, double dt, const double *c, double *kappa) {
  double dx = 2.0 / n;
  size_t n3 = (size_t)n * n * n;
  for (size_t i = 0; i < n3; ++i) {
    double r = c[i] * dt / dx;
    kappa[i] = r * r;
  }
}

double ffo_max(size_t len, const double *a) {
  double m = -INFINITY;
  for (size_t i = 0; i < len; ++i)
    if (a[i] > m) m = a[i];
  return m;
}

/* ---------------------------------------------------- wave operator W_T -- */

/* W_T h = p(., T) (eq. (3)) for the wave equation (1)-(2): p^0 = h; the zero
 * initial velocity gives p^1 = p^0 + 1/2 kappa L4 p^0; then the leapfrog
 * p^{n+1} = 2 p^n - p^{n-1} + kappa L4 p^n up to n + 1 = nt.  kappa carries
 * dt, so this runs any number of steps nt >= 1 for the given kappa. */
void ffo_wave(int n, int nt, const double *kappa, const double *h, double *out) {
  size_t n3 = (size_t)n * n * n;
  double *prev = malloc(n3 * sizeof(double));
  double *cur = malloc(n3 * sizeof(double));
  double *lap = malloc(n3 * sizeof(double));
  memcpy(prev, h, n3 * sizeof(double));
  lap4(prev, n, lap);
  for (size_t i = 0; i < n3; ++i) cur[i] = prev[i] + 0.5 * kappa[i] * lap[i];
  for (int step = 1; step < nt; ++step) {
    lap4(cur, n, lap);
    for (size_t i = 0; i < n3; ++i) {
      double next = 2.0 * cur[i] - prev[i] + kappa[i] * lap[i];
      prev[i] = cur[i];
      cur[i] = next;
    }
  }
  memcpy(out, cur, n3 * sizeof(double));
  free(prev);
  free(cur);
  free(lap);
}

/* The transpose of W_T (Sec. 3.1: the adjoint runs the wave equation backwards
 * from (q, q_t)|_T = (g, 0) to t = 0).  For the exact Euclidean transpose of
 * the discrete W the sound speed sits inside the Laplacian, q_tt = Delta(c^2 q):
 * q^{nt} = g, q^{nt-1} = q^{nt} + 1/2 L4(kappa q^{nt}), and
 * q^{n-1} = 2 q^n - q^{n+1} + L4(kappa q^n) down to q^0, the output. */
void ffo_wave_adjoint(int n, int nt, const double *kappa, const double *g, double *out) {
  size_t n3 = (size_t)n * n * n;
  double *later = malloc(n3 * sizeof(double)); /* q^{n+1} */
  double *cur = malloc(n3 * sizeof(double));   /* q^n */
  double *kq = malloc(n3 * sizeof(double));
  double *lap = malloc(n3 * sizeof(double));
  memcpy(later, g, n3 * sizeof(double));
  for (size_t i = 0; i < n3; ++i) kq[i] = kappa[i] * later[i];
  lap4(kq, n, lap);
  for (size_t i = 0; i < n3; ++i) cur[i] = later[i] + 0.5 * lap[i];
  for (int step = 1; step < nt; ++step) {
    for (size_t i = 0; i < n3; ++i) kq[i] = kappa[i] * cur[i];
    lap4(kq, n, lap);
    for (size_t i = 0; i < n3; ++i) {
      double earlier = 2.0 * cur[i] - later[i] + lap[i];
      later[i] = cur[i];
      cur[i] = earlier;
    }
  }
  memcpy(out, cur, n3 * sizeof(double));
  free(later);
  free(cur);
  free(kq);
  free(lap);
}

/* ------------------------------------------------- X-ray transform X / P -- */

/* theta_j = pi j / n_angles, j < n_angles (the paper's 1D set of directions,
 * Sec. 4.1: equidistant in [0, 180 degrees)). */
void ffo_angles(int nth, double *cs, double *sn) {
  for (int j = 0; j < nth; ++j) {
    double th = (FFO_PI * j) / nth;
    cs[j] = cos(th);
    sn[j] = sin(th);
  }
}

/* number of ray samples: 2 ceil(N / sqrt 2), spacing dx, covering |s| <~ sqrt 2 */
int ffo_ray_samples(int n) { return 2 * (int)ceil((double)n / sqrt(2.0)); }

/* bilinear interpolation weights of the sample point (xi_k theta + s_m theta_perp)
 * in slice coordinates; returns the lower-left corner through i0/j0.  The
 * slice has ng cells per axis of physical size dx = 2 / nimg, so it spans
 * [-L, L] with L = ng / nimg (ng = nimg: the box [-1, 1]); detectors and ray
 * samples are spaced dx. */
static void sample_point_g(int ng, int nimg, double cs, double sn, int k, int m, int ns, int *i0,
                           int *j0, double *fx, double *fy) {
  double dx = 2.0 / nimg;
  double L = (double)ng / nimg;
  double xi = -L + (k + 0.5) * dx;             /* detector centre xi_k */
  double s = (m + 0.5 - ns / 2) * dx;          /* ray sample s_m */
  double x = xi * cs - s * sn;                 /* xi theta + s theta_perp, theta_perp = (-sin, cos) */
  double y = xi * sn + s * cs;
  double half = nimg / 2.0;
  double gx = (x + L) * half - 0.5;            /* continuous grid index of x */
  double gy = (y + L) * half - 0.5;
  double fl_x = floor(gx), fl_y = floor(gy);
  *i0 = (int)fl_x;
  *j0 = (int)fl_y;
  *fx = gx - fl_x;
  *fy = gy - fl_y;
}

/* exposes the sample arithmetic for the bit-exact index-table check */
void ffo_sample_points_g(int n, int nimg, int nth, int count, const int32_t *jkm, int32_t *ij,
                         double *f) {
  double *cs = malloc(nth * sizeof(double)), *sn = malloc(nth * sizeof(double));
  int ns = ffo_ray_samples(n);
  ffo_angles(nth, cs, sn);
  for (int t = 0; t < count; ++t) {
    int j = jkm[3 * t], k = jkm[3 * t + 1], m = jkm[3 * t + 2];
    int i0, j0;
    double fx, fy;
    sample_point_g(n, nimg, cs[j], sn[j], k, m, ns, &i0, &j0, &fx, &fy);
    ij[2 * t] = i0;
    ij[2 * t + 1] = j0;
    f[2 * t] = fx;
    f[2 * t + 1] = fy;
  }
  free(cs);
  free(sn);
}

void ffo_sample_points(int n, int nth, int count, const int32_t *jkm, int32_t *ij, double *f) {
  ffo_sample_points_g(n, n, nth, count, jkm, ij, f);
}

static double slice_at(const double *slice, int n, int iy, int ix) {
  if (ix < 0 || iy < 0 || ix >= n || iy >= n) return 0.0;
  return slice[(size_t)iy * n + ix];
}

/* P: g[j][l][k] = ds sum_m B(p[l]; xi_k theta_j + s_m theta_j^perp), eq. (4)
 * applied in each horizontal plane z_l (the X-ray transform is the 2D Radon
 * transform per plane), with zero-extended bilinear interpolation B.  The
 * planes have ng cells per axis of size ds = 2 / nimg (see sample_point_g);
 * ng detectors, Ns = 2 ceil(ng / sqrt 2) samples per ray. */
void ffo_project_g(int ng, int nimg, int nth, const double *p, double *g) {
  int n = ng;
  double *cs = malloc(nth * sizeof(double)), *sn = malloc(nth * sizeof(double));
  int ns = ffo_ray_samples(n);
  double ds = 2.0 / nimg;
  ffo_angles(nth, cs, sn);
  int jl;
#pragma omp parallel for schedule(static)
  for (jl = 0; jl < nth * n; ++jl) {
    int j = jl / n, l = jl % n;
    const double *slice = p + (size_t)l * n * n;
    for (int k = 0; k < n; ++k) {
      double acc = 0.0;
      for (int m = 0; m < ns; ++m) {
        int i0, j0;
        double fx, fy;
        sample_point_g(n, nimg, cs[j], sn[j], k, m, ns, &i0, &j0, &fx, &fy);
        double b = (1.0 - fx) * (1.0 - fy) * slice_at(slice, n, j0, i0) +
                   fx * (1.0 - fy) * slice_at(slice, n, j0, i0 + 1) +
                   (1.0 - fx) * fy * slice_at(slice, n, j0 + 1, i0) +
                   fx * fy * slice_at(slice, n, j0 + 1, i0 + 1);
        acc += b;
      }
      g[((size_t)j * n + l) * n + k] = ds * acc;
    }
  }
  free(cs);
  free(sn);
}

void ffo_project(int n, int nth, const double *p, double *g) { ffo_project_g(n, n, nth, p, g); }

/* selected rays of ffo_project: out[t] = g[j][l][k] for jlk[3t..3t+2] = (j, l, k);
 * the same loop as ffo_project, restricted, for spot checks on large grids */
void ffo_project_rays(int n, int nth, const double *p, int count, const int32_t *jlk, double *out) {
  double *cs = malloc(nth * sizeof(double)), *sn = malloc(nth * sizeof(double));
  int ns = ffo_ray_samples(n);
  double ds = 2.0 / n;
  ffo_angles(nth, cs, sn);
  for (int t = 0; t < count; ++t) {
    int j = jlk[3 * t], l = jlk[3 * t + 1], k = jlk[3 * t + 2];
    const double *slice = p + (size_t)l * n * n;
    double acc = 0.0;
    for (int m = 0; m < ns; ++m) {
      int i0, j0;
      double fx, fy;
      sample_point_g(n, n, cs[j], sn[j], k, m, ns, &i0, &j0, &fx, &fy);
      double b = (1.0 - fx) * (1.0 - fy) * slice_at(slice, n, j0, i0) +
                 fx * (1.0 - fy) * slice_at(slice, n, j0, i0 + 1) +
                 (1.0 - fx) * fy * slice_at(slice, n, j0 + 1, i0) +
                 fx * fy * slice_at(slice, n, j0 + 1, i0 + 1);
      acc += b;
    }
    out[t] = ds * acc;
  }
  free(cs);
  free(sn);
}

static void scatter(double *slice, int n, int iy, int ix, double v) {
  if (ix < 0 || iy < 0 || ix >= n || iy >= n) return;
  slice[(size_t)iy * n + ix] += v;
}

/* P^T: the matrix transpose of ffo_project (the discrete counterpart of the
 * backprojection X* of Sec. 3.1): every sample spreads ds g[j][l][k] onto its
 * four bilinear corners with the same weights. */
void ffo_backproject_g(int ng, int nimg, int nth, const double *g, double *out) {
  int n = ng;
  double *cs = malloc(nth * sizeof(double)), *sn = malloc(nth * sizeof(double));
  int ns = ffo_ray_samples(n);
  double ds = 2.0 / nimg;
  ffo_angles(nth, cs, sn);
  memset(out, 0, (size_t)n * n * n * sizeof(double));
  int l;
#pragma omp parallel for schedule(static)
  for (l = 0; l < n; ++l) {
    double *slice = out + (size_t)l * n * n;
    for (int j = 0; j < nth; ++j)
      for (int k = 0; k < n; ++k) {
        double w = ds * g[((size_t)j * n + l) * n + k];
        for (int m = 0; m < ns; ++m) {
          int i0, j0;
          double fx, fy;
          sample_point_g(n, nimg, cs[j], sn[j], k, m, ns, &i0, &j0, &fx, &fy);
          scatter(slice, n, j0, i0, (1.0 - fx) * (1.0 - fy) * w);
          scatter(slice, n, j0, i0 + 1, fx * (1.0 - fy) * w);
          scatter(slice, n, j0 + 1, i0, (1.0 - fx) * fy * w);
          scatter(slice, n, j0 + 1, i0 + 1, fx * fy * w);
        }
      }
  }
  free(cs);
  free(sn);
}

void ffo_backproject(int n, int nth, const double *g, double *out) {
  ffo_backproject_g(n, n, nth, g, out);
}

/* ------------------------------------------------ preconditioner Lambda -- */

/* Filter tap t_d of Lambda (Sec. 3.1, F Lambda Phi = |omega|/(4 pi) F Phi in
 * the detector variable): half the band-limited ramp filter on the detector
 * spacing dxi = 2 / nimg, times the quadrature weight dxi. */
double ffo_ramp_tap(int nimg, int d) {
  double dxi = 2.0 / nimg;
  if (d < 0) d = -d;
  if (d == 0) return 1.0 / (8.0 * dxi);
  if (d % 2 == 0) return 0.0;
  return -1.0 / (2.0 * FFO_PI * FFO_PI * (double)d * (double)d * dxi);
}

/* (Lambda r)[j][l][k] = sum_{k'} t_{k-k'} r[j][l][k'] along each detector row
 * of ng detectors (nth ng rows) */
void ffo_ramp_g(int ng, int nimg, int nth, const double *r, double *out) {
  int n = ng;
  int row;
  int rows = nth * n;
#pragma omp parallel for schedule(static)
  for (row = 0; row < rows; ++row) {
    const double *rr = r + (size_t)row * n;
    double *oo = out + (size_t)row * n;
    for (int k = 0; k < n; ++k) {
      double acc = 0.0;
      for (int kk = 0; kk < n; ++kk) acc += ffo_ramp_tap(nimg, k - kk) * rr[kk];
      oo[k] = acc;
    }
  }
}

void ffo_ramp(int n, int nth, const double *r, double *out) { ffo_ramp_g(n, n, nth, r, out); }

/* ------------------------------- gradient regulariser R = 1/2 |grad h|^2 -- */

/* The discrete R of the paper's experiments (Sec. 5): forward differences
 * between neighbouring cells of the box, none across its faces (h lives on the
 * box V only), scaled by 1/dx:  R(h) = 1/2 sum_axes sum (h[i+1] - h[i])^2 / dx^2
 * = 1/2 <D h, D h> / dx^2.  This returns <D h, D h> (no 1/dx^2). */
double ffo_grad_energy(int n, const double *h) {
  double acc = 0.0;
  for (int z = 0; z < n; ++z)
    for (int y = 0; y < n; ++y)
      for (int x = 0; x < n; ++x) {
        double u = h[at3(n, z, y, x)];
        if (x + 1 < n) acc += (h[at3(n, z, y, x + 1)] - u) * (h[at3(n, z, y, x + 1)] - u);
        if (y + 1 < n) acc += (h[at3(n, z, y + 1, x)] - u) * (h[at3(n, z, y + 1, x)] - u);
        if (z + 1 < n) acc += (h[at3(n, z + 1, y, x)] - u) * (h[at3(n, z + 1, y, x)] - u);
      }
  return acc;
}

/* D^T D h for the difference operator D of ffo_grad_energy: every pair of
 * neighbouring box cells (i, i + 1) along x, y and z contributes its
 * difference d = h[i + 1] - h[i] as D^T d, i.e. -d at i and +d at i + 1 (no
 * pair crosses a face of the box).  Serial, in a fixed order. */
static void dtd_apply(int n, const double *h, double *out) {
  size_t n3 = (size_t)n * n * n;
  for (size_t i = 0; i < n3; ++i) out[i] = 0.0;
  for (int z = 0; z < n; ++z)
    for (int y = 0; y < n; ++y)
      for (int x = 0; x < n; ++x) {
        size_t i = at3(n, z, y, x);
        if (x + 1 < n) {
          size_t j = at3(n, z, y, x + 1);
          double d = h[j] - h[i];
          out[i] -= d;
          out[j] += d;
        }
        if (y + 1 < n) {
          size_t j = at3(n, z, y + 1, x);
          double d = h[j] - h[i];
          out[i] -= d;
          out[j] += d;
        }
        if (z + 1 < n) {
          size_t j = at3(n, z + 1, y, x);
          double d = h[j] - h[i];
          out[i] -= d;
          out[j] += d;
        }
      }
}

/* prox of a R with a = s lambda / dx^2 (the proximal map of Sec. 3.2 for the
 * regulariser of the experiments, Sec. 5): argmin 1/2 ||h - f||^2
 * + a/2 <D h, D h>, i.e. the solution of the symmetric positive definite
 * system (I + a D^T D) h = f, solved by plain conjugate gradients from h = f
 * with D^T D applied from the difference definition above.  The spectrum of
 * I + a D^T D lies in [1, 1 + 12 a], so the iteration converges at any size;
 * it runs until the residual is below 1e-15 ||f|| (or stops decreasing). */
void ffo_prox_grad(int n, double a, const double *f, double *out) {
  size_t n3 = (size_t)n * n * n;
  double *r = malloc(n3 * sizeof(double)), *p = malloc(n3 * sizeof(double));
  double *q = malloc(n3 * sizeof(double));
  double ff = 0.0;
  for (size_t i = 0; i < n3; ++i) ff += f[i] * f[i];
  /* h = f, r = f - (I + a D^T D) f = -a D^T D f */
  memcpy(out, f, n3 * sizeof(double));
  dtd_apply(n, out, q);
  double rr = 0.0;
  for (size_t i = 0; i < n3; ++i) {
    r[i] = -a * q[i];
    p[i] = r[i];
    rr += r[i] * r[i];
  }
  const double stop = 1e-30 * ff;  /* (1e-15 ||f||)^2 */
  double best = rr;
  int stalled = 0;
  for (int it = 0; it < 100000 && rr > stop && stalled < 50; ++it) {
    dtd_apply(n, p, q);
    double pq = 0.0;
    for (size_t i = 0; i < n3; ++i) {
      q[i] = p[i] + a * q[i];
      pq += p[i] * q[i];
    }
    if (!(pq > 0.0)) break;
    double alpha = rr / pq, rr_new = 0.0;
    for (size_t i = 0; i < n3; ++i) {
      out[i] += alpha * p[i];
      r[i] -= alpha * q[i];
      rr_new += r[i] * r[i];
    }
    double beta = rr_new / rr;
    for (size_t i = 0; i < n3; ++i) p[i] = r[i] + beta * p[i];
    rr = rr_new;
    if (rr < best) {
      best = rr;
      stalled = 0;
    } else {
      ++stalled;
    }
  }
  free(r);
  free(p);
  free(q);
}

/* --------------------------------------------- forward operator A = P W -- */

typedef struct {
  int n, pad, nw, nth, nt, precond;
  double dt, T, cfl;
  double *kappa; /* on the wave grid, nw^3 */
} ffo_setup_t;

/* The wave grid: the image box [-1,1]^3 (n cells per axis, dx = 2/n) enlarged
 * by pad cells of the same size on every side, nw = n + 2 pad.  This is the
 * V_T of the wave model (Sec. 2.1: W_T maps sources supported in V to fields
 * supported in a larger V_T, and the X-ray transform acts on V_T); the
 * paper's experiments compute on such an enlarged domain (Sec. 5).  c is
 * given on the wave grid and Nt follows from its maximum and dx; the data
 * are the projections of the whole wave grid: nw planes of nw detectors of
 * spacing dx.  pad = 0 is the box itself. */
static int setup(ffo_setup_t *s, int n, int pad, double T, double cfl, int nth, int precond,
                 const double *c) {
  s->n = n;
  s->pad = pad;
  s->nw = n + 2 * pad;
  size_t nw3 = (size_t)s->nw * s->nw * s->nw;
  s->nth = nth;
  s->T = T;
  s->cfl = cfl;
  s->precond = precond;
  s->nt = ffo_time_steps(n, T, cfl, ffo_max(nw3, c), &s->dt);
  s->kappa = malloc(nw3 * sizeof(double));
  double dx = 2.0 / n;
  for (size_t i = 0; i < nw3; ++i) {
    double r = c[i] * s->dt / dx;
    s->kappa[i] = r * r;
  }
  return s->nt;
}

static size_t wave_len(const ffo_setup_t *s) { return (size_t)s->nw * s->nw * s->nw; }
static size_t data_len(const ffo_setup_t *s) { return (size_t)s->nth * s->nw * s->nw; }

/* zero-extension E of an image-grid volume (n^3) to the wave grid (nw^3) */
static void embed(int n, int pad, const double *in, double *out) {
  int nw = n + 2 * pad;
  memset(out, 0, (size_t)nw * nw * nw * sizeof(double));
  for (int z = 0; z < n; ++z)
    for (int y = 0; y < n; ++y)
      for (int x = 0; x < n; ++x) out[at3(nw, z + pad, y + pad, x + pad)] = in[at3(n, z, y, x)];
}

/* its transpose E^T: the box cells of a wave-grid volume */
static void restrict_box(int n, int pad, const double *in, double *out) {
  int nw = n + 2 * pad;
  for (int z = 0; z < n; ++z)
    for (int y = 0; y < n; ++y)
      for (int x = 0; x < n; ++x) out[at3(n, z, y, x)] = in[at3(nw, z + pad, y + pad, x + pad)];
}

/* W_T E h: the field on the wave grid (nw^3) at time T of the source h on the box */
static void wave_out(const ffo_setup_t *s, const double *h, double *out) {
  if (s->pad == 0) {
    ffo_wave(s->n, s->nt, s->kappa, h, out);
    return;
  }
  double *a = malloc(wave_len(s) * sizeof(double));
  embed(s->n, s->pad, h, a);
  ffo_wave(s->nw, s->nt, s->kappa, a, out);
  free(a);
}

/* its transpose E^T W_T^T: a wave-grid volume to the box */
static void wave_back(const ffo_setup_t *s, const double *g, double *out) {
  if (s->pad == 0) {
    ffo_wave_adjoint(s->n, s->nt, s->kappa, g, out);
    return;
  }
  double *b = malloc(wave_len(s) * sizeof(double));
  ffo_wave_adjoint(s->nw, s->nt, s->kappa, g, b);
  restrict_box(s->n, s->pad, b, out);
  free(b);
}

/* transpose = 0: out (nw^3) = W_T E in (in: n^3); transpose = 1: out (n^3)
 * = E^T W_T^T in (in: nw^3).  Returns Nt. */
int ffo_wave_pad(int n, int pad, double T, double cfl, const double *c, const double *in,
                 double *out, int transpose) {
  ffo_setup_t s;
  setup(&s, n, pad, T, cfl, 0, 0, c);
  if (transpose)
    wave_back(&s, in, out);
  else
    wave_out(&s, in, out);
  free(s.kappa);
  return s.nt;
}

/* g = P W_T E h (Problem 1 with full data, M = R^2): g is n_angles x nw x nw */
int ffo_forward_pad(int n, int pad, double T, double cfl, int nth, const double *c,
                    const double *h, double *g) {
  ffo_setup_t s;
  setup(&s, n, pad, T, cfl, nth, 0, c);
  double *p = malloc(wave_len(&s) * sizeof(double));
  wave_out(&s, h, p);
  ffo_project_g(s.nw, n, nth, p, g);
  free(p);
  free(s.kappa);
  return s.nt;
}

int ffo_forward(int n, double T, double cfl, int nth, const double *c, const double *h, double *g) {
  return ffo_forward_pad(n, 0, T, cfl, nth, c, h, g);
}

/* h = E^T W_T^T P^T g */
int ffo_adjoint_pad(int n, int pad, double T, double cfl, int nth, const double *c,
                    const double *g, double *h) {
  ffo_setup_t s;
  setup(&s, n, pad, T, cfl, nth, 0, c);
  double *a = malloc(wave_len(&s) * sizeof(double));
  ffo_backproject_g(s.nw, n, nth, g, a);
  wave_back(&s, a, h);
  free(a);
  free(s.kappa);
  return s.nt;
}

int ffo_adjoint(int n, double T, double cfl, int nth, const double *c, const double *g, double *h) {
  return ffo_adjoint_pad(n, 0, T, cfl, nth, c, g, h);
}

static double dot(size_t len, const double *a, const double *b) {
  double acc = 0.0;
  for (size_t i = 0; i < len; ++i) acc += a[i] * b[i];
  return acc;
}

/* grad = A^T chi Lambda chi (A h - g) with the data mask chi (Problem 1:
 * chi_M, NULL = full data); r_out = chi (A h - g); lr_out = chi Lambda r.
 * work: a wave-grid volume. */
static void data_gradient_m(const ffo_setup_t *s, const double *h, const double *g,
                            const double *mask, double *r, double *lr, double *grad,
                            double *work) {
  int n = s->n, nw = s->nw, nth = s->nth;
  size_t nd = data_len(s);
  wave_out(s, h, work);
  ffo_project_g(nw, n, nth, work, r);
  for (size_t i = 0; i < nd; ++i) r[i] = (r[i] - g[i]) * (mask ? mask[i] : 1.0);
  if (s->precond)
    ffo_ramp_g(nw, n, nth, r, lr);
  else
    memcpy(lr, r, nd * sizeof(double));
  if (mask)
    for (size_t i = 0; i < nd; ++i) lr[i] *= mask[i];
  ffo_backproject_g(nw, n, nth, lr, work);
  wave_back(s, work, grad);
}

/* Largest eigenvalue of A^T chi Lambda chi A (mask = chi_M, NULL = full data)
 * by power iteration from v0 (the step size bound 1/L; not in the paper,
 * which fixes s = 0.2 for its own scaling). */
double ffo_power_ex(int n, int pad, double T, double cfl, int nth, int precond, const double *c,
                    const double *mask, const double *v0, int iters) {
  ffo_setup_t s;
  size_t n3 = (size_t)n * n * n;
  setup(&s, n, pad, T, cfl, nth, precond, c);
  size_t nd = data_len(&s);
  double *v = malloc(n3 * sizeof(double)), *w = malloc(n3 * sizeof(double));
  double *work3 = malloc(wave_len(&s) * sizeof(double));
  double *r = malloc(nd * sizeof(double)), *lr = malloc(nd * sizeof(double));
  double *zero = calloc(nd, sizeof(double));
  double nv = sqrt(dot(n3, v0, v0));
  for (size_t i = 0; i < n3; ++i) v[i] = v0[i] / nv;
  double lam = 0.0;
  for (int it = 0; it < iters; ++it) {
    data_gradient_m(&s, v, zero, mask, r, lr, w, work3); /* w = A^T chi Lambda chi A v */
    double nw = sqrt(dot(n3, w, w));
    lam = nw;
    for (size_t i = 0; i < n3; ++i) v[i] = w[i] / nw;
  }
  free(v);
  free(w);
  free(work3);
  free(r);
  free(lr);
  free(zero);
  free(s.kappa);
  return lam;
}

double ffo_power(int n, double T, double cfl, int nth, int precond, const double *c,
                 const double *v0, int iters) {
  return ffo_power_ex(n, 0, T, cfl, nth, precond, c, NULL, v0, iters);
}

/* Algorithm 8 (preconditioned proximal forward-backward, Sec. 3.2) with
 * R = ||h||_1 + indicator(h >= 0), the data mask chi_M of Problem 1 (mask,
 * NULL = full data) and the source support chi_V (support, NULL = the whole
 * grid): r_k = A^T chi Lambda chi (A h_k - g) and
 * h_{k+1} = chi_V max(h_k - s r_k - s lambda, 0) (the prox of
 * s lambda (||.||_1 + i_{>=0}) + i_V).  With mask and support NULL this is
 * the plain Algorithm 8.  reg = 1 takes the paper's experimental regulariser
 * R = 1/2 |grad h|^2 instead (ffo_prox_grad; support must be NULL): then
 * h_{k+1} = prox_{s lambda R}(h_k - s r_k) and the objective carries
 * lambda R(h_k).
 * stats[4 k + {0,1,2,3}] = objective 1/2 <Lambda r, r> + lambda ||h_k||_1,
 * ||chi (A h_k - g)||_2, ||h_{k+1} - h_k|| / max(||h_k||, 1e-300), ||h_{k+1}||_2.
 * Returns the number of iterations run (stops early when tol > 0 and the
 * relative change drops below tol). */
int ffo_fb_ex(int n, int pad, double T, double cfl, int nth, int precond, const double *c,
              const double *g, const double *mask, const double *support, int reg,
              double lambda, double step, int iters, double tol, double *h, double *stats) {
  ffo_setup_t s;
  size_t n3 = (size_t)n * n * n;
  if (reg == 1 && support) return -1; /* the smoothing prox is defined on the whole box */
  setup(&s, n, pad, T, cfl, nth, precond, c);
  size_t nd = data_len(&s);
  double *grad = malloc(n3 * sizeof(double)), *work3 = malloc(wave_len(&s) * sizeof(double));
  double *r = malloc(nd * sizeof(double)), *lr = malloc(nd * sizeof(double));
  double dx = 2.0 / n;
  int k;
  for (k = 0; k < iters; ++k) {
    data_gradient_m(&s, h, g, mask, r, lr, grad, work3);
    double l1 = 0.0, hh = 0.0, dd = 0.0, nn = 0.0;
    if (reg == 1) {
      /* h_{k+1} = prox_{s lambda R}(h_k - s r_k), R = 1/2 |grad h|^2 */
      l1 = 0.5 * ffo_grad_energy(n, h) / (dx * dx);
      for (size_t i = 0; i < n3; ++i) grad[i] = h[i] - step * grad[i];
      ffo_prox_grad(n, step * lambda / (dx * dx), grad, work3);
    }
    for (size_t i = 0; i < n3; ++i) {
      double hn;
      if (reg == 1) {
        hn = work3[i];
      } else {
        double f = h[i] - step * grad[i] - step * lambda;
        hn = f > 0.0 ? f : 0.0;
        if (support) hn *= support[i];
        l1 += fabs(h[i]);
      }
      hh += h[i] * h[i];
      dd += (hn - h[i]) * (hn - h[i]);
      nn += hn * hn;
      h[i] = hn;
    }
    double rel = sqrt(dd) / (sqrt(hh) > 1e-300 ? sqrt(hh) : 1e-300);
    if (stats) {
      stats[4 * k + 0] = 0.5 * dot(nd, lr, r) + lambda * l1;
      stats[4 * k + 1] = sqrt(dot(nd, r, r));
      stats[4 * k + 2] = rel;
      stats[4 * k + 3] = sqrt(nn);
    }
    if (tol > 0.0 && rel < tol) {
      ++k;
      break;
    }
  }
  free(grad);
  free(work3);
  free(r);
  free(lr);
  free(s.kappa);
  return k;
}

int ffo_fb(int n, double T, double cfl, int nth, int precond, const double *c, const double *g,
           double lambda, double step, int iters, double tol, double *h, double *stats) {
  return ffo_fb_ex(n, 0, T, cfl, nth, precond, c, g, NULL, NULL, 0, lambda, step, iters, tol, h,
                   stats);
}

/* ------------------------------------------- gradient with respect to c -- */

/* Gradient of the scalar <grad_g, A h> with respect to c (the differentiated
 * forward operator, chain rule through kappa = (c dt / dx)^2 with dt held
 * fixed): keep every p^n of W, run the transposed recurrence backwards
 * (lambda^{Nt} = P^T grad_g, lambda^n = 2 lambda^{n+1} - lambda^{n+2}
 * + L4(kappa lambda^{n+1}), lambda^0 = lambda^1 + 1/2 L4(kappa lambda^1)
 * - lambda^2), and sum the kappa-derivatives of every step:
 * d/dkappa = sum_{n>=1} lambda^{n+1} L4 p^n + 1/2 lambda^1 L4 p^0.
 * grad_h (optional) receives lambda^0 = A^T grad_g. */
int ffo_grad(int n, double T, double cfl, int nth, const double *c, const double *h,
             const double *grad_g, double *grad_h, double *grad_c) {
  ffo_setup_t s;
  size_t n3 = (size_t)n * n * n;
  setup(&s, n, 0, T, cfl, nth, 0, c);
  int nt = s.nt;
  double *ps = malloc((size_t)(nt + 1) * n3 * sizeof(double)); /* p^0 .. p^nt */
  double *lap = malloc(n3 * sizeof(double));
  memcpy(ps, h, n3 * sizeof(double));
  lap4(ps, n, lap);
  for (size_t i = 0; i < n3; ++i) ps[n3 + i] = ps[i] + 0.5 * s.kappa[i] * lap[i];
  for (int k = 1; k < nt; ++k) {
    const double *cur = ps + (size_t)k * n3, *prev = ps + (size_t)(k - 1) * n3;
    double *next = ps + (size_t)(k + 1) * n3;
    lap4(cur, n, lap);
    for (size_t i = 0; i < n3; ++i) next[i] = 2.0 * cur[i] - prev[i] + s.kappa[i] * lap[i];
  }
  double *later = calloc(n3, sizeof(double)); /* lambda^{n+2} */
  double *cur = malloc(n3 * sizeof(double));  /* lambda^{n+1} */
  double *kl = malloc(n3 * sizeof(double));
  double *gk = calloc(n3, sizeof(double));    /* d/dkappa */
  ffo_backproject(n, nth, grad_g, cur);       /* lambda^{nt} */
  for (int k = nt - 1; k >= 0; --k) {         /* lambda^{k+1} in cur -> lambda^k */
    lap4(ps + (size_t)k * n3, n, lap);
    double w = k >= 1 ? 1.0 : 0.5;
    for (size_t i = 0; i < n3; ++i) gk[i] += w * cur[i] * lap[i];
    for (size_t i = 0; i < n3; ++i) kl[i] = s.kappa[i] * cur[i];
    lap4(kl, n, lap);
    for (size_t i = 0; i < n3; ++i) {
      double earlier = k >= 1 ? 2.0 * cur[i] - later[i] + lap[i] : cur[i] + 0.5 * lap[i] - later[i];
      later[i] = cur[i];
      cur[i] = earlier;
    }
  }
  if (grad_h) memcpy(grad_h, cur, n3 * sizeof(double));
  if (grad_c)
    for (size_t i = 0; i < n3; ++i) grad_c[i] = gk[i] * 2.0 * s.kappa[i] / c[i];
  free(ps);
  free(lap);
  free(later);
  free(cur);
  free(kl);
  free(gk);
  free(s.kappa);
  return nt;
}

/* ------------------------------------------------- two-step method (Alg. 9) -- */

/* X^{-1} G = X^* Lambda G applied plane by plane (Sec. 3.1: filtered
 * backprojection); the discrete form (2 pi / (n_angles dx)) P^T Lambda G,
 * where 2 pi / n_angles is the angle weight of the backprojection over S^1
 * and 1/dx undoes the sample length of P^T. */
void ffo_fbp_g(int ng, int nimg, int nth, const double *G, double *out) {
  size_t nd = (size_t)nth * ng * ng, n3 = (size_t)ng * ng * ng;
  double *lr = malloc(nd * sizeof(double));
  ffo_ramp_g(ng, nimg, nth, G, lr);
  ffo_backproject_g(ng, nimg, nth, lr, out);
  double w = 2.0 * FFO_PI / (nth * (2.0 / nimg));
  for (size_t i = 0; i < n3; ++i) out[i] *= w;
  free(lr);
}

void ffo_fbp(int n, int nth, const double *G, double *out) { ffo_fbp_g(n, n, nth, G, out); }

/* Algorithm 9: g = X^{-1} G (on the wave grid), then
 * h_{k+1} = prox_{s lambda R}(h_k - s W^T (W h_k - g)) with W = W_T E (box to
 * wave grid) and R = ||h||_1 + indicator(h >= 0) (reg = 0) or
 * R = 1/2 |grad h|^2 (reg = 1).  stats[4 k + 0..3]: objective
 * 1/2 ||W h_k - g||^2 + lambda R(h_k), ||W h_k - g||, relative change,
 * ||h_{k+1}||. */
int ffo_fb_two_step(int n, int pad, double T, double cfl, int nth, const double *c,
                    const double *G, int reg, double lambda, double step, int iters, double tol,
                    double *h, double *stats) {
  ffo_setup_t s;
  size_t n3 = (size_t)n * n * n;
  setup(&s, n, pad, T, cfl, nth, 0, c);
  size_t nw3 = wave_len(&s);
  double *g = malloc(nw3 * sizeof(double)), *r = malloc(nw3 * sizeof(double));
  double *grad = malloc(n3 * sizeof(double)), *prox = malloc(n3 * sizeof(double));
  double dx = 2.0 / n;
  ffo_fbp_g(s.nw, n, nth, G, g);
  int k;
  for (k = 0; k < iters; ++k) {
    wave_out(&s, h, r);
    for (size_t i = 0; i < nw3; ++i) r[i] -= g[i];
    wave_back(&s, r, grad);
    double l1 = 0.0, hh = 0.0, dd = 0.0, nn = 0.0;
    if (reg == 1) {
      l1 = 0.5 * ffo_grad_energy(n, h) / (dx * dx);
      for (size_t i = 0; i < n3; ++i) grad[i] = h[i] - step * grad[i];
      ffo_prox_grad(n, step * lambda / (dx * dx), grad, prox);
    }
    for (size_t i = 0; i < n3; ++i) {
      double hn;
      if (reg == 1) {
        hn = prox[i];
      } else {
        double f = h[i] - step * grad[i] - step * lambda;
        hn = f > 0.0 ? f : 0.0;
        l1 += fabs(h[i]);
      }
      hh += h[i] * h[i];
      dd += (hn - h[i]) * (hn - h[i]);
      nn += hn * hn;
      h[i] = hn;
    }
    double rel = sqrt(dd) / (sqrt(hh) > 1e-300 ? sqrt(hh) : 1e-300);
    if (stats) {
      stats[4 * k + 0] = 0.5 * dot(nw3, r, r) + lambda * l1;
      stats[4 * k + 1] = sqrt(dot(nw3, r, r));
      stats[4 * k + 2] = rel;
      stats[4 * k + 3] = sqrt(nn);
    }
    if (tol > 0.0 && rel < tol) {
      ++k;
      break;
    }
  }
  free(g);
  free(r);
  free(grad);
  free(prox);
  free(s.kappa);
  return k;
}
