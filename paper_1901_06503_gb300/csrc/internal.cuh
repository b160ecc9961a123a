// internal.cuh -- shared declarations of the ffpat CUDA library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include <nvtx3/nvToolsExt.h>

#include "../../include/ffpat.h"

namespace ffpat {

constexpr int kNumSMs = 152;           // GB300: 2 dies x 76 SMs
constexpr int kReduceBlocks = 4 * kNumSMs;  // fixed grid of every deterministic reduction
constexpr int kReduceThreads = 256;
constexpr int kNumQuant = 8;           // quantities one reduction pass can carry

// Derived, validated problem plus the carve of the caller's workspace.
// Grid fields (n, n3, kap) describe the image box (the source domain V);
// with padding the wave runs on a grid of nw = n + 2 pad points per axis (the
// V_T of the wave model) whose view wave_plan() gives.  The data are always
// the projections of the wave grid: nd = nth nw^2 values, ns samples per ray.
struct Plan {
  int n = 0, nth = 0, ns = 0, nt = 0, prec = 0, precond = 0;
  int pad = 0, nw = 0;    // cells of padding per side; wave grid points per axis
  int nimg = 0;           // box points per axis in every view (cell size 2 / nimg)
  double T = 0, cfl = 0, dx = 0, dt = 0, cmax = 0;
  size_t n3 = 0, nd = 0, esize = 0, nw3 = 0;
  // workspace carve (device)
  void* kap = nullptr;    // kappa / 12 on the image box
  void* kapw = nullptr;   // kappa / 12 on the wave grid (== kap without padding)
  void* s[6] = {};        // wavefield state (wave grid): three-term p^{n-1}, p^n; increment form p, p', d, e, d', e'
  void* xw = nullptr;     // wave-grid input of a padded W or W^T
  void* xo = nullptr;     // image-box result of a padded W^T
  void* xg = nullptr;     // wave-grid scratch (the FBP of Algorithm 9 when padded)
  void* x = nullptr;      // image-domain scratch (adjoint input / gradient)
  void* v = nullptr;      // image-domain scratch (power iteration vector)
  void* r = nullptr;      // data-domain scratch (residual)
  void* r2 = nullptr;     // data-domain scratch (Lambda residual)
  double* partials = nullptr;  // kNumQuant * kReduceBlocks doubles
  double* scal = nullptr;      // small device scalars
  double* hist = nullptr;      // per-iteration FB statistics (8 doubles / iteration, up to kMaxHist)
  double* tab = nullptr;       // cos[nth], sin[nth] (double, host libm)
  float* tabf = nullptr;       // cos[nth], sin[nth] rounded to float
  int32_t* tabi = nullptr;     // cos[nth], sin[nth] in fixed point, round(. * 2^30)
  void* dct = nullptr;         // DCT-II matrix C and C^T (n^2 each, element type), then mu[n] (double)
  const double* dct_mu = nullptr;
  unsigned* sync = nullptr;    // step flags of the resident time loop (kResidentMaxItems)
};
// The plan as the wave kernels see it: the wave grid and its kappa.
inline Plan wave_plan(const Plan& pl) {
  Plan w = pl;
  w.n = pl.nw;
  w.n3 = pl.nw3;
  w.kap = pl.kapw;
  return w;
}
// bytes of the three angle tables (double, float, fixed point) for nth angles
inline size_t table_bytes(int nth) { return (size_t)nth * 2 * (8 + 4 + 4); }
constexpr int kMaxHist = 4096;
constexpr int kResidentMaxItems = 1024;  // work items (step flags) of the resident time loop
constexpr int kScal = 64;

// api.cu helpers shared with the server and the gradient path
int setup(const ffpat_problem* pr, Plan& pl, const void* c, void* ws, size_t ws_bytes,
          cudaStream_t st);
// one three-term leapfrog launch (TMA kernel when the layout allows)
int step3(const Plan& pl, bool tma, bool start, const void* p, const void* qin, void* qout,
          void* copy0, cudaStream_t st);
// whether a three-term FP32 time loop takes two steps per pass (W's own rule)
bool two_step_three_term(const Plan& pl, bool tma);
int attach(const ffpat_problem* pr, Plan& pl, void* ws, size_t ws_bytes);
int time_steps(const Plan& pl, double cmax, int* nt, double* dt);
void fill_tables_host(int nth, unsigned char* buf);  // table_bytes(nth) bytes

// An NVTX range for the lifetime of a scope: the library's phases (entry
// points, wave time loops, the data-side kernels, FB iterations, serving
// ticks) appear by name in profiler timelines.  Without a profiler attached
// the push and pop cost a few nanoseconds.
struct Trace {
  explicit Trace(const char* name) { nvtxRangePushA(name); }
  ~Trace() { nvtxRangePop(); }
  Trace(const Trace&) = delete;
  Trace& operator=(const Trace&) = delete;
};

// While an object of this type lives, wave time loops on this host thread are
// not captured into CUDA graphs (used by the allocation-free entry point).
struct NoGraphs {
  NoGraphs();
  ~NoGraphs();
  NoGraphs(const NoGraphs&) = delete;
  NoGraphs& operator=(const NoGraphs&) = delete;
};

// ---------------------------------------------------------------- launches --
void count_launch(int k = 1);
// FFPAT_OK, or FFPAT_ECUDA with the pending launch error recorded for ffpat_last_error()
int check_launch(const char* what);
// record a formatted message for ffpat_last_error() and return `code`
int report(int code, const char* fmt, ...);

// stencil.cu
// three-term form.  start: out_p1 = p0 + kap*L(p0)/2 and copy_p0 = p0 (may be null)
int launch_step3(const Plan& pl, const void* p, const void* qin, void* qout, bool start,
                 void* copy_p0, cudaStream_t st);
// increment form (FP32 only).  start: d = kap L(p)/2, e = Kahan carry, pout = p + d.
int launch_step_inc(const Plan& pl, const void* pin, void* pout, void* d, void* e, bool start,
                    cudaStream_t st);

// stencil_tma.cu: the same steps fed by TMA (needs N % 4 == 0 for float, N % 2
// == 0 for double, 16-byte aligned arrays).  form 0: three-term, q = {p^{n-1},
// kap} (start: {kap}), o0 = p^{n+1}, o1 = copy of p^0 at start; form 1:
// increment, q = {d, e, kap} (start: {kap}), o0 = p^{n+1}, o1 = d, o2 = e.
bool tma_supported(const Plan& pl, const void* const* ptrs, int count);
int launch_step_tma(const Plan& pl, int form, bool start, const void* p, const void* const* q,
                    void* o0, void* o1, void* o2, cudaStream_t st);
// One FP32-Kahan leapfrog step for each of `count` independent problems in a
// single launch (same arithmetic as launch_step_tma form 1).  start: the step
// p^1 = p^0 + d^1 with d, e written, else the regular step reading d, e.
struct BatchStep {
  const float* p;   // p^n (N^3, 16-byte aligned, N % 4 == 0)
  float* pout;      // p^{n+1}
  float* d;         // increment, updated in place
  float* e;         // Kahan carry, updated in place
  const float* kap; // kappa / 12
  int n;
  bool start;
};
int launch_step_batch(const BatchStep* steps, int count, cudaStream_t st);
// Two FP32-Kahan steps for several problems in one launch (the two-step pass
// of launch_step2_kahan per problem; d and e are read with a halo, so they go
// to separate output buffers).
struct BatchStep2 {
  const float* p;    // p^n
  float* pout;       // p^{n+2}
  const float* d;    // d^n, e^n
  const float* e;
  float* dout;       // d^{n+2}, e^{n+2}
  float* eout;
  const float* kap;  // kappa / 12
  int n;
};
int launch_step2_batch(const BatchStep2* steps, int count, cudaStream_t st);
// The two-step passes address a grid with 32-bit offsets: N^3 < 2^32, N <= 1624
// (larger grids take single steps, whose offsets are 64-bit).
constexpr int kTwoStepMaxN = 1624;
constexpr int kMaxBatchRequests = 28;

// Two FP32-Kahan steps in one pass (temporal blocking): reads (p, d, e) at
// level n with halos, writes level n + 2 to (po, dout, eout), which must not
// alias the inputs.  TMA layout rules as launch_step_tma.
int launch_step2_kahan(const Plan& pl, const void* p, const void* d, const void* e, void* po,
                       void* dout, void* eout, cudaStream_t st);
// The whole FP32 time loop of W in one cooperative launch (grids whose work
// items fit the GPU's CTA slots, N <= 128 on GB300; see stencil_tma.cu):
// form 1 increment with Kahan carry, form 0 three-term.  Reads p^0 from `in`,
// ping-pongs p through b0 (even steps) and b1 (odd steps), writes the last
// step to `out` when non-null; *result = the buffer holding p^{nt}.  Bit for
// bit the single-step loop.  resident_zc: the z-range of its work items, 0
// when the grid does not fit (the step-by-step loop runs instead).  *refused
// (may be null) is set when the cooperative launch was turned down because
// the grid cannot be co-resident at the moment: nothing ran.
int resident_zc(const Plan& pl, int form);
int launch_wave_resident(const Plan& pl, int form, const void* in, void* out, void* b0, void* b1,
                         const void** result, cudaStream_t st, bool* refused = nullptr);
// Two FP32 three-term leapfrog steps in one HBM pass (needs N % 4 == 0, 16-byte
// aligned arrays): reads p^{n-1} (pm) and p^n (p), writes p^{n+1} (o1) and
// p^{n+2} (o2); o1, o2 alias neither input.  Bit-identical to two single steps.
int launch_step2_f32(const Plan& pl, const void* pm, const void* p, void* o1, void* o2,
                     cudaStream_t st);

// device status word of the TMA kernels (0 = ok, else -FFPAT_* of the first error)
int read_device_status(unsigned* out, bool clear);
int launch_wait_timeout(long long cycles, cudaStream_t st);

// xray.cu
// g = mask .* (P p - sub)  (sub, mask nullable)
// scratch (nullable): a volume of the plan's grid that aliases neither p nor
// g; when the planes are too large for shared memory it receives a transposed
// copy of p, from which the steep angles read (same result, coalesced loads).
int launch_project(const Plan& pl, const void* p, void* g, const void* sub, cudaStream_t st,
                   const void* mask = nullptr, void* scratch = nullptr);
// bytes of that scratch (0 when the shared-memory kernel is used)
size_t project_scratch_bytes(const Plan& pl);
// h = mult * scale .* P^T g  (scale nullable)
int launch_backproject(const Plan& pl, const void* g, void* h, const void* scale, cudaStream_t st,
                       double mult = 1.0);
// out = mask .* (Lambda r)  (mask nullable)
int launch_ramp(const Plan& pl, const void* r, void* out, cudaStream_t st,
                const void* mask = nullptr);
int launch_debug_samples(const Plan& pl, int count, const int32_t* jkm, int32_t* ij, double* f,
                         cudaStream_t st);

// fb.cu
int launch_speed_stats(const Plan& pl, const void* c, double* out3, cudaStream_t st);
int launch_kappa(const Plan& pl, const void* c, cudaStream_t st);
// out[i] = a[i] * kap[i] (mul = true) or a[i] / kap[i]
// prox.cu: prox of the gradient regulariser, (I + a D^T D)^{-1} in -> out
// through the scratch volumes s0, s1 (in, out != s0, s1; in == out allowed).
size_t dct_bytes(int n, size_t esize);
int upload_dct(const Plan& pl, cudaStream_t st);  // fills pl.dct (synchronises)
int launch_prox_grad(const Plan& pl, double a, const void* in, void* out, void* s0, void* s1,
                     cudaStream_t st);
// FB step with that prox: x = h - s w / kap; then, after the prox wrote hn,
// the statistics rows (R(h), ||h||^2, ||hn - h||^2, ||hn||^2) and h = hn.
int launch_prox_prep(const Plan& pl, const void* h, const void* w, double step, void* x,
                     cudaStream_t st, const double* step_dev = nullptr);
int launch_prox_finish(const Plan& pl, void* h, const void* hn, double* dst, cudaStream_t st);
// padding: box (n^3) -> wave grid (zero outside the box), and wave grid -> box
int launch_embed(const Plan& pl, const void* box, void* wave, cudaStream_t st);
int launch_restrict(const Plan& pl, const void* wave, void* box, cudaStream_t st);
int launch_kscale(const Plan& pl, const void* a, void* out, bool mul, cudaStream_t st);
// out[i] = a[i] * s  (s a device double)
int launch_scale_dev(const Plan& pl, size_t len, const void* a, void* out, const double* s,
                     cudaStream_t st);
// scal[q] = deterministic FP64 dot products over `len` elements
int launch_dot(const Plan& pl, size_t len, const void* a, const void* b, double* result,
               cudaStream_t st);
// FB update + partial norms; results land in dst[0..3]
// step_dev (optional): read the step from device memory instead of `step`
// support (nullable): the iterate is multiplied by it (projection onto the source support)
int launch_fb_update(const Plan& pl, void* h, const void* w, double step, double lambda,
                     double* dst, cudaStream_t st, const double* step_dev = nullptr,
                     const void* support = nullptr);
int launch_inv_sqrt(const double* src, double* dst, cudaStream_t st);
int launch_sub_div(const Plan& pl, const void* a, const void* b, void* out, cudaStream_t st);
// x = kap (w - g), dst[0] = dst[1] = sum (w - g)^2
int launch_resid_kap(const Plan& pl, const void* w, const void* g, void* x, double* dst,
                     cudaStream_t st);
int launch_scale_div(const Plan& pl, const void* a, const void* c, double s, void* out,
                     cudaStream_t st);
// stencil.cu: acc += w * u * L(p)
int launch_lap_accum(const Plan& pl, void* acc, const void* u, const void* p, double w,
                     cudaStream_t st);
int launch_hash_fill(const Plan& pl, void* out, uint64_t seed, cudaStream_t st);

}  // namespace ffpat
