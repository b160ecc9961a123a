// api.cu -- the extern "C" boundary of the library (include/ffpat.h): argument
// validation, workspace carve, the time loops of W and W^T, and the host
// driver of Algorithm 8 (Sec. 3.2).
//
// The adjoint wave operator is applied as W^T = K^-1 W K with K = diag(kap):
// W = T_Nt(I + K L4 / 2) is a polynomial in K L4 (the leapfrog with the zero-
// velocity start step is the Chebyshev recurrence), so its transpose is the
// same polynomial in L4 K = K^-1 (K L4) K.  One stencil kernel therefore
// serves both directions; the K scalings are fused into the backprojection
// (on entry) and the gradient step (on exit).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <mutex>
#include <vector>

#include "internal.cuh"

namespace ffpat {

static thread_local char g_err[512] = "";
static std::atomic<long long> g_launches{0};
static std::atomic<long long> g_prof_launches{0};
static std::atomic<int> g_prof_on{0};
// 0 auto, 1 plain 2.5D kernel, 2 single-step TMA kernel, 3 two-step TMA kernel (FP32-Kahan),
// 4 resident time loop (FP32, FP32-Kahan)
static std::atomic<int> g_stencil_path{0};

struct ProfRec {
  cudaEvent_t a, b;
  long long steps;     // leapfrog steps timed
  long long launches;  // kernel launches (one HBM pass each) timed
  double bytes;        // algorithmic bytes: one pass of the state per launch
};
static std::mutex g_prof_mu;
static std::vector<ProfRec> g_prof;

void count_launch(int k) {
  g_launches += k;
  if (g_prof_on.load(std::memory_order_relaxed)) g_prof_launches += k;
}

static int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
  return code;
}

int report(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
  return code;
}

int check_launch(const char* what) {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(FFPAT_ECUDA, "%s: %s", what, cudaGetErrorString(e));
  return FFPAT_OK;
}

#define CK(call)                                                                       \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return fail(FFPAT_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));        \
  } while (0)

#define TRY(expr)                \
  do {                           \
    const int r_ = (expr);       \
    if (r_ != FFPAT_OK) return r_; \
  } while (0)

static size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

// Validate the problem and fill the size fields of the plan.
static int validate(const ffpat_problem* pr, Plan& pl) {
  g_err[0] = 0;
  if (!pr) return fail(FFPAT_EINVAL, "problem is NULL");
  if (pr->n < 1 || pr->n > 2048) return fail(FFPAT_EINVAL, "n = %d outside [1, 2048]", pr->n);
  if (!(pr->T > 0.0) || !isfinite(pr->T)) return fail(FFPAT_EINVAL, "T must be finite and > 0");
  if (!(pr->cfl > 0.0) || !(pr->cfl <= 0.5))
    return fail(FFPAT_EINVAL, "cfl = %g outside (0, 0.5] (leapfrog stability of L4)", pr->cfl);
  if (pr->n_angles < 1 || pr->n_angles > 65535)
    return fail(FFPAT_EINVAL, "n_angles = %d outside [1, 65535]", pr->n_angles);
  if (pr->precision < FFPAT_FP64 || pr->precision > FFPAT_FP32_KAHAN)
    return fail(FFPAT_EINVAL, "unknown precision %d", pr->precision);
  if (pr->precond < FFPAT_PRECOND_NONE || pr->precond > FFPAT_PRECOND_RAMP)
    return fail(FFPAT_EINVAL, "unknown preconditioner %d", pr->precond);
  if (pr->pad < 0 || pr->pad > 2048 || pr->n + 2 * pr->pad > 4096)
    return fail(FFPAT_EINVAL, "pad = %d outside [0, 2048] or N + 2 pad > 4096", pr->pad);
  pl.n = pr->n;
  pl.nimg = pr->n;
  pl.nth = pr->n_angles;
  pl.ns = 2 * (int)ceil((double)(pr->n + 2 * pr->pad) / sqrt(2.0));
  pl.prec = pr->precision;
  pl.precond = pr->precond;
  pl.T = pr->T;
  pl.cfl = pr->cfl;
  pl.dx = 2.0 / pr->n;
  pl.n3 = (size_t)pl.n * pl.n * pl.n;
  pl.pad = pr->pad;
  pl.nw = pr->n + 2 * pr->pad;
  pl.nw3 = (size_t)pl.nw * pl.nw * pl.nw;
  pl.nd = (size_t)pl.nth * pl.nw * pl.nw;
  pl.esize = pl.prec == FFPAT_FP64 ? 8 : 4;
  return FFPAT_OK;
}

// state volumes: FP32-Kahan p, p' and double-buffered d, e; FP32 two pairs
// (p^{n-1}, p^n in, p^{n+1}, p^{n+2} out of a two-step pass); FP64 one pair
static int nstate(const Plan& pl) {
  return pl.prec == FFPAT_FP32_KAHAN ? 6 : (pl.prec == FFPAT_FP32 ? 4 : 2);
}

// Carve the workspace (ws == nullptr: size only).
static size_t carve(Plan& pl, void* ws) {
  char* b = (char*)ws;
  size_t off = 0;
  auto take = [&](size_t bytes) -> void* {
    void* p = b ? (void*)(b + off) : nullptr;
    off += up256(bytes);
    return p;
  };
  const size_t vol = pl.n3 * pl.esize, dat = pl.nd * pl.esize, wvol = pl.nw3 * pl.esize;
  pl.kap = take(vol);
  pl.kapw = pl.pad ? take(wvol) : pl.kap;
  for (int i = 0; i < 6; ++i) pl.s[i] = i < nstate(pl) ? take(wvol) : nullptr;
  pl.x = take(vol);
  pl.v = take(vol);
  pl.xw = pl.pad ? take(wvol) : nullptr;
  pl.xo = pl.pad ? take(vol) : nullptr;
  pl.xg = pl.pad ? take(wvol) : nullptr;
  pl.r = take(dat);
  pl.r2 = take(dat);
  pl.partials = (double*)take(sizeof(double) * kNumQuant * kReduceBlocks);
  pl.scal = (double*)take(sizeof(double) * kScal);
  pl.hist = (double*)take(sizeof(double) * 8 * kMaxHist);
  void* tabs = take(table_bytes(pl.nth));
  pl.tab = (double*)tabs;
  pl.tabf = tabs ? (float*)((char*)tabs + 16 * (size_t)pl.nth) : nullptr;
  pl.tabi = tabs ? (int32_t*)((char*)tabs + 24 * (size_t)pl.nth) : nullptr;
  pl.dct = take(dct_bytes(pl.n, pl.esize));
  pl.dct_mu = pl.dct ? (const double*)((char*)pl.dct + 2 * (size_t)pl.n * pl.n * pl.esize) : nullptr;
  pl.sync = (unsigned*)take(128 * (size_t)kResidentMaxItems);
  return off;
}

int attach(const ffpat_problem* pr, Plan& pl, void* ws, size_t ws_bytes) {
  TRY(validate(pr, pl));
  const size_t need = carve(pl, nullptr);
  if (!ws) return fail(FFPAT_EINVAL, "workspace is NULL (%zu bytes needed)", need);
  if (((uintptr_t)ws & 255) != 0) return fail(FFPAT_EINVAL, "workspace not 256-byte aligned");
  if (ws_bytes < need)
    return fail(FFPAT_ENOMEM, "workspace of %zu bytes < %zu needed", ws_bytes, need);
  carve(pl, ws);
  return FFPAT_OK;
}

void host_angles(int nth, std::vector<double>& cs_sn) {
  cs_sn.resize(2 * (size_t)nth);
  for (int j = 0; j < nth; ++j) {
    const double th = (M_PI * j) / nth;
    cs_sn[j] = cos(th);
    cs_sn[nth + j] = sin(th);
  }
}

// Fill the three angle tables at `base` (device, table_bytes(nth) bytes):
// double cos/sin, their float roundings, and round(cos/sin * 2^30) as int32
// for the fixed-point sample coordinates of the FP32 projection pair.
void fill_tables_host(int nth, unsigned char* buf) {
  std::vector<double> t;
  host_angles(nth, t);
  const size_t m = t.size();
  double* d = (double*)buf;
  float* f = (float*)(buf + 8 * m);
  int32_t* q = (int32_t*)(buf + 12 * m);
  for (size_t i = 0; i < m; ++i) {
    d[i] = t[i];
    f[i] = (float)t[i];
    q[i] = (int32_t)llrint(t[i] * 1073741824.0);
  }
}

static int upload_tables(Plan& pl, void* base, cudaStream_t st) {
  const size_t m = 2 * (size_t)pl.nth;
  std::vector<unsigned char> buf(table_bytes(pl.nth));
  fill_tables_host(pl.nth, buf.data());
  pl.tab = (double*)base;
  pl.tabf = (float*)((char*)base + 8 * m);
  pl.tabi = (int32_t*)((char*)base + 12 * m);
  CK(cudaMemcpyAsync(base, buf.data(), buf.size(), cudaMemcpyHostToDevice, st));
  // the host buffer dies at return: make sure the copy has consumed it
  CK(cudaStreamSynchronize(st));
  return FFPAT_OK;
}

int time_steps(const Plan& pl, double cmax, int* nt, double* dt) {
  const double x = pl.T * cmax / (pl.cfl * pl.dx);
  const double steps = ceil(x * (1.0 - 1e-12));
  if (!(steps < 2e9)) return fail(FFPAT_EINVAL, "T c_max / (cfl dx) = %g steps is too many", x);
  *nt = steps < 1.0 ? 1 : (int)steps;
  *dt = pl.T / *nt;
  return FFPAT_OK;
}

// c statistics -> Nt, dt, kappa (one device-to-host read of three doubles).
// c and kapw live on the wave grid; kap is kapw's restriction to the box.
static int setup_speed(Plan& pl, const void* c, cudaStream_t st) {
  if (!c) return fail(FFPAT_EINVAL, "c is NULL");
  TRY(launch_speed_stats(wave_plan(pl), c, pl.scal, st));
  double h3[3];
  CK(cudaMemcpyAsync(h3, pl.scal, sizeof h3, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (h3[2] != 0.0)
    return fail(FFPAT_EINVAL, "sound speed has %.0f entries that are not finite and > 0", h3[2]);
  pl.cmax = h3[0];
  TRY(time_steps(pl, pl.cmax, &pl.nt, &pl.dt));
  TRY(launch_kappa(wave_plan(pl), c, st));
  if (pl.pad) TRY(launch_restrict(pl, pl.kapw, pl.kap, st));
  return FFPAT_OK;
}

int setup(const ffpat_problem* pr, Plan& pl, const void* c, void* ws, size_t ws_bytes,
          cudaStream_t st) {
  g_err[0] = 0;
  TRY(attach(pr, pl, ws, ws_bytes));
  TRY(upload_tables(pl, pl.tab, st));
  TRY(setup_speed(pl, c, st));
  return FFPAT_OK;
}

// FP32 and FP32-Kahan run two steps per pass (where the resident time loop
// does not run): measured on GB300 the two-step passes win at every size from
// 128^3 to 384^3 (FP32-Kahan 15.5 / 47.5 / 133 against 18.1 / 82.5 / 262 us per
// step at 160^3 / 256^3 / 384^3; FP32 three-term 14.0 / 42.3 / 118 against
// 15.4 / 46.9 / 135), and tie at 144^3, whose 64-wide tiles are a third empty
constexpr int kTwoStepMinN = 128;

// Whether a three-term FP32 time loop takes two steps per pass: the rule of
// W's own loop (TMA layout, N in the two-step kernel's range, automatic
// choice from kTwoStepMinN or the two-step path requested)
bool two_step_three_term(const Plan& pl, bool tma) {
  const int path = g_stencil_path.load();
  return pl.prec == FFPAT_FP32 && tma && pl.n <= kTwoStepMaxN &&
         (path == 3 || (path == 0 && pl.n >= kTwoStepMinN));
}

// algorithmic HBM bytes per point of a two-step pass beyond a single step's:
// FP32-Kahan moves its 28 B once for both steps, FP32 20 B against 16 B
static double pass_extra_bytes(const Plan& pl) { return pl.prec == FFPAT_FP32 ? 4.0 : 0.0; }

static double bytes_per_point(const Plan& pl) {
  return pl.prec == FFPAT_FP64 ? 32.0 : (pl.prec == FFPAT_FP32 ? 16.0 : 28.0);
}

// One leapfrog launch, through the TMA kernel when the layout allows it.
int step3(const Plan& pl, bool tma, bool start, const void* p, const void* qin, void* qout,
          void* copy0, cudaStream_t st) {
  if (tma) {
    const void* q[2] = {start ? pl.kap : qin, pl.kap};
    return launch_step_tma(pl, 0, start, p, q, qout, copy0, nullptr, st);
  }
  return launch_step3(pl, p, qin, qout, start, copy0, st);
}

static int step_inc(const Plan& pl, bool tma, bool start, const void* pin, void* pout, void* d,
                    void* e, cudaStream_t st) {
  if (tma) {
    const void* q[3] = {start ? pl.kap : d, e, pl.kap};
    return launch_step_tma(pl, 1, start, pin, q, pout, d, e, st);
  }
  return launch_step_inc(pl, pin, pout, d, e, start, st);
}

// The launches of W applied to `in` (N^3): the result goes to `out` if
// non-null, else it stays in a state buffer whose address is returned through
// *result; *launches counts the leapfrog launches (one HBM pass each).
static int wave_sequence(const Plan& pl, const void* in, void* out, const void** result,
                         long long* nlaunch, long long* npairs, cudaStream_t st) {
  const int nt = pl.nt;
  const void* ptrs[10] = {in, out, pl.kap, pl.s[0], pl.s[1], pl.s[2], pl.s[3], pl.s[4], pl.s[5]};
  const int path = g_stencil_path.load();
  const bool tma = path != 1 && tma_supported(pl, ptrs, 9);
  if (path >= 2 && !tma)
    return fail(FFPAT_EINVAL, "TMA stencil requested but N = %d or an array alignment rules it out",
                pl.n);
  if (path == 3 && pl.prec != FFPAT_FP64 && pl.n > kTwoStepMaxN)
    return fail(FFPAT_EINVAL, "two-step pass requested but N = %d > %d", pl.n, kTwoStepMaxN);
  long long launches = 0, pairs = 0;
  if (pl.prec == FFPAT_FP32_KAHAN) {
    // two steps per pass halve the HBM bytes (kTwoStepMinN)
    const bool two = tma && pl.n <= kTwoStepMaxN &&
                     (path == 3 || (path == 0 && pl.n >= kTwoStepMinN));
    void* P[2] = {pl.s[0], pl.s[1]};
    void* D[2] = {pl.s[2], pl.s[4]};
    void* E[2] = {pl.s[3], pl.s[5]};
    int c = 0;  // index of the buffers holding the current level
    void* first = (nt == 1 && out) ? out : P[0];
    TRY(step_inc(pl, tma, true, in, first, D[0], E[0], st));
    ++launches;
    const void* cur = first;
    int left = nt - 1;
    while (left > 0) {
      const int o = 1 - c;
      if (two && left >= 2) {
        void* dst = (left == 2 && out) ? out : (cur == P[0] ? P[1] : P[0]);
        TRY(launch_step2_kahan(pl, cur, D[c], E[c], dst, D[o], E[o], st));
        ++pairs;
        cur = dst;
        c = o;
        left -= 2;
      } else {
        // one step; d and e are read halo-free, so they update in place
        void* dst = (left == 1 && out) ? out : (cur == P[0] ? P[1] : P[0]);
        TRY(step_inc(pl, tma, false, cur, dst, D[c], E[c], st));
        cur = dst;
        left -= 1;
      }
      ++launches;
    }
    if (result) *result = cur;
  } else if (nt >= 3 && two_step_three_term(pl, tma)) {
    // FP32 three-term, two steps per pass (kTwoStepMinN): 20 B per point per
    // two steps against 32 B.  The pairs (S0, S1) and (S2, S3) alternate as
    // (p^{n-1}, p^n) inputs and (p^{n+1}, p^{n+2}) outputs
    void* S[4] = {pl.s[0], pl.s[1], pl.s[2], pl.s[3]};
    TRY(step3(pl, tma, true, in, nullptr, S[1], S[0], st));  // S1 = p^1, S0 = p^0
    ++launches;
    int prev = 0, cur = 1;
    int left = nt - 1;
    const void* res = nullptr;
    while (left >= 2) {
      const int n1 = cur == 1 ? 2 : 0, n2 = n1 + 1;
      void* d2 = (left == 2 && out) ? out : S[n2];
      TRY(launch_step2_f32(pl, S[prev], S[cur], S[n1], d2, st));
      ++launches;
      ++pairs;
      left -= 2;
      prev = n1;
      cur = n2;
      res = d2;
    }
    if (left == 1) {
      // p^{n+1} over p^{n-1}, in place as in the single-step loop
      void* dst = out ? out : S[prev];
      TRY(step3(pl, tma, false, S[cur], S[prev], dst, nullptr, st));
      ++launches;
      res = dst;
    }
    if (result) *result = res;
  } else {
    void* A = pl.s[0];  // p^{n-1}
    void* B = pl.s[1];  // p^n
    if (nt == 1) {
      void* dst = out ? out : B;
      TRY(step3(pl, tma, true, in, nullptr, dst, nullptr, st));
      ++launches;
      if (result) *result = dst;
    } else {
      TRY(step3(pl, tma, true, in, nullptr, B, A, st));
      ++launches;
      for (int s = 1; s < nt; ++s) {
        void* dst = (s == nt - 1 && out) ? out : A;
        TRY(step3(pl, tma, false, B, A, dst, nullptr, st));
        A = B;
        B = dst;
        ++launches;
      }
      if (result) *result = B;
    }
  }
  *nlaunch = launches;
  *npairs = pairs;
  return FFPAT_OK;
}

// ---- CUDA graphs of the time loop.  The second time the same W (same
// buffers, step count, precision and kernel path) runs, its launch sequence is
// captured on a private stream into a graph and from then on replayed with one
// cudaGraphLaunch on the caller's stream: the host no longer issues one launch
// per step, which bounds small grids (128^3 steps take ~10 us).  FFPAT_GRAPHS=0
// turns this off; a caller that is itself capturing gets plain launches.
struct GraphEntry {
  std::vector<const void*> key;
  cudaGraphExec_t exec = nullptr;
  const void* result = nullptr;
  long long launches = 0;
  long long pairs = 0;  // two-step passes among the launches
  int device = -1;
};
static std::mutex g_graph_mu;
static std::vector<GraphEntry> g_graphs;  // most recently used last
constexpr size_t kMaxGraphs = 32;

// NoGraphs scopes on this host thread: while one is open, time loops are
// launched step by step and never captured (capture creates a stream and an
// executable graph, both of which allocate)
static thread_local int g_no_graphs = 0;
NoGraphs::NoGraphs() { ++g_no_graphs; }
NoGraphs::~NoGraphs() { --g_no_graphs; }

static bool graphs_enabled() {
  static const bool on = [] {
    const char* e = getenv("FFPAT_GRAPHS");
    return !(e && e[0] == '0');
  }();
  return on;
}

static int run_wave(const Plan& pl, const void* in, void* out, const void** result,
                    cudaStream_t st) {
  Trace trace_("W (leapfrog time loop)");
  ProfRec rec{};
  const bool prof = g_prof_on.load();
  if (prof) {
    CK(cudaEventCreate(&rec.a));
    CK(cudaEventCreate(&rec.b));
    CK(cudaEventRecord(rec.a, st));
  }
  long long launches = 0, pairs = 0;
  const void* res = nullptr;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  CK(cudaStreamIsCapturing(st, &cap));
  // grids that fit the GPU's CTA slots run the whole loop in one cooperative
  // launch (no graph: there is one launch to make; a caller that is capturing
  // gets the step-by-step loop)
  const int path = g_stencil_path.load();
  const int form = pl.prec == FFPAT_FP32_KAHAN ? 1 : 0;
  if (pl.prec != FFPAT_FP64 && (path == 4 || (path == 0 && cap == cudaStreamCaptureStatusNone))) {
    const void* ptrs[5] = {in, out, pl.kap, pl.s[0], pl.s[1]};
    const bool fits = tma_supported(pl, ptrs, 5) && resident_zc(pl, form) > 0;
    if (path == 4 && !fits)
      return fail(FFPAT_EINVAL,
                  "resident time loop requested but N = %d, the precision or an array alignment "
                  "rules it out", pl.n);
    bool refused = false;
    const int rc = fits ? launch_wave_resident(pl, form, in, out, pl.s[0], pl.s[1], &res, st,
                                               &refused)
                        : FFPAT_EINVAL;
    // a cooperative launch turned down for lack of room falls back to the
    // step-by-step loop below unless the resident loop was asked for
    if (fits && rc != FFPAT_OK && !(refused && path == 0)) return rc;
    if (fits && rc == FFPAT_OK) {
      if (result) *result = res;
      if (prof) {
        CK(cudaEventRecord(rec.b, st));
        rec.steps = pl.nt;
        rec.launches = 1;
        rec.bytes = (double)pl.nt * bytes_per_point(pl) * (double)pl.n3;
        std::lock_guard<std::mutex> g(g_prof_mu);
        g_prof.push_back(rec);
      }
      return FFPAT_OK;
    }
  }
  int dev = 0;
  CK(cudaGetDevice(&dev));
  bool done = false, replay_only = false;
  if (graphs_enabled() && g_no_graphs == 0 && cap == cudaStreamCaptureStatusNone && pl.nt >= 8) {
    std::vector<const void*> key = {in, out, pl.kap, pl.s[0], pl.s[1], pl.s[2], pl.s[3],
                                    pl.s[4], pl.s[5], (const void*)(intptr_t)pl.nt,
                                    (const void*)(intptr_t)pl.prec,
                                    (const void*)(intptr_t)g_stencil_path.load(),
                                    (const void*)(intptr_t)pl.n, (const void*)(intptr_t)dev};
    std::unique_lock<std::mutex> lk(g_graph_mu);
    int hit = -1;
    for (int i = (int)g_graphs.size() - 1; i >= 0; --i)
      if (g_graphs[i].key == key) {
        hit = i;
        break;
      }
    if (hit >= 0) {
      GraphEntry e = g_graphs[hit];
      g_graphs.erase(g_graphs.begin() + hit);
      replay_only = e.exec != nullptr;
      if (!e.exec) {
        // second use: capture the sequence and keep the executable graph
        static thread_local cudaStream_t cs = nullptr;
        if (!cs) CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        const int rc = wave_sequence(pl, in, out, &e.result, &e.launches, &e.pairs, cs);
        cudaGraph_t graph = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(cs, &graph);
        if (rc != FFPAT_OK) return rc;
        if (ec != cudaSuccess) return fail(FFPAT_ECUDA, "graph capture: %s", cudaGetErrorString(ec));
        const cudaError_t ei = cudaGraphInstantiate(&e.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) return fail(FFPAT_ECUDA, "graph instantiate: %s", cudaGetErrorString(ei));
        e.device = dev;
      }
      CK(cudaGraphLaunch(e.exec, st));
      res = e.result;
      launches = e.launches;
      pairs = e.pairs;
      g_graphs.push_back(e);
      done = true;
    } else {
      GraphEntry e;
      e.key = key;
      g_graphs.push_back(e);
      if (g_graphs.size() > kMaxGraphs) {
        if (g_graphs.front().exec) cudaGraphExecDestroy(g_graphs.front().exec);
        g_graphs.erase(g_graphs.begin());
      }
    }
  }
  if (!done) TRY(wave_sequence(pl, in, out, &res, &launches, &pairs, st));
  if (replay_only) count_launch((int)launches);  // the graph's kernels run again
  if (result) *result = res;
  if (prof) {
    CK(cudaEventRecord(rec.b, st));
    rec.steps = pl.nt;
    rec.launches = launches;
    rec.bytes = ((double)launches * bytes_per_point(pl) + (double)pairs * pass_extra_bytes(pl)) *
                (double)pl.n3;
    std::lock_guard<std::mutex> g(g_prof_mu);
    g_prof.push_back(rec);
  }
  return FFPAT_OK;
}


// W E v: the wave-grid field at T of the box source v, left in a state
// buffer returned through *pN (pad = 0: W v).
static int wave_fwd(const Plan& pl, const void* v, const void** pN, cudaStream_t st) {
  if (pl.pad == 0) return run_wave(pl, v, nullptr, pN, st);
  TRY(launch_embed(pl, v, pl.xw, st));
  return run_wave(wave_plan(pl), pl.xw, nullptr, pN, st);
}

// The wave-grid input buffer of wave_back (pl.x without padding).
static void* wave_in(const Plan& pl) { return pl.pad ? pl.xw : pl.x; }

// E^T W x for a wave-grid x (already scaled by kappa: W^T = K^-1 W K), the
// box result returned through *w (a state buffer, or pl.xo when padded).
static int wave_back(const Plan& pl, const void* x, const void** w, cudaStream_t st) {
  if (pl.pad == 0) return run_wave(pl, x, nullptr, w, st);
  const void* r = nullptr;
  TRY(run_wave(wave_plan(pl), x, nullptr, &r, st));
  TRY(launch_restrict(pl, r, pl.xo, st));
  *w = pl.xo;
  return FFPAT_OK;
}

// h = E^T W^T P^T g  ->  x = K P^T g ; w = E^T W x ; h = w / K
static int apply_adjoint(const Plan& pl, const void* g, void* h, cudaStream_t st) {
  const Plan wp = wave_plan(pl);
  TRY(launch_backproject(wp, g, wave_in(pl), wp.kap, st));
  const void* w = nullptr;
  TRY(wave_back(pl, wave_in(pl), &w, st));
  TRY(launch_kscale(pl, w, h, false, st));
  return FFPAT_OK;
}

// x-domain result of A^T chi Lambda chi (A v - g) without the final 1/kap:
// returns the buffer holding E^T W K P^T chi Lambda r, r = chi (A v - g)
// (chi = the data mask, nullable).  dots[0] = <Lambda r, r>, dots[1] = <r, r>.
static int data_gradient(const Plan& pl, const void* v, const void* g, const void** w,
                         double* dots, cudaStream_t st, const void* mask = nullptr) {
  const Plan wp = wave_plan(pl);
  const void* pN = nullptr;
  TRY(wave_fwd(pl, v, &pN, st));
  {
    Trace trace_data("P, residual, Lambda, P^T");
    TRY(launch_project(wp, pN, pl.r, g, st, mask, wave_in(pl)));
    const void* lr = pl.r;
    if (pl.precond == FFPAT_PRECOND_RAMP) {
      TRY(launch_ramp(wp, pl.r, pl.r2, st, mask));
      lr = pl.r2;
    }
    if (dots) TRY(launch_dot(pl, pl.nd, lr, pl.r, dots, st));
    TRY(launch_backproject(wp, lr, wave_in(pl), wp.kap, st));
  }
  TRY(wave_back(pl, wave_in(pl), w, st));
  return FFPAT_OK;
}

// power iteration on A^T chi Lambda chi A, vector in pl.v; returns the estimate
static int power_iteration(const Plan& pl, int iters, double* est, cudaStream_t st,
                           const void* mask = nullptr) {
  double* sq = pl.scal + 8;
  TRY(launch_dot(pl, pl.n3, pl.v, pl.v, sq, st));
  TRY(launch_scale_dev(pl, pl.n3, pl.v, pl.v, sq, st));
  for (int it = 0; it < iters; ++it) {
    const void* w = nullptr;
    TRY(data_gradient(pl, pl.v, nullptr, &w, nullptr, st, mask));
    TRY(launch_kscale(pl, w, pl.v, false, st));
    TRY(launch_dot(pl, pl.n3, pl.v, pl.v, sq, st));
    TRY(launch_scale_dev(pl, pl.n3, pl.v, pl.v, sq, st));
  }
  double h;
  CK(cudaMemcpyAsync(&h, sq, sizeof h, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  *est = sqrt(h);
  return FFPAT_OK;
}

// validate the regulariser choice; the gradient one needs the DCT tables
static int check_regulariser(const Plan& pl, int32_t reg, const void* support, cudaStream_t st) {
  if (reg != FFPAT_REG_L1_POS && reg != FFPAT_REG_GRAD2)
    return fail(FFPAT_EINVAL, "unknown regulariser %d", reg);
  if (reg == FFPAT_REG_GRAD2) {
    if (support) return fail(FFPAT_EINVAL, "the gradient regulariser takes no support mask");
    TRY(upload_dct(pl, st));
  }
  return FFPAT_OK;
}

// h <- prox_{s lambda R}(h - s w / kap), R = 1/2 |grad h|^2, with the
// statistics rows at dst (R(h), ||h||^2, ||h+ - h||^2, ||h+||^2)
static int prox_grad_step(const Plan& pl, void* h, const void* w, double step, double lambda,
                          double* dst, cudaStream_t st) {
  TRY(launch_prox_prep(pl, h, w, step, pl.x, st));
  TRY(launch_prox_grad(pl, step * lambda / (pl.dx * pl.dx), pl.x, pl.x, pl.s[0], pl.s[1], st));
  TRY(launch_prox_finish(pl, h, pl.x, dst, st));
  return FFPAT_OK;
}

// After k FB iterations: one device-to-host read of the per-iteration rows
// (8 doubles: <Lambda r, r>, <r, r>, R(h_k), ||h_k||^2, ||h_{k+1} - h_k||^2,
// ||h_{k+1}||^2, ...) into the caller's history (4 per iteration: objective,
// residual norm, relative change, ||h_{k+1}||) and summary.  Synchronises.
static int report_fb(const Plan& pl, int k, double lambda, double step, double opn,
                     ffpat_fb_stats* stats, double* history, cudaStream_t st) {
  std::vector<double> hh(8 * (size_t)(k > 0 ? k : 1), 0.0);
  if (k > 0) CK(cudaMemcpyAsync(hh.data(), pl.hist, 8 * sizeof(double) * k, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  for (int i = 0; i < k && history; ++i) {
    const double* q = &hh[8 * (size_t)i];
    history[4 * i + 0] = 0.5 * q[0] + lambda * q[2];
    history[4 * i + 1] = sqrt(q[1]);
    history[4 * i + 2] = sqrt(q[4]) / fmax(sqrt(q[3]), 1e-300);
    history[4 * i + 3] = sqrt(q[5]);
  }
  if (stats) {
    memset(stats, 0, sizeof *stats);
    stats->iters_done = k;
    stats->step = step;
    stats->opnorm_sq = opn;
    if (k > 0) {
      const double* q = &hh[8 * (size_t)(k - 1)];
      stats->objective = 0.5 * q[0] + lambda * q[2];
      stats->resid_norm = sqrt(q[1]);
      stats->rel_change = sqrt(q[4]) / fmax(sqrt(q[3]), 1e-300);
    }
  }
  return FFPAT_OK;
}

}  // namespace ffpat

using namespace ffpat;

extern "C" {

const char* ffpat_last_error(void) { return g_err; }

const char* ffpat_version(void) { return "ffpat 0.1 (sm_103a)"; }

size_t ffpat_workspace_bytes(const ffpat_problem* problem) {
  Plan pl;
  if (validate(problem, pl) != FFPAT_OK) return 0;
  return carve(pl, nullptr);
}

int ffpat_problem_info(const ffpat_problem* problem, double c_max, int32_t* nt, double* dt,
                       int32_t* n_samples) {
  Plan pl;
  g_err[0] = 0;
  TRY(validate(problem, pl));
  if (!(c_max > 0.0) || !isfinite(c_max)) return fail(FFPAT_EINVAL, "c_max must be finite and > 0");
  int n_t;
  double d_t;
  TRY(time_steps(pl, c_max, &n_t, &d_t));
  if (nt) *nt = n_t;
  if (dt) *dt = d_t;
  if (n_samples) *n_samples = pl.ns;
  return FFPAT_OK;
}

int ffpat_debug_tables(const ffpat_problem* problem, double* cos_sin) {
  Plan pl;
  g_err[0] = 0;
  TRY(validate(problem, pl));
  if (!cos_sin) return fail(FFPAT_EINVAL, "cos_sin is NULL");
  std::vector<double> t;
  host_angles(pl.nth, t);
  for (int j = 0; j < pl.nth; ++j) {
    cos_sin[2 * j] = t[j];
    cos_sin[2 * j + 1] = t[pl.nth + j];
  }
  return FFPAT_OK;
}

int ffpat_debug_samples(const ffpat_problem* problem, int32_t count, const int32_t* jkm,
                        int32_t* ij, double* f, void* stream) {
  Plan pl;
  g_err[0] = 0;
  TRY(validate(problem, pl));
  if (count < 0 || (count > 0 && (!jkm || !ij || !f)))
    return fail(FFPAT_EINVAL, "bad sample list");
  cudaStream_t st = (cudaStream_t)stream;
  void* tabs = nullptr;
  CK(cudaMallocAsync(&tabs, table_bytes(pl.nth), st));
  int rc = upload_tables(pl, tabs, st);
  if (rc == FFPAT_OK) rc = launch_debug_samples(wave_plan(pl), count, jkm, ij, f, st);
  CK(cudaFreeAsync(tabs, st));
  TRY(rc);
  CK(cudaStreamSynchronize(st));
  return FFPAT_OK;
}

int ffpat_forward(const ffpat_problem* problem, const void* c, const void* h, void* g, void* ws,
                  size_t ws_bytes, void* stream) {
  Trace trace_("ffpat_forward");
  cudaStream_t st = (cudaStream_t)stream;
  Plan pl;
  TRY(setup(problem, pl, c, ws, ws_bytes, st));
  if (!h || !g) return fail(FFPAT_EINVAL, "h or g is NULL");
  const void* pN = nullptr;
  TRY(wave_fwd(pl, h, &pN, st));
  TRY(launch_project(wave_plan(pl), pN, g, nullptr, st, nullptr, wave_in(pl)));
  return FFPAT_OK;
}

int ffpat_adjoint(const ffpat_problem* problem, const void* c, const void* g, void* h, void* ws,
                  size_t ws_bytes, void* stream) {
  Trace trace_("ffpat_adjoint");
  cudaStream_t st = (cudaStream_t)stream;
  Plan pl;
  TRY(setup(problem, pl, c, ws, ws_bytes, st));
  if (!h || !g) return fail(FFPAT_EINVAL, "h or g is NULL");
  TRY(apply_adjoint(pl, g, h, st));
  return FFPAT_OK;
}

int ffpat_wave(const ffpat_problem* problem, const void* c, const void* in, void* out,
               int32_t transpose, void* ws, size_t ws_bytes, void* stream) {
  Trace trace_("ffpat_wave");
  cudaStream_t st = (cudaStream_t)stream;
  Plan pl;
  TRY(setup(problem, pl, c, ws, ws_bytes, st));
  if (!in || !out) return fail(FFPAT_EINVAL, "in or out is NULL");
  if (!transpose) {
    if (pl.pad == 0) {
      // out may overlap in: then the loop ends in a state buffer and is
      // copied out (a step must not write the array it reads)
      const size_t bytes = pl.n3 * pl.esize;
      const char *a = (const char*)in, *b = (const char*)out;
      if (a < b + bytes && b < a + bytes) {
        const void* w = nullptr;
        TRY(run_wave(pl, in, nullptr, &w, st));
        CK(cudaMemcpyAsync(out, w, bytes, cudaMemcpyDeviceToDevice, st));
      } else {
        TRY(run_wave(pl, in, out, nullptr, st));
      }
    } else {
      TRY(launch_embed(pl, in, pl.xw, st));
      TRY(run_wave(wave_plan(pl), pl.xw, out, nullptr, st));
    }
  } else {
    TRY(launch_kscale(wave_plan(pl), in, wave_in(pl), true, st));
    const void* w = nullptr;
    TRY(wave_back(pl, wave_in(pl), &w, st));
    TRY(launch_kscale(pl, w, out, false, st));
  }
  return FFPAT_OK;
}

int ffpat_project(const ffpat_problem* problem, const void* p, void* g, void* stream) {
  Trace trace_("ffpat_project");
  cudaStream_t st = (cudaStream_t)stream;
  Plan pl;
  g_err[0] = 0;
  TRY(validate(problem, pl));
  if (!p || !g) return fail(FFPAT_EINVAL, "p or g is NULL");
  void* tabs = nullptr;
  void* tr = nullptr;
  const size_t trb = project_scratch_bytes(wave_plan(pl));
  CK(cudaMallocAsync(&tabs, table_bytes(pl.nth), st));
  if (trb) CK(cudaMallocAsync(&tr, trb, st));
  int rc = upload_tables(pl, tabs, st);
  if (rc == FFPAT_OK) rc = launch_project(wave_plan(pl), p, g, nullptr, st, nullptr, tr);
  if (tr) CK(cudaFreeAsync(tr, st));
  CK(cudaFreeAsync(tabs, st));
  TRY(rc);
  CK(cudaStreamSynchronize(st));
  return FFPAT_OK;
}

int ffpat_backproject(const ffpat_problem* problem, const void* g, void* h, void* stream) {
  Trace trace_("ffpat_backproject");
  cudaStream_t st = (cudaStream_t)stream;
  Plan pl;
  g_err[0] = 0;
  TRY(validate(problem, pl));
  if (!h || !g) return fail(FFPAT_EINVAL, "g or h is NULL");
  void* tabs = nullptr;
  CK(cudaMallocAsync(&tabs, table_bytes(pl.nth), st));
  int rc = upload_tables(pl, tabs, st);
  if (rc == FFPAT_OK) rc = launch_backproject(wave_plan(pl), g, h, nullptr, st);
  CK(cudaFreeAsync(tabs, st));
  TRY(rc);
  CK(cudaStreamSynchronize(st));
  return FFPAT_OK;
}

int ffpat_ramp(const ffpat_problem* problem, const void* r, void* out, void* stream) {
  Trace trace_("ffpat_ramp");
  cudaStream_t st = (cudaStream_t)stream;
  Plan pl;
  g_err[0] = 0;
  TRY(validate(problem, pl));
  if (!r || !out) return fail(FFPAT_EINVAL, "r or out is NULL");
  if (r == out) return fail(FFPAT_EINVAL, "ramp cannot run in place");
  TRY(launch_ramp(wave_plan(pl), r, out, st));
  return FFPAT_OK;
}

int ffpat_prox_grad(const ffpat_problem* problem, double a, const void* f, void* out, void* ws,
                    size_t ws_bytes, void* stream) {
  Trace trace_("ffpat_prox_grad");
  cudaStream_t st = (cudaStream_t)stream;
  Plan pl;
  g_err[0] = 0;
  TRY(attach(problem, pl, ws, ws_bytes));
  if (!f || !out) return fail(FFPAT_EINVAL, "f or out is NULL");
  if (!(a >= 0.0) || !isfinite(a)) return fail(FFPAT_EINVAL, "a = %g must be finite and >= 0", a);
  TRY(upload_dct(pl, st));
  TRY(launch_prox_grad(pl, a, f, out, pl.s[0], pl.s[1], st));
  return FFPAT_OK;
}

int ffpat_opnorm(const ffpat_problem* problem, const void* c, const void* v0, int32_t iters,
                 double* opnorm_sq, void* ws, size_t ws_bytes, void* stream) {
  Trace trace_("ffpat_opnorm");
  cudaStream_t st = (cudaStream_t)stream;
  Plan pl;
  TRY(setup(problem, pl, c, ws, ws_bytes, st));
  if (!v0 || !opnorm_sq || iters < 1) return fail(FFPAT_EINVAL, "bad power-iteration arguments");
  CK(cudaMemcpyAsync(pl.v, v0, pl.n3 * pl.esize, cudaMemcpyDeviceToDevice, st));
  TRY(power_iteration(pl, iters, opnorm_sq, st));
  return FFPAT_OK;
}

int ffpat_fb_solve(const ffpat_problem* problem, const void* c, const void* g, double lambda,
                   double step, int32_t max_iters, double tol, void* h_inout,
                   ffpat_fb_stats* stats, double* history, void* ws, size_t ws_bytes,
                   void* stream) {
  return ffpat_fb_solve_ex(problem, c, g, nullptr, nullptr, FFPAT_REG_L1_POS, lambda, step,
                           max_iters, tol, h_inout, stats, history, ws, ws_bytes, stream);
}

int ffpat_fb_solve_ex(const ffpat_problem* problem, const void* c, const void* g,
                      const void* mask, const void* support, int32_t regulariser, double lambda,
                      double step, int32_t max_iters, double tol, void* h_inout,
                      ffpat_fb_stats* stats, double* history, void* ws, size_t ws_bytes,
                      void* stream) {
  Trace trace_("ffpat_fb_solve");
  cudaStream_t st = (cudaStream_t)stream;
  Plan pl;
  TRY(setup(problem, pl, c, ws, ws_bytes, st));
  if (!g || !h_inout) return fail(FFPAT_EINVAL, "g or h is NULL");
  TRY(check_regulariser(pl, regulariser, support, st));
  if (max_iters < 0 || max_iters > kMaxHist)
    return fail(FFPAT_EINVAL, "max_iters = %d outside [0, %d]", max_iters, kMaxHist);
  if (!(lambda >= 0.0) || !isfinite(lambda)) return fail(FFPAT_EINVAL, "lambda must be >= 0");
  if (!(tol >= 0.0)) return fail(FFPAT_EINVAL, "tol must be >= 0");
  double opn = 0.0;
  if (!(step > 0.0)) {
    TRY(launch_hash_fill(pl, pl.v, 0x5eed1901ull, st));
    TRY(power_iteration(pl, 20, &opn, st, mask));
    if (!(opn > 0.0) || !isfinite(opn)) return fail(FFPAT_EINVAL, "operator norm estimate %g", opn);
    step = 1.0 / opn;
  }
  if (!isfinite(step)) return fail(FFPAT_EINVAL, "step is not finite");
  int k = 0;
  for (; k < max_iters; ++k) {
    Trace trace_it("FB iteration (Algorithm 8)");
    double* hk = pl.hist + 8 * (size_t)k;
    const void* w = nullptr;
    TRY(data_gradient(pl, h_inout, g, &w, hk, st, mask));
    if (regulariser == FFPAT_REG_GRAD2)
      TRY(prox_grad_step(pl, h_inout, w, step, lambda, hk + 2, st));
    else
      TRY(launch_fb_update(pl, h_inout, w, step, lambda, hk + 2, st, nullptr, support));
    if (tol > 0.0) {
      double q[4];
      CK(cudaMemcpyAsync(q, hk + 2, sizeof q, cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      const double rel = sqrt(q[2]) / fmax(sqrt(q[1]), 1e-300);
      if (rel < tol) {
        ++k;
        break;
      }
    }
  }
  return report_fb(pl, k, lambda, step, opn, stats, history, st);
}

int ffpat_fbp(const ffpat_problem* problem, const void* G, void* out, void* ws, size_t ws_bytes,
              void* stream) {
  Trace trace_("ffpat_fbp");
  cudaStream_t st = (cudaStream_t)stream;
  Plan pl;
  g_err[0] = 0;
  TRY(attach(problem, pl, ws, ws_bytes));
  if (!G || !out) return fail(FFPAT_EINVAL, "G or out is NULL");
  TRY(upload_tables(pl, pl.tab, st));
  const Plan wp = wave_plan(pl);
  TRY(launch_ramp(wp, G, pl.r2, st));
  TRY(launch_backproject(wp, pl.r2, out, nullptr, st, 2.0 * M_PI / (pl.nth * pl.dx)));
  return FFPAT_OK;
}

// power iteration on W^T W (vector in pl.v); W^T = K^-1 W K
static int power_iteration_w(const Plan& pl, int iters, double* est, cudaStream_t st) {
  double* sq = pl.scal + 8;
  TRY(launch_dot(pl, pl.n3, pl.v, pl.v, sq, st));
  TRY(launch_scale_dev(pl, pl.n3, pl.v, pl.v, sq, st));
  for (int it = 0; it < iters; ++it) {
    const void* w = nullptr;
    TRY(wave_fwd(pl, pl.v, &w, st));
    TRY(launch_kscale(wave_plan(pl), w, wave_in(pl), true, st));
    TRY(wave_back(pl, wave_in(pl), &w, st));
    TRY(launch_kscale(pl, w, pl.v, false, st));
    TRY(launch_dot(pl, pl.n3, pl.v, pl.v, sq, st));
    TRY(launch_scale_dev(pl, pl.n3, pl.v, pl.v, sq, st));
  }
  double h;
  CK(cudaMemcpyAsync(&h, sq, sizeof h, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  *est = sqrt(h);
  return FFPAT_OK;
}

int ffpat_fb_two_step(const ffpat_problem* problem, const void* c, const void* G, double lambda,
                      double step, int32_t max_iters, double tol, void* h_inout,
                      ffpat_fb_stats* stats, double* history, void* ws, size_t ws_bytes,
                      void* stream) {
  return ffpat_fb_two_step_ex(problem, c, G, FFPAT_REG_L1_POS, lambda, step, max_iters, tol,
                              h_inout, stats, history, ws, ws_bytes, stream);
}

int ffpat_fb_two_step_ex(const ffpat_problem* problem, const void* c, const void* G,
                         int32_t regulariser, double lambda, double step, int32_t max_iters,
                         double tol, void* h_inout, ffpat_fb_stats* stats, double* history,
                         void* ws, size_t ws_bytes, void* stream) {
  Trace trace_("ffpat_fb_two_step");
  cudaStream_t st = (cudaStream_t)stream;
  Plan pl;
  TRY(setup(problem, pl, c, ws, ws_bytes, st));
  if (!G || !h_inout) return fail(FFPAT_EINVAL, "G or h is NULL");
  TRY(check_regulariser(pl, regulariser, nullptr, st));
  if (max_iters < 0 || max_iters > kMaxHist)
    return fail(FFPAT_EINVAL, "max_iters = %d outside [0, %d]", max_iters, kMaxHist);
  if (!(lambda >= 0.0) || !isfinite(lambda)) return fail(FFPAT_EINVAL, "lambda must be >= 0");
  if (!(tol >= 0.0)) return fail(FFPAT_EINVAL, "tol must be >= 0");
  double opn = 0.0;
  if (!(step > 0.0)) {
    TRY(launch_hash_fill(pl, pl.v, 0x5eed1901ull, st));
    TRY(power_iteration_w(pl, 20, &opn, st));
    if (!(opn > 0.0) || !isfinite(opn)) return fail(FFPAT_EINVAL, "operator norm estimate %g", opn);
    step = 1.0 / opn;
  }
  // g~ = X^{-1} G on the wave grid, kept for the whole solve (pl.v, or pl.xg
  // when padded)
  const Plan wp = wave_plan(pl);
  void* gt = pl.pad ? pl.xg : pl.v;
  TRY(launch_ramp(wp, G, pl.r2, st));
  TRY(launch_backproject(wp, pl.r2, gt, nullptr, st, 2.0 * M_PI / (pl.nth * pl.dx)));
  int k = 0;
  for (; k < max_iters; ++k) {
    Trace trace_it("FB iteration (Algorithm 9)");
    double* hk = pl.hist + 8 * (size_t)k;
    const void* w = nullptr;
    TRY(wave_fwd(pl, h_inout, &w, st));
    TRY(launch_resid_kap(wp, w, gt, wave_in(pl), hk, st));
    TRY(wave_back(pl, wave_in(pl), &w, st));
    if (regulariser == FFPAT_REG_GRAD2)
      TRY(prox_grad_step(pl, h_inout, w, step, lambda, hk + 2, st));
    else
      TRY(launch_fb_update(pl, h_inout, w, step, lambda, hk + 2, st));
    if (tol > 0.0) {
      double q[4];
      CK(cudaMemcpyAsync(q, hk + 2, sizeof q, cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      if (sqrt(q[2]) / fmax(sqrt(q[1]), 1e-300) < tol) {
        ++k;
        break;
      }
    }
  }
  return report_fb(pl, k, lambda, step, opn, stats, history, st);
}

int ffpat_profile_enable(int32_t on) {
  g_prof_on = on ? 1 : 0;
  return FFPAT_OK;
}

int ffpat_profile_read(ffpat_profile* out) {
  g_err[0] = 0;
  if (!out) return fail(FFPAT_EINVAL, "out is NULL");
  std::vector<ProfRec> recs;
  {
    std::lock_guard<std::mutex> g(g_prof_mu);
    recs.swap(g_prof);
  }
  memset(out, 0, sizeof *out);
  int rc = FFPAT_OK;
  for (auto& r : recs) {
    float ms = 0.f;
    if (rc == FFPAT_OK) {
      cudaError_t e = cudaEventSynchronize(r.b);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.a, r.b);
      if (e != cudaSuccess) rc = fail(FFPAT_ECUDA, "profile events: %s", cudaGetErrorString(e));
    }
    out->step_launches += r.launches;
    out->steps += r.steps;
    out->step_ms += ms;
    out->step_bytes += r.bytes;
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  out->kernel_launches = g_prof_launches.exchange(0);
  return rc;
}

int64_t ffpat_launch_count(void) { return g_launches.load(); }

int ffpat_set_stencil_path(int32_t path) {
  g_err[0] = 0;
  if (path < 0 || path > 4) return fail(FFPAT_EINVAL, "stencil path %d not in {0, ..., 4}", path);
  g_stencil_path = path;
  return FFPAT_OK;
}

int ffpat_debug_wait_timeout(int32_t microseconds, void* stream) {
  g_err[0] = 0;
  if (microseconds < 1 || microseconds > 2000000)
    return fail(FFPAT_EINVAL, "timeout %d us outside [1, 2e6]", microseconds);
  int khz = 0, dev = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev) != cudaSuccess || khz <= 0) khz = 2070000;
  TRY(launch_wait_timeout((long long)microseconds * (khz / 1000), (cudaStream_t)stream));
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  return FFPAT_OK;
}

int ffpat_device_status(int32_t clear) {
  g_err[0] = 0;
  unsigned v = 0;
  TRY(read_device_status(&v, clear != 0));
  if (v) fail(-(int)v, "a device-side wait timed out in an earlier launch");
  return -(int)v;
}

}  // extern "C"
