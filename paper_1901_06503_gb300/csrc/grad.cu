// grad.cu -- the differentiated forward operator: g = P W(c) h with
// wavefield checkpoints, and the backward pass giving grad_h = A^T grad_g and
// grad_c = d<grad_g, A(c) h>/dc (dt held fixed: Nt is piecewise constant in c).
//
// Forward: the three-term leapfrog of the wave model (Sec. 2.1) saves the
// pair (p^{sk}, p^{sk+1}) every k steps.  Backward: the transposed recurrence
// runs from lambda^{Nt} = P^T grad_g down to lambda^0 = grad_h; written for
// mu = (kappa/12) lambda it is the forward three-term step again
// (mu^n = 2 mu^{n+1} - mu^{n+2} + kappa L mu^{n+1}).  Segment by segment, from
// the last, the states p^n of the segment are recomputed from its checkpoint
// and the kappa-derivatives mu^{n+1} L(p^n) (weight 1/2 for the start step)
// are accumulated; grad_c = 2 acc / c because dkappa/dc = 2 kappa / c and the
// factors kappa/12 and 12 cancel.  Memory: 2 ceil(Nt/k) + k + 2 volumes.
#include "internal.cuh"

namespace ffpat {
namespace {

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Ckpt {
  size_t vol = 0;
  int nseg = 0, every = 0;
  unsigned char* base = nullptr;
  void* a(int s) const { return base + (size_t)(2 * s) * vol; }
  void* b(int s) const { return base + (size_t)(2 * s + 1) * vol; }
  void* seg(int j) const { return base + (size_t)(2 * nseg + j) * vol; }  // j = 0 .. every
  void* acc() const { return base + (size_t)(2 * nseg + every + 1) * vol; }
  size_t bytes() const { return (size_t)(2 * nseg + every + 2) * vol; }
};

int ckpt_layout(const Plan& pl, int nt, int every, void* base, Ckpt* ck) {
  if (pl.pad != 0) return report(FFPAT_EINVAL, "the differentiated operator needs pad = 0");
  if (every < 1 || every > 4096) return report(FFPAT_EINVAL, "checkpoint interval %d", every);
  ck->vol = up256(pl.n3 * pl.esize);
  ck->every = every;
  ck->nseg = (nt + every - 1) / every;
  ck->base = (unsigned char*)base;
  return FFPAT_OK;
}

// the three-term stepper runs this path for every precision (FP32-Kahan
// problems take FP32 three-term steps: the same discrete operator)
void as_three_term(Plan& pl) {
  if (pl.prec == FFPAT_FP32_KAHAN) pl.prec = FFPAT_FP32;
}

bool use_tma(const Plan& pl, const Ckpt& ck, const void* a, const void* b) {
  const void* ptrs[9] = {a, b, pl.kap, pl.s[0], pl.s[1], pl.s[2], pl.s[3], pl.x, ck.base};
  return tma_supported(pl, ptrs, 9) && (ck.vol % 16) == 0;
}

// two steps per pass in the checkpointed loops: W's rule, and checkpoints at
// even steps (the passes advance the pair (p^m, p^{m+1}) by two)
bool use_two(const Plan& pl, const Ckpt& ck, bool tma) {
  return two_step_three_term(pl, tma) && ck.every % 2 == 0 && pl.s[2] && pl.s[3];
}

}  // namespace
}  // namespace ffpat

using namespace ffpat;

extern "C" {

size_t ffpat_ckpt_bytes(const ffpat_problem* problem, int32_t nt, int32_t every) {
  Plan pl;
  if (ffpat_workspace_bytes(problem) == 0 || nt < 1) return 0;
  if (attach(problem, pl, (void*)256, ffpat_workspace_bytes(problem)) != FFPAT_OK) return 0;
  Ckpt ck;
  if (ckpt_layout(pl, nt, every, nullptr, &ck) != FFPAT_OK) return 0;
  return ck.bytes();
}

int ffpat_forward_ckpt(const ffpat_problem* problem, const void* c, const void* h, void* g,
                       int32_t every, void* ckpt, size_t ckpt_bytes, void* ws, size_t ws_bytes,
                       void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  Plan pl;
  const int rc0 = setup(problem, pl, c, ws, ws_bytes, st);
  if (rc0 != FFPAT_OK) return rc0;
  if (!h || !g || !ckpt) return report(FFPAT_EINVAL, "h, g or ckpt is NULL");
  as_three_term(pl);
  Ckpt ck;
  if (ckpt_layout(pl, pl.nt, every, ckpt, &ck) != FFPAT_OK) return FFPAT_EINVAL;
  if (ckpt_bytes < ck.bytes())
    return report(FFPAT_ENOMEM, "checkpoint buffer %zu < %zu bytes", ckpt_bytes, ck.bytes());
  const bool tma = use_tma(pl, ck, h, g);
  const bool two = use_two(pl, ck, tma);
  // S[a] = p^m, S[b] = p^{m+1}; a two-step pass writes the other pair
  void* S[4] = {pl.s[0], pl.s[1], pl.s[2], pl.s[3]};
  int a = 0, b = 1;
  int rc = step3(pl, tma, true, h, nullptr, S[b], S[a], st);  // p^0, p^1
  if (rc != FFPAT_OK) return rc;
  const size_t vb = pl.n3 * pl.esize;
  if (cudaMemcpyAsync(ck.a(0), S[a], vb, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(ck.b(0), S[b], vb, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return check_launch("checkpoint copy");
  for (int m = 0; m + 1 < pl.nt;) {
    if (two && m + 3 <= pl.nt) {
      rc = launch_step2_f32(pl, S[a], S[b], S[a ^ 2], S[b ^ 2], st);  // p^{m+2}, p^{m+3}
      a ^= 2;
      b ^= 2;
      m += 2;
    } else {
      rc = step3(pl, tma, false, S[b], S[a], S[a], nullptr, st);  // p^{m+2} over p^m
      const int t = a;
      a = b;
      b = t;
      m += 1;
    }
    if (rc != FFPAT_OK) return rc;
    if (m % every == 0) {
      const int s = m / every;
      if (cudaMemcpyAsync(ck.a(s), S[a], vb, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
          cudaMemcpyAsync(ck.b(s), S[b], vb, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return check_launch("checkpoint copy");
    }
  }
  return launch_project(pl, S[b], g, nullptr, st, nullptr, pl.x);
}

int ffpat_backward(const ffpat_problem* problem, const void* c, const void* grad_g, void* grad_h,
                   void* grad_c, int32_t every, void* ckpt, size_t ckpt_bytes, void* ws,
                   size_t ws_bytes, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  Plan pl;
  const int rc0 = setup(problem, pl, c, ws, ws_bytes, st);
  if (rc0 != FFPAT_OK) return rc0;
  if (!grad_g || !ckpt) return report(FFPAT_EINVAL, "grad_g or ckpt is NULL");
  as_three_term(pl);
  Ckpt ck;
  if (ckpt_layout(pl, pl.nt, every, ckpt, &ck) != FFPAT_OK) return FFPAT_EINVAL;
  if (ckpt_bytes < ck.bytes())
    return report(FFPAT_ENOMEM, "checkpoint buffer %zu < %zu bytes", ckpt_bytes, ck.bytes());
  const bool tma = use_tma(pl, ck, grad_h, c);
  const bool two = use_two(pl, ck, tma);
  const size_t vb = pl.n3 * pl.esize;
  // mu^{Nt} = (kappa / 12) P^T grad_g, mu^{Nt+1} = 0
  // B[u] = mu^{n+1}, B[v] = mu^{n+2}; a two-step pass writes mu^n, mu^{n-1}
  // into the other two buffers
  void* B[4] = {pl.x, pl.s[0], pl.s[1], pl.s[2]};
  const bool two_t = two_step_three_term(pl, tma) && pl.s[1] && pl.s[2];
  int u = 0, v = 1;
  int rc = launch_backproject(pl, grad_g, B[u], pl.kap, st);
  if (rc != FFPAT_OK) return rc;
  if (cudaMemsetAsync(B[v], 0, vb, st) != cudaSuccess ||
      cudaMemsetAsync(ck.acc(), 0, vb, st) != cudaSuccess)
    return check_launch("backward init");
  for (int s = ck.nseg - 1; s >= 0; --s) {
    const int lo = s * every;
    const int hi = (lo + every - 1 < pl.nt - 1) ? lo + every - 1 : pl.nt - 1;
    auto P = [&](int j) -> void* { return j == 0 ? ck.a(s) : (j == 1 ? ck.b(s) : ck.seg(j)); };
    // recompute p^{lo+2} .. p^{hi} from the checkpoint, two steps per pass
    // where allowed
    for (int j = 1; j + 1 <= hi - lo;) {
      if (two && j + 2 <= hi - lo) {
        rc = launch_step2_f32(pl, P(j - 1), P(j), P(j + 1), P(j + 2), st);
        j += 2;
      } else {
        rc = step3(pl, tma, false, P(j), P(j - 1), P(j + 1), nullptr, st);
        j += 1;
      }
      if (rc != FFPAT_OK) return rc;
    }
    for (int n = hi; n >= lo;) {
      const void* pn = P(n - lo);
      if (two_t && n - 1 >= lo && n - 1 >= 1) {
        // mu^n, mu^{n-1} in one pass; the accumulations in the order of
        // the single steps (mu^{n+1} L(p^n), then mu^n L(p^{n-1}))
        int x = 0;
        while (x == u || x == v) ++x;
        int y = x + 1;
        while (y == u || y == v) ++y;
        rc = launch_step2_f32(pl, B[v], B[u], B[x], B[y], st);
        if (rc == FFPAT_OK) rc = launch_lap_accum(pl, ck.acc(), B[u], pn, 1.0, st);
        if (rc == FFPAT_OK) rc = launch_lap_accum(pl, ck.acc(), B[x], P(n - 1 - lo), 1.0, st);
        if (rc != FFPAT_OK) return rc;
        u = y;  // mu^{n-1}
        v = x;  // mu^n
        n -= 2;
      } else if (n >= 1) {
        rc = launch_lap_accum(pl, ck.acc(), B[u], pn, 1.0, st);
        if (rc == FFPAT_OK) rc = step3(pl, tma, false, B[u], B[v], B[v], nullptr, st);  // mu^n
        if (rc != FFPAT_OK) return rc;
        const int t = u;
        u = v;
        v = t;
        n -= 1;
      } else {
        rc = launch_lap_accum(pl, ck.acc(), B[u], pn, 0.5, st);
        void* tmp = ck.seg(0);
        if (rc == FFPAT_OK) rc = step3(pl, tma, true, B[u], nullptr, tmp, nullptr, st);
        if (rc == FFPAT_OK && grad_h) rc = launch_sub_div(pl, tmp, B[v], grad_h, st);
        if (rc != FFPAT_OK) return rc;
        n -= 1;
      }
    }
  }
  if (grad_c) return launch_scale_div(pl, ck.acc(), c, 2.0, grad_c, st);
  return FFPAT_OK;
}

}  // extern "C"
