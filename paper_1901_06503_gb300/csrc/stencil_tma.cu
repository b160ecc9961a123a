// stencil_tma.cu -- the leapfrog step of p_tt = c^2 Delta p (Sec. 2.1,
// eq. (1)-(2)) as a TMA-fed, z-streaming persistent kernel for sm_103a.
//
// Same arithmetic as stencil.cu (see there for the two time-update forms);
// what changes is how the data reach the SM:
//   * every CTA owns a 64 x (8 RPT) (x, y) column tile and a z-range (RPT =
//     2 rows per thread by default: 64 x 16 tiles); a persistent grid walks
//     the (tile, z-range) work items;
//   * one thread issues cp.async.bulk.tensor (TMA) copies: the plane of p^n
//     with its two-point x/y halo (a 72 x 20 float box for 64 x 16 tiles,
//     starting 16-byte aligned at x0 - 4) into an 8-deep ring of
//     shared-memory planes, and the halo-free tiles of the per-point streams
//     (p^{n-1}, or d and e, and kap) into a 4-deep ring; an mbarrier per
//     round counts the bytes in;
//   * the ring runs three planes ahead of the plane being computed;
//   * zero ghost values outside the box come for free: TMA fills boxes that
//     cross the tensor bounds with zeros, including whole planes z < 0, z >= N;
//   * the z-neighbours z +- 1, z +- 2 are read from the neighbouring ring
//     planes, so each plane of p^n comes from HBM once per step.
// Every mbarrier wait is bounded (about a second of clock64 time); on a
// timeout the CTA records FFPAT_ETIMEDOUT in a device status word, waits a
// bounded time for its own copies in flight, and returns.
//
// Also here: the batched step of the server (k_step_batch), two steps per
// pass (k_step2_kahan, k_step2_f32: one kernel body for both forms), and, for
// grids whose work items all fit the GPU at once (N <= 128), the whole time
// loop in one cooperative launch
// (k_wave_resident: per-point state on chip, p^n through L2, neighbour step
// flags between steps).  All FP32 kernels share the packed two-lane pair
// arithmetic below, so they agree bit for bit.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <stdlib.h>
#include <string.h>

#include <mutex>
#include <unordered_map>

#include "internal.cuh"

namespace ffpat {

__device__ unsigned int g_tma_status;  // 0 = ok, else the first error code (as unsigned)

namespace {

constexpr int TBX = 64, TBY = 8;   // output tile
constexpr int NTX = 32, NTY = 8;   // threads: each computes x and x + 32
constexpr int SP = 8;              // ring of p planes: z-2 .. z+5
constexpr int SQ = 4;              // ring of per-point stream planes: z .. z+3
constexpr long long kWaitCycles = 1LL << 31;

// Tile geometry for RPT rows per thread: the output tile is TBX x (TBY RPT)
template <typename T, int RPT = 1>
struct Geo {
  static constexpr int XH = 16 / (int)sizeof(T);  // x halo rounded up to 16 bytes
  static constexpr int TH = TBY * RPT;            // tile height
  static constexpr int BXH = TBX + 2 * XH;
  static constexpr int BYH = TH + 4;
  static constexpr int PBYTES = BXH * BYH * (int)sizeof(T);
  static constexpr int QBYTES = TBX * TH * (int)sizeof(T);
};

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

// Let the dependent grid launch, then wait until the grid this one depends on
// (programmatic stream serialization) has completed with its memory visible.
// Without a programmatic dependency both return at once.
__device__ __forceinline__ void grid_dependency_sync() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// try_wait with a suspend-time hint: a thread whose phase has not completed
// is suspended (it takes no issue slots) until the phase completes or about
// `ns` nanoseconds have passed
__device__ __forceinline__ bool mbar_try_wait_ns(uint64_t* bar, unsigned parity, unsigned ns) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(ns)
      : "memory");
  return ok != 0;
}

// bounded wait: false if the phase did not complete within `cycles` (the
// latency-bound resident loop measured slower with the suspend-time hint of
// mbar_try_wait_ns, 4.86 against 4.70 us per step at 128^3, so this one polls)
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, long long cycles) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (true) {
    for (int i = 0; i < 64; ++i)
      if (mbar_try_wait(bar, parity)) return true;
    if (clock64() - t0 > cycles) return false;
  }
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

struct Maps {
  CUtensorMap p;     // p^n with the halo box
  CUtensorMap q[3];  // halo-free per-point streams
};

// FORM 0: three-term (q = {p^{n-1}, kap} or, at START, {kap});
// FORM 1: increment with Kahan carry (q = {d, e, kap} or, at START, {kap});
// FORM 2: the kappa-derivative accumulation of the differentiated operator,
//         acc += w mu L(p) with w = 1/2 at START, else 1 (q = {mu, acc}; FP32).
template <typename T, int FORM, bool START>
struct Streams {
  static constexpr int NQ = FORM == 2 ? 2 : (START ? 1 : (FORM == 0 ? 2 : 3));
};

__device__ __forceinline__ double lap12_sum(const double* P0, const double* Pm1, const double* Pp1,
                                            const double* Pm2, const double* Pp2, int o, int row) {
  const double c = P0[o];
  double s1 = P0[o - 1] + P0[o + 1];
  s1 += P0[o - row];
  s1 += P0[o + row];
  s1 += Pm1[o];
  s1 += Pp1[o];
  double s2 = fma(90.0, c, P0[o - 2]);
  s2 += P0[o + 2];
  s2 += P0[o - 2 * row];
  s2 += P0[o + 2 * row];
  s2 += Pm2[o];
  s2 += Pp2[o];
  return fma(16.0, s1, -s2);
}

// Two x-adjacent points are updated together with the packed two-lane FP32
// instructions of sm_100+ (lane x: the point at o, lane y: o + 1).  Each lane
// is exactly the IEEE single-precision operation (round to nearest even), so a
// pair computes what two scalar updates with the same operation order would;
// the packed forms halve the arithmetic instructions of a step.  They are
// written as PTX with an explicit rounding mode, which the compiler never
// contracts (a multiply followed by an add stays two roundings in every
// kernel), so all stencil kernels agree bit for bit whatever their code shape.
// bit copies between a float pair and the 64-bit register the packed
// instructions take (no instruction: the pair already is a register pair)
__device__ __forceinline__ unsigned long long pk2(float2 a) {
  unsigned long long r;
  memcpy(&r, &a, sizeof r);
  return r;
}
__device__ __forceinline__ float2 up2(unsigned long long r) {
  float2 a;
  memcpy(&a, &r, sizeof a);
  return a;
}
// a + b and a - b as one packed fused multiply-add each, a * 1 + b and
// b * (-1) + a: the exact sum rounded once, i.e. the IEEE addition and
// subtraction bit for bit (signed zeros included)
__device__ __forceinline__ float2 add2(float2 a, float2 b) {
  unsigned long long r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;"
      : "=l"(r)
      : "l"(pk2(a)), "l"(pk2(make_float2(1.0f, 1.0f))), "l"(pk2(b)));
  return up2(r);
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  unsigned long long r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;"
      : "=l"(r)
      : "l"(pk2(b)), "l"(pk2(make_float2(-1.0f, -1.0f))), "l"(pk2(a)));
  return up2(r);
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
  unsigned long long r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pk2(a)), "l"(pk2(b)));
  return up2(r);
}
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  unsigned long long r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(pk2(a)), "l"(pk2(b)), "l"(pk2(c)));
  return up2(r);
}

__device__ __forceinline__ float2 lds2(const float* p) { return *reinterpret_cast<const float2*>(p); }

// Neighbourhood of a pair of points for the FP32 difference-form Laplacian.
struct Nb2 {
  float2 c, xm1, xp1, ym1, yp1, zm1, zp1, xm2, xp2, ym2, yp2, zm2, zp2;
};

// 12 (h^2 L4 p) at both points, difference form:
// 16 sum_axes (p(-1) - c + p(+1) - c) - sum_axes (p(-2) - c + p(+2) - c).
// The far sum is accumulated negated, as (c - p(-2)) + (c - p(+2)) ..., which
// is exactly its negative (a - b = -(b - a) in IEEE arithmetic), so the last
// step is one fused 16 d1 + (-d2) without a separate negation.
__device__ __forceinline__ float2 lap12_pair(const Nb2& v) {
  float2 d1 = add2(sub2(v.xm1, v.c), sub2(v.xp1, v.c));
  d1 = add2(d1, add2(sub2(v.ym1, v.c), sub2(v.yp1, v.c)));
  d1 = add2(d1, add2(sub2(v.zm1, v.c), sub2(v.zp1, v.c)));
  float2 nd2 = add2(sub2(v.c, v.xm2), sub2(v.c, v.xp2));
  nd2 = add2(nd2, add2(sub2(v.c, v.ym2), sub2(v.c, v.yp2)));
  nd2 = add2(nd2, add2(sub2(v.c, v.zm2), sub2(v.c, v.zp2)));
  return fma2(make_float2(16.0f, 16.0f), d1, nd2);
}

// the neighbourhoods of the points at o and o + 1 (o even), read with eleven
// 64-bit shared-memory loads
__device__ __forceinline__ void gather_pair(const float* P0, const float* Pm1, const float* Pp1,
                                            const float* Pm2, const float* Pp2, int o, int row,
                                            Nb2& v) {
  const float2 C = lds2(P0 + o), XM = lds2(P0 + o - 2), XP = lds2(P0 + o + 2);
  v.c = C;
  v.xm1 = make_float2(XM.y, C.x);
  v.xp1 = make_float2(C.y, XP.x);
  v.xm2 = XM;
  v.xp2 = XP;
  v.ym1 = lds2(P0 + o - row);
  v.yp1 = lds2(P0 + o + row);
  v.ym2 = lds2(P0 + o - 2 * row);
  v.yp2 = lds2(P0 + o + 2 * row);
  v.zm1 = lds2(Pm1 + o);
  v.zp1 = lds2(Pp1 + o);
  v.zm2 = lds2(Pm2 + o);
  v.zp2 = lds2(Pp2 + o);
}

// Kahan-compensated increment update of a pair: p' = p + d' with carry e',
// d' = k L + d (start: d' = k L / 2, no carry in)
struct Kp2 {
  float2 p, d, e;
};
__device__ __forceinline__ Kp2 kahan_pair(float2 c, float2 k, float2 L, float2 dold, float2 eold,
                                          bool start) {
  const float2 dn = start ? mul2(mul2(make_float2(0.5f, 0.5f), k), L) : fma2(k, L, dold);
  const float2 yv = start ? dn : sub2(dn, eold);
  const float2 tv = add2(c, yv);
  return Kp2{tv, dn, sub2(sub2(tv, c), yv)};
}

// three-term update of a pair: p^{n+1} = p^n + (k L + (p^n - p^{n-1}));
// start: p^1 = p^0 + (k / 2) L
__device__ __forceinline__ float2 three_term_pair(float2 c, float2 k, float2 L, float2 pm) {
  return add2(c, fma2(k, L, sub2(c, pm)));
}
__device__ __forceinline__ float2 start_pair(float2 c, float2 k, float2 L) {
  return add2(c, mul2(mul2(make_float2(0.5f, 0.5f), k), L));
}

// Round R brings p plane R (needed while R <= z1 + 1) and the per-point
// stream planes R - 2 (needed while z0 <= R - 2 < z1) of the item's tile.
template <typename T, int NQ, int RPT>
__device__ __forceinline__ void issue_round(const Maps& maps, T* pst, T* qst, uint64_t* bar, int R,
                                            int z0, int z1, int x0, int y0) {
  using G = Geo<T, RPT>;
  const bool wp = R <= z1 + 1;
  const bool wq = (R - 2 >= z0) && (R - 2 < z1);
  if (!wp && !wq) return;
  uint64_t* b = &bar[R & (SP - 1)];
  mbar_expect_tx(b, (wp ? G::PBYTES : 0) + (wq ? NQ * G::QBYTES : 0));
  if (wp)
    tma_load_3d(pst + (size_t)(R & (SP - 1)) * (G::PBYTES / sizeof(T)), &maps.p, x0 - G::XH,
                y0 - 2, R, b);
  if (wq) {
    const int s = (R - 2) & (SQ - 1);
#pragma unroll
    for (int q = 0; q < NQ; ++q)
      tma_load_3d(qst + (size_t)(s * NQ + q) * (G::QBYTES / sizeof(T)), &maps.q[q], x0, y0, R - 2,
                  b);
  }
}

template <typename T, int FORM, bool START, int RPT>
__global__ void __launch_bounds__(NTX* NTY, 2)
    k_step_tma(const __grid_constant__ Maps maps, T* __restrict__ o0, T* __restrict__ o1,
               T* __restrict__ o2, int n, int zc, int tiles_x, int tiles_y, int nitems) {
  using G = Geo<T, RPT>;
  constexpr int NQ = Streams<T, FORM, START>::NQ;
  extern __shared__ unsigned char smem_raw[];
  // TMA destinations must be 128-byte aligned: align the dynamic window to 1 KB
  unsigned char* smem =
      smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  T* pst = reinterpret_cast<T*>(smem);                                   // SP planes
  T* qst = reinterpret_cast<T*>(smem + SP * G::PBYTES);                  // SQ x NQ tiles
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + SP * G::PBYTES + SQ * NQ * G::QBYTES);

  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * NTX + tx;
  if (tid == 0) {
    for (int i = 0; i < SP; ++i) mbar_init(&bar[i], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // programmatic dependent launch: the next step's grid may be scheduled as
  // this one's CTAs retire and run the prologue above; no global memory is
  // touched before the previous grid has completed and its writes are visible
  grid_dependency_sync();
  // after a device-side failure, later launches return at once (the host
  // reports the status word) instead of repeating bounded waits
  if (*(volatile unsigned*)&g_tma_status != 0u) return;
  __syncthreads();
  unsigned phase = 0;  // one parity bit per barrier slot
  const size_t plane = (size_t)n * n;

  for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
    const int tix = item % tiles_x;
    const int tiy = (item / tiles_x) % tiles_y;
    const int z0 = (item / (tiles_x * tiles_y)) * zc;
    const int z1 = min(n, z0 + zc);
    const int x0 = tix * TBX, y0 = tiy * G::TH;

    if (tid == 0)
      for (int R = z0 - 2; R <= z0 + SP - 3; ++R)
        issue_round<T, NQ, RPT>(maps, pst, qst, bar, R, z0, z1, x0, y0);

    bool timed_out = false;
    int waited_upto = z0 - 3;  // last round this thread has waited for
    for (int z = z0; z < z1; ++z) {
      for (int R = waited_upto + 1; R <= z + 2; ++R) {
        const int b = R & (SP - 1);
        if (!mbar_wait(&bar[b], (phase >> b) & 1u, kWaitCycles)) timed_out = true;
        phase ^= 1u << b;
      }
      waited_upto = z + 2;

      const T* P0 = pst + (size_t)(z & (SP - 1)) * (G::PBYTES / sizeof(T));
      const T* Pm1 = pst + (size_t)((z - 1) & (SP - 1)) * (G::PBYTES / sizeof(T));
      const T* Pp1 = pst + (size_t)((z + 1) & (SP - 1)) * (G::PBYTES / sizeof(T));
      const T* Pm2 = pst + (size_t)((z - 2) & (SP - 1)) * (G::PBYTES / sizeof(T));
      const T* Pp2 = pst + (size_t)((z + 2) & (SP - 1)) * (G::PBYTES / sizeof(T));
      const T* Q = qst + (size_t)((z & (SQ - 1)) * NQ) * (G::QBYTES / sizeof(T));
#pragma unroll
      for (int rr = 0; rr < RPT; ++rr) {
        const int ry = ty + TBY * rr;  // tile row of this thread
        const int y = y0 + ry;
        if constexpr (sizeof(T) == 4) {
          // two x-adjacent points per thread, 64-bit shared and global accesses
          const int xl = 2 * tx;
          const int x = x0 + xl;
          const int o = (ry + 2) * G::BXH + xl + G::XH;
          const int qo = ry * TBX + xl;
          constexpr int QS = G::QBYTES / 4;
          Nb2 v;
          gather_pair(P0, Pm1, Pp1, Pm2, Pp2, o, G::BXH, v);
          const float2 L = lap12_pair(v);
          if constexpr (FORM == 2) {
            // acc + (w mu) L, one rounding of w mu and one fused multiply-add
            const float w = START ? 0.5f : 1.0f;
            const float2 wu = mul2(make_float2(w, w), lds2(Q + qo));
            if (x < n && y < n)
              *reinterpret_cast<float2*>(o0 + (size_t)z * plane + (size_t)y * n + x) =
                  fma2(wu, L, lds2(Q + QS + qo));
            continue;
          }
          const float2 K = lds2(Q + (NQ - 1) * QS + qo);
          if (x < n && y < n) {  // N is even, so x + 1 < n as well
            const size_t gi = (size_t)z * plane + (size_t)y * n + x;
            if constexpr (FORM == 0) {
              if constexpr (START) {
                *reinterpret_cast<float2*>(o0 + gi) = start_pair(v.c, K, L);
                if (o1) *reinterpret_cast<float2*>(o1 + gi) = v.c;
              } else {
                *reinterpret_cast<float2*>(o0 + gi) = three_term_pair(v.c, K, L, lds2(Q + qo));
              }
            } else {
              float2 D = make_float2(0.f, 0.f), E = make_float2(0.f, 0.f);
              if constexpr (!START) {
                D = lds2(Q + qo);
                E = lds2(Q + QS + qo);
              }
              const Kp2 r = kahan_pair(v.c, K, L, D, E, START);
              *reinterpret_cast<float2*>(o0 + gi) = r.p;
              *reinterpret_cast<float2*>(o1 + gi) = r.d;
              *reinterpret_cast<float2*>(o2 + gi) = r.e;
            }
          }
        } else {
  #pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int xl = tx + 32 * h;
            const int x = x0 + xl;
            const int o = (ry + 2) * G::BXH + xl + G::XH;
            const int qo = ry * TBX + xl;
            const T L = lap12_sum(P0, Pm1, Pp1, Pm2, Pp2, o, G::BXH);
            const T c = P0[o];
            const T k = Q[(NQ - 1) * (G::QBYTES / sizeof(T)) + qo];
            if (x < n && y < n) {
              const size_t gi = (size_t)z * plane + (size_t)y * n + x;
              if constexpr (START) {
                o0[gi] = c + T(0.5) * k * L;
                if (o1) o1[gi] = c;
              } else {
                const T pm = Q[qo];
                o0[gi] = fma(k, L, fma(2.0, c, -pm));
              }
            }
          }
        }
      }  // rows of this thread
      if (__syncthreads_or(timed_out)) {
        if (tid == 0) {
          atomicCAS(&g_tma_status, 0u, (unsigned)(-FFPAT_ETIMEDOUT));
          // bounded wait for this CTA's copies still in flight
          for (int R = waited_upto + 1; R <= min(z1 + 1, z + SP - 3); ++R) {
            const int b = R & (SP - 1);
            mbar_wait(&bar[b], (phase >> b) & 1u, 1 << 24);
            phase ^= 1u << b;
          }
        }
        return;
      }
      if (tid == 0) issue_round<T, NQ, RPT>(maps, pst, qst, bar, z + SP - 2, z0, z1, x0, y0);
    }
  }
}

// ---------------------------------------------- batched step (serving) --
// One launch advances several independent problems (different N) by one
// FP32-Kahan leapfrog step each: the work items of all requests are
// concatenated and the persistent grid walks them.  The per-point arithmetic
// is the one of k_step_tma<float, 1, *>, so a request's result does not depend
// on which other requests share its launches.  Start steps (which read only
// kap besides p) and regular steps (d, e, kap) may share a launch.
constexpr int kMaxBatch = 28;

struct BatchReq {
  CUtensorMap p;     // p^n with the halo box
  CUtensorMap q[3];  // d, e, kap (halo-free)
  float* o0;         // p^{n+1}
  float* o1;         // d^{n+1}
  float* o2;         // e^{n+1}
  int n, zc, tiles_x, tiles_y, start;
};

struct BatchParams {
  int count;
  int item_end[kMaxBatch];  // exclusive prefix of the requests' item counts
  BatchReq r[kMaxBatch];
};

// the batched kernel's tile: 64 x 16, as the single-step kernel's
constexpr int kBatchRPT = 2;

__global__ void __launch_bounds__(NTX* NTY, 2) k_step_batch(const __grid_constant__ BatchParams bp) {
  using G = Geo<float, kBatchRPT>;
  constexpr int NQ = 3;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  float* pst = reinterpret_cast<float*>(smem);
  float* qst = reinterpret_cast<float*>(smem + SP * G::PBYTES);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + SP * G::PBYTES + SQ * NQ * G::QBYTES);
  if (*(volatile unsigned*)&g_tma_status != 0u) return;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * NTX + tx;
  if (tid == 0) {
    for (int i = 0; i < SP; ++i) mbar_init(&bar[i], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  unsigned phase = 0;
  const int nitems = bp.item_end[bp.count - 1];
  for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
    int r = 0;
    while (item >= bp.item_end[r]) ++r;
    const BatchReq& q = bp.r[r];
    const int local = item - (r ? bp.item_end[r - 1] : 0);
    const int n = q.n;
    const int tix = local % q.tiles_x;
    const int tiy = (local / q.tiles_x) % q.tiles_y;
    const int z0 = (local / (q.tiles_x * q.tiles_y)) * q.zc;
    const int z1 = min(n, z0 + q.zc);
    const int x0 = tix * TBX, y0 = tiy * G::TH;
    const bool start = q.start != 0;
    const size_t plane = (size_t)n * n;
    // round R: p plane R and the stream planes R - 2 (kap only at a start step)
    auto issue = [&](int R) {
      const bool wp = R <= z1 + 1;
      const bool wq = (R - 2 >= z0) && (R - 2 < z1);
      if (!wp && !wq) return;
      uint64_t* b = &bar[R & (SP - 1)];
      mbar_expect_tx(b, (wp ? G::PBYTES : 0) + (wq ? (start ? 1 : NQ) * G::QBYTES : 0));
      if (wp)
        tma_load_3d(pst + (size_t)(R & (SP - 1)) * (G::PBYTES / 4), &q.p, x0 - G::XH, y0 - 2, R, b);
      if (wq) {
        const int sl = (R - 2) & (SQ - 1);
        for (int k = start ? 2 : 0; k < NQ; ++k)
          tma_load_3d(qst + (size_t)(sl * NQ + k) * (G::QBYTES / 4), &q.q[k], x0, y0, R - 2, b);
      }
    };
    if (tid == 0)
      for (int R = z0 - 2; R <= z0 + SP - 3; ++R) issue(R);
    bool timed_out = false;
    int waited_upto = z0 - 3;
    for (int z = z0; z < z1; ++z) {
      for (int R = waited_upto + 1; R <= z + 2; ++R) {
        const int b = R & (SP - 1);
        if (!mbar_wait(&bar[b], (phase >> b) & 1u, kWaitCycles)) timed_out = true;
        phase ^= 1u << b;
      }
      waited_upto = z + 2;
      const float* P0 = pst + (size_t)(z & (SP - 1)) * (G::PBYTES / 4);
      const float* Pm1 = pst + (size_t)((z - 1) & (SP - 1)) * (G::PBYTES / 4);
      const float* Pp1 = pst + (size_t)((z + 1) & (SP - 1)) * (G::PBYTES / 4);
      const float* Pm2 = pst + (size_t)((z - 2) & (SP - 1)) * (G::PBYTES / 4);
      const float* Pp2 = pst + (size_t)((z + 2) & (SP - 1)) * (G::PBYTES / 4);
      const float* Qd = qst + (size_t)((z & (SQ - 1)) * NQ) * (G::QBYTES / 4);
#pragma unroll
      for (int rr = 0; rr < kBatchRPT; ++rr) {
        const int ry = ty + TBY * rr;  // tile row of this thread
        const int y = y0 + ry;
        const int xl = 2 * tx;
        const int x = x0 + xl;
        const int o = (ry + 2) * G::BXH + xl + G::XH;
        const int qo = ry * TBX + xl;
        constexpr int QS = G::QBYTES / 4;
        Nb2 v;
        gather_pair(P0, Pm1, Pp1, Pm2, Pp2, o, G::BXH, v);
        const float2 L = lap12_pair(v);
        const float2 K = lds2(Qd + 2 * QS + qo);
        if (x < n && y < n) {
          const size_t gi = (size_t)z * plane + (size_t)y * n + x;
          float2 D = make_float2(0.f, 0.f), E = make_float2(0.f, 0.f);
          if (!start) {
            D = lds2(Qd + qo);
            E = lds2(Qd + QS + qo);
          }
          const Kp2 r = kahan_pair(v.c, K, L, D, E, start);
          *reinterpret_cast<float2*>(q.o0 + gi) = r.p;
          *reinterpret_cast<float2*>(q.o1 + gi) = r.d;
          *reinterpret_cast<float2*>(q.o2 + gi) = r.e;
        }
      }
      if (__syncthreads_or(timed_out)) {
        if (tid == 0) {
          atomicCAS(&g_tma_status, 0u, (unsigned)(-FFPAT_ETIMEDOUT));
          for (int R = waited_upto + 1; R <= min(z1 + 1, z + SP - 3); ++R) {
            const int b = R & (SP - 1);
            mbar_wait(&bar[b], (phase >> b) & 1u, 1 << 24);
            phase ^= 1u << b;
          }
        }
        return;
      }
      if (tid == 0) issue(z + SP - 2);
    }
  }
}

// ------------------------------------------------ two steps per pass ----
// Temporal blocking: one launch advances the leapfrog by two steps.  Step A
// recomputes level n + 1 on the 64 x 16 tile plus a two-point x/y halo (the
// 68 x 20 extended tile) from a halo-4 box of p^n (72 x 24, starting 16-byte
// aligned at x0 - 4) and halo-2 boxes (72 x 20) of the per-point streams;
// step B then forms level n + 2 on the tile from the level-(n+1) planes.
//   * FP32-Kahan (k_step2_kahan): the streams are d^n, e^n, kap; the pass
//     writes p, d, e of level n + 2: 28 B per point per TWO steps (d and e are
//     read with a halo, so they are double-buffered, no in place);
//   * FP32 three-term (k_step2_f32): the streams are p^{n-1}, kap; the pass
//     writes p^{n+1} (step A, tile points) and p^{n+2} (step B): 20 B per point
//     per two steps, against 32 B for two single steps.
// Each point's arithmetic is that of the single-step kernel (same Laplacian
// order, same update), so results are bit-identical to single steps.  Points
// outside the grid read kap = 0 and zero state and therefore produce level
// n + 1 = 0 there: the zero ghost values of step B come out of step A.
//
// Organisation (one CTA per SM walks whole z-columns of its tile):
//   * a producer warp issues the TMA copies, one round per plane z: p^n and
//     the stream planes of z into slot z mod 8 of an 8-deep ring; it refills
//     a slot once every compute thread has reported the iteration that last
//     read it (iteration-done mbarriers), so copies run up to about five
//     planes ahead of the planes being computed;
//   * 22 compute warps, one point pair per thread: 16 warps own the tile's
//     rows and compute both steps of their pair, 6 warps the 168 halo pairs
//     (step A only).  The thread that computes step B of a pair computed its
//     step A as well, so the pair's level-(n+1) z-column and the point values
//     step B needs (d^{n+1}, e^{n+1} or p^n; kap) stay in registers; p^n's
//     z-column too (one new value per plane).  Only the x/y neighbours come
//     from shared memory: six 64-bit loads per step, plus the streams in
//     step A;
//   * level n + 1 goes through a 4-deep shared ring; a plane written in
//     iteration i is read by step B in iteration i + 2, after the
//     iteration-done barrier of iteration i, which every compute thread has
//     long passed by then (split arrive / wait, no block-wide barrier);
//   * the z-loop is unrolled by the ring depth, so every ring slot and
//     barrier index is a compile-time constant.
// Every wait is bounded (about a second of clock64 time) and gives up early
// once another thread of the CTA has recorded a timeout; the producer then
// waits a bounded time for its copies in flight, and the CTA returns after
// recording FFPAT_ETIMEDOUT in the device status word.
namespace tb2 {
constexpr int TH2 = 16;                  // output tile 64 x 16
constexpr int PW = 72, PH = TH2 + 8;     // p^n box (x0-4 .., y0-4 ..)
constexpr int QW = 72, QH = TH2 + 4;     // stream boxes (x0-4 .., y0-2 ..)
constexpr int AW = 68, AH = TH2 + 4;     // level-(n+1) planes on the extended tile (x0-2 .., y0-2 ..)
constexpr int PB = PW * PH * 4, QB = QW * QH * 4, AB = AW * AH * 4;
constexpr int RING = 8;                  // rounds in flight: p^n and stream planes
constexpr int RA = 4;                    // level-(n+1) planes
constexpr int NIN = TH2;                 // compute warps owning one tile row each
constexpr int NCW = NIN + 6;             // + the halo warps
constexpr int NHALO = 2 * 34 * 2 + 2 * TH2;  // 168 halo pairs of the 34 x 20 pair grid
constexpr int NCT = NCW * 32;            // compute threads (arrivals per iteration)
constexpr int NT2 = NCT + 32;            // + the producer warp
// streams per plane: d, e, kap (FP32-Kahan) or p^{n-1}, kap (three-term)
template <int FORM>
constexpr int NQ = FORM == 1 ? 3 : 2;
template <int FORM>
constexpr size_t bar_off() {
  return (size_t)RING * PB + (size_t)RING * NQ<FORM> * QB + (size_t)RA * AB;
}
template <int FORM>
constexpr size_t smem_bytes() {
  return bar_off<FORM>() + 2 * RING * 8 + 16;
}
static_assert(PB % 128 == 0 && QB % 128 == 0, "TMA destinations stay 128-byte aligned");
static_assert(NCW * 32 - NIN * 32 >= NHALO, "halo warps cover the halo pairs");
}  // namespace tb2

struct Maps2 {
  CUtensorMap p;     // p^n, 72 x 24 box
  CUtensorMap q[3];  // the streams, 72 x 20 boxes (kap last)
};

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Bounded wait that also gives up once another thread of the CTA recorded a
// failure in *abort.  Waiting threads sleep in the barrier instead of
// spinning, so the warps that have work keep the issue slots.
__device__ __forceinline__ bool tb2_wait(uint64_t* bar, unsigned parity, volatile int* abort) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (true) {
    for (int i = 0; i < 8; ++i)
      if (mbar_try_wait_ns(bar, parity, 20000u)) return true;
    if (*abort) return false;
    if (clock64() - t0 > kWaitCycles) return false;
  }
}

__device__ __forceinline__ void tb2_fail(volatile int* abort) {
  *abort = 1;
  atomicCAS(&g_tma_status, 0u, (unsigned)(-FFPAT_ETIMEDOUT));
}

// One work item of a two-step pass: a 64 x 16 tile and a z-range of one
// problem, with that problem's tensor maps and outputs.
// FORM 1: FP32-Kahan, o0/o1/o2 = p, d, e of level n + 2.
// FORM 0: three-term, o0 = p^{n+1}, o1 = p^{n+2} (o2 unused).
struct Step2Item {
  const Maps2* maps;
  float* o0;
  float* o1;
  float* o2;
  int n, x0, y0, z0, z1;
};

// a single problem: items are (tile, z-range) in x, y, z order
struct Step2One {
  const Maps2* maps;
  float *o0, *o1, *o2;
  int n, zc, tiles_x, tiles_y;
  __device__ Step2Item operator()(int item) const {
    const int tix = item % tiles_x;
    const int tiy = (item / tiles_x) % tiles_y;
    const int z0 = (item / (tiles_x * tiles_y)) * zc;
    return Step2Item{maps, o0, o1, o2, n, tix * TBX, tiy * tb2::TH2, z0, min(n, z0 + zc)};
  }
};

template <int FORM, class Items>
__device__ __forceinline__ void step2_body(const Items& items, int nitems) {
  using namespace tb2;
  constexpr int NQF = NQ<FORM>;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  float* P = reinterpret_cast<float*>(sm);
  float* Q = reinterpret_cast<float*>(sm + RING * PB);
  float* A = reinterpret_cast<float*>(sm + RING * PB + RING * NQF * QB);
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + bar_off<FORM>());  // round landed
  uint64_t* done = full + RING;                                         // iteration finished
  volatile int* abort = reinterpret_cast<volatile int*>(done + RING);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int i = 0; i < RING; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&done[i], NCT);
    }
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  grid_dependency_sync();
  if (*(volatile unsigned*)&g_tma_status != 0u) return;
  __syncthreads();

  // this thread's point pair on the 34 x 20 pair grid of the extended tile
  const bool inner = warp < NIN;
  int qx = 0, qy = 0;
  bool active = inner;
  if (inner) {
    qx = lane + 1;
    qy = warp + 2;
  } else if (warp < NCW) {
    const int t = (warp - NIN) * 32 + lane;
    active = t < NHALO;
    if (t < 136) {  // the two rows above and the two below the tile
      const int row = t / 34;
      qx = t - 34 * row;
      qy = row < 2 ? row : row + TH2;
    } else if (t < 136 + TH2) {  // the pair left of each tile row
      qy = 2 + (t - 136);
    } else if (t < NHALO) {  // and the pair right of it
      qx = 33;
      qy = 2 + (t - 136 - TH2);
    }
  }
  const int o = (qy + 2) * PW + 2 * qx + 2;  // in the p^n box
  const int qo = qy * QW + 2 * qx + 2;       // in the stream boxes
  const int ao = qy * AW + 2 * qx;           // in the level-(n+1) planes

  for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
    const Step2Item it = items(item);
    const Maps2& maps = *it.maps;
    float* __restrict__ o0 = it.o0;
    float* __restrict__ o1 = it.o1;
    float* __restrict__ o2 = it.o2;
    const int n = it.n, x0 = it.x0, y0 = it.y0, z0 = it.z0, z1 = it.z1;
    const unsigned plane = (unsigned)n * (unsigned)n;
    // iteration i computes step A at plane z0 - 2 + i and step B at z0 - 4 + i;
    // round r brings plane z0 - 4 + r of p^n (for r <= M + 3) and of the
    // streams (for 2 <= r <= M + 1)
    const int M = z1 - z0 + 4;
    bool ok = true;
    if (warp == NCW) {
      // ---- producer
      if (lane == 0) {
        int issued = 0;
        for (int r = 0; r < M + 4; ++r) {
          if (r >= RING) {
            // slot r mod 8 was last read in iteration r - 10 (iteration 0
            // follows every thread's read of the first planes)
            const int ir = r - 10 > 0 ? r - 10 : 0;
            if (!tb2_wait(&done[ir & (RING - 1)], (unsigned)(ir >> 3) & 1u, abort)) {
              ok = false;
              break;
            }
          }
          const int s = r & (RING - 1), z = z0 - 4 + r;
          const bool wq = r >= 2 && r <= M + 1;
          uint64_t* b = &full[s];
          mbar_expect_tx(b, PB + (wq ? NQF * QB : 0));
          tma_load_3d(P + s * (PB / 4), &maps.p, x0 - 4, y0 - 4, z, b);
          if (wq) {
#pragma unroll
            for (int k = 0; k < NQF; ++k)
              tma_load_3d(Q + (NQF * s + k) * (QB / 4), &maps.q[k], x0 - 4, y0 - 2, z, b);
          }
          issued = r + 1;
        }
        if (!ok) {
          tb2_fail(abort);
          // bounded wait for the copies still in flight
          for (int r = issued - RING > 0 ? issued - RING : 0; r < issued; ++r)
            mbar_wait(&full[r & (RING - 1)], (unsigned)(r >> 3) & 1u, 1 << 24);
        }
      }
      __syncwarp();
    } else {
      // ---- compute warps
      for (int r = 0; r < 4 && ok; ++r) ok = tb2_wait(&full[r], 0u, abort);
      if (!ok) tb2_fail(abort);
      // z-columns of the pair: p^n at z - 2 .. z + 1 of the step-A plane z,
      // level n + 1 at zB - 2 .. zB + 1 of the step-B plane zB, and the point
      // values step B takes from the last two step-A planes: d^{n+1} and
      // e^{n+1} (Kahan) or p^n (three-term), and kap
      float2 c0 = lds2(P + 0 * (PB / 4) + o), c1 = lds2(P + 1 * (PB / 4) + o);
      float2 c2 = lds2(P + 2 * (PB / 4) + o), c3 = lds2(P + 3 * (PB / 4) + o);
      const float2 zero = make_float2(0.f, 0.f);
      float2 a0 = zero, a1 = zero, a2 = zero, a3 = zero;
      float2 uq0 = zero, uq1 = zero, vq0 = zero, vq1 = zero, kq0 = zero, kq1 = zero;
      const int x = x0 + 2 * lane, y = y0 + warp;
      const bool store = inner && x < n && y < n;  // N % 4 == 0: x + 1 < n as well
      // offset of plane z0 - 4 + i (unsigned arithmetic: early values wrap and are
      // unused; N <= kTwoStepMaxN keeps every used offset below 2^32)
      unsigned gi = (unsigned)z0 * plane + (unsigned)y * (unsigned)n + (unsigned)x - 4u * plane;
      for (int ib = 0; ib < M; ib += RING) {
#pragma unroll
        for (int u = 0; u < RING; ++u) {
          const int i = ib + u;
          if (i < M) {
            // round i + 4 brings p^n at z + 2 (the column's new value)
            if (ok && !(ok = tb2_wait(&full[(u + 4) & 7], (unsigned)((i + 4) >> 3) & 1u, abort)))
              tb2_fail(abort);
            // ---- step A: level n + 1 at plane z = z0 - 2 + i
            const float* P0 = P + ((u + 2) & 7) * (PB / 4);
            const float* Qz = Q + NQF * ((u + 2) & 7) * (QB / 4);
            const float2 c4 = lds2(P + ((u + 4) & 7) * (PB / 4) + o);
            Nb2 v;
            const float2 XM = lds2(P0 + o - 2), XP = lds2(P0 + o + 2);
            v.c = c2;
            v.xm1 = make_float2(XM.y, c2.x);
            v.xp1 = make_float2(c2.y, XP.x);
            v.xm2 = XM;
            v.xp2 = XP;
            v.ym1 = lds2(P0 + o - PW);
            v.yp1 = lds2(P0 + o + PW);
            v.ym2 = lds2(P0 + o - 2 * PW);
            v.yp2 = lds2(P0 + o + 2 * PW);
            v.zm1 = c1;
            v.zp1 = c3;
            v.zm2 = c0;
            v.zp2 = c4;
            const float2 L = lap12_pair(v);
            const float2 Kv = lds2(Qz + (NQF - 1) * (QB / 4) + qo);
            float2 an, un, vn;  // level n + 1 at the pair; the values step B takes
            if constexpr (FORM == 1) {
              const Kp2 ra = kahan_pair(c2, Kv, L, lds2(Qz + qo), lds2(Qz + QB / 4 + qo), false);
              an = ra.p;
              un = ra.d;
              vn = ra.e;
            } else {
              an = three_term_pair(c2, Kv, L, lds2(Qz + qo));
              un = c2;
              vn = zero;
              // p^{n+1} of the tile's planes is an output of the pass
              if (store && i >= 2 && i < M - 2)
                *reinterpret_cast<float2*>(o0 + (gi + 2u * plane)) = an;
            }
            // the level-(n+1) slot of this plane was last read by step B of
            // iteration i - 2, and step B below reads the plane iteration
            // i - 2 wrote: both wait for iteration i - 2 to be done everywhere
            if (i >= 2 && ok &&
                !(ok = tb2_wait(&done[(u + 6) & 7], (unsigned)((i - 2) >> 3) & 1u, abort)))
              tb2_fail(abort);
            if (active) *reinterpret_cast<float2*>(A + (u & 3) * (AB / 4) + ao) = an;
            // ---- step B: level n + 2 at plane zB = z - 2 (tile rows only)
            if (inner && i >= 4) {
              const float* A0 = A + ((u + 2) & 3) * (AB / 4);
              Nb2 w;
              const float2 YM = lds2(A0 + ao - 2), YP = lds2(A0 + ao + 2);
              w.c = a2;
              w.xm1 = make_float2(YM.y, a2.x);
              w.xp1 = make_float2(a2.y, YP.x);
              w.xm2 = YM;
              w.xp2 = YP;
              w.ym1 = lds2(A0 + ao - AW);
              w.yp1 = lds2(A0 + ao + AW);
              w.ym2 = lds2(A0 + ao - 2 * AW);
              w.yp2 = lds2(A0 + ao + 2 * AW);
              w.zm1 = a1;
              w.zp1 = a3;
              w.zm2 = a0;
              w.zp2 = an;
              const float2 LB = lap12_pair(w);
              if constexpr (FORM == 1) {
                const Kp2 rb = kahan_pair(a2, kq0, LB, uq0, vq0, false);
                if (store) {
                  *reinterpret_cast<float2*>(o0 + gi) = rb.p;
                  *reinterpret_cast<float2*>(o1 + gi) = rb.d;
                  *reinterpret_cast<float2*>(o2 + gi) = rb.e;
                }
              } else {
                const float2 pb = three_term_pair(a2, kq0, LB, uq0);
                if (store) *reinterpret_cast<float2*>(o1 + gi) = pb;
              }
            }
            gi += plane;
            c0 = c1;
            c1 = c2;
            c2 = c3;
            c3 = c4;
            a0 = a1;
            a1 = a2;
            a2 = a3;
            a3 = an;
            uq0 = uq1;
            uq1 = un;
            vq0 = vq1;
            vq1 = vn;
            kq0 = kq1;
            kq1 = Kv;
            mbar_arrive(&done[u]);
          }
        }
      }
    }
    // every round issued was waited for by the compute warps: the rings are idle
    if (__syncthreads_or(!ok)) return;
    if (tid == 0) {
      for (int i = 0; i < RING; ++i) {
        mbar_inval(&full[i]);
        mbar_inval(&done[i]);
        mbar_init(&full[i], 1);
        mbar_init(&done[i], NCT);
      }
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(tb2::NT2, 1)
    k_step2_kahan(const __grid_constant__ Maps2 maps, float* __restrict__ po,
                  float* __restrict__ dout, float* __restrict__ eout, int n, int zc, int tiles_x,
                  int tiles_y, int nitems) {
  step2_body<1>(Step2One{&maps, po, dout, eout, n, zc, tiles_x, tiles_y}, nitems);
}

__global__ void __launch_bounds__(tb2::NT2, 1)
    k_step2_f32(const __grid_constant__ Maps2 maps, float* __restrict__ o1,
                float* __restrict__ o2, int n, int zc, int tiles_x, int tiles_y, int nitems) {
  step2_body<0>(Step2One{&maps, o1, o2, nullptr, n, zc, tiles_x, tiles_y}, nitems);
}

// ---- two FP32-Kahan steps per pass for several problems in one launch
// (the serving path): the work items of all problems are concatenated; every
// item carries its problem's tensor maps and outputs, so a problem's result
// does not depend on which others share the launch.
struct Batch2Req {
  Maps2 maps;
  float *o0, *o1, *o2;  // p, d, e of level n + 2
  int n, zc, tiles_x, tiles_y;
};

struct Batch2Params {
  int count;
  int item_end[kMaxBatch];  // exclusive prefix of the problems' item counts
  Batch2Req r[kMaxBatch];
};

struct Step2Batch {
  const Batch2Params* bp;
  __device__ Step2Item operator()(int item) const {
    int r = 0;
    while (item >= bp->item_end[r]) ++r;
    const Batch2Req& q = bp->r[r];
    const int local = item - (r ? bp->item_end[r - 1] : 0);
    return Step2One{&q.maps, q.o0, q.o1, q.o2, q.n, q.zc, q.tiles_x, q.tiles_y}(local);
  }
};

__global__ void __launch_bounds__(tb2::NT2, 1)
    k_step2_batch(const __grid_constant__ Batch2Params bp) {
  step2_body<1>(Step2Batch{&bp}, bp.item_end[bp.count - 1]);
}

// ------------------------------------ resident time loop (small grids) --
// When the work items of a grid fit the CTA slots of the GPU at one item per
// CTA, one cooperative launch runs the whole time loop.  Every CTA keeps its
// item (a 64 x 16 tile and up to rs::ZM planes) for all steps: the per-point
// state that no other CTA reads -- d and e of the increment form, p^{n-1} of
// the three-term form -- stays in registers, kap / 12 in shared memory, and
// only p^n moves through memory, in two ping-pong buffers that live in L2 at
// these sizes.  Between steps a CTA waits only for its neighbouring items
// (neighbour_sync), not for the whole grid.  Each step loads the
// item's zc + 4 halo planes of p^n by TMA at once (one mbarrier per plane) and
// computes the planes as they arrive, with the single-step kernel's
// arithmetic (gather_pair, lap12_pair, kahan_pair or the three-term update),
// so the result is bit for bit that of the step-by-step loop.  A step-by-step
// launch pays the launch, the ring's fill and its drain every step (about
// 3 us plus 0.55 us per plane of a work item on GB300), which at N <= 128 is
// most of the step.
namespace rs {
constexpr int ZM = 7;          // planes of one work item at most (registers)
constexpr int NPL = ZM + 4;    // p planes one item reads per step
using G = Geo<float, 2>;       // 64 x 16 tiles, 72 x 20 halo boxes
constexpr int PF = G::PBYTES / 4, QF = G::QBYTES / 4;
// the Kahan carries of each thread's second row live in shared memory (the
// first row's, and every d, in registers): the rest fits 128 registers
// without spilling
constexpr int EBYTES = ZM * TBY * NTX * 8;
constexpr size_t kSmem =
    (size_t)NPL * G::PBYTES + (size_t)ZM * G::QBYTES + EBYTES + (NPL + 1) * 8 + 1024;
}  // namespace rs

struct ResParams {
  CUtensorMap pin;    // p^0 (halo box)
  CUtensorMap pb[2];  // the state buffers (halo box)
  CUtensorMap kap;    // kap / 12 (tile box)
  float* buf[2];      // step s writes buf[s & 1] ...
  float* out;         // ... except the last step, which writes here when non-null
  unsigned* sync;     // one step flag per work item, zero at launch
  int n, zc, tiles_x, tiles_y, nt;
};

// Step boundary of the resident loop, point to point: a CTA publishes that
// it finished step s (its stores of p^{s+1} done, its loads of p^s complete)
// in its own flag, and before step s + 1 waits only for the items whose
// regions its halo reads (the neighbours within one tile in x and y and
// within two planes in z).  That covers both hazards of the two ping-pong
// buffers: the neighbours' p^{s+1} is written before it is read, and the
// buffer step s + 1 overwrites (p^{s-1}) is no longer read by any neighbour.
// Bounded: false when a neighbour did not arrive in time.
constexpr int kFlagStride = 32;  // one flag per 128-byte line

__device__ __forceinline__ bool neighbour_sync(unsigned* flags, unsigned s1, int tix, int tiy,
                                               int tz, int tiles_x, int tiles_y, int nzc,
                                               int zr) {
  const int tid = threadIdx.y * NTX + threadIdx.x;
  // this thread's generic-proxy stores before any later async-proxy (TMA) read
  asm volatile("fence.proxy.async.global;" ::: "memory");
  __syncthreads();
  if (tid == 0) {
    unsigned* f = flags + kFlagStride * ((tz * tiles_y + tiy) * tiles_x + tix);
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(f), "r"(s1) : "memory");
  }
  int fail = 0;
  const int nzr = 2 * zr + 1;
  if (tid < 9 * nzr) {
    const int jx = tix + tid % 3 - 1, jy = tiy + (tid / 3) % 3 - 1, jz = tz + tid / 9 - zr;
    const bool self = jx == tix && jy == tiy && jz == tz;
    if (!self && jx >= 0 && jx < tiles_x && jy >= 0 && jy < tiles_y && jz >= 0 && jz < nzc) {
      const unsigned* f = flags + kFlagStride * ((jz * tiles_y + jy) * tiles_x + jx);
      const long long t0 = clock64();
      while (true) {
        unsigned v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(f) : "memory");
        if ((int)(v - s1) >= 0) break;
        if (clock64() - t0 > kWaitCycles) {
          fail = 1;
          break;
        }
        __nanosleep(64);
      }
      asm volatile("fence.proxy.async.global;" ::: "memory");
    }
  }
  return __syncthreads_or(fail) == 0;
}

// One step of the resident loop over the item's planes.  sa, sb, es: the
// state of the thread's points (form 1: d in sa, e in sb for the first row
// and in shared memory es for the second; form 0: p^{n-1} in sa; moving its
// second row to es as well measured slower).
// Rows outer, planes inner: a thread walks the z-column of each of its two
// rows and keeps the four column values it already read (z-2 .. z+1) in
// registers, so each plane costs one new column load (z+2) and the six x/y
// neighbour loads; the arithmetic is gather_pair's, value for value.
template <int FORM, bool START>
__device__ __forceinline__ bool res_step(const float* pst, const float* kst, uint64_t* bar,
                                         unsigned parity, float2 (&sa)[rs::ZM][2],
                                         float2 (&sb)[rs::ZM], float2* __restrict__ es,
                                         float* __restrict__ dst,
                                         int n, int nz, int z0, int x0, int y0) {
  using G = rs::G;
  const int tx = threadIdx.x, ty = threadIdx.y;
  bool ok = true;
#pragma unroll
  for (int i = 0; i < 4; ++i)
    if (ok) ok = mbar_wait(&bar[i], parity, kWaitCycles);
  const int xl = 2 * tx, x = x0 + xl;
#pragma unroll
  for (int rr = 0; rr < 2; ++rr) {
    const int ry = ty + TBY * rr, y = y0 + ry;
    const int o = (ry + 2) * G::BXH + xl + G::XH;
    float2 c0 = lds2(pst + o), c1 = lds2(pst + rs::PF + o);
    float2 c2 = lds2(pst + 2 * rs::PF + o), c3 = lds2(pst + 3 * rs::PF + o);
#pragma unroll
    for (int zi = 0; zi < rs::ZM; ++zi) {
      if (zi < nz) {
        // the first row's pass waits for each plane; the second finds them complete
        if (rr == 0 && ok) ok = mbar_wait(&bar[zi + 4], parity, kWaitCycles);
        const float* P0 = pst + (zi + 2) * rs::PF;
        const float2 c4 = lds2(pst + (zi + 4) * rs::PF + o);
        const float2 XM = lds2(P0 + o - 2), XP = lds2(P0 + o + 2);
        Nb2 v;
        v.c = c2;
        v.xm1 = make_float2(XM.y, c2.x);
        v.xp1 = make_float2(c2.y, XP.x);
        v.xm2 = XM;
        v.xp2 = XP;
        v.ym1 = lds2(P0 + o - G::BXH);
        v.yp1 = lds2(P0 + o + G::BXH);
        v.ym2 = lds2(P0 + o - 2 * G::BXH);
        v.yp2 = lds2(P0 + o + 2 * G::BXH);
        v.zm1 = c1;
        v.zp1 = c3;
        v.zm2 = c0;
        v.zp2 = c4;
        const float2 L = lap12_pair(v);
        const float2 K = lds2(kst + zi * rs::QF + ry * TBX + xl);
        float2 w;
        if constexpr (FORM == 1) {
          float2* ep = es + (zi * TBY + ty) * NTX + tx;
          const Kp2 r = kahan_pair(v.c, K, L, sa[zi][rr], rr == 0 ? sb[zi] : *ep, START);
          sa[zi][rr] = r.d;
          if (rr == 0)
            sb[zi] = r.e;
          else
            *ep = r.e;
          w = r.p;
        } else {
          w = START ? start_pair(v.c, K, L) : three_term_pair(v.c, K, L, sa[zi][rr]);
          sa[zi][rr] = v.c;
        }
        if (x < n && y < n)  // N % 4 == 0, so x + 1 < n as well
          *reinterpret_cast<float2*>(dst + (size_t)(z0 + zi) * n * n + (size_t)y * n + x) = w;
        c0 = c1;
        c1 = c2;
        c2 = c3;
        c3 = c4;
        // keep the next plane's loads behind this one (register pressure)
        asm volatile("" ::: "memory");
      }
    }
  }
  return ok;
}

template <int FORM>
__global__ void __launch_bounds__(NTX* NTY, 2) k_wave_resident(const __grid_constant__ ResParams rp) {
  using G = rs::G;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  float* pst = reinterpret_cast<float*>(smem);                          // NPL halo planes
  float* kst = reinterpret_cast<float*>(smem + rs::NPL * G::PBYTES);    // ZM kap tiles
  float2* es = reinterpret_cast<float2*>(smem + rs::NPL * G::PBYTES + rs::ZM * G::QBYTES);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + rs::NPL * G::PBYTES + rs::ZM * G::QBYTES +
                                              rs::EBYTES);
  const int tid = threadIdx.y * NTX + threadIdx.x;
  const int n = rp.n, item = blockIdx.x;
  const int tix = item % rp.tiles_x, tiy = (item / rp.tiles_x) % rp.tiles_y;
  const int tz = item / (rp.tiles_x * rp.tiles_y);
  const int z0 = tz * rp.zc;
  const int nz = min(n - z0, rp.zc);
  const int nzc = (n + rp.zc - 1) / rp.zc;
  const int zr = rp.zc >= 2 ? 1 : 2;  // z-chunks a two-plane halo reaches
  const int x0 = tix * TBX, y0 = tiy * G::TH;
  if (tid == 0) {
    for (int i = 0; i <= rs::NPL; ++i) mbar_init(&bar[i], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // after a device-side failure of an earlier launch every CTA returns at once
  if (*(volatile unsigned*)&g_tma_status != 0u) return;
  if (tid == 0) {
    mbar_expect_tx(&bar[rs::NPL], (unsigned)(nz * G::QBYTES));
    for (int zi = 0; zi < nz; ++zi)
      tma_load_3d(kst + zi * rs::QF, &rp.kap, x0, y0, z0 + zi, &bar[rs::NPL]);
  }
  float2 sa[rs::ZM][2], sb[rs::ZM];
#pragma unroll
  for (int zi = 0; zi < rs::ZM; ++zi) {
    sa[zi][0] = sa[zi][1] = sb[zi] = make_float2(0.f, 0.f);
    es[(zi * TBY + threadIdx.y) * NTX + threadIdx.x] = make_float2(0.f, 0.f);
  }
  bool ok = mbar_wait(&bar[rs::NPL], 0, kWaitCycles);
  if (__syncthreads_or(!ok)) {
    if (tid == 0) {
      atomicCAS(&g_tma_status, 0u, (unsigned)(-FFPAT_ETIMEDOUT));
      mbar_wait(&bar[rs::NPL], 0, 1 << 24);
    }
    return;
  }
  for (int s = 0; s < rp.nt; ++s) {
    const CUtensorMap* src = s == 0 ? &rp.pin : &rp.pb[(s - 1) & 1];
    float* dst = (s == rp.nt - 1 && rp.out) ? rp.out : rp.buf[s & 1];
    // one lane of warp 0 per plane issues its copy (after its own proxy fence:
    // the neighbours' generic-proxy stores before this async-proxy read)
    if (tid < nz + 4) {
      asm volatile("fence.proxy.async.global;" ::: "memory");
      mbar_expect_tx(&bar[tid], G::PBYTES);
      tma_load_3d(pst + tid * rs::PF, src, x0 - G::XH, y0 - 2, z0 - 2 + tid, &bar[tid]);
    }
    const unsigned parity = (unsigned)s & 1u;
    ok = s == 0 ? res_step<FORM, true>(pst, kst, bar, parity, sa, sb, es, dst, n, nz, z0, x0, y0)
                : res_step<FORM, false>(pst, kst, bar, parity, sa, sb, es, dst, n, nz, z0, x0, y0);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicCAS(&g_tma_status, 0u, (unsigned)(-FFPAT_ETIMEDOUT));
        // bounded wait for this CTA's copies of the step still in flight
        for (int i = 0; i < nz + 4; ++i) mbar_wait(&bar[i], parity, 1 << 24);
      }
      return;
    }
    if (s + 1 < rp.nt && !neighbour_sync(rp.sync, (unsigned)(s + 1), tix, tiy, tz, rp.tiles_x,
                                         rp.tiles_y, nzc, zr)) {
      if (tid == 0) atomicCAS(&g_tma_status, 0u, (unsigned)(-FFPAT_ETIMEDOUT));
      return;
    }
  }
}

// ------------------------------------------------------------- host side --

// FFPAT_ZCHUNK=<planes> fixes the z-range of one work item of the TMA
// stencil kernels (a tuning knob for measurements; 0 or unset = automatic)
int zchunk_override() {
  static int v = [] {
    const char* e = getenv("FFPAT_ZCHUNK");
    return e ? atoi(e) : 0;
  }();
  return v;
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

struct MapKey {
  const void* ptr;
  int n, esize, bx, by;
  bool operator==(const MapKey& o) const {
    return ptr == o.ptr && n == o.n && esize == o.esize && bx == o.bx && by == o.by;
  }
};
struct MapKeyHash {
  size_t operator()(const MapKey& k) const {
    return std::hash<const void*>()(k.ptr) ^ ((size_t)k.n << 1) ^ ((size_t)k.esize << 13) ^
           ((size_t)k.bx << 17) ^ ((size_t)k.by << 27);
  }
};

int make_map_box(CUtensorMap* m, const void* base, int n, int esize, int bx, int by);

// the single-step kernels' boxes: p^n with the two-point halo, or the bare tile
int make_map(CUtensorMap* m, const void* base, int n, int esize, bool halo, int th = TBY) {
  const int xh = 16 / esize;
  return make_map_box(m, base, n, esize, halo ? TBX + 2 * xh : TBX, halo ? th + 4 : th);
}

int make_map_box(CUtensorMap* m, const void* base, int n, int esize, int bx, int by) {
  static thread_local std::unordered_map<MapKey, CUtensorMap, MapKeyHash> cache;
  const MapKey key{base, n, esize, bx, by};
  auto it = cache.find(key);
  if (it != cache.end()) {
    *m = it->second;
    return FFPAT_OK;
  }
  std::call_once(g_encode_once, [] {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  });
  if (!g_encode) return FFPAT_ECUDA;
  cuuint64_t dims[3] = {(cuuint64_t)n, (cuuint64_t)n, (cuuint64_t)n};
  cuuint64_t strides[2] = {(cuuint64_t)n * esize, (cuuint64_t)n * n * esize};
  cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = g_encode(
      m, esize == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3,
      const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
      CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return FFPAT_ECUDA;
  if (cache.size() > 256) cache.clear();
  cache.emplace(key, *m);
  return FFPAT_OK;
}

// Launch with programmatic stream serialization, so that consecutive leapfrog
// launches overlap one's tail with the next one's prologue (the kernels wait
// in grid_dependency_sync before touching global memory).
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                       cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

// z-range of one work item of the single-step kernel: every work item costs
// its zc planes plus the ring's 4 halo planes, and the grid runs
// ceil(items / slots) rounds of items; pick the zc (>= 6) of least
// rounds x (zc + 4) among those that keep at least 90 % of the CTA slots
// busy.  Grids too small for that keep ranges of N / 8.. planes as before.
int choose_zchunk(int n, int tiles, int slots) {
  int best = 0;
  long long best_cost = 0;
  for (int zc = 6; zc <= n; ++zc) {
    const long long items = (long long)tiles * ((n + zc - 1) / zc);
    if (items * 10 < (long long)slots * 9) break;  // items only shrink as zc grows
    const long long rounds = (items + slots - 1) / slots;
    const long long cost = rounds * (zc + 4);
    if (best == 0 || cost < best_cost) {
      best = zc;
      best_cost = cost;
    }
  }
  if (best > 0) return best;
  int zchunks = (4 * slots + tiles - 1) / tiles;
  const int zmax = n / 8 > 0 ? n / 8 : 1;
  if (zchunks > zmax) zchunks = zmax;
  if (zchunks < 1) zchunks = 1;
  return (n + zchunks - 1) / zchunks;
}

// z-range (planes) of the items of a batched pass over several problems.
// The persistent grid walks the items in rounds of `slots`, and an item costs
// its planes plus a fixed halo of 4, so the launch takes about
// ceil(items / slots) x (len + 4) plane times: take the len of least such
// cost (the longest among equals: the least halo work).  Tiles are TBX points
// wide and tile_h high.  The choice depends only on the sizes, which change
// only when a request joins or leaves: the last two are kept.
template <class Batch>
int batch_zrange(const Batch* steps, int count, int tile_h, int slots) {
  struct Memo {
    int count, tile_h, slots, len;
    int n[kMaxBatch];
  };
  static thread_local Memo memo[2] = {};
  static thread_local int next = 0;
  for (Memo& m : memo) {
    if (m.count != count || m.tile_h != tile_h || m.slots != slots) continue;
    bool same = true;
    for (int i = 0; i < count && same; ++i) same = m.n[i] == steps[i].n;
    if (same) return m.len;
  }
  int nmax = 1;
  for (int i = 0; i < count; ++i) nmax = steps[i].n > nmax ? steps[i].n : nmax;
  int best = nmax;
  long long best_cost = -1;
  for (int len = 1; len <= nmax; ++len) {
    long long items = 0;
    for (int i = 0; i < count; ++i) {
      const int n = steps[i].n;
      items += (long long)((n + TBX - 1) / TBX) * ((n + tile_h - 1) / tile_h) * ((n + len - 1) / len);
    }
    const long long cost = (items + slots - 1) / slots * (len + 4);
    if (best_cost < 0 || cost <= best_cost) {
      best = len;
      best_cost = cost;
    }
  }
  Memo& m = memo[next];
  next ^= 1;
  m.count = count;
  m.tile_h = tile_h;
  m.slots = slots;
  m.len = best;
  for (int i = 0; i < count; ++i) m.n[i] = steps[i].n;
  return best;
}

template <typename T, int FORM, bool START, int RPT>
int launch_one(const Plan& pl, const Maps& maps, void* o0, void* o1, void* o2, cudaStream_t st) {
  using G = Geo<T, RPT>;
  constexpr int NQ = Streams<T, FORM, START>::NQ;
  const size_t smem = (size_t)SP * G::PBYTES + (size_t)SQ * NQ * G::QBYTES + SP * 8 + 1024;
  auto kern = k_step_tma<T, FORM, START, RPT>;
  static int occ = 0;  // per instantiation
  static std::once_flag once;
  std::call_once(once, [&] {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NTX * NTY, smem);
    if (occ < 1) occ = 1;
  });
  const int n = pl.n;
  const int tiles_x = (n + TBX - 1) / TBX, tiles_y = (n + G::TH - 1) / G::TH;
  const int slots = kNumSMs * occ;
  int zc = choose_zchunk(n, tiles_x * tiles_y, slots);
  if (zchunk_override() > 0) zc = zchunk_override() < n ? zchunk_override() : n;
  const int zchunks = (n + zc - 1) / zc;
  const int nitems = tiles_x * tiles_y * zchunks;
  const int grid = nitems < slots ? nitems : slots;
  const cudaError_t e =
      launch_pdl(kern, dim3(grid), dim3(NTX, NTY), smem, st, maps, (T*)o0, (T*)o1, (T*)o2, n, zc,
                 tiles_x, tiles_y, nitems);
  count_launch();
  if (e != cudaSuccess) {
    cudaGetLastError();
    return report(FFPAT_ECUDA, "k_step_tma launch: %s", cudaGetErrorString(e));
  }
  return check_launch("k_step_tma");
}

}  // namespace

bool tma_supported(const Plan& pl, const void* const* ptrs, int count) {
  if (pl.esize == 4 ? (pl.n % 4) : (pl.n % 2)) return false;
  for (int i = 0; i < count; ++i)
    if (ptrs[i] && ((uintptr_t)ptrs[i] & 15)) return false;
  return true;
}

// FFPAT_RPT=<1|2> fixes the rows per thread of the single-step kernel (a
// tuning knob for measurements; 0 or unset = 2: the 64 x 16 tile, measured
// faster on GB300 at 128^3 - 384^3 in every precision: fewer halo rows per
// output row and the per-plane waits and barrier shared by twice the points)
static int rpt_override() {
  static int v = [] {
    const char* e = getenv("FFPAT_RPT");
    return e ? atoi(e) : 0;
  }();
  return v;
}

template <int RPT>
static int launch_step_tma_r(const Plan& pl, int form, bool start, const void* p,
                             const void* const* q, void* o0, void* o1, void* o2, cudaStream_t st) {
  Maps maps;
  const int es = (int)pl.esize;
  const int th = TBY * RPT;
  if (make_map(&maps.p, p, pl.n, es, true, th) != FFPAT_OK) return check_launch("tensor map (p)");
  const int nq = form == 2 ? 2 : (start ? 1 : (form == 0 ? 2 : 3));
  for (int i = 0; i < 3; ++i) {
    if (i < nq) {
      if (make_map(&maps.q[i], q[i], pl.n, es, false, th) != FFPAT_OK)
        return check_launch("tensor map (q)");
    } else {
      maps.q[i] = maps.p;
    }
  }
  if (pl.prec == FFPAT_FP64) {
    return start ? launch_one<double, 0, true, RPT>(pl, maps, o0, o1, o2, st)
                 : launch_one<double, 0, false, RPT>(pl, maps, o0, o1, o2, st);
  }
  if (form == 2)
    return start ? launch_one<float, 2, true, RPT>(pl, maps, o0, o1, o2, st)
                 : launch_one<float, 2, false, RPT>(pl, maps, o0, o1, o2, st);
  if (form == 0)
    return start ? launch_one<float, 0, true, RPT>(pl, maps, o0, o1, o2, st)
                 : launch_one<float, 0, false, RPT>(pl, maps, o0, o1, o2, st);
  return start ? launch_one<float, 1, true, RPT>(pl, maps, o0, o1, o2, st)
               : launch_one<float, 1, false, RPT>(pl, maps, o0, o1, o2, st);
}

int launch_step_tma(const Plan& pl, int form, bool start, const void* p, const void* const* q,
                    void* o0, void* o1, void* o2, cudaStream_t st) {
  const int rpt = rpt_override() == 1 ? 1 : 2;
  if (rpt == 2) return launch_step_tma_r<2>(pl, form, start, p, q, o0, o1, o2, st);
  return launch_step_tma_r<1>(pl, form, start, p, q, o0, o1, o2, st);
}

int launch_step_batch(const BatchStep* steps, int count, cudaStream_t st) {
  if (count < 1) return FFPAT_OK;
  if (count > kMaxBatch) return report(FFPAT_EINVAL, "batched step: %d requests > %d", count, kMaxBatch);
  using G = Geo<float, kBatchRPT>;
  const size_t smem = (size_t)SP * G::PBYTES + (size_t)SQ * 3 * G::QBYTES + SP * 8 + 1024;
  static int occ = 0;
  static std::once_flag once;
  std::call_once(once, [&] {
    cudaFuncSetAttribute(k_step_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_step_batch, NTX * NTY, smem);
    if (occ < 1) occ = 1;
  });
  static thread_local BatchParams bp;
  int total = 0;
  const int slots = kNumSMs * occ;
  const int len = batch_zrange(steps, count, G::TH, slots);
  bp.count = count;
  for (int i = 0; i < count; ++i) {
    const BatchStep& b = steps[i];
    BatchReq& r = bp.r[i];
    if (make_map(&r.p, b.p, b.n, 4, true, G::TH) != FFPAT_OK ||
        make_map(&r.q[2], b.kap, b.n, 4, false, G::TH) != FFPAT_OK)
      return report(FFPAT_ECUDA, "batched step: tensor map");
    if (!b.start) {
      if (make_map(&r.q[0], b.d, b.n, 4, false, G::TH) != FFPAT_OK ||
          make_map(&r.q[1], b.e, b.n, 4, false, G::TH) != FFPAT_OK)
        return report(FFPAT_ECUDA, "batched step: tensor map");
    } else {
      r.q[0] = r.q[2];
      r.q[1] = r.q[2];
    }
    r.o0 = b.pout;
    r.o1 = b.d;
    r.o2 = b.e;
    r.n = b.n;
    r.start = b.start ? 1 : 0;
    r.tiles_x = (b.n + TBX - 1) / TBX;
    r.tiles_y = (b.n + G::TH - 1) / G::TH;
    r.zc = len < b.n ? len : b.n;
    const int zchunks = (b.n + r.zc - 1) / r.zc;
    total += r.tiles_x * r.tiles_y * zchunks;
    bp.item_end[i] = total;
  }
  const int grid = total < slots ? total : slots;
  k_step_batch<<<grid, dim3(NTX, NTY), smem, st>>>(bp);
  count_launch();
  return check_launch("k_step_batch");
}

// A one-CTA kernel whose mbarrier never completes (nothing arrives on it):
// the bounded wait runs out after `cycles` and the kernel records
// FFPAT_ETIMEDOUT in the status word, exactly as the stencil kernels do, then
// returns.  Used to test failure detection without faulting or hanging.
__global__ void k_wait_timeout(long long cycles) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (!mbar_wait(&bar, 0u, cycles)) atomicCAS(&g_tma_status, 0u, (unsigned)(-FFPAT_ETIMEDOUT));
  }
}

int launch_wait_timeout(long long cycles, cudaStream_t st) {
  k_wait_timeout<<<1, 32, 0, st>>>(cycles);
  count_launch();
  return check_launch("k_wait_timeout");
}

// One two-step pass: grid of one CTA per SM over (64 x 16 tile, z-range) items.
template <typename Kern, typename... Outs>
int launch_step2(Kern kern, size_t smem_need, const char* name, const Plan& pl, const Maps2& maps,
                 cudaStream_t st, Outs... outs) {
  const size_t smem = smem_need + 1024;
  // the shared-memory opt-in, once per kernel (per instantiation of this template)
  static cudaError_t attr = cudaErrorUnknown;
  static std::once_flag once;
  std::call_once(once, [&] {
    attr = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  if (attr != cudaSuccess) {
    cudaGetLastError();
    return report(FFPAT_ECUDA, "%s: %zu bytes of shared memory refused", name, smem);
  }
  const int n = pl.n;
  const int tiles_x = (n + TBX - 1) / TBX, tiles_y = (n + tb2::TH2 - 1) / tb2::TH2;
  const int slots = kNumSMs;  // one CTA per SM
  // z-ranges: step A repeats 4 planes per range, the same cost model as the
  // single-step kernel (at 384^3 whole columns: 144 items for 152 slots)
  int zc = choose_zchunk(n, tiles_x * tiles_y, slots);
  if (zchunk_override() > 0) zc = zchunk_override() < n ? zchunk_override() : n;
  const int zchunks = (n + zc - 1) / zc;
  const int nitems = tiles_x * tiles_y * zchunks;
  const int grid = nitems < slots ? nitems : slots;
  const cudaError_t le = launch_pdl(kern, dim3(grid), dim3(tb2::NT2), smem, st, maps, outs..., n,
                                    zc, tiles_x, tiles_y, nitems);
  count_launch();
  if (le != cudaSuccess) {
    cudaGetLastError();
    return report(FFPAT_ECUDA, "%s launch: %s", name, cudaGetErrorString(le));
  }
  return check_launch(name);
}

int launch_step2_kahan(const Plan& pl, const void* p, const void* d, const void* e, void* po,
                       void* dout, void* eout, cudaStream_t st) {
  if (pl.n > kTwoStepMaxN)
    return report(FFPAT_EINVAL, "two-step pass: N = %d > %d (32-bit offsets)", pl.n, kTwoStepMaxN);
  Maps2 maps;
  if (make_map_box(&maps.p, p, pl.n, 4, tb2::PW, tb2::PH) != FFPAT_OK ||
      make_map_box(&maps.q[0], d, pl.n, 4, tb2::QW, tb2::QH) != FFPAT_OK ||
      make_map_box(&maps.q[1], e, pl.n, 4, tb2::QW, tb2::QH) != FFPAT_OK ||
      make_map_box(&maps.q[2], pl.kap, pl.n, 4, tb2::QW, tb2::QH) != FFPAT_OK)
    return report(FFPAT_ECUDA, "two-step kernel: tensor map");
  return launch_step2(k_step2_kahan, tb2::smem_bytes<1>(), "k_step2_kahan", pl, maps, st,
                      (float*)po, (float*)dout, (float*)eout);
}

int launch_step2_f32(const Plan& pl, const void* pm, const void* p, void* o1, void* o2,
                     cudaStream_t st) {
  if (pl.n > kTwoStepMaxN)
    return report(FFPAT_EINVAL, "two-step pass: N = %d > %d (32-bit offsets)", pl.n, kTwoStepMaxN);
  Maps2 maps;
  if (make_map_box(&maps.p, p, pl.n, 4, tb2::PW, tb2::PH) != FFPAT_OK ||
      make_map_box(&maps.q[0], pm, pl.n, 4, tb2::QW, tb2::QH) != FFPAT_OK ||
      make_map_box(&maps.q[1], pl.kap, pl.n, 4, tb2::QW, tb2::QH) != FFPAT_OK)
    return report(FFPAT_ECUDA, "two-step kernel: tensor map");
  maps.q[2] = maps.q[1];
  return launch_step2(k_step2_f32, tb2::smem_bytes<0>(), "k_step2_f32", pl, maps, st,
                      (float*)o1, (float*)o2);
}

int launch_step2_batch(const BatchStep2* steps, int count, cudaStream_t st) {
  if (count < 1) return FFPAT_OK;
  if (count > kMaxBatch)
    return report(FFPAT_EINVAL, "batched two-step pass: %d requests > %d", count, kMaxBatch);
  const size_t smem = tb2::smem_bytes<1>() + 1024;
  static cudaError_t attr = cudaErrorUnknown;
  static std::once_flag once;
  std::call_once(once, [&] {
    attr = cudaFuncSetAttribute(k_step2_batch, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem);
  });
  if (attr != cudaSuccess) {
    cudaGetLastError();
    return report(FFPAT_ECUDA, "k_step2_batch: %zu bytes of shared memory refused", smem);
  }
  static thread_local Batch2Params bp;
  const int slots = kNumSMs;  // one CTA per SM
  const int len = batch_zrange(steps, count, tb2::TH2, slots);
  int total = 0;
  bp.count = count;
  for (int i = 0; i < count; ++i) {
    const BatchStep2& b = steps[i];
    if (b.n > kTwoStepMaxN)
      return report(FFPAT_EINVAL, "batched two-step pass: N = %d > %d (32-bit offsets)", b.n,
                    kTwoStepMaxN);
    Batch2Req& r = bp.r[i];
    if (make_map_box(&r.maps.p, b.p, b.n, 4, tb2::PW, tb2::PH) != FFPAT_OK ||
        make_map_box(&r.maps.q[0], b.d, b.n, 4, tb2::QW, tb2::QH) != FFPAT_OK ||
        make_map_box(&r.maps.q[1], b.e, b.n, 4, tb2::QW, tb2::QH) != FFPAT_OK ||
        make_map_box(&r.maps.q[2], b.kap, b.n, 4, tb2::QW, tb2::QH) != FFPAT_OK)
      return report(FFPAT_ECUDA, "batched two-step pass: tensor map");
    r.o0 = b.pout;
    r.o1 = b.dout;
    r.o2 = b.eout;
    r.n = b.n;
    r.tiles_x = (b.n + TBX - 1) / TBX;
    r.tiles_y = (b.n + tb2::TH2 - 1) / tb2::TH2;
    r.zc = len < b.n ? len : b.n;
    const int zchunks = (b.n + r.zc - 1) / r.zc;
    total += r.tiles_x * r.tiles_y * zchunks;
    bp.item_end[i] = total;
  }
  const int grid = total < slots ? total : slots;
  k_step2_batch<<<grid, tb2::NT2, smem, st>>>(bp);
  count_launch();
  return check_launch("k_step2_batch");
}

// ---- the resident time loop (host side)
namespace {
template <int FORM>
int resident_slots(int* occ_out) {
  static int occ = 0, sms = 0;
  static std::once_flag once;
  std::call_once(once, [] {
    auto kern = k_wave_resident<FORM>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rs::kSmem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NTX * NTY, rs::kSmem) !=
        cudaSuccess)
      occ = 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      sms = 0;
    cudaGetLastError();
  });
  if (occ_out) *occ_out = occ;
  return occ * sms;
}

// z-range of the resident loop's items: one item per CTA slot, at most rs::ZM
// planes; among the ranges that fit, the least (items per SM) x (zc + 2), the
// longer range on ties.  0 if none fits.
int resident_zchunk(int n, int slots, int sms) {
  const int tiles = ((n + TBX - 1) / TBX) * ((n + rs::G::TH - 1) / rs::G::TH);
  const int ov = zchunk_override();
  int best = 0;
  long long best_cost = 0;
  for (int zc = 1; zc <= rs::ZM; ++zc) {
    const long long items = (long long)tiles * ((n + zc - 1) / zc);
    if (items > slots || items > kResidentMaxItems) continue;
    if (ov > 0 && zc != ov) continue;
    const long long cost = ((items + sms - 1) / sms) * (zc + 2);
    if (best == 0 || cost <= best_cost) {
      best = zc;
      best_cost = cost;
    }
  }
  return best;
}
}  // namespace

int resident_zc(const Plan& pl, int form) {
  if (pl.esize != 4 || pl.n % 4 != 0 || pl.n < 4 || !pl.sync) return 0;
  int occ = 0;
  const int slots = form == 1 ? resident_slots<1>(&occ) : resident_slots<0>(&occ);
  if (slots <= 0 || occ <= 0) return 0;
  return resident_zchunk(pl.n, slots, slots / occ);
}

int launch_wave_resident(const Plan& pl, int form, const void* in, void* out, void* b0, void* b1,
                         const void** result, cudaStream_t st, bool* refused) {
  if (refused) *refused = false;
  const int zc = resident_zc(pl, form);
  if (zc <= 0) return report(FFPAT_EINVAL, "resident time loop: N = %d does not fit", pl.n);
  static thread_local ResParams rp;
  const int n = pl.n;
  if (make_map(&rp.pin, in, n, 4, true, rs::G::TH) != FFPAT_OK ||
      make_map(&rp.pb[0], b0, n, 4, true, rs::G::TH) != FFPAT_OK ||
      make_map(&rp.pb[1], b1, n, 4, true, rs::G::TH) != FFPAT_OK ||
      make_map(&rp.kap, pl.kap, n, 4, false, rs::G::TH) != FFPAT_OK)
    return report(FFPAT_ECUDA, "resident time loop: tensor map");
  rp.buf[0] = (float*)b0;
  rp.buf[1] = (float*)b1;
  rp.out = (float*)out;
  rp.sync = pl.sync;
  rp.n = n;
  rp.zc = zc;
  rp.tiles_x = (n + TBX - 1) / TBX;
  rp.tiles_y = (n + rs::G::TH - 1) / rs::G::TH;
  rp.nt = pl.nt;
  const int items = rp.tiles_x * rp.tiles_y * ((n + zc - 1) / zc);
  if (items > kResidentMaxItems)
    return report(FFPAT_EINVAL, "resident time loop: %d work items > %d", items, kResidentMaxItems);
  if (cudaMemsetAsync(pl.sync, 0, sizeof(unsigned) * kFlagStride * items, st) != cudaSuccess)
    return check_launch("resident time loop: barrier reset");
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(items);
  cfg.blockDim = dim3(NTX, NTY);
  cfg.dynamicSmemBytes = rs::kSmem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const cudaError_t e = form == 1 ? cudaLaunchKernelEx(&cfg, k_wave_resident<1>, rp)
                                  : cudaLaunchKernelEx(&cfg, k_wave_resident<0>, rp);
  if (e != cudaSuccess) {
    cudaGetLastError();
    // the grid could not be made co-resident now (fewer SMs than the
    // occupancy query promised): nothing ran, the caller may step instead
    if (refused && e == cudaErrorCooperativeLaunchTooLarge) *refused = true;
    return report(FFPAT_ECUDA, "k_wave_resident launch: %s", cudaGetErrorString(e));
  }
  count_launch();
  if (result) *result = (pl.nt >= 1 && out) ? out : (pl.nt >= 1 ? rp.buf[(pl.nt - 1) & 1] : in);
  return check_launch("k_wave_resident");
}

int read_device_status(unsigned* out, bool clear) {
  unsigned v = 0;
  cudaError_t e = cudaMemcpyFromSymbol(&v, g_tma_status, sizeof v);
  if (e != cudaSuccess) return check_launch("read device status");
  if (clear && v) {
    const unsigned z = 0;
    cudaMemcpyToSymbol(g_tma_status, &z, sizeof z);
  }
  *out = v;
  return FFPAT_OK;
}

}  // namespace ffpat
