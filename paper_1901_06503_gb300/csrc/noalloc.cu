// noalloc.cu -- ffpat_forward_noalloc: the forward operator g = P W h for
// callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc or hand the library a workspace: code
// that runs inside an application whose memory is owned by someone else (a
// plugin or an embedded pipeline with a fixed memory budget), real-time loops
// that must never enter the allocator, or host code holding device pointers it
// received but no allocator of its own.  For them this entry point runs the
// same forward operator as ffpat_forward, with its scratch in a file-scope
// device array instead of a caller workspace, and with the time loop launched
// step by step (ffpat_forward replays repeated time loops from CUDA graphs,
// whose capture and instantiation allocate).
//
// The array is kScratchBytes (32 MiB) of device memory on every GPU where
// the library's device code is loaded, held until the process exits.  The
// array is committed when that module is loaded on a device; under CUDA's
// lazy module loading (the default) that happens during the first call on
// each device, which may therefore allocate device memory once; later calls
// allocate nothing.  Problems whose workspace (ffpat_workspace_bytes) is larger
// are rejected.  The workspace grows with the wave grid N_w = N + 2 pad:
// without padding, N <= 64 with up to 180 angles fits in every precision
// (N_w <= 64 with up to 180 angles in general).
//
// In host code the array's name is only a host-side stand-in, not a device
// address, so the first call on each device (made with that device current)
// looks up the real address with cudaGetSymbolAddress and keeps it; make that
// first call before any stream capture.  All calls on a device share the one
// array: calls that overlap on the GPU (different streams, or host threads
// without ordering) race on it and must be serialised by the caller.  The
// forward operator needs no scratch contents from an earlier call (nothing has
// to start at zero); the array keeps whatever the last call left in it.
#include <mutex>

#include "internal.cuh"

namespace ffpat {
namespace {

constexpr size_t kScratchBytes = 32u << 20;
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the static scratch on the current device (looked up once).
int scratch_address(void** out) {
  int dev = 0;
  const cudaError_t eg = cudaGetDevice(&dev);
  if (eg != cudaSuccess) {
    cudaGetLastError();
    return report(FFPAT_ECUDA, "ffpat_forward_noalloc: cudaGetDevice: %s", cudaGetErrorString(eg));
  }
  if (dev < 0 || dev >= kMaxDevices)
    return report(FFPAT_EINVAL, "ffpat_forward_noalloc: device %d >= %d (the static scratch "
                  "addresses are kept for devices 0 .. %d)", dev, kMaxDevices, kMaxDevices - 1);
  std::lock_guard<std::mutex> g(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return report(FFPAT_ECUDA, "ffpat_forward_noalloc: cudaGetSymbolAddress of the static "
                    "scratch: %s", cudaGetErrorString(e));
    }
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return FFPAT_OK;
}

}  // namespace
}  // namespace ffpat

extern "C" int ffpat_forward_noalloc(const ffpat_problem* problem, const void* c, const void* h,
                                     void* g, void* stream) {
  const size_t need = ffpat_workspace_bytes(problem);
  if (need == 0) return FFPAT_EINVAL;  // invalid problem; ffpat_last_error() says why
  if (need > ffpat::kScratchBytes)
    return ffpat::report(FFPAT_EINVAL,
                         "ffpat_forward_noalloc: the problem needs %zu bytes of scratch but the "
                         "static scratch holds %zu (a wave grid N + 2 pad <= 64 with <= 180 "
                         "angles fits every precision)",
                         need, ffpat::kScratchBytes);
  void* ws = nullptr;
  const int rc = ffpat::scratch_address(&ws);
  if (rc != FFPAT_OK) return rc;
  // launch the time loop step by step: the library's CUDA-graph replay would
  // create a capture stream and instantiate a graph, which allocate
  ffpat::NoGraphs no_graphs;
  return ffpat_forward(problem, c, h, g, ws, ffpat::kScratchBytes, stream);
}
