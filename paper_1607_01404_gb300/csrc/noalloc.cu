// Allocation-free variant of the Gram entry point (phsvds_gram_noalloc).
//
// Some callers cannot call cudaMalloc or any allocating routine: code running
// inside a host callback or a custom allocator hook, plug-ins that must not
// touch the device heap of their host application, and drivers that budget
// every device allocation up front.  For them this entry point takes its
// scratch (the per-CTA partial sums of the Gram reduction) from a file-scope
// device array of fixed size instead of a caller-provided buffer.
//
// The array lives in this translation unit; every GPU that loads the library
// holds it until the process exits.  Host code cannot use the array's name as
// a device address (it is a host-side stand-in), so the first call on each
// device, with that device current, resolves the address with
// cudaGetSymbolAddress and caches it.  Make that first call before any stream
// capture.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/phsvds.h"
#include "../../include/phsvds_kernels.h"
#include "engine.h"
#include "kernels.h"

namespace {

// Largest shapes the static scratch serves: P^T Q with p <= 64 and q <= 8
// (the block widths of the solver); the partials of one launch take
// gram_default_blocks() * p * q * 8 bytes = 608 * 64 * 8 * 8 = 2,490,368 bytes.
constexpr int kMaxP = 64;
constexpr int kMaxQ = 8;
constexpr size_t kScratchBytes = (size_t)152 * 4 * kMaxP * kMaxQ * 8;

static __device__ __align__(256) unsigned char g_gram_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (set-up on first use).
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_gram_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" int phsvds_gram_noalloc(int prec, int64_t r0, int64_t r1, const void* P, int64_t ldp, int p, const void* Q,
                                   int64_t ldq, int q, double* G, void* stream) {
  using namespace phsvds;
  if (prec != kF32 && prec != kDF64 && prec != kF64) return SVDS_ERR_ARG;
  if (p < 1 || q < 1 || r0 < 0 || r1 < r0 || !P || !Q || !G || ldp < p || ldq < q) return SVDS_ERR_ARG;
  if (p > kMaxP || q > kMaxQ) {
    set_last_error("phsvds_gram_noalloc: p <= 64 and q <= 8 are the largest shapes its static scratch serves");
    return SVDS_ERR_ARG;
  }
  void* scratch = nullptr;
  cudaError_t e = scratch_address(&scratch);
  if (e != cudaSuccess) {
    set_last_error(std::string(cudaGetErrorString(e)) + " at cudaGetSymbolAddress");
    cudaGetLastError();
    return SVDS_ERR_CUDA;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  SegV Ps{P, ldp, p};
  SegV Qs{Q, ldq, q};
  int nb = 0;
  // every CTA overwrites all of its p * q partials, so nothing needs clearing
  e = launch_gram(prec, r0, r1, &Ps, 1, Qs, scratch, gram_default_blocks(), &nb, st);
  if (e == cudaSuccess) e = launch_gram_reduce(prec, scratch, nb, p * q, G, st);
  if (e != cudaSuccess) {
    set_last_error(std::string(cudaGetErrorString(e)) + " in phsvds_gram_noalloc");
    cudaGetLastError();
    return SVDS_ERR_CUDA;
  }
  return SVDS_OK;
}
