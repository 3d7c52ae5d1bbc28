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
// a device address (it is a host-side stand-in), so every call resolves the
// address in the current context with cudaGetSymbolAddress, which allocates
// nothing.  Resolving per call (instead of caching one address per device)
// stays correct after cudaDeviceReset or when the caller switches contexts.
// The first call in a context also loads the library's device code into it:
// make that first call before any stream capture.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "../../include/phsvds.h"
#include "../../include/phsvds_kernels.h"
#include "engine.h"
#include "kernels.h"

namespace {

// Largest shapes the static scratch serves: P^T Q with p <= 64 and q <= 8
// (the block widths of the solver).  One launch writes nblocks * p * q
// accumulators of 8 bytes; the array holds kScratchBlocks of the largest
// shape, and every launch bounds its grid by what the array holds for its own
// shape, so no grid size can write past the end.
constexpr int kMaxP = 64;
constexpr int kMaxQ = 8;
constexpr int kScratchBlocks = 152 * 4;
constexpr size_t kScratchBytes = (size_t)kScratchBlocks * kMaxP * kMaxQ * 8;  // 2,490,368 bytes

static __device__ __align__(256) unsigned char g_gram_scratch[kScratchBytes];

// Device address of the scratch array in the current context.
cudaError_t scratch_address(void** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_gram_scratch);
  if (e != cudaSuccess) return e;
  *out = p;
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
  // the grid is bounded by the blocks whose partials fit the array
  const int fit = (int)(kScratchBytes / gram_partial_bytes(1, p, q));
  const int max_blocks = std::min(gram_default_blocks(), fit);
  int nb = 0;
  // every CTA overwrites all of its p * q partials, so nothing needs clearing
  e = launch_gram(prec, r0, r1, &Ps, 1, Qs, scratch, max_blocks, &nb, st);
  if (e == cudaSuccess) e = launch_gram_reduce(prec, scratch, nb, p * q, G, st);
  if (e != cudaSuccess) {
    set_last_error(std::string(cudaGetErrorString(e)) + " in phsvds_gram_noalloc");
    cudaGetLastError();
    return SVDS_ERR_CUDA;
  }
  return SVDS_OK;
}
