// Tile-streamed tall-skinny kernels (internal interface; see tiled.cu).
#pragma once
#include <cuda_runtime.h>

#include "kernels.h"

namespace phsvds {

// Row windows of up to four row-major blocks copied into one shared-memory
// tile row (16-byte granules).  Requirements: every block's row stride is a
// multiple of 16 bytes and its row 0 starts on a 16-byte boundary.
struct TileDesc {
  const char* base[4];  // 16-byte aligned start of the window in row 0
  long long ldB[4];     // row stride in bytes
  int g16[4];           // granules per row
  int soffw[4];         // word offset of the window inside a tile row
  int leadw[4];         // words from the window start to column 0 of the segment
  int nc[4];            // columns of the segment
  int nseg;
  int g16tot;           // granules per row (<= 64)
  int rowwords;         // words per tile row (padded)
};

bool make_tiles(const SegV* segs, int nseg, size_t esz, bool conflict_pad, TileDesc* T);

cudaError_t tiled_gram(int prec, const TileDesc& T, long long r0, long long r1, int p, int q, void* partial,
                       int max_blocks, int* nblocks, cudaStream_t st);
cudaError_t tiled_reduce(int prec, const void* partial, int nblocks, int pq, double* G, cudaStream_t st);
cudaError_t tiled_combine(int prec, const TileDesc& T, long long L, int p, const void* coef, const void* In,
                          long long ldin, int alpha_one, void* Out, long long ldout, int q, const void* Rinv,
                          void* Out2, long long ldout2, cudaStream_t st);
cudaError_t tiled_ritz(int prec, const TileDesc& T, long long L, int g, const void* Y, const void* theta, void* X,
                       void* R, long long ldb, int nb, const void* dscale, void* Tout, void* partial, int max_blocks,
                       int* nblocks, cudaStream_t st);

}  // namespace phsvds
