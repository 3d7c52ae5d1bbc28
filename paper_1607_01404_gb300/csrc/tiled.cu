// Tile-streamed tall-skinny kernels (sm_103a): Gram (P^T Q), combine
// (alpha In + P C, then * R^-1) and the fused Ritz-vector / residual / norm
// kernel.  These are the dense O((m+n) g) operations of the paper's Table 3
// ("MV, MM, inner products") and the residual kernel of Sec. 3.3.
//
// Each CTA of a persistent grid streams row tiles of the operand blocks into
// shared memory with 16-byte cp.async copies, double buffered so that the next
// tile is in flight while the current one is consumed.  Row windows of the
// row-major blocks are copied at 16-byte granularity (the window is widened to
// 16-byte boundaries inside its row), so a tile costs exactly the bytes the
// computation needs up to that rounding.
//
// The Gram accumulators are FP64-class in every mode: in the F32 mode the
// products are exact as double-floats (TwoProd) and are accumulated with
// TwoSum into a hi/lo pair whose low part collects the rounding errors (the
// compensated dot product of Ogita, Rump and Oishi, "Accurate sum and dot
// product", 2005), renormalised once per tile; the DF64 mode adds the cross
// terms of the double-float product.  The cross-CTA reduction sums per-CTA
// partials in a fixed order, so results are deterministic.
#include <cuda_runtime.h>

#include <cstdint>

#include "common.cuh"
#include "kernels.h"
#include "tiled.h"

namespace phsvds {

namespace {

constexpr int kT = 256;     // threads per CTA
constexpr int kRows = 64;   // rows per tile

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void cp_async16(unsigned dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// element read from a shared-memory tile (word index must be element aligned)
template <class P>
__device__ __forceinline__ typename P::A lds(const float* sm, int w);
template <>
__device__ __forceinline__ float lds<PF32>(const float* sm, int w) {
  return sm[w];
}
template <>
__device__ __forceinline__ df lds<PDF64>(const float* sm, int w) {
  const float2 v = *reinterpret_cast<const float2*>(sm + w);
  return {v.x, v.y};
}
template <>
__device__ __forceinline__ double lds<PF64>(const float* sm, int w) {
  return *reinterpret_cast<const double*>(sm + w);
}

template <class P>
__host__ __device__ constexpr int ew() {
  return P::id == kF32 ? 1 : 2;  // words per element
}

// Per-thread description of the granules it copies in each tile row.
struct LaneGran {
  int seg[2], gk[2], n;
};

__device__ __forceinline__ LaneGran lane_grans(const TileDesc& T, int lane) {
  LaneGran lg;
  lg.n = 0;
  for (int it = 0; it < 2; ++it) {
    int k = lane + 32 * it;
    if (k >= T.g16tot) break;
    int s = 0;
    while (k >= T.g16[s]) {
      k -= T.g16[s];
      ++s;
    }
    lg.seg[lg.n] = s;
    lg.gk[lg.n] = k;
    ++lg.n;
  }
  return lg;
}

__device__ __forceinline__ void tile_load(const TileDesc& T, const LaneGran& lg, long long row0, int nrows, float* buf,
                                          int warp, int nwarps) {
  // granule sources/destinations of this lane resolved once (no dynamic indexing in the loop)
  const char* b0 = lg.n > 0 ? T.base[lg.seg[0]] + lg.gk[0] * 16 : nullptr;
  const char* b1 = lg.n > 1 ? T.base[lg.seg[1]] + lg.gk[1] * 16 : nullptr;
  const long long l0 = lg.n > 0 ? T.ldB[lg.seg[0]] : 0, l1 = lg.n > 1 ? T.ldB[lg.seg[1]] : 0;
  const int d0 = lg.n > 0 ? T.soffw[lg.seg[0]] + lg.gk[0] * 4 : 0, d1 = lg.n > 1 ? T.soffw[lg.seg[1]] + lg.gk[1] * 4 : 0;
  for (int r = warp; r < nrows; r += nwarps) {
    if (lg.n > 0) cp_async16(smem_u32(buf + r * T.rowwords + d0), b0 + (row0 + r) * l0);
    if (lg.n > 1) cp_async16(smem_u32(buf + r * T.rowwords + d1), b1 + (row0 + r) * l1);
  }
}

// Dot2-style accumulation: hi + lo, lo collects the TwoSum errors.
template <class P>
struct GAcc;
template <>
struct GAcc<PF32> {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float x, float y) {
    const df p = two_prod(x, y);
    const df s = two_sum(hi, p.hi);
    hi = s.hi;
    lo = __fadd_rn(lo, __fadd_rn(s.lo, p.lo));
  }
  __device__ __forceinline__ void norm() {
    const df s = fast_two_sum(hi, lo);
    hi = s.hi;
    lo = s.lo;
  }
  __device__ __forceinline__ df get() const { return fast_two_sum(hi, lo); }
};
template <>
struct GAcc<PDF64> {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(df x, df y) {
    const df p = two_prod(x.hi, y.hi);
    const float pl = __fmaf_rn(x.hi, y.lo, __fmaf_rn(x.lo, y.hi, p.lo));
    const df s = two_sum(hi, p.hi);
    hi = s.hi;
    lo = __fadd_rn(lo, __fadd_rn(s.lo, pl));
  }
  __device__ __forceinline__ void norm() {
    const df s = fast_two_sum(hi, lo);
    hi = s.hi;
    lo = s.lo;
  }
  __device__ __forceinline__ df get() const { return fast_two_sum(hi, lo); }
};
template <>
struct GAcc<PF64> {
  double v = 0.0;
  __device__ __forceinline__ void add(double x, double y) { v = fma(x, y, v); }
  __device__ __forceinline__ void norm() {}
  __device__ __forceinline__ double get() const { return v; }
};

// ---------------------------------------------------------------------------
// Gram: partial[blk][i][j] = sum_r P[r, i] Q[r, j]; segments 0..nseg-2 form P,
// the last segment is Q.
// ---------------------------------------------------------------------------
template <class P, int NQ>
__global__ void __launch_bounds__(kT) k_gram_t(TileDesc T, long long r0, long long r1, int p, int q,
                                               typename P::G* __restrict__ partial) {
  using G = typename P::G;
  extern __shared__ __align__(16) float sm[];
  float* buf0 = sm;
  float* buf1 = sm + kRows * T.rowwords;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = kT / 32;
  const LaneGran lg = lane_grans(T, lane);
  const int NG = kT / p;
  const int i = tid % p, rg = tid / p;
  const bool active = rg < NG;
  // smem word offset of column i of P and of column 0 of Q
  int ci = i, s = 0;
  while (s < T.nseg - 2 && ci >= T.nc[s]) {
    ci -= T.nc[s];
    ++s;
  }
  const int offi = T.soffw[s] + T.leadw[s] + ci * ew<P>();
  const int qs = T.nseg - 1;
  const int offq = T.soffw[qs] + T.leadw[qs];
  GAcc<P> acc[NQ];
  const long long ntiles = (r1 - r0 + kRows - 1) / kRows;
  long long t = blockIdx.x;
  if (t < ntiles) tile_load(T, lg, r0 + t * kRows, (int)min((long long)kRows, r1 - r0 - t * kRows), buf0, warp, nwarps);
  cp_commit();
  for (int it = 0; t < ntiles; t += gridDim.x, ++it) {
    const long long tn = t + gridDim.x;
    float* cur = (it & 1) ? buf1 : buf0;
    float* nxt = (it & 1) ? buf0 : buf1;
    if (tn < ntiles) tile_load(T, lg, r0 + tn * kRows, (int)min((long long)kRows, r1 - r0 - tn * kRows), nxt, warp, nwarps);
    cp_commit();
    cp_wait1();
    __syncthreads();
    const int nrows = (int)min((long long)kRows, r1 - r0 - t * kRows);
    if (active) {
      for (int r = rg; r < nrows; r += NG) {
        const float* row = cur + r * T.rowwords;
        const auto x = lds<P>(row, offi);
#pragma unroll
        for (int j = 0; j < NQ; ++j)
          if (j < q) acc[j].add(x, lds<P>(row, offq + j * ew<P>()));
      }
#pragma unroll
      for (int j = 0; j < NQ; ++j) acc[j].norm();
    }
    __syncthreads();
  }
  cp_wait0();
  __syncthreads();
  // reduce over the row groups in a fixed order (reusing the tile buffers)
  G* red = reinterpret_cast<G*>(sm);
  if (active)
#pragma unroll
    for (int j = 0; j < NQ; ++j)
      if (j < q) red[(rg * p + i) * q + j] = acc[j].get();
  __syncthreads();
  const int pq = p * q;
  for (int e = tid; e < pq; e += kT) {
    G v = red[e];
    for (int g = 1; g < NG; ++g) v = P::gadd(v, red[g * pq + e]);
    partial[(long long)blockIdx.x * pq + e] = v;
  }
}

// ---------------------------------------------------------------------------
// Combine: Out = alpha In + P coef, optionally Out <- Out Rinv.
// ---------------------------------------------------------------------------
template <class P>
__global__ void __launch_bounds__(kT) k_combine_t(TileDesc T, long long L, int p, const typename P::C* __restrict__ coef,
                                                  const typename P::S* In, long long ldin, int alpha_one,
                                                  typename P::S* Out, long long ldout, int q,
                                                  const typename P::C* __restrict__ Rinv, typename P::S* Out2,
                                                  long long ldout2) {
  using A = typename P::A;
  using C = typename P::C;
  extern __shared__ __align__(16) float sm[];
  float* buf0 = sm;
  float* buf1 = sm + kRows * T.rowwords;
  C* Cs = reinterpret_cast<C*>(buf1 + kRows * T.rowwords);
  C* Rs = Cs + p * q;
  A* Os = reinterpret_cast<A*>(Rs + (Rinv ? q * q : 0));
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = kT / 32;
  for (int e = tid; e < p * q; e += kT) Cs[e] = coef[e];
  if (Rinv)
    for (int e = tid; e < q * q; e += kT) Rs[e] = Rinv[e];
  const LaneGran lg = lane_grans(T, lane);
  const int r = tid >> 2, jg = tid & 3;
  const long long ntiles = (L + kRows - 1) / kRows;
  long long t = blockIdx.x;
  if (t < ntiles) tile_load(T, lg, t * kRows, (int)min((long long)kRows, L - t * kRows), buf0, warp, nwarps);
  cp_commit();
  for (int it = 0; t < ntiles; t += gridDim.x, ++it) {
    const long long tn = t + gridDim.x;
    float* cur = (it & 1) ? buf1 : buf0;
    float* nxt = (it & 1) ? buf0 : buf1;
    if (tn < ntiles) tile_load(T, lg, tn * kRows, (int)min((long long)kRows, L - tn * kRows), nxt, warp, nwarps);
    cp_commit();
    cp_wait1();
    __syncthreads();
    const int nrows = (int)min((long long)kRows, L - t * kRows);
    const long long grow = t * kRows + r;
    if (r < nrows) {
      const float* row = cur + r * T.rowwords;
      for (int j = jg; j < q; j += 4) {
        A acc = alpha_one ? P::load(In + grow * ldin + j) : P::zero();
        int c = 0;
        for (int s = 0; s < T.nseg; ++s) {
          const int base = T.soffw[s] + T.leadw[s];
          for (int cc = 0; cc < T.nc[s]; ++cc, ++c) acc = P::fmac(acc, lds<P>(row, base + cc * ew<P>()), Cs[c * q + j]);
        }
        if (Rinv) {
          Os[r * q + j] = acc;
        } else {
          P::store(Out + grow * ldout + j, acc);
          if (Out2) P::store(Out2 + grow * ldout2 + j, acc);
        }
      }
    }
    if (Rinv) {
      __syncthreads();
      if (r < nrows) {
        for (int j = jg; j < q; j += 4) {
          A acc = P::zero();
          for (int l = 0; l <= j; ++l) acc = P::fmac(acc, Os[r * q + l], Rs[l * q + j]);
          P::store(Out + grow * ldout + j, acc);
          if (Out2) P::store(Out2 + grow * ldout2 + j, acc);
        }
      }
    }
    __syncthreads();
  }
  cp_wait0();
}

// ---------------------------------------------------------------------------
// Fused Ritz vectors / residuals / norms: X = V Y, R = W Y - X diag(theta),
// optional T = diag(dscale) R, per-CTA partial sums of R^2 per column.
// Segment 0 is the V window, segment 1 the W window (g columns each).
// ---------------------------------------------------------------------------
template <class P>
__global__ void __launch_bounds__(kT) k_ritz_t(TileDesc T, long long L, int g, const typename P::C* __restrict__ Y,
                                               const typename P::C* __restrict__ theta, typename P::S* X,
                                               typename P::S* R, long long ldb, int nb,
                                               const typename P::S* __restrict__ dscale, typename P::S* Tout,
                                               typename P::G* __restrict__ partial) {
  using A = typename P::A;
  using C = typename P::C;
  using G = typename P::G;
  extern __shared__ __align__(16) float sm[];
  float* buf0 = sm;
  float* buf1 = sm + kRows * T.rowwords;
  C* Ys = reinterpret_cast<C*>(buf1 + kRows * T.rowwords);
  C* Th = Ys + g * nb;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = kT / 32;
  for (int e = tid; e < g * nb; e += kT) Ys[e] = Y[e];
  for (int e = tid; e < nb; e += kT) Th[e] = theta[e];
  const LaneGran lg = lane_grans(T, lane);
  const int r = tid >> 2, jg = tid & 3;
  const int vb = T.soffw[0] + T.leadw[0], wb = T.soffw[1] + T.leadw[1];
  G nacc[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) nacc[a] = P::gzero();
  const long long ntiles = (L + kRows - 1) / kRows;
  long long t = blockIdx.x;
  if (t < ntiles) tile_load(T, lg, t * kRows, (int)min((long long)kRows, L - t * kRows), buf0, warp, nwarps);
  cp_commit();
  for (int it = 0; t < ntiles; t += gridDim.x, ++it) {
    const long long tn = t + gridDim.x;
    float* cur = (it & 1) ? buf1 : buf0;
    float* nxt = (it & 1) ? buf0 : buf1;
    if (tn < ntiles) tile_load(T, lg, tn * kRows, (int)min((long long)kRows, L - tn * kRows), nxt, warp, nwarps);
    cp_commit();
    cp_wait1();
    __syncthreads();
    const int nrows = (int)min((long long)kRows, L - t * kRows);
    if (r < nrows) {
      const float* row = cur + r * T.rowwords;
      const long long grow = t * kRows + r;
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const int j = jg + 4 * a;
        if (j >= nb) break;
        A x = P::zero(), w = P::zero();
        for (int c = 0; c < g; ++c) {
          const C y = Ys[c * nb + j];
          x = P::fmac(x, lds<P>(row, vb + c * ew<P>()), y);
          w = P::fmac(w, lds<P>(row, wb + c * ew<P>()), y);
        }
        const A res = P::sub(w, P::mulc(x, Th[j]));
        P::store(X + grow * ldb + j, x);
        P::store(R + grow * ldb + j, res);
        if (Tout) P::store(Tout + grow * ldb + j, P::mulc(res, P::load(dscale + grow)));
        nacc[a] = P::gfma(nacc[a], res, res);
      }
    }
    __syncthreads();
  }
  cp_wait0();
  __syncthreads();
  // fixed-order reduction of the 64 row threads of each column
  G* red = reinterpret_cast<G*>(sm);
#pragma unroll
  for (int a = 0; a < 4; ++a) red[(a * 4 + jg) * kRows + r] = nacc[a];
  __syncthreads();
  for (int j = tid; j < nb; j += kT) {
    const int a = j / 4, jj = j % 4;
    G v = red[(a * 4 + jj) * kRows];
    for (int rr = 1; rr < kRows; ++rr) v = P::gadd(v, red[(a * 4 + jj) * kRows + rr]);
    partial[(long long)blockIdx.x * nb + j] = v;
  }
}

// Fixed-order parallel reduction of per-CTA partials: one CTA per output.
template <class P>
__global__ void __launch_bounds__(128) k_reduce_t(const typename P::G* __restrict__ partial, int nblocks, int pq,
                                                  double* __restrict__ G) {
  using GT = typename P::G;
  __shared__ GT red[128];
  const int e = blockIdx.x;
  GT v = P::gzero();
  for (int b = threadIdx.x; b < nblocks; b += 128) v = P::gadd(v, partial[(long long)b * pq + e]);
  red[threadIdx.x] = v;
  __syncthreads();
  for (int w = 64; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] = P::gadd(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) G[e] = P::gval(red[0]);
}

// ===========================================================================
// Register-blocked variants.  Preconditions (checked on the host): every P
// segment window starts on a 16-byte boundary (lead 0), so each 16-byte
// granule holds whole elements of one segment.
// ===========================================================================

template <class P>
__host__ __device__ constexpr int epg() {
  return P::id == kF32 ? 4 : 2;  // elements per 16-byte granule
}

// Elements of one 16-byte shared-memory granule.
template <class P>
__device__ __forceinline__ void unpack(const float4 v, typename P::A (&e)[epg<P>()]);
template <>
__device__ __forceinline__ void unpack<PF32>(const float4 v, float (&e)[4]) {
  e[0] = v.x;
  e[1] = v.y;
  e[2] = v.z;
  e[3] = v.w;
}
template <>
__device__ __forceinline__ void unpack<PDF64>(const float4 v, df (&e)[2]) {
  e[0] = df{v.x, v.y};
  e[1] = df{v.z, v.w};
}
template <>
__device__ __forceinline__ void unpack<PF64>(const float4 v, double (&e)[2]) {
  e[0] = __hiloint2double(__float_as_int(v.y), __float_as_int(v.x));
  e[1] = __hiloint2double(__float_as_int(v.w), __float_as_int(v.z));
}

// Tile load with the granule index of each row XOR-swizzled by (row & 7):
// reading one granule per thread for 8 consecutive rows touches 8 distinct
// 16-byte bank groups.  RG = granules per tile row (a multiple of 8).
__device__ __forceinline__ void tile_load_swz(const TileDesc& T, const LaneGran& lg, int RG, long long row0, int nrows,
                                              float* buf, int warp, int nwarps, int lane) {
  const char* b0 = lg.n > 0 ? T.base[lg.seg[0]] + lg.gk[0] * 16 : nullptr;
  const char* b1 = lg.n > 1 ? T.base[lg.seg[1]] + lg.gk[1] * 16 : nullptr;
  const long long l0 = lg.n > 0 ? T.ldB[lg.seg[0]] : 0, l1 = lg.n > 1 ? T.ldB[lg.seg[1]] : 0;
  for (int r = warp; r < nrows; r += nwarps) {
    if (lg.n > 0) cp_async16(smem_u32(buf + (r * RG + (lane ^ (r & 7))) * 4), b0 + (row0 + r) * l0);
    if (lg.n > 1) cp_async16(smem_u32(buf + (r * RG + ((lane + 32) ^ (r & 7))) * 4), b1 + (row0 + r) * l1);
  }
}

__device__ __forceinline__ float4 lds4_swz(const float* buf, int RG, int r, int k) {
  return *reinterpret_cast<const float4*>(buf + (r * RG + (k ^ (r & 7))) * 4);
}

template <int N>
__device__ __forceinline__ void cp_wait_n() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Gram, each thread owns the elements of one granule of P (4 F32 or 2 wider
// columns) for all NQ columns of Q.  S-stage cp.async pipeline.
template <class P, int NQ, int S>
__global__ void __launch_bounds__(kT) k_gram_b(TileDesc T, long long r0, long long r1, int p, int q,
                                               typename P::G* __restrict__ partial) {
  using G = typename P::G;
  using A = typename P::A;
  constexpr int E = epg<P>();
  extern __shared__ __align__(16) float sm[];
  const int tw = kRows * T.rowwords;  // words per stage
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = kT / 32;
  const LaneGran lg = lane_grans(T, lane);
  const int npseg = T.nseg - 1;
  int TPR = 0;
  for (int s = 0; s < npseg; ++s) TPR += T.g16[s];
  const int NG = kT / TPR;
  const int cb = tid % TPR, rg = tid / TPR;
  const bool active = rg < NG;
  int s = 0, kk = cb, c0 = 0;
  while (s < npseg - 1 && kk >= T.g16[s]) {
    kk -= T.g16[s];
    c0 += T.nc[s];
    ++s;
  }
  const int goff = T.soffw[s] + kk * 4;
  const int col0 = c0 + kk * E;
  const int nvalid = min(E, T.nc[s] - kk * E);
  const int qs = T.nseg - 1;
  const int offq = T.soffw[qs] + T.leadw[qs];
  GAcc<P> acc[E][NQ];
  const long long ntiles = (r1 - r0 + kRows - 1) / kRows;
  const long long t0 = blockIdx.x, step = gridDim.x;
#pragma unroll
  for (int i = 0; i < S - 1; ++i) {
    const long long ti = t0 + i * step;
    if (ti < ntiles) tile_load(T, lg, r0 + ti * kRows, (int)min((long long)kRows, r1 - r0 - ti * kRows), sm + i * tw, warp, nwarps);
    cp_commit();
  }
  for (int it = 0;; ++it) {
    const long long t = t0 + it * step;
    if (t >= ntiles) break;
    cp_wait_n<S - 2>();
    __syncthreads();
    {
      const long long tl = t0 + (it + S - 1) * step;
      if (tl < ntiles)
        tile_load(T, lg, r0 + tl * kRows, (int)min((long long)kRows, r1 - r0 - tl * kRows), sm + ((it + S - 1) % S) * tw,
                  warp, nwarps);
      cp_commit();
    }
    const float* cur = sm + (it % S) * tw;
    const int nrows = (int)min((long long)kRows, r1 - r0 - t * kRows);
    if (active) {
      for (int r = rg; r < nrows; r += NG) {
        const float* row = cur + r * T.rowwords;
        A e[E];
        unpack<P>(*reinterpret_cast<const float4*>(row + goff), e);
        A y[NQ];
#pragma unroll
        for (int j = 0; j < NQ; ++j) y[j] = j < q ? lds<P>(row, offq + j * ew<P>()) : P::zero();
#pragma unroll
        for (int u = 0; u < E; ++u)
#pragma unroll
          for (int j = 0; j < NQ; ++j) acc[u][j].add(e[u], y[j]);
      }
#pragma unroll
      for (int u = 0; u < E; ++u)
#pragma unroll
        for (int j = 0; j < NQ; ++j) acc[u][j].norm();
    }
  }
  cp_wait0();
  __syncthreads();
  G* red = reinterpret_cast<G*>(sm);
  if (active)
    for (int u = 0; u < nvalid; ++u)
#pragma unroll
      for (int j = 0; j < NQ; ++j)
        if (j < q) red[(rg * p + col0 + u) * q + j] = acc[u][j].get();
  __syncthreads();
  const int pq = p * q;
  for (int e = tid; e < pq; e += kT) {
    G v = red[e];
    for (int g = 1; g < NG; ++g) v = P::gadd(v, red[g * pq + e]);
    partial[(long long)blockIdx.x * pq + e] = v;
  }
}

constexpr int kRowThreads = 128;

// Combine: TPR threads per row, each produces the output columns j = sub, sub +
// TPR, ... (TPR == 1 when Rinv is fused, which needs all outputs of a row).
template <class P, int NQ, int TPR, int S>
__global__ void __launch_bounds__(kRowThreads) k_combine_rows(TileDesc T, int RG, long long L, int p,
                                                              const typename P::C* __restrict__ coef,
                                                              const typename P::S* In, long long ldin, int alpha_one,
                                                              typename P::S* Out, long long ldout, int q,
                                                              const typename P::C* __restrict__ Rinv,
                                                              typename P::S* Out2, long long ldout2) {
  using A = typename P::A;
  using C = typename P::C;
  constexpr int E = epg<P>();
  constexpr int RT = kRowThreads / TPR;
  extern __shared__ __align__(16) float sm[];
  const int tw = RT * RG * 4;
  C* Cs = reinterpret_cast<C*>(sm + S * tw);
  C* Rs = Cs + p * q;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = kRowThreads / 32;
  for (int e = tid; e < p * q; e += kRowThreads) Cs[e] = coef[e];
  if (Rinv)
    for (int e = tid; e < q * q; e += kRowThreads) Rs[e] = Rinv[e];
  const LaneGran lg = lane_grans(T, lane);
  const int r = tid / TPR, sub = tid % TPR;
  const long long ntiles = (L + RT - 1) / RT;
  const long long t0 = blockIdx.x, step = gridDim.x;
#pragma unroll
  for (int i = 0; i < S - 1; ++i) {
    const long long ti = t0 + i * step;
    if (ti < ntiles) tile_load_swz(T, lg, RG, ti * RT, (int)min((long long)RT, L - ti * RT), sm + i * tw, warp, nwarps, lane);
    cp_commit();
  }
  for (int it = 0;; ++it) {
    const long long t = t0 + it * step;
    if (t >= ntiles) break;
    cp_wait_n<S - 2>();
    __syncthreads();
    {
      const long long tl = t0 + (it + S - 1) * step;
      if (tl < ntiles)
        tile_load_swz(T, lg, RG, tl * RT, (int)min((long long)RT, L - tl * RT), sm + ((it + S - 1) % S) * tw, warp,
                      nwarps, lane);
      cp_commit();
    }
    const float* cur = sm + (it % S) * tw;
    const int nrows = (int)min((long long)RT, L - t * RT);
    if (r < nrows) {
      const long long grow = t * RT + r;
      for (int jc = sub; jc < q; jc += NQ * TPR) {
        // outputs jc, jc + TPR, ..., jc + (NQ - 1) TPR
        A acc[NQ];
#pragma unroll
        for (int u = 0; u < NQ; ++u) {
          const int j = jc + u * TPR;
          acc[u] = (alpha_one && j < q) ? P::load(In + grow * ldin + j) : P::zero();
        }
        int c = 0, k = 0;
        for (int s = 0; s < T.nseg; ++s) {
          const int ns = T.nc[s];
          for (int kk = 0; kk < T.g16[s]; ++kk, ++k) {
            A e[E];
            unpack<P>(lds4_swz(cur, RG, r, k), e);
#pragma unroll
            for (int v = 0; v < E; ++v) {
              const int cc = kk * E + v;
              if (cc < ns) {
                const C* cr = Cs + (c + cc) * q + jc;
#pragma unroll
                for (int u = 0; u < NQ; ++u)
                  if (jc + u * TPR < q) acc[u] = P::fmac(acc[u], e[v], cr[u * TPR]);
              }
            }
          }
          c += ns;
        }
        if (TPR == 1 && Rinv) {
          A out[NQ];
#pragma unroll
          for (int j = 0; j < NQ; ++j) {
            out[j] = P::zero();
#pragma unroll
            for (int l = 0; l <= j; ++l)
              if (j < q) out[j] = P::fmac(out[j], acc[l], Rs[l * q + j]);
          }
#pragma unroll
          for (int j = 0; j < NQ; ++j) acc[j] = out[j];
        }
#pragma unroll
        for (int u = 0; u < NQ; ++u) {
          const int j = jc + u * TPR;
          if (j < q) {
            P::store(Out + grow * ldout + j, acc[u]);
            if (Out2) P::store(Out2 + grow * ldout2 + j, acc[u]);
          }
        }
      }
    }
  }
  cp_wait0();
}

// Fused Ritz vectors / residuals / norms: TPR threads per row, output column
// j handled by thread sub = j % TPR (segment 0 = V window, 1 = W window).
template <class P, int NB, int TPR, int S>
__global__ void __launch_bounds__(kRowThreads) k_ritz_rows(TileDesc T, int RG, long long L, int g,
                                                           const typename P::C* __restrict__ Y,
                                                           const typename P::C* __restrict__ theta, typename P::S* X,
                                                           typename P::S* R, long long ldb, int nb,
                                                           const typename P::S* __restrict__ dscale,
                                                           typename P::S* Tout, typename P::G* __restrict__ partial) {
  using A = typename P::A;
  using C = typename P::C;
  using G = typename P::G;
  constexpr int E = epg<P>();
  constexpr int RT = kRowThreads / TPR;
  constexpr int NJ = NB / TPR;  // outputs per thread
  extern __shared__ __align__(16) float sm[];
  const int tw = RT * RG * 4;
  C* Ys = reinterpret_cast<C*>(sm + S * tw);
  C* Th = Ys + g * nb;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = kRowThreads / 32;
  for (int e = tid; e < g * nb; e += kRowThreads) Ys[e] = Y[e];
  for (int e = tid; e < nb; e += kRowThreads) Th[e] = theta[e];
  const LaneGran lg = lane_grans(T, lane);
  const int r = tid / TPR, sub = tid % TPR;
  G nacc[NJ];
#pragma unroll
  for (int u = 0; u < NJ; ++u) nacc[u] = P::gzero();
  const long long ntiles = (L + RT - 1) / RT;
  const long long t0 = blockIdx.x, step = gridDim.x;
  const int gv = T.g16[0];
#pragma unroll
  for (int i = 0; i < S - 1; ++i) {
    const long long ti = t0 + i * step;
    if (ti < ntiles) tile_load_swz(T, lg, RG, ti * RT, (int)min((long long)RT, L - ti * RT), sm + i * tw, warp, nwarps, lane);
    cp_commit();
  }
  for (int it = 0;; ++it) {
    const long long t = t0 + it * step;
    if (t >= ntiles) break;
    cp_wait_n<S - 2>();
    __syncthreads();
    {
      const long long tl = t0 + (it + S - 1) * step;
      if (tl < ntiles)
        tile_load_swz(T, lg, RG, tl * RT, (int)min((long long)RT, L - tl * RT), sm + ((it + S - 1) % S) * tw, warp,
                      nwarps, lane);
      cp_commit();
    }
    const float* cur = sm + (it % S) * tw;
    const int nrows = (int)min((long long)RT, L - t * RT);
    if (r < nrows) {
      const long long grow = t * RT + r;
      A x[NJ], w[NJ];
#pragma unroll
      for (int u = 0; u < NJ; ++u) x[u] = w[u] = P::zero();
      for (int kk = 0; kk < gv; ++kk) {
        A ev[E], eW[E];
        unpack<P>(lds4_swz(cur, RG, r, kk), ev);
        unpack<P>(lds4_swz(cur, RG, r, gv + kk), eW);
#pragma unroll
        for (int v = 0; v < E; ++v) {
          const int c = kk * E + v;
          if (c < g) {
            const C* yr = Ys + c * nb + sub;
#pragma unroll
            for (int u = 0; u < NJ; ++u)
              if (sub + u * TPR < nb) {
                x[u] = P::fmac(x[u], ev[v], yr[u * TPR]);
                w[u] = P::fmac(w[u], eW[v], yr[u * TPR]);
              }
          }
        }
      }
      const A ds = Tout ? P::load(dscale + grow) : P::zero();
#pragma unroll
      for (int u = 0; u < NJ; ++u) {
        const int j = sub + u * TPR;
        if (j < nb) {
          const A res = P::sub(w[u], P::mulc(x[u], Th[j]));
          P::store(X + grow * ldb + j, x[u]);
          P::store(R + grow * ldb + j, res);
          if (Tout) P::store(Tout + grow * ldb + j, P::mulc(res, ds));
          nacc[u] = P::gfma(nacc[u], res, res);
        }
      }
    }
  }
  cp_wait0();
  __syncthreads();
  G* red = reinterpret_cast<G*>(sm);
  // red[j][row]: fixed-order sum over the rows of the tile grid
#pragma unroll
  for (int u = 0; u < NJ; ++u) {
    const int j = sub + u * TPR;
    if (j < nb) red[j * RT + r] = nacc[u];
  }
  __syncthreads();
  for (int j = tid; j < nb; j += kRowThreads) {
    G v = red[j * RT];
    for (int rr = 1; rr < RT; ++rr) v = P::gadd(v, red[j * RT + rr]);
    partial[(long long)blockIdx.x * nb + j] = v;
  }
}

int g_blocks_per_sm = 4;

}  // namespace

bool make_tiles(const SegV* segs, int nseg, size_t esz, bool conflict_pad, TileDesc* T) {
  if (nseg < 1 || nseg > 4) return false;
  int words = 0;
  for (int s = 0; s < nseg; ++s) {
    const uintptr_t a = reinterpret_cast<uintptr_t>(segs[s].p);
    if ((segs[s].ld * (long long)esz) % 16 != 0 || segs[s].nc < 1) return false;
    const int mis = (int)(a % 16);
    if (mis % esz != 0) return false;
    T->base[s] = reinterpret_cast<const char*>(a - mis);
    T->ldB[s] = segs[s].ld * (long long)esz;
    const int wb = mis + segs[s].nc * (int)esz;
    T->g16[s] = (wb + 15) / 16;
    T->soffw[s] = words;
    T->leadw[s] = mis / 4;
    T->nc[s] = segs[s].nc;
    words += T->g16[s] * 4;
  }
  T->nseg = nseg;
  T->g16tot = words / 4;
  if (T->g16tot > 64) return false;
  if (conflict_pad) words = ((words + 27) / 32) * 32 + 4;  // rows land on distinct bank groups
  T->rowwords = words;
  return true;
}

int tiled_grid(long long ntiles) {
  long long g = ntiles;
  const long long cap = 152LL * g_blocks_per_sm;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

template <class P>
static cudaError_t gram_tp(const TileDesc& T, long long r0, long long r1, int p, int q, void* partial, int max_blocks,
                           int* nblocks, cudaStream_t st) {
  const long long ntiles = (r1 - r0 + kRows - 1) / kRows;
  int grid = tiled_grid(ntiles);
  if (grid > max_blocks) grid = max_blocks;
  *nblocks = grid;
  const int NG = kT / p;
  size_t smem = sizeof(float) * 2 * kRows * T.rowwords;
  const size_t red = sizeof(typename P::G) * (size_t)NG * p * q;
  if (red > smem) smem = red;
  using G = typename P::G;
  G* out = reinterpret_cast<G*>(partial);
#define GRAM_LAUNCH(NQv, idx)                                                               \
  do {                                                                                   \
    const cudaError_t e_ = smem_optin(reinterpret_cast<const void*>(k_gram_t<P, NQv>), 200 * 1024); \
    if (e_ != cudaSuccess) return e_;                                                   \
    k_gram_t<P, NQv><<<grid, kT, smem, st>>>(T, r0, r1, p, q, out);                               \
  } while (0)
  if (q <= 1)
    GRAM_LAUNCH(1, 0);
  else if (q <= 2)
    GRAM_LAUNCH(2, 1);
  else if (q <= 4)
    GRAM_LAUNCH(4, 2);
  else
    GRAM_LAUNCH(8, 3);
#undef GRAM_LAUNCH
  return cudaGetLastError();
}

static bool leads_zero(const TileDesc& T, int nseg) {
  for (int s = 0; s < nseg; ++s)
    if (T.leadw[s] != 0) return false;
  return true;
}

template <class P>
static cudaError_t gram_bp(const TileDesc& T, long long r0, long long r1, int p, int q, void* partial, int max_blocks,
                           int* nblocks, cudaStream_t st) {
  constexpr int S = 4;
  int TPR = 0;
  for (int s = 0; s < T.nseg - 1; ++s) TPR += T.g16[s];
  const int NG = kT / TPR;
  const long long ntiles = (r1 - r0 + kRows - 1) / kRows;
  int grid = tiled_grid(ntiles);
  if (grid > max_blocks) grid = max_blocks;
  *nblocks = grid;
  size_t smem = sizeof(float) * S * kRows * T.rowwords;
  const size_t red = sizeof(typename P::G) * (size_t)NG * p * q;
  if (red > smem) smem = red;
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  using G = typename P::G;
  G* out = reinterpret_cast<G*>(partial);
#define GRAMB_LAUNCH(NQv, idx)                                                               \
  do {                                                                                   \
    const cudaError_t e_ = smem_optin(reinterpret_cast<const void*>(k_gram_b<P, NQv, S>), 200 * 1024); \
    if (e_ != cudaSuccess) return e_;                                                   \
    k_gram_b<P, NQv, S><<<grid, kT, smem, st>>>(T, r0, r1, p, q, out);                               \
  } while (0)
  if (q <= 1)
    GRAMB_LAUNCH(1, 0);
  else if (q <= 2)
    GRAMB_LAUNCH(2, 1);
  else if (q <= 4)
    GRAMB_LAUNCH(4, 2);
  else
    GRAMB_LAUNCH(8, 3);
#undef GRAMB_LAUNCH
  return cudaGetLastError();
}

cudaError_t tiled_gram(int prec, const TileDesc& T, long long r0, long long r1, int p, int q, void* partial,
                       int max_blocks, int* nblocks, cudaStream_t st) {
  if (p < 1 || p > kT || q < 1 || q > 8) return cudaErrorInvalidValue;
  if (leads_zero(T, T.nseg - 1)) {
    int TPR = 0;
    for (int s = 0; s < T.nseg - 1; ++s) TPR += T.g16[s];
    if (TPR <= kT) {
      cudaError_t e = cudaErrorInvalidValue;
      switch (prec) {
        case kF32: e = gram_bp<PF32>(T, r0, r1, p, q, partial, max_blocks, nblocks, st); break;
        case kDF64: e = gram_bp<PDF64>(T, r0, r1, p, q, partial, max_blocks, nblocks, st); break;
        case kF64: e = gram_bp<PF64>(T, r0, r1, p, q, partial, max_blocks, nblocks, st); break;
      }
      if (e != cudaErrorInvalidValue) return e;
    }
  }
  switch (prec) {
    case kF32: return gram_tp<PF32>(T, r0, r1, p, q, partial, max_blocks, nblocks, st);
    case kDF64: return gram_tp<PDF64>(T, r0, r1, p, q, partial, max_blocks, nblocks, st);
    case kF64: return gram_tp<PF64>(T, r0, r1, p, q, partial, max_blocks, nblocks, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t tiled_reduce(int prec, const void* partial, int nblocks, int pq, double* G, cudaStream_t st) {
  if (pq < 1) return cudaSuccess;
  switch (prec) {
    case kF32: k_reduce_t<PF32><<<pq, 128, 0, st>>>(reinterpret_cast<const df*>(partial), nblocks, pq, G); break;
    case kDF64: k_reduce_t<PDF64><<<pq, 128, 0, st>>>(reinterpret_cast<const df*>(partial), nblocks, pq, G); break;
    case kF64: k_reduce_t<PF64><<<pq, 128, 0, st>>>(reinterpret_cast<const double*>(partial), nblocks, pq, G); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <class P>
static cudaError_t combine_tp(const TileDesc& T, long long L, int p, const void* coef, const void* In, long long ldin,
                              int alpha_one, void* Out, long long ldout, int q, const void* Rinv, void* Out2,
                              long long ldout2, cudaStream_t st) {
  using S = typename P::S;
  using C = typename P::C;
  using A = typename P::A;
  const size_t smem = sizeof(float) * 2 * kRows * T.rowwords + sizeof(C) * ((size_t)p * q + (Rinv ? (size_t)q * q : 0)) +
                      (Rinv ? sizeof(A) * (size_t)kRows * q : 0);
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  {
    const cudaError_t e = smem_optin(reinterpret_cast<const void*>(k_combine_t<P>), 200 * 1024);
    if (e != cudaSuccess) return e;
  }
  const long long ntiles = (L + kRows - 1) / kRows;
  k_combine_t<P><<<tiled_grid(ntiles), kT, smem, st>>>(
      T, L, p, reinterpret_cast<const C*>(coef), reinterpret_cast<const S*>(In), ldin, alpha_one,
      reinterpret_cast<S*>(Out), ldout, q, reinterpret_cast<const C*>(Rinv), reinterpret_cast<S*>(Out2), ldout2);
  return cudaGetLastError();
}

template <class P, int TPR>
static cudaError_t combine_rp(const TileDesc& T, long long L, int p, const void* coef, const void* In, long long ldin,
                              int alpha_one, void* Out, long long ldout, int q, const void* Rinv, void* Out2,
                              long long ldout2, cudaStream_t st) {
  using S_ = typename P::S;
  using C = typename P::C;
  constexpr int S = 3;
  constexpr int RT = kRowThreads / TPR;
  const int RG = ((T.g16tot + 7) / 8) * 8;
  const size_t smem = (size_t)S * RT * RG * 16 + sizeof(C) * ((size_t)p * q + (Rinv ? (size_t)q * q : 0));
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  {
    const cudaError_t e = smem_optin(reinterpret_cast<const void*>(k_combine_rows<P, 8 / TPR, TPR, S>), 200 * 1024);
    if (e != cudaSuccess) return e;
  }
  const long long ntiles = (L + RT - 1) / RT;
  long long grid = ntiles < 152LL * 8 ? ntiles : 152LL * 8;
  if (grid < 1) grid = 1;
  k_combine_rows<P, 8 / TPR, TPR, S><<<(int)grid, kRowThreads, smem, st>>>(
      T, RG, L, p, reinterpret_cast<const C*>(coef), reinterpret_cast<const S_*>(In), ldin, alpha_one,
      reinterpret_cast<S_*>(Out), ldout, q, reinterpret_cast<const C*>(Rinv), reinterpret_cast<S_*>(Out2), ldout2);
  return cudaGetLastError();
}

cudaError_t tiled_combine(int prec, const TileDesc& T, long long L, int p, const void* coef, const void* In,
                          long long ldin, int alpha_one, void* Out, long long ldout, int q, const void* Rinv, void* Out2,
                          long long ldout2, cudaStream_t st) {
  if (leads_zero(T, T.nseg) && (Rinv == nullptr || q <= 8)) {
    cudaError_t e = cudaErrorInvalidValue;
    switch (prec) {
      case kF32: e = combine_rp<PF32, 1>(T, L, p, coef, In, ldin, alpha_one, Out, ldout, q, Rinv, Out2, ldout2, st); break;
      case kDF64:
        e = Rinv ? combine_rp<PDF64, 1>(T, L, p, coef, In, ldin, alpha_one, Out, ldout, q, Rinv, Out2, ldout2, st)
                 : combine_rp<PDF64, 2>(T, L, p, coef, In, ldin, alpha_one, Out, ldout, q, Rinv, Out2, ldout2, st);
        break;
      case kF64:
        e = Rinv ? combine_rp<PF64, 1>(T, L, p, coef, In, ldin, alpha_one, Out, ldout, q, Rinv, Out2, ldout2, st)
                 : combine_rp<PF64, 2>(T, L, p, coef, In, ldin, alpha_one, Out, ldout, q, Rinv, Out2, ldout2, st);
        break;
    }
    if (e != cudaErrorInvalidValue) return e;
  }
  switch (prec) {
    case kF32: return combine_tp<PF32>(T, L, p, coef, In, ldin, alpha_one, Out, ldout, q, Rinv, Out2, ldout2, st);
    case kDF64: return combine_tp<PDF64>(T, L, p, coef, In, ldin, alpha_one, Out, ldout, q, Rinv, Out2, ldout2, st);
    case kF64: return combine_tp<PF64>(T, L, p, coef, In, ldin, alpha_one, Out, ldout, q, Rinv, Out2, ldout2, st);
  }
  return cudaErrorInvalidValue;
}

template <class P>
static cudaError_t ritz_tp(const TileDesc& T, long long L, int g, const void* Y, const void* theta, void* X, void* R,
                           long long ldb, int nb, const void* dscale, void* Tout, void* partial, int max_blocks,
                           int* nblocks, cudaStream_t st) {
  using S = typename P::S;
  using C = typename P::C;
  using G = typename P::G;
  size_t smem = sizeof(float) * 2 * kRows * T.rowwords + sizeof(C) * ((size_t)g * nb + nb);
  const size_t red = sizeof(G) * 16 * kRows;
  if (red > smem) smem = red;
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  {
    const cudaError_t e = smem_optin(reinterpret_cast<const void*>(k_ritz_t<P>), 200 * 1024);
    if (e != cudaSuccess) return e;
  }
  const long long ntiles = (L + kRows - 1) / kRows;
  int grid = tiled_grid(ntiles);
  if (grid > max_blocks) grid = max_blocks;
  *nblocks = grid;
  k_ritz_t<P><<<grid, kT, smem, st>>>(T, L, g, reinterpret_cast<const C*>(Y), reinterpret_cast<const C*>(theta),
                                      reinterpret_cast<S*>(X), reinterpret_cast<S*>(R), ldb, nb,
                                      reinterpret_cast<const S*>(dscale), reinterpret_cast<S*>(Tout),
                                      reinterpret_cast<G*>(partial));
  return cudaGetLastError();
}

template <class P, int NB, int TPR>
static cudaError_t ritz_rp(const TileDesc& T, long long L, int g, const void* Y, const void* theta, void* X, void* R,
                           long long ldb, int nb, const void* dscale, void* Tout, void* partial, int max_blocks,
                           int* nblocks, cudaStream_t st) {
  using S_ = typename P::S;
  using C = typename P::C;
  using G = typename P::G;
  constexpr int S = 3;
  constexpr int RT = kRowThreads / TPR;
  const int RG = ((T.g16tot + 7) / 8) * 8;
  size_t smem = (size_t)S * RT * RG * 16 + sizeof(C) * ((size_t)g * nb + nb);
  const size_t red = sizeof(G) * (size_t)NB * RT;
  if (red > smem) smem = red;
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  {
    const cudaError_t e = smem_optin(reinterpret_cast<const void*>(k_ritz_rows<P, NB, TPR, S>), 200 * 1024);
    if (e != cudaSuccess) return e;
  }
  const long long ntiles = (L + RT - 1) / RT;
  long long grid = ntiles < 152LL * 8 ? ntiles : 152LL * 8;
  if (grid > max_blocks) grid = max_blocks;
  if (grid < 1) grid = 1;
  *nblocks = (int)grid;
  k_ritz_rows<P, NB, TPR, S><<<(int)grid, kRowThreads, smem, st>>>(
      T, RG, L, g, reinterpret_cast<const C*>(Y), reinterpret_cast<const C*>(theta), reinterpret_cast<S_*>(X),
      reinterpret_cast<S_*>(R), ldb, nb, reinterpret_cast<const S_*>(dscale), reinterpret_cast<S_*>(Tout),
      reinterpret_cast<G*>(partial));
  return cudaGetLastError();
}

cudaError_t tiled_ritz(int prec, const TileDesc& T, long long L, int g, const void* Y, const void* theta, void* X,
                       void* R, long long ldb, int nb, const void* dscale, void* Tout, void* partial, int max_blocks,
                       int* nblocks, cudaStream_t st) {
  if (nb < 1 || nb > 16) return cudaErrorInvalidValue;
  if (leads_zero(T, 2) && T.g16[0] == T.g16[1] && nb <= 8) {
    cudaError_t e = cudaErrorInvalidValue;
#define RITZ_ARGS T, L, g, Y, theta, X, R, ldb, nb, dscale, Tout, partial, max_blocks, nblocks, st
    switch (prec) {
      case kF32: e = nb <= 4 ? ritz_rp<PF32, 4, 1>(RITZ_ARGS) : ritz_rp<PF32, 8, 1>(RITZ_ARGS); break;
      case kDF64: e = nb <= 4 ? ritz_rp<PDF64, 4, 2>(RITZ_ARGS) : ritz_rp<PDF64, 8, 2>(RITZ_ARGS); break;
      case kF64: e = nb <= 4 ? ritz_rp<PF64, 4, 2>(RITZ_ARGS) : ritz_rp<PF64, 8, 2>(RITZ_ARGS); break;
    }
#undef RITZ_ARGS
    if (e != cudaErrorInvalidValue) return e;
  }
  switch (prec) {
    case kF32: return ritz_tp<PF32>(T, L, g, Y, theta, X, R, ldb, nb, dscale, Tout, partial, max_blocks, nblocks, st);
    case kDF64: return ritz_tp<PDF64>(T, L, g, Y, theta, X, R, ldb, nb, dscale, Tout, partial, max_blocks, nblocks, st);
    case kF64: return ritz_tp<PF64>(T, L, g, Y, theta, X, R, ldb, nb, dscale, Tout, partial, max_blocks, nblocks, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace phsvds
