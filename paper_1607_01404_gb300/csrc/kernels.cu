// Device kernels of the PHSVDS hot path (sm_103a).
//
// * k_spmm            : CSR SpMM Y = A X over row-major blocks (the user matvec
//                       of the paper's Sec. 3.4 with transpose 0/1 through an
//                       explicit CSR of A^T, Sec. 3.3 "operations with both the
//                       matrix and its transpose").
// * k_gram / reduce   : tall-skinny projections [P0 P1 P2]^T Q (Rayleigh-Ritz
//                       projection V^T W, CGS and CholQR Gram matrices; Table 3
//                       "Inner Prods"), deterministic two-level reduction.
// * k_combine         : tall-skinny times small (Table 3 "MM": V Y, restart
//                       V <- V Z in place, T <- (T - V C) R^-1).
// * k_ritz_residual   : fused Ritz vectors, residuals and norms (Sec. 3.3: the
//                       residual kernel that minimises memory accesses).
// * setup kernels     : deterministic CSR transpose, value formats, diagonal of
//                       A^T A, validation.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <cmath>
#include <cstring>

#include "common.cuh"
#include "kernels.h"
#include "spmm_dev.cuh"
#include "tiled.h"

namespace phsvds {

namespace {

constexpr int kThreads = 256;

inline int grid_for(long long n, int threads) {
  long long g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > 2147483647LL) g = 2147483647LL;
  return (int)g;
}

struct SegArr {
  const void* p[3];
  long long ld[3];
  int nc[3];
  int n;
};

template <class S>
__device__ __forceinline__ const S* seg_col(const SegArr& sa, int c, long long* ld) {
  int s = 0;
  while (s < sa.n - 1 && c >= sa.nc[s]) {
    c -= sa.nc[s];
    ++s;
  }
  *ld = sa.ld[s];
  return reinterpret_cast<const S*>(sa.p[s]) + c;
}

// ---------------------------------------------------------------------------
// SpMM
// ---------------------------------------------------------------------------
template <class P, int NB, int VMODE, bool VEC>
__global__ void __launch_bounds__(kThreads) k_spmm(long long rows, const int* __restrict__ rowptr,
                                                   const int* __restrict__ colidx, const float* __restrict__ v32,
                                                   const float* __restrict__ v32lo, const double* __restrict__ v64,
                                                   const typename P::S* __restrict__ X, long long ldx,
                                                   typename P::S* __restrict__ Y, long long ldy, int yvec) {
  using A = typename P::A;
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= rows) return;
  A acc[NB];
#pragma unroll
  for (int c = 0; c < NB; ++c) acc[c] = P::zero();
  row_product<P, NB, VMODE, VEC, spmm_unroll<P, NB>()>(__ldg(rowptr + i), __ldg(rowptr + i + 1), colidx, v32, v32lo,
                                                        v64, X, ldx, acc);
  store_yrow<P, NB, VEC>(Y + i * ldy, acc, yvec != 0);
}

// Short rows (at most a few nonzeros): each thread handles two consecutive rows
// and interleaves their gathers, doubling the loads in flight per thread.
template <class P, int NB, int VMODE, bool VEC>
__global__ void __launch_bounds__(kThreads) k_spmm2(long long rows, const int* __restrict__ rowptr,
                                                    const int* __restrict__ colidx, const float* __restrict__ v32,
                                                    const float* __restrict__ v32lo, const double* __restrict__ v64,
                                                    const typename P::S* __restrict__ X, long long ldx,
                                                    typename P::S* __restrict__ Y, long long ldy, int yvec) {
  using A = typename P::A;
  const long long i0 = 2 * (blockIdx.x * (long long)blockDim.x + threadIdx.x);
  if (i0 >= rows) return;
  const bool two = i0 + 1 < rows;
  const int ka = __ldg(rowptr + i0), kb = __ldg(rowptr + i0 + 1), kc = two ? __ldg(rowptr + i0 + 2) : kb;
  A acc0[NB], acc1[NB];
#pragma unroll
  for (int c = 0; c < NB; ++c) acc0[c] = acc1[c] = P::zero();
  const int na = kb - ka, nbn = kc - kb;
  const int nmax = na > nbn ? na : nbn;
  for (int t = 0; t < nmax; ++t) {
    const bool ua = t < na, ub = t < nbn;
    const int ja = ua ? __ldg(colidx + ka + t) : 0;
    const int jb = ub ? __ldg(colidx + kb + t) : 0;
    A xa[NB], xb[NB];
    if (ua) load_xrow<P, NB, VEC>(X + (long long)ja * ldx, xa);
    if (ub) load_xrow<P, NB, VEC>(X + (long long)jb * ldx, xb);
    if (ua) spmm_accum<P, NB, VMODE, VEC>(ka + t, v32, v32lo, v64, xa, acc0);
    if (ub) spmm_accum<P, NB, VMODE, VEC>(kb + t, v32, v32lo, v64, xb, acc1);
  }
  store_yrow<P, NB, VEC>(Y + i0 * ldy, acc0, yvec != 0);
  if (two) store_yrow<P, NB, VEC>(Y + (i0 + 1) * ldy, acc1, yvec != 0);
}

template <class P, int NB, bool VEC>
cudaError_t spmm_nbv(const CsrDev& A, const void* X, long long ldx, void* Y, long long ldy, int yvec,
                     cudaStream_t st) {
  if (P::id == kF32 && A.rows > 0 && A.nnz <= 4 * A.rows) {  // short rows (FP32): two rows per thread
    using S = typename P::S;
    const int grid = grid_for((A.rows + 1) / 2, kThreads);
    const S* x = reinterpret_cast<const S*>(X);
    S* y = reinterpret_cast<S*>(Y);
    if constexpr (P::id == kF32) {
      if (A.v16)
        k_spmm2<P, NB, 4, VEC><<<grid, kThreads, 0, st>>>(A.rows, A.rowptr, A.colidx,
                                                          reinterpret_cast<const float*>(A.v16), nullptr, nullptr, x,
                                                          ldx, y, ldy, yvec);
      else
        k_spmm2<P, NB, 0, VEC><<<grid, kThreads, 0, st>>>(A.rows, A.rowptr, A.colidx, A.v32, nullptr, nullptr, x, ldx,
                                                          y, ldy, yvec);
    } else if constexpr (P::id == kDF64) {
      if (A.v32lo == nullptr)
        k_spmm2<P, NB, 1, VEC><<<grid, kThreads, 0, st>>>(A.rows, A.rowptr, A.colidx, A.v32, nullptr, nullptr, x, ldx,
                                                          y, ldy, yvec);
      else
        k_spmm2<P, NB, 2, VEC><<<grid, kThreads, 0, st>>>(A.rows, A.rowptr, A.colidx, A.v32, A.v32lo, nullptr, x, ldx,
                                                          y, ldy, yvec);
    } else {
      k_spmm2<P, NB, 3, VEC><<<grid, kThreads, 0, st>>>(A.rows, A.rowptr, A.colidx, nullptr, nullptr, A.v64, x, ldx, y,
                                                        ldy, yvec);
    }
    return cudaGetLastError();
  }
  using S = typename P::S;
  const int grid = grid_for(A.rows, kThreads);
  const S* x = reinterpret_cast<const S*>(X);
  S* y = reinterpret_cast<S*>(Y);
  if constexpr (P::id == kF32) {
    if (A.v16)
      k_spmm<P, NB, 4, VEC><<<grid, kThreads, 0, st>>>(A.rows, A.rowptr, A.colidx,
                                                       reinterpret_cast<const float*>(A.v16), nullptr, nullptr, x, ldx,
                                                       y, ldy, yvec);
    else
      k_spmm<P, NB, 0, VEC><<<grid, kThreads, 0, st>>>(A.rows, A.rowptr, A.colidx, A.v32, nullptr, nullptr, x, ldx, y,
                                                       ldy, yvec);
  } else if constexpr (P::id == kDF64) {
    if (A.v32lo == nullptr)
      k_spmm<P, NB, 1, VEC><<<grid, kThreads, 0, st>>>(A.rows, A.rowptr, A.colidx, A.v32, nullptr, nullptr, x, ldx, y,
                                                       ldy, yvec);
    else
      k_spmm<P, NB, 2, VEC><<<grid, kThreads, 0, st>>>(A.rows, A.rowptr, A.colidx, A.v32, A.v32lo, nullptr, x, ldx, y,
                                                       ldy, yvec);
  } else {
    k_spmm<P, NB, 3, VEC><<<grid, kThreads, 0, st>>>(A.rows, A.rowptr, A.colidx, nullptr, nullptr, A.v64, x, ldx, y,
                                                     ldy, yvec);
  }
  return cudaGetLastError();
}

template <class P, int NB>
cudaError_t spmm_nb(const CsrDev& A, const void* X, long long ldx, void* Y, long long ldy, cudaStream_t st) {
  constexpr size_t es = sizeof(typename P::S);
  // 16-byte gathers need X's rows on 16-byte boundaries; 16-byte stores need
  // Y's (decided per launch inside the kernel)
  const bool vec = (NB * es) % 16 == 0 && (ldx * es) % 16 == 0 && reinterpret_cast<uintptr_t>(X) % 16 == 0;
  const int yvec = (ldy * es) % 16 == 0 && reinterpret_cast<uintptr_t>(Y) % 16 == 0 ? 1 : 0;
  if constexpr ((NB * es) % 16 == 0) {
    if (vec) return spmm_nbv<P, NB, true>(A, X, ldx, Y, ldy, yvec, st);
  }
  return spmm_nbv<P, NB, false>(A, X, ldx, Y, ldy, 0, st);
}

template <class P>
cudaError_t spmm_p(const CsrDev& A, const void* X, long long ldx, void* Y, long long ldy, int b, cudaStream_t st) {
  using S = typename P::S;
  int c0 = 0;
  while (c0 < b) {
    const int rem = b - c0;
    const S* x = reinterpret_cast<const S*>(X) + c0;
    S* y = reinterpret_cast<S*>(Y) + c0;
    cudaError_t e;
    int w;
    if (rem >= 8) {
      w = 8;
      e = spmm_nb<P, 8>(A, x, ldx, y, ldy, st);
    } else if (rem >= 4) {
      w = 4;
      e = spmm_nb<P, 4>(A, x, ldx, y, ldy, st);
    } else if (rem >= 2) {
      w = 2;
      e = spmm_nb<P, 2>(A, x, ldx, y, ldy, st);
    } else {
      w = 1;
      e = spmm_nb<P, 1>(A, x, ldx, y, ldy, st);
    }
    if (e != cudaSuccess) return e;
    c0 += w;
  }
  return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Gram: partial[blk][i][j] = sum over the block's rows of P[r, i] Q[r, j]
// ---------------------------------------------------------------------------
constexpr int kGramThreads = 256;
constexpr int kGramQ = 8;

template <class P>
__global__ void __launch_bounds__(kGramThreads) k_gram(long long r0, long long r1, SegArr segs, int p,
                                                       const typename P::S* __restrict__ Q, long long ldq, int q,
                                                       typename P::G* __restrict__ partial) {
  using S = typename P::S;
  using G = typename P::G;
  __shared__ G sm[kGramThreads * kGramQ];
  const int t = threadIdx.x;
  const int ngroups = kGramThreads / p;
  const int i = t % p, rg = t / p;
  const bool active = rg < ngroups;
  long long ld;
  const S* base = seg_col<S>(segs, active ? i : 0, &ld);
  const long long total = r1 - r0;
  const long long per = (total + gridDim.x - 1) / gridDim.x;
  const long long cr0 = r0 + (long long)blockIdx.x * per;
  const long long cr1 = cr0 + per < r1 ? cr0 + per : r1;
  G acc[kGramQ];
#pragma unroll
  for (int j = 0; j < kGramQ; ++j) acc[j] = P::gzero();
  if (active) {
#pragma unroll 2
    for (long long r = cr0 + rg; r < cr1; r += ngroups) {
      const auto x = P::load(base + r * ld);
      const S* qr = Q + r * ldq;
#pragma unroll
      for (int j = 0; j < kGramQ; ++j)
        if (j < q) acc[j] = P::gfma(acc[j], x, P::load(qr + j));
    }
    for (int j = 0; j < q; ++j) sm[(rg * p + i) * q + j] = acc[j];
  }
  __syncthreads();
  const int pq = p * q;
  for (int e = t; e < pq; e += kGramThreads) {
    G s = sm[e];
    for (int g = 1; g < ngroups; ++g) s = P::gadd(s, sm[g * pq + e]);
    partial[(long long)blockIdx.x * pq + e] = s;
  }
}

template <class P>
cudaError_t gram_p(long long r0, long long r1, const SegArr& sa, int p, SegV Q, void* partial, int max_blocks,
                   int* nblocks, cudaStream_t st) {
  long long rows = r1 - r0;
  long long want = (rows + 255) / 256;  // at least ~256 rows per block
  int nb = (int)(want < max_blocks ? want : max_blocks);
  if (nb < 1) nb = 1;
  *nblocks = nb;
  k_gram<P><<<nb, kGramThreads, 0, st>>>(r0, r1, sa, p, reinterpret_cast<const typename P::S*>(Q.p), Q.ld, Q.nc,
                                         reinterpret_cast<typename P::G*>(partial));
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Combine: Out = alpha In + P coef, then Out <- Out Rinv
// ---------------------------------------------------------------------------
constexpr int kCmbRows = 32;
constexpr int kCmbThreads = 128;

template <class P>
__global__ void __launch_bounds__(kCmbThreads) k_combine(long long L, SegArr segs, int p,
                                                         const typename P::C* __restrict__ coef,
                                                         const typename P::S* In, long long ldin, int alpha_one,
                                                         typename P::S* Out, long long ldout, int q,
                                                         const typename P::C* __restrict__ Rinv,
                                                         typename P::S* Out2, long long ldout2) {
  using S = typename P::S;
  using A = typename P::A;
  using C = typename P::C;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int pst = p + 1;
  A* Ps = reinterpret_cast<A*>(smraw);
  C* Cs = reinterpret_cast<C*>(Ps + kCmbRows * pst);
  A* Os = reinterpret_cast<A*>(Cs + p * q);
  C* Rs = reinterpret_cast<C*>(Os + kCmbRows * q);
  const int t = threadIdx.x;
  for (int e = t; e < p * q; e += kCmbThreads) Cs[e] = coef[e];
  if (Rinv)
    for (int e = t; e < q * q; e += kCmbThreads) Rs[e] = Rinv[e];
  for (long long row0 = (long long)blockIdx.x * kCmbRows; row0 < L; row0 += (long long)gridDim.x * kCmbRows) {
    const int nrows = (int)(L - row0 < kCmbRows ? L - row0 : kCmbRows);
    __syncthreads();
    for (int e = t; e < nrows * p; e += kCmbThreads) {
      const int r = e / p, c = e % p;
      long long ld;
      const S* b = seg_col<S>(segs, c, &ld);
      Ps[r * pst + c] = P::load(b + (row0 + r) * ld);
    }
    __syncthreads();
    for (int e = t; e < nrows * q; e += kCmbThreads) {
      const int r = e / q, j = e % q;
      A acc = alpha_one ? P::load(In + (row0 + r) * ldin + j) : P::zero();
      for (int c = 0; c < p; ++c) acc = P::fmac(acc, Ps[r * pst + c], Cs[c * q + j]);
      if (Rinv) {
        Os[r * q + j] = acc;
      } else {
        P::store(Out + (row0 + r) * ldout + j, acc);
        if (Out2) P::store(Out2 + (row0 + r) * ldout2 + j, acc);
      }
    }
    if (Rinv) {
      __syncthreads();
      for (int e = t; e < nrows * q; e += kCmbThreads) {
        const int r = e / q, j = e % q;
        A acc = P::zero();
        for (int l = 0; l <= j; ++l) acc = P::fmac(acc, Os[r * q + l], Rs[l * q + j]);
        P::store(Out + (row0 + r) * ldout + j, acc);
        if (Out2) P::store(Out2 + (row0 + r) * ldout2 + j, acc);
      }
    }
  }
}

template <class P>
size_t combine_smem(int p, int q, bool rinv) {
  return sizeof(typename P::A) * (size_t)kCmbRows * (p + 1) + sizeof(typename P::C) * (size_t)p * q +
         sizeof(typename P::A) * (size_t)kCmbRows * q + (rinv ? sizeof(typename P::C) * (size_t)q * q : 0);
}

// ---------------------------------------------------------------------------
// Fused Ritz vectors / residuals / norms
// ---------------------------------------------------------------------------
template <class P>
__global__ void __launch_bounds__(kCmbThreads) k_ritz_residual(long long L, const typename P::S* V, long long ldv,
                                                               const typename P::S* W, long long ldw, int g,
                                                               const typename P::C* __restrict__ Y,
                                                               const typename P::C* __restrict__ theta,
                                                               typename P::S* X, typename P::S* R, long long ldb,
                                                               int nb, const typename P::S* __restrict__ dscale,
                                                               typename P::S* T, typename P::G* __restrict__ partial) {
  using A = typename P::A;
  using C = typename P::C;
  using G = typename P::G;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int gst = g + 1;
  A* Vs = reinterpret_cast<A*>(smraw);
  A* Ws = Vs + kCmbRows * gst;
  C* Ys = reinterpret_cast<C*>(Ws + kCmbRows * gst);
  C* Th = Ys + g * nb;
  G* Ns = reinterpret_cast<G*>(Th + nb);
  const int t = threadIdx.x;
  for (int e = t; e < g * nb; e += kCmbThreads) Ys[e] = Y[e];
  for (int e = t; e < nb; e += kCmbThreads) Th[e] = theta[e];
  G nacc = P::gzero();  // thread j < nb accumulates column j
  for (long long row0 = (long long)blockIdx.x * kCmbRows; row0 < L; row0 += (long long)gridDim.x * kCmbRows) {
    const int nrows = (int)(L - row0 < kCmbRows ? L - row0 : kCmbRows);
    __syncthreads();
    for (int e = t; e < nrows * g; e += kCmbThreads) {
      const int r = e / g, c = e % g;
      Vs[r * gst + c] = P::load(V + (row0 + r) * ldv + c);
      Ws[r * gst + c] = P::load(W + (row0 + r) * ldw + c);
    }
    __syncthreads();
    for (int e = t; e < nrows * nb; e += kCmbThreads) {
      const int r = e / nb, j = e % nb;
      A x = P::zero(), w = P::zero();
      for (int c = 0; c < g; ++c) {
        x = P::fmac(x, Vs[r * gst + c], Ys[c * nb + j]);
        w = P::fmac(w, Ws[r * gst + c], Ys[c * nb + j]);
      }
      const A res = P::sub(w, P::mulc(x, Th[j]));
      const long long o = (row0 + r) * ldb + j;
      P::store(X + o, x);
      P::store(R + o, res);
      if (T) P::store(T + o, P::mulc(res, P::load(dscale + row0 + r)));
      Ns[r * nb + j] = P::gfma(P::gzero(), res, res);
    }
    __syncthreads();
    if (t < nb)
      for (int r = 0; r < nrows; ++r) nacc = P::gadd(nacc, Ns[r * nb + t]);
  }
  if (t < nb) partial[(long long)blockIdx.x * nb + t] = nacc;
}

// ---------------------------------------------------------------------------
// Stage-2 split residual norms
// ---------------------------------------------------------------------------
template <class P>
__global__ void __launch_bounds__(kThreads) k_split_resnorm(long long L, long long n, const typename P::S* X,
                                                            const typename P::S* BX, long long ldb, int nb,
                                                            const typename P::C* __restrict__ cf,
                                                            typename P::G* __restrict__ partial) {
  using A = typename P::A;
  using G = typename P::G;
  __shared__ G sm[kThreads * 8];
  G acc[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) acc[j] = P::gzero();
  const long long total = L * nb;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += stride) {
    const long long r = e / nb;
    const int j = (int)(e % nb);
    const int off = r < n ? 0 : 2 * nb;
    const A v = P::sub(P::mulc(P::load(BX + r * ldb + j), cf[off + j]), P::mulc(P::load(X + r * ldb + j), cf[off + nb + j]));
#pragma unroll
    for (int jj = 0; jj < 8; ++jj)
      if (jj == j) acc[jj] = P::gfma(acc[jj], v, v);
  }
  for (int j = 0; j < nb; ++j) sm[threadIdx.x * 8 + j] = acc[j];
  __syncthreads();
  if (threadIdx.x < nb) {
    G s = sm[threadIdx.x];
    for (int tt = 1; tt < blockDim.x; ++tt) s = P::gadd(s, sm[tt * 8 + threadIdx.x]);
    partial[(long long)blockIdx.x * nb + threadIdx.x] = s;
  }
}

// ---------------------------------------------------------------------------
// Elementwise helpers
// ---------------------------------------------------------------------------
template <class P>
__global__ void k_scale_rows(long long L, const typename P::S* d, const typename P::S* R, long long ldr,
                             typename P::S* T, long long ldt, int nb) {
  const long long total = L * nb;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const long long r = e / nb;
    const int j = (int)(e % nb);
    auto dv = P::load(d + r);
    auto rv = P::load(R + r * ldr + j);
    if constexpr (P::id == kDF64)
      P::store(T + r * ldt + j, df_mul(rv, dv));
    else
      P::store(T + r * ldt + j, rv * dv);
  }
}

template <class P>
__global__ void k_copy_cols(long long L, const typename P::S* Src, long long lds, typename P::S* Dst, long long ldd,
                            int nb) {
  const long long total = L * nb;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const long long r = e / nb;
    const int j = (int)(e % nb);
    Dst[r * ldd + j] = Src[r * lds + j];
  }
}

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
  // Steele, Lea, Flood, "Fast splittable pseudorandom number generators", 2014.
  x += 0x9E3779B97F4A7C15ULL;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ULL;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBULL;
  return x ^ (x >> 31);
}

template <class P>
__global__ void k_fill_normal(long long L, typename P::S* Dst, long long ldd, int nb, unsigned long long seed) {
  const long long total = L * nb;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const long long r = e / nb;
    const int j = (int)(e % nb);
    unsigned long long h = splitmix64(seed ^ splitmix64((unsigned long long)e));
    double u1 = ((h >> 11) + 1.0) * (1.0 / 9007199254740993.0);  // (0, 1]
    unsigned long long h2 = splitmix64(h);
    double u2 = (h2 >> 11) * (1.0 / 9007199254740992.0);
    double z = sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
    if constexpr (P::id == kF32) {
      Dst[r * ldd + j] = (float)z;
    } else if constexpr (P::id == kDF64) {
      float hi = (float)z;
      Dst[r * ldd + j] = df{hi, (float)(z - (double)hi)};
    } else {
      Dst[r * ldd + j] = z;
    }
  }
}

template <class P>
__global__ void k_from_f64(long long L, int nc, const double* src, long long lds, typename P::S* dst, long long ldd,
                           double scale) {
  const long long total = L * nc;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const long long r = e % L;
    const int j = (int)(e / L);
    const double z = src[(long long)j * lds + r] * scale;
    if constexpr (P::id == kF32) {
      dst[r * ldd + j] = (float)z;
    } else if constexpr (P::id == kDF64) {
      float hi = (float)z;
      dst[r * ldd + j] = df{hi, (float)(z - (double)hi)};
    } else {
      dst[r * ldd + j] = z;
    }
  }
}

// Row-major blocks in the mode's storage <-> row-major FP64 blocks (the
// interface of caller-supplied operators): element (r, j) at r * ld + j.
template <class P>
__global__ void k_rows_f64(long long L, int nc, const typename P::S* src, long long lds, double* dst, long long ldd) {
  const long long total = L * nc;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const long long r = e / nc;
    const int j = (int)(e - r * nc);
    const typename P::S v = src[r * lds + j];
    if constexpr (P::id == kDF64)
      dst[r * ldd + j] = (double)v.hi + (double)v.lo;
    else
      dst[r * ldd + j] = (double)v;
  }
}
template <class P>
__global__ void k_rows_from_f64(long long L, int nc, const double* src, long long lds, typename P::S* dst,
                                long long ldd) {
  const long long total = L * nc;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const long long r = e / nc;
    const int j = (int)(e - r * nc);
    const double z = src[r * lds + j];
    if constexpr (P::id == kF32) {
      dst[r * ldd + j] = (float)z;
    } else if constexpr (P::id == kDF64) {
      const float hi = (float)z;
      dst[r * ldd + j] = df{hi, (float)(z - (double)hi)};
    } else {
      dst[r * ldd + j] = z;
    }
  }
}

template <class P>
__global__ void k_to_f64(long long L, int nc, const typename P::S* src, long long lds, double* dst, long long ldd,
                         double scale) {
  const long long total = L * nc;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const long long r = e % L;
    const int j = (int)(e / L);
    double z;
    if constexpr (P::id == kDF64) {
      df v = src[r * lds + j];
      z = (double)v.hi + (double)v.lo;
    } else {
      z = (double)src[r * lds + j];
    }
    dst[(long long)j * ldd + r] = z * scale;
  }
}

template <class P>
__global__ void k_make_dscale(long long L, const double* s, int use_sqrt, typename P::S* d) {
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < L; r += (long long)gridDim.x * blockDim.x) {
    double v = s[r];
    if (use_sqrt) v = sqrt(v);
    double z = v > 0 ? 1.0 / v : 1.0;
    if constexpr (P::id == kF32) {
      d[r] = (float)z;
    } else if constexpr (P::id == kDF64) {
      float hi = (float)z;
      d[r] = df{hi, (float)(z - (double)hi)};
    } else {
      d[r] = z;
    }
  }
}

// ---------------------------------------------------------------------------
// Setup kernels
// ---------------------------------------------------------------------------
__global__ void k_absmax(long long nnz, const double* vals, unsigned long long* out) {
  unsigned long long m = 0;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nnz; k += (long long)gridDim.x * blockDim.x) {
    double a = fabs(vals[k]);
    unsigned long long b = (unsigned long long)__double_as_longlong(a);
    m = b > m ? b : m;
  }
  atomicMax(out, m);
}

__global__ void k_csr_values(long long nnz, const double* vals, double scale, float* v32, float* v32lo, double* v64,
                             int* flags) {
  int any = 0;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nnz; k += (long long)gridDim.x * blockDim.x) {
    const double z = vals[k] * scale;
    const float hi = (float)z;
    const float lo = (float)(z - (double)hi);
    v32[k] = hi;
    v32lo[k] = lo;
    v64[k] = z;
    any |= (lo != 0.f);
  }
  if (any) atomicOr(flags, 1);
}

__global__ void k_count_cols(long long nnz, const int* colidx, int* cnt) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nnz; k += (long long)gridDim.x * blockDim.x)
    atomicAdd(cnt + colidx[k], 1);
}

constexpr int kScanChunk = 2048;

__global__ void k_scan_block_sums(long long n, const int* in, long long* bsum) {
  __shared__ long long sm[kThreads];
  const long long base = (long long)blockIdx.x * kScanChunk;
  long long s = 0;
  for (int e = threadIdx.x; e < kScanChunk; e += kThreads)
    if (base + e < n) s += in[base + e];
  sm[threadIdx.x] = s;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) bsum[blockIdx.x] = sm[0];
}

// Exclusive scan of bsum (nb entries) by one block, sequential over chunks.
__global__ void k_scan_bsums(int nb, long long* bsum) {
  __shared__ long long sm[1024];
  long long carry = 0;
  for (int c0 = 0; c0 < nb; c0 += 1024) {
    const int i = c0 + threadIdx.x;
    long long v = i < nb ? bsum[i] : 0;
    sm[threadIdx.x] = v;
    __syncthreads();
    for (int w = 1; w < 1024; w <<= 1) {  // Hillis-Steele inclusive scan
      long long add = threadIdx.x >= w ? sm[threadIdx.x - w] : 0;
      __syncthreads();
      sm[threadIdx.x] += add;
      __syncthreads();
    }
    if (i < nb) bsum[i] = carry + sm[threadIdx.x] - v;
    carry += sm[1023];
    __syncthreads();
  }
}

// out[0] = 0, out[i + 1] = sum_{t <= i} in[t] (int32 result, checked on host).
__global__ void k_scan_apply(long long n, const int* in, const long long* boff, int* out) {
  __shared__ long long sm[kScanChunk];
  const long long base = (long long)blockIdx.x * kScanChunk;
  for (int e = threadIdx.x; e < kScanChunk; e += kThreads) sm[e] = base + e < n ? in[base + e] : 0;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long s = boff[blockIdx.x];
    for (int e = 0; e < kScanChunk; ++e) {
      s += sm[e];
      sm[e] = s;
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kScanChunk; e += kThreads)
    if (base + e < n) out[base + e + 1] = (int)sm[e];
  if (blockIdx.x == 0 && threadIdx.x == 0) out[0] = 0;
}

__global__ void k_scatter_t(long long rows, const int* rowptr, const int* colidx, const double* vals,
                            const int* rowptrT, int* cursor, int* colidxT, double* valsT) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < rows; i += (long long)gridDim.x * blockDim.x) {
    for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      const int j = colidx[k];
      const int pos = rowptrT[j] + atomicAdd(cursor + j, 1);
      colidxT[pos] = (int)i;
      valsT[pos] = vals[k];
    }
  }
}

__device__ void sift_down(int* key, double* val, int start, int end) {
  int root = start;
  while (2 * root + 1 <= end) {
    int child = 2 * root + 1, sw = root;
    if (key[sw] < key[child]) sw = child;
    if (child + 1 <= end && key[sw] < key[child + 1]) sw = child + 1;
    if (sw == root) return;
    int tk = key[root];
    key[root] = key[sw];
    key[sw] = tk;
    double tv = val[root];
    val[root] = val[sw];
    val[sw] = tv;
    root = sw;
  }
}

// Sort each row segment of the transposed CSR by index (makes the atomic
// scatter order irrelevant, so the result is deterministic).
__global__ void k_sort_segments(long long rowsT, const int* rowptrT, int* colidxT, double* valsT) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < rowsT; j += (long long)gridDim.x * blockDim.x) {
    const int k0 = rowptrT[j], len = rowptrT[j + 1] - k0;
    int* key = colidxT + k0;
    double* val = valsT + k0;
    if (len <= 32) {
      for (int a = 1; a < len; ++a) {
        int kk = key[a];
        double vv = val[a];
        int b = a - 1;
        while (b >= 0 && key[b] > kk) {
          key[b + 1] = key[b];
          val[b + 1] = val[b];
          --b;
        }
        key[b + 1] = kk;
        val[b + 1] = vv;
      }
    } else {  // heapsort
      for (int s = (len - 2) / 2; s >= 0; --s) sift_down(key, val, s, len - 1);
      for (int end = len - 1; end > 0; --end) {
        int tk = key[end];
        key[end] = key[0];
        key[0] = tk;
        double tv = val[end];
        val[end] = val[0];
        val[0] = tv;
        sift_down(key, val, 0, end - 1);
      }
    }
  }
}

__global__ void k_precond_check(long long n, const int* __restrict__ rowptr, const int* __restrict__ colidx,
                                const float* __restrict__ v32, const double* __restrict__ v64, int* flags) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride) {
    int f = 2;  // until a positive diagonal entry is seen
    for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      const double v = v32 ? (double)v32[k] : v64[k];
      if (!isfinite(v)) f |= 1;
      if (colidx[k] == i && v > 0) f &= ~2;
    }
    if (f) atomicOr(flags, f);
  }
}

__global__ void k_row_sumsq(long long rows, const int* rowptr, const double* vals, double* out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < rows; i += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) s += vals[k] * vals[k];
    out[i] = s;
  }
}

__global__ void k_csr_validate(long long rows, long long cols, const int* rowptr, const int* colidx, const double* vals,
                               int* flags) {
  int f = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < rows; i += (long long)gridDim.x * blockDim.x) {
    const int k0 = rowptr[i], k1 = rowptr[i + 1];
    if (k1 < k0) {
      f |= 2;
      continue;
    }
    int prev = -1;
    for (int k = k0; k < k1; ++k) {
      const int c = colidx[k];
      if (c < 0 || c >= cols || c <= prev) f |= 2;
      prev = c;
      if (!isfinite(vals[k])) f |= 4;
    }
  }
  if (f) atomicOr(flags, f);
}

// ---------------------------------------------------------------------------
// Small dense steps of the block orthogonalisation, on the device so that the
// CGS2 + CholQR2 sequence needs no host round trip.  One CTA of 64 threads.
//   stage 1: G = [V T]^T T ((g+nb) x nb): coef = -G[0:g], work[0:nb] = diag(T^T T)
//   stage 2: G = [V T']^T T': C2 = G[0:g], S = G[g:] - C2^T C2, R1 = chol(S);
//            coef = -C2, rinv = R1^-1; status bit 1 if a column kept less than
//            sqrt(drop2) of its norm, bit 2 if S is not positive definite
//   stage 3: G = T''^T T'' (nb x nb): R2 = chol(G), coef = R2^-1
// Coefficients are written in the mode's coefficient format (row-major).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void store_coef(int prec, void* out, int idx, double v) {
  if (prec == kF32) {
    reinterpret_cast<float*>(out)[idx] = (float)v;
  } else if (prec == kDF64) {
    const float hi = (float)v;
    reinterpret_cast<float*>(out)[2 * idx] = hi;
    reinterpret_cast<float*>(out)[2 * idx + 1] = (float)(v - (double)hi);
  } else {
    reinterpret_cast<double*>(out)[idx] = v;
  }
}

// Upper Cholesky of the nb x nb row-major matrix S into R (row-major) and its
// inverse into Ri; returns false if S is not numerically positive definite.
// Cholesky factor R (upper, S = R^T R) and its inverse; false when a pivot
// keeps at most tau of its column's squared norm S_jj (the column depends on
// the earlier ones: for a duplicated column the pivot is the FP64 rounding of
// the factorisation, about 1e-16 S_jj, of either sign) or is not finite.
__device__ bool dev_chol_inv(int nb, const double* S, double* R, double* Ri, double tau) {
  for (int e = 0; e < nb * nb; ++e) R[e] = Ri[e] = 0.0;
  for (int j = 0; j < nb; ++j) {
    double d = S[j * nb + j];
    for (int k = 0; k < j; ++k) d -= R[k * nb + j] * R[k * nb + j];
    if (!(d > tau * S[j * nb + j]) || !isfinite(d)) return false;
    const double rjj = sqrt(d);
    R[j * nb + j] = rjj;
    for (int i = j + 1; i < nb; ++i) {
      double t = 0.5 * (S[j * nb + i] + S[i * nb + j]);
      for (int k = 0; k < j; ++k) t -= R[k * nb + j] * R[k * nb + i];
      R[j * nb + i] = t / rjj;
    }
  }
  for (int j = 0; j < nb; ++j) {
    Ri[j * nb + j] = 1.0 / R[j * nb + j];
    for (int i = j - 1; i >= 0; --i) {
      double t = 0.0;
      for (int k = i + 1; k <= j; ++k) t += R[i * nb + k] * Ri[k * nb + j];
      Ri[i * nb + j] = -t / R[i * nb + i];
    }
  }
  return true;
}

__global__ void __launch_bounds__(64) k_ortho_small(int stage, int prec, int g, int nb, const double* __restrict__ G,
                                                    double* work, void* coef, void* rinv, int* status, double drop2) {
  __shared__ double S[64], R[64], Ri[64];
  const int t = threadIdx.x;
  if (stage == 1) {
    for (int e = t; e < g * nb; e += blockDim.x) store_coef(prec, coef, e, -G[e]);
    if (t < nb) work[t] = G[(g + t) * nb + t];
    return;
  }
  if (stage == 2) {
    for (int e = t; e < g * nb; e += blockDim.x) store_coef(prec, coef, e, -G[e]);
    for (int e = t; e < nb * nb; e += blockDim.x) {
      const int i = e / nb, j = e % nb;
      double v = G[(g + i) * nb + j];
      for (int l = 0; l < g; ++l) v -= G[l * nb + i] * G[l * nb + j];
      S[e] = v;
    }
  } else {
    for (int e = t; e < nb * nb; e += blockDim.x) S[e] = G[e];
  }
  __syncthreads();
  if (t == 0) {
    int st = 0;
    if (stage == 2)
      for (int j = 0; j < nb; ++j)
        if (!(S[j * nb + j] > drop2 * fmax(work[j], 1e-300))) st |= 1;
    if (!dev_chol_inv(nb, S, R, Ri, 1e-14)) {  // the host repair's rank rule
      st |= 2;
      for (int e = 0; e < nb * nb; ++e) Ri[e] = (e / nb == e % nb) ? 1.0 : 0.0;
    }
    if (st) atomicOr(status, st);
  }
  __syncthreads();
  for (int e = t; e < nb * nb; e += blockDim.x) store_coef(prec, stage == 2 ? rinv : coef, e, Ri[e]);
}

// CTAs of `kernel` that are resident on the whole GPU at once (per device and
// kernel, cached): a grid-stride kernel launched with more CTAs than this runs
// a partial last wave.
inline int resident_ctas(const void* kernel, int threads) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, int> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find({dev, kernel});
  if (it != cache.end()) return it->second;
  int per_sm = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess) {
    cudaGetLastError();
    per_sm = 1;
  }
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    sms = 152;
  }
  const int r = std::max(1, per_sm) * std::max(1, sms);
  cache[{dev, kernel}] = r;
  return r;
}

inline int persistent_grid(long long work_items, int per_block) {
  long long g = (work_items + per_block - 1) / per_block;
  const long long cap = 152LL * 16;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

template <class P, class F>
cudaError_t dispatch(int prec, F&& f) {
  (void)sizeof(P);
  return f();
}

}  // namespace

// ===========================================================================
// Launch wrappers
// ===========================================================================
#define PHSVDS_DISPATCH(prec, CALL)        \
  switch (prec) {                          \
    case kF32: {                           \
      using P = PF32;                      \
      return CALL;                         \
    }                                      \
    case kDF64: {                          \
      using P = PDF64;                     \
      return CALL;                         \
    }                                      \
    case kF64: {                           \
      using P = PF64;                      \
      return CALL;                         \
    }                                      \
    default:                               \
      return cudaErrorInvalidValue;        \
  }

static SegArr make_segs(const SegV* P, int nseg, int* ptotal) {
  SegArr sa{};
  int tot = 0;
  for (int s = 0; s < 3; ++s) {
    sa.p[s] = s < nseg ? P[s].p : nullptr;
    sa.ld[s] = s < nseg ? P[s].ld : 0;
    sa.nc[s] = s < nseg ? P[s].nc : 0;
    if (s < nseg) tot += P[s].nc;
  }
  sa.n = nseg;
  *ptotal = tot;
  return sa;
}

cudaError_t launch_spmm(int prec, const CsrDev& A, const void* X, long long ldx, void* Y, long long ldy, int b,
                        cudaStream_t st) {
  if (A.rows == 0 || b == 0) return cudaSuccess;
  PHSVDS_DISPATCH(prec, spmm_p<P>(A, X, ldx, Y, ldy, b, st))
}

// ---------------------------------------------------------------------------
// Row Gram: partial[blk] = P^T Q over rows [r0, r1) for P of at most
// kRowGramP columns (up to 3 segments) and Q of at most 8.  TPR lanes share a
// row: lane `part` owns the columns part + TPR k (k < KP) of P and all
// columns of Q, so the loads of a row are coalesced across its lanes and nothing is
// staged in shared memory.  Products are accumulated FP64-class as in the
// tiled Gram (Dot2: exact product, TwoSum into hi, the rounding errors into
// lo, renormalised every 2 rows); the rows of a CTA are reduced in a fixed
// order (shuffles within a warp, then the warps in turn), so results are
// deterministic.
// ---------------------------------------------------------------------------
constexpr int kRowGramP = 64;

template <class P>
struct RAcc;
template <>
struct RAcc<PF32> {
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
struct RAcc<PDF64> {
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
struct RAcc<PF64> {
  double v = 0.0;
  __device__ __forceinline__ void add(double x, double y) { v = fma(x, y, v); }
  __device__ __forceinline__ void norm() {}
  __device__ __forceinline__ double get() const { return v; }
};

template <class P>
__device__ __forceinline__ typename P::G shfl_down_g(typename P::G v, int delta) {
  if constexpr (P::id == kF64) {
    return __shfl_down_sync(0xffffffffu, v, delta);
  } else {
    return df{__shfl_down_sync(0xffffffffu, v.hi, delta), __shfl_down_sync(0xffffffffu, v.lo, delta)};
  }
}

template <class P, int TPR, int KP, int NQ>
__global__ void __launch_bounds__(kThreads) k_gram_row(long long r0, long long r1, SegArr segs, int p,
                                                       const typename P::S* __restrict__ Q, long long ldq, int q,
                                                       typename P::G* __restrict__ partial) {
  using S = typename P::S;
  using A = typename P::A;
  using G = typename P::G;
  constexpr int RPC = kThreads / TPR;  // rows of a CTA pass
  constexpr int NW = kThreads / 32;
  __shared__ G red[NW * kRowGramP * 8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int part = lane % TPR;
  // the P columns of this lane: base pointer and row stride, resolved once
  const S* cb[KP];
  long long cl[KP];
  bool cv[KP];
#pragma unroll
  for (int k = 0; k < KP; ++k) {
    int c = part + TPR * k;
    cv[k] = c < p;
    int s = 0;
    while (s < segs.n - 1 && c >= segs.nc[s]) {
      c -= segs.nc[s];
      ++s;
    }
    cb[k] = cv[k] ? reinterpret_cast<const S*>(segs.p[s]) + c : nullptr;
    cl[k] = cv[k] ? segs.ld[s] : 0;
  }
  RAcc<P> acc[KP][NQ];
  const long long stride = (long long)gridDim.x * RPC;
  // two rows per iteration (loads of both issued before the products), then
  // the accumulators are renormalised
  for (long long ra = r0 + (long long)blockIdx.x * RPC + threadIdx.x / TPR; ra < r1; ra += 2 * stride) {
    const long long rb = ra + stride;
    const bool hb = rb < r1;
    A xa[KP], xb[KP], ya[NQ], yb[NQ];
#pragma unroll
    for (int k = 0; k < KP; ++k) {
      xa[k] = cv[k] ? P::load(cb[k] + ra * cl[k]) : P::zero();
      xb[k] = (cv[k] && hb) ? P::load(cb[k] + rb * cl[k]) : P::zero();
    }
#pragma unroll
    for (int j = 0; j < NQ; ++j) {
      ya[j] = j < q ? P::load(Q + ra * ldq + j) : P::zero();
      yb[j] = (j < q && hb) ? P::load(Q + rb * ldq + j) : P::zero();
    }
#pragma unroll
    for (int k = 0; k < KP; ++k)
#pragma unroll
      for (int j = 0; j < NQ; ++j) {
        acc[k][j].add(xa[k], ya[j]);
        acc[k][j].add(xb[k], yb[j]);
        acc[k][j].norm();
      }
  }
  // lanes of equal `part` in a warp: tree of shuffles in a fixed order
#pragma unroll
  for (int k = 0; k < KP; ++k)
#pragma unroll
    for (int j = 0; j < NQ; ++j) {
      G v = acc[k][j].get();
#pragma unroll
      for (int off = 16; off >= TPR; off >>= 1) v = P::gadd(v, shfl_down_g<P>(v, off));
      const int c = part + TPR * k;
      if (lane < TPR && c < p && j < q) red[(warp * p + c) * q + j] = v;
    }
  __syncthreads();
  const int pq = p * q;
  for (int e = threadIdx.x; e < pq; e += kThreads) {
    G v = red[e];
    for (int w = 1; w < NW; ++w) v = P::gadd(v, red[w * pq + e]);
    partial[(long long)blockIdx.x * pq + e] = v;
  }
}

// ---------------------------------------------------------------------------
// Anchored row Gram (F32 storage): the row Gram's layout (TPR lanes
// per row, lane `part` owns P columns part + TPR k and every Q column) with a
// cheaper FP64-class accumulation.  Pair (i, j) of a lane accumulates into
// s = sigma_ij + (partial sum), where sigma_ij = a_i b_j is a power of two of
// at least 4 times the Cauchy-Schwarz bound sqrt(SP_i SQ_j) of every partial
// sum of the lane (SP, SQ: running sums of squares of the lane's entries).
// s then stays within a factor 2 of sigma at every step, so
//     s' = fma(p, q, s),  z = s' - s  (exact: Sterbenz),  d = fma(p, q, -z)
// is the rounding error of the update to FP32 precision, and d is summed in
// c: 4 FP32 operations per product instead of the 10 of Dot2 (double-float
// data keeps Dot2: this scheme's 2^-43 falls short of its 2^-48).  When a running sum of squares outgrows its anchor, the
// anchor is raised with 4x headroom and the pairs concerned move to it by an
// error-free FastTwoSum; every 8 rows c is folded into s (FastTwoSum), so |c|
// stays within a few units of sigma's last place.  The error of a product is
// about 2^-47 sigma_ij, i.e. 2^-43 of the Cauchy-Schwarz bound of the lane's
// rows.  Lane results are reduced in double-float in a fixed order as in the
// row Gram (deterministic).  Entries must be below 2^50 in magnitude (the
// anchors and sums of squares stay finite); the solver's blocks are far inside.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float hi_part(float x) { return x; }
__device__ __forceinline__ float hi_part(df x) { return x.hi; }

__device__ __forceinline__ void anc_add(float& s, float& c, float x, float y) {
  const float t = s;
  s = __fmaf_rn(x, y, t);
  const float z = __fsub_rn(s, t);
  c = __fadd_rn(c, __fmaf_rn(x, y, -z));
}

// Smallest power of two a with a^2 >= 18 sp (4x headroom over a^2 >= 4.5 sp),
// and at least 2^-58: the floor keeps the bound valid for entries whose
// squares underflow (below 2^-75) over up to 2^32 rows.
__device__ __forceinline__ float anc_anchor(float sp) {
  const unsigned u = __float_as_uint(18.0f * sp);
  int e = (int)(u >> 23) - 127;
  if (u & 0x7fffffu) ++e;  // ceil(log2 x) (conservative for subnormal x)
  int ea = (e + 1) >> 1;   // ceil(e / 2)
  ea = max(ea, -58);
  return __uint_as_float((unsigned)(ea + 127) << 23);
}

template <class P, int TPR, int KP, int NQ>
__global__ void __launch_bounds__(kThreads) k_gram_anc(long long r0, long long r1, SegArr segs, int p,
                                                       const typename P::S* __restrict__ Q, long long ldq, int q,
                                                       df* __restrict__ partial) {
  using S = typename P::S;
  using A = typename P::A;
  constexpr int RPC = kThreads / TPR;  // rows of a CTA pass
  constexpr int NW = kThreads / 32;
  constexpr float kFloor = 3.4694470e-18f;  // 2^-58
  __shared__ df red[NW * kRowGramP * 8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int part = lane % TPR;
  const S* cb[KP];
  long long cl[KP];
  bool cv[KP];
#pragma unroll
  for (int k = 0; k < KP; ++k) {
    int c = part + TPR * k;
    cv[k] = c < p;
    int sg = 0;
    while (sg < segs.n - 1 && c >= segs.nc[sg]) {
      c -= segs.nc[sg];
      ++sg;
    }
    cb[k] = cv[k] ? reinterpret_cast<const S*>(segs.p[sg]) + c : nullptr;
    cl[k] = cv[k] ? segs.ld[sg] : 0;
  }
  float sa[KP][NQ], ca[KP][NQ];
  float an[KP], bn[NQ], ta[KP], tb[NQ], sp[KP], sq[NQ];
  const float thr0 = kFloor * kFloor * (1.0f / 4.5f);
#pragma unroll
  for (int k = 0; k < KP; ++k) {
    an[k] = kFloor;
    ta[k] = thr0;
    sp[k] = 0.f;
  }
#pragma unroll
  for (int j = 0; j < NQ; ++j) {
    bn[j] = kFloor;
    tb[j] = thr0;
    sq[j] = 0.f;
  }
#pragma unroll
  for (int k = 0; k < KP; ++k)
#pragma unroll
    for (int j = 0; j < NQ; ++j) {
      sa[k][j] = kFloor * kFloor;
      ca[k][j] = 0.f;
    }
  const long long stride = (long long)gridDim.x * RPC;
  int it = 0;
  for (long long ra = r0 + (long long)blockIdx.x * RPC + threadIdx.x / TPR; ra < r1; ra += 2 * stride) {
    const long long rb = ra + stride;
    const bool hb = rb < r1;
    A xa[KP], xb[KP], ya[NQ], yb[NQ];
#pragma unroll
    for (int k = 0; k < KP; ++k) {
      xa[k] = cv[k] ? P::load(cb[k] + ra * cl[k]) : P::zero();
      xb[k] = (cv[k] && hb) ? P::load(cb[k] + rb * cl[k]) : P::zero();
    }
#pragma unroll
    for (int j = 0; j < NQ; ++j) {
      ya[j] = j < q ? P::load(Q + ra * ldq + j) : P::zero();
      yb[j] = (j < q && hb) ? P::load(Q + rb * ldq + j) : P::zero();
    }
    // running sums of squares, then raise the anchors that they outgrew
#pragma unroll
    for (int k = 0; k < KP; ++k) {
      sp[k] = __fmaf_rn(hi_part(xa[k]), hi_part(xa[k]), sp[k]);
      sp[k] = __fmaf_rn(hi_part(xb[k]), hi_part(xb[k]), sp[k]);
    }
#pragma unroll
    for (int j = 0; j < NQ; ++j) {
      sq[j] = __fmaf_rn(hi_part(ya[j]), hi_part(ya[j]), sq[j]);
      sq[j] = __fmaf_rn(hi_part(yb[j]), hi_part(yb[j]), sq[j]);
    }
#pragma unroll
    for (int k = 0; k < KP; ++k)
      if (sp[k] > ta[k]) {
        const float a1 = anc_anchor(sp[k]);
#pragma unroll
        for (int j = 0; j < NQ; ++j) {
          const float so = an[k] * bn[j], sn = a1 * bn[j];
          const float v = __fsub_rn(sa[k][j], so);
          const float t = __fadd_rn(sn, v);
          ca[k][j] = __fadd_rn(ca[k][j], __fsub_rn(v, __fsub_rn(t, sn)));
          sa[k][j] = t;
        }
        an[k] = a1;
        ta[k] = a1 * a1 * (1.0f / 4.5f);
      }
#pragma unroll
    for (int j = 0; j < NQ; ++j)
      if (sq[j] > tb[j]) {
        const float b1 = anc_anchor(sq[j]);
#pragma unroll
        for (int k = 0; k < KP; ++k) {
          const float so = an[k] * bn[j], sn = an[k] * b1;
          const float v = __fsub_rn(sa[k][j], so);
          const float t = __fadd_rn(sn, v);
          ca[k][j] = __fadd_rn(ca[k][j], __fsub_rn(v, __fsub_rn(t, sn)));
          sa[k][j] = t;
        }
        bn[j] = b1;
        tb[j] = b1 * b1 * (1.0f / 4.5f);
      }
#pragma unroll
    for (int k = 0; k < KP; ++k)
#pragma unroll
      for (int j = 0; j < NQ; ++j) {
        anc_add(sa[k][j], ca[k][j], xa[k], ya[j]);
        anc_add(sa[k][j], ca[k][j], xb[k], yb[j]);
      }
    if ((++it & 3) == 0) {  // every 8 rows: fold c into s (|s| >= |c|)
#pragma unroll
      for (int k = 0; k < KP; ++k)
#pragma unroll
        for (int j = 0; j < NQ; ++j) {
          const float t = __fadd_rn(sa[k][j], ca[k][j]);
          ca[k][j] = __fsub_rn(ca[k][j], __fsub_rn(t, sa[k][j]));
          sa[k][j] = t;
        }
    }
  }
  // lanes of equal `part` in a warp: tree of shuffles in a fixed order
#pragma unroll
  for (int k = 0; k < KP; ++k)
#pragma unroll
    for (int j = 0; j < NQ; ++j) {
      const float v = __fsub_rn(sa[k][j], an[k] * bn[j]);  // exact
      df g = two_sum(v, ca[k][j]);
#pragma unroll
      for (int off = 16; off >= TPR; off >>= 1)
        g = df_add(g, df{__shfl_down_sync(0xffffffffu, g.hi, off), __shfl_down_sync(0xffffffffu, g.lo, off)});
      const int c = part + TPR * k;
      if (lane < TPR && c < p && j < q) red[(warp * p + c) * q + j] = g;
    }
  __syncthreads();
  const int pq = p * q;
  for (int e = threadIdx.x; e < pq; e += kThreads) {
    df v = red[e];
    for (int w = 1; w < NW; ++w) v = df_add(v, red[w * pq + e]);
    partial[(long long)blockIdx.x * pq + e] = v;
  }
}

template <class P>
cudaError_t gram_row_p(long long r0, long long r1, const SegArr& sa, int p, SegV Q, void* partial, int max_blocks,
                       int* nblocks, cudaStream_t st) {
  using S = typename P::S;
  using G = typename P::G;
  const S* q = reinterpret_cast<const S*>(Q.p);
  G* out = reinterpret_cast<G*>(partial);
  const long long rows = r1 > r0 ? r1 - r0 : 0;
#define ROWG(TPRV, KPV, NQV)                                                                              \
  {                                                                                                       \
    int grid = persistent_grid((rows + kThreads / TPRV - 1) / (kThreads / TPRV), 1);                      \
    if (grid > max_blocks) grid = max_blocks;                                                             \
    if (grid < 1) grid = 1;                                                                               \
    *nblocks = grid;                                                                                      \
    if constexpr (P::id != kF32) {                                                                        \
      k_gram_row<P, TPRV, KPV, NQV><<<grid, kThreads, 0, st>>>(r0, r1, sa, p, q, Q.ld, Q.nc, out);        \
    } else {                                                                                              \
      k_gram_anc<P, TPRV, KPV, NQV><<<grid, kThreads, 0, st>>>(r0, r1, sa, p, q, Q.ld, Q.nc, out);        \
    }                                                                                                     \
    return cudaGetLastError();                                                                            \
  }
#define ROWG_Q4(TPRV, KPV)           \
  {                                  \
    if (Q.nc <= 1) ROWG(TPRV, KPV, 1) \
    if (Q.nc <= 2) ROWG(TPRV, KPV, 2) \
    ROWG(TPRV, KPV, 4)               \
  }
#define ROWG_Q(TPRV, KPV)  \
  {                        \
    if (Q.nc <= 4) ROWG_Q4(TPRV, KPV) \
    ROWG(TPRV, KPV, 8)     \
  }
  // lanes per row and P columns per lane: few idle lanes for p up to 64 at
  // moderate register use (6 columns of 8 lanes when p <= 48 and q <= 4)
  if (p <= 8) ROWG_Q(2, 4)
  if (p <= 16) ROWG_Q(4, 4)
  if (p <= 32) ROWG_Q(8, 4)
  if (p <= 48 && Q.nc <= 4) ROWG_Q4(8, 6)
  ROWG_Q(16, 4)
#undef ROWG_Q
#undef ROWG_Q4
#undef ROWG
}

cudaError_t launch_precond_check(long long n, const int* rowptr, const int* colidx, const float* v32,
                                 const double* v64, int* flags, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (!v32 && !v64) return cudaErrorInvalidValue;
  k_precond_check<<<std::min(grid_for(n, kThreads), 152 * 8), kThreads, 0, st>>>(n, rowptr, colidx, v32, v64, flags);
  return cudaGetLastError();
}

size_t gram_partial_bytes(int max_blocks, int p, int q) { return (size_t)max_blocks * p * q * 8; }
int gram_default_blocks() { return 152 * 4; }

cudaError_t launch_gram(int prec, long long r0, long long r1, const SegV* Pp, int nseg, SegV Q, void* partial,
                        int max_blocks, int* nblocks, cudaStream_t st) {
  int p;
  SegArr sa = make_segs(Pp, nseg, &p);
  if (p < 1 || p > kGramThreads || Q.nc < 1 || Q.nc > kGramQ || nseg < 1 || nseg > 3) return cudaErrorInvalidValue;
  if (r1 <= r0) {  // empty row range: one block of zeros
    r1 = r0;
  }
  if (p <= kRowGramP && Q.nc <= 8) {
    if (prec != kF64) {
      const cudaError_t e = launch_gram_tma(prec, r0, r1, Pp, nseg, Q, partial, max_blocks, nblocks, st);
      if (e != cudaErrorNotSupported) return e;
      cudaGetLastError();
    }
    PHSVDS_DISPATCH(prec, gram_row_p<P>(r0, r1, sa, p, Q, partial, max_blocks, nblocks, st))
  }
  {
    SegV all[4];
    for (int s = 0; s < nseg; ++s) all[s] = Pp[s];
    all[nseg] = Q;
    TileDesc T;
    if (make_tiles(all, nseg + 1, elem_bytes(prec), false, &T))
      return tiled_gram(prec, T, r0, r1, p, Q.nc, partial, max_blocks, nblocks, st);
  }
  PHSVDS_DISPATCH(prec, gram_p<P>(r0, r1, sa, p, Q, partial, max_blocks, nblocks, st))
}

cudaError_t launch_gram_reduce(int prec, const void* partial, int nblocks, int pq, double* G, cudaStream_t st) {
  return tiled_reduce(prec, partial, nblocks, pq, G, st);
}

template <class P>
static cudaError_t combine_p(long long L, const SegArr& sa, int p, const void* coef, const void* In, long long ldin,
                             int alpha_one, void* Out, long long ldout, int q, const void* Rinv, void* Out2,
                             long long ldout2, cudaStream_t st) {
  using S = typename P::S;
  using C = typename P::C;
  const size_t sm = combine_smem<P>(p, q, Rinv != nullptr);
  if (sm > 200 * 1024) return cudaErrorInvalidValue;
  {
    const cudaError_t e = smem_optin(reinterpret_cast<const void*>(k_combine<P>), 200 * 1024);
    if (e != cudaSuccess) return e;
  }
  const int grid = persistent_grid((L + kCmbRows - 1) / kCmbRows, 1);
  k_combine<P><<<grid, kCmbThreads, sm, st>>>(L, sa, p, reinterpret_cast<const C*>(coef), reinterpret_cast<const S*>(In),
                                              ldin, alpha_one, reinterpret_cast<S*>(Out), ldout, q,
                                              reinterpret_cast<const C*>(Rinv), reinterpret_cast<S*>(Out2), ldout2);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Row combine: one thread per row streams its p inputs (16-byte loads when
// every segment row is 16-byte aligned), keeps the q outputs in registers and
// writes them after all reads, so Out may alias an input segment or In.  The
// coefficients (and R^-1) sit in shared memory and are read as broadcasts.
// ---------------------------------------------------------------------------
constexpr int kRowCombP = 64;

template <class P>
__device__ __forceinline__ typename P::A mul_a(typename P::A a, typename P::A b) {
  if constexpr (P::id == kDF64) {
    return df_mul(a, b);
  } else {
    return a * b;
  }
}

template <class P>
__device__ __forceinline__ typename P::G shfl_down_gacc(typename P::G v, int o) {
  if constexpr (P::id == kF64) {
    return __shfl_down_sync(0xffffffffu, v, o);
  } else {
    return df{__shfl_down_sync(0xffffffffu, v.hi, o), __shfl_down_sync(0xffffffffu, v.lo, o)};
  }
}


template <class P>
__device__ __forceinline__ typename P::A shfl_a(typename P::A v, int lane) {
  if constexpr (P::id == kDF64) {
    return df{__shfl_sync(0xffffffffu, v.hi, lane), __shfl_sync(0xffffffffu, v.lo, lane)};
  } else {
    return __shfl_sync(0xffffffffu, v, lane);
  }
}

// one 16-byte load of W = 16 / sizeof(S) consecutive elements (no local array)
template <class P>
__device__ __forceinline__ void load16(const typename P::S* p, typename P::A (&x)[16 / sizeof(typename P::S)]) {
  if constexpr (P::id == kF32) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    x[0] = t.x;
    x[1] = t.y;
    x[2] = t.z;
    x[3] = t.w;
  } else if constexpr (P::id == kDF64) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    x[0] = df{t.x, t.y};
    x[1] = df{t.z, t.w};
  } else {
    const double2 t = *reinterpret_cast<const double2*>(p);
    x[0] = t.x;
    x[1] = t.y;
  }
}

// One thread per row: it streams the row's p inputs (16-byte loads for the
// aligned bulk of each segment, scalar loads for the tail), keeps its QT >= q
// outputs in registers and writes them after all reads, so Out may alias an
// input segment or In.  The coefficients (and R^-1) sit in shared memory and
// every lane of a warp reads the same address (a broadcast).
template <class P, int QT, bool VEC>
__global__ void __launch_bounds__(kThreads, (QT <= 4 && P::id != kDF64) ? 4 : 2) k_combine_row(long long L, SegArr segs, int p, int q,
                                                          const typename P::C* __restrict__ coef,
                                                          const typename P::S* In, long long ldin, int alpha_one,
                                                          typename P::S* Out, long long ldout,
                                                          const typename P::C* __restrict__ Rinv,
                                                          typename P::S* Out2, long long ldout2) {
  using S = typename P::S;
  using A = typename P::A;
  using C = typename P::C;
  constexpr int QR = QT <= 8 ? QT : 1;  // R^-1 is applied for q <= 8 only
  __shared__ C cs[kRowCombP * QT];
  __shared__ C rs[QR * QR];
  for (int e = threadIdx.x; e < p * QT; e += kThreads) {
    const int c = e / QT, j = e % QT;
    cs[e] = j < q ? coef[(long long)c * q + j] : C{};
  }
  if (QT <= 8 && Rinv)
    for (int e = threadIdx.x; e < QT * QT; e += kThreads) {
      const int i = e / QT, j = e % QT;
      rs[e] = (i < q && j < q) ? Rinv[i * q + j] : C{};
    }
  __syncthreads();
  const long long stride = (long long)gridDim.x * kThreads;
  for (long long r = (long long)blockIdx.x * kThreads + threadIdx.x; r < L; r += stride) {
    A acc[QT];
#pragma unroll
    for (int j = 0; j < QT; ++j) acc[j] = (alpha_one && j < q) ? P::load(In + r * ldin + j) : P::zero();
    int c0 = 0;
    for (int sg = 0; sg < segs.n; ++sg) {
      const S* row = reinterpret_cast<const S*>(segs.p[sg]) + r * segs.ld[sg];
      const int nc = segs.nc[sg];
      int c1 = 0;  // first column of the scalar tail
      if constexpr (VEC) {
        constexpr int W = (int)(16 / sizeof(S));
        constexpr int U = QT <= 8 ? 4 : 2;  // 16-byte loads in flight per thread
        c1 = nc - nc % W;
        int c = 0;
        for (; c + U * W <= c1; c += U * W) {
          A xs[U][W];
#pragma unroll
          for (int u = 0; u < U; ++u) load16<P>(row + c + u * W, xs[u]);
#pragma unroll
          for (int u = 0; u < U; ++u)
#pragma unroll
            for (int w = 0; w < W; ++w) {
              const C* cr = cs + (c0 + c + u * W + w) * QT;
#pragma unroll
              for (int j = 0; j < QT; ++j) acc[j] = P::fmac(acc[j], xs[u][w], cr[j]);
            }
        }
        for (; c < c1; c += W) {
          A xs[W];
          load16<P>(row + c, xs);
#pragma unroll
          for (int w = 0; w < W; ++w) {
            const C* cr = cs + (c0 + c + w) * QT;
#pragma unroll
            for (int j = 0; j < QT; ++j) acc[j] = P::fmac(acc[j], xs[w], cr[j]);
          }
        }
      }
      for (int c = c1; c < nc; ++c) {
        const A x = P::load(row + c);
        const C* cr = cs + (c0 + c) * QT;
#pragma unroll
        for (int j = 0; j < QT; ++j) acc[j] = P::fmac(acc[j], x, cr[j]);
      }
      c0 += nc;
    }
    if constexpr (QT <= 8) {
      if (Rinv) {  // acc_j <- sum_{i <= j} acc_i Rinv_ij, in place from the last column down
#pragma unroll
        for (int j = QT - 1; j >= 0; --j) {
          A t = P::zero();
#pragma unroll
          for (int i = 0; i <= j; ++i) t = P::fmac(t, acc[i], rs[i * QT + j]);
          acc[j] = t;
        }
      }
    }
#pragma unroll
    for (int j = 0; j < QT; ++j)
      if (j < q) {
        P::store(Out + r * ldout + j, acc[j]);
        if (Out2) P::store(Out2 + r * ldout2 + j, acc[j]);
      }
  }
}

template <class P>
cudaError_t combine_row_p(long long L, const SegArr& sa, int p, const void* coef, const void* In, long long ldin,
                          int alpha_one, void* Out, long long ldout, int q, const void* Rinv, void* Out2,
                          long long ldout2, cudaStream_t st) {
  using S = typename P::S;
  using C = typename P::C;
  // 16-byte loads for the aligned bulk of each segment's row, scalar loads for
  // its last columns (segment widths need not be multiples of 16 bytes)
  bool vec = true;
  for (int sg = 0; sg < sa.n; ++sg)
    vec = vec && (reinterpret_cast<uintptr_t>(sa.p[sg]) % 16 == 0) && ((sa.ld[sg] * sizeof(S)) % 16 == 0);
  const C* cf = reinterpret_cast<const C*>(coef);
  const C* ri = reinterpret_cast<const C*>(Rinv);
  const S* in = reinterpret_cast<const S*>(In);
  S* out = reinterpret_cast<S*>(Out);
  S* out2 = reinterpret_cast<S*>(Out2);
#define ROWC(QTV)                                                                                                  \
  {                                                                                                                \
    const int grid = persistent_grid((L + kThreads - 1) / kThreads, 1);                                           \
    if (vec)                                                                                                       \
      k_combine_row<P, QTV, true><<<grid, kThreads, 0, st>>>(L, sa, p, q, cf, in, ldin, alpha_one, out, ldout, ri,  \
                                                             out2, ldout2);                                        \
    else                                                                                                           \
      k_combine_row<P, QTV, false><<<grid, kThreads, 0, st>>>(L, sa, p, q, cf, in, ldin, alpha_one, out, ldout, ri, \
                                                              out2, ldout2);                                       \
    return cudaGetLastError();                                                                                     \
  }
  if (q <= 4) ROWC(4)
  if (q <= 8) ROWC(8)
  if (q <= 16) ROWC(16)
  if (q <= 24) ROWC(24)
  if (q <= 32) ROWC(32)
#undef ROWC
  return cudaErrorInvalidValue;
}

cudaError_t launch_combine(int prec, long long L, const SegV* Pp, int nseg, const void* coef, const void* In,
                           long long ldin, int alpha_one, void* Out, long long ldout, int q, const void* Rinv,
                           void* Out2, long long ldout2, cudaStream_t st) {
  if (L == 0 || q == 0) return cudaSuccess;
  int p;
  SegArr sa = make_segs(Pp, nseg, &p);
  if (nseg < 1 || nseg > 3 || p < 1) return cudaErrorInvalidValue;
  if (prec != kF64) {
    const cudaError_t e =
        launch_combine_tma(prec, L, Pp, nseg, coef, In, ldin, alpha_one, Out, ldout, q, Rinv, Out2, ldout2, st);
    if (e != cudaErrorNotSupported) return e;
  }
  if (p <= kRowCombP && q <= 32 && (!Rinv || q <= 8)) {
    PHSVDS_DISPATCH(prec, combine_row_p<P>(L, sa, p, coef, In, ldin, alpha_one, Out, ldout, q, Rinv, Out2, ldout2,
                                           st))
  }
  {
    TileDesc T;
    if (make_tiles(Pp, nseg, elem_bytes(prec), true, &T)) {
      cudaError_t e = tiled_combine(prec, T, L, p, coef, In, ldin, alpha_one, Out, ldout, q, Rinv, Out2, ldout2, st);
      if (e != cudaErrorInvalidValue) return e;
    }
  }
  PHSVDS_DISPATCH(prec, combine_p<P>(L, sa, p, coef, In, ldin, alpha_one, Out, ldout, q, Rinv, Out2, ldout2, st))
}

template <class P>
static cudaError_t ritz_p(long long L, SegV V, SegV W, int g, const void* Y, const void* theta, void* X, void* R,
                          long long ldb, int nb, const void* dscale, void* T, void* partial, int max_blocks,
                          int* nblocks, cudaStream_t st) {
  using S = typename P::S;
  using C = typename P::C;
  using A = typename P::A;
  using G = typename P::G;
  const size_t sm = sizeof(A) * 2 * (size_t)kCmbRows * (g + 1) + sizeof(C) * ((size_t)g * nb + nb) +
                    sizeof(G) * (size_t)kCmbRows * nb + 16;
  if (sm > 200 * 1024) return cudaErrorInvalidValue;
  {
    const cudaError_t e = smem_optin(reinterpret_cast<const void*>(k_ritz_residual<P>), 200 * 1024);
    if (e != cudaSuccess) return e;
  }
  int grid = persistent_grid((L + kCmbRows - 1) / kCmbRows, 1);
  if (grid > max_blocks) grid = max_blocks;
  *nblocks = grid;
  k_ritz_residual<P><<<grid, kCmbThreads, sm, st>>>(
      L, reinterpret_cast<const S*>(V.p), V.ld, reinterpret_cast<const S*>(W.p), W.ld, g,
      reinterpret_cast<const C*>(Y), reinterpret_cast<const C*>(theta), reinterpret_cast<S*>(X),
      reinterpret_cast<S*>(R), ldb, nb, reinterpret_cast<const S*>(dscale), reinterpret_cast<S*>(T),
      reinterpret_cast<G*>(partial));
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Row Ritz kernel: TPR lanes share a row (lane part owns the block columns
// 4 part .. 4 part + 3); X = V Y and R = W Y - X diag(theta) from streamed rows
// of V and W, optional T = diag(d) R, and FP64-class partial sums of R^2 per
// column (fixed shuffle butterfly, then warps in order): partial[blk][j].
// ---------------------------------------------------------------------------
template <class P, int TPR, bool VEC>
__global__ void __launch_bounds__(kThreads) k_ritz_row(long long L, const typename P::S* __restrict__ V,
                                                       const typename P::S* __restrict__ W, long long ldv, int g,
                                                       const typename P::C* __restrict__ Y,
                                                       const typename P::C* __restrict__ theta,
                                                       typename P::S* __restrict__ X, typename P::S* __restrict__ R,
                                                       long long ldb, int nb, const typename P::S* __restrict__ dscale,
                                                       typename P::S* __restrict__ T, typename P::G* __restrict__ partial) {
  using S = typename P::S;
  using A = typename P::A;
  using C = typename P::C;
  using G = typename P::G;
  constexpr int QT = 4, Q = QT * TPR;
  __shared__ C ys[kRowCombP * Q];
  __shared__ C th[Q];
  for (int e = threadIdx.x; e < g * Q; e += kThreads) {
    const int c = e / Q, j = e % Q;
    ys[e] = j < nb ? Y[(long long)c * nb + j] : C{};
  }
  if (threadIdx.x < Q) th[threadIdx.x] = threadIdx.x < nb ? theta[threadIdx.x] : C{};
  __syncthreads();
  const int part = threadIdx.x % TPR, j0 = part * QT;
  G nrm[QT];
#pragma unroll
  for (int j = 0; j < QT; ++j) nrm[j] = P::gzero();
  const long long rows_per_pass = (long long)gridDim.x * (kThreads / TPR);
  for (long long r = (long long)blockIdx.x * (kThreads / TPR) + threadIdx.x / TPR; r < L; r += rows_per_pass) {
    A ax[QT], ar[QT];
#pragma unroll
    for (int j = 0; j < QT; ++j) ax[j] = ar[j] = P::zero();
    const S* vr = V + r * ldv;
    const S* wr = W + r * ldv;
    int c1 = 0;  // first column of the scalar tail
    if constexpr (VEC) {
      constexpr int WW = (int)(16 / sizeof(S));
      constexpr int U = 2;  // row segments of V and W in flight per thread
      c1 = g - g % WW;
      int c = 0;
      for (; c + U * WW <= c1; c += U * WW) {
        A xv[U][WW], xw[U][WW];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          load16<P>(vr + c + u * WW, xv[u]);
          load16<P>(wr + c + u * WW, xw[u]);
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
          for (int w = 0; w < WW; ++w) {
            const C* yr = ys + (c + u * WW + w) * Q + j0;
#pragma unroll
            for (int j = 0; j < QT; ++j) {
              ax[j] = P::fmac(ax[j], xv[u][w], yr[j]);
              ar[j] = P::fmac(ar[j], xw[u][w], yr[j]);
            }
          }
      }
      for (; c < c1; c += WW) {
        A xv[WW], xw[WW];
        load16<P>(vr + c, xv);
        load16<P>(wr + c, xw);
#pragma unroll
        for (int w = 0; w < WW; ++w) {
          const C* yr = ys + (c + w) * Q + j0;
#pragma unroll
          for (int j = 0; j < QT; ++j) {
            ax[j] = P::fmac(ax[j], xv[w], yr[j]);
            ar[j] = P::fmac(ar[j], xw[w], yr[j]);
          }
        }
      }
    }
    {
      for (int c = c1; c < g; ++c) {
        const A xv = P::load(vr + c), xw = P::load(wr + c);
        const C* yr = ys + c * Q + j0;
#pragma unroll
        for (int j = 0; j < QT; ++j) {
          ax[j] = P::fmac(ax[j], xv, yr[j]);
          ar[j] = P::fmac(ar[j], xw, yr[j]);
        }
      }
    }
    A dr = P::zero();
    if (T) dr = P::load(dscale + r);
#pragma unroll
    for (int j = 0; j < QT; ++j)
      if (j0 + j < nb) {
        const A rj = P::sub(ar[j], P::mulc(ax[j], th[j0 + j]));
        P::store(X + r * ldb + j0 + j, ax[j]);
        P::store(R + r * ldb + j0 + j, rj);
        if (T) P::store(T + r * ldb + j0 + j, mul_a<P>(dr, rj));
        nrm[j] = P::gfma(nrm[j], rj, rj);
      }
  }
  // lanes of the same part across the warp's rows, then the warps in order
#pragma unroll
  for (int j = 0; j < QT; ++j)
    for (int o = 16; o >= TPR; o >>= 1) nrm[j] = P::gadd(nrm[j], shfl_down_gacc<P>(nrm[j], o));
  __shared__ G red[kThreads / 32][Q];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane < TPR)
#pragma unroll
    for (int j = 0; j < QT; ++j) red[warp][lane * QT + j] = nrm[j];
  __syncthreads();
  if ((int)threadIdx.x < nb) {
    G v = red[0][threadIdx.x];
    for (int w = 1; w < kThreads / 32; ++w) v = P::gadd(v, red[w][threadIdx.x]);
    partial[(long long)blockIdx.x * nb + threadIdx.x] = v;
  }
}

template <class P>
cudaError_t ritz_row_p(long long L, SegV V, SegV W, int g, const void* Y, const void* theta, void* X, void* R,
                       long long ldb, int nb, const void* dscale, void* T, void* partial, int max_blocks,
                       int* nblocks, cudaStream_t st) {
  using S = typename P::S;
  using C = typename P::C;
  using G = typename P::G;
  // 16-byte loads for the aligned bulk of each row, scalar loads for its last columns
  const bool vec = reinterpret_cast<uintptr_t>(V.p) % 16 == 0 && reinterpret_cast<uintptr_t>(W.p) % 16 == 0 &&
                   (V.ld * sizeof(S)) % 16 == 0;
  const S* vp = reinterpret_cast<const S*>(V.p);
  const S* wp = reinterpret_cast<const S*>(W.p);
  const C* yp = reinterpret_cast<const C*>(Y);
  const C* tp = reinterpret_cast<const C*>(theta);
  S* xp = reinterpret_cast<S*>(X);
  S* rp = reinterpret_cast<S*>(R);
  const S* dp = reinterpret_cast<const S*>(dscale);
  S* tq = reinterpret_cast<S*>(T);
  G* pd = reinterpret_cast<G*>(partial);
#define RITZR(TPRV)                                                                                                \
  {                                                                                                                \
    long long grid = (L + kThreads / TPRV - 1) / (kThreads / TPRV);                                                \
    if (grid > max_blocks) grid = max_blocks;                                                                      \
    {                                                                                                              \
      const int res = resident_ctas(vec ? reinterpret_cast<const void*>(k_ritz_row<P, TPRV, true>)                 \
                                        : reinterpret_cast<const void*>(k_ritz_row<P, TPRV, false>), kThreads);    \
      if (grid > res) grid = res; /* one full wave: no partial last wave */                                        \
    }                                                                                                              \
    if (grid < 1) grid = 1;                                                                                        \
    *nblocks = (int)grid;                                                                                          \
    if (vec)                                                                                                       \
      k_ritz_row<P, TPRV, true><<<(int)grid, kThreads, 0, st>>>(L, vp, wp, V.ld, g, yp, tp, xp, rp, ldb, nb, dp,   \
                                                                 tq, pd);                                          \
    else                                                                                                           \
      k_ritz_row<P, TPRV, false><<<(int)grid, kThreads, 0, st>>>(L, vp, wp, V.ld, g, yp, tp, xp, rp, ldb, nb, dp,  \
                                                                  tq, pd);                                         \
    return cudaGetLastError();                                                                                     \
  }
  if (nb <= 4) RITZR(1)
  if (nb <= 8) RITZR(2)
#undef RITZR
  return cudaErrorInvalidValue;
}

cudaError_t launch_ritz_residual(int prec, long long L, SegV V, SegV W, int g, const void* Y, const void* theta,
                                 void* X, void* R, long long ldb, int nb, const void* dscale, void* T,
                                 void* norm_partial, int max_blocks, int* nblocks, cudaStream_t st) {
  if (g < 1 || nb < 1) return cudaErrorInvalidValue;
  if (prec != kF64) {
    const cudaError_t e = launch_ritz_tma(prec, L, V, W, g, Y, theta, X, R, ldb, nb, dscale, T, norm_partial,
                                          max_blocks, nblocks, st);
    if (e != cudaErrorNotSupported) return e;
  }
  if (g <= kRowCombP && nb <= 8 && V.ld == W.ld) {
    PHSVDS_DISPATCH(prec, ritz_row_p<P>(L, V, W, g, Y, theta, X, R, ldb, nb, dscale, T, norm_partial, max_blocks,
                                        nblocks, st))
  }
  {
    SegV vw[2] = {SegV{V.p, V.ld, g}, SegV{W.p, W.ld, g}};
    TileDesc TD;
    if (nb <= 16 && make_tiles(vw, 2, elem_bytes(prec), true, &TD)) {
      cudaError_t e = tiled_ritz(prec, TD, L, g, Y, theta, X, R, ldb, nb, dscale, T, norm_partial, max_blocks, nblocks, st);
      if (e != cudaErrorInvalidValue) return e;
    }
  }
  PHSVDS_DISPATCH(prec, ritz_p<P>(L, V, W, g, Y, theta, X, R, ldb, nb, dscale, T, norm_partial, max_blocks, nblocks, st))
}

template <class P>
static cudaError_t split_p(long long L, long long n, const void* X, const void* BX, long long ldb, int nb,
                           const void* coefs, void* partial, int max_blocks, int* nblocks, cudaStream_t st) {
  int grid = persistent_grid(L * nb, kThreads * 8);
  if (grid > max_blocks) grid = max_blocks;
  *nblocks = grid;
  k_split_resnorm<P><<<grid, kThreads, 0, st>>>(L, n, reinterpret_cast<const typename P::S*>(X),
                                                reinterpret_cast<const typename P::S*>(BX), ldb, nb,
                                                reinterpret_cast<const typename P::C*>(coefs),
                                                reinterpret_cast<typename P::G*>(partial));
  return cudaGetLastError();
}

cudaError_t launch_split_resnorm(int prec, long long L, long long n, const void* X, const void* BX, long long ldb,
                                 int nb, const void* coefs, void* partial, int max_blocks, int* nblocks,
                                 cudaStream_t st) {
  if (nb < 1 || nb > 8) return cudaErrorInvalidValue;
  PHSVDS_DISPATCH(prec, split_p<P>(L, n, X, BX, ldb, nb, coefs, partial, max_blocks, nblocks, st))
}

template <class P>
static cudaError_t scale_rows_p(long long L, const void* d, const void* R, long long ldr, void* T, long long ldt,
                                int nb, cudaStream_t st) {
  using S = typename P::S;
  k_scale_rows<P><<<persistent_grid(L * nb, kThreads), kThreads, 0, st>>>(
      L, reinterpret_cast<const S*>(d), reinterpret_cast<const S*>(R), ldr, reinterpret_cast<S*>(T), ldt, nb);
  return cudaGetLastError();
}
cudaError_t launch_scale_rows(int prec, long long L, const void* d, const void* R, long long ldr, void* T,
                              long long ldt, int nb, cudaStream_t st) {
  if (L * nb == 0) return cudaSuccess;
  PHSVDS_DISPATCH(prec, scale_rows_p<P>(L, d, R, ldr, T, ldt, nb, st))
}

template <class P>
static cudaError_t copy_cols_p(long long L, const void* Src, long long lds, void* Dst, long long ldd, int nb,
                               cudaStream_t st) {
  using S = typename P::S;
  k_copy_cols<P><<<persistent_grid(L * nb, kThreads), kThreads, 0, st>>>(L, reinterpret_cast<const S*>(Src), lds,
                                                                         reinterpret_cast<S*>(Dst), ldd, nb);
  return cudaGetLastError();
}
cudaError_t launch_copy_cols(int prec, long long L, const void* Src, long long lds, void* Dst, long long ldd, int nb,
                             cudaStream_t st) {
  if (L * nb == 0) return cudaSuccess;
  PHSVDS_DISPATCH(prec, copy_cols_p<P>(L, Src, lds, Dst, ldd, nb, st))
}

template <class P>
static cudaError_t fill_p(long long L, void* Dst, long long ldd, int nb, unsigned long long seed, cudaStream_t st) {
  k_fill_normal<P><<<persistent_grid(L * nb, kThreads), kThreads, 0, st>>>(L, reinterpret_cast<typename P::S*>(Dst),
                                                                           ldd, nb, seed);
  return cudaGetLastError();
}
cudaError_t launch_fill_normal(int prec, long long L, void* Dst, long long ldd, int nb, unsigned long long seed,
                               cudaStream_t st) {
  if (L * nb == 0) return cudaSuccess;
  PHSVDS_DISPATCH(prec, fill_p<P>(L, Dst, ldd, nb, seed, st))
}

template <class P>
static cudaError_t from_p(long long L, int nc, const double* src, long long lds, void* dst, long long ldd,
                          double scale, cudaStream_t st) {
  k_from_f64<P><<<persistent_grid(L * nc, kThreads), kThreads, 0, st>>>(L, nc, src, lds,
                                                                        reinterpret_cast<typename P::S*>(dst), ldd, scale);
  return cudaGetLastError();
}
cudaError_t launch_rows_to_f64(int prec, long long L, int nc, const void* src, long long lds, double* dst,
                               long long ldd, cudaStream_t st) {
  if (L * nc == 0) return cudaSuccess;
  PHSVDS_DISPATCH(prec, (k_rows_f64<P><<<persistent_grid(L * nc, kThreads), kThreads, 0, st>>>(
                            L, nc, reinterpret_cast<const typename P::S*>(src), lds, dst, ldd),
                        cudaGetLastError()))
}

cudaError_t launch_rows_from_f64(int prec, long long L, int nc, const double* src, long long lds, void* dst,
                                 long long ldd, cudaStream_t st) {
  if (L * nc == 0) return cudaSuccess;
  PHSVDS_DISPATCH(prec, (k_rows_from_f64<P><<<persistent_grid(L * nc, kThreads), kThreads, 0, st>>>(
                            L, nc, src, lds, reinterpret_cast<typename P::S*>(dst), ldd),
                        cudaGetLastError()))
}

cudaError_t launch_from_f64_colmajor(int prec, long long L, int nc, const double* src, long long lds, void* dst,
                                     long long ldd, double scale, cudaStream_t st) {
  if (L * nc == 0) return cudaSuccess;
  PHSVDS_DISPATCH(prec, from_p<P>(L, nc, src, lds, dst, ldd, scale, st))
}

template <class P>
static cudaError_t to_p(long long L, int nc, const void* src, long long lds, double* dst, long long ldd, double scale,
                        cudaStream_t st) {
  k_to_f64<P><<<persistent_grid(L * nc, kThreads), kThreads, 0, st>>>(
      L, nc, reinterpret_cast<const typename P::S*>(src), lds, dst, ldd, scale);
  return cudaGetLastError();
}
cudaError_t launch_to_f64_colmajor(int prec, long long L, int nc, const void* src, long long lds, double* dst,
                                   long long ldd, double scale, cudaStream_t st) {
  if (L * nc == 0) return cudaSuccess;
  PHSVDS_DISPATCH(prec, to_p<P>(L, nc, src, lds, dst, ldd, scale, st))
}

size_t coef_bytes(int prec) { return prec == kF32 ? 4 : 8; }

void host_coef_convert(int prec, const double* src, size_t count, void* dst) {
  if (prec == kF32) {
    float* d = reinterpret_cast<float*>(dst);
    for (size_t i = 0; i < count; ++i) d[i] = (float)src[i];
  } else if (prec == kDF64) {
    float* d = reinterpret_cast<float*>(dst);
    for (size_t i = 0; i < count; ++i) {
      float hi = (float)src[i];
      d[2 * i] = hi;
      d[2 * i + 1] = (float)(src[i] - (double)hi);
    }
  } else {
    std::memcpy(dst, src, count * sizeof(double));
  }
}

cudaError_t launch_absmax(long long nnz, const double* vals, unsigned long long* out_bits, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(out_bits, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  if (nnz == 0) return cudaSuccess;
  k_absmax<<<persistent_grid(nnz, kThreads), kThreads, 0, st>>>(nnz, vals, out_bits);
  return cudaGetLastError();
}

cudaError_t launch_csr_values(long long nnz, const double* vals, double scale, float* v32, float* v32lo, double* v64,
                              int* flags, cudaStream_t st) {
  if (nnz == 0) return cudaSuccess;
  k_csr_values<<<persistent_grid(nnz, kThreads), kThreads, 0, st>>>(nnz, vals, scale, v32, v32lo, v64, flags);
  return cudaGetLastError();
}

size_t transpose_work_ints(long long cols) {
  const long long nb = (cols + kScanChunk - 1) / kScanChunk + 1;
  return (size_t)(2 * (cols + 1) + 2 * nb + 4);
}

cudaError_t launch_csr_transpose(long long rows, long long cols, long long nnz, const int* rowptr, const int* colidx,
                                 const double* vals, int* rowptrT, int* colidxT, double* valsT, int* work,
                                 cudaStream_t st) {
  int* cnt = work;
  int* cursor = work + (cols + 1);
  long long* bsum = reinterpret_cast<long long*>(work + 2 * (cols + 1) + ((2 * (cols + 1)) & 1));
  const int nb = (int)((cols + kScanChunk - 1) / kScanChunk);
  cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(int) * 2 * (cols + 1), st);
  if (e != cudaSuccess) return e;
  if (nnz > 0) k_count_cols<<<persistent_grid(nnz, kThreads), kThreads, 0, st>>>(nnz, colidx, cnt);
  if (nb > 0) {
    k_scan_block_sums<<<nb, kThreads, 0, st>>>(cols, cnt, bsum);
    k_scan_bsums<<<1, 1024, 0, st>>>(nb, bsum);
    k_scan_apply<<<nb, kThreads, 0, st>>>(cols, cnt, bsum, rowptrT);
  } else {
    e = cudaMemsetAsync(rowptrT, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
  }
  if (rows > 0 && nnz > 0) {
    k_scatter_t<<<persistent_grid(rows, kThreads), kThreads, 0, st>>>(rows, rowptr, colidx, vals, rowptrT, cursor,
                                                                      colidxT, valsT);
    k_sort_segments<<<persistent_grid(cols, kThreads), kThreads, 0, st>>>(cols, rowptrT, colidxT, valsT);
  }
  return cudaGetLastError();
}

cudaError_t launch_exclusive_scan(long long n, const int* in, int* out, int* work, cudaStream_t st) {
  long long* bsum = reinterpret_cast<long long*>(work);
  const int nb = (int)((n + kScanChunk - 1) / kScanChunk);
  if (nb > 0) {
    k_scan_block_sums<<<nb, kThreads, 0, st>>>(n, in, bsum);
    k_scan_bsums<<<1, 1024, 0, st>>>(nb, bsum);
    k_scan_apply<<<nb, kThreads, 0, st>>>(n, in, bsum, out);
  } else {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

size_t scan_work_ints(long long n) { return (size_t)(2 * ((n + kScanChunk - 1) / kScanChunk) + 4); }

// ---------------------------------------------------------------------------
// C = A^T A in CSR: row j merges the sorted rows i of A listed in row j of A^T
// (a k-way merge of at most kMergeMax lists per thread, deterministic order).
// ---------------------------------------------------------------------------
constexpr int kMergeMax = 64;

// Row j of C merges the sorted rows i of A with a_ij != 0 (the entries of row j
// of A^T); count = number of distinct columns.
__global__ void k_c_count(long long n, const int* __restrict__ rpT, const int* __restrict__ ciT,
                          const int* __restrict__ rp, const int* __restrict__ ci, int* __restrict__ cnt,
                          int* __restrict__ err) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x) {
    const int t0 = rpT[j], nl = rpT[j + 1] - t0;
    if (nl > kMergeMax) {
      atomicOr(err, 1);
      cnt[j] = 0;
      continue;
    }
    int cur[kMergeMax], end[kMergeMax];
    for (int t = 0; t < nl; ++t) {
      const int i = ciT[t0 + t];
      cur[t] = rp[i];
      end[t] = rp[i + 1];
    }
    int count = 0;
    while (true) {
      int mn = 0x7fffffff;
      for (int t = 0; t < nl; ++t)
        if (cur[t] < end[t] && ci[cur[t]] < mn) mn = ci[cur[t]];
      if (mn == 0x7fffffff) break;
      ++count;
      for (int t = 0; t < nl; ++t)
        if (cur[t] < end[t] && ci[cur[t]] == mn) ++cur[t];
    }
    cnt[j] = count;
  }
}

__global__ void k_c_fill(long long n, const int* __restrict__ rpT, const int* __restrict__ ciT,
                         const double* __restrict__ vT, const int* __restrict__ rp, const int* __restrict__ ci,
                         const double* __restrict__ va, double scale, const int* __restrict__ cptr,
                         int* __restrict__ cidx, double* __restrict__ cval) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x) {
    const int t0 = rpT[j], nl = rpT[j + 1] - t0;
    if (nl > kMergeMax) continue;
    int cur[kMergeMax], end[kMergeMax];
    for (int t = 0; t < nl; ++t) {
      const int i = ciT[t0 + t];
      cur[t] = rp[i];
      end[t] = rp[i + 1];
    }
    int o = cptr[j];
    while (true) {
      int mn = 0x7fffffff;
      for (int t = 0; t < nl; ++t)
        if (cur[t] < end[t] && ci[cur[t]] < mn) mn = ci[cur[t]];
      if (mn == 0x7fffffff) break;
      double v = 0.0;
      for (int t = 0; t < nl; ++t)
        if (cur[t] < end[t] && ci[cur[t]] == mn) {
          v += vT[t0 + t] * va[cur[t]];  // a_{i j} a_{i mn}
          ++cur[t];
        }
      cidx[o] = mn;
      cval[o] = v * scale;
      ++o;
    }
  }
}

cudaError_t launch_normal_count(long long n, const int* rpT, const int* ciT, const int* rp, const int* ci, int* cnt,
                                int* err, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_c_count<<<persistent_grid(n, kThreads), kThreads, 0, st>>>(n, rpT, ciT, rp, ci, cnt, err);
  return cudaGetLastError();
}

cudaError_t launch_normal_fill(long long n, const int* rpT, const int* ciT, const double* vT, const int* rp,
                               const int* ci, const double* va, double scale, const int* cptr, int* cidx,
                               double* cval, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_c_fill<<<persistent_grid(n, kThreads), kThreads, 0, st>>>(n, rpT, ciT, vT, rp, ci, va, scale, cptr, cidx, cval);
  return cudaGetLastError();
}

int normal_merge_max() { return kMergeMax; }

// FP32 -> bfloat16, round to nearest even (finite inputs); flags[0] |= 1 when
// some value is not exactly representable.
__global__ void k_to_bf16(long long n, const float* __restrict__ x, unsigned short* __restrict__ y,
                          int* __restrict__ flags) {
  int inexact = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const unsigned u = __float_as_uint(x[i]);
    const unsigned r = (u + 0x7fffu + ((u >> 16) & 1u)) >> 16;
    y[i] = (unsigned short)r;
    inexact |= (r << 16) != u;
  }
  if (inexact) atomicOr(flags, 1);
}

cudaError_t launch_to_bf16(long long n, const float* x, uint16_t* y, int* flags, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_to_bf16<<<persistent_grid(n, kThreads), kThreads, 0, st>>>(n, x, reinterpret_cast<unsigned short*>(y), flags);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Output sign convention: per column j of a column-major block, the entry of
// largest magnitude in rows [r0, r0 + len) (lowest index on ties) is made
// positive by scaling the whole column (rows [0, rows)).
// ---------------------------------------------------------------------------
// Out[:, jj] = X[r0 : r0 + len, perm[jj]] for jj < k (column-major, ld len):
// the returned block in the caller's column order, contiguous.
__global__ void k_gather_cols(long long len, int k, const double* __restrict__ X, long long ldx, long long r0,
                              const int* __restrict__ perm, double* __restrict__ Out) {
  const long long total = len * k;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const long long r = e % len;
    const int jj = (int)(e / len);
    Out[e] = X[(long long)perm[jj] * ldx + r0 + r];
  }
}

cudaError_t launch_gather_cols(long long len, int k, const double* X, long long ldx, long long r0, const int* perm,
                               double* Out, cudaStream_t st) {
  if (len <= 0 || k <= 0) return cudaSuccess;
  k_gather_cols<<<persistent_grid(len * k, kThreads), kThreads, 0, st>>>(len, k, X, ldx, r0, perm, Out);
  return cudaGetLastError();
}

// phase 1: per (row chunk, column) the largest |x| and its lowest index
__global__ void __launch_bounds__(kThreads) k_col_absmax(long long ld, long long r0, long long len, int chunks,
                                                         const double* __restrict__ X, double* __restrict__ pv,
                                                         long long* __restrict__ pi) {
  __shared__ double sv[kThreads];
  __shared__ long long si[kThreads];
  const int j = blockIdx.y, c = blockIdx.x;
  const long long per = (len + chunks - 1) / chunks;
  const long long a = (long long)c * per, b = a + per < len ? a + per : len;
  const double* col = X + j * ld + r0;
  double best = -1.0;
  long long bi = -1;
  for (long long r = a + threadIdx.x; r < b; r += kThreads) {
    const double v = fabs(col[r]);
    if (v > best) {  // strictly larger: the first index of a tie stays
      best = v;
      bi = r;
    }
  }
  sv[threadIdx.x] = best;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      const double v = sv[threadIdx.x + w];
      const long long iv = si[threadIdx.x + w];
      if (iv >= 0 && (v > sv[threadIdx.x] || (v == sv[threadIdx.x] && (si[threadIdx.x] < 0 || iv < si[threadIdx.x])))) {
        sv[threadIdx.x] = v;
        si[threadIdx.x] = iv;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    pv[(long long)j * chunks + c] = sv[0];
    pi[(long long)j * chunks + c] = si[0];
  }
}

// phase 2: chunks in order (a later chunk wins only when strictly larger), sign
__global__ void k_col_sign_pick(long long ld, long long r0, int k, int chunks, const double* __restrict__ X,
                                const double* __restrict__ pv, const long long* __restrict__ pi,
                                double* __restrict__ sign) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= k) return;
  double best = -1.0;
  long long bi = -1;
  for (int c = 0; c < chunks; ++c) {
    const long long i = pi[(long long)j * chunks + c];
    if (i >= 0 && pv[(long long)j * chunks + c] > best) {
      best = pv[(long long)j * chunks + c];
      bi = i;
    }
  }
  sign[j] = (bi >= 0 && X[j * ld + r0 + bi] < 0.0) ? -1.0 : 1.0;
}

// phase 3: X[:, j] *= sign[j]
__global__ void k_col_flip(long long rows, long long ld, int k, const double* __restrict__ sign, double* __restrict__ X) {
  const long long total = rows * k;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(e / rows);
    const long long r = e % rows;
    if (sign[j] < 0.0) X[j * ld + r] = -X[j * ld + r];
  }
}

cudaError_t launch_col_sign(long long rows, long long ld, int k, long long r0, long long len, double* X, double* work,
                            cudaStream_t st) {
  if (k <= 0 || rows <= 0) return cudaSuccess;
  const int chunks = (int)std::max<long long>(1, std::min<long long>(256, (len + 65535) / 65536));
  double* pv = work;
  long long* pi = reinterpret_cast<long long*>(work + (size_t)k * chunks);
  double* sign = work + (size_t)2 * k * chunks;
  k_col_absmax<<<dim3(chunks, k), kThreads, 0, st>>>(ld, r0, len, chunks, X, pv, pi);
  k_col_sign_pick<<<(k + 127) / 128, 128, 0, st>>>(ld, r0, k, chunks, X, pv, pi, sign);
  k_col_flip<<<persistent_grid(rows * k, kThreads), kThreads, 0, st>>>(rows, ld, k, sign, X);
  return cudaGetLastError();
}

size_t col_sign_work_doubles(int k, long long len) {
  const int chunks = (int)std::max<long long>(1, std::min<long long>(256, (len + 65535) / 65536));
  return (size_t)2 * k * chunks + k;
}

cudaError_t launch_row_sumsq(long long rows, const int* rowptr, const double* vals, double* out, cudaStream_t st) {
  if (rows == 0) return cudaSuccess;
  k_row_sumsq<<<persistent_grid(rows, kThreads), kThreads, 0, st>>>(rows, rowptr, vals, out);
  return cudaGetLastError();
}

template <class P>
static cudaError_t dscale_p(long long L, const double* s, int use_sqrt, void* d, cudaStream_t st) {
  k_make_dscale<P><<<persistent_grid(L, kThreads), kThreads, 0, st>>>(L, s, use_sqrt, reinterpret_cast<typename P::S*>(d));
  return cudaGetLastError();
}
cudaError_t launch_make_dscale(int prec, long long L, const double* s, int use_sqrt, void* d, cudaStream_t st) {
  if (L == 0) return cudaSuccess;
  PHSVDS_DISPATCH(prec, dscale_p<P>(L, s, use_sqrt, d, st))
}

cudaError_t launch_csr_validate(long long rows, long long cols, const int* rowptr, const int* colidx,
                                const double* vals, int* flags, cudaStream_t st) {
  if (rows == 0) return cudaSuccess;
  k_csr_validate<<<persistent_grid(rows, kThreads), kThreads, 0, st>>>(rows, cols, rowptr, colidx, vals, flags);
  return cudaGetLastError();
}

cudaError_t launch_ortho_small(int stage, int prec, int g, int nb, const double* G, double* work, void* coef,
                               void* rinv, int* status, double drop2, cudaStream_t st) {
  if (nb < 1 || nb > 8 || g < 0) return cudaErrorInvalidValue;
  k_ortho_small<<<1, 64, 0, st>>>(stage, prec, g, nb, G, work, coef, rinv, status, drop2);
  return cudaGetLastError();
}

void kernels_init() {}

}  // namespace phsvds
