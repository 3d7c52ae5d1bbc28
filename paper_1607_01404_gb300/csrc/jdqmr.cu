// Inner solver of JDQMR: symmetric QMR (quasi-minimal residual smoothing of
// preconditioned CG, Freund & Nachtigal 1994) on the Jacobi-Davidson
// correction equation
//     (I - x x^T)(op - eta I)(I - x x^T) t = -r,   t orthogonal to x,
// for a block of nb columns at once (one independent system per column), with
// the projected preconditioner K~^-1 z = K^-1 z - K^-1 x (x^T K^-1 z)/(x^T K^-1 x)
// (K^-1 = Jacobi diagonal, identity, or a sparse symmetric matrix such as the
// learned approximate inverse, applied by SpMM).  The paper runs JDQMR as the stage-2
// method (Sec. 3.4) and uses it in stage 1 in its experiments (Sec. 4).
//
// The vectors use the storage/arithmetic of one mode: FP32 by default (the
// correction only needs about one digit, and the outer iteration keeps its own
// precision), or the FP64-class mode.  Per inner step: one operator apply and
// three streaming kernels with fixed-order FP64-class reductions; the scalar
// recurrences run in one-thread-per-column kernels, so no host round trip is
// needed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <atomic>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "common.cuh"
#include "jdqmr.h"
#include "kernels.h"
#include "spmm_dev.cuh"

namespace phsvds {

namespace {

constexpr int kT = 256;
constexpr int kMaxNb = 8;

// Persistent grids: every SM holds as many 256-thread CTAs of the kernel as
// its register and shared-memory use allow (queried once per kernel), so
// there is no tail wave; at most kMaxGrid CTAs (partial-sum storage).
constexpr int kMaxGrid = 2048;

int sm_count() {
  static std::atomic<int> sms{0};
  int v = sms.load(std::memory_order_relaxed);
  if (!v) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) {
      cudaGetLastError();
      v = 152;
    }
    sms.store(v, std::memory_order_relaxed);
  }
  return v;
}

// resident 256-thread CTAs per SM of one kernel (cached by kernel address)
template <class K>
int blocks_per_sm(K kernel) {
  static std::mutex mu;
  static std::unordered_map<const void*, int> cache;
  const void* key = reinterpret_cast<const void*>(kernel);
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  int v = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kernel, kT, 0) != cudaSuccess || v < 1) {
    cudaGetLastError();
    v = 1;
  }
  cache[key] = v;
  return v;
}

template <class K>
int occ_grid(K kernel, long long work) {
  long long g = (work + kT - 1) / kT;
  const long long cap = std::min<long long>((long long)sm_count() * blocks_per_sm(kernel), kMaxGrid);
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

// grid of the plain elementwise kernels
int qmr_grid(long long L) {
  long long g = (L + kT - 1) / kT;
  const long long cap = (long long)sm_count() * 4;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}


// conversion of a double scalar to the mode's coefficient type
template <class P>
__device__ __forceinline__ typename P::C to_c(double v);
template <>
__device__ __forceinline__ float to_c<PF32>(double v) {
  return (float)v;
}
template <>
__device__ __forceinline__ df to_c<PDF64>(double v) {
  const float hi = (float)v;
  return df{hi, (float)(v - (double)hi)};
}
template <>
__device__ __forceinline__ double to_c<PF64>(double v) {
  return v;
}

__device__ __forceinline__ df shfl_down(df v, int o) {
  return df{__shfl_down_sync(0xffffffffu, v.hi, o), __shfl_down_sync(0xffffffffu, v.lo, o)};
}
__device__ __forceinline__ double shfl_down(double v, int o) { return __shfl_down_sync(0xffffffffu, v, o); }

// Per-thread accumulators of the dot products: plain FP32 in the FP32 inner
// mode (its vectors are FP32 and a thread sums a few dozen rows; the block and
// grid levels stay FP64-class), the mode's FP64-class type otherwise.
template <class P>
struct TAcc {
  using T = typename P::G;
  __device__ static T zero() { return P::gzero(); }
  __device__ static T fma(T a, typename P::A x, typename P::A y) { return P::gfma(a, x, y); }
  __device__ static typename P::G g(T a) { return a; }
};
template <>
struct TAcc<PF32> {
  using T = float;
  __device__ static float zero() { return 0.f; }
  __device__ static float fma(float a, float x, float y) { return fmaf(x, y, a); }
  __device__ static df g(float a) { return df{a, 0.f}; }
};

// Per-CTA partial sums of ND dot products for each of the NW <= 8 columns
// (FP64-class accumulation, fixed order), written to partial[blk][d * nb + j].
template <class P, int ND, int NW>
__device__ __forceinline__ void block_reduce_store(typename TAcc<P>::T (&acc)[ND][NW], int nb, typename P::G* partial) {
  using G = typename P::G;
  __shared__ G red[kT / 32][ND * kMaxNb];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int d = 0; d < ND; ++d)
#pragma unroll
    for (int j = 0; j < NW; ++j) {
      G v = TAcc<P>::g(acc[d][j]);
      for (int o = 16; o > 0; o >>= 1) v = P::gadd(v, shfl_down(v, o));
      if (lane == 0) red[warp][d * kMaxNb + j] = v;
    }
  __syncthreads();
  for (int e = threadIdx.x; e < ND * nb; e += kT) {
    const int d = e / nb, j = e % nb;
    G v = red[0][d * kMaxNb + j];
    for (int w = 1; w < kT / 32; ++w) v = P::gadd(v, red[w][d * kMaxNb + j]);
    partial[(long long)blockIdx.x * ND * nb + e] = v;
  }
}

__device__ void qmr_scalars1(int j, int nb, const double* __restrict__ dots, const double* __restrict__ eta,
                             QmrState* S);
__device__ void qmr_scalars2(int j, int nb, const double* __restrict__ dots, double xi, int maxk, QmrState* S);

// The last CTA of a grid to finish (counted with an atomic ticket after every
// CTA has stored its partial sums) reduces the partials in a fixed order into
// dots[0, n) and runs the scalar step: mode 1 = scalars1, 2 = none,
// 3 = scalars2 (with the dots of the whole step), then rearms the ticket.
// No CTA waits for another, so the tail cannot stall.
struct Tail {
  unsigned* tick = nullptr;
  double* out = nullptr;   // reduced values go to out[0, n)
  double* dots = nullptr;  // the step's dots (for the scalar step)
  int mode = 0;
  int nb = 0;
  const double* eta = nullptr;
  double xi = 0.0;
  int maxk = 0;
  QmrState* S = nullptr;
};

template <class P>
__device__ void grid_tail(const typename P::G* partial, int n, const Tail& t) {
  using G = typename P::G;
  __shared__ unsigned s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(t.tick, 1u) == gridDim.x - 1 ? 1u : 0u;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // kT / n threads per value (n divides kT): thread t sums the partials of
  // value t % n of CTAs t / n, t / n + kT / n, ... (coalesced, four loads in
  // flight), then a fixed tree over the threads of each value
  __shared__ G red[kT];
  const int per = kT / n, e = threadIdx.x % n;
  const long long tot = (long long)gridDim.x * n;
  auto ld = [&](long long i) -> G {
    if constexpr (P::id != kF64) {
      const float2 f = __ldcg(reinterpret_cast<const float2*>(partial + i));
      return G{f.x, f.y};
    } else {
      return __ldcg(reinterpret_cast<const double*>(partial + i));
    }
  };
  G v = P::gzero();
  long long i = threadIdx.x;
  for (; i + 3LL * kT < tot; i += 4LL * kT) {
    const G a0 = ld(i), a1 = ld(i + kT), a2 = ld(i + 2LL * kT), a3 = ld(i + 3LL * kT);
    v = P::gadd(P::gadd(P::gadd(P::gadd(v, a0), a1), a2), a3);
  }
  for (; i < tot; i += kT) v = P::gadd(v, ld(i));
  red[threadIdx.x] = v;
  __syncthreads();
  for (int w = per / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w * n) red[threadIdx.x] = P::gadd(red[threadIdx.x], red[threadIdx.x + w * n]);
    __syncthreads();
  }
  if ((int)threadIdx.x < n) t.out[threadIdx.x] = P::gval(red[threadIdx.x]);
  (void)e;
  __syncthreads();
  if ((int)threadIdx.x < t.nb) {
    if (t.mode == 1) qmr_scalars1(threadIdx.x, t.nb, t.dots, t.eta, t.S);
    if (t.mode == 3) qmr_scalars2(threadIdx.x, t.nb, t.dots, t.xi, t.maxk, t.S);
  }
  if (threadIdx.x == 0) *t.tick = 0u;
}

template <class P>
__device__ __forceinline__ typename P::A ld_or_one(const typename P::S* p, long long i) {
  if (p) return P::load(p + i);
  if constexpr (P::id == kDF64)
    return df{1.f, 0.f};
  else
    return (typename P::A)1;
}

template <class P>
__device__ __forceinline__ typename P::A mul(typename P::A a, typename P::A b) {
  if constexpr (P::id == kDF64)
    return df_mul(a, b);
  else
    return a * b;
}

// Row access of an L x nb block with leading dimension nb: NB (>= nb) slots,
// 16-byte vector loads when VEC (nb == NB and rows are 16-byte multiples).
template <class P, int NB, bool VEC>
__device__ __forceinline__ void ldrow(const typename P::S* __restrict__ p, long long row, int nb,
                                      typename P::A (&v)[NB]) {
  using S = typename P::S;
  const S* rp = p + row * nb;
  if constexpr (VEC) {
    constexpr int W = (int)(NB * sizeof(S) / 16);
    const float4* q4 = reinterpret_cast<const float4*>(rp);
    float buf[NB * sizeof(S) / 4];
#pragma unroll
    for (int i = 0; i < W; ++i) {
      const float4 t = q4[i];
      buf[4 * i] = t.x;
      buf[4 * i + 1] = t.y;
      buf[4 * i + 2] = t.z;
      buf[4 * i + 3] = t.w;
    }
#pragma unroll
    for (int j = 0; j < NB; ++j) v[j] = P::load(reinterpret_cast<const S*>(buf) + j);
  } else {
#pragma unroll
    for (int j = 0; j < NB; ++j) v[j] = j < nb ? P::load(rp + j) : P::zero();
  }
}

template <class P, int NB, bool VEC>
__device__ __forceinline__ void strow(typename P::S* __restrict__ p, long long row, int nb,
                                      const typename P::A (&v)[NB]) {
  using S = typename P::S;
  S* rp = p + row * nb;
  if constexpr (VEC) {
    constexpr int W = (int)(NB * sizeof(S) / 16);
    float buf[NB * sizeof(S) / 4];
#pragma unroll
    for (int j = 0; j < NB; ++j) P::store(reinterpret_cast<S*>(buf) + j, v[j]);
    float4* q4 = reinterpret_cast<float4*>(rp);
#pragma unroll
    for (int i = 0; i < W; ++i) q4[i] = make_float4(buf[4 * i], buf[4 * i + 1], buf[4 * i + 2], buf[4 * i + 3]);
  } else {
#pragma unroll
    for (int j = 0; j < NB; ++j)
      if (j < nb) P::store(rp + j, v[j]);
  }
}

// ---- initialisation ----
// kx = K^-1 x, u = K^-1 b, dots: x^T kx, x^T u, b^T b, b^T u, b^T kx
// (upre != nullptr: kx = K^-1 x and upre = K^-1 b were computed by SpMM)
template <class P>
__global__ void __launch_bounds__(kT) k_qmr_init(long long L, int nb, const typename P::S* __restrict__ x,
                                                 const typename P::S* __restrict__ b,
                                                 const typename P::S* __restrict__ dinv, typename P::S* __restrict__ kx,
                                                 const typename P::S* __restrict__ upre,
                                                 typename P::G* __restrict__ partial) {
  using G = typename P::G;
  typename TAcc<P>::T acc[5][kMaxNb];
#pragma unroll
  for (int d = 0; d < 5; ++d)
#pragma unroll
    for (int j = 0; j < kMaxNb; ++j) acc[d][j] = TAcc<P>::zero();
  for (long long r = blockIdx.x * (long long)kT + threadIdx.x; r < L; r += (long long)gridDim.x * kT) {
    const auto s = ld_or_one<P>(dinv, r);
#pragma unroll
    for (int j = 0; j < kMaxNb; ++j)
      if (j < nb) {
        const long long o = r * nb + j;
        const auto xv = P::load(x + o), bv = P::load(b + o);
        typename P::A kv, uv;
        if (upre) {
          kv = P::load(kx + o);
          uv = P::load(upre + o);
        } else {
          kv = mul<P>(s, xv);
          uv = mul<P>(s, bv);
          P::store(kx + o, kv);
        }
        acc[0][j] = TAcc<P>::fma(acc[0][j], xv, kv);
        acc[1][j] = TAcc<P>::fma(acc[1][j], xv, uv);
        acc[2][j] = TAcc<P>::fma(acc[2][j], bv, bv);
        acc[3][j] = TAcc<P>::fma(acc[3][j], bv, uv);
        acc[4][j] = TAcc<P>::fma(acc[4][j], bv, kv);
      }
  }
  block_reduce_store<P, 5, kMaxNb>(acc, nb, partial);
}

__global__ void k_qmr_init_scalars(int nb, const double* __restrict__ dots, QmrState* S) {
  const int j = threadIdx.x;
  if (j >= nb) return;
  const double xkx = dots[0 * nb + j], xu = dots[1 * nb + j], bb = dots[2 * nb + j], bu = dots[3 * nb + j],
               bkx = dots[4 * nb + j];
  QmrState s{};
  s.xkx = xkx > 0 ? xkx : 1.0;
  s.gamma = xu / s.xkx;
  s.rho = bu - bkx * s.gamma;
  s.tau = sqrt(bb);
  s.tau0 = s.tau;
  s.theta = 0.0;
  s.active = (s.tau > 0 && s.rho != 0.0) ? 1 : 0;
  s.k = 0;
  S[j] = s;
}

// q = K^-1 b - kx gamma ; r = b ; d = 0 ; sol = 0
template <class P>
__global__ void __launch_bounds__(kT) k_qmr_init_vec(long long L, int nb, const typename P::S* __restrict__ b,
                                                     const typename P::S* __restrict__ dinv,
                                                     const typename P::S* __restrict__ kx,
                                                     const typename P::S* __restrict__ upre,
                                                     const QmrState* __restrict__ S, typename P::S* __restrict__ q,
                                                     typename P::S* __restrict__ r, typename P::S* __restrict__ d,
                                                     typename P::S* __restrict__ sol) {
  __shared__ typename P::C gm[kMaxNb];
  if (threadIdx.x < nb) gm[threadIdx.x] = to_c<P>(S[threadIdx.x].gamma);
  __syncthreads();
  const long long total = L * nb;
  for (long long e = blockIdx.x * (long long)kT + threadIdx.x; e < total; e += (long long)gridDim.x * kT) {
    const long long row = e / nb;
    const int j = (int)(e % nb);
    const auto bv = P::load(b + e);
    const auto ub = upre ? P::load(upre + e) : mul<P>(ld_or_one<P>(dinv, row), bv);
    P::store(q + e, P::sub(ub, P::mulc(P::load(kx + e), gm[j])));
    P::store(r + e, bv);
    P::store(d + e, P::zero());
    P::store(sol + e, P::zero());
  }
}

// ---- per inner step ----
// after w = op(q): dots x^T w, q^T w, x^T q, q^T q (one thread per row)
template <class P, int NB, bool VEC>
__global__ void __launch_bounds__(kT) k_qmr_dots1(long long L, int nb, const typename P::S* __restrict__ x,
                                                  const typename P::S* __restrict__ q,
                                                  const typename P::S* __restrict__ w,
                                                  typename P::G* __restrict__ partial) {
  using G = typename P::G;
  using A = typename P::A;
  typename TAcc<P>::T acc[4][NB];
#pragma unroll
  for (int d = 0; d < 4; ++d)
#pragma unroll
    for (int j = 0; j < NB; ++j) acc[d][j] = TAcc<P>::zero();
  for (long long r = blockIdx.x * (long long)kT + threadIdx.x; r < L; r += (long long)gridDim.x * kT) {
    A xv[NB], qv[NB], wv[NB];
    ldrow<P, NB, VEC>(x, r, nb, xv);
    ldrow<P, NB, VEC>(q, r, nb, qv);
    ldrow<P, NB, VEC>(w, r, nb, wv);
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      acc[0][j] = TAcc<P>::fma(acc[0][j], xv[j], wv[j]);
      acc[1][j] = TAcc<P>::fma(acc[1][j], qv[j], wv[j]);
      acc[2][j] = TAcc<P>::fma(acc[2][j], xv[j], qv[j]);
      acc[3][j] = TAcc<P>::fma(acc[3][j], qv[j], qv[j]);
    }
  }
  block_reduce_store<P, 4, NB>(acc, nb, partial);
}

// sigma = q^T t with t = w - eta q - x (x^T w - eta x^T q); alpha = rho / sigma
__device__ void qmr_scalars1(int j, int nb, const double* __restrict__ dots, const double* __restrict__ eta,
                             QmrState* S) {
  QmrState s = S[j];
  const double xw = dots[0 * nb + j], qw = dots[1 * nb + j], xq = dots[2 * nb + j], qq = dots[3 * nb + j];
  s.c1 = xw - eta[j] * xq;
  const double sigma = (qw - eta[j] * qq) - xq * s.c1;
  if (s.active && sigma != 0.0 && isfinite(sigma)) {
    s.alpha = s.rho / sigma;
  } else {
    s.alpha = 0.0;
    s.active = 0;
  }
  S[j] = s;
}

__global__ void k_qmr_scalars1(int nb, const double* __restrict__ dots, const double* __restrict__ eta,
                               QmrState* S) {
  if ((int)threadIdx.x < nb) qmr_scalars1(threadIdx.x, nb, dots, eta, S);
}

// t = w - eta q - x c1 ; r -= alpha t ; u = K^-1 r ; dots r^T r, r^T u, x^T u, r^T kx
template <class P, int NB, bool VEC>
__global__ void __launch_bounds__(kT) k_qmr_update1(long long L, int nb, const typename P::S* __restrict__ x,
                                                    const typename P::S* __restrict__ q,
                                                    const typename P::S* __restrict__ w,
                                                    const typename P::S* __restrict__ kx,
                                                    const typename P::S* __restrict__ dinv,
                                                    const double* __restrict__ eta, const QmrState* __restrict__ S,
                                                    typename P::S* __restrict__ r, typename P::G* __restrict__ partial,
                                                    Tail tail) {
  using G = typename P::G;
  using C = typename P::C;
  using A = typename P::A;
  __shared__ C sa[kMaxNb], sc[kMaxNb], se[kMaxNb];
  if (threadIdx.x < kMaxNb) {
    const bool ok = threadIdx.x < nb;
    sa[threadIdx.x] = to_c<P>(ok && S[threadIdx.x].active ? S[threadIdx.x].alpha : 0.0);
    sc[threadIdx.x] = to_c<P>(ok ? S[threadIdx.x].c1 : 0.0);
    se[threadIdx.x] = to_c<P>(ok ? eta[threadIdx.x] : 0.0);
  }
  __syncthreads();
  typename TAcc<P>::T acc[4][NB];
#pragma unroll
  for (int d = 0; d < 4; ++d)
#pragma unroll
    for (int j = 0; j < NB; ++j) acc[d][j] = TAcc<P>::zero();
  for (long long row = blockIdx.x * (long long)kT + threadIdx.x; row < L; row += (long long)gridDim.x * kT) {
    const auto sv = ld_or_one<P>(dinv, row);
    A xv[NB], qv[NB], wv[NB], rv[NB], kv[NB];
    ldrow<P, NB, VEC>(x, row, nb, xv);
    ldrow<P, NB, VEC>(q, row, nb, qv);
    ldrow<P, NB, VEC>(w, row, nb, wv);
    ldrow<P, NB, VEC>(r, row, nb, rv);
    ldrow<P, NB, VEC>(kx, row, nb, kv);
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      const A t = P::sub(P::sub(wv[j], P::mulc(qv[j], se[j])), P::mulc(xv[j], sc[j]));
      rv[j] = P::sub(rv[j], P::mulc(t, sa[j]));
      const A uv = mul<P>(sv, rv[j]);
      acc[0][j] = TAcc<P>::fma(acc[0][j], rv[j], rv[j]);
      acc[1][j] = TAcc<P>::fma(acc[1][j], rv[j], uv);
      acc[2][j] = TAcc<P>::fma(acc[2][j], xv[j], uv);
      acc[3][j] = TAcc<P>::fma(acc[3][j], rv[j], kv[j]);
    }
    strow<P, NB, VEC>(r, row, nb, rv);
  }
  block_reduce_store<P, 4, NB>(acc, nb, partial);
  if (tail.tick) grid_tail<P>(partial, 4 * nb, tail);
}

// dots r^T u, x^T u for u = K^-1 r computed by SpMM (sparse K^-1)
template <class P, int NB, bool VEC>
__global__ void __launch_bounds__(kT) k_qmr_dots_u(long long L, int nb, const typename P::S* __restrict__ x,
                                                   const typename P::S* __restrict__ r,
                                                   const typename P::S* __restrict__ u,
                                                   typename P::G* __restrict__ partial) {
  using G = typename P::G;
  using A = typename P::A;
  typename TAcc<P>::T acc[2][NB];
#pragma unroll
  for (int d = 0; d < 2; ++d)
#pragma unroll
    for (int j = 0; j < NB; ++j) acc[d][j] = TAcc<P>::zero();
  for (long long row = blockIdx.x * (long long)kT + threadIdx.x; row < L; row += (long long)gridDim.x * kT) {
    A xv[NB], rv[NB], uv[NB];
    ldrow<P, NB, VEC>(x, row, nb, xv);
    ldrow<P, NB, VEC>(r, row, nb, rv);
    ldrow<P, NB, VEC>(u, row, nb, uv);
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      acc[0][j] = TAcc<P>::fma(acc[0][j], rv[j], uv[j]);
      acc[1][j] = TAcc<P>::fma(acc[1][j], xv[j], uv[j]);
    }
  }
  block_reduce_store<P, 2, NB>(acc, nb, partial);
}

// Fused Y = K X (CSR, rows L, Y row-major with ld NB) and the dot products
// of Y with two row-major blocks E1, E2 (ld NB): d0 = E1^T Y, d1 = E2^T Y and,
// for ND = 4, d2 = E1^T E2, d3 = E2^T E2 (per column, FP64-class partials).
// With (E1, E2) = (x, q) these are the four dots of k_qmr_dots1 for w = op q;
// with (E1, E2) = (r, x) the two dots of k_qmr_dots_u for u = K^-1 r.
// Tuning of k_spmm_dots in the F32 mode: CTAs per SM the register allocation
// must allow, and the number of row gathers a thread keeps in flight.  The
// gathers are latency-bound: 6 CTAs of 256 threads per SM (at most 40
// registers, a few spilled) with 2 gathers in flight beat 4 CTAs with 4
// gathers on the 7-nonzero rows of a 3D-grid A^T A.  Wider accumulators get
// looser bounds so that nothing spills heavily: F32 blocks of 8 columns 3 CTAs
// per SM (80 registers), double-float and FP64 blocks of up to 4 columns 3
// CTAs (80 registers), of 8 columns 1 CTA (up to 168 registers); these keep the
// default unroll.
#ifndef PHSVDS_DOTS_MINB
#define PHSVDS_DOTS_MINB 6
#endif
#ifndef PHSVDS_DOTS_U
#define PHSVDS_DOTS_U 2
#endif
template <class P, int NB>
__host__ __device__ constexpr int dots_minb() {
  return P::id == kF32 ? (NB >= 8 ? 3 : PHSVDS_DOTS_MINB) : (NB >= 8 ? 1 : 3);
}
template <class P, int NB>
__host__ __device__ constexpr int dots_unroll() {
  return (P::id == kF32 && NB < 8 && PHSVDS_DOTS_U > 0) ? PHSVDS_DOTS_U : spmm_unroll<P, NB>();
}

template <class P, int NB, int VMODE, bool VEC, int ND>
__global__ void __launch_bounds__(kT, dots_minb<P, NB>()) k_spmm_dots(long long L, const int* __restrict__ rowptr,
                                                  const int* __restrict__ colidx, const float* __restrict__ v32,
                                                  const float* __restrict__ v32lo, const double* __restrict__ v64,
                                                  const typename P::S* __restrict__ X, long long ldx,
                                                  typename P::S* __restrict__ Y, const typename P::S* __restrict__ E1,
                                                  const typename P::S* __restrict__ E2,
                                                  typename P::G* __restrict__ partial, Tail tail) {
  using G = typename P::G;
  using A = typename P::A;
  typename TAcc<P>::T acc[ND][NB];
#pragma unroll
  for (int d = 0; d < ND; ++d)
#pragma unroll
    for (int j = 0; j < NB; ++j) acc[d][j] = TAcc<P>::zero();
  for (long long row = blockIdx.x * (long long)kT + threadIdx.x; row < L; row += (long long)gridDim.x * kT) {
    A y[NB];
#pragma unroll
    for (int c = 0; c < NB; ++c) y[c] = P::zero();
    row_product<P, NB, VMODE, VEC, dots_unroll<P, NB>()>(__ldg(rowptr + row), __ldg(rowptr + row + 1), colidx, v32,
                                                          v32lo, v64, X, ldx, y);
    store_yrow<P, NB, VEC>(Y + row * NB, y);
    A e1[NB], e2[NB];
    ldrow<P, NB, VEC>(E1, row, NB, e1);
    ldrow<P, NB, VEC>(E2, row, NB, e2);
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      acc[0][j] = TAcc<P>::fma(acc[0][j], e1[j], y[j]);
      acc[1][j] = TAcc<P>::fma(acc[1][j], e2[j], y[j]);
      if constexpr (ND == 4) {
        acc[2][j] = TAcc<P>::fma(acc[2][j], e1[j], e2[j]);
        acc[3][j] = TAcc<P>::fma(acc[3][j], e2[j], e2[j]);
      }
    }
  }
  block_reduce_store<P, ND, NB>(acc, NB, partial);
  if (tail.tick) grid_tail<P>(partial, ND * NB, tail);
}

// launch k_spmm_dots for the value format of K; returns its grid (the number
// of partial sums), or 0 when nb or the alignment has no fused form
template <class P, int NB, int ND>
int spmm_dots_nb(long long L, const CsrDev& K, const void* X, long long ldx, void* Y, const void* E1, const void* E2,
                 void* partial, const Tail& tail, cudaStream_t st) {
  using SS = typename P::S;
  using GG = typename P::G;
  constexpr bool vec = (NB * sizeof(SS)) % 16 == 0;
  if (vec && ((ldx * sizeof(SS)) % 16 != 0 || reinterpret_cast<uintptr_t>(X) % 16 != 0 ||
              reinterpret_cast<uintptr_t>(Y) % 16 != 0 || reinterpret_cast<uintptr_t>(E1) % 16 != 0 ||
              reinterpret_cast<uintptr_t>(E2) % 16 != 0))
    return 0;
  const SS *x = (const SS*)X, *e1 = (const SS*)E1, *e2 = (const SS*)E2;
  SS* y = (SS*)Y;
  GG* pd = (GG*)partial;
  auto go = [&](auto kern, const float* a32, const float* a32lo, const double* a64) {
    const int g = occ_grid(kern, L);
    kern<<<g, kT, 0, st>>>(L, K.rowptr, K.colidx, a32, a32lo, a64, x, ldx, y, e1, e2, pd, tail);
    return g;
  };
  if constexpr (P::id == kF32) {
    if (K.v16) return go(k_spmm_dots<P, NB, 4, vec, ND>, reinterpret_cast<const float*>(K.v16), nullptr, nullptr);
    return go(k_spmm_dots<P, NB, 0, vec, ND>, K.v32, nullptr, nullptr);
  } else if constexpr (P::id == kDF64) {
    if (K.v32lo == nullptr) return go(k_spmm_dots<P, NB, 1, vec, ND>, K.v32, nullptr, nullptr);
    return go(k_spmm_dots<P, NB, 2, vec, ND>, K.v32, K.v32lo, nullptr);
  } else {
    return go(k_spmm_dots<P, NB, 3, vec, ND>, nullptr, nullptr, K.v64);
  }
}

template <class P, int ND>
int spmm_dots_p(int nb, long long L, const CsrDev& K, const void* X, long long ldx, void* Y, const void* E1,
                const void* E2, void* partial, const Tail& tail, cudaStream_t st) {
  switch (nb) {
    case 1: return spmm_dots_nb<P, 1, ND>(L, K, X, ldx, Y, E1, E2, partial, tail, st);
    case 2: return spmm_dots_nb<P, 2, ND>(L, K, X, ldx, Y, E1, E2, partial, tail, st);
    case 4: return spmm_dots_nb<P, 4, ND>(L, K, X, ldx, Y, E1, E2, partial, tail, st);
    case 8: return spmm_dots_nb<P, 8, ND>(L, K, X, ldx, Y, E1, E2, partial, tail, st);
  }
  return 0;
}

// QMR smoothing scalars, stopping test, next search-direction coefficients
__device__ void qmr_scalars2(int j, int nb, const double* __restrict__ dots, double xi, int maxk, QmrState* S) {
  QmrState s = S[j];
  s.coefd = 0.0;
  s.coefq = 0.0;
  s.beta = 0.0;
  s.upd = 0;
  if (s.active) {
    const double rr = dots[0 * nb + j], ru = dots[1 * nb + j], xu = dots[2 * nb + j], rkx = dots[3 * nb + j];
    const double theta = sqrt(fmax(rr, 0.0)) / s.tau;
    const double c = 1.0 / sqrt(1.0 + theta * theta);
    s.coefd = c * c * s.theta * s.theta;
    s.coefq = c * c * s.alpha;
    s.theta = theta;
    s.tau = s.tau * theta * c;
    s.k += 1;
    s.upd = 1;
    s.gamma = xu / s.xkx;
    const double rho_new = ru - rkx * s.gamma;
    // stop: QMR residual bound tau sqrt(k + 1) below xi ||b||, or budget, or breakdown
    if (s.tau * sqrt((double)s.k + 1.0) <= xi * s.tau0 || s.k >= maxk || rho_new == 0.0 || !isfinite(rho_new)) {
      s.active = 0;
    } else {
      s.beta = rho_new / s.rho;
      s.rho = rho_new;
    }
  }
  S[j] = s;
}

__global__ void k_qmr_scalars2(int nb, const double* __restrict__ dots, double xi, int maxk, QmrState* S) {
  if ((int)threadIdx.x < nb) qmr_scalars2(threadIdx.x, nb, dots, xi, maxk, S);
}


// d = coefd d + coefq q ; sol += d ; q = (K^-1 r - kx gamma) + beta q   (active columns)
template <class P, int NB, bool VEC>
__global__ void __launch_bounds__(kT) k_qmr_update2(long long L, int nb, const typename P::S* __restrict__ r,
                                                    const typename P::S* __restrict__ kx,
                                                    const typename P::S* __restrict__ dinv,
                                                    const typename P::S* __restrict__ upre,
                                                    const QmrState* __restrict__ S, typename P::S* __restrict__ q,
                                                    typename P::S* __restrict__ d, typename P::S* __restrict__ sol) {
  using C = typename P::C;
  using A = typename P::A;
  __shared__ C cd[kMaxNb], cq[kMaxNb], gm[kMaxNb], bt[kMaxNb];
  __shared__ int up[kMaxNb], ac[kMaxNb];
  if (threadIdx.x < kMaxNb) {
    const bool ok = threadIdx.x < nb;
    const QmrState s = ok ? S[threadIdx.x] : QmrState{};
    cd[threadIdx.x] = to_c<P>(ok ? s.coefd : 0.0);
    cq[threadIdx.x] = to_c<P>(ok ? s.coefq : 0.0);
    gm[threadIdx.x] = to_c<P>(ok ? s.gamma : 0.0);
    bt[threadIdx.x] = to_c<P>(ok ? s.beta : 0.0);
    up[threadIdx.x] = ok ? s.upd : 0;
    ac[threadIdx.x] = ok ? s.active : 0;
  }
  __syncthreads();
  bool anyup = false;
#pragma unroll
  for (int j = 0; j < NB; ++j) anyup = anyup || up[j];
  if (!anyup) return;
  for (long long row = blockIdx.x * (long long)kT + threadIdx.x; row < L; row += (long long)gridDim.x * kT) {
    A qv[NB], dv[NB], sv_[NB], rv[NB], kv[NB];
    ldrow<P, NB, VEC>(q, row, nb, qv);
    ldrow<P, NB, VEC>(d, row, nb, dv);
    ldrow<P, NB, VEC>(sol, row, nb, sv_);
    ldrow<P, NB, VEC>(upre ? upre : r, row, nb, rv);
    ldrow<P, NB, VEC>(kx, row, nb, kv);
    const auto s = upre ? ld_or_one<P>(nullptr, row) : ld_or_one<P>(dinv, row);
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      if (!up[j]) continue;
      dv[j] = P::add(P::mulc(dv[j], cd[j]), P::mulc(qv[j], cq[j]));
      sv_[j] = P::add(sv_[j], dv[j]);
      if (ac[j]) qv[j] = P::add(P::sub(mul<P>(s, rv[j]), P::mulc(kv[j], gm[j])), P::mulc(qv[j], bt[j]));
    }
    strow<P, NB, VEC>(q, row, nb, qv);
    strow<P, NB, VEC>(d, row, nb, dv);
    strow<P, NB, VEC>(sol, row, nb, sv_);
  }
}

template <class P>
__global__ void k_reduce_g(const typename P::G* __restrict__ partial, int nblocks, int n, double* __restrict__ out) {
  using G = typename P::G;
  __shared__ G red[128];
  const int e = blockIdx.x;
  G v = P::gzero();
  for (int b = threadIdx.x; b < nblocks; b += 128) v = P::gadd(v, partial[(long long)b * n + e]);
  red[threadIdx.x] = v;
  __syncthreads();
  for (int w = 64; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] = P::gadd(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) out[e] = P::gval(red[0]);
}

// convert columns between modes with a per-column scale
template <class PS, class PD>
__global__ void k_convert_cols(long long L, int nc, const typename PS::S* src, long long lds, typename PD::S* dst,
                               long long ldd, const double* __restrict__ scale) {
  const long long total = L * nc;
  for (long long e = blockIdx.x * (long long)kT + threadIdx.x; e < total; e += (long long)gridDim.x * kT) {
    const long long row = e / nc;
    const int j = (int)(e % nc);
    double v;
    const typename PS::S sv = src[row * lds + j];
    if constexpr (PS::id == kDF64)
      v = (double)sv.hi + (double)sv.lo;
    else
      v = (double)sv;
    v *= scale[j];
    if constexpr (PD::id == kDF64) {
      const float hi = (float)v;
      dst[row * ldd + j] = df{hi, (float)(v - (double)hi)};
    } else {
      dst[row * ldd + j] = (typename PD::S)v;
    }
  }
}

template <class P>
cudaError_t init_p(long long L, int nb, const void* x, const void* b, const void* dinv, const CsrDev* K, void* u,
                   void* kx, void* q, void* r, void* d, void* sol, QmrState* S, void* partial, double* dots,
                   cudaStream_t st) {
  using SS = typename P::S;
  using G = typename P::G;
  const int g = occ_grid(k_qmr_init<P>, L);
  G* pd = reinterpret_cast<G*>(partial);
  const SS* upre = nullptr;
  if (K) {
    cudaError_t e = launch_spmm(P::id, *K, x, nb, kx, nb, nb, st);
    if (e == cudaSuccess) e = launch_spmm(P::id, *K, b, nb, u, nb, nb, st);
    if (e != cudaSuccess) return e;
    upre = (const SS*)u;
    dinv = nullptr;
  }
  k_qmr_init<P><<<g, kT, 0, st>>>(L, nb, (const SS*)x, (const SS*)b, (const SS*)dinv, (SS*)kx, upre, pd);
  k_reduce_g<P><<<5 * nb, 128, 0, st>>>(pd, g, 5 * nb, dots);
  k_qmr_init_scalars<<<1, 32, 0, st>>>(nb, dots, S);
  k_qmr_init_vec<P><<<qmr_grid(L * nb), kT, 0, st>>>(L, nb, (const SS*)b, (const SS*)dinv, (const SS*)kx, upre, S,
                                                     (SS*)q, (SS*)r, (SS*)d, (SS*)sol);
  return cudaGetLastError();
}

template <class P, int NB, bool VEC>
cudaError_t step_nb(long long L, int nb, const void* x, const void* w, int ready, unsigned* ticks, const void* kx,
                    const void* dinv, const CsrDev* K, void* u, const double* eta, double xi, int maxk, void* q,
                    void* r, void* d, void* sol, QmrState* S, void* partial, double* dots, cudaStream_t st) {
  using SS = typename P::S;
  using G = typename P::G;
  G* pd = reinterpret_cast<G*>(partial);
  if (K) dinv = nullptr;
  if (nb & (nb - 1)) ticks = nullptr;  // the tail reduction needs 4 nb to divide the CTA size
  if (ready < 1) {
    const int g = occ_grid(k_qmr_dots1<P, NB, VEC>, L);
    k_qmr_dots1<P, NB, VEC><<<g, kT, 0, st>>>(L, nb, (const SS*)x, (const SS*)q, (const SS*)w, pd);
    k_reduce_g<P><<<4 * nb, 128, 0, st>>>(pd, g, 4 * nb, dots);
  }
  if (ready < 2) k_qmr_scalars1<<<1, 32, 0, st>>>(nb, dots, eta, S);
  // with tickets the reductions and scalar steps run in the tails of the
  // producing kernels; otherwise as separate launches
  Tail t1;
  if (ticks) {
    t1.tick = ticks + 1;
    t1.out = dots;
    t1.dots = dots;
    t1.mode = K ? 2 : 3;
    t1.nb = nb;
    t1.xi = xi;
    t1.maxk = maxk;
    t1.S = S;
  }
  {
    const int g = occ_grid(k_qmr_update1<P, NB, VEC>, L);
    k_qmr_update1<P, NB, VEC><<<g, kT, 0, st>>>(L, nb, (const SS*)x, (const SS*)q, (const SS*)w, (const SS*)kx,
                                                (const SS*)dinv, eta, S, (SS*)r, pd, t1);
    if (!ticks) k_reduce_g<P><<<4 * nb, 128, 0, st>>>(pd, g, 4 * nb, dots);
  }
  bool scal2_done = ticks && !K;
  if (K) {
    // u = K^-1 r by SpMM; r^T u and x^T u replace dots 1 and 2
    Tail t2;
    if (ticks) {
      t2 = t1;
      t2.tick = ticks + 2;
      t2.out = dots + nb;
      t2.mode = 3;
    }
    int g = spmm_dots_p<P, 2>(nb, L, *K, r, nb, u, r, x, pd, t2, st);
    if (g && ticks) {
      scal2_done = true;
    } else {
      if (!g) {
        const cudaError_t e = launch_spmm(P::id, *K, r, nb, u, nb, nb, st);
        if (e != cudaSuccess) return e;
        g = occ_grid(k_qmr_dots_u<P, NB, VEC>, L);
        k_qmr_dots_u<P, NB, VEC><<<g, kT, 0, st>>>(L, nb, (const SS*)x, (const SS*)r, (const SS*)u, pd);
      }
      k_reduce_g<P><<<2 * nb, 128, 0, st>>>(pd, g, 2 * nb, dots + nb);
    }
  }
  if (!scal2_done) k_qmr_scalars2<<<1, 32, 0, st>>>(nb, dots, xi, maxk, S);
  k_qmr_update2<P, NB, VEC><<<occ_grid(k_qmr_update2<P, NB, VEC>, L), kT, 0, st>>>(
      L, nb, (const SS*)r, (const SS*)kx, (const SS*)dinv, K ? (const SS*)u : nullptr, S, (SS*)q, (SS*)d, (SS*)sol);
  return cudaGetLastError();
}

template <class P>
cudaError_t step_p(long long L, int nb, const void* x, const void* w, int dr, unsigned* tk, const void* kx,
                   const void* dinv, const CsrDev* K, void* u, const double* eta, double xi, int maxk, void* q,
                   void* r, void* d, void* sol, QmrState* S, void* partial, double* dots, cudaStream_t st) {
  constexpr size_t es = sizeof(typename P::S);
#define STEP(NBv)                                                                                                  \
  ((nb == NBv && (NBv * es) % 16 == 0)                                                                            \
       ? step_nb<P, NBv, true>(L, nb, x, w, dr, tk, kx, dinv, K, u, eta, xi, maxk, q, r, d, sol, S, partial, dots, \
                               st)                                                                                \
       : step_nb<P, NBv, false>(L, nb, x, w, dr, tk, kx, dinv, K, u, eta, xi, maxk, q, r, d, sol, S, partial,     \
                                dots, st))
  if (nb <= 1) return STEP(1);
  if (nb <= 2) return STEP(2);
  if (nb <= 4) return STEP(4);
  return STEP(8);
#undef STEP
}

}  // namespace

cudaError_t qmr_init(int prec, long long L, int nb, const void* x, const void* b, const void* dinv, const CsrDev* K,
                     void* u, void* kx, void* q, void* r, void* d, void* sol, QmrState* S, void* partial,
                     double* dots, cudaStream_t st) {
  if (nb < 1 || nb > kMaxNb || (K && !u)) return cudaErrorInvalidValue;
  switch (prec) {
    case kF32: return init_p<PF32>(L, nb, x, b, dinv, K, u, kx, q, r, d, sol, S, partial, dots, st);
    case kDF64: return init_p<PDF64>(L, nb, x, b, dinv, K, u, kx, q, r, d, sol, S, partial, dots, st);
    case kF64: return init_p<PF64>(L, nb, x, b, dinv, K, u, kx, q, r, d, sol, S, partial, dots, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t qmr_step(int prec, long long L, int nb, const void* x, const void* w, int ready, unsigned* ticks,
                     const void* kx, const void* dinv, const CsrDev* K, void* u, const double* eta, double xi,
                     int maxk, void* q, void* r, void* d, void* sol, QmrState* S, void* partial, double* dots,
                     cudaStream_t st) {
  if (nb < 1 || nb > kMaxNb || (K && !u) || ready < 0 || ready > 2) return cudaErrorInvalidValue;
  const int dr = ready;
  unsigned* tk = ticks;
  switch (prec) {
    case kF32:
      return step_p<PF32>(L, nb, x, w, dr, tk, kx, dinv, K, u, eta, xi, maxk, q, r, d, sol, S, partial, dots, st);
    case kDF64:
      return step_p<PDF64>(L, nb, x, w, dr, tk, kx, dinv, K, u, eta, xi, maxk, q, r, d, sol, S, partial, dots, st);
    case kF64:
      return step_p<PF64>(L, nb, x, w, dr, tk, kx, dinv, K, u, eta, xi, maxk, q, r, d, sol, S, partial, dots, st);
  }
  return cudaErrorInvalidValue;
}

namespace {
int spmm_chunks(int b) {
  int c = 0;
  while (b > 0) {
    b -= b >= 8 ? 8 : b >= 4 ? 4 : b >= 2 ? 2 : 1;
    ++c;
  }
  return c;
}
}  // namespace

int qmr_step_launches(int nb, bool sparse_k, int ready, bool ticks) {
  const bool fused = nb == 1 || nb == 2 || nb == 4 || nb == 8;
  int n = 2;                                   // update1, update2
  if (ready < 1) n += 2;                       // dots1 + reduce
  if (ready < 2) n += 1;                       // scalars1
  if (!ticks) n += 1;                          // reduce after update1
  if (sparse_k) n += fused ? (ticks ? 1 : 2) : spmm_chunks(nb) + 2;
  if (!(ticks && (!sparse_k || fused))) n += 1;  // scalars2
  return n;
}

cudaError_t qmr_op_dots(int prec, long long L, int nb, const CsrDev& K, const void* X, long long ldx, void* w,
                        const void* x, const void* q, void* partial, double* dots, unsigned* ticks,
                        const double* eta, QmrState* S, int* ready, cudaStream_t st) {
  *ready = 0;
  if (nb < 1 || nb > kMaxNb) return cudaErrorInvalidValue;
  Tail t;
  if (ticks) {
    t.tick = ticks;
    t.out = dots;
    t.dots = dots;
    t.mode = 1;
    t.nb = nb;
    t.eta = eta;
    t.S = S;
  }
  int g = 0;
  switch (prec) {
    case kF32: g = spmm_dots_p<PF32, 4>(nb, L, K, X, ldx, w, x, q, partial, t, st); break;
    case kDF64: g = spmm_dots_p<PDF64, 4>(nb, L, K, X, ldx, w, x, q, partial, t, st); break;
    case kF64: g = spmm_dots_p<PF64, 4>(nb, L, K, X, ldx, w, x, q, partial, t, st); break;
    default: return cudaErrorInvalidValue;
  }
  if (!g) return cudaSuccess;
  if (ticks) {
    *ready = 2;  // dots reduced and scalars1 done in the kernel's tail
    return cudaGetLastError();
  }
  switch (prec) {
    case kF32: k_reduce_g<PF32><<<4 * nb, 128, 0, st>>>(reinterpret_cast<const PF32::G*>(partial), g, 4 * nb, dots); break;
    case kDF64:
      k_reduce_g<PDF64><<<4 * nb, 128, 0, st>>>(reinterpret_cast<const PDF64::G*>(partial), g, 4 * nb, dots);
      break;
    default: k_reduce_g<PF64><<<4 * nb, 128, 0, st>>>(reinterpret_cast<const PF64::G*>(partial), g, 4 * nb, dots); break;
  }
  *ready = 1;
  return cudaGetLastError();
}
int qmr_init_launches(int nb, bool sparse_k) { return 4 + (sparse_k ? 2 * spmm_chunks(nb) : 0); }

int jd_solve(int prec, const CsrDev& K, int nb, const void* X, const void* Bv, const double* eta_host,
             const void* dinv, int maxit, double xi, void* T, int* steps, cudaStream_t st) {
  const long long n = K.rows;
  const size_t es = prec == kF32 ? 4 : 8;
  std::vector<void*> mem;
  auto take = [&](size_t bytes) -> void* {
    void* p = nullptr;
    if (cudaMalloc(&p, bytes ? bytes : 1) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    mem.push_back(p);
    return p;
  };
  auto done = [&](int code) {
    cudaStreamSynchronize(st);
    for (void* p : mem) cudaFree(p);
    return code;
  };
  const size_t blk = (size_t)n * nb * es;
  void *kx = take(blk), *q = take(blk), *r = take(blk), *d = take(blk), *w = take(blk), *u = take(blk);
  QmrState* S = static_cast<QmrState*>(take(sizeof(QmrState) * kMaxNb));
  double* dots = static_cast<double*>(take(sizeof(double) * 64));
  double* deta = static_cast<double*>(take(sizeof(double) * kMaxNb));
  unsigned* ticks = static_cast<unsigned*>(take(64));
  void* partial = take((size_t)kMaxGrid * 5 * kMaxNb * 8);
  if (!kx || !q || !r || !d || !w || !u || !S || !dots || !deta || !ticks || !partial) return done(-5);
  if (cudaMemsetAsync(ticks, 0, 64, st) != cudaSuccess ||
      cudaMemcpyAsync(deta, eta_host, sizeof(double) * nb, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      qmr_init(prec, n, nb, X, Bv, dinv, nullptr, u, kx, q, r, d, T, S, partial, dots, st) != cudaSuccess)
    return done(-6);
  int k = 0;
  for (; k < maxit; ++k) {
    int ready = 0;
    if (qmr_op_dots(prec, n, nb, K, q, nb, w, X, q, partial, dots, ticks, deta, S, &ready, st) != cudaSuccess)
      return done(-6);
    if (!ready && launch_spmm(prec, K, q, nb, w, nb, nb, st) != cudaSuccess) return done(-6);
    if (qmr_step(prec, n, nb, X, w, ready, ticks, kx, dinv, nullptr, u, deta, xi, maxit, q, r, d, T, S, partial, dots,
                 st) != cudaSuccess)
      return done(-6);
    if ((k + 1) % 8 == 0) {
      QmrState hs[kMaxNb];
      if (cudaMemcpyAsync(hs, S, sizeof(QmrState) * nb, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess)
        return done(-6);
      bool any = false;
      for (int j = 0; j < nb; ++j) any = any || hs[j].active;
      if (!any) {
        ++k;
        break;
      }
    }
  }
  if (steps) *steps = k;
  if (cudaStreamSynchronize(st) != cudaSuccess) return done(-6);
  return done(0);
}

cudaError_t convert_cols(int src_prec, const void* src, long long lds, int dst_prec, void* dst, long long ldd,
                         long long L, int nc, const double* scale, cudaStream_t st) {
  const int g = qmr_grid(L * nc);
#define CONV(PS_, PD_)                                                                                           \
  k_convert_cols<PS_, PD_><<<g, kT, 0, st>>>(L, nc, reinterpret_cast<const typename PS_::S*>(src), lds,      \
                                             reinterpret_cast<typename PD_::S*>(dst), ldd, scale)
  if (src_prec == kDF64 && dst_prec == kF32)
    CONV(PDF64, PF32);
  else if (src_prec == kF64 && dst_prec == kF32)
    CONV(PF64, PF32);
  else if (src_prec == kF32 && dst_prec == kF32)
    CONV(PF32, PF32);
  else if (src_prec == kF32 && dst_prec == kDF64)
    CONV(PF32, PDF64);
  else if (src_prec == kF32 && dst_prec == kF64)
    CONV(PF32, PF64);
  else if (src_prec == kDF64 && dst_prec == kDF64)
    CONV(PDF64, PDF64);
  else if (src_prec == kF64 && dst_prec == kF64)
    CONV(PF64, PF64);
  else
    return cudaErrorInvalidValue;
#undef CONV
  return cudaGetLastError();
}

}  // namespace phsvds
