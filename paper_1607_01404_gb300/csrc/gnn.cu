// Learned sparse-approximate-inverse preconditioner: graph of C = A^T A,
// forward and backward kernels of the message-passing network, Adam.  The
// network and the loss are described in include/phsvds_gnn.h.  Node features
// are FP32; all reductions (weight gradients, loss dots) go through the
// FP64-class Gram kernel with a fixed summation order.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/phsvds.h"
#include "../../include/phsvds_gnn.h"
#include "common.cuh"
#include "engine.h"
#include "gnn.h"
#include "kernels.h"

namespace phsvds {

namespace {

constexpr int kW = 32;      // width
constexpr int kLayers = 4;
constexpr float kRho = 0.9f;
constexpr int kT = 256;

int grid1(long long n) {
  long long g = (n + kT - 1) / kT;
  if (g < 1) g = 1;
  if (g > 152LL * 16) g = 152LL * 16;
  return (int)g;
}

// ---- graph of C = A^T A ----------------------------------------------------
__global__ void k_diag_deg(long long n, const int* __restrict__ cptr, const int* __restrict__ cidx,
                           const double* __restrict__ cval, double* __restrict__ cdiag, float* __restrict__ deg,
                           int* __restrict__ degmax) {
  int dm = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double d = 0.0;
    int k = 0;
    for (int p = cptr[i]; p < cptr[i + 1]; ++p) {
      if (cidx[p] == i)
        d = cval[p];
      else
        ++k;
    }
    cdiag[i] = d > 0 ? d : 1.0;
    deg[i] = (float)k;
    dm = k > dm ? k : dm;
  }
  atomicMax(degmax, dm);
}

// e_ij = c_ij / sqrt(c_ii c_jj) (0 on the diagonal), weighted degree
// E_i = sum_j |e_ij|, transpose positions, log c_ii
__global__ void k_edges(long long n, const int* __restrict__ cptr, const int* __restrict__ cidx,
                        const double* __restrict__ cval, const double* __restrict__ cdiag, float* __restrict__ e,
                        float* __restrict__ wdeg, int* __restrict__ tpos, float* __restrict__ logc) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    logc[i] = (float)log(cdiag[i]);
    double wd = 0.0;
    for (int p = cptr[i]; p < cptr[i + 1]; ++p) {
      const int j = cidx[p];
      const float ev = j == i ? 0.f : (float)(cval[p] / sqrt(cdiag[i] * cdiag[j]));
      e[p] = ev;
      wd += fabs((double)ev);
      // position of (j, i): binary search in the sorted row j
      int lo = cptr[j], hi = cptr[j + 1] - 1, pos = -1;
      while (lo <= hi) {
        const int mid = (lo + hi) >> 1;
        const int c = cidx[mid];
        if (c == i) {
          pos = mid;
          break;
        }
        if (c < i)
          lo = mid + 1;
        else
          hi = mid - 1;
      }
      if (tpos) tpos[p] = pos >= 0 ? pos : p;
    }
    wdeg[i] = (float)wd;
  }
}

__global__ void k_x0(long long n, const float* __restrict__ logc, const float* __restrict__ deg, float logmean,
                     float degmax, float* __restrict__ x0) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    x0[2 * i] = logc[i] - logmean;
    x0[2 * i + 1] = deg[i] / degmax;
  }
}

// ---- forward ----------------------------------------------------------------
// The layer weights W1, W2 are used in bfloat16 (round to nearest even of the
// FP32 master copy; FP32 products and accumulation), in the forward pass and
// in the backward pass alike; biases and heads stay FP32.
__device__ __forceinline__ float bf16r(float x) {
  const unsigned u = __float_as_uint(x);
  return __uint_as_float(((u + 0x7fffu + ((u >> 16) & 1u)) >> 16) << 16);
}

// z = h W1 + Eh W2 + b, hout = relu(z).  A CTA takes tiles of 128 rows: h and
// Eh of the tile are staged in shared memory with coalesced 16-byte loads
// (rows padded against bank conflicts).  Thread t computes outputs
// [8 (t mod 4), 8 (t mod 4) + 8) of rows t / 4 and t / 4 + 64, so each pair of
// 16-byte weight loads from shared memory serves two rows (the weights, not
// the rows, were the shared-memory traffic of one row per thread); z and hout
// leave as 32-byte row segments (a warp writes 8 whole rows at a time).  The
// multiply-adds of an output run in column order, as in the backward pass.
constexpr int kLRows = 128;
template <int FIN>
__global__ void __launch_bounds__(kT) k_layer_fwd(long long n, const float* __restrict__ h,
                                                  const float* __restrict__ Eh, const float* __restrict__ W1,
                                                  const float* __restrict__ W2, const float* __restrict__ b,
                                                  float* __restrict__ z, float* __restrict__ hout) {
  static_assert(2 * kT == 4 * kLRows, "four threads per row, two rows per thread");
  // staged row stride: FIN + 4 floats (rows start on 16-byte boundaries for
  // 16-byte staging, 8 consecutive rows on distinct banks) when FIN is a
  // multiple of 4, else FIN + 1
  constexpr int HS = FIN % 4 == 0 ? FIN + 4 : FIN + 1;
  __shared__ __align__(16) float w1[FIN * kW], w2[FIN * kW];
  __shared__ float bb[kW];
  __shared__ __align__(16) float hs[kLRows * HS], es[kLRows * HS];
  for (int e = threadIdx.x; e < FIN * kW; e += blockDim.x) {
    w1[e] = bf16r(W1[e]);
    w2[e] = bf16r(W2[e]);
  }
  if (threadIdx.x < kW) bb[threadIdx.x] = b[threadIdx.x];
  const int row = threadIdx.x >> 2, j0 = 8 * (threadIdx.x & 3);
  for (long long r0 = (long long)blockIdx.x * kLRows; r0 < n; r0 += (long long)gridDim.x * kLRows) {
    const int rows = (int)(n - r0 < kLRows ? n - r0 : kLRows);
    __syncthreads();  // weights staged / previous tile consumed
    if constexpr (FIN % 4 == 0) {
      const float4* h4 = reinterpret_cast<const float4*>(h + r0 * FIN);
      const float4* e4 = reinterpret_cast<const float4*>(Eh + r0 * FIN);
      for (int e = threadIdx.x; e < rows * (FIN / 4); e += kT) {
        const int rr = e / (FIN / 4), c = 4 * (e % (FIN / 4));
        *reinterpret_cast<float4*>(hs + rr * HS + c) = h4[e];
        *reinterpret_cast<float4*>(es + rr * HS + c) = e4[e];
      }
    } else {
      for (int e = threadIdx.x; e < rows * FIN; e += kT) {
        const int rr = e / FIN, c = e % FIN;
        hs[rr * HS + c] = h[r0 * FIN + e];
        es[rr * HS + c] = Eh[r0 * FIN + e];
      }
    }
    __syncthreads();
    float a0[8], a1[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) a0[j] = a1[j] = bb[j0 + j];
    const int rb = row + kLRows / 2;
    const int ra_s = row < rows ? row : 0, rb_s = rb < rows ? rb : 0;  // rows past the tile read row 0
#pragma unroll 4
    for (int c = 0; c < FIN; ++c) {
      const float4 u0 = *reinterpret_cast<const float4*>(w1 + c * kW + j0);
      const float4 u1 = *reinterpret_cast<const float4*>(w1 + c * kW + j0 + 4);
      const float4 v0 = *reinterpret_cast<const float4*>(w2 + c * kW + j0);
      const float4 v1 = *reinterpret_cast<const float4*>(w2 + c * kW + j0 + 4);
      const float wa[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
      const float wb[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
      const float ha = hs[ra_s * HS + c], ea = es[ra_s * HS + c];
      const float hb = hs[rb_s * HS + c], eb = es[rb_s * HS + c];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        a0[j] = fmaf(ha, wa[j], fmaf(ea, wb[j], a0[j]));
        a1[j] = fmaf(hb, wa[j], fmaf(eb, wb[j], a1[j]));
      }
    }
    for (int t = 0; t < 2; ++t) {
      const int rr = t == 0 ? row : rb;
      if (rr >= rows) continue;
      const float* a = t == 0 ? a0 : a1;
      float4* zo = reinterpret_cast<float4*>(z + (r0 + rr) * kW + j0);
      float4* ho = reinterpret_cast<float4*>(hout + (r0 + rr) * kW + j0);
      zo[0] = make_float4(a[0], a[1], a[2], a[3]);
      zo[1] = make_float4(a[4], a[5], a[6], a[7]);
      ho[0] = make_float4(fmaxf(a[0], 0.f), fmaxf(a[1], 0.f), fmaxf(a[2], 0.f), fmaxf(a[3], 0.f));
      ho[1] = make_float4(fmaxf(a[4], 0.f), fmaxf(a[5], 0.f), fmaxf(a[6], 0.f), fmaxf(a[7], 0.f));
    }
  }
}

// |e_ij| / max(E_i, E_j): the off-diagonal weight that keeps M diagonally dominant
__device__ __forceinline__ float edge_weight(float e, float Ei, float Ej) {
  const float mx = fmaxf(Ei, Ej);
  return mx > 0.f ? fabsf(e) / mx : 0.f;
}

__device__ __forceinline__ float softplusf(float x) { return x > 20.f ? x : log1pf(expf(x)); }
__device__ __forceinline__ float sigmoidf_(float x) { return 1.f / (1.f + expf(-x)); }

__global__ void k_heads_node(long long n, const float* __restrict__ h, const float* __restrict__ ws,
                             const float* __restrict__ wd, const float* __restrict__ bd,
                             const double* __restrict__ cdiag, float* __restrict__ u, float* __restrict__ gpre,
                             float* __restrict__ delta) {
  __shared__ float sws[kW], swd[kW];
  if (threadIdx.x < kW) {
    sws[threadIdx.x] = ws[threadIdx.x];
    swd[threadIdx.x] = wd[threadIdx.x];
  }
  __syncthreads();
  const float b = *bd;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    float a = 0.f, g = b;
#pragma unroll
    for (int c = 0; c < kW; ++c) {
      a = fmaf(h[i * kW + c], sws[c], a);
      g = fmaf(h[i * kW + c], swd[c], g);
    }
    u[i] = a;
    gpre[i] = g;
    delta[i] = (float)(softplusf(g) / cdiag[i]);
  }
}

__global__ void k_heads_edge(long long n, const int* __restrict__ cptr, const int* __restrict__ cidx,
                             const float* __restrict__ e, const float* __restrict__ u, const float* __restrict__ delta,
                             const float* __restrict__ wdeg, const float* __restrict__ we, const float* __restrict__ bs,
                             float* __restrict__ s, float* __restrict__ m) {
  const float w = *we, b = *bs;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    for (int p = cptr[i]; p < cptr[i + 1]; ++p) {
      const int j = cidx[p];
      if (j == i) {
        s[p] = 0.f;
        m[p] = delta[i];
      } else {
        const float sv = tanhf(u[i] + u[j] + w * e[p] + b);
        const float mu = fminf(delta[i], delta[j]);
        s[p] = sv;
        m[p] = kRho * sv * mu * edge_weight(e[p], wdeg[i], wdeg[j]);
      }
    }
  }
}

// ---- backward ---------------------------------------------------------------
// dm[k] (+)= sum_p c_p R[i, p] R[j, p] for entry k = (i, j) (R row-major n x P)
__global__ void k_dm_outer(long long n, const int* __restrict__ cptr, const int* __restrict__ cidx,
                           const double* __restrict__ R, const double* __restrict__ c, int P, int accumulate,
                           float* __restrict__ dm) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double ri[8];
    for (int p = 0; p < P; ++p) ri[p] = c[p] * R[i * P + p];
    for (int k = cptr[i]; k < cptr[i + 1]; ++k) {
      const long long j = cidx[k];
      double acc = 0.0;
      for (int p = 0; p < P; ++p) acc += ri[p] * R[j * P + p];
      dm[k] = accumulate ? dm[k] + (float)acc : (float)acc;
    }
  }
}

// x <- x - omega z (n x P row-major)
__global__ void k_axpy_neg(long long total, double omega, const double* __restrict__ z, double* __restrict__ x) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x)
    x[e] -= omega * z[e];
}

// heads backward per row: ddelta_i, du_i; per-entry da_k = dm_k rho mu w_ij (1 - s^2)
// for the we / bs gradients (written to da and dae = da * e).
__global__ void k_heads_bwd(long long n, const int* __restrict__ cptr, const int* __restrict__ cidx,
                            const int* __restrict__ tpos, const float* __restrict__ dm, const float* __restrict__ s,
                            const float* __restrict__ delta, const float* __restrict__ wdeg,
                            const float* __restrict__ e, float* __restrict__ ddelta, float* __restrict__ du,
                            float* __restrict__ da, float* __restrict__ dae) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    float dd = 0.f, duu = 0.f;
    for (int k = cptr[i]; k < cptr[i + 1]; ++k) {
      const int j = cidx[k];
      if (j == i) {
        dd += dm[k];
        da[k] = 0.f;
        dae[k] = 0.f;
        continue;
      }
      const float di = delta[i], dj = delta[j];
      const float mu = fminf(di, dj);
      const float w = edge_weight(e[k], wdeg[i], wdeg[j]);
      const float sv = s[k];
      const float dpair = dm[k] + dm[tpos[k]];
      const float t = 1.f - sv * sv;
      duu += dpair * kRho * mu * w * t;
      const bool to_i = (di < dj) || (di == dj && i < j);
      if (to_i) dd += dpair * kRho * sv * w;
      const float dak = dm[k] * kRho * mu * w * t;
      da[k] = dak;
      dae[k] = dak * e[k];
    }
    ddelta[i] = dd;
    du[i] = duu;
  }
}

// dg = ddelta / c_ii * sigmoid(gpre); dh[i, c] = dg wd[c] + du ws[c]; gu = [dg, du]
__global__ void k_node_bwd(long long n, const float* __restrict__ ddelta, const float* __restrict__ du,
                           const float* __restrict__ gpre, const double* __restrict__ cdiag,
                           const float* __restrict__ ws, const float* __restrict__ wd, float* __restrict__ gu,
                           float* __restrict__ dh) {
  __shared__ float sws[kW], swd[kW];
  if (threadIdx.x < kW) {
    sws[threadIdx.x] = ws[threadIdx.x];
    swd[threadIdx.x] = wd[threadIdx.x];
  }
  __syncthreads();
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float dg = (float)(ddelta[i] / cdiag[i]) * sigmoidf_(gpre[i]);
    const float dv = du[i];
    gu[2 * i] = dg;
    gu[2 * i + 1] = dv;
#pragma unroll
    for (int c = 0; c < kW; ++c) dh[i * kW + c] = dg * swd[c] + dv * sws[c];
  }
}

__global__ void k_relu_bwd(long long total, const float* __restrict__ z, const float* __restrict__ dh,
                           float* __restrict__ dz) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x)
    dz[e] = z[e] > 0.f ? dh[e] : 0.f;
}

// out[i, c] = (add ? add[i, c] : 0) + sum_j dz[i, j] W[c, j]   (W: FOUT x 32, i.e. dz W^T)
template <int FOUT>
__global__ void __launch_bounds__(kT) k_rowmat_t(long long n, const float* __restrict__ dz, const float* __restrict__ W,
                                                 const float* __restrict__ add, float* __restrict__ out) {
  __shared__ float w[FOUT * kW];
  for (int e = threadIdx.x; e < FOUT * kW; e += blockDim.x) w[e] = bf16r(W[e]);  // the forward's weights
  __syncthreads();
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    float d[kW];
#pragma unroll
    for (int j = 0; j < kW; ++j) d[j] = dz[i * kW + j];
    for (int c = 0; c < FOUT; ++c) {
      float acc = add ? add[i * FOUT + c] : 0.f;
#pragma unroll
      for (int j = 0; j < kW; ++j) acc = fmaf(d[j], w[c * kW + j], acc);
      out[i * FOUT + c] = acc;
    }
  }
}

__global__ void k_to_f64(long long n, const float* __restrict__ x, double* __restrict__ y) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = (double)x[i];
}

// t <- t - omega (C t) / c_ii (damped Jacobi smoothing, row-major n x P)
__global__ void k_smooth(long long n, int P, const double* __restrict__ ct, const double* __restrict__ cdiag,
                         double omega, double* __restrict__ t) {
  const long long total = n * P;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x)
    t[e] -= omega * ct[e] / cdiag[e / P];
}

__global__ void k_fill1(long long n, float* __restrict__ x) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] = 1.f;
}

__global__ void k_adam(int np, float* __restrict__ p, const double* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  const float gi = (float)g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

struct Offsets {
  int W1[kLayers], W2[kLayers], b[kLayers], ws, wd, we, bs, bd, total;
  Offsets() {
    int o = 0;
    for (int l = 0; l < kLayers; ++l) {
      const int fin = l == 0 ? 2 : kW;
      W1[l] = o;
      o += fin * kW;
      W2[l] = o;
      o += fin * kW;
      b[l] = o;
      o += kW;
    }
    ws = o;
    o += kW;
    wd = o;
    o += kW;
    we = o++;
    bs = o++;
    bd = o++;
    total = o;
  }
};

}  // namespace
}  // namespace phsvds

using namespace phsvds;

struct phsvds_gnn {
  cudaStream_t st = nullptr;
  bool own_stream = false;
  long long n = 0, nnz = 0;
  std::vector<void*> allocs;
  int *cptr = nullptr, *cidx = nullptr, *tpos = nullptr;
  double *cval = nullptr, *cdiag = nullptr;
  float *deg = nullptr, *wdeg = nullptr, *e = nullptr, *x0 = nullptr, *logc = nullptr;
  float* prm = nullptr;  // device parameters
  float* h[kLayers + 1] = {};
  float* Eh[kLayers] = {};
  float* z[kLayers] = {};
  float *u = nullptr, *gpre = nullptr, *delta = nullptr, *s = nullptr, *m = nullptr;
  float *dm = nullptr, *da = nullptr, *dae = nullptr, *ddelta = nullptr, *du = nullptr, *gu = nullptr;
  float *dh = nullptr, *dz = nullptr, *tmp = nullptr, *tmp2 = nullptr, *ones = nullptr;
  double* kb[6] = {};  // n x 8 FP64 blocks of the loss (samples and products)
  double *dcoef = nullptr, *dG = nullptr, *dstage = nullptr, *grad = nullptr;
  float *am = nullptr, *av = nullptr;
  double* m64 = nullptr;  // FP64 copy of M for the FP64 solver mode
  double *w0 = nullptr, *w1 = nullptr, *w2 = nullptr;  // n x 8 FP64 work blocks (pairs, C products)
  void* partial = nullptr;
  bool train = false;
  long long launches = 0;
  Offsets off;
};

namespace {

int gfail(cudaError_t e, const char* where) {
  phsvds::set_last_error(std::string(cudaGetErrorString(e)) + " at " + where);
  cudaGetLastError();
  return SVDS_ERR_CUDA;
}
#define GK(x)                                    \
  do {                                           \
    cudaError_t _e = (x);                        \
    if (_e != cudaSuccess) return gfail(_e, #x); \
  } while (0)

template <class T>
int galloc(phsvds_gnn* g, T** p, size_t count) {
  if (count == 0) count = 1;
  void* q = nullptr;
  if (cudaMalloc(&q, sizeof(T) * count) != cudaSuccess) {
    cudaGetLastError();
    return SVDS_ERR_NOMEM;
  }
  g->allocs.push_back(q);
  *p = reinterpret_cast<T*>(q);
  return 0;
}

CsrDev Ecsr(const phsvds_gnn* g, const float* vals) {
  CsrDev c;
  c.rows = g->n;
  c.cols = g->n;
  c.nnz = g->nnz;
  c.rowptr = g->cptr;
  c.colidx = g->cidx;
  c.v32 = vals;
  return c;
}

// C = A^T A on its pattern (FP64 values)
CsrDev Ccsr(const phsvds_gnn* g) {
  CsrDev c = Ecsr(g, nullptr);
  c.v64 = g->cval;
  return c;
}


// G (p x q row-major, host) = P^T Q over all rows (FP64-class accumulation)
int gram_host(phsvds_gnn* g, const float* P, int p, const float* Q, int ldq, int q0, int q, std::vector<double>& out) {
  out.assign((size_t)p * q, 0.0);
  for (int c0 = 0; c0 < q; c0 += 8) {
    const int qc = q - c0 < 8 ? q - c0 : 8;
    SegV Ps{P, p, p};
    SegV Qs{Q + q0 + c0, ldq, qc};
    int nb = 0;
    GK(launch_gram(kF32, 0, g->n, &Ps, 1, Qs, g->partial, gram_default_blocks(), &nb, g->st));
    GK(launch_gram_reduce(kF32, g->partial, nb, p * qc, g->dG, g->st));
    std::vector<double> h((size_t)p * qc);
    GK(cudaMemcpyAsync(h.data(), g->dG, sizeof(double) * p * qc, cudaMemcpyDeviceToHost, g->st));
    GK(cudaStreamSynchronize(g->st));
    for (int i = 0; i < p; ++i)
      for (int j = 0; j < qc; ++j) out[(size_t)i * q + c0 + j] = h[(size_t)i * qc + j];
  }
  return 0;
}

int forward_impl(phsvds_gnn* g, const float* params_host) {
  const Offsets& o = g->off;
  GK(cudaMemcpyAsync(g->prm, params_host, sizeof(float) * o.total, cudaMemcpyHostToDevice, g->st));
  const long long n = g->n;
  const int gr = grid1(n);
  for (int l = 0; l < kLayers; ++l) {
    const int fin = l == 0 ? 2 : kW;
    GK(launch_spmm(kF32, Ecsr(g, g->e), g->h[l], fin, g->Eh[l], fin, fin, g->st));
    if (l == 0)
      k_layer_fwd<2><<<gr, kT, 0, g->st>>>(n, g->h[l], g->Eh[l], g->prm + o.W1[l], g->prm + o.W2[l], g->prm + o.b[l],
                                           g->z[l], g->h[l + 1]);
    else
      k_layer_fwd<kW><<<gr, kT, 0, g->st>>>(n, g->h[l], g->Eh[l], g->prm + o.W1[l], g->prm + o.W2[l],
                                            g->prm + o.b[l], g->z[l], g->h[l + 1]);
  }
  k_heads_node<<<gr, kT, 0, g->st>>>(n, g->h[kLayers], g->prm + o.ws, g->prm + o.wd, g->prm + o.bd, g->cdiag, g->u,
                                     g->gpre, g->delta);
  k_heads_edge<<<gr, kT, 0, g->st>>>(n, g->cptr, g->cidx, g->e, g->u, g->delta, g->wdeg, g->prm + o.we,
                                     g->prm + o.bs, g->s, g->m);
  GK(cudaGetLastError());
  g->launches += 1 + 4 + 3 * 5 + 2;  // SpMM chunks of 2 and 4 x 8 columns, layers, heads
  return 0;
}

CsrDev Mcsr64(const phsvds_gnn* g) {
  CsrDev c = Ecsr(g, nullptr);
  c.v64 = g->m64;
  return c;
}

// diag of P^T Q for row-major n x q FP64 blocks (host result)
int gram_diag64(phsvds_gnn* g, const double* P, const double* Q, int q, std::vector<double>& out) {
  SegV Ps{P, q, q}, Qs{Q, q, q};
  int nb = 0;
  GK(launch_gram(kF64, 0, g->n, &Ps, 1, Qs, g->partial, gram_default_blocks(), &nb, g->st));
  GK(launch_gram_reduce(kF64, g->partial, nb, q * q, g->dG, g->st));
  std::vector<double> h((size_t)q * q);
  GK(cudaMemcpyAsync(h.data(), g->dG, sizeof(double) * q * q, cudaMemcpyDeviceToHost, g->st));
  GK(cudaStreamSynchronize(g->st));
  out.resize(q);
  for (int p = 0; p < q; ++p) out[p] = h[(size_t)p * q + p];
  return 0;
}

// rho_p = <M C t_p, C t_p> / <C t_p, t_p> for the columns of the device block T;
// leaves R = C T in Rb.
int rayleigh_dev(phsvds_gnn* g, const double* T, int q, double* Rb, double* Zb, std::vector<double>& rho,
                 std::vector<double>& rt) {
  GK(launch_spmm(kF64, Ccsr(g), T, q, Rb, q, q, g->st));
  GK(launch_spmm(kF64, Mcsr64(g), Rb, q, Zb, q, q, g->st));
  std::vector<double> zr;
  int rc;
  if ((rc = gram_diag64(g, Zb, Rb, q, zr)) || (rc = gram_diag64(g, Rb, T, q, rt))) return rc;
  rho.resize(q);
  for (int p = 0; p < q; ++p) rho[p] = zr[p] / rt[p];
  return 0;
}

// Condition-number loss of M C from start blocks T0 (n x P) and X0 (n x Q)
// (host FP64 column-major): T = (M C)^ps T0, X = (I - omega M C)^ss X0 with
// omega = 1 / max rho(T); L = log mean rho(T) - log mean rho(X).  dL/dm with
// the samples held fixed is written to g->dm.
int kappa_term(phsvds_gnn* g, const double* T0, int P, int ps, const double* X0, int Q, int ss, double* loss) {
  const long long n = g->n;
  double *T = g->kb[0], *X = g->kb[1], *W = g->kb[2], *Z = g->kb[3], *R = g->kb[4], *Y = g->kb[5];
  k_to_f64<<<grid1(g->nnz), kT, 0, g->st>>>(g->nnz, g->m, g->m64);
  GK(cudaMemcpyAsync(W, T0, sizeof(double) * n * P, cudaMemcpyHostToDevice, g->st));
  GK(launch_from_f64_colmajor(kF64, n, P, W, n, T, P, 1.0, g->st));
  for (int s = 0; s < ps; ++s) {
    GK(launch_spmm(kF64, Ccsr(g), T, P, W, P, P, g->st));
    GK(launch_spmm(kF64, Mcsr64(g), W, P, T, P, P, g->st));
  }
  std::vector<double> ra, rta, rb, rtb;
  int rc;
  if ((rc = rayleigh_dev(g, T, P, R, Z, ra, rta))) return rc;
  double amax = 0.0, sa = 0.0;
  for (double v : ra) {
    amax = std::max(amax, v);
    sa += v;
  }
  if (!(amax > 0) || !std::isfinite(sa)) {
    phsvds::set_last_error("phsvds_gnn_loss_grad: M C T vanishes or is not finite");
    return SVDS_ERR_NUMERIC;
  }
  const double omega = 1.0 / amax;
  GK(cudaMemcpyAsync(W, X0, sizeof(double) * n * Q, cudaMemcpyHostToDevice, g->st));
  GK(launch_from_f64_colmajor(kF64, n, Q, W, n, X, Q, 1.0, g->st));
  for (int s = 0; s < ss; ++s) {
    GK(launch_spmm(kF64, Ccsr(g), X, Q, W, Q, Q, g->st));
    GK(launch_spmm(kF64, Mcsr64(g), W, Q, Z, Q, Q, g->st));
    k_axpy_neg<<<grid1(n * Q), kT, 0, g->st>>>(n * Q, omega, Z, X);
  }
  if ((rc = rayleigh_dev(g, X, Q, Y, Z, rb, rtb))) return rc;
  double sb = 0.0;
  for (double v : rb) sb += v;
  if (!(sb > 0) || !std::isfinite(sb)) {
    phsvds::set_last_error("phsvds_gnn_loss_grad: M C X vanishes or is not finite");
    return SVDS_ERR_NUMERIC;
  }
  *loss = std::log(sa / P) - std::log(sb / Q);
  // d rho_p / d m_ij = r_ip r_jp / <r_p, t_p>
  std::vector<double> cc(16, 0.0);
  for (int p = 0; p < P; ++p) cc[p] = 1.0 / (sa * rta[p]);
  for (int q = 0; q < Q; ++q) cc[8 + q] = -1.0 / (sb * rtb[q]);
  GK(cudaMemcpyAsync(g->dcoef, cc.data(), sizeof(double) * 16, cudaMemcpyHostToDevice, g->st));
  k_dm_outer<<<grid1(n), kT, 0, g->st>>>(n, g->cptr, g->cidx, R, g->dcoef, P, 0, g->dm);
  k_dm_outer<<<grid1(n), kT, 0, g->st>>>(n, g->cptr, g->cidx, Y, g->dcoef + 8, Q, 1, g->dm);
  GK(cudaGetLastError());
  GK(cudaStreamSynchronize(g->st));  // cc is read by the copy above
  return 0;
}

}  // namespace

namespace phsvds {

int gnn_build(phsvds_gnn** out, const DevMatrix& D, bool user_orientation, bool train, cudaStream_t st) {
  int rc = 0;
  phsvds_gnn* g = new phsvds_gnn();
  g->st = st;
  // nodes = columns of the user's matrix (user_orientation), else of the
  // device matrix (the operator C of stage 1)
  const bool tr = user_orientation && D.transposed;
  const long long n = tr ? D.m : D.n;
  const int* rp = tr ? D.rowptrT : D.rowptr;   // rows of the user's A
  const int* ci = tr ? D.colidxT : D.colidx;
  const int* rpT = tr ? D.rowptr : D.rowptrT;  // rows of the user's A^T
  const int* ciT = tr ? D.colidx : D.colidxT;
  const double* va = tr ? D.v64T : D.v64;
  const double* vT = tr ? D.v64 : D.v64T;
  g->n = n;
  int *cnt = nullptr, *err = nullptr, *work = nullptr, *dmax = nullptr;
  auto fail = [&](int code) {
    for (void* p : g->allocs) cudaFree(p);
    delete g;
    return code;
  };
  if ((rc = galloc(g, &g->cptr, n + 1)) || (rc = galloc(g, &cnt, n + 1)) || (rc = galloc(g, &err, 4)) ||
      (rc = galloc(g, &work, scan_work_ints(n) + 4)) || (rc = galloc(g, &dmax, 4)))
    return fail(rc);
  if (cudaMemsetAsync(err, 0, 4 * sizeof(int), st) != cudaSuccess ||
      cudaMemsetAsync(dmax, 0, 4 * sizeof(int), st) != cudaSuccess)
    return fail(gfail(cudaGetLastError(), "memset"));
  if (launch_normal_count(n, rpT, ciT, rp, ci, cnt, err, st) != cudaSuccess)
    return fail(gfail(cudaGetLastError(), "normal count"));
  if (launch_exclusive_scan(n, cnt, g->cptr, work, st) != cudaSuccess) return fail(gfail(cudaGetLastError(), "scan"));
  int herr = 0, hnnz = 0;
  cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(&hnnz, g->cptr + n, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) return fail(gfail(cudaGetLastError(), "graph count"));
  if (herr) {
    phsvds::set_last_error("phsvds_gnn_create: a column of A has more nonzeros than the merge supports");
    return fail(SVDS_ERR_SHAPE);
  }
  g->nnz = hnnz;
  const long long nnz = hnnz;
  if ((rc = galloc(g, &g->cidx, nnz)) || (rc = galloc(g, &g->cval, nnz)) || (rc = galloc(g, &g->cdiag, n)) ||
      (rc = galloc(g, &g->deg, n)) || (rc = galloc(g, &g->wdeg, n)) || (rc = galloc(g, &g->e, nnz)) ||
      (rc = galloc(g, &g->logc, n)) ||
      (rc = galloc(g, &g->prm, g->off.total)) || (rc = galloc(g, &g->u, n)) || (rc = galloc(g, &g->gpre, n)) ||
      (rc = galloc(g, &g->delta, n)) || (rc = galloc(g, &g->s, nnz)) || (rc = galloc(g, &g->m, nnz)) ||
      (rc = galloc(g, &g->ones, n > nnz ? n : nnz)) || (rc = galloc(g, &g->dG, 64 * 64)))
    return fail(rc);
  // training buffers (backward pass, loss, Adam)
  if (train &&
      ((rc = galloc(g, &g->tpos, nnz)) || (rc = galloc(g, &g->dm, nnz)) || (rc = galloc(g, &g->da, nnz)) ||
       (rc = galloc(g, &g->dae, nnz)) || (rc = galloc(g, &g->ddelta, n)) || (rc = galloc(g, &g->du, n)) ||
       (rc = galloc(g, &g->gu, 2 * n)) || (rc = galloc(g, &g->dh, n * kW)) || (rc = galloc(g, &g->dz, n * kW)) ||
       (rc = galloc(g, &g->tmp, n * kW)) || (rc = galloc(g, &g->tmp2, n * kW)) || (rc = galloc(g, &g->dcoef, 64)) ||
       (rc = galloc(g, &g->dstage, n * 8)) || (rc = galloc(g, &g->grad, g->off.total)) ||
       (rc = galloc(g, &g->am, g->off.total)) || (rc = galloc(g, &g->av, g->off.total))))
    return fail(rc);
  g->train = train;
  if ((rc = galloc(g, reinterpret_cast<char**>(&g->partial), gram_partial_bytes(gram_default_blocks(), kW, 8))))
    return fail(rc);
  g->h[0] = nullptr;
  if ((rc = galloc(g, &g->x0, 2 * n))) return fail(rc);
  g->h[0] = g->x0;
  for (int l = 0; l < kLayers; ++l) {
    const int fin = l == 0 ? 2 : kW;
    if ((rc = galloc(g, &g->Eh[l], n * fin)) || (rc = galloc(g, &g->z[l], n * kW)) ||
        (rc = galloc(g, &g->h[l + 1], n * kW)))
      return fail(rc);
  }
  // device values are scale * A (a power of two): C in the user's units is exact
  if (launch_normal_fill(n, rpT, ciT, vT, rp, ci, va, 1.0 / (D.scale * D.scale), g->cptr, g->cidx, g->cval, st) !=
      cudaSuccess)
    return fail(gfail(cudaGetLastError(), "normal fill"));
  k_diag_deg<<<grid1(n), kT, 0, st>>>(n, g->cptr, g->cidx, g->cval, g->cdiag, g->deg, dmax);
  k_edges<<<grid1(n), kT, 0, st>>>(n, g->cptr, g->cidx, g->cval, g->cdiag, g->e, g->wdeg, g->tpos, g->logc);
  k_fill1<<<grid1(n > nnz ? n : nnz), kT, 0, st>>>(n > nnz ? n : nnz, g->ones);
  if (cudaGetLastError() != cudaSuccess) return fail(gfail(cudaGetLastError(), "graph kernels"));
  // mean of log c_ii (FP64-class Gram of the ones vector with log c)
  {
    SegV Ps{g->ones, 1, 1}, Qs{g->logc, 1, 1};
    int nb = 0;
    launch_gram(kF32, 0, n, &Ps, 1, Qs, g->partial, gram_default_blocks(), &nb, st);
    launch_gram_reduce(kF32, g->partial, nb, 1, g->dG, st);
  }
  double hsum = 0;
  int hdmax = 0;
  cudaMemcpyAsync(&hsum, g->dG, sizeof(double), cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(&hdmax, dmax, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) return fail(gfail(cudaGetLastError(), "graph features"));
  k_x0<<<grid1(n), kT, 0, st>>>(n, g->logc, g->deg, (float)(hsum / n), (float)(hdmax > 0 ? hdmax : 1), g->x0);
  g->launches += 12;  // count, scan (3), fill, diagonal, edges, ones, Gram + reduce, features
  if (cudaStreamSynchronize(st) != cudaSuccess) return fail(gfail(cudaGetLastError(), "graph x0"));
  *out = g;
  return SVDS_OK;
}


int gnn_precond(phsvds_gnn* g, const float* params, CsrDev* f32, CsrDev* f64) {
  if (!g || !params || !f32) return SVDS_ERR_ARG;
  int rc = forward_impl(g, params);
  if (rc) return rc;
  *f32 = Ecsr(g, g->m);
  if (f64) {
    if (!g->m64 && (rc = galloc(g, &g->m64, g->nnz))) return rc;
    k_to_f64<<<grid1(g->nnz), kT, 0, g->st>>>(g->nnz, g->m, g->m64);
    GK(cudaGetLastError());
    g->launches += 1;
    *f64 = Ecsr(g, nullptr);
    f64->v64 = g->m64;
  }
  return SVDS_OK;
}

long long gnn_launches(const phsvds_gnn* g) { return g ? g->launches : 0; }

}  // namespace phsvds

extern "C" {

int phsvds_gnn_num_params(void) { return Offsets().total; }

int phsvds_gnn_init(uint64_t seed, float* params) {
  if (!params) return SVDS_ERR_ARG;
  uint64_t st = seed;
  auto next = [&]() {  // splitmix64
    st += 0x9E3779B97F4A7C15ULL;
    uint64_t z = st;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
  };
  auto normal = [&]() {  // Box-Muller on two uniforms in (0, 1]
    const double u1 = ((next() >> 11) + 1.0) * (1.0 / 9007199254740992.0);
    const double u2 = (next() >> 11) * (1.0 / 9007199254740992.0);
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
  };
  const Offsets o;
  for (int e = 0; e < o.total; ++e) params[e] = 0.f;
  for (int l = 0; l < kLayers; ++l) {
    const int fin = l == 0 ? 2 : kW;
    const double sd = std::sqrt(2.0 / (fin + kW));
    for (int e = 0; e < fin * kW; ++e) params[o.W1[l] + e] = (float)(sd * normal());
    for (int e = 0; e < fin * kW; ++e) params[o.W2[l] + e] = (float)(sd * normal());
  }
  for (int c = 0; c < kW; ++c) params[o.wd + c] = (float)(std::sqrt(1.0 / kW) * normal());
  for (int c = 0; c < kW; ++c) params[o.ws + c] = (float)(0.1 * std::sqrt(1.0 / kW) * normal());
  params[o.bd] = 0.5f;
  params[o.bs] = 1.f;
  return SVDS_OK;
}

int phsvds_gnn_create(phsvds_gnn** out, const svds_csr* A, void* stream) {
  if (!out || !A || A->m < 1 || A->n < 1 || A->nnz < 0 || !A->rowptr) return SVDS_ERR_ARG;
  *out = nullptr;
  // the device copy, transpose and validation of svds_create are reused
  svds_opts o;
  svds_opts_default(&o);
  o.stream = stream;
  svds_handle* h = nullptr;
  int rc = svds_create(&h, A, &o);
  if (rc) return rc;
  phsvds_gnn* g = nullptr;
  rc = gnn_build(&g, h->A, true, true, h->stream);
  if (rc == 0 && h->own_stream) {
    // the temporary handle's stream goes away with it
    cudaStream_t s2;
    if (cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking) != cudaSuccess) {
      rc = gfail(cudaGetLastError(), "stream");
      phsvds_gnn_destroy(g);
      g = nullptr;
    } else {
      g->st = s2;
      g->own_stream = true;
    }
  }
  svds_destroy(h);
  if (rc) return rc;
  *out = g;
  return SVDS_OK;
}

void phsvds_gnn_destroy(phsvds_gnn* g) {
  if (!g) return;
  if (g->st) cudaStreamSynchronize(g->st);
  for (void* p : g->allocs) cudaFree(p);
  if (g->own_stream) cudaStreamDestroy(g->st);
  delete g;
}

int phsvds_gnn_shape(const phsvds_gnn* g, int64_t* n, int64_t* nnz) {
  if (!g || !n || !nnz) return SVDS_ERR_ARG;
  *n = g->n;
  *nnz = g->nnz;
  return SVDS_OK;
}

int phsvds_gnn_pattern(const phsvds_gnn* g, int32_t* rowptr, int32_t* colidx) {
  if (!g || !rowptr || !colidx) return SVDS_ERR_ARG;
  GK(cudaMemcpyAsync(rowptr, g->cptr, sizeof(int) * (g->n + 1), cudaMemcpyDeviceToHost, g->st));
  GK(cudaMemcpyAsync(colidx, g->cidx, sizeof(int) * g->nnz, cudaMemcpyDeviceToHost, g->st));
  GK(cudaStreamSynchronize(g->st));
  return SVDS_OK;
}

int phsvds_gnn_forward(phsvds_gnn* g, const float* params, float* mvals) {
  if (!g || !params) return SVDS_ERR_ARG;
  int rc = forward_impl(g, params);
  if (rc) return rc;
  if (mvals) GK(cudaMemcpyAsync(mvals, g->m, sizeof(float) * g->nnz, cudaMemcpyDeviceToHost, g->st));
  GK(cudaStreamSynchronize(g->st));
  return SVDS_OK;
}

int phsvds_gnn_loss_grad(phsvds_gnn* g, const float* params, const double* T0, int P, int power_steps,
                         const double* X0, int Q, int smooth_steps, double* loss, double* grad) {
  if (!g || !g->train || !params || !T0 || !X0 || P < 1 || P > 8 || Q < 1 || Q > 8 || power_steps < 0 ||
      power_steps > 100 || smooth_steps < 0 || smooth_steps > 1000 || !loss || !grad)
    return SVDS_ERR_ARG;
  const Offsets& o = g->off;
  const long long n = g->n;
  const int gr = grid1(n);
  int rc = forward_impl(g, params);
  if (rc) return rc;
  if (!g->m64 && (rc = galloc(g, &g->m64, g->nnz))) return rc;
  for (int i = 0; i < 6; ++i)
    if (!g->kb[i] && (rc = galloc(g, &g->kb[i], g->n * 8))) return rc;
  double L = 0.0;
  if ((rc = kappa_term(g, T0, P, power_steps, X0, Q, smooth_steps, &L))) return rc;
  std::vector<double> gr_h(o.total, 0.0);
  // heads
  k_heads_bwd<<<gr, kT, 0, g->st>>>(n, g->cptr, g->cidx, g->tpos, g->dm, g->s, g->delta, g->wdeg, g->e, g->ddelta,
                                    g->du, g->da, g->dae);
  k_node_bwd<<<gr, kT, 0, g->st>>>(n, g->ddelta, g->du, g->gpre, g->cdiag, g->prm + o.ws, g->prm + o.wd, g->gu,
                                   g->dh);
  GK(cudaGetLastError());
  std::vector<double> G;
  // we, bs: sums over the entries of the pattern, against the ones vector (length >= nnz)
  {
    SegV Ps{g->ones, 1, 1};
    for (int w = 0; w < 2; ++w) {
      SegV Qs{w == 0 ? g->dae : g->da, 1, 1};
      int nb = 0;
      GK(launch_gram(kF32, 0, g->nnz, &Ps, 1, Qs, g->partial, gram_default_blocks(), &nb, g->st));
      GK(launch_gram_reduce(kF32, g->partial, nb, 1, g->dG + w, g->st));
    }
    double hv[2];
    GK(cudaMemcpyAsync(hv, g->dG, sizeof(double) * 2, cudaMemcpyDeviceToHost, g->st));
    GK(cudaStreamSynchronize(g->st));
    gr_h[o.we] = hv[0];
    gr_h[o.bs] = hv[1];
  }
  // wd, ws from h4^T [dg du]; bd = sum dg
  if ((rc = gram_host(g, g->h[kLayers], kW, g->gu, 2, 0, 2, G))) return rc;
  for (int c = 0; c < kW; ++c) {
    gr_h[o.wd + c] = G[(size_t)c * 2 + 0];
    gr_h[o.ws + c] = G[(size_t)c * 2 + 1];
  }
  if ((rc = gram_host(g, g->ones, 1, g->gu, 2, 0, 1, G))) return rc;
  gr_h[o.bd] = G[0];
  // layers
  for (int l = kLayers - 1; l >= 0; --l) {
    const int fin = l == 0 ? 2 : kW;
    k_relu_bwd<<<grid1(n * kW), kT, 0, g->st>>>(n * kW, g->z[l], g->dh, g->dz);
    GK(cudaGetLastError());
    if ((rc = gram_host(g, g->h[l], fin, g->dz, kW, 0, kW, G))) return rc;
    for (int e = 0; e < fin * kW; ++e) gr_h[o.W1[l] + e] = G[e];
    if ((rc = gram_host(g, g->Eh[l], fin, g->dz, kW, 0, kW, G))) return rc;
    for (int e = 0; e < fin * kW; ++e) gr_h[o.W2[l] + e] = G[e];
    if ((rc = gram_host(g, g->ones, 1, g->dz, kW, 0, kW, G))) return rc;
    for (int e = 0; e < kW; ++e) gr_h[o.b[l] + e] = G[e];
    if (l > 0) {
      // dh_l = dz W1^T + E (dz W2^T)
      k_rowmat_t<kW><<<gr, kT, 0, g->st>>>(n, g->dz, g->prm + o.W2[l], nullptr, g->tmp);
      GK(launch_spmm(kF32, Ecsr(g, g->e), g->tmp, kW, g->tmp2, kW, kW, g->st));
      k_rowmat_t<kW><<<gr, kT, 0, g->st>>>(n, g->dz, g->prm + o.W1[l], g->tmp2, g->dh);
      GK(cudaGetLastError());
    }
  }
  *loss = L;
  std::memcpy(grad, gr_h.data(), sizeof(double) * o.total);
  return SVDS_OK;
}

}  // extern "C"

namespace {

int ensure_work(phsvds_gnn* g) {
  int rc;
  if (!g->w0 && ((rc = galloc(g, &g->w0, g->n * 8)) || (rc = galloc(g, &g->w1, g->n * 8)) ||
                 (rc = galloc(g, &g->w2, g->n * 8))))
    return rc;
  return 0;
}

// device row-major n x q (ld q) -> host column-major
int to_host_cm(phsvds_gnn* g, const double* dsrc, int q, double* host) {
  GK(launch_to_f64_colmajor(kF64, g->n, q, dsrc, q, g->w2, g->n, 1.0, g->st));
  GK(cudaMemcpyAsync(host, g->w2, sizeof(double) * g->n * q, cudaMemcpyDeviceToHost, g->st));
  return 0;
}

}  // namespace

extern "C" {

int phsvds_gnn_pairs(phsvds_gnn* g, int P, int smooth, uint64_t seed, double* R, double* T) {
  if (!g || P < 1 || P > 8 || smooth < 0 || smooth > 1000 || !R || !T) return SVDS_ERR_ARG;
  int rc = ensure_work(g);
  if (rc) return rc;
  const long long n = g->n;
  GK(launch_fill_normal(kF64, n, g->w0, P, P, seed, g->st));
  for (int s = 0; s < smooth; ++s) {
    GK(launch_spmm(kF64, Ccsr(g), g->w0, P, g->w1, P, P, g->st));
    k_smooth<<<grid1(n * P), kT, 0, g->st>>>(n, P, g->w1, g->cdiag, 2.0 / 3.0, g->w0);
    GK(cudaGetLastError());
  }
  GK(launch_spmm(kF64, Ccsr(g), g->w0, P, g->w1, P, P, g->st));
  if ((rc = to_host_cm(g, g->w0, P, T))) return rc;
  GK(cudaStreamSynchronize(g->st));
  if ((rc = to_host_cm(g, g->w1, P, R))) return rc;
  GK(cudaStreamSynchronize(g->st));
  return SVDS_OK;
}

int phsvds_gnn_apply_c(phsvds_gnn* g, const double* X, int q, double* Y) {
  if (!g || q < 1 || q > 8 || !X || !Y) return SVDS_ERR_ARG;
  int rc = ensure_work(g);
  if (rc) return rc;
  const long long n = g->n;
  GK(cudaMemcpyAsync(g->w2, X, sizeof(double) * n * q, cudaMemcpyHostToDevice, g->st));
  GK(launch_from_f64_colmajor(kF64, n, q, g->w2, n, g->w0, q, 1.0, g->st));
  GK(launch_spmm(kF64, Ccsr(g), g->w0, q, g->w1, q, q, g->st));
  if ((rc = to_host_cm(g, g->w1, q, Y))) return rc;
  GK(cudaStreamSynchronize(g->st));
  return SVDS_OK;
}

int phsvds_gnn_save(const char* path, const float* params) {
  if (!path || !params) return SVDS_ERR_ARG;
  std::FILE* f = std::fopen(path, "wb");
  if (!f) return SVDS_ERR_ARG;
  const int32_t cnt = Offsets().total;
  bool ok = std::fwrite("PHSGNN01", 1, 8, f) == 8 && std::fwrite(&cnt, sizeof(cnt), 1, f) == 1 &&
            std::fwrite(params, sizeof(float), cnt, f) == (size_t)cnt;
  ok = (std::fclose(f) == 0) && ok;
  return ok ? SVDS_OK : SVDS_ERR_ARG;
}

int phsvds_gnn_load(const char* path, float* params) {
  if (!path || !params) return SVDS_ERR_ARG;
  std::FILE* f = std::fopen(path, "rb");
  if (!f) return SVDS_ERR_ARG;
  char tag[8];
  int32_t cnt = 0;
  const int32_t want = Offsets().total;
  std::vector<float> buf(want);
  bool ok = std::fread(tag, 1, 8, f) == 8 && std::memcmp(tag, "PHSGNN01", 8) == 0 &&
            std::fread(&cnt, sizeof(cnt), 1, f) == 1 && cnt == want &&
            std::fread(buf.data(), sizeof(float), want, f) == (size_t)want;
  std::fclose(f);
  if (!ok) return SVDS_ERR_ARG;
  for (float v : buf)
    if (!std::isfinite(v)) return SVDS_ERR_ARG;
  std::memcpy(params, buf.data(), sizeof(float) * want);
  return SVDS_OK;
}

int phsvds_gnn_adam(phsvds_gnn* g, float* params, const double* grad, float* m, float* v, int step, float lr) {
  if (!g || !g->train || !params || !grad || !m || !v || step < 1 || !(lr > 0)) return SVDS_ERR_ARG;
  const int np = g->off.total;
  float* dp = g->prm;
  GK(cudaMemcpyAsync(dp, params, sizeof(float) * np, cudaMemcpyHostToDevice, g->st));
  GK(cudaMemcpyAsync(g->grad, grad, sizeof(double) * np, cudaMemcpyHostToDevice, g->st));
  GK(cudaMemcpyAsync(g->am, m, sizeof(float) * np, cudaMemcpyHostToDevice, g->st));
  GK(cudaMemcpyAsync(g->av, v, sizeof(float) * np, cudaMemcpyHostToDevice, g->st));
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  k_adam<<<(np + 255) / 256, 256, 0, g->st>>>(np, dp, g->grad, g->am, g->av, lr, b1, b2, 1e-8f, c1, c2);
  GK(cudaGetLastError());
  GK(cudaMemcpyAsync(params, dp, sizeof(float) * np, cudaMemcpyDeviceToHost, g->st));
  GK(cudaMemcpyAsync(m, g->am, sizeof(float) * np, cudaMemcpyDeviceToHost, g->st));
  GK(cudaMemcpyAsync(v, g->av, sizeof(float) * np, cudaMemcpyDeviceToHost, g->st));
  GK(cudaStreamSynchronize(g->st));
  return SVDS_OK;
}

}  // extern "C"
