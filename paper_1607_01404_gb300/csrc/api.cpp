// C-ABI of the PHSVDS library (include/phsvds.h, include/phsvds_kernels.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/phsvds.h"
#include "../../include/phsvds_gnn.h"
#include "../../include/phsvds_kernels.h"
#include "engine.h"
#include "bjacobi.h"
#include "jdqmr.h"
#include "hostla.h"
#include "kernels.h"

using namespace phsvds;

namespace phsvds {
const char* last_error_cstr();
}

namespace {

int cuda_fail(cudaError_t e, const char* where) {
  phsvds::set_last_error(std::string(cudaGetErrorString(e)) + " at " + where);
  cudaGetLastError();
  return SVDS_ERR_CUDA;
}

#define CKR(x)                                   \
  do {                                           \
    cudaError_t _e = (x);                        \
    if (_e != cudaSuccess) return cuda_fail(_e, #x); \
  } while (0)

template <class T>
int dalloc(svds_handle* h, T** p, size_t count) {
  if (count == 0) count = 1;
  void* q = nullptr;
  if (cudaMalloc(&q, sizeof(T) * count) != cudaSuccess) {
    cudaGetLastError();
    return SVDS_ERR_NOMEM;
  }
  h->allocs.push_back(q);
  *p = reinterpret_cast<T*>(q);
  return 0;
}

int validate_host_csr(const svds_csr* A) {
  const int32_t* rp = A->rowptr;
  if (rp[0] != 0 || rp[A->m] != A->nnz) return SVDS_ERR_CSR;
  for (int64_t i = 0; i < A->m; ++i) {
    if (rp[i + 1] < rp[i]) return SVDS_ERR_CSR;
    int64_t prev = -1;
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
      const int64_t c = A->colidx[k];
      if (c < 0 || c >= A->n || c <= prev) return SVDS_ERR_CSR;
      prev = c;
      if (!std::isfinite(A->vals[k])) return SVDS_ERR_VALUE;
    }
  }
  return 0;
}

void release(svds_handle* h) {
  for (void* p : h->allocs) cudaFree(p);
  h->allocs.clear();
  if (h->arena.base) cudaFree(h->arena.base);
  h->arena = phsvds::Arena{};
  if (h->hpin) cudaFreeHost(h->hpin);
  h->hpin = nullptr;
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  h->stream = nullptr;
}

int create_impl(svds_handle* h, const svds_csr* A) {
  cudaStream_t st = h->stream;
  const long long mu = A->m, nu = A->n, nnz = A->nnz;
  int *rp = nullptr, *ci = nullptr, *rpT = nullptr, *ciT = nullptr, *work = nullptr, *flags = nullptr;
  double *vals = nullptr, *valsT = nullptr;
  int rc;
  if ((rc = dalloc(h, &rp, mu + 1)) || (rc = dalloc(h, &ci, nnz)) || (rc = dalloc(h, &vals, nnz)) ||
      (rc = dalloc(h, &rpT, nu + 1)) || (rc = dalloc(h, &ciT, nnz)) || (rc = dalloc(h, &valsT, nnz)) ||
      (rc = dalloc(h, &work, transpose_work_ints(nu))) || (rc = dalloc(h, &flags, 4)))
    return rc;
  const cudaMemcpyKind kind = A->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  CKR(cudaMemcpyAsync(rp, A->rowptr, sizeof(int) * (mu + 1), kind, st));
  if (nnz > 0) {
    CKR(cudaMemcpyAsync(ci, A->colidx, sizeof(int) * nnz, kind, st));
    CKR(cudaMemcpyAsync(vals, A->vals, sizeof(double) * nnz, kind, st));
  }
  CKR(cudaMemsetAsync(flags, 0, sizeof(int) * 4, st));
  if (A->on_device) {
    // validation on the device before anything else uses the arrays
    int hrp[2] = {0, 0};
    CKR(cudaMemcpyAsync(&hrp[0], rp, sizeof(int), cudaMemcpyDeviceToHost, st));
    CKR(cudaMemcpyAsync(&hrp[1], rp + mu, sizeof(int), cudaMemcpyDeviceToHost, st));
    CKR(cudaStreamSynchronize(st));
    if (hrp[0] != 0 || hrp[1] != nnz) return SVDS_ERR_CSR;
    CKR(launch_csr_validate(mu, nu, rp, ci, vals, flags, st));
    int hf = 0;
    CKR(cudaMemcpyAsync(&hf, flags, sizeof(int), cudaMemcpyDeviceToHost, st));
    CKR(cudaStreamSynchronize(st));
    if (hf & 2) return SVDS_ERR_CSR;
    if (hf & 4) return SVDS_ERR_VALUE;
  }
  CKR(launch_csr_transpose(mu, nu, nnz, rp, ci, vals, rpT, ciT, valsT, work, st));
  // power-of-two scaling keeps the double-float format far from float overflow
  unsigned long long* amax = reinterpret_cast<unsigned long long*>(flags + 2);
  CKR(launch_absmax(nnz, vals, amax, st));
  unsigned long long hbits = 0;
  CKR(cudaMemcpyAsync(&hbits, amax, sizeof(hbits), cudaMemcpyDeviceToHost, st));
  CKR(cudaStreamSynchronize(st));
  double amaxv;
  std::memcpy(&amaxv, &hbits, sizeof(double));
  double scale = 1.0;
  if (amaxv > 0 && std::isfinite(amaxv)) scale = std::ldexp(1.0, -std::ilogb(amaxv));
  DevMatrix& D = h->A;
  D.transposed = mu < nu;
  D.m = D.transposed ? nu : mu;
  D.n = D.transposed ? mu : nu;
  D.nnz = nnz;
  D.scale = scale;
  D.rowptr = D.transposed ? rpT : rp;
  D.colidx = D.transposed ? ciT : ci;
  D.rowptrT = D.transposed ? rp : rpT;
  D.colidxT = D.transposed ? ci : ciT;
  const double* va = D.transposed ? valsT : vals;
  const double* vaT = D.transposed ? vals : valsT;
  int rc2;
  if ((rc2 = dalloc(h, &D.v32, nnz)) || (rc2 = dalloc(h, &D.v32lo, nnz)) || (rc2 = dalloc(h, &D.v64, nnz)) ||
      (rc2 = dalloc(h, &D.v32T, nnz)) || (rc2 = dalloc(h, &D.v32loT, nnz)) || (rc2 = dalloc(h, &D.v64T, nnz)) ||
      (rc2 = dalloc(h, &D.colsq, D.n)) || (rc2 = dalloc(h, &D.rowsq, D.m)))
    return rc2;
  CKR(cudaMemsetAsync(flags, 0, sizeof(int), st));
  CKR(launch_csr_values(nnz, va, scale, D.v32, D.v32lo, D.v64, flags, st));
  CKR(launch_csr_values(nnz, vaT, scale, D.v32T, D.v32loT, D.v64T, flags, st));
  CKR(launch_row_sumsq(D.n, D.rowptrT, D.v64T, D.colsq, st));
  CKR(launch_row_sumsq(D.m, D.rowptr, D.v64, D.rowsq, st));
  int hf = 0;
  CKR(cudaMemcpyAsync(&hf, flags, sizeof(int), cudaMemcpyDeviceToHost, st));
  CKR(cudaStreamSynchronize(st));
  D.exact32 = (hf & 1) == 0;
  return 0;
}

int check_opts(const svds_opts& o) {
  if (o.stage1_precision != SVDS_DF64 && o.stage1_precision != SVDS_FP32 && o.stage1_precision != SVDS_BF16 &&
      o.stage1_precision != SVDS_NATIVE_FP64)
    return SVDS_ERR_ARG;
  if (o.maxBlockSize < 0 || o.maxBlockSize > 64 || o.maxBasisSize < 0 || o.minRestartSize < 0) return SVDS_ERR_ARG;
  if ((o.method_stage1 != SVDS_GDPK && o.method_stage1 != SVDS_JDQMR && o.method_stage1 != SVDS_DYNAMIC) ||
      (o.method_stage2 != SVDS_GDPK && o.method_stage2 != SVDS_JDQMR) || o.innerMaxIt < 0 || o.innerRelTol < 0)
    return SVDS_ERR_ARG;
  if (o.innerPrecision != 0 && o.innerPrecision != SVDS_FP32 && o.innerPrecision != SVDS_DF64) return SVDS_ERR_ARG;
  if (o.initSize < 0 || (o.initSize > 0 && !o.initV)) return SVDS_ERR_ARG;
  if (o.precond != SVDS_PRECOND_NONE && o.precond != SVDS_PRECOND_JACOBI && o.precond != SVDS_PRECOND_LEARNED &&
      o.precond != SVDS_PRECOND_BLOCKJACOBI)
    return SVDS_ERR_ARG;
  if (o.normalOperator != SVDS_NORMAL_AUTO && o.normalOperator != SVDS_NORMAL_TWOPASS &&
      o.normalOperator != SVDS_NORMAL_EXPLICIT)
    return SVDS_ERR_ARG;
  if (!(o.relTol >= 0) || !std::isfinite(o.relTol)) return SVDS_ERR_ARG;
  if (o.precondBlockSize < 0 || o.precondBlockSize > phsvds::kBjMaxBlock) return SVDS_ERR_ARG;
  return 0;
}

}  // namespace

extern "C" {

int svds_opts_default(svds_opts* o) {
  if (!o) return SVDS_ERR_ARG;
  std::memset(o, 0, sizeof(*o));
  o->maxBlockSize = 1;
  o->method_stage1 = SVDS_GDPK;
  o->method_stage2 = SVDS_GDPK;
  o->stage1_precision = SVDS_DF64;
  o->stage1_polish = 1;
  o->precond = SVDS_PRECOND_JACOBI;
  o->seed = 1;
  o->innerPrecision = SVDS_FP32;
  return SVDS_OK;
}

int svds_create(svds_handle** out, const svds_csr* A, const svds_opts* opts) {
  if (!out || !A) return SVDS_ERR_ARG;
  *out = nullptr;
  if (A->m < 1 || A->n < 1 || A->nnz < 0 || A->nnz > 2147483647LL || A->m > 2147483646LL || A->n > 2147483646LL)
    return SVDS_ERR_SHAPE;
  if (!A->rowptr || (A->nnz > 0 && (!A->colidx || !A->vals))) return SVDS_ERR_ARG;
  svds_opts o;
  if (opts)
    o = *opts;
  else
    svds_opts_default(&o);
  if (check_opts(o)) return SVDS_ERR_ARG;
  std::vector<float> gnn_params;
  if (o.precond == SVDS_PRECOND_LEARNED) {
    gnn_params.resize(phsvds_gnn_num_params());
    if (o.precondParams) {
      std::memcpy(gnn_params.data(), o.precondParams, sizeof(float) * gnn_params.size());
    } else if (!o.precondModel || phsvds_gnn_load(o.precondModel, gnn_params.data()) != SVDS_OK) {
      phsvds::set_last_error("SVDS_PRECOND_LEARNED needs precondParams or a readable precondModel");
      return SVDS_ERR_ARG;
    }
  }
  if (!A->on_device) {
    int rc = validate_host_csr(A);
    if (rc) return rc;
  }
  svds_handle* h = new svds_handle();
  h->opts = o;
  h->opts.initV = nullptr;  // initial guesses are per solve: copied from opts at solve time
  h->opts.initSize = 0;
  h->opts.precondParams = nullptr;  // kept in gnn_params
  h->opts.precondModel = nullptr;
  h->gnn_params.swap(gnn_params);
  cudaGetDevice(&h->device);
  if (o.stream) {
    h->stream = reinterpret_cast<cudaStream_t>(o.stream);
  } else {
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete h;
      return cuda_fail(cudaGetLastError(), "cudaStreamCreateWithFlags");
    }
    h->own_stream = true;
  }
  int rc = create_impl(h, A);
  if (rc) {
    release(h);
    delete h;
    return rc;
  }
  if (o.initSize > 0) {
    h->initV.assign(o.initV, o.initV + (size_t)o.initSize * A->n);
    h->opts.initV = h->initV.data();
    h->opts.initSize = o.initSize;
  }
  *out = h;
  return SVDS_OK;
}

int svds_create_op(svds_handle** out, int64_t m, int64_t n, svds_apply_fn apply, void* ctx, const double* diagC,
                   const svds_opts* opts) {
  if (!out || !apply) return SVDS_ERR_ARG;
  *out = nullptr;
  if (n < 1 || m < n || m > 2147483646LL) return SVDS_ERR_SHAPE;
  svds_opts o;
  if (opts)
    o = *opts;
  else
    svds_opts_default(&o);
  if (check_opts(o)) return SVDS_ERR_ARG;
  // no matrix values: no bfloat16 rounding, no explicit A^T A, and only the
  // Jacobi preconditioner from the caller's diagonal of A^T A
  if (o.stage1_precision == SVDS_BF16) return SVDS_ERR_ARG;
  if (o.precond != SVDS_PRECOND_NONE && o.precond != SVDS_PRECOND_JACOBI) return SVDS_ERR_ARG;
  if (o.precond == SVDS_PRECOND_JACOBI && !diagC) return SVDS_ERR_ARG;
  if (diagC)
    for (int64_t i = 0; i < n; ++i)
      if (!std::isfinite(diagC[i]) || diagC[i] < 0) return SVDS_ERR_VALUE;
  svds_handle* h = new svds_handle();
  h->opts = o;
  h->opts.initV = nullptr;
  h->opts.initSize = 0;
  h->opts.precondParams = nullptr;
  h->opts.precondModel = nullptr;
  cudaGetDevice(&h->device);
  if (o.stream) {
    h->stream = reinterpret_cast<cudaStream_t>(o.stream);
  } else {
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete h;
      return cuda_fail(cudaGetLastError(), "cudaStreamCreateWithFlags");
    }
    h->own_stream = true;
  }
  phsvds::DevMatrix& D = h->A;
  D.m = m;
  D.n = n;
  D.nnz = 0;
  D.nnzC = 0;  // C is the caller's operator
  D.user = apply;
  D.user_ctx = ctx;
  if (diagC) {
    int rc = dalloc(h, &D.colsq, n);
    if (!rc) {
      const cudaError_t e = cudaMemcpyAsync(D.colsq, diagC, sizeof(double) * n, cudaMemcpyHostToDevice, h->stream);
      if (e == cudaSuccess && cudaStreamSynchronize(h->stream) == cudaSuccess) rc = 0;
      else rc = cuda_fail(e != cudaSuccess ? e : cudaGetLastError(), "diagC upload");
    }
    if (rc) {
      release(h);
      delete h;
      return rc;
    }
  }
  if (o.initSize > 0) {
    h->initV.assign(o.initV, o.initV + (size_t)o.initSize * n);
    h->opts.initV = h->initV.data();
    h->opts.initSize = o.initSize;
  }
  *out = h;
  return SVDS_OK;
}

int svds_solve(svds_handle* h, int k, int target, double tol, double* sigma, double* U, double* V, double* rnorm,
               int* numConverged, svds_stats* stats) {
  if (!h || !sigma) return SVDS_ERR_ARG;
  if (target != SVDS_LARGEST && target != SVDS_SMALLEST) return SVDS_ERR_ARG;
  if (!(tol > 0) || !std::isfinite(tol)) return SVDS_ERR_ARG;
  if (k < 1 || k > h->A.n) return SVDS_ERR_SHAPE;
  if (h->opts.initSize > 0 && h->A.transposed) return SVDS_ERR_ARG;  // guesses are right vectors of the tall matrix
  cudaSetDevice(h->device);
  return phsvds::solve(h, k, target, tol, sigma, U, V, rnorm, numConverged, stats);
}

int svds_condest(svds_handle* h, double relTol, double* sigma_max, double* sigma_min, double* kappa,
                 svds_stats* stats) {
  if (!h || !sigma_max || !sigma_min || !kappa || !(relTol > 0) || !std::isfinite(relTol)) return SVDS_ERR_ARG;
  if (h->opts.initSize > 0) return SVDS_ERR_ARG;  // guesses belong to k-triplet solves
  const svds_opts saved = h->opts;
  h->opts.relTol = relTol;
  h->opts.maxBlockSize = 1;
  h->opts.maxBasisSize = 0;
  h->opts.minRestartSize = 0;
  h->opts.aNorm = 0.0;
  double smax = 0.0, smin = 0.0;
  int nc = 0;
  svds_stats st[2] = {};
  int rc = svds_solve(h, 1, SVDS_LARGEST, relTol, &smax, nullptr, nullptr, nullptr, &nc, &st[0]);
  if (rc == SVDS_OK) {
    h->opts.aNorm = smax;
    rc = svds_solve(h, 1, SVDS_SMALLEST, relTol, &smin, nullptr, nullptr, nullptr, &nc, &st[1]);
  }
  h->opts = saved;
  if (stats) {
    stats[0] = st[0];
    stats[1] = st[1];
  }
  *sigma_max = smax;
  *sigma_min = smin;
  *kappa = smin > 0 ? smax / smin : INFINITY;
  return rc;
}

void svds_destroy(svds_handle* h) {
  if (!h) return;
  cudaSetDevice(h->device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  release(h);
  delete h;
}

const char* svds_strerror(int code) {
  switch (code) {
    case SVDS_OK: return "success";
    case SVDS_ERR_ARG: return "invalid argument";
    case SVDS_ERR_SHAPE: return "inconsistent sizes (m, n, nnz or k)";
    case SVDS_ERR_CSR: return "malformed CSR (row pointers, or column indices unsorted / out of range)";
    case SVDS_ERR_VALUE: return "non-finite matrix value";
    case SVDS_ERR_NOMEM: return "out of memory";
    case SVDS_ERR_CUDA: return "CUDA error";
    case SVDS_ERR_NUMERIC: return "numerical breakdown";
    case SVDS_ERR_OPERATOR: return "the caller-supplied operator failed";
    case SVDS_ERR_MAXIT: return "matvec or time budget exhausted";
    default: return "unknown error";
  }
}

const char* svds_last_error(void) { return phsvds::last_error_cstr(); }

// ---------------------------------------------------------------------------
// kernel-level entry points
// ---------------------------------------------------------------------------
static bool prec_ok(int p) { return p == kF32 || p == kDF64 || p == kF64; }

int phsvds_spmm(int prec, int64_t rows, int64_t cols, int64_t nnz, const int32_t* rowptr, const int32_t* colidx,
                const float* v32, const float* v32lo, const double* v64, const void* X, int64_t ldx, void* Y,
                int64_t ldy, int b, void* stream) {
  if (!prec_ok(prec) || rows < 0 || cols < 0 || nnz < 0 || b < 0 || ldx < b || ldy < b) return SVDS_ERR_ARG;
  if (rows > 0 && (!rowptr || !Y)) return SVDS_ERR_ARG;
  if (nnz > 0 && (!colidx || !X)) return SVDS_ERR_ARG;
  if (prec == kF64 ? (nnz > 0 && !v64) : (nnz > 0 && !v32)) return SVDS_ERR_ARG;
  CsrDev A;
  A.rows = rows;
  A.cols = cols;
  A.nnz = nnz;
  A.rowptr = rowptr;
  A.colidx = colidx;
  A.v32 = v32;
  A.v32lo = v32lo;
  A.v64 = v64;
  CKR(launch_spmm(prec, A, X, ldx, Y, ldy, b, reinterpret_cast<cudaStream_t>(stream)));
  return 0;
}

int phsvds_spmm_bf16(int64_t rows, int64_t cols, int64_t nnz, const int32_t* rowptr, const int32_t* colidx,
                     const uint16_t* v16, const float* X, int64_t ldx, float* Y, int64_t ldy, int b, void* stream) {
  if (rows < 0 || cols < 0 || nnz < 0 || b < 0 || ldx < b || ldy < b) return SVDS_ERR_ARG;
  if (rows > 0 && (!rowptr || !Y)) return SVDS_ERR_ARG;
  if (nnz > 0 && (!colidx || !X || !v16)) return SVDS_ERR_ARG;
  CsrDev A;
  A.rows = rows;
  A.cols = cols;
  A.nnz = nnz;
  A.rowptr = rowptr;
  A.colidx = colidx;
  A.v16 = v16;
  CKR(launch_spmm(kF32, A, X, ldx, Y, ldy, b, reinterpret_cast<cudaStream_t>(stream)));
  return 0;
}

int64_t phsvds_block_jacobi_nnz(int64_t n, int bs) {
  return (bs < 1 || bs > phsvds::kBjMaxBlock) ? 0 : phsvds::bj_nnz(n, bs);
}

int phsvds_block_jacobi(int64_t n, const int32_t* rowptrT, const int32_t* colidxT, const double* valsT, int bs,
                        int32_t* rowptr, int32_t* colidx, double* v64, float* v32, void* stream) {
  if (n < 1 || bs < 1 || bs > phsvds::kBjMaxBlock || !rowptrT || !rowptr || !colidx || (!v64 && !v32))
    return SVDS_ERR_ARG;
  CKR(phsvds::launch_bj_build(n, bs, rowptrT, colidxT, valsT, rowptr, colidx, v32, v64,
                              reinterpret_cast<cudaStream_t>(stream)));
  return SVDS_OK;
}

size_t phsvds_spmm_dots_scratch_bytes(int nb) { return (size_t)2048 * 4 * (nb > 0 ? nb : 1) * 8; }

int phsvds_spmm_dots(int prec, int64_t n, int64_t nnz, const int32_t* rowptr, const int32_t* colidx,
                     const float* v32, const float* v32lo, const double* v64, int nb, const void* X, int64_t ldx,
                     void* W, const void* E1, const void* E2, double* dots, void* scratch, size_t scratch_bytes,
                     void* stream) {
  if (!prec_ok(prec) || n < 1 || nnz < 0 || !(nb == 1 || nb == 2 || nb == 4 || nb == 8) || !rowptr || !X || !W ||
      !E1 || !E2 || !dots || !scratch || scratch_bytes < phsvds_spmm_dots_scratch_bytes(nb) || ldx < nb)
    return SVDS_ERR_ARG;
  if (nnz > 0 && (!colidx || (prec == kF64 ? !v64 : !v32))) return SVDS_ERR_ARG;
  CsrDev K;
  K.rows = n;
  K.cols = n;
  K.nnz = nnz;
  K.rowptr = rowptr;
  K.colidx = colidx;
  K.v32 = v32;
  K.v32lo = v32lo;
  K.v64 = v64;
  int ready = 0;
  CKR(qmr_op_dots(prec, n, nb, K, X, ldx, W, E1, E2, scratch, dots, nullptr, nullptr, nullptr, &ready,
                  reinterpret_cast<cudaStream_t>(stream)));
  return ready ? SVDS_OK : SVDS_ERR_ARG;
}

int phsvds_ortho(int prec, int64_t L, const void* V, int64_t ldv, int g, void* T, int64_t ldt, int nb, int* status,
                 void* stream) {
  if (!prec_ok(prec) || L < 1 || !V || !T || g < 1 || nb < 1 || nb > 8 || g + nb > 256 || ldv < g || ldt < nb)
    return SVDS_ERR_ARG;
  return ortho_block(prec, L, V, ldv, g, T, ldt, nb, status, reinterpret_cast<cudaStream_t>(stream));
}

int phsvds_ortho_repair(int prec, int64_t L, const void* V, int64_t ldv, int g, void* T, int64_t ldt, int nb,
                        uint64_t seed, int* status, int* replaced, void* stream) {
  if (!prec_ok(prec) || L < 1 || !V || !T || g < 1 || nb < 1 || nb > 8 || g + nb > 256 || ldv < g || ldt < nb)
    return SVDS_ERR_ARG;
  return ortho_block(prec, L, V, ldv, g, T, ldt, nb, status, reinterpret_cast<cudaStream_t>(stream), true, seed,
                     replaced);
}

int phsvds_jd_solve(int prec, int64_t n, int64_t nnz, const int32_t* rowptr, const int32_t* colidx,
                    const float* v32, const float* v32lo, const double* v64, int nb, const void* X, const void* Bv,
                    const double* eta, const void* dinv, int maxit, double xi, void* T, int* steps, void* stream) {
  if (!prec_ok(prec) || n < 1 || nnz < 0 || nb < 1 || nb > 8 || maxit < 0 || !(xi >= 0) || !rowptr || !X || !Bv ||
      !eta || !T)
    return SVDS_ERR_ARG;
  if (nnz > 0 && (!colidx || (prec == kF64 ? !v64 : !v32))) return SVDS_ERR_ARG;
  CsrDev K;
  K.rows = n;
  K.cols = n;
  K.nnz = nnz;
  K.rowptr = rowptr;
  K.colidx = colidx;
  K.v32 = v32;
  K.v32lo = v32lo;
  K.v64 = v64;
  const int rc = jd_solve(prec, K, nb, X, Bv, eta, dinv, maxit, xi, T, steps, reinterpret_cast<cudaStream_t>(stream));
  if (rc == -6) {
    phsvds::set_last_error("phsvds_jd_solve: CUDA error");
    return SVDS_ERR_CUDA;
  }
  return rc == -5 ? SVDS_ERR_NOMEM : rc;
}

int phsvds_to_bf16(int64_t nnz, const float* v32, uint16_t* v16, int* flags, void* stream) {
  if (nnz < 0 || (nnz > 0 && (!v32 || !v16 || !flags))) return SVDS_ERR_ARG;
  CKR(launch_to_bf16(nnz, v32, v16, flags, reinterpret_cast<cudaStream_t>(stream)));
  return 0;
}

size_t phsvds_gram_scratch_bytes(int p, int q) {
  // partial sums of one column chunk, plus a p x 8 staging block when q > 8
  return gram_partial_bytes(gram_default_blocks(), p, std::min(q, 8)) + (q > 8 ? sizeof(double) * p * 8 : 0);
}

int phsvds_gram(int prec, int64_t r0, int64_t r1, const void* P, int64_t ldp, int p, const void* Q, int64_t ldq,
                int q, double* G, void* scratch, size_t scratch_bytes, void* stream) {
  if (!prec_ok(prec) || p < 1 || p > 256 || q < 1 || r0 < 0 || r1 < r0 || !P || !Q || !G || !scratch) return SVDS_ERR_ARG;
  if (ldp < p || ldq < q) return SVDS_ERR_ARG;
  if (scratch_bytes < phsvds_gram_scratch_bytes(p, q)) return SVDS_ERR_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const size_t e = elem_bytes(prec);
  SegV Ps{P, ldp, p};
  // column chunks of Q land in consecutive p x qc row-major blocks of a
  // device staging area; G is then assembled by a strided copy
  for (int c0 = 0; c0 < q; c0 += 8) {
    const int qc = std::min(8, q - c0);
    SegV Qc{reinterpret_cast<const char*>(Q) + c0 * e, ldq, qc};
    int nb = 0;
    CKR(launch_gram(prec, r0, r1, &Ps, 1, Qc, scratch, gram_default_blocks(), &nb, st));
    if (qc == q) {
      CKR(launch_gram_reduce(prec, scratch, nb, p * qc, G, st));
    } else {
      // reduce into the columns [c0, c0 + qc) of G (row-major p x q) via a 2D copy
      double* tmp = reinterpret_cast<double*>(reinterpret_cast<char*>(scratch) +
                                              gram_partial_bytes(gram_default_blocks(), p, 8));
      CKR(launch_gram_reduce(prec, scratch, nb, p * qc, tmp, st));
      CKR(cudaMemcpy2DAsync(G + c0, sizeof(double) * q, tmp, sizeof(double) * qc, sizeof(double) * qc, p,
                            cudaMemcpyDeviceToDevice, st));
    }
  }
  return 0;
}

int phsvds_combine(int prec, int64_t L, const void* P, int64_t ldp, int p, const void* coef, const void* In,
                   int64_t ldin, int alpha_one, void* Out, int64_t ldout, int q, const void* Rinv, void* stream) {
  if (!prec_ok(prec) || L < 0 || p < 1 || q < 1 || !P || !coef || !Out || ldp < p || ldout < q) return SVDS_ERR_ARG;
  if (alpha_one && (!In || ldin < q)) return SVDS_ERR_ARG;
  SegV Ps{P, ldp, p};
  CKR(launch_combine(prec, L, &Ps, 1, coef, In, ldin, alpha_one, Out, ldout, q, Rinv, nullptr, 0,
                     reinterpret_cast<cudaStream_t>(stream)));
  return 0;
}

size_t phsvds_ritz_scratch_bytes(int nb) { return (size_t)152 * 16 * (size_t)nb * 8; }

int phsvds_ritz_residual(int prec, int64_t L, const void* V, const void* W, int64_t ldv, int g, const void* Y,
                         const void* theta, void* X, void* R, int64_t ldb, int nb, double* norms2, void* scratch,
                         size_t scratch_bytes, void* stream) {
  if (!prec_ok(prec) || L < 0 || g < 1 || nb < 1 || !V || !W || !Y || !theta || !X || !R || !norms2 || !scratch)
    return SVDS_ERR_ARG;
  if (ldv < g || ldb < nb || scratch_bytes < phsvds_ritz_scratch_bytes(nb)) return SVDS_ERR_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int nbl = 0;
  CKR(launch_ritz_residual(prec, L, SegV{V, ldv, g}, SegV{W, ldv, g}, g, Y, theta, X, R, ldb, nb, nullptr, nullptr,
                           scratch, 152 * 16, &nbl, st));
  CKR(launch_gram_reduce(prec, scratch, nbl, nb, norms2, st));
  return 0;
}

int phsvds_from_f64(int prec, int64_t L, int nc, const double* src, int64_t lds, void* dst, int64_t ldd, void* stream) {
  if (!prec_ok(prec) || L < 0 || nc < 0 || lds < L || ldd < nc || (L * nc > 0 && (!src || !dst))) return SVDS_ERR_ARG;
  CKR(launch_from_f64_colmajor(prec, L, nc, src, lds, dst, ldd, 1.0, reinterpret_cast<cudaStream_t>(stream)));
  return 0;
}

int phsvds_to_f64(int prec, int64_t L, int nc, const void* src, int64_t lds, double* dst, int64_t ldd, void* stream) {
  if (!prec_ok(prec) || L < 0 || nc < 0 || ldd < L || lds < nc || (L * nc > 0 && (!src || !dst))) return SVDS_ERR_ARG;
  CKR(launch_to_f64_colmajor(prec, L, nc, src, lds, dst, ldd, 1.0, reinterpret_cast<cudaStream_t>(stream)));
  return 0;
}

size_t phsvds_csr_transpose_work_bytes(int64_t cols) { return transpose_work_ints(cols) * sizeof(int); }

int phsvds_csr_transpose(int64_t rows, int64_t cols, int64_t nnz, const int32_t* rowptr, const int32_t* colidx,
                         const double* vals, int32_t* rowptrT, int32_t* colidxT, double* valsT, void* work,
                         size_t work_bytes, void* stream) {
  if (rows < 0 || cols < 0 || nnz < 0 || !rowptr || !rowptrT || !work) return SVDS_ERR_ARG;
  if (nnz > 0 && (!colidx || !vals || !colidxT || !valsT)) return SVDS_ERR_ARG;
  if (work_bytes < phsvds_csr_transpose_work_bytes(cols)) return SVDS_ERR_ARG;
  CKR(launch_csr_transpose(rows, cols, nnz, rowptr, colidx, vals, rowptrT, colidxT, valsT,
                           reinterpret_cast<int*>(work), reinterpret_cast<cudaStream_t>(stream)));
  return 0;
}

int phsvds_csr_values(int64_t nnz, const double* vals, float* v32, float* v32lo, double* v64, int* flags, void* stream) {
  if (nnz < 0 || (nnz > 0 && (!vals || !v32 || !v32lo || !v64 || !flags))) return SVDS_ERR_ARG;
  CKR(launch_csr_values(nnz, vals, 1.0, v32, v32lo, v64, flags, reinterpret_cast<cudaStream_t>(stream)));
  return 0;
}

int phsvds_coef_convert(int prec, const double* src, size_t count, void* dst) {
  if (!prec_ok(prec) || (count > 0 && (!src || !dst))) return SVDS_ERR_ARG;
  host_coef_convert(prec, src, count, dst);
  return 0;
}

int phsvds_host_symeig(int n, const double* A, double* w, double* Z) {
  if (n < 0 || n > 512 || (n > 0 && (!A || !w || !Z))) return SVDS_ERR_ARG;
  return hla::sym_eig(n, A, w, Z) ? 0 : SVDS_ERR_NUMERIC;
}

int phsvds_host_svd(int n, const double* R, double* s, double* Yr) {
  if (n < 0 || n > 512 || (n > 0 && (!R || !s || !Yr))) return SVDS_ERR_ARG;
  return hla::svd_right(n, R, s, Yr) ? 0 : SVDS_ERR_NUMERIC;
}

}  // extern "C"
