// PHSVDS solver engine: the host control loop of Algorithm 1 driving the
// device kernels.  Long vectors never leave the device; per outer iteration
// only the small projections (Gram blocks and residual norms) are copied to
// the host and only small coefficient matrices are copied back (Sec. 3.3: the
// small objects are replicated, the long ones distributed / device-resident).
#include "engine.h"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/phsvds_gnn.h"
#include "gnn.h"
#include "hostla.h"
#include "bjacobi.h"
#include "jdqmr.h"

namespace phsvds {

namespace {

using Clock = std::chrono::steady_clock;

struct CudaFail {
  cudaError_t e;
  const char* where;
};
// a caller-supplied operator returned non-zero
struct OpFail {
  int rc;
};
struct NumFail {
  const char* what;
};
struct BudgetOut {};

#define CK(x)                                   \
  do {                                          \
    cudaError_t _e = (x);                       \
    if (_e != cudaSuccess) throw CudaFail{_e, #x}; \
  } while (0)

enum { OP_C = 0, OP_B = 1 };

// Unit roundoff of each storage/arithmetic mode (double-float: the sloppy
// addition of two double-words keeps about 2^-48 relative accuracy).
double unit_roundoff(int prec) {
  if (prec == kF32) return std::ldexp(1.0, -24);
  if (prec == kDF64) return std::ldexp(1.0, -48);
  return std::ldexp(1.0, -53);
}

// ---------------------------------------------------------------------------
// Per-solve device context
// ---------------------------------------------------------------------------
struct Ctx {
  svds_handle* h = nullptr;
  cudaStream_t st = nullptr;
  const DevMatrix* A = nullptr;
  double* ux = nullptr;  // FP64 staging of a caller-supplied operator's input and output blocks
  double* uy = nullptr;
  void* partial = nullptr;
  int maxblk = 0;
  double* dG = nullptr;
  double* hG = nullptr;
  size_t gcap = 0;  // doubles
  char* hstage = nullptr;
  char* dstage = nullptr;
  int nslots = 0;
  size_t slot_bytes = 0;
  int next_slot = 0;
  std::vector<long long> slot_epoch;
  long long epoch = 1;
  long long mv = 0;
  long long launches = 0;
  long long max_mv = 0;
  double max_sec = 0;
  Clock::time_point t0;
  int print = 0;
  unsigned long long seed = 0, seed_ctr = 0;
  long long restarts = 0, resets = 0;
  // device-side orthogonalisation scratch
  double* dGo = nullptr;   // Gram results of the device CGS2 + CholQR2
  double* dwork = nullptr;
  void* dco[4] = {nullptr, nullptr, nullptr, nullptr};
  int* dstatus = nullptr;  // breakdown flags raised by the device steps
  int* dflag = nullptr;    // result of the learned preconditioner's check
  int* hstatus = nullptr;  // pinned copy
  bool device_ortho = true;
  long long inner = 0;     // JDQMR inner steps
  bool bf16 = false;       // F32-mode operator applications use the bfloat16 values
  // the learned preconditioner was replaced by Jacobi: 1 = M failed its
  // check (a non-finite value or a non-positive diagonal), 2 = stall
  int precond_fallback = 0;
  // CSR of A (which 0), A^T (1) or the explicit C (2) in the value format of prec
  CsrDev op(int prec, int which) const {
    CsrDev m = which == 2 ? A->csrC() : A->csr(which == 1);
    if (bf16 && prec == kF32) m.v16 = which == 2 ? A->v16C : (which == 1 ? A->v16T : A->v16);
    return m;
  }

  double t_sync = 0, t_eig = 0;
  long long nsync = 0;
  void sync() {
    const auto a = Clock::now();
    CK(cudaStreamSynchronize(st));
    t_sync += std::chrono::duration<double>(Clock::now() - a).count();
    ++nsync;
    ++epoch;
  }
  double elapsed() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
  void budget() {
    if (max_mv > 0 && mv >= max_mv) throw BudgetOut{};
    if (max_sec > 0 && elapsed() > max_sec) throw BudgetOut{};
  }
  // Upload a coefficient array (host doubles, the kernel's row-major layout)
  // converted to the mode's coefficient format; stream-ordered.
  const void* upload(int prec, const double* src, size_t count) {
    const size_t bytes = count * coef_bytes(prec);
    if (bytes > slot_bytes) throw NumFail{"coefficient block larger than the staging slot"};
    const int s = next_slot;
    next_slot = (next_slot + 1) % nslots;
    if (slot_epoch[s] == epoch) sync();
    host_coef_convert(prec, src, count, hstage + (size_t)s * slot_bytes);
    CK(cudaMemcpyAsync(dstage + (size_t)s * slot_bytes, hstage + (size_t)s * slot_bytes, bytes,
                       cudaMemcpyHostToDevice, st));
    slot_epoch[s] = epoch;
    return dstage + (size_t)s * slot_bytes;
  }
};

inline char* off(void* p, long long elems, int prec) { return reinterpret_cast<char*>(p) + elems * (long long)elem_bytes(prec); }
inline const char* off(const void* p, long long elems, int prec) {
  return reinterpret_cast<const char*>(p) + elems * (long long)elem_bytes(prec);
}

int spmm_launches(int b) {
  int n = 0;
  while (b > 0) {
    b -= b >= 8 ? 8 : b >= 4 ? 4 : b >= 2 ? 2 : 1;
    ++n;
  }
  return n;
}

// Gram G = [P...]^T Q over rows [r0, r1); result p x q row-major (host).
std::vector<double> gram(Ctx& c, int prec, long long r0, long long r1, const std::vector<SegV>& P, SegV Q) {
  int p = 0;
  for (auto& s : P) p += s.nc;
  const int q = Q.nc;
  if (p > 256 || p < 1 || q < 1) throw NumFail{"gram shape out of range"};
  if ((size_t)p * q > c.gcap) throw NumFail{"gram result larger than the staging buffer"};
  std::vector<double> out((size_t)p * q);
  for (int c0 = 0; c0 < q; c0 += 8) {
    const int qc = std::min(8, q - c0);
    SegV Qc{off(Q.p, c0, prec), Q.ld, qc};
    int nb = 0;
    CK(launch_gram(prec, r0, r1, P.data(), (int)P.size(), Qc, c.partial, c.maxblk, &nb, c.st));
    CK(launch_gram_reduce(prec, c.partial, nb, p * qc, c.dG + (size_t)p * c0, c.st));
    c.launches += 2;
  }
  CK(cudaMemcpyAsync(c.hG, c.dG, sizeof(double) * p * q, cudaMemcpyDeviceToHost, c.st));
  c.sync();
  for (int c0 = 0; c0 < q; c0 += 8) {
    const int qc = std::min(8, q - c0);
    for (int i = 0; i < p; ++i)
      for (int j = 0; j < qc; ++j) out[(size_t)i * q + c0 + j] = c.hG[(size_t)p * c0 + (size_t)i * qc + j];
  }
  return out;
}

// Gram into device memory (no host round trip): dst = [P...]^T Q, p x q row-major, q <= 8.
void gram_dev(Ctx& c, int prec, long long r0, long long r1, const std::vector<SegV>& P, SegV Q, double* dst) {
  int p = 0;
  for (auto& sgm : P) p += sgm.nc;
  if (p > 256 || p < 1 || Q.nc < 1 || Q.nc > 8) throw NumFail{"device gram shape out of range"};
  int nb = 0;
  CK(launch_gram(prec, r0, r1, P.data(), (int)P.size(), Q, c.partial, c.maxblk, &nb, c.st));
  CK(launch_gram_reduce(prec, c.partial, nb, p * Q.nc, dst, c.st));
  c.launches += 2;
}

void combine(Ctx& c, int prec, long long L, const std::vector<SegV>& P, const std::vector<double>& coef_rm,
             const void* In, long long ldin, bool alpha_one, void* Out, long long ldout, int q,
             const std::vector<double>* Rinv_rm = nullptr, void* Out2 = nullptr, long long ldout2 = 0) {
  const void* dcoef = c.upload(prec, coef_rm.data(), coef_rm.size());
  const void* dR = Rinv_rm ? c.upload(prec, Rinv_rm->data(), Rinv_rm->size()) : nullptr;
  CK(launch_combine(prec, L, P.data(), (int)P.size(), dcoef, In, ldin, alpha_one ? 1 : 0, Out, ldout, q, dR, Out2,
                    ldout2, c.st));
  c.launches += 1;
}

// Apply C = A^T A (through tmp, m x nb, ld nb) or B = [0 A^T; A 0].
void apply_op(Ctx& c, int prec, int op, const void* X, long long ldx, void* Y, long long ldy, int nb, void* tmp,
              int tmp_cols) {
  const DevMatrix& A = *c.A;
  if (A.user) {
    // the caller's operator on row-major FP64 blocks (converted from and to
    // the mode's storage unless the mode is native FP64)
    const long long rows = op == OP_C ? A.n : A.n + A.m;
    for (int c0 = 0; c0 < nb; c0 += tmp_cols) {
      const int w = std::min(tmp_cols, nb - c0);
      const void* Xc = off(X, c0, prec);
      void* Yc = off(Y, c0, prec);
      const bool direct = prec == kF64;
      if (!direct) {
        CK(launch_rows_to_f64(prec, rows, w, Xc, ldx, c.ux, w, c.st));
        c.launches += 1;
      }
      const int rc = A.user(op == OP_C ? SVDS_OP_C : SVDS_OP_B, rows, w,
                            direct ? static_cast<const double*>(Xc) : c.ux, direct ? ldx : w,
                            direct ? static_cast<double*>(Yc) : c.uy, direct ? ldy : w, c.st, A.user_ctx);
      if (rc) throw OpFail{rc};
      if (!direct) {
        CK(launch_rows_from_f64(prec, rows, w, c.uy, w, Yc, ldy, c.st));
        c.launches += 1;
      }
      c.mv += 2LL * w;
    }
    return;
  }
  for (int c0 = 0; c0 < nb; c0 += tmp_cols) {
    const int w = std::min(tmp_cols, nb - c0);
    const void* Xc = off(X, c0, prec);
    void* Yc = off(Y, c0, prec);
    if (op == OP_C && A.nnzC > 0) {
      CK(launch_spmm(prec, c.op(prec, 2), Xc, ldx, Yc, ldy, w, c.st));
      c.launches -= spmm_launches(w);
    } else if (op == OP_C) {
      CK(launch_spmm(prec, c.op(prec, 0), Xc, ldx, tmp, w, w, c.st));
      CK(launch_spmm(prec, c.op(prec, 1), tmp, w, Yc, ldy, w, c.st));
    } else {
      CK(launch_spmm(prec, c.op(prec, 1), off(Xc, A.n * ldx, prec), ldx, Yc, ldy, w, c.st));
      CK(launch_spmm(prec, c.op(prec, 0), Xc, ldx, off(Yc, A.n * ldy, prec), ldy, w, c.st));
    }
    c.launches += 2 * spmm_launches(w);
    c.mv += 2LL * w;
  }
}

// Decide (once per handle) whether C = A^T A is applied as an explicit CSR
// matrix, and build it.  Bytes per C apply of a block of b FP32 columns:
// two passes 2 nnz(A) (4 + 4) + 4 (m + n + 2) + 4 b (2 m + 2 n); explicit
// nnz(C) (4 + 4) + 4 (n + 1) + 8 b n.  AUTO takes the explicit form below 0.8
// of the two-pass bytes.
void ensure_normal(svds_handle* h, cudaStream_t st, int mode, int b, long long& launches) {
  DevMatrix& A = h->A;
  if (A.nnzC >= 0) return;
  A.nnzC = 0;
  if (mode == SVDS_NORMAL_TWOPASS || A.n < 1) return;
  const long long n = A.n, m = A.m;
  std::vector<void*> tmp;
  auto take = [&](size_t bytes) -> void* {
    void* p = nullptr;
    if (cudaMalloc(&p, bytes ? bytes : 1) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    tmp.push_back(p);
    return p;
  };
  auto drop = [&]() {
    cudaStreamSynchronize(st);
    for (void* p : tmp) cudaFree(p);
    tmp.clear();
  };
  int* cnt = static_cast<int*>(take(sizeof(int) * (n + 1)));
  int* err = static_cast<int*>(take(sizeof(int) * 4));
  int* work = static_cast<int*>(take(sizeof(int) * scan_work_ints(n)));
  int* rp = static_cast<int*>(take(sizeof(int) * (n + 1)));
  if (!cnt || !err || !work || !rp) {
    drop();
    return;  // not enough memory: the two-pass form needs none
  }
  CK(cudaMemsetAsync(err, 0, sizeof(int) * 4, st));
  CK(launch_normal_count(n, A.rowptrT, A.colidxT, A.rowptr, A.colidx, cnt, err, st));
  CK(launch_exclusive_scan(n, cnt, rp, work, st));
  int herr = 0, hnnz = 0;
  CK(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&hnnz, rp + n, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  launches += 4;
  const double two = 2.0 * A.nnz * 8 + 4.0 * (m + n + 2) + 4.0 * b * (2.0 * m + 2.0 * n);
  const double one = (double)hnnz * 8 + 4.0 * (n + 1) + 8.0 * b * n;
  if (herr || hnnz <= 0 || (mode == SVDS_NORMAL_AUTO && one > 0.8 * two)) {
    drop();
    return;
  }
  int* ci = static_cast<int*>(take(sizeof(int) * hnnz));
  double* cv = static_cast<double*>(take(sizeof(double) * hnnz));
  float* v32 = static_cast<float*>(take(sizeof(float) * hnnz));
  float* v32lo = static_cast<float*>(take(sizeof(float) * hnnz));
  double* v64 = static_cast<double*>(take(sizeof(double) * hnnz));
  if (!ci || !cv || !v32 || !v32lo || !v64) {
    drop();
    return;
  }
  CK(launch_normal_fill(n, A.rowptrT, A.colidxT, A.v64T, A.rowptr, A.colidx, A.v64, 1.0, rp, ci, cv, st));
  CK(cudaMemsetAsync(err, 0, sizeof(int) * 4, st));
  CK(launch_csr_values(hnnz, cv, 1.0, v32, v32lo, v64, err, st));
  CK(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  launches += 2;
  // keep the matrix with the handle, release the temporaries
  for (void* p : {static_cast<void*>(rp), static_cast<void*>(ci), static_cast<void*>(v32), static_cast<void*>(v32lo),
                  static_cast<void*>(v64)}) {
    h->allocs.push_back(p);
    tmp.erase(std::find(tmp.begin(), tmp.end(), p));
  }
  drop();
  A.rowptrC = rp;
  A.colidxC = ci;
  A.v32C = v32;
  A.v32loC = v32lo;
  A.v64C = v64;
  A.exactC = herr == 0;
  A.nnzC = hnnz;
}

// bfloat16 copies of the FP32 values of A, A^T and the explicit C (once per handle).
void ensure_bf16(svds_handle* h, cudaStream_t st, long long& launches) {
  DevMatrix& A = h->A;
  if (A.v16 && (A.nnzC <= 0 || A.v16C)) return;
  auto take = [&](long long count) -> uint16_t* {
    void* p = nullptr;
    if (cudaMalloc(&p, sizeof(uint16_t) * (count > 0 ? count : 1)) != cudaSuccess) {
      cudaGetLastError();
      throw CudaFail{cudaErrorMemoryAllocation, "bfloat16 values"};
    }
    h->allocs.push_back(p);
    return static_cast<uint16_t*>(p);
  };
  int* flags = nullptr;
  if (cudaMalloc(&flags, sizeof(int) * 4) != cudaSuccess) {
    cudaGetLastError();
    throw CudaFail{cudaErrorMemoryAllocation, "bfloat16 flags"};
  }
  CK(cudaMemsetAsync(flags, 0, sizeof(int) * 4, st));
  if (!A.v16) {
    A.v16 = take(A.nnz);
    A.v16T = take(A.nnz);
    CK(launch_to_bf16(A.nnz, A.v32, A.v16, flags, st));
    CK(launch_to_bf16(A.nnz, A.v32T, A.v16T, flags, st));
    launches += 2;
  }
  if (A.nnzC > 0 && !A.v16C) {
    A.v16C = take(A.nnzC);
    CK(launch_to_bf16(A.nnzC, A.v32C, A.v16C, flags, st));
    launches += 1;
  }
  int hf = 0;
  CK(cudaMemcpyAsync(&hf, flags, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  cudaFree(flags);
  A.exact16 = A.exact16 && hf == 0;
}

// small helpers on column-major host matrices
std::vector<double> rowmajor(int rows, int cols, const double* cm, int ld) {
  std::vector<double> r((size_t)rows * cols);
  for (int i = 0; i < rows; ++i)
    for (int j = 0; j < cols; ++j) r[(size_t)i * cols + j] = cm[(size_t)j * ld + i];
  return r;
}

struct OrthoRes {
  std::vector<double> C;  // p x nb row-major: coefficients on the basis
  std::vector<double> R;  // nb x nb row-major upper triangular
  bool replaced = false;
};

// Orthonormalise T (L x nb, ld ldt) against the orthonormal basis segments:
// classical Gram-Schmidt twice, then Cholesky-QR twice (the second CGS Gram is
// fused with the first Cholesky Gram).  T0 = basis * C + T_final * R.
OrthoRes ortho(Ctx& c, int prec, long long L, const std::vector<SegV>& basis, void* T, long long ldt, int nb,
               void* Out2, long long ldo2, int depth = 0) {
  int p = 0;
  for (auto& s : basis) p += s.nc;
  SegV Ts{T, ldt, nb};
  std::vector<SegV> PT = basis;
  PT.push_back(Ts);
  OrthoRes res;
  res.C.assign((size_t)p * nb, 0.0);
  std::vector<double> G = gram(c, prec, 0, L, PT, Ts);  // (p + nb) x nb
  std::vector<double> norms0(nb);
  for (int j = 0; j < nb; ++j) norms0[j] = G[(size_t)(p + j) * nb + j];
  std::vector<double> S((size_t)nb * nb);  // row-major
  std::vector<double> C2((size_t)p * nb, 0.0);
  if (p > 0) {
    std::vector<double> negC((size_t)p * nb);
    for (size_t e = 0; e < negC.size(); ++e) {
      negC[e] = -G[e];
      res.C[e] = G[e];
    }
    combine(c, prec, L, basis, negC, T, ldt, true, T, ldt, nb);
    G = gram(c, prec, 0, L, PT, Ts);
    for (size_t e = 0; e < C2.size(); ++e) C2[e] = G[e];
    for (int i = 0; i < nb; ++i)
      for (int j = 0; j < nb; ++j) {
        double s = G[(size_t)(p + i) * nb + j];
        for (int l = 0; l < p; ++l) s -= C2[(size_t)l * nb + i] * C2[(size_t)l * nb + j];
        S[(size_t)i * nb + j] = s;
      }
    for (size_t e = 0; e < C2.size(); ++e) res.C[e] += C2[e];
  } else {
    for (int i = 0; i < nb; ++i)
      for (int j = 0; j < nb; ++j) S[(size_t)i * nb + j] = G[(size_t)i * nb + j];
  }
  // breakdown: a column that lost (almost) all of its norm is replaced by a
  // random vector and the whole block is orthonormalised again
  std::vector<int> bad;
  for (int j = 0; j < nb; ++j)
    if (!(S[(size_t)j * nb + j] > 1e-20 * std::max(norms0[j], 1e-300))) bad.push_back(j);
  if (bad.empty()) {
    // numerical rank of the block itself: Cholesky of S in column order; a
    // column whose pivot keeps at most tau of its squared norm depends on the
    // earlier columns of the block (a duplicated correction, say) and is
    // replaced in the same way.  A duplicate's pivot is the FP64 rounding of
    // this factorisation (about 1e-16 of the squared norm), not zero; tau
    // stays well below the pivots of merely ill-conditioned blocks, which the
    // shifted Cholesky-QR below handles
    const double tau = 1e-14;
    std::vector<double> Lc((size_t)nb * nb, 0.0);  // lower factor, row-major; skipped columns stay 0
    for (int j = 0; j < nb; ++j) {
      const double sjj = S[(size_t)j * nb + j];
      double d = sjj;
      for (int l = 0; l < j; ++l) d -= Lc[(size_t)j * nb + l] * Lc[(size_t)j * nb + l];
      if (!(d > tau * sjj)) {
        bad.push_back(j);
        continue;
      }
      const double ljj = std::sqrt(d);
      Lc[(size_t)j * nb + j] = ljj;
      for (int i = j + 1; i < nb; ++i) {
        double v = 0.5 * (S[(size_t)i * nb + j] + S[(size_t)j * nb + i]);
        for (int l = 0; l < j; ++l) v -= Lc[(size_t)i * nb + l] * Lc[(size_t)j * nb + l];
        Lc[(size_t)i * nb + j] = v / ljj;
      }
    }
  }
  if (!bad.empty()) {
    if (depth >= 3) throw NumFail{"orthogonalisation breakdown persists"};
    for (int j : bad) {
      CK(launch_fill_normal(prec, L, off(T, j, prec), ldt, 1, c.seed + 0x1000 + (++c.seed_ctr), c.st));
      c.launches += 1;
    }
    OrthoRes r2 = ortho(c, prec, L, basis, T, ldt, nb, Out2, ldo2, depth + 1);
    r2.replaced = true;
    return r2;
  }
  // first Cholesky-QR (shifted if needed, Fukaya et al. 2020)
  std::vector<double> Scm((size_t)nb * nb), R1((size_t)nb * nb), R1i((size_t)nb * nb);
  for (int i = 0; i < nb; ++i)
    for (int j = 0; j < nb; ++j) Scm[(size_t)j * nb + i] = S[(size_t)i * nb + j];
  bool extra = false;
  if (!hla::chol_upper(nb, Scm.data(), R1.data())) {
    double tr = 0;
    for (int j = 0; j < nb; ++j) tr += std::fabs(Scm[(size_t)j * nb + j]);
    const double shift = 11.0 * ((double)L * nb + (double)nb * (nb + 1)) * unit_roundoff(prec) * tr;
    for (int j = 0; j < nb; ++j) Scm[(size_t)j * nb + j] += shift;
    if (!hla::chol_upper(nb, Scm.data(), R1.data())) throw NumFail{"shifted Cholesky-QR failed"};
    extra = true;
  }
  hla::tri_inv_upper(nb, R1.data(), R1i.data());
  std::vector<double> R1i_rm = rowmajor(nb, nb, R1i.data(), nb);
  if (p > 0) {
    std::vector<double> negC2((size_t)p * nb);
    for (size_t e = 0; e < C2.size(); ++e) negC2[e] = -C2[e];
    combine(c, prec, L, basis, negC2, T, ldt, true, T, ldt, nb, &R1i_rm);
  } else {
    combine(c, prec, L, {Ts}, R1i_rm, nullptr, 0, false, T, ldt, nb);
  }
  std::vector<double> Rtot = R1;  // column-major
  const int passes = extra ? 2 : 1;
  for (int pass = 0; pass < passes; ++pass) {
    std::vector<double> G3 = gram(c, prec, 0, L, {Ts}, Ts);
    std::vector<double> G3cm((size_t)nb * nb), R2((size_t)nb * nb), R2i((size_t)nb * nb);
    for (int i = 0; i < nb; ++i)
      for (int j = 0; j < nb; ++j) G3cm[(size_t)j * nb + i] = G3[(size_t)i * nb + j];
    if (!hla::chol_upper(nb, G3cm.data(), R2.data())) throw NumFail{"second Cholesky-QR failed"};
    hla::tri_inv_upper(nb, R2.data(), R2i.data());
    const bool last = pass + 1 == passes;
    combine(c, prec, L, {Ts}, rowmajor(nb, nb, R2i.data(), nb), nullptr, 0, false, T, ldt, nb, nullptr,
            last ? Out2 : nullptr, ldo2);
    std::vector<double> Rn((size_t)nb * nb, 0.0);
    hla::gemm_nn(nb, nb, nb, R2.data(), nb, Rtot.data(), nb, Rn.data(), nb);
    Rtot = Rn;
  }
  res.R = rowmajor(nb, nb, Rtot.data(), nb);
  return res;
}

// Device-side CGS2 + CholQR2 of T (L x nb, nb <= 8) against one orthonormal
// basis segment: the same passes as ortho(), with the small dense steps
// (negated coefficients, Cholesky factors and their inverses) computed by a
// one-CTA kernel, so no host round trip is needed.  A breakdown (a column that
// lost almost all of its norm, or a Gram that is not positive definite) sets
// c.dstatus; the caller checks it at its next synchronisation and redoes the
// step with ortho().  The result is written to T and to Out2.
void ortho_dev(Ctx& c, int prec, long long L, SegV basis, void* T, long long ldt, int nb, void* Out2, long long ldo2) {
  const int g = basis.nc;
  SegV Ts{T, ldt, nb};
  const std::vector<SegV> PT = {basis, Ts};
  gram_dev(c, prec, 0, L, PT, Ts, c.dGo);
  CK(launch_ortho_small(1, prec, g, nb, c.dGo, c.dwork, c.dco[0], nullptr, c.dstatus, 0.0, c.st));
  CK(launch_combine(prec, L, &basis, 1, c.dco[0], T, ldt, 1, T, ldt, nb, nullptr, nullptr, 0, c.st));
  gram_dev(c, prec, 0, L, PT, Ts, c.dGo);
  CK(launch_ortho_small(2, prec, g, nb, c.dGo, c.dwork, c.dco[1], c.dco[2], c.dstatus, 1e-20, c.st));
  CK(launch_combine(prec, L, &basis, 1, c.dco[1], T, ldt, 1, T, ldt, nb, c.dco[2], nullptr, 0, c.st));
  gram_dev(c, prec, 0, L, {Ts}, Ts, c.dGo);
  CK(launch_ortho_small(3, prec, 0, nb, c.dGo, c.dwork, c.dco[3], nullptr, c.dstatus, 0.0, c.st));
  CK(launch_combine(prec, L, &Ts, 1, c.dco[3], nullptr, 0, 0, T, ldt, nb, nullptr, Out2, ldo2, c.st));
  c.launches += 6;
}

// Copy the device status word to the host with the next synchronisation and
// clear it; returns the flags.
int take_status(Ctx& c) {
  CK(cudaMemcpyAsync(c.hstatus, c.dstatus, sizeof(int), cudaMemcpyDeviceToHost, c.st));
  c.sync();
  const int v = *c.hstatus;
  if (v) CK(cudaMemsetAsync(c.dstatus, 0, sizeof(int), c.st));
  return v;
}

// ---------------------------------------------------------------------------
// Buffers of one eigensolver run
// ---------------------------------------------------------------------------
struct RunBufs {
  int prec = kDF64;
  long long L = 0;
  long long ldv = 0;
  int b = 1;
  void* V = nullptr;
  void* W = nullptr;
  void* Q = nullptr;      // refined extraction only
  void* Xb = nullptr;     // L x b
  void* Rb = nullptr;     // L x b
  void* Tb = nullptr;     // L x b
  void* Zb = nullptr;     // L x b (refined)
  void* BXb = nullptr;    // L x b (stage-2 checks)
  void* tmp = nullptr;    // m x b (C op)
  void* Xlock = nullptr;  // L x k (refined)
  // JDQMR inner-solve scratch (L x b each, inner mode): x, rhs, K^-1 x, q, r, d, sol, op(q)
  void* jd[8] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  void* jtmp = nullptr;  // m x b (inner-mode C op)
  void* ju = nullptr;    // L x b (inner-mode K^-1 r for a sparse preconditioner)
  unsigned* jtick = nullptr;  // tickets of the fused reduction tails (zeroed per correction)
  QmrState* jS = nullptr;
  double* jdots = nullptr;
};

using ConvFn = std::function<void(const double* theta, const double* rn, int off, int nc, char* ok)>;

struct RunCfg {
  int op = OP_C;
  int k = 1, b = 1, mb = 15, mr = 6;
  bool smallest = true;
  double normop = 0, u = 0;
  const void* dscale = nullptr;
  const void* V0 = nullptr;
  long long ldv0 = 0;
  int b0 = 1;
  ConvFn conv;
  const char* name = "";
  // JDQMR corrections instead of the preconditioned residual
  bool jd = false;
  int jd_prec = kF32;            // mode of the inner solves
  const void* jdinv = nullptr;   // Jacobi diagonal in the inner mode's storage, or nullptr
  const CsrDev* K = nullptr;     // sparse preconditioner (learned M) in the outer mode, or nullptr
  const CsrDev* jdK = nullptr;   // the same in the inner mode
  int jd_maxk = 30;
  double jd_xi = 0.1;
  // DYNAMIC: choose between the two corrections per outer iteration
  bool dyn = false;
  // fallback of a learned preconditioner (K / jdK) to Jacobi: after stall_its
  // outer iterations in which the smallest residual of the corrected block
  // did not fall below 0.99 of its best since the last newly converged pair
  // (0 = never), K and jdK are dropped for the Jacobi scalings below
  int stall_its = 0;
  const void* fb_dscale = nullptr;  // Jacobi diagonal in the outer mode's storage
  const void* fb_jdinv = nullptr;   // the same in the inner mode's storage
};

struct RunOut {
  std::vector<double> theta;
  long long outer = 0;
  long long outer_jd = 0;  // outer iterations whose correction came from JDQMR
};

// DYNAMIC method of stage 1 (Sec. 3.4: switch between GD+k and JDQMR so as to
// minimise time).  The paper gives no rule; this one measures.  Progress of
// an outer iteration is the decrease of log ||r|| summed over the Ritz
// indices whose residual was computed both at that iteration and at the one
// before, and it is charged, with the wall time between the two, to the
// method that made the correction in between.  Schedule: a JDQMR trial of 2
// outer iterations, a GD+k trial of at least 3 iterations and at least the
// JDQMR trial's time, then the method with the higher rate for 4 times the
// trials' time, a re-trial of the other method (its minimum iterations and its
// last trial time), the better one again for a window twice as long, and so
// on.  Every iteration stays a valid GD+k iteration, so the choice only
// affects time, never the returned triplets.
struct DynState {
  int cur = 1;    // method of the next correction: 0 GD+k, 1 JDQMR
  int stage = 0;  // 0 JDQMR trial, 1 GD+k trial, 2 exploit, 3 re-trial
  int its = 0;
  double t_win = 0, prog_win = 0;
  double rate[2] = {0, 0}, trial_t[2] = {0, 0};
  double exploit_len = 0;
  double t_last = -1;
  std::vector<std::pair<int, double>> last;
  // the window closed by the last choose(), for the iteration log
  bool closed = false;
  int closed_m = 0, closed_its = 0;
  double closed_t = 0;

  void drop() {
    t_last = -1;
    last.clear();
  }
  void observe(double now, const std::vector<std::pair<int, double>>& res) {
    if (t_last >= 0) {
      double prog = 0;
      for (const auto& a : res)
        for (const auto& b : last)
          if (a.first == b.first && a.second > 0 && b.second > 0) prog += std::log(b.second / a.second);
      t_win += now - t_last;
      prog_win += prog;
      ++its;
    }
    last = res;
    t_last = now;
  }
  static int min_its(int m) { return m == 1 ? 2 : 3; }
  int best() const { return rate[0] > rate[1] ? 0 : 1; }
  void close(int next) {
    closed = true;
    closed_m = cur;
    closed_its = its;
    closed_t = t_win;
    rate[cur] = t_win > 0 ? prog_win / t_win : 0.0;
    cur = next;
    its = 0;
    t_win = prog_win = 0;
  }
  int choose() {
    closed = false;
    switch (stage) {
      case 0:
        if (its >= 2) {
          trial_t[1] = t_win;
          close(0);
          stage = 1;
        }
        break;
      case 1:
        if ((its >= 3 && t_win >= trial_t[1]) || its >= 200) {
          trial_t[0] = t_win;
          exploit_len = 4.0 * (trial_t[0] + trial_t[1]);
          close(0);
          cur = best();
          stage = 2;
        }
        break;
      case 2:
        if (t_win >= exploit_len && its >= min_its(cur)) {
          close(1 - cur);
          stage = 3;
        }
        break;
      default:
        if (its >= min_its(cur) && t_win >= trial_t[cur]) {
          trial_t[cur] = t_win;
          close(cur);
          cur = best();
          exploit_len *= 2.0;
          stage = 2;
        }
    }
    return cur;
  }
};

void put_block_rm(std::vector<double>& dst, int g, const double* Ycm, int ldy, const std::vector<int>& cols) {
  const int q = (int)cols.size();
  dst.assign((size_t)g * q, 0.0);
  for (int i = 0; i < g; ++i)
    for (int j = 0; j < q; ++j) dst[(size_t)i * q + j] = Ycm[(size_t)cols[j] * ldy + i];
}

// Ritz vectors / residuals / norms for the coefficient block Ysel (g x nt,
// row-major) into columns [o, o + nt) of Xb and Rb.
std::vector<double> ritz_block(Ctx& c, RunBufs& B, int g, const std::vector<double>& Ysel,
                               const std::vector<double>& th, int o, const void* dscale = nullptr);

// Ritz vectors / residuals / norms for the coefficient columns `cols` of Y
// (column-major g x g) into columns [o, o + |cols|) of Xb and Rb.
std::vector<double> ritz_cols(Ctx& c, RunBufs& B, int g, const std::vector<double>& Ycm,
                              const std::vector<double>& theta, const std::vector<int>& cols, int o,
                              const void* dscale = nullptr) {
  const int nt = (int)cols.size();
  std::vector<double> Ysel;
  put_block_rm(Ysel, g, Ycm.data(), g, cols);
  std::vector<double> th(nt);
  for (int j = 0; j < nt; ++j) th[j] = theta[cols[j]];
  return ritz_block(c, B, g, Ysel, th, o, dscale);
}

std::vector<double> ritz_block(Ctx& c, RunBufs& B, int g, const std::vector<double>& Ysel,
                               const std::vector<double>& th, int o, const void* dscale) {
  const int prec = B.prec;
  const int nt = (int)th.size();
  const void* dY = c.upload(prec, Ysel.data(), Ysel.size());
  const void* dT = c.upload(prec, th.data(), th.size());
  int nbl = 0;
  CK(launch_ritz_residual(prec, B.L, SegV{B.V, B.ldv, g}, SegV{B.W, B.ldv, g}, g, dY, dT, off(B.Xb, o, prec),
                          off(B.Rb, o, prec), B.b, nt, dscale, dscale ? off(B.Tb, o, prec) : nullptr, c.partial,
                          c.maxblk, &nbl, c.st));
  CK(launch_gram_reduce(prec, c.partial, nbl, nt, c.dG, c.st));
  c.launches += 2;
  CK(cudaMemcpyAsync(c.hG, c.dG, sizeof(double) * nt, cudaMemcpyDeviceToHost, c.st));
  c.sync();
  std::vector<double> rn(nt);
  for (int j = 0; j < nt; ++j) rn[j] = std::sqrt(std::max(c.hG[j], 0.0));
  return rn;
}

void init_basis(Ctx& c, RunBufs& B, const RunCfg& cfg, int op, int& g, std::vector<double>& H,
                const std::vector<SegV>& against) {
  const int prec = B.prec;
  CK(launch_copy_cols(prec, B.L, cfg.V0, cfg.ldv0, B.V, B.ldv, cfg.b0, c.st));
  c.launches += 1;
  ortho(c, prec, B.L, against, B.V, B.ldv, cfg.b0, nullptr, 0);
  apply_op(c, prec, op, B.V, B.ldv, B.W, B.ldv, cfg.b0, B.tmp, B.b);
  g = cfg.b0;
  std::vector<double> Hr = gram(c, prec, 0, B.L, {SegV{B.V, B.ldv, g}}, SegV{B.W, B.ldv, g});
  H.assign((size_t)g * g, 0.0);
  for (int i = 0; i < g; ++i)
    for (int j = 0; j < g; ++j) H[(size_t)j * g + i] = 0.5 * (Hr[(size_t)i * g + j] + Hr[(size_t)j * g + i]);
}

void extend_H(std::vector<double>& H, int g, int nbk, const std::vector<double>& Hext /*(g+nbk) x nbk rm*/) {
  const int gn = g + nbk;
  std::vector<double> Hn((size_t)gn * gn, 0.0);
  for (int j = 0; j < g; ++j)
    for (int i = 0; i < g; ++i) Hn[(size_t)j * gn + i] = H[(size_t)j * g + i];
  for (int i = 0; i < g; ++i)
    for (int j = 0; j < nbk; ++j) {
      const double v = Hext[(size_t)i * nbk + j];
      Hn[(size_t)(g + j) * gn + i] = v;
      Hn[(size_t)i * gn + (g + j)] = v;
    }
  for (int i = 0; i < nbk; ++i)
    for (int j = 0; j < nbk; ++j)
      Hn[(size_t)(g + j) * gn + (g + i)] =
          0.5 * (Hext[(size_t)(g + i) * nbk + j] + Hext[(size_t)(g + j) * nbk + i]);
  H.swap(Hn);
}

// Z^T H Z for column-major H (g x g) and Z (g x gz).
std::vector<double> project_H(const std::vector<double>& H, int g, const std::vector<double>& Z, int gz) {
  std::vector<double> HZ((size_t)g * gz), Hn((size_t)gz * gz);
  hla::gemm_nn(g, gz, g, H.data(), g, Z.data(), g, HZ.data(), g);
  hla::gemm_tn(gz, gz, g, Z.data(), g, HZ.data(), g, Hn.data(), gz);
  for (int i = 0; i < gz; ++i)
    for (int j = i + 1; j < gz; ++j) {
      const double v = 0.5 * (Hn[(size_t)j * gz + i] + Hn[(size_t)i * gz + j]);
      Hn[(size_t)j * gz + i] = v;
      Hn[(size_t)i * gz + j] = v;
    }
  return Hn;
}

void reset_basis(Ctx& c, RunBufs& B, int op, int g, std::vector<double>& H, const std::vector<SegV>& against) {
  const int prec = B.prec;
  ortho(c, prec, B.L, against, B.V, B.ldv, g, nullptr, 0);
  apply_op(c, prec, op, B.V, B.ldv, B.W, B.ldv, g, B.tmp, B.b);
  std::vector<double> Hr = gram(c, prec, 0, B.L, {SegV{B.V, B.ldv, g}}, SegV{B.W, B.ldv, g});
  H.assign((size_t)g * g, 0.0);
  for (int i = 0; i < g; ++i)
    for (int j = 0; j < g; ++j) H[(size_t)j * g + i] = 0.5 * (Hr[(size_t)i * g + j] + Hr[(size_t)j * g + i]);
  c.resets += 1;
}

// ---------------------------------------------------------------------------
// JDQMR correction for the nbk block columns of (Xb, Rb): approximate solution
// of (I - x x^T)(op - eta I)(I - x x^T) t = -r (t orthogonal to x) by block
// symmetric QMR in FP32, with right-hand sides scaled to unit norm (the outer
// basis is orthonormalised afterwards, so the scale of t is immaterial).
// Result in B.Tb in the outer precision.
// ---------------------------------------------------------------------------
void jd_correction(Ctx& c, RunBufs& B, const RunCfg& cfg, int nbk, const std::vector<double>& eta,
                   const std::vector<double>& rn) {
  const int prec = B.prec, pin = cfg.jd_prec;
  const long long L = B.L;
  std::vector<double> one(nbk, 1.0), scr(nbk);
  for (int j = 0; j < nbk; ++j) scr[j] = rn[j] > 0 ? -1.0 / rn[j] : 0.0;
  const double* d1 = reinterpret_cast<const double*>(c.upload(kF64, one.data(), nbk));
  const double* d2 = reinterpret_cast<const double*>(c.upload(kF64, scr.data(), nbk));
  const double* de = reinterpret_cast<const double*>(c.upload(kF64, eta.data(), nbk));
  void *x = B.jd[0], *bv = B.jd[1], *kx = B.jd[2], *q = B.jd[3], *r = B.jd[4], *d = B.jd[5], *sol = B.jd[6],
       *w = B.jd[7];
  CK(convert_cols(prec, B.Xb, B.b, pin, x, nbk, L, nbk, d1, c.st));
  CK(convert_cols(prec, B.Rb, B.b, pin, bv, nbk, L, nbk, d2, c.st));
  CK(cudaMemsetAsync(B.jtick, 0, 64, c.st));
  CK(qmr_init(pin, L, nbk, x, bv, cfg.jdinv, cfg.jdK, B.ju, kx, q, r, d, sol, B.jS, c.partial, B.jdots, c.st));
  c.launches += 2 + qmr_init_launches(nbk, cfg.jdK != nullptr);
  const DevMatrix& Am = *c.A;
  for (int k = 0; k < cfg.jd_maxk; ++k) {
    // w = op(q), fused with the step's first dot products when op is C
    int ready = 0;
    if (cfg.op == OP_C && !Am.user) {
      if (Am.nnzC > 0) {
        CK(qmr_op_dots(pin, L, nbk, c.op(pin, 2), q, nbk, w, x, q, c.partial, B.jdots, B.jtick, de, B.jS, &ready,
                       c.st));
      } else {
        CK(launch_spmm(pin, c.op(pin, 0), q, nbk, B.jtmp, nbk, nbk, c.st));
        CK(qmr_op_dots(pin, L, nbk, c.op(pin, 1), B.jtmp, nbk, w, x, q, c.partial, B.jdots, B.jtick, de, B.jS,
                       &ready, c.st));
        if (ready) {
          c.launches += spmm_launches(nbk);
        } else {
          CK(launch_spmm(pin, c.op(pin, 1), B.jtmp, nbk, w, nbk, nbk, c.st));
          c.launches += 2 * spmm_launches(nbk);
        }
        c.mv += 2LL * nbk;
      }
      if (ready) {
        c.launches += ready == 2 ? 1 : 2;
        if (Am.nnzC > 0) c.mv += 2LL * nbk;
      }
    }
    if (!ready && (Am.user || !(cfg.op == OP_C && Am.nnzC <= 0)))
      apply_op(c, pin, cfg.op, q, nbk, w, nbk, nbk, B.jtmp, nbk);
    CK(qmr_step(pin, L, nbk, x, w, ready, B.jtick, kx, cfg.jdinv, cfg.jdK, B.ju, de, cfg.jd_xi, cfg.jd_maxk, q, r, d,
                sol, B.jS, c.partial, B.jdots, c.st));
    c.launches += qmr_step_launches(nbk, cfg.jdK != nullptr, ready, (nbk & (nbk - 1)) == 0);
    c.inner += 1;
    if ((k + 1) % 8 == 0 && k + 1 < cfg.jd_maxk) {
      CK(cudaMemcpyAsync(c.hG, B.jS, sizeof(QmrState) * nbk, cudaMemcpyDeviceToHost, c.st));
      c.sync();
      const QmrState* hs = reinterpret_cast<const QmrState*>(c.hG);
      bool any = false;
      for (int j = 0; j < nbk; ++j) any = any || hs[j].active;
      if (!any) break;
    }
  }
  CK(convert_cols(pin, sol, nbk, prec, B.Tb, B.b, L, nbk, d1, c.st));
  c.launches += 1;
}

// ---------------------------------------------------------------------------
// GD+k with Rayleigh-Ritz and soft locking (stage 1 on C; stage 2 largest on B)
// ---------------------------------------------------------------------------
RunOut run_gdk_rr(Ctx& c, RunBufs& B, const RunCfg& cfg0, void* Xout, long long ldx) {
  RunCfg cfg = cfg0;  // the preconditioner may fall back to Jacobi during the run
  const int prec = B.prec;
  const int k = cfg.k, b = cfg.b;
  RunOut out;
  int g = 0;
  std::vector<double> H;
  init_basis(c, B, cfg, cfg.op, g, H, {});
  std::vector<char> flags(k, 0);
  std::vector<double> Yprev;  // g x nprev column-major
  int nprev = 0;
  int rsr = 0;
  std::vector<double> w, Z;
  DynState dyn;
  std::vector<std::pair<int, double>> tested;  // (Ritz index, residual) of this iteration
  // stall detector of a learned preconditioner
  double stall_best = 1e300;
  int stall_since = 0, stall_nconv = -1;
  while (true) {
    c.budget();
    ++out.outer;
    w.assign(g, 0.0);
    Z.assign((size_t)g * g, 0.0);
    {
      const auto a = Clock::now();
      if (!hla::sym_eig(g, H.data(), w.data(), Z.data())) throw NumFail{"projected eigenproblem did not converge"};
      c.t_eig += std::chrono::duration<double>(Clock::now() - a).count();
    }
    std::vector<double> theta(g), Y((size_t)g * g);
    for (int j = 0; j < g; ++j) {
      const int src = cfg.smallest ? j : g - 1 - j;
      theta[j] = w[src];
      std::memcpy(&Y[(size_t)j * g], &Z[(size_t)src * g], sizeof(double) * g);
    }
    const int ncand = std::min(k, g);
    std::vector<int> block;
    std::vector<double> rnb;
    std::vector<int> cand;
    for (int j = 0; j < ncand; ++j)
      if (!flags[j]) cand.push_back(j);
    size_t ci = 0;
    int nbk = 0;
    tested.clear();
    auto test_and_compact = [&](const std::vector<int>& take, const std::vector<double>& rn) {
      std::vector<double> th(take.size());
      for (size_t t = 0; t < take.size(); ++t) th[t] = theta[take[t]];
      std::vector<char> ok(take.size(), 0);
      cfg.conv(th.data(), rn.data(), nbk, (int)take.size(), ok.data());
      int wpos = nbk;
      for (size_t t = 0; t < take.size(); ++t) {
        if (ok[t]) {
          flags[take[t]] = 1;
          continue;
        }
        const int src = nbk + (int)t;
        if (src != wpos) {
          CK(launch_copy_cols(prec, B.L, off(B.Xb, src, prec), b, off(B.Xb, wpos, prec), b, 1, c.st));
          CK(launch_copy_cols(prec, B.L, off(B.Rb, src, prec), b, off(B.Rb, wpos, prec), b, 1, c.st));
          c.launches += 2;
        }
        block.push_back(take[t]);
        rnb.push_back(rn[t]);
        ++wpos;
      }
      nbk = wpos;
    };
    while (ci < cand.size() && nbk < b) {
      std::vector<int> take;
      while (ci < cand.size() && (int)take.size() < b - nbk) take.push_back(cand[ci++]);
      std::vector<double> rn = ritz_cols(c, B, g, Y, theta, take, nbk);
      for (size_t t = 0; t < take.size(); ++t) tested.emplace_back(take[t], rn[t]);
      test_and_compact(take, rn);
    }
    bool allflag = ncand == k;
    for (int j = 0; j < k && allflag; ++j) allflag = flags[j] != 0;
    if (allflag) {
      // verification of all k flagged pairs together
      std::vector<int> fails;
      for (int c0 = 0; c0 < k; c0 += b) {
        std::vector<int> chunk;
        for (int j = c0; j < std::min(k, c0 + b); ++j) chunk.push_back(j);
        std::vector<double> rn = ritz_cols(c, B, g, Y, theta, chunk, 0);
        std::vector<double> th(chunk.size());
        for (size_t t = 0; t < chunk.size(); ++t) th[t] = theta[chunk[t]];
        std::vector<char> ok(chunk.size(), 0);
        cfg.conv(th.data(), rn.data(), 0, (int)chunk.size(), ok.data());
        for (size_t t = 0; t < chunk.size(); ++t)
          if (!ok[t]) fails.push_back(chunk[t]);
      }
      if (fails.empty()) {
        std::vector<int> all(k);
        for (int j = 0; j < k; ++j) all[j] = j;
        std::vector<double> Yk;
        put_block_rm(Yk, g, Y.data(), g, all);
        combine(c, prec, B.L, {SegV{B.V, B.ldv, g}}, Yk, nullptr, 0, false, Xout, ldx, k);
        out.theta.assign(theta.begin(), theta.begin() + k);
        return out;
      }
      for (int j = 0; j < k; ++j) flags[j] = 1;
      for (int j : fails) flags[j] = 0;
      block.clear();
      rnb.clear();
      std::vector<int> take(fails.begin(), fails.begin() + std::min((int)fails.size(), b));
      rnb = ritz_cols(c, B, g, Y, theta, take, 0);
      block = take;
      nbk = (int)take.size();
    }
    if (nbk == 0) {
      std::vector<int> take;
      for (int j = 0; j < std::min(b, ncand); ++j) take.push_back(j);
      rnb = ritz_cols(c, B, g, Y, theta, take, 0);
      block = take;
      nbk = (int)take.size();
    }
    if (c.print >= 3) {
      double mn = 1e300;
      for (double r : rnb) mn = std::min(mn, r);
      int nf = 0;
      for (char f : flags) nf += f;
      std::fprintf(stderr, "[%s] it %lld g %d conv %d/%d theta0 %.10e minres %.3e mv %lld\n", cfg.name, out.outer, g,
                   nf, k, theta[0], mn, c.mv);
    }
    if (cfg.stall_its > 0 && (cfg.K || cfg.jdK)) {
      int nf = 0;
      for (char f : flags) nf += f;
      double rmin = 1e300;
      for (double r : rnb) rmin = std::min(rmin, r);
      if (nf > stall_nconv) {
        stall_nconv = nf;
        stall_best = rmin;
        stall_since = 0;
      } else if (rmin < 0.99 * stall_best) {
        stall_best = rmin;
        stall_since = 0;
      } else if (++stall_since >= cfg.stall_its) {
        cfg.K = nullptr;
        cfg.jdK = nullptr;
        cfg.dscale = cfg.fb_dscale;
        cfg.jdinv = cfg.fb_jdinv;
        c.precond_fallback = 2;
        if (c.print >= 1)
          std::fprintf(stderr, "[%s] learned preconditioner stalled for %d outer iterations: Jacobi from here on\n",
                       cfg.name, cfg.stall_its);
      }
    }
    bool use_jd = cfg.jd;
    if (cfg.dyn) {
      dyn.observe(c.elapsed(), tested);
      use_jd = dyn.choose() == 1;
      if (dyn.closed && c.print >= 2)
        std::fprintf(stderr, "[%s] dynamic: %s window of %d its, %.4f s; rates GD+k %.4g, JDQMR %.4g /s -> %s\n",
                     cfg.name, dyn.closed_m ? "JDQMR" : "GD+k", dyn.closed_its, dyn.closed_t, dyn.rate[0],
                     dyn.rate[1], use_jd ? "JDQMR" : "GD+k");
    }
    // reset of V and W (Sec. 3.2)
    double rmin = 1e300;
    for (double r : rnb) rmin = std::min(rmin, r);
    if (rsr > 0 && cfg.u > 0 && rmin < std::sqrt((double)rsr) * cfg.normop * cfg.u) {
      reset_basis(c, B, cfg.op, g, H, {});
      rsr = 0;
      nprev = 0;
      Yprev.clear();
      dyn.drop();
      continue;
    }
    // correction: JDQMR, or T = M R (learned sparse M, or Jacobi), or T = R
    void* T = B.Rb;
    if (use_jd) {
      ++out.outer_jd;
      std::vector<double> eta(nbk);
      for (int j = 0; j < nbk; ++j) eta[j] = theta[block[j]];
      jd_correction(c, B, cfg, nbk, eta, rnb);
      T = B.Tb;
    } else if (cfg.K) {
      CK(launch_spmm(prec, *cfg.K, B.Rb, b, B.Tb, b, nbk, c.st));
      c.launches += spmm_launches(nbk);
      T = B.Tb;
    } else if (cfg.dscale) {
      CK(launch_scale_rows(prec, B.L, cfg.dscale, B.Rb, b, B.Tb, b, nbk, c.st));
      c.launches += 1;
      T = B.Tb;
    }
    std::vector<double> Ycur((size_t)g * nbk);
    for (int j = 0; j < nbk; ++j) std::memcpy(&Ycur[(size_t)j * g], &Y[(size_t)block[j] * g], sizeof(double) * g);
    if (g + nbk > cfg.mb) {
      // GD+k restart: the min_restart Ritz vectors plus the previous block's
      const int mr = std::min(cfg.mr, g);
      std::vector<double> cols((size_t)g * (mr + nprev));
      std::memcpy(cols.data(), Y.data(), sizeof(double) * g * mr);
      if (nprev) std::memcpy(&cols[(size_t)g * mr], Yprev.data(), sizeof(double) * g * nprev);
      const int gz = hla::orth_cols(g, mr + nprev, cols.data(), 1e-12);
      std::vector<double> Zr = rowmajor(g, gz, cols.data(), g);
      combine(c, prec, B.L, {SegV{B.V, B.ldv, g}}, Zr, nullptr, 0, false, B.V, B.ldv, gz);
      combine(c, prec, B.L, {SegV{B.W, B.ldv, g}}, Zr, nullptr, 0, false, B.W, B.ldv, gz);
      H = project_H(H, g, cols, gz);
      std::vector<double> Yn((size_t)gz * nbk);
      hla::gemm_tn(gz, nbk, g, cols.data(), g, Ycur.data(), g, Yn.data(), gz);
      Ycur.swap(Yn);
      g = gz;
      ++rsr;
      c.restarts += 1;
    }
    std::vector<double> Hext;
    if (c.device_ortho && nbk <= 8 && g + nbk <= 256) {
      ortho_dev(c, prec, B.L, SegV{B.V, B.ldv, g}, T, b, nbk, off(B.V, g, prec), B.ldv);
      apply_op(c, prec, cfg.op, T, b, off(B.W, g, prec), B.ldv, nbk, B.tmp, b);
      gram_dev(c, prec, 0, B.L, {SegV{B.V, B.ldv, g + nbk}}, SegV{off(B.W, g, prec), B.ldv, nbk}, c.dG);
      CK(cudaMemcpyAsync(c.hG, c.dG, sizeof(double) * (g + nbk) * nbk, cudaMemcpyDeviceToHost, c.st));
      if (take_status(c) == 0) {
        Hext.assign(c.hG, c.hG + (size_t)(g + nbk) * nbk);
      } else {
        // breakdown in the device orthogonalisation: rebuild the block and
        // redo the step with the host-driven path (random replacements)
        std::vector<double> Yb = rowmajor(g, nbk, Ycur.data(), g), thb(nbk);
        for (int j = 0; j < nbk; ++j) thb[j] = theta[block[j]];
        ritz_block(c, B, g, Yb, thb, 0);
        T = B.Rb;
        if (cfg.K) {
          CK(launch_spmm(prec, *cfg.K, B.Rb, b, B.Tb, b, nbk, c.st));
          T = B.Tb;
        } else if (cfg.dscale) {
          CK(launch_scale_rows(prec, B.L, cfg.dscale, B.Rb, b, B.Tb, b, nbk, c.st));
          T = B.Tb;
        }
      }
    }
    if (Hext.empty()) {
      ortho(c, prec, B.L, {SegV{B.V, B.ldv, g}}, T, b, nbk, off(B.V, g, prec), B.ldv);
      apply_op(c, prec, cfg.op, T, b, off(B.W, g, prec), B.ldv, nbk, B.tmp, b);
      Hext = gram(c, prec, 0, B.L, {SegV{B.V, B.ldv, g + nbk}}, SegV{off(B.W, g, prec), B.ldv, nbk});
    }
    extend_H(H, g, nbk, Hext);
    // previous-iteration coefficients padded with zeros for the new columns
    nprev = nbk;
    Yprev.assign((size_t)(g + nbk) * nbk, 0.0);
    for (int j = 0; j < nbk; ++j) std::memcpy(&Yprev[(size_t)j * (g + nbk)], &Ycur[(size_t)j * g], sizeof(double) * g);
    g += nbk;
  }
}

// ---------------------------------------------------------------------------
// Stage 2 smallest: simplified refined extraction (constant shift per target,
// incremental QR of (B - tau I) V) with hard locking (Sec. 3.2)
// ---------------------------------------------------------------------------
struct RefinedCfg : RunCfg {
  std::vector<double> taus;
};

// Fresh QR of (W - tau V): Q <- W - tau V, then CholQR2; returns R (column-major).
std::vector<double> fresh_qr(Ctx& c, RunBufs& B, int g, double tau) {
  const int prec = B.prec;
  // Q = W - tau V in column blocks of 32: each block is a combine of the two
  // matching column blocks with the coefficient [I; -tau I], whose table
  // stays small for any basis width
  for (int j0 = 0; j0 < g; j0 += 32) {
    const int w = std::min(32, g - j0);
    std::vector<double> coef((size_t)2 * w * w, 0.0);
    for (int j = 0; j < w; ++j) {
      coef[(size_t)j * w + j] = 1.0;         // W rows of the coefficient (first w rows)
      coef[(size_t)(w + j) * w + j] = -tau;  // V rows
    }
    combine(c, prec, B.L, {SegV{off(B.W, j0, prec), B.ldv, w}, SegV{off(B.V, j0, prec), B.ldv, w}}, coef, nullptr,
            0, false, off(B.Q, j0, prec), B.ldv, w);
  }
  OrthoRes o = ortho(c, prec, B.L, {}, B.Q, B.ldv, g, nullptr, 0);
  std::vector<double> R((size_t)g * g);
  for (int i = 0; i < g; ++i)
    for (int j = 0; j < g; ++j) R[(size_t)j * g + i] = o.R[(size_t)i * g + j];
  return R;
}

RunOut run_refined(Ctx& c, RunBufs& B, const RefinedCfg& cfg, std::vector<double>& locked_theta) {
  const int prec = B.prec;
  const int k = cfg.k, b = cfg.b;
  RunOut out;
  int g = 0;
  std::vector<double> H;
  init_basis(c, B, cfg, OP_B, g, H, {});
  int i = 0;
  std::vector<double> Rq = fresh_qr(c, B, g, cfg.taus[0]);
  std::vector<double> Yprev;
  int nprev = 0, rsr = 0;
  locked_theta.clear();
  while (i < k) {
    c.budget();
    ++out.outer;
    const double tau = cfg.taus[i];
    std::vector<double> s(g), Yr((size_t)g * g);
    hla::svd_right(g, Rq.data(), s.data(), Yr.data());
    const int nbk = std::min(b, g);
    std::vector<double> theta(g, 0.0);
    for (int j = 0; j < nbk; ++j) {
      const double* y = &Yr[(size_t)j * g];
      double acc = 0;
      for (int a = 0; a < g; ++a) {
        double hy = 0;
        for (int bb = 0; bb < g; ++bb) hy += H[(size_t)bb * g + a] * y[bb];
        acc += y[a] * hy;
      }
      theta[j] = acc;
    }
    std::vector<int> cols(nbk);
    for (int j = 0; j < nbk; ++j) cols[j] = j;
    std::vector<double> rn = ritz_cols(c, B, g, Yr, theta, cols, 0);
    std::vector<char> ok(1, 0);
    cfg.conv(theta.data(), rn.data(), 0, 1, ok.data());
    if (c.print >= 3)
      std::fprintf(stderr, "[%s] it %lld g %d locked %d tau %.10e theta %.10e res %.3e smin %.3e mv %lld\n", cfg.name,
                   out.outer, g, i, tau, theta[0], rn[0], s[0], c.mv);
    if (ok[0]) {
      CK(launch_copy_cols(prec, B.L, B.Xb, b, off(B.Xlock, i, prec), k, 1, c.st));
      c.launches += 1;
      locked_theta.push_back(theta[0]);
      ++i;
      if (i == k) break;
      // forced restart without the locked direction; QR recomputed with the next shift
      const int gk = std::min(g - 1, cfg.mr);
      std::vector<double> keep((size_t)g * gk);
      std::memcpy(keep.data(), &Yr[(size_t)g], sizeof(double) * g * gk);
      std::vector<double> Kr = rowmajor(g, gk, keep.data(), g);
      combine(c, prec, B.L, {SegV{B.V, B.ldv, g}}, Kr, nullptr, 0, false, B.V, B.ldv, gk);
      combine(c, prec, B.L, {SegV{B.W, B.ldv, g}}, Kr, nullptr, 0, false, B.W, B.ldv, gk);
      H = project_H(H, g, keep, gk);
      g = gk;
      if (g == 0) throw NumFail{"refined extraction lost its basis"};
      Rq = fresh_qr(c, B, g, cfg.taus[i]);
      nprev = 0;
      Yprev.clear();
      ++rsr;
      c.restarts += 1;
      continue;
    }
    if (rsr > 0 && rn[0] < std::sqrt((double)rsr) * cfg.normop * cfg.u) {
      std::vector<SegV> ag;
      if (i > 0) ag.push_back(SegV{B.Xlock, k, i});
      reset_basis(c, B, OP_B, g, H, ag);
      Rq = fresh_qr(c, B, g, tau);
      rsr = 0;
      nprev = 0;
      Yprev.clear();
      continue;
    }
    std::vector<double> Ycur((size_t)g * nbk);
    std::memcpy(Ycur.data(), Yr.data(), sizeof(double) * g * nbk);
    if (g + nbk > cfg.mb) {
      const int mr = std::min(cfg.mr, g);
      std::vector<double> zc((size_t)g * (mr + nprev));
      std::memcpy(zc.data(), Yr.data(), sizeof(double) * g * mr);
      if (nprev) std::memcpy(&zc[(size_t)g * mr], Yprev.data(), sizeof(double) * g * nprev);
      const int gz = hla::orth_cols(g, mr + nprev, zc.data(), 1e-12);
      std::vector<double> Zr = rowmajor(g, gz, zc.data(), g);
      combine(c, prec, B.L, {SegV{B.V, B.ldv, g}}, Zr, nullptr, 0, false, B.V, B.ldv, gz);
      combine(c, prec, B.L, {SegV{B.W, B.ldv, g}}, Zr, nullptr, 0, false, B.W, B.ldv, gz);
      H = project_H(H, g, zc, gz);
      // QR restart: R Z = Qt Rt, Q <- Q Qt, R <- Rt
      std::vector<double> RZ((size_t)g * gz);
      hla::gemm_nn(g, gz, g, Rq.data(), g, zc.data(), g, RZ.data(), g);
      std::vector<double> Qt = RZ;
      const int kept = hla::orth_cols(g, gz, Qt.data(), 1e-14);
      std::vector<double> Yn((size_t)gz * nbk);
      hla::gemm_tn(gz, nbk, g, zc.data(), g, Ycur.data(), g, Yn.data(), gz);
      Ycur.swap(Yn);
      if (kept == gz) {
        std::vector<double> Rt((size_t)gz * gz);
        hla::gemm_tn(gz, gz, g, Qt.data(), g, RZ.data(), g, Rt.data(), gz);
        for (int jj = 0; jj < gz; ++jj)
          for (int ii = jj + 1; ii < gz; ++ii) Rt[(size_t)jj * gz + ii] = 0.0;
        combine(c, prec, B.L, {SegV{B.Q, B.ldv, g}}, rowmajor(g, gz, Qt.data(), g), nullptr, 0, false, B.Q, B.ldv, gz);
        g = gz;
        Rq = Rt;
      } else {
        g = gz;
        Rq = fresh_qr(c, B, g, tau);
      }
      ++rsr;
      c.restarts += 1;
    }
    void* Tc = B.Rb;
    if (cfg.jd) {
      // the lower bound tau is the shift of the correction equation (Sec. 3.1)
      jd_correction(c, B, cfg, nbk, std::vector<double>(nbk, tau), rn);
      Tc = B.Tb;
    }
    std::vector<SegV> basis;
    if (i > 0) basis.push_back(SegV{B.Xlock, k, i});
    basis.push_back(SegV{B.V, B.ldv, g});
    ortho(c, prec, B.L, basis, Tc, b, nbk, off(B.V, g, prec), B.ldv);
    apply_op(c, prec, OP_B, Tc, b, off(B.W, g, prec), B.ldv, nbk, B.tmp, b);
    // Z = W T - tau T, orthonormalised against Q: extends (B - tau I)V = QR
    std::vector<double> coef((size_t)2 * nbk * nbk, 0.0);
    for (int j = 0; j < nbk; ++j) {
      coef[(size_t)j * nbk + j] = 1.0;
      coef[(size_t)(nbk + j) * nbk + j] = -tau;
    }
    combine(c, prec, B.L, {SegV{off(B.W, g, prec), B.ldv, nbk}, SegV{Tc, b, nbk}}, coef, nullptr, 0, false, B.Zb, b,
            nbk);
    OrthoRes oz = ortho(c, prec, B.L, {SegV{B.Q, B.ldv, g}}, B.Zb, b, nbk, off(B.Q, g, prec), B.ldv);
    std::vector<double> Hext = gram(c, prec, 0, B.L, {SegV{B.V, B.ldv, g + nbk}}, SegV{off(B.W, g, prec), B.ldv, nbk});
    extend_H(H, g, nbk, Hext);
    const int gn = g + nbk;
    if (oz.replaced) {
      g = gn;
      Rq = fresh_qr(c, B, g, tau);
    } else {
      std::vector<double> Rn((size_t)gn * gn, 0.0);
      for (int jj = 0; jj < g; ++jj)
        for (int ii = 0; ii <= jj; ++ii) Rn[(size_t)jj * gn + ii] = Rq[(size_t)jj * g + ii];
      for (int jj = 0; jj < nbk; ++jj) {
        for (int ii = 0; ii < g; ++ii) Rn[(size_t)(g + jj) * gn + ii] = oz.C[(size_t)ii * nbk + jj];
        for (int ii = 0; ii <= jj; ++ii) Rn[(size_t)(g + jj) * gn + g + ii] = oz.R[(size_t)ii * nbk + jj];
      }
      Rq.swap(Rn);
      g = gn;
    }
    nprev = nbk;
    Yprev.assign((size_t)g * nbk, 0.0);
    for (int j = 0; j < nbk; ++j)
      std::memcpy(&Yprev[(size_t)j * g], &Ycur[(size_t)j * (g - nbk)], sizeof(double) * (g - nbk));
  }
  out.theta = locked_theta;
  return out;
}

// Sizes: paper defaults (Sec. 3.4) with the reading for larger k and b.
void default_sizes(int k, int b, bool smallest, int& mb, int& mr) {
  if (!smallest && k < 10) {
    mb = 15;
    mr = 6;
  } else {
    mb = 35;
    mr = 14;
  }
  mr = std::max(mr, k + b);
  mb = std::max(mb, mr + 2 * b);
}

}  // namespace

static thread_local std::string g_last_error;
void set_last_error(const std::string& s) { g_last_error = s; }
const char* last_error_cstr() { return g_last_error.c_str(); }

// ===========================================================================
// Algorithm 1
// ===========================================================================
// The device-side CGS2 + CholQR2 of the solver on caller buffers, with its own
// scratch (the kernel-level entry point phsvds_ortho).
int ortho_block(int prec, long long L, const void* V, long long ldv, int g, void* T, long long ldt, int nb,
                int* status, cudaStream_t st, bool repair, unsigned long long seed, int* replaced) {
  Ctx c;
  c.st = st;
  c.maxblk = gram_default_blocks();
  c.seed = seed;
  std::vector<void*> mem;
  void* hpin = nullptr;
  auto take = [&](size_t bytes) -> void* {
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    mem.push_back(p);
    return p;
  };
  auto done = [&](int code) {
    cudaStreamSynchronize(st);
    for (void* p : mem) cudaFree(p);
    if (hpin) cudaFreeHost(hpin);
    return code;
  };
  c.partial = take(gram_partial_bytes(c.maxblk, 256, 8));
  c.dGo = static_cast<double*>(take(sizeof(double) * 264 * 8));
  c.dwork = static_cast<double*>(take(sizeof(double) * 128));
  for (int i = 0; i < 4; ++i) c.dco[i] = take(sizeof(double) * 264 * 8);
  c.dstatus = static_cast<int*>(take(256));
  if (!c.partial || !c.dGo || !c.dwork || !c.dco[0] || !c.dco[1] || !c.dco[2] || !c.dco[3] || !c.dstatus)
    return done(SVDS_ERR_NOMEM);
  // the host-driven repair needs a copy of the block, the Gram staging and
  // coefficient slots (as in a solve)
  void* T0 = nullptr;
  if (repair) {
    c.gcap = 264 * 8;
    c.nslots = 8;
    c.slot_bytes = 264 * 8 * 8;  // a (g + nb) x nb coefficient block
    c.dG = static_cast<double*>(take(sizeof(double) * c.gcap));
    c.dstage = static_cast<char*>(take((size_t)c.nslots * c.slot_bytes));
    T0 = take((size_t)L * nb * elem_bytes(prec));
    if (cudaMallocHost(&hpin, sizeof(double) * c.gcap + (size_t)c.nslots * c.slot_bytes) != cudaSuccess) {
      cudaGetLastError();
      hpin = nullptr;
    }
    if (!c.dG || !c.dstage || !T0 || !hpin) return done(SVDS_ERR_NOMEM);
    c.hG = static_cast<double*>(hpin);
    c.hstage = static_cast<char*>(hpin) + sizeof(double) * c.gcap;
    c.slot_epoch.assign(c.nslots, 0);
  }
  if (replaced) *replaced = 0;
  try {
    CK(cudaMemsetAsync(c.dstatus, 0, sizeof(int), st));
    if (repair) CK(launch_copy_cols(prec, L, T, ldt, T0, nb, nb, st));
    ortho_dev(c, prec, L, SegV{V, ldv, g}, T, ldt, nb, nullptr, 0);
    int hs = 0;
    CK(cudaMemcpyAsync(&hs, c.dstatus, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (status) *status = hs;
    if (repair && hs != 0) {
      // the solver's breakdown path: the block as given, orthonormalised by the
      // host-driven CGS2 + CholQR2 that replaces dependent columns
      CK(launch_copy_cols(prec, L, T0, nb, T, ldt, nb, st));
      OrthoRes r = ortho(c, prec, L, {SegV{V, ldv, g}}, T, ldt, nb, nullptr, 0);
      if (replaced) *replaced = r.replaced ? 1 : 0;
    }
  } catch (const CudaFail& f) {
    set_last_error(std::string(cudaGetErrorString(f.e)) + " at " + f.where);
    cudaGetLastError();
    return done(SVDS_ERR_CUDA);
  } catch (const NumFail& f) {
    set_last_error(f.what);
    return done(SVDS_ERR_NUMERIC);
  }
  return done(SVDS_OK);
}

int solve(svds_handle* h, int k, int target, double tol, double* sigma, double* Uout, double* Vout, double* rnorm,
          int* numConverged, svds_stats* stats) {
  const auto tstart = Clock::now();
  DevMatrix& A = h->A;
  const svds_opts& o = h->opts;
  const long long m = A.m, n = A.n, L2 = m + n;
  const bool smallest = target == SVDS_SMALLEST;
  const int b = std::max(1, o.maxBlockSize);
  int mb, mr;
  default_sizes(k, b, smallest, mb, mr);
  if (o.maxBasisSize > 0) mb = o.maxBasisSize;
  if (o.minRestartSize > 0) mr = o.minRestartSize;
  if (mr < k + b - 1 || mb < mr + b || mb > 240) return SVDS_ERR_ARG;
  const bool bf16 = o.stage1_precision == SVDS_BF16;
  const bool lowprec = o.stage1_precision == SVDS_FP32 || bf16;
  const int p2 = o.stage1_precision == SVDS_NATIVE_FP64 ? kF64 : kDF64;  // FP64-class mode
  const int p1a = lowprec ? kF32 : p2;
  const bool polish = !lowprec || o.stage1_polish;
  const long long ldv = (mb + 3) & ~3LL;
  // columns of the stage-1 blocks: k vectors, and with a reduced-precision
  // first phase b more for the start of the FP64-class phase
  const int kk = std::max(std::max(k, b), std::min(std::max(o.initSize, 0), k)) +
                 ((o.stage1_precision == SVDS_FP32 || o.stage1_precision == SVDS_BF16) ? b : 0);

  Ctx c;
  c.h = h;
  c.st = h->stream;
  c.A = &A;
  c.max_mv = o.maxMatvecs;
  c.max_sec = o.maxSeconds;
  c.t0 = tstart;
  c.print = o.printLevel;
  c.seed = o.seed;
  svds_stats S{};
  struct GnnGuard {
    phsvds_gnn* g = nullptr;
    ~GnnGuard() { phsvds_gnn_destroy(g); }
  } gnn_guard;
  struct BjGuard {  // device arrays of the block-Jacobi preconditioner
    void* p[4] = {nullptr, nullptr, nullptr, nullptr};
    ~BjGuard() {
      for (void* q : p)
        if (q) cudaFree(q);
    }
  } bj_guard;
  try {
    // ---- workspace ----
    struct Req {
      void** p;
      size_t bytes;
    };
    std::vector<Req> reqs;
    RunBufs B1a, B1, B2;
    auto plan_run = [&](RunBufs& R, int prec, long long L, bool refined, bool jdrun) {
      const size_t e = elem_bytes(prec);
      R.prec = prec;
      R.L = L;
      R.ldv = ldv;
      R.b = b;
      reqs.push_back({&R.V, (size_t)L * ldv * e});
      reqs.push_back({&R.W, (size_t)L * ldv * e});
      reqs.push_back({&R.Xb, (size_t)L * b * e});
      reqs.push_back({&R.Rb, (size_t)L * b * e});
      reqs.push_back({&R.Tb, (size_t)L * b * e});
      reqs.push_back({&R.BXb, (size_t)L * b * e});
      reqs.push_back({&R.tmp, (size_t)m * b * e});
      if (jdrun) {
        for (int i = 0; i < 8; ++i) reqs.push_back({&R.jd[i], (size_t)L * b * 8});
        reqs.push_back({&R.ju, (size_t)L * b * 8});
        reqs.push_back({(void**)&R.jtick, 64});
        reqs.push_back({&R.jtmp, (size_t)m * b * 8});
        reqs.push_back({(void**)&R.jS, sizeof(QmrState) * 8});
        reqs.push_back({(void**)&R.jdots, sizeof(double) * 64});
      }
      if (refined) {
        reqs.push_back({&R.Q, (size_t)L * ldv * e});
        reqs.push_back({&R.Zb, (size_t)L * b * e});
        reqs.push_back({&R.Xlock, (size_t)L * k * e});
      }
    };
    const bool dyn1 = o.method_stage1 == SVDS_DYNAMIC;
    const bool jd1 = o.method_stage1 == SVDS_JDQMR || dyn1, jd2 = o.method_stage2 == SVDS_JDQMR;
    if (lowprec) plan_run(B1a, kF32, n, false, jd1);
    plan_run(B1, p2, n, false, jd1);
    plan_run(B2, p2, L2, smallest, jd2);
    float* dj32 = nullptr;
    if (jd1) reqs.push_back({(void**)&dj32, (size_t)n * 4});
    const size_t e2 = elem_bytes(p2);
    void *X1a = nullptr, *X1 = nullptr, *CX = nullptr, *Xfin = nullptr, *BXfin = nullptr, *R2 = nullptr,
         *Xout2 = nullptr, *d1a = nullptr, *d1 = nullptr, *dout = nullptr;
    if (lowprec) reqs.push_back({&X1a, (size_t)n * kk * 4});
    reqs.push_back({&X1, (size_t)n * kk * e2});
    reqs.push_back({&CX, (size_t)n * kk * e2});
    reqs.push_back({&R2, (size_t)n * kk * e2});
    reqs.push_back({&Xfin, (size_t)L2 * kk * e2});
    reqs.push_back({&BXfin, (size_t)L2 * kk * e2});
    reqs.push_back({&Xout2, (size_t)L2 * kk * e2});
    if (lowprec) reqs.push_back({&d1a, (size_t)n * 4});
    reqs.push_back({&d1, (size_t)n * e2});
    reqs.push_back({&dout, (size_t)L2 * kk * 8});
    void* dout2 = nullptr;  // the returned U and V blocks, contiguous, in output order
    reqs.push_back({&dout2, (size_t)L2 * kk * 8 + sizeof(int) * kk + 256});
    c.maxblk = gram_default_blocks();
    c.gcap = 256 * 256;
    reqs.push_back({&c.partial, gram_partial_bytes(std::max(c.maxblk, 152 * 16), 256, 8)});
    reqs.push_back({(void**)&c.dG, c.gcap * 8});
    if (A.user) {  // FP64 staging of the caller's operator: blocks of up to b columns of B
      reqs.push_back({(void**)&c.ux, (size_t)L2 * b * 8});
      reqs.push_back({(void**)&c.uy, (size_t)L2 * b * 8});
    }
    reqs.push_back({(void**)&c.dGo, sizeof(double) * 264 * 8});
    reqs.push_back({(void**)&c.dwork, sizeof(double) * 128});
    for (int i = 0; i < 4; ++i) reqs.push_back({&c.dco[i], sizeof(double) * 264 * 8});
    reqs.push_back({(void**)&c.dstatus, 256});
    reqs.push_back({(void**)&c.dflag, 256});
    c.nslots = 64;
    // one slot holds the largest coefficient block (8-byte coefficients): a
    // basis-by-basis restart matrix of the widest basis, or the 2g x g block of
    // the refined extraction's fresh QR of W - tau V
    c.slot_bytes = std::max<size_t>({(size_t)2 * 256 * 256, (size_t)(ldv + 8) * (ldv + 8) * 8,
                                     (size_t)2 * ldv * ldv * 8});
    c.slot_bytes = (c.slot_bytes + 255) & ~size_t(255);
    reqs.push_back({(void**)&c.dstage, (size_t)c.nslots * c.slot_bytes});
    size_t total = 0;
    for (auto& r : reqs) total += (r.bytes + 255) & ~size_t(255);
    total += 4096;
    if (h->arena.cap < total) {
      if (h->arena.base) cudaFree(h->arena.base);
      h->arena = Arena{};
      if (cudaMalloc(&h->arena.base, total) != cudaSuccess) {
        cudaGetLastError();
        set_last_error("workspace allocation failed");
        return SVDS_ERR_NOMEM;
      }
      h->arena.cap = total;
    }
    h->arena.used = 0;
    for (auto& r : reqs) *r.p = h->arena.take(r.bytes);
    const size_t hneed = c.gcap * 8 + (size_t)c.nslots * c.slot_bytes + 256;
    if (h->hpin_bytes < hneed) {
      if (h->hpin) cudaFreeHost(h->hpin);
      h->hpin = nullptr;
      h->hpin_bytes = 0;
      if (cudaMallocHost(&h->hpin, hneed) != cudaSuccess) {
        cudaGetLastError();
        return SVDS_ERR_NOMEM;
      }
      h->hpin_bytes = hneed;
    }
    c.hG = reinterpret_cast<double*>(h->hpin);
    c.hstage = reinterpret_cast<char*>(h->hpin) + c.gcap * 8;
    c.slot_epoch.assign(c.nslots, 0);
    c.hstatus = reinterpret_cast<int*>(c.hstage + (size_t)c.nslots * c.slot_bytes);
    CK(cudaMemsetAsync(c.dstatus, 0, sizeof(int), c.st));
    B1.Xlock = nullptr;

    // ---- C = A^T A as one sparse matrix when that moves fewer bytes ----
    ensure_normal(h, c.st, o.normalOperator, b, c.launches);
    if (bf16) {
      ensure_bf16(h, c.st, c.launches);
      c.bf16 = true;
    }

    // ---- ||A|| (reading: estimate when not given; raised by later Ritz values) ----
    double normA = o.aNorm > 0 ? o.aNorm * A.scale : 0.0;
    // relative mode (condition-number estimate, Sec. 5) for the largest value:
    // no estimate needed, the Ritz value itself gives ||A|| at the end
    const double relTol = o.relTol;
    const double t_norm0 = c.elapsed();
    if (normA <= 0 && !(relTol > 0 && !smallest)) {
      // Lanczos (Arnoldi with full reorthogonalisation) on C from a seeded
      // random vector.  theta_max of the projected matrix is a lower bound of
      // ||C||, so the stopping tolerance ||r|| <= tol ||A|| can only get
      // stricter; it converges fast at the top of the spectrum.  Stop when it
      // changed by at most 1e-3 relative in two consecutive steps, on an
      // invariant subspace, or after 50 steps: ||A|| only scales tolerances,
      // so an estimate a few 1e-3 low (measured 2.3e-3 on the 2-D grid
      // Laplacian, half the steps of a 1e-5 rule) tightens them by that much.
      RunBufs& Bn = lowprec ? B1a : B1;
      const int pn = Bn.prec;
      const int maxs = (int)std::min<long long>(50, Bn.ldv - 1);  // columns of the basis buffer
      CK(launch_fill_normal(pn, n, Bn.V, Bn.ldv, 1, o.seed ^ 0x5eedULL, c.st));
      c.launches += 1;
      ortho(c, pn, n, {}, Bn.V, Bn.ldv, 1, nullptr, 0);
      std::vector<double> H((size_t)(maxs + 1) * (maxs + 1), 0.0);  // column-major, ld maxs + 1
      CK(cudaMemsetAsync(c.dstatus, 0, sizeof(int), c.st));
      double theta = 0.0;
      int calm = 0;
      for (int j = 0; j < maxs; ++j) {
        apply_op(c, pn, OP_C, off(Bn.V, j, pn), Bn.ldv, Bn.W, Bn.ldv, 1, Bn.tmp, Bn.b);
        // h = V^T w in a Gram, then the device-side CGS2 + CholQR2 of w into
        // the next basis column: one host round trip per step
        gram_dev(c, pn, 0, n, {SegV{Bn.V, Bn.ldv, j + 1}}, SegV{Bn.W, Bn.ldv, 1}, c.dG);
        if (j + 1 < maxs) ortho_dev(c, pn, n, SegV{Bn.V, Bn.ldv, j + 1}, Bn.W, Bn.ldv, 1, off(Bn.V, j + 1, pn), Bn.ldv);
        CK(cudaMemcpyAsync(c.hG, c.dG, sizeof(double) * (j + 1), cudaMemcpyDeviceToHost, c.st));
        const bool breakdown = take_status(c) != 0;
        for (int i = 0; i <= j; ++i) H[(size_t)j * (maxs + 1) + i] = c.hG[i];
        const int g = j + 1;
        // V^T C V from the upper triangle of the Arnoldi coefficients (C symmetric)
        std::vector<double> Hs((size_t)g * g), w(g), Z((size_t)g * g);
        for (int a = 0; a < g; ++a)
          for (int bb = 0; bb < g; ++bb)
            Hs[(size_t)bb * g + a] = H[(size_t)std::max(a, bb) * (maxs + 1) + std::min(a, bb)];
        if (!hla::sym_eig(g, Hs.data(), w.data(), Z.data())) throw NumFail{"norm estimate eigenproblem failed"};
        const double th = w[g - 1];
        calm = (theta > 0 && std::fabs(th - theta) <= 1e-3 * std::fabs(th)) ? calm + 1 : 0;
        theta = std::max(theta, th);
        S.norm_steps = j + 1;
        if (breakdown || calm >= 2) break;
      }
      normA = std::sqrt(std::fabs(theta));
      S.seconds_norm = c.elapsed() - t_norm0;
    }
    const double normC = normA * normA;
    S.seconds_setup = c.elapsed();

    // ---- stage 1 on C (Algorithm 1 lines 1-3) ----
    // relative mode: ||r^C|| <= relTol |lambda| (Sec. 5), floor 10 u max(||C||, |lambda|)
    auto stage1_conv = [&](double u) {
      return [=](const double* th, const double* rn, int, int nc, char* ok) {
        for (int j = 0; j < nc; ++j) {
          const double lam = std::fabs(th[j]);
          ok[j] = relTol > 0 ? rn[j] <= std::max(relTol * lam, 10.0 * u * std::max(normC, lam))
                             : rn[j] <= std::max(std::sqrt(lam * normC) * tol, 10.0 * u * normC);
        }
      };
    };
    const bool jac = smallest && o.precond == SVDS_PRECOND_JACOBI;
    // learned sparse approximate inverse on the pattern of C (stage 1 only,
    // smallest values; its scale is immaterial to GD+k and to the sQMR
    // iterates); the plain Jacobi preconditioner is its fallback, so the
    // Jacobi scalings are built for it too
    bool learned = smallest && o.precond == SVDS_PRECOND_LEARNED && !h->gnn_params.empty();
    if (jac || learned) {
      if (lowprec) CK(launch_make_dscale(kF32, n, A.colsq, 0, d1a, c.st));
      CK(launch_make_dscale(p2, n, A.colsq, 0, d1, c.st));
      c.launches += lowprec ? 2 : 1;
      if (jd1) {
        CK(launch_make_dscale(kF32, n, A.colsq, 0, dj32, c.st));
        c.launches += 1;
      }
    }
    CsrDev K32, K64;
    if (learned) {
      const double tp = c.elapsed();
      phsvds_gnn* gg = nullptr;
      int grc = gnn_build(&gg, A, false, false, c.st);
      if (grc == 0) {
        gnn_guard.g = gg;
        grc = gnn_precond(gg, h->gnn_params.data(), &K32, p2 == kF64 ? &K64 : nullptr);
      }
      if (grc == SVDS_ERR_NOMEM) return SVDS_ERR_NOMEM;
      if (grc) throw CudaFail{cudaErrorUnknown, "learned preconditioner"};
      c.launches += gnn_launches(gg);
      // M must be usable: finite values and a positive diagonal (its
      // construction guarantees both for finite parameters unless the
      // diagonal underflows); otherwise Jacobi replaces it for the whole solve
      CK(cudaMemsetAsync(c.dflag, 0, sizeof(int), c.st));
      CK(launch_precond_check(n, K32.rowptr, K32.colidx, K32.v32, nullptr, c.dflag, c.st));
      if (p2 == kF64) CK(launch_precond_check(n, K64.rowptr, K64.colidx, nullptr, K64.v64, c.dflag, c.st));
      c.launches += p2 == kF64 ? 2 : 1;
      CK(cudaMemcpyAsync(c.hstatus + 1, c.dflag, sizeof(int), cudaMemcpyDeviceToHost, c.st));
      c.sync();
      if (c.hstatus[1] != 0) {
        learned = false;
        c.precond_fallback = 1;
        if (c.print >= 1)
          std::fprintf(stderr, "[setup] learned preconditioner rejected (%s): Jacobi instead\n",
                       (c.hstatus[1] & 1) ? "non-finite value" : "non-positive diagonal");
      }
      S.seconds_precond = c.elapsed() - tp;
    }
    // Jacobi where the learned preconditioner was asked for and rejected
    const bool jac_fb = c.precond_fallback == 1;
    // block Jacobi on C (Sec. 4), stage 1, smallest values: a CSR matrix with
    // dense diagonal blocks, applied by the same SpMM kernels as the learned M
    const bool bjac = smallest && o.precond == SVDS_PRECOND_BLOCKJACOBI;
    if (bjac) {
      const double tp = c.elapsed();
      const int bs = o.precondBlockSize > 0 ? o.precondBlockSize : 32;
      const long long nz = bj_nnz(n, bs);
      const bool want64 = p2 == kF64;
      const size_t sz[4] = {sizeof(int) * (size_t)(n + 1), sizeof(int) * (size_t)nz, sizeof(float) * (size_t)nz,
                            want64 ? sizeof(double) * (size_t)nz : 0};
      for (int i = 0; i < 4; ++i)
        if (sz[i] && cudaMalloc(&bj_guard.p[i], sz[i]) != cudaSuccess) {
          cudaGetLastError();
          set_last_error("block-Jacobi allocation failed");
          return SVDS_ERR_NOMEM;
        }
      int* brp = static_cast<int*>(bj_guard.p[0]);
      int* bci = static_cast<int*>(bj_guard.p[1]);
      float* b32 = static_cast<float*>(bj_guard.p[2]);
      double* b64 = static_cast<double*>(bj_guard.p[3]);
      CK(launch_bj_build(n, bs, A.rowptrT, A.colidxT, A.v64T, brp, bci, b32, b64, c.st));
      c.launches += 1;
      for (CsrDev* Kd : {&K32, &K64}) {
        Kd->rows = n;
        Kd->cols = n;
        Kd->nnz = nz;
        Kd->rowptr = brp;
        Kd->colidx = bci;
      }
      K32.v32 = b32;
      K64.v64 = b64;
      c.sync();
      S.seconds_precond = c.elapsed() - tp;
    }
    const bool sparseM = learned || bjac;
    const CsrDev* Kouter = sparseM ? (p2 == kF64 ? &K64 : &K32) : nullptr;
    const int jd_prec = o.innerPrecision == SVDS_DF64 ? p2 : kF32;
    const CsrDev* Kinner = sparseM ? (jd_prec == kF64 ? &K64 : &K32) : nullptr;
    const int jd_maxk = o.innerMaxIt > 0 ? o.innerMaxIt : 30;
    const double jd_xi = o.innerRelTol > 0 ? o.innerRelTol : 0.1;
    // initial block: user guesses then seeded N(0,1) columns
    // initial block (ncols columns, leading dimension ld): user guesses first
    // (initSize, initV), then seeded N(0,1) columns
    auto init_block = [&](int prec, void* dst, long long ld, int ncols) {
      int given = 0;
      if (o.initV && o.initSize > 0) {
        given = std::min(o.initSize, ncols);
        double* dtmp = reinterpret_cast<double*>(dout);
        CK(cudaMemcpyAsync(dtmp, o.initV, sizeof(double) * n * given, cudaMemcpyHostToDevice, c.st));
        CK(launch_from_f64_colmajor(prec, n, given, dtmp, n, dst, ld, 1.0, c.st));
        c.launches += 1;
      }
      if (given < ncols) {
        CK(launch_fill_normal(prec, n, off(dst, given, prec), ld, ncols - given, o.seed, c.st));
        c.launches += 1;
      }
    };
    const int b0 = std::max(b, std::min(o.initSize, k));
    const double t1 = c.elapsed();
    const long long mv0 = c.mv;
    RunCfg c1;
    c1.op = OP_C;
    c1.k = k;
    c1.b = b;
    c1.mb = mb;
    c1.mr = mr;
    c1.smallest = smallest;
    c1.normop = normC;
    c1.b0 = b0;
    // the relative mode (block 1, loose stop) keeps GD+k corrections: JDQMR
    // corrections there can settle on an interior eigenvalue (Sec. 5 notes the
    // risk of missing the extreme pair at low accuracy)
    c1.jd = jd1 && !dyn1 && !(relTol > 0);
    c1.dyn = dyn1 && !(relTol > 0);
    c1.jd_prec = jd_prec;
    const void* jd_jacobi = jd_prec == kF32 ? static_cast<const void*>(dj32) : static_cast<const void*>(d1);
    c1.jdinv = (jac || jac_fb) ? jd_jacobi : nullptr;
    if (learned) {
      c1.stall_its = o.precondStallIts == 0 ? 50 : std::max(0, o.precondStallIts);
      c1.fb_jdinv = jd_jacobi;
    }
    c1.jd_maxk = jd_maxk;
    c1.jd_xi = jd_xi;
    c1.jdK = Kinner;
    if (lowprec) {
      init_block(kF32, X1a, kk, b0);
      // bfloat16 values that round A (or C) perturb the operator by ~2^-8 of
      // ||C||: for the largest values the FP32 phase stops at that floor.  The
      // smallest eigenvalues of the rounded operator move far less than that
      // bound (random rounding errors), but a pair accepted at a 2^-8 ||C||
      // residual has no accuracy at all when its value is far below it, and
      // such vectors steer the FP64-class phase away from the smallest pair;
      // for the smallest values the phase runs to its arithmetic's floor
      const bool exact_vals = A.exact16 && (A.nnzC > 0 ? A.exactC : A.exact32);
      c1.u = (bf16 && !exact_vals && !smallest) ? std::ldexp(1.0, -8) : unit_roundoff(kF32);
      c1.conv = stage1_conv(c1.u);
      c1.dscale = (jac || jac_fb) ? d1a : nullptr;
      c1.fb_dscale = d1a;
      c1.K = sparseM ? &K32 : nullptr;
      c1.V0 = X1a;
      c1.ldv0 = kk;
      c1.name = "stage1-fp32";
      RunOut ra = run_gdk_rr(c, B1a, c1, X1a, kk);
      S.outer_stage1 += ra.outer;
      S.outer_stage1_jdqmr += ra.outer_jd;
      S.matvecs_stage1_lowprec = c.mv - mv0;
      // hand the FP32 Ritz vectors to the FP64-class phase
      double* dtmp = reinterpret_cast<double*>(dout);
      CK(launch_to_f64_colmajor(kF32, n, k, X1a, kk, dtmp, n, 1.0, c.st));
      CK(launch_from_f64_colmajor(p2, n, k, dtmp, n, X1, kk, 1.0, c.st));
      // b seeded random columns beside them: a direction that the reduced-
      // precision operator could not resolve (a value below its floor) can
      // still enter the FP64-class basis
      CK(launch_fill_normal(p2, n, off(X1, k, p2), kk, b, o.seed ^ 0xB0B0ULL, c.st));
      c.launches += 3;
    } else {
      init_block(p2, X1, kk, b0);
    }
    std::vector<double> lam;
    if (polish) {
      c1.u = unit_roundoff(p2);
      c1.conv = stage1_conv(c1.u);
      c1.dscale = (jac || jac_fb) ? d1 : nullptr;
      c1.fb_dscale = d1;
      c1.K = Kouter;
      if (c.precond_fallback == 2) {  // the FP32 phase stalled with the learned M
        c1.dscale = d1;
        c1.K = nullptr;
        c1.jdK = nullptr;
        c1.jdinv = jd_jacobi;
      }
      c1.V0 = X1;
      c1.ldv0 = kk;
      c1.b0 = lowprec ? k + b : b0;
      c1.name = "stage1";
      RunOut r1 = run_gdk_rr(c, B1, c1, X1, kk);
      S.outer_stage1 += r1.outer;
      S.outer_stage1_jdqmr += r1.outer_jd;
      lam = r1.theta;
    }
    // ---- Algorithm 1 lines 4-5: Rayleigh-Ritz on the returned vectors ----
    ortho(c, p2, n, {}, X1, kk, k, nullptr, 0);
    apply_op(c, p2, OP_C, X1, kk, CX, kk, k, B1.tmp, b);
    std::vector<double> Hk = gram(c, p2, 0, n, {SegV{X1, kk, k}}, SegV{CX, kk, k});
    std::vector<double> Hkc((size_t)k * k), wk(k), Zk((size_t)k * k);
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < k; ++j) Hkc[(size_t)j * k + i] = 0.5 * (Hk[(size_t)i * k + j] + Hk[(size_t)j * k + i]);
    if (!hla::sym_eig(k, Hkc.data(), wk.data(), Zk.data())) throw NumFail{"final Rayleigh-Ritz failed"};
    std::vector<double> lk(k), Yk((size_t)k * k);
    for (int j = 0; j < k; ++j) {
      const int src = smallest ? j : k - 1 - j;
      lk[j] = wk[src];
      std::memcpy(&Yk[(size_t)j * k], &Zk[(size_t)src * k], sizeof(double) * k);
    }
    std::vector<double> rC(k), sig(k);
    // v = x (top n rows of Xfin), r^C = C x - lambda x, in blocks of up to 8 Ritz vectors
    for (int c0 = 0; c0 < k; c0 += 8) {
      const int w = std::min(8, k - c0);
      std::vector<double> Ych((size_t)k * w);  // rows of Yk, columns c0 .. c0 + w (row-major)
      for (int i = 0; i < k; ++i)
        for (int j = 0; j < w; ++j) Ych[(size_t)i * w + j] = Yk[(size_t)(c0 + j) * k + i];
      const void* dY = c.upload(p2, Ych.data(), Ych.size());
      const void* dth = c.upload(p2, lk.data() + c0, w);
      int nbl = 0;
      CK(launch_ritz_residual(p2, n, SegV{X1, kk, k}, SegV{CX, kk, k}, k, dY, dth, off(Xfin, c0, p2), off(R2, c0, p2),
                              kk, w, nullptr, nullptr, c.partial, c.maxblk, &nbl, c.st));
      CK(launch_gram_reduce(p2, c.partial, nbl, w, c.dG, c.st));
      c.launches += 2;
      CK(cudaMemcpyAsync(c.hG, c.dG, sizeof(double) * w, cudaMemcpyDeviceToHost, c.st));
      c.sync();
      for (int j = 0; j < w; ++j) rC[c0 + j] = std::sqrt(std::max(c.hG[j], 0.0));
    }
    for (int j = 0; j < k; ++j) sig[j] = std::sqrt(std::fabs(lk[j]));
    for (int j = 0; j < k; ++j) normA = std::max(normA, smallest ? 0.0 : sig[j]);
    // u = A v / sigma (bottom m rows of Xfin)
    void* Ufin = off(Xfin, n * kk, p2);
    if (A.user) {
      // [0; A v] = B [v; 0]: the lower rows of B applied to x with a zero left part
      CK(cudaMemsetAsync(Ufin, 0, (size_t)m * kk * e2, c.st));
      apply_op(c, p2, OP_B, Xfin, kk, BXfin, kk, k, B2.tmp, b);
      CK(launch_copy_cols(p2, m, off(BXfin, n * kk, p2), kk, Ufin, kk, k, c.st));
      c.launches += 1;
    } else {
      CK(launch_spmm(p2, A.csr(false), Xfin, kk, Ufin, kk, k, c.st));
      c.launches += spmm_launches(k);
      c.mv += k;
    }
    {
      std::vector<double> D((size_t)k * k, 0.0);
      for (int j = 0; j < k; ++j) D[(size_t)j * k + j] = sig[j] > 0 ? 1.0 / sig[j] : 1.0;
      combine(c, p2, m, {SegV{Ufin, kk, k}}, D, nullptr, 0, false, Ufin, kk, k);
    }
    // Eq. (res) for the stage-1 triplets, recomputed with fresh products
    auto triplet_res = [&](void* X, const std::vector<double>& s, int nc) {
      apply_op(c, p2, OP_B, X, kk, BXfin, kk, nc, B2.tmp, b);
      std::vector<double> cf((size_t)4 * nc);
      for (int j = 0; j < nc; ++j) {
        cf[j] = 1.0;
        cf[nc + j] = s[j];
        cf[2 * nc + j] = 1.0;
        cf[3 * nc + j] = s[j];
      }
      std::vector<double> r(nc, 0.0);
      for (int c0 = 0; c0 < nc; c0 += 8) {
        const int w = std::min(8, nc - c0);
        std::vector<double> cfc((size_t)4 * w);
        for (int j = 0; j < w; ++j) {
          cfc[j] = 1.0;
          cfc[w + j] = s[c0 + j];
          cfc[2 * w + j] = 1.0;
          cfc[3 * w + j] = s[c0 + j];
        }
        const void* dcf = c.upload(p2, cfc.data(), cfc.size());
        int nb2 = 0;
        CK(launch_split_resnorm(p2, L2, n, off(X, c0, p2), off(BXfin, c0, p2), kk, w, dcf, c.partial, c.maxblk, &nb2,
                                c.st));
        CK(launch_gram_reduce(p2, c.partial, nb2, w, c.dG, c.st));
        c.launches += 2;
        CK(cudaMemcpyAsync(c.hG, c.dG, sizeof(double) * w, cudaMemcpyDeviceToHost, c.st));
        c.sync();
        for (int j = 0; j < w; ++j) r[c0 + j] = std::sqrt(std::max(c.hG[j], 0.0));
      }
      return r;
    };
    std::vector<double> res = triplet_res(Xfin, sig, k);
    S.matvecs_stage1 = c.mv - mv0;
    S.seconds_stage1 = c.elapsed() - t1;
    bool all_ok = true;
    for (int j = 0; j < k; ++j) all_ok = all_ok && res[j] < normA * tol;
    if (relTol > 0) all_ok = true;  // the relative mode stops after stage 1
    void* Xres = Xfin;
    if (!all_ok) {
      // ---- stage 2 on B (Algorithm 1 lines 9-20) ----
      S.stage2_used = 1;
      const double t2 = c.elapsed();
      const long long mv2 = c.mv;
      RunCfg c2;
      c2.op = OP_B;
      c2.k = k;
      c2.b = b;
      int mb2, mr2;
      default_sizes(k, b, smallest, mb2, mr2);
      c2.mb = o.maxBasisSize > 0 ? mb : mb2;
      c2.mr = o.minRestartSize > 0 ? mr : mr2;
      if (c2.mb > mb) c2.mb = mb;  // buffers sized for mb
      c2.mr = std::min(c2.mr, c2.mb - b);
      c2.smallest = smallest;
      c2.normop = normA;
      c2.u = unit_roundoff(p2);
      c2.V0 = Xfin;
      c2.ldv0 = kk;
      c2.b0 = k;
      c2.name = "stage2";
      c2.jd = jd2;
      c2.jd_prec = jd_prec;
      c2.jd_maxk = jd_maxk;
      c2.jd_xi = jd_xi;
      RunBufs& Bs = B2;
      const double thr1 = std::sqrt(2.0) * normA * tol;
      // second level: Eq. (res) with a margin of the evaluation's own rounding
      // noise (a few units of the mode's roundoff times ||A||), so that a pair
      // accepted here also passes the final recomputation
      const double thr2 = normA * std::max(tol - 4.0 * unit_roundoff(p2), 0.5 * tol);
      // Eq. B_secondCriterion then Eq. (res) on the normalised halves
      c2.conv = [&](const double* th, const double* rn, int o0, int nc, char* ok) {
        bool any = false;
        for (int j = 0; j < nc; ++j) {
          ok[j] = rn[j] <= thr1;
          any = any || ok[j];
        }
        if (!any) return;
        void* Xc = off(Bs.Xb, o0, p2);
        apply_op(c, p2, OP_B, Xc, b, Bs.BXb, b, nc, Bs.tmp, b);
        std::vector<double> Gv = gram(c, p2, 0, n, {SegV{Xc, b, nc}}, SegV{Xc, b, nc});
        std::vector<double> Gu = gram(c, p2, n, L2, {SegV{Xc, b, nc}}, SegV{Xc, b, nc});
        std::vector<double> Gd = gram(c, p2, n, L2, {SegV{Xc, b, nc}}, SegV{Bs.BXb, b, nc});
        std::vector<double> cf((size_t)4 * nc);
        for (int j = 0; j < nc; ++j) {
          const double nv = std::sqrt(std::max(Gv[(size_t)j * nc + j], 1e-300));
          const double nu = std::sqrt(std::max(Gu[(size_t)j * nc + j], 1e-300));
          const double s = Gd[(size_t)j * nc + j] / (nv * nu);
          cf[j] = 1.0 / nu;           // rows < n: A^T u = (Bx)_v / ||x_u||
          cf[nc + j] = s / nv;        //           sigma v
          cf[2 * nc + j] = 1.0 / nv;  // rows >= n: A v = (Bx)_u / ||x_v||
          cf[3 * nc + j] = s / nu;    //           sigma u
        }
        const void* dcf = c.upload(p2, cf.data(), cf.size());
        int nb2 = 0;
        CK(launch_split_resnorm(p2, L2, n, Xc, Bs.BXb, b, nc, dcf, c.partial, c.maxblk, &nb2, c.st));
        CK(launch_gram_reduce(p2, c.partial, nb2, nc, c.dG, c.st));
        c.launches += 2;
        CK(cudaMemcpyAsync(c.hG, c.dG, sizeof(double) * nc, cudaMemcpyDeviceToHost, c.st));
        c.sync();
        for (int j = 0; j < nc; ++j) ok[j] = ok[j] && std::sqrt(std::max(c.hG[j], 0.0)) < thr2;
      };
      void* XB = nullptr;
      if (smallest) {
        RefinedCfg cr;
        static_cast<RunCfg&>(cr) = c2;
        cr.taus.resize(k);
        for (int j = 0; j < k; ++j) {
          // Algorithm 1 line 15: tau_i = max(s_i - sqrt(2) ||r^C_i|| / s_i, ||A|| eps)
          const double lb = sig[j] > 0 ? sig[j] - std::sqrt(2.0) * rC[j] / sig[j] : 0.0;
          cr.taus[j] = std::max(lb, normA * unit_roundoff(p2));
        }
        std::vector<double> lt;
        RunOut r2 = run_refined(c, Bs, cr, lt);
        S.outer_stage2 = r2.outer;
        XB = Bs.Xlock;
      } else {
        RunOut r2 = run_gdk_rr(c, Bs, c2, Xout2, kk);
        S.outer_stage2 = r2.outer;
        XB = Xout2;
      }
      // Algorithm 1 line 19: normalise the halves; sigma = u^T A v (reading)
      long long ldxb = smallest ? k : kk;
      std::vector<double> Gv = gram(c, p2, 0, n, {SegV{XB, ldxb, k}}, SegV{XB, ldxb, k});
      std::vector<double> Gu = gram(c, p2, n, L2, {SegV{XB, ldxb, k}}, SegV{XB, ldxb, k});
      std::vector<double> Dv((size_t)k * k, 0.0), Du((size_t)k * k, 0.0);
      for (int j = 0; j < k; ++j) {
        Dv[(size_t)j * k + j] = 1.0 / std::sqrt(std::max(Gv[(size_t)j * k + j], 1e-300));
        Du[(size_t)j * k + j] = 1.0 / std::sqrt(std::max(Gu[(size_t)j * k + j], 1e-300));
      }
      combine(c, p2, n, {SegV{XB, ldxb, k}}, Dv, nullptr, 0, false, Xfin, kk, k);
      combine(c, p2, m, {SegV{off(XB, n * ldxb, p2), ldxb, k}}, Du, nullptr, 0, false, off(Xfin, n * kk, p2), kk, k);
      apply_op(c, p2, OP_B, Xfin, kk, BXfin, kk, k, B2.tmp, b);
      // sigma_j = u_j^T (A v_j): rows [n, n + m) of Xfin against those of B Xfin
      std::vector<double> Gs = gram(c, p2, n, L2, {SegV{Xfin, kk, k}}, SegV{BXfin, kk, k});
      for (int j = 0; j < k; ++j) sig[j] = Gs[(size_t)j * k + j];
      res = triplet_res(Xfin, sig, k);
      S.matvecs_stage2 = c.mv - mv2;
      S.seconds_stage2 = c.elapsed() - t2;
    }
    // ---- outputs ----
    const double t_out = c.elapsed();
    std::vector<int> order(k);
    for (int j = 0; j < k; ++j) order[j] = j;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int bb) { return smallest ? sig[a] < sig[bb] : sig[a] > sig[bb]; });
    double* dtmp = reinterpret_cast<double*>(dout);
    const long long mu = A.transposed ? n : m;  // user rows
    const long long nu = A.transposed ? m : n;  // user cols
    const long long voff = A.transposed ? n : 0, uoff = A.transposed ? 0 : n;  // user v / u rows of x
    if (Uout || Vout) {
      // FP64 column-major copy, sign convention on the device (largest-|.|
      // entry of each v positive), then one copy per returned column
      CK(launch_to_f64_colmajor(p2, L2, k, Xres, kk, dtmp, L2, 1.0, c.st));
      // (the gather buffer is free until the gather below: the sign search uses it)
      CK(launch_col_sign(L2, L2, k, voff, nu, dtmp, reinterpret_cast<double*>(dout2), c.st));
      c.launches += 4;
      if (c.print >= 2) {
        c.sync();
        std::fprintf(stderr, "[output] conversion and signs done at %.4f s\n", c.elapsed() - t_out);
      }
      // gather the columns in output order so that U and V each leave in one
      // copy (many small copies into fresh pageable memory are far slower)
      int* dperm = reinterpret_cast<int*>(reinterpret_cast<char*>(dout2) + (size_t)L2 * k * 8);
      {
        std::vector<int> perm(order.begin(), order.end());
        CK(cudaMemcpyAsync(dperm, perm.data(), sizeof(int) * k, cudaMemcpyHostToDevice, c.st));
        double* Vblk = reinterpret_cast<double*>(dout2);
        double* Ublk = Vblk + (size_t)nu * k;
        CK(launch_gather_cols(nu, k, dtmp, L2, voff, dperm, Vblk, c.st));
        CK(launch_gather_cols(mu, k, dtmp, L2, uoff, dperm, Ublk, c.st));
        c.launches += 2;
        if (Vout) CK(cudaMemcpyAsync(Vout, Vblk, sizeof(double) * nu * k, cudaMemcpyDeviceToHost, c.st));
        if (Uout) CK(cudaMemcpyAsync(Uout, Ublk, sizeof(double) * mu * k, cudaMemcpyDeviceToHost, c.st));
        c.sync();  // perm stays alive until here
      }
    }
    int nconv = 0;
    bool prefix = true;
    for (int jj = 0; jj < k; ++jj) {
      const int j = order[jj];
      sigma[jj] = sig[j] / A.scale;
      if (rnorm) rnorm[jj] = res[j] / A.scale;
      const bool ok = relTol > 0 ? rC[j] <= std::max(relTol * std::fabs(lk[j]),
                                                      10.0 * unit_roundoff(p2) * std::max(normA * normA, std::fabs(lk[j])))
                                 : res[j] < normA * tol;
      if (prefix && ok)
        ++nconv;
      else
        prefix = false;
    }
    if (numConverged) *numConverged = nconv;
    S.aNorm = normA / A.scale;
    S.restarts = c.restarts;
    S.resets = c.resets;
    S.kernel_launches = c.launches;
    S.seconds_total = c.elapsed();
    S.seconds_host_eig = c.t_eig;
    S.seconds_sync_wait = c.t_sync;
    S.host_syncs = c.nsync;
    S.inner_steps = c.inner;
    S.normal_nnz = A.nnzC > 0 ? A.nnzC : 0;
    S.seconds_output = c.elapsed() - t_out;
    S.precond_fallback = c.precond_fallback;
    if (stats) *stats = S;
    h->launches += c.launches;
    return SVDS_OK;
  } catch (const CudaFail& f) {
    set_last_error(std::string(cudaGetErrorString(f.e)) + " at " + f.where);
    cudaGetLastError();
    if (stats) *stats = S;
    return SVDS_ERR_CUDA;
  } catch (const NumFail& f) {
    set_last_error(f.what);
    if (stats) *stats = S;
    return SVDS_ERR_NUMERIC;
  } catch (const OpFail& f) {
    set_last_error("the caller-supplied operator returned " + std::to_string(f.rc));
    if (stats) *stats = S;
    return SVDS_ERR_OPERATOR;
  } catch (const BudgetOut&) {
    cudaStreamSynchronize(c.st);
    if (numConverged) *numConverged = 0;
    S.seconds_total = c.elapsed();
    S.kernel_launches = c.launches;
    S.precond_fallback = c.precond_fallback;
    if (stats) *stats = S;
    return SVDS_ERR_MAXIT;
  }
}

}  // namespace phsvds
