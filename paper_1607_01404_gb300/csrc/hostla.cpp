// Small dense FP64 linear algebra on the host; see hostla.h.
#include "hostla.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

namespace phsvds {
namespace hla {

namespace {
inline double& at(double* A, int n, int i, int j) { return A[(size_t)j * n + i]; }
inline double at(const double* A, int n, int i, int j) { return A[(size_t)j * n + i]; }
}  // namespace

bool sym_eig(int n, const double* Ain, double* w, double* Z) {
  if (n == 0) return true;
  std::vector<double> A(Ain, Ain + (size_t)n * n);
  // symmetrise from the lower triangle
  for (int j = 0; j < n; ++j)
    for (int i = j + 1; i < n; ++i) {
      double v = 0.5 * (at(A.data(), n, i, j) + at(A.data(), n, j, i));
      at(A.data(), n, i, j) = v;
      at(A.data(), n, j, i) = v;
    }
  // Z = I
  std::fill(Z, Z + (size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) at(Z, n, i, i) = 1.0;
  // --- Householder tridiagonalisation: A <- H A H with H = I - beta v v^T ---
  std::vector<double> v(n), p(n), q(n);
  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - k - 1;  // length of the column below the diagonal
    double alpha = 0.0;
    for (int i = 0; i < m; ++i) alpha += at(A.data(), n, k + 1 + i, k) * at(A.data(), n, k + 1 + i, k);
    alpha = std::sqrt(alpha);
    if (alpha == 0.0) continue;
    const double x0 = at(A.data(), n, k + 1, k);
    const double s = x0 >= 0 ? -alpha : alpha;  // target value of the first entry
    for (int i = 0; i < m; ++i) v[i] = at(A.data(), n, k + 1 + i, k);
    v[0] -= s;
    double vnorm2 = 0.0;
    for (int i = 0; i < m; ++i) vnorm2 += v[i] * v[i];
    if (vnorm2 == 0.0) continue;
    const double beta = 2.0 / vnorm2;
    // p = beta * A22 v
    for (int i = 0; i < m; ++i) {
      double acc = 0.0;
      for (int j = 0; j < m; ++j) acc += at(A.data(), n, k + 1 + i, k + 1 + j) * v[j];
      p[i] = beta * acc;
    }
    double pv = 0.0;
    for (int i = 0; i < m; ++i) pv += p[i] * v[i];
    const double c = 0.5 * beta * pv;
    for (int i = 0; i < m; ++i) q[i] = p[i] - c * v[i];
    // A22 <- A22 - v q^T - q v^T
    for (int j = 0; j < m; ++j)
      for (int i = 0; i < m; ++i)
        at(A.data(), n, k + 1 + i, k + 1 + j) -= v[i] * q[j] + q[i] * v[j];
    at(A.data(), n, k + 1, k) = s;
    at(A.data(), n, k, k + 1) = s;
    for (int i = 1; i < m; ++i) {
      at(A.data(), n, k + 1 + i, k) = 0.0;
      at(A.data(), n, k, k + 1 + i) = 0.0;
    }
    // Z <- Z H  (columns k+1 .. n-1)
    for (int r = 0; r < n; ++r) {
      double acc = 0.0;
      for (int i = 0; i < m; ++i) acc += at(Z, n, r, k + 1 + i) * v[i];
      acc *= beta;
      for (int i = 0; i < m; ++i) at(Z, n, r, k + 1 + i) -= acc * v[i];
    }
  }
  std::vector<double> d(n), e(n, 0.0);
  for (int i = 0; i < n; ++i) d[i] = at(A.data(), n, i, i);
  for (int i = 0; i + 1 < n; ++i) e[i] = at(A.data(), n, i + 1, i);
  // --- implicit symmetric QR with Wilkinson shift on (d, e) ---
  const double eps = 2.220446049250313e-16;
  int hi = n - 1;
  int iter = 0;
  const int maxiter = 60 * n;
  while (hi > 0) {
    if (std::fabs(e[hi - 1]) <= eps * (std::fabs(d[hi - 1]) + std::fabs(d[hi])) || e[hi - 1] == 0.0) {
      e[hi - 1] = 0.0;
      --hi;
      continue;
    }
    int lo = hi - 1;
    while (lo > 0 && std::fabs(e[lo - 1]) > eps * (std::fabs(d[lo - 1]) + std::fabs(d[lo]))) --lo;
    if (++iter > maxiter) return false;
    // Wilkinson shift from the trailing 2x2 block
    const double dd = 0.5 * (d[hi - 1] - d[hi]);
    const double eh = e[hi - 1];
    const double den = dd + (dd >= 0 ? 1.0 : -1.0) * std::hypot(dd, eh);
    const double mu = d[hi] - eh * eh / den;
    double x = d[lo] - mu;
    double z = e[lo];
    for (int k = lo; k < hi; ++k) {
      // Givens rotation zeroing z against x
      double c, s;
      if (z == 0.0) {
        c = 1.0;
        s = 0.0;
      } else {
        const double r = std::hypot(x, z);
        c = x / r;
        s = -z / r;
      }
      // T <- G^T T G on rows/cols k, k+1 (G = [c s; -s c])
      if (k > lo) e[k - 1] = c * e[k - 1] - s * z;
      const double dk = d[k], dk1 = d[k + 1], ek = e[k];
      const double a = c * dk - s * ek;
      const double b = c * ek - s * dk1;
      d[k] = c * a - s * b;
      e[k] = s * a + c * b;
      const double a2 = s * dk + c * ek;
      const double b2 = s * ek + c * dk1;
      d[k + 1] = s * a2 + c * b2;
      if (k + 1 < hi) {
        x = e[k];
        z = -s * e[k + 1];
        e[k + 1] = c * e[k + 1];
      }
      for (int r = 0; r < n; ++r) {
        const double zk = at(Z, n, r, k), zk1 = at(Z, n, r, k + 1);
        at(Z, n, r, k) = c * zk - s * zk1;
        at(Z, n, r, k + 1) = s * zk + c * zk1;
      }
    }
  }
  // sort ascending
  std::vector<int> idx(n);
  std::iota(idx.begin(), idx.end(), 0);
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return d[a] < d[b]; });
  std::vector<double> Zs((size_t)n * n);
  for (int j = 0; j < n; ++j) {
    w[j] = d[idx[j]];
    std::memcpy(&Zs[(size_t)j * n], &Z[(size_t)idx[j] * n], sizeof(double) * n);
  }
  std::memcpy(Z, Zs.data(), sizeof(double) * (size_t)n * n);
  return true;
}

bool svd_right(int n, const double* R, double* s, double* Yr) {
  std::vector<double> Wm(R, R + (size_t)n * n);
  std::fill(Yr, Yr + (size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) at(Yr, n, i, i) = 1.0;
  const double eps = 2.220446049250313e-16;
  bool conv = false;
  for (int sweep = 0; sweep < 60 && !conv; ++sweep) {
    conv = true;
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j) {
        double a = 0, b = 0, g = 0;
        for (int r = 0; r < n; ++r) {
          const double wi = at(Wm.data(), n, r, i), wj = at(Wm.data(), n, r, j);
          a += wi * wi;
          b += wj * wj;
          g += wi * wj;
        }
        if (std::fabs(g) <= eps * std::sqrt(a * b) || g == 0.0) continue;
        conv = false;
        const double zeta = (b - a) / (2.0 * g);
        const double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / std::sqrt(1.0 + t * t), sn = c * t;
        for (int r = 0; r < n; ++r) {
          const double wi = at(Wm.data(), n, r, i), wj = at(Wm.data(), n, r, j);
          at(Wm.data(), n, r, i) = c * wi - sn * wj;
          at(Wm.data(), n, r, j) = sn * wi + c * wj;
          const double yi = at(Yr, n, r, i), yj = at(Yr, n, r, j);
          at(Yr, n, r, i) = c * yi - sn * yj;
          at(Yr, n, r, j) = sn * yi + c * yj;
        }
      }
  }
  std::vector<double> sv(n);
  for (int j = 0; j < n; ++j) {
    double a = 0;
    for (int r = 0; r < n; ++r) a += at(Wm.data(), n, r, j) * at(Wm.data(), n, r, j);
    sv[j] = std::sqrt(a);
  }
  std::vector<int> idx(n);
  std::iota(idx.begin(), idx.end(), 0);
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return sv[a] < sv[b]; });
  std::vector<double> Ys((size_t)n * n);
  for (int j = 0; j < n; ++j) {
    s[j] = sv[idx[j]];
    std::memcpy(&Ys[(size_t)j * n], &Yr[(size_t)idx[j] * n], sizeof(double) * n);
  }
  std::memcpy(Yr, Ys.data(), sizeof(double) * (size_t)n * n);
  return conv;
}

bool chol_upper(int n, const double* G, double* R) {
  std::fill(R, R + (size_t)n * n, 0.0);
  for (int j = 0; j < n; ++j) {
    double s = at(G, n, j, j);
    for (int k = 0; k < j; ++k) s -= at(R, n, k, j) * at(R, n, k, j);
    if (!(s > 0.0) || !std::isfinite(s)) return false;
    const double rjj = std::sqrt(s);
    at(R, n, j, j) = rjj;
    for (int i = j + 1; i < n; ++i) {
      double t = 0.5 * (at(G, n, j, i) + at(G, n, i, j));
      for (int k = 0; k < j; ++k) t -= at(R, n, k, j) * at(R, n, k, i);
      at(R, n, j, i) = t / rjj;
    }
  }
  return true;
}

void tri_inv_upper(int n, const double* R, double* Ri) {
  std::fill(Ri, Ri + (size_t)n * n, 0.0);
  for (int j = 0; j < n; ++j) {
    at(Ri, n, j, j) = 1.0 / at(R, n, j, j);
    for (int i = j - 1; i >= 0; --i) {
      double s = 0.0;
      for (int k = i + 1; k <= j; ++k) s += at(R, n, i, k) * at(Ri, n, k, j);
      at(Ri, n, i, j) = -s / at(R, n, i, i);
    }
  }
}

int orth_cols(int n, int c, double* Y, double tol) {
  int kept = 0;
  for (int j = 0; j < c; ++j) {
    double* y = Y + (size_t)j * n;
    double n0 = 0;
    for (int r = 0; r < n; ++r) n0 += y[r] * y[r];
    n0 = std::sqrt(n0);
    for (int pass = 0; pass < 2; ++pass)
      for (int k = 0; k < kept; ++k) {
        const double* q = Y + (size_t)k * n;
        double d = 0;
        for (int r = 0; r < n; ++r) d += q[r] * y[r];
        for (int r = 0; r < n; ++r) y[r] -= d * q[r];
      }
    double nn = 0;
    for (int r = 0; r < n; ++r) nn += y[r] * y[r];
    nn = std::sqrt(nn);
    if (nn <= tol * std::max(n0, 1e-300) || nn == 0.0) continue;
    double* dst = Y + (size_t)kept * n;
    for (int r = 0; r < n; ++r) dst[r] = y[r] / nn;
    ++kept;
  }
  return kept;
}

void gemm_tn(int m, int n, int k, const double* A, int lda, const double* B, int ldb, double* C, int ldc) {
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < m; ++i) {
      double s = 0;
      for (int l = 0; l < k; ++l) s += A[(size_t)i * lda + l] * B[(size_t)j * ldb + l];
      C[(size_t)j * ldc + i] = s;
    }
}

void gemm_nn(int m, int n, int k, const double* A, int lda, const double* B, int ldb, double* C, int ldc) {
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < m; ++i) {
      double s = 0;
      for (int l = 0; l < k; ++l) s += A[(size_t)l * lda + i] * B[(size_t)j * ldb + l];
      C[(size_t)j * ldc + i] = s;
    }
}

}  // namespace hla
}  // namespace phsvds
