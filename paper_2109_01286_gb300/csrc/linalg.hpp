// Dense FP64 linear algebra and host threading shared by the 2D and 3D preprocessing: a
// work-sharing parallel loop, Hestenes' one-sided Jacobi SVD, Householder QR with column
// pivoting for rows of a least-squares pseudo-inverse, the minimum-norm pseudo-inverse by SVD,
// and Dekker's double-double arithmetic.
#pragma once
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <thread>
#include <vector>

#include "hfd.h"

namespace hfd {

template <class F>
inline void parallel_for(int64_t n, int nthreads, F f) {
  if (nthreads <= 1 || n < 256) {
    for (int64_t i = 0; i < n; ++i) f(i, 0);
    return;
  }
  std::atomic<int64_t> next(0);
  const int64_t chunk = 64;
  std::vector<std::thread> th;
  for (int t = 0; t < nthreads; ++t)
    th.emplace_back([&, t] {
      for (;;) {
        int64_t s = next.fetch_add(chunk);
        if (s >= n) break;
        int64_t e = std::min(n, s + chunk);
        for (int64_t i = s; i < e; ++i) f(i, t);
      }
    });
  for (auto& x : th) x.join();
}

// ------------------------------------------------------------------ one-sided Jacobi SVD
// Hestenes' method on the columns of A (m x n, column-major): A V = U diag(s).  On return A
// holds U diag(s) (columns sorted by decreasing s), V the right singular vectors.
inline void jacobi_svd(int m, int n, double* A, double* V, double* s) {
  for (int i = 0; i < n * n; ++i) V[i] = 0.0;
  for (int i = 0; i < n; ++i) V[i + i * n] = 1.0;
  for (int sweep = 0; sweep < 80; ++sweep) {
    bool rotated = false;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        double al = 0, be = 0, ga = 0;
        double* ap = A + (size_t)p * m;
        double* aq = A + (size_t)q * m;
        for (int i = 0; i < m; ++i) {
          al += ap[i] * ap[i];
          be += aq[i] * aq[i];
          ga += ap[i] * aq[i];
        }
        if (al == 0.0 || be == 0.0) continue;
        if (std::fabs(ga) <= 1e-16 * std::sqrt(al * be)) continue;
        rotated = true;
        double zeta = (be - al) / (2.0 * ga);
        double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
        double c = 1.0 / std::sqrt(1.0 + t * t), sn = c * t;
        for (int i = 0; i < m; ++i) {
          double u = ap[i], w = aq[i];
          ap[i] = c * u - sn * w;
          aq[i] = sn * u + c * w;
        }
        double* vp = V + (size_t)p * n;
        double* vq = V + (size_t)q * n;
        for (int i = 0; i < n; ++i) {
          double u = vp[i], w = vq[i];
          vp[i] = c * u - sn * w;
          vq[i] = sn * u + c * w;
        }
      }
    if (!rotated) break;
  }
  std::vector<int> ord(n);
  for (int j = 0; j < n; ++j) {
    double t = 0;
    for (int i = 0; i < m; ++i) t += A[i + (size_t)j * m] * A[i + (size_t)j * m];
    s[j] = std::sqrt(t);
    ord[j] = j;
  }
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return s[a] > s[b]; });
  std::vector<double> A2((size_t)m * n), V2((size_t)n * n), s2(n);
  for (int j = 0; j < n; ++j) {
    std::memcpy(&A2[(size_t)j * m], A + (size_t)ord[j] * m, sizeof(double) * m);
    std::memcpy(&V2[(size_t)j * n], V + (size_t)ord[j] * n, sizeof(double) * n);
    s2[j] = s[ord[j]];
  }
  std::memcpy(A, A2.data(), sizeof(double) * m * n);
  std::memcpy(V, V2.data(), sizeof(double) * n * n);
  std::memcpy(s, s2.data(), sizeof(double) * n);
}

// ------------------------------------------------------------------ Householder QR (pivoted)
// Rows of the pseudo-inverse of a full-column-rank A (m x n, column-major): for each target
// pair (i1, i2) the row (e_i1 + e_i2)^T A^+ (i2 < 0: e_i1 only).  A P = Q R, so the row is
// Q z with R^T z = P^T e.  Returns |R_nn| / |R_11| as the conditioning estimate.
inline double ls_rows(int m, int n, std::vector<double>& A, const int (*targets)[2], int ntarg,
                      double* rows /* ntarg x m */) {
  std::vector<int> perm(n);
  for (int j = 0; j < n; ++j) perm[j] = j;
  std::vector<double> beta(n, 0.0), v0s(n, 0.0);
  auto col = [&](int j) { return &A[(size_t)j * m]; };
  for (int k = 0; k < n; ++k) {
    int best = k;
    double bn = -1;
    for (int j = k; j < n; ++j) {
      double t = 0;
      const double* c = col(j);
      for (int i = k; i < m; ++i) t += c[i] * c[i];
      if (t > bn) { bn = t; best = j; }
    }
    if (best != k) {
      std::swap_ranges(col(k), col(k) + m, col(best));
      std::swap(perm[k], perm[best]);
    }
    double* c = col(k);
    double nx = std::sqrt(bn);
    if (nx == 0.0) { beta[k] = 0.0; continue; }
    double alpha = c[k] >= 0 ? -nx : nx;
    double v0 = c[k] - alpha;
    // v = (v0, c[k+1..m-1]); v^T v = 2 (nx^2 - alpha c[k])
    double vtv = v0 * v0;
    for (int i = k + 1; i < m; ++i) vtv += c[i] * c[i];
    double b = 2.0 / vtv;
    for (int j = k + 1; j < n; ++j) {
      double* cj = col(j);
      double dot = v0 * cj[k];
      for (int i = k + 1; i < m; ++i) dot += c[i] * cj[i];
      dot *= b;
      cj[k] -= dot * v0;
      for (int i = k + 1; i < m; ++i) cj[i] -= dot * c[i];
    }
    c[k] = alpha;          // R_kk; the reflector tail stays below the diagonal
    beta[k] = b;
    v0s[k] = v0;
  }
  double r11 = std::fabs(A[0]), rnn = std::fabs(A[(size_t)(n - 1) * m + (n - 1)]);
  std::vector<double> f(n), z(n), yv(m);
  for (int t = 0; t < ntarg; ++t) {
    for (int k = 0; k < n; ++k) {
      int j = perm[k];
      f[k] = (j == targets[t][0] ? 1.0 : 0.0) + (j == targets[t][1] ? 1.0 : 0.0);
    }
    for (int k = 0; k < n; ++k) {           // R^T z = f (forward substitution)
      double acc = f[k];
      for (int i = 0; i < k; ++i) acc -= A[(size_t)k * m + i] * z[i];
      z[k] = acc / A[(size_t)k * m + k];
    }
    for (int i = 0; i < m; ++i) yv[i] = i < n ? z[i] : 0.0;
    for (int k = n - 1; k >= 0; --k) {      // y = H_0 ... H_{n-1} [z; 0]
      const double* c = col(k);
      double dot = v0s[k] * yv[k];
      for (int i = k + 1; i < m; ++i) dot += c[i] * yv[i];
      dot *= beta[k];
      yv[k] -= dot * v0s[k];
      for (int i = k + 1; i < m; ++i) yv[i] -= dot * c[i];
    }
    std::memcpy(rows + (size_t)t * m, yv.data(), sizeof(double) * m);
  }
  return rnn / r11;
}

// Minimum-norm rows e_t^T A^+ of a possibly rank-deficient A (m x n, column-major) by the
// one-sided Jacobi SVD of A (singular values <= max(m, n) * eps * sigma_max count as zero, the
// convention of numpy's pinv): A^+ = V diag(1/s) U^T with U diag(s) = A V.
inline void pinv_rows_svd(int m, int n, const std::vector<double>& A, const int* targets,
                          int ntarg, double* rows /* ntarg x m */) {
  std::vector<double> W(A), V((size_t)n * n), s(n);
  jacobi_svd(m, n, W.data(), V.data(), s.data());
  double tol = std::max(m, n) * 2.220446049250313e-16 * s[0];
  for (int t = 0; t < ntarg; ++t) {
    double* r = rows + (size_t)t * m;
    for (int i = 0; i < m; ++i) r[i] = 0.0;
    for (int k = 0; k < n; ++k) {
      if (!(s[k] > tol)) break;
      double f = V[targets[t] + (size_t)k * n] / (s[k] * s[k]);   // V[t,k] U[:,k] / s_k
      for (int i = 0; i < m; ++i) r[i] += f * W[i + (size_t)k * m];
    }
  }
}

// ------------------------------------------------------------------ double-double (Dekker)
struct dd { double hi, lo; };
inline dd two_sum(double a, double b) {
  double s = a + b, bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
inline dd quick_two_sum(double a, double b) {
  double s = a + b;
  return {s, b - (s - a)};
}
inline dd two_prod(double a, double b) {
  double p = a * b;
  return {p, std::fma(a, b, -p)};
}
inline dd dd_add(dd x, dd y) {
  dd s = two_sum(x.hi, y.hi), t = two_sum(x.lo, y.lo);
  s.lo += t.hi;
  s = quick_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return quick_two_sum(s.hi, s.lo);
}
inline dd dd_neg(dd x) { return {-x.hi, -x.lo}; }
inline dd dd_mul(dd x, dd y) {
  dd p = two_prod(x.hi, y.hi);
  p.lo += x.hi * y.lo + x.lo * y.hi;
  return quick_two_sum(p.hi, p.lo);
}
inline dd dd_from(double a) { return {a, 0.0}; }
inline dd dd_div(dd a, dd b) {          // long division, three quotient terms
  double q1 = a.hi / b.hi;
  dd r = dd_add(a, dd_neg(dd_mul(dd_from(q1), b)));
  double q2 = r.hi / b.hi;
  r = dd_add(r, dd_neg(dd_mul(dd_from(q2), b)));
  double q3 = r.hi / b.hi;
  dd q = quick_two_sum(q1, q2);
  return dd_add(q, dd_from(q3));
}

// The first error raised by any worker of a parallel loop.
struct ErrorSlot {
  std::mutex mu;
  hfd_status st = HFD_OK;
  char msg[512] = "";
  void set(hfd_status s, const char* m) {
    std::lock_guard<std::mutex> g(mu);
    if (st == HFD_OK) {
      st = s;
      snprintf(msg, sizeof msg, "%s", m);
    }
  }
};

}  // namespace hfd
