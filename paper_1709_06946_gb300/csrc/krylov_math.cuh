// Small dense FP64 algebra of the Krylov iterations, compiled for the host and
// the device (the device copy runs inside the Lanczos control kernel).
#pragma once

#include <cuda_runtime.h>
#include <math.h>

namespace pse {

// Symmetric tridiagonal eigen-decomposition by the implicit QL method with
// shifts from the leading 2x2 block (Wilkinson).  d[0..n): diagonal, replaced
// by the eigenvalues; e[0..n): off-diagonal in e[0..n-1), destroyed; Z: n x n
// row-major, Z[i*n+k] = component i of eigenvector k.  Returns false when an
// eigenvalue needs more than 100 sweeps.
__host__ __device__ inline bool tql_eigen(int n, double *d, double *e, double *Z) {
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k) Z[i * n + k] = i == k ? 1.0 : 0.0;
  if (n > 0) e[n - 1] = 0.0;
  const double eps = 2.220446049250313e-16;
  for (int l = 0; l < n; ++l) {
    for (int iter = 0;; ++iter) {
      int m = l;
      for (; m < n - 1; ++m) {
        double dd = fabs(d[m]) + fabs(d[m + 1]);
        if (fabs(e[m]) <= eps * dd) break;
      }
      if (m == l) break;
      if (iter > 100) return false;
      double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
      double rr = hypot(g, 1.0);
      g = d[m] - d[l] + e[l] / (g + (g >= 0 ? rr : -rr));
      double s = 1.0, c = 1.0, pp = 0.0;
      bool deflated = false;
      for (int i = m - 1; i >= l; --i) {
        double f = s * e[i], b = c * e[i];
        rr = hypot(f, g);
        e[i + 1] = rr;
        if (rr == 0.0) {  // underflow: split the problem
          d[i + 1] -= pp;
          e[m] = 0.0;
          deflated = true;
          break;
        }
        s = f / rr;
        c = g / rr;
        g = d[i + 1] - pp;
        rr = (d[i] - g) * s + 2.0 * c * b;
        pp = s * rr;
        d[i + 1] = g + pp;
        g = c * rr - b;
        for (int k = 0; k < n; ++k) {  // rotate columns i, i+1 of Z
          double zf = Z[k * n + i + 1];
          Z[k * n + i + 1] = s * Z[k * n + i] + c * zf;
          Z[k * n + i] = c * Z[k * n + i] - s * zf;
        }
      }
      if (deflated) continue;
      d[l] -= pp;
      e[l] = g;
      e[m] = 0.0;
    }
  }
  return true;
}

// cvec = T^{1/2} e1 for the symmetric tridiagonal T = tridiag(beta, alpha, beta)
// of order n (eigenvalues clamped at zero); work: 2n + n^2 doubles.
__host__ __device__ inline bool tridiag_sqrt_e1(int n, const double *alpha, const double *beta, double *work,
                                                double *cvec) {
  double *d = work, *e = work + n, *Z = work + 2 * n;
  for (int i = 0; i < n; ++i) {
    d[i] = alpha[i];
    e[i] = i < n - 1 ? beta[i] : 0.0;
  }
  if (!tql_eigen(n, d, e, Z)) return false;
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    for (int k = 0; k < n; ++k) s += Z[i * n + k] * sqrt(d[k] > 0.0 ? d[k] : 0.0) * Z[k];
    cvec[i] = s;
  }
  return true;
}

}  // namespace pse
