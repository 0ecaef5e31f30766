// Symmetric tridiagonal eigen-decomposition for the Gauss quadrature of SLQ.
//
// Stochastic Lanczos quadrature (Eq. 1 with M = I; Ubaru et al. 2017) needs,
// for each probe's Lanczos matrix T = U Lambda U^T, the eigenvalues lambda_j and
// the first components U_1j of the eigenvectors:
//     z^T log(Kh) z  ~  ||z||^2 sum_j U_1j^2 log(lambda_j).
// This is the implicit symmetric QR iteration with Wilkinson shifts on an
// unreduced tridiagonal window (Golub & Van Loan, Matrix Computations, §8.3),
// written for this library: Givens rotations chase the bulge down the window,
// and only the first row of the accumulated orthogonal factor is kept.
// FP64 throughout; m is at most a few dozen, one thread per probe.
#pragma once

#include <math.h>

namespace gp {

#ifdef __CUDACC__
#define GP_HD __host__ __device__ __forceinline__
#else
#define GP_HD inline
#endif

// c, s with [c s; -s c]^T [x; z] = [r; 0], r = sqrt(x^2 + z^2): c = x / r,
// s = -z / r from one reciprocal hypotenuse (an FP64 division or square root is
// a long dependent instruction sequence, and this sits on the serial path of
// every rotation).
GP_HD void givens_cs(double x, double z, double& c, double& s) {
  if (z == 0.0) {
    c = 1.0;
    s = 0.0;
    return;
  }
#ifdef __CUDA_ARCH__
  const double r = rhypot(x, z);
#else
  const double r = 1.0 / hypot(x, z);
#endif
  c = x * r;
  s = -z * r;
}

// a[0..m-1]: diagonal (overwritten by the eigenvalues); b[0..m-2]: off-diagonal
// (destroyed); q[0..m-1]: receives the first row of the eigenvector matrix.
// Returns false if the iteration cap was reached.
GP_HD bool tridiag_eig_first_row(double* a, double* b, double* q, int m) {
  const double eps = 1e-15;
  for (int j = 0; j < m; ++j) q[j] = (j == 0) ? 1.0 : 0.0;
  int hi = m - 1;
  int sweeps = 0;
  const int max_sweeps = 40 * (m > 0 ? m : 1);
  while (hi > 0) {
    if (fabs(b[hi - 1]) <= eps * (fabs(a[hi - 1]) + fabs(a[hi]))) {
      b[hi - 1] = 0.0;
      --hi;
      continue;
    }
    if (++sweeps > max_sweeps) return false;
    int lo = hi - 1;
    while (lo > 0 && fabs(b[lo - 1]) > eps * (fabs(a[lo - 1]) + fabs(a[lo]))) --lo;
    if (lo > 0) b[lo - 1] = 0.0;
    // Wilkinson shift: the eigenvalue of the trailing 2x2 closer to a[hi].
    const double dd = 0.5 * (a[hi - 1] - a[hi]);
    const double bb = b[hi - 1];
    const double den = dd + copysign(hypot(dd, bb), dd);
    const double mu = a[hi] - bb * bb / den;
    double x = a[lo] - mu;
    double z = b[lo];
    for (int k = lo; k < hi; ++k) {
      double c, s;
      givens_cs(x, z, c, s);
      if (k > lo) b[k - 1] = c * x - s * z;
      const double p = a[k], r = a[k + 1], e = b[k];
      const double cc = c * c, ss = s * s, cs = c * s;
      a[k] = cc * p - 2.0 * cs * e + ss * r;
      a[k + 1] = ss * p + 2.0 * cs * e + cc * r;
      b[k] = cs * (p - r) + (cc - ss) * e;
      if (k + 1 < hi) {
        z = -s * b[k + 1];
        b[k + 1] = c * b[k + 1];
        x = b[k];
      }
      const double q0 = q[k], q1 = q[k + 1];
      q[k] = c * q0 - s * q1;
      q[k + 1] = s * q0 + c * q1;
    }
  }
  return true;
}

// Gauss quadrature of log from one probe's Lanczos coefficients: T has
// diagonal alpha[0..m-1] and off-diagonal beta[0..m-2] (read with stride
// `stride`).  Returns ||z||^2 * sum_j U_1j^2 log(lambda_j); sets *ok = false on
// a non-positive eigenvalue or a non-converged eigen-iteration.
GP_HD double lanczos_logquad(const double* alpha, const double* beta, int stride, int m,
                             double znorm2, double* a, double* b, double* q, bool* ok) {
  *ok = true;
  if (m <= 0) return 0.0;
  for (int j = 0; j < m; ++j) {
    a[j] = alpha[j * stride];
    if (j + 1 < m) b[j] = beta[j * stride];
  }
  if (!tridiag_eig_first_row(a, b, q, m)) *ok = false;
  double acc = 0.0;
  for (int j = 0; j < m; ++j) {
    if (!(a[j] > 0.0)) {
      *ok = false;
      continue;
    }
    acc += q[j] * q[j] * log(a[j]);
  }
  return znorm2 * acc;
}

}  // namespace gp
