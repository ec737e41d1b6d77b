// Transform plans of the fast Poisson preconditioner (Algorithm 1 uses sine transforms for
// Dirichlet edges; Example 1 replaces them by cosine transforms for Neumann edges; Example 2 by
// discrete Fourier transforms for periodic edges).  Each axis gets a dense orthonormal
// eigenvector matrix Q of its 1-D second difference T (T = Q diag(lambda) Q^T), built in FP64 on
// the host with exact integer argument reduction, padded with zeros to a multiple of 128 and
// rounded once to the storage type.
#include "plan.h"

#include <cmath>
#include <cstdint>

namespace bx {

static const double kPi = 3.14159265358979323846;

// cos(pi * m / d) and sin(pi * m / d) with m reduced modulo 2d first.
static double cospi_frac(int64_t m, int64_t d) {
  m %= 2 * d;
  if (m < 0) m += 2 * d;
  return std::cos(kPi * (double)m / (double)d);
}
static double sinpi_frac(int64_t m, int64_t d) {
  m %= 2 * d;
  if (m < 0) m += 2 * d;
  return std::sin(kPi * (double)m / (double)d);
}

AxisBasis make_axis_basis(int n, int bc) {
  AxisBasis B;
  B.n = n;
  B.bc = bc;
  B.Q.assign((size_t)n * n, 0.0);
  B.lam.assign(n, 0.0);
  auto Q = [&](int i, int k) -> double& { return B.Q[(size_t)i * n + k]; };
  if (bc == 0) {  // symmetric: DCT-II basis, T with T[0][0] = T[n-1][n-1] = 1
    for (int k = 0; k < n; ++k) {
      const double c = (k == 0) ? std::sqrt(1.0 / n) : std::sqrt(2.0 / n);
      for (int i = 0; i < n; ++i) Q(i, k) = c * cospi_frac((int64_t)k * (2 * i + 1), 2 * (int64_t)n);
      B.lam[k] = 2.0 - 2.0 * cospi_frac(k, n);
    }
  } else if (bc == 1) {  // periodic: real Fourier basis (constant, cos/sin pairs, Nyquist)
    int col = 0;
    for (int i = 0; i < n; ++i) Q(i, col) = std::sqrt(1.0 / n);
    B.lam[col++] = 0.0;
    for (int j = 1; 2 * j < n; ++j) {
      const double c = std::sqrt(2.0 / n);
      for (int i = 0; i < n; ++i) {
        Q(i, col) = c * cospi_frac(2 * (int64_t)j * i, n);
        Q(i, col + 1) = c * sinpi_frac(2 * (int64_t)j * i, n);
      }
      const double l = 2.0 - 2.0 * cospi_frac(2 * (int64_t)j, n);
      B.lam[col] = l;
      B.lam[col + 1] = l;
      col += 2;
    }
    if (n % 2 == 0) {
      for (int i = 0; i < n; ++i) Q(i, col) = ((i & 1) ? -1.0 : 1.0) * std::sqrt(1.0 / n);
      B.lam[col++] = 4.0;
    }
  } else {  // Dirichlet: DST-I basis, T = tridiag(-1, 2, -1)
    const double c = std::sqrt(2.0 / (n + 1));
    for (int k = 0; k < n; ++k) {
      for (int i = 0; i < n; ++i) Q(i, k) = c * sinpi_frac((int64_t)(i + 1) * (k + 1), n + 1);
      B.lam[k] = 2.0 - 2.0 * cospi_frac(k + 1, n + 1);
    }
  }
  return B;
}

int pad_to(int n, int m) { return (n + m - 1) / m * m; }

void padded_df(const AxisBasis& B, int np, std::vector<float>& q, std::vector<float>& qt) {
  const size_t plane = (size_t)np * np;
  q.assign(2 * plane, 0.f);
  qt.assign(2 * plane, 0.f);
  for (int i = 0; i < B.n; ++i)
    for (int k = 0; k < B.n; ++k) {
      const double v = B.Q[(size_t)i * B.n + k];
      const float hi = (float)v, lo = (float)(v - (double)hi);
      q[(size_t)i * np + k] = hi;
      q[plane + (size_t)i * np + k] = lo;
      qt[(size_t)k * np + i] = hi;
      qt[plane + (size_t)k * np + i] = lo;
    }
}

}  // namespace bx
