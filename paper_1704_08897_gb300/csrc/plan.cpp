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

// The mirror i -> n-1-i maps every second-difference matrix T of this file onto itself, so T has
// an eigenbasis whose vectors are each even (Q[n-1-i][k] = Q[i][k]) or odd (= -Q[i][k]) under it:
// the DCT-II and DST-I bases as they are (parity of k), and for the periodic rule the real Fourier
// basis sampled at i + 1/2 (cosines even, sines and the alternating vector odd), which spans the
// same eigenspaces as make_axis_basis's.  For r on the n nodes and an even column k,
// sum_i r[i] Q[i][k] = sum_{i<h} (r[i] + r[n-1-i]) Q[i][k] (r[i] alone at a middle node), and for an
// odd column the same with r[i] - r[n-1-i]; conversely E = Q_even c_even and O = Q_odd c_odd
// on the first h nodes give Q c = E + O there and E - O at the mirrored nodes.  So the transform
// pairs of one axis split into two of half size (Sec. 2.2's O(n log n) transforms rest on the same
// symmetry).
static void mirror_basis(int n, int bc, std::vector<double>& Q, std::vector<double>& lam,
                         std::vector<int>& odd) {
  if (bc != 1) {
    AxisBasis B = make_axis_basis(n, bc);
    Q = std::move(B.Q);
    lam = std::move(B.lam);
    odd.assign(n, 0);
    for (int k = 0; k < n; ++k) odd[k] = k & 1;
    return;
  }
  Q.assign((size_t)n * n, 0.0);
  lam.assign(n, 0.0);
  odd.assign(n, 0);
  auto at = [&](int i, int k) -> double& { return Q[(size_t)i * n + k]; };
  int col = 0;
  for (int i = 0; i < n; ++i) at(i, col) = std::sqrt(1.0 / n);
  lam[col++] = 0.0;
  for (int j = 1; 2 * j < n; ++j) {
    const double c = std::sqrt(2.0 / n);
    for (int i = 0; i < n; ++i) {
      // angle 2 pi j (i + 1/2) / n = pi * j (2i + 1) / n
      at(i, col) = c * cospi_frac((int64_t)j * (2 * i + 1), n);
      at(i, col + 1) = c * sinpi_frac((int64_t)j * (2 * i + 1), n);
    }
    const double l = 2.0 - 2.0 * cospi_frac(2 * (int64_t)j, n);
    lam[col] = l;
    lam[col + 1] = l;
    odd[col + 1] = 1;
    col += 2;
  }
  if (n % 2 == 0) {
    for (int i = 0; i < n; ++i) at(i, col) = ((i & 1) ? -1.0 : 1.0) * std::sqrt(1.0 / n);
    lam[col] = 4.0;
    odd[col++] = 1;
  }
}

int mirror_half(int n) { return (n + 1) / 2; }

bool mirror_pays(int n, int pad) { return 2 * pad_to(mirror_half(n), pad) <= pad_to(n, pad); }

AxisBasis make_class_basis(int n, int bc, int cls) {
  std::vector<double> Qf, lf;
  std::vector<int> odd;
  mirror_basis(n, bc, Qf, lf, odd);
  const int h = mirror_half(n);
  AxisBasis B;
  B.n = h;
  B.bc = bc;
  B.Q.assign((size_t)h * h, 0.0);
  B.lam.assign(h, 0.0);  // columns beyond the class's modes stay zero
  int j = 0;
  for (int k = 0; k < n; ++k) {
    if (odd[k] != cls) continue;
    for (int i = 0; i < h; ++i) B.Q[(size_t)i * h + j] = Qf[(size_t)i * n + k];
    B.lam[j++] = lf[k];
  }
  // the middle node of an odd n is its own mirror: odd vectors vanish there
  if (cls == 1 && (n & 1))
    for (int jj = 0; jj < h; ++jj) B.Q[(size_t)(h - 1) * h + jj] = 0.0;
  return B;
}

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
