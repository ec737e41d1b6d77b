// Host-side construction of the per-axis transform bases (internal).
#pragma once

#include <vector>

namespace bx {

struct AxisBasis {
  int n = 0, bc = 0;
  std::vector<double> Q;    // [n][n], Q[i][k] = k-th orthonormal eigenvector at node i
  std::vector<double> lam;  // eigenvalue of column k (h = 1)
};

AxisBasis make_axis_basis(int n, int bc);
int pad_to(int n, int m);
// Zero-padded np x np double-float copies of Q and Q^T (row-major): the hi plane, then the lo
// plane (the FP64 entry minus its FP32 rounding).
void padded_df(const AxisBasis& B, int np, std::vector<float>& q, std::vector<float>& qt);

}  // namespace bx
