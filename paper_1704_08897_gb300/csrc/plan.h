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
// Mirror classes of an axis (i -> n-1-i): h = ceil(n/2) nodes per class; cls 0 = the even vectors,
// 1 = the odd ones, each an h x h basis (zero columns where the class has fewer than h modes) with
// its eigenvalues in ascending order.
int mirror_half(int n);
bool mirror_pays(int n, int pad);  // both classes padded fit in the padded axis
AxisBasis make_class_basis(int n, int bc, int cls);
// Zero-padded np x np double-float copies of Q and Q^T (row-major): the hi plane, then the lo
// plane (the FP64 entry minus its FP32 rounding).
void padded_df(const AxisBasis& B, int np, std::vector<float>& q, std::vector<float>& qt);

}  // namespace bx
