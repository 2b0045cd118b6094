// Small dense symmetric eigensolver (host, FP64) for the projected
// Lanczos matrix and the b x b Gram matrices of the block QR.
//
// Method (Golub & Van Loan, "Matrix Computations", Sec. 8.3): Householder
// reduction to tridiagonal form, accumulating the reflections, then the
// implicit symmetric QR iteration with Wilkinson shifts and Givens
// rotations, deflating negligible off-diagonal entries.
#pragma once

#include <vector>

namespace ci {

// A: n x n row-major symmetric (only read).  On return w holds the
// eigenvalues ascending and Z (n x n row-major) the eigenvectors as
// columns: A Z[:,i] = w[i] Z[:,i].  Returns false if the QR iteration did
// not converge.
bool sym_eig(int n, const std::vector<double> &A, std::vector<double> &w, std::vector<double> &Z);

}  // namespace ci
