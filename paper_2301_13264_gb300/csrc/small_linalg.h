// Small dense FP64 linear algebra for the solvers' subspace problems
// (DIIS equations, Davidson projected eigenproblem, biorthonormalisation).
#pragma once

#include <complex>
#include <vector>

namespace ccsd {

// Solve A x = b (n x n, row-major) by LU with partial pivoting; returns false if singular.
bool lu_solve(int n, std::vector<double> A, std::vector<double>& b);
// Inverse of a small matrix (row-major); returns false if singular.
bool invert(int n, const std::vector<double>& A, std::vector<double>& Ainv);
// All eigenvalues of a real n x n matrix (row-major): Hessenberg reduction and
// shifted QR iterations in complex arithmetic.
std::vector<std::complex<double>> eigenvalues(int n, const std::vector<double>& A);
// Right eigenvector for a real eigenvalue lam by inverse iteration; unit 2-norm.
std::vector<double> eigenvector(int n, const std::vector<double>& A, double lam);

}  // namespace ccsd
