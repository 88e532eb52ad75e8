// The Davidson subspace eigenproblem and the biorthonormalisation inverse on the GPU (FP64,
// subspace.cu): one warp per small dense problem.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

namespace ccsd {

// Bytes of device scratch launch_subspace_step needs for an m x m subspace matrix.
size_t subspace_work_bytes(int m);

// The subspace step of a block Davidson solve for the projected matrix G (m x m, row-major,
// leading dimension ldg, device): all eigenvalues (Hessenberg reduction and shifted QR in
// complex arithmetic), sorted by real part; the wanted nroots are the lowest, or, with
// targets (device, nroots values), the ones nearest each target.  out (device) receives
//   out[k]                       Re omega_k
//   out[nroots + k]              Im omega_k
//   out[2 nroots + i nroots + k] coefficient i of the Ritz vector of root k (U[m][nroots]):
//                                the real eigenvector by inverse iteration, or, for the second
//                                member of a complex pair a +- ib, (G - a) u of the first
//                                member's vector u, both spanning the pair's real invariant
//                                subspace
//   out[2 nroots + m nroots]     the largest |eigenvalue|
// work: subspace_work_bytes(m) bytes of device scratch.
void launch_subspace_step(int m, const double* G, int ldg, int nroots, const double* targets, double* out, void* work,
                          cudaStream_t st);

// Bytes of device scratch launch_small_inverse needs for an n x n matrix.
size_t small_inverse_work_bytes(int n);

// Ainv = A^-1 (n x n, row-major, device) by LU with partial pivoting; flag[0] = 1 (device) if A
// is singular.
void launch_small_inverse(int n, const double* A, double* Ainv, int* flag, void* work, cudaStream_t st);

}  // namespace ccsd
