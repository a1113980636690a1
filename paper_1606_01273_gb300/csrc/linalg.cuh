// FP64 dense helpers (internal): GEMM and symmetric eigensolver.
#pragma once
#include <algorithm>

#include "common.cuh"

namespace caspt2 {

// Row-major C = alpha * op(A) op(B) + beta * C, op = transpose when the flag is set.
// Batched over `batch` with element strides sA, sB, sC.
cudaError_t dgemm(int M, int N, int K, double alpha, const double* A, int lda, bool ta,
                  const double* B, int ldb, bool tb, double beta, double* C, int ldc,
                  cudaStream_t s, int batch = 1, long sA = 0, long sB = 0, long sC = 0);

// Eigenpairs of a symmetric m x m matrix by parallel cyclic Jacobi.  A is destroyed
// (left holding the diagonalised matrix); w[m] eigenvalues (unsorted), V[m][m] with
// eigenvectors as columns; work >= 2*m*m + 2 doubles.  Returns CASPT2_OK, ENOTCONV,
// ENAN or ECUDA.  Synchronises the stream once per sweep.
int sym_eig_jacobi(double* A, int m, double* w, double* V, double* work, cudaStream_t s);

}  // namespace caspt2
