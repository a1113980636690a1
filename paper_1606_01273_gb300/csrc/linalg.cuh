// FP64 dense helpers (internal): GEMM and symmetric eigensolver.
#pragma once
#include <vector>
#include <algorithm>

#include "common.cuh"

namespace caspt2 {

// Optional device-time accounting for one kernel (CUDA events on the launching stream).
struct KernelTimer {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  double ms = 0.0;       // summed device time
  double flops = 0.0;    // summed algorithmic flops
  double bytes = 0.0;    // summed algorithmic DRAM bytes
  long launches = 0;
  // the panel launches of the blocked reduction alone (k_latrd): an event pair per launch
  // (grown on demand, owned by the timer's holder), device time and the bytes of the
  // trailing matrix its matrix-vector products read (8 n1^2 per column)
  std::vector<cudaEvent_t> pev;
  double pms = 0.0, pbytes = 0.0;
  long plaunches = 0;
};

// Optional record of the FP64 GEMM launches of one host thread: an event pair around each
// launch (device time) and its algorithmic flops (2 M N K; the symmetric-output form its
// computed tiles).  Up to kGemmTimerPairs launches per collection; later ones run untimed.
constexpr int kGemmTimerPairs = 4096;
struct GemmTimer {
  cudaEvent_t ev[2 * kGemmTimerPairs] = {};
  double flops[kGemmTimerPairs] = {};
  int used = 0;
  bool ready = false;
};
cudaError_t gemm_timer_init(GemmTimer& t);
void gemm_timer_release(GemmTimer& t);
void set_gemm_timer(GemmTimer* t);   // this thread's dgemm launches are recorded (nullptr: off)
// Sum of the recorded launches (call after the stream has synchronised); resets the record.
cudaError_t gemm_timer_collect(GemmTimer& t, double* ms, double* flops, long* launches);

// Row-major C = alpha * op(A) op(B) + beta * C, op = transpose when the flag is set.
// Batched over `batch` with element strides sA, sB, sC.
cudaError_t dgemm(int M, int N, int K, double alpha, const double* A, int lda, bool ta,
                  const double* B, int ldb, bool tb, double beta, double* C, int ldc,
                  cudaStream_t s, int batch = 1, long sA = 0, long sB = 0, long sC = 0);
// Same product when the N x N result is known to be symmetric (A^T A, X^T F X): only the
// upper-triangle tiles are computed, each written to both triangles.
cudaError_t dgemm_sym(int N, int K, double alpha, const double* A, int lda, bool ta,
                      const double* B, int ldb, bool tb, double beta, double* C, int ldc,
                      cudaStream_t s);

// Eigenpairs of a symmetric m x m matrix by parallel cyclic Jacobi.  A is destroyed
// (left holding the diagonalised matrix); w[m] eigenvalues (ascending), V[m][m] with
// eigenvectors as columns; work >= 2*m*m + 2 doubles.  Returns CASPT2_OK, ENOTCONV,
// ENAN or ECUDA.  Synchronises the stream once per sweep.
int sym_eig_jacobi(double* A, int m, double* w, double* V, double* work, cudaStream_t s);

// Eigenpairs of a symmetric m x m matrix by Householder tridiagonalisation, bisection,
// inverse iteration and back-transformation (eig_tridiag.cu).  A is destroyed; w[m]
// ascending; V[m][m] eigenvectors as columns.  work >= sym_eig_tridiag_work(m) doubles.
size_t sym_eig_tridiag_work(int m);
// oz (optional, on): the Newton-Schulz correction Z (1/2)(I - Z^T Z), a term of the size of
// the orthogonality error, runs as a split-BF16 product with just enough slices.
struct OzWork;
int sym_eig_tridiag(double* A, int m, double* w, double* V, double* work, cudaStream_t s,
                    KernelTimer* tm = nullptr, OzWork* oz = nullptr);

// Dispatch: Jacobi for small matrices, tridiagonal method otherwise.
inline int sym_eig(double* A, int m, double* w, double* V, double* work, cudaStream_t s,
                   KernelTimer* tm = nullptr, OzWork* oz = nullptr) {
  return m <= 32 ? sym_eig_jacobi(A, m, w, V, work, s)
                 : sym_eig_tridiag(A, m, w, V, work, s, tm, oz);
}
inline size_t sym_eig_work(int m) {
  return std::max<size_t>((size_t)2 * m * m + 2, sym_eig_tridiag_work(m));
}

}  // namespace caspt2
