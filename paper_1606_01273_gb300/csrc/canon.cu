// Canonical closed and virtual orbitals for a Fock matrix whose closed-closed or
// virtual-virtual block is not diagonal (Sec. II.A/II.B: the energies are invariant under
// rotations among the closed and among the virtual orbitals, so the solve may run in the
// basis that diagonalises those blocks).
//
// C = blockdiag(Q_c, 1_act, Q_v), Q_c and Q_v the eigenvectors of f's closed and virtual
// blocks; the solve takes f' = C^T f C and B'_P = C^T B_P C.  A quantity M[p][q] that is
// a derivative with respect to f, h or B_P in the rotated basis is C M C^T in the
// caller's basis.
#include <algorithm>
#include <cmath>
#include <vector>

#include "class_dev.cuh"
#include "kernels.cuh"
#include "linalg.cuh"

namespace caspt2 {

namespace {

// A[i][j] = f[off + i][off + j], i, j < m
__global__ void k_canon_extract(const double* __restrict__ f, int nmo, int off, int m,
                                double* __restrict__ A) {
  const long total = (long)m * m;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    const int i = e / m, j = e % m;
    A[e] = f[(long)(off + i) * nmo + off + j];
  }
}

// C = blockdiag(Qc, 1, Qv)
__global__ void k_canon_build(const double* __restrict__ Qc, int c, int a,
                              const double* __restrict__ Qv, int v, double* __restrict__ C) {
  const int nmo = c + a + v;
  const long total = (long)nmo * nmo;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    const int p = e / nmo, q = e % nmo;
    double x = 0.0;
    if (p < c && q < c) x = Qc ? Qc[(long)p * c + q] : (p == q ? 1.0 : 0.0);
    else if (p >= c + a && q >= c + a) {
      const int i = p - c - a, j = q - c - a;
      x = Qv ? Qv[(long)i * v + j] : (i == j ? 1.0 : 0.0);
    } else if (p == q) x = 1.0;
    C[e] = x;
  }
}

// out = the block-diagonal canonical part of the rotated T: the closed and virtual
// diagonals and the (symmetrised) active block; every other entry is rounding of the
// rotation and set to zero.
__global__ void k_canon_clean(const double* __restrict__ T, int c, int a, int nmo,
                              double* __restrict__ out) {
  const long total = (long)nmo * nmo;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    const int p = e / nmo, q = e % nmo;
    const bool act = p >= c && p < c + a && q >= c && q < c + a;
    out[e] = (p == q || act) ? 0.5 * (T[e] + T[(long)q * nmo + p]) : 0.0;
  }
}

// Eigenvectors (columns) of the m x m block of f at offset off into Q (m >= 2).
int block_eigvecs(const double* f, int nmo, int off, int m, double* Q, cudaStream_t s) {
  double *A = nullptr, *w = nullptr, *work = nullptr;
  const size_t wsz = sym_eig_work(m);
  if (cudaMalloc(&A, sizeof(double) * m * m) != cudaSuccess) return CASPT2_ENOMEM;
  if (cudaMalloc(&w, sizeof(double) * m) != cudaSuccess) {
    cudaFree(A);
    return CASPT2_ENOMEM;
  }
  if (cudaMalloc(&work, sizeof(double) * wsz) != cudaSuccess) {
    cudaFree(A);
    cudaFree(w);
    return CASPT2_ENOMEM;
  }
  ++launch_counter();
  k_canon_extract<<<launch_blocks((long)m * m), 256, 0, s>>>(f, nmo, off, m, A);
  int st = cudaGetLastError() == cudaSuccess ? CASPT2_OK : CASPT2_ECUDA;
  if (st == CASPT2_OK) st = sym_eig(A, m, w, Q, work, s);
  if (st == CASPT2_OK && cudaStreamSynchronize(s) != cudaSuccess) st = CASPT2_ECUDA;
  cudaFree(A);
  cudaFree(w);
  cudaFree(work);
  return st;
}

}  // namespace

int classify_fock(const double* f, const Dims& d) {
  const int nmo = d.nmo();
  double fmax = 0.0;
  for (long k = 0; k < (long)nmo * nmo; ++k) {
    if (!(f[k] == f[k]) || std::fabs(f[k]) > 1e300) return CASPT2_ENAN;
    fmax = std::max(fmax, std::fabs(f[k]));
  }
  const double tol = 1e-10 * std::max(1.0, fmax);
  auto space = [&](int p) { return p < d.c ? 0 : (p < d.c + d.a ? 1 : 2); };
  bool rotated = false;
  for (int p = 0; p < nmo; ++p)
    for (int q = 0; q < nmo; ++q) {
      const double x = f[(long)p * nmo + q];
      if (std::fabs(x - f[(long)q * nmo + p]) > tol) return CASPT2_EINVAL;
      if (p == q) continue;
      const int sp = space(p), sq = space(q);
      if (sp != sq && std::fabs(x) > tol) return CASPT2_EINVAL;      // inter-space coupling
      if (sp == sq && sp != 1 && std::fabs(x) > tol) rotated = true;
    }
  return rotated ? 1 : 0;
}

int canonicalize_inputs(double* f, double* B, const Dims& d, double* C, cudaStream_t s) {
  const int nmo = d.nmo(), c = d.c, a = d.a, v = d.v;
  const long nn = (long)nmo * nmo;
  double *Qc = nullptr, *Qv = nullptr, *T1 = nullptr, *T2 = nullptr;
  int st = CASPT2_OK;
  auto cleanup = [&]() {
    cudaFree(Qc);
    cudaFree(Qv);
    cudaFree(T1);
    cudaFree(T2);
  };
  if (c >= 2) {
    if (cudaMalloc(&Qc, sizeof(double) * c * c) != cudaSuccess) return CASPT2_ENOMEM;
    st = block_eigvecs(f, nmo, 0, c, Qc, s);
  }
  if (st == CASPT2_OK && v >= 2) {
    if (cudaMalloc(&Qv, sizeof(double) * v * v) != cudaSuccess) st = CASPT2_ENOMEM;
    else st = block_eigvecs(f, nmo, c + a, v, Qv, s);
  }
  if (st != CASPT2_OK) {
    cleanup();
    return st;
  }
  ++launch_counter();
  k_canon_build<<<launch_blocks(nn), 256, 0, s>>>(Qc, c, a, Qv, v, C);
  if (cudaGetLastError() != cudaSuccess) {
    cleanup();
    return CASPT2_ECUDA;
  }
  // B_P <- C^T B_P C in chunks of matrices (work array of at most 2^27 doubles)
  const int qc = (int)std::max<long>(1, std::min<long>(d.X, (1L << 27) / std::max<long>(nn, 1)));
  const long tsz = std::max<long>((long)qc * nn, 2 * nn);
  if (cudaMalloc(&T1, sizeof(double) * tsz) != cudaSuccess ||
      cudaMalloc(&T2, sizeof(double) * nn) != cudaSuccess) {
    cleanup();
    return CASPT2_ENOMEM;
  }
  cudaError_t e = cudaSuccess;
  for (int q0 = 0; q0 < d.X && e == cudaSuccess; q0 += qc) {
    const int qb = std::min(qc, d.X - q0);
    double* Bq = B + (long)q0 * nn;
    e = dgemm(nmo, nmo, nmo, 1.0, Bq, nmo, false, C, nmo, false, 0.0, T1, nmo, s, qb, nn, 0, nn);
    if (e == cudaSuccess)
      e = dgemm(nmo, nmo, nmo, 1.0, C, nmo, true, T1, nmo, false, 0.0, Bq, nmo, s, qb, 0, nn, nn);
  }
  // f <- canonical part of C^T f C
  if (e == cudaSuccess)
    e = dgemm(nmo, nmo, nmo, 1.0, f, nmo, false, C, nmo, false, 0.0, T1, nmo, s);
  if (e == cudaSuccess)
    e = dgemm(nmo, nmo, nmo, 1.0, C, nmo, true, T1, nmo, false, 0.0, T2, nmo, s);
  if (e == cudaSuccess) {
    ++launch_counter();
    k_canon_clean<<<launch_blocks(nn), 256, 0, s>>>(T2, c, a, nmo, f);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cleanup();
  return e == cudaSuccess ? CASPT2_OK : CASPT2_ECUDA;
}

cudaError_t canon_back(const double* C, const double* M, int nmo, int batch, double* tmp,
                       double* out, cudaStream_t s) {
  const long nn = (long)nmo * nmo;
  cudaError_t e = dgemm(nmo, nmo, nmo, 1.0, M, nmo, false, C, nmo, true, 0.0, tmp, nmo, s, batch,
                        nn, 0, nn);
  if (e != cudaSuccess) return e;
  return dgemm(nmo, nmo, nmo, 1.0, C, nmo, false, tmp, nmo, false, 0.0, out, nmo, s, batch, 0, nn,
               nn);
}

}  // namespace caspt2
