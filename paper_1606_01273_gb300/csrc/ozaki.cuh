// FP64-accurate GEMM on the tcgen05 tensor cores by exact BF16 splitting (internal).
//
// Each row x of an operand is scaled by a power of two sigma_x > max|x| and written as
// S integer slices, x / sigma_x = sum_s a_s 2^(-7(s+1)) + r with |a_0| <= 128,
// |a_s| <= 64 (s >= 1), |r| <= 2^(-7S-1) (the signed 7-bit digits of x / sigma_x as a
// 2^56 fixed-point integer, rounded to nearest): every a_s is exact in BF16.  A product of two
// slices is an integer below 2^14, so the tensor core's FP32 accumulation of any level
// l = s + t (at most l + 1 slice pairs) over a K chunk of 256 stays an exact integer below
// 2^24.  Per chunk the S level sums are read from TMEM and added, as exact integers shifted
// to a common scale, into two int64 accumulators (levels 0-2 and 3..S-1), so that
//   C_ij = sigma_i tau_j sum_l 2^(-7(l+2)) L_l(ij)
// is rounded to FP64 only once, at the end.
// Dropped terms (pairs with s + t >= S and the residuals) bound the error by about
// 2^(-7S+1) K max|a| max|b| per element (S = 5: ~3e-11 relative to that scale).
#pragma once
#include <cuda_bf16.h>

#include "common.cuh"

namespace caspt2 {

constexpr int kOzMaxSlices = 7;
constexpr int kOzKChunk = 256;     // exact FP32 accumulation span
constexpr int kOzKStage = 32;      // K per shared-memory stage

// Operand addressing: element (r, k) of an R x K operand is X[r * rs + (k / kin) * kout +
// (k % kin) * cs] (kin = K, kout = 0 for a plain strided matrix).
struct OzView {
  const double* X;
  long rs, cs, kin, kout;
};

// Slices of an operand: out[s][r][Kp] (BF16, K padded with zeros to Kp, a multiple of
// kOzKStage) and scale[r] = sigma_r.
cudaError_t oz_split(const OzView& v, int R, int K, int Kp, int S, __nv_bfloat16* out,
                     double* scale, cudaStream_t s);

// C[i][j] (ldc) = alpha * sum_k A(i,k) B(j,k) + beta * C[i][j] from the slices of A
// (M x Kp) and B (N x Kp).  err receives a nonzero code if a bounded wait gave up.
// nsplit > 1 splits K (in exact chunks) over CTAs; part then holds nsplit * M * N doubles.
cudaError_t oz_gemm(const __nv_bfloat16* As, const double* sa, const __nv_bfloat16* Bs,
                    const double* sb, int M, int N, int Kp, int S, double alpha, double beta,
                    double* C, long ldc, int* err, cudaStream_t s, int nsplit = 1,
                    double* part = nullptr);

// Device workspace of the split GEMMs, grown on demand (growth synchronises the device)
// and owned by the caller.  on = false selects the plain FP64 paths.
struct OzWork {
  bool on = false;
  int S = 7;
  __nv_bfloat16* sl = nullptr;
  size_t sl_bytes = 0;
  double* sc = nullptr;
  size_t sc_n = 0;
  int* err = nullptr;
  double* part = nullptr;   // split-K partial sums
  size_t part_n = 0;
};
void oz_release(OzWork& w);

// C (ldc) = alpha * A B^T + beta * C for an M x K view A and an N x K view B (same: B is A,
// sliced once).
cudaError_t oz_matmul(OzWork& w, const OzView& A, const OzView& B, bool same, int M, int N,
                      int K, double alpha, double beta, double* C, long ldc, cudaStream_t s);

// Bytes of BF16 slice storage for an R x K operand.
inline size_t oz_slice_bytes(int R, int K, int S) {
  const long Kp = (K + kOzKStage - 1) / kOzKStage * kOzKStage;
  return (size_t)S * R * Kp * sizeof(__nv_bfloat16);
}
inline int oz_kpad(int K) { return (K + kOzKStage - 1) / kOzKStage * kOzKStage; }

}  // namespace caspt2
