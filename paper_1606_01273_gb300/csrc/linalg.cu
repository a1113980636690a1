// FP64 dense building blocks: a tiled GEMM and a parallel cyclic Jacobi
// eigensolver for symmetric matrices (used for the per-class overlap and Fock
// eigenproblems, Sec. II.B: truncation of the overlap eigenvalues).
#include "linalg.cuh"

namespace caspt2 {

// C[i][j] = alpha * sum_k A(i,k) B(k,j) + beta * C[i][j]
// A(i,k) = ta ? A[k*lda + i] : A[i*lda + k]; B(k,j) = tb ? B[j*ldb + k] : B[k*ldb + j]
constexpr int kGT = 64, kGK = 16;
__global__ void __launch_bounds__(256)
k_dgemm(int M, int N, int K, double alpha, const double* __restrict__ A, int lda, int ta,
        const double* __restrict__ B, int ldb, int tb, double beta, double* __restrict__ C, int ldc,
        long sA, long sB, long sC, int sym) {
  __shared__ double sa[kGK][kGT + 1], sb[kGK][kGT + 1];
  A += blockIdx.z * sA;
  B += blockIdx.z * sB;
  C += blockIdx.z * sC;
  int by = blockIdx.y, bx = blockIdx.x;
  if (sym) {          // symmetric result: upper-triangle tiles only, blockIdx.x linear
    const int T = (N + kGT - 1) / kGT;
    int rem = blockIdx.x;
    by = 0;
    while (rem >= T - by) { rem -= T - by; ++by; }
    bx = by + rem;
  }
  const int i0 = by * kGT, j0 = bx * kGT;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += kGK) {
    for (int l = threadIdx.x; l < kGK * kGT; l += 256) {
      int kk, ii;
      if (ta) { ii = l % kGT; kk = l / kGT; } else { kk = l % kGK; ii = l / kGK; }
      const int gi = i0 + ii, gk = k0 + kk;
      double v = 0.0;
      if (gi < M && gk < K) v = ta ? A[(long)gk * lda + gi] : A[(long)gi * lda + gk];
      sa[kk][ii] = v;
    }
    for (int l = threadIdx.x; l < kGK * kGT; l += 256) {
      int kk, jj;
      if (tb) { kk = l % kGK; jj = l / kGK; } else { jj = l % kGT; kk = l / kGT; }
      const int gj = j0 + jj, gk = k0 + kk;
      double v = 0.0;
      if (gj < N && gk < K) v = tb ? B[(long)gj * ldb + gk] : B[(long)gk * ldb + gj];
      sb[kk][jj] = v;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < kGK; ++kk) {
      double ra[4], rb[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) { ra[q] = sa[kk][ty + 16 * q]; rb[q] = sb[kk][tx + 16 * q]; }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = fma(ra[p], rb[q], acc[p][q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int gi = i0 + ty + 16 * p, gj = j0 + tx + 16 * q;
      if (gi < M && gj < N) {
        double* c = C + (long)gi * ldc + gj;
        *c = alpha * acc[p][q] + (beta == 0.0 ? 0.0 : beta * *c);
        if (sym && bx != by) {
          double* ct = C + (long)gj * ldc + gi;
          *ct = alpha * acc[p][q] + (beta == 0.0 ? 0.0 : beta * *ct);
        }
      }
    }
}

// Small-tile variant for products with a short edge: a TM x TN tile (each <= 32,
// fitted to M and N) per block, up to 4 outputs per thread, K in chunks of 8.
constexpr int kST = 32, kSK = 8;
__global__ void __launch_bounds__(256)
k_dgemm_s(int M, int N, int K, double alpha, const double* __restrict__ A, int lda, int ta,
          const double* __restrict__ B, int ldb, int tb, double beta, double* __restrict__ C,
          int ldc, int TM, int TN, int tn, long sA, long sB, long sC) {
  __shared__ double sa[kSK][kST + 1], sb[kSK][kST + 1];
  A += blockIdx.y * sA;
  B += blockIdx.y * sB;
  C += blockIdx.y * sC;
  const int i0 = (int)(blockIdx.x / tn) * TM, j0 = (int)(blockIdx.x % tn) * TN;
  const int nout = TM * TN;
  int oi[4], oj[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int q = threadIdx.x + 256 * r;
    oi[r] = q < nout ? q / TN : 0;
    oj[r] = q < nout ? q % TN : 0;
  }
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int k0 = 0; k0 < K; k0 += kSK) {
    for (int l = threadIdx.x; l < kSK * TM; l += 256) {
      int kk, ii;
      if (ta) { ii = l % TM; kk = l / TM; } else { kk = l % kSK; ii = l / kSK; }
      const int gi = i0 + ii, gk = k0 + kk;
      double v = 0.0;
      if (gi < M && gk < K) v = ta ? A[(long)gk * lda + gi] : A[(long)gi * lda + gk];
      sa[kk][ii] = v;
    }
    for (int l = threadIdx.x; l < kSK * TN; l += 256) {
      int kk, jj;
      if (tb) { kk = l % kSK; jj = l / kSK; } else { jj = l % TN; kk = l / TN; }
      const int gj = j0 + jj, gk = k0 + kk;
      double v = 0.0;
      if (gj < N && gk < K) v = tb ? B[(long)gj * ldb + gk] : B[(long)gk * ldb + gj];
      sb[kk][jj] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kSK; ++kk) {
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[r] = fma(sa[kk][oi[r]], sb[kk][oj[r]], acc[r]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int q = threadIdx.x + 256 * r;
    const int gi = i0 + oi[r], gj = j0 + oj[r];
    if (q < nout && gi < M && gj < N) {
      double* c = C + (long)gi * ldc + gj;
      *c = alpha * acc[r] + (beta == 0.0 ? 0.0 : beta * *c);
    }
  }
}

namespace {
thread_local GemmTimer* tl_gemm_timer = nullptr;

// Start of a timed launch: the slot of its event pair, or -1.
int gemm_timer_begin(cudaStream_t s) {
  GemmTimer* t = tl_gemm_timer;
  if (!t || !t->ready || t->used >= kGemmTimerPairs) return -1;
  const int slot = t->used++;
  cudaEventRecord(t->ev[2 * slot], s);
  return slot;
}
void gemm_timer_end(int slot, double flops, cudaStream_t s) {
  if (slot < 0) return;
  GemmTimer* t = tl_gemm_timer;
  cudaEventRecord(t->ev[2 * slot + 1], s);
  t->flops[slot] = flops;
}
}  // namespace

cudaError_t gemm_timer_init(GemmTimer& t) {
  if (t.ready) return cudaSuccess;
  for (auto& e : t.ev) {
    const cudaError_t r = cudaEventCreate(&e);
    if (r != cudaSuccess) return r;
  }
  t.used = 0;
  t.ready = true;
  return cudaSuccess;
}

void gemm_timer_release(GemmTimer& t) {
  for (auto& e : t.ev)
    if (e) cudaEventDestroy(e);
  t.ready = false;
}

void set_gemm_timer(GemmTimer* t) { tl_gemm_timer = t; }

cudaError_t gemm_timer_collect(GemmTimer& t, double* ms, double* flops, long* launches) {
  double tot = 0.0, fl = 0.0;
  for (int k = 0; k < t.used; ++k) {
    float x = 0.f;
    const cudaError_t r = cudaEventElapsedTime(&x, t.ev[2 * k], t.ev[2 * k + 1]);
    if (r != cudaSuccess) return r;
    tot += x;
    fl += t.flops[k];
  }
  *ms = tot;
  *flops = fl;
  *launches = t.used;
  t.used = 0;
  return cudaSuccess;
}

cudaError_t dgemm(int M, int N, int K, double alpha, const double* A, int lda, bool ta,
                  const double* B, int ldb, bool tb, double beta, double* C, int ldc,
                  cudaStream_t s, int batch, long sA, long sB, long sC) {
  if (M <= 0 || N <= 0 || batch <= 0) return cudaSuccess;
  const int slot = gemm_timer_begin(s);
  // padded work of the 64 x 64 tiles against tiles fitted to M and N (<= 32)
  const double pad64 = (double)((M + kGT - 1) / kGT * kGT) * ((N + kGT - 1) / kGT * kGT) /
                       ((double)M * N);
  ++launch_counter();
  if (pad64 > 1.3 || (M + kGT - 1) / kGT > 65535) {
    const int tm = (M + kST - 1) / kST, tn = (N + kST - 1) / kST;
    const int TM = (M + tm - 1) / tm, TN = (N + tn - 1) / tn;
    dim3 grid((unsigned)((long)tm * tn), batch);
    k_dgemm_s<<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, ta ? 1 : 0, B, ldb, tb ? 1 : 0, beta, C,
                                   ldc, TM, TN, tn, sA, sB, sC);
  } else {
    dim3 grid((N + kGT - 1) / kGT, (M + kGT - 1) / kGT, batch);
    k_dgemm<<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, ta ? 1 : 0, B, ldb, tb ? 1 : 0, beta, C,
                                 ldc, sA, sB, sC, 0);
  }
  gemm_timer_end(slot, 2.0 * M * N * (double)K * batch, s);
  return cudaGetLastError();
}

cudaError_t dgemm_sym(int N, int K, double alpha, const double* A, int lda, bool ta,
                      const double* B, int ldb, bool tb, double beta, double* C, int ldc,
                      cudaStream_t s) {
  const int T = (N + kGT - 1) / kGT;
  const double pad64 = (double)T * kGT * T * kGT / ((double)N * N);
  if (N <= 0 || pad64 > 1.3 || T > 2048)
    return dgemm(N, N, K, alpha, A, lda, ta, B, ldb, tb, beta, C, ldc, s);
  ++launch_counter();
  const int slot = gemm_timer_begin(s);
  dim3 grid((unsigned)((long)T * (T + 1) / 2), 1, 1);
  k_dgemm<<<grid, 256, 0, s>>>(N, N, K, alpha, A, lda, ta ? 1 : 0, B, ldb, tb ? 1 : 0, beta, C,
                               ldc, 0, 0, 0, 1);
  gemm_timer_end(slot, 2.0 * kGT * kGT * (double)K * ((double)T * (T + 1) / 2), s);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- Jacobi
// Round-robin ("circle") pairing over mp = m rounded up to even positions: in round r
// position 0 is fixed and positions 1..mp-1 rotate; pair k joins positions k and
// mp-1-k.  Indices >= m are padding (zero rows/columns, never rotated).
__device__ __forceinline__ int jac_index(int pos, int r, int mp) {
  return pos == 0 ? 0 : ((pos - 1 + r) % (mp - 1)) + 1;
}

__device__ __forceinline__ void jac_pair(int k, int r, int mp, int& p, int& q) {
  int a = jac_index(k, r, mp), b = jac_index(mp - 1 - k, r, mp);
  p = a < b ? a : b;
  q = a < b ? b : a;
}

__device__ __forceinline__ void jac_rot(const double* A, int m, int p, int q, double& c, double& s) {
  c = 1.0;
  s = 0.0;
  if (q >= m) return;
  const double apq = A[(long)p * m + q];
  if (apq == 0.0) return;
  const double app = A[(long)p * m + p], aqq = A[(long)q * m + q];
  const double theta = (aqq - app) / (2.0 * apq);
  double t;
  if (fabs(theta) > 1e150) t = 0.5 / theta;
  else t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
  c = 1.0 / sqrt(t * t + 1.0);
  s = t * c;
}

// A' = J^T A J for the disjoint rotations of round r (one thread per 2x2 block of pairs),
// V' = V J.  Reads A, V; writes A2, V2 (ping-pong buffers).
__global__ void k_jacobi_round(const double* __restrict__ A, double* __restrict__ A2,
                               const double* __restrict__ V, double* __restrict__ V2, int m,
                               int mp, int r) {
  const int npair = mp / 2;
  const long nblk = (long)npair * npair;
  const long total = nblk + (long)m * npair;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total;
       t += (long)gridDim.x * blockDim.x) {
    if (t < nblk) {
      const int I = t / npair, J = t % npair;
      int pI, qI, pJ, qJ;
      jac_pair(I, r, mp, pI, qI);
      jac_pair(J, r, mp, pJ, qJ);
      double cI, sI, cJ, sJ;
      jac_rot(A, m, pI, qI, cI, sI);
      jac_rot(A, m, pJ, qJ, cJ, sJ);
      const bool vq_I = qI < m, vq_J = qJ < m;
      const double a00 = A[(long)pI * m + pJ];
      const double a01 = vq_J ? A[(long)pI * m + qJ] : 0.0;
      const double a10 = vq_I ? A[(long)qI * m + pJ] : 0.0;
      const double a11 = (vq_I && vq_J) ? A[(long)qI * m + qJ] : 0.0;
      // rows: [c -s; s c] * A_sub ; columns: * [c s; -s c]
      const double r00 = cI * a00 - sI * a10, r01 = cI * a01 - sI * a11;
      const double r10 = sI * a00 + cI * a10, r11 = sI * a01 + cI * a11;
      double n00 = r00 * cJ - r01 * sJ, n01 = r00 * sJ + r01 * cJ;
      double n10 = r10 * cJ - r11 * sJ, n11 = r10 * sJ + r11 * cJ;
      if (I == J && vq_I) { n01 = 0.0; n10 = 0.0; }   // the rotated pair is annihilated
      A2[(long)pI * m + pJ] = n00;
      if (vq_J) A2[(long)pI * m + qJ] = n01;
      if (vq_I) A2[(long)qI * m + pJ] = n10;
      if (vq_I && vq_J) A2[(long)qI * m + qJ] = n11;
    } else {
      const long u = t - nblk;
      const int row = u / npair, J = u % npair;
      int pJ, qJ;
      jac_pair(J, r, mp, pJ, qJ);
      double cJ, sJ;
      jac_rot(A, m, pJ, qJ, cJ, sJ);
      const double vp = V[(long)row * m + pJ];
      if (qJ < m) {
        const double vq = V[(long)row * m + qJ];
        V2[(long)row * m + pJ] = cJ * vp - sJ * vq;
        V2[(long)row * m + qJ] = sJ * vp + cJ * vq;
      } else {
        V2[(long)row * m + pJ] = vp;
      }
    }
  }
}

__global__ void k_eye(double* V, int m) {
  long total = (long)m * m;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total;
       t += (long)gridDim.x * blockDim.x)
    V[t] = (t / m == t % m) ? 1.0 : 0.0;
}

// off = sum_{i != j} A_ij^2, dia = sum_i A_ii^2 (fixed-order block reduction)
__global__ void k_offnorm(const double* __restrict__ A, int m, double* out) {
  __shared__ double red[32];
  double off = 0.0, dia = 0.0;
  const long total = (long)m * m;
  for (long t = threadIdx.x; t < total; t += blockDim.x) {
    const double x = A[t];
    if (t / m == t % m) dia += x * x; else off += x * x;
  }
  off = block_sum(off, red);
  if (threadIdx.x == 0) out[0] = off;
  dia = block_sum(dia, red);
  if (threadIdx.x == 0) out[1] = dia;
}

__global__ void k_diag_out(const double* __restrict__ A, int m, double* w) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) w[i] = A[(long)i * m + i];
}

// Sort eigenpairs ascending (one block; rank by counting, ties by index): w2, V2 from w, V.
__global__ void k_sort_pairs(const double* __restrict__ w, const double* __restrict__ V, int m,
                             double* __restrict__ w2, double* __restrict__ V2) {
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    int r = 0;
    for (int k = 0; k < m; ++k) r += (w[k] < w[j] || (w[k] == w[j] && k < j)) ? 1 : 0;
    w2[r] = w[j];
    for (int i = 0; i < m; ++i) V2[(long)i * m + r] = V[(long)i * m + j];
  }
}

// The whole cyclic Jacobi iteration of one small matrix (m <= kJacobiFusedMax) in one
// block with A and V resident in shared memory: the rounds of k_jacobi_round, a fixed-order
// off-diagonal norm after each sweep with the same stopping rule as the multi-launch path,
// then the eigenvalues, and the pairs sorted ascending into w and V (A is left rotated).
// status[0] = 1 when converged, 0 otherwise, -1 on NaN.
constexpr int kJacobiFusedMax = 32;
__global__ void __launch_bounds__(256)
k_jacobi_fused(double* __restrict__ A, int m, double* __restrict__ w, double* __restrict__ V,
               int* __restrict__ status) {
  constexpr int MM = kJacobiFusedMax * kJacobiFusedMax;
  __shared__ double sA[2][MM], sV[2][MM];
  __shared__ double red[32];
  __shared__ double sw[kJacobiFusedMax];
  __shared__ int flag;
  const long mm = (long)m * m;
  for (long t = threadIdx.x; t < mm; t += blockDim.x) {
    sA[0][t] = A[t];
    sV[0][t] = (t / m == t % m) ? 1.0 : 0.0;
  }
  if (threadIdx.x == 0) flag = (m == 1) ? 1 : 0;
  __syncthreads();
  const int mp = m + (m & 1);
  const int npair = mp / 2;
  const long nblk = (long)npair * npair;
  const long total = nblk + (long)m * npair;
  int cur = 0;
  double prev = -1.0;
  for (int sweep = 0; sweep < 60 && flag == 0; ++sweep) {
    for (int r = 0; r < mp - 1; ++r) {
      const double* Ac = sA[cur];
      double* An = sA[cur ^ 1];
      const double* Vc = sV[cur];
      double* Vn = sV[cur ^ 1];
      for (long t = threadIdx.x; t < total; t += blockDim.x) {
        if (t < nblk) {
          const int I = t / npair, J = t % npair;
          int pI, qI, pJ, qJ;
          jac_pair(I, r, mp, pI, qI);
          jac_pair(J, r, mp, pJ, qJ);
          double cI, sI, cJ, sJ;
          jac_rot(Ac, m, pI, qI, cI, sI);
          jac_rot(Ac, m, pJ, qJ, cJ, sJ);
          const bool vq_I = qI < m, vq_J = qJ < m;
          const double a00 = Ac[pI * m + pJ];
          const double a01 = vq_J ? Ac[pI * m + qJ] : 0.0;
          const double a10 = vq_I ? Ac[qI * m + pJ] : 0.0;
          const double a11 = (vq_I && vq_J) ? Ac[qI * m + qJ] : 0.0;
          const double r00 = cI * a00 - sI * a10, r01 = cI * a01 - sI * a11;
          const double r10 = sI * a00 + cI * a10, r11 = sI * a01 + cI * a11;
          double n00 = r00 * cJ - r01 * sJ, n01 = r00 * sJ + r01 * cJ;
          double n10 = r10 * cJ - r11 * sJ, n11 = r10 * sJ + r11 * cJ;
          if (I == J && vq_I) { n01 = 0.0; n10 = 0.0; }
          An[pI * m + pJ] = n00;
          if (vq_J) An[pI * m + qJ] = n01;
          if (vq_I) An[qI * m + pJ] = n10;
          if (vq_I && vq_J) An[qI * m + qJ] = n11;
        } else {
          const long u = t - nblk;
          const int row = u / npair, J = u % npair;
          int pJ, qJ;
          jac_pair(J, r, mp, pJ, qJ);
          double cJ, sJ;
          jac_rot(Ac, m, pJ, qJ, cJ, sJ);
          const double vp = Vc[row * m + pJ];
          if (qJ < m) {
            const double vq = Vc[row * m + qJ];
            Vn[row * m + pJ] = cJ * vp - sJ * vq;
            Vn[row * m + qJ] = sJ * vp + cJ * vq;
          } else {
            Vn[row * m + pJ] = vp;
          }
        }
      }
      __syncthreads();
      cur ^= 1;
    }
    double off = 0.0, dia = 0.0;
    for (long t = threadIdx.x; t < mm; t += blockDim.x) {
      const double x = sA[cur][t];
      if (t / m == t % m) dia += x * x; else off += x * x;
    }
    off = block_sum(off, red);
    __syncthreads();
    dia = block_sum(dia, red);
    if (threadIdx.x == 0) {
      if (!(off == off)) flag = -1;
      else if (off == 0.0 || off <= 1e-34 * dia) flag = 1;
      else if (off <= 1e-20 * dia && prev >= 0.0 && off > 0.25 * prev) flag = 1;
      prev = off;
    }
    __syncthreads();
  }
  for (long t = threadIdx.x; t < mm; t += blockDim.x) A[t] = sA[cur][t];
  for (int i = threadIdx.x; i < m; i += blockDim.x) sw[i] = sA[cur][i * m + i];
  __syncthreads();
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    int rk = 0;
    for (int k = 0; k < m; ++k) rk += (sw[k] < sw[j] || (sw[k] == sw[j] && k < j)) ? 1 : 0;
    w[rk] = sw[j];
    for (int i = 0; i < m; ++i) V[(long)i * m + rk] = sV[cur][i * m + j];
  }
  if (threadIdx.x == 0) status[0] = flag;
}

// Eigenpairs of symmetric A (m x m, row-major, overwritten): w[m], V[m][m] (columns).
// work: 2*m*m doubles + 2.  Ascending.  Synchronises the stream once per sweep.
int sym_eig_jacobi(double* A, int m, double* w, double* V, double* work, cudaStream_t s) {
  if (m <= 0) return CASPT2_OK;
  if (m <= kJacobiFusedMax) {
    int* st_dev = reinterpret_cast<int*>(work + 2L * m * m);
    ++launch_counter();
    k_jacobi_fused<<<1, 256, 0, s>>>(A, m, w, V, st_dev);
    CASPT2_CUDA_TRY(cudaGetLastError());
    int st = 0;
    CASPT2_CUDA_TRY(cudaMemcpyAsync(&st, st_dev, sizeof(int), cudaMemcpyDeviceToHost, s));
    CASPT2_CUDA_TRY(cudaStreamSynchronize(s));
    if (st < 0) return CASPT2_ENAN;
    return st == 1 ? CASPT2_OK : CASPT2_ENOTCONV;
  }
  double* A2 = work;
  double* V2 = work + (long)m * m;
  double* nrm = work + 2L * m * m;
  const int mp = m + (m & 1);
  const long total = (long)(mp / 2) * (mp / 2) + (long)m * (mp / 2);
  const int threads = 256;
  const int blocks = (int)std::min<long>((total + threads - 1) / threads, 152L * 16);
  ++launch_counter();
  k_eye<<<(int)std::min<long>(((long)m * m + 255) / 256, 152L * 16), 256, 0, s>>>(V, m);
  CASPT2_CUDA_TRY(cudaGetLastError());
  CASPT2_CUDA_TRY(cudaMemcpyAsync(A2, A, sizeof(double) * m * m, cudaMemcpyDeviceToDevice, s));
  CASPT2_CUDA_TRY(cudaMemcpyAsync(V2, V, sizeof(double) * m * m, cudaMemcpyDeviceToDevice, s));
  double* cur = A;
  double* nxt = A2;
  double* vc = V;
  double* vn = V2;
  bool conv = (m == 1);
  double prev = -1.0;
  // Sweep until the off-diagonal norm reaches the rounding floor: it is exactly zero,
  // below 1e-34 of the diagonal, or (once below 1e-20) it no longer drops by 4x.
  for (int sweep = 0; sweep < 60 && !conv; ++sweep) {
    for (int r = 0; r < mp - 1; ++r) {
      ++launch_counter();
      k_jacobi_round<<<blocks, threads, 0, s>>>(cur, nxt, vc, vn, m, mp, r);
      std::swap(cur, nxt);
      std::swap(vc, vn);
    }
    CASPT2_CUDA_TRY(cudaGetLastError());
    ++launch_counter();
    k_offnorm<<<1, 1024, 0, s>>>(cur, m, nrm);
    double h[2];
    CASPT2_CUDA_TRY(cudaMemcpyAsync(h, nrm, sizeof(h), cudaMemcpyDeviceToHost, s));
    CASPT2_CUDA_TRY(cudaStreamSynchronize(s));
    if (!(h[0] == h[0])) return CASPT2_ENAN;
    if (h[0] == 0.0 || h[0] <= 1e-34 * h[1]) conv = true;
    else if (h[0] <= 1e-20 * h[1] && prev >= 0.0 && h[0] > 0.25 * prev) conv = true;
    prev = h[0];
  }
  if (cur != A) {
    CASPT2_CUDA_TRY(cudaMemcpyAsync(A, cur, sizeof(double) * m * m, cudaMemcpyDeviceToDevice, s));
    CASPT2_CUDA_TRY(cudaMemcpyAsync(V, vc, sizeof(double) * m * m, cudaMemcpyDeviceToDevice, s));
  }
  // eigenvalues into A2's first row, sorted pairs back into w and V
  ++launch_counter();
  k_diag_out<<<(m + 127) / 128, 128, 0, s>>>(A, m, A2);
  CASPT2_CUDA_TRY(cudaMemcpyAsync(V2, V, sizeof(double) * m * m, cudaMemcpyDeviceToDevice, s));
  ++launch_counter();
  k_sort_pairs<<<1, 256, 0, s>>>(A2, V2, m, w, V);
  CASPT2_CUDA_TRY(cudaGetLastError());
  return conv ? CASPT2_OK : CASPT2_ENOTCONV;
}

}  // namespace caspt2
