// Setup kernels of the (X)MS-CASPT2 path, FP64:
//   state-averaged density and the mean field g(d) (Sec. II.B),
//   core energy, XMS Fock matrix and its diagonalisation (Sec. II.A),
//   rotated RDMs and the reference Hamiltonian H^ref (Sec. II.A),
//   effective Hamiltonian assembly (Sec. II.B).
// These are small next to the class kernels; they are written for clarity,
// coalesced along the fastest index, with fixed-order reductions.
#include "kernels.cuh"

namespace caspt2 {

// ---------------------------------------------------------------- d_sa (active)
__global__ void k_dsa(const double* __restrict__ rdm1, int n, int a, double* __restrict__ dact) {
  int rs = blockIdx.x * blockDim.x + threadIdx.x;
  if (rs >= a * a) return;
  double acc = 0.0;
  for (int N = 0; N < n; ++N) acc += rdm1[((long)N * n + N) * a * a + rs];
  dact[rs] = acc / n;
}

cudaError_t launch_dsa(const double* rdm1, const Dims& d, double* dact, cudaStream_t s) {
  int aa = d.a * d.a;
  if (aa == 0) return cudaSuccess;
  ++launch_counter();
  k_dsa<<<(aa + 127) / 128, 128, 0, s>>>(rdm1, d.n, d.a, dact);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- g(d_act)
// gam[P] = sum_tu B[P][c+t][c+u] d[t][u]
__global__ void k_gammaP(const double* __restrict__ B, const double* __restrict__ dact, int nmo,
                         int c, int a, double* __restrict__ gam) {
  __shared__ double red[32];
  const int P = blockIdx.x;
  const double* Bp = B + (long)P * nmo * nmo;
  double acc = 0.0;
  for (int tu = threadIdx.x; tu < a * a; tu += blockDim.x) {
    int t = tu / a, u = tu % a;
    acc += Bp[(long)(c + t) * nmo + c + u] * dact[tu];
  }
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) gam[P] = acc;
}

// Y[P][x][u] = sum_t B[P][x][c+t] d[t][u]
__global__ void k_Yact(const double* __restrict__ B, const double* __restrict__ dact, int X,
                       int nmo, int c, int a, double* __restrict__ Y) {
  long total = (long)X * nmo * a;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total;
       idx += (long)gridDim.x * blockDim.x) {
    int u = idx % a;
    long px = idx / a;
    int x = px % nmo;
    long P = px / nmo;
    const double* row = B + (P * nmo + x) * nmo + c;
    double acc = 0.0;
    for (int t = 0; t < a; ++t) acc += row[t] * dact[t * a + u];
    Y[idx] = acc;
  }
}

// g[x][y] = sum_P B[P][x][y] gam[P] - 1/2 sum_P sum_u Y[P][x][u] B[P][c+u][y]
__global__ void k_gfull(const double* __restrict__ B, const double* __restrict__ gam,
                        const double* __restrict__ Y, int X, int nmo, int c, int a,
                        double* __restrict__ g) {
  long total = (long)nmo * nmo;
  for (long xy = blockIdx.x * (long)blockDim.x + threadIdx.x; xy < total;
       xy += (long)gridDim.x * blockDim.x) {
    int x = xy / nmo, y = xy % nmo;
    double j = 0.0, k = 0.0;
    for (int P = 0; P < X; ++P) {
      const double* Bp = B + (long)P * nmo * nmo;
      j += Bp[xy] * gam[P];
      const double* yp = Y + ((long)P * nmo + x) * a;
      for (int u = 0; u < a; ++u) k += yp[u] * Bp[(long)(c + u) * nmo + y];
    }
    g[xy] = j - 0.5 * k;
  }
}

cudaError_t launch_gmat(const double* B, const double* dact, const Dims& d, double* gam,
                        double* Y, double* g, cudaStream_t s) {
  const int nmo = d.nmo();
  if (d.a == 0) {
    cudaError_t e = cudaMemsetAsync(g, 0, sizeof(double) * nmo * nmo, s);
    return e;
  }
  ++launch_counter();
  k_gammaP<<<d.X, 128, 0, s>>>(B, dact, nmo, d.c, d.a, gam);
  long ty = (long)d.X * nmo * d.a;
  ++launch_counter();
  k_Yact<<<(int)std::min<long>((ty + 255) / 256, 152 * 16), 256, 0, s>>>(B, dact, d.X, nmo, d.c, d.a, Y);
  long tg = (long)nmo * nmo;
  ++launch_counter();
  k_gfull<<<(int)std::min<long>((tg + 127) / 128, 152 * 32), 128, 0, s>>>(B, gam, Y, d.X, nmo, d.c, d.a, g);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- E_core
// bsum[P] = sum_i B[P][i][i], bfro[P] = sum_ij B[P][i][j]^2 over closed i, j
__global__ void k_core_parts(const double* __restrict__ B, int nmo, int c, double* bsum,
                             double* bfro) {
  __shared__ double red[32];
  const int P = blockIdx.x;
  const double* Bp = B + (long)P * nmo * nmo;
  double s1 = 0.0, s2 = 0.0;
  for (int ij = threadIdx.x; ij < c * c; ij += blockDim.x) {
    int i = ij / c, j = ij % c;
    double b = Bp[(long)i * nmo + j];
    s2 += b * b;
    if (i == j) s1 += b;
  }
  s1 = block_sum(s1, red);
  if (threadIdx.x == 0) bsum[P] = s1;
  s2 = block_sum(s2, red);
  if (threadIdx.x == 0) bfro[P] = s2;
}

// E_core = sum_i (2 f_ii - 2 g_ii) - sum_ij [2 (ii|jj) - (ij|ji)]
__global__ void k_ecore(const double* __restrict__ f, const double* __restrict__ g,
                        const double* __restrict__ bsum, const double* __restrict__ bfro, int X,
                        int nmo, int c, double* ecore) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < c; i += blockDim.x)
    acc += 2.0 * f[(long)i * nmo + i] - 2.0 * g[(long)i * nmo + i];
  for (int P = threadIdx.x; P < X; P += blockDim.x) acc -= 2.0 * bsum[P] * bsum[P] - bfro[P];
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) *ecore = acc;
}

cudaError_t launch_ecore(const double* f, const double* g, const double* B, const Dims& d,
                         double* bsum, double* bfro, double* ecore, cudaStream_t s) {
  ++launch_counter();
  k_core_parts<<<d.X, 128, 0, s>>>(B, d.nmo(), d.c, bsum, bfro);
  ++launch_counter();
  k_ecore<<<1, 256, 0, s>>>(f, g, bsum, bfro, d.X, d.nmo(), d.c, ecore);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- XMS Fock
__global__ void k_fref(const double* __restrict__ f, const double* __restrict__ rdm1, int n,
                       int a, int nmo, int c, double* fref) {
  __shared__ double red[32];
  const int MN = blockIdx.x;
  const double* g1 = rdm1 + (long)MN * a * a;
  double acc = 0.0;
  for (int rs = threadIdx.x; rs < a * a; rs += blockDim.x) {
    int r = rs / a, s = rs % a;
    acc += f[(long)(c + r) * nmo + c + s] * g1[rs];
  }
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) fref[MN] = acc;
}

cudaError_t launch_fref(const double* f, const double* rdm1, const Dims& d, double* fref,
                        cudaStream_t s) {
  ++launch_counter();
  k_fref<<<d.n * d.n, 64, 0, s>>>(f, rdm1, d.n, d.a, d.nmo(), d.c, fref);
  return cudaGetLastError();
}

// Cyclic Jacobi for a small symmetric matrix, one thread (n <= 16, deterministic).
// Eigenvalues ascending; each eigenvector signed so its largest-|.| entry is positive.
__global__ void k_sym_eig(const double* __restrict__ Ain, int n, double* V, double* w,
                          int identity, int* status) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double A[kMaxStates * kMaxStates], Q[kMaxStates * kMaxStates];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      A[i * n + j] = 0.5 * (Ain[i * n + j] + Ain[j * n + i]);
      Q[i * n + j] = (i == j) ? 1.0 : 0.0;
    }
  if (identity) {  // U = 1 (MS): keep the state order, no sorting
    for (int i = 0; i < n; ++i) {
      w[i] = A[i * n + i];
      for (int j = 0; j < n; ++j) V[i * n + j] = (i == j) ? 1.0 : 0.0;
    }
    return;
  }
  {
    bool conv = false;
    for (int sweep = 0; sweep < 100 && !conv; ++sweep) {
      double off = 0.0, dia = 0.0;
      for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) (i == j ? dia : off) += A[i * n + j] * A[i * n + j];
      if (off <= 1e-30 * (dia + 1e-300) || off == 0.0) { conv = true; break; }
      for (int p = 0; p < n - 1; ++p)
        for (int q = p + 1; q < n; ++q) {
          double apq = A[p * n + q];
          if (apq == 0.0) continue;
          double app = A[p * n + p], aqq = A[q * n + q];
          double theta = (aqq - app) / (2.0 * apq);
          double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
          double cs = 1.0 / sqrt(t * t + 1.0), sn = t * cs;
          for (int k = 0; k < n; ++k) {  // A <- J^T A J
            double akp = A[k * n + p], akq = A[k * n + q];
            A[k * n + p] = cs * akp - sn * akq;
            A[k * n + q] = sn * akp + cs * akq;
          }
          for (int k = 0; k < n; ++k) {
            double apk = A[p * n + k], aqk = A[q * n + k];
            A[p * n + k] = cs * apk - sn * aqk;
            A[q * n + k] = sn * apk + cs * aqk;
          }
          for (int k = 0; k < n; ++k) {
            double qkp = Q[k * n + p], qkq = Q[k * n + q];
            Q[k * n + p] = cs * qkp - sn * qkq;
            Q[k * n + q] = sn * qkp + cs * qkq;
          }
        }
    }
    if (!conv) atomicExch(status, CASPT2_ENOTCONV);
  }
  // sort ascending (selection sort on columns)
  double ev[kMaxStates];
  for (int i = 0; i < n; ++i) ev[i] = A[i * n + i];
  for (int i = 0; i < n; ++i) {
    int m = i;
    for (int j = i + 1; j < n; ++j)
      if (ev[j] < ev[m]) m = j;
    if (m != i) {
      double t = ev[i]; ev[i] = ev[m]; ev[m] = t;
      for (int k = 0; k < n; ++k) { double q = Q[k * n + i]; Q[k * n + i] = Q[k * n + m]; Q[k * n + m] = q; }
    }
  }
  for (int j = 0; j < n; ++j) {
    int im = 0;
    for (int k = 1; k < n; ++k)
      if (fabs(Q[k * n + j]) > fabs(Q[im * n + j])) im = k;
    double sg = Q[im * n + j] < 0 ? -1.0 : 1.0;
    for (int k = 0; k < n; ++k) V[k * n + j] = sg * Q[k * n + j];
    w[j] = ev[j];
  }
}

cudaError_t launch_sym_eig(const double* A, int n, double* V, double* w, int identity,
                           int* status, cudaStream_t s) {
  ++launch_counter();
  k_sym_eig<<<1, 32, 0, s>>>(A, n, V, w, identity, status);
  return cudaGetLastError();
}

__global__ void k_congruence(const double* __restrict__ A, const double* __restrict__ U, int n,
                             double* out) {
  int idx = threadIdx.x;
  if (idx >= n * n) return;
  int M = idx / n, N = idx % n;
  double acc = 0.0;
  for (int K = 0; K < n; ++K)
    for (int L = 0; L < n; ++L) acc += U[K * n + M] * A[K * n + L] * U[L * n + N];
  out[idx] = acc;
}

cudaError_t launch_congruence(const double* A, const double* U, int n, double* out, cudaStream_t s) {
  ++launch_counter();
  k_congruence<<<1, kMaxStates * kMaxStates, 0, s>>>(A, U, n, out);
  return cudaGetLastError();
}

__global__ void k_diag(const double* __restrict__ A, int n, double* e0) {
  int i = threadIdx.x;
  if (i < n) e0[i] = A[i * n + i];
}

cudaError_t launch_diag(const double* A, int n, double* e0, cudaStream_t s) {
  ++launch_counter();
  k_diag<<<1, 32, 0, s>>>(A, n, e0);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- RDM rotation
// One thread per element e: the n x n block src[.][.][e] is read once (coalesced
// over e) and all n^2 rotated values are written.
__global__ void k_rotate_rdm(const double* __restrict__ src, const double* __restrict__ U, int n,
                             long len, double* __restrict__ dst) {
  __shared__ double Us[kMaxStates * kMaxStates];
  for (int i = threadIdx.x; i < n * n; i += blockDim.x) Us[i] = U[i];
  __syncthreads();
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < len;
       e += (long)gridDim.x * blockDim.x) {
    double t[kMaxStates * kMaxStates];  // t[K][N] = sum_L src[K][L][e] U[L][N]
    for (int K = 0; K < n; ++K)
      for (int N = 0; N < n; ++N) t[K * n + N] = 0.0;
    for (int K = 0; K < n; ++K)
      for (int L = 0; L < n; ++L) {
        double sv = src[((long)K * n + L) * len + e];
        for (int N = 0; N < n; ++N) t[K * n + N] += sv * Us[L * n + N];
      }
    for (int M = 0; M < n; ++M)
      for (int N = 0; N < n; ++N) {
        double acc = 0.0;
        for (int K = 0; K < n; ++K) acc += Us[K * n + M] * t[K * n + N];
        dst[((long)M * n + N) * len + e] = acc;
      }
  }
}

cudaError_t launch_rotate_rdm(const double* src, const double* U, int n, long len, double* dst,
                              cudaStream_t s) {
  if (len == 0) return cudaSuccess;
  int blocks = (int)std::min<long>((len + 127) / 128, 152 * 16);
  ++launch_counter();
  k_rotate_rdm<<<blocks, 128, 0, s>>>(src, U, n, len, dst);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- active ERIs, H^ref
__global__ void k_eri_act(const double* __restrict__ B, int X, int nmo, int c, int a,
                          double* __restrict__ eri) {
  int aa = a * a;
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= aa * aa) return;
  int rs = idx / aa, tu = idx % aa;
  int r = rs / a, s_ = rs % a, t = tu / a, u = tu % a;
  double acc = 0.0;
  for (int P = 0; P < X; ++P) {
    const double* Bp = B + (long)P * nmo * nmo;
    acc += Bp[(long)(c + r) * nmo + c + s_] * Bp[(long)(c + t) * nmo + c + u];
  }
  eri[idx] = acc;
}

cudaError_t launch_eri_act(const double* B, const Dims& d, double* eri, cudaStream_t s) {
  int tot = d.a * d.a * d.a * d.a;
  if (tot == 0) return cudaSuccess;
  ++launch_counter();
  k_eri_act<<<(tot + 127) / 128, 128, 0, s>>>(B, d.X, d.nmo(), d.c, d.a, eri);
  return cudaGetLastError();
}

__global__ void k_href(const double* __restrict__ f, const double* __restrict__ g,
                       const double* __restrict__ rdm1r, const double* __restrict__ rdm2r,
                       const double* __restrict__ eri, const double* __restrict__ ecore,
                       double enuc, int n, int a, int nmo, int c, double* href) {
  __shared__ double red[32];
  const int MN = blockIdx.x;
  const int M = MN / n, N = MN % n;
  const int aa = a * a;
  double acc = 0.0;
  for (int rs = threadIdx.x; rs < aa; rs += blockDim.x) {
    int r = rs / a, s_ = rs % a;
    long xy = (long)(c + r) * nmo + c + s_;
    acc += (f[xy] - g[xy]) * rdm1r[(long)MN * aa + rs];
  }
  const double* g2 = rdm2r + (long)MN * aa * aa;
  for (long k = threadIdx.x; k < (long)aa * aa; k += blockDim.x) acc += 0.5 * eri[k] * g2[k];
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) href[MN] = acc + (M == N ? (*ecore + enuc) : 0.0);
}

cudaError_t launch_href(const double* f, const double* g, const double* rdm1r, const double* rdm2r,
                        const double* eri, const double* ecore, double enuc, const Dims& d,
                        double* href, cudaStream_t s) {
  ++launch_counter();
  k_href<<<d.n * d.n, 128, 0, s>>>(f, g, rdm1r, rdm2r, eri, ecore, enuc, d.n, d.a, d.nmo(), d.c,
                                  href);
  return cudaGetLastError();
}

__global__ void k_active_block(const double* __restrict__ f, int nmo, int c, int a, double* out) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < a * a) out[idx] = f[(long)(c + idx / a) * nmo + c + idx % a];
}

cudaError_t launch_active_block(const double* f, const Dims& d, double* out, cudaStream_t s) {
  if (d.a == 0) return cudaSuccess;
  ++launch_counter();
  k_active_block<<<(d.a * d.a + 127) / 128, 128, 0, s>>>(f, d.nmo(), d.c, d.a, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- H^eff
__global__ void k_heff(const double* __restrict__ href, const double* __restrict__ ecls,
                       const double* __restrict__ ncls, unsigned mask, double shift, int n,
                       double* heff) {
  int idx = threadIdx.x;
  if (idx >= n * n) return;
  int L = idx / n, Lp = idx % n;
  double acc = href[idx];
  for (int k = 0; k < CASPT2_NCLASS; ++k) {
    if (!(mask >> k & 1u)) continue;
    const double* e = ecls + (long)k * n * n;
    acc += 0.5 * (e[L * n + Lp] + e[Lp * n + L]);
    if (L == Lp) acc -= shift * ncls[k * n + L];
  }
  heff[idx] = acc;
}

cudaError_t launch_heff(const double* href, const double* ecls, const double* ncls, unsigned mask,
                        double shift, int n, double* heff, cudaStream_t s) {
  ++launch_counter();
  k_heff<<<1, kMaxStates * kMaxStates, 0, s>>>(href, ecls, ncls, mask, shift, n, heff);
  return cudaGetLastError();
}

}  // namespace caspt2
