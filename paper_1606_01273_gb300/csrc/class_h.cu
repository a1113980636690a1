// Class H (E_ai,bj, Eq. class) of the first-order amplitudes, FP64, direct.
//
// For block-diagonal f the E_ai,bj E_Omega|N~> functions couple to the
// reference index only through the active Fock matrix: with U^T Fref U =
// W diag(omega) W^T, the amplitude equation (Eq. ampeq) for state L becomes, in
// the eigenbasis nu, a closed-shell pair equation with denominator
//     D = e_a + e_b - e_i - e_j + omega_nu - E0_L + E_s.
// The contributions to the effective Hamiltonian (Sec. II.B) are then
//     <Psi1_L|H|L'~>_H = -sum_nu W_Lnu W_L'nu sum_ijab K(2K - K')/D
//     <Psi1_L|Psi1_L>_H =  sum_nu W_Lnu^2     sum_ijab K(2K - K')/D^2
// with K = (ai|bj) = sum_P B_Pai B_Pbj, K' = (aj|bi).  Under SS-SR (Eq. wfp2) only
// nu = L survives and D = e_a + e_b - e_i - e_j + E_s.
//
// The amplitudes are never stored: one CTA forms a 64x64 tile of K_ij (and the
// mirrored tile) over the DF index, and the epilogue applies every
// denominator shift and reduces the energy and norm sums.  Per-CTA partial
// sums are reduced afterwards in a fixed order, so results are bitwise
// reproducible run to run.
#include "kernels.cuh"
#include "class_ag.cuh"
#include "ozaki.cuh"

namespace caspt2 {

constexpr int kHT = 64;   // tile edge in a and in b
constexpr int kHK = 16;   // DF-index chunk
constexpr int kHThreads = 256;
constexpr int kMaxShift = kMaxStates * kMaxStates;

// Bp[i][P][a] = B[P][i][vo + a]
__global__ void k_pack_cv(const double* __restrict__ B, int c, int v, int X, int nmo, int vo,
                          double* __restrict__ Bp) {
  long total = (long)c * X * v;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total;
       idx += (long)gridDim.x * blockDim.x) {
    int a = idx % v;
    long iP = idx / v;
    int P = iP % X;
    int i = iP / X;
    Bp[idx] = B[((long)P * nmo + i) * nmo + vo + a];
  }
}

// eps[0..c) = closed orbital energies, eps[c..c+v) = virtual orbital energies
__global__ void k_eps_cv(const double* __restrict__ f, int nmo, int c, int a, int v, double* eps) {
  int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x < c) eps[x] = f[(long)x * nmo + x];
  else if (x < c + v) eps[x] = f[(long)(x + a) * nmo + x + a];
}

// shifts[nu*n + L] = omega_nu - E0_L + E_s (MS-MR) ; shifts[0] = E_s (SS-SR)
__global__ void k_classH_shifts(const double* __restrict__ omega, const double* __restrict__ E0,
                                double shift, int n, int scheme, double* shifts) {
  int k = threadIdx.x;
  if (scheme == CASPT2_SSSR) {
    if (k == 0) shifts[0] = shift;
    return;
  }
  if (k < n * n) shifts[k] = omega[k / n] - E0[k % n] + shift;
}

// One CTA = (pair i <= j, tile pair ta <= tb).  It forms T1[a][b] = K_ij^ab over
// a in tile ta, b in tile tb and, when ta < tb, T2[a][b] = K_ij^ba = sum_P B_ib B_ja,
// so each thread holds both K_ij^ab and K_ij^ba for its elements and the K_ij block
// is computed exactly once.  On a diagonal tile (ta == tb) K_ij^ba is read from the
// transposed tile staged in shared memory.  Block (j, i) equals block (i, j) with a
// and b swapped, so i < j carries weight 2; for i == j, K_ii^ba = K_ii^ab.
__global__ void __launch_bounds__(kHThreads)
k_classH(const double* __restrict__ Bp, const double* __restrict__ eps,
         const double* __restrict__ shifts, int nshift, int c, int v, int X, int ntile,
         int pair0, double* __restrict__ partial) {
  __shared__ double sbuf[4 * kHK * kHT];   // operand tiles; reused for the diagonal transpose
  __shared__ double sEa[kHT], sEb[kHT];
  __shared__ double sShift[kMaxShift];
  __shared__ double red[32];
  double (*sAi)[kHT] = reinterpret_cast<double (*)[kHT]>(sbuf);
  double (*sBj)[kHT] = reinterpret_cast<double (*)[kHT]>(sbuf + kHK * kHT);
  double (*sAj)[kHT] = reinterpret_cast<double (*)[kHT]>(sbuf + 2 * kHK * kHT);
  double (*sBi)[kHT] = reinterpret_cast<double (*)[kHT]>(sbuf + 3 * kHK * kHT);

  const int ntp = ntile * (ntile + 1) / 2;
  long bid = blockIdx.x;
  int tp = bid % ntp;
  int pair = pair0 + (int)(bid / ntp), i = 0;
  while (pair >= c - i) { pair -= c - i; ++i; }
  const int j = i + pair;
  int ta = 0;
  while (tp >= ntile - ta) { tp -= ntile - ta; ++ta; }
  const int tb = ta + tp;
  const bool same = (i == j);
  const bool diag = (ta == tb);
  const bool need_t2 = !same && !diag;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int a0 = ta * kHT, b0 = tb * kHT;
  const double* bi = Bp + (long)i * X * v;
  const double* bj = Bp + (long)j * X * v;

  for (int k = threadIdx.x; k < nshift; k += kHThreads) sShift[k] = shifts[k];
  for (int k = threadIdx.x; k < kHT; k += kHThreads) {
    sEa[k] = (a0 + k < v) ? eps[c + a0 + k] : 0.0;   // eps holds closed then virtual energies
    sEb[k] = (b0 + k < v) ? eps[c + b0 + k] : 0.0;
  }
  __syncthreads();

  double t1[4][4], t2[4][4];
#pragma unroll
  for (int ii = 0; ii < 4; ++ii)
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) t1[ii][jj] = t2[ii][jj] = 0.0;

  for (int P0 = 0; P0 < X; P0 += kHK) {
    for (int l = threadIdx.x; l < kHK * kHT; l += kHThreads) {
      const int kk = l / kHT, col = l % kHT;
      const int P = P0 + kk;
      const bool okP = P < X;
      const int a = a0 + col, b = b0 + col;
      sAi[kk][col] = (okP && a < v) ? bi[(long)P * v + a] : 0.0;
      sBj[kk][col] = (okP && b < v) ? bj[(long)P * v + b] : 0.0;
      if (need_t2) {
        sAj[kk][col] = (okP && a < v) ? bj[(long)P * v + a] : 0.0;
        sBi[kk][col] = (okP && b < v) ? bi[(long)P * v + b] : 0.0;
      }
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < kHK; ++kk) {
      double ra[4], rb[4];
#pragma unroll
      for (int ii = 0; ii < 4; ++ii) ra[ii] = sAi[kk][ty + 16 * ii];
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) rb[jj] = sBj[kk][tx + 16 * jj];
#pragma unroll
      for (int ii = 0; ii < 4; ++ii)
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) t1[ii][jj] = fma(ra[ii], rb[jj], t1[ii][jj]);
      if (need_t2) {
#pragma unroll
        for (int ii = 0; ii < 4; ++ii) ra[ii] = sAj[kk][ty + 16 * ii];
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) rb[jj] = sBi[kk][tx + 16 * jj];
#pragma unroll
        for (int ii = 0; ii < 4; ++ii)
#pragma unroll
          for (int jj = 0; jj < 4; ++jj) t2[ii][jj] = fma(ra[ii], rb[jj], t2[ii][jj]);
      }
    }
    __syncthreads();
  }

  if (same) {
#pragma unroll
    for (int ii = 0; ii < 4; ++ii)
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) t2[ii][jj] = t1[ii][jj];
  } else if (diag) {
    // K_ij^ba of this thread's (a, b) is T1 at (b, a): stage T1 (64 x 64) and read it transposed
    double* sT = sbuf;
#pragma unroll
    for (int ii = 0; ii < 4; ++ii)
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) sT[(ty + 16 * ii) * kHT + tx + 16 * jj] = t1[ii][jj];
    __syncthreads();
#pragma unroll
    for (int ii = 0; ii < 4; ++ii)
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) t2[ii][jj] = sT[(tx + 16 * jj) * kHT + ty + 16 * ii];
  }

  // epilogue: numerators and shift-free denominators of this thread's 16 (a, b)
  const double wij = same ? 1.0 : 2.0;
  const double ei = eps[i], ej = eps[j];
  double num[16], d0[16];
#pragma unroll
  for (int ii = 0; ii < 4; ++ii)
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
      const int la = ty + 16 * ii, lb = tx + 16 * jj;
      const bool ok = (a0 + la < v) && (b0 + lb < v);
      const double k1 = t1[ii][jj];          // K_ij^ab
      const double k2 = t2[ii][jj];          // K_ij^ba
      // element (a, b); when ta < tb also element (b, a), which lives in no other CTA
      double nm = k1 * (2.0 * k1 - k2);
      if (!diag) nm += k2 * (2.0 * k2 - k1);
      num[ii * 4 + jj] = ok ? wij * nm : 0.0;
      d0[ii * 4 + jj] = ok ? (sEa[la] + sEb[lb] - ei - ej) : 1.0;
    }
  double* out = partial + blockIdx.x * (long)(3 * nshift + 1);
  double dmin = 1e300;
  for (int k = 0; k < nshift; ++k) {
    const double sh = sShift[k];
    double e = 0.0, nr = 0.0, n3 = 0.0;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const double inv = 1.0 / (d0[q] + sh);
      const double x = num[q] * inv;
      e += x;
      nr = fma(x, inv, nr);
      n3 = fma(x * inv, inv, n3);
      if (num[q] != 0.0) dmin = fmin(dmin, fabs(d0[q] + sh));
    }
    e = block_sum(e, red);
    if (threadIdx.x == 0) out[k] = e;
    nr = block_sum(nr, red);
    if (threadIdx.x == 0) out[nshift + k] = nr;
    n3 = block_sum(n3, red);
    if (threadIdx.x == 0) out[2 * nshift + k] = n3;
  }
  dmin = block_min(dmin, red);
  if (threadIdx.x == 0) out[3 * nshift] = dmin;
}

// sums[col] = fixed-order reduction of partial[.][col]; the last column is a min.
__global__ void k_reduce_cols(const double* __restrict__ partial, long nblocks, int ncol,
                              double* __restrict__ sums) {
  __shared__ double red[32];
  const int col = blockIdx.x;
  const bool is_min = (col == ncol - 1);
  double acc = is_min ? 1e300 : 0.0;
  for (long b = threadIdx.x; b < nblocks; b += blockDim.x) {
    double x = partial[b * ncol + col];
    acc = is_min ? fmin(acc, x) : acc + x;
  }
  acc = is_min ? block_min(acc, red) : block_sum(acc, red);
  if (threadIdx.x == 0) sums[col] = acc;
}

// Moments of class H from the sums Sk[nu,L] = sum num / D^k (k = 1, 2, 3):
//   M1[L][N][L'] = sum_nu W_Nnu W_L'nu S1[nu,L], M2[L][N] = sum_nu W_Nnu W_Lnu S2[nu,L],
//   M3[L] = sum_nu W_Lnu^2 S3[nu,L]; under SS-SR only N = L' = L with S_k[0].
// e[L][L'] = -M1[L][L][L'], norm[L] = M2[L][L].
__global__ void k_classH_combine(const double* __restrict__ sums, const double* __restrict__ W,
                                 int n, int scheme, double* ecls, double* ncls, double* mom,
                                 double* mindenom, int* status) {
  const int nshift = (scheme == CASPT2_SSSR) ? 1 : n * n;
  const double* S1 = sums;
  const double* S2 = sums + nshift;
  const double* S3 = sums + 2 * nshift;
  for (int idx = threadIdx.x; idx < n * n * n; idx += blockDim.x) {
    const int L = idx / (n * n), N = (idx / n) % n, Lp = idx % n;
    double v = 0.0;
    if (scheme == CASPT2_SSSR) v = (N == L && Lp == L) ? S1[0] : 0.0;
    else
      for (int nu = 0; nu < n; ++nu) v += W[N * n + nu] * W[Lp * n + nu] * S1[nu * n + L];
    mom[idx] = v;
    if (N == L) ecls[L * n + Lp] = -v;
  }
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int L = idx / n, N = idx % n;
    double v = 0.0;
    if (scheme == CASPT2_SSSR) v = (N == L) ? S2[0] : 0.0;
    else
      for (int nu = 0; nu < n; ++nu) v += W[N * n + nu] * W[L * n + nu] * S2[nu * n + L];
    mom[n * n * n + idx] = v;
    if (N == L) ncls[L] = v;
  }
  for (int L = threadIdx.x; L < n; L += blockDim.x) {
    double v = 0.0;
    if (scheme == CASPT2_SSSR) v = S3[0];
    else
      for (int nu = 0; nu < n; ++nu) v += W[L * n + nu] * W[L * n + nu] * S3[nu * n + L];
    mom[n * n * n + n * n + L] = v;
  }
  if (threadIdx.x == 0) {
    const double dm = sums[3 * nshift];
    *mindenom = fmin(*mindenom, dm);
    if (!(dm == dm)) atomicExch(status, CASPT2_ENAN);
  }
}

// Split form: KK[(ia)][(jb)] = K_ij^ab (2 K_ij^ab - K_ij^ba) from the full K matrix.
__global__ void k_classH_num(const double* __restrict__ K, int c, int v, int i0, int i1,
                             double* __restrict__ KK) {
  const long cv = (long)c * v, e0 = (long)i0 * v * cv, total = (long)i1 * v * cv;
  for (long e = e0 + blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    const long ia = e / cv, jb = e % cv;
    const int i = ia / v, a = ia % v, j = jb / v, b = jb % v;
    const double k1 = K[e];
    KK[e] = k1 * (2.0 * k1 - K[((long)i * v + b) * cv + (long)j * v + a]);
  }
}

// Split form: per-shift sums over all (i, j, a, b) of KK / D, KK / D^2, KK / D^3 and the
// smallest |D| with KK != 0; grid (nblk, nshift), one row of partial per block with only
// its own shift's columns set (the others zero, the min column +inf for no element), so the
// fixed-order column reduction of the fused kernel applies unchanged.
__global__ void k_classH_sums(const double* __restrict__ KK, const double* __restrict__ eps,
                              const double* __restrict__ shifts, int nshift, int c, int v,
                              int i0, int i1, double* __restrict__ partial) {
  __shared__ double red[32];
  const int k = blockIdx.y;
  const double sh = shifts[k];
  const long cv = (long)c * v;
  double e = 0.0, nr = 0.0, n3 = 0.0;
  // smallest |D| with KK != 0, kept as the bit pattern of |D| (non-negative doubles order
  // like their bit patterns, so the minimum runs on the integer units)
  unsigned long long dminb = 0x7FF0000000000000ull;
  // rows (i, a) over the blocks, (j, b) of a row over the threads: index arithmetic once
  // per row and per j, not per element
  for (long ia = (long)i0 * v + blockIdx.x; ia < (long)i1 * v; ia += gridDim.x) {
    const int i = (int)(ia / v), a = (int)(ia % v);
    const double base = eps[c + a] - eps[i] + sh;
    const double* row = KK + ia * cv;
    for (int j = 0; j < c; ++j) {
      const double bj = base - eps[j];
      const double* rj = row + (long)j * v;
      for (int b = threadIdx.x; b < v; b += blockDim.x) {
        const double num = rj[b];
        const double D = bj + eps[c + b];
        const double inv = recip(D);
        const double x = num * inv;
        e += x;
        nr = fma(x, inv, nr);
        n3 = fma(x * inv, inv, n3);
        const unsigned long long db =
            (unsigned long long)__double_as_longlong(D) & 0x7FFFFFFFFFFFFFFFull;
        if ((__double_as_longlong(num) << 1) != 0 && db < dminb) dminb = db;
      }
    }
  }
  double dmin = dminb < 0x7FF0000000000000ull ? __longlong_as_double((long long)dminb) : 1e300;
  const int ncol = 3 * nshift + 1;
  double* out = partial + ((long)blockIdx.y * gridDim.x + blockIdx.x) * ncol;
  for (int t = threadIdx.x; t < 3 * nshift; t += blockDim.x) out[t] = 0.0;
  __syncthreads();
  e = block_sum(e, red);
  if (threadIdx.x == 0) out[k] = e;
  nr = block_sum(nr, red);
  if (threadIdx.x == 0) out[nshift + k] = nr;
  n3 = block_sum(n3, red);
  if (threadIdx.x == 0) out[2 * nshift + k] = n3;
  dmin = block_min(dmin, red);
  if (threadIdx.x == 0) out[3 * nshift] = dmin;
}

cudaError_t launch_eps_cv(const double* f, const Dims& d, double* eps, cudaStream_t s) {
  if (d.c + d.v == 0) return cudaSuccess;
  ++launch_counter();
  k_eps_cv<<<(d.c + d.v + 127) / 128, 128, 0, s>>>(f, d.nmo(), d.c, d.a, d.v, eps);
  return cudaGetLastError();
}

long classH_blocks(const Dims& d) {
  long ntile = (d.v + kHT - 1) / kHT;
  long npair = (long)d.c * (d.c + 1) / 2;
  return npair * (ntile * (ntile + 1) / 2);
}

int classH_nshift(const Dims& d, int scheme) { return scheme == CASPT2_SSSR ? 1 : d.n * d.n; }

cudaError_t launch_classH(const double* f, const double* B, const double* Ftil, const double* E0,
                          double shift, int scheme, const Dims& d, ClassHWork& w, int* status,
                          double* ecls, double* ncls, double* mom, double* mindenom,
                          cudaStream_t s, int i0, int i1) {
  const int n = d.n, nmo = d.nmo();
  const int nshift = classH_nshift(d, scheme);
  cudaError_t e;
  if (d.c == 0 || d.v == 0) {
    e = cudaMemsetAsync(ecls, 0, sizeof(double) * n * n, s);
    if (e != cudaSuccess) return e;
    return cudaMemsetAsync(ncls, 0, sizeof(double) * n, s);
  }
  ++launch_counter();
  k_eps_cv<<<(d.c + d.v + 127) / 128, 128, 0, s>>>(f, nmo, d.c, d.a, d.v, w.eps);
  long tp = (long)d.c * d.X * d.v;
  ++launch_counter();
  k_pack_cv<<<(int)std::min<long>((tp + 255) / 256, 152 * 32), 256, 0, s>>>(
      B, d.c, d.v, d.X, nmo, d.c + d.a, w.Bp);
  e = launch_sym_eig(Ftil, n, w.W, w.omega, 0, status, s);
  if (e != cudaSuccess) return e;
  ++launch_counter();
  k_classH_shifts<<<1, kMaxShift, 0, s>>>(w.omega, E0, shift, n, scheme, w.shifts);
  const int ntile = (d.v + kHT - 1) / kHT;
  if (i1 < 0 || i1 > d.c) i1 = d.c;
  // pairs (i <= j) with i in [i0, i1): a contiguous run of the row-major pair order
  auto start = [&](long i) { return i * d.c - i * (i - 1) / 2; };
  const long pair0 = start(i0), npair = start(i1) - start(i0);
  const long nb = npair * ((long)ntile * (ntile + 1) / 2);
  if (nb == 0) {
    e = cudaMemsetAsync(ecls, 0, sizeof(double) * n * n, s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(mom, 0, sizeof(double) * (n * n * n + n * n + n), s);
    if (e != cudaSuccess) return e;
    return cudaMemsetAsync(ncls, 0, sizeof(double) * n, s);
  }
  if (w.ev_gemm0) cudaEventRecord(w.ev_gemm0, s);
  ++launch_counter();
  k_classH<<<(unsigned)nb, kHThreads, 0, s>>>(w.Bp, w.eps, w.shifts, nshift, d.c, d.v, d.X, ntile,
                                             (int)pair0, w.partial);
  if (w.ev_gemm1) cudaEventRecord(w.ev_gemm1, s);
  const int ncol = 3 * nshift + 1;
  ++launch_counter();
  k_reduce_cols<<<ncol, 256, 0, s>>>(w.partial, nb, ncol, w.sums);
  ++launch_counter();
  k_classH_combine<<<1, 256, 0, s>>>(w.sums, w.W, n, scheme, ecls, ncls, mom, mindenom, status);
  return cudaGetLastError();
}

cudaError_t launch_classH_split(const double* f, const double* B, const double* Ftil,
                                const double* E0, double shift, int scheme, const Dims& d,
                                ClassHWork& w, int* status, double* ecls, double* ncls,
                                double* mom, double* mindenom, OzWork& oz, double* pack,
                                double* K, double* KK, cudaStream_t s, int i0, int i1) {
  const int n = d.n, nmo = d.nmo();
  const int nshift = classH_nshift(d, scheme);
  cudaError_t e;
  if (d.c == 0 || d.v == 0) {
    e = cudaMemsetAsync(ecls, 0, sizeof(double) * n * n, s);
    if (e != cudaSuccess) return e;
    return cudaMemsetAsync(ncls, 0, sizeof(double) * n, s);
  }
  ++launch_counter();
  k_eps_cv<<<(d.c + d.v + 127) / 128, 128, 0, s>>>(f, nmo, d.c, d.a, d.v, w.eps);
  e = launch_sym_eig(Ftil, n, w.W, w.omega, 0, status, s);
  if (e != cudaSuccess) return e;
  ++launch_counter();
  k_classH_shifts<<<1, kMaxShift, 0, s>>>(w.omega, E0, shift, n, scheme, w.shifts);
  const long cv = (long)d.c * d.v;
  if (i1 < 0 || i1 > d.c) i1 = d.c;
  if (i1 <= i0) {
    e = cudaMemsetAsync(ecls, 0, sizeof(double) * n * n, s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(mom, 0, sizeof(double) * (n * n * n + n * n + n), s);
    if (e != cudaSuccess) return e;
    return cudaMemsetAsync(ncls, 0, sizeof(double) * n, s);
  }
  if ((e = launch_pack_block(B, d, SP_C, SP_V, pack, s)) != cudaSuccess) return e;
  if (w.ev_gemm0) cudaEventRecord(w.ev_gemm0, s);
  // rows (ia) with i in [i0, i1) of K = Bcv^T Bcv (the whole K for the full range); the
  // exchange partner K(aj|bi) = K(bi|aj) lies in the same rows
  const long r0 = (long)i0 * d.v, nr = (long)(i1 - i0) * d.v;
  const OzView vp{pack, 1, cv, (long)d.X, 0};     // rows (ia), K = Q
  const OzView vr{pack + r0, 1, cv, (long)d.X, 0};
  if (nr == cv) {
    if ((e = oz_matmul(oz, vp, vp, true, (int)cv, (int)cv, d.X, 1.0, 0.0, K, cv, s)) != cudaSuccess)
      return e;
  } else if ((e = oz_matmul(oz, vr, vp, false, (int)nr, (int)cv, d.X, 1.0, 0.0, K + r0 * cv, cv,
                            s)) != cudaSuccess) {
    return e;
  }
  if (w.ev_gemm1) cudaEventRecord(w.ev_gemm1, s);
  const long total = nr * cv;
  ++launch_counter();
  k_classH_num<<<(int)std::min<long>((total + 255) / 256, 152L * 32), 256, 0, s>>>(K, d.c, d.v, i0,
                                                                                  i1, KK);
  const int nblk = (int)std::max<long>(1, std::min<long>(w.nblocks / nshift, 152L * 4));
  // one pass over b per (i, a, j) when v fits a block (no idle tail of lanes)
  const int hthreads = d.v <= 1024 ? std::max(64, (d.v + 31) / 32 * 32) : 256;
  ++launch_counter();
  k_classH_sums<<<dim3(nblk, nshift), hthreads, 0, s>>>(KK, w.eps, w.shifts, nshift, d.c, d.v, i0,
                                                        i1, w.partial);
  const int ncol = 3 * nshift + 1;
  ++launch_counter();
  k_reduce_cols<<<ncol, 256, 0, s>>>(w.partial, (long)nblk * nshift, ncol, w.sums);
  ++launch_counter();
  k_classH_combine<<<1, 256, 0, s>>>(w.sums, w.W, n, scheme, ecls, ncls, mom, mindenom, status);
  return cudaGetLastError();
}

}  // namespace caspt2
