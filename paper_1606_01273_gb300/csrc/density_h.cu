// Class H (E_ai,bj) share of the densities of a target state P (Sec. II.D).
//
// In the eigenbasis nu of U^T Fref U (W, omega) the first-order function of state L is a
// closed-shell pair function per nu with amplitudes
//   t(L, nu)   = W_Lnu u,  u = -K / D,  K_ij^ab = (ai|bj),
//   lam(L, nu) = (r_L c_nu + 2 E_s r_L^2 W_Lnu / D) u,   c = W^T r,  r = R[:, P],
//   D = e_a + e_b - e_i - e_j + sigma_(L,nu),  sigma = omega_nu - E0_L + E_s
// (SS-SR: nu = L, W = 1, sigma = E_s; the states then share one denominator and their
// lambda amplitudes add).  With tt = 2 t - t^(a<->b) the pieces are
//   d2_ab += 2 sum_s sum_ijc lam_s[ijac] tt_s[ijbc],  d2_ij -= 2 sum_s sum_kab lam_s[jkab] tt_s[ikab],
//   d2_rs += sum_(L,nu,nu') <lam_(L,nu)|tt_(L,nu')> <nu|E_rs|nu'> - N_L <L~|E_rs|L~>   (MS-MR),
//   GDF[Q][ia] = -2 sum_jb phi(D0) (2 K_ij^ab - K_ij^ba) B_Q,jb,
//   phi(D0) = sum_s alpha_s / D_s + beta_s / D_s^2,  alpha = 2 r_L c_nu W_Lnu, beta = 2 E_s r_L^2 W_Lnu^2,
// the last from the source multiplier w = r_L' sum_L r_L t + lam over the |L'~> component.
// K is formed once ([i][a][j][b], FP64 GEMM over the DF index); the d2 blocks are split-K
// Gram products per shift s.
#include <cmath>

#include "class_ag.cuh"
#include "class_dev.cuh"
#include "kernels.cuh"
#include "linalg.cuh"
#include "ozaki.cuh"

namespace caspt2 {

namespace {

// coef[s][6] = {sigma, alpha, beta, gamma, delta, wt} per pair s; returns through ns
// the number of pairs (n^2 under MS-MR, 1 under SS-SR).
__global__ void k_h_coef(const double* __restrict__ W, const double* __restrict__ shifts,
                         const double* __restrict__ R, int P, int n, int scheme, double shift,
                         double* __restrict__ coef) {
  const int idx = threadIdx.x;
  if (scheme == CASPT2_SSSR) {
    if (idx != 0) return;
    double r2 = 0.0;
    for (int L = 0; L < n; ++L) r2 += R[L * n + P] * R[L * n + P];
    double* o = coef;
    o[0] = shift;
    o[1] = 2.0 * r2;
    o[2] = 2.0 * shift * r2;
    o[3] = r2;
    o[4] = 2.0 * shift * r2;
    o[5] = 1.0;
    return;
  }
  if (idx >= n * n) return;
  const int L = idx / n, nu = idx % n;
  double cnu = 0.0;
  for (int N = 0; N < n; ++N) cnu += W[N * n + nu] * R[N * n + P];
  const double rl = R[L * n + P], wl = W[L * n + nu];
  double* o = coef + 6 * idx;
  o[0] = shifts[nu * n + L];
  o[1] = 2.0 * rl * cnu * wl;
  o[2] = 2.0 * shift * rl * rl * wl * wl;
  o[3] = rl * cnu;
  o[4] = 2.0 * shift * rl * rl * wl;
  o[5] = wl;
}

// Per element (ia, jb): Wt = phi(D0) (2K - K^x) and KK = K (2K - K^x), K^x = K_ij^ba.
__global__ void k_h_wt(const double* __restrict__ Kb, const double* __restrict__ eps, int c, int v,
                       const double* __restrict__ coef, int ns, double* __restrict__ Wt,
                       double* __restrict__ KK) {
  const long cv = (long)c * v;
  const long total = cv * cv;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    const long ia = e / cv, jb = e % cv;
    const int i = ia / v, a = ia % v, j = jb / v, b = jb % v;
    const double K = Kb[e];
    const double Kx = Kb[((long)i * v + b) * cv + (long)j * v + a];
    const double D0 = eps[c + a] + eps[c + b] - eps[i] - eps[j];
    double phi = 0.0;
    for (int s = 0; s < ns; ++s) {
      const double inv = 1.0 / (D0 + coef[6 * s]);
      phi += (coef[6 * s + 1] + coef[6 * s + 2] * inv) * inv;
    }
    const double tk = 2.0 * K - Kx;
    Wt[e] = phi * tk;
    KK[e] = K * tk;
  }
}

// Pair s: Lb = 2 lam_s = 2 (gamma + delta / D) (-K / D), Tb = tt_s = wt (-(2K - K^x) / D).
__global__ void k_h_lt(const double* __restrict__ Kb, const double* __restrict__ eps, int c, int v,
                       const double* __restrict__ cf, double* __restrict__ Lb,
                       double* __restrict__ Tb) {
  const long cv = (long)c * v;
  const long total = cv * cv;
  const double sig = cf[0], gam = cf[3], del = cf[4], wt = cf[5];
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    const long ia = e / cv, jb = e % cv;
    const int i = ia / v, a = ia % v, j = jb / v, b = jb % v;
    const double K = Kb[e];
    const double Kx = Kb[((long)i * v + b) * cv + (long)j * v + a];
    const double inv = 1.0 / (eps[c + a] + eps[c + b] - eps[i] - eps[j] + sig);
    Lb[e] = -2.0 * (gam + del * inv) * K * inv;
    Tb[e] = -wt * (2.0 * K - Kx) * inv;
  }
}

// Sums over all elements of KK / (D1 D2) and KK / (D1^2 D2) for every triple
// (L, nu, nu'), D1 = D0 + sigma_(L,nu), D2 = D0 + sigma_(L,nu').  grid = (blocks, n^3);
// part[triple][block][2].
__global__ void k_h_ov(const double* __restrict__ KK, const double* __restrict__ eps, int c, int v,
                       const double* __restrict__ coef, int n, double* __restrict__ part) {
  __shared__ double red[32];
  const int tr = blockIdx.y;
  const int L = tr / (n * n), nu = (tr / n) % n, nu2 = tr % n;
  const double s1 = coef[6 * (L * n + nu)], s2 = coef[6 * (L * n + nu2)];
  const long cv = (long)c * v;
  const long total = cv * cv;
  double sa = 0.0, sb = 0.0;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    const long ia = e / cv, jb = e % cv;
    const int i = ia / v, a = ia % v, j = jb / v, b = jb % v;
    const double D0 = eps[c + a] + eps[c + b] - eps[i] - eps[j];
    const double i1 = 1.0 / (D0 + s1), i2 = 1.0 / (D0 + s2);
    const double x = KK[e] * i1 * i2;
    sa += x;
    sb += x * i1;
  }
  sa = block_sum(sa, red);
  sb = block_sum(sb, red);
  if (threadIdx.x == 0) {
    double* o = part + ((long)tr * gridDim.x + blockIdx.x) * 2;
    o[0] = sa;
    o[1] = sb;
  }
}

// Same sums for n <= NM with one division per (element, shift): grid = (blocks, n), block
// y = L; every thread holds 1 / (D0 + sigma_(L,nu)) for all nu and accumulates the 2 n^2
// pair sums in registers.  part[(L, nu, nu')][block][2] as above.
template <int NM>
__global__ void k_h_ov_reg(const double* __restrict__ KK, const double* __restrict__ eps, int c,
                           int v, const double* __restrict__ coef, int n,
                           double* __restrict__ part) {
  __shared__ double red[32];
  const int L = blockIdx.y;
  double sig[NM];
#pragma unroll
  for (int q = 0; q < NM; ++q) sig[q] = q < n ? coef[6 * (L * n + q)] : 0.0;
  double sa[NM][NM], sb[NM][NM];
#pragma unroll
  for (int p = 0; p < NM; ++p)
#pragma unroll
    for (int q = 0; q < NM; ++q) sa[p][q] = sb[p][q] = 0.0;
  const long cv = (long)c * v;
  const long total = cv * cv;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    const long ia = e / cv, jb = e % cv;
    const int i = ia / v, a = ia % v, j = jb / v, b = jb % v;
    const double D0 = eps[c + a] + eps[c + b] - eps[i] - eps[j];
    const double kk = KK[e];
    double inv[NM];
#pragma unroll
    for (int q = 0; q < NM; ++q) inv[q] = q < n ? 1.0 / (D0 + sig[q]) : 0.0;
#pragma unroll
    for (int p = 0; p < NM; ++p) {
      const double x1 = kk * inv[p];
#pragma unroll
      for (int q = 0; q < NM; ++q) {
        const double x = x1 * inv[q];
        sa[p][q] += x;
        sb[p][q] += x * inv[p];
      }
    }
  }
#pragma unroll
  for (int p = 0; p < NM; ++p)
#pragma unroll
    for (int q = 0; q < NM; ++q) {
      if (p >= n || q >= n) continue;
      const double ta = block_sum(sa[p][q], red);
      const double tb = block_sum(sb[p][q], red);
      if (threadIdx.x == 0) {
        double* o = part + ((long)((L * n + p) * n + q) * gridDim.x + blockIdx.x) * 2;
        o[0] = ta;
        o[1] = tb;
      }
    }
}

// Active block: d2[c + r][c + s] += sum_(L,nu,nu') W_Lnu' (gamma Sa + delta Sb)_(L,nu)
// g1nu[nu][nu'][rs] - sum_L NL[L] Gamma1[L][L][rs],  g1nu = W^T Gamma1 W.
__global__ void k_h_act_finish(const double* __restrict__ part, int nblk,
                               const double* __restrict__ coef, const double* __restrict__ W,
                               const double* __restrict__ g1, const double* __restrict__ NL,
                               int n, int a, int c, int nmo, double* __restrict__ d2) {
  __shared__ double ov[kMaxStates * kMaxStates * kMaxStates];
  const int n3 = n * n * n;
  for (int tr = threadIdx.x; tr < n3; tr += blockDim.x) {
    double sa = 0.0, sb = 0.0;
    for (int b = 0; b < nblk; ++b) {
      sa += part[((long)tr * nblk + b) * 2];
      sb += part[((long)tr * nblk + b) * 2 + 1];
    }
    const int L = tr / (n * n), nu = (tr / n) % n, nu2 = tr % n;
    const double* cf = coef + 6 * (L * n + nu);
    ov[tr] = W[L * n + nu2] * (cf[3] * sa + cf[4] * sb);
  }
  __syncthreads();
  const int a2 = a * a;
  for (int rs = threadIdx.x; rs < a2; rs += blockDim.x) {
    double acc = 0.0;
    for (int tr = 0; tr < n3; ++tr) {
      const int nu = (tr / n) % n, nu2 = tr % n;
      double g = 0.0;
      for (int M = 0; M < n; ++M)
        for (int N = 0; N < n; ++N)
          g += W[M * n + nu] * W[N * n + nu2] * g1[((long)M * n + N) * a2 + rs];
      acc += ov[tr] * g;
    }
    for (int L = 0; L < n; ++L) acc -= NL[L] * g1[((long)L * n + L) * a2 + rs];
    d2[(long)(c + rs / a) * nmo + c + rs % a] += acc;
  }
}

}  // namespace

int classH_densities(const double* B, const Dims& d, const ClassHWork& hw, int scheme,
                     double shift, const double* R, int P, const double* NL, const double* g1,
                     const HDensWork& hd, double* d2, double* gdf, OzWork* oz, bool k_ready,
                     cudaStream_t s) {
  const int c = d.c, v = d.v, n = d.n, a = d.a, nmo = d.nmo();
  if (c == 0 || v == 0) return CASPT2_OK;
  const long cv = (long)c * v, total = cv * cv;
  if (total > hd.size) return CASPT2_EINVAL;
  const int ns = scheme == CASPT2_SSSR ? 1 : n * n;
  ++launch_counter();
  k_h_coef<<<1, kMaxStates * kMaxStates, 0, s>>>(hw.W, hw.shifts, R, P, n, scheme, shift, hd.coef);
  CASPT2_CUDA_TRY(cudaGetLastError());
  const bool split = oz && oz->on;
  // K[(ia)][(jb)] = sum_Q B[Q][i][a] B[Q][j][b]
  CASPT2_CUDA_TRY(launch_pack_block(B, d, SP_C, SP_V, hd.pack, s));
  if (!k_ready) {
    if (split) {
      const OzView vp{hd.pack, 1, cv, (long)d.X, 0};     // rows (ia), K = Q
      CASPT2_CUDA_TRY(oz_matmul(*oz, vp, vp, true, (int)cv, (int)cv, d.X, 1.0, 0.0, hd.K, cv, s));
    } else {
      CASPT2_CUDA_TRY(dgemm((int)cv, (int)cv, d.X, 1.0, hd.pack, (int)cv, true, hd.pack, (int)cv,
                            false, 0.0, hd.K, (int)cv, s));
    }
  }
  ++launch_counter();
  k_h_wt<<<launch_blocks(total), 256, 0, s>>>(hd.K, hw.eps, c, v, hd.coef, ns, hd.B1, hd.B2);
  CASPT2_CUDA_TRY(cudaGetLastError());
  // GDF[Q][i][a] += -2 sum_jb B[Q][jb] Wt[ia][jb]
  if (split) {
    const OzView vq{hd.pack, cv, 1, cv, 0}, vw{hd.B1, cv, 1, cv, 0};   // rows Q / (ia), K = (jb)
    CASPT2_CUDA_TRY(oz_matmul(*oz, vq, vw, false, d.X, (int)cv, (int)cv, -2.0, 0.0, hd.tmp, cv, s));
  } else {
    CASPT2_CUDA_TRY(dgemm(d.X, (int)cv, (int)cv, -2.0, hd.pack, (int)cv, false, hd.B1, (int)cv,
                          true, 0.0, hd.tmp, (int)cv, s));
  }
  CASPT2_CUDA_TRY(launch_unpack_add(hd.tmp, d, SP_C, SP_V, gdf, s));
  // active block (MS-MR): pairs nu, nu' of the same state through <nu|E_rs|nu'>
  if (scheme != CASPT2_SSSR && a > 0) {
    const int nblk = (int)std::min<long>(n <= 4 ? 152L * 2 : 64L, (total + 255) / 256);
    const int n3 = n * n * n;
    if ((long)n3 * nblk * 2 > hd.partmax) return CASPT2_EINVAL;
    ++launch_counter();
    if (n <= 4)
      k_h_ov_reg<4><<<dim3(nblk, n), 256, 0, s>>>(hd.B2, hw.eps, c, v, hd.coef, n, hd.part);
    else
      k_h_ov<<<dim3(nblk, n3), 256, 0, s>>>(hd.B2, hw.eps, c, v, hd.coef, n, hd.part);
    ++launch_counter();
    k_h_act_finish<<<1, 256, 0, s>>>(hd.part, nblk, hd.coef, hw.W, g1, NL, n, a, c, nmo, d2);
    CASPT2_CUDA_TRY(cudaGetLastError());
  }
  // closed and virtual blocks, one Gram product per pair s
  for (int q = 0; q < ns; ++q) {
    ++launch_counter();
    k_h_lt<<<launch_blocks(total), 256, 0, s>>>(hd.K, hw.eps, c, v, hd.coef + 6 * q, hd.B1, hd.B2);
    CASPT2_CUDA_TRY(cudaGetLastError());
    int st = gram_product(hd.B1, hd.B2, c, v, cv, 2, d2, nmo, c + a, hd.part, hd.partmax, s, oz);
    if (st != CASPT2_OK) return st;
    st = gram_product(hd.B1, hd.B2, 1, c, (long)v * cv, 1, d2, nmo, 0, hd.part, hd.partmax, s, oz);
    if (st != CASPT2_OK) return st;
  }
  return CASPT2_OK;
}

}  // namespace caspt2
