// Energy gradient of the target MS state with respect to the library's inputs f and B
// (Sec. II.D densities chained through the definitions the solve uses), reference RDMs
// held fixed, for MS (U = 1; the XMS rotation response is not formed).
//
// With h = f - g(B, d_sa) (d_sa: closed 2 delta + state-averaged active 1-RDM) the solve's
// energy E = R_P^T H^eff R_P depends on
//   h      through the sources (d1) and H^ref (gamma_P = <P|E_xy|P>, closed 2 delta);
//   f      through eps_i, eps_a, F_act and E0 (d2 on the closed-closed, active-active and
//          virtual-virtual blocks: the blocks of an f without coupling between the spaces,
//          whose closed and virtual parts the solve takes through their eigenvalues);
//   B      through the (pq|rt) blocks and class H (Gamma), H^ref at fixed h (core energy,
//          g(d_core) and the active 2-electron term), and h.
// Hence
//   dE/df = gamma_P + d1 + d2 on those blocks
//   dE/dB_Qpq = Gamma_Qpq + ref_Qpq - [D_pq Gd_Q + dsa_pq GD_Q - (M_Q + M_Q^T)_pq / 2],
//   D = gamma_P + d1, Gd_Q = sum B_Q dsa, GD_Q = sum B_Q D, M_Q = D B_Q dsa,
// ref_Qpq the derivative of <P|H|P> at fixed h:
//   closed p, q: 4 bsum_Q delta_pq - 2 B_Qqp + 2 t_Q delta_pq  (t_Q = sum_rs G1_rs B_Qrs)
//   active r, s: 2 bsum_Q G1_rs + sum_tu G2_rstu B_Qtu
//   active r, closed j: -sum_s G1_rs B_Qjs;  closed j, active s: -sum_r G1_rs B_Qrj
// with G1, G2 the target state's active 1- and 2-RDMs (sum_MN R_MP R_NP Gamma^MN).
// Both gradients are returned symmetrised.
#include "class_ag.cuh"
#include "class_dev.cuh"
#include "kernels.cuh"
#include "linalg.cuh"

namespace caspt2 {

namespace {

// G1[rs] = sum_MN R_MP R_NP rdm1[M][N][rs], G2[rstu] likewise from rdm2.
__global__ void k_target_rdms(const double* __restrict__ rdm1, const double* __restrict__ rdm2,
                              const double* __restrict__ R, int P, int n, int a,
                              double* __restrict__ g1, double* __restrict__ g2) {
  const long a2 = (long)a * a, a4 = a2 * a2;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < a2 + a4;
       e += (long)gridDim.x * blockDim.x) {
    const bool one = e < a2;
    const long k = one ? e : e - a2;
    const double* src = one ? rdm1 : rdm2;
    const long len = one ? a2 : a4;
    double acc = 0.0;
    for (int M = 0; M < n; ++M)
      for (int N = 0; N < n; ++N) acc += R[M * n + P] * R[N * n + P] * src[((long)M * n + N) * len + k];
    if (one) g1[k] = acc;
    else g2[k] = acc;
  }
}

// D = gamma_P + d1 (full nmo x nmo), dsa (closed 2, active d_act) and
// grad_f = gamma_P + d1 + d2 on the blocks of f the solve takes.
__global__ void k_grad_f(const double* __restrict__ d1, const double* __restrict__ d2,
                         const double* __restrict__ g1, const double* __restrict__ dact, int c,
                         int a, int nmo, double* __restrict__ D, double* __restrict__ dsa,
                         double* __restrict__ gf) {
  const long total = (long)nmo * nmo;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    const int x = e / nmo, y = e % nmo;
    const bool xc = x < c, yc = y < c, xa = x >= c && x < c + a, ya = y >= c && y < c + a;
    double gp = 0.0, ds = 0.0;
    if (xc && yc && x == y) gp = ds = 2.0;
    if (xa && ya) {
      gp = g1[(x - c) * a + (y - c)];
      ds = dact[(x - c) * a + (y - c)];
    }
    // the closed-closed, active-active and virtual-virtual blocks (an f without coupling
    // between the spaces: off-diagonal closed/virtual entries are solved through the
    // canonical orbitals of those blocks)
    const bool xv = x >= c + a, yv = y >= c + a;
    const bool read = (xa && ya) || (xc && yc) || (xv && yv);
    D[e] = gp + d1[e];
    dsa[e] = ds;
    gf[e] = gp + d1[e] + (read ? d2[e] : 0.0);
  }
}

// Per Q: GD_Q = sum_xy D_xy B_Qxy and t_Q = sum_rs G1_rs B_Q[c+r][c+s].
__global__ void k_grad_scalars(const double* __restrict__ B, const double* __restrict__ D,
                               const double* __restrict__ g1, int c, int a, int nmo,
                               double* __restrict__ gD, double* __restrict__ tq) {
  __shared__ double red[32];
  const int Q = blockIdx.x;
  const double* Bq = B + (long)Q * nmo * nmo;
  double s1 = 0.0, s2 = 0.0;
  for (long e = threadIdx.x; e < (long)nmo * nmo; e += blockDim.x) s1 += D[e] * Bq[e];
  for (int rs = threadIdx.x; rs < a * a; rs += blockDim.x)
    s2 += g1[rs] * Bq[(long)(c + rs / a) * nmo + c + rs % a];
  s1 = block_sum(s1, red);
  if (threadIdx.x == 0) gD[Q] = s1;
  s2 = block_sum(s2, red);
  if (threadIdx.x == 0) tq[Q] = s2;
}

// T_Q = B_Q dsa: columns of closed j are 2 B_Q[:, j], active columns B_Q[:, act] d_act.
__global__ void k_b_dsa(const double* __restrict__ B, const double* __restrict__ dact, int X,
                        int c, int a, int nmo, double* __restrict__ T) {
  const long total = (long)X * nmo * nmo;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    const int y = e % nmo;
    const long row = e - y;                       // start of row x of matrix Q
    double v = 0.0;
    if (y < c) v = 2.0 * B[e];
    else if (y < c + a) {
      for (int u = 0; u < a; ++u) v += B[row + c + u] * dact[u * a + (y - c)];
    }
    T[e] = v;
  }
}

// grad_B[Q][p][q] = Gamma + ref - [D Gd_Q + dsa GD_Q - (M + M^T)/2] (symmetrised later).
__global__ void k_grad_b(const double* __restrict__ B, const double* __restrict__ gdf,
                         const double* __restrict__ D, const double* __restrict__ dsa,
                         const double* __restrict__ Mq, const double* __restrict__ g1,
                         const double* __restrict__ g2, const double* __restrict__ bsum,
                         const double* __restrict__ gam, const double* __restrict__ gD,
                         const double* __restrict__ tq, int X, int c, int a, int nmo,
                         double* __restrict__ gb) {
  const long nn = (long)nmo * nmo, total = (long)X * nn;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    const long Q = e / nn, pq = e % nn;
    const int p = pq / nmo, q = pq % nmo;
    const double* Bq = B + Q * nn;
    const bool pc = p < c, qc = q < c;
    const bool pa = p >= c && p < c + a, qa = q >= c && q < c + a;
    double ref = 0.0;
    if (pc && qc) {
      ref = -2.0 * Bq[(long)q * nmo + p];
      if (p == q) ref += 4.0 * bsum[Q] + 2.0 * tq[Q];
    } else if (pa && qa) {
      const int r = p - c, s = q - c;
      ref = 2.0 * bsum[Q] * g1[r * a + s];
      const double* g2rs = g2 + ((long)r * a + s) * a * a;
      for (int tu = 0; tu < a * a; ++tu) ref += g2rs[tu] * Bq[(long)(c + tu / a) * nmo + c + tu % a];
    } else if (pa && qc) {
      const int r = p - c;
      for (int s = 0; s < a; ++s) ref -= g1[r * a + s] * Bq[(long)q * nmo + c + s];
    } else if (pc && qa) {
      const int s = q - c;
      for (int r = 0; r < a; ++r) ref -= g1[r * a + s] * Bq[(long)(c + r) * nmo + p];
    }
    const double gd = 2.0 * bsum[Q] + (a > 0 ? gam[Q] : 0.0);
    const double term = D[pq] * gd + dsa[pq] * gD[Q] -
                        0.5 * (Mq[Q * nn + pq] + Mq[Q * nn + (long)q * nmo + p]);
    gb[e] = gdf[e] + ref - term;
  }
}

// Orbital derivative (Sec. II.D, Eq. orbderiv): dL/dh over every block,
// gf = gamma_P + d1 + d2, and D = -d2, the density whose mean-field derivative
// k_grad_b subtracts (so that it adds d2 : dg(B, d_sa)/dB, the f = h + g(B, d_sa) chain at
// fixed h); dsa as k_grad_f.
__global__ void k_orb_prep(const double* __restrict__ d1, const double* __restrict__ d2,
                           const double* __restrict__ g1, const double* __restrict__ dact, int c,
                           int a, int nmo, double* __restrict__ D, double* __restrict__ dsa,
                           double* __restrict__ gf) {
  const long total = (long)nmo * nmo;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    const int x = e / nmo, y = e % nmo;
    const bool xc = x < c, yc = y < c, xa = x >= c && x < c + a, ya = y >= c && y < c + a;
    double gp = 0.0, ds = 0.0;
    if (xc && yc && x == y) gp = ds = 2.0;
    if (xa && ya) {
      gp = g1[(x - c) * a + (y - c)];
      ds = dact[(x - c) * a + (y - c)];
    }
    D[e] = -d2[e];
    dsa[e] = ds;
    gf[e] = gp + d1[e] + d2[e];
  }
}

// Y[e] += alpha * sum_b part[b][e], b in increasing order.
__global__ void k_add_partials(const double* __restrict__ part, int nparts, long len,
                               double alpha, double* __restrict__ Y) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < len;
       e += (long)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int b = 0; b < nparts; ++b) acc += part[(long)b * len + e];
    Y[e] += alpha * acc;
  }
}

}  // namespace

int assemble_gradient(const Dims& d, const double* B, const double* R, int P,
                      const double* rdm1, const double* rdm2, const double* dact,
                      const double* bsum, const double* gam, const double* d1, const double* d2,
                      const double* gdf, const GradWork& gw, double* grad_f, double* grad_B,
                      cudaStream_t s) {
  const int nmo = d.nmo(), c = d.c, a = d.a, n = d.n;
  const long nn = (long)nmo * nmo;
  const long a2 = (long)a * a;
  if (a > 0) {
    ++launch_counter();
    k_target_rdms<<<launch_blocks(a2 + a2 * a2), 256, 0, s>>>(rdm1, rdm2, R, P, n, a, gw.g1, gw.g2);
  }
  ++launch_counter();
  k_grad_f<<<launch_blocks(nn), 256, 0, s>>>(d1, d2, gw.g1, dact, c, a, nmo, gw.D, gw.dsa, grad_f);
  ++launch_counter();
  k_grad_scalars<<<d.X, 256, 0, s>>>(B, gw.D, gw.g1, c, a, nmo, gw.gD, gw.tq);
  ++launch_counter();
  k_b_dsa<<<launch_blocks((long)d.X * nn), 256, 0, s>>>(B, dact, d.X, c, a, nmo, gw.T);
  CASPT2_CUDA_TRY(cudaGetLastError());
  // M_Q = D T_Q for every Q (batched FP64 GEMM)
  CASPT2_CUDA_TRY(dgemm(nmo, nmo, nmo, 1.0, gw.D, nmo, false, gw.T, nmo, false, 0.0, gw.M, nmo, s,
                        d.X, 0, nn, nn));
  ++launch_counter();
  k_grad_b<<<launch_blocks((long)d.X * nn), 256, 0, s>>>(B, gdf, gw.D, gw.dsa, gw.M, gw.g1, gw.g2,
                                                         bsum, gam, gw.gD, gw.tq, d.X, c, a, nmo,
                                                         grad_B);
  CASPT2_CUDA_TRY(cudaGetLastError());
  CASPT2_CUDA_TRY(launch_symmetrize(grad_f, nmo, 1, s));
  CASPT2_CUDA_TRY(launch_symmetrize(grad_B, nmo, d.X, s));
  return CASPT2_OK;
}

}  // namespace caspt2

namespace caspt2 {

// Y = 2 [h gf + sum_Q B_Q gBh_Q], gf = dL/dh and gBh = dL/dB at fixed h, both over every
// block (see k_orb_prep).  Under phi'_y = phi_y + sum_x phi_x k_xy the integrals change as
// h' = C^T h C and B'_Q = C^T B_Q C (C = 1 + k); with symmetric h, B_Q, gf and gBh_Q the
// first-order change of L is sum_xy k_xy Y_xy.
int assemble_orbital_derivative(const Dims& d, const double* f, const double* g_act,
                                const double* B, const double* R, int P, const double* rdm1,
                                const double* rdm2, const double* dact, const double* bsum,
                                const double* gam, const double* d1, const double* d2,
                                const double* gdf, const GradWork& gw, double* h, double* gf,
                                double* gBh, double* Y, cudaStream_t s) {
  const int nmo = d.nmo(), c = d.c, a = d.a, n = d.n;
  const long nn = (long)nmo * nmo;
  const long a2 = (long)a * a;
  if (a > 0) {
    ++launch_counter();
    k_target_rdms<<<launch_blocks(a2 + a2 * a2), 256, 0, s>>>(rdm1, rdm2, R, P, n, a, gw.g1, gw.g2);
  }
  ++launch_counter();
  k_orb_prep<<<launch_blocks(nn), 256, 0, s>>>(d1, d2, gw.g1, dact, c, a, nmo, gw.D, gw.dsa, gf);
  ++launch_counter();
  k_grad_scalars<<<d.X, 256, 0, s>>>(B, gw.D, gw.g1, c, a, nmo, gw.gD, gw.tq);
  ++launch_counter();
  k_b_dsa<<<launch_blocks((long)d.X * nn), 256, 0, s>>>(B, dact, d.X, c, a, nmo, gw.T);
  CASPT2_CUDA_TRY(cudaGetLastError());
  CASPT2_CUDA_TRY(dgemm(nmo, nmo, nmo, 1.0, gw.D, nmo, false, gw.T, nmo, false, 0.0, gw.M, nmo, s,
                        d.X, 0, nn, nn));
  ++launch_counter();
  k_grad_b<<<launch_blocks((long)d.X * nn), 256, 0, s>>>(B, gdf, gw.D, gw.dsa, gw.M, gw.g1, gw.g2,
                                                         bsum, gam, gw.gD, gw.tq, d.X, c, a, nmo,
                                                         gBh);
  CASPT2_CUDA_TRY(cudaGetLastError());
  CASPT2_CUDA_TRY(launch_symmetrize(gf, nmo, 1, s));
  CASPT2_CUDA_TRY(launch_symmetrize(gBh, nmo, d.X, s));
  // h = f - g(d_sa) over all orbital pairs (plain FP64 form)
  CASPT2_CUDA_TRY(launch_hcore(f, g_act, B, bsum, d, h, s, nullptr, nullptr));
  CASPT2_CUDA_TRY(dgemm(nmo, nmo, nmo, 2.0, h, nmo, false, gf, nmo, false, 0.0, Y, nmo, s));
  // sum_Q B_Q gBh_Q = B^T gBh with B and gBh read as (X nmo) x nmo matrices (row (Q, q));
  // partial products over chunks of Q (into gw.M, free again) summed in chunk order
  const int nb = std::min(d.X, 32);
  const int chunk = (d.X + nb - 1) / nb;
  const int nfull = d.X / chunk, rem = d.X - nfull * chunk;
  const long cstr = (long)chunk * nn;
  CASPT2_CUDA_TRY(dgemm(nmo, nmo, chunk * nmo, 1.0, B, nmo, true, gBh, nmo, false, 0.0, gw.M, nmo,
                        s, nfull, cstr, cstr, nn));
  if (rem > 0)
    CASPT2_CUDA_TRY(dgemm(nmo, nmo, rem * nmo, 1.0, B + nfull * cstr, nmo, true, gBh + nfull * cstr,
                          nmo, false, 0.0, gw.M + (long)nfull * nn, nmo, s));
  ++launch_counter();
  k_add_partials<<<launch_blocks(nn), 256, 0, s>>>(gw.M, nfull + (rem > 0 ? 1 : 0), nn, 2.0, Y);
  CASPT2_CUDA_TRY(cudaGetLastError());
  return CASPT2_OK;
}

}  // namespace caspt2
