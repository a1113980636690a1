// Internal launcher declarations (host side) for the CASPT2 kernels.
#pragma once
#include "common.cuh"

namespace caspt2 {

struct Dims {
  int c, a, v, X, n;
  __host__ __device__ int nmo() const { return c + a + v; }
};

// Host check of the Fock matrix the solve accepts (api.cu): symmetric, with zero
// closed-active, active-virtual and closed-virtual blocks and diagonal closed and
// virtual blocks, each to 1e-10 x max(1, max|f|).  f is a host copy [nmo][nmo].
// Returns CASPT2_OK, CASPT2_EINVAL (coupling found) or CASPT2_ENAN.
int check_block_diagonal_fock(const double* f, const Dims& d);

// ---- canonical closed and virtual orbitals (canon.cu) ------------------------
// Host classification of f [nmo][nmo]: 0 = block diagonal with diagonal closed and
// virtual blocks; 1 = no closed-active, active-virtual or closed-virtual coupling but an
// off-diagonal closed-closed or virtual-virtual entry (tolerance as above); CASPT2_EINVAL
// (asymmetric, or coupling between the spaces) or CASPT2_ENAN.
int classify_fock(const double* f, const Dims& d);
// Rotate the device inputs in place to the eigenvectors of f's closed and virtual blocks:
// C [nmo][nmo] = blockdiag(Q_c, 1, Q_v), f <- canonical part of C^T f C, B_P <- C^T B_P C.
// Synchronises s.  Returns CASPT2_OK, ENOMEM, ENOTCONV, ENAN or ECUDA.
int canonicalize_inputs(double* f, double* B, const Dims& d, double* C, cudaStream_t s);
// out[b] = C M[b] C^T for `batch` nmo x nmo matrices (tmp: batch * nmo^2 doubles).
cudaError_t canon_back(const double* C, const double* M, int nmo, int batch, double* tmp,
                       double* out, cudaStream_t s);

// ---- setup (setup.cu) --------------------------------------------------------
// d_act = (1/n) sum_N rdm1[N][N]                         (Sec. II.B, d^(0)sa)
cudaError_t launch_dsa(const double* rdm1, const Dims& d, double* dact, cudaStream_t s);
// g = g(d_act) over all nmo x nmo (Sec. II.B, g(d) with d nonzero in the active block)
cudaError_t launch_gmat(const double* B, const double* dact, const Dims& d, double* gam,
                        double* Y, double* g, cudaStream_t s);
// E_core = <core|H|core>, with h = f - g(d_sa)
cudaError_t launch_ecore(const double* f, const double* g, const double* B, const Dims& d,
                         double* bsum, double* bfro, double* ecore, cudaStream_t s);
// Fref[M][N] = sum_rs f_rs rdm1[M][N][r][s]             (Sec. II.A, XMS Fock)
cudaError_t launch_fref(const double* f, const double* rdm1, const Dims& d, double* fref,
                        cudaStream_t s);
// symmetric eigenpairs of an n x n matrix (n <= 16), ascending, canonical column signs
cudaError_t launch_sym_eig(const double* A, int n, double* V, double* w, int identity,
                           int* status, cudaStream_t s);
// out = U^T A U (n x n)
cudaError_t launch_congruence(const double* A, const double* U, int n, double* out,
                              cudaStream_t s);
// E0[L] = out[L][L]
cudaError_t launch_diag(const double* A, int n, double* e0, cudaStream_t s);
// dst[M][N][e] = sum_KL U[K][M] U[L][N] src[K][L][e]     (Sec. II.A, rotated RDMs)
cudaError_t launch_rotate_rdm(const double* src, const double* U, int n, long len, double* dst,
                              cudaStream_t s);
// eri[r][s][t][u] = (rs|tu) over the active block
cudaError_t launch_eri_act(const double* B, const Dims& d, double* eri, cudaStream_t s);
// H^ref_MN = d_MN (E_core + E_nuc) + sum fc_rs G1~ + 1/2 sum (rs|tu) G2~      (Sec. II.A)
cudaError_t launch_href(const double* f, const double* g, const double* rdm1r, const double* rdm2r,
                        const double* eri, const double* ecore, double enuc, const Dims& d,
                        double* href, cudaStream_t s);
// H^eff = H^ref + 1/2 (e + e^T) - diag(E_s * norm) summed over enabled classes (Sec. II.B)
cudaError_t launch_heff(const double* href, const double* ecls, const double* ncls, unsigned mask,
                        double shift, int n, double* heff, cudaStream_t s);

// ---- class H (class_h.cu) ----------------------------------------------------
struct ClassHWork {
  double* Bp;        // [c][X][v]   packed (ai|P) factors
  double* eps;       // [nmo]       diagonal of f
  double* W;         // [n][n]      eigenvectors of U^T Fref U
  double* omega;     // [n]
  double* shifts;    // [nshift]    omega_nu - E0_L + E_s
  double* partial;   // [nblocks][3*nshift + 1]
  double* sums;      // [3*nshift + 1]
  long    nblocks;
  cudaEvent_t ev_gemm0 = nullptr, ev_gemm1 = nullptr;  // optional: bracket the GEMM kernel
};
long classH_blocks(const Dims& d);

// Work space of the class-H densities: K, B1, B2 hold (c v)^2 doubles each (size),
// pack and tmp X c v, coef 6 n^2, part partmax.
struct HDensWork {
  double *K = nullptr, *B1 = nullptr, *B2 = nullptr, *pack = nullptr, *tmp = nullptr,
         *coef = nullptr, *part = nullptr;
  long size = 0, partmax = 0;
};
// Class-H share of d2 (closed, active, virtual blocks) and GDF of target state P
// (Sec. II.D), accumulated; needs the W, shifts and eps left by launch_classH.
struct OzWork;
// Class H with K[(ia)][(jb)] (cv x cv, in K) formed by the split BF16 tensor-core GEMM
// and the energy sums taken over the stored matrix (KK: cv x cv work, pack: X c v).
cudaError_t launch_classH_split(const double* f, const double* B, const double* Ftil,
                                const double* E0, double shift, int scheme, const Dims& d,
                                ClassHWork& w, int* status, double* ecls, double* ncls,
                                double* mom, double* mindenom, OzWork& oz, double* pack,
                                double* K, double* KK, cudaStream_t s, int i0 = 0, int i1 = -1);
// oz (optional, on): the DF and Gram products run as split BF16 GEMMs; k_ready: hd.K
// already holds K[(ia)][(jb)] (formed by the split class-H energy path).
int classH_densities(const double* B, const Dims& d, const ClassHWork& hw, int scheme,
                     double shift, const double* R, int P, const double* NL, const double* g1,
                     const HDensWork& hd, double* d2, double* gdf, OzWork* oz, bool k_ready,
                     cudaStream_t s);
// eps[0..c) closed and eps[c..c+v) virtual orbital energies (diagonal of f)
cudaError_t launch_eps_cv(const double* f, const Dims& d, double* eps, cudaStream_t s);
// out[r][s] = f[c + r][c + s] (active block, compact)
cudaError_t launch_active_block(const double* f, const Dims& d, double* out, cudaStream_t s);
int  classH_nshift(const Dims& d, int scheme);
cudaError_t launch_classH(const double* f, const double* B, const double* Ftil, const double* E0,
                          double shift, int scheme, const Dims& d, ClassHWork& w, int* status,
                          double* ecls, double* ncls, double* mom, double* mindenom,
                          cudaStream_t s, int i0 = 0, int i1 = -1);

}  // namespace caspt2
