// Classes A-G (internal): device structures and the per-class solve.
#pragma once
#include <vector>

#include "kernels.cuh"
#include "linalg.cuh"
#include "ozaki.cuh"
#include "terms.h"

namespace caspt2 {

struct DevClass {
  int nfam, nslot, next, nact;
  int slot_space[4];
  int ext[3], act[3];
  int pair0, pair1;
};

struct RdmPtrs { const double* p[5]; };      // p[k] = rotated k-RDM [n][n][a^{2k}]
struct EriBlocks { const double* p[81]; };   // (pq|rt) blocks keyed by the spaces of p,q,r,t
struct ExtDims { int d[3]; };
constexpr int kMaxPresum = 64;
struct PresumBlocks { const double* p[kMaxPresum]; };   // pre-summed (pq|rt) blocks by spec

__device__ __forceinline__ void atomicMin_double(double* addr, double v) {
  if (!(v >= 0.0)) return;
  atomicMin(reinterpret_cast<unsigned long long*>(addr),
            static_cast<unsigned long long>(__double_as_longlong(v)));
}

// Sector eigenbasis kept from the energy pass for the densities: Y (msec x nk, the
// first nk columns used), omega (nk) and the sources Vt = Y^T V (nk x ntup * n).
struct SectorKeep {
  int sec = 0, Lsel = -1, msec = 0, nk = 0;
  long ntup = 0;
  double *Y = nullptr, *omega = nullptr, *Vt = nullptr;
};

struct ClassWork {
  int cls = -1;
  DevClass dc{};
  int m = 0;             // nfam * a^nact * n
  long A = 0;            // a^nact
  ExtDims ed{};
  long vsize = 0;
  ActPlan* dS = nullptr; int nS = 0;
  ActPlan* dF = nullptr; int nF = 0;
  SrcPlan* dV = nullptr; int nV = 0;
  SrcPlan* dVs = nullptr; int nVs = 0;   // the solve's variant: loop-only integrals pre-summed,
  std::vector<SrcPlan> hVs;              // without the terms that run as GEMM groups
  std::vector<SrcGemmGroup> hG;          // source terms as X G products (see terms.h)
  SrcXTerm* dX = nullptr;                // every group's X terms, group g at dX + gx_off[g]
  std::vector<int> gx_off;
  double *Sact = nullptr, *Fact = nullptr, *V = nullptr;
  std::vector<SectorKeep> keep;   // one per (sector, SS-SR state), see class_keep_layout
};

struct SectorWork {
  double *Ssec = nullptr, *Fsec = nullptr, *s = nullptr, *Qs = nullptr, *X = nullptr,
         *FX = nullptr, *Ft = nullptr, *Qf = nullptr, *jac = nullptr, *W = nullptr,
         *part = nullptr, *part2 = nullptr;
  long wcap = 0, pcap = 0;   // doubles held by W and part (the sector pass runs in tuple
                             // chunks that fit them)
  long nb2 = 0;              // row blocks of the first column-sum stage (part2: nb2 x pcol)
  long p2size = 0;           // doubles held by part2
  double *srcX = nullptr, *srcG = nullptr;   // source GEMM groups: X rows chunk, G
  long srcXcap = 0, srcGcap = 0;
};
// Upper bounds on the solve's sector work arrays W and part (doubles): larger sectors are
// processed in tuple chunks.
constexpr long kSectorWCap = 1L << 28;
constexpr long kSectorPartCap = 1L << 27;
constexpr long kColsumBlocks = 1216;
// Sector eigenvalues whose smallest |denominator| is below this (Eh) are refined by a
// double-double Rayleigh quotient before the energies are formed.
constexpr double kRefineDenom = 1e-2;
// Sector size from which the precision form (7 slices) runs the sector transforms F X,
// X^T F X and X Q as split-BF16 tensor-core products.
constexpr int kOzTransformMin = 1024;

// Work space of the class densities (sized by the caller, see density_ag.cu).
struct DensWork {
  double *T = nullptr, *Lam = nullptr;   // all-tuple amplitudes [tuple][L][row], tall each
  double *U1 = nullptr, *U2 = nullptr;   // S^id T, S^sw T (U1 later holds W)
  double *Tsw = nullptr;                 // a tuple-swapped copy
  double *sec = nullptr;                 // sector amplitudes and lambda [2][secmax]
  double *tmp = nullptr;                 // back-transformed sector rows [2][secmax]
  double *Dm = nullptr;                  // D^id, D^sw [2][m^2]
  double *part = nullptr;                // split-K / block partial sums, partmax
  long tall = 0, secmax = 0, partmax = 0;
};
constexpr long kDensPartMax = 152L * 4 * 64 * 64;

// Device doubles a class needs in DensWork (all-tuple arrays).
long class_dens_tall(const ClassWork& w, const Dims& d);

// Sizes the context must allocate (doubles).
struct ClassSizes {
  long m2max = 0;        // max m^2 over enabled classes
  long wmax = 0;         // max msec * ntuple * n over sectors
  long partmax = 0;      // max ntuple * n * n
};

void class_setup(int cls, const Dims& d, ClassWork& w);   // host-only: sizes and plans
// Fill w.keep with the sectors of the scheme (device pointers left to the caller).
void class_keep_layout(ClassWork& w, const Dims& d, int scheme);
long class_sector_wsize(const ClassWork& w, const Dims& d, int scheme, long* partsize);
// Upload plans (allocated by the caller with cudaMalloc into w.dS/dF/dV).
cudaError_t class_upload_plans(ClassWork& w, const std::vector<ActPlan>& S,
                               const std::vector<ActPlan>& F, const std::vector<SrcPlan>& V);

// Evaluate S, F_act, V of a class and solve it; accumulates the moment sums
// mom = [M1: n^3][M2: n^2][M3: n] (see k_sector_energy).
int class_solve(ClassWork& w, SectorWork& sw, const Dims& d, int scheme, double shift,
                double thresh, RdmPtrs rdm, const double* f, const double* h, const EriBlocks& eri,
                const PresumBlocks& pb, const double* E0, const double* eps_cv, double* mom,
                double* mindenom, cudaStream_t s, KernelTimer* tm = nullptr,
                OzWork* oz = nullptr, int ci0 = 0, int ci1 = -1);
// Doubles of a pre-summed block, and its evaluation from the (pq|rt) block of its spaces.
long presum_size(const Dims& d, const PresumSpec& sp);
cudaError_t presum_block(const Dims& d, const PresumSpec& sp, const double* src, double* out,
                         cudaStream_t s);
// e = -M1[L][L][.], norm = M2[L][L] of one class
cudaError_t launch_moments_to_e(const double* mom, int n, double* e, double* nr, cudaStream_t s);
// lambda pieces of the target state P of one class from its moments and R
cudaError_t launch_lambda(const double* mom, const double* R, int n, int P, double shift, double* NL,
                          double* lv, cudaStream_t s);

// Class share of the densities of target state P (Sec. II.D) accumulated into
// d1[nmo][nmo] (source derivative w.r.t. h), d2[nmo][nmo] (closed, active and
// virtual blocks of dL/df) and the adjoint integral blocks G (same keys and layout
// as the (pq|rt) blocks of the solve).  Uses the sector bases kept by class_solve;
// NL = this class's <lambda_L|S|T_L>.
// First-order amplitudes T_L and lambda_L (target state P) of every sector of a class,
// back-transformed to all index tuples: dw.T and dw.Lam [tuple][L][(fam, act..., N)].
int class_tuple_amplitudes(ClassWork& w, DensWork& dw, const Dims& d, double shift,
                           const double* E0, const double* eps_cv, const double* R, int P,
                           OzWork* oz, cudaStream_t s);
// out[fam][ext...][act...] = src[tuple][L][(fam, act..., N)] for one (L, N).
cudaError_t gather_amplitudes(const ClassWork& w, const Dims& d, const double* src, int L, int N,
                              double* out, cudaStream_t s);
int class_densities(ClassWork& w, DensWork& dw, const Dims& d, int scheme, double shift,
                    RdmPtrs rdm, const double* E0, const double* eps_cv, const double* R, int P,
                    const double* NL, const EriBlocks& G, double* d1, double* d2, OzWork* oz,
                    cudaStream_t s);

// GDF[Q][p][q] += sum_rt G[pq][rt] B[Q][rt] and GDF[Q][r][t] += sum_pq G[pq][rt] B[Q][pq]
// for one adjoint block with spaces sp; pack0/pack1/tmp hold X * (block pair) doubles.
cudaError_t gdf_from_block(const double* B, const Dims& d, const int sp[4], const double* G,
                           double* pack0, double* pack1, double* tmp, double* gdf, cudaStream_t s,
                           OzWork* oz = nullptr);

// Split-K FP64 Gram product over [pre][Ns][post] tensors:
//   X[x][y] = sum_(p, q) A[(p Ns + x) post + q] B[(p Ns + y) post + q],
// finished into out by mode: 0 out[x][y] = X; 1 out[off+y][off+x] -= X; 2 out[off+x][off+y] += X.
// part holds the split partials (partmax doubles, >= Ns^2).
// oz (optional, on): the product runs as a split BF16 GEMM on the tensor cores.
int gram_product(const double* A, const double* B, long pre, long Ns, long post, int mode,
                 double* out, long ld, long off, double* part, long partmax, cudaStream_t s,
                 OzWork* oz = nullptr);

// out[Q][x][y] = B[Q][off(sp0) + x][off(sp1) + y];  gdf[Q][off(sp0) + x][off(sp1) + y] += tmp[Q][x][y]
cudaError_t launch_pack_block(const double* B, const Dims& d, int sp0, int sp1, double* out,
                              cudaStream_t s);
cudaError_t launch_unpack_add(const double* tmp, const Dims& d, int sp0, int sp1, double* gdf,
                              cudaStream_t s);

// Work space of the energy gradient (gradient.cu): target-state active RDMs g1 [a^2], g2
// [a^4]; D, dsa [nmo^2]; per-Q scalars gD, tq [X]; T, M [X][nmo][nmo].
struct GradWork {
  double *g1 = nullptr, *g2 = nullptr, *D = nullptr, *dsa = nullptr, *gD = nullptr,
         *tq = nullptr, *T = nullptr, *M = nullptr;
};
// grad_f [nmo][nmo] and grad_B [X][nmo][nmo] of E_P (MS) from the densities d1, d2, Gamma
// (gdf) and the reference pieces (see gradient.cu).
int assemble_gradient(const Dims& d, const double* B, const double* R, int P,
                      const double* rdm1, const double* rdm2, const double* dact,
                      const double* bsum, const double* gam, const double* d1, const double* d2,
                      const double* gdf, const GradWork& gw, double* grad_f, double* grad_B,
                      cudaStream_t s);

// Orbital derivative Y [nmo][nmo] of the Lagrangian (Sec. II.D, Eq. orbderiv) from the
// densities d1, d2 (every block), Gamma (gdf) and the reference pieces; also returns
// gf = dL/dh [nmo][nmo], gBh = dL/dB at fixed h [X][nmo][nmo] and h (see gradient.cu).
int assemble_orbital_derivative(const Dims& d, const double* f, const double* g_act,
                                const double* B, const double* R, int P, const double* rdm1,
                                const double* rdm2, const double* dact, const double* bsum,
                                const double* gam, const double* d1, const double* d2,
                                const double* gdf, const GradWork& gw, double* h, double* gf,
                                double* gBh, double* Y, cudaStream_t s);

// x <- (x + x^T) / 2 for `batch` square nmo x nmo matrices.
cudaError_t launch_symmetrize(double* x, int nmo, long batch, cudaStream_t s);

// DF integral block out[p][q][r][t] = sum_P B[P][p][q] B[P][r][t] for the given spaces.
cudaError_t eri_block(const double* B, const Dims& d, const int sp[4], double* pack0, double* pack1,
                      double* out, cudaStream_t s, OzWork* oz = nullptr);

// h = f - g(d_core) - g(d_act), g(d_core)_xy = sum_j [2 (xy|jj) - (xj|jy)]
// oz (on, 7 slices) with ktmp [nmo][nmo]: the core exchange as a split Gram product.
cudaError_t launch_hcore(const double* f, const double* g_act, const double* B, const double* bsum,
                         const Dims& d, double* h, cudaStream_t s, OzWork* oz = nullptr,
                         double* ktmp = nullptr);

}  // namespace caspt2
