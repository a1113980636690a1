// Classes A-G (internal): device structures and the per-class solve.
#pragma once
#include <vector>

#include "kernels.cuh"
#include "linalg.cuh"
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

__device__ __forceinline__ void atomicMin_double(double* addr, double v) {
  if (!(v >= 0.0)) return;
  atomicMin(reinterpret_cast<unsigned long long*>(addr),
            static_cast<unsigned long long>(__double_as_longlong(v)));
}

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
  double *Sact = nullptr, *Fact = nullptr, *V = nullptr;
};

struct SectorWork {
  double *Ssec = nullptr, *Fsec = nullptr, *s = nullptr, *Qs = nullptr, *X = nullptr,
         *FX = nullptr, *Ft = nullptr, *omega = nullptr, *Qf = nullptr, *Y = nullptr,
         *mask = nullptr, *jac = nullptr, *W = nullptr, *Vt = nullptr, *part = nullptr,
         *partn = nullptr;
};

// Sizes the context must allocate (doubles).
struct ClassSizes {
  long m2max = 0;        // max m^2 over enabled classes
  long wmax = 0;         // max msec * ntuple * n over sectors
  long partmax = 0;      // max ntuple * n * n
};

void class_setup(int cls, const Dims& d, ClassWork& w);   // host-only: sizes and plans
long class_sector_wsize(const ClassWork& w, const Dims& d, int scheme, long* partsize);
// Upload plans (allocated by the caller with cudaMalloc into w.dS/dF/dV).
cudaError_t class_upload_plans(ClassWork& w, const std::vector<ActPlan>& S,
                               const std::vector<ActPlan>& F, const std::vector<SrcPlan>& V);

// Evaluate S, F_act, V of a class and solve it; accumulates the moment sums
// mom = [M1: n^3][M2: n^2][M3: n] (see k_sector_energy).
int class_solve(ClassWork& w, SectorWork& sw, const Dims& d, int scheme, double shift,
                double thresh, RdmPtrs rdm, const double* f, const double* h, const EriBlocks& eri,
                const double* E0, const double* eps_cv, double* mom, double* mindenom,
                cudaStream_t s, KernelTimer* tm = nullptr);
// e = -M1[L][L][.], norm = M2[L][L] of one class
cudaError_t launch_moments_to_e(const double* mom, int n, double* e, double* nr, cudaStream_t s);
// lambda pieces of the target state P of one class from its moments and R
cudaError_t launch_lambda(const double* mom, const double* R, int n, int P, double shift, double* NL,
                          double* lv, cudaStream_t s);

// DF integral block out[p][q][r][t] = sum_P B[P][p][q] B[P][r][t] for the given spaces.
cudaError_t eri_block(const double* B, const Dims& d, const int sp[4], double* pack0, double* pack1,
                      double* out, cudaStream_t s);

// h = f - g(d_core) - g(d_act), g(d_core)_xy = sum_j [2 (xy|jj) - (xj|jy)]
cudaError_t launch_hcore(const double* f, const double* g_act, const double* B, const double* bsum,
                         const Dims& d, double* h, cudaStream_t s);

}  // namespace caspt2
