// One-body couplings between excitation classes (internal; see cross.cu).
#pragma once
#include <vector>

#include "class_ag.cuh"
#include "terms.h"

namespace caspt2 {

// Layout of a class's all-tuple arrays [(tuple, L)][(fam, active..., N)] (classes A-G as in
// DensWork; class H with tuples (i, j, a, b) and rows N).
struct XCls {
  int nfam, nact, next;
  int ext_dim[4];
  long ntup;            // product of the external dimensions
  long A;               // a^nact
  int m;                // nfam * A * n
};
XCls make_xcls(int cls, const Dims& d);   // cls 0..7

struct XGroupDev {
  int side, nfe;
  int fe_xy[2], fe_pos[2];
  int ket_src[4];
};

struct CrossGroupHost {
  CrossGroup g;         // pattern (terms moved to the device plan array)
  int off = 0, nplan = 0, maxrank = 0;
};

struct CrossWork {
  std::vector<CrossGroupHost> groups;
  CrossPlan* plans = nullptr;   // device copy of every group's terms (owned by the caller)
};

constexpr int kCrossChunks = 64;  // row chunks of one reduction (fixed: results reproducible)

// Generate the groups of all six space pairs; `all` receives their terms (group h at
// all[h.off .. h.off + h.nplan)), which the caller copies to xw.plans on the device.
void cross_setup(CrossWork& xw, std::vector<CrossPlan>& all);
// Work sizes (doubles): W of the largest group, the largest GEMM product, the partials.
long cross_work_size(const CrossWork& xw, const Dims& d, long* wmax, long* zmax, long* partmax);
// dbar2 off-diagonal blocks (closed-active, active-virtual, closed-virtual and transposes)
// accumulated into d2 [nmo][nmo]: T[cls], Lam[cls] are the all-tuple amplitude and lambda
// arrays of the eight classes (nullptr: class left out).
int cross_dbar2(const CrossWork& xw, const Dims& d, RdmPtrs rdm, double* const* T,
                double* const* Lam, double* Wb, double* Zb, double* part, long wmax, long zmax,
                long partmax, double* d2, cudaStream_t s);
// Class-H all-tuple amplitudes and lambda [(i, j, a, b)][L][N] from K[(ia)][(jb)] = (ai|bj)
// and the class-H pair bases (W, shifts) of the solve.
cudaError_t launch_h_tuple_amps(const double* K, const double* eps, const double* W,
                                const double* shifts, const double* R, int P, const Dims& d,
                                int scheme, double shift, double* T, double* Lam, cudaStream_t s);

}  // namespace caspt2
