// Classes A-G of Eq. (class): overlap, active Fock and source matrices from the
// rotated RDMs (plans from terms.cpp), then the amplitude equation (Eq. ampeq) per
// external tuple for block-diagonal f.  The overlap and Fock matrices couple
// external tuples only through identity and (for classes with two closed or two
// virtual indices) the swap of that pair, so each class is solved in the symmetric
// and antisymmetric combinations:
//   S^+- = S^id +- S^sw,   F^+- = e_ext S^+- + F_act^+-,
//   X = Q_S s^(-1/2) over overlap eigenvalues >= threshold (Sec. II.B),
//   X^T F_act X = Q diag(omega) Q^T,  Y = X Q,
//   T(tuple, L) = -Y diag(1/(e_ext + omega - E0_L + E_s)) Y^T V(tuple, L),
// and the pieces of the effective Hamiltonian are
//   e[L][L'] = sum_tuples V(L')^T T(L),  norm[L] = T(L)^T S T(L).
#include <cmath>
#include <vector>

#include "class_ag.cuh"
#include "class_dev.cuh"
#include "linalg.cuh"

namespace caspt2 {


// S or F_act for all (row, col) of the m x m class matrix; out[pi][row][col].
// row = ((fam * a^nact + act) * n + M), act digits in slot order (first slot slowest).
__global__ void k_act_eval(const ActPlan* __restrict__ plans, int nplan, DevClass C, int a, int n,
                           RdmPtrs g, const double* __restrict__ f_act, double* __restrict__ out,
                           int m) {
  const long total = (long)m * m;
  const long A = ipow(a, C.nact);
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    const int row = e / m, col = e % m;
    int vals[24];
    const int M = row % n, N = col % n;
    long ab = row / n, ak = col / n;
    const int fb = ab / A, fk = ak / A;
    ab %= A;
    ak %= A;
    for (int k = C.nact - 1; k >= 0; --k) {
      vals[kRefBra + k] = ab % a;
      ab /= a;
      vals[kRefKet + k] = ak % a;
      ak /= a;
    }
    double acc0 = 0.0, acc1 = 0.0;
    for (int t = 0; t < nplan; ++t) {
      const ActPlan& P = plans[t];
      if (P.fb != fb || P.fk != fk) continue;
      bool ok = true;
      for (int q = 0; q < P.neq; ++q)
        if (vals[P.eq[q][0]] != vals[P.eq[q][1]]) ok = false;
      if (!ok) continue;
      const int nl = P.nloop;
      const int niter = nl == 0 ? 1 : (nl == 1 ? a : a * a);
      double s = 0.0;
      for (int it = 0; it < niter; ++it) {
        if (nl >= 1) vals[kRefLoop] = it % a;
        if (nl >= 2) vals[kRefLoop + 1] = it / a;
        double x = rdm_at(g.p, P.rank, n, a, M, N, vals, P.idx);
        if (P.has_f) x *= f_act[vals[P.fidx[0]] * a + vals[P.fidx[1]]];
        s += x;
      }
      if (P.pi == 0) acc0 += P.coeff * s; else acc1 += P.coeff * s;
    }
    out[e] = acc0;
    out[total + e] = acc1;
  }
}

// Sources V[fam][ext...][act...][M][L] = <M~|E_Omega^dag H|L~> (Eq. ampeq).
__global__ void k_src_eval(const SrcPlan* __restrict__ plans, int nplan, DevClass C, Dims d,
                           RdmPtrs g, const double* __restrict__ h, EriBlocks eri,
                           PresumBlocks pb, double* __restrict__ V, long total) {
  const int n = d.n, a = d.a, nmo = d.nmo();
  const int dimsp[4] = {d.c, d.a, d.v, 1};
  const int offsp[3] = {0, d.c, d.c + d.a};
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    long r = e;
    const int L = r % n; r /= n;
    const int M = r % n; r /= n;
    int vals[24];
    vals[kRefZero] = 0;
    for (int k = C.nact - 1; k >= 0; --k) {
      vals[kRefBra + C.act[k]] = r % a;
      r /= a;
    }
    for (int k = C.next - 1; k >= 0; --k) {
      const int dm = dimsp[C.slot_space[C.ext[k]]];
      vals[kRefBra + C.ext[k]] = r % dm;
      r /= dm;
    }
    const int fam = (int)r;
    double acc = 0.0;
    for (int t = 0; t < nplan; ++t) {
      const SrcPlan& P = plans[t];
      if (P.fb != fam) continue;
      bool ok = true;
      for (int q = 0; q < P.neq; ++q)
        if (vals[P.eq[q][0]] != vals[P.eq[q][1]]) ok = false;
      if (!ok) continue;
      long niter = 1;
      for (int j = 0; j < P.nloop; ++j) niter *= dimsp[P.loop_space[j]];
      const double* blk = nullptr;
      long bd[4] = {1, 1, 1, 1};
      if (P.kind == 1) {
        const int key = ((P.ispace[0] * 3 + P.ispace[1]) * 3 + P.ispace[2]) * 3 + P.ispace[3];
        blk = eri.p[key];
        for (int j = 0; j < 4; ++j) bd[j] = dimsp[P.ispace[j]];
      } else if (P.kind == 2) {
        blk = pb.p[P.cb];
        for (int j = 0; j < 4; ++j) bd[j] = dimsp[P.ispace[j]];
      }
      double s = 0.0;
      for (long it = 0; it < niter; ++it) {
        long q = it;
        for (int j = 0; j < P.nloop; ++j) {
          const int dm = dimsp[P.loop_space[j]];
          vals[kRefLoop + j] = q % dm;
          q /= dm;
        }
        double x;
        if (P.kind == 0) {
          x = h[(long)(offsp[P.ispace[0]] + vals[P.iidx[0]]) * nmo + offsp[P.ispace[1]] +
                vals[P.iidx[1]]];
        } else {
          x = blk[((vals[P.iidx[0]] * bd[1] + vals[P.iidx[1]]) * bd[2] + vals[P.iidx[2]]) * bd[3] +
                  vals[P.iidx[3]]];
        }
        if (x != 0.0) x *= rdm_at(g.p, P.rank, n, a, M, L, vals, P.idx);
        s += x;
      }
      acc += P.coeff * s;
    }
    V[e] = acc;
  }
}

// Source GEMM groups (terms.h, split_src_plans): X[(row)][k] over the external tuples
// row0 .. row0 + nrow (row-major in the class's external order) and k over the shared loops
// (a^ns, the first loop slowest): the group's integral terms summed, each with its
// integral-only loops and external deltas.
__global__ void k_src_x(const SrcXTerm* __restrict__ xt, int nx, DevClass C, Dims d, int ns,
                        const double* __restrict__ h, EriBlocks eri, PresumBlocks pb, long row0,
                        long nrow, double* __restrict__ X) {
  const int a = d.a, nmo = d.nmo();
  const int dimsp[4] = {d.c, d.a, d.v, 1};
  const int offsp[3] = {0, d.c, d.c + d.a};
  const long K = ipow(a, ns);
  const long total = nrow * K;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    int vals[32];
    vals[kRefZero] = 0;
    long q = e % K;
    for (int p = ns - 1; p >= 0; --p) {
      vals[kRefLoop + p] = (int)(q % a);
      q /= a;
    }
    long r = row0 + e / K;
    for (int k = C.next - 1; k >= 0; --k) {
      const int dm = dimsp[C.slot_space[C.ext[k]]];
      vals[kRefBra + C.ext[k]] = (int)(r % dm);
      r /= dm;
    }
    double acc = 0.0;
    for (int t = 0; t < nx; ++t) {
      const SrcXTerm& T = xt[t];
      bool ok = true;
      for (int u = 0; u < T.neq; ++u)
        if (vals[T.eq[u][0]] != vals[T.eq[u][1]]) ok = false;
      if (!ok) continue;
      const double* blk = nullptr;
      long bd[4] = {1, 1, 1, 1};
      if (T.kind == 1) {
        const int key = ((T.ispace[0] * 3 + T.ispace[1]) * 3 + T.ispace[2]) * 3 + T.ispace[3];
        blk = eri.p[key];
        for (int j = 0; j < 4; ++j) bd[j] = dimsp[T.ispace[j]];
      } else if (T.kind == 2) {
        blk = pb.p[T.cb];
        for (int j = 0; j < 4; ++j) bd[j] = dimsp[T.ispace[j]];
      }
      long niter = 1;
      for (int j = 0; j < T.nloop; ++j) niter *= dimsp[T.loop_space[j]];
      double sum = 0.0;
      for (long it = 0; it < niter; ++it) {
        long w = it;
        for (int j = 0; j < T.nloop; ++j) {
          const int dm = dimsp[T.loop_space[j]];
          vals[kRefLoop + ns + j] = (int)(w % dm);
          w /= dm;
        }
        if (T.kind == 0)
          sum += h[(long)(offsp[T.ispace[0]] + vals[T.iidx[0]]) * nmo + offsp[T.ispace[1]] +
                   vals[T.iidx[1]]];
        else
          sum += blk[((vals[T.iidx[0]] * bd[1] + vals[T.iidx[1]]) * bd[2] + vals[T.iidx[2]]) *
                         bd[3] + vals[T.iidx[3]]];
      }
      acc += T.coeff * sum;
    }
    X[e] = acc;
  }
}

// G[k][(act..., M, L)] of a source GEMM group: the RDM element (bra state M, ket L) summed
// over the RDM-only loops, zero where an active delta fails.
__global__ void k_src_g(SrcGSig g, DevClass C, Dims d, RdmPtrs rdm, double* __restrict__ G) {
  const int n = d.n, a = d.a;
  const long A = ipow(a, C.nact);
  const long ncol = A * n * n;
  const long total = ipow(a, g.ns) * ncol;
  const long nit = ipow(a, g.nloop);
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    int vals[32];
    vals[kRefZero] = 0;
    long col = e % ncol;
    const int L = (int)(col % n);
    const int M = (int)((col / n) % n);
    long r = col / ((long)n * n);
    for (int k = C.nact - 1; k >= 0; --k) {
      vals[kRefBra + C.act[k]] = (int)(r % a);
      r /= a;
    }
    long q = e / ncol;
    for (int p = g.ns - 1; p >= 0; --p) {
      vals[kRefLoop + p] = (int)(q % a);
      q /= a;
    }
    bool ok = true;
    for (int u = 0; u < g.neq; ++u)
      if (vals[g.eq[u][0]] != vals[g.eq[u][1]]) ok = false;
    double sum = 0.0;
    if (ok)
      for (long it = 0; it < nit; ++it) {
        long w = it;
        for (int j = 0; j < g.nloop; ++j) {
          vals[kRefLoop + g.ns + j] = (int)(w % a);
          w /= a;
        }
        sum += rdm_at(rdm.p, g.rank, n, a, M, L, vals, g.idx);
      }
    G[e] = sum;
  }
}

// Same sources with one thread per (fam, ext, act) holding all n^2 (M, L) results (n <=
// NS): each plan term's integral value and RDM offset are formed once and applied to the
// n^2 state pairs (Gamma[M][L][off] at stride a^(2 rank)).
template <int NS>
__global__ void k_src_eval_ml(const SrcPlan* __restrict__ plans, int nplan, DevClass C, Dims d,
                              RdmPtrs g, const double* __restrict__ h, EriBlocks eri,
                              PresumBlocks pb, double* __restrict__ V, long total2) {
  const int n = d.n, a = d.a, nmo = d.nmo();
  const int dimsp[4] = {d.c, d.a, d.v, 1};
  const int offsp[3] = {0, d.c, d.c + d.a};
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total2;
       e += (long)gridDim.x * blockDim.x) {
    long r = e;
    int vals[24];
    vals[kRefZero] = 0;
    for (int k = C.nact - 1; k >= 0; --k) {
      vals[kRefBra + C.act[k]] = r % a;
      r /= a;
    }
    for (int k = C.next - 1; k >= 0; --k) {
      const int dm = dimsp[C.slot_space[C.ext[k]]];
      vals[kRefBra + C.ext[k]] = r % dm;
      r /= dm;
    }
    const int fam = (int)r;
    double acc[NS * NS];
#pragma unroll
    for (int q = 0; q < NS * NS; ++q) acc[q] = 0.0;
    for (int t = 0; t < nplan; ++t) {
      const SrcPlan& P = plans[t];
      if (P.fb != fam) continue;
      bool ok = true;
      for (int q = 0; q < P.neq; ++q)
        if (vals[P.eq[q][0]] != vals[P.eq[q][1]]) ok = false;
      if (!ok) continue;
      long niter = 1;
      for (int j = 0; j < P.nloop; ++j) niter *= dimsp[P.loop_space[j]];
      const double* blk = nullptr;
      long bd[4] = {1, 1, 1, 1};
      if (P.kind == 1) {
        const int key = ((P.ispace[0] * 3 + P.ispace[1]) * 3 + P.ispace[2]) * 3 + P.ispace[3];
        blk = eri.p[key];
        for (int j = 0; j < 4; ++j) bd[j] = dimsp[P.ispace[j]];
      } else if (P.kind == 2) {
        blk = pb.p[P.cb];
        for (int j = 0; j < 4; ++j) bd[j] = dimsp[P.ispace[j]];
      }
      const long stride = ipow(a, 2 * P.rank);
      for (long it = 0; it < niter; ++it) {
        long q = it;
        for (int j = 0; j < P.nloop; ++j) {
          const int dm = dimsp[P.loop_space[j]];
          vals[kRefLoop + j] = q % dm;
          q /= dm;
        }
        double x;
        if (P.kind == 0) {
          x = h[(long)(offsp[P.ispace[0]] + vals[P.iidx[0]]) * nmo + offsp[P.ispace[1]] +
                vals[P.iidx[1]]];
        } else {
          x = blk[((vals[P.iidx[0]] * bd[1] + vals[P.iidx[1]]) * bd[2] + vals[P.iidx[2]]) * bd[3] +
                  vals[P.iidx[3]]];
        }
        if (x == 0.0) continue;
        x *= P.coeff;
        if (P.rank == 0) {
#pragma unroll
          for (int M = 0; M < NS; ++M)
            if (M < n) acc[M * NS + M] += x;
        } else {
          long off = 0;
          for (int j = 0; j < 2 * P.rank; ++j) off = off * a + vals[P.idx[j]];
          const double* gp = g.p[P.rank] + off;
#pragma unroll
          for (int M = 0; M < NS; ++M)
#pragma unroll
            for (int L = 0; L < NS; ++L)
              if (M < n && L < n) acc[M * NS + L] += x * gp[(long)(M * n + L) * stride];
        }
      }
    }
    double* out = V + e * n * n;
#pragma unroll
    for (int M = 0; M < NS; ++M)
#pragma unroll
      for (int L = 0; L < NS; ++L)
        if (M < n && L < n) out[M * n + L] = acc[M * NS + L];
  }
}

// Sources with one thread per (fam, ext, act, M) holding the n results over L (n <= NS):
// fewer registers than the all-(M, L) variant, for larger state counts.
template <int NS>
__global__ void k_src_eval_m(const SrcPlan* __restrict__ plans, int nplan, DevClass C, Dims d,
                              RdmPtrs g, const double* __restrict__ h, EriBlocks eri,
                              PresumBlocks pb, double* __restrict__ V, long total2) {
  const int n = d.n, a = d.a, nmo = d.nmo();
  const int dimsp[4] = {d.c, d.a, d.v, 1};
  const int offsp[3] = {0, d.c, d.c + d.a};
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total2 * n;
       e += (long)gridDim.x * blockDim.x) {
    const int Mt = (int)(e % n);
    long r = e / n;
    int vals[24];
    vals[kRefZero] = 0;
    for (int k = C.nact - 1; k >= 0; --k) {
      vals[kRefBra + C.act[k]] = r % a;
      r /= a;
    }
    for (int k = C.next - 1; k >= 0; --k) {
      const int dm = dimsp[C.slot_space[C.ext[k]]];
      vals[kRefBra + C.ext[k]] = r % dm;
      r /= dm;
    }
    const int fam = (int)r;
    double acc[NS];
#pragma unroll
    for (int q = 0; q < NS; ++q) acc[q] = 0.0;
    for (int t = 0; t < nplan; ++t) {
      const SrcPlan& P = plans[t];
      if (P.fb != fam) continue;
      bool ok = true;
      for (int q = 0; q < P.neq; ++q)
        if (vals[P.eq[q][0]] != vals[P.eq[q][1]]) ok = false;
      if (!ok) continue;
      long niter = 1;
      for (int j = 0; j < P.nloop; ++j) niter *= dimsp[P.loop_space[j]];
      const double* blk = nullptr;
      long bd[4] = {1, 1, 1, 1};
      if (P.kind == 1) {
        const int key = ((P.ispace[0] * 3 + P.ispace[1]) * 3 + P.ispace[2]) * 3 + P.ispace[3];
        blk = eri.p[key];
        for (int j = 0; j < 4; ++j) bd[j] = dimsp[P.ispace[j]];
      } else if (P.kind == 2) {
        blk = pb.p[P.cb];
        for (int j = 0; j < 4; ++j) bd[j] = dimsp[P.ispace[j]];
      }
      const long stride = ipow(a, 2 * P.rank);
      for (long it = 0; it < niter; ++it) {
        long q = it;
        for (int j = 0; j < P.nloop; ++j) {
          const int dm = dimsp[P.loop_space[j]];
          vals[kRefLoop + j] = q % dm;
          q /= dm;
        }
        double x;
        if (P.kind == 0) {
          x = h[(long)(offsp[P.ispace[0]] + vals[P.iidx[0]]) * nmo + offsp[P.ispace[1]] +
                vals[P.iidx[1]]];
        } else {
          x = blk[((vals[P.iidx[0]] * bd[1] + vals[P.iidx[1]]) * bd[2] + vals[P.iidx[2]]) * bd[3] +
                  vals[P.iidx[3]]];
        }
        if (x == 0.0) continue;
        x *= P.coeff;
        if (P.rank == 0) {
#pragma unroll
          for (int L = 0; L < NS; ++L)
            if (L == Mt) acc[L] += x;
        } else {
          long off = 0;
          for (int j = 0; j < 2 * P.rank; ++j) off = off * a + vals[P.idx[j]];
          const double* gp = g.p[P.rank] + off + (long)Mt * n * stride;
#pragma unroll
          for (int L = 0; L < NS; ++L)
            if (L < n) acc[L] += x * gp[(long)L * stride];
        }
      }
    }
    double* out = V + (e / n) * n * n + (long)Mt * n;
#pragma unroll
    for (int L = 0; L < NS; ++L)
      if (L < n) out[L] = acc[L];
  }
}

// Pre-summed block: out[i0][i1][i2][i3] (summed positions of size 1) = sum over the
// summed variables' values of src at those indices (fixed order).
__global__ void k_presum(const double* __restrict__ src, PresumSpec sp, int d0, int d1, int d2,
                         int d3, double* __restrict__ out) {
  const int sd[4] = {d0, d1, d2, d3};
  int od[4], vd[2] = {1, 1};
  for (int p = 0; p < 4; ++p) {
    od[p] = sp.var[p] < 0 ? sd[p] : 1;
    if (sp.var[p] >= 0) vd[sp.var[p]] = sd[p];
  }
  const long total = (long)od[0] * od[1] * od[2] * od[3];
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    int r[4];
    long q = e;
    for (int p = 3; p >= 0; --p) {
      r[p] = (int)(q % od[p]);
      q /= od[p];
    }
    double acc = 0.0;
    for (int s0 = 0; s0 < vd[0]; ++s0)
      for (int s1 = 0; s1 < vd[1]; ++s1) {
        int x[4];
        for (int p = 0; p < 4; ++p)
          x[p] = sp.var[p] < 0 ? r[p] : (sp.var[p] == 0 ? s0 : s1);
        acc += src[(((long)x[0] * sd[1] + x[1]) * sd[2] + x[2]) * sd[3] + x[3]];
      }
    out[e] = acc;
  }
}

// Pack B[P][off0 + x][off1 + y] -> out[P][x][y]
__global__ void k_pack_block(const double* __restrict__ B, int X, int nmo, int off0, int n0,
                             int off1, int n1, double* __restrict__ out) {
  const long total = (long)X * n0 * n1;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    const int y = e % n1;
    const long r = e / n1;
    const int x = r % n0;
    const long P = r / n0;
    out[e] = B[(P * nmo + off0 + x) * nmo + off1 + y];
  }
}

__global__ void k_fill(double* __restrict__ x, long n, double v) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    x[i] = v;
}

// Sector matrices: out = sym(S_id + sgn S_sw) restricted to rows/cols with state Lsel
// (Lsel < 0: all), into an msec x msec buffer.
__global__ void k_sector(const double* __restrict__ in, int m, int n, double sgn, int Lsel,
                         double* __restrict__ out, int msec) {
  const long total = (long)msec * msec;
  const long mm = (long)m * m;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    const int i = e / msec, j = e % msec;
    const int ri = Lsel < 0 ? i : i * n + Lsel;
    const int rj = Lsel < 0 ? j : j * n + Lsel;
    const double x = in[(long)ri * m + rj] + sgn * in[mm + (long)ri * m + rj];
    const double y = in[(long)rj * m + ri] + sgn * in[mm + (long)rj * m + ri];
    out[e] = 0.5 * (x + y);
  }
}

// Eigenvalues ascending: the kept overlap directions are the last nk columns.
// X[i][c] = Q[i][m - nk + c] / sqrt(s[m - nk + c])   (m x nk, row-major)
__global__ void k_range_basis(const double* __restrict__ Q, const double* __restrict__ s, int m,
                              int nk, double* __restrict__ X) {
  const long total = (long)m * nk;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    const int i = e / nk, c = e % nk, k = m - nk + c;
    X[e] = Q[(long)i * m + k] / sqrt(s[k]);
  }
}

// W[row][(tuple - t0, L')] for the sector tuples t0 .. t0 + nt - 1: rows (fam, act, M)
// (M == Lsel under SS-SR)
__global__ void k_sector_src(const double* __restrict__ V, DevClass C, ExtDims ed, int a, int n,
                             int sector, int Lsel, long t0, long nt, int msec,
                             double* __restrict__ W) {
  // one thread per (tuple, row prefix fam * A + act), the tuple fastest (coalesced writes of
  // W); the tuple is decoded once and the n x n (M, L') block of V read contiguously
  const long A = ipow(a, C.nact);
  const long ncol = nt * n;
  const long nfa = Lsel < 0 ? msec / n : msec;
  const long total = nt * nfa;
  const double isq2 = 0.70710678118654752440;
  const long nn = (long)n * n;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    const long tl = e % nt;
    const long fa = e / nt;                     // fam * A + act
    const long t = t0 + tl;
    int co[3], cs[3];
    sector_tuple(C, ed.d, sector, t, co, cs);
    const int fam = (int)(fa / A);
    const long act = fa % A;
    long off = fam, offs = fam;
    for (int k = 0; k < C.next; ++k) {
      off = off * ed.d[k] + co[k];
      offs = offs * ed.d[k] + cs[k];
    }
    const long ia0 = off * A * nn + act * nn, ib0 = offs * A * nn + act * nn;
    const int m0 = Lsel < 0 ? 0 : Lsel, m1 = Lsel < 0 ? n : Lsel + 1;
    for (int M = m0; M < m1; ++M) {
      const long row = Lsel < 0 ? fa * n + M : fa;
      double* wr = W + row * ncol + tl * n;
      for (int Lp = 0; Lp < n; ++Lp) {
        const long ia = ia0 + (long)M * n + Lp, ib = ib0 + (long)M * n + Lp;
        double w;
        if (C.pair0 < 0) w = V[ia];
        else if (sector == 0) w = (ia == ib) ? V[ia] : (V[ia] + V[ib]) * isq2;
        else w = (V[ia] - V[ib]) * isq2;
        wr[Lp] = w;
      }
    }
  }
}

// Moment sums of the sector for each (tuple t, L, N) over the kept eigenvectors mu:
//   M1[L][N][L'] += Vt_N Vt_L' / D_L (all L'),  M2[L][N] += Vt_N Vt_L / D_L^2,
//   M3[L] += Vt_L^2 / D_L^3 (N == L),   D_L = e_ext(t) + omega_mu - E0_L + E_s.
// part[t][Li][N][n + 2] (Li = L, or 0 under SS-SR where L = Lsel).
// Same moment sums with one thread per (tuple, L) holding all N (n <= NS): each
// denominator and its reciprocal are formed once and the row of Vt is read once.
template <int NS>
__global__ void k_sector_energy_ml(const double* __restrict__ Vt, const double* __restrict__ omega,
                                   const double* __restrict__ E0, const double* __restrict__ eps,
                                   DevClass C, ExtDims ed, int c, int n, int sector, int Lsel,
                                   long ntup, long t0, long nt, int msec, double shift,
                                   double* __restrict__ part, double* __restrict__ mindenom) {
  const long ncol = ntup * n;
  const int nL = Lsel < 0 ? n : 1;
  const long total = nt * nL;
  const int w = n + 2;
  double dmin = 1e300;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    const int Li = e % nL;
    const long tl = e / nL;
    const long t = t0 + tl;
    const int L = Lsel < 0 ? Li : Lsel;
    int co[3], cs[3];
    sector_tuple(C, ed.d, sector, t, co, cs);
    double ee = 0.0;
    for (int k = 0; k < C.next; ++k)
      ee += (C.slot_space[C.ext[k]] == SP_V) ? eps[c + co[k]] : -eps[co[k]];
    const double base = ee - E0[L] + shift;
    double m1[NS * NS], m2[NS], m3 = 0.0;
#pragma unroll
    for (int q = 0; q < NS * NS; ++q) m1[q] = 0.0;
#pragma unroll
    for (int q = 0; q < NS; ++q) m2[q] = 0.0;
    for (int mu = 0; mu < msec; ++mu) {
      const double D = base + omega[mu];
      const double inv = recip(D);
      const double* row = Vt + (long)mu * ncol + t * n;
      double r[NS];
#pragma unroll
      for (int q = 0; q < NS; ++q) r[q] = q < n ? row[q] : 0.0;
      double rL = 0.0;
#pragma unroll
      for (int q = 0; q < NS; ++q) if (q == L) rL = r[q];
      const double wL = rL * inv * inv;
#pragma unroll
      for (int N = 0; N < NS; ++N) {
        const double vn = r[N] * inv;
#pragma unroll
        for (int q = N; q < NS; ++q) m1[N * NS + q] = fma(vn, r[q], m1[N * NS + q]);   // q >= N
        m2[N] = fma(r[N], wL, m2[N]);
      }
      m3 = fma(rL * rL * inv, inv * inv, m3);
      dmin = fmin(dmin, fabs(D));
    }
#pragma unroll
    for (int N = 0; N < NS; ++N) {
      if (N >= n) continue;
      double* o = part + (((tl * nL + Li) * n) + N) * w;
#pragma unroll
      for (int q = 0; q < NS; ++q)
        if (q < n) o[q] = q >= N ? m1[N * NS + q] : m1[q * NS + N];   // M1 symmetric in (N, q)
      o[n] = m2[N];
      o[n + 1] = (N == L) ? m3 : 0.0;
    }
  }
  __shared__ double red[32];
  dmin = block_min(dmin, red);
  if (threadIdx.x == 0) atomicMin_double(mindenom, dmin);
}

// e_ext(t) of every tuple of a sector (one decode per tuple), for k_mu_mindenom_ee.
__global__ void k_sector_eext(const double* __restrict__ eps, DevClass C, ExtDims ed, int c,
                              int sector, long ntup, double* __restrict__ ee) {
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < ntup;
       t += (long)gridDim.x * blockDim.x) {
    int co[3], cs[3];
    sector_tuple(C, ed.d, sector, t, co, cs);
    double x = 0.0;
    for (int k = 0; k < C.next; ++k)
      x += (C.slot_space[C.ext[k]] == SP_V) ? eps[c + co[k]] : -eps[co[k]];
    ee[t] = x;
  }
}

// k_mu_mindenom from the stored e_ext of the tuples.
__global__ void k_mu_mindenom_ee(const double* __restrict__ omega, const double* __restrict__ E0,
                                 const double* __restrict__ ee, int n, int Lsel, long ntup,
                                 double shift, double* __restrict__ mdn) {
  __shared__ double red[32];
  const int mu = blockIdx.y;
  const int nL = Lsel < 0 ? n : 1;
  double dmin = 1e300;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < ntup;
       t += (long)gridDim.x * blockDim.x) {
    const double x = ee[t] + omega[mu];
    for (int Li = 0; Li < nL; ++Li) dmin = fmin(dmin, fabs(x - E0[Lsel < 0 ? Li : Lsel] + shift));
  }
  dmin = block_min(dmin, red);
  if (threadIdx.x == 0) atomicMin_double(mdn + mu, dmin);
}

// Smallest |e_ext(t) + omega_mu - E0_L + E_s| over the tuples of the sector and the states
// L of the scheme, for every eigenvector mu: mdn[mu] (order-independent minimum).
__global__ void k_mu_mindenom(const double* __restrict__ omega, const double* __restrict__ E0,
                              const double* __restrict__ eps, DevClass C, ExtDims ed, int c,
                              int n, int sector, int Lsel, long ntup, int nk, double shift,
                              double* __restrict__ mdn) {
  __shared__ double red[32];
  const int mu = blockIdx.y;
  const int nL = Lsel < 0 ? n : 1;
  double dmin = 1e300;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < ntup;
       t += (long)gridDim.x * blockDim.x) {
    int co[3], cs[3];
    sector_tuple(C, ed.d, sector, t, co, cs);
    double ee = 0.0;
    for (int k = 0; k < C.next; ++k)
      ee += (C.slot_space[C.ext[k]] == SP_V) ? eps[c + co[k]] : -eps[co[k]];
    for (int Li = 0; Li < nL; ++Li) {
      const int L = Lsel < 0 ? Li : Lsel;
      dmin = fmin(dmin, fabs(ee + omega[mu] - E0[L] + shift));
    }
  }
  dmin = block_min(dmin, red);
  if (threadIdx.x == 0) atomicMin_double(mdn + mu, dmin);
}

// Double-double arithmetic from error-free transformations (Knuth's two-sum; the
// product error of a fused multiply-add): a value is hi + lo with |lo| <= ulp(hi) / 2.
struct DD { double hi, lo; };
__device__ __forceinline__ DD dd_from_sum(double a, double b) {
  const double s = a + b, bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ DD dd_add(DD x, DD y) {
  DD s = dd_from_sum(x.hi, y.hi);
  const double e = s.lo + x.lo + y.lo;
  const double hi = s.hi + e;
  return {hi, e - (hi - s.hi)};
}
// x + a * b with the product kept exactly
__device__ __forceinline__ DD dd_add_prod(DD x, double a, double b) {
  const double p = a * b, pe = fma(a, b, -p);
  DD s = dd_from_sum(x.hi, p);
  const double e = s.lo + x.lo + pe;
  const double hi = s.hi + e;
  return {hi, e - (hi - s.hi)};
}
__device__ __forceinline__ DD dd_shfl_down(DD x, int o) {
  return {__shfl_down_sync(0xffffffffu, x.hi, o), __shfl_down_sync(0xffffffffu, x.lo, o)};
}

// Rayleigh quotient omega_mu = y^T F y / y^T S y of the sector eigenvectors y = Y[:, mu]
// listed in `list`, in double-double.  The eigenvalue of a vector that is accurate to eps
// is accurate to O(eps^2) in the quotient, so this removes the eigensolver's rounding from
// the eigenvalues that sit next to a small denominator.  Stage 1: grid (row blocks,
// eigenvectors), one warp per row, each block's partial sums (dd) of y_i (F y)_i and
// y_i (S y)_i in a fixed order -> part[(list index * nrb + row block) * 4]; stage 2 sums
// the row blocks in order and divides.
constexpr int kRqThreads = 256;
__global__ void __launch_bounds__(kRqThreads)
k_rq_partial(const double* __restrict__ S, const double* __restrict__ F, int msec,
             const double* __restrict__ Y, int nk, const int* __restrict__ list,
             double* __restrict__ part) {
  __shared__ DD accF[kRqThreads / 32], accS[kRqThreads / 32];
  const int mu = list[blockIdx.y];
  const int nrb = gridDim.x;
  const int rows = (msec + nrb - 1) / nrb;
  const int r0 = blockIdx.x * rows, r1 = min(msec, r0 + rows);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  DD nf{0.0, 0.0}, ns{0.0, 0.0};
  for (int i = r0 + warp; i < r1; i += nw) {
    DD uf{0.0, 0.0}, us{0.0, 0.0};
    const double* fr = F + (long)i * msec;
    const double* sr = S + (long)i * msec;
    for (int j = lane; j < msec; j += 32) {
      const double yj = Y[(long)j * nk + mu];
      uf = dd_add_prod(uf, fr[j], yj);
      us = dd_add_prod(us, sr[j], yj);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      uf = dd_add(uf, dd_shfl_down(uf, o));
      us = dd_add(us, dd_shfl_down(us, o));
    }
    if (lane == 0) {
      const double yi = Y[(long)i * nk + mu];
      nf = dd_add(dd_add_prod(nf, yi, uf.hi), DD{yi * uf.lo, 0.0});
      ns = dd_add(dd_add_prod(ns, yi, us.hi), DD{yi * us.lo, 0.0});
    }
  }
  if (lane == 0) { accF[warp] = nf; accS[warp] = ns; }
  __syncthreads();
  if (threadIdx.x == 0) {
    DD tf = accF[0], ts = accS[0];
    for (int w = 1; w < nw; ++w) { tf = dd_add(tf, accF[w]); ts = dd_add(ts, accS[w]); }
    double* o = part + ((long)blockIdx.y * nrb + blockIdx.x) * 4;
    o[0] = tf.hi; o[1] = tf.lo; o[2] = ts.hi; o[3] = ts.lo;
  }
}

__global__ void k_rq_finish(const double* __restrict__ part, int nrb, const int* __restrict__ list,
                            int nlist, double* __restrict__ omega) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nlist) return;
  DD tf{0.0, 0.0}, ts{0.0, 0.0};
  for (int b = 0; b < nrb; ++b) {
    const double* o = part + ((long)q * nrb + b) * 4;
    tf = dd_add(tf, DD{o[0], o[1]});
    ts = dd_add(ts, DD{o[2], o[3]});
  }
  // (tf.hi + tf.lo) / (ts.hi + ts.lo) to double precision: one Newton correction
  const double r0 = tf.hi / ts.hi;
  const double p = r0 * ts.hi, pe = fma(r0, ts.hi, -p);
  const double r = ((tf.hi - p) - pe + tf.lo - r0 * ts.lo) / ts.hi;
  omega[list[q]] = r0 + r;
}

// Residual of the refined eigenpairs, r = F y - omega S y, in double-double per row
// (a warp per row), rounded to double: R[i * nl + q] for list entry q.  Grid (row blocks,
// list entries).
__global__ void __launch_bounds__(kRqThreads)
k_rq_resid(const double* __restrict__ S, const double* __restrict__ F, int msec,
           const double* __restrict__ Y, int nk, const int* __restrict__ list, int nl,
           const double* __restrict__ omega, double* __restrict__ R) {
  const int q = blockIdx.y;
  const int mu = list[q];
  const double w = omega[mu];
  const int nrb = gridDim.x;
  const int rows = (msec + nrb - 1) / nrb;
  const int r0 = blockIdx.x * rows, r1 = min(msec, r0 + rows);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int i = r0 + warp; i < r1; i += nw) {
    DD uf{0.0, 0.0}, us{0.0, 0.0};
    const double* fr = F + (long)i * msec;
    const double* sr = S + (long)i * msec;
    for (int j = lane; j < msec; j += 32) {
      const double yj = Y[(long)j * nk + mu];
      uf = dd_add_prod(uf, fr[j], yj);
      us = dd_add_prod(us, sr[j], yj);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      uf = dd_add(uf, dd_shfl_down(uf, o));
      us = dd_add(us, dd_shfl_down(us, o));
    }
    if (lane == 0) {
      // (F y)_i - w (S y)_i with the product w (S y)_i kept exactly
      DD r = dd_add_prod(uf, -w, us.hi);
      r = dd_add(r, DD{-w * us.lo, 0.0});
      R[(long)i * nl + q] = r.hi + r.lo;
    }
  }
}

// First-order correction coefficients of the refined eigenvectors from the other sector
// eigenvectors: c_j = (y_j . r) / (omega_k - omega_j), zero for j = k and for eigenvalues
// within 1e-12 of omega_k (a rotation inside a degenerate pair leaves the energies
// unchanged).  Cm[j * nl + q] holds y_j . r on input.
__global__ void k_rq_coef(double* __restrict__ Cm, int nk, const int* __restrict__ list, int nl,
                          const double* __restrict__ omega) {
  const long total = (long)nk * nl;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    const int j = (int)(e / nl), q = (int)(e % nl);
    const int k = list[q];
    const double gap = omega[k] - omega[j];
    const double tol = 1e-12 * fmax(1.0, fabs(omega[k]));
    Cm[e] = (j == k || fabs(gap) <= tol) ? 0.0 : Cm[e] / gap;
  }
}

// Y[i][list[q]] += Dl[i * nl + q]
__global__ void k_rq_apply(double* __restrict__ Y, int msec, int nk, const int* __restrict__ list,
                           int nl, const double* __restrict__ Dl) {
  const long total = (long)msec * nl;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    const int i = (int)(e / nl), q = (int)(e % nl);
    Y[(long)i * nk + list[q]] += Dl[e];
  }
}

// Tuples t0 .. t0 + nt - 1 of the sector (ntup in all; Vt has ntup * n columns); part
// rows are local to the chunk.
__global__ void k_sector_energy(const double* __restrict__ Vt, const double* __restrict__ omega,
                                const double* __restrict__ E0,
                                const double* __restrict__ eps, DevClass C, ExtDims ed, int c,
                                int n, int sector, int Lsel, long ntup, long t0, long nt, int msec,
                                double shift, double* __restrict__ part,
                                double* __restrict__ mindenom) {
  const long ncol = ntup * n;
  const int nL = Lsel < 0 ? n : 1;
  const long total = nt * nL * n;
  const int w = n + 2;
  double dmin = 1e300;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    const int N = e % n;
    const int Li = (e / n) % nL;
    const long tl = e / ((long)n * nL);
    const long t = t0 + tl;
    const int L = Lsel < 0 ? Li : Lsel;
    int co[3], cs[3];
    sector_tuple(C, ed.d, sector, t, co, cs);
    double ee = 0.0;
    for (int k = 0; k < C.next; ++k)
      ee += (C.slot_space[C.ext[k]] == SP_V) ? eps[c + co[k]] : -eps[co[k]];
    double m1[kMaxStates], m2 = 0.0, m3 = 0.0;
    for (int q = 0; q < n; ++q) m1[q] = 0.0;
    for (int mu = 0; mu < msec; ++mu) {
      const double D = ee + omega[mu] - E0[L] + shift;
      const double inv = 1.0 / D;
      const double* row = Vt + (long)mu * ncol + t * n;
      const double vn = row[N] * inv;
      for (int q = 0; q < n; ++q) m1[q] += vn * row[q];
      m2 += vn * row[L] * inv;
      if (N == L) m3 += row[L] * row[L] * inv * inv * inv;
      dmin = fmin(dmin, fabs(D));
    }
    double* o = part + (((tl * nL + Li) * n) + N) * w;
    for (int q = 0; q < n; ++q) o[q] = m1[q];
    o[n] = m2;
    o[n + 1] = m3;
  }
  __shared__ double red[32];
  dmin = block_min(dmin, red);
  if (threadIdx.x == 0) atomicMin_double(mindenom, dmin);
}

// First stage of the fixed-order column sums: block b sums rows [b R, (b + 1) R) of
// part[rows][ncol] (R = ceil(rows / gridDim.x)), one thread per column, rows in order
// (reads coalesced across the columns) -> out[b][ncol].
__global__ void k_colsum_rows(const double* __restrict__ part, long rows, int ncol,
                              double* __restrict__ out) {
  const long R = (rows + gridDim.x - 1) / gridDim.x;
  const long r0 = (long)blockIdx.x * R;
  const long r1 = r0 + R < rows ? r0 + R : rows;
  for (int col = threadIdx.x; col < ncol; col += blockDim.x) {
    double acc = 0.0;
    for (long r = r0; r < r1; ++r) acc += part[r * ncol + col];
    out[(long)blockIdx.x * ncol + col] = acc;
  }
}

// Fixed-order column sums of part[rows][nL][n][n+2] accumulated into the class moments
// mom = [M1: n^3][M2: n^2][M3: n].
__global__ void k_moment_colsum(const double* __restrict__ part, long rows, int n, int nL, int Lsel,
                                double* __restrict__ mom) {
  __shared__ double red[32];
  const int w = n + 2;
  const int col = blockIdx.x;          // (Li, N, q)
  const int ncol = nL * n * w;
  const int q = col % w, N = (col / w) % n, Li = col / (w * n);
  const int L = Lsel < 0 ? Li : Lsel;
  double acc = 0.0;
  for (long r = threadIdx.x; r < rows; r += blockDim.x) acc += part[r * ncol + col];
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) {
    if (q < n) mom[(L * n + N) * n + q] += acc;
    else if (q == n) mom[n * n * n + L * n + N] += acc;
    else if (N == L) mom[n * n * n + n * n + L] += acc;
  }
}

// column sums of part[rows][ncol] in fixed order -> out[ncol] (accumulated: out += sum)
__global__ void k_colsum_acc(const double* __restrict__ part, long rows, int ncol,
                             double* __restrict__ out, int stride_out, int offset_out) {
  __shared__ double red[32];
  const int col = blockIdx.x;
  double acc = 0.0;
  for (long r = threadIdx.x; r < rows; r += blockDim.x) acc += part[r * ncol + col];
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) out[offset_out + col * stride_out] += acc;
}

}  // namespace caspt2

// ============================================================== host side
namespace caspt2 {


// g(d_core)_xy = sum_P B_Pxy bsum_P * 2 - sum_P sum_j B_Pxj B_Pjy; h = f - g_act - g_core
__global__ void k_hcore(const double* __restrict__ f, const double* __restrict__ gact,
                        const double* __restrict__ B, const double* __restrict__ bsum, int X,
                        int nmo, int c, double* __restrict__ h) {
  const long total = (long)nmo * nmo;
  for (long xy = blockIdx.x * (long)blockDim.x + threadIdx.x; xy < total;
       xy += (long)gridDim.x * blockDim.x) {
    const int x = xy / nmo, y = xy % nmo;
    double jc = 0.0, kc = 0.0;
    for (int P = 0; P < X; ++P) {
      const double* Bp = B + (long)P * nmo * nmo;
      jc += Bp[xy] * bsum[P];
      for (int j = 0; j < c; ++j) kc += Bp[(long)x * nmo + j] * Bp[(long)j * nmo + y];
    }
    h[xy] = f[xy] - gact[xy] - (2.0 * jc - kc);
  }
}

// e[L][L'] = -M1[L][L][L'], norm[L] = M2[L][L] of one class
__global__ void k_moments_to_e(const double* __restrict__ mom, int n, double* e, double* nr) {
  const int idx = threadIdx.x;
  if (idx < n * n) {
    const int L = idx / n, Lp = idx % n;
    e[idx] = -mom[(L * n + L) * n + Lp];
  }
  if (idx < n) nr[idx] = mom[n * n * n + idx * n + idx];
}

cudaError_t launch_moments_to_e(const double* mom, int n, double* e, double* nr, cudaStream_t s) {
  ++launch_counter();
  k_moments_to_e<<<1, kMaxStates * kMaxStates, 0, s>>>(mom, n, e, nr);
  return cudaGetLastError();
}

// lambda of the target state P from the moments (Eq. lambdaeq differentiated w.r.t. T):
//   NL[L] = R_LP sum_N R_NP M2[L][N] + 2 E_s R_LP^2 M3[L]
//   lv[L][L'] = -R_LP sum_N R_NP M1[L][N][L'] - 2 E_s R_LP^2 M2[L][L']
__global__ void k_lambda_from_moments(const double* __restrict__ mom, const double* __restrict__ R,
                                      int n, int P, double shift, double* NL, double* lv) {
  const int idx = threadIdx.x;
  if (idx < n * n) {
    const int L = idx / n, Lp = idx % n;
    const double rl = R[L * n + P];
    double acc = 0.0;
    for (int N = 0; N < n; ++N) acc += R[N * n + P] * mom[(L * n + N) * n + Lp];
    lv[idx] = -rl * acc - 2.0 * shift * rl * rl * mom[n * n * n + L * n + Lp];
  }
  if (idx < n) {
    const int L = idx;
    const double rl = R[L * n + P];
    double acc = 0.0;
    for (int N = 0; N < n; ++N) acc += R[N * n + P] * mom[n * n * n + L * n + N];
    NL[L] = rl * acc + 2.0 * shift * rl * rl * mom[n * n * n + n * n + L];
  }
}

cudaError_t launch_lambda(const double* mom, const double* R, int n, int P, double shift, double* NL,
                          double* lv, cudaStream_t s) {
  ++launch_counter();
  k_lambda_from_moments<<<1, kMaxStates * kMaxStates, 0, s>>>(mom, R, n, P, shift, NL, lv);
  return cudaGetLastError();
}

// h = f - g_act - 2 J + Kc with the exchange part Kc[x][y] = sum_(P, j) B_Pxj B_Pjy given
__global__ void k_hcore_j(const double* __restrict__ f, const double* __restrict__ gact,
                          const double* __restrict__ B, const double* __restrict__ bsum, int X,
                          int nmo, const double* __restrict__ Kc, double* __restrict__ h) {
  const long total = (long)nmo * nmo;
  for (long xy = blockIdx.x * (long)blockDim.x + threadIdx.x; xy < total;
       xy += (long)gridDim.x * blockDim.x) {
    double jc = 0.0;
    for (int P = 0; P < X; ++P) jc += B[(long)P * total + xy] * bsum[P];
    h[xy] = f[xy] - gact[xy] - (2.0 * jc - Kc[xy]);
  }
}

cudaError_t launch_hcore(const double* f, const double* g_act, const double* B, const double* bsum,
                         const Dims& d, double* h, cudaStream_t s, OzWork* oz, double* ktmp) {
  const long tot = (long)d.nmo() * d.nmo();
  if (oz && oz->on && oz->S >= kOzMaxSlices && ktmp && d.c > 0) {
    // precision form: the core exchange sum_(P, j) B_Pxj B_Pjy as one split Gram product
    // over K = (P, j) (B symmetric in its orbital pair)
    const int nmo = d.nmo();
    const OzView vb{B, 1, nmo, d.c, (long)nmo * nmo};        // rows x, K = (P, j)
    cudaError_t e = oz_matmul(*oz, vb, vb, true, nmo, nmo, d.X * d.c, 1.0, 0.0, ktmp, nmo, s);
    if (e != cudaSuccess) return e;
    ++launch_counter();
    k_hcore_j<<<launch_blocks(tot, 128), 128, 0, s>>>(f, g_act, B, bsum, d.X, nmo, ktmp, h);
    return cudaGetLastError();
  }
  ++launch_counter();
  k_hcore<<<launch_blocks(tot, 128), 128, 0, s>>>(f, g_act, B, bsum, d.X, d.nmo(), d.c, h);
  return cudaGetLastError();
}

// gdf[Q][off0 + x][off1 + y] += tmp[Q][x][y]
__global__ void k_unpack_add(const double* __restrict__ tmp, int X, int nmo, int off0, int n0,
                             int off1, int n1, double* __restrict__ gdf) {
  const long total = (long)X * n0 * n1;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    const int y = e % n1;
    const long r = e / n1;
    const int x = r % n0;
    const long P = r / n0;
    gdf[(P * nmo + off0 + x) * nmo + off1 + y] += tmp[e];
  }
}

cudaError_t launch_pack_block(const double* B, const Dims& d, int sp0, int sp1, double* out,
                              cudaStream_t s) {
  const int n0 = space_dim(d, sp0), n1 = space_dim(d, sp1);
  const long t = (long)d.X * n0 * n1;
  if (t == 0) return cudaSuccess;
  ++launch_counter();
  k_pack_block<<<launch_blocks(t), 256, 0, s>>>(B, d.X, d.nmo(), space_off(d, sp0), n0,
                                               space_off(d, sp1), n1, out);
  return cudaGetLastError();
}

cudaError_t launch_unpack_add(const double* tmp, const Dims& d, int sp0, int sp1, double* gdf,
                              cudaStream_t s) {
  const int n0 = space_dim(d, sp0), n1 = space_dim(d, sp1);
  const long t = (long)d.X * n0 * n1;
  if (t == 0) return cudaSuccess;
  ++launch_counter();
  k_unpack_add<<<launch_blocks(t), 256, 0, s>>>(tmp, d.X, d.nmo(), space_off(d, sp0), n0,
                                               space_off(d, sp1), n1, gdf);
  return cudaGetLastError();
}

cudaError_t gdf_from_block(const double* B, const Dims& d, const int sp[4], const double* G,
                           double* pack0, double* pack1, double* tmp, double* gdf, cudaStream_t s,
                           OzWork* oz) {
  const int n0 = space_dim(d, sp[0]), n1 = space_dim(d, sp[1]);
  const int n2 = space_dim(d, sp[2]), n3 = space_dim(d, sp[3]);
  if ((long)n0 * n1 * n2 * n3 == 0) return cudaSuccess;
  const int n01 = n0 * n1, n23 = n2 * n3;
  const long t0 = (long)d.X * n01, t1 = (long)d.X * n23;
  ++launch_counter();
  k_pack_block<<<launch_blocks(t0), 256, 0, s>>>(B, d.X, d.nmo(), space_off(d, sp[0]), n0,
                                                space_off(d, sp[1]), n1, pack0);
  ++launch_counter();
  k_pack_block<<<launch_blocks(t1), 256, 0, s>>>(B, d.X, d.nmo(), space_off(d, sp[2]), n2,
                                                space_off(d, sp[3]), n3, pack1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const bool split = oz && oz->on;
  // d/dB[Q][pq] = sum_rt G[pq][rt] B[Q][rt]
  if (split) {
    const OzView vb{pack1, n23, 1, n23, 0}, vg{G, n23, 1, n23, 0};   // rows Q / pq, K = rt
    e = oz_matmul(*oz, vb, vg, false, d.X, n01, n23, 1.0, 0.0, tmp, n01, s);
  } else {
    e = dgemm(d.X, n01, n23, 1.0, pack1, n23, false, G, n23, true, 0.0, tmp, n01, s);
  }
  if (e != cudaSuccess) return e;
  ++launch_counter();
  k_unpack_add<<<launch_blocks(t0), 256, 0, s>>>(tmp, d.X, d.nmo(), space_off(d, sp[0]), n0,
                                                space_off(d, sp[1]), n1, gdf);
  // d/dB[Q][rt] = sum_pq G[pq][rt] B[Q][pq]
  if (split) {
    const OzView va{pack0, n01, 1, n01, 0}, vg{G, 1, n23, n01, 0};   // rows Q / rt, K = pq
    e = oz_matmul(*oz, va, vg, false, d.X, n23, n01, 1.0, 0.0, tmp, n23, s);
  } else {
    e = dgemm(d.X, n23, n01, 1.0, pack0, n01, false, G, n23, false, 0.0, tmp, n23, s);
  }
  if (e != cudaSuccess) return e;
  ++launch_counter();
  k_unpack_add<<<launch_blocks(t1), 256, 0, s>>>(tmp, d.X, d.nmo(), space_off(d, sp[2]), n2,
                                                space_off(d, sp[3]), n3, gdf);
  return cudaGetLastError();
}

cudaError_t eri_block(const double* B, const Dims& d, const int sp[4], double* pack0, double* pack1,
                      double* out, cudaStream_t s, OzWork* oz) {
  const int n0 = space_dim(d, sp[0]), n1 = space_dim(d, sp[1]);
  const int n2 = space_dim(d, sp[2]), n3 = space_dim(d, sp[3]);
  if ((long)n0 * n1 * n2 * n3 == 0) return cudaSuccess;
  const long t0 = (long)d.X * n0 * n1, t1 = (long)d.X * n2 * n3;
  ++launch_counter();
  k_pack_block<<<launch_blocks(t0), 256, 0, s>>>(B, d.X, d.nmo(), space_off(d, sp[0]), n0,
                                                space_off(d, sp[1]), n1, pack0);
  ++launch_counter();
  k_pack_block<<<launch_blocks(t1), 256, 0, s>>>(B, d.X, d.nmo(), space_off(d, sp[2]), n2,
                                                space_off(d, sp[3]), n3, pack1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (oz && oz->on) {
    // rows pq (K = P): pack0[P][pq]; rows rt: pack1[P][rt]
    const OzView va{pack0, 1, (long)n0 * n1, (long)d.X, 0}, vb{pack1, 1, (long)n2 * n3, (long)d.X, 0};
    return oz_matmul(*oz, va, vb, false, n0 * n1, n2 * n3, d.X, 1.0, 0.0, out, (long)n2 * n3, s);
  }
  return dgemm(n0 * n1, n2 * n3, d.X, 1.0, pack0, n0 * n1, true, pack1, n2 * n3, false, 0.0, out,
               n2 * n3, s);
}

void class_setup(int cls, const Dims& d, ClassWork& w) {
  const ClassDef& C = class_def(cls);
  w.cls = cls;
  DevClass& dc = w.dc;
  dc.nfam = C.nfam;
  dc.nslot = C.nslot;
  dc.next = C.next;
  dc.nact = C.nact;
  for (int k = 0; k < 4; ++k) dc.slot_space[k] = C.slot_space[k];
  for (int k = 0; k < 3; ++k) {
    dc.ext[k] = C.ext[k];
    dc.act[k] = C.act[k];
  }
  dc.pair0 = C.pair0;
  dc.pair1 = C.pair1;
  w.A = 1;
  for (int k = 0; k < C.nact; ++k) w.A *= d.a;
  w.m = (int)(C.nfam * w.A * d.n);
  long ext = 1;
  for (int k = 0; k < C.next; ++k) {
    w.ed.d[k] = space_dim(d, C.slot_space[C.ext[k]]);
    ext *= w.ed.d[k];
  }
  w.vsize = C.nfam * ext * w.A * d.n * d.n;
}

long class_sector_wsize(const ClassWork& w, const Dims& d, int scheme, long* partsize) {
  long wmax = 0, pmax = 0;
  for (int sec = 0; sec < 2; ++sec) {
    const long nt = sector_tuples(w, sec);
    const long msec = scheme == CASPT2_SSSR ? w.m / d.n : w.m;
    wmax = std::max(wmax, msec * nt * d.n);
    pmax = std::max(pmax, nt * (long)d.n * d.n * (d.n + 2));
  }
  if (partsize) *partsize = pmax;
  return wmax;
}

void class_keep_layout(ClassWork& w, const Dims& d, int scheme) {
  const int nsec = w.dc.pair0 < 0 ? 1 : 2;
  const int nsel = scheme == CASPT2_SSSR ? d.n : 1;
  w.keep.assign((size_t)nsec * nsel, SectorKeep{});
  for (int sec = 0; sec < nsec; ++sec)
    for (int is = 0; is < nsel; ++is) {
      SectorKeep& K = w.keep[sec * nsel + is];
      K.sec = sec;
      K.Lsel = scheme == CASPT2_SSSR ? is : -1;
      K.msec = scheme == CASPT2_SSSR ? w.m / d.n : w.m;
      K.ntup = sector_tuples(w, sec);
    }
}

long presum_size(const Dims& d, const PresumSpec& sp) {
  long n = 1;
  for (int p = 0; p < 4; ++p) n *= sp.var[p] < 0 ? space_dim(d, sp.space[p]) : 1;
  return n;
}

cudaError_t presum_block(const Dims& d, const PresumSpec& sp, const double* src, double* out,
                         cudaStream_t s) {
  const long total = presum_size(d, sp);
  if (total == 0) return cudaSuccess;
  ++launch_counter();
  k_presum<<<launch_blocks(total), 256, 0, s>>>(src, sp, space_dim(d, sp.space[0]),
                                                space_dim(d, sp.space[1]),
                                                space_dim(d, sp.space[2]),
                                                space_dim(d, sp.space[3]), out);
  return cudaGetLastError();
}

cudaError_t class_upload_plans(ClassWork& w, const std::vector<ActPlan>& S,
                               const std::vector<ActPlan>& F, const std::vector<SrcPlan>& V) {
  cudaError_t e;
  if ((e = cudaMemcpy(w.dS, S.data(), sizeof(ActPlan) * S.size(), cudaMemcpyHostToDevice)) != cudaSuccess) return e;
  if ((e = cudaMemcpy(w.dF, F.data(), sizeof(ActPlan) * F.size(), cudaMemcpyHostToDevice)) != cudaSuccess) return e;
  if ((e = cudaMemcpy(w.dV, V.data(), sizeof(SrcPlan) * V.size(), cudaMemcpyHostToDevice)) != cudaSuccess) return e;
  if (w.dVs && (e = cudaMemcpy(w.dVs, w.hVs.data(), sizeof(SrcPlan) * w.hVs.size(),
                               cudaMemcpyHostToDevice)) != cudaSuccess)
    return e;
  w.nVs = (int)w.hVs.size();
  if (w.dX) {
    std::vector<SrcXTerm> all;
    w.gx_off.clear();
    for (const SrcGemmGroup& G : w.hG) {
      w.gx_off.push_back((int)all.size());
      all.insert(all.end(), G.x.begin(), G.x.end());
    }
    if ((e = cudaMemcpy(w.dX, all.data(), sizeof(SrcXTerm) * all.size(),
                        cudaMemcpyHostToDevice)) != cudaSuccess)
      return e;
  }
  w.nS = (int)S.size();
  w.nF = (int)F.size();
  w.nV = (int)V.size();
  return cudaSuccess;
}

int class_solve(ClassWork& w, SectorWork& sw, const Dims& d, int scheme, double shift,
                double thresh, RdmPtrs rdm, const double* f_act, const double* h,
                const EriBlocks& eri, const PresumBlocks& pb, const double* E0,
                const double* eps_cv, double* mom, double* mindenom, cudaStream_t s,
                KernelTimer* tm, OzWork* oz, int ci0, int ci1) {
  const int m = w.m, n = d.n;
  if (w.vsize == 0 || m == 0) return CASPT2_OK;
  const long mm = (long)m * m;
  // overlap, active Fock, sources
  ++launch_counter();
  k_act_eval<<<launch_blocks(mm), 256, 0, s>>>(w.dS, w.nS, w.dc, d.a, n, rdm, f_act, w.Sact, m);
  ++launch_counter();
  k_act_eval<<<launch_blocks(mm), 256, 0, s>>>(w.dF, w.nF, w.dc, d.a, n, rdm, f_act, w.Fact, m);
  ++launch_counter();
  if (n <= 4) {
    const long total2 = w.vsize / ((long)n * n);
    k_src_eval_ml<4><<<launch_blocks(total2), 256, 0, s>>>(w.dVs, w.nVs, w.dc, d, rdm, h, eri, pb,
                                                          w.V, total2);
  } else if (n <= 8) {
    const long total2 = w.vsize / ((long)n * n);
    k_src_eval_m<8><<<launch_blocks(total2 * n), 256, 0, s>>>(w.dVs, w.nVs, w.dc, d, rdm, h, eri,
                                                              pb, w.V, total2);
  } else {
    k_src_eval<<<launch_blocks(w.vsize), 256, 0, s>>>(w.dVs, w.nVs, w.dc, d, rdm, h, eri, pb,
                                                      w.V, w.vsize);
  }
  CASPT2_CUDA_TRY(cudaGetLastError());
  // the terms of the GEMM groups: V[fam] += X G, X in row chunks
  if (!w.hG.empty()) {
    const long rows = all_tuples(w);
    const long ncol = w.A * n * n;
    for (size_t gi = 0; gi < w.hG.size(); ++gi) {
      const SrcGemmGroup& G = w.hG[gi];
      const long K = ipow_host(d.a, G.g.ns);
      if (K * ncol > sw.srcGcap) return CASPT2_EINVAL;
      ++launch_counter();
      k_src_g<<<launch_blocks(K * ncol), 256, 0, s>>>(G.g, w.dc, d, rdm, sw.srcG);
      CASPT2_CUDA_TRY(cudaGetLastError());
      const long chunk = std::min<long>(rows, sw.srcXcap / K);
      if (chunk < 1) return CASPT2_EINVAL;
      for (long r0 = 0; r0 < rows; r0 += chunk) {
        const long nr = std::min(chunk, rows - r0);
        ++launch_counter();
        k_src_x<<<launch_blocks(nr * K), 256, 0, s>>>(w.dX + w.gx_off[gi], (int)G.x.size(), w.dc,
                                                      d, G.g.ns, h, eri, pb, r0, nr, sw.srcX);
        CASPT2_CUDA_TRY(cudaGetLastError());
        double* Vc = w.V + ((long)G.fb * rows + r0) * ncol;
        if (oz && oz->on && oz->S >= kOzMaxSlices) {
          const OzView vx{sw.srcX, K, 1, K, 0}, vg{sw.srcG, 1, ncol, K, 0};
          CASPT2_CUDA_TRY(oz_matmul(*oz, vx, vg, false, (int)nr, (int)ncol, (int)K, 1.0, 1.0, Vc,
                                    ncol, s));
        } else {
          CASPT2_CUDA_TRY(dgemm((int)nr, (int)ncol, (int)K, 1.0, sw.srcX, (int)K, false, sw.srcG,
                                (int)ncol, false, 1.0, Vc, (int)ncol, s));
        }
      }
    }
  }

  const int nsec = w.dc.pair0 < 0 ? 1 : 2;
  for (int sec = 0; sec < nsec; ++sec) {
    const long ntup = sector_tuples(w, sec);
    if (ntup == 0) continue;
    const double sgn = w.dc.pair0 < 0 ? 0.0 : (sec == 0 ? 1.0 : -1.0);
    const int nsel = scheme == CASPT2_SSSR ? n : 1;
    for (int is = 0; is < nsel; ++is) {
      const int Lsel = scheme == CASPT2_SSSR ? is : -1;
      const int msec = scheme == CASPT2_SSSR ? m / n : m;
      const long ms2 = (long)msec * msec;
      ++launch_counter();
      k_sector<<<launch_blocks(ms2), 256, 0, s>>>(w.Sact, m, n, sgn, Lsel, sw.Ssec, msec);
      ++launch_counter();
      k_sector<<<launch_blocks(ms2), 256, 0, s>>>(w.Fact, m, n, sgn, Lsel, sw.Fsec, msec);
      CASPT2_CUDA_TRY(cudaGetLastError());
      SectorKeep& K = w.keep[sec * nsel + is];
      K.nk = 0;
      OzWork* ozn = (oz && oz->on && oz->S >= kOzMaxSlices) ? oz : nullptr;
      int st = sym_eig(sw.Ssec, msec, sw.s, sw.Qs, sw.jac, s, tm, ozn);
      if (st != CASPT2_OK) return st;
      // number of overlap eigenvalues at or above the threshold (ascending order)
      std::vector<double> hs(msec);
      CASPT2_CUDA_TRY(cudaMemcpyAsync(hs.data(), sw.s, sizeof(double) * msec,
                                      cudaMemcpyDeviceToHost, s));
      CASPT2_CUDA_TRY(cudaStreamSynchronize(s));
      int nk = 0;
      for (int k = 0; k < msec; ++k) nk += hs[k] >= thresh ? 1 : 0;
      if (nk == 0) continue;
      K.nk = nk;
      ++launch_counter();
      k_range_basis<<<launch_blocks((long)msec * nk), 256, 0, s>>>(sw.Qs, sw.s, msec, nk, sw.X);
      CASPT2_CUDA_TRY(cudaGetLastError());
      const bool ozx = oz && oz->on && oz->S >= kOzMaxSlices && msec >= kOzTransformMin;
      if (ozx) {
        // precision form, FP64-accurate split products (7 slices) for the sector
        // transforms F X, X^T (F X) and X Q of the large sectors
        const OzView vf{sw.Fsec, msec, 1, msec, 0}, vxt{sw.X, 1, nk, msec, 0};
        CASPT2_CUDA_TRY(oz_matmul(*oz, vf, vxt, false, msec, nk, msec, 1.0, 0.0, sw.FX, nk, s));
        const OzView vfx{sw.FX, 1, nk, msec, 0};
        CASPT2_CUDA_TRY(oz_matmul(*oz, vxt, vfx, false, nk, nk, msec, 1.0, 0.0, sw.Ft, nk, s));
        CASPT2_CUDA_TRY(launch_symmetrize(sw.Ft, nk, 1, s));
      } else {
        CASPT2_CUDA_TRY(dgemm(msec, nk, msec, 1.0, sw.Fsec, msec, false, sw.X, nk, false, 0.0,
                              sw.FX, nk, s));
        CASPT2_CUDA_TRY(dgemm_sym(nk, msec, 1.0, sw.X, nk, true, sw.FX, nk, false, 0.0, sw.Ft, nk,
                                  s));
      }
      st = sym_eig(sw.Ft, nk, K.omega, sw.Qf, sw.jac, s, tm, ozn);
      if (st != CASPT2_OK) return st;
      if (ozx) {
        const OzView vx{sw.X, nk, 1, nk, 0}, vq{sw.Qf, 1, nk, nk, 0};
        CASPT2_CUDA_TRY(oz_matmul(*oz, vx, vq, false, msec, nk, nk, 1.0, 0.0, K.Y, nk, s));
      } else {
        CASPT2_CUDA_TRY(dgemm(msec, nk, nk, 1.0, sw.X, nk, false, sw.Qf, nk, false, 0.0, K.Y, nk,
                              s));
      }
      {
        // eigenvalues next to small denominators: Rayleigh quotients in double-double
        // against the sector's S (rebuilt into Qs, free once X is formed) and F
        double* mdn = sw.part2;      // nk minima (free until the column sums below)
        if (nk > sw.p2size) return CASPT2_EINVAL;
        const double big = 1e300;
        ++launch_counter();
        k_fill<<<launch_blocks(nk), 256, 0, s>>>(mdn, nk, big);
        if (ntup <= sw.wcap) {
          // the tuples' external energies once into W (free until the sector sources)
          ++launch_counter();
          k_sector_eext<<<launch_blocks(ntup), 256, 0, s>>>(eps_cv, w.dc, w.ed, d.c, sec, ntup,
                                                            sw.W);
          ++launch_counter();
          k_mu_mindenom_ee<<<dim3((unsigned)std::min<long>((ntup + 255) / 256, 64), nk), 256, 0,
                             s>>>(K.omega, E0, sw.W, n, Lsel, ntup, shift, mdn);
        } else {
          ++launch_counter();
          k_mu_mindenom<<<dim3((unsigned)std::min<long>((ntup + 255) / 256, 64), nk), 256, 0,
                          s>>>(K.omega, E0, eps_cv, w.dc, w.ed, d.c, n, sec, Lsel, ntup, nk,
                               shift, mdn);
        }
        CASPT2_CUDA_TRY(cudaGetLastError());
        std::vector<double> hm(nk);
        CASPT2_CUDA_TRY(cudaMemcpyAsync(hm.data(), mdn, sizeof(double) * nk, cudaMemcpyDeviceToHost, s));
        CASPT2_CUDA_TRY(cudaStreamSynchronize(s));
        std::vector<int> list;
        for (int k = 0; k < nk; ++k)
          if (hm[k] < kRefineDenom) list.push_back(k);
        if (!list.empty()) {
          // list (ints) at the start of part2, the stage-1 partials in W (free here)
          const int nl = (int)list.size();
          const int nrb = (int)std::max<long>(1, std::min<long>(
              {(long)(msec + 63) / 64, 1216L / nl + 1, sw.wcap / (4L * nl)}));
          if ((long)nl > sw.p2size || 4L * nl * nrb > sw.wcap) return CASPT2_EINVAL;
          int* dlist = reinterpret_cast<int*>(sw.part2);
          CASPT2_CUDA_TRY(cudaMemcpyAsync(dlist, list.data(), sizeof(int) * nl,
                                          cudaMemcpyHostToDevice, s));
          ++launch_counter();
          k_sector<<<launch_blocks(ms2), 256, 0, s>>>(w.Sact, m, n, sgn, Lsel, sw.Qs, msec);
          ++launch_counter();
          k_rq_partial<<<dim3(nrb, nl), kRqThreads, 0, s>>>(sw.Qs, sw.Fsec, msec, K.Y, nk, dlist,
                                                           sw.W);
          ++launch_counter();
          k_rq_finish<<<(nl + 127) / 128, 128, 0, s>>>(sw.W, nrb, dlist, nl, K.omega);
          CASPT2_CUDA_TRY(cudaGetLastError());
          // eigenvectors: y_k += sum_j c_j y_j with the double-double residual of (F, S)
          double* R = sw.W;                                  // [msec][nl]
          double* Cm = R + (long)msec * nl;                  // [nk][nl]
          double* Dl = Cm + (long)nk * nl;                   // [msec][nl]
          if ((long)(2 * msec + nk) * nl > sw.wcap) return CASPT2_EINVAL;
          ++launch_counter();
          k_rq_resid<<<dim3(nrb, nl), kRqThreads, 0, s>>>(sw.Qs, sw.Fsec, msec, K.Y, nk, dlist, nl,
                                                         K.omega, R);
          CASPT2_CUDA_TRY(cudaGetLastError());
          CASPT2_CUDA_TRY(dgemm(nk, nl, msec, 1.0, K.Y, nk, true, R, nl, false, 0.0, Cm, nl, s));
          ++launch_counter();
          k_rq_coef<<<launch_blocks((long)nk * nl), 256, 0, s>>>(Cm, nk, dlist, nl, K.omega);
          CASPT2_CUDA_TRY(cudaGetLastError());
          CASPT2_CUDA_TRY(dgemm(msec, nl, nk, 1.0, K.Y, nk, false, Cm, nl, false, 0.0, Dl, nl, s));
          ++launch_counter();
          k_rq_apply<<<launch_blocks((long)msec * nl), 256, 0, s>>>(K.Y, msec, nk, dlist, nl, Dl);
          CASPT2_CUDA_TRY(cudaGetLastError());
          CASPT2_CUDA_TRY(cudaStreamSynchronize(s));   // the host list is released below
        }
      }
      const long ncol = ntup * n;
      const int nL = Lsel < 0 ? n : 1;
      const int pcol = nL * n * (n + 2);
      // tuples in chunks so that the sector sources W (msec x chunk n) and the moment
      // partials (chunk x pcol) stay within the work arrays the context holds
      long chunk = std::min<long>(ntup, sw.wcap / ((long)msec * n));
      chunk = std::min<long>(chunk, sw.pcap / pcol);
      if (chunk < 1 || (long)nk * ncol > (1L << 62)) return CASPT2_EINVAL;
      // class G under a closed-orbital range: the sector tuples are ordered with the
      // closed index slowest, so the range is a contiguous run of them
      long tb = 0, te = ntup;
      if (w.cls == CASPT2_CLASS_G && (ci0 > 0 || (ci1 >= 0 && ci1 < d.c))) {
        const long per_i = ntup / d.c;
        tb = (long)ci0 * per_i;
        te = (long)(ci1 < 0 || ci1 > d.c ? d.c : ci1) * per_i;
      }
      for (long t0 = tb; t0 < te; t0 += chunk) {
        const long nt = std::min(chunk, te - t0);
        ++launch_counter();
        k_sector_src<<<launch_blocks((long)(scheme == CASPT2_SSSR ? msec : msec / n) * nt), 256, 0, s>>>(
            w.V, w.dc, w.ed, d.a, n, sec, Lsel, t0, nt, msec, sw.W);
        CASPT2_CUDA_TRY(cudaGetLastError());
        if (oz && oz->on && oz->S >= kOzMaxSlices) {
          // precision form with every product FP64-accurate (7 slices): the sector
          // transform as a split-BF16 tensor-core product (fewer slices keep it in FP64:
          // the energies are first order in its rounding)
          const OzView vy{K.Y, 1, nk, msec, 0};               // rows mu, K = sector row
          const OzView vw{sw.W, 1, nt * n, msec, 0};           // rows (t, L'), K = sector row
          CASPT2_CUDA_TRY(oz_matmul(*oz, vy, vw, false, nk, (int)(nt * n), msec, 1.0, 0.0,
                                    K.Vt + t0 * n, ncol, s));
        } else {
          CASPT2_CUDA_TRY(dgemm(nk, (int)(nt * n), msec, 1.0, K.Y, nk, true, sw.W,
                                (int)(nt * n), false, 0.0, K.Vt + t0 * n, (int)ncol, s));
        }
        ++launch_counter();
        if (n <= 4) {
          k_sector_energy_ml<4><<<launch_blocks(nt * nL), 256, 0, s>>>(
              K.Vt, K.omega, E0, eps_cv, w.dc, w.ed, d.c, n, sec, Lsel, ntup, t0, nt, nk, shift,
              sw.part, mindenom);
        } else if (n <= 6) {
          k_sector_energy_ml<6><<<launch_blocks(nt * nL), 256, 0, s>>>(
              K.Vt, K.omega, E0, eps_cv, w.dc, w.ed, d.c, n, sec, Lsel, ntup, t0, nt, nk, shift,
              sw.part, mindenom);
        } else {
          const long ne = nt * nL * n;
          k_sector_energy<<<launch_blocks(ne), 256, 0, s>>>(K.Vt, K.omega, E0, eps_cv, w.dc, w.ed,
                                                            d.c, n, sec, Lsel, ntup, t0, nt, nk,
                                                            shift, sw.part, mindenom);
        }
        // fixed-order column sums: row blocks, then the block partials in order
        const long nb = std::min<long>(sw.nb2, std::max<long>(1, nt / 64));
        ++launch_counter();
        k_colsum_rows<<<(unsigned)nb, 256, 0, s>>>(sw.part, nt, pcol, sw.part2);
        ++launch_counter();
        k_moment_colsum<<<pcol, 256, 0, s>>>(sw.part2, nb, n, nL, Lsel, mom);
        CASPT2_CUDA_TRY(cudaGetLastError());
      }
    }
  }
  return CASPT2_OK;
}

}  // namespace caspt2
