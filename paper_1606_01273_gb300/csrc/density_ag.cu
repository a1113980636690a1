// Classes A-G: the class share of the correlated densities of a target state P
// (Sec. II.D) from the sector bases kept by the energy pass.
//
// With R the eigenvectors of H^eff, r = R[:, P], and T_L, lambda_L the first-order
// amplitudes and the lambda amplitudes (Eq. lambdaeq) over all index tuples,
//   W_L'   = r_L' sum_L r_L T_L + lambda_L'                (source multiplier)
//   d1_pq  = sum W <M~|E_Omega^dag E_pq|L'~>                (d/dh of the sources)
//   G_pqrt = sum W <M~|E_Omega^dag 1/2 E_pq,rt|L'~>         (d/d(pq|rt))
//   d2     = d L / d f on the closed, active and virtual blocks:
//            closed/virtual: one external slot of T moves (hole or particle line of
//            f), contracted through the overlap (identity or pair swap);
//            active: lambda x T contracted with the d/df_uw of F_act, minus
//            N_L <L~|E_uw|L~> from the E0 dependence of the denominators.
// All contractions reuse the access plans of the solve (transposed), so the device
// path shares the solve's normal ordering and index conventions.
#include <cmath>
#include <vector>

#include "class_ag.cuh"
#include "class_dev.cuh"
#include "linalg.cuh"

namespace caspt2 {

namespace {

constexpr double kInvSqrt2 = 0.70710678118654752440;
constexpr long kActAdjSmem = 96L * 1024;

// Sector amplitudes and lambda in the eigenbasis mu of the sector, for every
// (tuple t, state L): amp = -Vt_L / D_L, lam = -(r_L sum_N r_N Vt_N - 2 E_s r_L^2 amp) / D_L,
// D_L = e_ext(t) + omega_mu - E0_L + E_s.  Layout [mu][t][Li] (Li = L, or 0 for SS-SR).
__global__ void k_sector_amp(const double* __restrict__ Vt, const double* __restrict__ omega,
                             const double* __restrict__ E0, const double* __restrict__ eps,
                             const double* __restrict__ R, int P, DevClass C, ExtDims ed, int c,
                             int n, int sector, int Lsel, long ntup, int nk, double shift,
                             double* __restrict__ amp, double* __restrict__ lam) {
  const int nL = Lsel < 0 ? n : 1;
  const long ncolV = ntup * n;
  const long total = (long)nk * ntup * nL;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    const int Li = e % nL;
    const long t = (e / nL) % ntup;
    const long mu = e / (nL * ntup);
    const int L = Lsel < 0 ? Li : Lsel;
    int co[3], cs[3];
    sector_tuple(C, ed.d, sector, t, co, cs);
    double ee = 0.0;
    for (int k = 0; k < C.next; ++k)
      ee += (C.slot_space[C.ext[k]] == SP_V) ? eps[c + co[k]] : -eps[co[k]];
    const double D = ee + omega[mu] - E0[L] + shift;
    const double* row = Vt + mu * ncolV + t * n;
    const double am = -row[L] / D;
    double acc = 0.0;
    for (int N = 0; N < n; ++N) acc += R[N * n + P] * row[N];
    const double rl = R[L * n + P];
    amp[e] = am;
    lam[e] = -(rl * acc - 2.0 * shift * rl * rl * am) / D;
  }
}

// Sector rows src[i][(t, Li)] (i over the sector rows) -> all-tuple arrays
// dst[tuple][L][row]; pair classes: a pair (x, y), x < y, receives (T+ + T-)/sqrt2 and its
// swap (T+ - T-)/sqrt2, x = y receives T+.  Two arrays (T and lambda) per launch.
__global__ void k_tuple_scatter(const double* __restrict__ src0, const double* __restrict__ src1,
                                DevClass C, ExtDims ed, int n, int m, int sector, int Lsel,
                                long ntup, int msec, double* __restrict__ dst0,
                                double* __restrict__ dst1) {
  const int nL = Lsel < 0 ? n : 1;
  const long ncol = ntup * nL;
  const long total = (long)msec * ncol;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    const long i = e / ncol, col = e % ncol;
    const long t = col / nL;
    const int Li = col % nL;
    const int L = Lsel < 0 ? Li : Lsel;
    const long row = Lsel < 0 ? i : i * n + Lsel;
    int co[3], cs[3];
    sector_tuple(C, ed.d, sector, t, co, cs);
    const long ia = (tuple_index(C, ed.d, co) * n + L) * m + row;
    const long ib = (tuple_index(C, ed.d, cs) * n + L) * m + row;
    const double x0 = src0[e], x1 = src1[e];
    if (C.pair0 < 0) {
      dst0[ia] = x0;
      dst1[ia] = x1;
    } else if (ia == ib) {
      dst0[ia] += x0;
      dst1[ia] += x1;
    } else {
      const double sg = sector == 0 ? kInvSqrt2 : -kInvSqrt2;
      dst0[ia] += kInvSqrt2 * x0;
      dst1[ia] += kInvSqrt2 * x1;
      dst0[ib] += sg * x0;
      dst1[ib] += sg * x1;
    }
  }
}

// dst[t][inner] = src[swap(t)][inner], swap exchanging the pair slots of the tuple.
__global__ void k_swap_tuples(const double* __restrict__ src, DevClass C, ExtDims ed, long ntot,
                              long inner, double* __restrict__ dst) {
  int ip = 0, jp = 0;
  for (int k = 0; k < C.next; ++k) {
    if (C.ext[k] == C.pair0) ip = k;
    if (C.ext[k] == C.pair1) jp = k;
  }
  const long total = ntot * inner;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    long t = e / inner;
    const long r = e % inner;
    int co[3];
    for (int k = C.next - 1; k >= 0; --k) {
      co[k] = t % ed.d[k];
      t /= ed.d[k];
    }
    const int x = co[ip];
    co[ip] = co[jp];
    co[jp] = x;
    dst[e] = src[tuple_index(C, ed.d, co) * inner + r];
  }
}

// Split-K Gram product over a tensor viewed as [pre][Ns][post]:
//   part[z][x][y] = sum_{k in chunk z} A(x, k) B(y, k),  k = (p, q) over pre x post,
//   A(x, (p, q)) = A[(p * Ns + x) * post + q].
// Output tile TS x TS per block (TS <= 32 fitted to Ns), up to 4 outputs per thread,
// K staged in chunks of 16 through shared memory; FP64 FMA.
constexpr int kGS = 32, kGK = 16;
__global__ void __launch_bounds__(256)
k_gram(const double* __restrict__ A, const double* __restrict__ B, long Ns, unsigned post,
       unsigned K, unsigned chunk, int TS, double* __restrict__ part) {
  __shared__ double sa[kGK][kGS + 1], sb[kGK][kGS + 1];
  const long x0 = (long)blockIdx.y * TS, y0 = (long)blockIdx.x * TS;
  const unsigned kbeg = blockIdx.z * chunk;
  const unsigned kend = min(K, kbeg + chunk);
  const bool xfast = post == 1u;
  const int nout = TS * TS;
  int ox[4], oy[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int q = threadIdx.x + 256 * r;
    ox[r] = q < nout ? q / TS : 0;
    oy[r] = q < nout ? q % TS : 0;
  }
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (unsigned k0 = kbeg; k0 < kend; k0 += kGK) {
    for (int l = threadIdx.x; l < kGK * TS; l += 256) {
      int kk, ii;
      if (xfast) { ii = l % TS; kk = l / TS; } else { kk = l % kGK; ii = l / kGK; }
      const unsigned gk = k0 + kk;
      const long gx = x0 + ii, gy = y0 + ii;
      double va = 0.0, vb = 0.0;
      if (gk < kend) {
        const unsigned p = gk / post, q = gk - p * post;
        const long base = (long)p * Ns * post + q;
        if (gx < Ns) va = A[base + gx * post];
        if (gy < Ns) vb = B[base + gy * post];
      }
      sa[kk][ii] = va;
      sb[kk][ii] = vb;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < kGK; ++kk) {
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[r] = fma(sa[kk][ox[r]], sb[kk][oy[r]], acc[r]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int q = threadIdx.x + 256 * r;
    const long gx = x0 + ox[r], gy = y0 + oy[r];
    if (q < nout && gx < Ns && gy < Ns) part[((long)blockIdx.z * Ns + gx) * Ns + gy] = acc[r];
  }
}

// Fixed-order sum of the split-K partials.  mode 0: out[x][y] = X; mode 1 (closed
// block): out[off + y][off + x] -= X; mode 2 (virtual block): out[off + x][off + y] += X.
__global__ void k_gram_finish(const double* __restrict__ part, int nsplit, long Ns, int mode,
                              double* __restrict__ out, long ld, long off) {
  const long total = Ns * Ns;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int z = 0; z < nsplit; ++z) s += part[(long)z * total + e];
    const long x = e / Ns, y = e % Ns;
    if (mode == 0) out[x * ld + y] = s;
    else if (mode == 1) out[(off + y) * ld + off + x] -= s;
    else out[(off + x) * ld + off + y] += s;
  }
}

// Active block of d2: partial sums over (row, col) of D^pi[row][col] dF_act^pi/df_uw.
// Each thread takes its own (row, col) elements, evaluates every plan term once (as the
// forward evaluation does) and adds coeff * D * Gamma into its private column of
// acc[uw][thread] in shared memory at uw = (f index 0, f index 1); a fixed-order sum over
// the threads gives part[block][a^2].
__global__ void k_act_adj(const ActPlan* __restrict__ plans, int nplan, DevClass C, int a, int n,
                          RdmPtrs g, const double* __restrict__ Dm, int m,
                          double* __restrict__ part) {
  extern __shared__ double acc[];   // [a^2][blockDim.x]
  const int a2 = a * a, nt = blockDim.x, tid = threadIdx.x;
  for (int q = 0; q < a2; ++q) acc[q * nt + tid] = 0.0;
  const long total = (long)m * m;
  const long A = ipow(a, C.nact);
  for (long e = (long)blockIdx.x * nt + tid; e < total; e += (long)gridDim.x * nt) {
    const double D0 = Dm[e], D1 = Dm[total + e];
    if (D0 == 0.0 && D1 == 0.0) continue;
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
    for (int t = 0; t < nplan; ++t) {
      const ActPlan& P = plans[t];
      if (!P.has_f || P.fb != fb || P.fk != fk) continue;
      const double Dv = P.pi == 0 ? D0 : D1;
      if (Dv == 0.0) continue;
      bool ok = true;
      for (int q = 0; q < P.neq; ++q)
        if (vals[P.eq[q][0]] != vals[P.eq[q][1]]) ok = false;
      if (!ok) continue;
      const int nl = P.nloop;
      const int niter = nl == 0 ? 1 : (nl == 1 ? a : a * a);
      const double cd = P.coeff * Dv;
      for (int it = 0; it < niter; ++it) {
        if (nl >= 1) vals[kRefLoop] = it % a;
        if (nl >= 2) vals[kRefLoop + 1] = it / a;
        const double x = rdm_at(g.p, P.rank, n, a, M, N, vals, P.idx);
        const int uw = vals[P.fidx[0]] * a + vals[P.fidx[1]];
        acc[uw * nt + tid] += cd * x;
      }
    }
  }
  __syncthreads();
  for (int q = tid; q < a2; q += nt) {
    double t = 0.0;
    for (int j = 0; j < nt; ++j) t += acc[q * nt + j];
    part[(long)blockIdx.x * a2 + q] = t;
  }
}

// d2[c + u][c + w] += sum_blocks part[b][uw] - sum_L NL[L] Gamma1[L][L][u][w]
__global__ void k_act_finish(const double* __restrict__ part, int nblk, int a, int c, int nmo,
                             const double* __restrict__ NL, const double* __restrict__ g1, int n,
                             double* __restrict__ d2) {
  const int a2 = a * a;
  for (int uw = threadIdx.x; uw < a2; uw += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += part[(long)b * a2 + uw];
    for (int L = 0; L < n; ++L) s -= NL[L] * g1[((long)L * n + L) * a2 + uw];
    d2[(long)(c + uw / a) * nmo + c + uw % a] += s;
  }
}

// W[t][L'][row] = r_L' sum_L r_L T[t][L][row] + Lam[t][L'][row]
__global__ void k_wsrc(const double* __restrict__ T, const double* __restrict__ Lam,
                       const double* __restrict__ R, int P, int n, long m, long total,
                       double* __restrict__ W) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    const long row = e % m;
    const int Lp = (e / m) % n;
    const long t = e / (m * n);
    double acc = 0.0;
    for (int L = 0; L < n; ++L) acc += R[L * n + P] * T[(t * n + L) * m + row];
    W[e] = R[Lp * n + P] * acc + Lam[e];
  }
}

__device__ __forceinline__ void flush_add(double* p, double v) {
  if (p != nullptr && v != 0.0) atomicAdd(p, v);
}

// Adjoint of the sources: for every V element (fam, ext, act, M, L') with multiplier
// W, each plan term coeff * I[...] * Gamma adds coeff * W * Gamma to dI[...] (d1 for the
// one-electron part, G blocks for (pq|rt)).  Runs of equal targets are summed before
// the atomic add.
__global__ void k_src_adj(const SrcPlan* __restrict__ plans, int nplan, DevClass C, Dims d,
                          RdmPtrs g, const double* __restrict__ W, long m, long vtotal,
                          double* __restrict__ d1, EriBlocks G) {
  const int n = d.n, a = d.a, nmo = d.nmo();
  const int dimsp[3] = {d.c, d.a, d.v};
  const int offsp[3] = {0, d.c, d.c + d.a};
  const long A = ipow(a, C.nact);
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < vtotal;
       e += (long)gridDim.x * blockDim.x) {
    long r = e;
    const int L = r % n; r /= n;
    const int M = r % n; r /= n;
    const long actlin = r % A; r /= A;
    int vals[24];
    long q = actlin;
    for (int k = C.nact - 1; k >= 0; --k) {
      vals[kRefBra + C.act[k]] = q % a;
      q /= a;
    }
    int co[3];
    for (int k = C.next - 1; k >= 0; --k) {
      const int dm = dimsp[C.slot_space[C.ext[k]]];
      co[k] = r % dm;
      vals[kRefBra + C.ext[k]] = co[k];
      r /= dm;
    }
    const int fam = (int)r;
    long t = 0;
    for (int k = 0; k < C.next; ++k) t = t * dimsp[C.slot_space[C.ext[k]]] + co[k];
    const double Wv = W[(t * n + L) * m + (fam * A + actlin) * n + M];
    if (Wv == 0.0) continue;
    double* last = nullptr;
    double run = 0.0;
    for (int tp = 0; tp < nplan; ++tp) {
      const SrcPlan& P = plans[tp];
      if (P.fb != fam) continue;
      bool ok = true;
      for (int qq = 0; qq < P.neq; ++qq)
        if (vals[P.eq[qq][0]] != vals[P.eq[qq][1]]) ok = false;
      if (!ok) continue;
      long niter = 1;
      for (int j = 0; j < P.nloop; ++j) niter *= dimsp[P.loop_space[j]];
      double* blk = nullptr;
      long bd[4] = {1, 1, 1, 1};
      if (P.kind == 1) {
        const int key = ((P.ispace[0] * 3 + P.ispace[1]) * 3 + P.ispace[2]) * 3 + P.ispace[3];
        blk = const_cast<double*>(G.p[key]);
        for (int j = 0; j < 4; ++j) bd[j] = dimsp[P.ispace[j]];
      }
      const double cw = P.coeff * Wv;
      for (long it = 0; it < niter; ++it) {
        long qi = it;
        for (int j = 0; j < P.nloop; ++j) {
          const int dm = dimsp[P.loop_space[j]];
          vals[kRefLoop + j] = qi % dm;
          qi /= dm;
        }
        const double x = rdm_at(g.p, P.rank, n, a, M, L, vals, P.idx);
        if (x == 0.0) continue;
        double* tgt;
        if (P.kind == 0) {
          tgt = d1 + (long)(offsp[P.ispace[0]] + vals[P.iidx[0]]) * nmo + offsp[P.ispace[1]] +
                vals[P.iidx[1]];
        } else {
          tgt = blk + ((vals[P.iidx[0]] * bd[1] + vals[P.iidx[1]]) * bd[2] + vals[P.iidx[2]]) *
                          bd[3] + vals[P.iidx[3]];
        }
        if (tgt != last) {
          flush_add(last, run);
          last = tgt;
          run = 0.0;
        }
        run += cw * x;
      }
    }
    flush_add(last, run);
  }
}

// Source adjoint with one thread per (fam, ext, act) and the n^2 multipliers W[M][L'] (n <=
// NS) in registers: each plan term adds coeff * sum_(M,L') W Gamma[M][L'][off] to its
// target with one atomic per run of equal targets.
template <int NS>
__global__ void k_src_adj_ml(const SrcPlan* __restrict__ plans, int nplan, DevClass C, Dims d,
                             RdmPtrs g, const double* __restrict__ W, long m, long total2,
                             double* __restrict__ d1, EriBlocks G) {
  const int n = d.n, a = d.a, nmo = d.nmo();
  const int dimsp[3] = {d.c, d.a, d.v};
  const int offsp[3] = {0, d.c, d.c + d.a};
  const long A = ipow(a, C.nact);
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total2;
       e += (long)gridDim.x * blockDim.x) {
    long r = e;
    const long actlin = r % A;
    r /= A;
    int vals[24];
    long q = actlin;
    for (int k = C.nact - 1; k >= 0; --k) {
      vals[kRefBra + C.act[k]] = q % a;
      q /= a;
    }
    int co[3];
    for (int k = C.next - 1; k >= 0; --k) {
      const int dm = dimsp[C.slot_space[C.ext[k]]];
      co[k] = r % dm;
      vals[kRefBra + C.ext[k]] = co[k];
      r /= dm;
    }
    const int fam = (int)r;
    long t = 0;
    for (int k = 0; k < C.next; ++k) t = t * dimsp[C.slot_space[C.ext[k]]] + co[k];
    double wv[NS * NS];
    bool any = false;
#pragma unroll
    for (int M = 0; M < NS; ++M)
#pragma unroll
      for (int L = 0; L < NS; ++L) {
        const double x = (M < n && L < n) ? W[(t * n + L) * m + (fam * A + actlin) * n + M] : 0.0;
        wv[M * NS + L] = x;
        any = any || x != 0.0;
      }
    if (!any) continue;
    double* last = nullptr;
    double run = 0.0;
    for (int tp = 0; tp < nplan; ++tp) {
      const SrcPlan& P = plans[tp];
      if (P.fb != fam) continue;
      bool ok = true;
      for (int qq = 0; qq < P.neq; ++qq)
        if (vals[P.eq[qq][0]] != vals[P.eq[qq][1]]) ok = false;
      if (!ok) continue;
      long niter = 1;
      for (int j = 0; j < P.nloop; ++j) niter *= dimsp[P.loop_space[j]];
      double* blk = nullptr;
      long bd[4] = {1, 1, 1, 1};
      if (P.kind == 1) {
        const int key = ((P.ispace[0] * 3 + P.ispace[1]) * 3 + P.ispace[2]) * 3 + P.ispace[3];
        blk = const_cast<double*>(G.p[key]);
        for (int j = 0; j < 4; ++j) bd[j] = dimsp[P.ispace[j]];
      }
      const long stride = ipow(a, 2 * P.rank);
      for (long it = 0; it < niter; ++it) {
        long qi = it;
        for (int j = 0; j < P.nloop; ++j) {
          const int dm = dimsp[P.loop_space[j]];
          vals[kRefLoop + j] = qi % dm;
          qi /= dm;
        }
        double gs = 0.0;
        if (P.rank == 0) {
#pragma unroll
          for (int M = 0; M < NS; ++M) gs += wv[M * NS + M];
        } else {
          long off = 0;
          for (int j = 0; j < 2 * P.rank; ++j) off = off * a + vals[P.idx[j]];
          const double* gp = g.p[P.rank] + off;
#pragma unroll
          for (int M = 0; M < NS; ++M)
#pragma unroll
            for (int L = 0; L < NS; ++L)
              if (M < n && L < n) gs += wv[M * NS + L] * gp[(long)(M * n + L) * stride];
        }
        if (gs == 0.0) continue;
        double* tgt;
        if (P.kind == 0) {
          tgt = d1 + (long)(offsp[P.ispace[0]] + vals[P.iidx[0]]) * nmo + offsp[P.ispace[1]] +
                vals[P.iidx[1]];
        } else {
          tgt = blk + ((vals[P.iidx[0]] * bd[1] + vals[P.iidx[1]]) * bd[2] + vals[P.iidx[2]]) *
                          bd[3] + vals[P.iidx[3]];
        }
        if (tgt != last) {
          flush_add(last, run);
          last = tgt;
          run = 0.0;
        }
        run += P.coeff * gs;
      }
    }
    flush_add(last, run);
  }
}

__global__ void k_symmetrize(double* __restrict__ x, int nmo, long batch) {
  const long nn = (long)nmo * nmo;
  const long total = batch * nn;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    const long r = e % nn;
    const int i = r / nmo, j = r % nmo;
    if (i >= j) continue;
    double* m = x + (e - r);
    const double s = 0.5 * (m[(long)i * nmo + j] + m[(long)j * nmo + i]);
    m[(long)i * nmo + j] = s;
    m[(long)j * nmo + i] = s;
  }
}

}  // namespace

// X = sum over (pre, post) of A(x, .) B(y, .) for [pre][Ns][post] tensors, finished
// into `out` according to `mode` (see k_gram_finish).
int gram_product(const double* A, const double* B, long pre, long Ns, long post, int mode,
                 double* out, long ld, long off, double* part, long partmax, cudaStream_t s,
                 OzWork* oz) {
  if (pre * Ns * post == 0) return CASPT2_OK;
  const long K = pre * post;
  if (K >= (1L << 31) || Ns * Ns > partmax) return CASPT2_EINVAL;
  if (oz && oz->on) {
    // element (x, (p, q)) of a [pre][Ns][post] tensor: x * post + p * Ns * post + q
    const OzView va{A, post, 1, post, Ns * post}, vb{B, post, 1, post, Ns * post};
    CASPT2_CUDA_TRY(oz_matmul(*oz, va, vb, A == B, (int)Ns, (int)Ns, (int)K, 1.0, 0.0, part, Ns,
                              s));
    ++launch_counter();
    k_gram_finish<<<launch_blocks(Ns * Ns), 256, 0, s>>>(part, 1, Ns, mode, out, ld, off);
    CASPT2_CUDA_TRY(cudaGetLastError());
    return CASPT2_OK;
  }
  const long ntile = (Ns + kGS - 1) / kGS;
  const int TS = (int)((Ns + ntile - 1) / ntile);        // tile edge fitted to Ns
  const long tiles = ntile * ntile;
  long nsplit = std::max<long>(1, (152L * 4 + tiles - 1) / tiles);
  nsplit = std::min(nsplit, std::max<long>(1, K / 256));
  nsplit = std::min(nsplit, partmax / (Ns * Ns));
  long chunk = (K + nsplit - 1) / nsplit;
  chunk = (chunk + kGK - 1) / kGK * kGK;
  nsplit = (K + chunk - 1) / chunk;
  dim3 grid((unsigned)ntile, (unsigned)ntile, (unsigned)nsplit);
  ++launch_counter();
  k_gram<<<grid, 256, 0, s>>>(A, B, Ns, (unsigned)post, (unsigned)K, (unsigned)chunk, TS, part);
  ++launch_counter();
  k_gram_finish<<<launch_blocks(Ns * Ns), 256, 0, s>>>(part, (int)nsplit, Ns, mode, out, ld, off);
  CASPT2_CUDA_TRY(cudaGetLastError());
  return CASPT2_OK;
}

long class_dens_tall(const ClassWork& w, const Dims& d) {
  if (w.vsize == 0 || w.m == 0) return 0;
  return all_tuples(w) * d.n * w.m;
}

cudaError_t launch_symmetrize(double* x, int nmo, long batch, cudaStream_t s) {
  const long total = batch * (long)nmo * nmo;
  if (total == 0) return cudaSuccess;
  ++launch_counter();
  k_symmetrize<<<launch_blocks(total), 256, 0, s>>>(x, nmo, batch);
  return cudaGetLastError();
}

int class_tuple_amplitudes(ClassWork& w, DensWork& dw, const Dims& d, double shift,
                           const double* E0, const double* eps_cv, const double* R, int P,
                           OzWork* oz, cudaStream_t s) {
  const int m = w.m, n = d.n;
  if (w.vsize == 0 || m == 0) return CASPT2_OK;
  const DevClass& C = w.dc;
  const long ntot = all_tuples(w);
  const long tall = ntot * n * m;
  if (tall > dw.tall) return CASPT2_EINVAL;
  CASPT2_CUDA_TRY(cudaMemsetAsync(dw.T, 0, sizeof(double) * tall, s));
  CASPT2_CUDA_TRY(cudaMemsetAsync(dw.Lam, 0, sizeof(double) * tall, s));

  // ---- amplitudes and lambda of every sector, back-transformed to all tuples
  for (const SectorKeep& K : w.keep) {
    if (K.nk == 0 || K.ntup == 0) continue;
    const int nL = K.Lsel < 0 ? n : 1;
    const long ncol = K.ntup * nL;
    if ((long)K.nk * ncol > dw.secmax || (long)K.msec * ncol > dw.secmax) return CASPT2_EINVAL;
    double* amp = dw.sec;
    double* lam = dw.sec + dw.secmax;
    ++launch_counter();
    k_sector_amp<<<launch_blocks((long)K.nk * ncol), 256, 0, s>>>(
        K.Vt, K.omega, E0, eps_cv, R, P, C, w.ed, d.c, n, K.sec, K.Lsel, K.ntup, K.nk, shift, amp,
        lam);
    CASPT2_CUDA_TRY(cudaGetLastError());
    // rows = Y (msec x nk) times sector columns, for amp and lam together
    if (oz && oz->on) {
      const OzView vy{K.Y, K.nk, 1, K.nk, 0};                   // rows i, K = mu
      for (int q = 0; q < 2; ++q) {
        const OzView vs{dw.sec + q * dw.secmax, 1, ncol, K.nk, 0};   // rows col, K = mu
        CASPT2_CUDA_TRY(oz_matmul(*oz, vy, vs, false, K.msec, (int)ncol, K.nk, 1.0, 0.0,
                                  dw.tmp + q * dw.secmax, ncol, s));
      }
    } else {
      CASPT2_CUDA_TRY(dgemm(K.msec, (int)ncol, K.nk, 1.0, K.Y, K.nk, false, dw.sec, (int)ncol,
                            false, 0.0, dw.tmp, (int)ncol, s, 2, 0, dw.secmax, dw.secmax));
    }
    ++launch_counter();
    k_tuple_scatter<<<launch_blocks((long)K.msec * ncol), 256, 0, s>>>(
        dw.tmp, dw.tmp + dw.secmax, C, w.ed, n, m, K.sec, K.Lsel, K.ntup, K.msec, dw.T, dw.Lam);
    CASPT2_CUDA_TRY(cudaGetLastError());
  }
  return CASPT2_OK;
}

int class_densities(ClassWork& w, DensWork& dw, const Dims& d, int scheme, double shift,
                    RdmPtrs rdm, const double* E0, const double* eps_cv, const double* R, int P,
                    const double* NL, const EriBlocks& G, double* d1, double* d2, OzWork* oz,
                    cudaStream_t s) {
  (void)scheme;
  const int m = w.m, n = d.n, a = d.a, nmo = d.nmo();
  if (w.vsize == 0 || m == 0) return CASPT2_OK;
  const DevClass& C = w.dc;
  const long ntot = all_tuples(w);
  const long tall = ntot * n * m;
  if (a * a > 256) return CASPT2_EINVAL;
  {
    const int st = class_tuple_amplitudes(w, dw, d, shift, E0, eps_cv, R, P, oz, s);
    if (st != CASPT2_OK) return st;
  }
  const bool pair = C.pair0 >= 0;
  const long mm = (long)m * m;
  // ---- overlap applied to T: U1 = S^id T, U2 = S^sw T (rows of T are (tuple, L))
  if (oz && oz->on) {
    const OzView vt{dw.T, m, 1, m, 0}, vs1{w.Sact, m, 1, m, 0}, vs2{w.Sact + mm, m, 1, m, 0};
    CASPT2_CUDA_TRY(oz_matmul(*oz, vt, vs1, false, (int)(ntot * n), m, m, 1.0, 0.0, dw.U1, m, s));
    if (pair)
      CASPT2_CUDA_TRY(oz_matmul(*oz, vt, vs2, false, (int)(ntot * n), m, m, 1.0, 0.0, dw.U2, m, s));
  } else {
    CASPT2_CUDA_TRY(dgemm((int)(ntot * n), m, m, 1.0, dw.T, m, false, w.Sact, m, true, 0.0, dw.U1,
                          m, s));
    if (pair)
      CASPT2_CUDA_TRY(dgemm((int)(ntot * n), m, m, 1.0, dw.T, m, false, w.Sact + mm, m, true, 0.0,
                            dw.U2, m, s));
  }
  // ---- closed and virtual blocks: one external slot moves
  auto slot_blocks = [&](const double* Lm, const double* U) -> int {
    long pre = 1;
    for (int k = 0; k < C.next; ++k) {
      const long Ns = w.ed.d[k];
      long post = (long)n * m;
      for (int k2 = k + 1; k2 < C.next; ++k2) post *= w.ed.d[k2];
      const int sp = C.slot_space[C.ext[k]];
      const int st = gram_product(Lm, U, pre, Ns, post, sp == SP_C ? 1 : 2, d2, nmo,
                                  space_off(d, sp), dw.part, dw.partmax, s, oz);
      if (st != CASPT2_OK) return st;
      pre *= Ns;
    }
    return CASPT2_OK;
  };
  int st = slot_blocks(dw.Lam, dw.U1);
  if (st != CASPT2_OK) return st;
  if (pair) {
    ++launch_counter();
    k_swap_tuples<<<launch_blocks(tall), 256, 0, s>>>(dw.Lam, C, w.ed, ntot, (long)n * m, dw.Tsw);
    CASPT2_CUDA_TRY(cudaGetLastError());
    st = slot_blocks(dw.Tsw, dw.U2);
    if (st != CASPT2_OK) return st;
  }
  // ---- active block: D^pi = sum_(tuple, L) lambda x T^pi, contracted with dF_act/df
  st = gram_product(dw.Lam, dw.T, ntot * n, m, 1, 0, dw.Dm, m, 0, dw.part, dw.partmax, s, oz);
  if (st != CASPT2_OK) return st;
  if (pair) {
    ++launch_counter();
    k_swap_tuples<<<launch_blocks(tall), 256, 0, s>>>(dw.T, C, w.ed, ntot, (long)n * m, dw.Tsw);
    CASPT2_CUDA_TRY(cudaGetLastError());
    st = gram_product(dw.Lam, dw.Tsw, ntot * n, m, 1, 0, dw.Dm + mm, m, 0, dw.part, dw.partmax,
                      s, oz);
    if (st != CASPT2_OK) return st;
  } else {
    CASPT2_CUDA_TRY(cudaMemsetAsync(dw.Dm + mm, 0, sizeof(double) * mm, s));
  }
  if (a > 0) {
    const int a2 = a * a;
    // per-thread accumulator columns: at most 96 KB of shared memory per block
    const int nt = std::max(32, std::min(256, (int)(kActAdjSmem / (8L * a2)) / 32 * 32));
    const size_t smem = 8ull * a2 * nt;
    if (smem > (size_t)kActAdjSmem) return CASPT2_EINVAL;
    const long nblk = std::max<long>(1, std::min<long>(152L * 4, (mm + nt - 1) / nt));
    if (nblk * a2 > dw.partmax) return CASPT2_EINVAL;
    CASPT2_CUDA_TRY(cudaFuncSetAttribute(k_act_adj, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kActAdjSmem));
    ++launch_counter();
    k_act_adj<<<(unsigned)nblk, nt, smem, s>>>(w.dF, w.nF, C, a, n, rdm, dw.Dm, m, dw.part);
    ++launch_counter();
    k_act_finish<<<1, 256, 0, s>>>(dw.part, (int)nblk, a, d.c, nmo, NL, rdm.p[1], n, d2);
    CASPT2_CUDA_TRY(cudaGetLastError());
  }
  // ---- sources: d1 and the adjoint integral blocks
  ++launch_counter();
  k_wsrc<<<launch_blocks(tall), 256, 0, s>>>(dw.T, dw.Lam, R, P, n, m, tall, dw.U1);
  ++launch_counter();
  if (n <= 4) {
    const long total2 = w.vsize / ((long)n * n);
    k_src_adj_ml<4><<<launch_blocks(total2), 256, 0, s>>>(w.dV, w.nV, C, d, rdm, dw.U1, m, total2,
                                                         d1, G);
  } else {
    k_src_adj<<<launch_blocks(w.vsize), 256, 0, s>>>(w.dV, w.nV, C, d, rdm, dw.U1, m, w.vsize, d1,
                                                     G);
  }
  CASPT2_CUDA_TRY(cudaGetLastError());
  return CASPT2_OK;
}

namespace {
// out[fam][ext...][act...] = src[tuple][L][(fam, act..., N)] for one (L, N)
__global__ void k_gather_amp(const double* __restrict__ src, int nfam, long ntot, long A, int n,
                             int L, int N, double* __restrict__ out) {
  const long total = (long)nfam * ntot * A;
  const long m = (long)nfam * A * n;
  for (long o = blockIdx.x * (long)blockDim.x + threadIdx.x; o < total;
       o += (long)gridDim.x * blockDim.x) {
    const long act = o % A;
    const long t = (o / A) % ntot;
    const long fam = o / (A * ntot);
    out[o] = src[(t * n + L) * m + (fam * A + act) * n + N];
  }
}
}  // namespace

cudaError_t gather_amplitudes(const ClassWork& w, const Dims& d, const double* src, int L, int N,
                              double* out, cudaStream_t s) {
  const long total = (long)w.dc.nfam * all_tuples(w) * w.A;
  if (total == 0) return cudaSuccess;
  ++launch_counter();
  k_gather_amp<<<launch_blocks(total), 256, 0, s>>>(src, w.dc.nfam, all_tuples(w), w.A, d.n, L, N,
                                                    out);
  return cudaGetLastError();
}

}  // namespace caspt2
