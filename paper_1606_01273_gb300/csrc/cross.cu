// One-body couplings between excitation classes (Sec. II.B, II.D).
//
// E_xy with x and y in different orbital spaces (closed-active, active-virtual,
// closed-virtual and the transposes) maps a first-order function of class K' to the
// (closed holes, virtual particles) count of class K.  Its matrix elements
//   C^{xy}_{K K'} = <M~| E_bra(K)^dag E_xy E_ket(K') |N~>
// are generated in terms.cpp, grouped by their external pattern: every closed or virtual
// index is tied to exactly one other, so a group factorises into Kronecker deltas between
// the bra tuple, the ket tuple and the external f index (or indices), times an active
// factor.  The active factor of a group is formed once as a dense matrix
//   W[(fk, ket active, N)][(t, fb, bra active, M)]      (t: the active one of x, y)
// from the rotated RDMs, so that the coupling of a whole class pair is one GEMM over the
// ket (or bra) rows plus a gather over the external indices.
//
// Here the couplings give the off-diagonal blocks of the density
//   dbar2_xy = sum_L <Psi_lambda_L| E_xy |Psi1_L>     (Sec. II.D, the dbar(2) definition)
// from the amplitudes and lambda of every class over all index tuples.  With the f index
// tied to a bra slot (side 0):
//   Z[(kt, L)][(t, br)] = sum_kr T^{K'}[(kt, L)][kr] W[kr][(t, br)]
//   dbar2[e][t]        += sum_{bt: bt_f = e} sum_{L, br} lambda^K[(bt, L)][br] Z[(kt(bt), L)][(t, br)]
// and with it tied to a ket slot (side 1) the roles of the two classes swap:
//   Lt[(bt, L)][(t, kr)] = sum_br lambda^K[(bt, L)][br] W'[(t, kr)][br]
//   dbar2[e][t]        += sum_{bt, L, kr} T^{K'}[(kt(bt, e), L)][kr] Lt[(bt, L)][(t, kr)].
// Every sum runs in a fixed order (block partials finished in order), so the result is
// bitwise reproducible.
#include <algorithm>
#include <vector>

#include "class_ag.cuh"
#include "class_dev.cuh"
#include "cross.cuh"
#include "linalg.cuh"

namespace caspt2 {

namespace {

constexpr int kMaxT = 16;   // active orbitals (the densities need a <= 16)

// W of one group: layout 0 W[kr][t][br], layout 1 W[t][kr][br].
__global__ void k_cross_w(const CrossPlan* __restrict__ plans, int nplan, XCls B, XCls Kc, int a,
                          int n, int at, int layout, RdmPtrs g, double* __restrict__ W) {
  const long m = B.m, mp = Kc.m;
  const long total = mp * at * m;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    const long br = e % m;
    long kr;
    int t;
    if (layout == 0) {
      t = (int)((e / m) % at);
      kr = e / (m * at);
    } else {
      kr = (e / m) % mp;
      t = (int)(e / (m * mp));
    }
    int vals[32];
    const int M = (int)(br % n), N = (int)(kr % n);
    long ab = br / n, ak = kr / n;
    const int fb = (int)(ab / B.A), fk = (int)(ak / Kc.A);
    ab %= B.A;
    ak %= Kc.A;
    for (int k = B.nact - 1; k >= 0; --k) {
      vals[kRefBra + k] = (int)(ab % a);
      ab /= a;
    }
    for (int k = Kc.nact - 1; k >= 0; --k) {
      vals[kRefKet + k] = (int)(ak % a);
      ak /= a;
    }
    vals[kRefT] = t;
    double acc = 0.0;
    for (int q = 0; q < nplan; ++q) {
      const CrossPlan& P = plans[q];
      if (P.fb != fb || P.fk != fk) continue;
      bool ok = true;
      for (int r = 0; r < P.neq; ++r)
        if (vals[P.eq[r][0]] != vals[P.eq[r][1]]) ok = false;
      if (!ok) continue;
      acc += P.coeff * rdm_at(g.p, P.rank, n, a, M, N, vals, P.idx);
    }
    W[e] = acc;
  }
}

// Row-major tuple index of coordinates co over dims.
__device__ __forceinline__ long xtuple(const XCls& C, const int* co) {
  long t = 0;
  for (int k = 0; k < C.next; ++k) t = t * C.ext_dim[k] + co[k];
  return t;
}

// Partial sums of one group's dbar2 block.  Block (combo, chunk): combo fixes the values of
// the external f index positions (bra positions for side 0, ket positions for side 1); the
// block runs over its chunk of (free bra coordinates) x L x row and accumulates, per t,
//   Ab[(bt n + L) rb + t sbt + r] * Ak[(kt n + L) rk + t skt + r].
__global__ void __launch_bounds__(256)
k_cross_reduce(const double* __restrict__ Ab, long rb, long sbt, const double* __restrict__ Ak,
               long rk, long skt, long R, XCls B, XCls Kc, XGroupDev G, int n, int at, long nfree,
               long chunk, double* __restrict__ part) {
  __shared__ double red[32];
  const int combo = blockIdx.x;
  int fixv[2] = {0, 0};
  {
    const XCls& F = G.side == 0 ? B : Kc;
    int rem = combo;
    for (int k = G.nfe - 1; k >= 0; --k) {
      const int dk = F.ext_dim[G.fe_pos[k]];
      fixv[k] = rem % dk;
      rem /= dk;
    }
  }
  const long niter = nfree * n * R;
  const long it0 = (long)blockIdx.y * chunk, it1 = min(niter, it0 + chunk);
  double acc[kMaxT];
#pragma unroll
  for (int t = 0; t < kMaxT; ++t) acc[t] = 0.0;
  for (long it = it0 + threadIdx.x; it < it1; it += blockDim.x) {
    const long r = it % R;
    const long rest = it / R;
    const int L = (int)(rest % n);
    long fr = rest / n;
    int bt[4], kt[4];
    for (int k = B.next - 1; k >= 0; --k) {
      bool fixed = false;
      if (G.side == 0)
        for (int q = 0; q < G.nfe; ++q)
          if (G.fe_pos[q] == k) { bt[k] = fixv[q]; fixed = true; }
      if (!fixed) {
        bt[k] = (int)(fr % B.ext_dim[k]);
        fr /= B.ext_dim[k];
      }
    }
    for (int k = 0; k < Kc.next; ++k) {
      if (G.ket_src[k] >= 0) {
        kt[k] = bt[G.ket_src[k]];
      } else {
        kt[k] = 0;
        for (int q = 0; q < G.nfe; ++q)
          if (G.fe_pos[q] == k) kt[k] = fixv[q];
      }
    }
    const double* pb = Ab + (xtuple(B, bt) * n + L) * rb + r;
    const double* pk = Ak + (xtuple(Kc, kt) * n + L) * rk + r;
    if (sbt == 0) {
      const double vb = *pb;
#pragma unroll
      for (int t = 0; t < kMaxT; ++t)
        if (t < at) acc[t] = fma(vb, pk[t * skt], acc[t]);
    } else {
      const double vk = *pk;
#pragma unroll
      for (int t = 0; t < kMaxT; ++t)
        if (t < at) acc[t] = fma(pb[t * sbt], vk, acc[t]);
    }
  }
  for (int t = 0; t < at; ++t) {
    const double s = block_sum(acc[t], red);
    if (threadIdx.x == 0) part[((long)combo * gridDim.y + blockIdx.y) * at + t] = s;
  }
}

// dbar2[x][y] += sum over the chunks (in order) of each (combo, t).
__global__ void k_cross_finish(const double* __restrict__ part, int ncombo, int nchunk, int at,
                               XCls B, XCls Kc, XGroupDev G, int offx, int offy, int nmo,
                               double* __restrict__ d2) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= ncombo * at) return;
  const int combo = idx / at, t = idx % at;
  double s = 0.0;
  for (int q = 0; q < nchunk; ++q) s += part[((long)combo * nchunk + q) * at + t];
  const XCls& F = G.side == 0 ? B : Kc;
  int fixv[2] = {0, 0};
  int rem = combo;
  for (int k = G.nfe - 1; k >= 0; --k) {
    const int dk = F.ext_dim[G.fe_pos[k]];
    fixv[k] = rem % dk;
    rem /= dk;
  }
  int x = t, y = t;
  for (int k = 0; k < G.nfe; ++k) {
    if (G.fe_xy[k] == 0) x = fixv[k];
    else y = fixv[k];
  }
  d2[(long)(offx + x) * nmo + offy + y] += s;
}

// Class H over all tuples (i, j, a, b): T[(tuple, L)][N] and lambda, the coefficients of
// E_ai,bj |N~> in |Psi1_L> and |Psi_lambda_L> (unrestricted sums over i, j, a, b):
//   T_LN = 1/2 sum_nu W_Nnu W_Lnu u,   u = -K / D,   D = e_a + e_b - e_i - e_j + s_(nu, L)
//   lambda_LN = 1/2 sum_nu W_Nnu (r_L c_nu + 2 E_s r_L^2 W_Lnu / D) u,  c_nu = sum_L' W_L'nu r_L'
// (SS-SR: nu = L only, W = 1, s = E_s).
__global__ void k_h_tuple_amps(const double* __restrict__ K, const double* __restrict__ eps,
                               const double* __restrict__ W, const double* __restrict__ shifts,
                               const double* __restrict__ R, int P, int c, int v, int n,
                               int scheme, double shift, double* __restrict__ T,
                               double* __restrict__ Lam) {
  const long cv = (long)c * v;
  const long total = cv * cv;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    const int b = (int)(e % v);
    const int a = (int)((e / v) % v);
    const int j = (int)((e / ((long)v * v)) % c);
    const int i = (int)(e / ((long)v * v * c));
    const double Kv = K[((long)i * v + a) * cv + (long)j * v + b];
    const double D0 = eps[c + a] + eps[c + b] - eps[i] - eps[j];
    double* To = T + e * n * n;
    double* Lo = Lam + e * n * n;
    if (scheme == CASPT2_SSSR) {
      for (int L = 0; L < n; ++L) {
        const double D = D0 + shift;
        const double u = -Kv / D;
        const double rl = R[L * n + P];
        for (int N = 0; N < n; ++N) {
          To[L * n + N] = N == L ? 0.5 * u : 0.0;
          Lo[L * n + N] = N == L ? 0.5 * (rl * rl + 2.0 * shift * rl * rl / D) * u : 0.0;
        }
      }
      continue;
    }
    for (int L = 0; L < n; ++L) {
      const double rl = R[L * n + P];
      for (int N = 0; N < n; ++N) {
        double tv = 0.0, lv = 0.0;
        for (int nu = 0; nu < n; ++nu) {
          double cnu = 0.0;
          for (int Q = 0; Q < n; ++Q) cnu += W[Q * n + nu] * R[Q * n + P];
          const double D = D0 + shifts[nu * n + L];
          const double u = -Kv / D;
          tv += W[N * n + nu] * W[L * n + nu] * u;
          lv += W[N * n + nu] * (rl * cnu + 2.0 * shift * rl * rl * W[L * n + nu] / D) * u;
        }
        To[L * n + N] = 0.5 * tv;
        Lo[L * n + N] = 0.5 * lv;
      }
    }
  }
}

int space_offset(const Dims& d, int sp) { return sp == SP_C ? 0 : (sp == SP_A ? d.c : d.c + d.a); }

}  // namespace

XCls make_xcls(int cls, const Dims& d) {
  const XClassInfo I = xclass_info(cls);
  XCls C{};
  C.nfam = I.nfam;
  C.nact = I.nact;
  C.next = I.next;
  C.ntup = 1;
  for (int k = 0; k < I.next; ++k) {
    C.ext_dim[k] = I.ext_space[k] == SP_C ? d.c : d.v;
    C.ntup *= C.ext_dim[k];
  }
  C.A = 1;
  for (int k = 0; k < I.nact; ++k) C.A *= d.a;
  C.m = (int)(C.nfam * C.A * d.n);
  return C;
}

void cross_setup(CrossWork& xw, std::vector<CrossPlan>& all) {
  xw.groups.clear();
  all.clear();
  const int pairs[6][2] = {{SP_C, SP_A}, {SP_A, SP_C}, {SP_A, SP_V},
                           {SP_V, SP_A}, {SP_C, SP_V}, {SP_V, SP_C}};
  for (auto& p : pairs) {
    std::vector<CrossGroup> gs;
    build_cross_groups(p[0], p[1], gs);
    for (auto& g : gs) {
      CrossGroupHost h{};
      h.g = g;
      h.off = (int)all.size();
      h.nplan = (int)g.terms.size();
      for (const CrossPlan& P : g.terms) h.maxrank = std::max<int>(h.maxrank, P.rank);
      all.insert(all.end(), g.terms.begin(), g.terms.end());
      h.g.terms.clear();
      xw.groups.push_back(h);
    }
  }
}

long cross_work_size(const CrossWork& xw, const Dims& d, long* wmax, long* zmax, long* partmax) {
  *wmax = *zmax = *partmax = 1;
  const int n = d.n;
  for (const CrossGroupHost& h : xw.groups) {
    const XCls B = make_xcls(h.g.K, d), Kc = make_xcls(h.g.Kp, d);
    if (B.ntup == 0 || Kc.ntup == 0 || B.m == 0 || Kc.m == 0) continue;
    const int at = h.g.t_xy >= 0 ? d.a : 1;
    *wmax = std::max(*wmax, (long)Kc.m * at * B.m);
    const long z = h.g.side == 0 ? Kc.ntup * n * (long)at * B.m : B.ntup * n * (long)at * Kc.m;
    *zmax = std::max(*zmax, z);
    const XCls& F = h.g.side == 0 ? B : Kc;
    long ncombo = 1;
    for (int k = 0; k < h.g.nfe; ++k) ncombo *= F.ext_dim[h.g.fe_pos[k]];
    *partmax = std::max(*partmax, ncombo * kCrossChunks * at);
  }
  return *wmax + *zmax + *partmax;
}

int cross_dbar2(const CrossWork& xw, const Dims& d, RdmPtrs rdm, double* const* T,
                double* const* Lam, double* Wb, double* Zb, double* part, long wmax, long zmax,
                long partmax, double* d2, cudaStream_t s) {
  const int n = d.n, a = d.a, nmo = d.nmo();
  if (a > kMaxT) return CASPT2_EINVAL;
  for (const CrossGroupHost& h : xw.groups) {
    const CrossGroup& g = h.g;
    const XCls B = make_xcls(g.K, d), Kc = make_xcls(g.Kp, d);
    if (B.ntup == 0 || Kc.ntup == 0 || B.m == 0 || Kc.m == 0) continue;
    if (!T[g.Kp] || !Lam[g.K]) continue;             // a class left out of the densities
    if (h.maxrank > 0 && !rdm.p[h.maxrank]) return CASPT2_EINVAL;
    const int at = g.t_xy >= 0 ? a : 1;
    if (at == 0) continue;
    const long wsize = (long)Kc.m * at * B.m;
    if (wsize > wmax) return CASPT2_EINVAL;
    ++launch_counter();
    k_cross_w<<<launch_blocks(wsize), 256, 0, s>>>(xw.plans + h.off, h.nplan, B, Kc, a, n, at,
                                                   g.side, rdm, Wb);
    CASPT2_CUDA_TRY(cudaGetLastError());
    XGroupDev G{};
    G.side = g.side;
    G.nfe = g.nfe;
    for (int k = 0; k < 2; ++k) {
      G.fe_xy[k] = g.fe_xy[k];
      G.fe_pos[k] = g.fe_pos[k];
    }
    for (int k = 0; k < 4; ++k) G.ket_src[k] = g.ket_src[k];
    const XCls& F = g.side == 0 ? B : Kc;
    long ncombo = 1;
    for (int k = 0; k < g.nfe; ++k) ncombo *= F.ext_dim[g.fe_pos[k]];
    long nfree = 1;
    for (int k = 0; k < B.next; ++k) {
      bool fixed = false;
      if (g.side == 0)
        for (int q = 0; q < g.nfe; ++q) fixed = fixed || g.fe_pos[q] == k;
      if (!fixed) nfree *= B.ext_dim[k];
    }
    const double *Ab, *Ak;
    long rb, sbt, rk, skt, R;
    if (g.side == 0) {
      // Z[(kt, L)][(t, br)] = T^{K'} W
      const long rows = Kc.ntup * n, cols = (long)at * B.m;
      if (rows * cols > zmax || rows > INT32_MAX) return CASPT2_EINVAL;
      CASPT2_CUDA_TRY(dgemm((int)rows, (int)cols, Kc.m, 1.0, T[g.Kp], Kc.m, false, Wb, (int)cols,
                            false, 0.0, Zb, (int)cols, s));
      Ab = Lam[g.K]; rb = B.m; sbt = 0;
      Ak = Zb; rk = cols; skt = B.m;
      R = B.m;
    } else {
      // Lt[(bt, L)][(t, kr)] = lambda^K W'^T
      const long rows = B.ntup * n, cols = (long)at * Kc.m;
      if (rows * cols > zmax || rows > INT32_MAX) return CASPT2_EINVAL;
      CASPT2_CUDA_TRY(dgemm((int)rows, (int)cols, B.m, 1.0, Lam[g.K], B.m, false, Wb, B.m, true,
                            0.0, Zb, (int)cols, s));
      Ab = Zb; rb = cols; sbt = Kc.m;
      Ak = T[g.Kp]; rk = Kc.m; skt = 0;
      R = Kc.m;
    }
    const long niter = nfree * n * R;
    const int nchunk = (int)std::max<long>(1, std::min<long>(kCrossChunks, (niter + 2047) / 2048));
    const long chunk = (niter + nchunk - 1) / nchunk;
    if (ncombo * nchunk * at > partmax || ncombo > INT32_MAX) return CASPT2_EINVAL;
    ++launch_counter();
    k_cross_reduce<<<dim3((unsigned)ncombo, nchunk), 256, 0, s>>>(Ab, rb, sbt, Ak, rk, skt, R, B,
                                                                  Kc, G, n, at, nfree, chunk, part);
    CASPT2_CUDA_TRY(cudaGetLastError());
    const int nout = (int)(ncombo * at);
    ++launch_counter();
    k_cross_finish<<<(nout + 255) / 256, 256, 0, s>>>(part, (int)ncombo, nchunk, at, B, Kc, G,
                                                      space_offset(d, g.X), space_offset(d, g.Y),
                                                      nmo, d2);
    CASPT2_CUDA_TRY(cudaGetLastError());
  }
  return CASPT2_OK;
}

cudaError_t launch_h_tuple_amps(const double* K, const double* eps, const double* W,
                                const double* shifts, const double* R, int P, const Dims& d,
                                int scheme, double shift, double* T, double* Lam, cudaStream_t s) {
  const long total = (long)d.c * d.c * d.v * d.v;
  if (total == 0) return cudaSuccess;
  ++launch_counter();
  k_h_tuple_amps<<<launch_blocks(total), 256, 0, s>>>(K, eps, W, shifts, R, P, d.c, d.v, d.n,
                                                      scheme, shift, T, Lam);
  return cudaGetLastError();
}

}  // namespace caspt2
