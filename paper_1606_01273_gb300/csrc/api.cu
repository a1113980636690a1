// C ABI of the CASPT2 library: context lifetime, input staging and the solve
// pipeline.  Host code only orchestrates; every arithmetic step runs in the
// kernels of setup.cu and class_*.cu on the caller's stream.
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include <algorithm>
#include <cmath>
#include <map>

#include "class_ag.cuh"
#include "cross.cuh"
#include "class_dev.cuh"
#include "kernels.cuh"
#include "linalg.cuh"
#include "ozaki.cuh"

using namespace caspt2;

namespace {

constexpr int kNumStages = 4;  // setup, class H, classes A-G, H^eff
constexpr int kNumTimes = kNumStages + 12;  // + class-H kernel, tridiagonalisation ms/flops/launches,
                                            //   densities, tridiagonalisation bytes, FP64 GEMM
                                            //   ms/flops/launches, blocked-reduction panels
                                            //   ms/bytes/launches

}  // namespace

struct caspt2_ctx {
  Dims d{};
  caspt2_options opt{};
  int device = 0;
  bool have_inputs = false;
  bool have_rdm3 = false, have_rdm4 = false;
  bool solved = false;
  int last_status = CASPT2_ESTATE;   // of the last caspt2_solve (ESTATE before the first)
  unsigned warnings = 0;             // CASPT2_WARN_* of the last solve
  bool partial() const {             // a closed-orbital range narrower than all orbitals
    return opt.closed_begin > 0 || (opt.closed_end >= 0 && opt.closed_end < d.c);
  }
  double min_e0_gap = 0.0;           // smallest |E0_M - E0_N| of the last solve
  std::vector<void*> allocs;

  // inputs (device copies)
  double *f = nullptr, *B = nullptr, *rdm1 = nullptr, *rdm2 = nullptr, *rdm3 = nullptr,
         *rdm4 = nullptr;
  // setup work
  double *dact = nullptr, *gam = nullptr, *Y = nullptr, *g = nullptr, *bsum = nullptr,
         *bfro = nullptr, *ecore = nullptr, *fref = nullptr, *U = nullptr, *Etil = nullptr,
         *Ftil = nullptr, *E0 = nullptr, *rdm1r = nullptr, *rdm2r = nullptr, *eri = nullptr,
         *href = nullptr;
  // classes
  double *ecls = nullptr, *ncls = nullptr, *mindenom = nullptr;
  double *mom = nullptr, *lamNL = nullptr, *lamLV = nullptr;   // per class moments, lambda
  ClassHWork hw{};
  // classes A-G
  int kmax = 2;                       // highest RDM rank the enabled classes read
  ClassWork cw[7];
  bool cw_on[7] = {};
  SectorWork sw{};
  double *rdm3r = nullptr, *rdm4r = nullptr, *h = nullptr, *fact = nullptr, *eps = nullptr;
  double* hk = nullptr;               // precision form: core exchange block for h
  double *pack0 = nullptr, *pack1 = nullptr;
  std::map<int, double*> eri_blk;     // canonical space key -> (pq|rt) block
  EriBlocks eri_tab{};
  std::vector<PresumSpec> presum;     // pre-summed blocks of the solve's source plans
  std::vector<double*> presum_blk;
  PresumBlocks presum_tab{};
  long wmax = 0, m2max = 0, packmax = 0;
  // densities (allocated on the first caspt2_densities call)
  bool dens_alloc = false, dens_done = false;
  DensWork dw{};
  HDensWork hd{};
  std::map<int, double*> gblk;        // adjoint (pq|rt) blocks, keys of eri_blk
  EriBlocks g_tab{};
  double *dd1 = nullptr, *dd2 = nullptr, *dgdf = nullptr, *gtmp = nullptr;
  // precision form: split BF16 tensor-core GEMMs, class-H pair integrals kept for the densities
  OzWork oz{};
  double *hK = nullptr, *hKK = nullptr, *hpack = nullptr;
  // one-body couplings between classes: dbar2 off-diagonal blocks (opt.dens_offdiag)
  bool x_alloc = false;
  CrossWork xw{};
  double* xT[8] = {};
  double* xL[8] = {};
  double *xW = nullptr, *xZ = nullptr, *xpart = nullptr;
  long xwmax = 0, xzmax = 0, xpartmax = 0;
  // energy gradient (allocated on the first caspt2_gradient call)
  bool grad_alloc = false;
  GradWork gw{};
  double *gradf = nullptr, *gradB = nullptr;
  // canonical closed/virtual orbitals: the inputs were rotated by canonC (set_inputs with
  // an f whose closed or virtual block is not diagonal); outputs are rotated back
  bool canon = false;
  double *canonC = nullptr, *canon_t1 = nullptr, *canon_t2 = nullptr;
  long canon_chunk = 0;
  // orbital derivative (allocated on the first caspt2_orbital_derivative call)
  bool orb_alloc = false;
  double *orb_h = nullptr, *orb_gf = nullptr, *orb_y = nullptr;
  cudaEvent_t dev0 = nullptr, dev1 = nullptr;
  // results
  double *heff = nullptr, *ems = nullptr, *R = nullptr;
  int* status = nullptr;
  cudaEvent_t ev[kNumStages + 1] = {};

  // host copies of the last results
  std::vector<double> hU, hE0, hHref, hHeff, hEms, hR, hEcls, hNcls, hLamNL, hLamLV;
  double hEcore = 0.0, hMinDenom = 0.0;
  double times[kNumTimes] = {};
  long launches = 0;
  KernelTimer tri{};
  GemmTimer* gemm = nullptr;          // FP64 GEMM launches of a solve (device time, flops)

  template <class T>
  int alloc(T** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    void* q = nullptr;
    if (cudaMalloc(&q, count * sizeof(T)) != cudaSuccess) return CASPT2_ENOMEM;
    allocs.push_back(q);
    *p = static_cast<T*>(q);
    return CASPT2_OK;
  }
};

namespace caspt2 {

int check_block_diagonal_fock(const double* f, const Dims& d) {
  // the canonical case of classify_fock; rotated closed/virtual blocks are refused here
  const int st = classify_fock(f, d);
  return st == 1 ? CASPT2_EINVAL : st;
}

}  // namespace caspt2

extern "C" {

void caspt2_default_options(caspt2_options* o) {
  if (!o) return;
  o->xms = 1;
  o->scheme = CASPT2_MSMR;
  o->shift = 0.0;
  o->ovl_thresh = 1e-9;
  o->enuc = 0.0;
  o->target_state = 0;
  o->class_mask = caspt2_supported_classes();
  o->precision = CASPT2_FP64;
  o->slices = 7;
  o->degen_thresh = 1e-8;
  o->closed_begin = 0;
  o->closed_end = -1;
  o->dens_offdiag = 0;
}

unsigned caspt2_supported_classes(void) { return (1u << CASPT2_NCLASS) - 1u; }

const char* caspt2_strerror(int st) {
  switch (st) {
    case CASPT2_OK: return "ok";
    case CASPT2_EINVAL: return "invalid argument (sizes, options or pointers)";
    case CASPT2_ENOMEM: return "device allocation failed";
    case CASPT2_ENOTCONV: return "an eigensolver or iteration did not converge";
    case CASPT2_ENAN: return "NaN or Inf in inputs or results";
    case CASPT2_ETIMEOUT: return "a bounded device wait gave up";
    case CASPT2_ECUDA: return "CUDA runtime error";
    case CASPT2_ESTATE: return "call out of order";
    case CASPT2_ESCRATCH:
      return "problem exceeds the fixed 4 MiB device scratch of caspt2_classH_noalloc";
    case CASPT2_WINTRUDER: return "warning: a denominator is below 1e-3 Eh (intruder state)";
    case CASPT2_WDEGEN:
      return "warning: two XMS zeroth-order energies are degenerate (rotation not unique there)";
    default: return "unknown status";
  }
}

void caspt2_destroy(caspt2_ctx* ctx) {
  if (!ctx) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(ctx->device);
  for (void* p : ctx->allocs) cudaFree(p);
  for (auto& e : ctx->ev)
    if (e) cudaEventDestroy(e);
  if (ctx->hw.ev_gemm0) cudaEventDestroy(ctx->hw.ev_gemm0);
  if (ctx->hw.ev_gemm1) cudaEventDestroy(ctx->hw.ev_gemm1);
  if (ctx->tri.e0) cudaEventDestroy(ctx->tri.e0);
  if (ctx->dev0) cudaEventDestroy(ctx->dev0);
  oz_release(ctx->oz);
  if (ctx->gemm) {
    gemm_timer_release(*ctx->gemm);
    delete ctx->gemm;
  }
  if (ctx->dev1) cudaEventDestroy(ctx->dev1);
  if (ctx->tri.e1) cudaEventDestroy(ctx->tri.e1);
  for (cudaEvent_t e : ctx->tri.pev)
    if (e) cudaEventDestroy(e);
  cudaSetDevice(cur);
  delete ctx;
}

int caspt2_create(caspt2_ctx** out, const caspt2_dims* dims, const caspt2_options* opt) {
  if (!out || !dims) return CASPT2_EINVAL;
  *out = nullptr;
  const caspt2_dims& q = *dims;
  if (q.nclosed < 0 || q.nact < 0 || q.nvirt < 0 || q.naux <= 0 || q.nstate <= 0 ||
      q.nstate > kMaxStates)
    return CASPT2_EINVAL;
  caspt2_options o;
  caspt2_default_options(&o);
  if (opt) o = *opt;
  if (o.scheme != CASPT2_MSMR && o.scheme != CASPT2_SSSR) return CASPT2_EINVAL;
  if (!(o.shift >= 0.0) || !(o.ovl_thresh > 0.0)) return CASPT2_EINVAL;
  if (o.class_mask & ~caspt2_supported_classes()) return CASPT2_EINVAL;
  if (o.target_state >= q.nstate) return CASPT2_EINVAL;
  if (o.precision != CASPT2_FP64 && o.precision != CASPT2_BF16X) return CASPT2_EINVAL;
  if (o.precision == CASPT2_BF16X && (o.slices < 1 || o.slices > 7)) return CASPT2_EINVAL;
  if (!(o.degen_thresh >= 0.0)) return CASPT2_EINVAL;
  if (o.closed_begin < 0 || o.closed_begin > q.nclosed ||
      (o.closed_end >= 0 && (o.closed_end < o.closed_begin || o.closed_end > q.nclosed)))
    return CASPT2_EINVAL;

  caspt2_ctx* c = new (std::nothrow) caspt2_ctx();
  if (!c) return CASPT2_ENOMEM;
  c->d = Dims{q.nclosed, q.nact, q.nvirt, q.naux, q.nstate};
  c->opt = o;
  cudaGetDevice(&c->device);
  const Dims& d = c->d;
  const size_t nmo = d.nmo(), n = d.n, a = d.a, X = d.X;
  const size_t a2 = a * a, a4 = a2 * a2;
  int st = CASPT2_OK;
#define ALLOC(ptr, cnt) \
  if (st == CASPT2_OK) st = c->alloc(&(ptr), (cnt))
  ALLOC(c->f, nmo * nmo);
  ALLOC(c->B, X * nmo * nmo);
  ALLOC(c->rdm1, n * n * a2);
  ALLOC(c->rdm2, n * n * a4);
  ALLOC(c->dact, a2);
  ALLOC(c->gam, X);
  ALLOC(c->Y, X * nmo * (a ? a : 1));
  ALLOC(c->g, nmo * nmo);
  ALLOC(c->bsum, X);
  ALLOC(c->bfro, X);
  ALLOC(c->ecore, 1);
  ALLOC(c->fref, n * n);
  ALLOC(c->U, n * n);
  ALLOC(c->Etil, n);
  ALLOC(c->Ftil, n * n);
  ALLOC(c->E0, n);
  ALLOC(c->rdm1r, n * n * a2);
  ALLOC(c->rdm2r, n * n * a4);
  ALLOC(c->eri, a4);
  ALLOC(c->href, n * n);
  ALLOC(c->ecls, (size_t)CASPT2_NCLASS * n * n);
  ALLOC(c->ncls, (size_t)CASPT2_NCLASS * n);
  ALLOC(c->mindenom, 1);
  ALLOC(c->heff, n * n);
  ALLOC(c->ems, n);
  ALLOC(c->R, n * n);
  ALLOC(c->status, 1);
  // class H work
  c->hw.nblocks = classH_blocks(d);
  const size_t nshift = (size_t)classH_nshift(d, o.scheme);
  ALLOC(c->hw.Bp, (size_t)d.c * X * d.v);
  ALLOC(c->hw.eps, nmo);
  ALLOC(c->hw.W, n * n);
  ALLOC(c->hw.omega, n);
  ALLOC(c->hw.shifts, nshift);
  ALLOC(c->hw.partial, (size_t)c->hw.nblocks * (3 * nshift + 1));
  ALLOC(c->hw.sums, 3 * nshift + 1);
  ALLOC(c->mom, (size_t)CASPT2_NCLASS * (n * n * n + n * n + n));
  if (o.precision == CASPT2_BF16X) {
    c->oz.on = true;
    c->oz.S = o.slices;
    if ((o.class_mask >> CASPT2_CLASS_H & 1u) && d.c > 0 && d.v > 0) {
      const size_t cv = (size_t)d.c * d.v;
      ALLOC(c->hK, cv * cv);
      ALLOC(c->hKK, cv * cv);
      ALLOC(c->hpack, (size_t)d.X * cv);
    }
  }
  ALLOC(c->lamNL, (size_t)CASPT2_NCLASS * n);
  ALLOC(c->lamLV, (size_t)CASPT2_NCLASS * n * n);
  // classes A-G: plans, class matrices, sources, sector work space, integral blocks
  {
    long m2max = 0, wmax = 0, pmax = 0, vmax = 0, srcx_max = 0, srcg_max = 0;
    long packmax = 0;
    std::map<int, long> eri_need;
    for (int k = 0; k < 7 && st == CASPT2_OK; ++k) {
      if (!(o.class_mask >> k & 1u)) continue;
      ClassWork& w = c->cw[k];
      class_setup(k, d, w);
      if (w.vsize == 0 || a == 0) continue;
      c->cw_on[k] = true;
      std::vector<ActPlan> S, F;
      std::vector<SrcPlan> V;
      build_act_plans(k, false, S);
      build_act_plans(k, true, F);
      build_src_plans(k, V);
      for (auto& t : S) c->kmax = std::max<int>(c->kmax, t.rank);
      for (auto& t : F) c->kmax = std::max<int>(c->kmax, t.rank);
      for (auto& t : V) {
        c->kmax = std::max<int>(c->kmax, t.rank);
        if (t.kind == 1) {
          const int dims3[3] = {d.c, d.a, d.v};
          int key = ((t.ispace[0] * 3 + t.ispace[1]) * 3 + t.ispace[2]) * 3 + t.ispace[3];
          eri_need[key] = (long)dims3[t.ispace[0]] * dims3[t.ispace[1]] * dims3[t.ispace[2]] *
                          dims3[t.ispace[3]];
          packmax = std::max(packmax, (long)X * dims3[t.ispace[0]] * dims3[t.ispace[1]]);
          packmax = std::max(packmax, (long)X * dims3[t.ispace[2]] * dims3[t.ispace[3]]);
        }
      }
      {
        std::vector<SrcPlan> pre;
        presum_src_plans(V, pre, c->presum);
        split_src_plans(k, pre, w.hVs, w.hG);
      }
      if (c->presum.size() > (size_t)kMaxPresum) st = CASPT2_EINVAL;
      ALLOC(w.dS, S.size());
      ALLOC(w.dF, F.size());
      ALLOC(w.dV, V.size());
      ALLOC(w.dVs, w.hVs.size());
      {
        size_t nx = 0;
        const long ncol = w.A * n * n;
        for (const SrcGemmGroup& G : w.hG) {
          nx += G.x.size();
          long K = 1;
          for (int q = 0; q < G.g.ns; ++q) K *= a;
          srcg_max = std::max(srcg_max, K * ncol);
          srcx_max = std::max(srcx_max, K * all_tuples(w));
        }
        if (nx > 0) ALLOC(w.dX, nx);
      }
      if (st == CASPT2_OK && class_upload_plans(w, S, F, V) != cudaSuccess) st = CASPT2_ECUDA;
      ALLOC(w.Sact, 2 * (size_t)w.m * w.m);
      ALLOC(w.Fact, 2 * (size_t)w.m * w.m);
      vmax = std::max(vmax, w.vsize);   // the sources live only during the class's solve
      // sector bases kept for the densities
      class_keep_layout(w, d, o.scheme);
      for (SectorKeep& K : w.keep) {
        if (K.ntup == 0) continue;
        ALLOC(K.Y, (size_t)K.msec * K.msec);
        ALLOC(K.omega, (size_t)K.msec);
        ALLOC(K.Vt, (size_t)K.msec * K.ntup * n);
      }
      m2max = std::max(m2max, (long)w.m * w.m);
      long ps = 0;
      wmax = std::max(wmax, class_sector_wsize(w, d, o.scheme, &ps));
      pmax = std::max(pmax, ps);
    }
    c->wmax = wmax;
    c->m2max = m2max;
    c->packmax = packmax;
    if (vmax > 0) {
      double* vb = nullptr;
      ALLOC(vb, (size_t)vmax);
      for (int k = 0; k < 7; ++k)
        if (c->cw_on[k]) c->cw[k].V = vb;
    }
    if (m2max > 0) {
      SectorWork& q = c->sw;
      const long mx = (long)std::sqrt((double)m2max) + 1;
      ALLOC(q.Ssec, m2max); ALLOC(q.Fsec, m2max); ALLOC(q.s, mx); ALLOC(q.Qs, m2max);
      ALLOC(q.X, m2max); ALLOC(q.FX, m2max); ALLOC(q.Ft, m2max);
      ALLOC(q.Qf, m2max); ALLOC(q.jac, sym_eig_work((int)mx));
      // the sector pass works in tuple chunks: W and the moment partials are capped
      const long pcol = (long)n * n * (n + 2);
      q.wcap = std::max<long>(std::min(wmax, kSectorWCap), mx * (long)n);
      q.pcap = std::max<long>(std::min(pmax, kSectorPartCap), pcol);
      q.nb2 = kColsumBlocks;
      // part2 also holds the per-eigenvector denominator minima and the refinement list
      q.p2size = std::max<long>(q.nb2 * pcol, mx + 1);
      ALLOC(q.W, q.wcap); ALLOC(q.part, q.pcap); ALLOC(q.part2, q.p2size);
      // source GEMM groups: X in row chunks of at most 2^26 doubles
      q.srcXcap = std::max<long>(1, std::min<long>(srcx_max, 1L << 26));
      q.srcGcap = std::max<long>(1, srcg_max);
      ALLOC(q.srcX, q.srcXcap); ALLOC(q.srcG, q.srcGcap);
      ALLOC(c->h, nmo * nmo);
      if (o.precision == CASPT2_BF16X) ALLOC(c->hk, nmo * nmo);
      ALLOC(c->fact, a2);
      ALLOC(c->eps, nmo);
      if (packmax > 0) {
        ALLOC(c->pack0, packmax);
        ALLOC(c->pack1, packmax);
      }
      for (auto& kv : eri_need) {
        double* p = nullptr;
        ALLOC(p, (size_t)std::max<long>(kv.second, 1));
        c->eri_blk[kv.first] = p;
        c->eri_tab.p[kv.first] = p;
      }
      for (size_t k = 0; k < c->presum.size() && st == CASPT2_OK; ++k) {
        double* p = nullptr;
        ALLOC(p, (size_t)std::max<long>(presum_size(d, c->presum[k]), 1));
        c->presum_blk.push_back(p);
        c->presum_tab.p[k] = p;
      }
      if (c->kmax >= 3) {
        ALLOC(c->rdm3, n * n * a2 * a2 * a2);
        ALLOC(c->rdm3r, n * n * a2 * a2 * a2);
      }
      if (c->kmax >= 4) {
        ALLOC(c->rdm4, n * n * a4 * a4);
        ALLOC(c->rdm4r, n * n * a4 * a4);
      }
    }
  }
#undef ALLOC
  for (auto& e : c->ev)
    if (st == CASPT2_OK && cudaEventCreate(&e) != cudaSuccess) st = CASPT2_ECUDA;
  if (st == CASPT2_OK && (cudaEventCreate(&c->hw.ev_gemm0) != cudaSuccess ||
                          cudaEventCreate(&c->hw.ev_gemm1) != cudaSuccess ||
                          cudaEventCreate(&c->tri.e0) != cudaSuccess ||
                          cudaEventCreate(&c->tri.e1) != cudaSuccess ||
                          cudaEventCreate(&c->dev0) != cudaSuccess ||
                          cudaEventCreate(&c->dev1) != cudaSuccess))
    st = CASPT2_ECUDA;
  if (st != CASPT2_OK) {
    caspt2_destroy(c);
    return st;
  }
  c->hU.assign(n * n, 0.0);
  c->hE0.assign(n, 0.0);
  c->hHref.assign(n * n, 0.0);
  c->hHeff.assign(n * n, 0.0);
  c->hEms.assign(n, 0.0);
  c->hR.assign(n * n, 0.0);
  c->hEcls.assign((size_t)CASPT2_NCLASS * n * n, 0.0);
  c->hNcls.assign((size_t)CASPT2_NCLASS * n, 0.0);
  c->hLamNL.assign((size_t)CASPT2_NCLASS * n, 0.0);
  c->hLamLV.assign((size_t)CASPT2_NCLASS * n * n, 0.0);
  *out = c;
  return CASPT2_OK;
}

int caspt2_set_inputs(caspt2_ctx* c, int mem, const double* fock, const double* dfB,
                      const double* rdm1, const double* rdm2, const double* rdm3,
                      const double* rdm4) {
  if (!c || !fock || !dfB || !rdm1 || !rdm2) return CASPT2_EINVAL;
  if (mem != CASPT2_MEM_HOST && mem != CASPT2_MEM_DEVICE) return CASPT2_EINVAL;
  const Dims& d = c->d;
  const size_t nmo = d.nmo(), n = d.n, a2 = (size_t)d.a * d.a;
  const cudaMemcpyKind k = mem == CASPT2_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  CASPT2_CUDA_TRY(cudaSetDevice(c->device));
  c->have_inputs = false;
  c->solved = false;
  c->dens_done = false;
  c->canon = false;
  int fclass = 0;
  {
    // the classes decouple only without closed-active, active-virtual and closed-virtual
    // coupling: refuse any other f; rotated closed/virtual blocks are canonicalised below
    std::vector<double> hf(nmo * nmo);
    CASPT2_CUDA_TRY(cudaMemcpy(hf.data(), fock, sizeof(double) * nmo * nmo,
                               mem == CASPT2_MEM_HOST ? cudaMemcpyHostToHost
                                                      : cudaMemcpyDeviceToHost));
    fclass = classify_fock(hf.data(), d);
    if (fclass < 0) return fclass;
  }
  CASPT2_CUDA_TRY(cudaMemcpy(c->f, fock, sizeof(double) * nmo * nmo, k));
  CASPT2_CUDA_TRY(cudaMemcpy(c->B, dfB, sizeof(double) * d.X * nmo * nmo, k));
  if (fclass == 1) {
    if (!c->canonC) {
      const int st = c->alloc(&c->canonC, nmo * nmo);
      if (st != CASPT2_OK) return st;
    }
    const int st = canonicalize_inputs(c->f, c->B, d, c->canonC, cudaStreamPerThread);
    if (st != CASPT2_OK) return st;
    c->canon = true;
  }
  CASPT2_CUDA_TRY(cudaMemcpy(c->rdm1, rdm1, sizeof(double) * n * n * a2, k));
  CASPT2_CUDA_TRY(cudaMemcpy(c->rdm2, rdm2, sizeof(double) * n * n * a2 * a2, k));
  if ((c->kmax >= 3 && !rdm3) || (c->kmax >= 4 && !rdm4)) return CASPT2_EINVAL;
  if (c->kmax >= 3)
    CASPT2_CUDA_TRY(cudaMemcpy(c->rdm3, rdm3, sizeof(double) * n * n * a2 * a2 * a2, k));
  if (c->kmax >= 4)
    CASPT2_CUDA_TRY(cudaMemcpy(c->rdm4, rdm4, sizeof(double) * n * n * a2 * a2 * a2 * a2, k));
  c->have_rdm3 = rdm3 != nullptr;
  c->have_rdm4 = rdm4 != nullptr;
  c->have_inputs = true;
  c->solved = false;
  return CASPT2_OK;
}

}  // extern "C"

namespace {
int solve_impl(caspt2_ctx* c, void* stream);
}  // namespace

extern "C" {

int caspt2_solve(caspt2_ctx* c, void* stream) {
  if (!c) return CASPT2_EINVAL;
  c->warnings = 0;
  c->min_e0_gap = 0.0;
  const int st = solve_impl(c, stream);
  c->last_status = st;
  return st;
}

int caspt2_get_status(caspt2_ctx* c, caspt2_report* out) {
  if (!c || !out) return CASPT2_EINVAL;
  std::memset(out, 0, sizeof(*out));
  out->last_status = c->last_status;
  out->solved = c->solved ? 1 : 0;
  out->densities_done = c->dens_done ? 1 : 0;
  out->min_denominator = c->solved ? c->hMinDenom : 0.0;
  out->kernel_launches = c->launches;
  const int k = kNumTimes < CASPT2_REPORT_TIMES ? kNumTimes : CASPT2_REPORT_TIMES;
  for (int i = 0; i < k; ++i) out->times_ms[i] = c->times[i];
  out->warnings = c->solved ? c->warnings : 0u;
  out->min_e0_gap = c->solved ? c->min_e0_gap : 0.0;
  return CASPT2_OK;
}

}  // extern "C"

namespace {

int solve_impl(caspt2_ctx* c, void* stream) {
  if (!c) return CASPT2_EINVAL;
  if (!c->have_inputs) return CASPT2_ESTATE;
  CASPT2_CUDA_TRY(cudaSetDevice(c->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const Dims& d = c->d;
  const caspt2_options& o = c->opt;
  const int n = d.n;
  const long a2 = (long)d.a * d.a;
  const double big = 1e300;
  const long launches0 = launch_counter();
  c->tri.ms = c->tri.flops = c->tri.bytes = 0.0;
  c->tri.launches = 0;
  c->tri.pms = c->tri.pbytes = 0.0;
  c->tri.plaunches = 0;
  if (!c->gemm) {
    c->gemm = new (std::nothrow) GemmTimer();
    if (c->gemm && gemm_timer_init(*c->gemm) != cudaSuccess) {
      gemm_timer_release(*c->gemm);
      delete c->gemm;
      c->gemm = nullptr;
    }
  }
  if (c->gemm) c->gemm->used = 0;
  struct TimerScope {
    explicit TimerScope(GemmTimer* t) { set_gemm_timer(t); }
    ~TimerScope() { set_gemm_timer(nullptr); }
  } timer_scope(c->gemm);
  CASPT2_CUDA_TRY(cudaMemsetAsync(c->status, 0, sizeof(int), s));
  CASPT2_CUDA_TRY(cudaMemcpyAsync(c->mindenom, &big, sizeof(double), cudaMemcpyHostToDevice, s));
  CASPT2_CUDA_TRY(cudaMemsetAsync(c->ecls, 0, sizeof(double) * CASPT2_NCLASS * n * n, s));
  CASPT2_CUDA_TRY(cudaMemsetAsync(c->ncls, 0, sizeof(double) * CASPT2_NCLASS * n, s));
  const long msz = (long)n * n * n + n * n + n;
  CASPT2_CUDA_TRY(cudaMemsetAsync(c->mom, 0, sizeof(double) * CASPT2_NCLASS * msz, s));
  CASPT2_CUDA_TRY(cudaMemsetAsync(c->lamNL, 0, sizeof(double) * CASPT2_NCLASS * n, s));
  CASPT2_CUDA_TRY(cudaMemsetAsync(c->lamLV, 0, sizeof(double) * CASPT2_NCLASS * n * n, s));

  // ---- stage 0: setup (Sec. II.A, II.B)
  CASPT2_CUDA_TRY(cudaEventRecord(c->ev[0], s));
  CASPT2_CUDA_TRY(launch_dsa(c->rdm1, d, c->dact, s));
  CASPT2_CUDA_TRY(launch_gmat(c->B, c->dact, d, c->gam, c->Y, c->g, s));
  CASPT2_CUDA_TRY(launch_ecore(c->f, c->g, c->B, d, c->bsum, c->bfro, c->ecore, s));
  CASPT2_CUDA_TRY(launch_fref(c->f, c->rdm1, d, c->fref, s));
  CASPT2_CUDA_TRY(launch_sym_eig(c->fref, n, c->U, c->Etil, o.xms ? 0 : 1, c->status, s));
  CASPT2_CUDA_TRY(launch_congruence(c->fref, c->U, n, c->Ftil, s));
  CASPT2_CUDA_TRY(launch_diag(c->Ftil, n, c->E0, s));
  CASPT2_CUDA_TRY(launch_rotate_rdm(c->rdm1, c->U, n, a2, c->rdm1r, s));
  CASPT2_CUDA_TRY(launch_rotate_rdm(c->rdm2, c->U, n, a2 * a2, c->rdm2r, s));
  CASPT2_CUDA_TRY(launch_eri_act(c->B, d, c->eri, s));
  CASPT2_CUDA_TRY(launch_href(c->f, c->g, c->rdm1r, c->rdm2r, c->eri, c->ecore, o.enuc, d,
                              c->href, s));
  CASPT2_CUDA_TRY(cudaEventRecord(c->ev[1], s));

  // ---- stage 1: class H (direct)
  if ((o.class_mask >> CASPT2_CLASS_H & 1u) && c->oz.on) {
    CASPT2_CUDA_TRY(launch_classH_split(c->f, c->B, c->Ftil, c->E0, o.shift, o.scheme, d, c->hw,
                                        c->status, c->ecls + (long)CASPT2_CLASS_H * n * n,
                                        c->ncls + (long)CASPT2_CLASS_H * n,
                                        c->mom + (long)CASPT2_CLASS_H * msz, c->mindenom, c->oz,
                                        c->hpack, c->hK, c->hKK, s, o.closed_begin,
                                        o.closed_end));
  } else if (o.class_mask >> CASPT2_CLASS_H & 1u) {
    CASPT2_CUDA_TRY(launch_classH(c->f, c->B, c->Ftil, c->E0, o.shift, o.scheme, d, c->hw,
                                  c->status, c->ecls + (long)CASPT2_CLASS_H * n * n,
                                  c->ncls + (long)CASPT2_CLASS_H * n,
                                  c->mom + (long)CASPT2_CLASS_H * msz, c->mindenom, s,
                                  o.closed_begin, o.closed_end));
  }
  CASPT2_CUDA_TRY(cudaEventRecord(c->ev[2], s));
  // ---- stage 2: classes A-G
  {
    bool any = false;
    for (int k = 0; k < 7; ++k) any = any || c->cw_on[k];
    if (any) {
      CASPT2_CUDA_TRY(launch_hcore(c->f, c->g, c->B, c->bsum, d, c->h, s, &c->oz, c->hk));
      CASPT2_CUDA_TRY(launch_active_block(c->f, d, c->fact, s));
      CASPT2_CUDA_TRY(launch_eps_cv(c->f, d, c->eps, s));
      if (c->kmax >= 3)
        CASPT2_CUDA_TRY(launch_rotate_rdm(c->rdm3, c->U, n, a2 * a2 * a2, c->rdm3r, s));
      if (c->kmax >= 4)
        CASPT2_CUDA_TRY(launch_rotate_rdm(c->rdm4, c->U, n, a2 * a2 * a2 * a2, c->rdm4r, s));
      for (auto& kv : c->eri_blk) {
        int sp4[4] = {kv.first / 27, (kv.first / 9) % 3, (kv.first / 3) % 3, kv.first % 3};
        CASPT2_CUDA_TRY(eri_block(c->B, d, sp4, c->pack0, c->pack1, kv.second, s, &c->oz));
      }
      for (size_t k = 0; k < c->presum.size(); ++k) {
        const PresumSpec& sp = c->presum[k];
        const int key = ((sp.space[0] * 3 + sp.space[1]) * 3 + sp.space[2]) * 3 + sp.space[3];
        CASPT2_CUDA_TRY(presum_block(d, sp, c->eri_blk.at(key), c->presum_blk[k], s));
      }
      RdmPtrs g{{nullptr, c->rdm1r, c->rdm2r, c->rdm3r, c->rdm4r}};
      for (int k = 0; k < 7; ++k) {
        if (!c->cw_on[k]) continue;
        // partial solves: classes A-F belong to the partition that starts at closed 0
        if (k != CASPT2_CLASS_G && o.closed_begin > 0) continue;
        int st = class_solve(c->cw[k], c->sw, d, o.scheme, o.shift, o.ovl_thresh, g, c->fact, c->h,
                             c->eri_tab, c->presum_tab, c->E0, c->eps, c->mom + (long)k * msz,
                             c->mindenom, s, &c->tri, &c->oz, o.closed_begin, o.closed_end);
        if (st != CASPT2_OK) return st;
        CASPT2_CUDA_TRY(launch_moments_to_e(c->mom + (long)k * msz, n, c->ecls + (long)k * n * n,
                                            c->ncls + (long)k * n, s));
      }
    }
  }
  CASPT2_CUDA_TRY(cudaEventRecord(c->ev[3], s));
  // ---- stage 3: effective Hamiltonian and its eigenpairs (Sec. II.B)
  CASPT2_CUDA_TRY(launch_heff(c->href, c->ecls, c->ncls, o.class_mask, o.shift, n, c->heff, s));
  CASPT2_CUDA_TRY(launch_sym_eig(c->heff, n, c->R, c->ems, 0, c->status, s));
  // lambda of the target state from the class moments (Eq. lambdaeq)
  if (o.target_state >= 0) {
    for (int k = 0; k < CASPT2_NCLASS; ++k) {
      if (!(o.class_mask >> k & 1u)) continue;
      CASPT2_CUDA_TRY(launch_lambda(c->mom + (long)k * msz, c->R, n, o.target_state, o.shift,
                                    c->lamNL + (long)k * n, c->lamLV + (long)k * n * n, s));
    }
  }
  CASPT2_CUDA_TRY(cudaEventRecord(c->ev[4], s));

  // results back to the host copies
  int hst = 0;
  CASPT2_CUDA_TRY(cudaMemcpyAsync(c->hU.data(), c->U, sizeof(double) * n * n, cudaMemcpyDeviceToHost, s));
  CASPT2_CUDA_TRY(cudaMemcpyAsync(c->hE0.data(), c->E0, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
  CASPT2_CUDA_TRY(cudaMemcpyAsync(c->hHref.data(), c->href, sizeof(double) * n * n, cudaMemcpyDeviceToHost, s));
  CASPT2_CUDA_TRY(cudaMemcpyAsync(c->hHeff.data(), c->heff, sizeof(double) * n * n, cudaMemcpyDeviceToHost, s));
  CASPT2_CUDA_TRY(cudaMemcpyAsync(c->hEms.data(), c->ems, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
  CASPT2_CUDA_TRY(cudaMemcpyAsync(c->hR.data(), c->R, sizeof(double) * n * n, cudaMemcpyDeviceToHost, s));
  CASPT2_CUDA_TRY(cudaMemcpyAsync(c->hEcls.data(), c->ecls, sizeof(double) * CASPT2_NCLASS * n * n, cudaMemcpyDeviceToHost, s));
  CASPT2_CUDA_TRY(cudaMemcpyAsync(c->hNcls.data(), c->ncls, sizeof(double) * CASPT2_NCLASS * n, cudaMemcpyDeviceToHost, s));
  CASPT2_CUDA_TRY(cudaMemcpyAsync(c->hLamNL.data(), c->lamNL, sizeof(double) * CASPT2_NCLASS * n, cudaMemcpyDeviceToHost, s));
  CASPT2_CUDA_TRY(cudaMemcpyAsync(c->hLamLV.data(), c->lamLV, sizeof(double) * CASPT2_NCLASS * n * n, cudaMemcpyDeviceToHost, s));
  CASPT2_CUDA_TRY(cudaMemcpyAsync(&c->hEcore, c->ecore, sizeof(double), cudaMemcpyDeviceToHost, s));
  CASPT2_CUDA_TRY(cudaMemcpyAsync(&c->hMinDenom, c->mindenom, sizeof(double), cudaMemcpyDeviceToHost, s));
  CASPT2_CUDA_TRY(cudaMemcpyAsync(&hst, c->status, sizeof(int), cudaMemcpyDeviceToHost, s));
  int ozerr = 0;
  if (c->oz.err)
    CASPT2_CUDA_TRY(cudaMemcpyAsync(&ozerr, c->oz.err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CASPT2_CUDA_TRY(cudaStreamSynchronize(s));
  if (ozerr != 0) return CASPT2_ETIMEOUT;
  for (int k = 0; k < kNumStages; ++k) {
    float ms = 0.f;
    CASPT2_CUDA_TRY(cudaEventElapsedTime(&ms, c->ev[k], c->ev[k + 1]));
    c->times[k] = ms;
  }
  c->times[kNumStages] = 0.0;
  if ((o.class_mask >> CASPT2_CLASS_H & 1u) && d.c > 0 && d.v > 0) {
    float ms = 0.f;
    CASPT2_CUDA_TRY(cudaEventElapsedTime(&ms, c->hw.ev_gemm0, c->hw.ev_gemm1));
    c->times[kNumStages] = ms;
  }
  c->times[kNumStages + 1] = c->tri.ms;
  c->times[kNumStages + 2] = c->tri.flops;
  c->times[kNumStages + 3] = (double)c->tri.launches;
  c->times[kNumStages + 5] = c->tri.bytes;
  c->times[kNumStages + 4] = 0.0;
  c->times[kNumStages + 6] = c->times[kNumStages + 7] = c->times[kNumStages + 8] = 0.0;
  if (c->gemm) {
    double gms = 0.0, gfl = 0.0;
    long gn = 0;
    CASPT2_CUDA_TRY(gemm_timer_collect(*c->gemm, &gms, &gfl, &gn));
    c->times[kNumStages + 6] = gms;
    c->times[kNumStages + 7] = gfl;
    c->times[kNumStages + 8] = (double)gn;
  }
  c->times[kNumStages + 9] = c->tri.pms;
  c->times[kNumStages + 10] = c->tri.pbytes;
  c->times[kNumStages + 11] = (double)c->tri.plaunches;
  c->launches = launch_counter() - launches0;
  c->solved = true;
  c->dens_done = false;
  if (hst != 0) return hst;
  for (double x : c->hEms)
    if (!(x == x) || x > 1e300 || x < -1e300) return CASPT2_ENAN;
  // warnings: intruder denominators; XMS zeroth-order energies that are degenerate
  // (the rotation inside such a pair is arbitrary; energies do not depend on it)
  double gap = 0.0;
  bool first = true;
  for (int M = 0; M < n; ++M)
    for (int N = M + 1; N < n; ++N) {
      const double g = std::fabs(c->hE0[M] - c->hE0[N]);
      gap = first ? g : std::min(gap, g);
      first = false;
    }
  c->min_e0_gap = gap;
  if (c->hMinDenom < 1e-3) c->warnings |= CASPT2_WARN_INTRUDER;
  if (o.xms && n > 1 && gap < o.degen_thresh) c->warnings |= CASPT2_WARN_DEGEN;
  if (c->warnings & CASPT2_WARN_INTRUDER) return CASPT2_WINTRUDER;
  if (c->warnings & CASPT2_WARN_DEGEN) return CASPT2_WDEGEN;
  return CASPT2_OK;
}

}  // namespace

extern "C" {

int caspt2_get_energies(caspt2_ctx* c, double* U, double* E0, double* Href, double* Heff,
                        double* Ems, double* R) {
  if (!c) return CASPT2_EINVAL;
  if (!c->solved) return CASPT2_ESTATE;
  const size_t n = c->d.n;
  if (U) std::memcpy(U, c->hU.data(), sizeof(double) * n * n);
  if (E0) std::memcpy(E0, c->hE0.data(), sizeof(double) * n);
  if (Href) std::memcpy(Href, c->hHref.data(), sizeof(double) * n * n);
  if (Heff) std::memcpy(Heff, c->hHeff.data(), sizeof(double) * n * n);
  if (Ems) std::memcpy(Ems, c->hEms.data(), sizeof(double) * n);
  if (R) std::memcpy(R, c->hR.data(), sizeof(double) * n * n);
  return CASPT2_OK;
}

int caspt2_get_class_energy(caspt2_ctx* c, int cls, double* e, double* norm) {
  if (!c || cls < 0 || cls >= CASPT2_NCLASS) return CASPT2_EINVAL;
  if (!(c->opt.class_mask >> cls & 1u)) return CASPT2_EINVAL;
  if (!c->solved) return CASPT2_ESTATE;
  const size_t n = c->d.n;
  if (e) std::memcpy(e, c->hEcls.data() + cls * n * n, sizeof(double) * n * n);
  if (norm) std::memcpy(norm, c->hNcls.data() + cls * n, sizeof(double) * n);
  return CASPT2_OK;
}

int caspt2_get_class_lambda(caspt2_ctx* c, int cls, double* NL, double* lv) {
  if (!c || cls < 0 || cls >= CASPT2_NCLASS) return CASPT2_EINVAL;
  if (!(c->opt.class_mask >> cls & 1u) || c->opt.target_state < 0) return CASPT2_EINVAL;
  if (!c->solved) return CASPT2_ESTATE;
  const size_t n = c->d.n;
  if (NL) std::memcpy(NL, c->hLamNL.data() + cls * n, sizeof(double) * n);
  if (lv) std::memcpy(lv, c->hLamLV.data() + cls * n * n, sizeof(double) * n * n);
  return CASPT2_OK;
}

int caspt2_get_core_energy(caspt2_ctx* c, double* ecore) {
  if (!c || !ecore) return CASPT2_EINVAL;
  if (!c->solved) return CASPT2_ESTATE;
  *ecore = c->hEcore;
  return CASPT2_OK;
}

int caspt2_get_timings(caspt2_ctx* c, double* times, int* count) {
  if (!c || !count) return CASPT2_EINVAL;
  int m = *count < kNumTimes ? *count : kNumTimes;
  for (int k = 0; k < m && times; ++k) times[k] = c->times[k];
  *count = kNumTimes;
  return CASPT2_OK;
}

long caspt2_get_kernel_launches(caspt2_ctx* c) { return c ? c->launches : -1; }

int caspt2_get_moments(caspt2_ctx* c, double* mom) {
  if (!c || !mom) return CASPT2_EINVAL;
  if (!c->solved) return CASPT2_ESTATE;
  const long n = c->d.n, msz = n * n * n + n * n + n;
  CASPT2_CUDA_TRY(cudaSetDevice(c->device));
  CASPT2_CUDA_TRY(cudaMemcpy(mom, c->mom, sizeof(double) * CASPT2_NCLASS * msz,
                             cudaMemcpyDeviceToHost));
  return CASPT2_OK;
}

int caspt2_finalize_moments(caspt2_ctx* c, const double* mom, void* stream) {
  if (!c || !mom) return CASPT2_EINVAL;
  if (!c->solved) return CASPT2_ESTATE;
  CASPT2_CUDA_TRY(cudaSetDevice(c->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const caspt2_options& o = c->opt;
  const int n = c->d.n;
  const long msz = (long)n * n * n + n * n + n;
  CASPT2_CUDA_TRY(cudaMemsetAsync(c->status, 0, sizeof(int), s));
  CASPT2_CUDA_TRY(cudaMemcpyAsync(c->mom, mom, sizeof(double) * CASPT2_NCLASS * msz,
                                  cudaMemcpyHostToDevice, s));
  CASPT2_CUDA_TRY(cudaMemsetAsync(c->ecls, 0, sizeof(double) * CASPT2_NCLASS * n * n, s));
  CASPT2_CUDA_TRY(cudaMemsetAsync(c->ncls, 0, sizeof(double) * CASPT2_NCLASS * n, s));
  for (int k = 0; k < CASPT2_NCLASS; ++k) {
    if (!(o.class_mask >> k & 1u)) continue;
    CASPT2_CUDA_TRY(launch_moments_to_e(c->mom + (long)k * msz, n, c->ecls + (long)k * n * n,
                                        c->ncls + (long)k * n, s));
  }
  CASPT2_CUDA_TRY(launch_heff(c->href, c->ecls, c->ncls, o.class_mask, o.shift, n, c->heff, s));
  CASPT2_CUDA_TRY(launch_sym_eig(c->heff, n, c->R, c->ems, 0, c->status, s));
  CASPT2_CUDA_TRY(cudaMemsetAsync(c->lamNL, 0, sizeof(double) * CASPT2_NCLASS * n, s));
  CASPT2_CUDA_TRY(cudaMemsetAsync(c->lamLV, 0, sizeof(double) * CASPT2_NCLASS * n * n, s));
  if (o.target_state >= 0) {
    for (int k = 0; k < CASPT2_NCLASS; ++k) {
      if (!(o.class_mask >> k & 1u)) continue;
      CASPT2_CUDA_TRY(launch_lambda(c->mom + (long)k * msz, c->R, n, o.target_state, o.shift,
                                    c->lamNL + (long)k * n, c->lamLV + (long)k * n * n, s));
    }
  }
  int hst = 0;
  CASPT2_CUDA_TRY(cudaMemcpyAsync(c->hHeff.data(), c->heff, sizeof(double) * n * n, cudaMemcpyDeviceToHost, s));
  CASPT2_CUDA_TRY(cudaMemcpyAsync(c->hEms.data(), c->ems, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
  CASPT2_CUDA_TRY(cudaMemcpyAsync(c->hR.data(), c->R, sizeof(double) * n * n, cudaMemcpyDeviceToHost, s));
  CASPT2_CUDA_TRY(cudaMemcpyAsync(c->hEcls.data(), c->ecls, sizeof(double) * CASPT2_NCLASS * n * n, cudaMemcpyDeviceToHost, s));
  CASPT2_CUDA_TRY(cudaMemcpyAsync(c->hNcls.data(), c->ncls, sizeof(double) * CASPT2_NCLASS * n, cudaMemcpyDeviceToHost, s));
  CASPT2_CUDA_TRY(cudaMemcpyAsync(c->hLamNL.data(), c->lamNL, sizeof(double) * CASPT2_NCLASS * n, cudaMemcpyDeviceToHost, s));
  CASPT2_CUDA_TRY(cudaMemcpyAsync(c->hLamLV.data(), c->lamLV, sizeof(double) * CASPT2_NCLASS * n * n, cudaMemcpyDeviceToHost, s));
  CASPT2_CUDA_TRY(cudaMemcpyAsync(&hst, c->status, sizeof(int), cudaMemcpyDeviceToHost, s));
  CASPT2_CUDA_TRY(cudaStreamSynchronize(s));
  c->dens_done = false;
  if (hst != 0) return hst;
  for (double x : c->hEms)
    if (!(x == x) || x > 1e300 || x < -1e300) return CASPT2_ENAN;
  return CASPT2_OK;
}

}  // extern "C"

namespace {

// Device work space of the densities, sized from the solved classes.
int alloc_densities(caspt2_ctx* c) {
  const Dims& d = c->d;
  const size_t nmo = d.nmo(), n = d.n;
  int st = CASPT2_OK;
#define ALLOC(ptr, cnt) \
  if (st == CASPT2_OK) st = c->alloc(&(ptr), (cnt))
  ALLOC(c->dd1, nmo * nmo);
  ALLOC(c->dd2, nmo * nmo);
  ALLOC(c->dgdf, (size_t)d.X * nmo * nmo);
  long tall = 0;
  for (int k = 0; k < 7; ++k)
    if (c->cw_on[k]) tall = std::max(tall, class_dens_tall(c->cw[k], d));
  const bool h_on = (c->opt.class_mask >> CASPT2_CLASS_H & 1u) && d.c > 0 && d.v > 0;
  long partmax = std::max<long>(kDensPartMax, 4 * c->m2max);
  if (h_on) {
    partmax = std::max<long>(partmax, (long)d.v * d.v);
    partmax = std::max<long>(partmax, 2L * 64 * (long)n * n * n);
  }
  partmax = std::max<long>(partmax, 152L * 4 * 256);
  ALLOC(c->dw.part, (size_t)partmax);
  c->dw.partmax = partmax;
  if (tall > 0) {
    DensWork& w = c->dw;
    w.tall = tall;
    w.secmax = std::max<long>(c->wmax, 1);
    ALLOC(w.T, (size_t)tall);
    ALLOC(w.Lam, (size_t)tall);
    ALLOC(w.U1, (size_t)tall);
    ALLOC(w.U2, (size_t)tall);
    ALLOC(w.Tsw, (size_t)tall);
    ALLOC(w.sec, 2 * (size_t)w.secmax);
    ALLOC(w.tmp, 2 * (size_t)w.secmax);
    ALLOC(w.Dm, 2 * (size_t)std::max<long>(c->m2max, 1));
    ALLOC(c->gtmp, (size_t)std::max<long>(c->packmax, 1));
    for (auto& kv : c->eri_blk) {
      const int dims3[3] = {d.c, d.a, d.v};
      const int sp4[4] = {kv.first / 27, (kv.first / 9) % 3, (kv.first / 3) % 3, kv.first % 3};
      const long sz = (long)dims3[sp4[0]] * dims3[sp4[1]] * dims3[sp4[2]] * dims3[sp4[3]];
      double* p = nullptr;
      ALLOC(p, (size_t)std::max<long>(sz, 1));
      c->gblk[kv.first] = p;
      c->g_tab.p[kv.first] = p;
    }
  }
  if (h_on) {
    HDensWork& h = c->hd;
    const long cv = (long)d.c * d.v;
    h.size = cv * cv;
    if (c->hK) h.K = c->hK;          // the split energy path keeps K for the densities
    else ALLOC(h.K, (size_t)h.size);
    ALLOC(h.B1, (size_t)h.size);
    ALLOC(h.B2, (size_t)h.size);
    ALLOC(h.pack, (size_t)d.X * cv);
    ALLOC(h.tmp, (size_t)d.X * cv);
    ALLOC(h.coef, 6 * n * n);
    h.part = c->dw.part;
    h.partmax = partmax;
  }
#undef ALLOC
  if (st == CASPT2_OK) c->dens_alloc = true;
  return st;
}

// The closed-active, active-virtual and closed-virtual blocks of d2 (dbar2 through the
// one-body couplings between classes) for the classes of class_mask, added to c->dd2.
int dens_offdiag(caspt2_ctx* c, unsigned class_mask, cudaStream_t s) {
  const Dims& d = c->d;
  const caspt2_options& o = c->opt;
  const int n = d.n, P = o.target_state;
  const bool h_on = (class_mask >> CASPT2_CLASS_H & 1u) && d.c > 0 && d.v > 0;
  if (!c->x_alloc) {
    std::vector<CrossPlan> all;
    cross_setup(c->xw, all);
    int st = c->alloc(&c->xw.plans, all.size());
    if (st != CASPT2_OK) return st;
    CASPT2_CUDA_TRY(cudaMemcpy(c->xw.plans, all.data(), sizeof(CrossPlan) * all.size(),
                               cudaMemcpyHostToDevice));
    cross_work_size(c->xw, d, &c->xwmax, &c->xzmax, &c->xpartmax);
    for (int k = 0; k < 7 && st == CASPT2_OK; ++k) {
      if (!c->cw_on[k]) continue;
      const size_t sz = (size_t)all_tuples(c->cw[k]) * n * c->cw[k].m;
      st = c->alloc(&c->xT[k], sz);
      if (st == CASPT2_OK) st = c->alloc(&c->xL[k], sz);
    }
    if (st == CASPT2_OK && (c->opt.class_mask >> CASPT2_CLASS_H & 1u) && d.c > 0 && d.v > 0) {
      const size_t sz = (size_t)d.c * d.c * d.v * d.v * n * n;
      st = c->alloc(&c->xT[7], sz);
      if (st == CASPT2_OK) st = c->alloc(&c->xL[7], sz);
    }
    if (st == CASPT2_OK) st = c->alloc(&c->xW, (size_t)c->xwmax);
    if (st == CASPT2_OK) st = c->alloc(&c->xZ, (size_t)c->xzmax);
    if (st == CASPT2_OK) st = c->alloc(&c->xpart, (size_t)c->xpartmax);
    if (st != CASPT2_OK) return st;
    c->x_alloc = true;
  }
  double* T[8] = {};
  double* L[8] = {};
  for (int k = 0; k < 7; ++k) {
    if (!(class_mask >> k & 1u) || !c->cw_on[k] || !c->xT[k]) continue;
    DensWork tmp = c->dw;
    tmp.T = c->xT[k];
    tmp.Lam = c->xL[k];
    tmp.tall = all_tuples(c->cw[k]) * n * c->cw[k].m;
    const int st = class_tuple_amplitudes(c->cw[k], tmp, d, o.shift, c->E0, c->eps, c->R, P,
                                          &c->oz, s);
    if (st != CASPT2_OK) return st;
    T[k] = c->xT[k];
    L[k] = c->xL[k];
  }
  if (h_on && c->xT[7]) {
    CASPT2_CUDA_TRY(launch_h_tuple_amps(c->hd.K, c->hw.eps, c->hw.W, c->hw.shifts, c->R, P, d,
                                        o.scheme, o.shift, c->xT[7], c->xL[7], s));
    T[7] = c->xT[7];
    L[7] = c->xL[7];
  }
  RdmPtrs g{{nullptr, c->rdm1r, c->rdm2r, c->rdm3r, c->rdm4r}};
  return cross_dbar2(c->xw, d, g, T, L, c->xW, c->xZ, c->xpart, c->xwmax, c->xzmax, c->xpartmax,
                     c->dd2, s);
}

// Copy `batch` nmo x nmo device matrices src (derivatives in the orbital basis the solve
// used) to dst in the caller's basis: C M C^T after a canonicalisation of the inputs, a
// plain copy otherwise.
int copy_out(caspt2_ctx* c, const double* src, long batch, double* dst, cudaMemcpyKind k) {
  const int nmo = c->d.nmo();
  const long nn = (long)nmo * nmo;
  if (!c->canon) {
    CASPT2_CUDA_TRY(cudaMemcpy(dst, src, sizeof(double) * batch * nn, k));
    return CASPT2_OK;
  }
  if (!c->canon_t1) {
    c->canon_chunk = std::max<long>(1, std::min<long>(std::max(c->d.X, 1), (1L << 26) / nn));
    int st = c->alloc(&c->canon_t1, (size_t)(c->canon_chunk * nn));
    if (st == CASPT2_OK) st = c->alloc(&c->canon_t2, (size_t)(c->canon_chunk * nn));
    if (st != CASPT2_OK) return st;
  }
  cudaStream_t s = cudaStreamPerThread;
  for (long b0 = 0; b0 < batch; b0 += c->canon_chunk) {
    const int nb = (int)std::min<long>(c->canon_chunk, batch - b0);
    CASPT2_CUDA_TRY(canon_back(c->canonC, src + b0 * nn, nmo, nb, c->canon_t1, c->canon_t2, s));
    CASPT2_CUDA_TRY(cudaStreamSynchronize(s));
    CASPT2_CUDA_TRY(cudaMemcpy(dst + b0 * nn, c->canon_t2, sizeof(double) * nb * nn, k));
  }
  return CASPT2_OK;
}

long block_size(const Dims& d, int key) {
  const int dims3[3] = {d.c, d.a, d.v};
  return (long)dims3[key / 27] * dims3[(key / 9) % 3] * dims3[(key / 3) % 3] * dims3[key % 3];
}

}  // namespace

extern "C" {

int caspt2_densities(caspt2_ctx* c, unsigned class_mask, void* stream) {
  if (!c) return CASPT2_EINVAL;
  if (!c->solved) return CASPT2_ESTATE;
  const caspt2_options& o = c->opt;
  if (o.target_state < 0 || (class_mask & ~o.class_mask) || c->d.a > 16 || c->partial())
    return CASPT2_EINVAL;
  CASPT2_CUDA_TRY(cudaSetDevice(c->device));
  if (!c->dens_alloc) {
    const int st = alloc_densities(c);
    if (st != CASPT2_OK) return st;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const Dims& d = c->d;
  const int n = d.n, P = o.target_state;
  const size_t nmo = d.nmo();
  const long launches0 = launch_counter();
  CASPT2_CUDA_TRY(cudaEventRecord(c->dev0, s));
  CASPT2_CUDA_TRY(cudaMemsetAsync(c->dd1, 0, sizeof(double) * nmo * nmo, s));
  CASPT2_CUDA_TRY(cudaMemsetAsync(c->dd2, 0, sizeof(double) * nmo * nmo, s));
  CASPT2_CUDA_TRY(cudaMemsetAsync(c->dgdf, 0, sizeof(double) * d.X * nmo * nmo, s));
  bool any_ag = false;
  for (int k = 0; k < 7; ++k) any_ag = any_ag || ((class_mask >> k & 1u) && c->cw_on[k]);
  if (any_ag) {
    for (auto& kv : c->gblk)
      CASPT2_CUDA_TRY(cudaMemsetAsync(kv.second, 0, sizeof(double) * block_size(d, kv.first), s));
    RdmPtrs g{{nullptr, c->rdm1r, c->rdm2r, c->rdm3r, c->rdm4r}};
    for (int k = 0; k < 7; ++k) {
      if (!(class_mask >> k & 1u) || !c->cw_on[k]) continue;
      const int st = class_densities(c->cw[k], c->dw, d, o.scheme, o.shift, g, c->E0, c->eps, c->R,
                                     P, c->lamNL + (long)k * n, c->g_tab, c->dd1, c->dd2, &c->oz,
                                     s);
      if (st != CASPT2_OK) return st;
    }
    for (auto& kv : c->gblk) {
      const int sp4[4] = {kv.first / 27, (kv.first / 9) % 3, (kv.first / 3) % 3, kv.first % 3};
      CASPT2_CUDA_TRY(gdf_from_block(c->B, d, sp4, kv.second, c->pack0, c->pack1, c->gtmp,
                                     c->dgdf, s, &c->oz));
    }
  }
  if ((class_mask >> CASPT2_CLASS_H & 1u) && d.c > 0 && d.v > 0) {
    const int st = classH_densities(c->B, d, c->hw, o.scheme, o.shift, c->R, P,
                                    c->lamNL + (long)CASPT2_CLASS_H * n, c->rdm1r, c->hd, c->dd2,
                                    c->dgdf, &c->oz, c->hK != nullptr && c->hd.K == c->hK, s);
    if (st != CASPT2_OK) return st;
  }
  if (o.dens_offdiag) {
    const int st = dens_offdiag(c, class_mask, s);
    if (st != CASPT2_OK) return st;
  }
  CASPT2_CUDA_TRY(launch_symmetrize(c->dd1, (int)nmo, 1, s));
  CASPT2_CUDA_TRY(launch_symmetrize(c->dd2, (int)nmo, 1, s));
  CASPT2_CUDA_TRY(launch_symmetrize(c->dgdf, (int)nmo, d.X, s));
  CASPT2_CUDA_TRY(cudaEventRecord(c->dev1, s));
  int ozerr = 0;
  if (c->oz.err)
    CASPT2_CUDA_TRY(cudaMemcpyAsync(&ozerr, c->oz.err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CASPT2_CUDA_TRY(cudaStreamSynchronize(s));
  if (ozerr != 0) return CASPT2_ETIMEOUT;
  float ms = 0.f;
  CASPT2_CUDA_TRY(cudaEventElapsedTime(&ms, c->dev0, c->dev1));
  c->times[kNumStages + 4] = ms;
  c->launches += launch_counter() - launches0;
  c->dens_done = true;
  return CASPT2_OK;
}

long caspt2_amplitude_size(const caspt2_ctx* c, int cls) {
  if (!c || cls < 0 || cls > CASPT2_CLASS_H) return CASPT2_EINVAL;
  if (cls == CASPT2_CLASS_H) return (long)c->d.c * c->d.c * c->d.v * c->d.v;
  if (!c->cw_on[cls]) return 0;
  const ClassWork& w = c->cw[cls];
  return (long)w.dc.nfam * all_tuples(w) * w.A;
}

}  // extern "C"

namespace {
// T_LN (lam = false) or lambda_LN of the target state (lam = true) of a class A-G, rebuilt
// from the sector eigenbases kept by the solve and gathered into out[fam][ext...][act...].
int get_class_vector(caspt2_ctx* c, int cls, int L, int N, int mem, double* out, bool lam,
                     void* stream) {
  if (!c || !out || cls < 0 || cls >= CASPT2_CLASS_H) return CASPT2_EINVAL;
  if (mem != CASPT2_MEM_HOST && mem != CASPT2_MEM_DEVICE) return CASPT2_EINVAL;
  if (!c->solved) return CASPT2_ESTATE;
  const caspt2_options& o = c->opt;
  const Dims& d = c->d;
  if (!c->cw_on[cls] || L < 0 || L >= d.n || N < 0 || N >= d.n || d.a > 16 || c->partial())
    return CASPT2_EINVAL;
  if (lam && o.target_state < 0) return CASPT2_EINVAL;
  // amplitudes carry closed and virtual indices of the canonical orbitals the solve used
  if (c->canon) return CASPT2_EINVAL;
  CASPT2_CUDA_TRY(cudaSetDevice(c->device));
  if (!c->dens_alloc) {
    const int st = alloc_densities(c);
    if (st != CASPT2_OK) return st;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ClassWork& w = c->cw[cls];
  const long size = (long)w.dc.nfam * all_tuples(w) * w.A;
  if (size == 0) return CASPT2_OK;
  const int P = o.target_state >= 0 ? o.target_state : 0;
  int st = class_tuple_amplitudes(w, c->dw, d, o.shift, c->E0, c->eps, c->R, P, &c->oz, s);
  if (st != CASPT2_OK) return st;
  // device output directly; host output through the (free) S T buffer, which holds
  // ntuples * n * m >= size doubles
  double* dst = mem == CASPT2_MEM_DEVICE ? out : c->dw.U1;
  CASPT2_CUDA_TRY(gather_amplitudes(w, d, lam ? c->dw.Lam : c->dw.T, L, N, dst, s));
  if (mem == CASPT2_MEM_HOST)
    CASPT2_CUDA_TRY(cudaMemcpyAsync(out, dst, sizeof(double) * size, cudaMemcpyDeviceToHost, s));
  int ozerr = 0;
  if (c->oz.err)
    CASPT2_CUDA_TRY(cudaMemcpyAsync(&ozerr, c->oz.err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CASPT2_CUDA_TRY(cudaStreamSynchronize(s));
  return ozerr != 0 ? CASPT2_ETIMEOUT : CASPT2_OK;
}
}  // namespace

extern "C" {

int caspt2_get_amplitudes(caspt2_ctx* c, int cls, int L, int N, int mem, double* out,
                          void* cuda_stream) {
  return get_class_vector(c, cls, L, N, mem, out, false, cuda_stream);
}

int caspt2_get_lambda(caspt2_ctx* c, int cls, int L, int N, int mem, double* out,
                      void* cuda_stream) {
  return get_class_vector(c, cls, L, N, mem, out, true, cuda_stream);
}

int caspt2_get_densities(caspt2_ctx* c, int mem, double* d1, double* d2, double* NL,
                         double* gdf) {
  if (!c) return CASPT2_EINVAL;
  if (mem != CASPT2_MEM_HOST && mem != CASPT2_MEM_DEVICE) return CASPT2_EINVAL;
  if (!c->dens_done) return CASPT2_ESTATE;
  CASPT2_CUDA_TRY(cudaSetDevice(c->device));
  const cudaMemcpyKind k = mem == CASPT2_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  const size_t nmo = c->d.nmo();
  int st = CASPT2_OK;
  if (d1 && st == CASPT2_OK) st = copy_out(c, c->dd1, 1, d1, k);
  if (d2 && st == CASPT2_OK) st = copy_out(c, c->dd2, 1, d2, k);
  if (st != CASPT2_OK) return st;
  if (NL) {
    // N_L summed over the classes in a fixed order (per-class shares of the last solve)
    const int n = c->d.n;
    std::vector<double> tot(n, 0.0);
    for (int cls = 0; cls < CASPT2_NCLASS; ++cls)
      if (c->opt.class_mask >> cls & 1u)
        for (int L = 0; L < n; ++L) tot[L] += c->hLamNL[(size_t)cls * n + L];
    CASPT2_CUDA_TRY(cudaMemcpy(NL, tot.data(), sizeof(double) * n,
                               mem == CASPT2_MEM_HOST ? cudaMemcpyHostToHost
                                                      : cudaMemcpyHostToDevice));
  }
  if (gdf) return copy_out(c, c->dgdf, c->d.X, gdf, k);
  return CASPT2_OK;
}

}  // extern "C"

namespace {
// Work arrays of the gradient and orbital-derivative assembly (first call only).
int alloc_grad_work(caspt2_ctx* c) {
  if (c->grad_alloc) return CASPT2_OK;
  const Dims& d = c->d;
  const size_t nmo = d.nmo(), a = d.a, X = d.X;
  int e = CASPT2_OK;
#define ALLOC(ptr, cnt) \
  if (e == CASPT2_OK) e = c->alloc(&(ptr), (cnt))
  ALLOC(c->gw.g1, a * a);
  ALLOC(c->gw.g2, a * a * a * a);
  ALLOC(c->gw.D, nmo * nmo);
  ALLOC(c->gw.dsa, nmo * nmo);
  ALLOC(c->gw.gD, X);
  ALLOC(c->gw.tq, X);
  ALLOC(c->gw.T, X * nmo * nmo);
  ALLOC(c->gw.M, X * nmo * nmo);
  ALLOC(c->gradf, nmo * nmo);
  ALLOC(c->gradB, X * nmo * nmo);
#undef ALLOC
  if (e != CASPT2_OK) return e;
  c->grad_alloc = true;
  return CASPT2_OK;
}
}  // namespace

extern "C" int caspt2_gradient(caspt2_ctx* c, int mem, double* grad_f, double* grad_B,
                               void* stream) {
  if (!c) return CASPT2_EINVAL;
  if (mem != CASPT2_MEM_HOST && mem != CASPT2_MEM_DEVICE) return CASPT2_EINVAL;
  if (!c->solved) return CASPT2_ESTATE;
  const caspt2_options& o = c->opt;
  if (o.xms != 0 || o.target_state < 0) return CASPT2_EINVAL;
  CASPT2_CUDA_TRY(cudaSetDevice(c->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int st = caspt2_densities(c, o.class_mask, stream);
  if (st != CASPT2_OK) return st;
  const Dims& d = c->d;
  const size_t nmo = d.nmo(), X = d.X;
  st = alloc_grad_work(c);
  if (st != CASPT2_OK) return st;
  if (d.a == 0) {
    CASPT2_CUDA_TRY(cudaMemsetAsync(c->gw.g1, 0, sizeof(double), s));
  }
  st = assemble_gradient(d, c->B, c->R, o.target_state, c->rdm1r, c->rdm2r, c->dact, c->bsum,
                         c->gam, c->dd1, c->dd2, c->dgdf, c->gw, c->gradf, c->gradB, s);
  if (st != CASPT2_OK) return st;
  CASPT2_CUDA_TRY(cudaStreamSynchronize(s));
  const cudaMemcpyKind k = mem == CASPT2_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  if (grad_f) {
    st = copy_out(c, c->gradf, 1, grad_f, k);
    if (st != CASPT2_OK) return st;
  }
  if (grad_B) return copy_out(c, c->gradB, X, grad_B, k);
  return CASPT2_OK;
}

// Orbital derivative Y_xy = dL/dk_xy of the target state's Lagrangian (Sec. II.D, Eq.
// orbderiv) from the densities of every block: see include/caspt2.h.
extern "C" int caspt2_orbital_derivative(caspt2_ctx* c, int mem, double* Y, void* stream) {
  if (!c || !Y) return CASPT2_EINVAL;
  if (mem != CASPT2_MEM_HOST && mem != CASPT2_MEM_DEVICE) return CASPT2_EINVAL;
  if (!c->solved) return CASPT2_ESTATE;
  const caspt2_options& o = c->opt;
  if (o.target_state < 0) return CASPT2_EINVAL;
  // the closed-active, active-virtual and closed-virtual blocks of d2 enter Y
  if (c->d.a > 0 && !o.dens_offdiag) return CASPT2_EINVAL;
  CASPT2_CUDA_TRY(cudaSetDevice(c->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int st = caspt2_densities(c, o.class_mask, stream);
  if (st != CASPT2_OK) return st;
  const Dims& d = c->d;
  const size_t nmo = d.nmo();
  st = alloc_grad_work(c);
  if (st != CASPT2_OK) return st;
  if (!c->orb_alloc) {
    int e = c->alloc(&c->orb_h, nmo * nmo);
    if (e == CASPT2_OK) e = c->alloc(&c->orb_gf, nmo * nmo);
    if (e == CASPT2_OK) e = c->alloc(&c->orb_y, nmo * nmo);
    if (e != CASPT2_OK) return e;
    c->orb_alloc = true;
  }
  if (d.a == 0) {
    CASPT2_CUDA_TRY(cudaMemsetAsync(c->gw.g1, 0, sizeof(double), s));
  }
  st = assemble_orbital_derivative(d, c->f, c->g, c->B, c->R, o.target_state, c->rdm1r,
                                   c->rdm2r, c->dact, c->bsum, c->gam, c->dd1, c->dd2, c->dgdf,
                                   c->gw, c->orb_h, c->orb_gf, c->gradB, c->orb_y, s);
  if (st != CASPT2_OK) return st;
  CASPT2_CUDA_TRY(cudaStreamSynchronize(s));
  const cudaMemcpyKind k = mem == CASPT2_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  return copy_out(c, c->orb_y, 1, Y, k);
}
