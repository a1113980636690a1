/*
 * caspt2.h -- C ABI of the GB300 (sm_103a) library for the (X)MS-CASPT2
 * amplitude / effective-Hamiltonian path of Vlaisavljevich & Shiozaki,
 * "Nuclear energy gradients for internally contracted complete active space
 * second-order perturbation theory: multistate extensions".
 *
 * Conventions (all calls):
 *   - orbitals are ordered [closed | active | virtual]; nmo = nclosed + nact + nvirt;
 *     i, j closed; r, s, t, u active; a, b virtual; x, y, z, w general (Sec. II).
 *   - every array is row-major FP64 (double).
 *   - spin-free RDMs between reference states M, N (unrotated, as supplied):
 *       rdm1[M][N][r][s]          = <M|E_rs|N>
 *       rdm2[M][N][r][s][t][u]    = <M|E_rs,tu|N>,  E_rs,tu = sum a+_r a+_t a_u a_s
 *       rdm3 / rdm4 likewise with 6 / 8 active indices.
 *   - the caller owns every buffer it passes; the library keeps no caller
 *     pointer once a call returns (inputs are copied into the context).
 *   - return value: 0 = OK, negative = error (CASPT2_E*), positive = warning.
 *     No call exits or aborts the process.
 *   - one context serves one stream at a time; contexts are independent.
 */
#ifndef CASPT2_H
#define CASPT2_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define CASPT2_OK            0
#define CASPT2_EINVAL      (-1)   /* bad sizes, options or pointers               */
#define CASPT2_ENOMEM      (-2)   /* device allocation failed                     */
#define CASPT2_ENOTCONV    (-3)   /* an eigensolver or iteration did not converge */
#define CASPT2_ENAN        (-4)   /* NaN/Inf found in inputs or results           */
#define CASPT2_ETIMEOUT    (-5)   /* a bounded device wait gave up                */
#define CASPT2_ECUDA       (-6)   /* a CUDA runtime call failed                   */
#define CASPT2_ESTATE      (-7)   /* call out of order (e.g. solve before inputs) */
#define CASPT2_ESCRATCH    (-8)   /* too large for the fixed scratch of caspt2_classH_noalloc */
#define CASPT2_WINTRUDER     1    /* smallest |denominator| below 1e-3 Eh          */
#define CASPT2_WDEGEN        2    /* XMS: two zeroth-order energies closer than    */
                                  /* options.degen_thresh (U not unique there)     */

/* memory kinds for caspt2_set_inputs */
#define CASPT2_MEM_HOST      0
#define CASPT2_MEM_DEVICE    1

/* contraction schemes (Sec. II.B, Eq. wfp and Eq. wfp2) */
#define CASPT2_MSMR          0
#define CASPT2_SSSR          1
/* precision forms */
#define CASPT2_FP64          0   /* plain FP64 on the FP64 pipe                              */
#define CASPT2_BF16X         1   /* exact BF16 splitting on the tcgen05 tensor cores: the DF  */
                                 /* integral contractions, the class-H pair integrals and the */
                                 /* density Gram products run as S-slice split GEMMs (see    */
                                 /* options.slices); eigensolvers, H^eff and reductions stay  */
                                 /* FP64                                                      */

/* excitation classes (Eq. class): A E_ri,st  B E_ri,sj  C E_ar,st  D E_ai,rs + E_ar,si
 *                                  E E_ai,rj  F E_ar,bs  G E_ar,bi  H E_ai,bj        */
enum { CASPT2_CLASS_A = 0, CASPT2_CLASS_B, CASPT2_CLASS_C, CASPT2_CLASS_D,
       CASPT2_CLASS_E, CASPT2_CLASS_F, CASPT2_CLASS_G, CASPT2_CLASS_H, CASPT2_NCLASS };

typedef struct caspt2_ctx caspt2_ctx;

typedef struct {
    int nclosed, nact, nvirt, naux, nstate;
} caspt2_dims;

typedef struct {
    int    xms;          /* 1: XMS rotation U from <L|f|M> (Sec. II.A); 0: MS, U = 1           */
    int    scheme;       /* CASPT2_MSMR or CASPT2_SSSR                                         */
    double shift;        /* vertical shift E_s >= 0, enters as (f - E0_L + E_s), Eq. (ampeq)  */
    double ovl_thresh;   /* overlap eigenvalue cut, default 1e-9 (Sec. II.B)                   */
    double enuc;         /* constant added to the diagonal of H^ref                            */
    int    target_state; /* P for lambda and densities; -1 = energies only                     */
    unsigned class_mask; /* bit k set = class k is included (default: all supported)           */
    int    precision;    /* CASPT2_FP64 (default) or CASPT2_BF16X                               */
    int    slices;       /* BF16 slices per operand for CASPT2_BF16X, 1..7 (default 7: every   */
                         /* product within FP64 rounding of the plain form; 5: ~2e-12 of the   */
                         /* row x column scale)                                                */
    double degen_thresh; /* XMS: |E0_M - E0_N| (Eh) below which the pair counts as degenerate */
                         /* (default 1e-8).  The rotation U is then fixed only up to a        */
                         /* rotation inside the degenerate subspace, which leaves every energy */
                         /* unchanged (Sec. II.D: the XMS response of such a pair is taken as  */
                         /* zero); the solve returns WDEGEN as a warning.                      */
    int    closed_begin; /* partial solve for splitting one solve over GPUs: the class-H     */
    int    closed_end;   /* pairs (i <= j) and class-G tuples (a, b, i) with closed_begin <=  */
                         /* i < closed_end; classes A-F only when closed_begin == 0.  The     */
                         /* per-class moments of the partitions summed (caspt2_get_moments)   */
                         /* and passed to caspt2_finalize_moments give the whole solve.       */
                         /* Default 0, -1 (all closed orbitals).                              */
    int    dens_offdiag; /* 1: caspt2_densities also forms the closed-active, active-virtual   */
                         /* and closed-virtual blocks of d2 (the one-body couplings between    */
                         /* classes, Sec. II.D); needs every class's amplitudes and lambda    */
                         /* over all index tuples in device memory at once (class H: c^2 v^2  */
                         /* n^2 doubles each).  Default 0 (those blocks are zero).            */
} caspt2_options;

/* Fill *opt with defaults: XMS, MS-MR, shift 0, 1e-9, enuc 0, target 0, all classes,
 * plain FP64, 7 slices, degen_thresh 1e-8. */
void caspt2_default_options(caspt2_options* opt);

/* Create a context for the given sizes.  Allocates its device buffers
 * (sizes fixed by dims) on the current device.  Errors: EINVAL, ENOMEM, ECUDA. */
int caspt2_create(caspt2_ctx** ctx, const caspt2_dims* dims, const caspt2_options* opt);

/* Copy the inputs into the context (Sec. II.A, II.B: reference states through their
 * RDMs, the state-averaged Fock matrix f and the DF factors defining (xy|zw)).
 *   mem   CASPT2_MEM_HOST or CASPT2_MEM_DEVICE (pointers on the context's device)
 *   fock  [nmo][nmo] symmetric SA Fock matrix f = h + g(d_sa) with zero closed-active,
 *         active-virtual and closed-virtual blocks.  The classes then decouple and each is
 *         solved exactly in one step (Eq. ampeq); a Fock matrix with coupling between the
 *         spaces needs the iterative solve of Sec. II.B, which this library does not do,
 *         so such an f is refused rather than solved with its coupling dropped.  If the
 *         closed or the virtual block is not diagonal (orbitals not canonical), the call
 *         rotates the closed and the virtual orbitals on the device to the eigenvectors of
 *         those blocks (f <- C^T f C, B_P <- C^T B_P C, C = blockdiag(Q_c, 1, Q_v)): every
 *         energy is invariant under such rotations (Sec. II.A), and the densities,
 *         caspt2_gradient and caspt2_orbital_derivative return their results rotated back
 *         to the caller's orbitals (C M C^T); caspt2_get_amplitudes / caspt2_get_lambda
 *         then return EINVAL (their closed and virtual indices would be the rotated ones).
 *   dfB   [naux][nmo][nmo] DF factors, (xy|zw) = sum_P B[P][x][y] B[P][z][w], symmetric in x,y
 *   rdm1  [n][n][a][a], rdm2 [n][n][a^4]   (required)
 *   rdm3, rdm4 may be NULL while only classes that do not need them are enabled.
 * Errors: EINVAL (NULL required pointer; f not symmetric, or an entry of a coupling block
 * above 1e-10 x max(1, max|f|) in magnitude — the context then holds no inputs), ENOMEM,
 * ENOTCONV (the eigensolver of a closed or virtual block), ECUDA. */
int caspt2_set_inputs(caspt2_ctx* ctx, int mem, const double* fock, const double* dfB,
                      const double* rdm1, const double* rdm2, const double* rdm3,
                      const double* rdm4);

/* Run the path on `cuda_stream` (a cudaStream_t, NULL = legacy default stream):
 * SA density and core Fock (Sec. II.B), XMS rotation and H^ref (Sec. II.A),
 * first-order amplitudes of the enabled classes (Eq. ampeq), the effective
 * Hamiltonian and its eigenpairs (Sec. II.B).  Synchronises the stream before
 * returning.  Returns WINTRUDER if a denominator fell below 1e-3 Eh, else WDEGEN if XMS
 * met two zeroth-order energies closer than opt.degen_thresh (both are reported in
 * caspt2_get_status's warnings).
 * Errors: ESTATE (no inputs), ENOTCONV, ENAN, ECUDA. */
int caspt2_solve(caspt2_ctx* ctx, void* cuda_stream);

/* Copy results of the last solve to host buffers (any pointer may be NULL):
 *   U [n][n] XMS rotation (columns = rotated states), E0 [n] zeroth-order energies,
 *   Href [n][n], Heff [n][n], Ems [n] ascending, R [n][n] (columns = eigenvectors;
 *   each column signed so that its largest-|.| entry is positive). */
int caspt2_get_energies(caspt2_ctx* ctx, double* U, double* E0, double* Href, double* Heff,
                        double* Ems, double* R);

/* Per-class pieces of the last solve (Sec. II.B effective Hamiltonian):
 *   e[L][L'] = <Psi1_L|H|L'~> restricted to class cls, norm[L] = <Psi1_L|Psi1_L> of that class.
 * Either pointer may be NULL.  Errors: EINVAL (class not enabled / out of range). */
int caspt2_get_class_energy(caspt2_ctx* ctx, int cls, double* e, double* norm);

/* lambda of the last solve for target state P = opt.target_state (the Lagrange multipliers
 * of Eq. lambdaeq, solution of the lambda equation obtained by differentiating the
 * Lagrangian with respect to T), per class, in gauge-invariant form:
 *   NL[L]     = <lambda_L|T_L> in the overlap metric (the class's share of N_L, Sec. II.D)
 *   lv[L][L'] = <Psi_lambda_L|H|L'~>, Psi_lambda_L = sum_N lambda_LN |N~>
 * Either pointer may be NULL.  Errors: EINVAL (class not enabled, or target_state < 0). */
int caspt2_get_class_lambda(caspt2_ctx* ctx, int cls, double* NL, double* lv);

/* Number of first-order amplitudes of a class per (L, N): nfam * (external tuples) *
 * a^(active indices) for the classes A-G (0 if the class is not enabled), c^2 v^2 for
 * class H.  Negative (EINVAL) for a null context or a bad class index. */
long caspt2_amplitude_size(const caspt2_ctx* ctx, int cls);

/* First-order amplitudes T_LN (Eq. ampeq, Sec. II.B: the solution of the class's amplitude
 * equation for reference state L, component N of the MS-MR basis;
 * SS-SR: zero for N != L) and the Lagrange multipliers lambda_LN of the target state
 * P = opt.target_state (Eq. lambdaeq, Sec. II.C), of a class A-G, in the range-projected gauge (the
 * amplitudes are expanded in the class's orthonormalised basis Y = X Q, X = V s^(-1/2) over
 * the overlap eigenvalues kept by the threshold).  out[amplitude_size] is laid out
 * [family][external indices in slot order][active indices], row-major, in the caller's
 * memory (mem = CASPT2_MEM_HOST or CASPT2_MEM_DEVICE).  The vector is rebuilt from the
 * sector eigenbases the solve keeps (the solve never stores amplitudes); the call runs on
 * cuda_stream and returns after the result is in out.  Errors: EINVAL (bad index, class H
 * (its amplitudes are never formed), class not enabled, lambda with target_state < 0, or
 * inputs canonicalised by caspt2_set_inputs), ESTATE (no solve yet), ETIMEOUT (a bounded
 * wait of a split GEMM gave up). */
int caspt2_get_amplitudes(caspt2_ctx* ctx, int cls, int L, int N, int mem, double* out,
                          void* cuda_stream);
int caspt2_get_lambda(caspt2_ctx* ctx, int cls, int L, int N, int mem, double* out,
                      void* cuda_stream);

/* Core energy E_core = <core|H|core> (closed orbitals doubly occupied) of the last solve. */
int caspt2_get_core_energy(caspt2_ctx* ctx, double* ecore);

/* Device time in milliseconds of the last solve, measured with CUDA events on the
 * solve stream: times[0] setup, [1] class H stage, [2] classes A-G, [3] effective
 * Hamiltonian and lambda, [4] the class-H DF-GEMM kernel alone (0 if class H is off),
 * [5] the Householder tridiagonalisation kernel summed over its launches, [6] its
 * algorithmic flops (4/3 m^3 per launch), [7] its number of launches, [8] the last
 * caspt2_densities call (0 before one), [9] the tridiagonalisation's algorithmic DRAM bytes
 * (the matrix read and the reflectors written once: 8 m^2 + 4 m (m - 1) per launch),
 * [10] the FP64 GEMM launches of the solve summed (device time by event pairs, the first
 * 4096 launches), [11] their algorithmic flops (2 M N K), [12] their number, [13] the panel
 * launches of the blocked Householder reduction (sectors too wide for shared memory) summed,
 * [14] the bytes of the trailing matrix their matrix-vector products read (8 n1^2 per
 * column, n1 the trailing size), [15] their number.
 *   times[k] is written for k < *count on input; *count = number of entries on output. */
int caspt2_get_timings(caspt2_ctx* ctx, double* times, int* count);

/* State of a context after its last calls: the last caspt2_solve's status (OK, WINTRUDER
 * or the error it returned; ESTATE before the first solve), whether a solve and a density
 * pass have completed, the smallest |denominator| e_ext + omega - E0_L + E_s of the last
 * solve (Eh; below 1e-3 the solve returned WINTRUDER; 0 before a solve), the library
 * kernels launched by the last solve, and the timings of caspt2_get_timings.
 * Errors: EINVAL (NULL pointer). */
#define CASPT2_REPORT_TIMES 10
#define CASPT2_WARN_INTRUDER 1u   /* warnings bit: WINTRUDER condition met */
#define CASPT2_WARN_DEGEN    2u   /* warnings bit: WDEGEN condition met    */
typedef struct {
  int last_status;
  int solved;
  int densities_done;
  double min_denominator;
  long kernel_launches;
  double times_ms[CASPT2_REPORT_TIMES];
  unsigned warnings;      /* CASPT2_WARN_* bits of the last solve                        */
  double min_e0_gap;      /* smallest |E0_M - E0_N| over M != N of the last solve (Eh;     */
                          /* 0 for one state)                                             */
} caspt2_report;
int caspt2_get_status(caspt2_ctx* ctx, caspt2_report* out);

/* Correlated densities of the target state P = opt.target_state (Sec. II.D: the
 * derivatives of the Lagrangian L = sum_LL' R_LP R_L'P Heff_LL' + sum <lambda|..> at the
 * converged amplitudes and lambda), computed on the device for the classes in
 * class_mask (a subset of the solved classes; CASPT2_CLASS_* bits), summed over them:
 *   d1[p][q]      derivative of the source terms <Omega|H|L'~> with respect to the
 *                 one-electron operator h (h = f minus the core and state-averaged active
 *                 mean fields, Sec. II.F) — classes A-G;
 *   d2[p][q]      derivative with respect to the Fock matrix f on the closed-closed,
 *                 active-active and virtual-virtual blocks (the blocks that the
 *                 block-diagonal f of the solve carries), including the E0 dependence of
 *                 the denominators (-N_L <L~|E_pq|L~>); with opt.dens_offdiag also the
 *                 closed-active, active-virtual and closed-virtual blocks
 *                 dbar2_xy = sum_L <Psi_lambda_L|E_xy|Psi1_L> (the couplings between
 *                 classes that an off-diagonal f would bring), else those blocks are zero;
 *   gdf[Q][p][q]  derivative with respect to the DF factors B[Q][p][q] of the two-electron
 *                 source terms (D(1) contracted with B, Sec. II.D DF form).
 * All three are returned symmetrised (x + x^T)/2 per matrix: the integrals are
 * symmetric, so only the symmetric part enters a gradient.
 * Call after a successful (or WINTRUDER) caspt2_solve with target_state >= 0; runs on
 * cuda_stream (NULL = default stream) and synchronises it.  The first call allocates
 * the density work space (about 6 x the largest class's amplitude array plus 3 (c v)^2
 * doubles for class H; with dens_offdiag, the all-tuple amplitude and lambda arrays of
 * every class).  Errors: EINVAL (mask outside the solved classes, target_state < 0,
 * nact > 16), ESTATE (no solve), ENOMEM, ECUDA. */
int caspt2_densities(caspt2_ctx* ctx, unsigned class_mask, void* cuda_stream);

/* Copy the densities of the last caspt2_densities call: d1 and d2 [nmo][nmo], NL [n], gdf
 * [naux][nmo][nmo] (the layout of the dfB input), to host (mem = CASPT2_MEM_HOST) or
 * device (CASPT2_MEM_DEVICE) buffers owned by the caller.  Any pointer may be NULL.
 *   NL[L] = sum_MN <M~|lambda_LM^dag T_LN|N~> over all eight classes (Sec. II.D, the
 *           normalisation term that multiplies <L~|E_xy|L~> in d(2)).
 * Errors: EINVAL, ESTATE (no densities computed since the last solve). */
int caspt2_get_densities(caspt2_ctx* ctx, int mem, double* d1, double* d2, double* NL,
                         double* gdf);

/* Gradient of the target state's MS energy E_P (opt.target_state) with respect to the
 * library's inputs, the Fock matrix f and the DF factors B, with the reference RDMs held
 * fixed (Sec. II.D: the densities chained through h = f - g(B, d_sa), the reference
 * Hamiltonian and the denominators):
 *   grad_f[p][q]     = dE_P/df_pq  = gamma_P + d1 + d2 on the closed-closed,
 *                      active-active and virtual-virtual blocks (the blocks of an f the
 *                      solve takes, see caspt2_set_inputs; off-diagonal closed and
 *                      virtual entries included);
 *   grad_B[Q][p][q]  = dE_P/dB_Qpq at fixed f;
 * both symmetrised, in the layouts of the inputs, to host or device buffers (mem).  MS
 * only (opt.xms = 0): the XMS rotation response is not formed.  The closed-active,
 * active-virtual and closed-virtual entries of grad_f are left zero: an f with those
 * blocks is refused, and their derivative is d-bar(2) of those blocks (caspt2_densities
 * with opt.dens_offdiag).  Recomputes the densities of all solved classes.
 * Errors: EINVAL (xms, target_state < 0), ESTATE (no solve), ENOMEM, ECUDA. */
int caspt2_gradient(caspt2_ctx* ctx, int mem, double* grad_f, double* grad_B, void* cuda_stream);

/* Orbital derivative of the target state's CASPT2 Lagrangian (Sec. II.D, Eq. orbderiv:
 * Y_xy = dL_PT2/dkappa_xy, the orbital part of the Z-vector source), from the relaxed
 * densities, in the density-fitted form
 *   Y = 2 [ h G + sum_Q B_Q Gb_Q ],
 *   G     = dL/dh   = gamma_P + d1 + d2        (every block of d2),
 *   Gb_Q  = dL/dB_Q at fixed h (the DF form of D(1), the reference two-electron part and
 *           d2 through f = h + g(B, d_sa)),
 * h = f - g(B, d_sa).  Convention: the orbitals change as phi'_y = phi_y + sum_x phi_x
 * kappa_xy with the reference CI vectors, the XMS rotation U and d_sa held fixed, every
 * integral following the orbitals; along an antisymmetric generator the change of L is
 * sum_xy kappa_xy (Y_xy - Y_yx).  For XMS this is the derivative at fixed rotated states
 * |M~>; the XMS term Y' (through w_MN, which needs the CI derivative) is not included.
 *   Y   [nmo][nmo] (not symmetric), to a host or device buffer (mem).
 * Needs opt.target_state >= 0 and, when nact > 0, opt.dens_offdiag = 1 (the closed-active,
 * active-virtual and closed-virtual blocks of d2 enter G).  Recomputes the densities of all
 * solved classes.  Errors: EINVAL (NULL, target_state < 0, dens_offdiag off), ESTATE (no
 * solve), ENOMEM, ECUDA. */
int caspt2_orbital_derivative(caspt2_ctx* ctx, int mem, double* Y, void* cuda_stream);

/* Per-class moment sums of the last solve (Sec. II.B, Eq. ampeq solved in each class's
 * orthonormal sector basis mu: M1[L][N][L'] = sum Vt_N Vt_L' / D_L, M2[L][N] =
 * sum Vt_N Vt_L / D_L^2, M3[L] = sum Vt_L^2 / D_L^3), laid out [class][n^3 + n^2 + n], to
 * a host buffer of CASPT2_NCLASS * (n^3 + n^2 + n) doubles.  They are sums over the
 * external index tuples, so the moments of partial solves over disjoint closed-orbital
 * ranges (options.closed_begin/closed_end) add up to those of the whole solve.
 * Errors: EINVAL, ESTATE (no solve). */
int caspt2_get_moments(caspt2_ctx* ctx, double* mom);

/* Replace the last solve's moments by `mom` (host, the layout of caspt2_get_moments; e.g.
 * summed over the partitions of one solve in a fixed order) and recompute from them the
 * per-class pieces, H^eff, E^MS, R and the lambda pieces of the target state, on
 * cuda_stream (synchronised).  The getters then return the combined results; the
 * densities and amplitude getters stay unavailable after a partial solve.
 * Errors: EINVAL, ESTATE (no solve), ENOTCONV, ENAN, ECUDA. */
int caspt2_finalize_moments(caspt2_ctx* ctx, const double* mom, void* cuda_stream);

/* Number of CUDA kernels the library launched during the last solve (-1 if ctx is NULL). */
long caspt2_get_kernel_launches(caspt2_ctx* ctx);

/* Bitmask of the classes this build implements. */
unsigned caspt2_supported_classes(void);

void caspt2_destroy(caspt2_ctx* ctx);
const char* caspt2_strerror(int status);

/* Size of the fixed device scratch array used by caspt2_classH_noalloc. */
#define CASPT2_NOALLOC_SCRATCH_BYTES ((size_t)4 << 20)

/* Class-H pieces e[L][L'] = <Psi1_L|H|L'~>_H and norm[L] = <Psi1_L|Psi1_L>_H (the same
 * values caspt2_get_class_energy returns for class H after caspt2_solve), computed
 * without allocating any device memory.  The paper has no counterpart: this entry
 * point exists for callers that cannot call cudaMalloc (code running inside another
 * framework's memory pool or a pre-sized arena, plugins in hosts that forbid
 * allocation after start-up, loops that must never enter the allocator).
 *   dims, opt     as for caspt2_create (opt->xms, scheme, shift are used)
 *   fock, dfB     device pointers, layouts as in caspt2_set_inputs
 *   rdm1          device pointer [n][n][a][a] (may be NULL when nact = 0)
 *   e, norm       device pointers to [n][n] and [n] outputs (written, caller-owned)
 *   cuda_stream   cudaStream_t to run on; the call synchronises it before returning
 * All intermediates live in one file-scope device array of CASPT2_NOALLOC_SCRATCH_BYTES
 * that every GPU loading the library keeps until the process exits.  The first call on
 * each device looks up that array's device address (cudaGetSymbolAddress) with the
 * device current; make that first call before any stream capture.  Calls share the
 * array: calls that overlap on the GPU (other threads or streams) race and must be
 * serialised by the caller.  Returns ESCRATCH when the problem needs more scratch than
 * the array holds (about 4 MiB: n <= 16 and nclosed + nvirt up to ~2e5 fit), EINVAL for
 * bad sizes, NULL pointers or an f that is not block diagonal with diagonal closed and
 * virtual blocks (this entry point takes canonical orbitals only; f is read back to host
 * memory for that check), ENOTCONV / ENAN / ECUDA, or WINTRUDER as caspt2_solve. */
int caspt2_classH_noalloc(const caspt2_dims* dims, const caspt2_options* opt,
                          const double* fock, const double* dfB, const double* rdm1,
                          double* e, double* norm, void* cuda_stream);

/* ---------------------------------------------------------------- serving form
 * A server that admits (X)MS-CASPT2 requests of different sizes while others run:
 * max_slots host workers, each with its own non-blocking CUDA stream on the device that
 * is current at creation, take queued requests in submission order as soon as a slot is
 * free and the request's estimated device memory fits the remaining budget, run
 * caspt2_create / set_inputs / solve (and caspt2_densities if requested) on their stream,
 * copy the results to host memory and free the request's device memory.  Work of
 * different requests overlaps on the device (separate streams); each request's
 * arithmetic is the same as a solve alone.  The paper has no counterpart (it distributes
 * one solve over MPI ranks). */
typedef struct caspt2_server caspt2_server;

typedef struct {
    caspt2_dims    dims;
    caspt2_options opt;
    /* host pointers, layouts as in caspt2_set_inputs; copied by caspt2_server_submit */
    const double *fock, *dfB, *rdm1, *rdm2, *rdm3, *rdm4;
    int densities;          /* 1: also caspt2_densities for opt.target_state (all classes) */
} caspt2_request;

typedef struct {
    int status;             /* status of the request's solve (OK, WINTRUDER, or an error) */
    double latency_ms;      /* submit -> results ready, measured by the server */
    double queue_ms;        /* submit -> admitted to a slot */
    /* caller-owned host outputs, any may be NULL: Ems [n], R and Heff [n][n],
       d1 and d2 [nmo][nmo], gdf [naux][nmo][nmo] */
    double *Ems, *R, *Heff, *d1, *d2, *gdf;
} caspt2_result;

/* hbm_budget_bytes: device memory the server may hold for requests at once (0: 90% of
 * the free memory at creation); max_slots: concurrent requests (1..64).
 * Errors: EINVAL, ENOMEM, ECUDA. */
int caspt2_server_create(caspt2_server** srv, size_t hbm_budget_bytes, int max_slots);

/* Queue a request (its inputs are copied; the caller may free them on return) and get
 * its ticket.  EINVAL for bad sizes/options/pointers or a request whose estimate exceeds
 * the whole budget; ESTATE after destroy has begun. */
int caspt2_server_submit(caspt2_server* srv, const caspt2_request* req, long* ticket);

/* Wait up to timeout_ms (< 0: no limit) for a ticket, copy its results into *out and
 * release it.  Returns the request's status, ETIMEOUT if it is not done yet (the ticket
 * stays valid), EINVAL for an unknown ticket. */
int caspt2_server_wait(caspt2_server* srv, long ticket, int timeout_ms, caspt2_result* out);

/* Finish the queued and running requests, then free the server. */
void caspt2_server_destroy(caspt2_server* srv);

#ifdef __cplusplus
}
#endif
#endif /* CASPT2_H */
