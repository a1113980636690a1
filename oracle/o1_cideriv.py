"""CI derivative of the CASPT2 Lagrangian and the XMS response (Sec. II.D: Eq. cideriv,
Eq. cideriv2, Eq. xmseq and the XMS terms Y', y~' and d-check), in the full determinant
space of o1_determinant.

TEST INFRASTRUCTURE (see oracle/__init__.py).

ytil[I][M] = dL_PT2/dc~_{I,M} at fixed amplitudes, multipliers and R, with c~ = c U the
rotated reference CI vectors and I an active-space determinant.  L_PT2 (Eq. lambdaeq)
is written out with explicit vectors:
    E_P   = <P|H|P> + <psi_P|H|P> - E_s sum_L R_LP^2 <psi_L|psi_L>,
    L_PT2 = E_P + sum_L [ <chi_L|(f^ - E0_L + E_s)|psi_L> + <chi_L|H|L~> ],
    psi_L = sum_(Omega, N) t_(Omega,LN) E_Omega|N~>,  chi_L likewise with lambda,
    |P> = sum_L R_LP |L~>, psi_P = sum_L R_LP psi_L,  E0_L = <L~|f^|L~>,
and f = h + g(d_sa) carries the state-averaged density of the references
(d_sa = (1/n) sum_N <N|E|N>), so f^ depends on the CI vectors too.  Each term is
differentiated with respect to every place a reference vector enters: the bra or ket
|L~>, the reference inside E_Omega|N~>, E0_L and d_sa.  (For the shift term the
Lagrangian's sum_L R_LP^2 <psi_L|psi_L> is used; the paper prints it with the mixed
amplitudes.)

The XMS rotation enters through the constraint sum_(M != N) w_MN <M~|f^|N~> = 0;
stationarity with respect to rotations of c~ gives Eq. xmseq
    w_MN = -sum_I (c~_IM ytil_IN - ytil_IM c~_IN) / (2 (E0_M - E0_N)),
zero for pairs closer than degen_thresh, and the constraint adds
    ytil'[I][N] = dC/dc~_{I,N}  (C = sum w_MN <M~|f^|N~>, through the bra, ket and d_sa),
    Y'           = the orbital derivative of C (f = h + g(d_sa) follows the orbitals),
    d-check_xy   = sum_MN w_MN <M~|E_xy|N~>.
The CI derivative with respect to the unrotated coefficients is y = (ytil [+ ytil']) U^T
(Eq. cideriv2).
"""
from __future__ import annotations

import numpy as np

from .o1_determinant import FullSpace, g_matrix, operator_tuples
from .o1_orbderiv import orbital_derivative


def _column_ops(space, tup):
    """E_Omega and E_Omega^dag as callables on full-space vectors, E_Omega = E_pq E_rs -
    delta_qr E_ps (Eq. class)."""
    p, q, r, s = tup

    def op(x):
        y = space.E[p, q] @ (space.E[r, s] @ x)
        return y - space.E[p, s] @ x if q == r else y

    def adj(x):
        y = space.E[s, r] @ (space.E[q, p] @ x)
        return y - space.E[s, p] @ x if q == r else y
    return op, adj


def _g_transpose(eri, d):
    """G with sum_xy d_xy g(D)_xy = sum_zw G_zw D_zw for every D (g of o1_determinant)."""
    return (np.einsum("xy,xyzw->zw", d, eri)
            - 0.25 * np.einsum("xy,xwzy->zw", d, eri)
            - 0.25 * np.einsum("xy,xzwy->zw", d, eri))


class _Derivs:
    """Everything the CI derivative needs, rebuilt from a problem and its O1 result."""

    def __init__(self, prob, res, shift, enuc=0.0):
        p = prob
        self.p, self.res, self.shift = p, res, shift
        nmo, n = p.nmo, p.nstate
        self.space = space = FullSpace(nmo, 2 * p.nclosed + p.nelact)
        self.eri = np.einsum("Ppq,Prs->pqrs", p.B, p.B)
        ref = space.embed(p.nclosed, p.ci, p.det_alpha, p.det_beta)
        self.rot = ref @ res.U
        ndet = p.ci.shape[0]
        self.emb = space.embed(p.nclosed, np.eye(ndet), p.det_alpha, p.det_beta)   # |I>
        self.f = res.h + g_matrix(self.eri, res.d_sa)
        nc = p.nclosed
        self.fhat = space.one_body(self.f, const=-2.0 * float(np.trace(self.f[:nc, :nc])))
        self.enuc = enuc
        tuples = operator_tuples(p.nclosed, p.nact, p.nvirt)
        self.ops = {}
        for cls, tl in tuples.items():
            for tup in tl:
                self.ops[(cls, tup)] = _column_ops(space, tup)
        # psi_L, chi_L and their per-reference parts
        self.psi, self.chi = [], []
        for L in range(n):
            ps = np.zeros(space.dim)
            ch = np.zeros(space.dim)
            for k, (cls, tup, N) in enumerate(res.cols[L]):
                v = self.ops[(cls, tup)][0](self.rot[:, N])
                ps += res.t[L][k] * v
                ch += res.lam[L][k] * v
            self.psi.append(ps)
            self.chi.append(ch)

    def H(self, x):
        r = self.res
        return self.space.apply_h(x, r.h, self.eri, self.enuc)

    def adj_ref(self, coef, L, M, y):
        """sum over the columns of state L on reference M of coef * E_Omega^dag y."""
        out = np.zeros(self.space.dim)
        for k, (cls, tup, N) in enumerate(self.res.cols[L]):
            if N == M and coef[L][k] != 0.0:
                out += coef[L][k] * self.ops[(cls, tup)][1](y)
        return out

    def dsa_term(self, d, M):
        """d/dc~_{.,M} of sum_xy d_xy f_xy(d_sa): W_M <I|E(G + G^T)|M~> with G = g^T(d)."""
        n = self.p.nstate
        G = _g_transpose(self.eri, d)
        return (1.0 / n) * (self.space.one_body(G + G.T) @ self.rot[:, M])


def ci_derivative(prob, res, shift, target=0):
    """ytil [ndet][n] = dL_PT2/dc~ (module docstring) for an O1Result with densities of
    target state `target` (res.d2 is dL/df over every block)."""
    return _ytil(_Derivs(prob, res, shift), res, shift, target)[0]


def _ytil(D, res, shift, target):
    n = D.p.nstate
    rP = res.R[:, target]
    mixP = D.rot @ rP
    psiP = sum(rP[L] * D.psi[L] for L in range(n))
    HP = D.H(mixP)
    NL = np.array([D.chi[L] @ D.psi[L] for L in range(n)])
    E0 = np.array([D.rot[:, L] @ (D.fhat @ D.rot[:, L]) for L in range(n)])
    out = np.zeros((D.emb.shape[1], n))
    for M in range(n):
        acc = 2.0 * rP[M] * HP                                   # <P|H|P>
        acc = acc + rP[M] * D.H(psiP)                            # <psi_P|H|P>, ket
        for L in range(n):                                       # ... refs inside psi_P
            acc = acc + rP[L] * D.adj_ref(res.t, L, M, HP)
        for L in range(n):                                       # -E_s R^2 <psi|psi>
            acc = acc - 2.0 * shift * rP[L] ** 2 * D.adj_ref(res.t, L, M, D.psi[L])
        acc = acc + D.H(D.chi[M])                                # <chi_L|H|L~>, ket
        for L in range(n):                                       # ... refs inside chi_L
            acc = acc + D.adj_ref(res.lam, L, M, D.H(D.rot[:, L]))
        for L in range(n):                                       # <chi|(f - E0 + Es)|psi>
            op_chi = D.fhat @ D.chi[L] + (shift - E0[L]) * D.chi[L]
            op_psi = D.fhat @ D.psi[L] + (shift - E0[L]) * D.psi[L]
            acc = acc + D.adj_ref(res.t, L, M, op_chi) + D.adj_ref(res.lam, L, M, op_psi)
        acc = acc - 2.0 * NL[M] * (D.fhat @ D.rot[:, M])         # E0_M = <M~|f^|M~>
        acc = acc + D.dsa_term(res.d2, M)                        # f = h + g(d_sa)
        out[:, M] = D.emb.T @ acc
    return out, D


def xms_response(prob, res, shift, target=0, degen_thresh=1e-8):
    """(ytil, w, ytil', dcheck, Y') for an O1Result with densities of target state
    `target`: Eq. cideriv, Eq. xmseq and the XMS terms (module docstring).  ytil' and Y'
    are zero when w is."""
    ytil, D = _ytil(_Derivs(prob, res, shift), res, shift, target)
    n = prob.nstate
    ct = D.emb.T @ D.rot                                         # c~ [ndet][n]
    E0 = np.array([D.rot[:, L] @ (D.fhat @ D.rot[:, L]) for L in range(n)])
    w = np.zeros((n, n))
    for M in range(n):
        for N in range(n):
            if M != N and abs(E0[M] - E0[N]) >= degen_thresh:
                w[M, N] = -(ct[:, M] @ ytil[:, N] - ytil[:, M] @ ct[:, N]) / (2.0 * (E0[M] - E0[N]))
    nc = prob.nclosed
    dcheck = np.zeros((prob.nmo, prob.nmo))
    for M in range(n):
        for N in range(n):
            if w[M, N] != 0.0:
                t = D.space.tdm1(D.rot[:, M], D.rot[:, N])
                t[np.arange(nc), np.arange(nc)] -= 2.0 * (D.rot[:, M] @ D.rot[:, N])
                dcheck += w[M, N] * t
    yprime = np.zeros_like(ytil)
    for N in range(n):
        acc = np.zeros(D.space.dim)
        for M in range(n):
            if w[M, N] != 0.0:
                acc = acc + 2.0 * w[M, N] * (D.fhat @ D.rot[:, M])
        acc = acc + D.dsa_term(dcheck, N)
        yprime[:, N] = D.emb.T @ acc
    # orbital derivative of C = sum_xy f_xy dcheck_xy (+ the vacuum constant, already in
    # dcheck's closed diagonal): f = h + g(d_sa) with h and (pq|rs) following the orbitals
    Yp = _constraint_orbital_derivative(res.h, D.eri, res.d_sa, dcheck)
    return ytil, w, yprime, dcheck, Yp


def _constraint_orbital_derivative(h, eri, dsa, dcheck):
    """d/dk_xy of sum_xy f_xy dcheck_xy, f = h + g((pq|rs), d_sa), the orbitals transformed
    as in o1_orbderiv (h' = C^T h C, (pq|rs) on all four indices, d_sa fixed)."""
    W = np.einsum("pq,rs->pqrs", dcheck, dsa) - 0.25 * np.einsum("ps,rq->pqrs", dcheck, dsa + dsa.T)
    Y = h @ dcheck.T + h.T @ dcheck
    Y = Y + np.einsum("pqrs,tqrs->tp", W, eri)
    Y = Y + np.einsum("qprs,qtrs->tp", W, eri)
    Y = Y + np.einsum("qrps,qrts->tp", W, eri)
    Y = Y + np.einsum("qrsp,qrst->tp", W, eri)
    return Y


def total_ci_derivative(prob, res, shift, target=0, xms=True, degen_thresh=1e-8):
    """dE_MS_P/dc [ndet][n] with respect to the unrotated CI coefficients (Eq. cideriv2):
    (ytil + ytil') U^T under XMS, ytil U^T with w = 0 under MS."""
    if xms:
        ytil, w, yp, _, _ = xms_response(prob, res, shift, target, degen_thresh)
        return (ytil + yp) @ res.U.T
    return ci_derivative(prob, res, shift, target) @ res.U.T


def total_orbital_derivative(prob, res, shift, target=0, xms=True, degen_thresh=1e-8):
    """Y + Y' (XMS) or Y (MS): the orbital derivative of the whole XMS-CASPT2 Lagrangian."""
    Y = orbital_derivative(res, prob.B)
    if xms:
        Y = Y + xms_response(prob, res, shift, target, degen_thresh)[4]
    return Y
