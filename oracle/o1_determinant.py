"""O1 -- (X)MS-CASPT2 amplitudes, lambda and densities by brute force in the
full determinant space.

TEST INFRASTRUCTURE (see oracle/__init__.py).  Nothing here is fast or clever:
every quantity is formed from explicit many-electron vectors, so that each
step can be checked against the paper by eye.  Sizes: a few 10^4
determinants at most.

Steps, in the paper's order (Sec. II):
  * reference states |M> embedded with closed orbitals doubly occupied and
    virtuals empty (Sec. II.A);
  * XMS: diagonalise <L|f|M> -> U, E~; rotated states |M~> = sum_N |N> U_NM;
    H^ref_MN = <M~|H|N~>; MS is U = 1 (Sec. II.A);
  * f^ = sum_xy f_xy {E_xy}_C with the closed-vacuum normal ordering read as
    subtracting the vacuum expectation value: f^ = sum f_xy E_xy - 2 sum_i f_ii
    (Sec. II.B, definition of {E_xy}_C); H = E_nuc + sum h_pq E_pq +
    1/2 sum (pq|rs) E_pq,rs with h = f - g(d_sa) (Sec. II.B, Fock definition);
  * first-order space: the nine operator families of Eq. (class) applied to
    every |N~> (MS-MR, Eq. wfp) or to |L~> only (SS-SR, Eq. wfp2);
  * amplitude equation Eq. (ampeq): (F - (E0_L - E_s) S) t_L = -V^T H |L~>,
    solved on the range of S after dropping overlap eigenvalues below the
    threshold (1e-9 by default), per class;
  * effective Hamiltonian, its diagonalisation and the explicit E^MS
    (Sec. II.B);
  * lambda equation (derivative of Eq. lambdaeq with respect to T);
  * correlated densities d(1), D(1), d(2), N_L (Sec. II.D).
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

CLASSES = ("A", "B", "C", "D", "E", "F", "G", "H")


def _strings(norb: int, nel: int):
    out = []
    for occ in itertools.combinations(range(norb), nel):
        m = 0
        for o in occ:
            m |= 1 << o
        out.append(m)
    return sorted(out)


def _bits_below(s: int, p: int) -> int:
    return bin(s & ((1 << p) - 1)).count("1")


class FullSpace:
    """Sz = 0 determinants of nelec electrons in nmo orbitals; index = ia*ns + ib,
    alpha creators left of beta creators, each string in ascending orbital order."""

    def __init__(self, nmo: int, nelec: int):
        assert nelec % 2 == 0
        self.nmo = nmo
        self.nhalf = nelec // 2
        self.str = _strings(nmo, self.nhalf)
        self.ns = len(self.str)
        self.dim = self.ns * self.ns
        self.index = {s: i for i, s in enumerate(self.str)}
        eye = sp.identity(self.ns, format="csr")
        self.E = {}
        for p in range(nmo):
            for q in range(nmo):
                e = self._string_exc(p, q)
                self.E[p, q] = (sp.kron(e, eye) + sp.kron(eye, e)).tocsr()

    def _string_exc(self, p: int, q: int):
        rows, cols, vals = [], [], []
        for j, s in enumerate(self.str):
            if not (s >> q & 1):
                continue
            sign = (-1) ** _bits_below(s, q)
            t = s ^ (1 << q)
            if t >> p & 1:
                continue
            sign *= (-1) ** _bits_below(t, p)
            u = t | (1 << p)
            rows.append(self.index[u])
            cols.append(j)
            vals.append(float(sign))
        return sp.csr_matrix((vals, (rows, cols)), shape=(self.ns, self.ns))

    def embed(self, nclosed: int, ci: np.ndarray, det_alpha, det_beta) -> np.ndarray:
        core = (1 << nclosed) - 1
        out = np.zeros((self.dim, ci.shape[1]))
        for k in range(ci.shape[0]):
            ia = self.index[core | (int(det_alpha[k]) << nclosed)]
            ib = self.index[core | (int(det_beta[k]) << nclosed)]
            out[ia * self.ns + ib] = ci[k]
        return out

    def one_body(self, m: np.ndarray, const: float = 0.0):
        """sum_pq m_pq E_pq + const as a sparse matrix."""
        acc = sp.identity(self.dim, format="csr") * const
        for (p, q), e in self.E.items():
            if m[p, q] != 0.0:
                acc = acc + m[p, q] * e
        return acc.tocsr()

    def apply_h(self, x: np.ndarray, h: np.ndarray, eri: np.ndarray, enuc: float) -> np.ndarray:
        """H x, H = E_nuc + sum h_pq E_pq + 1/2 sum (pq|rs)(E_pq E_rs - delta_qr E_ps)."""
        n = self.nmo
        k = h - 0.5 * np.einsum("prrq->pq", eri)
        u = np.stack([self.E[r, s] @ x for r in range(n) for s in range(n)])
        w = 0.5 * np.tensordot(eri.reshape(n * n, n * n), u, axes=(1, 0))
        w += k.reshape(n * n, *([1] * x.ndim)) * x[None]
        y = enuc * x
        for p in range(n):
            for q in range(n):
                y = y + self.E[p, q] @ w[p * n + q]
        return y

    def two_body(self, x: np.ndarray, p, q, r, s) -> np.ndarray:
        """E_{pq,rs} x = E_pq E_rs x - delta_qr E_ps x."""
        y = self.E[p, q] @ (self.E[r, s] @ x)
        if q == r:
            y = y - self.E[p, s] @ x
        return y

    def tdm1(self, bra: np.ndarray, ket: np.ndarray) -> np.ndarray:
        """<bra|E_xy|ket> for all x, y."""
        n = self.nmo
        out = np.zeros((n, n))
        for (p, q), e in self.E.items():
            out[p, q] = bra @ (e @ ket)
        return out

    def tdm2(self, bra: np.ndarray, ket: np.ndarray) -> np.ndarray:
        """<bra|E_{xy,zw}|ket> for all x, y, z, w."""
        n = self.nmo
        left = np.stack([self.E[y, x] @ bra for x in range(n) for y in range(n)])   # (E_yx bra) ~ <bra|E_xy
        right = np.stack([self.E[z, w] @ ket for z in range(n) for w in range(n)])
        g = (left @ right.T).reshape(n, n, n, n)
        g -= np.einsum("yz,xw->xyzw", np.eye(n), self.tdm1(bra, ket))
        return g


def operator_tuples(nclosed: int, nact: int, nvirt: int) -> dict:
    """Index tuples (p, q, r, s) of E_{pq,rs} for each class, Eq. (class).

    A: E_ri,st   B: E_ri,sj   C: E_ar,st   D: E_ai,rs and E_ar,si
    E: E_ai,rj   F: E_ar,bs   G: E_ar,bi   H: E_ai,bj
    (i, j closed; r, s, t active; a, b virtual)."""
    C = range(nclosed)
    A = range(nclosed, nclosed + nact)
    V = range(nclosed + nact, nclosed + nact + nvirt)
    P = itertools.product
    return {
        "A": [(r, i, s, t) for i, r, s, t in P(C, A, A, A)],
        "B": [(r, i, s, j) for i, j, r, s in P(C, C, A, A)],
        "C": [(a, r, s, t) for a, r, s, t in P(V, A, A, A)],
        "D": [(a, i, r, s) for a, i, r, s in P(V, C, A, A)]
             + [(a, r, s, i) for a, i, r, s in P(V, C, A, A)],
        "E": [(a, i, r, j) for a, i, j, r in P(V, C, C, A)],
        "F": [(a, r, b, s) for a, b, r, s in P(V, V, A, A)],
        "G": [(a, r, b, i) for a, b, r, i in P(V, V, A, C)],
        "H": [(a, i, b, j) for a, b, i, j in P(V, V, C, C)],
    }


def g_matrix(eri: np.ndarray, d: np.ndarray) -> np.ndarray:
    """[g(d)]_xy = sum_zw (xy|zw) d_zw - 1/4 (xw|zy)(d_zw + d_wz) (Sec. II.B)."""
    return (np.einsum("xyzw,zw->xy", eri, d)
            - 0.25 * np.einsum("xwzy,zw->xy", eri, d + d.T))


def _canon_columns(v: np.ndarray) -> np.ndarray:
    """Sign each eigenvector so that its largest-|.| component is positive."""
    v = v.copy()
    for j in range(v.shape[1]):
        if v[np.argmax(np.abs(v[:, j])), j] < 0:
            v[:, j] *= -1
    return v


@dataclass
class O1Result:
    U: np.ndarray
    E0: np.ndarray
    Href: np.ndarray
    Heff: np.ndarray
    Ems: np.ndarray
    R: np.ndarray
    Ems_explicit: float
    Ecore: float
    e_class: dict          # class -> [L, L'] contribution <Psi1_L|H|L'~> of that class
    norm_class: dict       # class -> [L] <Psi1_L|Psi1_L> of that class
    t: list                # per L: amplitude vector in the column basis of V_L
    lam: list              # per L: lambda vector (target state P)
    cols: list             # per L: list of (class, tuple, N) column labels
    S: list                # per L: overlap matrix
    b_src: list            # per L: [L'] -> V_L^T H |L'~>
    d1: np.ndarray = None
    D1: np.ndarray = None
    D1df: np.ndarray = None     # sum_zw D1[x,y,z,w] B[P,z,w]
    d2: np.ndarray = None
    dbar2: np.ndarray = None
    NL: np.ndarray = None
    gammaP: np.ndarray = None   # <P|E_xy|P>
    Gamma2P: np.ndarray = None  # <P|E_xy,zw|P>
    h: np.ndarray = None        # one-electron operator of H (f - g(d_sa) unless given)
    d_sa: np.ndarray = None     # state-averaged density over all orbitals (closed 2 delta)
    X: list = None              # per L: orthonormal basis of range(S), classes side by side
    A: list = None              # per L: X^T F X - (E0_L - E_s) 1 (every class coupling)
    Xcls: list = None           # per L: the class of each column of X


def solve(nclosed: int, nact: int, nvirt: int, nelact: int, f: np.ndarray, B: np.ndarray,
          ci: np.ndarray, det_alpha, det_beta, *, xms: bool = True, scheme: str = "msmr",
          shift: float = 0.0, thresh: float = 1e-9, target: int = 0, enuc: float = 0.0,
          h: np.ndarray | None = None, densities: bool = True, space: FullSpace | None = None,
          density_classes: str = "ABCDEFGH", U_fixed: np.ndarray | None = None) -> O1Result:
    """U_fixed: use this rotation of the reference states instead of the one XMS
    determines (for derivatives at fixed rotated states |M~>, Sec. II.D)."""
    nmo = nclosed + nact + nvirt
    n = ci.shape[1]
    eri = np.einsum("Ppq,Prs->pqrs", B, B)
    if space is None:
        space = FullSpace(nmo, 2 * nclosed + nelact)
    ref = space.embed(nclosed, ci, det_alpha, det_beta)          # |N>

    # state-averaged density over all orbitals (Sec. II.B) and h = f - g(d_sa)
    d_sa = np.zeros((nmo, nmo))
    for m in range(n):
        d_sa += space.tdm1(ref[:, m], ref[:, m]) / n
    if h is None:
        h = f - g_matrix(eri, d_sa)
    fhat = space.one_body(f, const=-2.0 * float(np.trace(f[:nclosed, :nclosed])))

    # XMS rotation (Sec. II.A)
    fref = ref.T @ (fhat @ ref)
    if U_fixed is not None:
        U = np.array(U_fixed, dtype=float)
    elif xms:
        w, U = np.linalg.eigh(0.5 * (fref + fref.T))
        U = _canon_columns(U)
    else:
        U = np.eye(n)
    rot = ref @ U                                                   # |M~>
    E0 = np.array([rot[:, l] @ (fhat @ rot[:, l]) for l in range(n)])
    Hrot = space.apply_h(rot, h, eri, enuc)                          # H|M~>
    Href = rot.T @ Hrot
    cc = np.arange(nclosed)
    Ecore = float(enuc + 2.0 * h[cc, cc].sum()
                  + 2.0 * np.einsum("iijj->", eri[:nclosed, :nclosed, :nclosed, :nclosed])
                  - np.einsum("ijji->", eri[:nclosed, :nclosed, :nclosed, :nclosed]))

    # first-order space (Eq. class, Eq. wfp / wfp2)
    tuples = operator_tuples(nclosed, nact, nvirt)
    ers = {}

    def column(tup, N):
        p, q, r, s = tup
        key = (r, s, N)
        if key not in ers:
            ers[key] = space.E[r, s] @ rot[:, N]
        y = space.E[p, q] @ ers[key]
        if q == r:
            y = y - space.E[p, s] @ rot[:, N]
        return y

    cols_all, vecs_all = [], []
    for cls in CLASSES:
        for tup in tuples[cls]:
            for N in range(n):
                cols_all.append((cls, tup, N))
                vecs_all.append(column(tup, N))
    Vall = np.stack(vecs_all, axis=1) if vecs_all else np.zeros((space.dim, 0))

    ts, lams, colsL, SL, bL, AL_solve = [], [], [], [], [], []
    XL, AL, XclsL = [], [], []
    for L in range(n):
        sel = [k for k, c in enumerate(cols_all) if scheme == "msmr" or c[2] == L]
        V = Vall[:, sel]
        cols = [cols_all[k] for k in sel]
        S = V.T @ V
        F = V.T @ (fhat @ V)
        b = {Lp: V.T @ Hrot[:, Lp] for Lp in range(n)}
        # orthonormal basis of range(S), per class (overlap eigenvalues < thresh dropped)
        blocks, xcls = [], []
        for cls in CLASSES:
            idx = [k for k, c in enumerate(cols) if c[0] == cls]
            if not idx:
                continue
            s_, q_ = np.linalg.eigh(S[np.ix_(idx, idx)])
            keep = s_ >= thresh
            x = np.zeros((len(cols), int(keep.sum())))
            x[idx] = q_[:, keep] / np.sqrt(s_[keep])
            blocks.append(x)
            xcls += [cls] * int(keep.sum())
        X = np.concatenate(blocks, axis=1) if blocks else np.zeros((len(cols), 0))
        A = X.T @ F @ X - (E0[L] - shift) * np.eye(X.shape[1])
        A = 0.5 * (A + A.T)

        def solver(rhs, X=X, A=A):
            return X @ np.linalg.solve(A, X.T @ rhs)

        t = -solver(b[L])
        ts.append(t)
        colsL.append(cols)
        SL.append(S)
        bL.append(b)
        AL_solve.append(solver)
        XL.append(X)
        AL.append(A)
        XclsL.append(xcls)

    # effective Hamiltonian (Sec. II.B)
    Heff = Href.copy()
    for L in range(n):
        for Lp in range(n):
            Heff[L, Lp] += 0.5 * (ts[L] @ bL[L][Lp] + bL[Lp][L] @ ts[Lp])
        Heff[L, L] -= shift * ts[L] @ SL[L] @ ts[L]
    Heff = 0.5 * (Heff + Heff.T)
    Ems, R = np.linalg.eigh(Heff)
    R = _canon_columns(R)
    P = target
    Ems_explicit = float(R[:, P] @ Href @ R[:, P]
                         + sum(R[L, P] * R[N, P] * (ts[L] @ bL[L][N]) for L in range(n) for N in range(n))
                         - shift * sum(R[L, P] ** 2 * ts[L] @ SL[L] @ ts[L] for L in range(n)))

    e_class, norm_class = {}, {}
    for cls in CLASSES:
        e = np.zeros((n, n))
        nm = np.zeros(n)
        for L in range(n):
            idx = [k for k, c in enumerate(colsL[L]) if c[0] == cls]
            if idx:
                for Lp in range(n):
                    e[L, Lp] = ts[L][idx] @ bL[L][Lp][idx]
                nm[L] = ts[L][idx] @ SL[L][np.ix_(idx, idx)] @ ts[L][idx]
        e_class[cls] = e
        norm_class[cls] = nm

    # lambda equation (derivative of Eq. lambdaeq with respect to T)
    for L in range(n):
        src = R[L, P] * sum(R[N, P] * bL[L][N] for N in range(n)) \
            - 2.0 * shift * R[L, P] ** 2 * (SL[L] @ ts[L])
        lams.append(-AL_solve[L](src))

    res = O1Result(U, E0, Href, Heff, Ems, R, Ems_explicit, Ecore, e_class, norm_class,
                   ts, lams, colsL, SL, bL)
    res.h, res.d_sa = h, d_sa
    res.X, res.A, res.Xcls = XL, AL, XclsL
    if not densities:
        return res

    # correlated densities (Sec. II.D)
    def full(vec, L):
        sel = [k for k, c in enumerate(cols_all) if scheme == "msmr" or c[2] == L]
        return Vall[:, sel] @ vec

    def only(vec, L):
        # restrict an amplitude vector to the columns of the requested classes
        sel = [k for k, c in enumerate(cols_all) if scheme == "msmr" or c[2] == L]
        mask = np.array([cols_all[k][0] in density_classes for k in sel], dtype=float)
        return vec * mask

    psi1 = [full(only(ts[L], L), L) for L in range(n)]
    psil = [full(only(lams[L], L), L) for L in range(n)]
    mixP = rot @ R[:, P]                                  # |P>
    psiT = sum(R[L, P] * psi1[L] for L in range(n))       # sum_M T_PM |M~> (mixed amplitudes)
    d1 = space.tdm1(psiT, mixP) + sum(space.tdm1(psil[N], rot[:, N]) for N in range(n))
    D1 = space.tdm2(psiT, mixP) + sum(space.tdm2(psil[N], rot[:, N]) for N in range(n))
    dbar2 = sum(space.tdm1(psil[L], psi1[L]) for L in range(n))
    NL = np.array([psil[L] @ psi1[L] for L in range(n)])
    res.D1df = np.einsum("xyzw,Pzw->Pxy", D1, B)
    d2 = dbar2.copy()
    act = slice(nclosed, nclosed + nact)
    for L in range(n):
        d2[act, act] -= NL[L] * space.tdm1(rot[:, L], rot[:, L])[act, act]
    # f^ = sum f_xy E_xy - 2 sum_i f_ii: the closed diagonal carries the -2 of the vacuum term
    d2[np.arange(nclosed), np.arange(nclosed)] -= 2.0 * NL.sum()
    res.d1, res.D1, res.d2, res.dbar2, res.NL = d1, D1, d2, dbar2, NL
    res.gammaP = space.tdm1(mixP, mixP)
    res.Gamma2P = space.tdm2(mixP, mixP)
    return res


def solve_problem(prob, **kw) -> O1Result:
    """Convenience wrapper for a synth.Problem."""
    return solve(prob.nclosed, prob.nact, prob.nvirt, prob.nelact, kw.pop("f", prob.f),
                 kw.pop("B", prob.B), kw.pop("ci", prob.ci), prob.det_alpha, prob.det_beta, **kw)
