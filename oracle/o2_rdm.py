"""O2 -- the same quantities as O1 written with RDMs and orbital-space tensors,
for sizes where the determinant space is out of reach.

TEST INFRASTRUCTURE (see oracle/__init__.py).  Plain numpy FP64, one einsum
per formula, no blocking.  Each function is pinned against O1 on tiny spaces
(tests/test_oracle_o2.py).

Reading of the closed-vacuum normal ordering (Sec. II.B): f^ = sum f_xy E_xy -
2 sum_i f_ii, so the zeroth-order energies are active-only (E0_L =
sum_rs f_rs <L~|E_rs|L~>) and a closed hole carries -e_i.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def _canon(v):
    v = v.copy()
    for j in range(v.shape[1]):
        if v[np.argmax(np.abs(v[:, j])), j] < 0:
            v[:, j] *= -1
    return v


@dataclass
class Setup:
    U: np.ndarray       # XMS rotation (columns = rotated states)
    Fref: np.ndarray    # <M|f|N> over the input states
    Ftil: np.ndarray    # U^T Fref U
    E0: np.ndarray      # zeroth-order energies (Sec. II.B)
    g: np.ndarray       # g(d_sa) over the active density (all orbital pairs)
    Ecore: float
    Href: np.ndarray
    rdm: dict           # rotated RDMs, k -> [n][n][a]*2k


def g_of(B: np.ndarray, d: np.ndarray) -> np.ndarray:
    """[g(d)]_xy = sum_zw (xy|zw) d_zw - 1/4 (xw|zy)(d_zw + d_wz), with (xy|zw) = B.B."""
    ds = d + d.T
    J = np.einsum("Pxy,Pzw,zw->xy", B, B, d, optimize=True)
    K = np.einsum("Pxw,Pzy,zw->xy", B, B, ds, optimize=True)
    return J - 0.25 * K


def setup(prob, xms: bool = True, enuc: float = 0.0, kmax: int = 2) -> Setup:
    c, a, n, nmo = prob.nclosed, prob.nact, prob.nstate, prob.nmo
    f, B = prob.f, prob.B
    act = slice(c, c + a)
    g1 = prob.rdm[1].reshape(n, n, a, a)
    # d_sa restricted to the active block; the closed block 2 delta is the core (Sec. II.B)
    d_act = np.zeros((nmo, nmo))
    d_act[act, act] = sum(g1[m, m] for m in range(n)) / n
    d_core = np.zeros((nmo, nmo))
    d_core[np.arange(c), np.arange(c)] = 2.0
    g_act = g_of(B, d_act)
    h = f - g_of(B, d_core + d_act)
    gc = g_of(B, d_core)
    Ecore = float(enuc + np.trace(h[:c, :c]) + np.trace((h + gc)[:c, :c]))
    # XMS (Sec. II.A)
    Fref = np.einsum("rs,mnrs->mn", f[act, act], g1)
    if xms:
        _, U = np.linalg.eigh(0.5 * (Fref + Fref.T))
        U = _canon(U)
    else:
        U = np.eye(n)
    Ftil = U.T @ Fref @ U
    E0 = np.diag(Ftil).copy()
    rdm = {}
    for k in range(1, kmax + 1):
        gk = prob.rdm[k].reshape(n, n, -1)
        rdm[k] = np.einsum("km,ln,kle->mne", U, U, gk).reshape((n, n) + (a,) * (2 * k))
    fc_act = (f - g_act)[act, act]
    eri = np.einsum("Prs,Ptu->rstu", B[:, act, act], B[:, act, act])
    Href = (np.einsum("rs,mnrs->mn", fc_act, rdm[1])
            + 0.5 * np.einsum("rstu,mnrstu->mn", eri, rdm[2]))
    Href += Ecore * np.eye(n)
    return Setup(U, Fref, Ftil, E0, g_act, Ecore, Href, rdm)


def class_h(prob, st: Setup, shift: float = 0.0, scheme: str = "msmr"):
    """Class E_ai,bj with block-diagonal f (Eq. ampeq restricted to the class).

    In the eigenbasis of U^T Fref U (W, omega) the equation for state L is the
    closed-shell pair equation with D = e_a + e_b - e_i - e_j + omega_nu - E0_L + E_s;
    returns (e[L, L'] = <Psi1_L|H|L'~>_H, norm[L] = <Psi1_L|Psi1_L>_H)."""
    c, a, v, n = prob.nclosed, prob.nact, prob.nvirt, prob.nstate
    if c == 0 or v == 0:
        return np.zeros((n, n)), np.zeros(n)
    vo = c + a
    eps = np.diag(prob.f)
    ec, ev = eps[:c], eps[vo:]
    X = prob.B.shape[0]
    Bcv = np.ascontiguousarray(prob.B[:, :c, vo:]).reshape(X, c * v)   # [P, (i, a)]
    K = (Bcv.T @ Bcv).reshape(c, v, c, v)                             # (ai|bj)
    num = K * (2.0 * K - K.transpose(0, 3, 2, 1))               # K (2K - (aj|bi))
    D = (ev[None, :, None, None] + ev[None, None, None, :]
         - ec[:, None, None, None] - ec[None, None, :, None])
    if scheme == "sssr":
        s1 = np.sum(num / (D + shift))
        s2 = np.sum(num / (D + shift) ** 2)
        return -s1 * np.eye(n), s2 * np.ones(n)
    omega, W = np.linalg.eigh(0.5 * (st.Ftil + st.Ftil.T))
    e = np.zeros((n, n))
    nr = np.zeros(n)
    for L in range(n):
        for nu in range(n):
            dd = D + omega[nu] - st.E0[L] + shift
            s1 = np.sum(num / dd)
            s2 = np.sum(num / dd ** 2)
            e[L, :] -= W[L, nu] * W[:, nu] * s1
            nr[L] += W[L, nu] ** 2 * s2
    return e, nr


def class_h_moments(prob, st: Setup, shift: float = 0.0, scheme: str = "msmr",
                    i_chunk: int | None = None, i_groups: int | None = None):
    """Moment sums (M1, M2, M3) of class E_ai,bj in the eigenbasis nu of U^T Fref U, where the
    sources are Vt_N(nu) = W_N nu k and sum_tuples k^2 = sum_ijab K(2K - K'):
      M1[L,N,L'] = sum_nu W_Nnu W_L'nu S1[nu,L],  M2[L,N] = sum_nu W_Nnu W_Lnu S2[nu,L],
      M3[L] = sum_nu W_Lnu^2 S3[nu,L],  Sk[nu,L] = sum_ijab K(2K - K') / D^k.
    i_chunk: the sums over i are taken for groups of i_chunk closed orbitals at a time
    (K(ai|bj) and its exchange partner K(aj|bi) = K(bi|aj) share the row index i, so a group
    needs only its own rows of K).  i_groups: stop after that many groups (a partial sum,
    for timing samples only)."""
    c, a, v, n = prob.nclosed, prob.nact, prob.nvirt, prob.nstate
    M1, M2, M3 = np.zeros((n, n, n)), np.zeros((n, n)), np.zeros(n)
    if c == 0 or v == 0:
        return M1, M2, M3
    vo = c + a
    eps = np.diag(prob.f)
    ec, ev = eps[:c], eps[vo:]
    X = prob.B.shape[0]
    Bcv = np.ascontiguousarray(prob.B[:, :c, vo:]).reshape(X, c * v)
    step = c if i_chunk is None else i_chunk
    if scheme == "sssr":
        shifts = [(L, None) for L in range(n)]
    else:
        omega, W = np.linalg.eigh(0.5 * (st.Ftil + st.Ftil.T))
        shifts = [(L, nu) for L in range(n) for nu in range(n)]
    sums = {key: np.zeros(3) for key in shifts}
    for g, i0 in enumerate(range(0, c, step)):
        if i_groups is not None and g >= i_groups:
            break
        i1 = min(c, i0 + step)
        K = (Bcv[:, i0 * v:i1 * v].T @ Bcv).reshape(i1 - i0, v, c, v)    # (ai|bj), i in group
        num = K * (2.0 * K - K.transpose(0, 3, 2, 1))               # K (2K - (aj|bi))
        del K
        D = (ev[None, :, None, None] + ev[None, None, None, :]
             - ec[i0:i1, None, None, None] - ec[None, None, :, None])
        for L, nu in shifts:
            dd = D + shift + (0.0 if nu is None else omega[nu] - st.E0[L])
            sums[(L, nu)] += [np.sum(num / dd), np.sum(num / dd ** 2), np.sum(num / dd ** 3)]
    if scheme == "sssr":
        for L in range(n):
            s1, s2, s3 = sums[(L, None)]
            M1[L, L, L] = s1
            M2[L, L] = s2
            M3[L] = s3
        return M1, M2, M3
    for L in range(n):
        for nu in range(n):
            s1, s2, s3 = sums[(L, nu)]
            M1[L] += np.outer(W[:, nu], W[:, nu]) * s1
            M2[L] += W[:, nu] * W[L, nu] * s2
            M3[L] += W[L, nu] ** 2 * s3
    return M1, M2, M3


def heff(st: Setup, parts: dict, shift: float):
    """H^eff = H^ref + 1/2 (e + e^T) - E_s diag(norm), summed over the given classes
    (Sec. II.B); returns (Heff, Ems ascending, R with canonical column signs)."""
    H = st.Href.copy()
    for e, nr in parts.values():
        H += 0.5 * (e + e.T) - shift * np.diag(nr)
    w, R = np.linalg.eigh(0.5 * (H + H.T))
    return H, w, _canon(R)


def class_h_densities(prob, st: Setup, R: np.ndarray, P: int, shift: float = 0.0,
                      scheme: str = "msmr"):
    """Class E_ai,bj share of the densities of target state P (Sec. II.D).

    In the eigenbasis nu of U^T Fref U the first-order functions of state L are closed-shell
    pair functions |Psi(t)> = 1/2 sum t_ij^ab E_ai E_bj |0> times |nu> = sum_N W_Nnu |N~>, with
      t(L, nu)   = -W_Lnu K / D,                      D = e_a + e_b - e_i - e_j + omega_nu - E0_L + E_s
      lam(L, nu) = -[R_LP c_nu + 2 E_s R_LP^2 W_Lnu / D] K / D,   c_nu = sum_N R_NP W_Nnu
    (under SS-SR only nu = L with W = 1 and D = e_a + e_b - e_i - e_j + E_s).  For two pair
    functions <Psi(l)|E_ab|Psi(t)> = 2 sum_ijc l_ij^ac (2 t_ij^bc - t_ij^cb),
    <Psi(l)|E_ij - 2 delta_ij|Psi(t)> = -2 sum_kab l_jk^ab (2 t_ik^ab - t_ik^ba),
    <Psi(l)|Psi(t)> = sum l (2t - t'), and the source functional sum w (2K - K') gives
    GDF[Q][a][i] = 2 sum_jb (2 w_ij^ab - w_ij^ba) B_Qbj with w the reference-projected
    combination R_L'P sum_L R_LP t + lam over the component along |L'~>.
    The active block of d2 pairs nu and nu' through <nu|E_rs|nu'> and carries -N_L <L~|E_rs|L~>.
    Returns (d2 closed, active and virtual blocks, GDF, NL)."""
    c, a, v, n, nmo = prob.nclosed, prob.nact, prob.nvirt, prob.nstate, prob.nmo
    d2 = np.zeros((nmo, nmo))
    GDF = np.zeros_like(prob.B)
    NL = np.zeros(n)
    if c == 0 or v == 0:
        return d2, GDF, NL
    vo = c + a
    eps = np.diag(prob.f)
    ec, ev = eps[:c], eps[vo:]
    X = prob.B.shape[0]
    Bcv = np.ascontiguousarray(prob.B[:, :c, vo:])          # [Q, i, a] = B_Q,ia = B_Q,ai
    K = np.einsum("Qia,Qjb->ijab", Bcv, Bcv)                  # (ai|bj)
    D0 = (ev[None, None, :, None] + ev[None, None, None, :]
          - ec[:, None, None, None] - ec[None, :, None, None])
    r = R[:, P]
    if scheme == "sssr":
        W = np.eye(n)
        shifts = lambda nu, L: shift
        pairs = [(L, L) for L in range(n)]
    else:
        omega, W = np.linalg.eigh(0.5 * (st.Ftil + st.Ftil.T))
        shifts = lambda nu, L: omega[nu] - st.E0[L] + shift
        pairs = [(L, nu) for L in range(n) for nu in range(n)]
    cnu = W.T @ r
    wsum = np.zeros_like(K)
    # active block: E_rs acts on |nu>, coupling nu and nu' of the same state L
    g1nu = np.einsum("mu,nw,mnrs->uwrs", W, W, st.rdm[1])      # <nu|E_rs|nu'>
    if scheme != "sssr":
        for L in range(n):
            for nu in range(n):
                Dl = D0 + shifts(nu, L)
                lam = (r[L] * cnu[nu] + 2.0 * shift * r[L] ** 2 * W[L, nu] / Dl) * (-K / Dl)
                for nu2 in range(n):
                    Dt = D0 + shifts(nu2, L)
                    t = W[L, nu2] * (-K / Dt)
                    ov = np.sum(lam * (2.0 * t - t.transpose(0, 1, 3, 2)))
                    d2[c:vo, c:vo] += ov * g1nu[nu, nu2]
    for L, nu in pairs:
        D = D0 + shifts(nu, L)
        u = -K / D
        t = W[L, nu] * u
        lam = (r[L] * cnu[nu] + 2.0 * shift * r[L] ** 2 * W[L, nu] / D) * u
        tt = 2.0 * t - t.transpose(0, 1, 3, 2)
        NL[L] += np.sum(lam * tt)
        d2[vo:, vo:] += 2.0 * np.einsum("ijac,ijbc->ab", lam, tt)
        d2[:c, :c] -= 2.0 * np.einsum("jkab,ikab->ij", lam, tt)
        # component along |L'~> of the IC amplitude: sum_nu W_L'nu (amplitude at nu)
        for Lp in range(n):
            if scheme == "sssr" and Lp != L:
                continue
            wsum += W[Lp, nu] * (r[Lp] * r[L] * t + (lam if Lp == L else 0.0))
    if scheme != "sssr":   # under SS-SR <lam_L|E_rs|T_L> = N_L <L~|E_rs|L~> cancels the E0 term
        for L in range(n):
            d2[c:vo, c:vo] -= NL[L] * st.rdm[1][L, L]
    # the lambda term pairs lambda_L' with reference L' only (Sec. II.D d(1)/D(1) definition)
    GDF[:, vo:, :c] = 2.0 * np.einsum("ijab,Qjb->Qai", 2.0 * wsum - wsum.transpose(0, 1, 3, 2), Bcv)
    return d2, GDF, NL
