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


def class_h_moments(prob, st: Setup, shift: float = 0.0, scheme: str = "msmr"):
    """Moment sums (M1, M2, M3) of class E_ai,bj in the eigenbasis nu of U^T Fref U, where the
    sources are Vt_N(nu) = W_N nu k and sum_tuples k^2 = sum_ijab K(2K - K'):
      M1[L,N,L'] = sum_nu W_Nnu W_L'nu S1[nu,L],  M2[L,N] = sum_nu W_Nnu W_Lnu S2[nu,L],
      M3[L] = sum_nu W_Lnu^2 S3[nu,L],  Sk[nu,L] = sum_ijab K(2K - K') / D^k."""
    c, a, v, n = prob.nclosed, prob.nact, prob.nvirt, prob.nstate
    M1, M2, M3 = np.zeros((n, n, n)), np.zeros((n, n)), np.zeros(n)
    if c == 0 or v == 0:
        return M1, M2, M3
    vo = c + a
    eps = np.diag(prob.f)
    ec, ev = eps[:c], eps[vo:]
    X = prob.B.shape[0]
    Bcv = np.ascontiguousarray(prob.B[:, :c, vo:]).reshape(X, c * v)
    K = (Bcv.T @ Bcv).reshape(c, v, c, v)
    num = K * (2.0 * K - K.transpose(0, 3, 2, 1))
    D = (ev[None, :, None, None] + ev[None, None, None, :]
         - ec[:, None, None, None] - ec[None, None, :, None])
    if scheme == "sssr":
        for L in range(n):
            dd = D + shift
            M1[L, L, L] = np.sum(num / dd)
            M2[L, L] = np.sum(num / dd ** 2)
            M3[L] = np.sum(num / dd ** 3)
        return M1, M2, M3
    omega, W = np.linalg.eigh(0.5 * (st.Ftil + st.Ftil.T))
    for L in range(n):
        for nu in range(n):
            dd = D + omega[nu] - st.E0[L] + shift
            s1, s2, s3 = np.sum(num / dd), np.sum(num / dd ** 2), np.sum(num / dd ** 3)
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
