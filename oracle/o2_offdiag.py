"""O2: the off-diagonal blocks of the density d-bar(2) (Sec. II.D),

  dbar2_xy = sum_L <Psi_lambda_L| E_xy |Psi1_L>,   x and y in different orbital spaces
             (closed-active, active-virtual, closed-virtual and their transposes).

TEST INFRASTRUCTURE (see oracle/__init__.py).  E_xy with x, y in different spaces changes
the (closed holes, virtual particles) count of an excitation, so it couples the first-order
functions of two different classes K' -> K:

  dh = [y closed] - [x closed],   dp = [x virtual] - [y virtual],   (h, p)_K = (h, p)_K' + (dh, dp)

Each coupling <M~| E_Omega(K)^dag E_xy E_Omega'(K')|N~> is reduced to Kronecker deltas and
rotated RDMs by the normal-ordering engine (oracle/wick.py) and contracted with the class
amplitude tensors T^K'_L and multipliers lambda^K_L (o2_classes.class_amplitudes for the
classes A-G; class H from the closed-shell pair form of o2_rdm, recast on E_ai,bj |N~>).
With the block-diagonal f of the solve these blocks are not read by the energy; they are
the derivative of the Lagrangian with respect to the off-diagonal f elements."""
from __future__ import annotations

import string
from functools import lru_cache

import numpy as np

from .o2_classes import CLASS_DEF, _bra_ops, _ket_ops, class_amplitudes
from .wick import Builder, expect

# (closed holes, virtual particles) of each class's excitation (Eq. class)
COUNTS = {"A": (1, 0), "B": (2, 0), "C": (0, 1), "D": (1, 1), "E": (2, 1), "F": (0, 2),
          "G": (1, 2), "H": (2, 2)}
# class H as a family for the engine: E_ai,bj, external slots in the order (i, j, a, b)
DEFS = dict(CLASS_DEF)
DEFS["H"] = ([(("a", "v"), ("i", "c"), ("b", "v"), ("j", "c"))], ["i", "j", "a", "b"],
             ("i", "j"), [])
OFFDIAG = [("c", "a"), ("a", "c"), ("a", "v"), ("v", "a"), ("c", "v"), ("v", "c")]


def _slot_space(cls):
    sp = {}
    for fam in DEFS[cls][0]:
        for slot, s in fam:
            sp[slot] = s
    return sp


@lru_cache(maxsize=None)
def cross_terms(K, fb, Kp, fk, X, Y):
    """Terms of <M| E_bra(K, fb)^dag E_xy E_ket(K', fk) |N> with x in space X, y in Y."""
    sp = {slot + "_b": s for slot, s in _slot_space(K).items()}
    sp.update({slot + "_k": s for slot, s in _slot_space(Kp).items()})
    sp.update({"x": X, "y": Y})
    b = Builder()
    ops = _bra_ops(b, DEFS[K][0][fb], "_b") + b.E("x", "y") + _ket_ops(b, DEFS[Kp][0][fk], "_k")
    return tuple(expect(ops, sp))


def class_h_amplitudes(prob, st, shift, scheme, R, P):
    """T^H_L and lambda^H_L as coefficients of E_ai,bj |N~> (unrestricted sum over i, j, a,
    b): arrays [L][1, i, j, a, b, N].  With the pair functions |Psi(t)> = 1/2 sum t E_ai E_bj
    |0> |nu> of o2_rdm.class_h_densities and |nu> = sum_N W_Nnu |N~>, the coefficient of
    E_ai,bj |N~> is 1/2 sum_nu W_Nnu t(L, nu)_ij^ab."""
    c, a, v, n = prob.nclosed, prob.nact, prob.nvirt, prob.nstate
    T = np.zeros((n, 1, c, c, v, v, n))
    Lam = np.zeros_like(T)
    if c == 0 or v == 0:
        return T, Lam
    vo = c + a
    eps = np.diag(prob.f)
    ec, ev = eps[:c], eps[vo:]
    Bcv = np.ascontiguousarray(prob.B[:, :c, vo:])
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
    for L, nu in pairs:
        D = D0 + shifts(nu, L)
        u = -K / D
        t = W[L, nu] * u
        lam = (r[L] * cnu[nu] + 2.0 * shift * r[L] ** 2 * W[L, nu] / D) * u
        for N in range(n):
            T[L, 0, :, :, :, :, N] += 0.5 * W[N, nu] * t
            Lam[L, 0, :, :, :, :, N] += 0.5 * W[N, nu] * lam
    return T, Lam


def _einsum_term(t, K, Kp, lamK, ampKp, rdm, n):
    """One engine term contracted with lambda^K (bra), T^K' (ket) and the RDM: [x][y]."""
    parent = {}

    def find(u):
        parent.setdefault(u, u)
        while parent[u] != u:
            u = parent[u]
        return u

    for u, w in t.deltas:
        parent[find(u)] = find(w)
    pool = iter(string.ascii_letters.replace("M", "").replace("N", ""))
    letters = {}

    def L(label):
        rt = find(label)
        if rt not in letters:
            letters[rt] = next(pool)
        return letters[rt]

    _, extK, _, actK = DEFS[K]
    _, extKp, _, actKp = DEFS[Kp]
    sb = "".join(L(e + "_b") for e in extK) + "".join(L(s + "_b") for s in actK) + "M"
    sk = "".join(L(e + "_k") for e in extKp) + "".join(L(s + "_k") for s in actKp) + "N"
    if t.rdm:
        sr = "MN" + "".join(L(p) + L(q) for p, q in t.rdm)
        g = rdm[len(t.rdm)]
    else:
        sr = "MN"
        g = np.eye(n)
    out = L("x") + L("y")
    return t.coeff * np.einsum(f"{sb},{sk},{sr}->{out}", lamK, ampKp, g, optimize=True)


def offdiag_dbar2(prob, st, shift, scheme, R, P, thresh=1e-9):
    """The closed-active, active-virtual and closed-virtual blocks (both orders) of
    dbar2 = sum_L <Psi_lambda_L|E_xy|Psi1_L> of target state P; zero elsewhere."""
    c, a, v, n, nmo = prob.nclosed, prob.nact, prob.nvirt, prob.nstate, prob.nmo
    rng = {"c": slice(0, c), "a": slice(c, c + a), "v": slice(c + a, nmo)}
    dims = {"c": c, "a": a, "v": v}
    amps = {cls: class_amplitudes(prob, st, cls, shift, scheme, R, P, thresh)
            for cls in "ABCDEFG"}
    amps["H"] = class_h_amplitudes(prob, st, shift, scheme, R, P)
    out = np.zeros((nmo, nmo))
    for X, Y in OFFDIAG:
        if dims[X] == 0 or dims[Y] == 0:
            continue
        dh = (Y == "c") - (X == "c")
        dp = (X == "v") - (Y == "v")
        for Kp, (h, p) in COUNTS.items():
            K = next((k for k, hp in COUNTS.items() if hp == (h + dh, p + dp)), None)
            if K is None:
                continue
            lam_all = amps[K][1]
            amp_all = amps[Kp][0]
            if not lam_all.size or not amp_all.size:
                continue
            for fb in range(len(DEFS[K][0])):
                for fk in range(len(DEFS[Kp][0])):
                    for t in cross_terms(K, fb, Kp, fk, X, Y):
                        for L in range(n):
                            out[rng[X], rng[Y]] += _einsum_term(
                                t, K, Kp, lam_all[L][fb], amp_all[L][fk], st.rdm, n)
    return out
