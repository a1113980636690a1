"""Active-space determinant machinery for the seeded input generator.

This module prepares the reference states that the method takes as input
(Sec. II.A: CASSCF-type reference states |M> = sum_I c_IM |I>, eigenfunctions
of the Hamiltonian inside the active space) and their spin-free reduced
density matrices.  It is input preparation only: nothing here belongs to the
perturbation method itself.

Determinant ordering (the layout of every CI vector this package writes):
  * an alpha (or beta) string is a bitmask over the nact active orbitals,
    bit p set = orbital p occupied; strings of a given electron count are
    listed in ascending integer order;
  * determinant index = ia * nstr_beta + ib (alpha-major);
  * the determinant is a+_{alpha strings, ascending orbital} a+_{beta strings,
    ascending orbital} |vac>, i.e. all alpha creators to the left of all beta
    creators.

RDM convention: Gamma^{MN}_{p1q1,...,pkqk} = <M| E_{p1q1,...,pkqk} |N> with
E_{p1q1,...,pkqk} = sum_{s1..sk} a+_{p1 s1} ... a+_{pk sk} a_{qk sk} ... a_{q1 s1};
stored as [n][n][p1][q1]...[pk][qk] (row-major, FP64).
"""
from __future__ import annotations

from functools import lru_cache
import itertools

import numpy as np


@lru_cache(maxsize=None)
def strings(norb: int, nel: int) -> np.ndarray:
    """All bitmasks over norb bits with nel set bits, ascending."""
    if nel < 0 or nel > norb:
        return np.zeros(0, dtype=np.int64)
    out = []
    for occ in itertools.combinations(range(norb), nel):
        m = 0
        for o in occ:
            m |= 1 << o
        out.append(m)
    return np.array(sorted(out), dtype=np.int64)


def _popcount_below(s: int, p: int) -> int:
    return bin(s & ((1 << p) - 1)).count("1")


@lru_cache(maxsize=None)
def _string_index(norb: int, nel: int) -> dict:
    return {int(s): i for i, s in enumerate(strings(norb, nel))}


@lru_cache(maxsize=None)
def _ann_table(norb: int, nel: int, p: int):
    """a_p on strings with nel electrons -> (src idx, dst idx, sign)."""
    src, dst, sgn = [], [], []
    tgt = _string_index(norb, nel - 1)
    for i, s in enumerate(strings(norb, nel)):
        s = int(s)
        if s >> p & 1:
            src.append(i)
            dst.append(tgt[s ^ (1 << p)])
            sgn.append(-1.0 if _popcount_below(s, p) % 2 else 1.0)
    return np.array(src, dtype=np.int64), np.array(dst, dtype=np.int64), np.array(sgn)


@lru_cache(maxsize=None)
def _cre_table(norb: int, nel: int, p: int):
    """a+_p on strings with nel electrons -> (src idx, dst idx, sign)."""
    src, dst, sgn = [], [], []
    tgt = _string_index(norb, nel + 1)
    for i, s in enumerate(strings(norb, nel)):
        s = int(s)
        if not (s >> p & 1):
            src.append(i)
            dst.append(tgt[s | (1 << p)])
            sgn.append(-1.0 if _popcount_below(s, p) % 2 else 1.0)
    return np.array(src, dtype=np.int64), np.array(dst, dtype=np.int64), np.array(sgn)


def apply_op(x: np.ndarray, norb: int, na: int, nb: int, kind: str, spin: int, p: int):
    """Apply a_{p spin} (kind 'a') or a+_{p spin} (kind 'c') to a batch of
    determinant vectors x[na_str, nb_str, ...] in sector (na, nb).

    Returns (y, na', nb').  Beta operators carry the (-1)^na sign of passing
    the alpha string."""
    if spin == 0:
        n = na
        tab = _ann_table(norb, n, p) if kind == "a" else _cre_table(norb, n, p)
        nn = n - 1 if kind == "a" else n + 1
        src, dst, sgn = tab
        y = np.zeros((len(strings(norb, nn)),) + x.shape[1:], dtype=x.dtype)
        if len(src):
            y[dst] = x[src] * sgn.reshape((-1,) + (1,) * (x.ndim - 1))
        return y, nn, nb
    n = nb
    tab = _ann_table(norb, n, p) if kind == "a" else _cre_table(norb, n, p)
    nn = n - 1 if kind == "a" else n + 1
    src, dst, sgn = tab
    y = np.zeros((x.shape[0], len(strings(norb, nn))) + x.shape[2:], dtype=x.dtype)
    if len(src):
        s = sgn * (-1.0 if na % 2 else 1.0)
        y[:, dst] = x[:, src] * s.reshape((1, -1) + (1,) * (x.ndim - 2))
    return y, na, nn


def string_excitation_matrices(norb: int, nel: int) -> np.ndarray:
    """Dense e_pq = a+_p a_q on one spin's strings: shape [norb, norb, nstr, nstr]."""
    ns = len(strings(norb, nel))
    e = np.zeros((norb, norb, ns, ns))
    for q in range(norb):
        s1, d1, g1 = _ann_table(norb, nel, q)
        for p in range(norb):
            s2, d2, g2 = _cre_table(norb, nel - 1, p)
            # compose: a_q maps s1->d1, then a+_p maps s2->d2 on (nel-1) strings
            inv = -np.ones(len(strings(norb, nel - 1)), dtype=np.int64)
            inv[s2] = np.arange(len(s2))
            for k in range(len(s1)):
                j = inv[d1[k]]
                if j >= 0:
                    e[p, q, d2[j], s1[k]] += g1[k] * g2[j]
    return e


class ActiveSpace:
    """Sz=0 determinant space of nel electrons in norb active orbitals."""

    def __init__(self, norb: int, nel: int):
        assert nel % 2 == 0, "singlet references with Sz = 0 need an even electron count"
        self.norb, self.nel = norb, nel
        self.na = self.nb = nel // 2
        self.astr = strings(norb, self.na)
        self.bstr = strings(norb, self.nb)
        self.ndet = len(self.astr) * len(self.bstr)
        self.e = string_excitation_matrices(norb, self.na)  # same for beta (na == nb)

    def det_strings(self):
        a = np.repeat(self.astr, len(self.bstr))
        b = np.tile(self.bstr, len(self.astr))
        return a, b

    # --- operators on [ndet, m] blocks -------------------------------------------
    def _as3(self, x):
        return x.reshape(len(self.astr), len(self.bstr), -1)

    def epq(self, x: np.ndarray, p: int, q: int) -> np.ndarray:
        """E_pq (spin-summed) applied to columns of x[ndet, m]."""
        x3 = self._as3(x)
        e = self.e[p, q]
        y = np.einsum("ij,jkm->ikm", e, x3, optimize=True)
        y += np.einsum("ij,kjm->kim", e, x3, optimize=True)
        return y.reshape(x.shape)

    def sigma(self, x: np.ndarray, h1: np.ndarray, eri: np.ndarray) -> np.ndarray:
        """H x with H = sum h1_rs E_rs + 1/2 sum (rs|tu) E_{rs,tu}."""
        n = self.norb
        # E_{rs,tu} = E_rs E_tu - delta_st E_ru
        k = h1 - 0.5 * np.einsum("rsst->rt", eri)
        ex = np.stack([self.epq(x, t, u) for t in range(n) for u in range(n)])  # [tu, ndet, m]
        w = 0.5 * np.tensordot(eri.reshape(n * n, n * n), ex, axes=(1, 0))
        w += k.reshape(n * n, 1, 1) * x[None]
        y = np.zeros_like(x)
        for r in range(n):
            for s in range(n):
                y += self.epq(w[r * n + s], r, s)
        return y

    def s_squared(self, x: np.ndarray) -> np.ndarray:
        """S^2 x = S- S+ x for Sz = 0 vectors, with S+ = sum_p a+_{p alpha} a_{p beta}."""
        x3 = self._as3(x)
        na, nb = self.na, self.nb
        sp = None
        for p in range(self.norb):
            y, a1, b1 = apply_op(x3, self.norb, na, nb, "a", 1, p)
            y, a1, b1 = apply_op(y, self.norb, a1, b1, "c", 0, p)
            sp = y if sp is None else sp + y
        out = None
        for p in range(self.norb):  # S- = sum_p a+_{p beta} a_{p alpha}
            y, a1, b1 = apply_op(sp, self.norb, na + 1, nb - 1, "a", 0, p)
            y, a1, b1 = apply_op(y, self.norb, a1, b1, "c", 1, p)
            out = y if out is None else out + y
        return out.reshape(x.shape)

    # --- reduced density matrices ---------------------------------------------
    def rdm(self, ci: np.ndarray, k: int) -> np.ndarray:
        """Spin-free k-RDM for all state pairs: [n][n][p1][q1]...[pk][qk].

        Gamma_{p..,q..} = sum over spins of <a_{pk}..a_{p1} M | a_{qk}..a_{q1} N>."""
        n = ci.shape[1]
        a = self.norb
        x0 = self._as3(ci)
        total = np.zeros((a,) * k + (n,) + (a,) * k + (n,))
        for spins in itertools.product((0, 1), repeat=k):
            # batch layout of vec: [sa, sb, n, p1, ..., pj]
            vecs = x0
            na, nb = self.na, self.nb
            for j in range(k):
                outs = []
                for p in range(a):
                    y, na2, nb2 = apply_op(vecs, a, na, nb, "a", spins[j], p)
                    outs.append(y)
                vecs = np.stack(outs, axis=-1)
                na, nb = na2, nb2
            if vecs.shape[0] == 0 or vecs.shape[1] == 0:
                continue
            flat = vecs.reshape(vecs.shape[0] * vecs.shape[1], -1)  # [dim, n*a^k]
            g = flat.T @ flat  # [(n,p1..pk), (n,q1..qk)]
            g = g.reshape((n,) + (a,) * k + (n,) + (a,) * k)
            # -> [p1..pk, M, q1..qk, N]
            perm = tuple(range(1, k + 1)) + (0,) + tuple(range(k + 2, 2 * k + 2)) + (k + 1,)
            total += g.transpose(perm)
        # reorder to [M][N][p1][q1]...[pk][qk]
        perm = [k, 2 * k + 1]
        for j in range(k):
            perm += [j, k + 1 + j]
        return np.ascontiguousarray(total.transpose(perm))


def hamiltonian_matrix(space: ActiveSpace, h1: np.ndarray, eri: np.ndarray) -> np.ndarray:
    """Dense H = sum h1_rs E_rs + 1/2 sum (rs|tu) E_{rs,tu} over the Sz = 0 determinants.

    With E_rs = e^a_rs + e^b_rs: H = H_a (x) 1 + 1 (x) H_b + sum (rs|tu) e_rs (x) e_tu,
    H_s = sum k_rs e_rs + 1/2 sum (rs|tu) e_rs e_tu, k = h1 - 1/2 sum_s (rs|st)."""
    n = space.norb
    e = space.e.reshape(n * n, *space.e.shape[2:])          # [rs, I, J]
    ns = e.shape[1]
    k = (h1 - 0.5 * np.einsum("rsst->rt", eri)).reshape(n * n)
    v = eri.reshape(n * n, n * n)
    g = np.tensordot(v, e, axes=(1, 0))                      # G_rs = sum_tu (rs|tu) e_tu
    hs = np.tensordot(k, e, axes=(0, 0)) + 0.5 * np.einsum("rij,rjk->ik", e, g)
    eye = np.eye(ns)
    hm = np.kron(hs, eye) + np.kron(eye, hs)
    ab = np.tensordot(e.reshape(n * n, ns * ns).T, g.reshape(n * n, ns * ns), axes=(1, 0))
    hm += ab.reshape(ns, ns, ns, ns).transpose(0, 2, 1, 3).reshape(ns * ns, ns * ns)
    return 0.5 * (hm + hm.T)


def s2_matrix(space: ActiveSpace) -> np.ndarray:
    """S^2 = N_b - sum_pq e^a_qp (x) e^b_pq  (Sz = 0)."""
    n = space.norb
    ns = space.e.shape[2]
    ea = space.e.transpose(1, 0, 2, 3).reshape(n * n, ns * ns)   # e_qp at index (p, q)
    eb = space.e.reshape(n * n, ns * ns)                          # e_pq
    m = -(ea.T @ eb).reshape(ns, ns, ns, ns).transpose(0, 2, 1, 3).reshape(ns * ns, ns * ns)
    m += space.nb * np.eye(ns * ns)
    return 0.5 * (m + m.T)


def lowest_singlets(space: ActiveSpace, h1: np.ndarray, eri: np.ndarray, nstate: int,
                    penalty: float = 1.0, tol: float = 1e-6):
    """Lowest nstate singlet eigenvectors of the active-space Hamiltonian.

    H + penalty * S^2 is diagonalised exactly (dense, lowest eigenpairs only);
    states with <S^2> above tol are skipped.  Each vector is signed so that its
    largest-|.| component is positive.  Returns (energies without the penalty,
    ci[ndet, nstate])."""
    import scipy.linalg as sl
    nd = space.ndet
    if nd > 20000:
        raise ValueError("dense CASCI limited to 20000 determinants")
    hm = hamiltonian_matrix(space, h1, eri)
    s2 = s2_matrix(space)
    keep_e, keep_v = [], []
    nwant = min(nd, 4 * nstate + 4)
    while True:
        w, v = sl.eigh(hm + penalty * s2, subset_by_index=[0, nwant - 1])
        keep_e, keep_v = [], []
        for j in range(v.shape[1]):
            c = v[:, j]
            if float(c @ s2 @ c) < tol:
                keep_e.append(float(c @ hm @ c))
                keep_v.append(c)
            if len(keep_v) == nstate:
                break
        if len(keep_v) == nstate or nwant == nd:
            break
        nwant = min(nd, 2 * nwant)
    if len(keep_v) < nstate:
        raise ValueError("not enough singlet states in the active space")
    ci = np.stack(keep_v, axis=1)
    for j in range(nstate):
        if ci[np.argmax(np.abs(ci[:, j])), j] < 0:
            ci[:, j] *= -1
    return np.array(keep_e), ci
