"""Active-space reference states and RDMs for large active spaces (input preparation).

The dense path of synth.casci builds the full active-space Hamiltonian and every
spin pattern of annihilated vectors; both grow too fast past ~2e4 determinants.  This
module prepares the same inputs for larger spaces (10 orbitals, 10 electrons: 63504
determinants), in torch so that it can use a GPU when one is present:

  * CI vectors are matrices X[alpha string, beta string] (the determinant order of
    synth.casci: alpha-major, alpha creators left of beta creators);
  * H X and S^2 X are applied through the dense one-spin excitation matrices
    e_pq[I, J] of synth.casci (E_pq = e_pq (x) 1 + 1 (x) e_pq, no sign for beta because
    E_pq moves an even number of operators past the alpha string);
  * the lowest singlets come from a block Davidson iteration on H + penalty * S^2
    (diagonal preconditioner), each vector signed so that its largest-|.| entry is
    positive, as in synth.casci.lowest_singlets;
  * the spin-free k-RDMs use one Gram matrix per number of alpha annihilators: a
    product of k annihilators a_{qk sk} ... a_{q1 s1} is, up to the sign of the
    permutation that sorts it, one canonical product (beta annihilators in descending
    orbital order to the left of alpha annihilators in descending order) of distinct
    spin-orbitals, and Gamma_{p1q1..pkqk} = sum over spins <a_pk..a_p1 M|a_qk..a_q1 N>
    is gathered from those Gram matrices with the two permutation signs.

Nothing here belongs to the perturbation method.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

from .casci import strings, string_excitation_matrices, _ann_table


def _torch():
    import torch
    return torch


class BigSpace:
    """Sz = 0 space of nel electrons in norb orbitals on a torch device."""

    def __init__(self, norb: int, nel: int, device: str = "cpu"):
        assert nel % 2 == 0
        torch = _torch()
        self.norb, self.nel = norb, nel
        self.na = self.nb = nel // 2
        self.ns = len(strings(norb, self.na))
        self.ndet = self.ns * self.ns
        self.dev = torch.device(device)
        e = string_excitation_matrices(norb, self.na)
        self.e = torch.tensor(e.reshape(norb * norb, self.ns, self.ns), dtype=torch.float64,
                              device=self.dev)
        occ = np.array([[(int(s) >> p) & 1 for p in range(norb)] for s in strings(norb, self.na)],
                       dtype=np.float64)
        self.occ = torch.tensor(occ, device=self.dev)          # [ns, norb]

    # --- operators on X[ns, ns, m] ---------------------------------------------
    def _e_all(self, X):
        """E_pq X for every (p, q): [norb^2, ns, ns, m]."""
        torch = _torch()
        return (torch.einsum("xij,jkm->xikm", self.e, X)
                + torch.einsum("xij,kjm->xkim", self.e, X))

    def sigma(self, X, h1, eri):
        """H X, H = sum h1_rs E_rs + 1/2 sum (rs|tu) E_{rs,tu} (E_{rs,tu} = E_rs E_tu -
        delta_st E_ru)."""
        torch = _torch()
        n = self.norb
        k = torch.as_tensor(h1 - 0.5 * np.einsum("rsst->rt", eri), device=self.dev).reshape(-1)
        v = torch.as_tensor(eri.reshape(n * n, n * n), device=self.dev)
        ex = self._e_all(X)
        w = 0.5 * torch.einsum("xy,yikm->xikm", v, ex) + k[:, None, None, None] * X[None]
        return (torch.einsum("xij,xjkm->ikm", self.e, w)
                + torch.einsum("xij,xkjm->kim", self.e, w))

    def s2(self, X):
        """S^2 X = N_b X - sum_pq e_qp X e_pq^T (Sz = 0)."""
        torch = _torch()
        n = self.norb
        et = self.e.reshape(n, n, self.ns, self.ns).transpose(0, 1).reshape(n * n, self.ns, self.ns)
        y = torch.einsum("xij,jkm->xikm", et, X)                 # e_qp X at index (p, q)
        y = torch.einsum("xikm,xlk->ilm", y, self.e)             # ... e_pq^T
        return self.nb * X - y

    def diag(self, h1, eri, penalty):
        """Diagonal of H + penalty S^2 over the determinants, [ns, ns]."""
        torch = _torch()
        J = torch.as_tensor(np.einsum("ppqq->pq", eri), device=self.dev)
        K = torch.as_tensor(np.einsum("pqqp->pq", eri), device=self.dev)
        h = torch.as_tensor(np.diag(h1).copy(), device=self.dev)
        na, nb = self.occ[:, None, :], self.occ[None, :, :]       # [ns, 1, n], [1, ns, n]
        ntot = na + nb
        d = (ntot * h).sum(-1)
        d = d + 0.5 * torch.einsum("abp,pq,abq->ab", ntot, J, ntot)
        exa = 0.5 * torch.einsum("ap,pq,aq->a", self.occ, K, self.occ)
        d = d - exa[:, None] - exa[None, :]
        s2 = self.nb - torch.einsum("ap,bp->ab", self.occ, self.occ)
        return d + penalty * s2


def _orthonormal(V, drop=None):
    """Orthonormal basis of the columns of V (tall, few columns): Cholesky of the Gram
    matrix on the host, twice; columns whose pivot falls below drop x the largest are
    left out."""
    torch = _torch()
    for _ in range(2):
        G = (V.T @ V).cpu().numpy()
        G = 0.5 * (G + G.T)
        if drop is not None:
            d = np.sqrt(np.maximum(np.diag(G), 0.0))
            keep = d > drop * d.max()
            V, G = V[:, torch.as_tensor(keep, device=V.device)], G[np.ix_(keep, keep)]
        w, Q = np.linalg.eigh(G)
        ok = w > 1e-12 * w.max()
        T = Q[:, ok] / np.sqrt(w[ok])
        V = V @ torch.as_tensor(T, device=V.device)
    return V


def davidson_singlets(space: BigSpace, h1, eri, nstate: int, penalty: float = 1.0,
                      tol: float = 1e-9, max_iter: int = 400, seed: int = 0):
    """Lowest nstate singlets of the active-space H (Davidson on H + penalty S^2).
    Returns (energies without the penalty, ci[ndet, nstate]) as numpy arrays."""
    torch = _torch()
    ns, nd = space.ns, space.ndet
    nroot = min(nd, 2 * nstate + 4)
    dg = space.diag(h1, eri, penalty).reshape(-1)

    def op(V):                                   # V [nd, m]
        X = V.reshape(ns, ns, -1)
        return (space.sigma(X, h1, eri) + penalty * space.s2(X)).reshape(nd, -1)

    # initial guesses: unit vectors on the lowest diagonal entries, symmetrised in
    # alpha <-> beta (singlets are symmetric under that exchange for an even count)
    order = torch.argsort(dg)
    V = torch.zeros((nd, nroot), dtype=torch.float64, device=space.dev)
    gen = torch.Generator(device="cpu").manual_seed(seed)
    used, col = set(), 0
    for idx in order.tolist():
        ia, ib = divmod(idx, ns)
        key = (min(ia, ib), max(ia, ib))
        if key in used:
            continue
        used.add(key)
        V[ia * ns + ib, col] += 1.0
        V[ib * ns + ia, col] += 1.0
        col += 1
        if col == nroot:
            break
    V = V + 1e-3 * torch.randn(V.shape, generator=gen, dtype=torch.float64).to(space.dev)
    V = _orthonormal(V)
    AV = op(V)
    for it in range(max_iter):
        Hs = (V.T @ AV).cpu().numpy()
        w, c = np.linalg.eigh(0.5 * (Hs + Hs.T))       # small dense problems on the host
        w = torch.as_tensor(w[:nroot], device=space.dev)
        c = torch.as_tensor(c[:, :nroot], device=space.dev)
        X = V @ c
        R = AV @ c - X * w
        rn = torch.sqrt((R * R).sum(dim=0))
        if float(rn.max()) < tol:
            break
        act = rn >= tol
        den = w[act][None, :] - dg[:, None]
        den = torch.where(den.abs() < 1e-8, torch.full_like(den, 1e-8), den)
        Rn = R[:, act] / den
        if V.shape[1] + Rn.shape[1] > 8 * nroot:      # restart on the current Ritz vectors
            V, AV = X, AV @ c
        Rn = Rn / torch.sqrt((Rn * Rn).sum(dim=0))
        for _ in range(2):                            # orthogonalise twice against V
            Rn = Rn - V @ (V.T @ Rn)
        keep = torch.sqrt((Rn * Rn).sum(dim=0)) > 1e-6   # drop directions already in span(V)
        Rn = Rn[:, keep]
        if Rn.shape[1] == 0 or V.shape[1] >= nd:
            break
        Rn = _orthonormal(Rn, drop=1e-6)
        Rn = Rn - V @ (V.T @ Rn)
        Rn = Rn / torch.sqrt((Rn * Rn).sum(dim=0))
        V = torch.cat([V, Rn], dim=1)
        AV = torch.cat([AV, op(Rn)], dim=1)
    else:
        raise RuntimeError("Davidson did not converge")
    # singlets: <S^2> below 1e-6
    keep_e, keep_v = [], []
    S2X = space.s2(X.reshape(ns, ns, -1)).reshape(nd, -1)
    HX = space.sigma(X.reshape(ns, ns, -1), h1, eri).reshape(nd, -1)
    for j in range(X.shape[1]):
        if float(X[:, j] @ S2X[:, j]) < 1e-6:
            keep_e.append(float(X[:, j] @ HX[:, j]))
            keep_v.append(X[:, j])
        if len(keep_v) == nstate:
            break
    if len(keep_v) < nstate:
        raise ValueError("not enough singlet states among the Davidson roots")
    ci = torch.stack(keep_v, dim=1).cpu().numpy()
    for j in range(nstate):
        if ci[np.argmax(np.abs(ci[:, j])), j] < 0:
            ci[:, j] *= -1
    return np.array(keep_e), ci


# --- RDMs from canonical annihilated vectors --------------------------------------

def _annihilate(X, norb, na, nb, spin, p):
    """a_{p spin} on X[sa, sb, m] in sector (na, nb) (torch): returns (Y, na', nb');
    beta operators carry (-1)^na for passing the alpha string (as synth.casci)."""
    torch = _torch()
    n = na if spin == 0 else nb
    src, dst, sgn = _ann_table(norb, n, p)
    nn = len(strings(norb, n - 1))
    dev = X.device
    s_t = torch.as_tensor(sgn, dtype=torch.float64, device=dev)
    if spin == 0:
        Y = torch.zeros((nn,) + tuple(X.shape[1:]), dtype=X.dtype, device=dev)
        if len(src):
            Y[torch.as_tensor(dst, device=dev)] = X[torch.as_tensor(src, device=dev)] * \
                s_t.reshape((-1,) + (1,) * (X.dim() - 1))
        return Y, na - 1, nb
    Y = torch.zeros((X.shape[0], nn) + tuple(X.shape[2:]), dtype=X.dtype, device=dev)
    if len(src):
        s_t = s_t * (-1.0 if na % 2 else 1.0)
        Y[:, torch.as_tensor(dst, device=dev)] = X[:, torch.as_tensor(src, device=dev)] * \
            s_t.reshape((1, -1) + (1,) * (X.dim() - 2))
    return Y, na, nb - 1


def _canonical_vectors(X0, norb, na, nb, nalpha, nbeta):
    """W[(A, B), M] = a_{B beta, desc} ... a_{A alpha, desc} |M>: the alpha annihilators of
    the sorted set A applied in ascending order, then the beta ones of B.  X0 [sa, sb, n].
    Returns (W [dim, nA * nB * n] with column ((A, B), M), list of A, list of B)."""
    torch = _torch()
    As = list(itertools.combinations(range(norb), nalpha))
    Bs = list(itertools.combinations(range(norb), nbeta))
    cols = []
    for A in As:
        Y, a1, b1 = X0, na, nb
        for p in A:
            Y, a1, b1 = _annihilate(Y, norb, a1, b1, 0, p)
        for B in Bs:
            Z, a2, b2 = Y, a1, b1
            for q in B:
                Z, a2, b2 = _annihilate(Z, norb, a2, b2, 1, q)
            cols.append(Z.reshape(-1, Z.shape[-1]))
    W = torch.stack(cols, dim=1)                   # [dim, nA*nB, n]
    return W.reshape(W.shape[0], -1), As, Bs


def _perm_parity(keys):
    inv = 0
    for i in range(len(keys)):
        for j in range(i + 1, len(keys)):
            if keys[i] > keys[j]:
                inv += 1
    return -1.0 if inv % 2 else 1.0


def _pattern_maps(norb, k, spins, As, Bs):
    """For one spin pattern: map each index tuple (q1..qk) to (row of the canonical set,
    sign), row -1 when two annihilators of one spin coincide."""
    aidx = {A: i for i, A in enumerate(As)}
    bidx = {B: i for i, B in enumerate(Bs)}
    nB = len(Bs)
    rows = np.full(norb ** k, -1, dtype=np.int64)
    sgn = np.zeros(norb ** k)
    for t, q in enumerate(itertools.product(range(norb), repeat=k)):
        A = sorted(q[j] for j in range(k) if spins[j] == 0)
        B = sorted(q[j] for j in range(k) if spins[j] == 1)
        if len(set(A)) < len(A) or len(set(B)) < len(B):
            continue
        # operator string left to right: a_{qk sk} ... a_{q1 s1}; canonical order has
        # key (0, -q) for beta and (1, -q) for alpha, ascending left to right
        keys = [(0 if spins[j] == 1 else 1, -q[j]) for j in range(k - 1, -1, -1)]
        rows[t] = aidx[tuple(A)] * nB + bidx[tuple(B)]
        sgn[t] = _perm_parity(keys)
    return rows, sgn


def rdms(space: BigSpace, ci: np.ndarray, kmax: int = 4, out_device=None):
    """Spin-free 1..kmax RDMs for all state pairs, {k: tensor [n, n, a^(2k)]} laid out
    [M][N][p1][q1]...[pk][qk] as synth.casci.ActiveSpace.rdm (on out_device, default the
    space's device)."""
    torch = _torch()
    a, n = space.norb, ci.shape[1]
    X0 = torch.as_tensor(ci, device=space.dev).reshape(space.ns, space.ns, n)
    out = {}
    for k in range(1, kmax + 1):
        total = torch.zeros((a ** k, n, a ** k, n), dtype=torch.float64, device=space.dev)
        for nalpha in range(k + 1):
            nbeta = k - nalpha
            if nalpha > space.na or nbeta > space.nb:
                continue
            W, As, Bs = _canonical_vectors(X0, a, space.na, space.nb, nalpha, nbeta)
            G = (W.T @ W).reshape(len(As) * len(Bs), n, len(As) * len(Bs), n)
            rows_q = max(1, int(2 ** 27 // max(1, n * n * a ** k)))   # ~1 GB temporaries
            for spins in itertools.product((0, 1), repeat=k):
                if sum(1 for s in spins if s == 0) != nalpha:
                    continue
                rows, sg = _pattern_maps(a, k, spins, As, Bs)
                r = torch.as_tensor(np.where(rows >= 0, rows, 0), device=space.dev)
                s = torch.as_tensor(sg, device=space.dev)         # 0 where rows < 0
                Gq = G.index_select(2, r) * s[None, None, :, None]
                # total[p, M, q, N] += s_p s_q G[r_p, M, r_q, N], in row chunks of p
                for p0 in range(0, a ** k, rows_q):
                    p1 = min(a ** k, p0 + rows_q)
                    total[p0:p1] += Gq.index_select(0, r[p0:p1]) * s[p0:p1, None, None, None]
                del Gq
            del W, G
        # -> [M][N][p1][q1]...[pk][qk]
        t = total.reshape((a,) * k + (n,) + (a,) * k + (n,))
        perm = [k, 2 * k + 1]
        for j in range(k):
            perm += [j, k + 1 + j]
        t = t.permute(perm).contiguous().reshape(n, n, -1)
        out[k] = t if out_device is None else t.to(out_device)
        del total
    return out
