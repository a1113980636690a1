"""Input variants shared by the oracle pins and the GPU tests (input construction only:
nothing here computes a result of the method)."""
from __future__ import annotations

import copy

import numpy as np


def degenerate_xms_problem(p):
    """A copy of the synth.Problem `p` (two or more states) whose Fock matrix is changed
    in its active block only, by the smallest symmetric change that makes the XMS Fock
    matrix F_MN = sum_rs f_rs <M|E_rs|N> a multiple of the identity: every pair of
    zeroth-order energies is then degenerate and any rotation of the states is an XMS
    rotation.  The active block is the only part of f that F depends on."""
    n, a, c = p.nstate, p.nact, p.nclosed
    g1 = p.rdm[1].reshape(n, n, a, a)
    g1s = 0.5 * (g1 + g1.transpose(0, 1, 3, 2))
    iu = np.triu_indices(a)
    wgt = np.where(iu[0] == iu[1], 1.0, 2.0)            # symmetric delta: (r,s) and (s,r)

    def fref(fa):
        return np.einsum("rs,mnrs->mn", fa, g1s)

    # constraints: F_MM - F_00 = 0 (M > 0) and F_MN = 0 (M < N), linear in the delta
    rows, rhs = [], []
    fa0 = p.f[c:c + a, c:c + a]
    F0 = fref(fa0)
    for M in range(1, n):
        rows.append((g1s[M, M] - g1s[0, 0])[iu] * wgt)
        rhs.append(-(F0[M, M] - F0[0, 0]))
    for M in range(n):
        for N in range(M + 1, n):
            rows.append(g1s[M, N][iu] * wgt)
            rhs.append(-F0[M, N])
    x, *_ = np.linalg.lstsq(np.array(rows), np.array(rhs), rcond=None)
    delta = np.zeros((a, a))
    delta[iu] = x
    delta = delta + np.triu(delta, 1).T
    q = copy.copy(p)
    q.f = p.f.copy()
    q.f[c:c + a, c:c + a] = fa0 + delta
    return q


def rotated_fock(p, seed=1):
    """f rotated inside the closed and inside the virtual space (off-diagonal
    closed-closed and virtual-virtual entries), and f with a closed-virtual coupling."""
    rng = np.random.default_rng(seed)
    Q = np.eye(p.nmo)
    for lo, hi in ((0, p.nclosed), (p.nclosed + p.nact, p.nmo)):
        q, _ = np.linalg.qr(rng.standard_normal((hi - lo, hi - lo)))
        Q[lo:hi, lo:hi] = q
    f_rot = Q.T @ p.f @ Q
    f_cpl = p.f.copy()
    i, b = 0, p.nclosed + p.nact
    f_cpl[i, b] = f_cpl[b, i] = 1e-3
    return np.ascontiguousarray(f_rot), np.ascontiguousarray(f_cpl)
