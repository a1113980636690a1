"""Iterative solution of the amplitude equation with coupling between the classes (Sec. II.B:
for an f with closed-active, active-virtual or closed-virtual entries, or with non-diagonal
closed/virtual blocks, the equation is solved by subspace residual minimisation with a
preconditioner), in the orthonormal range basis of o1_determinant.

TEST INFRASTRUCTURE (see oracle/__init__.py).

For state L, with X the per-class orthonormal basis of range(S) (overlap eigenvalues below
the threshold dropped) and g = X^T b_L the source in that basis, the equation is
    A y = -g,   A = X^T F X - (E0_L - E_s) 1,   t = X y.
The preconditioner M is the part of A inside each class (the couplings between classes
dropped), applied exactly: for an f without coupling between the spaces M = A and the
first step is the exact one-step solution.  Each iteration adds the preconditioned
residual -M^-1 r to the subspace (orthonormalised against it) and takes the y of the
subspace that minimises ||A y + g||.  A start vector y0 (a warm start from a nearby
problem) replaces zero.
"""
from __future__ import annotations

import numpy as np


def block_preconditioner(A: np.ndarray, cls: list):
    """M^-1 as a callable: the class-diagonal blocks of A, each solved exactly."""
    labels = np.array(cls)
    blocks = []
    for c in dict.fromkeys(cls):
        idx = np.nonzero(labels == c)[0]
        blocks.append((idx, np.linalg.inv(A[np.ix_(idx, idx)])))

    def apply(r):
        z = np.zeros_like(r)
        for idx, inv in blocks:
            z[idx] = inv @ r[idx]
        return z
    return apply


def residual_minimisation(A, g, precond, y0=None, tol=1e-12, max_iter=200):
    """Solve A y = -g; returns (y, iterations, residual norms relative to ||g||)."""
    y0 = np.zeros_like(g) if y0 is None else np.array(y0, dtype=float)
    gn = max(float(np.linalg.norm(g)), 1e-300)
    r = A @ y0 + g
    hist = [float(np.linalg.norm(r)) / gn]
    W = np.zeros((len(g), 0))
    AW = np.zeros((len(g), 0))
    y = y0
    it = 0
    while hist[-1] > tol and it < max_iter:
        z = -precond(r)
        for _ in range(2):                                   # Gram-Schmidt twice
            z = z - W @ (W.T @ z)
        nz = float(np.linalg.norm(z))
        if nz == 0.0:
            break
        z /= nz
        W = np.column_stack([W, z])
        AW = np.column_stack([AW, A @ z])
        rhs = -(A @ y0 + g)
        c, *_ = np.linalg.lstsq(AW, rhs, rcond=None)
        y = y0 + W @ c
        r = A @ y + g
        hist.append(float(np.linalg.norm(r)) / gn)
        it += 1
    return y, it, hist


def solve_state(res, L, y0=None, tol=1e-12):
    """t_L = X y of an O1Result by the iterative solve (with its iteration count)."""
    A, X, cls = res.A[L], res.X[L], res.Xcls[L]
    g = X.T @ res.b_src[L][L]
    y, it, hist = residual_minimisation(A, g, block_preconditioner(A, cls), y0, tol)
    return X @ y, y, it, hist
