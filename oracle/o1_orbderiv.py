"""Orbital derivative Y_xy of the CASPT2 Lagrangian (Sec. II.D, Eq. orbderiv) from the
determinant-space densities of o1_determinant.

TEST INFRASTRUCTURE (see oracle/__init__.py).

Definition used here.  The orbitals are transformed as phi'_y = phi_y + sum_x phi_x k_xy
(C = 1 + k, k a general matrix; the unitary generator of Eq. orbderiv is its
antisymmetric part), the reference CI vectors and the XMS rotation U are held fixed,
and every integral follows the orbitals:
    h' = C^T h C,   (pq|rs)' = sum C_xp C_yq C_zr C_ws (xy|zw),   f' = h' + g(d_sa)'
with d_sa the state-averaged density of the fixed reference states.  Then
    Y_xy = dL_PT2 / dk_xy   at k = 0,
and the orbital gradient along an antisymmetric generator is Y_xy - Y_yx.

L_PT2 depends on
  * h through H (the reference part <P|E_xy|P> and the first-order part d1);
  * f through the zeroth-order operator f^ (d2 = dL/df, every block);
  * (pq|rs) through H (1/2 <P|E_pq,rs|P> + 1/2 D1) and through f = h + g((pq|rs), d_sa).
With G = dL/dh|_(pq|rs) and W = dL/d(pq|rs)|_h written out from those densities, the
first-order change of L under the transformation is a sum over every index that the
transformation touches: two for h, four for (pq|rs).  Nothing here is blocked or
reordered beyond that sum.
"""
from __future__ import annotations

import numpy as np


def lagrangian_partials(res, eri: np.ndarray):
    """G[x][y] = dL/dh_xy and W[p][q][r][s] = dL/d(pq|rs) at fixed h (entries taken as
    independent), from an O1Result computed with densities."""
    dsa = res.d_sa
    G = res.gammaP + res.d1 + res.d2
    # g(d)_xy = sum_zw (xy|zw) d_zw - 1/4 sum_zw (xw|zy)(d_zw + d_wz)  (o1_determinant.g_matrix)
    W = 0.5 * (res.Gamma2P + res.D1)
    W = W + np.einsum("pq,rs->pqrs", res.d2, dsa)
    W = W - 0.25 * np.einsum("ps,rq->pqrs", res.d2, dsa + dsa.T)
    return G, W


def orbital_derivative(res, B: np.ndarray) -> np.ndarray:
    """Y[x][y] = dL_PT2/dk_xy (module docstring) for an O1Result with densities, whose
    problem had the DF factors B[P][p][q]."""
    eri = np.einsum("Ppq,Prs->pqrs", B, B)
    h = res.h
    G, W = lagrangian_partials(res, eri)
    # h'_pq = h_pq + sum_t (k_tp h_tq + h_pt k_tq)
    Y = h @ G.T + h.T @ G
    # (pq|rs)' = (pq|rs) + sum_t (k_tp (tq|rs) + k_tq (pt|rs) + k_tr (pq|ts) + k_ts (pq|rt))
    Y = Y + np.einsum("pqrs,tqrs->tp", W, eri)
    Y = Y + np.einsum("qprs,qtrs->tp", W, eri)
    Y = Y + np.einsum("qrps,qrts->tp", W, eri)
    Y = Y + np.einsum("qrsp,qrst->tp", W, eri)
    return Y
