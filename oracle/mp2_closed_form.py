"""Closed-shell MP2 in canonical orbitals -- the nact = 0 special case of the method.

TEST INFRASTRUCTURE (see oracle/__init__.py).  With no active orbitals only the
E_ai,bj family of Eq. (class) survives, the reference is the closed-shell
determinant and the first-order equations reduce to the textbook pair
amplitudes t_ij^ab = -(ai|bj) / (e_a + e_b - e_i - e_j + E_s).  The energy is
<Psi1|H|0> - E_s <Psi1|Psi1> (effective Hamiltonian with the shift correction,
Sec. II.B), which in closed form is

  E2 = -sum_ijab K(2K - K') [1/(D + E_s) + E_s/(D + E_s)^2],
  K = (ai|bj), K' = (aj|bi), D = e_a + e_b - e_i - e_j.
"""
import numpy as np


def mp2_energy(eps_closed: np.ndarray, eps_virt: np.ndarray, Kiajb: np.ndarray, shift: float = 0.0):
    """Kiajb[i, a, j, b] = (ai|bj) over closed i, j and virtual a, b."""
    d = (eps_virt[None, :, None, None] + eps_virt[None, None, None, :]
         - eps_closed[:, None, None, None] - eps_closed[None, None, :, None])
    kx = Kiajb.transpose(0, 3, 2, 1)  # (aj|bi) placed at [i, a, j, b]
    num = Kiajb * (2.0 * Kiajb - kx)
    return float(-np.sum(num * (1.0 / (d + shift) + shift / (d + shift) ** 2)))
