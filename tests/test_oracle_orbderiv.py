"""Pin of the oracle's orbital derivative Y (Sec. II.D, Eq. orbderiv; oracle/o1_orbderiv.py)
against central finite differences of the determinant-space energy.

The orbitals are transformed by C = 1 + e K (K a random general matrix, so that the
symmetric and the antisymmetric part of Y are both checked); h and the DF factors follow
the orbitals (h' = C^T h C, B'_P = C^T B_P C), f' = h' + g(d_sa) with the state-averaged
density of the fixed reference CI vectors, and the energy is recomputed from scratch by
o1_determinant with a general (non-block-diagonal) f'.  For XMS the rotation U is held
at its unperturbed value (Y is the derivative at fixed rotated reference states; the
XMS response enters through w_MN, which is not part of Y).  dE/de must equal
sum_xy K_xy Y_xy."""
import numpy as np
import pytest

from synth import make_problem
from oracle import o1_determinant as o1
from oracle.o1_orbderiv import orbital_derivative

STEP = 2e-4


@pytest.fixture(scope="module")
def prob():
    return make_problem(nclosed=2, nact=4, nvirt=2, naux=24, nstate=2, seed=5)


def _energy(p, base, K, e, U, opt):
    C = np.eye(p.nmo) + e * K
    h = C.T @ base.h @ C
    B = np.einsum("xp,Pxy,yq->Ppq", C, p.B, C)
    eri = np.einsum("Ppq,Prs->pqrs", B, B)
    f = h + o1.g_matrix(eri, base.d_sa)
    r = o1.solve(p.nclosed, p.nact, p.nvirt, p.nelact, f, B, p.ci, p.det_alpha, p.det_beta,
                 h=h, densities=False, U_fixed=U, **opt)
    return r.Ems[opt.get("target", 0)]


def _fd(p, base, K, U, opt):
    """Central differences at steps h and h/2, Richardson-combined (error O(h^4))."""
    def central(s):
        return (_energy(p, base, K, s, U, opt) - _energy(p, base, K, -s, U, opt)) / (2 * s)
    return (4.0 * central(STEP / 2) - central(STEP)) / 3.0


@pytest.mark.parametrize("opt", [dict(xms=False, scheme="msmr", shift=0.2),
                                 dict(xms=True, scheme="msmr", shift=0.0),
                                 dict(xms=True, scheme="sssr", shift=0.2, target=1)],
                         ids=["ms_msmr_s0.2", "xms_msmr_s0", "xms_sssr_s0.2_P1"])
def test_orbital_derivative_matches_finite_differences(prob, opt):
    p = prob
    base = o1.solve_problem(p, **opt)
    Y = orbital_derivative(base, p.B)
    assert np.abs(Y - Y.T).max() > 1e-4         # not symmetric: the orbital gradient is nonzero
    rng = np.random.default_rng(11)
    for _ in range(2):
        K = rng.standard_normal((p.nmo, p.nmo))
        want = float(np.sum(K * Y))
        got = _fd(p, base, K, base.U, opt)
        assert abs(got - want) <= 1e-7 * max(1.0, abs(want)), (got, want)


def test_orbital_derivative_mixes_every_block(prob):
    """Rotations between the closed, active and virtual spaces move the energy (the
    inter-space blocks of Y are populated), so the check above is not blind to them."""
    p = prob
    base = o1.solve_problem(p, xms=False, shift=0.2)
    Y = orbital_derivative(base, p.B)
    c, a = p.nclosed, p.nact
    sl = (slice(0, c), slice(c, c + a), slice(c + a, p.nmo))
    for i in range(3):
        for j in range(3):
            assert np.abs(Y[sl[i], sl[j]]).max() > 1e-6, (i, j)
