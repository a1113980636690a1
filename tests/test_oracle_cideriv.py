"""Pins of the oracle's CI derivative and XMS response (Sec. II.D: Eq. cideriv, Eq.
cideriv2, Eq. xmseq, the XMS terms; oracle/o1_cideriv.py) against central finite
differences of the determinant-space energy.

The reference CI coefficients c are moved along a random direction (every determinant
and state, normalisation not kept: the Lagrangian is defined for any c), with h and the
DF factors fixed and f = h + g(d_sa(c)) following the references' state-averaged density;
O1 recomputes everything from the moved references.  Then
  * at fixed U (MS, and XMS with U held):     dE/de = sum delta . (ytil U^T)
  * XMS with U re-determined by the rotation:  dE/de = sum delta . ((ytil + ytil') U^T),
which pins w_MN (Eq. xmseq) and ytil';
  * orbital transformations with U re-determined: dE/de = sum K . (Y + Y').
A dropped term, a wrong sign of w or a missing d_sa chain shows up at the percent level."""
import numpy as np
import pytest

from synth import make_problem
from oracle import o1_determinant as o1
from oracle.o1_cideriv import ci_derivative, xms_response, total_orbital_derivative

STEP = 2e-4


@pytest.fixture(scope="module")
def prob():
    return make_problem(nclosed=2, nact=4, nvirt=2, naux=24, nstate=2, seed=5)


@pytest.fixture(scope="module")
def space(prob):
    return o1.FullSpace(prob.nmo, 2 * prob.nclosed + prob.nelact)


def _dsa(space, p, ci):
    ref = space.embed(p.nclosed, ci, p.det_alpha, p.det_beta)
    return sum(space.tdm1(ref[:, m], ref[:, m]) for m in range(ci.shape[1])) / ci.shape[1]


def _energy(p, space, h, ci, B, opt, U=None):
    eri = np.einsum("Ppq,Prs->pqrs", B, B)
    f = h + o1.g_matrix(eri, _dsa(space, p, ci))
    r = o1.solve(p.nclosed, p.nact, p.nvirt, p.nelact, f, B, ci, p.det_alpha, p.det_beta, h=h,
                 densities=False, space=space, U_fixed=U, **opt)
    return r.Ems[opt.get("target", 0)]


def _richardson(fun):
    def central(s):
        return (fun(s) - fun(-s)) / (2 * s)
    return (4.0 * central(STEP / 2) - central(STEP)) / 3.0


OPTS = [dict(xms=False, scheme="msmr", shift=0.2),
        dict(xms=True, scheme="msmr", shift=0.0),
        dict(xms=True, scheme="sssr", shift=0.2, target=1)]
IDS = ["ms_msmr_s0.2", "xms_msmr_s0", "xms_sssr_s0.2_P1"]


@pytest.mark.parametrize("opt", OPTS, ids=IDS)
def test_ci_derivative_at_fixed_rotation(prob, space, opt):
    p = prob
    base = o1.solve_problem(p, space=space, **opt)
    y = ci_derivative(p, base, opt["shift"], opt.get("target", 0)) @ base.U.T
    rng = np.random.default_rng(4)
    for _ in range(2):
        delta = rng.standard_normal(p.ci.shape)
        delta /= np.linalg.norm(delta)
        want = float(np.sum(delta * y))
        got = _richardson(lambda e: _energy(p, space, base.h, p.ci + e * delta, p.B, opt, U=base.U))
        assert abs(got - want) <= 1e-7 * max(1.0, abs(want)), (got, want)


@pytest.mark.parametrize("opt", OPTS[1:], ids=IDS[1:])
def test_total_ci_derivative_with_xms_response(prob, space, opt):
    p = prob
    base = o1.solve_problem(p, space=space, **opt)
    ytil, w, yp, dcheck, _ = xms_response(p, base, opt["shift"], opt.get("target", 0))
    assert np.abs(w).max() > 1e-6 and np.allclose(w, w.T)
    y_fixed = ytil @ base.U.T
    y_tot = (ytil + yp) @ base.U.T
    rng = np.random.default_rng(6)
    for _ in range(2):
        delta = rng.standard_normal(p.ci.shape)
        delta /= np.linalg.norm(delta)
        want = float(np.sum(delta * y_tot))
        got = _richardson(lambda e: _energy(p, space, base.h, p.ci + e * delta, p.B, opt))
        assert abs(got - want) <= 1e-7 * max(1.0, abs(want)), (got, want)
        # the XMS response is not negligible along these directions
        assert abs(float(np.sum(delta * (y_tot - y_fixed)))) > 1e-5


@pytest.mark.parametrize("opt", OPTS[1:], ids=IDS[1:])
def test_total_orbital_derivative_with_xms_response(prob, space, opt):
    p = prob
    base = o1.solve_problem(p, space=space, **opt)
    Y = total_orbital_derivative(p, base, opt["shift"], opt.get("target", 0), xms=True)
    rng = np.random.default_rng(8)
    for _ in range(2):
        K = rng.standard_normal((p.nmo, p.nmo))

        def fun(e):
            C = np.eye(p.nmo) + e * K
            B = np.einsum("xp,Pxy,yq->Ppq", C, p.B, C)
            return _energy(p, space, C.T @ base.h @ C, p.ci, B, opt)
        want = float(np.sum(K * Y))
        got = _richardson(fun)
        assert abs(got - want) <= 1e-7 * max(1.0, abs(want)), (got, want)
