"""The oracle's iterative amplitude solve for coupled Fock matrices (Sec. II.B, subspace
residual minimisation with the class-diagonal preconditioner; oracle/o1_iterative.py)
against the determinant-space direct solve of the same coupled equations: the same
amplitudes for an f with closed-active, active-virtual and closed-virtual entries (MS-MR
and SS-SR), one step when f has no such coupling (the preconditioner is then the whole
operator: the one-step class solve), and a warm start from a nearby problem's solution
needs fewer steps than a start from zero."""
import numpy as np
import pytest

from synth import make_problem
from oracle import o1_determinant as o1
from oracle.o1_iterative import solve_state


@pytest.fixture(scope="module")
def prob():
    return make_problem(nclosed=2, nact=4, nvirt=2, naux=24, nstate=2, seed=5)


def _coupling(p, seed=3):
    rng = np.random.default_rng(seed)
    sp = np.array([0] * p.nclosed + [1] * p.nact + [2] * p.nvirt)
    K = rng.standard_normal((p.nmo, p.nmo))
    K = 0.5 * (K + K.T)
    K[sp[:, None] == sp[None, :]] = 0.0             # only the blocks between the spaces
    return K


def test_uncoupled_f_is_one_step(prob):
    r = o1.solve_problem(prob, xms=True, shift=0.2, densities=False)
    for L in range(prob.nstate):
        t, _, it, _ = solve_state(r, L)
        assert it == 1
        assert np.abs(t - r.t[L]).max() <= 1e-12 * np.abs(r.t[L]).max()


@pytest.mark.parametrize("scheme", ["msmr", "sssr"])
def test_coupled_f_matches_direct_solve(prob, scheme):
    f = prob.f + 0.05 * _coupling(prob)
    r = o1.solve_problem(prob, f=f, xms=True, scheme=scheme, shift=0.2, densities=False)
    for L in range(prob.nstate):
        t, _, it, hist = solve_state(r, L)
        assert it > 1 and hist[-1] <= 1e-12
        assert np.abs(t - r.t[L]).max() <= 1e-10 * np.abs(r.t[L]).max()


def test_warm_start_takes_fewer_steps(prob):
    K = _coupling(prob)
    r1 = o1.solve_problem(prob, f=prob.f + 0.05 * K, xms=False, shift=0.2, densities=False)
    r2 = o1.solve_problem(prob, f=prob.f + 0.051 * K, xms=False, shift=0.2, densities=False)
    for L in range(prob.nstate):
        _, y1, _, _ = solve_state(r1, L)
        t_cold, _, it_cold, _ = solve_state(r2, L)
        t_warm, _, it_warm, _ = solve_state(r2, L, y0=y1)
        assert it_warm < it_cold
        assert np.abs(t_warm - t_cold).max() <= 1e-10 * np.abs(t_cold).max()
