"""Orbital derivative Y_xy = dL/dkappa_xy (Sec. II.D, Eq. orbderiv; the orbital part of the
Z-vector source) from caspt2_orbital_derivative against the determinant-space oracle
(oracle/o1_orbderiv.py: Y from O1's explicit densities, itself pinned against central
finite differences of the O1 energy under orbital transformations that carry h, B and f).

Every element of Y, at nact 4, 5 and 6, XMS (at fixed rotated states) and MS, MS-MR and
SS-SR, shifts 0 and 0.2.  The library forms Y in the density-fitted form 2 [h G +
sum_Q B_Q Gb_Q]; the oracle sums the first-order change of L over every index of h and of
the four-index integrals, so the two share no arithmetic beyond the definition."""
import os

import numpy as np
import pytest

from synth import make_problem
from oracle import o1_determinant as o1
from oracle.o1_orbderiv import orbital_derivative

pytestmark = pytest.mark.gpu

PROBLEMS = {
    "c2a4v3n2": dict(nclosed=2, nact=4, nvirt=3, naux=24, nstate=2, seed=5),
    "c1a6v1n2": dict(nclosed=1, nact=6, nvirt=1, naux=20, nstate=2, seed=33),
    "c2a5v2n3": dict(nclosed=2, nact=5, nvirt=2, naux=24, nstate=3, seed=36, nelact=4),
}
OPTS = [dict(xms=x, scheme=s, shift=e) for x in (1, 0) for s in (0, 1) for e in (0.0, 0.2)]
RTOL = 1e-9


@pytest.fixture(scope="module")
def cp():
    from paper_1606_01273_gb300 import build as b
    if not os.path.exists(b.LIB):
        b.build()
    import paper_1606_01273_gb300 as cp
    return cp


_cache = {}


def _problem(name):
    if name not in _cache:
        _cache[name] = make_problem(**PROBLEMS[name])
    return _cache[name]


def _gpu_y(cp, p, opt, calls=1, offdiag=1):
    ctx = cp.Context(p.nclosed, p.nact, p.nvirt, p.naux, p.nstate, dens_offdiag=offdiag, **opt)
    try:
        ctx.set_inputs(*cp.problem_inputs(p))
        assert ctx.solve() == cp.OK
        return [ctx.orbital_derivative() for _ in range(calls)]
    finally:
        ctx.close()


@pytest.mark.parametrize("name", list(PROBLEMS))
@pytest.mark.parametrize("opt", OPTS, ids=lambda o: f"xms{o['xms']}_sch{o['scheme']}_s{o['shift']}")
def test_orbital_derivative_vs_brute_force(cp, name, opt):
    p = _problem(name)
    (Y,) = _gpu_y(cp, p, opt)
    ref = o1.solve_problem(p, xms=bool(opt["xms"]), scheme="sssr" if opt["scheme"] else "msmr",
                           shift=opt["shift"])
    want = orbital_derivative(ref, p.B)
    scale = max(1.0, float(np.abs(want).max()))
    err = float(np.abs(Y - want).max())
    assert err <= RTOL * scale, f"Y max |diff| {err:.3e} (scale {scale:.3e})"
    # the orbital gradient (antisymmetric part) is populated, not only the symmetric part
    assert float(np.abs(want - want.T).max()) > 1e-4


# more DF factors than the 32 partial products of sum_Q B_Q Gb_Q (chunks of two, one
# left over), and no active orbitals (class H alone; no inter-space blocks of d2 exist, so
# the off-diagonal density option is not needed)
EXTRA = {
    "c2a4v3x37n2": (dict(nclosed=2, nact=4, nvirt=3, naux=37, nstate=2, seed=5), 1),
    "c3a0v4x30n1": (dict(nclosed=3, nact=0, nvirt=4, naux=30, nstate=1, seed=3), 0),
}


@pytest.mark.parametrize("name", list(EXTRA))
@pytest.mark.parametrize("opt", [dict(xms=1, scheme=0, shift=0.2), dict(xms=0, scheme=1, shift=0.0)],
                         ids=["xms_msmr_s0.2", "ms_sssr_s0"])
def test_orbital_derivative_chunks_and_no_active(cp, name, opt):
    spec, offdiag = EXTRA[name]
    if name not in _cache:
        _cache[name] = make_problem(**spec)
    p = _cache[name]
    (Y,) = _gpu_y(cp, p, opt, offdiag=offdiag)
    ref = o1.solve_problem(p, xms=bool(opt["xms"]), scheme="sssr" if opt["scheme"] else "msmr",
                           shift=opt["shift"])
    want = orbital_derivative(ref, p.B)
    scale = max(1.0, float(np.abs(want).max()))
    err = float(np.abs(Y - want).max())
    assert err <= RTOL * scale, f"Y max |diff| {err:.3e} (scale {scale:.3e})"


def test_orbital_derivative_contract(cp):
    """Two calls in a row give the same Y (the densities are recomputed each time, up to
    the last bits of their atomic scatter sums); without the inter-space blocks of d2
    (dens_offdiag off) the call is refused."""
    p = _problem("c2a4v3n2")
    opt = dict(xms=1, scheme=0, shift=0.2)
    Y1, Y2 = _gpu_y(cp, p, opt, calls=2)
    assert float(np.abs(Y1 - Y2).max()) <= 1e-12 * max(1.0, float(np.abs(Y1).max()))
    ctx = cp.Context(p.nclosed, p.nact, p.nvirt, p.naux, p.nstate, **opt)
    try:
        ctx.set_inputs(*cp.problem_inputs(p))
        assert ctx.solve() == cp.OK
        with pytest.raises(cp.CASPT2Error) as e:
            ctx.orbital_derivative()
        assert e.value.status == cp.EINVAL
    finally:
        ctx.close()
