"""The closed-active, active-virtual and closed-virtual blocks of d2 (Sec. II.D: dbar2_xy =
sum_L <Psi_lambda_L|E_xy|Psi1_L> for x, y in different spaces), formed on the GPU through
the one-body couplings between classes (opt.dens_offdiag), against

  * the determinant-space brute force (O1), which forms <Psi_lambda_L|E_xy|Psi1_L> from
    explicit many-electron vectors and shares no algebra with the library: nact 4, 5 and
    6, XMS and MS, MS-MR and SS-SR, shifts 0 and 0.2, every element of d2;
  * the RDM-form oracle (oracle/o2_offdiag.py) at nact 8 with several closed and virtual
    orbitals (ragged reduction chunks, both pair sectors populated), every element.

The diagonal blocks do not change when the option is on (to the last bits of the atomic
scatter sums of d1)."""
import os

import numpy as np
import pytest

from synth import make_problem
from oracle import o1_determinant as o1

pytestmark = pytest.mark.gpu

PROBLEMS = {
    "c2a4v3n2": dict(nclosed=2, nact=4, nvirt=3, naux=24, nstate=2, seed=5),
    "c1a6v1n2": dict(nclosed=1, nact=6, nvirt=1, naux=20, nstate=2, seed=33),
    "c2a5v2n3": dict(nclosed=2, nact=5, nvirt=2, naux=24, nstate=3, seed=36, nelact=4),
}
OPTS = [dict(xms=x, scheme=s, shift=e) for x in (1, 0) for s in (0, 1) for e in (0.0, 0.2)]


@pytest.fixture(scope="module")
def cp():
    from paper_1606_01273_gb300 import build as b
    if not os.path.exists(b.LIB):
        b.build()
    import paper_1606_01273_gb300 as cp
    return cp


_cache = {}


def _problem(name, spec):
    if name not in _cache:
        _cache[name] = make_problem(**spec)
    return _cache[name]


def _sym(x):
    return 0.5 * (x + x.T)


def _blocks(p):
    c, a = p.nclosed, p.nact
    diag = np.zeros((p.nmo, p.nmo))
    diag[:c, :c] = diag[c:c + a, c:c + a] = diag[c + a:, c + a:] = 1.0
    return diag, 1.0 - diag


def _densities(cp, p, opt, offdiag):
    ctx = cp.Context(p.nclosed, p.nact, p.nvirt, p.naux, p.nstate, dens_offdiag=offdiag, **opt)
    try:
        ctx.set_inputs(*cp.problem_inputs(p))
        st = ctx.solve()
        assert st == cp.OK
        ctx.compute_densities()
        d1, d2, _ = ctx.get_densities(with_gdf=False)
    finally:
        ctx.close()
    return d1, d2


@pytest.mark.parametrize("name", list(PROBLEMS))
@pytest.mark.parametrize("opt", OPTS, ids=lambda o: f"xms{o['xms']}_sch{o['scheme']}_s{o['shift']}")
def test_offdiag_vs_brute_force(cp, name, opt):
    p = _problem(name, PROBLEMS[name])
    _, d2 = _densities(cp, p, opt, 1)
    ref = o1.solve_problem(p, xms=bool(opt["xms"]), scheme="sssr" if opt["scheme"] else "msmr",
                           shift=opt["shift"])
    want = _sym(ref.d2)
    scale = max(1.0, float(np.abs(want).max()))
    err = float(np.abs(d2 - want).max())
    assert err <= 1e-9 * scale, f"d2 max |diff| {err:.3e} (scale {scale:.3e})"
    _, off = _blocks(p)
    assert float(np.abs(want * off).max()) > 1e-6       # the blocks are populated


@pytest.mark.parametrize("opt", [dict(xms=1, scheme=0, shift=0.2), dict(xms=0, scheme=1, shift=0.0)],
                         ids=["xms_msmr", "ms_sssr"])
def test_offdiag_vs_rdm_oracle_nact8(cp, opt):
    from oracle import o2_rdm as o2
    from oracle import o2_classes as oc
    from oracle.o2_offdiag import offdiag_dbar2
    p = _problem("c3a8v5n2", dict(nclosed=3, nact=8, nvirt=5, naux=30, nstate=2, seed=12))
    d1_off, d2_off = _densities(cp, p, opt, 0)
    d1_on, d2_on = _densities(cp, p, opt, 1)
    diag, off = _blocks(p)
    # d1 carries atomic scatter sums (last bits vary run to run); d2's diagonal blocks do not
    # depend on the option
    assert float(np.abs(d1_on - d1_off).max()) <= 1e-12 * max(1.0, float(np.abs(d1_off).max()))
    assert float(np.abs((d2_on - d2_off) * diag).max()) <= 1e-12 * max(1.0, float(np.abs(d2_off).max()))
    assert float(np.abs(d2_off * off).max()) == 0.0
    scheme = "sssr" if opt["scheme"] else "msmr"
    st = o2.setup(p, xms=bool(opt["xms"]), kmax=4)
    mom = oc.all_moments(p, st, shift=opt["shift"], scheme=scheme)
    parts = {c: (-np.einsum("llk->lk", M1), np.diagonal(M2).copy())
             for c, (M1, M2, M3) in mom.items()}
    _, _, R = o2.heff(st, parts, opt["shift"])
    want = _sym(offdiag_dbar2(p, st, opt["shift"], scheme, R, 0))
    scale = max(1.0, float(np.abs(want).max()))
    err = float(np.abs(d2_on * off - want).max())
    assert err <= 1e-9 * scale, f"off-diagonal d2 max |diff| {err:.3e} (scale {scale:.3e})"
