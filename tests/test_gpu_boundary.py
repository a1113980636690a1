"""The C-ABI contract at its edges: the Fock matrices the solve refuses (coupling between
the closed, active and virtual spaces, which the one-step class solve would drop), the
degenerate-XMS warning, and
N_L through caspt2_get_densities, each against the determinant-space brute force."""
import os

import numpy as np
import pytest

from synth import make_problem
from oracle import o1_determinant as o1
from tests.cases import degenerate_xms_problem, rotated_fock

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cp():
    from paper_1606_01273_gb300 import build as b
    if not os.path.exists(b.LIB):
        b.build()
    import paper_1606_01273_gb300 as cp
    return cp


@pytest.fixture(scope="module")
def small():
    return make_problem(2, 4, 2, 24, 2, seed=5)


@pytest.mark.parametrize("device", [False, True], ids=["host", "device"])
def test_coupled_fock_is_refused(cp, small, device):
    """An f with one closed-virtual coupling entry is refused with EINVAL (host and device
    inputs); the block-diagonal f and a closed/virtual-rotated f (solved through the
    canonical orbitals of those blocks) are accepted."""
    import torch
    p = small
    f_rot, f_cpl = rotated_fock(p)
    _, B, *rd = cp.problem_inputs(p)
    ctx = cp.Context(p.nclosed, p.nact, p.nvirt, p.naux, p.nstate)
    try:
        for f in (f_cpl, f_rot, f_cpl, p.f):
            args = [f, B, *rd]
            if device:
                args = [None if x is None else torch.from_numpy(np.ascontiguousarray(x)).cuda()
                        for x in args]
            if f is p.f or f is f_rot:
                ctx.set_inputs(*args)
            else:
                with pytest.raises(cp.CASPT2Error) as e:
                    ctx.set_inputs(*args)
                assert e.value.status == cp.EINVAL
                # the context keeps no inputs after a refusal
                assert cp.lib().caspt2_solve(ctx._h, None) == cp.ESTATE
        assert ctx.solve() in (cp.OK, cp.WINTRUDER)
    finally:
        ctx.close()


def test_degenerate_xms_warns_and_matches_brute_force(cp, small):
    """Degenerate XMS zeroth-order energies: the solve returns WDEGEN, get_status carries
    the warning and the gap, and the energies (shift 0: independent of the rotation
    chosen inside the pair) equal the brute force's."""
    p = degenerate_xms_problem(small)
    ctx = cp.Context(p.nclosed, p.nact, p.nvirt, p.naux, p.nstate, xms=1, shift=0.0)
    try:
        ctx.set_inputs(*cp.problem_inputs(p))
        st = ctx.solve()
        r = ctx.result(st)
        s = ctx.status()
    finally:
        ctx.close()
    assert st == cp.WDEGEN
    assert s["warnings"] & cp.WARN_DEGEN and s["min_e0_gap"] < 1e-8
    ref = o1.solve_problem(p, shift=0.0, densities=False)
    assert np.abs(r.Ems - ref.Ems).max() <= 1e-8
    # a non-degenerate problem carries no such warning
    ctx = cp.Context(small.nclosed, small.nact, small.nvirt, small.naux, small.nstate, xms=1)
    try:
        ctx.set_inputs(*cp.problem_inputs(small))
        assert ctx.solve() == cp.OK
        assert ctx.status()["warnings"] == 0 and ctx.status()["min_e0_gap"] > 1e-3
    finally:
        ctx.close()


@pytest.mark.parametrize("opt", [dict(xms=1, scheme=0, shift=0.2), dict(xms=0, scheme=1, shift=0.1)],
                         ids=["xms_msmr", "ms_sssr"])
def test_NL_matches_brute_force(cp, small, opt):
    """N_L = sum_MN <M~|lambda_LM^dag T_LN|N~> (Sec. II.D) from caspt2_get_densities
    equals the determinant-space value and the sum of the per-class shares."""
    p = small
    ctx = cp.Context(p.nclosed, p.nact, p.nvirt, p.naux, p.nstate, **opt)
    try:
        ctx.set_inputs(*cp.problem_inputs(p))
        st = ctx.solve()
        r = ctx.result(st)
        ctx.compute_densities()
        *_, nl = ctx.get_densities(with_gdf=False, with_nl=True)
    finally:
        ctx.close()
    sch = "sssr" if opt["scheme"] == 1 else "msmr"
    ref = o1.solve_problem(p, xms=bool(opt["xms"]), scheme=sch, shift=opt["shift"])
    scale = max(1e-12, np.abs(ref.NL).max())
    assert np.abs(nl - ref.NL).max() <= 1e-9 * scale
    assert np.abs(nl - sum(r.lam_NL.values())).max() <= 1e-13 * scale
