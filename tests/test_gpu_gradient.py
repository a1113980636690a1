"""Differentiation form: dE_MS/df and dE_MS/dB of the target state (MS, reference RDMs
fixed) from caspt2_gradient and through torch.autograd, checked against central finite
differences of the library's own energies in random symmetric directions (for f, on the
closed and virtual diagonals and the active block; directions with off-diagonal closed or
virtual entries, which the library solves through canonical orbitals, are checked in
test_gpu_canonical.py) and, on the closed-closed, active-active and virtual-virtual
blocks, against the determinant-space oracle's densities."""
import os

import numpy as np
import pytest

from synth import make_problem
from oracle import o1_determinant as o1

pytestmark = pytest.mark.gpu

CASES = [dict(nclosed=2, nact=4, nvirt=2, naux=24, nstate=2, seed=5),
         dict(nclosed=3, nact=3, nvirt=10, naux=30, nstate=2, seed=41, nelact=2)]
STEP = 2e-4


@pytest.fixture(scope="module")
def cp():
    from paper_1606_01273_gb300 import build as b
    if not os.path.exists(b.LIB):
        b.build()
    import paper_1606_01273_gb300 as cp
    return cp


def _fd(cp, p, opt, df=None, dB=None):
    """Central difference of E along (df, dB), Richardson-extrapolated over steps h and
    h/2 so that the truncation error is O(h^4)."""
    def central(h):
        ep = _energy(cp, p, p.f + h * df if df is not None else p.f,
                     p.B + h * dB if dB is not None else p.B, opt)
        em = _energy(cp, p, p.f - h * df if df is not None else p.f,
                     p.B - h * dB if dB is not None else p.B, opt)
        return (ep - em) / (2 * h)
    return (4.0 * central(STEP / 2) - central(STEP)) / 3.0


def _read_mask(p):
    c, a = p.nclosed, p.nact
    m = np.eye(p.nmo)
    m[c:c + a, c:c + a] = 1.0
    return m


def _energy(cp, p, f, B, opt):
    ctx = cp.Context(p.nclosed, p.nact, p.nvirt, p.naux, p.nstate, **opt)
    try:
        _, _, *rd = cp.problem_inputs(p)
        ctx.set_inputs(np.ascontiguousarray(f), np.ascontiguousarray(B), *rd)
        st = ctx.solve()
        return ctx.result(st).Ems[opt.get("target_state", 0)]
    finally:
        ctx.close()


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("opt", [dict(xms=0, scheme=0, shift=0.2), dict(xms=0, scheme=1, shift=0.1),
                                 dict(xms=0, scheme=0, shift=0.0, target_state=1)],
                         ids=["msmr", "sssr", "msmr_P1"])
def test_gradient_matches_finite_differences(cp, case, opt):
    p = make_problem(**CASES[case])
    ctx = cp.Context(p.nclosed, p.nact, p.nvirt, p.naux, p.nstate, **opt)
    try:
        ctx.set_inputs(*cp.problem_inputs(p))
        ctx.solve()
        gf, gB = ctx.gradient()
    finally:
        ctx.close()
    rng = np.random.default_rng(case * 10 + opt.get("target_state", 0) + 7 * opt["scheme"])
    for _ in range(2):
        # directions on the closed and virtual diagonals and the active block (a direction
        # with a closed-active, active-virtual or closed-virtual entry makes f one that
        # caspt2_set_inputs refuses)
        df = rng.standard_normal(p.f.shape)
        df = df + df.T
        df *= _read_mask(p)
        df /= np.linalg.norm(df)
        fd = _fd(cp, p, opt, df=df)
        an = np.sum(gf * df)
        assert abs(fd - an) <= 1e-6 * abs(an) + 1e-8, ("f", fd, an)
        dB = rng.standard_normal(p.B.shape)
        dB = dB + dB.transpose(0, 2, 1)
        dB /= np.linalg.norm(dB)
        fd = _fd(cp, p, opt, dB=dB)
        an = np.sum(gB * dB)
        assert abs(fd - an) <= 1e-6 * abs(an) + 1e-8, ("B", fd, an)


def test_gradient_vs_determinant_oracle(cp):
    """On the closed-closed, active-active and virtual-virtual blocks of f (the blocks of
    an f the library takes; off-diagonal closed/virtual entries are solved through the
    canonical orbitals), dE/df = gamma_P + d(1) + d(2) of the brute-force oracle
    (h = f - g(B, d_sa) is held consistent through d(1))."""
    p = make_problem(**CASES[0])
    opt = dict(xms=0, scheme=0, shift=0.2)
    ctx = cp.Context(p.nclosed, p.nact, p.nvirt, p.naux, p.nstate, **opt)
    try:
        ctx.set_inputs(*cp.problem_inputs(p))
        ctx.solve()
        gf, _ = ctx.gradient()
    finally:
        ctx.close()
    r = o1.solve_problem(p, xms=False, scheme="msmr", shift=0.2)
    ref = r.gammaP + r.d1 + r.d2
    ref = 0.5 * (ref + ref.T)
    c, a = p.nclosed, p.nact
    mask = np.zeros_like(gf, dtype=bool)
    mask[:c, :c] = mask[c:c + a, c:c + a] = mask[c + a:, c + a:] = True
    assert np.abs((gf - ref)[mask]).max() <= 1e-9 * max(1.0, np.abs(ref).max())


def test_autograd_function(cp):
    """torch.autograd through ms_energy gives caspt2_gradient's dE/df and dE/dB."""
    import torch
    p = make_problem(**CASES[1])
    dev = torch.device("cuda", 0)
    f, B, *rd = (None if x is None else torch.from_numpy(x).to(dev) for x in cp.problem_inputs(p))
    f.requires_grad_(True)
    B.requires_grad_(True)
    e = cp.ms_energy(f, B, rd, p.nclosed, target_state=0, scheme=0, shift=0.2)
    gf, gB = torch.autograd.grad(e, (f, B))
    ctx = cp.Context(p.nclosed, p.nact, p.nvirt, p.naux, p.nstate, xms=0, scheme=0, shift=0.2)
    try:
        ctx.set_inputs(*cp.problem_inputs(p))
        ctx.solve()
        rf, rB = ctx.gradient()
    finally:
        ctx.close()
    assert np.abs(gf.cpu().numpy() - rf).max() <= 1e-12 * max(1.0, np.abs(rf).max())
    assert np.abs(gB.cpu().numpy() - rB).max() <= 1e-12 * max(1.0, np.abs(rB).max())
