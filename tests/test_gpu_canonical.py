"""Fock matrices whose closed-closed or virtual-virtual block is not diagonal (orbitals that
are not canonical, Sec. II.A/II.B), which caspt2_set_inputs solves through the canonical
orbitals of those blocks:

  * orbital-rotation invariance on the GPU: f and B rotated together inside the closed and
    inside the virtual space give the same energies as the unrotated inputs, and the
    densities and the gradient come back rotated the same way (the caller's basis), with
    both eigensolver paths (Jacobi for blocks up to 32, the tridiagonal method above);
  * f alone rotated (a different, non-canonical problem) against the determinant-space
    oracle, which solves the coupled amplitude equations of that f directly;
  * dE/df along directions with off-diagonal closed and virtual entries against central
    finite differences of the library's energies;
  * an f with coupling between the spaces is still refused, and the amplitude getters
    refuse canonicalised inputs."""
import os

import numpy as np
import pytest

from synth import make_problem
from oracle import o1_determinant as o1
from tests.cases import rotated_fock

pytestmark = pytest.mark.gpu

SMALL = dict(nclosed=2, nact=4, nvirt=3, naux=24, nstate=2, seed=5)
WIDE = dict(nclosed=4, nact=3, nvirt=40, naux=60, nstate=2, seed=1, nelact=2)
OPTS = [dict(xms=1, scheme=0, shift=0.2), dict(xms=0, scheme=1, shift=0.1)]


@pytest.fixture(scope="module")
def cp():
    from paper_1606_01273_gb300 import build as b
    if not os.path.exists(b.LIB):
        b.build()
    import paper_1606_01273_gb300 as cp
    return cp


_cache = {}


def _problem(spec):
    key = tuple(sorted(spec.items()))
    if key not in _cache:
        _cache[key] = make_problem(**spec)
    return _cache[key]


def _space_rotation(p, seed):
    rng = np.random.default_rng(seed)
    Q = np.eye(p.nmo)
    for lo, hi in ((0, p.nclosed), (p.nclosed + p.nact, p.nmo)):
        q, _ = np.linalg.qr(rng.standard_normal((hi - lo, hi - lo)))
        Q[lo:hi, lo:hi] = q
    return Q


def _run(cp, p, f, B, opt, grad=False):
    ctx = cp.Context(p.nclosed, p.nact, p.nvirt, p.naux, p.nstate, **opt)
    try:
        _, _, *rd = cp.problem_inputs(p)
        ctx.set_inputs(np.ascontiguousarray(f), np.ascontiguousarray(B), *rd)
        st = ctx.solve()
        assert st in (cp.OK, cp.WINTRUDER)
        r = ctx.result(st)
        ctx.compute_densities()
        r.d1, r.d2, r.gdf = ctx.get_densities()
        if grad:
            r.gf, r.gB = ctx.gradient()
        return r
    finally:
        ctx.close()


def _close(got, ref, rtol, what):
    scale = max(1.0, float(np.abs(ref).max()))
    err = float(np.abs(got - ref).max())
    assert err <= rtol * scale, f"{what}: max |diff| {err:.3e} (scale {scale:.3e})"


@pytest.mark.parametrize("spec", [SMALL, WIDE], ids=["c2a4v3", "c4a3v40"])
@pytest.mark.parametrize("opt", OPTS, ids=["xms_msmr_s0.2", "ms_sssr_s0.1"])
def test_orbital_rotation_invariance(cp, spec, opt):
    p = _problem(spec)
    Q = _space_rotation(p, 7)
    f_in = Q.T @ p.f @ Q
    B_in = np.einsum("xp,Pxy,yq->Ppq", Q, p.B, Q)
    want = _run(cp, p, p.f, p.B, dict(opt, target_state=0), grad=opt["xms"] == 0)
    got = _run(cp, p, f_in, B_in, dict(opt, target_state=0), grad=opt["xms"] == 0)
    assert np.abs(got.Ems - want.Ems).max() <= 1e-10
    assert np.abs(got.Heff - want.Heff).max() <= 1e-10
    for cls in "ABCDEFGH":
        _close(got.e_class[cls], want.e_class[cls], 1e-11, f"{cls} e")
    # derivatives with respect to f, h and B_P in the caller's basis: Q^T M Q
    _close(got.d1, Q.T @ want.d1 @ Q, 1e-10, "d1")
    _close(got.d2, Q.T @ want.d2 @ Q, 1e-10, "d2")
    _close(got.gdf, np.einsum("xp,Pxy,yq->Ppq", Q, want.gdf, Q), 1e-10, "GDF")
    if opt["xms"] == 0:
        _close(got.gf, Q.T @ want.gf @ Q, 1e-10, "dE/df")
        _close(got.gB, np.einsum("xp,Pxy,yq->Ppq", Q, want.gB, Q), 1e-10, "dE/dB")


@pytest.mark.parametrize("opt", OPTS + [dict(xms=0, scheme=0, shift=0.2)],
                         ids=["xms_msmr_s0.2", "ms_sssr_s0.1", "ms_msmr_s0.2"])
def test_noncanonical_fock_vs_brute_force(cp, opt):
    p = _problem(SMALL)
    f_rot, _ = rotated_fock(p)
    assert np.abs(f_rot[:p.nclosed, :p.nclosed] - np.diag(np.diag(f_rot[:p.nclosed, :p.nclosed]))).max() > 1e-2
    got = _run(cp, p, f_rot, p.B, dict(opt, target_state=0))
    ref = o1.solve_problem(p, f=f_rot, xms=bool(opt["xms"]),
                           scheme="sssr" if opt["scheme"] else "msmr", shift=opt["shift"])
    assert np.abs(got.Ems - ref.Ems).max() <= 1e-8
    assert np.abs(got.Heff - ref.Heff).max() <= 1e-8
    c, a = p.nclosed, p.nact
    mask = np.zeros((p.nmo, p.nmo))
    mask[:c, :c] = mask[c:c + a, c:c + a] = mask[c + a:, c + a:] = 1.0
    sym = lambda x: 0.5 * (x + np.swapaxes(x, -1, -2))   # noqa: E731
    _close(got.d1, sym(ref.d1), 1e-9, "d1")
    _close(got.d2, sym(ref.d2) * mask, 1e-9, "d2")
    _close(got.gdf, sym(ref.D1df), 1e-9, "GDF")


def _energy(cp, p, f, opt):
    ctx = cp.Context(p.nclosed, p.nact, p.nvirt, p.naux, p.nstate, **opt)
    try:
        _, B, *rd = cp.problem_inputs(p)
        ctx.set_inputs(np.ascontiguousarray(f), B, *rd)
        st = ctx.solve()
        return ctx.result(st).Ems[opt.get("target_state", 0)]
    finally:
        ctx.close()


def test_gradient_off_diagonal_closed_virtual(cp):
    """dE/df on the off-diagonal closed-closed and virtual-virtual entries (MS) against
    Richardson-combined central differences: every perturbed f is non-canonical and goes
    through the canonicalisation."""
    p = _problem(SMALL)
    opt = dict(xms=0, scheme=0, shift=0.2, target_state=0)
    ctx = cp.Context(p.nclosed, p.nact, p.nvirt, p.naux, p.nstate, **opt)
    try:
        ctx.set_inputs(*cp.problem_inputs(p))
        ctx.solve()
        gf, _ = ctx.gradient()
    finally:
        ctx.close()
    c, a = p.nclosed, p.nact
    mask = np.zeros((p.nmo, p.nmo))
    mask[:c, :c] = mask[c + a:, c + a:] = 1.0
    mask -= np.eye(p.nmo) * mask                     # off-diagonal closed and virtual entries
    rng = np.random.default_rng(3)
    step = 2e-4
    for _ in range(2):
        df = rng.standard_normal(p.f.shape)
        df = (df + df.T) * mask
        df /= np.linalg.norm(df)

        def central(h):
            return (_energy(cp, p, p.f + h * df, opt) - _energy(cp, p, p.f - h * df, opt)) / (2 * h)
        fd = (4.0 * central(step / 2) - central(step)) / 3.0
        an = float(np.sum(gf * df))
        assert abs(an) > 1e-6
        assert abs(fd - an) <= 1e-6 * abs(an) + 1e-8, (fd, an)


def test_coupling_refused_and_amplitudes_refused(cp):
    p = _problem(SMALL)
    f_rot, f_cpl = rotated_fock(p)
    _, B, *rd = cp.problem_inputs(p)
    ctx = cp.Context(p.nclosed, p.nact, p.nvirt, p.naux, p.nstate)
    try:
        with pytest.raises(cp.CASPT2Error) as e:
            ctx.set_inputs(f_cpl, B, *rd)
        assert e.value.status == cp.EINVAL
        ctx.set_inputs(f_rot, B, *rd)
        assert ctx.solve() in (cp.OK, cp.WINTRUDER)
        with pytest.raises(cp.CASPT2Error) as e:
            ctx.amplitudes(0, 0, 0)
        assert e.value.status == cp.EINVAL
    finally:
        ctx.close()
