"""The whole C-ABI path against the determinant-space brute force (O1) at nact 5 and 6.

The library's class algebra (its contraction plans) and the RDM-form oracle come from
the same normal-ordering derivation, so agreement between those two checks arithmetic,
not algebra.  O1 shares nothing with either: it applies the excitation operators of
Eq. (class) to explicit determinant-space vectors.  These spaces have more active
orbitals than the four at which an index placement can coincide by accident:

  * c1 a6 v1, 6 active electrons, 2 states: 8 orbitals, 4900 determinants;
  * c2 a5 v2, 4 active electrons, 3 states: 9 orbitals, 15876 determinants, with two
    closed and two virtual orbitals so that the antisymmetric pair sectors of classes
    B, E, F, G and H are populated.

For XMS and MS, MS-MR and SS-SR, shifts 0 and 0.2: every class's <Psi1_L|H|L'~> and
<Psi1_L|Psi1_L>, the lambda pieces, H^eff, E^MS, N_L and the densities d1, d2 (closed,
active and virtual blocks) and GDF are compared element by element.  Seeds were chosen
with no near-intruder (largest class norm below 1.3) and no overlap eigenvalue within
[1e-12, 1e-6] of the truncation."""
import os

import numpy as np
import pytest

from synth import make_problem
from oracle import o1_determinant as o1

pytestmark = pytest.mark.gpu

PROBLEMS = {
    "c1a6v1n2": dict(nclosed=1, nact=6, nvirt=1, naux=20, nstate=2, seed=33),
    "c2a5v2n3": dict(nclosed=2, nact=5, nvirt=2, naux=24, nstate=3, seed=36, nelact=4),
}
OPTS = [dict(xms=x, scheme=s, shift=e) for x in (1, 0) for s in (0, 1) for e in (0.0, 0.2)]
ETOL = 1e-8


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


def _sym(x):
    return 0.5 * (x + np.swapaxes(x, -1, -2))


def _close(got, ref, rtol, what):
    scale = max(1.0, float(np.abs(ref).max()))
    err = float(np.abs(got - ref).max())
    assert err <= rtol * scale, f"{what}: max |diff| {err:.3e} (scale {scale:.3e})"


@pytest.mark.parametrize("name", list(PROBLEMS))
@pytest.mark.parametrize("opt", OPTS, ids=lambda o: f"xms{o['xms']}_sch{o['scheme']}_s{o['shift']}")
def test_path_vs_brute_force(cp, name, opt):
    p = _problem(name)
    ctx = cp.Context(p.nclosed, p.nact, p.nvirt, p.naux, p.nstate, **opt)
    try:
        ctx.set_inputs(*cp.problem_inputs(p))
        st = ctx.solve()
        assert st == cp.OK
        r = ctx.result(st)
        ctx.compute_densities()
        d1, d2, gdf, nl = ctx.get_densities(with_nl=True)
    finally:
        ctx.close()
    ref = o1.solve_problem(p, xms=bool(opt["xms"]), scheme="sssr" if opt["scheme"] else "msmr",
                           shift=opt["shift"])
    n = p.nstate
    for cls in "ABCDEFGH":
        _close(r.e_class[cls], ref.e_class[cls], 1e-10, f"{cls} e")
        _close(r.norm_class[cls], ref.norm_class[cls], 1e-10, f"{cls} norm")
        for L in range(n):
            idx = [k for k, c in enumerate(ref.cols[L]) if c[0] == cls]
            if not idx:
                continue
            lam, t = ref.lam[L][idx], ref.t[L][idx]
            nlc = lam @ ref.S[L][np.ix_(idx, idx)] @ t
            assert abs(r.lam_NL[cls][L] - nlc) <= 1e-9 * max(1.0, abs(nlc)), (cls, L)
            for Lp in range(n):
                lv = lam @ ref.b_src[L][Lp][idx]
                assert abs(r.lam_lv[cls][L, Lp] - lv) <= 1e-9 * max(1.0, abs(lv)), (cls, L, Lp)
    assert np.abs(r.U - ref.U).max() <= 1e-10
    assert np.abs(r.Heff - ref.Heff).max() <= ETOL
    assert np.abs(r.Ems - ref.Ems).max() <= ETOL
    _close(nl, ref.NL, 1e-9, "N_L")
    c, a = p.nclosed, p.nact
    mask = np.zeros((p.nmo, p.nmo))
    mask[:c, :c] = mask[c:c + a, c:c + a] = mask[c + a:, c + a:] = 1.0
    _close(d1, _sym(ref.d1), 1e-9, "d1")
    _close(d2, _sym(ref.d2) * mask, 1e-9, "d2")
    _close(gdf, _sym(ref.D1df), 1e-9, "GDF")
