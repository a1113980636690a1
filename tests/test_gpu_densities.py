"""GPU parity of the correlated densities of the target state (Sec. II.D) through the C ABI
(caspt2_densities / caspt2_get_densities): per class against the RDM-form oracle at the
parity sizes, all classes against the determinant-space brute force on a tiny space, and
at the full bench workload through identities that hold at any size (occupation-change
traces of d2 against N_L, and Euler's theorem for d1 and GDF against the energy path's
e and lambda pieces).  The library returns each density symmetrised, so the oracle's
matrices are symmetrised the same way before comparing."""
import os

import numpy as np
import pytest

from synth import make_problem, WORKLOADS
from oracle import o1_determinant as o1
from oracle import o2_rdm as o2
from oracle import o2_classes as oc

pytestmark = pytest.mark.gpu

CASES = {
    "c4a4v20x84n2": WORKLOADS["c4a4v20x84n2"],
    "ragged_c5a3v70x37n3": dict(nclosed=5, nact=3, nvirt=70, naux=37, nstate=3, seed=21, nelact=2),
}
OPTS = [dict(xms=1, scheme=0, shift=0.2), dict(xms=0, scheme=0, shift=0.0),
        dict(xms=1, scheme=1, shift=0.1)]
OCC_CHANGE = {"A": (-1, 1, 0), "B": (-2, 2, 0), "C": (0, -1, 1), "D": (-1, 0, 1),
              "E": (-2, 1, 1), "F": (0, -2, 2), "G": (-1, -1, 2), "H": (-2, 0, 2)}
RTOL = 1e-9


@pytest.fixture(scope="module")
def cp():
    from paper_1606_01273_gb300 import build as b
    if not os.path.exists(b.LIB):
        b.build()
    import paper_1606_01273_gb300 as cp
    return cp


def _sym(x):
    return 0.5 * (x + np.swapaxes(x, -1, -2))


def _close(got, ref, what):
    scale = max(1.0, float(np.abs(ref).max()))
    err = float(np.abs(got - ref).max())
    assert err <= RTOL * scale, f"{what}: max |diff| {err:.3e} (scale {scale:.3e})"


def _oracle_state(p, opt):
    st = o2.setup(p, xms=bool(opt["xms"]), kmax=4)
    sch = "sssr" if opt["scheme"] == 1 else "msmr"
    mom = oc.all_moments(p, st, shift=opt["shift"], scheme=sch)
    parts = {c: (-np.einsum("llk->lk", M1), np.diagonal(M2).copy()) for c, (M1, M2, M3) in mom.items()}
    _, _, R = o2.heff(st, parts, opt["shift"])
    return st, R, sch


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("opt", OPTS, ids=lambda o: f"xms{o['xms']}_sch{o['scheme']}_s{o['shift']}")
def test_class_densities_vs_rdm_oracle(cp, name, opt):
    p = make_problem(**CASES[name])
    st, R, sch = _oracle_state(p, opt)
    ctx = cp.Context(p.nclosed, p.nact, p.nvirt, p.naux, p.nstate, **opt)
    try:
        ctx.set_inputs(*cp.problem_inputs(p))
        ctx.solve()
        assert np.abs(ctx.result().R - R).max() < 1e-9
        for k, cls in enumerate("ABCDEFGH"):
            d1, d2, gdf = ctx.densities(1 << k)
            if cls == "H":
                rd2, rG, _ = o2.class_h_densities(p, st, R, 0, opt["shift"], sch)
                rd1 = np.zeros_like(rd2)
            else:
                rd1, rG, rd2, _ = oc.class_densities(p, st, cls, opt["shift"], sch, R, 0)
            _close(d1, _sym(rd1), f"{cls} d1")
            _close(d2, _sym(rd2), f"{cls} d2")
            _close(gdf, _sym(rG), f"{cls} GDF")
    finally:
        ctx.close()


@pytest.mark.parametrize("opt", OPTS, ids=lambda o: f"xms{o['xms']}_sch{o['scheme']}_s{o['shift']}")
def test_total_densities_vs_brute_force(cp, opt):
    """All classes at once against O1's densities from explicit determinant-space vectors."""
    p = make_problem(2, 4, 2, 24, 2, seed=5)
    r = cp.solve_problem(p, densities=True, **opt)
    ref = o1.solve_problem(p, xms=bool(opt["xms"]), scheme="sssr" if opt["scheme"] else "msmr",
                           shift=opt["shift"])
    c, a = p.nclosed, p.nact
    mask = np.zeros((p.nmo, p.nmo))
    mask[:c, :c] = mask[c:c + a, c:c + a] = mask[c + a:, c + a:] = 1.0
    _close(r.d1, _sym(ref.d1), "d1")
    _close(r.gdf, _sym(ref.D1df), "GDF")
    _close(r.d2, _sym(ref.d2) * mask, "d2")


def _h_of(p):
    c, a, n = p.nclosed, p.nact, p.nstate
    d = np.zeros((p.nmo, p.nmo))
    d[np.arange(c), np.arange(c)] = 2.0
    g1 = p.rdm[1].reshape(n, n, a, a)
    d[c:c + a, c:c + a] = sum(g1[m, m] for m in range(n)) / n
    return p.f - o2.g_of(p.B, d)


@pytest.mark.parametrize("opt", [dict(xms=1, scheme=0, shift=0.2), dict(xms=1, scheme=1, shift=0.2)],
                         ids=["xms_msmr", "xms_sssr"])
def test_densities_identities_at_bench_size(cp, opt):
    """The benchmark workload (c20 a8 v200, naux 700, 3 states): per class, the block
    traces of d2 equal the occupation change times sum_L N_L, and sum d1 h + 1/2 sum GDF B
    equals sum r r e + tr(lv), with N_L, e and lv from the solve's moment path."""
    p = make_problem(**WORKLOADS["c20a8v200x700n3"])
    h = _h_of(p)
    c, a = p.nclosed, p.nact
    ctx = cp.Context(p.nclosed, p.nact, p.nvirt, p.naux, p.nstate, **opt)
    try:
        ctx.set_inputs(*cp.problem_inputs(p))
        st = ctx.solve()
        res = ctx.result(st)
        r = res.R[:, 0]
        for k, cls in enumerate("ABCDEFGH"):
            d1, d2, gdf = ctx.densities(1 << k)
            NL = res.lam_NL[cls].sum()
            tr = [np.trace(d2[:c, :c]), np.trace(d2[c:c + a, c:c + a]),
                  np.trace(d2[c + a:, c + a:])]
            scale = max(1.0, float(np.abs(d2).max()))
            for q in range(3):
                assert abs(tr[q] - OCC_CHANGE[cls][q] * NL) <= 1e-9 * scale, (cls, q, tr, NL)
            src = r @ res.e_class[cls] @ r + np.trace(res.lam_lv[cls])
            val = np.sum(d1 * h) + 0.5 * np.sum(gdf * p.B)
            assert abs(val - src) <= 1e-9 * max(1.0, abs(src)), (cls, val, src)
    finally:
        ctx.close()
