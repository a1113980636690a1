"""First-order amplitudes T_LN and the target state's lambda_LN of the classes A-G through
the C ABI (caspt2_get_amplitudes / caspt2_get_lambda), against the RDM-form oracle's
amplitudes and multipliers in the same range-projected gauge (the oracle expands them in
the orthonormalised basis Y = X Q of each sector, as the library does), for every (L, N),
MS-MR and SS-SR, at the small workload and a ragged case.

Tolerance: 1e-9 of the class's largest element, widened for ill-conditioned classes.  An
amplitude is a source divided by its denominators, so near an intruder it inherits the
rounding of the sector eigenvalues amplified by E/|D|; the library's and the oracle's
eigensolvers round differently at up to ~1e-13 relative.  The test measures each class's
conditioning with the oracle itself (the relative change of its T and lambda under a
seeded 1e-15 relative perturbation of f) and allows 1000 times that (1e-13 / 1e-15 with a
factor 10 of margin)."""
import os

import numpy as np
import pytest

from synth import make_problem, WORKLOADS
from oracle import o2_rdm as o2
from oracle import o2_classes as oc

pytestmark = pytest.mark.gpu

CASES = {
    "c4a4v20x84n2": WORKLOADS["c4a4v20x84n2"],
    "ragged_c5a3v70x37n3": dict(nclosed=5, nact=3, nvirt=70, naux=37, nstate=3, seed=21, nelact=2),
}
OPTS = [dict(xms=1, scheme=0, shift=0.2, target_state=0),
        dict(xms=1, scheme=1, shift=0.1, target_state=1)]


@pytest.fixture(scope="module")
def cp():
    from paper_1606_01273_gb300 import build as b
    if not os.path.exists(b.LIB):
        b.build()
    import paper_1606_01273_gb300 as cp
    return cp


def _oracle_vectors(p, opt, P, perturb=0.0):
    if perturb:
        import copy
        p = copy.deepcopy(p)
        d = np.random.default_rng(3).standard_normal(p.f.shape)
        p.f = p.f * (1.0 + perturb * 0.5 * (d + d.T))
    st = o2.setup(p, xms=bool(opt["xms"]), kmax=4)
    sch = "sssr" if opt["scheme"] == 1 else "msmr"
    mom = oc.all_moments(p, st, shift=opt["shift"], scheme=sch)
    parts = {c: (-np.einsum("llk->lk", M1), np.diagonal(M2).copy()) for c, (M1, M2, M3) in mom.items()}
    _, _, R = o2.heff(st, parts, opt["shift"])
    return {cls: oc.class_amplitudes(p, st, cls, opt["shift"], sch, R, P) for cls in "ABCDEFG"}


def _rel(a, b):
    return float(np.abs(a - b).max()) / max(1e-300, float(np.abs(b).max()))


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("opt", OPTS, ids=["xms_msmr_P0", "xms_sssr_P1"])
def test_amplitudes_and_lambda_vs_oracle(cp, name, opt):
    p = make_problem(**CASES[name])
    P = opt["target_state"]
    ref = _oracle_vectors(p, opt, P)
    probe = _oracle_vectors(p, opt, P, perturb=1e-15)
    ctx = cp.Context(p.nclosed, p.nact, p.nvirt, p.naux, p.nstate, **opt)
    try:
        ctx.set_inputs(*cp.problem_inputs(p))
        ctx.solve()
        for k, cls in enumerate("ABCDEFG"):
            T, Lam = ref[cls]
            tt = max(1e-9, 1e3 * _rel(probe[cls][0], T))
            tl = max(1e-9, 1e3 * _rel(probe[cls][1], Lam))
            assert ctx.amplitude_size(k) == T[0][..., 0].size, cls
            ts = max(1e-300, float(np.abs(T).max()))
            ls = max(1e-300, float(np.abs(Lam).max()))
            for L in range(p.nstate):
                for N in range(p.nstate):
                    t = ctx.amplitudes(k, L, N)
                    lam = ctx.lambdas(k, L, N)
                    assert np.abs(t - T[L][..., N].ravel()).max() <= tt * ts, (cls, L, N, tt)
                    assert np.abs(lam - Lam[L][..., N].ravel()).max() <= tl * ls, (cls, L, N, tl)
        with pytest.raises(cp.CASPT2Error):
            ctx.amplitudes(7, 0, 0)                      # class H amplitudes are never formed
    finally:
        ctx.close()


def test_status_report(cp):
    """caspt2_get_status after create, solve and densities."""
    p = make_problem(**CASES["c4a4v20x84n2"])
    ctx = cp.Context(p.nclosed, p.nact, p.nvirt, p.naux, p.nstate, xms=1, scheme=0, shift=0.2,
                     target_state=0)
    try:
        r0 = ctx.status()
        assert r0["last_status"] == cp.ESTATE and not r0["solved"]
        ctx.set_inputs(*cp.problem_inputs(p))
        st = ctx.solve()
        r1 = ctx.status()
        assert r1["last_status"] == st and r1["solved"] and not r1["densities_done"]
        assert r1["min_denominator"] > 0.0 and r1["kernel_launches"] > 0
        assert (st == 1) == (r1["min_denominator"] < 1e-3)
        ctx.densities()
        assert ctx.status()["densities_done"]
    finally:
        ctx.close()
