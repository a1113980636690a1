"""GPU parity of all eight classes (A-G from plan-driven RDM contractions, H direct),
H^eff and E^MS through the C ABI: against the RDM-form oracle at the parity sizes and
directly against the determinant-space brute force on a tiny space."""
import os

import numpy as np
import pytest

from synth import make_problem, WORKLOADS
from oracle import o1_determinant as o1
from oracle import o2_rdm as o2
from oracle import o2_classes as oc

pytestmark = pytest.mark.gpu

ETOL = 1e-8
CASES = {
    "c4a4v20x84n2": WORKLOADS["c4a4v20x84n2"],
    "ragged_c5a3v70x37n3": dict(nclosed=5, nact=3, nvirt=70, naux=37, nstate=3, seed=21, nelact=2),
}
OPTS = [dict(xms=1, scheme=0, shift=0.2), dict(xms=0, scheme=0, shift=0.0),
        dict(xms=1, scheme=1, shift=0.1)]


@pytest.fixture(scope="module")
def cp():
    from paper_1606_01273_gb300 import build as b
    if not os.path.exists(b.LIB):
        b.build()
    import paper_1606_01273_gb300 as cp
    return cp


_probs = {}


def _prob(name):
    if name not in _probs:
        _probs[name] = make_problem(**CASES[name])
    return _probs[name]


def _check(r, ref_parts, st, shift, etol_rel=1e-10):
    for cls, (e, nr) in ref_parts.items():
        scale = max(1.0, np.abs(e).max())
        assert np.abs(r.e_class[cls] - e).max() <= min(ETOL, etol_rel * scale), cls
        assert np.abs(r.norm_class[cls] - nr).max() <= etol_rel * max(1.0, np.abs(nr).max()), cls
    H, w, R = o2.heff(st, ref_parts, shift)
    assert np.abs(r.Heff - H).max() <= ETOL
    assert np.abs(r.Ems - w).max() <= ETOL


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("opt", OPTS, ids=lambda o: f"xms{o['xms']}_sch{o['scheme']}_s{o['shift']}")
def test_all_classes_vs_rdm_oracle(cp, name, opt):
    p = _prob(name)
    r = cp.solve_problem(p, **opt)
    st = o2.setup(p, xms=bool(opt["xms"]), kmax=4)
    sch = "sssr" if opt["scheme"] == 1 else "msmr"
    mom = oc.all_moments(p, st, shift=opt["shift"], scheme=sch)
    parts = {c: (-np.einsum("llk->lk", M1), np.diagonal(M2).copy()) for c, (M1, M2, M3) in mom.items()}
    _check(r, parts, st, opt["shift"])
    # lambda of target state 0 (Eq. lambdaeq), per class
    H, w, R = o2.heff(st, parts, opt["shift"])
    for cls in "ABCDEFGH":
        NL, lv = oc.lambda_pieces(*mom[cls], R, 0, opt["shift"])
        assert np.abs(r.lam_NL[cls] - NL).max() <= 1e-9 * max(1.0, np.abs(NL).max()), cls
        assert np.abs(r.lam_lv[cls] - lv).max() <= 1e-9 * max(1.0, np.abs(lv).max()), cls


@pytest.mark.parametrize("opt", OPTS, ids=lambda o: f"xms{o['xms']}_sch{o['scheme']}_s{o['shift']}")
def test_all_classes_vs_brute_force(cp, opt):
    """The CUDA path against explicit determinant-space vectors (no RDM algebra)."""
    p = make_problem(2, 4, 2, 24, 2, seed=5)
    r = cp.solve_problem(p, **opt)
    ref = o1.solve_problem(p, xms=bool(opt["xms"]), scheme="sssr" if opt["scheme"] else "msmr",
                           shift=opt["shift"], densities=False)
    for cls in "ABCDEFGH":
        scale = max(1.0, np.abs(ref.e_class[cls]).max())
        assert np.abs(r.e_class[cls] - ref.e_class[cls]).max() <= 1e-10 * scale, cls
        assert np.abs(r.norm_class[cls] - ref.norm_class[cls]).max() <= 1e-10, cls
        # lambda against the explicit determinant-space vectors
        n = p.nstate
        for L in range(n):
            idx = [k for k, c in enumerate(ref.cols[L]) if c[0] == cls]
            if not idx:
                continue
            lam, t = ref.lam[L][idx], ref.t[L][idx]
            nl = lam @ ref.S[L][np.ix_(idx, idx)] @ t
            assert abs(r.lam_NL[cls][L] - nl) <= 1e-9 * max(1.0, abs(nl)), cls
            for Lp in range(n):
                lv = lam @ ref.b_src[L][Lp][idx]
                assert abs(r.lam_lv[cls][L, Lp] - lv) <= 1e-9 * max(1.0, abs(lv)), cls
    assert np.abs(r.Heff - ref.Heff).max() <= ETOL
    assert np.abs(r.Ems - ref.Ems).max() <= ETOL


def test_bench_workload_all_classes(cp):
    """The full benzophenone-like bench workload (XMS, MS-MR, shift 0.2).  Class C has a
    near-intruder denominator here (min |D| = 2.7e-4 Eh), so the shift-correction term
    E_s <T|T> is ill-conditioned: the oracle's own class-C norm moves by ~3e-6 between two
    LAPACK eigensolver drivers.  The pieces are compared to 1e-8 relative and E^MS to
    1e-8 Eh + E_s * 1e-8 * sum_X max|norm_X| (the relative bound carried through the shift
    term); the library reports the near-intruder as WINTRUDER."""
    p = make_problem(**WORKLOADS["c20a8v200x700n3"])
    r = cp.solve_problem(p, xms=1, scheme=0, shift=0.2)
    assert r.status == cp.WINTRUDER
    st = o2.setup(p, xms=True, kmax=4)
    parts = oc.all_classes(p, st, shift=0.2, scheme="msmr")
    nsum = 0.0
    for cls, (e, nr) in parts.items():
        assert np.abs(r.e_class[cls] - e).max() <= 1e-8 * max(1.0, np.abs(e).max()), cls
        assert np.abs(r.norm_class[cls] - nr).max() <= 1e-8 * max(1.0, np.abs(nr).max()), cls
        nsum += np.abs(nr).max()
    H, w, R = o2.heff(st, parts, 0.2)
    assert np.abs(r.Ems - w).max() <= 1e-8 + 0.2 * 1e-8 * nsum
