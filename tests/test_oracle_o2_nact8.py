"""O2 (RDM-form oracle) against O1 (determinant-space brute force) at eight active
orbitals, the active size of the c20 a8 v200 workload (no GPU).

O2's class matrices come from the normal-ordering engine (oracle/wick.py), whose algebra
the library's plan generator shares; O1 applies the operators of Eq. (class) to explicit
vectors and shares nothing with either.  At four active orbitals an index placement
error can coincide with the right one by accident; at eight it cannot.  The problem is
c1 a8 v1 with 6 active electrons and 2 states (10 orbitals, 44100 determinants; every
RDM up to rank 4 populated), seed 41 (no near-intruder: the largest class norm is 0.13).
With one closed and one virtual orbital only the symmetric pair sectors occur; the
antisymmetric ones are pinned at c2 v2 (test_oracle_o2.py) and, against the GPU, at
nact 5 (test_gpu_vs_brute_force.py)."""
import numpy as np
import pytest

from synth import make_problem
from oracle import o1_determinant as o1
from oracle import o2_rdm as o2
from oracle import o2_classes as oc


@pytest.fixture(scope="module")
def p8():
    return make_problem(nclosed=1, nact=8, nvirt=1, naux=30, nstate=2, seed=41, nelact=6)


@pytest.mark.parametrize("xms,scheme,shift", [(True, "msmr", 0.2), (False, "sssr", 0.0)])
def test_o2_matches_brute_force_at_nact8(p8, xms, scheme, shift):
    r = o1.solve_problem(p8, xms=xms, scheme=scheme, shift=shift, densities=False)
    st = o2.setup(p8, xms=xms, kmax=4)
    mom = oc.all_moments(p8, st, shift=shift, scheme=scheme)
    parts = {c: (-np.einsum("llk->lk", M1), np.diagonal(M2).copy()) for c, (M1, M2, M3) in mom.items()}
    for cls in "ABCDEFGH":
        e, nr = parts[cls]
        scale = max(1.0, np.abs(r.e_class[cls]).max())
        assert np.abs(e - r.e_class[cls]).max() <= 1e-11 * scale, cls
        assert np.abs(nr - r.norm_class[cls]).max() <= 1e-11 * max(1.0, np.abs(nr).max()), cls
    H, w, R = o2.heff(st, parts, shift)
    assert np.abs(H - r.Heff).max() <= 1e-10
    assert np.abs(w - r.Ems).max() <= 1e-10
    for cls in "ABCDEFGH":
        NL, lv = oc.lambda_pieces(*mom[cls], R, 0, shift)
        for L in range(p8.nstate):
            idx = [k for k, c in enumerate(r.cols[L]) if c[0] == cls]
            if not idx:
                continue
            lam, t = r.lam[L][idx], r.t[L][idx]
            assert abs(NL[L] - lam @ r.S[L][np.ix_(idx, idx)] @ t) <= 1e-10 * max(1.0, abs(NL[L])), cls
            for Lp in range(p8.nstate):
                ref = lam @ r.b_src[L][Lp][idx]
                assert abs(lv[L, Lp] - ref) <= 1e-10 * max(1.0, abs(ref)), cls
