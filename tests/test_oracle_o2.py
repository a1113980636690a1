"""Pins of the RDM-form oracle O2 against the brute-force oracle O1 (no GPU)."""
import numpy as np
import pytest

from synth import make_problem
from oracle import o1_determinant as o1
from oracle import o2_rdm as o2

CASES = [
    dict(nclosed=2, nact=4, nvirt=2, naux=24, nstate=2, seed=5),
    dict(nclosed=2, nact=3, nvirt=3, naux=20, nstate=3, seed=8, nelact=2),
    dict(nclosed=3, nact=0, nvirt=4, naux=30, nstate=1, seed=3),
]


@pytest.fixture(scope="module", params=range(len(CASES)))
def prob(request):
    return make_problem(**CASES[request.param])


@pytest.mark.parametrize("xms", [True, False])
def test_setup_matches_o1(prob, xms):
    """U, E0 and H^ref (Sec. II.A) from RDMs equal the determinant-space values."""
    r = o1.solve_problem(prob, xms=xms, densities=False)
    st = o2.setup(prob, xms=xms)
    assert np.allclose(st.U, r.U, atol=1e-12)
    assert np.allclose(st.E0, r.E0, atol=1e-12)
    assert np.allclose(st.Href, r.Href, atol=1e-11)
    assert abs(st.Ecore - r.Ecore) < 1e-11


@pytest.mark.parametrize("xms,scheme,shift", [(True, "msmr", 0.0), (True, "msmr", 0.3),
                                              (False, "msmr", 0.2), (True, "sssr", 0.2),
                                              (False, "sssr", 0.0)])
def test_class_h_matches_o1(prob, xms, scheme, shift):
    """Class E_ai,bj contributions to H^eff and <Psi1|Psi1> equal O1's."""
    r = o1.solve_problem(prob, xms=xms, scheme=scheme, shift=shift, densities=False)
    st = o2.setup(prob, xms=xms)
    e, nr = o2.class_h(prob, st, shift=shift, scheme=scheme)
    scale = max(1.0, np.abs(r.e_class["H"]).max())
    assert np.allclose(e, r.e_class["H"], atol=1e-11 * scale)
    assert np.allclose(nr, r.norm_class["H"], atol=1e-11)
