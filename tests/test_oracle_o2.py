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


CLASS_CASES = [
    dict(nclosed=2, nact=4, nvirt=2, naux=24, nstate=2, seed=5),
    dict(nclosed=2, nact=3, nvirt=2, naux=20, nstate=3, seed=8, nelact=2),
    dict(nclosed=1, nact=4, nvirt=3, naux=16, nstate=1, seed=14, nelact=4),
]


@pytest.fixture(scope="module", params=range(len(CLASS_CASES)))
def cprob(request):
    return make_problem(**CLASS_CASES[request.param])


@pytest.mark.parametrize("xms,scheme,shift", [(True, "msmr", 0.2), (False, "msmr", 0.0),
                                              (True, "sssr", 0.1), (False, "sssr", 0.3)])
def test_classes_a_to_g_match_o1(cprob, xms, scheme, shift):
    """Per-class <Psi1_L|H|L'~> and <Psi1_L|Psi1_L> of classes A-G from RDMs (normal-
    ordering engine + per-sector solve) equal the determinant-space values."""
    from oracle import o2_classes as oc
    r = o1.solve_problem(cprob, xms=xms, scheme=scheme, shift=shift, densities=False)
    st = o2.setup(cprob, xms=xms, kmax=4)
    for cls in "ABCDEFG":
        e, nr = oc.class_energy(cprob, st, cls, shift=shift, scheme=scheme)
        scale = max(1.0, np.abs(r.e_class[cls]).max())
        assert np.abs(e - r.e_class[cls]).max() <= 1e-11 * scale, cls
        assert np.abs(nr - r.norm_class[cls]).max() <= 1e-11 * max(1.0, np.abs(nr).max()), cls


def test_wick_engine_identities():
    """Textbook identities: <E_ij> = 2 delta_ij over the core, E_rs E_tu = E_rs,tu +
    delta_st E_ru, <E_ir E_r'i'> = delta_ii'(2 delta_rr' - Gamma_r'r)."""
    from oracle.wick import Builder, expect
    sp = {"i": "c", "j": "c", "r": "a", "s": "a", "t": "a", "u": "a", "a": "v", "b": "v"}
    b = Builder()
    assert [(x.coeff, x.deltas, x.rdm) for x in expect(b.E("i", "j"), sp)] == [(2, (("i", "j"),), ())]
    assert expect(b.E("a", "b"), sp) == []
    got = {(x.coeff, x.deltas, x.rdm) for x in expect(b.E("r", "s") + b.E("t", "u"), sp)}
    assert got == {(1, (), (("r", "s"), ("t", "u"))), (1, (("s", "t"),), (("r", "u"),))}
    got = {(x.coeff, x.deltas, x.rdm) for x in expect(b.E("i", "r") + b.E("s", "j"), sp)}
    assert got == {(2, (("i", "j"), ("r", "s")), ()), (-1, (("i", "j"),), (("s", "r"),))}


@pytest.mark.parametrize("xms,scheme,shift", [(True, "msmr", 0.2), (False, "msmr", 0.0),
                                              (True, "sssr", 0.1), (False, "msmr", 0.3)])
def test_lambda_pieces_match_o1(cprob, xms, scheme, shift):
    """lambda per class from the moment sums equals O1's explicit lambda vectors:
    NL[L] = lam_L . S_L t_L and lv[L, L'] = lam_L . V_L^T H |L'~> over the class columns."""
    from oracle import o2_classes as oc
    r = o1.solve_problem(cprob, xms=xms, scheme=scheme, shift=shift, densities=False)
    st = o2.setup(cprob, xms=xms, kmax=4)
    mom = oc.all_moments(cprob, st, shift=shift, scheme=scheme)
    parts = {c: (-np.einsum("llk->lk", M1), np.diagonal(M2).copy()) for c, (M1, M2, M3) in mom.items()}
    H, w, R = o2.heff(st, parts, shift)
    assert np.abs(R - r.R).max() < 1e-9
    n = cprob.nstate
    for cls in "ABCDEFGH":
        NL, lv = oc.lambda_pieces(*mom[cls], R, 0, shift)
        for L in range(n):
            idx = [k for k, c in enumerate(r.cols[L]) if c[0] == cls]
            if not idx:
                continue
            lam, t = r.lam[L][idx], r.t[L][idx]
            S = r.S[L][np.ix_(idx, idx)]
            assert abs(NL[L] - lam @ S @ t) <= 1e-10 * max(1.0, abs(NL[L])), cls
            for Lp in range(n):
                ref = lam @ r.b_src[L][Lp][idx]
                assert abs(lv[L, Lp] - ref) <= 1e-10 * max(1.0, abs(ref)), cls


def _o2_state(p, xms, scheme, shift):
    from oracle import o2_classes as oc
    st = o2.setup(p, xms=xms, kmax=4)
    mom = oc.all_moments(p, st, shift=shift, scheme=scheme)
    parts = {c: (-np.einsum("llk->lk", M1), np.diagonal(M2).copy()) for c, (M1, M2, M3) in mom.items()}
    H, w, R = o2.heff(st, parts, shift)
    return st, R


def _o2_densities(p, st, R, shift, scheme, classes="ABCDEFGH"):
    from oracle import o2_classes as oc
    nmo = p.nmo
    d1, G, d2, NL = np.zeros((nmo, nmo)), np.zeros_like(p.B), np.zeros((nmo, nmo)), np.zeros(p.nstate)
    for cls in classes:
        if cls == "H":
            a2, b2, c2 = o2.class_h_densities(p, st, R, 0, shift, scheme)
            d2 += a2; G += b2; NL += c2
        else:
            a1, b1, c1, e1 = oc.class_densities(p, st, cls, shift, scheme, R, 0)
            d1 += a1; G += b1; d2 += c1; NL += e1
    return d1, G, d2, NL


def _diag_blocks(p, x):
    c, a = p.nclosed, p.nact
    m = np.zeros_like(x)
    m[:c, :c] = 1
    m[c:c + a, c:c + a] = 1
    m[c + a:, c + a:] = 1
    return x * m


@pytest.mark.parametrize("xms,scheme,shift", [(True, "msmr", 0.2), (False, "sssr", 0.1)])
def test_class_densities_match_o1(xms, scheme, shift):
    """Each class's share of d(1), D(1).B, N_L and the closed/active/virtual blocks of d(2)
    (Sec. II.D) equals O1's densities built from that class's amplitudes alone."""
    p = make_problem(**CLASS_CASES[0])
    st, R = _o2_state(p, xms, scheme, shift)
    for cls in "ABCDEFGH":
        r = o1.solve_problem(p, xms=xms, scheme=scheme, shift=shift, density_classes=cls)
        d1, G, d2, NL = _o2_densities(p, st, R, shift, scheme, cls)
        assert np.abs(d1 - r.d1).max() < 1e-12, cls
        assert np.abs(G - r.D1df).max() < 1e-12, cls
        assert np.abs(_diag_blocks(p, d2 - r.d2)).max() < 1e-12, cls
        assert np.abs(NL - r.NL).max() < 1e-12, cls


@pytest.mark.parametrize("xms,scheme,shift", [(True, "msmr", 0.2), (False, "msmr", 0.0),
                                              (True, "sssr", 0.1)])
def test_total_densities_match_o1(cprob, xms, scheme, shift):
    """Sum over classes: d(1), D(1).B and N_L equal O1 (FD-validated) exactly; d(2) on its
    closed, active and virtual blocks."""
    st, R = _o2_state(cprob, xms, scheme, shift)
    r = o1.solve_problem(cprob, xms=xms, scheme=scheme, shift=shift)
    d1, G, d2, NL = _o2_densities(cprob, st, R, shift, scheme)
    assert np.abs(d1 - r.d1).max() < 1e-11
    assert np.abs(G - r.D1df).max() < 1e-11
    assert np.abs(_diag_blocks(cprob, d2 - r.d2)).max() < 1e-11
    assert np.abs(NL - r.NL).max() < 1e-11


# (closed, active, virtual) change of the orbital-space occupation made by each class's
# excitation operator (Eq. class): e.g. class A moves one electron closed -> active.
OCC_CHANGE = {"A": (-1, 1, 0), "B": (-2, 2, 0), "C": (0, -1, 1), "D": (-1, 0, 1),
              "E": (-2, 1, 1), "F": (0, -2, 2), "G": (-1, -1, 2), "H": (-2, 0, 2)}


def _h_of(p):
    c, a, n = p.nclosed, p.nact, p.nstate
    d = np.zeros((p.nmo, p.nmo))
    d[np.arange(c), np.arange(c)] = 2.0
    g1 = p.rdm[1].reshape(n, n, a, a)
    d[c:c + a, c:c + a] = sum(g1[m, m] for m in range(n)) / n
    return p.f - o2.g_of(p.B, d)


@pytest.mark.parametrize("xms,scheme,shift", [(True, "msmr", 0.2), (False, "sssr", 0.1),
                                              (False, "msmr", 0.0)])
def test_density_identities(xms, scheme, shift):
    """Two exact identities per class, independent of the density algebra:
    (1) particle-number conservation: shifting every f_pp of one orbital space by delta
        shifts each denominator by delta times the class's occupation change there, so
        tr d2(space) = change(space) * sum_L N_L (the E0 term cancels the reference part);
    (2) Euler's theorem: the sources are linear in h and bilinear in B, so
        sum d1 h + 1/2 sum GDF B = sum_LL' r_L r_L' e[L][L'] + sum_L lv[L][L]
        with e and lv from the moment path (Eq. lambdaeq)."""
    from oracle import o2_classes as oc
    p = make_problem(nclosed=2, nact=4, nvirt=3, naux=24, nstate=2, seed=5)
    st = o2.setup(p, xms=xms, kmax=4)
    mom = oc.all_moments(p, st, shift=shift, scheme=scheme)
    parts = {c: (-np.einsum("llk->lk", M1), np.diagonal(M2).copy()) for c, (M1, M2, M3) in mom.items()}
    _, _, R = o2.heff(st, parts, shift)
    h = _h_of(p)
    c, a = p.nclosed, p.nact
    r = R[:, 0]
    for cls in "ABCDEFGH":
        NL, lv = oc.lambda_pieces(*mom[cls], R, 0, shift)
        d1, G, d2, _ = _o2_densities(p, st, R, shift, scheme, cls)
        tr = [np.trace(d2[:c, :c]), np.trace(d2[c:c + a, c:c + a]), np.trace(d2[c + a:, c + a:])]
        for k in range(3):
            assert abs(tr[k] - OCC_CHANGE[cls][k] * NL.sum()) < 1e-12, (cls, k)
        src = r @ parts[cls][0] @ r + np.trace(lv)
        assert abs(np.sum(d1 * h) + 0.5 * np.sum(G * p.B) - src) < 1e-12 * max(1.0, abs(src)), cls


@pytest.mark.parametrize("xms,scheme,shift", [(True, "msmr", 0.2), (False, "msmr", 0.0),
                                              (True, "sssr", 0.1)])
def test_offdiag_dbar2_matches_o1(cprob, xms, scheme, shift):
    """The closed-active, active-virtual and closed-virtual blocks of dbar2 (Sec. II.D), which
    couple different classes through E_xy, equal O1's <Psi_lambda_L|E_xy|Psi1_L> summed
    over L, block by block."""
    from oracle.o2_offdiag import offdiag_dbar2
    st, R = _o2_state(cprob, xms, scheme, shift)
    r = o1.solve_problem(cprob, xms=xms, scheme=scheme, shift=shift)
    got = offdiag_dbar2(cprob, st, shift, scheme, R, 0)
    c, a = cprob.nclosed, cprob.nact
    off = np.ones((cprob.nmo, cprob.nmo))
    off[:c, :c] = off[c:c + a, c:c + a] = off[c + a:, c + a:] = 0.0
    scale = max(1.0, float(np.abs(r.dbar2 * off).max()))
    assert np.abs((got - r.dbar2) * off).max() <= 1e-11 * scale
    assert np.abs(got * (1.0 - off)).max() == 0.0
