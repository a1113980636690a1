"""The large-active-space input generator (synth.casci_fast: Davidson CASCI, RDMs from
canonical annihilated-vector Gram matrices) against the dense generator (synth.casci:
full Hamiltonian matrix, every spin pattern of annihilated vectors) on spaces both can
build (no GPU; torch on the CPU)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from synth.casci import ActiveSpace, lowest_singlets, hamiltonian_matrix, s2_matrix
from synth.casci_fast import BigSpace, davidson_singlets, rdms


@pytest.mark.parametrize("a,ne,n", [(4, 4, 2), (5, 4, 3), (6, 6, 2)])
def test_fast_generator_matches_dense(a, ne, n):
    rng = np.random.default_rng(a)
    t = rng.uniform(-0.3, 0.3, (a, a))
    h1 = np.triu(t) + np.triu(t, 1).T
    B = rng.standard_normal((12, a, a))
    B = 0.15 * (B + B.transpose(0, 2, 1))
    eri = np.einsum("Ppq,Prs->pqrs", B, B)
    sp = ActiveSpace(a, ne)
    bs = BigSpace(a, ne, "cpu")
    X = rng.standard_normal((sp.ndet, 3))
    Xt = torch.tensor(X).reshape(bs.ns, bs.ns, 3)
    hm = hamiltonian_matrix(sp, h1, eri)
    s2m = s2_matrix(sp)
    assert np.abs(bs.sigma(Xt, h1, eri).reshape(sp.ndet, 3).numpy() - hm @ X).max() < 1e-12
    assert np.abs(bs.s2(Xt).reshape(sp.ndet, 3).numpy() - s2m @ X).max() < 1e-12
    assert np.abs(bs.diag(h1, eri, 1.0).reshape(-1).numpy() - np.diag(hm + s2m)).max() < 1e-12
    e0, c0 = lowest_singlets(sp, h1, eri, n)
    e1, c1 = davidson_singlets(bs, h1, eri, n)
    assert np.abs(e0 - e1).max() < 1e-10
    assert np.abs(np.abs(np.sum(c0 * c1, axis=0)) - 1.0).max() < 1e-10
    r1 = rdms(bs, c1, 4)
    for k in range(1, 5):
        r0 = sp.rdm(c1, k).reshape(n, n, -1)
        assert np.abs(r1[k].numpy() - r0).max() < 1e-13, k
