"""Seeded synthetic inputs for the (X)MS-CASPT2 amplitude / lambda / density path.

The paper's molecules, basis sets and integrals are not available, so every
input is synthetic and seeded (numpy PCG64):

  * DF factors  B[P,p,q] = alpha sum_k U[P,k] sigma_k W_k[p,q]   (U ~ N(0,1),
    W_k = (G + G^T)/2 with G ~ N(0,1), sigma_k = exp(-k/decay), alpha chosen so
    that the mean (pp|pp) is about c0 = 0.5 Eh);
  * orbital energies: closed U[-2.5, -0.4] (sorted), virtual log-uniform on
    [0.2, 4.0] Eh (sorted), an active symmetric block with entries U[-0.3, 0.3];
  * reference states: the lowest nstate singlets of the active-space
    Hamiltonian (exact diagonalisation), spin-free 1- to 4-RDMs between all of
    them.

The Fock matrix f returned here is block diagonal (closed and virtual blocks
diagonal, no closed-active, active-virtual or closed-virtual coupling).  Its
active block is made consistent with the reference states: the CASCI is run
with the core-dressed one-electron operator fc, and then f_act = fc_act +
J/K(d_sa) over the active block, so that the states are eigenfunctions of the
Hamiltonian built from h = f - g(d_sa) restricted to the active space
(Sec. II.A).  This file only prepares inputs; none of the perturbation method
is computed here.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

from .casci import ActiveSpace, lowest_singlets


@dataclass
class Problem:
    nclosed: int
    nact: int
    nvirt: int
    naux: int
    nstate: int
    nelact: int
    seed: int
    f: np.ndarray            # [nmo, nmo] state-averaged Fock, block diagonal
    B: np.ndarray            # [naux, nmo, nmo] DF factors, symmetric in (p, q)
    ci: np.ndarray           # [ndet, nstate] CASCI vectors (determinant order: synth.casci)
    det_alpha: np.ndarray    # [ndet] alpha bitmask of each active determinant
    det_beta: np.ndarray     # [ndet] beta bitmask
    e_cas: np.ndarray        # [nstate] active-space energies (without core energy)
    rdm: dict = field(default_factory=dict)   # k -> [n][n][a^{2k}] spin-free RDMs

    @property
    def nmo(self) -> int:
        return self.nclosed + self.nact + self.nvirt

    def rdms(self, kmax: int = 4):
        return [self.rdm[k] for k in range(1, kmax + 1)]


def df_factors(rng: np.random.Generator, naux: int, nmo: int, decay: float, c0: float = 0.5,
               device: str | None = None):
    """device: None forms the product with numpy (the stored oracle results depend on those
    bytes); a torch device name forms the same product there (other rounding)."""
    k = np.arange(naux)
    sigma = np.exp(-k / decay)
    alpha = math.sqrt(c0 / (naux * float(np.sum(sigma ** 2))))
    U = rng.standard_normal((naux, naux))
    G = rng.standard_normal((naux, nmo, nmo))
    W = 0.5 * (G + G.transpose(0, 2, 1))
    if device is not None:
        import torch
        Ut = torch.from_numpy(U * sigma[None, :]).to(device)
        Wt = torch.from_numpy(W.reshape(naux, nmo * nmo)).to(device)
        B = (alpha * (Ut @ Wt)).cpu().numpy().reshape(naux, nmo, nmo)
        del Ut, Wt
        _release_device(device)
        return B
    B = alpha * ((U * sigma[None, :]) @ W.reshape(naux, nmo * nmo)).reshape(naux, nmo, nmo)
    return B


def _active_meanfield(eri_act: np.ndarray, d: np.ndarray) -> np.ndarray:
    # Coulomb minus half exchange of a symmetric active density, used only to
    # dress the active-space one-electron operator for the CASCI.
    return np.einsum("rstu,tu->rs", eri_act, d) - 0.5 * np.einsum("ruts,tu->rs", eri_act, d)


DENSE_CASCI_MAX = 20000     # determinants: dense CASCI and spin-pattern RDMs up to here


def _default_device() -> str:
    try:
        import torch
        return "cuda" if torch.cuda.is_available() else "cpu"
    except ImportError:
        return "cpu"


def _release_device(dev: str) -> None:
    if str(dev).startswith("cuda"):
        import torch
        torch.cuda.empty_cache()


def make_problem(nclosed: int, nact: int, nvirt: int, naux: int, nstate: int,
                 seed: int, nelact: int | None = None, decay: float = 10.0,
                 kmax: int = 4, device: str | None = None, fast: bool | None = None,
                 df_device: str | None = None) -> Problem:
    """Build one seeded problem.  nelact defaults to nact (half filling).  Active spaces
    above DENSE_CASCI_MAX determinants (or any, with fast=True) use the Davidson /
    Gram-matrix path of synth.casci_fast on `device` (default: the GPU when present).
    df_device: form the DF factors' product on that torch device (see df_factors)."""
    if nelact is None:
        nelact = nact
    rng = np.random.Generator(np.random.PCG64(seed))
    nmo = nclosed + nact + nvirt
    B = df_factors(rng, naux, nmo, decay, device=df_device)
    eps_c = np.sort(rng.uniform(-2.5, -0.4, nclosed))
    eps_v = np.sort(np.exp(rng.uniform(math.log(0.2), math.log(4.0), nvirt)))
    t = rng.uniform(-0.3, 0.3, (nact, nact))
    t_act = np.triu(t) + np.triu(t, 1).T

    f = np.zeros((nmo, nmo))
    f[np.arange(nclosed), np.arange(nclosed)] = eps_c
    ov = nclosed + nact
    f[np.arange(ov, nmo), np.arange(ov, nmo)] = eps_v

    if nact == 0:
        return Problem(nclosed, 0, nvirt, naux, 1 if nstate < 1 else nstate, 0, seed, f, B,
                       np.ones((1, 1)), np.zeros(1, dtype=np.int64), np.zeros(1, dtype=np.int64),
                       np.zeros(1), {k: np.zeros((1, 1, 0)) for k in range(1, kmax + 1)})

    act = slice(nclosed, ov)
    Bact = B[:, act, act].reshape(naux, nact * nact)
    eri_act = (Bact.T @ Bact).reshape(nact, nact, nact, nact)
    d_guess = (nelact / nact) * np.eye(nact)
    fc_act = t_act - _active_meanfield(eri_act, d_guess)

    space = ActiveSpace(nact, nelact)
    if not fast and (fast is not None or space.ndet <= DENSE_CASCI_MAX):
        e_cas, ci = lowest_singlets(space, fc_act, eri_act, nstate)
        rdm = {k: space.rdm(ci, k) for k in range(1, kmax + 1)}
    else:
        # large active spaces: Davidson CASCI and Gram-matrix RDMs (on a GPU when present)
        from .casci_fast import BigSpace, davidson_singlets, rdms
        dev = device if device is not None else _default_device()
        big = BigSpace(nact, nelact, dev)
        e_cas, ci = davidson_singlets(big, fc_act, eri_act, nstate)
        rdm = {k: v.cpu().numpy() for k, v in rdms(big, ci, kmax).items()}
        del big
        _release_device(dev)
    g1 = rdm[1].reshape(nstate, nstate, nact, nact)
    d_sa = sum(g1[m, m] for m in range(nstate)) / nstate
    f[act, act] = fc_act + _active_meanfield(eri_act, d_sa)
    da, db = space.det_strings()
    return Problem(nclosed, nact, nvirt, naux, nstate, nelact, seed, f, B, ci, da, db, e_cas,
                   {k: v.reshape(nstate, nstate, -1) for k, v in rdm.items()})


# Named workloads (sizes follow the synthetic copper-corrole / benzophenone
# shapes and the small parity case).
WORKLOADS = {
    "c4a4v20x84n2": dict(nclosed=4, nact=4, nvirt=20, naux=84, nstate=2, seed=0, decay=10.0),
    "c20a8v200x700n3": dict(nclosed=20, nact=8, nvirt=200, naux=700, nstate=3, seed=1, decay=10.0),
    # copper-corrole shape: 10 active orbitals, 10 electrons (63504 determinants)
    "c70a10v600x2000n5": dict(nclosed=70, nact=10, nvirt=600, naux=2000, nstate=5, seed=4,
                              decay=40.0),
    # benzophenone shape: 12 active orbitals, 12 electrons (853776 determinants)
    "c42a12v350x1200n4": dict(nclosed=42, nact=12, nvirt=350, naux=1200, nstate=4, seed=3,
                              decay=10.0),
}
