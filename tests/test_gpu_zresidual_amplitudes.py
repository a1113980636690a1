"""A bound on the library's first-order amplitudes that does not depend on the
conditioning of the denominators: the residual of the GPU's T_LN (caspt2_get_amplitudes,
classes A-G, every L and N) in the amplitude equation of the RDM-form oracle (Eq. ampeq,
in each class's own sector metric: oracle/o2_classes.class_residual), relative to the
sources.

The element-by-element comparison in test_gpu_amplitudes.py allows, for ill-conditioned
classes, 1000 times the oracle's own response to a 1e-15 perturbation of f: an error of a
sector eigenvalue at the rounding level moves T along the directions where the equation
is nearly singular.  Such an error leaves the residual near the rounding level, while an
error of the algebra or of the arithmetic would not: the oracle's own amplitudes give
1e-16 to 4e-12 here; the oracle's amplitudes for f perturbed by 1e-15 to 1e-12 relative
(which move the ill-conditioned class-B amplitudes of the ragged SS-SR case by up to
4e-9) give at most 3e-11 in the unperturbed metric; a 1e-6 relative change of T gives 3e-7
or more.  The bound applied, 5e-9, leaves room for the library's S, F and sources, whose
rounding is up to ~30 times the oracle's, and is still far below what the widened
element tolerance admits."""
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
BOUND = 5e-9


@pytest.fixture(scope="module")
def cp():
    from paper_1606_01273_gb300 import build as b
    if not os.path.exists(b.LIB):
        b.build()
    import paper_1606_01273_gb300 as cp
    return cp


def _oracle(p, opt):
    st = o2.setup(p, xms=bool(opt["xms"]), kmax=4)
    sch = "sssr" if opt["scheme"] == 1 else "msmr"
    mom = oc.all_moments(p, st, shift=opt["shift"], scheme=sch)
    parts = {c: (-np.einsum("llk->lk", M1), np.diagonal(M2).copy()) for c, (M1, M2, M3) in mom.items()}
    _, _, R = o2.heff(st, parts, opt["shift"])
    return st, sch, R


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("opt", OPTS, ids=["xms_msmr_P0", "xms_sssr_P1"])
def test_amplitude_residual_in_oracle_metric(cp, name, opt):
    p = make_problem(**CASES[name])
    st, sch, R = _oracle(p, opt)
    n = p.nstate
    ctx = cp.Context(p.nclosed, p.nact, p.nvirt, p.naux, p.nstate, **opt)
    try:
        ctx.set_inputs(*cp.problem_inputs(p))
        ctx.solve()
        for k, cls in enumerate("ABCDEFG"):
            Tref, _ = oc.class_amplitudes(p, st, cls, opt["shift"], sch, R, opt["target_state"])
            if Tref.size == 0 or not np.abs(Tref).max() > 0.0:
                continue
            own = oc.class_residual(p, st, cls, opt["shift"], sch, Tref)
            assert own <= 1e-11, (cls, own)                 # the oracle's own solve
            T = np.zeros_like(Tref)
            for L in range(n):
                for N in range(n):
                    T[L][..., N] = ctx.amplitudes(k, L, N).reshape(Tref[L][..., N].shape)
            res = oc.class_residual(p, st, cls, opt["shift"], sch, T)
            assert res <= BOUND, (cls, res)
    finally:
        ctx.close()
