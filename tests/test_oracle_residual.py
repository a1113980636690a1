"""The oracle's amplitude-equation residual (oracle/o2_classes.class_residual, Eq. ampeq
in each class's sector metric) on the oracle's own amplitudes: zero to rounding for the
amplitudes of the same problem (class_amplitudes solves in the sector eigenbasis; the
residual multiplies the explicit S and F), and clearly nonzero for the amplitudes of
another shift or after a 1e-6 relative change."""
import numpy as np
import pytest

from synth import make_problem, WORKLOADS
from oracle import o2_rdm as o2
from oracle import o2_classes as oc


@pytest.mark.parametrize("sch", ["msmr", "sssr"])
def test_class_residual(sch):
    p = make_problem(**WORKLOADS["c4a4v20x84n2"])
    st = o2.setup(p, xms=True, kmax=4)
    mom = oc.all_moments(p, st, shift=0.2, scheme=sch)
    parts = {c: (-np.einsum("llk->lk", M1), np.diagonal(M2).copy()) for c, (M1, M2, M3) in mom.items()}
    _, _, R = o2.heff(st, parts, 0.2)
    rng = np.random.default_rng(2)
    for cls in "ABCDEFG":
        T, _ = oc.class_amplitudes(p, st, cls, 0.2, sch, R, 0)
        assert oc.class_residual(p, st, cls, 0.2, sch, T) <= 1e-12, cls
        T2, _ = oc.class_amplitudes(p, st, cls, 0.25, sch, R, 0)
        assert oc.class_residual(p, st, cls, 0.2, sch, T2) >= 1e-4, cls
        T3 = T * (1.0 + 1e-6 * rng.standard_normal(T.shape))
        assert oc.class_residual(p, st, cls, 0.2, sch, T3) >= 1e-7, cls
