"""One solve split over closed-orbital ranges (the multi-GPU design of the path, run here
as consecutive partial solves on one GPU): each partition solves the class-H pairs and
class-G tuples of its closed orbitals (classes A-F on the partition that starts at 0),
the per-class moments of the partitions are summed in partition order, and H^eff, E_MS,
R and the lambda pieces formed from the sum equal the whole solve's."""
import os

import numpy as np
import pytest

from synth import make_problem
from paper_1606_01273_gb300.shard import closed_range, sum_moments_fixed_order

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cp():
    from paper_1606_01273_gb300 import build as b
    if not os.path.exists(b.LIB):
        b.build()
    import paper_1606_01273_gb300 as cp
    return cp


@pytest.mark.parametrize("parts", [2, 3])
@pytest.mark.parametrize("opt", [dict(xms=1, scheme=0, shift=0.2), dict(xms=0, scheme=1, shift=0.1),
                                 dict(xms=1, scheme=0, shift=0.2, precision=1, slices=7)],
                         ids=["xms_msmr", "ms_sssr", "xms_msmr_split_bf16"])
def test_partial_solves_sum_to_the_whole(cp, parts, opt):
    p = make_problem(nclosed=5, nact=3, nvirt=70, naux=37, nstate=3, seed=21, nelact=2)
    whole = cp.solve_problem(p, **opt)
    ctxs, moms = [], []
    try:
        for r in range(parts):
            lo, hi = closed_range(p.nclosed, r, parts)
            ctx = cp.Context(p.nclosed, p.nact, p.nvirt, p.naux, p.nstate, closed_begin=lo,
                             closed_end=hi, **opt)
            ctx.set_inputs(*cp.problem_inputs(p))
            ctx.solve()
            moms.append(ctx.moments())
            ctxs.append(ctx)
        tot = moms[0].copy()
        for m in moms[1:]:
            tot += m
        assert np.array_equal(tot, sum_moments_fixed_order(tot))    # one process: identity
        st = ctxs[0].finalize_moments(tot)
        r = ctxs[0].result(st)
        # a partial solve has no densities or amplitudes of its own
        with pytest.raises(cp.CASPT2Error):
            ctxs[1].compute_densities()
    finally:
        for c in ctxs:
            c.close()
    scale = max(1.0, np.abs(whole.Ems).max())
    assert np.abs(r.Ems - whole.Ems).max() <= 1e-11 * scale
    assert np.abs(r.Heff - whole.Heff).max() <= 1e-11 * scale
    assert np.abs(r.R - whole.R).max() <= 1e-9
    for cls in "ABCDEFGH":
        s = max(1.0, np.abs(whole.e_class[cls]).max())
        assert np.abs(r.e_class[cls] - whole.e_class[cls]).max() <= 1e-11 * s, cls
        assert np.abs(r.lam_NL[cls] - whole.lam_NL[cls]).max() <= 1e-10 * max(1.0, np.abs(whole.lam_NL[cls]).max()), cls
