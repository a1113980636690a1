"""GPU parity of the setup stage and the direct class-H kernel against the RDM-form
oracle (itself pinned to brute force), through the C ABI."""
import numpy as np
import pytest

from synth import make_problem, WORKLOADS
from oracle import o2_rdm as o2

pytestmark = pytest.mark.gpu

# (name, generator kwargs): the small parity workload, a ragged case (virtuals not a
# multiple of the 64-wide tile, DF index not a multiple of the 16-deep chunk, odd
# state count), nact = 0, and the full benzophenone-like bench workload.
CASES = {
    "c4a4v20x84n2": WORKLOADS["c4a4v20x84n2"],
    "ragged_c5a3v70x37n3": dict(nclosed=5, nact=3, nvirt=70, naux=37, nstate=3, seed=21, nelact=2),
    "nact0_c6v50x40": dict(nclosed=6, nact=0, nvirt=50, naux=40, nstate=1, seed=22),
    "c20a8v200x700n3": WORKLOADS["c20a8v200x700n3"],
}
H_ONLY = 1 << 7
OPTS = [dict(xms=1, scheme=0, shift=0.0, class_mask=H_ONLY), dict(xms=1, scheme=0, shift=0.2, class_mask=H_ONLY),
        dict(xms=0, scheme=0, shift=0.2, class_mask=H_ONLY), dict(xms=1, scheme=1, shift=0.2, class_mask=H_ONLY)]

ETOL = 1e-8   # |dE| bound on energies (Eh)


@pytest.fixture(scope="module")
def cp():
    import os
    from paper_1606_01273_gb300 import build as b
    if not os.path.exists(b.LIB):
        b.build()
    import paper_1606_01273_gb300 as cp
    return cp


_probs = {}


def _prob(name):
    if name not in _probs:
        _probs[name] = make_problem(**CASES[name], kmax=2)
    return _probs[name]


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("opt", OPTS, ids=lambda o: f"xms{o['xms']}_sch{o['scheme']}_s{o['shift']}")
def test_class_h_parity(cp, name, opt):
    p = _prob(name)
    if p.nstate == 1 and opt["xms"] == 0 and opt["scheme"] == 1:
        pytest.skip("identical to the n = 1 XMS case")
    r = cp.solve_problem(p, **opt)
    st = o2.setup(p, xms=bool(opt["xms"]))
    sch = "sssr" if opt["scheme"] == 1 else "msmr"
    e, nr = o2.class_h(p, st, shift=opt["shift"], scheme=sch)
    H, w, R = o2.heff(st, {"H": (e, nr)}, opt["shift"])
    scale = max(1.0, np.abs(e).max())
    assert abs(r.Ecore - st.Ecore) <= 1e-10 * max(1.0, abs(st.Ecore))
    assert np.allclose(r.U, st.U, atol=1e-12)
    assert np.allclose(r.E0, st.E0, atol=1e-12)
    assert np.abs(r.Href - st.Href).max() <= min(ETOL, 1e-11 * max(1.0, np.abs(st.Href).max()))
    assert np.abs(r.e_class["H"] - e).max() <= min(ETOL, 1e-11 * scale)
    assert np.abs(r.norm_class["H"] - nr).max() <= 1e-11 * max(1.0, np.abs(nr).max())
    assert np.abs(r.Heff - H).max() <= ETOL
    assert np.abs(r.Ems - w).max() <= ETOL
    assert np.allclose(np.abs(r.R), np.abs(R), atol=1e-8)
    assert r.launches > 0


def test_bitwise_reproducible(cp):
    p = _prob("ragged_c5a3v70x37n3")
    a = cp.solve_problem(p, shift=0.2, class_mask=H_ONLY)
    b = cp.solve_problem(p, shift=0.2, class_mask=H_ONLY)
    assert np.array_equal(a.Ems, b.Ems) and np.array_equal(a.e_class["H"], b.e_class["H"])


def test_device_resident_inputs_and_stream(cp):
    """Inputs passed as device pointers and a caller stream give the host-path result."""
    import torch
    p = _prob("c4a4v20x84n2")
    host = cp.problem_inputs(p, kmax=2)[:4]
    dev = [torch.from_numpy(x).cuda() for x in host]
    ctx = cp.Context(p.nclosed, p.nact, p.nvirt, p.naux, p.nstate, shift=0.1, class_mask=H_ONLY)
    s = torch.cuda.Stream()
    ctx.set_inputs(*dev)
    ctx.solve(stream=s.cuda_stream)
    r_dev = ctx.result()
    ctx.close()
    r_host = cp.solve_problem(p, shift=0.1, class_mask=H_ONLY)
    assert np.array_equal(r_dev.Ems, r_host.Ems)


def test_errors_are_status_codes(cp):
    import ctypes as C
    L = cp.lib()
    h = C.c_void_p()
    bad = cp.Dims(2, 2, 2, 4, 0)
    assert L.caspt2_create(C.byref(h), C.byref(bad), None) == cp.EINVAL
    ctx = cp.Context(2, 2, 2, 4, 1, class_mask=H_ONLY)
    assert L.caspt2_solve(ctx._h, None) == cp.ESTATE
    assert L.caspt2_get_energies(ctx._h, None, None, None, None, None, None) == cp.ESTATE
    with pytest.raises(cp.CASPT2Error):
        cp.Context(2, 2, 2, 4, 1, class_mask=1 << 9)   # no such class
    ctx.close()
