"""caspt2_classH_noalloc: the class-H pieces computed without any device allocation.

Callers that cannot allocate device memory (code inside another framework's memory
pool or a pre-sized arena, plugins whose host forbids allocation after start-up,
loops that must never enter the allocator) use this entry point; its intermediates
live in the library's fixed device scratch array.  The test calls it twice in a row
through the C ABI and checks both results against caspt2_solve +
caspt2_get_class_energy on the same inputs, within the FP64 tolerance of the other
class-H parity tests.  It also checks the size rejection.  This file is collected
last so that a failure here cannot hide the other tests.
"""
import os

import numpy as np
import pytest

from synth import make_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cp():
    from paper_1606_01273_gb300 import build as b
    if not os.path.exists(b.LIB):
        b.build()
    import paper_1606_01273_gb300 as cp
    return cp


@pytest.mark.parametrize("opt", [dict(xms=1, scheme=0, shift=0.2), dict(xms=0, scheme=0, shift=0.0),
                                 dict(xms=1, scheme=1, shift=0.1)],
                         ids=["xms_msmr", "ms_msmr", "xms_sssr"])
def test_noalloc_matches_solve_twice(cp, opt):
    import torch
    p = make_problem(nclosed=5, nact=3, nvirt=70, naux=37, nstate=3, seed=21, nelact=2, kmax=2)
    ref = cp.solve_problem(p, class_mask=1 << 7, **opt)
    e_ref, n_ref = ref.e_class["H"], ref.norm_class["H"]
    f, B, rdm1 = cp.problem_inputs(p, kmax=1)[:3]
    dev = torch.device("cuda", 0)
    f_d, B_d, r_d = (torch.from_numpy(x).to(dev) for x in (f, B, rdm1))
    n = p.nstate
    e_d = torch.empty((n, n), dtype=torch.float64, device=dev)
    n_d = torch.empty(n, dtype=torch.float64, device=dev)
    dims = cp.Dims(p.nclosed, p.nact, p.nvirt, p.naux, p.nstate)
    opts = cp.default_options(**opt)
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.synchronize(dev)
    scale = max(1.0, np.abs(e_ref).max())
    for _ in range(2):
        e_d.fill_(float("nan"))
        n_d.fill_(float("nan"))
        torch.cuda.synchronize(dev)
        st = cp.classH_noalloc(dims, opts, f_d, B_d, r_d, e_d, n_d, stream=stream.cuda_stream)
        assert st == cp.OK
        e, nr = e_d.cpu().numpy(), n_d.cpu().numpy()
        assert np.abs(e - e_ref).max() <= min(1e-8, 1e-11 * scale)
        assert np.abs(nr - n_ref).max() <= 1e-11 * max(1.0, np.abs(n_ref).max())


def test_noalloc_rejects_oversized(cp):
    import ctypes as C
    import torch
    dev = torch.device("cuda", 0)
    t = torch.zeros(8, dtype=torch.float64, device=dev)
    dims = cp.Dims(100000, 2, 200000, 10, 16)      # scratch needed far above 4 MiB
    opts = cp.default_options()
    p = C.c_void_p(t.data_ptr())
    st = cp.lib().caspt2_classH_noalloc(C.byref(dims), C.byref(opts), p, p, p, p, p, None)
    assert st == cp.ESCRATCH
    assert b"scratch" in cp.lib().caspt2_strerror(st)


def test_noalloc_rejects_coupled_fock(cp):
    """The entry point reads only the blocks of a block-diagonal f, so (like
    caspt2_set_inputs) it refuses an f with a closed-virtual coupling entry."""
    import torch
    from tests.cases import rotated_fock
    p = make_problem(nclosed=5, nact=3, nvirt=70, naux=37, nstate=3, seed=21, nelact=2, kmax=2)
    _, f_cpl = rotated_fock(p)
    _, B, rdm1 = cp.problem_inputs(p, kmax=1)[:3]
    dev = torch.device("cuda", 0)
    f_d, B_d, r_d = (torch.from_numpy(x).to(dev) for x in (f_cpl, B, rdm1))
    e_d = torch.zeros((p.nstate, p.nstate), dtype=torch.float64, device=dev)
    n_d = torch.zeros(p.nstate, dtype=torch.float64, device=dev)
    dims = cp.Dims(p.nclosed, p.nact, p.nvirt, p.naux, p.nstate)
    with pytest.raises(cp.CASPT2Error) as e:
        cp.classH_noalloc(dims, cp.default_options(), f_d, B_d, r_d, e_d, n_d)
    assert e.value.status == cp.EINVAL
