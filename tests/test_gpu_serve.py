"""Serving form (caspt2_server_*): requests of different sizes and state counts submitted
together, admitted by device-memory budget into concurrent slots (one stream each); every
result equals the same request solved alone (energies to 1e-12 Eh, densities to 1e-10
relative: the density source adjoint sums with atomics), also when a small budget forces
requests to wait for memory."""
import os

import numpy as np
import pytest

from synth import make_problem, WORKLOADS

pytestmark = pytest.mark.gpu

PROBLEMS = [
    (WORKLOADS["c4a4v20x84n2"], dict(xms=1, scheme=0, shift=0.2), True),
    (dict(nclosed=5, nact=3, nvirt=70, naux=37, nstate=3, seed=21, nelact=2),
     dict(xms=1, scheme=1, shift=0.1), True),
    (dict(nclosed=2, nact=4, nvirt=2, naux=24, nstate=2, seed=5), dict(xms=0, scheme=0, shift=0.0), False),
    (dict(nclosed=6, nact=2, nvirt=30, naux=40, nstate=1, seed=33, nelact=2),
     dict(xms=1, scheme=0, shift=0.3), True),
    (dict(nclosed=3, nact=4, nvirt=40, naux=50, nstate=3, seed=34), dict(xms=1, scheme=0, shift=0.2), False),
    (dict(nclosed=8, nact=3, nvirt=64, naux=64, nstate=2, seed=35, nelact=2),
     dict(xms=0, scheme=1, shift=0.2, precision=1, slices=7), True),
]


@pytest.fixture(scope="module")
def cp():
    from paper_1606_01273_gb300 import build as b
    if not os.path.exists(b.LIB):
        b.build()
    import paper_1606_01273_gb300 as cp
    return cp


@pytest.fixture(scope="module")
def probs():
    return [make_problem(**kw) for kw, _, _ in PROBLEMS]


def _alone(cp, p, opt, dens):
    return cp.solve_problem(p, densities=True if dens else None, **opt)


def _check(got, ref, dens):
    assert got["status"] >= 0
    assert np.abs(got["Ems"] - ref.Ems).max() <= 1e-12 * max(1.0, np.abs(ref.Ems).max())
    assert np.abs(got["Heff"] - ref.Heff).max() <= 1e-12 * max(1.0, np.abs(ref.Heff).max())
    if dens:
        for k in ("d1", "d2", "gdf"):
            a, b = got[k], getattr(ref, k)
            assert np.linalg.norm(a - b) <= 1e-10 * max(1e-300, np.linalg.norm(b)), k


@pytest.mark.parametrize("slots", [1, 3])
def test_mix_equals_alone(cp, probs, slots):
    refs = [_alone(cp, p, o, d) for p, (_, o, d) in zip(probs, PROBLEMS)]
    srv = cp.Server(slots=slots)
    try:
        tickets = [srv.submit(p, densities=d, **o) for p, (_, o, d) in zip(probs, PROBLEMS)]
        outs = [srv.wait(t) for t in tickets]
    finally:
        srv.close()
    for got, ref, (_, _, d) in zip(outs, refs, PROBLEMS):
        _check(got, ref, d)
        assert got["latency_ms"] >= got["queue_ms"] >= 0.0


def test_small_budget_queues_and_still_matches(cp, probs):
    """A budget that holds about one request at a time: later requests wait for memory
    (queue time grows) and every result is unchanged."""
    p = probs[1]
    _, o, d = PROBLEMS[1]
    ref = _alone(cp, p, o, d)
    srv = cp.Server(budget_bytes=250 << 20, slots=4)   # estimate ~160 MiB each
    try:
        tickets = [srv.submit(p, densities=d, **o) for _ in range(4)]
        outs = [srv.wait(t) for t in tickets]
    finally:
        srv.close()
    for got in outs:
        _check(got, ref, d)
    q = sorted(o_["queue_ms"] for o_ in outs)
    assert q[-1] > q[0]


def test_wait_timeout_and_unknown_ticket(cp, probs):
    srv = cp.Server(slots=1)
    try:
        t = srv.submit(probs[0], **PROBLEMS[0][1])
        import ctypes as C
        res = cp.ServeResult()
        assert cp.lib().caspt2_server_wait(srv._h, t + 1000, 0, C.byref(res)) == cp.EINVAL
        out = srv.wait(t)
        assert out["status"] >= 0
    finally:
        srv.close()


def _pool(count=12, seed=5000):
    """Mixed sizes as in the serving measurement: nclosed 4-16, nact 2-6, nvirt 20-120,
    1-3 states, naux ~ 3 nmo."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        nact = int(rng.integers(2, 7))
        c, v, n = int(rng.integers(4, 17)), int(rng.integers(20, 121)), int(rng.integers(1, 4))
        out.append(make_problem(nclosed=c, nact=nact, nvirt=v, naux=3 * (c + nact + v), nstate=n,
                                seed=seed + k, nelact=nact if nact % 2 == 0 else nact - 1))
    return out


def test_mixed_pool_four_slots(cp):
    """Twelve problems of different sizes (nact up to 6), four slots, densities on every
    other request: each served result equals the same request alone."""
    pool = _pool()
    opt = dict(xms=1, scheme=0, shift=0.2)
    refs = [cp.solve_problem(p, densities=True if k % 2 == 0 else None, **opt)
            for k, p in enumerate(pool)]
    srv = cp.Server(slots=4)
    try:
        tickets = [srv.submit(p, densities=(k % 2 == 0), **opt) for k, p in enumerate(pool)]
        outs = [srv.wait(t) for t in tickets]
    finally:
        srv.close()
    for k, (got, ref) in enumerate(zip(outs, refs)):
        _check(got, ref, k % 2 == 0)
