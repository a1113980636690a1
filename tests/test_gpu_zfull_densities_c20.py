"""Correlated densities of target state 0 (Sec. II.D: d1, d2 on the closed-closed,
active-active and virtual-virtual blocks, GDF = D1 contracted with B) at the workload
nclosed 20, nact 8 (8 electrons), nvirt 200, naux 700, 3 states (XMS, MS-MR, shift
0.2 Eh), through the C ABI, element by element against the RDM-form oracle's stored
values (tests/golden/c20a8v200x700n3_densities.json, written by
make_c20a8v200x700n3_densities.py from synth and oracle/ alone), in the plain FP64 form
and in the split-BF16 form with 7 slices.

Tolerance 1e-6 relative (the densities' bar): the Frobenius norm of every block, and a
seeded sample of elements of every nonzero block against the largest sampled magnitude of
that block (GDF: a sample over all of it).  The stored file records sums of the inputs;
the regenerated inputs must agree with them to 1e-10 relative (the generator's linear
algebra may round differently from one machine to another, far below what moves the
densities at this tolerance)."""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(ROOT, "tests", "golden", "c20a8v200x700n3_densities.json")
RTOL = 1e-6


@pytest.fixture(scope="module")
def golden():
    with open(GOLDEN) as fh:
        return json.load(fh)


@pytest.fixture(scope="module")
def prob(golden):
    from synth import make_problem, WORKLOADS
    p = make_problem(**WORKLOADS[golden["workload"]])
    arrays = {"f": p.f, "B": p.B, **{f"rdm{k}": p.rdm[k] for k in p.rdm}}
    for key, want in golden["inputs"].items():
        base = key[:-4] if key.endswith("_abs") else key
        x = arrays[base]
        got = float(np.sum(np.abs(x))) if key.endswith("_abs") else float(np.sum(x))
        scale = golden["inputs"][base + "_abs"]
        assert abs(got - want) <= 1e-10 * scale, (key, got, want)
    return p


@pytest.fixture(scope="module")
def cp():
    from paper_1606_01273_gb300 import build as b
    if not os.path.exists(b.LIB):
        b.build()
    import paper_1606_01273_gb300 as cp
    return cp


def _spaces(p):
    c, a = p.nclosed, p.nact
    return {"c": slice(0, c), "a": slice(c, c + a), "v": slice(c + a, p.nmo)}


@pytest.mark.parametrize("precision", ["fp64", "bf16x"])
def test_densities_vs_stored_oracle(cp, golden, prob, precision):
    p = prob
    o = golden["options"]
    opt = dict(xms=int(o["xms"]), scheme=0 if o["scheme"] == "msmr" else 1, shift=o["shift"],
               target_state=o["target"],
               precision=cp.BF16X if precision == "bf16x" else cp.FP64, slices=7)
    r = cp.solve_problem(p, densities=True, **opt)
    assert np.abs(r.R - np.array(golden["R"])).max() <= 1e-6
    sp = _spaces(p)
    mats = {"d1": r.d1, "d2": r.d2}
    top = {}
    for key, ent in golden["blocks"].items():
        top[key.split("_")[0]] = max(top.get(key.split("_")[0], 0.0), ent["fro"])
    for key, ent in golden["blocks"].items():
        name, (x, y) = key.split("_")[0], key.split("_")[1]
        blk = r.gdf[:, sp[x], sp[y]] if name == "gdf" else mats[name][sp[x], sp[y]]
        fro = float(np.linalg.norm(blk))
        if ent["fro"] == 0.0:
            # blocks the method leaves empty (d2 between spaces without dens_offdiag)
            assert fro <= 1e-12 * top[name], (key, fro)
            continue
        assert abs(fro - ent["fro"]) <= RTOL * ent["fro"], (key, fro, ent["fro"])
        if "val" in ent:
            want = np.array(ent["val"])
            got = blk[np.array(ent["i"]), np.array(ent["j"])]
            scale = float(np.abs(want).max())
            assert float(np.abs(got - want).max()) <= RTOL * scale, (key, scale)
    s = golden["gdf_sample"]
    want = np.array(s["val"])
    got = r.gdf[np.array(s["q"]), np.array(s["i"]), np.array(s["j"])]
    assert float(np.abs(got - want).max()) <= RTOL * float(np.abs(want).max())
