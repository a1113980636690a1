"""Write tests/golden/c20a8v200x700n3_densities.json: the RDM-form oracle's correlated
densities of target state 0 (Sec. II.D: d1, d2 on the closed-closed, active-active and
virtual-virtual blocks, GDF = D1 contracted with B) for the workload nclosed 20, nact 8
(8 electrons), nvirt 200, naux 700, 3 states; XMS, MS-MR, vertical shift 0.2 Eh.

Calls only synth (the seeded inputs) and oracle/ (O2: every class's densities, summed in
class order A..H, each symmetrised as the library returns them).  The file keeps what a
test needs to compare element by element without storing whole matrices: the Frobenius
norm of every block of d1 and d2 and of every orbital-space block of GDF, a fixed seeded
sample of elements from every nonzero block, the oracle's E_MS, and sums of the inputs (so
that a test can tell that the regenerated inputs are the same to rounding).

Run: python tests/golden/make_c20a8v200x700n3_densities.py   (a few minutes on 8 cores)
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from synth import make_problem, WORKLOADS                  # noqa: E402
from oracle import o2_rdm as o2                            # noqa: E402
from oracle import o2_classes as oc                        # noqa: E402

NAME = "c20a8v200x700n3"
OPTS = dict(xms=True, scheme="msmr", shift=0.2, target=0)
SAMPLES = 300          # elements per block of d1 / d2
GDF_SAMPLES = 2000


def spaces(p):
    c, a = p.nclosed, p.nact
    return {"c": slice(0, c), "a": slice(c, c + a), "v": slice(c + a, p.nmo)}


def input_sums(p):
    return {"f": float(np.sum(p.f)), "f_abs": float(np.sum(np.abs(p.f))),
            "B": float(np.sum(p.B)), "B_abs": float(np.sum(np.abs(p.B))),
            **{f"rdm{k}": float(np.sum(p.rdm[k])) for k in sorted(p.rdm)},
            **{f"rdm{k}_abs": float(np.sum(np.abs(p.rdm[k]))) for k in sorted(p.rdm)}}


def main(out_path: str) -> None:
    t0 = time.time()
    p = make_problem(**WORKLOADS[NAME])
    t_gen = time.time() - t0
    t = time.time()
    st = o2.setup(p, xms=OPTS["xms"], kmax=4)
    mom = oc.all_moments(p, st, shift=OPTS["shift"], scheme=OPTS["scheme"])
    parts = {c: (-np.einsum("llk->lk", M1), np.diagonal(M2).copy()) for c, (M1, M2, M3) in mom.items()}
    _, w, R = o2.heff(st, parts, OPTS["shift"])
    d1 = np.zeros((p.nmo, p.nmo))
    d2 = np.zeros((p.nmo, p.nmo))
    gdf = np.zeros_like(p.B)
    for cls in "ABCDEFG":
        r1, rG, r2, _ = oc.class_densities(p, st, cls, OPTS["shift"], OPTS["scheme"], R, OPTS["target"])
        d1 += r1
        d2 += r2
        gdf += rG
        print(cls, "%.1fs" % (time.time() - t), flush=True)
    r2, rG, _ = o2.class_h_densities(p, st, R, OPTS["target"], OPTS["shift"], OPTS["scheme"])
    d2 += r2
    gdf += rG
    oracle_s = time.time() - t
    sym = lambda x: 0.5 * (x + np.swapaxes(x, -1, -2))   # noqa: E731
    d1, d2, gdf = sym(d1), sym(d2), sym(gdf)
    sp = spaces(p)
    rng = np.random.default_rng(20)
    blocks = {}
    for name, m in (("d1", d1), ("d2", d2)):
        for x in "cav":
            for y in "cav":
                blk = m[sp[x], sp[y]]
                ent = {"fro": float(np.linalg.norm(blk))}
                if ent["fro"] > 0.0:
                    i = rng.integers(0, blk.shape[0], SAMPLES)
                    j = rng.integers(0, blk.shape[1], SAMPLES)
                    ent["i"] = i.tolist()
                    ent["j"] = j.tolist()
                    ent["val"] = blk[i, j].tolist()
                blocks[f"{name}_{x}{y}"] = ent
    for x in "cav":
        for y in "cav":
            blk = gdf[:, sp[x], sp[y]]
            blocks[f"gdf_{x}{y}"] = {"fro": float(np.linalg.norm(blk))}
    q = rng.integers(0, p.naux, GDF_SAMPLES)
    i = rng.integers(0, p.nmo, GDF_SAMPLES)
    j = rng.integers(0, p.nmo, GDF_SAMPLES)
    res = {
        "workload": NAME, "options": OPTS, "inputs": input_sums(p),
        "Ems": w.tolist(), "R": R.tolist(), "blocks": blocks,
        "gdf_sample": {"q": q.tolist(), "i": i.tolist(), "j": j.tolist(),
                       "val": gdf[q, i, j].tolist()},
        "oracle_seconds": oracle_s, "generation_seconds": t_gen,
        "host_cores": len(os.sched_getaffinity(0)),
    }
    with open(out_path, "w") as fh:
        json.dump(res, fh)
    print("wrote", out_path, "E_MS", w, "oracle %.0fs" % oracle_s, flush=True)


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else
         os.path.join(os.path.dirname(os.path.abspath(__file__)), NAME + "_densities.json"))
