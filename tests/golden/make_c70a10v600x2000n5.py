"""Write tests/golden/c70a10v600x2000n5.json: the RDM-form oracle's results for the
copper-corrole-shaped workload (nclosed 70, nact 10 with 10 electrons, nvirt 600, naux
2000, 5 states; XMS, MS-MR, vertical shift 0.3 Eh, target state 0).

Calls only synth (the seeded inputs) and oracle/ (O2: the class matrices from the
normal-ordering engine, evaluated with numpy).  Classes D, E, F and G take their sources
in groups of one external index and class H its pair integrals in groups of closed
orbitals (oracle options that only order the sums), so that the host holds one group at a
time.  The inputs are generated on the GPU when one is present (the Davidson CASCI and
the RDM Gram matrices of synth.casci_fast), so the file records fingerprints of the
inputs; the tests compare against these values only when the regenerated inputs match.

Run: python tests/golden/make_c70a10v600x2000n5.py   (about 15-30 min; ~100 GB host RAM)
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
from synth.fingerprint import input_fingerprint            # noqa: E402
from oracle import o2_rdm as o2                            # noqa: E402
from oracle import o2_classes as oc                        # noqa: E402

NAME = "c70a10v600x2000n5"
OPTS = dict(xms=True, scheme="msmr", shift=0.3, target=0)
CHUNKS = {"D": ("i", 10), "E": ("a", 60), "G": ("i", 5)}
I_CHUNK = 10


def main(out_path: str) -> None:
    t0 = time.time()
    p = make_problem(**WORKLOADS[NAME])
    t_gen = time.time() - t0
    fp = input_fingerprint(p)
    t = time.time()
    st = o2.setup(p, xms=OPTS["xms"], kmax=4)
    timing = {"setup": time.time() - t}
    mom = {}
    for cls in "ABCDEFG":
        t = time.time()
        mom[cls] = oc.class_moments(p, st, cls, OPTS["shift"], OPTS["scheme"], chunk=CHUNKS.get(cls))
        timing[cls] = time.time() - t
        print(cls, "%.1fs" % timing[cls], flush=True)
    t = time.time()
    mom["H"] = o2.class_h_moments(p, st, shift=OPTS["shift"], scheme=OPTS["scheme"],
                                  i_chunk=I_CHUNK)
    timing["H"] = time.time() - t
    parts = {c: (-np.einsum("llk->lk", M1), np.diagonal(M2).copy()) for c, (M1, M2, M3) in mom.items()}
    H, w, R = o2.heff(st, parts, OPTS["shift"])
    lam = {c: oc.lambda_pieces(*mom[c], R, OPTS["target"], OPTS["shift"]) for c in mom}
    res = {
        "workload": NAME, "options": OPTS, "fingerprint": fp,
        "U": st.U.tolist(), "E0": st.E0.tolist(), "Href": st.Href.tolist(), "Ecore": st.Ecore,
        "Heff": H.tolist(), "Ems": w.tolist(), "R": R.tolist(),
        "e_class": {c: parts[c][0].tolist() for c in parts},
        "norm_class": {c: parts[c][1].tolist() for c in parts},
        "M3": {c: np.asarray(mom[c][2]).tolist() for c in mom},
        "lam_NL": {c: lam[c][0].tolist() for c in lam},
        "lam_lv": {c: lam[c][1].tolist() for c in lam},
        "oracle_seconds": timing, "generation_seconds": t_gen,
        "host_cores": len(os.sched_getaffinity(0)),
    }
    with open(out_path, "w") as fh:
        json.dump(res, fh, indent=1)
    print("wrote", out_path, "E_MS", w, flush=True)


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else
         os.path.join(os.path.dirname(os.path.abspath(__file__)), NAME + ".json"))
