"""Fingerprints of a generated problem's inputs (to tell whether two runs of the
generator produced the same bytes): SHA-256 of f, of the 1-3 RDMs and of a fixed strided
sample of B and of the 4-RDM, with their full sums."""
from __future__ import annotations

import hashlib

import numpy as np


def _digest(x: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(x).tobytes()).hexdigest()[:32]


def input_fingerprint(p) -> dict:
    fp = {"f": _digest(p.f)}
    for k in (1, 2, 3):
        if k in p.rdm:
            fp[f"rdm{k}"] = _digest(p.rdm[k])
    for name, arr in (("B", p.B), ("rdm4", p.rdm.get(4))):
        if arr is None:
            continue
        flat = arr.reshape(-1)
        step = max(1, flat.size // 1000003)
        fp[name + "_sample"] = _digest(flat[::step])
        fp[name + "_sum"] = float(np.sum(flat))
    return fp
