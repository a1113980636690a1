"""Spin-free matrix elements <M| E ... E |N> between reference states, reduced to
active-space RDMs.

TEST INFRASTRUCTURE (see oracle/__init__.py).  The reference states have the
closed orbitals doubly occupied and the virtual orbitals empty (Sec. II.A), so a
product of spin-free generators factorises into three strings:

  * closed-orbital operators: full contraction against the filled core,
    <a+_x a_y> = delta_xy (creator on the left), every other pairing zero;
  * virtual-orbital operators: full contraction against the empty space,
    <a_x a+_y> = delta_xy (annihilator on the left), every other pairing zero;
  * active operators: normal-ordered with a_p a+_q = delta_pq - a+_q a_p and read
    as spin-free RDMs Gamma_{p1q1,...,pkqk} = <M|sum a+_p1..a+_pk a_qk..a_q1|N>.

Each generator E_pq = sum_s a+_ps a_qs carries its own spin variable; contractions
identify spin variables, a variable left on no operator contributes a factor 2, and
the remaining active string pairs every creator with the annihilator of the same
variable, which fixes the RDM index order.  The output is a list of integer-weighted
terms (coefficient, Kronecker deltas between index labels, RDM index pairs).
"""
from __future__ import annotations

import itertools
from collections import defaultdict
from dataclasses import dataclass


@dataclass(frozen=True)
class Op:
    cre: bool      # True: creator a+, False: annihilator a
    label: str     # orbital index label
    spin: int      # spin variable


class Builder:
    """Generates fermion strings for products of spin-free generators."""

    def __init__(self):
        self._spin = itertools.count()

    def E(self, p: str, q: str):
        """E_pq = sum_s a+_ps a_qs."""
        s = next(self._spin)
        return [Op(True, p, s), Op(False, q, s)]

    def E2(self, p: str, q: str, r: str, t: str):
        """E_pq,rt = sum_{s,u} a+_ps a+_ru a_tu a_qs."""
        s, u = next(self._spin), next(self._spin)
        return [Op(True, p, s), Op(True, r, u), Op(False, t, u), Op(False, q, s)]


def _parity(perm):
    p = list(perm)
    sign = 1
    for i in range(len(p)):
        while p[i] != i:
            j = p[i]
            p[i], p[j] = p[j], p[i]
            sign = -sign
    return sign


def _full_contractions(ops, left_cre: bool):
    """All complete pairings of a string against a filled (left_cre=True: nonzero
    pairs are creator-left) or empty (left_cre=False: annihilator-left) vacuum.
    Yields (sign, label deltas, spin merges)."""
    if not ops:
        yield 1, [], []
        return
    if len(ops) % 2:
        return
    first = ops[0]
    if first.cre != left_cre:
        return
    for k in range(1, len(ops)):
        other = ops[k]
        if other.cre == first.cre:
            continue
        sign = -1 if (k - 1) % 2 else 1
        rest = ops[1:k] + ops[k + 1:]
        for s, d, m in _full_contractions(rest, left_cre):
            yield sign * s, [(first.label, other.label)] + d, [(first.spin, other.spin)] + m


def _normal_order(ops):
    """Creators to the left.  Returns [(coeff, label deltas, spin merges, ops)]."""
    for i in range(len(ops) - 1):
        if not ops[i].cre and ops[i + 1].cre:
            a, c = ops[i], ops[i + 1]
            out = [(-co, d, m, o) for co, d, m, o in _normal_order(ops[:i] + [c, a] + ops[i + 2:])]
            for co, d, m, o in _normal_order(ops[:i] + ops[i + 2:]):
                out.append((co, [(a.label, c.label)] + d, [(a.spin, c.spin)] + m, o))
            return out
    return [(1, [], [], ops)]


class _UF:
    def __init__(self):
        self.p = {}

    def find(self, x):
        self.p.setdefault(x, x)
        while self.p[x] != x:
            self.p[x] = self.p[self.p[x]]
            x = self.p[x]
        return x

    def union(self, a, b):
        ra, rb = self.find(a), self.find(b)
        if ra != rb:
            self.p[ra] = rb


@dataclass(frozen=True)
class Term:
    coeff: int
    deltas: tuple          # sorted tuple of sorted (label, label) pairs
    rdm: tuple             # ((p1, q1), ..., (pk, qk)) active labels; () = overlap <M|N>


def expect(ops, space: dict) -> list:
    """<M| ops |N> as a list of Terms.  `space` maps each label to 'c', 'a' or 'v'."""
    order = {"c": 0, "v": 1, "a": 2}
    idx = sorted(range(len(ops)), key=lambda i: (order[space[ops[i].label]], i))
    sign0 = _parity(idx)
    srt = [ops[i] for i in idx]
    core = [o for o in srt if space[o.label] == "c"]
    virt = [o for o in srt if space[o.label] == "v"]
    act = [o for o in srt if space[o.label] == "a"]
    all_spins = {o.spin for o in ops}
    acc = defaultdict(int)
    for s1, d1, m1 in _full_contractions(core, True):
        for s2, d2, m2 in _full_contractions(virt, False):
            for co, d3, m3, no in _normal_order(act):
                uf = _UF()
                for a, b in m1 + m2 + m3:
                    uf.union(a, b)
                cre = [o for o in no if o.cre]
                ann = [o for o in no if not o.cre]
                if len(cre) != len(ann):
                    continue
                live = {uf.find(o.spin) for o in no}
                free = {uf.find(s) for s in all_spins} - live
                # pair creator j with the annihilator of the same spin class
                pos = {}
                for j, o in enumerate(ann):
                    pos.setdefault(uf.find(o.spin), []).append(j)
                k = len(cre)
                target = []
                ok = True
                for j, o in enumerate(cre):
                    lst = pos.get(uf.find(o.spin), [])
                    if len(lst) != 1:
                        ok = False
                        break
                    target.append(lst[0])
                if not ok:
                    raise AssertionError("spin class not paired one creator / one annihilator")
                # annihilators must read a_{q_k} ... a_{q_1}: creator j pairs with ann slot k-1-j
                perm = [0] * k
                for j in range(k):
                    perm[k - 1 - j] = target[j]
                sgn = _parity(perm)
                rdm = tuple((cre[j].label, ann[target[j]].label) for j in range(k))
                deltas = tuple(sorted(tuple(sorted(x)) for x in d1 + d2 + d3))
                acc[(deltas, rdm)] += sign0 * s1 * s2 * co * sgn * (2 ** len(free))
    return [Term(c, d, r) for (d, r), c in acc.items() if c != 0]
