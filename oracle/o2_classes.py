"""O2 for the excitation classes A-G: overlap, Fock and source matrices from RDMs.

TEST INFRASTRUCTURE (see oracle/__init__.py).  Every matrix element is produced by
the normal-ordering engine in oracle/wick.py from the operator families of
Eq. (class) and evaluated with numpy.einsum over the rotated RDMs (Sec. II.F: the
RDMs <M~|E..|N~> are the only reference-state information the contractions use).

For block-diagonal f (closed and virtual blocks diagonal) a class's overlap and
Fock matrices couple external index tuples only through Kronecker deltas, i.e.
through the identity or, for classes with two closed (or two virtual) indices, the
swap of that pair.  The class is then solved per external tuple in the symmetric (+)
and antisymmetric (-) combinations of the pair:

  S^+- = S^id +- S^sw ,  F^+- = e_ext S^+- + F_act^+- ,
  T = -Y diag(1/(e_ext + omega - E0_L + E_s)) Y^T V,   Y = X Q,

with X = V_S s^(-1/2) over overlap eigenvalues >= threshold (Sec. II.B) and
(Q, omega) the eigenpairs of X^T F_act X.  The + sector includes the tuples with
coinciding pair indices (i = j or a = b).
"""
from __future__ import annotations

import itertools
import string
from functools import lru_cache

import numpy as np

from .wick import Builder, expect

# class -> (families, external slots, pair slots, active slots); a family lists the
# (slot, space) of E_{pq,rs} in the order p, q, r, s (Eq. class)
CLASS_DEF = {
    "A": ([(("r", "a"), ("i", "c"), ("s", "a"), ("t", "a"))], ["i"], None, ["r", "s", "t"]),
    "B": ([(("r", "a"), ("i", "c"), ("s", "a"), ("j", "c"))], ["i", "j"], ("i", "j"), ["r", "s"]),
    "C": ([(("a", "v"), ("r", "a"), ("s", "a"), ("t", "a"))], ["a"], None, ["r", "s", "t"]),
    "D": ([(("a", "v"), ("i", "c"), ("r", "a"), ("s", "a")),
           (("a", "v"), ("r", "a"), ("s", "a"), ("i", "c"))], ["a", "i"], None, ["r", "s"]),
    "E": ([(("a", "v"), ("i", "c"), ("r", "a"), ("j", "c"))], ["a", "i", "j"], ("i", "j"), ["r"]),
    "F": ([(("a", "v"), ("r", "a"), ("b", "v"), ("s", "a"))], ["a", "b"], ("a", "b"), ["r", "s"]),
    "G": ([(("a", "v"), ("r", "a"), ("b", "v"), ("i", "c"))], ["a", "b", "i"], ("a", "b"), ["r"]),
}


def _space_of_slot(cls):
    fams = CLASS_DEF[cls][0]
    sp = {}
    for fam in fams:
        for slot, s in fam:
            sp[slot] = s
    return sp


def _ket_ops(b, fam, tag):
    (p, _), (q, _), (r, _), (s, _) = fam
    return b.E2(p + tag, q + tag, r + tag, s + tag)


def _bra_ops(b, fam, tag):
    # (E_{pq,rs})^dagger = E_{qp,sr}
    (p, _), (q, _), (r, _), (s, _) = fam
    return b.E2(q + tag, p + tag, s + tag, r + tag)


@lru_cache(maxsize=None)
def overlap_terms(cls, fb, fk, with_fock):
    """Terms of <M|E_bra^dag (E_uw) E_ket|N> for families fb, fk of a class."""
    fams = CLASS_DEF[cls][0]
    sp = {}
    for slot, s in _space_of_slot(cls).items():
        sp[slot + "_b"] = s
        sp[slot + "_k"] = s
    b = Builder()
    ops = _bra_ops(b, fams[fb], "_b")
    if with_fock:
        sp["u"] = sp["w"] = "a"
        ops = ops + b.E("u", "w")
    ops = ops + _ket_ops(b, fams[fk], "_k")
    return tuple(expect(ops, sp))


@lru_cache(maxsize=None)
def source_terms(cls, fb):
    """Terms of <M|E_bra^dag H|L> with H = sum h_pq E_pq + 1/2 sum (pq|rt) E_pq,rt, the
    general indices split over closed / active / virtual."""
    fams = CLASS_DEF[cls][0]
    out = []
    base = {slot + "_b": s for slot, s in _space_of_slot(cls).items()}
    for sp1 in itertools.product("cav", repeat=2):
        b = Builder()
        sp = dict(base)
        sp.update({"p": sp1[0], "q": sp1[1]})
        for t in expect(_bra_ops(b, fams[fb], "_b") + b.E("p", "q"), sp):
            out.append(("h", sp1, 1.0, t))
    for sp2 in itertools.product("cav", repeat=4):
        b = Builder()
        sp = dict(base)
        sp.update({"p": sp2[0], "q": sp2[1], "r": sp2[2], "t": sp2[3]})
        for t in expect(_bra_ops(b, fams[fb], "_b") + b.E2("p", "q", "r", "t"), sp):
            out.append(("g", sp2, 0.5, t))
    return tuple(out)


class _Letters:
    def __init__(self):
        self.m = {}
        self.pool = iter(string.ascii_letters.replace("M", "").replace("N", "").replace("P", ""))

    def __call__(self, label):
        if label not in self.m:
            self.m[label] = next(self.pool)
        return self.m[label]


def _ext_perm(cls, deltas):
    """'id' or 'sw' from the bra-ket deltas between external labels."""
    ext = CLASS_DEF[cls][1]
    pair = CLASS_DEF[cls][2]
    mp = {}
    for x, y in deltas:
        for u, w in ((x, y), (y, x)):
            if u.endswith("_b") and w.endswith("_k") and u[:-2] in ext and w[:-2] in ext:
                mp[u[:-2]] = w[:-2]
    if all(mp.get(e) == e for e in ext):
        return "id"
    if pair is not None:
        i, j = pair
        if mp.get(i) == j and mp.get(j) == i and all(mp.get(e) == e for e in ext if e not in pair):
            return "sw"
    raise AssertionError(f"unexpected external pattern {deltas} for class {cls}")


def active_matrices(cls, rdm, n, a, f_act=None):
    """S_act^pi (and F_act^pi if f_act is given) as arrays
    [fam_b, act_b..., M, fam_k, act_k..., N] for pi in ('id', 'sw')."""
    fams, ext, pair, act = CLASS_DEF[cls]
    nf = len(fams)
    shape = (nf,) + (a,) * len(act) + (n,) + (nf,) + (a,) * len(act) + (n,)
    out = {}
    for which in (("S", False),) + ((("F", True),) if f_act is not None else ()):
        name, fock = which
        mats = {"id": np.zeros(shape), "sw": np.zeros(shape)}
        for fb in range(nf):
            for fk in range(nf):
                for t in overlap_terms(cls, fb, fk, fock):
                    pi = _ext_perm(cls, t.deltas)
                    L = _Letters()
                    subs, opnds = [], []
                    k = len(t.rdm)
                    if k == 0:
                        subs.append("MN")
                        opnds.append(np.eye(n))
                    else:
                        subs.append("MN" + "".join(L(p) + L(q) for p, q in t.rdm))
                        opnds.append(rdm[k])
                    for x, y in t.deltas:
                        if x[:-2] in ext and (x.endswith("_b") or x.endswith("_k")):
                            continue
                        subs.append(L(x) + L(y))
                        opnds.append(np.eye(a))
                    if fock:
                        subs.append(L("u") + L("w"))
                        opnds.append(f_act)
                    outsub = ("".join(L(s + "_b") for s in act) + "M"
                              + "".join(L(s + "_k") for s in act) + "N")
                    val = np.einsum(",".join(subs) + "->" + outsub, *opnds, optimize=True)
                    idx = (fb,) + (slice(None),) * (len(act) + 1) + (fk,)
                    mats[pi][idx] += t.coeff * val
        out[name] = mats
    return out


def sources(cls, rdm, n, a, blocks, ext_range=None):
    """V[fam, ext..., act..., M, L] = <M~|E_Omega^dag H|L~> (Eq. ampeq source).
    ext_range = (external label, lo, hi): only the values lo..hi-1 of that external index
    (every operand axis carrying the label is restricted to them)."""
    fams, ext, pair, act = CLASS_DEF[cls]
    dims = blocks["dims"]
    sp = _space_of_slot(cls)
    ext_dims = [dims[sp[e]] for e in ext]
    if ext_range is not None:
        ext_dims[ext.index(ext_range[0])] = ext_range[2] - ext_range[1]
    shape = (len(fams),) + tuple(ext_dims) + (a,) * len(act) + (n, n)
    V = np.zeros(shape)
    for fb in range(len(fams)):
        for kind, spc, w, t in source_terms(cls, fb):
            L = _Letters()
            subs, opnds = [], []
            k = len(t.rdm)
            if k == 0:
                subs.append("MN")
                opnds.append(np.eye(n))
            else:
                subs.append("MN" + "".join(L(p) + L(q) for p, q in t.rdm))
                opnds.append(rdm[k])
            lab_space = {"p": spc[0], "q": spc[1]} if kind == "h" else \
                dict(zip("pqrt", spc))
            for s_ in sp:
                lab_space[s_ + "_b"] = sp[s_]
            if kind == "h":
                subs.append(L("p") + L("q"))
                opnds.append(blocks["h"][spc[0] + spc[1]])
            else:
                subs.append("P" + L("p") + L("q"))
                opnds.append(blocks["B"][spc[0] + spc[1]])
                subs.append("P" + L("r") + L("t"))
                opnds.append(blocks["B"][spc[2] + spc[3]])
            for x, y in t.deltas:
                subs.append(L(x) + L(y))
                opnds.append(np.eye(dims[lab_space[x]]))
            outsub = ("".join(L(e + "_b") for e in ext) + "".join(L(s + "_b") for s in act) + "MN")
            if ext_range is not None:
                ch, lo, hi = L(ext_range[0] + "_b"), ext_range[1], ext_range[2]
                opnds = [_restrict(op, sub, ch, lo, hi) for op, sub in zip(opnds, subs)]
            val = np.einsum(",".join(subs) + "->" + outsub, *opnds, optimize=True)
            V[fb] += w * t.coeff * val
    return V


def _restrict(op, sub, ch, lo, hi):
    """op with every axis labelled ch restricted to lo..hi-1."""
    if ch not in sub:
        return op
    idx = tuple(slice(lo, hi) if x == ch else slice(None) for x in sub)
    return op[idx]


def integral_blocks(prob, h):
    c, a, v = prob.nclosed, prob.nact, prob.nvirt
    sl = {"c": slice(0, c), "a": slice(c, c + a), "v": slice(c + a, c + a + v)}
    hb = {x + y: h[sl[x], sl[y]] for x in "cav" for y in "cav"}
    Bb = {x + y: prob.B[:, sl[x], sl[y]] for x in "cav" for y in "cav"}
    return {"h": hb, "B": Bb, "dims": {"c": c, "a": a, "v": v}}


def all_classes(prob, st, shift=0.0, scheme="msmr", thresh=1e-9):
    """{class: (e, norm)} for A-G from RDMs and H from the closed form (o2_rdm.class_h)."""
    from .o2_rdm import class_h
    out = {cls: class_energy(prob, st, cls, shift, scheme, thresh) for cls in "ABCDEFG"}
    out["H"] = class_h(prob, st, shift=shift, scheme=scheme)
    return out


def all_moments(prob, st, shift=0.0, scheme="msmr", thresh=1e-9, chunks=None, i_chunk=None):
    """{class: (M1, M2, M3)} for all eight classes.  chunks: {class: (label, size)} for
    classes whose sources are taken in groups (class_moments); i_chunk: closed orbitals
    per group of class H (o2_rdm.class_h_moments)."""
    from .o2_rdm import class_h_moments
    chunks = chunks or {}
    out = {cls: class_moments(prob, st, cls, shift, scheme, thresh, chunk=chunks.get(cls))
           for cls in "ABCDEFG"}
    out["H"] = class_h_moments(prob, st, shift=shift, scheme=scheme, i_chunk=i_chunk)
    return out


def class_energy(prob, st, cls, shift=0.0, scheme="msmr", thresh=1e-9, h=None, chunk=None):
    """(e, norm) of a class; see class_moments for the definitions."""
    M1, M2, M3 = class_moments(prob, st, cls, shift, scheme, thresh, h, chunk)
    n = prob.nstate
    e = -np.array([[M1[L, L, Lp] for Lp in range(n)] for L in range(n)])
    nr = np.array([M2[L, L] for L in range(n)])
    return e, nr


def lambda_pieces(M1, M2, M3, R, P, shift):
    """lambda of the Lagrangian (Eq. lambdaeq differentiated with respect to T) in each
    sector's orthonormal basis: lam_L = -[R_LP sum_N R_NP Vt_N - 2 E_s R_LP^2 amp_L] / D_L
    with amp_L = -Vt_L / D_L.  Returns NL[L] = <lam_L|S|T_L> and
    lv[L, L'] = <Psi_lam_L|H|L'~> of the class."""
    n = R.shape[0]
    r = R[:, P]
    NL = np.array([r[L] * np.sum(r * M2[L]) + 2.0 * shift * r[L] ** 2 * M3[L] for L in range(n)])
    lv = np.array([[-r[L] * np.sum(r * M1[L, :, Lp]) - 2.0 * shift * r[L] ** 2 * M2[L, Lp]
                    for Lp in range(n)] for L in range(n)])
    return NL, lv


def class_moments(prob, st, cls, shift=0.0, scheme="msmr", thresh=1e-9, h=None, chunk=None):
    """Moment sums over the external tuples and sector eigenvectors mu of a class:
      M1[L, N, L'] = sum Vt_N Vt_L' / D_L,  M2[L, N] = sum Vt_N Vt_L / D_L^2,
      M3[L] = sum Vt_L^2 / D_L^3,   D_L = e_ext + omega_mu - E0_L + E_s,
    with Vt = Y^T V the sources in the orthonormal eigenbasis of the sector.  Then
    <Psi1_L|H|L'~> = -M1[L, L, L'] and <Psi1_L|Psi1_L> = M2[L, L].  For block-diagonal f,
    from the rotated RDMs of `st` (an o2_rdm.Setup with kmax >= 4).

    chunk = (external label, size), for classes too large to hold all sources at once:
    the tuples are taken in groups of `size` values of that external index (one that is
    not part of the swapped pair), sources of one group at a time.  Tuples are solved
    independently in the sector basis, so the grouping only orders the sums."""
    from .o2_rdm import g_of
    c, a, v, n = prob.nclosed, prob.nact, prob.nvirt, prob.nstate
    fams, ext, pair, act = CLASS_DEF[cls]
    sp = _space_of_slot(cls)
    dims = {"c": c, "a": a, "v": v}
    if any(dims[sp[e]] == 0 for e in ext) or a == 0:
        return np.zeros((n, n, n)), np.zeros((n, n)), np.zeros(n)
    if h is None:
        nmo = prob.nmo
        d = np.zeros((nmo, nmo))
        d[np.arange(c), np.arange(c)] = 2.0
        g1 = prob.rdm[1].reshape(n, n, a, a)
        d[c:c + a, c:c + a] = sum(g1[m, m] for m in range(n)) / n
        h = prob.f - g_of(prob.B, d)
    f_act = prob.f[c:c + a, c:c + a]
    rdm = st.rdm
    mats = active_matrices(cls, rdm, n, a, f_act)
    blocks = integral_blocks(prob, h)
    eps = np.diag(prob.f)
    ec, ev = eps[:c], eps[c + a:]
    nf = len(fams)
    m = nf * a ** len(act) * n
    S = {k: x.reshape(m, m) for k, x in mats["S"].items()}
    F = {k: x.reshape(m, m) for k, x in mats["F"].items()}
    M1 = np.zeros((n, n, n))
    M2 = np.zeros((n, n))
    M3 = np.zeros(n)
    sectors = [("+", 1.0), ("-", -1.0)] if pair is not None else [("id", 0.0)]

    # orthonormalised sector bases (independent of the external tuples)
    bases = {}
    for name, sgn in sectors:
        if pair is None:
            Ssec, Fsec = S["id"], F["id"]
        else:
            Ssec, Fsec = S["id"] + sgn * S["sw"], F["id"] + sgn * F["sw"]
        Ssec = 0.5 * (Ssec + Ssec.T)
        Fsec = 0.5 * (Fsec + Fsec.T)
        for Lsel in (range(n) if scheme == "sssr" else [None]):
            keep_idx = np.arange(m) if Lsel is None else np.arange(Lsel, m, n)
            Ss = Ssec[np.ix_(keep_idx, keep_idx)]
            Fs = Fsec[np.ix_(keep_idx, keep_idx)]
            s_, q_ = np.linalg.eigh(Ss)
            keep = s_ >= thresh
            if not keep.any():
                continue
            X = q_[:, keep] / np.sqrt(s_[keep])
            om, Q = np.linalg.eigh(X.T @ Fs @ X)
            bases[(name, Lsel)] = (keep_idx, X @ Q, om)

    # external tuples, in groups of one external index when chunked
    full = [dims[sp[e]] for e in ext]
    if chunk is None:
        groups = [None]
    else:
        lab, size = chunk
        assert lab in ext and (pair is None or lab not in pair)
        dim = full[ext.index(lab)]
        groups = [(lab, lo, min(dim, lo + size)) for lo in range(0, dim, size)]
    for grp in groups:
        V = sources(cls, rdm, n, a, blocks, ext_range=grp)
        ext_shape = list(full)
        offs = [0] * len(ext)
        if grp is not None:
            k_ = ext.index(grp[0])
            ext_shape[k_] = grp[2] - grp[1]
            offs[k_] = grp[1]
        grids = np.meshgrid(*[np.arange(r) for r in ext_shape], indexing="ij")
        tup_all = np.stack([g.ravel() for g in grids], axis=1)            # [ntup, next]
        eext_all = np.zeros(len(tup_all))
        for k, e_ in enumerate(ext):
            idx = tup_all[:, k] + offs[k]
            eext_all += ev[idx] if sp[e_] == "v" else -ec[idx]
        Vflat = V.reshape((nf, int(np.prod(ext_shape)), a ** len(act), n, n))
        del V

        def flat(tups):
            return np.ravel_multi_index(tuple(tups.T), ext_shape)

        for name, sgn in sectors:
            if pair is None:
                sel = np.arange(len(tup_all))
                vmat = Vflat[:, sel]                                          # [nf, T, A, M, L]
            else:
                pi_, pj_ = ext.index(pair[0]), ext.index(pair[1])
                ti, tj = tup_all[:, pi_], tup_all[:, pj_]
                sel = np.nonzero((ti < tj) if name == "-" else (ti <= tj))[0]
                swp = tup_all[sel].copy()
                swp[:, [pi_, pj_]] = swp[:, [pj_, pi_]]
                v1 = Vflat[:, sel]
                v2 = Vflat[:, flat(swp)]
                diag = (ti[sel] == tj[sel])[None, :, None, None, None]
                vmat = np.where(diag, v1, (v1 + sgn * v2) / np.sqrt(2.0))
            ee_sel = eext_all[sel]
            # rows (fam, act, M), columns (tuple, L)
            Vm = np.moveaxis(vmat, 1, 3).reshape(m, len(sel), n)
            del vmat
            for Lsel in (range(n) if scheme == "sssr" else [None]):
                if (name, Lsel) not in bases or len(sel) == 0:
                    continue
                keep_idx, Y, om = bases[(name, Lsel)]
                Vt = np.einsum("ku,ktl->utl", Y, Vm[keep_idx])              # [mu, tuple, L']
                Ls = range(n) if Lsel is None else [Lsel]
                for L in Ls:
                    D = ee_sel[None, :] + om[:, None] - st.E0[L] + shift      # [mu, tuple]
                    M1[L] += np.einsum("utn,utl->nl", Vt / D[:, :, None], Vt)
                    M2[L] += np.einsum("utn,ut->n", Vt, Vt[:, :, L] / D ** 2)
                    M3[L] += np.sum(Vt[:, :, L] ** 2 / D ** 3)
    return M1, M2, M3


def class_amplitudes(prob, st, cls, shift, scheme, R, P, thresh=1e-9, h=None):
    """T_L and lambda_L (target state P) of class cls in the basis of all index tuples:
    arrays [L][fam, ext..., act..., M].  Each sector is solved as in class_moments; the
    sector amplitudes Y amp and Y lam are mapped back to the tuples (a pair (x, y), x < y,
    takes (T+ + T-)/sqrt2 and its swap (T+ - T-)/sqrt2; x = y takes T+)."""
    from .o2_rdm import g_of
    c, a, v, n = prob.nclosed, prob.nact, prob.nvirt, prob.nstate
    fams, ext, pair, act = CLASS_DEF[cls]
    sp = _space_of_slot(cls)
    dims = {"c": c, "a": a, "v": v}
    nf = len(fams)
    ext_shape = [dims[sp[e]] for e in ext]
    T = np.zeros((n, nf) + tuple(ext_shape) + (a,) * len(act) + (n,))
    Lam = np.zeros_like(T)
    if any(d_ == 0 for d_ in ext_shape) or a == 0:
        return T, Lam
    if h is None:
        nmo = prob.nmo
        d = np.zeros((nmo, nmo))
        d[np.arange(c), np.arange(c)] = 2.0
        g1 = prob.rdm[1].reshape(n, n, a, a)
        d[c:c + a, c:c + a] = sum(g1[m, m] for m in range(n)) / n
        h = prob.f - g_of(prob.B, d)
    mats = active_matrices(cls, st.rdm, n, a, prob.f[c:c + a, c:c + a])
    V = sources(cls, st.rdm, n, a, integral_blocks(prob, h))
    eps = np.diag(prob.f)
    ec, ev = eps[:c], eps[c + a:]
    m = nf * a ** len(act) * n
    S = {k: x_.reshape(m, m) for k, x_ in mats["S"].items()}
    F = {k: x_.reshape(m, m) for k, x_ in mats["F"].items()}
    ntot = int(np.prod(ext_shape))
    grids = np.meshgrid(*[np.arange(r_) for r_ in ext_shape], indexing="ij")
    tup_all = np.stack([g_.ravel() for g_ in grids], axis=1)
    eext_all = np.zeros(len(tup_all))
    for k, e_ in enumerate(ext):
        eext_all += ev[tup_all[:, k]] if sp[e_] == "v" else -ec[tup_all[:, k]]
    Vflat = V.reshape((nf, ntot, a ** len(act), n, n))
    Tf = np.zeros((n, nf, ntot, a ** len(act), n))
    Lf = np.zeros_like(Tf)
    r = R[:, P]
    sectors = [("+", 1.0), ("-", -1.0)] if pair is not None else [("id", 0.0)]
    for name, sgn in sectors:
        if pair is None:
            Ssec, Fsec = S["id"], F["id"]
            sel = np.arange(ntot)
            partner = sel
            vmat = Vflat[:, sel]
        else:
            Ssec, Fsec = S["id"] + sgn * S["sw"], F["id"] + sgn * F["sw"]
            pi_, pj_ = ext.index(pair[0]), ext.index(pair[1])
            ti, tj = tup_all[:, pi_], tup_all[:, pj_]
            sel = np.nonzero((ti < tj) if name == "-" else (ti <= tj))[0]
            swp = tup_all[sel].copy()
            swp[:, [pi_, pj_]] = swp[:, [pj_, pi_]]
            partner = np.ravel_multi_index(tuple(swp.T), ext_shape)
            v1, v2 = Vflat[:, sel], Vflat[:, partner]
            diag = (ti[sel] == tj[sel])[None, :, None, None, None]
            vmat = np.where(diag, v1, (v1 + sgn * v2) / np.sqrt(2.0))
        Ssec = 0.5 * (Ssec + Ssec.T)
        Fsec = 0.5 * (Fsec + Fsec.T)
        ee = eext_all[sel]
        Vm = np.moveaxis(vmat, 1, 3).reshape(m, len(sel), n)
        isdiag = np.zeros(len(sel), dtype=bool) if pair is None else (partner == sel)
        for Lsel in (range(n) if scheme == "sssr" else [None]):
            keep_idx = np.arange(m) if Lsel is None else np.arange(Lsel, m, n)
            Ss = Ssec[np.ix_(keep_idx, keep_idx)]
            Fs = Fsec[np.ix_(keep_idx, keep_idx)]
            s_, q_ = np.linalg.eigh(Ss)
            keep = s_ >= thresh
            if not keep.any() or len(sel) == 0:
                continue
            X = q_[:, keep] / np.sqrt(s_[keep])
            om, Q = np.linalg.eigh(X.T @ Fs @ X)
            Y = X @ Q
            Vt = np.einsum("ku,ktl->utl", Y, Vm[keep_idx])
            for L in (range(n) if Lsel is None else [Lsel]):
                D = ee[None, :] + om[:, None] - st.E0[L] + shift
                amp = -Vt[:, :, L] / D
                src = r[L] * np.einsum("n,utn->ut", r, Vt) - 2.0 * shift * r[L] ** 2 * amp
                lam = -src / D
                tsec, lsec = Y @ amp, Y @ lam          # [rows(keep_idx), sel]
                full_t = np.zeros((m, len(sel)))
                full_l = np.zeros((m, len(sel)))
                full_t[keep_idx], full_l[keep_idx] = tsec, lsec
                # rows (fam, act, M) -> [fam, act, M]
                ft = full_t.reshape(nf, a ** len(act), n, len(sel))
                fl = full_l.reshape(nf, a ** len(act), n, len(sel))
                if pair is None:
                    Tf[L][:, sel] += np.moveaxis(ft, 3, 1)
                    Lf[L][:, sel] += np.moveaxis(fl, 3, 1)
                else:
                    w1 = np.where(isdiag, 1.0, 1.0 / np.sqrt(2.0))
                    w2 = np.where(isdiag, 0.0, sgn / np.sqrt(2.0))
                    for arr, src_ in ((Tf, ft), (Lf, fl)):
                        arr[L][:, sel] += np.moveaxis(src_ * w1, 3, 1)
                        np.add.at(arr[L], (slice(None), partner),
                                  np.moveaxis(src_ * w2, 3, 1))
    T = Tf.reshape((n, nf) + tuple(ext_shape) + (a,) * len(act) + (n,))
    Lam = Lf.reshape(T.shape)
    return T, Lam


def class_densities(prob, st, cls, shift, scheme, R, P, thresh=1e-9):
    """Class cls's share of the correlated densities of target state P (Sec. II.D):
      d1[x, y]     = sum W <M~|E_Omega^dag E_xy|L'~>,  W = R_L'P sum_L R_LP T_L + lambda_L'
      GDF[Q, x, y] = d/dB_Qxy of sum W <M~|E_Omega^dag H_2|L'~>  (= sum_zw D1_xy,zw B_Qzw)
      d2[x, y]     = d L_PT2 / d f_xy on the closed-closed, active-active and virtual-virtual
                     blocks (the closed-vacuum normal-ordered f^), with the E0 term
      NL[L]        = <lambda_L|S|T_L>."""
    from .o2_rdm import g_of
    c, a, v, n, nmo = prob.nclosed, prob.nact, prob.nvirt, prob.nstate, prob.nmo
    fams, ext, pair, act = CLASS_DEF[cls]
    sp = _space_of_slot(cls)
    d1 = np.zeros((nmo, nmo))
    GDF = np.zeros_like(prob.B)
    d2 = np.zeros((nmo, nmo))
    NL = np.zeros(n)
    dims = {"c": c, "a": a, "v": v}
    if any(dims[sp[e]] == 0 for e in ext) or a == 0:
        return d1, GDF, d2, NL
    d = np.zeros((nmo, nmo))
    d[np.arange(c), np.arange(c)] = 2.0
    g1 = prob.rdm[1].reshape(n, n, a, a)
    d[c:c + a, c:c + a] = sum(g1[m_, m_] for m_ in range(n)) / n
    h = prob.f - g_of(prob.B, d)
    T, Lam = class_amplitudes(prob, st, cls, shift, scheme, R, P, thresh, h)
    r = R[:, P]
    nf = len(fams)
    # W[fam, ext..., act..., M, L'] (the source contraction pairs M with the bra and L' with the ket)
    W = (np.einsum("l,k,l...->...k", r, r, T) + np.moveaxis(Lam, 0, -1))
    off = {"c": 0, "a": c, "v": c + a}
    rng = {s_: slice(off[s_], off[s_] + dims[s_]) for s_ in "cav"}
    blocks = integral_blocks(prob, h)
    for fb in range(nf):
        for kind, spc, w, t in source_terms(cls, fb):
            L_ = _Letters()
            subs, opnds = [], []
            subs.append("".join(L_(e_ + "_b") for e_ in ext) + "".join(L_(s_ + "_b") for s_ in act) + "MN")
            opnds.append(W[fb])
            k = len(t.rdm)
            if k == 0:
                subs.append("MN")
                opnds.append(np.eye(n))
            else:
                subs.append("MN" + "".join(L_(p_) + L_(q_) for p_, q_ in t.rdm))
                opnds.append(st.rdm[k])
            lab_space = {"p": spc[0], "q": spc[1]} if kind == "h" else dict(zip("pqrt", spc))
            for s_ in sp:
                lab_space[s_ + "_b"] = sp[s_]
            for x_, y_ in t.deltas:
                subs.append(L_(x_) + L_(y_))
                opnds.append(np.eye(dims[lab_space[x_]]))
            if kind == "h":
                out = L_("p") + L_("q")
                val = np.einsum(",".join(subs) + "->" + out, *opnds, optimize=True)
                d1[rng[spc[0]], rng[spc[1]]] += w * t.coeff * val
            else:
                out = L_("p") + L_("q") + L_("r") + L_("t")
                G = w * t.coeff * np.einsum(",".join(subs) + "->" + out, *opnds, optimize=True)
                B1 = prob.B[:, rng[spc[0]], rng[spc[1]]]
                B2 = prob.B[:, rng[spc[2]], rng[spc[3]]]
                GDF[:, rng[spc[0]], rng[spc[1]]] += np.einsum("pqrt,Qrt->Qpq", G, B2)
                GDF[:, rng[spc[2]], rng[spc[3]]] += np.einsum("pqrt,Qpq->Qrt", G, B1)
    # overlap-metric contractions
    mats = active_matrices(cls, st.rdm, n, a, None)["S"]
    m = nf * a ** len(act) * n
    next_ = len(ext)
    ax_ext = list(range(2, 2 + next_))                 # ext axes of T[L] arrays (after L, fam)

    def apply_S(Spi, arr):   # arr [L][fam, ext..., act..., M] -> S applied over (fam, act, M)
        Sm = Spi.reshape(m, m)
        ext_axes = list(range(2, 2 + next_))
        x_ = np.moveaxis(arr, ext_axes, list(range(1, 1 + next_)))   # [L, ext..., fam, act..., M]
        shp = x_.shape
        y_ = (x_.reshape(shp[:1 + next_] + (m,)) @ Sm.T).reshape(shp)
        return np.moveaxis(y_, list(range(1, 1 + next_)), ext_axes)

    def swap_pair(arr):
        if pair is None:
            return arr
        i_, j_ = ext.index(pair[0]), ext.index(pair[1])
        return np.swapaxes(arr, 2 + i_, 2 + j_)

    U = {"id": apply_S(mats["id"], T), "sw": apply_S(mats["sw"], T)}
    ax = tuple(range(1, T.ndim))
    NL = np.sum(Lam * U["id"], axis=ax)
    if pair is not None:
        NL = NL + np.sum(Lam * swap_pair(U["sw"]), axis=ax)
    # external blocks: one slot of the ket tuple moves (hole for closed, particle for virtual)
    letters = "abcdefghijk"
    for si, s_ in enumerate(ext):
        blk = sp[s_]
        for pi_name, Lm in (("id", Lam), ("sw", swap_pair(Lam) if pair is not None else None)):
            if Lm is None:
                continue
            rank = Lm.ndim
            sl = list(letters[:rank])
            su = list(sl)
            sl[2 + si] = "x"
            su[2 + si] = "y"
            X = np.einsum("".join(sl) + "," + "".join(su) + "->xy", Lm, U[pi_name])
            if blk == "c":
                d2[rng["c"], rng["c"]] -= X.T        # d2[i][j] = -sum lam(s=j) S T(s=i)
            else:
                d2[rng["v"], rng["v"]] += X          # d2[a][b] = +sum lam(s=a) S T(s=b)
    # active block: lambda x T contracted with the Fock-type terms (E_uw between IC functions)
    Dm = {}
    for pi_name in ("id", "sw"):
        Tp = T if pi_name == "id" else swap_pair(T)
        if pi_name == "sw" and pair is None:
            continue
        nb = 2 + next_
        sl = "L" + "f" + "".join("e" + str(k) for k in range(next_))
        # einsum over L and ext: rows (fam_b, act_b, M), cols (fam_k, act_k, N)
        A_ = Lam.reshape((n, nf, -1, a ** len(act) * n))
        B_ = Tp.reshape((n, nf, -1, a ** len(act) * n))
        Dm[pi_name] = np.einsum("lfer,lgec->frgc", A_, B_).reshape(
            (nf,) + (a,) * len(act) + (n,) + (nf,) + (a,) * len(act) + (n,))
    for fb in range(nf):
        for fk in range(nf):
            for t in overlap_terms(cls, fb, fk, True):
                pi = _ext_perm(cls, t.deltas)
                if pi not in Dm:
                    continue
                L_ = _Letters()
                subs, opnds = [], []
                subs.append("".join(L_(s_ + "_b") for s_ in act) + "M" + "".join(L_(s_ + "_k") for s_ in act) + "N")
                opnds.append(Dm[pi][(fb,) + (slice(None),) * (len(act) + 1) + (fk,)])
                k = len(t.rdm)
                if k == 0:
                    subs.append("MN")
                    opnds.append(np.eye(n))
                else:
                    subs.append("MN" + "".join(L_(p_) + L_(q_) for p_, q_ in t.rdm))
                    opnds.append(st.rdm[k])
                for x_, y_ in t.deltas:
                    if x_[:-2] in ext and (x_.endswith("_b") or x_.endswith("_k")):
                        continue
                    subs.append(L_(x_) + L_(y_))
                    opnds.append(np.eye(a))
                val = np.einsum(",".join(subs) + "->" + L_("u") + L_("w"), *opnds, optimize=True)
                d2[rng["a"], rng["a"]] += t.coeff * val
    g1r = st.rdm[1]
    for L in range(n):
        d2[rng["a"], rng["a"]] -= NL[L] * g1r[L, L]
    return d1, GDF, d2, NL


def class_residual(prob, st, cls, shift, scheme, T, thresh=1e-9, h=None):
    """Relative residual of given first-order amplitudes in the amplitude equation of
    class cls (Eq. ampeq with block-diagonal f), in the class's own metric:
        r = X^T [ (F + (e_ext - E0_L + E_s) S) t + V ]   per sector, tuple and state L,
    t the sector amplitudes of T (layout of class_amplitudes: [L][fam, ext..., act..., M];
    a pair (x, y) enters the + and - sectors as (T(x,y) +- T(y,x))/sqrt2, x = y the +
    sector as T(x,x)), X the orthonormalised basis of the kept overlap eigenvalues.
    Returns ||r|| / ||X^T V|| over all sectors, tuples and states: about the unit
    roundoff for an exact solve, whatever the conditioning of the denominators, because a
    rounding error of a sector eigenvalue moves t along directions where the equation is
    nearly singular and leaves r small."""
    from .o2_rdm import g_of
    c, a, v, n = prob.nclosed, prob.nact, prob.nvirt, prob.nstate
    fams, ext, pair, act = CLASS_DEF[cls]
    sp = _space_of_slot(cls)
    dims = {"c": c, "a": a, "v": v}
    nf = len(fams)
    ext_shape = [dims[sp[e]] for e in ext]
    if any(d_ == 0 for d_ in ext_shape) or a == 0:
        return 0.0
    if h is None:
        nmo = prob.nmo
        d = np.zeros((nmo, nmo))
        d[np.arange(c), np.arange(c)] = 2.0
        g1 = prob.rdm[1].reshape(n, n, a, a)
        d[c:c + a, c:c + a] = sum(g1[m, m] for m in range(n)) / n
        h = prob.f - g_of(prob.B, d)
    mats = active_matrices(cls, st.rdm, n, a, prob.f[c:c + a, c:c + a])
    V = sources(cls, st.rdm, n, a, integral_blocks(prob, h))
    eps = np.diag(prob.f)
    ec, ev = eps[:c], eps[c + a:]
    m = nf * a ** len(act) * n
    S = {k: x_.reshape(m, m) for k, x_ in mats["S"].items()}
    F = {k: x_.reshape(m, m) for k, x_ in mats["F"].items()}
    ntot = int(np.prod(ext_shape))
    grids = np.meshgrid(*[np.arange(r_) for r_ in ext_shape], indexing="ij")
    tup_all = np.stack([g_.ravel() for g_ in grids], axis=1)
    eext_all = np.zeros(len(tup_all))
    for k, e_ in enumerate(ext):
        eext_all += ev[tup_all[:, k]] if sp[e_] == "v" else -ec[tup_all[:, k]]
    Vflat = V.reshape((nf, ntot, a ** len(act), n, n))
    Tflat = np.asarray(T).reshape((n, nf, ntot, a ** len(act), n))
    num = den = 0.0
    sectors = [("+", 1.0), ("-", -1.0)] if pair is not None else [("id", 0.0)]
    for name, sgn in sectors:
        if pair is None:
            Ssec, Fsec = S["id"], F["id"]
            sel = np.arange(ntot)
            vmat = Vflat[:, sel]
            tmat = Tflat[:, :, sel]
        else:
            Ssec, Fsec = S["id"] + sgn * S["sw"], F["id"] + sgn * F["sw"]
            pi_, pj_ = ext.index(pair[0]), ext.index(pair[1])
            ti, tj = tup_all[:, pi_], tup_all[:, pj_]
            sel = np.nonzero((ti < tj) if name == "-" else (ti <= tj))[0]
            swp = tup_all[sel].copy()
            swp[:, [pi_, pj_]] = swp[:, [pj_, pi_]]
            partner = np.ravel_multi_index(tuple(swp.T), ext_shape)
            diag = (ti[sel] == tj[sel])
            v1, v2 = Vflat[:, sel], Vflat[:, partner]
            vmat = np.where(diag[None, :, None, None, None], v1, (v1 + sgn * v2) / np.sqrt(2.0))
            t1, t2 = Tflat[:, :, sel], Tflat[:, :, partner]
            tmat = np.where(diag[None, None, :, None, None], t1, (t1 + sgn * t2) / np.sqrt(2.0))
        if len(sel) == 0:
            continue
        Ssec = 0.5 * (Ssec + Ssec.T)
        Fsec = 0.5 * (Fsec + Fsec.T)
        ee = eext_all[sel]
        Vm = np.moveaxis(vmat, 1, 3).reshape(m, len(sel), n)               # rows (fam, act, M)
        Tm = np.moveaxis(tmat, 2, 4).reshape(n, m, len(sel))               # [L][rows, tuple]
        for Lsel in (range(n) if scheme == "sssr" else [None]):
            keep_idx = np.arange(m) if Lsel is None else np.arange(Lsel, m, n)
            Ss = Ssec[np.ix_(keep_idx, keep_idx)]
            Fs = Fsec[np.ix_(keep_idx, keep_idx)]
            s_, q_ = np.linalg.eigh(Ss)
            keep = s_ >= thresh
            if not keep.any():
                continue
            X = q_[:, keep] / np.sqrt(s_[keep])
            for L in (range(n) if Lsel is None else [Lsel]):
                t = Tm[L][keep_idx]
                r = Fs @ t + (Ss @ t) * (ee - st.E0[L] + shift)[None, :] + Vm[keep_idx, :, L]
                num += float(np.sum((X.T @ r) ** 2))
                den += float(np.sum((X.T @ Vm[keep_idx, :, L]) ** 2))
    return float(np.sqrt(num / den)) if den > 0 else 0.0
