"""Python binding of libcaspt2.so (argument marshalling only).

Every computation runs in the CUDA library; this module converts arrays to
pointers, calls the C ABI declared in include/caspt2.h and raises on error.
There is no CPU fallback: if the library is missing, importing the binding
functions raises.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(HERE, "libcaspt2.so")

OK, EINVAL, ENOMEM, ENOTCONV, ENAN, ETIMEOUT, ECUDA, ESTATE, ESCRATCH = 0, -1, -2, -3, -4, -5, -6, -7, -8
WINTRUDER, WDEGEN = 1, 2
WARN_INTRUDER, WARN_DEGEN = 1, 2
MEM_HOST, MEM_DEVICE = 0, 1
MSMR, SSSR = 0, 1
FP64, BF16X = 0, 1
CLASSES = "ABCDEFGH"


class Dims(C.Structure):
    _fields_ = [("nclosed", C.c_int), ("nact", C.c_int), ("nvirt", C.c_int),
                ("naux", C.c_int), ("nstate", C.c_int)]


class Options(C.Structure):
    _fields_ = [("xms", C.c_int), ("scheme", C.c_int), ("shift", C.c_double),
                ("ovl_thresh", C.c_double), ("enuc", C.c_double), ("target_state", C.c_int),
                ("class_mask", C.c_uint), ("precision", C.c_int), ("slices", C.c_int),
                ("degen_thresh", C.c_double), ("closed_begin", C.c_int),
                ("closed_end", C.c_int), ("dens_offdiag", C.c_int)]


class Request(C.Structure):
    _fields_ = [("dims", Dims), ("opt", Options),
                ("fock", C.c_void_p), ("dfB", C.c_void_p), ("rdm1", C.c_void_p),
                ("rdm2", C.c_void_p), ("rdm3", C.c_void_p), ("rdm4", C.c_void_p),
                ("densities", C.c_int)]


class ServeResult(C.Structure):
    _fields_ = [("status", C.c_int), ("latency_ms", C.c_double), ("queue_ms", C.c_double),
                ("Ems", C.c_void_p), ("R", C.c_void_p), ("Heff", C.c_void_p),
                ("d1", C.c_void_p), ("d2", C.c_void_p), ("gdf", C.c_void_p)]


_lib = None


def lib():
    """Load libcaspt2.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIBPATH):
            raise RuntimeError(f"{LIBPATH} is missing: build it with "
                               "`python -m paper_1606_01273_gb300.build`")
        L = C.CDLL(LIBPATH)
        P = C.c_void_p
        dp = C.POINTER(C.c_double)
        L.caspt2_default_options.argtypes = [C.POINTER(Options)]
        L.caspt2_default_options.restype = None
        L.caspt2_create.argtypes = [C.POINTER(P), C.POINTER(Dims), C.POINTER(Options)]
        L.caspt2_set_inputs.argtypes = [P, C.c_int, P, P, P, P, P, P]
        L.caspt2_solve.argtypes = [P, P]
        L.caspt2_get_energies.argtypes = [P, dp, dp, dp, dp, dp, dp]
        L.caspt2_get_class_energy.argtypes = [P, C.c_int, dp, dp]
        L.caspt2_get_core_energy.argtypes = [P, dp]
        L.caspt2_get_class_lambda.argtypes = [P, C.c_int, dp, dp]
        L.caspt2_get_timings.argtypes = [P, dp, C.POINTER(C.c_int)]
        L.caspt2_get_kernel_launches.argtypes = [P]
        L.caspt2_get_kernel_launches.restype = C.c_long
        L.caspt2_supported_classes.argtypes = []
        L.caspt2_supported_classes.restype = C.c_uint
        L.caspt2_destroy.argtypes = [P]
        L.caspt2_destroy.restype = None
        L.caspt2_densities.argtypes = [P, C.c_uint, P]
        L.caspt2_get_densities.argtypes = [P, C.c_int, P, P, P, P]
        L.caspt2_gradient.argtypes = [P, C.c_int, P, P, P]
        L.caspt2_orbital_derivative.argtypes = [P, C.c_int, P, P]
        L.caspt2_get_status.argtypes = [P, C.POINTER(Report)]
        L.caspt2_amplitude_size.argtypes = [P, C.c_int]
        L.caspt2_amplitude_size.restype = C.c_long
        L.caspt2_get_amplitudes.argtypes = [P, C.c_int, C.c_int, C.c_int, C.c_int, P, P]
        L.caspt2_get_lambda.argtypes = [P, C.c_int, C.c_int, C.c_int, C.c_int, P, P]
        L.caspt2_server_create.argtypes = [C.POINTER(P), C.c_size_t, C.c_int]
        L.caspt2_server_submit.argtypes = [P, C.POINTER(Request), C.POINTER(C.c_long)]
        L.caspt2_server_wait.argtypes = [P, C.c_long, C.c_int, C.POINTER(ServeResult)]
        L.caspt2_server_destroy.argtypes = [P]
        L.caspt2_server_destroy.restype = None
        L.caspt2_classH_noalloc.argtypes = [C.POINTER(Dims), C.POINTER(Options), P, P, P, P, P, P]
        L.caspt2_get_moments.argtypes = [P, P]
        L.caspt2_finalize_moments.argtypes = [P, P, P]
        L.caspt2_strerror.argtypes = [C.c_int]
        L.caspt2_strerror.restype = C.c_char_p
        _lib = L
    return _lib


class Report(C.Structure):
    """caspt2_report (caspt2_get_status)."""
    _fields_ = [("last_status", C.c_int), ("solved", C.c_int), ("densities_done", C.c_int),
                ("min_denominator", C.c_double), ("kernel_launches", C.c_long),
                ("times_ms", C.c_double * 10), ("warnings", C.c_uint),
                ("min_e0_gap", C.c_double)]


class CASPT2Error(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {lib().caspt2_strerror(status).decode()} ({status})")
        self.status = status


def _check(st: int, where: str, warn_ok: bool = False) -> int:
    if st < 0 or (st > 0 and not warn_ok):
        raise CASPT2Error(st, where)
    return st


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ptr(x):
    """Host numpy array (C-contiguous float64) or torch CUDA tensor -> (void*, mem kind)."""
    if x is None:
        return None, None
    if isinstance(x, np.ndarray):
        assert x.dtype == np.float64 and x.flags.c_contiguous
        return C.c_void_p(x.ctypes.data), MEM_HOST
    # torch tensor on the device
    assert x.dtype.is_floating_point and x.element_size() == 8 and x.is_contiguous()
    return C.c_void_p(x.data_ptr()), (MEM_DEVICE if x.is_cuda else MEM_HOST)


def default_options(**kw) -> Options:
    o = Options()
    lib().caspt2_default_options(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def supported_classes() -> str:
    m = lib().caspt2_supported_classes()
    return "".join(c for k, c in enumerate(CLASSES) if m >> k & 1)


@dataclass
class Result:
    U: np.ndarray
    E0: np.ndarray
    Href: np.ndarray
    Heff: np.ndarray
    Ems: np.ndarray
    R: np.ndarray
    Ecore: float
    e_class: dict
    norm_class: dict
    status: int
    timings_ms: list
    launches: int
    lam_NL: dict = None
    lam_lv: dict = None
    d1: np.ndarray = None
    d2: np.ndarray = None
    gdf: np.ndarray = None


class Context:
    """One library context (device buffers sized for `dims`)."""

    def __init__(self, nclosed, nact, nvirt, naux, nstate, **opts):
        self.dims = Dims(nclosed, nact, nvirt, naux, nstate)
        self.opts = default_options(**opts)
        h = C.c_void_p()
        _check(lib().caspt2_create(C.byref(h), C.byref(self.dims), C.byref(self.opts)),
               "caspt2_create")
        self._h = h
        self.n = nstate

    def close(self):
        if getattr(self, "_h", None):
            lib().caspt2_destroy(self._h)
            self._h = None

    __del__ = close

    def set_inputs(self, fock, dfB, rdm1, rdm2, rdm3=None, rdm4=None):
        ptrs = [_ptr(x) for x in (fock, dfB, rdm1, rdm2, rdm3, rdm4)]
        mems = {m for p, m in ptrs if m is not None}
        if len(mems) != 1:
            raise ValueError("all inputs must live in the same memory (host or device)")
        self._keep = (fock, dfB, rdm1, rdm2, rdm3, rdm4)
        _check(lib().caspt2_set_inputs(self._h, mems.pop(), *[p for p, _ in ptrs]),
               "caspt2_set_inputs")

    def solve(self, stream=None) -> int:
        s = C.c_void_p(stream) if stream is not None else None
        return _check(lib().caspt2_solve(self._h, s), "caspt2_solve", warn_ok=True)

    def result(self, status: int = 0) -> Result:
        n = self.n
        U, Href, Heff, R = (np.zeros((n, n)) for _ in range(4))
        E0, Ems = np.zeros(n), np.zeros(n)
        _check(lib().caspt2_get_energies(self._h, _dp(U), _dp(E0), _dp(Href), _dp(Heff),
                                         _dp(Ems), _dp(R)), "caspt2_get_energies")
        ec = C.c_double()
        _check(lib().caspt2_get_core_energy(self._h, C.byref(ec)), "caspt2_get_core_energy")
        e_cls, n_cls = {}, {}
        for k, name in enumerate(CLASSES):
            if self.opts.class_mask >> k & 1:
                e, nr = np.zeros((n, n)), np.zeros(n)
                _check(lib().caspt2_get_class_energy(self._h, k, _dp(e), _dp(nr)),
                       "caspt2_get_class_energy")
                e_cls[name], n_cls[name] = e, nr
        lam_NL, lam_lv = {}, {}
        if self.opts.target_state >= 0:
            for k, name in enumerate(CLASSES):
                if self.opts.class_mask >> k & 1:
                    a_, b_ = np.zeros(n), np.zeros((n, n))
                    _check(lib().caspt2_get_class_lambda(self._h, k, _dp(a_), _dp(b_)),
                           "caspt2_get_class_lambda")
                    lam_NL[name], lam_lv[name] = a_, b_
        t = np.zeros(32)
        cnt = C.c_int(32)
        _check(lib().caspt2_get_timings(self._h, _dp(t), C.byref(cnt)), "caspt2_get_timings")
        return Result(U, E0, Href, Heff, Ems, R, ec.value, e_cls, n_cls, status,
                      list(t[: cnt.value]), int(lib().caspt2_get_kernel_launches(self._h)),
                      lam_NL, lam_lv)


    def compute_densities(self, class_mask=None, stream=None):
        """caspt2_densities for the classes in class_mask (default: all solved classes);
        the results stay on the device until get_densities."""
        mask = self.opts.class_mask if class_mask is None else class_mask
        s = C.c_void_p(stream) if stream is not None else None
        _check(lib().caspt2_densities(self._h, mask, s), "caspt2_densities")

    def get_densities(self, with_gdf: bool = True, with_nl: bool = False):
        """Host copies (d1, d2, gdf) of the last densities (gdf None if not requested);
        with_nl: (d1, d2, gdf, NL), NL[L] summed over the classes."""
        nmo = self.dims.nclosed + self.dims.nact + self.dims.nvirt
        d1, d2 = np.zeros((nmo, nmo)), np.zeros((nmo, nmo))
        nl = np.zeros(self.n)
        gdf = np.zeros((self.dims.naux, nmo, nmo)) if with_gdf else None
        gp = C.c_void_p(gdf.ctypes.data) if with_gdf else None
        _check(lib().caspt2_get_densities(self._h, MEM_HOST, C.c_void_p(d1.ctypes.data),
                                          C.c_void_p(d2.ctypes.data),
                                          C.c_void_p(nl.ctypes.data), gp),
               "caspt2_get_densities")
        return (d1, d2, gdf, nl) if with_nl else (d1, d2, gdf)

    def gradient(self, stream=None):
        """caspt2_gradient: host copies (dE/df [nmo][nmo], dE/dB [naux][nmo][nmo]) of the
        target state's MS energy (MS only, reference RDMs fixed)."""
        nmo = self.dims.nclosed + self.dims.nact + self.dims.nvirt
        gf = np.zeros((nmo, nmo))
        gB = np.zeros((self.dims.naux, nmo, nmo))
        s = C.c_void_p(stream) if stream is not None else None
        _check(lib().caspt2_gradient(self._h, MEM_HOST, C.c_void_p(gf.ctypes.data),
                                     C.c_void_p(gB.ctypes.data), s), "caspt2_gradient")
        return gf, gB

    def orbital_derivative(self, stream=None):
        """caspt2_orbital_derivative: host copy of Y [nmo][nmo] = dL/dkappa (the orbital
        part of the Z-vector source) of the target state; needs dens_offdiag=1."""
        nmo = self.dims.nclosed + self.dims.nact + self.dims.nvirt
        Y = np.zeros((nmo, nmo))
        s = C.c_void_p(stream) if stream is not None else None
        _check(lib().caspt2_orbital_derivative(self._h, MEM_HOST, C.c_void_p(Y.ctypes.data), s),
               "caspt2_orbital_derivative")
        return Y

    def densities(self, class_mask=None, stream=None):
        """compute_densities + get_densities: host copies (d1, d2, gdf), each symmetrised."""
        self.compute_densities(class_mask, stream)
        return self.get_densities()

    def status(self) -> dict:
        """caspt2_get_status: last solve status, flags, smallest |denominator|, launches,
        timings."""
        r = Report()
        _check(lib().caspt2_get_status(self._h, C.byref(r)), "caspt2_get_status")
        return {"last_status": r.last_status, "solved": bool(r.solved),
                "densities_done": bool(r.densities_done), "min_denominator": r.min_denominator,
                "kernel_launches": r.kernel_launches, "times_ms": list(r.times_ms),
                "warnings": int(r.warnings), "min_e0_gap": r.min_e0_gap}

    def moments(self) -> np.ndarray:
        """caspt2_get_moments: per-class moment sums [8][n^3 + n^2 + n] of the last solve."""
        n = self.n
        out = np.zeros((8, n ** 3 + n ** 2 + n))
        _check(lib().caspt2_get_moments(self._h, C.c_void_p(out.ctypes.data)),
               "caspt2_get_moments")
        return out

    def finalize_moments(self, mom: np.ndarray, stream=None) -> int:
        """caspt2_finalize_moments: H^eff, E_MS, R and lambda from (summed) moments."""
        m = np.ascontiguousarray(mom, dtype=np.float64)
        s = C.c_void_p(stream) if stream is not None else None
        return _check(lib().caspt2_finalize_moments(self._h, C.c_void_p(m.ctypes.data), s),
                      "caspt2_finalize_moments", warn_ok=True)

    def amplitude_size(self, cls: int) -> int:
        """caspt2_amplitude_size: elements of T_LN (or lambda_LN) of class index cls."""
        n = int(lib().caspt2_amplitude_size(self._h, cls))
        if n < 0:
            raise CASPT2Error(n, "caspt2_amplitude_size")
        return n

    def _class_vector(self, fn, name, cls, L, N, stream):
        out = np.zeros(self.amplitude_size(cls))
        s = C.c_void_p(stream) if stream is not None else None
        _check(fn(self._h, cls, L, N, MEM_HOST, C.c_void_p(out.ctypes.data), s), name)
        return out

    def amplitudes(self, cls: int, L: int, N: int, stream=None) -> np.ndarray:
        """T_LN of class cls (0-6 = A-G), flat [family][external...][active...]."""
        return self._class_vector(lib().caspt2_get_amplitudes, "caspt2_get_amplitudes", cls, L,
                                  N, stream)

    def lambdas(self, cls: int, L: int, N: int, stream=None) -> np.ndarray:
        """lambda_LN of the target state, class cls (0-6 = A-G), same layout as amplitudes."""
        return self._class_vector(lib().caspt2_get_lambda, "caspt2_get_lambda", cls, L, N,
                                  stream)


def classH_noalloc(dims: Dims, opts: Options, fock, dfB, rdm1, e, norm, stream=None) -> int:
    """caspt2_classH_noalloc on device tensors (no device allocation inside the call).

    For callers that cannot allocate device memory: every intermediate lives in the
    library's fixed 4 MiB device scratch array.  Returns the status (warnings > 0);
    raises on errors."""
    ptr = lambda t: None if t is None else C.c_void_p(t.data_ptr())
    s = C.c_void_p(stream) if stream is not None else None
    st = lib().caspt2_classH_noalloc(C.byref(dims), C.byref(opts), ptr(fock), ptr(dfB),
                                     ptr(rdm1), ptr(e), ptr(norm), s)
    return _check(st, "caspt2_classH_noalloc", warn_ok=True)


def problem_inputs(prob, kmax: int = 4):
    """Host arrays (f, B, rdm1, rdm2, rdm3, rdm4) of a synth.Problem in the layout of
    caspt2_set_inputs; RDMs above kmax (or absent) are None."""
    n = prob.nstate
    r = [np.ascontiguousarray(prob.rdm[k].reshape(n, n, -1)) if (k <= kmax and k in prob.rdm)
         else None for k in (1, 2, 3, 4)]
    return (np.ascontiguousarray(prob.f), np.ascontiguousarray(prob.B), *r)


def solve_problem(prob, densities=None, **opts) -> Result:
    """Create a context, copy a synth.Problem from host memory, solve, fetch results.
    densities: a class mask (or True for all solved classes) to also compute the
    densities of opts' target_state."""
    ctx = Context(prob.nclosed, prob.nact, prob.nvirt, prob.naux, prob.nstate, **opts)
    try:
        ctx.set_inputs(*problem_inputs(prob))
        st = ctx.solve()
        r = ctx.result(st)
        if densities is not None and densities is not False:
            mask = None if densities is True else int(densities)
            r.d1, r.d2, r.gdf = ctx.densities(mask)
            r.timings_ms = ctx.result(st).timings_ms
        return r
    finally:
        ctx.close()


class Server:
    """caspt2_server_*: concurrent requests admitted by device-memory budget."""

    def __init__(self, budget_bytes: int = 0, slots: int = 4):
        h = C.c_void_p()
        _check(lib().caspt2_server_create(C.byref(h), budget_bytes, slots), "caspt2_server_create")
        self._h = h

    def submit(self, prob, densities: bool = False, **opts) -> int:
        """Queue a synth.Problem (inputs copied by the library); returns the ticket."""
        f, B, r1, r2, r3, r4 = problem_inputs(prob)
        req = Request()
        req.dims = Dims(prob.nclosed, prob.nact, prob.nvirt, prob.naux, prob.nstate)
        req.opt = default_options(**opts)
        ptr = lambda x: None if x is None else C.c_void_p(x.ctypes.data)
        req.fock, req.dfB, req.rdm1, req.rdm2, req.rdm3, req.rdm4 = (ptr(x) for x in (f, B, r1, r2, r3, r4))
        req.densities = 1 if densities else 0
        t = C.c_long()
        _check(lib().caspt2_server_submit(self._h, C.byref(req), C.byref(t)), "caspt2_server_submit")
        self._shapes = getattr(self, "_shapes", {})
        self._shapes[t.value] = (prob.nstate, prob.nmo, prob.naux, densities)
        return t.value

    def wait(self, ticket: int, timeout_ms: int = -1) -> dict:
        n, nmo, X, dens = self._shapes.pop(ticket)
        out = {"Ems": np.zeros(n), "R": np.zeros((n, n)), "Heff": np.zeros((n, n))}
        if dens:
            out.update(d1=np.zeros((nmo, nmo)), d2=np.zeros((nmo, nmo)), gdf=np.zeros((X, nmo, nmo)))
        res = ServeResult()
        for k, v in out.items():
            setattr(res, k, C.c_void_p(v.ctypes.data))
        st = lib().caspt2_server_wait(self._h, ticket, timeout_ms, C.byref(res))
        _check(st, "caspt2_server_wait", warn_ok=True)
        out.update(status=st, latency_ms=res.latency_ms, queue_ms=res.queue_ms)
        return out

    def close(self):
        if getattr(self, "_h", None):
            lib().caspt2_server_destroy(self._h)
            self._h = None

    __del__ = close


def ms_energy(f, B, rdms, nclosed, target_state=0, **opts):
    """E_MS of `target_state` as a differentiable function of the Fock matrix f and the DF
    factors B (CUDA float64 tensors; the RDMs (rdm1..rdm4, device tensors in the layouts of
    caspt2_set_inputs, higher ranks may be None) are held fixed).  The forward pass is a
    caspt2_solve; the backward pass is caspt2_gradient (densities chained through the
    solve's definitions), so torch.autograd gives dE/df and dE/dB.  MS only (xms = 0)."""
    import torch

    nmo = f.shape[0]
    X = B.shape[0]
    n = rdms[0].shape[0]
    a = int(round(np.sqrt(rdms[0][0, 0].numel()))) if rdms[0].numel() else 0
    dims = (nclosed, a, nmo - nclosed - a, X, n)
    kw = dict(opts, xms=0, target_state=target_state)

    class _E(torch.autograd.Function):
        @staticmethod
        def forward(fctx, f_, B_):
            ctx = Context(*dims, **kw)
            ctx.set_inputs(f_.contiguous(), B_.contiguous(), *[r.contiguous() if r is not None
                                                                 else None for r in rdms])
            st = ctx.solve()
            r = ctx.result(st)
            fctx.lib_ctx = ctx
            return torch.tensor(r.Ems[target_state], dtype=f_.dtype, device=f_.device)

        @staticmethod
        def backward(fctx, g):
            ctx = fctx.lib_ctx
            gf = torch.empty((nmo, nmo), dtype=torch.float64, device=g.device)
            gB = torch.empty((X, nmo, nmo), dtype=torch.float64, device=g.device)
            torch.cuda.synchronize(g.device)
            _check(lib().caspt2_gradient(ctx._h, MEM_DEVICE, C.c_void_p(gf.data_ptr()),
                                         C.c_void_p(gB.data_ptr()), None), "caspt2_gradient")
            ctx.close()
            return g * gf, g * gB

    return _E.apply(f, B)
