"""Thin Python binding of the wfft C ABI (include/wfft.h).

Argument marshalling only: every step of the solver runs in the CUDA library
libwfft.so built in-tree by ``paper_2211_08263_gb300.build``.  There is no
CPU fallback -- importing the library raises if it has not been built or if
the CUDA runtime cannot be loaded.
"""
from __future__ import annotations

import ctypes as C
import os
import re
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libwfft.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "wfft.h")

OK, EINVAL, ENOMEM, ECUDA, ENOTCONV, ENUMERIC, ETIMEOUT, EUNSUPPORTED = range(8)
KERNEL_KINDS = ["xfwd_plain", "xfwd_pupd", "xfwd_rupd", "xfwd_conv", "xinv_apply", "xinv_resid", "xinv_prec",
                "xmid", "col_fwd", "col_inv", "col_grad", "col_div", "col_prec", "newmark", "scalar"]
FP64, MIXED = 0, 1
WARM_PREV, WARM_TAYLOR, WARM_LEARNED = 0, 1, 2
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ENOTCONV", 5: "ENUMERIC", 6: "ETIMEOUT",
                7: "EUNSUPPORTED"}


class WfftError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"wfft error {STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class Grid(C.Structure):
    _fields_ = [("ndim", C.c_int), ("n", C.c_int * 3), ("h", C.c_double * 3)]


class Options(C.Structure):
    _fields_ = [("precision", C.c_int), ("tol", C.c_double), ("maxit", C.c_int), ("warm_start", C.c_int),
                ("inner_tol", C.c_double), ("max_sweeps", C.c_int), ("check_every", C.c_int),
                ("watchdog_iters", C.c_int)]


class StepInfo(C.Structure):
    _fields_ = [("status", C.c_int), ("iters", C.c_int), ("outer_applies", C.c_int), ("sweeps", C.c_int),
                ("ref", C.c_double), ("rel_res", C.c_double), ("reaction", C.c_double * 3), ("ms", C.c_double)]

    def as_dict(self):
        return {"status": self.status, "iters": self.iters, "outer_applies": self.outer_applies,
                "sweeps": self.sweeps, "ref": self.ref, "rel_res": self.rel_res,
                "reaction": list(self.reaction), "ms": self.ms}


_lib = None


def declared_symbols(header: str = HEADER):
    """Names of the functions declared in include/wfft.h."""
    txt = open(header).read()
    return sorted(set(re.findall(r"^WFFT_API\s+[\w\s\*]+?\b(wfft_\w+)\s*\(", txt, flags=re.M)))


def load(path: str = LIB_PATH):
    """Load libwfft.so (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"the wfft CUDA library is not built ({path}); run "
                          f"`python -m paper_2211_08263_gb300.build` (or __graft_entry__.build())")
    lib = C.CDLL(path)
    vp, i, d = C.c_void_p, C.c_int, C.c_double
    P = C.POINTER
    lib.wfft_default_options.argtypes = [P(Options)]
    lib.wfft_create.argtypes = [P(Grid), vp, vp, i, vp, vp, d, d, d, P(Options), vp, P(vp)]
    lib.wfft_destroy.argtypes = [vp]
    lib.wfft_destroy.restype = None
    lib.wfft_last_error.argtypes = [vp]
    lib.wfft_last_error.restype = C.c_char_p
    lib.wfft_set_state.argtypes = [vp, vp, vp, vp, C.c_longlong]
    lib.wfft_get_state.argtypes = [vp, vp, vp, vp, P(C.c_longlong)]
    lib.wfft_set_state_dev.argtypes = [vp, vp, vp, vp, C.c_longlong]
    lib.wfft_get_state_dev.argtypes = [vp, vp, vp, vp]
    lib.wfft_step.argtypes = [vp, P(d), P(StepInfo)]
    lib.wfft_solve.argtypes = [vp, vp, vp, d, i, P(StepInfo)]
    lib.wfft_apply.argtypes = [vp, i, vp, vp, i]
    lib.wfft_precond.argtypes = [vp, i, vp, vp, i]
    lib.wfft_rfft3.argtypes = [vp, i, i, i, vp, vp]
    lib.wfft_spectral_pitch.argtypes = [vp, P(i)]
    lib.wfft_batch_step.argtypes = [P(vp), i, P(d), P(StepInfo)]
    lib.wfft_get_sizes.argtypes = [vp, P(i), P(i), P(C.c_longlong)]
    lib.wfft_device_bytes.argtypes = [vp, P(C.c_size_t)]
    lib.wfft_profile.argtypes = [vp, i]
    lib.wfft_profile_read.argtypes = [vp, i, i, P(C.c_longlong), P(C.c_longlong), P(d), P(d), P(d)]
    lib.wfft_launch_count.argtypes = [vp, P(C.c_longlong)]
    lib.wfft_precond_noalloc.argtypes = [P(Grid), P(d), d, d, vp, vp, vp]
    _lib = lib
    return lib


def default_options(**kw) -> Options:
    o = Options()
    load().wfft_default_options(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _dptr(t) -> C.c_void_p:
    """Device pointer of a torch CUDA tensor (or an int address)."""
    return C.c_void_p(t if isinstance(t, int) else t.data_ptr())


class Solver:
    """One wfft handle.  Host arrays use the [c][N3][N2][N1] layout."""

    def __init__(self, ndim: int, n, h, C_table: np.ndarray, rho: np.ndarray, phase: Optional[np.ndarray],
                 mask: Optional[np.ndarray], dt: float, beta: float = 0.25, gamma: float = 0.5,
                 options: Optional[Options] = None, stream: int = 0):
        lib = load()
        self.lib = lib
        self.ndim = ndim
        self.n = tuple(int(v) for v in n)
        self.V = self.n[0] * self.n[1] * self.n[2]
        self.shape = (ndim, self.n[2], self.n[1], self.n[0])
        g = Grid(ndim, (C.c_int * 3)(*self.n), (C.c_double * 3)(*[float(v) for v in h]))
        self._C = np.ascontiguousarray(C_table, dtype=np.float64)
        self._rho = np.ascontiguousarray(rho, dtype=np.float64)
        self._phase = None if phase is None else np.ascontiguousarray(phase, dtype=np.uint16)
        self._mask = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
        nphase = 0 if phase is None else int(self._C.shape[0])
        self.options = options if options is not None else default_options()
        hnd = C.c_void_p()
        rc = lib.wfft_create(C.byref(g), _ptr(self._C), None if self._phase is None else _ptr(self._phase), nphase,
                             _ptr(self._rho), None if self._mask is None else _ptr(self._mask), float(dt),
                             float(beta), float(gamma), C.byref(self.options), C.c_void_p(stream), C.byref(hnd))
        if rc != OK:
            raise WfftError(rc, lib.wfft_last_error(None).decode())
        self.h = hnd

    @classmethod
    def from_problem(cls, prob, options: Optional[Options] = None, stream: int = 0, **kw) -> "Solver":
        if options is None:
            options = default_options(tol=prob.tol, **kw)
        return cls(prob.ndim, prob.n, prob.h, prob.C, prob.rho, prob.phase, prob.mask, prob.dt, prob.beta,
                   prob.gamma, options, stream)

    def _check(self, rc):
        if rc != OK:
            raise WfftError(rc, self.lib.wfft_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.wfft_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- state
    def set_state(self, u=None, v=None, a=None, n: int = 0):
        arrs = [None if x is None else np.ascontiguousarray(x, dtype=np.float64).reshape(self.shape)
                for x in (u, v, a)]
        self._check(self.lib.wfft_set_state(self.h, *[None if x is None else _ptr(x) for x in arrs], n))

    def get_state(self):
        u, v, a = (np.empty(self.shape) for _ in range(3))
        n = C.c_longlong()
        self._check(self.lib.wfft_get_state(self.h, _ptr(u), _ptr(v), _ptr(a), C.byref(n)))
        return u, v, a, n.value

    def download_u(self, out: np.ndarray) -> int:
        """Copy u_n into `out` (host, [c][N3][N2][N1] float64, may be pinned); returns n."""
        n = C.c_longlong()
        self._check(self.lib.wfft_get_state(self.h, _ptr(out), None, None, C.byref(n)))
        return n.value

    def set_state_dev(self, u, v, a, n: int = 0):
        self._check(self.lib.wfft_set_state_dev(self.h, _dptr(u), _dptr(v), _dptr(a), n))

    def get_state_dev(self, u, v, a):
        self._check(self.lib.wfft_get_state_dev(self.h, _dptr(u), _dptr(v), _dptr(a)))

    # ---- stepping
    def step(self, U, raise_on_error: bool = True) -> dict:
        Uv = (C.c_double * 3)(*[float(x) for x in list(U)[:3]] + [0.0] * (3 - min(3, len(U))))
        info = StepInfo()
        rc = self.lib.wfft_step(self.h, Uv, C.byref(info))
        if raise_on_error:
            self._check(rc)
        d = info.as_dict()
        d["rc"] = rc
        return d

    def solve(self, b: np.ndarray, x: np.ndarray, tol: float = 0.0, maxit: int = 0) -> dict:
        b = np.ascontiguousarray(b, dtype=np.float64).reshape(self.shape)
        xo = np.ascontiguousarray(x, dtype=np.float64).reshape(self.shape).copy()
        info = StepInfo()
        rc = self.lib.wfft_solve(self.h, _ptr(b), _ptr(xo), float(tol), int(maxit), C.byref(info))
        self._check(rc)
        d = info.as_dict()
        d["x"] = xo
        return d

    # ---- raw operators on device arrays (torch tensors)
    def apply(self, p, q, precision: int = FP64, masked: bool = False):
        self._check(self.lib.wfft_apply(self.h, precision, _dptr(p), _dptr(q), int(masked)))

    def precond(self, r, z, precision: int = FP64, masked: bool = False):
        self._check(self.lib.wfft_precond(self.h, precision, _dptr(r), _dptr(z), int(masked)))

    def rfft3(self, inp, out, precision: int = FP64, direction: int = -1, ncomp: int = 1):
        self._check(self.lib.wfft_rfft3(self.h, precision, direction, ncomp, _dptr(inp), _dptr(out)))

    # ---- launch accounting
    def profile(self, enable: bool):
        self._check(self.lib.wfft_profile(self.h, int(enable)))

    def profile_read(self):
        """{(precision, kind): {launches, timed, ms, bytes, flops}} for kinds with launches."""
        out = {}
        for prec in (FP64, MIXED):
            for k, name in enumerate(KERNEL_KINDS):
                n, t = C.c_longlong(), C.c_longlong()
                ms, by, fl = C.c_double(), C.c_double(), C.c_double()
                self._check(self.lib.wfft_profile_read(self.h, prec, k, C.byref(n), C.byref(t), C.byref(ms),
                                                       C.byref(by), C.byref(fl)))
                if n.value:
                    out[("fp64" if prec == FP64 else "fp32", name)] = {
                        "launches": n.value, "timed": t.value, "ms": ms.value, "bytes": by.value, "flops": fl.value}
        return out

    def launch_count(self) -> int:
        n = C.c_longlong()
        self._check(self.lib.wfft_launch_count(self.h, C.byref(n)))
        return n.value

    def spectral_pitch(self) -> int:
        p = C.c_int()
        self._check(self.lib.wfft_spectral_pitch(self.h, C.byref(p)))
        return p.value


def precond_noalloc(ndim: int, n, h, cbar21, rho_bar: float, theta: float, r, z, stream: int = 0):
    """z = M r (FP64, unmasked) through the allocation-free entry point; r, z are device arrays."""
    lib = load()
    g = Grid(ndim, (C.c_int * 3)(*[int(v) for v in n]), (C.c_double * 3)(*[float(v) for v in h]))
    cb = (C.c_double * 21)(*[float(v) for v in cbar21])
    rc = lib.wfft_precond_noalloc(C.byref(g), cb, float(rho_bar), float(theta), _dptr(r), _dptr(z),
                                  C.c_void_p(stream))
    if rc != OK:
        raise WfftError(rc, lib.wfft_last_error(None).decode())


def batch_step(solvers, U: np.ndarray):
    """Advance every solver by one step (U: n x 3)."""
    lib = load()
    n = len(solvers)
    hs = (C.c_void_p * n)(*[s.h for s in solvers])
    Ua = np.ascontiguousarray(U, dtype=np.float64).reshape(n, 3)
    infos = (StepInfo * n)()
    rc = lib.wfft_batch_step(hs, n, Ua.ctypes.data_as(C.POINTER(C.c_double)), infos)
    return rc, [infos[i].as_dict() for i in range(n)]
