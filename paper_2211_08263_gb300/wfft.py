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
                "xmid", "col_fwd", "col_inv", "col_grad", "col_div", "col_prec", "newmark", "scalar", "net_conv",
                "net_aux", "xinv_pupd"]
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
                ("watchdog_iters", C.c_int), ("use_graphs", C.c_int), ("inner_floor", C.c_double),
                ("incr_resid", C.c_int)]


class PlanChoice(C.Structure):
    _fields_ = [("radix", (C.c_int * 7) * 3), ("bx", (C.c_int * 5) * 3), ("xelems", C.c_int)]


class StepInfo(C.Structure):
    _fields_ = [("status", C.c_int), ("iters", C.c_int), ("outer_applies", C.c_int), ("sweeps", C.c_int),
                ("ref", C.c_double), ("rel_res", C.c_double), ("reaction", C.c_double * 3), ("ms", C.c_double),
                ("incr_resids", C.c_int), ("energy", C.c_double)]

    def as_dict(self):
        return {"status": self.status, "iters": self.iters, "outer_applies": self.outer_applies,
                "sweeps": self.sweeps, "ref": self.ref, "rel_res": self.rel_res,
                "reaction": list(self.reaction), "ms": self.ms, "incr_resids": self.incr_resids,
                "energy": self.energy}


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
    lib.wfft_autotune.argtypes = [vp, i, P(i)]
    lib.wfft_set_radix.argtypes = [vp, i, i, P(i)]
    lib.wfft_get_plan.argtypes = [vp, i, P(PlanChoice)]
    lib.wfft_set_plan.argtypes = [vp, i, P(PlanChoice)]
    lib.wfft_green_setup.argtypes = [vp, C.c_longlong]
    lib.wfft_green_step.argtypes = [vp, P(d), P(StepInfo)]
    lib.wfft_explicit_step.argtypes = [vp, P(d), P(StepInfo)]
    lib.wfft_explicit_dt.argtypes = [i, P(d), vp, vp, C.c_longlong, P(d)]
    lib.wfft_download_async.argtypes = [vp, vp, vp, vp]
    lib.wfft_download_wait.argtypes = [vp]
    lib.wfft_operator_bound.argtypes = [i, P(i), P(d), vp, vp, C.c_longlong, d, P(d)]
    lib.wfft_axis_plan.argtypes = [i, P(i), P(i)]
    lib.wfft_precond_noalloc.argtypes = [P(Grid), P(d), d, d, vp, vp, vp]
    lib.wfft_net_conv_kernel.argtypes = [i]
    lib.wfft_model_bytes.argtypes = [i]
    lib.wfft_model_bytes.restype = C.c_size_t
    lib.wfft_model_init.argtypes = [i, C.c_ulonglong, vp, C.c_size_t]
    lib.wfft_set_model.argtypes = [vp, vp, C.c_size_t]
    lib.wfft_trainer_create.argtypes = [vp, C.c_size_t, vp, P(vp)]
    lib.wfft_trainer_collect.argtypes = [vp, vp, P(d), i, P(StepInfo)]
    lib.wfft_trainer_samples.argtypes = [vp]
    lib.wfft_trainer_samples.restype = C.c_longlong
    lib.wfft_trainer_fit.argtypes = [vp, i, i, d, C.c_ulonglong, P(d)]
    lib.wfft_trainer_get_model.argtypes = [vp, vp, C.c_size_t]
    lib.wfft_trainer_error.argtypes = [vp]
    lib.wfft_trainer_error.restype = C.c_char_p
    lib.wfft_trainer_destroy.argtypes = [vp]
    lib.wfft_trainer_destroy.restype = None
    lib.wfft_net_forward.argtypes = [vp, C.c_size_t, P(i), vp, vp]
    lib.wfft_net_loss_grad.argtypes = [vp, C.c_size_t, P(i), i, vp, vp, vp, vp, P(d)]
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

    def download_async(self, u: Optional[np.ndarray] = None, v: Optional[np.ndarray] = None,
                       a: Optional[np.ndarray] = None) -> None:
        """Start copying the state into host arrays ([c][N3][N2][N1] float64, contiguous;
        pinned memory overlaps with the next step).  The arrays must stay alive and unread
        until download_wait() (wfft_download_async)."""
        ptrs = []
        for x in (u, v, a):
            if x is None:
                ptrs.append(None)
                continue
            if x.dtype != np.float64 or not x.flags["C_CONTIGUOUS"] or x.size != self.shape[0] * self.V:
                raise ValueError("download buffers must be contiguous float64 arrays of the state's size")
            ptrs.append(_ptr(x))
        self._check(self.lib.wfft_download_async(self.h, *ptrs))

    def download_wait(self) -> None:
        """Block until the latest download_async has landed (wfft_download_wait)."""
        self._check(self.lib.wfft_download_wait(self.h))

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

    def explicit_step(self, Udot, raise_on_error: bool = True) -> dict:
        """One explicit central-difference step (handle created with beta = 0, gamma = 1/2)
        with the velocity Udot(t_n) prescribed on Gamma."""
        Uv = (C.c_double * 3)(*[float(x) for x in list(Udot)[:3]] + [0.0] * (3 - min(3, len(Udot))))
        info = StepInfo()
        rc = self.lib.wfft_explicit_step(self.h, Uv, C.byref(info))
        if raise_on_error:
            self._check(rc)
        d = info.as_dict()
        d["rc"] = rc
        return d

    def green_setup(self, max_dofs: int = 0) -> None:
        """Build and invert the Green's matrix of the prescribed region (wfft_green_setup)."""
        self._check(self.lib.wfft_green_setup(self.h, int(max_dofs)))

    def green_step(self, U) -> dict:
        """One Newmark step through the Green's matrix (wfft_green_step)."""
        Uv = (C.c_double * 3)(*[float(x) for x in list(U)[:3]] + [0.0] * (3 - min(3, len(U))))
        info = StepInfo()
        self._check(self.lib.wfft_green_step(self.h, Uv, C.byref(info)))
        return info.as_dict()

    def get_plan(self, precision: int) -> dict:
        """{"radix": 3 x 7 stage counts, "bx": 3 x 5 column-tile widths, "xelems": x-pass tile
        size} (wfft_get_plan)."""
        pc = PlanChoice()
        self._check(self.lib.wfft_get_plan(self.h, int(precision), C.byref(pc)))
        return {"radix": [list(r) for r in pc.radix], "bx": [list(r) for r in pc.bx], "xelems": pc.xelems}

    def set_plan(self, precision: int, plan: dict) -> None:
        """Apply plan choices read by get_plan (wfft_set_plan)."""
        pc = PlanChoice()
        for a in range(3):
            for r in range(7):
                pc.radix[a][r] = int(plan["radix"][a][r])
            for o in range(5):
                pc.bx[a][o] = int(plan["bx"][a][o])
        pc.xelems = int(plan.get("xelems", 0))
        self._check(self.lib.wfft_set_plan(self.h, int(precision), C.byref(pc)))

    def set_radix(self, precision: int, axis: int, counts) -> None:
        """Stages of radix 8, 4, 2, 3, 5, 7, 16 (counts, 7 entries) for one axis (wfft_set_radix)."""
        c = (C.c_int * 7)(*[int(x) for x in counts])
        self._check(self.lib.wfft_set_radix(self.h, int(precision), int(axis), c))

    def autotune(self, reps: int = 3) -> int:
        """Time and keep the fastest radix decompositions and column-tile widths
        (wfft_autotune); returns how many choices changed."""
        ch = C.c_int()
        self._check(self.lib.wfft_autotune(self.h, int(reps), C.byref(ch)))
        return ch.value

    # ---- learned warm start
    def set_model(self, blob: Optional[np.ndarray]):
        """Load a model blob (uint8 array) for warm_start = WARM_LEARNED; None unloads."""
        if blob is None:
            self._check(self.lib.wfft_set_model(self.h, None, 0))
        else:
            b = np.ascontiguousarray(blob, dtype=np.uint8)
            self._check(self.lib.wfft_set_model(self.h, _ptr(b), b.nbytes))

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


def _check_dev_f64(name: str, t, count: int):
    """Refuse anything but a contiguous CUDA float64 tensor of `count` elements: the library
    cannot see the size of a device buffer it is handed."""
    ok = (hasattr(t, "is_cuda") and t.is_cuda and str(t.dtype) == "torch.float64" and t.is_contiguous()
          and t.numel() == count)
    if not ok:
        raise WfftError(EINVAL, f"{name} must be a contiguous CUDA float64 tensor of {count} elements")


def precond_noalloc(ndim: int, n, h, cbar21, rho_bar: float, theta: float, r, z, stream: int = 0):
    """z = M r (FP64, unmasked) through the allocation-free entry point; r, z are contiguous
    CUDA float64 tensors of ndim * N1 * N2 * N3 elements (checked here before the call)."""
    count = int(ndim) * int(n[0]) * int(n[1]) * int(n[2])
    _check_dev_f64("r", r, count)
    _check_dev_f64("z", z, count)
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


# ---------------------------------------------------------------------------
# learned warm start: model blobs, GPU trainer, single-call network evaluation
# ---------------------------------------------------------------------------
NET_IN, NET_OUT, NET_OUT_PAD, NET_LAYERS = 16, 3, 16, 4
_HEADER_INTS = 8


def _raise_global(rc: int):
    if rc != OK:
        raise WfftError(rc, load().wfft_last_error(None).decode())


def net_conv_kernel(kind: int) -> int:
    """Network forward convolutions: 0 = tcgen05 where the grid allows, 1 = mma.sync
    (wfft_net_conv_kernel); returns the previous setting."""
    return load().wfft_net_conv_kernel(int(kind))


def model_bytes(hidden: int) -> int:
    return int(load().wfft_model_bytes(int(hidden)))


def model_init(hidden: int = 32, seed: int = 0) -> np.ndarray:
    """Seeded initial model blob (uint8); its last layer is zero (Taylor warm start)."""
    nb = model_bytes(hidden)
    if nb == 0:
        raise WfftError(EINVAL, "hidden width must be 16 or 32")
    b = np.zeros(nb, dtype=np.uint8)
    _raise_global(load().wfft_model_init(int(hidden), int(seed), _ptr(b), nb))
    return b


def layer_shapes(hidden: int):
    """(cout, cin) of the four layers as stored."""
    return [(hidden, NET_IN), (hidden, hidden), (hidden, hidden), (NET_OUT_PAD, hidden)]


def blob_params(blob: np.ndarray):
    """Model blob -> (hidden, [(W[27, cout, cin], b[cout]) per layer]) as float32 copies."""
    b = np.ascontiguousarray(blob, dtype=np.uint8)
    hd = b[:4 * _HEADER_INTS].view(np.int32)
    hidden = int(hd[4])
    th = b[4 * _HEADER_INTS:].view(np.float32)
    out, off = [], 0
    for co, ci in layer_shapes(hidden):
        nw = 27 * co * ci
        W = th[off:off + nw].reshape(27, co, ci).copy()
        off += nw
        out.append((W, th[off:off + co].copy()))
        off += co
    return hidden, out


def params_blob(hidden: int, params) -> np.ndarray:
    """Inverse of blob_params."""
    hd = np.array([0x314E4657, 1, NET_LAYERS, NET_IN, hidden, NET_OUT, NET_OUT_PAD, 0], dtype=np.int32)
    parts = [hd.view(np.uint8)]
    for (W, bias), (co, ci) in zip(params, layer_shapes(hidden)):
        parts.append(np.ascontiguousarray(W, dtype=np.float32).reshape(27 * co * ci).view(np.uint8))
        parts.append(np.ascontiguousarray(bias, dtype=np.float32).reshape(co).view(np.uint8))
    return np.concatenate(parts)


def grad_params(hidden: int, grad: np.ndarray):
    """Flat FP32 gradient (parameter layout) -> [(dW, db)] per layer."""
    out, off = [], 0
    for co, ci in layer_shapes(hidden):
        nw = 27 * co * ci
        dW = grad[off:off + nw].reshape(27, co, ci)
        off += nw
        out.append((dW, grad[off:off + co]))
        off += co
    return out


def net_forward(blob: np.ndarray, n, x: np.ndarray) -> np.ndarray:
    """Network output y [V, 3] for host features x [V, 16] on the periodic grid n = (N1, N2, N3)."""
    b = np.ascontiguousarray(blob, dtype=np.uint8)
    nn = (C.c_int * 3)(*[int(v) for v in n])
    V = int(n[0]) * int(n[1]) * int(n[2])
    xf = np.ascontiguousarray(x, dtype=np.float32).reshape(V, NET_IN)
    y = np.empty((V, NET_OUT), dtype=np.float32)
    _raise_global(load().wfft_net_forward(_ptr(b), b.nbytes, nn, _ptr(xf), _ptr(y)))
    return y


def net_loss_grad(blob: np.ndarray, n, c: int, x: np.ndarray, target: np.ndarray, mask: Optional[np.ndarray] = None):
    """(loss, flat FP32 gradient) of one training pair."""
    b = np.ascontiguousarray(blob, dtype=np.uint8)
    hidden = int(b[:32].view(np.int32)[4])
    nn = (C.c_int * 3)(*[int(v) for v in n])
    V = int(n[0]) * int(n[1]) * int(n[2])
    xf = np.ascontiguousarray(x, dtype=np.float32).reshape(V, NET_IN)
    tf = np.ascontiguousarray(target, dtype=np.float32).reshape(V, NET_OUT)
    mk = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8).reshape(V)
    nparam = (model_bytes(hidden) - 4 * _HEADER_INTS) // 4
    g = np.empty(nparam, dtype=np.float32)
    loss = C.c_double()
    _raise_global(load().wfft_net_loss_grad(_ptr(b), b.nbytes, nn, int(c), _ptr(xf), _ptr(tf),
                                            None if mk is None else _ptr(mk), _ptr(g), C.byref(loss)))
    return loss.value, g


class Trainer:
    """GPU trainer of the warm-start network (wfft_trainer_*)."""

    def __init__(self, blob: np.ndarray, stream: int = 0):
        self.lib = load()
        b = np.ascontiguousarray(blob, dtype=np.uint8)
        self.nbytes = b.nbytes
        t = C.c_void_p()
        _raise_global(self.lib.wfft_trainer_create(_ptr(b), b.nbytes, C.c_void_p(stream or None), C.byref(t)))
        self.t = t

    def _check(self, rc):
        if rc != OK:
            raise WfftError(rc, self.lib.wfft_trainer_error(self.t).decode())

    def collect(self, solver: Solver, U: np.ndarray):
        """Step `solver` through U (nsteps x 3), keeping one training pair per step; returns the step infos."""
        Ua = np.ascontiguousarray(np.asarray(U, dtype=np.float64).reshape(-1, 3))
        infos = (StepInfo * max(1, Ua.shape[0]))()
        self._check(self.lib.wfft_trainer_collect(self.t, solver.h, Ua.ctypes.data_as(C.POINTER(C.c_double)),
                                                  Ua.shape[0], infos))
        return [infos[i].as_dict() for i in range(Ua.shape[0])]

    @property
    def samples(self) -> int:
        return int(self.lib.wfft_trainer_samples(self.t))

    def fit(self, epochs: int, batch: int = 4, lr: float = 1e-3, seed: int = 0) -> float:
        loss = C.c_double()
        self._check(self.lib.wfft_trainer_fit(self.t, int(epochs), int(batch), float(lr), int(seed), C.byref(loss)))
        return loss.value

    def model(self) -> np.ndarray:
        b = np.zeros(self.nbytes, dtype=np.uint8)
        self._check(self.lib.wfft_trainer_get_model(self.t, _ptr(b), b.nbytes))
        return b

    def close(self):
        if getattr(self, "t", None):
            self.lib.wfft_trainer_destroy(self.t)
            self.t = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def operator_bound(ndim: int, n, h, C_table: np.ndarray, rho: np.ndarray, theta: float) -> float:
    """Upper bound of the largest eigenvalue of A = rho + theta B^T C B (wfft_operator_bound)."""
    Ct = np.ascontiguousarray(C_table, dtype=np.float64).reshape(-1, 21)
    r = np.ascontiguousarray(rho, dtype=np.float64).reshape(-1)
    nn = (C.c_int * 3)(*[int(x) for x in list(n)[:3]] + [1] * (3 - min(3, len(n))))
    hh = (C.c_double * 3)(*[float(x) for x in list(h)[:3]] + [1.0] * (3 - min(3, len(h))))
    out = C.c_double()
    _raise_global(load().wfft_operator_bound(int(ndim), nn, hh, _ptr(Ct), _ptr(r), Ct.shape[0], float(theta),
                                             C.byref(out)))
    return out.value


def axis_plan(n: int):
    """Built-in FFT decomposition of an axis of n points (wfft_axis_plan): (stage counts of
    radix 8, 4, 2, 3, 5, 7, 16, prime factor above 7 taken by the direct stage or 0)."""
    cnt = (C.c_int * 7)()
    prime = C.c_int()
    _raise_global(load().wfft_axis_plan(int(n), cnt, C.byref(prime)))
    return list(cnt), prime.value


def explicit_dt(ndim: int, h, C_table: np.ndarray, rho: np.ndarray) -> float:
    """Largest stable increment of the explicit scheme over the material rows (wfft_explicit_dt)."""
    Ct = np.ascontiguousarray(C_table, dtype=np.float64).reshape(-1, 21)
    r = np.ascontiguousarray(rho, dtype=np.float64).reshape(-1)
    hh = (C.c_double * 3)(*[float(x) for x in list(h)[:3]] + [1.0] * (3 - min(3, len(h))))
    out = C.c_double()
    _raise_global(load().wfft_explicit_dt(int(ndim), hh, _ptr(Ct), _ptr(r), Ct.shape[0], C.byref(out)))
    return out.value
