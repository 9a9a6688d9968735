"""Oracle work run in spawned CPU processes by the full-size GPU tests.

One FP64 oracle Newmark step at 256^3 takes minutes on the host cores, most of it in
single-threaded NumPy; independent steps (from different saved states) therefore run in
parallel processes, each with a share of the cores for scipy.fft.  The processes are
started with the 'spawn' method, so no CUDA state of the test process is inherited.
Only the oracle computes here; the seeded inputs are regenerated in each process."""
import os

import numpy as np

_CACHE = {}


def _oracle(kind, tol, workers):
    from oracle import newmark, spectral
    from paper_2211_08263_gb300 import inputs
    spectral.WORKERS = max(1, int(workers))
    key = (kind, tol)
    if key not in _CACHE:
        if kind == "c3":
            prob = inputs.config_c3(nsteps=400, n=256)
        else:
            raise ValueError(kind)
        _CACHE[key] = (prob, newmark.oracle_from_problem(prob, tol=tol, maxit=2000))
    return _CACHE[key]


def oracle_step(kind, state_path, out_path, n, tol, workers):
    """Load (u, v, a) = the state after step n - 1 ([c][N3][N2][N1] arrays in an .npz),
    take oracle step n (U = U(t_n)) and save u_n in the same layout; returns the step's
    PCG record."""
    from oracle import newmark
    prob, nm = _oracle(kind, tol, workers)
    z = np.load(state_path)
    st = newmark.state_from_abi(prob, z["u"], z["v"], z["a"])
    ns, info = nm.step(st, prob.U[n - 1])
    np.save(out_path, ns.u.reshape(z["u"].shape))
    os.remove(state_path)
    return {"iters": int(info["iters"]), "ref": float(info["ref"]), "rel_res": float(info["rel_res"]),
            "converged": bool(info["converged"])}


def oracle_apply(kind, u_path, workers):
    """A u with the oracle's operator (Eq. Fourier_ND_A), in the [c][N3][N2][N1] layout."""
    prob, nm = _oracle(kind, 1e-13, workers)
    from oracle.medium import field_to_oracle
    u = np.load(u_path)
    return nm.A(field_to_oracle(prob, u)).reshape(u.shape)
