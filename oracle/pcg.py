"""Preconditioned conjugate gradient (Sec. 2.2.3: CG on the real field, valid
because the operator is Hermitian; preconditioned with M of Eq. precond).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

``masked_pcg`` solves the constrained problem that the paper's Green's-matrix
construction (Eqs. lin_prob1, u_p, deconvolution, L-determination_ND) reaches:
u|_Gamma = U and (A u - b) = 0 on every free DOF.  P zeroes the prescribed
DOFs.  Stopping test (reading of the paper's unspecified "tolerance"): the
2-norm of the masked true-recursion residual relative to
ref = || P (b - A x_Gamma) ||, x_Gamma = U on Gamma and 0 elsewhere.
"""
from __future__ import annotations

import numpy as np


def dot(a: np.ndarray, b: np.ndarray) -> float:
    return float(np.dot(a.reshape(-1), b.reshape(-1)))


def masked_pcg(Aop, Mop, b: np.ndarray, x0: np.ndarray, mask: np.ndarray, xgam: np.ndarray,
               tol: float, maxit: int = 1000):
    """Masked PCG.

    Aop(v): operator A;  Mop(v): preconditioner M;  b: right-hand side;
    x0: warm start (its Gamma values are overwritten);  mask: bool, True on
    prescribed DOFs;  xgam: field holding the prescribed values on Gamma.
    Returns (x, info) with info = {iters, ref, rel_res, converged}.
    Iteration count = number of applications q = P A p.
    """
    P = lambda v: np.where(mask, 0.0, v)
    x = np.where(mask, xgam, x0)
    x_g = np.where(mask, xgam, 0.0)
    ref = np.sqrt(dot(P(b - Aop(x_g)), P(b - Aop(x_g))))
    if ref == 0.0:
        return x_g, {"iters": 0, "ref": 0.0, "rel_res": 0.0, "converged": True}
    r = P(b - Aop(x))
    rn = np.sqrt(dot(r, r))
    if rn <= tol * ref:
        return x, {"iters": 0, "ref": ref, "rel_res": rn / ref, "converged": True}
    z = P(Mop(r))
    p = z.copy()
    rz = dot(r, z)
    it = 0
    converged = False
    while it < maxit:
        q = P(Aop(p))
        alpha = rz / dot(p, q)
        x = x + alpha * p
        r = r - alpha * q
        it += 1
        rn = np.sqrt(dot(r, r))
        if rn <= tol * ref:
            converged = True
            break
        z = P(Mop(r))
        rz_new = dot(r, z)
        beta = rz_new / rz
        p = z + beta * p
        rz = rz_new
    return x, {"iters": it, "ref": ref, "rel_res": rn / ref, "converged": converged}


def pcg(Aop, Mop, b: np.ndarray, x0: np.ndarray, tol: float, maxit: int = 1000):
    """Plain PCG for A x = b with relative residual ||r|| <= tol ||b||
    (the unconstrained solves of Alg. 2)."""
    x = x0.copy()
    r = b - Aop(x)
    bn = np.sqrt(dot(b, b))
    if bn == 0.0:
        return np.zeros_like(b), {"iters": 0, "rel_res": 0.0, "converged": True}
    z = Mop(r)
    p = z.copy()
    rz = dot(r, z)
    it = 0
    rn = np.sqrt(dot(r, r))
    while rn > tol * bn and it < maxit:
        q = Aop(p)
        alpha = rz / dot(p, q)
        x = x + alpha * p
        r = r - alpha * q
        it += 1
        rn = np.sqrt(dot(r, r))
        if rn <= tol * bn:
            break
        z = Mop(r)
        rz_new = dot(r, z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, {"iters": it, "rel_res": rn / bn, "converged": rn <= tol * bn}
