"""The paper's literal Green's-matrix treatment of the prescribed-displacement
region (Sec. 2.2.3, Eqs. f_discrete, solve_green, g, G, Vt,
L-determination_ND; Alg. 2), for tiny grids.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Preprocessing: for every prescribed DOF (point p, direction j) solve
A u_(p,j) = e_(p,j) (unit force, Eq. f_discrete) with PCG, and store the
responses at the prescribed DOFs as column (p,j) of G (row = responding DOF
(q,i), column = forcing DOF (p,j); reading of the garbled index formula of
Eq. G); LU-factorise G once.
Per step: u_b = A^-1 b (PCG), V = U - u_b|_Gamma (Eq. Vt),
F = theta^-1 G^-1 V (Eq. L-determination_ND), u_f = theta A^-1 f with f = F
on Gamma, u_n = u_b + u_f; then the Newmark corrector.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .pcg import pcg


class GreenNewmark:
    def __init__(self, nm, tol: float = 1e-14, maxit: int = 2000):
        """nm: oracle.newmark.NewmarkOracle (medium, mask, constants, A and M)."""
        self.nm = nm
        self.tol, self.maxit = tol, maxit
        self.gam = np.flatnonzero(nm.mask.reshape(-1))
        shape = (nm.med.d,) + tuple(nm.med.shape)
        cols = []
        for g in self.gam:
            e = np.zeros(shape)
            e.reshape(-1)[g] = 1.0
            u, info = pcg(nm.A, nm.M, e, np.zeros(shape), tol, maxit)
            cols.append(u.reshape(-1)[self.gam])
        self.G = np.stack(cols, axis=1)
        self.lu = sla.lu_factor(self.G)

    def step(self, s, Uvec):
        nm = self.nm
        ut, b = nm.predictor(s)
        ub, _ = pcg(nm.A, nm.M, b, s.u, self.tol, self.maxit)
        Ug = nm.gamma_field(Uvec).reshape(-1)[self.gam]
        V = Ug - ub.reshape(-1)[self.gam]
        F = sla.lu_solve(self.lu, V) / nm.theta
        f = np.zeros_like(b)
        f.reshape(-1)[self.gam] = F
        uf, _ = pcg(nm.A, nm.M, f, np.zeros_like(b), self.tol, self.maxit)
        x = ub + nm.theta * uf
        return nm.corrector(s, x, ut), F

    def run(self, U, nsteps=None, state=None):
        s = self.nm.zero_state() if state is None else state
        nsteps = U.shape[0] if nsteps is None else nsteps
        forces = []
        for n in range(nsteps):
            s, F = self.step(s, U[n])
            forces.append(F)
        return s, forces
