"""Explicit central-difference FFT scheme (Sec. 2.3: Eq. Central_diff_rule,
Eq. Explicit_linear_momentum_arranged_3D with the spectral operator of
Eq. b_explicit), FP64: the beta = 0, gamma = 1/2 member of the Newmark family.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Per step n, with the velocity Udot(t_n) prescribed on Gamma:
  u_n  = u + dt v + dt^2/2 a                          (every DOF, explicit)
  v_b  = v + dt/2 a + dt/(2 rho) div(C : grad^s u_n)  (the known part of v_n)
  f_n  = 2 rho/dt (Udot - v_b) on Gamma, 0 elsewhere  (the force that enforces Udot)
  v_n  = v_b + dt/(2 rho) f_n                         (= Udot on Gamma)
  a_n  = 2 (v_n - v)/dt - a                            (gamma = 1/2 solved for a_n)
so that rho a_n = div sigma(u_n) + f_n.  Reaction per component: the sum of f_n
over the grid (= sum of rho a_n, the divergence summing to zero on the torus).

Stable increment (Eq. Courant_stable with Eq. Eigenvalues_1D_homogeneo):
dt <= 2 / omega_max, omega_max^2 the largest eigenvalue of
Q_ik = C_ijkl xi_j xi_l / rho at xi_i = N_i pi / L_i; for a heterogeneous medium
this reading takes the largest value over the voxels' (C, rho) pairs.
"""
from __future__ import annotations

import numpy as np

from . import spectral
from .medium import Medium
from .newmark import State


def div_sigma(med: Medium, sp: spectral.Spectral, u: np.ndarray) -> np.ndarray:
    """div(C : grad^s u) through the spectral derivatives (Eq. b_explicit)."""
    return spectral.divergence(sp, spectral.hooke(med, spectral.strain(sp, u)))


class ExplicitOracle:
    """Central-difference stepper on a Medium; mask: bool (d, *shape), True on Gamma."""

    def __init__(self, med: Medium, mask: np.ndarray, dt: float):
        self.med = med
        self.sp = spectral.Spectral(med)
        self.mask = mask.astype(bool)
        self.dt = dt

    def zero_state(self) -> State:
        z = np.zeros((self.med.d,) + tuple(self.med.shape))
        return State(z, z.copy(), z.copy())

    def step(self, s: State, Udot):
        dt, rho = self.dt, self.med.rho[None]
        u = s.u + dt * s.v + 0.5 * dt * dt * s.a
        vb = s.v + 0.5 * dt * s.a + dt / (2.0 * rho) * div_sigma(self.med, self.sp, u)
        g = np.stack([np.full(self.med.shape, float(Udot[j])) for j in range(self.med.d)])
        f = np.where(self.mask, 2.0 * rho / dt * (g - vb), 0.0)
        vn = vb + dt / (2.0 * rho) * f
        an = 2.0 * (vn - s.v) / dt - s.a
        reaction = [float(f[j].sum()) for j in range(self.med.d)]
        return State(u, vn, an), reaction

    def run(self, Udot: np.ndarray, nsteps: int = None, state: State = None):
        """Advance from `state` (rest by default); Udot[n-1] = Udot(t_n)."""
        s = self.zero_state() if state is None else state
        nsteps = Udot.shape[0] if nsteps is None else nsteps
        reactions = []
        for n in range(nsteps):
            s, r = self.step(s, Udot[n])
            reactions.append(r)
        return s, reactions


def omega_max(med: Medium) -> float:
    """sqrt of the largest eigenvalue of C_ijkl xi_j xi_l / rho at xi_i = N_i pi / L_i
    over the voxels' (C, rho) pairs."""
    d = med.d
    xi = np.array([med.shape[d - 1 - i] * np.pi / med.L[i] for i in range(d)])
    best = 0.0
    for p in np.unique(med.phase):
        rho_min = float(med.rho[med.phase == p].min())
        Q = np.einsum("ijkl,j,l->ik", med.Ctab[p], xi, xi) / rho_min
        best = max(best, float(np.linalg.eigvalsh(0.5 * (Q + Q.T)).max()))
    return float(np.sqrt(best))


def stable_dt(med: Medium) -> float:
    """Largest stable increment of the explicit scheme, 2 / omega_max."""
    return 2.0 / omega_max(med)
