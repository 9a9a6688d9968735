"""beta-Newmark time stepping of the implicit FFT method (Eq. Newmark,
Eq. ND_consv_lm_Newmark_ord, Alg. 2), FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Per step n (t_n = n dt):
  predictor   u~ = u_{n-1} + dt v_{n-1} + dt^2 (1/2 - beta) a_{n-1},  b = rho u~
  solve       u_n with u_n|_Gamma = U(t_n) and (A u_n - b)|_free = 0
              (masked PCG, or the dense / Green's-matrix variants)
  corrector   a_n = (u_n - u~) / (beta dt^2)
              v_n = v_{n-1} + dt ((1 - gamma) a_{n-1} + gamma a_n)
Reaction on Gamma: f_n = (A u_n - b) / theta (zero off Gamma up to the
tolerance); its sum per component equals sum_x rho a_n (momentum balance).
Initial acceleration: every workload starts at rest, a_0 = 0 (reading of the
garbled preprocessing line of Alg. 2: a_0 = rho^-1 div(C : grad^s u_0)).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import spectral
from .medium import Medium, medium_from_problem, field_to_oracle, mask_to_oracle
from .pcg import masked_pcg


@dataclass
class State:
    u: np.ndarray
    v: np.ndarray
    a: np.ndarray

    def copy(self):
        return State(self.u.copy(), self.v.copy(), self.a.copy())


class NewmarkOracle:
    """Masked-PCG Newmark stepper on a Medium.

    mask: bool (d, *shape), True on prescribed DOFs.
    warm: 'prev' (x0 = u_{n-1}, the paper's choice) or 'taylor'
          (x0 = u~ + beta dt^2 a_{n-1} = u + dt v + dt^2/2 a).
    """

    def __init__(self, med: Medium, mask: np.ndarray, dt: float, beta: float = 0.25,
                 gamma: float = 0.5, tol: float = 1e-10, maxit: int = 1000, warm: str = "prev"):
        self.med = med
        self.sp = spectral.Spectral(med)
        self.mask = mask.astype(bool)
        self.dt, self.beta, self.gamma = dt, beta, gamma
        self.theta = beta * dt * dt
        self.tol, self.maxit, self.warm = tol, maxit, warm
        self.Cbar = med.C_mean()
        self.rhobar = med.rho_mean()

    def A(self, u):
        return spectral.apply_A(self.med, self.sp, u, self.theta)

    def M(self, r):
        return spectral.apply_M(self.med, self.sp, r, self.theta, self.Cbar, self.rhobar)

    def zero_state(self) -> State:
        z = np.zeros((self.med.d,) + tuple(self.med.shape))
        return State(z, z.copy(), z.copy())

    def gamma_field(self, Uvec) -> np.ndarray:
        """Field holding U_j on the prescribed DOFs of component j."""
        d = self.med.d
        g = np.zeros((d,) + tuple(self.med.shape))
        for j in range(d):
            g[j] = np.where(self.mask[j], Uvec[j], 0.0)
        return g

    def predictor(self, s: State):
        dt, beta = self.dt, self.beta
        ut = s.u + dt * s.v + dt * dt * (0.5 - beta) * s.a
        b = self.med.rho[None] * ut
        return ut, b

    def warm_start(self, s: State, ut):
        if self.warm == "prev":
            return s.u.copy()
        if self.warm == "taylor":
            return ut + self.theta * s.a
        raise ValueError(self.warm)

    def solve(self, b, x0, Uvec, tol=None):
        return masked_pcg(self.A, self.M, b, x0, self.mask, self.gamma_field(Uvec),
                          self.tol if tol is None else tol, self.maxit)

    def corrector(self, s: State, x, ut) -> State:
        a_new = (x - ut) / self.theta
        v_new = s.v + self.dt * ((1.0 - self.gamma) * s.a + self.gamma * a_new)
        return State(x, v_new, a_new)

    def step(self, s: State, Uvec, x0=None):
        ut, b = self.predictor(s)
        if x0 is None:
            x0 = self.warm_start(s, ut)
        x, info = self.solve(b, x0, Uvec)
        ns = self.corrector(s, x, ut)
        d = self.med.d
        info["reaction"] = [float(np.sum(self.med.rho * ns.a[j])) for j in range(d)]
        return ns, info

    def reaction_field(self, s_new: State, b) -> np.ndarray:
        """f_n = (A u_n - b)/theta (supported on Gamma)."""
        return (self.A(s_new.u) - b) / self.theta

    def energy(self, s: State) -> float:
        """E_n = 1/2 sum rho |v|^2 + 1/2 sum eps : C : eps."""
        return spectral.kinetic_energy(self.med, s.v) + spectral.strain_energy(self.med, self.sp, s.u)

    def run(self, U: np.ndarray, nsteps: int = None, state: State = None, callback=None):
        """Advance nsteps steps from `state` (rest by default); U[n-1] = U(t_n)."""
        s = self.zero_state() if state is None else state
        nsteps = U.shape[0] if nsteps is None else nsteps
        infos = []
        for n in range(nsteps):
            s, info = self.step(s, U[n])
            infos.append(info)
            if callback is not None:
                callback(n + 1, s, info)
        return s, infos


def oracle_from_problem(prob, tol=None, warm="prev", maxit=1000) -> NewmarkOracle:
    med = medium_from_problem(prob)
    return NewmarkOracle(med, mask_to_oracle(prob), prob.dt, prob.beta, prob.gamma,
                         prob.tol if tol is None else tol, maxit, warm)


def state_to_abi(prob, s: State):
    """Oracle state -> [c][N3][N2][N1] arrays."""
    shp = (prob.ndim, prob.n[2], prob.n[1], prob.n[0])
    return s.u.reshape(shp), s.v.reshape(shp), s.a.reshape(shp)


def state_from_abi(prob, u, v, a) -> State:
    return State(field_to_oracle(prob, u).copy(), field_to_oracle(prob, v).copy(),
                 field_to_oracle(prob, a).copy())
