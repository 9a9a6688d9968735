"""Closed forms used to pin the oracle.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

* Elastic plane waves (Christoffel problem; the acoustic tensor of Eq. acous
  and the eigenvalue problem of Eq. Eigenvalues_1D_homogeneo):
  rho omega^2 a = K(xi) a,  K_ik = C_ijkl xi_j xi_l.
* Discrete beta-Newmark phase of a single mode (gamma = 1/2): with
  Omega = omega dt, u_n = u_0 cos(n phi) for v_0 = 0, a_0 = -omega^2 u_0, where
  cos(phi) = (1 - (1/2 - beta) Omega^2) / (1 + beta Omega^2).
* Isotropic wave speeds c_L = sqrt((lambda + 2 mu)/rho), c_S = sqrt(mu/rho)
  (Eq. wave_velocity-nd).
* Cubic-crystal speeds along [100], [110], [111] (textbook).
* 1-D d'Alembert solution with periodic images and reflection /
  transmission coefficients at an interface (App. C), and the layered bar's
  solution built from them wave by wave (pinned by the homogeneous closed form
  and by the interface conditions of Eq. wave_boundary).
"""
from __future__ import annotations

import numpy as np


def christoffel(C: np.ndarray, rho: float, xi: np.ndarray):
    """Eigenpairs of K(xi)/rho for a (d,d,d,d) tensor: returns (omega^2, vectors)."""
    d = len(xi)
    K = np.einsum("ijkl,j,l->ik", C[(slice(0, d),) * 4], xi, xi)
    w2, vecs = np.linalg.eigh(K / rho)
    return w2, vecs


def newmark_cos_phi(Omega: float, beta: float = 0.25) -> float:
    return (1.0 - (0.5 - beta) * Omega * Omega) / (1.0 + beta * Omega * Omega)


def isotropic_speeds(lam: float, mu: float, rho: float):
    return np.sqrt((lam + 2 * mu) / rho), np.sqrt(mu / rho)


def lame(E: float, nu: float):
    return E * nu / ((1 + nu) * (1 - 2 * nu)), E / (2 * (1 + nu))


def cubic_speeds(c11: float, c12: float, c44: float, rho: float):
    """rho c^2 for the three propagation directions of a cubic crystal."""
    return {
        "100": sorted([c11 / rho, c44 / rho, c44 / rho]),
        "110": sorted([(c11 + c12 + 2 * c44) / (2 * rho), c44 / rho, (c11 - c12) / (2 * rho)]),
        "111": sorted([(c11 + 2 * c12 + 4 * c44) / (3 * rho), (c11 - c12 + c44) / (3 * rho),
                       (c11 - c12 + c44) / (3 * rho)]),
    }


def dalembert_periodic(x: np.ndarray, t: float, x0: float, c0: float, L: float, Ufun) -> np.ndarray:
    """Displacement of a periodic homogeneous bar driven at x0 by u(x0, t) = U(t):
    a right-going wave U(t - s/c0) and a left-going one U(t - (L - s)/c0),
    s = (x - x0) mod L; valid until the waves return to x0 (t < L/c0 + pulse)."""
    s = np.mod(x - x0, L)
    return Ufun(t - s / c0) + Ufun(t - (L - s) / c0)


def layered_dalembert_periodic(x: np.ndarray, t: float, bounds, c, Z, Ufun) -> np.ndarray:
    """Displacement of a periodic layered bar [bounds[0], bounds[-1]) driven at x = bounds[0]
    (= bounds[-1]) by u(0, t) = U(t), by superposing d'Alembert waves (App. C, Eq.
    soL_wave_eq) ray by ray: layer k spans [bounds[k], bounds[k+1]) with speed c[k] and
    impedance Z[k].  A wave leaves the source both ways; at an interface it splits into a
    reflected and a transmitted wave with the amplitude ratios of App. C (Eq.
    wave_transmission_reflection); at the source point, held at U(t) = 0 once the pulse has
    passed, it reflects with ratio -1.  Waves whose front reaches a boundary after t are not
    split further.  U must vanish for negative arguments."""
    x = np.asarray(x, dtype=np.float64)
    nl = len(c)
    L = bounds[-1]
    u = np.zeros_like(x)
    # each wave: amplitude, direction (+1 right), layer, the point and time its front leaves
    waves = [(1.0, +1, 0, bounds[0], 0.0), (1.0, -1, nl - 1, L, 0.0)]
    while waves:
        a, d, k, xs, ts = waves.pop()
        lo, hi = bounds[k], bounds[k + 1]
        ahead = (x >= lo) & (x < hi) & ((x - xs) * d >= 0)
        u[ahead] += a * Ufun(t - ts - np.abs(x[ahead] - xs) / c[k])
        xe = hi if d > 0 else lo
        th = ts + abs(xe - xs) / c[k]
        if th > t:
            continue
        if (d > 0 and k == nl - 1) or (d < 0 and k == 0):
            waves.append((-a, -d, k, xe, th))  # the source point
            continue
        r, tr = reflection_transmission(Z[k], Z[k + d])
        waves.append((a * r, -d, k, xe, th))
        waves.append((a * tr, d, k + d, xe, th))
    return u


def reflection_transmission(Z1: float, Z2: float):
    """Amplitude ratios of a displacement wave from medium 1 into medium 2 (App. C):
    A_T / A_I = 2 / (1 + Z2/Z1),  A_R / A_I = (1 - Z2/Z1) / (1 + Z2/Z1)."""
    r = Z2 / Z1
    return (1 - r) / (1 + r), 2.0 / (1 + r)
