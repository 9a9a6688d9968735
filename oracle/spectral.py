"""Spectral operator, right-hand side and preconditioner of the implicit FFT
method, FP64, written from the paper's equations with scipy.fft.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

* Discrete frequencies: Eq. frequencies / Eq. freq3D (Sec. 2.1.3, 2.2.3).
  Reading for even N (the paper only runs odd N): the unpaired frequency
  -N/2 (k = N/2 in FFT order) gets derivative multiplier 0, in the operator
  and in the preconditioner alike.  This makes every spectral derivative a
  real, skew-symmetric matrix (it equals the closed-form periodic
  differentiation matrix, see oracle.dense).
* Operator A: Eq. Fourier_ND_A (Sec. 2.2.2), evaluated in real space:
      eps_lm = F^-1{ (i/2)(u^_l xi_m + u^_m xi_l) },  sig_jk = C_jklm(x) eps_lm,
      (A u)_j = -theta F^-1{ i xi_k F{sig_jk} } + rho(x) u_j,  theta = beta dt^2.
* Right-hand side b: Eq. Fourier_ND_b, b = rho (u + dt v + dt^2 (1/2 - beta) a).
* Preconditioner: Eq. precond / Eq. acous (Sec. 2.2.3),
      M^(xi) = (theta K(xi) + rho_bar I)^-1,  K_ij = Cbar_ikjm xi_k xi_m,
  Cbar, rho_bar volume averages; solved per frequency with numpy.linalg.solve.
"""
from __future__ import annotations

import os

import numpy as np
import scipy.fft as sfft

from .medium import Medium

WORKERS = os.cpu_count() or 1
_CHUNK = 1 << 18


def wavenumbers(N: int, L: float) -> np.ndarray:
    """Discrete frequencies xi_k in FFT order (Eq. frequencies), Nyquist -> 0."""
    k = np.arange(N)
    kk = np.where(k <= (N - 1) // 2, k, k - N).astype(np.float64)
    xi = 2.0 * np.pi * kk / L
    if N % 2 == 0:
        xi[N // 2] = 0.0
    return xi


class Spectral:
    """Real-to-complex transforms over the d spatial axes of a medium and the
    frequency vector xi on the half spectrum (last array axis = x_1 is the
    real-FFT axis)."""

    def __init__(self, med: Medium):
        self.d = med.d
        self.shape = tuple(med.shape)
        self.axes = tuple(range(-self.d, 0))
        self.xi = []
        for i in range(self.d):
            ax = self.d - 1 - i  # position of axis x_{i+1} in the spatial shape
            N = self.shape[ax]
            x = wavenumbers(N, med.L[i])
            if i == 0:
                x = x[: N // 2 + 1]
            bshape = [1] * self.d
            bshape[ax] = x.size
            self.xi.append(x.reshape(bshape))
        self.hshape = tuple(self.shape[:-1]) + (self.shape[-1] // 2 + 1,)

    def fwd(self, f: np.ndarray) -> np.ndarray:
        return sfft.rfftn(f, axes=self.axes, workers=WORKERS)

    def inv(self, F: np.ndarray) -> np.ndarray:
        return sfft.irfftn(F, s=self.shape, axes=self.axes, workers=WORKERS)

    def deriv(self, f: np.ndarray, i: int) -> np.ndarray:
        """d f / d x_{i+1} = F^-1{ i xi_i F{f} } (Eq. Fourier_derivatives)."""
        return self.inv(1j * self.xi[i] * self.fwd(f))


def hooke(med: Medium, eps: np.ndarray) -> np.ndarray:
    """sigma_ij(x) = C_ijkl(x) eps_kl(x) voxel by voxel; eps is (d, d, *shape)."""
    d = med.d
    e = eps.reshape(d, d, -1)
    out = np.empty_like(e)
    ph = med.phase.reshape(-1)
    V = ph.size
    for s in range(0, V, _CHUNK):
        C = med.Ctab[ph[s:s + _CHUNK]]
        out[:, :, s:s + _CHUNK] = np.einsum("vijkl,klv->ijv", C, e[:, :, s:s + _CHUNK])
    return out.reshape(eps.shape)


def strain(sp: Spectral, u: np.ndarray) -> np.ndarray:
    """eps_lm = F^-1{ (i/2)(u^_l xi_m + u^_m xi_l) } (inner term of Eq. Fourier_ND_A)."""
    d = sp.d
    uh = [sp.fwd(u[l]) for l in range(d)]
    eps = np.empty((d, d) + sp.shape)
    for l in range(d):
        for m in range(d):
            eps[l, m] = sp.inv(0.5j * (uh[l] * sp.xi[m] + uh[m] * sp.xi[l]))
    return eps


def divergence(sp: Spectral, sig: np.ndarray) -> np.ndarray:
    """t_j = F^-1{ i xi_k F{sig_jk} } (outer term of Eq. Fourier_ND_A)."""
    d = sp.d
    t = np.empty((d,) + sp.shape)
    for j in range(d):
        acc = np.zeros(sp.hshape, dtype=np.complex128)
        for k in range(d):
            acc += 1j * sp.xi[k] * sp.fwd(sig[j, k])
        t[j] = sp.inv(acc)
    return t


def apply_A(med: Medium, sp: Spectral, u: np.ndarray, theta: float) -> np.ndarray:
    """Operator A of Eq. Fourier_ND_A in real space:
    (A u)_j = -theta div(C : grad^s u)_j + rho u_j."""
    sig = hooke(med, strain(sp, u))
    return -theta * divergence(sp, sig) + med.rho[None] * u


def rhs_b(med: Medium, u, v, a, dt: float, beta: float) -> np.ndarray:
    """b = rho (u_{n-1} + dt v_{n-1} + dt^2 (1/2 - beta) a_{n-1})  (Eq. Fourier_ND_b)."""
    return med.rho[None] * (u + dt * v + dt * dt * (0.5 - beta) * a)


def acoustic_tensor(sp: Spectral, Cbar: np.ndarray) -> np.ndarray:
    """K_ij(xi) = Cbar_ikjm xi_k xi_m on the half spectrum, shape (*hshape, d, d) (Eq. acous)."""
    d = sp.d
    xi = [np.broadcast_to(sp.xi[k], sp.hshape) for k in range(d)]
    K = np.zeros(sp.hshape + (d, d))
    for i in range(d):
        for j in range(d):
            for k in range(d):
                for m in range(d):
                    if Cbar[i, k, j, m] != 0.0:
                        K[..., i, j] += Cbar[i, k, j, m] * xi[k] * xi[m]
    return K


def apply_M(med: Medium, sp: Spectral, r: np.ndarray, theta: float,
            Cbar: np.ndarray = None, rhobar: float = None) -> np.ndarray:
    """Preconditioner z = F^-1{ (theta K(xi) + rho_bar I)^-1 F{r} } (Eq. precond)."""
    d = sp.d
    if Cbar is None:
        Cbar = med.C_mean()
    if rhobar is None:
        rhobar = med.rho_mean()
    K = acoustic_tensor(sp, Cbar).reshape(-1, d, d)
    Mmat = theta * K + rhobar * np.eye(d)[None]
    rh = np.stack([sp.fwd(r[i]).reshape(-1) for i in range(d)], axis=-1)
    zh = np.empty_like(rh)
    n = rh.shape[0]
    for s in range(0, n, _CHUNK):
        zh[s:s + _CHUNK] = np.linalg.solve(Mmat[s:s + _CHUNK].astype(np.complex128),
                                           rh[s:s + _CHUNK][..., None])[..., 0]
    return np.stack([sp.inv(zh[:, i].reshape(sp.hshape)) for i in range(d)])


def strain_energy(med: Medium, sp: Spectral, u: np.ndarray) -> float:
    """(1/2) sum_x eps : C : eps with the spectral strain of u."""
    eps = strain(sp, u)
    sig = hooke(med, eps)
    return 0.5 * float(np.sum(eps * sig))


def kinetic_energy(med: Medium, v: np.ndarray) -> float:
    return 0.5 * float(np.sum(med.rho[None] * v * v))
