"""Voxel medium for the oracle (Sec. 2.2.1 and 2.2.3: C(x) and rho(x) sampled
at voxel centres).

The oracle works on ``d``-dimensional arrays whose spatial axes are ordered
(x_d, ..., x_2, x_1): displacement component ``i`` (0-based) differentiates
along array axis ``-1 - i``.  A 2-D problem is plane strain: its stiffness is
the in-plane block C_ijkl, i,j,k,l in {1,2}, of the 3-D tensor.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Optional

import numpy as np

# Voigt index of the symmetric pair (i, j), order 11,22,33,23,13,12.
_VOIGT = {(0, 0): 0, (1, 1): 1, (2, 2): 2, (1, 2): 3, (2, 1): 3, (0, 2): 4, (2, 0): 4, (0, 1): 5, (1, 0): 5}


def tensor_from_voigt21(v21: np.ndarray) -> np.ndarray:
    """Full 3x3x3x3 stiffness tensor(s) from 21 upper-triangle Voigt values.

    C_ijkl = Cv[I, J] with I = voigt(i, j), J = voigt(k, l): no factor 2,
    the tensor is minor- and major-symmetric by construction.
    Accepts (..., 21) and returns (..., 3, 3, 3, 3).
    """
    v21 = np.asarray(v21, dtype=np.float64)
    lead = v21.shape[:-1]
    m = np.zeros(lead + (6, 6))
    k = 0
    for I in range(6):
        for J in range(I, 6):
            m[..., I, J] = v21[..., k]
            m[..., J, I] = v21[..., k]
            k += 1
    c = np.zeros(lead + (3, 3, 3, 3))
    for i in range(3):
        for j in range(3):
            for kk in range(3):
                for ll in range(3):
                    c[..., i, j, kk, ll] = m[..., _VOIGT[(i, j)], _VOIGT[(kk, ll)]]
    return c


@dataclass
class Medium:
    """d-dimensional periodic voxel medium.

    shape: spatial array shape (N_d, ..., N_1);  L: cell lengths (L_1..L_d);
    Ctab: (nphase, d, d, d, d) stiffness tensors;  phase: int array of
    ``shape`` (index into Ctab / rhotab);  rho: density field of ``shape``.
    """
    d: int
    shape: tuple
    L: tuple
    Ctab: np.ndarray
    phase: np.ndarray
    rho: np.ndarray

    @property
    def nvox(self):
        return int(np.prod(self.shape))

    def C_mean(self) -> np.ndarray:
        """Volume average of C(x) (Sec. 2.2.3, reference medium of Eq. precond)."""
        counts = np.bincount(self.phase.reshape(-1), minlength=self.Ctab.shape[0]).astype(np.float64)
        return np.einsum("p,pijkl->ijkl", counts, self.Ctab) / self.nvox

    def rho_mean(self) -> float:
        return float(self.rho.mean())


def medium_from_problem(prob) -> Medium:
    """Build the oracle's medium from a ``paper_2211_08263_gb300.inputs.Problem``."""
    d = prob.ndim
    n1, n2, n3 = prob.n
    if d == 3:
        shape = (n3, n2, n1)
    elif d == 2:
        assert n3 == 1
        shape = (n2, n1)
    else:
        raise ValueError("ndim must be 2 or 3")
    L = tuple(prob.n[i] * prob.h[i] for i in range(d))
    C3 = tensor_from_voigt21(prob.C)
    Ctab = C3[(slice(None),) + (slice(0, d),) * 4].copy()
    if prob.phase is None:
        phase = np.arange(prob.nvox, dtype=np.int64).reshape(shape)
        rho = np.asarray(prob.rho, dtype=np.float64).reshape(shape)
    else:
        phase = prob.phase.astype(np.int64).reshape(shape)
        rho = np.asarray(prob.rho, dtype=np.float64)[phase]
    return Medium(d, shape, L, Ctab, phase, rho)


def field_to_oracle(prob, arr: np.ndarray) -> np.ndarray:
    """[c][N3][N2][N1] array -> oracle vector field (d, *shape)."""
    arr = np.asarray(arr, dtype=np.float64)
    if prob.ndim == 2:
        return arr.reshape(2, prob.n[1], prob.n[0])
    return arr.reshape(3, prob.n[2], prob.n[1], prob.n[0])


def mask_to_oracle(prob) -> np.ndarray:
    return field_to_oracle(prob, prob.mask).astype(bool)


def homogeneous_medium(d: int, shape: tuple, L: tuple, C: np.ndarray, rho: float) -> Medium:
    """Single-phase medium; C is a (3,3,3,3) tensor (its first d indices are used)."""
    Ct = np.asarray(C)[(slice(0, d),) * 4][None].copy()
    return Medium(d, tuple(shape), tuple(L), Ct, np.zeros(shape, dtype=np.int64),
                  np.full(shape, float(rho)))
