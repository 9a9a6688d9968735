"""Dense-matrix form of the discrete operator, with no FFT anywhere.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The DFT derivative of Eq. Fourier_derivatives on N equispaced points with the
Nyquist multiplier set to zero (reading for even N) is the periodic spectral
differentiation matrix, written in closed form (Trefethen, "Spectral Methods
in MATLAB", SIAM 2000, ch. 3), with h = 2 pi / N and period L:
    N even:  D_jk = (2 pi / L) * 1/2 (-1)^(j-k) cot((j-k) h / 2),  j != k
    N odd:   D_jk = (2 pi / L) * 1/2 (-1)^(j-k) csc((j-k) h / 2),  j != k
    D_jj = 0.
Grid derivatives are Kronecker products of the 1-D matrices.  The operator
of Eq. Fourier_ND_A is assembled as A = -theta Div S Eps + diag(rho), with
Eps the symmetric-gradient matrix, S the block-diagonal stiffness and Div
the divergence matrix; the constrained step problem
    A_FF u_F = b_F - A_FG U_G
is solved with one LU factorisation (A does not change in time).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sps

from .medium import Medium


def diff_matrix_1d(N: int, L: float) -> np.ndarray:
    """Closed-form periodic spectral differentiation matrix (see module doc)."""
    D = np.zeros((N, N))
    if N == 1:
        return D
    h = 2.0 * np.pi / N
    for j in range(N):
        for k in range(N):
            if j == k:
                continue
            m = j - k
            sgn = -1.0 if (m % 2) else 1.0
            if N % 2 == 0:
                D[j, k] = 0.5 * sgn / np.tan(m * h / 2.0)
            else:
                D[j, k] = 0.5 * sgn / np.sin(m * h / 2.0)
    return D * (2.0 * np.pi / L)


def grid_derivatives(shape, L):
    """Sparse matrices D_i (i = 0 for x_1) acting on C-ordered fields of `shape`
    (spatial axes ordered x_d ... x_1)."""
    d = len(shape)
    mats = []
    for i in range(d):
        ax = d - 1 - i
        M = sps.identity(1, format="csr")
        for a in range(d):
            blk = sps.csr_matrix(diff_matrix_1d(shape[a], L[i])) if a == ax else sps.identity(shape[a], format="csr")
            M = sps.kron(M, blk, format="csr")
        mats.append(M)
    return mats


def dense_operator(med: Medium, theta: float) -> np.ndarray:
    """Assembled A (dV x dV) on the stacked DOF vector [u_1; ...; u_d]."""
    d, V = med.d, med.nvox
    D = grid_derivatives(med.shape, med.L)
    # symmetric gradient: eps_kl = 1/2 (D_l u_k + D_k u_l), rows (k, l)
    rows = []
    for k in range(d):
        for l in range(d):
            blocks = [None] * d
            for c in range(d):
                blk = None
                if c == k:
                    blk = 0.5 * D[l]
                if c == l:
                    blk = 0.5 * D[k] if blk is None else blk + 0.5 * D[k]
                blocks[c] = blk if blk is not None else sps.csr_matrix((V, V))
            rows.append(blocks)
    Eps = sps.bmat(rows, format="csr")
    # stiffness: sig_ij = C_ijkl(x) eps_kl
    ph = med.phase.reshape(-1)
    srows = []
    for i in range(d):
        for j in range(d):
            srows.append([sps.diags(med.Ctab[ph, i, j, k, l]) for k in range(d) for l in range(d)])
    S = sps.bmat(srows, format="csr")
    # divergence: t_i = D_j sig_ij
    drows = []
    for i in range(d):
        blocks = []
        for a in range(d):
            for b in range(d):
                blocks.append(D[b] if a == i else sps.csr_matrix((V, V)))
        drows.append(blocks)
    Div = sps.bmat(drows, format="csr")
    SE = (S @ Eps).toarray()
    A = -theta * (Div @ SE)
    A += np.diag(np.tile(med.rho.reshape(-1), d))
    return A


class DenseConstrainedSolver:
    """Direct solve of A u = b on the free DOFs with u fixed on Gamma."""

    def __init__(self, A: np.ndarray, mask_flat: np.ndarray):
        self.A = A
        self.G = np.flatnonzero(mask_flat)
        self.F = np.flatnonzero(~mask_flat)
        self.lu = sla.lu_factor(A[np.ix_(self.F, self.F)])
        self.AFG = A[np.ix_(self.F, self.G)]

    def solve(self, b: np.ndarray, xgam_flat: np.ndarray) -> np.ndarray:
        x = np.zeros_like(b)
        Ug = xgam_flat[self.G]
        x[self.G] = Ug
        x[self.F] = sla.lu_solve(self.lu, b[self.F] - self.AFG @ Ug)
        return x


class DenseNewmark:
    """Newmark stepping with the dense constrained solve (exact discrete reference)."""

    def __init__(self, nm):
        """nm: an oracle.newmark.NewmarkOracle supplying medium, mask and constants."""
        self.nm = nm
        self.A = dense_operator(nm.med, nm.theta)
        self.solver = DenseConstrainedSolver(self.A, nm.mask.reshape(-1))

    def step(self, s, Uvec):
        ut, b = self.nm.predictor(s)
        x = self.solver.solve(b.reshape(-1), self.nm.gamma_field(Uvec).reshape(-1)).reshape(b.shape)
        return self.nm.corrector(s, x, ut)

    def run(self, U, nsteps=None, state=None):
        s = self.nm.zero_state() if state is None else state
        nsteps = U.shape[0] if nsteps is None else nsteps
        for n in range(nsteps):
            s = self.step(s, U[n])
        return s
