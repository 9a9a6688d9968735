"""Mistakes planted in the FP64 oracle, on the CPU, must fail its pins.

Each case replaces one function of the oracle's spectral operator (Eq. Fourier_ND_A),
preconditioner (Eq. precond), Newmark update (Eq. Newmark) or masked conjugate gradient
(Sec. 2.2.3) by a copy with one plausible
slip -- a dropped factor or term, a wrong sign, a wrong index -- and runs a few fast pins
of tests/test_oracle_pins.py against it: at least one must fail.  The pins compare the oracle with things outside it
(the dense operator assembled from the closed-form differentiation matrix, the exact
inverse of a homogeneous medium, the discrete Newmark phase of a plane wave), so this
checks that they would notice.  CPU only."""
import numpy as np
import pytest

from oracle import newmark, pcg, spectral
from tests import test_oracle_pins as pins

# a planted mistake may overflow or divide by zero on its way to failing a pin
pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _strain_no_half(sp, u):
    d = sp.d
    uh = [sp.fwd(u[l]) for l in range(d)]
    eps = np.empty((d, d) + sp.shape)
    for l in range(d):
        for m in range(d):
            eps[l, m] = sp.inv(1j * (uh[l] * sp.xi[m] + uh[m] * sp.xi[l]))  # the 1/2 dropped
    return eps


def _divergence_sign(sp, sig):
    d = sp.d
    t = np.empty((d,) + sp.shape)
    for j in range(d):
        acc = np.zeros(sp.hshape, dtype=np.complex128)
        for k in range(d):
            acc -= 1j * sp.xi[k] * sp.fwd(sig[j, k])  # sign flipped
        t[j] = sp.inv(acc)
    return t


def _divergence_index(sp, sig):
    d = sp.d
    t = np.empty((d,) + sp.shape)
    for j in range(d):
        acc = np.zeros(sp.hshape, dtype=np.complex128)
        for k in range(d):
            acc += 1j * sp.xi[j] * sp.fwd(sig[j, k])  # xi_j instead of xi_k
        t[j] = sp.inv(acc)
    return t


def _hooke_swapped(med, eps):
    d = med.d
    e = eps.reshape(d, d, -1)
    C = med.Ctab[med.phase.reshape(-1)]
    return np.einsum("vikjl,klv->ijv", C, e).reshape(eps.shape)  # C_ikjl instead of C_ijkl


def _apply_A_no_mass(med, sp, u, theta):
    return -theta * spectral.divergence(sp, spectral.hooke(med, spectral.strain(sp, u)))  # rho u dropped


def _acoustic_transposed(sp, Cbar):
    d = sp.d
    xi = [np.broadcast_to(sp.xi[k], sp.hshape) for k in range(d)]
    K = np.zeros(sp.hshape + (d, d))
    for i in range(d):
        for j in range(d):
            for k in range(d):
                for m in range(d):
                    K[..., i, j] += Cbar[i, j, k, m] * xi[k] * xi[m]  # C_ijkm instead of C_ikjm
    return K


_ORIG_APPLY_M = spectral.apply_M


def _apply_M_no_theta(med, sp, r, theta, Cbar=None, rhobar=None):
    # theta folded away: (K + rho_bar I)^-1, i.e. theta = 1
    return _ORIG_APPLY_M(med, sp, r, 1.0, Cbar, rhobar)


def _predictor_sign(self, s):
    ut = s.u + self.dt * s.v + self.dt * self.dt * (0.5 + self.beta) * s.a  # + beta instead of - beta
    return ut, self.med.rho[None] * ut


def _corrector_no_old_acceleration(self, s, x, ut):
    a_new = (x - ut) / self.theta
    v_new = s.v + self.dt * self.gamma * a_new  # the (1 - gamma) a_{n-1} term dropped
    return newmark.State(x, v_new, a_new)


def _corrector_without_beta(self, s, x, ut):
    a_new = (x - ut) / (self.dt * self.dt)  # dt^2 instead of beta dt^2
    v_new = s.v + self.dt * ((1.0 - self.gamma) * s.a + self.gamma * a_new)
    return newmark.State(x, v_new, a_new)


def _pcg(project_q=True, beta_inverted=False):
    """The masked PCG with one slip switched on (else the same steps as oracle.pcg)."""
    def run(Aop, Mop, b, x0, mask, xgam, tol, maxit=1000):
        P = lambda v: np.where(mask, 0.0, v)
        x = np.where(mask, xgam, x0)
        x_g = np.where(mask, xgam, 0.0)
        ref = np.sqrt(pcg.dot(P(b - Aop(x_g)), P(b - Aop(x_g))))
        if ref == 0.0:
            return x_g, {"iters": 0, "ref": 0.0, "rel_res": 0.0, "converged": True}
        r = P(b - Aop(x))
        z = P(Mop(r))
        p = z.copy()
        rz = pcg.dot(r, z)
        it, rn = 0, np.sqrt(pcg.dot(r, r))
        while it < maxit and rn > tol * ref:
            q = P(Aop(p)) if project_q else Aop(p)
            alpha = rz / pcg.dot(p, q)
            x = x + alpha * p
            r = r - alpha * q
            it += 1
            rn = np.sqrt(pcg.dot(r, r))
            z = P(Mop(r))
            rz_new = pcg.dot(r, z)
            p = z + (rz / rz_new if beta_inverted else rz_new / rz) * p
            rz = rz_new
        return x, {"iters": it, "ref": ref, "rel_res": rn / ref, "converged": rn <= tol * ref}
    return run


PCG_MUTATIONS = {
    "A p not projected": _pcg(project_q=False),
    "beta inverted": _pcg(beta_inverted=True),
}

NEWMARK_MUTATIONS = {
    "predictor sign": ("predictor", _predictor_sign),
    "corrector drops the old acceleration": ("corrector", _corrector_no_old_acceleration),
    "corrector without beta": ("corrector", _corrector_without_beta),
}

MUTATIONS = {
    "strain without 1/2": ("strain", _strain_no_half),
    "divergence sign": ("divergence", _divergence_sign),
    "divergence index": ("divergence", _divergence_index),
    "Hooke indices swapped": ("hooke", _hooke_swapped),
    "mass term dropped": ("apply_A", _apply_A_no_mass),
    "acoustic tensor transposed": ("acoustic_tensor", _acoustic_transposed),
    "preconditioner without theta": ("apply_M", _apply_M_no_theta),
}

PINS = [
    lambda: pins.test_fft_operator_equals_dense_operator(*pins.CASES[0]),
    lambda: pins.test_fft_operator_equals_dense_operator(*pins.CASES[-1]),
    lambda: pins.test_preconditioner_is_exact_inverse_for_homogeneous_medium(3, True),
    lambda: pins.test_plane_wave_follows_discrete_newmark_closed_form(3, True, 0),
]


NEWMARK_PINS = [
    lambda: pins.test_plane_wave_follows_discrete_newmark_closed_form(3, True, 0),
    lambda: pins.test_plane_wave_follows_discrete_newmark_closed_form(2, False, 1),
    pins.test_energy_conserved_in_free_vibration,
]


def _failures(pins_):
    failed = 0
    for pin in pins_:
        try:
            pin()
        except (AssertionError, np.linalg.LinAlgError, ValueError, FloatingPointError):
            failed += 1
    return failed


PCG_PINS = [
    lambda: pins.test_green_matrix_masked_pcg_and_dense_agree(2, (8, 8, 1), 2),
    lambda: pins.test_green_matrix_masked_pcg_and_dense_agree(3, (6, 6, 6), 1),
]


def test_pins_pass_on_the_unchanged_oracle():
    for pin in PINS + NEWMARK_PINS + PCG_PINS:
        pin()


def test_unchanged_copy_of_the_pcg_passes_the_pins(monkeypatch):
    """The copy used for the PCG mutations, with no slip, is the oracle's algorithm."""
    monkeypatch.setattr(newmark, "masked_pcg", _pcg())
    assert _failures(PCG_PINS) == 0


@pytest.mark.parametrize("name", list(PCG_MUTATIONS))
def test_planted_pcg_mistake_fails_a_pin(monkeypatch, name):
    monkeypatch.setattr(newmark, "masked_pcg", PCG_MUTATIONS[name])
    assert _failures(PCG_PINS) >= 1, f"no pin noticed: {name}"


@pytest.mark.parametrize("name", list(NEWMARK_MUTATIONS))
def test_planted_newmark_mistake_fails_a_pin(monkeypatch, name):
    attr, bad = NEWMARK_MUTATIONS[name]
    monkeypatch.setattr(newmark.NewmarkOracle, attr, bad)
    assert _failures(NEWMARK_PINS) >= 1, f"no pin noticed: {name}"


@pytest.mark.parametrize("name", list(MUTATIONS))
def test_planted_mistake_fails_a_pin(monkeypatch, name):
    attr, bad = MUTATIONS[name]
    monkeypatch.setattr(spectral, attr, bad)
    assert _failures(PINS) >= 1, f"no pin noticed: {name}"
