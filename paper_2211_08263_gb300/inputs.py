"""Seeded synthetic inputs for the implicit FFT elastodynamics solver.

This module is shared by the FP64 oracle and the CUDA path.  It holds only
input construction: microstructures (phase maps, per-phase stiffness and
density tables), Dirichlet masks and prescribed-displacement time series.
None of the solver's arithmetic (operator, preconditioner, Krylov solve,
Newmark update) lives here.

Array conventions (shared with the C ABI):
  * scalar voxel fields are C-ordered ``[N3][N2][N1]`` (x fastest);
    2-D problems use ``N3 = 1``;
  * vector fields are ``[c][N3][N2][N1]`` with ``c = ndim``;
  * a stiffness is 21 Voigt upper-triangle values in the order
    (11,22,33,23,13,12) x (11,22,33,23,13,12), row by row:
    C11 C12 C13 C14 C15 C16 C22 C23 ... C66, with no factor 2 anywhere
    (C_IJ = C_ijkl where I=(ij), J=(kl));
  * a Dirichlet mask is uint8 ``[c][N3][N2][N1]``, 1 = prescribed.

The material recipes stand in for the paper's microstructures (Sec. 4:
spherical inclusions in a matrix, a weighted-Voronoi nickel polycrystal);
the pulses are the time functions of Sec. 3.1 (Eq. prescribed_displacement)
and the sin^2 / Gaussian pulses of the synthetic workloads.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

VOIGT_PAIRS = ((0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1))


def voigt21_from_matrix(m: np.ndarray) -> np.ndarray:
    """Pack a symmetric 6x6 Voigt matrix into 21 upper-triangle values."""
    out = []
    for i in range(6):
        for j in range(i, 6):
            out.append(m[i, j])
    return np.asarray(out, dtype=np.float64)


def matrix_from_voigt21(v: np.ndarray) -> np.ndarray:
    m = np.zeros((6, 6))
    k = 0
    for i in range(6):
        for j in range(i, 6):
            m[i, j] = m[j, i] = v[k]
            k += 1
    return m


def isotropic_voigt(E: float, nu: float) -> np.ndarray:
    """6x6 Voigt stiffness of an isotropic solid from Young's modulus and
    Poisson's ratio (Lame constants lambda, mu)."""
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    m = np.zeros((6, 6))
    m[:3, :3] = lam
    for i in range(3):
        m[i, i] = lam + 2 * mu
        m[3 + i, 3 + i] = mu
    return m


def isotropic_lame_voigt(lam: float, mu: float) -> np.ndarray:
    m = np.zeros((6, 6))
    m[:3, :3] = lam
    for i in range(3):
        m[i, i] = lam + 2 * mu
        m[3 + i, 3 + i] = mu
    return m


def cubic_voigt(c11: float, c12: float, c44: float) -> np.ndarray:
    m = np.zeros((6, 6))
    m[:3, :3] = c12
    for i in range(3):
        m[i, i] = c11
        m[3 + i, 3 + i] = c44
    return m


def _tensor_from_voigt_matrix(m: np.ndarray) -> np.ndarray:
    c = np.zeros((3, 3, 3, 3))
    for I, (i, j) in enumerate(VOIGT_PAIRS):
        for J, (k, l) in enumerate(VOIGT_PAIRS):
            v = m[I, J]
            for a, b in ((i, j), (j, i)):
                for cc, d in ((k, l), (l, k)):
                    c[a, b, cc, d] = v
    return c


def _voigt_matrix_from_tensor(c: np.ndarray) -> np.ndarray:
    m = np.zeros((6, 6))
    for I, (i, j) in enumerate(VOIGT_PAIRS):
        for J, (k, l) in enumerate(VOIGT_PAIRS):
            m[I, J] = c[i, j, k, l]
    return m


def rotate_voigt(m: np.ndarray, R: np.ndarray) -> np.ndarray:
    """Stiffness of a crystal rotated by R: C'_ijkl = R_ia R_jb R_kc R_ld C_abcd."""
    c = _tensor_from_voigt_matrix(m)
    cr = np.einsum("ia,jb,kc,ld,abcd->ijkl", R, R, R, R, c, optimize=True)
    return _voigt_matrix_from_tensor(cr)


def random_rotations(rng: np.random.Generator, n: int) -> np.ndarray:
    """Uniformly distributed rotations from uniform random unit quaternions
    (Shoemake, Graphics Gems III, 1992): three uniforms per rotation."""
    u = rng.random((n, 3))
    q1 = np.sqrt(1 - u[:, 0]) * np.sin(2 * np.pi * u[:, 1])
    q2 = np.sqrt(1 - u[:, 0]) * np.cos(2 * np.pi * u[:, 1])
    q3 = np.sqrt(u[:, 0]) * np.sin(2 * np.pi * u[:, 2])
    q0 = np.sqrt(u[:, 0]) * np.cos(2 * np.pi * u[:, 2])
    w, x, y, z = q0, q1, q2, q3
    R = np.empty((n, 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - z * w)
    R[:, 0, 2] = 2 * (x * z + y * w)
    R[:, 1, 0] = 2 * (x * y + z * w)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - x * w)
    R[:, 2, 0] = 2 * (x * z - y * w)
    R[:, 2, 1] = 2 * (y * z + x * w)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


# ----------------------------------------------------------------------------
# microstructures
# ----------------------------------------------------------------------------

def voxel_centres(shape_xyz, h=(1.0, 1.0, 1.0)):
    """Voxel centre coordinates x_i = h_i (1/2 + idx_i) (Sec. 2.2.3)."""
    n1, n2, n3 = shape_xyz
    x = (np.arange(n1) + 0.5) * h[0]
    y = (np.arange(n2) + 0.5) * h[1]
    z = (np.arange(n3) + 0.5) * h[2]
    return x, y, z


def periodic_voronoi(shape_xyz, nseeds: int, rng: np.random.Generator) -> tuple:
    """Periodic Voronoi grain map (grain id per voxel, uint16).

    Seeds are uniform in [0, N_i) (units of voxels); each voxel centre takes
    the id of the nearest seed under the periodic minimum-image distance.
    Returns (ids[N3,N2,N1], seeds[nseeds,3]).
    """
    from scipy.spatial import cKDTree

    n1, n2, n3 = shape_xyz
    seeds = rng.random((nseeds, 3)) * np.array([n1, n2, n3], dtype=np.float64)
    tree = cKDTree(seeds, boxsize=[n1, n2, n3])
    ids = np.empty((n3, n2, n1), dtype=np.uint16)
    xs = np.arange(n1) + 0.5
    ys = np.arange(n2) + 0.5
    gx, gy = np.meshgrid(xs, ys, indexing="xy")  # [n2, n1]
    plane = np.stack([gx.ravel(), gy.ravel(), np.zeros(gx.size)], axis=1)
    for k in range(n3):
        plane[:, 2] = k + 0.5
        _, idx = tree.query(plane, k=1, workers=-1)
        ids[k] = idx.reshape(n2, n1).astype(np.uint16)
    return ids, seeds


def sphere_composite(shape_xyz, nsph: int, rmin: float, rmax: float, rng: np.random.Generator,
                     max_attempts: int = 100000):
    """Two-phase map: phase 0 inside non-overlapping periodic spheres, 1 outside.

    Per attempt the centre (x, y, z uniform in [0, N_i)) is drawn, then the
    radius (uniform in [rmin, rmax]); a candidate is kept when its periodic
    minimum-image distance to every kept sphere exceeds r1 + r2 + 1.
    """
    n = np.array(shape_xyz, dtype=np.float64)
    cs, rs = [], []
    att = 0
    while len(cs) < nsph:
        att += 1
        if att > max_attempts:
            raise RuntimeError("sphere packing failed")
        c = rng.random(3) * n
        r = rmin + (rmax - rmin) * rng.random()
        ok = True
        for c2, r2 in zip(cs, rs):
            d = c - c2
            d -= n * np.round(d / n)
            if np.sqrt((d * d).sum()) <= r + r2 + 1:
                ok = False
                break
        if ok:
            cs.append(c)
            rs.append(r)
    n1, n2, n3 = shape_xyz
    ids = np.ones((n3, n2, n1), dtype=np.uint16)
    x = np.arange(n1) + 0.5
    y = np.arange(n2) + 0.5
    z = np.arange(n3) + 0.5
    for c, r in zip(cs, rs):
        dx = x - c[0]
        dx -= n1 * np.round(dx / n1)
        dy = y - c[1]
        dy -= n2 * np.round(dy / n2)
        dz = z - c[2]
        dz -= n3 * np.round(dz / n3)
        d2 = dz[:, None, None] ** 2 + dy[None, :, None] ** 2 + dx[None, None, :] ** 2
        ids[d2 <= r * r] = 0
    return ids, np.array(cs), np.array(rs)


# ----------------------------------------------------------------------------
# time functions U(t)
# ----------------------------------------------------------------------------

def sin2_pulse(t, amp, period):
    """amp * sin^2(pi t / period) for 0 <= t < period, else 0."""
    t = np.asarray(t, dtype=np.float64)
    return np.where((t >= 0) & (t < period), amp * np.sin(np.pi * t / period) ** 2, 0.0)


def gaussian_pulse(t, amp, width, centre):
    t = np.asarray(t, dtype=np.float64)
    return amp * np.exp(-((t - centre) ** 2) / (2 * width * width))


def bell_pulse(t, amp, omega, alpha):
    """Bell-shaped pulse of Sec. 3.1 (Eq. prescribed_displacement):
    amp (t (pi/omega - t))^alpha / ((pi/omega)^2/4)^alpha on [0, pi/omega]."""
    t = np.asarray(t, dtype=np.float64)
    T = np.pi / omega
    val = amp * (t * (T - t)) ** alpha / ((T * T / 4.0) ** alpha)
    return np.where((t >= 0) & (t <= T), val, 0.0)


# ----------------------------------------------------------------------------
# problem description
# ----------------------------------------------------------------------------

@dataclass
class Problem:
    """One periodic elastodynamics problem on a voxel grid.

    n = (N1, N2, N3) (N3 = 1 for ndim = 2), h = voxel size per axis (m).
    phase: uint16 [N3,N2,N1] grain/phase id, or None for per-voxel tables
    (then C has V rows and rho has V entries).  C: [nphase, 21] Voigt;
    rho: [nphase].  mask: uint8 [c,N3,N2,N1].  U: [nsteps, 3] prescribed
    displacement U(t_n) for n = 1..nsteps (component j applies to DOFs of
    component j on the mask).
    """
    name: str
    ndim: int
    n: tuple
    h: tuple
    dt: float
    beta: float
    gamma: float
    C: np.ndarray
    rho: np.ndarray
    phase: Optional[np.ndarray]
    mask: np.ndarray
    U: np.ndarray
    tol: float = 1e-10
    extra: dict = field(default_factory=dict)

    @property
    def nsteps(self):
        return self.U.shape[0]

    @property
    def nvox(self):
        return int(self.n[0] * self.n[1] * self.n[2])

    @property
    def spatial_shape(self):
        return (self.n[2], self.n[1], self.n[0])

    def C_field(self):
        """Per-voxel Voigt table rows (V, 21) (materialises a dense copy)."""
        if self.phase is None:
            return self.C
        return self.C[self.phase.reshape(-1)]

    def rho_field(self):
        if self.phase is None:
            return self.rho.reshape(self.spatial_shape)
        return self.rho[self.phase]

    def truncated(self, nsteps: int) -> "Problem":
        import copy
        p = copy.copy(self)
        p.U = self.U[:nsteps].copy()
        return p


def slab_mask(ndim, n, width, comps=None):
    """Mask of the x-face slab x_idx < width (all components by default)."""
    c = ndim
    m = np.zeros((c, n[2], n[1], n[0]), dtype=np.uint8)
    comps = range(c) if comps is None else comps
    for j in comps:
        m[j, :, :, :width] = 1
    return m


def _U_series(nsteps, dt, fn):
    t = dt * np.arange(1, nsteps + 1)
    U = np.zeros((nsteps, 3))
    U[:, 0] = fn(t)
    return U


def config_c1(nsteps: int = 50) -> Problem:
    """2-D plane strain 64x64, homogeneous isotropic steel-like medium,
    strip x_idx < 3 prescribed u_x = 1e-6 sin^2(pi t / 2e-5), u_y = 0."""
    n = (64, 64, 1)
    Cv = voigt21_from_matrix(isotropic_voigt(200e9, 0.3))[None, :]
    rho = np.array([7800.0])
    phase = np.zeros((1, 64, 64), dtype=np.uint16)
    dt = 2e-7
    U = _U_series(nsteps, dt, lambda t: sin2_pulse(t, 1e-6, 2e-5))
    return Problem("c1_2d_64", 2, n, (1e-3, 1e-3, 1e-3), dt, 0.25, 0.5, Cv, rho, phase,
                   slab_mask(2, n, 3), U, tol=1e-10)


MATRIX_PHASE = (70e9, 0.33, 2700.0)
INCLUSION_PHASE = (400e9, 0.25, 3900.0)


def config_c2(nsteps: int = 200, n: int = 128, nsph: int = 20, rmin=8.0, rmax=14.0, seed=2) -> Problem:
    """3-D two-phase composite: non-overlapping periodic spheres (phase 0,
    E=400 GPa, nu=0.25, rho=3900) in a matrix (phase 1, 70 GPa, 0.33, 2700);
    x-face slab of 4 voxels, sin^2 pulse (period 2e-5 s) on u_x."""
    rng = np.random.default_rng(seed)
    ids, cs, rs = sphere_composite((n, n, n), nsph, rmin, rmax, rng)
    Cv = np.stack([voigt21_from_matrix(isotropic_voigt(INCLUSION_PHASE[0], INCLUSION_PHASE[1])),
                   voigt21_from_matrix(isotropic_voigt(MATRIX_PHASE[0], MATRIX_PHASE[1]))])
    rho = np.array([INCLUSION_PHASE[2], MATRIX_PHASE[2]])
    dt = 2e-7
    U = _U_series(nsteps, dt, lambda t: sin2_pulse(t, 1e-6, 2e-5))
    return Problem(f"c2_composite_{n}", 3, (n, n, n), (1e-3,) * 3, dt, 0.25, 0.5, Cv, rho, ids,
                   slab_mask(3, (n, n, n), 4), U, tol=1e-10, extra={"centres": cs, "radii": rs})


NI_CUBIC = (168.4e9, 121.4e9, 75.4e9)
NI_RHO = 8960.0


def polycrystal(n_xyz, ngrains, seed):
    rng = np.random.default_rng(seed)
    ids, _ = periodic_voronoi(n_xyz, ngrains, rng)
    Rs = random_rotations(rng, ngrains)
    base = cubic_voigt(*NI_CUBIC)
    Cv = np.stack([voigt21_from_matrix(rotate_voigt(base, R)) for R in Rs])
    rho = np.full(ngrains, NI_RHO)
    return ids, Cv, rho


def config_c3(nsteps: int = 400, n: int = 256, ngrains: int = 500, seed: int = 3,
              width_steps: float = 50.0, nz: Optional[int] = None, ny: Optional[int] = None) -> Problem:
    """3-D nickel polycrystal: periodic Voronoi grains with uniformly random
    orientations of a cubic crystal (C11=168.4, C12=121.4, C44=75.4 GPa,
    rho=8960); Gaussian pulse (sigma = 50 dt, centre 4 sigma) on u_x of the
    4-voxel x-face slab.  ny, nz: n x ny x nz voxels instead of the cube
    (smaller cases with some of the cube's transforms, e.g. for profiler captures)."""
    shape = (n, ny if ny else n, nz if nz else n)
    ids, Cv, rho = polycrystal(shape, ngrains, seed)
    dt = 2e-7
    w = width_steps * dt
    U = _U_series(nsteps, dt, lambda t: gaussian_pulse(t, 1e-6, w, 4 * w))
    name = (f"c3_polycrystal_{n}" if shape[1] == n and shape[2] == n
            else f"c3_polycrystal_{n}x{shape[1]}x{shape[2]}")
    return Problem(name, 3, shape, (1e-3,) * 3, dt, 0.25, 0.5, Cv, rho, ids,
                   slab_mask(3, shape, 4), U, tol=1e-10, extra={"seed": seed, "ngrains": ngrains})


# nickel single crystal of the polycrystalline bar (Sec. 4.3)
NI_BAR_CUBIC = (249e9, 155e9, 114e9)
NI_BAR_RHO = 8908.0


def config_bar567(nsteps: int = 60, pulse_grains: float = 20.0, seed: int = 567,
                  dt_cfl: float = 10.0) -> Problem:
    """The polycrystalline bar of Sec. 4.3: 35 x 35 x 567 voxels of 10 um (0.35 x 0.35 x
    5.67 mm), nickel grains (C11 = 249, C12 = 155, C44 = 114 GPa, rho = 8908) with random
    orientations; bell pulse (Eq. prescribed_displacement, alpha = 4, A = 5.67e-6 m,
    omega = pi c / (pulse_grains d_g), c = sqrt(C11 / rho), d_g = 100 um) on u_3 of the
    plane x_3 = 0, u_1 = u_2 = 0 there.  Synthetic stand-in for the paper's microstructure:
    a periodic Voronoi map with as many grains as spheres of 100 um fill the bar (the
    paper's weighted, log-normal tessellation is not reproduced).  dt = dt_cfl * CFL with
    CFL = h / c (Sec. 3.1); pulse_grains = 3 is the paper's short pulse, 20 its long one."""
    n = (35, 35, 567)
    h = 1e-5
    dg = 1e-4
    V = n[0] * n[1] * n[2]
    ngrains = int(round(V * h ** 3 / (np.pi / 6.0 * dg ** 3)))
    rng = np.random.default_rng(seed)
    ids, _ = periodic_voronoi(n, ngrains, rng)
    Rs = random_rotations(rng, ngrains)
    base = cubic_voigt(*NI_BAR_CUBIC)
    Cv = np.stack([voigt21_from_matrix(rotate_voigt(base, R)) for R in Rs])
    rho = np.full(ngrains, NI_BAR_RHO)
    c0 = np.sqrt(NI_BAR_CUBIC[0] / NI_BAR_RHO)
    dt = dt_cfl * h / c0
    omega = np.pi * c0 / (pulse_grains * dg)
    t = dt * np.arange(1, nsteps + 1)
    U = np.zeros((nsteps, 3))
    U[:, 2] = bell_pulse(t, 5.67e-6, omega, 4.0)
    mask = np.zeros((3, n[2], n[1], n[0]), dtype=np.uint8)
    mask[:, 0, :, :] = 1
    return Problem("bar_polycrystal_35x35x567", 3, n, (h,) * 3, dt, 0.25, 0.5, Cv, rho, ids, mask, U,
                   tol=1e-10, extra={"seed": seed, "ngrains": ngrains, "pulse_grains": pulse_grains})


# Aluminium of the paper's material table (Sec. 3.1): E, nu, rho
AL_E_NU_RHO = (70.3e9, 0.345, 2700.0)


def config_sphere129(nsteps: int = 6, pulse_steps: float = 12.0) -> Problem:
    """Spherical waves in a homogeneous solid (Sec. 4.1): a 1 m aluminium cube of
    129^3 voxels (129 = 3 x 43), dt = 1.52e-6 s, the bell pulse (Eq.
    prescribed_displacement, alpha = 4, amplitude 1 mm) on u_1 of the voxels whose
    centres lie within R = 1 cm of the centre of the cube (the centre voxel and its six
    face neighbours at h = 7.75 mm), u_2 = u_3 = 0 there.  The pulse frequency is not
    printed for this case: omega = pi / (pulse_steps dt), a pulse of pulse_steps steps."""
    n = (129, 129, 129)
    h = 1.0 / 129
    E, nu, rho = AL_E_NU_RHO
    Cv = voigt21_from_matrix(isotropic_voigt(E, nu))[None, :]
    dt = 1.52e-6
    x = (np.arange(129) + 0.5) * h - 0.5
    r2 = x[:, None, None] ** 2 + x[None, :, None] ** 2 + x[None, None, :] ** 2
    mask = np.zeros((3, 129, 129, 129), dtype=np.uint8)
    mask[:, r2 <= 0.01 ** 2] = 1
    t = dt * np.arange(1, nsteps + 1)
    U = np.zeros((nsteps, 3))
    U[:, 0] = bell_pulse(t, 1e-3, np.pi / (pulse_steps * dt), 4.0)
    phase = np.zeros((129, 129, 129), dtype=np.uint16)
    return Problem("sphere_al_129", 3, n, (h,) * 3, dt, 0.25, 0.5, Cv, np.array([rho]), phase, mask, U,
                   tol=1e-10, extra={"pulse_steps": pulse_steps})


FE_E_NU_RHO = (211.4e9, 0.293, 7850.0)


def config_plate1025(nsteps: int = 4, framed: bool = False, n: int = 1025, pulse_steps: float = 12.0) -> Problem:
    """Circular waves in a plate (Sec. 4.1): 0.001 x 1 x 1 m discretised in 1 x n x n voxels
    (n = 1025 = 5^2 x 41 in the paper), aluminium, or (framed) an aluminium square of
    0.39 x 0.39 m in the centre of an iron frame; dt = 1.9e-6 s; the bell pulse (Eq.
    prescribed_displacement, alpha = 4, amplitude 1 mm) on u_1 (perpendicular to the plate)
    of the voxels whose centres lie within R = 2.5 mm of the plate's centre, u_2 = u_3 = 0
    there.  The pulse frequency is not printed: omega = pi / (pulse_steps dt)."""
    shape_xyz = (1, n, n)
    h = (1e-3, 1.0 / n, 1.0 / n)
    mats = [AL_E_NU_RHO, FE_E_NU_RHO]
    Cv = np.stack([voigt21_from_matrix(isotropic_voigt(E, nu)) for E, nu, _ in mats])
    rho = np.array([r for _, _, r in mats])
    y = (np.arange(n) + 0.5) / n - 0.5  # centres along x_2 and x_3, origin at the plate's centre
    phase = np.zeros((n, n, 1), dtype=np.uint16)  # [N3][N2][N1]
    if framed:
        inside = (np.abs(y)[:, None] < 0.195) & (np.abs(y)[None, :] < 0.195)
        phase[:, :, 0] = np.where(inside, 0, 1)
    r2 = y[:, None] ** 2 + y[None, :] ** 2
    mask = np.zeros((3, n, n, 1), dtype=np.uint8)
    mask[:, r2 <= 2.5e-3 ** 2, 0] = 1
    dt = 1.9e-6
    t = dt * np.arange(1, nsteps + 1)
    U = np.zeros((nsteps, 3))
    U[:, 0] = bell_pulse(t, 1e-3, np.pi / (pulse_steps * dt), 4.0)
    return Problem(f"plate_{'framed' if framed else 'al'}_{n}", 3, shape_xyz, h, dt, 0.25, 0.5, Cv, rho, phase,
                   mask, U, tol=1e-10, extra={"pulse_steps": pulse_steps})


BATCH_SIZES = (64, 80, 96, 128, 144, 160, 192)


def config_c4_specs(ninst: int = 48, seed: int = 48):
    """Sizes and grain counts of the uneven batch (drawn, not built)."""
    rng = np.random.default_rng(seed)
    sizes = rng.choice(np.array(BATCH_SIZES), size=ninst)
    grains = rng.integers(50, 801, size=ninst)
    return [(int(s), int(g), 1000 + i) for i, (s, g) in enumerate(zip(sizes, grains))]


def config_c4_instance(size: int, ngrains: int, seed: int, nsteps: int = 100) -> Problem:
    ids, Cv, rho = polycrystal((size, size, size), ngrains, seed)
    dt = 2e-7
    U = _U_series(nsteps, dt, lambda t: gaussian_pulse(t, 1e-6, 10 * dt, 40 * dt))
    return Problem(f"c4_inst_{size}_{seed}", 3, (size,) * 3, (1e-3,) * 3, dt, 0.25, 0.5, Cv, rho, ids,
                   slab_mask(3, (size,) * 3, 4), U, tol=1e-10)


def random_problem(rng: np.random.Generator, ndim: int, n, nphase: int = 3, mask_width: int = 1,
                   nsteps: int = 3, dense: bool = False, contrast: float = 3.0, dt: float = 2e-7,
                   h: float = 1e-3, anisotropic: bool = True) -> Problem:
    """Small random heterogeneous problem for parity tests: random phase map,
    random (rotated cubic or isotropic) stiffnesses, random densities."""
    n = tuple(n)
    shape = (n[2], n[1], n[0])
    mats = []
    for p in range(nphase):
        scale = 1.0 + (contrast - 1.0) * rng.random()
        if anisotropic:
            base = cubic_voigt(*(np.array(NI_CUBIC) * scale / 1.5))
            mats.append(rotate_voigt(base, random_rotations(rng, 1)[0]))
        else:
            E = 70e9 * scale
            nu = 0.2 + 0.15 * rng.random()
            mats.append(isotropic_voigt(E, nu))
    Cv = np.stack([voigt21_from_matrix(m) for m in mats])
    rho = 2700.0 + 6000.0 * rng.random(nphase)
    phase = rng.integers(0, nphase, size=shape).astype(np.uint16)
    if dense:
        V = int(np.prod(shape))
        Cv = Cv[phase.reshape(-1)]
        rho = rho[phase.reshape(-1)]
        phase = None
    mask = slab_mask(ndim, n, mask_width) if mask_width > 0 else np.zeros((ndim,) + shape, np.uint8)
    U = np.zeros((nsteps, 3))
    U[:, :ndim] = 1e-6 * rng.standard_normal((nsteps, ndim))
    return Problem(f"rand_{ndim}d_{'x'.join(map(str, n))}", ndim, n, (h,) * 3, dt, 0.25, 0.5, Cv, rho,
                   phase, mask, U, tol=1e-12)
