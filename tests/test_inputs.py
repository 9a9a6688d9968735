"""Seeded input generators: determinism and the stated recipes (CPU)."""
import numpy as np

from paper_2211_08263_gb300 import inputs


def test_rotations_are_proper_orthogonal():
    R = inputs.random_rotations(np.random.default_rng(0), 50)
    assert np.allclose(np.einsum("nij,nkj->nik", R, R), np.eye(3)[None], atol=1e-14)
    assert np.allclose(np.linalg.det(R), 1.0)


def test_voronoi_matches_brute_force_periodic_nearest_seed():
    rng = np.random.default_rng(4)
    n = (9, 7, 5)
    ids, seeds = inputs.periodic_voronoi(n, 11, rng)
    box = np.array(n, float)
    for z in range(n[2]):
        for y in range(n[1]):
            for x in range(n[0]):
                p = np.array([x + 0.5, y + 0.5, z + 0.5])
                d = p - seeds
                d -= box * np.round(d / box)
                dist = np.sqrt((d * d).sum(1))
                assert dist[ids[z, y, x]] <= dist.min() + 1e-12


def test_spheres_do_not_overlap_and_inputs_are_deterministic():
    p1 = inputs.config_c2(nsteps=3, n=48, nsph=6, rmin=4, rmax=6)
    p2 = inputs.config_c2(nsteps=3, n=48, nsph=6, rmin=4, rmax=6)
    assert np.array_equal(p1.phase, p2.phase)
    cs, rs = p1.extra["centres"], p1.extra["radii"]
    box = np.full(3, 48.0)
    for i in range(len(cs)):
        for j in range(i + 1, len(cs)):
            d = cs[i] - cs[j]
            d -= box * np.round(d / box)
            assert np.linalg.norm(d) > rs[i] + rs[j] + 1
    frac = (p1.phase == 0).mean()
    expect = sum(4 / 3 * np.pi * r ** 3 for r in rs) / 48 ** 3
    assert abs(frac - expect) < 0.1 * expect


def test_polycrystal_tables_are_rotated_cubic():
    ids, Cv, rho = inputs.polycrystal((16, 16, 16), 20, 3)
    assert ids.max() < 20 and Cv.shape == (20, 21) and np.all(rho == inputs.NI_RHO)
    base = inputs.cubic_voigt(*inputs.NI_CUBIC)
    # rotation invariants of the 6x6 matrix are not preserved in general, but the
    # bulk modulus (1/9 sum_{ij<=3} C_iijj) is
    kb = base[:3, :3].sum() / 9
    for v in Cv:
        m = inputs.matrix_from_voigt21(v)
        assert abs(m[:3, :3].sum() / 9 - kb) < 1e-6 * kb


def test_pulses():
    t = np.linspace(0, 3e-5, 301)
    s = inputs.sin2_pulse(t, 1e-6, 2e-5)
    assert s.max() <= 1e-6 and abs(s[100] - 1e-6) < 1e-18 and np.all(s[t >= 2e-5] == 0)
    b = inputs.bell_pulse(t, 1.0, np.pi / 2e-5, 4)
    assert abs(b[100] - 1.0) < 1e-12 and np.all(b[t > 2e-5] == 0)
    g = inputs.gaussian_pulse(t, 2.0, 1e-6, 1e-5)
    assert abs(g[100] - 2.0) < 1e-12


def test_config_c1_shape():
    p = inputs.config_c1()
    assert p.ndim == 2 and p.n == (64, 64, 1) and p.mask.shape == (2, 1, 64, 64)
    assert p.mask[:, :, :, :3].all() and not p.mask[:, :, :, 3:].any()
    assert p.U.shape == (50, 3) and np.all(p.U[:, 1:] == 0)
