"""The C-ABI library builds, loads and exports every symbol include/wfft.h
declares; host-side validation answers without a GPU (no compute calls)."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from paper_2211_08263_gb300 import inputs


@pytest.fixture(scope="module")
def lib():
    from paper_2211_08263_gb300 import build, wfft
    if not os.path.exists(build.LIB):
        build.build()
    return wfft.load()


def test_every_declared_symbol_is_exported(lib):
    from paper_2211_08263_gb300 import build, wfft
    declared = wfft.declared_symbols()
    assert len(declared) >= 15
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = [s for s in declared if s not in exported]
    assert not missing, missing
    for s in declared:
        assert hasattr(lib, s)


def test_default_options(lib):
    from paper_2211_08263_gb300 import wfft
    o = wfft.default_options()
    assert o.precision == wfft.FP64 and o.tol == 1e-10 and o.maxit == 1000 and o.check_every >= 1


@pytest.mark.parametrize("case", ["ndim", "n2d", "dt", "rho", "spd", "nphase", "allmasked", "prime", "bigprime",
                                  "1d", "long"])
def test_create_rejects_bad_inputs_before_device_work(lib, case):
    from paper_2211_08263_gb300 import wfft
    p = inputs.config_c1(2)
    kw = dict(ndim=2, n=(64, 64, 1), h=p.h, C_table=p.C, rho=p.rho, phase=p.phase, mask=p.mask, dt=p.dt)
    expect = wfft.EINVAL
    if case == "ndim":
        kw["ndim"] = 4
    elif case == "n2d":
        kw["n"] = (64, 64, 2)
    elif case == "dt":
        kw["dt"] = -1.0
    elif case == "rho":
        kw["rho"] = np.array([0.0])
    elif case == "spd":
        bad = p.C.copy()
        bad[0, 1] = 10 * bad[0, 0]  # C12 >> C11: indefinite
        kw["C_table"] = bad
    elif case == "nphase":
        ph = p.phase.copy()
        ph[0, 0, 0] = 3
        kw["phase"] = ph
    elif case == "allmasked":
        kw["mask"] = np.ones_like(p.mask)
    elif case == "prime":
        # 143 = 11 x 13: two prime factors above 7 (one general prime stage per axis)
        kw["n"] = (143, 64, 1)
        kw["phase"] = np.zeros((1, 64, 143), np.uint16)
        kw["mask"] = None
        expect = wfft.EUNSUPPORTED
    elif case == "bigprime":
        # 2 x 131: a prime factor above the largest direct DFT stage (127)
        kw["n"] = (262, 64, 1)
        kw["phase"] = np.zeros((1, 64, 262), np.uint16)
        kw["mask"] = None
        expect = wfft.EUNSUPPORTED
    elif case == "long":
        # 3^7: 7-smooth, but longer than any radix schedule is made for
        kw["n"] = (2187, 64, 1)
        kw["phase"] = np.zeros((1, 64, 2187), np.uint16)
        kw["mask"] = None
        expect = wfft.EUNSUPPORTED
    elif case == "1d":
        kw["ndim"] = 3
        kw["n"] = (64, 1, 1)
        kw["phase"] = np.zeros((1, 1, 64), np.uint16)
        kw["mask"] = None
        expect = wfft.EUNSUPPORTED
    with pytest.raises(wfft.WfftError) as e:
        wfft.Solver(**kw)
    assert e.value.code == expect


def test_last_error_without_handle_is_text(lib):
    assert isinstance(lib.wfft_last_error(None), bytes)


def test_model_blob_layout_and_initial_model(lib):
    """Host-only parts of the learned warm start: blob size, header, the zero
    output layer of an initial model (it reproduces the Taylor warm start) and the
    He scale of the hidden layers; round trip through the Python (un)packing."""
    from paper_2211_08263_gb300 import wfft
    assert wfft.model_bytes(8) == 0 and wfft.model_bytes(64) == 0
    for H in (16, 32):
        nparam = sum(27 * co * ci + co for co, ci in wfft.layer_shapes(H))
        assert wfft.model_bytes(H) == 32 + 4 * nparam
        blob = wfft.model_init(H, seed=3)
        hd = blob[:32].view(np.int32)
        assert list(hd) == [0x314E4657, 1, 4, 16, H, 3, 16, 0]
        hidden, params = wfft.blob_params(blob)
        assert hidden == H
        assert not params[3][0].any() and not params[3][1].any()
        for (W, b), (co, ci) in zip(params[:3], wfft.layer_shapes(H)[:3]):
            assert W.shape == (27, co, ci) and not b.any()
            assert abs(W.std() - np.sqrt(2.0 / (27 * ci))) < 0.1 * np.sqrt(2.0 / (27 * ci))
        assert np.array_equal(wfft.params_blob(H, params), blob)
        assert np.array_equal(wfft.model_init(H, seed=3), blob)
        assert not np.array_equal(wfft.model_init(H, seed=4), blob)


def test_trainer_and_network_calls_fail_cleanly(lib):
    from paper_2211_08263_gb300 import wfft
    blob = wfft.model_init(16, 0)
    with pytest.raises(wfft.WfftError) as e:
        wfft.Trainer(blob[:-4])
    assert e.value.code == wfft.EINVAL
    bad = blob.copy()
    bad[:4] = 0
    with pytest.raises(wfft.WfftError) as e:
        wfft.net_forward(bad, (4, 4, 4), np.zeros((64, 16), np.float32))
    assert e.value.code == wfft.EINVAL
    with pytest.raises(wfft.WfftError) as e:
        wfft.net_forward(blob, (0, 4, 4), np.zeros((0, 16), np.float32))
    assert e.value.code == wfft.EINVAL
    assert lib.wfft_set_model(None, None, 0) == wfft.EINVAL


@pytest.mark.parametrize("ndim", [2, 3])
def test_explicit_stable_increment_matches_the_reference(lib, ndim):
    """wfft_explicit_dt (host only) against the reference's 2 / omega_max over
    random rotated-cubic and isotropic phases with different densities."""
    from oracle import explicit, medium
    from paper_2211_08263_gb300 import inputs, wfft
    rng = np.random.default_rng(81 + ndim)
    n = (8, 6, 4) if ndim == 3 else (8, 6, 1)
    prob = inputs.random_problem(rng, ndim, n, nphase=4, mask_width=1, nsteps=1, h=7e-4)
    dt = wfft.explicit_dt(ndim, prob.h, prob.C, prob.rho)
    ref = explicit.stable_dt(medium.medium_from_problem(prob))
    assert abs(dt - ref) <= 1e-12 * ref, (dt, ref)


@pytest.mark.parametrize("ndim,n,dense_tables", [(2, (8, 6, 1), False), (3, (6, 5, 4), False), (3, (4, 5, 3), True),
                                                 (2, (7, 9, 1), True)])
def test_operator_bound_covers_the_dense_operator(lib, ndim, n, dense_tables):
    """wfft_operator_bound (host only) is an upper bound of the largest eigenvalue of the
    assembled operator of the oracle (Eq. A_oper), and not a loose one."""
    from oracle import dense, medium
    from paper_2211_08263_gb300 import inputs, wfft
    rng = np.random.default_rng(5 * ndim + sum(n))
    prob = inputs.random_problem(rng, ndim, n, nphase=4, mask_width=1, nsteps=1, dense=dense_tables,
                                 contrast=4.0, dt=4e-7)
    th = prob.beta * prob.dt ** 2
    A = dense.dense_operator(medium.medium_from_problem(prob), th)
    lam = np.linalg.eigvalsh(A.toarray() if hasattr(A, "toarray") else A).max()
    bound = wfft.operator_bound(ndim, prob.n, prob.h, prob.C, prob.rho, th)
    assert lam <= bound * (1 + 1e-12), (lam, bound)
    assert bound <= 4.0 * lam, (lam, bound)


def test_operator_bound_homogeneous_isotropic_closed_form(lib):
    """Isotropic C on symmetric tensors has eigenvalues 3 lambda + 2 mu (once) and 2 mu:
    the bound is rho + theta (3 lambda + 2 mu) |xi|_max^2 with the largest discrete
    frequency 2 pi floor((N-1)/2) / L per axis."""
    from paper_2211_08263_gb300 import inputs, wfft
    E, nu, rho = 200e9, 0.3, 7800.0
    lam_, mu = E * nu / ((1 + nu) * (1 - 2 * nu)), E / (2 * (1 + nu))
    Cv = inputs.voigt21_from_matrix(inputs.isotropic_voigt(E, nu))[None]
    n, h, th = (16, 9, 8), (1e-3, 2e-3, 1.5e-3), 1e-14
    xi2 = sum((2 * np.pi / (n[i] * h[i]) * ((n[i] - 1) // 2)) ** 2 for i in range(3))
    expect = rho + th * (3 * lam_ + 2 * mu) * xi2
    got = wfft.operator_bound(3, n, h, Cv, np.array([rho]), th)
    assert abs(got - expect) <= 1e-12 * expect, (got, expect)


@pytest.mark.parametrize("n,cnt,prime", [
    (256, [2, 1, 0, 0, 0, 0, 0], 0),    # 8 8 4
    (129, [0, 0, 0, 1, 0, 0, 0], 43),   # 3 x 43: the paper's spherical-wave grid
    (1025, [0, 0, 0, 0, 2, 0, 0], 41),  # 5^2 x 41: the paper's plate grid
    (176, [0, 2, 0, 0, 0, 0, 0], 11),   # 2^4 (as 4 x 4) x 11
    (127, [0, 0, 0, 0, 0, 0, 0], 127),  # the largest direct stage
    (567, [0, 0, 0, 4, 0, 1, 0], 0),    # 3^4 x 7: the paper's polycrystal bar
    (1, [0, 0, 0, 0, 0, 0, 0], 0)])
def test_axis_plan_factorizes_with_one_prime_stage(lib, n, cnt, prime):
    """wfft_axis_plan (host only): the built-in decomposition multiplies back to n, with at
    most one prime factor above 7 as the direct stage."""
    from paper_2211_08263_gb300 import wfft
    got, p = wfft.axis_plan(n)
    assert (got, p) == (cnt, prime)
    rad = [8, 4, 2, 3, 5, 7, 16]
    assert int(np.prod([r ** c for r, c in zip(rad, got)])) * max(p, 1) == n


@pytest.mark.parametrize("n", [143, 262, 11 * 11, 2049, 0, 6561])
def test_axis_plan_refuses_unsupported_lengths(lib, n):
    """Two prime factors above 7 (143 = 11 x 13, 121 = 11^2), one above 127 (262 = 2 x 131),
    and lengths outside 1..2048 (6561 = 3^8, the paper's 1-D bar) are refused."""
    from paper_2211_08263_gb300 import wfft
    with pytest.raises(wfft.WfftError) as e:
        wfft.axis_plan(n)
    assert e.value.code == wfft.EUNSUPPORTED

