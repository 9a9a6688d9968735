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


@pytest.mark.parametrize("case", ["ndim", "n2d", "dt", "rho", "spd", "nphase", "allmasked", "prime", "1d"])
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
        kw["n"] = (11, 64, 1)
        kw["phase"] = np.zeros((1, 64, 11), np.uint16)
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
