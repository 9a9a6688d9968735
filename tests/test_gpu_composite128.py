"""The 128^3 two-phase composite (20 periodic spheres of 400 GPa in a 70 GPa matrix, 4-voxel
x-face slab, sin^2 pulse, 200 steps) in FP64 and in mixed precision (FP32 inner PCG with FP64
refinement), against the FP64 oracle's trajectory of the same workload.

The oracle trajectory (masked PCG to 1e-13, Alg. 2, Eq. ND_consv_lm_Newmark_ord) takes hours
of host time, so it is stored: tests/golden/make_c2_oracle.py (which calls only the oracle)
writes, at steps 10 ... 200, u_n at 2048 seeded DOFs, each component's 2-norm over the grid
and each component's mean over every x-plane, plus every step's iteration count.  Bars
(relative L2): FP64 solved to 1e-13 <= 1e-10, mixed at tol 1e-10 <= 1e-6, on the sampled DOFs,
the norms and the plane means; the FP64-vs-mixed difference over the whole grid is printed
per checkpoint."""
import importlib.util
import os

import numpy as np
import pytest

from paper_2211_08263_gb300 import inputs
from tests.gpu_util import solver_lib, torch_cuda

pytestmark = pytest.mark.gpu

FIXTURE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "c2_composite128_oracle.txt")


def _fixture():
    spec = importlib.util.spec_from_file_location(
        "make_c2_oracle", os.path.join(os.path.dirname(FIXTURE), "make_c2_oracle.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod.read(FIXTURE)


def _summary(u, dofs):
    vals = u[dofs[:, 0], dofs[:, 1], dofs[:, 2], dofs[:, 3]]
    norms = np.sqrt(np.sum(u.reshape(3, -1) ** 2, axis=1))
    planes = u.mean(axis=(1, 2))
    return vals, norms, planes


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.skipif(not os.path.exists(FIXTURE), reason="stored oracle trajectory not generated")
def test_composite_128_fp64_and_mixed_match_the_oracle_trajectory():
    torch = torch_cuda()
    wfft = solver_lib()
    fx = _fixture()
    prob = inputs.config_c2()
    ck = sorted(fx["checkpoints"])
    runs = {}
    for name, prec, tol in (("fp64", wfft.FP64, 1e-13), ("mixed", wfft.MIXED, 1e-10)):
        s = wfft.Solver.from_problem(prob, options=wfft.default_options(precision=prec, tol=tol, maxit=1000))
        out, iters = {}, []
        u = torch.empty(s.shape, dtype=torch.float64, device="cuda")
        v, a = torch.empty_like(u), torch.empty_like(u)
        for n in range(1, prob.nsteps + 1):
            info = s.step(prob.U[n - 1])
            assert info["status"] == 0 and info["rel_res"] <= tol
            iters.append(info["iters"])
            if n in ck:
                s.get_state_dev(u, v, a)
                out[n] = u.cpu().numpy()
        s.close()
        runs[name] = (out, iters)
    rows = []
    for n in ck:
        vo, no, po = fx["checkpoints"][n]
        row = {"step": n}
        for name in runs:
            vg, ng, pg = _summary(runs[name][0][n], fx["dofs"])
            row[name] = max(_rel(vg, vo), _rel(ng, no), _rel(pg, po))
        row["mixed_vs_fp64_grid"] = _rel(runs["mixed"][0][n], runs["fp64"][0][n])
        rows.append(row)
    print()
    for r in rows:
        print(r)
    oracle_iters = [it for _, it, _, _ in fx["steps"]]
    gap = max(abs(g - o) for g, o in zip(runs["fp64"][1], oracle_iters))
    print("FP64 iterations per step, GPU vs oracle, largest gap:", gap,
          "mean GPU FP64 / mixed:", np.mean(runs["fp64"][1]), np.mean(runs["mixed"][1]))
    for r in rows:
        assert r["fp64"] <= 1e-10, r
        assert r["mixed"] <= 1e-6, r
    assert gap <= 2
