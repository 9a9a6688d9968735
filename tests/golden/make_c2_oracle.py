"""Writes tests/golden/c2_composite128_oracle.txt: the FP64 oracle's trajectory of the
128^3 two-phase composite (20 periodic spheres, E 400 / 70 GPa, nu 0.25 / 0.33, rho
3900 / 2700; 4-voxel x-face slab, sin^2 pulse of period 2e-5 s on u_x; dt 2e-7 s,
beta 1/4, gamma 1/2; 200 steps), solved by the oracle's masked PCG (Alg. 2 loop body,
Eq. ND_consv_lm_Newmark_ord, Eq. precond) to a relative residual of 1e-13.

Only ``oracle/`` computes; ``paper_2211_08263_gb300.inputs`` only generates the seeded
medium and load.  The full field is 6.3 M values per step, so the file keeps, at each
checkpoint step: u_n at 2048 seeded random DOFs, the 2-norm of each component, and the
mean of each component over every x-plane (N1 x 3 values), plus the iteration count,
reference norm and final relative residual of every step.  About 75 s per step on eight
x86 cores (31-32 PCG iterations); --state-dir keeps the state after every checkpoint so
that an interrupted run resumes.

    python tests/golden/make_c2_oracle.py --state-dir /tmp/c2_state
"""
import argparse
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import newmark  # noqa: E402
from paper_2211_08263_gb300 import inputs  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c2_composite128_oracle.txt")
CHECKPOINTS = (10, 25, 50, 75, 100, 150, 200)
NSAMPLES = 2048
SAMPLE_SEED = 12801
TOL = 1e-13


def sample_dofs(prob):
    """Seeded DOFs (component, z, y, x), sorted; the same recipe the test reads back."""
    rng = np.random.default_rng(SAMPLE_SEED)
    total = prob.ndim * prob.nvox
    flat = np.sort(rng.choice(total, size=NSAMPLES, replace=False))
    c, rem = np.divmod(flat, prob.nvox)
    z, rem = np.divmod(rem, prob.n[0] * prob.n[1])
    y, x = np.divmod(rem, prob.n[0])
    return np.stack([c, z, y, x], axis=1)


def summarise(u, dofs):
    """u: oracle field (3, N3, N2, N1)."""
    vals = u[dofs[:, 0], dofs[:, 1], dofs[:, 2], dofs[:, 3]]
    norms = np.sqrt(np.sum(u.reshape(3, -1) ** 2, axis=1))
    planes = u.mean(axis=(1, 2))  # (3, N1)
    return vals, norms, planes


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--state-dir", default=None)
    ap.add_argument("--nsteps", type=int, default=200)
    args = ap.parse_args()
    prob = inputs.config_c2(nsteps=args.nsteps)
    nm = newmark.oracle_from_problem(prob, tol=TOL)
    dofs = sample_dofs(prob)
    state = nm.zero_state()
    done = 0
    records = {}
    steps = []
    sd = args.state_dir
    if sd:
        os.makedirs(sd, exist_ok=True)
        ck = os.path.join(sd, "resume.npz")
        if os.path.exists(ck):
            z = np.load(ck, allow_pickle=True)
            state = newmark.State(z["u"], z["v"], z["a"])
            done = int(z["n"])
            records = z["records"].item()
            steps = [tuple(s) for s in z["steps"]]
            print(f"resumed at step {done}", flush=True)
    for n in range(done + 1, args.nsteps + 1):
        t0 = time.time()
        state, info = nm.step(state, prob.U[n - 1])
        assert info["converged"], (n, info)
        steps.append((n, info["iters"], info["ref"], info["rel_res"]))
        print(f"step {n}: {info['iters']} iterations, rel_res {info['rel_res']:.3e}, {time.time() - t0:.1f} s",
              flush=True)
        if n in CHECKPOINTS:
            records[n] = summarise(state.u, dofs)
            if sd:
                np.savez(os.path.join(sd, "resume.tmp.npz"), u=state.u, v=state.v, a=state.a, n=n,
                         records=np.array(records, dtype=object), steps=np.array(steps))
                os.replace(os.path.join(sd, "resume.tmp.npz"), os.path.join(sd, "resume.npz"))
    write(prob, dofs, records, steps)


def write(prob, dofs, records, steps):
    with open(OUT, "w") as f:
        f.write("# FP64 oracle trajectory of the 128^3 two-phase composite (inputs.config_c2, 200 steps),\n")
        f.write(f"# masked PCG to relative residual {TOL:g} (Alg. 2, Eq. ND_consv_lm_Newmark_ord, Eq. precond).\n")
        f.write("# Written by tests/golden/make_c2_oracle.py (calls only oracle/ and the seeded inputs).\n")
        f.write("# Indices: component c (0 = x), z, y, x of the [c][N3][N2][N1] field.\n")
        f.write(f"checkpoints {' '.join(str(k) for k in sorted(records))}\n")
        f.write(f"dofs {len(dofs)}\n")
        for d in dofs:
            f.write(f"{d[0]} {d[1]} {d[2]} {d[3]}\n")
        for k in sorted(records):
            vals, norms, planes = records[k]
            f.write(f"step {k}\n")
            f.write("norms " + " ".join(f"{v:.17e}" for v in norms) + "\n")
            for c in range(3):
                f.write(f"planes{c} " + " ".join(f"{v:.17e}" for v in planes[c]) + "\n")
            f.write("values " + " ".join(f"{v:.17e}" for v in vals) + "\n")
        f.write(f"iterations {len(steps)}\n")
        for n, it, ref, rr in steps:
            f.write(f"{int(n)} {int(it)} {ref:.17e} {rr:.17e}\n")


def read(path=OUT):
    """Parse the fixture: dict with dofs (K x 4), checkpoints {step: (values, norms, planes)},
    steps (n, iters, ref, rel_res)."""
    out = {"checkpoints": {}, "steps": []}
    with open(path) as f:
        lines = [ln.rstrip("\n") for ln in f if not ln.startswith("#")]
    i = 0
    i += 1  # checkpoints line
    nd = int(lines[i].split()[1])
    i += 1
    out["dofs"] = np.array([[int(v) for v in lines[i + j].split()] for j in range(nd)], dtype=np.int64)
    i += nd
    while lines[i].startswith("step "):
        k = int(lines[i].split()[1])
        norms = np.array([float(v) for v in lines[i + 1].split()[1:]])
        planes = np.array([[float(v) for v in lines[i + 2 + c].split()[1:]] for c in range(3)])
        vals = np.array([float(v) for v in lines[i + 5].split()[1:]])
        out["checkpoints"][k] = (vals, norms, planes)
        i += 6
    ns = int(lines[i].split()[1])
    for j in range(ns):
        p = lines[i + 1 + j].split()
        out["steps"].append((int(p[0]), int(p[1]), float(p[2]), float(p[3])))
    return out


if __name__ == "__main__":
    main()
