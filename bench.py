#!/usr/bin/env python
"""Benchmark of the implicit FFT beta-Newmark solver on the 256^3 nickel
polycrystal (500 seeded Voronoi grains, rotated cubic C11/C12/C44 =
168.4/121.4/75.4 GPa, rho = 8960, Gaussian pulse of width 50 dt on the 4-voxel
x-face slab), one GB300.

A step is one Newmark step of the whole hot path: predictor, the masked
preconditioned Krylov solve to 1e-10 (FFT operator + reference-medium
preconditioner) and the corrector.  The headline `value` is voxel *
Krylov-iterations / s of the mixed+learned solve (FP32 inner PCG, FP64 dots,
FP64 true-residual refinement, FP64 state; warm start = Taylor extrapolation
plus the BF16 network's correction, trained on the GPU beforehand -- untimed --
on 2000 step pairs of new-seed polycrystal runs at 48^3); the plain FP64
solve, the mixed solve from u_{n-1} and the mixed solve from the Taylor
extrapolation alone are measured beside it.  The mixed forms run every step of the
400-step pulse; the timed region (`--steps` K steps, CUDA events on the solver's stream,
a device synchronisation on both sides) is the window centred on the pulse's peak
(step 200), after `--warmup` untimed steps; per-window figures (onset, peak, tail) and
whole-run iterations per step are reported beside it.  Plain FP64 runs the same three
windows from states the first form kept.  Every field is >= 64 MB, so the working set
of each pass exceeds L2.

`--impl reference` times the FP64 CPU oracle (the plain NumPy/SciPy restatement of
the method that the tests check the GPU path against) on the host cores: one oracle
PCG iteration of the same 256^3 workload per step.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "s per Newmark step, voxel·Krylov-iters/s at 256³; plain FP64 vs mixed+learned"
UNIT = "voxel·Krylov-iters/s"
WORKLOAD = ("256^3 nickel polycrystal: 500 periodic Voronoi grains (seed 3), uniformly random orientations of "
            "cubic C11/C12/C44 = 168.4/121.4/75.4 GPa, rho 8960; Gaussian pulse (sigma 50 dt, centre 200 dt) on "
            "u_x of the 4-voxel x-face slab; dt 2e-7 s, h 1 mm, beta 1/4, gamma 1/2; PCG to 1e-10 relative "
            "residual")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=256, help="grid edge (the workload is 256)")
    ap.add_argument("--nsteps", type=int, default=400, help="steps of the pulse (the workload is 400)")
    ap.add_argument("--fp64-whole", action="store_true",
                    help="run every step of the pulse in FP64 too (default: its three windows only)")
    ap.add_argument("--modes", default="learned,mixed,taylor,fp64",
                    help="learned = mixed + learned warm start, taylor = mixed + Taylor warm start, "
                         "mixed = mixed from u_{n-1}, fp64 = plain FP64 from u_{n-1}")
    ap.add_argument("--hidden", type=int, default=32, help="warm-start network width (16 or 32)")
    ap.add_argument("--train-pairs", type=int, default=2000)
    ap.add_argument("--train-n", type=int, default=48)
    ap.add_argument("--epochs", type=int, default=4)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-small", action="store_true", help="skip the launch-bound C1 (64^2) measurement")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default FFT plans (no wfft_autotune)")
    ap.add_argument("--no-explicit", action="store_true", help="skip the explicit-scheme measurement")
    ap.add_argument("--no-sphere", action="store_true", help="skip the 129^3 sphere (prime-length stage) measurement")
    ap.add_argument("--no-batch", action="store_true", help="skip the 48-instance uneven batch")
    ap.add_argument("--batch-inst", type=int, default=48, help="instances of the uneven batch")
    ap.add_argument("--plan", default=None,
                    help="plan choices to apply instead of autotuning: a JSON file, or the JSON text itself")
    ap.add_argument("--save-plan", default=None, help="write the plan choices of the timed handles (JSON)")
    ap.add_argument("--inner-floor", type=float, default=None,
                    help="mixed modes: stop an inner solve at this fraction of the outer target")
    ap.add_argument("--inner-tol", type=float, default=None, help="mixed mode: FP32 inner-solve reduction")
    ap.add_argument("--nz", type=int, default=None, help="z extent of an n x n x nz slab instead of the cube")
    ap.add_argument("--ny", type=int, default=None, help="y extent (n x ny x nz) instead of the cube's")
    ap.add_argument("--xelems", type=int, default=None,
                    help="x-pass tile size (complex elements) applied after tuning / plan loading")
    ap.add_argument("--no-incr-resid", action="store_true",
                    help="mixed modes: every residual is a full FP64 application (no incremental residual)")
    return ap.parse_args()


def aggregate_over_ranks(ms, iters, world, device):
    """Whole-job figures of the replicas: the slowest rank's timed milliseconds (max over
    ranks) and the Krylov iterations all ranks ran (sum).  device: "cuda" under NCCL,
    "cpu" under gloo."""
    if world <= 1:
        return float(ms), float(iters)
    import torch
    mx = torch.tensor([float(ms)], device=device, dtype=torch.float64)
    sm = torch.tensor([float(iters)], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(mx, op=torch.distributed.ReduceOp.MAX)
    torch.distributed.all_reduce(sm, op=torch.distributed.ReduceOp.SUM)
    return float(mx.item()), float(sm.item())


def whole_job_value(V, iters, ms):
    """voxel x Krylov iterations of all ranks per second of the slowest rank."""
    return V * iters / (ms * 1e-3)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms in the background."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1])]
        mx = [num(r[2]) for r in rows if num(r[2])]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        pw = [num(r[3]) for r in rows if num(r[3])]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "power_w_max": max(pw) if pw else None}


def csrc_hash(files=None):
    """Hash of the kernel sources (all of csrc/, or the listed files of it)."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2211_08263_gb300", "csrc")
    for f in sorted(files if files else os.listdir(d)):
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def bf16_peak():
    """Dense BF16 tensor peak (TFLOP/s) for a kernel timed inside a long step: the
    sustained cuBLAS figure."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("bf16_tflops_sustained", d.get("bf16_tflops", 1700.0)), "measured (sustained)"
    return 1700.0, "fallback (sustained)"


def net_roofline(prof):
    """The warm-start convolutions (BF16 tensor-core contraction) against the BF16 peak."""
    d = prof.get(("fp32", "net_conv"))
    if not d or not d["timed"]:
        return None
    peak, src = bf16_peak()
    per = d["ms"] / d["timed"]
    ach = d["flops"] / d["timed"] / (per * 1e-3) / 1e12
    return {"kernel": "net_conv (bf16 tcgen05.mma, f32 accumulators in tensor memory)", "bound": "tensor",
            "achieved": ach, "peak": peak,
            "unit": "TFLOP/s", "frac": ach / peak, "peak_source": src, "ms_per_launch": per,
            "launches": d["timed"], "ms_total": d["ms"], "traffic": None}


def pcg_roofline(prof, V, hbm_peak, peak_kind):
    """The FP32 operator and preconditioner passes of the inner Krylov solve taken together
    (every FP32 pass kind but the network's): their algorithmic bytes over their summed
    CUDA-event time, against the measured HBM bandwidth, and per operator application
    (one x middle pass per application)."""
    kinds = {k: d for (prec, k), d in prof.items() if prec == "fp32" and not k.startswith("net") and d["timed"]}
    if not kinds:
        return None
    ms = sum(d["ms"] for d in kinds.values())
    by = sum(d["bytes"] for d in kinds.values())
    napp = kinds.get("xmid", {}).get("timed", 0)
    ach = by / (ms * 1e-3) / 1e9
    return {"kernels": "FP32 operator + preconditioner passes of the inner PCG (all kinds)", "bound": "hbm",
            "achieved": ach, "peak": hbm_peak, "unit": "GB/s", "frac": ach / hbm_peak, "peak_source": peak_kind,
            "ms_per_application": ms / napp if napp else None,
            "alg_bytes_per_voxel_application": by / napp / V if napp else None}


# FP64 FMA throughput of a GB300, measured with an FMA-chain microbenchmark
# (152 SMs x 2 FP64 FMA/clk/SM x 2 flop x ~1.97 GHz); the FP64 kernels are
# bound by it rather than by HBM.
FP64_PEAK_GFLOPS = 1195.2


MODES = {"learned": ("mixed+learned", "MIXED", "WARM_LEARNED"), "taylor": ("mixed+taylor", "MIXED", "WARM_TAYLOR"),
         "mixed": ("mixed", "MIXED", "WARM_PREV"), "fp64": ("fp64", "FP64", "WARM_PREV")}


def train_warm_start(wfft, args, stream):
    """GPU training of the warm-start network (untimed): step pairs collected from
    runs of the same kind of workload with new seeds -- polycrystals at
    train_n^3 with 6..21 grains, Gaussian pulses of widths 10..50 dt."""
    from paper_2211_08263_gb300 import inputs
    nruns = 16
    steps = max(1, -(-args.train_pairs // nruns))
    t0 = time.perf_counter()
    tr = wfft.Trainer(wfft.model_init(args.hidden, seed=0), stream=stream.cuda_stream)
    opt = wfft.default_options(precision=wfft.MIXED, tol=1e-10, maxit=500, check_every=4)
    for r in range(nruns):
        width = 10.0 + 40.0 * r / (nruns - 1)
        p = inputs.config_c3(nsteps=steps, n=args.train_n, ngrains=6 + r, seed=1000 + r, width_steps=width)
        s = wfft.Solver.from_problem(p, options=opt, stream=stream.cuda_stream)
        tr.collect(s, p.U)
        s.close()
    t1 = time.perf_counter()
    loss0 = tr.fit(1, batch=8, lr=1e-3, seed=1)
    loss = tr.fit(max(0, args.epochs - 1), batch=8, lr=1e-3, seed=2) if args.epochs > 1 else loss0
    blob = tr.model()
    info = {"hidden": args.hidden, "pairs": tr.samples, "grid": args.train_n, "runs": nruns,
            "epochs": args.epochs, "batch": 8, "lr": 1e-3, "loss_first_epoch": loss0, "loss_last_epoch": loss,
            "collect_s": round(t1 - t0, 2), "fit_s": round(time.perf_counter() - t1, 2)}
    tr.close()
    return blob, info


PROF_STEPS = 3
INNER_FLOOR = None  # None: the library default
PLAN = None         # plan choices to apply instead of tuning (--plan)
PLANS_USED = {}     # plan choices of the timed handles, per precision
NO_INCR = False     # --no-incr-resid: full FP64 residuals only
XELEMS = None       # --xelems: x-pass tile size set after tuning


def windows(nsteps, W, K):
    """Timed windows of K steps, each after W untimed warm-up steps: the pulse's onset
    (right after the first W steps), its peak (centred on the Gaussian's centre, step 200 of
    400) and its tail (the last K steps).  Steps are numbered from 1."""
    peak0 = max(W + 1, min(nsteps - K + 1, nsteps // 2 - K // 2 + 1))
    return {"onset": (W + 1, W + K), "peak": (peak0, peak0 + K - 1), "tail": (nsteps - K + 1, nsteps)}


def _events(torch):
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def run_mode(wfft, torch, prob, mode, blob, W, K, world, e2e: bool, inner_tol=None, autotune=True,
             whole=True, states=None):
    """One solver form on the pulse.  whole=True: every step of the pulse is run, each timed with
    CUDA events on the solver's stream; the headline region is the K steps of the peak window
    after its W warm-up steps, bracketed by a device synchronisation (and a barrier across
    ranks) on both sides; the per-launch profile is taken on the PROF_STEPS steps after it
    (their times are left out of the per-window figures).  States at the start of each
    window's warm-up are kept in `states` (device copies) for forms that run windows only.
    whole=False: each window runs from the kept state, W warm-up steps then K timed steps."""
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    _, prec, warm = MODES[mode]
    opt = wfft.default_options(precision=getattr(wfft, prec), tol=1e-10, maxit=500, check_every=4,
                               warm_start=getattr(wfft, warm))
    if inner_tol:
        opt.inner_tol = inner_tol
    if INNER_FLOOR is not None:
        opt.inner_floor = INNER_FLOOR
    if NO_INCR:
        opt.incr_resid = 0

    def make():
        sv = wfft.Solver.from_problem(prob, options=opt, stream=stream.cuda_stream)
        if mode == "learned":
            sv.set_model(blob)
        return sv

    s = make()
    precs = [wfft.FP64] + ([wfft.MIXED] if prec == "MIXED" else [])
    if PLAN is not None:
        for pr in precs:
            s.set_plan(pr, PLAN["fp64" if pr == wfft.FP64 else "fp32"])
        tuned = "from plan file"
    else:
        tuned = s.autotune(3) if autotune else None
    if XELEMS:
        for pr in precs:
            pl = s.get_plan(pr)
            pl["xelems"] = XELEMS
            s.set_plan(pr, pl)
    for pr in precs:
        PLANS_USED["fp64" if pr == wfft.FP64 else "fp32"] = s.get_plan(pr)
    nsteps = prob.nsteps
    wins = windows(nsteps, W, K)
    t0, t1 = wins["peak"]
    shape = s.shape
    per_ms, per_it, infos_all = {}, {}, {}
    res = {"autotune_changed": tuned}

    def timed_region(first, last):
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        l0 = s.launch_count()
        ev0, ev1 = _events(torch)
        infos = []
        ev0.record(stream)
        for n in range(first, last + 1):
            infos.append(s.step(prob.U[n - 1]))
        ev1.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        return ev0.elapsed_time(ev1), infos, s.launch_count() - l0

    def keep_state(n):
        if states is not None and n not in states:
            u = torch.empty(shape, dtype=torch.float64, device="cuda")
            v, a = torch.empty_like(u), torch.empty_like(u)
            s.get_state_dev(u, v, a)
            states[n] = (u, v, a)

    prof_steps = set(range(t1 + 1, min(nsteps, t1 + PROF_STEPS) + 1))
    if whole:
        starts = {w[0] - W - 1 for w in wins.values()}
        n = 1
        evs = {}
        while n <= nsteps:
            if n - 1 in starts:
                keep_state(n - 1)
            if n == t0 - W:
                # warm-up of the headline window, then the timed region
                for k in range(n, t0):
                    e0, e1 = _events(torch)
                    e0.record(stream)
                    infos_all[k] = s.step(prob.U[k - 1])
                    e1.record(stream)
                    evs[k] = (e0, e1)
                ms, infos, launches = timed_region(t0, t1)
                for k, inf in zip(range(t0, t1 + 1), infos):
                    infos_all[k] = inf
                    per_ms[k] = ms / K
                res.update({"ms_total": ms, "iters": sum(i["iters"] for i in infos), "launches": launches,
                            "outer_applies": sum(i["outer_applies"] for i in infos),
                            "sweeps": sum(i["sweeps"] for i in infos),
                            "rel_res_max": max(i["rel_res"] for i in infos),
                            "incr_resids": sum(i["incr_resids"] for i in infos),
                            "iters_per_step": [i["iters"] for i in infos]})
                n = t1 + 1
                # per-kernel CUDA-event times (kernel table, roofline) on the steps after the
                # timed ones: event pairs around every launch would perturb the timed region
                s.profile(True)
                for k in sorted(prof_steps):
                    infos_all[k] = s.step(prob.U[k - 1])
                res["profile"] = s.profile_read()
                s.profile(False)
                n = max(prof_steps) + 1 if prof_steps else n
                continue
            e0, e1 = _events(torch)
            e0.record(stream)
            infos_all[n] = s.step(prob.U[n - 1])
            e1.record(stream)
            evs[n] = (e0, e1)
            n += 1
        torch.cuda.synchronize()
        for k, (e0, e1) in evs.items():
            per_ms[k] = e0.elapsed_time(e1)
        for k, inf in infos_all.items():
            per_it[k] = inf["iters"]
        out_w = {}
        for name, (a, b) in wins.items():
            ks = [k for k in range(a, b + 1) if k in per_ms]
            out_w[name] = {"steps": [a, b], "ms_per_step": sum(per_ms[k] for k in ks) / len(ks) if ks else None,
                           "krylov_iters_per_step": sum(per_it[k] for k in range(a, b + 1)) / (b - a + 1)}
        ks = [k for k in per_ms if k not in prof_steps]
        res["windows"] = out_w
        res["whole_run"] = {"steps": nsteps, "ms_per_step": sum(per_ms[k] for k in ks) / len(ks),
                            "krylov_iters_per_step": sum(per_it.values()) / len(per_it),
                            "fp64_applies_per_step": sum(i["outer_applies"] for i in infos_all.values()) / nsteps,
                            "max_rel_res": max(i["rel_res"] for i in infos_all.values()),
                            "note": "every step of the pulse; the profiled steps' times left out"}
    else:
        out_w = {}
        for name, (a, b) in wins.items():
            u, v, a_ = states[a - W - 1]
            s.set_state_dev(u, v, a_, a - W - 1)
            for k in range(a - W, a):
                s.step(prob.U[k - 1])
            ms, infos, launches = timed_region(a, b)
            out_w[name] = {"steps": [a, b], "ms_per_step": ms / K,
                           "krylov_iters_per_step": sum(i["iters"] for i in infos) / K}
            if name == "peak":
                res.update({"ms_total": ms, "iters": sum(i["iters"] for i in infos), "launches": launches,
                            "outer_applies": sum(i["outer_applies"] for i in infos),
                            "sweeps": sum(i["sweeps"] for i in infos),
                            "rel_res_max": max(i["rel_res"] for i in infos),
                            "incr_resids": sum(i["incr_resids"] for i in infos),
                            "iters_per_step": [i["iters"] for i in infos]})
                s.profile(True)
                for k in range(b + 1, min(nsteps, b + PROF_STEPS) + 1):
                    s.step(prob.U[k - 1])
                res["profile"] = s.profile_read()
                s.profile(False)
        res["windows"] = out_w
    if e2e:
        # end to end through the C ABI over the headline window: U(t_n) from host memory in,
        # the displacement field u_n copied back to pinned host memory after every step
        host_u = torch.empty((2,) + tuple(s.shape), dtype=torch.float64, pin_memory=True).numpy()
        s2 = make()
        for pr in precs:
            s2.set_plan(pr, PLANS_USED["fp64" if pr == wfft.FP64 else "fp32"])
        u, v, a_ = states[t0 - W - 1]
        s2.set_state_dev(u, v, a_, t0 - W - 1)
        for n in range(t0 - W, t0):
            s2.step(prob.U[n - 1])
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        h0 = time.perf_counter()
        it2 = 0
        for n in range(t0, t1 + 1):
            it2 += s2.step(prob.U[n - 1])["iters"]
            # u_n to pinned host memory on the library's copy stream, overlapping the next
            # step's solve (the next corrector waits for the copy); one buffer per step in
            # flight, so the host reads u_n only after the wait below
            s2.download_async(host_u[(n - t0) % 2])
        s2.download_wait()
        torch.cuda.synchronize()
        h1 = time.perf_counter()
        res["e2e_s"] = h1 - h0
        res["e2e_iters"] = it2
        res["d2h_bytes"] = int(host_u[0].nbytes)
        s2.close()
    s.close()
    return res


def roofline(prof, V, hbm_peak, peak_kind):
    """Dominant kernel (largest device time in the timed region) against its roofline:
    the warm-start convolutions against the BF16 tensor peak, FP32 passes against HBM,
    FP64 passes against the FP64 FMA rate."""
    best = max(prof.items(), key=lambda kv: kv[1]["ms"])
    (prec, kind), d = best
    if kind == "net_conv":
        return net_roofline(prof)
    per = d["ms"] / max(1, d["timed"])
    if prec == "fp32":
        achieved = d["bytes"] / max(1, d["timed"]) / (per * 1e-3) / 1e9
        return {"kernel": f"{kind} ({prec})", "bound": "hbm", "achieved": achieved, "peak": hbm_peak,
                "unit": "GB/s", "frac": achieved / hbm_peak, "peak_source": peak_kind,
                "alg_bytes_per_launch": d["bytes"] / max(1, d["timed"]), "ms_per_launch": per,
                "launches": d["timed"], "traffic": None}
    achieved = d["flops"] / max(1, d["timed"]) / (per * 1e-3) / 1e9
    return {"kernel": f"{kind} ({prec})", "bound": "alu", "achieved": achieved, "peak": FP64_PEAK_GFLOPS,
            "unit": "GFLOP/s (FP64)", "frac": achieved / FP64_PEAK_GFLOPS, "peak_source": "measured FP64 FMA",
            "alg_flops_per_launch": d["flops"] / max(1, d["timed"]), "ms_per_launch": per,
            "launches": d["timed"], "traffic": None}


def kernel_table(prof, hbm_peak, total_ms):
    out = {}
    for (prec, kind), d in sorted(prof.items(), key=lambda kv: -kv[1]["ms"]):
        if not d["timed"]:
            continue
        per = d["ms"] / d["timed"]
        gbs = d["bytes"] / d["timed"] / (per * 1e-3) / 1e9 if per > 0 else 0.0
        gfl = d["flops"] / d["timed"] / (per * 1e-3) / 1e9 if per > 0 else 0.0
        out[f"{prec}:{kind}"] = {"launches": d["timed"], "ms": round(d["ms"], 3),
                                 "share": round(d["ms"] / total_ms, 4) if total_ms else None,
                                 "alg_GBps": round(gbs, 1), "frac_hbm": round(gbs / hbm_peak, 3),
                                 "alg_GFLOPs": round(gfl, 1)}
    return out


def small_grid(wfft, torch, steps=50):
    """The launch-bound end of the workloads: C1 (2-D plane strain 64 x 64, homogeneous steel,
    sin^2 strip load, FP64 to 1e-10), microseconds per Newmark step with the PCG iteration
    blocks as CUDA graphs and as plain launches."""
    from paper_2211_08263_gb300 import inputs
    prob = inputs.config_c1(nsteps=steps)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    out = {"workload": "C1: 2-D plane strain 64x64, E 200 GPa, nu 0.3, rho 7800, strip x<3 u_x = 1e-6 "
                       "sin^2(pi t / 2e-5), dt 2e-7 s, %d steps, FP64, tol 1e-10" % steps}
    for g in (1, 0):
        s = wfft.Solver.from_problem(prob, options=wfft.default_options(precision=wfft.FP64, tol=1e-10, use_graphs=g),
                                     stream=stream.cuda_stream)
        for k in range(5):
            s.step(prob.U[k])
        s.set_state()
        torch.cuda.synchronize()
        l0 = s.launch_count()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        its = sum(s.step(prob.U[k])["iters"] for k in range(steps))
        ev1.record(stream)
        torch.cuda.synchronize()
        key = "graphs" if g else "plain"
        out["us_per_step_" + key] = 1e3 * ev0.elapsed_time(ev1) / steps
        out["kernels_per_step"] = (s.launch_count() - l0) / steps
        out["krylov_iters_per_step"] = its / steps
        s.close()
    # launch floor: a CUDA graph of as many one-element kernels as a C1 step launches, replayed
    # once per step, without and with one host synchronisation per step (a step waits on the
    # device at least once, for its convergence flag)
    nk = max(1, int(round(out["kernels_per_step"])))
    try:
        x = torch.zeros(1, device="cuda")
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            for _ in range(nk):
                x.add_(1.0)
        for sync in (False, True):
            for _ in range(3):
                graph.replay()
            torch.cuda.synchronize()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            for _ in range(steps):
                graph.replay()
                if sync:
                    stream.synchronize()
            ev1.record(stream)
            torch.cuda.synchronize()
            out["launch_floor_us" + ("_sync" if sync else "")] = 1e3 * ev0.elapsed_time(ev1) / steps
        out["launch_floor_note"] = ("%d one-element kernels per step in one CUDA graph (the step's launch count), "
                                    "replayed per step; _sync adds one host synchronisation per step" % nk)
    except RuntimeError as e:  # the floor is context for the C1 figures, not part of them
        out["launch_floor_error"] = str(e).splitlines()[0]
    return out


def sphere129(wfft, torch, W=3, K=10):
    """The paper's spherical waves in a homogeneous aluminium cube (Sec. 4.1): 129^3 voxels,
    129 = 3 x 43, so every axis runs the direct 43-point DFT stage ahead of its radix-3
    stage; central u_1 bell pulse, dt 1.52e-6 s.  Milliseconds per Newmark step (CUDA events
    on the solver's stream) and Krylov iterations per step, FP64 and mixed, tol 1e-10."""
    from paper_2211_08263_gb300 import inputs
    prob = inputs.config_sphere129(nsteps=W + K)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    out = {"workload": "129^3 Al cube (E 70.3 GPa, nu 0.345, rho 2700), u_1 bell pulse within 1 cm of the "
                       "centre, dt 1.52e-6 s, tol 1e-10; axes 3 x 43 (direct 43-point DFT stage)",
           "steps": K, "warmup": W}
    for name, prec in (("fp64", wfft.FP64), ("mixed", wfft.MIXED)):
        s = wfft.Solver.from_problem(prob, options=wfft.default_options(precision=prec, tol=1e-10, maxit=400),
                                     stream=stream.cuda_stream)
        for k in range(W):
            s.step(prob.U[k])
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        its = sum(s.step(prob.U[k])["iters"] for k in range(W, W + K))
        ev1.record(stream)
        torch.cuda.synchronize()
        out[name] = {"ms_per_step": ev0.elapsed_time(ev1) / K, "krylov_iters_per_step": its / K}
        s.close()
    return out


def explicit_scheme(wfft, torch, prob, W, K):
    """The paper's explicit central-difference variant (Sec. 2.3) on the same 256^3 medium:
    one FP64 operator application per step at 0.9 of the CFL increment."""
    import numpy as np
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    dtc = wfft.explicit_dt(prob.ndim, prob.h, prob.C, prob.rho)
    dt = 0.9 * dtc
    s = wfft.Solver(prob.ndim, prob.n, prob.h, prob.C, prob.rho, prob.phase, prob.mask, dt, beta=0.0, gamma=0.5,
                    stream=stream.cuda_stream)
    t = dt * np.arange(1, W + K + 1)
    Ud = np.zeros((W + K, 3))
    w = 50 * prob.dt  # the workload's Gaussian pulse (sigma 50 dt, centre 4 sigma, amplitude 1e-6 m), differentiated
    Ud[:, 0] = -(t - 4 * w) / w ** 2 * 1e-6 * np.exp(-((t - 4 * w) ** 2) / (2 * w * w))
    for k in range(W):
        s.explicit_step(Ud[k])
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for k in range(W, W + K):
        s.explicit_step(Ud[k])
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / K
    s.close()
    return {"ms_per_step": ms, "dt": dt, "cfl_dt": dtc, "implicit_dt": prob.dt,
            "ms_per_implicit_dt_of_simulated_time": ms * prob.dt / dt,
            "note": "explicit central difference (beta 0, gamma 1/2), FP64, prescribed u_x velocity on the slab"}


def batch_leg(wfft, torch, rank, world, W, K, ninst=48, nsteps=100):
    """The batched workload of uneven grids: 48 polycrystal instances of 64^3 ... 192^3 (seeded
    sizes, 50-800 grains, the 256^3 workload's cubic nickel), Gaussian pulse of sigma 10 dt
    centred at step 40 on each x-face slab, mixed precision to 1e-10.  Instances are
    partitioned across ranks by their FFT work (no collective on the data path); each rank
    steps its instances together (wfft_batch_step: one grouped launch per pass, each
    instance with its own autotuned radix schedule and column-tile widths, grouped PCG
    blocks replayed as CUDA graphs).  Timed: K grouped steps centred on the pulse's peak,
    after the steps before them (untimed), CUDA events on the solvers' stream; value =
    voxel x Krylov iterations of all instances / slowest rank's time."""
    import numpy as np
    from paper_2211_08263_gb300 import batch, inputs
    specs = inputs.config_c4_specs(ninst)
    costs = [batch.instance_cost((sz, sz, sz)) for sz, _, _ in specs]
    mine = batch.partition(costs, world)[rank]
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    t0 = time.perf_counter()
    probs, solvers = [], []
    for i in mine:
        sz, ng, seed = specs[i]
        p = inputs.config_c4_instance(sz, ng, seed, nsteps)
        sv = wfft.Solver.from_problem(p, options=wfft.default_options(precision=wfft.MIXED, tol=1e-10, maxit=500,
                                                                      check_every=4),
                                      stream=stream.cuda_stream)
        sv.autotune(3)  # timed once per grid size and precision, then taken from the cache
        probs.append(p)
        solvers.append(sv)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    first = max(W + 1, 40 - K // 2 + 1)
    last = min(nsteps, first + K - 1)
    local = {}
    ms = 0.0
    vox_it = 0.0
    if solvers:
        Ustep = lambda k: np.stack([p.U[k - 1] for p in probs])  # noqa: E731
        for k in range(1, first):
            rc, _ = wfft.batch_step(solvers, Ustep(k))
            if rc != wfft.OK:
                raise RuntimeError(f"batched step {k} failed: {rc}")
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    if solvers:
        ev0, ev1 = _events(torch)
        recs = []
        ev0.record(stream)
        for k in range(first, last + 1):
            rc, infos = wfft.batch_step(solvers, Ustep(k))
            if rc != wfft.OK:
                raise RuntimeError(f"batched step {k} failed: {rc}")
            recs.append(infos)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        for j, i in enumerate(mine):
            its = [r[j]["iters"] for r in recs]
            V = probs[j].nvox
            vox_it += V * sum(its)
            local[i] = {"size": probs[j].n[0], "iters_per_step": sum(its) / len(its),
                        "max_rel_res": max(r[j]["rel_res"] for r in recs)}
    if world > 1:
        torch.distributed.barrier()
    ms_all, vox_all = aggregate_over_ranks(ms, vox_it, world, "cuda")
    allrec = batch.gather_records(local, world)
    for sv in solvers:
        sv.close()
    nk = last - first + 1
    sizes = sorted({r["size"] for r in allrec.values()})
    return {"workload": f"{ninst} polycrystals of {min(sizes)}^3..{max(sizes)}^3 (seeded sizes from "
                        "64, 80, 96, 128, 144, 160, 192; 50-800 grains), sigma 10 dt pulse centred at step 40, "
                        "mixed, tol 1e-10",
            "instances": len(allrec), "ranks": world, "voxels": int(sum(s ** 3 for s, _, _ in specs)),
            "timed_steps": [first, last], "ms_per_step": ms_all / nk,
            "voxel_iters_per_s": vox_all / (ms_all * 1e-3) if ms_all > 0 else None,
            "krylov_iters_per_step_mean": float(np.mean([r["iters_per_step"] for r in allrec.values()])),
            "max_rel_res": max(r["max_rel_res"] for r in allrec.values()),
            "setup_s": round(setup_s, 1), "scaling": "weak (instances partitioned by FFT work)"}


def cpu_oracle_iteration(prob, reps=1):
    """One FP64 oracle PCG iteration (operator + preconditioner + updates) on the workload."""
    import numpy as np
    from oracle import newmark, pcg
    nm = newmark.oracle_from_problem(prob, tol=1e-10)
    rng = np.random.default_rng(0)
    shape = (3,) + tuple(nm.med.shape)
    p = rng.standard_normal(shape)
    r = rng.standard_normal(shape)
    x = np.zeros(shape)
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        q = np.where(nm.mask, 0.0, nm.A(p))
        alpha = pcg.dot(r, r) / pcg.dot(p, q)
        x = x + alpha * p
        r = r - alpha * q
        z = np.where(nm.mask, 0.0, nm.M(r))
        beta = pcg.dot(r, z)
        p = z + 1e-3 * beta * p
        times.append(time.perf_counter() - t0)
    return times


def run_reference(args, prob, rank, world):
    if rank != 0:
        return 0
    V = prob.nvox
    W, K = args.warmup, args.steps
    t = cpu_oracle_iteration(prob, reps=W + K)[W:]
    total = sum(t)
    value = V * K / total
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": K, "warmup": W, "ms_per_step": 1e3 * total / K, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": [prob.n[0], prob.n[1], prob.n[2]],
                       "step": "one FP64 oracle PCG iteration (operator + preconditioner + updates)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{K} PCG iterations of the FP64 NumPy/SciPy oracle at "
                                       f"{prob.n[0]}^3, scipy.fft workers={cores}"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    global INNER_FLOOR, PLAN, NO_INCR, XELEMS
    if args.inner_floor is not None:
        INNER_FLOOR = args.inner_floor
    NO_INCR = args.no_incr_resid
    XELEMS = args.xelems
    if args.plan:
        PLAN = json.loads(args.plan) if args.plan.lstrip().startswith("{") else json.load(open(args.plan))
    rank, world, local = dist_env()
    from paper_2211_08263_gb300 import inputs
    W, K = args.warmup, args.steps
    prob = inputs.config_c3(nsteps=max(args.nsteps, 2 * (W + K + PROF_STEPS) + K), n=args.n, nz=args.nz, ny=args.ny)
    if args.impl == "reference":
        return run_reference(args, prob, rank, world)

    import torch
    torch.cuda.set_device(local)
    if world > 1:
        torch.distributed.init_process_group("nccl")
    from paper_2211_08263_gb300 import build, wfft
    if not os.path.exists(build.LIB):
        build.build()
    wfft.load()
    hbm_peak, peak_kind = load_peaks()
    V = prob.nvox
    modes = [m.strip() for m in args.modes.split(",") if m.strip()]
    for m in modes:
        if m not in MODES:
            raise SystemExit(f"unknown mode {m!r}; choose from {sorted(MODES)}")
    blob, learned = None, None
    if "learned" in modes:
        blob, learned = train_warm_start(wfft, args, torch.cuda.current_stream())
    clocks = ClockSampler(local)
    results = {}
    states = {}
    # forms whose every step is run: the mixed ones (tens of ms per step); plain FP64 runs the
    # three windows from the states the first form kept, unless --fp64-whole
    order = [m for m in modes if m != "fp64" or args.fp64_whole] + [m for m in modes if m == "fp64" and
                                                                       not args.fp64_whole]
    for m in order:
        if m == modes[0]:
            clocks.start()
        whole = m != "fp64" or args.fp64_whole
        results[m] = run_mode(wfft, torch, prob, m, blob, W, K, world, e2e=(m == modes[0] and not args.no_e2e),
                              inner_tol=args.inner_tol, autotune=not args.no_autotune, whole=whole,
                              states=states)
        if m == modes[0]:
            clk = clocks.stop()
    states.clear()
    head = results[modes[0]]
    ms, iters = aggregate_over_ranks(head["ms_total"], head["iters"], world, "cuda")
    value = whole_job_value(V, iters, ms)
    modes_out = {}
    for m in modes:
        r = results[m]
        modes_out[MODES[m][0]] = {"ms_per_step": r["ms_total"] / K, "s_per_step": r["ms_total"] / K / 1e3,
                        "voxel_iters_per_s": V * r["iters"] / (r["ms_total"] * 1e-3),
                        "krylov_iters_per_step": r["iters"] / K, "fp64_applies_per_step": r["outer_applies"] / K,
                        "incr_resids_per_step": r["incr_resids"] / K,
                        "sweeps_per_step": r["sweeps"] / K, "max_rel_res": r["rel_res_max"],
                        "autotune_changed": r["autotune_changed"],
                        "iters_per_step": r["iters_per_step"], "windows": r["windows"]}
        if "whole_run" in r:
            modes_out[MODES[m][0]]["whole_run"] = r["whole_run"]
    rl = roofline(head["profile"], V, hbm_peak, peak_kind)
    # DRAM bytes per launch from an ncu capture, used only while the kernel's source
    # files still hash to the captured version
    traffic_file = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if os.path.exists(traffic_file) and rl:
        ent = json.load(open(traffic_file)).get("kernels", {}).get(rl["kernel"])
        if ent and ent.get("sha") == csrc_hash(ent.get("files")):
            rl["traffic"] = ent["bytes_per_launch"]
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64",
                      "mixed": "f32 (inner PCG) + f64 (dots, residual refinement, state)",
                      "taylor": "f32 (inner PCG) + f64 (dots, residual refinement, state)",
                      "learned": "f32 (inner PCG) + f64 (dots, residual refinement, state) + bf16 (warm-start "
                                 "network, f32 accumulate)"}[modes[0]],
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": [prob.n[0], prob.n[1], prob.n[2]],
                       "mode": MODES[modes[0]][0],
                       "timed_steps": list(windows(prob.nsteps, W, K)["peak"]), "tol": 1e-10,
                       "fp64_ms_per_step": round(results["fp64"]["ms_total"] / K, 2) if "fp64" in results else None,
                       "l2": "inputs larger than L2 (every field >= 64 MB)",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "fp64_ms_per_step": results["fp64"]["ms_total"] / K if "fp64" in results else None,
            "fp64_value": (V * results["fp64"]["iters"] / (results["fp64"]["ms_total"] * 1e-3)
                           if "fp64" in results else None),
            "modes": modes_out, "roofline": rl,
            "kernels": kernel_table(head["profile"], hbm_peak,
                                    sum(d["ms"] for d in head["profile"].values())),
            "gpu_launches": head["launches"], "clocks": clk}
    if learned:
        line["learned"] = learned
        nr = net_roofline(results["learned"]["profile"])
        if nr:
            line["roofline_net"] = nr
    pr = pcg_roofline(head["profile"], V, hbm_peak, peak_kind)
    if pr:
        line["roofline_pcg"] = pr
    line["plans"] = PLANS_USED
    if args.save_plan and rank == 0:
        with open(args.save_plan, "w") as f:
            json.dump(PLANS_USED, f)
    if not args.no_small:
        line["small_grid"] = small_grid(wfft, torch)
    if not args.no_explicit:
        line["explicit"] = explicit_scheme(wfft, torch, prob, W, K)
    if not args.no_sphere:
        line["sphere129"] = sphere129(wfft, torch)
    if not args.no_batch:
        line["batch"] = batch_leg(wfft, torch, rank, world, W, K, ninst=args.batch_inst)
    if "e2e_s" in head:
        line["e2e"] = {"value": V * head["e2e_iters"] * world / head["e2e_s"], "unit": UNIT,
                       "h2d_bytes_per_step": 24, "d2h_bytes_per_step": head["d2h_bytes"],
                       "note": "wfft_step with host U(t_n) + u_n copied to pinned host memory every step (wfft_download_async, overlapping the next step; timed to the last copy landing)"}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        t = cpu_oracle_iteration(prob, reps=1)
        line["cpu_baseline"] = {"value": V / t[0], "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                                "sample": f"1 PCG iteration of the FP64 oracle at {prob.n[0]}^3 "
                                          f"({t[0]:.1f} s, scipy.fft workers={os.cpu_count()})"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
