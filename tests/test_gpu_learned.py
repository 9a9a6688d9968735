"""Learned warm start: the BF16 network kernels against the FP64 reference of
oracle/conv.py (forward and gradients), the warm start inside the step (it
changes only the initial guess: results stay within the solver tolerance of
the oracle), and the training loop on trajectories of the solver itself."""
import numpy as np
import pytest

from paper_2211_08263_gb300 import inputs
from tests.gpu_util import oracle_field, rel, solver_lib, torch_cuda

pytestmark = pytest.mark.gpu


def bf16(a):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def random_blob(wfft, hidden, seed, last_scale=0.2):
    rng = np.random.default_rng(seed)
    _, params = wfft.blob_params(wfft.model_init(hidden, seed))
    W4 = last_scale * rng.standard_normal(params[3][0].shape) / np.sqrt(27 * hidden)
    params[3] = (W4.astype(np.float32), (0.1 * rng.standard_normal(16)).astype(np.float32))
    params = [(W, (0.05 * rng.standard_normal(b.shape)).astype(np.float32) if i < 3 else b)
              for i, (W, b) in enumerate(params)]
    return wfft.params_blob(hidden, params)


def oracle_params(wfft, blob):
    hidden, params = wfft.blob_params(blob)
    return hidden, [(bf16(W), b.astype(np.float64)) for W, b in params]


GRIDS = [(20, 12, 6), (5, 3, 1), (32, 16, 4), (16, 32, 8), (8, 16, 1), (24, 48, 40)]


@pytest.mark.parametrize("hidden", [16, 32])
@pytest.mark.parametrize("n", GRIDS)
def test_net_forward_matches_fp64_reference(hidden, n):
    from oracle import conv
    torch_cuda()
    wfft = solver_lib()
    rng = np.random.default_rng(11)
    V = n[0] * n[1] * n[2]
    x = bf16(rng.standard_normal((V, 16)))
    blob = random_blob(wfft, hidden, 3)
    y = wfft.net_forward(blob, n, x)
    _, P = oracle_params(wfft, blob)
    yo, _ = conv.net_forward(x.reshape(n[2], n[1], n[0], 16), P)
    yo = yo.reshape(V, 16)[:, :3]
    assert np.all(np.isfinite(y))
    assert rel(y, yo) < 2e-2, rel(y, yo)


@pytest.mark.parametrize("n", [(32, 16, 4), (8, 16, 1), (24, 48, 40), (16, 32, 35)])
def test_tcgen05_and_mma_sync_forward_kernels_agree(n):
    """Grids of whole 8 x 16 tiles run the hidden-32 network's forward convolutions on the
    tcgen05 kernel (z chunks of 32 planes, periodic wrap in every axis); the mma.sync kernel
    computes the same products in another order: both agree with each other to the BF16
    rounding of the hidden activations, and with the FP64 reference."""
    from oracle import conv
    torch_cuda()
    wfft = solver_lib()
    rng = np.random.default_rng(12)
    V = n[0] * n[1] * n[2]
    x = bf16(rng.standard_normal((V, 16)))
    blob = random_blob(wfft, 32, 4)
    prev = wfft.net_conv_kernel(0)
    try:
        y_tc = wfft.net_forward(blob, n, x)
        wfft.net_conv_kernel(1)
        y_ms = wfft.net_forward(blob, n, x)
    finally:
        wfft.net_conv_kernel(prev)
    _, P = oracle_params(wfft, blob)
    yo, _ = conv.net_forward(x.reshape(n[2], n[1], n[0], 16), P)
    yo = yo.reshape(V, 16)[:, :3]
    assert np.all(np.isfinite(y_tc))
    assert rel(y_tc, y_ms) < 1e-2, rel(y_tc, y_ms)
    assert rel(y_tc, yo) < 2e-2 and rel(y_ms, yo) < 2e-2


def bf16_pipeline_grads(conv, X, P, t16, free):
    """The reference forward / backward of oracle/conv.py composed with BF16 rounding
    at the points where the kernels store BF16: hidden activations and the
    gradients handed from layer to layer (the output and the loss stay FP32)."""
    hs, h = [X], X
    for i, (W, b) in enumerate(P):
        z = conv.conv_forward(h, W, b)
        if i < 3:
            h = bf16(np.maximum(z, 0.0))
            hs.append(h)
        else:
            y = z.astype(np.float32).astype(np.float64)
    L, d = conv.masked_mse(y, t16, free)
    g = bf16(d)
    grads = [None] * 4
    for i in range(3, -1, -1):
        dx, dW, db = conv.conv_backward(hs[i], P[i][0], g)
        grads[i] = (dW, db)
        if i > 0:
            g = bf16(dx * (hs[i] > 0))
    return L, grads


@pytest.mark.parametrize("hidden", [16, 32])
def test_net_gradients_match_fp64_reference(hidden):
    from oracle import conv
    torch_cuda()
    wfft = solver_lib()
    n = (20, 12, 6)
    V = n[0] * n[1] * n[2]
    rng = np.random.default_rng(5)
    x = bf16(rng.standard_normal((V, 16)))
    target = rng.standard_normal((V, 3)).astype(np.float32)
    mask = (rng.random(V) < 0.2).astype(np.uint8) * 7  # all three components prescribed
    mask[rng.random(V) < 0.1] |= 2
    blob = random_blob(wfft, hidden, 8, last_scale=1.0)
    loss, g = wfft.net_loss_grad(blob, n, 3, x, target, mask)
    _, P = oracle_params(wfft, blob)
    X = x.reshape(n[2], n[1], n[0], 16)
    out, cache = conv.net_forward(X, P)
    t16 = np.zeros((V, 16))
    t16[:, :3] = target
    t16 = t16.reshape(out.shape)
    free = np.zeros((V, 16), dtype=bool)
    for k in range(3):
        free[:, k] = ((mask >> k) & 1) == 0
    free = free.reshape(out.shape)
    Lo, dout = conv.masked_mse(out, t16, free)
    grads, _ = conv.net_backward(P, cache, dout)
    Lb, gb = bf16_pipeline_grads(conv, X, P, t16, free)
    assert abs(loss - Lo) <= 1e-2 * Lo
    assert abs(loss - Lb) <= 1e-4 * Lb
    for (dW, db), (dWo, dbo), (dWb, dbb) in zip(wfft.grad_params(hidden, g), grads, gb):
        # same rounding points: FP32-vs-FP64 accumulation only
        assert rel(dW, dWb) < 5e-3, rel(dW, dWb)
        assert rel(db, dbb) < 5e-3, rel(db, dbb)
        # against exact FP64 arithmetic: the BF16 rounding of activations and
        # gradients costs up to ~4% on the first layer's weight gradient
        assert rel(dW, dWo) < 6e-2, rel(dW, dWo)
        assert rel(db, dbo) < 2e-2, rel(db, dbo)


def _traj_problem(n, seed, nsteps, width=10.0, ndim=3):
    """Small polycrystal (rotated cubic nickel grains) with a Gaussian pulse on the x-face slab."""
    if ndim == 3:
        ids, Cv, rho = inputs.polycrystal((n, n, n), max(8, n ** 3 // 2000), seed)
        shape = (n, n, n)
    else:
        rng = np.random.default_rng(seed)
        return inputs.random_problem(rng, 2, (n, n, 1), nphase=4, mask_width=3, nsteps=nsteps, contrast=3.0)
    dt = 2e-7
    U = inputs._U_series(nsteps, dt, lambda t: inputs.gaussian_pulse(t, 1e-6, width * dt, 3 * width * dt))
    return inputs.Problem(f"traj{n}_{seed}", 3, shape, (1e-3,) * 3, dt, 0.25, 0.5, Cv, rho, ids,
                          inputs.slab_mask(3, shape, 4), U, tol=1e-10)


def _run(wfft, prob, precision, warm, blob=None, tol=1e-10):
    s = wfft.Solver.from_problem(prob, options=wfft.default_options(precision=precision, tol=tol, warm_start=warm))
    if blob is not None:
        s.set_model(blob)
    infos = [s.step(prob.U[k]) for k in range(prob.nsteps)]
    u = s.get_state()[0]
    s.close()
    return u, infos


def test_untrained_model_reproduces_taylor_warm_start_bitwise():
    torch_cuda()
    wfft = solver_lib()
    prob = _traj_problem(24, 4, 12)
    blob = wfft.model_init(16, 1)   # zero last layer: y = 0
    u_t, it_t = _run(wfft, prob, wfft.MIXED, wfft.WARM_TAYLOR)
    u_l, it_l = _run(wfft, prob, wfft.MIXED, wfft.WARM_LEARNED, blob)
    assert np.array_equal(u_t, u_l)
    assert [i["iters"] for i in it_t] == [i["iters"] for i in it_l]


@pytest.mark.parametrize("n", [20, 32])
@pytest.mark.parametrize("precision,bar", [(0, 1e-10), (1, 1e-6)])
def test_learned_warm_start_keeps_the_solution(precision, bar, n):
    """Any network (here a random one) only moves the initial guess: the converged
    displacements match the oracle and the plain solver within the solver bars (n = 32: the
    tcgen05 convolutions, n = 20: the mma.sync ones)."""
    from oracle import newmark
    torch_cuda()
    wfft = solver_lib()
    prob = _traj_problem(n, 6, 8)
    blob = random_blob(wfft, 32, 2, last_scale=3.0)
    tol = 1e-12 if precision == 0 else 1e-10
    u_l, infos = _run(wfft, prob, precision, wfft.WARM_LEARNED, blob, tol=tol)
    u_p, _ = _run(wfft, prob, precision, wfft.WARM_PREV, tol=tol)
    assert all(i["status"] == 0 for i in infos)
    so, _ = newmark.oracle_from_problem(prob, tol=1e-13).run(prob.U)
    assert rel(oracle_field(prob, u_l), so.u) < bar
    assert rel(u_l, u_p) < bar


def test_learned_warm_start_plane_strain():
    from oracle import newmark
    torch_cuda()
    wfft = solver_lib()
    prob = _traj_problem(24, 3, 6, ndim=2)
    blob = random_blob(wfft, 16, 4, last_scale=2.0)
    u_l, infos = _run(wfft, prob, wfft.MIXED, wfft.WARM_LEARNED, blob)
    so, _ = newmark.oracle_from_problem(prob, tol=1e-13).run(prob.U)
    assert rel(oracle_field(prob, u_l), so.u) < 1e-6


def test_set_model_rejects_malformed_blobs_and_learned_needs_a_model():
    torch_cuda()
    wfft = solver_lib()
    prob = _traj_problem(16, 1, 1)
    s = wfft.Solver.from_problem(prob, options=wfft.default_options(warm_start=wfft.WARM_LEARNED))
    with pytest.raises(wfft.WfftError):
        s.step(prob.U[0])
    blob = wfft.model_init(16, 0)
    for bad in (blob[:-4], np.concatenate([blob, np.zeros(4, np.uint8)])):
        with pytest.raises(wfft.WfftError):
            s.set_model(bad)
    broken = blob.copy()
    broken[40:44] = np.frombuffer(np.float32(np.nan).tobytes(), np.uint8)
    with pytest.raises(wfft.WfftError):
        s.set_model(broken)
    s.set_model(blob)
    assert s.step(prob.U[0])["status"] == 0
    s.close()


def test_training_on_solver_trajectories_lowers_loss_and_iterations():
    """Train on trajectories of three small polycrystals (pulse widths 6-12 steps),
    then A/B on a fourth (new seed): Krylov iterations with the learned warm start vs
    the paper's warm start u_{n-1} (and the Taylor extrapolation it builds on)."""
    torch_cuda()
    wfft = solver_lib()
    tr = wfft.Trainer(wfft.model_init(16, 7))
    for seed, width in ((21, 6.0), (22, 9.0), (23, 12.0)):
        p = _traj_problem(32, seed, 40, width)
        s = wfft.Solver.from_problem(p, options=wfft.default_options(precision=wfft.MIXED))
        infos = tr.collect(s, p.U)
        assert all(i["status"] == 0 for i in infos)
        s.close()
    assert tr.samples == 120
    first = tr.fit(1, batch=4, lr=2e-3, seed=1)
    last = tr.fit(12, batch=4, lr=2e-3, seed=2)
    assert np.isfinite(first) and last < first
    blob = tr.model()
    tr.close()
    test = _traj_problem(32, 29, 40, 8.0)
    runs = {}
    for name, warm, b in (("prev", wfft.WARM_PREV, None), ("taylor", wfft.WARM_TAYLOR, None),
                          ("learned", wfft.WARM_LEARNED, blob)):
        u, infos = _run(wfft, test, wfft.MIXED, warm, b)
        runs[name] = (u, sum(i["iters"] for i in infos))
    print({k: v[1] for k, v in runs.items()})
    assert runs["learned"][1] < runs["prev"][1]
    assert rel(runs["learned"][0], runs["prev"][0]) < 1e-6
