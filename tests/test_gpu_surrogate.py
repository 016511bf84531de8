"""MLP surrogate of the hills sum: the hand-written inference, gradient and
Adam kernels against the FP64 MLP oracle (oracle/mlp.py, bfloat16-rounded
weights emulated), the step path (network for hills [0, K) + exact sum over
the rest) against the oracle, and a fit on the hills of an oracle
metadynamics run whose held-out error is checked against the oracle's exact
hills sum."""
import numpy as np
import pytest

import synth
from systems import gpu_handle, oracle_system, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

NORM = np.array([0.2, -0.1, 0.3, 1.5, 0.8, 2.0, 1.7, 3.0])  # mu[3], inv_s[3], Vm, Vs


def _wt():
    import paper_2301_04835_b300 as wt
    return wt


def _theta(seed, scale=0.35):
    return synth.rng(seed).normal(scale=scale, size=4481)


def _handle(d=3, W=4, capacity=1000, sigma=0.3, **kw):
    spec = dict(engine="none", walker_sizes=[1] * W, sigma=(sigma,) * d, capacity=capacity,
                cvs=[dict(kind="component", a=[0], axis=k) for k in range(d)], **kw)
    return gpu_handle(spec, "f32"), spec


def _abs_scales(theta_b, norm, xi):
    """Tolerance scales: magnitudes of the terms that make V and dV/dxi."""
    from oracle import mlp

    W1, b1, W2, b2, w3, b3 = mlp.unpack(theta_b)
    d = xi.shape[1]
    X = np.zeros((xi.shape[0], 3))
    X[:, :d] = (xi - norm[:d]) * norm[3:3 + d]
    z1 = X @ W1.T + b1
    a1, d1 = mlp.silu(z1), mlp.silu_d1(z1)
    z2 = a1 @ W2.T + b2
    g2 = np.abs(mlp.silu_d1(z2) * w3)
    SV = abs(norm[7]) * ((np.abs(a1) @ np.abs(W2.T) + np.abs(b2)) @ np.abs(w3) + abs(b3)) + abs(norm[6])
    h1 = g2 @ np.abs(W2)
    SG = np.abs(norm[7] * norm[3:3 + d]) * ((np.abs(d1) * h1) @ np.abs(W1))[:, :d]
    return SV, SG


@pytest.mark.parametrize("d", [3, 2])
def test_mlp_eval_matches_oracle(d):
    from oracle import mlp

    m, _ = _handle(d=d)
    th = _theta(1)
    m.mlp_params(th, NORM)
    xi = synth.rng(2).normal(size=(777, d))
    V, dV = m.mlp_eval(torch.tensor(xi, device="cuda"))
    tb = mlp.bf16_round(th)
    Vr, dVr = mlp.bias(tb, NORM, xi)
    SV, SG = _abs_scales(tb, NORM, xi)
    assert np.all(np.abs(to_np(V) - Vr) <= 1e-5 * SV), np.max(np.abs(to_np(V) - Vr) / SV)
    assert np.all(np.abs(to_np(dV) - dVr) <= 1e-5 * SG + 1e-30), np.max(np.abs(to_np(dV) - dVr) / SG)


def test_mlp_params_roundtrip_and_bf16_copy():
    from oracle import mlp

    m, _ = _handle()
    th = _theta(3).astype(np.float32)
    out, nrm = m.mlp_params(th, NORM)
    assert np.array_equal(out, th) and np.array_equal(nrm, NORM)
    # a network whose only path is b3: V_nn = Vs * bf16(b3) + Vm exactly
    t = np.zeros(4481, np.float32)
    t[-1] = 0.1
    m.mlp_params(t)
    V, dV = m.mlp_eval(torch.zeros(3, 3, dtype=torch.float64, device="cuda"))
    assert np.allclose(to_np(V), NORM[7] * mlp.bf16_round(0.1) + NORM[6], rtol=1e-7)
    assert np.all(to_np(dV) == 0)


def _batch(seed, B, d=3):
    r = synth.rng(seed)
    x = np.zeros((B, 3))
    x[:, :d] = r.normal(size=(B, d))
    V = r.normal(loc=2.0, scale=3.0, size=B).astype(np.float32)
    G = np.zeros((B, 3), np.float32)
    G[:, :d] = r.normal(scale=2.0, size=(B, d))
    return x, V, G


def _oracle_targets(x, V, G, norm, d=3):
    X = np.zeros_like(x)
    X[:, :d] = (x[:, :d] - norm[:d]) * norm[3:3 + d]
    Vt = (V.astype(np.float64) - norm[6]) / norm[7]
    Gt = np.zeros_like(x)
    Gt[:, :d] = G[:, :d].astype(np.float64) / (norm[7] * norm[3:3 + d])
    return X, Vt, Gt


@pytest.mark.parametrize("d", [3, 2])
def test_sobolev_gradient_matches_oracle(d):
    """Weight gradient of the Sobolev loss, forward + double backward, over a
    ragged batch (300 samples over 4-warp blocks)."""
    from oracle import mlp

    m, _ = _handle(d=d)
    th = _theta(4)
    m.mlp_params(th, NORM)
    x, V, G = _batch(5, 300, d)
    g, L = m.mlp_grad(torch.tensor(x, device="cuda"), torch.tensor(V, device="cuda"),
                      torch.tensor(G, device="cuda"), 0.3)
    X, Vt, Gt = _oracle_targets(x, V, G, NORM, d)
    Lr, gr = mlp.loss_grad(mlp.bf16_round(th), X, Vt, Gt, 0.3)
    assert abs(float(L) - Lr) <= 1e-5 * Lr
    g = to_np(g)
    blocks = [(0, 192), (192, 256), (256, 4352), (4352, 4416), (4416, 4480), (4480, 4481)]
    for a, b in blocks:
        err = np.linalg.norm(g[a:b] - gr[a:b]) / np.linalg.norm(gr[a:b])
        assert err < 2e-4, (a, b, err)


def test_adam_steps_match_oracle():
    """Adam on the FP32 master with bfloat16 working weights, emulated in the
    oracle.  One step: each parameter moves by lr g / (|g| + eps); five
    steps: the loss sequence and the weights follow the oracle."""
    from oracle import mlp

    m, _ = _handle()
    th = _theta(6).astype(np.float32).astype(np.float64)
    x, V, G = _batch(7, 256)
    xt, Vt_, Gt_ = (torch.tensor(a, device="cuda") for a in (x, V, G))
    X, Vt, Gt = _oracle_targets(x, V, G, NORM)
    lr = 1e-3
    m.mlp_params(th, NORM)
    m.mlp_train(xt, Vt_, Gt_, 256, 1, lr, 0.1)
    t1 = m.mlp_params()[0].astype(np.float64)
    _, g = mlp.loss_grad(mlp.bf16_round(th), X, Vt, Gt, 0.1)
    ref, _, _ = mlp.adam(th, np.zeros_like(th), np.zeros_like(th), g, 1, lr)
    big = np.abs(g) > 1e-3 * np.abs(g).max()
    assert big.mean() > 0.8
    assert np.all(np.abs(t1 - ref)[big] <= 1e-6 * np.abs(th[big]) + 1e-3 * lr)
    assert np.all(np.abs(t1 - th) <= lr * (1 + 1e-5) + 1e-7)
    # five steps from the same start
    m.mlp_params(th, NORM)
    losses = []
    for _ in range(5):
        losses.append(float(m.mlp_train(xt, Vt_, Gt_, 256, 1, lr, 0.1)))
    t5 = m.mlp_params()[0].astype(np.float64)
    tt, mm, vv = th.copy(), np.zeros_like(th), np.zeros_like(th)
    ref_losses = []
    for k in range(1, 6):
        L, g = mlp.loss_grad(mlp.bf16_round(tt.astype(np.float32)), X, Vt, Gt, 0.1)
        ref_losses.append(L)
        tt, mm, vv = mlp.adam(tt, mm, vv, g, k, lr)
        tt = tt.astype(np.float32).astype(np.float64)
    assert np.allclose(losses, ref_losses, rtol=1e-4)
    close = np.abs(t5 - tt) <= 1e-2 * lr
    assert close.mean() > 0.98, close.mean()


def _oracle_bias(theta_b, norm, xi, hills, sigma, k0):
    import oracle as o
    from oracle import mlp

    Vn, dVn = mlp.bias(theta_b, norm, xi)
    Vt, dVt = o.hills_sum(xi, hills[k0:], sigma)
    return Vn + Vt, dVn + dVt


def test_step_path_network_plus_exact_tail():
    """bias_eval with the surrogate active: V = V_nn + sum over hills
    [512, H); inactive: the exact sum over all hills."""
    from oracle import mlp

    wt = _wt()
    m, spec = _handle(d=2, W=5, capacity=1000, sigma=0.3)
    hills = synth.uniform_hills(700, [-1, -1], [1, 1], seed=8, w_range=(0.05, 0.5))
    m.hills_load(hills)
    th = _theta(9)
    m.mlp_params(th, NORM)
    m.surrogate_set(512, True)
    x = np.zeros((5, 3))
    x[:, :2] = synth.rng(10).uniform(-1, 1, size=(5, 2))
    pos = wt.particles(x, torch.float32)
    F = torch.zeros_like(pos)
    V, xi, dV = m.bias_eval(pos, F)
    xi = to_np(xi)
    Vr, dVr = _oracle_bias(mlp.bf16_round(th), NORM, xi, hills, (0.3, 0.3), 512)
    SV, SG = _abs_scales(mlp.bf16_round(th), NORM, xi)
    SH = (hills[512:, 3][None, :] * np.exp(-((xi[:, None, :] - hills[None, 512:, :2]) ** 2).sum(-1) / 0.18)).sum(1)
    assert np.all(np.abs(to_np(V) - Vr) <= 1e-5 * (SV + SH))
    assert np.all(np.abs(to_np(dV) - dVr) <= 1e-5 * (SG + SH[:, None] * 20))
    assert np.allclose(to_np(F)[:, :2], -to_np(dV), rtol=1e-6, atol=1e-7)
    # inactive: exact sum over every hill
    m.surrogate_set(512, False)
    V2, xi2, dV2 = m.bias_eval(pos)
    import oracle as o

    Ve, dVe = o.hills_sum(to_np(xi2), hills, (0.3, 0.3))
    assert np.allclose(to_np(V2), Ve, rtol=1e-5)


def test_deposit_height_uses_the_surrogate_bias():
    """A step that deposits takes the well-tempered height from the hybrid
    bias V_nn + tail at the new CVs."""
    from oracle import mlp

    wt = _wt()
    spec = dict(engine="mb", walker_sizes=[1, 1], dims=2, dt=1e-4, kT=15.0, sigma=(0.3, 0.3), w0=1.0, gamma=10.0,
                stride=1, capacity=2000, cvs=[dict(kind="component", a=[0], axis=k) for k in range(2)])
    m = gpu_handle(spec, "f32")
    hills = synth.uniform_hills(600, [-1, -0.5], [1, 2], seed=11, w_range=(0.05, 0.5))
    m.hills_load(hills)
    th = _theta(12)
    m.mlp_params(th, NORM)
    m.surrogate_set(512, True)
    pos = wt.particles([[-0.558, 1.442, 0], [0.623, 0.028, 0]], torch.float32)
    vel, F = torch.zeros_like(pos), torch.zeros_like(pos)
    m.bind(pos, vel, F)
    m.step_n(1)
    h = m.hills_read()
    assert h.shape[0] == 602
    Vr, _ = _oracle_bias(mlp.bf16_round(th), NORM, h[600:, :2], hills, (0.3, 0.3), 512)
    href = 1.0 * np.exp(-Vr / (15.0 * 9.0))
    assert np.allclose(h[600:, 3], href, rtol=2e-5)


def _oracle_wtmd_hills():
    """5120 hills of a well-tempered metadynamics run of 16 walkers on the
    three-well landscape (CVs = x, y, z), by the FP64 oracle."""
    import oracle as o

    W = 16
    spec = dict(engine="wells3", walker_sizes=[1] * W, dims=3, dt=5e-3, friction=1.0, kT=1.0, seed=3,
                sigma=(1.0, 1.0, 1.0), w0=0.1, gamma=4.0, stride=5, capacity=8192,
                cvs=[dict(kind="component", a=[0], axis=k) for k in range(3)])
    centres = np.array([[-1, 0, 0], [1, 0.2, -0.3], [0.1, 1.3, 0.6]])
    x = synth.rng(1).normal(scale=0.3, size=(W, 3)) + centres[np.arange(W) % 3]
    sim = o.Sim(oracle_system(spec), x=x, v=np.zeros_like(x))
    sim.forces()
    assert sim.run(1600) == 0
    return spec, sim.hills[: sim.n_hills].copy()


def test_fit_on_oracle_metadynamics_hills():
    """Fit on the GPU (samples, exact labels, Adam, held-out check) to the
    hills of an oracle run; the held-out error the fit reports agrees with
    the error against the oracle's exact hills sum at fresh points, and the
    network part is switched on exactly when that error is within tol."""
    import oracle as o

    spec, hills = _oracle_wtmd_hills()
    assert hills.shape[0] == 5120
    m = gpu_handle(dict(spec, engine="none", capacity=8192), "f32")
    m.hills_load(hills)
    m.surrogate_config(n_samples=40000, iters=6000, batch=2048, lr=2e-3, lam=0.1)
    m.surrogate(True, tol_kT=0.3, retrain_every=0)
    st = m.surrogate_fit()
    assert st["K"] == 5120 and st["fits"] == 1
    assert st["rms_kT"] < 0.3, st
    assert st["active"] == 1.0
    # fresh points: jittered hill centres, exact V by the oracle
    r = synth.rng(21)
    pts = hills[r.integers(0, 5120, 400), :3] + r.normal(size=(400, 3))
    Vr, _ = o.hills_sum(pts, hills, (1.0, 1.0, 1.0))
    Vn, _ = m.mlp_eval(torch.tensor(pts, device="cuda"))
    e = to_np(Vn) - Vr
    e -= e.mean()
    rms = np.sqrt(np.mean(e ** 2))
    assert rms < 0.3 and abs(rms - st["rms_kT"]) <= 0.5 * st["rms_kT"] + 0.02, (rms, st)
    # an unreachable tolerance: the exact sum stays in use
    m.surrogate(True, tol_kT=1e-6, retrain_every=0)
    st2 = m.surrogate_fit()
    assert st2["active"] == 0.0
    wt = _wt()
    pos = wt.particles(pts[:4], torch.float32)
    m2 = gpu_handle(dict(spec, engine="none", capacity=8192, walker_sizes=[1] * 4), "f32")
    m2.hills_load(hills)
    m2.surrogate(True, tol_kT=1e-6, retrain_every=0)
    m2.surrogate_fit()
    V, xi, _ = m2.bias_eval(pos)
    Ve, _ = o.hills_sum(to_np(xi), hills, (1.0, 1.0, 1.0))
    assert np.allclose(to_np(V), Ve, rtol=1e-5)


def wells3_hills_gpu(wt, H=1_000_000, W=2048, sigma=0.4, w0=0.05, gamma=3.0, seed=5):
    """A long hill list from a well-tempered run of W walkers on the
    three-well landscape in CV space (x, y, z), made by the library itself
    (inputs of the GPU-only gain test)."""
    m = wt.Wtmd(precision="f32", sigma=(sigma,) * 3, w0=w0, gamma=gamma, kT=1.0, stride=10, capacity=H + W,
                seed=seed, engine="wells3", walker_sizes=[1] * W, dims=3, dt=5e-3, friction=1.0)
    for k in range(3):
        m.cv_define(wt.CV_COMPONENT, a=[0], axis=k)
    centres = np.array([[-1, 0, 0], [1, 0.2, -0.3], [0.1, 1.3, 0.6]])
    x = synth.rng(1).normal(scale=0.3, size=(W, 3)) + centres[np.arange(W) % 3]
    pos, vel = wt.particles(x, torch.float32), wt.particles(np.zeros_like(x), torch.float32)
    F = torch.zeros_like(pos)
    m.bind(pos, vel, F)
    m.step_n((H // W) * 10)
    return m


def test_gain_at_1e6_hills():
    """What the trained network gains: at ~1e6 hills the fitted network is
    within 0.05 kT (held out) and evaluates bias and gradient at 4096 points
    many times faster than the exact hills sum; the step path with the
    surrogate active gives the same bias as the exact path to that
    tolerance."""
    wt = _wt()
    m = wells3_hills_gpu(wt)
    K = m.counters()[1]
    assert K > 990000
    m.surrogate(True, tol_kT=0.05, retrain_every=0)
    st = m.surrogate_fit()
    assert st["active"] == 1.0 and st["rms_kT"] <= 0.05, st
    h = m.hills_read()
    r = synth.rng(3)
    P = 4096
    pts = h[r.integers(0, h.shape[0], P), :3] + 0.4 * r.normal(size=(P, 3))
    x64 = torch.tensor(pts, device="cuda")
    x32 = x64.float()
    Ve = torch.empty(P, dtype=torch.float32, device="cuda")
    dVe = torch.empty(P, 3, dtype=torch.float32, device="cuda")

    def timed(fn, reps=10):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    t_exact = timed(lambda: m.hills_eval_into(x32, Ve, dVe))
    t_nn = timed(lambda: m.mlp_eval(x64))
    Vn, dVn = m.mlp_eval(x64)
    e = to_np(Vn) - to_np(Ve)
    e -= e.mean()
    assert np.sqrt(np.mean(e ** 2)) <= 0.05  # fresh points, exact GPU sum as reference
    assert t_exact / t_nn > 10.0, (t_exact, t_nn)
    # step path: bias of the 2048 walkers, surrogate vs exact
    pos = m._bound[0]
    V1, xi1, _ = m.bias_eval(pos)
    m.surrogate(False)
    V0, xi0, _ = m.bias_eval(pos)
    d = to_np(V1) - to_np(V0)
    d -= d.mean()
    assert np.sqrt(np.mean(d ** 2)) <= 0.1


def test_refits_are_scheduled_inside_step_n():
    """With retrain_every = 512 the network is refitted inside step_n each
    time 512 more hills exist (64 walkers deposit every step), continuing
    from the current weights, and the step counters stay consistent."""
    wt = _wt()
    W = 64
    spec = dict(engine="wells3", walker_sizes=[1] * W, dims=3, dt=5e-3, kT=1.0, sigma=(0.5, 0.5, 0.5), w0=0.05,
                gamma=3.0, stride=1, capacity=8192, cvs=[dict(kind="component", a=[0], axis=k) for k in range(3)])
    m = gpu_handle(spec, "f32")
    x = synth.rng(2).normal(scale=0.5, size=(W, 3))
    pos, vel = wt.particles(x, torch.float32), wt.particles(np.zeros_like(x), torch.float32)
    F = torch.zeros_like(pos)
    m.bind(pos, vel, F)
    m.surrogate_config(n_samples=4000, iters=300, batch=512, lr=3e-3, lam=0.1)
    m.surrogate(True, tol_kT=10.0, retrain_every=512)
    m.step_n(40)  # 2560 hills: fits at 512 (first chance), 1024, 1536, 2048, 2560
    st = m.surrogate_status()
    assert m.counters() == (40, 2560)
    assert st["fits"] >= 4 and st["K"] % 256 == 0 and st["K"] >= 2048, st
    assert st["active"] == 1.0 and st["iters"] == 300 * st["fits"]
    # the bias the step path uses agrees with the exact sum to the fit's error
    V1, xi, _ = m.bias_eval(pos)
    m.surrogate(False)
    V0, _, _ = m.bias_eval(pos)
    d = to_np(V1) - to_np(V0)
    d -= d.mean()
    assert np.sqrt(np.mean(d ** 2)) <= 3 * st["rms_kT"] + 0.05


def test_domain_exit_falls_back_to_the_exact_sum():
    """The network is used only inside the box of the inputs it was trained
    on.  A walker moved outside it gets, in the same evaluation, the exact sum
    over the fitted hills (plus the exact tail): its V and dV/dxi equal the
    exact path's; the network is then switched off on the device (the status
    reports it) and the exact sum serves every walker until the next fit."""
    wt = _wt()
    W = 64
    spec = dict(engine="wells3", walker_sizes=[1] * W, dims=3, dt=5e-3, kT=1.0, sigma=(0.5, 0.5, 0.5), w0=0.05,
                gamma=3.0, stride=1, capacity=8192, cvs=[dict(kind="component", a=[0], axis=k) for k in range(3)])
    m = gpu_handle(spec, "f32")
    x = synth.rng(2).normal(scale=0.5, size=(W, 3))
    pos, vel = wt.particles(x, torch.float32), wt.particles(np.zeros_like(x), torch.float32)
    F = torch.zeros_like(pos)
    m.bind(pos, vel, F)
    m.step_n(40)  # 2560 hills, no surrogate yet
    m.surrogate_config(n_samples=4000, iters=300, batch=512, lr=3e-3, lam=0.1)
    m.surrogate(True, tol_kT=10.0, retrain_every=0)
    st = m.surrogate_fit()
    assert st["active"] == 1.0
    h = m.hills_read()
    far = h[:, :3].max(0) + 2.0  # beyond every hill centre and every jittered sample
    with torch.no_grad():
        pos[0, :3] = torch.tensor(far, dtype=torch.float32, device="cuda")
    V1, xi1, dV1 = m.bias_eval(pos)
    assert m.surrogate_status()["active"] == 0.0
    V2, _, dV2 = m.bias_eval(pos)  # network off: the exact sum everywhere
    m.surrogate(False)
    V0, xi0, dV0 = m.bias_eval(pos)
    v0, v1, v2 = to_np(V0), to_np(V1), to_np(V2)
    g0, g1, g2 = to_np(dV0), to_np(dV1), to_np(dV2)
    scale = np.abs(v0).max() + 1e-30
    assert v0[0] > 0.0  # the far walker still feels the nearest hills' tails
    assert abs(v1[0] - v0[0]) <= 1e-5 * v0[0]
    assert np.abs(g1[0] - g0[0]).max() <= 1e-4 * np.abs(g0[0]).max()
    assert np.allclose(v2, v0, rtol=1e-5, atol=1e-5 * scale)
    assert np.allclose(g2, g0, rtol=1e-5, atol=1e-5 * (np.abs(g0).max() + 1e-30))
