"""GPU grid-read bias (Sec. 2.1.5: the bias kept on a pre-defined grid) against
the FP64 oracle, through the C ABI.

The oracle builds its own grid from the same hills (orc_grid_add) and reads
the bias from it (orc_grid_interp); the GPU builds its grid on the device
(wtmd_hills_load rebuilds it) and reads it with wtmd_grid_eval, or inside
bias_eval / step_n after wtmd_bias_source(WTMD_BIAS_GRID).

Tolerances: the read is a weighted sum of grid values with weights in
[0, 1] that sum to 1, so its FP64 rounding error is a few ulps of the
largest grid value G = max|grid|, and that of the gradient a few ulps of
G / dx.  FP64 handles: 1e-12 of those scales.  FP32 handles compute in FP64
and round once on the store: 1e-5 relative (V) and 1e-5 of the gradient
scale.  Trajectories (FP64): 1e-6 over the run, as for the hills sum.
"""
import numpy as np
import pytest

import synth
from systems import gpu_handle, lj_fluid_spec, oracle_system, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _wt():
    import paper_2301_04835_b300 as wt
    return wt


def _f32(x):
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def _oracle_grid(hills, bins, lo, hi, sigma, per):
    import oracle as o

    g = np.zeros(int(np.prod(bins)))
    for h in hills:
        o.grid_add(g, bins, lo, hi, sigma, h[: len(bins)], h[3], per)
    return g


GRID_CASES = [(1, False), (2, False), (2, True), (3, False), (3, True)]


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("d,periodic", GRID_CASES)
def test_grid_eval_matches_oracle(prec, d, periodic):
    """Points inside the grid, beyond its edges (clamped or wrapped), on the
    nodes themselves and across the periodic seam; uneven bin counts."""
    wt = _wt()
    import oracle as o

    sigma = [0.35, 0.3, 0.5][:d] if periodic else [0.05, 0.1, 0.07][:d]
    lo, hi = ([-np.pi] * d, [np.pi] * d) if periodic else ([-1.0, 0.5, 2.0][:d], [1.5, 2.0, 3.0][:d])
    per = [2 * np.pi] * d if periodic else [0.0] * d
    bins = [37, 29, 23][:d]
    H = 300
    hills = synth.uniform_hills(H, lo, hi, seed=17 * d + periodic)
    span = np.asarray(hi) - np.asarray(lo)
    pts = synth.uniform_points(700, list(np.asarray(lo) - 0.2 * span), list(np.asarray(hi) + 0.2 * span),
                               seed=5 * d + periodic)
    nodes = np.stack([c[:: max(1, len(c) // 7)][:7] for c in o.grid_centres(bins, lo, hi)], axis=1)
    seam = np.tile(np.asarray(hi) - 1e-3 * span, (1, 1))
    pts = np.concatenate([pts, nodes, seam])
    m = wt.Wtmd(precision=prec, sigma=sigma, capacity=H + 3, walker_sizes=[1], grid=(bins, lo, hi))
    for i in range(d):
        m.cv_define(wt.CV_COMPONENT, a=[0], axis=i, period=per[i])
    m.hills_load(hills)
    g_ref = _oracle_grid(hills, bins, lo, hi, sigma, per)
    g_gpu = m.grid_read().ravel()
    G = np.abs(g_ref).max()
    assert np.all(np.abs(g_gpu - g_ref) <= 1e-12 * G)
    dt = torch.float32 if prec == "f32" else torch.float64
    V, dV = m.grid_eval(torch.tensor(pts, dtype=dt, device="cuda"))
    torch.cuda.synchronize()
    xr = _f32(pts) if prec == "f32" else pts
    Vr, dVr = o.grid_interp(g_ref, bins, lo, hi, xr, per)
    Vg, dVg = to_np(V), to_np(dV)
    dxm = np.min(span / np.asarray(bins))
    if prec == "f64":
        assert np.all(np.abs(Vg - Vr) <= 1e-12 * G)
        assert np.all(np.abs(dVg - dVr) <= 1e-12 * G / dxm)
    else:
        assert np.all(np.abs(Vg - Vr) <= 1e-5 * np.abs(Vr) + 1e-12 * G)
        assert np.all(np.abs(dVg - dVr) <= 1e-5 * np.abs(dVr) + 1e-9 * G / dxm)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_bias_eval_from_grid_lj(prec):
    """bias_eval with the grid as the bias source on a 500-atom LJ fluid with
    the coordination and Rg CVs: CVs, V, dV/dxi and the scattered force
    against the oracle's grid-read bias."""
    wt = _wt()
    import oracle as o

    spec, x, L = lj_fluid_spec(n=500, n_tag=37, n_rg=20, seed=4, jitter=0.1)
    xin = _f32(x) if prec == "f32" else x
    sim0 = o.Sim(oracle_system(spec), x=xin)
    _, xi0, _, _ = sim0.bias(xin, hills=np.zeros((0, 4)))
    sig = np.asarray(spec["sigma"])
    hills = synth.walk_hills(301, xi0[0, :2] - 3 * sig, xi0[0, :2] + 3 * sig, 0.5 * sig, seed=3)
    lo, hi = list(xi0[0, :2] - 5 * sig), list(xi0[0, :2] + 5 * sig)
    spec.update(grid=((61, 47), lo, hi), bias_grid=True)
    sim = o.Sim(oracle_system(spec), x=xin, hills=hills)
    g_ref = _oracle_grid(hills, [61, 47], lo, hi, spec["sigma"], [0.0, 0.0])
    Fr, xir, Vr, dVr = sim.bias_grid(xin, grid=g_ref)
    m = gpu_handle(spec, prec)
    m.hills_load(hills)
    dt = torch.float32 if prec == "f32" else torch.float64
    pos = wt.particles(xin, dt)
    F = torch.zeros_like(pos)
    V, xi, dV = m.bias_eval(pos, F)
    torch.cuda.synchronize()
    tol = 1e-12 if prec == "f64" else 1e-5
    xig = to_np(xi)
    assert np.allclose(xig, xir[:, :2], rtol=1e-12 if prec == "f64" else 1e-6, atol=0)
    Fg = to_np(F)[:, :3]
    if prec == "f64":
        assert np.allclose(to_np(V), Vr, rtol=tol, atol=0)
        assert np.allclose(to_np(dV), dVr[:, :2], rtol=tol, atol=tol * np.abs(dVr).max())
        assert np.linalg.norm(Fg - Fr) <= tol * np.linalg.norm(Fr)
    else:
        # FP32 handles: the CVs carry FP32 rounding (within 1e-6 relative,
        # asserted above), which the bias curvature (sigma = 0.05) amplifies.  The
        # bound is 1e-5 relative plus that CV error propagated through the grid
        # read: dxi_j = 1e-6 |xi_j|, |dV| <= sum_j |d2V/dxi_i dxi_j| dxi_j, with the
        # Hessian by central differences of the oracle's read.
        bins, dxi = [61, 47], 1e-6 * np.abs(xir[0, :2])
        Hs = np.zeros((2, 2))
        for j in range(2):
            e = np.zeros((1, 2))
            e[0, j] = 1e-4 * spec["sigma"][j]
            Hs[:, j] = (o.grid_interp(g_ref, bins, lo, hi, xir[:, :2] + e)[1][0]
                        - o.grid_interp(g_ref, bins, lo, hi, xir[:, :2] - e)[1][0]) / (2 * e[0, j])
        tV = tol * abs(Vr[0]) + np.abs(dVr[0, :2]) @ dxi
        tdV = tol * np.abs(dVr[0, :2]) + np.abs(Hs) @ dxi
        assert abs(to_np(V)[0] - Vr[0]) <= tV
        assert np.all(np.abs(to_np(dV)[0] - dVr[0, :2]) <= tdV)
        Js = [o.cv_eval(cv, xin, list(spec["box"]))[1] for cv in sim.sys.cvs]
        tF = tol * np.linalg.norm(Fr) + sum(tdV[c] * np.linalg.norm(Js[c]) for c in range(2))
        assert np.linalg.norm(Fg - Fr) <= tF


def test_trajectory_mueller_brown_grid_bias_fp64():
    """Mueller-Brown walkers (kT = 15, dt = 1e-4) whose bias, and whose hill
    heights, come from the grid; 300 steps with a hill every 10: positions,
    hills and grid against the oracle's grid-sourced run."""
    wt = _wt()
    import oracle as o

    spec = dict(engine="mb", walker_sizes=[1, 1, 1], dims=2, dt=1e-4, friction=1.0, kT=15.0, seed=0,
                sigma=(0.05, 0.05), w0=1.0, gamma=10.0, stride=10, capacity=200,
                grid=((108, 96), (-1.5, -0.5), (1.2, 2.2)), bias_grid=True,
                cvs=[dict(kind="component", a=[0], axis=0), dict(kind="component", a=[0], axis=1)])
    x = np.array([[-0.558, 1.442, 0], [0.623, 0.028, 0], [-0.05, 0.467, 0]])
    v = np.zeros_like(x)
    sim = o.Sim(oracle_system(spec), x=x, v=v)
    sim.forces()
    assert sim.run(300) == 0
    m = gpu_handle(spec, "f64")
    pos, vel = wt.particles(x, torch.float64), wt.particles(v, torch.float64)
    F = torch.zeros_like(pos)
    m.bind(pos, vel, F)
    m.step_n(300)
    torch.cuda.synchronize()
    X = to_np(pos)[:, :3]
    assert np.max(np.abs(X - sim.x)) < 1e-6
    h = m.hills_read()
    assert h.shape[0] == sim.n_hills == 90
    assert np.allclose(h, sim.hills[:90], rtol=1e-10, atol=1e-12)
    g = m.grid_read().ravel()
    assert np.allclose(g, sim.grid, rtol=1e-10, atol=1e-12 * np.abs(sim.grid).max())
    assert np.all(h[:, 3] > 0) and np.all(h[:, 3] <= 1.0)


def test_grid_bias_source_is_validated():
    wt = _wt()
    m = wt.Wtmd(precision="f64", sigma=[0.1, 0.1], walker_sizes=[1])
    m.cv_define(wt.CV_COMPONENT, a=[0], axis=0)
    m.cv_define(wt.CV_COMPONENT, a=[0], axis=1)
    with pytest.raises(wt.WtmdError):
        m.bias_source(wt.BIAS_GRID)  # no grid
    with pytest.raises(wt.WtmdError):
        m.grid_eval(torch.zeros(3, 2, dtype=torch.float64, device="cuda"))
    with pytest.raises(wt.WtmdError):
        m.bias_source(7)
    m.bias_source(wt.BIAS_HILLS)
    one = wt.Wtmd(precision="f64", sigma=[0.1, 0.1], walker_sizes=[1], grid=((1, 8), (0.0, 0.0), (1.0, 1.0)))
    one.cv_define(wt.CV_COMPONENT, a=[0], axis=0)
    one.cv_define(wt.CV_COMPONENT, a=[0], axis=1)
    with pytest.raises(wt.WtmdError):
        one.bias_source(wt.BIAS_GRID)  # an axis of one cell
    dih = wt.Wtmd(precision="f64", sigma=[0.3], walker_sizes=[4], grid=((32,), (-np.pi,), (3.0,)))
    dih.cv_define(wt.CV_DIHEDRAL, a=[0, 1, 2, 3], period=2 * np.pi)
    with pytest.raises(wt.WtmdError):
        dih.bias_source(wt.BIAS_GRID)  # periodic CV, grid not one period
    # an empty point set is a no-op
    ok = wt.Wtmd(precision="f32", sigma=[0.1], walker_sizes=[1], grid=((8,), (0.0,), (1.0,)))
    ok.cv_define(wt.CV_COMPONENT, a=[0], axis=0)
    V, dV = ok.grid_eval(torch.zeros(0, 1, dtype=torch.float32, device="cuda"))
    assert V.numel() == 0 and dV.numel() == 0


def test_trajectory_chain_dihedrals_periodic_grid_bias_fp64():
    """16 chain replicas with two periodic dihedral CVs, the bias and the hill
    heights read from a periodic 48x40 grid over [-pi, pi)^2 (FP64): 200 steps
    with a hill every 10 per walker, positions, hills and grid against the
    oracle's grid-sourced run."""
    wt = _wt()
    import oracle as o

    W = 16
    x = synth.chain_replicas(W, 22, seed=6)
    spec = dict(engine="chain", walker_sizes=[22] * W, dt=1e-3, friction=1.0, kT=1.0, seed=2,
                sigma=(0.35, 0.35), w0=0.5, gamma=6.0, stride=10, capacity=512,
                grid=((48, 40), (-np.pi, -np.pi), (np.pi, np.pi)), bias_grid=True,
                cvs=[dict(kind="dihedral", a=[5, 7, 9, 15], period=2 * np.pi),
                     dict(kind="dihedral", a=[7, 9, 15, 17], period=2 * np.pi)])
    v = np.zeros_like(x)
    sim = o.Sim(oracle_system(spec), x=x, v=v)
    sim.forces()
    assert sim.run(200) == 0
    m = gpu_handle(spec, "f64")
    pos, vel = wt.particles(x, torch.float64), wt.particles(v, torch.float64)
    m.bind(pos, vel, torch.zeros_like(pos))
    m.step_n(200)
    torch.cuda.synchronize()
    assert np.max(np.abs(to_np(pos)[:, :3] - sim.x)) < 1e-6
    h = m.hills_read()
    assert h.shape[0] == sim.n_hills == 20 * W
    dh = h - sim.hills[: 20 * W]
    dh[:, :2] = np.mod(dh[:, :2] + np.pi, 2 * np.pi) - np.pi  # centres compared modulo the period
    assert np.abs(dh).max() < 1e-9
    g = m.grid_read().ravel()
    assert np.allclose(g, sim.grid, rtol=1e-9, atol=1e-12 * np.abs(sim.grid).max())
