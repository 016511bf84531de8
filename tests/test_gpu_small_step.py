"""Small FP64 analytic systems stepped by one CTA, many steps per launch
(wtmd_small_step), against the per-kernel step of the same handle and
against the FP64 oracle.

The two GPU paths run the same operations in the same order except the
hills sum, which the single CTA adds in another fixed order: with the hills
source they agree to rounding (1e-12 relative over the runs here); with the
grid or harmonic windows as the source the arithmetic is the same."""
import numpy as np
import pytest

import synth
from systems import gpu_handle, oracle_system, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _wt():
    import paper_2301_04835_b300 as wt
    return wt


MB_CVS = [dict(kind="component", a=[0], axis=0), dict(kind="component", a=[0], axis=1)]


def _mb_spec(W=3, stride=10, grid=True, **kw):
    spec = dict(engine="mb", walker_sizes=[1] * W, dims=2, dt=1e-4, friction=1.0, kT=15.0, seed=0,
                sigma=(0.05, 0.05), w0=1.0, gamma=10.0, stride=stride, capacity=1000, cvs=MB_CVS)
    if grid:
        spec["grid"] = ((64, 48), (-1.5, -0.5), (1.2, 2.2))
    spec.update(kw)
    return spec


def _mb_start(W):
    base = np.array([[-0.558, 1.442, 0.0], [0.623, 0.028, 0.0], [-0.05, 0.467, 0.0]])
    return base[np.arange(W) % 3] + 0.01 * np.arange(W)[:, None] * np.array([1.0, -1.0, 0.0])


def _run(spec, x, v, n, small, setup=None):
    wt = _wt()
    m = gpu_handle(spec, "f64")
    if setup:
        setup(m)
    assert m.small_step(small) == small
    pos, vel = wt.particles(x, torch.float64), wt.particles(v, torch.float64)
    F = torch.zeros_like(pos)
    m.bind(pos, vel, F)
    m.step_n(n)
    torch.cuda.synchronize()
    m.check()
    return m, to_np(pos)[:, :3], to_np(vel)[:, :3], to_np(F)[:, :3]


def test_small_step_form():
    """On by default for an FP64 Mueller-Brown handle with component CVs;
    not for FP32, not for the LJ engine; enable = 0 turns it off."""
    wt = _wt()
    m = gpu_handle(_mb_spec(), "f64")
    assert m.small_step() is True
    assert m.small_step(False) is False
    assert m.small_step(True) is True
    assert gpu_handle(_mb_spec(), "f32").small_step() is False
    assert gpu_handle(_mb_spec(capacity=4000), "f64").small_step() is False  # hills sum beyond one SM's share
    lj = dict(engine="lj", walker_sizes=[64], box=(6.0, 6.0, 6.0), dt=0.005, kT=1.0, sigma=(0.1,),
              cvs=[dict(kind="rg")])
    assert gpu_handle(lj, "f64").small_step() is False
    assert wt.lib().wtmd_small_step(m.h, 2, None) == wt.EINVAL


def test_small_step_matches_per_kernel_hills_and_grid():
    """2000 steps, 3 walkers, a hill every 10 steps (600 hills) with the
    FP64 grid kept: positions, velocities, forces, hills and grid of the
    single-CTA path against the per-kernel path."""
    spec = _mb_spec(W=3, stride=10)
    x = _mb_start(3)
    v = np.zeros_like(x)
    ms, Xs, Vs, Fs = _run(spec, x, v, 2000, True)
    mk, Xk, Vk, Fk = _run(spec, x, v, 2000, False)
    assert ms.counters() == mk.counters() == (2000, 600)
    # the orders of the hills sum differ by rounding (~1e-16 relative in
    # dV/dxi); the same noise drives both, so the trajectories stay together
    # up to the growth of that difference over 2000 steps
    assert np.max(np.abs(Xs - Xk)) < 1e-8
    assert np.max(np.abs(Vs - Vk)) < 1e-5
    assert np.linalg.norm(Fs - Fk) <= 1e-7 * np.linalg.norm(Fk)
    np.testing.assert_allclose(ms.hills_read(), mk.hills_read(), rtol=1e-9, atol=1e-10)
    gs, gk = ms.grid_read(), mk.grid_read()
    np.testing.assert_allclose(gs, gk, rtol=1e-9, atol=1e-10 * np.abs(gk).max())


def test_small_step_trajectory_against_oracle():
    """100 steps with deposits against the FP64 oracle (as the per-kernel
    path is held to)."""
    import oracle as o

    spec = _mb_spec(W=3, stride=10, capacity=100)
    x = _mb_start(3)
    v = np.zeros_like(x)
    sim = o.Sim(oracle_system(spec), x=x, v=v)
    sim.forces()
    assert sim.run(100) == 0
    m, X, _, _ = _run(spec, x, v, 100, True)
    assert np.max(np.abs(X - sim.x)) < 1e-10
    h = m.hills_read()
    assert h.shape[0] == sim.n_hills == 30
    np.testing.assert_allclose(h, sim.hills[:30], rtol=1e-12, atol=1e-13)
    g = m.grid_read().ravel()
    np.testing.assert_allclose(g, sim.grid, rtol=1e-12, atol=1e-12 * np.abs(sim.grid).max())


@pytest.mark.parametrize("source", ["grid", "harmonic"])
def test_small_step_grid_and_windows_match_per_kernel(source):
    """The grid-read bias (hills still deposited and added to the grid) and
    harmonic windows (16 walkers, window sums and sample count) through the
    single-CTA path against the per-kernel path."""
    wt = _wt()
    W = 16 if source == "harmonic" else 3
    spec = _mb_spec(W=W, stride=5, grid=True)
    if source == "grid":
        spec["bias_grid"] = True
    x = _mb_start(W)
    v = np.zeros_like(x)
    centres = x[:, :2] + 0.02

    def setup(m):
        if source == "harmonic":
            m.harmonic((4000.0, 4000.0), centres)

    ms, Xs, Vs, _ = _run(spec, x, v, 500, True, setup)
    mk, Xk, Vk, _ = _run(spec, x, v, 500, False, setup)
    assert ms.counters() == mk.counters()
    assert np.max(np.abs(Xs - Xk)) < 1e-12
    assert np.max(np.abs(Vs - Vk)) < 1e-9
    if source == "harmonic":
        (a, na), (b, nb) = ms.umbrella_stats(), mk.umbrella_stats()
        assert na == nb == 500 and ms.counters()[1] == 0
        np.testing.assert_allclose(a, b, rtol=1e-13, atol=1e-13)
    else:
        np.testing.assert_allclose(ms.grid_read(), mk.grid_read(), rtol=1e-12, atol=1e-13)


def test_small_step_wells3_three_cvs():
    """The three-well landscape in 3-D with three component CVs and hills."""
    W = 4
    spec = dict(engine="wells3", walker_sizes=[1] * W, dims=3, dt=5e-3, friction=1.0, kT=1.0, seed=3,
                sigma=(0.3, 0.3, 0.3), w0=0.2, gamma=6.0, stride=5, capacity=2000,
                cvs=[dict(kind="component", a=[0], axis=k) for k in range(3)])
    x = synth.uniform_points(W, [-1.0, -0.5, -0.5], [1.0, 1.0, 0.5], seed=4)
    v = np.zeros_like(x)
    ms, Xs, _, _ = _run(spec, x, v, 1000, True)
    mk, Xk, _, _ = _run(spec, x, v, 1000, False)
    assert ms.counters() == mk.counters() == (1000, 800)
    assert np.max(np.abs(Xs - Xk)) < 1e-9
    np.testing.assert_allclose(ms.hills_read(), mk.hills_read(), rtol=1e-10, atol=1e-12)


def test_small_step_runs_past_one_launch():
    """70000 steps cross the 65536-step launch boundary: the step counter,
    the hill count and the trajectory continue as one run (against two
    step_n calls that split it elsewhere)."""
    spec = _mb_spec(W=1, stride=1000, grid=False, capacity=100)
    x = _mb_start(1)
    v = np.zeros_like(x)
    ma, Xa, Va, _ = _run(spec, x, v, 70000, True)
    wt = _wt()
    mb = gpu_handle(spec, "f64")
    pos, vel = wt.particles(x, torch.float64), wt.particles(v, torch.float64)
    F = torch.zeros_like(pos)
    mb.bind(pos, vel, F)
    mb.step_n(30000)
    mb.step_n(40000)
    torch.cuda.synchronize()
    assert ma.counters() == mb.counters() == (70000, 70)
    assert np.array_equal(Xa, to_np(pos)[:, :3]) and np.array_equal(Va, to_np(vel)[:, :3])
