"""Harmonic bias and umbrella windows (Sec. 2.1.1 harmonic biasing, Sec. 2.1.2
umbrella sampling / integration) on the GPU against the FP64 oracle, through
the C ABI: one window per walker.

Tolerances as for the hills sum: FP64 1e-12 relative; FP32 CVs carry FP32
rounding (dihedrals: 1e-5 rad asserted), which the spring constant carries
into dV/dxi, so FP32 forces are held to 1e-5 relative plus k times that CV
error through the Jacobian.
"""
import numpy as np
import pytest

import synth
from systems import gpu_handle, oracle_system, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _wt():
    import paper_2301_04835_b300 as wt
    return wt


def _f32(x):
    return np.asarray(x, dtype=np.float32).astype(np.float64)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_harmonic_windows_bias_eval_chain_dihedrals(prec):
    """64 replicas of the 22-bead chain, two periodic dihedral CVs, each replica
    a window with its own centre (some across the -pi / pi seam)."""
    import oracle as o

    wt = _wt()
    W = 64
    x = synth.chain_replicas(W, 22, seed=3)
    cvs = [dict(kind="dihedral", a=[5, 7, 9, 15], period=2 * np.pi),
           dict(kind="dihedral", a=[7, 9, 15, 17], period=2 * np.pi)]
    spec = dict(engine="chain", walker_sizes=[22] * W, sigma=(0.35, 0.35), cvs=cvs, capacity=16)
    centres = synth.uniform_points(W, [-np.pi, -np.pi], [np.pi, np.pi], seed=8)
    k = (50.0, 20.0)
    xin = _f32(x) if prec == "f32" else x
    osys = oracle_system(spec)
    osys.umb_k, osys.umb_centres = k, centres
    Fr, xir, Vr, dVr = o.Sim(osys, x=xin).bias(xin)
    m = gpu_handle(spec, prec)
    m.harmonic(k, centres)
    dt = torch.float32 if prec == "f32" else torch.float64
    pos = wt.particles(xin, dt)
    F = torch.zeros_like(pos)
    V, xi, dV = m.bias_eval(pos, F)
    torch.cuda.synchronize()
    dphi = np.mod(to_np(xi) - xir[:, :2] + np.pi, 2 * np.pi) - np.pi
    eps = 1e-12 if prec == "f64" else 1e-5
    assert np.abs(dphi).max() <= eps
    kk = np.asarray(k)
    if prec == "f64":
        np.testing.assert_allclose(to_np(V), Vr, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(to_np(dV), dVr[:, :2], rtol=1e-12, atol=1e-11)
        assert np.linalg.norm(to_np(F)[:, :3] - Fr) <= 1e-12 * np.linalg.norm(Fr)
    else:
        D = np.abs(dVr[:, :2]) / kk  # |xi - xi0| per window
        assert np.all(np.abs(to_np(V) - Vr) <= 1e-5 * Vr + (kk * D * eps).sum(1) + 1e-6)
        assert np.all(np.abs(to_np(dV) - dVr[:, :2]) <= 1e-5 * np.abs(dVr[:, :2]) + kk * eps)
        assert np.linalg.norm(to_np(F)[:, :3] - Fr) <= 1e-4 * np.linalg.norm(Fr)


def test_umbrella_windows_mueller_brown_trajectory_and_integration():
    """16 Mueller-Brown windows on the segment between two minima (FP64):
    trajectories, window means and the integrated profile against the oracle
    run, and no hills deposited."""
    import oracle as o

    wt = _wt()
    a, b = np.array([0.623, 0.028]), np.array([-0.05, 0.467])
    W = 16
    centres = a[None, :] + np.linspace(0, 1, W)[:, None] * (b - a)[None, :]
    cvs = [dict(kind="component", a=[0], axis=0), dict(kind="component", a=[0], axis=1)]
    spec = dict(engine="mb", walker_sizes=[1] * W, dims=2, dt=2e-4, friction=5.0, kT=15.0, seed=1,
                sigma=(0.05, 0.05), stride=10, capacity=64, cvs=cvs)
    k = (40000.0, 40000.0)
    x = np.zeros((W, 3))
    x[:, :2] = centres
    osys = oracle_system(spec)
    osys.umb_k, osys.umb_centres = k, centres
    sim = o.Sim(osys, x=x)
    sim.forces()
    assert sim.run(300) == 0
    m = gpu_handle(spec, "f64")
    m.harmonic(k, centres)
    pos, vel = wt.particles(x, torch.float64), wt.particles(np.zeros_like(x), torch.float64)
    F = torch.zeros_like(pos)
    m.bind(pos, vel, F)
    m.step_n(300)
    torch.cuda.synchronize()
    assert np.max(np.abs(to_np(pos)[:, :3] - sim.x)) < 1e-6
    mean, n = m.umbrella_stats()
    assert n == sim.n_samples == 300
    om, og, oA = sim.umbrella()
    np.testing.assert_allclose(mean, om, rtol=0, atol=1e-9)
    g, A = m.umbrella_integrate()
    np.testing.assert_allclose(g, og, rtol=1e-6, atol=1e-6 * np.abs(og).max())
    np.testing.assert_allclose(A, oA, rtol=0, atol=1e-6 * max(1.0, np.abs(oA).max()))
    assert m.counters()[1] == 0  # windows deposit no hills
    _, n2 = m.umbrella_stats(reset=True)
    assert m.umbrella_stats()[1] == 0 and n2 == 300


def test_harmonic_windows_are_validated():
    wt = _wt()
    m = wt.Wtmd(precision="f64", sigma=[0.1], walker_sizes=[1, 1])
    with pytest.raises(wt.WtmdError):
        m.harmonic([1.0], [[0.0], [1.0]])  # CVs not defined yet
    m.cv_define(wt.CV_COMPONENT, a=[0], axis=0)
    for k, c in (([0.0], [[0.0], [1.0]]), ([-1.0], [[0.0], [1.0]]), ([1.0], [[0.0], [np.nan]])):
        with pytest.raises(wt.WtmdError):
            m.harmonic(k, c)
    with pytest.raises(wt.WtmdError):
        m.bias_source(wt.BIAS_HARMONIC)  # no windows set
    with pytest.raises(wt.WtmdError):
        m.umbrella_integrate()  # no windows
    m.harmonic([5.0], [[0.0], [1.0]])
    with pytest.raises(wt.WtmdError):
        m.umbrella_integrate()  # no samples yet
    m.bias_source(wt.BIAS_HILLS)
    m.bias_source(wt.BIAS_HARMONIC)
