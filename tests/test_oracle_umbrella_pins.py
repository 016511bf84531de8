"""Pins of the oracle's harmonic bias and umbrella integration (Sec. 2.1.1
harmonic biasing, Sec. 2.1.2 umbrella sampling / integration).

Closed forms of the bias and its force (with the periodic minimum image),
the exact BAOAB variance kT/k of a harmonically confined free particle in
every window, exactness of the trapezoidal integral for a linear mean force,
and recovery of the Mueller-Brown energy profile (the free energy in the
particle's own coordinates) along a path of windows.
"""
import numpy as np
import pytest

import oracle as o


def _windows_system(engine, centres, k, cvs, **kw):
    W = len(centres)
    return o.System(engine=engine, walker_n=[1] * W, cvs=cvs, umb_k=tuple(k), umb_centres=np.asarray(centres),
                    stride=0, **kw)


def test_harmonic_bias_closed_forms():
    cvs = [o.CV(o.CV_COMPONENT, a=[0], axis=0), o.CV(o.CV_COMPONENT, a=[0], axis=1)]
    s = _windows_system(o.ENGINE_NONE, [[0.3, -0.2], [1.0, 1.0]], (50.0, 20.0), cvs)
    x = np.array([[0.5, 0.1, 0.0], [0.0, 2.0, 0.0]])
    f, xi, V, dV = o.Sim(s, x=x).bias(x)
    d = x[:, :2] - np.array([[0.3, -0.2], [1.0, 1.0]])
    k = np.array([50.0, 20.0])
    np.testing.assert_allclose(V, 0.5 * (k * d * d).sum(1), rtol=1e-14)
    np.testing.assert_allclose(dV[:, :2], k * d, rtol=1e-14)
    np.testing.assert_allclose(f[:, :2], -k * d, rtol=1e-14)
    # periodic CV: a dihedral just below pi, centre just above -pi: the
    # difference is the short way round
    dih = [o.CV(o.CV_DIHEDRAL, a=[0, 1, 2, 3], period=2 * np.pi)]
    phi = np.pi - 0.05
    xd = np.array([[1, 0, 0], [0, 0, 0], [0, 0, 1], [np.cos(phi), np.sin(phi), 1.0]])
    sd = o.System(engine=o.ENGINE_NONE, walker_n=[4], cvs=dih, umb_k=(10.0,), umb_centres=[[-np.pi + 0.05]],
                  stride=0)
    _, xi, V, dV = o.Sim(sd, x=xd).bias(xd)
    assert abs(xi[0, 0]) == pytest.approx(np.pi - 0.05, abs=1e-12)
    D = xi[0, 0] - (-np.pi + 0.05)
    D -= 2 * np.pi * np.rint(D / (2 * np.pi))
    assert abs(D) < 0.2
    assert V[0] == pytest.approx(0.5 * 10.0 * D * D, rel=1e-12)
    assert dV[0, 0] == pytest.approx(10.0 * D, rel=1e-12)


def test_windows_sample_the_exact_harmonic_variance():
    """A free particle held by the bias alone: BAOAB samples the harmonic
    configurational distribution exactly at any stable dt (Leimkuhler &
    Matthews 2013): mean xi0 and variance kT/k in every window."""
    centres = [[-1.0], [0.0], [0.5], [2.0]]
    k, kT = 40.0, 1.5
    s = _windows_system(o.ENGINE_NONE, centres, (k,), [o.CV(o.CV_COMPONENT, a=[0], axis=0)], kT=kT, dt=0.05,
                        friction=2.0, seed=3)
    x = np.zeros((4, 3))
    sim = o.Sim(s, x=x)
    sim.forces()
    assert sim.run(400) == 0
    sim.xi_sum[:] = 0.0
    sim.n_samples = 0
    xs = []
    for _ in range(200):
        sim.run(100)
        xs.append(sim.x[:, 0].copy())
    xs = np.array(xs)
    se_mean = np.sqrt(kT / k / 200) * 4
    np.testing.assert_allclose(xs.mean(0), np.ravel(centres), atol=se_mean)
    np.testing.assert_allclose(xs.var(0), kT / k, rtol=0.25)
    mean, g, A = sim.umbrella()
    np.testing.assert_allclose(mean[:, 0], np.ravel(centres), atol=se_mean)
    assert sim.n_samples == 20000


def test_trapezoid_is_exact_for_a_linear_mean_force():
    """A(xi) = a xi^2 / 2 along a line: mean forces a xi_bar are linear, so
    the trapezoidal integral reproduces a (xi_bar_i^2 - xi_bar_0^2) / 2."""
    lib = o.lib()
    W, a, k = 7, 3.0, 25.0
    xb = np.linspace(-1.0, 2.0, W)
    # windows whose mean sits where -k (xi_bar - xi0) = a xi_bar
    centres = xb + a * xb / k
    mean = np.zeros((W, 3))
    cen = np.zeros((W, 3))
    mean[:, 0], cen[:, 0] = xb, centres
    g, A = np.zeros((W, 3)), np.zeros(W)
    kk = np.array([k, 0.0, 0.0])
    per = np.zeros(3)
    lib.orc_umbrella_integrate(W, 1, o._dp(mean), o._dp(cen), o._dp(kk), o._dp(per), o._dp(g), o._dp(A))
    np.testing.assert_allclose(g[:, 0], a * xb, rtol=1e-12)
    np.testing.assert_allclose(A, a * (xb ** 2 - xb[0] ** 2) / 2, atol=1e-12)


def test_umbrella_integration_recovers_the_mueller_brown_profile():
    """Windows along the segment between two Mueller-Brown minima (CVs = the
    particle's x, y, so the free energy is U_MB itself): the integrated mean
    forces reproduce U_MB(xi_bar_i) - U_MB(xi_bar_0) (a 2.4 kT barrier) within
    0.25 kT.  The lowest-order estimate equates -k (xi_bar - xi0), which is
    exactly the window average of grad U, with grad U at xi_bar: stiff
    windows (width sqrt(kT/k) = 0.02) keep that difference small."""
    a, b = np.array([0.623, 0.028]), np.array([-0.05, 0.467])
    W = 16
    centres = a[None, :] + np.linspace(0, 1, W)[:, None] * (b - a)[None, :]
    kT = 15.0
    cvs = [o.CV(o.CV_COMPONENT, a=[0], axis=0), o.CV(o.CV_COMPONENT, a=[0], axis=1)]
    s = _windows_system(o.ENGINE_MB, centres, (40000.0, 40000.0), cvs, dims=2, kT=kT, dt=2e-4, friction=5.0,
                        seed=1)
    x = np.zeros((W, 3))
    x[:, :2] = centres
    sim = o.Sim(s, x=x)
    sim.forces()
    sim.run(2000)
    sim.xi_sum[:] = 0.0
    sim.n_samples = 0
    sim.run(40000)
    mean, g, A = sim.umbrella()
    U = np.array([o.mb(*m)[0] for m in mean])
    assert (U.max() - U.min()) > 2.0 * kT
    assert np.max(np.abs(A - (U - U[0]))) < 0.25 * kT, np.abs(A - (U - U[0])).max() / kT
