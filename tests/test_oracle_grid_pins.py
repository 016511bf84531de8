"""Pins of the oracle's grid-read bias (Sec. 2.1.5: the bias potential kept on a
pre-defined grid, trading accuracy for speed).

The reading (central-difference node gradients, multilinear interpolation,
clamped non-periodic edges, wrapped periodic axes) is checked against closed
forms it must reproduce exactly (polynomials it interpolates without error,
the central difference of a cosine across the periodic seam), against the
exact hills sum it approximates (second-order convergence as the grid is
refined), and, through the step loop, against the well-tempered recursion of a
walker frozen on a grid node.  A wrong corner weight, a swapped axis, a wrong
sign or an off-by-one node index breaks at least one of them.
"""
import numpy as np
import pytest

import oracle as o


def _nodes(bins, lo, hi):
    return o.grid_centres(bins, lo, hi)


def test_quadratic_1d_value_and_gradient_closed_forms():
    """V = x^2 on nodes: linear interpolation gives x^2 + (x - c_k)(c_{k+1} - x);
    central differences of a quadratic are exact, so dV = 2x between interior
    nodes; beyond the last node the edge value and the one-sided slope
    c_{n-1} + c_{n-2} hold."""
    bins, lo, hi = [16], [-1.0], [1.0]
    c = _nodes(bins, lo, hi)[0]
    dx = c[1] - c[0]
    rng = np.random.default_rng(0)
    x = rng.uniform(c[1], c[-2], 200)
    V, dV = o.grid_interp(c ** 2, bins, lo, hi, x[:, None])
    k = np.floor((x - c[0]) / dx).astype(int)
    np.testing.assert_allclose(V, x ** 2 + (x - c[k]) * (c[k + 1] - x), rtol=0, atol=1e-14)
    np.testing.assert_allclose(dV[:, 0], 2 * x, rtol=0, atol=1e-13)
    Ve, dVe = o.grid_interp(c ** 2, bins, lo, hi, np.array([[hi[0] + 0.3], [lo[0] - 5.0]]))
    assert Ve[0] == pytest.approx(c[-1] ** 2, abs=1e-15)
    assert dVe[0, 0] == pytest.approx(c[-1] + c[-2], abs=1e-13)
    assert Ve[1] == pytest.approx(c[0] ** 2, abs=1e-15)
    assert dVe[1, 0] == pytest.approx(c[0] + c[1], abs=1e-13)


def test_multilinear_functions_are_reproduced_exactly():
    """A function linear in each CV separately (a + b x + c y + e x y, and the
    trilinear 3-D analogue with distinct coefficients per axis) is
    interpolated without error, value and gradient, inside the node range:
    distinct coefficients catch a swapped axis or node-order error."""
    rng = np.random.default_rng(1)
    bins, lo, hi = [7, 11], [-1.0, 0.5], [2.0, 1.5]
    cx, cy = _nodes(bins, lo, hi)
    X, Y = np.meshgrid(cx, cy, indexing="ij")
    f = lambda x, y: 0.3 + 1.7 * x - 2.9 * y + 4.1 * x * y
    pts = np.stack([rng.uniform(cx[1], cx[-2], 300), rng.uniform(cy[1], cy[-2], 300)], axis=1)
    V, dV = o.grid_interp(f(X, Y), bins, lo, hi, pts)
    x, y = pts[:, 0], pts[:, 1]
    np.testing.assert_allclose(V, f(x, y), rtol=0, atol=1e-12)
    np.testing.assert_allclose(dV[:, 0], 1.7 + 4.1 * y, rtol=0, atol=1e-11)
    np.testing.assert_allclose(dV[:, 1], -2.9 + 4.1 * x, rtol=0, atol=1e-11)

    bins3, lo3, hi3 = [5, 6, 9], [0.0, -1.0, 2.0], [1.0, 1.0, 3.5]
    ax = _nodes(bins3, lo3, hi3)
    G = np.meshgrid(*ax, indexing="ij")
    g = lambda x, y, z: 1.0 + 2.0 * x - 3.0 * y + 5.0 * z + 7.0 * x * y * z - 0.5 * y * z
    pts = np.stack([rng.uniform(a[1], a[-2], 300) for a in ax], axis=1)
    V, dV = o.grid_interp(g(*G), bins3, lo3, hi3, pts)
    x, y, z = pts.T
    np.testing.assert_allclose(V, g(x, y, z), rtol=0, atol=1e-11)
    np.testing.assert_allclose(dV[:, 0], 2.0 + 7.0 * y * z, rtol=0, atol=1e-10)
    np.testing.assert_allclose(dV[:, 1], -3.0 + 7.0 * x * z - 0.5 * z, rtol=0, atol=1e-10)
    np.testing.assert_allclose(dV[:, 2], 5.0 + 7.0 * x * y - 0.5 * y, rtol=0, atol=1e-10)


def test_periodic_axis_wraps_across_the_seam():
    """V = cos(theta) on one period [-pi, pi): at a node the value is exact and
    the gradient is the central difference -sin(theta) sin(h) / h, h = dx,
    also at the first and last nodes whose neighbours lie across the seam; a
    point and its periodic image give the same result."""
    n = 24
    bins, lo, hi = [n], [-np.pi], [np.pi]
    c = _nodes(bins, lo, hi)[0]
    dx = 2 * np.pi / n
    V, dV = o.grid_interp(np.cos(c), bins, lo, hi, c[:, None], period=[2 * np.pi])
    np.testing.assert_allclose(V, np.cos(c), rtol=0, atol=1e-14)
    np.testing.assert_allclose(dV[:, 0], -np.sin(c) * np.sin(dx) / dx, rtol=0, atol=1e-13)
    x = np.array([-np.pi + 0.1 * dx, np.pi - 0.2 * dx, 2.9])
    Va, dVa = o.grid_interp(np.cos(c), bins, lo, hi, x[:, None], period=[2 * np.pi])
    Vb, dVb = o.grid_interp(np.cos(c), bins, lo, hi, (x + 2 * np.pi)[:, None], period=[2 * np.pi])
    np.testing.assert_allclose(Va, Vb, rtol=0, atol=1e-13)
    np.testing.assert_allclose(dVa, dVb, rtol=0, atol=1e-12)
    # between the last node and the first one across the seam: linear in t
    t = 0.3
    Vs, _ = o.grid_interp(np.cos(c), bins, lo, hi, np.array([[c[-1] + t * dx]]), period=[2 * np.pi])
    assert Vs[0] == pytest.approx((1 - t) * np.cos(c[-1]) + t * np.cos(c[0]), abs=1e-14)


def test_grid_bias_converges_to_the_hills_sum_at_second_order():
    """The grid holds the hills sum at its nodes (orc_grid_add); the value and
    gradient read from it approach the exact sum (orc_hills_sum) with errors
    that fall about fourfold per halving of the cell size."""
    rng = np.random.default_rng(2)
    sigma = (0.3, 0.2)
    hills = np.column_stack([rng.uniform(-1, 1, 40), rng.uniform(-1, 1, 40), np.zeros(40), rng.uniform(0.1, 1, 40)])
    lo, hi = [-2.0, -2.0], [2.0, 2.0]
    pts = np.stack([rng.uniform(-1, 1, 200), rng.uniform(-1, 1, 200)], axis=1)
    Vx, dVx = o.hills_sum(pts, hills, sigma)
    errs = []
    for n in (40, 80, 160):
        bins = [n, n]
        grid = np.zeros(n * n)
        for h in hills:
            o.grid_add(grid, bins, lo, hi, sigma, h[:2], h[3])
        V, dV = o.grid_interp(grid, bins, lo, hi, pts)
        errs.append((np.max(np.abs(V - Vx)), np.max(np.abs(dV - dVx))))
    errs = np.array(errs)
    assert errs[-1, 0] < 2e-3 * np.max(np.abs(Vx)) and errs[-1, 1] < 2e-2 * np.max(np.abs(dVx))
    ratios = errs[:-1] / errs[1:]
    assert np.all(ratios > 3.0) and np.all(ratios < 5.0), ratios


def test_grid_interp_rejects_single_cell_axes():
    with pytest.raises(ValueError):
        o.grid_interp(np.zeros(5), [1, 5], [0.0, 0.0], [1.0, 1.0], np.zeros((1, 2)))


def test_grid_sourced_step_follows_the_wt_recursion_on_a_node():
    """A walker frozen on a grid node: the grid value there is the sum of the
    heights (each Gaussian is 1 at its centre), so with the bias read from
    the grid the heights still follow V_{k+1} = V_k + w0 exp(-V_k / dT)."""
    gamma, w0, kT = 6.0, 1.0, 2.0
    dT = kT * (gamma - 1)
    s = o.System(engine=o.ENGINE_NONE, walker_n=[1], cvs=[o.CV(o.CV_COMPONENT, a=[0], axis=0)], mass=1e30,
                 kT=kT, sigma=(0.2,), w0=w0, gamma=gamma, stride=3, hill_cap=1000, dt=0.01,
                 grid_bins=(10,), grid_lo=(0.0,), grid_hi=(1.0,), bias_grid=True)
    sim = o.Sim(s, x=[[0.45, 0.0, 0.0]])
    sim.forces()
    assert sim.run(60) == 0
    assert sim.n_hills == 20
    V = 0.0
    for k in range(sim.n_hills):
        assert sim.hills[k, 3] == pytest.approx(w0 * np.exp(-V / dT), rel=1e-12)
        V += sim.hills[k, 3]
    # the last step's bias was read before its own deposit
    assert sim.V[0] == pytest.approx(V - sim.hills[sim.n_hills - 1, 3], rel=1e-12)
    assert sim.grid[4] == pytest.approx(V, rel=1e-12)
