"""Pins of the FP64 oracle against facts fixed outside it.

Each test checks the oracle against something other than itself: published
known-answer vectors, literature values, closed forms, finite differences,
invariances, or a physical limit the method must reach.  A plausible slip in
the oracle (a dropped term, a sign, an index, a transposed operand) breaks at
least one of them.
"""
import os

import numpy as np
import pytest

import oracle as o
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# Random numbers
# --------------------------------------------------------------------------
def test_philox_known_answers():
    """Philox4x32-10 against the published known-answer vectors (SC'11)."""
    rows = [l.split() for l in open(os.path.join(GOLD, "philox4x32_10_kat.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) == 3
    for r in rows:
        w = [int(v, 16) for v in r]
        out = o.philox4x32_10(w[0:4], w[4:6])
        assert list(out) == w[6:10]


def test_noise_moments_and_independence():
    """Box-Muller normals: mean 0, variance 1, uncorrelated across particles
    and steps; different seeds give different streams."""
    g = np.array([o.noise3(7, t, p) for t in range(200) for p in range(50)])
    assert abs(g.mean()) < 0.03
    assert abs(g.var() - 1.0) < 0.04
    assert abs(np.corrcoef(g[:, 0], g[:, 1])[0, 1]) < 0.05
    assert not np.allclose(o.noise3(1, 0, 0), o.noise3(2, 0, 0))
    assert not np.allclose(o.noise3(1, 0, 0), o.noise3(1, 1, 0))
    assert not np.allclose(o.noise3(1, 0, 0), o.noise3(1, 0, 1))
    assert not np.allclose(o.noise3(1, 0, 0), o.noise3(1, 1 << 32, 0))


# --------------------------------------------------------------------------
# Engines
# --------------------------------------------------------------------------
def test_mueller_brown_minima_match_literature():
    from scipy.optimize import minimize

    rows = [list(map(float, l.split())) for l in open(os.path.join(GOLD, "mueller_brown_minima.txt"))
            if l.strip() and l[0] != "#"]
    for x, y, U in rows:
        r = minimize(lambda p: o.mb(p[0], p[1])[0], [x + 0.02, y - 0.02], jac=lambda p: -o.mb(p[0], p[1])[1],
                     tol=1e-12, method="BFGS")
        assert abs(r.x[0] - x) < 1.5e-3 and abs(r.x[1] - y) < 1.5e-3
        assert abs(r.fun - U) < 0.01


def _fd_force(energy, x, h=1e-6):
    g = np.zeros_like(x)
    for idx in np.ndindex(x.shape):
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        g[idx] = -(energy(xp) - energy(xm)) / (2 * h)
    return g


def test_mueller_brown_force_is_minus_gradient():
    for x, y in [(-0.3, 0.8), (0.4, 0.2), (-1.0, 1.3)]:
        U, f = o.mb(x, y)
        fd = _fd_force(lambda p: o.mb(p[0], p[1])[0], np.array([x, y]))
        assert np.allclose(f, fd, rtol=1e-7, atol=1e-6)


def test_lj_two_atom_closed_forms():
    box = [10.0, 10.0, 10.0]
    # force zero at the minimum r = 2^(1/6) sigma; energy there -eps + shift
    x = np.array([[1.0, 1.0, 1.0], [1.0 + 2 ** (1 / 6), 1.0, 1.0]])
    U, f = o.lj(x, box)
    assert np.allclose(f, 0.0, atol=1e-12)
    shift = 4 * (2.5 ** -12 - 2.5 ** -6)
    assert U == pytest.approx(-1.0 - shift, abs=1e-12)
    # at r = sigma the repulsive force magnitude is 24 eps / sigma
    x = np.array([[0.2, 5.0, 5.0], [9.2, 5.0, 5.0]])  # separated by 1.0 through the boundary
    U, f = o.lj(x, box)
    assert f[0, 0] == pytest.approx(24.0, rel=1e-12) and f[1, 0] == pytest.approx(-24.0, rel=1e-12)
    # beyond the cutoff nothing
    x = np.array([[0.0, 0.0, 0.0], [2.6, 0.0, 0.0]])
    U, f = o.lj(x, box)
    assert U == 0.0 and np.all(f == 0.0)


def test_lj_force_matches_energy_gradient():
    x, L = synth.fcc_lattice(32, 0.8, seed=3, jitter=0.08)
    box = [L, L, L]
    U, f = o.lj(x, box)
    fd = _fd_force(lambda p: o.lj(p, box)[0], x)
    assert np.allclose(f, fd, rtol=1e-6, atol=1e-6)
    assert np.allclose(f.sum(0), 0.0, atol=1e-10)


def test_chain_force_matches_energy_gradient():
    x = synth.chain_replicas(1, 8, seed=5)
    x += synth.rng(1).normal(scale=0.05, size=x.shape)
    U, f = o.chain(x)
    fd = _fd_force(lambda p: o.chain(p)[0], x)
    assert np.allclose(f, fd, rtol=1e-6, atol=1e-5)
    assert np.allclose(f.sum(0), 0.0, atol=1e-9)


def test_chain_dimer_closed_form():
    """A stretched dimer: only the bond term, U = kb/2 (r - r0)^2 and a
    central force of magnitude kb |r - r0|."""
    kb, r0 = 100.0, 1.0
    for r in (0.8, 1.0, 1.3):
        d = np.array([0.3, -0.4, 1.2])
        d *= r / np.linalg.norm(d)
        x = np.array([[0.2, 0.1, -0.3], [0.2, 0.1, -0.3]]) + np.array([[0, 0, 0], d])
        U, f = o.chain(x, kb=kb, r0=r0, ka=50.0, kt=1.0)
        assert U == pytest.approx(0.5 * kb * (r - r0) ** 2, rel=1e-13, abs=1e-14)
        F1 = -kb * (r - r0) * d / r  # on bead 1, along +d when compressed
        assert np.allclose(f[1], F1, rtol=1e-12, atol=1e-13)
        assert np.allclose(f[0], -F1, rtol=1e-12, atol=1e-13)


def test_chain_trimer_closed_form():
    """A bent trimer with both bonds at r0: only the angle term,
    U = ka/2 (theta - theta0)^2 with theta0 in radians; bead 0 on the x axis
    and bead 2 at angle theta in the xy plane feel tangential forces of size
    ka |theta - theta0| / r0."""
    ka, r0, th0 = 50.0, 1.0, np.deg2rad(109.47)
    for th in (np.deg2rad(90.0), np.deg2rad(109.47), np.deg2rad(150.0)):
        x = np.array([[r0, 0.0, 0.0], [0.0, 0.0, 0.0], [r0 * np.cos(th), r0 * np.sin(th), 0.0]])
        U, f = o.chain(x, kb=100.0, r0=r0, ka=ka, th0=th0, kt=1.0)
        assert U == pytest.approx(0.5 * ka * (th - th0) ** 2, rel=1e-12, abs=1e-14)
        g = ka * (th - th0) / r0  # dU/dtheta / r0
        # moving bead 0 by +y closes the angle; moving bead 2 along
        # (-sin th, cos th) opens it
        assert np.allclose(f[0], [0.0, g, 0.0], rtol=1e-12, atol=1e-12)
        assert np.allclose(f[2], -g * np.array([-np.sin(th), np.cos(th), 0.0]), rtol=1e-12, atol=1e-12)
        assert np.allclose(f[1], -(f[0] + f[2]), rtol=1e-12, atol=1e-12)


def _tetramer(r0, th0, phi):
    """Four beads with bonds r0, both angles th0 and dihedral phi (cis = 0)."""
    return np.array([
        [r0 * np.cos(th0), r0 * np.sin(th0), 0.0],
        [0.0, 0.0, 0.0],
        [r0, 0.0, 0.0],
        [r0 - r0 * np.cos(th0), r0 * np.sin(th0) * np.cos(phi), r0 * np.sin(th0) * np.sin(phi)],
    ])


def test_chain_tetramer_torsion_closed_form():
    """A tetramer with bonds r0 and angles theta0 has only the torsion term
    kt (1 + cos 3 phi): 2 kt at phi = 0, 0 at pi/3 and pi, kt at pi/2; the end
    beads feel |dU/dphi| / (r0 sin theta0), normal to their bond plane."""
    kt, r0, th0 = 1.0, 1.0, np.deg2rad(109.47)
    for phi, Uc in ((0.0, 2.0), (np.pi / 3, 0.0), (np.pi, 0.0), (np.pi / 2, 1.0), (-np.pi / 2, 1.0)):
        x = _tetramer(r0, th0, phi)
        U, f = o.chain(x, kb=100.0, r0=r0, ka=50.0, th0=th0, kt=kt)
        assert U == pytest.approx(kt * Uc, abs=1e-12)
        mag = abs(3 * kt * np.sin(3 * phi)) / (r0 * np.sin(th0))
        assert np.linalg.norm(f[0]) == pytest.approx(mag, rel=1e-10, abs=1e-10)
        assert np.linalg.norm(f[3]) == pytest.approx(mag, rel=1e-10, abs=1e-10)
        n012 = np.cross(x[0] - x[1], x[2] - x[1])
        n123 = np.cross(x[1] - x[2], x[3] - x[2])
        assert abs(np.dot(f[0], n012)) == pytest.approx(mag * np.linalg.norm(n012), rel=1e-10, abs=1e-10)
        assert abs(np.dot(f[3], n123)) == pytest.approx(mag * np.linalg.norm(n123), rel=1e-10, abs=1e-10)
        assert np.allclose(f.sum(0), 0.0, atol=1e-12)
        assert np.allclose(np.cross(x, f).sum(0), 0.0, atol=1e-12)


def test_coordination_refuses_m_not_2n():
    """The switching function is defined here for m = 2n only; other exponent
    pairs are refused instead of being evaluated as m = 2n."""
    x = synth.rng(3).normal(size=(6, 3))
    with pytest.raises(ValueError):
        o.cv_eval(o.CV(o.CV_COORDINATION, a=[0, 1], r0=1.5, nn=6, mm=10), x)
    with pytest.raises(ValueError):
        o.cv_eval(o.CV(o.CV_QPAIRS, a=[0, 1, 2, 3], r0=1.5, nn=4, mm=12), x)
    o.cv_eval(o.CV(o.CV_COORDINATION, a=[0, 1], r0=1.5, nn=5, mm=10), x)


# --------------------------------------------------------------------------
# Collective variables (Sec. 2.2)
# --------------------------------------------------------------------------
def _fd_jac(cv, x, box=None, h=1e-6):
    J = np.zeros_like(x)
    for idx in np.ndindex(x.shape):
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        J[idx] = (o.cv_eval(cv, xp, box)[0] - o.cv_eval(cv, xm, box)[0]) / (2 * h)
    return J


def _cases():
    r = synth.rng(11)
    xl, L = synth.fcc_lattice(32, 0.8, seed=2, jitter=0.1)
    box = [L, L, L]
    yield "component", o.CV(o.CV_COMPONENT, a=[3], axis=1), xl, box
    yield "dihedral", o.CV(o.CV_DIHEDRAL, a=[5, 1, 9, 2]), r.normal(size=(12, 3)), None
    yield "dihedral_pbc", o.CV(o.CV_DIHEDRAL, a=[0, 1, 2, 3]), xl, box
    yield "coord_subset", o.CV(o.CV_COORDINATION, a=[0, 4, 7, 9], r0=1.5, nn=6, mm=12), xl, box
    yield "coord_all", o.CV(o.CV_COORDINATION, a=None, r0=1.2, nn=6, mm=12), xl, box
    yield "coord_ab", o.CV(o.CV_COORDINATION, a=[1, 2], b=[2, 3, 5, 8], r0=1.5, nn=8, mm=16), xl, box
    yield "rg_subset", o.CV(o.CV_RG, a=[0, 3, 5, 6, 11]), xl, box
    yield "rg_intensive", o.CV(o.CV_RG, a=None, flags=o.CV_INTENSIVE), r.normal(size=(9, 3)), None
    yield "qpairs", o.CV(o.CV_QPAIRS, a=[0, 1, 2, 5, 7, 3], r0=1.5, nn=6, mm=12), xl, box
    yield "distance_pbc", o.CV(o.CV_DISTANCE, a=[0, 3, 5], b=[9, 11]), xl, box
    yield "distance_open", o.CV(o.CV_DISTANCE, a=[1], b=[2, 4, 7, 8]), r.normal(size=(10, 3)), None
    yield "angle", o.CV(o.CV_ANGLE, a=[4, 0, 7]), r.normal(size=(9, 3)), None
    yield "angle_pbc", o.CV(o.CV_ANGLE, a=[2, 5, 6]), xl, box
    xg = r.normal(size=(11, 3)) * np.array([1.5, 1.0, 0.6])
    for q, nm in enumerate(("l1", "l2", "l3", "asphericity", "acylindricity", "anisotropy")):
        yield "gyration_" + nm, o.CV(o.CV_GYRATION, a=None, axis=q), xg, None
    yield "gyration_pbc", o.CV(o.CV_GYRATION, a=[0, 3, 5, 6, 11, 12], axis=o.GY_ANISOTROPY), xl, box


@pytest.mark.parametrize("name,cv,x,box", list(_cases()), ids=[c[0] for c in _cases()])
def test_cv_jacobian_matches_finite_differences(name, cv, x, box):
    xi, J = o.cv_eval(cv, x, box)
    fd = _fd_jac(cv, x, box)
    assert np.allclose(J, fd, rtol=1e-6, atol=1e-8), np.abs(J - fd).max()


@pytest.mark.parametrize("name,cv,x,box", [c for c in _cases() if c[0] != "component"],
                         ids=[c[0] for c in _cases() if c[0] != "component"])
def test_cv_translation_invariance_zero_net_force(name, cv, x, box):
    """Translation-invariant CVs: sum_j d xi / d r_j = 0 (no net bias force)."""
    xi, J = o.cv_eval(cv, x, box)
    assert np.allclose(J.sum(0), 0.0, atol=1e-10)
    xi2, _ = o.cv_eval(cv, x + np.array([0.37, -1.1, 2.3]), box)
    assert xi2 == pytest.approx(xi, abs=1e-11)


@pytest.mark.parametrize("name,cv,x,box", [c for c in _cases() if c[3] is None],
                         ids=[c[0] for c in _cases() if c[3] is None])
def test_cv_rotation_invariance_zero_net_torque(name, cv, x, box):
    """Rotation-invariant CVs (open boundaries): sum_j r_j x J_j = 0."""
    xi, J = o.cv_eval(cv, x, box)
    assert np.allclose(np.cross(x, J).sum(0), 0.0, atol=1e-10)
    q, _ = np.linalg.qr(synth.rng(4).normal(size=(3, 3)))
    if np.linalg.det(q) < 0:
        q[:, 0] *= -1
    xi2, _ = o.cv_eval(cv, x @ q.T, box)
    assert xi2 == pytest.approx(xi, abs=1e-11)


def test_distance_and_angle_closed_forms():
    # centres (0,0,0) and (3,4,0): distance 5, whatever the group sizes
    x = np.array([[1, 0, 0], [-1, 0, 0], [3, 4, 1], [3, 4, -1], [3, 4, 0.0]])
    xi, J = o.cv_eval(o.CV(o.CV_DISTANCE, a=[0, 1], b=[2, 3, 4]), x)
    assert xi == pytest.approx(5.0, abs=1e-14)
    assert np.allclose(J[0], -np.array([0.6, 0.8, 0]) / 2) and np.allclose(J[4], np.array([0.6, 0.8, 0]) / 3)
    # the centre difference uses the minimum image: groups 9 apart in a box of 10
    xb = np.array([[0.5, 0, 0], [9.5, 0, 0.0]])
    assert o.cv_eval(o.CV(o.CV_DISTANCE, a=[0], b=[1]), xb, [10.0, 10.0, 10.0])[0] == pytest.approx(1.0)
    tri = np.array([[1.0, 0, 0], [0, 0, 0], [0.5, np.sqrt(3) / 2, 0]])
    for pts, th in ((tri, np.pi / 3), (np.array([[1.0, 0, 0], [0, 0, 0], [0, 2.0, 0]]), np.pi / 2),
                    (np.array([[1.0, 0, 0], [0, 0, 0], [-3.0, 0, 0]]), np.pi)):
        assert o.cv_eval(o.CV(o.CV_ANGLE, a=[0, 1, 2]), pts)[0] == pytest.approx(th, abs=1e-14)
    # unit-length arms at a right angle: moving either end towards the other closes the angle at rate 1
    xi, J = o.cv_eval(o.CV(o.CV_ANGLE, a=[0, 1, 2]), np.array([[1.0, 0, 0], [0, 0, 0], [0, 1.0, 0]]))
    assert np.allclose(J[0], [0, -1, 0]) and np.allclose(J[2], [-1, 0, 0]) and np.allclose(J[1], [1, 1, 0])


def test_gyration_tensor_closed_forms():
    """Rod of n atoms spaced a: l3 = a^2 (n^2-1)/12, l1 = l2 = 0, asphericity
    l3, acylindricity 0, anisotropy 1.  Square of side a: l = (0, a^2/4,
    a^2/4), asphericity a^2/8, acylindricity a^2/4, anisotropy 1/4.  Cube
    corners: isotropic, asphericity = acylindricity = anisotropy = 0.  In
    every case l1 + l2 + l3 = Rg^2."""
    def q(x, k):
        return o.cv_eval(o.CV(o.CV_GYRATION, a=None, axis=k), x)[0]

    rot, _ = np.linalg.qr(synth.rng(8).normal(size=(3, 3)))
    n, a = 7, 0.8
    rod = (np.arange(n)[:, None] * a * np.array([[1.0, 0, 0]])) @ rot.T + 2.0
    l3 = a * a * (n * n - 1) / 12
    assert q(rod, 2) == pytest.approx(l3, rel=1e-12)
    assert abs(q(rod, 0)) < 1e-13 and abs(q(rod, 1)) < 1e-13
    assert q(rod, 3) == pytest.approx(l3, rel=1e-12) and abs(q(rod, 4)) < 1e-13
    assert q(rod, 5) == pytest.approx(1.0, rel=1e-12)
    sq = (np.array([[1, 1, 0], [1, -1, 0], [-1, 1, 0], [-1, -1, 0.0]]) * a / 2) @ rot.T
    assert [q(sq, k) for k in range(3)] == pytest.approx([0.0, a * a / 4, a * a / 4], abs=1e-13)
    assert q(sq, 3) == pytest.approx(a * a / 8, rel=1e-12) and q(sq, 4) == pytest.approx(a * a / 4, rel=1e-12)
    assert q(sq, 5) == pytest.approx(0.25, rel=1e-12)
    cube = np.array([[i, j, k] for i in (-1, 1) for j in (-1, 1) for k in (-1, 1)], float) @ rot.T
    for k in (3, 4, 5):
        assert abs(q(cube, k)) < 1e-12
    x = synth.rng(9).normal(size=(13, 3))
    rg = o.cv_eval(o.CV(o.CV_RG, a=None), x)[0]
    assert sum(q(x, k) for k in range(3)) == pytest.approx(rg * rg, rel=1e-12)


def test_dihedral_conventions():
    """IUPAC: cis = 0, trans = pi, and +90 deg when, looking along b->c, the
    a-b bond turns clockwise onto c-d."""
    cv = o.CV(o.CV_DIHEDRAL, a=[0, 1, 2, 3])
    p = lambda d: np.array([[0, 1, 0], [0, 0, 0], [1, 0, 0], d], dtype=float)
    assert o.cv_eval(cv, p([1, 1, 0]))[0] == pytest.approx(0.0, abs=1e-15)
    assert abs(o.cv_eval(cv, p([1, -1, 0]))[0]) == pytest.approx(np.pi, abs=1e-15)
    assert o.cv_eval(cv, p([1, 0, 1]))[0] == pytest.approx(np.pi / 2, abs=1e-15)
    assert o.cv_eval(cv, p([1, 0, -1]))[0] == pytest.approx(-np.pi / 2, abs=1e-15)


def test_switching_function_closed_forms():
    """s(r0) = n/m = 1/2 and s(2^(1/6) r0) = 1/(1+2) for n=6, m=12."""
    for r, want in [(1.5, 0.5), (1.5 * 2 ** (1 / 6), 1 / 3)]:
        x = np.array([[0.0, 0.0, 0.0], [r, 0.0, 0.0]])
        cv = o.CV(o.CV_COORDINATION, a=[0], r0=1.5, nn=6, mm=12)
        assert o.cv_eval(cv, x)[0] == pytest.approx(want, rel=1e-14)
        cv = o.CV(o.CV_COORDINATION, a=None, r0=1.5, nn=6, mm=12)  # each atom sees the other
        assert o.cv_eval(cv, x)[0] == pytest.approx(want, rel=1e-14)


def test_coordination_counts_neighbours_of_a_lattice():
    """Periodic 4x4x4 simple cubic lattice of spacing 1: along each axis the
    minimum-image separations from an atom to the 4 atoms of its row have
    magnitudes {0, 1, 1, 2}, so the partners of every atom are the 63 offsets
    of {0,1,1,2}^3 minus the origin, and the mean coordination is the sum of
    s(|offset|) over them."""
    g = np.stack(np.meshgrid(*[np.arange(4.0)] * 3, indexing="ij"), -1).reshape(-1, 3)
    axis = [0.0, 1.0, 1.0, 2.0]
    for r0, n in [(0.5, 24), (1.0, 6), (1.7, 8)]:
        want = 0.0
        for a in axis:
            for b in axis:
                for c in axis:
                    r2 = a * a + b * b + c * c
                    if r2 > 0:
                        want += 1.0 / (1.0 + (r2 / r0 ** 2) ** (n / 2))
        cv = o.CV(o.CV_COORDINATION, a=None, r0=r0, nn=n, mm=2 * n)
        xi, _ = o.cv_eval(cv, g, [4.0, 4.0, 4.0])
        assert xi == pytest.approx(want, rel=1e-13)


def test_rg_closed_forms_and_unwrapping():
    a = 1.3
    tet = a / np.sqrt(8) * np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], dtype=float)
    cv = o.CV(o.CV_RG, a=None)
    assert o.cv_eval(cv, tet)[0] == pytest.approx(a * np.sqrt(3 / 8), rel=1e-14)
    sq = np.array([[0, 0, 0], [a, 0, 0], [a, a, 0], [0, a, 0]], dtype=float)
    assert o.cv_eval(cv, sq)[0] == pytest.approx(a / np.sqrt(2), rel=1e-14)
    # a group straddling the periodic boundary
    L = 5.0
    shifted = np.mod(sq + np.array([4.5, 4.5, 1.0]), L)
    assert o.cv_eval(cv, shifted, [L, L, L])[0] == pytest.approx(a / np.sqrt(2), rel=1e-12)
    cvi = o.CV(o.CV_RG, a=None, flags=o.CV_INTENSIVE)
    assert o.cv_eval(cvi, sq)[0] == pytest.approx(a / np.sqrt(2) / 4 ** (1 / 3), rel=1e-14)


# --------------------------------------------------------------------------
# Hills sum (Sec. 2.1.5)
# --------------------------------------------------------------------------
def test_single_hill_closed_forms():
    sig = [0.05, 0.2, 0.7]
    h = np.array([[0.3, -1.0, 2.0, 1.7]])
    for d in (1, 2, 3):
        s = h[0, :d]
        V, dV = o.hills_sum(s[None], h, sig[:d])
        assert V[0] == pytest.approx(1.7, rel=1e-15) and np.all(dV == 0)
        for i in range(d):
            p = s.copy()
            p[i] += sig[i]
            V, dV = o.hills_sum(p[None], h, sig[:d])
            assert V[0] == pytest.approx(1.7 * np.exp(-0.5), rel=1e-14)
            assert dV[0, i] == pytest.approx(-1.7 * np.exp(-0.5) / sig[i], rel=1e-14)
            assert np.all(np.delete(dV[0], i) == 0)


def test_hills_gradient_matches_fd_and_sum_is_linear():
    sig = [0.3, 0.5, 0.4]
    hills = synth.uniform_hills(40, [-1, -1, -1], [1, 1, 1], seed=9)
    pts = synth.uniform_points(6, [-1, -1, -1], [1, 1, 1], seed=10)
    V, dV = o.hills_sum(pts, hills, sig)
    h = 1e-6
    for i in range(3):
        e = np.zeros(3)
        e[i] = h
        fd = (o.hills_sum(pts + e, hills, sig)[0] - o.hills_sum(pts - e, hills, sig)[0]) / (2 * h)
        assert np.allclose(dV[:, i], fd, rtol=1e-7, atol=1e-9)
    V1, dV1 = o.hills_sum(pts, hills[:17], sig)
    V2, dV2 = o.hills_sum(pts, hills[17:], sig)
    assert np.allclose(V, V1 + V2, rtol=1e-14) and np.allclose(dV, dV1 + dV2, rtol=1e-12, atol=1e-15)


def test_periodic_hills_wrap():
    sig = [0.35, 0.35]
    per = [2 * np.pi, 2 * np.pi]
    hills = synth.uniform_hills(30, [-np.pi, -np.pi], [np.pi, np.pi], seed=4)
    pts = synth.uniform_points(5, [-np.pi, -np.pi], [np.pi, np.pi], seed=5)
    V, dV = o.hills_sum(pts, hills, sig, per)
    V2, dV2 = o.hills_sum(pts + np.array([2 * np.pi, -4 * np.pi]), hills, sig, per)
    assert np.allclose(V, V2, rtol=1e-12) and np.allclose(dV, dV2, rtol=1e-10, atol=1e-12)
    # a hill at +pi - eps seen from -pi + eps is 2 eps away
    h = np.array([[np.pi - 0.01, 0.0, 0.0, 1.0]])
    V, _ = o.hills_sum(np.array([[-np.pi + 0.01, 0.0]]), h, sig, per)
    assert V[0] == pytest.approx(np.exp(-0.02 ** 2 / (2 * 0.35 ** 2)), rel=1e-12)


def test_grid_integral_matches_gaussian_volume():
    """Sum over a fine grid times the cell volume = w (2 pi)^(d/2) prod sigma."""
    bins, lo, hi, sig = (200, 160), (-2.0, -1.0), (2.0, 3.0), (0.15, 0.25)
    g = np.zeros(bins[0] * bins[1])
    o.grid_add(g, bins, lo, hi, sig, (0.1, 0.9), 2.5)
    vol = np.prod([(hi[i] - lo[i]) / bins[i] for i in range(2)])
    assert g.sum() * vol == pytest.approx(2.5 * 2 * np.pi * 0.15 * 0.25, rel=1e-9)
    # grid values are the hills sum at the cell centres
    cx, cy = o.grid_centres(bins, lo, hi)
    V, _ = o.hills_sum(np.array([[cx[17], cy[101]]]), np.array([[0.1, 0.9, 0, 2.5]]), sig)
    assert g.reshape(bins)[17, 101] == pytest.approx(V[0], rel=1e-14)


def test_fes_is_scaled_negative_bias_with_zero_minimum():
    grid = np.array([0.0, 3.0, 1.0, 2.5])
    assert np.allclose(o.fes(grid, 10.0), (-10 / 9) * grid + 10 / 9 * 3.0)
    assert np.allclose(o.fes(grid, 0.0), 3.0 - grid)  # standard metadynamics


# --------------------------------------------------------------------------
# Well-tempered deposition (Sec. 2.1.5) and the step loop
# --------------------------------------------------------------------------
def _frozen_walker(gamma, w0=1.0, kT=2.0, stride=3, steps=60):
    """A walker that cannot move (huge mass) deposits all hills at one point."""
    s = o.System(engine=o.ENGINE_NONE, walker_n=[1], cvs=[o.CV(o.CV_COMPONENT, a=[0], axis=0)],
                 mass=1e30, kT=kT, sigma=(0.2,), w0=w0, gamma=gamma, stride=stride, hill_cap=1000, dt=0.01)
    sim = o.Sim(s, x=[[0.4, 0.0, 0.0]])
    sim.forces()
    assert sim.run(steps) == 0
    return sim


def test_wt_heights_follow_fixed_point_recursion():
    """All hills at one point: V_{k+1} = V_k + w0 exp(-V_k / (kT (gamma-1))),
    and V_k stays between the continuous-time solutions
    dT ln(1 + k w0/dT) <= V_k <= w0 + dT ln(1 + (k-1) w0/dT)."""
    gamma, w0, kT = 6.0, 1.0, 2.0
    dT = kT * (gamma - 1)
    sim = _frozen_walker(gamma, w0, kT)
    assert sim.n_hills == 20
    w = sim.hills[: sim.n_hills, 3]
    V = 0.0
    for k in range(sim.n_hills):
        assert w[k] == pytest.approx(w0 * np.exp(-V / dT), rel=1e-12)
        V += w[k]
        n = k + 1
        assert dT * np.log1p(n * w0 / dT) - 1e-12 <= V <= w0 + dT * np.log1p((n - 1) * w0 / dT) + 1e-12
    assert np.all(np.diff(w) < 0)


def test_standard_metadynamics_has_fixed_heights():
    sim = _frozen_walker(0.0, w0=0.7)
    assert np.all(sim.hills[: sim.n_hills, 3] == 0.7)


def test_deposition_timing_and_capacity():
    s = o.System(engine=o.ENGINE_MB, walker_n=[1, 1, 1], dims=2,
                 cvs=[o.CV(o.CV_COMPONENT, a=[0], axis=0), o.CV(o.CV_COMPONENT, a=[0], axis=1)],
                 dt=1e-4, kT=15.0, sigma=(0.05, 0.05), w0=1.0, gamma=10.0, stride=10, hill_cap=12)
    x = np.array([[-0.558, 1.442, 0], [0.623, 0.028, 0], [-0.05, 0.467, 0]])
    sim = o.Sim(s, x=x)
    sim.forces()
    assert sim.run(9) == 0 and sim.n_hills == 0
    assert sim.run(1) == 0 and sim.n_hills == 3
    # hills carry the walkers' CVs in walker order
    assert np.allclose(sim.hills[:3, :2], sim.xi[:, :2], rtol=0, atol=0)
    assert sim.run(30) == 0 and sim.n_hills == 12
    assert sim.run(10) == -3 and sim.n_hills == 12  # capacity reached: reported, nothing written


def test_baoab_samples_harmonic_oscillator_exactly():
    """BAOAB gives the exact configurational variance kT/k for a harmonic
    oscillator at any stable time step (Leimkuhler & Matthews 2013)."""
    s = o.System(engine=o.ENGINE_HARMONIC, walker_n=[1], cvs=[], harm_k=4.0, kT=1.5, dt=0.4, friction=1.0,
                 seed=3, bias_on=False)
    sim = o.Sim(s, x=[[0.0, 0.0, 0.0]])
    sim.forces()
    xs = []
    for _ in range(2000):
        sim.run(50)
        xs.append(sim.x[0].copy())
    xs = np.array(xs)
    assert np.mean(xs ** 2) == pytest.approx(1.5 / 4.0, rel=0.05)


def test_lj_nve_conserves_energy():
    """friction 0: BAOAB reduces to velocity Verlet; total energy drifts only
    at O(dt^2)."""
    x, L = synth.fcc_lattice(108, 0.8, seed=1, jitter=0.05)
    v = synth.velocities(108, 1.0, 1.0, seed=2)
    v -= v.mean(0)
    s = o.System(engine=o.ENGINE_LJ, walker_n=[108], cvs=[], box=(L, L, L), dt=0.002, friction=0.0, bias_on=False)
    sim = o.Sim(s, x=x, v=v)
    sim.forces()

    def energy():
        return o.lj(sim.x, [L, L, L])[0] + 0.5 * np.sum(sim.v ** 2)

    e0 = energy()
    sim.run(300)
    assert abs(energy() - e0) / abs(e0) < 5e-4


def test_bias_force_is_minus_gradient_of_bias_energy():
    """The bias force f = -J^T dV/dxi equals -d V(xi(x)) / dx by finite
    differences (chain rule through CV and hills sum)."""
    xl, L = synth.fcc_lattice(32, 0.8, seed=6, jitter=0.1)
    box = (L, L, L)
    cvs = [o.CV(o.CV_COORDINATION, a=[0, 3, 8], r0=1.5), o.CV(o.CV_RG, a=[1, 2, 4, 5, 9])]
    s = o.System(engine=o.ENGINE_NONE, walker_n=[32], cvs=cvs, box=box, sigma=(0.05, 0.1))
    sim = o.Sim(s, x=xl)
    _, xi, _, _ = sim.bias(xl, hills=np.zeros((0, 4)))
    hills = synth.walk_hills(25, xi[0, :2] - 0.1, xi[0, :2] + 0.1, 0.02, seed=8)
    f, xi, V, dV = sim.bias(xl, hills=hills)
    fd = _fd_force(lambda p: sim.bias(p, hills=hills)[2][0], xl)
    # central differences with h = 1e-6 on hills of width 0.05: truncation
    # error ~1e-7 of the largest component
    assert np.allclose(f, fd, rtol=1e-6, atol=1e-7 * np.abs(f).max())


@pytest.mark.slow
def test_mueller_brown_free_energy_recovered_within_half_kT():
    """WTMD on (x, y) of a Mueller-Brown particle: -(gamma/(gamma-1)) V on
    the grid matches U_MB up to a constant within 0.5 kT on visited cells
    up to 5 kT above the global minimum (Sec. 2.1, Eq. (free-energy): the
    CVs are the only coordinates, so A = U + C)."""
    bins, lo, hi = (60, 60), (-1.5, -0.5), (1.2, 2.2)
    kT = 15.0
    s = o.System(engine=o.ENGINE_MB, walker_n=[1], dims=2,
                 cvs=[o.CV(o.CV_COMPONENT, a=[0], axis=0), o.CV(o.CV_COMPONENT, a=[0], axis=1)],
                 dt=2e-3, friction=5.0, kT=kT, sigma=(0.05, 0.05), w0=0.5, gamma=10.0, stride=20,
                 hill_cap=20000, grid_bins=bins, grid_lo=lo, grid_hi=hi, seed=0)
    sim = o.Sim(s, x=[[-0.558, 1.442, 0.0]])
    sim.forces()
    vis = np.zeros(bins, bool)
    for _ in range(3000):
        assert sim.run(100) == 0
        i = int((sim.x[0, 0] - lo[0]) / (hi[0] - lo[0]) * bins[0])
        j = int((sim.x[0, 1] - lo[1]) / (hi[1] - lo[1]) * bins[1])
        if 0 <= i < bins[0] and 0 <= j < bins[1]:
            vis[i, j] = True
    F = sim.fes().reshape(bins)
    cx, cy = o.grid_centres(bins, lo, hi)
    U = np.array([[o.mb(a, b)[0] for b in cy] for a in cx])
    m = vis & (U < U.min() + 5 * kT)
    assert m.sum() > 200
    d = (F - U)[m]
    d -= d.mean()
    assert np.abs(d).max() < 0.5 * kT
    assert np.sqrt(np.mean(d ** 2)) < 0.25 * kT


def test_three_well_landscape_force_and_minima():
    """The three-well landscape: force = -grad U by central differences, and
    a local minimum near each well centre, lower than the saddle region."""
    import oracle as o

    r = np.array([0.3, -0.2, 0.4])
    h = 1e-6
    u, f = o.wells3(r)
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        fd = -(o.wells3(r + e)[0] - o.wells3(r - e)[0]) / (2 * h)
        assert abs(fd - f[k]) < 1e-7 * max(1.0, abs(f[k]))
    for c in ([-1.0, 0.0, 0.0], [1.0, 0.2, -0.3], [0.1, 1.3, 0.6]):
        x = np.array(c, float)
        for _ in range(2000):  # steepest descent
            x = x + 0.01 * o.wells3(x)[1]
        assert np.linalg.norm(o.wells3(x)[1]) < 1e-6
        assert np.linalg.norm(x - np.array(c)) < 0.5
        assert o.wells3(x)[0] < o.wells3((x + np.zeros(3)) * 0.0 + np.array([0.0, 0.5, 0.0]))[0]
