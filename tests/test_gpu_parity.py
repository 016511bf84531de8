"""GPU (libwtmd, through the C ABI) against the FP64 oracle on the same seeded
inputs.

Tolerances:
  * FP64 handles: 1e-12 relative (V, dV/dxi, CVs, forces norm-wise).
  * FP32 handles: 1e-5 relative.  V is a sum of positive terms: plain
    relative error.  dV/dxi and the bias force are signed sums whose terms
    can cancel (a walker inside a filled basin sits where the bias is flat);
    there the bound is 1e-5 of the sum of the absolute terms,
    S_c = sum_k w_k e_k |D_kc| / sigma_c^2 for dV/dxi_c and
    F_scale,i = sum_c S_c |J_ci| for the force (norm-wise).  Without
    cancellation these equal |dV| and |F|: the plain relative bound.
The oracle always receives the inputs exactly as the GPU sees them (FP32
handles: positions and points rounded to float first).
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


def _close_V(Vg, Vr, prec):
    tol = 1e-12 if prec == "f64" else 1e-5
    assert np.all(np.abs(Vg - Vr) <= tol * np.abs(Vr) + 1e-300), np.max(np.abs(Vg - Vr) / np.maximum(np.abs(Vr), 1e-300))


def grad_scale(pts, hills, sigma, period=None):
    """S[p, c] = sum_k w_k e_k |D_kc| / sigma_c^2 (tolerance scale only)."""
    pts = np.atleast_2d(pts)
    d = pts.shape[1]
    sig = np.asarray(sigma, float)[:d]
    per = np.zeros(d) if period is None else np.asarray(period, float)[:d]
    out = np.zeros((pts.shape[0], d))
    for p in range(pts.shape[0]):
        D = pts[p][None, :] - hills[:, :d]
        D = np.where(per > 0, D - per * np.rint(D / np.where(per > 0, per, 1.0)), D)
        e = hills[:, 3] * np.exp(-(D ** 2 / (2 * sig ** 2)).sum(1))
        out[p] = (e[:, None] * np.abs(D)).sum(0) / sig ** 2
    return out


def _close_dV(dg, dr, S, prec):
    """FP64: 1e-12 of |dV|; FP32: 1e-5 of the absolute-term sum S."""
    if prec == "f64":
        err = np.abs(dg - dr) / np.maximum(np.abs(dr), 1e-300)
        ok = np.abs(dg - dr) <= 1e-12 * np.abs(dr) + 1e-13 * S
    else:
        err = np.abs(dg - dr) / np.maximum(S, 1e-300)
        ok = err <= 1e-5
    assert np.all(ok), err.max()


def _close_F(Fg, Fr, prec, Fscale=None):
    """FP64: ||dF|| <= 1e-12 ||F||.  FP32: ||dF|| <= 1e-5 ||F_scale||, where
    F_scale,i = sum_c S_c |J_ci| and S_c = sum_k w_k e_k |D_kc| / sigma_c^2 is
    the sum of the absolute gradient terms: a bias gradient that cancels to
    a small fraction of its terms (a walker inside a filled basin) cannot be
    resolved to 1e-5 of itself in FP32, only to 1e-5 of its terms.  Without
    cancellation F_scale = |F| and this is the plain relative bound."""
    tol = 1e-12 if prec == "f64" else 1e-5
    den = np.linalg.norm(Fr) if (prec == "f64" or Fscale is None) else np.linalg.norm(Fscale)
    assert np.linalg.norm(Fg - Fr) <= tol * den, np.linalg.norm(Fg - Fr) / den


def force_scale(sim, x, hills, cvs_period):
    """F_scale of _close_F from the oracle's CV Jacobians (tolerance only)."""
    import oracle as o

    sysd = sim.sys
    sig = np.asarray(sysd.sigma[: len(sysd.cvs)])
    per = np.asarray(cvs_period)
    out = np.zeros_like(x)
    off = 0
    box = list(sysd.box)
    for n in sysd.walker_n:
        xw = x[off: off + n]
        xi, Js = [], []
        for cv in sysd.cvs:
            v, J = o.cv_eval(cv, xw, box)
            xi.append(v)
            Js.append(J)
        D = np.asarray(xi)[None, :] - hills[:, : len(xi)]
        D = np.where(per > 0, D - per * np.rint(D / np.where(per > 0, per, 1.0)), D)
        e = hills[:, 3] * np.exp(-(D ** 2 / (2 * sig ** 2)).sum(1))
        S = (e[:, None] * np.abs(D)).sum(0) / sig ** 2
        out[off: off + n] = sum(S[c] * np.abs(Js[c]) for c in range(len(xi)))
        off += n
    return out


# --------------------------------------------------------------------------
def test_philox_bitwise():
    wt = _wt()
    import oracle as o

    r = synth.rng(5)
    q = r.integers(0, 2 ** 32, size=(257, 6), dtype=np.uint64).astype(np.uint32)
    out = wt.philox(q)
    for i in range(q.shape[0]):
        assert list(out[i]) == list(o.philox4x32_10(q[i, :4], q[i, 4:]))


# --------------------------------------------------------------------------
# hills sum
# --------------------------------------------------------------------------
HILL_CASES = [
    # d, periodic, P, H
    (1, False, 1, 1),
    (2, False, 1, 1001),
    (2, False, 5, 257),
    (2, False, 40, 3001),
    (2, True, 300, 2049),
    (3, False, 2100, 513),
    (3, True, 7, 999),
    (1, True, 1100, 4097),
    (3, False, 1, 200001),   # few-points kernel: hundreds of splits, odd count
    (2, True, 8, 100003),
]


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("d,periodic,P,H", HILL_CASES)
def test_hills_eval_matches_oracle(prec, d, periodic, P, H):
    wt = _wt()
    import oracle as o

    sigma = [0.35, 0.2, 0.5][:d] if periodic else [0.05, 0.1, 0.07][:d]
    lo, hi = ([-np.pi] * d, [np.pi] * d) if periodic else ([-1.0, 0.5, 2.0][:d], [1.5, 2.0, 3.0][:d])
    per = [2 * np.pi] * d if periodic else [0.0] * d
    hills = synth.uniform_hills(H, lo, hi, seed=d * 100 + P)
    pts = synth.uniform_points(P, lo, hi, seed=d * 100 + P + 1)
    m = wt.Wtmd(precision=prec, sigma=sigma, capacity=H + 3, walker_sizes=[1])
    for i in range(d):
        m.cv_define(wt.CV_COMPONENT, a=[0], axis=i, period=per[i])
    m.hills_load(hills)
    dt = torch.float32 if prec == "f32" else torch.float64
    x = torch.tensor(pts, dtype=dt, device="cuda")
    V, dV = m.hills_eval(x)
    torch.cuda.synchronize()
    xr = _f32(pts) if prec == "f32" else pts
    Vr, dVr = o.hills_sum(xr, hills, sigma, per)
    _close_V(to_np(V), Vr, prec)
    _close_dV(to_np(dV), dVr, grad_scale(xr, hills, sigma, per), prec)


CLUSTER_CASES = [
    # d, periodic, P, H, cluster size
    (1, False, 1, 1, 8),
    (2, False, 1, 100001, 8),
    (2, False, 1, 100001, 16),
    (3, True, 3, 4097, 16),
    (2, True, 8, 200003, 16),
    (3, False, 1, 0, 8),
]


@pytest.mark.parametrize("d,periodic,P,H,cl", CLUSTER_CASES)
def test_hills_cluster_kernel_matches_oracle(d, periodic, P, H, cl):
    """The few-points sum on one thread-block cluster (split sums met in
    distributed shared memory), forced by wtmd_hills_plan; twice in a row,
    bitwise equal."""
    wt = _wt()
    import oracle as o

    sigma = [0.35, 0.2, 0.5][:d] if periodic else [0.05, 0.1, 0.07][:d]
    lo, hi = ([-np.pi] * d, [np.pi] * d) if periodic else ([-1.0, 0.5, 2.0][:d], [1.5, 2.0, 3.0][:d])
    per = [2 * np.pi] * d if periodic else [0.0] * d
    hills = synth.uniform_hills(H, lo, hi, seed=d * 100 + P + 7)
    pts = synth.uniform_points(P, lo, hi, seed=d * 100 + P + 8)
    if H == 1:  # a point near the one hill (far away, V underflows FP32)
        pts = hills[:1, :d] + 0.3 * np.asarray(sigma)
    m = wt.Wtmd(precision="f32", sigma=sigma, capacity=max(H, 1) + 3, walker_sizes=[1])
    for i in range(d):
        m.cv_define(wt.CV_COMPONENT, a=[0], axis=i, period=per[i])
    if H:
        m.hills_load(hills)
    try:
        m.hills_plan(P, -1, cl)
    except wt.WtmdError:
        assert cl == 16
        pytest.skip("clusters of 16 CTAs are not available on this device")
    x = torch.tensor(pts, dtype=torch.float32, device="cuda")
    V, dV = m.hills_eval(x)
    V2, dV2 = m.hills_eval(x)
    torch.cuda.synchronize()
    assert torch.equal(V, V2) and torch.equal(dV, dV2)
    xr = _f32(pts)
    if H == 0:
        assert torch.all(V == 0) and torch.all(dV == 0)
        return
    Vr, dVr = o.hills_sum(xr, hills, sigma, per)
    _close_V(to_np(V), Vr, "f32")
    _close_dV(to_np(dV), dVr, grad_scale(xr, hills, sigma, per), "f32")


def test_hills_plan_rejects_bad_values():
    wt = _wt()
    m = wt.Wtmd(precision="f32", sigma=[0.1], capacity=10, walker_sizes=[1])
    m.cv_define(wt.CV_COMPONENT, a=[0], axis=0)
    for P, lanes, splits in ((9, 0, 8), (9, -1, 8), (1, -1, 12), (1, 3, 8), (1, 4, 0), (0, 4, 8)):
        with pytest.raises(wt.WtmdError):
            m.hills_plan(P, lanes, splits)
    m64 = wt.Wtmd(precision="f64", sigma=[0.1], capacity=10, walker_sizes=[1])
    m64.cv_define(wt.CV_COMPONENT, a=[0], axis=0)
    with pytest.raises(wt.WtmdError):
        m64.hills_plan(1, -1, 8)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_hills_eval_edge_cases(prec):
    wt = _wt()
    dt = torch.float32 if prec == "f32" else torch.float64
    m = wt.Wtmd(precision=prec, sigma=[0.1, 0.2], capacity=10, walker_sizes=[1])
    m.cv_define(wt.CV_COMPONENT, a=[0], axis=0)
    m.cv_define(wt.CV_COMPONENT, a=[0], axis=1)
    x = torch.tensor([[0.25, 0.375], [1.0, -2.0]], dtype=dt, device="cuda")  # exact in FP32
    V, dV = m.hills_eval(x)  # no hills
    assert torch.all(V == 0) and torch.all(dV == 0)
    m.hills_load([[0.25, 0.375, 0.0, 2.0]])  # one hill: V(s) = w, dV(s) = 0
    V, dV = m.hills_eval(x[:1])
    assert abs(V.item() - 2.0) <= (1e-6 if prec == "f32" else 1e-15) * 2
    assert torch.all(dV.abs() <= 1e-6)
    V, dV = m.hills_eval(x[:0])  # zero points
    assert V.numel() == 0
    with pytest.raises(wt.WtmdError):
        m.hills_load(np.zeros((11, 4)) + [0, 0, 0, 1])  # over capacity
    with pytest.raises(wt.WtmdError):
        m.hills_load([[0.0, 0.0, 0.0, -1.0]])  # negative height


# --------------------------------------------------------------------------
# bias_eval: CVs + hills + scatter on LJ systems
# --------------------------------------------------------------------------
def _bias_case(spec, x, prec, n_hills, seed=3):
    wt = _wt()
    import oracle as o

    dt = torch.float32 if prec == "f32" else torch.float64
    xin = _f32(x) if prec == "f32" else x
    osys = oracle_system(spec)
    sim = o.Sim(osys, x=xin)
    _, xi0, _, _ = sim.bias(xin, hills=np.zeros((0, 4)))
    d = len(spec["cvs"])
    sig = np.asarray(spec["sigma"])
    hills = synth.walk_hills(n_hills, xi0[0, :d] - 3 * sig, xi0[0, :d] + 3 * sig, 0.5 * sig, seed=seed)
    Fr, xir, Vr, dVr = sim.bias(xin, hills=hills)
    m = gpu_handle(spec, prec)
    m.hills_load(hills)
    pos = wt.particles(xin, dt)
    F = torch.zeros_like(pos)
    V, xi, dV = m.bias_eval(pos, F)
    torch.cuda.synchronize()
    per = [c.get("period", 0.0) for c in spec["cvs"]]
    Fs = force_scale(sim, xin, hills, per)
    S = grad_scale(xir[:, :d], hills, spec["sigma"], per)
    return (to_np(F)[:, :3], to_np(xi), to_np(V), to_np(dV)), (Fr, xir[:, :d], Vr, dVr[:, :d], Fs, S)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_bias_eval_lj_small(prec):
    spec, x, L = lj_fluid_spec(n=500, n_tag=37, n_rg=20, seed=4, jitter=0.1)
    (F, xi, V, dV), (Fr, xir, Vr, dVr, Fs, S) = _bias_case(spec, x, prec, 301)
    tol = 1e-12 if prec == "f64" else 1e-6
    assert np.allclose(xi, xir, rtol=tol, atol=0)
    _close_V(V, Vr, prec)
    _close_dV(dV, dVr, S, prec)
    _close_F(F, Fr, prec, Fs)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_bias_eval_lj_4096_full_size(prec):
    """The 4096-atom workload (512 tagged, 64-atom Rg) with 1e5 hills."""
    spec, x, L = lj_fluid_spec(n=4096, seed=0)
    (F, xi, V, dV), (Fr, xir, Vr, dVr, Fs, S) = _bias_case(spec, x, prec, 100000)
    tol = 1e-12 if prec == "f64" else 1e-6
    assert np.allclose(xi, xir, rtol=tol, atol=0)
    _close_V(V, Vr, prec)
    _close_dV(dV, dVr, S, prec)
    _close_F(F, Fr, prec, Fs)


CV_CASES = {
    "component": [dict(kind="component", a=[7], axis=2)],
    "dihedral_pbc": [dict(kind="dihedral", a=[3, 10, 11, 40], period=2 * np.pi)],
    "coord_all": [dict(kind="coordination", a=None, r0=1.2, nn=6, mm=12)],
    "coord_ab": [dict(kind="coordination", a=[1, 5, 9, 200], b=list(range(0, 300, 2)), r0=1.5, nn=8, mm=16)],
    "rg_all_intensive": [dict(kind="rg", a=None, flags=1)],
    "qpairs": [dict(kind="qpairs", a=[0, 1, 2, 5, 7, 3, 1, 9, 40, 41], r0=1.5, nn=6, mm=12)],
    "distance": [dict(kind="distance", a=list(range(0, 40, 3)), b=[100, 101, 250])],
    "angle": [dict(kind="angle", a=[3, 10, 11])],
    "gyration_shape": [dict(kind="gyration", a=list(range(100, 164)), axis=5),
                       dict(kind="gyration", a=list(range(100, 164)), axis=3),
                       dict(kind="gyration", a=None, axis=2)],
    "gyration_moments": [dict(kind="gyration", a=list(range(200, 232)), axis=0),
                         dict(kind="gyration", a=list(range(200, 232)), axis=1),
                         dict(kind="gyration", a=list(range(200, 232)), axis=4)],
    "three_cvs": [dict(kind="coordination", a=list(range(0, 500, 5)), r0=1.5),
                  dict(kind="rg", a=list(range(100, 164))),
                  dict(kind="qpairs", a=[0, 1, 2, 5, 7, 3, 1, 9], r0=1.5)],
}


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("name", list(CV_CASES))
def test_bias_eval_each_cv(prec, name):
    x, L = synth.fcc_lattice(500, 0.8, seed=9, jitter=0.1)
    cvs = CV_CASES[name]
    sig = [0.05, 0.1, 0.02][: len(cvs)]
    if name == "dihedral_pbc":
        sig = [0.35]
    spec = dict(engine="lj", walker_sizes=[500], box=(L, L, L), sigma=sig, cvs=cvs, capacity=2000)
    (F, xi, V, dV), (Fr, xir, Vr, dVr, Fs, S) = _bias_case(spec, x, prec, 777)
    tol = 1e-12 if prec == "f64" else 1e-6
    assert np.allclose(xi, xir, rtol=tol, atol=tol)
    _close_V(V, Vr, prec)
    _close_F(F, Fr, prec, Fs)


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("with_b", [False, True])
def test_bias_eval_walkers_coordination_tiles(prec, with_b):
    """Three walkers of uneven size sharing one box: the coordination tile
    path (an explicit tagged list, partners all atoms of the walker or an
    explicit list) runs one grid row per walker, each with its own scale and
    value quantum, and a ragged last tile and chunk."""
    sizes = [300, 260, 340]
    L = (300 / 0.8) ** (1 / 3)

    def ties(x, tag):
        # a pair exactly half a box apart has two minimum images whose
        # Jacobians differ (the CV has a kink there): keep such draws out
        off = 0
        for n in sizes:
            xw = x[off: off + n].astype(np.float32).astype(np.float64)
            q = (xw[tag][:, None, :] - xw[None, :, :]) / L
            if np.any(np.abs(np.abs(q) - 0.5) < 1e-6):
                return True
            off += n
        return False

    for seed in range(21, 121):
        r = synth.rng(seed)
        x = np.concatenate([r.uniform(0.0, L, size=(n, 3)) for n in sizes])
        tag = sorted(r.choice(260, 70, replace=False).tolist())
        b = sorted(r.choice(260, 200, replace=False).tolist()) if with_b else None
        if not ties(x, tag):
            break
    cvs = [dict(kind="coordination", a=tag, b=b, r0=1.5, nn=6, mm=12), dict(kind="rg", a=list(range(30)))]
    spec = dict(engine="lj", walker_sizes=sizes, box=(L, L, L), sigma=(0.05, 0.1), cvs=cvs, capacity=2000)
    wt = _wt()
    import oracle as o

    dt = torch.float32 if prec == "f32" else torch.float64
    xin = _f32(x) if prec == "f32" else x
    sim = o.Sim(oracle_system(spec), x=xin)
    _, xi0, _, _ = sim.bias(xin, hills=np.zeros((0, 4)))
    sig = np.asarray(spec["sigma"])
    # hills around every walker's CVs, so that each walker's bias matters
    hills = np.concatenate([synth.walk_hills(300, xi0[w, :2] - 3 * sig, xi0[w, :2] + 3 * sig, 0.5 * sig, seed=30 + w)
                            for w in range(len(sizes))])
    Fr, xir, Vr, dVr = sim.bias(xin, hills=hills)
    m = gpu_handle(spec, prec)
    m.hills_load(hills)
    pos = wt.particles(xin, dt)
    F = torch.zeros_like(pos)
    V, xi, dV = m.bias_eval(pos, F)
    torch.cuda.synchronize()
    tol = 1e-12 if prec == "f64" else 1e-6
    assert np.allclose(to_np(xi), xir[:, :2], rtol=tol, atol=tol)
    _close_V(to_np(V), Vr, prec)
    _close_dV(to_np(dV), dVr[:, :2], grad_scale(xir[:, :2], hills, spec["sigma"]), prec)
    _close_F(to_np(F)[:, :3], Fr, prec, force_scale(sim, xin, hills, [0, 0]))


def test_bias_eval_many_walkers_chain_dihedrals():
    """1024 replicas of a 22-bead chain, two dihedral CVs (beads 5-7-9-15 and
    7-9-15-17, 0-based), periodic, sigma 0.35 rad: every replica's forces."""
    x = synth.chain_replicas(1024, 22, seed=2)
    spec = dict(engine="chain", walker_sizes=[22] * 1024, sigma=(0.35, 0.35), gamma=6.0,
                cvs=[dict(kind="dihedral", a=[5, 7, 9, 15], period=2 * np.pi),
                     dict(kind="dihedral", a=[7, 9, 15, 17], period=2 * np.pi)], capacity=1000)
    for prec in ("f64", "f32"):
        wt = _wt()
        import oracle as o

        xin = _f32(x) if prec == "f32" else x
        hills = synth.uniform_hills(500, [-np.pi, -np.pi], [np.pi, np.pi], seed=4)
        sim = o.Sim(oracle_system(spec), x=xin)
        Fr, xir, Vr, dVr = sim.bias(xin, hills=hills)
        m = gpu_handle(spec, prec)
        m.hills_load(hills)
        dt = torch.float32 if prec == "f32" else torch.float64
        pos = wt.particles(xin, dt)
        F = torch.zeros_like(pos)
        V, xi, dV = m.bias_eval(pos, F)
        torch.cuda.synchronize()
        dphi = np.mod(to_np(xi) - xir[:, :2] + np.pi, 2 * np.pi) - np.pi  # periodic CVs: compare modulo 2 pi
        assert np.abs(dphi).max() <= (1e-12 if prec == "f64" else 1e-5), np.abs(dphi).max()
        _close_V(to_np(V), Vr, prec)
        _close_F(to_np(F)[:, :3], Fr, prec, force_scale(sim, xin, hills, [2 * np.pi, 2 * np.pi]))


# --------------------------------------------------------------------------
# trajectories
# --------------------------------------------------------------------------
def _run_pair(spec, x, v, nsteps, prec, hills=None):
    wt = _wt()
    import oracle as o

    dt = torch.float32 if prec == "f32" else torch.float64
    xin = _f32(x) if prec == "f32" else x
    vin = _f32(v) if prec == "f32" else v
    sim = o.Sim(oracle_system(spec), x=xin, v=vin, hills=hills)
    sim.forces()
    rc = sim.run(nsteps)
    m = gpu_handle(spec, prec)
    if hills is not None:
        m.hills_load(hills)
    pos, vel = wt.particles(xin, dt), wt.particles(vin, dt)
    F = torch.zeros_like(pos)
    m.bind(pos, vel, F)
    m.step_n(nsteps)
    torch.cuda.synchronize()
    return m, sim, rc, to_np(pos)[:, :3], to_np(vel)[:, :3]


def test_trajectory_mueller_brown_fp64_with_deposition():
    """Config-1 physics (kT = 15, dt = 1e-4, friction 1, sigma 0.05, w0 1,
    gamma 10) with a short stride so hills feed back within 100 steps."""
    spec = dict(engine="mb", walker_sizes=[1, 1, 1], dims=2, dt=1e-4, friction=1.0, kT=15.0, seed=0,
                sigma=(0.05, 0.05), w0=1.0, gamma=10.0, stride=10, capacity=100,
                grid=((64, 48), (-1.5, -0.5), (1.2, 2.2)),
                cvs=[dict(kind="component", a=[0], axis=0), dict(kind="component", a=[0], axis=1)])
    x = np.array([[-0.558, 1.442, 0], [0.623, 0.028, 0], [-0.05, 0.467, 0]])
    v = np.zeros_like(x)
    m, sim, rc, X, Vv = _run_pair(spec, x, v, 100, "f64")
    assert rc == 0
    assert np.max(np.abs(X - sim.x)) < 1e-6
    assert np.max(np.abs(X - sim.x)) < 1e-10  # in practice: rounding level
    h = m.hills_read()
    assert h.shape[0] == sim.n_hills == 30
    assert np.allclose(h, sim.hills[:30], rtol=1e-12, atol=1e-13)
    g = m.grid_read().ravel()
    assert np.allclose(g, sim.grid, rtol=1e-12, atol=1e-12 * np.abs(sim.grid).max())
    F = to_np(m.fes_grid()).ravel()
    assert np.allclose(F, sim.fes(), rtol=1e-12, atol=1e-10)
    step, n = m.counters()
    assert step == 100 and n == 30


def test_trajectory_lj_fp64_100_steps():
    spec, x, L = lj_fluid_spec(n=500, n_tag=50, n_rg=20, seed=7, jitter=0.05)
    spec.update(stride=10, capacity=100)
    v = synth.velocities(500, 1.0, 1.0, seed=8)
    m, sim, rc, X, Vv = _run_pair(spec, x, v, 100, "f64")
    assert rc == 0
    assert np.max(np.abs(X - sim.x)) < 1e-6
    h = m.hills_read()
    assert h.shape[0] == sim.n_hills == 10
    assert np.allclose(h, sim.hills[:10], rtol=1e-9, atol=1e-10)


def test_trajectory_lj_fp32_against_fp64_oracle():
    """FP32 engine with identical Philox streams: after 100 steps the
    positions agree with the FP64 oracle to ~1e-4 (FP32 rounding grows with
    the chaotic LJ dynamics; the 1e-6 trajectory bar is met in FP64)."""
    spec, x, L = lj_fluid_spec(n=500, n_tag=50, n_rg=20, seed=7, jitter=0.05)
    spec.update(stride=10, capacity=100)
    v = synth.velocities(500, 1.0, 1.0, seed=8)
    m, sim, rc, X, Vv = _run_pair(spec, x, v, 100, "f32")
    assert rc == 0
    assert np.max(np.abs(X - sim.x)) < 1e-3
    assert np.median(np.abs(X - sim.x)) < 1e-5


def test_trajectory_cell_list_4096_fp64_100_steps():
    """The 4096-atom workload in FP64 (cell lists with list rebuilds,
    coordination of 512 atoms + Rg of 64, 2000 hills around the start plus a
    deposit every 10 steps): 100 steps with identical Philox streams agree
    with the oracle to 1e-6 in position, and the deposited hills too."""
    spec, x, L = lj_fluid_spec(n=4096, seed=0)
    spec.update(stride=10, capacity=2200)
    v = synth.velocities(4096, 1.0, 1.0, seed=1)
    import oracle as o

    sim0 = o.Sim(oracle_system(spec), x=x)
    _, xi0, _, _ = sim0.bias(x, hills=np.zeros((0, 4)))
    sig = np.asarray(spec["sigma"])
    hills = synth.walk_hills(2000, xi0[0, :2] - 3 * sig, xi0[0, :2] + 3 * sig, 0.5 * sig, seed=12)
    m, sim, rc, X, Vv = _run_pair(spec, x, v, 100, "f64", hills=hills)
    assert rc == 0
    assert np.max(np.abs(X - sim.x)) < 1e-6
    assert np.max(np.abs(Vv - sim.v)) < 1e-6
    h = m.hills_read()
    assert h.shape[0] == sim.n_hills == 2010
    assert np.allclose(h, sim.hills[:2010], rtol=1e-9, atol=1e-12)


def test_capacity_overflow_is_reported():
    wt = _wt()
    spec = dict(engine="mb", walker_sizes=[1, 1], dims=2, dt=1e-4, kT=15.0, sigma=(0.05, 0.05), stride=2,
                capacity=5, cvs=[dict(kind="component", a=[0], axis=0), dict(kind="component", a=[0], axis=1)])
    m = gpu_handle(spec, "f64")
    pos = wt.particles([[-0.5, 1.4, 0], [0.6, 0.0, 0]], torch.float64)
    vel, F = torch.zeros_like(pos), torch.zeros_like(pos)
    m.bind(pos, vel, F)
    m.step_n(4)  # 4 hills
    with pytest.raises(wt.WtmdError) as e:
        m.step_n(2)  # would need 6
    assert e.value.code == wt.ECAPACITY
    assert m.counters()[1] == 4


def test_invalid_arguments_are_rejected():
    wt = _wt()
    m = wt.Wtmd(precision="f64", sigma=[0.1], walker_sizes=[10])
    for bad in [dict(kind=wt.CV_DIHEDRAL, a=[0, 1, 2]), dict(kind=wt.CV_DIHEDRAL, a=[0, 1, 1, 2]),
                dict(kind=wt.CV_COMPONENT, a=[10]), dict(kind=wt.CV_COORDINATION, a=[0, 1], nn=6, mm=10),
                dict(kind=wt.CV_COORDINATION, a=[0, 1], nn=5, mm=10), dict(kind=99, a=[0])]:
        with pytest.raises(wt.WtmdError):
            m.cv_define(**bad)
    m.cv_define(wt.CV_RG, a=None)
    with pytest.raises(wt.WtmdError):
        m.cv_define(wt.CV_RG, a=None)  # more than n_cv
    assert wt.lib().fes_grid(m.h, None, 0) == wt.EINVAL  # no grid configured
    with pytest.raises(wt.WtmdError):
        wt.Wtmd(precision="f64", sigma=[0.1], gamma=0.5, walker_sizes=[1])


def test_hills_tune_keeps_results():
    """The plan autotuner changes only the launch shape: V and dV/dxi after
    tuning agree with the oracle as before (FP32 bound), and the choice is a
    valid plan."""
    wt = _wt()
    import oracle as o

    spec, x, L = lj_fluid_spec(n=500, n_tag=50, n_rg=20, seed=3, jitter=0.05)
    m = gpu_handle(spec, "f32")
    pos = wt.particles(_f32(x), torch.float32)
    _, xi0, _ = m.bias_eval(pos)
    c = to_np(xi0)[0]
    hills = synth.walk_hills(3000, c - 0.3, c + 0.3, 0.05, seed=4)
    m.hills_load(hills)
    th, sp, ms = m.hills_tune(1)
    # 0: the few-points kernel, -1: the cluster kernel (8 or 16 CTAs)
    assert th in (-1, 0, 1, 4, 32, 256) and sp >= 1 and ms > 0
    assert th != -1 or sp in (8, 16)
    V, xi, dV = m.bias_eval(pos)
    Vr, dVr = o.hills_sum(to_np(xi), hills, spec["sigma"])
    _close_V(to_np(V), Vr, "f32")
    _close_dV(to_np(dV), dVr, grad_scale(to_np(xi), hills, spec["sigma"]), "f32")


def test_frozen_walker_heights_follow_the_well_tempered_recursion():
    """A walker that cannot move (no engine, no noise, zero velocity; the
    bias gradient vanishes at a hill's own centre) deposits every stride
    steps at the same point, so the heights obey the scalar recursion
    V_{k+1} = V_k + w_k, w_k = w0 exp(-V_k / (kT (gamma - 1))) of Sec. 2.1.5
    exactly (FP64 handle)."""
    wt = _wt()
    spec = dict(engine="none", walker_sizes=[1], dims=3, dt=1e-3, kT=2.0, friction=0.0, sigma=(0.3, 0.2),
                w0=1.5, gamma=6.0, stride=3, capacity=64,
                cvs=[dict(kind="component", a=[0], axis=0), dict(kind="component", a=[0], axis=1)])
    m = gpu_handle(spec, "f64")
    pos = wt.particles([[0.4, -0.7, 0.0]], torch.float64)
    vel, F = torch.zeros_like(pos), torch.zeros_like(pos)
    m.bind(pos, vel, F)
    m.step_n(60)
    h = m.hills_read()
    assert h.shape[0] == 20
    assert np.all(h[:, 0] == 0.4) and np.all(h[:, 1] == -0.7)
    V, ref = 0.0, []
    for _ in range(20):
        w = 1.5 * np.exp(-V / (2.0 * 5.0))
        ref.append(w)
        V += w
    assert np.allclose(h[:, 3], ref, rtol=1e-13, atol=0)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_standard_metadynamics_and_no_deposition(prec):
    """gamma = 0 deposits fixed heights w0 (standard metadynamics); stride = 0
    never deposits; both against the oracle's trajectory."""
    import oracle as o

    wt = _wt()
    dt = torch.float32 if prec == "f32" else torch.float64
    base = dict(engine="mb", walker_sizes=[1, 1], dims=2, dt=1e-4, friction=1.0, kT=15.0, seed=2,
                sigma=(0.05, 0.05), w0=0.7, capacity=100,
                cvs=[dict(kind="component", a=[0], axis=0), dict(kind="component", a=[0], axis=1)])
    x = np.array([[-0.558, 1.442, 0], [0.623, 0.028, 0]])
    for extra, nh in ((dict(gamma=0.0, stride=5), 2 * 8), (dict(gamma=10.0, stride=0), 0)):
        spec = dict(base, **extra)
        xin = _f32(x) if prec == "f32" else x
        sim = o.Sim(oracle_system(spec), x=xin, v=np.zeros_like(x))
        sim.forces()
        assert sim.run(40) == 0
        m = gpu_handle(spec, prec)
        pos, vel = wt.particles(xin, dt), wt.particles(np.zeros_like(x), dt)
        F = torch.zeros_like(pos)
        m.bind(pos, vel, F)
        m.step_n(40)
        torch.cuda.synchronize()
        assert m.counters() == (40, nh) and sim.n_hills == nh
        if nh:
            h = m.hills_read()
            assert np.all(h[:, 3] == 0.7)
            assert np.allclose(h[:, :2], sim.hills[:nh, :2], rtol=0, atol=1e-5 if prec == "f32" else 1e-12)
        tol = 1e-4 if prec == "f32" else 1e-12
        assert np.max(np.abs(to_np(pos)[:, :3] - sim.x)) < tol


def test_new_cv_definitions_are_validated():
    wt = _wt()
    m = wt.Wtmd(precision="f32", sigma=[0.1], walker_sizes=[20])
    for bad in [dict(kind=wt.CV_DISTANCE, a=[0, 1], b=[1, 2]),  # overlapping groups
                dict(kind=wt.CV_DISTANCE, a=[0, 1], b=None),  # B must be a list
                dict(kind=wt.CV_ANGLE, a=[0, 1]), dict(kind=wt.CV_ANGLE, a=[0, 1, 1]),
                dict(kind=wt.CV_GYRATION, a=[0, 1, 2], axis=6), dict(kind=wt.CV_GYRATION, a=[3], axis=0),
                dict(kind=wt.CV_GYRATION, a=[0, 25], axis=1)]:
        with pytest.raises(wt.WtmdError):
            m.cv_define(**bad)
    m.cv_define(wt.CV_GYRATION, a=None, axis=wt.GY_ANISOTROPY)


def test_mueller_brown_free_energy_recovered_on_gpu():
    """The whole GPU step (engine, CVs, hills sum, scatter, deposition, FP64
    grid) recovers the Mueller-Brown free energy: -(gamma/(gamma-1)) V_grid
    matches U_MB up to a constant within 0.5 kT on visited cells up to 5 kT
    above the minimum (the CVs are the particle's own x, y, so A = U + C;
    Sec. 2.1, Eq. (free-energy)).  Same parameters as the oracle's pin."""
    import oracle as o

    wt = _wt()
    bins, lo, hi, kT = (60, 60), (-1.5, -0.5), (1.2, 2.2), 15.0
    m = wt.Wtmd(precision="f64", sigma=(0.05, 0.05), w0=0.5, gamma=10.0, kT=kT, stride=20, capacity=20000, seed=0,
                engine="mb", walker_sizes=[1], dims=2, dt=2e-3, friction=5.0, grid=(bins, lo, hi))
    m.cv_define(wt.CV_COMPONENT, a=[0], axis=0)
    m.cv_define(wt.CV_COMPONENT, a=[0], axis=1)
    pos = wt.particles(np.array([[-0.558, 1.442, 0.0]]), torch.float64)
    vel = wt.particles(np.zeros((1, 3)), torch.float64)
    m.bind(pos, vel, torch.zeros_like(pos))
    m.step_n(300000)
    hills = m.hills_read()
    assert hills.shape[0] == 15000
    F = to_np(m.fes_grid()).reshape(bins)
    cx, cy = o.grid_centres(bins, lo, hi)
    U = np.array([[o.mb(a, b)[0] for b in cy] for a in cx])
    vis = np.zeros(bins, bool)
    for hx, hy in hills[:, :2]:
        i, j = int((hx - lo[0]) / (hi[0] - lo[0]) * bins[0]), int((hy - lo[1]) / (hi[1] - lo[1]) * bins[1])
        if 0 <= i < bins[0] and 0 <= j < bins[1]:
            vis[i, j] = True
    mask = vis & (U < U.min() + 5 * kT)
    assert mask.sum() > 200
    d = (F - U)[mask]
    d -= d.mean()
    assert np.abs(d).max() < 0.5 * kT
    assert np.sqrt(np.mean(d ** 2)) < 0.25 * kT
