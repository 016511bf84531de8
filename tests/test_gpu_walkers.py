"""Persistent multi-walker step (one cooperative launch per MD step over all
walkers) and its autotuner, against the FP64 oracle and against the generic
FP32 launch sequence on the same handle.

Workload: 37 Lennard-Jones clusters in open space, sizes log-uniform in
[38, 600] atoms (ragged: several target tiles per walker and a partial last
tile), compact FCC-site clusters at rho* = 0.9, T* = 0.3, CVs = mean
coordination number (all atoms, r0 = 1.5, n = 6, m = 12) and Rg (all atoms),
hills shared by all walkers (multiple walkers, Sec. 2)."""
import numpy as np
import pytest

import synth
from systems import gpu_handle, oracle_system, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

W = 37


def _wt():
    import paper_2301_04835_b300 as wt
    return wt


def cluster_spec(W=W, lo=38, hi=600, seed=0, capacity=4000, grid=None, stride=5):
    sizes = synth.log_uniform_sizes(W, lo, hi, seed)
    x = np.concatenate([synth.fcc_cluster(int(n), 0.9, seed=100 + w) for w, n in enumerate(sizes)])
    v = synth.velocities(x.shape[0], 0.3, 1.0, seed=seed + 1)
    spec = dict(engine="lj", walker_sizes=[int(n) for n in sizes], box=(0, 0, 0), dt=0.005, kT=0.3, friction=1.0,
                sigma=(0.2, 0.05), gamma=8.0, w0=0.3, stride=stride, capacity=capacity, seed=seed, grid=grid,
                cvs=[dict(kind="coordination", r0=1.5, nn=6, mm=12), dict(kind="rg")])
    return spec, x, v


def walker_cvs(spec, x):
    import oracle as o

    sysd = oracle_system(spec)
    out, off = [], 0
    for n in spec["walker_sizes"]:
        out.append([o.cv_eval(cv, x[off: off + n], [0, 0, 0])[0] for cv in sysd.cvs])
        off += n
    return np.asarray(out)


def shared_hills(spec, x, H=1500, seed=5):
    xi = walker_cvs_box(spec, x)
    return synth.uniform_hills(H, xi.min(0) - 0.3, xi.max(0) + 0.3, seed=seed, w_range=(0.01, 0.3))


def _f32(a):
    return np.asarray(a, np.float32).astype(np.float64)


def _setup(spec, x, v, hills, persistent):
    wt = _wt()
    m = gpu_handle(spec, "f32")
    if hills is not None:
        m.hills_load(hills)
    pos, vel = wt.particles(_f32(x), torch.float32), wt.particles(_f32(v), torch.float32)
    F = torch.zeros_like(pos)
    m.bind(pos, vel, F)
    if persistent:
        m.walkers_persistent(True)
    return m, pos, vel, F


def test_persistent_step_matches_generic_fp32_path():
    """Same handle set-up, same Philox streams: one step of the persistent
    kernel against one step of the generic launch sequence (forces, CVs, hills
    sum, deposit).  Both are FP32; only summation orders differ."""
    spec, x, v = cluster_spec(stride=1)
    hills = shared_hills(spec, x)
    ms = [_setup(spec, x, v, hills, p) for p in (False, True)]
    for m, *_ in ms:
        m.step_n(3)
    torch.cuda.synchronize()
    (mg, pg, vg, Fg), (mp, pp, vp, Fp) = ms
    assert mg.counters() == mp.counters() == (3, 1500 + 3 * W)
    assert torch.allclose(pp, pg, rtol=0, atol=2e-6)
    assert torch.allclose(vp, vg, rtol=0, atol=1e-4)
    dF = torch.linalg.norm(Fp - Fg) / torch.linalg.norm(Fg)
    assert dF < 1e-5, float(dF)
    hg, hp = mg.hills_read(), mp.hills_read()
    assert np.allclose(hp[:, :3], hg[:, :3], rtol=1e-5, atol=1e-6)
    assert np.allclose(hp[:, 3], hg[:, 3], rtol=1e-4)


def test_persistent_trajectory_against_fp64_oracle():
    """20 steps with a deposit every 5 steps: positions within the FP32 bar
    of the FP64 oracle; the deposited hills (centres = CVs, heights =
    w0 exp(-V/(kT(gamma-1))), Eq. 4) agree to FP32 accuracy."""
    import oracle as o

    spec, x, v = cluster_spec()
    hills = shared_hills(spec, x)
    sim = o.Sim(oracle_system(spec), x=_f32(x), v=_f32(v), hills=hills)
    sim.forces()
    assert sim.run(20) == 0
    m, pos, vel, F = _setup(spec, x, v, hills, True)
    m.step_n(20)
    torch.cuda.synchronize()
    X = to_np(pos)[:, :3]
    assert np.max(np.abs(X - sim.x)) < 1e-3
    assert np.median(np.abs(X - sim.x)) < 1e-5
    assert m.counters() == (20, 1500 + 4 * W)
    h = m.hills_read()
    ref = sim.hills[: sim.n_hills]
    assert h.shape[0] == sim.n_hills
    assert np.allclose(h[1500:, :2], ref[1500:, :2], rtol=1e-4, atol=1e-4)
    assert np.allclose(h[1500:, 3], ref[1500:, 3], rtol=1e-3)


def test_persistent_grid_update_against_oracle():
    """The FP64 bias grid, updated after each persistent step that deposits."""
    import oracle as o

    grid = ((32, 24), (7.0, 1.0), (15.0, 4.0))
    spec, x, v = cluster_spec(W=9, hi=300, grid=grid)
    sim = o.Sim(oracle_system(spec), x=_f32(x), v=_f32(v))
    sim.forces()
    assert sim.run(10) == 0
    m, pos, vel, F = _setup(spec, x, v, None, True)
    m.step_n(10)
    torch.cuda.synchronize()
    g = m.grid_read().ravel()
    assert np.allclose(g, sim.grid, rtol=1e-3, atol=1e-4 * np.abs(sim.grid).max())


def test_persistent_step_is_deterministic():
    spec, x, v = cluster_spec(stride=2)
    hills = shared_hills(spec, x)
    runs = []
    for _ in range(2):
        m, pos, vel, F = _setup(spec, x, v, hills, True)
        m.step_n(6)
        torch.cuda.synchronize()
        runs.append((pos.clone(), vel.clone(), F.clone(), m.hills_read()))
    assert all(torch.equal(a, b) for a, b in zip(runs[0][:3], runs[1][:3]))
    assert np.array_equal(runs[0][3], runs[1][3])


def test_autotune_leaves_state_and_picks_a_valid_plan():
    spec, x, v = cluster_spec(stride=1)
    hills = shared_hills(spec, x)
    m, pos, vel, F = _setup(spec, x, v, hills, True)
    m.step_n(2)
    torch.cuda.synchronize()
    before = (pos.clone(), vel.clone(), F.clone(), m.counters(), m.hills_read())
    T, bps, hm = m.autotune(steps=2)
    torch.cuda.synchronize()
    assert T in (32, 64, 128, 256) and 1 <= bps <= 4 and hm in (1, 2)
    assert torch.equal(pos, before[0]) and torch.equal(vel, before[1]) and torch.equal(F, before[2])
    assert m.counters() == before[3]
    assert np.array_equal(m.hills_read(), before[4])
    # the tuned plan steps on as the default plan does, to FP32 rounding
    m.step_n(3)
    m2, pos2, *_ = _setup(spec, x, v, hills, True)
    m2.step_n(5)
    torch.cuda.synchronize()
    assert m.counters() == m2.counters()
    assert torch.allclose(pos, pos2, rtol=0, atol=1e-5)


def test_persistent_rejects_unsupported_handles():
    wt = _wt()
    spec, x, v = cluster_spec(W=3, hi=100)
    m = gpu_handle(spec, "f64")
    with pytest.raises(wt.WtmdError):
        m.walkers_persistent(True)
    m = gpu_handle(dict(spec, cvs=[dict(kind="dihedral", a=[0, 1, 2, 3], period=2 * np.pi), dict(kind="rg")]),
                   "f32")
    with pytest.raises(wt.WtmdError):
        m.walkers_persistent(True)
    m = gpu_handle(spec, "f32")
    with pytest.raises(wt.WtmdError):
        m.autotune()
    m.surrogate_set(0, False)  # surrogate on (network inactive): the persistent step refuses
    with pytest.raises(wt.WtmdError):
        m.walkers_persistent(True)
    m.surrogate(False)
    m.walkers_persistent(True)
    with pytest.raises(wt.WtmdError):
        m.surrogate(True)


def test_full_size_cluster_workload_sampled_against_oracle():
    """The 256-cluster workload at full size (sizes 38..2048 atoms, 2e5
    shared hills, FP64 grid) in the benchmark's launch configuration
    (persistent step, autotuned plan), one step with a deposit: for sampled
    walkers (smallest, largest and four seeded others) the deposited CVs, the
    well-tempered heights and the total forces agree with the FP64 oracle
    evaluated at the GPU's own positions."""
    import oracle as o
    from test_gpu_parity import force_scale

    wt = _wt()
    sizes, x = synth.lj_clusters(256, 38, 2048, 0.9, seed=0)
    sizes = [int(n) for n in sizes]
    v = synth.velocities(x.shape[0], 0.3, 1.0, seed=7)
    sig = np.array([0.2, 0.01])
    spec = dict(engine="lj", walker_sizes=sizes, box=(0, 0, 0), dt=0.005, kT=0.3, friction=1.0, sigma=tuple(sig),
                gamma=8.0, w0=0.3, stride=1, capacity=200000 + 4096, seed=0,
                cvs=[dict(kind="coordination", r0=1.5, nn=6, mm=12), dict(kind="rg", flags=wt.CV_INTENSIVE)])
    m0 = gpu_handle(dict(spec, capacity=16), "f32")
    _, xi0, _ = m0.bias_eval(wt.particles(x, torch.float32))
    xi0 = to_np(xi0)
    lo, hi = xi0.min(0) - 3 * sig, xi0.max(0) + 3 * sig
    hills = synth.walk_hills(200000, lo, hi, 0.5 * sig, seed=8, w_range=(0.01, 0.3))
    grid = ((256, 256), tuple(lo - 10 * sig), tuple(hi + 10 * sig))
    m, pos, vel, F = _setup(dict(spec, grid=grid), x, v, hills, True)
    m.autotune(steps=2)
    m.step_n(1)
    torch.cuda.synchronize()
    X, Fg = to_np(pos)[:, :3], to_np(F)[:, :3]
    h = m.hills_read()
    assert h.shape[0] == 200000 + 256
    dep = h[200000:]
    off = np.concatenate([[0], np.cumsum(sizes)])
    r = np.random.default_rng(3)
    sample = sorted({int(np.argmin(sizes)), int(np.argmax(sizes)), *r.choice(256, 4, replace=False).tolist()})
    inv_dT = 1.0 / (0.3 * 7.0)
    for w in sample:
        n = sizes[w]
        xw = X[off[w]: off[w + 1]]
        sub = dict(spec, walker_sizes=[n])
        sim = o.Sim(oracle_system(sub), x=xw, hills=hills)
        Fr = sim.forces()
        _, xi_r, _, _ = sim.bias(xw)
        assert np.all(np.abs(dep[w, :2] - xi_r[0, :2]) <= 1e-5 * np.abs(xi_r[0, :2])), (w, dep[w], xi_r[0])
        Vr, _ = o.hills_sum(dep[w, :2][None, :], hills, tuple(sig))
        h_r = 0.3 * np.exp(-Vr[0] * inv_dT)
        assert abs(dep[w, 3] - h_r) <= h_r * 2e-5 * Vr[0] * inv_dT + 1e-12, (w, dep[w, 3], h_r)
        Fs = force_scale(sim, xw, hills, [0.0, 0.0])
        dF = np.linalg.norm(Fg[off[w]: off[w + 1]] - Fr)
        assert dF <= 1e-5 * (np.linalg.norm(Fr) + np.linalg.norm(Fs)), (w, n, dF / np.linalg.norm(Fr))


def periodic_spec(W=6, lo=120, hi=360, L=8.5, seed=0, stride=5, nn=6, capacity=4000):
    """W walkers, each a Lennard-Jones fluid in its own periodic box of edge
    L (ragged sizes, log-uniform in [lo, hi]: rho* 0.2-0.6), T* = 1, seeded
    random positions at least 0.9 sigma apart; CVs as for the clusters."""
    sizes = synth.log_uniform_sizes(W, lo, hi, seed)
    x = np.concatenate([synth.random_liquid(int(n), L, seed=300 + w) for w, n in enumerate(sizes)])
    v = synth.velocities(x.shape[0], 1.0, 1.0, seed=seed + 1)
    spec = dict(engine="lj", walker_sizes=[int(n) for n in sizes], box=(L, L, L), dt=0.004, kT=1.0, friction=1.0,
                sigma=(0.2, 0.05), gamma=8.0, w0=0.3, stride=stride, capacity=capacity, seed=seed,
                cvs=[dict(kind="coordination", r0=1.5, nn=nn, mm=2 * nn), dict(kind="rg")])
    return spec, x, v


def _dpos(X, Y, L):
    D = X - Y
    return D - L * np.rint(D / L)


@pytest.mark.parametrize("nn", [6, 10])
def test_persistent_periodic_boxes_match_generic_and_oracle(nn):
    """Walkers in periodic boxes (minimum-image pairs and Rg members): three
    steps with a deposit each against the generic FP32 launch sequence, and a
    20-step trajectory against the FP64 oracle.  n = 10 takes the kernel with
    the exponent read at run time."""
    import oracle as o

    spec, x, v = periodic_spec(stride=1, nn=nn)
    L = spec["box"][0]
    hills = shared_hills(spec, x)
    ms = [_setup(spec, x, v, hills, p) for p in (False, True)]
    for m, *_ in ms:
        m.step_n(3)
    torch.cuda.synchronize()
    (mg, pg, vg, Fg), (mp, pp, vp, Fp) = ms
    W = len(spec["walker_sizes"])
    assert mg.counters() == mp.counters() == (3, 1500 + 3 * W)
    assert np.abs(_dpos(to_np(pp)[:, :3], to_np(pg)[:, :3], L)).max() < 2e-6
    assert torch.allclose(vp, vg, rtol=0, atol=1e-4)
    assert torch.isfinite(Fp).all()
    dF = torch.linalg.norm(Fp - Fg) / torch.linalg.norm(Fg)
    assert dF < 1e-5, float(dF)
    hg, hp = mg.hills_read(), mp.hills_read()
    assert np.allclose(hp[:, :3], hg[:, :3], rtol=1e-5, atol=1e-6)
    assert np.allclose(hp[:, 3], hg[:, 3], rtol=1e-4)

    spec, x, v = periodic_spec(stride=5, nn=nn)
    sim = o.Sim(oracle_system(spec), x=_f32(x), v=_f32(v), hills=hills)
    sim.forces()
    assert sim.run(20) == 0
    m, pos, vel, F = _setup(spec, x, v, hills, True)
    m.step_n(20)
    torch.cuda.synchronize()
    D = np.abs(_dpos(to_np(pos)[:, :3], sim.x, L))
    assert D.max() < 1e-3 and np.median(D) < 1e-5, (D.max(), np.median(D))
    assert m.counters() == (20, 1500 + 4 * W)
    h, ref = m.hills_read(), sim.hills[: sim.n_hills]
    assert np.allclose(h[1500:, :2], ref[1500:, :2], rtol=1e-4, atol=1e-4)
    assert np.allclose(h[1500:, 3], ref[1500:, 3], rtol=1e-3)


def test_persistent_high_exponent_open_clusters():
    """Open clusters with n = 10, m = 20: the padding point of an odd-sized
    walker and each target's left-out self pair lie 1e4 away, where y^h
    exceeds FP32's range; the run-time-exponent kernel caps it, so forces
    stay finite and match the generic launch sequence."""
    spec, x, v = cluster_spec(W=9, hi=300, stride=1)
    spec["cvs"][0] = dict(kind="coordination", r0=1.5, nn=10, mm=20)
    hills = shared_hills(spec, x)
    ms = [_setup(spec, x, v, hills, p) for p in (False, True)]
    for m, *_ in ms:
        m.step_n(2)
    torch.cuda.synchronize()
    (mg, pg, vg, Fg), (mp, pp, vp, Fp) = ms
    assert torch.isfinite(Fp).all() and torch.isfinite(pp).all()
    assert torch.allclose(pp, pg, rtol=0, atol=2e-6)
    dF = torch.linalg.norm(Fp - Fg) / torch.linalg.norm(Fg)
    assert dF < 1e-5, float(dF)


def test_persistent_umbrella_windows_periodic_against_oracle():
    """Umbrella windows as walkers of the persistent launch (Sec. 2.1.1
    harmonic bias, Sec. 2.1.2 umbrella sampling): one window per periodic
    walker on (coordination, Rg), centres offset from the starting CVs.
    Against the generic launch sequence (forces, window sums) and against
    the FP64 oracle's run with the same windows (trajectory, window means,
    sample count, umbrella integration); no hill is deposited."""
    import oracle as o

    spec, x, v = periodic_spec(stride=5)
    L = spec["box"][0]
    W = len(spec["walker_sizes"])
    xi0 = walker_cvs_box(spec, x)
    centres = xi0 + np.array([0.4, -0.2])[None, :] * np.sign(np.arange(W) % 2 - 0.5)[:, None]
    k = (30.0, 8.0)

    def gpu(persistent):
        m, pos, vel, F = _setup(spec, x, v, None, False)
        m.harmonic(k, centres)
        if persistent:
            m.walkers_persistent(True)
        return m, pos, vel, F

    ms = [gpu(p) for p in (False, True)]
    for m, *_ in ms:
        m.step_n(3)
    torch.cuda.synchronize()
    (mg, pg, vg, Fg), (mp, pp, vp, Fp) = ms
    assert np.abs(_dpos(to_np(pp)[:, :3], to_np(pg)[:, :3], L)).max() < 2e-6
    dF = torch.linalg.norm(Fp - Fg) / torch.linalg.norm(Fg)
    assert dF < 1e-5, float(dF)
    (mean_g, n_g), (mean_p, n_p) = mg.umbrella_stats(), mp.umbrella_stats()
    assert n_g == n_p == 3
    np.testing.assert_allclose(mean_p, mean_g, rtol=1e-6)

    osys = oracle_system(spec)
    osys.umb_k, osys.umb_centres = k, centres
    sim = o.Sim(osys, x=_f32(x), v=_f32(v))
    sim.forces()
    assert sim.run(30) == 0
    m, pos, vel, F = gpu(True)
    m.step_n(30)
    torch.cuda.synchronize()
    D = np.abs(_dpos(to_np(pos)[:, :3], sim.x, L))
    assert D.max() < 1e-3 and np.median(D) < 1e-5, (D.max(), np.median(D))
    assert m.counters()[1] == 0  # windows deposit no hills
    mean, n = m.umbrella_stats()
    assert n == sim.n_samples == 30
    om, og, oA = sim.umbrella()
    # window means to the trajectories' FP32 agreement (as the deposited CVs
    # of the metadynamics runs)
    np.testing.assert_allclose(mean, om, rtol=1e-4, atol=1e-4)
    g, A = m.umbrella_integrate()
    kk = np.asarray(k)
    # mean force k (mean - centre): the means' error times k
    assert np.all(np.abs(g - og) <= kk[None, :] * 1e-4 * (1 + np.abs(om)) + 1e-6 * np.abs(og))
    assert np.all(np.isfinite(A))


def test_persistent_grid_read_bias_against_generic_and_oracle():
    """The bias read from the FP64 grid inside the persistent launch (Sec.
    2.1.5): the grid is updated after each step that deposits and read back
    at the next step's CVs.  Against the generic launch sequence with the
    same bias source (forces, hills, grid) and against the FP64 oracle run
    with the grid-read bias (trajectory and grid)."""
    import oracle as o

    grid = ((32, 24), (7.0, 1.0), (15.0, 4.0))
    spec, x, v = cluster_spec(W=9, hi=300, grid=grid, stride=2)
    spec["bias_grid"] = True
    ms = [_setup(spec, x, v, None, p) for p in (False, True)]
    for m, *_ in ms:
        m.step_n(8)
    torch.cuda.synchronize()
    (mg, pg, vg, Fg), (mp, pp, vp, Fp) = ms
    assert mg.counters() == mp.counters() == (8, 4 * 9)
    assert torch.allclose(pp, pg, rtol=0, atol=2e-6)
    dF = torch.linalg.norm(Fp - Fg) / torch.linalg.norm(Fg)
    assert dF < 1e-5, float(dF)
    assert np.allclose(mp.grid_read(), mg.grid_read(), rtol=1e-5, atol=1e-7)
    xi_g, xi_p = mg.hills_read()[:, :2], mp.hills_read()[:, :2]
    assert np.allclose(xi_p, xi_g, rtol=1e-5, atol=1e-6)

    sim = o.Sim(oracle_system(spec), x=_f32(x), v=_f32(v))
    sim.forces()
    assert sim.run(12) == 0
    m, pos, vel, F = _setup(spec, x, v, None, True)
    m.step_n(12)
    torch.cuda.synchronize()
    X = to_np(pos)[:, :3]
    assert np.max(np.abs(X - sim.x)) < 1e-3 and np.median(np.abs(X - sim.x)) < 1e-5
    assert m.counters() == (12, 6 * 9)
    g = m.grid_read().ravel()
    assert np.allclose(g, sim.grid, rtol=1e-3, atol=1e-4 * np.abs(sim.grid).max())


def walker_cvs_box(spec, x):
    import oracle as o

    sysd = oracle_system(spec)
    out, off = [], 0
    for n in spec["walker_sizes"]:
        out.append([o.cv_eval(cv, x[off: off + n], list(spec["box"]))[0] for cv in sysd.cvs])
        off += n
    return np.asarray(out)
