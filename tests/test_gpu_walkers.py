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
    xi = walker_cvs(spec, x)
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
    m = gpu_handle(dict(spec, box=(20.0, 20.0, 20.0)), "f32")
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
