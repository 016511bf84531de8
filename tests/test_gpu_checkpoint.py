"""Checkpoint / restart (the paper lists restarts as still to be added to
PySAGES, Conclusion) through the C ABI.

A run saved at step t and resumed, in a fresh handle or in the same one, must
reproduce the uninterrupted run bitwise: the thermostat noise is keyed by
(seed, step, particle) and the checkpoint holds the raw bytes of the hills,
grid, counters and particle arrays.  The resumed runs cross deposits, grid
updates and neighbour-list rebuilds.
"""
import ctypes as C

import numpy as np
import pytest

from systems import gpu_handle, lj_fluid_spec, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _wt():
    import paper_2301_04835_b300 as wt
    return wt


def _state(m, pos, vel, F):
    torch.cuda.synchronize()
    return dict(pos=pos.cpu().numpy().copy(), vel=vel.cpu().numpy().copy(), F=F.cpu().numpy().copy(),
                hills=m.hills_read(), grid=m.grid_read() if m.grid_shape else None, counters=m.counters())


def _same(a, b):
    for k in ("pos", "vel", "F", "hills"):
        assert a[k].shape == b[k].shape and np.array_equal(a[k], b[k]), k
    if a["grid"] is not None:
        assert np.array_equal(a["grid"], b["grid"])
    assert a["counters"] == b["counters"]


def _resume_bitwise(spec, x, v, prec, t_save, t_more):
    wt = _wt()
    dt = torch.float32 if prec == "f32" else torch.float64
    m = gpu_handle(spec, prec)
    pos, vel = wt.particles(x, dt), wt.particles(v, dt)
    F = torch.zeros_like(pos)
    m.bind(pos, vel, F)
    m.step_n(t_save)
    blob = m.checkpoint()
    n = C.c_int64()
    assert wt.lib().wtmd_checkpoint_size(m.h, C.byref(n)) == 0 and n.value == len(blob)
    m.step_n(t_more)
    ref = _state(m, pos, vel, F)
    assert ref["counters"][0] == t_save + t_more

    # a fresh handle with fresh arrays
    m2 = gpu_handle(spec, prec)
    p2, v2 = wt.particles(np.zeros_like(x), dt), wt.particles(np.zeros_like(x), dt)
    F2 = torch.zeros_like(p2)
    m2.bind(p2, v2, F2)
    m2.restore(blob)
    assert m2.counters()[0] == t_save
    m2.step_n(t_more)
    _same(ref, _state(m2, p2, v2, F2))

    # the same handle, rewound
    m.restore(blob)
    m.step_n(t_more)
    _same(ref, _state(m, pos, vel, F))
    return blob


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_lj_resume_is_bitwise(prec):
    """500-atom LJ fluid (cell list, Verlet lists), coordination + Rg CVs,
    hills every 20 steps into an FP64 grid; saved at step 60, 80 more."""
    spec, x, L = lj_fluid_spec(n=500, n_tag=37, n_rg=20, seed=4, jitter=0.1, capacity=4000)
    spec.update(stride=20, w0=0.5, grid=((32, 24), (0.0, 0.5), (40.0, 3.0)))
    from synth import velocities

    v = velocities(500, 1.0, 1.0, seed=9)
    _resume_bitwise(spec, x, v, prec, 60, 80)


def test_mueller_brown_grid_sourced_resume_is_bitwise():
    """Three Mueller-Brown walkers with the bias read from the grid (FP64):
    the grid itself, not the hill list, feeds the forces and heights."""
    wt = _wt()
    spec = dict(engine="mb", walker_sizes=[1, 1, 1], dims=2, dt=1e-4, friction=1.0, kT=15.0, seed=0,
                sigma=(0.05, 0.05), w0=1.0, gamma=10.0, stride=10, capacity=200,
                grid=((108, 96), (-1.5, -0.5), (1.2, 2.2)), bias_grid=True,
                cvs=[dict(kind="component", a=[0], axis=0), dict(kind="component", a=[0], axis=1)])
    x = np.array([[-0.558, 1.442, 0], [0.623, 0.028, 0], [-0.05, 0.467, 0]])
    _resume_bitwise(spec, x, np.zeros_like(x), "f64", 150, 250)


def test_checkpoint_is_validated():
    wt = _wt()
    spec, x, L = lj_fluid_spec(n=500, n_tag=37, n_rg=20, seed=4, jitter=0.1, capacity=4000)
    m = gpu_handle(spec, "f32")
    with pytest.raises(wt.WtmdError):
        m.checkpoint()  # nothing bound
    pos = wt.particles(x, torch.float32)
    m.bind(pos, torch.zeros_like(pos), torch.zeros_like(pos))
    blob = m.checkpoint()
    with pytest.raises(wt.WtmdError):
        m.restore(blob[:-1])  # truncated
    with pytest.raises(wt.WtmdError):
        m.restore(b"X" + blob[1:])  # not a checkpoint
    with pytest.raises(wt.WtmdError):
        m.restore(blob[:16])
    other = gpu_handle(dict(spec, capacity=5000), "f32")
    p2 = wt.particles(x, torch.float32)
    other.bind(p2, torch.zeros_like(p2), torch.zeros_like(p2))
    with pytest.raises(wt.WtmdError):
        other.restore(blob)  # another hill capacity
    f64 = gpu_handle(spec, "f64")
    p3 = wt.particles(x, torch.float64)
    f64.bind(p3, torch.zeros_like(p3), torch.zeros_like(p3))
    with pytest.raises(wt.WtmdError):
        f64.restore(blob)  # another precision
    m.restore(blob)  # the handle is still usable after the refusals
    m.step_n(5)
    m.check()


def test_persistent_walkers_resume_is_bitwise():
    """The persistent multi-walker step (LJ clusters of uneven size sharing one
    hill list, a hill per walker every 2 steps, FP64 grid) saved and resumed
    in a fresh handle reproduces the uninterrupted run bitwise."""
    from test_gpu_walkers import _setup, cluster_spec, shared_hills

    spec, x, v = cluster_spec(stride=2, grid=((32, 32), (0.0, 0.0), (12.0, 1.0)))
    hills = shared_hills(spec, x)
    m, pos, vel, F = _setup(spec, x, v, hills, True)
    m.step_n(6)
    blob = m.checkpoint()
    m.step_n(8)
    ref = _state(m, pos, vel, F)
    m2, p2, v2, F2 = _setup(spec, x, v, hills, True)
    m2.restore(blob)
    m2.step_n(8)
    _same(ref, _state(m2, p2, v2, F2))


def _resume_vs_oracle(spec, x, v, t_save, t_more):
    """GPU: t_save steps, checkpoint, a fresh handle restored from it and
    t_more steps; oracle: t_save + t_more steps straight.  Returns both."""
    import oracle as o
    from systems import oracle_system

    wt = _wt()
    m = gpu_handle(spec, "f64")
    pos, vel = wt.particles(x, torch.float64), wt.particles(v, torch.float64)
    F = torch.zeros_like(pos)
    m.bind(pos, vel, F)
    m.step_n(t_save)
    blob = m.checkpoint()
    m.close()
    m2 = gpu_handle(spec, "f64")
    p2, v2 = wt.particles(np.zeros_like(x), torch.float64), wt.particles(np.zeros_like(x), torch.float64)
    F2 = torch.zeros_like(p2)
    m2.bind(p2, v2, F2)
    m2.restore(blob)
    m2.step_n(t_more)
    got = _state(m2, p2, v2, F2)
    sim = o.Sim(oracle_system(spec), x=x, v=v)
    sim.forces()
    assert sim.run(t_save + t_more) == 0
    return got, sim


def test_lj_resume_matches_the_oracle_fp64():
    """FP64 LJ fluid with coordination + Rg CVs and an FP64 grid, saved at
    step 60 and resumed in a fresh handle for 80 more steps (3 deposits before
    the save, 4 after), against the oracle run straight for 140 steps."""
    from synth import velocities

    spec, x, L = lj_fluid_spec(n=500, n_tag=37, n_rg=20, seed=4, jitter=0.1, capacity=4000)
    spec.update(stride=20, w0=0.5, grid=((32, 24), (0.0, 0.5), (40.0, 3.0)))
    v = velocities(500, 1.0, 1.0, seed=9)
    got, sim = _resume_vs_oracle(spec, x, v, 60, 80)
    assert got["counters"] == (140, sim.n_hills) and sim.n_hills == 7
    assert np.max(np.abs(got["pos"][:, :3] - sim.x)) < 1e-9
    assert np.max(np.abs(got["vel"][:, :3] - sim.v)) < 1e-9
    assert np.allclose(got["hills"], sim.hills[:7], rtol=1e-9, atol=1e-12)
    g = got["grid"].ravel()
    assert np.allclose(g, sim.grid, rtol=1e-9, atol=1e-9 * np.abs(sim.grid).max())


def test_mueller_brown_grid_sourced_resume_matches_the_oracle():
    """Three Mueller-Brown walkers whose bias is read from the FP64 grid,
    saved at step 150 and resumed for 250 more: the oracle's straight run of
    400 steps gives the same positions, hills and grid."""
    spec = dict(engine="mb", walker_sizes=[1, 1, 1], dims=2, dt=1e-4, friction=1.0, kT=15.0, seed=0,
                sigma=(0.05, 0.05), w0=1.0, gamma=10.0, stride=10, capacity=200,
                grid=((108, 96), (-1.5, -0.5), (1.2, 2.2)), bias_grid=True,
                cvs=[dict(kind="component", a=[0], axis=0), dict(kind="component", a=[0], axis=1)])
    x = np.array([[-0.558, 1.442, 0], [0.623, 0.028, 0], [-0.05, 0.467, 0]])
    got, sim = _resume_vs_oracle(spec, x, np.zeros_like(x), 150, 250)
    assert got["counters"] == (400, 120) and sim.n_hills == 120
    assert np.max(np.abs(got["pos"][:, :2] - sim.x[:, :2])) < 1e-10
    assert np.allclose(got["hills"], sim.hills[:120], rtol=1e-10, atol=1e-12)
    g = got["grid"].ravel()
    assert np.allclose(g, sim.grid, rtol=1e-10, atol=1e-10 * np.abs(sim.grid).max())
