"""GPU tests of the single-launch persistent step (wtmd_fused_step): the MD
step of one periodic FP32 system with LJ Verlet lists, tile coordination and
Rg CVs and the exact hills sum, run as one cooperative kernel per step.

* It is off by default; once allowed it is used when the handle has that
  form, and not otherwise.
* Its trajectory, hills and heights match the FP64 oracle (Sec. 3.2.1 steps
  (a)-(f) with the Sec. 2.1.5 update) to the FP32 trajectory bounds of the
  per-kernel step, through neighbour-list rebuilds and deposits.
* It agrees with the per-kernel step on the same inputs (they differ only in
  the order of the hills reduction) and is bitwise reproducible.
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


def _f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def _hills(spec, x, n, seed):
    import oracle as o

    sim = o.Sim(oracle_system(spec), x=x)
    _, xi0, _, _ = sim.bias(x, hills=np.zeros((0, 4)))
    sig = np.asarray(spec["sigma"])
    return synth.walk_hills(n, xi0[0, :2] - 3 * sig, xi0[0, :2] + 3 * sig, 0.5 * sig, seed=seed)


def _run(spec, x, v, hills, nsteps, fused):
    wt = _wt()
    m = gpu_handle(spec, "f32")
    m.hills_load(hills)
    pos, vel = wt.particles(x, torch.float32), wt.particles(v, torch.float32)
    F = torch.zeros_like(pos)
    m.bind(pos, vel, F)
    assert m.fused_step(fused) == fused
    m.step_n(nsteps)
    torch.cuda.synchronize()
    out = (to_np(pos)[:, :3], to_np(vel)[:, :3], to_np(F)[:, :3], m.hills_read(), m.counters())
    m.close()
    return out


def _system(n=4096, seed=3):
    spec, x, L = lj_fluid_spec(n=n, seed=seed)
    spec.update(stride=5, capacity=4000)
    x = _f32(x)
    v = _f32(synth.velocities(n, 1.0, 1.0, seed=seed + 1))
    return spec, x, v


def test_fused_step_is_used_only_for_its_form():
    wt = _wt()
    spec, x, v = _system(n=500)
    m = gpu_handle(spec, "f32")
    assert m.fused_step() is False  # off by default
    assert m.fused_step(True) is True
    assert m.fused_step() is True
    assert m.fused_step(False) is False
    m.close()
    m = gpu_handle(spec, "f64")
    assert m.fused_step(True) is False
    m.close()
    # a grid-read bias or open clusters take the per-kernel step
    spec_g = dict(spec, grid=((32, 32), (0.0, 0.0), (10.0, 5.0)), bias_grid=True)
    m = gpu_handle(spec_g, "f32")
    assert m.fused_step(True) is False
    m.close()
    spec_c = dict(spec, box=(0, 0, 0))
    m = gpu_handle(spec_c, "f32")
    assert m.fused_step(True) is False
    m.close()


def test_fused_step_matches_the_fp64_oracle_4096():
    import oracle as o

    spec, x, v = _system()
    hills = _hills(spec, x, 2000, seed=9)
    nsteps = 20
    X, Vv, F, h, (step, nh) = _run(spec, x, v, hills, nsteps, True)
    sim = o.Sim(oracle_system(spec), x=x, v=v, hills=hills)
    sim.forces()
    assert sim.run(nsteps) == 0
    assert step == nsteps and nh == sim.n_hills == 2000 + nsteps // 5
    d = np.abs(X - sim.x)
    assert d.max() < 1e-3 and np.median(d) < 1e-5, (d.max(), np.median(d))
    ref = sim.hills[:nh]
    # deposited centres are the CVs (FP32 path, FP64 CV values), heights
    # w0 exp(-V / (kT (gamma - 1))) with the FP32 hills sum
    assert np.allclose(h[:2000], ref[:2000], rtol=0, atol=0)
    assert np.allclose(h[2000:, :2], ref[2000:, :2], rtol=1e-4, atol=1e-6)
    assert np.allclose(h[2000:, 3], ref[2000:, 3], rtol=1e-2)


def test_fused_and_per_kernel_steps_agree():
    spec, x, v = _system()
    hills = _hills(spec, x, 2000, seed=10)
    a = _run(spec, x, v, hills, 20, True)
    b = _run(spec, x, v, hills, 20, False)
    assert np.abs(a[0] - b[0]).max() < 1e-4
    assert np.median(np.abs(a[0] - b[0])) < 1e-6
    assert a[4] == b[4]
    assert np.allclose(a[3], b[3], rtol=1e-5, atol=1e-7)


def test_fused_step_is_bitwise_reproducible():
    spec, x, v = _system(seed=5)
    hills = _hills(spec, x, 1000, seed=11)
    a = _run(spec, x, v, hills, 30, True)
    b = _run(spec, x, v, hills, 30, True)
    for p, q in zip(a[:4], b[:4]):
        assert np.array_equal(p, q)
