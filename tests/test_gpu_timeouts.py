"""Failure detection without a GPU fault: every wait of the persistent
launches is bounded, and a wait that runs out is reported as WTMD_ETIMEOUT
with the device and the handle left usable.

* A cooperative grid in which one CTA never reaches the grid barrier: the
  others give up after the limit and report it (a flag that nothing sets).
* The multi-walker step and the single-system step with a wait limit far
  below the barrier's normal latency: the step reports WTMD_ETIMEOUT, every
  CTA leaves, and after a restore from a checkpoint the handle reproduces an
  uninterrupted run bitwise.
"""
import numpy as np
import pytest

import synth
from systems import gpu_handle, lj_fluid_spec, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _wt():
    import paper_2301_04835_b300 as wt

    return wt


def test_grid_barrier_gives_up_on_an_absent_block():
    wt = _wt()
    assert wt.barrier_probe(8, 3, 1_000_000) is True
    assert wt.barrier_probe(8, -1, 1 << 31) is False
    assert wt.barrier_probe(8, 7, 200_000) is True
    # the device is still usable: a plain hills sum
    m = wt.Wtmd(precision="f32", sigma=[0.1], capacity=4, walker_sizes=[1])
    m.cv_define(wt.CV_COMPONENT, a=[0], axis=0)
    m.hills_load([[0.25, 0.0, 0.0, 2.0]])
    V, dV = m.hills_eval(torch.tensor([[0.25]], dtype=torch.float32, device="cuda"))
    assert abs(V.item() - 2.0) < 1e-5
    with pytest.raises(wt.WtmdError):
        wt.barrier_probe(8, 8, 1000)  # absent CTA outside the grid


def _state(pos, vel, F, m):
    torch.cuda.synchronize()
    return [to_np(pos), to_np(vel), to_np(F), m.hills_read(), np.array(m.counters())]


def _timeout_then_recover(m, pos, vel, F, steps):
    wt = _wt()
    m.step_n(2)
    blob = m.checkpoint()
    m.step_n(steps)
    ref = _state(pos, vel, F, m)
    m.restore(blob)
    m.wait_limit(100)  # far below one barrier round trip
    m.step_n(1, check=False)
    with pytest.raises(wt.WtmdError) as e:
        m.check()
    assert e.value.code == wt.ETIMEOUT
    m.wait_limit(0)
    m.restore(blob)
    m.step_n(steps)
    got = _state(pos, vel, F, m)
    for a, b in zip(ref, got):
        assert np.array_equal(a, b)
    with pytest.raises(wt.WtmdError):
        m.wait_limit(-1)


def test_walkers_step_timeout_is_reported_and_recovered():
    from test_gpu_walkers import _setup, cluster_spec, shared_hills

    spec, x, v = cluster_spec(stride=2)
    hills = shared_hills(spec, x)
    m, pos, vel, F = _setup(spec, x, v, hills, True)
    _timeout_then_recover(m, pos, vel, F, 5)


def test_single_system_step_timeout_is_reported_and_recovered():
    wt = _wt()
    spec, x, L = lj_fluid_spec(n=4096, seed=6)
    spec.update(stride=3, capacity=3000)
    m = gpu_handle(spec, "f32")
    x = np.asarray(x, dtype=np.float32).astype(np.float64)
    pos, vel = wt.particles(x, torch.float32), wt.particles(synth.velocities(4096, 1.0, 1.0, seed=7), torch.float32)
    F = torch.zeros_like(pos)
    m.bind(pos, vel, F)
    assert m.fused_step(True) is True
    _timeout_then_recover(m, pos, vel, F, 6)
