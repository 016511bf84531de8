"""GPU tests of the LJ engine's Verlet neighbour lists and of the FP32
coordination path's reproducibility (the lists are an implementation device
of the engine; the oracle evaluates every pair inside the cutoff directly).

* A trajectory cut by a forced list rebuild (re-binding the same arrays
  recomputes the forces with fresh lists) is bitwise the trajectory of an
  uninterrupted run: the force depends only on the pairs inside the cutoff,
  never on when the lists were built.
* Atoms moved by the caller between calls, by more than half the skin, are
  picked up: the forces after the next step match the oracle's at the
  positions the step produced.
* The FP32 coordination value (exact quantized FP64 atomics) and the forces
  of two evaluations of the same positions are bitwise equal.
* A cell that overflows its capacity is reported (WTMD_ECELL); atoms left
  without a list read none (list counts start at 0 and are clamped).
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


def _state(spec, x, v, prec):
    wt = _wt()
    dt = torch.float32 if prec == "f32" else torch.float64
    pos, vel = wt.particles(x, dt), wt.particles(v, dt)
    return pos, vel, torch.zeros_like(pos)


def _hills(spec, x, n=2000, seed=11):
    import oracle as o

    sim = o.Sim(oracle_system(spec), x=x)
    _, xi0, _, _ = sim.bias(x, hills=np.zeros((0, 4)))
    sig = np.asarray(spec["sigma"])
    d = len(spec["cvs"])
    return synth.walk_hills(n, xi0[0, :d] - 3 * sig, xi0[0, :d] + 3 * sig, 0.5 * sig, seed=seed)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_forced_rebuild_leaves_the_trajectory_bitwise_unchanged(prec):
    spec, x, L = lj_fluid_spec(n=4096, seed=2)
    spec.update(stride=5, capacity=3000)
    v = synth.velocities(4096, 1.0, 1.0, seed=3)
    hills = _hills(spec, x)
    runs = []
    for cut in (None, 7):
        m = gpu_handle(spec, prec)
        m.hills_load(hills)
        pos, vel, F = _state(spec, x, v, prec)
        m.bind(pos, vel, F)
        if cut is None:
            m.step_n(20)
        else:
            m.step_n(cut)
            m.bind(pos, vel, F)  # forces recomputed now, with freshly built lists
            m.step_n(20 - cut)
        torch.cuda.synchronize()
        runs.append((pos.clone(), vel.clone(), F.clone(), m.hills_read()))
        m.close()
    a, b = runs
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1]) and torch.equal(a[2], b[2])
    assert np.array_equal(a[3], b[3]) and a[3].shape[0] == 2000 + 4


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_atoms_moved_by_the_caller_are_seen_by_the_lists(prec):
    import oracle as o

    spec, x, L = lj_fluid_spec(n=4096, seed=4)
    v = synth.velocities(4096, 1.0, 1.0, seed=5)
    m = gpu_handle(spec, prec)
    pos, vel, F = _state(spec, x, v, prec)
    m.bind(pos, vel, F)
    m.step_n(3)
    # a different configuration of the same fluid: every atom moves far
    # beyond half the skin (0.15 sigma)
    x2, _ = synth.lattice(4096, 0.8, seed=40, jitter=0.05)
    x2 = (x2 + 0.37 * L) % L
    with torch.no_grad():
        pos[:, :3] = torch.as_tensor(x2, dtype=pos.dtype, device=pos.device)
    m.step_n(1)
    torch.cuda.synchronize()
    xf = to_np(pos)[:, :3]
    assert np.max(np.abs(xf - x2)) > 0.0  # the step moved them
    sim = o.Sim(oracle_system(spec), x=xf)
    Fr = sim.forces()  # LJ + bias (no hills loaded: the bias force is 0)
    Fg = to_np(F)[:, :3]
    tol = 1e-12 if prec == "f64" else 2e-5
    err = np.linalg.norm(Fg - Fr, axis=1) / max(1.0, np.linalg.norm(Fr, axis=1).max())
    assert err.max() < tol, err.max()
    m.close()


def test_fp32_coordination_is_bitwise_reproducible():
    wt = _wt()
    spec, x, L = lj_fluid_spec(n=4096, seed=6)
    m = gpu_handle(spec, "f32")
    m.hills_load(_hills(spec, x))
    pos = wt.particles(x, torch.float32)
    outs = []
    for _ in range(3):
        F = torch.zeros_like(pos)
        V, xi, dV = m.bias_eval(pos, F)
        torch.cuda.synchronize()
        outs.append((xi.clone(), V.clone(), dV.clone(), F.clone()))
    for o in outs[1:]:
        assert all(torch.equal(p, q) for p, q in zip(outs[0], o))
    m.close()


def test_cell_overflow_is_reported():
    """A dense block of 64 atoms inside one cell of a dilute box (cell
    capacity 24) overflows the cell list: the step reports WTMD_ECELL."""
    wt = _wt()
    L = 20.0
    cell = L / 7  # cells at least rc + skin = 2.8 wide
    g = np.arange(4) * 0.65 + 0.4
    block = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3) + 3 * cell
    r = synth.rng(12)
    far = 3 * cell + np.array([[7.5, 0.0, 0.0]]) + np.stack(np.meshgrid(np.arange(5), np.arange(5), np.arange(6),
                                                                        indexing="ij"), -1).reshape(-1, 3) * 1.6
    x = np.concatenate([block, far[:136] + r.normal(scale=0.02, size=(136, 3))]) % L
    spec = dict(engine="lj", walker_sizes=[200], box=(L, L, L), dt=0.005, kT=1.0, friction=1.0, sigma=(0.1,),
                cvs=[dict(kind="component", a=[0], axis=0)])
    m = gpu_handle(spec, "f32")
    pos, vel, F = _state(spec, x, np.zeros_like(x), "f32")
    m.bind(pos, vel, F)
    with pytest.raises(wt.WtmdError) as e:
        m.step_n(1)
    assert e.value.code == -7
    m.close()
