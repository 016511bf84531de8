"""Hand-written adjoint of the CV map (wtmd_cv_adjoint) and its
torch.autograd.Function, against the FP64 oracle's Jacobians and finite
differences.  The paper differentiates CVs with jax.grad (Sec. 2); here the
vector-Jacobian product grad_r = J^T grad_xi is a CUDA kernel.

Workload: 1024 replicas of a 22-bead chain (bond 1.0, angle 109.47 deg,
random torsions), CVs = dihedrals of beads 5-7-9-15 and 7-9-15-17 (0-based).
"""
import numpy as np
import pytest

import synth
from systems import gpu_handle, lj_fluid_spec, oracle_system, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CHAIN = dict(engine="chain", walker_sizes=[22] * 1024, sigma=(0.35, 0.35), gamma=6.0, capacity=100,
             cvs=[dict(kind="dihedral", a=[5, 7, 9, 15], period=2 * np.pi),
                  dict(kind="dihedral", a=[7, 9, 15, 17], period=2 * np.pi)])


def _wt():
    import paper_2301_04835_b300 as wt
    return wt


def _oracle_vjp(spec, x, g):
    """J^T g per walker from the oracle's analytic Jacobians."""
    import oracle as o

    sysd = oracle_system(spec)
    out = np.zeros_like(x)
    off = 0
    for w, n in enumerate(spec["walker_sizes"]):
        for c, cv in enumerate(sysd.cvs):
            _, J = o.cv_eval(cv, x[off: off + n], list(sysd.box))
            out[off: off + n] += g[w, c] * J
        off += n
    return out


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_adjoint_matches_oracle_chain_replicas(prec):
    wt = _wt()
    x = synth.chain_replicas(1024, 22, seed=2)
    if prec == "f32":
        x = x.astype(np.float32).astype(np.float64)
    dt = torch.float32 if prec == "f32" else torch.float64
    m = gpu_handle(CHAIN, prec)
    pos = wt.particles(x, dt)
    xi = m.cv_forward(pos)
    g = synth.rng(3).normal(size=(1024, 2))
    gt = torch.tensor(g, dtype=dt, device="cuda")
    out = to_np(m.cv_adjoint(gt))
    assert np.all(out[:, 3] == 0)
    ref = _oracle_vjp(CHAIN, x, g)
    err = np.linalg.norm(out[:, :3] - ref) / np.linalg.norm(ref)
    assert err < (1e-12 if prec == "f64" else 1e-5), err


def test_adjoint_matches_finite_differences_of_gpu_forward():
    """d/dr of sum_c g_c xi_c(r) by central differences of the FP64 forward."""
    wt = _wt()
    spec = dict(CHAIN, walker_sizes=[22] * 3)
    x = synth.chain_replicas(3, 22, seed=7)
    m = gpu_handle(spec, "f64")
    g = synth.rng(8).normal(size=(3, 2))
    gt = torch.tensor(g, dtype=torch.float64, device="cuda")
    m.cv_forward(wt.particles(x, torch.float64))
    adj = to_np(m.cv_adjoint(gt))[:, :3]
    h = 1e-6
    for i in [5, 7, 9, 15, 17, 22 + 9, 44 + 15]:
        for k in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, k] += h
            xm[i, k] -= h
            fp = (to_np(m.cv_forward(wt.particles(xp, torch.float64))) * g).sum()
            fm = (to_np(m.cv_forward(wt.particles(xm, torch.float64))) * g).sum()
            assert abs((fp - fm) / (2 * h) - adj[i, k]) < 1e-7 * max(1.0, abs(adj[i, k]))
    # atoms not in any dihedral get nothing
    assert np.all(adj[0] == 0) and np.all(adj[21] == 0)


def test_cv_function_gradcheck():
    wt = _wt()
    spec = dict(CHAIN, walker_sizes=[22] * 2)
    x = torch.tensor(synth.chain_replicas(2, 22, seed=9), dtype=torch.float64, device="cuda", requires_grad=True)
    m = gpu_handle(spec, "f64")
    assert torch.autograd.gradcheck(lambda p: wt.cv_apply(p, m), (x,), eps=1e-6, atol=1e-6, rtol=1e-5)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_cv_function_backward_coordination_and_rg(prec):
    """autograd through coordination (list against all atoms) and Rg, against
    the oracle's J^T g; a second forward in between forces the recompute."""
    wt = _wt()
    spec, x, L = lj_fluid_spec(n=500, n_tag=37, n_rg=20, seed=4, jitter=0.1)
    if prec == "f32":
        x = x.astype(np.float32).astype(np.float64)
    dt = torch.float32 if prec == "f32" else torch.float64
    m = gpu_handle(spec, prec)
    p = torch.tensor(x, dtype=dt, device="cuda", requires_grad=True)
    xi = wt.cv_apply(p, m)
    m.cv_forward(wt.particles(x + 0.1, dt))  # another forward on the handle
    g = np.array([[0.7, -1.3]])
    xi.backward(torch.tensor(g, dtype=dt, device="cuda"))
    ref = _oracle_vjp(spec, x, g)
    err = np.linalg.norm(to_np(p.grad) - ref) / np.linalg.norm(ref)
    assert err < (1e-12 if prec == "f64" else 1e-5), err


def test_adjoint_bias_force_identity():
    """cv_adjoint(-dV/dxi) equals the force bias_eval scatters."""
    wt = _wt()
    x = synth.chain_replicas(1024, 22, seed=2).astype(np.float32).astype(np.float64)
    m = gpu_handle(dict(CHAIN, capacity=1000), "f32")
    m.hills_load(synth.uniform_hills(500, [-np.pi, -np.pi], [np.pi, np.pi], seed=4))
    pos = wt.particles(x, torch.float32)
    F = torch.zeros_like(pos)
    V, xi, dV = m.bias_eval(pos, F)
    adj = m.cv_adjoint(-dV)
    assert torch.equal(adj[:, :3], F[:, :3])


SHAPES = dict(engine="none", walker_sizes=[40] * 64, sigma=(0.1, 0.1, 0.1), capacity=16,
              cvs=[dict(kind="gyration", a=None, axis=5), dict(kind="distance", a=[0, 1, 2, 3], b=list(range(20, 40))),
                   dict(kind="angle", a=[5, 17, 30])])


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_adjoint_matches_oracle_shape_cvs(prec):
    """64 walkers of 40 atoms: gyration anisotropy, Distance between group
    centres and Angle: J^T g against the oracle's Jacobians."""
    wt = _wt()
    x = synth.rng(12).normal(size=(64 * 40, 3)) * np.array([2.0, 1.2, 0.8])
    if prec == "f32":
        x = x.astype(np.float32).astype(np.float64)
    dt = torch.float32 if prec == "f32" else torch.float64
    m = gpu_handle(SHAPES, prec)
    m.cv_forward(wt.particles(x, dt))
    g = synth.rng(5).normal(size=(64, 3))
    out = to_np(m.cv_adjoint(torch.tensor(g, dtype=dt, device="cuda")))
    ref = _oracle_vjp(SHAPES, x, g)
    err = np.linalg.norm(out[:, :3] - ref) / np.linalg.norm(ref)
    assert err < (1e-12 if prec == "f64" else 1e-5), err
