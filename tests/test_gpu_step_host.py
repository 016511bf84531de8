"""wtmd_step_host: steps whose state lives in host memory, through the C ABI.

The state [3][N][4] (positions, velocities, forces) is copied in, stepped and
copied back by the library.  Every path -- one captured graph per call
(packed device block, pinned buffer, one step), the copy-around-step_n path
(pageable buffer or separate device arrays) and several steps per call --
must reproduce the trajectory of the same handle stepped on the device alone,
bitwise: the copies move bytes and the steps are the same kernels.
"""
import numpy as np
import pytest

from systems import gpu_handle, lj_fluid_spec

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _wt():
    import paper_2301_04835_b300 as wt
    return wt


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_host_buffer_steps_match_device_steps_bitwise(prec):
    wt = _wt()
    from synth import velocities

    spec, x, L = lj_fluid_spec(n=500, n_tag=37, n_rg=20, seed=4, jitter=0.1, capacity=4000)
    spec.update(stride=7, w0=0.5)
    v = velocities(500, 1.0, 1.0, seed=9)
    dt = torch.float32 if prec == "f32" else torch.float64

    def packed_handle():
        m = gpu_handle(spec, prec)
        st = torch.stack([wt.particles(x, dt), wt.particles(v, dt), torch.zeros_like(wt.particles(x, dt))]).contiguous()
        m.bind(st[0], st[1], st[2])
        m.step_n(5)
        return m, st

    ref, sref = packed_handle()
    ref.step_n(20)
    torch.cuda.synchronize()
    want = sref.cpu().numpy()

    # one captured graph per call: packed device block, pinned buffer, in == out
    m, st = packed_handle()
    hst = st.cpu().pin_memory()
    for _ in range(20):
        m.step_host(hst, wait=True)
    assert np.array_equal(hst.numpy(), want)
    assert np.array_equal(st.cpu().numpy(), want)
    assert m.counters() == ref.counters()

    # several steps per call, separate in and out buffers
    m2, st2 = packed_handle()
    hin = st2.cpu().pin_memory()
    hout = torch.empty_like(hin).pin_memory()
    m2.step_host(hin, hout, n=20)
    assert np.array_equal(hout.numpy(), want)

    # separate device arrays and a pageable numpy buffer: copies around step_n
    m3 = gpu_handle(spec, prec)
    p3, v3 = wt.particles(x, dt), wt.particles(v, dt)
    f3 = torch.zeros_like(p3)
    m3.bind(p3, v3, f3)
    m3.step_n(5)
    torch.cuda.synchronize()
    buf = np.ascontiguousarray(np.stack([p3.cpu().numpy(), v3.cpu().numpy(), f3.cpu().numpy()]))
    for _ in range(4):
        m3.step_host(buf, n=5)
    assert np.array_equal(buf, want)


def test_step_host_is_validated():
    wt = _wt()
    spec, x, L = lj_fluid_spec(n=500, n_tag=37, n_rg=20, seed=4, jitter=0.1, capacity=100)
    m = gpu_handle(spec, "f32")
    buf = np.zeros((3, 500, 4), np.float32)
    with pytest.raises(wt.WtmdError):
        m.step_host(buf)  # nothing bound
    p = wt.particles(x, torch.float32)
    m.bind(p, torch.zeros_like(p), torch.zeros_like(p))
    with pytest.raises(wt.WtmdError):
        m.step_host(buf, n=0)
