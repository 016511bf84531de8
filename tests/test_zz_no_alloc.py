"""The allocation-free hills sum (wtmd_hills_eval_static) gives the same V and
dV/dxi as hills_eval on an FP64 handle.

wtmd_hills_eval_static serves callers that must not allocate device memory
(for example an engine plugin restricted to the buffers it is handed).  It
keeps its partial sums in one fixed library-owned device array shared by all
calls, so this test makes two calls in a row with different sizes: if the
second call read anything the first left behind, its result would differ.
The file is named to be collected last.
"""
import ctypes as C

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def _static_call(wt, sigma, period, hills_d, xi_d, V, dV):
    d = len(sigma)
    sg = (C.c_double * d)(*sigma)
    pr = (C.c_double * d)(*period)
    return wt.lib().wtmd_hills_eval_static(d, sg, pr, _ptr(hills_d), hills_d.shape[0], _ptr(xi_d), xi_d.shape[0],
                                           _ptr(V), _ptr(dV), C.c_void_p(torch.cuda.current_stream().cuda_stream))


def _abs_term_scale(pts, hills, sigma, period):
    sig, per = np.asarray(sigma), np.asarray(period)
    out = np.zeros_like(pts)
    for p in range(pts.shape[0]):
        D = pts[p][None, :] - hills[:, : pts.shape[1]]
        D = np.where(per > 0, D - per * np.rint(D / np.where(per > 0, per, 1.0)), D)
        e = hills[:, 3] * np.exp(-(D ** 2 / (2 * sig ** 2)).sum(1))
        out[p] = (e[:, None] * np.abs(D)).sum(0) / sig ** 2
    return out


def test_static_hills_sum_matches_hills_eval_twice():
    import paper_2301_04835_b300 as wt

    cases = [  # (sigma, period, box, H, P): second call smaller and periodic
        ((0.05, 0.1, 0.07), (0.0, 0.0, 0.0), ([-1.0, 0.5, 2.0], [1.5, 2.0, 3.0]), 20001, 3000),
        ((0.35, 0.2), (2 * np.pi, 2 * np.pi), ([-np.pi, -np.pi], [np.pi, np.pi]), 777, 17),
    ]
    for k, (sigma, period, (lo, hi), H, P) in enumerate(cases):
        d = len(sigma)
        hills = synth.uniform_hills(H, lo, hi, seed=40 + k)
        pts = synth.uniform_points(P, lo, hi, seed=50 + k)
        m = wt.Wtmd(precision="f64", sigma=sigma, capacity=H, walker_sizes=[1])
        for i in range(d):
            m.cv_define(wt.CV_COMPONENT, a=[0], axis=i, period=period[i])
        m.hills_load(hills)
        xi_d = torch.tensor(pts, dtype=torch.float64, device="cuda")
        V_ref, dV_ref = m.hills_eval(xi_d)

        hills_d = torch.tensor(hills, dtype=torch.float64, device="cuda")
        V = torch.full((P,), float("nan"), dtype=torch.float64, device="cuda")
        dV = torch.full((P, d), float("nan"), dtype=torch.float64, device="cuda")
        assert _static_call(wt, sigma, period, hills_d, xi_d, V, dV) == wt.OK
        torch.cuda.synchronize()
        Vr, dVr, Vg, dVg = (t.cpu().numpy() for t in (V_ref, dV_ref, V, dV))
        S = _abs_term_scale(pts, hills, sigma, period)
        assert np.all(np.abs(Vg - Vr) <= 1e-12 * np.abs(Vr)), np.max(np.abs(Vg - Vr) / np.abs(Vr))
        assert np.all(np.abs(dVg - dVr) <= 1e-12 * np.abs(dVr) + 1e-13 * S)
        m.close()


def test_static_hills_sum_rejects_too_many_points():
    import paper_2301_04835_b300 as wt

    P = wt_max = 32768 + 1
    hills_d = torch.zeros(4, 4, dtype=torch.float64, device="cuda")
    hills_d[:, 3] = 1.0
    xi_d = torch.zeros(P, 1, dtype=torch.float64, device="cuda")
    V = torch.zeros(P, dtype=torch.float64, device="cuda")
    dV = torch.zeros(P, 1, dtype=torch.float64, device="cuda")
    assert wt_max > 32768
    assert _static_call(wt, (0.1,), (0.0,), hills_d, xi_d, V, dV) == wt.EINVAL
    torch.cuda.synchronize()
    assert torch.all(V == 0)
