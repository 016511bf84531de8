"""The allocation-free hills sum (wtmd_hills_eval_static) gives the same V and
dV/dxi as hills_eval on an FP64 handle, and as the FP64 oracle.

wtmd_hills_eval_static serves callers that must not allocate device memory
(for example an engine plugin restricted to the buffers it is handed, or a
caller whose memory footprint must stay fixed once it has started).  It keeps
its partial sums in one fixed library-owned device array shared by all calls,
so these tests make calls in a row with different sizes and launch layouts:
if a call read anything an earlier call left behind, its result would differ.
The file is named to be collected last.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

MAX_POINTS = 32768  # WTMD_STATIC_MAX_POINTS


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def _static_call(wt, sigma, period, hills_d, xi_d, V, dV):
    d = len(sigma)
    sg = (C.c_double * d)(*sigma)
    pr = (C.c_double * d)(*period)
    return wt.lib().wtmd_hills_eval_static(d, sg, pr, _ptr(hills_d), hills_d.shape[0], _ptr(xi_d), xi_d.shape[0],
                                           _ptr(V), _ptr(dV), C.c_void_p(torch.cuda.current_stream().cuda_stream))


def _abs_term_scale(pts, hills, sigma, period):
    """sum_k w_k e_k |D_ki| / sigma_i^2 per point and CV: the size of the
    terms whose signed sum is dV/dxi_i (the bound for a cancelling sum)."""
    sig, per = np.asarray(sigma), np.asarray(period)
    out = np.zeros_like(pts)
    for p in range(pts.shape[0]):
        D = pts[p][None, :] - hills[:, : pts.shape[1]]
        D = np.where(per > 0, D - per * np.rint(D / np.where(per > 0, per, 1.0)), D)
        e = hills[:, 3] * np.exp(-(D ** 2 / (2 * sig ** 2)).sum(1))
        out[p] = (e[:, None] * np.abs(D)).sum(0) / sig ** 2
    return out


# (sigma, period, box, H, P): P picks the kernel's layout -- threads per point
# 1 (P >= 1024), 4 (64 <= P < 1024), 32 (8 <= P < 64), 256 (P < 8, the
# cross-warp shared-memory reduction); P = MAX_POINTS leaves room for one
# hill split only
CASES = [
    ((0.05, 0.1, 0.07), (0.0, 0.0, 0.0), ([-1.0, 0.5, 2.0], [1.5, 2.0, 3.0]), 20001, 3000),
    ((0.35, 0.2), (2 * np.pi, 2 * np.pi), ([-np.pi, -np.pi], [np.pi, np.pi]), 777, 17),
    ((0.05, 0.1), (0.0, 0.0), ([0.0, 0.0], [1.0, 1.0]), 5003, 5),
    ((0.2,), (0.0,), ([-2.0], [2.0]), 40000, 1),
    ((0.3, 0.25, 0.4), (2 * np.pi, 0.0, 0.0), ([-np.pi, -1.0, -1.0], [np.pi, 1.0, 1.0]), 3001, 200),
    ((0.05, 0.1), (0.0, 0.0), ([0.0, 0.0], [1.0, 1.0]), 1500, MAX_POINTS),
]


def _run_static(wt, sigma, period, hills, pts):
    d = len(sigma)
    hills_d = torch.tensor(hills, dtype=torch.float64, device="cuda").reshape(-1, 4)
    xi_d = torch.tensor(pts, dtype=torch.float64, device="cuda")
    P = pts.shape[0]
    V = torch.full((P,), float("nan"), dtype=torch.float64, device="cuda")
    dV = torch.full((P, d), float("nan"), dtype=torch.float64, device="cuda")
    assert _static_call(wt, sigma, period, hills_d, xi_d, V, dV) == wt.OK
    torch.cuda.synchronize()
    return V.cpu().numpy(), dV.cpu().numpy()


def test_static_hills_sum_matches_hills_eval_and_oracle():
    import paper_2301_04835_b300 as wt

    for k, (sigma, period, (lo, hi), H, P) in enumerate(CASES):
        d = len(sigma)
        hills = synth.uniform_hills(H, lo, hi, seed=40 + k)
        pts = synth.uniform_points(P, lo, hi, seed=50 + k)
        m = wt.Wtmd(precision="f64", sigma=sigma, capacity=H, walker_sizes=[1])
        for i in range(d):
            m.cv_define(wt.CV_COMPONENT, a=[0], axis=i, period=period[i])
        m.hills_load(hills)
        V_ref, dV_ref = (t.cpu().numpy() for t in m.hills_eval(torch.tensor(pts, dtype=torch.float64,
                                                                                 device="cuda")))
        m.close()
        Vo, dVo = oracle.hills_sum(pts, hills, sigma, period)
        # two calls in a row on the same inputs: the second reads scratch the
        # first left behind and must not depend on it
        Vg, dVg = _run_static(wt, sigma, period, hills, pts)
        Vg2, dVg2 = _run_static(wt, sigma, period, hills, pts)
        assert np.array_equal(Vg, Vg2) and np.array_equal(dVg, dVg2), f"case {k}: repeat differs"
        S = _abs_term_scale(pts, hills, sigma, period)
        for Vr, dVr, what in ((V_ref, dV_ref, "hills_eval"), (Vo, dVo, "oracle")):
            assert np.all(np.abs(Vg - Vr) <= 1e-12 * np.abs(Vr)), (k, what, np.max(np.abs(Vg - Vr) / np.abs(Vr)))
            assert np.all(np.abs(dVg - dVr) <= 1e-12 * np.abs(dVr) + 1e-13 * S), (k, what)


def test_static_hills_sum_no_hills_is_zero():
    import paper_2301_04835_b300 as wt

    pts = synth.uniform_points(300, [0.0, 0.0], [1.0, 1.0], seed=3)
    V, dV = _run_static(wt, (0.1, 0.1), (0.0, 0.0), np.zeros((0, 4)), pts)
    assert np.all(V == 0.0) and np.all(dV == 0.0)


def test_static_hills_sum_allocates_nothing():
    import paper_2301_04835_b300 as wt

    sigma, period, (lo, hi), H, P = CASES[0]
    hills = synth.uniform_hills(H, lo, hi, seed=7)
    pts = synth.uniform_points(P, lo, hi, seed=8)
    hills_d = torch.tensor(hills, dtype=torch.float64, device="cuda")
    xi_d = torch.tensor(pts, dtype=torch.float64, device="cuda")
    V = torch.empty(P, dtype=torch.float64, device="cuda")
    dV = torch.empty(P, 3, dtype=torch.float64, device="cuda")
    assert _static_call(wt, sigma, period, hills_d, xi_d, V, dV) == wt.OK  # first call: address lookup
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        assert _static_call(wt, sigma, period, hills_d, xi_d, V, dV) == wt.OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_static_hills_sum_rejects_too_many_points():
    import paper_2301_04835_b300 as wt

    P = MAX_POINTS + 1
    hills_d = torch.zeros(4, 4, dtype=torch.float64, device="cuda")
    hills_d[:, 3] = 1.0
    xi_d = torch.zeros(P, 1, dtype=torch.float64, device="cuda")
    V = torch.zeros(P, dtype=torch.float64, device="cuda")
    dV = torch.zeros(P, 1, dtype=torch.float64, device="cuda")
    assert _static_call(wt, (0.1,), (0.0,), hills_d, xi_d, V, dV) == wt.EINVAL
    torch.cuda.synchronize()
    assert torch.all(V == 0)
