"""FP64 CPU oracle for the well-tempered metadynamics bias-force path.

TEST INFRASTRUCTURE ONLY: `tests/`, `__graft_entry__.smoke()` and the
CPU-baseline leg of `bench.py` are the only callers.  The product library
(`paper_2301_04835_b300`) never imports this package and this package never
imports it; they share only the seeded input generators in `synth`.

The arithmetic lives in `wtmd_oracle.c` (plain C, double precision); this
module compiles it with gcc on first use and wraps it with ctypes/numpy.
Each wrapper names the passage of the PySAGES paper it follows (Sec. 2.1.5
for the metadynamics bias, Sec. 2.2 for the collective variables, Sec. 2.1
Eq. (free-energy) for the meaning of the free-energy estimate).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wtmd_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

CV_COMPONENT, CV_DIHEDRAL, CV_COORDINATION, CV_RG, CV_QPAIRS = 1, 2, 3, 4, 5
CV_DISTANCE, CV_ANGLE, CV_GYRATION = 6, 7, 8
# CV_GYRATION quantities (axis): principal moments l1 <= l2 <= l3, asphericity,
# acylindricity, relative shape anisotropy
GY_L1, GY_L2, GY_L3, GY_ASPHERICITY, GY_ACYLINDRICITY, GY_ANISOTROPY = 0, 1, 2, 3, 4, 5
CV_INTENSIVE = 1
ENGINE_NONE, ENGINE_MB, ENGINE_LJ, ENGINE_CHAIN, ENGINE_HARMONIC, ENGINE_WELLS3 = 0, 1, 2, 3, 4, 5


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/liboracle.so (gcc, -O2, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _CV(C.Structure):
    _fields_ = [
        ("kind", C.c_int64), ("n_a", C.c_int64), ("a", C.POINTER(C.c_int32)),
        ("n_b", C.c_int64), ("b", C.POINTER(C.c_int32)), ("axis", C.c_int64),
        ("r0", C.c_double), ("nn", C.c_int64), ("mm", C.c_int64), ("scale", C.c_double),
        ("flags", C.c_int64), ("period", C.c_double),
    ]


class _Sys(C.Structure):
    _fields_ = [
        ("engine", C.c_int64), ("dims", C.c_int64), ("n_walkers", C.c_int64),
        ("walker_off", C.POINTER(C.c_int64)), ("walker_n", C.POINTER(C.c_int64)),
        ("box", C.c_double * 3), ("dt", C.c_double), ("friction", C.c_double), ("mass", C.c_double),
        ("kT", C.c_double), ("seed", C.c_uint64),
        ("lj_eps", C.c_double), ("lj_sig", C.c_double), ("lj_rc", C.c_double),
        ("bond_k", C.c_double), ("bond_r0", C.c_double), ("angle_k", C.c_double), ("angle_t0", C.c_double),
        ("tors_k", C.c_double), ("harm_k", C.c_double),
        ("n_cv", C.c_int64), ("cv", C.POINTER(_CV)), ("sigma", C.c_double * 3),
        ("w0", C.c_double), ("gamma", C.c_double), ("stride", C.c_int64), ("hill_cap", C.c_int64),
        ("grid_bins", C.c_int64 * 3), ("grid_lo", C.c_double * 3), ("grid_hi", C.c_double * 3),
        ("bias_on", C.c_int64), ("bias_grid", C.c_int64),
        ("bias_harm", C.c_int64), ("harm_kcv", C.c_double * 3), ("harm_centre", C.POINTER(C.c_double)),
    ]


class _State(C.Structure):
    _fields_ = [
        ("x", C.POINTER(C.c_double)), ("v", C.POINTER(C.c_double)), ("f", C.POINTER(C.c_double)),
        ("hills", C.POINTER(C.c_double)), ("n_hills", C.c_int64), ("grid", C.POINTER(C.c_double)),
        ("step", C.c_int64), ("xi", C.POINTER(C.c_double)), ("V", C.POINTER(C.c_double)),
        ("dV", C.POINTER(C.c_double)), ("xi_sum", C.POINTER(C.c_double)), ("n_samples", C.c_int64),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        d, i64, u32p, dp = C.c_double, C.c_int64, C.POINTER(C.c_uint32), C.POINTER(C.c_double)
        _lib.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
        _lib.orc_noise3.argtypes = [C.c_uint64, C.c_uint64, C.c_uint32, dp]
        _lib.orc_mb.argtypes = [d, d, dp, dp]
        _lib.orc_mb.restype = d
        _lib.orc_wells3.argtypes = [dp, dp]
        _lib.orc_wells3.restype = d
        _lib.orc_lj.argtypes = [i64, dp, dp, d, d, d, dp]
        _lib.orc_lj.restype = d
        _lib.orc_chain.argtypes = [i64, dp, d, d, d, d, d, dp]
        _lib.orc_chain.restype = d
        _lib.orc_cv_eval.argtypes = [C.POINTER(_CV), i64, dp, dp, dp, dp]
        _lib.orc_hills_sum.argtypes = [i64, i64, dp, i64, dp, dp, dp, dp, dp]
        _lib.orc_wt_height.argtypes = [d, d, d, d]
        _lib.orc_wt_height.restype = d
        _lib.orc_grid_add.argtypes = [i64, C.POINTER(i64), dp, dp, dp, dp, dp, d, dp]
        _lib.orc_fes.argtypes = [i64, dp, d, dp]
        _lib.orc_grid_interp.argtypes = [i64, C.POINTER(i64), dp, dp, dp, dp, i64, dp, dp, dp]
        _lib.orc_grid_interp.restype = C.c_int
        _lib.orc_bias.argtypes = [C.POINTER(_Sys), dp, dp, i64, dp, dp, dp, dp]
        _lib.orc_bias_grid.argtypes = [C.POINTER(_Sys), dp, dp, dp, dp, dp, dp]
        _lib.orc_forces.argtypes = [C.POINTER(_Sys), C.POINTER(_State)]
        _lib.orc_run.argtypes = [C.POINTER(_Sys), C.POINTER(_State), i64]
        _lib.orc_umbrella_integrate.argtypes = [i64, i64, dp, dp, dp, dp, dp, dp]
        _lib.orc_num_threads.restype = C.c_int
        _lib.orc_set_threads.argtypes = [C.c_int]
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


# --------------------------------------------------------------------------
# Primitives
# --------------------------------------------------------------------------
def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 block (Salmon et al., SC'11) -> four uint32 words."""
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return np.array(list(o), dtype=np.uint32)


def noise3(seed: int, step: int, particle: int) -> np.ndarray:
    g = np.zeros(3)
    lib().orc_noise3(seed, step, particle, _dp(g))
    return g


def mb(x: float, y: float):
    """Mueller-Brown energy and force (fx, fy)."""
    fx, fy = C.c_double(), C.c_double()
    u = lib().orc_mb(x, y, C.byref(fx), C.byref(fy))
    return u, np.array([fx.value, fy.value])


def wells3(r):
    """Three-well test landscape: energy and force [3] at r [3]."""
    r = _f64(np.asarray(r, float).reshape(3))
    f = np.zeros(3)
    u = lib().orc_wells3(_dp(r), _dp(f))
    return u, f


def lj(x, box, eps=1.0, sig=1.0, rc=2.5):
    """All-pairs Lennard-Jones energy and forces (minimum image, cut at rc)."""
    x = _f64(x)
    f = np.zeros_like(x)
    b = _f64(box if box is not None else [0, 0, 0])
    u = lib().orc_lj(x.shape[0], _dp(x), _dp(b), eps, sig, rc, _dp(f))
    return u, f


def chain(x, kb=100.0, r0=1.0, ka=50.0, th0=np.deg2rad(109.47), kt=1.0):
    x = _f64(x)
    f = np.zeros_like(x)
    u = lib().orc_chain(x.shape[0], _dp(x), kb, r0, ka, th0, kt, _dp(f))
    return u, f


@dataclass
class CV:
    """One collective variable (Sec. 2.2).  Indices are walker-local."""
    kind: int
    a: np.ndarray | None = None  # None = all atoms of the walker
    b: np.ndarray | None = None
    axis: int = 0
    r0: float = 1.5
    nn: int = 6
    mm: int = 12
    scale: float = 0.0
    flags: int = 0
    period: float = 0.0
    _keep: list = field(default_factory=list, repr=False)

    def to_c(self) -> _CV:
        c = _CV()
        c.kind, c.axis, c.r0, c.nn, c.mm = self.kind, self.axis, self.r0, self.nn, self.mm
        c.scale, c.flags, c.period = self.scale, self.flags, self.period
        for nm in ("a", "b"):
            arr = getattr(self, nm)
            if arr is None:
                setattr(c, "n_" + nm, -1)
            else:
                arr = np.ascontiguousarray(np.asarray(arr, dtype=np.int32))
                self._keep.append(arr)
                setattr(c, "n_" + nm, arr.size)
                setattr(c, nm, arr.ctypes.data_as(C.POINTER(C.c_int32)))
        return c


def cv_eval(cv: CV, x, box=None):
    """xi and its dense Jacobian d xi / d x  ([n][3]) for one walker."""
    x = _f64(x)
    J = np.zeros_like(x)
    xi = C.c_double()
    b = _f64(box if box is not None else [0, 0, 0])
    c = cv.to_c()
    rc = lib().orc_cv_eval(C.byref(c), x.shape[0], _dp(x), _dp(b), C.byref(xi), _dp(J))
    if rc != 0:
        raise ValueError("bad CV")
    return xi.value, J


def hills_sum(xi, hills, sigma, period=None):
    """Bias V and dV/dxi at points xi [P][d] over hills [H][4] (Sec. 2.1.5)."""
    xi = _f64(np.atleast_2d(xi))
    P, d = xi.shape
    hills = _f64(hills).reshape(-1, 4)
    sig = _f64(list(sigma) + [1.0] * (3 - len(sigma)))
    per = _f64((list(period) if period is not None else [0.0] * d) + [0.0] * (3 - d))
    V = np.zeros(P)
    dV = np.zeros((P, d))
    lib().orc_hills_sum(d, P, _dp(xi), hills.shape[0], _dp(hills), _dp(sig), _dp(per), _dp(V), _dp(dV))
    return V, dV


def wt_height(V, w0, kT, gamma):
    return lib().orc_wt_height(V, w0, kT, gamma)


def grid_add(grid, bins, lo, hi, sigma, s, w, period=None):
    d = len(bins)
    b = (C.c_int64 * 3)(*(list(bins) + [1] * (3 - d)))
    pad = lambda v, fill: _f64(list(v) + [fill] * (3 - d))
    per = pad(period if period is not None else [0.0] * d, 0.0)
    assert grid.dtype == np.float64 and grid.flags.c_contiguous
    lib().orc_grid_add(d, b, _dp(pad(lo, 0.0)), _dp(pad(hi, 1.0)), _dp(per), _dp(pad(sigma, 1.0)),
                       _dp(pad(s, 0.0)), w, _dp(grid))


def grid_interp(grid, bins, lo, hi, xi, period=None):
    """Bias V and dV/dxi at points xi [P][d] read from a grid of V (Sec. 2.1.5,
    bias stored on a pre-defined grid): central-difference node gradients and
    multilinear interpolation of V and of the gradient (reading stated in
    wtmd_oracle.c, orc_grid_interp)."""
    xi = _f64(np.atleast_2d(xi))
    P, d = xi.shape
    b = (C.c_int64 * 3)(*(list(bins) + [1] * (3 - d)))
    pad = lambda v, fill: _f64(list(v) + [fill] * (3 - d))
    per = pad(period if period is not None else [0.0] * d, 0.0)
    g = _f64(grid).reshape(-1)
    V = np.zeros(P)
    dV = np.zeros((P, d))
    if lib().orc_grid_interp(d, b, _dp(pad(lo, 0.0)), _dp(pad(hi, 1.0)), _dp(per), _dp(g), P, _dp(xi), _dp(V),
                             _dp(dV)) != 0:
        raise ValueError("grid_interp: every axis needs at least 2 cells")
    return V, dV


def fes(grid, gamma):
    g = _f64(grid)
    out = np.zeros_like(g)
    lib().orc_fes(g.size, _dp(g), gamma, _dp(out))
    return out


def grid_centres(bins, lo, hi):
    """Cell-centre coordinates of each grid axis."""
    return [lo[i] + (np.arange(bins[i]) + 0.5) * (hi[i] - lo[i]) / bins[i] for i in range(len(bins))]


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


# --------------------------------------------------------------------------
# Whole system
# --------------------------------------------------------------------------
@dataclass
class System:
    """Engine + WTMD method parameters for the oracle's step loop."""
    engine: int
    walker_n: list
    cvs: list
    dims: int = 3
    box: tuple = (0.0, 0.0, 0.0)
    dt: float = 1e-3
    friction: float = 1.0
    mass: float = 1.0
    kT: float = 1.0
    seed: int = 0
    lj_eps: float = 1.0
    lj_sig: float = 1.0
    lj_rc: float = 2.5
    bond_k: float = 100.0
    bond_r0: float = 1.0
    angle_k: float = 50.0
    angle_t0: float = float(np.deg2rad(109.47))
    tors_k: float = 1.0
    harm_k: float = 1.0
    sigma: tuple = (0.1, 0.1, 0.1)
    w0: float = 1.0
    gamma: float = 10.0
    stride: int = 100
    hill_cap: int = 100000
    grid_bins: tuple = (0, 0, 0)
    grid_lo: tuple = (0.0, 0.0, 0.0)
    grid_hi: tuple = (1.0, 1.0, 1.0)
    bias_on: bool = True
    bias_grid: bool = False
    umb_k: tuple | None = None         # harmonic bias: spring constant per CV (None: metadynamics)
    umb_centres: object = None         # [W][d] window centres


class Sim:
    """Oracle simulation state; arrays are numpy float64, positions [N][3]."""

    def __init__(self, sys: System, x, v=None, hills=None):
        self.sys = sys
        W = len(sys.walker_n)
        self._wn = np.ascontiguousarray(np.asarray(sys.walker_n, dtype=np.int64))
        self._wo = np.ascontiguousarray(np.concatenate([[0], np.cumsum(self._wn)[:-1]]).astype(np.int64))
        N = int(self._wn.sum())
        self.x = _f64(x).reshape(N, 3).copy()
        self.v = np.zeros((N, 3)) if v is None else _f64(v).reshape(N, 3).copy()
        self.f = np.zeros((N, 3))
        self.hills = np.zeros((sys.hill_cap, 4))
        self.n_hills = 0
        if hills is not None:
            h = _f64(hills).reshape(-1, 4)
            self.hills[: h.shape[0]] = h
            self.n_hills = h.shape[0]
        nb = [b for b in sys.grid_bins if b > 0]
        self.grid = np.zeros(int(np.prod(nb))) if nb else np.zeros(1)
        self.xi = np.zeros((W, 3))
        self.V = np.zeros(W)
        self.dV = np.zeros((W, 3))
        self.step = 0
        self._cvs = [c.to_c() for c in sys.cvs]
        self._cvarr = (_CV * max(1, len(self._cvs)))(*self._cvs)
        s = _Sys()
        s.engine, s.dims, s.n_walkers = sys.engine, sys.dims, W
        s.walker_off = self._wo.ctypes.data_as(C.POINTER(C.c_int64))
        s.walker_n = self._wn.ctypes.data_as(C.POINTER(C.c_int64))
        s.box = (C.c_double * 3)(*sys.box)
        for nm in ("dt", "friction", "mass", "kT", "lj_eps", "lj_sig", "lj_rc", "bond_k", "bond_r0", "angle_k",
                   "angle_t0", "tors_k", "harm_k", "w0", "gamma"):
            setattr(s, nm, float(getattr(sys, nm)))
        s.seed = int(sys.seed)
        s.n_cv = len(sys.cvs)
        s.cv = C.cast(self._cvarr, C.POINTER(_CV))
        s.sigma = (C.c_double * 3)(*(list(sys.sigma) + [1.0] * (3 - len(sys.sigma))))
        s.stride, s.hill_cap = int(sys.stride), int(sys.hill_cap)
        s.grid_bins = (C.c_int64 * 3)(*(list(sys.grid_bins) + [0] * (3 - len(sys.grid_bins))))
        s.grid_lo = (C.c_double * 3)(*(list(sys.grid_lo) + [0.0] * (3 - len(sys.grid_lo))))
        s.grid_hi = (C.c_double * 3)(*(list(sys.grid_hi) + [1.0] * (3 - len(sys.grid_hi))))
        s.bias_on = 1 if sys.bias_on else 0
        s.bias_grid = 1 if sys.bias_grid else 0
        self.xi_sum = np.zeros((W, 3))
        self.n_samples = 0
        if sys.umb_k is not None:
            d = len(sys.cvs)
            s.bias_harm = 1
            s.harm_kcv = (C.c_double * 3)(*(list(sys.umb_k) + [0.0] * (3 - len(sys.umb_k))))
            cen = np.zeros((W, 3))
            cen[:, :d] = np.asarray(sys.umb_centres, dtype=np.float64).reshape(W, d)
            self._centres = np.ascontiguousarray(cen)
            s.harm_centre = _dp(self._centres)
        self._sys = s

    def _state(self) -> _State:
        st = _State()
        st.x, st.v, st.f = _dp(self.x), _dp(self.v), _dp(self.f)
        st.hills, st.n_hills = _dp(self.hills), self.n_hills
        st.grid = _dp(self.grid)
        st.step = self.step
        st.xi, st.V, st.dV = _dp(self.xi), _dp(self.V), _dp(self.dV)
        st.xi_sum, st.n_samples = _dp(self.xi_sum), self.n_samples
        return st

    def _pull(self, st: _State):
        self.n_hills = st.n_hills
        self.step = st.step
        self.n_samples = st.n_samples

    def umbrella(self):
        """Umbrella integration over the windows' statistics (Sec. 2.1.2):
        (mean xi [W][d], mean force dA/dxi [W][d], A along the path [W])."""
        d = len(self.sys.cvs)
        W = len(self._wn)
        mean = np.ascontiguousarray(self.xi_sum / max(self.n_samples, 1))
        per = _f64([c.period for c in self.sys.cvs] + [0.0] * (3 - d))
        k = _f64(list(self.sys.umb_k) + [0.0] * (3 - d))
        g, A = np.zeros((W, 3)), np.zeros(W)
        lib().orc_umbrella_integrate(W, d, _dp(mean), _dp(self._centres), _dp(k), _dp(per), _dp(g), _dp(A))
        return mean[:, :d], g[:, :d], A

    def forces(self):
        st = self._state()
        if lib().orc_forces(C.byref(self._sys), C.byref(st)) != 0:
            raise ValueError("oracle forces failed")
        self._pull(st)
        return self.f

    def run(self, n: int) -> int:
        st = self._state()
        rc = lib().orc_run(C.byref(self._sys), C.byref(st), int(n))
        self._pull(st)
        return rc

    def bias(self, x, f=None, hills=None):
        """One bias evaluation at x: returns (f - J^T dV, xi [W][3], V [W], dV [W][3])."""
        x = _f64(x).reshape(-1, 3)
        f = np.zeros_like(x) if f is None else _f64(f).reshape(-1, 3).copy()
        h = self.hills[: self.n_hills] if hills is None else _f64(hills).reshape(-1, 4)
        h = np.ascontiguousarray(h)
        W = len(self._wn)
        xi, V, dV = np.zeros((W, 3)), np.zeros(W), np.zeros((W, 3))
        if lib().orc_bias(C.byref(self._sys), _dp(x), _dp(h), h.shape[0], _dp(f), _dp(xi), _dp(V), _dp(dV)) != 0:
            raise ValueError("oracle bias failed")
        return f, xi, V, dV

    def bias_grid(self, x, f=None, grid=None):
        """One bias evaluation at x with V and dV/dxi read from the grid (the
        current one, or `grid`): returns (f - J^T dV, xi [W][3], V [W], dV [W][3])."""
        x = _f64(x).reshape(-1, 3)
        f = np.zeros_like(x) if f is None else _f64(f).reshape(-1, 3).copy()
        g = self.grid if grid is None else _f64(grid).reshape(-1)
        W = len(self._wn)
        xi, V, dV = np.zeros((W, 3)), np.zeros(W), np.zeros((W, 3))
        if lib().orc_bias_grid(C.byref(self._sys), _dp(x), _dp(g), _dp(f), _dp(xi), _dp(V), _dp(dV)) != 0:
            raise ValueError("oracle grid bias failed")
        return f, xi, V, dV

    def fes(self):
        return fes(self.grid, self.sys.gamma)
