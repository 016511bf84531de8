"""Python binding of libwtmd, the B300 well-tempered metadynamics library.

Argument marshalling only: every step of the bias-force path runs in the
CUDA kernels of libwtmd.so (built from csrc/ by `build.py`).  PyTorch
provides device memory and the stream; there is no CPU fallback -- importing
the binding without the built library raises.

    import paper_2301_04835_b300 as wt
    m = wt.Wtmd(precision="f32", sigma=(0.05, 0.1), w0=1.0, gamma=8.0, kT=1.0,
                stride=100, capacity=100000, walker_sizes=[N], engine="lj",
                box=(L, L, L), dt=0.005)
    m.cv_define(wt.CV_COORDINATION, a=tagged, r0=1.5, nn=6, mm=12)
    m.cv_define(wt.CV_RG, a=subset)
    m.bind(pos, vel, force)          # torch CUDA tensors [N, 4]
    m.step_n(1000)
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libwtmd.so")

OK, EINVAL, ENOMEM, ECAPACITY, ENUMERIC, ETIMEOUT, ECUDA, ECELL = 0, -1, -2, -3, -4, -5, -6, -7
F32, F64 = 0, 1
ENGINE_NONE, ENGINE_MB, ENGINE_LJ, ENGINE_CHAIN = 0, 1, 2, 3
CV_COMPONENT, CV_DIHEDRAL, CV_COORDINATION, CV_RG, CV_QPAIRS = 1, 2, 3, 4, 5
CV_DISTANCE, CV_ANGLE, CV_GYRATION = 6, 7, 8
GY_L1, GY_L2, GY_L3, GY_ASPHERICITY, GY_ACYLINDRICITY, GY_ANISOTROPY = 0, 1, 2, 3, 4, 5
CV_INTENSIVE = 1
ENGINE_WELLS3 = 5
_ENGINES = {"none": ENGINE_NONE, "mb": ENGINE_MB, "lj": ENGINE_LJ, "chain": ENGINE_CHAIN, "wells3": ENGINE_WELLS3}


class WtmdError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libwtmd error {code}: {msg}")
        self.code = code


class Config(C.Structure):
    """Mirror of wtmd_config (include/wtmd.h)."""
    _fields_ = [
        ("precision", C.c_int32), ("n_cv", C.c_int32), ("sigma", C.c_double * 3), ("w0", C.c_double),
        ("gamma", C.c_double), ("kT", C.c_double), ("stride", C.c_int64), ("hill_capacity", C.c_int64),
        ("seed", C.c_uint64), ("grid_bins", C.c_int32 * 3), ("engine", C.c_int32),
        ("grid_lo", C.c_double * 3), ("grid_hi", C.c_double * 3), ("dims", C.c_int32), ("n_walkers", C.c_int32),
        ("walker_size", C.POINTER(C.c_int64)), ("dt", C.c_double), ("friction", C.c_double), ("mass", C.c_double),
        ("box", C.c_double * 3), ("lj_eps", C.c_double), ("lj_sigma", C.c_double), ("lj_rc", C.c_double),
        ("bond_k", C.c_double), ("bond_r0", C.c_double), ("angle_k", C.c_double), ("angle_theta0", C.c_double),
        ("torsion_k", C.c_double),
    ]


class CvDesc(C.Structure):
    """Mirror of wtmd_cv_desc (include/wtmd.h)."""
    _fields_ = [
        ("kind", C.c_int32), ("axis", C.c_int32), ("n_a", C.c_int64), ("a", C.POINTER(C.c_int32)),
        ("n_b", C.c_int64), ("b", C.POINTER(C.c_int32)), ("r0", C.c_double), ("nn", C.c_int32), ("mm", C.c_int32),
        ("scale", C.c_double), ("flags", C.c_int32), ("reserved", C.c_int32), ("period", C.c_double),
    ]


EXPORTS = ["wtmd_create", "wtmd_destroy", "wtmd_last_error", "wtmd_set_stream", "cv_define", "wtmd_bind", "step_n",
           "wtmd_check", "bias_eval", "hills_eval", "fes_grid", "wtmd_hills_load", "wtmd_hills_read",
           "wtmd_counters", "wtmd_grid_read", "wtmd_philox", "wtmd_profile_step", "wtmd_probe_peak",
           "wtmd_hills_eval_static", "wtmd_cv_forward", "wtmd_cv_adjoint", "wtmd_walkers_persistent",
           "wtmd_autotune", "wtmd_surrogate", "wtmd_surrogate_config", "wtmd_surrogate_fit", "wtmd_surrogate_status",
           "wtmd_surrogate_set", "wtmd_mlp_params", "wtmd_mlp_eval", "wtmd_mlp_grad", "wtmd_mlp_train", "wtmd_hills_tune",
           "wtmd_grid_eval", "wtmd_bias_source", "wtmd_checkpoint_size", "wtmd_checkpoint_save",
           "wtmd_checkpoint_load", "wtmd_harmonic", "wtmd_umbrella_stats", "wtmd_umbrella_integrate",
           "wtmd_step_host", "wtmd_fused_step", "wtmd_small_step", "wtmd_hills_plan", "wtmd_wait_limit", "wtmd_barrier_probe"]

BIAS_HILLS, BIAS_GRID, BIAS_HARMONIC = 0, 1, 2

MLP_PARAMS = 4481

_lib = None


def lib() -> C.CDLL:
    """Load libwtmd.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2301_04835_b300.build`")
    L = C.CDLL(LIB_PATH)
    vp, i64, i32 = C.c_void_p, C.c_int64, C.c_int32
    L.wtmd_create.argtypes = [C.POINTER(Config), C.POINTER(vp)]
    L.wtmd_destroy.argtypes = [vp]
    L.wtmd_last_error.argtypes = [vp]
    L.wtmd_last_error.restype = C.c_char_p
    L.wtmd_set_stream.argtypes = [vp, vp]
    L.cv_define.argtypes = [vp, C.POINTER(CvDesc), C.POINTER(i32)]
    L.wtmd_bind.argtypes = [vp, vp, vp, vp, i64]
    L.step_n.argtypes = [vp, i64]
    L.wtmd_check.argtypes = [vp]
    L.bias_eval.argtypes = [vp, vp, vp, vp, vp, vp]
    L.hills_eval.argtypes = [vp, vp, i64, vp, vp]
    L.fes_grid.argtypes = [vp, vp, i64]
    L.wtmd_hills_load.argtypes = [vp, C.POINTER(C.c_double), i64]
    L.wtmd_hills_read.argtypes = [vp, C.POINTER(C.c_double), i64, C.POINTER(i64)]
    L.wtmd_counters.argtypes = [vp, C.POINTER(i64), C.POINTER(i64)]
    L.wtmd_grid_read.argtypes = [vp, C.POINTER(C.c_double), i64]
    L.wtmd_philox.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), i64]
    L.wtmd_profile_step.argtypes = [vp, i64, C.c_char_p, C.POINTER(C.c_double), i32, C.POINTER(i32)]
    L.wtmd_probe_peak.argtypes = [i32, C.POINTER(C.c_double), C.POINTER(C.c_double)]
    L.wtmd_walkers_persistent.argtypes = [vp, i32]
    L.wtmd_fused_step.argtypes = [vp, i32, C.POINTER(i32)]
    L.wtmd_small_step.argtypes = [vp, i32, C.POINTER(i32)]
    L.wtmd_hills_plan.argtypes = [vp, i64, i32, i32]
    L.wtmd_wait_limit.argtypes = [vp, i64]
    L.wtmd_barrier_probe.argtypes = [i32, i32, i64, C.POINTER(i32)]
    L.wtmd_autotune.argtypes = [vp, i64, C.POINTER(i32)]
    dp, fp = C.POINTER(C.c_double), C.POINTER(C.c_float)
    L.wtmd_surrogate.argtypes = [vp, i32, C.c_double, i64]
    L.wtmd_surrogate_config.argtypes = [vp, i64, i64, i64, C.c_double, C.c_double]
    L.wtmd_surrogate_fit.argtypes = [vp, dp]
    L.wtmd_surrogate_status.argtypes = [vp, dp]
    L.wtmd_surrogate_set.argtypes = [vp, i64, i32]
    L.wtmd_mlp_params.argtypes = [vp, fp, fp, dp, dp]
    L.wtmd_mlp_eval.argtypes = [vp, vp, i64, vp, vp]
    L.wtmd_mlp_grad.argtypes = [vp, vp, vp, vp, i64, C.c_double, vp]
    L.wtmd_mlp_train.argtypes = [vp, vp, vp, vp, i64, i64, i64, C.c_double, C.c_double, vp]
    L.wtmd_hills_tune.argtypes = [vp, i64, C.POINTER(i32), C.POINTER(C.c_double)]
    L.wtmd_grid_eval.argtypes = [vp, vp, i64, vp, vp]
    L.wtmd_bias_source.argtypes = [vp, i32]
    L.wtmd_checkpoint_size.argtypes = [vp, C.POINTER(i64)]
    L.wtmd_checkpoint_save.argtypes = [vp, vp, i64]
    L.wtmd_checkpoint_load.argtypes = [vp, vp, i64]
    L.wtmd_harmonic.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_double)]
    L.wtmd_step_host.argtypes = [vp, vp, vp, i64, i32]
    L.wtmd_umbrella_stats.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(i64), i32]
    L.wtmd_umbrella_integrate.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_double)]
    L.wtmd_cv_forward.argtypes = [vp, vp, vp]
    L.wtmd_cv_adjoint.argtypes = [vp, vp, vp]
    L.wtmd_hills_eval_static.argtypes = [i32, C.POINTER(C.c_double), C.POINTER(C.c_double), vp, i64, vp, i64, vp,
                                         vp, vp]
    for name in EXPORTS:
        if not hasattr(L, name):
            raise ImportError(f"libwtmd.so lacks {name}")
        if name != "wtmd_last_error":
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _torch():
    import torch
    return torch


def philox(ctr_key: np.ndarray) -> np.ndarray:
    """Philox4x32-10 on the device: [n][6] uint32 (ctr0..3, key0..1) -> [n][4]."""
    a = np.ascontiguousarray(ctr_key, dtype=np.uint32)
    out = np.zeros((a.shape[0], 4), dtype=np.uint32)
    rc = lib().wtmd_philox(a.ctypes.data_as(C.POINTER(C.c_uint32)), out.ctypes.data_as(C.POINTER(C.c_uint32)),
                           a.shape[0])
    if rc:
        raise WtmdError(rc, "wtmd_philox")
    return out


class Wtmd:
    """One WTMD handle (wtmd_t).  Tensors passed in are CUDA tensors of the
    handle's precision, [n_atoms, 4] for particle arrays."""

    def __init__(self, *, precision="f32", sigma, w0=1.0, gamma=10.0, kT=1.0, stride=100, capacity=100000,
                 seed=0, grid=None, engine="none", dims=0, walker_sizes, dt=1e-3, friction=1.0, mass=1.0,
                 box=(0.0, 0.0, 0.0), lj=(1.0, 1.0, 2.5), chain=(100.0, 1.0, 50.0, float(np.deg2rad(109.47)), 1.0)):
        torch = _torch()
        self.prec = F32 if precision in ("f32", F32) else F64
        self.dtype = torch.float32 if self.prec == F32 else torch.float64
        self.d = len(sigma)
        self.W = len(walker_sizes)
        self.N = int(np.sum(walker_sizes))
        self._ws = (C.c_int64 * self.W)(*[int(v) for v in walker_sizes])
        c = Config()
        c.precision, c.n_cv = self.prec, self.d
        c.sigma = (C.c_double * 3)(*(list(sigma) + [1.0] * (3 - self.d)))
        c.w0, c.gamma, c.kT = w0, gamma, kT
        c.stride, c.hill_capacity, c.seed = int(stride), int(capacity), int(seed)
        if grid is not None:
            bins, lo, hi = grid
            c.grid_bins = (C.c_int32 * 3)(*(list(bins) + [0] * (3 - len(bins))))
            c.grid_lo = (C.c_double * 3)(*(list(lo) + [0.0] * (3 - len(lo))))
            c.grid_hi = (C.c_double * 3)(*(list(hi) + [1.0] * (3 - len(hi))))
            self.grid_shape = tuple(bins)
        else:
            self.grid_shape = None
        c.engine = _ENGINES[engine] if isinstance(engine, str) else int(engine)
        c.dims, c.n_walkers = int(dims), self.W
        c.walker_size = C.cast(self._ws, C.POINTER(C.c_int64))
        c.dt, c.friction, c.mass = dt, friction, mass
        c.box = (C.c_double * 3)(*box)
        c.lj_eps, c.lj_sigma, c.lj_rc = lj
        c.bond_k, c.bond_r0, c.angle_k, c.angle_theta0, c.torsion_k = chain
        self.cfg = c
        h = C.c_void_p()
        torch.cuda.init()
        rc = lib().wtmd_create(C.byref(c), C.byref(h))
        if rc:
            raise WtmdError(rc, "wtmd_create rejected the configuration")
        self.h = h
        self._keep = []

    # ------------------------------------------------------------------
    def _err(self, rc, what):
        if rc:
            msg = lib().wtmd_last_error(self.h)
            raise WtmdError(rc, f"{what}: {msg.decode() if msg else ''}")

    def _stream(self):
        s = _torch().cuda.current_stream().cuda_stream
        lib().wtmd_set_stream(self.h, C.c_void_p(s))

    def close(self):
        if getattr(self, "h", None):
            lib().wtmd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check_tensor(self, t, shape=None):
        torch = _torch()
        if t is None:
            return None
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == self.dtype and t.is_contiguous()):
            raise TypeError(f"expected a contiguous CUDA {self.dtype} tensor")
        if shape is not None and tuple(t.shape) != tuple(shape):
            raise ValueError(f"expected shape {shape}, got {tuple(t.shape)}")
        return C.c_void_p(t.data_ptr())

    @staticmethod
    def _dev(t, shape, dtype):
        """Validate a contiguous CUDA tensor of `dtype`; None in `shape` matches any size."""
        torch = _torch()
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()):
            raise TypeError(f"expected a contiguous CUDA {dtype} tensor")
        if len(t.shape) != len(shape) or any(w is not None and w != g for w, g in zip(shape, t.shape)):
            raise ValueError(f"expected shape {shape}, got {tuple(t.shape)}")
        return t

    # ------------------------------------------------------------------
    def cv_define(self, kind, a=None, b=None, axis=0, r0=1.5, nn=6, mm=12, scale=0.0, flags=0, period=0.0) -> int:
        d = CvDesc()
        d.kind, d.axis, d.r0, d.nn, d.mm, d.scale, d.flags, d.period = kind, axis, r0, nn, mm, scale, flags, period
        for nm in ("a", "b"):
            arr = locals()[nm]
            if arr is None:
                setattr(d, "n_" + nm, -1)
            else:
                arr = np.ascontiguousarray(np.asarray(arr, dtype=np.int32))
                self._keep.append(arr)
                setattr(d, "n_" + nm, arr.size)
                setattr(d, nm, arr.ctypes.data_as(C.POINTER(C.c_int32)))
        cid = C.c_int32()
        self._err(lib().cv_define(self.h, C.byref(d), C.byref(cid)), "cv_define")
        return cid.value

    def bind(self, pos, vel, force):
        self._bound = (pos, vel, force)
        self._err(lib().wtmd_bind(self.h, self._check_tensor(pos, (self.N, 4)), self._check_tensor(vel, (self.N, 4)),
                                  self._check_tensor(force, (self.N, 4)), self.N), "wtmd_bind")

    def step_n(self, n: int, check: bool = True):
        self._stream()
        self._err(lib().step_n(self.h, int(n)), "step_n")
        if check:
            self.check()

    def step_host(self, state_in, state_out=None, n: int = 1, wait: bool = True):
        """n steps with the state [3][N][4] (positions, velocities, forces) in
        host memory: a CPU tensor or array, pinned for the single-graph path;
        state_out defaults to state_in."""
        self._stream()
        out = state_in if state_out is None else state_out

        def ptr(a):
            return a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data

        self._err(lib().wtmd_step_host(self.h, C.c_void_p(ptr(state_in)), C.c_void_p(ptr(out)), int(n),
                                       1 if wait else 0), "wtmd_step_host")

    def check(self):
        self._stream()
        self._err(lib().wtmd_check(self.h), "wtmd_check")

    def bias_eval(self, pos, force=None):
        """Returns (V [W], xi [W, d], dV [W, d]); force (if given) -= J^T dV."""
        torch = _torch()
        self._stream()
        V = torch.empty(self.W, dtype=self.dtype, device=pos.device)
        xi = torch.empty(self.W, self.d, dtype=self.dtype, device=pos.device)
        dV = torch.empty(self.W, self.d, dtype=self.dtype, device=pos.device)
        self._err(lib().bias_eval(self.h, self._check_tensor(pos, (self.N, 4)),
                                  self._check_tensor(force, (self.N, 4)) if force is not None else None,
                                  C.c_void_p(V.data_ptr()), C.c_void_p(xi.data_ptr()), C.c_void_p(dV.data_ptr())),
                  "bias_eval")
        return V, xi, dV

    def hills_tune(self, P: int):
        """Time the hills-sum plans for P points and keep the fastest; returns
        (lanes per point, splits, ms per sum)."""
        self._stream()
        ch = (C.c_int32 * 2)()
        ms = C.c_double()
        self._err(lib().wtmd_hills_tune(self.h, int(P), ch, C.byref(ms)), "wtmd_hills_tune")
        return ch[0], ch[1], ms.value

    def fused_step(self, enable=None) -> bool:
        """Allow (True) or forbid (False, the default) the single-launch
        persistent step (None leaves the setting); returns whether the next
        step uses it."""
        act = C.c_int32()
        self._err(lib().wtmd_fused_step(self.h, -1 if enable is None else (1 if enable else 0), C.byref(act)),
                  "wtmd_fused_step")
        return bool(act.value)

    def small_step(self, enable=None) -> bool:
        """Allow (True, the default) or forbid (False) the single-CTA
        many-steps launch for small FP64 analytic systems (None leaves the
        setting); returns whether the next step uses it."""
        act = C.c_int32()
        self._err(lib().wtmd_small_step(self.h, -1 if enable is None else (1 if enable else 0), C.byref(act)),
                  "wtmd_small_step")
        return bool(act.value)

    def hills_plan(self, P: int, lanes: int, splits: int):
        """Set the hills-sum plan for P points (lanes per point 1/4/32/256,
        0 = few-points kernel, -1 = cluster kernel; splits)."""
        self._err(lib().wtmd_hills_plan(self.h, int(P), int(lanes), int(splits)), "wtmd_hills_plan")

    def wait_limit(self, cycles: int = 0):
        """Grid-barrier wait bound of the persistent launches (SM cycles; 0 = default)."""
        self._err(lib().wtmd_wait_limit(self.h, int(cycles)), "wtmd_wait_limit")

    def walkers_persistent(self, enable: bool = True):
        """Run each step as one persistent launch over all walkers."""
        self._err(lib().wtmd_walkers_persistent(self.h, 1 if enable else 0), "wtmd_walkers_persistent")

    def autotune(self, steps: int = 5):
        """Pick the persistent step's tiles by timing; returns (T, CTAs/SM, split factor)."""
        self._stream()
        ch = (C.c_int32 * 3)()
        self._err(lib().wtmd_autotune(self.h, int(steps), ch), "wtmd_autotune")
        return tuple(ch)

    # ---- MLP surrogate of the hills sum ----
    _STATS = ("K", "rms_kT", "max_kT", "grad_rel_rms", "loss", "active", "fits", "iters")

    def surrogate(self, enable: bool = True, tol_kT: float = 0.05, retrain_every: int = 10000):
        """Network for the older hills + exact tail, refitted every `retrain_every` hills."""
        self._stream()
        self._err(lib().wtmd_surrogate(self.h, 1 if enable else 0, float(tol_kT), int(retrain_every)),
                  "wtmd_surrogate")

    def surrogate_config(self, n_samples=65540, iters=80000, batch=4096, lr=6e-3, lam=0.1):
        self._err(lib().wtmd_surrogate_config(self.h, int(n_samples), int(iters), int(batch), float(lr), float(lam)),
                  "wtmd_surrogate_config")

    def surrogate_fit(self) -> dict:
        self._stream()
        st = (C.c_double * 8)()
        self._err(lib().wtmd_surrogate_fit(self.h, st), "wtmd_surrogate_fit")
        return dict(zip(self._STATS, list(st)))

    def surrogate_status(self) -> dict:
        st = (C.c_double * 8)()
        self._err(lib().wtmd_surrogate_status(self.h, st), "wtmd_surrogate_status")
        return dict(zip(self._STATS, list(st)))

    def surrogate_set(self, k0: int, active: bool = True):
        self._stream()
        self._err(lib().wtmd_surrogate_set(self.h, int(k0), 1 if active else 0), "wtmd_surrogate_set")

    def mlp_params(self, params=None, norm=None):
        """Load (if given) and return (FP32 master weights [4481], norm [8])."""
        self._stream()
        fp, dp = C.POINTER(C.c_float), C.POINTER(C.c_double)
        pin = None
        if params is not None:
            pin = np.ascontiguousarray(np.asarray(params, dtype=np.float32).reshape(MLP_PARAMS))
        nin = None if norm is None else np.ascontiguousarray(np.asarray(norm, dtype=np.float64).reshape(8))
        out = np.zeros(MLP_PARAMS, dtype=np.float32)
        nout = np.zeros(8)
        self._err(lib().wtmd_mlp_params(self.h, pin.ctypes.data_as(fp) if pin is not None else None,
                                        out.ctypes.data_as(fp), nin.ctypes.data_as(dp) if nin is not None else None,
                                        nout.ctypes.data_as(dp)), "wtmd_mlp_params")
        return out, nout

    def mlp_eval(self, xi):
        """V_nn [P] and dV_nn/dxi [P][d] (float32) at CV points xi (CUDA FP64 [P][d])."""
        torch = _torch()
        self._stream()
        xi = self._dev(xi, (None, self.d), torch.float64)
        P = xi.shape[0]
        V = torch.empty(P, dtype=torch.float32, device=xi.device)
        dV = torch.empty(P, self.d, dtype=torch.float32, device=xi.device)
        self._err(lib().wtmd_mlp_eval(self.h, C.c_void_p(xi.data_ptr()), P, C.c_void_p(V.data_ptr()),
                                      C.c_void_p(dV.data_ptr())), "wtmd_mlp_eval")
        return V, dV

    def mlp_grad(self, x, V, G, lam):
        """Sobolev-loss gradient [4481] and loss over one batch (x FP64 [B][3], V [B], G [B][3] FP32)."""
        torch = _torch()
        self._stream()
        x = self._dev(x, (None, 3), torch.float64)
        B = x.shape[0]
        V = self._dev(V, (B,), torch.float32)
        G = self._dev(G, (B, 3), torch.float32)
        out = torch.empty(MLP_PARAMS + 1, dtype=torch.float32, device=x.device)
        self._err(lib().wtmd_mlp_grad(self.h, C.c_void_p(x.data_ptr()), C.c_void_p(V.data_ptr()),
                                      C.c_void_p(G.data_ptr()), B, float(lam), C.c_void_p(out.data_ptr())),
                  "wtmd_mlp_grad")
        return out[:MLP_PARAMS], out[MLP_PARAMS]

    def mlp_train(self, x, V, G, batch, iters, lr, lam):
        """`iters` Adam steps over cyclic batches of the given samples; returns the last loss (tensor)."""
        torch = _torch()
        self._stream()
        x = self._dev(x, (None, 3), torch.float64)
        n = x.shape[0]
        V = self._dev(V, (n,), torch.float32)
        G = self._dev(G, (n, 3), torch.float32)
        loss = torch.zeros(1, dtype=torch.float32, device=x.device)
        self._err(lib().wtmd_mlp_train(self.h, C.c_void_p(x.data_ptr()), C.c_void_p(V.data_ptr()),
                                       C.c_void_p(G.data_ptr()), n, int(batch), int(iters), float(lr), float(lam),
                                       C.c_void_p(loss.data_ptr())), "wtmd_mlp_train")
        return loss

    def cv_forward(self, pos):
        """CV values [W, d] at pos; keeps the Jacobians for cv_adjoint."""
        torch = _torch()
        self._stream()
        xi = torch.empty(self.W, self.d, dtype=self.dtype, device=pos.device)
        self._err(lib().wtmd_cv_forward(self.h, self._check_tensor(pos, (self.N, 4)), C.c_void_p(xi.data_ptr())),
                  "wtmd_cv_forward")
        self._gen = getattr(self, "_gen", 0) + 1
        return xi

    def cv_adjoint(self, grad_xi):
        """J^T grad_xi of the latest forward: [N, 4] (last column 0)."""
        torch = _torch()
        self._stream()
        g = grad_xi.to(self.dtype).contiguous()
        out = torch.empty(self.N, 4, dtype=self.dtype, device=g.device)
        self._err(lib().wtmd_cv_adjoint(self.h, self._check_tensor(g, (self.W, self.d)), C.c_void_p(out.data_ptr())),
                  "wtmd_cv_adjoint")
        return out

    def hills_eval(self, xi):
        torch = _torch()
        self._stream()
        P = xi.shape[0]
        V = torch.empty(P, dtype=self.dtype, device=xi.device)
        dV = torch.empty(P, self.d, dtype=self.dtype, device=xi.device)
        self._err(lib().hills_eval(self.h, self._check_tensor(xi, (P, self.d)), P, C.c_void_p(V.data_ptr()),
                                   C.c_void_p(dV.data_ptr())), "hills_eval")
        return V, dV

    def grid_eval(self, xi):
        """V and dV/dxi at points xi [P][n_cv] read from the FP64 bias grid
        (central-difference node gradients, multilinear interpolation)."""
        torch = _torch()
        self._stream()
        P = xi.shape[0]
        V = torch.empty(P, dtype=self.dtype, device=xi.device)
        dV = torch.empty(P, self.d, dtype=self.dtype, device=xi.device)
        self._err(lib().wtmd_grid_eval(self.h, self._check_tensor(xi, (P, self.d)), P, C.c_void_p(V.data_ptr()),
                                       C.c_void_p(dV.data_ptr())), "wtmd_grid_eval")
        return V, dV

    def grid_eval_into(self, xi, V, dV):
        """grid_eval into preallocated outputs (no allocation; for timing)."""
        self._err(lib().wtmd_grid_eval(self.h, C.c_void_p(xi.data_ptr()), xi.shape[0], C.c_void_p(V.data_ptr()),
                                       C.c_void_p(dV.data_ptr())), "wtmd_grid_eval")

    def bias_source(self, source: int):
        """Where step_n and bias_eval take the bias from: BIAS_HILLS (exact
        sum) or BIAS_GRID (read from the grid)."""
        self._err(lib().wtmd_bias_source(self.h, int(source)), "wtmd_bias_source")

    def harmonic(self, k, centres):
        """Harmonic windows: spring constants k [n_cv], centres [W][n_cv]."""
        kk = np.ascontiguousarray(np.asarray(k, dtype=np.float64).reshape(self.d))
        cc = np.ascontiguousarray(np.asarray(centres, dtype=np.float64).reshape(self.W, self.d))
        dp = C.POINTER(C.c_double)
        self._err(lib().wtmd_harmonic(self.h, kk.ctypes.data_as(dp), cc.ctypes.data_as(dp)), "wtmd_harmonic")

    def umbrella_stats(self, reset: bool = False):
        """(mean CVs [W][n_cv], samples) of the windows."""
        self._stream()
        mean = np.zeros((self.W, self.d))
        n = C.c_int64()
        self._err(lib().wtmd_umbrella_stats(self.h, mean.ctypes.data_as(C.POINTER(C.c_double)), C.byref(n),
                                            1 if reset else 0), "wtmd_umbrella_stats")
        return mean, n.value

    def umbrella_integrate(self):
        """(mean forces [W][n_cv], A along the window path [W])."""
        self._stream()
        g, A = np.zeros((self.W, self.d)), np.zeros(self.W)
        dp = C.POINTER(C.c_double)
        self._err(lib().wtmd_umbrella_integrate(self.h, g.ctypes.data_as(dp), A.ctypes.data_as(dp)),
                  "wtmd_umbrella_integrate")
        return g, A

    def checkpoint(self) -> bytes:
        """The run's state as bytes (hills, grid, counters, bound particle
        arrays); load it with restore() to resume bitwise."""
        n = C.c_int64()
        self._err(lib().wtmd_checkpoint_size(self.h, C.byref(n)), "wtmd_checkpoint_size")
        buf = C.create_string_buffer(n.value)
        self._err(lib().wtmd_checkpoint_save(self.h, buf, n.value), "wtmd_checkpoint_save")
        return buf.raw

    def restore(self, blob: bytes):
        """Load a checkpoint() of a handle with the same configuration."""
        buf = C.create_string_buffer(bytes(blob), len(blob))
        self._err(lib().wtmd_checkpoint_load(self.h, buf, len(blob)), "wtmd_checkpoint_load")

    def hills_eval_into(self, xi, V, dV):
        """hills_eval into preallocated outputs (no allocation; for timing)."""
        self._err(lib().hills_eval(self.h, C.c_void_p(xi.data_ptr()), xi.shape[0], C.c_void_p(V.data_ptr()),
                                   C.c_void_p(dV.data_ptr())), "hills_eval")

    def profile_step(self, n_steps: int = 20):
        """Mean device time per kernel of an MD step ({name: ms}), measured
        with CUDA events on the launching stream (eager launches)."""
        self._stream()
        cap = 64
        names = C.create_string_buffer(32 * cap)
        ms = (C.c_double * cap)()
        n = C.c_int32()
        self._err(lib().wtmd_profile_step(self.h, int(n_steps), names, ms, cap, C.byref(n)), "wtmd_profile_step")
        out = []
        for i in range(n.value):
            nm = names.raw[32 * i: 32 * i + 32].split(b"\0", 1)[0].decode()
            out.append((nm, ms[i]))
        return out

    def fes_grid(self):
        torch = _torch()
        self._stream()
        n = int(np.prod(self.grid_shape))
        out = torch.empty(n, dtype=torch.float64, device="cuda")
        self._err(lib().fes_grid(self.h, C.c_void_p(out.data_ptr()), n), "fes_grid")
        return out.reshape(self.grid_shape)

    def hills_load(self, hills):
        self._stream()
        h = np.ascontiguousarray(np.asarray(hills, dtype=np.float64).reshape(-1, 4))
        self._err(lib().wtmd_hills_load(self.h, h.ctypes.data_as(C.POINTER(C.c_double)), h.shape[0]),
                  "wtmd_hills_load")

    def hills_read(self) -> np.ndarray:
        self._stream()
        cnt = C.c_int64()
        self._err(lib().wtmd_hills_read(self.h, None, 0, C.byref(cnt)), "wtmd_hills_read")
        out = np.zeros((max(cnt.value, 1), 4))
        self._err(lib().wtmd_hills_read(self.h, out.ctypes.data_as(C.POINTER(C.c_double)), cnt.value, C.byref(cnt)),
                  "wtmd_hills_read")
        return out[: cnt.value]

    def counters(self):
        self._stream()
        s, c = C.c_int64(), C.c_int64()
        self._err(lib().wtmd_counters(self.h, C.byref(s), C.byref(c)), "wtmd_counters")
        return s.value, c.value

    def grid_read(self) -> np.ndarray:
        self._stream()
        n = int(np.prod(self.grid_shape))
        out = np.zeros(n)
        self._err(lib().wtmd_grid_read(self.h, out.ctypes.data_as(C.POINTER(C.c_double)), n), "wtmd_grid_read")
        return out.reshape(self.grid_shape)


def _cv_function():
    import torch

    class CVFunction(torch.autograd.Function):
        """xi = CVs(positions) with the hand-written adjoint as backward.

        Forward: pos [N, 3] (or [N, 4]) -> xi [W, d] through wtmd_cv_forward;
        backward: grad_pos = J^T grad_xi through the wtmd_cv_adjoint kernel.
        If another forward ran on the handle in between, the forward is
        recomputed at the saved positions first (the adjoint uses the
        handle's latest Jacobians)."""

        @staticmethod
        def forward(ctx, pos, handle):
            p4 = pos if pos.shape[-1] == 4 else torch.nn.functional.pad(pos, (0, 1))
            p4 = p4.detach().to(handle.dtype).contiguous()
            xi = handle.cv_forward(p4)
            ctx.handle, ctx.gen, ctx.ncol = handle, handle._gen, pos.shape[-1]
            ctx.save_for_backward(p4)
            return xi

        @staticmethod
        def backward(ctx, grad_xi):
            h = ctx.handle
            (p4,) = ctx.saved_tensors
            if h._gen != ctx.gen:
                h.cv_forward(p4)
            g = h.cv_adjoint(grad_xi)
            return g[:, : ctx.ncol].to(grad_xi.dtype), None

    return CVFunction


def load_config(name: str | None = None) -> dict:
    """The five workloads of this library as data (configs.json beside this
    module): method, engine and CV parameters and the recipe of the seeded
    synthetic inputs.  name: one of mueller_brown, lj4096, chain1024,
    walkers256, surrogate32768; None returns all of them."""
    import json

    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "configs.json")) as f:
        cfg = json.load(f)
    return cfg if name is None else cfg[name]


def cv_apply(pos, handle):
    """Differentiable CV evaluation: xi = cv_apply(pos, handle)."""
    return _cv_function().apply(pos, handle)


def probe_peak(kind: int):
    """Measured pipe throughput: kind 0 = MUFU ex2/s, 1 = FP32 FMA lane-ops/s."""
    v, ms = C.c_double(), C.c_double()
    rc = lib().wtmd_probe_peak(kind, C.byref(v), C.byref(ms))
    if rc:
        raise WtmdError(rc, "wtmd_probe_peak")
    return v.value, ms.value


def barrier_probe(blocks: int, absent: int, limit_cycles: int) -> bool:
    """Cooperative grid where CTA `absent` never reaches the grid barrier:
    True if the others' bounded wait gave up (wtmd_barrier_probe)."""
    out = C.c_int32()
    rc = lib().wtmd_barrier_probe(int(blocks), int(absent), int(limit_cycles), C.byref(out))
    if rc != OK:
        raise WtmdError(rc, "wtmd_barrier_probe")
    return bool(out.value)


def particles(x, dtype, device="cuda"):
    """[N,3] array -> contiguous [N,4] CUDA tensor of the handle's precision."""
    torch = _torch()
    x = np.asarray(x, dtype=np.float64).reshape(-1, 3)
    t = torch.zeros(x.shape[0], 4, dtype=dtype)
    t[:, :3] = torch.from_numpy(x).to(dtype)
    return t.to(device).contiguous()
