"""Python binding of the C ABI in include/mhd.h (argument marshalling only).

Every step of the method runs in the CUDA library built from csrc/ for sm_103a; this
module loads it with ctypes and raises if it is missing: there is no CPU fallback.
Names follow the C entry points (mhd_create -> Solver(), mhd_step -> Solver.step, ...).
PyTorch supplies device memory (tensors for device-side upload/download) and streams.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

LIB_PATH = _build.LIB

MHD_OK, MHD_ERR_INVALID, MHD_ERR_OOM, MHD_ERR_CUDA, MHD_ERR_UNPHYSICAL, MHD_ERR_TIMEOUT = range(6)
PERIODIC, OUTFLOW = 0, 1
FP32, FP64 = 0, 1
PRESSURE_FP32, PRESSURE_FP64, PRESSURE_COMPENSATED = 0, 1, 2   # mhd_pressure_mode

# every symbol include/mhd.h declares; tests check the library exports them all
EXPORTS = ("mhd_create", "mhd_init_fields", "mhd_upload", "mhd_step", "mhd_apply", "mhd_cmax",
           "mhd_read", "mhd_download", "mhd_sums", "mhd_state", "mhd_set_state", "mhd_sync",
           "mhd_info", "mhd_stream", "mhd_profile", "mhd_profile_read", "mhd_destroy",
           "mhd_status_str", "mhd_last_error", "mhd_sums_noalloc", "mhd_batch_create",
           "mhd_batch_step", "mhd_batch_step_each", "mhd_batch_sync", "mhd_batch_info",
           "mhd_batch_destroy", "mhd_batch_selftest_timeout", "mhd_batch_configure",
           "mhd_vis_curve",
           "mhd_vis_slice", "mhd_vis_volume", "mhd_vis_range")


class MhdConfig(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("h", C.c_double),
                ("gamma", C.c_double), ("cfl", C.c_double), ("bc", C.c_int * 3),
                ("prec", C.c_int), ("fp64_pressure", C.c_int), ("cuda_stream", C.c_void_p)]


class BatchShape(C.Structure):
    """mhd_batch_shape: launch shape of one context inside a batch (0 = default)."""
    _fields_ = [("march_len", C.c_int), ("ct_march", C.c_int), ("seg_k", C.c_int),
                ("z_warps", C.c_int), ("alone", C.c_int)]


class MhdError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(msg)
        self.status = status


_lib = None


def load_library(path: str | None = None) -> C.CDLL:
    """Load the built library; raises if it was not built (run build.build())."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise ImportError(f"CUDA library not built: {p} (run paper_0908_4362_gb300.build.build())")
    lib = C.CDLL(p)
    vp, ip, dp = C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_double)
    sig = {
        "mhd_create": ([C.POINTER(MhdConfig), C.POINTER(vp)], C.c_int),
        "mhd_init_fields": ([vp, C.POINTER(vp), C.c_double], C.c_int),
        "mhd_upload": ([vp, C.POINTER(vp), C.c_int, C.c_int, C.c_double], C.c_int),
        "mhd_step": ([vp, C.c_int, C.c_double, ip, dp], C.c_int),
        "mhd_apply": ([vp, C.c_int, C.c_int, C.c_double], C.c_int),
        "mhd_cmax": ([vp, dp], C.c_int),
        "mhd_read": ([vp, C.POINTER(vp)], C.c_int),
        "mhd_download": ([vp, C.POINTER(vp), C.c_int, C.c_int], C.c_int),
        "mhd_sums": ([vp, dp], C.c_int),
        "mhd_state": ([vp, dp, dp, ip, ip], C.c_int),
        "mhd_set_state": ([vp, C.c_double, C.c_int, C.c_int], C.c_int),
        "mhd_sync": ([vp], C.c_int),
        "mhd_info": ([vp, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)], C.c_int),
        "mhd_stream": ([vp, C.POINTER(vp)], C.c_int),
        "mhd_profile": ([vp, C.c_int], C.c_int),
        "mhd_profile_read": ([vp, dp, C.POINTER(C.c_longlong), C.c_int], C.c_int),
        "mhd_destroy": ([vp], None),
        "mhd_sums_noalloc": ([C.POINTER(vp), C.c_int, C.c_longlong, dp, vp], C.c_int),
        "mhd_batch_create": ([C.POINTER(vp), C.c_int, C.c_int, C.c_int, C.POINTER(vp)], C.c_int),
        "mhd_batch_step": ([vp, C.c_int], C.c_int),
        "mhd_batch_step_each": ([vp, ip], C.c_int),
        "mhd_vis_curve": ([vp, C.c_int, vp], C.c_int),
        "mhd_vis_slice": ([vp, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, vp], C.c_int),
        "mhd_vis_volume": ([vp, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, vp],
                           C.c_int),
        "mhd_vis_range": ([vp, C.c_int, dp, dp], C.c_int),
        "mhd_batch_sync": ([vp], C.c_int),
        "mhd_batch_info": ([vp, ip, C.POINTER(C.c_longlong), C.POINTER(vp)], C.c_int),
        "mhd_batch_destroy": ([vp], None),
        "mhd_batch_selftest_timeout": ([C.c_longlong], C.c_int),
        "mhd_batch_configure": ([vp, C.c_int, C.c_int, C.c_longlong, C.POINTER(BatchShape)],
                                C.c_int),
        "mhd_status_str": ([C.c_int], C.c_char_p),
        "mhd_last_error": ([vp], C.c_char_p),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    if path is None:
        _lib = lib
    return lib


def _ptrs8(arrs) -> C.Array:
    return (C.c_void_p * 8)(*[C.c_void_p(a) for a in arrs])


class Solver:
    """One grid on the GPU (mhd_create ... mhd_destroy)."""

    def __init__(self, n, bc=(PERIODIC,) * 3, h=1.0, gamma=5.0 / 3.0, cfl=0.7, prec=FP32,
                 fp64_pressure=False, stream=None, pressure=None):
        """pressure: PRESSURE_FP32 / PRESSURE_FP64 / PRESSURE_COMPENSATED (mhd_pressure_mode);
        fp64_pressure=True is PRESSURE_FP64."""
        self.lib = load_library()
        pm = int(pressure) if pressure is not None else (PRESSURE_FP64 if fp64_pressure
                                                         else PRESSURE_FP32)
        cfg = MhdConfig(int(n[0]), int(n[1]), int(n[2]), float(h), float(gamma), float(cfl),
                        (C.c_int * 3)(*[int(b) for b in bc]), int(prec), pm,
                        C.c_void_p(stream if stream else None))
        h_ = C.c_void_p()
        st = self.lib.mhd_create(C.byref(cfg), C.byref(h_))
        if st != MHD_OK:
            raise MhdError(st, f"mhd_create: {self.lib.mhd_status_str(st).decode()}")
        self.ctx = h_
        self.n = tuple(int(v) for v in n)
        self.ncells = self.n[0] * self.n[1] * self.n[2]
        self.prec = prec
        self.dtype = np.float32 if prec == FP32 else np.float64

    @classmethod
    def from_problem(cls, prob, prec=FP32, **kw):
        s = cls(prob.n, prob.bc, prob.h, prob.gamma, prob.cfl, prec=prec, **kw)
        s.init_fields(prob.fields)
        return s

    def _check(self, st: int, what: str) -> int:
        if st not in (MHD_OK,):
            err = self.lib.mhd_last_error(self.ctx).decode()
            raise MhdError(st, f"{what}: {self.lib.mhd_status_str(st).decode()} {err}".strip())
        return st

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.mhd_destroy(self.ctx)
            self.ctx = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # --- state in/out ---------------------------------------------------------------
    def init_fields(self, fields, t0: float = 0.0, check: bool = True):
        f = np.ascontiguousarray(np.asarray(fields, dtype=np.float64).reshape(8, -1))
        assert f.shape[1] == self.ncells
        st = self.lib.mhd_init_fields(self.ctx, _ptrs8([f[k].ctypes.data for k in range(8)]), t0)
        return self._check(st, "mhd_init_fields") if check else st

    def upload(self, arrays, t0: float = 0.0, on_device: bool | None = None):
        """8 arrays (numpy or torch tensors, float32/float64, host or device)."""
        ptrs, dtype, dev = [], None, on_device
        for a in arrays:
            if hasattr(a, "data_ptr"):
                ptrs.append(a.data_ptr())
                d = 0 if str(a.dtype) == "torch.float32" else 1
                dv = a.is_cuda
            else:
                ptrs.append(a.ctypes.data)
                d = 0 if a.dtype == np.float32 else 1
                dv = False
            dtype = d if dtype is None else dtype
            dev = dv if dev is None else dev
        st = self.lib.mhd_upload(self.ctx, _ptrs8(ptrs), dtype, int(bool(dev)), t0)
        return self._check(st, "mhd_upload")

    def read(self, check: bool = True) -> np.ndarray:
        out = np.empty((8, self.ncells), dtype=np.float64)
        st = self.lib.mhd_read(self.ctx, _ptrs8([out[k].ctypes.data for k in range(8)]))
        if check:
            self._check(st, "mhd_read")
        self.last_status = st
        return out

    def download(self, arrays, check: bool = True) -> int:
        ptrs, dtype, dev = [], None, None
        for a in arrays:
            if hasattr(a, "data_ptr"):
                ptrs.append(a.data_ptr())
                d = 0 if str(a.dtype) == "torch.float32" else 1
                dv = a.is_cuda
            else:
                ptrs.append(a.ctypes.data)
                d = 0 if a.dtype == np.float32 else 1
                dv = False
            dtype = d if dtype is None else dtype
            dev = dv if dev is None else dev
        st = self.lib.mhd_download(self.ctx, _ptrs8(ptrs), dtype, int(bool(dev)))
        return self._check(st, "mhd_download") if check else st

    # --- stepping -------------------------------------------------------------------
    def step(self, nsteps: int = 1, t_end: float = -1.0, sync: bool = False, check: bool = True):
        if sync or t_end >= 0:
            done, t = C.c_int(0), C.c_double(0)
            st = self.lib.mhd_step(self.ctx, int(nsteps), float(t_end), C.byref(done), C.byref(t))
            if check:
                self._check(st, "mhd_step")
            return done.value
        st = self.lib.mhd_step(self.ctx, int(nsteps), -1.0, None, None)
        if check:
            self._check(st, "mhd_step")
        return nsteps

    def run_to(self, t_end: float, max_steps: int = 10 ** 7) -> int:
        return self.step(max_steps, t_end)

    def apply(self, op: int, axis: int, dt: float):
        return self._check(self.lib.mhd_apply(self.ctx, op, axis, dt), "mhd_apply")

    def cmax(self) -> float:
        v = C.c_double(0)
        self._check(self.lib.mhd_cmax(self.ctx, C.byref(v)), "mhd_cmax")
        return v.value

    def sums(self) -> np.ndarray:
        out = np.zeros(8)
        self._check(self.lib.mhd_sums(self.ctx, out.ctypes.data_as(C.POINTER(C.c_double))),
                    "mhd_sums")
        return out

    def state(self):
        t, dtl, stp, ph = C.c_double(), C.c_double(), C.c_int(), C.c_int()
        self._check(self.lib.mhd_state(self.ctx, C.byref(t), C.byref(dtl), C.byref(stp),
                                       C.byref(ph)), "mhd_state")
        return t.value, dtl.value, stp.value, ph.value

    def set_state(self, t: float, step: int, phase: int):
        return self._check(self.lib.mhd_set_state(self.ctx, t, step, phase), "mhd_set_state")

    def sync(self, check: bool = True) -> int:
        st = self.lib.mhd_sync(self.ctx)
        return self._check(st, "mhd_sync") if check else st

    def info(self):
        n, b = C.c_longlong(), C.c_longlong()
        self._check(self.lib.mhd_info(self.ctx, C.byref(n), C.byref(b)), "mhd_info")
        return n.value, b.value

    def profile(self, enable: bool = True):
        return self._check(self.lib.mhd_profile(self.ctx, int(bool(enable))), "mhd_profile")

    KINDS = ("fluid_x", "fluid_y", "fluid_z", "ct_x", "ct_y", "ct_z", "dt", "other")

    def profile_read(self, reset: bool = True) -> dict:
        ms = np.zeros(8)
        cnt = (C.c_longlong * 8)()
        self._check(self.lib.mhd_profile_read(self.ctx, ms.ctypes.data_as(C.POINTER(C.c_double)),
                                              cnt, int(bool(reset))), "mhd_profile_read")
        return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(self.KINDS)}

    def stream_handle(self) -> int:
        s = C.c_void_p()
        self._check(self.lib.mhd_stream(self.ctx, C.byref(s)), "mhd_stream")
        return s.value or 0

    # --- visualization (device buffers from torch; results returned as torch tensors) ---
    QUANTITIES = {"rho": 0, "p": 1, "E": 2, "vmag": 3, "bmag": 4}

    def _q(self, quantity) -> int:
        return self.QUANTITIES[quantity] if isinstance(quantity, str) else int(quantity)

    def vis_range(self, quantity="rho"):
        lo, hi = C.c_double(), C.c_double()
        self._check(self.lib.mhd_vis_range(self.ctx, self._q(quantity), C.byref(lo),
                                           C.byref(hi)), "mhd_vis_range")
        return lo.value, hi.value

    def _image_shape(self, axis: int):
        if axis not in (0, 1, 2):
            raise MhdError(MHD_ERR_INVALID, f"axis {axis} is not 0, 1 or 2")
        u, v = [a for a in range(3) if a != axis]
        return self.n[v], self.n[u]

    def vis_curve(self, quantity="rho"):
        import torch
        n = max(self.n)
        xy = torch.empty((n, 2), dtype=torch.float32, device="cuda")
        self._check(self.lib.mhd_vis_curve(self.ctx, self._q(quantity), C.c_void_p(xy.data_ptr())),
                    "mhd_vis_curve")
        return xy

    def vis_slice(self, quantity="rho", axis=2, index=0, vmin=None, vmax=None):
        import torch
        if vmin is None or vmax is None:
            lo, hi = self.vis_range(quantity)
            vmin = lo if vmin is None else vmin
            vmax = (hi if hi > lo else lo + 1.0) if vmax is None else vmax
        h, w = self._image_shape(axis)
        img = torch.empty((h, w, 4), dtype=torch.uint8, device="cuda")
        self._check(self.lib.mhd_vis_slice(self.ctx, self._q(quantity), int(axis), int(index),
                                           float(vmin), float(vmax),
                                           C.c_void_p(img.data_ptr())), "mhd_vis_slice")
        return img

    def vis_volume(self, quantity="rho", axis=2, vmin=None, vmax=None, opacity=0.05):
        import torch
        if vmin is None or vmax is None:
            lo, hi = self.vis_range(quantity)
            vmin = lo if vmin is None else vmin
            vmax = (hi if hi > lo else lo + 1.0) if vmax is None else vmax
        h, w = self._image_shape(axis)
        img = torch.empty((h, w, 4), dtype=torch.float32, device="cuda")
        self._check(self.lib.mhd_vis_volume(self.ctx, self._q(quantity), int(axis), float(vmin),
                                            float(vmax), float(opacity),
                                            C.c_void_p(img.data_ptr())), "mhd_vis_volume")
        return img


class Batch:
    """Many solvers advanced together by one persistent launch per step call
    (mhd_batch_create / mhd_batch_step / mhd_batch_sync / mhd_batch_destroy)."""

    def __init__(self, solvers, z_tile_warps: int = 0, ctas_per_sm: int = 0):
        self.lib = load_library()
        self.solvers = list(solvers)
        arr = (C.c_void_p * len(self.solvers))(*[s.ctx for s in self.solvers])
        h_ = C.c_void_p()
        st = self.lib.mhd_batch_create(arr, len(self.solvers), int(z_tile_warps), int(ctas_per_sm),
                                       C.byref(h_))
        if st != MHD_OK:
            raise MhdError(st, f"mhd_batch_create: {self.lib.mhd_status_str(st).decode()}")
        self.b = h_

    def step(self, nsteps: int):
        st = self.lib.mhd_batch_step(self.b, int(nsteps))
        if st != MHD_OK:
            raise MhdError(st, f"mhd_batch_step: {self.lib.mhd_status_str(st).decode()}")

    def step_each(self, counts):
        """Advance solver i by counts[i] steps (0: not at all) in one persistent launch."""
        arr = (C.c_int * len(self.solvers))(*[int(c) for c in counts])
        st = self.lib.mhd_batch_step_each(self.b, arr)
        if st != MHD_OK:
            raise MhdError(st, f"mhd_batch_step_each: {self.lib.mhd_status_str(st).decode()}")

    def sync(self) -> int:
        return self.lib.mhd_batch_sync(self.b)

    def configure(self, threads_per_cta: int = 0, ctas_per_sm: int = 0, spin_cycles: int = 0,
                  shapes=None):
        """mhd_batch_configure.  shapes: None, or one dict (or BatchShape) per solver with
        any of march_len, ct_march, seg_k, z_warps, alone (missing keys: 0 = default)."""
        arr = None
        if shapes is not None:
            if len(shapes) != len(self.solvers):
                raise ValueError("one shape per solver")
            arr = (BatchShape * len(shapes))()
            for a, sh in zip(arr, shapes):
                for k, v in (sh.items() if isinstance(sh, dict) else
                             ((f, getattr(sh, f)) for f, _ in BatchShape._fields_)):
                    setattr(a, k, int(v))
        st = self.lib.mhd_batch_configure(self.b, int(threads_per_cta), int(ctas_per_sm),
                                          int(spin_cycles), arr)
        if st != MHD_OK:
            raise MhdError(st, f"mhd_batch_configure: {self.lib.mhd_status_str(st).decode()}")

    def info(self):
        c, n, s = C.c_int(), C.c_longlong(), C.c_void_p()
        self.lib.mhd_batch_info(self.b, C.byref(c), C.byref(n), C.byref(s))
        return c.value, n.value

    def stream_handle(self) -> int:
        s = C.c_void_p()
        self.lib.mhd_batch_info(self.b, None, None, C.byref(s))
        return s.value or 0

    def close(self):
        if getattr(self, "b", None):
            self.lib.mhd_batch_destroy(self.b)
            self.b = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
