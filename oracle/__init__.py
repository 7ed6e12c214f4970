"""FP64 CPU oracle of the relaxing-TVD MHD step (arXiv:0908.4362, Sect. 3 and 4.2).

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package.  The product path (the CUDA library
and its binding) never imports it, and this package never imports the product.

The arithmetic lives in ``mhd_oracle.c`` (plain C, double precision, no FMA contraction).
This module only compiles it with gcc and marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mhd_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LOCK = threading.Lock()
_LIBS: dict = {}

UNPHYSICAL = 1
NONFINITE = 2


class Grid(C.Structure):
    _fields_ = [("n", C.c_int * 3), ("bc", C.c_int * 3), ("h", C.c_double),
                ("gamma", C.c_double), ("cfl", C.c_double)]


def lib_path(mutant: int = 0, openmp: bool = True) -> str:
    tag = f"m{mutant}" + ("_omp" if openmp else "")
    return os.path.join(_BUILD, f"liborc_{tag}.so")


def build(mutant: int = 0, openmp: bool = True, force: bool = False) -> str:
    """Compile the oracle (optionally a planted-mistake variant) into oracle/_build."""
    out = lib_path(mutant, openmp)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    os.makedirs(_BUILD, exist_ok=True)
    tmp = out + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           f"-DORC_MUTANT={mutant}", _SRC, "-o", tmp, "-lm"]
    if openmp:
        cmd.insert(1, "-fopenmp")
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def load(mutant: int = 0, openmp: bool = True) -> C.CDLL:
    key = (mutant, openmp)
    with _LOCK:
        if key not in _LIBS:
            lib = C.CDLL(build(mutant, openmp))
            dp = C.POINTER(C.c_double)
            pp = C.POINTER(dp)
            g = C.POINTER(Grid)
            lib.orc_vanleer.restype = C.c_double
            lib.orc_vanleer.argtypes = [C.c_double, C.c_double]
            lib.orc_cell_flux.restype = C.c_int
            lib.orc_cell_flux.argtypes = [dp, dp, C.c_double, dp, dp, dp, dp]
            for name in ("orc_fluid", "orc_ct"):
                fn = getattr(lib, name)
                fn.restype = C.c_int
                fn.argtypes = [g, pp, C.c_int, C.c_double]
            lib.orc_ct_one.restype = C.c_int
            lib.orc_ct_one.argtypes = [g, pp, C.c_int, C.c_int, C.c_double]
            lib.orc_cmax.restype = C.c_double
            lib.orc_cmax.argtypes = [g, pp, C.POINTER(C.c_int)]
            lib.orc_step_dt.restype = C.c_int
            lib.orc_step_dt.argtypes = [g, pp, C.c_int, C.c_double]
            lib.orc_dt.restype = C.c_double
            lib.orc_dt.argtypes = [g, pp, C.c_double, C.c_double, C.POINTER(C.c_int),
                                   C.POINTER(C.c_int)]
            lib.orc_step.restype = C.c_int
            lib.orc_step.argtypes = [g, pp, dp, C.POINTER(C.c_int), C.c_double, dp]
            lib.orc_run.restype = C.c_int
            lib.orc_run.argtypes = [g, pp, dp, C.POINTER(C.c_int), C.c_int, C.c_double,
                                    C.POINTER(C.c_int)]
            lib.orc_divb_max.restype = C.c_double
            lib.orc_divb_max.argtypes = [g, pp]
            lib.orc_mutant.restype = C.c_int
            _LIBS[key] = lib
        return _LIBS[key]


def set_threads(n: int) -> None:
    """Thread count of the OpenMP build (results do not depend on it)."""
    os.environ["OMP_NUM_THREADS"] = str(n)


class Oracle:
    """A grid state advanced by the C oracle.

    ``fields`` is an (8, nx*ny*nz) float64 array in the paper's order
    (rho, mx, my, mz, E, Bx, By, Bz), flat index (x*ny + y)*nz + z.
    """

    def __init__(self, n, bc, h, gamma, cfl, fields, t=0.0, phase=0, mutant=0, openmp=True,
                 copy=True):
        self.lib = load(mutant, openmp)
        self.grid = Grid((C.c_int * 3)(*n), (C.c_int * 3)(*bc), float(h), float(gamma),
                         float(cfl))
        self.n = tuple(int(v) for v in n)
        if copy:
            self.f = np.ascontiguousarray(np.array(fields, dtype=np.float64).reshape(8, -1))
        else:   # advance the caller's float64 array in place
            self.f = np.asarray(fields, dtype=np.float64).reshape(8, -1)
            assert self.f.flags["C_CONTIGUOUS"]
        assert self.f.shape[1] == self.n[0] * self.n[1] * self.n[2]
        self.t = float(t)
        self.phase = int(phase)
        self.status = 0
        self.steps = 0

    @classmethod
    def from_problem(cls, prob, **kw):
        return cls(prob.n, prob.bc, prob.h, prob.gamma, prob.cfl, prob.fields, **kw)

    def _ptrs(self):
        dp = C.POINTER(C.c_double)
        arr = (dp * 8)(*[self.f[k].ctypes.data_as(dp) for k in range(8)])
        return arr

    def cmax(self) -> float:
        st = C.c_int(0)
        v = self.lib.orc_cmax(C.byref(self.grid), self._ptrs(), C.byref(st))
        self.status |= st.value
        return v

    def dt(self, t_end: float = -1.0) -> float:
        st, cl = C.c_int(0), C.c_int(0)
        v = self.lib.orc_dt(C.byref(self.grid), self._ptrs(), self.t, t_end, C.byref(cl),
                            C.byref(st))
        self.status |= st.value
        return v

    def fluid(self, axis: int, dt: float) -> None:
        self.status |= self.lib.orc_fluid(C.byref(self.grid), self._ptrs(), axis, dt)

    def ct(self, axis: int, dt: float) -> None:
        self.status |= self.lib.orc_ct(C.byref(self.grid), self._ptrs(), axis, dt)

    def ct_one(self, axis: int, tsel: int, dt: float) -> None:
        self.status |= self.lib.orc_ct_one(C.byref(self.grid), self._ptrs(), axis, tsel, dt)

    def step_dt(self, dt: float, phase: int | None = None) -> None:
        ph = self.phase if phase is None else phase
        self.status |= self.lib.orc_step_dt(C.byref(self.grid), self._ptrs(), ph, dt)

    def step(self, nsteps: int = 1, t_end: float = -1.0) -> int:
        t = C.c_double(self.t)
        ph = C.c_int(self.phase)
        done = C.c_int(0)
        self.status |= self.lib.orc_run(C.byref(self.grid), self._ptrs(), C.byref(t),
                                        C.byref(ph), nsteps, t_end, C.byref(done))
        self.t, self.phase = t.value, ph.value
        self.steps += done.value
        return done.value

    def run_to(self, t_end: float, max_steps: int = 10 ** 7) -> int:
        return self.step(max_steps, t_end)

    def divb_max(self) -> float:
        return self.lib.orc_divb_max(C.byref(self.grid), self._ptrs())

    def sums(self) -> np.ndarray:
        return self.f.sum(axis=1)

    def field(self, k: int) -> np.ndarray:
        return self.f[k].reshape(self.n)


def vanleer(a: float, b: float, mutant: int = 0) -> float:
    return load(mutant).orc_vanleer(float(a), float(b))


def cell_flux(u, b, gamma, mutant: int = 0):
    """(FR, FL, c, F) of one cell in local coordinates."""
    lib = load(mutant)
    dp = C.POINTER(C.c_double)
    u = np.ascontiguousarray(u, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    fr, fl, F = np.zeros(5), np.zeros(5), np.zeros(5)
    c = C.c_double(0)
    st = lib.orc_cell_flux(u.ctypes.data_as(dp), b.ctypes.data_as(dp), float(gamma),
                           fr.ctypes.data_as(dp), fl.ctypes.data_as(dp), C.byref(c),
                           F.ctypes.data_as(dp))
    return fr, fl, c.value, F, st
