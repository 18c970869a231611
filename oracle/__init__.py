"""ctypes wrapper of the plain-C FP64 oracle (``fvlbm_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
CPU-baseline leg are the only users.  Nothing in the library imports it, and it
imports nothing from the library.  See the header of ``fvlbm_oracle.c`` for the
paper passages each routine follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fvlbm_oracle.c")
_LIB = os.path.join(_HERE, "libfvlbm_oracle.so")

SCHEMES = {"euler": 0, "rk2": 1, "ab2": 2, "rk4": 3}

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (strict IEEE evaluation: no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", "-fopenmp", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = C.CDLL(build())
    P = C.c_void_p
    dp = C.POINTER(C.c_double)
    i32p = C.POINTER(C.c_int32)
    i64p = C.POINTER(C.c_int64)
    lib.orc_create.restype = P
    lib.orc_create.argtypes = [C.c_int64, dp, C.c_int64, i64p, i32p, C.c_int64, i32p, i32p,
                               C.c_int32, i32p, i32p, dp, dp, dp, i32p, dp, C.c_char_p, C.c_int]
    lib.orc_destroy.argtypes = [P]
    lib.orc_geometry.argtypes = [P, dp, dp, dp]
    lib.orc_n_faces.restype = C.c_int64
    lib.orc_n_faces.argtypes = [P]
    lib.orc_feq.argtypes = [C.c_double, C.c_double, C.c_double, dp]
    lib.orc_set_f.argtypes = [P, dp]
    lib.orc_get_f.argtypes = [P, dp]
    lib.orc_set_equilibrium.argtypes = [P, dp, dp]
    lib.orc_macros.argtypes = [P, dp, dp]
    lib.orc_mass.restype = C.c_double
    lib.orc_mass.argtypes = [P]
    lib.orc_residual.restype = C.c_double
    lib.orc_residual.argtypes = [P, dp]
    lib.orc_rhs.argtypes = [P, dp, C.c_double, dp]
    lib.orc_run.argtypes = [P, C.c_int, C.c_double, C.c_double, C.c_int64]
    lib.orc_stencil_point.restype = C.c_int
    lib.orc_stencil_point.argtypes = [P, C.c_int64, C.c_int, dp]
    lib.orc_threads.restype = C.c_int
    lib.orc_threads.argtypes = [C.c_int]
    lib.orc_cfl_dt.restype = C.c_double
    lib.orc_cfl_dt.argtypes = [P, C.c_double, C.c_double, C.c_double, C.c_int]
    _lib = lib
    return lib


def _d(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _i32(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def _i64(a):
    return a.ctypes.data_as(C.POINTER(C.c_int64))


def threads(n: int = 0) -> int:
    """Threads the oracle's loops use from now on (n <= 0: unchanged); returns
    the number in effect.  A timing control only."""
    return int(_load().orc_threads(int(n)))


def feq(rho: float, ux: float, uy: float) -> np.ndarray:
    out = np.zeros(9)
    _load().orc_feq(rho, ux, uy, _d(out))
    return out


class Oracle:
    """FP64 CPU reference solver on one mesh (cells kept in the caller's order)."""

    def __init__(self, mesh):
        lib = _load()
        self._lib = lib
        kind, ext, uw, rinf, uinf, partner, shift = mesh.bc_arrays()
        self._keep = [np.ascontiguousarray(x) for x in (
            mesh.xy, mesh.cell_ptr.astype(np.int64), mesh.cell_vert.astype(np.int32),
            mesh.bedge.astype(np.int32), mesh.btag.astype(np.int32),
            kind, ext, uw, rinf, uinf, partner, shift)]
        xy, cp, cv, be, bt, kind, ext, uw, rinf, uinf, partner, shift = self._keep
        err = C.create_string_buffer(256)
        self.n_cell = mesh.n_cell
        h = lib.orc_create(mesh.n_vert, _d(xy), mesh.n_cell, _i64(cp), _i32(cv), mesh.n_bedge,
                           _i32(be), _i32(bt), len(kind), _i32(kind), _i32(ext), _d(uw),
                           _d(rinf), _d(uinf), _i32(partner), _d(shift), err, 256)
        if not h:
            raise ValueError("oracle mesh rejected: " + err.value.decode())
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.orc_destroy(h)
            self._h = None

    def geometry(self):
        a = np.zeros(self.n_cell)
        c = np.zeros((self.n_cell, 2))
        l = np.zeros((self.n_cell, 2))
        self._lib.orc_geometry(self._h, _d(a), _d(c), _d(l))
        return a, c, l

    def n_faces(self) -> int:
        return int(self._lib.orc_n_faces(self._h))

    def set_f(self, f):
        f = np.ascontiguousarray(f, np.float64).reshape(self.n_cell, 9)
        self._lib.orc_set_f(self._h, _d(f))

    def get_f(self) -> np.ndarray:
        f = np.zeros((self.n_cell, 9))
        self._lib.orc_get_f(self._h, _d(f))
        return f

    def set_equilibrium(self, rho, u):
        rho = np.ascontiguousarray(np.broadcast_to(rho, (self.n_cell,)), np.float64)
        u = np.ascontiguousarray(np.broadcast_to(u, (self.n_cell, 2)), np.float64)
        self._lib.orc_set_equilibrium(self._h, _d(rho), _d(u))

    def macros(self):
        rho = np.zeros(self.n_cell)
        u = np.zeros((self.n_cell, 2))
        self._lib.orc_macros(self._h, _d(rho), _d(u))
        return rho, u

    def mass(self) -> float:
        return float(self._lib.orc_mass(self._h))

    def residual(self, u_old) -> float:
        u_old = np.ascontiguousarray(u_old, np.float64).reshape(self.n_cell, 2)
        return float(self._lib.orc_residual(self._h, _d(u_old)))

    def rhs(self, f, tau: float) -> np.ndarray:
        f = np.ascontiguousarray(f, np.float64).reshape(self.n_cell, 9)
        out = np.zeros((self.n_cell, 9))
        self._lib.orc_rhs(self._h, _d(f), float(tau), _d(out))
        return out

    def run(self, scheme: str, tau: float, dt: float, nsteps: int):
        rc = self._lib.orc_run(self._h, SCHEMES[scheme], float(tau), float(dt), int(nsteps))
        if rc != 0:
            raise MemoryError("oracle run failed")

    def stencil_point(self, c: int, k: int):
        """(kind, position) of the least-squares stencil point of face k of cell c;
        kind is the boundary kind, or 10 interior / 11 periodic."""
        xy = np.zeros(2)
        kind = self._lib.orc_stencil_point(self._h, int(c), int(k), _d(xy))
        return kind, xy

    def cfl_dt(self, cfl: float, umax: float, tau: float, scheme: str) -> float:
        return float(self._lib.orc_cfl_dt(self._h, cfl, umax, tau, SCHEMES[scheme]))
