"""Python binding of libfvlbm (ctypes over the C ABI in include/fvlbm.h).

Argument marshalling only: every step of the solver runs in the library's CUDA
kernels.  PyTorch supplies the device workspace and the stream.  There is no
fallback: if the shared library is missing or cannot be loaded, importing this
module raises.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Iterable, List, Optional, Sequence, Union

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfvlbm.so")

EULER, RK2, AB2, RK4 = 0, 1, 2, 3
FP64, FP32_DEV, FP16_DEV, BF16_DEV = 0, 1, 2, 3
SCHEMES = {"euler": EULER, "rk2": RK2, "ab2": AB2, "rk4": RK4}
PRECISIONS = {"fp64": FP64, "fp32": FP32_DEV, "fp16": FP16_DEV, "bf16": BF16_DEV}

ERRORS = {
    -1: "ARG", -2: "MESH_TOPOLOGY", -3: "DEGENERATE_CELL", -4: "UNTAGGED_BOUNDARY",
    -5: "UNSTABLE_DT", -6: "OOM", -7: "CUDA", -8: "DIVERGED", -9: "TIMEOUT", -10: "UNSUPPORTED",
}


class FvlbmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        self.code = code
        self.name = ERRORS.get(code, str(code))
        super().__init__(f"FVLBM_ERR_{self.name}: {msg}")


class BcT(C.Structure):
    _fields_ = [("kind", C.c_int32), ("external", C.c_int32), ("u_w", C.c_double * 2),
                ("rho_inf", C.c_double), ("u_inf", C.c_double * 2), ("partner", C.c_int32),
                ("reserved", C.c_int32), ("shift", C.c_double * 2)]


class ParamsT(C.Structure):
    _fields_ = [("tau", C.c_double), ("dt", C.c_double), ("cfl", C.c_double), ("u_max", C.c_double),
                ("scheme", C.c_int32), ("precision", C.c_int32), ("rho0", C.c_double),
                ("u0", C.c_double * 2), ("device", C.c_int32), ("kernel", C.c_int32)]


class MeshInfoT(C.Structure):
    _fields_ = [("n_cell", C.c_int64), ("n_face", C.c_int64), ("n_bface", C.c_int64),
                ("n_periodic", C.c_int64), ("max_faces", C.c_int32), ("n_instances", C.c_int32),
                ("total_area", C.c_double), ("min_cfl_length", C.c_double)]


class PartInfoT(C.Structure):
    _fields_ = [("n_owned", C.c_int64), ("n_ring1", C.c_int64), ("n_ring2", C.c_int64),
                ("n_recv", C.c_int64), ("n_send", C.c_int64), ("n_neighbours", C.c_int32)]


class PlanInfoT(C.Structure):
    _fields_ = [("stage_kernel", C.c_int32), ("slots", C.c_int32), ("n_tiles", C.c_int64),
                ("short_tiles", C.c_int64), ("max_local_cells", C.c_int32), ("max_faces", C.c_int32),
                ("mean_tile_cells", C.c_double), ("mean_ring1_cells", C.c_double),
                ("mean_local_cells", C.c_double), ("face_table_waves", C.c_double),
                ("gather_waves", C.c_double), ("violations", C.c_int64)]


class ServerConfigT(C.Structure):
    _fields_ = [("device", C.c_int32), ("n_streams", C.c_int32), ("arena_bytes", C.c_size_t),
                ("max_active", C.c_int32), ("check_interval", C.c_int32), ("residual_tol", C.c_double),
                ("max_steps", C.c_int64)]


class RequestInfoT(C.Structure):
    _fields_ = [("state", C.c_int32), ("status", C.c_int32), ("steps", C.c_int64), ("n_cell", C.c_int64),
                ("residual", C.c_double), ("t_submit", C.c_double), ("t_admit", C.c_double),
                ("t_done", C.c_double), ("workspace_bytes", C.c_size_t)]


class ServerStatsT(C.Structure):
    _fields_ = [("queued", C.c_int32), ("active", C.c_int32), ("arena_free", C.c_size_t),
                ("arena_free_largest", C.c_size_t), ("cell_steps", C.c_int64), ("t_now", C.c_double)]


#: every symbol include/fvlbm.h declares
EXPORTS = ["fvlbm_mesh_create", "fvlbm_mesh_concat", "fvlbm_mesh_destroy", "fvlbm_mesh_info",
           "fvlbm_suggest_dt", "fvlbm_workspace_bytes", "fvlbm_plan_info", "fvlbm_init", "fvlbm_step", "fvlbm_macros",
           "fvlbm_residual", "fvlbm_mass", "fvlbm_mass_noalloc", "fvlbm_get_f", "fvlbm_set_f", "fvlbm_host_transfer", "fvlbm_stage_kernel", "fvlbm_sync",
           "fvlbm_get_dt", "fvlbm_profile", "fvlbm_autotune", "fvlbm_fma_peak", "fvlbm_launches_per_step", "fvlbm_solver_destroy",
           "fvlbm_server_create", "fvlbm_server_submit", "fvlbm_server_poll", "fvlbm_server_request",
           "fvlbm_server_stats", "fvlbm_server_destroy", "fvlbm_mesh_partition", "fvlbm_partition_destroy",
           "fvlbm_partition_info", "fvlbm_partition_cells", "fvlbm_partition_halo", "fvlbm_dd_create",
           "fvlbm_dd_step", "fvlbm_dd_macros", "fvlbm_dd_get_f", "fvlbm_dd_set_f", "fvlbm_dd_mass",
           "fvlbm_dd_residual", "fvlbm_dd_stage_kernel", "fvlbm_dd_sync", "fvlbm_dd_destroy",
           "fvlbm_last_error"]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built; run __graft_entry__.build() "
                          "(the solver has no CPU fallback)")
    lib = C.CDLL(LIB_PATH)
    P = C.c_void_p
    PP = C.POINTER(C.c_void_p)
    dp = C.POINTER(C.c_double)
    i32p = C.POINTER(C.c_int32)
    i64p = C.POINTER(C.c_int64)
    sig = {
        "fvlbm_mesh_create": [dp, C.c_int64, i64p, i32p, C.c_int64, i32p, i32p, C.c_int64,
                              C.POINTER(BcT), C.c_int32, PP],
        "fvlbm_mesh_concat": [PP, C.c_int32, PP],
        "fvlbm_mesh_destroy": [P],
        "fvlbm_mesh_info": [P, C.POINTER(MeshInfoT)],
        "fvlbm_suggest_dt": [P, C.c_int32, C.c_double, C.c_double, C.c_double, C.c_int32, dp],
        "fvlbm_workspace_bytes": [P, C.POINTER(ParamsT), C.c_int32, C.POINTER(C.c_size_t)],
        "fvlbm_plan_info": [P, C.POINTER(ParamsT), C.c_int32, C.POINTER(PlanInfoT)],
        "fvlbm_init": [P, C.POINTER(ParamsT), C.c_int32, P, P, C.c_size_t, PP],
        "fvlbm_step": [P, C.c_int64],
        "fvlbm_macros": [P, dp, dp],
        "fvlbm_residual": [P, dp],
        "fvlbm_mass": [P, dp],
        "fvlbm_mass_noalloc": [P, dp],
        "fvlbm_get_f": [P, dp],
        "fvlbm_set_f": [P, dp],
        "fvlbm_sync": [P],
        "fvlbm_get_dt": [P, C.c_int32, dp],
        "fvlbm_profile": [P, C.c_int64, dp, C.c_int32, i32p, i64p],
        "fvlbm_launches_per_step": [P, i64p],
        "fvlbm_autotune": [P, C.POINTER(ParamsT), C.c_int32, P, C.c_int32, i32p, dp],
        "fvlbm_fma_peak": [C.c_int32, C.c_int32, dp],
        "fvlbm_host_transfer": [P, C.c_int32, i32p],
        "fvlbm_stage_kernel": [P, i32p],
        "fvlbm_solver_destroy": [P],
        "fvlbm_server_create": [C.POINTER(ServerConfigT), PP],
        "fvlbm_server_submit": [P, P, C.POINTER(ParamsT), C.c_int32, i64p],
        "fvlbm_server_poll": [P, i32p],
        "fvlbm_server_request": [P, C.c_int64, C.POINTER(RequestInfoT), dp, dp],
        "fvlbm_server_stats": [P, C.POINTER(ServerStatsT)],
        "fvlbm_server_destroy": [P],
        "fvlbm_mesh_partition": [P, C.c_int32, PP],
        "fvlbm_partition_destroy": [P],
        "fvlbm_partition_info": [P, C.c_int32, C.POINTER(PartInfoT)],
        "fvlbm_partition_cells": [P, C.c_int32, i64p],
        "fvlbm_partition_halo": [P, C.c_int32, C.c_int32, i64p, i32p, i32p],
        "fvlbm_dd_create": [P, C.POINTER(ParamsT), C.c_int32, P, PP],
        "fvlbm_dd_step": [P, C.c_int64],
        "fvlbm_dd_macros": [P, dp, dp],
        "fvlbm_dd_get_f": [P, dp],
        "fvlbm_dd_set_f": [P, dp],
        "fvlbm_dd_mass": [P, dp],
        "fvlbm_dd_residual": [P, dp],
        "fvlbm_dd_stage_kernel": [P, i32p, i64p],
        "fvlbm_dd_sync": [P],
        "fvlbm_dd_destroy": [P],
        "fvlbm_last_error": [],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = C.c_int
    lib.fvlbm_mesh_destroy.restype = None
    lib.fvlbm_solver_destroy.restype = None
    lib.fvlbm_server_destroy.restype = None
    lib.fvlbm_partition_destroy.restype = None
    lib.fvlbm_dd_destroy.restype = None
    lib.fvlbm_last_error.restype = C.c_char_p
    return lib


lib = _load()


def _check(rc: int):
    if rc != 0:
        raise FvlbmError(rc, (lib.fvlbm_last_error() or b"").decode())


def _d(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


class Mesh:
    """A mesh handle built from a meshgen.Mesh (or any object with the same arrays)."""

    def __init__(self, m=None, _handle=None, _n_cell=None):
        if _handle is not None:
            self._h = _handle
            self.n_cell = _n_cell
            return
        xy = np.ascontiguousarray(m.xy, np.float64)
        cp = np.ascontiguousarray(m.cell_ptr, np.int64)
        cv = np.ascontiguousarray(m.cell_vert, np.int32)
        be = np.ascontiguousarray(m.bedge, np.int32)
        bt = np.ascontiguousarray(m.btag, np.int32)
        bcs = (BcT * max(1, len(m.bcs)))()
        for i, b in enumerate(m.bcs):
            bcs[i].kind = b.kind
            bcs[i].external = b.external
            bcs[i].u_w[:] = list(b.u_w)
            bcs[i].rho_inf = b.rho_inf
            bcs[i].u_inf[:] = list(b.u_inf)
            bcs[i].partner = b.partner
            bcs[i].shift[:] = list(b.shift)
        h = C.c_void_p()
        _check(lib.fvlbm_mesh_create(_d(xy), xy.shape[0], cp.ctypes.data_as(C.POINTER(C.c_int64)),
                                     cv.ctypes.data_as(C.POINTER(C.c_int32)), cp.shape[0] - 1,
                                     be.ctypes.data_as(C.POINTER(C.c_int32)),
                                     bt.ctypes.data_as(C.POINTER(C.c_int32)), be.shape[0], bcs,
                                     len(m.bcs), C.byref(h)))
        self._h = h
        self.n_cell = int(cp.shape[0] - 1)

    @classmethod
    def concat(cls, meshes: Sequence["Mesh"]) -> "Mesh":
        arr = (C.c_void_p * len(meshes))(*[m._h.value for m in meshes])
        h = C.c_void_p()
        _check(lib.fvlbm_mesh_concat(arr, len(meshes), C.byref(h)))
        return cls(_handle=h, _n_cell=sum(m.n_cell for m in meshes))

    def info(self) -> dict:
        i = MeshInfoT()
        _check(lib.fvlbm_mesh_info(self._h, C.byref(i)))
        return {k: getattr(i, k) for k, _ in MeshInfoT._fields_}

    def suggest_dt(self, tau: float, cfl: float = 0.5, u_max: float = 0.1, scheme="euler",
                   instance: int = 0) -> float:
        dt = C.c_double()
        _check(lib.fvlbm_suggest_dt(self._h, instance, tau, cfl, u_max, _scheme(scheme), C.byref(dt)))
        return dt.value

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib.fvlbm_mesh_destroy(h)
            self._h = None


def _scheme(s) -> int:
    return SCHEMES[s] if isinstance(s, str) else int(s)


def _prec(p) -> int:
    return PRECISIONS[p] if isinstance(p, str) else int(p)


def make_params(tau: float, dt: float = 0.0, scheme="euler", precision="fp64", rho0: float = 1.0,
                u0=(0.0, 0.0), cfl: float = 0.0, u_max: float = 0.0, device: int = 0,
                kernel: int = 0) -> ParamsT:
    p = ParamsT()
    p.tau, p.dt, p.cfl, p.u_max = tau, dt, cfl, u_max
    p.scheme, p.precision = _scheme(scheme), _prec(precision)
    p.rho0 = rho0
    p.u0[:] = list(u0)
    p.device = device
    p.kernel = kernel
    return p


class Solver:
    """Solver of one mesh (possibly a concatenation of instances) on one GPU.

    params: one ParamsT (all instances) or one per instance.  The device
    workspace is a torch uint8 tensor on the solver's device, kept alive by this
    object; the stream is torch's current stream on that device unless given.
    """

    def __init__(self, mesh: Mesh, params: Union[ParamsT, Sequence[ParamsT]], stream=None,
                 use_torch_workspace: bool = True):
        import torch
        plist = [params] if isinstance(params, ParamsT) else list(params)
        arr = (ParamsT * len(plist))(*plist)
        dev = plist[0].device
        self.device = dev
        self.mesh = mesh
        self.n_cell = mesh.n_cell
        self.n_inst = mesh.info()["n_instances"]
        if stream is None:
            # a stream of its own (not the legacy default stream, which cannot
            # be captured into the CUDA graphs fvlbm_step replays)
            stream = torch.cuda.Stream(device=dev)
        self.stream = stream
        sh = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream or 0)
        nbytes = C.c_size_t()
        _check(lib.fvlbm_workspace_bytes(mesh._h, arr, len(plist), C.byref(nbytes)))
        self.workspace_bytes = nbytes.value
        if use_torch_workspace:
            self._ws = torch.empty(nbytes.value, dtype=torch.uint8, device=f"cuda:{dev}")
            ws_ptr = self._ws.data_ptr()
        else:
            self._ws = None
            ws_ptr = None
        h = C.c_void_p()
        _check(lib.fvlbm_init(mesh._h, arr, len(plist), C.c_void_p(sh), C.c_void_p(ws_ptr),
                              nbytes.value, C.byref(h)))
        self._h = h

    def step(self, n: int = 1):
        _check(lib.fvlbm_step(self._h, int(n)))

    def sync(self):
        _check(lib.fvlbm_sync(self._h))

    def macros(self):
        rho = np.zeros(self.n_cell)
        u = np.zeros((self.n_cell, 2))
        return self.macros_into(rho, u)

    def macros_into(self, rho: np.ndarray, u: np.ndarray):
        """rho [n_cell] and u [n_cell, 2] (C-contiguous float64 arrays the
        caller owns, e.g. pinned host memory) written in place."""
        for a, shape in ((rho, (self.n_cell,)), (u, (self.n_cell, 2))):
            if a.dtype != np.float64 or a.shape != shape or not a.flags.c_contiguous:
                raise ValueError(f"macros_into: need a C-contiguous float64 array of shape {shape}")
        _check(lib.fvlbm_macros(self._h, _d(rho), _d(u)))
        return rho, u

    def residual(self) -> np.ndarray:
        e = np.zeros(self.n_inst)
        _check(lib.fvlbm_residual(self._h, _d(e)))
        return e

    def mass(self) -> np.ndarray:
        m = np.zeros(self.n_inst)
        _check(lib.fvlbm_mass(self._h, _d(m)))
        return m

    def mass_noalloc(self) -> np.ndarray:
        """fvlbm_mass computed without any allocation by the call (fixed
        library scratch; calls on one device must not overlap)."""
        m = np.zeros(self.n_inst)
        _check(lib.fvlbm_mass_noalloc(self._h, _d(m)))
        return m

    def get_f(self) -> np.ndarray:
        f = np.zeros((self.n_cell, 9))
        _check(lib.fvlbm_get_f(self._h, _d(f)))
        return f

    def set_f(self, f):
        f = np.ascontiguousarray(f, np.float64).reshape(self.n_cell, 9)
        _check(lib.fvlbm_set_f(self._h, _d(f)))

    def stage_kernel(self) -> int:
        """1 for the two-kernel stage, else the fused stage's threads per CTA."""
        k = C.c_int32()
        _check(lib.fvlbm_stage_kernel(self._h, C.byref(k)))
        return k.value

    def host_transfer(self, mode: str = "auto") -> bool:
        """How set_f reads the caller's buffer: "auto" (the kernel reads it
        directly when the GPU can reach pageable host memory) or "staged" (one
        copy to a device buffer).  get_f and macros always copy through the
        device buffer.  Returns True when set_f reads directly."""
        d = C.c_int32()
        _check(lib.fvlbm_host_transfer(self._h, {"auto": 0, "staged": 1}[mode], C.byref(d)))
        return bool(d.value)

    def dt(self, instance: int = 0) -> float:
        d = C.c_double()
        _check(lib.fvlbm_get_dt(self._h, instance, C.byref(d)))
        return d.value

    def profile(self, n: int):
        """Mean device ms of each kernel kind over n steps, and kernels launched."""
        ms = np.zeros(8)
        nk = C.c_int32()
        nl = C.c_int64()
        _check(lib.fvlbm_profile(self._h, int(n), _d(ms), 8, C.byref(nk), C.byref(nl)))
        return ms[:nk.value].copy(), nl.value

    def launches_per_step(self) -> int:
        n = C.c_int64()
        _check(lib.fvlbm_launches_per_step(self._h, C.byref(n)))
        return n.value

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib.fvlbm_solver_destroy(h)
            self._h = None

    def __del__(self):
        self.close()


KERNEL_VARIANTS = (1, 128, 256, 512, 1024)


def fma_peak(device: int = 0, fp64: bool = True) -> float:
    """Sustained FMA throughput of the device in TFLOP/s (FP64 or FP32)."""
    t = C.c_double()
    _check(lib.fvlbm_fma_peak(device, 1 if fp64 else 0, C.byref(t)))
    return t.value


def plan_info(mesh: Mesh, params) -> dict:
    """The stage plan fvlbm_init would build, checked on the host (no GPU):
    tile statistics, modelled shared-memory wavefronts, failed checks (and,
    if any, the first one's description under "first_violation")."""
    plist = [params] if isinstance(params, ParamsT) else list(params)
    arr = (ParamsT * len(plist))(*plist)
    i = PlanInfoT()
    _check(lib.fvlbm_plan_info(mesh._h, arr, len(plist), C.byref(i)))
    out = {k: getattr(i, k) for k, _ in PlanInfoT._fields_}
    if out["violations"]:
        out["first_violation"] = (lib.fvlbm_last_error() or b"").decode()
    return out


def autotune(mesh: Mesh, params, steps: int = 10, stream=None):
    """Fastest stage-kernel variant for this mesh: (params.kernel value, {variant: ms per step})."""
    import torch
    plist = [params] if isinstance(params, ParamsT) else list(params)
    arr = (ParamsT * len(plist))(*plist)
    if stream is None:
        stream = torch.cuda.Stream(device=plist[0].device)
    sh = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream or 0)
    best = C.c_int32()
    ms = np.zeros(5)
    _check(lib.fvlbm_autotune(mesh._h, arr, len(plist), C.c_void_p(sh), steps, C.byref(best), _d(ms)))
    return best.value, dict(zip(KERNEL_VARIANTS, ms.tolist()))


class Partition:
    """Domain decomposition plan of a one-instance mesh (host only): recursive
    coordinate bisection into n_parts parts, two ghost rings per part, and the
    halo messages that fill them after every stage."""

    def __init__(self, mesh: Mesh, n_parts: int):
        h = C.c_void_p()
        _check(lib.fvlbm_mesh_partition(mesh._h, int(n_parts), C.byref(h)))
        self._h = h
        self.mesh = mesh
        self.n_parts = int(n_parts)
        self.n_cell = mesh.n_cell

    def info(self, part: int) -> dict:
        i = PartInfoT()
        _check(lib.fvlbm_partition_info(self._h, int(part), C.byref(i)))
        return {k: getattr(i, k) for k, _ in PartInfoT._fields_}

    def cells(self, part: int) -> np.ndarray:
        """Whole-mesh cell numbers of the part's local cells: owned, ring 1, ring 2."""
        i = self.info(part)
        out = np.zeros(i["n_owned"] + i["n_ring1"] + i["n_ring2"], np.int64)
        _check(lib.fvlbm_partition_cells(self._h, int(part), out.ctypes.data_as(C.POINTER(C.c_int64))))
        return out

    def halo(self, src: int, dst: int):
        """(src_local, dst_local) of the message src sends dst after every stage."""
        n = C.c_int64()
        _check(lib.fvlbm_partition_halo(self._h, int(src), int(dst), C.byref(n), None, None))
        a, b = np.zeros(n.value, np.int32), np.zeros(n.value, np.int32)
        if n.value:
            _check(lib.fvlbm_partition_halo(self._h, int(src), int(dst), C.byref(n),
                                            a.ctypes.data_as(C.POINTER(C.c_int32)),
                                            b.ctypes.data_as(C.POINTER(C.c_int32))))
        return a, b

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib.fvlbm_partition_destroy(h)
            self._h = None

    def __del__(self):
        self.close()


class DDSolver:
    """Partitioned solve of one mesh on one GPU (fvlbm_dd_* in the header): one
    solver per part of `plan`, the halo exchange after every stage."""

    def __init__(self, plan: Partition, params: ParamsT, stream=None):
        import torch
        if stream is None:
            stream = torch.cuda.Stream(device=params.device)
        self.stream = stream
        self.plan = plan                      # must outlive the solver
        self.n_cell = plan.n_cell
        sh = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream or 0)
        h = C.c_void_p()
        _check(lib.fvlbm_dd_create(plan._h, C.byref(params), 1, C.c_void_p(sh), C.byref(h)))
        self._h = h

    def step(self, n: int = 1):
        _check(lib.fvlbm_dd_step(self._h, int(n)))

    def sync(self):
        _check(lib.fvlbm_dd_sync(self._h))

    def macros(self):
        rho, u = np.zeros(self.n_cell), np.zeros((self.n_cell, 2))
        _check(lib.fvlbm_dd_macros(self._h, _d(rho), _d(u)))
        return rho, u

    def get_f(self) -> np.ndarray:
        f = np.zeros((self.n_cell, 9))
        _check(lib.fvlbm_dd_get_f(self._h, _d(f)))
        return f

    def set_f(self, f):
        f = np.ascontiguousarray(f, np.float64).reshape(self.n_cell, 9)
        _check(lib.fvlbm_dd_set_f(self._h, _d(f)))

    def mass(self) -> float:
        m = C.c_double()
        _check(lib.fvlbm_dd_mass(self._h, C.byref(m)))
        return m.value

    def residual(self) -> float:
        e = C.c_double()
        _check(lib.fvlbm_dd_residual(self._h, C.byref(e)))
        return e.value

    def stage_kernel(self):
        """(stage kernel of the parts, kernel launches per time step)."""
        k, n = C.c_int32(), C.c_int64()
        _check(lib.fvlbm_dd_stage_kernel(self._h, C.byref(k), C.byref(n)))
        return k.value, n.value

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib.fvlbm_dd_destroy(h)
            self._h = None

    def __del__(self):
        self.close()


REQ_QUEUED, REQ_ACTIVE, REQ_DONE, REQ_FAILED = 0, 1, 2, 3


class Server:
    """Continuous-batching solve server on one GPU (see fvlbm_server_* in the header)."""

    def __init__(self, arena_bytes: int, device: int = 0, n_streams: int = 4, max_active: int = 16,
                 check_interval: int = 1000, residual_tol: float = 1e-8, max_steps: int = 20000):
        cfg = ServerConfigT(device, n_streams, int(arena_bytes), max_active, check_interval, residual_tol, max_steps)
        h = C.c_void_p()
        _check(lib.fvlbm_server_create(C.byref(cfg), C.byref(h)))
        self._h = h
        self._meshes = {}

    def submit(self, mesh: Mesh, params) -> int:
        plist = [params] if isinstance(params, ParamsT) else list(params)
        arr = (ParamsT * len(plist))(*plist)
        rid = C.c_int64()
        _check(lib.fvlbm_server_submit(self._h, mesh._h, arr, len(plist), C.byref(rid)))
        self._meshes[rid.value] = mesh          # the mesh must outlive the request
        return rid.value

    def poll(self) -> int:
        n = C.c_int32()
        _check(lib.fvlbm_server_poll(self._h, C.byref(n)))
        return n.value

    def request(self, rid: int, fields: bool = False):
        info = RequestInfoT()
        _check(lib.fvlbm_server_request(self._h, rid, C.byref(info), None, None))
        d = {k: getattr(info, k) for k, _ in RequestInfoT._fields_}
        if fields and info.state == REQ_DONE:
            rho = np.zeros(info.n_cell)
            u = np.zeros((info.n_cell, 2))
            _check(lib.fvlbm_server_request(self._h, rid, C.byref(info), _d(rho), _d(u)))
            d["rho"], d["u"] = rho, u
        if info.state in (REQ_DONE, REQ_FAILED):
            self._meshes.pop(rid, None) if fields else None
        return d

    def stats(self) -> dict:
        st = ServerStatsT()
        _check(lib.fvlbm_server_stats(self._h, C.byref(st)))
        return {k: getattr(st, k) for k, _ in ServerStatsT._fields_}

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib.fvlbm_server_destroy(h)
            self._h = None

    def __del__(self):
        self.close()
