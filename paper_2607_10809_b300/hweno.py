"""Thin Python binding of the C ABI in include/hweno.h (argument marshalling only).

Every step of the scheme runs in the CUDA library; this module only converts
numpy arrays to pointers, allocates the device workspace as a torch uint8
tensor and passes torch's current CUDA stream.  It fails loudly when the
library has not been built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libhweno.so")

HW_OK, HW_EINVAL, HW_ENOMEM, HW_ECUDA, HW_EMESH, HW_ENONFINITE, HW_ETIMEOUT, HW_ESTATE = range(8)
STATUS_NAMES = ["HW_OK", "HW_EINVAL", "HW_ENOMEM", "HW_ECUDA", "HW_EMESH", "HW_ENONFINITE", "HW_ETIMEOUT",
                "HW_ESTATE"]
EQUATIONS = {"advection": 0, "burgers": 1, "euler": 2}
PRECISIONS = {"fp64": 0, "fp32": 1}

# every symbol declared in include/hweno.h
EXPORTED = ["hw_options_default", "hw_mesh_create", "hw_mesh_set_boundary", "hw_mesh_destroy", "hw_mesh_ntri", "hw_mesh_neighbors",
            "hw_mesh_permutation", "hw_workspace_bytes", "hw_state_init", "hw_set_state", "hw_step", "hw_run_to",
            "hw_get_state", "hw_conservation", "hw_status_flags", "hw_time", "hw_profile", "hw_profile_read",
            "hw_solver_destroy", "hw_step_kernels", "hw_last_error", "hw_step_static_scratch", "hw_batch_schedule_default",
            "hw_batch_workspace_bytes", "hw_batch_create", "hw_batch_set_schedule", "hw_batch_get_schedule",
            "hw_batch_autotune", "hw_batch_run_to", "hw_batch_steps", "hw_batch_reset", "hw_batch_get_state",
            "hw_batch_destroy", "hw_state_bytes", "hw_state_export", "hw_state_import", "hw_state_row_words",
            "hw_state_rows_export", "hw_state_rows_import", "hw_host_to_internal",
            "hw_internal_to_host", "hw_pb_bytes", "hw_step_keep", "hw_adjoint_scratch_bytes", "hw_step_adjoint"]


class HwError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")
        self.status = status


class Options(ctypes.Structure):
    _fields_ = [("eq", ctypes.c_int32), ("positivity", ctypes.c_int32), ("time_rule", ctypes.c_int32),
                ("step_kernels", ctypes.c_int32), ("ax", ctypes.c_double),
                ("ay", ctypes.c_double), ("gamma_gas", ctypes.c_double), ("cfl", ctypes.c_double),
                ("gamma_lin", ctypes.c_double * 4), ("eps", ctypes.c_double), ("inflow", ctypes.c_double * 4)]


class Schedule(ctypes.Structure):
    _fields_ = [("blocks_per_sm", ctypes.c_int32), ("tile_order", ctypes.c_int32),
                ("steps_per_launch", ctypes.c_int32), ("withhold_block", ctypes.c_int32),
                ("spin_limit", ctypes.c_int64), ("launch_mode", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None


def load():
    """Load libhweno.so (built by paper_2607_10809_b300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: run paper_2607_10809_b300/build.py (no CPU fallback exists)")
    L = ctypes.CDLL(LIB_PATH)
    vp, i64, i32, d, sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_size_t
    P = ctypes.POINTER
    sig = {
        "hw_options_default": (None, [P(Options)]),
        "hw_mesh_create": (ctypes.c_int, [vp, i64, vp, i64, d, d, i32, P(vp)]),
        "hw_mesh_destroy": (ctypes.c_int, [vp]),
        "hw_mesh_set_boundary": (ctypes.c_int, [vp, vp]),
        "hw_mesh_ntri": (i64, [vp]),
        "hw_mesh_neighbors": (ctypes.c_int, [vp, vp, vp]),
        "hw_mesh_permutation": (ctypes.c_int, [vp, vp]),
        "hw_workspace_bytes": (ctypes.c_int, [vp, P(Options), i32, P(sz)]),
        "hw_state_init": (ctypes.c_int, [vp, P(Options), i32, vp, vp, vp, vp, sz, vp, P(vp)]),
        "hw_set_state": (ctypes.c_int, [vp, vp, vp, vp, d]),
        "hw_step": (ctypes.c_int, [vp, d]),
        "hw_run_to": (ctypes.c_int, [vp, d, P(i64)]),
        "hw_get_state": (ctypes.c_int, [vp, vp, vp, vp, P(d)]),
        "hw_conservation": (ctypes.c_int, [vp, vp]),
        "hw_status_flags": (ctypes.c_int, [vp, P(ctypes.c_uint32)]),
        "hw_time": (ctypes.c_int, [vp, P(d), P(d), P(i64)]),
        "hw_profile": (ctypes.c_int, [vp, i32]),
        "hw_profile_read": (ctypes.c_int, [vp, vp, P(i64)]),
        "hw_solver_destroy": (ctypes.c_int, [vp]),
        "hw_step_kernels": (ctypes.c_int, [vp, P(i32)]),
        "hw_last_error": (ctypes.c_char_p, []),
        "hw_step_static_scratch": (ctypes.c_int, [vp, d]),
        "hw_batch_schedule_default": (None, [P(Schedule)]),
        "hw_batch_workspace_bytes": (ctypes.c_int, [vp, i32, P(Options), i32, P(sz)]),
        "hw_batch_create": (ctypes.c_int, [vp, i32, P(Options), i32, vp, vp, vp, vp, sz, vp, P(vp)]),
        "hw_batch_set_schedule": (ctypes.c_int, [vp, P(Schedule)]),
        "hw_batch_get_schedule": (ctypes.c_int, [vp, P(Schedule), P(i32)]),
        "hw_batch_autotune": (ctypes.c_int, [vp, i32, P(Schedule), P(d)]),
        "hw_batch_run_to": (ctypes.c_int, [vp, d, P(i64)]),
        "hw_batch_steps": (ctypes.c_int, [vp, i32, P(d)]),
        "hw_batch_reset": (ctypes.c_int, [vp]),
        "hw_batch_get_state": (ctypes.c_int, [vp, i32, vp, vp, vp, P(d), P(i64), P(i32)]),
        "hw_batch_destroy": (ctypes.c_int, [vp]),
        "hw_state_bytes": (ctypes.c_int, [vp, P(sz)]),
        "hw_state_export": (ctypes.c_int, [vp, vp]),
        "hw_state_import": (ctypes.c_int, [vp, vp, d]),
        "hw_state_row_words": (ctypes.c_int, [vp, P(i32)]),
        "hw_state_rows_export": (ctypes.c_int, [vp, vp, i64, vp]),
        "hw_state_rows_import": (ctypes.c_int, [vp, vp, i64, vp, i32]),
        "hw_host_to_internal": (ctypes.c_int, [vp, vp, vp, vp, vp]),
        "hw_internal_to_host": (ctypes.c_int, [vp, vp, vp, vp, vp]),
        "hw_adjoint_scratch_bytes": (ctypes.c_int, [vp, P(sz)]),
        "hw_pb_bytes": (ctypes.c_int, [vp, P(sz)]),
        "hw_step_keep": (ctypes.c_int, [vp, d, vp]),
        "hw_step_adjoint": (ctypes.c_int, [vp, d, vp, vp, vp, vp, vp, sz]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(rc):
    if rc != HW_OK:
        raise HwError(rc, load().hw_last_error().decode())


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


TIME_RULES = {"lobatto": 0, "gauss": 1}
STEP_KERNELS = {"default": 0, "separate": 1, "fused": 2, "edge_once": 3}


def options(eq="advection", a=(1.0, 1.0), gamma_gas=1.4, cfl=0.5, gamma_lin=(0.94, 0.02, 0.02, 0.02), eps=1e-8,
            positivity=False, time_rule="lobatto", step_kernels="default", inflow=None):
    o = Options()
    load().hw_options_default(ctypes.byref(o))
    o.eq = EQUATIONS[eq]
    o.positivity = int(bool(positivity))
    o.time_rule = TIME_RULES[time_rule]
    o.step_kernels = STEP_KERNELS[step_kernels]
    o.ax, o.ay = a
    o.gamma_gas = gamma_gas
    o.cfl = cfl
    for k in range(4):
        o.gamma_lin[k] = gamma_lin[k]
    o.eps = eps
    if inflow is not None:
        for k, v in enumerate(np.asarray(inflow, dtype=np.float64).ravel()[:4]):
            o.inflow[k] = v
    return o


# ------------------------------------------------------------------ C-ABI names
def hw_mesh_create(xy, tri, Lx=0.0, Ly=0.0, bc=0):
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    tri = np.ascontiguousarray(tri, dtype=np.int32)
    h = ctypes.c_void_p()
    _check(load().hw_mesh_create(_ptr(xy), xy.shape[0], _ptr(tri), tri.shape[0], float(Lx), float(Ly), int(bc),
                                 ctypes.byref(h)))
    return h


def hw_mesh_neighbors(h, nt):
    nbr = np.empty((nt, 3), np.int32); nbe = np.empty((nt, 3), np.int32)
    _check(load().hw_mesh_neighbors(h, _ptr(nbr), _ptr(nbe)))
    return nbr, nbe


def hw_mesh_permutation(h, nt):
    p = np.empty(nt, np.int32)
    _check(load().hw_mesh_permutation(h, _ptr(p)))
    return p


def hw_workspace_bytes(h, opt, precision):
    n = ctypes.c_size_t()
    _check(load().hw_workspace_bytes(h, ctypes.byref(opt), PRECISIONS[precision], ctypes.byref(n)))
    return n.value


class Mesh:
    """Host mesh handle (hw_mesh)."""

    def __init__(self, mesh):
        self.src = mesh
        self.nt = mesh.nt
        self.h = hw_mesh_create(mesh.xy, mesh.tri, mesh.Lx, mesh.Ly, mesh.bc)
        if getattr(mesh, "edge_bc", None) is not None:
            self._ebc = np.ascontiguousarray(mesh.edge_bc, dtype=np.int32)
            _check(load().hw_mesh_set_boundary(self.h, _ptr(self._ebc)))

    def neighbors(self):
        return hw_mesh_neighbors(self.h, self.nt)

    def permutation(self):
        return hw_mesh_permutation(self.h, self.nt)

    def __del__(self):
        if getattr(self, "h", None) is not None and _lib is not None:
            _lib.hw_mesh_destroy(self.h)
            self.h = None


class Solver:
    """One solve on the current CUDA device (hw_solver).  State arrays follow
    the host layout U[k, c, i] (k: Wbar, Vbar, Ybar) in the caller's numbering."""

    def __init__(self, mesh, U0, eq="advection", precision="fp64", stream=None, **opt_kw):
        import torch
        self.mesh = mesh if isinstance(mesh, Mesh) else Mesh(mesh)
        self.m = 4 if eq == "euler" else 1
        self.eq = eq
        self.precision = precision
        self.opt = options(eq, **opt_kw)
        nbytes = hw_workspace_bytes(self.mesh.h, self.opt, precision)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        U0 = np.ascontiguousarray(U0, dtype=np.float64)
        assert U0.shape == (3, self.m, self.mesh.nt), U0.shape
        h = ctypes.c_void_p()
        _check(load().hw_state_init(self.mesh.h, ctypes.byref(self.opt), PRECISIONS[precision], _ptr(U0[0]),
                                    _ptr(U0[1]), _ptr(U0[2]), ctypes.c_void_p(self.workspace.data_ptr()), nbytes,
                                    ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)))
        self.h = h

    def set_state(self, U, t=0.0):
        U = np.ascontiguousarray(U, dtype=np.float64)
        _check(load().hw_set_state(self.h, _ptr(U[0]), _ptr(U[1]), _ptr(U[2]), float(t)))
        self._keep = U   # the copy is asynchronous

    def step(self, dt=0.0):
        _check(load().hw_step(self.h, float(dt)))

    def step_static_scratch(self, dt=0.0):
        """hw_step with the step's scratch in the library's static device array
        (for callers that cannot allocate device memory; see include/hweno.h)."""
        _check(load().hw_step_static_scratch(self.h, float(dt)))

    def run_to(self, T):
        n = ctypes.c_int64()
        _check(load().hw_run_to(self.h, float(T), ctypes.byref(n)))
        return n.value

    def get_state(self, out=None):
        """Returns (U, t); ``out`` may be a preallocated float64 array [3, m, nt]
        (pinned memory makes the device-to-host copy direct)."""
        U = np.empty((3, self.m, self.mesh.nt)) if out is None else out
        assert U.shape == (3, self.m, self.mesh.nt) and U.dtype == np.float64 and U.flags.c_contiguous
        t = ctypes.c_double()
        _check(load().hw_get_state(self.h, _ptr(U[0]), _ptr(U[1]), _ptr(U[2]), ctypes.byref(t)))
        return U, t.value

    def conservation(self):
        s = np.empty(self.m)
        _check(load().hw_conservation(self.h, _ptr(s)))
        return s

    def status_flags(self):
        f = ctypes.c_uint32()
        _check(load().hw_status_flags(self.h, ctypes.byref(f)))
        return f.value

    def time(self):
        t = ctypes.c_double(); dt = ctypes.c_double(); n = ctypes.c_int64()
        _check(load().hw_time(self.h, ctypes.byref(t), ctypes.byref(dt), ctypes.byref(n)))
        return t.value, dt.value, n.value

    # ---- device-side state buffers (internal order / precision, torch uint8 tensors)
    def state_buffer(self):
        import torch
        n = ctypes.c_size_t()
        _check(load().hw_state_bytes(self.h, ctypes.byref(n)))
        return torch.empty(n.value, dtype=torch.uint8, device="cuda")

    def export_state(self, buf):
        _check(load().hw_state_export(self.h, ctypes.c_void_p(buf.data_ptr())))

    def import_state(self, buf, t=0.0):
        _check(load().hw_state_import(self.h, ctypes.c_void_p(buf.data_ptr()), float(t)))

    def state_row_words(self):
        """Values per row of hw_state_rows_export / import (record, then in
        FP32 the compensation words)."""
        w = ctypes.c_int32()
        _check(load().hw_state_row_words(self.h, ctypes.byref(w)))
        return w.value

    def state_rows_export(self, rows, out):
        """out[k] = row rows[k] of the current state (rows: int32 CUDA tensor of
        internal cell indices; out: CUDA tensor [len(rows), state_row_words()]
        of the solver's precision)."""
        _check(load().hw_state_rows_export(self.h, ctypes.c_void_p(rows.data_ptr()), rows.numel(),
                                           ctypes.c_void_p(out.data_ptr())))

    def state_rows_import(self, rows=None, buf=None, refresh=False):
        """Row rows[k] of the current state = buf[k]; refresh: then recompute
        the CFL step (rows may be None for a refresh alone)."""
        n = 0 if rows is None else rows.numel()
        _check(load().hw_state_rows_import(self.h, ctypes.c_void_p(rows.data_ptr() if n else None), n,
                                           ctypes.c_void_p(buf.data_ptr() if n else None), int(bool(refresh))))

    def host_to_internal(self, U, buf):
        U = np.ascontiguousarray(U, dtype=np.float64)
        _check(load().hw_host_to_internal(self.h, _ptr(U[0]), _ptr(U[1]), _ptr(U[2]), ctypes.c_void_p(buf.data_ptr())))

    def internal_to_host(self, buf, out=None):
        """``out``: optional float64 array [3, m, nt] (pinned memory makes the
        device-to-host copy direct)."""
        U = np.empty((3, self.m, self.mesh.nt)) if out is None else out
        assert U.shape == (3, self.m, self.mesh.nt) and U.dtype == np.float64 and U.flags.c_contiguous
        _check(load().hw_internal_to_host(self.h, ctypes.c_void_p(buf.data_ptr()), _ptr(U[0]), _ptr(U[1]), _ptr(U[2])))
        return U

    def pb_buffer(self):
        """Edge-point buffer (torch uint8 tensor) for step_keep / step_adjoint."""
        import torch
        n = ctypes.c_size_t()
        _check(load().hw_pb_bytes(self.h, ctypes.byref(n)))
        return torch.empty(n.value, dtype=torch.uint8, device="cuda")

    def step_keep(self, dt, pb):
        """hw_step that leaves the edge-point data of the pre-step state in pb."""
        _check(load().hw_step_keep(self.h, float(dt), ctypes.c_void_p(pb.data_ptr())))

    def adjoint_scratch(self):
        import torch
        n = ctypes.c_size_t()
        _check(load().hw_adjoint_scratch_bytes(self.h, ctypes.byref(n)))
        return torch.empty(n.value, dtype=torch.uint8, device="cuda")

    def step_adjoint(self, dt, U_n, Ubar_next, Ubar_n, scratch, pb=None):
        """Ubar_n = (dU^{n+1}/dU^n)^T Ubar_next for a step of size dt (buffers:
        state_buffer() tensors; scratch: adjoint_scratch(); pb: the
        pb_buffer() that step_keep(dt, pb) filled from U_n, or None)."""
        _check(load().hw_step_adjoint(self.h, float(dt), ctypes.c_void_p(U_n.data_ptr()),
                                      ctypes.c_void_p(pb.data_ptr() if pb is not None else None),
                                      ctypes.c_void_p(Ubar_next.data_ptr()), ctypes.c_void_p(Ubar_n.data_ptr()),
                                      ctypes.c_void_p(scratch.data_ptr()), scratch.numel()))

    def step_kernels(self):
        """'separate', 'fused' or 'edge_once': the kernels this solver's steps run."""
        p = ctypes.c_int32()
        _check(load().hw_step_kernels(self.h, ctypes.byref(p)))
        return {1: "separate", 2: "fused", 3: "edge_once"}[p.value]

    def profile(self, enable=True):
        _check(load().hw_profile(self.h, int(enable)))

    def profile_read(self):
        ms = np.zeros(2); n = ctypes.c_int64()
        _check(load().hw_profile_read(self.h, _ptr(ms), ctypes.byref(n)))
        return {"recon_ms": float(ms[0]), "edge_ms": float(ms[1]), "steps": n.value}

    def close(self):
        if getattr(self, "h", None) is not None and _lib is not None:
            _lib.hw_solver_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()


class Batch:
    """Many independent solves advanced together in one persistent launch
    (hw_batch).  meshes: list of inputs.Mesh; states: list of U[3, m, nt]."""

    def __init__(self, meshes, states, eq="euler", precision="fp32", stream=None, **opt_kw):
        import torch
        self.meshes = [m if isinstance(m, Mesh) else Mesh(m) for m in meshes]
        self.n = len(self.meshes)
        self.m = 4 if eq == "euler" else 1
        self.opt = options(eq, **opt_kw)
        self.precision = precision
        hs = (ctypes.c_void_p * self.n)(*[mm.h.value for mm in self.meshes])
        self._hs = hs
        n = ctypes.c_size_t()
        _check(load().hw_batch_workspace_bytes(hs, self.n, ctypes.byref(self.opt), PRECISIONS[precision],
                                               ctypes.byref(n)))
        self.workspace = torch.empty(n.value, dtype=torch.uint8, device="cuda")
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._states = [np.ascontiguousarray(U, dtype=np.float64) for U in states]
        for U, mm in zip(self._states, self.meshes):
            assert U.shape == (3, self.m, mm.nt), U.shape
        W = (ctypes.c_void_p * self.n)(*[U[0].ctypes.data for U in self._states])
        V = (ctypes.c_void_p * self.n)(*[U[1].ctypes.data for U in self._states])
        Y = (ctypes.c_void_p * self.n)(*[U[2].ctypes.data for U in self._states])
        h = ctypes.c_void_p()
        _check(load().hw_batch_create(hs, self.n, ctypes.byref(self.opt), PRECISIONS[precision], W, V, Y,
                                      ctypes.c_void_p(self.workspace.data_ptr()), n.value,
                                      ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)))
        self.h = h

    def schedule(self):
        s = Schedule(); g = ctypes.c_int32()
        _check(load().hw_batch_get_schedule(self.h, ctypes.byref(s), ctypes.byref(g)))
        d = s.as_dict(); d["grid_blocks"] = g.value
        return d

    def set_schedule(self, **kw):
        s = Schedule(); g = ctypes.c_int32()
        _check(load().hw_batch_get_schedule(self.h, ctypes.byref(s), ctypes.byref(g)))
        for k, v in kw.items():
            setattr(s, k, v)
        _check(load().hw_batch_set_schedule(self.h, ctypes.byref(s)))

    def autotune(self, trial_steps=8):
        s = Schedule(); ms = ctypes.c_double()
        _check(load().hw_batch_autotune(self.h, int(trial_steps), ctypes.byref(s), ctypes.byref(ms)))
        d = s.as_dict(); d["trial_ms"] = ms.value
        return d

    def run_to(self, T):
        cs = ctypes.c_int64()
        _check(load().hw_batch_run_to(self.h, float(T), ctypes.byref(cs)))
        return cs.value

    def steps(self, k):
        ms = ctypes.c_double()
        _check(load().hw_batch_steps(self.h, int(k), ctypes.byref(ms)))
        return ms.value

    def reset(self):
        _check(load().hw_batch_reset(self.h))

    def get_state(self, k):
        U = np.empty((3, self.m, self.meshes[k].nt))
        t = ctypes.c_double(); ns = ctypes.c_int64(); f = ctypes.c_int32()
        _check(load().hw_batch_get_state(self.h, int(k), U[0].ctypes.data_as(ctypes.c_void_p),
                                         U[1].ctypes.data_as(ctypes.c_void_p), U[2].ctypes.data_as(ctypes.c_void_p),
                                         ctypes.byref(t), ctypes.byref(ns), ctypes.byref(f)))
        return U, t.value, ns.value, bool(f.value)

    def close(self):
        if getattr(self, "h", None) is not None and _lib is not None:
            _lib.hw_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

