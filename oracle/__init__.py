"""Python access to the plain FP64 CPU oracle (oracle.cpp).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline / reference leg load this module; the library never does.

State arrays follow the host layout U[k, c, i] (k = 0: Wbar, 1: Vbar, 2: Ybar).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")

EQ = {"advection": 0, "burgers": 1, "euler": 2}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc: no fast-math, no FMA contraction."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math",
                               "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        d, i64, i32 = ctypes.c_double, ctypes.c_int64, ctypes.c_int32
        vp = ctypes.c_void_p
        _lib.orc_create.argtypes = [vp, i64, vp, i64, d, d, ctypes.c_int, ctypes.c_int, d, d, d, d, vp, d,
                                    ctypes.c_int, P(vp)]
        _lib.orc_destroy.argtypes = [vp]
        _lib.orc_set_positivity.argtypes = [vp, ctypes.c_int]
        _lib.orc_set_time_rule.argtypes = [vp, ctypes.c_int]
        _lib.orc_neighbors.argtypes = [vp, vp, vp]
        _lib.orc_cell_geometry.argtypes = [vp, vp]
        _lib.orc_cfl_dt.argtypes = [vp, vp]
        _lib.orc_cfl_dt.restype = d
        _lib.orc_step.argtypes = [vp, vp, d, vp, vp]
        _lib.orc_run_to.argtypes = [vp, vp, d, d, i64, P(i64), vp]
        _lib.orc_run_dual.argtypes = [vp, vp, vp, vp, i64]
        _lib.orc_reconstruct_cell.argtypes = [vp, vp, i64, ctypes.c_int, vp, vp, vp, vp, vp]
        _lib.orc_lax_wendroff.argtypes = [ctypes.c_int, d, d, d, vp, vp]
        _lib.orc_cell_taylor.argtypes = [vp, vp, d, i64, vp]
        _lib.orc_flux_derivs.argtypes = [ctypes.c_int, d, d, d, vp, vp, vp, vp]
        _lib.orc_step_cells.argtypes = [vp, vp, d, vp, i64, vp]
        _lib.orc_set_boundary.argtypes = [vp, vp]
        _lib.orc_set_inflow.argtypes = [vp, vp]
        _lib.orc_spectral_radius.argtypes = [ctypes.c_int, d, d, d, vp, d, d, vp]
        _lib.orc_admissible_fraction.argtypes = [d, vp, vp, d]
        _lib.orc_admissible_fraction.restype = d
        _lib.orc_last_error.restype = ctypes.c_char_p
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(rc):
    if rc != 0:
        raise RuntimeError(f"oracle error {rc}: {lib().orc_last_error().decode()}")


class Oracle:
    """One mesh + equation.  All arrays are float64 in the caller's numbering."""

    def __init__(self, mesh, eq: str = "advection", a=(1.0, 1.0), gamma_gas: float = 1.4, cfl: float = 0.5,
                 gamma_lin=(0.94, 0.02, 0.02, 0.02), eps: float = 1e-8, linear_only: bool = False,
                 positivity: bool = False, time_rule: str = "lobatto", inflow=None):
        L = lib()
        self.mesh = mesh
        self.eq = EQ[eq]
        self.m = 4 if eq == "euler" else 1
        self.nt = mesh.nt
        self._xy = np.ascontiguousarray(mesh.xy, dtype=np.float64)
        self._tri = np.ascontiguousarray(mesh.tri, dtype=np.int32)
        self._gl = np.asarray(gamma_lin, dtype=np.float64)
        h = ctypes.c_void_p()
        _check(L.orc_create(_ptr(self._xy), mesh.nv, _ptr(self._tri), mesh.nt, mesh.Lx, mesh.Ly, mesh.bc,
                            self.eq, a[0], a[1], gamma_gas, cfl, _ptr(self._gl), eps, int(linear_only),
                            ctypes.byref(h)))
        self._h = h
        if positivity:
            # True: scale limiter + flux blending; "scale_only": the scale limiter alone
            _check(L.orc_set_positivity(h, 2 if positivity == "scale_only" else 1))
        if getattr(mesh, "edge_bc", None) is not None:
            self._ebc = np.ascontiguousarray(mesh.edge_bc, dtype=np.int32)
            _check(L.orc_set_boundary(h, _ptr(self._ebc)))
        if inflow is not None:
            self._win = np.ascontiguousarray(inflow, dtype=np.float64)
            _check(L.orc_set_inflow(h, _ptr(self._win)))
        if time_rule != "lobatto":
            _check(L.orc_set_time_rule(h, {"gauss": 1}[time_rule]))
        self.a = a
        self.gamma_gas = gamma_gas

    def __del__(self):
        if getattr(self, "_h", None):
            lib().orc_destroy(self._h)
            self._h = None

    def neighbors(self):
        nbr = np.empty((self.nt, 3), np.int32); nbe = np.empty((self.nt, 3), np.int32)
        _check(lib().orc_neighbors(self._h, _ptr(nbr), _ptr(nbe)))
        return nbr, nbe

    def cell_geometry(self):
        out = np.empty((4, self.nt))
        _check(lib().orc_cell_geometry(self._h, _ptr(out)))
        return {"area": out[0], "cx": out[1], "cy": out[2], "inradius": out[3]}

    def _u(self, U):
        U = np.ascontiguousarray(U, dtype=np.float64)
        assert U.shape == (3, self.m, self.nt), U.shape
        return U

    def cfl_dt(self, U):
        return float(lib().orc_cfl_dt(self._h, _ptr(self._u(U))))

    def step(self, U, dt, mask=None):
        U = self._u(U)
        out = np.empty_like(U)
        mk = None
        if mask is not None:
            mk = np.ascontiguousarray(mask, dtype=np.uint8)
        _check(lib().orc_step(self._h, _ptr(U), dt, _ptr(out), _ptr(mk) if mk is not None else None))
        return out

    def step_cells(self, U, dt, cells):
        """One step of the given cells only -> their new values [3, m, len(cells)]
        (cells ascending; the cost grows with their number, not the mesh's)."""
        U = self._u(U)
        c = np.ascontiguousarray(np.sort(np.asarray(cells, dtype=np.int64)))
        out = np.empty((3, self.m, c.size))
        _check(lib().orc_step_cells(self._h, _ptr(U), float(dt), _ptr(c), c.size, _ptr(out)))
        return out

    def run_to(self, U, T, t0=0.0, max_steps=10 ** 9):
        U = self._u(U).copy()
        n = ctypes.c_int64()
        cap = 200000
        dts = np.zeros(cap)
        _check(lib().orc_run_to(self._h, _ptr(U), t0, T, min(max_steps, cap), ctypes.byref(n), _ptr(dts)))
        return U, dts[: n.value].copy()

    def run_dts(self, U, dts):
        U = self._u(U).copy()
        out = U
        for dt in dts:
            out = self.step(out, float(dt))
        return out

    def run_dual(self, U, dU, dts):
        U = self._u(U).copy(); dU = self._u(dU).copy()
        dts = np.ascontiguousarray(dts, dtype=np.float64)
        _check(lib().orc_run_dual(self._h, _ptr(U), _ptr(dU), _ptr(dts), len(dts)))
        return U, dU

    def cell_taylor(self, U, dt, cell: int):
        """Taylor data (W, Wt, Wtt) at the six edge Gauss points of a cell,
        after the limiter when it is on -> [6, 3, m]."""
        U = self._u(U)
        out = np.empty((6, 3, self.m))
        _check(lib().orc_cell_taylor(self._h, _ptr(U), float(dt), int(cell), _ptr(out)))
        return out

    def reconstruct_cell(self, U, cell: int, comp: int = 0):
        U = self._u(U)
        polys = np.empty((4, 6, 6)); rec = np.empty((6, 6)); beta = np.empty(4); om = np.empty(4)
        gp = np.empty((6, 2))
        _check(lib().orc_reconstruct_cell(self._h, _ptr(U), cell, comp, _ptr(polys), _ptr(rec), _ptr(beta),
                                          _ptr(om), _ptr(gp)))
        return {"polys": polys, "recon": rec, "beta": beta, "omega": om, "gp": gp}


def lax_wendroff(eq: str, jet, a=(1.0, 1.0), gamma_gas: float = 1.4):
    """jet[6, m] = (W, Wx, Wy, Wxx, Wxy, Wyy) -> [4, m] = (Wt, Wtx, Wty, Wtt)."""
    jet = np.ascontiguousarray(jet, dtype=np.float64)
    m = jet.shape[1]
    out = np.empty((4, m))
    _check(lib().orc_lax_wendroff(EQ[eq], a[0], a[1], gamma_gas, _ptr(jet), _ptr(out)))
    return out


def flux_derivs(eq: str, W, da, db, a=(1.0, 1.0), gamma_gas: float = 1.4):
    """-> [6, m] = f'a, f'b, f''[a]b, g'a, g'b, g''[a]b at W."""
    W = np.ascontiguousarray(W, dtype=np.float64)
    da = np.ascontiguousarray(da, dtype=np.float64); db = np.ascontiguousarray(db, dtype=np.float64)
    out = np.empty((6, W.shape[0]))
    _check(lib().orc_flux_derivs(EQ[eq], a[0], a[1], gamma_gas, _ptr(W), _ptr(da), _ptr(db), _ptr(out)))
    return out


def spectral_radius(eq: str, W, n, a=(1.0, 1.0), gamma_gas: float = 1.4):
    """(largest |eigenvalue| of d(F.n)/dW for the unit normal n, largest over all directions)."""
    W = np.ascontiguousarray(W, dtype=np.float64)
    out = np.empty(2)
    _check(lib().orc_spectral_radius(EQ[eq], a[0], a[1], gamma_gas, _ptr(W), float(n[0]), float(n[1]), _ptr(out)))
    return float(out[0]), float(out[1])


def admissible_fraction(Wb, w, eps, gamma_gas: float = 1.4):
    """Largest f in [0, 1] with density and pressure >= eps on Wb + f (w - Wb)."""
    Wb = np.ascontiguousarray(Wb, dtype=np.float64); w = np.ascontiguousarray(w, dtype=np.float64)
    return float(lib().orc_admissible_fraction(gamma_gas, _ptr(Wb), _ptr(w), float(eps)))
