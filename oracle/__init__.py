"""ctypes front end of the plain C FP64 oracle (lmood_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the benchmark's
CPU-baseline / reference leg. The product path (the CUDA library and its binding) never
imports this package, and this package imports nothing from the product path.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lmood_oracle.c")
_LIB = os.path.join(_HERE, "liblmood_oracle.so")
_TSRC = os.path.join(_HERE, "lmood_tangent.cpp")
_TLIB = os.path.join(_HERE, "liblmood_tangent.so")

F_X, F_VP, F_VSTAR, F_V, F_E, F_F, F_TAU, F_ORDER, F_MASS, F_PKM, F_PKR = range(11)
ERR = {0: "ok", 1: "bad argument", 2: "bad mesh", 5: "parachute failure", 6: "MOOD iteration limit"}


def _stale(lib: str, *srcs: str) -> bool:
    return not os.path.exists(lib) or any(os.path.getmtime(lib) < os.path.getmtime(f) for f in srcs)


def build(force: bool = False) -> str:
    """Compile the oracle with plain gcc (-O2, no FP contraction, OpenMP), and its tangent
    build (the same source as C++ with dual numbers, lmood_tangent.cpp) with g++."""
    if force or _stale(_LIB, _SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    if force or _stale(_TLIB, _SRC, _TSRC):
        tmp = _TLIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _TSRC, "-lm"], cwd=_HERE)
        os.replace(tmp, _TLIB)
    return _LIB


class Params(C.Structure):
    _fields_ = [("cfl", C.c_double), ("Cv", C.c_double), ("Ci", C.c_double),
                ("delta0", C.c_double), ("delta1", C.c_double), ("dt_fixed", C.c_double),
                ("max_mood_iters", C.c_int), ("order", C.c_int), ("mood", C.c_int),
                ("vol_coeff", C.c_int), ("cascade", C.c_int), ("shear_a", C.c_double),
                ("eos", C.c_int), ("gamma", C.c_double), ("p_inf", C.c_double), ("p0", C.c_double)]


class Info(C.Structure):
    _fields_ = [("t", C.c_double), ("dt_used", C.c_double), ("dt_next", C.c_double),
                ("step", C.c_long), ("n_troubled", C.c_int), ("n_p0", C.c_int),
                ("mood_iters", C.c_int), ("n_parachute", C.c_int), ("n_p0_eps", C.c_int), ("n_lim", C.c_int),
                ("mass", C.c_double),
                ("mom", C.c_double * 3), ("energy", C.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        dp = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
        ip = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
        L = _lib
        L.orc_mesh_new.argtypes = [C.c_int, C.c_long, dp, C.c_long, ip, C.c_long, C.c_void_p,
                                   C.c_void_p, C.POINTER(C.c_void_p)]
        L.orc_mesh_free.argtypes = [C.c_void_p]
        L.orc_state_new.argtypes = [C.c_void_p, C.c_double, C.c_double, dp, dp, C.c_void_p,
                                    C.POINTER(Params), C.POINTER(C.c_void_p)]
        L.orc_state_free.argtypes = [C.c_void_p]
        L.orc_step.argtypes = [C.c_void_p, C.POINTER(Info)]
        L.orc_get.argtypes = [C.c_void_p, C.c_int, dp]
        L.orc_get_dt.argtypes = [C.c_void_p]
        L.orc_get_dt.restype = C.c_double
        L.orc_get_t.argtypes = [C.c_void_p]
        L.orc_get_t.restype = C.c_double
        L.orc_set_state.argtypes = [C.c_void_p] + [C.c_void_p] * 5 + [C.c_double]
        L.orc_cell_geometry.argtypes = [C.c_int, dp, dp, dp, dp, dp, dp]
        L.orc_stress.argtypes = [C.c_int, dp, C.c_double, C.c_double, dp]
        L.orc_free_energy.argtypes = [C.c_int, dp, C.c_double, C.c_double, C.c_double]
        L.orc_free_energy.restype = C.c_double
        L.orc_stress_a.argtypes = [C.c_int, dp, C.c_double, C.c_double, C.c_double, dp]
        L.orc_free_energy_a.argtypes = [C.c_int, dp, C.c_double, C.c_double, C.c_double, C.c_double]
        L.orc_free_energy_a.restype = C.c_double
        L.orc_sound_speed.argtypes = [C.c_int, dp, C.c_double, C.c_double, C.c_double]
        L.orc_sound_speed.restype = C.c_double
        L.orc_mesh_stencil.argtypes = [C.c_void_p, C.c_long, np.ctypeslib.ndpointer(np.int64), C.c_long]
        L.orc_mesh_stencil.restype = C.c_long
        L.orc_debug_corner_values.argtypes = [C.c_void_p, C.c_long, C.c_int, dp, dp, dp]
        L.orc_debug_predictor.argtypes = [C.c_void_p, C.c_int, C.c_double, dp, dp]
        L.orc_debug_rdmp.argtypes = [C.c_void_p, C.c_long, C.c_double, C.POINTER(C.c_double),
                                     C.POINTER(C.c_double)]
        L.orc_debug_pad.argtypes = [C.c_void_p, C.c_long, dp, C.c_double, dp, C.c_double]
        L.orc_threads.restype = C.c_int
        L.orc_mesh_bc_ndof.argtypes = [C.c_void_p, C.c_long]
        L.orc_mesh_bc_ndof.restype = C.c_int
        L.orc_mesh_set_bc_values.argtypes = [C.c_void_p, dp]
        L.orc_mesh_set_btag.argtypes = [C.c_void_p, ip]
        L.orc_mesh_set_contact.argtypes = [C.c_void_p, C.c_int, dp, C.c_double]
    return _lib


def default_params(cfl=0.4, **kw) -> Params:
    p = Params(cfl=cfl, Cv=0.2, Ci=0.1, delta0=1e-4, delta1=1e-3, dt_fixed=0.0,
               max_mood_iters=100000, order=2, mood=1, vol_coeff=0, cascade=2, shear_a=-1.0)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def threads() -> int:
    """threads of the oracle's OpenMP loops"""
    return lib().orc_threads()


# ----------------------------------------------------------------------------- unit functions
def cell_geometry(xs: np.ndarray):
    """xs [d+1, d] -> (V, xc[d], N[d+1,d] outward face area vectors, ln[d+1,d], Lc)."""
    xs = np.ascontiguousarray(xs, dtype=np.float64)
    nv, d = xs.shape
    V, xc, N, ln, Lc = np.zeros(1), np.zeros(d), np.zeros(nv * d), np.zeros(nv * d), np.zeros(1)
    lib().orc_cell_geometry(d, xs.ravel(), V, xc, N, ln, Lc)
    return V[0], xc, N.reshape(nv, d), ln.reshape(nv, d), Lc[0]


def stress(F: np.ndarray, mu: float, kappa: float) -> np.ndarray:
    F = np.ascontiguousarray(F, dtype=np.float64)
    d = F.shape[0]
    T = np.zeros(d * d)
    lib().orc_stress(d, F.ravel(), mu, kappa, T)
    return T.reshape(d, d)


def free_energy(F, rho0, mu, kappa) -> float:
    F = np.ascontiguousarray(F, dtype=np.float64)
    return lib().orc_free_energy(F.shape[0], F.ravel(), rho0, mu, kappa)


def stress_a(F: np.ndarray, mu: float, kappa: float, a: float) -> np.ndarray:
    """stress of the shear energy family (Eq. familiy_energies) with parameter a"""
    F = np.ascontiguousarray(F, dtype=np.float64)
    d = F.shape[0]
    T = np.zeros(d * d)
    lib().orc_stress_a(d, F.ravel(), mu, kappa, a, T)
    return T.reshape(d, d)


def free_energy_a(F, rho0, mu, kappa, a) -> float:
    F = np.ascontiguousarray(F, dtype=np.float64)
    return lib().orc_free_energy_a(F.shape[0], F.ravel(), rho0, mu, kappa, a)


def sound_speed(F, rho, mu, kappa) -> float:
    F = np.ascontiguousarray(F, dtype=np.float64)
    return lib().orc_sound_speed(F.shape[0], F.ravel(), rho, mu, kappa)


# ----------------------------------------------------------------------------- step driver
class OracleError(RuntimeError):
    pass


@dataclass
class _Handles:
    mesh: C.c_void_p
    state: C.c_void_p


class Oracle:
    """One mesh + state advanced by the oracle. Arrays are SoA like the library's ABI."""

    def __init__(self, problem, params: Params | None = None, **kw):
        L = lib()
        m = problem.mesh
        self.d = m.dim
        self.nc, self.np = m.n_cells, m.n_nodes
        self.params = params or default_params(problem.cfl, **kw)
        if params is None and "shear_a" not in kw:
            self.params.shear_a = getattr(problem, "shear_a", -1.0)
        sg = getattr(problem, "stiffened_gas", None)
        if params is None and sg is not None:
            self.params.eos = 1
            self.params.gamma, self.params.p_inf, self.params.p0 = sg
        x = np.ascontiguousarray(m.x, dtype=np.float64)
        c2n = np.ascontiguousarray(m.c2n, dtype=np.int32)
        bf = np.ascontiguousarray(m.bface, dtype=np.int32)
        bt = np.ascontiguousarray(m.btag, dtype=np.int32)
        self._keep = (bf, bt)
        hm = C.c_void_p()
        rc = L.orc_mesh_new(self.d, self.np, x.ravel(), self.nc, c2n.ravel(), bt.size,
                            bf.ctypes.data if bt.size else None, bt.ctypes.data if bt.size else None,
                            C.byref(hm))
        if rc:
            raise OracleError(f"orc_mesh_new: {ERR.get(rc, rc)}")
        bcval = getattr(problem, "bcval", None)
        if bcval is not None:
            L.orc_mesh_set_bc_values(hm, np.ascontiguousarray(bcval, dtype=np.float64).ravel())
        contact = getattr(problem, "contact", None)
        if contact is not None:
            planes, eps = contact
            pl = np.ascontiguousarray(planes, dtype=np.float64).ravel()
            L.orc_mesh_set_contact(hm, len(planes), pl, eps)
        hs = C.c_void_p()
        mu = np.ascontiguousarray(problem.mu, dtype=np.float64)
        v = np.ascontiguousarray(problem.v, dtype=np.float64)
        F = None if problem.F is None else np.ascontiguousarray(problem.F, dtype=np.float64)
        rc = L.orc_state_new(hm, problem.rho0, problem.lam, mu, v.ravel(),
                             None if F is None else F.ctypes.data, C.byref(self.params), C.byref(hs))
        if rc:
            L.orc_mesh_free(hm)
            raise OracleError(f"orc_state_new: {ERR.get(rc, rc)}")
        self._h = _Handles(hm, hs)
        self.info = Info()

    def close(self):
        if getattr(self, "_h", None) is not None:
            lib().orc_state_free(self._h.state)
            lib().orc_mesh_free(self._h.mesh)
            self._h = None

    def __del__(self):
        self.close()

    def step(self, n: int = 1, check: bool = True) -> int:
        rc = 0
        for _ in range(n):
            rc = lib().orc_step(self._h.state, C.byref(self.info))
            if rc:
                if check:
                    raise OracleError(f"orc_step: {ERR.get(rc, rc)}")
                break
        return rc

    def get(self, field: int) -> np.ndarray:
        d, nc, np_, nv = self.d, self.nc, self.np, self.d + 1
        shape = {F_X: (d, np_), F_VP: (d, np_), F_VSTAR: (d, np_), F_V: (d, nc), F_E: (nc,),
                 F_F: (d * d, nc), F_TAU: (nc,), F_ORDER: (nc,), F_MASS: (nc,),
                 F_PKM: (d * d, nv, nc), F_PKR: (d, nv, nc)}[field]
        out = np.zeros(int(np.prod(shape)))
        lib().orc_get(self._h.state, field, out)
        return out.reshape(shape)

    def set_state(self, x=None, vp=None, v=None, e=None, F=None, dt=0.0):
        keep = []

        def ptr(a):
            if a is None:
                return None
            a = np.ascontiguousarray(a, dtype=np.float64)
            keep.append(a)
            return a.ctypes.data
        lib().orc_set_state(self._h.state, ptr(x), ptr(vp), ptr(v), ptr(e), ptr(F), float(dt))

    @property
    def dt(self) -> float:
        return lib().orc_get_dt(self._h.state)

    @property
    def t(self) -> float:
        return lib().orc_get_t(self._h.state)

    def stencil(self, c: int) -> np.ndarray:
        buf = np.zeros(4096, dtype=np.int64)
        n = lib().orc_mesh_stencil(self._h.mesh, c, buf, buf.size)
        return buf[:n].copy()

    def corner_values(self, c: int, level: int):
        d = self.d
        nq = d + d * d
        out, lo, hi = np.zeros((d + 1) * nq), np.zeros(nq), np.zeros(nq)
        lib().orc_debug_corner_values(self._h.state, c, level, out, lo, hi)
        return out.reshape(d + 1, nq), lo, hi

    def predictor(self, level: int, dt: float):
        """(v* [nc][nv][d], F* [nc][nv][d][d]): the predictor's corner values of every cell at
        the given level (1, 2 or 3) from the current state with time step dt (reading R8)"""
        d, nc = self.d, self.nc
        ov, oF = np.zeros(nc * (d + 1) * d), np.zeros(nc * (d + 1) * d * d)
        if lib().orc_debug_predictor(self._h.state, level, dt, ov, oF) != 0:
            raise OracleError("orc_debug_predictor: bad level")
        return ov.reshape(nc, d + 1, d), oF.reshape(nc, d + 1, d, d)

    def rdmp(self, c: int, rho_new: float):
        """(admissible, lo, hi): the RDMP decision of Eq. RDMP for a candidate density of cell
        c, and the density range at the current positions over the cell's stencil and itself"""
        lo, hi = C.c_double(), C.c_double()
        ok = lib().orc_debug_rdmp(self._h.state, c, rho_new, C.byref(lo), C.byref(hi))
        if ok < 0:
            raise OracleError("orc_debug_rdmp: bad cell")
        return bool(ok), lo.value, hi.value

    def pad(self, c: int, v, e: float, F, V: float) -> int:
        """Eq. PAD for a candidate of cell c (its material): 0 admissible, 1 only eps below the
        tolerance, 2 not computable (non-finite, V <= 0, det F <= 0)"""
        r = lib().orc_debug_pad(self._h.state, c, np.ascontiguousarray(v, dtype=np.float64).ravel(), e,
                                np.ascontiguousarray(F, dtype=np.float64).ravel(), V)
        if r < 0:
            raise OracleError("orc_debug_pad: bad cell")
        return r

    def bc_ndof(self, p: int) -> int:
        return lib().orc_mesh_bc_ndof(self._h.mesh, p)

    def set_bc_values(self, values):
        """boundary-face values [d][n_bfaces] (traction / pressure / prescribed velocity)"""
        rc = lib().orc_mesh_set_bc_values(self._h.mesh, np.ascontiguousarray(values, dtype=np.float64).ravel())
        if rc:
            raise OracleError(f"orc_mesh_set_bc_values: {ERR.get(rc, rc)}")

    def set_contact(self, planes, eps):
        """contact walls [n][2d] (point, unit normal into the body) and threshold eps"""
        pl = np.ascontiguousarray(planes, dtype=np.float64).ravel()
        rc = lib().orc_mesh_set_contact(self._h.mesh, len(planes), pl, eps)
        if rc:
            raise OracleError(f"orc_mesh_set_contact: {ERR.get(rc, rc)}")

    def set_btag(self, btag):
        """new boundary-face tags [n_bfaces]; per-node conditions re-derived"""
        rc = lib().orc_mesh_set_btag(self._h.mesh, np.ascontiguousarray(btag, dtype=np.int32).ravel())
        if rc:
            raise OracleError(f"orc_mesh_set_btag: {ERR.get(rc, rc)}")

    def state(self) -> dict:
        return {"x": self.get(F_X), "vp": self.get(F_VP), "v": self.get(F_V), "e": self.get(F_E),
                "F": self.get(F_F), "tau": self.get(F_TAU)}


# ----------------------------------------------------------------------------- tangent build
_tlib = None


def tangent_lib():
    global _tlib
    if _tlib is None:
        build()
        _tlib = C.CDLL(_TLIB)
        vp = C.c_void_p
        _tlib.orct_run.argtypes = [C.c_int, C.c_long, vp, vp, C.c_double, C.c_long, vp, C.c_long, vp, vp, vp, C.c_int, vp,
                                   C.c_double, C.c_double, C.c_double, vp, vp, vp, vp, vp, vp, C.POINTER(Params),
                                   C.c_long] + [vp] * 12
        _tlib.orct_run.restype = C.c_int
    return _tlib


def tangent(problem, n_steps: int, dv=None, dmu=None, dF=None, dx=None, x_shift: float = 0.0,
            params: Params | None = None, **kw) -> dict:
    """The oracle's n-step map and its directional derivative (forward mode, dual numbers):
    the final state x, vp [d][np], v [d][nc], F [d*d][nc], e [nc] and their derivatives dx,
    dvp, dv, dF, de along the direction (dv [d][nc], dmu [nc], dF [d*d][nc], dx [d][np] of the positions at
    fixed cell masses; None = 0) of the initial data, with each step's order mask and dt held
    at the run's own (masks [n][nc] int8, dts [n]). The problem's boundary values and contact
    walls apply as constants. x_shift: start from the positions x + x_shift dx (masses and slip
    directions of x), for central differences along dx."""
    m = problem.mesh
    d, nc, npn = m.dim, m.n_cells, m.n_nodes
    sgkw = {}
    sg = getattr(problem, "stiffened_gas", None)
    if sg is not None:
        sgkw = {"eos": 1, "gamma": sg[0], "p_inf": sg[1], "p0": sg[2]}
    prm = params or default_params(problem.cfl, **{"shear_a": getattr(problem, "shear_a", -1.0), **sgkw, **kw})
    keep = []

    def arr(a, dtype=np.float64):
        if a is None:
            return None
        a = np.ascontiguousarray(a, dtype=dtype)
        keep.append(a)
        return a.ctypes.data

    out = {k: np.zeros(shape) for k, shape in (("x", (d, npn)), ("dx", (d, npn)), ("vp", (d, npn)),
                                                ("dvp", (d, npn)), ("v", (d, nc)), ("dv", (d, nc)),
                                                ("F", (d * d, nc)), ("dF", (d * d, nc)), ("e", (nc,)),
                                                ("de", (nc,)))}
    out["masks"] = np.zeros((n_steps, nc), np.int8)
    out["dts"] = np.zeros(n_steps)
    nb = m.btag.size
    bcval = getattr(problem, "bcval", None)
    contact = getattr(problem, "contact", None)
    planes, ceps = (np.asarray(contact[0], dtype=np.float64), float(contact[1])) if contact is not None else (None, 0.0)
    rc = tangent_lib().orct_run(d, npn, arr(m.x), arr(dx), x_shift, nc, arr(m.c2n, np.int32), nb,
                                arr(m.bface, np.int32) if nb else None, arr(m.btag, np.int32) if nb else None,
                                arr(bcval) if (bcval is not None and nb) else None,
                                0 if planes is None else len(planes), arr(planes), ceps,
                                problem.rho0, problem.lam, arr(problem.mu), arr(dmu), arr(problem.v), arr(dv),
                                arr(problem.F), arr(dF), C.byref(prm), n_steps,
                                *(out[k].ctypes.data for k in ("x", "dx", "vp", "dvp", "v", "dv", "F", "dF", "e", "de")),
                                out["masks"].ctypes.data, out["dts"].ctypes.data)
    if rc:
        raise OracleError(f"orct_run: {ERR.get(rc, rc)}")
    return out
