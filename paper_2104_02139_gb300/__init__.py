"""Thin Python binding of the GB300 Lagrangian ADER-MOOD library (C ABI in include/lmood.h).

Argument marshalling only: every step of the scheme runs in the CUDA kernels of
liblmood.so. Host arrays are numpy; device buffers may be torch CUDA tensors (their data
pointers are passed through), and the CUDA stream defaults to torch's current stream when
torch has a device. There is no CPU fallback: without the compiled library every call raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import LIB, build  # noqa: F401  (build() compiles the library in-tree)

OK, ERR_ARG, ERR_MESH, ERR_CUDA, ERR_OOM, ERR_PARACHUTE, ERR_MOOD_ITERS, ERR_TIMEOUT, ERR_STATE = range(9)
FIELD_X, FIELD_VP, FIELD_VSTAR, FIELD_V, FIELD_E, FIELD_F, FIELD_TAU, FIELD_ORDER, FIELD_MASS, \
    FIELD_PKM, FIELD_PKR, FIELD_DT = range(12)


class LmoodError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"[{status}] {msg}")
        self.status = status


class Material(C.Structure):
    _fields_ = [("rho0", C.c_double), ("lambda_", C.c_double), ("vol_coeff", C.c_int32), ("eos", C.c_int32),
                ("shear_a", C.c_double), ("gamma", C.c_double), ("p_inf", C.c_double), ("p0", C.c_double)]


class Params(C.Structure):
    _fields_ = [("cfl", C.c_double), ("Cv", C.c_double), ("Ci", C.c_double), ("delta0", C.c_double),
                ("delta1", C.c_double), ("dt_fixed", C.c_double), ("max_mood_iters", C.c_int32),
                ("order", C.c_int32), ("mood", C.c_int32), ("graph", C.c_int32), ("cascade", C.c_int32),
                ("barrier_polls", C.c_int32)]


class StepInfo(C.Structure):
    _fields_ = [("t", C.c_double), ("dt_used", C.c_double), ("dt_next", C.c_double), ("step", C.c_int64),
                ("n_troubled", C.c_int32), ("n_p0", C.c_int32), ("mood_iters", C.c_int32),
                ("n_parachute", C.c_int32), ("n_p0_eps", C.c_int32), ("n_lim", C.c_int32),
                ("syncs", C.c_int32)]


_lib = None
EXPORTS = ("lmood_params_default", "lmood_mesh_create", "lmood_mesh_destroy", "lmood_mesh_info",
           "lmood_mesh_set_bc_values", "lmood_mesh_set_btag", "lmood_mesh_set_contact",
           "lmood_state_init", "lmood_state_init_device", "lmood_state_destroy", "lmood_step", "lmood_run", "lmood_get", "lmood_set",
           "lmood_get_fields", "lmood_set_fields",
           "lmood_totals", "lmood_timing", "lmood_timing_read", "lmood_autotune", "lmood_autotune_schedule",
           "lmood_totals_noalloc",
           "lmood_tape_record",
           "lmood_tape_backward", "lmood_tape_backward_e", "lmood_tape_replay", "lmood_tape_info", "lmood_tape_destroy", "lmood_last_error")
K_PREDICT, K_NODES, K_UPDATE, K_MOOD, K_FINALIZE, K_MOMENTS, NK = range(7)
K_NAMES = ("predict", "nodes", "update", "mood", "finalize", "moments")


def lib():
    """Load liblmood.so (raises if it has not been built; see build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError(f"CUDA library {LIB} is missing: run paper_2104_02139_gb300.build()")
        L = C.CDLL(LIB)
        vp = C.c_void_p
        L.lmood_params_default.argtypes = [C.c_int, C.POINTER(Params)]
        L.lmood_mesh_create.argtypes = [C.c_int, C.c_int64, vp, C.c_int64, vp, C.c_int64, vp, vp, vp, C.c_int32,
                                        vp, C.POINTER(vp)]
        L.lmood_mesh_destroy.argtypes = [vp]
        L.lmood_mesh_info.argtypes = [vp, C.POINTER(C.c_int64)]
        L.lmood_mesh_set_bc_values.argtypes = [vp, vp, C.c_int]
        L.lmood_mesh_set_btag.argtypes = [vp, vp]
        L.lmood_mesh_set_contact.argtypes = [vp, C.c_int, vp, C.c_double]
        L.lmood_state_init.argtypes = [vp, C.POINTER(Material), vp, vp, vp, C.POINTER(Params), C.POINTER(vp)]
        L.lmood_state_init_device.argtypes = [vp, C.POINTER(Material), vp, vp, vp, C.POINTER(Params),
                                              C.POINTER(vp)]
        L.lmood_state_destroy.argtypes = [vp]
        L.lmood_step.argtypes = [vp, C.POINTER(StepInfo)]
        L.lmood_run.argtypes = [vp, C.c_int64, C.POINTER(StepInfo)]
        L.lmood_get.argtypes = [vp, C.c_int, vp, C.c_int]
        L.lmood_set.argtypes = [vp, C.c_int, vp, C.c_int]
        L.lmood_get_fields.argtypes = [vp, C.c_int, C.POINTER(C.c_int), C.POINTER(vp), C.c_int]
        L.lmood_set_fields.argtypes = [vp, C.c_int, C.POINTER(C.c_int), C.POINTER(vp), C.c_int]
        L.lmood_totals.argtypes = [vp, C.POINTER(C.c_double)]
        L.lmood_timing.argtypes = [vp, C.c_int]
        L.lmood_timing_read.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_int64)]
        L.lmood_totals_noalloc.argtypes = [C.c_int, C.c_int64, vp, vp, vp, vp, vp]
        L.lmood_autotune.argtypes = [vp, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_int32)]
        L.lmood_autotune_schedule.argtypes = [vp, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_int32),
                                              C.POINTER(C.c_double), C.POINTER(C.c_int32)]
        L.lmood_tape_record.argtypes = [vp, C.c_int64, C.c_int64, C.POINTER(vp), C.POINTER(StepInfo)]
        L.lmood_tape_backward.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, C.c_int]
        L.lmood_tape_backward_e.argtypes = [vp] + [vp] * 11 + [C.c_int]
        L.lmood_tape_replay.argtypes = [vp, vp, C.c_int64]
        L.lmood_tape_info.argtypes = [vp, C.POINTER(C.c_int64)]
        L.lmood_tape_destroy.argtypes = [vp]
        L.lmood_last_error.restype = C.c_char_p
        for name in EXPORTS:
            if name != "lmood_last_error":
                getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def _check(rc: int):
    if rc != OK:
        raise LmoodError(rc, lib().lmood_last_error().decode(errors="replace"))


def _host(a, dtype):
    return None if a is None else np.ascontiguousarray(a, dtype=dtype)


def _ptr(a):
    return None if a is None else a.ctypes.data


def _is_torch(a) -> bool:
    return hasattr(a, "data_ptr") and hasattr(a, "is_cuda")


def _numel(shape) -> int:
    """element count of a field's shape; None (an id the library rejects without copying): any"""
    return -1 if shape is None else int(np.prod(shape, dtype=np.int64))


def _out_buffer(a, shape, what: str):
    """Check a destination the library writes prod(shape) doubles into: a writeable
    C-contiguous float64 numpy array (host) or a contiguous float64 CUDA tensor (device) of
    exactly that many elements. Returns (pointer, is_device). Anything else raises before the
    library is called, so no copy can run past the end of the buffer."""
    n = _numel(shape)
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags.c_contiguous or not a.flags.writeable:
            raise ValueError(f"{what}: host destination must be a writeable C-contiguous float64 array "
                             f"(got {a.dtype}, contiguous={a.flags.c_contiguous})")
        if n >= 0 and a.size != n:
            raise ValueError(f"{what}: destination has {a.size} elements, the field needs {n} {tuple(shape)}")
        return a.ctypes.data, 0
    if _is_torch(a):
        import torch
        if a.dtype != torch.float64 or not a.is_cuda or not a.is_contiguous():
            raise ValueError(f"{what}: device destination must be a contiguous float64 CUDA tensor "
                             f"(got {a.dtype}, cuda={a.is_cuda}, contiguous={a.is_contiguous()})")
        if n >= 0 and a.numel() != n:
            raise ValueError(f"{what}: destination has {a.numel()} elements, the field needs {n} {tuple(shape)}")
        return a.data_ptr(), 1
    raise TypeError(f"{what}: destination must be a numpy array or a torch CUDA tensor, not {type(a).__name__}")


def _in_buffer(a, shape, what: str):
    """A source the library reads prod(shape) doubles from. Host data (anything numpy accepts)
    is converted to a C-contiguous float64 copy when needed; a torch tensor must be a CUDA
    tensor and is made contiguous float64 when needed. Returns (keep, pointer, is_device,
    copied): keep must stay alive until the library has read it -- for a device copy that is
    until the mesh's stream has passed the call (the caller synchronises when copied)."""
    n = _numel(shape)
    if _is_torch(a):
        import torch
        if not a.is_cuda:
            raise ValueError(f"{what}: a torch source must be a CUDA tensor (host data: pass numpy)")
        t = a if (a.dtype == torch.float64 and a.is_contiguous()) else a.to(torch.float64).contiguous()
        if n >= 0 and t.numel() != n:
            raise ValueError(f"{what}: source has {t.numel()} elements, the field needs {n} {tuple(shape)}")
        return t, t.data_ptr(), 1, t is not a
    h = np.ascontiguousarray(a, dtype=np.float64)
    if n >= 0 and h.size != n:
        raise ValueError(f"{what}: source has {h.size} elements, the field needs {n} {tuple(shape)}")
    return h, h.ctypes.data, 0, False


def _sync_after_copy():
    """A temporary device copy was handed to the library: wait until every stream (the mesh's
    included) has finished with it before it can be freed and reused by torch's allocator."""
    import torch
    torch.cuda.synchronize()


def current_stream_handle():
    """torch's current CUDA stream as a raw handle (None for the legacy default stream)."""
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream or None
    except Exception:
        pass
    return None


def params_default(dim: int, **kw) -> Params:
    """lmood_params_default, then the given fields (unknown names raise TypeError)"""
    p = Params()
    _check(lib().lmood_params_default(dim, C.byref(p)))
    known = {name for name, _ in Params._fields_}
    for k, v in kw.items():
        if k not in known:
            raise TypeError(f"unknown step parameter {k!r} (lmood_params has {sorted(known)})")
        setattr(p, k, v)
    return p


class Mesh:
    """lmood_mesh_create / lmood_mesh_destroy."""

    def __init__(self, dim, x, c2n, bface=None, btag=None, cell_inst=None, n_inst=1, stream=None):
        x = _host(x, np.float64)
        c2n = _host(c2n, np.int32)
        bface = _host(bface, np.int32)
        btag = _host(btag, np.int32)
        ci = _host(cell_inst, np.int32)
        nb = 0 if btag is None else btag.size
        self.dim, self.n_nodes, self.n_cells, self.n_bfaces = dim, x.shape[-1], c2n.shape[-1], nb
        self.n_inst = n_inst if ci is not None else 1
        self.stream = current_stream_handle() if stream is None else stream
        h = C.c_void_p()
        _check(lib().lmood_mesh_create(dim, self.n_nodes, _ptr(x), self.n_cells, _ptr(c2n), nb,
                                       _ptr(bface) if nb else None, _ptr(btag) if nb else None, _ptr(ci),
                                       self.n_inst, self.stream, C.byref(h)))
        self.h = h

    def set_bc_values(self, values):
        """boundary-face values [dim, n_bfaces]: traction vectors (tag 3), pressures in row 0
        (tag 4), prescribed velocities (tag 5); numpy (host) or a torch CUDA tensor"""
        keep, ptr, dev, copied = _in_buffer(values, (self.dim, self.n_bfaces), "set_bc_values")
        _check(lib().lmood_mesh_set_bc_values(self.h, C.c_void_p(ptr), dev))
        if copied:
            _sync_after_copy()
        del keep

    def set_contact(self, planes, eps: float):
        """contact walls [n][2 dim] (a point, the unit normal into the body) and threshold eps
        for the faces tagged 6"""
        a = np.ascontiguousarray(planes, dtype=np.float64)
        _check(lib().lmood_mesh_set_contact(self.h, len(a), a.ctypes.data if len(a) else None, eps))

    def set_btag(self, btag):
        """new boundary-face tags [n_bfaces] (0-6); per-node conditions re-derived"""
        a = np.ascontiguousarray(btag, dtype=np.int32)
        _check(lib().lmood_mesh_set_btag(self.h, a.ctypes.data))

    def info(self) -> dict:
        o = (C.c_int64 * 6)()
        _check(lib().lmood_mesh_info(self.h, o))
        return dict(zip(("n_nodes", "n_cells", "dim", "stencil_nnz", "max_corners", "n_inst"), list(o)))

    def close(self):
        if getattr(self, "h", None):
            lib().lmood_mesh_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()


class State:
    """lmood_state_init / step / run / get / set / totals / destroy."""

    def __init__(self, mesh: Mesh, rho0, lam, mu, v, F=None, params: Params | None = None, vol_coeff=0,
                 shear_a=-1.0, stiffened_gas=None):
        """stiffened_gas: None, or (gamma, p_inf, p0) for the stiffened-gas volumetric law.
        mu, v, F: host arrays, or torch CUDA tensors (all of them; lmood_state_init_device, the
        data never leaves the device)"""
        self.mesh = mesh
        self.params = params or params_default(mesh.dim)
        mat = Material(rho0=rho0, lambda_=lam, vol_coeff=vol_coeff, shear_a=shear_a)
        if stiffened_gas is not None:
            mat.eos = 1
            mat.gamma, mat.p_inf, mat.p0 = stiffened_gas
        h = C.c_void_p()
        nc, d = mesh.n_cells, mesh.dim
        if _is_torch(mu) or _is_torch(v) or _is_torch(F):
            if not (_is_torch(mu) and _is_torch(v) and (F is None or _is_torch(F))):
                raise TypeError("State: mu, v and F must be all host arrays or all CUDA tensors")
            import torch
            kept = [_in_buffer(a, shp, f"State ({k})") for a, shp, k in
                    ((mu, (nc,), "mu"), (v, (d, nc), "v"), (F, (d * d, nc), "F")) if a is not None]
            torch.cuda.current_stream().synchronize()  # the inputs are ready before the mesh's stream reads them
            ptrs = [C.c_void_p(k[1]) for k in kept] + ([None] if F is None else [])
            _check(lib().lmood_state_init_device(mesh.h, C.byref(mat), *ptrs, C.byref(self.params), C.byref(h)))
            if any(k[3] for k in kept):
                _sync_after_copy()
            del kept
        else:
            mu = _host(mu, np.float64)
            v = _host(v, np.float64)
            F = _host(F, np.float64)
            _check(lib().lmood_state_init(mesh.h, C.byref(mat), _ptr(mu), _ptr(v), _ptr(F), C.byref(self.params),
                                          C.byref(h)))
        self.h = h
        self.info = StepInfo()

    def close(self):
        if getattr(self, "h", None):
            lib().lmood_state_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def step(self) -> StepInfo:
        _check(lib().lmood_step(self.h, C.byref(self.info)))
        return self.info

    def step_status(self) -> int:
        """lmood_step without raising: returns the status code."""
        return lib().lmood_step(self.h, C.byref(self.info))

    def run(self, n: int) -> StepInfo:
        _check(lib().lmood_run(self.h, n, C.byref(self.info)))
        return self.info

    def shape(self, field: int) -> tuple:
        d, nc, npn, nv = self.mesh.dim, self.mesh.n_cells, self.mesh.n_nodes, self.mesh.dim + 1
        if not 0 <= field <= FIELD_DT:
            return None  # the library rejects the id and copies nothing
        return {FIELD_X: (d, npn), FIELD_VP: (d, npn), FIELD_VSTAR: (d, npn), FIELD_V: (d, nc), FIELD_E: (nc,),
                FIELD_F: (d * d, nc), FIELD_TAU: (nc,), FIELD_ORDER: (nc,), FIELD_MASS: (nc,),
                FIELD_PKM: (d * (d + 1) // 2, nv, nc), FIELD_PKR: (d, nv, nc), FIELD_DT: (self.mesh.n_inst,)}[field]

    def get(self, field: int, out=None):
        """Host copy as numpy (out None or a numpy array), or into a torch CUDA tensor; out
        must be float64, contiguous and of the field's size (checked before the copy)."""
        if out is None:
            out = np.empty(self.shape(field) or (1,))
        ptr, dev = _out_buffer(out, self.shape(field), "get")
        _check(lib().lmood_get(self.h, field, C.c_void_p(ptr), dev))
        return out

    def set(self, field: int, src):
        """Replace a field from host data (numpy-convertible) or a torch CUDA tensor of the
        field's size."""
        keep, ptr, dev, copied = _in_buffer(src, self.shape(field), "set")
        _check(lib().lmood_set(self.h, field, C.c_void_p(ptr), dev))
        if copied:
            _sync_after_copy()
        del keep

    def get_fields(self, outs: dict) -> dict:
        """lmood_get_fields: {field id: destination} all numpy (one synchronisation at the end)
        or all torch CUDA tensors"""
        ids = list(outs)
        checked = [_out_buffer(outs[f], self.shape(f), f"get_fields (field {f})") for f in ids]
        if len({dev for _, dev in checked}) > 1:
            raise ValueError("get_fields: destinations must be all host or all device")
        _check(lib().lmood_get_fields(self.h, len(ids), (C.c_int * len(ids))(*ids),
                                      (C.c_void_p * len(ids))(*[p for p, _ in checked]), checked[0][1]))
        return outs

    def set_fields(self, srcs: dict):
        """lmood_set_fields: {field id: source}, all host arrays or all torch CUDA tensors"""
        ids = list(srcs)
        checked = [_in_buffer(srcs[f], self.shape(f), f"set_fields (field {f})") for f in ids]
        if len({c[2] for c in checked}) > 1:
            raise ValueError("set_fields: sources must be all host or all device")
        _check(lib().lmood_set_fields(self.h, len(ids), (C.c_int * len(ids))(*ids),
                                      (C.c_void_p * len(ids))(*[c[1] for c in checked]), checked[0][2]))
        if any(c[3] for c in checked):
            _sync_after_copy()
        del checked

    def totals(self) -> np.ndarray:
        o = (C.c_double * 5)()
        _check(lib().lmood_totals(self.h, o))
        return np.array(list(o))

    def autotune(self, reps: int = 5) -> dict:
        """lmood_autotune: per kernel class the candidate block sizes' mean times (ms) and the
        chosen size"""
        ms = (C.c_double * 12)()
        ch = (C.c_int32 * 4)()
        _check(lib().lmood_autotune(self.h, reps, ms, ch))
        cand = ((128, 256, 512), (64, 128, 256), (128, 256, 512), (64, 128, 256))
        out = {}
        for k, name in enumerate(("moments", "predict", "nodes", "update")):
            out[name] = {"chosen": ch[k], "ms": {cand[k][v]: ms[k * 3 + v] for v in range(3)}}
        return out

    def autotune_schedule(self, reps: int = 5) -> dict:
        """lmood_autotune_schedule: node-window size of the whole-mesh node kernels (32, 256,
        2048, 0 = own order) and the step form (graph 1 or 2), each timed and the fastest kept"""
        msw = (C.c_double * 4)()
        w = C.c_int32()
        msf = (C.c_double * 2)()
        fm = C.c_int32()
        _check(lib().lmood_autotune_schedule(self.h, reps, msw, C.byref(w), msf, C.byref(fm)))
        if fm.value > 0:
            self.params.graph = fm.value
        return {"node_window": {"chosen": w.value, "ms": dict(zip((32, 256, 2048, 0), list(msw)))},
                "step_form": {"chosen": fm.value, "ms": {1: msf[0], 2: msf[1]}}}

    def timing(self, enable: bool):
        _check(lib().lmood_timing(self.h, 1 if enable else 0))

    def timing_read(self) -> dict:
        ms = (C.c_double * NK)()
        n = (C.c_int64 * NK)()
        _check(lib().lmood_timing_read(self.h, ms, n))
        return {K_NAMES[i]: (ms[i], n[i]) for i in range(NK)}

    def state(self) -> dict:
        return {"x": self.get(FIELD_X), "vp": self.get(FIELD_VP), "v": self.get(FIELD_V), "e": self.get(FIELD_E),
                "F": self.get(FIELD_F), "tau": self.get(FIELD_TAU)}


class Tape:
    """lmood_tape_record / backward / info / destroy: reverse-mode gradients of n steps of a
    state with each step's MOOD order mask and dt frozen at their recorded values."""

    def __init__(self, state: State, n_steps: int, checkpoint_every: int = 0):
        """checkpoint_every = 0 keeps every state and step product (no replay in backward);
        C >= 1 keeps a checkpoint every C steps and replays."""
        self.state = state
        h = C.c_void_p()
        _check(lib().lmood_tape_record(state.h, n_steps, checkpoint_every, C.byref(h), C.byref(state.info)))
        self.h = h

    def info(self) -> dict:
        o = (C.c_int64 * 4)()
        _check(lib().lmood_tape_info(self.h, o))
        return dict(zip(("steps", "checkpoint_every", "through_init", "bytes"), list(o)))

    def backward(self, lam_x=None, lam_vp=None, lam_v=None, lam_F=None, lam_e=None, out=None) -> dict:
        """Adjoints of the final state in (numpy host arrays, or torch CUDA tensors; None = 0);
        gradients with respect to the start of the tape out, as a dict x, vp, v, F, e, mu of the
        same kind (numpy unless the inputs are torch tensors, or given in out)."""
        st = self.state
        shapes = {"x": st.shape(FIELD_X), "vp": st.shape(FIELD_VP), "v": st.shape(FIELD_V), "F": st.shape(FIELD_F),
                  "e": (st.mesh.n_cells,), "mu": (st.mesh.n_cells,)}
        ins = (lam_x, lam_vp, lam_v, lam_F, lam_e)
        dev = any(a is not None and hasattr(a, "data_ptr") for a in ins)
        if out is None:
            if dev:
                import torch
                out = {k: torch.empty(v, dtype=torch.float64, device="cuda") for k, v in shapes.items()}
            else:
                out = {k: np.empty(v) for k, v in shapes.items()}

        kept, args = [], []
        for a, k in zip(ins, ("x", "vp", "v", "F", "e")):
            if a is None:
                args.append(None)
                continue
            if dev != _is_torch(a):
                raise TypeError("backward: adjoint inputs must be all host arrays or all CUDA tensors")
            kept.append(_in_buffer(a, shapes[k], f"backward (lam_{k})"))
            args.append(C.c_void_p(kept[-1][1]))
        optr = []
        for k in ("x", "vp", "v", "F", "e", "mu"):
            o = out.get(k)
            if o is None:
                optr.append(None)
                continue
            ptr, odev = _out_buffer(o, shapes[k], f"backward (grad_{k})")
            if odev != int(dev):
                raise ValueError("backward: gradients must live where the adjoint inputs do (host or device)")
            optr.append(C.c_void_p(ptr))
        _check(lib().lmood_tape_backward_e(self.h, *args, *optr, 1 if dev else 0))
        if any(c[3] for c in kept):
            _sync_after_copy()
        del kept
        return out

    def replay(self, state: State, n_steps: int | None = None) -> State:
        """Advance another state (same mesh sizes) by the recorded steps with the recorded
        orders and dt: the frozen-mask map that backward() differentiates."""
        n = self.info()["steps"] if n_steps is None else n_steps
        _check(lib().lmood_tape_replay(self.h, state.h, n))
        return state

    def close(self):
        if getattr(self, "h", None):
            lib().lmood_tape_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()


def rollout(problem, n_steps: int, v0, mu, F0=None, checkpoint_every: int = 0, **params):
    """Differentiable rollout (torch.autograd.Function): the state after n_steps steps of the
    scheme on problem's mesh and material, started from the per-cell initial velocity v0
    [dim, n_cells], shear modulus mu [n_cells] and deformation gradient F0 [dim*dim, n_cells]
    (None: identity), given as float64 torch CUDA tensors. Returns (x, vp, v, F) at t^N as
    torch CUDA tensors; gradients flow back to v0, mu and F0 through the recorded steps (MOOD
    orders and dt frozen). The forward and the reverse pass run in the library's kernels."""
    import torch

    class _Rollout(torch.autograd.Function):
        @staticmethod
        def forward(ctx, v0_, mu_, F0_):
            pb = problem
            m = pb.mesh
            mesh = Mesh(m.dim, m.x, m.c2n, m.bface, m.btag)
            if getattr(pb, "bcval", None) is not None:
                mesh.set_bc_values(pb.bcval)
            if getattr(pb, "contact", None) is not None:
                mesh.set_contact(*pb.contact)
            p = params_default(m.dim, cfl=pb.cfl)
            for k, v in params.items():
                setattr(p, k, v)
            # the initial data stay on the device (lmood_state_init_device)
            state = State(mesh, pb.rho0, pb.lam, mu_.detach(), v0_.detach(), None if F0_ is None else F0_.detach(),
                          p, shear_a=getattr(pb, "shear_a", -1.0))
            tape = Tape(state, n_steps, checkpoint_every)
            outs = []
            for fid in (FIELD_X, FIELD_VP, FIELD_V, FIELD_F):
                t = torch.empty(state.shape(fid), dtype=torch.float64, device="cuda")
                state.get(fid, t)
                outs.append(t)
            torch.cuda.current_stream().synchronize()
            ctx.tape, ctx.state, ctx.mesh, ctx.has_F = tape, state, mesh, F0_ is not None
            return tuple(outs)

        @staticmethod
        def backward(ctx, gx, gvp, gv, gF):
            def dense(g):
                return None if g is None else g.contiguous().to(torch.float64)

            out = ctx.tape.backward(*(dense(g) if g is not None else None for g in (gx, gvp, gv, gF)))
            if isinstance(out["v"], np.ndarray):  # all output gradients were None
                out = {k: torch.as_tensor(v, device="cuda") for k, v in out.items()}
            torch.cuda.current_stream().synchronize()
            return out["v"], out["mu"], (out["F"] if ctx.has_F else None)

    return _Rollout.apply(v0, mu, F0)


def simulation(problem, stream=None, cell_inst=None, n_inst=1, **params) -> State:
    """Mesh + state of a workload problem (anything with .mesh, .rho0, .lam, .mu, .v, .F, .cfl);
    cell_inst / n_inst describe a batch of independent instances concatenated into one mesh."""
    m = problem.mesh
    mesh = Mesh(m.dim, m.x, m.c2n, m.bface, m.btag, cell_inst=cell_inst, n_inst=n_inst, stream=stream)
    if getattr(problem, "bcval", None) is not None:
        mesh.set_bc_values(problem.bcval)
    if getattr(problem, "contact", None) is not None:
        mesh.set_contact(*problem.contact)
    p = params_default(m.dim, **{"cfl": problem.cfl, **params})
    return State(mesh, problem.rho0, problem.lam, problem.mu, problem.v, problem.F, p,
                 shear_a=getattr(problem, "shear_a", -1.0), stiffened_gas=getattr(problem, "stiffened_gas", None))
