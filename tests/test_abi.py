"""The C ABI library loads without a GPU and exports every entry point include/lmood.h declares."""
import os
import re

import paper_2104_02139_gb300 as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "lmood.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return set(re.findall(r"\b(lmood_[a-z_]+)\s*\(", src))


def test_header_and_exports_agree():
    L.build()
    lib = L.lib()
    declared = _declared()
    assert declared == set(L.EXPORTS)
    for name in declared:
        assert hasattr(lib, name), name


def test_params_default_without_gpu():
    p = L.params_default(3)
    assert p.cfl == 0.25 and p.Cv == 0.2 and p.Ci == 0.1 and p.delta0 == 1e-4 and p.delta1 == 1e-3
    assert p.order == 2 and p.mood == 1 and p.max_mood_iters == 100000
    try:
        L.params_default(4)
    except L.LmoodError as e:
        assert e.status == L.ERR_ARG
    else:
        raise AssertionError("dim 4 accepted")


def test_mesh_size_limits_checked_before_any_device_work():
    """The kernels index with 32-bit integers: meshes whose corner matrices, F or node moments
    would overflow them are refused with LMOOD_ERR_ARG (the sizes are checked before the arrays
    are read or any device call is made; the limits are 3D 89,478,485 cells / 37,025,580 nodes,
    2D 238,609,294 cells / 89,478,485 nodes)."""
    import ctypes as C
    lib = L.lib()
    x = (C.c_double * 12)()
    c2n = (C.c_int32 * 4)(0, 1, 2, 3)
    out = C.c_void_p()
    for dim, nodes, cells in ((3, 4, 89_478_486), (3, 37_025_581, 1), (2, 3, 238_609_295), (2, 89_478_486, 1)):
        rc = lib.lmood_mesh_create(dim, nodes, x, cells, c2n, 0, None, None, None, 1, None, C.byref(out))
        assert rc == L.ERR_ARG, (dim, nodes, cells)
        assert "too large" in lib.lmood_last_error().decode()


def test_unknown_step_parameter_is_an_error():
    import pytest
    with pytest.raises(TypeError):
        L.params_default(2, grpah=2)
    assert L.params_default(2, graph=2, barrier_polls=7).barrier_polls == 7


def _fake_state(dim=2, n_cells=3, n_nodes=4, n_inst=1):
    """A State whose handle is never used: every buffer check runs before the library call."""
    from types import SimpleNamespace
    s = L.State.__new__(L.State)
    s.mesh = SimpleNamespace(dim=dim, n_cells=n_cells, n_nodes=n_nodes, n_inst=n_inst)
    s.h = None
    return s


def test_field_copies_check_their_destinations_on_the_host():
    """get_fields refuses mixed or non-float64 destinations before any library call."""
    import numpy as np
    import pytest
    s = _fake_state(n_cells=3, n_nodes=3)
    with pytest.raises(ValueError):
        s.get_fields({L.FIELD_X: np.zeros((2, 3)), L.FIELD_V: np.zeros((2, 3), dtype=np.float32)})
    with pytest.raises(ValueError):
        s.get_fields({L.FIELD_X: np.zeros((3, 2)).T})  # not C-contiguous


def test_buffers_are_checked_before_the_library_copies():
    """Every get / set / get_fields / set_fields / set_bc_values / backward buffer is checked for
    dtype, host-or-device kind, contiguity and element count before the library is called: a
    float32 or short buffer would otherwise be read or written past its end."""
    import numpy as np
    import pytest
    torch = pytest.importorskip("torch")
    s = _fake_state(dim=2, n_cells=5, n_nodes=4)
    bad_out = [np.zeros((2, 5), dtype=np.float32),          # wrong dtype
               np.zeros((2, 4)),                            # too short for V [2][5]
               np.zeros((2, 6)),                            # too long
               np.zeros((5, 2)).T,                          # not C-contiguous
               torch.zeros((2, 5), dtype=torch.float64),    # a host torch tensor is not a device buffer
               [0.0] * 10]                                  # not a buffer at all
    for o in bad_out:
        with pytest.raises((ValueError, TypeError)):
            s.get(L.FIELD_V, out=o)
        with pytest.raises((ValueError, TypeError)):
            s.get_fields({L.FIELD_V: o})
    for src in (np.zeros(9), np.zeros((2, 4)), torch.zeros(10, dtype=torch.float64)):
        with pytest.raises(ValueError):
            s.set(L.FIELD_V, src)
        with pytest.raises(ValueError):
            s.set_fields({L.FIELD_V: src})
    with pytest.raises(ValueError):
        s.set(L.FIELD_E, np.zeros(4))                       # E is [n_cells]
    with pytest.raises(ValueError):
        s.set(L.FIELD_DT, np.zeros(2))                      # DT is [n_instances]
    with pytest.raises(ValueError):                         # host and device mixed in one call
        s.get_fields({L.FIELD_E: np.zeros(5), L.FIELD_TAU: np.zeros(5, dtype=np.float32)})
    m = L.Mesh.__new__(L.Mesh)
    m.dim, m.n_bfaces, m.h = 2, 3, None
    for v in (np.zeros(5), np.zeros((3, 2)).T[:, :2], torch.zeros(6, dtype=torch.float64)):
        with pytest.raises(ValueError):
            m.set_bc_values(v)
    tape = L.Tape.__new__(L.Tape)
    tape.state, tape.h = s, None
    with pytest.raises(ValueError):
        tape.backward(lam_v=np.zeros((2, 4)))
    with pytest.raises(ValueError):
        tape.backward(lam_v=np.zeros((2, 5)), out={"v": np.zeros((2, 5), dtype=np.float32)})
    with pytest.raises(ValueError):
        tape.backward(lam_v=np.zeros((2, 5)), out={"mu": np.zeros(4)})
