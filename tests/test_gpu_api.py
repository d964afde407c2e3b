"""Error paths of the C ABI on a device: each returns a status, none faults the GPU (-m gpu)."""
import numpy as np
import pytest

import paper_2104_02139_gb300 as L
import workloads as W

pytestmark = pytest.mark.gpu


def _status(fn):
    try:
        fn()
    except L.LmoodError as e:
        return e.status
    return L.OK


def test_mesh_errors():
    m = W.tri_mesh(6, 1, bc={"x0": W.SLIP})
    bad = m.c2n.copy()
    bad[[1, 2]] = bad[[2, 1]]  # clockwise triangles
    assert _status(lambda: L.Mesh(2, m.x, bad)) == L.ERR_MESH
    oob = m.c2n.copy()
    oob[0, 3] = m.n_nodes
    assert _status(lambda: L.Mesh(2, m.x, oob)) == L.ERR_MESH
    assert _status(lambda: L.Mesh(4, m.x, m.c2n)) == L.ERR_ARG
    btag = np.full(m.btag.size, 7, np.int32)
    assert _status(lambda: L.Mesh(2, m.x, m.c2n, m.bface, btag)) == L.ERR_ARG


def test_state_and_field_errors():
    pb = W.plain2d(n=8)
    s = L.simulation(pb)
    assert _status(lambda: s.get(99)) == L.ERR_ARG
    assert _status(lambda: s.set(L.FIELD_TAU, np.zeros(pb.mesh.n_cells))) == L.ERR_ARG
    mesh = L.Mesh(2, pb.mesh.x, pb.mesh.c2n)
    assert _status(lambda: L.State(mesh, 1.0, 2.0, -np.ones(pb.mesh.n_cells), pb.v)) == L.ERR_ARG
    assert _status(lambda: L.State(mesh, 0.0, 2.0, pb.mu, pb.v)) == L.ERR_ARG


def test_parachute_leaves_state_unchanged():
    """A dt far above the CFL bound inverts cells even with the first-order scheme: the step
    reports the parachute failure and the state is the one before the call."""
    pb = W.impact2d(n=12)
    s = L.simulation(pb, dt_fixed=50.0, order=1)
    before = s.state()
    assert s.step_status() == L.ERR_PARACHUTE
    after = s.state()
    for k in before:
        assert np.array_equal(before[k], after[k]), k
    assert s.step_status() == L.ERR_PARACHUTE  # and it stays usable


def test_set_and_replay():
    """Setting a state from host buffers and stepping equals stepping the original."""
    pb = W.impact2d(n=30)
    a = L.simulation(pb)
    a.run(3)
    snap = a.state()
    dt = a.get(L.FIELD_DT)
    b = L.simulation(pb)
    for f, k in ((L.FIELD_X, "x"), (L.FIELD_VP, "vp"), (L.FIELD_V, "v"), (L.FIELD_E, "e"), (L.FIELD_F, "F")):
        b.set(f, snap[k])
    b.set(L.FIELD_DT, dt)
    a.step()
    b.step()
    for k, v in a.state().items():
        assert np.array_equal(v, b.state()[k]), k


def test_empty_and_null_inputs():
    m = W.tri_mesh(5, 1)
    assert _status(lambda: L.Mesh(2, np.zeros((2, 0)), np.zeros((3, 0), np.int32))) == L.ERR_ARG
    assert _status(lambda: L.Mesh(2, m.x, np.zeros((3, 0), np.int32))) == L.ERR_ARG
    lib = L.lib()
    import ctypes as C
    h = C.c_void_p()
    assert lib.lmood_mesh_create(2, 3, None, 1, None, 0, None, None, None, 1, None, C.byref(h)) == L.ERR_ARG
    assert lib.lmood_step(None, None) == L.ERR_ARG
    assert lib.lmood_get(None, 0, None, 0) == L.ERR_ARG


def test_destruction_in_any_order():
    """A mesh destroyed before its state, a state before its tape (as a garbage collector may
    order them): the dependent handles stay destroyable, every other call on them is an error."""
    pb = W.plain2d(n=8)
    st = L.simulation(pb)
    tape = L.Tape(st, 2)
    st.close()  # the state goes first: its tape is an orphan
    with pytest.raises(L.LmoodError):
        tape.backward(lam_v=np.ones((2, pb.mesh.n_cells)))
    tape.close()
    st2 = L.simulation(pb)
    tape2 = L.Tape(st2, 2)
    st2.mesh.close()  # the mesh goes first: its state can only be destroyed now
    assert st2.step_status() == L.ERR_STATE
    with pytest.raises(L.LmoodError) as e:
        st2.get(L.FIELD_V)
    assert e.value.status == L.ERR_STATE
    st2.close()
    tape2.close()
