"""The persistent step (params.graph = 2: the whole step, MOOD rounds included, as one
cooperative launch with grid-wide barriers between the stages) and the graph-captured step
whose MOOD loop is one cooperative kernel node (params.graph = 3) against the graph-captured
step with the conditional while node (graph = 1), which the parity tests pin to the oracle:
bitwise identical states and reports, in 2D and 3D, with MOOD active, the three-level
cascade, batched instances, boundary faces, contact walls and (graph = 3) the other
materials; the error paths (MOOD iteration limit, a barrier wait that gives up) leave the
state unchanged (-m gpu)."""
import dataclasses

import numpy as np
import pytest

import oracle as O
import paper_2104_02139_gb300 as L
import workloads as W
from parity_util import Pair

pytestmark = pytest.mark.gpu

REPORT = ("n_troubled", "mood_iters", "n_p0", "n_parachute", "n_p0_eps", "n_lim", "dt_used", "dt_next")
FIELDS = (L.FIELD_X, L.FIELD_VP, L.FIELD_VSTAR, L.FIELD_V, L.FIELD_E, L.FIELD_F, L.FIELD_ORDER, L.FIELD_PKM,
          L.FIELD_DT)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available()
    L.build()
    O.build()


def _same(pb, steps, mode=2, **kw):
    a = L.simulation(pb, graph=mode, **kw)
    b = L.simulation(pb, graph=1, **kw)
    tot = {k: 0 for k in REPORT}
    for s in range(steps):
        ia, ib = a.step(), b.step()
        for k in REPORT:
            assert getattr(ia, k) == getattr(ib, k), (s, k)
            tot[k] += getattr(ia, k)
    for f in FIELDS:
        assert np.array_equal(a.get(f), b.get(f)), f
    return tot


def test_persistent_equals_graph_2d_mood():
    tot = _same(W.impact2d(n=120), 8)
    assert tot["n_troubled"] > 0 and tot["mood_iters"] > 0


def test_persistent_equals_graph_3d_mood():
    tot = _same(W.cube3d(n=6), 6)
    assert tot["n_troubled"] > 0


def test_persistent_equals_graph_cascade3():
    tot = _same(W.impact2d(n=60), 15, cascade=3)
    assert tot["n_lim"] > 0


def test_persistent_equals_graph_first_order_and_unlimited():
    _same(W.plain2d(n=30), 5, order=1)
    _same(W.plain2d(n=30), 5, mood=0)


def test_persistent_equals_graph_batched():
    probs = W.batched2d(n_inst=5, lo=200, hi=5000, steps=12)
    pb, inst = W.concat(probs)
    a = L.simulation(pb, cell_inst=inst, n_inst=len(probs), graph=2)
    b = L.simulation(pb, cell_inst=inst, n_inst=len(probs), graph=1)
    for _ in range(10):
        a.step()
        b.step()
    for f in FIELDS:
        assert np.array_equal(a.get(f), b.get(f)), f
    assert np.unique(a.get(L.FIELD_DT)).size == len(probs)


def test_persistent_equals_graph_boundary_faces_and_contact():
    _same(W.piston2d(n=16), 10)
    _same(W.rebound2d(n=11, gap=0.02), 40)


def test_persistent_matches_oracle():
    """one run side by side with the oracle, the same bar as the other parity tests"""
    pb = W.impact2d(n=40)
    p = Pair.__new__(Pair)
    p.pb, p.g, p.o = pb, L.simulation(pb, graph=2), O.Oracle(pb)
    st = p.run_compare(20)
    assert st["troubled"] > 0 and st["worst"] <= 1e-8


def test_persistent_mood_iteration_limit():
    s = L.simulation(W.cube3d(n=6), graph=2, max_mood_iters=2)
    before = s.state()
    assert s.step_status() == L.ERR_MOOD_ITERS
    for k, v in before.items():
        assert np.array_equal(v, s.state()[k]), k


def test_barrier_wait_that_gives_up_reports_timeout():
    """With a one-poll bound on every grid-barrier wait, blocks that arrive early give up: the
    launch ends, the step returns LMOOD_ERR_TIMEOUT and the state stays at t^n; the context
    stays usable (the same state steps normally once the bound is the default again)."""
    pb = W.plain2d(n=60)
    s = L.simulation(pb, graph=2, barrier_polls=1)
    before = s.state()
    codes = [s.step_status() for _ in range(5)]
    assert set(codes) <= {L.OK, L.ERR_TIMEOUT}
    assert L.ERR_TIMEOUT in codes
    if L.OK not in codes:
        for k, v in before.items():
            assert np.array_equal(v, s.state()[k]), k
    ref = L.simulation(pb, graph=1)
    ok = L.simulation(pb, graph=2)
    ref.run(3)
    ok.run(3)
    for f in FIELDS:
        assert np.array_equal(ref.get(f), ok.get(f)), f


def test_persistent_refuses_other_materials():
    for kw in ({"shear_a": 0.0}, {"stiffened_gas": (4.4, 0.6, 1e-4)}):
        with pytest.raises(L.LmoodError) as e:
            L.simulation(dataclasses.replace(W.plain2d(n=8), **kw), graph=2)
        assert e.value.status == L.ERR_ARG
    with pytest.raises(L.LmoodError) as e:
        L.simulation(W.plain2d(n=8), graph=4)
    assert e.value.status == L.ERR_ARG


MODE3 = [("impact2d", lambda: W.impact2d(n=120), 8, {}), ("cube3d", lambda: W.cube3d(n=6), 6, {}),
         ("cascade3", lambda: W.impact2d(n=60), 15, {"cascade": 3}),
         ("piston", lambda: W.piston2d(n=16), 10, {}), ("rebound", lambda: W.rebound2d(n=11, gap=0.02), 40, {}),
         ("family", lambda: dataclasses.replace(W.impact2d(n=60), shear_a=0.0), 10, {}),
         ("jellydrop", lambda: W.jellydrop3d(n=5, steps=30), 30, {})]


@pytest.mark.parametrize("name,make,steps,kw", MODE3, ids=[m[0] for m in MODE3])
def test_mood_kernel_node_equals_graph(name, make, steps, kw):
    tot = _same(make(), steps, mode=3, **kw)
    if name in ("impact2d", "cube3d", "cascade3"):
        assert tot["n_troubled"] > 0


def test_mood_kernel_node_batched():
    probs = W.batched2d(n_inst=5, lo=200, hi=5000, steps=12)
    pb, inst = W.concat(probs)
    a = L.simulation(pb, cell_inst=inst, n_inst=len(probs), graph=3)
    b = L.simulation(pb, cell_inst=inst, n_inst=len(probs), graph=1)
    for _ in range(10):
        a.step()
        b.step()
    for f in FIELDS:
        assert np.array_equal(a.get(f), b.get(f)), f


def test_mood_kernel_node_errors():
    """iteration limit and a barrier wait that gives up (one-poll bound) in the MOOD node"""
    s = L.simulation(W.cube3d(n=6), graph=3, max_mood_iters=2)
    before = s.state()
    assert s.step_status() == L.ERR_MOOD_ITERS
    for k, v in before.items():
        assert np.array_equal(v, s.state()[k]), k
    s = L.simulation(W.impact2d(n=60), graph=3, barrier_polls=1)
    before = s.state()
    codes = [s.step_status() for _ in range(5)]
    assert set(codes) <= {L.OK, L.ERR_TIMEOUT}
    assert L.ERR_TIMEOUT in codes
    if L.OK not in codes:
        for k, v in before.items():
            assert np.array_equal(v, s.state()[k]), k
