"""lmood_autotune (-m gpu): the chosen launch shapes are among the candidates, the state is not
changed by tuning, and the steps that follow are bitwise the same as without tuning (the
arithmetic per cell and node does not depend on the block size), in both step modes."""
import numpy as np
import pytest

import paper_2104_02139_gb300 as L
import workloads as W

pytestmark = pytest.mark.gpu

FIELDS = (L.FIELD_X, L.FIELD_VP, L.FIELD_V, L.FIELD_E, L.FIELD_F, L.FIELD_ORDER, L.FIELD_DT)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available()
    L.build()


@pytest.mark.parametrize("graph", [1, 0])
def test_tuned_steps_are_bitwise_the_same(graph):
    for pb in (W.impact2d(n=120), W.cube3d(n=6)):
        a, b = L.simulation(pb, graph=graph), L.simulation(pb, graph=graph)
        a.run(3)
        b.run(3)
        before = {f: a.get(f) for f in FIELDS}
        res = a.autotune(reps=2)
        for f, v in before.items():
            assert np.array_equal(a.get(f), v), f
        cand = {"moments": (128, 256, 512), "predict": (64, 128, 256), "nodes": (128, 256, 512),
                "update": (64, 128, 256)}
        for k, r in res.items():
            assert r["chosen"] in cand[k]
            assert all(t > 0 for t in r["ms"].values())
            assert r["ms"][r["chosen"]] == min(r["ms"].values())
        for _ in range(8):
            ia, ib = a.step(), b.step()
            assert ia.n_troubled == ib.n_troubled and ia.dt_used == ib.dt_used
        for f in FIELDS:
            assert np.array_equal(a.get(f), b.get(f)), f


@pytest.mark.parametrize("case", ["impact2d", "cube3d", "batch"])
def test_tuned_schedule_is_bitwise_the_same(case):
    """lmood_autotune_schedule (node-window size, step form): the state is unchanged by the
    trial steps, the choices are among the candidates, and the steps after tuning are bitwise
    those of an untuned twin."""
    kw = {}
    if case == "impact2d":
        pb = W.impact2d(n=120)
    elif case == "cube3d":
        pb = W.cube3d(n=6)
    else:
        probs = W.batched2d(n_inst=6, lo=300, hi=4000)
        pb, inst = W.concat(probs)
        kw = {"cell_inst": inst, "n_inst": len(probs)}
    a, b = L.simulation(pb, **kw), L.simulation(pb, **kw)
    a.run(3)
    b.run(3)
    before = {f: a.get(f) for f in FIELDS}
    t_before = a.info.t
    res = a.autotune_schedule(reps=3)
    for f, v in before.items():
        assert np.array_equal(a.get(f), v), f
    assert res["node_window"]["chosen"] in (32, 256, 2048, 0)
    assert res["step_form"]["chosen"] in (1, 2)
    assert all(t > 0 for t in res["step_form"]["ms"].values())
    for _ in range(8):
        ia, ib = a.step(), b.step()
        assert ia.n_troubled == ib.n_troubled and ia.dt_used == ib.dt_used and ia.step == ib.step
    assert ia.t == ib.t and ia.t > t_before
    for f in FIELDS:
        assert np.array_equal(a.get(f), b.get(f)), f


def test_schedule_keeps_a_form_it_cannot_time():
    """the shear family (a = 0) has no persistent form: only the node order is tuned"""
    import dataclasses
    pb = dataclasses.replace(W.impact2d(n=60), shear_a=0.0)
    a = L.simulation(pb)
    res = a.autotune_schedule(reps=2)
    assert res["step_form"]["chosen"] == -1 and res["step_form"]["ms"] == {1: -1.0, 2: -1.0}
    a.run(2)
