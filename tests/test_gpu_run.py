"""lmood_run chains its steps on the device (-m gpu): nsteps step graphs launched back to back
behind a device-side gate, one host synchronisation for the whole run. The result must be
bitwise that of nsteps lmood_step calls -- fields, next dt, time, step count and the last
report -- and a run whose k-th step fails must stop there with the same error and the state
of the k - 1 accepted steps."""
import numpy as np
import pytest

import paper_2104_02139_gb300 as L
import workloads as W

pytestmark = pytest.mark.gpu

FIELDS = (L.FIELD_X, L.FIELD_VP, L.FIELD_V, L.FIELD_E, L.FIELD_F, L.FIELD_TAU, L.FIELD_ORDER, L.FIELD_DT,
          L.FIELD_PKM, L.FIELD_VSTAR)
REPORT = ("t", "dt_used", "dt_next", "step", "n_troubled", "n_p0", "mood_iters", "n_parachute", "n_p0_eps", "n_lim")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available()
    L.build()


def _same(a, b):
    for f in FIELDS:
        assert np.array_equal(a.get(f), b.get(f)), f


@pytest.mark.parametrize("case", ["plain2d_config1", "impact2d_mood", "cube3d", "batch"])
def test_run_is_bitwise_the_steps(case):
    kw = {}
    if case == "plain2d_config1":
        pb, n = W.plain2d(), 200          # the 40 x 40 configuration: 3,042 triangles, 200 steps
    elif case == "impact2d_mood":
        pb, n = W.impact2d(n=60), 30
    elif case == "cube3d":
        pb, n = W.cube3d(n=5), 12
        pb.v *= 4.0
    else:
        probs = W.batched2d(n_inst=6, lo=300, hi=4000, steps=20)
        pb, inst = W.concat(probs)
        kw = {"cell_inst": inst, "n_inst": len(probs)}
        n = 20
    a, b = L.simulation(pb, **kw), L.simulation(pb, **kw)
    ra = a.run(n)
    ra = {k: getattr(ra, k) for k in REPORT + ("syncs",)}
    for _ in range(n):
        rb = b.step()
    assert ra["syncs"] == 1, "the run was not chained on the device"
    for k in REPORT:
        assert ra[k] == getattr(rb, k), k
    _same(a, b)
    # and it goes on from there like the stepped state
    a.run(3)
    b.run(1), b.step(), b.step()
    _same(a, b)


def test_run_stops_at_the_failing_step():
    """impact2d on a 60 x 60 lattice needs 1, 1, 2, 3 MOOD rounds in its first four steps: with
    max_mood_iters = 2 the fourth step fails (LMOOD_ERR_MOOD_ITERS) and the state is that of
    the first three, in the chained run as step by step."""
    pb = W.impact2d(n=60)
    a = L.simulation(pb, max_mood_iters=2)
    b = L.simulation(pb, max_mood_iters=2)
    with pytest.raises(L.LmoodError) as ea:
        a.run(10)
    assert ea.value.status == L.ERR_MOOD_ITERS
    for k in range(3):
        b.step()
    assert b.step_status() == L.ERR_MOOD_ITERS
    assert a.info.step == b.info.step == 3 and a.info.mood_iters == b.info.mood_iters
    _same(a, b)


def test_run_with_timing_or_other_step_forms_steps_one_at_a_time():
    pb = W.plain2d(n=20)
    for graph in (0, 2, 3):
        a, b = L.simulation(pb, graph=graph), L.simulation(pb, graph=1)
        ia = a.run(6)
        assert ia.syncs >= 6
        b.run(6)
        _same(a, b)
    c = L.simulation(pb)
    c.timing(True)
    assert c.run(4).syncs >= 4
    c.timing(False)
    assert c.run(4).syncs == 1
