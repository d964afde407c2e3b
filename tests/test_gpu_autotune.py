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
