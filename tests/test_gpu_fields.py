"""lmood_get_fields / lmood_set_fields (several fields per call, one synchronisation) give the
same results as field-by-field lmood_get / lmood_set, host and device; arguments are all
checked before the first copy (-m gpu)."""
import numpy as np
import pytest

import paper_2104_02139_gb300 as L
import workloads as W

pytestmark = pytest.mark.gpu

STATE = (L.FIELD_X, L.FIELD_VP, L.FIELD_V, L.FIELD_E, L.FIELD_F, L.FIELD_DT)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available()
    L.build()


def test_get_fields_equals_get():
    s = L.simulation(W.impact2d(n=50))
    s.run(4)
    ids = STATE + (L.FIELD_ORDER, L.FIELD_TAU, L.FIELD_PKM)
    outs = s.get_fields({f: np.empty(s.shape(f)) for f in ids})
    for f in ids:
        assert np.array_equal(outs[f], s.get(f)), f


def test_set_fields_restart_is_bitwise():
    """a run restarted from its own state through one set_fields call (host, then device)
    continues bitwise like the uninterrupted run"""
    import torch
    pb = W.cube3d(n=5)
    a = L.simulation(pb)
    a.run(3)
    st = {f: a.get(f) for f in STATE}
    b = L.simulation(pb)
    b.set_fields(st)
    c = L.simulation(pb)
    c.set_fields({f: torch.tensor(v, device="cuda") for f, v in st.items()})
    torch.cuda.synchronize()
    for s in (a, b, c):
        s.run(4)
    for f in STATE + (L.FIELD_TAU, L.FIELD_ORDER):
        assert np.array_equal(a.get(f), b.get(f)), f
        assert np.array_equal(a.get(f), c.get(f)), f


def test_device_get_fields():
    import torch
    s = L.simulation(W.plain2d(n=20))
    s.run(2)
    outs = s.get_fields({f: torch.empty(s.shape(f), dtype=torch.float64, device="cuda") for f in STATE})
    torch.cuda.synchronize()
    for f in STATE:
        assert np.array_equal(outs[f].cpu().numpy(), s.get(f)), f


def test_field_arguments_checked_first():
    s = L.simulation(W.plain2d(n=10))
    x0 = s.get(L.FIELD_X)
    for bad in ({L.FIELD_X: x0 + 1.0, L.FIELD_TAU: np.ones(s.shape(L.FIELD_TAU))},  # read-only
                {L.FIELD_X: x0 + 1.0, 42: np.ones(3)}):  # unknown id
        with pytest.raises(L.LmoodError) as e:
            s.set_fields(bad)
        assert e.value.status == L.ERR_ARG
        assert np.array_equal(s.get(L.FIELD_X), x0)  # nothing was copied
    with pytest.raises(L.LmoodError) as e:
        s.get_fields({L.FIELD_X: np.empty(s.shape(L.FIELD_X)), -1: np.empty(3)})
    assert e.value.status == L.ERR_ARG
