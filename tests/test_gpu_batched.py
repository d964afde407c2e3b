"""Batched instances (independent meshes of uneven sizes, own dt each) advanced by one launch
per stage give exactly the per-instance results (-m gpu)."""
import numpy as np
import pytest

import paper_2104_02139_gb300 as L
import workloads as W

pytestmark = pytest.mark.gpu


def test_batch_equals_instances_bitwise():
    probs = W.batched2d(n_inst=5, lo=200, hi=5000, steps=12)
    pb, inst = W.concat(probs)
    b = L.simulation(pb, cell_inst=inst, n_inst=len(probs))
    singles = [L.simulation(q) for q in probs]
    for _ in range(pb.steps):
        b.step()
        for s in singles:
            s.step()
    dt = b.get(L.FIELD_DT)
    assert dt.shape == (len(probs),) and np.unique(dt).size == len(probs)
    full = {f: b.get(f) for f in (L.FIELD_X, L.FIELD_V, L.FIELD_E, L.FIELD_F, L.FIELD_ORDER)}
    c0 = n0 = 0
    for i, (q, s) in enumerate(zip(probs, singles)):
        nc, nn = q.mesh.n_cells, q.mesh.n_nodes
        assert np.array_equal(full[L.FIELD_X][:, n0:n0 + nn], s.get(L.FIELD_X))
        assert np.array_equal(full[L.FIELD_V][:, c0:c0 + nc], s.get(L.FIELD_V))
        assert np.array_equal(full[L.FIELD_E][c0:c0 + nc], s.get(L.FIELD_E))
        assert np.array_equal(full[L.FIELD_F][:, c0:c0 + nc], s.get(L.FIELD_F))
        assert np.array_equal(full[L.FIELD_ORDER][c0:c0 + nc], s.get(L.FIELD_ORDER))
        assert dt[i] == s.get(L.FIELD_DT)[0]
        c0 += nc
        n0 += nn


def test_batch_rejects_shared_nodes():
    probs = W.batched2d(n_inst=2, lo=200, hi=400)
    pb, inst = W.concat(probs)
    inst = inst.copy()
    inst[0] = 1  # a cell of instance 0 claims instance 1 while its nodes belong to instance 0
    with pytest.raises(L.LmoodError) as e:
        L.simulation(pb, cell_inst=inst, n_inst=2)
    assert e.value.status == L.ERR_MESH
