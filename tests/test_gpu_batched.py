"""Batched instances (independent meshes of uneven sizes, own dt each) advanced by one launch
per stage give exactly the per-instance results; at the full 256-instance size, sampled
instances match the oracle stepping them one by one (-m gpu)."""
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


def test_full_size_batch_sampled_instances_match_oracle():
    """The 256-instance configuration at full size (11.6M cells, one launch per stage for all
    instances, own dt each): the smallest, the largest and two more instances, sampled, are
    stepped by the oracle one by one and compared element by element with their slices of the
    batch after every step (masks identical, state within 1e-11 after the first step and 1e-8
    after three)."""
    import oracle as O
    from parity_util import relerr
    O.build()
    probs = W.batched2d()
    pb, inst = W.concat(probs)
    b = L.simulation(pb, cell_inst=inst, n_inst=len(probs))
    cells = np.asarray(pb.meta["cells"])
    c_off = np.concatenate([[0], np.cumsum(cells)])
    n_off = np.concatenate([[0], np.cumsum(pb.meta["nodes"])])
    rng = np.random.default_rng(11)
    pick = sorted({int(cells.argmin()), int(cells.argmax()), *rng.choice(len(probs), 2, replace=False).tolist()})
    oracles = {i: O.Oracle(probs[i]) for i in pick}
    pairs = ((L.FIELD_X, O.F_X, "node"), (L.FIELD_VP, O.F_VP, "node"), (L.FIELD_V, O.F_V, "cell"),
             (L.FIELD_E, O.F_E, "cell"), (L.FIELD_F, O.F_F, "cell"), (L.FIELD_TAU, O.F_TAU, "cell"))
    for s in range(3):
        b.step()
        full = {fg: b.get(fg) for fg, _, _ in pairs}
        order = b.get(L.FIELD_ORDER).astype(int)
        dt = b.get(L.FIELD_DT)
        for i, o in oracles.items():
            o.step()
            cs, ns = slice(c_off[i], c_off[i + 1]), slice(n_off[i], n_off[i + 1])
            assert np.array_equal(order[cs], o.get(O.F_ORDER).astype(int)), (s, i)
            tol = 1e-11 if s == 0 else 1e-8
            for fg, fo, kind in pairs:
                g = full[fg][..., ns] if kind == "node" else full[fg][..., cs]
                assert relerr(g, o.get(fo)) <= tol, (s, i, fg)
            assert abs(dt[i] - o.dt) <= tol * o.dt, (s, i)
