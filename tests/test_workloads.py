"""The seeded input generators: sizes of the named workloads, orientation, determinism."""
import numpy as np

import workloads as W


def test_tri_mesh_counts_and_orientation():
    m = W.tri_mesh(40, 1, bc={"x0": W.SLIP})
    assert m.n_cells == 2 * 39 ** 2 == 3042 and m.n_nodes == 1600
    x = m.x.T[m.c2n.T]
    e1, e2 = x[:, 1] - x[:, 0], x[:, 2] - x[:, 0]
    assert np.all(e1[:, 0] * e2[:, 1] - e1[:, 1] * e2[:, 0] > 0)
    assert m.btag.size == 39 and np.all(m.x[0, m.bface.ravel()] == 0.0)


def test_tet_mesh_counts_and_orientation():
    m = W.tet_mesh(3, 4, 5, 3, bc={"z0": W.CLAMPED})
    assert m.n_cells == 6 * 60 and m.n_nodes == 4 * 5 * 6
    x = m.x.T[m.c2n.T]
    assert np.all(np.linalg.det(x[:, 1:] - x[:, :1]) > 0)
    assert m.btag.size == 2 * 3 * 4 and np.all(m.x[2, m.bface.ravel()] == 0.0)


def test_seeded_determinism():
    a, b = W.impact2d(n=30), W.impact2d(n=30)
    assert np.array_equal(a.mesh.x, b.mesh.x) and np.array_equal(a.mesh.c2n, b.mesh.c2n)
    c = W.cube3d(n=4)
    assert np.all(np.abs(c.mu - 1) < 1.0) and c.mu.std() > 0.05


def test_concat_offsets():
    probs = W.batched2d(n_inst=3, lo=100, hi=300)
    pb, inst = W.concat(probs)
    assert pb.mesh.n_cells == sum(q.mesh.n_cells for q in probs) == inst.size
    assert np.array_equal(np.bincount(inst), [q.mesh.n_cells for q in probs])
    # no node is shared between instances
    owner = np.full(pb.mesh.n_nodes, -1)
    for k in range(3):
        owner[pb.mesh.c2n[k]] = inst
    for k in range(3):
        assert np.array_equal(owner[pb.mesh.c2n[k]], inst)
