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


def _volumes(m):
    x = m.x.T[m.c2n.T]  # [nc, d+1, d]
    e = x[:, 1:] - x[:, :1]
    return np.linalg.det(e) if m.dim == 3 else e[:, 0, 0] * e[:, 1, 1] - e[:, 0, 1] * e[:, 1, 0]


def test_paper_problem_meshes():
    """the beryllium plate, Blake's needle and the swinging cube: positively oriented cells
    that fill their domains, boundary faces tagged as the problems state"""
    be = W.be_plate(nx=13, ny=4)
    assert be.mesh.n_cells == 2 * 12 * 3 and be.mesh.btag.size == 0  # free boundaries only
    assert np.all(_volumes(be.mesh) > 0)
    assert abs(_volumes(be.mesh).sum() / 2 - 0.06 * 0.01) < 1e-15
    cube = W.swinging_cube(3)
    assert cube.mesh.n_cells == 6 * 27 and np.all(_volumes(cube.mesh) > 0)
    assert abs(_volumes(cube.mesh).sum() / 6 - 8.0) < 1e-12
    assert np.all(cube.mesh.btag == W.SLIP) and cube.mesh.btag.size == 6 * 2 * 9
    # Blake's needle: the lateral slip faces lie in planes through the centre, the pressure
    # face on the sphere r = 0.1, the free outer face on r = 1 (not tagged)
    bl = W.blake3d(nr=6, nlat=2)
    m = bl.mesh
    assert np.all(_volumes(m) > 0)
    xf = m.x.T[m.bface.T]  # [nb, 3, 3]
    slip = m.btag == W.SLIP
    nrm = np.cross(xf[:, 1] - xf[:, 0], xf[:, 2] - xf[:, 0])
    nrm /= np.linalg.norm(nrm, axis=1)[:, None]
    assert np.abs((nrm[slip, None, :] * xf[slip]).sum(axis=2)).max() < 1e-14  # n . x = 0
    pr = m.btag == W.PRESSURE
    assert pr.sum() == 2 * 2 * 2 and np.abs(np.linalg.norm(xf[pr], axis=2) - 0.1).max() < 1e-15
    assert np.all(bl.bcval[0, pr] == 1e6) and np.all(bl.bcval[:, ~pr] == 0.0)
    r = np.linalg.norm(m.x, axis=0)
    assert abs(r.min() - 0.1) < 1e-15 and abs(r.max() - 1.0) < 1e-15
