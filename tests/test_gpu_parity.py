"""CUDA path vs the CPU oracle, element by element, on the same seeded inputs (-m gpu).

Tolerances: a state relative error of at most 1e-11 after one step and 1e-8 after the
configured run, with identical MOOD order masks at every step. Both sides
compute in FP64; the differences come from FMA contraction and the two math libraries'
log/cbrt (a few ulp), i.e. ~1e-15 relative per step.
"""
import numpy as np
import pytest

import oracle as O
import paper_2104_02139_gb300 as L
import workloads as W
from parity_util import Pair, relerr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available()
    L.build()
    O.build()


def test_init_parity():
    for pb in (W.plain2d(n=20), W.cube3d(n=4), W.column3d(nxy=3, nz=9)):
        p = Pair(pb)
        np.testing.assert_allclose(p.g.get(L.FIELD_MASS), p.o.get(O.F_MASS), rtol=1e-14)
        err = p.errors()
        assert max(err.values()) <= 1e-13, err


@pytest.mark.parametrize("case", ["plain2d", "impact2d", "cube3d", "column3d"])
def test_kernel_level_parity(case):
    """Corner packets (M_cp, rhs_cp) and nodal velocities v*_p after one step."""
    pb = {"plain2d": lambda: W.plain2d(n=24),
          "impact2d": lambda: W.impact2d(n=40),
          "cube3d": lambda: W.cube3d(n=5),
          "column3d": lambda: W.column3d(nxy=3, nz=12)}[case]()
    pb.v *= 3.0
    p = Pair(pb)
    p.step()
    d = pb.mesh.dim
    nv = d + 1
    oM = p.o.get(O.F_PKM).reshape(d, d, nv, -1)
    gM = p.g.get(L.FIELD_PKM)
    s = 0
    for a in range(d):
        for b in range(a, d):
            assert relerr(gM[s], oM[a, b]) <= 1e-12, (a, b)
            s += 1
    assert relerr(p.g.get(L.FIELD_PKR), p.o.get(O.F_PKR)) <= 1e-11
    assert relerr(p.g.get(L.FIELD_VSTAR), p.o.get(O.F_VSTAR)) <= 1e-11
    mg, mo = p.masks()
    assert np.array_equal(mg, mo)


def test_plain2d_full_run():
    """40x40 lattice, 3,042 triangles, slip walls, 200 steps (MOOD active in the first steps)."""
    pb = W.plain2d()
    stats = Pair(pb).run_compare(pb.steps)
    assert stats["troubled"] > 0


def test_impact2d_small_run():
    pb = W.impact2d(n=60)
    stats = Pair(pb).run_compare(60)
    assert stats["troubled"] > 0


def test_3d_runs():
    Pair(W.cube3d(n=6)).run_compare(30)
    pb = W.column3d(nxy=4, nz=24)
    pb.v *= 5
    Pair(pb).run_compare(30)


def test_first_order_and_unlimited_modes():
    pb = W.impact2d(n=30)
    Pair(pb, order=1).run_compare(20)
    Pair(W.plain2d(n=16), mood=0).run_compare(20)


def test_impact2d_full_size_steps():
    """999,698 triangles (the benchmark workload): first steps, element by element."""
    pb = W.impact2d()
    Pair(pb).run_compare(3)


def test_cube3d_full_size_step():
    """511,104 tetrahedra: first step, element by element."""
    pb = W.cube3d()
    Pair(pb).run_compare(1)


def test_determinism():
    pb = W.impact2d(n=80)
    a, b = L.simulation(pb), L.simulation(pb)
    a.run(15)
    b.run(15)
    for f in (L.FIELD_X, L.FIELD_V, L.FIELD_E, L.FIELD_F, L.FIELD_ORDER):
        assert np.array_equal(a.get(f), b.get(f))


def test_energy_conservation_full_size():
    pb = W.impact2d()
    g = L.simulation(pb)
    t0 = g.totals()
    g.run(20)
    t1 = g.totals()
    assert abs(t1[4] - t0[4]) <= 1e-12 * abs(t0[4])
    assert t1[0] == pytest.approx(t0[0], rel=1e-14)


def test_graph_and_host_modes_bitwise():
    """The graph-captured step (MOOD loop as a device-side while node) and the host-driven
    MOOD rounds give bitwise identical results and reports."""
    for pb in (W.impact2d(n=120), W.cube3d(n=5)):
        a, b = L.simulation(pb, graph=1), L.simulation(pb, graph=0)
        for _ in range(8):
            ia, ib = a.step(), b.step()
            for k in ("n_troubled", "mood_iters", "n_p0", "dt_used", "dt_next"):
                assert getattr(ia, k) == getattr(ib, k), k
        for f in (L.FIELD_X, L.FIELD_VP, L.FIELD_V, L.FIELD_E, L.FIELD_F, L.FIELD_ORDER, L.FIELD_PKM):
            assert np.array_equal(a.get(f), b.get(f)), f


def test_mood_iteration_limit_reports_error():
    """A step that would need more MOOD rounds than allowed returns LMOOD_ERR_MOOD_ITERS and
    leaves the state unchanged (both modes)."""
    pb = W.cube3d(n=6)
    for graph in (1, 0):
        s = L.simulation(pb, graph=graph, max_mood_iters=2)
        before = s.state()
        assert s.step_status() == L.ERR_MOOD_ITERS
        for k, v in before.items():
            assert np.array_equal(v, s.state()[k]), k


def test_column3d_full_size_first_steps():
    """5,989,500 tetrahedra (the 3D column configuration): the first two steps from the
    seeded initial data, element by element (masks identical, state within 1e-11 after the
    first step)."""
    Pair(W.column3d()).run_compare(2)


def test_tiny_meshes():
    """One triangle, two triangles and one tetrahedron (empty or one-cell stencils, every node
    on the boundary): same results as the oracle."""
    for x, c2n, d in ((np.array([[0.0, 1.0, 0.0], [0.0, 0.0, 1.0]]), np.array([[0], [1], [2]]), 2),
                      (np.array([[0.0, 1.0, 1.0, 0.0], [0.0, 0.0, 1.0, 1.0]]), np.array([[0, 0], [1, 2], [2, 3]]), 2),
                      (np.array([[0.0, 1, 0, 0], [0.0, 0, 1, 0], [0.0, 0, 0, 1]]), np.array([[0], [1], [2], [3]]), 3)):
        m = W.Mesh(d, x, c2n.astype(np.int32), np.zeros((d, 0), np.int32), np.zeros(0, np.int32))
        nc = c2n.shape[1]
        v = np.arange(1, d * nc + 1, dtype=float).reshape(d, nc) * 0.01
        pb = W.Problem("tiny", m, 1.0, 2.0, np.ones(nc), v, 0.4, 5)
        Pair(pb).run_compare(5)


def test_clamped_everywhere_stays_put():
    pb = W.plain2d(n=10)
    pb.mesh.btag[:] = W.CLAMPED
    p = Pair(pb)
    x0 = p.g.get(L.FIELD_X)
    p.run_compare(5)
    assert np.array_equal(p.g.get(L.FIELD_X)[:, np.unique(pb.mesh.bface)], x0[:, np.unique(pb.mesh.bface)])


def test_three_level_cascade_parity():
    """P1 -> P1 with Barth-Jespersen slopes -> P0: identical order masks (codes 2, 3, 1) and
    states as the oracle, in 2D and 3D; graph and host-driven modes agree bitwise."""
    pb = W.impact2d(n=60)
    stats = Pair(pb, cascade=3).run_compare(30)
    assert stats["troubled"] > 0
    pb3 = W.column3d(nxy=4, nz=24)
    pb3.v *= 5
    Pair(pb3, cascade=3).run_compare(15)
    a, b = L.simulation(pb, cascade=3, graph=1), L.simulation(pb, cascade=3, graph=0)
    lim = 0
    for _ in range(15):
        lim += a.step().n_lim
        b.step()
    assert lim > 0
    for f in (L.FIELD_X, L.FIELD_V, L.FIELD_F, L.FIELD_ORDER):
        assert np.array_equal(a.get(f), b.get(f)), f
