"""Pins of the oracle's traction, pressure and prescribed-velocity boundary conditions
(Appendix B, Eqs. pBC, vBC1, vBC; reading R15), of boundary conditions that change type
during a run and of contact walls (Sect. "Boundary condition treatments"; reading R17). CPU
only.

Each pin is fixed by mechanics, not by the oracle's own formulas: a uniformly stressed block
held by the matching pressure stays at rest; the momentum a free block gains equals the
impulse of the applied tractions; the energy it gains equals their work on the nodes; a
prescribed normal velocity is met exactly at every node of the face, corners with a slip wall
included; a block translating with the piston's velocity stays a rigid translation; a block
rebounding from a contact wall keeps its energy and never reaches the wall.
"""
import dataclasses

import numpy as np
import pytest

import oracle as O
import workloads as W


def _block(n=8, seed=3, bc=None, v=(0.0, 0.0), F=None, mu=1.0, lam=2.0):
    m = W.tri_mesh(n, seed, bc=bc or {})
    v0 = np.tile(np.asarray(v, dtype=float)[:, None], (1, m.n_cells))
    return W.Problem("block", m, 1.0, lam, np.full(m.n_cells, mu), v0, 0.4, 10, F=F)


def _face_vectors(m, x):
    """outward area vector of every boundary face at positions x [d][np] (orientation from
    the cell on the face's inner side)"""
    c2n = m.c2n.T
    bf = m.bface.T
    out = np.zeros((bf.shape[0], m.dim))
    for i, (q0, q1) in enumerate(bf):
        N = np.array([x[1, q1] - x[1, q0], x[0, q0] - x[0, q1]])
        cells = np.where(np.isin(c2n, [q0, q1]).sum(axis=1) == 2)[0]
        opp = [q for q in c2n[cells[0]] if q not in (q0, q1)][0]
        mid = 0.5 * (x[:, q0] + x[:, q1])
        if N @ (mid - x[:, opp]) < 0:
            N = -N
        out[i] = N
    return out


def test_pressure_holds_a_uniformly_stressed_block_at_rest():
    """F = s I (plane strain) gives a uniform in-plane stress sigma I; the pressure -sigma on
    every face balances it exactly, so nothing moves. Without it the block springs back."""
    s = 0.97
    F = np.zeros((4, 1))
    F[0] = F[3] = s
    kappa = 2.0 + 2.0 / 3.0
    T = O.stress(np.array([[s, 0.0], [0.0, s]]), 1.0, kappa)
    sigma = T[0, 0]
    assert abs(T[0, 1]) < 1e-15 and abs(T[1, 1] - sigma) < 1e-15
    pb = _block(bc={k: W.PRESSURE for k in ("x0", "x1", "y0", "y1")})
    pb = dataclasses.replace(pb, F=np.tile(F, (1, pb.mesh.n_cells)),
                             bcval=W.side_values(pb.mesh, W.PRESSURE, (-sigma, 0.0)))
    o = O.Oracle(pb)
    x0 = o.get(O.F_X).copy()
    for _ in range(5):
        o.step()
    assert np.abs(o.get(O.F_V)).max() < 1e-13
    assert np.abs(o.get(O.F_VP)).max() < 1e-13
    assert np.abs(o.get(O.F_X) - x0).max() < 1e-14
    free = O.Oracle(dataclasses.replace(pb, bcval=None))
    for _ in range(5):
        free.step()
    assert np.abs(free.get(O.F_V)).max() > 1e-4


def test_traction_impulse_and_work():
    """Free block at rest, random tractions on its faces: after one step the momentum equals
    dt sum_f |N_f| t_f and the total energy change equals dt sum_p F_p . v*_p, F_p the
    nodes' shares |N_f| t_f / 2 of the faces around them."""
    pb = _block(n=9, bc={k: W.TRACTION for k in ("x0", "x1", "y0", "y1")})
    rng = np.random.default_rng(4)
    t = rng.normal(size=(2, pb.mesh.btag.size)) * 0.01
    pb = dataclasses.replace(pb, bcval=t)
    o = O.Oracle(pb)
    x0 = o.get(O.F_X).copy()
    m = o.get(O.F_MASS)
    e0 = o.get(O.F_E).copy()
    dt = o.dt
    o.step()
    Nf = _face_vectors(pb.mesh, x0)
    area = np.linalg.norm(Nf, axis=1)
    impulse = dt * (area[None, :] * t).sum(axis=1)
    mom = (m[None, :] * o.get(O.F_V)).sum(axis=1)
    np.testing.assert_allclose(mom, impulse, rtol=1e-12, atol=1e-16)
    Fp = np.zeros_like(x0)
    for i, q in enumerate(pb.mesh.bface.T):
        for p in q:
            Fp[:, p] += area[i] * t[:, i] / 2
    work = dt * (Fp * o.get(O.F_VSTAR)).sum()
    dE = (m * (o.get(O.F_E) - e0)).sum()
    assert abs(dE - work) <= 1e-12 * abs(work)


def test_piston_normal_velocity_is_met_exactly():
    """The x = 0 face moves with the prescribed V at every node, including the two corners
    that also lie on a slip wall (whose normal velocity stays zero)."""
    pb = W.piston2d(n=10)
    V = pb.bcval[0, pb.mesh.btag == W.VELOCITY][0]
    o = O.Oracle(pb)
    x = o.get(O.F_X)
    on = np.where(np.abs(x[0]) < 1e-15)[0]
    corners = on[(np.abs(x[1, on]) < 1e-15) | (np.abs(x[1, on] - 1.0) < 1e-15)]
    assert on.size == 10 and corners.size == 2
    for _ in range(6):
        o.step()
        vs = o.get(O.F_VSTAR)
        np.testing.assert_allclose(vs[0, on], V, rtol=1e-13)
        assert np.abs(vs[1, corners]).max() < 1e-15
    assert np.abs(o.get(O.F_X)[0, on] - V * o.t).max() < 1e-14


def test_piston_with_the_block_velocity_is_a_rigid_translation():
    pb = _block(n=8, bc={"x0": W.VELOCITY}, v=(0.03, -0.01))
    pb = dataclasses.replace(pb, bcval=W.side_values(pb.mesh, W.VELOCITY, (0.03, -0.01)))
    o = O.Oracle(pb)
    for _ in range(5):
        o.step()
    v = o.get(O.F_V)
    assert np.abs(v[0] - 0.03).max() < 1e-14 and np.abs(v[1] + 0.01).max() < 1e-14
    F = o.get(O.F_F)
    assert np.abs(F[0] - 1).max() < 1e-13 and np.abs(F[1]).max() < 1e-13 and np.abs(F[3] - 1).max() < 1e-13


def test_piston_prescribed_velocity_differs_from_the_block():
    """A piston slower than the block decelerates the nodes on its face to V, and the
    compression wave it starts raises the density next to it."""
    pb = _block(n=8, bc={"x0": W.VELOCITY}, v=(-0.05, 0.0))
    pb = dataclasses.replace(pb, bcval=W.side_values(pb.mesh, W.VELOCITY, (0.0, 0.0)))
    o = O.Oracle(pb)
    x = o.get(O.F_X)
    on = np.where(np.abs(x[0]) < 1e-15)[0]
    for _ in range(4):
        o.step()
    assert np.abs(o.get(O.F_VSTAR)[0, on]).max() < 1e-15
    assert (1.0 / o.get(O.F_TAU)).max() > 1.0 + 1e-3


def test_boundary_tags_can_change_during_a_run():
    """Slip walls replaced by clamped ones between two steps: the wall nodes stop."""
    pb = W.plain2d(n=10)
    pb = dataclasses.replace(pb, v=pb.v * 50)
    o = O.Oracle(pb)
    o.step()
    x = o.get(O.F_X)
    wall = np.where((np.abs(x[0]) < 1e-12) | (np.abs(x[0] - 1) < 1e-12) | (np.abs(x[1]) < 1e-12)
                    | (np.abs(x[1] - 1) < 1e-12))[0]
    assert np.abs(o.get(O.F_VSTAR)[:, wall]).max() > 1e-5
    o.set_btag(np.full(pb.mesh.btag.size, W.CLAMPED))
    assert all(o.bc_ndof(p) == 0 for p in wall)
    o.step()
    assert np.abs(o.get(O.F_VSTAR)[:, wall]).max() == 0.0
    with pytest.raises(O.OracleError):
        o.set_btag(np.full(pb.mesh.btag.size, 7))


def test_contact_wall_rebound():
    """A block flying at a wall through its contact face (reading R17): free flight until the
    face comes within eps of the wall, no node closer than the capture distance minus one
    step's travel, total energy conserved to round-off (the wall does no work), the normal
    momentum reversed, and after the face has detached the momentum is constant again."""
    gap = 0.1
    pb = W.rebound2d(n=11, gap=gap)
    eps = pb.contact[1]
    o = O.Oracle(pb)
    m = o.get(O.F_MASS)
    E0 = (m * o.get(O.F_E)).sum()
    face = np.where(o.get(O.F_X)[0] == 0.0)[0]
    contact_seen = detached_at = None
    p_after = []
    for s in range(400):
        o.step()
        x = o.get(O.F_X)
        px = (m * o.get(O.F_V)[0]).sum()
        d = x[0, face] + gap
        assert abs((m * o.get(O.F_E)).sum() - E0) <= 1e-14 * E0
        assert (x[0] + gap).min() >= eps - 0.1 * o.dt - 1e-15
        if contact_seen is None:
            if (d < eps).any():
                contact_seen = s
            else:
                assert px == pytest.approx(-0.1 * m.sum(), rel=1e-13)
        elif detached_at is None and (d > eps).all() and px > 0:
            detached_at = s
        elif detached_at is not None:
            p_after.append(px)
    assert contact_seen is not None and detached_at is not None
    assert min(p_after) > 0.3 * 0.1 * m.sum()
    assert max(p_after) - min(p_after) <= 1e-13 * max(p_after)


def test_contact_face_without_walls_is_free():
    """The same block without contact walls flies through the plane."""
    gap = 0.1
    pb = dataclasses.replace(W.rebound2d(n=11, gap=gap), contact=None)
    o = O.Oracle(pb)
    for _ in range(200):
        o.step()
    assert (o.get(O.F_X)[0] + gap).min() < -0.02


def test_piston_in_3d_meets_its_velocity_exactly():
    """A box pushed through its x = 0 face (prescribed normal velocity V, Eq. vBC; reading R15)
    with slip walls at y = 0, y = 1: every node of the face, those on its edges with the slip
    walls included, moves with v*_x = V exactly, and the edge nodes keep zero velocity across
    their slip wall."""
    m = W.tet_mesh(4, 4, 4, 9, bc={"x0": W.VELOCITY, "y0": W.SLIP, "y1": W.SLIP})
    V = 0.03
    pb = W.Problem("piston3d", m, 1.0, 2.0, np.full(m.n_cells, 1.0), np.zeros((3, m.n_cells)), 0.25, 5,
                   bcval=W.side_values(m, W.VELOCITY, (V, 0.0, 0.0)))
    o = O.Oracle(pb)
    x = o.get(O.F_X)
    face = np.where(np.abs(x[0]) < 1e-15)[0]
    edges = face[(np.abs(x[1, face]) < 1e-15) | (np.abs(x[1, face] - 1.0) < 1e-15)]
    assert face.size == 25 and edges.size == 10
    for _ in range(4):
        o.step()
        vs = o.get(O.F_VSTAR)
        np.testing.assert_allclose(vs[0, face], V, rtol=1e-13)
        assert np.abs(vs[1, edges]).max() == 0.0
    assert np.abs(o.get(O.F_X)[0, face] - V * o.t).max() < 1e-14


def test_contact_floor_in_3d():
    """A block falling onto a floor through its contact face (reading R17) in 3D: free fall
    until the face comes within eps of the floor, then no node closer than eps less one step's
    travel, total energy conserved to round-off (the floor does no work), the vertical momentum
    reversed by the contact and constant again once the face has detached."""
    m = W.tet_mesh(4, 4, 4, 9, bc={"z0": W.CONTACT})
    v = np.zeros((3, m.n_cells))
    v[2] = -0.1
    gap, eps = 0.15, 0.125
    planes = np.array([[0.0, 0.0, -gap, 0.0, 0.0, 1.0]])
    pb = W.Problem("drop3d", m, 1.0, 2.0, np.full(m.n_cells, 1.0), v, 0.25, 10, contact=(planes, eps))
    o = O.Oracle(pb)
    mass = o.get(O.F_MASS)
    E0 = (mass * o.get(O.F_E)).sum()
    touched = False
    pz = []
    for _ in range(200):
        o.step()
        z = o.get(O.F_X)[2]
        assert (z + gap).min() >= eps - 0.1 * o.dt - 1e-15
        assert abs((mass * o.get(O.F_E)).sum() - E0) <= 1e-14 * E0
        touched = touched or (z + gap).min() < eps
        pz.append((mass * o.get(O.F_V)[2]).sum() / mass.sum())
    assert touched
    # rebounded and detached: upward, constant momentum in the last steps
    assert min(pz[-25:]) > 0.3 * 0.1
    assert max(pz[-25:]) - min(pz[-25:]) <= 1e-13 * max(pz[-25:])


def _face_vectors_3d(m, x):
    """outward area vector of every boundary triangle at positions x [3, np] (orientation from
    the tetrahedron on the face's inner side)"""
    c2n = m.c2n.T
    out = np.zeros((m.bface.shape[1], 3))
    for i, (q0, q1, q2) in enumerate(m.bface.T):
        N = 0.5 * np.cross(x[:, q1] - x[:, q0], x[:, q2] - x[:, q0])
        cell = np.where(np.isin(c2n, [q0, q1, q2]).sum(axis=1) == 3)[0][0]
        opp = [q for q in c2n[cell] if q not in (q0, q1, q2)][0]
        if N @ (x[:, q0] - x[:, opp]) < 0:
            N = -N
        out[i] = N
    return out


def test_pressure_and_traction_in_3d():
    """3D counterparts of the 2D pins: a block under F = s I held by the pressure -sigma on all
    six sides stays at rest; a free block at rest under random face tractions gains the momentum
    dt sum_f |N_f| t_f and the energy dt sum_p F_p . v*_p (F_p the nodes' thirds of the faces
    around them) in one step."""
    s = 0.97
    kappa = 2.0 + 2.0 / 3.0
    sigma = O.stress(s * np.eye(3), 1.0, kappa)[0, 0]
    sides = ("x0", "x1", "y0", "y1", "z0", "z1")
    m = W.tet_mesh(3, 3, 3, 5, bc={k: W.PRESSURE for k in sides})
    F = np.tile((s * np.eye(3)).reshape(9, 1), (1, m.n_cells))
    pb = W.Problem("block3d", m, 1.0, 2.0, np.full(m.n_cells, 1.0), np.zeros((3, m.n_cells)), 0.25, 5, F=F,
                   bcval=W.side_values(m, W.PRESSURE, (-sigma, 0.0, 0.0)))
    o = O.Oracle(pb)
    for _ in range(4):
        o.step()
    assert np.abs(o.get(O.F_V)).max() < 1e-13 and np.abs(o.get(O.F_VP)).max() < 1e-13

    m = W.tet_mesh(3, 3, 3, 6, bc={k: W.TRACTION for k in sides})
    t = np.random.default_rng(7).normal(size=(3, m.btag.size)) * 0.01
    pb = W.Problem("free3d", m, 1.0, 2.0, np.full(m.n_cells, 1.0), np.zeros((3, m.n_cells)), 0.25, 5, bcval=t)
    o = O.Oracle(pb)
    x0, mass, e0, dt = o.get(O.F_X).copy(), o.get(O.F_MASS), o.get(O.F_E).copy(), o.dt
    o.step()
    Nf = _face_vectors_3d(m, x0)
    area = np.linalg.norm(Nf, axis=1)
    np.testing.assert_allclose((mass[None, :] * o.get(O.F_V)).sum(axis=1), dt * (area[None, :] * t).sum(axis=1),
                               rtol=1e-12, atol=1e-16)
    Fp = np.zeros_like(x0)
    for i, q in enumerate(m.bface.T):
        for p in q:
            Fp[:, p] += area[i] * t[:, i] / 3
    work = dt * (Fp * o.get(O.F_VSTAR)).sum()
    assert abs((mass * (o.get(O.F_E) - e0)).sum() - work) <= 1e-12 * abs(work)
