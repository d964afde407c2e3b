"""Pins of the oracle's full step: conservation, GCL, invariance, nodal balance, exactness on
affine fields, observed second order on the swinging plate (and the paper's error table),
first order of the parachute scheme, MOOD behaviour under an injected fault."""
import math
import os
import subprocess
import sys

import numpy as np
import pytest

import workloads as W


def _geom_all(orc, x, c2n):
    """(V, ln) of every cell at positions x [d, np] from the oracle's unit geometry."""
    d = x.shape[0]
    nc = c2n.shape[1]
    V = np.zeros(nc)
    ln = np.zeros((nc, d + 1, d))
    for c in range(nc):
        V[c], _, _, ln[c], _ = orc.cell_geometry(x[:, c2n[:, c]].T)
    return V, ln


def _totals(o, orc):
    m = o.get(orc.F_MASS)
    return (m * o.get(orc.F_E)).sum(), (m * o.get(orc.F_V)).sum(axis=1)


# ----------------------------------------------------------------------------- GCL / mass
@pytest.mark.parametrize("d", [2, 3])
def test_gcl(orc, d):
    """V^{n+1} - V^n = dt sum_p l n (x^{n+1/2}) . v*_p exactly in 2D (area is quadratic in x);
    in 3D with Simpson's rule in time (volume is cubic). tau^{n+1} m_c = V(x^{n+1})."""
    pb = W.plain2d(n=10) if d == 2 else W.cube3d(n=3)
    pb.v *= 40.0  # visible motion
    o = orc.Oracle(pb, mood=0)
    m = o.get(orc.F_MASS)
    c2n = pb.mesh.c2n
    for _ in range(3):
        x0 = o.get(orc.F_X)
        V0 = o.get(orc.F_TAU) * m
        dt = o.dt
        o.step()
        x1 = o.get(orc.F_X)
        vs = o.get(orc.F_VSTAR)
        V1 = o.get(orc.F_TAU) * m
        np.testing.assert_allclose(_geom_all(orc, x1, c2n)[0], V1, rtol=1e-15)
        vsc = vs[:, c2n]                                   # [d, nv, nc]
        flux = lambda ln: np.einsum("cka,akc->c", ln, vsc)
        if d == 2:
            rhs = dt * flux(_geom_all(orc, 0.5 * (x0 + x1), c2n)[1])
        else:
            rhs = dt * (flux(_geom_all(orc, x0, c2n)[1]) + 4 * flux(_geom_all(orc, 0.5 * (x0 + x1), c2n)[1])
                        + flux(_geom_all(orc, x1, c2n)[1])) / 6
        np.testing.assert_allclose(V1 - V0, rhs, rtol=0, atol=1e-13 * V0.max())
        assert np.abs(V1 - V0).max() > 1e-9 * V0.max()    # the mesh did move


# ----------------------------------------------------------------------------- conservation
@pytest.mark.parametrize("case", ["slip2d", "free2d", "clamped3d", "slip3d"])
def test_energy_conservation(orc, case):
    """Total energy sum m e is conserved to round-off with free, slip and clamped nodes:
    sum_c f_cp . v*_p vanishes node by node (Eq. sum_fcp with the BC projections)."""
    if case == "slip2d":
        pb = W.plain2d(n=14); pb.v *= 50
    elif case == "free2d":
        pb = W.impact2d(n=14)
        pb.mesh.btag[:] = W.FREE
    elif case == "clamped3d":
        pb = W.column3d(nxy=2, nz=6)
        pb.v *= 5
    else:
        pb = W.cube3d(n=3); pb.v *= 5
    o = orc.Oracle(pb)
    E0, _ = _totals(o, orc)
    for _ in range(5):
        o.step()
    E1, _ = _totals(o, orc)
    assert abs(E1 - E0) <= 1e-14 * abs(E0) * 10


@pytest.mark.parametrize("d", [2, 3])
def test_momentum_conservation_free(orc, d):
    """With traction-free boundaries sum_c f_cp = 0 at every node, so sum m v is conserved."""
    pb = W.plain2d(n=12) if d == 2 else W.cube3d(n=3)
    pb.mesh.btag[:] = W.FREE
    pb.v *= 30
    o = orc.Oracle(pb)
    _, P0 = _totals(o, orc)
    scale = (o.get(orc.F_MASS) * np.abs(o.get(orc.F_V)).max()).sum()
    for _ in range(5):
        o.step()
    _, P1 = _totals(o, orc)
    np.testing.assert_allclose(P1, P0, rtol=0, atol=1e-15 * scale * 10)


# ----------------------------------------------------------------------------- invariance
@pytest.mark.parametrize("d", [2, 3])
def test_uniform_translation(orc, d):
    pb = W.plain2d(n=9) if d == 2 else W.cube3d(n=2)
    pb.mesh.btag[:] = W.FREE
    vel = np.array([0.3, -0.2, 0.1][:d])
    pb.v = np.repeat(vel[:, None], pb.mesh.n_cells, axis=1)
    o = orc.Oracle(pb)
    x0 = o.get(orc.F_X)
    for _ in range(4):
        o.step()
    np.testing.assert_allclose(o.get(orc.F_V), pb.v, rtol=0, atol=1e-15)
    np.testing.assert_allclose(o.get(orc.F_X), x0 + o.t * vel[:, None], rtol=0, atol=1e-14)
    F = o.get(orc.F_F)
    np.testing.assert_allclose(F, np.eye(d).reshape(-1, 1) * np.ones((1, F.shape[1])), rtol=0, atol=1e-15)
    assert o.info.n_troubled == 0


@pytest.mark.parametrize("d", [2, 3])
def test_rotation_objectivity(orc, d):
    """step(R problem) = R step(problem): x -> R x, v -> R v, F -> R F R^t, e and tau unchanged
    (slip walls rotate with the body)."""
    pb = W.plain2d(n=10) if d == 2 else W.cube3d(n=3)
    pb.v *= 30
    rng = np.random.default_rng(2)
    if d == 2:
        th = 0.7
        R = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    else:
        R, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        if np.linalg.det(R) < 0:
            R[:, 0] *= -1
    pr = W.translate_rotate(pb, R, np.arange(1, d + 1) * 0.5)
    a, b = orc.Oracle(pb, mood=0), orc.Oracle(pr, mood=0)
    a.step(3)
    b.step(3)
    sa, sb = a.state(), b.state()
    np.testing.assert_allclose(sb["v"], R @ sa["v"], atol=1e-12 * np.abs(sa["v"]).max())
    np.testing.assert_allclose(sb["x"], R @ sa["x"] + np.arange(1, d + 1)[:, None] * 0.5, atol=1e-13)
    Fa = sa["F"].T.reshape(-1, d, d)
    Fb = sb["F"].T.reshape(-1, d, d)
    np.testing.assert_allclose(Fb, R @ Fa @ R.T, atol=1e-12)
    np.testing.assert_allclose(sb["e"], sa["e"], rtol=1e-9, atol=1e-12 * np.abs(sa["e"]).max())
    np.testing.assert_allclose(sb["tau"], sa["tau"], rtol=1e-12)


# ----------------------------------------------------------------------------- nodal solver
def test_nodal_balance_and_bcs(orc):
    """After a step, node by node: M_p SPD; free nodes: M_p v*_p = b_p (so sum_c f_cp = 0);
    slip nodes: zero normal velocity and zero tangential residual; clamped: v* = 0."""
    for pb in (W.impact2d(n=12), W.column3d(nxy=2, nz=4)):
        pb.v[:] *= 3
        o = orc.Oracle(pb)
        o.step()
        d = pb.mesh.dim
        nv = d + 1
        pkM = o.get(orc.F_PKM).reshape(d, d, nv, -1)
        pkR = o.get(orc.F_PKR)
        vs = o.get(orc.F_VSTAR)
        c2n = pb.mesh.c2n
        Mp = np.zeros((pb.mesh.n_nodes, d, d))
        bp = np.zeros((pb.mesh.n_nodes, d))
        for k in range(nv):
            np.add.at(Mp, c2n[k], pkM[:, :, k, :].transpose(2, 0, 1))
            np.add.at(bp, c2n[k], pkR[:, k, :].T)
        assert np.all(np.linalg.eigvalsh(Mp) > 0)
        res = np.einsum("pab,bp->pa", Mp, vs) - bp
        scale = np.abs(bp).max() + 1e-300
        for p in range(pb.mesh.n_nodes):
            ndof = o.bc_ndof(p)
            if ndof == d:
                assert np.abs(res[p]).max() <= 1e-12 * scale
            elif ndof == 0:
                assert np.all(vs[:, p] == 0)
        if d == 2:  # slip wall x = 0: exactly zero normal velocity, tangential residual zero
            wall = np.where(pb.mesh.x[0] == 0.0)[0]
            assert wall.size and np.all(vs[0, wall] == 0.0)
            assert np.abs(res[wall, 1]).max() <= 1e-12 * scale


# ----------------------------------------------------------------------------- reconstruction
@pytest.mark.parametrize("d", [2, 3])
def test_reconstruction_exact_on_affine_fields(orc, d):
    """Least-squares slopes reproduce an affine velocity exactly, so the predictor's corner
    value v*_cp = v_h(x_p) = G x_p + b (with F = I and a vanishing dt, T* = 0), recovered from
    the packet as M_cp^{-1} rhs_cp, in interior and boundary cells alike."""
    pb = W.plain2d(n=8) if d == 2 else W.cube3d(n=3)
    G = np.random.default_rng(4).normal(size=(d, d))
    b = np.arange(1, d + 1) * 0.1
    xc = W.cell_points(pb.mesh)
    pb.v = (xc @ G.T + b).T.copy()
    o = orc.Oracle(pb, mood=0, dt_fixed=1e-30)
    o.step()
    nv = d + 1
    pkM = o.get(orc.F_PKM).reshape(d, d, nv, -1)
    pkR = o.get(orc.F_PKR)
    x = pb.mesh.x
    for k in range(nv):
        Mk = pkM[:, :, k, :].transpose(2, 0, 1)
        vstar = np.linalg.solve(Mk, pkR[:, k, :].T[..., None])[..., 0]
        xp = x[:, pb.mesh.c2n[k]].T
        np.testing.assert_allclose(vstar, xp @ G.T + b, rtol=0, atol=1e-12)


def test_first_order_F_update_is_mesh_deformation(orc):
    """P0 cells: F^{n+1} = (I + dt L*) F^n with L* the velocity gradient of v*_p on x^n
    (Eqs. div_grad_v, firstB). From F = I this is exactly the deformation gradient of the
    cell's affine map x^n -> x^{n+1}; a transposed L (the printed ln (x) v) fails."""
    for pb in (W.plain2d(n=9), W.cube3d(n=2)):
        d = pb.mesh.dim
        pb.v *= 100
        o = orc.Oracle(pb, order=1)
        x0 = o.get(orc.F_X)
        o.step()
        x1 = o.get(orc.F_X)
        F = o.get(orc.F_F).T.reshape(-1, d, d)
        c2n = pb.mesh.c2n
        E0 = (x0[:, c2n[1:]] - x0[:, c2n[:1]]).transpose(2, 0, 1)   # columns = edge vectors
        E1 = (x1[:, c2n[1:]] - x1[:, c2n[:1]]).transpose(2, 0, 1)
        Fgeo = E1 @ np.linalg.inv(E0)
        np.testing.assert_allclose(F, Fgeo, rtol=0, atol=1e-13)
        assert np.abs(Fgeo - np.eye(d)).max() > 1e-8


# ----------------------------------------------------------------------------- order of accuracy
def _plate_error(orc, n, order):
    pb = W.swinging_plate(n, jitter=0.25)
    o0 = orc.Oracle(pb, mood=0)
    dt0 = o0.dt
    o0.close()
    tf = pb.meta["t_final"]
    ns = int(math.ceil(tf / dt0))
    o = orc.Oracle(pb, mood=0, order=order, dt_fixed=tf / ns)
    o.step(ns)
    s = o.state()
    xc = s["x"][:, pb.mesh.c2n].mean(axis=1)
    V = s["tau"] * o.get(orc.F_MASS)
    a, om = pb.meta["amp"], pb.meta["omega"]
    uex = a * math.cos(om * o.t) * (-np.sin(0.5 * np.pi * xc[0]) * np.cos(0.5 * np.pi * xc[1]))
    eu = math.sqrt((V * (s["v"][0] - uex) ** 2).sum())
    F = s["F"]
    eB = math.sqrt((V * (F[0] ** 2 + F[1] ** 2 - 1.0) ** 2).sum())
    # in-sphere diameters at t_final
    Lc = np.array([orc.cell_geometry(s["x"][:, pb.mesh.c2n[:, c]].T)[4] for c in range(pb.mesh.n_cells)])
    return eu, eB, Lc.mean()


def test_swinging_plate_order_and_magnitude(orc):
    """Sect. "2D swinging plate": observed order of eps(u) and eps(B11) at t_final >= 1.8 on the
    two finest meshes for the second-order scheme (the paper's table shows 1.82-2.06), about 1
    for the first-order parachute scheme; and eps(u) within a factor 3 of the paper's table
    interpolated at the same in-sphere diameter (golden values in tests/golden)."""
    res2 = [_plate_error(orc, n, 2) for n in (17, 33, 65)]
    o_u = math.log(res2[1][0] / res2[2][0]) / math.log(res2[1][2] / res2[2][2])
    o_B = math.log(res2[1][1] / res2[2][1]) / math.log(res2[1][2] / res2[2][2])
    assert o_u >= 1.8 and o_B >= 1.8, (res2, o_u, o_B)
    res1 = [_plate_error(orc, n, 1) for n in (17, 33)]
    o1 = math.log(res1[0][0] / res1[1][0]) / math.log(res1[0][2] / res1[1][2])
    assert o1 < 1.3 and res1[1][0] > 5 * res2[1][0], (res1, o1)
    tab = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", "swinging_plate_table.txt"))
    for eu, _, Lc in res2[:2]:
        ref = math.exp(np.interp(math.log(Lc), np.log(tab[::-1, 0]), np.log(tab[::-1, 1]),
                                 left=np.nan, right=np.nan))
        if not math.isnan(ref):
            assert ref / 3 < eu < 3 * ref, (eu, ref, Lc)


def _cube_error(orc, n, order):
    """L2 error of the cell velocities at t_final = pi / omega (half a period) on the swinging
    cube, fixed dt from the acoustic dt of the initial state, unlimited scheme"""
    pb = W.swinging_cube(n)
    o0 = orc.Oracle(pb, mood=0)
    dt0 = o0.dt
    o0.close()
    tf = pb.meta["t_final"]
    ns = int(math.ceil(tf / dt0))
    o = orc.Oracle(pb, mood=0, order=order, dt_fixed=tf / ns)
    o.step(ns)
    s = o.state()
    xc = s["x"][:, pb.mesh.c2n].mean(axis=1)
    V = s["tau"] * o.get(orc.F_MASS)
    k, a, om = pb.meta["k"], pb.meta["amp"], pb.meta["omega"]
    sn, cs = np.sin(k * xc), np.cos(k * xc)
    vex = a * math.cos(om * o.t) * np.stack([sn[0] * cs[1] * cs[2], -cs[0] * sn[1] * cs[2], 0.0 * sn[0]])
    o.close()
    return math.sqrt((V * ((s["v"] - vex) ** 2).sum(axis=0)).sum())


@pytest.mark.slow
def test_swinging_cube_order(orc):
    """The whole 3D scheme on a smooth standing shear wave with slip walls (the swinging plate's
    3D counterpart, exact solution v = omega U0 cos(omega t) U(x)): the observed order of the
    velocity error on 8^3 -> 16^3 cubes (3,072 -> 24,576 tets) is >= 1.65 and above the order on
    4^3 -> 8^3 (1.05 -> 1.74 measured: still rising toward 2 at these sizes); the first-order
    scheme's error on 8^3 cubes is far larger (the wave is nearly damped out)."""
    e = [_cube_error(orc, n, 2) for n in (4, 8, 16)]
    o1, o2 = math.log2(e[0] / e[1]), math.log2(e[1] / e[2])
    assert o2 >= 1.65 and o2 > o1 + 0.3, (e, o1, o2)
    assert _cube_error(orc, 8, 1) > 1.5 * e[1]


# ----------------------------------------------------------------------------- MOOD
def test_mood_injected_fault(orc):
    """A resting block with one cell kicked hard: the candidate violates the RDMP around it,
    those cells drop to P0, nothing far away does, and energy stays conserved."""
    pb = W.plain2d(n=16)
    pb.v[:] = 0.0
    xc = W.cell_points(pb.mesh)
    c0 = int(np.argmin(((xc - 0.5) ** 2).sum(axis=1)))
    pb.v[0, c0] = 0.5
    o = orc.Oracle(pb)
    E0, _ = _totals(o, orc)
    o.step()
    order = o.get(orc.F_ORDER)
    bad = np.where(order == 1)[0]
    assert o.info.n_troubled >= 1 and c0 in bad
    assert np.sqrt(((xc[bad] - xc[c0]) ** 2).sum(axis=1)).max() < 0.25
    E1, _ = _totals(o, orc)
    assert abs(E1 - E0) <= 1e-13 * E0
    # unlimited P1 on the same data yields a candidate the detector rejects
    u = orc.Oracle(pb, mood=0)
    u.step()
    assert u.info.n_troubled == 0


def test_parachute_first_order_has_no_troubled_cells(orc):
    pb = W.impact2d(n=20)
    o = orc.Oracle(pb, order=1)
    o.step(5)
    assert o.info.n_troubled == 0 and o.info.n_p0 == pb.mesh.n_cells


def test_parachute_failure_leaves_the_state(orc):
    """a cell whose first-order candidate cannot be computed (Sect. "Limiting: a posteriori MOOD
    loop": the parachute scheme must produce an admissible state): a NaN velocity, or an
    inverted F (det F < 0) that the first-order update keeps inverted; the step reports the
    parachute failure and leaves the state and the time as they were, and the oracle stays
    usable: from the clean state it steps as a fresh run does"""
    pb = W.plain2d(n=12)
    clean = orc.Oracle(pb)
    clean.step(2)
    s0, t0, dt0 = clean.state(), clean.t, clean.dt
    clean.step()
    ref = clean.state()
    for field, bad in (("v", lambda a: a.__setitem__((0, 5), np.nan)),
                       ("F", lambda a: a.__setitem__((slice(0, 1), 7), -a[0, 7]))):
        o = orc.Oracle(pb)
        o.step(2)
        arr = o.state()[field].copy()
        bad(arr)
        o.set_state(**{field: arr})
        before = o.state()
        rc = o.step(check=False)
        assert orc.ERR[rc] == "parachute failure" and o.info.n_parachute >= 1, (field, rc)
        after = o.state()
        for k in before:
            assert np.array_equal(after[k], before[k], equal_nan=True), (field, k)
        assert o.t == t0
        o.set_state(x=s0["x"], vp=s0["vp"], v=s0["v"], e=s0["e"], F=s0["F"], dt=dt0)
        o.step()
        for k in ref:
            assert np.array_equal(o.state()[k], ref[k]), (field, k)


# ----------------------------------------------------------------------------- time step
def test_dt_rules(orc):
    """dt^0 = C_CFL min L_c/a_c with a = sqrt((lambda + 2 mu)/rho0) at rest (Eq. CFL2);
    dt^{n+1} <= (1 + C_i) dt^n."""
    pb = W.impact2d(n=12)
    o = orc.Oracle(pb)
    x = pb.mesh.x
    Lc = np.array([orc.cell_geometry(x[:, pb.mesh.c2n[:, c]].T)[4] for c in range(pb.mesh.n_cells)])
    a = math.sqrt((pb.lam + 2 * pb.mu[0]) / pb.rho0)
    assert o.dt == pytest.approx(0.4 * Lc.min() / a, rel=1e-14)
    for _ in range(4):
        dt = o.dt
        o.step()
        assert o.dt <= 1.1 * dt * (1 + 1e-15)


def test_thread_count_independence(orc):
    code = ("import sys, hashlib; sys.path.insert(0, %r); import numpy as np, oracle as O, workloads as W;"
            "pb = W.impact2d(n=24); o = O.Oracle(pb); o.step(6); s = o.state();"
            "h = hashlib.sha256(); [h.update(a.tobytes()) for a in s.values()];"
            "sys.stdout.write(h.hexdigest())") % os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    outs = []
    for nt in ("1", "3"):
        env = dict(os.environ, OMP_NUM_THREADS=nt)
        outs.append(subprocess.check_output([sys.executable, "-c", code], env=env))
    assert outs[0] == outs[1]


# ----------------------------------------------------------------------------- BJ level
def test_barth_jespersen_bounds_and_linear_preservation(orc):
    """Level 3 (Barth-Jespersen slopes, Sect. "Limiting: a posteriori MOOD loop"): the
    reconstructed values at a cell's nodes stay within the field's range over the stencil and
    the cell; on an affine field interior cells keep the unlimited (exact) reconstruction."""
    pb = W.impact2d(n=40)
    o = orc.Oracle(pb)
    o.step(8)   # a state with a compression front
    rng = np.random.default_rng(3)
    for c in rng.choice(pb.mesh.n_cells, 200, replace=False):
        vals, lo, hi = o.corner_values(int(c), 3)
        span = np.maximum(hi - lo, 1e-300)
        assert np.all(vals >= lo - 1e-12 * span) and np.all(vals <= hi + 1e-12 * span)
    # affine velocity field, F = I: interior cells unchanged by the limiter
    pb = W.plain2d(n=12)
    G = np.array([[0.3, -0.2], [0.1, 0.4]])
    xc = W.cell_points(pb.mesh)
    pb.v = (xc @ G.T).T.copy()
    o = orc.Oracle(pb)
    bnd = set(pb.mesh.bface.ravel().tolist())
    for c in range(pb.mesh.n_cells):
        if any(int(p) in bnd for p in pb.mesh.c2n[:, c]):
            continue
        v2, _, _ = o.corner_values(c, 2)
        v3, _, _ = o.corner_values(c, 3)
        np.testing.assert_allclose(v3, v2, rtol=0, atol=1e-15)


def test_three_level_cascade(orc):
    """With the three-level cascade, troubled P1 cells first try the limited scheme; fewer
    cells end at first order than with P1 -> P0, energy is still conserved."""
    pb = W.impact2d(n=60)
    res = {}
    for cas in (2, 3):
        o = orc.Oracle(pb, cascade=cas)
        E0, _ = _totals(o, orc)
        for _ in range(20):
            o.step()
        E1, _ = _totals(o, orc)
        assert abs(E1 - E0) <= 1e-13 * E0
        order = o.get(orc.F_ORDER)
        res[cas] = (int((order == 1).sum()), int((order == 3).sum()))
    assert res[2][1] == 0 and res[3][1] > 0 and res[3][0] < res[2][0]


# ----------------------------------------------------------------------------- entropy
def _thermal(o, orc, pb):
    """specific internal energy not stored elastically, e - |v|^2/2 - Psi(F) (theta d eta)"""
    d = pb.mesh.dim
    v, e, F = o.get(orc.F_V), o.get(orc.F_E), o.get(orc.F_F)
    kap = pb.lam + 2.0 * pb.mu / 3.0
    psi = np.array([orc.free_energy(F[:, c].reshape(d, d), pb.rho0, pb.mu[c], kap[c]) for c in range(F.shape[1])])
    return e - 0.5 * (v * v).sum(axis=0) - psi


def _dissipation(o, orc, pb, v_n):
    """sum over the cell's corners of M_cp (v*_p - v_c) . (v*_p - v_c), v_c at t^n"""
    d, c2n = pb.mesh.dim, pb.mesh.c2n
    pk, vs = o.get(orc.F_PKM), o.get(orc.F_VSTAR)
    out = np.zeros(pb.mesh.n_cells)
    for c in range(pb.mesh.n_cells):
        for k in range(d + 1):
            w = vs[:, c2n[k, c]] - v_n[:, c]
            out[c] += w @ pk[:, k, c].reshape(d, d) @ w
    return out


@pytest.mark.parametrize("d", [2, 3])
def test_first_order_entropy_production(orc, d):
    """Sect. "Semi-discrete entropy analysis - Subcell force" (Eq. theta_deta_discr2): with the
    subcell force of the scheme, m_c theta_c d eta_c / dt = sum_p M_cp (v_p - v_c) . (v_p - v_c)
    >= 0, theta d eta being the change of e - |v|^2/2 - Psi(F). First-order steps from the same
    state: every cell's production is >= 0 (to rounding) at the CFL step, and its ratio to the
    right-hand side evaluated with the step's packets and v*_p tends to 1 linearly in dt. A sign
    error in M_cp, a stress inconsistent with Psi or a wrong energy update fails it."""
    pb = W.impact2d(n=16) if d == 2 else W.cube3d(n=4)
    if d == 3:
        pb.v *= 20
    o = orc.Oracle(pb, order=1, mood=0)
    o.step()  # a state with node velocities and a strained mesh
    st, dt0 = o.state(), o.dt
    errs = []
    for scale in (1.0, 0.1, 0.01):
        s = orc.Oracle(pb, order=1, mood=0, dt_fixed=dt0 * scale)
        s.set_state(x=st["x"], vp=st["vp"], v=st["v"], e=st["e"], F=st["F"], dt=dt0 * scale)
        h0, v_n, m = _thermal(s, orc, pb), s.get(orc.F_V).copy(), s.get(orc.F_MASS)
        s.step()
        dh = _thermal(s, orc, pb) - h0
        D = _dissipation(s, orc, pb, v_n) * (dt0 * scale) / m
        if scale == 1.0:
            assert dh.min() >= -1e-15 * np.abs(s.get(orc.F_E)).max()
            assert (m * dh).sum() > 0.0
        sel = D > 1e-3 * D.max()
        assert sel.sum() >= 20
        errs.append(np.abs(dh[sel] / D[sel] - 1.0).max())
    assert errs[1] < 0.05 and errs[2] < 0.005
    assert 5.0 < errs[1] / errs[2] < 20.0  # first order in dt


def test_slip_planes_in_3d_leave_their_intersection(orc):
    """Reading R14 on a cube with slip walls on all six faces: after a step a node on one wall
    has exactly zero velocity across it and moves freely along it (zero residual of the
    Galerkin solve in the wall's plane); a node on an edge (two walls) moves along the edge
    only; a corner node (three walls) does not move."""
    pb = W.cube3d(n=4)
    pb.v *= 20
    o = orc.Oracle(pb)
    o.step()
    d, nv = 3, 4
    x0 = pb.mesh.x
    pkM = o.get(orc.F_PKM).reshape(d, d, nv, -1)
    pkR = o.get(orc.F_PKR)
    vs = o.get(orc.F_VSTAR)
    Mp = np.zeros((pb.mesh.n_nodes, d, d))
    bp = np.zeros((pb.mesh.n_nodes, d))
    for k in range(nv):
        np.add.at(Mp, pb.mesh.c2n[k], pkM[:, :, k, :].transpose(2, 0, 1))
        np.add.at(bp, pb.mesh.c2n[k], pkR[:, k, :].T)
    res = np.einsum("pab,bp->pa", Mp, vs) - bp
    scale = np.abs(bp).max()
    on = (np.abs(x0) < 1e-14) | (np.abs(x0 - 1.0) < 1e-14)  # [3, np]: on the wall normal to axis a
    counts = {1: 0, 2: 0, 3: 0}
    for p in range(pb.mesh.n_nodes):
        walls = np.where(on[:, p])[0]
        if walls.size == 0:
            continue
        counts[walls.size] += 1
        assert np.all(vs[walls, p] == 0.0), (p, walls, vs[:, p])
        free = [a for a in range(d) if a not in walls]
        assert o.bc_ndof(p) == len(free)
        if free:
            assert np.abs(res[p, free]).max() <= 1e-12 * scale
            assert np.abs(vs[free, p]).max() > 0.0
    assert counts[1] > 0 and counts[2] > 0 and counts[3] == 8


def test_three_level_cascade_3d(orc):
    """The three-level cascade on tetrahedra: limited-slope cells appear, fewer cells end at first
    order than with P1 -> P0, and energy is conserved."""
    pb = W.column3d(nxy=4, nz=24)
    pb.v *= 5
    res = {}
    for cas in (2, 3):
        o = orc.Oracle(pb, cascade=cas)
        E0, _ = _totals(o, orc)
        for _ in range(10):
            o.step()
        E1, _ = _totals(o, orc)
        assert abs(E1 - E0) <= 1e-13 * abs(E0)
        order = o.get(orc.F_ORDER)
        res[cas] = (int((order == 1).sum()), int((order == 3).sum()))
    assert res[2][1] == 0 and res[3][1] > 0 and res[3][0] < res[2][0]
