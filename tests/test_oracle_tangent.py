"""The oracle's tangent build (lmood_tangent.cpp: the oracle's source compiled with dual numbers)
as a CPU reference derivative of the step map (CPU).

Pins: its value parts are bitwise those of the plain oracle (the same source, the same
operations); its derivative parts equal central differences of the plain oracle's n-step map
(step 1e-6, masks of the perturbed runs checked equal to the tangent run's, dt fixed so that
the differenced map is the frozen-dt map the tangent differentiates) to 1e-6 relative, in 2D
and 3D, with MOOD active and first-order cells in the mask, for directions of v0, mu and F0;
and they are linear in the direction. With traction, pressure and prescribed-velocity faces
and contact walls (the piston, the block rebounding on a wall, a block under pressure and
traction, a 3D box with every kind of face) the same holds for directions of v0, mu, F0 and
of the initial node positions at fixed masses (central differences of the tangent build's
values from displaced starts), checked per output field.
"""
import dataclasses

import numpy as np
import pytest

import workloads as W
from adjoint_cases import bc_case, sg_case, smooth_positions_direction

FIELDS = ("x", "vp", "v", "F")


def _case(name):
    if name == "plain2d":
        pb = W.plain2d(n=10)
        pb.v *= 40.0
        return pb
    if name == "impact2d":
        return W.impact2d(n=14)
    pb = W.cube3d(n=3)
    pb.v *= 6.0
    return pb


def _with_F(pb, rng):
    d, nc = pb.mesh.dim, pb.mesh.n_cells
    F = np.zeros((d * d, nc))
    for a in range(d):
        F[a * d + a] = 1.0
    F += 0.01 * rng.standard_normal((d * d, nc))
    mu = np.asarray(pb.mu, dtype=float) * (1.0 + 0.1 * rng.random(nc))
    return dataclasses.replace(pb, F=F, mu=mu)


def _plain(orc, pb, n, **prm):
    o = orc.Oracle(pb, **prm)
    masks = []
    for _ in range(n):
        o.step()
        masks.append(o.get(orc.F_ORDER).astype(np.int8))
    return {"x": o.get(orc.F_X), "vp": o.get(orc.F_VP), "v": o.get(orc.F_V), "F": o.get(orc.F_F)}, masks


@pytest.mark.parametrize("name", ["plain2d", "impact2d", "cube3d"])
def test_tangent_values_are_the_oracle(orc, name):
    pb = _with_F(_case(name), np.random.default_rng(3))
    n = 6
    rng = np.random.default_rng(4)
    t = orc.tangent(pb, n, dv=rng.standard_normal(pb.v.shape))
    ref, masks = _plain(orc, pb, n)
    for k in FIELDS:
        assert np.array_equal(t[k], ref[k]), k
    for s in range(n):
        assert np.array_equal(t["masks"][s], masks[s]), s
    assert (t["masks"] == 1).any(), "no first-order cell in the run"


@pytest.mark.parametrize("name", ["plain2d", "impact2d", "cube3d"])
def test_tangent_against_central_differences(orc, name):
    rng = np.random.default_rng(11)
    pb = _with_F(_case(name), rng)
    n = 5
    d, nc, npn = pb.mesh.dim, pb.mesh.n_cells, pb.mesh.n_nodes
    dt = 0.5 * orc.Oracle(pb).dt
    prm = {"dt_fixed": dt}
    lam = {"x": rng.standard_normal((d, npn)), "vp": rng.standard_normal((d, npn)),
           "v": rng.standard_normal((d, nc)), "F": rng.standard_normal((d * d, nc))}
    dirs = {"v": rng.standard_normal((d, nc)), "mu": rng.standard_normal(nc) * pb.mu,
            "F": rng.standard_normal((d * d, nc))}
    h = 1e-6
    for name_dir, delta in dirs.items():
        t = orc.tangent(pb, n, **{"d" + name_dir: delta}, **prm)
        assert (t["masks"] == 1).any() and (t["masks"] == 2).any(), "the mask must mix P1 and P0 cells"
        ad = sum(float((t["d" + k] * lam[k]).sum()) for k in FIELDS)
        runs = []
        for sgn in (1.0, -1.0):
            base = {"v": pb.v, "mu": pb.mu, "F": pb.F}[name_dir]
            st, masks = _plain(orc, dataclasses.replace(pb, **{name_dir: base + sgn * h * delta}), n, **prm)
            for s in range(n):
                assert np.array_equal(masks[s], t["masks"][s]), f"mask changed under the perturbation at step {s}"
            runs.append(st)
        fd = sum(float(((runs[0][k] - runs[1][k]) * lam[k]).sum()) for k in FIELDS) / (2 * h)
        assert abs(ad - fd) <= 1e-6 * max(abs(ad), abs(fd)), (name_dir, ad, fd)


def test_tangent_is_linear_in_the_direction(orc):
    rng = np.random.default_rng(5)
    pb = _with_F(_case("cube3d"), rng)
    a, b = rng.standard_normal(pb.v.shape), rng.standard_normal(pb.v.shape)
    ta, tb = orc.tangent(pb, 4, dv=a), orc.tangent(pb, 4, dv=b)
    tab = orc.tangent(pb, 4, dv=a + b)
    for k in FIELDS:
        np.testing.assert_allclose(tab["d" + k], ta["d" + k] + tb["d" + k], rtol=0,
                                   atol=1e-11 * np.abs(tab["d" + k]).max())
    t0 = orc.tangent(pb, 4)
    for k in FIELDS:
        assert not np.any(t0["d" + k]), k


@pytest.mark.parametrize("name", ["piston2d", "rebound2d", "pressure_traction2d", "box3d_bc", "blake_needle"])
def test_tangent_with_boundary_faces_against_central_differences(orc, name):
    """traction, pressure and prescribed-velocity faces and contact walls (their multiplier
    steps differentiated with the contact set frozen), slip walls in oblique planes (Blake's
    needle at rest under its pressure, with the unlimited scheme: its first steps put cells at
    the detection thresholds, where a perturbation changes the mask), and a direction of the
    initial node positions at fixed masses (central differences of the tangent build's values
    from displaced starts)"""
    rng = np.random.default_rng(17)
    pb = bc_case(name)
    d, nc, npn = pb.mesh.dim, pb.mesh.n_cells, pb.mesh.n_nodes
    pb = dataclasses.replace(pb, mu=np.asarray(pb.mu, dtype=float) * (1.0 + 0.1 * rng.random(nc)),
                             F=np.tile(np.eye(d).ravel()[:, None], (1, nc)))
    n = 5
    prm = {"dt_fixed": 0.5 * orc.Oracle(pb).dt}
    if name == "blake_needle":
        prm["mood"] = 0
    lam = {"x": rng.standard_normal((d, npn)), "vp": rng.standard_normal((d, npn)),
           "v": rng.standard_normal((d, nc)), "F": rng.standard_normal((d * d, nc))}
    dirs = {"v": rng.standard_normal((d, nc)), "mu": rng.standard_normal(nc) * pb.mu,
            "F": rng.standard_normal((d * d, nc)), "x": smooth_positions_direction(pb.mesh)}
    for name_dir, delta in dirs.items():
        h = 1e-5  # (these small runs are weakly sensitive to some directions: a larger step keeps rounding small)
        if name == "blake_needle" and name_dir == "F":
            h = 1e-6  # strongly curved in F at 2 % strain: the difference's h^2 error is 3e-6 at 1e-5, 3e-8 here
        t = orc.tangent(pb, n, **{"d" + name_dir: delta}, **prm)
        ad = {k: float((t["d" + k] * lam[k]).sum()) for k in FIELDS}
        runs = []
        for sgn in (1.0, -1.0):
            if name_dir == "x":
                r = orc.tangent(pb, n, dx=delta, x_shift=sgn * h, **prm)
                st, masks = {k: r[k] for k in FIELDS}, list(r["masks"])
            else:
                base = {"v": pb.v, "mu": pb.mu, "F": pb.F}[name_dir]
                st, masks = _plain(orc, dataclasses.replace(pb, **{name_dir: base + sgn * h * delta}), n, **prm)
            for s in range(n):
                assert np.array_equal(masks[s], t["masks"][s]), f"mask changed under the perturbation at step {s}"
            runs.append(st)
        # per output field (their sum cancels in part, and the rounding of the differenced runs
        # is relative to the largest of them)
        fd = {k: float(((runs[0][k] - runs[1][k]) * lam[k]).sum()) / (2 * h) for k in FIELDS}
        scale = max(abs(v) for v in ad.values())
        for k in FIELDS:
            assert abs(ad[k] - fd[k]) <= 1e-6 * scale, (name, name_dir, k, ad[k], fd[k])


@pytest.mark.parametrize("name", ["sgwave2d", "sgdrop3d"])
def test_tangent_stiffened_gas_against_central_differences(orc, name):
    """the stiffened gas, whose pressure depends on the internal energy: the derivative of the
    final (x, v_p, v, F, e) along directions of v0, mu, F0 and of the initial positions"""
    rng = np.random.default_rng(23)
    pb = sg_case(name)
    d, nc, npn = pb.mesh.dim, pb.mesh.n_cells, pb.mesh.n_nodes
    pb = dataclasses.replace(pb, mu=np.asarray(pb.mu, dtype=float) * (1.0 + 0.1 * rng.random(nc)),
                             F=np.tile(np.eye(d).ravel()[:, None], (1, nc)))
    n = 4
    prm = {"dt_fixed": 0.5 * orc.Oracle(pb).dt}
    fields = FIELDS + ("e",)
    lam = {"x": rng.standard_normal((d, npn)), "vp": rng.standard_normal((d, npn)),
           "v": rng.standard_normal((d, nc)), "F": rng.standard_normal((d * d, nc)), "e": rng.standard_normal(nc)}
    dirs = {"v": rng.standard_normal((d, nc)), "mu": rng.standard_normal(nc) * pb.mu,
            "F": 0.1 * rng.standard_normal((d * d, nc)), "x": 0.1 * smooth_positions_direction(pb.mesh)}
    h = 1e-5  # (the rounding of the differenced runs dominates at 1e-6 for the weaker directions)
    for name_dir, delta in dirs.items():
        t = orc.tangent(pb, n, **{"d" + name_dir: delta}, **prm)
        ad = {k: float((t["d" + k] * lam[k]).sum()) for k in fields}
        runs = []
        for sgn in (1.0, -1.0):
            if name_dir == "x":
                r = orc.tangent(pb, n, dx=delta, x_shift=sgn * h, **prm)
            else:
                base = {"v": pb.v, "mu": pb.mu, "F": pb.F}[name_dir]
                r = orc.tangent(dataclasses.replace(pb, **{name_dir: base + sgn * h * delta}), n, **prm)
            for s in range(n):
                assert np.array_equal(r["masks"][s], t["masks"][s]), f"mask changed under the perturbation at step {s}"
            runs.append(r)
        fd = {k: float(((runs[0][k] - runs[1][k]) * lam[k]).sum()) / (2 * h) for k in fields}
        scale = max(abs(v) for v in ad.values())
        for k in fields:
            assert abs(ad[k] - fd[k]) <= 1e-6 * scale, (name, name_dir, k, ad[k], fd[k])


def test_tangent_position_direction_at_rest_shift_is_the_oracle(orc):
    """x_shift = 0 with a position direction leaves the values those of the plain oracle (the
    initial nodal solve done again at the same positions gives the same v_p^0)"""
    pb = bc_case("piston2d")
    rng = np.random.default_rng(20)
    t = orc.tangent(pb, 4, dx=rng.standard_normal((pb.mesh.dim, pb.mesh.n_nodes)))
    ref, _ = _plain(orc, pb, 4)
    for k in FIELDS:
        assert np.array_equal(t[k], ref[k]), k
