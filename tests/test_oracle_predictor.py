"""Pins of the oracle's ADER predictor (reading R8: v*_cp = v_h(x_p) + dt/2 (1/m) sum_q
T(F_h(x_q)) (l n)_q, F*_cp = F_h(x_p) + dt/2 L^ F_c), independent of the step's other parts.

1. An exact solution it must reproduce to round-off: the homogeneous motion with constant
   particle velocities, x = (I + t L) F0 X (F(t) = (I + t L) F0 uniform, so the stress is
   uniform: no acceleration). From a state at t0 > 0 the corner values at t0 + dt/2 are
   v*_cp = L F0 X_p and F*_cp = (I + (t0 + dt/2) L) F0, on any mesh and in every cell. A dt
   in place of dt/2, a dropped dF/dt, a transposed L^ or F_c L^ in place of L^ F_c (L is not
   symmetric and F0 does not commute with it), or a normal of the wrong corner in the stress
   sum (the sum of a uniform T over the corners vanishes only with each corner's own l n_q)
   makes it fail.
2. Its local order on a smooth solution: small-amplitude plane P and S waves, where the
   neo-Hookean law reduces to linear elasticity with the Lame constants (lambda, mu), have the
   exact solution u = a_p sin(k.X - w_p t) k^ + a_s sin(k.X - w_s t) s^; the predicted corner
   values must approach v and F at (X_p, dt/2) at second order in h (dt proportional to h).
   A dropped or sign-flipped acceleration term, a dt in place of dt/2 or a dropped dF/dt leaves
   an O(dt) error (first order), and a normal of the wrong corner an O(1) one.
"""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W


@pytest.fixture(scope="module")
def orc():
    O.build()
    return O


def _mesh_problem(d, n, seed=3):
    """A jittered mesh of the unit square / cube with homogeneous material rho0 = 2.5, mu = 1,
    lambda = 2 (reference configuration X; rho0 != 1 so that mass and volume differ)."""
    if d == 2:
        pb = W.plain2d(n=n, seed=seed)
    else:
        pb = W.cube3d(n=n, seed=seed)
        h = 1.0 / n
        rng = np.random.default_rng(seed)
        pb.mesh.x = np.ascontiguousarray(pb.mesh.x + rng.uniform(-0.08 * h, 0.08 * h, pb.mesh.x.shape))
    pb.rho0 = 2.5
    pb.mu = np.ones(pb.mesh.n_cells)
    pb.v = np.zeros((d, pb.mesh.n_cells))
    return pb


def _corner_X(pb):
    """reference positions of every cell's corners, [nc][nv][d]"""
    return pb.mesh.x.T[pb.mesh.c2n.T]


@pytest.mark.parametrize("d", [2, 3])
def test_predictor_exact_on_homogeneous_motion(orc, d):
    pb = _mesh_problem(d, 8 if d == 2 else 3)
    L = np.array([[0.11, 0.23], [-0.17, 0.05]]) if d == 2 else \
        np.array([[0.11, 0.23, -0.07], [-0.17, 0.05, 0.13], [0.09, -0.21, 0.04]])
    # a constant pre-deformation that does not commute with L: x = (I + t L) F0 X
    F0 = np.array([[1.1, 0.2], [-0.1, 0.95]]) if d == 2 else \
        np.array([[1.1, 0.2, 0.05], [-0.1, 0.95, 0.15], [0.0, -0.12, 1.05]])
    assert np.abs(L @ F0 - F0 @ L).max() > 0.01
    t0, dt = 0.5, 0.02
    X = pb.mesh.x
    Ft = (np.eye(d) + t0 * L) @ F0
    Xc = W.cell_points(pb.mesh)            # cell vertex averages in X (the map is affine)
    o = orc.Oracle(pb)
    nc = pb.mesh.n_cells
    o.set_state(x=Ft @ X, vp=L @ F0 @ X, v=L @ F0 @ Xc.T, e=np.ones(nc),
                F=np.repeat(Ft.reshape(-1, 1), nc, axis=1))
    vs, Fs = o.predictor(2, dt)
    Xp = _corner_X(pb)
    np.testing.assert_allclose(vs, Xp @ (L @ F0).T, rtol=0, atol=1e-13)
    Fex = (np.eye(d) + (t0 + 0.5 * dt) * L) @ F0
    np.testing.assert_allclose(Fs, np.broadcast_to(Fex, Fs.shape), rtol=0, atol=1e-13)
    # first order (P0) keeps the cell values
    v1, F1 = o.predictor(1, dt)
    np.testing.assert_allclose(v1, np.broadcast_to((Xc @ (L @ F0).T)[:, None, :], v1.shape), rtol=0, atol=1e-14)
    np.testing.assert_allclose(F1, np.broadcast_to(Ft, F1.shape), rtol=0, atol=1e-14)
    o.close()


def _waves(d):
    """wave vector k (|k| = 2 pi), P direction k^, S direction s^ (s^ . k^ = 0), amplitudes"""
    if d == 2:
        kh = np.array([math.cos(0.3), math.sin(0.3)])
        sh = np.array([-kh[1], kh[0]])
    else:
        kh = np.array([1.0, 0.6, 0.3]) / math.sqrt(1.45)
        sh = np.cross(kh, [0.0, 0.0, 1.0])
        sh /= np.linalg.norm(sh)
    return 2 * math.pi * kh, kh, sh, 1e-6, 0.7e-6


def _wave_state(X, t, d, lam, mu, rho0):
    """displacement-derived velocity [n][d] and deformation gradient [n][d][d] at reference
    points X [n][d] and time t, and the displacement [n][d]"""
    k, kh, sh, ap, as_ = _waves(d)
    wp, ws = np.linalg.norm(k) * math.sqrt((lam + 2 * mu) / rho0), np.linalg.norm(k) * math.sqrt(mu / rho0)
    ph = X @ k
    u = ap * np.sin(ph - wp * t)[:, None] * kh + as_ * np.sin(ph - ws * t)[:, None] * sh
    v = -ap * wp * np.cos(ph - wp * t)[:, None] * kh - as_ * ws * np.cos(ph - ws * t)[:, None] * sh
    F = (np.eye(d) + ap * np.cos(ph - wp * t)[:, None, None] * np.outer(kh, k)
         + as_ * np.cos(ph - ws * t)[:, None, None] * np.outer(sh, k))
    return u, v, F


def _wave_errors(orc, d, n):
    pb = _mesh_problem(d, n)
    lam, mu, rho0 = pb.lam, 1.0, pb.rho0
    X = pb.mesh.x.T
    u0, vp0, _ = _wave_state(X, 0.0, d, lam, mu, rho0)
    Xc = W.cell_points(pb.mesh)
    _, vc, Fc = _wave_state(Xc, 0.0, d, lam, mu, rho0)
    nc = pb.mesh.n_cells
    o = orc.Oracle(pb)
    o.set_state(x=(X + u0).T, vp=vp0.T, v=vc.T, e=np.ones(nc), F=Fc.reshape(nc, d * d).T)
    dt = 0.3 / n / math.sqrt((lam + 2 * mu) / rho0)
    vs, Fs = o.predictor(2, dt)
    o.close()
    Xp = _corner_X(pb).reshape(-1, d)
    _, vex, Fex = _wave_state(Xp, 0.5 * dt, d, lam, mu, rho0)
    k, _, _, ap, _ = _waves(d)
    sv = ap * np.linalg.norm(k) * math.sqrt((lam + 2 * mu) / rho0)   # velocity scale a w_p
    sF = ap * np.linalg.norm(k)                                       # strain scale a |k|
    ev = math.sqrt(np.mean(np.sum((vs.reshape(-1, d) - vex) ** 2, axis=1))) / sv
    eF = math.sqrt(np.mean(np.sum((Fs.reshape(-1, d, d) - Fex) ** 2, axis=(1, 2)))) / sF
    return ev, eF


@pytest.mark.parametrize("d", [2, 3])
def test_predictor_second_order_on_elastic_waves(orc, d):
    ns = (16, 32, 64) if d == 2 else (6, 12, 24)
    errs = [_wave_errors(orc, d, n) for n in ns]
    for j in range(2):
        ov = math.log2(errs[j][0] / errs[j + 1][0])
        oF = math.log2(errs[j][1] / errs[j + 1][1])
        assert ov >= 1.7 and oF >= 1.7, (errs, ov, oF)
    # and the errors themselves are small at the finest mesh (relative to the wave's scales)
    assert errs[-1][0] < 0.02 and errs[-1][1] < 0.02, errs
