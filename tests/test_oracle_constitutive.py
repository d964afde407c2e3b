"""Pins of the oracle's geometry and constitutive functions against closed forms, finite
differences of independently written energies, and identities the paper states."""
import dataclasses
import math

import numpy as np
import pytest

import oracle as O
import workloads as W


# ----------------------------------------------------------------------------- geometry
def test_unit_triangle_closed_form(orc):
    xs = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    V, xc, N, ln, Lc = orc.cell_geometry(xs)
    assert V == 0.5
    np.testing.assert_allclose(xc, [1 / 3, 1 / 3], rtol=0, atol=1e-16)
    # outward edge normals scaled by edge length, face k opposite vertex k
    np.testing.assert_allclose(N, [[1, 1], [-1, 0], [0, -1]], atol=1e-16)
    # corner vector = dV/dx_p (Eq. def_lcpncp): dV/dx0 = (-1/2,-1/2), dV/dx1 = (1/2,0), dV/dx2 = (0,1/2)
    np.testing.assert_allclose(ln, [[-0.5, -0.5], [0.5, 0.0], [0.0, 0.5]], atol=1e-16)
    # in-circle diameter of the right isoceles triangle = 2 (a+b-c)/2 with legs 1
    assert Lc == pytest.approx(2 - math.sqrt(2), rel=1e-15)


def test_unit_tet_closed_form(orc):
    xs = np.array([[0.0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]])
    V, xc, N, ln, Lc = orc.cell_geometry(xs)
    assert V == pytest.approx(1 / 6, rel=1e-15)
    np.testing.assert_allclose(xc, [0.25] * 3, atol=1e-16)
    np.testing.assert_allclose(N[1], [-0.5, 0, 0], atol=1e-16)
    np.testing.assert_allclose(N[0], [0.5, 0.5, 0.5], atol=1e-16)
    np.testing.assert_allclose(ln[0], [-1 / 6] * 3, atol=1e-16)
    np.testing.assert_allclose(ln[1], [1 / 6, 0, 0], atol=1e-16)
    # in-sphere radius of the corner tet = 1/(3+sqrt3)
    assert Lc == pytest.approx(2 / (3 + math.sqrt(3)), rel=1e-14)


@pytest.mark.parametrize("d", [2, 3])
def test_corner_vector_is_volume_gradient(orc, d):
    """l_cp n_cp = d|w_c|/dx_p (Eq. def_lcpncp) and sum_p l_cp n_cp = 0, checked by central
    differences on random simplices."""
    rng = np.random.default_rng(11 + d)
    for _ in range(20):
        xs = rng.normal(size=(d + 1, d))
        V, _, _, ln, _ = orc.cell_geometry(xs)
        if V < 0:
            xs[[1, 2]] = xs[[2, 1]]
            V, _, _, ln, _ = orc.cell_geometry(xs)
        np.testing.assert_allclose(ln.sum(axis=0), 0, atol=1e-14 * np.abs(ln).max())
        h = 1e-6
        for p in range(d + 1):
            for a in range(d):
                xp = xs.copy(); xp[p, a] += h
                xm = xs.copy(); xm[p, a] -= h
                fd = (orc.cell_geometry(xp)[0] - orc.cell_geometry(xm)[0]) / (2 * h)
                assert fd == pytest.approx(ln[p, a], rel=1e-7, abs=1e-9)


# ----------------------------------------------------------------------------- stress
def _rand_F(rng, d, amp=0.3):
    while True:
        F = np.eye(d) + amp * rng.normal(size=(d, d))
        if np.linalg.det(F) > 0.2:
            return F


def _W_independent(F, rho0, mu, kappa):
    """Stored energy per reference volume rho0 Psi written from Eqs. EOS_neoHook and
    familiy_energies (a = -1) with numpy, independently of the oracle's C code."""
    d = F.shape[0]
    F3 = np.eye(3)
    F3[:d, :d] = F
    J = np.linalg.det(F3)
    I1bar = J ** (-2 / 3) * np.trace(F3 @ F3.T)
    return kappa / 4 * ((J - 1) ** 2 + np.log(J) ** 2) + mu / 2 * (I1bar - 3)


@pytest.mark.parametrize("d", [2, 3])
def test_stress_is_energy_derivative(orc, d):
    """T = 2 rho dPsi/dB B (Eq. const_law) is equivalent to T = (1/J) P F^t with the first
    Piola-Kirchhoff stress P = d(rho0 Psi)/dF; P by central differences of an independently
    written energy."""
    rng = np.random.default_rng(5 + d)
    mu, kappa, rho0 = 1.3, 2.7, 1.9
    for _ in range(10):
        F = _rand_F(rng, d)
        P = np.zeros((d, d))
        h = 1e-6
        for i in range(d):
            for j in range(d):
                Fp = F.copy(); Fp[i, j] += h
                Fm = F.copy(); Fm[i, j] -= h
                P[i, j] = (_W_independent(Fp, rho0, mu, kappa) - _W_independent(Fm, rho0, mu, kappa)) / (2 * h)
        T_fd = P @ F.T / np.linalg.det(F)
        T = orc.stress(F, mu, kappa)
        np.testing.assert_allclose(T, T_fd, rtol=0, atol=2e-8 * (1 + np.abs(T).max()))
        # the oracle's own free energy agrees with the independent one
        assert orc.free_energy(F, rho0, mu, kappa) * rho0 == pytest.approx(
            _W_independent(F, rho0, mu, kappa), rel=1e-12, abs=1e-14)


@pytest.mark.parametrize("d", [2, 3])
def test_stress_identities(orc, d):
    rng = np.random.default_rng(3)
    mu, kappa = 0.8, 3.1
    np.testing.assert_array_equal(orc.stress(np.eye(d), mu, kappa), np.zeros((d, d)))
    for _ in range(10):
        F = _rand_F(rng, d)
        T = orc.stress(F, mu, kappa)
        np.testing.assert_allclose(T, T.T, atol=1e-14 * np.abs(T).max())          # symmetry
        B = F @ F.T
        np.testing.assert_allclose(T @ B, B @ T, atol=1e-13 * np.abs(T @ B).max())  # T B = B T
        # objectivity: T(R F) = R T(F) R^t
        if d == 2:
            th = rng.uniform(0, 2 * np.pi)
            R = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
        else:
            R, _ = np.linalg.qr(rng.normal(size=(3, 3)))
            if np.linalg.det(R) < 0:
                R[:, 0] *= -1
        np.testing.assert_allclose(orc.stress(R @ F, mu, kappa), R @ T @ R.T, atol=1e-13 * (1 + np.abs(T).max()))


def test_pure_dilation_pressure_closed_form(orc):
    """F = s I in 3D: deviator vanishes, T = -p I with p = -(kappa/2)(J - 1 + log J / J)."""
    for s in (0.8, 0.97, 1.0, 1.05, 1.3):
        J = s ** 3
        T = orc.stress(s * np.eye(3), 0.7, 2.2)
        p = -0.5 * 2.2 * (J - 1 + math.log(J) / J)
        np.testing.assert_allclose(T, -p * np.eye(3), atol=1e-15 * (1 + abs(p)))


@pytest.mark.parametrize("d", [2, 3])
def test_small_strain_limit_is_lame(orc, d):
    """With kappa = lambda + 2 mu / 3 the stress linearises to lambda tr(eps) I + 2 mu eps."""
    lam, mu = 2.0, 0.7
    kappa = lam + 2 * mu / 3
    rng = np.random.default_rng(1)
    G = rng.normal(size=(d, d))
    eps_sym = 0.5 * (G + G.T)
    for h in (1e-4, 1e-5):
        T = orc.stress(np.eye(d) + h * G, mu, kappa) / h
        lin = lam * np.trace(eps_sym) * np.eye(d) + 2 * mu * eps_sym
        np.testing.assert_allclose(T, lin, atol=20 * h * np.abs(G).max() ** 2 * (lam + mu))


def test_sound_speed(orc):
    """a^2 = (K(J) + 4 mu / (3 J)) / rho with K = -J dp/dJ; at J = 1: (lambda + 2 mu)/rho."""
    lam, mu, rho = 1.06, 0.46, 8.93
    kappa = lam + 2 * mu / 3
    assert orc.sound_speed(np.eye(2), rho, mu, kappa) == pytest.approx(math.sqrt((lam + 2 * mu) / rho), rel=1e-15)
    s = 1.1
    J = s ** 3
    p = lambda J: -0.5 * kappa * (J - 1 + math.log(J) / J)
    K = -J * (p(J + 1e-6) - p(J - 1e-6)) / 2e-6
    a = orc.sound_speed(s * np.eye(3), rho, mu, kappa)
    assert a * a * rho == pytest.approx(K + 4 * mu / (3 * J), rel=1e-8)


# ----------------------------------------------------------------------------- energy family
def _W_family(F, mu, kappa, a):
    """rho0 Psi of Eqs. EOS_neoHook and familiy_energies for parameter a, written with numpy
    from the invariants of Bbar = J^{-2/3} F F^t (plane strain in 2D), independently of the
    oracle's C code"""
    d = F.shape[0]
    F3 = np.eye(3)
    F3[:d, :d] = F
    J = np.linalg.det(F3)
    Bb = J ** (-2 / 3) * F3 @ F3.T
    I1 = np.trace(Bb)
    I2 = 0.5 * (I1 ** 2 - np.trace(Bb @ Bb))
    return kappa / 4 * ((J - 1) ** 2 + np.log(J) ** 2) + mu / 4 * (-2 * a * (I1 - 3) + (1 + a) / 3 * (I2 ** 2 - 9))


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("a", [-1.0, 0.0, 0.4])
def test_energy_family_stress_is_energy_derivative(d, a):
    """T = (1/J) P F^t with P = d(rho0 Psi)/dF by central differences of the independently
    written energy of the family; a = -1 reproduces the neo-Hookean stress exactly."""
    rng = np.random.default_rng(21 + d)
    mu, kappa, rho0 = 1.3, 2.7, 1.9
    for _ in range(8):
        F = _rand_F(rng, d)
        P = np.zeros((d, d))
        h = 1e-6
        for i in range(d):
            for j in range(d):
                Fp = F.copy(); Fp[i, j] += h
                Fm = F.copy(); Fm[i, j] -= h
                P[i, j] = (_W_family(Fp, mu, kappa, a) - _W_family(Fm, mu, kappa, a)) / (2 * h)
        T_fd = P @ F.T / np.linalg.det(F)
        T = O.stress_a(F, mu, kappa, a)
        np.testing.assert_allclose(T, T_fd, rtol=0, atol=2e-8 * (1 + np.abs(T).max()))
        assert O.free_energy_a(F, rho0, mu, kappa, a) * rho0 == pytest.approx(_W_family(F, mu, kappa, a),
                                                                              rel=1e-12, abs=1e-14)
        if a == -1.0:
            assert np.array_equal(T, O.stress(F, mu, kappa))


@pytest.mark.parametrize("a", [0.0, 0.4])
def test_energy_family_small_strain_shear_modulus_is_mu(a):
    """Every member of the family has shear modulus mu and bulk modulus kappa at small strain:
    T = 2 mu dev(E) + kappa tr(E) I + O(|E|^2), E the small strain (3D)."""
    rng = np.random.default_rng(3)
    mu, kappa = 0.8, 2.1
    G = rng.normal(size=(3, 3))
    for eps in (1e-4, 1e-5):
        F = np.eye(3) + eps * G
        E = 0.5 * (F + F.T) - np.eye(3)
        T_lin = 2 * mu * (E - np.trace(E) / 3 * np.eye(3)) + kappa * np.trace(E) * np.eye(3)
        T = O.stress_a(F, mu, kappa, a)
        assert np.abs(T - T_lin).max() < 50 * eps ** 2 * (mu + kappa)


def test_energy_family_scheme_conserves_energy():
    """a = 0 through the whole scheme: an initially strained block at rest in slip walls
    conserves total energy (which starts from the family's free energy) and stays different
    from the neo-Hookean run."""
    m = W.tri_mesh(10, 2, bc={k: W.SLIP for k in ("x0", "x1", "y0", "y1")})
    rng = np.random.default_rng(5)
    F = np.zeros((4, m.n_cells))
    F[0] = 1.0 + 0.02 * rng.standard_normal(m.n_cells)
    F[3] = 1.0 + 0.02 * rng.standard_normal(m.n_cells)
    pb = W.Problem("fam", m, 1.0, 2.0, np.full(m.n_cells, 1.0), np.zeros((2, m.n_cells)), 0.4, 10, F=F)
    o0 = O.Oracle(dataclasses.replace(pb, shear_a=0.0))
    o1 = O.Oracle(pb)
    e0 = (o0.get(O.F_MASS) * o0.get(O.F_E)).sum()
    assert e0 != (o1.get(O.F_MASS) * o1.get(O.F_E)).sum()
    for _ in range(10):
        o0.step()
        o1.step()
    e1 = (o0.get(O.F_MASS) * o0.get(O.F_E)).sum()
    assert abs(e1 - e0) <= 1e-12 * abs(e0)
    assert np.abs(o0.get(O.F_V) - o1.get(O.F_V)).max() > 1e-6


def test_energy_family_scheme_conserves_energy_3d():
    """The same in 3D: a = 0, an initially strained cube at rest in slip walls conserves its total
    energy through the scheme and moves differently from the neo-Hookean run."""
    sides = ("x0", "x1", "y0", "y1", "z0", "z1")
    m = W.tet_mesh(3, 3, 3, 2, bc={k: W.SLIP for k in sides})
    rng = np.random.default_rng(6)
    F = np.zeros((9, m.n_cells))
    for q in (0, 4, 8):
        F[q] = 1.0 + 0.02 * rng.standard_normal(m.n_cells)
    pb = W.Problem("fam3d", m, 1.0, 2.0, np.full(m.n_cells, 1.0), np.zeros((3, m.n_cells)), 0.25, 10, F=F)
    o0 = O.Oracle(dataclasses.replace(pb, shear_a=0.0))
    o1 = O.Oracle(pb)
    e0 = (o0.get(O.F_MASS) * o0.get(O.F_E)).sum()
    for _ in range(10):
        o0.step()
        o1.step()
    assert abs((o0.get(O.F_MASS) * o0.get(O.F_E)).sum() - e0) <= 1e-12 * abs(e0)
    assert np.abs(o0.get(O.F_V) - o1.get(O.F_V)).max() > 1e-6
