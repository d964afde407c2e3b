"""Pins of the oracle's stiffened-gas volumetric law (Eq. EOS_stiffened_gas; reading R18). CPU
only. Fixed by mechanics: a compression wave driven by a piston travels at the sound speed
a = sqrt((gamma (p + p_inf) + 4 mu / 3) / rho0) and carries the density jump rho0 V / a (the
momentum balance across an acoustic front); a uniformly strained block held by the outer
pressure equal to its own stress stays at rest; total energy is conserved."""
import dataclasses

import numpy as np
import pytest

import oracle as O
import workloads as W


def _front(gamma, pinf, p0, n=41, V=0.01, mu=1e-3):
    """piston at x = 0, the outer pressure p0 held at x = 1; run until the front has travelled
    0.6 (before it reaches x = 1); returns (a t, front position, density jump, rho0 V / a)"""
    T = 0.6 / np.sqrt((gamma * (p0 + pinf) + 4 * mu / 3) / 1.0)
    bc = {"x0": W.VELOCITY, "y0": W.SLIP, "y1": W.SLIP, "x1": W.PRESSURE}
    m = W.tri_mesh(n, 11, bc=bc)
    val = W.side_values(m, W.VELOCITY, (V, 0.0)) + W.side_values(m, W.PRESSURE, (p0, 0.0))
    pb = W.Problem("sgwave", m, 1.0, 0.0, np.full(m.n_cells, mu), np.zeros((2, m.n_cells)), 0.4, 10,
                   bcval=val, stiffened_gas=(gamma, pinf, p0))
    o = O.Oracle(pb)
    while o.t < T:
        o.step()
    xc = o.get(O.F_X)[0][m.c2n].mean(axis=0)
    rho = 1.0 / o.get(O.F_TAU)
    bins = np.linspace(0, 1, 41)
    idx = np.digitize(xc, bins)
    prof = np.array([rho[idx == i].mean() for i in range(1, len(bins))])
    mid = 0.5 * (bins[1:] + bins[:-1])
    a = np.sqrt((gamma * (p0 + pinf) + 4 * mu / 3) / 1.0)
    drho = V / a
    front = mid[np.where(prof > 1 + 0.5 * drho)[0].max()]
    return a * o.t, front, prof[:6].mean() - 1, drho


@pytest.mark.parametrize("gamma, pinf, p0", [(2.2, 1.0, 0.0), (1.4, 1.0, 0.0), (2.2, 0.5, 0.5), (3.0, 2.0, 0.3)])
def test_acoustic_front_speed_and_jump(gamma, pinf, p0):
    at, front, jump, drho = _front(gamma, pinf, p0)
    assert abs(front - at) <= 0.04  # within one and a half bins of the 40 along x
    assert jump == pytest.approx(drho, rel=0.02)


def test_strained_block_held_by_its_own_stress_stays_at_rest():
    s, gamma, pinf, p0, mu, a = 0.98, 2.2, 1.0, 0.3, 0.2, -1.0
    F = np.zeros((4, 1))
    F[0] = F[3] = s
    Ts = O.stress_a(np.array([[s, 0.0], [0.0, s]]), mu, 0.0, a)  # shear part alone
    P = p0 - Ts[0, 0]  # sigma_xx = -p0 + Ts_xx; the outer pressure balances it
    m = W.tri_mesh(9, 4, bc={k: W.PRESSURE for k in ("x0", "x1", "y0", "y1")})
    pb = W.Problem("sgblock", m, 1.0, 0.0, np.full(m.n_cells, mu), np.zeros((2, m.n_cells)), 0.4, 10,
                   F=np.tile(F, (1, m.n_cells)), bcval=W.side_values(m, W.PRESSURE, (P, 0.0)),
                   stiffened_gas=(gamma, pinf, p0))
    o = O.Oracle(pb)
    x0 = o.get(O.F_X).copy()
    for _ in range(5):
        o.step()
    assert np.abs(o.get(O.F_V)).max() < 1e-13
    assert np.abs(o.get(O.F_X) - x0).max() < 1e-14
    # a wrong outer pressure sets it moving
    o2 = O.Oracle(dataclasses.replace(pb, bcval=W.side_values(m, W.PRESSURE, (P + 0.05, 0.0))))
    for _ in range(5):
        o2.step()
    assert np.abs(o2.get(O.F_V)).max() > 1e-4


def test_energy_conserved_with_stiffened_gas():
    m = W.tri_mesh(12, 5, bc={k: W.SLIP for k in ("x0", "x1", "y0", "y1")})
    rng = np.random.default_rng(2)
    pts = m.x[:, m.c2n].mean(axis=1)
    v = 0.05 * np.stack([np.sin(np.pi * pts[0]) * np.cos(np.pi * pts[1]), -np.cos(np.pi * pts[0]) * np.sin(np.pi * pts[1])])
    pb = W.Problem("sgbox", m, 1.0, 0.0, np.full(m.n_cells, 0.3) + 0.05 * rng.random(m.n_cells), v, 0.4, 10,
                   stiffened_gas=(2.2, 1.0, 0.2))
    o = O.Oracle(pb)
    mass = o.get(O.F_MASS)
    E0 = (mass * o.get(O.F_E)).sum()
    for _ in range(30):
        o.step()
    assert abs((mass * o.get(O.F_E)).sum() - E0) <= 1e-13 * abs(E0)


def test_bad_stiffened_gas_parameters_are_rejected():
    m = W.tri_mesh(5, 1)
    pb = W.Problem("bad", m, 1.0, 0.0, np.full(m.n_cells, 1.0), np.zeros((2, m.n_cells)), 0.4, 1,
                   stiffened_gas=(0.9, 1.0, 0.0))
    with pytest.raises(O.OracleError):
        O.Oracle(pb)


def test_stiffened_gas_in_3d_rest_and_energy():
    """3D counterparts: a compressed block held by the outer pressure that balances its stiffened
    gas pressure and shear stress stays at rest; in a box with slip walls and a swirling
    velocity the total energy is conserved to round-off."""
    s, gamma, pinf, p0, mu = 0.98, 2.2, 1.0, 0.3, 0.2
    Ts = O.stress_a(s * np.eye(3), mu, 0.0, -1.0)  # shear part alone (zero for a pure dilation)
    P = p0 - Ts[0, 0]
    sides = ("x0", "x1", "y0", "y1", "z0", "z1")
    m = W.tet_mesh(3, 3, 3, 4, bc={k: W.PRESSURE for k in sides})
    pb = W.Problem("sgblock3d", m, 1.0, 0.0, np.full(m.n_cells, mu), np.zeros((3, m.n_cells)), 0.25, 5,
                   F=np.tile((s * np.eye(3)).reshape(9, 1), (1, m.n_cells)),
                   bcval=W.side_values(m, W.PRESSURE, (P, 0.0, 0.0)), stiffened_gas=(gamma, pinf, p0))
    o = O.Oracle(pb)
    x0 = o.get(O.F_X).copy()
    for _ in range(4):
        o.step()
    assert np.abs(o.get(O.F_V)).max() < 1e-13 and np.abs(o.get(O.F_X) - x0).max() < 1e-14
    o2 = O.Oracle(dataclasses.replace(pb, bcval=W.side_values(m, W.PRESSURE, (P + 0.05, 0.0, 0.0))))
    for _ in range(4):
        o2.step()
    assert np.abs(o2.get(O.F_V)).max() > 1e-4  # a wrong outer pressure sets it moving

    m = W.tet_mesh(4, 4, 4, 5, bc={k: W.SLIP for k in sides})
    pts = m.x[:, m.c2n].mean(axis=1)
    v = 0.05 * np.stack([np.sin(np.pi * pts[0]) * np.cos(np.pi * pts[1]), -np.cos(np.pi * pts[0]) * np.sin(np.pi * pts[1]),
                         0.3 * np.sin(np.pi * pts[2])])
    pb = W.Problem("sgbox3d", m, 1.0, 0.0, np.full(m.n_cells, 0.3), v, 0.25, 10, stiffened_gas=(2.2, 1.0, 0.2))
    o = O.Oracle(pb)
    mass = o.get(O.F_MASS)
    E0 = (mass * o.get(O.F_E)).sum()
    for _ in range(20):
        o.step()
    assert abs((mass * o.get(O.F_E)).sum() - E0) <= 1e-13 * abs(E0)
