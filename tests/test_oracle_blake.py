"""Oracle pin on Blake's problem (Sect. "Blake's problem"): a spherical cavity of radius a in an
elastic medium, at rest, whose face carries a pressure p0 from t = 0, against its exact solution.

The exact solution of small-strain elasticity (the paper's reference solution; here derived, not
read off a figure). The motion is radial and irrotational, u = grad phi, and the outgoing
solution of the wave equation is phi = F(tau) / r with tau = t - (r - a) / c, c the P-wave speed.
Then
  u_r = -F / r^2 - F' / (c r),   v_r = -F' / r^2 - F'' / (c r),
  sigma_rr = 4 mu F / r^3 + 4 mu F' / (c r^2) + rho F'' / r,
  p = -K div u = -K F'' / (c^2 r)                    (K = lambda + 2 mu / 3),
and sigma_rr(a, t) = -p0 for t > 0 with F(0) = F'(0) = 0 makes F a damped oscillator,
  F'' + 2 zeta w0 F' + w0^2 F = -p0 a / rho,   w0^2 = 4 mu / (rho a^2),   zeta = c_s / c,
  F = -(p0 a^3 / (4 mu)) S(tau),  S = 1 - exp(-zeta w0 tau) (cos wd tau + zeta w0 / wd sin wd tau),
with wd = w0 sqrt(1 - zeta^2): the front tau = 0 carries the jump v_r = p0 a / (rho c r).

The needle of the shell (`workloads.blake3d`) has slip walls on its lateral planes through the
centre, the pressure on its inner face and a free outer face; the oracle runs the paper's
scheme (P1 -> P0 MOOD cascade) to t = 1.6e-4, when the front reaches r = 0.9. Its radial
velocity, pressure and radial deviatoric stress (the paper's figures plot the last two) must
approach the exact ones as the mesh is refined: behind the front, away from the first cells at
the loaded face (where the paper also sees perturbations), and over all cells with the front
smeared over a few cells; the front must stand where c puts it."""
import math

import numpy as np
import pytest

import workloads as W


def blake_exact(r, t, a, p0, rho, E, nu):
    """(u_r, v_r, p) of the exact solution at radii r and time t"""
    mu = E / (2 * (1 + nu))
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    K = lam + 2 * mu / 3
    c, cs = math.sqrt((lam + 2 * mu) / rho), math.sqrt(mu / rho)
    w0 = math.sqrt(4 * mu / (rho * a * a))
    zeta = cs / c
    wd = w0 * math.sqrt(1 - zeta * zeta)
    C = p0 * a ** 3 / (4 * mu)
    r = np.asarray(r, dtype=float)
    tau = t - (r - a) / c
    on = tau > 0
    tp = np.where(on, tau, 0.0)
    e = np.exp(-zeta * w0 * tp)
    S0 = 1.0 - e * (np.cos(wd * tp) + zeta * w0 / wd * np.sin(wd * tp))
    S1 = (w0 * w0 / wd) * e * np.sin(wd * tp)
    S2 = (w0 * w0 / wd) * e * (wd * np.cos(wd * tp) - zeta * w0 * np.sin(wd * tp))
    ur = np.where(on, C * (S0 / r ** 2 + S1 / (c * r)), 0.0)
    vr = np.where(on, C * (S1 / r ** 2 + S2 / (c * r)), 0.0)
    p = np.where(on, K * C * S2 / (c * c * r), 0.0)
    return ur, vr, p


def test_exact_solution_meets_its_equations():
    """the closed form against the equations it solves, by central differences of u_r: v_r is
    its time derivative, the radial momentum equation rho dv_r/dt = d sigma_rr/dr +
    2 (sigma_rr - sigma_tt) / r holds behind the front, sigma_rr = -p0 at r = a, p = -K div u,
    and v_r jumps from 0 to p0 a / (rho c r) at the front"""
    a, p0, rho, E, nu = 0.1, 1e6, 3000.0, 62.5e9, 0.25
    mu = E / (2 * (1 + nu))
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    K = lam + 2 * mu / 3
    c = math.sqrt((lam + 2 * mu) / rho)
    t = 1.0e-4
    ex = lambda r, s: blake_exact(r, s, a, p0, rho, E, nu)  # noqa: E731
    r = np.array([a, 0.15, 0.3, 0.45])
    ht, hr = 1e-9, 1e-6
    u, v, p = ex(r, t)
    vmax = p0 / (rho * c)
    assert np.abs((ex(r, t + ht)[0] - ex(r, t - ht)[0]) / (2 * ht) - v).max() < 1e-6 * vmax

    def stresses(rr, s):
        uu = ex(rr, s)[0]
        ur = (ex(rr + hr, s)[0] - ex(rr - hr, s)[0]) / (2 * hr)
        return (lam + 2 * mu) * ur + 2 * lam * uu / rr, lam * (ur + 2 * uu / rr) + 2 * mu * uu / rr, ur + 2 * uu / rr

    ri = r[1:]
    srr, stt, div = stresses(ri, t)
    dsrr = (stresses(ri + 1e-4, t)[0] - stresses(ri - 1e-4, t)[0]) / 2e-4
    acc = (ex(ri, t + ht)[1] - ex(ri, t - ht)[1]) / (2 * ht)
    scale = rho * np.abs(acc).max()
    assert np.abs(rho * acc - (dsrr + 2 * (srr - stt) / ri)).max() < 1e-4 * scale
    assert np.abs(p[1:] + K * div).max() < 1e-6 * np.abs(p).max()
    # at the loaded face (one-sided differences of second order)
    u0, u1, u2 = ex(np.array([a, a + hr, a + 2 * hr]), t)[0]
    srr_a = (lam + 2 * mu) * (-3 * u0 + 4 * u1 - u2) / (2 * hr) + 2 * lam * u0 / a
    assert srr_a == pytest.approx(-p0, rel=1e-6)
    # the front
    rf = a + c * t
    vin = ex(np.array([rf - 1e-9]), t)[1][0]
    vout = ex(np.array([rf + 1e-9]), t)[1][0]
    assert vout == 0.0 and vin == pytest.approx(p0 * a / (rho * c * rf), rel=1e-6)


def _radial_fields(orc, pb, mu, K):
    """radius, radial velocity, pressure -tr(T)/3 and radial deviatoric stress r.T.r + p of each
    cell after the run (T from the cell's F by the oracle's stress)"""
    o = orc.Oracle(pb)
    tf = pb.meta["t_final"]
    while o.t < tf:
        o.step()
    x = o.get(orc.F_X)
    xc = x[:, pb.mesh.c2n].mean(axis=1)
    r = np.sqrt((xc * xc).sum(axis=0))
    vr = (o.get(orc.F_V) * xc).sum(axis=0) / r
    F = o.get(orc.F_F)
    p, srr = np.empty(r.size), np.empty(r.size)
    for c in range(r.size):
        T = orc.stress(F[:, c].reshape(3, 3), mu, K)
        p[c] = -np.trace(T) / 3.0
        rh = xc[:, c] / r[c]
        srr[c] = rh @ T @ rh + p[c]
    t = o.t
    o.close()
    return r, vr, p, srr, t


def _front(r, vr, nr, a=0.1, b=1.0):
    """where the front stands: v_r averaged over each radial layer of cells ((b - a) / nr wide),
    and the radius, coming from the outer face, at which that profile first reaches half its peak
    (linear interpolation between layers); a smeared step has it at the step"""
    edges = np.linspace(a, b, nr + 1)
    k = np.clip(np.searchsorted(edges, r) - 1, 0, nr - 1)
    prof = np.bincount(k, weights=vr, minlength=nr) / np.maximum(np.bincount(k, minlength=nr), 1)
    mid = 0.5 * (edges[1:] + edges[:-1])
    half = 0.5 * prof[mid > 0.5].max()
    j = np.nonzero(prof >= half)[0].max()
    return mid[j] + (prof[j] - half) / (prof[j] - prof[j + 1]) * (mid[j + 1] - mid[j])


@pytest.mark.slow
def test_oracle_converges_to_blakes_solution(orc):
    m = W.blake3d(nr=4).meta
    a, p0 = m["r_in"], m["p0"]
    rho, E, nu = 3000.0, m["E"], m["nu"]
    mu = E / (2 * (1 + nu))
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    K = lam + 2 * mu / 3
    c = math.sqrt((lam + 2 * mu) / rho)
    err = {k: [] for k in ("v_smooth", "v_whole", "front", "p_smooth", "p_whole", "s_smooth", "s_whole")}
    for nr in (50, 100):
        r, vr, p, srr, t = _radial_fields(orc, W.blake3d(nr=nr), mu, K)
        ue, ve, pe = blake_exact(r, t, a, p0, rho, E, nu)
        h = 1e-6
        dudr = (blake_exact(r + h, t, a, p0, rho, E, nu)[0] - blake_exact(r - h, t, a, p0, rho, E, nu)[0]) / (2 * h)
        se = (lam + 2 * mu) * dudr + 2 * lam * ue / r + pe  # sigma_rr + p
        front = a + c * t
        vmax = p0 * a / (rho * c * front)  # the jump of v_r at the front, the largest |v_r|
        smax = p0 * a / front  # the jump of sigma_rr at the front
        behind = (r > 1.5 * a) & (r < front - 0.1)
        err["v_smooth"].append(np.abs(vr - ve)[behind].mean() / vmax)
        err["v_whole"].append(np.abs(vr - ve).mean() / vmax)
        err["front"].append(abs(_front(r, vr, nr) - front))
        err["p_smooth"].append(np.abs(p - pe)[behind].mean() / smax)
        err["p_whole"].append(np.abs(p - pe).mean() / smax)
        err["s_smooth"].append(np.abs(srr - se)[behind].mean() / smax)
        err["s_whole"].append(np.abs(srr - se).mean() / smax)
    # 1,200 and 2,400 tetrahedra: radial cells of 0.018 and 0.009. Measured: v_r 1.8 % and 0.63 %
    # of its jump behind the front, 8.2 % and 3.4 % over all cells; the front 0.027 and 0.014
    # ahead of a + c t; p 2.8 % and 1.4 %, 7.4 % and 4.0 %, and the radial deviatoric stress
    # 1.2 % and 0.45 %, 3.7 % and 1.9 % of the jump of sigma_rr
    bars = {"v_smooth": (0.01, 2.0), "v_whole": (0.05, 1.8), "p_smooth": (0.02, 1.7), "p_whole": (0.06, 1.6),
            "s_smooth": (0.01, 2.0), "s_whole": (0.03, 1.7)}
    for k, (bar, ratio) in bars.items():
        assert err[k][1] < bar and err[k][0] / err[k][1] > ratio, (k, err[k])
    assert err["front"][1] < 0.025 and err["front"][1] < 0.7 * err["front"][0], err["front"]
