"""Oracle pin on the paper's beryllium plate (Sect. "Elastic vibration of a beryllium plate"):
the frequency of its first free bending mode.

The paper's initial velocity is the first free-free bending mode of an Euler-Bernoulli plate:
alpha L is the first root b of cos(b) cosh(b) = 1, a1 / a2 = (cosh b - cos b) / (sinh b - sin b),
and omega = alpha^2 sqrt(E' H^2 / (12 rho0)) with the plane-strain modulus E' = E / (1 - nu^2).
The plate is thick (L / H = 6), so its exact first bending frequency in plane-strain elasticity
lies below omega (shear deformation and rotary inertia). That frequency is computed here by an
independent quadratic (P2) finite-element eigen-solve of linear plane-strain elasticity, itself
pinned by its three rigid modes, by its convergence, and by the Euler-Bernoulli frequency of a
slender plate. The oracle (the unlimited scheme at a small amplitude, where the law is linear
elasticity with lambda and mu) must vibrate at that frequency, with an error that falls with
the mesh size at about second order."""
import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as sla
from scipy.optimize import brentq

import workloads as W

RHO0, E, NU = 1845.0, 3.1827e11, 0.0539
L_BE, H_BE = 0.06, 0.01


def _lame(E, nu):
    return E * nu / ((1 + nu) * (1 - 2 * nu)), E / (2 * (1 + nu))


def _euler_bernoulli(b, L, H, rho, E, nu):
    """first free-free bending frequency of a plane-strain Euler-Bernoulli plate"""
    return (b / L) ** 2 * math.sqrt(E / (1 - nu * nu) * H * H / (12.0 * rho))


def _first_root():
    return brentq(lambda b: math.cos(b) * math.cosh(b) - 1.0, 4.0, 5.0, xtol=1e-14)


# six-point degree-4 quadrature on the reference triangle (weights sum to 1/2)
_QW = [(0.223381589678011, 0.445948490915965), (0.109951743655322, 0.091576213509771)]
_QP = [((1 - 2 * a, a, a), w / 2) for w, a in _QW] + [((a, 1 - 2 * a, a), w / 2) for w, a in _QW] + \
      [((a, a, 1 - 2 * a), w / 2) for w, a in _QW]


def _p2_reference_matrices():
    """values and barycentric derivatives of the six P2 shape functions (vertices 0-2, then
    the midpoints of edges 12, 20, 01) at the quadrature points, derivatives w.r.t. (L1, L2)"""
    out = []
    for (l1, l2, l3), w in _QP:
        N = np.array([l1 * (2 * l1 - 1), l2 * (2 * l2 - 1), l3 * (2 * l3 - 1), 4 * l2 * l3, 4 * l3 * l1, 4 * l1 * l2])
        dL = np.array([[4 * l1 - 1, 0, 0], [0, 4 * l2 - 1, 0], [0, 0, 4 * l3 - 1],
                       [0, 4 * l3, 4 * l2], [4 * l3, 0, 4 * l1], [4 * l2, 4 * l1, 0]])
        out.append((N, np.stack([dL[:, 0] - dL[:, 2], dL[:, 1] - dL[:, 2]], 1), w))
    return out


def plate_frequencies(nx, ny, L, H, rho, E, nu, k=6):
    """Lowest k angular eigenfrequencies of a free rectangular plate [-L/2, L/2] x [-H/2, H/2]
    in linear plane-strain elasticity (K u = w^2 M u), P2 triangles on an nx x ny grid of
    rectangles each cut in two; the first three are the rigid modes (zero)."""
    lam, mu = _lame(E, nu)
    NX, NY = 2 * nx + 1, 2 * ny + 1
    X, Y = np.meshgrid(np.linspace(-L / 2, L / 2, NX), np.linspace(-H / 2, H / 2, NY), indexing="ij")
    xy = np.stack([X.ravel(), Y.ravel()], 1)

    def nid(p):
        return p[0] * NY + p[1]

    def mid(p, q):
        return ((p[0] + q[0]) // 2, (p[1] + q[1]) // 2)

    tris = []
    for i in range(nx):
        for j in range(ny):
            a, b, c, d = (2 * i, 2 * j), (2 * i + 2, 2 * j), (2 * i + 2, 2 * j + 2), (2 * i, 2 * j + 2)
            for p, q, r in ((a, b, c), (a, c, d)):
                tris.append([nid(p), nid(q), nid(r), nid(mid(q, r)), nid(mid(r, p)), nid(mid(p, q))])
    tris = np.array(tris)
    Dm = np.array([[lam + 2 * mu, lam, 0.0], [lam, lam + 2 * mu, 0.0], [0.0, 0.0, mu]])
    ref = _p2_reference_matrices()
    rows, cols, kv, mv = [], [], [], []
    for t in tris:
        P = xy[t[:3]]
        Jm = np.array([P[0] - P[2], P[1] - P[2]]).T  # d x / d (L1, L2)
        dj, Ji = abs(np.linalg.det(Jm)), np.linalg.inv(Jm)
        Ke, Me = np.zeros((12, 12)), np.zeros((12, 12))
        for N, dref, w in ref:
            g = dref @ Ji  # d N / d (x, y)
            B = np.zeros((3, 12))
            B[0, 0::2], B[1, 1::2] = g[:, 0], g[:, 1]
            B[2, 0::2], B[2, 1::2] = g[:, 1], g[:, 0]
            Nn = np.zeros((2, 12))
            Nn[0, 0::2], Nn[1, 1::2] = N, N
            Ke += (B.T @ Dm @ B) * (w * dj)
            Me += (Nn.T @ Nn) * (rho * w * dj)
        dof = np.stack([2 * t, 2 * t + 1], 1).ravel()
        rows.append(np.repeat(dof, 12))
        cols.append(np.tile(dof, 12))
        kv.append(Ke.ravel())
        mv.append(Me.ravel())
    n = 2 * xy.shape[0]
    r, c = np.concatenate(rows), np.concatenate(cols)
    K = sp.csc_matrix((np.concatenate(kv), (r, c)), shape=(n, n))
    M = sp.csc_matrix((np.concatenate(mv), (r, c)), shape=(n, n))
    # shift-invert about -(w_EB / 2)^2: K - sigma M is then as well conditioned as the modes near
    # the bending one (a shift far below them leaves K + |sigma| M nearly singular)
    sigma = -0.25 * _euler_bernoulli(_first_root(), L, H, rho, E, nu) ** 2
    w2 = sla.eigsh(K, k=k, M=M, sigma=sigma, which="LM", return_eigenvectors=False)
    return np.sqrt(np.clip(np.sort(w2), 0.0, None))


def test_paper_plate_data_is_the_first_euler_bernoulli_mode():
    pb = W.be_plate(nx=5, ny=3)
    b = _first_root()
    m = pb.meta
    assert m["alpha"] * m["L"] == pytest.approx(b, rel=2e-5)
    a1, a2 = 56.6368, 57.6455
    assert a1 / a2 == pytest.approx((math.cosh(b) - math.cos(b)) / (math.sinh(b) - math.sin(b)), rel=2e-5)
    assert _euler_bernoulli(b, L_BE, H_BE, RHO0, E, NU) == pytest.approx(m["omega"], rel=1e-4)


def test_finite_element_reference():
    wEB = _euler_bernoulli(_first_root(), L_BE, H_BE, RHO0, E, NU)
    w = plate_frequencies(24, 4, L_BE, H_BE, RHO0, E, NU)
    assert np.all(w[:3] < 1e-5 * wEB)  # two translations and a rotation
    assert w[3] > 0.5 * wEB
    w_fine = plate_frequencies(48, 8, L_BE, H_BE, RHO0, E, NU)
    assert w_fine[3] == pytest.approx(w[3], rel=1e-4)
    # the thick plate bends below the Euler-Bernoulli frequency (shear and rotary inertia)
    assert 0.85 < w[3] / wEB < 0.97
    # a slender plate (L / H = 40) bends at the Euler-Bernoulli frequency, slightly below it
    Ls = 40 * H_BE
    ws = plate_frequencies(80, 2, Ls, H_BE, RHO0, E, NU, k=4)
    r = ws[3] / _euler_bernoulli(_first_root(), Ls, H_BE, RHO0, E, NU)
    assert 0.995 < r < 1.0


def _bending_frequency(orc, pb):
    """angular frequency of the first mode from the oracle: the amplitude of the initial mode,
    a(t) = sum_c m_c v_y,c(t) phi_c / sum_c m_c phi_c^2 with phi the initial vertical velocity
    (cells are material points), crosses zero at T/4 and 3T/4"""
    o = orc.Oracle(pb, mood=0)
    m = o.get(orc.F_MASS)
    phi = pb.v[1].copy()
    den = float((m * phi * phi).sum())
    ts, amp = [0.0], [1.0]
    zeros = []
    while len(zeros) < 2 and o.t < pb.meta["t_final"]:
        o.step()
        ts.append(o.t)
        amp.append(float((m * o.get(orc.F_V)[1] * phi).sum()) / den)
        if amp[-2] * amp[-1] < 0.0:
            zeros.append(ts[-2] - amp[-2] * (ts[-1] - ts[-2]) / (amp[-1] - amp[-2]))
    o.close()
    assert len(zeros) == 2
    return math.pi / (zeros[1] - zeros[0])


def test_oracle_first_bending_frequency(orc):
    w_fe = plate_frequencies(24, 4, L_BE, H_BE, RHO0, E, NU)[3]
    err = []
    for nx, ny in ((31, 6), (61, 11)):
        # 1e-3 of the paper's amplitude (whose bending strains reach ~12 % at the surfaces): strains
        # ~1e-4, where the neo-Hookean law is linear elasticity
        w = _bending_frequency(orc, W.be_plate(nx=nx, ny=ny, amp=1e-3))
        err.append(abs(w / w_fe - 1.0))
    # 300 and 1,200 triangles (6 and 11 points through the thickness)
    assert err[1] < 0.03
    assert err[0] / err[1] > 3.0  # h halved: about second order
