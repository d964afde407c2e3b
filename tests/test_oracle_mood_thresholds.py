"""Pins of the oracle's MOOD detection thresholds (CPU): Eqs. PAD and RDMP of Sect. "Limiting:
a posteriori MOOD loop", with the paper's delta0 = 1e-4 and delta1 = 1e-3 and readings R11 /
R12 (RDMP on the density over the stencil and the cell itself, delta0 absolute; the PAD
tolerance on eps = e - |v|^2/2 is 1e-10 max(|e|, |v|^2/2, a0^2) with a0^2 the squared P-wave
speed at rest).

Every expected flag below is derived by hand from a hand-built state, with candidates placed
at a threshold times (1 -+ 1e-3): far outside rounding, close enough that each of these
mistakes fails a test -- delta0 and delta1 swapped, delta0 taken relative to the density,
the cell itself left out of the RDMP range, the a0^2 floor of the PAD tolerance dropped
(checked by mutating the oracle's source). A last test ties these decisions to the step: the
first MOOD round of a full step flags exactly the cells whose unlimited candidate fails them.
"""
import dataclasses

import numpy as np
import pytest

import workloads as W

# two counter-clockwise triangles c0 = (0, 1, 2), c1 = (1, 3, 2) on the unit square; moving
# node 3 to (1 + s, 1 + s) makes |c1| = (1 + 2 s) / 2 while |c0| = 1/2 stays
X0 = np.array([[0.0, 1.0, 0.0, 1.0], [0.0, 0.0, 1.0, 1.0]])
C2N = np.array([[0, 1], [1, 3], [2, 2]], np.int32)


def _two_triangles(orc, rho0, mu=1.0, lam=2.0, **kw):
    mesh = W.Mesh(2, X0.copy(), C2N.copy(), np.zeros((2, 0), np.int32), np.zeros(0, np.int32))
    pb = W.Problem("two_triangles", mesh, rho0, lam, np.full(2, mu), np.zeros((2, 2)), 0.4, 1)
    return orc.Oracle(dataclasses.replace(pb, **kw))


def _stretch(o, s):
    """node 3 to (1 + s, 1 + s): densities rho0 (c0) and rho0 / (1 + 2 s) (c1)"""
    x = X0.copy()
    x[:, 3] = 1.0 + s
    o.set_state(x=x)


# ----------------------------------------------------------------------------- Eq. RDMP
@pytest.mark.parametrize("rho0", [1.0, 8.93])
def test_rdmp_range_includes_the_cell_itself(orc, rho0):
    o = _two_triangles(orc, rho0)
    _stretch(o, 0.25)  # rho(c1) = rho0 / 1.5
    for c in (0, 1):
        _, lo, hi = o.rdmp(c, rho0)
        # c0 is the densest and c1 the lightest cell: each one's own density is an end of its range
        assert lo == pytest.approx(rho0 / 1.5, rel=1e-14) and hi == pytest.approx(rho0, rel=1e-14)


def _rdmp_cases(rho0, s):
    """the candidate densities around the two ends of the admissible interval, as (rho, flag
    expected for cells 0 and 1); delta by hand for the range [rho0 / (1 + 2 s), rho0]"""
    lo, hi = rho0 / (1 + 2 * s), rho0
    delta = max(1e-4, 1e-3 * (hi - lo))
    eps = 1e-3 * delta
    return lo, hi, delta, [(lo - delta - eps, False), (lo - delta + eps, True),
                           (hi + delta - eps, True), (hi + delta + eps, False)]


@pytest.mark.parametrize("rho0, s", [(8.93, 0.002), (1.0, 0.01)])
def test_rdmp_absolute_delta0_when_the_range_is_narrow(orc, rho0, s):
    """delta1 (M - m) < delta0: delta = delta0 = 1e-4 exactly, absolute (with rho0 = 8.93 a
    delta0 relative to the density would be ~9e-4 and admit m - 1e-4 - 1e-7)."""
    lo, hi, delta, cases = _rdmp_cases(rho0, s)
    assert 1e-3 * (hi - lo) < 1e-4 and delta == 1e-4
    o = _two_triangles(orc, rho0)
    _stretch(o, s)
    for c in (0, 1):
        for rho, ok in cases:
            assert o.rdmp(c, rho)[0] is ok, (c, rho, ok)


@pytest.mark.parametrize("rho0, s", [(8.93, 0.5), (1.0, 0.25)])
def test_rdmp_relative_delta1_when_the_range_is_wide(orc, rho0, s):
    """delta1 (M - m) > delta0: delta = 1e-3 (M - m) (rho0 = 8.93, s = 0.5: 4.465e-3)."""
    lo, hi, delta, cases = _rdmp_cases(rho0, s)
    assert delta == 1e-3 * (hi - lo) > 1e-4
    o = _two_triangles(orc, rho0)
    _stretch(o, s)
    for c in (0, 1):
        for rho, ok in cases:
            assert o.rdmp(c, rho)[0] is ok, (c, rho, ok)


def test_rdmp_uniform_density(orc):
    """A uniform mesh at rest: range [rho0, rho0], delta = delta0."""
    o = _two_triangles(orc, 2.0)
    for c in (0, 1):
        ok, lo, hi = o.rdmp(c, 2.0)
        assert ok and lo == hi == 2.0
        assert o.rdmp(c, 2.0 + 1e-4 * 0.999)[0] and not o.rdmp(c, 2.0 + 1e-4 * 1.001)[0]
        assert o.rdmp(c, 2.0 - 1e-4 * 0.999)[0] and not o.rdmp(c, 2.0 - 1e-4 * 1.001)[0]


# ----------------------------------------------------------------------------- Eq. PAD
I2 = np.eye(2)


def test_pad_tolerance_floor_in_a_cell_at_rest(orc):
    """At rest (v = 0) the tolerance is 1e-10 a0^2, a0^2 = (kappa + 4 mu / 3) / rho0: with
    rho0 = 1, mu = 1, lambda = 2, kappa = lambda + 2 mu / 3 = 8/3 and a0^2 = 4, so tol = 4e-10.
    (Without the floor the tolerance would be 1e-10 |e| ~ 4e-20 and both candidates fail.)"""
    o = _two_triangles(orc, 1.0, mu=1.0, lam=2.0)
    v0 = np.zeros(2)
    assert o.pad(0, v0, -4e-10 * (1 - 1e-3), I2, 0.5) == 0
    assert o.pad(0, v0, -4e-10 * (1 + 1e-3), I2, 0.5) == 1
    assert o.pad(0, v0, 0.0, I2, 0.5) == 0


def test_pad_tolerance_floor_follows_the_material(orc):
    """a0^2 for other materials: vol_coeff = 1 (kappa = mu = 1.5, rho0 = 2): a0^2 =
    (1.5 + 2) / 2 = 1.75; the stiffened gas (gamma = 2, p_inf = 1, p0 = 1, mu = 1.5, rho0 = 2):
    a0^2 = (gamma (p0 + p_inf) + 4 mu / 3) / rho0 = (4 + 2) / 2 = 3."""
    v0 = np.zeros(2)
    o = orc.Oracle(_problem_two(2.0, 1.5, 0.0), orc.default_params(vol_coeff=1))
    assert o.pad(1, v0, -1.75e-10 * (1 - 1e-3), I2, 0.5) == 0
    assert o.pad(1, v0, -1.75e-10 * (1 + 1e-3), I2, 0.5) == 1
    sg = orc.Oracle(dataclasses.replace(_problem_two(2.0, 1.5, 0.0), stiffened_gas=(2.0, 1.0, 1.0)))
    assert sg.pad(0, v0, -3e-10 * (1 - 1e-3), I2, 0.5) == 0
    assert sg.pad(0, v0, -3e-10 * (1 + 1e-3), I2, 0.5) == 1


def _problem_two(rho0, mu, lam):
    mesh = W.Mesh(2, X0.copy(), C2N.copy(), np.zeros((2, 0), np.int32), np.zeros(0, np.int32))
    return W.Problem("two_triangles", mesh, rho0, lam, np.full(2, mu), np.zeros((2, 2)), 0.4, 1)


def test_pad_tolerance_in_a_moving_cell(orc):
    """v = (3, 4): |v|^2 / 2 = 12.5 > a0^2 = 4, so tol = 1e-10 x 12.5 = 1.25e-9."""
    o = _two_triangles(orc, 1.0, mu=1.0, lam=2.0)
    v = np.array([3.0, 4.0])
    assert o.pad(0, v, 12.5 - 1.25e-9 * (1 - 1e-3), I2, 0.5) == 0
    assert o.pad(0, v, 12.5 - 1.25e-9 * (1 + 1e-3), I2, 0.5) == 1
    # a 3D moving cell: v = (1, 2, 2), |v|^2 / 2 = 4.5, same material: tol = 4.5e-10
    x3 = np.array([[0.0, 1, 0, 0], [0.0, 0, 1, 0], [0.0, 0, 0, 1]])
    mesh = W.Mesh(3, x3, np.array([[0], [1], [2], [3]], np.int32), np.zeros((3, 0), np.int32),
                  np.zeros(0, np.int32))
    t = orc.Oracle(W.Problem("tet", mesh, 1.0, 2.0, np.ones(1), np.zeros((3, 1)), 0.25, 1))
    v3 = np.array([1.0, 2.0, 2.0])
    assert t.pad(0, v3, 4.5 - 4.5e-10 * (1 - 1e-3), np.eye(3), 1 / 6) == 0
    assert t.pad(0, v3, 4.5 - 4.5e-10 * (1 + 1e-3), np.eye(3), 1 / 6) == 1


def test_pad_not_computable(orc):
    o = _two_triangles(orc, 1.0)
    v0 = np.zeros(2)
    assert o.pad(0, v0, 0.1, I2, 0.0) == 2                       # tau <= 0
    assert o.pad(0, v0, 0.1, I2, -0.5) == 2
    assert o.pad(0, v0, 0.1, np.array([[1.0, 0], [0, -1]]), 0.5) == 2   # det F < 0
    assert o.pad(0, v0, 0.1, np.array([[1.0, 1], [1, 1]]), 0.5) == 2    # det F = 0
    assert o.pad(0, np.array([np.nan, 0]), 0.1, I2, 0.5) == 2
    assert o.pad(0, v0, np.inf, I2, 0.5) == 2
    assert o.pad(0, v0, 0.1, np.array([[1.0, np.inf], [0, 1]]), 0.5) == 2


# ----------------------------------------------------------------------------- the step uses them
@pytest.mark.parametrize("case", ["impact2d", "cube3d"])
def test_first_mood_round_flags_what_the_thresholds_reject(orc, case):
    """The cells that the first MOOD round of a full step flags are exactly those whose
    unlimited candidate (the same step with detection off) fails Eq. PAD or Eq. RDMP as
    decided by the functions pinned above."""
    pb = W.impact2d(n=24) if case == "impact2d" else W.cube3d(n=4)
    if case == "cube3d":
        pb.v *= 4.0
    o = orc.Oracle(pb)
    o.step(2)
    st = o.state()
    free = orc.Oracle(pb, mood=0)
    free.set_state(**{k: st[k] for k in ("x", "vp", "v", "e", "F")}, dt=o.dt)
    free.step()
    cand = free.state()
    first = orc.Oracle(pb, max_mood_iters=0)
    first.set_state(**{k: st[k] for k in ("x", "vp", "v", "e", "F")}, dt=o.dt)
    rc = first.step(check=False)
    mask = first.get(orc.F_ORDER)
    d, nc = pb.mesh.dim, pb.mesh.n_cells
    m = first.get(orc.F_MASS)
    expect = np.zeros(nc, bool)
    for c in range(nc):
        F = cand["F"][:, c].reshape(d, d)
        V = orc.cell_geometry(cand["x"][:, pb.mesh.c2n[:, c]].T)[0]  # |w_c(x^{n+1})|, as the step has it
        bad_pad = first.pad(c, cand["v"][:, c], cand["e"][c], F, V) != 0
        expect[c] = bad_pad or not first.rdmp(c, m[c] / V)[0]
    assert expect.sum() > 0, "no troubled cell: the case does not exercise the detection"
    assert rc == 6  # the first round flagged cells and max_mood_iters = 0 stops there
    np.testing.assert_array_equal(mask == 1, expect)
