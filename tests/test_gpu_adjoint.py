"""Reverse-mode gradients of recorded steps (lmood_tape_*) against central finite differences
(-m gpu). The MOOD order mask and dt are frozen: the runs use a fixed dt, and every finite
difference pair checks that its order masks equal the recorded ones, so the difference
quotient and the adjoint differentiate the same smooth map.

Objective: J = <lam, state(t^N)> with seeded random adjoints lam of x, v_p, v and F; checked
as the directional derivative <grad, delta> for seeded random directions delta of each input.
The two perturbed runs' fields are differenced element by element before the contraction
with lam. Steps of 1e-6 (absolute: the map's nonlinear scales -- sound speed, F ~ I, mu --
are O(1)) leave a truncation error ~1e-12 and a rounding error ~1e-16 |field| / eps ~ 1e-10,
relative; the bar is 1e-6.
"""
import dataclasses

import numpy as np
import pytest

import oracle as O
import paper_2104_02139_gb300 as L
import workloads as W
from adjoint_cases import bc_case, family_case, sg_case

pytestmark = pytest.mark.gpu

OUT_FIELDS = (("x", L.FIELD_X), ("vp", L.FIELD_VP), ("v", L.FIELD_V), ("F", L.FIELD_F), ("e", L.FIELD_E))


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available()
    L.build()
    O.build()


def _setup(pb, seed):
    """Heterogeneous mu and a non-trivial initial F; seeded adjoints of the final state."""
    rng = np.random.default_rng(seed)
    d, nc, npn = pb.mesh.dim, pb.mesh.n_cells, pb.mesh.n_nodes
    F = np.zeros((d * d, nc))
    for a in range(d):
        F[a * d + a] = 1.0
    F += 0.01 * rng.standard_normal((d * d, nc))
    mu = np.asarray(pb.mu, dtype=float) * (1.0 + 0.1 * rng.random(nc))
    pb = dataclasses.replace(pb, F=F, mu=mu)
    lam = {"x": rng.standard_normal((d, npn)), "vp": rng.standard_normal((d, npn)),
           "v": rng.standard_normal((d, nc)), "F": rng.standard_normal((d * d, nc)), "e": rng.standard_normal(nc)}
    return pb, lam, rng


def _dt_fixed(pb, frac=0.5):
    s = L.simulation(pb)
    return frac * float(s.get(L.FIELD_DT)[0])


def _fields(st):
    return {k: st.get(fid) for k, fid in OUT_FIELDS}


def _run(pb, n, prm, pre=0, setter=None):
    """pre steps, optional setter(state), then n steps; returns (state, masks of the n steps)."""
    st = L.simulation(pb, **prm)
    if pre:
        st.run(pre)
    if setter:
        setter(st)
    masks = []
    for _ in range(n):
        st.step()
        masks.append(st.get(L.FIELD_ORDER).astype(np.int8))
    return st, masks


def _fd(pb, n, prm, lam, masks, make, eps, pre=0, tape=None):
    """central difference of J along the perturbation make(sign * eps): through ordinary steps
    (whose masks must equal the recorded ones), or through tape.replay (orders and dt frozen)"""
    vals = []
    for sgn in (+1.0, -1.0):
        pbp, setter = make(sgn * eps)
        if tape is None:
            st, mk = _run(pbp, n, prm, pre=pre, setter=setter)
            for j, (a, b) in enumerate(zip(mk, masks)):
                assert np.array_equal(a, b), f"order mask changed under the perturbation at step {j}"
        else:
            st = L.simulation(pbp, **prm)
            tape.replay(st)
        vals.append(_fields(st))
    # difference the fields first, then contract with lam (no cancellation in a large sum)
    return sum(float(((vals[0][k] - vals[1][k]) * lam[k]).sum()) for k in lam) / (2 * eps)


def _grad(pb, n, prm, lam, pre=0, ckpt=0):
    st = L.simulation(pb, **prm)
    if pre:
        st.run(pre)
    tape = L.Tape(st, n, ckpt)
    g = tape.backward(lam_x=lam["x"], lam_vp=lam["vp"], lam_v=lam["v"], lam_F=lam["F"], lam_e=lam.get("e"))
    return st, tape, g


def _rel(a, b):
    return abs(a - b) / max(abs(a), abs(b), 1e-300)


def _check_init_grads(pb, n, prm, seed, tol=1e-6, eps=1e-6, frozen=False):
    """frozen: finite differences through the tape's replay (any dt rule; MOOD masks of the
    recorded run); else through ordinary steps at a fixed dt"""
    pb, lam, rng = _setup(pb, seed)
    if not frozen:
        prm = dict(prm, dt_fixed=_dt_fixed(pb))
    st, tape, g = _grad(pb, n, prm, lam)
    assert tape.info()["through_init"] == 1
    _, masks = _run(pb, n, prm)
    d, nc = pb.mesh.dim, pb.mesh.n_cells
    dv = rng.standard_normal((d, nc))
    dmu = rng.standard_normal(nc) * np.asarray(pb.mu)
    dF = rng.standard_normal((d * d, nc))
    sv = smu = sF = eps  # absolute: the nonlinear scales (sound speed ~ 1, F ~ I, mu ~ 1) are O(1)
    cases = [
        ("v", lambda e: (dataclasses.replace(pb, v=pb.v + e * dv), None), sv, float((g["v"] * dv).sum())),
        ("mu", lambda e: (dataclasses.replace(pb, mu=pb.mu + e * dmu), None), smu, float((g["mu"] * dmu).sum())),
        ("F", lambda e: (dataclasses.replace(pb, F=pb.F + e * dF), None), sF, float((g["F"] * dF).sum())),
    ]
    assert np.all(g["vp"] == 0.0) and np.all(g["e"] == 0.0)  # the start's v_p and e are derived
    out = {}
    for name, make, eps, ad in cases:
        fd = _fd(pb, n, prm, lam, masks, make, eps, tape=tape if frozen else None)
        out[name] = (ad, fd)
        assert _rel(ad, fd) <= tol, (name, ad, fd)
    return out, masks


def test_adjoint_fd_2d_p1():
    out, masks = _check_init_grads(W.plain2d(n=10), 6, {"mood": 0}, seed=11)
    assert all(np.all(m == 2) for m in masks)


def test_adjoint_fd_2d_p0_scheme():
    out, masks = _check_init_grads(W.plain2d(n=9), 5, {"order": 1}, seed=12)
    assert all(np.all(m == 1) for m in masks)


def test_adjoint_fd_2d_mood_mask():
    """An impact with MOOD active and the adaptive dt: some cells recomputed at first order
    in the recorded steps. RDMP has cells within ~1e-6 of its threshold, so the finite
    differences go through the tape's replay (the map with the recorded masks and dt)."""
    pb = W.impact2d(n=24)
    out, masks = _check_init_grads(pb, 6, {}, seed=13, frozen=True)
    assert sum(int((m == 1).sum()) for m in masks) > 0, "no first-order cells: the mixed mask is not exercised"


def test_adjoint_fd_3d_mood_mask():
    pb = W.cube3d(n=4)
    pb.v *= 4.0
    out, masks = _check_init_grads(pb, 5, {}, seed=23, frozen=True)
    assert sum(int((m == 1).sum()) for m in masks) > 0, "no first-order cells: the mixed mask is not exercised"


def test_replay_reproduces_the_recorded_run():
    """The frozen-mask replay of a state's own initial data lands on the recorded run."""
    for pb in (W.impact2d(n=24), W.cube3d(n=4)):
        pb.v *= 1.0 if pb.mesh.dim == 2 else 4.0
        st = L.simulation(pb)
        tape = L.Tape(st, 5, 2)
        other = tape.replay(L.simulation(pb))
        for k, fid in OUT_FIELDS:
            a, b = st.get(fid), other.get(fid)
            assert np.abs(a - b).max() <= 1e-13 * max(np.abs(a).max(), 1e-300), k
        assert np.array_equal(st.get(L.FIELD_DT), other.get(L.FIELD_DT)) or \
            abs(st.get(L.FIELD_DT)[0] / other.get(L.FIELD_DT)[0] - 1) < 1e-12


def test_adjoint_fd_3d_slip():
    out, masks = _check_init_grads(W.cube3d(n=3), 4, {}, seed=14)


def test_adjoint_fd_3d_clamped_column():
    pb = W.column3d(nxy=2, nz=6)
    out, masks = _check_init_grads(pb, 4, {}, seed=15)


@pytest.mark.parametrize("name", ["piston2d", "rebound2d", "pressure_traction2d", "box3d_bc"])
def test_adjoint_fd_boundary_faces(name):
    """Traction, pressure and prescribed-velocity faces and contact walls, MOOD active, the
    finite differences through the tape's replay (recorded masks and dt)."""
    _check_init_grads(bc_case(name), 5, {}, seed=24, frozen=True)


@pytest.mark.parametrize("name", ["cube3d_a0", "impact2d_a05"])
def test_adjoint_fd_shear_family(name):
    """the shear energy family (a != -1): its stress and product in the predictor's reverse"""
    _check_init_grads(family_case(name), 5, {}, seed=25, frozen=True)


def test_adjoint_fd_limited_level():
    """the three-level cascade: cells at the limited level (Barth-Jespersen slopes) in the
    recorded masks, finite differences through the tape's replay (which recomputes them with
    their limited slopes)"""
    pb = W.impact2d(n=24)
    pb.v += 1e-3 * np.random.default_rng(30).standard_normal(pb.v.shape)  # no ties in the stencils' ranges
    out, masks = _check_init_grads(pb, 6, {"cascade": 3}, seed=29, frozen=True)
    assert sum(int((m == 3).sum()) for m in masks) > 0, "no cell at the limited level"


@pytest.mark.parametrize("name", ["sgwave2d", "sgdrop3d"])
def test_adjoint_fd_stiffened_gas(name):
    """the stiffened gas (its pressure depends on e, which carries an adjoint)"""
    _check_init_grads(sg_case(name), 5, {}, seed=26, frozen=True)


@pytest.mark.parametrize("name", ["plain2d", "piston2d", "rebound2d", "box3d_bc", "sgwave2d"])
def test_adjoint_fd_mid_run_state(name):
    """A tape that starts after some steps: gradients of x, v_p, v, F, e (via lmood_set) and
    mu; with boundary faces the position direction moves them (their forces and multipliers);
    with the stiffened gas e enters the pressure."""
    pb = W.plain2d(n=10) if name == "plain2d" else (sg_case(name) if name.startswith("sg") else bc_case(name))
    pb, lam, rng = _setup(pb, 16)
    prm = {"dt_fixed": _dt_fixed(pb), "mood": 0}
    pre, n = 3, 5
    st, tape, g = _grad(pb, n, prm, lam, pre=pre)
    assert tape.info()["through_init"] == 0
    _, masks = _run(pb, n, prm, pre=pre)
    base = L.simulation(pb, **prm)
    base.run(pre)
    x0, vp0, v0, F0, e0 = (base.get(f) for f in (L.FIELD_X, L.FIELD_VP, L.FIELD_V, L.FIELD_F, L.FIELD_E))
    d, nc, npn = pb.mesh.dim, pb.mesh.n_cells, pb.mesh.n_nodes
    h = np.sqrt((base.get(L.FIELD_TAU) * base.get(L.FIELD_MASS)).mean())  # a cell size
    dirs = {"x": rng.standard_normal((d, npn)), "vp": rng.standard_normal((d, npn)),
            "v": rng.standard_normal((d, nc)), "F": rng.standard_normal((d * d, nc)), "e": rng.standard_normal(nc)}
    scale = {"x": 1e-5 * h, "vp": 1e-6, "v": 1e-6, "F": 1e-6, "e": 1e-6}
    fields = {"x": (L.FIELD_X, x0), "vp": (L.FIELD_VP, vp0), "v": (L.FIELD_V, v0), "F": (L.FIELD_F, F0),
              "e": (L.FIELD_E, e0)}
    for k, (fid, val) in fields.items():
        dk = dirs[k]

        def make(e, fid=fid, val=val, dk=dk):
            return pb, (lambda s: s.set(fid, val + e * dk))
        fd = _fd(pb, n, prm, lam, masks, make, scale[k], pre=pre)
        ad = float((g[k] * dk).sum())
        assert _rel(ad, fd) <= 1e-6, (k, ad, fd)


def test_adjoint_vs_oracle_fd():
    """The CUDA adjoint against finite differences of the CPU oracle (an independent forward)."""
    pb, lam, rng = _setup(W.plain2d(n=8), 17)
    n = 4
    prm = {"dt_fixed": _dt_fixed(pb), "mood": 0}
    st, tape, g = _grad(pb, n, prm, lam)
    dv = rng.standard_normal(pb.v.shape)
    dmu = rng.standard_normal(pb.mesh.n_cells)
    ofields = (("x", O.F_X), ("vp", O.F_VP), ("v", O.F_V), ("F", O.F_F), ("e", O.F_E))

    def Jo(p):
        o = O.Oracle(p, **prm)
        for _ in range(n):
            o.step()
        return {k: o.get(fid) for k, fid in ofields}
    for name, d, eps, ad in (("v", dv, 1e-6, float((g["v"] * dv).sum())),
                             ("mu", dmu, 1e-6, float((g["mu"] * dmu).sum()))):
        plus = Jo(dataclasses.replace(pb, **{name: getattr(pb, name) + eps * d}))
        minus = Jo(dataclasses.replace(pb, **{name: getattr(pb, name) - eps * d}))
        fd = sum(float(((plus[k] - minus[k]) * lam[k]).sum()) for k in lam) / (2 * eps)
        assert _rel(ad, fd) <= 1e-6, (name, ad, fd)


def test_checkpoint_interval_is_bitwise_invariant():
    pb, lam, _ = _setup(W.impact2d(n=16), 18)
    prm = {"dt_fixed": _dt_fixed(pb)}
    n = 7
    ref = None
    for C in (0, 1, 2, 3, 7, 100):
        _, tape, g = _grad(pb, n, prm, lam, ckpt=C)
        assert tape.info()["checkpoint_every"] == min(C, n)
        if ref is None:
            ref = g
        else:
            for k in ref:
                assert np.array_equal(ref[k], g[k]), (C, k)


def test_backward_restores_the_state_and_repeats():
    for C in (0, 2):
        _restore_case(C)


def _restore_case(C):
    pb, lam, _ = _setup(W.plain2d(n=12), 19)
    st = L.simulation(pb)
    twin = L.simulation(pb)
    tape = L.Tape(st, 4, C)
    twin.run(4)
    before = {f: st.get(f) for f in (L.FIELD_X, L.FIELD_VP, L.FIELD_V, L.FIELD_E, L.FIELD_F, L.FIELD_TAU,
                                      L.FIELD_DT, L.FIELD_ORDER)}
    g1 = tape.backward(lam_x=lam["x"], lam_v=lam["v"])
    g2 = tape.backward(lam_x=lam["x"], lam_v=lam["v"])
    for k in g1:
        assert np.array_equal(g1[k], g2[k]), k
    for f, a in before.items():
        assert np.array_equal(st.get(f), a), f
    st.run(3)
    twin.run(3)
    for f in (L.FIELD_X, L.FIELD_V, L.FIELD_F, L.FIELD_E):
        assert np.array_equal(st.get(f), twin.get(f)), f


def test_backward_linear_in_the_adjoints():
    pb, lam, rng = _setup(W.cube3d(n=3), 20)
    _, tape, _ = _grad(pb, 3, {}, lam)
    ga = tape.backward(lam_v=lam["v"])
    gb = tape.backward(lam_F=lam["F"])
    gab = tape.backward(lam_v=lam["v"], lam_F=lam["F"])
    for k in ga:
        np.testing.assert_allclose(gab[k], ga[k] + gb[k], rtol=1e-12, atol=1e-12 * np.abs(gab[k]).max())
    g0 = tape.backward()
    for k in g0:
        assert not np.any(g0[k]), k


def test_torch_rollout_autograd():
    import torch
    pb, lam, rng = _setup(W.plain2d(n=10), 21)
    prm = {"dt_fixed": _dt_fixed(pb)}
    n = 4
    dev = "cuda"
    v0 = torch.tensor(pb.v, dtype=torch.float64, device=dev, requires_grad=True)
    mu = torch.tensor(pb.mu, dtype=torch.float64, device=dev, requires_grad=True)
    F0 = torch.tensor(pb.F, dtype=torch.float64, device=dev, requires_grad=True)
    w = torch.tensor(lam["x"], device=dev)
    x, vp, v, F = L.rollout(pb, n, v0, mu, F0, checkpoint_every=2, **prm)
    loss = (v * v).sum() + (x * w).sum() + F.sum()
    loss.backward()
    # the same gradient from the tape with the adjoints written out
    st = L.simulation(pb, **prm)
    tape = L.Tape(st, n)
    vN = st.get(L.FIELD_V)
    g = tape.backward(lam_x=lam["x"], lam_v=2 * vN, lam_F=np.ones((pb.mesh.dim ** 2, pb.mesh.n_cells)))
    np.testing.assert_allclose(v0.grad.cpu().numpy(), g["v"], rtol=1e-12, atol=1e-14 * np.abs(g["v"]).max())
    np.testing.assert_allclose(mu.grad.cpu().numpy(), g["mu"], rtol=1e-12, atol=1e-14 * np.abs(g["mu"]).max())
    np.testing.assert_allclose(F0.grad.cpu().numpy(), g["F"], rtol=1e-12, atol=1e-14 * np.abs(g["F"]).max())
    # and a finite difference of the rollout along v0
    d = torch.tensor(rng.standard_normal(pb.v.shape), device=dev)
    eps = 1e-6
    with torch.no_grad():
        xp_, _, vp_, Fp_ = L.rollout(pb, n, v0 + eps * d, mu, F0, **prm)
        xm_, _, vm_, Fm_ = L.rollout(pb, n, v0 - eps * d, mu, F0, **prm)
        fd = float(((vp_ - vm_) * (vp_ + vm_)).sum() + ((xp_ - xm_) * w).sum() + (Fp_ - Fm_).sum()) / (2 * eps)
    ad = float((v0.grad * d).sum())
    assert _rel(ad, fd) <= 1e-6, (ad, fd)


def test_state_init_from_device_tensors():
    """lmood_state_init_device (the rollout's path: the initial data stay on the device) gives
    the state lmood_state_init gives from the same values in host memory, bitwise, and refuses
    a non-positive mu on the device"""
    import torch
    pb, lam, rng = _setup(bc_case("piston2d"), 27)
    host = L.simulation(pb)
    m = pb.mesh
    mesh = L.Mesh(m.dim, m.x, m.c2n, m.bface, m.btag)
    mesh.set_bc_values(pb.bcval)
    dev = L.State(mesh, pb.rho0, pb.lam, torch.tensor(pb.mu, device="cuda"), torch.tensor(pb.v, device="cuda"),
                  torch.tensor(pb.F, device="cuda"), L.params_default(m.dim, cfl=pb.cfl))
    for _ in range(2):
        for k, fid in OUT_FIELDS:
            assert np.array_equal(host.get(fid), dev.get(fid)), k
        host.step()
        dev.step()
    bad = np.array(pb.mu)
    bad[5] = 0.0
    with pytest.raises(L.LmoodError) as e:
        L.State(mesh, pb.rho0, pb.lam, torch.tensor(bad, device="cuda"), torch.tensor(pb.v, device="cuda"), None,
                L.params_default(m.dim, cfl=pb.cfl))
    assert e.value.status == L.ERR_ARG


def test_torch_rollout_boundary_faces():
    """the rollout on a problem with prescribed-velocity faces (the piston): gradients of v0 and
    mu equal the tape's"""
    import torch
    pb, lam, rng = _setup(bc_case("piston2d"), 28)
    n = 4
    v0 = torch.tensor(pb.v, dtype=torch.float64, device="cuda", requires_grad=True)
    mu = torch.tensor(pb.mu, dtype=torch.float64, device="cuda", requires_grad=True)
    x, vp, v, F = L.rollout(pb, n, v0, mu, torch.tensor(pb.F, device="cuda"), checkpoint_every=2)
    ((v * v).sum() + x.sum()).backward()
    st = L.simulation(pb)
    tape = L.Tape(st, n)
    g = tape.backward(lam_x=np.ones((pb.mesh.dim, pb.mesh.n_nodes)), lam_v=2 * st.get(L.FIELD_V))
    np.testing.assert_allclose(v0.grad.cpu().numpy(), g["v"], rtol=1e-12, atol=1e-14 * np.abs(g["v"]).max())
    np.testing.assert_allclose(mu.grad.cpu().numpy(), g["mu"], rtol=1e-12, atol=1e-14 * np.abs(g["mu"]).max())


def test_tape_errors():
    pb = W.plain2d(n=6)
    st = L.simulation(pb)
    with pytest.raises(L.LmoodError) as e:
        L.Tape(st, 0)
    assert e.value.status == L.ERR_ARG
    with pytest.raises(L.LmoodError) as e:
        L.Tape(st, 2, -1)
    assert e.value.status == L.ERR_ARG
