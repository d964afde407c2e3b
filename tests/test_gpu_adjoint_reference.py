"""The CUDA adjoint against independent references (-m gpu).

1. The oracle's tangent build (the oracle's own source compiled with dual numbers, a CPU
   forward-mode derivative of the same frozen-mask map that shares nothing with the CUDA
   adjoint): for seeded adjoints lam of the final state (x, v_p, v, F, e) and seeded
   directions delta of the initial v0, mu, F0 and node positions (at fixed masses, through the
   initial nodal solve), <grad, delta> from the tape's reverse pass must equal <lam, J delta>
   from the tangent to 1e-6 relative, over 12 steps with MOOD active (first-order cells in the
   masks) and the adaptive dt: in 2D (slip walls; the impact against a wall) and 3D (slip
   walls; the clamped column); with traction, pressure and prescribed-velocity faces and
   contact walls (the piston, a block rebounding on a wall, a block under pressure and
   traction, a 3D box with every kind of face); with the shear energy family (a = 0, a = 0.5);
   with the stiffened gas (a 2D piston against a pressure; a 3D block on a contact floor); and
   with the three-level cascade, whose limited level (Barth-Jespersen slopes) is differentiated
   with the limiter's choices frozen (the impact in 2D, the column in 3D).
   The two runs' masks must be identical at every step and their dt equal to 1e-12, so both
   differentiate the same map.
2. The adjoint configuration at full size (511,104 tetrahedra, 400 steps, a checkpoint every
   20 steps): the gradient of J = sum over cells with initial centroid z > 0.5 of m |v|^2 / 2
   along two random directions of v0 and two of mu (each cell's mu direction scaled by its mu,
   so that the step h = 1e-6 is relative), against central differences through the tape's
   replay (the recorded masks and dt), to 1e-6 relative.
"""
import dataclasses

import numpy as np
import pytest

import oracle as O
import paper_2104_02139_gb300 as L
import workloads as W
from adjoint_cases import bc_case, family_case, sg_case, smooth_positions_direction

pytestmark = pytest.mark.gpu

STATE = (("x", L.FIELD_X), ("vp", L.FIELD_VP), ("v", L.FIELD_V), ("F", L.FIELD_F))


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available()
    L.build()
    O.build()


def _case(name):
    if name == "plain2d":
        pb = W.plain2d(n=12)
        pb.v *= 40.0
    elif name == "impact2d":
        pb = W.impact2d(n=20)
    elif name == "cube3d":
        pb = W.cube3d(n=4)
        pb.v *= 4.0
    elif name == "column3d":
        pb = W.column3d(nxy=3, nz=12)
        pb.v *= 8.0
    elif name in ("cube3d_a0", "impact2d_a05"):
        pb = family_case(name)
    elif name in ("sgwave2d", "sgdrop3d"):
        pb = sg_case(name)
    elif name == "impact2d_bj":
        # (a uniform field would give the oracle slopes of exactly zero where the GPU's are at
        # rounding level: at that tie the limiter's branch, and so the one-sided derivative,
        # differ; small noise in v0 removes the ties)
        pb = W.impact2d(n=20)
        pb.v = pb.v + 1e-3 * np.random.default_rng(5).standard_normal(pb.v.shape)
    elif name == "column3d_bj":
        pb = W.column3d(nxy=3, nz=12)
        pb.v *= 8.0
    else:
        pb = bc_case(name)
    return pb


def _perturbed_material(pb, rng):
    """heterogeneous mu and a non-trivial initial F"""
    d, nc = pb.mesh.dim, pb.mesh.n_cells
    F = np.zeros((d * d, nc))
    for a in range(d):
        F[a * d + a] = 1.0
    F += 0.01 * rng.standard_normal((d * d, nc))
    mu = np.asarray(pb.mu, dtype=float) * (1.0 + 0.1 * rng.random(nc))
    return dataclasses.replace(pb, F=F, mu=mu)


@pytest.mark.parametrize("name", ["plain2d", "impact2d", "cube3d", "column3d", "piston2d", "rebound2d",
                                  "pressure_traction2d", "box3d_bc", "cube3d_a0", "impact2d_a05", "sgwave2d",
                                  "sgdrop3d", "impact2d_bj", "column3d_bj"])
def test_adjoint_matches_the_oracle_tangent(name):
    rng = np.random.default_rng(31)
    pb = _perturbed_material(_case(name), rng)
    prm = {"cascade": 3} if name.endswith("_bj") else {}  # the three-level cascade
    n = 12
    d, nc, npn = pb.mesh.dim, pb.mesh.n_cells, pb.mesh.n_nodes
    lam = {"x": rng.standard_normal((d, npn)), "vp": rng.standard_normal((d, npn)),
           "v": rng.standard_normal((d, nc)), "F": rng.standard_normal((d * d, nc)), "e": rng.standard_normal(nc)}
    st = L.simulation(pb, **prm)
    tape = L.Tape(st, n, 4)
    g = tape.backward(lam_x=lam["x"], lam_vp=lam["vp"], lam_v=lam["v"], lam_F=lam["F"], lam_e=lam["e"])
    twin = L.simulation(pb, **prm)
    masks, dts = [], []
    for _ in range(n):
        dts.append(twin.step().dt_used)
        masks.append(twin.get(L.FIELD_ORDER).astype(np.int8))
    dirs = {"v": rng.standard_normal((d, nc)), "mu": rng.standard_normal(nc) * pb.mu,
            "F": rng.standard_normal((d * d, nc)), "x": smooth_positions_direction(pb.mesh)}
    out = {}
    for k, delta in dirs.items():
        t = O.tangent(pb, n, **{"d" + k: delta}, **prm)
        for s in range(n):
            assert np.array_equal(t["masks"][s], masks[s]), f"step {s}: the oracle's mask differs from the GPU's"
            assert abs(t["dts"][s] - dts[s]) <= 1e-12 * dts[s], (s, t["dts"][s], dts[s])
        ref = sum(float((t["d" + f] * lam[f]).sum()) for f in lam)
        ad = float((g[k] * delta).sum())
        rel = abs(ad - ref) / max(abs(ad), abs(ref))
        out[k] = rel
        assert rel <= 1e-6, (name, k, ad, ref)
    p0 = sum(int((m == 1).sum()) for m in masks)
    assert p0 > 0, "no first-order cell in the recorded masks: the mixed mask is not exercised"
    if prm:
        lim = sum(int((m == 3).sum()) for m in masks)
        assert lim > 0, "no cell at the limited level in the recorded masks"
        print(f"  ({lim} cell-steps at the limited level)")
    print(f"adjoint vs oracle tangent, {name} ({nc} cells, {n} steps, {p0} first-order cell-steps): "
          + ", ".join(f"{k} {v:.1e}" for k, v in out.items()))


def test_adjoint_configuration_full_size_against_central_differences():
    pb = W.cube3d()
    n, ckpt, h = 400, 20, 1e-6
    d, nc = pb.mesh.dim, pb.mesh.n_cells
    zc = pb.mesh.x[2][pb.mesh.c2n].mean(axis=0)  # initial centroid height of each cell
    st = L.simulation(pb)
    tape = L.Tape(st, n, ckpt)
    m = st.get(L.FIELD_MASS)
    w = np.where(zc > 0.5, m, 0.0)
    vN = st.get(L.FIELD_V)
    J = float((0.5 * w * (vN * vN).sum(0)).sum())
    g = tape.backward(lam_v=w * vN)
    rng = np.random.default_rng(41)
    cases = [("v", rng.standard_normal((d, nc))) for _ in range(2)]
    cases += [("mu", rng.standard_normal(nc) * pb.mu) for _ in range(2)]  # h relative to mu
    res = []
    for k, delta in cases:
        vs = []
        for sgn in (1.0, -1.0):
            base = pb.v if k == "v" else pb.mu
            s2 = L.simulation(dataclasses.replace(pb, **{k: base + sgn * h * delta}))
            tape.replay(s2)
            vs.append(s2.get(L.FIELD_V))
            s2.close()
            s2.mesh.close()
        fd = float((0.5 * w * ((vs[0] - vs[1]) * (vs[0] + vs[1])).sum(0)).sum()) / (2 * h)
        ad = float((g[k] * delta).sum())
        res.append((k, ad, fd, abs(ad - fd) / max(abs(ad), abs(fd))))
    print(f"adjoint configuration (511,104 tets, 400 steps, checkpoint every 20), J = {J:.6e}: "
          + "; ".join(f"d{k}: adjoint {a:.6e} FD {f:.6e} rel {r:.1e}" for k, a, f, r in res))
    for k, ad, fd, rel in res:
        assert rel <= 1e-6, (k, ad, fd, rel)
