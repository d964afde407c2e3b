"""The stiffened-gas volumetric law (Eq. EOS_stiffened_gas; reading R18) on the CUDA path
against the oracle (-m gpu): identical MOOD masks, state error <= 1e-11 after one step and
<= 1e-8 over the run; parameter checks (its adjoint is checked with the adjoint tests)."""
import dataclasses

import numpy as np
import pytest

import oracle as O
import paper_2104_02139_gb300 as L
import workloads as W
from parity_util import Pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available()
    L.build()
    O.build()


def _wave2d(n=24, gamma=2.2, pinf=1.0, p0=0.3, V=0.02, a=-1.0):
    bc = {"x0": W.VELOCITY, "y0": W.SLIP, "y1": W.SLIP, "x1": W.PRESSURE}
    m = W.tri_mesh(n, 11, bc=bc)
    val = W.side_values(m, W.VELOCITY, (V, 0.0)) + W.side_values(m, W.PRESSURE, (p0, 0.0))
    return W.Problem("sgwave", m, 1.0, 0.0, np.full(m.n_cells, 0.1), np.zeros((2, m.n_cells)), 0.4, 10,
                     bcval=val, stiffened_gas=(gamma, pinf, p0), shear_a=a)


@pytest.mark.parametrize("a", [-1.0, 0.0])
def test_stiffened_gas_wave_parity(a):
    st = Pair(_wave2d(a=a)).run_compare(60)
    assert st["worst"] <= 1e-8


def test_stiffened_gas_swirl_2d_and_3d_parity():
    m = W.tri_mesh(16, 5, bc={k: W.SLIP for k in ("x0", "x1", "y0", "y1")})
    pts = m.x[:, m.c2n].mean(axis=1)
    v = 0.2 * np.stack([np.sin(np.pi * pts[0]) * np.cos(np.pi * pts[1]), -np.cos(np.pi * pts[0]) * np.sin(np.pi * pts[1])])
    pb = W.Problem("sgbox", m, 1.0, 0.0, np.full(m.n_cells, 0.3), v, 0.4, 10, stiffened_gas=(2.2, 1.0, 0.2))
    Pair(pb).run_compare(40)
    pb3 = dataclasses.replace(W.cube3d(n=5), stiffened_gas=(1.8, 2.0, 0.5))
    pb3.v *= 4
    Pair(pb3).run_compare(20)


def test_jelly_drop_parity():
    """the paper's last configuration on a box: stiffened gas, symmetry walls, contact floor"""
    for a in (-1.0, 0.0):
        pb = W.jellydrop3d(n=5, shear_a=a)
        p = Pair(pb)
        p.run_compare(40)
        z = p.g.get(L.FIELD_X)[2] + 2e-4  # distance to the floor
        assert z.min() < pb.contact[1]  # touched down
        assert z.min() >= pb.contact[1] - 2.0 * p.o.dt - 1e-12


def test_stiffened_gas_arguments_and_adjoint():
    with pytest.raises(L.LmoodError) as e:
        L.simulation(dataclasses.replace(_wave2d(n=6), stiffened_gas=(1.0, 1.0, 0.0)))
    assert e.value.status == L.ERR_ARG
    with pytest.raises(L.LmoodError) as e:
        L.simulation(dataclasses.replace(_wave2d(n=6), stiffened_gas=(2.0, 1.0, -2.0)))
    assert e.value.status == L.ERR_ARG
    m = W.tri_mesh(6, 2, bc={k: W.SLIP for k in ("x0", "x1", "y0", "y1")})
    pb = W.Problem("sg", m, 1.0, 0.0, np.full(m.n_cells, 0.3), np.zeros((2, m.n_cells)), 0.4, 2,
                   stiffened_gas=(2.2, 1.0, 0.0))
    st = L.simulation(pb)
    g = L.Tape(st, 2).backward(lam_e=np.ones(m.n_cells))  # e carries an adjoint: it enters p
    assert np.isfinite(g["mu"]).all() and np.abs(g["F"]).max() > 0.0 and not np.any(g["e"])
