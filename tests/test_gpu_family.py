"""The shear energy family of Eq. familiy_energies (a != -1) on the CUDA path against the
oracle (-m gpu): identical MOOD masks, state error <= 1e-11 after one step and <= 1e-8 over
the run; the material range check; the adjoint's refusal."""
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


def _strained_block(n, a, seed=2):
    m = W.tri_mesh(n, seed, bc={k: W.SLIP for k in ("x0", "x1", "y0", "y1")})
    rng = np.random.default_rng(seed)
    F = np.zeros((4, m.n_cells))
    F[0] = 1.0 + 0.05 * rng.standard_normal(m.n_cells)
    F[3] = 1.0 + 0.05 * rng.standard_normal(m.n_cells)
    F[1] = 0.03 * rng.standard_normal(m.n_cells)
    return W.Problem("fam", m, 1.0, 2.0, np.full(m.n_cells, 1.0), np.zeros((2, m.n_cells)), 0.4, 10, F=F, shear_a=a)


@pytest.mark.parametrize("a", [0.0, 0.5])
def test_family_2d_parity(a):
    Pair(_strained_block(16, a)).run_compare(40)
    pb = dataclasses.replace(W.impact2d(n=40), shear_a=a)
    st = Pair(pb).run_compare(30)
    assert st["troubled"] > 0


def test_family_3d_parity():
    pb = W.cube3d(n=5)
    pb = dataclasses.replace(pb, v=pb.v * 4, shear_a=0.0)
    Pair(pb).run_compare(20)


def test_family_differs_from_neo_hookean():
    a = L.simulation(_strained_block(12, 0.0))
    b = L.simulation(_strained_block(12, -1.0))
    a.run(5)
    b.run(5)
    assert np.abs(a.get(L.FIELD_V) - b.get(L.FIELD_V)).max() > 1e-6


def test_family_range_and_adjoint():
    """a outside [-1, 1/2] is refused; a tape of the family records and runs backward (its
    gradients are checked against the oracle's tangent and finite differences in the adjoint
    tests)"""
    with pytest.raises(L.LmoodError) as e:
        L.simulation(_strained_block(6, 0.7))
    assert e.value.status == L.ERR_ARG
    st = L.simulation(_strained_block(6, 0.0))
    g = L.Tape(st, 2).backward(lam_v=np.ones((2, st.mesh.n_cells)))
    assert np.isfinite(g["mu"]).all() and np.abs(g["v"]).max() > 0.0
