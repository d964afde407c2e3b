"""CUDA path vs the CPU oracle on the paper's beryllium plate (Sect. "Elastic vibration of a
beryllium plate"; -m gpu): free boundaries, the paper's material scale (E = 3.2e11 Pa,
rho0 = 1845) and amplitude, the three-level cascade; 60 steps of 1,200 triangles (12,752
troubled cell-events, 6,250 P0 and 252 limited updates) with identical MOOD order masks at every
step and a state within 1e-11 after one step and 1e-8 over the run."""
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


def test_be_plate_parity():
    stats = Pair(W.be_plate(nx=61, ny=11), cascade=3).run_compare(60)
    assert stats["troubled"] > 0

