"""lmood_totals_noalloc -- the totals reduction for callers that do not let the library
allocate device memory (their application owns every device allocation) -- against the
allocating lmood_totals, through the C ABI, on two calls in a row (-m gpu). Collected last on
purpose: it shares a file-scope device scratch array with nothing else, and runs the same
whether alone in a fresh process or after the other tests."""
import ctypes as C

import numpy as np
import pytest

import paper_2104_02139_gb300 as L
import workloads as W

pytestmark = pytest.mark.gpu


def _device_fields(sim, torch):
    n = sim.mesh.n_cells
    d = sim.mesh.dim
    m = torch.empty(n, dtype=torch.float64, device="cuda")
    v = torch.empty((d, n), dtype=torch.float64, device="cuda")
    e = torch.empty(n, dtype=torch.float64, device="cuda")
    sim.get(L.FIELD_MASS, out=m)
    sim.get(L.FIELD_V, out=v)
    sim.get(L.FIELD_E, out=e)
    return m, v, e


@pytest.mark.parametrize("case", ["impact2d", "cube3d"])
def test_totals_noalloc_matches_totals(case):
    import torch
    L.build()
    lib = L.lib()
    pb = W.impact2d(n=120) if case == "impact2d" else W.cube3d(n=6)
    sim = L.simulation(pb, stream=0)
    for call in range(2):
        sim.run(2)
        ref = sim.totals()
        m, v, e = _device_fields(sim, torch)
        out = torch.full((5,), float("nan"), dtype=torch.float64, device="cuda")
        rc = lib.lmood_totals_noalloc(pb.mesh.dim, pb.mesh.n_cells, C.c_void_p(m.data_ptr()),
                                      C.c_void_p(v.data_ptr()), C.c_void_p(e.data_ptr()),
                                      C.c_void_p(out.data_ptr()), None)
        assert rc == L.OK, lib.lmood_last_error()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        scale = np.abs(ref).max()
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-14 * scale)


def test_totals_noalloc_rejects_oversize_and_bad_args():
    import torch
    L.build()
    lib = L.lib()
    buf = torch.zeros(8, dtype=torch.float64, device="cuda")
    p = C.c_void_p(buf.data_ptr())
    assert lib.lmood_totals_noalloc(2, 16_777_217, p, p, p, p, None) == L.ERR_ARG
    assert b"no-allocation limit" in lib.lmood_last_error()
    assert lib.lmood_totals_noalloc(4, 10, p, p, p, p, None) == L.ERR_ARG
    assert lib.lmood_totals_noalloc(2, 10, None, p, p, p, None) == L.ERR_ARG
    assert lib.lmood_totals_noalloc(2, 0, p, p, p, p, None) == L.ERR_ARG
