"""Host logic of bench.py on the CPU: the reference arm (the oracle over the run's own warm-up
and timed steps, each the workload's first time step from its initial data, the state restored
before each) and the FP64 counts per cell that its roofline uses, which belong to the kernel
sources they were captured on."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_steps_restore_the_initial_state(orc):
    sys.path.insert(0, ROOT)
    import bench
    import workloads as W
    pb = W.plain2d()
    r = bench.reference_steps(pb, steps=3, warmup=2)
    assert r["kind"] == "oracle" and r["unit"] == "cell-steps/s" and r["cores"] >= 1
    assert r["value"] > 0 and r["ms_per_step"] > 0
    assert r["value"] == pytest.approx(pb.mesh.n_cells * 1e3 / r["ms_per_step"], rel=1e-12)
    assert "each of the 3 timed steps (after 2 untimed)" in r["sample"]

    # what every sampled step computes: one step from the initial data, whatever ran before
    a = orc.Oracle(pb)
    s0, dt0 = a.state(), a.dt
    a.step()
    first = a.state()
    b = orc.Oracle(pb)
    b.step(3)
    b.set_state(x=s0["x"], vp=s0["vp"], v=s0["v"], e=s0["e"], F=s0["F"], dt=dt0)
    b.step()
    again = b.state()
    for k in ("x", "vp", "v", "e", "F"):
        assert np.array_equal(first[k], again[k]), k
    a.close()
    b.close()



def test_fp64_counts_belong_to_the_current_kernel_sources():
    """the roofline's FP64 FLOP / instruction counts per cell and the DRAM bytes per cell were
    captured on the kernel sources whose digest COUNTS_SRC records: a kernel change without a new
    capture would make the bench report stale counts ("counts_stale")"""
    sys.path.insert(0, ROOT)
    import bench
    digest = bench.kernel_source_digest()
    for dim in (2, 3):
        assert bench.COUNTS_SRC[dim] == digest, dim
        for table in (bench.FP64_FLOP_PER_CELL, bench.FP64_INSTR_PER_CELL, bench.TRAFFIC_PER_CELL):
            assert set(table[dim]) == {"predict", "update", "nodes", "moments"}
        for k, flop in bench.FP64_FLOP_PER_CELL[dim].items():
            # one instruction is 1 (add, mul) or 2 (fma) FLOP
            assert bench.FP64_INSTR_PER_CELL[dim][k] <= flop <= 2 * bench.FP64_INSTR_PER_CELL[dim][k]
