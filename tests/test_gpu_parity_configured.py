"""Parity of the CUDA path with the oracle over the configured run lengths at full size
(-m gpu; opt-in: set LMOOD_CONFIGURED_RUNS=1, since the oracle takes minutes to tens of
minutes of host time for them).

The oracle advances along its own trajectory from the seeded initial data; a free-running
CUDA state takes the same steps. Its MOOD masks must equal the oracle's after every step and
its state must be within 1e-8 (relative, field-wise) after the run and at checkpoints along
it; a second CUDA state set to the oracle's state at intervals must take that step within
1e-11 of the oracle's step (the per-step bar, field-wise; per component within 1e-10). Configurations: the 2D impact (999,698
triangles, 2000 steps), the 3D cube of the adjoint configuration (511,104 tetrahedra, 400
steps), the 256-instance batch's smallest, largest and two random instances (500 steps, the
batch free-running), and the bending column (5,989,500 tetrahedra) over its first 100 steps
of 500 (the oracle recomputes the whole column for every MOOD round of its later steps).
"""
import os

import numpy as np
import pytest

import oracle as O
import paper_2104_02139_gb300 as L
import workloads as W
from parity_util import push_oracle_state, relerr, step_errors

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(os.environ.get("LMOOD_CONFIGURED_RUNS") != "1",
                                 reason="long: set LMOOD_CONFIGURED_RUNS=1 to run the configured lengths")]

# the state's relative error per step (field-wise) and after the run; each component of a
# field on its own scale (rows) is reported and held to TOL_ROWS: in the column the transverse
# rows of v_p and v*_p are far smaller than the lateral one, and its rounding shows at
# ~1e-11 of them
TOL_STEP, TOL_RUN, TOL_ROWS = 1e-11, 1e-8, 1e-10
STATE = ((L.FIELD_X, O.F_X), (L.FIELD_VP, O.F_VP), (L.FIELD_V, O.F_V), (L.FIELD_E, O.F_E), (L.FIELD_F, O.F_F),
         (L.FIELD_TAU, O.F_TAU))


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available()
    L.build()
    O.build()


def _configured(pb, n, resync_every, check_every):
    o = O.Oracle(pb)
    g = L.simulation(pb)
    h = L.simulation(pb)
    worst_step, worst_rows, worst_run, troubled, rounds = 0.0, 0.0, 0.0, 0, 0
    for s in range(n):
        before = push_oracle_state(h, o) if s % resync_every == resync_every - 1 else None
        ig = g.step()
        o.step()
        troubled += o.info.n_troubled
        rounds += o.info.mood_iters
        mg, mo = g.get(L.FIELD_ORDER).astype(int), o.get(O.F_ORDER).astype(int)
        assert np.array_equal(mg, mo), (s + 1, int((mg != mo).sum()))
        assert ig.n_troubled == o.info.n_troubled, s + 1
        if before is not None:
            h.step()
            err = step_errors(h, o, before)
            err["dt"] = abs(h.get(L.FIELD_DT)[0] - o.dt) / o.dt
            fw = max(v for k, v in err.items() if not k.endswith("_rows"))
            rw = max(v for k, v in err.items() if k.endswith("_rows"))
            assert fw <= TOL_STEP and rw <= TOL_ROWS, (s + 1, err)
            worst_step, worst_rows = max(worst_step, fw), max(worst_rows, rw)
        if (s + 1) % check_every == 0 or s == n - 1:
            e = max(relerr(g.get(fg), o.get(fo)) for fg, fo in STATE)
            assert e <= TOL_RUN, (s + 1, e)
            worst_run = max(worst_run, e)
    return worst_step, worst_run, troubled, rounds, e, worst_rows


def _report(name, n, r):
    print(f"{name} {n} steps: state after the run {r[4]:.2e} (worst along it {r[1]:.2e}), per-step worst "
          f"{r[0]:.2e} (per component {r[5]:.2e}), troubled cell-events {r[2]}, MOOD rounds {r[3]}, masks "
          f"identical at every step")


def test_impact2d_2000_steps():
    r = _configured(W.impact2d(), 2000, 100, 200)
    _report("impact2d (999,698 triangles)", 2000, r)


def test_cube3d_400_steps():
    r = _configured(W.cube3d(), 400, 40, 40)
    _report("cube3d (511,104 tets)", 400, r)


def test_column3d_first_100_steps():
    r = _configured(W.column3d(), 100, 25, 25)
    _report("column3d (5,989,500 tets)", 100, r)


def test_batch_sampled_instances_500_steps():
    """the batch free-running for 500 steps; the sampled instances' slices against their
    oracles (masks every step, state after the run)"""
    probs = W.batched2d()
    pb, inst = W.concat(probs)
    b = L.simulation(pb, cell_inst=inst, n_inst=len(probs))
    cells = np.asarray(pb.meta["cells"])
    c_off = np.concatenate([[0], np.cumsum(cells)])
    n_off = np.concatenate([[0], np.cumsum(pb.meta["nodes"])])
    rng = np.random.default_rng(12)
    pick = sorted({int(cells.argmin()), int(cells.argmax()), *rng.choice(len(probs), 2, replace=False).tolist()})
    oracles = {i: O.Oracle(probs[i]) for i in pick}
    troubled = 0
    for s in range(500):
        b.step()
        order = b.get(L.FIELD_ORDER).astype(int)
        for i, o in oracles.items():
            o.step()
            troubled += o.info.n_troubled
            assert np.array_equal(order[c_off[i]:c_off[i + 1]], o.get(O.F_ORDER).astype(int)), (s + 1, i)
    worst = 0.0
    for fg, fo in STATE:
        a = b.get(fg)
        node = fg in (L.FIELD_X, L.FIELD_VP)
        for i, o in oracles.items():
            sl = slice(n_off[i], n_off[i + 1]) if node else slice(c_off[i], c_off[i + 1])
            e = relerr(a[..., sl], o.get(fo))
            assert e <= TOL_RUN, (i, fg, e)
            worst = max(worst, e)
    print(f"batch instances {pick} ({[int(cells[i]) for i in pick]} cells), 500 steps free-running: state after "
          f"the run {worst:.2e}, troubled cell-events {troubled}, masks identical at every step")
