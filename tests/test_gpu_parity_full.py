"""Full-size parity of the CUDA path with the oracle over long stretches of the configured
runs (-m gpu).

Two bars, as the configurations state them: every step within 1e-11 (relative, identical
MOOD masks), and the state within 1e-8 after a run. The oracle always advances along its own
trajectory from the seeded initial data (nothing flows from the CUDA path into it). The
per-step bar is checked on a second CUDA state that is set to the oracle's state (x, v_p, v,
e, F and the next dt, through lmood_set_fields) before the compared step: both then take that
step from the same state, so the difference is that step's alone. Errors are measured
field-wise (max |g - o| / max |o|), per component (each row of a SoA field on its own scale)
and, for the nodes, on the nodal solver's velocity v*_p (the step's displacement over dt); all
three are held to 1e-11.
"""
import numpy as np
import pytest

import oracle as O
import paper_2104_02139_gb300 as L
import workloads as W
from parity_util import push_oracle_state, relerr, step_errors

pytestmark = pytest.mark.gpu

TOL_STEP = 1e-11


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available()
    L.build()
    O.build()


def _masks_equal(g, o, label):
    mg, mo = g.get(L.FIELD_ORDER).astype(int), o.get(O.F_ORDER).astype(int)
    if not np.array_equal(mg, mo):
        bad = np.where(mg != mo)[0]
        raise AssertionError(f"{label}: MOOD masks differ in {bad.size} cells, e.g. {bad[:8]}")


def _run(pb, n, resync_at, check_every):
    """The oracle advances n steps from the initial data. Beside it, a free CUDA state g takes
    the same n steps (masks compared after every step, state within 1e-8 every check_every
    steps), and a second CUDA state h is set to the oracle's state before each step in
    resync_at and takes that one step (within 1e-11 of the oracle's step, masks and step
    reports identical)."""
    o = O.Oracle(pb)
    g = L.simulation(pb)
    h = L.simulation(pb)
    worst_step, worst_run, troubled, resynced = 0.0, 0.0, 0, 0
    for s in range(n):
        before = push_oracle_state(h, o) if s in resync_at else None
        ig = g.step()
        o.step()
        troubled += o.info.n_troubled
        _masks_equal(g, o, f"free run, step {s + 1}")
        assert ig.n_troubled == o.info.n_troubled and ig.mood_iters == o.info.mood_iters, s
        if before is not None:
            ih = h.step()
            _masks_equal(h, o, f"step {s + 1} from the oracle's state")
            assert ih.n_troubled == o.info.n_troubled and ih.mood_iters == o.info.mood_iters, s
            err = step_errors(h, o, before)
            err["dt"] = abs(h.get(L.FIELD_DT)[0] - o.dt) / o.dt
            assert max(err.values()) <= TOL_STEP, (s + 1, err)
            worst_step = max(worst_step, max(err.values()))
            resynced += 1
        if (s + 1) % check_every == 0 or s == n - 1:
            e = max(relerr(g.get(fg), o.get(fo)) for fg, fo in ((L.FIELD_X, O.F_X), (L.FIELD_VP, O.F_VP),
                                                             (L.FIELD_V, O.F_V), (L.FIELD_E, O.F_E),
                                                             (L.FIELD_F, O.F_F), (L.FIELD_TAU, O.F_TAU)))
            assert e <= 1e-8, (s + 1, e)
            worst_run = max(worst_run, e)
    return {"worst_step": worst_step, "worst_run": worst_run, "troubled": troubled, "resynced": resynced}


def test_impact2d_full_size_200_steps():
    """999,698 triangles (the 2D impact configuration), 200 steps: every one of steps 1-50 and
    every 10th step after, taken from the oracle's state, within 1e-11 of the oracle's step;
    the free-running CUDA state's masks identical at every step and its state within 1e-8 at
    every 20th step and after step 200."""
    st = _run(W.impact2d(), 200, set(range(50)) | set(range(59, 200, 10)), 20)
    assert st["troubled"] > 0 and st["resynced"] == 65
    print(f"impact2d 200 steps: per-step worst {st['worst_step']:.2e} over {st['resynced']} steps, "
          f"free run worst {st['worst_run']:.2e}, troubled cell-events {st['troubled']}")


def test_cube3d_full_size_20_steps():
    """511,104 tetrahedra (the adjoint configuration's cube, heterogeneous mu): 20 steps, each
    from the oracle's state within 1e-11, free run within 1e-8 after them."""
    st = _run(W.cube3d(), 20, set(range(20)), 10)
    print(f"cube3d 20 steps: per-step worst {st['worst_step']:.2e}, free run worst {st['worst_run']:.2e}, "
          f"troubled {st['troubled']}")


def test_full_size_batch_sampled_instances_50_steps():
    """The 256-instance batch (11.6M cells, one launch per stage, own dt each): the smallest,
    the largest and two random instances follow their oracles. Before each of 50 steps the
    sampled instances' slices of the batch are set to their oracles' states (the other
    instances keep their own); each step is then within 1e-11 of the oracles' steps, masks
    identical."""
    import torch
    probs = W.batched2d()
    pb, inst = W.concat(probs)
    b = L.simulation(pb, cell_inst=inst, n_inst=len(probs))
    cells = np.asarray(pb.meta["cells"])
    c_off = np.concatenate([[0], np.cumsum(cells)])
    n_off = np.concatenate([[0], np.cumsum(pb.meta["nodes"])])
    rng = np.random.default_rng(12)
    pick = sorted({int(cells.argmin()), int(cells.argmax()), *rng.choice(len(probs), 2, replace=False).tolist()})
    oracles = {i: O.Oracle(probs[i]) for i in pick}
    fields = ((L.FIELD_X, O.F_X, "node"), (L.FIELD_VP, O.F_VP, "node"), (L.FIELD_V, O.F_V, "cell"),
              (L.FIELD_E, O.F_E, "cell"), (L.FIELD_F, O.F_F, "cell"))
    dev = {fg: torch.empty(b.shape(fg), dtype=torch.float64, device="cuda") for fg, _, _ in fields}
    worst, troubled = 0.0, 0
    for s in range(50):
        b.get_fields(dev)
        dt = b.get(L.FIELD_DT)
        for i, o in oracles.items():
            cs, ns = slice(c_off[i], c_off[i + 1]), slice(n_off[i], n_off[i + 1])
            for fg, fo, kind in fields:
                dev[fg][..., ns if kind == "node" else cs] = torch.as_tensor(o.get(fo), device="cuda")
            dt[i] = o.dt
        b.set_fields(dev)
        b.set(L.FIELD_DT, dt)
        b.step()
        after = {fg: b.get(fg) for fg in (L.FIELD_X, L.FIELD_VP, L.FIELD_V, L.FIELD_E, L.FIELD_F, L.FIELD_TAU,
                                          L.FIELD_VSTAR)}
        order = b.get(L.FIELD_ORDER).astype(int)
        dt1 = b.get(L.FIELD_DT)
        for i, o in oracles.items():
            o.step()
            troubled += o.info.n_troubled
            cs, ns = slice(c_off[i], c_off[i + 1]), slice(n_off[i], n_off[i + 1])
            assert np.array_equal(order[cs], o.get(O.F_ORDER).astype(int)), (s, i)
            for fg, fo in ((L.FIELD_X, O.F_X), (L.FIELD_VP, O.F_VP), (L.FIELD_V, O.F_V), (L.FIELD_E, O.F_E),
                           (L.FIELD_F, O.F_F), (L.FIELD_TAU, O.F_TAU), (L.FIELD_VSTAR, O.F_VSTAR)):
                node = fg in (L.FIELD_X, L.FIELD_VP, L.FIELD_VSTAR)
                g = after[fg][..., ns] if node else after[fg][..., cs]
                e = relerr(g, o.get(fo))
                worst = max(worst, e)
                assert e <= TOL_STEP, (s, i, fg, e)
            assert abs(dt1[i] - o.dt) <= TOL_STEP * o.dt, (s, i)
    assert troubled > 0
    print(f"batch instances {pick}: 50 steps from their oracles' states, worst {worst:.2e}, troubled {troubled}")
