"""Side-by-side stepping of the CUDA library and the CPU oracle on the same seeded inputs."""
from __future__ import annotations

import numpy as np

import oracle as O
import paper_2104_02139_gb300 as L

FIELDS = (("x", O.F_X, L.FIELD_X), ("vp", O.F_VP, L.FIELD_VP), ("v", O.F_V, L.FIELD_V),
          ("e", O.F_E, L.FIELD_E), ("F", O.F_F, L.FIELD_F), ("tau", O.F_TAU, L.FIELD_TAU))


def relerr(g: np.ndarray, o: np.ndarray) -> float:
    """max |g - o| / max |o| (field-wise relative error; 0 for an all-zero reference)."""
    scale = np.abs(o).max()
    d = np.abs(g - o).max()
    if scale == 0:
        return float(d)
    return float(d / scale)


def relerr_rows(g: np.ndarray, o: np.ndarray) -> float:
    """max over components (rows of the SoA field) of max |g - o| / max |o| over that
    component: each component is held to its own scale (a small velocity component or an
    off-diagonal of F is not measured against the largest one)."""
    g2, o2 = g.reshape(-1, g.shape[-1]), o.reshape(-1, o.shape[-1])
    floor = 1e-300 + 1e-12 * np.abs(o2).max()
    return float(max(np.abs(g2[r] - o2[r]).max() / max(np.abs(o2[r]).max(), floor) for r in range(o2.shape[0])))


def push_oracle_state(g, o):
    """Give the CUDA state g the oracle o's dynamic state (x, v_p, v, e, F) and next dt, so
    that both take their next step from the same state. The oracle's trajectory stays its own
    (nothing flows from the CUDA path into the oracle). Returns the state."""
    st = o.state()
    g.set_fields({L.FIELD_X: st["x"], L.FIELD_VP: st["vp"], L.FIELD_V: st["v"], L.FIELD_E: st["e"],
                  L.FIELD_F: st["F"], L.FIELD_DT: np.array([o.dt])})
    return st


def step_errors(g, o, before: dict) -> dict:
    """After one step of both sides from the same state `before`: the field-wise relative
    errors, the per-component relative errors, and the nodal solver's velocity v*_p (the
    step's displacement divided by dt, compared on its own scale: x itself is ~1 while a step
    moves it by ~1e-5, so x^{n+1} alone hides the displacement below its last bits)."""
    out = {}
    for name, fo, fg in FIELDS:
        a, b = g.get(fg), o.get(fo)
        out[name] = relerr(a, b)
        out[name + "_rows"] = relerr_rows(a, b)
    out["vstar_rows"] = relerr_rows(g.get(L.FIELD_VSTAR), o.get(O.F_VSTAR))
    return out


class Pair:
    def __init__(self, problem, **params):
        """params: step parameters of both sides; graph (the library's step form) goes to the
        CUDA side only"""
        self.pb = problem
        self.g = L.simulation(problem, **params)
        self.o = O.Oracle(problem, **{k: v for k, v in params.items() if k != "graph"})

    def errors(self) -> dict:
        out = {}
        for name, fo, fg in FIELDS:
            out[name] = relerr(self.g.get(fg), self.o.get(fo))
        out["dt"] = abs(self.g.get(L.FIELD_DT)[0] - self.o.dt) / self.o.dt
        return out

    def masks(self):
        return self.g.get(L.FIELD_ORDER).astype(int), self.o.get(O.F_ORDER).astype(int)

    def step(self):
        ig = self.g.step()
        self.o.step()
        return ig, self.o.info

    def run_compare(self, nsteps: int, tol_step: float = 1e-11, tol_run: float = 1e-8, check_every: int = 1):
        """Advance both sides; order masks must match at every step, the state must agree to
        tol_step after the first step and to tol_run over the run. Returns stats."""
        worst = 0.0
        troubled = 0
        for s in range(nsteps):
            ig, io = self.step()
            mg, mo = self.masks()
            if not np.array_equal(mg, mo):
                bad = np.where(mg != mo)[0]
                raise AssertionError(f"step {s}: MOOD masks differ in {bad.size} cells, e.g. {bad[:10]}")
            assert ig.n_troubled == io.n_troubled and ig.mood_iters == io.mood_iters, (s, ig.n_troubled, io.n_troubled)
            troubled += io.n_troubled
            if s % check_every == 0 or s == nsteps - 1:
                err = self.errors()
                e = max(err.values())
                worst = max(worst, e)
                lim = tol_step if s == 0 else tol_run
                assert e <= lim, (s, err)
        return {"worst": worst, "troubled": troubled}
