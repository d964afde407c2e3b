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
