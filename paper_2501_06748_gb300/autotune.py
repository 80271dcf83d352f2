"""Schedule autotuner (a harness around the library; not part of the paper's method).

For one model and one shot batch, ``tune`` times every element kernel (tensor-core,
FP64, and on meshes with uneven elements the per-class mix of the two) with every global-solve schedule (dataflow, barrier, per-level launches) on a
few steps of the caller's own problem -- a forward pass that stores its velocities and
the adjoint pass with the gradient, the two time loops of a misfit-and-gradient
evaluation, whose element launches differ (store vs gradient) -- keeps the fastest on the model
(``sbfwi.set_schedule``) and reports all candidates.  Candidates the shapes do not
allow (no tensor-core kernel for this n_b or shot count) are reported as such.  Every
candidate computes the same method; results agree within rounding.
"""

from __future__ import annotations

import time

import numpy as np

from . import sbfwi

ELEMENTS = {"tensor": sbfwi.ELEMENT_TENSOR, "fp64": sbfwi.ELEMENT_FP64, "mixed": sbfwi.ELEMENT_MIXED}
SOLVES = {"dataflow": sbfwi.SOLVE_DATAFLOW, "barrier": sbfwi.SOLVE_BARRIER, "levels": sbfwi.SOLVE_LEVELS}


def tune(model, src_nodes, wavelets, rec_nodes, steps: int = 16, repeats: int = 3,
         elements=("tensor", "fp64", "mixed"), solves=("dataflow", "barrier", "levels"),
         shots_per_pass: int = 8) -> dict:
    """Time the candidates on ``steps`` steps of a misfit-and-gradient evaluation of these
    shots (passes of ``shots_per_pass``: forward with stored velocities + adjoint with the
    gradient) and set the fastest; returns {"element", "solve", "s_per_step" (the whole
    evaluation per step), "candidates": [...]}."""
    wav = wavelets[:, :max(1, min(steps, wavelets.shape[1]))]
    K = wav.shape[1]
    out = []
    for en in elements:
        for sn in solves:
            sbfwi.set_schedule(model, ELEMENTS[en], SOLVES[sn])

            def evaluation():                          # the passes of a misfit-and-gradient evaluation
                for lo in range(0, len(src_nodes), max(1, shots_per_pass)):
                    hi = min(len(src_nodes), lo + max(1, shots_per_pass))
                    tr, st = sbfwi.forward(model, src_nodes[lo:hi], wav[lo:hi], rec_nodes)
                    sbfwi.adjoint_gradient(model, st, tr)   # synchronous: the gradient comes back
                    del st

            try:
                evaluation()                               # warm-up, first-use preparation
            except sbfwi.SbfwiError as err:
                if err.code != sbfwi.EUNSUPPORTED:
                    raise
                out.append({"element": en, "solve": sn, "s_per_step": None, "note": str(err)})
                continue
            best = np.inf
            for _ in range(repeats):
                t0 = time.perf_counter()
                evaluation()
                best = min(best, time.perf_counter() - t0)
            out.append({"element": en, "solve": sn, "s_per_step": best / K})
    ok = [c for c in out if c["s_per_step"] is not None]
    if not ok:
        sbfwi.set_schedule(model)
        raise RuntimeError("no schedule ran")
    win = min(ok, key=lambda c: c["s_per_step"])
    sbfwi.set_schedule(model, ELEMENTS[win["element"]], SOLVES[win["solve"]])
    return {"element": win["element"], "solve": win["solve"], "s_per_step": win["s_per_step"], "candidates": out}


def apply(model, choice: dict) -> None:
    """Set a choice returned by ``tune`` on another model of the same mesh."""
    sbfwi.set_schedule(model, ELEMENTS[choice["element"]], SOLVES[choice["solve"]])
