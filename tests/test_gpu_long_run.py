"""GPU path vs the oracle over the full 2000-step time axis of the size recipe.

Per-step rounding of the two implementations accumulates in the free-surface
problem's rigid-body mode roughly linearly in time, so agreement over a few steps
does not imply agreement over the recipe's 2000 steps.  This runs an 8 x 8 sub-mesh
of the size recipe (p = 4, N_r = 32, 8 shots in one pass, the default element
kernel and solve schedule, as the benchmark times them) for all 2000 steps:
set-up, forward, misfit, adjoint and gradient against ``oracle.fwi``.
"""

import numpy as np
import pytest
import torch

from oracle import fwi
from sbfwi_inputs import size_workload

pytestmark = pytest.mark.gpu

TRACE_TOL = 1e-10
GRAD_TOL = 1e-8


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def test_size_recipe_submesh_all_2000_steps(lib):
    w = size_workload(nx=8, K=2000, n_shots=8)
    dev = torch.device("cuda", 0)
    M = lib.Mesh.from_inputs(w.mesh, w.n_r)
    # the flawed model, zero observed data (the adjoint is driven by the traces themselves)
    md = lib.Model(M, w.c, torch.tensor(w.rho_true, device=dev), w.dt)
    tr, st = lib.forward(md, w.src_nodes, torch.tensor(w.wavelets, device=dev), w.rec_nodes)
    E, res = lib.misfit(tr, torch.zeros_like(tr), w.dt)
    g = lib.adjoint_gradient(md, st, res).cpu().numpy()
    tr = tr.cpu().numpy()

    om = fwi.build_model(w.mesh, w.n_r, w.c, w.rho_true, w.dt)
    to, store, _ = fwi.forward(om, w.src_nodes, w.wavelets, w.rec_nodes)
    Eo, reso = fwi.misfit(to, np.zeros_like(to), w.dt)
    go = fwi.gradient_to_grid(om, fwi.adjoint_gradient(om, store, reso, w.rec_nodes), w.gx, w.gy)

    assert np.abs(to).max() > 1e-3
    assert rel(tr, to) <= TRACE_TOL
    assert abs(E - Eo) <= 1e-10 * abs(Eo)
    assert rel(g, go) <= GRAD_TOL
