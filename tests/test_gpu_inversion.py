"""The inversion loop around the library (harness): sharded misfit + gradient on one
rank equals the direct calls, and projected L-BFGS lowers the misfit on the tiny
workload."""

import numpy as np
import pytest

from sbfwi_inputs import tiny_workload

pytestmark = pytest.mark.gpu


def test_single_rank_misfit_and_gradient_match_direct_calls(lib):
    from paper_2501_06748_gb300 import shots
    w = tiny_workload(K=120)
    M = lib.Mesh.from_inputs(w.mesh, w.n_r)
    mt = lib.Model(M, w.c, w.rho_true, w.dt)
    obs, _ = lib.forward(mt, w.src_nodes, w.wavelets, w.rec_nodes, keep=False)
    md = lib.Model(M, w.c, w.rho_start, w.dt)
    E, g = shots.misfit_and_gradient(md, w.src_nodes, w.wavelets, w.rec_nodes, obs, ckpt_every=lib.CKPT_AUTO)
    tr, st = lib.forward(md, w.src_nodes, w.wavelets, w.rec_nodes)
    E2, res = lib.misfit(tr, obs, w.dt)
    g2 = lib.adjoint_gradient(md, st, res)
    assert E == pytest.approx(E2, rel=1e-14)
    assert np.array_equal(g, g2)


def test_projected_lbfgs_lowers_the_misfit(lib):
    torch = pytest.importorskip("torch")
    from paper_2501_06748_gb300 import inversion
    w = tiny_workload(K=200)
    M = lib.Mesh.from_inputs(w.mesh, w.n_r)
    mt = lib.Model(M, w.c, w.rho_true, w.dt)
    obs, _ = lib.forward(mt, w.src_nodes, torch.tensor(w.wavelets, device="cuda"), w.rec_nodes, keep=False)
    fg = inversion.objective(M, w.c, w.dt, w.src_nodes, torch.tensor(w.wavelets, device="cuda"), w.rec_nodes, obs)
    x0 = torch.tensor(w.rho_start, device="cuda")
    x, hist = inversion.lbfgs(fg, x0, 1e-6, 2.0, iters=3)
    assert len(hist) == 4
    assert all(b <= a for a, b in zip(hist, hist[1:]))
    assert hist[-1] < 0.9 * hist[0]
    assert float(x.min()) >= 1e-6 and float(x.max()) <= 2.0
