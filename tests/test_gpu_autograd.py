"""The misfit as a torch.autograd.Function whose backward is the library's adjoint:
same value and gradient as the direct calls, the oracle's gradient within 1e-8, the
incoming gradient scales it, checkpointed and stored forward fields agree bitwise, and
L-BFGS driven through autograd lowers the misfit."""

import numpy as np
import pytest

from oracle import fwi
from sbfwi_inputs import tiny_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup(lib):
    torch = pytest.importorskip("torch")
    from paper_2501_06748_gb300 import autograd
    w = tiny_workload(K=120)
    M = lib.Mesh.from_inputs(w.mesh, w.n_r)
    obs, _ = lib.forward(lib.Model(M, w.c, w.rho_true, w.dt), w.src_nodes, w.wavelets, w.rec_nodes, keep=False)
    return torch, autograd, w, M, obs


def _problem(setup, device, **kw):
    torch, autograd, w, M, obs = setup
    wav, ob = w.wavelets, obs
    if device == "cuda":
        wav, ob = torch.tensor(wav, device="cuda"), torch.tensor(obs, device="cuda")
    return autograd.Problem(M, w.c, w.dt, w.src_nodes, wav, w.rec_nodes, ob, **kw)


@pytest.mark.parametrize("device", ["cuda", "cpu"])
def test_value_and_gradient_match_direct_calls_and_oracle(lib, setup, device):
    torch, autograd, w, M, obs = setup
    rho = torch.tensor(w.rho_start, device=device, requires_grad=True)
    E = autograd.misfit(rho, _problem(setup, device))
    E.backward()
    md = lib.Model(M, w.c, w.rho_start, w.dt)
    tr, st = lib.forward(md, w.src_nodes, w.wavelets, w.rec_nodes)
    E2, res = lib.misfit(tr, obs, w.dt)
    g2 = lib.adjoint_gradient(md, st, res)
    assert float(E.detach()) == pytest.approx(E2, rel=1e-14)
    g = rho.grad.cpu().numpy()
    assert np.array_equal(g, g2)
    om = fwi.build_model(w.mesh, w.n_r, w.c, w.rho_start, w.dt)
    to, store, _ = fwi.forward(om, w.src_nodes, w.wavelets, w.rec_nodes)
    go = fwi.gradient_to_grid(om, fwi.adjoint_gradient(om, store, obs - to, w.rec_nodes), w.gx, w.gy)
    assert np.linalg.norm(g - go) <= 1e-8 * np.linalg.norm(go)


def test_incoming_gradient_scales_and_checkpoints_agree(lib, setup):
    torch, autograd, w, M, obs = setup
    rho = torch.tensor(w.rho_start, device="cuda", requires_grad=True)
    (2.5 * autograd.misfit(rho, _problem(setup, "cuda"))).backward()
    r2 = torch.tensor(w.rho_start, device="cuda", requires_grad=True)
    autograd.misfit(r2, _problem(setup, "cuda", ckpt_every=lib.CKPT_AUTO)).backward()
    assert torch.equal(rho.grad, 2.5 * r2.grad)


def test_lbfgs_through_autograd_lowers_the_misfit(lib, setup):
    torch, autograd, w, M, obs = setup
    from paper_2501_06748_gb300 import inversion
    fg = autograd.objective(_problem(setup, "cuda"))
    x, hist = inversion.lbfgs(fg, torch.tensor(w.rho_start, device="cuda"), 1e-6, 2.0, iters=3)
    assert all(b <= a for a, b in zip(hist, hist[1:]))
    assert hist[-1] < 0.9 * hist[0]
