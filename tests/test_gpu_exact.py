"""The exact discrete adjoint on the GPU (SBFWI_GRAD_EXACT), through the C ABI.

The reference is ``oracle.modex``: reverse-mode differentiation of the uncondensed time
loop (every element's rows -1..n+1 and the flux-balance rows, solved densely), whose
result is itself pinned by central finite differences on the CPU.  The GPU computes the
same derivative with the condensation's own operators transposed and run backwards in
time, the transposed multifrontal factors, and Gauss-point products of the derivative of
every block.  Tolerance: relative L2 1e-8 on the gradient, as for the paper's kernel.
Beyond the oracle's reach (uneven meshes, many steps), the GPU gradient is checked against
central finite differences of the GPU's own misfit.
"""

import numpy as np
import pytest
import torch

from oracle import fwi, modex, sbfem
from sbfwi_inputs import boundary_nodes, quadtree_mesh, ricker, structured_mesh, tiny_workload

pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-8


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _problem(mesh, n_r, K, B, dt, f0, seed=3):
    """Nodal densities 1 + 0.3 U(0,1) (the oracle's nodal layout, which is the library's for
    meshes with one n_b), B Ricker shots on the top edge, receivers on the other edges,
    observed data small noise (the residual is then about the traces themselves)."""
    rng = np.random.default_rng(seed)
    els = sbfem.elements_from_mesh(mesh)
    xi = sbfem.radial_grid(n_r - 1, 1e-3, np.float64)
    pts, _ = fwi.nodal_points(mesh, els, xi)
    rho = 1.0 + 0.3 * rng.random(pts.shape[0])
    top = boundary_nodes(mesh, "top")
    src = top[np.linspace(1, len(top) - 2, B).astype(int)]
    recs = np.unique(np.concatenate([boundary_nodes(mesh, s) for s in ("bottom", "left", "right")]))[::2]
    wav = np.stack([ricker(f0, dt, K) for _ in range(B)])
    obs = 0.01 * rng.standard_normal((B, len(recs), K))
    return rho, src, recs, wav, obs


def _gpu_exact(lib, M, rho, dt, src, wav, recs, obs, ckpt=0, rho_kind=None):
    md = lib.Model(M, 1.0, rho, dt, rho_kind=lib.RHO_NODAL if rho_kind is None else rho_kind)
    lib.set_gradient_mode(md, lib.GRAD_EXACT)
    tr, st = lib.forward(md, src, wav, recs, ckpt_every=ckpt)
    E, res = lib.misfit(tr, obs, dt)
    return E, lib.adjoint_gradient(md, st, res, mode=lib.GRAD_EXACT), tr


CASES = {
    "2x2_p2_nr5_1shot": (lambda: structured_mesh(2, 2, 2), 5, 40, 1, 0.05, 1.5),
    "4x4_p2_nr8_2shots": (lambda: structured_mesh(4, 4, 2), 8, 100, 2, 0.0625, 0.8),
    "3x3_p3_nr6_3shots": (lambda: structured_mesh(3, 3, 3), 6, 80, 3, 0.04, 1.0),
    "6x5_p3_nr6_5shots_ragged": (lambda: structured_mesh(6, 5, 3, lx=1.2, ly=1.0), 6, 60, 5, 0.03, 1.2),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_exact_gradient_matches_the_oracle(lib, case):
    mk, n_r, K, B, dt, f0 = CASES[case]
    mesh = mk()
    rho, src, recs, wav, obs = _problem(mesh, n_r, K, B, dt, f0)
    M = lib.Mesh.from_inputs(mesh, n_r)
    E, g, tr = _gpu_exact(lib, M, rho, dt, src, wav, recs, obs)
    Eo, go = modex.misfit_and_gradient(mesh, n_r, 1.0, rho, dt, src, wav, recs, obs)
    assert abs(E - Eo) <= 1e-10 * abs(Eo)
    assert g.shape == go.shape
    assert rel(g, go) <= GRAD_TOL


def test_exact_gradient_with_checkpoints_is_the_stored_field_gradient(lib):
    """Checkpointed forward (recomputed window by window in the adjoint) against the stored
    u, u'' field: bit for bit, for several intervals."""
    mesh = structured_mesh(4, 4, 2)
    rho, src, recs, wav, obs = _problem(mesh, 8, 90, 3, 0.0625, 0.8, seed=5)
    M = lib.Mesh.from_inputs(mesh, 8)
    E0, g0, _ = _gpu_exact(lib, M, rho, 0.0625, src, wav, recs, obs)
    for c in (1, 7, 30, 90, lib.CKPT_AUTO):
        E, g, _ = _gpu_exact(lib, M, rho, 0.0625, src, wav, recs, obs, ckpt=c)
        assert E == E0
        assert np.array_equal(g, g0), c


def test_exact_gradient_on_the_fine_grid_is_the_transpose_of_the_map(lib):
    """Grid densities: the gradient is P^T of the nodal one (P the bilinear map)."""
    w = tiny_workload(K=120)
    M = lib.Mesh.from_inputs(w.mesh, w.n_r)
    om = fwi.build_model(w.mesh, w.n_r, w.c, w.rho_start, w.dt)
    obs = 0.01 * np.random.default_rng(2).standard_normal((w.n_shots, len(w.rec_nodes), w.K))
    _, g_grid, _ = _gpu_exact(lib, M, w.rho_start, w.dt, w.src_nodes, w.wavelets, w.rec_nodes, obs,
                              rho_kind=lib.RHO_GRID)
    _, go = modex.misfit_and_gradient(w.mesh, w.n_r, w.c, om.rho_nodal, w.dt, w.src_nodes, w.wavelets, w.rec_nodes,
                                      obs)
    assert rel(g_grid, fwi.gradient_to_grid(om, go, w.gx, w.gy)) <= GRAD_TOL


def _fd_check(lib, M, rho, dt, src, wav, recs, obs, n_dir, h, seed, rho_kind=None):
    dev = torch.device("cuda", 0)
    kind = lib.RHO_NODAL if rho_kind is None else rho_kind
    _, g, _ = _gpu_exact(lib, M, torch.tensor(rho, device=dev), dt, src, torch.tensor(wav, device=dev), recs,
                         torch.tensor(obs, device=dev), rho_kind=kind)
    g = g.cpu().numpy()

    def E(r):
        md = lib.Model(M, 1.0, torch.tensor(r, device=dev), dt, rho_kind=kind)
        tr, _ = lib.forward(md, src, torch.tensor(wav, device=dev), recs, keep=False)
        return lib.misfit(tr, torch.tensor(obs, device=dev), dt, want_residual=False)[0]

    rng = np.random.default_rng(seed)
    errs = []
    for _ in range(n_dir):
        d = rng.standard_normal(rho.shape)
        fd = (E(rho + h * d) - E(rho - h * d)) / (2 * h)
        errs.append(abs(float(np.sum(g * d)) - fd) / abs(fd))
    return max(errs)


def test_exact_gradient_matches_central_differences_on_an_uneven_mesh(lib):
    """Quadtree mesh with hanging vertices (n_b 8..12, padded elements): beyond the oracle's
    uniform-n_b reach, so <g, d> is checked against central differences of the GPU misfit
    along 6 random directions of the nodal densities (caller's unpadded layout)."""
    mesh = quadtree_mesh(4, 1, lambda x0, y0, x1, y1, lvl: x0 < 0.5 and y0 < 0.5, 2)
    n_r = 6
    M = lib.Mesh.from_inputs(mesh, n_r)
    rng = np.random.default_rng(1)
    rho = 1.0 + 0.3 * rng.random(M.n_nodal)
    top = boundary_nodes(mesh, "top")
    src = top[[1, len(top) - 2]]
    recs = np.unique(np.concatenate([boundary_nodes(mesh, s) for s in ("bottom", "left", "right")]))[::2]
    dt, K = 0.03, 120
    wav = np.stack([ricker(1.0, dt, K) for _ in src])
    obs = 0.01 * rng.standard_normal((len(src), len(recs), K))
    assert _fd_check(lib, M, rho, dt, src, wav, recs, obs, n_dir=6, h=1e-5, seed=4) <= 1e-6


def test_exact_gradient_through_autograd_matches_central_differences_in_16_directions(lib):
    """The exact mode of the autograd.Function: E.backward() fills rho.grad with the exact
    derivative of the discrete misfit, so <rho.grad, d> equals the central difference of the
    misfit along each of 16 random directions of the fine density grid (tiny workload,
    400 steps, two passes of one shot)."""
    from paper_2501_06748_gb300 import autograd
    w = tiny_workload()
    dev = torch.device("cuda", 0)
    M = lib.Mesh.from_inputs(w.mesh, w.n_r)
    wf = tiny_workload(refine=2)
    om = fwi.build_model(wf.mesh, wf.n_r, wf.c, wf.rho_true, w.dt)
    obs, _, _ = fwi.forward(om, wf.src_nodes, wf.wavelets, wf.rec_nodes, keep=False)
    src = np.concatenate([w.src_nodes, w.src_nodes])
    wav = torch.tensor(np.concatenate([w.wavelets, 0.5 * w.wavelets]), device=dev)
    obs = torch.tensor(np.concatenate([obs, 0.5 * obs]), device=dev)
    prob = autograd.Problem(M, w.c, w.dt, src, wav, w.rec_nodes, obs, shots_per_pass=1, gradient="exact")
    rho = torch.tensor(w.rho_start, device=dev, requires_grad=True)
    E = autograd.misfit(rho, prob)
    E.backward()
    g = rho.grad.cpu().numpy()
    rng = np.random.default_rng(16)
    h = 1e-5
    errs = []
    with torch.no_grad():
        for _ in range(16):
            d = torch.tensor(rng.standard_normal(w.rho_start.shape), device=dev)
            fd = (float(autograd.misfit(rho + h * d, prob)) - float(autograd.misfit(rho - h * d, prob))) / (2 * h)
            errs.append(abs(float(np.sum(g * d.cpu().numpy())) - fd) / abs(fd))
    assert max(errs) <= 1e-6


def test_exact_and_kernel_gradients_differ_and_state_errors(lib):
    """The paper's kernel is not the exact derivative (the radial FD operator is not
    symmetric); the forward state must be kept for the mode asked for."""
    mesh = structured_mesh(2, 2, 2)
    rho, src, recs, wav, obs = _problem(mesh, 5, 40, 1, 0.05, 1.5)
    M = lib.Mesh.from_inputs(mesh, 5)
    md = lib.Model(M, 1.0, rho, 0.05, rho_kind=lib.RHO_NODAL)
    tr, st = lib.forward(md, src, wav, recs)
    _, res = lib.misfit(tr, obs, 0.05)
    with pytest.raises(lib.SbfwiError) as ei:
        lib.adjoint_gradient(md, st, res, mode=lib.GRAD_EXACT)
    assert ei.value.code == lib.ESTATE
    gk = lib.adjoint_gradient(md, st, res)
    lib.set_gradient_mode(md, lib.GRAD_EXACT)
    tr2, st2 = lib.forward(md, src, wav, recs)
    assert rel(tr2, tr) <= 1e-12                      # the exact mode runs the FP64 element kernel
    with pytest.raises(lib.SbfwiError) as ei:
        lib.adjoint_gradient(md, st2, res)            # a stored exact field has no velocities
    assert ei.value.code == lib.ESTATE
    gx = lib.adjoint_gradient(md, st2, res, mode=lib.GRAD_EXACT)
    assert rel(gk, gx) > 1e-3
    with pytest.raises(lib.SbfwiError) as ei:
        lib.set_gradient_mode(md, 7)
    assert ei.value.code == lib.EINVAL
    ml = lib.Model(M, 1.0, rho, 0.05, rho_kind=lib.RHO_NODAL, lfe=True)
    with pytest.raises(lib.SbfwiError) as ei:
        lib.set_gradient_mode(ml, lib.GRAD_EXACT)
    assert ei.value.code == lib.EUNSUPPORTED
