"""The exact derivative of the discrete misfit (Mode X, ``oracle.modex``) against finite
differences, and the paper's velocity kernel (Mode K, ``oracle.fwi.adjoint_gradient``)
against the exact derivative of the inertia density."""

import numpy as np
import pytest

from oracle import fwi, modex, sbfem
from sbfwi_inputs import structured_mesh, boundary_nodes, ricker, tiny_workload
from test_oracle_dynamics import _lumped_nodal_areas


def _small_problem(seed=3):
    mesh = structured_mesh(2, 2, 2)
    n_r = 5
    rng = np.random.default_rng(seed)
    elements = sbfem.elements_from_mesh(mesh)
    xi = sbfem.radial_grid(n_r - 1, 1e-3, np.float64)
    pts, _ = fwi.nodal_points(mesh, elements, xi)
    rho = 1.0 + 0.3 * rng.random(pts.shape[0])
    src = np.array([boundary_nodes(mesh, "top")[1]])
    recs = np.unique(np.concatenate([boundary_nodes(mesh, s) for s in ("bottom", "left", "right")]))[:4]
    dt, K = 0.05, 40
    wav = np.stack([ricker(1.5, dt, K)])
    obs = 0.01 * rng.standard_normal((1, len(recs), K))
    return mesh, n_r, rho, src, recs, wav, obs, dt


def test_exact_gradient_matches_central_differences():
    """<g, d> against (E(rho + h d) - E(rho - h d)) / 2h of the same discrete misfit."""
    mesh, n_r, rho, src, recs, wav, obs, dt = _small_problem()
    E0, g = modex.misfit_and_gradient(mesh, n_r, 1.0, rho, dt, src, wav, recs, obs)
    assert E0 == pytest.approx(modex.misfit_only(mesh, n_r, 1.0, rho, dt, src, wav, recs, obs), rel=1e-13)
    rng = np.random.default_rng(11)
    for _ in range(4):
        d = rng.standard_normal(rho.size)
        h = 1e-6
        fd = (modex.misfit_only(mesh, n_r, 1.0, rho + h * d, dt, src, wav, recs, obs)
              - modex.misfit_only(mesh, n_r, 1.0, rho - h * d, dt, src, wav, recs, obs)) / (2 * h)
        assert abs(g @ d - fd) <= 1e-6 * abs(fd)


def test_exact_gradient_is_linear_in_the_residual():
    """With observed = traces + r, E and g scale as |r|^2 and r (the forward does not
    depend on the residual)."""
    mesh, n_r, rho, src, recs, wav, obs, dt = _small_problem(5)
    fs = modex.bruteforce.FullSystem(mesh, n_r, 1.0, rho, dt)
    tr, _ = fs.forward(src, wav, recs)
    r = obs
    E1, g1 = modex.misfit_and_gradient(mesh, n_r, 1.0, rho, dt, src, wav, recs, tr + r)
    E2, g2 = modex.misfit_and_gradient(mesh, n_r, 1.0, rho, dt, src, wav, recs, tr + 2 * r)
    assert E2 == pytest.approx(4 * E1, rel=1e-8)
    np.testing.assert_allclose(g2, 2 * g1, rtol=0, atol=1e-8 * np.abs(g1).max())


@pytest.mark.slow
def test_velocity_kernel_matches_the_exact_inertia_gradient():
    """Mode K weighted by the area each nodal point stands for against the exact
    derivative with respect to the density of the inertia term (tiny workload, 200
    steps): cosine similarity >= 0.99 (measured 0.9987) and norms within 10 %
    (measured 3 %).  The full exact derivative also differentiates the stiffness
    terms, which the paper's kernel drops, so it is only loosely aligned (measured
    cosine 0.59) and is not asserted."""
    w = tiny_workload(K=200)
    m0 = fwi.build_model(w.mesh, w.n_r, w.c, w.rho_start, w.dt)
    mt = fwi.build_model(w.mesh, w.n_r, w.c, w.rho_true, w.dt)
    obs, _, _ = fwi.forward(mt, w.src_nodes, w.wavelets, w.rec_nodes, keep=False)
    _, gx_mass = modex.misfit_and_gradient(w.mesh, w.n_r, w.c, m0.rho_nodal, w.dt, w.src_nodes, w.wavelets,
                                           w.rec_nodes, obs, part="mass")
    mn = fwi.build_model(w.mesh, w.n_r, w.c, m0.rho_nodal, w.dt, rho_kind="nodal")
    tr, store, _ = fwi.forward(mn, w.src_nodes, w.wavelets, w.rec_nodes)
    _, res = fwi.misfit(tr, obs, w.dt)
    gk = _lumped_nodal_areas(mn, w.mesh) * fwi.adjoint_gradient(mn, store, res, w.rec_nodes)
    cos = gk @ gx_mass / np.linalg.norm(gk) / np.linalg.norm(gx_mass)
    assert cos >= 0.99
    assert abs(np.linalg.norm(gk) / np.linalg.norm(gx_mass) - 1) <= 0.10
