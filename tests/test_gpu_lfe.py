"""The paper's comparison method (low-frequency expansion, Section 3.2) on the GPU against
the oracle's, through the C ABI: receiver traces, misfit and the boundary-node gradient,
on a structured mesh and on a quadtree with hanging vertices."""

import numpy as np
import pytest

from oracle import fwi, lfe
from sbfwi_inputs import boundary_nodes, min_spacing, nearest_node, quadtree_mesh, ricker, structured_mesh

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.mark.parametrize("kind", ["structured", "quadtree"])
def test_lfe_traces_and_gradient_match_the_oracle(lib, kind):
    if kind == "structured":
        m = structured_mesh(4, 4, 2)
    else:
        m = quadtree_mesh(4, 1, lambda x0, y0, x1, y1, lvl: x0 < 0.5 and y0 < 0.5, 3)
    gx = gy = 16
    rho = 0.8 + 0.4 * np.random.default_rng(3).random((gy, gx))
    s = min_spacing(m)
    dt, f0, K = 0.5 * s, 1.0 / (10 * s), 80
    top = boundary_nodes(m, "top")
    src = np.array([nearest_node(m, top, (0.3, 1.0)), nearest_node(m, top, (0.7, 1.0))])
    wav = np.stack([ricker(f0, dt, K, t0=1.2 / f0), 0.5 * ricker(f0, dt, K, t0=1.4 / f0)])
    rec = np.unique(np.concatenate([boundary_nodes(m, "bottom")[::2], boundary_nodes(m, "left")[1::3]]))
    rho_b = fwi.grid_to_points(rho, m.node_xy, 1.0, 1.0)
    obs = np.zeros((2, rec.size, K))
    to, Eo, go = lfe.forward_and_gradient(m, 1.0, rho_b, dt, src, wav, rec, obs)
    M = lib.Mesh.from_inputs(m, 5)
    md = lib.Model(M, 1.0, rho, dt, lfe=True)
    tr, st = lib.forward(md, src, wav, rec)
    assert np.abs(to).max() > 0
    assert rel(tr, to) <= 1e-10
    E, res = lib.misfit(tr, obs, dt)
    assert E == pytest.approx(Eo, rel=1e-10)
    g = lib.adjoint_gradient(md, st, res)
    assert rel(g, fwi.points_to_grid(go, m.node_xy, gx, gy, 1.0, 1.0)) <= 1e-8
    # the radial finite differences give different traces (the expansion is an approximation)
    tr_fd, _ = lib.forward(lib.Model(M, 1.0, rho, dt), src, wav, rec, keep=False)
    assert rel(tr_fd, tr) > 1e-3


def test_lfe_refuses_the_full_kernel(lib):
    m = structured_mesh(2, 2, 2)
    M = lib.Mesh.from_inputs(m, 5)
    md = lib.Model(M, 1.0, np.ones((8, 8)), 0.05, lfe=True)
    lib.set_kernel_terms(md, lib.TERMS_FULL)
    w = ricker(0.8, 0.05, 10)[None]
    with pytest.raises(lib.SbfwiError) as ei:
        lib.forward(md, [int(boundary_nodes(m, "top")[1])], w, boundary_nodes(m, "bottom"))
    assert ei.value.code == lib.EUNSUPPORTED
