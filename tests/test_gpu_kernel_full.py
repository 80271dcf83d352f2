"""The full Frechet kernel (velocity term + the gradient term the paper drops) on the GPU
against the oracle's, through the C ABI: grid and nodal parameters, both element
kernels, and the errors of the states it needs."""

import numpy as np
import pytest

from oracle import fwi
from sbfwi_inputs import tiny_workload, structured_mesh, boundary_nodes, ricker

pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-8


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def _oracle_full(w, rho, obs, rho_kind="grid"):
    om = fwi.build_model(w.mesh, w.n_r, w.c, rho, w.dt, rho_kind=rho_kind)
    to, store, _, su = fwi.forward(om, w.src_nodes, w.wavelets, w.rec_nodes, keep_u=True)
    g = fwi.adjoint_gradient(om, store, obs - to, w.rec_nodes, store_u=su)
    gv = fwi.adjoint_gradient(om, store, obs - to, w.rec_nodes)
    return om, g, gv


@pytest.mark.parametrize("element", ["tensor", "fp64"])
@pytest.mark.parametrize("rho_kind", ["grid", "nodal"])
def test_full_kernel_matches_the_oracle(lib, element, rho_kind):
    w = tiny_workload(K=120)
    wf = tiny_workload(refine=2, K=120)
    mt = fwi.build_model(wf.mesh, wf.n_r, 1.0, wf.rho_true, w.dt)
    obs, _, _ = fwi.forward(mt, wf.src_nodes, wf.wavelets, wf.rec_nodes, keep=False)
    rho = w.rho_start * (1.0 + 0.2 * np.sin(np.linspace(0, 3, w.rho_start.size)).reshape(w.rho_start.shape))
    om, go, gvo = _oracle_full(w, rho, obs)
    if rho_kind == "nodal":
        rho = np.asarray(om.rho_nodal, dtype=np.float64)
        om, go, gvo = _oracle_full(w, rho, obs, "nodal")
    M = lib.Mesh.from_inputs(w.mesh, w.n_r)
    md = lib.Model(M, w.c, rho, w.dt, rho_kind=lib.RHO_GRID if rho_kind == "grid" else lib.RHO_NODAL)
    lib.set_schedule(md, lib.ELEMENT_TENSOR if element == "tensor" else lib.ELEMENT_FP64)
    lib.set_kernel_terms(md, lib.TERMS_FULL)
    tr, st = lib.forward(md, w.src_nodes, w.wavelets, w.rec_nodes)
    _, res = lib.misfit(tr, obs, w.dt)
    g = lib.adjoint_gradient(md, st, res)
    if rho_kind == "grid":
        go = fwi.gradient_to_grid(om, go, w.gx, w.gy)
        gvo = fwi.gradient_to_grid(om, gvo, w.gx, w.gy)
    assert rel(g, go) <= GRAD_TOL
    assert rel(go, gvo) > 1e-3              # the gradient term is not negligible here


def test_full_kernel_state_errors(lib):
    w = tiny_workload(K=40)
    M = lib.Mesh.from_inputs(w.mesh, w.n_r)
    md = lib.Model(M, w.c, w.rho_start, w.dt)
    tr, st = lib.forward(md, w.src_nodes, w.wavelets, w.rec_nodes)          # velocities only
    lib.set_kernel_terms(md, lib.TERMS_FULL)
    with pytest.raises(lib.SbfwiError) as ei:
        lib.adjoint_gradient(md, st, -tr)
    assert ei.value.code == lib.ESTATE
    with pytest.raises(lib.SbfwiError) as ei:
        lib.set_kernel_terms(md, 5)
    assert ei.value.code == lib.EINVAL
    lib.set_kernel_terms(md, lib.TERMS_VELOCITY)
    g = lib.adjoint_gradient(md, st, -tr)                                     # back to the paper's kernel
    assert np.isfinite(g).all()


@pytest.mark.parametrize("p", [3, 5])
def test_full_kernel_on_uneven_meshes(lib, p):
    """Quadtree meshes with hanging vertices (p = 3: n_b 12 and 15; p = 5 with a cell of
    four finer neighbours: n_b 20..40, FP64 kernel): the padded layout's gradient operator
    against the grouped oracle's."""
    from oracle import uneven
    from sbfwi_inputs import min_spacing, nearest_node, quadtree_mesh
    if p == 3:
        m = quadtree_mesh(4, 1, lambda x0, y0, x1, y1, lvl: x0 < 0.5 and y0 < 0.5, 3)
    else:
        m = quadtree_mesh(3, 1, lambda x0, y0, x1, y1, lvl: not (1 / 3 <= x0 < 0.5 and 1 / 3 <= y0 < 0.5), 5)
    rho = 0.8 + 0.4 * np.random.default_rng(p).random((15, 15))
    s = min_spacing(m)
    dt, f0, K = 0.5 * s, 1.0 / (10 * s), 30
    src = np.array([nearest_node(m, boundary_nodes(m, "top"), (0.4, 1.0))])
    wav = ricker(f0, dt, K, t0=1.2 / f0)[None]
    rec = boundary_nodes(m, "bottom")[::2]
    om = uneven.build_model(m, 5, 1.0, rho, dt)
    to, store, _, su = uneven.forward(om, src, wav, rec, keep_u=True)
    go = uneven.gradient_to_grid(om, uneven.adjoint_gradient(om, store, -to, rec, store_u=su), 15, 15)
    M = lib.Mesh.from_inputs(m, 5)
    md = lib.Model(M, 1.0, rho, dt)
    lib.set_kernel_terms(md, lib.TERMS_FULL)
    tr, st = lib.forward(md, src, wav, rec)
    g = lib.adjoint_gradient(md, st, -tr)
    assert rel(g, go) <= GRAD_TOL


@pytest.mark.parametrize("element", ["tensor", "fp64"])
def test_full_kernel_with_checkpoints_is_the_stored_field_kernel(lib, element):
    """Checkpointed forward passes: the adjoint recomputes velocities and displacements window
    by window; the full kernel's gradient equals the stored-field one bit for bit."""
    w = tiny_workload(K=60)
    M = lib.Mesh.from_inputs(w.mesh, w.n_r)
    md = lib.Model(M, w.c, w.rho_true, w.dt)
    lib.set_schedule(md, lib.ELEMENT_TENSOR if element == "tensor" else lib.ELEMENT_FP64)
    lib.set_kernel_terms(md, lib.TERMS_FULL)
    tr, st = lib.forward(md, w.src_nodes, w.wavelets, w.rec_nodes)
    g0 = lib.adjoint_gradient(md, st, -tr)
    for c in (1, 7, 60, lib.CKPT_AUTO):
        tr_c, st_c = lib.forward(md, w.src_nodes, w.wavelets, w.rec_nodes, ckpt_every=c)
        assert np.array_equal(tr_c, tr)
        assert np.array_equal(lib.adjoint_gradient(md, st_c, -tr), g0), c
