"""GPU path vs the CPU oracle on meshes whose S-elements have different numbers of
boundary nodes (quadtree meshes with hanging vertices, n_b from 8 to 40), through the
C ABI.  The library pads every element to the mesh's largest n_b; these tests check
that the padding changes nothing: traces within 1e-10 and gradients within 1e-8
(relative L2) of the oracle, which handles each n_b group on its own."""

import numpy as np
import pytest

from oracle import uneven
from sbfwi_inputs import batching_workload, boundary_nodes, min_spacing, nearest_node, quadtree_mesh, ricker

pytestmark = pytest.mark.gpu

TRACE_TOL = 1e-10
GRAD_TOL = 1e-8


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _case(p, n_r, shots=3, K=40, seed=0, ring=False):
    """A small quadtree: the lower-left quarter refined once (n_b = 4p..5p), or with
    ``ring`` every cell but the centre one of a 3x3 grid (the centre has n_b = 8p)."""
    if ring:
        m = quadtree_mesh(3, 1, lambda x0, y0, x1, y1, lvl: not (1 / 3 <= x0 < 0.5 and 1 / 3 <= y0 < 0.5), p)
    else:
        m = quadtree_mesh(4, 1, lambda x0, y0, x1, y1, lvl: x0 < 0.5 and y0 < 0.5, p)
    rng = np.random.default_rng(seed)
    rho = 0.7 + 0.6 * rng.random((19, 21))
    s = min_spacing(m)
    dt, f0 = 0.5 * s, 1.0 / (10 * s)
    top = boundary_nodes(m, "top")
    src = np.array([nearest_node(m, top, ((k + 0.5) / shots, 1.0)) for k in range(shots)])
    wav = np.stack([ricker(f0, dt, K, t0=(1.2 + 0.2 * k) / f0) for k in range(shots)])
    rec = np.unique(np.concatenate([boundary_nodes(m, "bottom")[::3], boundary_nodes(m, "left")[1::4]]))
    return m, n_r, rho, dt, src, wav, rec


def _compare(lib, m, n_r, rho, dt, src, wav, rec, rho_kind="grid"):
    om = uneven.build_model(m, n_r, 1.0, rho, dt)
    M = lib.Mesh.from_inputs(m, n_r)
    assert M.n_nodal == om.n_int + om.n_nodes
    if rho_kind == "grid":
        md = lib.Model(M, 1.0, rho, dt, lx=1.0, ly=1.0)
    else:
        md = lib.Model(M, 1.0, om.rho_nodal, dt, rho_kind=lib.RHO_NODAL)
    tr, st = lib.forward(md, src, wav, rec)
    to, store, _ = uneven.forward(om, src, wav, rec)
    assert np.abs(to).max() > 0
    assert rel(tr, to) <= TRACE_TOL
    obs = 0.9 * to + 0.05 * np.roll(to, 3, axis=-1)
    _, res = lib.misfit(tr, obs, dt)
    reso = obs - to
    g = lib.adjoint_gradient(md, st, res)
    go = uneven.adjoint_gradient(om, store, reso, rec)
    if rho_kind == "grid":
        go = uneven.gradient_to_grid(om, go, rho.shape[1], rho.shape[0])
    assert g.shape == go.shape
    assert rel(g, go) <= GRAD_TOL
    return tr, g


@pytest.mark.parametrize("element", ["tensor", "fp64"])
@pytest.mark.parametrize("p", [2, 5])
def test_quadtree_both_element_kernels(lib, p, element, monkeypatch):
    """p = 2: n_b 8 and 10 padded to 10 (one-tile tensor-core kernel); p = 5: n_b 20 and
    25 padded to 25 (two-tile tensor-core kernel); and the FP64 kernel on both."""
    if element == "fp64":
        monkeypatch.setenv("SBFWI_ELEMENT", "fp64")
    m, n_r, rho, dt, src, wav, rec = _case(p, 6 if p < 5 else 5, K=40 if p < 5 else 25)
    assert set(m.n_b) == {4 * p, 5 * p}
    _compare(lib, m, n_r, rho, dt, src, wav, rec)


@pytest.mark.parametrize("rho_kind", ["grid", "nodal"])
def test_quadtree_order3_grid_and_nodal_density(lib, rho_kind):
    """n_b 12 and 15 (padded to 15); nodal density in the caller's unpadded layout, and
    the nodal gradient returned in it."""
    m, n_r, rho, dt, src, wav, rec = _case(3, 5, shots=2, seed=1)
    _compare(lib, m, n_r, rho, dt, src, wav, rec, rho_kind)


def test_quadtree_order5_up_to_forty_boundary_nodes(lib):
    """A cell with four finer neighbours: n_b = 40 next to n_b = 20 and 25 (padded to 40:
    the FP64 element kernel)."""
    m, n_r, rho, dt, src, wav, rec = _case(5, 5, shots=2, K=25, seed=2, ring=True)
    assert m.n_b.max() == 40 and m.n_b.min() == 20
    _compare(lib, m, n_r, rho, dt, src, wav, rec)


@pytest.mark.parametrize("index", [0, 1, 2])
def test_batching_meshes_full_size_few_steps(lib, index):
    """Each mesh of the batching recipe at full size (about 700 elements, p = 2, 3, 5,
    N_r = 16, 32, 48, padded n_b 12, 18, 30: one-tile tensor-core, FP64 and two-tile
    tensor-core element kernels)
    with 8 shots in one pass, the launch configuration of the benchmark, for 4 steps:
    traces and the grid gradient against the oracle."""
    w = batching_workload(index, K=4)
    src = w.src_nodes[:8]
    wav = np.stack([ricker(w.f0, w.dt, 4, t0=(2 + k) * w.dt) for k in range(src.size)])  # active from step 1
    om = uneven.build_model(w.mesh, w.n_r, w.c, w.rho_true, w.dt)
    M = lib.Mesh.from_inputs(w.mesh, w.n_r)
    md = lib.Model(M, w.c, w.rho_true, w.dt)
    tr, st = lib.forward(md, src, wav, w.rec_nodes)
    to, store, _ = uneven.forward(om, src, wav, w.rec_nodes)
    assert rel(tr, to) <= TRACE_TOL
    obs = 0.5 * to
    _, res = lib.misfit(tr, obs, w.dt)
    g = lib.adjoint_gradient(md, st, res)
    go = uneven.gradient_to_grid(om, uneven.adjoint_gradient(om, store, obs - to, w.rec_nodes), w.gx, w.gy)
    assert rel(g, go) <= GRAD_TOL


@pytest.mark.parametrize("intervals", [5, 7])
def test_voronoi_paper_plate(lib, intervals):
    """The paper's plate recipe on its own mesh type: about 100 centroidal Voronoi
    polygons (4 to 7 sides, n_b 8..14), 5 and 7 radial intervals, two sine-burst
    sources, receivers every 1 mm, all 200 steps: traces and gradient."""
    from sbfwi_inputs import paper_workload
    w = paper_workload(n_elem=100, intervals=intervals, mesh_kind="voronoi")
    assert len(set(w.mesh.n_b)) > 1
    L = w.mesh.lx
    om = uneven.build_model(w.mesh, w.n_r, w.c, w.rho_true, w.dt, lx=L, ly=L)
    to, store, _ = uneven.forward(om, w.src_nodes, w.wavelets, w.rec_nodes)
    M = lib.Mesh.from_inputs(w.mesh, w.n_r)
    md = lib.Model(M, w.c, w.rho_true, w.dt, lx=L, ly=L)
    tr, st = lib.forward(md, w.src_nodes, w.wavelets, w.rec_nodes)
    assert np.abs(to).max() > 0
    assert rel(tr, to) <= TRACE_TOL
    g = lib.adjoint_gradient(md, st, -tr)
    go = uneven.gradient_to_grid(om, uneven.adjoint_gradient(om, store, -to, w.rec_nodes), w.gx, w.gy, L, L)
    assert rel(g, go) <= GRAD_TOL


def test_voronoi_paper_plate_full_size_few_steps(lib):
    """1000 Voronoi polygons (the paper's smallest mesh), 5 intervals, 6 steps."""
    from sbfwi_inputs import paper_workload
    w = paper_workload(n_elem=1000, intervals=5, K=6, mesh_kind="voronoi")
    L = w.mesh.lx
    om = uneven.build_model(w.mesh, w.n_r, w.c, w.rho_true, w.dt, lx=L, ly=L)
    to, store, _ = uneven.forward(om, w.src_nodes, w.wavelets, w.rec_nodes)
    M = lib.Mesh.from_inputs(w.mesh, w.n_r)
    md = lib.Model(M, w.c, w.rho_true, w.dt, lx=L, ly=L)
    tr, st = lib.forward(md, w.src_nodes, w.wavelets, w.rec_nodes)
    assert np.abs(to).max() > 0
    assert rel(tr, to) <= TRACE_TOL
    g = lib.adjoint_gradient(md, st, -tr)
    go = uneven.gradient_to_grid(om, uneven.adjoint_gradient(om, store, -to, w.rec_nodes), w.gx, w.gy, L, L)
    assert rel(g, go) <= GRAD_TOL
