"""Pins of the oracle on meshes whose S-elements have different numbers of boundary
nodes (quadtree meshes with hanging vertices), CPU only."""

import numpy as np
import pytest

from oracle import fwi, sbfem, uneven
from sbfwi_inputs.mesh import min_spacing, quadtree_mesh, structured_mesh, voronoi_mesh
from sbfwi_inputs.wavelet import ricker


def _corner_refined(p, base=2, levels=1):
    return quadtree_mesh(base, levels, lambda x0, y0, x1, y1, lvl: x0 < 0.5 and y0 < 0.5, p)


def test_quadtree_mesh_is_conforming_and_balanced():
    m = quadtree_mesh(4, 2, lambda x0, y0, x1, y1, lvl: x0 < 0.3 < x1 + 0.1 and y0 < 0.6, 3)
    seen = {}
    for e in range(m.n_elem):
        for ln in m.line_nodes[m.elem_ptr[e]:m.elem_ptr[e + 1]]:
            key = (int(ln[0]), int(ln[-1]))
            assert key not in seen                    # no segment twice in the same direction
            seen[key] = tuple(ln)
    for (a, b), nodes in seen.items():
        on_edge = lambda q: np.isclose(m.node_xy[q], 0).any() or np.isclose(m.node_xy[q], 1).any()
        if (b, a) in seen:                            # interior segment: shared, reversed
            assert seen[(b, a)] == nodes[::-1]
        else:                                         # boundary segment lies on the domain edge
            mid = m.node_xy[list(nodes)].mean(axis=0)
            assert np.isclose(mid, 0).any() or np.isclose(mid, 1).any()
            assert on_edge(a) and on_edge(b)
    # 2:1 balance: cells sharing a side differ by at most one level
    lev = {tuple(c[1:]) + (c[0],): c[0] for c in m.cells}
    sizes = {int(c[0]) for c in m.cells}
    assert max(sizes) == 2 and min(sizes) == 0
    assert set(np.unique(np.diff(m.elem_ptr))) <= {4, 5, 6, 7, 8}
    assert np.all(m.n_b == 3 * np.diff(m.elem_ptr))
    # every node belongs to some line, and the cells tile the square
    assert np.unique(m.line_nodes).size == m.n_nodes
    area = sum((1.0 / (4 << int(c[0]))) ** 2 for c in m.cells)
    assert abs(area - 1.0) < 1e-12 and lev


@pytest.mark.parametrize("p", [1, 3])
def test_hanging_vertex_element_static_stiffness_annihilates_constants(p):
    """Partition of unity on a side split into two collinear lines: E1^T 1 = E2 1 = 0,
    so the static condensed stiffness of an element with hanging vertices maps the
    constant mode to zero."""
    m = _corner_refined(p)
    els = sbfem.elements_from_mesh(m)
    e = int(np.argmax([el.dofs.size for el in els]))
    el = els[e]
    assert el.dofs.size > 4 * p
    n = 6
    xi = sbfem.radial_grid(n, 1e-3, sbfem.XP)
    rho = np.ones((n + 1, el.dofs.size), dtype=sbfem.XP)
    mats = sbfem.coefficient_matrices(el, m.node_xy, p, 1.0, rho)
    one = np.ones(el.dofs.size)
    scale = float(np.abs(np.asarray(mats[0], dtype=np.float64)).max())
    assert np.abs(np.asarray(mats[1].transpose(0, 2, 1) @ one, dtype=np.float64)).max() < 1e-13 * scale
    assert np.abs(np.asarray(mats[2] @ one, dtype=np.float64)).max() < 1e-13 * scale
    cd = sbfem.condense(sbfem.element_system(*(q[None] for q in mats), xi, 1.0, 0.25, static=True))
    S = np.asarray(cd.S[0], dtype=np.float64)
    assert np.abs(S @ one).max() < 1e-10 * np.abs(S).max()


@pytest.mark.parametrize("p", [2, 3])
def test_uneven_condensed_path_equals_uncondensed_system(p):
    """Condensed path (elements grouped by n_b) against the uncondensed element systems
    with ghosts and flux-balance rows, solved directly each step."""
    m = _corner_refined(p)
    assert len(set(m.n_b)) == 2
    n_r, c = 5, 1.0
    s = min_spacing(m)
    dt, f0, K = 0.5 * s / c, c / (10 * s), 30
    w = np.stack([ricker(f0, dt, K), 0.7 * ricker(f0, dt, K, t0=1.2 / f0)])
    rho = 1.0 + 0.2 * np.random.default_rng(0).random((16, 16))
    src, rec = np.array([3, 20]), np.array([5, 9, 30])
    md = uneven.build_model(m, n_r, c, rho, dt)
    tr, _, st = uneven.forward(md, src, w, rec)
    fs = uneven.FullSystem(m, n_r, c, md.rho_nodal, dt)
    tr2, u2 = fs.forward(src, w, rec)
    assert np.linalg.norm(tr) > 0
    assert np.linalg.norm(tr - tr2) <= 1e-11 * np.linalg.norm(tr)
    for k, g in enumerate(md.groups):
        for q, e in enumerate(g.elems):
            assert np.linalg.norm(st.u[k][q] - u2[e]) <= 1e-11 * np.linalg.norm(u2[e])


def test_uneven_path_equals_uniform_oracle_on_structured_mesh():
    """On a mesh with one n_b the grouped path is the uniform one: traces, stored
    velocities and the velocity kernel agree to rounding."""
    m = structured_mesh(3, 2, 2)
    n_r, c = 6, 1.0
    dt, f0, K = 0.5 * 0.25 / c, c / (10 * 0.25), 25
    w = np.stack([ricker(f0, dt, K)])
    rho = 1.0 + 0.3 * np.random.default_rng(1).random((12, 12))
    src, rec = np.array([2]), np.array([0, 7, 11])
    a = fwi.build_model(m, n_r, c, rho, dt)
    b = uneven.build_model(m, n_r, c, rho, dt)
    tra, sta, _ = fwi.forward(a, src, w, rec)
    trb, stb, _ = uneven.forward(b, src, w, rec)
    assert np.linalg.norm(tra - trb) <= 1e-13 * np.linalg.norm(tra)
    assert np.linalg.norm(sta - stb) <= 1e-13 * np.linalg.norm(sta)
    obs = 1.1 * tra
    _, res = fwi.misfit(tra, obs, dt)
    ga = fwi.adjoint_gradient(a, sta, res, rec)
    gb = uneven.adjoint_gradient(b, stb, res, rec)
    assert np.linalg.norm(ga - gb) <= 1e-12 * np.linalg.norm(ga)


def test_voronoi_mesh_is_a_conforming_ccw_tiling():
    m = voronoi_mesh(60, 2, seed=3)
    sides = np.diff(m.elem_ptr)
    assert sides.min() >= 3 and sides.max() > sides.min()
    seen = set()
    area = 0.0
    for e in range(m.n_elem):
        ls = m.line_nodes[m.elem_ptr[e]:m.elem_ptr[e + 1]]
        c = m.centre_xy[e]
        for k, ln in enumerate(ls):
            assert ln[-1] == ls[(k + 1) % len(ls)][0]                  # closed loop
            a, b = m.node_xy[ln[0]], m.node_xy[ln[-1]]
            assert (a[0] - c[0]) * (b[1] - a[1]) - (a[1] - c[1]) * (b[0] - a[0]) > 0   # centre sees it CCW
            assert (ln[0], ln[-1]) not in seen
            seen.add((int(ln[0]), int(ln[-1])))
        P = m.node_xy[[ln[0] for ln in ls]]
        area += 0.5 * np.sum(P[:, 0] * np.roll(P[:, 1], -1) - np.roll(P[:, 0], -1) * P[:, 1])
    assert abs(area - 1.0) < 1e-12
    for a, b in seen:                                                   # interior sides shared, reversed
        if (b, a) not in seen:
            mid = 0.5 * (m.node_xy[a] + m.node_xy[b])
            assert np.isclose(mid, 0).any() or np.isclose(mid, 1).any()


@pytest.mark.parametrize("p", [1, 2])
def test_polygon_element_static_stiffness_annihilates_constants(p):
    m = voronoi_mesh(12, p, seed=5)
    for el in sbfem.elements_from_mesh(m)[:4]:
        xi = sbfem.radial_grid(5, 1e-3, sbfem.XP)
        mats = sbfem.coefficient_matrices(el, m.node_xy, p, 1.0, np.ones((6, el.dofs.size), dtype=sbfem.XP))
        cd = sbfem.condense(sbfem.element_system(*(q[None] for q in mats), xi, 1.0, 0.25, static=True))
        S = np.asarray(cd.S[0], dtype=np.float64)
        assert np.abs(S @ np.ones(el.dofs.size)).max() < 1e-10 * np.abs(S).max()


def test_voronoi_condensed_path_equals_uncondensed_system():
    m = voronoi_mesh(8, 2, seed=7)
    assert len(set(m.n_b)) > 1
    n_r, c = 5, 1.0
    s = min_spacing(m)
    dt, f0, K = 0.5 * s / c, c / (10 * s), 30
    w = np.stack([ricker(f0, dt, K, t0=1.0 / f0)])
    rho = 1.0 + 0.3 * np.random.default_rng(2).random((16, 16))
    src, rec = np.array([0]), np.array([1, 5, 9])
    md = uneven.build_model(m, n_r, c, rho, dt)
    tr, _, st = uneven.forward(md, src, w, rec)
    tr2, u2 = uneven.FullSystem(m, n_r, c, md.rho_nodal, dt).forward(src, w, rec)
    assert np.linalg.norm(tr) > 0
    assert np.linalg.norm(tr - tr2) <= 1e-11 * np.linalg.norm(tr)


def test_uneven_full_kernel_and_gradient_operator():
    """The full kernel's gradient term on grouped elements equals the uniform oracle's on a
    uniform mesh, and the nodal gradient is exact for quadratic fields on a quadtree with
    hanging vertices (lines of a split side are short: the operator takes each line's own
    geometry)."""
    m = structured_mesh(3, 2, 2)
    w = ricker(0.8, 0.125, 30)[None]
    rho = 1 + 0.3 * np.random.default_rng(1).random((12, 12))
    a = fwi.build_model(m, 6, 1.0, rho, 0.125)
    b = uneven.build_model(m, 6, 1.0, rho, 0.125)
    rec = [0, 7, 11]
    ta, sa, _, ua = fwi.forward(a, [2], w, rec, keep_u=True)
    tb, sb, _, ub = uneven.forward(b, [2], w, rec, keep_u=True)
    ga = fwi.adjoint_gradient(a, sa, 0.1 * ta, rec, store_u=ua)
    gb = uneven.adjoint_gradient(b, sb, 0.1 * tb, rec, store_u=ub)
    assert np.linalg.norm(ga - gb) <= 1e-12 * np.linalg.norm(ga)
    mq = _corner_refined(3, base=4)
    bq = uneven.build_model(mq, 5, 1.0, rho, 0.05)
    G = fwi.gradient_operator(bq)
    x, y = (np.asarray(bq.points[:, k], dtype=np.float64) for k in (0, 1))
    g = (G @ (x * x + x * y)).reshape(-1, 2)
    assert np.abs(g - np.c_[2 * x + y, x]).max() < 1e-9
