"""Host-side checks of libsbfwi: it builds, loads, exports every declared entry point,
and validates meshes and builds the elimination tree without a GPU."""

import ctypes
import os
import re

import numpy as np
import pytest

from sbfwi_inputs import structured_mesh

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def binding():
    from paper_2501_06748_gb300 import build
    build.build()
    from paper_2501_06748_gb300 import sbfwi
    return sbfwi


def test_library_exports_every_declared_symbol(binding):
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            names |= set(re.findall(r"^\w[\w\s\*]*?\b(sbfwi_\w+)\s*\(", text, flags=re.M))
    assert {"sbfwi_build_mesh", "sbfwi_set_model", "sbfwi_forward", "sbfwi_misfit",
            "sbfwi_adjoint_gradient"} <= names
    lib = ctypes.CDLL(binding.LIB_PATH)
    for n in sorted(names):
        assert hasattr(lib, n), n
    assert binding.version() >= 100


def test_mesh_info_and_elimination_tree(binding):
    m = structured_mesh(4, 4, 2)
    M = binding.Mesh.from_inputs(m, 8)
    assert (M.n_elem, M.n_nodes, M.n_b, M.n_r) == (16, 65, 8, 8)
    assert M.n_int == 16 * 7 * 8 and M.n_nodal == M.n_int + 65
    assert M.tree_levels == 5                          # 16 leaves -> 8 -> 4 -> 2 -> 1
    big = binding.Mesh.from_inputs(structured_mesh(64, 64, 4), 32)
    assert big.n_nodes == 29185 and big.tree_levels == 13
    # the factors of a 2-D nested dissection stay far below a dense matrix
    assert big.factor_entries < 0.02 * big.n_nodes ** 2


def test_mesh_info_of_elements_with_different_boundary_node_counts(binding):
    """Quadtree mesh with hanging vertices: n_b is the largest count, and the nodal
    layout seen by callers has no padding (n_int = n * sum of n_b(e))."""
    from sbfwi_inputs import quadtree_mesh
    m = quadtree_mesh(3, 1, lambda x0, y0, x1, y1, lvl: not (1 / 3 <= x0 < 0.5 and 1 / 3 <= y0 < 0.5), 5)
    nbs = m.n_b
    assert nbs.max() == 40 and nbs.min() == 20        # the centre cell has four finer neighbours
    M = binding.Mesh.from_inputs(m, 6)
    assert (M.n_elem, M.n_nodes, M.n_b) == (m.n_elem, m.n_nodes, 40)
    assert M.n_int == 5 * int(nbs.sum()) and M.n_nodal == M.n_int + m.n_nodes
    # more than 40 boundary nodes is outside this build
    m9 = quadtree_mesh(3, 1, lambda x0, y0, x1, y1, lvl: not (1 / 3 <= x0 < 0.5 and 1 / 3 <= y0 < 0.5), 6)
    with pytest.raises(binding.SbfwiError) as ei:
        binding.Mesh.from_inputs(m9, 6)
    assert ei.value.code == binding.EUNSUPPORTED


def test_voronoi_mesh_builds_with_its_elimination_tree(binding):
    """A centroidal Voronoi mesh (4 to 8 sides per polygon) passes the library's checks
    (closed CCW loops, straight equally spaced lines, det J_b > 0) and gets a tree."""
    from sbfwi_inputs import voronoi_mesh
    m = voronoi_mesh(400, 2, seed=2)
    M = binding.Mesh.from_inputs(m, 6)
    assert (M.n_elem, M.n_nodes, M.n_b) == (400, m.n_nodes, int(m.n_b.max()))
    assert M.n_int == 5 * int(m.n_b.sum())
    assert 8 <= M.tree_levels <= 12 and M.factor_entries > 0


def test_lfe_element_matrices_match_the_oracle(binding):
    """The comparison method's element K (Riccati, by the matrix sign function) and M
    (Lyapunov) computed by the library on the host agree with the oracle's (eigenvector
    Riccati basis, dense Kronecker Lyapunov) on square, quadtree, Voronoi and n_b = 40
    elements with a density that varies along the boundary."""
    from oracle import lfe, sbfem
    from sbfwi_inputs import quadtree_mesh, voronoi_mesh
    meshes = [structured_mesh(2, 2, 2), quadtree_mesh(4, 1, lambda *a: a[0] < 0.5 and a[1] < 0.5, 3),
              voronoi_mesh(30, 2, seed=1),
              quadtree_mesh(3, 1, lambda x0, y0, x1, y1, lvl: not (1 / 3 <= x0 < 0.5 and 1 / 3 <= y0 < 0.5), 5)]
    for m in meshes:
        for el in sbfem.elements_from_mesh(m)[:4]:
            nb = el.dofs.size
            rho = np.tile((1 + 0.3 * np.random.default_rng(nb).random(nb)).astype(sbfem.XP), (2, 1))
            E0, E1, E2, M0 = (np.asarray(q[-1], dtype=np.float64)
                              for q in sbfem.coefficient_matrices(el, m.node_xy, m.p, 1.0, rho))
            K, _ = lfe.riccati_stiffness(E0, E1, E2)
            M = lfe.lyapunov_mass(K, E0, E1, M0)
            K2, M2 = binding.lfe_element_matrices(E0, E1, E2, M0)
            assert np.abs(K2 - K).max() <= 1e-12 * np.abs(K).max()
            assert np.abs(M2 - M).max() <= 1e-12 * np.abs(M).max()
    with pytest.raises(binding.SbfwiError) as ei:
        binding.lfe_element_matrices(*(np.zeros((1, 1)),) * 4)
    assert ei.value.code == binding.EINVAL


def _bad(binding, **kw):
    m = structured_mesh(2, 2, 2)
    args = dict(node_xy=m.node_xy.copy(), elem_ptr=m.elem_ptr.copy(), line_nodes=m.line_nodes.copy(),
                centre_xy=m.centre_xy.copy(), p=2, n_r=5, xi0=1e-3)
    args.update(kw)
    with pytest.raises(binding.SbfwiError) as ei:
        binding.Mesh(**args)
    return ei.value


def test_mesh_validation_errors(binding):
    m = structured_mesh(2, 2, 2)
    e = _bad(binding, n_r=2)
    assert e.code == binding.EINVAL
    lines = m.line_nodes.copy()
    lines[0] = lines[0][::-1]                              # breaks the closed CCW loop
    assert _bad(binding, line_nodes=lines).code == binding.EINVAL
    cw = m.line_nodes.reshape(4, 4, 3)[:, ::-1, ::-1].reshape(-1, 3).copy()   # clockwise loops
    err = _bad(binding, line_nodes=cw)
    assert err.code == binding.EINVAL and "det J_b" in str(err)
    centres = m.centre_xy.copy()
    centres[1] = (5.0, 5.0)                                # centre outside its element
    assert "element 1" in str(_bad(binding, centre_xy=centres))
    xy = m.node_xy.copy()
    xy[m.line_nodes[0][1]] += (0.0, 0.01)                  # mid-node off the straight line
    assert _bad(binding, node_xy=xy).code == binding.EINVAL
    ln = m.line_nodes.copy()
    ln[3, 1] = 10_000
    assert _bad(binding, line_nodes=ln).code == binding.EINVAL


def test_compute_calls_fail_loudly_without_a_device(binding):
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a CUDA device is present")
    except ImportError:
        pass
    M = binding.Mesh.from_inputs(structured_mesh(2, 2, 1), 4)
    with pytest.raises(binding.SbfwiError) as ei:
        binding.Model(M, 1.0, np.ones((8, 8)), 0.1)
    assert ei.value.code == binding.ECUDA
    with pytest.raises(binding.SbfwiError):
        binding.misfit(np.zeros(3), np.ones(3), 0.1)
    with pytest.raises(binding.SbfwiError) as ei:
        binding.selftest_barrier(4, 1)
    assert ei.value.code == binding.ECUDA


def test_misfit_wrappers_check_lengths_before_the_call(binding):
    """The C entry points take one sample count n for every array; the binding refuses
    arrays of different lengths before calling them (a short device array would be read
    or written beyond its end)."""
    with pytest.raises(ValueError):
        binding.misfit(np.zeros(5), np.ones(4), 0.1)
    with pytest.raises(ValueError):
        binding.misfit(np.zeros(5), np.ones(5), 0.1, residual_out=np.zeros(3))


def test_lfe_refuses_an_element_whose_stable_subspace_has_the_wrong_rank(binding):
    """K is built from the n_b - 1 stable eigen-solutions plus the constant mode; that split
    exists because E1^T 1 = E2 1 = 0 gives the constant mode an exact zero pair.  Coefficient
    matrices that break it (E2 + 0.1 max|E2| I: the pair splits into +-0.73, one of them joins
    the stable side, 8 = n_b stable solutions) must be refused, not given a wrong subspace;
    a tiny perturbation that keeps the split is still accepted."""
    from oracle import sbfem
    m = structured_mesh(2, 2, 2)
    el = sbfem.elements_from_mesh(m)[0]
    nb = el.dofs.size
    E0, E1, E2, M0 = (np.asarray(q[0], dtype=np.float64)
                      for q in sbfem.coefficient_matrices(el, m.node_xy, m.p, 1.0, np.ones((1, nb), dtype=sbfem.XP)))
    binding.lfe_element_matrices(E0, E1, E2 + 1e-3 * np.abs(E2).max() * np.eye(nb), M0)
    with pytest.raises(binding.SbfwiError) as ei:
        binding.lfe_element_matrices(E0, E1, E2 + 0.1 * np.abs(E2).max() * np.eye(nb), M0)
    assert ei.value.code == binding.ESINGULAR and "n_b - 1" in str(ei.value)


def test_mesh3d_info_and_validation(binding):
    """sbfwi_build_mesh3d (host code): node and boundary-node counts of hexahedral
    S-elements, and the checks on face orientation, closure and size."""
    from sbfwi_inputs.mesh3d import structured_mesh3d
    m = structured_mesh3d(3, 2, 2, 2)
    M = binding.Mesh.from_inputs(m, 6)
    assert (M.dim, M.n_elem, M.n_nodes, M.n_b) == (3, 12, 7 * 5 * 5 - 12, 26)
    assert M.n_nodal == 5 * 26 * 12 + M.n_nodes and M.tree_levels >= 4
    M1 = binding.Mesh.from_inputs(structured_mesh3d(2, 2, 2, 1), 5)
    assert (M1.n_nodes, M1.n_b) == (27, 8)
    args = dict(node_xy=m.node_xyz, elem_ptr=m.elem_ptr, line_nodes=m.face_nodes, centre_xy=m.centre_xyz, p=2, n_r=6)
    # a face turned inward (eta and zeta swapped): det J_b < 0
    bad = m.face_nodes.copy()
    bad[0] = bad[0].reshape(3, 3).T.ravel()
    with pytest.raises(binding.SbfwiError) as ei:
        binding.Mesh(**{**args, "line_nodes": bad})
    assert ei.value.code == binding.EINVAL and "det J_b" in str(ei.value)
    # a missing face: the surface is not closed
    ep = m.elem_ptr.copy()
    ep[1:] -= 1
    with pytest.raises(binding.SbfwiError) as ei:
        binding.Mesh(**{**args, "line_nodes": m.face_nodes[1:], "elem_ptr": ep})
    assert ei.value.code == binding.EINVAL and "close" in str(ei.value)
    # p = 3 hexahedra have 56 boundary nodes, above the 40 the kernels take
    m3 = structured_mesh3d(1, 1, 1, 3)
    with pytest.raises(binding.SbfwiError) as ei:
        binding.Mesh.from_inputs(m3, 5)
    assert ei.value.code == binding.EUNSUPPORTED
