"""Pins of the oracle's element algebra (Section 3) against closed forms and identities.

These tests check the CPU oracle against facts fixed by the mathematics, not
against itself: shape-function identities, Gauss exactness, the boundary
Jacobian identity of Section 3 (Eq. (substitute)), the partition-of-unity
null spaces of E1^T and E2, the area carried by M0, and the static dynamic
stiffness annihilating constant fields.
"""

import math

import numpy as np
import pytest

from oracle import sbfem, fwi
from sbfwi_inputs import structured_mesh


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_lagrange_partition_of_unity_and_kronecker(p):
    eta = np.linspace(-1, 1, 37)
    phi, dphi = sbfem.lagrange(p, eta)
    assert np.allclose(phi.sum(axis=1), 1.0, atol=1e-13)
    assert np.allclose(dphi.sum(axis=1), 0.0, atol=1e-11)
    at_nodes, _ = sbfem.lagrange(p, sbfem.lagrange_nodes(p))
    assert np.allclose(at_nodes, np.eye(p + 1), atol=1e-13)
    # derivative against a central difference of the function itself
    h = 1e-6
    fp, _ = sbfem.lagrange(p, eta + h)
    fm, _ = sbfem.lagrange(p, eta - h)
    assert np.allclose(dphi, (fp - fm) / (2 * h), atol=1e-7)
    # reproduces eta^k exactly for k <= p
    nodes = sbfem.lagrange_nodes(p)
    for k in range(p + 1):
        assert np.allclose(phi @ nodes ** k, eta ** k, atol=1e-12)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
def test_gauss_rule_integrates_degree_3p(p):
    x, w = sbfem.gauss_points(p)
    for k in range(0, 3 * p + 1):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.sum(w * x ** k) - exact) < 1e-13


def _square_element(p, a=0.3, centre=(0.1, -0.2), shift=(0.0, 0.0)):
    """Square of side a around ``centre`` with the scaling centre shifted by ``shift``."""
    cx, cy = centre
    corners = np.array([(cx - a / 2, cy - a / 2), (cx + a / 2, cy - a / 2),
                        (cx + a / 2, cy + a / 2), (cx - a / 2, cy + a / 2)])
    nb = 4 * p
    xy = np.array([corners[k] + (corners[(k + 1) % 4] - corners[k]) * m / p
                   for k in range(4) for m in range(p)])
    lines = [np.array([(k * p + m) % nb for m in range(p + 1)]) for k in range(4)]
    el = sbfem.make_element(np.array([cx + shift[0], cy + shift[1]]), lines)
    return el, xy, a


@pytest.mark.parametrize("p", [1, 2, 4])
def test_boundary_jacobian_identity_and_area(p):
    el, xy, a = _square_element(p, shift=(0.03, -0.05))
    eta_g, w = sbfem.gauss_points(p)
    area = 0.0
    for ln in el.lines:
        _, _, det, b1, b2 = sbfem.line_geometry(xy[ln], el.centre, p, eta_g)
        assert np.all(det > 0)
        area += 0.5 * np.sum(w * det)          # dOmega = det J_b xi dxi deta
        # Eq. (substitute): d/deta (det J_b b2) = -det J_b b1, by central differences in eta
        e = np.linspace(-0.9, 0.9, 7)
        h = 1e-6
        _, _, dp, _, b2p = sbfem.line_geometry(xy[ln], el.centre, p, e + h)
        _, _, dm, _, b2m = sbfem.line_geometry(xy[ln], el.centre, p, e - h)
        _, _, d0, b10, _ = sbfem.line_geometry(xy[ln], el.centre, p, e)
        lhs = (dp[:, None] * b2p - dm[:, None] * b2m) / (2 * h)
        assert np.allclose(lhs, -d0[:, None] * b10, atol=1e-6)
    assert abs(area - a * a) < 1e-14


@pytest.mark.parametrize("p", [1, 2, 4])
def test_coefficient_matrix_identities(p):
    el, xy, a = _square_element(p, shift=(0.02, 0.04))
    nb = el.dofs.size
    rng = np.random.default_rng(3)
    rho = 0.5 + rng.random((3, nb))                  # variable density along eta
    E0, E1, E2, M0 = [np.asarray(a, dtype=np.float64) for a in sbfem.coefficient_matrices(el, xy, p, 1.7, rho)]
    one = np.ones(nb)
    for m in range(3):
        # partition of unity: sum_a d phi_a / d eta = 0
        assert np.abs(E1[m].T @ one).max() < 1e-13 * np.abs(E1[m]).max()
        assert np.abs(E2[m] @ one).max() < 1e-13 * np.abs(E2[m]).max()
        for M in (E0[m], E2[m], M0[m]):
            assert np.allclose(M, M.T, atol=1e-14 * np.abs(M).max())
        assert np.linalg.eigvalsh(E0[m]).min() > 0
        assert np.linalg.eigvalsh(M0[m]).min() > 0
    # homogeneous density: 1^T M0 1 = int rho det J_b deta = 2 rho * area
    E0h, E1h, E2h, M0h = [np.asarray(a, dtype=np.float64) for a in sbfem.coefficient_matrices(el, xy, p, 1.0, np.full((1, nb), 2.5))]
    assert abs(one @ M0h[0] @ one - 2 * 2.5 * a * a) < 1e-13
    # E-matrices are linear in the nodal density and c^2 scales E0..E2 only
    E0b, E1b, E2b, M0b = [np.asarray(a, dtype=np.float64) for a in sbfem.coefficient_matrices(el, xy, p, 2.0, np.full((1, nb), 2.5))]
    assert np.allclose(E0b, 4 * E0h) and np.allclose(M0b, M0h)


@pytest.mark.parametrize("nx,p,nr", [(2, 1, 4), (4, 2, 8), (3, 4, 6)])
def test_static_stiffness_annihilates_constants(nx, p, nr):
    mesh = structured_mesh(nx, nx, p)
    rng = np.random.default_rng(nx)
    rho = 0.6 + 0.8 * rng.random((16, 16))
    m = fwi.build_model(mesh, nr, 1.3, rho, 1.0, static=True)
    one = np.ones(m.S.shape[1])
    for S in m.S:
        assert np.abs(S @ one).max() < 1e-11 * np.abs(S).max()


def test_radial_grid_and_fd_of_E():
    xi = sbfem.radial_grid(7, 1e-3)
    assert xi[0] == 1e-3 and xi[-1] == 1.0
    assert np.allclose(np.diff(xi), (1 - 1e-3) / 7)
    # one-sided at the ends, central inside: exact for a linear function
    E = (2.0 + 3.0 * xi)[:, None, None] * np.ones((1, 2, 2))
    dE = sbfem.radial_derivative(E, (1 - 1e-3) / 7)
    assert np.allclose(dE, 3.0)
    # and second-order accurate inside for a quadratic
    E = (xi ** 2)[:, None, None] * np.ones((1, 1, 1))
    dE = sbfem.radial_derivative(E, (1 - 1e-3) / 7)
    assert np.allclose(dE[1:-1, 0, 0], 2 * xi[1:-1])
