"""Three-dimensional scaled-boundary elements (Section 3, carried from the 2-D derivation
to a boundary surface as the paper's Section 3 preamble says it can be), plain numpy.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

An S-element: scaling centre x0 and boundary faces, each a quadrilateral surface element
of Lagrange order p with (p+1)^2 nodes in tensor order, N_ab(eta, zeta) = phi_a(eta)
phi_b(zeta).  The coordinate map is x = x0 + xi (x_b(eta, zeta) - x0) (Eq.
(transformation) with a surface instead of a line).  With the boundary Jacobian

    J_b = [x_b - x0 ; d x_b / d eta ; d x_b / d zeta]        (rows)

the gradient is grad = b1 d/dxi + (1/xi) (b2 d/deta + b3 d/dzeta), b_k the columns of
J_b^{-1} (the counterpart of Eq. (partial3)), and dOmega = xi^2 det J_b dxi deta dzeta.
The Galerkin weak form of Eq. (wave) written as div(rho c^2 grad u) - rho u_tt = 0
with u = N(eta, zeta) u(xi) gives the coefficient matrices (the counterpart of Eq. (Es))

    E0 = int rho c^2 N^T (b1.b1) N det J_b
    E1 = int rho c^2 B2^T b1 N det J_b,     B2 = b2 N_eta + b3 N_zeta
    E2 = int rho c^2 B2^T B2 det J_b
    M0 = int rho N^T N det J_b

(integrals over the faces in eta, zeta), with rho(xi, eta, zeta) = sum_j N_j rho_j(xi),
and the radial equation (the counterpart of Eq. (ODE))

    xi^2 E0 u'' + xi (2 E0 + E1^T - E1 + xi E0') u' + (E1^T - E2 + xi E1^T') u
        - xi^2 M0 u_tt = 0,

internal source vector q = xi^2 E0 u' + xi E1^T u (the counterpart of Eq. (internal)).
Compared with 2-D, the u' coefficient has 2 E0 instead of E0 and the u coefficient gains
E1^T; at xi = 1 the boundary row is the same, and at xi0 the zero-flux row divided by
xi0 is the same as in 2-D.  The blocks, the condensation and the time loop are those of
``oracle.sbfem`` with ``element_system(..., dim=3)``.

Parity status: pinned by ``tests/test_oracle_3d.py``: Gauss exactness of the face rule,
the boundary-Jacobian volume identity, the constant-field identities of E1 and E2, the
mass identity 1^T M0 1 = 3 rho V, the static stiffness annihilating constants and
reproducing the flux of a linear field, free-vibration frequencies of a homogeneous cube
(Neumann Laplacian closed form) and of an exponentially graded density (closed form,
which exercises the d/dxi E terms), and the brute-force uncondensed solve.
"""

from dataclasses import dataclass

import numpy as np

from . import sbfem

XP = sbfem.XP


@dataclass
class Element3D:
    centre: np.ndarray            # (3,) scaling centre
    faces: list                   # list of ((p+1)^2,) global node ids, tensor order
    dofs: np.ndarray              # (n_b,) global ids of the element's boundary nodes
    face_local: list              # list of ((p+1)^2,) local indices into dofs


def make_element3d(centre, faces) -> Element3D:
    """Local boundary-node numbering: order of first appearance over the faces."""
    order, index = [], {}
    for f in faces:
        for g in f:
            g = int(g)
            if g not in index:
                index[g] = len(order)
                order.append(g)
    face_local = [np.array([index[int(g)] for g in f]) for f in faces]
    return Element3D(np.asarray(centre, dtype=np.float64), [np.asarray(f) for f in faces],
                     np.array(order, dtype=np.int64), face_local)


def elements_from_mesh3d(mesh):
    out = []
    for e in range(mesh.n_elem):
        fs = mesh.face_nodes[mesh.elem_ptr[e]:mesh.elem_ptr[e + 1]]
        out.append(make_element3d(mesh.centre_xyz[e], [fs[k] for k in range(fs.shape[0])]))
    return out


def face_rule(p: int, dtype=XP):
    """Tensor Gauss rule on [-1, 1]^2 and the face shape functions at its points.

    On a planar face with straight edges det J_b is constant, b1 constant and b2, b3
    linear in each variable, so every integrand above is a polynomial of degree <= 3p + 2
    in each of eta, zeta; (3p + 4) // 2 points per direction integrate it exactly.
    Returns eta, zeta, w (g,) and N, N_eta, N_zeta (g, (p+1)^2).
    """
    x, w1 = sbfem.legendre_gauss((3 * p + 4) // 2, dtype)
    phi, dphi = sbfem.lagrange(p, x)
    ng, pp = x.size, p + 1
    # point (ga, gb) at index ga + ng gb; node (a, b) at a + pp b
    eta = np.tile(x, ng)
    zeta = np.repeat(x, ng)
    w = np.tile(w1, ng) * np.repeat(w1, ng)
    N = np.einsum("ia,jb->jiba", phi, phi).reshape(ng * ng, pp * pp)
    Ne = np.einsum("ia,jb->jiba", dphi, phi).reshape(ng * ng, pp * pp)
    Nz = np.einsum("ia,jb->jiba", phi, dphi).reshape(ng * ng, pp * pp)
    return eta, zeta, w, N, Ne, Nz


def face_geometry(xyz_face: np.ndarray, centre: np.ndarray, N, Ne, Nz):
    """Boundary map of one face at the rule's points: r_b = x_b - x0, det J_b and the
    columns b1, b2, b3 of J_b^{-1} (each (g, 3)), in the floating type of N."""
    X = np.asarray(xyz_face).astype(N.dtype)
    c = np.asarray(centre).astype(N.dtype)
    rb = N @ X - c[None, :]
    xe = Ne @ X
    xz = Nz @ X
    # J_b rows (rb, xe, xz); its inverse columns by the cofactor formula
    det = np.einsum("gi,gi->g", rb, np.cross(xe, xz))
    b1 = np.cross(xe, xz) / det[:, None]
    b2 = np.cross(xz, rb) / det[:, None]
    b3 = np.cross(rb, xe) / det[:, None]
    return rb, det, b1, b2, b3


def coefficient_matrices3d(el: Element3D, node_xyz: np.ndarray, p: int, c: float, rho_local: np.ndarray,
                           dtype=XP):
    """E0, E1, E2, M0 of the 3-D element at one or more radial stations.

    ``rho_local`` (m, n_b): nodal densities rho_j(xi) at m radial stations; inside a face
    rho = sum_j N_j rho_j.  Returns four (m, n_b, n_b) arrays in ``dtype``.
    """
    rho_local = np.atleast_2d(np.asarray(rho_local)).astype(dtype)
    m, nb = rho_local.shape
    _, _, w, N, Ne, Nz = face_rule(p, dtype)
    out = [np.zeros((m, nb, nb), dtype=dtype) for _ in range(4)]
    c2 = dtype(c) * dtype(c)
    for f, loc in zip(el.faces, el.face_local):
        _, det, b1, b2, b3 = face_geometry(node_xyz[f], el.centre, N, Ne, Nz)
        rho_g = rho_local[:, loc] @ N.T                                   # (m, g)
        wd = w * det
        dot = lambda u, v: np.sum(u * v, axis=1)
        k0 = c2 * wd * dot(b1, b1)
        B2 = b2[:, :, None] * Ne[:, None, :] + b3[:, :, None] * Nz[:, None, :]    # (g, 3, nodes)
        ix = np.ix_(np.arange(m), loc, loc)
        out[0][ix] += np.einsum("mg,g,ga,gb->mab", rho_g, k0, N, N)
        out[1][ix] += np.einsum("mg,g,gka,gk,gb->mab", rho_g, c2 * wd, B2, b1, N)
        out[2][ix] += np.einsum("mg,g,gka,gkb->mab", rho_g, c2 * wd, B2, B2)
        out[3][ix] += np.einsum("mg,g,ga,gb->mab", rho_g, wd, N, N)
    return tuple(out)


def nodal_points3d(mesh, elements, xi):
    """Physical location of every nodal point: x0 + xi_i (x_j - x0) for i < n, then the
    global nodes (the same layout as ``oracle.fwi.nodal_points``)."""
    n = xi.size - 1
    pts, int_ptr = [], [0]
    for el in elements:
        xj = mesh.node_xyz[el.dofs].astype(xi.dtype)
        p_el = el.centre[None, None, :] + xi[:n, None, None] * (xj[None, :, :] - el.centre[None, None, :])
        pts.append(p_el.reshape(-1, 3))
        int_ptr.append(int_ptr[-1] + n * el.dofs.size)
    pts.append(mesh.node_xyz.astype(xi.dtype))
    return np.concatenate(pts, axis=0), np.asarray(int_ptr, dtype=np.int64)
