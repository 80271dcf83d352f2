"""Scaled-boundary element algebra of the paper's Section 3, in plain numpy.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Everything here follows the paper's notation:

* a 2-D S-element: scaling centre (x0, y0) and boundary line elements of Lagrange
  order p, coordinate map x = x0 + xi (x_b(eta) - x0) (Eq. (transformation));
* boundary Jacobian J_b, det J_b, b1 = [j11, j21], b2 = [j12, j22]
  (Section 3, Eq. (b1b2));
* coefficient matrices E0, E1, E2, M0 with rho(xi, eta) = sum_j phi_j(eta) rho_j(xi)
  (Eq. (Es));
* radial grid xi_i = xi0 + i h, i = 0..n, xi0 = 1e-3 (Section 3.3);
* radial derivative of E0, E1 by central differences inside and one-sided at
  i = 0 and i = n (Section 3.3);
* blocks theta_i, phi_i, psi_i of rows i = -1..n+1 of Eq. (system);
* condensation: rho_0 = theta_0 theta_{-1}^{-1}, Thomas sweep, rho_{n+1}, 2x2
  closure giving S and W = psi_{n+1} psi_n^{-1} (Section 3.3);
* per step: residual source p_i (Eq. (ODE_Newmark)), forward sweep of p, the
  effective source f_hat, and the back-substitution u_i.

Parity status: pinned by the tests in ``tests/test_oracle_*.py``: partition of
unity identities of E1, E2 (exact), the area identity of M0, the static S
annihilating constants, Gauss exactness, free-vibration frequencies of a
homogeneous square and of an exponentially graded density (closed forms), and
the brute-force uncondensed solve (``oracle.bruteforce``).
"""

from dataclasses import dataclass

import numpy as np


# ----------------------------------------------------------------------------
# 1-D Lagrange shape functions and Gauss quadrature on eta in [-1, 1]
# ----------------------------------------------------------------------------

#: Working precision of the set-up (density map, E-matrices, condensation).  The
#: condensation amplifies rounding of the coefficient matrices by about 1e4 (its
#: first pivot is theta_{-1} = -xi0 E0 / (2h) with xi0 = 1e-3), enough for an FP64
#: set-up alone to move receiver traces by ~5e-10 over 400 steps.  The set-up is
#: therefore carried in extended precision and its results rounded to FP64 for
#: the time loop.  numpy's long double is 80-bit extended on x86 and IEEE binary128
#: on AArch64.
XP = np.longdouble


def lagrange_nodes(p: int, dtype=np.float64) -> np.ndarray:
    """Equally spaced Lagrange nodes on [-1, 1] (node placement is not fixed by the paper)."""
    return np.array([-1 + 2 * dtype(k) / p for k in range(p + 1)], dtype=dtype)


def lagrange(p: int, eta: np.ndarray):
    """Shape functions phi_a(eta) and derivatives d phi_a / d eta, shapes (len(eta), p+1).

    Written from the product formula phi_a = prod_{b != a} (eta - eta_b)/(eta_a - eta_b);
    computed in the floating type of ``eta`` (at least float64).
    """
    eta = np.atleast_1d(np.asarray(eta))
    dt_ = np.result_type(eta.dtype, np.float64)
    eta = eta.astype(dt_)
    nodes = lagrange_nodes(p, dt_.type)
    phi = np.ones((eta.size, p + 1), dtype=dt_)
    dphi = np.zeros((eta.size, p + 1), dtype=dt_)
    for a in range(p + 1):
        others = [b for b in range(p + 1) if b != a]
        denom = dt_.type(1)
        for b in others:
            denom *= nodes[a] - nodes[b]
        for b in others:
            phi[:, a] *= (eta - nodes[b])
        phi[:, a] /= denom
        for m in others:               # derivative: sum over the factor that is differentiated
            term = np.ones(eta.size, dtype=dt_)
            for b in others:
                if b != m:
                    term *= (eta - nodes[b])
            dphi[:, a] += term
        dphi[:, a] /= denom
    return phi, dphi


def legendre_gauss(ng: int, dtype=XP):
    """Gauss-Legendre nodes and weights in ``dtype``.

    numpy's float64 rule is polished by Newton steps on P_ng (three-term recurrence);
    weights 2 / ((1 - x^2) P_ng'(x)^2).
    """
    x64, _ = np.polynomial.legendre.leggauss(ng)
    x = x64.astype(dtype)

    def legendre_and_derivative(x):
        p0, p1 = np.ones_like(x), x.copy()
        for k in range(2, ng + 1):
            p0, p1 = p1, ((2 * k - 1) * x * p1 - (k - 1) * p0) / k
        if ng == 1:
            p0 = np.ones_like(x)
        return p1, ng * (x * p1 - p0) / (x * x - 1)

    for _ in range(4):
        pn, dpn = legendre_and_derivative(x)
        x = x - pn / dpn
    _, dpn = legendre_and_derivative(x)
    return x, 2 / ((1 - x * x) * dpn * dpn)


def gauss_points(p: int, dtype=XP):
    """Gauss-Legendre rule exact for the E-matrix integrands of straight line elements.

    With straight edges det J_b and b1 are constant and b2 is linear in eta, so every
    integrand of Eq. (Es) is a polynomial of degree <= 3p; n_g = ceil((3p+1)/2)
    points integrate it exactly.
    """
    return legendre_gauss((3 * p + 2) // 2, dtype)


def inverse(A: np.ndarray) -> np.ndarray:
    """Inverse of a batch of square matrices by Gauss-Jordan with partial pivoting.

    Works in the floating type of ``A`` (numpy's linalg has no long-double routines).
    """
    A = np.asarray(A)
    batch = A.shape[:-2]
    n = A.shape[-1]
    M = np.concatenate([A.reshape(-1, n, n), np.broadcast_to(np.eye(n, dtype=A.dtype), (int(np.prod(batch, dtype=np.int64)), n, n))], axis=2).copy()
    rows = np.arange(M.shape[0])
    for k in range(n):
        piv = k + np.argmax(np.abs(M[:, k:, k]), axis=1)
        top = M[rows, k, :].copy()
        M[rows, k, :] = M[rows, piv, :]
        M[rows, piv, :] = top
        M[:, k, :] = M[:, k, :] / M[:, k, k][:, None]
        f = M[:, :, k].copy()
        f[:, k] = 0
        M = M - f[:, :, None] * M[:, k, None, :]
    return M[:, :, n:].reshape(A.shape)


# ----------------------------------------------------------------------------
# Element description
# ----------------------------------------------------------------------------

@dataclass
class Element:
    centre: np.ndarray            # (2,) scaling centre (x0, y0)
    lines: list                   # list of (p+1,) global node ids, CCW
    dofs: np.ndarray              # (n_b,) global ids of the element's boundary nodes
    line_local: list              # list of (p+1,) local indices into dofs


def make_element(centre, lines) -> Element:
    """Local boundary-node numbering: order of first appearance along the CCW lines."""
    order = []
    for ln in lines:
        for g in ln:
            g = int(g)
            if g not in order:
                order.append(g)
    index = {g: k for k, g in enumerate(order)}
    line_local = [np.array([index[int(g)] for g in ln]) for ln in lines]
    return Element(np.asarray(centre, dtype=np.float64), [np.asarray(l) for l in lines],
                   np.array(order, dtype=np.int64), line_local)


def elements_from_mesh(mesh):
    out = []
    for e in range(mesh.n_elem):
        ls = mesh.line_nodes[mesh.elem_ptr[e]:mesh.elem_ptr[e + 1]]
        out.append(make_element(mesh.centre_xy[e], [ls[k] for k in range(ls.shape[0])]))
    return out


def radial_grid(n: int, xi0: float = 1e-3, dtype=XP) -> np.ndarray:
    """xi_i = xi0 + i h, h = (1 - xi0)/n, i = 0..n, with xi_n set to exactly 1 (Section 3.3)."""
    xi0 = dtype(xi0)
    h = (1 - xi0) / n
    xi = xi0 + h * np.arange(n + 1).astype(dtype)
    xi[-1] = 1
    return xi


# ----------------------------------------------------------------------------
# Geometry and coefficient matrices
# ----------------------------------------------------------------------------

def line_geometry(xy_line: np.ndarray, centre: np.ndarray, p: int, eta: np.ndarray):
    """Boundary map of one line element at points eta (Section 3 preamble).

    Returns x_b - x0 (shape (g, 2)), d x_b / d eta (g, 2), det J_b (g,), b1 (g, 2), b2 (g, 2)
    with J_b = [[x_b - x0, y_b - y0], [x_b,eta, y_b,eta]],
    b1 = [j11, j21] = [y_b,eta, -x_b,eta] / det J_b and
    b2 = [j12, j22] = [-(y_b - y0), x_b - x0] / det J_b.
    Computed in the floating type of ``eta``.
    """
    phi, dphi = lagrange(p, eta)
    xy_line = np.asarray(xy_line).astype(phi.dtype)
    centre = np.asarray(centre).astype(phi.dtype)
    rb = phi @ xy_line - centre[None, :]
    xe = dphi @ xy_line
    det = rb[:, 0] * xe[:, 1] - rb[:, 1] * xe[:, 0]
    b1 = np.stack([xe[:, 1], -xe[:, 0]], axis=1) / det[:, None]
    b2 = np.stack([-rb[:, 1], rb[:, 0]], axis=1) / det[:, None]
    return rb, xe, det, b1, b2


def coefficient_matrices(el: Element, node_xy: np.ndarray, p: int, c: float, rho_local: np.ndarray,
                         dtype=XP):
    """E0, E1, E2, M0 of Eq. (Es) at one or more radial stations.

    ``rho_local`` has shape (m, n_b): the nodal densities rho_j(xi) of the element's
    boundary nodes at m radial stations.  The density inside a line element is
    rho(xi, eta) = sum_j phi_j(eta) rho_j(xi).  Returns four arrays (m, n_b, n_b) in
    ``dtype``:

      E0 = int rho c^2 phi^T (b1.b1) phi det J_b d eta
      E1 = int rho c^2 phi_eta^T (b2.b1) phi det J_b d eta
      E2 = int rho c^2 phi_eta^T (b2.b2) phi_eta det J_b d eta
      M0 = int rho phi^T phi det J_b d eta
    """
    rho_local = np.atleast_2d(np.asarray(rho_local)).astype(dtype)
    m, nb = rho_local.shape
    eta, w = gauss_points(p, dtype)
    phi, dphi = lagrange(p, eta)
    E0 = np.zeros((m, nb, nb), dtype=dtype)
    E1 = np.zeros((m, nb, nb), dtype=dtype)
    E2 = np.zeros((m, nb, nb), dtype=dtype)
    M0 = np.zeros((m, nb, nb), dtype=dtype)
    c2 = dtype(c) * dtype(c)
    for ln, loc in zip(el.lines, el.line_local):
        _, _, det, b1, b2 = line_geometry(node_xy[ln], el.centre, p, eta)
        rho_g = rho_local[:, loc] @ phi.T                      # (m, g)
        wd = w * det                                            # (g,)
        k0 = rho_g * (c2 * wd * np.sum(b1 * b1, axis=1))[None, :]
        k1 = rho_g * (c2 * wd * np.sum(b2 * b1, axis=1))[None, :]
        k2 = rho_g * (c2 * wd * np.sum(b2 * b2, axis=1))[None, :]
        km = rho_g * wd[None, :]
        ix = np.ix_(np.arange(m), loc, loc)
        E0[ix] += np.einsum("mg,ga,gb->mab", k0, phi, phi)
        E1[ix] += np.einsum("mg,ga,gb->mab", k1, dphi, phi)
        E2[ix] += np.einsum("mg,ga,gb->mab", k2, dphi, dphi)
        M0[ix] += np.einsum("mg,ga,gb->mab", km, phi, phi)
    return E0, E1, E2, M0


def radial_derivative(E: np.ndarray, h) -> np.ndarray:
    """d E / d xi over the radial axis (axis -3): forward difference at i = 0, backward at
    i = n, central inside."""
    dE = np.empty_like(E)
    dE[..., 0, :, :] = (E[..., 1, :, :] - E[..., 0, :, :]) / h
    dE[..., -1, :, :] = (E[..., -1, :, :] - E[..., -2, :, :]) / h
    dE[..., 1:-1, :, :] = (E[..., 2:, :, :] - E[..., :-2, :, :]) / (2 * h)
    return dE


# ----------------------------------------------------------------------------
# Blocks of Eq. (system) and the condensation (batched over elements)
# ----------------------------------------------------------------------------

def _T(A):
    return np.swapaxes(A, -1, -2)


@dataclass
class ElementSystem:
    """Rows i = -1..n+1 of Eq. (system), stored at index i+1, for a batch of elements."""
    xi: np.ndarray          # (n+1,)
    h: object
    theta: np.ndarray       # (E, n+3, n_b, n_b)
    phi: np.ndarray
    psi: np.ndarray
    M0: np.ndarray          # (E, n+1, n_b, n_b) at the radial points


def element_system(E0, E1, E2, M0, xi, dt, beta, static=False, dim=2) -> ElementSystem:
    """Blocks theta_i, phi_i, psi_i of the discretised radial ODE (Section 3.3).

    ``E0..M0`` have shape (E, n+1, n_b, n_b).  For i = 0..n (Eq. (discretized) with
    the central differences of Eq. (FD)):
      D_i     = E0 + E1^T - E1 + xi_i dE0/dxi
      theta_i = xi_i^2 E0 / h^2 - xi_i D_i / (2h)
      phi_i   = -2 xi_i^2 E0 / h^2 - E2 + xi_i (dE1/dxi)^T - xi_i^2 M0 / (beta dt^2)
      psi_i   = xi_i^2 E0 / h^2 + xi_i D_i / (2h)
    ``dim=3``: the radial equation of a 3-D element (``oracle.sbfem3d``), D_i with 2 E0
    instead of E0 and phi_i with + E1^T; the boundary-condition rows are unchanged.
    Boundary-condition rows (internal source vector q = xi E0 u' + E1^T u, Eq. (internal)):
      row -1 at xi_0: theta = -xi_0 E0(xi_0)/(2h), phi = E1(xi_0)^T, psi = xi_0 E0(xi_0)/(2h)
      row n+1 at xi_n: theta = -xi_n E0(xi_n)/(2h), phi = E1(xi_n)^T, psi = xi_n E0(xi_n)/(2h)
    ``static=True`` drops the mass term (the limit 1/(beta dt^2) -> 0).
    """
    dtype = E0.dtype.type
    n = xi.size - 1
    h = (1 - xi[0]) / n
    dE0 = radial_derivative(E0, h)
    dE1 = radial_derivative(E1, h)
    Ee, _, nb, _ = E0.shape
    theta = np.zeros((Ee, n + 3, nb, nb), dtype=E0.dtype)
    phi = np.zeros_like(theta)
    psi = np.zeros_like(theta)
    mass = dtype(0) if static else 1 / (dtype(beta) * dtype(dt) * dtype(dt))
    x = xi[None, :, None, None]
    if dim not in (2, 3):
        raise ValueError("dim must be 2 or 3")
    D = (dim - 1) * E0 + _T(E1) - E1 + x * dE0
    theta[:, 1:n + 2] = x * x * E0 / (h * h) - x * D / (2 * h)
    phi[:, 1:n + 2] = -2 * x * x * E0 / (h * h) - E2 + x * _T(dE1) - mass * x * x * M0
    if dim == 3:
        phi[:, 1:n + 2] += _T(E1)
    psi[:, 1:n + 2] = x * x * E0 / (h * h) + x * D / (2 * h)
    theta[:, 0] = -xi[0] * E0[:, 0] / (2 * h)
    phi[:, 0] = _T(E1[:, 0])
    psi[:, 0] = xi[0] * E0[:, 0] / (2 * h)
    theta[:, n + 2] = -xi[n] * E0[:, n] / (2 * h)
    phi[:, n + 2] = _T(E1[:, n])
    psi[:, n + 2] = xi[n] * E0[:, n] / (2 * h)
    return ElementSystem(xi, h, theta, phi, psi, M0)


@dataclass
class Condensed:
    """Result of the algorithmic condensation (Section 3.3), index i+1 for row i."""
    rho: np.ndarray          # (E, n+3, n_b, n_b): varrho_0..varrho_n at 1..n+1, varrho_{n+1} at n+2
    phi_t: np.ndarray        # modified phi_i (rows 0..n+1)
    psi_t: np.ndarray        # modified psi_i (psi_0 changed by the first pivot)
    W: np.ndarray            # (E, n_b, n_b) psi_{n+1} psi_n^{-1}
    S: np.ndarray            # (E, n_b, n_b) dynamic stiffness phi_{n+1} - psi_{n+1} psi_n^{-1} phi_n
    phi_t_inv: np.ndarray    # (E, n, n_b, n_b) inverses of the modified phi_i, rows 0..n-1


def condense(sys_: ElementSystem) -> Condensed:
    """Gaussian elimination of Eq. (system) onto the boundary unknowns u_n (Section 3.3).

    1. varrho_0 = theta_0 theta_{-1}^{-1}; phi_0 -= varrho_0 phi_{-1}; psi_0 -= varrho_0 psi_{-1}.
    2. Thomas sweep, i = 1..n: varrho_i = theta_i phi_{i-1}^{-1}; phi_i -= varrho_i psi_{i-1}.
    3. varrho_{n+1} = theta_{n+1} phi_{n-1}^{-1}; phi_{n+1} -= varrho_{n+1} psi_{n-1}.
    4. S = phi_{n+1} - psi_{n+1} psi_n^{-1} phi_n.
    """
    th, ph, ps = sys_.theta, sys_.phi.copy(), sys_.psi.copy()
    n = sys_.xi.size - 1
    rho = np.zeros_like(th)
    inv = np.zeros_like(th[:, :n])
    # step 1: eliminate u_{-1} from row 0 with row -1
    rho[:, 1] = th[:, 1] @ inverse(th[:, 0])
    ph[:, 1] = ph[:, 1] - rho[:, 1] @ ph[:, 0]
    ps[:, 1] = ps[:, 1] - rho[:, 1] @ ps[:, 0]
    # step 2: Thomas sweep on rows 1..n
    for i in range(1, n + 1):
        inv[:, i - 1] = inverse(ph[:, i])
        rho[:, i + 1] = th[:, i + 1] @ inv[:, i - 1]
        ph[:, i + 1] = ph[:, i + 1] - rho[:, i + 1] @ ps[:, i]
    # step 3: last row (n+1) couples to u_{n-1}
    rho[:, n + 2] = th[:, n + 2] @ inv[:, n - 1]
    ph[:, n + 2] = ph[:, n + 2] - rho[:, n + 2] @ ps[:, n]
    # step 4: 2x2 block closure
    W = ps[:, n + 2] @ inverse(ps[:, n + 1])
    S = ph[:, n + 2] - W @ ph[:, n + 1]
    return Condensed(rho, ph, ps, W, S, inv)


# ----------------------------------------------------------------------------
# Per-step right-hand-side sweeps (FP64, batched over elements and shots)
# ----------------------------------------------------------------------------

def residual_source(xi, M0, pred):
    """p_i = -xi_i^2 M0_i (u_i/(beta dt^2) + u'_i/(beta dt) - (1 - 1/(2 beta)) u''_i), i = 0..n.

    Eq. (ODE_Newmark); ``pred`` is the bracket, shape (E, n+1, n_b, B).
    """
    x2 = (xi ** 2)[None, :, None, None]
    return -x2 * np.einsum("eiab,eibs->eias", M0, pred)


def forward_sweep(rho, W, p):
    """Forward elimination of the right-hand side and the effective source (Section 3.3).

    p_0 is unchanged (row -1 has a zero right-hand side), p_i -= varrho_i p_{i-1}
    for i = 1..n, p_{n+1} = -varrho_{n+1} p_{n-1} and
    f_hat = p_{n+1} - psi_{n+1} psi_n^{-1} p_n (the external f is added globally).
    ``p`` has shape (E, n+1, n_b, B); returns (p_tilde, f_hat (E, n_b, B)).
    """
    n = p.shape[1] - 1
    pt = p.copy()
    for i in range(1, n + 1):
        pt[:, i] -= np.einsum("eab,ebs->eas", rho[:, i + 1], pt[:, i - 1])
    p_np1 = -np.einsum("eab,ebs->eas", rho[:, n + 2], pt[:, n - 1])
    f_hat = p_np1 - np.einsum("eab,ebs->eas", W, pt[:, n])
    return pt, f_hat


def back_substitute(phi_t_inv, psi_t, pt, u_n):
    """u_i = phi_i^{-1} (p_i - psi_i u_{i+1}) for i = n-1..0 (Section 3.3), u_n given."""
    n = pt.shape[1] - 1
    u = np.empty_like(pt)
    u[:, n] = u_n
    for i in range(n - 1, -1, -1):
        rhs = pt[:, i] - np.einsum("eab,ebs->eas", psi_t[:, i + 1], u[:, i + 1])
        u[:, i] = np.einsum("eab,ebs->eas", phi_t_inv[:, i], rhs)
    return u
