"""Forward, misfit, adjoint and Frechet kernel of the paper's Sections 2-4 (FP64 numpy/scipy).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Conventions (the readings the paper leaves open are listed with each function):

* Nodal points: every element's interior radial points i = 0..n-1 of its n_b
  rays, then every global boundary node once (the boundary point i = n is shared
  by the elements meeting there).  Index of interior point (e, i, j) is
  ``int_ptr[e] + i*n_b(e) + j``; global node g is ``n_int + g``.
* Density parameters: either nodal (the paper's choice, Section 4) or a
  cell-centred fine grid mapped to the nodal points by bilinear interpolation
  with clamping at the edges (forward rho_nodal = P rho_grid, gradient
  g_grid = P^T g_nodal).
* Sources: a point source adds +f(t_{k+1}) to the global right-hand side at its
  node for the step k -> k+1 (the external source vector f of the boundary row
  at xi = 1, Section 3.3, added once per node).
* Time axis: zero initial state; step k (0-based) produces the state at
  t_{k+1}; trace sample k is u at t_{k+1}.
"""

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import sbfem


# ----------------------------------------------------------------------------
# Newmark (Eq. (Newmark))
# ----------------------------------------------------------------------------

def newmark_predictor(u, ud, udd, dt, beta):
    """Bracket of the residual source: u/(beta dt^2) + u'/(beta dt) - (1 - 1/(2 beta)) u''."""
    return u / (beta * dt * dt) + ud / (beta * dt) - (1.0 - 1.0 / (2.0 * beta)) * udd


def newmark_update(u, ud, udd, u_new, dt, beta, gamma):
    """Velocity and acceleration at t + dt from the new displacement, Eq. (Newmark)."""
    du = u_new - u
    udd_new = du / (beta * dt * dt) - ud / (beta * dt) + (1.0 - 1.0 / (2.0 * beta)) * udd
    ud_new = gamma / (beta * dt) * du + (1.0 - gamma / beta) * ud + dt * (1.0 - gamma / (2.0 * beta)) * udd
    return ud_new, udd_new


# ----------------------------------------------------------------------------
# Density map
# ----------------------------------------------------------------------------

def bilinear_weights(points, gx, gy, lx, ly):
    """Cells and weights of bilinear interpolation of a cell-centred grid at ``points``.

    Grid value (ix, iy) sits at ((ix+1/2) lx/gx, (iy+1/2) ly/gy).  Points outside the
    band of cell centres are clamped to the edge value.  Returns (idx (m, 4), w (m, 4))
    with flat indices iy*gx + ix into the (gy, gx) array; the weights are in the
    floating type of ``points`` (at least float64).
    """
    points = np.asarray(points)
    points = points.astype(np.result_type(points.dtype, np.float64))
    ft = points.dtype.type
    fx = points[:, 0] * ft(gx) / ft(lx) - ft(0.5)
    fy = points[:, 1] * ft(gy) / ft(ly) - ft(0.5)
    ix = np.floor(fx).astype(np.int64)
    iy = np.floor(fy).astype(np.int64)
    tx = fx - ix
    ty = fy - iy
    lo = ix < 0
    ix[lo], tx[lo] = 0, 0.0
    hi = ix > gx - 2
    ix[hi], tx[hi] = gx - 2, 1.0
    lo = iy < 0
    iy[lo], ty[lo] = 0, 0.0
    hi = iy > gy - 2
    iy[hi], ty[hi] = gy - 2, 1.0
    idx = np.stack([iy * gx + ix, iy * gx + ix + 1, (iy + 1) * gx + ix, (iy + 1) * gx + ix + 1], axis=1)
    w = np.stack([(1 - tx) * (1 - ty), tx * (1 - ty), (1 - tx) * ty, tx * ty], axis=1)
    return idx, w


def grid_to_points(rho_grid, points, lx, ly):
    gy, gx = rho_grid.shape
    idx, w = bilinear_weights(points, gx, gy, lx, ly)
    return np.sum(rho_grid.ravel()[idx].astype(w.dtype) * w, axis=1)


def points_to_grid(g_points, points, gx, gy, lx, ly):
    """Adjoint (transpose) of ``grid_to_points``, in float64."""
    idx, w = bilinear_weights(points, gx, gy, lx, ly)
    out = np.zeros(gx * gy)
    np.add.at(out, idx.ravel(), (w.astype(np.float64) * np.asarray(g_points, dtype=np.float64)[:, None]).ravel())
    return out.reshape(gy, gx)


# ----------------------------------------------------------------------------
# Model set-up
# ----------------------------------------------------------------------------

@dataclass
class Model:
    mesh: object
    elements: list
    n: int                     # radial intervals; N_r = n + 1 points
    xi: np.ndarray
    c: float
    dt: float
    beta: float
    gamma: float
    int_ptr: np.ndarray        # (E+1,) offsets of interior nodal points
    points: np.ndarray         # (n_nodal, 2) physical location of every nodal point
    rho_nodal: np.ndarray      # (n_nodal,)
    # stacked per-element data, all elements share (n_b, n) in this oracle
    dofs: np.ndarray           # (E, n_b)
    M0: np.ndarray             # (E, n+1, n_b, n_b)
    rho_piv: np.ndarray        # (E, n+3, n_b, n_b)  varrho at index i+1
    psi_t: np.ndarray          # (E, n+3, n_b, n_b)
    phi_t_inv: np.ndarray      # (E, n, n_b, n_b)
    W: np.ndarray              # (E, n_b, n_b)
    S: np.ndarray              # (E, n_b, n_b)
    A: object                  # global sparse matrix sum_e Z_e^T S_e Z_e
    lu: object

    @property
    def n_int(self) -> int:
        return int(self.int_ptr[-1])

    @property
    def n_nodes(self) -> int:
        return int(self.mesh.n_nodes)


def nodal_points(mesh, elements, xi):
    """Physical location of every nodal point: x0 + xi_i (x_j - x0), i < n; x_j for i = n."""
    n = xi.size - 1
    pts = []
    int_ptr = [0]
    for el in elements:
        xj = mesh.node_xy[el.dofs].astype(xi.dtype)                        # (n_b, 2)
        p_el = el.centre[None, None, :] + xi[:n, None, None] * (xj[None, :, :] - el.centre[None, None, :])
        pts.append(p_el.reshape(-1, 2))
        int_ptr.append(int_ptr[-1] + n * el.dofs.size)
    pts.append(mesh.node_xy.astype(xi.dtype))
    return np.concatenate(pts, axis=0), np.asarray(int_ptr, dtype=np.int64)


def build_model(mesh, n_r, c, rho, dt, beta=0.25, gamma=0.5, xi0=1e-3,
                rho_kind="grid", lx=None, ly=None, static=False, rho_mass_nodal=None) -> Model:
    """Set-up of the path (no time stepping): nodal densities, E-matrices, blocks,
    condensation of every element, and the assembled global boundary matrix.

    ``rho`` is a (gy, gx) grid (rho_kind='grid') or a vector over nodal points
    (rho_kind='nodal').  ``rho_mass_nodal`` (tests only) gives M0 its own nodal
    densities while E0, E1, E2 keep ``rho``: the density of the inertia term alone,
    which is what the velocity part of the Frechet kernel differentiates.

    The set-up runs in extended precision (``sbfem.XP``); the matrices the time
    loop uses are then rounded once to float64.
    """
    XP = sbfem.XP
    n = n_r - 1
    if n < 2:
        raise ValueError("need at least 3 radial points")
    elements = sbfem.elements_from_mesh(mesh)
    nb = elements[0].dofs.size
    if any(el.dofs.size != nb for el in elements):
        raise ValueError("this oracle expects one boundary-node count for all elements")
    xi = sbfem.radial_grid(n, xi0, XP)
    points, int_ptr = nodal_points(mesh, elements, xi)
    lx = mesh.lx if lx is None else lx
    ly = mesh.ly if ly is None else ly
    if rho_kind == "grid":
        rho_nodal = grid_to_points(np.asarray(rho, dtype=np.float64), points, lx, ly)
    elif rho_kind == "nodal":
        rho_nodal = np.asarray(rho).astype(XP)
        if rho_nodal.shape != (points.shape[0],):
            raise ValueError("nodal density has the wrong length")
    else:
        raise ValueError(rho_kind)
    if np.any(rho_nodal <= 0):
        raise ValueError("density must be positive")
    n_int = int(int_ptr[-1])
    E = len(elements)

    def local(rn, e, el):
        r = np.empty((n + 1, nb), dtype=XP)
        r[:n] = rn[int_ptr[e]:int_ptr[e + 1]].reshape(n, nb)
        r[n] = rn[n_int + el.dofs]
        return r

    Es = [np.zeros((E, n + 1, nb, nb), dtype=XP) for _ in range(4)]
    for e, el in enumerate(elements):
        mats = sbfem.coefficient_matrices(el, mesh.node_xy, mesh.p, c, local(rho_nodal, e, el))
        if rho_mass_nodal is not None:
            rm = local(np.asarray(rho_mass_nodal).astype(XP), e, el)
            mats = mats[:3] + (sbfem.coefficient_matrices(el, mesh.node_xy, mesh.p, c, rm)[3],)
        for k in range(4):
            Es[k][e] = mats[k]
    sys_ = sbfem.element_system(*Es, xi, dt, beta, static=static)
    cd = sbfem.condense(sys_)
    f64 = lambda a: np.asarray(a, dtype=np.float64)
    dofs = np.stack([el.dofs for el in elements])
    S = f64(cd.S)
    rr = np.repeat(dofs, nb, axis=1).ravel()
    cc = np.tile(dofs, (1, nb)).ravel()
    N = mesh.n_nodes
    A = sp.coo_matrix((S.ravel(), (rr, cc)), shape=(N, N)).tocsc()
    lu = spla.splu(A)
    return Model(mesh, elements, n, f64(xi), c, dt, beta, gamma, int_ptr, points, f64(rho_nodal),
                 dofs, f64(sys_.M0), f64(cd.rho), f64(cd.psi_t), f64(cd.phi_t_inv), f64(cd.W), S, A, lu)


# ----------------------------------------------------------------------------
# Time stepping
# ----------------------------------------------------------------------------

@dataclass
class State:
    u: np.ndarray      # (E, n, n_b, B) interior radial points
    ud: np.ndarray
    udd: np.ndarray
    ub: np.ndarray     # (N, B) global boundary nodes
    udb: np.ndarray
    uddb: np.ndarray


def zero_state(model: Model, B: int) -> State:
    E, nb = model.dofs.shape
    z = lambda *s: np.zeros(s)
    return State(z(E, model.n, nb, B), z(E, model.n, nb, B), z(E, model.n, nb, B),
                 z(model.n_nodes, B), z(model.n_nodes, B), z(model.n_nodes, B))


def step(model: Model, st: State, f_ext: np.ndarray) -> State:
    """One Newmark step of every element and the global boundary system (Section 3.3).

    Per element: residual sources p_i (Eq. (ODE_Newmark)), forward sweep and
    effective source f_hat; globally: F = sum_e Z_e^T f_hat_e + f_ext and
    (sum_e Z_e^T S_e Z_e) u_n = F; per element: back-substitution for the interior
    u_i; Newmark update (Eq. (Newmark)) of every radial point.
    """
    dt, beta, gamma = model.dt, model.beta, model.gamma
    n = model.n
    E, nb = model.dofs.shape
    B = st.ub.shape[1]
    # residual source at radial points 0..n (point n from the shared boundary state)
    u = np.concatenate([st.u, st.ub[model.dofs][:, None]], axis=1)          # (E, n+1, nb, B)
    ud = np.concatenate([st.ud, st.udb[model.dofs][:, None]], axis=1)
    udd = np.concatenate([st.udd, st.uddb[model.dofs][:, None]], axis=1)
    p = sbfem.residual_source(model.xi, model.M0, newmark_predictor(u, ud, udd, dt, beta))
    pt, f_hat = sbfem.forward_sweep(model.rho_piv, model.W, p)
    # global assembly of the right-hand side and the boundary solve
    F = np.zeros((model.n_nodes, B))
    np.add.at(F, model.dofs.ravel(), f_hat.reshape(E * nb, B))
    F += f_ext
    ub_new = model.lu.solve(F)
    if ub_new.ndim == 1:
        ub_new = ub_new[:, None]
    un = sbfem.back_substitute(model.phi_t_inv, model.psi_t, pt, ub_new[model.dofs])
    ud_i, udd_i = newmark_update(st.u, st.ud, st.udd, un[:, :n], dt, beta, gamma)
    ud_b, udd_b = newmark_update(st.ub, st.udb, st.uddb, ub_new, dt, beta, gamma)
    return State(un[:, :n].copy(), ud_i, udd_i, ub_new, ud_b, udd_b)


def nodal_vector(model: Model, interior: np.ndarray, boundary: np.ndarray) -> np.ndarray:
    """Flatten (E, n, n_b, B) interior + (N, B) boundary values to (n_nodal, B)."""
    B = boundary.shape[1]
    return np.concatenate([interior.reshape(-1, B), boundary], axis=0)


def forward(model: Model, src_nodes, wavelets, rec_nodes, K=None, keep=True, state=None, keep_u=False):
    """Forward solve of B shots (Section 2, Eq. (main)); shot s has one point source.

    Returns traces (B, R, K) with sample k = u(t_{k+1}) at the receivers and, if
    ``keep``, the nodal velocities (K, n_nodal, B) after every step (stored for the
    adjoint, the memory strategy of Section 4).  With ``keep_u`` the nodal
    displacements of every step are returned as well (a 4th result), for the gradient
    term of the full Frechet kernel (``adjoint_gradient(..., store_u=...)``).
    """
    src_nodes = np.asarray(src_nodes)
    rec_nodes = np.asarray(rec_nodes)
    wavelets = np.atleast_2d(wavelets)
    B = src_nodes.size
    K = wavelets.shape[1] if K is None else K
    st = zero_state(model, B) if state is None else state
    traces = np.zeros((B, rec_nodes.size, K))
    store = np.zeros((K, model.n_int + model.n_nodes, B)) if keep else None
    store_u = np.zeros((K, model.n_int + model.n_nodes, B)) if keep_u else None
    for k in range(K):
        f = np.zeros((model.n_nodes, B))
        for s in range(B):
            f[src_nodes[s], s] += wavelets[s, k]
        st = step(model, st, f)
        traces[:, :, k] = st.ub[rec_nodes].T
        if keep:
            store[k] = nodal_vector(model, st.ud, st.udb)
        if keep_u:
            store_u[k] = nodal_vector(model, st.u, st.ub)
    if keep_u:
        return traces, store, st, store_u
    return traces, store, st


def misfit(traces, observed, dt):
    """E = 1/2 sum_r int (d - u)^2 dt with the rectangle rule on the trace samples (Eq. (misfit)).

    Returns (E, residual d - u)."""
    res = np.asarray(observed, dtype=np.float64) - np.asarray(traces, dtype=np.float64)
    return 0.5 * dt * float(np.sum(res * res)), res


def gradient_operator(model: Model):
    """Sparse G: (G u)[2q + d] is component d (x, y) of grad u at nodal point q, from nodal
    values u (the full Frechet kernel's c^2 grad(lambda).grad(u) term, Section 2).

    Readings (the paper gives no discretisation of the term it drops): at radial point
    xi_i of node j on one of the element's line elements, [u_xi; u_eta] = J [u_x; u_y]
    with J = [[x_b - x0, y_b - y0], [xi x_b,eta, xi y_b,eta]] (the coordinate map x = x0 +
    xi (x_b(eta) - x0), Section 3); u_xi by second-order finite differences on the radial
    grid (central inside, one-sided at xi_0 and xi_n = 1), u_eta by the derivative of the
    line's Lagrange interpolant at the node.  A point met by several (element, line)
    pairs -- a vertex node, or a boundary node shared by elements -- gets the mean of their
    gradients."""
    import scipy.sparse as sp_
    mesh, n, xi = model.mesh, model.n, model.xi
    h = float(xi[1] - xi[0])
    p = mesh.p
    _, dphi = sbfem.lagrange(p, sbfem.lagrange_nodes(p))
    n_int = model.n_int
    rows, cols, vals = [], [], []
    count = np.zeros(n_int + model.n_nodes)
    for e, el in enumerate(model.elements):
        nb = el.dofs.size
        idx = lambda i, j: model.int_ptr[e] + i * nb + j if i < n else n_int + el.dofs[j]
        x0 = el.centre
        for ln, loc in zip(el.lines, el.line_local):
            X = mesh.node_xy[ln]
            dX = dphi @ X
            for i in range(n + 1):
                if i == 0:
                    st = ((0, -3.0), (1, 4.0), (2, -1.0))
                elif i == n:
                    st = ((n, 3.0), (n - 1, -4.0), (n - 2, 1.0))
                else:
                    st = ((i + 1, 1.0), (i - 1, -1.0))
                for k in range(p + 1):
                    j = int(loc[k])
                    Jinv = np.linalg.inv(np.array([X[k] - x0, xi[i] * dX[k]]))
                    q = idx(i, j)
                    for d in range(2):
                        for ii, wgt in st:
                            rows.append(2 * q + d); cols.append(idx(ii, j)); vals.append(Jinv[d, 0] * wgt / (2 * h))
                        for mm in range(p + 1):
                            rows.append(2 * q + d); cols.append(idx(i, int(loc[mm]))); vals.append(Jinv[d, 1] * dphi[k, mm])
                    count[q] += 1
    rows = np.asarray(rows)
    vals = np.asarray(vals) / np.repeat(count, 2)[rows]
    npt = n_int + model.n_nodes
    return sp_.csr_matrix((vals, (rows, np.asarray(cols))), shape=(2 * npt, npt))


def adjoint_gradient(model: Model, store: np.ndarray, residual: np.ndarray, rec_nodes, store_u=None):
    """Adjoint solve in reversed time and zero-lag cross-correlation (Sections 2 and 4).

    The adjoint field lambda(T - t) is the forward operator run from a zero state
    with the residuals d - u injected at the receivers, last sample first:
    adjoint step m (0-based) uses residual sample j = K-1-m as its source.  The
    Frechet kernel keeps only the velocity term (the paper drops the
    c^2 grad(lambda).grad(u) term and uses the nodal solution fields directly):

        g_node = dt * sum_m sum_shots  udot_fwd[j = K-1-m](node) * lambdadot^{m+1}(node)

    With the forward written as M u'' + K u = f (the sign of the boundary source
    row) and the adjoint driven by +(d - u), this is +dE/drho of the mass term
    (reading of the sign of the reversed-time kernel).  Returns g on nodal points
    (n_nodal,).  Parity of this kernel against the paper is unpinned (the paper
    prints no values); its parts are pinned through the forward solver.

    With ``store_u`` (the forward displacements of every step, ``forward(...,
    keep_u=True)``) the gradient term the paper drops is added: the same reversed-time
    pairing of c^2 grad(u_fwd) . grad(lambda) (``gradient_operator``).  In reversed time
    the velocity term changes sign and the gradient term does not, so relative to the
    velocity term as computed here it enters with a plus sign (Section 2's kernel
    d_t lambda d_t u - c^2 grad lambda . grad u, with d_t lambda = -d lambda / d tau).
    """
    residual = np.asarray(residual)
    B, R, K = residual.shape
    st = zero_state(model, B)
    g = np.zeros(model.n_int + model.n_nodes)
    G = gradient_operator(model) if store_u is not None else None
    npt = model.n_int + model.n_nodes
    for m in range(K):
        j = K - 1 - m
        f = np.zeros((model.n_nodes, B))
        for s in range(B):
            np.add.at(f[:, s], rec_nodes, residual[s, :, j])
        st = step(model, st, f)
        lam_dot = nodal_vector(model, st.ud, st.udb)
        g += model.dt * np.sum(store[j] * lam_dot, axis=1)
        if G is not None:
            gu = (G @ store_u[j]).reshape(npt, 2, B)
            gl = (G @ nodal_vector(model, st.u, st.ub)).reshape(npt, 2, B)
            g += model.dt * model.c ** 2 * np.sum(gu * gl, axis=(1, 2))
    return g


def gradient_to_grid(model: Model, g_nodal, gx, gy, lx=None, ly=None):
    lx = model.mesh.lx if lx is None else lx
    ly = model.mesh.ly if ly is None else ly
    return points_to_grid(g_nodal, model.points, gx, gy, lx, ly)


# ----------------------------------------------------------------------------
# Three-dimensional meshes (``oracle.sbfem3d``)
# ----------------------------------------------------------------------------

def trilinear_weights(points, gx, gy, gz, lx, ly, lz):
    """Cells and weights of trilinear interpolation of a cell-centred grid rho[gz, gy, gx]
    (value (ix, iy, iz) at ((ix+1/2) lx/gx, (iy+1/2) ly/gy, (iz+1/2) lz/gz)), clamped at
    the edges like ``bilinear_weights``.  Returns (idx (m, 8), w (m, 8)), flat indices
    (iz gy + iy) gx + ix, corner c = cx + 2 cy + 4 cz."""
    points = np.asarray(points)
    points = points.astype(np.result_type(points.dtype, np.float64))
    ft = points.dtype.type
    ii, tt = [], []
    for d, (g, L) in enumerate(((gx, lx), (gy, ly), (gz, lz))):
        f = points[:, d] * ft(g) / ft(L) - ft(0.5)
        i = np.floor(f).astype(np.int64)
        t = f - i
        lo = i < 0
        i[lo], t[lo] = 0, 0.0
        hi = i > g - 2
        i[hi], t[hi] = g - 2, 1.0
        ii.append(i)
        tt.append(t)
    idx, w = [], []
    for cz in range(2):
        for cy in range(2):
            for cx in range(2):
                idx.append(((ii[2] + cz) * gy + ii[1] + cy) * gx + ii[0] + cx)
                w.append((tt[0] if cx else 1 - tt[0]) * (tt[1] if cy else 1 - tt[1]) * (tt[2] if cz else 1 - tt[2]))
    return np.stack(idx, axis=1), np.stack(w, axis=1)


def grid_to_points3d(rho_grid, points, lx, ly, lz):
    gz, gy, gx = rho_grid.shape
    idx, w = trilinear_weights(points, gx, gy, gz, lx, ly, lz)
    return np.sum(rho_grid.ravel()[idx].astype(w.dtype) * w, axis=1)


def points_to_grid3d(g_points, points, gx, gy, gz, lx, ly, lz):
    """Adjoint (transpose) of ``grid_to_points3d``, in float64."""
    idx, w = trilinear_weights(points, gx, gy, gz, lx, ly, lz)
    out = np.zeros(gx * gy * gz)
    np.add.at(out, idx.ravel(), (w.astype(np.float64) * np.asarray(g_points, dtype=np.float64)[:, None]).ravel())
    return out.reshape(gz, gy, gx)


def build_model3d(mesh, n_r, c, rho, dt, beta=0.25, gamma=0.5, xi0=1e-3, rho_kind="grid", static=False,
                  rho_mass_nodal=None) -> Model:
    """``build_model`` for a mesh of 3-D S-elements (``sbfwi_inputs.mesh3d``): nodal
    densities (trilinear map of a rho[gz, gy, gx] grid, or nodal), the 3-D coefficient
    matrices, the blocks of the 3-D radial equation, condensation and the global matrix.
    The time loop, misfit and velocity-kernel adjoint of this module apply unchanged.
    ``rho_mass_nodal`` (tests only) gives M0 its own nodal densities, as in ``build_model``."""
    from . import sbfem3d
    XP = sbfem.XP
    n = n_r - 1
    if n < 2:
        raise ValueError("need at least 3 radial points")
    elements = sbfem3d.elements_from_mesh3d(mesh)
    nb = elements[0].dofs.size
    if any(el.dofs.size != nb for el in elements):
        raise ValueError("this oracle expects one boundary-node count for all elements")
    xi = sbfem.radial_grid(n, xi0, XP)
    points, int_ptr = sbfem3d.nodal_points3d(mesh, elements, xi)
    if rho_kind == "grid":
        rho_nodal = grid_to_points3d(np.asarray(rho, dtype=np.float64), points, mesh.lx, mesh.ly, mesh.lz)
    elif rho_kind == "nodal":
        rho_nodal = np.asarray(rho).astype(XP)
        if rho_nodal.shape != (points.shape[0],):
            raise ValueError("nodal density has the wrong length")
    else:
        raise ValueError(rho_kind)
    if np.any(rho_nodal <= 0):
        raise ValueError("density must be positive")
    n_int = int(int_ptr[-1])
    E = len(elements)
    Es = [np.zeros((E, n + 1, nb, nb), dtype=XP) for _ in range(4)]
    def local(rn, e, el):
        r = np.empty((n + 1, nb), dtype=XP)
        r[:n] = rn[int_ptr[e]:int_ptr[e + 1]].reshape(n, nb)
        r[n] = rn[n_int + el.dofs]
        return r

    for e, el in enumerate(elements):
        mats = sbfem3d.coefficient_matrices3d(el, mesh.node_xyz, mesh.p, c, local(rho_nodal, e, el))
        if rho_mass_nodal is not None:
            rm = local(np.asarray(rho_mass_nodal).astype(XP), e, el)
            mats = mats[:3] + (sbfem3d.coefficient_matrices3d(el, mesh.node_xyz, mesh.p, c, rm)[3],)
        for k in range(4):
            Es[k][e] = mats[k]
    sys_ = sbfem.element_system(*Es, xi, dt, beta, static=static, dim=3)
    cd = sbfem.condense(sys_)
    f64 = lambda a: np.asarray(a, dtype=np.float64)
    dofs = np.stack([el.dofs for el in elements])
    S = f64(cd.S)
    rr = np.repeat(dofs, nb, axis=1).ravel()
    cc = np.tile(dofs, (1, nb)).ravel()
    N = mesh.n_nodes
    A = sp.coo_matrix((S.ravel(), (rr, cc)), shape=(N, N)).tocsc()
    lu = spla.splu(A)
    return Model(mesh, elements, n, f64(xi), c, dt, beta, gamma, int_ptr, f64(points), f64(rho_nodal),
                 dofs, f64(sys_.M0), f64(cd.rho), f64(cd.psi_t), f64(cd.phi_t_inv), f64(cd.W), S, A, lu)


def gradient_to_grid3d(model: Model, g_nodal, gx, gy, gz):
    m = model.mesh
    return points_to_grid3d(g_nodal, model.points, gx, gy, gz, m.lx, m.ly, m.lz)
