"""The condensed path of ``oracle.fwi`` on meshes whose S-elements have different
numbers of boundary nodes (quadtree meshes with hanging vertices, polygons).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Nothing in Sections 2-4 ties the elements of a mesh to one boundary-node count:
every element is set up, condensed, swept and back-substituted on its own
(Section 3.3), and only the global boundary system couples them.  This module
takes the same steps as ``oracle.fwi`` with the elements grouped by n_b: each
group is stacked and run through the same ``oracle.sbfem`` routines, and the
groups meet only in the global right-hand side and the global matrix.  Nodal
points are numbered as in ``oracle.fwi``: interior points of every element in
element order (n * n_b(e) of them, i-major), then the global nodes.

Pinned by ``tests/test_oracle_uneven.py``: against ``FullSystem`` below (the
uncondensed element systems plus the flux balance, solved directly, as in
``oracle.bruteforce``) on a quadtree mesh with hanging vertices, and against
``oracle.fwi`` on a uniform mesh (traces, states and kernel).
"""

from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fwi
from . import sbfem


@dataclass
class Group:
    elems: np.ndarray          # (Eg,) element ids with this n_b
    nb: int
    dofs: np.ndarray           # (Eg, nb)
    M0: np.ndarray             # (Eg, n+1, nb, nb)
    rho_piv: np.ndarray        # (Eg, n+3, nb, nb)
    psi_t: np.ndarray
    phi_t_inv: np.ndarray      # (Eg, n, nb, nb)
    W: np.ndarray              # (Eg, nb, nb)
    S: np.ndarray              # (Eg, nb, nb)
    interior: np.ndarray       # (Eg, n, nb) nodal-point index of each interior point


@dataclass
class Model:
    mesh: object
    elements: list
    n: int
    xi: np.ndarray
    c: float
    dt: float
    beta: float
    gamma: float
    int_ptr: np.ndarray
    points: np.ndarray
    rho_nodal: np.ndarray
    groups: list
    A: object
    lu: object

    @property
    def n_int(self) -> int:
        return int(self.int_ptr[-1])

    @property
    def n_nodes(self) -> int:
        return int(self.mesh.n_nodes)


def _local_density(rho_nodal, int_ptr, n_int, n, el, e):
    nb = el.dofs.size
    r = np.empty((n + 1, nb), dtype=rho_nodal.dtype)
    r[:n] = rho_nodal[int_ptr[e]:int_ptr[e + 1]].reshape(n, nb)
    r[n] = rho_nodal[n_int + el.dofs]
    return r


def build_model(mesh, n_r, c, rho, dt, beta=0.25, gamma=0.5, xi0=1e-3, rho_kind="grid", lx=None, ly=None) -> Model:
    """Set-up of every element (coefficient matrices, blocks, condensation) and the
    assembled global boundary matrix, as ``oracle.fwi.build_model``, group by group."""
    XP = sbfem.XP
    n = n_r - 1
    if n < 2:
        raise ValueError("need at least 3 radial points")
    elements = sbfem.elements_from_mesh(mesh)
    xi = sbfem.radial_grid(n, xi0, XP)
    points, int_ptr = fwi.nodal_points(mesh, elements, xi)
    lx = mesh.lx if lx is None else lx
    ly = mesh.ly if ly is None else ly
    if rho_kind == "grid":
        rho_nodal = fwi.grid_to_points(np.asarray(rho, dtype=np.float64), points, lx, ly)
    elif rho_kind == "nodal":
        rho_nodal = np.asarray(rho).astype(XP)
        if rho_nodal.shape != (points.shape[0],):
            raise ValueError("nodal density has the wrong length")
    else:
        raise ValueError(rho_kind)
    if np.any(rho_nodal <= 0):
        raise ValueError("density must be positive")
    n_int = int(int_ptr[-1])
    f64 = lambda a: np.asarray(a, dtype=np.float64)
    nbs = np.array([el.dofs.size for el in elements])
    groups, rows, cols, vals = [], [], [], []
    for nb in np.unique(nbs):
        idx = np.nonzero(nbs == nb)[0]
        Es = [np.zeros((idx.size, n + 1, nb, nb), dtype=XP) for _ in range(4)]
        for k, e in enumerate(idx):
            el = elements[e]
            mats = sbfem.coefficient_matrices(el, mesh.node_xy, mesh.p, c,
                                              _local_density(rho_nodal, int_ptr, n_int, n, el, e))
            for q in range(4):
                Es[q][k] = mats[q]
        sys_ = sbfem.element_system(*Es, xi, dt, beta)
        cd = sbfem.condense(sys_)
        dofs = np.stack([elements[e].dofs for e in idx])
        interior = np.stack([int_ptr[e] + np.arange(n * nb).reshape(n, nb) for e in idx])
        S = f64(cd.S)
        rows.append(np.repeat(dofs, nb, axis=1).ravel())
        cols.append(np.tile(dofs, (1, nb)).ravel())
        vals.append(S.ravel())
        groups.append(Group(idx, int(nb), dofs, f64(sys_.M0), f64(cd.rho), f64(cd.psi_t), f64(cd.phi_t_inv),
                            f64(cd.W), S, interior))
    N = mesh.n_nodes
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N)).tocsc()
    return Model(mesh, elements, n, f64(xi), c, dt, beta, gamma, int_ptr, points, f64(rho_nodal), groups, A,
                 spla.splu(A))


@dataclass
class State:
    u: list            # per group (Eg, n, nb, B)
    ud: list
    udd: list
    ub: np.ndarray     # (N, B)
    udb: np.ndarray
    uddb: np.ndarray


def zero_state(model: Model, B: int) -> State:
    z = lambda g: np.zeros((g.elems.size, model.n, g.nb, B))
    return State([z(g) for g in model.groups], [z(g) for g in model.groups], [z(g) for g in model.groups],
                 np.zeros((model.n_nodes, B)), np.zeros((model.n_nodes, B)), np.zeros((model.n_nodes, B)))


def step(model: Model, st: State, f_ext: np.ndarray) -> State:
    """One Newmark step (Section 3.3): per group the residual sources, forward sweep and
    effective sources; the global boundary solve; per group the back-substitution;
    the Newmark update of every radial point."""
    dt, beta, gamma, n = model.dt, model.beta, model.gamma, model.n
    B = st.ub.shape[1]
    F = np.array(f_ext, dtype=np.float64, copy=True)
    sweeps = []
    for k, g in enumerate(model.groups):
        u = np.concatenate([st.u[k], st.ub[g.dofs][:, None]], axis=1)
        ud = np.concatenate([st.ud[k], st.udb[g.dofs][:, None]], axis=1)
        udd = np.concatenate([st.udd[k], st.uddb[g.dofs][:, None]], axis=1)
        p = sbfem.residual_source(model.xi, g.M0, fwi.newmark_predictor(u, ud, udd, dt, beta))
        pt, f_hat = sbfem.forward_sweep(g.rho_piv, g.W, p)
        np.add.at(F, g.dofs.ravel(), f_hat.reshape(-1, B))
        sweeps.append(pt)
    ub_new = model.lu.solve(F)
    if ub_new.ndim == 1:
        ub_new = ub_new[:, None]
    u_n, ud_n, udd_n = [], [], []
    for k, g in enumerate(model.groups):
        un = sbfem.back_substitute(g.phi_t_inv, g.psi_t, sweeps[k], ub_new[g.dofs])
        a, b = fwi.newmark_update(st.u[k], st.ud[k], st.udd[k], un[:, :n], dt, beta, gamma)
        u_n.append(un[:, :n].copy())
        ud_n.append(a)
        udd_n.append(b)
    ud_b, udd_b = fwi.newmark_update(st.ub, st.udb, st.uddb, ub_new, dt, beta, gamma)
    return State(u_n, ud_n, udd_n, ub_new, ud_b, udd_b)


def nodal_vector(model: Model, interior: list, boundary: np.ndarray) -> np.ndarray:
    """Per-group interior values and (N, B) boundary values as (n_nodal, B) in nodal order."""
    B = boundary.shape[1]
    out = np.empty((model.n_int + model.n_nodes, B))
    for k, g in enumerate(model.groups):
        out[g.interior.ravel()] = interior[k].reshape(-1, B)
    out[model.n_int:] = boundary
    return out


def forward(model: Model, src_nodes, wavelets, rec_nodes, K=None, keep=True, keep_u=False):
    """Traces (B, R, K), the nodal velocities after every step (if ``keep``) and the
    final state; the conventions of ``oracle.fwi.forward`` (``keep_u``: the nodal
    displacements of every step as a 4th result, for the full kernel)."""
    src_nodes = np.asarray(src_nodes)
    rec_nodes = np.asarray(rec_nodes)
    wavelets = np.atleast_2d(wavelets)
    B = src_nodes.size
    K = wavelets.shape[1] if K is None else K
    st = zero_state(model, B)
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


def adjoint_gradient(model: Model, store: np.ndarray, residual: np.ndarray, rec_nodes, store_u=None):
    """Time-reversed adjoint and zero-lag velocity correlation on the nodal points, the
    conventions of ``oracle.fwi.adjoint_gradient``; with ``store_u`` the full kernel's
    gradient term too (``oracle.fwi.gradient_operator``, which takes each element's own
    n_b)."""
    residual = np.asarray(residual)
    B, R, K = residual.shape
    st = zero_state(model, B)
    npt = model.n_int + model.n_nodes
    g = np.zeros(npt)
    G = fwi.gradient_operator(model) if store_u is not None else None
    for m in range(K):
        j = K - 1 - m
        f = np.zeros((model.n_nodes, B))
        for s in range(B):
            np.add.at(f[:, s], rec_nodes, residual[s, :, j])
        st = step(model, st, f)
        g += model.dt * np.sum(store[j] * nodal_vector(model, st.ud, st.udb), axis=1)
        if G is not None:
            gu = (G @ store_u[j]).reshape(npt, 2, B)
            gl = (G @ nodal_vector(model, st.u, st.ub)).reshape(npt, 2, B)
            g += model.dt * model.c ** 2 * np.sum(gu * gl, axis=(1, 2))
    return g


def gradient_to_grid(model: Model, g_nodal, gx, gy, lx=None, ly=None):
    lx = model.mesh.lx if lx is None else lx
    ly = model.mesh.ly if ly is None else ly
    return fwi.points_to_grid(g_nodal, model.points, gx, gy, lx, ly)


class FullSystem:
    """Every element's uncondensed rows -1..n of Eq. (system) (ghosts included) plus the
    per-node flux balance of the rows n+1, assembled for elements of any n_b and
    solved densely each step: the independent route of ``oracle.bruteforce`` for
    uneven meshes (tiny meshes only)."""

    def __init__(self, mesh, n_r, c, rho_nodal, dt, beta=0.25, gamma=0.5, xi0=1e-3):
        XP = sbfem.XP
        self.mesh, self.n = mesh, n_r - 1
        n = self.n
        self.elements = sbfem.elements_from_mesh(mesh)
        xi = sbfem.radial_grid(n, xi0, XP)
        self.xi = np.asarray(xi, dtype=np.float64)
        self.dt, self.beta, self.gamma = dt, beta, gamma
        _, int_ptr = fwi.nodal_points(mesh, self.elements, xi)
        n_int = int(int_ptr[-1])
        rho_nodal = np.asarray(rho_nodal).astype(XP)
        nbs = [el.dofs.size for el in self.elements]
        self.off = np.concatenate([[0], np.cumsum([(n + 2) * nb for nb in nbs])]).astype(np.int64)
        self.n_elem_unknowns = int(self.off[-1])
        self.size = self.n_elem_unknowns + mesh.n_nodes
        self.M0 = []
        R, C, V = [], [], []

        def add(ri, ci, M):
            rr, cc = np.meshgrid(ri, ci, indexing="ij")
            R.append(rr.ravel())
            C.append(cc.ravel())
            V.append(np.asarray(M).ravel())

        for e, el in enumerate(self.elements):
            mats = sbfem.coefficient_matrices(el, mesh.node_xy, mesh.p, c,
                                              _local_density(rho_nodal, int_ptr, n_int, n, el, e))
            sys_ = sbfem.element_system(*(m[None] for m in mats), xi, dt, beta)
            self.M0.append(np.asarray(sys_.M0[0], dtype=np.float64))
            th, ph, ps = sys_.theta[0], sys_.phi[0], sys_.psi[0]
            for i in range(-1, n + 2):
                ri = self.row_index(e, i)
                k0 = min(max(i, 0), n) - 1          # rows -1 and n+1 couple the unknowns of rows 0 and n
                for d, M in enumerate((th[i + 1], ph[i + 1], ps[i + 1])):
                    add(ri, self.col_block(e, k0 + d), M)
        self._coo = (np.concatenate(R), np.concatenate(C), np.concatenate(V))
        r, cidx, v = self._coo
        self.matrix = sp.coo_matrix((np.asarray(v, dtype=np.float64), (r, cidx)), shape=(self.size, self.size)).toarray()
        self._lu = sla.lu_factor(self.matrix)

    def solve(self, rhs):
        """A x = rhs: dense LU in float64, refined with residuals in extended precision
        (the rows next to the scaling centre make A ill-conditioned, ~1e7)."""
        r, c, v = self._coo
        x = sla.lu_solve(self._lu, rhs).astype(v.dtype)
        for _ in range(3):
            res = np.asarray(rhs).astype(v.dtype)
            np.subtract.at(res, r, v[:, None] * x[c])
            x = x + sla.lu_solve(self._lu, np.asarray(res, dtype=np.float64))
        return np.asarray(x, dtype=np.float64)

    def col_block(self, e, k):
        """Columns of u_k (k = -1..n+1) of element e; u_n is the global boundary field."""
        el, n = self.elements[e], self.n
        nb = el.dofs.size
        if k == n:
            return self.n_elem_unknowns + el.dofs
        blk = k + 1 if k < n else n + 1
        return self.off[e] + blk * nb + np.arange(nb)

    def row_index(self, e, i):
        """Rows of element e's equation i = -1..n, or its flux-balance rows (i = n+1)."""
        el, n = self.elements[e], self.n
        nb = el.dofs.size
        if i == n + 1:
            return self.n_elem_unknowns + el.dofs
        return self.off[e] + (i + 1) * nb + np.arange(nb)

    def forward(self, src_nodes, wavelets, rec_nodes, K=None):
        """Traces (B, R, K) and the final interior displacements (list per element)."""
        src_nodes = np.asarray(src_nodes)
        rec_nodes = np.asarray(rec_nodes)
        wavelets = np.atleast_2d(wavelets)
        B = src_nodes.size
        K = wavelets.shape[1] if K is None else K
        n, N = self.n, self.mesh.n_nodes
        dt, beta, gamma = self.dt, self.beta, self.gamma
        zi = lambda: [np.zeros((n, el.dofs.size, B)) for el in self.elements]
        u, ud, udd = zi(), zi(), zi()
        ub, udb, uddb = np.zeros((N, B)), np.zeros((N, B)), np.zeros((N, B))
        traces = np.zeros((B, rec_nodes.size, K))
        for k in range(K):
            rhs = np.zeros((self.size, B))
            for e, el in enumerate(self.elements):
                ue = np.concatenate([u[e], ub[el.dofs][None]], axis=0)
                ude = np.concatenate([ud[e], udb[el.dofs][None]], axis=0)
                udde = np.concatenate([udd[e], uddb[el.dofs][None]], axis=0)
                pred = fwi.newmark_predictor(ue, ude, udde, dt, beta)
                for i in range(n + 1):
                    rhs[self.row_index(e, i)] = -(self.xi[i] ** 2) * (self.M0[e][i] @ pred[i])
            for s in range(B):
                rhs[self.n_elem_unknowns + src_nodes[s], s] += wavelets[s, k]
            x = self.solve(rhs)
            for e in range(len(self.elements)):
                un = np.stack([x[self.col_block(e, i)] for i in range(n)])
                ud[e], udd_new = fwi.newmark_update(u[e], ud[e], udd[e], un, dt, beta, gamma)
                udd[e], u[e] = udd_new, un
            ub_new = x[self.n_elem_unknowns:]
            udb, uddb = fwi.newmark_update(ub, udb, uddb, ub_new, dt, beta, gamma)
            ub = ub_new
            traces[:, :, k] = ub[rec_nodes].T
        return traces, u
