"""The uncondensed system of Eq. (system), assembled for the whole mesh and solved directly.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Unknowns: for every element its ghost u_{-1}, interior u_0..u_{n-1} and ghost
u_{n+1} (n_b values each), and the global boundary field (one value per node,
the shared u_n).  Equations: every element's rows i = -1..n of Eq. (system) and,
per global node, the sum over the elements meeting there of their row n+1
(the internal source vector at xi = 1) equated to the external source (flux
balance of the assembled boundary).  No condensation is performed, so solving
this system each step is an independent route to the solution of the condensed
algorithm in ``oracle.fwi``; it is small enough only for tiny meshes.

The same assembly without the Newmark mass term, with the mass rows
xi_i^2 M0_i collected separately, is the pencil (Omega, M) of the semi-discrete
radial ODE (Eq. (ODE)): Omega x = -omega^2 M x gives its free-vibration
frequencies.
"""

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import sbfem
from . import fwi


class FullSystem:
    def __init__(self, mesh, n_r, c, rho_nodal, dt, beta=0.25, gamma=0.5, xi0=1e-3, static=False):
        self.mesh = mesh
        self.n = n = n_r - 1
        dim = getattr(mesh, "dim", 2)        # 3: hexahedral S-elements (oracle.sbfem3d)
        if dim == 3:
            from . import sbfem3d
            self.elements = sbfem3d.elements_from_mesh3d(mesh)
            coefficients = lambda el, r: sbfem3d.coefficient_matrices3d(el, mesh.node_xyz, mesh.p, c, r)
        else:
            self.elements = sbfem.elements_from_mesh(mesh)
            coefficients = lambda el, r: sbfem.coefficient_matrices(el, mesh.node_xy, mesh.p, c, r)
        self.nb = nb = self.elements[0].dofs.size
        xi = sbfem.radial_grid(n, xi0, sbfem.XP)
        self.xi = np.asarray(xi, dtype=np.float64)
        self.dt, self.beta, self.gamma = dt, beta, gamma
        if dim == 3:
            pts, int_ptr = sbfem3d.nodal_points3d(mesh, self.elements, xi)
        else:
            pts, int_ptr = fwi.nodal_points(mesh, self.elements, xi)
        self.int_ptr = int_ptr
        n_int = int(int_ptr[-1])
        E = len(self.elements)
        self.E = E
        self.n_elem_unknowns = E * (n + 2) * nb
        self.size = self.n_elem_unknowns + mesh.n_nodes
        rows, cols, vals = [], [], []
        mrows, mcols, mvals = [], [], []
        rho_nodal = np.asarray(rho_nodal).astype(sbfem.XP)
        self.rho_nodal = rho_nodal
        Es = [np.zeros((E, n + 1, nb, nb), dtype=sbfem.XP) for _ in range(4)]
        for e, el in enumerate(self.elements):
            r = np.empty((n + 1, nb), dtype=sbfem.XP)
            r[:n] = rho_nodal[int_ptr[e]:int_ptr[e + 1]].reshape(n, nb)
            r[n] = rho_nodal[n_int + el.dofs]
            mats = coefficients(el, r)
            for k in range(4):
                Es[k][e] = mats[k]
        sysall = sbfem.element_system(*Es, xi, dt, beta, static=static, dim=dim)
        # blocks are kept in extended precision; float64 copies feed the factorisation
        self.theta, self.phi, self.psi, self.M0 = sysall.theta, sysall.phi, sysall.psi, sysall.M0
        self.M0_64 = np.asarray(sysall.M0, dtype=np.float64)

        def col_block(e, k):
            """Column indices of u_k (k = -1..n+1) of element e."""
            el = self.elements[e]
            if k == n:
                return self.n_elem_unknowns + el.dofs
            blk = k + 1 if k < n else n + 1          # u_{-1}->0, u_i->i+1, u_{n+1}->n+1
            return e * (n + 2) * nb + blk * nb + np.arange(nb)

        def add(r_idx, c_idx, M, R, C, V):
            rr, cc = np.meshgrid(r_idx, c_idx, indexing="ij")
            R.append(rr.ravel())
            C.append(cc.ravel())
            V.append(M.ravel())

        self.col_block = col_block
        for e, el in enumerate(self.elements):
            th, ph, ps, M0 = self.theta[e], self.phi[e], self.psi[e], self.M0[e]
            for i in range(-1, n + 1):               # element rows -1..n
                ridx = e * (n + 2) * nb + (i + 1) * nb + np.arange(nb)
                if i == -1:
                    add(ridx, col_block(e, -1), th[0], rows, cols, vals)
                    add(ridx, col_block(e, 0), ph[0], rows, cols, vals)
                    add(ridx, col_block(e, 1), ps[0], rows, cols, vals)
                else:
                    add(ridx, col_block(e, i - 1), th[i + 1], rows, cols, vals)
                    add(ridx, col_block(e, i), ph[i + 1], rows, cols, vals)
                    add(ridx, col_block(e, i + 1), ps[i + 1], rows, cols, vals)
                    add(ridx, col_block(e, i), self.xi[i] ** 2 * M0[i], mrows, mcols, mvals)
            ridx = self.n_elem_unknowns + el.dofs     # row n+1 -> flux balance rows
            add(ridx, col_block(e, n - 1), th[n + 2], rows, cols, vals)
            add(ridx, col_block(e, n), ph[n + 2], rows, cols, vals)
            add(ridx, col_block(e, n + 1), ps[n + 2], rows, cols, vals)
        cat = np.concatenate
        self._coo = (cat(rows), cat(cols), cat(vals))
        self._mcoo = (cat(mrows), cat(mcols), cat(mvals))
        f64 = lambda a: np.asarray(a, dtype=np.float64)
        self.matrix = sp.coo_matrix((f64(cat(vals)), (cat(rows), cat(cols))), shape=(self.size, self.size)).tocsc()
        self.mass = sp.coo_matrix((f64(cat(mvals)), (cat(mrows), cat(mcols))), shape=(self.size, self.size)).tocsc()

    def _matvec_xp(self, x, mass=False, transpose=False):
        """Extended-precision product of the assembled (uncondensed) matrix, or of the
        mass pencil matrix, or of its transpose, with x (shape (size,) or (size, B))."""
        r, c, v = self._mcoo if mass else self._coo
        if transpose:
            r, c = c, r
        x = np.asarray(x)
        out = np.zeros((self.size,) + x.shape[1:], dtype=v.dtype)
        vv = v.reshape((-1,) + (1,) * (x.ndim - 1))
        np.add.at(out, r, vv * x[c].astype(v.dtype))
        return out

    # -- time stepping with a direct solve of the whole system each step --------

    def solve(self, rhs, transpose=False):
        """x with A x = rhs (or A^T x = rhs): dense LU in float64 (condition number ~1e7
        from the xi0 = 1e-3 rows), then iterative refinement with residuals in extended
        precision."""
        if not hasattr(self, "_lu"):
            self._lu = sla.lu_factor(self.matrix.toarray())
        tr = 1 if transpose else 0
        x = sla.lu_solve(self._lu, rhs, trans=tr).astype(sbfem.XP)
        for _ in range(3):
            res = np.asarray(rhs).astype(sbfem.XP) - self._matvec_xp(x, transpose=transpose)
            x = x + sla.lu_solve(self._lu, np.asarray(res, dtype=np.float64), trans=tr)
        return np.asarray(x, dtype=np.float64)

    def row_index(self, e, i):
        """Rows of element e's equation i = -1..n (element rows) or n+1 (flux rows)."""
        nb, n = self.nb, self.n
        if i == n + 1:
            return self.n_elem_unknowns + self.elements[e].dofs
        return e * (n + 2) * nb + (i + 1) * nb + np.arange(nb)

    def step(self, st: fwi.State, f_ext: np.ndarray) -> fwi.State:
        return self.step_full(st, f_ext)[2]

    def step_full(self, st: fwi.State, f_ext: np.ndarray):
        """One Newmark step of the whole uncondensed system; returns (x, predictor
        (E, n+1, n_b, B) at radial points 0..n, new state)."""
        n, nb, E = self.n, self.nb, self.E
        B = st.ub.shape[1]
        rhs = np.zeros((self.size, B))
        dofs = np.stack([el.dofs for el in self.elements])
        u = np.concatenate([st.u, st.ub[dofs][:, None]], axis=1)
        ud = np.concatenate([st.ud, st.udb[dofs][:, None]], axis=1)
        udd = np.concatenate([st.udd, st.uddb[dofs][:, None]], axis=1)
        pred = fwi.newmark_predictor(u, ud, udd, self.dt, self.beta)
        pall = sbfem.residual_source(self.xi, self.M0_64, pred)
        for e in range(E):
            p = pall[e]
            for i in range(n + 1):
                rhs[self.row_index(e, i)] = p[i]
        rhs[self.n_elem_unknowns:] += f_ext
        x = self.solve(rhs)
        u_int = np.empty((E, n, nb, B))
        for e in range(E):
            for i in range(n):
                u_int[e, i] = x[self.col_block(e, i)]
        ub = x[self.n_elem_unknowns:]
        ud_i, udd_i = fwi.newmark_update(st.u, st.ud, st.udd, u_int, self.dt, self.beta, self.gamma)
        ud_b, udd_b = fwi.newmark_update(st.ub, st.udb, st.uddb, ub, self.dt, self.beta, self.gamma)
        return x, pred, fwi.State(u_int, ud_i, udd_i, ub, ud_b, udd_b)

    def forward(self, src_nodes, wavelets, rec_nodes, K=None):
        src_nodes = np.asarray(src_nodes)
        wavelets = np.atleast_2d(wavelets)
        B = src_nodes.size
        K = wavelets.shape[1] if K is None else K
        nb, n, E = self.nb, self.n, self.E
        z = lambda *s: np.zeros(s)
        st = fwi.State(z(E, n, nb, B), z(E, n, nb, B), z(E, n, nb, B),
                       z(self.mesh.n_nodes, B), z(self.mesh.n_nodes, B), z(self.mesh.n_nodes, B))
        traces = np.zeros((B, len(rec_nodes), K))
        for k in range(K):
            f = np.zeros((self.mesh.n_nodes, B))
            for s in range(B):
                f[src_nodes[s], s] += wavelets[s, k]
            st = self.step(st, f)
            traces[:, :, k] = st.ub[np.asarray(rec_nodes)].T
        return traces, st

    def forward_pencil(self, src_nodes, wavelets, rec_nodes, K=None, transpose=False):
        """The same time loop written for the assembled pencil: with M the assembled mass
        rows (xi_i^2 M0_i at element row i, unknown u_i) and A the assembled matrix, every
        step solves A x = -M (a0 u + a1 u' + a2 u'') + f and updates u, u', u'' of every
        entry by Eq. (Newmark).  ``transpose=True`` runs the transposed pencil (A^T, M^T),
        whose state lives on the equations' index set; sources act on the flux rows and
        receivers read the boundary unknowns of the same global node numbers."""
        src_nodes = np.asarray(src_nodes)
        rec_nodes = np.asarray(rec_nodes)
        wavelets = np.atleast_2d(wavelets)
        B = src_nodes.size
        K = wavelets.shape[1] if K is None else K
        M = self.mass.T.tocsc() if transpose else self.mass
        u, ud, udd = (np.zeros((self.size, B)) for _ in range(3))
        traces = np.zeros((B, len(rec_nodes), K))
        for k in range(K):
            rhs = -(M @ fwi.newmark_predictor(u, ud, udd, self.dt, self.beta))
            for s in range(B):
                rhs[self.n_elem_unknowns + src_nodes[s], s] += wavelets[s, k]
            x = self.solve(rhs, transpose=transpose)
            ud, udd = fwi.newmark_update(u, ud, udd, x, self.dt, self.beta, self.gamma)
            u = x
            traces[:, :, k] = x[self.n_elem_unknowns + rec_nodes].T
        return traces

    # -- free vibration ---------------------------------------------------------

    def refine_mode(self, x, omega2, iters=4):
        """Newton refinement of an eigenpair of Omega x = -omega^2 M x (static system).

        Bordered system [[Omega + omega^2 M, M x], [e_k^T, 0]] [dx; dw] = -[r; 0] with
        the residual r in extended precision and x normalised to 1 at its largest entry.
        """
        x = np.asarray(x, dtype=np.float64)
        k = int(np.argmax(np.abs(x)))
        x = (x / x[k]).astype(sbfem.XP)
        w2 = sbfem.XP(omega2)
        Om = self.matrix.toarray()
        Ms = self.mass.toarray()
        for _ in range(iters):
            Mx = self._matvec_xp(x, mass=True)
            r = self._matvec_xp(x) + w2 * Mx
            J = np.zeros((self.size + 1, self.size + 1))
            J[:-1, :-1] = Om + float(w2) * Ms
            J[:-1, -1] = np.asarray(Mx, dtype=np.float64)
            J[-1, k] = 1.0
            d = np.linalg.solve(J, -np.concatenate([np.asarray(r, dtype=np.float64), [0.0]]))
            x = x + d[:-1]
            w2 = w2 + d[-1]
        return np.asarray(x, dtype=np.float64), float(w2)

    def frequencies(self, count=8, sigma=-1e-3):
        """Smallest ``count`` omega of Omega x = -omega^2 M x (system built with static=True).

        Uses shift-invert Arnoldi around -omega^2 = sigma; returns sorted omega (real parts).
        """
        vals = spla.eigs(self.matrix, k=count, M=self.mass, sigma=sigma, which="LM",
                         return_eigenvectors=False)
        w2 = np.sort(-vals.real)
        return np.sqrt(np.maximum(w2, 0.0)), vals
