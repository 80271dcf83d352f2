"""Exact derivative of the discrete misfit with respect to the nodal densities ("Mode X").

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper's gradient (Section 2, Section 4) is the continuous adjoint: the forward
operator run backwards in time with the residuals as sources, correlated with the
forward velocity ("Mode K", ``oracle.fwi.adjoint_gradient``).  The radial finite-
difference operator is not symmetric, so that kernel is not the exact derivative of
the discrete misfit.  This module computes the exact derivative by reverse-mode
differentiation of the discrete time loop, written out step by step on the
uncondensed system of ``oracle.bruteforce`` (which solves the same discrete problem
as the condensed path without eliminating anything):

  forward step k:   A(rho) x_{k+1} = r_k,   r_k = [-xi_i^2 M0_i(rho) v_{k,i}] + f_k,
                    v_k = Newmark predictor of the state s_k (Eq. (ODE_Newmark)),
                    u_{k+1} = the radial points 0..n-1 and boundary nodes of x_{k+1},
                    u', u'' at k+1 by Eq. (Newmark), traces d_k = u_{k+1} at receivers;
  misfit:           E = 1/2 dt sum_k |d_obs,k - d_k|^2 (Eq. (misfit)).

Both A and M0 are linear in the nodal densities (the E-matrices of Eq. (Es) are
linear in rho_j(xi_i); the blocks of Eq. (system) are linear combinations of them),
so with mu_k = A^{-T} xbar_k the adjoint of x_{k+1},

  dE/drho_q = sum_k [ -mu_k^T (dA/drho_q) x_{k+1} - xi_i^2 mu_{k,(e,i)}^T (dM0_i/drho_q) v_{k,i} ],

where dA/drho_q and dM0/drho_q are the element blocks assembled with the unit
density at parameter q (exact, by linearity).  The outer products mu x^T and mu v^T
are accumulated per element over time, then contracted once per parameter.

Pinned by ``tests/test_oracle_gradient.py``: central finite differences of the same
discrete misfit along random directions agree to ~1e-7 relative.
"""

import numpy as np

from . import bruteforce
from . import fwi
from . import sbfem


def _element_block_matrix(fs, theta, phi, psi):
    """Dense matrix of one element's rows -1..n+1 against its unknowns u_{-1}..u_{n+1}
    (local row (i+1) n_b + a, local column (k+1) n_b + b)."""
    n, nb = fs.n, fs.nb
    m = (n + 3) * nb
    A = np.zeros((m, m), dtype=theta.dtype)
    for i in range(-1, n + 2):
        r = slice((i + 1) * nb, (i + 2) * nb)
        # row i = 0..n couples u_{i-1}, u_i, u_{i+1}; the boundary-condition rows -1 and
        # n+1 couple the same unknowns as rows 0 and n
        k0 = min(max(i, 0), n) - 1
        blk = i + 1
        for d, M in enumerate((theta[blk], phi[blk], psi[blk])):
            k = k0 + d
            A[r, (k + 1) * nb:(k + 2) * nb] = M
    return A


def _element_index(fs, e):
    """Global rows and columns of element e's local block matrix."""
    n = fs.n
    rows = np.concatenate([fs.row_index(e, i) for i in range(-1, n + 2)])
    cols = np.concatenate([fs.col_block(e, k) for k in range(-1, n + 2)])
    return rows, cols


def misfit_and_gradient(mesh, n_r, c, rho_nodal, dt, src_nodes, wavelets, rec_nodes, observed,
                        beta=0.25, gamma=0.5, xi0=1e-3, part="all"):
    """(E, dE/drho_nodal) of the discrete path, rho on the nodal points (the order of
    ``oracle.fwi``: interior points of every element, then the global nodes).

    ``part="mass"`` keeps only the density of the inertia term (M0; E0, E1, E2 held
    fixed), the quantity the paper's velocity kernel approximates."""
    fs = bruteforce.FullSystem(mesh, n_r, c, rho_nodal, dt, beta, gamma, xi0)
    n, nb, E = fs.n, fs.nb, fs.E
    N = mesh.n_nodes
    src_nodes = np.asarray(src_nodes)
    rec_nodes = np.asarray(rec_nodes)
    wavelets = np.atleast_2d(wavelets)
    observed = np.asarray(observed, dtype=np.float64)
    B, K = wavelets.shape
    dofs = np.stack([el.dofs for el in fs.elements])
    z = lambda *s: np.zeros(s)

    # ---- forward, keeping x_{k+1} and the predictors v_k -------------------------
    st = fwi.State(z(E, n, nb, B), z(E, n, nb, B), z(E, n, nb, B), z(N, B), z(N, B), z(N, B))
    xs, vs = [], []
    traces = np.zeros((B, rec_nodes.size, K))
    for k in range(K):
        f = np.zeros((N, B))
        for s in range(B):
            f[src_nodes[s], s] += wavelets[s, k]
        x, v, st = fs.step_full(st, f)
        xs.append(x)
        vs.append(v)
        traces[:, :, k] = st.ub[rec_nodes].T
    res = observed - traces
    Emis = 0.5 * dt * float(np.sum(res * res))

    # ---- reverse ------------------------------------------------------------------
    a0, a1 = 1.0 / (beta * dt * dt), 1.0 / (beta * dt)
    a2 = 1.0 / (2.0 * beta) - 1.0                       # predictor: a0 u + a1 u' + a2 u''
    cu, cud, cudd = gamma / (beta * dt), 1.0 - gamma / beta, dt * (1.0 - gamma / (2.0 * beta))
    du, dud, dudd = 1.0 / (beta * dt * dt), -1.0 / (beta * dt), 1.0 - 1.0 / (2.0 * beta)
    ub_ = [z(E, n, nb, B), z(N, B)]                     # adjoints of u_{k+1} (interior, boundary)
    ud_ = [z(E, n, nb, B), z(N, B)]
    udd_ = [z(E, n, nb, B), z(N, B)]
    idx = [_element_index(fs, e) for e in range(E)]
    m = (n + 3) * nb
    W = np.zeros((E, m, m))                             # sum_k mu x^T on each element's block
    V = np.zeros((E, n + 1, nb, nb))                    # sum_k mu_(e,i) v_(e,i)^T
    for k in range(K - 1, -1, -1):
        # misfit term of trace sample k (u at receivers after step k)
        ub_[1][rec_nodes] += -dt * res[:, :, k].T
        # Newmark update u', u'' (k+1) <- u (k+1), u (k), u' (k), u'' (k)
        tot = [ub_[j] + cu * ud_[j] + du * udd_[j] for j in range(2)]
        u_k = [-cu * ud_[j] - du * udd_[j] for j in range(2)]
        ud_k = [cud * ud_[j] + dud * udd_[j] for j in range(2)]
        udd_k = [cudd * ud_[j] + dudd * udd_[j] for j in range(2)]
        # u(k+1) is part of x(k+1)
        xbar = np.zeros((fs.size, B))
        for e in range(E):
            for i in range(n):
                xbar[fs.col_block(e, i)] += tot[0][e, i]
        xbar[fs.n_elem_unknowns:] += tot[1]
        mu = fs.solve(xbar, transpose=True)
        x, v = xs[k], vs[k]
        vbar = np.zeros((E, n + 1, nb, B))
        for e in range(E):
            r, cidx = idx[e]
            W[e] += mu[r] @ x[cidx].T
            for i in range(n + 1):
                mr = mu[fs.row_index(e, i)]                        # (nb, B)
                V[e, i] += mr @ v[e, i].T
                vbar[e, i] = -(fs.xi[i] ** 2) * (fs.M0_64[e, i].T @ mr)
        # predictor v = a0 u + a1 u' + a2 u'' at points 0..n (point n: the boundary node)
        for j, coef in ((0, a0), (1, a1), (2, a2)):
            tgt = (u_k, ud_k, udd_k)[j]
            tgt[0] += coef * vbar[:, :n]
            np.add.at(tgt[1], dofs.ravel(), (coef * vbar[:, n]).reshape(E * nb, B))
        ub_, ud_, udd_ = u_k, ud_k, udd_k

    # ---- contraction with the unit-density element blocks ------------------------
    XP = sbfem.XP
    n_int = int(fs.int_ptr[-1])
    g = np.zeros(n_int + N)
    for e, el in enumerate(fs.elements):
        for i in range(n + 1):
            for j in range(nb):
                unit = np.zeros((n + 1, nb), dtype=XP)
                unit[i, j] = 1
                mats = sbfem.coefficient_matrices(el, mesh.node_xy, mesh.p, c, unit)
                if part == "mass":
                    mats = (0 * mats[0], 0 * mats[1], 0 * mats[2], mats[3])
                elif part != "all":
                    raise ValueError(part)
                sys_ = sbfem.element_system(*(mm[None] for mm in mats), np.asarray(fs.xi, dtype=XP), dt, beta)
                Ae = np.asarray(_element_block_matrix(fs, sys_.theta[0], sys_.phi[0], sys_.psi[0]),
                                dtype=np.float64)
                val = -np.sum(Ae * W[e])
                M0i = np.asarray(mats[3][i], dtype=np.float64)
                val += -(fs.xi[i] ** 2) * np.sum(M0i * V[e, i])
                q = fs.int_ptr[e] + i * nb + j if i < n else n_int + el.dofs[j]
                g[q] += val
    return Emis, g


def misfit_only(mesh, n_r, c, rho_nodal, dt, src_nodes, wavelets, rec_nodes, observed,
                beta=0.25, gamma=0.5, xi0=1e-3):
    """E of the same discrete path (for finite-difference checks)."""
    fs = bruteforce.FullSystem(mesh, n_r, c, rho_nodal, dt, beta, gamma, xi0)
    tr, _ = fs.forward(src_nodes, wavelets, rec_nodes)
    res = np.asarray(observed, dtype=np.float64) - tr
    return 0.5 * dt * float(np.sum(res * res))
