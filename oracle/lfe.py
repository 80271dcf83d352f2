"""Low-frequency expansion of the reduced element equation (Section 3.2), the paper's
comparison method.  TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

With the density held constant along every radial line (it varies with eta only),
E0, E1, E2, M0 no longer depend on xi and the radial ODE reduces to Eq. (simplified).
Its dynamic stiffness S(omega) at the boundary is expanded as S ~ K - omega^2 M
(Eq. (S)):

* K solves the algebraic Riccati equation (K - E1) E0^-1 (K - E1^T) - E2 = 0.  With
  q = xi E0 u_xi + E1^T u (Eq. (internal)) the static ODE is the first-order system
  xi d/dxi [u; q] = -Z [u; q] with
      Z = [[E0^-1 E1^T, -E0^-1], [-E2 + E1 E0^-1 E1^T, -E1 E0^-1]];
  its solutions are eigenvectors of Z times xi^-lambda, and those bounded at the
  scaling centre (Re lambda < 0, plus the constant mode u = 1, q = 0 of the double
  zero eigenvalue, exact because E1^T 1 = E2 1 = 0) span q = K u, so K = Q_q Q_u^-1.
* M solves the Lyapunov equation (K - E1) E0^-1 M + M E0^-1 (K - E1^T) + 2 M - M0 = 0,
  as one dense linear system in the n_b^2 entries of M.

The comparison method's time loop assembles K and M (symmetric) over the mesh and
steps M u'' + K u = f with Newmark (``element_matrices``, ``assemble``, ``newmark``).

Pinned by ``tests/test_oracle_lfe.py``: the radial finite-difference condensation of
the same reduced element (``oracle.sbfem``, density constant in xi) converges to K
(static S) and to M (derivative of S with respect to the Newmark mass factor) as N_r
grows -- two independent discretisations of one equation; 1^T M 1 is the element's
(and the plate's) mass; K and M are symmetric with one rigid mode; the Newmark loop
conserves the discrete energy; and on a homogeneous plate the radial-FD traces approach
the expansion's as N_r grows at a low source frequency.
"""

import numpy as np
import scipy.linalg as sla


def riccati_stiffness(E0, E1, E2):
    """K with (K - E1) E0^-1 (K - E1^T) - E2 = 0 from the bounded solutions of Z."""
    nb = E0.shape[0]
    E0i = np.linalg.inv(E0)
    Z = np.block([[E0i @ E1.T, -E0i], [-E2 + E1 @ E0i @ E1.T, -E1 @ E0i]])
    lam, V = np.linalg.eig(Z)
    order = np.argsort(lam.real)
    # the two eigenvalues closest to zero are the constant mode and its unbounded
    # (log xi) partner; the n_b - 1 most negative ones decay towards the centre
    near_zero = set(np.argsort(np.abs(lam))[:2])
    keep = [k for k in order if k not in near_zero][:nb - 1]
    Q = np.concatenate([V[:, keep], np.concatenate([np.ones(nb), np.zeros(nb)])[:, None]], axis=1)
    K = Q[nb:] @ np.linalg.inv(Q[:nb])
    return K.real, float(np.abs(K.imag).max() / np.abs(K.real).max())


def lyapunov_mass(K, E0, E1, M0):
    """M with (K - E1) E0^-1 M + M E0^-1 (K - E1^T) + 2 M - M0 = 0 (row-major vec)."""
    nb = E0.shape[0]
    E0i = np.linalg.inv(E0)
    A = (K - E1) @ E0i
    B = E0i @ (K - E1.T)
    I = np.eye(nb)
    L = np.kron(A, I) + np.kron(I, B.T) + 2.0 * np.eye(nb * nb)
    return np.linalg.solve(L, M0.reshape(-1)).reshape(nb, nb)


# ----------------------------------------------------------------------------
# The low-frequency-expansion time loop (the paper's comparison method)
# ----------------------------------------------------------------------------

def element_matrices(mesh, c, rho_boundary_nodal, xi0=1e-3, rho_mass=None):
    """K_e, M_e of every element with its density taken constant along xi (the values at
    its boundary nodes, Section 3.2): E0..M0 at xi = 1 (any xi: they do not depend on it
    then) -> Riccati K, Lyapunov M.  ``rho_mass`` (tests only) gives M0 its own boundary
    densities while E0, E1, E2 keep ``rho_boundary_nodal``: the density of the inertia
    term alone."""
    from . import sbfem
    els = sbfem.elements_from_mesh(mesh)
    out = []
    for el in els:
        rho = np.tile(np.asarray(rho_boundary_nodal, dtype=sbfem.XP)[el.dofs], (2, 1))
        E0, E1, E2, M0 = (np.asarray(q[-1], dtype=np.float64)
                          for q in sbfem.coefficient_matrices(el, mesh.node_xy, mesh.p, c, rho))
        if rho_mass is not None:
            rm = np.tile(np.asarray(rho_mass, dtype=sbfem.XP)[el.dofs], (2, 1))
            M0 = np.asarray(sbfem.coefficient_matrices(el, mesh.node_xy, mesh.p, c, rm)[3][-1], dtype=np.float64)
        K, _ = riccati_stiffness(E0, E1, E2)
        out.append((el.dofs, K, lyapunov_mass(K, E0, E1, M0)))
    return out


def assemble(mesh, elem):
    """Global K and M (dense; tiny meshes) from the element matrices."""
    N = mesh.n_nodes
    K, M = np.zeros((N, N)), np.zeros((N, N))
    for dofs, Ke, Me in elem:
        K[np.ix_(dofs, dofs)] += Ke
        M[np.ix_(dofs, dofs)] += Me
    return K, M


def newmark(K, M, f, dt, beta=0.25, gamma=0.5, u0=None, v0=None):
    """M u'' + K u = f by Newmark (Eq. (Newmark)) from rest, or from u0, v0 with the
    consistent initial acceleration; f[k] (steps, N) is the load at the end of step k.
    Returns u, u' after every step."""
    N = K.shape[0]
    u = np.zeros(N) if u0 is None else np.array(u0, dtype=np.float64)
    v = np.zeros(N) if v0 is None else np.array(v0, dtype=np.float64)
    a = np.linalg.solve(M, -K @ u)               # at rest, or free vibration from u0 (no load at t = 0)
    a0, a1, a2 = 1 / (beta * dt * dt), 1 / (beta * dt), 1 / (2 * beta) - 1
    lu = sla.lu_factor(K + a0 * M)
    us, vs = [], []
    for k in range(f.shape[0]):
        un = sla.lu_solve(lu, f[k] + M @ (a0 * u + a1 * v + a2 * a))
        an = a0 * (un - u) - a1 * v - a2 * a
        v = v + dt * ((1 - gamma) * a + gamma * an)
        u, a = un, an
        us.append(u.copy())
        vs.append(v.copy())
    return np.array(us), np.array(vs)


def forward_and_gradient(mesh, c, rho_boundary_nodal, dt, src_nodes, wavelets, rec_nodes, observed, beta=0.25,
                         gamma=0.5, rho_mass=None, fields=False):
    """The comparison method's misfit pipeline on the boundary nodes: Newmark traces of
    every shot, E = 1/2 dt sum (d - u)^2, and the reversed-time adjoint (the same
    symmetric pencil driven by the residuals, last sample first) correlated with the
    forward velocities: g(node) = dt sum_m sum_shots u'_fwd[K-1-m] lambda'[m] (the
    conventions of ``oracle.fwi``; the expansion has nodal points on the boundary only).
    ``rho_mass`` as in ``element_matrices``.  Returns (traces (B, R, K), E, g (n_nodes,)),
    and with ``fields`` also the forward velocities (B, K, N) after every step and the
    adjoint velocities (B, K, N) after every adjoint step.

    The nodal product is the paper's convention (Section 4: the fields at the nodal points
    used directly).  The exact derivative of E with respect to the density of the inertia
    term is the consistent form dt sum_m u'_fwd[K-1-m]^T (dM/drho_j) lambda'[m] of the same
    fields (pinned by finite differences in the tests); with only boundary nodes, whose
    density sets the mass of a whole sector of the element, the nodal product is a coarse
    stand-in for it."""
    K_, M_ = assemble(mesh, element_matrices(mesh, c, rho_boundary_nodal, rho_mass=rho_mass))
    src_nodes, rec_nodes = np.asarray(src_nodes), np.asarray(rec_nodes)
    wavelets = np.atleast_2d(wavelets)
    B, K = wavelets.shape
    N = mesh.n_nodes
    traces = np.zeros((B, rec_nodes.size, K))
    vel = np.zeros((B, K, N))
    for s in range(B):
        F = np.zeros((K, N))
        F[:, src_nodes[s]] = wavelets[s]
        us, vs = newmark(K_, M_, F, dt, beta, gamma)
        traces[s] = us[:, rec_nodes].T
        vel[s] = vs
    res = np.asarray(observed, dtype=np.float64) - traces
    E = 0.5 * dt * float(np.sum(res * res))
    g = np.zeros(N)
    lvel = np.zeros((B, K, N))
    for s in range(B):
        F = np.zeros((K, N))
        for m in range(K):
            np.add.at(F[m], rec_nodes, res[s, :, K - 1 - m])
        _, lv = newmark(K_, M_, F, dt, beta, gamma)
        lvel[s] = lv
        for m in range(K):
            g += dt * vel[s, K - 1 - m] * lv[m]
    if fields:
        return traces, E, g, vel, lvel
    return traces, E, g
