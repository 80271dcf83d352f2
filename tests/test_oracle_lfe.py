"""Pins of the low-frequency-expansion oracle (Section 3.2) and of the radial
finite-difference condensation on the reduced (density constant along xi) element."""

import numpy as np
import pytest

from oracle import lfe, sbfem
from sbfwi_inputs import structured_mesh


def _reduced_element(p, n_r, rho_boundary):
    """E0..M0 of element 0 of a 2 x 2 mesh with the density constant along every
    radial line (its boundary values), and the FD condensation's S as a function of
    the Newmark mass factor eps = 1/(beta dt^2)."""
    m = structured_mesh(2, 2, p)
    el = sbfem.elements_from_mesh(m)[0]
    n = n_r - 1
    xi = sbfem.radial_grid(n, 1e-3, sbfem.XP)
    rho = np.tile(np.asarray(rho_boundary, dtype=sbfem.XP), (n + 1, 1))
    mats = sbfem.coefficient_matrices(el, m.node_xy, p, 1.0, rho)

    def S(eps):
        if eps == 0:
            sys_ = sbfem.element_system(*(q[None] for q in mats), xi, 1.0, 0.25, static=True)
        else:                                   # mass factor 1/(beta dt^2) = eps with dt = 1
            sys_ = sbfem.element_system(*(q[None] for q in mats), xi, 1.0, 1.0 / eps)
        return np.asarray(sbfem.condense(sys_).S[0], dtype=np.float64)

    E = [np.asarray(q[0], dtype=np.float64) for q in mats]
    return E, S, m


@pytest.mark.parametrize("p", [2, 3])
def test_riccati_stiffness_is_the_limit_of_the_fd_static_stiffness(p):
    """Static S of the radial FD condensation -> K of the Riccati equation, second order
    in the radial spacing; K is symmetric and annihilates constants."""
    nb = 4 * p
    rho_b = 1.0 + 0.5 * np.random.default_rng(p).random(nb)
    errs = []
    for n_r in (9, 17, 33, 65):
        (E0, E1, E2, M0), S, _ = _reduced_element(p, n_r, rho_b)
        K, imag = lfe.riccati_stiffness(E0, E1, E2)
        assert imag < 1e-12
        errs.append(np.linalg.norm(S(0) - K) / np.linalg.norm(K))
    assert np.abs(K - K.T).max() < 1e-12 * np.abs(K).max()
    assert np.abs(K @ np.ones(nb)).max() < 1e-12 * np.abs(K).max()
    ratios = [a / b for a, b in zip(errs, errs[1:])]
    assert all(r > 3.0 for r in ratios), (errs, ratios)     # h halves: error / ~4
    assert errs[-1] < 2e-3


@pytest.mark.parametrize("p", [2, 3])
def test_lyapunov_mass_is_the_limit_of_the_fd_mass_derivative(p):
    """dS/d(eps) of the FD condensation at eps = 0 -> M of the Lyapunov equation
    (S ~ K - omega^2 M with -omega^2 in the place of the Newmark mass factor)."""
    nb = 4 * p
    rho_b = 1.0 + 0.5 * np.random.default_rng(10 + p).random(nb)
    errs = []
    for n_r in (9, 17, 33, 65):
        (E0, E1, E2, M0), S, _ = _reduced_element(p, n_r, rho_b)
        K, _ = lfe.riccati_stiffness(E0, E1, E2)
        M = lfe.lyapunov_mass(K, E0, E1, M0)
        eps = 1e-3 * np.abs(E2).max() / np.abs(M0).max()
        dS = (S(eps) - S(-eps)) / (2 * eps)
        errs.append(np.linalg.norm(dS - M) / np.linalg.norm(M))
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 3e-3
    assert np.abs(M - M.T).max() < 1e-10 * np.abs(M).max()


def test_lyapunov_mass_carries_the_element_mass():
    """For a homogeneous element the constant mode's kinetic mass is the element's mass:
    1^T M 1 = rho * area (here a square of side 1/2)."""
    p, rho0 = 3, 2.7
    (E0, E1, E2, M0), _, m = _reduced_element(p, 5, np.full(4 * p, rho0))
    K, _ = lfe.riccati_stiffness(E0, E1, E2)
    M = lfe.lyapunov_mass(K, E0, E1, M0)
    one = np.ones(4 * p)
    assert one @ M @ one == pytest.approx(rho0 * 0.25, rel=1e-12)


def _plate(nx=3, p=2, rho=None):
    m = structured_mesh(nx, nx, p)
    rho = np.ones(m.n_nodes) if rho is None else rho(m)
    K, M = lfe.assemble(m, lfe.element_matrices(m, 1.0, rho))
    return m, K, M


def test_lfe_global_matrices_are_symmetric_and_definite():
    m, K, M = _plate(rho=lambda m: 1.0 + 0.3 * np.random.default_rng(0).random(m.n_nodes))
    assert np.abs(K - K.T).max() < 1e-12 * np.abs(K).max()
    assert np.abs(M - M.T).max() < 1e-12 * np.abs(M).max()
    assert np.linalg.eigvalsh(M).min() > 0
    ev = np.sort(np.linalg.eigvalsh(K))
    assert abs(ev[0]) < 1e-12 * ev[-1] and ev[1] > 1e-3 * ev[-1]      # one rigid (constant) mode


def test_lfe_total_mass_of_a_homogeneous_plate():
    m, K, M = _plate(rho=lambda m: np.full(m.n_nodes, 1.7))
    one = np.ones(m.n_nodes)
    assert one @ M @ one == pytest.approx(1.7 * 1.0, rel=1e-12)    # unit square
    assert np.abs(K @ one).max() < 1e-12 * np.abs(K).max()


def test_lfe_newmark_conserves_the_discrete_energy():
    """Average-acceleration Newmark on a symmetric pencil: 1/2 u'^T M u' + 1/2 u^T K u stays
    at its initial value in free vibration (400 steps)."""
    m, K, M = _plate(rho=lambda m: 1.0 + 0.3 * np.random.default_rng(0).random(m.n_nodes))
    u0 = np.random.default_rng(1).standard_normal(m.n_nodes)
    us, vs = lfe.newmark(K, M, np.zeros((400, m.n_nodes)), 0.05, u0=u0, v0=np.zeros(m.n_nodes))
    E = 0.5 * np.einsum("ki,ij,kj->k", vs, M, vs) + 0.5 * np.einsum("ki,ij,kj->k", us, K, us)
    E0 = 0.5 * u0 @ K @ u0
    assert np.abs(E / E0 - 1).max() < 1e-12


def test_fd_traces_approach_the_lfe_traces_at_low_frequency():
    """Homogeneous plate (density constant along xi, so both methods solve the same
    equation): the radial-FD receiver traces converge towards the low-frequency expansion's
    as N_r grows when the source frequency is low, and stay apart at a higher frequency
    where the one-term expansion itself is inaccurate (a trend, not a number)."""
    from oracle import fwi
    from sbfwi_inputs import boundary_nodes, ricker
    m = structured_mesh(4, 4, 2)
    src = int(boundary_nodes(m, "top")[4])
    rec = np.array([int(boundary_nodes(m, "bottom")[3]), int(boundary_nodes(m, "left")[5])])
    K, M = lfe.assemble(m, lfe.element_matrices(m, 1.0, np.ones(m.n_nodes)))
    dt, steps = 0.0625, 300
    err = {}
    for f0 in (0.2, 0.4):
        w = ricker(f0, dt, steps)
        F = np.zeros((steps, m.n_nodes))
        F[:, src] = w
        tl = lfe.newmark(K, M, F, dt)[0][:, rec].T
        for n_r in (5, 9, 17):
            tr, _, _ = fwi.forward(fwi.build_model(m, n_r, 1.0, np.ones((8, 8)), dt), [src], w[None], rec, keep=False)
            err[(f0, n_r)] = np.linalg.norm(tr[0] - tl) / np.linalg.norm(tl)
    assert err[(0.2, 5)] > err[(0.2, 9)] > err[(0.2, 17)]
    assert err[(0.2, 17)] < 0.05
    assert err[(0.4, 17)] > 3 * err[(0.2, 17)]


def test_lfe_adjoint_fields_give_the_exact_inertia_derivative():
    """The comparison method's gradient correlates forward and time-reversed adjoint
    velocities.  Its consistent form, dt sum_m u'_fwd[K-1-m]^T (dM/drho) lambda'[m] with
    dM/drho the Lyapunov mass's derivative along a direction of the inertia density (M is
    linear in that density when K is held), must equal the central finite difference of the
    misfit along that direction: this pins the adjoint's source, sign and time pairing.
    The paper's nodal product (each boundary node's own velocities, weighted by the mass it
    carries) is a lumped stand-in for that form: on this 4 x 4 order-2 plate it differs
    from the exact derivative by 20-100 % along a direction (the boundary nodes' densities
    each set the mass of a whole sector of an element), which is recorded, not asserted
    beyond the sign of the smooth direction."""
    from sbfwi_inputs import boundary_nodes, ricker
    m = structured_mesh(4, 4, 2)
    N = m.n_nodes
    rho = 1.0 + 0.2 * np.sin(2 * np.pi * m.node_xy[:, 0]) * np.cos(np.pi * m.node_xy[:, 1])
    top = boundary_nodes(m, "top")
    src = [int(top[len(top) // 2])]
    recs = np.unique(np.concatenate([boundary_nodes(m, s) for s in ("bottom", "left", "right")]))[::3]
    dt, K = 0.0625, 96
    wav = ricker(0.8, dt, K)[None]
    obs = np.zeros((1, len(recs), K))
    _, E, g, vel, lvel = lfe.forward_and_gradient(m, 1.0, rho, dt, src, wav, recs, obs, fields=True)
    C = sum(dt * np.outer(vel[0, K - 1 - k], lvel[0, k]) for k in range(K))
    _, M0 = lfe.assemble(m, lfe.element_matrices(m, 1.0, rho, rho_mass=rho))
    one = np.ones(N)
    mass = np.array([one @ (lfe.assemble(m, lfe.element_matrices(m, 1.0, rho, rho_mass=rho + e))[1] - M0) @ one
                     for e in np.eye(N)])
    assert mass.sum() == pytest.approx(1.0, rel=1e-12)          # the unit square's area
    h = 1e-5
    rng = np.random.default_rng(0)
    for d in (np.cos(np.pi * m.node_xy[:, 0]), rng.standard_normal(N)):
        dM = lfe.assemble(m, lfe.element_matrices(m, 1.0, rho, rho_mass=rho + d))[1] - M0
        fd = (lfe.forward_and_gradient(m, 1.0, rho, dt, src, wav, recs, obs, rho_mass=rho + h * d)[1]
              - lfe.forward_and_gradient(m, 1.0, rho, dt, src, wav, recs, obs, rho_mass=rho - h * d)[1]) / (2 * h)
        assert np.sum(dM * C) == pytest.approx(fd, rel=1e-6)
    smooth = np.cos(np.pi * m.node_xy[:, 0])
    fd_s = (lfe.forward_and_gradient(m, 1.0, rho, dt, src, wav, recs, obs, rho_mass=rho + h * smooth)[1]
            - lfe.forward_and_gradient(m, 1.0, rho, dt, src, wav, recs, obs, rho_mass=rho - h * smooth)[1]) / (2 * h)
    assert np.sign((mass * g) @ smooth) == np.sign(fd_s)
