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
