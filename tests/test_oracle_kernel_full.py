"""Pins of the full Frechet kernel in the oracle (Section 2: d_t lambda d_t u -
c^2 grad lambda . grad u; the paper keeps only the first term, Section 4)."""

import numpy as np
import pytest

from oracle import fwi
from sbfwi_inputs import structured_mesh, tiny_workload

from test_oracle_dynamics import _lumped_nodal_areas


@pytest.mark.parametrize("p", [2, 3])
def test_nodal_gradient_reproduces_linear_and_quadratic_fields(p):
    """Second-order radial differences and the line's Lagrange derivative are exact for
    fields that are quadratic along every radial line and of degree <= p along the lines."""
    m = structured_mesh(3, 2, p)
    om = fwi.build_model(m, 6, 1.0, np.ones((8, 8)), 0.1)
    G = fwi.gradient_operator(om)
    x, y = (np.asarray(om.points[:, k], dtype=np.float64) for k in (0, 1))
    for u, ex in [(2 * x - 3 * y, np.c_[np.full_like(x, 2.0), np.full_like(x, -3.0)]),
                  (x * x + x * y, np.c_[2 * x + y, x])]:
        g = (G @ u).reshape(-1, 2)
        assert np.abs(g - ex).max() < 1e-10


def test_gradient_term_matches_the_stiffness_density_derivative():
    """<a . g_grad, drho> ~ dE/d(rho in E0, E1, E2), <a . g_vel, drho> ~ dE/d(rho in M0) and
    their sum ~ dE/drho along smooth directions (within 10 %; measured 2-8 %): the
    gradient term the paper drops carries the stiffness part of the derivative, with the
    sign and time pairing of the reversed-time kernel."""
    w = tiny_workload(K=200)
    wf = tiny_workload(refine=2, K=200)
    mt = fwi.build_model(wf.mesh, wf.n_r, 1.0, wf.rho_true, w.dt)
    d, _, _ = fwi.forward(mt, wf.src_nodes, wf.wavelets, wf.rec_nodes, keep=False)
    m0 = fwi.build_model(w.mesh, w.n_r, 1.0, w.rho_start, w.dt)
    tr, store, _, su = fwi.forward(m0, w.src_nodes, w.wavelets, w.rec_nodes, keep_u=True)
    _, res = fwi.misfit(tr, d, w.dt)
    gv = fwi.adjoint_gradient(m0, store, res, w.rec_nodes)
    gf = fwi.adjoint_gradient(m0, store, res, w.rec_nodes, store_u=su)
    gg = gf - gv
    a = _lumped_nodal_areas(m0, w.mesh)
    r0 = np.asarray(m0.rho_nodal, dtype=np.float64)

    def E(rs, rm):
        mm = fwi.build_model(w.mesh, w.n_r, 1.0, rs, w.dt, rho_kind="nodal", rho_mass_nodal=rm)
        t, _, _ = fwi.forward(mm, w.src_nodes, w.wavelets, w.rec_nodes, keep=False)
        return fwi.misfit(t, d, w.dt)[0]

    pts = np.asarray(m0.points, dtype=np.float64)
    eps = 1e-5
    for dirn in [np.sin(2 * np.pi * pts[:, 0]) * np.cos(np.pi * pts[:, 1]),
                 np.exp(-((pts[:, 0] - 0.5) ** 2 + (pts[:, 1] - 0.7) ** 2) / 0.02)]:
        up, dn = r0 * (1 + eps * dirn), r0 * (1 - eps * dirn)
        fd_stiff = (E(up, r0) - E(dn, r0)) / (2 * eps)
        fd_all = (E(up, up) - E(dn, dn)) / (2 * eps)
        assert abs(np.sum(gg * a * dirn * r0) / fd_stiff - 1) < 0.10
        assert abs(np.sum(gf * a * dirn * r0) / fd_all - 1) < 0.10
