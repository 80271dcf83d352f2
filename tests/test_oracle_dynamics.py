"""Pins of the oracle's time stepping, global solve, misfit and gradient (Sections 2-4).

Each test checks the oracle against something other than itself:

* the condensed algorithm against the brute-force uncondensed solve;
* free-vibration frequencies of the semi-discrete radial ODE against the Neumann
  Laplacian closed form (homogeneous density) and against the closed form for an
  exponentially graded density (which exercises the d/dxi E terms);
* average-acceleration Newmark against its textbook amplification and period
  (scalar oscillator), and the full condensed stepper started on an eigenmode
  against the same closed form;
* the misfit against a hand-summable case;
* the bilinear density map against linear reproduction and its transpose;
* the velocity part of the Frechet kernel against the finite-difference
  derivative of the misfit with respect to the inertia density.
"""

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from oracle import bruteforce, fwi, sbfem
from sbfwi_inputs import structured_mesh, tiny_workload


@pytest.fixture(scope="module")
def tiny():
    return tiny_workload()


def test_condensed_equals_bruteforce(tiny):
    w = tiny
    m = fwi.build_model(w.mesh, w.n_r, w.c, w.rho_true, w.dt)
    tr, _, st = fwi.forward(m, w.src_nodes, w.wavelets, w.rec_nodes, K=80, keep=False)
    fs = bruteforce.FullSystem(w.mesh, w.n_r, w.c, m.rho_nodal, w.dt)
    tb, sb = fs.forward(w.src_nodes, w.wavelets, w.rec_nodes, K=80)
    assert np.linalg.norm(tb - tr) <= 1e-11 * np.linalg.norm(tr)
    assert np.linalg.norm(sb.u - st.u) <= 1e-11 * np.linalg.norm(st.u)
    assert np.linalg.norm(sb.udb - st.udb) <= 1e-11 * np.linalg.norm(st.udb)


def test_global_solve_residual(tiny):
    w = tiny
    m = fwi.build_model(w.mesh, w.n_r, w.c, w.rho_true, w.dt)
    rng = np.random.default_rng(0)
    F = rng.standard_normal((m.n_nodes, 3))
    x = m.lu.solve(F)
    assert np.linalg.norm(m.A @ x - F) <= 1e-13 * np.linalg.norm(F)


def _neumann_square(count):
    vals = sorted(np.pi * np.hypot(a, b) for a in range(5) for b in range(5))
    return np.array(vals[:count])


def test_free_vibration_homogeneous_square_converges():
    exact = _neumann_square(8)
    errs = []
    for nx, p, nr in [(4, 2, 8), (8, 4, 16)]:
        mesh = structured_mesh(nx, nx, p)
        m = fwi.build_model(mesh, nr, 1.0, np.ones((8, 8)), 1.0, static=True)
        fs = bruteforce.FullSystem(mesh, nr, 1.0, m.rho_nodal, 1.0, static=True)
        om, _ = fs.frequencies(count=8)
        errs.append(np.abs(om[1:] - exact[1:]) / exact[1:])
    assert errs[1].max() < 5e-4
    assert errs[1].max() < errs[0].max()


def test_free_vibration_graded_density_closed_form():
    """rho = exp(alpha x), c = 1 on the unit square with free edges.

    u = exp(-alpha x/2) (cos(k x) + alpha/(2k) sin(k x)) cos(n pi y), k = m pi, gives
    omega^2 = (m pi)^2 + alpha^2/4 + (n pi)^2 for m >= 1 and (n pi)^2 for m = 0.
    """
    alpha = 1.5
    w2 = sorted([(np.pi * n) ** 2 for n in range(4)] +
                [(np.pi * m) ** 2 + alpha ** 2 / 4 + (np.pi * n) ** 2 for m in range(1, 4) for n in range(4)])
    exact = np.sqrt(w2[:8])
    mesh = structured_mesh(8, 8, 4)
    els = sbfem.elements_from_mesh(mesh)
    xi = sbfem.radial_grid(15)
    pts, _ = fwi.nodal_points(mesh, els, xi)
    fs = bruteforce.FullSystem(mesh, 16, 1.0, np.exp(alpha * pts[:, 0]), 1.0, static=True)
    om, _ = fs.frequencies(count=8)
    assert np.abs(om[1:] - exact[1:]).max() / exact[1] < 1e-3
    # dropping the variable-density terms would miss alpha^2/4 in the m >= 1 modes
    assert abs(om[2] - exact[2]) < 0.1 * (exact[2] - np.pi)


def _newmark_scalar(omega, dt, K, beta=0.25, gamma=0.5):
    """The oracle's Newmark formulas on m u'' + k u = 0 (m = 1, k = omega^2)."""
    u, ud, udd = 1.0, 0.0, -omega ** 2
    out = []
    for _ in range(K):
        pred = fwi.newmark_predictor(u, ud, udd, dt, beta)
        u_new = pred / (omega ** 2 + 1.0 / (beta * dt * dt))     # (k + m/(beta dt^2)) u = m * pred
        ud, udd = fwi.newmark_update(u, ud, udd, u_new, dt, beta, gamma)
        u = u_new
        out.append(u)
    return np.array(out)


@pytest.mark.parametrize("wdt", [0.1, 1.0, 3.0])
def test_newmark_scalar_oscillator_closed_form(wdt):
    """Average acceleration: unit amplification, tan(wbar dt / 2) = w dt / 2."""
    omega, dt, K = 2.0, wdt / 2.0, 500
    u = _newmark_scalar(omega, dt, K)
    wbar = 2.0 * np.arctan(omega * dt / 2.0) / dt
    t = dt * np.arange(1, K + 1)
    assert np.abs(u - np.cos(wbar * t)).max() < 1e-11


def test_condensed_stepper_on_eigenmode_follows_newmark_closed_form():
    """Start the full condensed stepper on a free-vibration mode (u = x, u' = 0, u'' = -w^2 x).

    Average-acceleration Newmark then gives u_k = x cos(wbar t_k) exactly, with
    tan(wbar dt/2) = w dt/2; this pins the residual source, condensation, global
    solve, back-substitution and Newmark update together.
    """
    mesh = structured_mesh(4, 4, 2)
    nr, dt = 8, 0.0625
    m = fwi.build_model(mesh, nr, 1.0, np.ones((8, 8)), dt)
    fs = bruteforce.FullSystem(mesh, nr, 1.0, m.rho_nodal, dt, static=True)
    vals, vecs = sla.eig(fs.matrix.toarray(), fs.mass.toarray())
    fin = np.isfinite(vals)
    vals, vecs = vals[fin], vecs[:, fin]
    w2 = -vals.real
    j = int(np.argsort(w2)[3])                       # the sqrt(2) pi mode (simple)
    x0 = vecs[:, j]
    x0 = (x0 / x0[np.argmax(np.abs(x0))]).real
    x, omega2 = fs.refine_mode(x0, w2[j])            # QZ gives ~1e-8; Newton with extended residuals
    omega = np.sqrt(omega2)
    E = len(fs.elements)
    u0 = np.stack([np.stack([x[fs.col_block(e, i)] for i in range(fs.n)]) for e in range(E)])[..., None]
    ub0 = x[fs.n_elem_unknowns:][:, None]
    st = fwi.State(u0.copy(), np.zeros_like(u0), -omega ** 2 * u0, ub0.copy(), np.zeros_like(ub0), -omega ** 2 * ub0)
    K = 400
    rec = np.arange(m.n_nodes)
    tr, _, _ = fwi.forward(m, np.array([0]), np.zeros((1, K)), rec, keep=False, state=st)
    wbar = 2.0 * np.arctan(omega * dt / 2.0) / dt
    expect = ub0[:, 0][:, None] * np.cos(wbar * dt * np.arange(1, K + 1))[None, :]
    err = np.abs(tr[0] - expect).max()
    assert err < 1e-11, err


def test_misfit_closed_form():
    tr = np.zeros((2, 3, 4))
    ob = np.zeros((2, 3, 4))
    ob[0, 1, 2] = 3.0
    ob[1, 2, 0] = -4.0
    E, res = fwi.misfit(tr, ob, 0.5)
    assert E == pytest.approx(0.5 * 0.5 * (9 + 16))
    assert res[0, 1, 2] == 3.0 and res[1, 2, 0] == -4.0


def test_density_map_linear_reproduction_and_transpose():
    gx, gy, lx, ly = 17, 11, 1.0, 0.7
    xc = (np.arange(gx) + 0.5) * lx / gx
    yc = (np.arange(gy) + 0.5) * ly / gy
    X, Y = np.meshgrid(xc, yc)
    grid = 1.0 + 2.0 * X - 3.0 * Y
    rng = np.random.default_rng(1)
    pts = np.c_[rng.uniform(xc[0], xc[-1], 50), rng.uniform(yc[0], yc[-1], 50)]
    vals = fwi.grid_to_points(grid, pts, lx, ly)
    assert np.allclose(vals, 1.0 + 2.0 * pts[:, 0] - 3.0 * pts[:, 1], atol=1e-13)
    # clamped outside the band of cell centres
    edge = fwi.grid_to_points(grid, np.array([[0.0, 0.0]]), lx, ly)
    assert edge[0] == pytest.approx(grid[0, 0])
    gpt = rng.standard_normal(50)
    assert np.dot(vals, gpt) == pytest.approx(np.sum(grid * fwi.points_to_grid(gpt, pts, gx, gy, lx, ly)))


def _lumped_nodal_areas(m: fwi.Model, mesh):
    """Area that each nodal point stands for (trapezoid in xi, consistent weights in eta)."""
    n, xi = m.n, m.xi
    h = xi[1] - xi[0]
    a = np.zeros(m.n_int + m.n_nodes)
    eta, wq = sbfem.gauss_points(mesh.p)
    phi, _ = sbfem.lagrange(mesh.p, eta)
    for e, el in enumerate(m.elements):
        s = np.zeros(el.dofs.size)
        for ln, loc in zip(el.lines, el.line_local):
            _, _, det, _, _ = sbfem.line_geometry(mesh.node_xy[ln], el.centre, mesh.p, eta)
            s[loc] += phi.T @ (wq * det)
        for i in range(n):
            wi = xi[i] * h if i > 0 else xi[0] * h / 2 + h * h / 8
            a[m.int_ptr[e] + i * el.dofs.size:m.int_ptr[e] + (i + 1) * el.dofs.size] = s * wi
        a[m.n_int + el.dofs] += s * (h / 2) * (1 - h / 4)
    return a


@pytest.mark.slow
def test_kernel_matches_inertia_density_derivative(tiny):
    """<a . g, drho> ~ dE/d(rho in M0) along smooth directions (within 6%).

    g is the velocity part of the Frechet kernel on nodal points (Section 4) and a
    the area each nodal point stands for; the finite difference perturbs only the
    density of the inertia term, so the dropped gradient term plays no role.  A
    wrong sign or a reversed time pairing fails this.
    """
    w = tiny
    wf = tiny_workload(refine=2)
    mt = fwi.build_model(wf.mesh, wf.n_r, 1.0, wf.rho_true, w.dt)
    d, _, _ = fwi.forward(mt, wf.src_nodes, wf.wavelets, wf.rec_nodes, keep=False)
    m0 = fwi.build_model(w.mesh, w.n_r, 1.0, w.rho_start, w.dt)
    tr, store, _ = fwi.forward(m0, w.src_nodes, w.wavelets, w.rec_nodes)
    _, res = fwi.misfit(tr, d, w.dt)
    g = fwi.adjoint_gradient(m0, store, res, w.rec_nodes)
    a = _lumped_nodal_areas(m0, w.mesh)
    assert abs(a.sum() - 1.0) < 1e-5

    def E_mass(rm):
        mm = fwi.build_model(w.mesh, w.n_r, 1.0, w.rho_start, w.dt, rho_mass_nodal=rm)
        t, _, _ = fwi.forward(mm, w.src_nodes, w.wavelets, w.rec_nodes, keep=False)
        return fwi.misfit(t, d, w.dt)[0]

    pts = m0.points
    for dirn in [np.sin(2 * np.pi * pts[:, 0]) * np.cos(np.pi * pts[:, 1]),
                 np.exp(-((pts[:, 0] - 0.5) ** 2 + (pts[:, 1] - 0.7) ** 2) / 0.02)]:
        eps = 1e-5
        fd = (E_mass(1 + eps * dirn) - E_mass(1 - eps * dirn)) / (2 * eps)
        gk = np.sum(g * a * dirn)
        assert abs(gk / fd - 1.0) < 0.06


def test_kernel_linear_in_residual_and_additive_over_shots(tiny):
    w = tiny
    m0 = fwi.build_model(w.mesh, w.n_r, 1.0, w.rho_start, w.dt)
    K = 60
    srcs = np.array([w.src_nodes[0], w.rec_nodes[0]])
    wav = np.stack([w.wavelets[0, :K], 0.5 * w.wavelets[0, :K]])
    tr, store, _ = fwi.forward(m0, srcs, wav, w.rec_nodes)
    rng = np.random.default_rng(2)
    res = rng.standard_normal(tr.shape)
    g = fwi.adjoint_gradient(m0, store, res, w.rec_nodes)
    g2 = fwi.adjoint_gradient(m0, store, 2.5 * res, w.rec_nodes)
    assert np.allclose(g2, 2.5 * g, rtol=1e-12, atol=1e-14 * np.abs(g).max())
    parts = sum(fwi.adjoint_gradient(m0, store[:, :, s:s + 1], res[s:s + 1], w.rec_nodes) for s in range(2))
    assert np.allclose(parts, g, rtol=1e-11, atol=1e-13 * np.abs(g).max())


def test_sharp_high_contrast_is_unstable_for_the_radial_fd_scheme(tiny):
    """The workloads' flaw contrast is limited by the scheme itself.

    With the density jumping to 1e-3 of the background the semi-discrete pencil
    has real negative omega^2 (exponentially growing modes), while the paper's
    weak-inclusion contrast of 1/2 has none.
    """
    import scipy.linalg as sla
    w = tiny
    X, Y = np.meshgrid((np.arange(64) + 0.5) / 64, (np.arange(64) + 0.5) / 64)
    cx, cy = w.info["flaw"]["centre"]
    inside = np.hypot(X - cx, Y - cy) <= 0.1
    mins = []
    for f in (1e-3, 0.5):
        rho = np.where(inside, f, 1.0)
        m = fwi.build_model(w.mesh, w.n_r, 1.0, rho, w.dt, static=True)
        fs = bruteforce.FullSystem(w.mesh, w.n_r, 1.0, m.rho_nodal, w.dt, static=True)
        vals = sla.eigvals(fs.matrix.toarray(), fs.mass.toarray())
        w2 = -vals[np.isfinite(vals)]
        mins.append(w2.real.min())
    assert mins[0] < -1e3
    assert mins[1] > -1e-6


def test_a_tapered_edge_does_not_stabilise_the_1e3_contrast(tiny):
    """Grading the flaw's edge does not rescue the configs' 1e-3 contrast: with the density
    falling log-linearly from 1 to 1e-3 over one radius outside the flaw the pencil still
    has negative omega^2, while 1e-2 with the same taper has none (sharp 1e-2 does)."""
    import scipy.linalg as sla
    w = tiny
    X, Y = np.meshgrid((np.arange(64) + 0.5) / 64, (np.arange(64) + 0.5) / 64)
    cx, cy = w.info["flaw"]["centre"]
    r = np.hypot(X - cx, Y - cy)
    s = np.clip((0.2 - r) / 0.1, 0.0, 1.0)            # 1 inside r <= 0.1, 0 beyond 0.2
    mins = {}
    for f in (1e-3, 1e-2):
        rho = np.exp(np.log(f) * s)
        m = fwi.build_model(w.mesh, w.n_r, 1.0, rho, w.dt, static=True)
        fs = bruteforce.FullSystem(w.mesh, w.n_r, 1.0, m.rho_nodal, w.dt, static=True)
        vals = sla.eigvals(fs.matrix.toarray(), fs.mass.toarray())
        mins[f] = (-vals[np.isfinite(vals)]).real.min()
    assert mins[1e-3] < -1e3
    assert mins[1e-2] > -1e-6
