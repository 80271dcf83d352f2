"""Pins of the oracle's 3-D scaled-boundary elements (``oracle.sbfem3d``; Section 3 carried to
a boundary surface).

Each test checks the oracle against something other than itself:

* the face rule integrates the degree it is chosen for, and the boundary Jacobian sums
  to three times the element's volume (divergence theorem);
* the coefficient matrices annihilate constants where the continuous operators do, and
  1^T M0 1 = 3 rho V;
* the static condensed stiffness annihilates constants and maps the nodal values of a
  linear field to the consistent boundary flux of that field (exact up to the zero-flux
  condition on the tiny sphere xi0 around the scaling centre), which the 2-D radial
  coefficients would miss by O(1);
* free-vibration frequencies of a homogeneous cube against the Neumann Laplacian closed
  form, exactly degenerate where the cube's symmetry makes them so, converging with p;
* the frequency shift alpha^2/4 of an exponentially graded density (closed form), which
  exercises the d/dxi E terms;
* the condensed time loop against the brute-force uncondensed solve;
* the trilinear density map against linear reproduction and its transpose.
"""

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import bruteforce, fwi, sbfem, sbfem3d
from sbfwi_inputs.mesh3d import structured_mesh3d, boundary_nodes3d, nearest_node3d
from sbfwi_inputs import ricker


def _skewed(nx, p):
    """A structured mesh under an affine map (planar parallelogram faces, skewed cells)."""
    m = structured_mesh3d(nx, nx, nx, p)
    A = np.array([[1.0, 0.2, 0.1], [0.0, 0.9, 0.15], [0.05, 0.0, 1.1]])
    m.node_xyz = m.node_xyz @ A.T
    m.centre_xyz = m.centre_xyz @ A.T
    return m, abs(np.linalg.det(A))


def _f64(*a):
    return [np.asarray(x, dtype=np.float64) for x in a]


@pytest.mark.parametrize("p", [1, 2, 3])
def test_face_rule_exact_and_jacobian_volume(p):
    eta, zeta, w, N, Ne, Nz = _f64(*sbfem3d.face_rule(p))
    # exact for eta^a zeta^b, a, b <= 3p + 2
    for a in range(3 * p + 3):
        for b in (0, 3 * p + 2):
            ex = (1 - (-1) ** (a + 1)) / (a + 1) * (1 - (-1) ** (b + 1)) / (b + 1)
            assert abs(np.sum(w * eta ** a * zeta ** b) - ex) < 1e-13
    # partition of unity of the face shape functions
    assert np.allclose(N.sum(1), 1.0) and np.allclose(Ne.sum(1), 0.0) and np.allclose(Nz.sum(1), 0.0)
    m, detA = _skewed(1, p)
    el = sbfem3d.elements_from_mesh3d(m)[0]
    tot = 0.0
    for f in el.faces:
        _, det, _, _, _ = sbfem3d.face_geometry(m.node_xyz[f], el.centre, N, Ne, Nz)
        assert det.min() > 0
        tot += float(np.sum(w * det))
    assert abs(tot - 3 * detA) < 1e-13


@pytest.mark.parametrize("p", [1, 2])
def test_coefficient_matrix_identities_3d(p):
    m, detA = _skewed(1, p)
    el = sbfem3d.elements_from_mesh3d(m)[0]
    nb = el.dofs.size
    rng = np.random.default_rng(p)
    rho = 0.5 + rng.random((3, nb))
    E0, E1, E2, M0 = _f64(*sbfem3d.coefficient_matrices3d(el, m.node_xyz, p, 1.3, rho))
    one = np.ones(nb)
    for k in range(3):
        assert np.abs(E1[k].T @ one).max() < 1e-13 * np.abs(E1[k]).max()
        assert np.abs(E2[k] @ one).max() < 1e-13 * np.abs(E2[k]).max()
        for A in (E0[k], E2[k], M0[k]):
            assert np.allclose(A, A.T, atol=1e-15 * np.abs(A).max())
        assert np.linalg.eigvalsh(E0[k]).min() > 0 and np.linalg.eigvalsh(M0[k]).min() > 0
    # homogeneous: 1^T M0 1 = int rho det J_b = 3 rho V; c^2 scales E0..E2 only
    E0h, _, _, M0h = _f64(*sbfem3d.coefficient_matrices3d(el, m.node_xyz, p, 1.0, np.full((1, nb), 2.5)))
    assert abs(one @ M0h[0] @ one - 3 * 2.5 * detA) < 1e-13
    E0c, _, _, M0c = _f64(*sbfem3d.coefficient_matrices3d(el, m.node_xyz, p, 2.0, np.full((1, nb), 2.5)))
    assert np.allclose(E0c, 4 * E0h) and np.allclose(M0c, M0h)


def _linear_flux(m, el, p, rho, d):
    """int_faces N rho c^2 n_d dA (c = 1) by the face rule, independent of the E-matrices."""
    _, _, w, N, Ne, Nz = _f64(*sbfem3d.face_rule(p))
    f = np.zeros(el.dofs.size)
    for fc, loc in zip(el.faces, el.face_local):
        X = m.node_xyz[fc]
        nA = np.cross(Ne @ X, Nz @ X)
        f[loc] += (N * (w * nA[:, d] * rho)[:, None]).sum(0)
    return f


@pytest.mark.parametrize("p", [1, 2])
def test_static_stiffness_constants_and_linear_flux(p):
    m, _ = _skewed(2, p)
    md = fwi.build_model3d(m, 8, 1.0, np.full((6, 6, 6), 1.7), 1.0, static=True)
    one = np.ones(md.S.shape[1])
    for S in md.S:
        assert np.abs(S @ one).max() < 1e-11 * np.abs(S).max()
    el = md.elements[0]
    S = md.S[0]
    for d in range(3):
        a = m.node_xyz[el.dofs, d] - el.centre[d]
        f = _linear_flux(m, el, p, 1.7, d)
        assert np.abs(S @ a - f).max() < 1e-5 * np.abs(f).max()
    # the 2-D radial coefficients on the same E-matrices miss the linear field by O(1)
    XP = sbfem.XP
    xi = sbfem.radial_grid(7, 1e-3, XP)
    Es = sbfem3d.coefficient_matrices3d(el, m.node_xyz, p, 1.0, np.full((8, el.dofs.size), 1.7))
    Es = [np.asarray(E)[None] for E in Es]
    S2 = np.asarray(sbfem.condense(sbfem.element_system(*Es, xi, 1.0, 0.25, static=True, dim=2)).S[0], dtype=float)
    a = m.node_xyz[el.dofs, 0] - el.centre[0]
    f = _linear_flux(m, el, p, 1.7, 0)
    assert np.abs(S2 @ a - f).max() > 1e-2 * np.abs(f).max()


def _dense_frequencies(fs, count):
    """Smallest ``count`` omega of Omega x = -omega^2 M x by a dense QZ (the pencil is
    nonsymmetric, and shift-invert Arnoldi splits its degenerate eigenvalues)."""
    v = sla.eig(fs.matrix.toarray(), -fs.mass.toarray(), right=False)
    v = v[np.isfinite(v)]
    v = v[np.argsort(np.abs(v))][:count]
    assert np.abs(v.imag).max() < 1e-8 * np.abs(v).max()
    return np.sort(np.sqrt(np.abs(v.real)) * np.sign(v.real))


_FREQ = {}


def _cube_frequencies(p, alpha=0.0):
    key = (p, alpha)
    if key not in _FREQ:
        m = structured_mesh3d(2, 2, 2, p)
        els = sbfem3d.elements_from_mesh3d(m)
        pts, _ = sbfem3d.nodal_points3d(m, els, sbfem.radial_grid(5))
        fs = bruteforce.FullSystem(m, 6, 1.0, np.exp(alpha * np.asarray(pts[:, 0], dtype=float)), 1.0, static=True)
        _FREQ[key] = _dense_frequencies(fs, 11)
    return _FREQ[key]


def test_free_vibration_homogeneous_cube():
    """Neumann Laplacian on the unit cube: omega = pi sqrt(l^2 + m^2 + n^2): 0, pi (x3),
    pi sqrt 2 (x3), pi sqrt 3, 2 pi (x3)."""
    exact = np.pi * np.array([0, 1, 1, 1, np.sqrt(2), np.sqrt(2), np.sqrt(2), np.sqrt(3), 2, 2, 2])
    errs = []
    for p in (1, 2):
        om = _cube_frequencies(p)
        assert abs(om[0]) < 1e-4                             # omega^2 at rounding level
        for lo, hi in ((1, 4), (4, 7), (8, 11)):            # the symmetric triplets stay degenerate
            assert np.ptp(om[lo:hi]) < 1e-8 * om[lo]
        errs.append(np.abs(om[1:8] - exact[1:8]) / exact[1:8])
    assert errs[1].max() < 5e-3
    assert errs[1].max() < 0.2 * errs[0].max()


def test_free_vibration_graded_density_3d():
    """rho = exp(alpha x): omega^2 = (m pi)^2 + alpha^2/4 + (n pi)^2 + (l pi)^2 for m >= 1,
    (n pi)^2 + (l pi)^2 for m = 0.  The (1,0,0) mode moves by the alpha^2/4 term; measured
    against the same mesh's homogeneous (0,1,0) mode the discretisation error cancels."""
    alpha = 1.0
    om_h = _cube_frequencies(2)
    om = _cube_frequencies(2, alpha)
    # modes: 0, (0,1,0), (0,0,1) at pi (unmoved by the grading, up to a small fraction of
    # the 3e-3 discretisation error), (1,0,0) at sqrt(pi^2 + alpha^2/4)
    assert abs(om[1] - om_h[1]) < 1e-4 * om[1] and abs(om[2] - om_h[2]) < 1e-4 * om[2]
    shift_exact = np.sqrt(np.pi ** 2 + alpha ** 2 / 4) - np.pi
    assert abs((om[3] - om_h[1]) - shift_exact) < 0.02 * shift_exact
    # (0,1,1) at pi sqrt 2 unaffected; (1,1,0), (1,0,1) shifted
    assert abs(om[4] - om_h[4]) < 1e-4 * om[4]
    shift2 = np.sqrt(2 * np.pi ** 2 + alpha ** 2 / 4) - np.sqrt(2) * np.pi
    assert abs((om[5] - om_h[4]) - shift2) < 0.02 * shift2


def test_condensed_equals_bruteforce_3d():
    m = structured_mesh3d(2, 2, 2, 1)
    rng = np.random.default_rng(3)
    rho = 0.7 + 0.6 * rng.random((6, 6, 6))
    dt = 0.05
    md = fwi.build_model3d(m, 5, 1.0, rho, dt)
    src = [nearest_node3d(m, boundary_nodes3d(m, "z1"), (0.5, 0.5, 1.0))]
    rec = boundary_nodes3d(m, "z0")[:4]
    wav = ricker(2.0, dt, 60)[None]
    tr, _, st = fwi.forward(md, src, wav, rec, keep=False)
    fs = bruteforce.FullSystem(m, 5, 1.0, md.rho_nodal, dt)
    tb, sb = fs.forward(src, wav, rec)
    assert np.abs(tr).max() > 0
    assert np.linalg.norm(tb - tr) <= 1e-11 * np.linalg.norm(tr)
    assert np.linalg.norm(sb.u - st.u) <= 1e-11 * np.linalg.norm(st.u)


def test_trilinear_map_linear_reproduction_and_transpose():
    gx, gy, gz, lx, ly, lz = 7, 5, 6, 1.0, 0.8, 1.2
    xc = (np.arange(gx) + 0.5) * lx / gx
    yc = (np.arange(gy) + 0.5) * ly / gy
    zc = (np.arange(gz) + 0.5) * lz / gz
    Z, Y, X = np.meshgrid(zc, yc, xc, indexing="ij")
    lin = 0.3 + 1.1 * X - 0.7 * Y + 0.4 * Z
    rng = np.random.default_rng(5)
    pts = np.stack([rng.uniform(xc[0], xc[-1], 50), rng.uniform(yc[0], yc[-1], 50), rng.uniform(zc[0], zc[-1], 50)], 1)
    v = fwi.grid_to_points3d(lin, pts, lx, ly, lz)
    assert np.allclose(v, 0.3 + 1.1 * pts[:, 0] - 0.7 * pts[:, 1] + 0.4 * pts[:, 2], atol=1e-13)
    g = rng.standard_normal(50)
    r = rng.standard_normal((gz, gy, gx))
    lhs = np.dot(fwi.grid_to_points3d(r, pts, lx, ly, lz), g)
    rhs = np.sum(r * fwi.points_to_grid3d(g, pts, gx, gy, gz, lx, ly, lz))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def _lumped_nodal_volumes3d(m, mesh):
    """Volume each nodal point stands for: the face integrals of its shape function times
    det J_b, times the trapezoid weight of int xi^2 dxi at its radial point."""
    n, xi = m.n, m.xi
    h = xi[1] - xi[0]
    v = np.zeros(m.n_int + m.n_nodes)
    _, _, w, N, Ne, Nz = _f64(*sbfem3d.face_rule(mesh.p))
    for e, el in enumerate(m.elements):
        s = np.zeros(el.dofs.size)
        for f, loc in zip(el.faces, el.face_local):
            _, det, _, _, _ = sbfem3d.face_geometry(mesh.node_xyz[f], el.centre, N, Ne, Nz)
            s[loc] += N.T @ (w * det)
        for i in range(n):
            wi = xi[i] ** 2 * (h if i > 0 else h / 2)
            v[m.int_ptr[e] + i * el.dofs.size:m.int_ptr[e] + (i + 1) * el.dofs.size] = s * wi
        v[m.n_int + el.dofs] += s * xi[n] ** 2 * h / 2
    return v


@pytest.mark.slow
def test_kernel_matches_inertia_density_derivative_3d():
    """In 3-D as in 2-D: <a . g, drho> ~ dE/d(rho in M0) along smooth directions (within 8 %;
    measured 4 %), g the velocity part of the Frechet kernel on nodal points and a the volume
    each nodal point stands for; a wrong sign or a reversed time pairing fails this.  The
    agreement needs the wave resolved: at two nodes per wavelength (2 x 2 x 2 elements of
    order 2 at f0 = 2) the ratio is about 2, as it is in 2-D on equally coarse meshes."""
    m = structured_mesh3d(3, 3, 3, 2)            # about 4 nodes per dominant wavelength (f0 = 1.5)
    dt = 0.04
    rho_true = np.ones((8, 8, 8))
    rho_true[2:5, 3:6, 2:6] = 0.6
    src = [nearest_node3d(m, boundary_nodes3d(m, "z1"), (0.5, 0.5, 1.0))]
    rec = boundary_nodes3d(m, "z0")[::3]
    wav = ricker(1.5, dt, 75)[None]
    mt = fwi.build_model3d(m, 6, 1.0, rho_true, dt)
    d, _, _ = fwi.forward(mt, src, wav, rec, keep=False)
    m0 = fwi.build_model3d(m, 6, 1.0, np.ones((8, 8, 8)), dt)
    tr, store, _ = fwi.forward(m0, src, wav, rec)
    _, res = fwi.misfit(tr, d, dt)
    g = fwi.adjoint_gradient(m0, store, res, rec)
    a = _lumped_nodal_volumes3d(m0, m)
    assert abs(a.sum() - 1.0) < 2e-2

    def E_mass(rm):
        mm = fwi.build_model3d(m, 6, 1.0, np.ones((8, 8, 8)), dt, rho_mass_nodal=rm)
        t, _, _ = fwi.forward(mm, src, wav, rec, keep=False)
        return fwi.misfit(t, d, dt)[0]

    pts = m0.points
    for dirn in [np.ones(pts.shape[0]),
                 np.exp(-((pts[:, 0] - 0.5) ** 2 + (pts[:, 1] - 0.4) ** 2 + (pts[:, 2] - 0.6) ** 2) / 0.05)]:
        eps = 1e-5
        fd = (E_mass(1 + eps * dirn) - E_mass(1 - eps * dirn)) / (2 * eps)
        gk = np.sum(g * a * dirn)
        assert abs(gk / fd - 1.0) < 0.08, (gk, fd)
