"""GPU path vs the CPU oracle, element by element, through the C ABI.

Tolerances are the ones the path is held to: relative L2 1e-10 on receiver
traces and 1e-8 on the gradient.
"""

import numpy as np
import pytest

from oracle import fwi
from sbfwi_inputs import structured_mesh, tiny_workload, size_workload, boundary_nodes, ricker

pytestmark = pytest.mark.gpu

TRACE_TOL = 1e-10
GRAD_TOL = 1e-8


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def tiny():
    return tiny_workload()


@pytest.fixture(scope="module")
def tiny_observed(tiny):
    """Observed data: the oracle on the same set-up with twice the elements and radial points."""
    wf = tiny_workload(refine=2)
    mt = fwi.build_model(wf.mesh, wf.n_r, wf.c, wf.rho_true, tiny.dt)
    d, _, _ = fwi.forward(mt, wf.src_nodes, wf.wavelets, wf.rec_nodes, keep=False)
    return d


def test_forward_traces_tiny_flawed_model(lib, tiny):
    w = tiny
    M = lib.Mesh.from_inputs(w.mesh, w.n_r)
    md = lib.Model(M, w.c, w.rho_true, w.dt)
    tr, _ = lib.forward(md, w.src_nodes, w.wavelets, w.rec_nodes, keep=False)
    om = fwi.build_model(w.mesh, w.n_r, w.c, w.rho_true, w.dt)
    to, _, _ = fwi.forward(om, w.src_nodes, w.wavelets, w.rec_nodes, keep=False)
    assert np.abs(to).max() > 0.1
    assert rel(tr, to) <= TRACE_TOL


@pytest.mark.parametrize("rho_kind", ["grid", "nodal"])
def test_misfit_and_gradient_tiny(lib, tiny, tiny_observed, rho_kind):
    w = tiny
    om = fwi.build_model(w.mesh, w.n_r, w.c, w.rho_start, w.dt)
    M = lib.Mesh.from_inputs(w.mesh, w.n_r)
    if rho_kind == "grid":
        md = lib.Model(M, w.c, w.rho_start, w.dt)
    else:
        md = lib.Model(M, w.c, om.rho_nodal, w.dt, rho_kind=lib.RHO_NODAL)
    tr, st = lib.forward(md, w.src_nodes, w.wavelets, w.rec_nodes)
    to, store, _ = fwi.forward(om, w.src_nodes, w.wavelets, w.rec_nodes)
    assert rel(tr, to) <= TRACE_TOL
    E, res = lib.misfit(tr, tiny_observed, w.dt)
    Eo, reso = fwi.misfit(to, tiny_observed, w.dt)
    assert abs(E - Eo) <= 1e-10 * abs(Eo)
    assert rel(res, reso) <= TRACE_TOL
    g = lib.adjoint_gradient(md, st, res)
    go = fwi.adjoint_gradient(om, store, reso, w.rec_nodes)
    if rho_kind == "grid":
        go = fwi.gradient_to_grid(om, go, w.gx, w.gy)
    assert g.shape == go.shape
    assert rel(g, go) <= GRAD_TOL


def _ragged_case():
    """6 x 5 elements of order 3 (n_b = 12), N_r = 6, five shots: odd tree splits,
    partial CTAs and task tails."""
    mesh = structured_mesh(6, 5, 3, lx=1.2, ly=1.0)
    rng = np.random.default_rng(7)
    gx, gy = 23, 17
    rho = 0.6 + 0.8 * rng.random((gy, gx))
    top = boundary_nodes(mesh, "top")
    srcs = rng.choice(top, size=5, replace=False)
    bnd = np.concatenate([boundary_nodes(mesh, s) for s in ("bottom", "left", "right")])
    recs = rng.choice(np.unique(bnd), size=7, replace=False)
    dt = 0.5 * 0.2 / 3
    K = 60
    wav = np.stack([ricker(1.0 / (10 * 0.2 / 3) * (1 + 0.1 * s), dt, K) for s in range(5)])
    return mesh, rho, srcs, recs, wav, dt


def test_ragged_multishot_forward_and_gradient(lib):
    mesh, rho, srcs, recs, wav, dt = _ragged_case()
    n_r = 6
    om = fwi.build_model(mesh, n_r, 1.3, rho, dt, lx=1.2, ly=1.0)
    to, store, _ = fwi.forward(om, srcs, wav, recs)
    M = lib.Mesh.from_inputs(mesh, n_r)
    md = lib.Model(M, 1.3, rho, dt, lx=1.2, ly=1.0)
    tr, st = lib.forward(md, srcs, wav, recs)
    assert rel(tr, to) <= TRACE_TOL
    rng = np.random.default_rng(3)
    res = rng.standard_normal(tr.shape)
    g = lib.adjoint_gradient(md, st, res)
    go = fwi.gradient_to_grid(om, fwi.adjoint_gradient(om, store, res, recs), rho.shape[1], rho.shape[0], 1.2, 1.0)
    assert rel(g, go) <= GRAD_TOL


def test_shots_are_independent_in_a_batch(lib):
    """A shot's traces are the same alone and inside a batch of five."""
    mesh, rho, srcs, recs, wav, dt = _ragged_case()
    M = lib.Mesh.from_inputs(mesh, 6)
    md = lib.Model(M, 1.3, rho, dt, lx=1.2, ly=1.0)
    tr, _ = lib.forward(md, srcs, wav, recs, keep=False)
    for s in (0, 3):
        t1, _ = lib.forward(md, srcs[s:s + 1], wav[s:s + 1], recs, keep=False)
        assert rel(t1[0], tr[s]) <= 1e-13


def test_device_and_host_memory_give_identical_results(lib, tiny):
    torch = pytest.importorskip("torch")
    w = tiny
    M = lib.Mesh.from_inputs(w.mesh, w.n_r)
    md_h = lib.Model(M, w.c, w.rho_true, w.dt)
    md_d = lib.Model(M, w.c, torch.tensor(w.rho_true, device="cuda"), w.dt)
    K = 50
    th, sh = lib.forward(md_h, w.src_nodes, w.wavelets[:, :K], w.rec_nodes)
    td, sd = lib.forward(md_d, w.src_nodes, torch.tensor(w.wavelets[:, :K], device="cuda"), w.rec_nodes)
    assert np.array_equal(th, td.cpu().numpy())
    gh = lib.adjoint_gradient(md_h, sh, th)
    gd = lib.adjoint_gradient(md_d, sd, td)
    assert np.array_equal(gh, gd.cpu().numpy())
    E, _ = lib.misfit(td, torch.zeros_like(td), w.dt)
    assert E == pytest.approx(0.5 * w.dt * float(np.sum(th * th)), rel=1e-13)


def test_errors_are_reported(lib, tiny):
    w = tiny
    M = lib.Mesh.from_inputs(w.mesh, w.n_r)
    with pytest.raises(lib.SbfwiError) as ei:
        lib.Model(M, w.c, -w.rho_true, w.dt)
    assert ei.value.code == lib.EINVAL
    md = lib.Model(M, w.c, w.rho_true, w.dt)
    with pytest.raises(lib.SbfwiError):
        lib.forward(md, [10_000], w.wavelets, w.rec_nodes)
    with pytest.raises(lib.SbfwiError):
        lib.forward(md, w.src_nodes, w.wavelets, [w.rec_nodes[0], w.rec_nodes[0]])
    tr, st = lib.forward(md, w.src_nodes, w.wavelets[:, :5], w.rec_nodes)
    with pytest.raises(lib.SbfwiError) as ei:       # the forward state was not kept for the exact adjoint
        lib.adjoint_gradient(md, st, tr, mode=lib.GRAD_EXACT)
    assert ei.value.code == lib.ESTATE
    with pytest.raises(lib.SbfwiError) as ei:
        lib.adjoint_gradient(md, st, tr, mode=5)
    assert ei.value.code == lib.EINVAL


@pytest.mark.slow
def test_full_size_workload_few_steps(lib):
    """The bench's workload and launch configuration (64x64 elements, p = 4, N_r = 32,
    8 shots in one pass) for 8 Newmark steps: traces on the flawed model and the
    gradient on the starting model, element by element against the oracle."""
    w = size_workload(K=8)
    M = lib.Mesh.from_inputs(w.mesh, w.n_r)
    md = lib.Model(M, w.c, w.rho_true, w.dt)
    tr, _ = lib.forward(md, w.src_nodes, w.wavelets, w.rec_nodes, keep=False)
    om = fwi.build_model(w.mesh, w.n_r, w.c, w.rho_true, w.dt)
    to, _, _ = fwi.forward(om, w.src_nodes, w.wavelets, w.rec_nodes, keep=False)
    assert np.abs(to).max() > 0
    assert rel(tr, to) <= TRACE_TOL
    m0 = lib.Model(M, w.c, w.rho_start, w.dt)
    t0, st = lib.forward(m0, w.src_nodes, w.wavelets, w.rec_nodes)
    o0 = fwi.build_model(w.mesh, w.n_r, w.c, w.rho_start, w.dt)
    to0, store, _ = fwi.forward(o0, w.src_nodes, w.wavelets, w.rec_nodes)
    assert rel(t0, to0) <= TRACE_TOL
    res = to - to0                          # residual: flawed minus starting model (oracle traces)
    g = lib.adjoint_gradient(m0, st, res)
    go = fwi.gradient_to_grid(o0, fwi.adjoint_gradient(o0, store, res, w.rec_nodes), w.gx, w.gy)
    assert rel(g, go) <= GRAD_TOL


@pytest.mark.parametrize("case", ["ragged", "size8"])
def test_dataflow_barrier_and_per_level_global_solves_agree(lib, monkeypatch, case):
    """The one-launch dataflow solve (default), the one-launch solve with grid barriers
    between levels and the one-launch-per-level solve give the same traces (same
    arithmetic, different launch structure)."""
    if case == "ragged":
        mesh, rho, srcs, recs, wav, dt = _ragged_case()
        n_r, c, lx, ly = 6, 1.3, 1.2, 1.0
    else:
        w = size_workload(K=8)
        mesh, rho, srcs, recs, wav, dt = w.mesh, w.rho_true, w.src_nodes, w.rec_nodes, w.wavelets, w.dt
        n_r, c, lx, ly = w.n_r, w.c, 1.0, 1.0
    M = lib.Mesh.from_inputs(mesh, n_r)
    md = lib.Model(M, c, rho, dt, lx=lx, ly=ly)
    t_flow, _ = lib.forward(md, srcs, wav, recs, keep=False)
    t_flow2, _ = lib.forward(md, srcs, wav, recs, keep=False)
    monkeypatch.setenv("SBFWI_SOLVE", "barrier")
    t_barrier, _ = lib.forward(md, srcs, wav, recs, keep=False)
    monkeypatch.setenv("SBFWI_SOLVE", "levels")
    t_levels, _ = lib.forward(md, srcs, wav, recs, keep=False)
    assert np.abs(t_flow).max() > 0
    assert np.array_equal(t_flow, t_flow2)
    assert np.array_equal(t_flow, t_barrier)
    assert np.array_equal(t_flow, t_levels)


@pytest.mark.parametrize("case", ["tiny", "ragged"])
def test_tensor_core_and_fp64_element_kernels_agree(lib, tiny, monkeypatch, case):
    """The element step on the FP16 tensor cores (error-free digit splitting) and the
    FP64 element step give the same traces and gradient to FP64 rounding."""
    if case == "tiny":
        w = tiny
        mesh, rho, srcs, recs, wav, dt, c, lx, ly, n_r = (w.mesh, w.rho_true, w.src_nodes, w.rec_nodes,
                                                          w.wavelets, w.dt, w.c, 1.0, 1.0, w.n_r)
    else:
        mesh, rho, srcs, recs, wav, dt = _ragged_case()
        c, lx, ly, n_r = 1.3, 1.2, 1.0, 6
    M = lib.Mesh.from_inputs(mesh, n_r)
    md = lib.Model(M, c, rho, dt, lx=lx, ly=ly)
    t_tc, s_tc = lib.forward(md, srcs, wav, recs)
    g_tc = lib.adjoint_gradient(md, s_tc, t_tc)
    monkeypatch.setenv("SBFWI_ELEMENT", "fp64")
    t_64, s_64 = lib.forward(md, srcs, wav, recs)
    g_64 = lib.adjoint_gradient(md, s_64, t_64)
    assert rel(t_tc, t_64) <= 1e-12
    assert rel(g_tc, g_64) <= 1e-11
