"""3-D hexahedral S-elements: the GPU path vs the CPU oracle (``oracle.sbfem3d``) through the
C ABI (sbfwi_build_mesh3d, sbfwi_set_model3d).

Tolerances as for the 2-D path: relative L2 1e-10 on receiver traces, 1e-8 on the
gradient.  Cases span several elements per direction, a ragged element count per axis,
both face orders (n_b 8 on the one-tile and 26 on the two-tile tensor-core kernel), 5
shots (a partial shot tile), grid and nodal densities.
"""

import numpy as np
import pytest

from oracle import fwi
from sbfwi_inputs import ricker
from sbfwi_inputs.mesh3d import structured_mesh3d, boundary_nodes3d, nearest_node3d, flawed_density_sphere

pytestmark = pytest.mark.gpu

TRACE_TOL = 1e-10
GRAD_TOL = 1e-8


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _case(nx, ny, nz, p, n_r, shots, K, seed=0):
    mesh = structured_mesh3d(nx, ny, nz, p, lx=1.0, ly=0.9, lz=1.1)
    rho, _ = flawed_density_sphere(10, 9, 11, lx=1.0, ly=0.9, lz=1.1, radius=0.2, factor=0.5, seed=seed)
    h = min(1.0 / nx, 0.9 / ny, 1.1 / nz) / p
    dt = 0.4 * h
    top = boundary_nodes3d(mesh, "z1")
    rng = np.random.default_rng(seed)
    src = np.array([int(s) for s in rng.choice(top, size=shots, replace=False)], dtype=np.int64)
    rec = np.array(sorted(set(int(nearest_node3d(mesh, boundary_nodes3d(mesh, side), c))
                              for side, c in (("z0", (0.3, 0.4, 0.0)), ("z0", (0.7, 0.5, 0.0)),
                                              ("x0", (0.0, 0.45, 0.5)), ("y1", (0.5, 0.9, 0.6))))), dtype=np.int64)
    wav = np.stack([ricker(1.0 / (6 * h), dt, K) * (1.0 + 0.1 * s) for s in range(shots)])
    return mesh, rho, dt, src, rec, wav, n_r


@pytest.mark.parametrize("shape", [(2, 2, 2, 2, 6, 2, 60), (3, 2, 2, 1, 5, 5, 80)])
def test_forward_traces_3d(lib, shape):
    mesh, rho, dt, src, rec, wav, n_r = _case(*shape)
    M = lib.Mesh.from_inputs(mesh, n_r)
    md = lib.Model(M, 1.0, rho, dt, lx=1.0, ly=0.9, lz=1.1)
    tr, _ = lib.forward(md, src, wav, rec, keep=False)
    om = fwi.build_model3d(mesh, n_r, 1.0, rho, dt)
    to, _, _ = fwi.forward(om, src, wav, rec, keep=False)
    assert np.abs(to).max() > 0
    assert rel(tr, to) <= TRACE_TOL


@pytest.mark.parametrize("rho_kind", ["grid", "nodal"])
def test_misfit_and_gradient_3d(lib, rho_kind):
    mesh, rho, dt, src, rec, wav, n_r = _case(2, 2, 2, 2, 6, 3, 50, seed=1)
    rho0 = np.ones_like(rho)
    om_true = fwi.build_model3d(mesh, n_r, 1.0, rho, dt)
    obs, _, _ = fwi.forward(om_true, src, wav, rec, keep=False)
    om = fwi.build_model3d(mesh, n_r, 1.0, rho0, dt)
    M = lib.Mesh.from_inputs(mesh, n_r)
    if rho_kind == "grid":
        md = lib.Model(M, 1.0, rho0, dt, lx=1.0, ly=0.9, lz=1.1)
    else:
        md = lib.Model(M, 1.0, om.rho_nodal, dt, rho_kind=lib.RHO_NODAL)
    tr, st = lib.forward(md, src, wav, rec)
    to, store, _ = fwi.forward(om, src, wav, rec)
    assert rel(tr, to) <= TRACE_TOL
    E, res = lib.misfit(tr, obs, dt)
    Eo, reso = fwi.misfit(to, obs, dt)
    assert Eo > 0 and abs(E - Eo) <= 1e-10 * abs(Eo)
    g = lib.adjoint_gradient(md, st, res)
    go = fwi.adjoint_gradient(om, store, reso, rec)
    if rho_kind == "grid":
        go = fwi.gradient_to_grid3d(om, go, 10, 9, 11)
    assert g.shape == go.shape
    assert rel(g, go) <= GRAD_TOL


def test_3d_schedules_and_kernels_agree(lib):
    mesh, rho, dt, src, rec, wav, n_r = _case(2, 3, 2, 2, 6, 4, 40, seed=2)
    M = lib.Mesh.from_inputs(mesh, n_r)
    md = lib.Model(M, 1.0, rho, dt, lx=1.0, ly=0.9, lz=1.1)
    out = {}
    for el in (lib.ELEMENT_TENSOR, lib.ELEMENT_FP64):
        for so in (lib.SOLVE_DATAFLOW, lib.SOLVE_BARRIER, lib.SOLVE_LEVELS):
            lib.set_schedule(md, el, so)
            out[(el, so)], _ = lib.forward(md, src, wav, rec, keep=False)
    for el in (lib.ELEMENT_TENSOR, lib.ELEMENT_FP64):
        assert np.array_equal(out[(el, lib.SOLVE_DATAFLOW)], out[(el, lib.SOLVE_BARRIER)])
        assert np.array_equal(out[(el, lib.SOLVE_DATAFLOW)], out[(el, lib.SOLVE_LEVELS)])
    a, b = out[(lib.ELEMENT_TENSOR, lib.SOLVE_DATAFLOW)], out[(lib.ELEMENT_FP64, lib.SOLVE_DATAFLOW)]
    assert rel(a, b) <= 1e-12


def test_3d_refuses_what_is_built_for_2d_only(lib):
    mesh, rho, dt, *_ = _case(2, 2, 2, 1, 5, 1, 10)
    M = lib.Mesh.from_inputs(mesh, 5)
    md = lib.Model(M, 1.0, rho, dt, lx=1.0, ly=0.9, lz=1.1)
    with pytest.raises(lib.SbfwiError) as ei:
        lib.set_gradient_mode(md, lib.GRAD_EXACT)
    assert ei.value.code == lib.EUNSUPPORTED
    with pytest.raises(ValueError):
        lib.Model(M, 1.0, rho, dt, lfe=True)


def test_3d_checkpoints_and_sessions_match_the_plain_path(lib):
    """The memory strategies and the continuous-batching sessions are dimension-blind: on a
    3-D model the checkpointed adjoint is bit for bit the stored-field one, and a shot run as
    a session slot gives the traces and gradient of the same shot run alone."""
    import torch
    mesh, rho, dt, src, rec, wav, n_r = _case(2, 2, 2, 2, 6, 2, 40, seed=3)
    M = lib.Mesh.from_inputs(mesh, n_r)
    md = lib.Model(M, 1.0, rho, dt, lx=1.0, ly=0.9, lz=1.1)
    rng = np.random.default_rng(4)
    res = rng.standard_normal((len(src), len(rec), wav.shape[1]))
    t0, s0 = lib.forward(md, src, wav, rec, ckpt_every=0)
    g0 = lib.adjoint_gradient(md, s0, res)
    for c in (1, 7, lib.CKPT_AUTO):
        t, s = lib.forward(md, src, wav, rec, ckpt_every=c)
        assert np.array_equal(t, t0), c
        assert np.array_equal(lib.adjoint_gradient(md, s, res), g0), c
    # one shot through a forward and an adjoint session
    dev = torch.device("cuda", 0)
    t1, s1 = lib.forward(md, src[:1], wav[:1], rec)
    g1 = lib.adjoint_gradient(md, s1, res[:1])
    fs = lib.Session(md, lib.SESSION_FORWARD, 2, rec, 8)
    K = wav.shape[1]
    field = torch.empty((K, fs.field_stride), dtype=torch.float64, device=dev)
    fs.admit(1, torch.tensor(wav[0], device=dev), src_node=int(src[0]), field=field)
    done = []
    while not done:
        done = fs.step()
    tr = fs.collect(1).cpu().numpy()
    assert np.abs(tr - t1[0]).max() <= 1e-13 * np.abs(t1).max()
    adj = lib.Session(md, lib.SESSION_ADJOINT, 2, rec, 8)
    adj.admit(0, torch.tensor(res[0], device=dev), field=field)
    done = []
    while not done:
        done = adj.step()
    g = adj.collect(0).cpu().numpy()
    assert g.shape == g1.shape
    assert np.linalg.norm(g - g1) <= 1e-13 * np.linalg.norm(g1)
