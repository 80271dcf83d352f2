"""Schedules of the time loop (element kernel x global-solve schedule) chosen through the
C ABI, and the autotuner that times them: every schedule computes the same traces,
the choice is checked against the shapes, and the autotuner keeps a valid fastest one."""

import numpy as np
import pytest

from oracle import fwi, uneven
from sbfwi_inputs import boundary_nodes, min_spacing, nearest_node, quadtree_mesh, ricker

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def _problem(p=3, shots=3, K=30):
    m = quadtree_mesh(4, 1, lambda x0, y0, x1, y1, lvl: x0 < 0.5 and y0 < 0.5, p)
    rho = 0.8 + 0.4 * np.random.default_rng(5).random((17, 17))
    s = min_spacing(m)
    dt, f0 = 0.5 * s, 1.0 / (10 * s)
    top = boundary_nodes(m, "top")
    src = np.array([nearest_node(m, top, ((k + 0.5) / shots, 1.0)) for k in range(shots)])
    wav = np.stack([ricker(f0, dt, K, t0=(1.1 + 0.1 * k) / f0) for k in range(shots)])
    rec = boundary_nodes(m, "bottom")[::2]
    return m, rho, dt, src, wav, rec


def test_every_schedule_gives_the_same_traces(lib):
    """Quadtree of order 3 (n_b 12, 15 padded to 15): both element kernels under all
    three solve schedules; one element kernel gives bitwise the same traces under every
    solve schedule, and the kernels agree within 1e-12."""
    m, rho, dt, src, wav, rec = _problem()
    M = lib.Mesh.from_inputs(m, 5)
    md = lib.Model(M, 1.0, rho, dt)
    out = {}
    for e in (lib.ELEMENT_TENSOR, lib.ELEMENT_FP64):
        for s in (lib.SOLVE_DATAFLOW, lib.SOLVE_BARRIER, lib.SOLVE_LEVELS):
            lib.set_schedule(md, e, s)
            out[(e, s)], _ = lib.forward(md, src, wav, rec, keep=False)
    for e in (lib.ELEMENT_TENSOR, lib.ELEMENT_FP64):
        assert np.array_equal(out[(e, lib.SOLVE_DATAFLOW)], out[(e, lib.SOLVE_BARRIER)])
        assert np.array_equal(out[(e, lib.SOLVE_DATAFLOW)], out[(e, lib.SOLVE_LEVELS)])
    assert rel(out[(lib.ELEMENT_TENSOR, 1)], out[(lib.ELEMENT_FP64, 1)]) <= 1e-12


def test_tensor_kernel_on_request_where_the_default_is_mixed(lib):
    """Padded n_b = 18 runs the mixed kernels by default (n_b <= 16 on the one-tile
    tensor-core kernel, the n_b = 18 elements on FP64); asking for the two-tile tensor-core
    kernel prepares its operator digits on first use, and both match the oracle."""
    m = quadtree_mesh(4, 1, lambda x0, y0, x1, y1, lvl: x0 < 0.25 or y0 < 0.25, 3)    # corner cell: n_b 18
    assert m.n_b.max() == 18
    _, rho, dt, src, wav, rec = _problem()
    om = uneven.build_model(m, 5, 1.0, rho, dt)
    to, _, _ = uneven.forward(om, src, wav, rec, keep=False)
    M = lib.Mesh.from_inputs(m, 5)
    md = lib.Model(M, 1.0, rho, dt)
    tr_auto, _ = lib.forward(md, src, wav, rec, keep=False)
    lib.set_schedule(md, lib.ELEMENT_TENSOR)
    tr_tc, _ = lib.forward(md, src, wav, rec, keep=False)
    assert rel(tr_auto, to) <= 1e-10 and rel(tr_tc, to) <= 1e-10
    assert not np.array_equal(tr_auto, tr_tc)          # a different kernel ran


def test_schedule_errors(lib):
    m, rho, dt, src, wav, rec = _problem()
    M = lib.Mesh.from_inputs(m, 5)
    md = lib.Model(M, 1.0, rho, dt)
    with pytest.raises(lib.SbfwiError) as ei:
        lib.set_schedule(md, 7, 0)
    assert ei.value.code == lib.EINVAL
    with pytest.raises(lib.SbfwiError) as ei:
        lib.set_schedule(md, 0, 9)
    assert ei.value.code == lib.EINVAL
    lib.set_schedule(md, lib.ELEMENT_TENSOR)               # nine shots: no tensor-core kernel
    src9 = np.resize(src, 9)
    wav9 = np.resize(wav, (9, wav.shape[1]))
    with pytest.raises(lib.SbfwiError) as ei:
        lib.forward(md, src9, wav9, rec, keep=False)
    assert ei.value.code == lib.EUNSUPPORTED
    # checkpoints written by one element kernel cannot feed an adjoint on the other
    lib.set_schedule(md, lib.ELEMENT_TENSOR)
    tr, st = lib.forward(md, src, wav, rec, ckpt_every=7)
    lib.set_schedule(md, lib.ELEMENT_FP64)
    with pytest.raises(lib.SbfwiError) as ei:
        lib.adjoint_gradient(md, st, -tr)
    assert ei.value.code == lib.ESTATE


def test_autotuner_keeps_a_valid_fastest_schedule(lib):
    from paper_2501_06748_gb300 import autotune
    m, rho, dt, src, wav, rec = _problem()
    M = lib.Mesh.from_inputs(m, 5)
    md = lib.Model(M, 1.0, rho, dt)
    ref, _ = lib.forward(md, src, wav, rec, keep=False)
    choice = autotune.tune(md, src, wav, rec, steps=8, repeats=2)
    assert len(choice["candidates"]) == 9
    times = [c["s_per_step"] for c in choice["candidates"] if c["s_per_step"] is not None]
    # padded n_b 15: every element fits one tile, so the mixed kernels do not apply
    assert len(times) == 6 and choice["s_per_step"] == min(times)
    assert all(c["s_per_step"] is None for c in choice["candidates"] if c["element"] == "mixed")
    tr, _ = lib.forward(md, src, wav, rec, keep=False)
    assert rel(tr, ref) <= 1e-12


def test_mixed_element_kernels_on_uneven_elements(lib):
    """A quadtree whose corner cells have n_b = 18 (the rest 12 and 15): the elements of
    n_b <= 16 run the one-tile tensor-core kernel and the others the FP64 kernel, two
    launches per step over element lists.  Traces and gradient match the oracle (1e-10 /
    1e-8) and the all-FP64 run (1e-12); checkpointed = stored field bit for bit."""
    m = quadtree_mesh(4, 1, lambda x0, y0, x1, y1, lvl: x0 < 0.25 or y0 < 0.25, 3)
    nbs = m.n_b
    assert nbs.max() == 18 and (nbs <= 16).sum() > 0
    _, rho, dt, src, wav, rec = _problem()
    om = uneven.build_model(m, 5, 1.0, rho, dt)
    to, store, _ = uneven.forward(om, src, wav, rec)
    obs = 0.01 * np.random.default_rng(3).standard_normal(to.shape)
    Eo, reso = fwi.misfit(to, obs, dt)
    go = uneven.gradient_to_grid(om, uneven.adjoint_gradient(om, store, reso, rec), 17, 17)
    M = lib.Mesh.from_inputs(m, 5)
    md = lib.Model(M, 1.0, rho, dt)
    out = {}
    for e in (lib.ELEMENT_MIXED, lib.ELEMENT_FP64):
        lib.set_schedule(md, e)
        for c in (0, 7):
            tr, st = lib.forward(md, src, wav, rec, ckpt_every=c)
            _, res = lib.misfit(tr, obs, dt)
            out[(e, c)] = (tr, lib.adjoint_gradient(md, st, res))
    tr, g = out[(lib.ELEMENT_MIXED, 0)]
    assert rel(tr, to) <= 1e-10 and rel(g, go) <= 1e-8
    assert rel(tr, out[(lib.ELEMENT_FP64, 0)][0]) <= 1e-12
    assert not np.array_equal(tr, out[(lib.ELEMENT_FP64, 0)][0])          # the tensor cores ran
    assert np.array_equal(g, out[(lib.ELEMENT_MIXED, 7)][1])
    lib.set_schedule(md, lib.ELEMENT_AUTO)
    tr_auto, _ = lib.forward(md, src, wav, rec, keep=False)
    assert np.array_equal(tr_auto, tr)                                      # the default for padded n_b 18
