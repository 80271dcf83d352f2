"""Checkpoint-and-recompute memory strategy for the adjoint (the alternative to
storing the forward field, Section 4): traces and gradient must be bit for bit
those of the stored-field run, for every checkpoint interval and both element
kernels; the oracle pins the stored-field run."""

import numpy as np
import pytest

from oracle import fwi
from test_gpu_parity import _ragged_case, rel, GRAD_TOL, TRACE_TOL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ragged(lib):
    mesh, rho, srcs, recs, wav, dt = _ragged_case()
    M = lib.Mesh.from_inputs(mesh, 6)
    md = lib.Model(M, 1.3, rho, dt, lx=1.2, ly=1.0)
    rng = np.random.default_rng(5)
    res = rng.standard_normal((len(srcs), len(recs), wav.shape[1]))
    return md, srcs, recs, wav, res


@pytest.mark.parametrize("element", ["tc", "fp64"])
def test_checkpointed_gradient_is_bitwise_the_stored_field_gradient(lib, ragged, monkeypatch, element):
    md, srcs, recs, wav, res = ragged
    if element == "fp64":
        monkeypatch.setenv("SBFWI_ELEMENT", "fp64")
    t0, s0 = lib.forward(md, srcs, wav, recs, ckpt_every=0)
    g0 = lib.adjoint_gradient(md, s0, res)
    K = wav.shape[1]
    for c in (1, 7, 13, K - 1, K, K + 5, lib.CKPT_AUTO):
        t, s = lib.forward(md, srcs, wav, recs, ckpt_every=c)
        assert np.array_equal(t, t0), c
        g = lib.adjoint_gradient(md, s, res)
        assert np.array_equal(g, g0), c
        # the state can be used again
        assert np.array_equal(lib.adjoint_gradient(md, s, res), g0), c


def test_checkpointed_gradient_matches_the_oracle(lib):
    mesh, rho, srcs, recs, wav, dt = _ragged_case()
    M = lib.Mesh.from_inputs(mesh, 6)
    md = lib.Model(M, 1.3, rho, dt, lx=1.2, ly=1.0)
    tr, st = lib.forward(md, srcs, wav, recs, ckpt_every=9)
    om = fwi.build_model(mesh, 6, 1.3, rho, dt, lx=1.2, ly=1.0)
    to, store, _ = fwi.forward(om, srcs, wav, recs)
    assert rel(tr, to) <= TRACE_TOL
    res = -to
    g = lib.adjoint_gradient(md, st, res)
    go = fwi.gradient_to_grid(om, fwi.adjoint_gradient(om, store, res, recs), rho.shape[1], rho.shape[0], 1.2, 1.0)
    assert rel(g, go) <= GRAD_TOL


def test_checkpoints_from_the_other_element_kernel_are_refused(lib, ragged, monkeypatch):
    md, srcs, recs, wav, res = ragged
    _, s = lib.forward(md, srcs, wav, recs, ckpt_every=10)
    monkeypatch.setenv("SBFWI_ELEMENT", "fp64")
    with pytest.raises(lib.SbfwiError) as ei:
        lib.adjoint_gradient(md, s, res)
    assert ei.value.code == lib.ESTATE


def test_negative_interval_is_rejected(lib, ragged):
    md, srcs, recs, wav, res = ragged
    with pytest.raises(lib.SbfwiError) as ei:
        lib.forward(md, srcs, wav, recs, ckpt_every=-2)
    assert ei.value.code == lib.EINVAL


def test_cached_store_gives_identical_results(lib, ragged):
    """A destroyed forward state leaves its store in the library's cache; the next
    forward state of the same size takes it over.  Results do not depend on it."""
    md, srcs, recs, wav, res = ragged
    lib.release_cache()
    t1, s1 = lib.forward(md, srcs, wav, recs)
    g1 = lib.adjoint_gradient(md, s1, res)
    del s1                                   # store goes to the cache
    t2, s2 = lib.forward(md, srcs, wav, recs)  # takes it over
    g2 = lib.adjoint_gradient(md, s2, res)
    assert np.array_equal(t1, t2) and np.array_equal(g1, g2)
    del s2
    lib.release_cache()
    t3, s3 = lib.forward(md, srcs, wav, recs, ckpt_every=5)
    assert np.array_equal(t3, t1)
    assert np.array_equal(lib.adjoint_gradient(md, s3, res), g1)


def test_differentiation_recipe_at_full_size(lib):
    """The differentiation recipe at its full mesh size (128 x 128 elements, p = 4, N_r = 32,
    512^2 grid) in the benchmark's launch configuration (8 shots per pass), 24 steps:
    properties that hold at any size -- the checkpointed adjoint gradient is bitwise the
    stored-field one, traces are exactly linear in the wavelets (scaling by 2), and one
    shot alone gives its traces in the batch to rounding."""
    from sbfwi_inputs import diff_workload
    w = diff_workload(K=24)
    src, wav = w.src_nodes[:8], w.wavelets[:8]
    M = lib.Mesh.from_inputs(w.mesh, w.n_r)
    md = lib.Model(M, w.c, w.rho_start, w.dt)
    tr, st = lib.forward(md, src, wav, w.rec_nodes)
    assert np.abs(tr).max() > 0
    res = -tr
    g_store = lib.adjoint_gradient(md, st, res)
    tr_c, st_c = lib.forward(md, src, wav, w.rec_nodes, ckpt_every=lib.CKPT_AUTO)
    assert np.array_equal(tr, tr_c)
    g_ckpt = lib.adjoint_gradient(md, st_c, res)
    assert np.array_equal(g_store, g_ckpt)
    tr2, _ = lib.forward(md, src, 2.0 * wav, w.rec_nodes, keep=False)
    assert np.array_equal(tr2, 2.0 * tr)
    tr1, _ = lib.forward(md, src[3:4], wav[3:4], w.rec_nodes, keep=False)
    assert np.linalg.norm(tr1[0] - tr[3]) <= 1e-13 * np.linalg.norm(tr[3])
