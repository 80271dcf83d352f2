"""Serving engine (harness) with continuous batching over library sessions.

Requests share sessions per model: each is a slot (a shot column) admitted at a window
boundary while the other slots keep running.  Checked: requests are admitted while others
are in flight, forward traces and gradients equal the same shot run alone through
sbfwi_forward / sbfwi_adjoint_gradient (1e-13), and a memory budget bounds the requests
in flight."""

import numpy as np
import pytest

from sbfwi_inputs import structured_mesh, boundary_nodes, ricker, flawed_density_circle

pytestmark = pytest.mark.gpu


def _setup(lib, n_req=12, seed=4):
    from paper_2501_06748_gb300 import serving
    meshes = {}

    def build(key):
        nx, p, n_r, s = key
        if (nx, p, n_r) not in meshes:
            meshes[(nx, p, n_r)] = lib.Mesh.from_inputs(structured_mesh(nx, nx, p), n_r)
        rho, _ = flawed_density_circle(32, 32, radius=0.12, factor=0.5, seed=s)
        return lib.Model(meshes[(nx, p, n_r)], 1.0, rho, 0.5 / (nx * p))

    keys = [(4, 2, 6, 0), (3, 3, 5, 1)]
    rng = np.random.default_rng(seed)
    reqs = []
    for rid in range(n_req):
        key = keys[rid % 2]
        nx, p = key[0], key[1]
        mesh = structured_mesh(nx, nx, p)
        top = boundary_nodes(mesh, "top")
        recs = np.array(boundary_nodes(mesh, "bottom")[:3], dtype=np.int64)
        dt = 0.5 / (nx * p)
        K = 40 + 13 * (rid % 5)                  # uneven lengths: slots free up at different windows
        wav = ricker(1.0 / (10 / (nx * p)), dt, K)
        obs = 0.01 * rng.standard_normal((recs.size, K)) if rid % 3 == 0 else None
        reqs.append(serving.Request(rid, key, int(rng.choice(top)), wav, recs, arrival=0.0, observed=obs))
    return serving, build, reqs


def _solo(lib, build, r):
    md = build(r.model_key)
    if r.observed is None:
        tr, _ = lib.forward(md, [r.src_node], r.wavelet[None], r.rec_nodes, keep=False)
        return tr[0], None, None
    tr, st = lib.forward(md, [r.src_node], r.wavelet[None], r.rec_nodes)
    E, res = lib.misfit(tr, r.observed[None], md.dt)
    return tr[0], E, lib.adjoint_gradient(md, st, res)


def test_requests_join_running_sessions_and_match_solo_runs(lib):
    serving, build, reqs = _setup(lib)
    eng = serving.Engine(build, max_batch=2, window=8)
    eng.run(reqs)
    assert all(r.done >= 0 for r in reqs)
    # with two slots per session and uneven lengths, requests enter while another is mid-flight
    joined = [r for r in reqs if r.admitted_at[0] > 0 and r.admitted_at[1] > 0]
    assert joined, [r.admitted_at for r in reqs]
    assert max(eng.batches) == 2
    for r in reqs:
        tr, E, g = _solo(lib, build, r)
        assert np.abs(tr).max() > 0
        np.testing.assert_allclose(r.traces, tr, rtol=0, atol=1e-13 * np.abs(tr).max())
        if r.observed is not None:
            assert r.misfit == pytest.approx(E, rel=1e-13)
            assert np.linalg.norm(r.gradient - g) <= 1e-13 * np.linalg.norm(g)
    st = serving.latency_stats(reqs)
    assert 0 <= st["p50_s"] <= st["p99_s"]


def test_staggered_arrivals_are_admitted_between_windows(lib):
    """Requests arriving on the engine's clock while others run are admitted at the next
    window of their session."""
    serving, build, reqs = _setup(lib, n_req=8, seed=9)
    for k, r in enumerate(reqs):
        r.arrival = 0.004 * k
    eng = serving.Engine(build, max_batch=4, window=4)
    eng.run(reqs)
    assert all(r.done >= r.arrival for r in reqs)
    for r in reqs:
        tr, _, g = _solo(lib, build, r)
        np.testing.assert_allclose(r.traces, tr, rtol=0, atol=1e-13 * np.abs(tr).max())
        if g is not None:
            assert np.linalg.norm(r.gradient - g) <= 1e-13 * np.linalg.norm(g)


def test_memory_budget_bounds_the_requests_in_flight(lib):
    serving, build, reqs = _setup(lib, n_req=10, seed=2)
    reqs = [r for r in reqs if r.model_key == reqs[0].model_key]      # one model, equal lengths,
    for r in reqs:                                                     # every request keeps a field
        r.wavelet = r.wavelet[:40].copy()
        r.observed = np.zeros((r.rec_nodes.size, r.K))
    stride = lib.Session(build(reqs[0].model_key), lib.SESSION_FORWARD, 1, reqs[0].rec_nodes, 4).field_stride
    need = serving.request_bytes(stride, reqs[0])
    eng = serving.Engine(build, max_batch=4, window=8, mem_budget=2 * need)
    eng.run(reqs)
    assert all(r.done >= 0 for r in reqs)
    assert eng.max_in_flight <= 2
    # slots are reused: every later request starts from a clean slot
    for r in reqs:
        tr, _, g = _solo(lib, build, r)
        np.testing.assert_allclose(r.traces, tr, rtol=0, atol=1e-13 * np.abs(tr).max())
        assert np.linalg.norm(r.gradient - g) <= 1e-13 * np.linalg.norm(g)
