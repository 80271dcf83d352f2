"""Serving engine (harness): batched forward requests return the traces of the
same shots run one by one, and every request is served."""

import numpy as np
import pytest

from sbfwi_inputs import structured_mesh, boundary_nodes, ricker, flawed_density_circle

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("budget_requests", [None, 2])
def test_batched_requests_match_single_shot_forwards(lib, budget_requests):
    """Results are the same alone and in the mix; with a memory budget of two requests'
    worth, no batch holds more than two."""
    from paper_2501_06748_gb300 import serving
    meshes = {}

    def build(key):
        nx, p, n_r, seed = key
        if (nx, p, n_r) not in meshes:
            meshes[(nx, p, n_r)] = lib.Mesh.from_inputs(structured_mesh(nx, nx, p), n_r)
        rho, _ = flawed_density_circle(32, 32, radius=0.12, factor=0.5, seed=seed)
        return lib.Model(meshes[(nx, p, n_r)], 1.0, rho, 0.5 / (nx * p))

    keys = [(4, 2, 6, 0), (3, 3, 5, 1)]
    rng = np.random.default_rng(4)
    reqs = []
    for rid in range(11):
        key = keys[rid % 2]
        nx, p = key[0], key[1]
        mesh = structured_mesh(nx, nx, p)
        top = boundary_nodes(mesh, "top")
        recs = np.array(boundary_nodes(mesh, "bottom")[:3], dtype=np.int64)
        dt = 0.5 / (nx * p)
        wav = ricker(1.0 / (10 / (nx * p)), dt, 40 + 10 * (rid % 2))
        reqs.append(serving.Request(rid, key, int(rng.choice(top)), wav, recs, arrival=0.0))
    budget = None
    if budget_requests:
        need = max(serving.request_bytes(build(r.model_key), r) for r in reqs)
        budget = budget_requests * need
    eng = serving.Engine(build, max_batch=4, mem_budget=budget)
    eng.run(reqs)
    assert all(r.done >= 0 for r in reqs)
    assert max(eng.batches) > 1 and sum(eng.batches) == len(reqs)
    if budget_requests:
        assert max(eng.batches) <= budget_requests
    for r in reqs:
        md = build(r.model_key)
        tr, _ = lib.forward(md, [r.src_node], r.wavelet[None], r.rec_nodes, keep=False)
        assert np.abs(tr[0]).max() > 0
        np.testing.assert_allclose(r.traces, tr[0], rtol=0, atol=1e-13 * np.abs(tr[0]).max())
    st = serving.latency_stats(reqs)
    assert 0 <= st["p50_s"] <= st["p99_s"]
