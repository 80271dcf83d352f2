"""Edge cases of the GPU path against the oracle: a single element, the lowest
Lagrange order, the fewest radial points, one time step, no receivers, the largest
shot batch (16, FP64 element kernel), boundary-node counts above one tensor-core
tile (n_b = 20: FP64 element kernel; n_b = 24 and the largest, 32: two-tile kernel)."""

import numpy as np
import pytest

from oracle import fwi
from sbfwi_inputs import structured_mesh, boundary_nodes, ricker

pytestmark = pytest.mark.gpu

TRACE_TOL = 1e-10
GRAD_TOL = 1e-8


def rel(a, b):
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / (nb if nb > 0 else 1.0))


def _case(nx, ny, p, n_r, B, K, n_rec, seed=0):
    mesh = structured_mesh(nx, ny, p)
    rng = np.random.default_rng(seed)
    gx = gy = 12
    rho = 0.7 + 0.6 * rng.random((gy, gx))
    top = boundary_nodes(mesh, "top")
    srcs = rng.choice(top, size=B, replace=B > len(top))
    bnd = np.unique(np.concatenate([boundary_nodes(mesh, s) for s in ("bottom", "left", "right")]))
    recs = rng.choice(bnd, size=min(n_rec, len(bnd)), replace=False) if n_rec else np.zeros(0, dtype=np.int64)
    h = 1.0 / (max(nx, ny) * p)
    dt = 0.5 * h
    wav = np.stack([ricker(1.0 / (10 * h) * (1 + 0.05 * s), dt, K) for s in range(B)])
    return mesh, rho, srcs, recs, wav, dt


CASES = {
    "single_element_p2": (1, 1, 2, 6, 2, 40, 3),
    "p1_fewest_radial_points": (2, 2, 1, 3, 3, 40, 4),
    "one_time_step": (3, 2, 2, 5, 2, 1, 4),
    "sixteen_shots_fp64_kernel": (3, 3, 2, 5, 16, 30, 4),
    "nb20_fp64_kernel": (2, 2, 5, 5, 3, 30, 4),
    "nb24_two_tile_kernel": (2, 2, 6, 5, 3, 30, 4),
    "nb32_two_tile_kernel": (2, 2, 8, 4, 3, 20, 4),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_edge_case_matches_oracle(lib, name):
    nx, ny, p, n_r, B, K, n_rec = CASES[name]
    mesh, rho, srcs, recs, wav, dt = _case(nx, ny, p, n_r, B, K, n_rec)
    om = fwi.build_model(mesh, n_r, 1.0, rho, dt)
    to, store, _ = fwi.forward(om, srcs, wav, recs)
    M = lib.Mesh.from_inputs(mesh, n_r)
    md = lib.Model(M, 1.0, rho, dt)
    tr, st = lib.forward(md, srcs, wav, recs)
    assert tr.shape == to.shape
    if K > 5:
        assert np.abs(to).max() > 0
    assert rel(tr, to) <= TRACE_TOL
    res = np.random.default_rng(1).standard_normal(tr.shape)
    g = lib.adjoint_gradient(md, st, res)
    go = fwi.gradient_to_grid(om, fwi.adjoint_gradient(om, store, res, recs), rho.shape[1], rho.shape[0])
    assert rel(g, go) <= GRAD_TOL


def test_no_receivers_gives_empty_traces_and_zero_gradient(lib):
    mesh, rho, srcs, recs, wav, dt = _case(2, 2, 2, 5, 2, 20, 0)
    M = lib.Mesh.from_inputs(mesh, 5)
    md = lib.Model(M, 1.0, rho, dt)
    tr, st = lib.forward(md, srcs, wav, recs)
    assert tr.shape == (2, 0, 20)
    g = lib.adjoint_gradient(md, st, tr)
    assert np.all(g == 0)
    E, _ = lib.misfit(tr, tr, dt)
    assert E == 0.0


@pytest.mark.parametrize("intervals", [5, 7])
def test_paper_shaped_workload_matches_oracle(lib, intervals):
    """The paper's plate recipe (100 mm plate, c = 6000 m/s, rho = 2700 with a flaw, two
    2-cycle sine-burst sources, receivers every 1 mm, 200 steps of 0.2 us) with 5 and 7
    radial intervals, on about 100 square elements."""
    from sbfwi_inputs import paper_workload
    w = paper_workload(n_elem=100, intervals=intervals)
    L = w.mesh.lx
    om = fwi.build_model(w.mesh, w.n_r, w.c, w.rho_true, w.dt, lx=L, ly=L)
    to, store, _ = fwi.forward(om, w.src_nodes, w.wavelets, w.rec_nodes)
    M = lib.Mesh.from_inputs(w.mesh, w.n_r)
    md = lib.Model(M, w.c, w.rho_true, w.dt, lx=L, ly=L)
    tr, st = lib.forward(md, w.src_nodes, w.wavelets, w.rec_nodes)
    assert np.abs(to).max() > 0
    assert rel(tr, to) <= TRACE_TOL
    res = -to
    g = lib.adjoint_gradient(md, st, res)
    go = fwi.gradient_to_grid(om, fwi.adjoint_gradient(om, store, res, w.rec_nodes), w.gx, w.gy, L, L)
    assert rel(g, go) <= GRAD_TOL
