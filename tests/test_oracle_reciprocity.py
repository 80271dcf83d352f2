"""Source-receiver reciprocity of the discrete time loop (CPU oracle).

Newmark's average-acceleration scheme applied to M u'' + K u = f is a linear map from
source samples to displacement samples whose transfer function is a scalar rational
function of z times (c(z) M + K)^-1.  Replacing M, K by their transposes transposes the
map, so the trace at b from a source at a equals, sample by sample, the trace at a from
a source at b under the transposed pencil.  The radial finite-difference operator is
not symmetric, so the plain swap (same pencil) is only approximately reciprocal."""

import numpy as np

from oracle import bruteforce, fwi, sbfem
from sbfwi_inputs import boundary_nodes, structured_mesh, ricker


def _system():
    m = structured_mesh(2, 2, 2)
    n_r = 5
    els = sbfem.elements_from_mesh(m)
    xi = sbfem.radial_grid(n_r - 1, 1e-3, sbfem.XP)
    pts, _ = fwi.nodal_points(m, els, xi)
    rho = 1.0 + 0.4 * np.random.default_rng(3).random(pts.shape[0])
    dt = 0.5 * 0.25
    return m, bruteforce.FullSystem(m, n_r, 1.0, rho, dt), dt


def test_transposed_pencil_swaps_source_and_receiver():
    m, fs, dt = _system()
    a = int(boundary_nodes(m, "top")[1])
    b = int(boundary_nodes(m, "bottom")[3])
    w = ricker(1.0 / (10 * 0.25), dt, 60)[None]
    ab_steps, _ = fs.forward([a], w, [b])
    ab = fs.forward_pencil([a], w, [b])
    scale = np.linalg.norm(ab)
    assert scale > 0
    # the pencil form is the brute-force time loop itself
    assert np.linalg.norm(ab - ab_steps) <= 1e-12 * scale
    ba_t = fs.forward_pencil([b], w, [a], transpose=True)
    assert np.linalg.norm(ab - ba_t) <= 1e-12 * scale
    # the plain swap differs: the operator is not symmetric
    ba = fs.forward_pencil([b], w, [a])
    assert np.linalg.norm(ab - ba) > 1e-6 * scale
