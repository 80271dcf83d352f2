"""The sharded product path with two ranks: two processes (gloo on the host, both on the one
GPU of this machine), each running its shard of the shots through the library with
``shots.misfit_and_gradient`` (set-up, forward, misfit, adjoint and gradient in libsbfwi),
then the one all-reduce of misfit and gradient.  The sum equals the oracle's single-process
result over all shots.  The ranks' kernels never wait on each other: the only exchange is
the host all-reduce after both ranks' device work has finished."""

import os
import socket

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TRACE_TOL = 1e-10
GRAD_TOL = 1e-8


def _problem():
    from sbfwi_inputs import structured_mesh, boundary_nodes, ricker
    mesh = structured_mesh(4, 4, 2)
    rng = np.random.default_rng(21)
    rho = 0.7 + 0.6 * rng.random((16, 16))
    top = boundary_nodes(mesh, "top")
    srcs = np.array(top[1:6])
    bnd = np.unique(np.concatenate([boundary_nodes(mesh, s) for s in ("bottom", "left", "right")]))
    recs = rng.choice(bnd, size=6, replace=False)
    dt, K = 0.05, 60
    wav = np.stack([ricker(1.0 + 0.1 * s, dt, K) for s in range(5)])
    observed = 0.01 * rng.standard_normal((5, 6, K))
    return mesh, rho, srcs, recs, wav, dt, observed


def _worker(rank, world, port, n_shots, exact, out_dir):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch
    import torch.distributed as dist
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        from paper_2501_06748_gb300 import sbfwi, shots
        mesh, rho, srcs, recs, wav, dt, observed = _problem()
        M = sbfwi.Mesh.from_inputs(mesh, 6)
        md = sbfwi.Model(M, 1.0, rho, dt)
        E, g = shots.misfit_and_gradient(md, srcs[:n_shots], wav[:n_shots], recs, observed[:n_shots],
                                         shots_per_pass=2, exact=exact)
        np.save(os.path.join(out_dir, f"rank{rank}.npy"), np.concatenate([np.asarray(g).ravel(), [E]]))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("n_shots,exact", [(5, False), (1, False), (5, True)])
def test_two_ranks_through_the_library_sum_to_the_oracle(lib, tmp_path, n_shots, exact):
    import torch.multiprocessing as mp
    from oracle import fwi, modex
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), n_shots, exact, str(tmp_path)), nprocs=world,
                       start_method="spawn", join=True)
    mesh, rho, srcs, recs, wav, dt, observed = _problem()
    om = fwi.build_model(mesh, 6, 1.0, rho, dt)
    if exact:
        Eo, gn = modex.misfit_and_gradient(mesh, 6, 1.0, om.rho_nodal, dt, srcs[:n_shots], wav[:n_shots], recs,
                                           observed[:n_shots])
        go = fwi.gradient_to_grid(om, gn, rho.shape[1], rho.shape[0])
    else:
        tr, store, _ = fwi.forward(om, srcs[:n_shots], wav[:n_shots], recs)
        Eo, res = fwi.misfit(tr, observed[:n_shots], dt)
        go = fwi.gradient_to_grid(om, fwi.adjoint_gradient(om, store, res, recs), rho.shape[1], rho.shape[0])
    outs = [np.load(tmp_path / f"rank{r}.npy") for r in range(world)]
    assert np.array_equal(outs[0], outs[1])                 # both ranks hold the all-reduced result
    E, g = outs[0][-1], outs[0][:-1].reshape(go.shape)
    assert abs(E - Eo) <= 1e-10 * abs(Eo)
    assert np.linalg.norm(g - go) / np.linalg.norm(go) <= GRAD_TOL
