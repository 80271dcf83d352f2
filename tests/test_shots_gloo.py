"""Shot sharding over ranks: two gloo ranks on the CPU, each running its shard of
the shots through the oracle, then the one all-reduce of misfit and gradient; the
sum equals the single-process result over all shots."""

import os
import socket

import numpy as np
import pytest

from paper_2501_06748_gb300.shots import shard, allreduce_misfit_gradient


def test_shard_covers_every_shot_once():
    for n in range(0, 12):
        for world in range(1, 6):
            parts = [shard(n, r, world) for r in range(world)]
            flat = [i for p in parts for i in p]
            assert flat == list(range(n))
            sizes = [len(p) for p in parts]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard(4, 2, 2)


def _problem():
    from sbfwi_inputs import structured_mesh, boundary_nodes, ricker
    mesh = structured_mesh(3, 3, 2)
    rng = np.random.default_rng(11)
    rho = 0.7 + 0.6 * rng.random((12, 12))
    top = boundary_nodes(mesh, "top")
    srcs = np.array(top[1:4])
    bnd = np.unique(np.concatenate([boundary_nodes(mesh, s) for s in ("bottom", "left", "right")]))
    recs = rng.choice(bnd, size=4, replace=False)
    dt, K = 0.05, 30
    wav = np.stack([ricker(1.2 + 0.1 * s, dt, K) for s in range(3)])
    observed = 0.01 * rng.standard_normal((3, 4, K))
    return mesh, rho, srcs, recs, wav, dt, observed


def _rank_result(shots):
    """Misfit and grid gradient of the given shots with the oracle."""
    from oracle import fwi
    mesh, rho, srcs, recs, wav, dt, observed = _problem()
    g = np.zeros(rho.shape)
    E = 0.0
    if len(shots):
        om = fwi.build_model(mesh, 4, 1.0, rho, dt)
        sl = slice(shots.start, shots.stop)
        tr, store, _ = fwi.forward(om, srcs[sl], wav[sl], recs)
        E, res = fwi.misfit(tr, observed[sl], dt)
        g = fwi.gradient_to_grid(om, fwi.adjoint_gradient(om, store, res, recs), rho.shape[1], rho.shape[0])
    return E, g


def _worker(rank, world, port, n_shots, out_dir):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        E, g = _rank_result(shard(n_shots, rank, world))
        E, g = allreduce_misfit_gradient(E, g)
        np.save(os.path.join(out_dir, f"rank{rank}.npy"), np.concatenate([g.ravel(), [E]]))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("n_shots", [3, 1])
def test_two_gloo_ranks_sum_to_the_single_process_gradient(tmp_path, n_shots):
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), n_shots, str(tmp_path)), nprocs=world,
                       start_method="spawn", join=True)
    E1, g1 = _rank_result(range(0, n_shots))
    for r in range(world):
        out = np.load(tmp_path / f"rank{r}.npy")
        assert abs(out[-1] - E1) <= 1e-13 * abs(E1)
        np.testing.assert_allclose(out[:-1].reshape(g1.shape), g1, rtol=0, atol=1e-13 * np.abs(g1).max())
    assert np.abs(g1).max() > 0


def test_allreduce_without_a_process_group_is_the_identity():
    g = np.arange(6.0).reshape(2, 3)
    E, g2 = allreduce_misfit_gradient(2.5, g)
    assert E == 2.5 and g2 is g
