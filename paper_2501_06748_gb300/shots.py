"""Shot-parallel misfit and gradient over ranks (one process per GPU).

Every shot is an independent forward + adjoint pair on the same model (Section 2:
the misfit and its gradient are sums over sources), so shots are sharded across
ranks and each rank runs its own shots on its own GPU with a replica of the mesh,
model and factorisation.  The ranks exchange data once per misfit/gradient
evaluation: an all-reduce (sum) of the gradient and the misfit value.

``shard`` and ``allreduce_misfit_gradient`` are plain host logic (any
``torch.distributed`` backend: NCCL for CUDA tensors, gloo for host arrays);
``misfit_and_gradient`` composes them with the CUDA library.
"""

from __future__ import annotations

import numpy as np


def shard(n_shots: int, rank: int, world: int) -> range:
    """Contiguous, balanced block of shot indices for `rank` (the first n_shots % world
    ranks take one extra shot; ranks beyond n_shots get an empty range)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    if n_shots < 0:
        raise ValueError("n_shots < 0")
    base, extra = divmod(n_shots, world)
    lo = rank * base + min(rank, extra)
    return range(lo, lo + base + (1 if rank < extra else 0))


def _dist():
    import torch.distributed as dist
    return dist if dist.is_available() and dist.is_initialized() else None


def allreduce_misfit_gradient(E: float, grad, group=None):
    """Sum the misfit value and the gradient over the ranks of `group` (in place for
    the gradient).  `grad` is a numpy array (gloo) or a torch tensor on the device
    the backend serves.  Without an initialised process group this is the identity."""
    dist = _dist()
    if dist is None or dist.get_world_size(group) == 1:
        return float(E), grad
    import torch
    if isinstance(grad, np.ndarray):
        buf = torch.from_numpy(np.concatenate([np.ascontiguousarray(grad, dtype=np.float64).ravel(), [float(E)]]))
        dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
        out = buf.numpy()
        grad[...] = out[:-1].reshape(grad.shape)
        return float(out[-1]), grad
    buf = torch.cat([grad.reshape(-1).to(torch.float64),
                     torch.tensor([float(E)], dtype=torch.float64, device=grad.device)])
    dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
    grad.copy_(buf[:-1].view_as(grad))
    return float(buf[-1].item()), grad


def misfit_and_gradient(model, src_nodes, wavelets, rec_nodes, observed, shots_per_pass: int = 8, group=None,
                        ckpt_every: int = 0, exact: bool = False):
    """Misfit and density gradient of all shots, sharded over the ranks of `group`.

    `src_nodes` [S], `wavelets` [S][K] and `observed` [S][R][K] hold every shot; each
    rank takes its `shard`, runs it through the library in passes of at most
    `shots_per_pass` shots (forward with the velocity store, or with checkpoints every
    `ckpt_every` steps, misfit, adjoint with the gradient accumulated), then joins the
    one all-reduce.  Host arrays in, host arrays out; CUDA tensors in, CUDA tensors out.
    ``exact`` gives the exact derivative of the discrete misfit instead of the paper's kernel."""
    from . import sbfwi
    mode = sbfwi.GRAD_EXACT if exact else sbfwi.GRAD_KERNEL
    sbfwi.set_gradient_mode(model, mode)
    dist = _dist()
    rank = dist.get_rank(group) if dist else 0
    world = dist.get_world_size(group) if dist else 1
    src = np.asarray(src_nodes, dtype=np.int64)
    mine = shard(len(src), rank, world)
    shape = model.grad_shape
    if hasattr(wavelets, "is_cuda") and wavelets.is_cuda:
        import torch
        grad = torch.zeros(shape, dtype=torch.float64, device=wavelets.device)
    else:
        grad = np.zeros(shape)
    E = 0.0
    for lo in range(mine.start, mine.stop, max(1, shots_per_pass)):
        hi = min(mine.stop, lo + max(1, shots_per_pass))
        tr, st = sbfwi.forward(model, src[lo:hi], wavelets[lo:hi], rec_nodes, ckpt_every=ckpt_every)
        Ec, res = sbfwi.misfit(tr, observed[lo:hi], model.dt)
        sbfwi.adjoint_gradient(model, st, res, mode=mode, grad_out=grad, accumulate=True)
        E += Ec
        del st
    return allreduce_misfit_gradient(E, grad, group)
