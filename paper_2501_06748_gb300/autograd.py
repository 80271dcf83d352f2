"""The waveform misfit of a density model as a differentiable torch function (a harness
around the library: the forward solve, the misfit and the adjoint all run in its CUDA
kernels; this module only marshals arrays).

``misfit(rho, problem)`` returns E(rho) = 1/2 dt sum over shots, receivers and samples
of (d - u)^2 (Eq. (misfit)) as a 0-d float64 tensor.  Its backward is, with
``problem.gradient == "kernel"``, the paper's gradient (Sections 2 and 4): the forward
operator run in reversed time with the residuals as sources and the zero-lag correlation
of forward and adjoint velocities, with the c^2 grad(lambda).grad(u) term dropped as the
paper does; with ``"exact"`` the exact derivative of the discrete misfit (the library's
transposed condensation run backwards in time), which is what finite differences of E
measure.  Either lives on the fine density grid (or on the nodal points for
``SBFWI_RHO_NODAL``).  The forward pass keeps, per
pass of ``shots_per_pass`` shots, the forward field the adjoint needs: the velocities
of every step, or with ``ckpt_every`` > 0 (or ``sbfwi.CKPT_AUTO``) only checkpoints,
the forward being recomputed window by window during backward.

Arrays follow the library's memory rule: with ``rho`` a CUDA tensor, the wavelets and
observed traces must be CUDA tensors too and everything stays on the device; with a
CPU tensor, they are numpy arrays or CPU tensors and the work still runs on the GPU
through host buffers.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from . import sbfwi


@dataclass
class Problem:
    mesh: "sbfwi.Mesh"
    c: float
    dt: float
    src_nodes: np.ndarray          # (S,)
    wavelets: object               # (S, K)
    rec_nodes: np.ndarray          # (R,)
    observed: object               # (S, R, K)
    rho_kind: int = sbfwi.RHO_GRID
    lx: float = 1.0
    ly: float = 1.0
    shots_per_pass: int = 8
    ckpt_every: int = 0
    gradient: str = "kernel"       # "kernel" (the paper's) or "exact"


def _host(x):
    if isinstance(x, torch.Tensor):
        return x.detach().cpu().numpy()
    return np.asarray(x, dtype=np.float64)


class _Misfit(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rho, prob: Problem):
        dev = rho.is_cuda
        r = rho.detach().contiguous() if dev else np.ascontiguousarray(_host(rho), dtype=np.float64)
        wav = prob.wavelets if dev else _host(prob.wavelets)
        obs = prob.observed if dev else _host(prob.observed)
        if prob.gradient not in ("kernel", "exact"):
            raise ValueError("gradient must be 'kernel' or 'exact'")
        model = sbfwi.Model(prob.mesh, prob.c, r, prob.dt, rho_kind=prob.rho_kind, lx=prob.lx, ly=prob.ly)
        mode = sbfwi.GRAD_EXACT if prob.gradient == "exact" else sbfwi.GRAD_KERNEL
        sbfwi.set_gradient_mode(model, mode)
        src = np.asarray(prob.src_nodes, dtype=np.int64)
        per = max(1, int(prob.shots_per_pass))
        E, passes = 0.0, []
        for lo in range(0, src.size, per):
            hi = min(src.size, lo + per)
            tr, st = sbfwi.forward(model, src[lo:hi], wav[lo:hi], prob.rec_nodes, ckpt_every=prob.ckpt_every)
            e, res = sbfwi.misfit(tr, obs[lo:hi], prob.dt)
            E += e
            passes.append((st, res))
        ctx.model, ctx.passes, ctx.mode = model, passes, mode
        ctx.shape, ctx.device, ctx.cuda = tuple(rho.shape), rho.device, dev
        return torch.tensor(E, dtype=torch.float64, device=rho.device)

    @staticmethod
    def backward(ctx, grad_E):
        if ctx.passes is None:
            raise RuntimeError("the misfit's backward can run once (its forward fields are released)")
        if ctx.cuda:
            g = torch.zeros(ctx.shape, dtype=torch.float64, device=ctx.device)
        else:
            g = np.zeros(ctx.shape)
        for st, res in ctx.passes:
            sbfwi.adjoint_gradient(ctx.model, st, res, mode=ctx.mode, grad_out=g, accumulate=True)
        ctx.passes = None
        if not ctx.cuda:
            g = torch.from_numpy(g)
        return grad_E * g, None


def misfit(rho: torch.Tensor, problem: Problem) -> torch.Tensor:
    """E(rho) with the paper's adjoint gradient (or the exact one) as its backward."""
    return _Misfit.apply(rho, problem)


def objective(problem: Problem):
    """fg(rho) -> (E, dE/drho) through autograd, the form ``inversion.lbfgs`` takes."""
    def fg(rho):
        x = rho.detach().clone().requires_grad_(True)
        E = misfit(x, problem)
        E.backward()
        return float(E.detach()), x.grad.detach()
    return fg
