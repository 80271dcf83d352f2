"""Density inversion loop around the library's misfit and gradient (a harness, not
part of the method's arithmetic).

The paper minimises the waveform misfit over the density with a bounded quasi-
Newton method (Section 4: L-BFGS with box constraints on the density).  This module
gives the same kind of loop: a two-loop-recursion L-BFGS with memory ``m``, the box
``lo <= rho <= hi`` enforced by projection (clipping), the memory cleared whenever
the set of parameters on a bound changes, and a backtracking line search on the
projected step.  The objective is ``shots.misfit_and_gradient``: every shot's
forward and adjoint run in the CUDA library, sharded over ranks when a process
group is initialised; the vector updates of the loop run in torch on the device of
the parameters (or in numpy for host arrays).
"""

from __future__ import annotations

import numpy as np

from . import shots


def objective(mesh, c, dt, src_nodes, wavelets, rec_nodes, observed, lx=1.0, ly=1.0, shots_per_pass=8,
              ckpt_every=0, group=None, exact=False):
    """fg(rho_grid) -> (misfit, gradient on the grid): one model set-up and every shot's
    forward, misfit and adjoint through the library (the paper's kernel, or with ``exact``
    the exact derivative of the discrete misfit)."""
    from . import sbfwi

    def fg(rho):
        model = sbfwi.Model(mesh, c, rho, dt, lx=lx, ly=ly)
        return shots.misfit_and_gradient(model, src_nodes, wavelets, rec_nodes, observed,
                                         shots_per_pass=shots_per_pass, group=group, ckpt_every=ckpt_every,
                                         exact=exact)
    return fg


def misfit_only(mesh, c, dt, src_nodes, wavelets, rec_nodes, observed, lx=1.0, ly=1.0, shots_per_pass=8):
    """f(rho_grid) -> misfit: forward passes and the misfit only (finite-difference checks)."""
    from . import sbfwi

    def f(rho):
        model = sbfwi.Model(mesh, c, rho, dt, lx=lx, ly=ly)
        src = np.asarray(src_nodes, dtype=np.int64)
        E = 0.0
        for lo in range(0, src.size, max(1, shots_per_pass)):
            hi = min(src.size, lo + max(1, shots_per_pass))
            tr, _ = sbfwi.forward(model, src[lo:hi], wavelets[lo:hi], rec_nodes, keep=False)
            E += sbfwi.misfit(tr, observed[lo:hi], dt, want_residual=False)[0]
        return E
    return f


def _ops(x):
    if hasattr(x, "is_cuda"):
        import torch
        return (lambda a, b: float(torch.sum(a * b)), lambda a: a.clone(),
                lambda a, lo, hi: torch.clamp(a, lo, hi), lambda a: float(torch.max(torch.abs(a))))
    return (lambda a, b: float(np.sum(a * b)), lambda a: a.copy(), lambda a, lo, hi: np.clip(a, lo, hi),
            lambda a: float(np.max(np.abs(a))))


def lbfgs(fg, x0, lo, hi, iters, m=10, step0=0.05, max_backtracks=8, c1=1e-4, callback=None):
    """Projected L-BFGS; returns (x, history) with history[k] = misfit after iteration k
    (history[0] at x0).  ``step0`` is the first step's largest relative change of x."""
    dot, copy, clip, amax = _ops(x0)
    x = clip(copy(x0), lo, hi)
    E, g = fg(x)
    hist = [E]
    S, Y = [], []
    active = None
    for it in range(iters):
        # two-loop recursion for d = -H g
        q = copy(g)
        alphas = []
        for s_, y_ in reversed(list(zip(S, Y))):
            rho_ = 1.0 / dot(y_, s_)
            a_ = rho_ * dot(s_, q)
            q = q - a_ * y_
            alphas.append((rho_, a_, s_, y_))
        if S:
            q = q * (dot(S[-1], Y[-1]) / dot(Y[-1], Y[-1]))
        else:
            q = q * (step0 * amax(x) / max(amax(g), 1e-300))
        for rho_, a_, s_, y_ in reversed(alphas):
            b_ = rho_ * dot(y_, q)
            q = q + (a_ - b_) * s_
        d = -q
        if dot(d, g) >= 0:                      # not a descent direction: restart
            S, Y = [], []
            d = -g * (step0 * amax(x) / max(amax(g), 1e-300))
        # backtracking on the projected step
        t = 1.0
        accepted = False
        for _ in range(max_backtracks):
            xn = clip(x + t * d, lo, hi)
            En, gn = fg(xn)
            if En <= E + c1 * dot(g, xn - x):
                accepted = True
                break
            t *= 0.5
        if not accepted:
            S, Y = [], []
            if callback:
                callback(it, x, E)
            hist.append(E)
            continue
        s_, y_ = xn - x, gn - g
        on_bound = (xn <= lo) | (xn >= hi)
        if active is not None and bool((on_bound != active).any()):
            S, Y = [], []                        # active set changed
        active = on_bound
        if dot(s_, y_) > 1e-12 * dot(y_, y_) ** 0.5 * dot(s_, s_) ** 0.5:
            S.append(s_)
            Y.append(y_)
            if len(S) > m:
                S.pop(0)
                Y.pop(0)
        x, E, g = xn, En, gn
        hist.append(E)
        if callback:
            callback(it, x, E)
    return x, hist
