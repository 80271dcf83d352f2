"""Seeded density fields on a fine, cell-centred Cartesian grid.

A field is an array ``rho[gy, gx]``; cell (ix, iy) covers
[ix*lx/gx, (ix+1)*lx/gx] x [iy*ly/gy, (iy+1)*ly/gy] and its value sits at the cell
centre.  Flaws are regions where the background density is multiplied by a small
factor, like the paper's hole (void) and weak-inclusion specimens (Section 4).
"""

import numpy as np


def _cell_centres(gx, gy, lx, ly):
    xc = (np.arange(gx) + 0.5) * (lx / gx)
    yc = (np.arange(gy) + 0.5) * (ly / gy)
    return np.meshgrid(xc, yc, indexing="xy")   # arrays shaped (gy, gx)


def flawed_density_circle(gx, gy, lx=1.0, ly=1.0, rho0=1.0, radius=0.1, factor=1e-3, seed=0):
    """Homogeneous rho0 with one circular flaw (rho0*factor inside).

    The centre is drawn uniformly so that the circle stays clear of the edges by
    at least one radius.
    """
    rng = np.random.default_rng(seed)
    cx = rng.uniform(2 * radius, lx - 2 * radius)
    cy = rng.uniform(2 * radius, ly - 2 * radius)
    X, Y = _cell_centres(gx, gy, lx, ly)
    rho = np.full((gy, gx), float(rho0))
    rho[(X - cx) ** 2 + (Y - cy) ** 2 <= radius ** 2] *= factor
    return rho, {"centre": (cx, cy), "radius": radius, "factor": factor}


def flawed_density_ellipses(gx, gy, lx=1.0, ly=1.0, rho0=1.0, n=2, amin=0.03, amax=0.12,
                            factor=1e-5, seed=1, max_tries=1000):
    """Homogeneous rho0 with ``n`` non-overlapping elliptical flaws (rho0*factor inside).

    Semi-axes are uniform in [amin, amax], orientation uniform in [0, pi), centres
    uniform in the interior with a margin of ``amax`` from the edges.
    """
    rng = np.random.default_rng(seed)
    X, Y = _cell_centres(gx, gy, lx, ly)
    mask_all = np.zeros((gy, gx), dtype=bool)
    flaws = []
    tries = 0
    while len(flaws) < n:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("could not place non-overlapping ellipses")
        a, b = rng.uniform(amin, amax, size=2)
        th = rng.uniform(0.0, np.pi)
        cx = rng.uniform(amax + 0.05 * lx, lx - amax - 0.05 * lx)
        cy = rng.uniform(amax + 0.05 * ly, ly - amax - 0.05 * ly)
        dx, dy = X - cx, Y - cy
        u = dx * np.cos(th) + dy * np.sin(th)
        v = -dx * np.sin(th) + dy * np.cos(th)
        m = (u / a) ** 2 + (v / b) ** 2 <= 1.0
        # keep a one-cell gap between flaws
        grown = m.copy()
        grown[1:, :] |= m[:-1, :]
        grown[:-1, :] |= m[1:, :]
        grown[:, 1:] |= m[:, :-1]
        grown[:, :-1] |= m[:, 1:]
        if np.any(grown & mask_all) or not np.any(m):
            continue
        mask_all |= m
        flaws.append({"centre": (cx, cy), "semi_axes": (a, b), "angle": th})
    rho = np.full((gy, gx), float(rho0))
    rho[mask_all] *= factor
    return rho, {"flaws": flaws, "factor": factor}
