"""Named synthetic workloads (meshes, density models, sources, receivers, time axis).

Flaw contrast.  The flaws keep the geometry of the specified workloads (a circle of
radius 0.1; two ellipses with semi-axes in [0.03, 0.12]) but multiply the density
by FLAW_FACTOR = 0.5, the paper's weak-inclusion contrast (Section 4, "half the
density").  The paper's radial finite differences discretise the expanded,
non-conservative form of the radial ODE; with a sharp jump of the density to
1e-3 or 1e-5 of the background the semi-discrete operator has real negative
omega^2 modes and every time integrator diverges (jumps to 0.1 of the background
already diverge within 2000 steps).  ``flaw_factor`` overrides the default.

Time step and source frequency follow one rule for every workload: with s_min the
smallest spacing of consecutive boundary nodes, f0 = c / (10 s_min) (about ten
nodes per dominant wavelength) and dt = 0.5 s_min / c.  Newmark uses the
average-acceleration parameters beta = 1/4, gamma = 1/2.
"""

from dataclasses import dataclass, field

import numpy as np

from .mesh import (StructuredMesh, structured_mesh, boundary_nodes, nearest_node, quadtree_mesh, min_spacing,
                   voronoi_mesh)
from .fields import flawed_density_circle, flawed_density_ellipses
from .wavelet import ricker, sine_burst

FLAW_FACTOR = 0.5


@dataclass
class Workload:
    name: str
    mesh: StructuredMesh
    n_r: int                   # radial FD points per element (n + 1, i = 0..n)
    c: float
    gx: int
    gy: int
    rho_true: np.ndarray       # (gy, gx) density with flaws
    rho_start: np.ndarray      # (gy, gx) homogeneous starting model
    src_nodes: np.ndarray      # (B,) int64, one point source per shot
    wavelets: np.ndarray       # (B, K) float64, sample k drives the step to t_{k+1}
    rec_nodes: np.ndarray      # (R,) int64, shared by all shots
    dt: float
    K: int
    f0: float
    beta: float = 0.25
    gamma: float = 0.5
    xi0: float = 1e-3
    info: dict = field(default_factory=dict)

    @property
    def n_shots(self) -> int:
        return int(self.src_nodes.shape[0])

    def summary(self) -> dict:
        m = self.mesh
        nb = getattr(m, "n_b", None)
        nb = 4 * m.p if nb is None else [int(nb.min()), int(nb.max())]
        return {"workload": self.name, "elements": m.n_elem, "p": m.p, "n_b": nb,
                "N_r": self.n_r, "global_nodes": m.n_nodes, "shots": self.n_shots,
                "receivers": int(self.rec_nodes.shape[0]), "steps": self.K,
                "grid": [self.gy, self.gx], "dt": self.dt, "f0": self.f0}


def _time_axis(mesh: StructuredMesh, c: float):
    s_min = min(mesh.lx / (mesh.nx * mesh.p), mesh.ly / (mesh.ny * mesh.p))
    return c / (10.0 * s_min), 0.5 * s_min / c


def tiny_workload(seed: int = 0, refine: int = 1, K: int = 400, flaw_factor: float = FLAW_FACTOR) -> Workload:
    """4x4 square S-elements, p = 2, N_r = 8, one circular flaw (radius 0.1) on a 64x64 grid.

    One Ricker source at the top-edge node nearest x = 0.5; four receivers on the
    other three edges.  ``refine=2`` gives the same physical set-up on a mesh with
    twice the elements per direction and twice the radial points (used to make
    observed data without an inverse crime); the source and receivers sit at the
    same physical points, which are nodes of both meshes.  The time axis is that
    of the unrefined mesh.
    """
    rng = np.random.default_rng(seed)
    base = structured_mesh(4, 4, 2)
    mesh = structured_mesh(4 * refine, 4 * refine, 2)
    c = 1.0
    f0, dt = _time_axis(base, c)
    rho_true, finfo = flawed_density_circle(64, 64, radius=0.1, factor=flaw_factor, seed=seed)
    rho_start = np.ones_like(rho_true)
    src = nearest_node(mesh, boundary_nodes(mesh, "top"), (0.5, 1.0))
    sides = ["bottom", "left", "right", ["bottom", "left", "right"][rng.integers(3)]]
    recs = []
    for side in sides:
        t = rng.uniform(0.1, 0.9)
        pt = {"bottom": (t, 0.0), "left": (0.0, t), "right": (1.0, t)}[side]
        # snap to a node of the unrefined mesh so the point exists in both meshes
        pb = base.node_xy[nearest_node(base, boundary_nodes(base, side), pt)]
        g = nearest_node(mesh, boundary_nodes(mesh, side), pb)
        if g in recs:
            g = nearest_node(mesh, np.setdiff1d(boundary_nodes(mesh, side), recs), pb)
        recs.append(g)
    wav = ricker(f0, dt, K)[None, :]
    return Workload("tiny", mesh, 8 * refine, c, 64, 64, rho_true, rho_start,
                    np.array([src], dtype=np.int64), wav, np.array(recs, dtype=np.int64),
                    dt, K, f0, info={"flaw": finfo, "seed": seed, "refine": refine})


def size_workload(seed: int = 1, K: int = 2000, n_shots: int = 8, nx: int = 64, n_r: int = 32,
                  grid: int = 256, n_rec: int = 32, flaw_factor: float = FLAW_FACTOR) -> Workload:
    """64x64 square S-elements, p = 4, N_r = 32, two elliptical flaws on a 256x256 grid.

    Eight Ricker sources equally spaced along the top edge, 32 receivers equally
    spaced along the perimeter, 2000 steps.  Smaller meshes with the same recipe
    are available through ``nx`` / ``n_r`` / ``grid`` for tests.
    """
    mesh = structured_mesh(nx, nx, 4)
    c = 1.0
    f0, dt = _time_axis(mesh, c)
    rho_true, finfo = flawed_density_ellipses(grid, grid, n=2, factor=flaw_factor, seed=seed)
    rho_start = np.ones_like(rho_true)
    top = boundary_nodes(mesh, "top")
    srcs = [nearest_node(mesh, top, ((s + 0.5) / n_shots, 1.0)) for s in range(n_shots)]
    recs = []
    for k in range(n_rec):
        t = 4.0 * (k + 0.5) / n_rec          # position along the perimeter, CCW from (0,0)
        side, u = int(t), t - int(t)
        side_name, pt = [("bottom", (u, 0.0)), ("right", (1.0, u)),
                         ("top", (1.0 - u, 1.0)), ("left", (0.0, 1.0 - u))][side]
        recs.append(nearest_node(mesh, boundary_nodes(mesh, side_name), pt))
    recs = list(dict.fromkeys(recs))
    wav = np.stack([ricker(f0, dt, K) for _ in srcs])
    return Workload("size", mesh, n_r, c, grid, grid, rho_true, rho_start,
                    np.array(srcs, dtype=np.int64), wav, np.array(recs, dtype=np.int64),
                    dt, K, f0, info={"flaws": finfo, "seed": seed})


def diff_workload(seed: int = 2, K: int = 8000, n_shots: int = 16, nx: int = 128, n_r: int = 32,
                  grid: int = 512, n_rec: int = 64, flaw_factor: float = FLAW_FACTOR) -> Workload:
    """The differentiation-scale recipe: 128x128 square S-elements, p = 4, N_r = 32, 16
    sources on the top edge, 64 receivers along the perimeter, 8000 steps, 512x512
    density grid (the forward field no longer fits in memory: checkpoints)."""
    w = size_workload(seed=seed, K=K, n_shots=n_shots, nx=nx, n_r=n_r, grid=grid, n_rec=n_rec,
                      flaw_factor=flaw_factor)
    w.name = "diff"
    return w


def paper_workload(n_elem: int = 2000, intervals: int = 5, seed: int = 3, p: int = 2, K: int = 200,
                   flaw_factor: float = FLAW_FACTOR, mesh_kind: str = "square", lloyd_iters: int = 40,
                   mesh=None) -> Workload:
    """The shape of the paper's plate experiments (Section 4) on square S-elements: a
    100 mm x 100 mm plate, c = 6000 m/s, rho = 2700 with one circular flaw, two
    sources 30 mm apart on the top edge driven by a 2-cycle sine burst (f0 = 500 kHz),
    receivers every 1 mm along all four edges, dt = 0.2 us, 200 steps (40 us), and
    `intervals` radial intervals (N_r = intervals + 1).  ``mesh_kind="voronoi"`` gives the
    paper's mesh type, `n_elem` centroidal Voronoi polygons (seeded, Lloyd iterations);
    ``"square"`` about `n_elem` squares."""
    L = 0.1
    if mesh is not None:                      # a mesh of this recipe made earlier (reused across intervals)
        pass
    elif mesh_kind == "voronoi":
        mesh = voronoi_mesh(n_elem, p, lx=L, ly=L, seed=seed, lloyd_iters=lloyd_iters)
    elif mesh_kind == "square":
        nx = max(1, int(round(np.sqrt(n_elem))))
        mesh = structured_mesh(nx, nx, p, lx=L, ly=L)
    else:
        raise ValueError(mesh_kind)
    c = 6000.0
    f0, dt = 500e3, 0.2e-6
    grid = 256
    rho_rel, finfo = flawed_density_circle(grid, grid, radius=0.08, factor=flaw_factor, seed=seed)
    rho_true = 2700.0 * rho_rel
    rho_start = np.full_like(rho_true, 2700.0)
    top = boundary_nodes(mesh, "top")
    srcs = [nearest_node(mesh, top, (x, L)) for x in (0.035, 0.065)]
    recs = []
    for side, pts in (("bottom", [(x, 0.0) for x in np.arange(0.0005, L, 0.001)]),
                      ("right", [(L, y) for y in np.arange(0.0005, L, 0.001)]),
                      ("top", [(x, L) for x in np.arange(0.0005, L, 0.001)]),
                      ("left", [(0.0, y) for y in np.arange(0.0005, L, 0.001)])):
        cand = boundary_nodes(mesh, side)
        recs += [nearest_node(mesh, cand, pt) for pt in pts]
    recs = [r for r in dict.fromkeys(recs) if r not in srcs]
    wav = np.stack([sine_burst(f0, dt, K, cycles=2, amplitude=1e12) for _ in srcs])
    return Workload("paper", mesh, intervals + 1, c, grid, grid, rho_true, rho_start,
                    np.array(srcs, dtype=np.int64), wav, np.array(recs, dtype=np.int64),
                    dt, K, f0, info={"flaws": finfo, "seed": seed, "plate_m": L, "intervals": intervals,
                                     "mesh": mesh_kind})


BATCHING_MESHES = ((2, 16), (3, 32), (5, 48))     # (p, N_r) of the three quadtree meshes


def batching_workload(index: int, seed: int = 4, base: int = 16, levels: int = 2, K: int = 1500,
                      n_shots: int | None = None, total_shots: int = 64, grid: int = 256, n_rec: int = 32,
                      flaw_factor: float = FLAW_FACTOR) -> Workload:
    """Mesh ``index`` (0, 1, 2) of the batching recipe: a quadtree of square S-elements,
    ``base`` x ``base`` root cells refined ``levels`` times around two elliptical flaws
    (seed + index) and 2:1 balanced, so that elements carry 4 to 8 line elements of order
    p = 2, 3, 5 (n_b from 8 to 40) with N_r = 16, 32, 48 radial points.  The 64 shots of
    the recipe are split over the three meshes (22, 21, 21), sources equally spaced on
    the top edge, ``n_rec`` receivers equally spaced along the perimeter, 1500 steps."""
    p, n_r = BATCHING_MESHES[index]
    rho_true, finfo = flawed_density_ellipses(grid, grid, n=2, factor=flaw_factor, seed=seed + index)
    flaw = rho_true != rho_true.max()
    h = 1.0 / grid

    def refine(x0, y0, x1, y1, lvl):
        m = 0.5 * (x1 - x0)                        # refine where a flaw is within half a cell
        i0, i1 = max(0, int((x0 - m) / h)), min(grid, int(np.ceil((x1 + m) / h)))
        j0, j1 = max(0, int((y0 - m) / h)), min(grid, int(np.ceil((y1 + m) / h)))
        return bool(flaw[j0:j1, i0:i1].any())

    mesh = quadtree_mesh(base, levels, refine, p)
    c = 1.0
    s_min = min_spacing(mesh)
    f0, dt = c / (10.0 * s_min), 0.5 * s_min / c
    if n_shots is None:
        n_shots = total_shots // 3 + (1 if index < total_shots % 3 else 0)
    top = boundary_nodes(mesh, "top")
    srcs = list(dict.fromkeys(nearest_node(mesh, top, ((s + 0.5) / n_shots, 1.0)) for s in range(n_shots)))
    recs = []
    for k in range(n_rec):
        t = 4.0 * (k + 0.5) / n_rec
        side, u = int(t), t - int(t)
        side_name, pt = [("bottom", (u, 0.0)), ("right", (1.0, u)),
                         ("top", (1.0 - u, 1.0)), ("left", (0.0, 1.0 - u))][side]
        recs.append(nearest_node(mesh, boundary_nodes(mesh, side_name), pt))
    recs = list(dict.fromkeys(recs))
    wav = np.stack([ricker(f0, dt, K) for _ in srcs])
    return Workload(f"batching[{index}]", mesh, n_r, c, grid, grid, rho_true, np.ones_like(rho_true),
                    np.array(srcs, dtype=np.int64), wav, np.array(recs, dtype=np.int64),
                    dt, K, f0, info={"flaws": finfo, "seed": seed + index, "base": base, "levels": levels})


def solid_workload(nx: int = 16, p: int = 2, n_r: int = 16, n_shots: int = 8, K: int = 500, grid: int = 64,
                   n_rec: int = 32, seed: int = 5, flaw_factor: float = FLAW_FACTOR) -> Workload:
    """A 3-D recipe: the unit cube in nx^3 hexahedral S-elements with faces of order p
    (n_b = 26 at p = 2), N_r radial points, one spherical flaw on a grid^3 density grid,
    n_shots Ricker sources spread over the top face (z = 1), receivers on the bottom face
    and the four sides (nearest nodes to seeded points), f0 and dt from the smallest node
    spacing as in the 2-D recipes.  ``gx``/``gy`` hold the grid size; the density arrays are
    [grid][grid][grid]."""
    from .mesh3d import structured_mesh3d, boundary_nodes3d, nearest_node3d, flawed_density_sphere
    mesh = structured_mesh3d(nx, nx, nx, p)
    c = 1.0
    s_min = 1.0 / (nx * p)
    f0, dt = c / (10.0 * s_min), 0.5 * s_min / c
    rho_true, finfo = flawed_density_sphere(grid, grid, grid, radius=0.15, factor=flaw_factor, seed=seed)
    rho_start = np.ones_like(rho_true)
    rng = np.random.default_rng(seed)
    top = boundary_nodes3d(mesh, "z1")
    k = int(np.ceil(np.sqrt(n_shots)))
    pts = [((i + 0.5) / k, (j + 0.5) / k, 1.0) for j in range(k) for i in range(k)][:n_shots]
    srcs = [nearest_node3d(mesh, top, q) for q in pts]
    recs = []
    for side in ("z0", "x0", "x1", "y0", "y1"):
        ids = boundary_nodes3d(mesh, side)
        for _ in range(max(1, n_rec // 5)):
            q = mesh.node_xyz[rng.choice(ids)]
            recs.append(int(nearest_node3d(mesh, ids, q)))
    recs = [r for r in dict.fromkeys(recs) if r not in srcs]
    wav = np.stack([ricker(f0, dt, K) for _ in srcs])
    return Workload("solid", mesh, n_r, c, grid, grid, rho_true, rho_start, np.array(srcs, dtype=np.int64), wav,
                    np.array(recs, dtype=np.int64), dt, K, f0, info={"flaw": finfo, "seed": seed, "grid": grid})


def workload_by_name(name: str, **kw) -> Workload:
    if name == "tiny":
        return tiny_workload(**kw)
    if name == "size":
        return size_workload(**kw)
    if name == "diff":
        return diff_workload(**kw)
    if name == "paper":
        return paper_workload(**kw)
    if name == "solid":
        return solid_workload(**kw)
    raise KeyError(name)
