"""Seeded meshes of square scaled-boundary elements.

A mesh is given the way the library's ``sbfwi_build_mesh`` takes it:

* ``node_xy``   (n_nodes, 2) float64 -- global node coordinates;
* ``elem_ptr``  (n_elem + 1,) int64  -- element ``e`` owns line elements
  ``elem_ptr[e] .. elem_ptr[e+1]-1``;
* ``line_nodes`` (n_lines, p+1) int64 -- the ``p+1`` global node ids of each
  boundary line element, listed in the direction of travel, with every element's
  lines running counter-clockwise around its scaling centre;
* ``centre_xy`` (n_elem, 2) float64  -- scaling centre of each element.

Nodes inside a line element are equally spaced along it (the paper leaves the
node placement of the boundary Lagrange elements open).
"""

from dataclasses import dataclass

import numpy as np


@dataclass
class StructuredMesh:
    node_xy: np.ndarray
    elem_ptr: np.ndarray
    line_nodes: np.ndarray
    centre_xy: np.ndarray
    p: int
    lx: float
    ly: float
    nx: int
    ny: int

    @property
    def n_nodes(self) -> int:
        return int(self.node_xy.shape[0])

    @property
    def n_elem(self) -> int:
        return int(self.centre_xy.shape[0])


def structured_mesh(nx: int, ny: int, p: int, lx: float = 1.0, ly: float = 1.0) -> StructuredMesh:
    """nx x ny square S-elements on [0, lx] x [0, ly], boundary lines of order p.

    The scaling centre of each element is its cell centre.  Global node count is
    (nx+1)(ny+1) + (p-1)(nx(ny+1) + ny(nx+1)).
    """
    if nx < 1 or ny < 1 or p < 1:
        raise ValueError("nx, ny, p must be >= 1")
    dx, dy = lx / nx, ly / ny
    nv = (nx + 1) * (ny + 1)
    nh = nx * (ny + 1)          # horizontal edges
    nvert = ny * (nx + 1)       # vertical edges
    n_nodes = nv + (p - 1) * (nh + nvert)
    xy = np.zeros((n_nodes, 2))
    iy, ix = np.meshgrid(np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    xy[:nv, 0] = (ix * dx).ravel()
    xy[:nv, 1] = (iy * dy).ravel()
    base_h = nv
    base_v = nv + (p - 1) * nh

    def vid(i, j):
        return j * (nx + 1) + i

    def hnodes(i, j):           # edge (i,j)->(i+1,j), ascending x
        b = base_h + (j * nx + i) * (p - 1)
        return list(range(b, b + p - 1))

    def vnodes(i, j):           # edge (i,j)->(i,j+1), ascending y
        b = base_v + (j * (nx + 1) + i) * (p - 1)
        return list(range(b, b + p - 1))

    for j in range(ny + 1):
        for i in range(nx):
            for k, g in enumerate(hnodes(i, j)):
                xy[g] = ((i + (k + 1) / p) * dx, j * dy)
    for j in range(ny):
        for i in range(nx + 1):
            for k, g in enumerate(vnodes(i, j)):
                xy[g] = (i * dx, (j + (k + 1) / p) * dy)

    lines = []
    centres = np.zeros((nx * ny, 2))
    for j in range(ny):
        for i in range(nx):
            e = j * nx + i
            v00, v10, v11, v01 = vid(i, j), vid(i + 1, j), vid(i + 1, j + 1), vid(i, j + 1)
            lines.append([v00] + hnodes(i, j) + [v10])
            lines.append([v10] + vnodes(i + 1, j) + [v11])
            lines.append([v11] + hnodes(i, j + 1)[::-1] + [v01])
            lines.append([v01] + vnodes(i, j)[::-1] + [v00])
            centres[e] = ((i + 0.5) * dx, (j + 0.5) * dy)
    elem_ptr = np.arange(0, 4 * nx * ny + 1, 4, dtype=np.int64)
    return StructuredMesh(xy, elem_ptr, np.asarray(lines, dtype=np.int64), centres, p, lx, ly, nx, ny)


def boundary_nodes(mesh, side: str) -> np.ndarray:
    """Global ids of the nodes on one side of the rectangular domain, sorted along it."""
    x, y = mesh.node_xy[:, 0], mesh.node_xy[:, 1]
    tol = 1e-12 * max(mesh.lx, mesh.ly)
    if side == "top":
        ids = np.nonzero(np.abs(y - mesh.ly) < tol)[0]
        return ids[np.argsort(x[ids])]
    if side == "bottom":
        ids = np.nonzero(np.abs(y) < tol)[0]
        return ids[np.argsort(x[ids])]
    if side == "left":
        ids = np.nonzero(np.abs(x) < tol)[0]
        return ids[np.argsort(y[ids])]
    if side == "right":
        ids = np.nonzero(np.abs(x - mesh.lx) < tol)[0]
        return ids[np.argsort(y[ids])]
    raise ValueError(side)


def nearest_node(mesh, ids: np.ndarray, point) -> int:
    d = np.hypot(mesh.node_xy[ids, 0] - point[0], mesh.node_xy[ids, 1] - point[1])
    return int(ids[int(np.argmin(d))])


@dataclass
class QuadtreeMesh:
    """Square S-elements of a 2:1-balanced quadtree, same arrays as ``StructuredMesh``.

    Where a cell borders two cells of the next finer level, the side is split at
    the shared (hanging) vertex into two line elements, so an element has 4 to 8
    line elements and p * (number of lines) boundary nodes.  ``cells`` holds
    (level, ix, iy) of every element (ix, iy in units of that level's cell size).
    """
    node_xy: np.ndarray
    elem_ptr: np.ndarray
    line_nodes: np.ndarray
    centre_xy: np.ndarray
    p: int
    lx: float
    ly: float
    base: int
    levels: int
    cells: np.ndarray

    @property
    def n_nodes(self) -> int:
        return int(self.node_xy.shape[0])

    @property
    def n_elem(self) -> int:
        return int(self.centre_xy.shape[0])

    @property
    def n_b(self) -> np.ndarray:
        """Boundary nodes of every element."""
        return self.p * np.diff(self.elem_ptr)


def quadtree_mesh(base: int, levels: int, refine, p: int, lx: float = 1.0, ly: float = 1.0) -> QuadtreeMesh:
    """Quadtree of square S-elements on [0, lx] x [0, ly] with ``base`` x ``base`` root cells.

    ``refine(x0, y0, x1, y1, level)`` decides whether a cell of the given level
    (0 = root) is split; cells are split up to ``levels`` times, then further
    cells are split until every pair of cells sharing a side differs by at most
    one level (2:1 balance).  Scaling centres are the cell centres; lines run
    counter-clockwise from the lower-left corner; nodes inside a line element are
    equally spaced.
    """
    if base < 1 or levels < 0 or p < 1:
        raise ValueError("base >= 1, levels >= 0, p >= 1")
    F = 1 << levels                       # fine-lattice units per root cell
    M = base * F                          # fine cells per side
    leaves = {(0, i, j) for i in range(base) for j in range(base)}

    def box(c):
        l, i, j = c
        s = F >> l
        return i * s, j * s, s

    for lvl in range(levels):
        for c in sorted(x for x in leaves if x[0] == lvl):
            X, Y, s = box(c)
            if refine(X * lx / M, Y * ly / M, (X + s) * lx / M, (Y + s) * ly / M, lvl):
                leaves.remove(c)
                leaves.update({(lvl + 1, 2 * c[1] + a, 2 * c[2] + b) for a in (0, 1) for b in (0, 1)})

    def level_map():
        lev = np.zeros((M, M), dtype=np.int64)          # [fine x][fine y] -> level of the covering leaf
        for c in leaves:
            X, Y, s = box(c)
            lev[X:X + s, Y:Y + s] = c[0]
        return lev

    while True:                                          # 2:1 balance
        lev = level_map()
        split = []
        for c in leaves:
            X, Y, s = box(c)
            nb_levels = []
            if X > 0: nb_levels.append(lev[X - 1, Y:Y + s].max())
            if X + s < M: nb_levels.append(lev[X + s, Y:Y + s].max())
            if Y > 0: nb_levels.append(lev[X:X + s, Y - 1].max())
            if Y + s < M: nb_levels.append(lev[X:X + s, Y + s].max())
            if nb_levels and max(nb_levels) > c[0] + 1:
                split.append(c)
        if not split:
            break
        for c in split:
            leaves.remove(c)
            leaves.update({(c[0] + 1, 2 * c[1] + a, 2 * c[2] + b) for a in (0, 1) for b in (0, 1)})
    lev = level_map()

    vid = {}                                             # fine-lattice vertex -> node id
    xy = []

    def vertex(X, Y):
        if (X, Y) not in vid:
            vid[(X, Y)] = len(xy)
            xy.append((X * lx / M, Y * ly / M))
        return vid[(X, Y)]

    inner = {}                                           # segment -> its p-1 inner nodes, from the lower endpoint

    def segment(a, b):
        key = (min(a, b), max(a, b))
        if key not in inner:
            (Xa, Ya), (Xb, Yb) = key
            ids = []
            for k in range(1, p):
                ids.append(len(xy))
                xy.append(((Xa + (Xb - Xa) * k / p) * lx / M, (Ya + (Yb - Ya) * k / p) * ly / M))
            inner[key] = ids
        ids = inner[key]
        return [vertex(*a)] + (ids if a < b else ids[::-1]) + [vertex(*b)]

    cells = sorted(leaves, key=lambda c: (box(c)[1], box(c)[0], c[0]))   # rows bottom to top
    lines, ptr, centres = [], [0], []
    for c in cells:
        X, Y, s = box(c)
        h = s // 2
        corners = [(X, Y), (X + s, Y), (X + s, Y + s), (X, Y + s)]
        # a side gets its midpoint when the cell across it is finer
        finer = [Y > 0 and lev[X, Y - 1] > c[0],
                 X + s < M and lev[X + s, Y] > c[0],
                 Y + s < M and lev[X, Y + s] > c[0],
                 X > 0 and lev[X - 1, Y] > c[0]]
        mids = [(X + h, Y), (X + s, Y + h), (X + h, Y + s), (X, Y + h)]
        loop = []
        for k in range(4):
            loop.append(corners[k])
            if finer[k]:
                loop.append(mids[k])
        for k in range(len(loop)):
            lines.append(segment(loop[k], loop[(k + 1) % len(loop)]))
        ptr.append(len(lines))
        centres.append(((X + s / 2) * lx / M, (Y + s / 2) * ly / M))
    return QuadtreeMesh(np.asarray(xy, dtype=np.float64), np.asarray(ptr, dtype=np.int64),
                        np.asarray(lines, dtype=np.int64), np.asarray(centres, dtype=np.float64), p, lx, ly,
                        base, levels, np.asarray(cells, dtype=np.int64))


def min_spacing(mesh) -> float:
    """Smallest distance between consecutive nodes of any line element."""
    ln = mesh.line_nodes
    d = np.hypot(*(mesh.node_xy[ln[:, 1:]] - mesh.node_xy[ln[:, :-1]]).transpose(2, 0, 1))
    return float(d.min())


@dataclass
class PolygonMesh:
    """Convex polygonal S-elements (centroidal Voronoi cells), same arrays as
    ``StructuredMesh``: element e owns one straight line element of order p per polygon
    side, counter-clockwise around its centroid."""
    node_xy: np.ndarray
    elem_ptr: np.ndarray
    line_nodes: np.ndarray
    centre_xy: np.ndarray
    p: int
    lx: float
    ly: float
    seeds: np.ndarray

    @property
    def n_nodes(self) -> int:
        return int(self.node_xy.shape[0])

    @property
    def n_elem(self) -> int:
        return int(self.centre_xy.shape[0])

    @property
    def n_b(self) -> np.ndarray:
        return self.p * np.diff(self.elem_ptr)


def _polygon_centroid(V):
    x, y = V[:, 0], V[:, 1]
    xs, ys = np.roll(x, -1), np.roll(y, -1)
    cr = x * ys - xs * y
    a = cr.sum() / 2
    return np.array([((x + xs) * cr).sum() / (6 * a), ((y + ys) * cr).sum() / (6 * a)])


def voronoi_mesh(n_cells: int, p: int, lx: float = 1.0, ly: float = 1.0, seed: int = 0, lloyd_iters: int = 40,
                 min_edge: float = 0.2) -> PolygonMesh:
    """Centroidal Voronoi tessellation of [0, lx] x [0, ly] into ``n_cells`` convex polygons
    (the mesh type of the paper's experiments, Section 4).

    Seeds are drawn uniformly and moved to their cells' centroids ``lloyd_iters`` times
    (Lloyd's algorithm); cells are bounded by mirroring the seeds across the four sides.
    Sides shorter than ``min_edge`` times the mean cell size sqrt(lx ly / n) are collapsed
    (their two vertices merged: at a domain vertex or side if one lies there, else at the
    midpoint), so no line element is much shorter than the rest.  Each polygon side is one
    line element of order p with equally spaced nodes; scaling centres are the centroids.
    """
    from scipy.spatial import Voronoi

    if n_cells < 2 or p < 1:
        raise ValueError("n_cells >= 2, p >= 1")
    rng = np.random.default_rng(seed)
    pts = rng.random((n_cells, 2)) * [lx, ly]
    for it in range(lloyd_iters + 1):
        allp = np.concatenate([pts, pts * [-1, 1], pts * [1, -1], np.c_[2 * lx - pts[:, 0], pts[:, 1]],
                               np.c_[pts[:, 0], 2 * ly - pts[:, 1]]])
        vor = Voronoi(allp)
        regions = [vor.regions[vor.point_region[i]] for i in range(n_cells)]
        if it == lloyd_iters:
            break
        pts = np.array([_polygon_centroid(vor.vertices[r]) for r in regions])
    V = vor.vertices.copy()
    tol = 1e-9 * max(lx, ly)
    V[np.abs(V[:, 0]) < tol, 0] = 0.0
    V[np.abs(V[:, 0] - lx) < tol, 0] = lx
    V[np.abs(V[:, 1]) < tol, 1] = 0.0
    V[np.abs(V[:, 1] - ly) < tol, 1] = ly
    # counter-clockwise vertex loops
    cells = []
    for r in regions:
        c = V[r].mean(axis=0)
        ang = np.arctan2(V[r, 1] - c[1], V[r, 0] - c[0])
        cells.append([r[k] for k in np.argsort(ang)])
    on_x = lambda v: V[v, 0] == 0.0 or V[v, 0] == lx
    on_y = lambda v: V[v, 1] == 0.0 or V[v, 1] == ly
    # collapse short sides
    h = np.sqrt(lx * ly / n_cells)
    parent = list(range(V.shape[0]))

    def find(v):
        while parent[v] != v:
            parent[v] = parent[parent[v]]
            v = parent[v]
        return v

    changed = True
    while changed:
        changed = False
        for cell in cells:
            loop = [find(v) for v in cell]
            loop = [v for k, v in enumerate(loop) if v != loop[k - 1]] if len(set(loop)) > 1 else loop
            for k in range(len(loop)):
                a, b = loop[k], loop[(k + 1) % len(loop)]
                if a == b or np.hypot(*(V[a] - V[b])) >= min_edge * h:
                    continue
                ca, cb = on_x(a) + on_y(a), on_x(b) + on_y(b)    # 2: domain vertex, 1: on a side
                if ca == 2 and cb == 2:
                    continue
                if ca > cb or (ca == cb and ca == 1 and (on_x(a) != on_x(b))):
                    keep, drop = a, b
                elif cb > ca:
                    keep, drop = b, a
                else:
                    keep, drop = a, b
                    if ca == 0:
                        V[a] = 0.5 * (V[a] + V[b])
                parent[drop] = keep
                changed = True
                break
    loops = []
    for cell in cells:
        loop = [find(v) for v in cell]
        loop = [v for k, v in enumerate(loop) if v != loop[k - 1]]
        loops.append(loop)
    used = sorted({v for loop in loops for v in loop})
    ren = {v: k for k, v in enumerate(used)}
    xy = [tuple(V[v]) for v in used]
    inner = {}

    def segment(a, b):
        key = (min(a, b), max(a, b))
        if key not in inner:
            (xa, ya), (xb, yb) = xy[key[0]], xy[key[1]]
            ids = []
            for k in range(1, p):
                ids.append(len(xy))
                xy.append((xa + (xb - xa) * k / p, ya + (yb - ya) * k / p))
            inner[key] = ids
        ids = inner[key]
        return [a] + (ids if a < b else ids[::-1]) + [b]

    lines, ptr, centres = [], [0], []
    for loop in loops:
        lp = [ren[v] for v in loop]
        for k in range(len(lp)):
            lines.append(segment(lp[k], lp[(k + 1) % len(lp)]))
        ptr.append(len(lines))
        centres.append(_polygon_centroid(np.array([xy[v] for v in lp])))
    return PolygonMesh(np.asarray(xy, dtype=np.float64), np.asarray(ptr, dtype=np.int64),
                       np.asarray(lines, dtype=np.int64), np.asarray(centres, dtype=np.float64), p, lx, ly, pts)
