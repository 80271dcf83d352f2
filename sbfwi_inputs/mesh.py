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
