"""Structured 3-D meshes of hexahedral scaled-boundary elements (input generation only).

An element is a box cell with its scaling centre at the cell centre; its boundary is
the six faces, each a quadrilateral surface element of Lagrange order p with
(p+1)^2 nodes in tensor order: node (a, b) of a face sits at index a + (p+1) b, a
counting along the face's first direction (eta) and b along its second (zeta).  The
two directions are chosen so that eta x zeta points out of the element (the scaling
centre sees every face from its inner side).  Only nodes that lie on some face exist
(an S-element has no interior nodes); they are numbered in lattice order.
"""

from dataclasses import dataclass

import numpy as np


@dataclass
class StructuredMesh3D:
    node_xyz: np.ndarray      # (n_nodes, 3)
    elem_ptr: np.ndarray      # (n_elem+1,) element e owns faces elem_ptr[e]..elem_ptr[e+1]-1
    face_nodes: np.ndarray    # (n_faces, (p+1)^2) global node ids, tensor order
    centre_xyz: np.ndarray    # (n_elem, 3)
    p: int
    lx: float
    ly: float
    lz: float
    nx: int
    ny: int
    nz: int

    dim = 3

    @property
    def n_nodes(self) -> int:
        return int(self.node_xyz.shape[0])

    @property
    def n_elem(self) -> int:
        return int(self.centre_xyz.shape[0])


# (fixed axis, side, eta axis, zeta axis): eta x zeta is the outward normal
_FACES = [(0, 0, 2, 1), (0, 1, 1, 2), (1, 0, 0, 2), (1, 1, 2, 0), (2, 0, 1, 0), (2, 1, 0, 1)]


def structured_mesh3d(nx: int, ny: int, nz: int, p: int, lx: float = 1.0, ly: float = 1.0,
                      lz: float = 1.0) -> StructuredMesh3D:
    """nx x ny x nz box S-elements on [0, lx] x [0, ly] x [0, lz], faces of order p."""
    if min(nx, ny, nz, p) < 1:
        raise ValueError("nx, ny, nz, p must be >= 1")
    NX, NY, NZ = nx * p + 1, ny * p + 1, nz * p + 1
    lattice = lambda i, j, k: (k * NY + j) * NX + i
    pp = p + 1
    faces, centres = [], []
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                lo = (i * p, j * p, k * p)
                centres.append(((i + 0.5) * lx / nx, (j + 0.5) * ly / ny, (k + 0.5) * lz / nz))
                for axis, side, ea, za in _FACES:
                    ids = np.empty(pp * pp, dtype=np.int64)
                    for b in range(pp):
                        for a in range(pp):
                            c = list(lo)
                            c[axis] += side * p
                            c[ea] += a
                            c[za] += b
                            ids[a + pp * b] = lattice(*c)
                    faces.append(ids)
    faces = np.array(faces)
    used = np.unique(faces)
    renum = np.full(NX * NY * NZ, -1, dtype=np.int64)
    renum[used] = np.arange(used.size)
    kk, rem = np.divmod(used, NX * NY)
    jj, ii = np.divmod(rem, NX)
    xyz = np.stack([ii * (lx / (nx * p)), jj * (ly / (ny * p)), kk * (lz / (nz * p))], axis=1)
    E = nx * ny * nz
    return StructuredMesh3D(xyz, np.arange(0, 6 * E + 1, 6, dtype=np.int64), renum[faces],
                            np.array(centres, dtype=np.float64), p, lx, ly, lz, nx, ny, nz)


def boundary_nodes3d(mesh: StructuredMesh3D, side: str) -> np.ndarray:
    """Global ids of the nodes on one face of the box domain ('x0', 'x1', 'y0', 'y1',
    'z0', 'z1'), in lattice order."""
    axis = "xyz".index(side[0])
    ext = (mesh.lx, mesh.ly, mesh.lz)[axis]
    target = 0.0 if side[1] == "0" else ext
    tol = 1e-12 * max(mesh.lx, mesh.ly, mesh.lz)
    return np.nonzero(np.abs(mesh.node_xyz[:, axis] - target) < tol)[0]


def nearest_node3d(mesh: StructuredMesh3D, ids: np.ndarray, point) -> int:
    d = np.linalg.norm(mesh.node_xyz[ids] - np.asarray(point)[None, :], axis=1)
    return int(ids[int(np.argmin(d))])


def flawed_density_sphere(gx, gy, gz, lx=1.0, ly=1.0, lz=1.0, rho0=1.0, radius=0.15, factor=0.5, seed=0):
    """rho[gz, gy, gx] on cell centres: homogeneous rho0 with one spherical flaw (rho0 *
    factor inside), its centre drawn uniformly at least one radius clear of the faces."""
    rng = np.random.default_rng(seed)
    c = [rng.uniform(2 * radius, L - 2 * radius) for L in (lx, ly, lz)]
    zc = (np.arange(gz) + 0.5) * (lz / gz)
    yc = (np.arange(gy) + 0.5) * (ly / gy)
    xc = (np.arange(gx) + 0.5) * (lx / gx)
    Z, Y, X = np.meshgrid(zc, yc, xc, indexing="ij")
    rho = np.full((gz, gy, gx), float(rho0))
    rho[(X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2 <= radius ** 2] *= factor
    return rho, {"centre": tuple(c), "radius": radius, "factor": factor}
