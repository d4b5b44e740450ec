"""Structured subdomain meshes (test infrastructure; see ``oracle/__init__``).

Sec. 2.4 asks for a triangulation of each of Omega^P and Omega^E; Sec. 4.1 uses uniform
triangulations of the unit square.  The project partitions [0,1]^2 into an
``nsub_x`` x ``nsub_y`` grid of rectangular subdomains, numbered row-major from the
bottom (subdomain ``s = cy * nsub_x + cx``).  Partition row ``cy`` has ``cells_y[cy]``
cells vertically and partition column ``cx`` has ``cells_x[cx]`` cells horizontally, so
meshes match across every interface.  Each cell is cut by its '/' diagonal into the
triangles (v00, v10, v11) and (v00, v11, v01); element ``e = 2 * (j * nx + i) + t``.

Displacement nodes of order k live on the grid ``(k*nx+1) x (k*ny+1)`` (P2: vertices and
edge midpoints; P1: vertices); scalar P1 nodes on ``(nx+1) x (ny+1)``.  Node keys are
global grid indices, so a node shared by several subdomains has one key.

Pinned by tests/test_oracle_fem.py (areas sum to the domain, shared keys coincide in
coordinates).
"""
import numpy as np


class SubMesh:
    """Mesh of one subdomain."""

    def __init__(self, case, s):
        self.s = s
        self.cx = s % case.nsub_x
        self.cy = s // case.nsub_x
        self.nx = int(case.cells_x[self.cx])
        self.ny = int(case.cells_y[self.cy])
        self.k = int(case.order_k)
        self.x0 = self.cx / case.nsub_x
        self.x1 = (self.cx + 1) / case.nsub_x
        self.y0 = self.cy / case.nsub_y
        self.y1 = (self.cy + 1) / case.nsub_y
        self.hx = (self.x1 - self.x0) / self.nx
        self.hy = (self.y1 - self.y0) / self.ny
        self.is_poro = self.cy < case.poro_rows
        k = self.k
        # global grid offsets (u-node grid of order k, and P1 grid)
        self.I0 = k * int(sum(case.cells_x[: self.cx]))
        self.J0 = k * int(sum(case.cells_y[: self.cy]))
        self.i0 = int(sum(case.cells_x[: self.cx]))
        self.j0 = int(sum(case.cells_y[: self.cy]))
        self.nux = k * self.nx + 1
        self.nuy = k * self.ny + 1
        self.npx = self.nx + 1
        self.npy = self.ny + 1
        self.n_unode = self.nux * self.nuy
        self.n_pnode = self.npx * self.npy
        self._build_elements()

    # node coordinates -------------------------------------------------------------
    def unode_xy(self):
        I = np.arange(self.nux)
        J = np.arange(self.nuy)
        X = self.x0 + I * (self.hx / self.k)
        Y = self.y0 + J * (self.hy / self.k)
        XX, YY = np.meshgrid(X, Y)  # (nuy, nux)
        return XX.ravel(), YY.ravel()

    def pnode_xy(self):
        X = self.x0 + np.arange(self.npx) * self.hx
        Y = self.y0 + np.arange(self.npy) * self.hy
        XX, YY = np.meshgrid(X, Y)
        return XX.ravel(), YY.ravel()

    def unode_key(self, a):
        """Global (I, J) key of local u-node index a = J * nux + I."""
        return (self.I0 + a % self.nux, self.J0 + a // self.nux)

    def pnode_key(self, a):
        return (self.i0 + a % self.npx, self.j0 + a // self.npx)

    # elements ---------------------------------------------------------------------
    def _build_elements(self):
        nx, ny, k = self.nx, self.ny, self.k
        ne = 2 * nx * ny
        verts = np.zeros((ne, 3), dtype=np.int64)   # P1 node indices
        unodes = np.zeros((ne, 3 if k == 1 else 6), dtype=np.int64)
        for j in range(ny):
            for i in range(nx):
                v00 = j * self.npx + i
                v10 = v00 + 1
                v01 = v00 + self.npx
                v11 = v01 + 1
                e = 2 * (j * nx + i)
                verts[e] = (v00, v10, v11)
                verts[e + 1] = (v00, v11, v01)

                def U(I, J):
                    return J * self.nux + I
                if k == 1:
                    unodes[e] = (U(i, j), U(i + 1, j), U(i + 1, j + 1))
                    unodes[e + 1] = (U(i, j), U(i + 1, j + 1), U(i, j + 1))
                else:
                    I, J = 2 * i, 2 * j
                    # vertices a, b, c then midpoints (a,b), (b,c), (c,a)
                    unodes[e] = (U(I, J), U(I + 2, J), U(I + 2, J + 2),
                                 U(I + 1, J), U(I + 2, J + 1), U(I + 1, J + 1))
                    unodes[e + 1] = (U(I, J), U(I + 2, J + 2), U(I, J + 2),
                                     U(I + 1, J + 1), U(I + 1, J + 2), U(I, J + 1))
        self.elem_p = verts
        self.elem_u = unodes
        px, py = self.pnode_xy()
        self.elem_xy = np.stack([np.stack([px[verts[:, c]], py[verts[:, c]]], axis=-1)
                                 for c in range(3)], axis=1)  # (ne, 3, 2)


def build_meshes(case):
    return [SubMesh(case, s) for s in range(case.nsub_x * case.nsub_y)]
