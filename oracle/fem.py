"""Q1 finite elements on a voxel image (paper Section 2).

ORACLE -- test infrastructure only (see oracle/__init__.py).

* Eq. stiff_iso: isotropic stiffness from the Lame parameters
  lambda = E nu / ((1+nu)(1-2nu)), mu = E / (2(1+nu)).
* Eq. ls_all: Galerkin FEM with trilinear shape functions on unit voxels gives
  the symmetric system A_hat x_hat = b_hat.
* Eq. BC: Dirichlet displacements are eliminated from the unknowns (their
  coupling moves to the right-hand side); traction-free Neumann elsewhere; a
  uniform traction on a face adds t*h^2/4 to each corner node of every solid
  voxel face on that plane (the consistent load of a bilinear face).

Conventions (readings of points the paper leaves open):
* voxel (i,j,k) is mask[k, j, i]; node (i,j,k) in [0,nx]x[0,ny]x[0,nz] exists
  when one of its <= 8 adjacent voxels is solid; voxel size h = 1;
* element corner a = ax + 2 ay + 4 az sits at (i+ax, j+ay, k+az);
* Voigt order (xx, yy, zz, yz, xz, xy) with engineering shear strains;
* 2x2x2 Gauss-Legendre quadrature (exact for Q1 on a cube);
* nodes are numbered in lexicographic order (x fastest) over existing nodes;
  free DOFs node-major: (x,y,z) components of node 0, then node 1, ...
* faces are processed in the order x0,x1,y0,y1,z0,z1; a later face overrides
  the prescribed value of a component an earlier face also fixes.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

FACES = ("x0", "x1", "y0", "y1", "z0", "z1")


def lame(E, nu):
    """Eq. stiff_iso Lame parameters."""
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    return lam, mu


def elasticity_matrix(E, nu):
    """6x6 Voigt form of C_ijkl = lam d_ij d_kl + mu (d_ik d_jl + d_il d_jk)."""
    lam, mu = lame(E, nu)
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    for d in range(3):
        D[d, d] += 2.0 * mu
        D[3 + d, 3 + d] = mu
    return D


def corner_offset(a):
    return (a & 1, (a >> 1) & 1, (a >> 2) & 1)


def shape_gradients(xi):
    """Gradients of the 8 trilinear shape functions on the unit cube at point xi=(x,y,z)."""
    G = np.zeros((8, 3))
    for a in range(8):
        c = corner_offset(a)
        f = [xi[d] if c[d] else 1.0 - xi[d] for d in range(3)]
        s = [1.0 if c[d] else -1.0 for d in range(3)]
        G[a, 0] = s[0] * f[1] * f[2]
        G[a, 1] = f[0] * s[1] * f[2]
        G[a, 2] = f[0] * f[1] * s[2]
    return G


def strain_matrix(G):
    """B (6x24): Voigt strain from the 24 corner displacements (node-major, xyz)."""
    B = np.zeros((6, 24))
    for a in range(8):
        gx, gy, gz = G[a]
        c = 3 * a
        B[0, c] = gx
        B[1, c + 1] = gy
        B[2, c + 2] = gz
        B[3, c + 1] = gz
        B[3, c + 2] = gy
        B[4, c] = gz
        B[4, c + 2] = gx
        B[5, c] = gy
        B[5, c + 1] = gx
    return B


def reference_stiffness(nu, order=2):
    """K_ref(nu) = int_[0,1]^3 B^T D(E=1,nu) B dV by Gauss-Legendre quadrature."""
    x, w = np.polynomial.legendre.leggauss(order)
    x = 0.5 * (x + 1.0)
    w = 0.5 * w
    D = elasticity_matrix(1.0, nu)
    K = np.zeros((24, 24))
    for a in range(order):
        for b in range(order):
            for c in range(order):
                B = strain_matrix(shape_gradients((x[a], x[b], x[c])))
                K += w[a] * w[b] * w[c] * (B.T @ D @ B)
    return K


class Mesh:
    """Existing nodes and solid elements of a voxel mask."""

    def __init__(self, mask):
        mask = np.asarray(mask)
        self.nz, self.ny, self.nx = mask.shape
        nz, ny, nx = mask.shape
        self.solid = mask.astype(bool)
        pad = np.zeros((nz + 2, ny + 2, nx + 2), bool)
        pad[1:-1, 1:-1, 1:-1] = self.solid
        exists = np.zeros((nz + 1, ny + 1, nx + 1), bool)
        for dk in (0, 1):
            for dj in (0, 1):
                for di in (0, 1):
                    exists |= pad[dk:dk + nz + 1, dj:dj + ny + 1, di:di + nx + 1]
        self.exists = exists
        self.grid_to_node = np.full(exists.shape, -1, np.int64)
        self.n_nodes = int(exists.sum())
        self.grid_to_node[exists] = np.arange(self.n_nodes)
        kk, jj, ii = np.nonzero(exists)          # C order = lexicographic, x fastest
        self.node_ijk = np.stack([ii, jj, kk], axis=1)
        ek, ej, ei = np.nonzero(self.solid)
        self.elem_ijk = np.stack([ei, ej, ek], axis=1)
        self.n_elem = ek.size
        conn = np.empty((self.n_elem, 8), np.int64)
        for a in range(8):
            ox, oy, oz = corner_offset(a)
            conn[:, a] = self.grid_to_node[ek + oz, ej + oy, ei + ox]
        assert (conn >= 0).all()
        self.conn = conn

    def elem_dofs(self):
        return (3 * self.conn[:, :, None] + np.arange(3)[None, None, :]).reshape(self.n_elem, 24)


def assemble_full(mesh, E, nu):
    """A over all 3*n_nodes DOFs (no BCs): sum_e E_e K_ref(nu), Eq. ls_all."""
    K = reference_stiffness(nu)
    Ee = np.asarray(E, np.float64)[mesh.elem_ijk[:, 2], mesh.elem_ijk[:, 1], mesh.elem_ijk[:, 0]]
    dofs = mesh.elem_dofs()
    n = 3 * mesh.n_nodes
    A = sp.csr_matrix((n, n))
    chunk = 1 << 16
    for s in range(0, mesh.n_elem, chunk):
        d = dofs[s:s + chunk]
        rows = np.repeat(d, 24, axis=1).ravel()
        cols = np.tile(d, (1, 24)).ravel()
        vals = (Ee[s:s + chunk, None, None] * K[None, :, :]).ravel()
        A = A + sp.coo_matrix((vals, (rows, cols)), shape=(n, n)).tocsr()
    return A


def face_nodes(mesh, face):
    """Existing node ids on a face plane of the image box."""
    ax = "xyz".index(face[0])
    side = face[1] == "1"
    lim = (mesh.nx, mesh.ny, mesh.nz)[ax]
    sel = mesh.node_ijk[:, ax] == (lim if side else 0)
    return np.flatnonzero(sel)


def boundary_data(mesh, bcs):
    """Fixed-component mask, prescribed values and traction loads per node (n_nodes x 3)."""
    fixed = np.zeros((mesh.n_nodes, 3), bool)
    uD = np.zeros((mesh.n_nodes, 3))
    f = np.zeros((mesh.n_nodes, 3))
    for face in FACES:
        spec = bcs.get(face)
        if spec is None:
            continue
        nodes = face_nodes(mesh, face)
        for d in range(3):
            if spec["fix"][d]:
                fixed[nodes, d] = True
                uD[nodes, d] = spec["value"][d]
        t = np.asarray(spec["traction"], np.float64)
        if np.any(t != 0.0):
            ax = "xyz".index(face[0])
            side = face[1] == "1"
            lim = (mesh.nx, mesh.ny, mesh.nz)[ax]
            layer = lim - 1 if side else 0
            sel = np.flatnonzero(mesh.elem_ijk[:, ax] == layer)
            for a in range(8):
                if corner_offset(a)[ax] == (1 if side else 0):
                    np.add.at(f, mesh.conn[sel, a], t * 0.25)
    return fixed, uD, f


class System:
    """The eliminated free-DOF system A_hat x_hat = b_hat of Eq. ls_all."""

    def __init__(self, mask, E, nu, bcs):
        self.mesh = Mesh(mask)
        self.nu = float(nu)
        self.E = np.asarray(E, np.float64)
        A = assemble_full(self.mesh, self.E, nu)
        fixed, uD, f = boundary_data(self.mesh, bcs)
        self.fixed = fixed
        self.uD = uD
        fixed_flat = fixed.ravel()
        self.free = np.flatnonzero(~fixed_flat)          # full DOF index of each free DOF
        self.dirichlet = np.flatnonzero(fixed_flat)
        self.n_dof = self.free.size
        Acsr = A.tocsr()
        self.A_full = Acsr
        self.A = Acsr[self.free][:, self.free].tocsr()
        self.b = f.ravel()[self.free] - Acsr[self.free][:, self.dirichlet] @ uD.ravel()[self.dirichlet]
        self.full_to_free = np.full(3 * self.mesh.n_nodes, -1, np.int64)
        self.full_to_free[self.free] = np.arange(self.n_dof)

    def expand(self, x):
        """Free-DOF vector -> full nodal displacement (n_nodes x 3) including Dirichlet values."""
        u = self.uD.ravel().copy()
        u[self.free] = x
        return u.reshape(-1, 3)
