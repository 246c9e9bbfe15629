"""Grain grids, contact interfaces and the permutation W (paper Sections 3.1,
3.2 and 4.2, Eqs. WQP, permute, permute_blk_1/2).

ORACLE -- test infrastructure only (see oracle/__init__.py).

Readings of points the paper leaves open:
* Cartesian decomposition (Section 3.1): voxel (i,j,k) belongs to grain
  gx + px*(gy + py*gz) with gx = floor(i*px/nx), etc.
* S(node) = set of grains owning the node's solid adjacent voxels.  |S| = 1:
  the node is interior to that grain.  |S| >= 2: the node lies on a contact
  interface; Section 3.2 states an interface is shared by exactly two grains,
  so a node touching three or more grains (3D edges and corners) is given to
  the pair (min S, second-smallest S).
* Two grains may share several disconnected interfaces (Section 3.2): the
  interface nodes of one pair are split into connected components, two nodes
  being adjacent when they are corners of a common solid voxel.  Each
  component is one contact interface Gamma^{c_j}.
* Interface nodes must carry at least one free DOF (fully clamped nodes are
  not unknowns).
* Interfaces are ordered by (pair, smallest node id); W orders the free DOFs
  as grain 0 interior, ..., grain N^g-1 interior, interface 0, ..., each set
  in node order with components x,y,z inside a node (Eq. permute).
* Grain grid g is coupled to interface c when a node of c is a corner of a
  solid voxel of g (this contains every g with A^g_c != 0, so the discrete
  harmonic extension is exact); `strict_two_grain` keeps only the pair.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from scipy.sparse.csgraph import connected_components

BIG = np.iinfo(np.int64).max


def cartesian_partition(shape, grains):
    """Grain id per voxel for a (px,py,pz) Cartesian slicing of an (nz,ny,nx) image."""
    nz, ny, nx = shape
    px, py, pz = grains
    gx = (np.arange(nx) * px) // nx
    gy = (np.arange(ny) * py) // ny
    gz = (np.arange(nz) * pz) // nz
    return (gx[None, None, :] + px * (gy[None, :, None] + py * gz[:, None, None])).astype(np.int64)


class Decomposition:
    """Node classes, interfaces, W and grain/interface couplings."""

    def __init__(self, system, grain_of_voxel, n_grains, strict_two_grain=False):
        mesh = system.mesh
        self.n_grains = int(n_grains)
        nz, ny, nx = mesh.nz, mesh.ny, mesh.nx
        gpad = np.full((nz + 2, ny + 2, nx + 2), BIG, np.int64)
        gpad[1:-1, 1:-1, 1:-1] = np.where(mesh.solid, np.asarray(grain_of_voxel, np.int64), BIG)
        ii, jj, kk = mesh.node_ijk[:, 0], mesh.node_ijk[:, 1], mesh.node_ijk[:, 2]
        G8 = np.empty((mesh.n_nodes, 8), np.int64)
        t = 0
        for dk in (0, 1):
            for dj in (0, 1):
                for di in (0, 1):
                    G8[:, t] = gpad[kk + dk, jj + dj, ii + di]
                    t += 1
        G8.sort(axis=1)
        self.G8 = G8
        valid = G8 != BIG
        distinct = valid.copy()
        distinct[:, 1:] &= G8[:, 1:] != G8[:, :-1]
        nS = distinct.sum(axis=1)
        smin = G8[:, 0]
        other = valid & (G8 != smin[:, None])
        second = np.where(nS >= 2, G8[np.arange(mesh.n_nodes), np.argmax(other, axis=1)], -1)
        self.nS = nS
        self.smin = smin
        self.second = second

        has_free = (~system.fixed).any(axis=1)
        self.is_interface_node = (nS >= 2) & has_free
        self.is_grain_node = (nS == 1) & has_free

        # connected components of interface nodes of the same pair
        iface = self.is_interface_node
        pairkey = np.where(iface, smin * self.n_grains + second, -1)
        rows, cols = [], []
        conn = mesh.conn
        for a in range(8):
            for b in range(a + 1, 8):
                na, nb = conn[:, a], conn[:, b]
                ok = iface[na] & iface[nb] & (pairkey[na] == pairkey[nb])
                rows.append(na[ok])
                cols.append(nb[ok])
        rows = np.concatenate(rows)
        cols = np.concatenate(cols)
        graph = sp.coo_matrix((np.ones(rows.size), (rows, cols)), shape=(mesh.n_nodes, mesh.n_nodes))
        _, label = connected_components(graph, directed=False)
        inodes = np.flatnonzero(iface)
        # smallest node id of each component
        comp_min = np.full(label.max() + 1, BIG, np.int64)
        np.minimum.at(comp_min, label[inodes], inodes)
        root = comp_min[label[inodes]]
        keys = np.stack([smin[inodes], second[inodes], root], axis=1)
        uniq, inv = np.unique(keys, axis=0, return_inverse=True)   # lexicographic (a, b, min node)
        inv = inv.ravel()
        self.n_interfaces = uniq.shape[0]
        self.iface_pair = uniq[:, :2].copy()
        self.iface_root = uniq[:, 2].copy()
        self.iface_of_node = np.full(mesh.n_nodes, -1, np.int64)
        self.iface_of_node[inodes] = inv
        self.iface_nodes = [inodes[inv == c] for c in range(self.n_interfaces)]   # ascending node ids
        self.grain_of_node = np.where(self.is_grain_node, smin, -1)

        # free DOFs of each class, in node order, components inside a node
        full_to_free = system.full_to_free
        def dofs_of(nodes):
            d = (3 * nodes[:, None] + np.arange(3)[None, :]).ravel()
            f = full_to_free[d]
            return f[f >= 0]
        order_g = np.argsort(self.grain_of_node[self.is_grain_node], kind="stable")
        gnodes_all = np.flatnonzero(self.is_grain_node)[order_g]
        gid_sorted = self.grain_of_node[gnodes_all]
        self.grain_nodes = [gnodes_all[gid_sorted == g] for g in range(self.n_grains)]
        self.grain_dofs = [dofs_of(n) for n in self.grain_nodes]
        self.iface_dofs = [dofs_of(n) for n in self.iface_nodes]
        self.W = np.concatenate(self.grain_dofs + self.iface_dofs) if system.n_dof else np.zeros(0, np.int64)

        # couplings between grains and interfaces
        self.strict_two_grain = bool(strict_two_grain)
        coupled = []
        for c in range(self.n_interfaces):
            if strict_two_grain:
                gs = np.array(sorted(set(self.iface_pair[c].tolist())), np.int64)
            else:
                g8 = G8[self.iface_nodes[c]].ravel()
                gs = np.unique(g8[g8 != BIG])
            coupled.append(gs)
        self.iface_grains = coupled
        self.grain_ifaces = [[] for _ in range(self.n_grains)]
        for c, gs in enumerate(coupled):
            for g in gs:
                self.grain_ifaces[int(g)].append(c)
