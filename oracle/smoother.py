"""Contact-grain smoother M_CG (paper Section 4.3, Eqs. local_smoother_CG
and Mg_Mz; contact grids from Section 3.1).

ORACLE -- test infrastructure only (see oracle/__init__.py).

* Eq. Mg_Mz: both M_g and M_zeta are additive Schwarz operators
  sum_i E_i (R_i A_hat E_i)^{-1} R_i with exact local solves.
* Eq. local_smoother_CG: M_CG^{-1} = M_zeta^{-1} + M_g^{-1} (I - A_hat M_zeta^{-1}).
* Grain block i: the interior free DOFs of grain grid i (the same blocks
  A^{g_i}_{g_i} as the coarse space uses).
* Contact grid zeta_k (Section 3.1: a morphological dilation of interface
  c_k, not merged with its neighbours): every free DOF of the nodes within
  L-infinity node distance <= w of a node of c_k.  The paper uses 16 elements
  in total width for ~70-pixel grains; w is a parameter here.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla
from scipy import ndimage


def contact_grid_nodes(mesh, iface_nodes, w):
    """Node ids within L-infinity distance w of the given interface nodes (ascending)."""
    ijk = mesh.node_ijk[iface_nodes]
    lo = np.maximum(ijk.min(axis=0) - w, 0)
    hi = np.minimum(ijk.max(axis=0) + w, [mesh.nx, mesh.ny, mesh.nz])
    shape = (hi[2] - lo[2] + 1, hi[1] - lo[1] + 1, hi[0] - lo[0] + 1)
    box = np.zeros(shape, bool)
    box[ijk[:, 2] - lo[2], ijk[:, 1] - lo[1], ijk[:, 0] - lo[0]] = True
    if w > 0:
        box = ndimage.binary_dilation(box, structure=np.ones((2 * w + 1,) * 3, bool))
    kk, jj, ii = np.nonzero(box)
    ids = mesh.grid_to_node[kk + lo[2], jj + lo[1], ii + lo[0]]
    return np.sort(ids[ids >= 0])


class ContactGrainSmoother:
    def __init__(self, system, dec, coarse, w):
        A = system.A.tocsr()
        self.A = A
        self.w = int(w)
        self.grain_sets = []
        self.grain_lu = []
        for g in range(dec.n_grains):
            I = dec.grain_dofs[g]
            if I.size == 0:
                continue
            self.grain_sets.append(I)
            self.grain_lu.append(coarse.grain_lu[g])
        self.contact_sets = []
        self.contact_lu = []
        ftf = system.full_to_free
        for c in range(dec.n_interfaces):
            nodes = contact_grid_nodes(system.mesh, dec.iface_nodes[c], self.w)
            d = ftf[(3 * nodes[:, None] + np.arange(3)[None, :]).ravel()]
            Z = d[d >= 0]
            if Z.size == 0:
                continue
            self.contact_sets.append(Z)
            self.contact_lu.append(spla.splu(A[Z][:, Z].tocsc()))

    @staticmethod
    def _schwarz(sets, lus, r):
        z = np.zeros_like(r)
        for S, lu in zip(sets, lus):
            z[S] += lu.solve(r[S])
        return z

    def M_zeta(self, r):
        return self._schwarz(self.contact_sets, self.contact_lu, r)

    def M_g(self, r):
        return self._schwarz(self.grain_sets, self.grain_lu, r)

    def apply(self, r):
        """M_CG^{-1} r (Eq. local_smoother_CG): contact grids first, then grain grids."""
        z_zeta = self.M_zeta(r)
        r2 = r - self.A @ z_zeta
        return z_zeta + self.M_g(r2)
