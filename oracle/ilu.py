"""ILU(0) base smoother M_ILU(0): the black-box alternative to the contact-grain smoother that the paper
pairs with M_G in its smoother comparison (Section 4.1 names ILU(k) as a possible base smoother M_l of
Eq. local_smoother; Section 5 runs it with fill level k = 0 and n_st = 6 stages).

ORACLE -- test infrastructure only (see oracle/__init__.py).

Reading (the paper does not define the sparsity pattern): the pattern P of A_hat is structural.  Free DOFs
i and j are coupled when their nodes are corners of a common solid voxel, so entries of the element
matrices that happen to vanish still belong to P.  ILU(0) gives L (unit lower triangular) and U (upper
triangular), both supported on P, with (LU)_ij = A_ij for every (i, j) in P.  Rows are eliminated in the
free-DOF order of fem.System (node-major; nodes lexicographic, x fastest) by the row-oriented (IKJ) form
of Gaussian elimination, dropping every update that falls outside P (Saad, Iterative Methods for Sparse
Linear Systems, Section 10.3).  M_ILU(0)^{-1} r = U^{-1} L^{-1} r.

Pins (tests/test_oracle_ilu.py): (LU)_ij = A_ij on P and L, U vanish off P (the definition); P's row
counts on a full block (81 for an interior node) and its node-level symmetry; on a one-voxel column P is
closed under elimination, so ILU(0) is the exact LU and one stage solves A_hat x = b; the stage recursion
of Eq. local_smoother has error propagation (I - M_L^{-1} A) = (I - M_l^{-1} A)^{n_st}.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from scipy.sparse.linalg import spsolve_triangular


def structural_pattern(system):
    """Boolean CSR over the free DOFs (sorted columns): i ~ j when their nodes share a solid voxel."""
    mesh = system.mesh
    conn = mesh.conn
    rows = np.repeat(conn, 8, axis=1).ravel()
    cols = np.tile(conn, (1, 8)).ravel()
    nodes = sp.coo_matrix((np.ones(rows.size), (rows, cols)), shape=(mesh.n_nodes, mesh.n_nodes)).tocsr()
    nodes.data[:] = 1.0
    dofs = sp.kron(nodes, np.ones((3, 3)), format="csr")   # (3n + a, 3m + b) for coupled nodes n, m
    P = dofs[system.free][:, system.free].tocsr()
    P.sort_indices()
    P.data[:] = 1.0
    return P


class ILU0:
    """ILU(0) of A on the pattern P (both CSR over the same index set)."""

    def __init__(self, A, P):
        A = A.tocsr()
        n = A.shape[0]
        indptr, indices = P.indptr, P.indices
        val = np.zeros(indices.size)
        diag = np.full(n, -1, np.int64)
        w = np.zeros(n)
        for i in range(n):
            lo, hi = indptr[i], indptr[i + 1]
            cols = indices[lo:hi]
            a0, a1 = A.indptr[i], A.indptr[i + 1]
            w[A.indices[a0:a1]] = A.data[a0:a1]
            touched = [cols, A.indices[a0:a1]]
            # eliminate with every earlier row k in row i's pattern, in increasing k
            for k in cols[cols < i]:
                piv = val[diag[k]]
                if piv == 0.0:
                    raise ZeroDivisionError(f"ILU(0): zero pivot in row {k}")
                w[k] /= piv
                u0, u1 = diag[k] + 1, indptr[k + 1]
                ucols = indices[u0:u1]
                w[ucols] -= w[k] * val[u0:u1]          # positions outside P are never read: dropped
                touched.append(ucols)
            val[lo:hi] = w[cols]
            d = np.searchsorted(cols, i)
            if d >= cols.size or cols[d] != i:
                raise ValueError(f"ILU(0): row {i} has no diagonal in the pattern")
            diag[i] = lo + d
            for t in touched:
                w[t] = 0.0
        self.n = n
        self.F = sp.csr_matrix((val, indices.copy(), indptr.copy()), shape=(n, n))
        self.L = (sp.tril(self.F, -1) + sp.identity(n)).tocsr()
        self.U = sp.triu(self.F).tocsr()

    def apply(self, r):
        """z = U^{-1} L^{-1} r."""
        y = spsolve_triangular(self.L, r, lower=True, unit_diagonal=True)
        return spsolve_triangular(self.U, y, lower=False)


class ILU0Smoother:
    """M_ILU(0) over the free DOFs of a system (the base smoother M_l of Eq. local_smoother)."""

    def __init__(self, system):
        self.P = structural_pattern(system)
        self.ilu = ILU0(system.A, self.P)

    def apply(self, r):
        return self.ilu.apply(np.asarray(r, dtype=np.float64))
