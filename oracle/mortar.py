"""Mortar nodes, Gaussian mortar functions and the reduction block Q^o
(paper Section 3.3, Eqs. node_init and gauss; Section 4.2, Eq. reduced_defs).

ORACLE -- test infrastructure only (see oracle/__init__.py).

Mortar placement (Section 3.3).  The N^m_c mortar nodes of interface c are
chosen among its FEM nodes F^c, treated as like charges:
  1. the first two are the farthest pair of F^c;
  2. each further node minimises sum_{j<=i} 1/||y - x_j|| over the remaining
     nodes (Eq. node_init);
  3. sweeps then move each node in turn to the minimiser of the same energy
     summed over all other nodes, until a sweep changes nothing.
Readings: distances are in node-index units (h = 1); sweeps visit nodes in
ascending mortar index (the paper says "random order"), at most 100 sweeps;
every tie goes to the smallest node id (pairs: smallest (id_a, id_b)).
N^m_c = min(n, |F^c|); when N^m_c = |F^c| every node is a mortar; when it is
1 the node nearest the centroid is taken (its position does not matter since
the mortar function is then identically 1).  Energies are summed in
ascending mortar index; squared distances are exact integers.

Gaussian mortars (Eq. gauss): alpha_i(y) = exp(-||y-x_i||^2 / (beta *
min_{j != i} ||x_i - x_j||^2)) (the j = i term would be zero, so it is
excluded) and eta_i = alpha_i / sum_j alpha_j, evaluated as a softmax of the
exponents (algebraically identical).  eta_{i,gamma} = eta_i e_gamma in the
global xyz frame: because a Gaussian mortar is the same scalar on every
component, the span of {eta_i e_gamma} does not depend on the interface's
local (n, m) frame.

Algebraic mortars (Eq. algebra, and the Remark after Eq. reduced_defs): the column (mortar i, component
gamma) of interface c is the displacement field on the interface's free DOFs that equals 1 at DOF
(x_i, gamma), 0 at every other mortar DOF, and solves S^c w = 0 on the remaining DOFs: the rows and columns
of the mortar DOFs are removed, the column of the unit DOF moved to the right-hand side, and the reduced
system solved (a dense solve, as a library primitive).  S^c stands for the interface's own elasticity
operator of Eq. algebra, built from A_hat alone: for every pair of distinct interface nodes {y, y'} that
A_hat couples, the edge term (e_y - e_y')(e_y - e_y')^T (x) B_yy', where B_yy' = |-(A_yy' + A_yy'^T)/2|
(the matrix absolute value: eigenvectors kept, eigenvalues replaced by their magnitudes) and A_yy' is the
3x3 block of A_hat (zero where a DOF is fixed); then ALG_SHIFT times A_hat's diagonal is added.  Without
the shift S^c is symmetric positive semidefinite and annihilates rigid translations of the interface, so
the mortars of one component sum to e_gamma (Eq. algebra's partition of unity "by superposition"), and
with one mortar the column is the rigid translation, as for PLMM.  Where A_hat's coupling is attractive
(-sym(A_yy') positive semidefinite) the edge term carries A_hat's own coupling.  The shift (1e-8 of the
diagonal) makes S^c positive definite on interface pieces that carry no mortar node and moves the sums
away from e_gamma by about 1e-6 at most on the tested interfaces.  Other readings and why they were
left: the literal principal submatrix A^c_c (the Remark) gives mortars that decay within a node or two of
their mortar node; A^c_c with each diagonal block shifted by its block-row sum is not positive definite
where the couplings of the normal component between in-plane neighbours are positive (the normal-gradient
part of the 3D stiffness); and clipping negative eigenvalues instead of taking magnitudes leaves the
normal component of a planar interface coupled only along diagonals (a checkerboard of two decoupled
halves, one without mortars).  A column (i, gamma) exists only when DOF
(x_i, gamma) is free (a fixed DOF cannot carry the unit value).

Q^o (Eq. reduced_defs) is block-diagonal per interface: rows are the free
interface DOFs in W order, columns are (interface, mortar i, component gamma)
in that nesting order.  A column with no free DOF (every node of the
interface has component gamma fixed) is dropped, since it would make the
coarse matrix singular.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

MAX_SWEEPS = 100
ALG_SHIFT = 1e-8   # diagonal shift of the algebraic mortars' interface operator, relative to A_hat's diagonal


def _d2(P, q):
    d = P - q[None, :]
    return (d * d).sum(axis=1)


def _energy(coords, chosen, exclude_index=None):
    """sum_j 1/||y - x_j|| over the chosen mortars (skipping one index), summed in ascending j."""
    acc = np.zeros(coords.shape[0])
    for j, m in enumerate(chosen):
        if j == exclude_index:
            continue
        d2 = _d2(coords, coords[m]).astype(np.float64)
        with np.errstate(divide="ignore"):
            acc = acc + 1.0 / np.sqrt(d2)
    return acc


def _argmin_excluding(values, forbidden):
    v = values.copy()
    v[list(forbidden)] = np.inf
    return int(np.argmin(v))          # first occurrence = smallest node id on ties


def place_mortars(coords, n):
    """Indices (into the ascending node list of the interface) of its mortar nodes."""
    coords = np.asarray(coords, np.int64)
    F = coords.shape[0]
    nc = min(n, F)
    if nc == F:
        return list(range(F))
    if nc == 1:
        # nearest to the centroid: minimise ||F*y - sum(coords)||^2 in exact integers
        s = coords.sum(axis=0)
        return [int(np.argmin(_d2(F * coords, s)))]
    best, ia, ib = -1, 0, 0
    for a in range(F):
        d2 = _d2(coords[a + 1:], coords[a])
        if d2.size:
            j = int(np.argmax(d2))
            if d2[j] > best:
                best, ia, ib = int(d2[j]), a, a + 1 + j
    chosen = [ia, ib]
    while len(chosen) < nc:
        chosen.append(_argmin_excluding(_energy(coords, chosen), chosen))
    for _ in range(MAX_SWEEPS):
        changed = False
        for i in range(nc):
            others = [m for j, m in enumerate(chosen) if j != i]
            new = _argmin_excluding(_energy(coords, chosen, exclude_index=i), others)
            if new != chosen[i]:
                chosen[i] = new
                changed = True
        if not changed:
            break
    return chosen


def gaussian_mortars(coords, chosen, beta=4.0):
    """eta[y, i] for every interface node y and mortar i (Eq. gauss)."""
    coords = np.asarray(coords, np.int64)
    nc = len(chosen)
    F = coords.shape[0]
    if nc == 1:
        return np.ones((F, 1))
    X = coords[chosen]
    dmin2 = np.empty(nc)
    for i in range(nc):
        d2 = _d2(X, X[i]).astype(np.float64)
        d2[i] = np.inf
        dmin2[i] = d2.min()
    a = np.empty((F, nc))
    for i in range(nc):
        a[:, i] = -_d2(coords, X[i]).astype(np.float64) / (beta * dmin2[i])
    a -= a.max(axis=1, keepdims=True)
    e = np.exp(a)
    return e / e.sum(axis=1, keepdims=True)


class Mortars:
    """Mortar nodes, eta weights and Q^o for every interface of a decomposition."""

    def __init__(self, system, dec, n, beta=4.0, kind="gaussian"):
        mesh = system.mesh
        self.n = int(n)
        self.beta = float(beta)
        if kind not in ("gaussian", "algebraic"):
            raise ValueError(kind)
        self.kind = kind
        self._alg = {}
        self.mortar_nodes = []     # per interface: global node ids of its mortars, in mortar order
        self.eta = []              # per interface: |F^c| x n_c weights
        self.columns = []          # per interface: list of (mortar i, component gamma) kept
        fixed = system.fixed
        for c in range(dec.n_interfaces):
            nodes = dec.iface_nodes[c]
            coords = mesh.node_ijk[nodes]
            chosen = place_mortars(coords, self.n)
            self.mortar_nodes.append(nodes[chosen])
            self.eta.append(gaussian_mortars(coords, chosen, self.beta))
            if kind == "gaussian":
                free_comp = (~fixed[nodes]).any(axis=0)
                self.columns.append([(i, g) for i in range(len(chosen)) for g in range(3) if free_comp[g]])
            else:
                self.columns.append([(i, g) for i in range(len(chosen)) for g in range(3)
                                     if not fixed[nodes[chosen[i]], g]])
        self.iface_col_offset = np.zeros(dec.n_interfaces + 1, np.int64)
        for c in range(dec.n_interfaces):
            self.iface_col_offset[c + 1] = self.iface_col_offset[c] + len(self.columns[c])
        self.n_mortar_cols = int(self.iface_col_offset[-1])     # N^o_m

    def Qo_block(self, system, dec, c):
        """Dense block of Q^o for interface c: rows = its free DOFs (W order), cols = its kept columns."""
        nodes = dec.iface_nodes[c]
        rows = []
        for y, node in enumerate(nodes):
            for d in range(3):
                if not system.fixed[node, d]:
                    rows.append((y, d))
        if self.kind == "algebraic":
            return self._algebraic_block(system, dec, c, rows)
        Q = np.zeros((len(rows), len(self.columns[c])))
        for r, (y, d) in enumerate(rows):
            for k, (i, g) in enumerate(self.columns[c]):
                if g == d:
                    Q[r, k] = self.eta[c][y, i]
        return Q

    def _interface_operator(self, system, dec, c, rows):
        """S^c on the interface's free DOFs (rows in W order): a sum over coupled node pairs {y, y'} of
        (e_y - e_y')(e_y - e_y')^T (x) B_yy', B_yy' = |-(A_yy' + A_yy'^T)/2| (matrix absolute value; A_yy'
        the 3x3 block of A_hat, zero where a DOF is fixed), plus ALG_SHIFT times the diagonal of A_hat on
        those DOFs."""
        nodes = dec.iface_nodes[c]
        F = len(nodes)
        f2f = system.full_to_free
        J = np.array([f2f[3 * nodes[y] + d] for (y, d) in rows], np.int64)
        Acc = system.A[J][:, J].tocoo()
        # the interface block on all 3F node components, zero on fixed ones
        full_of_row = np.array([3 * y + d for (y, d) in rows], np.int64)
        Afull = np.zeros((3 * F, 3 * F))
        Afull[full_of_row[Acc.row], full_of_row[Acc.col]] = Acc.data
        ny, nz = full_of_row[Acc.row] // 3, full_of_row[Acc.col] // 3
        pairs = np.unique(np.stack([np.minimum(ny, nz), np.maximum(ny, nz)], axis=1), axis=0)
        pairs = pairs[pairs[:, 0] != pairs[:, 1]]
        S = np.zeros((3 * F, 3 * F))
        if len(pairs):
            blk = np.stack([Afull[3 * y:3 * y + 3, 3 * z:3 * z + 3] for (y, z) in pairs])
            B = -0.5 * (blk + blk.transpose(0, 2, 1))
            w, V = np.linalg.eigh(B)
            P = np.einsum("kij,kj,klj->kil", V, np.abs(w), V)
            for (y, z), Pk in zip(pairs, P):
                S[3 * y:3 * y + 3, 3 * y:3 * y + 3] += Pk
                S[3 * z:3 * z + 3, 3 * z:3 * z + 3] += Pk
                S[3 * y:3 * y + 3, 3 * z:3 * z + 3] -= Pk
                S[3 * z:3 * z + 3, 3 * y:3 * y + 3] -= Pk
        S = S[np.ix_(full_of_row, full_of_row)]
        S[np.diag_indices_from(S)] += ALG_SHIFT * system.A.diagonal()[J]
        return S

    def _algebraic_block(self, system, dec, c, rows):
        if c in self._alg:
            return self._alg[c]
        S = self._interface_operator(system, dec, c, rows)
        mortar_y = set(np.flatnonzero(np.isin(dec.iface_nodes[c], self.mortar_nodes[c])).tolist())
        pos = {yd: r for r, yd in enumerate(rows)}
        is_m = np.array([y in mortar_y for (y, d) in rows], dtype=bool)
        R = np.flatnonzero(~is_m)
        chosen_y = [int(np.flatnonzero(dec.iface_nodes[c] == m)[0]) for m in self.mortar_nodes[c]]
        Q = np.zeros((len(rows), len(self.columns[c])))
        for k, (i, g) in enumerate(self.columns[c]):
            r1 = pos[(chosen_y[i], g)]
            Q[r1, k] = 1.0
            if R.size:
                Q[R, k] = -np.linalg.solve(S[np.ix_(R, R)], S[R, r1])
        self._alg[c] = Q
        return Q

    def Qo(self, system, dec):
        """Q^o as a sparse (N^f_c x N^o_m) matrix, rows in W order of the interface DOFs."""
        blocks = [sp.csr_matrix(self.Qo_block(system, dec, c)) for c in range(dec.n_interfaces)]
        if not blocks:
            return sp.csr_matrix((0, 0))
        return sp.block_diag(blocks, format="csr")
