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
system solved (a dense solve, as a library primitive).  S^c is the interface block A^c_c of A_hat (its
principal submatrix on the interface's free DOFs) with each node's 3x3 diagonal block reduced by that node's
block-row sum over the interface, so that S^c annihilates rigid translations of the interface -- the
property Eq. algebra states (its mortars sum to e_gamma "by superposition"); with one mortar per interface
the column is then the rigid translation, as for PLMM.  (The unshifted principal submatrix gives mortars
that decay within a node or two of their mortar node.)  A column (i, gamma) exists only when DOF
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

    def _algebraic_block(self, system, dec, c, rows):
        if c in self._alg:
            return self._alg[c]
        J = dec.iface_dofs[c]
        Acc = system.A[J][:, J].toarray()
        # S^c: each node's diagonal block minus its block-row sum over the interface (translations -> 0)
        node_of = np.array([y for (y, d) in rows], np.int64)
        comp_of = np.array([d for (y, d) in rows], np.int64)
        S = Acc.copy()
        for r in range(len(rows)):
            for g in range(3):
                same_g = comp_of == g
                diag = np.flatnonzero((node_of == node_of[r]) & same_g)
                if diag.size:
                    S[r, diag[0]] -= Acc[r, same_g].sum()
        Acc = S
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
                Q[R, k] = -np.linalg.solve(Acc[np.ix_(R, R)], Acc[R, r1])
        self._alg[c] = Q
        return Q

    def Qo(self, system, dec):
        """Q^o as a sparse (N^f_c x N^o_m) matrix, rows in W order of the interface DOFs."""
        blocks = [sp.csr_matrix(self.Qo_block(system, dec, c)) for c in range(dec.n_interfaces)]
        if not blocks:
            return sp.csr_matrix((0, 0))
        return sp.block_diag(blocks, format="csr")
