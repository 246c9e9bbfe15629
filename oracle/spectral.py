"""Spectral k-way partition of a gray-scale voxel image into k grain grids (paper Section 3.1, "Spectral
partitioning"): the solid voxels become the vertices of a weighted graph; the k + 1 eigenvectors of its
normalized graph Laplacian with the smallest eigenvalues are computed and the first (eigenvalue zero) is
dropped; k-means clusters the vertices by their entries in the remaining k eigenvectors, and each cluster
is one grain grid.  The paper uses the k-way form, not recursive bisection.

ORACLE -- test infrastructure only (see oracle/__init__.py).

Readings (the paper refers elsewhere for the details):
* graph: one vertex per solid voxel; an edge between face neighbours (6-connectivity) weighted by the
  harmonic mean of the two moduli, 2 E_a E_b / (E_a + E_b) -- two springs in series -- so a compliant layer
  (a slit of E x 1e-4) is a weak link the partition cuts across, and a uniform image gives equal weights;
* Laplacian: L = I - D^{-1/2} W D^{-1/2} with D the diagonal of W's row sums;
* features: the raw entries of eigenvectors 2 .. k+1 of L (no row normalisation);
* k-means: Lloyd's iteration from k-means++ seeds whose k uniform random numbers are an input (the method's
  randomness is passed in); a vertex goes to the nearest centre, ties to the lower index; a cluster left
  empty takes the vertex farthest from its own centre (lowest index on ties); the iteration stops when no
  assignment changes (at most 300 sweeps);
* labels are renumbered in the order in which the clusters first occur in voxel order (z, y, x), void
  voxels get -1.

Pins (tests/test_oracle_spectral.py): the edge weights; the Laplacian's eigenvalues and eigenvectors on a
voxel bar against the closed forms of a path graph (1 - cos(pi j / (n - 1)), D^{1/2} cos(pi j x / (n - 1)))
and a two-way partition there equal to the brute-force k-means optimum of its features; blocks joined by
compliant layers: a near-zero eigenvalue per block, block-constant random-walk vectors, and no block split
when there are fewer grains than blocks; k-means at a fixed point of Lloyd's map and equal to brute force on
a small well-separated set; the label conventions; hPLMM built on a spectral partition converging.  Note
that the paper's recipe (k features, eigenvectors 2 .. k+1) makes its k-th feature the first mode inside a
block when an image has exactly k weakly linked blocks, and k-means may then split that block.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from scipy.sparse.linalg import eigsh


def voxel_graph(mask, E):
    """Symmetric CSR weight matrix W over the solid voxels (C order) and the voxel index of each vertex."""
    mask = np.asarray(mask).astype(bool)
    E = np.asarray(E, np.float64)
    vid = np.full(mask.shape, -1, np.int64)
    solid = np.flatnonzero(mask.ravel())
    vid.ravel()[solid] = np.arange(solid.size)
    rows, cols, vals = [], [], []
    for axis in range(3):
        a = [slice(None)] * 3
        b = [slice(None)] * 3
        a[axis] = slice(0, -1)
        b[axis] = slice(1, None)
        ok = mask[tuple(a)] & mask[tuple(b)]
        ea, eb = E[tuple(a)][ok], E[tuple(b)][ok]
        w = 2.0 * ea * eb / (ea + eb)
        ia, ib = vid[tuple(a)][ok], vid[tuple(b)][ok]
        rows += [ia, ib]
        cols += [ib, ia]
        vals += [w, w]
    n = solid.size
    W = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n)).tocsr()
    return W, solid


def normalized_laplacian(W):
    d = np.asarray(W.sum(axis=1)).ravel()
    if np.any(d <= 0):
        raise ValueError("the graph has an isolated vertex (a solid voxel without solid face neighbours)")
    s = sp.diags(1.0 / np.sqrt(d))
    return (sp.identity(W.shape[0]) - s @ W @ s).tocsr()


def smallest_eigenvectors(L, m):
    """The m smallest eigenpairs of the symmetric positive semidefinite L, ascending."""
    n = L.shape[0]
    if n <= 600 or m >= n - 1:
        lam, V = np.linalg.eigh(L.toarray())
        return lam[:m], V[:, :m]
    # shift-invert about a point just below the spectrum (L + 0.01 I is positive definite)
    lam, V = eigsh(L, k=m, sigma=-0.01, which="LM")
    order = np.argsort(lam)
    return lam[order], V[:, order]


def kmeans(X, k, u, max_sweeps=300):
    """Lloyd's k-means of the rows of X from k-means++ seeds drawn with the uniforms u[0..k-1]."""
    X = np.asarray(X, np.float64)
    n = X.shape[0]
    u = np.asarray(u, np.float64)
    centres = np.empty((k, X.shape[1]))
    centres[0] = X[min(int(u[0] * n), n - 1)]
    d2 = ((X - centres[0]) ** 2).sum(axis=1)
    for j in range(1, k):
        c = np.cumsum(d2)
        i = int(np.searchsorted(c, u[j] * c[-1], side="right"))
        centres[j] = X[min(i, n - 1)]
        d2 = np.minimum(d2, ((X - centres[j]) ** 2).sum(axis=1))
    label = None
    for _ in range(max_sweeps):
        dist = ((X[:, None, :] - centres[None, :, :]) ** 2).sum(axis=2)
        new = np.argmin(dist, axis=1)          # ties: lowest index
        for j in range(k):
            if not np.any(new == j):           # empty: take the vertex farthest from its own centre
                far = dist[np.arange(n), new]
                i = int(np.argmax(far))
                new[i] = j
        if label is not None and np.array_equal(new, label):
            break
        label = new
        for j in range(k):
            centres[j] = X[label == j].mean(axis=0)
    return label, centres


def spectral_partition(mask, E, k, u):
    """Grain id per voxel (-1 for void) of a k-way spectral partition of the solid voxels."""
    W, solid = voxel_graph(mask, E)
    if k == 1:
        label = np.zeros(solid.size, np.int64)
    else:
        L = normalized_laplacian(W)
        _, V = smallest_eigenvectors(L, k + 1)
        label, _ = kmeans(V[:, 1:], k, u)
    # renumber by first occurrence in voxel order
    first = {}
    for g in label:
        if g not in first:
            first[g] = len(first)
    out = np.full(np.asarray(mask).size, -1, np.int64)
    out[solid] = np.array([first[g] for g in label], np.int64)
    return out.reshape(np.asarray(mask).shape)
