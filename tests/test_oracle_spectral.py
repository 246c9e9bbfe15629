"""Pins for oracle/spectral.py: the spectral k-way partition of a gray-scale image into grain grids (paper
Section 3.1, "Spectral partitioning").  Closed forms (eigenvalues and eigenvectors of the normalized Laplacian
of a path graph), the spectrum of blocks joined by compliant layers and the clusters it forces, k-means
against its own fixed-point conditions and brute force, and an hPLMM solve on a spectral partition.
"""
import itertools

import numpy as np
import pytest

import synth
from oracle import gmres, precond
from oracle.fem import System
from oracle.precond import HPLMM
from oracle.spectral import kmeans, normalized_laplacian, smallest_eigenvectors, spectral_partition, voxel_graph


def test_path_graph_spectrum():
    # a bar of n voxels with equal moduli is the path graph P_n: its normalized Laplacian has the eigenvalues
    # 1 - cos(pi j / (n - 1)), j = 0 .. n-1 (the end vertices have degree 1, the others 2)
    n = 9
    mask = np.ones((1, 1, n), np.uint8)
    W, solid = voxel_graph(mask, np.full(mask.shape, 3.0))
    lam = np.linalg.eigvalsh(normalized_laplacian(W).toarray())
    ref = 1.0 - np.cos(np.pi * np.arange(n) / (n - 1))
    assert np.abs(np.sort(lam) - np.sort(ref)).max() < 1e-12
    # the smallest eigenvector is D^{1/2} 1 (eigenvalue 0) up to scale and sign
    lam2, V = smallest_eigenvectors(normalized_laplacian(W), 2)
    d = np.asarray(W.sum(axis=1)).ravel()
    v0 = np.sqrt(d) / np.linalg.norm(np.sqrt(d))
    assert abs(lam2[0]) < 1e-12 and abs(abs(V[:, 0] @ v0) - 1.0) < 1e-12


def test_graph_weights_are_series_springs():
    # two voxels: one edge of weight 2 E_a E_b / (E_a + E_b); a void voxel breaks the bar
    W, _ = voxel_graph(np.ones((1, 1, 2), np.uint8), np.array([[[1.0, 3.0]]]))
    assert W.nnz == 2 and abs(W[0, 1] - 1.5) < 1e-15 and abs(W[1, 0] - 1.5) < 1e-15
    mask = np.ones((2, 2, 3), np.uint8)
    W, solid = voxel_graph(mask, np.ones(mask.shape))
    # 2x2x3 block: edges along x 2*2*2, along y 2*1*3, along z 1*2*3 -> 8 + 6 + 6 = 20, each stored twice
    assert W.nnz == 40 and solid.size == 12


def test_path_graph_eigenvectors_and_features():
    # the eigenvectors of the path's normalized Laplacian are D^{1/2} cos(pi j x / (n - 1)) at the voxels
    # x = 0 .. n-1 (distinct eigenvalues: unique up to sign); the partition's features are eigenvectors
    # 2 .. k+1 of the computed set, so a k = 2 partition of a bar clusters the curve (cos, cos 2x) -- whose
    # k-means optima are 6/4 splits for n = 10, not the halves, since the second feature folds the ends together
    n = 10
    mask = np.ones((1, 1, n), np.uint8)
    W, _ = voxel_graph(mask, np.ones(mask.shape))
    lam, V = smallest_eigenvectors(normalized_laplacian(W), 4)
    d = np.asarray(W.sum(axis=1)).ravel()
    x = np.arange(n)
    for j in range(4):
        ref = np.sqrt(d) * np.cos(np.pi * j * x / (n - 1))
        ref /= np.linalg.norm(ref)
        assert abs(lam[j] - (1.0 - np.cos(np.pi * j / (n - 1)))) < 1e-12
        assert abs(abs(V[:, j] @ ref) - 1.0) < 1e-12
    # with these seeds Lloyd's iteration reaches the global optimum, found by enumerating all bipartitions
    g = spectral_partition(mask, np.ones(mask.shape), 2, [0.1, 0.9])[0, 0]
    X = V[:, 1:3]

    def wcss(lab):
        return sum(((X[lab == j] - X[lab == j].mean(axis=0)) ** 2).sum() for j in range(2) if np.any(lab == j))
    best = min(wcss(np.array((0,) + t)) for t in itertools.product(range(2), repeat=n - 1) if 1 in t)
    assert abs(wcss(g) - best) < 1e-12
    assert sorted(np.bincount(g).tolist()) == [4, 6]


def _blocks(m, rng):
    """m stiff blocks along x joined by one-voxel layers with E x 1e-4 (the slits of the fractured images)."""
    widths = [5, 4, 6, 5][:m]
    nx = sum(widths) + (m - 1)
    mask = np.ones((3, 3, nx), np.uint8)
    E = np.exp(0.3 * rng.standard_normal(mask.shape))
    blocks, x = [], 0
    for b, w in enumerate(widths):
        blocks.append(slice(x, x + w))
        x += w
        if b + 1 < m:
            E[:, :, x] *= 1e-4
            x += 1
    return mask, E, blocks


@pytest.mark.parametrize("m", [2, 3])
def test_compliant_layers_spectrum(m):
    # m blocks joined by compliant layers: m eigenvalues near zero (the weak links cost ~1e-4), then a gap;
    # the corresponding random-walk vectors D^{-1/2} v are constant on every block
    mask, E, blocks = _blocks(m, np.random.default_rng(4))
    W, solid = voxel_graph(mask, E)
    lam, V = smallest_eigenvectors(normalized_laplacian(W), m + 1)
    assert lam[m - 1] < 1e-3 and lam[m] > 0.05
    d = np.asarray(W.sum(axis=1)).ravel()
    F = V[:, :m] / np.sqrt(d)[:, None]
    vox = np.full(mask.size, -1)
    vox[solid] = np.arange(solid.size)
    vox = vox.reshape(mask.shape)
    for sl in blocks:
        rows = F[vox[:, :, sl].ravel()]
        assert np.abs(rows - rows.mean(axis=0)).max() <= 1e-2 * np.abs(F).max()


@pytest.mark.parametrize("m,k", [(3, 2), (4, 3)])
def test_blocks_are_not_split(m, k):
    # with fewer grains than blocks (k = m - 1) every feature (eigenvectors 2 .. k+1) is a block mode, so each
    # block is a tight point cloud in feature space and falls into one cluster whole; the compliant voxels
    # join either side.  (With k = m the last feature is the first mode inside a block, and k-means may split
    # that block rather than cut a layer -- the recipe as the paper states it.)
    rng = np.random.default_rng(5)
    mask, E, blocks = _blocks(m, rng)
    g = spectral_partition(mask, E, k, rng.uniform(size=k))
    used = set()
    for sl in blocks:
        vals = np.unique(g[:, :, sl])
        assert vals.size == 1
        used.add(int(vals[0]))
    assert used == set(range(k))


def test_labels_void_and_order():
    p = synth.make_workload("tiny8", 3)
    k = 4
    g = spectral_partition(p.mask, p.E, k, np.random.default_rng(0).uniform(size=k))
    assert (g[p.mask == 0] == -1).all()
    labels = g[p.mask != 0]
    assert set(np.unique(labels)) == set(range(k))
    # labels numbered in order of first occurrence in voxel order
    firsts = [int(np.flatnonzero(labels == j)[0]) for j in range(k)]
    assert firsts == sorted(firsts)


def test_kmeans_fixed_point_and_brute_force():
    rng = np.random.default_rng(8)
    # three well-separated blobs in 2D
    X = np.concatenate([rng.normal(c, 0.05, size=(4, 2)) for c in ((0, 0), (1, 0), (0, 1))])
    label, C = kmeans(X, 3, rng.uniform(size=3))
    # fixed point of Lloyd's map: every point at its nearest centre, every centre its cluster's mean
    d = ((X[:, None, :] - C[None]) ** 2).sum(axis=2)
    assert np.array_equal(label, np.argmin(d, axis=1))
    for j in range(3):
        assert np.allclose(C[j], X[label == j].mean(axis=0), atol=1e-15)
    # the global optimum of the within-cluster sum of squares, by enumerating all partitions into 3 groups
    def wcss(lab):
        return sum(((X[lab == j] - X[lab == j].mean(axis=0)) ** 2).sum() for j in range(3) if np.any(lab == j))
    best = min(wcss(np.array((0,) + t)) for t in itertools.product(range(3), repeat=X.shape[0] - 1)
               if len(set((0,) + t)) == 3)
    assert abs(wcss(label) - best) < 1e-12


def test_hplmm_on_a_spectral_partition_converges():
    # a gray-scale (all solid, log-normal moduli) block partitioned spectrally into 8 grain grids: the
    # two-level preconditioner is built on it and GMRES reaches the tolerance
    rng = np.random.default_rng(2)
    shape = (8, 8, 8)
    mask = np.ones(shape, np.uint8)
    E = synth.lognormal_modulus(shape, 1.5, rng).astype(np.float64)
    k = 8
    g = spectral_partition(mask, E, k, rng.uniform(size=k))
    sysm = System(mask, E, 0.3, synth.bcs_clamped_traction())
    M = HPLMM(sysm, g, k, precond.Options(n_mortar=2, contact_halfwidth=1))
    x, st = gmres.gmres(sysm.A, sysm.b, M.apply, tol=1e-8)
    assert np.linalg.norm(sysm.b - sysm.A @ x) <= 1e-8 * np.linalg.norm(sysm.b) * 1.001
