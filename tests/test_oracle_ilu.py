"""Pins for oracle/ilu.py: the ILU(0) base smoother of the paper's smoother comparison (Sections 4.1 and 5;
Eq. local_smoother with M_l = M_ILU(0) and n_st stages).

ILU(0) has a plain definition: L unit lower and U upper triangular, both supported on the pattern P, with
(LU)_ij = A_ij on P.  These tests check that definition on the output (not the elimination that produced
it), the pattern against the voxel connectivity it is defined by, and two closed forms: exactness where P is
closed under elimination, and the error propagation of n_st stages.
"""
import numpy as np
import pytest

import synth
from oracle import fem, precond
from oracle.ilu import ILU0, ILU0Smoother, structural_pattern


def _system(mask, E=None, nu=0.3):
    mask = np.asarray(mask, np.uint8)
    if E is None:
        E = np.ones(mask.shape)
    return fem.System(mask, E, nu, synth.bcs_clamped_traction())


@pytest.fixture(scope="module")
def porous():
    p = synth.make_workload("tiny8", 3)
    return fem.System(p.mask, p.E, p.nu, p.bcs)


def _on_pattern(M, P):
    """Entries of the dense matrix M at the stored positions of the CSR pattern P."""
    rows = np.repeat(np.arange(P.shape[0]), np.diff(P.indptr))
    return M[rows, P.indices]


def test_lu_equals_a_on_the_pattern(porous):
    # the definition of ILU(0): (LU)_ij = A_ij for (i, j) in P, L and U zero off P
    S = ILU0Smoother(porous)
    A = porous.A.toarray()
    L = S.ilu.L.toarray()
    U = S.ilu.U.toarray()
    P = S.P
    Pd = P.toarray() != 0
    assert np.allclose(np.diag(L), 1.0) and np.abs(np.triu(L, 1)).max() == 0.0 and np.abs(np.tril(U, -1)).max() == 0.0
    assert np.abs(L[~Pd]).max() == 0.0 and np.abs(U[~Pd]).max() == 0.0
    LU = L @ U
    scale = np.abs(A).max()
    assert np.abs(_on_pattern(LU, P) - _on_pattern(A, P)).max() <= 1e-12 * scale
    # ... and it is an incomplete factorisation: LU differs from A off P (the dropped fill)
    assert np.abs(LU[~Pd]).max() > 1e-6 * scale


def test_pattern_is_the_voxel_connectivity():
    # a full 3x3x3 block clamped at z = 0: the interior node (x, y, z) = (1, 1, 2) of the 4^3 node grid couples
    # to its 27 neighbours (3 x 27 = 81 DOFs), the interior node (1, 1, 1) to the 18 of them above the clamped
    # face (54), a corner node of the top face (3, 3, 3) to 8 nodes (24 DOFs); the pattern is symmetric and
    # contains A's numerical nonzeros (grid_to_node is indexed [z, y, x])
    sysm = _system(np.ones((3, 3, 3)))
    P = structural_pattern(sysm)
    counts = np.diff(P.indptr)
    g2f = sysm.full_to_free
    node = sysm.mesh.grid_to_node
    assert counts[g2f[3 * node[2, 1, 1]]] == 81
    assert counts[g2f[3 * node[1, 1, 1]]] == 54
    assert counts[g2f[3 * node[3, 3, 3] + 2]] == 24
    assert (P != P.T).nnz == 0
    A = sysm.A.tocoo()
    Pd = P.toarray() != 0
    assert Pd[A.row, A.col].all()
    # P also holds positions where the assembled A is exactly zero (structural, not numerical)
    assert P.nnz > sysm.A.nnz


def test_exact_on_a_one_voxel_column():
    # one voxel wide: every node of layer z shares a voxel with every node of layers z-1, z, z+1, so the fill
    # created by eliminating a node lies inside P: ILU(0) is the exact LU and one application solves A x = b
    rng = np.random.default_rng(3)
    sysm = _system(np.ones((6, 1, 1)), E=np.exp(rng.standard_normal((6, 1, 1))))
    S = ILU0Smoother(sysm)
    A = sysm.A.toarray()
    assert np.abs(S.ilu.L.toarray() @ S.ilu.U.toarray() - A).max() <= 1e-12 * np.abs(A).max()
    x = S.apply(sysm.b)
    assert np.linalg.norm(A @ x - sysm.b) <= 1e-12 * np.linalg.norm(sysm.b)


def test_two_voxel_row_is_not_exact():
    # two voxels wide: nodes x = 0 and x = 2 share no voxel, yet eliminating x = 1 couples them -- dropped
    sysm = _system(np.ones((3, 1, 2)))
    S = ILU0Smoother(sysm)
    A = sysm.A.toarray()
    assert np.abs(S.ilu.L.toarray() @ S.ilu.U.toarray() - A).max() > 1e-6 * np.abs(A).max()


def test_small_dense_case_matches_gaussian_elimination_with_dropping():
    # an independent formulation on a dense copy: right-looking (KIJ) elimination over the whole matrix,
    # updating only positions in P; same result as the row-oriented form in exact arithmetic
    rng = np.random.default_rng(7)
    mask = np.ones((2, 2, 2))
    mask[1, 1, 1] = 0
    sysm = _system(mask, E=np.exp(rng.standard_normal((2, 2, 2))))
    P = structural_pattern(sysm)
    Pd = P.toarray() != 0
    W = sysm.A.toarray().copy()
    W[~Pd] = 0.0
    n = W.shape[0]
    for k in range(n):
        for i in range(k + 1, n):
            if Pd[i, k]:
                W[i, k] /= W[k, k]
                for j in range(k + 1, n):
                    if Pd[i, j]:
                        W[i, j] -= W[i, k] * W[k, j]
    F = ILU0(sysm.A, P).F.toarray()
    assert np.abs(F - W).max() <= 1e-12 * np.abs(W).max()


def test_stages_compose_as_error_propagation():
    # Eq. local_smoother with n_st stages of one base smoother: I - M_L^{-1} A = (I - M_l^{-1} A)^{n_st}
    p = synth.make_workload("tiny6", 2)
    for n_st in (1, 3, 6):
        sysm, M = precond.build(p, precond.Options(n_mortar=2, contact_halfwidth=1, smoother="ilu0", n_st=n_st))
        n = sysm.n_dof
        A = sysm.A.toarray()
        I = np.eye(n)
        ML = np.stack([M.M_L(e) for e in I], axis=1)
        Ml = np.stack([M.smoother.apply(e) for e in I], axis=1)
        E1 = I - Ml @ A
        assert np.abs((I - ML @ A) - np.linalg.matrix_power(E1, n_st)).max() < 1e-10
        # and the two-level M with it: I - M^{-1} A = (I - M_L^{-1} A)(I - M_G^{-1} A) (Eq. error_prop)
        Minv = np.stack([M.apply(e) for e in I], axis=1)
        MG = np.stack([M.M_G(e) for e in I], axis=1)
        assert np.abs((I - Minv @ A) - (I - ML @ A) @ (I - MG @ A)).max() < 1e-10


def test_ilu_preconditioner_converges():
    # hPLMM with the ILU(0) smoother (n_st = 6) still solves the system (the paper finds it slower than with
    # M_CG, not divergent, on all but its highest-contrast image)
    from oracle import gmres
    p = synth.make_workload("tiny8", 3)
    sysm, M = precond.build(p, precond.Options(n_mortar=2, contact_halfwidth=1, smoother="ilu0", n_st=6))
    x, st = gmres.gmres(sysm.A, sysm.b, M.apply, tol=1e-10)
    assert np.linalg.norm(sysm.b - sysm.A @ x) <= 1e-10 * np.linalg.norm(sysm.b) * 1.001
