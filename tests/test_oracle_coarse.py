"""Pins for oracle/coarse.py: the prolongation P_hat = W Q P and the coarse
operator (paper Section 4.2).  Checked against properties the definitions
fix: harmonic extension of each shape vector (Eq. col_pk), the correction
equation (Eq. col_cg), partition of unity of the interface rows, Galerkin
orthogonality, exact reproduction of a rigid translation, and exactness
when every interface node is a mortar (Appendix B)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synth
from oracle import fem, precond
from oracle.decomposition import cartesian_partition


def _setup(problem, **kw):
    opt = precond.Options(n_mortar=kw.pop("n", problem.n_mortar), **kw)
    return precond.build(problem, opt)


@pytest.fixture(scope="module")
def tiny():
    return _setup(synth.make_workload("tiny8", 3))


def test_coarse_matrix_symmetric_spd(tiny):
    sysm, M = tiny
    cs = M.coarse
    assert cs.asymmetry < 1e-12
    assert np.linalg.eigvalsh(cs.A_o).min() > 0


def test_shape_vectors_are_discrete_harmonic(tiny):
    # A_hat p_hat_k vanishes on every grain's interior DOFs for mortar columns (Eq. col_pk),
    # and equals b^g on grain g for the correction column of g (Eq. col_cg)
    sysm, M = tiny
    dec, cs = M.dec, M.coarse
    AP = (sysm.A @ cs.P_hat).toarray()
    Pd = cs.P_hat.toarray()
    scale = np.abs(sysm.A).max() * np.abs(Pd).max()
    grain_rows = np.concatenate([d for d in dec.grain_dofs if d.size])
    assert np.abs(AP[grain_rows, :cs.n_m]).max() < 1e-12 * scale
    for j, g in enumerate(cs.correction_grain):
        I = dec.grain_dofs[g]
        col = AP[:, cs.n_m + j]
        assert np.allclose(col[I], sysm.b[I], rtol=0, atol=1e-12 * scale)
        other = np.setdiff1d(grain_rows, I)
        assert np.abs(col[other]).max() < 1e-12 * scale


def test_interface_rows_partition_of_unity(tiny):
    # summing the mortar columns of component gamma gives e_gamma on every interface DOF
    sysm, M = tiny
    dec, cs = M.dec, M.coarse
    Pd = cs.P_hat.toarray()
    iface_rows = np.concatenate(dec.iface_dofs)
    comp = sysm.free[iface_rows] % 3
    for gamma in range(3):
        cols = [M.mortars.iface_col_offset[c] + k for c in range(dec.n_interfaces)
                for k, (i, g) in enumerate(M.mortars.columns[c]) if g == gamma]
        s = Pd[np.ix_(iface_rows, cols)].sum(axis=1)
        assert np.allclose(s, (comp == gamma).astype(float), atol=1e-14)


def test_galerkin_orthogonality(tiny):
    sysm, M = tiny
    xa = M.M_G(sysm.b)
    res = M.coarse.restrict(sysm.b - sysm.A @ xa)
    assert np.abs(res).max() < 1e-12 * np.abs(M.coarse.restrict(sysm.b)).max()


def _translation_problem(gamma, grains=(2, 2, 2), shape=(6, 6, 6), seed=0):
    rng = np.random.default_rng(seed)
    mask = synth.porous_mask(shape, 0.2, 1.0, rng)
    E = synth.lognormal_modulus(shape, 1.0, rng)
    bcs = synth.bcs_clamped_traction((0.0, 0.0, 0.0))
    v = [0.0, 0.0, 0.0]
    v[gamma] = 1.0
    bcs["z0"] = {"fix": (True, True, True), "value": tuple(v), "traction": (0.0,) * 3}
    return synth.Problem("translation", mask, E, 0.3, grains, bcs, 2, seed)


@pytest.mark.parametrize("gamma", [0, 1, 2])
@pytest.mark.parametrize("n", [1, 2, 4])
def test_first_pass_reproduces_rigid_translation(gamma, n):
    # a prescribed rigid translation with no load: the exact solution is the translation itself,
    # which lies in range(P_hat) (mortars sum to one; the grain corrections carry the Dirichlet data)
    p = _translation_problem(gamma)
    sysm, M = _setup(p, n=n)
    xa = M.M_G(sysm.b)
    expect = np.zeros((sysm.mesh.n_nodes, 3))
    expect[:, gamma] = 1.0
    assert np.abs(xa - expect.ravel()[sysm.free]).max() < 1e-10


def test_all_interface_nodes_as_mortars_is_exact():
    # Appendix B: with n >= every interface's node count, Q^o is square and P_hat spans the solution
    shape = (3, 3, 4)     # nz, ny, nx: two grains along x, one 4x4 node interface
    rng = np.random.default_rng(7)
    mask = np.ones(shape, np.uint8)
    E = synth.lognormal_modulus(shape, 1.0, rng)
    p = synth.Problem("two_grain", mask, E, 0.3, (2, 1, 1), synth.bcs_clamped_traction((0.3, -0.2, 1.0)), 64, 0)
    sysm, M = _setup(p, n=64)
    assert M.dec.n_interfaces == 1
    assert M.mortars.n_mortar_cols == 3 * len(M.dec.iface_nodes[0])
    xs = spla.spsolve(sysm.A.tocsc(), sysm.b)
    xa = M.M_G(sysm.b)
    assert np.linalg.norm(xa - xs) / np.linalg.norm(xs) < 1e-9


def test_strict_two_grain_equals_default_without_cross_points():
    shape = (3, 3, 6)
    rng = np.random.default_rng(8)
    mask = np.ones(shape, np.uint8)
    E = synth.lognormal_modulus(shape, 1.0, rng)
    p = synth.Problem("two_grain", mask, E, 0.3, (2, 1, 1), synth.bcs_clamped_traction(), 2, 0)
    _, M1 = _setup(p)
    _, M2 = _setup(p, strict_two_grain=True)
    assert np.abs((M1.coarse.P_hat - M2.coarse.P_hat)).max() == 0
