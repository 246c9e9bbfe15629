"""Pins for oracle/smoother.py, oracle/precond.py, oracle/gmres.py and
oracle/accuracy.py (paper Sections 4.1, 4.3, 5 and Eqs. multi_precond,
local_smoother_CG, Mg_Mz, error_prop, err_metric)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synth
from oracle import accuracy, fem, gmres, precond
from oracle.smoother import contact_grid_nodes


@pytest.fixture(scope="module")
def tiny():
    p = synth.make_workload("tiny6", 2)
    return precond.build(p, precond.Options(n_mortar=2, contact_halfwidth=1))


def _dense(op, n):
    return np.stack([op(e) for e in np.eye(n)], axis=1)


def test_error_propagation_split(tiny):
    # Eq. error_prop: I - M^{-1} A = (I - M_L^{-1} A)(I - M_G^{-1} A), a consequence of Eq. multi_precond
    sysm, M = tiny
    n = sysm.n_dof
    A = sysm.A.toarray()
    Minv = _dense(M.apply, n)
    MG = _dense(M.M_G, n)
    ML = _dense(M.M_L, n)
    I = np.eye(n)
    E = (I - ML @ A) @ (I - MG @ A)
    assert np.abs((I - Minv @ A) - E).max() < 1e-10
    # (the paper reports rho(E) < 1 on its own domains; with the heavy contact-grid overlap at the
    # edges of 3-voxel Cartesian grains the additive M_zeta overshoots, so rho is not asserted here)


def test_contact_grain_split(tiny):
    # Eq. local_smoother_CG: I - M_CG^{-1} A = (I - M_g^{-1} A)(I - M_zeta^{-1} A)
    sysm, M = tiny
    n = sysm.n_dof
    A = sysm.A.toarray()
    S = M.smoother
    Mcg = _dense(S.apply, n)
    Mz = _dense(S.M_zeta, n)
    Mg = _dense(S.M_g, n)
    I = np.eye(n)
    assert np.abs((I - Mcg @ A) - (I - Mg @ A) @ (I - Mz @ A)).max() < 1e-10


def test_schwarz_local_exactness(tiny):
    # additive Schwarz with exact local solves: for v supported on subdomain i alone,
    # (M^{-1} A v) restricted to that subdomain equals v when no other subdomain overlaps it
    sysm, M = tiny
    S = M.smoother
    rng = np.random.default_rng(0)
    for sets, op in ((S.grain_sets, S.M_g),):
        for I in sets[:3]:
            v = np.zeros(sysm.n_dof)
            v[I] = rng.standard_normal(I.size)
            z = op(sysm.A @ v)
            assert np.allclose(z[I], v[I], atol=1e-10 * np.abs(v).max())


def test_contact_grid_local_exactness():
    # M_zeta with exact local solves on principal submatrices of A_hat (Eq. local_smoother_CG): on a bar cut
    # into three grains along x, the two contact grids (w = 1) are disjoint, so for v supported on one grid,
    # (M_zeta A v) restricted to that grid is v itself; a dropped grid gives 0 there, a wrong submatrix
    # (not principal, or a missing coupling) gives something else
    shape = (4, 4, 12)                                            # [z][y][x]
    bcs = synth.bcs_clamped_traction(traction=(0.0, 0.0, 1.0))
    p = synth.Problem("bar", np.ones(shape, np.uint8), np.linspace(0.5, 2.0, 192).reshape(shape).astype(np.float32),
                      0.3, (3, 1, 1), bcs, 2, 0)
    sysm, M = precond.build(p, precond.Options(n_mortar=2, contact_halfwidth=1))
    S = M.smoother
    assert len(S.contact_sets) == 2
    a, b = (set(np.asarray(c).tolist()) for c in S.contact_sets)
    assert not (a & b)
    rng = np.random.default_rng(1)
    for I in S.contact_sets:
        I = np.asarray(I)
        v = np.zeros(sysm.n_dof)
        v[I] = rng.standard_normal(I.size)
        z = S.M_zeta(sysm.A @ v)
        assert np.allclose(z[I], v[I], atol=1e-10 * np.abs(v).max())
        # and the grid is the L-inf dilation (w = 1) of its interface plane: three node layers in x
        xs = sysm.mesh.node_ijk[sysm.free[I] // 3, 0]
        assert xs.max() - xs.min() == 2 and xs.min() in (3, 7)


def test_contact_grid_is_linf_dilation():
    mask = np.ones((5, 5, 5), np.uint8)
    m = fem.Mesh(mask)
    centre = m.grid_to_node[2, 2, 2]
    nodes = contact_grid_nodes(m, np.array([centre]), 1)
    assert nodes.size == 27
    nodes = contact_grid_nodes(m, np.array([m.grid_to_node[0, 0, 0]]), 2)
    assert nodes.size == 27     # clipped at the box corner: 3x3x3


def test_single_grain_is_a_direct_solve():
    # one grain covering every free DOF: the correction column alone reproduces x, and the grain
    # smoother is the exact inverse, so GMRES converges in one step
    p = synth.make_workload("tiny6", 1)
    p.grains = (1, 1, 1)
    sysm, M = precond.build(p, precond.Options(n_mortar=2, contact_halfwidth=1))
    xs = spla.spsolve(sysm.A.tocsc(), sysm.b)
    assert np.linalg.norm(M.M_G(sysm.b) - xs) < 1e-10 * np.linalg.norm(xs)
    x, st = gmres.gmres(sysm.A, sysm.b, M.apply, tol=1e-10)
    assert st["iters"] == 1


@pytest.mark.parametrize("name,seed", [("tiny6", 0), ("tiny8", 4)])
def test_gmres_matches_dense_solve(name, seed):
    p = synth.make_workload(name, seed)
    sysm, M = precond.build(p)
    xs = np.linalg.solve(sysm.A.toarray(), sysm.b)
    x, st = gmres.gmres(sysm.A, sysm.b, M.apply, tol=1e-12)
    assert st["converged"]
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) < 1e-10


def test_gmres_restart_and_cap():
    rng = np.random.default_rng(3)
    n = 60
    Q = np.linalg.qr(rng.standard_normal((n, n)))[0]
    A = Q @ np.diag(np.linspace(1, 50, n)) @ Q.T
    b = rng.standard_normal(n)
    ident = lambda v: v.copy()
    x, st = gmres.gmres(A, b, ident, tol=1e-10, restart=5, max_iters=2000)
    assert st["converged"] and np.linalg.norm(A @ x - b) <= 1e-10 * np.linalg.norm(b) * 1.0001
    x, st = gmres.gmres(A, b, ident, tol=1e-14, restart=5, max_iters=7)
    assert not st["converged"] and st["iters"] == 7


def test_more_mortars_fewer_iterations():
    # the paper's qualitative trend (Table wct): n = 4 converges faster than n = 1 (PLMM)
    p = synth.make_workload("cube16", 0)
    its = {}
    for n in (1, 4):
        sysm, M = precond.build(p, precond.Options(n_mortar=n, contact_halfwidth=1))
        its[n] = gmres.gmres(sysm.A, sysm.b, M.apply, tol=1e-8)[1]["iters"]
    assert its[4] < its[1]


def test_max_shear_of_uniaxial_stress():
    # uniaxial tension sigma: principal stresses (sigma, 0, 0) -> max shear sigma/2 in every voxel
    shape = (3, 2, 2)
    bcs = {f: {"fix": (False,) * 3, "value": (0,) * 3, "traction": (0,) * 3} for f in fem.FACES}
    bcs["x0"] = {"fix": (True, False, False), "value": (0,) * 3, "traction": (0,) * 3}
    bcs["y0"] = {"fix": (False, True, False), "value": (0,) * 3, "traction": (0,) * 3}
    bcs["z0"] = {"fix": (False, False, True), "value": (0,) * 3, "traction": (0,) * 3}
    bcs["z1"] = {"fix": (False,) * 3, "value": (0,) * 3, "traction": (0, 0, 0.8)}
    sysm = fem.System(np.ones(shape, np.uint8), np.full(shape, 2.0), 0.3, bcs)
    x = spla.spsolve(sysm.A.tocsc(), sysm.b)
    S = accuracy.centroid_stress(sysm, x)
    assert np.allclose(S[:, 2, 2], 0.8, atol=1e-12)
    assert np.allclose(accuracy.max_shear(S), 0.4, atol=1e-12)
    eu, es = accuracy.e2_errors(sysm, x, x)
    assert eu == 0.0 and es == 0.0
    eu, _ = accuracy.e2_errors(sysm, 0.5 * x, x)
    u = sysm.expand(x)
    un = np.linalg.norm(u, axis=1)
    assert eu == pytest.approx(0.5 * np.sqrt(np.mean(un ** 2)) / un.max(), rel=1e-12)
