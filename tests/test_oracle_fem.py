"""Pins for oracle/fem.py: Q1 element stiffness, assembly, loads and Dirichlet
elimination (paper Section 2, Eqs. stiff_iso, BC, ls_all).

Each check rests on something other than the oracle's own formula: entries
of K_ref integrated by hand, the strain energy of a uniform strain, rigid-body
null vectors, and exact finite-element solutions (patch tests)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import fem

FACES = fem.FACES


def _bcs(**faces):
    out = {f: {"fix": (False,) * 3, "value": (0.0,) * 3, "traction": (0.0,) * 3} for f in FACES}
    out.update(faces)
    return out


@pytest.mark.parametrize("nu", [0.0, 0.25, 0.3, 0.45])
def test_kref_hand_integrated_entries(nu):
    # N_0 = (1-x)(1-y)(1-z): int (dN0/dx)^2 = 1/9, int dN0/dx dN0/dy = 1/12 over the unit cube,
    # so K[ux0,ux0] = (lam + 2mu + mu + mu)/9 and K[ux0,uy0] = (lam + mu)/12 (E = 1).
    lam, mu = fem.lame(1.0, nu)
    K = fem.reference_stiffness(nu)
    assert K[0, 0] == pytest.approx((lam + 4 * mu) / 9.0, rel=1e-14)
    assert K[0, 1] == pytest.approx((lam + mu) / 12.0, rel=1e-14)
    # corner 7 = (1,1,1) is the mirror image of corner 0: same diagonal, same coupling sign
    assert K[21, 21] == pytest.approx((lam + 4 * mu) / 9.0, rel=1e-14)
    assert K[21, 22] == pytest.approx((lam + mu) / 12.0, rel=1e-14)


def test_kref_symmetric_rank_18():
    K = fem.reference_stiffness(0.3)
    assert np.abs(K - K.T).max() < 1e-15
    ev = np.linalg.eigvalsh(K)
    assert (np.abs(ev) < 1e-12 * ev.max()).sum() == 6
    assert (ev > 1e-6).sum() == 18


def _corner_xyz():
    return np.array([fem.corner_offset(a) for a in range(8)], dtype=float)


def test_kref_rigid_modes_in_null_space():
    K = fem.reference_stiffness(0.27)
    X = _corner_xyz()
    for d in range(3):
        u = np.zeros((8, 3))
        u[:, d] = 1.0
        assert np.abs(K @ u.ravel()).max() < 1e-14
    for axis in np.eye(3):
        u = np.cross(axis, X - 0.5)              # infinitesimal rotation
        assert np.abs(K @ u.ravel()).max() < 1e-14


def test_kref_uniform_strain_energy():
    # u = G x: energy u^T K u = eps : C : eps over unit volume = lam tr(eps)^2 + 2 mu eps:eps
    rng = np.random.default_rng(3)
    nu = 0.31
    lam, mu = fem.lame(1.0, nu)
    K = fem.reference_stiffness(nu)
    X = _corner_xyz()
    for _ in range(5):
        G = rng.standard_normal((3, 3))
        eps = 0.5 * (G + G.T)
        u = X @ G.T
        e = u.ravel() @ K @ u.ravel()
        assert e == pytest.approx(lam * np.trace(eps) ** 2 + 2 * mu * np.sum(eps * eps), rel=1e-13)


def test_kref_quadrature_is_exact():
    assert np.abs(fem.reference_stiffness(0.3, 2) - fem.reference_stiffness(0.3, 3)).max() < 1e-14


def test_mesh_node_existence_and_numbering():
    mask = np.zeros((2, 2, 3), np.uint8)
    mask[0, 0, 0] = 1
    mask[1, 1, 2] = 1
    m = fem.Mesh(mask)
    assert m.n_nodes == 16                       # two isolated voxels, 8 corners each
    # lexicographic numbering, x fastest
    assert list(m.node_ijk[0]) == [0, 0, 0]
    assert list(m.node_ijk[1]) == [1, 0, 0]
    assert m.n_elem == 2


def test_unconstrained_matrix_rigid_null_space():
    rng = np.random.default_rng(0)
    mask = (rng.random((4, 5, 3)) < 0.8).astype(np.uint8)
    E = rng.uniform(0.5, 2.0, mask.shape)
    m = fem.Mesh(mask)
    A = fem.assemble_full(m, E, 0.3)
    X = m.node_ijk.astype(float)
    for d in range(3):
        u = np.zeros((m.n_nodes, 3))
        u[:, d] = 1
        assert np.abs(A @ u.ravel()).max() < 1e-12
    for axis in np.eye(3):
        u = np.cross(axis, X)
        assert np.abs(A @ u.ravel()).max() < 1e-11
    assert abs(A - A.T).max() < 1e-15


def test_patch_test_linear_dirichlet_field():
    # homogeneous block, all six faces prescribed u = G x + c: the FE solution is exact
    shape = (3, 4, 5)
    mask = np.ones(shape, np.uint8)
    E = np.full(shape, 2.5)
    G = np.array([[0.1, -0.2, 0.05], [0.3, 0.02, -0.1], [0.0, 0.15, 0.2]])
    c = np.array([0.5, -1.0, 0.25])
    m = fem.Mesh(mask)
    # build per-face prescribed values by running elimination with the exact field
    sysm = fem.System(mask, E, 0.3, _bcs(**{f: {"fix": (True,) * 3, "value": (0.0,) * 3,
                                                 "traction": (0.0,) * 3} for f in FACES}))
    exact = m.node_ijk.astype(float) @ G.T + c
    uD = sysm.uD.copy()
    uD[sysm.fixed.any(axis=1)] = exact[sysm.fixed.any(axis=1)]
    b = -sysm.A_full[sysm.free][:, sysm.dirichlet] @ uD.ravel()[sysm.dirichlet]
    x = spla.spsolve(sysm.A.tocsc(), b)
    assert np.abs(x - exact.ravel()[sysm.free]).max() < 1e-12


def test_uniaxial_traction_exact_solution():
    # rollers on x0 (ux), y0 (uy), z0 (uz); traction sigma e_z on z1 -> exact linear field
    shape = (4, 3, 2)        # nz, ny, nx
    mask = np.ones(shape, np.uint8)
    E0, nu, sig = 3.0, 0.28, 0.7
    bcs = _bcs(x0={"fix": (True, False, False), "value": (0, 0, 0), "traction": (0, 0, 0)},
               y0={"fix": (False, True, False), "value": (0, 0, 0), "traction": (0, 0, 0)},
               z0={"fix": (False, False, True), "value": (0, 0, 0), "traction": (0, 0, 0)},
               z1={"fix": (False, False, False), "value": (0, 0, 0), "traction": (0, 0, sig)})
    sysm = fem.System(mask, np.full(shape, E0), nu, bcs)
    x = spla.spsolve(sysm.A.tocsc(), sysm.b)
    u = sysm.expand(x)
    X = sysm.mesh.node_ijk.astype(float)
    exact = np.stack([-nu * sig * X[:, 0] / E0, -nu * sig * X[:, 1] / E0, sig * X[:, 2] / E0], axis=1)
    assert np.abs(u - exact).max() < 1e-12


def test_traction_total_force_and_dof_numbering():
    # the consistent loads on a face sum to traction x solid face area
    mask = np.ones((2, 3, 3), np.uint8)
    mask[1, 1, 1] = 0                          # a hole in the top layer
    bcs = _bcs(z0={"fix": (True,) * 3, "value": (0, 0, 0), "traction": (0, 0, 0)},
               z1={"fix": (False,) * 3, "value": (0, 0, 0), "traction": (0.5, -1.0, 2.0)})
    sysm = fem.System(mask, np.ones(mask.shape), 0.25, bcs)
    total = sysm.b.reshape(-1, 3).sum(axis=0) if sysm.n_dof % 3 == 0 else None
    assert total is not None
    assert np.allclose(total, np.array([0.5, -1.0, 2.0]) * 8)
    # all z0 nodes are fixed: every free DOF belongs to a node with k >= 1, node-major order
    nodes = sysm.free // 3
    assert (sysm.mesh.node_ijk[nodes, 2] >= 1).all()
    assert (np.diff(sysm.free) > 0).all()
