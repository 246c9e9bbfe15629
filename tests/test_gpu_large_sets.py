"""GPU parity on the paths only large sets of local problems take.

* 216 grains (porous24, 6x6x6 grains of 4^3 voxels): more problems than half the SMs, so each grain and
  contact grid is factored by one CTA (no two-CTA clusters);
* 512 grains (porous32, 8x8x8): more problems than two per SM, so the persistent factorisation queue
  hands every CTA several problems; 1,300+ contact grids;
* both give a deep elimination tree of the sparse coarse factor (many fronts per level, merged leaves,
  extend-adds of several children into one parent).

Every comparison is made norm-wise and element-wise (max |error| over the largest |oracle value|), in
FP64 (rounding of two different factorisations: 1e-10) and in the FP32 form (FP32 local factors, basis
and smoother; FP32 rounding amplified by local condition numbers of a few 1e4: 1e-3).
"""
import numpy as np
import pytest

from tests._cases import gpu_solver, maxrel, oracle_case, oracle_solution, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LARGE = ["porous24_g216", "porous32_g512"]


def _t(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def _n(t):
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("name", LARGE)
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-3)])
def test_large_set_apply(name, prec, tol):
    p, opt, sysm, M = oracle_case(name)
    s = gpu_solver(name, local_prec=prec, apply_prec=prec)
    r = np.random.default_rng(11).standard_normal(sysm.n_dof)
    rt = _t(r)
    for got, ref, what in ((s.apply_coarse(rt), M.M_G(r), "M_G"), (s.apply_smoother(rt), M.smoother.apply(r), "M_CG"),
                           (s.apply(rt), M.apply(r), "M")):
        g = _n(got)
        assert np.isfinite(g).all(), what
        assert rel(g, ref) < tol, (what, rel(g, ref))
        assert maxrel(g, ref) < 10 * tol, (what, maxrel(g, ref))
    s.close()


@pytest.mark.parametrize("name", LARGE)
@pytest.mark.parametrize("ctas", [1, 2])
def test_large_set_smoother_forms(name, ctas):
    # the smoother solve with one CTA per problem and with two-CTA clusters, FP32 factors
    p, opt, sysm, M = oracle_case(name)
    s = gpu_solver(name, local_prec="fp32", apply_prec="fp32", smoother_ctas=ctas)
    r = np.random.default_rng(12).standard_normal(sysm.n_dof)
    g = _n(s.apply_smoother(_t(r)))
    ref = M.smoother.apply(r)
    assert rel(g, ref) < 1e-3 and maxrel(g, ref) < 1e-2, (rel(g, ref), maxrel(g, ref))
    s.close()


@pytest.mark.parametrize("name", LARGE)
def test_large_set_coarse_space(name):
    # A^o (dense copy) and columns of P_hat element-wise; the solution of the FP64 form
    p, opt, sysm, M = oracle_case(name)
    s = gpu_solver(name)
    A = _n(s.coarse_matrix())
    assert np.abs(A - M.coarse.A_o).max() < 1e-10 * np.abs(M.coarse.A_o).max()
    P = M.coarse.P_hat.tocsc()
    n = P.shape[1]
    for col in sorted({0, n // 7, n // 2, n - 1}):
        ref = P[:, col].toarray().ravel()
        got = _n(s.prolongation_column(col))
        assert maxrel(got, ref) < 1e-10, col
    # the solution: the FP64 form's true residual (recomputed with the oracle's A_hat) and the oracle GMRES
    # iteration count at 1e-8 (the same Krylov space: CGS2 FGMRES against MGS GMRES, +-2)
    x_ref, st_ref = oracle_solution(name, tol=1e-8)
    x, rc, st = s.solve(tol=1e-8)
    assert rc == 0
    xn = _n(x)
    assert np.linalg.norm(sysm.b - sysm.A @ xn) / np.linalg.norm(sysm.b) <= 1e-8 * 1.001
    assert abs(st.iters - st_ref["iters"]) <= 2
    assert rel(xn, x_ref) < 1e-5
    s.close()
