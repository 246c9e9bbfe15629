"""Algebraic mortars (paper Section 3.3, Eq. algebra and the Remark after Eq. reduced_defs; Appendix B): the
CUDA path against the oracle, element-wise, on the objects they change -- the columns of P_hat (their
interface rows are the mortar functions), A^o, M^{-1} r and the solution -- and the comparison with Gaussian
mortars that Appendix B makes: first-pass accuracy and GMRES iterations as n grows.
"""
import numpy as np
import pytest

from tests._cases import gpu_solver, maxrel, oracle_case, oracle_solution, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _n(t):
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("name", ["tiny8_alg", "porous32_alg"])
def test_algebraic_mortars_match_oracle(name):
    p, opt, sysm, M = oracle_case(name)
    s = gpu_solver(name)
    assert s.sizes()["n_coarse"] == M.coarse.n_coarse
    P = M.coarse.P_hat.tocsc()
    n = P.shape[1]
    for col in sorted({0, 1, n // 3, n // 2, n - 2, n - 1}):
        ref = P[:, col].toarray().ravel()
        assert maxrel(_n(s.prolongation_column(col)), ref) < 1e-10, col
    A = _n(s.coarse_matrix())
    assert np.abs(A - M.coarse.A_o).max() < 1e-10 * np.abs(M.coarse.A_o).max()
    r = np.random.default_rng(41).standard_normal(sysm.n_dof)
    z = _n(s.apply(torch.from_numpy(r).cuda()))
    assert rel(z, M.apply(r)) < 1e-10
    x_ref, st_ref = oracle_solution(name)
    x, rc, st = s.solve(tol=1e-11)
    assert rc == 0 and rel(_n(x), x_ref) < 1e-8 and abs(st.iters - st_ref["iters"]) <= 2
    s.close()


def test_gaussian_and_algebraic_mortars_as_n_grows():
    # Appendix B: both kinds give first-pass solutions of similar accuracy; with one mortar per interface
    # they are the same (PLMM).  Reported: the first-pass error and the GMRES iterations per n and kind.
    import scipy.sparse.linalg as spla
    import synth
    from oracle import fem
    p = synth.make_workload("porous32", 1)
    sysm = fem.System(p.mask, p.E, p.nu, p.bcs)
    xs = spla.spsolve(sysm.A.tocsc(), sysm.b)
    out = {}
    for kind in ("gaussian", "algebraic"):
        for n in (1, 2, 4):
            s = gpu_solver("porous32_n4", n_mortar=n, mortar_kind=kind)
            xa = _n(s.apply_coarse(s.b))
            x, rc, st = s.solve(tol=1e-8)
            assert rc == 0
            out[(kind, n)] = (rel(xa, xs), st.iters)
            s.close()
    for n in (1, 2, 4):
        print(f"n={n}: first-pass error Gaussian {out[('gaussian', n)][0]:.3f} ({out[('gaussian', n)][1]} its), "
              f"algebraic {out[('algebraic', n)][0]:.3f} ({out[('algebraic', n)][1]} its)")
    # one mortar: the same translation, up to the algebraic operator's diagonal shift (1e-8 of A_hat's)
    assert abs(out[("gaussian", 1)][0] - out[("algebraic", 1)][0]) < 1e-5
    for kind in ("gaussian", "algebraic"):
        assert out[(kind, 4)][0] < out[(kind, 1)][0]
