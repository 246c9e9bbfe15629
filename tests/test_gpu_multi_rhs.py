"""Several loads on one set-up (paper Section 1 and Section 6.3: the set-up is paid once and reused for
further load cases; Section 7.4).

Four load cases on the same image and Dirichlet conditions (uniform tractions on the top face in z, x, y
and a combination) are solved with the preconditioner set up once for the first one.  The oracle builds
its preconditioner the same way (correction columns from the first load) and solves each load with its
GMRES; the GPU solves all four in lockstep (hplmm_solve_multi).  The multi-vector apply is also compared
vector by vector with the one-vector apply and with the oracle's M^{-1}.
"""
import numpy as np
import pytest

import synth
from oracle import fem, gmres, precond
from tests._cases import gpu_solver, maxrel, oracle_case, problem, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TRACTIONS = [(0.0, 0.0, 1.0), (1.0, 0.0, 0.0), (0.0, 0.7, 0.0), (0.3, -0.4, 0.5)]


def _loads(p):
    bs = []
    for t in TRACTIONS:
        sysm = fem.System(p.mask, p.E, p.nu, synth.bcs_clamped_traction(traction=t))
        bs.append(sysm.b)
    return np.stack(bs)


@pytest.mark.parametrize("name", ["porous32_n4", "fractured32_n2"])
def test_four_loads_one_setup_match_oracle(name):
    p, opt, sysm, M = oracle_case(name)
    B = _loads(p)
    s = gpu_solver(name)            # FP64 form, set up with the first load's b_hat
    X, rc, st = s.solve_multi(torch.from_numpy(B).cuda(), tol=1e-10)
    assert rc == 0
    Xn = X.cpu().numpy()
    for q in range(len(TRACTIONS)):
        x_ref, st_ref = gmres.gmres(sysm.A, B[q], M.apply, tol=1e-10)
        assert np.linalg.norm(B[q] - sysm.A @ Xn[q]) / np.linalg.norm(B[q]) <= 1e-10 * 1.001
        assert rel(Xn[q], x_ref) < 1e-8 and maxrel(Xn[q], x_ref) < 1e-7, q
        assert abs(st[q].iters - st_ref["iters"]) <= 2, (q, st[q].iters, st_ref["iters"])
    s.close()


@pytest.mark.parametrize("form,tol", [(dict(local_prec="fp64", apply_prec="fp64"), 1e-12),
                                      (dict(local_prec="fp32", apply_prec="fp32"), None),
                                      (dict(local_prec="fp32", apply_prec="bf16"), None)])
def test_multi_apply_matches_single_apply(form, tol):
    # the multi-vector apply uses the multi-right-hand-side banded solves for the smoother (the one-vector
    # apply the pipelined solve), so in FP32 the two differ by FP32 rounding only
    name = "porous32_n4"
    p, opt, sysm, M = oracle_case(name)
    s = gpu_solver(name, **form)
    Rn = np.random.default_rng(31).standard_normal((5, sysm.n_dof))
    Z = s.apply_multi(torch.from_numpy(Rn).cuda()).cpu().numpy()
    for q in range(Rn.shape[0]):
        z1 = s.apply(torch.from_numpy(Rn[q]).cuda()).cpu().numpy()
        ref = M.apply(Rn[q])
        e1, em = rel(z1, ref), rel(Z[q], ref)
        if form["apply_prec"] == "fp64":
            assert rel(Z[q], z1) < tol and em < 1e-10, (q, rel(Z[q], z1), em)
        else:
            # two different FP32 computations of the same operator (the multi-vector smoother uses other
            # kernels): each carries the form's error against the FP64 oracle, so they differ by at most the
            # sum of those errors, and neither is more than a few times the other
            assert rel(Z[q], z1) <= e1 + em and em <= 4 * e1, (q, rel(Z[q], z1), e1, em)
    s.close()


def test_multi_solve_fp32_form_reaches_fp64_residual():
    name = "porous32_n4"
    p, opt, sysm, M = oracle_case(name)
    B = _loads(p)
    s = gpu_solver(name, local_prec="fp32", apply_prec="fp32")
    X, rc, st = s.solve_multi(torch.from_numpy(B).cuda(), tol=1e-8)
    assert rc == 0
    Xn = X.cpu().numpy()
    for q in range(len(TRACTIONS)):
        assert np.linalg.norm(B[q] - sysm.A @ Xn[q]) / np.linalg.norm(B[q]) <= 1e-8
    # the same solves one at a time take the same iteration counts (same preconditioner up to rounding)
    for q in range(len(TRACTIONS)):
        x1, rc1, st1 = s.solve(torch.from_numpy(B[q]).cuda(), None, 1e-8)
        assert rc1 == 0 and abs(st1.iters - st[q].iters) <= 2
    s.close()


def test_multi_arguments_validated():
    import paper_2509_19777_gb300 as hp
    s = gpu_solver("tiny8_n2")
    B = torch.zeros((65, s.n_dof), dtype=torch.float64, device="cuda")
    with pytest.raises(hp.HplmmError) as ei:
        s.solve_multi(B)
    assert ei.value.code == hp.HPLMM_ERR_INVALID
    s.close()
