"""The Schur updates of the coarse multifrontal Cholesky on the tensor cores, in FP64 by the Ozaki splitting
scheme (options.tensor_coarse, the default), against the same factorisation on the FP64 CUDA cores and the
oracle's (A^o)^{-1}.

Each panel row is cut to 56-bit fixed point (error below 2^-56 of the row's largest entry) and the digit
groups kept cover the product to 2^-53 of |L_i||L_j|: the factor has the rounding errors of an FP64
factorisation, so the coarse solve (A^o)^{-1} t of the two paths agrees to the FP64 backward error times
the condition number of A^o (measured: a few 1e-15 to 1e-13 here), and both meet the oracle's 1e-10.
"""
import numpy as np
import pytest

from tests._cases import gpu_solver, maxrel, oracle_case, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name", ["porous32_n4", "fractured32_n2", "porous24_g216", "porous32_g512"])
def test_tensor_coarse_factor_matches_fp64_cores_and_oracle(name):
    p, opt, sysm, M = oracle_case(name)
    r = np.random.default_rng(17).standard_normal(sysm.n_dof)
    rt = torch.from_numpy(r).cuda()
    out = {}
    for key, tc in (("tc", True), ("cc", False)):
        s = gpu_solver(name, tensor_coarse=tc)
        out[key] = s.apply_coarse(rt).cpu().numpy()
        s.close()
    ref = M.M_G(r)
    d = rel(out["tc"], out["cc"])
    print(f"{name}: |tc - cc| {d:.2e}, |tc - oracle| {rel(out['tc'], ref):.2e}")
    assert d < 1e-11
    assert rel(out["tc"], ref) < 1e-10 and maxrel(out["tc"], ref) < 1e-9


def test_tensor_coarse_solve_bf16_form():
    # the BF16 form's solve with the tensor-core coarse factor reaches the FP64 residual
    name = "porous32_n4"
    p, opt, sysm, M = oracle_case(name)
    s = gpu_solver(name, local_prec="fp32", apply_prec="bf16", tensor_coarse=True)
    x, rc, st = s.solve(tol=1e-8)
    assert rc == 0
    xn = x.cpu().numpy()
    assert np.linalg.norm(sysm.b - sysm.A @ xn) / np.linalg.norm(sysm.b) <= 1e-8
    s.close()
