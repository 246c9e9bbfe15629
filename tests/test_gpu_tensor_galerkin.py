"""The Galerkin product A^o = P_hat^T A_hat P_hat (paper Section 4.2, Eq. mg_struct) of the FP32 forms on the
tensor cores (tcgen05.mma kind::tf32 with three TF32 products per pair of FP32 operands, accumulator in
tensor memory) against the same product on the FP32 CUDA cores and against the FP64 form and the oracle.

Both FP32 products sum the same FP32 terms P[r][a] Y[r][b] over the grain box's rows (M ~ 10^4 of them)
in different orders; the tensor-core one also drops the lo*lo term and truncates lo to TF32 (about 2^-22 of
each product).  The two differ by FP32 rounding of those sums, about sqrt(M) 2^-24 sum_r |P||Y|; with the
cancellation in A^o's entries (sum |P||Y| up to ~10^2 times the largest |A^o|) that is up to ~1e-5 of the
largest entry (measured: 6e-7 to 1e-5).  Both carry the FP32 basis error against the FP64 coarse matrix
(4e-6 to 4e-4 here), which the tensor path must not enlarge.
"""
import numpy as np
import pytest

from tests._cases import gpu_solver, oracle_case

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP32 = dict(local_prec="fp32", apply_prec="fp32")


@pytest.mark.parametrize("name", ["tiny8_n2", "porous32_n4", "fractured32_n2", "porous24_g216"])
def test_tensor_galerkin_matches_cuda_cores_and_fp64(name):
    p, opt, sysm, M = oracle_case(name)
    A_or = M.coarse.A_o
    scale = np.abs(A_or).max()
    out = {}
    for key, over in (("fp64", {}), ("tc", dict(FP32, tensor_galerkin=True)), ("cc", dict(FP32, tensor_galerkin=False))):
        s = gpu_solver(name, **over)
        out[key] = s.coarse_matrix().cpu().numpy()
        s.close()
    assert np.abs(out["fp64"] - A_or).max() <= 1e-10 * scale
    d_tc_cc = np.abs(out["tc"] - out["cc"]).max() / scale
    e_tc = np.abs(out["tc"] - out["fp64"]).max() / scale
    e_cc = np.abs(out["cc"] - out["fp64"]).max() / scale
    print(f"{name}: |tc - cc| {d_tc_cc:.2e}, |tc - fp64| {e_tc:.2e}, |cc - fp64| {e_cc:.2e} (of max |A^o|)")
    assert d_tc_cc <= 5e-5
    assert e_tc <= 1.1 * e_cc + 5e-5
    # symmetric to FP32 rounding (both triangles are summed separately)
    assert np.abs(out["tc"] - out["tc"].T).max() <= 5e-5 * scale


def test_tensor_galerkin_solve_matches_oracle():
    # the FP32 form with the tensor-core product reaches the oracle's solution at the FP64 residual
    name = "porous32_n4"
    p, opt, sysm, M = oracle_case(name)
    s = gpu_solver(name, tensor_galerkin=True, **FP32)
    x, rc, st = s.solve(tol=1e-10)
    assert rc == 0
    xn = x.cpu().numpy()
    assert np.linalg.norm(sysm.b - sysm.A @ xn) / np.linalg.norm(sysm.b) <= 1e-10 * 1.001
    s.close()
