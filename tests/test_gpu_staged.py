"""The staged set-up of the BF16 apply form: local factors computed in FP32 in chunks (each chunk of grains
used for its basis solves), then kept only as BF16.  A chunk with few problems is factored by two-CTA
clusters where the whole set is factored one CTA per problem, which orders some FP32 sums differently; a
factor element that lands on the other side of a BF16 rounding boundary then differs by one BF16 unit.  The
Galerkin product on the tensor cores (three TF32 products per FP32 pair, error up to 2^-22 of each product,
moving with the last bits of its inputs) turns FP32-rounding differences of the basis into differences of
A^o of about 2^-22 times the cancellation in its entries (up to ~10^2).  So a set-up split into many small
chunks gives the same preconditioner as a one-chunk set-up up to relative 3e-5 (measured 9e-6), against
the BF16 form's own error of about 1e-2, and both match the FP64 oracle within the BF16 form's error."""
import numpy as np
import pytest

from tests._cases import gpu_solver, maxrel, oracle_case, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _t(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


@pytest.mark.parametrize("name", ["porous32_n4", "porous32_g512"])
def test_staged_chunks_bit_identical(name):
    p, opt, sysm, M = oracle_case(name)
    r = _t(np.random.default_rng(21).standard_normal(sysm.n_dof))
    out = []
    for mb in (0, 1):  # one chunk (default budget) and chunks of at most 1 MiB of FP32 factors
        s = gpu_solver(name, local_prec="fp32", apply_prec="bf16", stage_mb=mb)
        z = s.apply(r).clone()
        x, rc, st = s.solve(tol=1e-8)
        out.append((z, x.clone(), st.iters))
        s.close()
    zn = out[0][0].cpu().numpy()
    assert rel(out[1][0].cpu().numpy(), zn) < 3e-5
    assert abs(out[0][2] - out[1][2]) <= 1
    assert rel(out[1][1].cpu().numpy(), out[0][1].cpu().numpy()) < 1e-6
    ref = M.apply(r.cpu().numpy())
    assert np.isfinite(zn).all()
    assert rel(zn, ref) < 0.2 and maxrel(zn, ref) < 1.0
    xn = out[0][1].cpu().numpy()
    assert np.linalg.norm(sysm.b - sysm.A @ xn) / np.linalg.norm(sysm.b) <= 1e-8


def test_bf16_prolongation_columns_are_the_rounded_fp32_basis():
    # after the set-up the BF16 form keeps only its column-major BF16 panels: a column of P_hat read back
    # from them is the FP32 form's column rounded to BF16 (unit roundoff 2^-8), up to the FP32 differences of
    # the staged factorisation (relative 1e-5 of the column's largest entry)
    name = "porous32_n4"
    s16 = gpu_solver(name, local_prec="fp32", apply_prec="bf16")
    s32 = gpu_solver(name, local_prec="fp32", apply_prec="fp32")
    n = s32.sizes()["n_coarse"]
    for col in sorted({0, 1, n // 3, n // 2, n - 1}):
        a = s16.prolongation_column(col).cpu().numpy()
        b = s32.prolongation_column(col).cpu().numpy()
        assert np.all(np.abs(a - b) <= 2.0 ** -8 * np.abs(b) + 1e-5 * np.abs(b).max()), col
    s16.close()
    s32.close()
