"""GPU: the two forms of the smoother solve (one CTA per local problem, or a two-CTA
cluster that splits each panel's far rows) and the Krylov kernels over the whole range of
basis sizes, through the C interface, against each other and the FP64 CPU oracle.

Bars: M_CG^{-1} r of the two forms agrees to the rounding of the form's precision (FP64:
1e-12 relative, only the order of additions differs; FP32: 1e-5; BF16 storage: 1e-3) and
matches the oracle's (FP64 form: 1e-10; FP32: 5e-3, the FP32 unit roundoff 6e-8 amplified by
local condition numbers of a few 1e4 on the heterogeneous porous grains, measured 1.3e-3;
BF16: the bound derived in test_bf16_error_follows_roundoff); FGMRES with restart lengths that
take the basis past 32 vectors (the largest register block and the generic update) reaches
the FP64 true residual and the oracle's solution.
"""
import numpy as np
import pytest

from tests._cases import gpu_solver, oracle_case, oracle_solution, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _t(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def _n(t):
    return t.detach().cpu().numpy()


FORMS = [
    (dict(local_prec="fp64", apply_prec="fp64"), 1e-12, 1e-10),
    (dict(local_prec="fp32", apply_prec="fp32"), 1e-5, 5e-3),
    (dict(local_prec="fp32", apply_prec="bf16"), 1e-3, None),
]
U32, U16 = 2.0 ** -24, 2.0 ** -8   # unit roundoffs of FP32 and BF16 (24- and 8-bit significands)


@pytest.mark.parametrize("name", ["cube16_n4", "porous32_n4", "tiny10_strict"])
@pytest.mark.parametrize("form,tol_forms,tol_oracle", FORMS)
def test_one_and_two_cta_smoothers_agree(name, form, tol_forms, tol_oracle):
    p, opt, sysm, M = oracle_case(name)
    rng = np.random.default_rng(17)
    r = rng.standard_normal(sysm.n_dof)
    z_ref = M.smoother.apply(r)
    out = {}
    for ctas in (1, 2):
        s = gpu_solver(name, smoother_ctas=ctas, **form)
        out[ctas] = _n(s.apply_smoother(_t(r)))
        s.close()
    assert rel(out[2], out[1]) < tol_forms
    for ctas in (1, 2):
        if tol_oracle is not None:
            assert rel(out[ctas], z_ref) < tol_oracle, ctas


@pytest.mark.parametrize("name", ["cube16_n4", "porous32_n4", "fractured32_n2"])
@pytest.mark.parametrize("form,tol_forms,tol_oracle", FORMS)
def test_bulk_warp_forms_agree(name, form, tol_forms, tol_oracle):
    # the one-CTA smoother with 8, 4, 2 or 1 warps streaming the far rows (ring sized for one, two, three or
    # four CTAs per SM): the same operator, summed in another order
    p, opt, sysm, M = oracle_case(name)
    r = np.random.default_rng(23).standard_normal(sysm.n_dof)
    z_ref = M.smoother.apply(r)
    out = {}
    for nbw in (8, 4, 2, 1):
        s = gpu_solver(name, smoother_ctas=1, smoother_bulk_warps=nbw, **form)
        out[nbw] = _n(s.apply_smoother(_t(r)))
        s.close()
    for nbw in (4, 2, 1):
        assert rel(out[nbw], out[8]) < tol_forms, nbw
    if tol_oracle is not None:
        for nbw in out:
            assert rel(out[nbw], z_ref) < tol_oracle, nbw


@pytest.mark.parametrize("nbw", [4, 1])
def test_bulk_warp_solve_matches_oracle(nbw):
    # the headline's smoother forms (4 bulk warps for the grains, 1 for the contact grids) inside FGMRES with
    # the graph replay
    name = "porous32_n4"
    x_ref, _ = oracle_solution(name)
    p, opt, sysm, M = oracle_case(name)
    s = gpu_solver(name, smoother_bulk_warps=nbw, local_prec="fp32", apply_prec="bf16", use_graph=True)
    x, rc, st = s.solve(tol=1e-10)
    xn = _n(x)
    assert rc == 0
    assert np.linalg.norm(sysm.b - sysm.A @ xn) / np.linalg.norm(sysm.b) <= 1e-10 * 1.001
    assert rel(xn, x_ref) < 1e-6
    s.close()


@pytest.mark.parametrize("name", ["cube16_n4", "porous32_n4", "fractured32_n2"])
def test_bf16_error_follows_roundoff(name):
    # The BF16 form computes exactly like the FP32 form (FP32 factorisation, FP32 arithmetic) and then stores
    # the factors rounded to BF16, each element with relative error at most U16.  To first order an error in
    # the stored factors reaches M_CG^{-1} r linearly, amplified by the local problems' conditioning; the
    # FP32 form's own error against the FP64 oracle, e32, carries the same amplification of its FP32 roundoff
    # (factorisation and solves, at least U32 per element).  Hence e16 <= e32 + (U16 / U32) e32, and the
    # BF16 rounding is visible: e16 > e32.
    p, opt, sysm, M = oracle_case(name)
    r = np.random.default_rng(19).standard_normal(sysm.n_dof)
    z_ref = M.smoother.apply(r)
    e = {}
    for ap in ("fp32", "bf16"):
        s = gpu_solver(name, local_prec="fp32", apply_prec=ap)
        e[ap] = rel(_n(s.apply_smoother(_t(r))), z_ref)
        s.close()
    print(f"{name}: M_CG^-1 r error vs FP64 oracle: FP32 {e['fp32']:.2e}, BF16 {e['bf16']:.2e}")
    assert e["fp32"] < e["bf16"] <= (1.0 + U16 / U32) * e["fp32"]


@pytest.mark.parametrize("ctas", [1, 2])
def test_two_cta_solve_matches_oracle(ctas):
    name = "porous32_n4"
    x_ref, _ = oracle_solution(name)
    p, opt, sysm, M = oracle_case(name)
    s = gpu_solver(name, smoother_ctas=ctas, local_prec="fp32", apply_prec="fp32", use_graph=True)
    x, rc, st = s.solve(tol=1e-8)
    xn = _n(x)
    assert rc == 0
    assert np.linalg.norm(sysm.b - sysm.A @ xn) / np.linalg.norm(sysm.b) <= 1e-8
    assert rel(xn, x_ref) < 1e-6
    s.close()


@pytest.mark.parametrize("restart", [3, 12, 45])
def test_krylov_basis_sizes(restart):
    # restart 45 builds bases of up to 46 vectors: every register block of the CGS2 kernels (1 .. 32) and,
    # past 32, the generic update followed by the 64-wide dot product
    name = "cube16_n4"
    x_ref, _ = oracle_solution(name)
    p, opt, sysm, M = oracle_case(name)
    s = gpu_solver(name, restart=restart)
    x, rc, st = s.solve(tol=1e-11)
    xn = _n(x)
    assert rc == 0
    assert np.linalg.norm(sysm.b - sysm.A @ xn) / np.linalg.norm(sysm.b) <= 1e-11
    assert rel(xn, x_ref) < 1e-8
    s.close()


def test_smoother_ctas_validated():
    import paper_2509_19777_gb300 as hp
    with pytest.raises(hp.HplmmError):
        hp.Solver(smoother_ctas=3)
    with pytest.raises(hp.HplmmError):
        hp.Solver(smoother_bulk_warps=4, smoother_ctas=2)
