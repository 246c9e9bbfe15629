"""The residual updates r - A_hat z of the FP32 and BF16 applies computed element by element from the voxel
moduli (options.matrix_free_updates, the default) against the same updates from the assembled FP32 copy of
A_hat (paper Section 2: A_hat is the sum over solid voxels of E_e times the reference element stiffness).

Both are FP32 products of the same operator: the assembled copy rounds each summed entry of A_hat to FP32,
the element-by-element one rounds E_e K_ref and sums in FP32, so a product differs by FP32 rounding (a few
2^-24 of |A_hat||z| per row); the residual update subtracts nearly equal vectors, so the applies differ by
about the FP32 form's own rounding error, which is what each carries against the FP64 oracle.
"""
import numpy as np
import pytest

from tests._cases import gpu_solver, maxrel, oracle_case, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,form", [("porous32_n4", dict(local_prec="fp32", apply_prec="fp32")),
                                       ("fractured32_n2", dict(local_prec="fp32", apply_prec="fp32")),
                                       ("porous32_n4", dict(local_prec="fp32", apply_prec="bf16"))])
def test_matrix_free_updates_match_assembled(name, form):
    p, opt, sysm, M = oracle_case(name)
    r = torch.from_numpy(np.random.default_rng(23).standard_normal(sysm.n_dof)).cuda()
    out = {}
    for key, mf in (("mf", True), ("as", False)):
        s = gpu_solver(name, matrix_free_updates=mf, **form)
        out[key] = s.apply(r).cpu().numpy()
        x, rc, st = s.solve(tol=1e-8)
        assert rc == 0
        xn = x.cpu().numpy()
        assert np.linalg.norm(sysm.b - sysm.A @ xn) / np.linalg.norm(sysm.b) <= 1e-8
        out[key + "_its"] = st.iters
        s.close()
    ref = M.apply(r.cpu().numpy())
    d = rel(out["mf"], out["as"])
    e_mf, e_as = rel(out["mf"], ref), rel(out["as"], ref)
    print(f"{name} {form['apply_prec']}: |mf - as| {d:.2e}, errors against the oracle {e_mf:.2e} / {e_as:.2e}, "
          f"iterations {out['mf_its']} / {out['as_its']}")
    # two FP32 computations of the same apply: they differ by at most the sum of their errors against the
    # oracle, and the element-by-element one is no less accurate
    assert d <= e_mf + e_as
    assert e_mf <= 1.5 * e_as + 1e-6
    assert abs(out["mf_its"] - out["as_its"]) <= 2
