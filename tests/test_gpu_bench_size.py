"""Parity at benchmark sizes: configuration 2 (porous64, 672,339 DOF, 64 grains, n = 4) and the reduced
fractured recipe (fractured64: the 256^3 recipe at 64^3 with its 16^3-voxel grains, slits and two-phase
Voronoi moduli, n = 2) -- the CUDA path's M^{-1} r element-wise against the oracle's (FP64 form, 1e-10), the
FP32 and BF16 forms within their bounds, and every form's solve at the FP64 true residual.  The oracle
builds its preconditioner in about three minutes per image on one core (marked slow).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

from tests._cases import maxrel, rel  # noqa: E402


def _solver(hp, p, n, **form):
    s = hp.Solver(n_mortar=n, contact_halfwidth=2, **form)
    mask, E = hp.problem_to_device(p)
    s.assemble(mask, E, p.nu, p.bcs)
    s.setup(grains=p.grains)
    return s


@pytest.mark.parametrize("name,seed,n", [("porous64", 0, 4), ("fractured64", 0, 2)])
def test_bench_size_apply_and_solve(name, seed, n):
    import paper_2509_19777_gb300 as hp
    import synth
    from oracle import precond
    p = synth.make_workload(name, seed)
    sysm, M = precond.build(p, precond.Options(n_mortar=n, contact_halfwidth=2))
    r = np.random.default_rng(5).standard_normal(sysm.n_dof)
    ref = M.apply(r)
    rt = torch.from_numpy(r).cuda()
    errs = {}
    for key, form in (("fp64", {}), ("fp32", dict(local_prec="fp32", apply_prec="fp32")),
                      ("bf16", dict(local_prec="fp32", apply_prec="bf16", use_graph=True, autotune=True))):
        s = _solver(hp, p, n, **form)
        assert s.n_dof == sysm.n_dof
        z = s.apply(rt).cpu().numpy()
        errs[key] = (rel(z, ref), maxrel(z, ref))
        x, rc, st = s.solve(tol=1e-8)
        assert rc == 0
        xn = x.cpu().numpy()
        assert np.linalg.norm(sysm.b - sysm.A @ xn) / np.linalg.norm(sysm.b) <= 1e-8
        s.close()
    print(f"{name}: apply error against the oracle FP64 {errs['fp64'][0]:.2e} (max {errs['fp64'][1]:.2e}), "
          f"FP32 form {errs['fp32'][0]:.2e}, BF16 form {errs['bf16'][0]:.2e}")
    assert errs["fp64"][0] < 1e-10 and errs["fp64"][1] < 1e-9
    assert errs["fp32"][0] < 1e-3
    # the BF16 form stores factors and panels with unit roundoff 2^-8 where the FP32 form has 2^-24: to first
    # order its error is at most 2^16 times the FP32 form's, and at least that error
    assert errs["fp32"][0] * 0.5 <= errs["bf16"][0] <= 2.0 ** 16 * errs["fp32"][0]
