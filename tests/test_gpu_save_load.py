"""Saving a set-up and loading it into a fresh context (the set-up is built once and reused: paper Sections 1,
6.3 and 7.4).  The loaded context applies the same preconditioner -- to rounding order of the atomics inside
one apply, which the saved context shows between two of its own applies -- and solves in the same
iterations; mismatched systems or options and bad files are refused with HPLMM_ERR_INVALID.
"""
import numpy as np
import pytest

from tests._cases import gpu_solver, oracle_case, problem, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FORMS = [("porous32_n4", {}), ("porous32_n4", dict(local_prec="fp32", apply_prec="fp32", use_graph=True)),
         ("porous32_n4", dict(local_prec="fp32", apply_prec="bf16", autotune=True)),
         ("tiny8_alg", {}), ("porous32_g512", {})]


def _fresh(name, **over):
    import paper_2509_19777_gb300 as hp
    p, opt = problem(name)
    kw = dict(n_mortar=opt["n_mortar"], contact_halfwidth=opt["contact_halfwidth"],
              strict_two_grain=opt.get("strict_two_grain", False), mortar_kind=opt.get("mortar_kind", "gaussian"))
    kw.update(over)
    s = hp.Solver(**kw)
    mask, E = hp.problem_to_device(p)
    s.assemble(mask, E, p.nu, p.bcs)
    return s


@pytest.mark.parametrize("name,form", FORMS)
def test_loaded_setup_applies_and_solves_the_same(tmp_path, name, form):
    p, opt, sysm, M = oracle_case(name)
    r = torch.from_numpy(np.random.default_rng(7).standard_normal(sysm.n_dof)).cuda()
    s1 = gpu_solver(name, **form)
    z1 = s1.apply(r).clone()
    z1b = s1.apply(r).clone()
    x1, rc1, st1 = s1.solve(tol=1e-8)
    path = str(tmp_path / "setup.bin")
    s1.save_setup(path)
    sizes1 = s1.sizes()
    s1.close()
    s2 = _fresh(name, **form)
    s2.load_setup(path)
    assert s2.sizes() == sizes1
    z2 = s2.apply(r).cpu().numpy()
    z1n, rep = z1.cpu().numpy(), rel(z1b.cpu().numpy(), z1.cpu().numpy())
    fp64 = form.get("apply_prec", "fp64") == "fp64"
    assert rel(z2, z1n) <= max(10 * rep, 1e-12 if fp64 else 1e-6), (rel(z2, z1n), rep)
    x2, rc2, st2 = s2.solve(tol=1e-8)
    assert rc2 == 0 and abs(st2.iters - st1.iters) <= 1
    xn = x2.cpu().numpy()
    assert np.linalg.norm(sysm.b - sysm.A @ xn) / np.linalg.norm(sysm.b) <= 1e-8
    s2.close()


def test_load_refuses_mismatches(tmp_path):
    import paper_2509_19777_gb300 as hp
    name = "tiny8_n2"
    s1 = gpu_solver(name)
    path = str(tmp_path / "setup.bin")
    s1.save_setup(path)
    s1.close()
    # other set-up options
    s2 = _fresh(name, n_mortar=3)
    with pytest.raises(hp.HplmmError) as ei:
        s2.load_setup(path)
    assert ei.value.code == hp.HPLMM_ERR_INVALID
    s2.close()
    # not assembled
    s3 = hp.Solver(n_mortar=2, contact_halfwidth=1)
    with pytest.raises(hp.HplmmError) as ei:
        s3.load_setup(path)
    assert ei.value.code == hp.HPLMM_ERR_STATE
    s3.close()
    # not a saved set-up, and a truncated one
    bad = tmp_path / "bad.bin"
    bad.write_bytes(b"not a set-up" * 10)
    cut = tmp_path / "cut.bin"
    cut.write_bytes(open(path, "rb").read()[:5000])
    for f in (bad, cut):
        s4 = _fresh(name)
        with pytest.raises(hp.HplmmError) as ei:
            s4.load_setup(str(f))
        assert ei.value.code == hp.HPLMM_ERR_INVALID
        s4.close()
    # nothing to save before a set-up
    s5 = _fresh(name)
    with pytest.raises(hp.HplmmError) as ei:
        s5.save_setup(str(tmp_path / "none.bin"))
    assert ei.value.code == hp.HPLMM_ERR_STATE
    s5.close()
