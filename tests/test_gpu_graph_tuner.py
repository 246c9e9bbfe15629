"""GPU: the preconditioner apply replayed from a captured CUDA graph, and the
set-up tuner of the smoother solve pipeline, against the plain launches and
the FP64 CPU oracle.

Bars: the graph replay computes the same operator as the launched apply
(relative 1e-12: only the order of floating-point atomic additions differs),
FP64 solutions within 1e-8 of the oracle's with the same iteration count, and
the tuned pipeline depths change timing only.
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


@pytest.mark.parametrize("name", ["tiny8_n2", "porous32_n4"])
def test_graph_apply_matches_launched_apply(name):
    import paper_2509_19777_gb300 as hp
    p, opt, sysm, M = oracle_case(name)
    s0 = gpu_solver(name)
    s1 = gpu_solver(name, use_graph=True)
    rng = np.random.default_rng(7)
    for rep in range(3):  # first call captures, later calls replay
        r = _t(rng.standard_normal(sysm.n_dof))
        l0 = hp.hplmm_kernel_launches()
        z1 = _n(s1.apply(r))
        torch.cuda.synchronize()
        assert hp.hplmm_kernel_launches() > l0  # the replay's kernels are counted
        z0 = _n(s0.apply(r))
        assert rel(z1, z0) < 1e-12
        assert rel(z1, M.apply(_n(r))) < 1e-10
    s0.close()
    s1.close()


@pytest.mark.parametrize("name", ["cube16_n4", "porous32_n4"])
def test_graph_solve_fp64_and_fp32(name):
    p, opt, sysm, M = oracle_case(name)
    x_ref, st_ref = oracle_solution(name)
    s = gpu_solver(name, use_graph=True)
    x, rc, st = s.solve(tol=1e-11)
    assert rc == 0
    assert rel(_n(x), x_ref) < 1e-8
    assert abs(st.iters - st_ref["iters"]) <= 2
    s.close()
    s = gpu_solver(name, use_graph=True, local_prec="fp32", apply_prec="fp32")
    x, rc, st = s.solve(tol=1e-8)
    xn = _n(x)
    assert rc == 0
    assert np.linalg.norm(sysm.b - sysm.A @ xn) / np.linalg.norm(sysm.b) <= 1e-8
    assert rel(xn, x_ref) < 1e-6
    s.close()


def test_graph_rebuilt_after_setup():
    # a second set-up invalidates the captured graph; the next apply captures it again
    import paper_2509_19777_gb300 as hp
    name = "tiny10_n1"
    p, opt, sysm, M = oracle_case(name)
    s = gpu_solver(name, use_graph=True)
    r = _t(np.random.default_rng(3).standard_normal(sysm.n_dof))
    z_a = _n(s.apply(r))
    s.setup(grains=p.grains)
    z_b = _n(s.apply(r))
    assert rel(z_b, z_a) < 1e-12
    assert rel(z_b, M.apply(_n(r))) < 1e-10
    s.close()


@pytest.mark.parametrize("name", ["porous32_n4"])
def test_autotune_keeps_results(name):
    p, opt, sysm, M = oracle_case(name)
    x_ref, st_ref = oracle_solution(name)
    s = gpu_solver(name, autotune=True)
    r = np.random.default_rng(5).standard_normal(sysm.n_dof)
    assert rel(_n(s.apply(_t(r))), M.apply(r)) < 1e-10
    x, rc, st = s.solve(tol=1e-11)
    assert rc == 0 and rel(_n(x), x_ref) < 1e-8
    s.close()
    s = gpu_solver(name, autotune=True, use_graph=True, local_prec="fp32", apply_prec="fp32")
    x, rc, st = s.solve(tol=1e-8)
    assert rc == 0 and rel(_n(x), x_ref) < 1e-6
    s.close()
