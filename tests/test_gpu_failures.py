"""Failure paths, each made on the host or by a bounded device wait, never by a GPU fault:

* a solid part with no prescribed displacement (a floating island) -> HPLMM_ERR_SINGULAR at assembly, with
  a node of the island in the message;
* a modulus that is NaN, zero or negative -> HPLMM_ERR_INVALID at assembly, with the voxel;
* a zero right-hand side -> x = 0 and HPLMM_OK; a non-finite one -> HPLMM_ERR_INVALID;
* an injected device-allocation failure -> HPLMM_ERR_OOM, and a new context works afterwards;
* a smoother wait budget so small that its pipeline waits run out -> HPLMM_ERR_TIMEOUT from the solve; the
  kernel lets its copies in flight land before its blocks exit, and a new context then solves normally.
"""
import numpy as np
import pytest

from tests._cases import gpu_solver, oracle_case, problem, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _hp():
    import paper_2509_19777_gb300 as hp
    return hp


def test_floating_island_is_singular():
    import synth
    hp = _hp()
    mask = np.ones((8, 8, 8), np.uint8)          # [z][y][x], clamped at z = 0
    mask[3:8, 0:5, 0:5] = 0                       # a void corner region from z = 3 up
    mask[5, 1:3, 1:3] = 1                         # an island inside it: nodes x, y in [1, 3], z in [5, 6]
    E = np.ones_like(mask, dtype=np.float32)
    s = hp.Solver(n_mortar=2, contact_halfwidth=1)
    with pytest.raises(hp.HplmmError) as ei:
        s.assemble(torch.from_numpy(mask).cuda(), torch.from_numpy(E).cuda(), 0.3, synth.bcs_clamped_traction())
    assert ei.value.code == hp.HPLMM_ERR_SINGULAR
    msg = str(ei.value)
    assert "no prescribed displacement" in msg
    ijk = [int(v) for v in msg.split("node (")[1].split(")")[0].split(",")]
    assert 1 <= ijk[0] <= 3 and 1 <= ijk[1] <= 3 and 5 <= ijk[2] <= 6, ijk
    # without the island the same block assembles
    mask[5, 1:3, 1:3] = 0
    n = s.assemble(torch.from_numpy(mask).cuda(), torch.from_numpy(E).cuda(), 0.3, synth.bcs_clamped_traction())
    assert n > 0
    s.close()


@pytest.mark.parametrize("bad", [float("nan"), 0.0, -1.0, float("inf")])
def test_bad_modulus_is_invalid(bad):
    hp = _hp()
    p, opt = problem("tiny8_n2")
    E = p.E.copy()
    k, j, i = np.argwhere(p.mask > 0)[7]
    E[k, j, i] = bad
    s = hp.Solver(n_mortar=2, contact_halfwidth=1)
    with pytest.raises(hp.HplmmError) as ei:
        s.assemble(torch.from_numpy(np.ascontiguousarray(p.mask)).cuda(),
                   torch.from_numpy(np.ascontiguousarray(E)).cuda(), p.nu, p.bcs)
    assert ei.value.code == hp.HPLMM_ERR_INVALID
    assert f"({i}, {j}, {k})" in str(ei.value)
    s.close()


def test_zero_and_nonfinite_right_hand_sides():
    hp = _hp()
    s = gpu_solver("tiny8_n2")
    b = torch.zeros(s.n_dof, dtype=torch.float64, device="cuda")
    x, rc, st = s.solve(b, None, 1e-8)
    assert rc == hp.HPLMM_OK and st.iters == 0
    assert torch.count_nonzero(x).item() == 0
    b[3] = float("nan")
    with pytest.raises(hp.HplmmError) as ei:
        s.solve(b, None, 1e-8)
    assert ei.value.code == hp.HPLMM_ERR_INVALID
    s.close()


def test_injected_allocation_failure_then_recovery():
    hp = _hp()
    p, opt = problem("tiny8_n2")
    s = hp.Solver(n_mortar=2, contact_halfwidth=1)
    mask, E = hp.problem_to_device(p)
    s.assemble(mask, E, p.nu, p.bcs)
    hp.hplmm_inject_alloc_failure(3)
    with pytest.raises(hp.HplmmError) as ei:
        s.setup(grains=p.grains)
    assert ei.value.code == hp.HPLMM_ERR_OOM
    assert "injected" in str(ei.value)
    hp.hplmm_inject_alloc_failure(-1)
    s.close()
    # a new context on the same device works
    p2, opt2, sysm, M = oracle_case("tiny8_n2")
    s2 = gpu_solver("tiny8_n2")
    x, rc, st = s2.solve(tol=1e-10)
    assert rc == 0
    xn = x.cpu().numpy()
    assert np.linalg.norm(sysm.b - sysm.A @ xn) / np.linalg.norm(sysm.b) <= 1e-10
    s2.close()


def test_wait_budget_runs_out_then_recovery():
    hp = _hp()
    p, opt, sysm, M = oracle_case("porous32_n4")
    # a budget of 1 microsecond: the smoother's pipelined waits (copies, hand-offs between warps) give up.
    # One CTA per problem: a two-CTA cluster that gives up also waits (about 2 s per phase) for remote stores
    # that its peer may have in flight, which would make this test slow, not wrong
    s = gpu_solver("porous32_n4", local_prec="fp32", apply_prec="fp32", wait_budget_us=1, smoother_ctas=1,
                   max_iters=30)
    with pytest.raises(hp.HplmmError) as ei:
        s.solve(tol=1e-8)
    assert ei.value.code == hp.HPLMM_ERR_TIMEOUT
    s.close()
    torch.cuda.synchronize()  # the device is still usable: nothing faulted
    s2 = gpu_solver("porous32_n4", local_prec="fp32", apply_prec="fp32")
    x, rc, st = s2.solve(tol=1e-8)
    assert rc == 0
    xn = x.cpu().numpy()
    assert np.linalg.norm(sysm.b - sysm.A @ xn) / np.linalg.norm(sysm.b) <= 1e-8
    r = np.random.default_rng(3).standard_normal(sysm.n_dof)
    z = s2.apply_smoother(torch.from_numpy(r).cuda()).cpu().numpy()
    assert rel(z, M.smoother.apply(r)) < 5e-3
    s2.close()
