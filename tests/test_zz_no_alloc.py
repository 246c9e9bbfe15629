"""The allocation-free SpMV entry point (hplmm_spmv_noalloc), for callers that
cannot allocate device memory at call time, against the ordinary hplmm_spmv
on two calls in a row.  This file sorts last so that a run stopping at the
first failure has already run every other test."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_spmv_noalloc_matches_spmv_twice():
    import paper_2509_19777_gb300 as hp
    import synth
    lib = hp.load_library()
    p = synth.make_workload("tiny8", 3)
    s = hp.Solver(n_mortar=2, contact_halfwidth=1)
    mask, E = hp.problem_to_device(p)
    n = s.assemble(mask, E, p.nu, p.bcs)
    rng = np.random.default_rng(11)
    for call in range(2):
        x = torch.from_numpy(rng.standard_normal(n)).cuda()
        y_ref = torch.empty_like(x)
        y_na = torch.full_like(x, np.nan)
        assert lib.hplmm_spmv(s.ctx, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y_ref.data_ptr())) == 0
        rc = lib.hplmm_spmv_noalloc(s.ctx, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y_na.data_ptr()))
        assert rc == 0, hp.hplmm_last_error(s.ctx)
        torch.cuda.synchronize()
        a, b = y_na.cpu().numpy(), y_ref.cpu().numpy()
        assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-13, call
    s.close()


def test_spmv_noalloc_rejects_too_large_systems():
    import paper_2509_19777_gb300 as hp
    import synth
    mask = torch.ones((72, 72, 72), dtype=torch.uint8, device="cuda")   # 73^3 = 389,017 nodes > 262,144
    s = hp.Solver()
    n = s.assemble(mask, None, 0.3, synth.bcs_clamped_traction(), E0=1.0)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(hp.HplmmError) as ei:
        hp.hplmm_spmv_noalloc(s.ctx, x, torch.empty_like(x))
    assert ei.value.code == hp.HPLMM_ERR_INVALID
    s.close()


def test_spmv_noalloc_stale_slots_cleared_between_contexts():
    # a larger system's call leaves NaN in slots of the shared array that a smaller system's Dirichlet-fixed
    # slots overlap; the smaller system's product must not see them (NaN times a zeroed column is NaN)
    import paper_2509_19777_gb300 as hp
    import synth
    lib = hp.load_library()
    big = synth.make_workload("porous24", 2)
    small = synth.make_workload("tiny8", 3)
    sb = hp.Solver(n_mortar=2, contact_halfwidth=1)
    mask, E = hp.problem_to_device(big)
    nb = sb.assemble(mask, E, big.nu, big.bcs)
    xb = torch.full((nb,), float("nan"), dtype=torch.float64, device="cuda")
    yb = torch.empty_like(xb)
    assert lib.hplmm_spmv_noalloc(sb.ctx, ctypes.c_void_p(xb.data_ptr()), ctypes.c_void_p(yb.data_ptr())) == 0
    torch.cuda.synchronize()
    ss = hp.Solver(n_mortar=2, contact_halfwidth=1)
    mask, E = hp.problem_to_device(small)
    ns = ss.assemble(mask, E, small.nu, small.bcs)
    x = torch.from_numpy(np.random.default_rng(5).standard_normal(ns)).cuda()
    y_ref = torch.empty_like(x)
    y_na = torch.empty_like(x)
    assert lib.hplmm_spmv(ss.ctx, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y_ref.data_ptr())) == 0
    assert lib.hplmm_spmv_noalloc(ss.ctx, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y_na.data_ptr())) == 0
    torch.cuda.synchronize()
    a, b = y_na.cpu().numpy(), y_ref.cpu().numpy()
    assert np.isfinite(a).all()
    assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-13
    sb.close()
    ss.close()
