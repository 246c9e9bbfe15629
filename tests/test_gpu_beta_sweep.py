"""The spread beta of the Gaussian mortars (paper Eq. gauss; Appendix A): through the CUDA path, the coarse
matrix's condition number, the first-pass error of M_G b and the FGMRES iterations as beta grows.

Appendix A: too small a beta makes the mortars nearly indicator functions of their neighbourhoods and the
first-pass error grows; too large a beta makes adjacent mortars overlap and A^o ill-conditioned.  The
oracle gives, on porous32 with n = 4 (beta 0.25 / 1 / 4 / 16 / 64): kappa(A^o) 9.5e4 / 3.0e5 / 5.6e7 /
4.4e10 / 1.9e14, first-pass error 0.261 / 0.130 / 0.133 / 0.139 / 0.147, 66 / 60 / 60 / 61 / 61 GMRES
iterations.  The GPU's A^o at each beta is compared with the oracle's at beta = 1 and 16 (relative 1e-10).
"""
import numpy as np
import pytest

from tests._cases import gpu_solver, problem, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BETAS = (0.25, 1.0, 4.0, 16.0, 64.0)


def test_beta_sweep_conditioning_and_first_pass():
    import scipy.sparse.linalg as spla
    from oracle import fem, precond
    p, opt = problem("porous32_n4")
    sysm = fem.System(p.mask, p.E, p.nu, p.bcs)
    xs = spla.spsolve(sysm.A.tocsc(), sysm.b)
    rows = []
    for beta in BETAS:
        s = gpu_solver("porous32_n4", beta=beta)
        Ao = s.coarse_matrix().cpu().numpy()
        if beta in (1.0, 16.0):
            _, M = precond.build(p, precond.Options(n_mortar=opt["n_mortar"], contact_halfwidth=opt["contact_halfwidth"],
                                                    beta=beta))
            assert np.abs(Ao - M.coarse.A_o).max() <= 1e-10 * np.abs(M.coarse.A_o).max()
        ev = np.linalg.eigvalsh(0.5 * (Ao + Ao.T))
        xa = s.apply_coarse(s.b).cpu().numpy()
        x, rc, st = s.solve(tol=1e-8)
        assert rc == 0
        rows.append((beta, ev[-1] / ev[0], rel(xa, xs), st.iters))
        s.close()
    for beta, kappa, e, its in rows:
        print(f"beta {beta:6.2f}: kappa(A^o) {kappa:.3e}, first-pass error {e:.4f}, {its} FGMRES iterations")
    kappas = [r[1] for r in rows]
    assert all(b > a for a, b in zip(kappas, kappas[1:])), kappas
    err = {r[0]: r[2] for r in rows}
    its = {r[0]: r[3] for r in rows}
    assert err[0.25] > 1.5 * err[4.0]          # too narrow: the first pass degrades
    assert its[4.0] <= its[0.25]
