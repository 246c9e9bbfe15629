"""The hPLMM preconditioner M (paper Section 4.1, Eqs. multi_precond and
local_smoother) and its set-up from an image.

ORACLE -- test infrastructure only (see oracle/__init__.py).

* Eq. multi_precond: M^{-1} = M_G^{-1} + M_L^{-1} (I - A_hat M_G^{-1}); M_G first.
* Eq. local_smoother: M_L^{-1} = sum_{i=1}^{n_st} M_l^{-1} prod_{j<i} (I - A_hat M_l^{-1})
  with base smoother M_l = M_CG (n_st = 1 in the paper's runs) or, for the paper's smoother comparison,
  M_l = M_ILU(0) (oracle/ilu.py; n_st = 6 there).
Applied to r this is: z1 = M_G^{-1} r; r1 = r - A_hat z1; then n_st stages of
t = M_l^{-1} res, s += t, res -= A_hat t; return z1 + s.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import fem
from .coarse import CoarseSpace
from .decomposition import Decomposition, cartesian_partition
from .ilu import ILU0Smoother
from .mortar import Mortars
from .smoother import ContactGrainSmoother


@dataclasses.dataclass
class Options:
    n_mortar: int = 4          # n: maximum mortar nodes per interface
    beta: float = 4.0          # Gaussian mortar spread (Eq. gauss; Appendix A)
    contact_halfwidth: int = 2  # w: contact grid = interface dilated by w nodes
    n_st: int = 1              # smoother stages (Eq. local_smoother)
    strict_two_grain: bool = False
    keep_corrections: bool = True
    mortar_kind: str = "gaussian"   # "gaussian" (Eq. gauss) or "algebraic" (Eq. algebra)
    smoother: str = "contact_grain"  # base smoother M_l: "contact_grain" (M_CG) or "ilu0" (M_ILU(0))


class HPLMM:
    """Set-up (T_MG + T_ML) and application of M for one system."""

    def __init__(self, system, grain_of_voxel, n_grains, opt=Options()):
        self.system = system
        self.opt = opt
        self.dec = Decomposition(system, grain_of_voxel, n_grains, opt.strict_two_grain)
        self.mortars = Mortars(system, self.dec, opt.n_mortar, opt.beta, opt.mortar_kind)
        self.coarse = CoarseSpace(system, self.dec, self.mortars, opt.keep_corrections)
        if opt.smoother == "ilu0":
            self.smoother = ILU0Smoother(system)
        else:
            self.smoother = ContactGrainSmoother(system, self.dec, self.coarse, opt.contact_halfwidth)
        self.A = system.A.tocsr()

    def M_G(self, r):
        return self.coarse.apply(r)

    def M_L(self, r):
        s = np.zeros_like(r)
        res = r
        for _ in range(self.opt.n_st):
            t = self.smoother.apply(res)
            s = s + t
            res = res - self.A @ t
        return s

    def apply(self, r):
        """z = M^{-1} r, Eq. multi_precond."""
        z1 = self.M_G(r)
        r1 = r - self.A @ z1
        return z1 + self.M_L(r1)


def build(problem, opt=None):
    """System + preconditioner for a synth.Problem (Cartesian grains)."""
    if opt is None:
        opt = Options(n_mortar=problem.n_mortar)
    system = fem.System(problem.mask, problem.E, problem.nu, problem.bcs)
    px, py, pz = problem.grains
    grains = cartesian_partition(problem.mask.shape, problem.grains)
    return system, HPLMM(system, grains, px * py * pz, opt)
