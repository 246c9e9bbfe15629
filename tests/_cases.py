"""Shared helpers for the GPU parity tests: seeded workloads, oracle runs cached
per process, and conversions between numpy and torch."""
import functools

import numpy as np

import synth
from oracle import fem, gmres, precond
from oracle.decomposition import cartesian_partition

# (workload, seed, options) -> small cases the oracle finishes in seconds, spanning several
# grains, porous geometry, heterogeneous moduli and the edge cases of the method
CASES = {
    "cube16_n4": ("cube16", 0, dict(n_mortar=4, contact_halfwidth=1)),
    "tiny8_n2": ("tiny8", 3, dict(n_mortar=2, contact_halfwidth=1)),
    "tiny10_n1": ("tiny10", 5, dict(n_mortar=1, contact_halfwidth=1)),
    "tiny10_strict": ("tiny10", 6, dict(n_mortar=3, contact_halfwidth=1, strict_two_grain=True)),
    "porous32_n4": ("porous32", 1, dict(n_mortar=4, contact_halfwidth=2)),
    # the fractured recipe at 32^3 (2x2x2 grains): Voronoi two-phase E in {1, 10} and three one-voxel slits
    # with E x 1e-4 crossing the grains and their interfaces
    "fractured32_n2": ("fractured32", 0, dict(n_mortar=2, contact_halfwidth=2)),
    # algebraic mortars (Eq. algebra)
    "tiny8_alg": ("tiny8", 3, dict(n_mortar=2, contact_halfwidth=1, mortar_kind="algebraic")),
    "porous32_alg": ("porous32", 1, dict(n_mortar=4, contact_halfwidth=2, mortar_kind="algebraic")),
    # large local sets: 216 grains of 4^3 voxels (more grains than half the SMs: one CTA per problem in the
    # factorisation) and 512 grains (more problems than two per SM: the persistent queue hands CTAs several
    # problems), both with more than 500 contact grids and a deep coarse elimination tree
    "porous24_g216": ("porous24", 1, dict(n_mortar=1, contact_halfwidth=1, grains=(6, 6, 6))),
    "porous32_g512": ("porous32", 1, dict(n_mortar=1, contact_halfwidth=1, grains=(8, 8, 8))),
    # the ILU(0) base smoother with the paper's six stages (its smoother comparison, Section 5)
    "tiny8_ilu": ("tiny8", 3, dict(n_mortar=2, contact_halfwidth=1, smoother="ilu0", n_st=6)),
    "cube16_ilu": ("cube16", 0, dict(n_mortar=4, contact_halfwidth=1, smoother="ilu0", n_st=6)),
    "porous32_ilu": ("porous32", 1, dict(n_mortar=4, contact_halfwidth=2, smoother="ilu0", n_st=6)),
}


def problem(name):
    wl, seed, opt = CASES[name]
    p = synth.make_workload(wl, seed)
    if "grains" in opt:
        p.grains = tuple(opt["grains"])
    return p, opt


@functools.lru_cache(maxsize=None)
def oracle_case(name):
    """(problem, options, oracle system, oracle preconditioner)."""
    p, opt = problem(name)
    o = precond.Options(n_mortar=opt["n_mortar"], contact_halfwidth=opt["contact_halfwidth"],
                        strict_two_grain=opt.get("strict_two_grain", False),
                        mortar_kind=opt.get("mortar_kind", "gaussian"),
                        smoother=opt.get("smoother", "contact_grain"), n_st=opt.get("n_st", 1))
    sysm, M = precond.build(p, o)
    return p, opt, sysm, M


@functools.lru_cache(maxsize=None)
def oracle_solution(name, tol=1e-11):
    p, opt, sysm, M = oracle_case(name)
    x, st = gmres.gmres(sysm.A, sysm.b, M.apply, tol=tol)
    return x, st


def maxrel(a, b):
    """Element-wise error: max |a - b| over the largest |b| (a wrong value on a few entries of a long vector
    shows here even when the norm-wise error stays small)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    m = np.abs(b).max() if b.size else 0.0
    d = np.abs(a - b).max() if b.size else 0.0
    return d / m if m > 0 else d


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    d = np.linalg.norm(a - b)
    n = np.linalg.norm(b)
    return d / n if n > 0 else d


def gpu_solver(name, **over):
    import torch
    import paper_2509_19777_gb300 as hp
    p, opt = problem(name)
    kw = dict(n_mortar=opt["n_mortar"], contact_halfwidth=opt["contact_halfwidth"],
              strict_two_grain=opt.get("strict_two_grain", False), mortar_kind=opt.get("mortar_kind", "gaussian"),
              smoother=opt.get("smoother", "contact_grain"), n_st=opt.get("n_st", 1))
    kw.update(over)
    s = hp.Solver(**kw)
    mask, E = hp.problem_to_device(p)
    s.assemble(mask, E, p.nu, p.bcs)
    s.setup(grains=p.grains)
    torch.cuda.synchronize()
    return s
