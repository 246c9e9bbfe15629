"""The node-level schedule of the GPU ILU(0) smoother (paper Sections 4.1 and 5; the factorisation and the two
triangular solves run one launch per level lambda = i + 2 j + 4 k, all nodes of a level at once), checked on
the CPU: every neighbour that precedes a node in the elimination order has a smaller level, and eliminating
level by level -- nodes of one level in any order -- gives the oracle's sequential ILU(0) factor.
"""
import itertools

import numpy as np

import synth
from oracle import fem
from oracle.ilu import ILU0, structural_pattern


def test_every_earlier_neighbour_has_a_smaller_level():
    # node ids grow with the grid index x + (nx+1)(y + (ny+1) z), so a neighbour (dx, dy, dz) comes earlier
    # exactly when (dz, dy, dx) is lexicographically negative; its level differs by dx + 2 dy + 4 dz
    for dx, dy, dz in itertools.product((-1, 0, 1), repeat=3):
        if (dx, dy, dz) == (0, 0, 0):
            continue
        earlier = (dz, dy, dx) < (0, 0, 0)
        dlev = dx + 2 * dy + 4 * dz
        assert (dlev < 0) == earlier and dlev != 0


def _levels(sysm):
    ijk = sysm.mesh.node_ijk
    lev_node = ijk[:, 0] + 2 * ijk[:, 1] + 4 * ijk[:, 2]
    node_of_dof = sysm.free // 3
    return lev_node[node_of_dof], node_of_dof


def test_level_order_elimination_equals_the_oracle():
    # row-oriented ILU(0) whose rows are taken level by level (nodes of a level in reverse id order, a node's
    # rows in component order): every row sees the same earlier rows, already final, as in the sequential order
    for name, seed in (("tiny8", 3), ("tiny10", 5)):
        p = synth.make_workload(name, seed)
        sysm = fem.System(p.mask, p.E, p.nu, p.bcs)
        P = structural_pattern(sysm)
        ref = ILU0(sysm.A, P).F.toarray()
        lev, node = _levels(sysm)
        order = sorted(range(sysm.n_dof), key=lambda i: (lev[i], -node[i], i))
        Pd = P.toarray() != 0
        F = np.where(Pd, sysm.A.toarray(), 0.0)
        done = np.zeros(sysm.n_dof, bool)
        for i in order:
            for k in np.flatnonzero(Pd[i, :i]):
                assert done[k], "row eliminated with an unfinished row"
                F[i, k] /= F[k, k]
                js = np.flatnonzero(Pd[i] & Pd[k])
                js = js[js > k]
                F[i, js] -= F[i, k] * F[k, js]
            done[i] = True
        assert np.abs(F - ref).max() <= 1e-12 * np.abs(ref).max()
