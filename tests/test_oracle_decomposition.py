"""Pins for oracle/decomposition.py: grain grids, interfaces, W (paper
Sections 3.1-3.2, Eq. permute).  Checked against a hand-derived census
(tests/golden/partition_4cube_2x2x2.txt) and structural invariants."""
import os

import numpy as np

from oracle import fem
from oracle.decomposition import Decomposition, cartesian_partition

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "partition_4cube_2x2x2.txt")
FREE = {f: {"fix": (False,) * 3, "value": (0.0,) * 3, "traction": (0.0,) * 3} for f in fem.FACES}


def _dec(mask, grains, strict=False, bcs=FREE):
    sysm = fem.System(mask, np.ones(mask.shape), 0.3, bcs)
    g = cartesian_partition(mask.shape, grains)
    return sysm, Decomposition(sysm, g, grains[0] * grains[1] * grains[2], strict)


def test_cartesian_partition_formula():
    g = cartesian_partition((4, 6, 5), (2, 3, 2))
    assert g[0, 0, 0] == 0
    assert g[0, 0, 4] == 1            # floor(4*2/5) = 1
    assert g[0, 0, 2] == 0            # floor(2*2/5) = 0
    assert g[0, 5, 0] == 2 * 2        # gy = floor(5*3/6) = 2
    assert g[3, 0, 0] == 2 * 3 * 1


def test_hand_derived_census_4cube():
    sysm, d = _dec(np.ones((4, 4, 4), np.uint8), (2, 2, 2))
    rows = [tuple(int(v) for v in l.split()) for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    got = [(int(d.iface_pair[c, 0]), int(d.iface_pair[c, 1]), len(d.iface_nodes[c])) for c in range(d.n_interfaces)]
    assert got == rows
    assert [len(n) for n in d.grain_nodes] == [8] * 8
    assert d.is_interface_node.sum() == 61
    # the centre node (2,2,2) touches all eight grains and lies on the (0,1) interface
    centre = sysm.mesh.grid_to_node[2, 2, 2]
    assert d.iface_of_node[centre] == 0
    assert list(d.iface_grains[0]) == list(range(8))


def test_strict_two_grain_coupling():
    _, d = _dec(np.ones((4, 4, 4), np.uint8), (2, 2, 2), strict=True)
    for c in range(d.n_interfaces):
        assert list(d.iface_grains[c]) == sorted(d.iface_pair[c].tolist())


def test_W_is_a_permutation_and_sets_partition_dofs():
    rng = np.random.default_rng(5)
    mask = (rng.random((6, 7, 8)) < 0.75).astype(np.uint8)
    bcs = dict(FREE)
    bcs["z0"] = {"fix": (True, False, True), "value": (0.0,) * 3, "traction": (0.0,) * 3}
    sysm, d = _dec(mask, (2, 2, 3), bcs=bcs)
    assert np.array_equal(np.sort(d.W), np.arange(sysm.n_dof))
    # grain DOFs first, then interfaces, each block in ascending DOF (= node) order
    pos = 0
    for S in d.grain_dofs + d.iface_dofs:
        assert np.array_equal(d.W[pos:pos + S.size], S)
        assert (np.diff(S) > 0).all()
        pos += S.size
    # a grain node has exactly one grain among its solid neighbours
    assert (d.nS[d.is_grain_node] == 1).all()
    assert (d.nS[d.is_interface_node] >= 2).all()


def test_split_interface_components():
    # grains 0 | 1 along x, touching through two separate bridges -> two interfaces for the pair
    mask = np.zeros((1, 5, 4), np.uint8)     # nz=1, ny=5, nx=4
    mask[0, :, :] = 1
    mask[0, 2, :] = 0                        # a void row splits the contact into two patches ...
    mask[0, 2, 0] = 1                        # ... but keeps the left grain connected
    sysm, d = _dec(mask, (2, 1, 1))
    pairs = [tuple(p) for p in d.iface_pair.tolist()]
    assert pairs == [(0, 1), (0, 1)]
    a, b = d.iface_nodes
    assert a.min() < b.min()                 # ordered by smallest node id
    assert np.intersect1d(a, b).size == 0
