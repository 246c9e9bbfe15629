"""Pins for oracle/mortar.py: mortar placement (Section 3.3, Eq. node_init)
and Gaussian mortars (Eq. gauss)."""
import itertools

import numpy as np
import pytest

from oracle.mortar import gaussian_mortars, place_mortars


def _energy(coords, sel):
    X = coords[list(sel)].astype(float)
    e = 0.0
    for a, b in itertools.combinations(range(len(sel)), 2):
        e += 1.0 / np.linalg.norm(X[a] - X[b])
    return e


def test_line_two_mortars_are_endpoints():
    coords = np.array([[3, k, 7] for k in range(11)])
    assert sorted(place_mortars(coords, 2)) == [0, 10]


def test_square_face_four_mortars_are_corners():
    coords = np.array([[i, j, 5] for j in range(5) for i in range(5)])     # x fastest, like node ids
    sel = place_mortars(coords, 4)
    got = sorted(tuple(coords[s][:2]) for s in sel)
    assert got == [(0, 0), (0, 4), (4, 0), (4, 4)]


def test_line_three_mortars_endpoints_and_middle():
    coords = np.array([[k, 0, 0] for k in range(9)])
    assert sorted(place_mortars(coords, 3)) == [0, 4, 8]


def test_all_nodes_when_n_exceeds_size():
    coords = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0]])
    assert place_mortars(coords, 4) == [0, 1, 2]
    assert place_mortars(coords, 3) == [0, 1, 2]


def test_single_mortar_nearest_centroid():
    coords = np.array([[k, 0, 0] for k in range(7)])
    assert place_mortars(coords, 1) == [3]
    coords = np.array([[k, 0, 0] for k in range(6)])       # tie between 2 and 3 -> smaller id
    assert place_mortars(coords, 1) == [2]


@pytest.mark.parametrize("seed", range(6))
def test_coordinatewise_optimum(seed):
    # after the sweeps stop, no single mortar can move to another free node and lower the energy
    rng = np.random.default_rng(seed)
    pts = {(int(a), int(b), 0) for a, b in rng.integers(0, 7, size=(40, 2))}
    coords = np.array(sorted(pts, key=lambda p: (p[2], p[1], p[0])))
    for n in (2, 3, 4, 5):
        sel = place_mortars(coords, n)
        e0 = _energy(coords, sel)
        for i in range(n):
            for y in range(len(coords)):
                if y in sel:
                    continue
                trial = list(sel)
                trial[i] = y
                assert _energy(coords, trial) >= e0 - 1e-12


def test_brute_force_report_small_interfaces():
    # the greedy + sweep placement is a local method; on tiny interfaces it matches the global optimum
    hits = 0
    total = 0
    for seed in range(8):
        rng = np.random.default_rng(100 + seed)
        pts = {(int(a), int(b), 0) for a, b in rng.integers(0, 5, size=(12, 2))}
        coords = np.array(sorted(pts, key=lambda p: (p[2], p[1], p[0])))
        if len(coords) < 4:
            continue
        sel = place_mortars(coords, 3)
        best = min(_energy(coords, c) for c in itertools.combinations(range(len(coords)), 3))
        total += 1
        hits += abs(_energy(coords, sel) - best) < 1e-12
    assert total > 0 and hits >= total // 2


@pytest.mark.parametrize("beta", [1.0, 4.0, 16.0])
def test_gaussian_partition_of_unity_and_peaks(beta):
    rng = np.random.default_rng(1)
    pts = {(int(a), int(b), int(c)) for a, b, c in rng.integers(0, 9, size=(60, 3))}
    coords = np.array(sorted(pts, key=lambda p: (p[2], p[1], p[0])))
    sel = place_mortars(coords, 4)
    eta = gaussian_mortars(coords, sel, beta)
    assert np.abs(eta.sum(axis=1) - 1.0).max() < 1e-15
    assert (eta > 0).all()
    for i, m in enumerate(sel):
        assert np.argmax(eta[m]) == i          # mortar i dominates at its own node


def test_gaussian_closed_form_two_mortars():
    # two mortars 4 apart on a line, beta = 4, min spacing^2 = 16: at the midpoint both weights
    # are 1/2; at node 1: a_0 = -1/64, a_1 = -9/64 -> eta_0 = 1/(1+exp(-1/8))
    coords = np.array([[k, 0, 0] for k in range(5)])
    eta = gaussian_mortars(coords, [0, 4], 4.0)
    assert eta[2, 0] == pytest.approx(0.5, abs=1e-15)
    assert eta[1, 0] == pytest.approx(1.0 / (1.0 + np.exp(-0.125)), rel=1e-15)


def test_single_mortar_is_constant_one():
    coords = np.array([[k, 1, 2] for k in range(5)])
    assert np.array_equal(gaussian_mortars(coords, [2]), np.ones((5, 1)))


# ---------------------------------------------------------------- algebraic mortars (Eq. algebra)
def _alg_case(n, name="tiny8", seed=3):
    import synth
    from oracle import precond
    p = synth.make_workload(name, seed)
    return precond.build(p, precond.Options(n_mortar=n, contact_halfwidth=1, mortar_kind="algebraic"))


@pytest.mark.parametrize("n", [2, 4])
def test_algebraic_mortars_partition_of_unity_and_constraints(n):
    # Eq. algebra: every mortar function is 1 in its own component at its own mortar node and 0 in every
    # component at the other mortar nodes, and the functions of one component sum to e_gamma on the
    # interface (the paper: "guaranteed automatically by superposition")
    sysm, M = _alg_case(n)
    mo, dec = M.mortars, M.dec
    for c in range(dec.n_interfaces):
        nodes = dec.iface_nodes[c]
        rows = [(y, d) for y, node in enumerate(nodes) for d in range(3) if not sysm.fixed[node, d]]
        Q = mo.Qo_block(sysm, dec, c)
        chosen = [int(np.flatnonzero(nodes == m)[0]) for m in mo.mortar_nodes[c]]
        for k, (i, g) in enumerate(mo.columns[c]):
            for r, (y, d) in enumerate(rows):
                if y in chosen:
                    want = 1.0 if (y == chosen[i] and d == g) else 0.0
                    assert Q[r, k] == want
        all_free = all(not sysm.fixed[nodes[ch], g] for ch in chosen for g in range(3))
        if all_free:
            for g in range(3):
                ks = [k for k, (i, gg) in enumerate(mo.columns[c]) if gg == g]
                tot = Q[:, ks].sum(axis=1)
                want = np.array([1.0 if d == g else 0.0 for (y, d) in rows])
                # exact without the diagonal shift; the shift (1e-8 of the diagonal) moves the sums slightly
                assert np.abs(tot - want).max() < 1e-5, (c, g)


def test_algebraic_one_mortar_is_plmm():
    # one mortar per interface: the algebraic function is the rigid translation, the same as the Gaussian
    # one (eta = 1), so both give PLMM's coarse matrix
    import synth
    from oracle import precond
    p = synth.make_workload("tiny8", 3)
    Ao = {}
    for kind in ("gaussian", "algebraic"):
        sysm, M = precond.build(p, precond.Options(n_mortar=1, contact_halfwidth=1, mortar_kind=kind))
        Ao[kind] = M.coarse.A_o
    # equal but for the diagonal shift of the interface operator (1e-8 of A_hat's diagonal)
    assert np.abs(Ao["gaussian"] - Ao["algebraic"]).max() < 1e-5 * np.abs(Ao["gaussian"]).max()


def _iface_operator_case(c_pick=None):
    sysm, M = _alg_case(4)
    mo, dec = M.mortars, M.dec
    out = []
    for c in range(dec.n_interfaces):
        nodes = dec.iface_nodes[c]
        rows = [(y, d) for y, node in enumerate(nodes) for d in range(3) if not sysm.fixed[node, d]]
        S = mo._interface_operator(sysm, dec, c, rows)
        f2f = sysm.full_to_free
        J = np.array([f2f[3 * nodes[y] + d] for (y, d) in rows])
        out.append((nodes, rows, S, J))
    return sysm, out


def test_algebraic_interface_operator_properties():
    # S^c - shift annihilates every rigid translation of the interface, is symmetric positive semidefinite,
    # and S^c itself is positive definite (so the band Cholesky of the reduced systems cannot break down)
    from oracle import mortar
    sysm, cases = _iface_operator_case()
    diagA = sysm.A.diagonal()
    for nodes, rows, S, J in cases:
        S0 = S - np.diag(mortar.ALG_SHIFT * diagA[J])
        scale = np.abs(S0).max()
        assert np.abs(S0 - S0.T).max() <= 1e-14 * scale
        for g in range(3):
            t = np.array([1.0 if d == g else 0.0 for (y, d) in rows])
            assert np.abs(S0 @ t).max() <= 1e-12 * scale
        ev = np.linalg.eigvalsh(S0)
        assert ev.min() >= -1e-12 * scale
        assert np.linalg.eigvalsh(S).min() > 0


def test_algebraic_interface_operator_edge_blocks():
    # the off-diagonal block of S^c for a node pair is -|B|, B = -sym(A_yy'), checked against what fixes the
    # matrix absolute value without computing it: |B| is the one positive semidefinite matrix whose square is
    # B^2; where B is itself positive semidefinite (an attractive coupling) the block is sym(A_yy'), A_hat's
    # own coupling.  Brute force over all node pairs of every interface
    sysm, cases = _iface_operator_case()
    A = sysm.A.toarray()
    n_att = n_mixed = 0
    for nodes, rows, S, J in cases:
        pos = {yd: r for r, yd in enumerate(rows)}
        F = len(nodes)
        for y in range(F):
            for z in range(F):
                if y == z:
                    continue
                free = [(d, e) for d in range(3) for e in range(3) if (y, d) in pos and (z, e) in pos]
                blk = np.zeros((3, 3))
                for d, e in free:
                    blk[d, e] = A[J[pos[(y, d)]], J[pos[(z, e)]]]
                if not blk.any():
                    continue
                B = -0.5 * (blk + blk.T)
                off = np.zeros((3, 3))
                for d, e in free:
                    off[d, e] = S[pos[(y, d)], pos[(z, e)]]
                scale = np.abs(B).max()
                if len(free) == 9:
                    absB = -off
                    assert np.abs(absB - absB.T).max() <= 1e-13 * scale
                    assert np.linalg.eigvalsh(absB).min() >= -1e-13 * scale
                    assert np.abs(absB @ absB - B @ B).max() <= 1e-12 * scale ** 2
                if np.linalg.eigvalsh(B).min() >= 0:
                    for d, e in free:
                        assert abs(off[d, e] + B[d, e]) <= 1e-13 * scale
                    n_att += 1
                else:
                    n_mixed += 1
    assert n_att > 0 and n_mixed > 0


def test_algebraic_all_nodes_mortars_is_identity():
    # n_c = |F|: every interface DOF is a mortar DOF, so Q^o is the identity and the first pass is exact
    import scipy.sparse.linalg as spla
    import synth
    from oracle import precond
    p = synth.make_workload("tiny6", 1)
    sysm, M = precond.build(p, precond.Options(n_mortar=10 ** 4, contact_halfwidth=1, mortar_kind="algebraic"))
    for c in range(M.dec.n_interfaces):
        Q = M.mortars.Qo_block(sysm, M.dec, c)
        assert Q.shape[0] == Q.shape[1] and np.array_equal(Q, np.eye(Q.shape[0]))
    xs = spla.spsolve(sysm.A.tocsc(), sysm.b)
    assert np.linalg.norm(M.M_G(sysm.b) - xs) < 1e-10 * np.linalg.norm(xs)


# ---------------------------------------------------------------- the spread beta (Appendix A)
def test_gaussian_mortars_beta_limits():
    # Eq. gauss as beta -> infinity: every exponent tends to 0, so the mortars flatten to 1/n_c on the whole
    # interface (linearly dependent columns); as beta -> 0 each node belongs to the mortar with the smallest
    # d^2 / dmin^2 (with a symmetric layout, the nearest mortar): indicator functions
    coords = np.array([[0, y, z] for y in range(7) for z in range(7)])
    chosen = [0, 6, 42, 48]                        # the four corners: equal nearest-mortar distances
    eta_inf = gaussian_mortars(coords, chosen, beta=1e12)
    assert np.abs(eta_inf - 0.25).max() < 1e-10
    eta_0 = gaussian_mortars(coords, chosen, beta=1e-3)
    X = coords[chosen]
    d2 = ((coords[:, None, :] - X[None, :, :]) ** 2).sum(axis=2)
    for y in range(len(coords)):
        order = np.sort(d2[y])
        if order[0] < order[1]:                    # a unique nearest mortar
            want = np.zeros(4)
            want[np.argmin(d2[y])] = 1.0
            assert np.abs(eta_0[y] - want).max() < 1e-12, y


def test_coarse_conditioning_grows_with_beta():
    # Appendix A: the larger beta, the more adjacent mortars overlap and the worse A^o is conditioned
    import synth
    from oracle import precond
    p = synth.make_workload("tiny8", 3)
    kappa = []
    for beta in (0.25, 1.0, 4.0, 16.0, 64.0):
        sysm, M = precond.build(p, precond.Options(n_mortar=2, contact_halfwidth=1, beta=beta))
        ev = np.linalg.eigvalsh(M.coarse.A_o)
        assert ev[0] > 0
        kappa.append(ev[-1] / ev[0])
    assert all(b > a for a, b in zip(kappa, kappa[1:])), kappa
