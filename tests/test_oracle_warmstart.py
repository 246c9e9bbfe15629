"""Pins for oracle/warmstart.py: the learned warm start of the local basis
solves and the preconditioned CG basis solver (no counterpart in the paper's
own runs, which solve the local problems exactly; Eqs. col_pk, col_cg)."""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import synth
from oracle import precond, warmstart as ws
from oracle.decomposition import cartesian_partition


def _toy(seed, B=2, D=4, channels=(2, 3, 3, 2)):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((B, channels[0], D, D, D))
    t = rng.standard_normal((B, channels[-1], D, D, D))
    valid = (rng.uniform(size=t.shape) < 0.7).astype(np.float64)
    theta = rng.standard_normal(ws.n_params(channels)) * 0.3
    return x, t, valid, theta


def test_gradient_matches_central_differences():
    channels = (2, 3, 3, 2)
    x, t, valid, theta = _toy(0, channels=channels)
    loss, g = ws.loss_and_grad(theta, x, t, valid, channels)
    rng = np.random.default_rng(1)
    idx = rng.choice(theta.size, size=40, replace=False)
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (ws.loss_and_grad(tp, x, t, valid, channels)[0] - ws.loss_and_grad(tm, x, t, valid, channels)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_delta_kernel_shifts_the_input():
    # a single tap (tz, ty, tx) = (2, 1, 0) with weight 1 gives y[z][y][x] = x[z+1][y][x-1] (zeros outside)
    rng = np.random.default_rng(2)
    x = rng.standard_normal((1, 1, 5, 5, 5))
    W = np.zeros((1, 1, 3, 3, 3))
    W[0, 0, 2, 1, 0] = 1.0
    y = ws.conv3d(x, W, np.zeros(1))
    ref = np.zeros_like(x)
    ref[0, 0, :4, :, 1:] = x[0, 0, 1:, :, :4]
    assert np.array_equal(y, ref)


def test_dilated_delta_kernel_shifts_by_the_dilation():
    rng = np.random.default_rng(9)
    x = rng.standard_normal((1, 1, 9, 9, 9))
    W = np.zeros((1, 1, 3, 3, 3))
    W[0, 0, 0, 2, 1] = 1.0  # offset (-d, +d, 0)
    y = ws.conv3d(x, W, np.zeros(1), dil=4)
    ref = np.zeros_like(x)
    ref[0, 0, 4:, :5, :] = x[0, 0, :5, 4:, :]
    assert np.array_equal(y, ref)


def test_shift_beyond_the_grid_is_zero():
    x = np.ones((1, 1, 5, 5, 5))
    assert not ws._shift(x, 8, 0, 0).any() and not ws._shift(x, 0, -5, 0).any()
    assert ws._shift(x, 4, 0, 0).sum() == 25


def test_receptive_field_spans_the_grain():
    # with dilations 1, 2, 4, 8 an output depends on inputs up to 15 nodes away along each axis, i.e. on
    # every node of a 16-voxel grain but the opposite corner row
    assert sum(ws.DILATIONS) == ws.GRID - 2


def test_conv_is_linear_and_bias_is_constant():
    rng = np.random.default_rng(3)
    x1, x2 = rng.standard_normal((2, 1, 2, 4, 4, 4))
    W = rng.standard_normal((3, 2, 3, 3, 3))
    b = rng.standard_normal(3)
    y = ws.conv3d(x1 + 2 * x2, W, b)
    y1 = ws.conv3d(x1, W, np.zeros(3))
    y2 = ws.conv3d(x2, W, np.zeros(3))
    assert np.allclose(y, y1 + 2 * y2 + b[None, :, None, None, None], atol=1e-12)


def test_adam_first_step_and_convergence():
    # the bias-corrected first step moves every coordinate by lr * g / (|g| + eps) ~ lr * sign(g)
    th = np.array([1.0, -2.0])
    g = np.array([0.5, -4.0])
    t1, m, v = ws.adam_step(th, g, np.zeros(2), np.zeros(2), 1, 0.1)
    assert np.allclose(t1, th - 0.1 * g / (np.abs(g) + 1e-8), atol=1e-15)
    # and it minimises (w - 3)^2
    w, m, v = np.array([0.0]), np.zeros(1), np.zeros(1)
    for k in range(1, 3001):
        w, m, v = ws.adam_step(w, 2 * (w - 3.0), m, v, k, 0.05)
    assert abs(w[0] - 3.0) < 1e-3


def test_param_count_and_packing():
    assert ws.n_params() == 32 * 5 * 27 + 32 + 2 * (32 * 32 * 27 + 32) + 3 * 32 * 27 + 3
    th = ws.init_params(4)
    assert th.dtype == np.float32 and th.size == ws.n_params()
    assert np.array_equal(ws.pack(ws.unpack(th)), th)


def test_sample_reproduces_the_basis_column():
    # the target channels of a grain's sample, mapped back to DOFs, are its exact basis column; the rhs
    # channels times s are the right-hand side, and every free DOF of the grain is a valid entry
    p = synth.make_workload("cube16", 0)
    sysm, M = precond.build(p, precond.Options(n_mortar=2, contact_halfwidth=1))
    part = cartesian_partition(p.mask.shape, p.grains)
    A = sysm.A.tocsr()
    g = 3
    I = M.dec.grain_dofs[g]
    o = ws.grain_box_origin(sysm, part, g)
    fields, ebar = ws.grain_fields(sysm, part, g, o)
    pos = ws.dof_positions(sysm, I, o)
    assert np.all((np.stack(pos[1:]) >= 0) & (np.stack(pos[1:]) < ws.GRID))
    rng = np.random.default_rng(5)
    rhs = rng.standard_normal(I.size)
    x = spla.spsolve(A[I][:, I].tocsc(), rhs)
    inp, tgt, valid = ws.make_sample(fields, pos, rhs, x)
    s = np.sqrt(np.mean(rhs * rhs))
    assert valid.sum() == I.size
    assert np.allclose(inp[2:][pos] * s, rhs, rtol=0, atol=1e-12)
    assert np.allclose(ws.guess_from_prediction(tgt, pos) * np.sqrt(np.mean(x * x)), x, rtol=1e-12, atol=0)
    # with the guess direction of the exact solution, the energy-optimal scaling reproduces the solution
    xg, its, rel0 = ws.pcg(A[I][:, I], rhs, sp.identity(I.size), x0=ws.guess_from_prediction(tgt, pos), tol=1e-9)
    assert its == 0 and rel0 < 1e-9
    assert inp[0].sum() == 16 * 16 * 16 / 8  # a solid 8^3 grain of cube16 (2x2x2 grains)


def test_pcg_matches_direct_solve_and_warm_start_helps():
    p = synth.make_workload("tiny10", 5)
    sysm, M = precond.build(p, precond.Options(n_mortar=2, contact_halfwidth=1))
    A = sysm.A.tocsr()
    I = M.dec.grain_dofs[0]
    Agg = A[I][:, I]
    node = sysm.free[I] // 3
    Dinv = ws.block_jacobi_inverse(Agg, node)
    rng = np.random.default_rng(6)
    b = rng.standard_normal(I.size)
    x_ref = spla.spsolve(Agg.tocsc(), b)
    x, its, rel0 = ws.pcg(Agg, b, Dinv, tol=1e-10)
    assert np.linalg.norm(x - x_ref) <= 1e-8 * np.linalg.norm(x_ref)
    assert rel0 == 1.0 and its > 0
    # a guess within 0.1% of the solution starts from a smaller residual and needs fewer iterations
    x0 = x_ref + 1e-3 * np.linalg.norm(x_ref) / np.sqrt(I.size) * rng.standard_normal(I.size)
    xw, its_w, rel0_w = ws.pcg(Agg, b, Dinv, x0=x0, tol=1e-10)
    assert rel0_w < rel0 and its_w < its
    assert np.linalg.norm(xw - x_ref) <= 1e-8 * np.linalg.norm(x_ref)
    # the scaled guess is never worse than the zero guess in the A-norm, even for a poor guess
    bad = rng.standard_normal(I.size)
    xs = bad * ((bad @ b) / (bad @ (Agg @ bad)))
    e0 = x_ref @ (Agg @ x_ref)
    es = (xs - x_ref) @ (Agg @ (xs - x_ref))
    assert es <= e0 * (1 + 1e-12)
    # the block-Jacobi operator is the inverse of the node-diagonal part
    Bd = Agg.toarray() * (node[:, None] == node[None, :])
    assert np.allclose(Dinv.toarray() @ Bd, np.eye(I.size), atol=1e-10)


def test_round_bf16_against_its_definition():
    # values the 8-bit significand holds exactly stay; halfway cases go to the even neighbour; others to the
    # nearest; the result always has 16 zero low bits and is within half a unit: 2^-8 relative (the unit
    # roundoff of an 8-bit significand)
    assert ws.round_bf16(1.0) == 1.0 and ws.round_bf16(-3.5) == -3.5
    assert ws.round_bf16(1.0 + 2.0 ** -8) == 1.0                       # tie: 1.0 is even
    assert ws.round_bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6       # tie: up to the even neighbour
    assert ws.round_bf16(1.0 + 2.0 ** -8 + 2.0 ** -20) == 1.0 + 2.0 ** -7
    rng = np.random.default_rng(0)
    v = rng.standard_normal(10000) * 10.0 ** rng.uniform(-5, 5, 10000)
    r = ws.round_bf16(v)
    bits = r.astype(np.float32).view(np.uint32)
    assert np.all(bits & 0xFFFF == 0)
    assert np.all(np.abs(r - v.astype(np.float32)) <= 2.0 ** -8 * np.abs(v.astype(np.float32)) * (1 + 1e-7))


def test_forward_bf16_is_forward_of_rounded_weights_when_activations_are_exact():
    # with weights that are already BF16 values and a one-layer network, the BF16 path equals the plain
    # forward of those weights (rounded to FP32 at the output)
    rng = np.random.default_rng(2)
    ch = (2, 3)
    theta = ws.round_bf16(rng.standard_normal(ws.n_params(ch)) * 0.1)
    x = ws.round_bf16(rng.standard_normal((1, 2, 5, 5, 5)))
    ref = ws.forward(theta, x, ch)[-1]
    got = ws.forward_bf16(theta, x, ch)
    assert np.abs(got - ref).max() <= 2.0 ** -23 * np.abs(ref).max()
