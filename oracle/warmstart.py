"""Learned warm start of the local basis solves, and the Jacobi-preconditioned
conjugate-gradient basis solver it feeds.

ORACLE -- test infrastructure only (see oracle/__init__.py).

The paper solves every local basis problem exactly (Eqs. col_pk and col_cg,
Section 6.3).  This module states, in plain FP64 numpy, the optional
iterative path: a small 3-D convolutional network maps a grain's geometry,
moduli and the right-hand side of one basis problem to an initial guess, and
block-Jacobi-preconditioned CG refines it (the exact local solve stays the
judge of its error and the fallback).

Sample of one basis problem (grain g, right-hand side column a):
  grid      the grain's voxel box origin o = minimum corner of its solid voxels
            (the box must fit in 16^3 voxels), nodes o + (i, j, k), 0 <= i,j,k <= 16
            (GRID = 17 per axis, arrays indexed [z][y][x])
  ch 0      1 on voxel (i,j,k) < 16 if it is a solid voxel of grain g, else 0
  ch 1      log E of that voxel (0 elsewhere)
  ch 2..4   the right-hand side's x, y, z components on the grain's free DOFs,
            divided by s = RMS of the right-hand side over those DOFs
  target    the basis column (exact local solve) divided by its RMS over the
            grain's free DOFs, on the same positions
  valid     1 where a free DOF of the grain sits, else 0
A prediction q, read at the valid positions, is the direction of the initial
guess: CG scales it by the factor that minimises the A-norm error along it,
so only the shape of the solution has to be learned.

Network: 4 layers of 3x3x3 convolutions with zero padding ("same" size) and
dilations 1, 2, 4, 8 (receptive field 31 nodes: an output sees inputs up to 15
nodes away along each axis, nearly the whole 17^3 grid), channels 5 -> 32 -> 32 -> 32 -> 3, bias per output channel, ReLU
after the first three.  Flat parameter vector (the exchange format with the library):
for each layer in order, W[co][ci][tz][ty][tx] (tap (tz,ty,tx) of a layer with
dilation d reads offset ((tz-1)d, (ty-1)d, (tx-1)d) in (z, y, x)), then bias[co].
Loss: sum over valid entries of (q - target)^2 divided by the number of valid
entries.  Optimiser: Adam (Kingma and Ba, 2015) with bias correction.

Pins (tests/test_oracle_warmstart.py): the analytic gradient against central
finite differences in FP64; a delta kernel reproducing a shifted input; the
Adam step against its closed form on a scalar quadratic; the sample of a grain
reproducing the oracle's own basis column; CG against a direct solve.
"""
from __future__ import annotations

import numpy as np

GRID = 17
CHANNELS = (5, 32, 32, 32, 3)
DILATIONS = (1, 2, 4, 8)


def layer_shapes(channels=CHANNELS):
    return [(channels[i + 1], channels[i]) for i in range(len(channels) - 1)]


def n_params(channels=CHANNELS):
    return sum(co * ci * 27 + co for co, ci in layer_shapes(channels))


def unpack(theta, channels=CHANNELS):
    """Flat parameter vector -> [(W[co][ci][3][3][3], b[co]), ...]."""
    out, pos = [], 0
    for co, ci in layer_shapes(channels):
        W = theta[pos:pos + co * ci * 27].reshape(co, ci, 3, 3, 3)
        pos += co * ci * 27
        b = theta[pos:pos + co]
        pos += co
        out.append((W, b))
    return out


def pack(layers):
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in layers])


def _shift(x, dz, dy, dx):
    """y[..., z, y, x] = x[..., z+dz, y+dy, x+dx] with zeros outside."""
    out = np.zeros_like(x)
    D = x.shape[-3:]
    if abs(dz) >= D[0] or abs(dy) >= D[1] or abs(dx) >= D[2]:
        return out  # the shifted grid lies entirely outside
    sz = slice(max(0, -dz), D[0] - max(0, dz))
    sy = slice(max(0, -dy), D[1] - max(0, dy))
    sx = slice(max(0, -dx), D[2] - max(0, dx))
    tz = slice(max(0, dz), D[0] - max(0, -dz))
    ty = slice(max(0, dy), D[1] - max(0, -dy))
    tx = slice(max(0, dx), D[2] - max(0, -dx))
    out[..., sz, sy, sx] = x[..., tz, ty, tx]
    return out


def conv3d(x, W, b, dil=1):
    """x [B][ci][D][D][D] -> y [B][co][D][D][D]:
    y[n][o][p] = b[o] + sum_{i, t} W[o][i][t] x[n][i][p + (t - 1) dil] (zero padding)."""
    B = x.shape[0]
    co = W.shape[0]
    y = np.broadcast_to(b[None, :, None, None, None], (B, co) + x.shape[2:]).astype(np.float64).copy()
    for tz in range(3):
        for ty in range(3):
            for tx in range(3):
                xs = _shift(x, (tz - 1) * dil, (ty - 1) * dil, (tx - 1) * dil)
                y += np.einsum("oi,nizyx->nozyx", W[:, :, tz, ty, tx], xs)
    return y


def conv3d_backward(x, W, gy, dil=1):
    """Gradients of conv3d: (dL/dx, dL/dW, dL/db) given dL/dy."""
    gx = np.zeros_like(x, dtype=np.float64)
    gW = np.zeros_like(W, dtype=np.float64)
    for tz in range(3):
        for ty in range(3):
            for tx in range(3):
                dz, dy, dx = (tz - 1) * dil, (ty - 1) * dil, (tx - 1) * dil
                xs = _shift(x, dz, dy, dx)
                gW[:, :, tz, ty, tx] = np.einsum("nozyx,nizyx->oi", gy, xs)
                # y[p] uses x[p + offset]: the adjoint moves gy by the opposite offset
                gx += _shift(np.einsum("oi,nozyx->nizyx", W[:, :, tz, ty, tx], gy), -dz, -dy, -dx)
    gb = gy.sum(axis=(0, 2, 3, 4))
    return gx, gW, gb


def forward(theta, x, channels=CHANNELS):
    """Activations [x, a1, a2, a3, q]; ReLU after every layer but the last."""
    acts = [np.asarray(x, np.float64)]
    layers = unpack(np.asarray(theta, np.float64), channels)
    for li, (W, b) in enumerate(layers):
        z = conv3d(acts[-1], W, b, DILATIONS[li])
        acts.append(np.maximum(z, 0.0) if li + 1 < len(layers) else z)
    return acts


def round_bf16(a):
    """Round to the nearest bfloat16 (8-bit significand, FP32 exponent range), ties to even: the FP32 value's
    low 16 bits are dropped after adding half a unit of the kept part (0x7fff plus the kept part's lowest
    bit).  Inputs are first rounded to FP32; NaN and infinities are not used here."""
    f = np.ascontiguousarray(np.asarray(a, np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def forward_bf16(theta, x, channels=CHANNELS):
    """The network as its BF16 inference path defines it: weights and biases rounded to BF16, the input kept
    in FP32, every hidden activation rounded to BF16 after its ReLU, the output kept in FP32; products and
    sums exact here (FP64), which the GPU's FP32 accumulation approximates."""
    a = np.asarray(np.asarray(x, np.float32), np.float64)
    layers = unpack(np.asarray(theta, np.float64), channels)
    for li, (W, b) in enumerate(layers):
        z = conv3d(a, round_bf16(W), round_bf16(b), DILATIONS[li])
        a = round_bf16(np.maximum(z, 0.0)) if li + 1 < len(layers) else np.asarray(z.astype(np.float32), np.float64)
    return a


def loss_and_grad(theta, x, target, valid, channels=CHANNELS):
    """Masked mean-squared error and its gradient with respect to the flat parameters."""
    acts = forward(theta, x, channels)
    q = acts[-1]
    m = np.asarray(valid, np.float64)
    cnt = max(m.sum(), 1.0)
    d = (q - target) * m
    loss = float((d * d).sum() / cnt)
    g = 2.0 * d / cnt
    layers = unpack(np.asarray(theta, np.float64), channels)
    grads = [None] * len(layers)
    for li in range(len(layers) - 1, -1, -1):
        W, b = layers[li]
        gx, gW, gb = conv3d_backward(acts[li], W, g, DILATIONS[li])
        grads[li] = (gW, gb)
        if li > 0:
            g = gx * (acts[li] > 0.0)  # through the ReLU that produced acts[li]
    return loss, pack(grads)


def adam_step(theta, grad, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (bias-corrected moments); returns new (theta, m, v). step counts from 1."""
    m = b1 * m + (1.0 - b1) * grad
    v = b2 * v + (1.0 - b2) * grad * grad
    mhat = m / (1.0 - b1 ** step)
    vhat = v / (1.0 - b2 ** step)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v


def init_params(seed, channels=CHANNELS):
    """Seeded initial parameters: the shared input generator synth.netinit (the library receives them)."""
    from synth.netinit import init_params as draw
    return draw(seed, channels)


# ------------------------------------------------------------------ samples of one grain
def grain_box_origin(system, grain_of_voxel, g):
    """Minimum corner (x, y, z) of grain g's solid voxels; raises if the box exceeds 16^3."""
    sel = (np.asarray(grain_of_voxel) == g) & system.mesh.solid
    kk, jj, ii = np.nonzero(sel)
    if ii.size == 0:
        return None
    lo = np.array([ii.min(), jj.min(), kk.min()])
    hi = np.array([ii.max(), jj.max(), kk.max()])
    if np.any(hi - lo + 1 > GRID - 1):
        raise ValueError(f"grain {g}: voxel box larger than {GRID - 1}^3")
    return lo


def grain_fields(system, grain_of_voxel, g, origin):
    """Channels 0 and 1 ([2][17][17][17]) and exp(mean log E) of grain g."""
    f = np.zeros((2, GRID, GRID, GRID))
    sel = (np.asarray(grain_of_voxel) == g) & system.mesh.solid
    kk, jj, ii = np.nonzero(sel)
    x, y, z = ii - origin[0], jj - origin[1], kk - origin[2]
    f[0, z, y, x] = 1.0
    logE = np.log(system.E[kk, jj, ii])
    f[1, z, y, x] = logE
    ebar = float(np.exp(logE.mean()))
    return f, ebar


def dof_positions(system, dofs, origin):
    """(component, z, y, x) grid position of each free DOF in `dofs`."""
    full = system.free[dofs]
    node, comp = full // 3, full % 3
    ijk = system.mesh.node_ijk[node]
    return comp, ijk[:, 2] - origin[2], ijk[:, 1] - origin[1], ijk[:, 0] - origin[0]


def make_sample(fields, pos, rhs, x_true=None):
    """(input [5][17]^3, target [3][17]^3 or None, valid [3][17]^3) for one right-hand side."""
    comp, z, y, x = pos
    s = float(np.sqrt(np.mean(rhs * rhs))) if rhs.size else 0.0
    inp = np.zeros((5, GRID, GRID, GRID))
    inp[:2] = fields
    valid = np.zeros((3, GRID, GRID, GRID))
    valid[comp, z, y, x] = 1.0
    tgt = None
    if s > 0.0:
        inp[2 + comp, z, y, x] = rhs / s
    if x_true is not None:
        tgt = np.zeros((3, GRID, GRID, GRID))
        sx = float(np.sqrt(np.mean(x_true * x_true))) if x_true.size else 0.0
        if s > 0.0 and sx > 0.0:
            tgt[comp, z, y, x] = x_true / sx
    return inp, tgt, valid


def guess_from_prediction(q, pos):
    """Direction of the initial guess on the grain's DOFs (CG rescales it, see pcg)."""
    comp, z, y, x = pos
    return q[comp, z, y, x]


# ------------------------------------------------------------------ iterative basis solve
def block_jacobi_inverse(A, dofs_comp_node):
    """Inverse of the diagonal block of each node (its free components) as a sparse operator."""
    import scipy.sparse as sp
    node = dofs_comp_node
    n = A.shape[0]
    rows, cols, vals = [], [], []
    A = A.tocsr()
    for nd in np.unique(node):
        idx = np.flatnonzero(node == nd)
        Bk = A[idx][:, idx].toarray()
        Bi = np.linalg.inv(Bk)
        r, c = np.meshgrid(idx, idx, indexing="ij")
        rows.append(r.ravel())
        cols.append(c.ravel())
        vals.append(Bi.ravel())
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))


def pcg(A, b, Minv, x0=None, tol=1e-6, max_iters=5000, scale_guess=True):
    """Preconditioned conjugate gradients (Hestenes-Stiefel), stop at ||b - A x|| <= tol ||b||.
    A guess x0 is first scaled by alpha0 = (x0 . b) / (x0 . A x0), the factor that minimises the A-norm
    error along x0 (so the scaled guess is never worse than zero in that norm).
    Returns (x, iterations, initial relative residual)."""
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    if scale_guess and x0 is not None:
        xax = x @ (A @ x)
        x *= (x @ b) / xax if xax > 0.0 else 0.0
    r = b - A @ x
    bn = np.linalg.norm(b)
    if bn == 0.0:
        return np.zeros_like(b), 0, 0.0
    rel0 = np.linalg.norm(r) / bn
    z = Minv @ r
    p = z.copy()
    rz = r @ z
    it = 0
    while np.linalg.norm(r) > tol * bn and it < max_iters:
        q = A @ p
        alpha = rz / (p @ q)
        x += alpha * p
        r -= alpha * q
        z = Minv @ r
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
        it += 1
    return x, it, rel0
