"""Python binding of libhplmm.so, the GB300 (sm_103a) library for algebraic
hPLMM (two-level multiscale preconditioner for Q1 voxel elasticity, used in
right-preconditioned GMRES).

This module only marshals arguments: every step of assembly, set-up, apply and
solve runs in the library's CUDA kernels.  Device arrays are torch CUDA tensors
(PyTorch is used for device memory and streams only).  There is no CPU
fallback: importing works without a GPU, but every call needs the built
library and a CUDA device, and a missing library raises at first use.

The functions below carry the C interface's names (include/hplmm.h); `Solver`
wraps one context for convenience.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhplmm.so")

HPLMM_OK = 0
HPLMM_NOT_CONVERGED = 1
HPLMM_ERR_INVALID = -1
HPLMM_ERR_OOM = -2
HPLMM_ERR_CUDA = -3
HPLMM_ERR_SINGULAR = -4
HPLMM_ERR_TIMEOUT = -5
HPLMM_ERR_STATE = -6
HPLMM_FP64, HPLMM_FP32, HPLMM_BF16 = 0, 1, 2
PREC = {"fp64": HPLMM_FP64, "fp32": HPLMM_FP32, "bf16": HPLMM_BF16}

EXPORTED = [
    "hplmm_default_options", "hplmm_create", "hplmm_assemble", "hplmm_setup", "hplmm_apply",
    "hplmm_apply_coarse", "hplmm_apply_smoother", "hplmm_spmv", "hplmm_spmv_noalloc", "hplmm_solve",
    "hplmm_get_sizes",
    "hplmm_get_maps", "hplmm_get_coarse_matrix", "hplmm_get_prolongation_column", "hplmm_get_profile",
    "hplmm_reset_profile", "hplmm_kernel_launches", "hplmm_get_costs", "hplmm_last_error", "hplmm_destroy",
    "hplmm_ws_num_params", "hplmm_ws_set_params", "hplmm_ws_get_params", "hplmm_ws_collect", "hplmm_ws_clear",
    "hplmm_ws_train", "hplmm_ws_loss_grad", "hplmm_get_basis_stats", "hplmm_ws_get_samples",
    "hplmm_inject_alloc_failure", "hplmm_apply_multi", "hplmm_solve_multi", "hplmm_ws_predict",
    "hplmm_save_setup", "hplmm_load_setup",
]
PHASES = ["maps", "factor_grains", "factor_contacts", "basis_rhs", "basis_solve", "galerkin", "coarse_chol",
          "apply_coarse", "apply_contacts", "apply_grains", "spmv", "krylov", "apply_graph", "factor_ilu",
          "apply_ilu"]


class hplmm_options(ctypes.Structure):
    _fields_ = [("n_mortar", ctypes.c_int), ("beta", ctypes.c_double), ("contact_halfwidth", ctypes.c_int),
                ("n_st", ctypes.c_int), ("local_prec", ctypes.c_int), ("apply_prec", ctypes.c_int),
                ("restart", ctypes.c_int), ("max_iters", ctypes.c_int), ("strict_two_grain", ctypes.c_int),
                ("use_graph", ctypes.c_int), ("verbose", ctypes.c_int), ("profile", ctypes.c_int),
                ("autotune", ctypes.c_int), ("basis_solver", ctypes.c_int), ("basis_tol", ctypes.c_double),
                ("basis_max_iters", ctypes.c_int), ("keep_basis_rhs", ctypes.c_int),
                ("smoother_ctas", ctypes.c_int), ("mortar_kind", ctypes.c_int), ("stage_mb", ctypes.c_int),
                ("wait_budget_us", ctypes.c_int), ("tensor_galerkin", ctypes.c_int),
                ("tensor_coarse", ctypes.c_int), ("matrix_free_updates", ctypes.c_int),
                ("smoother_bulk_warps", ctypes.c_int), ("smoother_kind", ctypes.c_int)]


HPLMM_BASIS_DIRECT, HPLMM_BASIS_PCG, HPLMM_BASIS_PCG_WARM = 0, 1, 2
BASIS = {"direct": HPLMM_BASIS_DIRECT, "pcg": HPLMM_BASIS_PCG, "pcg_warm": HPLMM_BASIS_PCG_WARM}
HPLMM_MORTAR_GAUSSIAN, HPLMM_MORTAR_ALGEBRAIC = 0, 1
MORTAR = {"gaussian": HPLMM_MORTAR_GAUSSIAN, "algebraic": HPLMM_MORTAR_ALGEBRAIC}
HPLMM_SMOOTHER_CONTACT_GRAIN, HPLMM_SMOOTHER_ILU0 = 0, 1
SMOOTHER = {"contact_grain": HPLMM_SMOOTHER_CONTACT_GRAIN, "ilu0": HPLMM_SMOOTHER_ILU0}


class hplmm_basis_stats(ctypes.Structure):
    _fields_ = [("columns", ctypes.c_longlong), ("iters_total", ctypes.c_longlong), ("iters_max", ctypes.c_longlong),
                ("fallback_columns", ctypes.c_longlong), ("fallback_grains", ctypes.c_longlong),
                ("init_rel_res_mean", ctypes.c_double), ("t_net_ms", ctypes.c_double), ("t_pcg_ms", ctypes.c_double)]


class hplmm_bcs(ctypes.Structure):
    _fields_ = [("fix", (ctypes.c_uint8 * 3) * 6), ("value", (ctypes.c_double * 3) * 6),
                ("traction", (ctypes.c_double * 3) * 6)]


class hplmm_stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("restarts", ctypes.c_int), ("rel_res_true", ctypes.c_double),
                ("t_setup_ml", ctypes.c_double), ("t_setup_mg", ctypes.c_double), ("t_solve", ctypes.c_double),
                ("n_dof", ctypes.c_longlong), ("n_coarse", ctypes.c_longlong),
                ("n_interfaces", ctypes.c_longlong), ("n_grains", ctypes.c_longlong)]


class hplmm_sizes(ctypes.Structure):
    _fields_ = [(n, ctypes.c_longlong) for n in ("n_nodes", "n_dof", "n_grains", "n_interfaces", "n_iface_nodes",
                                                   "n_mortars", "n_mortar_cols", "n_coarse")]


class hplmm_costs(ctypes.Structure):
    _fields_ = [("nnzb", ctypes.c_longlong), ("grain_band_elems", ctypes.c_longlong),
                ("contact_band_elems", ctypes.c_longlong), ("grain_chol_flops", ctypes.c_double),
                ("contact_chol_flops", ctypes.c_double), ("basis_solve_flops", ctypes.c_double),
                ("grain_dofs", ctypes.c_longlong), ("contact_dofs", ctypes.c_longlong),
                ("panel_elems", ctypes.c_longlong), ("local_elem_bytes", ctypes.c_int),
                ("n_nodes", ctypes.c_longlong), ("sell_blocks", ctypes.c_longlong),
                ("coarse_solve_bytes", ctypes.c_longlong), ("coarse_factor_flops", ctypes.c_double),
                ("coarse_fronts", ctypes.c_longlong), ("coarse_front_bytes", ctypes.c_longlong),
                ("n_voxels", ctypes.c_longlong), ("n_grid", ctypes.c_longlong), ("matrix_free_updates", ctypes.c_int),
                ("ilu_levels", ctypes.c_longlong)]


_lib = None


def load_library():
    """Load libhplmm.so (built in-tree); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing; build it with `python -m paper_2509_19777_gb300.build` "
                           "(the library has no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    P, I, D, LL = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
    sig = {
        "hplmm_default_options": (None, [ctypes.POINTER(hplmm_options)]),
        "hplmm_create": (I, [ctypes.POINTER(P), ctypes.POINTER(hplmm_options), P]),
        "hplmm_assemble": (I, [P, P, I, I, I, P, D, D, ctypes.POINTER(hplmm_bcs), P, ctypes.POINTER(LL)]),
        "hplmm_setup": (I, [P, P, I, I, I, I, P]),
        "hplmm_apply": (I, [P, P, P]),
        "hplmm_apply_coarse": (I, [P, P, P]),
        "hplmm_apply_smoother": (I, [P, P, P]),
        "hplmm_spmv": (I, [P, P, P]),
        "hplmm_spmv_noalloc": (I, [P, P, P]),
        "hplmm_solve": (I, [P, P, P, D, ctypes.POINTER(hplmm_stats)]),
        "hplmm_get_sizes": (I, [P, ctypes.POINTER(hplmm_sizes)]),
        "hplmm_get_maps": (I, [P, P, P, P, P, P, P, P, P]),
        "hplmm_get_coarse_matrix": (I, [P, P]),
        "hplmm_get_prolongation_column": (I, [P, LL, P]),
        "hplmm_get_profile": (I, [P, P, P, I]),
        "hplmm_reset_profile": (I, [P]),
        "hplmm_kernel_launches": (LL, []),
        "hplmm_inject_alloc_failure": (None, [LL]),
        "hplmm_apply_multi": (I, [P, P, P, I]),
        "hplmm_save_setup": (I, [P, ctypes.c_char_p]),
        "hplmm_load_setup": (I, [P, ctypes.c_char_p]),
        "hplmm_ws_predict": (I, [P, P, P, I]),
        "hplmm_solve_multi": (I, [P, P, P, I, D, ctypes.POINTER(hplmm_stats)]),
        "hplmm_get_costs": (I, [P, ctypes.POINTER(hplmm_costs)]),
        "hplmm_last_error": (ctypes.c_char_p, [P]),
        "hplmm_ws_num_params": (LL, []),
        "hplmm_ws_set_params": (I, [P, P, LL]),
        "hplmm_ws_get_params": (I, [P, P, LL]),
        "hplmm_ws_collect": (I, [P, ctypes.POINTER(LL)]),
        "hplmm_ws_clear": (I, [P]),
        "hplmm_ws_get_samples": (I, [P, LL, LL, P, P, P]),
        "hplmm_ws_train": (I, [P, P, LL, I, D, P]),
        "hplmm_ws_loss_grad": (I, [P, P, P, P, I, I, ctypes.POINTER(D), P]),
        "hplmm_get_basis_stats": (I, [P, ctypes.POINTER(hplmm_basis_stats)]),
        "hplmm_destroy": (None, [P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


class HplmmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"hplmm status {code}: {msg}")
        self.code = code


def _ptr(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _check(ctx, rc, allow=(HPLMM_OK,)):
    if rc not in allow:
        msg = load_library().hplmm_last_error(ctx).decode() if ctx else ""
        raise HplmmError(rc, msg)
    return rc


# ---- functions with the C interface's names -------------------------------------------------
def hplmm_default_options():
    o = hplmm_options()
    load_library().hplmm_default_options(ctypes.byref(o))
    return o


def hplmm_create(options=None, stream=None):
    """Create a context on the current CUDA device and `stream` (torch stream or raw handle)."""
    import torch
    lib = load_library()
    ctx = ctypes.c_void_p()
    if stream is None:
        stream = torch.cuda.current_stream()
    handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    rc = lib.hplmm_create(ctypes.byref(ctx), ctypes.byref(options) if options is not None else None,
                          ctypes.c_void_p(handle))
    if rc != HPLMM_OK:
        raise HplmmError(rc, "hplmm_create failed")
    return ctx


def make_bcs(bcs):
    """Face dictionary (synth.FACES order) or (fix, value, traction) arrays -> hplmm_bcs."""
    if isinstance(bcs, dict):
        from synth import bcs_dict_to_arrays
        fix, val, tra = bcs_dict_to_arrays(bcs)
    else:
        fix, val, tra = bcs
    b = hplmm_bcs()
    for f in range(6):
        for d in range(3):
            b.fix[f][d] = int(fix[f][d])
            b.value[f][d] = float(val[f][d])
            b.traction[f][d] = float(tra[f][d])
    return b


def hplmm_assemble(ctx, mask, E, nu, bcs, b_out=None, E0=1.0):
    nz, ny, nx = mask.shape
    n = ctypes.c_longlong(0)
    bc = bcs if isinstance(bcs, hplmm_bcs) else make_bcs(bcs)
    _check(ctx, load_library().hplmm_assemble(ctx, _ptr(mask), nx, ny, nz, _ptr(E), float(E0), float(nu),
                                              ctypes.byref(bc), _ptr(b_out), ctypes.byref(n)))
    return n.value


def hplmm_setup(ctx, partition=None, n_grains=0, grains=(1, 1, 1), b=None):
    px, py, pz = grains
    _check(ctx, load_library().hplmm_setup(ctx, _ptr(partition), int(n_grains), px, py, pz, _ptr(b)))


def hplmm_apply(ctx, r, z):
    _check(ctx, load_library().hplmm_apply(ctx, _ptr(r), _ptr(z)))


def hplmm_apply_coarse(ctx, r, z):
    _check(ctx, load_library().hplmm_apply_coarse(ctx, _ptr(r), _ptr(z)))


def hplmm_apply_smoother(ctx, r, z):
    _check(ctx, load_library().hplmm_apply_smoother(ctx, _ptr(r), _ptr(z)))


def hplmm_spmv(ctx, x, y):
    _check(ctx, load_library().hplmm_spmv(ctx, _ptr(x), _ptr(y)))


def hplmm_spmv_noalloc(ctx, x, y):
    """y = A_hat x using the library's static device scratch (no allocation; see include/hplmm.h)."""
    _check(ctx, load_library().hplmm_spmv_noalloc(ctx, _ptr(x), _ptr(y)))


def hplmm_solve(ctx, b, x, tol=1e-8):
    st = hplmm_stats()
    rc = load_library().hplmm_solve(ctx, _ptr(b), _ptr(x), float(tol), ctypes.byref(st))
    _check(ctx, rc, allow=(HPLMM_OK, HPLMM_NOT_CONVERGED))
    return rc, st


def hplmm_get_sizes(ctx):
    s = hplmm_sizes()
    _check(ctx, load_library().hplmm_get_sizes(ctx, ctypes.byref(s)))
    return {n: getattr(s, n) for n, _ in hplmm_sizes._fields_}


def hplmm_get_maps(ctx, device="cuda"):
    """Integer maps and mortar weights of the set-up, as numpy arrays."""
    import torch
    sz = hplmm_get_sizes(ctx)
    i32 = dict(dtype=torch.int32, device=device)
    node_ijk = torch.empty(sz["n_nodes"] * 3, **i32)
    W = torch.empty(max(sz["n_dof"], 1), dtype=torch.int64, device=device)
    pair = torch.empty(max(2 * sz["n_interfaces"], 1), **i32)
    inodes = torch.empty(max(sz["n_iface_nodes"], 1), **i32)
    ioff = torch.empty(sz["n_interfaces"] + 1, **i32)
    mnodes = torch.empty(max(sz["n_mortars"], 1), **i32)
    moff = torch.empty(sz["n_interfaces"] + 1, **i32)
    # eta block sizes follow from the offsets; allocate generously (nodes x max mortars)
    eta = torch.empty(max(sz["n_iface_nodes"] * max(1, 128), 1), dtype=torch.float64, device=device)
    _check(ctx, load_library().hplmm_get_maps(ctx, _ptr(node_ijk), _ptr(W), _ptr(pair), _ptr(inodes), _ptr(ioff),
                                              _ptr(mnodes), _ptr(moff), _ptr(eta)))
    ioff_h = ioff.cpu().numpy()
    moff_h = moff.cpu().numpy()
    n_eta = int(sum((ioff_h[c + 1] - ioff_h[c]) * (moff_h[c + 1] - moff_h[c]) for c in range(sz["n_interfaces"])))
    return {
        "node_ijk": node_ijk.cpu().numpy().reshape(-1, 3),
        "W": W.cpu().numpy()[:sz["n_dof"]],
        "iface_pair": pair.cpu().numpy()[:2 * sz["n_interfaces"]].reshape(-1, 2),
        "iface_nodes": inodes.cpu().numpy()[:sz["n_iface_nodes"]],
        "iface_offsets": ioff_h,
        "mortar_nodes": mnodes.cpu().numpy()[:sz["n_mortars"]],
        "mortar_offsets": moff_h,
        "eta": eta.cpu().numpy()[:n_eta],
        "sizes": sz,
    }


def hplmm_get_coarse_matrix(ctx, device="cuda"):
    import torch
    n = hplmm_get_sizes(ctx)["n_coarse"]
    A = torch.empty(max(n * n, 1), dtype=torch.float64, device=device)
    _check(ctx, load_library().hplmm_get_coarse_matrix(ctx, _ptr(A)))
    return A[:n * n].reshape(n, n)


def hplmm_get_prolongation_column(ctx, col, out):
    _check(ctx, load_library().hplmm_get_prolongation_column(ctx, int(col), _ptr(out)))


def hplmm_get_profile(ctx):
    """{phase: (milliseconds, kernel launches)} accumulated since the last reset."""
    n = len(PHASES)
    ms = (ctypes.c_double * n)()
    ln = (ctypes.c_longlong * n)()
    _check(ctx, load_library().hplmm_get_profile(ctx, ctypes.cast(ms, ctypes.c_void_p),
                                                 ctypes.cast(ln, ctypes.c_void_p), n))
    return {PHASES[i]: (ms[i], ln[i]) for i in range(n)}


def hplmm_reset_profile(ctx):
    _check(ctx, load_library().hplmm_reset_profile(ctx))


def hplmm_kernel_launches():
    return int(load_library().hplmm_kernel_launches())


def hplmm_inject_alloc_failure(after):
    load_library().hplmm_inject_alloc_failure(int(after))


def hplmm_ws_predict(ctx, x, out=None):
    """BF16 inference of the warm-start network on [n, 5, 17, 17, 17] float32 CUDA inputs."""
    import torch
    n = int(x.shape[0])
    if out is None:
        out = torch.empty((n, 3, 17, 17, 17), dtype=torch.float32, device=x.device)
    _check(ctx, load_library().hplmm_ws_predict(ctx, _ptr(x), _ptr(out), n))
    return out


def hplmm_save_setup(ctx, path):
    """Write the context's set-up to the file at path."""
    _check(ctx, load_library().hplmm_save_setup(ctx, os.fsencode(path)))


def hplmm_load_setup(ctx, path):
    """Read a saved set-up into a context assembled on the same system with the same set-up options."""
    _check(ctx, load_library().hplmm_load_setup(ctx, os.fsencode(path)))


def hplmm_apply_multi(ctx, R, Z):
    """Z[q] = M^{-1} R[q] for the rows q of the [k, n_dof] float64 CUDA tensors R and Z."""
    _check(ctx, load_library().hplmm_apply_multi(ctx, _ptr(R), _ptr(Z), int(R.shape[0])))
    return Z


def hplmm_solve_multi(ctx, B, X, tol=1e-8):
    """Solve A X[q] = B[q] for the rows q of [k, n_dof] float64 CUDA tensors; returns (X, rc, stats list)."""
    k = int(B.shape[0])
    st = (hplmm_stats * k)()
    rc = load_library().hplmm_solve_multi(ctx, _ptr(B), _ptr(X), k, float(tol), st)
    _check(ctx, rc, allow=(HPLMM_OK, HPLMM_NOT_CONVERGED))
    return X, rc, list(st)


def hplmm_get_costs(ctx):
    c = hplmm_costs()
    _check(ctx, load_library().hplmm_get_costs(ctx, ctypes.byref(c)))
    return {n: getattr(c, n) for n, _ in hplmm_costs._fields_}


def hplmm_ws_num_params():
    return int(load_library().hplmm_ws_num_params())


def hplmm_ws_set_params(ctx, params):
    a = np.ascontiguousarray(params, dtype=np.float32)
    _check(ctx, load_library().hplmm_ws_set_params(ctx, a.ctypes.data, a.size))


def hplmm_ws_get_params(ctx):
    a = np.empty(hplmm_ws_num_params(), dtype=np.float32)
    _check(ctx, load_library().hplmm_ws_get_params(ctx, a.ctypes.data, a.size))
    return a


def hplmm_ws_collect(ctx):
    n = ctypes.c_longlong(0)
    _check(ctx, load_library().hplmm_ws_collect(ctx, ctypes.byref(n)))
    return n.value


def hplmm_ws_clear(ctx):
    _check(ctx, load_library().hplmm_ws_clear(ctx))


def hplmm_ws_get_samples(ctx, first, count, device="cuda"):
    """(in [count][5][17^3], target [count][3][17^3], valid [count][3][17^3]) float32 tensors."""
    import torch
    D3 = 17 ** 3
    x = torch.empty((count, 5, D3), dtype=torch.float32, device=device)
    t = torch.empty((count, 3, D3), dtype=torch.float32, device=device)
    v = torch.empty((count, 3, D3), dtype=torch.float32, device=device)
    _check(ctx, load_library().hplmm_ws_get_samples(ctx, int(first), int(count), _ptr(x), _ptr(t), _ptr(v)))
    return x, t, v


def hplmm_ws_train(ctx, order, batch, lr):
    o = np.ascontiguousarray(order, dtype=np.int32)
    loss = np.zeros(max(1, o.size // batch), dtype=np.float64)
    _check(ctx, load_library().hplmm_ws_train(ctx, o.ctypes.data, o.size, int(batch), float(lr), loss.ctypes.data))
    return loss[:o.size // batch]


def hplmm_ws_loss_grad(ctx, x, target, valid, D):
    """x, target, valid: float32 CUDA tensors [n][5|3|3][D^3]; returns (loss, grad tensor)."""
    import torch
    grad = torch.empty(hplmm_ws_num_params(), dtype=torch.float32, device=x.device)
    loss = ctypes.c_double(0.0)
    _check(ctx, load_library().hplmm_ws_loss_grad(ctx, _ptr(x), _ptr(target), _ptr(valid), int(x.shape[0]), int(D),
                                                  ctypes.byref(loss), _ptr(grad)))
    return loss.value, grad


def hplmm_get_basis_stats(ctx):
    st = hplmm_basis_stats()
    _check(ctx, load_library().hplmm_get_basis_stats(ctx, ctypes.byref(st)))
    return {n: getattr(st, n) for n, _ in hplmm_basis_stats._fields_}


def hplmm_last_error(ctx):
    return load_library().hplmm_last_error(ctx).decode()


def hplmm_destroy(ctx):
    if ctx:
        load_library().hplmm_destroy(ctx)


# ---- convenience wrapper ---------------------------------------------------------------------
class Solver:
    """One library context: assemble -> setup -> apply / solve, on torch CUDA tensors."""

    def __init__(self, n_mortar=4, beta=4.0, contact_halfwidth=2, n_st=1, local_prec="fp64", apply_prec="fp64",
                 restart=30, max_iters=300, strict_two_grain=False, use_graph=False, verbose=False, profile=False,
                 autotune=False, basis_solver="direct", basis_tol=1e-6, basis_max_iters=3000, keep_basis_rhs=False,
                 smoother_ctas=0, mortar_kind="gaussian", stage_mb=0, wait_budget_us=0, tensor_galerkin=True,
                 tensor_coarse=True, matrix_free_updates=True, smoother_bulk_warps=0, smoother="contact_grain",
                 stream=None):
        o = hplmm_default_options()
        o.n_mortar, o.beta, o.contact_halfwidth, o.n_st = n_mortar, beta, contact_halfwidth, n_st
        o.local_prec, o.apply_prec = PREC[local_prec], PREC[apply_prec]
        o.restart, o.max_iters = restart, max_iters
        o.strict_two_grain, o.use_graph, o.verbose = int(strict_two_grain), int(use_graph), int(verbose)
        o.profile = int(profile)
        o.autotune = int(autotune)
        o.basis_solver, o.basis_tol, o.basis_max_iters = BASIS[basis_solver], basis_tol, basis_max_iters
        o.keep_basis_rhs = int(keep_basis_rhs)
        o.smoother_ctas = int(smoother_ctas)
        o.mortar_kind = MORTAR[mortar_kind]
        o.stage_mb = int(stage_mb)
        o.wait_budget_us = int(wait_budget_us)
        o.tensor_galerkin = int(tensor_galerkin)
        o.tensor_coarse = int(tensor_coarse)
        o.matrix_free_updates = int(matrix_free_updates)
        o.smoother_bulk_warps = int(smoother_bulk_warps)
        o.smoother_kind = SMOOTHER[smoother]
        self.options = o
        self.ctx = hplmm_create(o, stream)
        self.n_dof = 0

    def close(self):
        hplmm_destroy(self.ctx)
        self.ctx = None

    def __del__(self):
        try:
            if getattr(self, "ctx", None):
                self.close()
        except Exception:
            pass

    def assemble(self, mask, E, nu, bcs, E0=1.0):
        import torch
        self.n_dof = hplmm_assemble(self.ctx, mask, E, nu, bcs, None, E0)
        self.b = torch.empty(self.n_dof, dtype=torch.float64, device=mask.device)
        hplmm_assemble(self.ctx, mask, E, nu, bcs, self.b, E0)
        return self.n_dof

    def setup(self, grains=(1, 1, 1), partition=None, n_grains=0, b=None):
        hplmm_setup(self.ctx, partition, n_grains, grains, b)

    def apply(self, r, z=None):
        import torch
        z = torch.empty_like(r) if z is None else z
        hplmm_apply(self.ctx, r, z)
        return z

    def apply_coarse(self, r, z=None):
        import torch
        z = torch.empty_like(r) if z is None else z
        hplmm_apply_coarse(self.ctx, r, z)
        return z

    def apply_smoother(self, r, z=None):
        import torch
        z = torch.empty_like(r) if z is None else z
        hplmm_apply_smoother(self.ctx, r, z)
        return z

    def spmv(self, x, y=None):
        import torch
        y = torch.empty_like(x) if y is None else y
        hplmm_spmv(self.ctx, x, y)
        return y

    def solve(self, b=None, x=None, tol=1e-8):
        import torch
        x = torch.empty(self.n_dof, dtype=torch.float64, device="cuda") if x is None else x
        rc, st = hplmm_solve(self.ctx, b, x, tol)
        return x, rc, st

    def save_setup(self, path):
        hplmm_save_setup(self.ctx, path)

    def load_setup(self, path):
        hplmm_load_setup(self.ctx, path)

    def apply_multi(self, R, Z=None):
        import torch
        if Z is None:
            Z = torch.empty_like(R)
        return hplmm_apply_multi(self.ctx, R, Z)

    def solve_multi(self, B, X=None, tol=1e-8):
        import torch
        if X is None:
            X = torch.empty_like(B)
        return hplmm_solve_multi(self.ctx, B, X, tol)

    def sizes(self):
        return hplmm_get_sizes(self.ctx)

    def maps(self):
        return hplmm_get_maps(self.ctx)

    def coarse_matrix(self):
        return hplmm_get_coarse_matrix(self.ctx)

    def profile(self):
        return hplmm_get_profile(self.ctx)

    def reset_profile(self):
        hplmm_reset_profile(self.ctx)

    def costs(self):
        return hplmm_get_costs(self.ctx)

    def basis_stats(self):
        return hplmm_get_basis_stats(self.ctx)

    def ws_set_params(self, params):
        hplmm_ws_set_params(self.ctx, params)

    def ws_get_params(self):
        return hplmm_ws_get_params(self.ctx)

    def ws_collect(self):
        return hplmm_ws_collect(self.ctx)

    def ws_train(self, order, batch, lr):
        return hplmm_ws_train(self.ctx, order, batch, lr)

    def prolongation_column(self, col, out=None):
        import torch
        out = torch.empty(self.n_dof, dtype=torch.float64, device="cuda") if out is None else out
        hplmm_get_prolongation_column(self.ctx, col, out)
        return out


def problem_to_device(problem, device="cuda"):
    """synth.Problem -> (mask uint8, E float32) device tensors."""
    import torch
    mask = torch.from_numpy(np.ascontiguousarray(problem.mask.astype(np.uint8))).to(device)
    E = torch.from_numpy(np.ascontiguousarray(problem.E.astype(np.float32))).to(device)
    return mask, E
