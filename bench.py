#!/usr/bin/env python
"""Benchmark: set-up + FGMRES time-to-solution at relative residual 1e-8 for algebraic hPLMM on one GB300,
plain FP64 against the chosen mixed-precision form.

The default workload is the largest configuration that fits one GPU: the 256^3 fractured heterogeneous
block (porosity 0.25, two-phase Voronoi moduli 1 and 10, 20 one-voxel slits with E x 1e-4, 16^3 grains of
16^3 voxels, about 44M DOF).  Its plain FP64 form needs about 370 GB of FP64 local factors, more than the
GPU holds, so the plain FP64 comparison runs on the largest workload where it fits (128^3 porous, about
4.5M DOF) and is reported beside the headline with the chosen form timed on the same image.

One step = the whole hot path over one synthetic image: preconditioner set-up (maps, mortars, local
factorisations, basis solves, Galerkin product, sparse coarse Cholesky) and the right-preconditioned FGMRES
solve to 1e-8, with the assembled system resident in HBM.  `e2e` repeats the step through the C interface
from pinned host buffers (image upload, assembly, set-up, solve and solution download in the timed region).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl hplmm|reference] [--workload NAME]

Under torchrun each rank solves its own seeded replica (replicas only) and rank 0 prints one JSON line with
the maximum time over ranks.  `--impl reference` times the CPU oracle (there is no reference program: the
paper is the reference) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "setup+GMRES time-to-solution at rel. residual 1e-8, plain FP64 vs chosen form"
TOL = 1e-8
METHOD = dict(contact_halfwidth=2, n_st=1, restart=30, max_iters=600)

# forms: the chosen one per workload (BF16 local factors and panels where the FP32 ones would not fit,
# FP32 otherwise), the plain FP64 form, and FP64 with the same graph replay and tuner (to separate the
# precision gain from the scheduling gain)
FP32 = dict(local_prec="fp32", apply_prec="fp32", use_graph=True, autotune=True)
BF16 = dict(local_prec="fp32", apply_prec="bf16", use_graph=True, autotune=True)
PLAIN = dict(local_prec="fp64", apply_prec="fp64")
FP64_TUNED = dict(local_prec="fp64", apply_prec="fp64", use_graph=True, autotune=True)

WORKLOADS = {
    "fractured256": dict(image=[256, 256, 256], porosity=0.25, grains=[16, 16, 16], n_mortar=4, chosen=BF16,
                         plain_fits=False,
                         form_text=("BF16 local factors and basis panels (FP32 factorisation in chunks), "
                                    "element-by-element FP32 residual updates, FP32 arithmetic, FP64 sparse coarse "
                                    "Cholesky (Schur updates on tcgen05 by the Ozaki scheme) and FGMRES; Galerkin "
                                    "GEMM on tcgen05; apply replayed from a CUDA graph; smoother plans tuned at "
                                    "set-up")),
    "porous128": dict(image=[128, 128, 128], porosity=0.4, grains=[8, 8, 8], n_mortar=4, chosen=FP32,
                      plain_fits=True,
                      form_text=("FP32 local factors, basis panels and residual updates, FP64 sparse coarse "
                                 "Cholesky and FGMRES; apply replayed from a CUDA graph; smoother plans tuned")),
    "porous64": dict(image=[64, 64, 64], porosity=0.3, grains=[4, 4, 4], n_mortar=4, chosen=FP32,
                     plain_fits=True,
                     form_text="FP32 form as for porous128"),
    # the fractured256 recipe at 64^3 and 128^3 (the same 16^3-voxel grains, so the same local problem shapes,
    # 64 and 512 of them): profiling cases small enough for a full ncu capture, not bench lines
    "fractured64": dict(image=[64, 64, 64], porosity=0.25, grains=[4, 4, 4], n_mortar=2, chosen=BF16,
                        plain_fits=True, form_text="BF16 form as for fractured256"),
    "fractured128": dict(image=[128, 128, 128], porosity=0.25, grains=[8, 8, 8], n_mortar=2, chosen=BF16,
                         plain_fits=True, form_text="BF16 form as for fractured256"),
}
DEFAULT_WORKLOAD = "fractured256"
PLAIN_WORKLOAD = "porous128"   # largest workload whose plain FP64 form fits one GPU


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="hplmm", choices=["hplmm", "reference"])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP64 comparison")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-ws", action="store_true", help="skip the learned warm-start evaluation")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg")
    ap.add_argument("--quick", action="store_true",
                    help="profiling mode: time only the chosen form (no comparison, e2e or CPU legs)")
    ap.add_argument("--form", default=None, choices=["fp32", "bf16", "plain", "fp64_tuned"],
                    help="form timed by --quick runs (default: the workload's chosen form)")
    ap.add_argument("--n-mortar", type=int, default=None, help="override the workload's mortar count")
    return ap.parse_args()


FORM_BY_NAME = {"fp32": FP32, "bf16": BF16, "plain": PLAIN, "fp64_tuned": FP64_TUNED}


# ------------------------------------------------------------------ distributed plumbing
def dist_init():
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def reduce_max(x, world):
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ clocks during the timed region
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons, power = [], None, set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power) if power else None}


# ------------------------------------------------------------------ the GPU arm
def make_solver(hp, spec, form, stream, profile=False, n_mortar=None):
    # a form may override the method's defaults (the ILU(0) smoother runs n_st = 6 stages)
    return hp.Solver(n_mortar=n_mortar or spec["n_mortar"], **{**METHOD, **form}, profile=profile, stream=stream)


def run_form(hp, problem, spec, form, steps, warmup, flush, stream, profile=False, n_mortar=None, keep=False):
    """Time `steps` set-up + solve steps of one form (after `warmup` untimed ones); returns the solver (closed
    unless keep), the solution, per-step ms, the last stats, the phase profile, costs, sizes and the number of
    library kernel launches in the timed steps."""
    import torch
    s = make_solver(hp, spec, form, stream, profile, n_mortar)
    mask, E = hp.problem_to_device(problem)
    s.assemble(mask, E, problem.nu, problem.bcs)
    del mask, E
    x = torch.empty(s.n_dof, dtype=torch.float64, device="cuda")
    times, st, launches0 = [], None, None
    for it in range(warmup + steps):
        if it == warmup:
            if profile:
                s.reset_profile()
            launches0 = hp.hplmm_kernel_launches()
        flush.zero_()  # evict L2 between steps (outside the timed window)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.setup(grains=problem.grains)
        _, rc, st = s.solve(None, x, TOL)
        e1.record(stream)
        torch.cuda.synchronize()
        if rc != 0 or st.rel_res_true > TOL:
            raise RuntimeError(f"solve did not reach {TOL}: rc={rc} rel={st.rel_res_true}")
        if it >= warmup:
            times.append(e0.elapsed_time(e1))
    launches = hp.hplmm_kernel_launches() - launches0
    prof = s.profile() if profile else None
    costs, sizes = s.costs(), s.sizes()
    if not keep:
        s.close()
        s = None
    return s, x, times, st, prof, costs, sizes, launches


def time_applies(hp, s, n_dof, stream, reps=10):
    """Mean time of one preconditioner apply z = M^{-1} r (the captured graph in the chosen form) on the
    solver's last set-up, CUDA events on the library's stream, L2 state warm (the apply's own bytes are far
    larger than L2)."""
    import torch
    r = torch.randn(n_dof, dtype=torch.float64, device="cuda")
    z = torch.empty_like(r)
    for _ in range(2):
        s.apply(r, z)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        s.apply(r, z)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def apply_bytes(costs, form):
    """Algorithmic bytes of one preconditioner apply (Eq. multi_precond with one smoother stage): the two
    residual updates' SpMVs, the restriction and prolongation (basis panels read twice, interface weights
    neglected), the coarse solve (its factor read once forward, once backward), the contact-grid and grain
    solves (each factor read twice: forward and backward sweeps) with their gathered and scattered vectors,
    and the vector sums of the apply."""
    n3 = 3 * costs["n_nodes"]
    fb = {"fp64": 8, "fp32": 4, "bf16": 2}[form["apply_prec"]]      # local factors and panels
    ab = 8 if form["apply_prec"] == "fp64" else 4                    # A_hat of the residual updates
    vb = 8 if form["apply_prec"] == "fp64" else 4                    # local vectors of the smoother
    if form["apply_prec"] != "fp64" and costs.get("matrix_free_updates"):
        # element by element: the vectors (x, sub, y), the moduli and mask, the node map and coordinates
        spmv = 2 * (3 * n3 * 8 + 5 * costs["n_voxels"] + 4 * costs["n_grid"] + 12 * costs["n_nodes"] + n3)
    else:
        spmv = 2 * (costs["nnzb"] * (9 * ab + 4) + 3 * n3 * 8)
    coarse = 2 * costs["panel_elems"] * fb + costs["coarse_solve_bytes"] + 2 * n3 * 8
    local = 2 * (costs["grain_band_elems"] + costs["contact_band_elems"]) * fb
    local += (costs["grain_dofs"] + costs["contact_dofs"]) * (8 + 8 + 4 + 2 * vb)
    vec = 4 * 3 * n3 * 8
    return {"spmv": spmv, "coarse": coarse, "smoothers": local, "vectors": vec,
            "total": spmv + coarse + local + vec}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return d.get("hbm_gbs", 6800.0), d.get("sm_max_mhz", 2070.0), "measured"
    return 6800.0, 2070.0, "fallback"


# the smoother solve's device source: the device helpers at the head of local.cu (up to its first section of
# kernels) and the section that holds k_band_solve_ws.  Its recorded DRAM traffic stays valid while these are
# unchanged; host code (launch dispatch, tuner, options) does not change what a launch reads or writes.
SMOOTHER_FILE = "paper_2509_19777_gb300/csrc/local.cu"
SMOOTHER_REGIONS = ((None, "// ---------------------------------------------------------------- boxes"),
                    ("// ---------------------------------------------------------------- single-RHS smoother solves",
                     "int num_sms() {"))


def kernel_source_hash():
    txt = open(os.path.join(ROOT, SMOOTHER_FILE)).read()
    h = hashlib.sha256()
    for start, end in SMOOTHER_REGIONS:
        a = txt.index(start) if start else 0
        h.update(txt[a:txt.index(end, a)].encode())
    return h.hexdigest()[:16]


def traffic_for(workload, phase):
    """DRAM bytes per launch of the phase's kernel from the committed ncu summary, if still current."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    if not os.path.exists(path):
        return None
    try:
        d = json.load(open(path))
    except (OSError, ValueError):
        return None
    ent = d.get(f"{workload}:{phase}")
    if not ent or ent.get("kernel_source_hash") != kernel_source_hash():
        return None
    return ent.get("dram_bytes_per_launch")


def dominant_roofline(prof, costs, form, steps, workload):
    """Roofline of the dominant phase of the profiled steps: algorithmic units per launch over the mean
    launch time of the phase (CUDA events around each phase, on the library's stream)."""
    hbm, smax, src = measured_peaks()
    alu_peak = 152 * 128 * 2 * (smax * 1e6) / 1e12   # FP32 CUDA cores: 152 SMs x 128 lanes x 2 flops x clock
    fb = {"fp64": 8, "fp32": 4, "bf16": 2}[form["apply_prec"]]
    vb = 8 if form["apply_prec"] == "fp64" else 4
    cand = {ph: v for ph, v in prof.items() if v[0] > 0 and ph != "apply_graph"}
    dom = max(cand, key=lambda k: cand[k][0])
    ms, launches = cand[dom]
    per_launch_ms = ms / max(launches, 1)
    out = {"kernel_phase": dom, "ms_per_step": ms / steps, "launches_per_step": launches / steps,
           "ms_per_launch": per_launch_ms}
    if dom in ("apply_grains", "apply_contacts"):
        g = dom == "apply_grains"
        elems = costs["grain_band_elems"] if g else costs["contact_band_elems"]
        dofs = costs["grain_dofs"] if g else costs["contact_dofs"]
        per_launch = 2 * elems * fb + dofs * (8 + 8 + 4 + 2 * vb)
        out.update(bound="hbm", achieved=per_launch / (per_launch_ms * 1e-3) / 1e9, peak=hbm, unit="GB/s",
                   algorithmic_bytes_per_launch=per_launch,
                   kernel="k_band_solve_ws (" + ("grain" if g else "contact-grid") + " solves)")
    elif dom == "factor_grains":
        work = costs["grain_chol_flops"] + costs["contact_chol_flops"]
        out.update(bound="alu", achieved=work / (ms / steps * 1e-3) / 1e12, peak=alu_peak, unit="TFLOP/s",
                   kernel="k_band_chol32")
    elif dom == "basis_solve":
        out.update(bound="alu", achieved=costs["basis_solve_flops"] / (ms / steps * 1e-3) / 1e12,
                   peak=alu_peak, unit="TFLOP/s", kernel="k_band_solve_multi32")
    elif dom == "spmv":
        per_launch = costs["nnzb"] * (9 * 8 + 4) + 3 * 3 * costs["n_nodes"] * 8
        out.update(bound="hbm", achieved=per_launch / (per_launch_ms * 1e-3) / 1e9, peak=hbm, unit="GB/s",
                   kernel="k_spmv_sell")
    else:
        out.update(bound="hbm", achieved=None, peak=hbm, unit="GB/s")
    out["frac"] = (out["achieved"] / out["peak"]) if out.get("achieved") else None
    out["peak_source"] = src
    out["traffic"] = traffic_for(workload, dom)
    return out


def run_e2e(hp, problem, spec, form, steps, warmup, flush, stream, n_mortar=None):
    """The same step through the C interface from pinned host buffers, copies inside the timed region."""
    import numpy as np
    import torch
    s = make_solver(hp, spec, form, stream, n_mortar=n_mortar)
    mask_h = torch.from_numpy(np.ascontiguousarray(problem.mask.astype(np.uint8))).pin_memory()
    E_h = torch.from_numpy(np.ascontiguousarray(problem.E.astype(np.float32))).pin_memory()
    mask_d = torch.empty_like(mask_h, device="cuda")
    E_d = torch.empty_like(E_h, device="cuda")
    times = []
    x_h = None
    bcs = hp.make_bcs(problem.bcs)
    for it in range(warmup + steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        with torch.cuda.stream(stream):
            mask_d.copy_(mask_h, non_blocking=True)
            E_d.copy_(E_h, non_blocking=True)
        n = hp.hplmm_assemble(s.ctx, mask_d, E_d, problem.nu, bcs)
        s.n_dof = n
        s.setup(grains=problem.grains)
        x, rc, st = s.solve(None, None, TOL)
        if x_h is None:
            x_h = torch.empty(n, dtype=torch.float64).pin_memory()
        with torch.cuda.stream(stream):
            x_h.copy_(x, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        if rc != 0:
            raise RuntimeError("e2e solve did not converge")
        if it >= warmup:
            times.append(e0.elapsed_time(e1))
    h2d = mask_h.numel() * mask_h.element_size() + E_h.numel() * E_h.element_size()
    d2h = x_h.numel() * 8
    s.close()
    return times, h2d, d2h


def warm_start_eval(hp, stream, seed=0):
    """Learned warm start of the basis solves.  Training: the exact bases of the 16^3 cube (2x2x2 grains) and
    the 64^3 porous image (4x4x4 grains) -- the first two workloads -- with seeded initial weights and
    minibatch order drawn here and passed to the library.  Evaluation: the 64^3 corner (4x4x4 grains of 16^3
    voxels) of an unseen 192^3 image with porosity 0.35 (seed 100), whose basis problems are solved by
    block-Jacobi CG from the network's guess and from zero, next to the exact banded solve; CG iterations,
    starting residuals and basis-solve times are reported."""
    import numpy as np
    import torch
    import synth
    from synth.netinit import init_params
    from synth.voxels import _largest_component_touching_bottom
    kw = dict(METHOD, n_mortar=4, local_prec="fp32", apply_prec="fp32")
    tr = hp.Solver(**kw, keep_basis_rhs=True, stream=stream)
    n = 0
    for wl, sd in (("cube16", 0), ("porous64", 1)):
        p = synth.make_workload(wl, sd)
        mask, E = hp.problem_to_device(p)
        tr.assemble(mask, E, p.nu, p.bcs)
        tr.setup(grains=p.grains)
        n = tr.ws_collect()
    tr.ws_set_params(init_params(7 + seed))
    rng = np.random.default_rng(8 + seed)
    epochs = 3
    order = np.concatenate([rng.permutation(n) for _ in range(epochs)]).astype(np.int32)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    loss = tr.ws_train(order, 8, 1e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    theta = tr.ws_get_params()
    tr.close()
    full = synth.make_workload("porous192", 100)
    sub = _largest_component_touching_bottom(full.mask[:64, :64, :64].astype(bool))
    p = synth.Problem("porous192_corner64", sub, full.E[:64, :64, :64].copy(), full.nu, (4, 4, 4), full.bcs, 4, 100)
    out = {"train": {"images": "cube16 seed 0 and porous64 seed 1 (the first two workloads)", "samples": int(n),
                     "epochs": epochs, "steps": int(loss.size), "batch": 8, "lr": 1e-3,
                     "loss_first_10pct": float(loss[:max(1, loss.size // 10)].mean()),
                     "loss_last_10pct": float(loss[-max(1, loss.size // 10):].mean()), "seconds": t_train},
           "eval_image": "64^3 corner (4x4x4 grains) of an unseen 192^3 image, porosity 0.35, seed 100",
           "basis_tol": 1e-6}
    for mode in ("direct", "pcg", "pcg_warm"):
        s = hp.Solver(**kw, basis_solver=mode, basis_tol=1e-6, profile=True, stream=stream)
        if mode == "pcg_warm":
            s.ws_set_params(theta)
        mask, E = hp.problem_to_device(p)
        s.assemble(mask, E, p.nu, p.bcs)
        s.setup(grains=p.grains)
        s.reset_profile()
        s.setup(grains=p.grains)
        x, rc, st = s.solve(tol=TOL)
        bs = s.basis_stats()
        prof = s.profile()
        out[mode] = {"basis_ms": prof["basis_solve"][0], "cg_iters_total": bs["iters_total"],
                     "cg_iters_max": bs["iters_max"], "init_rel_res_mean": bs["init_rel_res_mean"],
                     "fallback_columns": bs["fallback_columns"], "net_ms": bs["t_net_ms"],
                     "fgmres_iters": st.iters, "rel_res_true": st.rel_res_true}
        s.close()
    c, w = out["pcg"]["cg_iters_total"], out["pcg_warm"]["cg_iters_total"]
    out["cg_iterations_saved"] = int(c - w)
    out["cg_iterations_saved_frac"] = (c - w) / c if c else None
    return out


# ------------------------------------------------------------------ the CPU oracle sample
def sample_problem(workload, seed):
    """Bounded sample of a workload for the CPU oracle: the corner of the image that holds its first 2 x 2 x 2
    grains (edge = two grain edges), with the same moduli, loads and grain size, the solid component touching
    z = 0 kept."""
    import synth
    from synth.voxels import _largest_component_touching_bottom
    p = synth.make_workload(workload, seed)
    e = 2 * (p.mask.shape[0] // p.grains[0])
    sub = _largest_component_touching_bottom(p.mask[:e, :e, :e].astype(bool))
    return synth.Problem(f"{workload}_corner{e}", sub, p.E[:e, :e, :e].copy(), p.nu, (2, 2, 2), p.bcs,
                         WORKLOADS[workload]["n_mortar"], seed), p


def oracle_samples(workload, seed, n):
    """Time the CPU oracle n times on the workload's sample: its full set-up (decomposition, mortars, exact
    local solves, Galerkin product, dense coarse Cholesky, smoother factorisations) and its GMRES(30) to 1e-8."""
    from oracle import gmres as og
    from oracle import precond
    q, full = sample_problem(workload, seed)
    out = []
    for _ in range(n):
        t0 = time.perf_counter()
        sysm, M = precond.build(q, precond.Options(n_mortar=q.n_mortar, contact_halfwidth=2))
        t1 = time.perf_counter()
        x, st = og.gmres(sysm.A, sysm.b, M.apply, tol=TOL, max_iters=METHOD["max_iters"])
        t2 = time.perf_counter()
        out.append({"setup_s": t1 - t0, "solve_s": t2 - t1, "total_s": t2 - t0, "iters": st["iters"],
                    "rel_res": st["rel_res"], "n_dof": sysm.n_dof, "grains": 8,
                    "full_grains": int(full.grains[0] * full.grains[1] * full.grains[2]),
                    "shape": list(q.mask.shape)})
    return out


def _oracle_subprocess(workload, seed, n, timeout=1800):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ("import json,sys; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench.oracle_samples(%r, %d, %d)))") % (ROOT, workload, seed, n)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=timeout)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def _oracle_concurrent(workload, seed, procs, timeout=1800):
    """The all-cores variant: `procs` single-threaded oracle processes at once, each timing the same sample;
    returns their runs and the wall time from the first start to the last finish."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ("import json,sys; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench.oracle_samples(%r, %d, 1)))") % (ROOT, workload, seed)
    t0 = time.perf_counter()
    ps = [subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True,
                           env=env) for _ in range(procs)]
    runs = []
    for pr in ps:
        out, err = pr.communicate(timeout=timeout)
        if pr.returncode != 0:
            raise RuntimeError(err[-2000:])
        runs.extend(json.loads(out.strip().splitlines()[-1]))
    return runs, time.perf_counter() - t0


def all_cores_json(runs, wall, procs):
    return {"cores": procs, "concurrent_samples": procs, "wall_s": wall,
            "per_sample_s": statistics.mean(r["total_s"] for r in runs),
            "host_time_per_sample_s": wall / procs,
            "how": (f"{procs} single-threaded oracle processes at once (one per host core), each timing the same "
                    "sample; host_time_per_sample_s = wall time / samples, the host's throughput with every "
                    "core busy (process start and imports included in the wall time)")}


def cpu_baseline_json(runs, workload, full_iters=None):
    """The measured oracle time of the sample (no extrapolation in `value`); an extrapolation to the full
    image -- set-up by the grain count, solve by the grain count and the iteration ratio -- is reported
    beside it and labelled as such."""
    v = statistics.mean(r["total_s"] for r in runs)
    r0 = runs[-1]
    scale = r0["full_grains"] / r0["grains"]
    its = (full_iters / r0["iters"]) if (full_iters and r0["iters"]) else 1.0
    ext = statistics.mean(r["setup_s"] for r in runs) * scale + statistics.mean(r["solve_s"] for r in runs) * scale * its
    return {"value": v, "unit": "s", "cores": 1, "host_cores": os.cpu_count(), "kind": "oracle",
            "sample": (f"oracle (numpy/scipy, 1 thread) set-up + GMRES(30) to 1e-8 on the {r0['shape'][0]}^3 corner "
                       f"of {workload} (2x2x2 of its {r0['full_grains']} grains, {r0['n_dof']} DOF, "
                       f"{r0['iters']} iterations), mean of {len(runs)} runs"),
            "setup_s": statistics.mean(r["setup_s"] for r in runs),
            "solve_s": statistics.mean(r["solve_s"] for r in runs),
            "extrapolated_full_image_s": ext,
            "extrapolation": (f"x{scale:.0f} grains for the set-up, x{scale:.0f} grains x {its:.2f} iterations "
                              "for the solve: an estimate, not a measurement")}


def reference_arm(args, rank, world):
    """The oracle on the workload's sample: each step is one timed oracle run (warm-up runs untimed)."""
    if rank != 0:
        return
    runs = _oracle_subprocess(args.workload, args.seed, args.warmup + args.steps)
    timed = runs[args.warmup:]
    cb = cpu_baseline_json(timed, args.workload)
    r0 = timed[-1]
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * cb["value"],
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{args.workload} sample: {r0['shape'][0]}^3 corner, 2x2x2 grains",
                       "n_dof": r0["n_dof"], "n_mortar": WORKLOADS[args.workload]["n_mortar"],
                       "contact_halfwidth": METHOD["contact_halfwidth"], "tol": TOL, "l2": "n/a (CPU)"},
            "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ main
def compare_forms(hp, np, torch, synth, spec_name, flush, stream, seed):
    """Plain FP64 against the chosen form (and FP64 with the same graph replay and tuner) on one image."""
    spec = WORKLOADS[spec_name]
    problem = synth.make_workload(spec_name, seed)
    out = {"workload": spec_name, "n_mortar": spec["n_mortar"]}
    xs = {}
    for name, form, w, k in (("plain_fp64", PLAIN, 1, 1), ("fp64_tuned", FP64_TUNED, 1, 1),
                             ("chosen", spec["chosen"], 1, 2)):
        _, x, t, st, _, _, _, _ = run_form(hp, problem, spec, form, k, w, flush, stream)
        xs[name] = x.cpu().numpy()
        out[name] = {"value": statistics.mean(t) / 1e3, "unit": "s", "iters": st.iters, "rel_res_true": st.rel_res_true,
                     "t_setup_ml": st.t_setup_ml, "t_setup_mg": st.t_setup_mg, "t_solve": st.t_solve,
                     "form": {k2: v for k2, v in form.items()}}
        del x
    ref = xs["plain_fp64"]
    for name in ("fp64_tuned", "chosen"):
        out[name]["rel_diff_vs_plain_fp64"] = float(np.linalg.norm(xs[name] - ref) / np.linalg.norm(ref))
    out["speedup_chosen_vs_plain_fp64"] = out["plain_fp64"]["value"] / out["chosen"]["value"]
    out["speedup_fp64_tuned_vs_plain_fp64"] = out["plain_fp64"]["value"] / out["fp64_tuned"]["value"]
    return out


def smoother_comparison(hp, np, synth, spec_name, flush, stream, seed):
    """The paper's smoother comparison (Section 5): hPLMM with the contact-grain smoother M_CG (n_st = 1)
    against the black-box ILU(0) base smoother (n_st = 6), same coarse space, FP64 form with graph replay."""
    spec = WORKLOADS[spec_name]
    problem = synth.make_workload(spec_name, seed)
    out = {"workload": spec_name, "n_mortar": spec["n_mortar"], "form": FP64_TUNED}
    xs = {}
    for name, over in (("contact_grain_nst1", {}), ("ilu0_nst6", dict(smoother="ilu0", n_st=6))):
        form = dict(FP64_TUNED, **over)
        _, x, t, st, prof, costs, _, launches = run_form(hp, problem, spec, form, 1, 1, flush, stream)
        xs[name] = x.cpu().numpy()
        out[name] = {"value": t[0] / 1e3, "unit": "s", "iters": st.iters, "rel_res_true": st.rel_res_true,
                     "t_setup_ml": st.t_setup_ml, "t_setup_mg": st.t_setup_mg, "t_solve": st.t_solve,
                     "ms_per_iteration": 1e3 * st.t_solve / max(1, st.iters), "gpu_launches": int(launches)}
        if over:
            out[name]["ilu_levels"] = costs["ilu_levels"]
        del x
    a, b = xs["contact_grain_nst1"], xs["ilu0_nst6"]
    out["ilu0_nst6"]["rel_diff_vs_contact_grain"] = float(np.linalg.norm(b - a) / np.linalg.norm(a))
    out["time_ratio_ilu0_over_contact_grain"] = out["ilu0_nst6"]["value"] / out["contact_grain_nst1"]["value"]
    out["iteration_ratio_ilu0_over_contact_grain"] = out["ilu0_nst6"]["iters"] / out["contact_grain_nst1"]["iters"]
    return out


def multi_load_eval(hp, torch, synth, spec_name, flush, stream, seed, k=4):
    """Load-step reuse: one set-up, then k load cases (top-face tractions in z, x, y and a combination) solved
    one at a time and all together in lockstep (hplmm_solve_multi), against k separate set-up + solve steps."""
    spec = WORKLOADS[spec_name]
    form = spec["chosen"]
    p = synth.make_workload(spec_name, seed)
    trs = [(0.0, 0.0, 1.0), (1.0, 0.0, 0.0), (0.0, 0.7, 0.0), (0.3, -0.4, 0.5)][:k]
    mask, E = hp.problem_to_device(p)
    B = []
    for t in trs:   # the right-hand sides of the load cases, assembled by the library itself
        sb = make_solver(hp, spec, form, stream)
        sb.assemble(mask, E, p.nu, synth.bcs_clamped_traction(traction=t))
        B.append(sb.b.clone())
        sb.close()
    B = torch.stack(B)
    s = make_solver(hp, spec, form, stream)
    s.assemble(mask, E, p.nu, p.bcs)

    def timed(fn):
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3, out

    s.setup(grains=p.grains)  # warm-up
    s.solve(B[0], None, TOL)
    t_setup, _ = timed(lambda: s.setup(grains=p.grains))
    singles = [timed(lambda q=q: s.solve(B[q], None, TOL)) for q in range(k)]
    s.solve_multi(B, None, TOL)  # warm-up of the multi-vector buffers
    t_multi, (_, rc, st) = timed(lambda: s.solve_multi(B, None, TOL))
    s.close()
    t_single = sum(t for t, _ in singles)
    return {"workload": spec_name, "loads": k, "form": form, "t_setup_s": t_setup,
            "t_solve_each_s": [t for t, _ in singles], "iters_each": [o[2].iters for _, o in singles],
            "t_solve_multi_s": t_multi, "iters_multi": [x.iters for x in st], "rc_multi": rc,
            "per_extra_load_s_one_at_a_time": t_single / k,
            "per_load_s_in_lockstep": t_multi / k,
            "k_separate_setup_and_solve_s": k * t_setup + t_single,
            "one_setup_and_lockstep_s": t_setup + t_multi}


def main():
    args = parse()
    rank, world, local = dist_init()
    if args.impl == "reference":
        reference_arm(args, rank, world)
        return
    import numpy as np
    import torch
    import paper_2509_19777_gb300 as hp
    import synth
    from paper_2509_19777_gb300.build import build_library
    build_library()
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")   # 256 MiB > 129 MB L2
    spec = WORKLOADS[args.workload]
    form = FORM_BY_NAME[args.form] if args.form else spec["chosen"]
    nm = args.n_mortar or spec["n_mortar"]
    problem = synth.make_workload(args.workload, args.seed + rank)
    if args.quick:
        s, _, tt, stt, _, costs, sizes, launches = run_form(hp, problem, spec, form, args.steps, args.warmup, flush,
                                                            stream, n_mortar=nm, keep=True)
        t_apply = time_applies(hp, s, sizes["n_dof"], stream)
        s.close()
        _, _, tq, _, prof, _, _, _ = run_form(hp, problem, spec, dict(form, use_graph=False), 1, 0, flush, stream,
                                              profile=True, n_mortar=nm)
        ab = apply_bytes(costs, form)
        print(json.dumps({"workload": args.workload, "n_mortar": nm, "form": form, "ms_per_step": statistics.mean(tt),
                          "iters": stt.iters, "t_setup": stt.t_setup_ml + stt.t_setup_mg, "t_solve": stt.t_solve,
                          "launches_per_step": launches / args.steps, "apply_ms": t_apply,
                          "apply_frac": ab["total"] / (t_apply * 1e-3) / 1e9 / measured_peaks()[0],
                          "apply_bytes": ab, "costs": costs, "n_coarse": sizes["n_coarse"],
                          "profile_ms_per_step": {k: v[0] for k, v in prof.items()},
                          "profile_launches": {k: v[1] for k, v in prof.items()}}), flush=True)
        return

    # the chosen form: timed steps with the clocks sampled, then one apply timed on the last set-up
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        s, xc, tc, stc, _, costs, sizes, launches = run_form(hp, problem, spec, form, args.steps, args.warmup, flush,
                                                             stream, n_mortar=nm, keep=True)
    barrier(world)
    torch.cuda.synchronize()
    ms_step = reduce_max(statistics.mean(tc), world)
    free_b, total_b = torch.cuda.mem_get_info()
    t_apply = time_applies(hp, s, sizes["n_dof"], stream)
    s.close()
    del xc
    hbm = measured_peaks()[0]
    ab = apply_bytes(costs, form)
    apply_rf = {"bound": "hbm", "achieved": ab["total"] / (t_apply * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                "frac": ab["total"] / (t_apply * 1e-3) / 1e9 / hbm, "ms_per_apply": t_apply,
                "algorithmic_bytes": ab, "peak_source": measured_peaks()[2]}
    # one profiled step (phase timers, the apply launched kernel by kernel) for the breakdown and the
    # dominant kernel's roofline
    _, _, tq, stq, prof, _, _, _ = run_form(hp, problem, spec, dict(form, use_graph=False), 1, 0, flush, stream,
                                            profile=True, n_mortar=nm)
    rf = dominant_roofline(prof, costs, form, 1, args.workload)
    clocks = clk.summary()
    line = {
        "metric": METRIC,
        "value": ms_step / 1e3,
        "unit": "s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_step,
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "bf16+f32+f64" if form["apply_prec"] == "bf16" else ("f32+f64" if form["apply_prec"] == "fp32" else "f64"),
        "data": "synthetic",
        "config": {"workload": args.workload, "image": spec["image"],
                   "porosity": spec["porosity"], "grains": spec["grains"], "n_mortar": nm,
                   "contact_halfwidth": METHOD["contact_halfwidth"], "restart": METHOD["restart"], "tol": TOL,
                   "n_dof": sizes["n_dof"], "n_coarse": sizes["n_coarse"], "n_interfaces": sizes["n_interfaces"],
                   "form": spec["form_text"], "l2": "flushed (256 MiB write) before every step",
                   "parallelism": "replicas"},
        "iters": stc.iters,
        "rel_res_true": stc.rel_res_true,
        "phases_s": {"t_setup_ml": stc.t_setup_ml, "t_setup_mg": stc.t_setup_mg, "t_solve": stc.t_solve},
        "profile_ms_per_step": {k: v[0] for k, v in prof.items()},
        "roofline": rf,
        "apply_roofline": apply_rf,
        "gpu_launches": int(launches),
        "gpu_launches_per_step": launches / max(1, args.steps),
        "clocks": clocks,
        "memory": {"device_gb_in_use_after_solve": (total_b - free_b) / 1e9, "device_gb_total": total_b / 1e9},
    }
    if not args.no_e2e:
        te2e, h2d, d2h = run_e2e(hp, problem, spec, form, args.steps, 1, flush, stream, n_mortar=nm)
        line["e2e"] = {"value": reduce_max(statistics.mean(te2e), world) / 1e3, "unit": "s",
                       "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}
    if rank == 0 and not args.no_plain:
        try:
            if spec["plain_fits"]:
                line["plain_fp64"] = compare_forms(hp, np, torch, synth, args.workload, flush, stream, args.seed)
            else:
                cmp = compare_forms(hp, np, torch, synth, PLAIN_WORKLOAD, flush, stream, args.seed)
                line["plain_fp64"] = {"value": None, "unavailable": (
                    f"the plain FP64 form of {args.workload} needs about "
                    f"{8 * (costs['grain_band_elems'] + costs['contact_band_elems']) / 1e9:.0f} GB of FP64 local "
                    "factors alone: it does not fit one GPU"), "largest_workload_where_it_fits": cmp}
            line["speedup_vs_plain_fp64"] = (line["plain_fp64"].get("speedup_chosen_vs_plain_fp64") or
                                             line["plain_fp64"]["largest_workload_where_it_fits"]
                                             ["speedup_chosen_vs_plain_fp64"])
        except Exception as e:  # reported, never required for the headline
            line["plain_fp64"] = {"error": str(e)[-300:]}
    if rank == 0 and not args.no_plain:
        try:
            line["multi_load"] = multi_load_eval(hp, torch, synth, PLAIN_WORKLOAD, flush, stream, args.seed)
        except Exception as e:
            line["multi_load"] = {"error": str(e)[-300:]}
        try:
            line["smoother_comparison"] = smoother_comparison(hp, np, synth, "porous64", flush, stream, args.seed)
        except Exception as e:
            line["smoother_comparison"] = {"error": str(e)[-300:]}
    if rank == 0 and not args.no_ws:
        try:
            line["warm_start"] = warm_start_eval(hp, stream)
        except Exception as e:
            line["warm_start"] = {"error": str(e)[-300:]}
    if rank == 0 and world == 1 and not args.no_cpu:
        try:
            runs = _oracle_subprocess(args.workload, args.seed, 2)
            line["cpu_baseline"] = cpu_baseline_json(runs[1:], args.workload, stc.iters)
            procs = os.cpu_count() or 1
            cruns, wall = _oracle_concurrent(args.workload, args.seed, procs)
            line["cpu_baseline"]["all_cores"] = all_cores_json(cruns, wall, procs)
        except Exception as e:  # the baseline is reported, never required
            line["cpu_baseline"] = {"value": None, "error": str(e)[-300:]}
    if rank == 0:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
