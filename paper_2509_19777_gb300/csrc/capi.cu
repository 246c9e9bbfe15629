// The library's C interface (include/hplmm.h): argument checks, phase
// ordering, timing and the conversion between the public free-DOF vectors
// and the padded [n_nodes][3] layout used internally.
#include "common.cuh"

#include <atomic>
#include <chrono>
#include <cstring>

using hp::Error;

namespace hp {
static std::atomic<long long> g_launches{0};
static std::atomic<long long> g_fail_after{-1};  // allocations left before the injected failure; -1: none
bool alloc_should_fail() {
  long long v = g_fail_after.load();
  while (v >= 0) {
    if (g_fail_after.compare_exchange_weak(v, v - 1)) return v == 0;
  }
  return false;
}
long long note_launch() { return ++g_launches; }
long long launch_count() { return g_launches.load(); }
void add_launches(long long n) { g_launches += n; }

cudaEvent_t prof_event(hplmm_ctx *c) {
  if (!c->ev_pool.empty()) {
    cudaEvent_t e = c->ev_pool.back();
    c->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  HP_CUDA(cudaEventCreate(&e));
  return e;
}

void prof_harvest(hplmm_ctx *c) {
  if (c->prof_pending.empty()) return;
  HP_CUDA(cudaEventSynchronize(c->prof_pending.back().e1));
  for (auto &r : c->prof_pending) {
    float ms = 0.f;
    HP_CUDA(cudaEventElapsedTime(&ms, r.e0, r.e1));
    c->prof_ms[r.ph] += ms;
    c->prof_launches[r.ph] += r.launches;
    c->ev_pool.push_back(r.e0);
    c->ev_pool.push_back(r.e1);
  }
  c->prof_pending.clear();
}
}  // namespace hp

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

template <typename F>
hplmm_status guarded(hplmm_ctx *c, F &&f) {
  if (!c) return HPLMM_ERR_INVALID;
  try {
    f();
    return HPLMM_OK;
  } catch (const Error &e) {
    c->err = e.what();
    return e.code;
  } catch (const std::exception &e) {
    c->err = e.what();
    return HPLMM_ERR_CUDA;
  }
}

void validate_options(const hplmm_options &o) {
  HP_REQUIRE(o.n_mortar >= 1 && o.n_mortar <= 128, HPLMM_ERR_INVALID, "n_mortar must lie in [1, 128]");
  HP_REQUIRE(o.beta > 0.0, HPLMM_ERR_INVALID, "beta must be positive");
  HP_REQUIRE(o.contact_halfwidth >= 0 && o.contact_halfwidth <= 16, HPLMM_ERR_INVALID,
             "contact_halfwidth must lie in [0, 16]");
  HP_REQUIRE(o.n_st >= 1 && o.n_st <= 16, HPLMM_ERR_INVALID, "n_st must lie in [1, 16]");
  HP_REQUIRE(o.local_prec == HPLMM_FP64 || o.local_prec == HPLMM_FP32, HPLMM_ERR_INVALID,
             "local_prec must be FP64 or FP32");
  HP_REQUIRE(o.apply_prec == HPLMM_FP64 || o.apply_prec == HPLMM_FP32 || o.apply_prec == HPLMM_BF16,
             HPLMM_ERR_INVALID, "apply_prec must be FP64, FP32 or BF16");
  HP_REQUIRE(o.apply_prec != HPLMM_BF16 || o.local_prec == HPLMM_FP32, HPLMM_ERR_INVALID,
             "the BF16 apply stores BF16 copies of FP32 local factors and panels: it needs local_prec = FP32");
  HP_REQUIRE(o.restart >= 1 && o.restart <= 60, HPLMM_ERR_INVALID, "restart must lie in [1, 60]");
  HP_REQUIRE(o.max_iters >= 1, HPLMM_ERR_INVALID, "max_iters must be positive");
  HP_REQUIRE(o.use_graph == 0 || o.use_graph == 1, HPLMM_ERR_INVALID, "use_graph must be 0 or 1");
  HP_REQUIRE(o.autotune == 0 || o.autotune == 1, HPLMM_ERR_INVALID, "autotune must be 0 or 1");
  HP_REQUIRE(o.basis_solver >= HPLMM_BASIS_DIRECT && o.basis_solver <= HPLMM_BASIS_PCG_WARM, HPLMM_ERR_INVALID,
             "basis_solver must be HPLMM_BASIS_DIRECT, HPLMM_BASIS_PCG or HPLMM_BASIS_PCG_WARM");
  HP_REQUIRE(o.basis_solver == HPLMM_BASIS_DIRECT || o.local_prec == HPLMM_FP32, HPLMM_ERR_INVALID,
             "the iterative basis solves run in FP32: they need local_prec = FP32");
  HP_REQUIRE(o.basis_tol > 0.0 && o.basis_tol < 1.0, HPLMM_ERR_INVALID, "basis_tol must lie in (0, 1)");
  HP_REQUIRE(o.basis_max_iters >= 1, HPLMM_ERR_INVALID, "basis_max_iters must be positive");
  HP_REQUIRE(o.smoother_ctas >= 0 && o.smoother_ctas <= 2, HPLMM_ERR_INVALID, "smoother_ctas must be 0, 1 or 2");
  HP_REQUIRE(o.mortar_kind == HPLMM_MORTAR_GAUSSIAN || o.mortar_kind == HPLMM_MORTAR_ALGEBRAIC, HPLMM_ERR_INVALID,
             "mortar_kind must be HPLMM_MORTAR_GAUSSIAN or HPLMM_MORTAR_ALGEBRAIC");
  HP_REQUIRE(o.stage_mb >= 0, HPLMM_ERR_INVALID, "stage_mb must be non-negative");
  HP_REQUIRE(o.wait_budget_us >= 0, HPLMM_ERR_INVALID, "wait_budget_us must be non-negative");
  HP_REQUIRE(o.tensor_galerkin == 0 || o.tensor_galerkin == 1, HPLMM_ERR_INVALID, "tensor_galerkin must be 0 or 1");
  HP_REQUIRE(o.tensor_coarse == 0 || o.tensor_coarse == 1, HPLMM_ERR_INVALID, "tensor_coarse must be 0 or 1");
  HP_REQUIRE(o.matrix_free_updates == 0 || o.matrix_free_updates == 1, HPLMM_ERR_INVALID,
             "matrix_free_updates must be 0 or 1");
  HP_REQUIRE(o.smoother_bulk_warps == 0 || o.smoother_bulk_warps == 1 || o.smoother_bulk_warps == 2 ||
                 o.smoother_bulk_warps == 4 || o.smoother_bulk_warps == 8,
             HPLMM_ERR_INVALID, "smoother_bulk_warps must be 0, 1, 2, 4 or 8");
  HP_REQUIRE(o.smoother_bulk_warps == 0 || o.smoother_bulk_warps == 8 || o.smoother_ctas != 2, HPLMM_ERR_INVALID,
             "smoother_bulk_warps 1, 2 or 4 runs one CTA per local problem: it excludes smoother_ctas = 2");
  HP_REQUIRE(o.smoother_kind == HPLMM_SMOOTHER_CONTACT_GRAIN || o.smoother_kind == HPLMM_SMOOTHER_ILU0,
             HPLMM_ERR_INVALID, "smoother_kind must be HPLMM_SMOOTHER_CONTACT_GRAIN or HPLMM_SMOOTHER_ILU0");
}

void require_setup(hplmm_ctx *c) {
  HP_REQUIRE(c->assembled, HPLMM_ERR_STATE, "call hplmm_assemble first");
  HP_REQUIRE(c->setup_done, HPLMM_ERR_STATE, "call hplmm_setup first");
}

void alloc_work(hplmm_ctx *c) {
  long long L = 3LL * c->n_nodes;
  for (auto *b : {&c->w_r1, &c->w_r2, &c->w_z1, &c->w_zz, &c->w_zg, &c->w_t, &c->w_w, &c->w_in, &c->w_out})
    b->alloc(L);
  long long No = std::max<long long>(c->n_coarse, 1);
  c->w_coarse_t.alloc(No);
  c->w_coarse_u.alloc(No);
  c->w_coarse_y.alloc(No);
  c->w_x32.alloc(L);  // allocated before any graph capture reads it
  int m = c->opt.restart;
  c->V.alloc((size_t)(m + 1) * L);
  c->Z.alloc((size_t)m * L);
  c->w_h.alloc(2 * 64 + 8);
  c->w_partial.alloc(304 * 64);
  if (c->w_ticket.n == 0) {
    c->w_ticket.alloc(1);
    c->w_ticket.zero(c->stream);
  }
}

}  // namespace

extern "C" {

void hplmm_default_options(hplmm_options *o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->n_mortar = 4;
  o->beta = 4.0;
  o->contact_halfwidth = 2;
  o->n_st = 1;
  o->local_prec = HPLMM_FP64;
  o->apply_prec = HPLMM_FP64;
  o->restart = 30;
  o->max_iters = 300;
  o->strict_two_grain = 0;
  o->use_graph = 0;
  o->verbose = 0;
  o->profile = 0;
  o->autotune = 0;
  o->basis_solver = HPLMM_BASIS_DIRECT;
  o->basis_tol = 1e-6;
  o->basis_max_iters = 3000;
  o->keep_basis_rhs = 0;
  o->smoother_ctas = 0;
  o->tensor_galerkin = 1;
  o->tensor_coarse = 1;
  o->matrix_free_updates = 1;
  o->smoother_bulk_warps = 0;
  o->smoother_kind = HPLMM_SMOOTHER_CONTACT_GRAIN;
}

hplmm_status hplmm_create(hplmm_ctx **ctx, const hplmm_options *opt, void *cuda_stream) {
  if (!ctx) return HPLMM_ERR_INVALID;
  *ctx = nullptr;
  hplmm_options o;
  hplmm_default_options(&o);
  if (opt) o = *opt;
  try {
    validate_options(o);
  } catch (const Error &) {
    return HPLMM_ERR_INVALID;
  }
  hplmm_ctx *c = new (std::nothrow) hplmm_ctx();
  if (!c) return HPLMM_ERR_OOM;
  c->opt = o;
  c->stream = (cudaStream_t)cuda_stream;
  if (cudaGetDevice(&c->device) != cudaSuccess) {
    delete c;
    return HPLMM_ERR_CUDA;
  }
  *ctx = c;
  return HPLMM_OK;
}

hplmm_status hplmm_assemble(hplmm_ctx *c, const uint8_t *mask, int nx, int ny, int nz, const float *E, double E0,
                            double nu, const hplmm_bcs *bcs, double *b_out, long long *n_dof_out) {
  return guarded(c, [&] {
    hp::assemble(c, mask, nx, ny, nz, E, E0, nu, bcs, b_out);
    if (n_dof_out) *n_dof_out = c->n_dof;
  });
}

hplmm_status hplmm_setup(hplmm_ctx *c, const int32_t *partition, int n_grains, int px, int py, int pz,
                         const double *b) {
  return guarded(c, [&] {
    HP_REQUIRE(c->assembled, HPLMM_ERR_STATE, "call hplmm_assemble first");
    if (partition) {
      HP_REQUIRE(n_grains >= 1, HPLMM_ERR_INVALID, "n_grains must be positive with an explicit partition");
      c->n_grains = n_grains;
      c->px = c->py = c->pz = 0;
    } else {
      HP_REQUIRE(px >= 1 && py >= 1 && pz >= 1 && px <= c->nx && py <= c->ny && pz <= c->nz, HPLMM_ERR_INVALID,
                 "Cartesian grain counts must lie in [1, image size] per axis");
      c->px = px;
      c->py = py;
      c->pz = pz;
      c->n_grains = px * py * pz;
    }
    c->setup_done = false;
    hp::drop_apply_graph(c);
    cudaStream_t s = c->stream;
    long long L = 3LL * c->n_nodes;
    c->b_corr.alloc(L);
    if (b)
      hp::scatter_free(c, b, c->b_corr.p);
    else
      HP_CUDA(cudaMemcpyAsync(c->b_corr.p, c->b_pad.p, sizeof(double) * L, cudaMemcpyDeviceToDevice, s));
    HP_CUDA(cudaStreamSynchronize(s));
    double t0 = now_s();
    {
      hp::ProfScope ps(c, HPLMM_PH_MAPS);
      hp::build_maps(c, partition);
      hp::build_mortars(c);
      if (c->opt.mortar_kind == HPLMM_MORTAR_ALGEBRAIC) {
        hp::build_algebraic_mortars(c);
        hp::check_status(c);
      }
      hp::build_local_sets(c);
    }
    double t1 = now_s(), t2, t3;
    const bool staged = c->opt.local_prec == HPLMM_FP32 && c->opt.apply_prec == HPLMM_BF16 &&
                        c->opt.basis_solver == HPLMM_BASIS_DIRECT;
    if (staged) {
      // BF16 form: FP32 factors in chunks, each chunk of grains used for its basis solves, then kept as
      // BF16 (the local factorisations and basis solves are timed together as the smoother build)
      hp::coarse_rhs(c, c->b_corr.p);
      hp::factor_staged(c, c->X32.p, c->panel_off, c->kg, c->h_kg);
      hp::check_status(c);
      t2 = now_s();
      hp::coarse_finish(c);
    } else {
      // smoother build (T_ML): exact local factorisations of grains and contact grids
      hp::factor_local_both(c, c->opt.local_prec);
      hp::check_status(c);
      t2 = now_s();
      // coarse build (T_MG): basis solves, Galerkin product, coarse Cholesky
      hp::build_coarse(c, c->b_corr.p);
    }
    alloc_work(c);
    hp::check_status(c);
    t3 = now_s();
    // the ILU(0) smoother's factorisation, or the pipeline depths of the contact-grain smoother's solves (both
    // part of the smoother build)
    if (c->opt.smoother_kind == HPLMM_SMOOTHER_ILU0) {
      hp::ilu_setup(c);
      hp::check_status(c);
    } else {
      hp::tune_local(c);
    }
    double t4 = now_s();
    t2 += t4 - t3;
    t3 = t4;
    c->t_ml = t2 - t1;
    c->t_mg = (t1 - t0) + (t3 - t2);
    if (c->opt.verbose)
      fprintf(stderr, "[hplmm] setup: maps %.3f ms, factor %.3f ms, coarse %.3f ms; N^o=%lld, ifaces=%d\n",
              1e3 * (t1 - t0), 1e3 * (t2 - t1), 1e3 * (t3 - t2), c->n_coarse, c->n_ifaces);
    hp::prof_harvest(c);
    c->setup_done = true;
  });
}

hplmm_status hplmm_apply(hplmm_ctx *c, const double *r, double *z) {
  return guarded(c, [&] {
    require_setup(c);
    HP_REQUIRE(r && z && r != z, HPLMM_ERR_INVALID, "apply: r and z must be distinct device vectors");
    hp::scatter_free(c, r, c->w_in.p);
    hp::precond_apply_any(c, c->w_in.p, c->w_out.p);
    hp::gather_free(c, c->w_out.p, z);
  });
}

hplmm_status hplmm_apply_coarse(hplmm_ctx *c, const double *r, double *z) {
  return guarded(c, [&] {
    require_setup(c);
    HP_REQUIRE(r && z, HPLMM_ERR_INVALID, "apply_coarse: null vector");
    hp::scatter_free(c, r, c->w_in.p);
    hp::coarse_apply(c, c->w_in.p, c->w_out.p);
    hp::gather_free(c, c->w_out.p, z);
  });
}

hplmm_status hplmm_apply_smoother(hplmm_ctx *c, const double *r, double *z) {
  return guarded(c, [&] {
    require_setup(c);
    HP_REQUIRE(r && z, HPLMM_ERR_INVALID, "apply_smoother: null vector");
    hp::scatter_free(c, r, c->w_in.p);
    hp::smoother_stage(c, c->w_in.p, c->w_out.p);
    hp::gather_free(c, c->w_out.p, z);
  });
}

hplmm_status hplmm_spmv(hplmm_ctx *c, const double *x, double *y) {
  return guarded(c, [&] {
    HP_REQUIRE(c->assembled, HPLMM_ERR_STATE, "call hplmm_assemble first");
    HP_REQUIRE(x && y, HPLMM_ERR_INVALID, "spmv: null vector");
    long long L = 3LL * c->n_nodes;
    if (c->w_in.n < (size_t)L) c->w_in.alloc(L);
    if (c->w_out.n < (size_t)L) c->w_out.alloc(L);
    hp::scatter_free(c, x, c->w_in.p);
    hp::spmv(c, c->w_in.p, c->w_out.p, HPLMM_FP64);
    hp::gather_free(c, c->w_out.p, y);
  });
}

hplmm_status hplmm_solve(hplmm_ctx *c, const double *b, double *x, double tol, hplmm_stats *st) {
  hplmm_status rc = HPLMM_OK;
  hplmm_status g = guarded(c, [&] {
    require_setup(c);
    HP_REQUIRE(x, HPLMM_ERR_INVALID, "solve: x is required");
    HP_REQUIRE(tol > 0.0, HPLMM_ERR_INVALID, "solve: tol must be positive");
    const double *bp = c->b_pad.p;
    if (b) {
      hp::scatter_free(c, b, c->w_in.p);
      bp = c->w_in.p;
    }
    double t0 = now_s();
    rc = (hplmm_status)hp::fgmres(c, bp, c->w_out.p, tol, st);
    hp::gather_free(c, c->w_out.p, x);
    HP_CUDA(cudaStreamSynchronize(c->stream));
    hp::prof_harvest(c);
    double t1 = now_s();
    if (st) {
      st->t_setup_ml = c->t_ml;
      st->t_setup_mg = c->t_mg;
      st->t_solve = t1 - t0;
      st->n_dof = c->n_dof;
      st->n_coarse = c->n_coarse;
      st->n_interfaces = c->n_ifaces;
      st->n_grains = c->n_grains;
    }
  });
  return g != HPLMM_OK ? g : rc;
}

hplmm_status hplmm_save_setup(hplmm_ctx *c, const char *path) {
  return guarded(c, [&] {
    require_setup(c);
    hp::save_setup(c, path);
  });
}

hplmm_status hplmm_load_setup(hplmm_ctx *c, const char *path) {
  return guarded(c, [&] {
    HP_REQUIRE(c->assembled, HPLMM_ERR_STATE, "call hplmm_assemble first");
    hp::load_setup(c, path);
    alloc_work(c);
    // the ILU(0) factor is not stored: it is recomputed from A_hat
    if (c->opt.smoother_kind == HPLMM_SMOOTHER_ILU0) {
      hp::ilu_setup(c);
      hp::check_status(c);
    }
    c->setup_done = true;
  });
}

hplmm_status hplmm_apply_multi(hplmm_ctx *c, const double *R, double *Z, int k) {
  return guarded(c, [&] {
    require_setup(c);
    HP_REQUIRE(R && Z && R != Z, HPLMM_ERR_INVALID, "apply_multi: R and Z must be distinct device arrays");
    HP_REQUIRE(k >= 1 && k <= 64, HPLMM_ERR_INVALID, "apply_multi: k must lie in [1, 64]");
    const long long L = 3LL * c->n_nodes;
    c->mw_pin.alloc(L * k);
    c->mw_pout.alloc(L * k);
    for (int q = 0; q < k; ++q) hp::scatter_free(c, R + q * c->n_dof, c->mw_pin.p + q * L);
    hp::precond_apply_multi(c, c->mw_pin.p, c->mw_pout.p, k);
    for (int q = 0; q < k; ++q) hp::gather_free(c, c->mw_pout.p + q * L, Z + q * c->n_dof);
  });
}

hplmm_status hplmm_solve_multi(hplmm_ctx *c, const double *B, double *X, int k, double tol, hplmm_stats *st) {
  hplmm_status rc = HPLMM_OK;
  hplmm_status g = guarded(c, [&] {
    require_setup(c);
    HP_REQUIRE(B && X && B != X, HPLMM_ERR_INVALID, "solve_multi: B and X must be distinct device arrays");
    HP_REQUIRE(k >= 1 && k <= 64, HPLMM_ERR_INVALID, "solve_multi: k must lie in [1, 64]");
    HP_REQUIRE(tol > 0.0, HPLMM_ERR_INVALID, "solve_multi: tol must be positive");
    const long long L = 3LL * c->n_nodes;
    c->mw_pin.alloc(L * k);
    c->mw_pout.alloc(L * k);
    for (int q = 0; q < k; ++q) hp::scatter_free(c, B + q * c->n_dof, c->mw_pin.p + q * L);
    double t0 = now_s();
    std::vector<hplmm_stats> sv(k);
    rc = (hplmm_status)hp::fgmres_multi(c, c->mw_pin.p, c->mw_pout.p, k, tol, sv.data());
    for (int q = 0; q < k; ++q) hp::gather_free(c, c->mw_pout.p + q * L, X + q * c->n_dof);
    HP_CUDA(cudaStreamSynchronize(c->stream));
    hp::prof_harvest(c);
    double t1 = now_s();
    if (st)
      for (int q = 0; q < k; ++q) {
        st[q] = sv[q];
        st[q].t_setup_ml = c->t_ml;
        st[q].t_setup_mg = c->t_mg;
        st[q].t_solve = t1 - t0;
        st[q].n_dof = c->n_dof;
        st[q].n_coarse = c->n_coarse;
        st[q].n_interfaces = c->n_ifaces;
        st[q].n_grains = c->n_grains;
      }
  });
  return g != HPLMM_OK ? g : rc;
}

hplmm_status hplmm_get_sizes(hplmm_ctx *c, hplmm_sizes *out) {
  return guarded(c, [&] {
    HP_REQUIRE(out, HPLMM_ERR_INVALID, "get_sizes: null output");
    std::memset(out, 0, sizeof(*out));
    out->n_nodes = c->n_nodes;
    out->n_dof = c->n_dof;
    if (c->setup_done) {
      out->n_grains = c->n_grains;
      out->n_interfaces = c->n_ifaces;
      out->n_iface_nodes = c->n_iface_nodes;
      out->n_mortars = c->n_mortars;
      out->n_mortar_cols = c->n_mortar_cols;
      out->n_coarse = c->n_coarse;
    }
  });
}

hplmm_status hplmm_get_maps(hplmm_ctx *c, int32_t *node_ijk, int64_t *W, int32_t *iface_pair, int32_t *iface_nodes,
                            int32_t *iface_offsets, int32_t *mortar_nodes, int32_t *mortar_offsets, double *eta) {
  return guarded(c, [&] {
    require_setup(c);
    cudaStream_t s = c->stream;
    auto cp = [&](void *dst, const void *src, size_t bytes) {
      if (dst && bytes) HP_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, s));
    };
    cp(node_ijk, c->node_ijk.p, sizeof(int) * 3 * (size_t)c->n_nodes);
    if (W) hp::compute_W(c, W);
    cp(iface_pair, c->iface_pair.p, sizeof(int) * 2 * (size_t)c->n_ifaces);
    cp(iface_nodes, c->iface_nodes.p, sizeof(int) * (size_t)c->n_iface_nodes);
    cp(iface_offsets, c->iface_off.p, sizeof(int) * (size_t)(c->n_ifaces + 1));
    cp(mortar_nodes, c->mortar_nodes.p, sizeof(int) * (size_t)c->n_mortars);
    cp(mortar_offsets, c->mortar_off.p, sizeof(int) * (size_t)(c->n_ifaces + 1));
    if (eta && c->n_ifaces) {
      long long last = 0;
      HP_CUDA(cudaMemcpyAsync(&last, c->eta_off.p + c->n_ifaces, sizeof(long long), cudaMemcpyDeviceToHost, s));
      HP_CUDA(cudaStreamSynchronize(s));
      cp(eta, c->eta.p, sizeof(double) * (size_t)last);
    }
    HP_CUDA(cudaStreamSynchronize(s));
  });
}

hplmm_status hplmm_get_coarse_matrix(hplmm_ctx *c, double *A_o) {
  return guarded(c, [&] {
    require_setup(c);
    HP_REQUIRE(A_o, HPLMM_ERR_INVALID, "get_coarse_matrix: null output");
    HP_REQUIRE(c->dense_ao || c->n_coarse == 0, HPLMM_ERR_INVALID,
               "get_coarse_matrix: the dense A^o is kept only for N^o <= 12288 (this set-up has " +
                   std::to_string(c->n_coarse) + ")");
    size_t bytes = sizeof(double) * (size_t)c->n_coarse * (size_t)c->n_coarse;
    if (bytes) HP_CUDA(cudaMemcpyAsync(A_o, c->Ao.p, bytes, cudaMemcpyDeviceToDevice, c->stream));
    HP_CUDA(cudaStreamSynchronize(c->stream));
  });
}

hplmm_status hplmm_get_prolongation_column(hplmm_ctx *c, long long col, double *out) {
  return guarded(c, [&] {
    require_setup(c);
    HP_REQUIRE(out && col >= 0 && col < c->n_coarse, HPLMM_ERR_INVALID, "get_prolongation_column: bad column");
    hp::prolong_column(c, col, c->w_out.p);
    hp::gather_free(c, c->w_out.p, out);
    HP_CUDA(cudaStreamSynchronize(c->stream));
  });
}

hplmm_status hplmm_get_profile(hplmm_ctx *c, double *ms, long long *launches, int n) {
  return guarded(c, [&] {
    HP_REQUIRE(n >= HPLMM_PH_COUNT, HPLMM_ERR_INVALID, "get_profile: arrays must hold HPLMM_PH_COUNT entries");
    hp::prof_harvest(c);
    for (int i = 0; i < HPLMM_PH_COUNT; ++i) {
      if (ms) ms[i] = c->prof_ms[i];
      if (launches) launches[i] = c->prof_launches[i];
    }
  });
}

hplmm_status hplmm_reset_profile(hplmm_ctx *c) {
  return guarded(c, [&] {
    hp::prof_harvest(c);
    for (int i = 0; i < HPLMM_PH_COUNT; ++i) {
      c->prof_ms[i] = 0.0;
      c->prof_launches[i] = 0;
    }
  });
}

long long hplmm_kernel_launches(void) { return hp::launch_count(); }

void hplmm_inject_alloc_failure(long long after) { hp::g_fail_after.store(after < 0 ? -1 : after); }

hplmm_status hplmm_get_costs(hplmm_ctx *c, hplmm_costs *out) {
  return guarded(c, [&] {
    require_setup(c);
    HP_REQUIRE(out, HPLMM_ERR_INVALID, "get_costs: null output");
    std::memset(out, 0, sizeof(*out));
    out->nnzb = c->nnzb;
    out->local_elem_bytes = c->opt.local_prec == HPLMM_FP64 ? 8 : (c->opt.apply_prec == HPLMM_BF16 ? 2 : 4);
    auto acc = [&](const hp::LocalSet &S, long long &elems, double &flops, long long &dofs) {
      elems = S.h_band_off.empty() ? 0 : S.h_band_off.back();
      for (int k = 0; k < S.count; ++k) {
        flops += (double)S.h_n[k] * S.h_bw[k] * S.h_bw[k];
        dofs += S.h_n[k];
      }
    };
    acc(c->grains, out->grain_band_elems, out->grain_chol_flops, out->grain_dofs);
    acc(c->contacts, out->contact_band_elems, out->contact_chol_flops, out->contact_dofs);
    for (int g = 0; g < c->grains.count; ++g)
      out->basis_solve_flops += 4.0 * c->grains.h_n[g] * c->grains.h_bw[g] * c->h_kg[g];
    out->panel_elems = c->h_panel_off.empty() ? 0 : c->h_panel_off.back();
    out->n_nodes = c->n_nodes;
    out->sell_blocks = (long long)c->sell_col.n;
    out->coarse_solve_bytes = c->cf.solve_bytes;
    out->coarse_factor_flops = c->cf.flops;
    out->coarse_fronts = c->cf.nf;
    out->coarse_front_bytes = 8LL * c->cf.F_total;
    out->n_voxels = (long long)c->nx * c->ny * c->nz;
    out->n_grid = c->n_grid;
    out->matrix_free_updates = c->opt.matrix_free_updates;
    out->ilu_levels = c->opt.smoother_kind == HPLMM_SMOOTHER_ILU0 ? (long long)c->h_ilu_off.size() - 1 : 0;
  });
}

long long hplmm_ws_num_params(void) { return hp::ws_num_params(); }

hplmm_status hplmm_ws_set_params(hplmm_ctx *c, const float *params, long long n) {
  return guarded(c, [&] {
    HP_REQUIRE(params && n == hp::ws_num_params(), HPLMM_ERR_INVALID,
               "ws_set_params: expected " + std::to_string(hp::ws_num_params()) + " parameters");
    hp::ws_set_params(c, params);
  });
}

hplmm_status hplmm_ws_get_params(hplmm_ctx *c, float *params, long long n) {
  return guarded(c, [&] {
    HP_REQUIRE(params && n == hp::ws_num_params(), HPLMM_ERR_INVALID,
               "ws_get_params: expected " + std::to_string(hp::ws_num_params()) + " parameters");
    hp::ws_get_params(c, params);
  });
}

hplmm_status hplmm_ws_collect(hplmm_ctx *c, long long *n_total) {
  return guarded(c, [&] {
    long long n = hp::ws_collect(c);
    if (n_total) *n_total = n;
  });
}

hplmm_status hplmm_ws_clear(hplmm_ctx *c) {
  return guarded(c, [&] {
    c->ws.n_samples = 0;
    c->ws.cap = 0;
    c->ws.tin.release();
    c->ws.ttgt.release();
    c->ws.tvalid.release();
  });
}

hplmm_status hplmm_ws_get_samples(hplmm_ctx *c, long long first, long long count, float *in, float *target,
                                  float *valid) {
  return guarded(c, [&] {
    HP_REQUIRE(first >= 0 && count >= 0 && first + count <= c->ws.n_samples, HPLMM_ERR_INVALID,
               "ws_get_samples: range outside the training set");
    const long long D3 = 17LL * 17 * 17;
    auto cp = [&](float *dst, const float *src, long long per) {
      if (dst && count)
        HP_CUDA(cudaMemcpyAsync(dst, src + first * per, sizeof(float) * count * per, cudaMemcpyDeviceToDevice,
                                c->stream));
    };
    cp(in, c->ws.tin.p, 5 * D3);
    cp(target, c->ws.ttgt.p, 3 * D3);
    cp(valid, c->ws.tvalid.p, 3 * D3);
    HP_CUDA(cudaStreamSynchronize(c->stream));
  });
}

hplmm_status hplmm_ws_train(hplmm_ctx *c, const int32_t *order, long long n_order, int batch, double lr,
                            double *loss) {
  return guarded(c, [&] {
    HP_REQUIRE(order && n_order >= 1 && lr > 0.0, HPLMM_ERR_INVALID, "ws_train: bad order or learning rate");
    hp::ws_train(c, order, n_order, batch, lr, loss);
  });
}

hplmm_status hplmm_ws_loss_grad(hplmm_ctx *c, const float *in, const float *target, const float *valid, int n,
                                int D, double *loss, float *grad) {
  return guarded(c, [&] {
    HP_REQUIRE(in && target && valid && grad && loss, HPLMM_ERR_INVALID, "ws_loss_grad: null argument");
    HP_REQUIRE(n >= 1 && n <= 256 && D >= 3 && D <= 17, HPLMM_ERR_INVALID, "ws_loss_grad: need 1 <= n <= 256, 3 <= D <= 17");
    HP_REQUIRE(c->ws.has_params, HPLMM_ERR_STATE, "ws_loss_grad: set the network parameters first");
    *loss = hp::ws_loss_grad(c, c->ws.theta.p, in, target, valid, n, D, grad);
  });
}

hplmm_status hplmm_ws_predict(hplmm_ctx *c, const float *in, float *out, int n) {
  return guarded(c, [&] {
    HP_REQUIRE(in && out && n >= 1 && n <= 4096, HPLMM_ERR_INVALID, "ws_predict: need inputs, outputs and 1 <= n <= 4096");
    HP_REQUIRE(c->ws.has_params, HPLMM_ERR_STATE, "ws_predict: set the network parameters first");
    hp::ws_infer(c, in, n, out);
    HP_CUDA(cudaStreamSynchronize(c->stream));
  });
}

hplmm_status hplmm_get_basis_stats(hplmm_ctx *c, hplmm_basis_stats *out) {
  return guarded(c, [&] {
    HP_REQUIRE(out, HPLMM_ERR_INVALID, "get_basis_stats: null output");
    *out = c->bstats;
  });
}

const char *hplmm_last_error(const hplmm_ctx *c) {
  if (!c) return "null context";
  return c->err.c_str();
}

void hplmm_destroy(hplmm_ctx *c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  if (c->apply_graph) cudaGraphExecDestroy(c->apply_graph);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->aux_stream) cudaStreamDestroy(c->aux_stream);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  for (auto &r : c->prof_pending) {
    cudaEventDestroy(r.e0);
    cudaEventDestroy(r.e1);
  }
  for (auto e : c->ev_pool) cudaEventDestroy(e);
  delete c;
}

}  // extern "C"
