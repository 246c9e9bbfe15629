// Preconditioner application and the outer Krylov solver.
//
// Eq. multi_precond: M^{-1} r = z1 + M_L^{-1}(r - A_hat z1), z1 = M_G^{-1} r.
// Eq. local_smoother: n_st stages of the base smoother on the running residual.
// Eq. local_smoother_CG: M_CG^{-1} r = z_zeta + M_g^{-1}(r - A_hat z_zeta),
//   z_zeta = M_zeta^{-1} r (contact grids, overlapping: atomic adds);
//   M_g^{-1} on disjoint grain interiors.
// Section 5: right-preconditioned GMRES.  Because the mixed-precision apply is
// not exactly linear, the flexible variant (FGMRES, storing Z_j = M^{-1} v_j) is
// used; classical Gram-Schmidt with one re-orthogonalisation (CGS2) keeps the
// Arnoldi basis orthogonal in FP64 with three passes over the basis per step
// (h1 = V^T w; w -= V h1 fused with h2 = V^T w; w -= V h2 fused with |w|^2),
// each reduced to its result inside the same launch.
#include "common.cuh"

#include <chrono>
#include <cmath>

namespace hp {
namespace {

__global__ void k_axpby(double *y, const double *x, double a, double b, long long n) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = a * x[i] + b * y[i];
}

__global__ void k_add2(double *z, const double *a, const double *b, long long n) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) z[i] = a[i] + b[i];
}

__global__ void k_scale_copy(double *y, const double *x, double a, long long n) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = a * x[i];
}

constexpr int MDOT_BLOCKS = 304;
constexpr int MAXV = 64;

// Block reduction of acc[0..nv) into partial[block][.], then the last block to finish (a ticket on
// *counter) sums the partials of all blocks into out[0..nv) in a fixed order (deterministic) and resets the
// ticket: thread (group g, lane j) sums blocks g, g+8, ... of output j, then the 8 groups are added in order.
template <int CAP>
__device__ void reduce_blocks(double (&acc)[CAP], int nv, double *partial, double *out, unsigned *counter) {
  __shared__ double red[8][CAP > 32 ? CAP : 32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < CAP; ++j) {
    if (j < nv) {
      double s = acc[j];
      for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      if (lane == 0) red[wid][j] = s;
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < nv; j += blockDim.x) {
    double s = 0.0;
    for (int w2 = 0; w2 < 8; ++w2) s += red[w2][j];
    partial[(long long)blockIdx.x * MAXV + j] = s;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(counter, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  for (int j0 = 0; j0 < nv; j0 += 32) {
    const int j = j0 + lane;
    double s = 0.0;
    if (j < nv) {
#pragma unroll 8
      for (int b = wid; b < (int)gridDim.x; b += 8) s += __ldcg(&partial[(long long)b * MAXV + j]);
    }
    red[wid][lane] = s;
    __syncthreads();
    if (threadIdx.x < 32 && j < nv) {
      double t = 0.0;
      for (int g = 0; g < 8; ++g) t += red[g][threadIdx.x];
      out[j] = t;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *counter = 0u;
}

// out[j] = V_j . w for j < nv <= CAP (accumulators in registers), U elements per thread per pass.  The
// grid-stride loop is software-pipelined: the next pass's CAP x U loads are issued before this pass's
// multiply-adds, which do not depend on them, so a thread always has a full pass of loads in flight.  The
// loads are branch-free: slots j >= nv read vector nv-1 again (the same addresses, served by L1) and their
// sums are discarded; elements past n are clamped to n-1 with a zero weight.
template <int CAP, int U>
__global__ void __launch_bounds__(256) k_cgs_dot(const double *V, long long ldv, int nv, const double *w, long long n,
                                                 double *partial, double *out, unsigned *counter) {
  double acc[CAP];
#pragma unroll
  for (int j = 0; j < CAP; ++j) acc[j] = 0.0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  auto load = [&](long long i0, double (&v)[U][CAP], double (&wv)[U]) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const long long i = i0 + u * stride;
      const long long ii = i < n ? i : n - 1;
      wv[u] = i < n ? w[ii] : 0.0;
#pragma unroll
      for (int j = 0; j < CAP; ++j) v[u][j] = V[(long long)min(j, nv - 1) * ldv + ii];
    }
  };
  long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double v[U][CAP], wv[U];
  load(i0, v, wv);
  for (; i0 < n; i0 += U * stride) {
    double vn[U][CAP], wn[U];
    load(i0 + U * stride, vn, wn);
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int j = 0; j < CAP; ++j) acc[j] += v[u][j] * wv[u];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      wv[u] = wn[u];
#pragma unroll
      for (int j = 0; j < CAP; ++j) v[u][j] = vn[u][j];
    }
  }
  reduce_blocks<CAP>(acc, nv, partial, out, counter);
}

// w <- w - V h over j < nv <= CAP, and in the same pass either out[j] = V_j . w_new (mode 0, the next CGS
// pass) or out[0] = w_new . w_new (mode 1)
template <int CAP, int U>
__global__ void __launch_bounds__(256) k_cgs_update(const double *V, long long ldv, int nv, const double *h, double *w,
                                                    long long n, int mode, double *partial, double *out,
                                                    unsigned *counter) {
  __shared__ double hs[CAP];
  for (int j = threadIdx.x; j < CAP; j += blockDim.x) hs[j] = j < nv ? h[j] : 0.0;
  __syncthreads();
  double acc[CAP];
#pragma unroll
  for (int j = 0; j < CAP; ++j) acc[j] = 0.0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += U * stride) {
    double v[U][CAP];  // slots j >= nv repeat vector nv-1 (finite) and meet hs[j] = 0
    double wv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const long long i = min(i0 + u * stride, n - 1);
      wv[u] = w[i];
#pragma unroll
      for (int j = 0; j < CAP; ++j) v[u][j] = V[(long long)min(j, nv - 1) * ldv + i];
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const long long i = i0 + u * stride;
      double s = wv[u];
#pragma unroll
      for (int j = 0; j < CAP; ++j) s -= v[u][j] * hs[j];
      if (i < n) {
        w[i] = s;
        if (mode == 0) {
#pragma unroll
          for (int j = 0; j < CAP; ++j) acc[j] += v[u][j] * s;
        } else {
          acc[0] += s * s;
        }
      }
    }
  }
  reduce_blocks<CAP>(acc, mode == 0 ? nv : 1, partial, out, counter);
}

// w -= sum_j V_j h[j] (any nv <= MAXV; the fused kernels cover nv <= 32)
__global__ void k_mupdate(double *w, const double *V, long long ldv, int nv, const double *h, long long n) {
  __shared__ double hs[MAXV];
  for (int j = threadIdx.x; j < nv; j += blockDim.x) hs[j] = h[j];
  __syncthreads();
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double s = w[i];
    for (int j = 0; j < nv; ++j) s -= V[j * ldv + i] * hs[j];
    w[i] = s;
  }
}

// x += sum_j Z_j y[j]
__global__ void k_mcombine(double *x, const double *Z, long long ldz, int nv, const double *y, long long n) {
  __shared__ double ys[MAXV];
  for (int j = threadIdx.x; j < nv; j += blockDim.x) ys[j] = y[j];
  __syncthreads();
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double s = x[i];
    for (int j = 0; j < nv; ++j) s += Z[j * ldz + i] * ys[j];
    x[i] = s;
  }
}

// Register-block shapes of the fused Gram-Schmidt kernels: capacity CAP (the smallest listed one >= nv is
// taken; the CAP - nv padded slots still cost an FP64 multiply-add per element, and the FP64 pipe is what
// bounds these kernels, so the capacities step by 2) and U elements per thread per pass, so that about
// CAP x U loads are in flight.
template <int C, int U>
struct CgsShape {
  static constexpr int cap = C, u = U;
};
template <typename F, typename S0, typename... Ss>
bool pick_cgs_shape(int nv, F &&f) {
  if (nv <= S0::cap) {
    f(S0{});
    return true;
  }
  if constexpr (sizeof...(Ss) > 0)
    return pick_cgs_shape<F, Ss...>(nv, static_cast<F &&>(f));
  else
    return false;
}
template <typename F>
bool for_cgs_shape(int nv, F &&f) {
  return pick_cgs_shape<F, CgsShape<1, 8>, CgsShape<2, 8>, CgsShape<3, 8>, CgsShape<4, 8>, CgsShape<6, 4>,
                        CgsShape<8, 4>, CgsShape<10, 2>, CgsShape<12, 2>, CgsShape<14, 2>, CgsShape<16, 2>,
                        CgsShape<18, 1>, CgsShape<20, 1>, CgsShape<22, 1>, CgsShape<24, 1>, CgsShape<26, 1>,
                        CgsShape<28, 1>, CgsShape<30, 1>, CgsShape<32, 1>>(nv, static_cast<F &&>(f));
}

// out[j] = V_j . w, j < nv (one launch)
void mdot(hplmm_ctx *c, const double *V, long long ldv, int nv, const double *w, long long n, double *out) {
  ProfScope ps(c, HPLMM_PH_KRYLOV);
  double *pp = c->w_partial.p;
  unsigned *ct = c->w_ticket.p;
  auto go = [&](auto kern) { kern<<<MDOT_BLOCKS, 256, 0, c->stream>>>(V, ldv, nv, w, n, pp, out, ct); };
  if (!for_cgs_shape(nv, [&](auto sh) { go(k_cgs_dot<decltype(sh)::cap, decltype(sh)::u>); }))
    go(k_cgs_dot<64, 1>);
  HP_CHECK_LAUNCH();
}

// w -= V h; then out = V^T w (mode 0) or out[0] = w . w (mode 1)
void cgs_update(hplmm_ctx *c, const double *V, long long ldv, int nv, const double *h, double *w, long long n, int mode,
                double *out) {
  ProfScope ps(c, HPLMM_PH_KRYLOV);
  double *pp = c->w_partial.p;
  unsigned *ct = c->w_ticket.p;
  auto go = [&](auto kern) { kern<<<MDOT_BLOCKS, 256, 0, c->stream>>>(V, ldv, nv, h, w, n, mode, pp, out, ct); };
  if (for_cgs_shape(nv, [&](auto sh) { go(k_cgs_update<decltype(sh)::cap, decltype(sh)::u>); })) {
    HP_CHECK_LAUNCH();
    return;
  }
  k_mupdate<<<MDOT_BLOCKS, 256, 0, c->stream>>>(w, V, ldv, nv, h, n);
  HP_CHECK_LAUNCH();
  if (mode == 0)
    mdot(c, V, ldv, nv, w, n, out);
  else
    mdot(c, w, 0, 1, w, n, out);
}

}  // namespace

void check_status(hplmm_ctx *c) {
  int w[4] = {0, 0, 0, 0};
  HP_CUDA(cudaMemcpyAsync(w, c->status.p, sizeof(w), cudaMemcpyDeviceToHost, c->stream));
  HP_CUDA(cudaStreamSynchronize(c->stream));
  int st = w[0];
  if (st != 0) {
    hplmm_status code = (hplmm_status)st;
    if (code == HPLMM_ERR_SINGULAR && w[1] == 5)
      throw Error(code, "zero or non-finite pivot in the ILU(0) factorisation (node " + std::to_string(w[2]) +
                            ", component " + std::to_string(w[3]) + ")");
    if (code == HPLMM_ERR_SINGULAR) {
      static const char *where[] = {"?", "grain-grid", "contact-grid", "coarse"};
      throw Error(code, std::string("non-positive pivot in the ") + where[(w[1] >= 1 && w[1] <= 3) ? w[1] : 0] +
                            " Cholesky factorisation (problem " + std::to_string(w[2]) + ", row " +
                            std::to_string(w[3]) + "): the matrix is singular or not positive definite");
    }
    if (code == HPLMM_ERR_TIMEOUT) throw Error(code, "a device-side wait ran out of its budget");
    if (code == HPLMM_ERR_INVALID && w[1] == 4)
      throw Error(code, "coarse factor: coarse column " + std::to_string(w[3]) + " is missing from front " +
                            std::to_string(w[2]) + " (inconsistent symbolic analysis)");
    throw Error(HPLMM_ERR_CUDA, "device error word " + std::to_string(st));
  }
}

void smoother_stage(hplmm_ctx *c, const double *r_pad, double *z_pad) {
  if (c->opt.smoother_kind == HPLMM_SMOOTHER_ILU0) {
    ilu_stage(c, r_pad, z_pad);
    return;
  }
  cudaStream_t s = c->stream;
  long long L = 3LL * c->n_nodes;
  // z_zeta = M_zeta^{-1} r
  HP_CUDA(cudaMemsetAsync(c->w_zz.p, 0, sizeof(double) * L, s));
  smoother_apply(c, c->contacts, r_pad, c->w_zz.p, true);
  // r2 = r - A z_zeta
  spmv(c, c->w_zz.p, c->w_r2.p, c->opt.apply_prec, r_pad);
  // z_g = M_g^{-1} r2 (disjoint grain interiors)
  HP_CUDA(cudaMemsetAsync(c->w_zg.p, 0, sizeof(double) * L, s));
  smoother_apply(c, c->grains, c->w_r2.p, c->w_zg.p, false);
  k_add2<<<grid_for(L, 256), 256, 0, s>>>(z_pad, c->w_zz.p, c->w_zg.p, L);
  HP_CHECK_LAUNCH();
}

void precond_apply(hplmm_ctx *c, const double *r_pad, double *z_pad) {
  cudaStream_t s = c->stream;
  long long L = 3LL * c->n_nodes;
  // z1 = M_G^{-1} r
  coarse_apply(c, r_pad, c->w_z1.p);
  // r1 = r - A z1
  spmv(c, c->w_z1.p, c->w_r1.p, c->opt.apply_prec, r_pad);
  // n_st stages of M_CG on the running residual
  HP_CUDA(cudaMemcpyAsync(z_pad, c->w_z1.p, sizeof(double) * L, cudaMemcpyDeviceToDevice, s));
  for (int st = 0; st < c->opt.n_st; ++st) {
    smoother_stage(c, c->w_r1.p, c->w_t.p);
    k_axpby<<<grid_for(L, 256), 256, 0, s>>>(z_pad, c->w_t.p, 1.0, 1.0, L);
    HP_CHECK_LAUNCH();
    if (st + 1 < c->opt.n_st) {
      // res <- res - A t
      spmv(c, c->w_t.p, c->w_r2.p, c->opt.apply_prec, c->w_r1.p);
      HP_CUDA(cudaMemcpyAsync(c->w_r1.p, c->w_r2.p, sizeof(double) * L, cudaMemcpyDeviceToDevice, s));
    }
  }
}

// M^{-1} for k vectors at stride L (Eq. multi_precond with n_st stages of M_CG): the multi-right-hand-side
// forms of the coarse correction, the SpMVs and the smoother solves read each matrix, panel and factor once
// per group of vectors instead of once per vector
void precond_apply_multi(hplmm_ctx *c, const double *R, double *Z, int k) {
  cudaStream_t s = c->stream;
  const long long L = 3LL * c->n_nodes, LK = L * k;
  if (c->opt.smoother_kind == HPLMM_SMOOTHER_ILU0) {
    // the level-scheduled ILU(0) solves have no multi-vector form: one vector at a time
    for (int v = 0; v < k; ++v) precond_apply(c, R + v * L, Z + v * L);
    return;
  }
  for (auto *b : {&c->mw_r1, &c->mw_r2, &c->mw_z1, &c->mw_zz, &c->mw_zg, &c->mw_t}) b->alloc(LK);
  coarse_apply_multi(c, R, c->mw_z1.p, k);
  spmv_multi(c, c->mw_z1.p, c->mw_r1.p, k, c->opt.apply_prec, R);
  HP_CUDA(cudaMemcpyAsync(Z, c->mw_z1.p, sizeof(double) * LK, cudaMemcpyDeviceToDevice, s));
  for (int st = 0; st < c->opt.n_st; ++st) {
    HP_CUDA(cudaMemsetAsync(c->mw_zz.p, 0, sizeof(double) * LK, s));
    smoother_apply_multi(c, c->contacts, c->mw_r1.p, c->mw_zz.p, k, true);
    spmv_multi(c, c->mw_zz.p, c->mw_r2.p, k, c->opt.apply_prec, c->mw_r1.p);
    HP_CUDA(cudaMemsetAsync(c->mw_zg.p, 0, sizeof(double) * LK, s));
    smoother_apply_multi(c, c->grains, c->mw_r2.p, c->mw_zg.p, k, false);
    k_add2<<<grid_for(LK, 256), 256, 0, s>>>(c->mw_t.p, c->mw_zz.p, c->mw_zg.p, LK);
    HP_CHECK_LAUNCH();
    k_axpby<<<grid_for(LK, 256), 256, 0, s>>>(Z, c->mw_t.p, 1.0, 1.0, LK);
    HP_CHECK_LAUNCH();
    if (st + 1 < c->opt.n_st) {
      spmv_multi(c, c->mw_t.p, c->mw_r2.p, k, c->opt.apply_prec, c->mw_r1.p);
      HP_CUDA(cudaMemcpyAsync(c->mw_r1.p, c->mw_r2.p, sizeof(double) * LK, cudaMemcpyDeviceToDevice, s));
    }
  }
}

void drop_apply_graph(hplmm_ctx *c) {
  if (c->apply_graph) {
    cudaStreamSynchronize(c->stream);
    cudaGraphExecDestroy(c->apply_graph);
    c->apply_graph = nullptr;
  }
  c->graph_kernels = 0;
}

// One apply replayed from a CUDA graph: the launches of precond_apply are captured once (on a private
// stream, reading the fixed work vector w_gin and writing w_gout) and the executable graph is launched on
// the context's stream for every apply, with the input and output copied in and out.
static void build_apply_graph(hplmm_ctx *c) {
  const long long L = 3LL * c->n_nodes;
  if (!c->cap_stream) HP_CUDA(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
  c->w_gin.alloc(L);
  c->w_gout.alloc(L);
  HP_CUDA(cudaStreamSynchronize(c->stream));
  cudaStream_t user = c->stream;
  const long long l0 = launch_count();
  cudaGraph_t g = nullptr;
  c->stream = c->cap_stream;
  c->capturing = true;
  cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    try {
      precond_apply(c, c->w_gin.p, c->w_gout.p);
    } catch (...) {
      cudaStreamEndCapture(c->cap_stream, &g);
      if (g) cudaGraphDestroy(g);
      c->stream = user;
      c->capturing = false;
      throw;
    }
    e = cudaStreamEndCapture(c->cap_stream, &g);
  }
  c->stream = user;
  c->capturing = false;
  HP_CUDA(e);
  const long long captured = launch_count() - l0;
  add_launches(-captured);  // recorded, not launched
  cudaError_t e2 = cudaGraphInstantiate(&c->apply_graph, g, 0);
  cudaGraphDestroy(g);
  HP_CUDA(e2);
  c->graph_kernels = captured;
}

void precond_apply_any(hplmm_ctx *c, const double *r_pad, double *z_pad) {
  if (!c->opt.use_graph) {
    precond_apply(c, r_pad, z_pad);
    return;
  }
  if (!c->apply_graph) build_apply_graph(c);
  const long long L = 3LL * c->n_nodes;
  ProfScope ps(c, HPLMM_PH_APPLY_GRAPH);
  HP_CUDA(cudaMemcpyAsync(c->w_gin.p, r_pad, sizeof(double) * L, cudaMemcpyDeviceToDevice, c->stream));
  HP_CUDA(cudaGraphLaunch(c->apply_graph, c->stream));
  add_launches(c->graph_kernels);
  HP_CUDA(cudaMemcpyAsync(z_pad, c->w_gout.p, sizeof(double) * L, cudaMemcpyDeviceToDevice, c->stream));
}

int fgmres(hplmm_ctx *c, const double *b_pad, double *x_pad, double tol, hplmm_stats *st) {
  cudaStream_t s = c->stream;
  long long L = 3LL * c->n_nodes;
  int m = c->opt.restart;
  int maxit = c->opt.max_iters;
  double *V = c->V.p, *Z = c->Z.p;
  double *w = c->w_w.p;
  double *dev_h = c->w_h.p;  // [0..m]: h1, [MAXV..]: h2, [2*MAXV]: norm^2
  std::vector<double> H((size_t)(m + 1) * m, 0.0), cs(m, 0.0), sn(m, 0.0), gv(m + 1, 0.0), y(m, 0.0);
  std::vector<double> hh(2 * MAXV + 1, 0.0);
  HP_CUDA(cudaMemsetAsync(x_pad, 0, sizeof(double) * L, s));
  mdot(c, b_pad, 0, 1, b_pad, L, dev_h);
  HP_CUDA(cudaMemcpyAsync(hh.data(), dev_h, sizeof(double), cudaMemcpyDeviceToHost, s));
  HP_CUDA(cudaStreamSynchronize(s));
  double bnorm = std::sqrt(hh[0]);
  HP_REQUIRE(std::isfinite(bnorm), HPLMM_ERR_INVALID, "solve: the right-hand side has non-finite entries");
  int its = 0, restarts = 0;
  double rel = 0.0;
  if (bnorm == 0.0) {
    if (st) {
      st->iters = 0;
      st->restarts = 0;
      st->rel_res_true = 0.0;
    }
    return HPLMM_OK;
  }
  for (;;) {
    // r = b - A x (true residual, FP64)
    spmv(c, x_pad, V, HPLMM_FP64, b_pad);
    mdot(c, V, 0, 1, V, L, dev_h);
    HP_CUDA(cudaMemcpyAsync(hh.data(), dev_h, sizeof(double), cudaMemcpyDeviceToHost, s));
    HP_CUDA(cudaStreamSynchronize(s));
    double beta = std::sqrt(hh[0]);
    rel = beta / bnorm;
    if (c->opt.verbose) fprintf(stderr, "[hplmm] fgmres cycle %d: its=%d true rel=%.3e\n", restarts, its, rel);
    if (rel <= tol || its >= maxit) break;
    k_scale_copy<<<grid_for(L, 256), 256, 0, s>>>(V, V, 1.0 / beta, L);
    HP_CHECK_LAUNCH();
    std::fill(gv.begin(), gv.end(), 0.0);
    gv[0] = beta;
    int k = 0;
    for (int j = 0; j < m; ++j) {
      double *vj = V + (long long)j * L;
      double *zj = Z + (long long)j * L;
      precond_apply_any(c, vj, zj);
      spmv(c, zj, w, HPLMM_FP64);
      ++its;
      // CGS2 in three passes over the basis: h1 = V^T w; w -= V h1 with h2 = V^T w; w -= V h2 with |w|^2
      mdot(c, V, L, j + 1, w, L, dev_h);
      cgs_update(c, V, L, j + 1, dev_h, w, L, 0, dev_h + MAXV);
      cgs_update(c, V, L, j + 1, dev_h + MAXV, w, L, 1, dev_h + 2 * MAXV);
      HP_CUDA(cudaMemcpyAsync(hh.data(), dev_h, sizeof(double) * (2 * MAXV + 1), cudaMemcpyDeviceToHost, s));
      HP_CUDA(cudaStreamSynchronize(s));
      for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = hh[i] + hh[MAXV + i];
      double hn = std::sqrt(std::max(hh[2 * MAXV], 0.0));
      H[(size_t)(j + 1) * m + j] = hn;
      for (int i = 0; i < j; ++i) {
        double a = H[(size_t)i * m + j], bb = H[(size_t)(i + 1) * m + j];
        H[(size_t)i * m + j] = cs[i] * a + sn[i] * bb;
        H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * bb;
      }
      double a = H[(size_t)j * m + j], bb = H[(size_t)(j + 1) * m + j];
      double den = std::hypot(a, bb);
      cs[j] = a / den;
      sn[j] = bb / den;
      H[(size_t)j * m + j] = den;
      H[(size_t)(j + 1) * m + j] = 0.0;
      gv[j + 1] = -sn[j] * gv[j];
      gv[j] = cs[j] * gv[j];
      k = j + 1;
      double est = std::fabs(gv[j + 1]) / bnorm;
      if (c->opt.verbose) fprintf(stderr, "[hplmm]   it %d est %.3e\n", its, est);
      if (hn > 0.0 && j + 1 < m + 1) {
        k_scale_copy<<<grid_for(L, 256), 256, 0, s>>>(V + (long long)(j + 1) * L, w, 1.0 / hn, L);
        HP_CHECK_LAUNCH();
      }
      if (est <= tol || hn == 0.0 || its >= maxit) break;
    }
    for (int i = k - 1; i >= 0; --i) {
      double t = gv[i];
      for (int q = i + 1; q < k; ++q) t -= H[(size_t)i * m + q] * y[q];
      y[i] = t / H[(size_t)i * m + i];
    }
    HP_CUDA(cudaMemcpyAsync(dev_h, y.data(), sizeof(double) * k, cudaMemcpyHostToDevice, s));
    k_mcombine<<<MDOT_BLOCKS, 256, 0, s>>>(x_pad, Z, L, k, dev_h, L);
    HP_CHECK_LAUNCH();
    ++restarts;
  }
  check_status(c);
  if (st) {
    st->iters = its;
    st->restarts = restarts;
    st->rel_res_true = rel;
  }
  return rel <= tol ? HPLMM_OK : HPLMM_NOT_CONVERGED;
}

}  // namespace hp

namespace hp {

// k right-preconditioned FGMRES(m) solves with one preconditioner, run in lockstep so that every Arnoldi
// step applies M^{-1} to the current basis vectors of all unfinished solves at once (precond_apply_multi) and
// multiplies them by A_hat together; each solve keeps its own basis, Hessenberg matrix, Givens rotations
// and restarts.  B and X hold k padded vectors at stride 3 n_nodes; st (host, may be NULL) k entries.
int fgmres_multi(hplmm_ctx *c, const double *B, double *X, int k, double tol, hplmm_stats *st) {
  cudaStream_t s = c->stream;
  const long long L = 3LL * c->n_nodes;
  const int m = c->opt.restart, maxit = c->opt.max_iters;
  const size_t per = (size_t)(2 * m + 1) * L;  // V (m + 1 vectors) and Z (m vectors) of one solve
  c->mV.alloc(per * k);
  c->mw_in.alloc(L * k);
  c->mw_out.alloc(L * k);
  c->mw_w.alloc(L * k);
  c->mh.alloc((size_t)(2 * MAXV + 8) * k);
  struct Rhs {
    double bnorm = 0, rel = 0;
    int its = 0, restarts = 0, kk = 0;
    bool done = false, cyc = false;
    std::vector<double> H, cs, sn, g, y;
  };
  std::vector<Rhs> R(k);
  std::vector<double> hh(2 * MAXV + 1, 0.0);
  auto V = [&](int i) { return c->mV.p + per * i; };
  auto Zb = [&](int i) { return c->mV.p + per * i + (size_t)(m + 1) * L; };
  auto dh = [&](int i) { return c->mh.p + (size_t)(2 * MAXV + 8) * i; };
  HP_CUDA(cudaMemsetAsync(X, 0, sizeof(double) * L * k, s));
  for (int i = 0; i < k; ++i) {
    R[i].H.assign((size_t)(m + 1) * m, 0.0);
    R[i].cs.assign(m, 0.0);
    R[i].sn.assign(m, 0.0);
    R[i].g.assign(m + 1, 0.0);
    R[i].y.assign(m, 0.0);
    mdot(c, B + i * L, 0, 1, B + i * L, L, dh(i));
    HP_CUDA(cudaMemcpyAsync(hh.data(), dh(i), sizeof(double), cudaMemcpyDeviceToHost, s));
    HP_CUDA(cudaStreamSynchronize(s));
    R[i].bnorm = std::sqrt(hh[0]);
    HP_REQUIRE(std::isfinite(R[i].bnorm), HPLMM_ERR_INVALID,
               "solve: right-hand side " + std::to_string(i) + " has non-finite entries");
    if (R[i].bnorm == 0.0) R[i].done = true;
  }
  for (;;) {
    // true residuals and the start of a cycle for every unfinished solve
    bool any = false;
    for (int i = 0; i < k; ++i) {
      Rhs &r = R[i];
      if (r.done) continue;
      spmv(c, X + i * L, V(i), HPLMM_FP64, B + i * L);
      mdot(c, V(i), 0, 1, V(i), L, dh(i));
      HP_CUDA(cudaMemcpyAsync(hh.data(), dh(i), sizeof(double), cudaMemcpyDeviceToHost, s));
      HP_CUDA(cudaStreamSynchronize(s));
      const double beta = std::sqrt(hh[0]);
      r.rel = beta / r.bnorm;
      if (r.rel <= tol || r.its >= maxit) {
        r.done = true;
        continue;
      }
      any = true;
      k_scale_copy<<<grid_for(L, 256), 256, 0, s>>>(V(i), V(i), 1.0 / beta, L);
      HP_CHECK_LAUNCH();
      std::fill(r.g.begin(), r.g.end(), 0.0);
      r.g[0] = beta;
      r.kk = 0;
      r.cyc = true;
    }
    if (!any) break;
    for (int j = 0; j < m; ++j) {
      std::vector<int> act;
      for (int i = 0; i < k; ++i)
        if (!R[i].done && R[i].cyc) act.push_back(i);
      if (act.empty()) break;
      const int na = (int)act.size();
      for (int q = 0; q < na; ++q)
        HP_CUDA(cudaMemcpyAsync(c->mw_in.p + q * L, V(act[q]) + (size_t)j * L, sizeof(double) * L,
                                cudaMemcpyDeviceToDevice, s));
      precond_apply_multi(c, c->mw_in.p, c->mw_out.p, na);
      spmv_multi(c, c->mw_out.p, c->mw_w.p, na, HPLMM_FP64);
      for (int q = 0; q < na; ++q) {
        const int i = act[q];
        Rhs &r = R[i];
        double *w = c->mw_w.p + q * L;
        HP_CUDA(cudaMemcpyAsync(Zb(i) + (size_t)j * L, c->mw_out.p + q * L, sizeof(double) * L,
                                cudaMemcpyDeviceToDevice, s));
        ++r.its;
        mdot(c, V(i), L, j + 1, w, L, dh(i));
        cgs_update(c, V(i), L, j + 1, dh(i), w, L, 0, dh(i) + MAXV);
        cgs_update(c, V(i), L, j + 1, dh(i) + MAXV, w, L, 1, dh(i) + 2 * MAXV);
        HP_CUDA(cudaMemcpyAsync(hh.data(), dh(i), sizeof(double) * (2 * MAXV + 1), cudaMemcpyDeviceToHost, s));
        HP_CUDA(cudaStreamSynchronize(s));
        for (int a = 0; a <= j; ++a) r.H[(size_t)a * m + j] = hh[a] + hh[MAXV + a];
        const double hn = std::sqrt(std::max(hh[2 * MAXV], 0.0));
        r.H[(size_t)(j + 1) * m + j] = hn;
        for (int a = 0; a < j; ++a) {
          const double u = r.H[(size_t)a * m + j], v = r.H[(size_t)(a + 1) * m + j];
          r.H[(size_t)a * m + j] = r.cs[a] * u + r.sn[a] * v;
          r.H[(size_t)(a + 1) * m + j] = -r.sn[a] * u + r.cs[a] * v;
        }
        const double u = r.H[(size_t)j * m + j], v = r.H[(size_t)(j + 1) * m + j];
        const double den = std::hypot(u, v);
        r.cs[j] = u / den;
        r.sn[j] = v / den;
        r.H[(size_t)j * m + j] = den;
        r.H[(size_t)(j + 1) * m + j] = 0.0;
        r.g[j + 1] = -r.sn[j] * r.g[j];
        r.g[j] = r.cs[j] * r.g[j];
        r.kk = j + 1;
        const double est = std::fabs(r.g[j + 1]) / r.bnorm;
        if (hn > 0.0) {
          k_scale_copy<<<grid_for(L, 256), 256, 0, s>>>(V(i) + (size_t)(j + 1) * L, w, 1.0 / hn, L);
          HP_CHECK_LAUNCH();
        }
        if (est <= tol || hn == 0.0 || r.its >= maxit) r.cyc = false;
      }
    }
    // x += Z y for every solve that ran this cycle
    for (int i = 0; i < k; ++i) {
      Rhs &r = R[i];
      if (r.done || r.kk == 0) continue;
      for (int a = r.kk - 1; a >= 0; --a) {
        double t = r.g[a];
        for (int q = a + 1; q < r.kk; ++q) t -= r.H[(size_t)a * m + q] * r.y[q];
        r.y[a] = t / r.H[(size_t)a * m + a];
      }
      HP_CUDA(cudaMemcpyAsync(dh(i), r.y.data(), sizeof(double) * r.kk, cudaMemcpyHostToDevice, s));
      k_mcombine<<<MDOT_BLOCKS, 256, 0, s>>>(X + i * L, Zb(i), L, r.kk, dh(i), L);
      HP_CHECK_LAUNCH();
      HP_CUDA(cudaStreamSynchronize(s));
      ++r.restarts;
      r.kk = 0;
    }
  }
  check_status(c);
  bool all = true;
  for (int i = 0; i < k; ++i) {
    if (st) {
      st[i].iters = R[i].its;
      st[i].restarts = R[i].restarts;
      st[i].rel_res_true = R[i].rel;
    }
    if (!(R[i].rel <= tol)) all = false;
  }
  return all ? HPLMM_OK : HPLMM_NOT_CONVERGED;
}

}  // namespace hp
