// Internal definitions shared by the hPLMM CUDA translation units.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <stdexcept>
#include <type_traits>
#include <string>
#include <vector>

#include "../../include/hplmm.h"

// NVTX ranges around the library's phases (header-only NVTX 3: free unless a profiler is attached); left out
// where the toolkit has no NVTX headers
#if defined(__has_include)
#if __has_include(<nvtx3/nvToolsExt.h>)
#include <nvtx3/nvToolsExt.h>
#define HP_HAVE_NVTX 1
#endif
#endif

namespace hp {

// ---------------------------------------------------------------- errors
struct Error : public std::runtime_error {
  hplmm_status code;
  Error(hplmm_status c, const std::string &m) : std::runtime_error(m), code(c) {}
};

#define HP_CUDA(call)                                                                      \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) {                                                               \
      (void)cudaGetLastError(); /* a non-sticky error must not resurface at a later check */ \
      throw ::hp::Error(e_ == cudaErrorMemoryAllocation ? HPLMM_ERR_OOM : HPLMM_ERR_CUDA,  \
                        std::string(#call) + ": " + cudaGetErrorString(e_) + " at " +      \
                            __FILE__ + ":" + std::to_string(__LINE__));                    \
    }                                                                                      \
  } while (0)

// every kernel launch site checks its launch; the check also counts launches
long long note_launch();
#define HP_CHECK_LAUNCH()          \
  do {                             \
    ::hp::note_launch();           \
    HP_CUDA(cudaGetLastError());   \
  } while (0)

#define HP_REQUIRE(cond, code, msg)        \
  do {                                     \
    if (!(cond)) throw ::hp::Error(code, msg); \
  } while (0)

// test hook (hplmm_inject_alloc_failure): true when this device allocation is to fail as if out of memory
bool alloc_should_fail();

// ---------------------------------------------------------------- device buffer
template <typename T>
struct Buf {
  T *p = nullptr;
  size_t n = 0;    // current size (elements)
  size_t cap = 0;  // allocated capacity (elements); alloc() keeps the memory when it fits
  Buf() = default;
  Buf(const Buf &) = delete;
  Buf &operator=(const Buf &) = delete;
  ~Buf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = cap = 0;
  }
  void alloc(size_t count) {
    if (count == 0) count = 1;
    if (p && count <= cap) {
      n = count;
      return;
    }
    release();
    if (alloc_should_fail())
      throw Error(HPLMM_ERR_OOM, "cudaMalloc of " + std::to_string(count * sizeof(T)) +
                                     " bytes failed: injected failure (hplmm_inject_alloc_failure)");
    cudaError_t e = cudaMalloc(&p, count * sizeof(T));
    if (e != cudaSuccess) {
      p = nullptr;
      throw Error(HPLMM_ERR_OOM, "cudaMalloc of " + std::to_string(count * sizeof(T)) + " bytes failed: " +
                                     cudaGetErrorString(e));
    }
    n = cap = count;
  }
  void zero(cudaStream_t s) { HP_CUDA(cudaMemsetAsync(p, 0, n * sizeof(T), s)); }
  void fill_bytes(int v, cudaStream_t s) { HP_CUDA(cudaMemsetAsync(p, v, n * sizeof(T), s)); }
  void upload(const std::vector<T> &h, cudaStream_t s) {
    alloc(h.size());
    if (!h.empty()) HP_CUDA(cudaMemcpyAsync(p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s));
  }
  std::vector<T> download(cudaStream_t s, size_t count = (size_t)-1) const {
    if (count == (size_t)-1) count = n;
    std::vector<T> h(count);
    if (count) HP_CUDA(cudaMemcpyAsync(h.data(), p, count * sizeof(T), cudaMemcpyDeviceToHost, s));
    HP_CUDA(cudaStreamSynchronize(s));
    return h;
  }
  T *get() const { return p; }
};

inline unsigned grid_for(long long n, int block) {
  long long g = (n + block - 1) / block;
  if (g < 1) g = 1;
  if (g > 2147483647LL) g = 2147483647LL;
  return (unsigned)g;
}

// ---------------------------------------------------------------- primitives (prims.cu)
// exclusive scan of int32 values (in may equal out); returns the total
long long exclusive_scan_i32(const int *in, int *out, long long n, cudaStream_t s);
// sort 64-bit unsigned keys ascending in place (n arbitrary; uses a power-of-two scratch)
void sort_u64(uint64_t *keys, long long n, cudaStream_t s);

// ---------------------------------------------------------------- local band problems
// A local problem (grain grid or contact grid) is a principal submatrix of A_hat on
// the nodes of a box, numbered in a permuted lexicographic order (slowest axis = the
// longest box extent) so that the matrix is banded; all three components of every
// member node are kept, fixed components becoming identity rows.
struct LocalSet {
  int count = 0;
  // host copies
  std::vector<int> h_n;        // local DOFs (3 * member nodes)
  std::vector<int> h_bw;       // half bandwidth in DOFs
  std::vector<long long> h_band_off;  // offset of the band storage (elements)
  std::vector<long long> h_node_off;  // offset into node lists (capacity = box volume)
  std::vector<long long> h_vec_off;   // offset of local vectors (n entries each)
  long long band_total = 0, node_total = 0, vec_total = 0;
  // device
  Buf<int> box;       // per problem: lo[3], ext[3], perm[3] (9 ints)
  Buf<int> n;         // local DOF count
  Buf<int> bw;        // half bandwidth (DOFs)
  Buf<long long> band_off, node_off, vec_off;
  Buf<int> lnodes;    // ordinal -> global node id (node_off based)
  Buf<int> lmap;      // box cell (permuted lexicographic) -> ordinal or -1 (node_off based)
  Buf<double> band64;   // FP64 factors (panel width 16; diagonal rows hold inv(L_kk))
  Buf<float> band32;    // FP32 factors (panel width 32)
  Buf<__nv_bfloat16> band16;  // BF16 copy of the FP32 factors, used by the apply in the BF16 form
  bool apply_bf16 = false;
  Buf<int> order;     // problems sorted by decreasing factorisation cost
  Buf<int> queue;     // work counter of the persistent factorisation
  Buf<int> gidx;      // global vector index of every local DOF (vec_off based)
  Buf<double> yscr;   // smoother scratch: forward-sweep result per local DOF (vec_off based; FP32 sets use
                      // it as a float array)
  int tuned_chunk_rows = 0;  // smoother solve plan picked by the tuner (0 = default): far chunk rows,
  int tuned_ring_rows = 0;   // far ring rows (0 = largest that fits) and diagonal-chunk stages
  int tuned_c0_stages = 0;
  int tuned_cluster = 0;     // CTAs per problem of the smoother solve (0 = default: 2 when the set is small)
  int tuned_bulk = 0;        // bulk warps per CTA of the smoother solve (0 = 8; with 4, two CTAs share an SM)
  hplmm_prec prec = HPLMM_FP64;
};

// ---------------------------------------------------------------- sparse coarse factor (cfactor.cu)
// Multifrontal FP64 Cholesky of A^o.  A^o = sum over grains of a dense block on the grain's coupled
// columns, so the grains play the part of finite elements: a recursive bisection of the grain centres
// gives a nested-dissection tree, every coarse column group (an interface's mortar columns, or a grain's
// correction column) is eliminated at the lowest tree node whose subtree holds every grain coupled to it,
// and nodes with few columns are merged into their parents.  Front f (dense, row-major m x m) holds its
// p pivot columns, padded with identity columns to P (a multiple of 64), then its b boundary columns,
// which belong to ancestors; its boundary block receives the Schur update and is added into the parent.
struct FTask {
  int f, a, b, c;  // front and up to three tile or block indices
};
struct FLaunch {
  int kind;        // kernel (see cfactor.cu)
  int kt;          // tile step of the factorisation
  long long off;   // first task
  int count;       // tasks
};
struct CoarseFactor {
  int nf = 0, nlev = 0;
  long long F_total = 0, Y_total = 0, D_total = 0, idx_total = 0;
  std::vector<int> h_m, h_P, h_p, h_b, h_parent, h_level;
  std::vector<long long> h_foff, h_yoff, h_doff, h_ioff;
  Buf<int> m, P, p, b, parent;
  Buf<long long> foff, yoff, doff, ioff, roff;
  const int *bdev() const { return b.p; }
  Buf<int> idx;     // coarse column of every front row (-1 on padding rows)
  Buf<int> rank;    // elimination rank of every front row (-1 on padding rows)
  Buf<int> rel;     // per front: row of each of its boundary rows in the parent's front
  Buf<int> erank, owner, fpos;  // per coarse column: elimination rank, front, row in that front
  Buf<double> F;    // fronts; after the factorisation their first P columns hold [L_pp; L_bp]
  Buf<double> Y;    // per front: inv(L_pp), P x P row-major
  Buf<double> D;    // per front: inverses of the 64 x 64 diagonal tiles of L_pp
  Buf<FTask> tasks;
  Buf<int> otask;                       // tensor-core Schur update tasks: f, kt, it, jt, slot(it), slot(jt)
  Buf<__nv_bfloat16> oz_S;              // base-256 digits of one step's panel tiles (7 per value)
  Buf<int> oz_E;                        // their per-row exponents
  long long oz_slots = 0;
  std::vector<FLaunch> fact;            // factorisation launches, in order
  std::vector<std::vector<FLaunch>> fwd, bwd;  // solve launches per level (forward ascending, backward
                                               // descending levels)
  double flops = 0;                     // factorisation flops (pivot block, panel and Schur update)
  long long solve_bytes = 0;            // bytes of L and inv(L_pp) read by one coarse solve
};

// device view of the front layout, for adding A^o entries into the fronts
struct CFView {
  const int *erank, *owner, *fpos, *m, *P, *rank;
  const long long *foff, *ioff;
  double *F;
  int *status;
};

// position of coarse column `col` among the rows of front f: a pivot row, or a boundary row found by
// binary search of its elimination rank among the front's boundary rows (sorted by rank)
__device__ __forceinline__ int cf_row(const CFView &v, int f, int col) {
  if (v.owner[col] == f) return v.fpos[col];
  const int r = v.erank[col];
  const int *rk = v.rank + v.ioff[f];
  int a = v.P[f], b = v.m[f];
  const int end = b;
  while (a < b) {
    const int mid = (a + b) >> 1;
    if (rk[mid] < r) a = mid + 1;
    else b = mid;
  }
  return (a < end && rk[a] == r) ? a : -1;
}

// A^o[ca][cb] += val, into the front of whichever of the two columns is eliminated first
__device__ __forceinline__ void cf_add(const CFView &v, int ca, int cb, double val) {
  const int x = v.erank[ca] <= v.erank[cb] ? ca : cb;
  const int f = v.owner[x];
  const long long m = v.m[f];
  const int ra = cf_row(v, f, ca), rb = cf_row(v, f, cb);
  if (ra < 0 || rb < 0) {  // not in the front: the symbolic analysis is inconsistent
    if (atomicCAS(v.status, 0, (int)HPLMM_ERR_INVALID) == 0) {
      v.status[1] = 4;
      v.status[2] = f;
      v.status[3] = ra < 0 ? ca : cb;
    }
    return;
  }
  atomicAdd(v.F + v.foff[f] + (long long)ra * m + rb, val);
}

}  // namespace hp

// ---------------------------------------------------------------- the context
struct hplmm_ctx {
  hplmm_options opt{};
  cudaStream_t stream = nullptr;
  std::string err;
  int device = 0;

  // ---- assembly (Section 2)
  bool assembled = false;
  int nx = 0, ny = 0, nz = 0;
  long long n_grid = 0;            // (nx+1)(ny+1)(nz+1)
  int n_nodes = 0;
  long long n_dof = 0;
  double nu = 0.3, E0 = 1.0;
  hp::Buf<uint8_t> mask;           // voxel mask copy
  hp::Buf<float> E;                // voxel modulus (E0 filled if none given)
  hp::Buf<int> grid_to_node;       // n_grid -> node id or -1
  hp::Buf<int> node_ijk;           // n_nodes*3
  hp::Buf<uint8_t> fixed;          // n_nodes*3
  hp::Buf<int> free_index;         // n_nodes*3 -> free DOF or -1
  hp::Buf<int> dof_slot;           // n_dof -> node*3+d
  hp::Buf<double> Kref;            // 24x24 reference element stiffness (E = 1)
  std::vector<float> h_kref32;     // its FP32 copy (host), for the element-by-element residual updates
  hp::Buf<int> row_ptr, col;       // BSR over nodes, 3x3 blocks
  long long nnzb = 0;
  hp::Buf<double> val64;           // nnzb*9, fixed rows/cols zeroed
  hp::Buf<float> val32;            // FP32 shadow (assembly only; released once the sliced copy exists)
  hp::Buf<int> sell_perm;          // sliced ELL: node of each row position (longest rows first per window)
  hp::Buf<int> sell_off;           // sliced ELL (32-row slices): entry offset of each slice, n_slices+1
  hp::Buf<int> sell_col;           // block column per entry (slot-major within a slice)
  hp::Buf<double> sell_val64;      // 9 values per entry, element-major within a slot
  hp::Buf<float> sell_val32;
  hp::Buf<double> b_pad;           // n_nodes*3 right-hand side, 0 on fixed slots
  hp::Buf<double> b_corr;          // right-hand side defining the correction columns (padded)

  // ---- decomposition (Sections 3.1-3.2)
  bool setup_done = false;
  int n_grains = 0, px = 0, py = 0, pz = 0;
  hp::Buf<int> vgrain;             // grain id per voxel (-1 void)
  hp::Buf<int> node_cls;           // >=0 grain of an interior node; -1 interface node; -2 none
  hp::Buf<int> iface_of_node;      // interface id or -1
  hp::Buf<int> iface_slot;         // position of the node inside its interface list
  int n_ifaces = 0;
  long long n_iface_nodes = 0;
  hp::Buf<int> iface_pair;         // n_ifaces*2
  hp::Buf<int> iface_off;          // n_ifaces+1
  hp::Buf<int> iface_nodes;        // n_iface_nodes
  std::vector<int> h_iface_off;
  // grain -> coupled interfaces (CSR) and column layout
  std::vector<int> h_gi_off, h_gi_iface, h_gi_colbase;
  hp::Buf<int> gi_off, gi_iface, gi_colbase;  // colbase = local column offset of the interface inside K_g
  std::vector<int> h_kg;           // columns per grain (incl. correction)
  std::vector<long long> h_panel_off;  // offsets of X_g panels (elements)
  hp::Buf<int> kg;
  hp::Buf<long long> panel_off;
  std::vector<int> h_corr_col;     // coarse column of grain g's correction, or -1
  std::vector<std::vector<int>> h_glists;  // per grain: its coupled interfaces (ascending)
  std::vector<int> h_grain_hasb;   // per grain: b^g != 0 (a correction column is kept)
  hp::Buf<int> corr_col;

  // ---- mortars (Section 3.3)
  int n_mortars = 0;
  hp::Buf<int> mortar_off;         // n_ifaces+1
  hp::Buf<int> mortar_nodes;       // slot -> node id
  hp::Buf<int> mortar_idx;         // slot -> index into its interface's node list
  hp::Buf<long long> eta_off;      // n_ifaces+1 (elements)
  hp::Buf<double> eta;             // per interface: F x nc row-major
  hp::Buf<int> comp_mask;          // per interface: bit gamma set if component gamma has a free DOF
  hp::Buf<int> col_off;            // n_ifaces+1: first coarse column of each interface
  std::vector<int> h_mortar_off, h_comp_mask, h_col_off;
  long long n_mortar_cols = 0, n_coarse = 0;

  // ---- local problems
  hp::LocalSet grains, contacts;
  hp::LocalSet ifsets;             // algebraic mortars: the interfaces as local problems on their own nodes
  hp::Buf<int> mslot_of_node;      // algebraic mortars: global mortar slot of a node, or -1
  hp::Buf<int> mfree;              // per mortar slot: bit gamma set when the mortar node's DOF gamma is free
  hp::Buf<int> mcol;               // per mortar slot: its first column within its interface
  hp::Buf<double> qblk;            // per interface: Q^o block, rows (slot, component) x its columns
  hp::Buf<long long> qoff;         // offsets of the blocks
  hp::Buf<float> stage32;          // FP32 chunk of the staged BF16 set-up

  // ---- coarse space (Section 4.2)
  hp::Buf<double> X64;             // basis panels X_g (local DOF rows x k_g), FP64
  hp::Buf<float> X32;              // FP32 copy/compute
  hp::Buf<__nv_bfloat16> X16;      // BF16 copy of X32 for the apply of the BF16 form, column-major per grain
  hp::Buf<long long> panel_off_cm;  // offsets of the column-major BF16 panels (leading dimension N_g rounded to 8)
  std::vector<long long> h_panel_off_cm;
  hp::Buf<double> Ao;              // N^o x N^o dense copy, kept only when N^o <= dense_coarse_max
  bool dense_ao = false;
  hp::Buf<double> gal64;           // Galerkin work: P and Y on the grains' node boxes (FP64 form)
  hp::Buf<float> gal32;            // (FP32 form)
  hp::CoarseFactor cf;             // sparse (multifrontal) Cholesky factor of A^o
  hp::Buf<int> gcol_off, gcol;     // global coarse column of each panel column
  hp::Buf<int> status;             // device error word

  // ---- ILU(0) base smoother (smoother_kind = HPLMM_SMOOTHER_ILU0)
  hp::Buf<double> ilu_val;         // L and U in A_hat's block storage (nnzb x 9)
  hp::Buf<int> ilu_diag;           // position of each node row's diagonal block
  hp::Buf<int> ilu_nodes;          // nodes ordered by level
  std::vector<int> h_ilu_off;      // first entry of each non-empty level in ilu_nodes, then n_nodes

  // ---- apply / GMRES work vectors (padded n_nodes*3)
  hp::Buf<double> w_r1, w_r2, w_z1, w_zz, w_zg, w_t, w_w;
  hp::Buf<double> w_coarse_t, w_coarse_u, w_coarse_y;
  // multi-right-hand-side work (k vectors each): coarse vectors, padded fine vectors, local panels
  hp::Buf<double> mw_ct, mw_cu, mw_r1, mw_r2, mw_z1, mw_zz, mw_zg, mw_t, mw_in, mw_out;
  hp::Buf<double> mloc64, mV, mw_w, mh, mw_pin, mw_pout;
  hp::Buf<float> mloc32;
  hp::Buf<double> w_loc64;         // local vectors for smoother
  hp::Buf<float> w_loc32;
  hp::Buf<double> w_in, w_out;     // padded copies of API vectors
  hp::Buf<float> w_x32;            // FP32 copy of the vector of an element-by-element residual update
  hp::Buf<double> V, Z, w_dots, w_h;
  int gmres_cap = 0;
  hp::Buf<double> w_partial;
  hp::Buf<unsigned> w_ticket;      // last-block ticket of the Krylov reductions (zero between launches)

  // graph of the apply (options.use_graph): captured on a private stream from fixed work vectors
  cudaGraphExec_t apply_graph = nullptr;
  cudaStream_t cap_stream = nullptr;
  cudaStream_t aux_stream = nullptr;   // second stream of the concurrent local factorisations
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  bool capturing = false;
  long long graph_kernels = 0;     // kernels in the captured apply
  hp::Buf<double> w_gin, w_gout;

  double t_ml = 0, t_mg = 0;

  // ---- learned warm start and iterative basis solves (ws.cu)
  hp::Buf<float> Xrhs;             // copy of the basis right-hand sides (iterative solves, sample collection)
  hplmm_basis_stats bstats{};
  struct WarmStart {
    hp::Buf<float> theta, m, v, grad;       // parameters (FP32), Adam moments, gradient
    hp::Buf<__nv_bfloat16> theta16;         // BF16 copy for inference
    long long adam_step = 0;
    bool has_params = false;
    hp::Buf<float> tin, ttgt, tvalid;       // training set [S][5|3|3][17^3]
    long long n_samples = 0, cap = 0;
    hp::Buf<float> a1, a2, a3, q, g32a, g32b, gq, wflip, bx, bt, bv;  // training/inference scratch
    hp::Buf<__nv_bfloat16> h1, h2;
    hp::Buf<double> sums;
    hp::Buf<int> sg, sa, vmin, vmax, nfree, iters, unconv, nb;
    hp::Buf<float> scale, tscale, rel0, blk, dinv, pcg_work;
    hp::Buf<long long> ell_off;
    long long S = 0;                        // samples of the current set-up
  } ws;

  // ---- phase profiling (options.profile)
  struct ProfRec {
    int ph;
    cudaEvent_t e0, e1;
    long long launches;
  };
  std::vector<cudaEvent_t> ev_pool;
  std::vector<ProfRec> prof_pending;
  double prof_ms[HPLMM_PH_COUNT] = {};
  long long prof_launches[HPLMM_PH_COUNT] = {};
};

namespace hp {
long long launch_count();
void add_launches(long long n);  // launches issued by a graph replay (negative: undo counts of a capture)
cudaEvent_t prof_event(hplmm_ctx *c);
void prof_harvest(hplmm_ctx *c);

// times the kernels queued on the context's stream between construction and destruction
inline const char *phase_name(int ph) {
  static const char *const names[] = {"hplmm:maps",         "hplmm:factor_grains", "hplmm:factor_contacts",
                                      "hplmm:basis_rhs",    "hplmm:basis_solve",   "hplmm:galerkin",
                                      "hplmm:coarse_chol",  "hplmm:apply_coarse",  "hplmm:apply_contacts",
                                      "hplmm:apply_grains", "hplmm:spmv",          "hplmm:krylov",
                                      "hplmm:apply_graph",  "hplmm:factor_ilu",    "hplmm:apply_ilu"};
  static_assert(sizeof(names) / sizeof(names[0]) == HPLMM_PH_COUNT, "one name per phase");
  return (ph >= 0 && ph < HPLMM_PH_COUNT) ? names[ph] : "hplmm:?";
}

// a phase: an NVTX range always, CUDA events on the context's stream when options.profile is set
struct ProfScope {
  hplmm_ctx *c;
  int ph;
  cudaEvent_t e0 = nullptr;
  long long l0 = 0;
  ProfScope(hplmm_ctx *ctx, int phase) : c(ctx), ph(phase) {
#ifdef HP_HAVE_NVTX
    nvtxRangePushA(phase_name(ph));
#endif
    if (!c->opt.profile || c->capturing) return;
    e0 = prof_event(c);
    cudaEventRecord(e0, c->stream);
    l0 = launch_count();
  }
  ~ProfScope() {
#ifdef HP_HAVE_NVTX
    nvtxRangePop();
#endif
    if (!c->opt.profile || !e0) return;
    cudaEvent_t e1 = prof_event(c);
    cudaEventRecord(e1, c->stream);
    c->prof_pending.push_back({ph, e0, e1, launch_count() - l0});
  }
};

// assemble.cu
void assemble(hplmm_ctx *c, const uint8_t *mask, int nx, int ny, int nz, const float *E, double E0, double nu,
              const hplmm_bcs *bcs, double *b_out);
void spmv(hplmm_ctx *c, const double *x_pad, double *y_pad, hplmm_prec prec, const double *sub = nullptr);
// k vectors at stride 3 n_nodes (the matrix read once per group of four)
void spmv_multi(hplmm_ctx *c, const double *X, double *Y, int k, hplmm_prec prec, const double *SUB = nullptr);
void gather_free(hplmm_ctx *c, const double *pad, double *dof);
void scatter_free(hplmm_ctx *c, const double *dof, double *pad);
// maps.cu
void check_anchored(hplmm_ctx *c);  // throws HPLMM_ERR_SINGULAR when a solid part has no prescribed displacement
void layout_columns(hplmm_ctx *c);  // grain panel columns and coarse columns from the interfaces' column counts
void build_maps(hplmm_ctx *c, const int32_t *partition);
void build_mortars(hplmm_ctx *c);
void build_algebraic_mortars(hplmm_ctx *c);  // local.cu: Eq. algebra mortars (options.mortar_kind = 1)
void compute_W(hplmm_ctx *c, int64_t *W);
// local.cu
void build_local_sets(hplmm_ctx *c);
void factor_local(hplmm_ctx *c, LocalSet &S, hplmm_prec prec);
void factor_local_both(hplmm_ctx *c, hplmm_prec prec);  // grains and contact grids concurrently
// elementwise FP32 -> BF16 copy (round to nearest even)
void to_bf16(const float *src, __nv_bfloat16 *dst, long long n, cudaStream_t s);
void solve_local_multi_f64(hplmm_ctx *c, LocalSet &S, double *X, const Buf<long long> &x_off, const Buf<int> &x_ld,
                           const std::vector<int> &h_ld);
void solve_local_multi_f32(hplmm_ctx *c, LocalSet &S, float *X, const Buf<long long> &x_off, const Buf<int> &x_ld,
                           const std::vector<int> &h_ld);
void smoother_apply(hplmm_ctx *c, LocalSet &S, const double *r_pad, double *z_pad, bool atomic);
void smoother_apply_multi(hplmm_ctx *c, LocalSet &S, const double *R, double *Z, int k, bool atomic);
void factor_staged(hplmm_ctx *c, float *X, const Buf<long long> &x_off, const Buf<int> &x_ld,
                   const std::vector<int> &h_ld);  // BF16 form: chunked FP32 factors + basis solves -> BF16
void solve_local_multi_f32_subset(hplmm_ctx *c, LocalSet &S, float *X, const Buf<long long> &x_off,
                                  const Buf<int> &x_ld, const std::vector<int> &h_ld, const std::vector<int> &grains);
// ws.cu
long long ws_num_params();
void ws_set_params(hplmm_ctx *c, const float *theta_host);
void ws_get_params(hplmm_ctx *c, float *theta_host);
long long ws_collect(hplmm_ctx *c);
void ws_train(hplmm_ctx *c, const int32_t *order, long long n_order, int batch, double lr, double *loss_out);
double ws_loss_grad(hplmm_ctx *c, const float *theta, const float *x, const float *tgt, const float *valid, int B,
                    int D, float *grad);
void ws_pcg_basis(hplmm_ctx *c, bool warm);
void ws_infer(hplmm_ctx *c, const float *x, int B, float *q);  // BF16 inference, D = 17
int num_sms();
// coarse.cu
void build_coarse(hplmm_ctx *c, const double *b_pad_for_corr);  // = the three steps below
void coarse_rhs(hplmm_ctx *c, const double *b_pad_for_corr);     // panels X_g = right-hand sides
void coarse_basis_solve(hplmm_ctx *c);                             // X_g <- (A^g_g)^{-1} X_g
void coarse_finish(hplmm_ctx *c);                                  // Galerkin product, coarse factor
// cfactor.cu: symbolic analysis from the grains' voxel boxes (lo[3], ext[3] per grain), numeric
// factorisation of the fronts the Galerkin product filled, and x = (A^o)^{-1} t (t is overwritten, y is
// work; all three of length N^o)
void cf_analyse(hplmm_ctx *c, const std::vector<int> &gbox);
void cf_factor(hplmm_ctx *c);
void cf_solve(hplmm_ctx *c, double *t, double *y, double *x);
void coarse_apply(hplmm_ctx *c, const double *r_pad, double *z_pad);
void coarse_apply_multi(hplmm_ctx *c, const double *R, double *Z, int k);  // k vectors at stride 3 n_nodes
void prolong_column(hplmm_ctx *c, long long col, double *out_pad);
// apply.cu
void precond_apply(hplmm_ctx *c, const double *r_pad, double *z_pad);
void precond_apply_any(hplmm_ctx *c, const double *r_pad, double *z_pad);  // graph replay when use_graph
void drop_apply_graph(hplmm_ctx *c);
// checkpoint.cu: the set-up's state to a file and back (the context must be assembled on the same system)
void save_setup(hplmm_ctx *c, const char *path);
void load_setup(hplmm_ctx *c, const char *path);
void tune_local(hplmm_ctx *c);
void smoother_stage(hplmm_ctx *c, const double *r_pad, double *z_pad);
void ilu_setup(hplmm_ctx *c);
void ilu_stage(hplmm_ctx *c, const double *r_pad, double *z_pad);
int fgmres(hplmm_ctx *c, const double *b_pad, double *x_pad, double tol, hplmm_stats *st);
void precond_apply_multi(hplmm_ctx *c, const double *R, double *Z, int k);
int fgmres_multi(hplmm_ctx *c, const double *B, double *X, int k, double tol, hplmm_stats *st);
void check_status(hplmm_ctx *c);
}  // namespace hp
