/*
 * hplmm.h -- C interface of the GB300 (sm_103a) library for algebraic hPLMM,
 * the two-level multiscale preconditioner of Khan & Mehmani, "High-order
 * Multiscale Preconditioner for Elasticity of Arbitrary Structures", used in
 * right-preconditioned GMRES for Q1 finite-element linear elasticity on voxel
 * images.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Status codes are returned, never exceptions.  After any HPLMM_ERR_* the
 *   context may only be destroyed, except HPLMM_NOT_CONVERGED (solve returns
 *   its best iterate) and HPLMM_ERR_INVALID raised by argument checks that
 *   ran before any work was queued.  hplmm_last_error() gives the message.
 * - Work is queued on the CUDA stream given to hplmm_create (0 = legacy
 *   default stream).  hplmm_assemble, hplmm_setup and hplmm_solve
 *   synchronise that stream before returning; hplmm_apply* are asynchronous.
 * - "device" pointers are CUDA device (or managed) memory owned by the caller;
 *   "host" pointers are ordinary host memory owned by the caller.  The context
 *   owns every internal buffer and frees it in hplmm_destroy.
 * - Vectors of length n_dof hold the free degrees of freedom in the paper's
 *   fine-grid numbering: existing nodes in lexicographic order (x fastest),
 *   the x,y,z components of a node consecutive, Dirichlet components removed
 *   (Section 2, Eq. ls_all).  All such vectors are float64.
 * - Voxel arrays are [nz][ny][nx] with x fastest; voxel (i,j,k) spans
 *   [i,i+1]x[j,j+1]x[k,k+1] (h = 1).
 */
#ifndef HPLMM_H
#define HPLMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hplmm_ctx hplmm_ctx;

typedef enum {
  HPLMM_OK = 0,
  HPLMM_NOT_CONVERGED = 1,
  HPLMM_ERR_INVALID = -1,   /* bad argument, size or call order detected on the host */
  HPLMM_ERR_OOM = -2,       /* a device allocation failed */
  HPLMM_ERR_CUDA = -3,      /* a CUDA runtime error */
  HPLMM_ERR_SINGULAR = -4,  /* a non-positive pivot in a local or coarse Cholesky factorisation */
  HPLMM_ERR_TIMEOUT = -5,   /* a device-side wait ran out of its iteration budget */
  HPLMM_ERR_STATE = -6      /* call out of order (e.g. apply before setup) */
} hplmm_status;

typedef enum { HPLMM_FP64 = 0, HPLMM_FP32 = 1, HPLMM_BF16 = 2 } hplmm_prec;

/* Options (zero-initialise, then call hplmm_default_options). */
typedef struct {
  int n_mortar;          /* n: maximum mortar nodes per contact interface (Section 3.3; paper sweeps 1,2,4,8) */
  double beta;           /* Gaussian mortar spread, Eq. gauss (paper: 4) */
  int contact_halfwidth; /* w: contact grid = nodes within L-inf distance w of an interface (Section 3.1) */
  int n_st;              /* smoother stages, Eq. local_smoother (paper: 1 with M_CG) */
  hplmm_prec local_prec; /* precision of local factorisations and basis solves: FP64 or FP32 */
  hplmm_prec apply_prec; /* precision of the preconditioner apply: FP64 (everything), FP32 (local factors,
                            basis panels and the A_hat of its residual updates stored in FP32, FP32
                            arithmetic) or BF16 (local factors and basis panels stored in BF16, the residual
                            updates' A_hat in FP32, FP32 arithmetic); the coarse solve is FP64 in every form */
  int restart;           /* GMRES restart length (default 30) */
  int max_iters;         /* cap on total GMRES iterations (paper: 300) */
  int strict_two_grain;  /* 1: shape vectors only on the two grains of each interface (the paper's
                            literal Eq. col_pk); 0 (default): on every grain whose voxels touch it */
  int use_graph;         /* 1: capture one preconditioner apply as a CUDA graph at its first use after
                            set-up and replay it for every apply (phase timings then report the replays as
                            HPLMM_PH_APPLY_GRAPH) */
  int verbose;           /* 1: print phase timings to stderr */
  int profile;           /* 1: time every phase with CUDA events on the context's stream (hplmm_get_profile) */
  int autotune;          /* 1: at set-up, time the smoother solve's pipeline depths on this problem's local
                            problems and keep the fastest (cached per problem-size bucket for the process);
                            no effect with the ILU(0) smoother */
  int basis_solver;      /* local basis solves (Eqs. col_pk, col_cg): HPLMM_BASIS_DIRECT (default, the exact
                            banded Cholesky solve), HPLMM_BASIS_PCG (block-Jacobi CG from a zero guess) or
                            HPLMM_BASIS_PCG_WARM (CG from the learned warm start); the iterative forms need
                            local_prec = FP32, and a column that misses basis_tol after basis_max_iters
                            iterations makes its grain fall back to the exact solve */
  double basis_tol;      /* relative residual of the iterative basis solves (default 1e-6) */
  int basis_max_iters;   /* iteration cap of the iterative basis solves (default 3000) */
  int keep_basis_rhs;    /* 1: keep a copy of the basis right-hand sides after set-up (hplmm_ws_collect) */
  int smoother_ctas;     /* CTAs per local problem in the smoother solves: 0 (default) the tuner's choice, or
                            two for a set with at most half as many problems as the GPU has SMs, else one;
                            1 or 2 force it (two: a cluster that splits each panel's far rows) */
  int mortar_kind;       /* mortar functions (Section 3.3): HPLMM_MORTAR_GAUSSIAN (default, Eq. gauss, spread
                            beta) or HPLMM_MORTAR_ALGEBRAIC (Eq. algebra: each interface's mortar functions solve
                            its own elasticity block with unit/zero values at the mortar DOFs; no parameter) */
  int stage_mb;          /* BF16 apply form (local_prec FP32, apply_prec BF16, exact basis solves): the local
                            factors are computed in FP32 in chunks of at most this many MiB, each chunk of grains
                            used for its basis solves, then kept only as BF16 (0 = default, 6144); the result does
                            not depend on it */
  int wait_budget_us;    /* budget of each bounded device-side wait in the smoother's pipelined solves, in
                            microseconds at the nominal 2,070 MHz SM clock (0 = default, about 2 s); a wait that
                            runs out makes the launch stop and the next synchronising call return
                            HPLMM_ERR_TIMEOUT (a small value is how the tests exercise that path) */
  int tensor_galerkin;   /* Galerkin product P_hat^T A_hat P_hat of the FP32 and BF16 forms: 1 (default) on the
                            tensor cores (tcgen05.mma kind::tf32, three TF32 products per pair of FP32 operands,
                            FP32 accumulation in tensor memory), 0 on the FP32 CUDA cores; the FP64 form always
                            uses FP64 CUDA cores */
  int tensor_coarse;     /* Schur updates of the coarse multifrontal Cholesky: 1 (default) on the tensor cores in
                            FP64 by the Ozaki splitting scheme (each row cut to 56-bit fixed point in seven BF16
                            digits, digit products exact in FP32, FP64 recombination; FP64-accurate), 0 on the
                            FP64 CUDA cores */
  int matrix_free_updates; /* residual updates r - A_hat z inside the apply of the FP32 and BF16 forms: 1
                            (default) element by element from the voxel moduli and the reference stiffness, in
                            FP32 (no matrix read), 0 from the FP32 copy of A_hat (sliced ELL); the FP64 form
                            and the Krylov products always use the assembled FP64 A_hat */
  int smoother_bulk_warps; /* warps per CTA that stream the far rows in the smoother solves: 0 (default) the
                            tuner's choice, else 8; 8, 4, 2 or 1 force it (4, 2 and 1 run one CTA per local
                            problem, with a ring sized for two, three or four CTAs per SM, and so exclude
                            smoother_ctas = 2); the result does not depend on it beyond the order of additions */
  int smoother_kind;     /* base smoother M_l of Eq. local_smoother: HPLMM_SMOOTHER_CONTACT_GRAIN (default, M_CG of
                            Section 4.3) or HPLMM_SMOOTHER_ILU0 (M_ILU(0), the black-box smoother of the paper's
                            smoother comparison, Sections 4.1 and 5; use it with n_st = 6 as the paper does):
                            ILU(0) of A_hat in FP64 on its structural pattern (DOFs coupled when their nodes share
                            a solid voxel), rows eliminated in free-DOF order; the contact grids are then not built,
                            and the set-up fails with HPLMM_ERR_SINGULAR on a zero pivot */
} hplmm_options;

enum { HPLMM_BASIS_DIRECT = 0, HPLMM_BASIS_PCG = 1, HPLMM_BASIS_PCG_WARM = 2 };
enum { HPLMM_MORTAR_GAUSSIAN = 0, HPLMM_MORTAR_ALGEBRAIC = 1 };
enum { HPLMM_SMOOTHER_CONTACT_GRAIN = 0, HPLMM_SMOOTHER_ILU0 = 1 };

/* Boundary conditions on the six faces of the image box, in the order
 * x=0, x=nx, y=0, y=ny, z=0, z=nz (Eq. BC).  fix[f][d] != 0 prescribes
 * displacement component d on face f to value[f][d] (a later face overrides
 * an earlier one on shared nodes); traction[f] is a uniform traction on the
 * solid part of face f, applied to components that are not fixed. */
typedef struct {
  uint8_t fix[6][3];
  double value[6][3];
  double traction[6][3];
} hplmm_bcs;

typedef struct {
  int iters;              /* Arnoldi steps taken */
  int restarts;           /* completed restart cycles */
  double rel_res_true;    /* ||b - A x|| / ||b|| recomputed in FP64 at exit */
  double t_setup_ml;      /* smoother build (local factorisations of grains and contact grids), s */
  double t_setup_mg;      /* coarse build (maps, mortars, basis solves, Galerkin, coarse Cholesky), s */
  double t_solve;         /* GMRES, s */
  long long n_dof;        /* free fine DOFs */
  long long n_coarse;     /* coarse dimension N^o = N^o_m + kept corrections */
  long long n_interfaces; /* contact interfaces N^c (= contact grids N^zeta) */
  long long n_grains;     /* grain grids N^g */
} hplmm_stats;

/* Fill `opt` with the defaults: n=4, beta=4, w=2, n_st=1, FP64 locals and apply,
 * restart 30, 300 iterations, default coupling, no graph. */
void hplmm_default_options(hplmm_options *opt);

/* Create a context bound to the current CUDA device and `cuda_stream`
 * (a cudaStream_t, or NULL for the legacy default stream).  `opt` may be NULL
 * for defaults; it is copied.  Returns HPLMM_ERR_INVALID on bad options. */
hplmm_status hplmm_create(hplmm_ctx **ctx, const hplmm_options *opt, void *cuda_stream);

/* Assemble A_hat and b_hat (Section 2, Eqs. stiff_iso, BC, ls_all) from a voxel
 * image.  mask: DEVICE uint8 [nz][ny][nx], 1 = solid (the caller keeps one
 * connected component attached to a Dirichlet face; otherwise a local or
 * coarse factorisation reports HPLMM_ERR_SINGULAR).  E: DEVICE float32 per
 * voxel, or NULL for the constant E0.  bcs: HOST.  n_dof_out: HOST, receives
 * the number of free DOFs.  b_out: DEVICE float64 [n_dof] or NULL.  Replaces
 * any earlier assembly and set-up in this context.  Synchronises. */
hplmm_status hplmm_assemble(hplmm_ctx *ctx, const uint8_t *mask, int nx, int ny, int nz,
                            const float *E, double E0, double nu, const hplmm_bcs *bcs,
                            double *b_out, long long *n_dof_out);

/* Build the preconditioner (T_MG + T_ML): grain grids, contact interfaces,
 * W, mortars and Gaussian Q^o (Sections 3.1-3.3, 4.2), shape and correction
 * vectors (Eqs. col_pk, col_cg), A^o = P_hat^T A_hat P_hat and its Cholesky
 * factor (Eq. mg_struct), and the local factorisations of the contact-grain
 * smoother (Eqs. local_smoother_CG, Mg_Mz).
 * partition: DEVICE int32 grain id per voxel (values in [0, n_grains), void
 * voxels ignored), or NULL for the Cartesian slicing into px*py*pz grains.
 * b: DEVICE float64 [n_dof] right-hand side defining the correction columns,
 * or NULL for the assembled b_hat.  Synchronises. */
hplmm_status hplmm_setup(hplmm_ctx *ctx, const int32_t *partition, int n_grains,
                         int px, int py, int pz, const double *b);

/* z = M^{-1} r, the full multiplicative preconditioner of Eq. multi_precond
 * (M_G first, then n_st stages of the base smoother: M_CG, or M_ILU(0) with
 * options.smoother_kind).  r, z: DEVICE float64 [n_dof];
 * they may not alias.  Asynchronous on the context's stream. */
hplmm_status hplmm_apply(hplmm_ctx *ctx, const double *r, double *z);

/* z = M_G^{-1} r = P_hat (A^o)^{-1} P_hat^T r (Eq. mg_struct); with r = b_hat
 * this is the first-pass solution of Section 6.1.  DEVICE float64 [n_dof]. */
hplmm_status hplmm_apply_coarse(hplmm_ctx *ctx, const double *r, double *z);

/* z = M_l^{-1} r, one stage of the base smoother: the contact-grain smoother
 * M_CG (Eq. local_smoother_CG), or M_ILU(0) = U^{-1} L^{-1} with
 * options.smoother_kind = HPLMM_SMOOTHER_ILU0.  DEVICE float64 [n_dof]. */
hplmm_status hplmm_apply_smoother(hplmm_ctx *ctx, const double *r, double *z);

/* y = A_hat x in FP64.  DEVICE float64 [n_dof]. */
hplmm_status hplmm_spmv(hplmm_ctx *ctx, const double *x, double *y);

/* y = A_hat x in FP64, like hplmm_spmv, but allocating nothing.  The paper has
 * no counterpart: this entry point exists for callers that cannot allocate
 * device memory at call time -- their memory is held by their own pool or
 * fixed budget, or their loop must not pay cudaMalloc's implicit device
 * synchronisation.  The padded work vectors live in one file-scope device
 * array of 786,432 float64 slots per vector, so the context must have
 * 3 * n_nodes <= 786,432 (262,144 fine nodes); larger systems get
 * HPLMM_ERR_INVALID.  The array (12 MiB) stays allocated on every device that
 * loads the library until the process exits.  The first call on a device looks
 * up the array's device address once (make that first call before any stream
 * capture).  All calls share the array and it keeps the previous call's
 * contents (the padded input is cleared each call); calls that overlap on the
 * GPU race.  The context's device must be the current device
 * (HPLMM_ERR_INVALID otherwise), and the cached address assumes the device's
 * primary context is not reset while the library is loaded.  x, y: DEVICE
 * float64 [n_dof].  Asynchronous on the context's stream. */
hplmm_status hplmm_spmv_noalloc(hplmm_ctx *ctx, const double *x, double *y);

/* Right-preconditioned FGMRES(restart) with CGS2 Arnoldi in FP64 (Section 5),
 * x_0 = 0, stopping when ||b - A x|| / ||b|| <= tol (true residual checked
 * at the end of each cycle) or after max_iters steps.  b: DEVICE float64
 * [n_dof] or NULL for b_hat; x: DEVICE float64 [n_dof] (output).  st: HOST,
 * may be NULL.  Returns HPLMM_OK or HPLMM_NOT_CONVERGED.  Synchronises. */
hplmm_status hplmm_solve(hplmm_ctx *ctx, const double *b, double *x, double tol, hplmm_stats *st);

/* Several loads on one set-up (the reuse the paper builds the preconditioner for: Section 1, Section 6.3
 * on front-loading the set-up cost, Section 7.4).  hplmm_apply_multi: Z_q = M^{-1} R_q for q < k, the k
 * vectors applied together: the coarse restriction and prolongation read each basis panel once per eight
 * vectors, the SpMVs read A_hat once per four, and the smoother's local solves read each factor once per 32
 * (the FP64 and FP32 forms; the BF16 form keeps only BF16 factors and solves vector by vector).
 * hplmm_solve_multi: k right-preconditioned FGMRES solves in lockstep, each Arnoldi step applying M^{-1} to
 * all unfinished solves' vectors at once; every solve keeps its own basis, restarts and stopping test
 * (||b_q - A x_q|| / ||b_q|| <= tol); st (HOST, may be NULL) receives k entries.  R, Z, B, X: DEVICE
 * float64 [k][n_dof] (vector q at offset q n_dof); 1 <= k <= 64; Z (X) may not alias R (B).  apply_multi is
 * asynchronous, solve_multi synchronises.  The correction columns of the coarse space stay those of the
 * set-up's right-hand side. */
hplmm_status hplmm_apply_multi(hplmm_ctx *ctx, const double *R, double *Z, int k);
hplmm_status hplmm_solve_multi(hplmm_ctx *ctx, const double *B, double *X, int k, double tol, hplmm_stats *st);

/* Saving and reloading a set-up (the set-up is built once and reused, Sections 1, 6.3 and 7.4).
 * hplmm_save_setup writes everything hplmm_setup computed -- decomposition and maps, mortars, local factors
 * and layouts, basis panels, the coarse factor and its schedules, the tuner's plans -- to the file at path
 * (HOST, NUL-terminated; overwritten), after a header with the set-up options and a fingerprint of the
 * assembled system.  hplmm_load_setup reads such a file into a context that has been assembled on the same
 * system with the same set-up options (n_mortar, beta, contact_halfwidth, n_st, local_prec, apply_prec,
 * strict_two_grain, basis_solver, mortar_kind): apply and solve then behave as on the saved context, and
 * no hplmm_setup is needed.  Errors: HPLMM_ERR_STATE (no set-up to save; not assembled before a load),
 * HPLMM_ERR_INVALID (file unreadable, unwritable or of another format, or saved for another system or
 * other options; the context's previous set-up is then gone and hplmm_setup or a good load must follow),
 * HPLMM_ERR_OOM.  Both synchronise.  The file holds the factors in their stored precision (about the
 * device memory the set-up uses). */
hplmm_status hplmm_save_setup(hplmm_ctx *ctx, const char *path);
hplmm_status hplmm_load_setup(hplmm_ctx *ctx, const char *path);

/* Sizes of the index maps, for hplmm_get_maps.  HOST outputs. */
typedef struct {
  long long n_nodes;        /* existing fine nodes */
  long long n_dof;
  long long n_grains;
  long long n_interfaces;
  long long n_iface_nodes;  /* nodes on contact interfaces (with a free DOF) */
  long long n_mortars;      /* mortar nodes over all interfaces */
  long long n_mortar_cols;  /* N^o_m */
  long long n_coarse;       /* N^o */
} hplmm_sizes;

hplmm_status hplmm_get_sizes(hplmm_ctx *ctx, hplmm_sizes *out);

/* Copy the set-up's integer maps and mortar weights into caller arrays
 * (any pointer may be NULL to skip it).  Arrays are DEVICE memory.
 *   node_ijk       int32 [n_nodes][3]    grid coordinates of each existing node
 *   W              int64 [n_dof]         free-DOF index at each position of the W order (Eq. permute)
 *   iface_pair     int32 [n_interfaces][2] grains (a < b) of each interface
 *   iface_nodes    int32 [n_iface_nodes] node ids of interface 0, then 1, ... (ascending within)
 *   iface_offsets  int32 [n_interfaces+1]
 *   mortar_nodes   int32 [n_mortars]     mortar node ids of interface 0, then 1, ... (mortar order)
 *   mortar_offsets int32 [n_interfaces+1]
 *   eta            float64 [n_iface_nodes x ...] weights eta_i(y): for interface c, a row-major
 *                  block (nodes of c) x (mortars of c), blocks in interface order
 * Synchronises. */
hplmm_status hplmm_get_maps(hplmm_ctx *ctx, int32_t *node_ijk, int64_t *W, int32_t *iface_pair,
                            int32_t *iface_nodes, int32_t *iface_offsets, int32_t *mortar_nodes,
                            int32_t *mortar_offsets, double *eta);

/* Copy the coarse matrix A^o (N^o x N^o, row-major float64, DEVICE) -- the
 * symmetrised Galerkin product of Eq. mg_struct.  Synchronises. */
hplmm_status hplmm_get_coarse_matrix(hplmm_ctx *ctx, double *A_o);

/* Copy column `col` of P_hat in the free-DOF numbering (DEVICE float64 [n_dof]). */
hplmm_status hplmm_get_prolongation_column(hplmm_ctx *ctx, long long col, double *out);

/* Phases timed when options.profile = 1 (CUDA events around each phase's launches). */
typedef enum {
  HPLMM_PH_MAPS = 0,          /* grain/interface maps and mortars (Sections 3.1-3.3) */
  HPLMM_PH_FACTOR_GRAINS,     /* banded Cholesky of the grain blocks A^g_g, together with the contact-grid
                                 blocks factored concurrently on a second stream */
  HPLMM_PH_FACTOR_CONTACTS,   /* (kept for compatibility: zero, the contact grids are timed above) */
  HPLMM_PH_BASIS_RHS,         /* right-hand sides of Eqs. col_pk and col_cg */
  HPLMM_PH_BASIS_SOLVE,       /* batched multi-RHS local solves building P */
  HPLMM_PH_GALERKIN,          /* A^o = P_hat^T A_hat P_hat */
  HPLMM_PH_COARSE_CHOL,       /* FP64 Cholesky of A^o */
  HPLMM_PH_APPLY_COARSE,      /* M_G^{-1}: restriction, coarse solve, prolongation */
  HPLMM_PH_APPLY_CONTACTS,    /* M_zeta^{-1}: contact-grid solves */
  HPLMM_PH_APPLY_GRAINS,      /* M_g^{-1}: grain-grid solves */
  HPLMM_PH_SPMV,              /* every A_hat x product */
  HPLMM_PH_KRYLOV,            /* FGMRES vector work (CGS2 products, updates) */
  HPLMM_PH_APPLY_GRAPH,       /* whole preconditioner applies replayed from a captured CUDA graph (use_graph) */
  HPLMM_PH_FACTOR_ILU,        /* ILU(0) factorisation of A_hat (smoother_kind = HPLMM_SMOOTHER_ILU0) */
  HPLMM_PH_APPLY_ILU,         /* M_ILU(0)^{-1}: the two level-scheduled triangular solves */
  HPLMM_PH_COUNT
} hplmm_phase;

/* Cumulative milliseconds and kernel launches per phase since the last reset
 * (arrays of n >= HPLMM_PH_COUNT entries, HOST).  Requires options.profile. */
hplmm_status hplmm_get_profile(hplmm_ctx *ctx, double *ms, long long *launches, int n);
hplmm_status hplmm_reset_profile(hplmm_ctx *ctx);

/* Process-wide number of CUDA kernels this library has launched. */
long long hplmm_kernel_launches(void);

/* Testing aid (the paper has no counterpart): after `after` more device allocations by the library, the next
 * one fails as if the device were out of memory, and the call that made it returns HPLMM_ERR_OOM; later
 * allocations succeed again.  A negative value cancels a pending failure.  Process-wide; it lets a caller
 * exercise its out-of-memory handling without exhausting the device. */
void hplmm_inject_alloc_failure(long long after);

/* Algorithmic sizes of the current set-up, for roofline accounting (HOST output). */
typedef struct {
  long long nnzb;                 /* 3x3 blocks of A_hat */
  long long grain_band_elems;     /* stored factor elements of all grain blocks */
  long long contact_band_elems;   /* stored factor elements of all contact-grid blocks */
  double grain_chol_flops;        /* sum N b^2 over grain blocks (banded Cholesky) */
  double contact_chol_flops;      /* sum N b^2 over contact-grid blocks */
  double basis_solve_flops;       /* sum 4 N b k over grains (forward + backward, k right-hand sides) */
  long long grain_dofs;           /* sum of local DOFs of the grain blocks */
  long long contact_dofs;         /* sum of local DOFs of the contact-grid blocks */
  long long panel_elems;          /* stored basis-panel elements sum N_g k_g */
  int local_elem_bytes;           /* bytes per local factor element read by the apply (8 FP64, 4 FP32, 2 in the
                                     BF16 form) */
  long long n_nodes;              /* existing fine nodes (vectors inside the library are 3 n_nodes long) */
  long long sell_blocks;          /* stored 3x3 blocks of the sliced-ELL copy of A_hat (padding included) */
  long long coarse_solve_bytes;   /* bytes of the coarse factor read by one coarse solve (L and inv(L_pp)) */
  double coarse_factor_flops;     /* flops of the multifrontal coarse Cholesky (pivot blocks, panels, updates) */
  long long coarse_fronts;        /* fronts of the coarse factor */
  long long coarse_front_bytes;   /* device bytes of the fronts (dense, m x m each) */
  long long n_voxels;             /* voxels of the image (nx ny nz) */
  long long n_grid;               /* grid points (nx+1)(ny+1)(nz+1) */
  int matrix_free_updates;        /* the apply's residual updates are element by element (options) */
  long long ilu_levels;           /* non-empty node levels of the ILU(0) factor and solves (0 without it); each
                                     triangular solve is one launch per level and reads nnzb 3x3 blocks in all */
} hplmm_costs;

hplmm_status hplmm_get_costs(hplmm_ctx *ctx, hplmm_costs *out);

/* ---- learned warm start of the local basis solves --------------------------------------------
 * The paper solves the local basis problems exactly.  The library can instead solve them by
 * block-Jacobi preconditioned conjugate gradients, optionally started from the guess of a small 3-D
 * convolutional network (options.basis_solver).  A sample of one basis problem lives on the 17^3 node
 * grid of its grain (origin = minimum corner of the grain's solid voxels, at most 16 voxels per axis):
 * channel 0 = solid voxels of the grain, channel 1 = their log E, channels 2-4 = the right-hand side
 * divided by its RMS; the network predicts the solution divided by its RMS (CG rescales the guess by the
 * factor that minimises its A-norm error, so only the solution's shape is learned).  Network:
 * 3x3x3 convolutions with dilations 1, 2, 4, 8, channels 5 -> 32 -> 32 -> 32 -> 3, ReLU after the first
 * three; parameters (FP32) per layer W[co][ci][tz][ty][tx] then bias[co].  Training (Adam) and inference run in the library's own
 * kernels; inference stores weights and activations in BF16. */

/* Number of network parameters (floats). */
long long hplmm_ws_num_params(void);

/* Set (HOST float32 [n], n = hplmm_ws_num_params()) or read the network parameters; setting resets the
 * optimiser state. */
hplmm_status hplmm_ws_set_params(hplmm_ctx *ctx, const float *params, long long n);
hplmm_status hplmm_ws_get_params(hplmm_ctx *ctx, float *params, long long n);

/* Append the current set-up's basis problems (right-hand sides and their exact solutions) to the context's
 * training set; needs a set-up with local_prec = FP32, basis_solver = HPLMM_BASIS_DIRECT and
 * keep_basis_rhs = 1.  n_total (HOST, may be NULL) receives the number of samples held.  Synchronises. */
hplmm_status hplmm_ws_collect(hplmm_ctx *ctx, long long *n_total);
hplmm_status hplmm_ws_clear(hplmm_ctx *ctx);

/* Copy samples [first, first + count) of the training set out (DEVICE float32: in [count][5][17^3],
 * target and valid [count][3][17^3]; any pointer may be NULL).  Synchronises. */
hplmm_status hplmm_ws_get_samples(hplmm_ctx *ctx, long long first, long long count, float *in, float *target,
                                  float *valid);

/* Adam steps (lr, beta1 0.9, beta2 0.999, eps 1e-8) over minibatches of `batch` samples taken in the
 * order given (HOST int32 [n_order], indices into the training set: the caller draws the shuffle).
 * loss (HOST double [n_order / batch], may be NULL) receives the loss before each step.  Synchronises. */
hplmm_status hplmm_ws_train(hplmm_ctx *ctx, const int32_t *order, long long n_order, int batch, double lr,
                            double *loss);

/* Masked mean-squared loss and its gradient with respect to the parameters (FP32, the training path)
 * for n samples on a D^3 grid (3 <= D <= 17): in DEVICE float32 [n][5][D^3], target and valid DEVICE
 * float32 [n][3][D^3], grad DEVICE float32 [hplmm_ws_num_params()], loss HOST.  Synchronises. */
hplmm_status hplmm_ws_loss_grad(hplmm_ctx *ctx, const float *in, const float *target, const float *valid, int n,
                                int D, double *loss, float *grad);

/* The network's inference path as the warm start uses it (BF16 weights and activations, FP32 products and
 * sums): out [n][3][17^3] from in [n][5][17^3], both DEVICE float32, 1 <= n <= 4096.  Synchronises. */
hplmm_status hplmm_ws_predict(hplmm_ctx *ctx, const float *in, float *out, int n);

typedef struct {
  long long columns;          /* basis problems solved */
  long long iters_total;      /* CG iterations summed over the columns (the cap for columns that missed it) */
  long long iters_max;
  long long fallback_columns; /* columns that missed basis_tol */
  long long fallback_grains;  /* grains re-solved exactly because of them */
  double init_rel_res_mean;   /* mean over columns of ||b - A x0|| / ||b|| (1 for a zero guess) */
  double t_net_ms;            /* network inference (warm start) */
  double t_pcg_ms;            /* CG iterations */
} hplmm_basis_stats;

/* Statistics of the last set-up's iterative basis solves (zeros after an exact one).  HOST output. */
hplmm_status hplmm_get_basis_stats(hplmm_ctx *ctx, hplmm_basis_stats *out);

/* Message of the most recent error in this context (never NULL). */
const char *hplmm_last_error(const hplmm_ctx *ctx);

/* Free every device and host resource of the context.  NULL is ignored. */
void hplmm_destroy(hplmm_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* HPLMM_H */
