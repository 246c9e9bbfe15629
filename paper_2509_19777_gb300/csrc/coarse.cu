// Coarse space of the preconditioner (paper Section 4.2, Eqs. mg_struct, WQP,
// reduced_defs, bc_matrix, col_cg, col_pk): shape and correction vectors from
// batched local solves, the Galerkin coarse matrix A^o = P_hat^T A_hat P_hat,
// its FP64 Cholesky factor, and the restriction / prolongation of the apply.
//
// Storage.  For grain g the panel X_g holds, row-major with leading dimension
// k_g, the local DOFs of g (its interior nodes in the grain problem's order,
// three components each) against the k_g coarse columns coupled to g: the
// mortar columns of every coupled interface (interfaces in ascending order,
// inside one interface (mortar i, kept component gamma)), then the grain's
// correction column when it is kept.  The interface rows of P_hat are the
// Gaussian weights eta_i(y) (Q^o, Eq. reduced_defs) and are never stored.
#include "common.cuh"

#include <algorithm>
#include <type_traits>

namespace hp {
namespace {

// local column of interface c inside grain g's panel, or -1 if not coupled
__device__ __forceinline__ int colbase_of(const int *gi_off, const int *gi_iface, const int *gi_colbase, int g, int c) {
  int a = gi_off[g], b = gi_off[g + 1];
  while (a < b) {  // ascending interface ids
    int m = (a + b) >> 1;
    int v = gi_iface[m];
    if (v == c) return gi_colbase[m];
    if (v < c) a = m + 1;
    else b = m;
  }
  return -1;
}

__device__ __forceinline__ int comp_rank(int mask, int gamma) { return __popc(mask & ((1 << gamma) - 1)); }

// Q^o of algebraic mortars (Eq. algebra): per interface a dense block, rows (interface slot, component),
// columns the interface's own; q == nullptr selects the Gaussian mortars (eta_i e_gamma)
struct QAlg {
  const double *q;
  const long long *qoff;
  const int *col_off;  // first coarse column of each interface (its column count = the difference)
};

// right-hand sides of Eq. col_pk (-A^g_c Q^o e_k) and Eq. col_cg (b^g), one thread per local node
template <typename T>
__global__ void k_basis_rhs(int G, const long long *node_off, const int *nloc, const int *lnodes, const int *row_ptr,
                            const int *col, const double *val, const int *iface_of_node, const int *iface_slot,
                            const int *iface_pair, const int *mortar_off, const long long *eta_off, const double *eta,
                            const int *comp_mask, const int *gi_off, const int *gi_iface, const int *gi_colbase,
                            const int *kg, const int *corr_col, const long long *panel_off, const double *b,
                            int strict, T *X, QAlg qa) {
  int g = blockIdx.y;
  int cnt = nloc[g] / 3;
  int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= cnt) return;
  int ld = kg[g];
  T *Xg = X + panel_off[g];
  int n = lnodes[node_off[g] + o];
  for (int p = row_ptr[n]; p < row_ptr[n + 1]; ++p) {
    int m = col[p];
    int c = iface_of_node[m];
    if (c < 0) continue;
    if (strict && iface_pair[2 * c] != g && iface_pair[2 * c + 1] != g) continue;
    int base = colbase_of(gi_off, gi_iface, gi_colbase, g, c);
    if (base < 0) continue;
    int nc = mortar_off[c + 1] - mortar_off[c];
    int cm = comp_mask[c];
    int ncomp = __popc(cm);
    int slot = iface_slot[m];
    const double *et = eta + eta_off[c] + (long long)slot * nc;
    const double *v = val + (long long)p * 9;
    if (qa.q) {
      const int ncol = qa.col_off[c + 1] - qa.col_off[c];
      const double *qr = qa.q + qa.qoff[c] + (long long)3 * slot * ncol;
      for (int kk = 0; kk < ncol; ++kk)
        for (int d = 0; d < 3; ++d) {
          const double a = v[3 * d] * qr[kk] + v[3 * d + 1] * qr[ncol + kk] + v[3 * d + 2] * qr[2 * ncol + kk];
          if (a != 0.0) Xg[(long long)(3 * o + d) * ld + base + kk] -= (T)a;
        }
      continue;
    }
    for (int i = 0; i < nc; ++i) {
      double w = et[i];
      for (int gam = 0; gam < 3; ++gam) {
        if (!((cm >> gam) & 1)) continue;
        int lc = base + i * ncomp + comp_rank(cm, gam);
        for (int d = 0; d < 3; ++d) {
          double a = v[3 * d + gam];
          if (a != 0.0) Xg[(long long)(3 * o + d) * ld + lc] -= (T)(a * w);
        }
      }
    }
  }
  if (corr_col[g] >= 0)
    for (int d = 0; d < 3; ++d) Xg[(long long)(3 * o + d) * ld + (ld - 1)] = (T)b[3LL * n + d];
}

// voxel bounding box of every grain (for the Galerkin sub-assembly)
__global__ void k_grain_vbox(const int *vg, int nx, int ny, int nz, int *vmin, int *vmax) {
  long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= (long long)nx * ny * nz) return;
  int g = vg[v];
  if (g < 0) return;
  int p[3] = {(int)(v % nx), (int)((v / nx) % ny), (int)(v / ((long long)nx * ny))};
  for (int a = 0; a < 3; ++a) {
    atomicMin(&vmin[3 * g + a], p[a]);
    atomicMax(&vmax[3 * g + a], p[a]);
  }
}

struct GalBox {
  int lo[3], ext[3];  // node box: lo .. lo+ext-1
};

// P_hat restricted to the corners of grain g's voxels: interior rows from X_g, interface rows eta
template <typename T>
__global__ void k_gal_fill(const int *gbox, const long long *gal_off, const int *kg, const int *grid_to_node, int nx,
                           int ny, const int *node_cls, const int *iface_of_node, const int *iface_slot,
                           const uint8_t *fixed, const int *gbox_grain, const long long *node_off_g,
                           const int *lmap_g, const long long *panel_off, const T *X, const int *mortar_off,
                           const long long *eta_off, const double *eta, const int *comp_mask, const int *gi_off,
                           const int *gi_iface, const int *gi_colbase, int g0, long long gbase, T *P, QAlg qa) {
  int g = g0 + blockIdx.y;
  const int *bx = gbox + 6 * g;
  int ex = bx[3], ey = bx[4], ez = bx[5];
  int vol = ex * ey * ez;
  int cell = blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= vol) return;
  int k = kg[g];
  int x = bx[0] + cell % ex, y = bx[1] + (cell / ex) % ey, z = bx[2] + cell / (ex * ey);
  long long NX = nx + 1, NY = ny + 1;
  int n = grid_to_node[((long long)z * NY + y) * NX + x];
  if (n < 0) return;
  T *Pr = P + (gal_off[g] - gbase) + (long long)3 * cell * k;
  if (node_cls[n] == g) {
    // ordinal of n in the grain problem: box of the grain set (lo, ext, perm)
    const int *b = gbox_grain + 9 * g;
    int pp[3] = {x - b[0], y - b[1], z - b[2]};
    int f = b[6], m = b[7], s = b[8];
    int gc = (pp[s] * b[3 + m] + pp[m]) * b[3 + f] + pp[f];
    int o = lmap_g[node_off_g[g] + gc];
    const T *Xr = X + panel_off[g] + (long long)3 * o * k;
    for (int e = 0; e < 3 * k; ++e) Pr[e] = Xr[e];
    return;
  }
  int c = iface_of_node[n];
  if (c < 0) return;
  int base = colbase_of(gi_off, gi_iface, gi_colbase, g, c);
  if (base < 0) return;
  if (qa.q) {
    const int ncol = qa.col_off[c + 1] - qa.col_off[c];
    const double *qr = qa.q + qa.qoff[c] + (long long)3 * iface_slot[n] * ncol;
    for (int d = 0; d < 3; ++d) {
      if (fixed[3 * n + d]) continue;
      for (int kk = 0; kk < ncol; ++kk) Pr[(long long)d * k + base + kk] = (T)qr[d * ncol + kk];
    }
    return;
  }
  int nc = mortar_off[c + 1] - mortar_off[c];
  int cm = comp_mask[c];
  int ncomp = __popc(cm);
  const double *et = eta + eta_off[c] + (long long)iface_slot[n] * nc;
  for (int d = 0; d < 3; ++d) {
    if (fixed[3 * n + d] || !((cm >> d) & 1)) continue;
    for (int i = 0; i < nc; ++i) Pr[(long long)d * k + base + i * ncomp + comp_rank(cm, d)] = (T)et[i];
  }
}

// Y = A^(g) P on the grain's node box, A^(g) = sum over the grain's solid voxels of E_v K_ref
template <typename T>
__global__ void k_gal_Y(const int *gbox, const long long *gal_off, const int *kg, const int *vg, const uint8_t *mask,
                        const float *E, int nx, int ny, int nz, const double *Kref, const uint8_t *fixed,
                        const int *grid_to_node, int g0, long long gbase, const T *P, T *Y) {
  __shared__ T K[576];
  int g = g0 + blockIdx.y;
  for (int e = threadIdx.x; e < 576; e += blockDim.x) K[e] = (T)Kref[e];
  __syncthreads();
  const int *bx = gbox + 6 * g;
  int ex = bx[3], ey = bx[4], ez = bx[5];
  int vol = ex * ey * ez;
  int cell = blockIdx.x;
  if (cell >= vol) return;
  int k = kg[g];
  int x = bx[0] + cell % ex, y = bx[1] + (cell / ex) % ey, z = bx[2] + cell / (ex * ey);
  const T *Pg = P + (gal_off[g] - gbase);
  T *Yr = Y + (gal_off[g] - gbase) + (long long)3 * cell * k;
  for (int a = threadIdx.x; a < k; a += blockDim.x) {
    T acc[3] = {0, 0, 0};
    for (int dz = -1; dz <= 0; ++dz)
      for (int dy = -1; dy <= 0; ++dy)
        for (int dx = -1; dx <= 0; ++dx) {
          int vx = x + dx, vy = y + dy, vz = z + dz;
          if (vx < 0 || vy < 0 || vz < 0 || vx >= nx || vy >= ny || vz >= nz) continue;
          long long v = ((long long)vz * ny + vy) * nx + vx;
          if (vg[v] != g) continue;
          T Ev = (T)E[v];
          int ca = (x - vx) + 2 * (y - vy) + 4 * (z - vz);
          for (int cb = 0; cb < 8; ++cb) {
            int nx_ = vx + (cb & 1), ny_ = vy + ((cb >> 1) & 1), nz_ = vz + ((cb >> 2) & 1);
            int bc = ((nz_ - bx[2]) * ey + (ny_ - bx[1])) * ex + (nx_ - bx[0]);
            const T *pr = Pg + (long long)3 * bc * k + a;
            T p0 = pr[0], p1 = pr[k], p2 = pr[2 * k];
            for (int d = 0; d < 3; ++d) {
              const T *kr = K + (3 * ca + d) * 24 + 3 * cb;
              acc[d] += Ev * (kr[0] * p0 + kr[1] * p1 + kr[2] * p2);
            }
          }
        }
    Yr[a] = acc[0];
    Yr[k + a] = acc[1];
    Yr[2 * k + a] = acc[2];
  }
}

// A^o[gcol(a)][gcol(b)] += sum_r P[r][a] Y[r][b] over the grain's box rows; 32x32 output tiles
template <typename T>
__global__ void __launch_bounds__(256) k_gal_gemm(const int *tiles, const int *gbox, const long long *gal_off,
                                                  const int *kg, const int *gcol_off, const int *gcol, const T *P,
                                                  const T *Y, long long gbase, CFView cf, double *Ao,
                                                  long long No) {
  __shared__ T Ps[32][33];
  __shared__ T Ys[32][33];
  int g = tiles[3 * blockIdx.x], a0 = tiles[3 * blockIdx.x + 1], b0 = tiles[3 * blockIdx.x + 2];
  const int *bx = gbox + 6 * g;
  long long M = 3LL * bx[3] * bx[4] * bx[5];
  int k = kg[g];
  const T *Pg = P + (gal_off[g] - gbase);
  const T *Yg = Y + (gal_off[g] - gbase);
  int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;  // 16 x 16 threads, 2x2 outputs each
  T acc[2][2] = {{0, 0}, {0, 0}};
  for (long long r0 = 0; r0 < M; r0 += 32) {
    for (int e = threadIdx.x; e < 1024; e += 256) {
      int rr = e >> 5, cc = e & 31;
      long long r = r0 + rr;
      Ps[rr][cc] = (r < M && a0 + cc < k) ? Pg[r * k + a0 + cc] : (T)0;
      Ys[rr][cc] = (r < M && b0 + cc < k) ? Yg[r * k + b0 + cc] : (T)0;
    }
    __syncthreads();
#pragma unroll 8
    for (int rr = 0; rr < 32; ++rr) {
      T p0 = Ps[rr][ty], p1 = Ps[rr][ty + 16];
      T y0 = Ys[rr][tx], y1 = Ys[rr][tx + 16];
      acc[0][0] += p0 * y0;
      acc[0][1] += p0 * y1;
      acc[1][0] += p1 * y0;
      acc[1][1] += p1 * y1;
    }
    __syncthreads();
  }
  const int *gc = gcol + gcol_off[g];
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      int a = a0 + ty + 16 * i, bb = b0 + tx + 16 * j;
      if (a < k && bb < k) {
        cf_add(cf, gc[a], gc[bb], (double)acc[i][j]);
        if (Ao) atomicAdd(&Ao[(long long)gc[a] * No + gc[bb]], (double)acc[i][j]);
      }
    }
}

// ---- the Galerkin product on the 5th-generation tensor cores (FP32 forms): C = P^T Y per grain with
// tcgen05.mma kind::tf32 and the accumulator in tensor memory.  Near-FP32 accuracy from three TF32 products
// per pair of operands (x = x_hi + x_lo with x_hi the value rounded to TF32 and x_lo = x - x_hi exact in
// FP32: hi*hi + hi*lo + lo*hi; the dropped lo*lo term and the TF32 truncation of lo are below 2^-22 of the
// product).
// CTA = (grain, 128 columns a of P, up to 256 columns b of Y): 128 threads stage 16 box rows of both operands
// per step into shared memory in the canonical K-major layout without swizzle (8-row x 16-byte core
// matrices; core matrices along K 128 bytes apart, 8-row groups 512 bytes apart), two stages; one thread
// issues the 2 x 3 MMAs of a step (M = 128, N = the tile's columns rounded to 16, K = 8) and commits them to
// the stage's mbarrier, which releases the stage for the step two later.  The 128 x N accumulator sits in
// 256 TMEM columns (two CTAs per SM at most, by shared memory); each warp reads its 32 lanes back with
// tcgen05.ld and adds them into the coarse fronts.
namespace tc {
constexpr int KC = 16;                                // box rows per stage (K of the stage)
constexpr int A_BYTES = 128 * KC * 4;                 // one TF32 part of the A tile (8 KB)
constexpr int B_BYTES = 256 * KC * 4;                 // one TF32 part of the B tile (16 KB)
constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;  // hi and lo of both
constexpr int SMEM_BYTES = 2 * STAGE_BYTES;           // 96 KB
constexpr int TMEM_COLS = 256;
constexpr long long WAIT_CYCLES = 2000000000LL;      // bounded waits: about a second of SM clock

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of element (row, kk) of a tile in the K-major no-swizzle layout
__device__ __forceinline__ int koff(int row, int kk) {
  return (row >> 3) * 512 + (kk >> 2) * 128 + (row & 7) * 16 + (kk & 3) * 4;
}

__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  const uint64_t lbo = 128 >> 4, sbo = 512 >> 4;
  return (uint64_t)((addr >> 4) & 0x3fff) | (lbo << 16) | (sbo << 32) | (1ull << 46);  // version 1, no swizzle
}

__device__ __forceinline__ uint32_t idesc_tf32(int n) {
  return (1u << 4)                    // D: F32
         | (2u << 7) | (2u << 10)     // A, B: TF32 (both K-major)
         | ((uint32_t)(n >> 3) << 17) // N / 8
         | ((uint32_t)(128 >> 4) << 24);  // M / 16
}

// x = hi + lo exactly, hi = x rounded to the nearest TF32 value (|lo| <= 2^-12 |x|); the tensor core then
// truncates lo to TF32, an error of at most 2^-23 |x|
__device__ __forceinline__ void split_tf32(float x, float &hi, float &lo) {
  uint32_t h;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
  hi = __uint_as_float(h);
  lo = x - hi;
}

__device__ __forceinline__ void mma_tf32(uint32_t dtm, uint64_t a, uint64_t b, uint32_t id, int acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtm),
      "l"(a), "l"(b), "r"(id), "r"(acc)
      : "memory");
}

__device__ __forceinline__ bool bar_wait(uint64_t *bar, uint32_t parity) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.b32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(su32(bar)), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > WAIT_CYCLES) return false;
  }
}
}  // namespace tc

__global__ void __launch_bounds__(128) k_gal_gemm_tc(const int *tiles, const int *gbox, const long long *gal_off,
                                                     const int *kg, const int *gcol_off, const int *gcol,
                                                     const float *P, const float *Y, long long gbase, CFView cf,
                                                     double *Ao, long long No, int *status) {
  extern __shared__ __align__(1024) unsigned char tsm[];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
  // tile: grain, first column of P, first column of Y, and the range [c_beg, c_end) of 16-row chunks of the
  // box (split-K: the partial products of one output tile are added into the fronts atomically)
  const int *tl = tiles + 5 * blockIdx.x;
  const int g = tl[0], a0 = tl[1], b0 = tl[2], c_beg = tl[3], c_end = tl[4];
  const int *bx = gbox + 6 * g;
  const long long M = 3LL * bx[3] * bx[4] * bx[5];
  const int k = kg[g];
  const int nb = min(256, k - b0);
  const int N = (nb + 15) & ~15;
  const float *Pg = P + (gal_off[g] - gbase);
  const float *Yg = Y + (gal_off[g] - gbase);
  if (wid == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::su32(&tmem_base)),
                 "r"(tc::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::su32(&bar[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::su32(&bar[1])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t dtm = tmem_base;
  const uint32_t id = tc::idesc_tf32(N);
  const int nchunks = c_end - c_beg;
  // this thread's values of one chunk: column a0 + tid of P, columns b0 + tid and b0 + tid + 128 of Y
  float ra[tc::KC], rb[2][tc::KC];
  auto fetch = [&](int ch) {
    const long long r0 = (long long)(c_beg + ch) * tc::KC;
#pragma unroll
    for (int e = 0; e < tc::KC; ++e) {
      const long long r = r0 + e;
      ra[e] = (r < M && a0 + tid < k) ? __ldg(Pg + r * k + a0 + tid) : 0.f;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int j = tid + 128 * h;
        rb[h][e] = (r < M && j < nb) ? __ldg(Yg + r * k + b0 + j) : 0.f;
      }
    }
  };
  if (nchunks > 0) fetch(0);
  bool ok = true;
  for (int ch = 0; ch < nchunks; ++ch) {
    const int st = ch & 1;
    // the stage's previous MMAs (step ch - 2) must have read it
    if (ch >= 2 && ok && !tc::bar_wait(&bar[st], (uint32_t)(((ch - 2) >> 1) & 1))) ok = false;
    unsigned char *base = tsm + st * tc::STAGE_BYTES;
    unsigned char *Ahi = base, *Alo = base + tc::A_BYTES;
    unsigned char *Bhi = base + 2 * tc::A_BYTES, *Blo = Bhi + tc::B_BYTES;
    // store this chunk (four consecutive box rows per 16-byte store), split into TF32 hi and lo
#pragma unroll
    for (int q = 0; q < tc::KC; q += 4) {
      float4 h, l;
      tc::split_tf32(ra[q], h.x, l.x);
      tc::split_tf32(ra[q + 1], h.y, l.y);
      tc::split_tf32(ra[q + 2], h.z, l.z);
      tc::split_tf32(ra[q + 3], h.w, l.w);
      *reinterpret_cast<float4 *>(Ahi + tc::koff(tid, q)) = h;
      *reinterpret_cast<float4 *>(Alo + tc::koff(tid, q)) = l;
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        const int j = tid + 128 * hh;
        if (j < N) {
          float4 bh, bl;
          tc::split_tf32(rb[hh][q], bh.x, bl.x);
          tc::split_tf32(rb[hh][q + 1], bh.y, bl.y);
          tc::split_tf32(rb[hh][q + 2], bh.z, bl.z);
          tc::split_tf32(rb[hh][q + 3], bh.w, bl.w);
          *reinterpret_cast<float4 *>(Bhi + tc::koff(j, q)) = bh;
          *reinterpret_cast<float4 *>(Blo + tc::koff(j, q)) = bl;
        }
      }
    }
    // the next chunk's loads are in flight while this one is handed to the tensor cores
    if (ch + 1 < nchunks) fetch(ch + 1);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    // every step is committed (with or without MMAs), so that the last commit always arrives
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int ks = 0; ks < tc::KC / 8; ++ks) {
        if (!ok) break;
        const uint32_t off = (uint32_t)ks * 256u;  // two core matrices along K per MMA
        const uint64_t ah = tc::sdesc(tc::su32(Ahi) + off), al = tc::sdesc(tc::su32(Alo) + off);
        const uint64_t bh = tc::sdesc(tc::su32(Bhi) + off), bl = tc::sdesc(tc::su32(Blo) + off);
        tc::mma_tf32(dtm, ah, bh, id, (ch > 0 || ks > 0) ? 1 : 0);
        tc::mma_tf32(dtm, ah, bl, id, 1);
        tc::mma_tf32(dtm, al, bh, id, 1);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       tc::su32(&bar[st]))
                   : "memory");
    }
  }
  // the last commit covers every MMA issued before it (an empty box issues none and adds nothing)
  const int last = nchunks - 1;
  if (nchunks == 0) ok = false;
  else if (ok && !tc::bar_wait(&bar[last & 1], (uint32_t)((last >> 1) & 1))) ok = false;
  if (!ok && nchunks > 0) {
    atomicCAS(status, 0, (int)HPLMM_ERR_TIMEOUT);
    // the MMAs must not outlive the tensor memory: wait for the last commit once more before freeing it
    tc::bar_wait(&bar[last & 1], (uint32_t)((last >> 1) & 1));
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const int a = a0 + 32 * wid + lane;
  const int *gc = gcol + gcol_off[g];
  for (int c0 = 0; c0 < N; c0 += 16) {
    uint32_t v[16];
    const uint32_t taddr = dtm + ((uint32_t)(32 * wid) << 16) + (uint32_t)c0;
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    if (ok && a < k) {
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int bb = b0 + c0 + i;
        if (c0 + i < nb) {
          const double val = (double)__uint_as_float(v[i]);
          cf_add(cf, gc[a], gc[bb], val);
          if (Ao) atomicAdd(&Ao[(long long)gc[a] * No + gc[bb]], val);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (wid == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(dtm), "r"(tc::TMEM_COLS) : "memory");
}

__global__ void k_symmetrize(double *A, long long N, double *asym) {
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * N) return;
  long long i = e / N, j = e % N;
  if (j >= i) return;
  double a = A[i * N + j], b = A[j * N + i];
  double m = 0.5 * (a + b);
  A[i * N + j] = m;
  A[j * N + i] = m;
}

// ---------------------------------------------------------------- restriction / prolongation
// t[gcol] += sum over grain rows of X_g[row][a] r_loc[row]; CTA = (grain, chunk of RCHUNK rows):
// the chunk's residual entries are gathered once into shared memory, then each thread owns columns and
// reads the panel rows coalesced.
// rows of a grain's panel per CTA of the restriction: each CTA adds its k partial sums into the coarse
// vector atomically, so larger chunks mean fewer atomics (1,024 rows: a 12k-row grain takes 12 CTAs)
constexpr int RCHUNK = 1024;
constexpr int RCHUNK8 = 128;  // the same for the eight-vector restriction (its staged residuals are 8 wide)
// largest coarse dimension for which the dense A^o is also kept (for inspection only)
constexpr long long DENSE_COARSE_MAX = 12288;
// elements of each of the Galerkin work arrays (P and Y on the grains' node boxes) per batch of grains
constexpr long long GAL_WORK_ELEMS = 1LL << 28;

template <typename T, typename A>
__global__ void __launch_bounds__(256) k_restrict_grain(const long long *node_off, const int *nloc, const int *lnodes,
                                                        const int *kg, const long long *panel_off, const T *X,
                                                        const int *gcol_off, const int *gcol, const double *r,
                                                        double *t) {
  __shared__ A rl[RCHUNK];
  int g = blockIdx.y;
  int N = nloc[g];
  int row0 = blockIdx.x * RCHUNK;
  if (row0 >= N) return;
  int cnt = min(RCHUNK, N - row0);
  int k = kg[g];
  const int *ln = lnodes + node_off[g];
  for (int rr = threadIdx.x; rr < cnt; rr += blockDim.x) {
    int row = row0 + rr;
    int o = row / 3, d = row - 3 * o;
    rl[rr] = (A)r[3LL * ln[o] + d];
  }
  __syncthreads();
  const T *Xg = X + panel_off[g] + (long long)row0 * k;
  for (int a = threadIdx.x; a < k; a += blockDim.x) {
    A s0 = 0, s1 = 0, s2 = 0, s3 = 0;
    const T *xa = Xg + a;
    int rr = 0;
    for (; rr + 3 < cnt; rr += 4) {  // four independent rows in flight per thread
      const A x0 = (A)xa[(long long)rr * k], x1 = (A)xa[(long long)(rr + 1) * k];
      const A x2 = (A)xa[(long long)(rr + 2) * k], x3 = (A)xa[(long long)(rr + 3) * k];
      s0 += x0 * rl[rr];
      s1 += x1 * rl[rr + 1];
      s2 += x2 * rl[rr + 2];
      s3 += x3 * rl[rr + 3];
    }
    for (; rr < cnt; ++rr) s0 += (A)xa[(long long)rr * k] * rl[rr];
    atomicAdd(&t[gcol[gcol_off[g] + a]], (double)((s0 + s1) + (s2 + s3)));
  }
}

// interface part of the restriction: t[(c,i,gamma)] += sum_y eta_i(y) r(y,gamma); thread per interface node
__global__ void k_restrict_iface(const int *iface_nodes, const int *iface_of_node, long long count,
                                 const int *iface_slot, const int *mortar_off, const long long *eta_off,
                                 const double *eta, const int *comp_mask, const int *col_off, const uint8_t *fixed,
                                 const double *r, double *t, QAlg qa) {
  long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= count) return;
  int n = iface_nodes[p];
  int c = iface_of_node[n];
  if (qa.q) {
    const int ncol = col_off[c + 1] - col_off[c];
    const double *qr = qa.q + qa.qoff[c] + (long long)3 * iface_slot[n] * ncol;
    const double r0 = r[3LL * n], r1 = r[3LL * n + 1], r2 = r[3LL * n + 2];
    for (int kk = 0; kk < ncol; ++kk) {
      const double v = qr[kk] * r0 + qr[ncol + kk] * r1 + qr[2 * ncol + kk] * r2;
      if (v != 0.0) atomicAdd(&t[col_off[c] + kk], v);
    }
    return;
  }
  int nc = mortar_off[c + 1] - mortar_off[c];
  int cm = comp_mask[c], ncomp = __popc(cm);
  const double *et = eta + eta_off[c] + (long long)iface_slot[n] * nc;
  for (int gam = 0; gam < 3; ++gam) {
    if (!((cm >> gam) & 1) || fixed[3 * n + gam]) continue;
    double rv = r[3LL * n + gam];
    if (rv == 0.0) continue;
    for (int i = 0; i < nc; ++i) atomicAdd(&t[col_off[c] + i * ncomp + comp_rank(cm, gam)], et[i] * rv);
  }
}

// z on grain rows = X_g u[K_g]: one warp per 8 consecutive rows (lanes over the k_g columns, coalesced;
// the 8 rows' loads issued together), the 8 partial sums reduced by a butterfly that halves the values per
// lane at each of the first three levels (9 shuffles for 8 rows)
template <typename T, typename A>
__global__ void __launch_bounds__(256) k_prolong_grain(const long long *node_off, const int *nloc, const int *lnodes,
                                                       const int *kg, const long long *panel_off, const T *X,
                                                       const int *gcol_off, const int *gcol, const double *u,
                                                       double *z) {
  constexpr int R = 8;
  __shared__ A ul[512];
  const int g = blockIdx.y;
  const int k = kg[g];
  for (int a = threadIdx.x; a < k; a += blockDim.x) ul[a] = (A)u[gcol[gcol_off[g] + a]];
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int N = nloc[g];
  const T *Xg = X + panel_off[g];
  const int *ln = lnodes + node_off[g];
  const int nw = blockDim.x >> 5;
  for (int row0 = R * (blockIdx.x * nw + wid); row0 < N; row0 += R * gridDim.x * nw) {
    A acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = 0;
    for (int a = lane; a < k; a += 32) {
      const A ua = ul[a];
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (row0 + r < N) acc[r] += (A)Xg[(long long)(row0 + r) * k + a] * ua;
    }
    // level xor 16: rows 0-3 stay on lanes with bit 4 clear, rows 4-7 on the others; then xor 8, xor 4
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const bool up = lane & 16;
      const A send = up ? acc[h] : acc[h + 4];
      const A keep = up ? acc[h + 4] : acc[h];
      acc[h] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const bool up = lane & 8;
      const A send = up ? acc[h] : acc[h + 2];
      const A keep = up ? acc[h + 2] : acc[h];
      acc[h] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    {
      const bool up = lane & 4;
      const A send = up ? acc[0] : acc[1];
      const A keep = up ? acc[1] : acc[0];
      acc[0] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    acc[0] += __shfl_xor_sync(0xffffffffu, acc[0], 2);
    acc[0] += __shfl_xor_sync(0xffffffffu, acc[0], 1);
    // lane l holds row 4 (bit 4) + 2 (bit 3) + (bit 2)
    const int row = row0 + ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
    if ((lane & 3) == 0 && row < N) {
      const int o = row / 3, d = row - 3 * o;
      z[3LL * ln[o] + d] = (double)acc[0];
    }
  }
}

__global__ void k_prolong_iface(const int *iface_nodes, const int *iface_of_node, long long count,
                                const int *iface_slot, const int *mortar_off, const long long *eta_off,
                                const double *eta, const int *comp_mask, const int *col_off, const uint8_t *fixed,
                                const double *u, double *z, QAlg qa) {
  long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= count) return;
  int n = iface_nodes[p];
  int c = iface_of_node[n];
  if (qa.q) {
    const int ncol = col_off[c + 1] - col_off[c];
    const double *qr = qa.q + qa.qoff[c] + (long long)3 * iface_slot[n] * ncol;
    const double *uc = u + col_off[c];
    for (int d = 0; d < 3; ++d) {
      double sum = 0.0;
      if (!fixed[3 * n + d])
        for (int kk = 0; kk < ncol; ++kk) sum += qr[d * ncol + kk] * uc[kk];
      z[3LL * n + d] = sum;
    }
    return;
  }
  int nc = mortar_off[c + 1] - mortar_off[c];
  int cm = comp_mask[c], ncomp = __popc(cm);
  const double *et = eta + eta_off[c] + (long long)iface_slot[n] * nc;
  for (int gam = 0; gam < 3; ++gam) {
    double s = 0.0;
    if (((cm >> gam) & 1) && !fixed[3 * n + gam])
      for (int i = 0; i < nc; ++i) s += et[i] * u[col_off[c] + i * ncomp + comp_rank(cm, gam)];
    z[3LL * n + gam] = s;
  }
}

// multi-right-hand-side restriction: t_q[gcol] += sum over grain rows of X_g[row][a] r_q[row] for q < kc
// (kc <= 8 vectors at stride L, their coarse vectors at stride No): each panel element read once per group
template <typename T, typename A>
__global__ void __launch_bounds__(256) k_restrict_grain8(const long long *node_off, const int *nloc,
                                                         const int *lnodes, const int *kg, const long long *panel_off,
                                                         const T *X, const int *gcol_off, const int *gcol,
                                                         const double *r, long long L, double *t, long long No,
                                                         int kc) {
  __shared__ A rl[8][RCHUNK8];
  const int g = blockIdx.y;
  const int N = nloc[g];
  const int row0 = blockIdx.x * RCHUNK8;
  if (row0 >= N) return;
  const int cnt = min(RCHUNK8, N - row0);
  const int k = kg[g];
  const int *ln = lnodes + node_off[g];
  for (int e = threadIdx.x; e < 8 * RCHUNK8; e += blockDim.x) {
    const int q = e / RCHUNK8, rr = e % RCHUNK8;
    A v = 0;
    if (q < kc && rr < cnt) {
      const int row = row0 + rr, o = row / 3, d = row - 3 * o;
      v = (A)r[q * L + 3LL * ln[o] + d];
    }
    rl[q][rr] = v;
  }
  __syncthreads();
  const T *Xg = X + panel_off[g] + (long long)row0 * k;
  for (int a = threadIdx.x; a < k; a += blockDim.x) {
    A acc[8] = {};
    for (int rr = 0; rr < cnt; ++rr) {
      const A x = (A)Xg[(long long)rr * k + a];
#pragma unroll
      for (int q = 0; q < 8; ++q) acc[q] += x * rl[q][rr];
    }
    const int col = gcol[gcol_off[g] + a];
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if (q < kc) atomicAdd(&t[q * No + col], (double)acc[q]);
  }
}

// multi-right-hand-side prolongation on grain rows: z_q[row] = X_g[row][.] u_q[K_g]; warp per row
template <typename T, typename A>
__global__ void __launch_bounds__(256) k_prolong_grain8(const long long *node_off, const int *nloc, const int *lnodes,
                                                        const int *kg, const long long *panel_off, const T *X,
                                                        const int *gcol_off, const int *gcol, const double *u,
                                                        long long No, double *z, long long L, int kc) {
  __shared__ A ul[8][512];
  const int g = blockIdx.y;
  const int k = kg[g];
  for (int e = threadIdx.x; e < 8 * k; e += blockDim.x) {
    const int q = e / k, a = e % k;
    ul[q][a] = q < kc ? (A)u[q * No + gcol[gcol_off[g] + a]] : (A)0;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int N = nloc[g];
  const T *Xg = X + panel_off[g];
  const int *ln = lnodes + node_off[g];
  for (int row = blockIdx.x * nw + wid; row < N; row += gridDim.x * nw) {
    A acc[8] = {};
    for (int a = lane; a < k; a += 32) {
      const A x = (A)Xg[(long long)row * k + a];
#pragma unroll
      for (int q = 0; q < 8; ++q) acc[q] += x * ul[q][a];
    }
#pragma unroll
    for (int q = 0; q < 8; ++q)
      for (int o = 16; o > 0; o >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
    if (lane < kc) {
      A v = acc[0];
#pragma unroll
      for (int q = 1; q < 8; ++q)
        if (lane == q) v = acc[q];
      const int o = row / 3, d = row - 3 * o;
      z[lane * L + 3LL * ln[o] + d] = (double)v;
    }
  }
}

// ---- column-major BF16 panels of the BF16 form's apply.  Column a of grain g sits at Xc[cm_off[g] + a ld_g]
// with ld_g = N_g rounded up to 8, so that every column starts on 16 bytes and a lane moves 8 rows (uint4) per
// load; the padding rows hold zeros.
__host__ __device__ inline int cm_ld(int n) { return (n + 7) & ~7; }

// exact BF16 -> FP32 of the two halves of a 32-bit word
__device__ __forceinline__ float bf_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf_hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }

__device__ __forceinline__ void bf8_to_f32(const uint4 v, float *x) {
  x[0] = bf_lo(v.x), x[1] = bf_hi(v.x), x[2] = bf_lo(v.y), x[3] = bf_hi(v.y);
  x[4] = bf_lo(v.z), x[5] = bf_hi(v.z), x[6] = bf_lo(v.w), x[7] = bf_hi(v.w);
}

// transpose-convert of the FP32 row-major panels (32 x 32 tiles through shared memory)
__global__ void k_panel_bf16_cm(const int *nloc, const int *kg, const long long *panel_off, const long long *cm_off,
                                const float *X, __nv_bfloat16 *Xc) {
  __shared__ float tile[32][33];
  const int g = blockIdx.z;
  const int N = nloc[g], k = kg[g], ld = cm_ld(N);
  const int r0 = blockIdx.x * 32, a0 = blockIdx.y * 32;
  if (r0 >= ld || a0 >= k) return;
  const float *Xg = X + panel_off[g];
  __nv_bfloat16 *Cg = Xc + cm_off[g];
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int row = r0 + i, a = a0 + threadIdx.x;
    tile[i][threadIdx.x] = (row < N && a < k) ? Xg[(long long)row * k + a] : 0.f;
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += 8) {
    const int a = a0 + j, row = r0 + threadIdx.x;
    if (row < ld && a < k) Cg[(long long)a * ld + row] = __float2bfloat16_rn(tile[threadIdx.x][j]);
  }
}

// Sums of 8 values over a warp (a butterfly that halves the values each lane carries at the first three levels:
// 9 shuffles).  On return v[0] of lane l holds the sum of value 4 b4 + 2 b3 + b2 (b = the bits of l).
__device__ __forceinline__ void warp_sum8(float *v, int lane) {
#pragma unroll
  for (int h = 0; h < 4; ++h) {
    const bool up = lane & 16;
    const float send = up ? v[h] : v[h + 4], keep = up ? v[h + 4] : v[h];
    v[h] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const bool up = lane & 8;
    const float send = up ? v[h] : v[h + 2], keep = up ? v[h + 2] : v[h];
    v[h] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  {
    const bool up = lane & 4;
    const float send = up ? v[0] : v[1], keep = up ? v[1] : v[0];
    v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
  v[0] += __shfl_xor_sync(0xffffffffu, v[0], 2);
  v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
}

constexpr int CM_ROWS = 2048;  // panel rows per CTA in the column-major restriction and prolongation (8 per thread)

// restriction t_q[gcol] += sum over the grain's rows of X_g[row][a] r_q[row] on column-major BF16 panels:
// CTA = (grain, 2,048 rows), lane = 8 consecutive rows whose residuals it keeps in registers, warps over the
// columns.  MULTI = false: one vector, 8 columns per step (8 loads in flight); MULTI = true: kc <= 8 vectors at
// stride L / No, one column per step.  The warp sums go to shared memory, then one atomic per column and vector.
template <bool MULTI>
__global__ void __launch_bounds__(256) k_restrict_grain_cm(const long long *node_off, const int *nloc,
                                                           const int *lnodes, const int *kg, const long long *cm_off,
                                                           const __nv_bfloat16 *Xc, const int *gcol_off,
                                                           const int *gcol, const double *r, long long L, double *t,
                                                           long long No, int kc) {
  constexpr int KQ = MULTI ? 8 : 1;
  __shared__ float colsum[KQ][512];
  const int g = blockIdx.y;
  const int N = nloc[g], ld = cm_ld(N), k = kg[g];
  const int row0 = blockIdx.x * CM_ROWS;
  if (row0 >= ld) return;
  for (int e = threadIdx.x; e < KQ * 512; e += blockDim.x) colsum[e / 512][e % 512] = 0.f;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int *ln = lnodes + node_off[g];
  const __nv_bfloat16 *Xg = Xc + cm_off[g];
  // the 8 warps split the CTA's rows: warp w takes rows row0 + 256 w + 8 lane + [0, 8)
  const int rs = row0 + 256 * wid + 8 * lane;
  const bool live = rs < ld;
  float rl[KQ][8];
#pragma unroll
  for (int q = 0; q < KQ; ++q)
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      float v = 0.f;
      const int row = rs + j;
      if (q < kc && row < N) {
        const int o = row / 3, d = row - 3 * o;
        v = (float)r[q * L + 3LL * ln[o] + d];
      }
      rl[q][j] = v;
    }
  __syncthreads();
  const int sel = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
  if (!MULTI) {
    for (int a0 = 0; a0 < k; a0 += 8) {
      float acc[8];
      uint4 xv[8];
#pragma unroll
      for (int c = 0; c < 8; ++c)
        xv[c] = (live && a0 + c < k) ? __ldg(reinterpret_cast<const uint4 *>(Xg + (long long)(a0 + c) * ld + rs))
                                     : make_uint4(0, 0, 0, 0);
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        float x[8];
        bf8_to_f32(xv[c], x);
        float s = 0.f;
#pragma unroll
        for (int j = 0; j < 8; ++j) s += x[j] * rl[0][j];
        acc[c] = s;
      }
      warp_sum8(acc, lane);
      if ((lane & 3) == 0 && a0 + sel < k) atomicAdd(&colsum[0][a0 + sel], acc[0]);
    }
  } else {
    for (int a = 0; a < k; ++a) {
      const uint4 xv = live ? __ldg(reinterpret_cast<const uint4 *>(Xg + (long long)a * ld + rs))
                            : make_uint4(0, 0, 0, 0);
      float x[8], acc[8];
      bf8_to_f32(xv, x);
#pragma unroll
      for (int q = 0; q < KQ; ++q) {
        float s = 0.f;
#pragma unroll
        for (int j = 0; j < 8; ++j) s += x[j] * rl[q][j];
        acc[q] = s;
      }
      warp_sum8(acc, lane);
      if ((lane & 3) == 0 && sel < kc) atomicAdd(&colsum[sel][a], acc[0]);
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < KQ * k; e += blockDim.x) {
    const int q = e / k, a = e % k;
    if (q < kc) {
      const float v = colsum[q][a];
      if (v != 0.f) atomicAdd(&t[q * No + gcol[gcol_off[g] + a]], (double)v);
    }
  }
}

// prolongation z_q[row] = X_g[row][.] u_q[K_g] on column-major BF16 panels: thread = 8 consecutive rows (one
// 16-byte load per column, coalesced over the warp), the grain's coarse values in shared memory; kc <= KQ vectors
template <bool MULTI>
__global__ void __launch_bounds__(256) k_prolong_grain_cm(const long long *node_off, const int *nloc,
                                                          const int *lnodes, const int *kg, const long long *cm_off,
                                                          const __nv_bfloat16 *Xc, const int *gcol_off,
                                                          const int *gcol, const double *u, long long No, double *z,
                                                          long long L, int kc) {
  constexpr int KQ = MULTI ? 8 : 1;
  __shared__ float ul[KQ][512];
  const int g = blockIdx.y;
  const int N = nloc[g], ld = cm_ld(N), k = kg[g];
  const int row0 = blockIdx.x * CM_ROWS;
  if (row0 >= ld) return;
  for (int e = threadIdx.x; e < KQ * k; e += blockDim.x) {
    const int q = e / k, a = e % k;
    ul[q][a] = q < kc ? (float)u[q * No + gcol[gcol_off[g] + a]] : 0.f;
  }
  __syncthreads();
  const int rs = row0 + 8 * threadIdx.x;
  if (rs >= ld) return;
  const __nv_bfloat16 *xr = Xc + cm_off[g] + rs;
  float acc[KQ][8];
#pragma unroll
  for (int q = 0; q < KQ; ++q)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[q][j] = 0.f;
  int a = 0;
  if (!MULTI) {
    for (; a + 3 < k; a += 4) {
      uint4 xv[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) xv[c] = __ldg(reinterpret_cast<const uint4 *>(xr + (long long)(a + c) * ld));
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        float x[8];
        bf8_to_f32(xv[c], x);
        const float uc = ul[0][a + c];
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[0][j] += x[j] * uc;
      }
    }
  }
  for (; a < k; ++a) {
    float x[8];
    bf8_to_f32(__ldg(reinterpret_cast<const uint4 *>(xr + (long long)a * ld)), x);
#pragma unroll
    for (int q = 0; q < KQ; ++q) {
      const float uq = ul[q][a];
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[q][j] += x[j] * uq;
    }
  }
  const int *ln = lnodes + node_off[g];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int row = rs + j;
    if (row >= N) break;
    const int o = row / 3, d = row - 3 * o;
    const long long dst = 3LL * ln[o] + d;
#pragma unroll
    for (int q = 0; q < KQ; ++q)
      if (q < kc) z[q * L + dst] = (double)acc[q][j];
  }
}

QAlg qalg(const hplmm_ctx *c) {
  return QAlg{c->opt.mortar_kind == HPLMM_MORTAR_ALGEBRAIC ? c->qblk.p : nullptr, c->qoff.p, c->col_off.p};
}

template <typename T>
Buf<T> &gal_buf(hplmm_ctx *c);
template <>
Buf<double> &gal_buf<double>(hplmm_ctx *c) { return c->gal64; }
template <>
Buf<float> &gal_buf<float>(hplmm_ctx *c) { return c->gal32; }

template <typename T>
T *panel_ptr(hplmm_ctx *c);
template <>
double *panel_ptr<double>(hplmm_ctx *c) { return c->X64.p; }
template <>
float *panel_ptr<float>(hplmm_ctx *c) { return c->X32.p; }

template <typename T>
void galerkin(hplmm_ctx *c, const Buf<int> &gbox, const std::vector<long long> &hgal, const Buf<long long> &gal_off,
              const Buf<int> &gcol_off, const Buf<int> &gcol, int maxvol) {
  cudaStream_t s = c->stream;
  int G = c->n_grains;
  Buf<T> &work = gal_buf<T>(c);
  // grains in batches whose P and Y on the node boxes fit the work budget (at least one grain per batch)
  long long most = 1;
  for (int g = 0; g < G; ++g) most = std::max(most, hgal[g + 1] - hgal[g]);
  const long long cap = std::max(most, std::min<long long>(hgal[G], GAL_WORK_ELEMS));
  work.alloc(2 * cap);
  const CoarseFactor &F = c->cf;
  CFView cv{F.erank.p, F.owner.p, F.fpos.p, F.m.p, F.P.p, F.rank.p, F.foff.p, F.ioff.p, F.F.p, c->status.p};
  Buf<int> tl;
  for (int g0 = 0; g0 < G;) {
    int g1 = g0 + 1;
    while (g1 < G && hgal[g1 + 1] - hgal[g0] <= cap) ++g1;
    const long long base = hgal[g0], tot = std::max<long long>(hgal[g1] - hgal[g0], 1);
    T *P = work.p, *Y = work.p + cap;
    HP_CUDA(cudaMemsetAsync(P, 0, sizeof(T) * tot, s));
    dim3 gf(grid_for(maxvol, 128), g1 - g0);
    k_gal_fill<T><<<gf, 128, 0, s>>>(gbox.p, gal_off.p, c->kg.p, c->grid_to_node.p, c->nx, c->ny, c->node_cls.p,
                                     c->iface_of_node.p, c->iface_slot.p, c->fixed.p, c->grains.box.p,
                                     c->grains.node_off.p, c->grains.lmap.p, c->panel_off.p, panel_ptr<T>(c),
                                     c->mortar_off.p, c->eta_off.p, c->eta.p, c->comp_mask.p, c->gi_off.p,
                                     c->gi_iface.p, c->gi_colbase.p, g0, base, P, qalg(c));
    HP_CHECK_LAUNCH();
    dim3 gy(maxvol, g1 - g0);
    k_gal_Y<T><<<gy, 128, 0, s>>>(gbox.p, gal_off.p, c->kg.p, c->vgrain.p, c->mask.p, c->E.p, c->nx, c->ny, c->nz,
                                  c->Kref.p, c->fixed.p, c->grid_to_node.p, g0, base, P, Y);
    HP_CHECK_LAUNCH();
    // output tiles: 128 x 256 on the tensor cores (each split along the box rows into enough pieces for
    // about four CTAs per SM over the batch), 32 x 32 on the CUDA cores
    const bool tensor = std::is_same<T, float>::value && c->opt.tensor_galerkin;
    const int ta = tensor ? 128 : 32, tb = tensor ? 256 : 32;
    std::vector<int> tiles;
    int ntile = 0;
    for (int g = g0; g < g1; ++g) ntile += ((c->h_kg[g] + ta - 1) / ta) * ((c->h_kg[g] + tb - 1) / tb);
    const int want = 4 * num_sms();
    for (int g = g0; g < g1; ++g) {
      int k = c->h_kg[g];
      const long long nch = ((hgal[g + 1] - hgal[g]) / std::max(k, 1) + 15) / 16;  // 16-row chunks of the box
      const int split = tensor ? (int)std::max<long long>(1, std::min<long long>(nch / 32, (want + ntile - 1) / std::max(ntile, 1))) : 1;
      for (int a0 = 0; a0 < k; a0 += ta)
        for (int b0 = 0; b0 < k; b0 += tb)
          for (int q = 0; q < split; ++q) {
            tiles.push_back(g);
            tiles.push_back(a0);
            tiles.push_back(b0);
            if (tensor) {
              tiles.push_back((int)(nch * q / split));
              tiles.push_back((int)(nch * (q + 1) / split));
            }
          }
    }
    if (!tiles.empty()) {
      HP_CUDA(cudaStreamSynchronize(s));  // the previous batch's tile list is still read until here
      tl.upload(tiles, s);
      if constexpr (std::is_same<T, float>::value) {
        if (tensor) {
          HP_CUDA(cudaFuncSetAttribute(k_gal_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SMEM_BYTES));
          k_gal_gemm_tc<<<(unsigned)(tiles.size() / 5), 128, tc::SMEM_BYTES, s>>>(
              tl.p, gbox.p, gal_off.p, c->kg.p, gcol_off.p, gcol.p, P, Y, base, cv, c->dense_ao ? c->Ao.p : nullptr,
              c->n_coarse, c->status.p);
          HP_CHECK_LAUNCH();
        }
      }
      if (!tensor) {
        k_gal_gemm<T><<<(unsigned)(tiles.size() / 3), 256, 0, s>>>(tl.p, gbox.p, gal_off.p, c->kg.p, gcol_off.p,
                                                                   gcol.p, P, Y, base, cv,
                                                                   c->dense_ao ? c->Ao.p : nullptr, c->n_coarse);
        HP_CHECK_LAUNCH();
      }
    }
    g0 = g1;
  }
  HP_CUDA(cudaStreamSynchronize(s));
  work.release();
}

}  // namespace

void coarse_rhs(hplmm_ctx *c, const double *b_corr) {
  cudaStream_t s = c->stream;
  int G = c->n_grains;
  bool f64 = c->opt.local_prec == HPLMM_FP64;
  // panels
  std::vector<long long> poff(G + 1, 0);
  for (int g = 0; g < G; ++g) poff[g + 1] = poff[g] + (long long)c->grains.h_n[g] * c->h_kg[g];
  c->h_panel_off = poff;
  c->panel_off.upload(poff, s);
  if (f64) {
    c->X64.alloc(std::max<long long>(poff[G], 1));
    c->X64.zero(s);
  } else {
    c->X32.alloc(std::max<long long>(poff[G], 1));
    c->X32.zero(s);
  }
  int maxn = 0, maxk = 0;
  for (int g = 0; g < G; ++g) {
    maxn = std::max(maxn, c->grains.h_n[g] / 3);
    maxk = std::max(maxk, c->h_kg[g]);
  }
  HP_REQUIRE(maxk <= 512, HPLMM_ERR_INVALID,
             "a grain couples to " + std::to_string(maxk) + " coarse columns (limit 512); use fewer mortars or larger grains");
  dim3 grid(grid_for(std::max(maxn, 1), 128), G);
  {
  ProfScope ps_rhs(c, HPLMM_PH_BASIS_RHS);
  if (f64)
    k_basis_rhs<double><<<grid, 128, 0, s>>>(G, c->grains.node_off.p, c->grains.n.p, c->grains.lnodes.p,
                                             c->row_ptr.p, c->col.p, c->val64.p, c->iface_of_node.p, c->iface_slot.p,
                                             c->iface_pair.p, c->mortar_off.p, c->eta_off.p, c->eta.p,
                                             c->comp_mask.p, c->gi_off.p, c->gi_iface.p, c->gi_colbase.p, c->kg.p,
                                             c->corr_col.p, c->panel_off.p, b_corr, c->opt.strict_two_grain, c->X64.p,
                                             qalg(c));
  else
    k_basis_rhs<float><<<grid, 128, 0, s>>>(G, c->grains.node_off.p, c->grains.n.p, c->grains.lnodes.p, c->row_ptr.p,
                                            c->col.p, c->val64.p, c->iface_of_node.p, c->iface_slot.p,
                                            c->iface_pair.p, c->mortar_off.p, c->eta_off.p, c->eta.p, c->comp_mask.p,
                                            c->gi_off.p, c->gi_iface.p, c->gi_colbase.p, c->kg.p, c->corr_col.p,
                                            c->panel_off.p, b_corr, c->opt.strict_two_grain, c->X32.p, qalg(c));
  HP_CHECK_LAUNCH();
  }
  if (!f64 && c->opt.basis_solver == HPLMM_BASIS_DIRECT && c->opt.keep_basis_rhs) {
    c->Xrhs.alloc(std::max<long long>(poff[G], 1));
    HP_CUDA(cudaMemcpyAsync(c->Xrhs.p, c->X32.p, sizeof(float) * poff[G], cudaMemcpyDeviceToDevice, s));
  } else if (f64 || c->opt.basis_solver == HPLMM_BASIS_DIRECT) {
    c->Xrhs.release();
  }
}

void coarse_basis_solve(hplmm_ctx *c) {
  // batched local solves (Eqs. col_pk, col_cg): X_g <- (A^g_g)^{-1} X_g, exactly by the banded factors, or by
  // block-Jacobi CG from a zero or a learned initial guess (FP32 locals only)
  c->bstats = hplmm_basis_stats{};
  if (c->opt.local_prec == HPLMM_FP64) {
    solve_local_multi_f64(c, c->grains, c->X64.p, c->panel_off, c->kg, c->h_kg);
  } else if (c->opt.basis_solver == HPLMM_BASIS_DIRECT) {
    solve_local_multi_f32(c, c->grains, c->X32.p, c->panel_off, c->kg, c->h_kg);
  } else {
    ProfScope ps_it(c, HPLMM_PH_BASIS_SOLVE);
    ws_pcg_basis(c, c->opt.basis_solver == HPLMM_BASIS_PCG_WARM);
  }
}

void coarse_finish(hplmm_ctx *c) {
  cudaStream_t s = c->stream;
  int G = c->n_grains;
  bool f64 = c->opt.local_prec == HPLMM_FP64;
  const std::vector<long long> &poff = c->h_panel_off;
  if (!f64 && c->opt.apply_prec == HPLMM_BF16) {
    // the apply's BF16 panels, column-major per grain with 16-byte aligned columns
    std::vector<long long> coff(G + 1, 0);
    int maxld = 8, maxk = 1;
    for (int g = 0; g < G; ++g) {
      coff[g + 1] = coff[g] + (long long)cm_ld(c->grains.h_n[g]) * c->h_kg[g];
      maxld = std::max(maxld, cm_ld(c->grains.h_n[g]));
      maxk = std::max(maxk, c->h_kg[g]);
    }
    c->h_panel_off_cm = coff;
    c->panel_off_cm.upload(coff, s);
    c->X16.alloc(std::max<long long>(coff[G], 8));
    k_panel_bf16_cm<<<dim3((maxld + 31) / 32, (maxk + 31) / 32, G), dim3(32, 8), 0, s>>>(
        c->grains.n.p, c->kg.p, c->panel_off.p, c->panel_off_cm.p, c->X32.p, c->X16.p);
    HP_CHECK_LAUNCH();
  } else {
    c->X16.release();
    c->panel_off_cm.release();
  }

  // global column of every local panel column
  std::vector<int> hgoff(G + 1, 0), hgcol;
  for (int g = 0; g < G; ++g) {
    for (int q = c->h_gi_off[g]; q < c->h_gi_off[g + 1]; ++q) {
      int ci = c->h_gi_iface[q];
      for (int col = c->h_col_off[ci]; col < c->h_col_off[ci + 1]; ++col) hgcol.push_back(col);
    }
    if (c->h_corr_col[g] >= 0) hgcol.push_back(c->h_corr_col[g]);
    hgoff[g + 1] = (int)hgcol.size();
  }
  if (hgcol.empty()) hgcol.push_back(0);
  c->gcol_off.upload(hgoff, s);
  c->gcol.upload(hgcol, s);

  // Galerkin product on each grain's node box
  Buf<int> vmin, vmax;
  vmin.alloc(3 * G);
  vmax.alloc(3 * G);
  vmin.fill_bytes(0x7f, s);
  vmax.fill_bytes(0x80, s);
  long long nv = (long long)c->nx * c->ny * c->nz;
  k_grain_vbox<<<grid_for(nv, 256), 256, 0, s>>>(c->vgrain.p, c->nx, c->ny, c->nz, vmin.p, vmax.p);
  HP_CHECK_LAUNCH();
  auto lo = vmin.download(s), hi = vmax.download(s);
  std::vector<int> hbox(6 * G, 0);
  std::vector<long long> hgal(G + 1, 0);
  int maxvol = 1;
  for (int g = 0; g < G; ++g) {
    int vol = 1;
    for (int a = 0; a < 3; ++a) {
      if (lo[3 * g + a] > hi[3 * g + a]) {
        hbox[6 * g + a] = 0;
        hbox[6 * g + 3 + a] = 0;
        vol = 0;
      } else {
        hbox[6 * g + a] = lo[3 * g + a];
        hbox[6 * g + 3 + a] = hi[3 * g + a] - lo[3 * g + a] + 2;
        vol *= hbox[6 * g + 3 + a];
      }
    }
    if (vol == 0)
      for (int a = 0; a < 3; ++a) hbox[6 * g + 3 + a] = 0;
    maxvol = std::max(maxvol, vol);
    hgal[g + 1] = hgal[g] + 3LL * vol * c->h_kg[g];
  }
  Buf<int> gbox;
  gbox.upload(hbox, s);
  Buf<long long> gal_off;
  gal_off.upload(hgal, s);
  long long No = c->n_coarse;
  // the dense A^o is kept only for inspection (hplmm_get_coarse_matrix) of small coarse spaces; the solver
  // uses the sparse factor
  c->dense_ao = No > 0 && No <= DENSE_COARSE_MAX;
  if (c->dense_ao) {
    c->Ao.alloc(No * No);
    c->Ao.zero(s);
  } else {
    c->Ao.release();
  }
  {
    ProfScope ps_sym(c, HPLMM_PH_COARSE_CHOL);
    cf_analyse(c, hbox);
  }
  {
    ProfScope ps_gal(c, HPLMM_PH_GALERKIN);
    if (f64)
      galerkin<double>(c, gbox, hgal, gal_off, c->gcol_off, c->gcol, maxvol);
    else
      galerkin<float>(c, gbox, hgal, gal_off, c->gcol_off, c->gcol, maxvol);
  }
  if (No > 0) {
    ProfScope ps_chol(c, HPLMM_PH_COARSE_CHOL);
    if (c->dense_ao) {
      k_symmetrize<<<grid_for(No * No, 256), 256, 0, s>>>(c->Ao.p, No, nullptr);
      HP_CHECK_LAUNCH();
    }
    cf_factor(c);
  }
  HP_CUDA(cudaStreamSynchronize(s));
  // BF16 form: after the Galerkin product (the last reader of the FP32 panels) the apply and the inspection
  // calls read only the BF16 copy; the FP32 panels stay only when the warm-start collection will read them
  // as training targets
  if (c->X16.p && !c->opt.keep_basis_rhs) c->X32.release();
}

void build_coarse(hplmm_ctx *c, const double *b_corr) {
  coarse_rhs(c, b_corr);
  coarse_basis_solve(c);
  coarse_finish(c);
}

void coarse_apply(hplmm_ctx *c, const double *r_pad, double *z_pad) {
  ProfScope ps(c, HPLMM_PH_APPLY_COARSE);
  cudaStream_t s = c->stream;
  long long No = c->n_coarse;
  int G = c->n_grains;
  bool f64 = c->opt.local_prec == HPLMM_FP64;
  HP_CUDA(cudaMemsetAsync(z_pad, 0, sizeof(double) * 3 * (size_t)c->n_nodes, s));
  if (No == 0) return;
  double *t = c->w_coarse_t.p;
  HP_CUDA(cudaMemsetAsync(t, 0, sizeof(double) * No, s));
  if (c->n_iface_nodes > 0) {
    k_restrict_iface<<<grid_for(c->n_iface_nodes, 128), 128, 0, s>>>(
        c->iface_nodes.p, c->iface_of_node.p, c->n_iface_nodes, c->iface_slot.p, c->mortar_off.p, c->eta_off.p,
        c->eta.p, c->comp_mask.p, c->col_off.p, c->fixed.p, r_pad, t, qalg(c));
    HP_CHECK_LAUNCH();
  }
  int nmax = 1;
  for (int g = 0; g < G; ++g) nmax = std::max(nmax, c->grains.h_n[g]);
  dim3 gr((nmax + RCHUNK - 1) / RCHUNK, G);
  const bool b16 = !f64 && c->opt.apply_prec == HPLMM_BF16;
  if (f64)
    k_restrict_grain<double, double><<<gr, 256, 0, s>>>(c->grains.node_off.p, c->grains.n.p, c->grains.lnodes.p,
                                                        c->kg.p, c->panel_off.p, c->X64.p, c->gcol_off.p, c->gcol.p,
                                                        r_pad, t);
  else if (b16)
    k_restrict_grain_cm<false><<<dim3((cm_ld(nmax) + CM_ROWS - 1) / CM_ROWS, G), 256, 0, s>>>(
        c->grains.node_off.p, c->grains.n.p, c->grains.lnodes.p, c->kg.p, c->panel_off_cm.p, c->X16.p,
        c->gcol_off.p, c->gcol.p, r_pad, 0, t, 0, 1);
  else
    k_restrict_grain<float, float><<<gr, 256, 0, s>>>(c->grains.node_off.p, c->grains.n.p, c->grains.lnodes.p,
                                                      c->kg.p, c->panel_off.p, c->X32.p, c->gcol_off.p, c->gcol.p,
                                                      r_pad, t);
  HP_CHECK_LAUNCH();
  // u = (A^o)^{-1} t by the sparse factor; the prolongation reads u
  double *u = c->w_coarse_u.p;
  cf_solve(c, t, c->w_coarse_y.p, u);
  t = u;
  dim3 gp(64, G);
  if (f64)
    k_prolong_grain<double, double><<<gp, 256, 0, s>>>(c->grains.node_off.p, c->grains.n.p, c->grains.lnodes.p,
                                                       c->kg.p, c->panel_off.p, c->X64.p, c->gcol_off.p, c->gcol.p, t,
                                                       z_pad);
  else if (b16)
    k_prolong_grain_cm<false><<<dim3((cm_ld(nmax) + CM_ROWS - 1) / CM_ROWS, G), 256, 0, s>>>(
        c->grains.node_off.p, c->grains.n.p, c->grains.lnodes.p, c->kg.p, c->panel_off_cm.p, c->X16.p,
        c->gcol_off.p, c->gcol.p, t, 0, z_pad, 0, 1);
  else
    k_prolong_grain<float, float><<<gp, 256, 0, s>>>(c->grains.node_off.p, c->grains.n.p, c->grains.lnodes.p,
                                                     c->kg.p, c->panel_off.p, c->X32.p, c->gcol_off.p, c->gcol.p, t,
                                                     z_pad);
  HP_CHECK_LAUNCH();
  if (c->n_iface_nodes > 0) {
    k_prolong_iface<<<grid_for(c->n_iface_nodes, 128), 128, 0, s>>>(
        c->iface_nodes.p, c->iface_of_node.p, c->n_iface_nodes, c->iface_slot.p, c->mortar_off.p, c->eta_off.p,
        c->eta.p, c->comp_mask.p, c->col_off.p, c->fixed.p, t, z_pad, qalg(c));
    HP_CHECK_LAUNCH();
  }
}

// M_G^{-1} for k vectors at stride L (Z_q = P_hat (A^o)^{-1} P_hat^T R_q): the basis panels are read once per
// group of eight vectors in the restriction and in the prolongation; the coarse solves run per vector
void coarse_apply_multi(hplmm_ctx *c, const double *R, double *Z, int k) {
  ProfScope ps(c, HPLMM_PH_APPLY_COARSE);
  cudaStream_t s = c->stream;
  const long long No = c->n_coarse, L = 3LL * c->n_nodes;
  const int G = c->n_grains;
  const bool f64 = c->opt.local_prec == HPLMM_FP64;
  const bool b16 = !f64 && c->opt.apply_prec == HPLMM_BF16;
  HP_CUDA(cudaMemsetAsync(Z, 0, sizeof(double) * L * k, s));
  if (No == 0) return;
  c->mw_ct.alloc((size_t)No * k);
  c->mw_cu.alloc((size_t)No * k);
  double *t = c->mw_ct.p, *u = c->mw_cu.p;
  HP_CUDA(cudaMemsetAsync(t, 0, sizeof(double) * No * k, s));
  int nmax = 1;
  for (int g = 0; g < G; ++g) nmax = std::max(nmax, c->grains.h_n[g]);
  for (int q0 = 0; q0 < k; q0 += 8) {
    const int kc = std::min(8, k - q0);
    dim3 gr((nmax + RCHUNK8 - 1) / RCHUNK8, G);
    if (f64)
      k_restrict_grain8<double, double><<<gr, 256, 0, s>>>(c->grains.node_off.p, c->grains.n.p, c->grains.lnodes.p,
                                                           c->kg.p, c->panel_off.p, c->X64.p, c->gcol_off.p,
                                                           c->gcol.p, R + q0 * L, L, t + q0 * No, No, kc);
    else if (b16)
      k_restrict_grain_cm<true><<<dim3((cm_ld(nmax) + CM_ROWS - 1) / CM_ROWS, G), 256, 0, s>>>(
          c->grains.node_off.p, c->grains.n.p, c->grains.lnodes.p, c->kg.p, c->panel_off_cm.p, c->X16.p,
          c->gcol_off.p, c->gcol.p, R + q0 * L, L, t + q0 * No, No, kc);
    else
      k_restrict_grain8<float, float><<<gr, 256, 0, s>>>(c->grains.node_off.p, c->grains.n.p, c->grains.lnodes.p,
                                                         c->kg.p, c->panel_off.p, c->X32.p, c->gcol_off.p, c->gcol.p,
                                                         R + q0 * L, L, t + q0 * No, No, kc);
    HP_CHECK_LAUNCH();
  }
  for (int q = 0; q < k; ++q) {
    if (c->n_iface_nodes > 0) {
      k_restrict_iface<<<grid_for(c->n_iface_nodes, 128), 128, 0, s>>>(
          c->iface_nodes.p, c->iface_of_node.p, c->n_iface_nodes, c->iface_slot.p, c->mortar_off.p, c->eta_off.p,
          c->eta.p, c->comp_mask.p, c->col_off.p, c->fixed.p, R + q * L, t + q * No, qalg(c));
      HP_CHECK_LAUNCH();
    }
    cf_solve(c, t + q * No, c->w_coarse_y.p, u + q * No);
  }
  for (int q0 = 0; q0 < k; q0 += 8) {
    const int kc = std::min(8, k - q0);
    dim3 gp(64, G);
    if (f64)
      k_prolong_grain8<double, double><<<gp, 256, 0, s>>>(c->grains.node_off.p, c->grains.n.p, c->grains.lnodes.p,
                                                          c->kg.p, c->panel_off.p, c->X64.p, c->gcol_off.p, c->gcol.p,
                                                          u + q0 * No, No, Z + q0 * L, L, kc);
    else if (b16)
      k_prolong_grain_cm<true><<<dim3((cm_ld(nmax) + CM_ROWS - 1) / CM_ROWS, G), 256, 0, s>>>(
          c->grains.node_off.p, c->grains.n.p, c->grains.lnodes.p, c->kg.p, c->panel_off_cm.p, c->X16.p,
          c->gcol_off.p, c->gcol.p, u + q0 * No, No, Z + q0 * L, L, kc);
    else
      k_prolong_grain8<float, float><<<gp, 256, 0, s>>>(c->grains.node_off.p, c->grains.n.p, c->grains.lnodes.p,
                                                        c->kg.p, c->panel_off.p, c->X32.p, c->gcol_off.p, c->gcol.p,
                                                        u + q0 * No, No, Z + q0 * L, L, kc);
    HP_CHECK_LAUNCH();
  }
  if (c->n_iface_nodes > 0)
    for (int q = 0; q < k; ++q) {
      k_prolong_iface<<<grid_for(c->n_iface_nodes, 128), 128, 0, s>>>(
          c->iface_nodes.p, c->iface_of_node.p, c->n_iface_nodes, c->iface_slot.p, c->mortar_off.p, c->eta_off.p,
          c->eta.p, c->comp_mask.p, c->col_off.p, c->fixed.p, u + q * No, Z + q * L, qalg(c));
      HP_CHECK_LAUNCH();
    }
}

void prolong_column(hplmm_ctx *c, long long col, double *out_pad) {
  cudaStream_t s = c->stream;
  long long No = c->n_coarse;
  int G = c->n_grains;
  bool f64 = c->opt.local_prec == HPLMM_FP64;
  HP_CUDA(cudaMemsetAsync(out_pad, 0, sizeof(double) * 3 * (size_t)c->n_nodes, s));
  double *u = c->w_coarse_u.p;
  HP_CUDA(cudaMemsetAsync(u, 0, sizeof(double) * No, s));
  double one = 1.0;
  HP_CUDA(cudaMemcpyAsync(u + col, &one, sizeof(double), cudaMemcpyHostToDevice, s));
  dim3 gp(64, G);
  int nmax = 1;
  for (int g = 0; g < G; ++g) nmax = std::max(nmax, c->grains.h_n[g]);
  if (f64)
    k_prolong_grain<double, double><<<gp, 256, 0, s>>>(c->grains.node_off.p, c->grains.n.p, c->grains.lnodes.p,
                                                       c->kg.p, c->panel_off.p, c->X64.p, c->gcol_off.p, c->gcol.p, u,
                                                       out_pad);
  else if (c->X16.p)
    k_prolong_grain_cm<false><<<dim3((cm_ld(nmax) + CM_ROWS - 1) / CM_ROWS, G), 256, 0, s>>>(
        c->grains.node_off.p, c->grains.n.p, c->grains.lnodes.p, c->kg.p, c->panel_off_cm.p, c->X16.p,
        c->gcol_off.p, c->gcol.p, u, 0, out_pad, 0, 1);
  else
    k_prolong_grain<float, float><<<gp, 256, 0, s>>>(c->grains.node_off.p, c->grains.n.p, c->grains.lnodes.p,
                                                     c->kg.p, c->panel_off.p, c->X32.p, c->gcol_off.p, c->gcol.p, u,
                                                     out_pad);
  HP_CHECK_LAUNCH();
  if (c->n_iface_nodes > 0) {
    k_prolong_iface<<<grid_for(c->n_iface_nodes, 128), 128, 0, s>>>(
        c->iface_nodes.p, c->iface_of_node.p, c->n_iface_nodes, c->iface_slot.p, c->mortar_off.p, c->eta_off.p,
        c->eta.p, c->comp_mask.p, c->col_off.p, c->fixed.p, u, out_pad, qalg(c));
    HP_CHECK_LAUNCH();
  }
  HP_CUDA(cudaStreamSynchronize(s));
}

}  // namespace hp
