// Local problems of the preconditioner: the grain-grid blocks A^{g_i}_{g_i}
// (Eqs. col_pk, col_cg and Mg_Mz) and the contact-grid blocks R A_hat E of
// Eq. Mg_Mz.  Each is a principal submatrix of A_hat, factorised once by an
// exact banded Cholesky (the paper precomputes exact local factorisations,
// Section 6.3) and then solved many times.
//
// Layout.  A problem's nodes are numbered in a permuted lexicographic order
// of its box (slowest axis = longest extent) which makes the matrix banded
// with half bandwidth bw.  The band is stored panel-blocked: panel p holds the
// NB columns [p*NB, p*NB+NB) and the NB+bw rows starting at p*NB, row-major,
// so every panel is one contiguous (NB+bw) x NB tile.  The inverse of each
// NB x NB diagonal factor block is stored beside it, turning the in-block
// triangular solves into small dense products.
#include "common.cuh"

#include <cuda_bf16.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <numeric>
#include <tuple>

namespace hp {

template <typename T> struct NBOf;
template <> struct NBOf<float> { static constexpr int v = 32; };
template <> struct NBOf<double> { static constexpr int v = 16; };

namespace {

constexpr int FACT_THREADS = 256;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// 16-byte asynchronous global->shared copies (cp.async), tracked per thread in commit groups
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// rank of this CTA in its cluster, and a barrier over every thread of the cluster with release/acquire
// ordering of the memory operations before and after it (not warp-aligned: lanes may be diverged)
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}
// the two halves of that barrier, for work in between
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire;" ::: "memory"); }
// wait until at most n of this thread's most recent cp.async groups are pending (n small, runtime)
__device__ __forceinline__ void cp_async_wait_pending(int n) {
  switch (n) {
    case 0: asm volatile("cp.async.wait_group 0;" ::: "memory"); break;
    case 1: asm volatile("cp.async.wait_group 1;" ::: "memory"); break;
    case 2: asm volatile("cp.async.wait_group 2;" ::: "memory"); break;
    case 3: asm volatile("cp.async.wait_group 3;" ::: "memory"); break;
    case 4: asm volatile("cp.async.wait_group 4;" ::: "memory"); break;
    case 5: asm volatile("cp.async.wait_group 5;" ::: "memory"); break;
    case 6: asm volatile("cp.async.wait_group 6;" ::: "memory"); break;
    default: asm volatile("cp.async.wait_group 7;" ::: "memory"); break;
  }
}


__device__ __forceinline__ long long panel_addr(int i, int j, int NB, int bw) {
  int p = j / NB, c = j - p * NB, r = i - p * NB;
  return (long long)p * (NB + bw) * NB + (long long)r * NB + c;
}

// box of problem k: lo[3], ext[3], perm[3] (perm[0] = fastest axis)
struct Box {
  int lo[3], ext[3], perm[3];
};

__device__ __forceinline__ Box load_box(const int *box, int k) {
  Box b;
  for (int a = 0; a < 3; ++a) {
    b.lo[a] = box[9 * k + a];
    b.ext[a] = box[9 * k + 3 + a];
    b.perm[a] = box[9 * k + 6 + a];
  }
  return b;
}

// cell index of grid point (x,y,z) in the box's permuted order, or -1 when outside
__device__ __forceinline__ int box_cell(const Box &b, int x, int y, int z) {
  int p[3] = {x - b.lo[0], y - b.lo[1], z - b.lo[2]};
  for (int a = 0; a < 3; ++a)
    if (p[a] < 0 || p[a] >= b.ext[a]) return -1;
  int f = b.perm[0], m = b.perm[1], s = b.perm[2];
  return (p[s] * b.ext[m] + p[m]) * b.ext[f] + p[f];
}

__device__ __forceinline__ void cell_xyz(const Box &b, int cell, int *xyz) {
  int f = b.perm[0], m = b.perm[1], s = b.perm[2];
  int pf = cell % b.ext[f];
  int t = cell / b.ext[f];
  int pm = t % b.ext[m];
  int ps = t / b.ext[m];
  int p[3];
  p[f] = pf;
  p[m] = pm;
  p[s] = ps;
  for (int a = 0; a < 3; ++a) xyz[a] = b.lo[a] + p[a];
}

// ---------------------------------------------------------------- boxes
__global__ void k_grain_bbox(const int *cls, const int *node_ijk, int n_nodes, int *bmin, int *bmax) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= n_nodes) return;
  int g = cls[n];
  if (g < 0) return;
  for (int a = 0; a < 3; ++a) {
    atomicMin(&bmin[3 * g + a], node_ijk[3 * n + a]);
    atomicMax(&bmax[3 * g + a], node_ijk[3 * n + a]);
  }
}

__global__ void k_iface_bbox(const int *iface_nodes, const int *iface_of_node, long long count, const int *node_ijk,
                             int *bmin, int *bmax) {
  long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= count) return;
  int n = iface_nodes[p];
  int c = iface_of_node[n];
  for (int a = 0; a < 3; ++a) {
    atomicMin(&bmin[3 * c + a], node_ijk[3 * n + a]);
    atomicMax(&bmax[3 * c + a], node_ijk[3 * n + a]);
  }
}

// mark the (2w+1)^3 neighbourhood of every interface node in its contact grid's box
__global__ void k_contact_mark(const int *iface_nodes, const int *iface_of_node, long long count, const int *node_ijk,
                               const int *box, const long long *node_off, int w, int *lmap) {
  long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= count) return;
  int n = iface_nodes[p];
  int c = iface_of_node[n];
  Box b = load_box(box, c);
  int x = node_ijk[3 * n], y = node_ijk[3 * n + 1], z = node_ijk[3 * n + 2];
  for (int dz = -w; dz <= w; ++dz)
    for (int dy = -w; dy <= w; ++dy)
      for (int dx = -w; dx <= w; ++dx) {
        int cell = box_cell(b, x + dx, y + dy, z + dz);
        if (cell >= 0) lmap[node_off[c] + cell] = 1;
      }
}

// one CTA per problem: enumerate member nodes in box order, assign ordinals
// kind 0: grain (member = interior node of grain k); kind 1: contact grid (member = marked, exists, free)
__global__ void k_local_enum(int kind, const int *box, const long long *node_off, int *lmap, int *lnodes, int *nloc,
                             const int *grid_to_node, int nx, int ny, const int *cls, const uint8_t *fixed) {
  __shared__ int warp_tot[32];
  __shared__ int running;
  int k = blockIdx.x;
  Box b = load_box(box, k);
  int vol = b.ext[0] * b.ext[1] * b.ext[2];
  long long off = node_off[k];
  if (threadIdx.x == 0) running = 0;
  __syncthreads();
  long long NX = nx + 1, NY = ny + 1;
  for (int base = 0; base < vol; base += blockDim.x) {
    int cell = base + threadIdx.x;
    int node = -1, member = 0;
    if (cell < vol) {
      int xyz[3];
      cell_xyz(b, cell, xyz);
      node = grid_to_node[((long long)xyz[2] * NY + xyz[1]) * NX + xyz[0]];
      if (node >= 0) {
        if (kind == 0) {
          member = cls[node] == k;
        } else {
          bool has_free = !fixed[3 * node] || !fixed[3 * node + 1] || !fixed[3 * node + 2];
          member = (lmap[off + cell] == 1) && has_free;
        }
      }
    }
    // block exclusive scan of member flags
    int v = member;
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = v;
    for (int o = 1; o < 32; o <<= 1) {
      int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      int nw = blockDim.x >> 5;
      int t = lane < nw ? warp_tot[lane] : 0;
      int s = t;
      for (int o = 1; o < 32; o <<= 1) {
        int u = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += u;
      }
      warp_tot[lane] = s - t;
    }
    __syncthreads();
    int excl = incl - v + warp_tot[wid] + running;
    if (cell < vol) {
      lmap[off + cell] = member ? excl : -1;
      if (member) lnodes[off + excl] = node;
    }
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) running = excl + v;
    __syncthreads();
  }
  if (threadIdx.x == 0) nloc[k] = 3 * running;
}

// half bandwidth: max |ord(n) - ord(m)| over coupled member pairs
__global__ void k_local_bw(const int *box, const long long *node_off, const int *nloc, const int *lmap,
                           const int *lnodes, const int *node_ijk, const int *row_ptr, const int *col, int *bw) {
  int k = blockIdx.x;
  Box b = load_box(box, k);
  long long off = node_off[k];
  int cnt = nloc[k] / 3;
  int best = 0;
  for (int o = threadIdx.x; o < cnt; o += blockDim.x) {
    int n = lnodes[off + o];
    for (int p = row_ptr[n]; p < row_ptr[n + 1]; ++p) {
      int m = col[p];
      int cell = box_cell(b, node_ijk[3 * m], node_ijk[3 * m + 1], node_ijk[3 * m + 2]);
      if (cell < 0) continue;
      int om = lmap[off + cell];
      if (om >= 0) best = max(best, abs(om - o));
    }
  }
  for (int o = 16; o > 0; o >>= 1) best = max(best, __shfl_down_sync(0xffffffffu, best, o));
  if ((threadIdx.x & 31) == 0) atomicMax(&bw[k], 3 * best + 2);
}

// scatter the lower band of the principal submatrix into panel-blocked storage
// global vector index of every local DOF: 3 * (global node of ordinal l / 3) + l mod 3
__global__ void k_local_gidx(const int *nloc, const long long *node_off, const long long *vec_off, const int *lnodes,
                             int *gidx) {
  const int k = blockIdx.x;
  const int n = nloc[k];
  const int *ln = lnodes + node_off[k];
  int *gk = gidx + vec_off[k];
  for (int l = threadIdx.x; l < n; l += blockDim.x) {
    const int o = l / 3;
    gk[l] = 3 * ln[o] + (l - 3 * o);
  }
}

template <typename T>
__global__ void k_local_extract(const int *box, const long long *node_off, const int *nloc, const int *bwv,
                                const long long *band_off, const int *lmap, const int *lnodes, const int *node_ijk,
                                const int *row_ptr, const int *col, const double *val, const uint8_t *fixed, T *band,
                                int NB, const int *plist, long long bbase) {
  int k = plist ? plist[blockIdx.x] : (int)blockIdx.x;
  Box b = load_box(box, k);
  long long off = node_off[k];
  int cnt = nloc[k] / 3;
  int bw = bwv[k];
  T *B = band + (band_off[k] - bbase);
  for (int o = threadIdx.x; o < cnt; o += blockDim.x) {
    int n = lnodes[off + o];
    for (int p = row_ptr[n]; p < row_ptr[n + 1]; ++p) {
      int m = col[p];
      int cell = box_cell(b, node_ijk[3 * m], node_ijk[3 * m + 1], node_ijk[3 * m + 2]);
      if (cell < 0) continue;
      int om = lmap[off + cell];
      if (om < 0 || om > o) continue;
      const double *v = val + (long long)p * 9;
      for (int d = 0; d < 3; ++d)
        for (int d2 = 0; d2 < 3; ++d2) {
          int i = 3 * o + d, j = 3 * om + d2;
          if (j > i) continue;
          B[panel_addr(i, j, NB, bw)] = (T)v[3 * d + d2];
        }
    }
    for (int d = 0; d < 3; ++d)
      if (fixed[3 * n + d]) {
        int i = 3 * o + d;
        B[panel_addr(i, i, NB, bw)] = (T)1.0;
      }
  }
}

// ---------------------------------------------------------------- factorisation
template <typename T>
__device__ __forceinline__ T dev_sqrt(T x);
template <>
__device__ __forceinline__ float dev_sqrt<float>(float x) { return sqrtf(x); }
template <>
__device__ __forceinline__ double dev_sqrt<double>(double x) { return sqrt(x); }

// persistent: each CTA takes problems from the cost-ordered queue
template <typename T, int NB>
__global__ void __launch_bounds__(FACT_THREADS) k_band_chol(const int *order, int count, int *queue,
                                                           const int *nloc, const int *bwv,
                                                           const long long *band_off, T *band, int *status,
                                                           int where) {
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr int LD = NB + (16 / sizeof(T));  // padded row stride
  T *P = reinterpret_cast<T *>(smraw);
  __shared__ T Dv[NB][NB + 1];
  __shared__ int s_job;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = FACT_THREADS / 32;
  for (;;) {
    if (threadIdx.x == 0) s_job = atomicAdd(queue, 1);
    __syncthreads();
    int job = s_job;
    __syncthreads();
    if (job >= count) return;
    int k = order[job];
    int N = nloc[k], bw = bwv[k];
    if (N == 0) continue;
    T *B = band + band_off[k];
    const int RP = NB + bw;
    for (int k0 = 0, p = 0; k0 < N; k0 += NB, ++p) {
      int nb = min(NB, N - k0);
      int R = min(N - k0, RP);
      T *Bp = B + (long long)p * RP * NB;
      // 1. load panel rows [0,R) into shared memory
      for (int e = threadIdx.x; e < R * NB; e += FACT_THREADS) {
        int r = e / NB, cc = e - r * NB;
        P[r * LD + cc] = Bp[e];
      }
      __syncthreads();
      // 2. factor the diagonal block (one warp), then invert it
      if (wid == 0) {
        for (int cc = 0; cc < nb; ++cc) {
          if (lane == 0) {
            T d = P[cc * LD + cc];
            if (!(d > (T)0)) {
              if (atomicCAS(status, 0, (int)HPLMM_ERR_SINGULAR) == 0) {
                status[1] = where;
                status[2] = k;
                status[3] = k0 + cc;
              }
              d = (T)1;
            }
            P[cc * LD + cc] = dev_sqrt<T>(d);
          }
          __syncwarp();
          T dd = P[cc * LD + cc];
          for (int r = cc + 1 + lane; r < nb; r += 32) P[r * LD + cc] /= dd;
          __syncwarp();
          for (int r = cc + 1 + lane; r < nb; r += 32) {
            T lr = P[r * LD + cc];
            for (int c2 = cc + 1; c2 <= r; ++c2) P[r * LD + c2] -= lr * P[c2 * LD + cc];
          }
          __syncwarp();
        }
        // zero the strict upper part and padding of the diagonal block
        for (int e = lane; e < NB * NB; e += 32) {
          int r = e / NB, cc = e % NB;
          if (cc > r || r >= nb || cc >= nb) P[r * LD + cc] = (T)0;
        }
        __syncwarp();
        // column j of inv(L_kk): solve L x = e_j (lane j)
        for (int j = lane; j < NB; j += 32) {
          for (int i = 0; i < NB; ++i) {
            T v;
            if (i < j || i >= nb || j >= nb) {
              v = (T)0;
            } else {
              T s = (i == j) ? (T)1 : (T)0;
              for (int q = j; q < i; ++q) s -= P[i * LD + q] * Dv[q][j];
              v = s / P[i * LD + i];
            }
            Dv[i][j] = v;
          }
        }
      }
      __syncthreads();
      // 3. L_panel = A_panel * inv(L_kk)^T for rows [nb, R)
      for (int r = nb + threadIdx.x; r < R; r += FACT_THREADS) {
        T out[NB];
#pragma unroll
        for (int cc = 0; cc < NB; ++cc) out[cc] = 0;
#pragma unroll
        for (int q = 0; q < NB; ++q) {
          T aq = P[r * LD + q];
          const volatile T *dcol = &Dv[0][q];
#pragma unroll
          for (int cc = q; cc < NB; ++cc) out[cc] += aq * dcol[cc * (NB + 1)];
        }
#pragma unroll
        for (int cc = 0; cc < NB; ++cc) P[r * LD + cc] = out[cc];
      }
      __syncthreads();
      // 4. write the panel back: inv(L_kk) in the diagonal rows (the solves only need the inverse), then L
      for (int e = threadIdx.x; e < NB * NB; e += FACT_THREADS) Bp[e] = Dv[e / NB][e % NB];
      for (int e = NB * NB + threadIdx.x; e < R * NB; e += FACT_THREADS) {
        int r = e / NB, cc = e - r * NB;
        Bp[e] = P[r * LD + cc];
      }
      // 5. trailing update of the (R-nb)^2 lower window: A[i][j] -= sum_c P[i][c] P[j][c].
      //    Warp tiles of 16 rows x 32 columns (lane = column), rows strided over warps.
      int Wn = R - nb;
      int nrt = (Wn + 15) / 16;
      int nct = (Wn + 31) / 32;
      int ntiles = 0;
      for (int tj = 0; tj < nct; ++tj) ntiles += max(0, nrt - 2 * tj);
      for (int t = wid; t < ntiles; t += nw) {
        // tile t -> (column tile tj, row tile ti), column-major over the lower window (ti >= 2 tj)
        int tj = 0, rem = t;
        while (rem >= nrt - 2 * tj) {
          rem -= nrt - 2 * tj;
          ++tj;
        }
        int ti = 2 * tj + rem;
        int jl = nb + tj * 32 + lane;
        T pj[NB];
#pragma unroll
        for (int cc = 0; cc < NB; ++cc) pj[cc] = (jl < R) ? P[jl * LD + cc] : (T)0;
        T acc[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          int il = nb + ti * 16 + q;
          int ir = il < R ? il : nb;  // rows past the window read a valid row; the result is discarded
          T s = 0;
#pragma unroll
          for (int cc = 0; cc < NB; ++cc) s += P[ir * LD + cc] * pj[cc];
          acc[q] = s;
        }
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          int il = nb + ti * 16 + q;
          if (il < R && jl < R && jl <= il) B[panel_addr(k0 + il, k0 + jl, NB, bw)] -= acc[q];
        }
      }
      __syncthreads();
    }
  }
}

// TF32 tensor-core helpers: round to TF32 (the value keeps the FP32 format with 13 low mantissa bits cleared),
// split x = hi + lo into two TF32 parts, and one m16n8k8 MMA with FP32 accumulation (d += a b)
__device__ __forceinline__ uint32_t tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ void split_tf32(float x, uint32_t &hi, uint32_t &lo) {
  hi = tf32_rna(x);
  lo = tf32_rna(x - __uint_as_float(hi));
}
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// FP32 banded Cholesky, one CTA per problem (persistent, problems taken from a cost-ordered queue).
// Per panel of NB = 32 columns:
//   1. the panel's rows [0, R) are loaded into shared memory (row stride 36 floats: rows start in
//      different 16-byte bank groups, so per-thread 16-byte row reads are conflict-free);
//   2. warp 0 factorises the 32x32 diagonal block with the rows held in registers (lane r = row r,
//      columns broadcast by shuffles) and forms inv(L_kk) column by column (lane j = column j);
//   3. every thread turns its rows of the sub-diagonal block into L rows: L_r = A_r inv(L_kk)^T;
//   4. the panel (inv(L_kk) in its first 32 rows, then the L rows) is written back;
//   5. the trailing update A_ij -= L_i . L_j of the (R-32)^2 lower window is done in 32x32 warp tiles on
//      the tensor cores (split-TF32 MMAs, FP32 accuracy), the tile's old values fetched into the warp's
//      staging area by cp.async before the arithmetic.
// CL = 2 (sets with at most half as many problems as SMs, where one SM per problem would leave most SMs
// idle): a cluster of two CTAs per problem.  Both CTAs load the panel and compute steps 2-3 (the same
// arithmetic on the same data, so the same values); rank 0 writes the panel back; the trailing tiles
// alternate between the two; a cluster barrier (release / acquire) ends each panel, so the next panel's
// loads, which read L2 only, see both CTAs' tile updates.  The factor is bit-identical to CL = 1.
constexpr int CHOL32_THREADS = 512;
// FP32 scratch of the staged BF16 set-up (floats): one chunk of local factors at a time
constexpr long long STAGE_ELEMS = 3LL << 29;
constexpr int CHOL32_LD = 36;
// row stride of a warp's staged 32x32 trailing tile: with 40 floats, the 8-byte pairs each lane reads in
// the MMA accumulator layout (row g8 (+8, +16), columns 2 tq, 2 tq + 1) fall on 32 distinct banks per
// half-warp, where a stride of 32 put 8 lanes on every bank
constexpr int CHOL32_CST_LD = 40;

template <int CL>
__global__ void __launch_bounds__(CHOL32_THREADS, 1) k_band_chol32(const int *order, int count, int *queue,
                                                                const int *nloc, const int *bwv,
                                                                const long long *band_off, float *band, int *status,
                                                                int where, int bwv_max, long long bbase) {
  constexpr int NB = 32, LD = CHOL32_LD;
  extern __shared__ __align__(16) unsigned char smraw[];
  float *P = reinterpret_cast<float *>(smraw);
  __shared__ __align__(16) float Lk[NB][LD];
  __shared__ __align__(16) float Dv[NB][LD];
  __shared__ int s_job;
  float *Cst = P + (size_t)(NB + bwv_max) * LD;  // per-warp 32x32 staging of the trailing tiles (row stride 40)
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = CHOL32_THREADS / 32;
  const int rank = CL == 2 ? (int)cluster_rank() : 0;
  for (int round = 0;; ++round) {
    int job;
    if constexpr (CL == 1) {
      if (threadIdx.x == 0) s_job = atomicAdd(queue, 1);
      __syncthreads();
      job = s_job;
      __syncthreads();
    } else {
      if (round > 0) return;
      job = blockIdx.x / CL;  // both CTAs of a cluster: the same problem, the same control flow
    }
    if (job >= count) return;
    const int k = order[job];
    const int N = nloc[k], bw = bwv[k];
    if (N == 0) continue;
    float *B = band + (band_off[k] - bbase);
    const int RP = NB + bw;
    for (int k0 = 0, p = 0; k0 < N; k0 += NB, ++p) {
      const int nb = min(NB, N - k0);
      const int R = min(N - k0, RP);
      float *Bp = B + (long long)p * RP * NB;
      // 1. load rows [0, R): 8 float4 per row
      {
        const float4 *src = reinterpret_cast<const float4 *>(Bp);
        const int n4 = R * 8;
        // the other CTA of a cluster updated some of these rows: read them from L2
        auto ld4 = [&](int i) { return CL == 2 ? __ldcg(src + i) : src[i]; };
        int e = threadIdx.x;
        for (; e + 3 * CHOL32_THREADS < n4; e += 4 * CHOL32_THREADS) {
          float4 v0 = ld4(e), v1 = ld4(e + CHOL32_THREADS), v2 = ld4(e + 2 * CHOL32_THREADS),
                 v3 = ld4(e + 3 * CHOL32_THREADS);
          *reinterpret_cast<float4 *>(P + (e >> 3) * LD + (e & 7) * 4) = v0;
          int e1 = e + CHOL32_THREADS, e2 = e + 2 * CHOL32_THREADS, e3 = e + 3 * CHOL32_THREADS;
          *reinterpret_cast<float4 *>(P + (e1 >> 3) * LD + (e1 & 7) * 4) = v1;
          *reinterpret_cast<float4 *>(P + (e2 >> 3) * LD + (e2 & 7) * 4) = v2;
          *reinterpret_cast<float4 *>(P + (e3 >> 3) * LD + (e3 & 7) * 4) = v3;
        }
        for (; e < n4; e += CHOL32_THREADS) *reinterpret_cast<float4 *>(P + (e >> 3) * LD + (e & 7) * 4) = ld4(e);
      }
      // this CTA has read the panel, which rank 0 overwrites in step 4 (the wait comes after steps 2-3)
      if constexpr (CL == 2) cluster_arrive();
      __syncthreads();
      // 2. diagonal block (warp 0)
      if (wid == 0) {
        const int r = lane;
        float a[NB];
#pragma unroll
        for (int c = 0; c < NB; ++c) a[c] = (r < nb && c < nb && c <= r) ? P[r * LD + c] : 0.f;
#pragma unroll
        for (int cc = 0; cc < NB; ++cc) {
          if (cc < nb) {
            float d = __shfl_sync(0xffffffffu, a[cc], cc);
            if (!(d > 0.f)) {
              if (lane == 0 && atomicCAS(status, 0, (int)HPLMM_ERR_SINGULAR) == 0) {
                status[1] = where;
                status[2] = k;
                status[3] = k0 + cc;
              }
              d = 1.f;
            }
            const float sd = sqrtf(d);
            const float l = (r > cc) ? a[cc] / sd : (r == cc ? sd : 0.f);
            a[cc] = l;
#pragma unroll
            for (int c2 = cc + 1; c2 < NB; ++c2) {
              const float l2 = __shfl_sync(0xffffffffu, l, c2);
              if (c2 <= r) a[c2] -= l * l2;
            }
          }
        }
        // L_kk rows to shared memory (identity on the padding rows, so the inverse stays defined)
#pragma unroll
        for (int c = 0; c < NB; ++c) Lk[r][c] = (r < nb) ? ((c <= r) ? a[c] : 0.f) : (c == r ? 1.f : 0.f);
        __syncwarp();
        // column j = lane of inv(L_kk): y_i = (delta_ij - sum_{q<i} L_iq y_q) / L_ii
        const int j = lane;
        float y[NB];
#pragma unroll
        for (int i = 0; i < NB; ++i) {
          float s = (i == j) ? 1.f : 0.f;
#pragma unroll
          for (int q = 0; q < i; ++q) s -= Lk[i][q] * y[q];
          y[i] = s / Lk[i][i];
        }
#pragma unroll
        for (int i = 0; i < NB; ++i) Dv[i][j] = (i < nb && j < nb) ? y[i] : 0.f;
      }
      __syncthreads();
      // 3. L rows of the sub-diagonal block: L_r[cc] = sum_{q <= cc} A_r[q] inv[cc][q] (row r is read into
      //    registers first, so each thread overwrites only its own row)
      for (int r = nb + threadIdx.x; r < R; r += CHOL32_THREADS) {
        float ar[NB];
#pragma unroll
        for (int g = 0; g < 8; ++g) {
          float4 t = *reinterpret_cast<const float4 *>(P + r * LD + 4 * g);
          ar[4 * g] = t.x; ar[4 * g + 1] = t.y; ar[4 * g + 2] = t.z; ar[4 * g + 3] = t.w;
        }
        // four columns per pass, stored as one 16-byte group (rows 144 bytes apart: 8 consecutive rows hit 8
        // distinct bank groups); the row's original values stay in registers
#pragma unroll 1
        for (int cg = 0; cg < NB / 4; ++cg) {
          float o[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int cc = 4 * cg + j;
            float s0 = 0.f, s1 = 0.f;
#pragma unroll
            for (int g = 0; g < 8; ++g) {
              if (4 * g <= cc) {
                float4 d = *reinterpret_cast<const float4 *>(&Dv[cc][4 * g]);
                s0 = fmaf(ar[4 * g], d.x, s0);
                s1 = fmaf(ar[4 * g + 1], d.y, s1);
                s0 = fmaf(ar[4 * g + 2], d.z, s0);
                s1 = fmaf(ar[4 * g + 3], d.w, s1);
              }
            }
            o[j] = s0 + s1;
          }
          *reinterpret_cast<float4 *>(P + r * LD + 4 * cg) = make_float4(o[0], o[1], o[2], o[3]);
        }
      }
      __syncthreads();
      // 4. write the panel back: inv(L_kk) in the first NB rows, then the L rows
      if constexpr (CL == 2) cluster_wait();
      if (rank == 0) {
        float4 *dst = reinterpret_cast<float4 *>(Bp);
        for (int e = threadIdx.x; e < R * 8; e += CHOL32_THREADS) {
          const int rr = e >> 3, g = e & 7;
          dst[e] = (rr < NB) ? *reinterpret_cast<const float4 *>(&Dv[rr][4 * g])
                             : *reinterpret_cast<const float4 *>(P + rr * LD + 4 * g);
        }
      }
      // 5. trailing update in 32x32 warp tiles over the lower window (column-major order of tiles); the
      //    tile's old values are fetched into the warp's staging area by cp.async before the arithmetic
      const int Wn = R - nb;
      const int nt = (Wn + 31) / 32;
      const int ntiles = nt * (nt + 1) / 2;
      float *cst = Cst + (size_t)wid * 32 * CHOL32_CST_LD;
      for (int t = wid * CL + rank; t < ntiles; t += nw * CL) {
        int tj = 0, rem = t;
        while (rem >= nt - tj) {
          rem -= nt - tj;
          ++tj;
        }
        const int ti = tj + rem;
        // window rows nb + ti*32 + q live in panel p+1+tj at row (ti - tj)*32 + q (here nb = NB)
        float *tile = B + (long long)(p + 1 + tj) * RP * NB + (long long)(ti - tj) * 32 * NB;
        const int rows_valid = min(32, R - (nb + ti * 32));
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int piece = u * 32 + lane;  // row piece >> 3, 16-byte group piece & 7
          if ((piece >> 3) < rows_valid) cp_async16(cst + (piece >> 3) * CHOL32_CST_LD + (piece & 7) * 4, tile + piece * 4);
        }
        cp_async_commit();
        // A_ij -= sum_k L_ik L_jk on the tensor cores: m16n8k8 TF32 products with each operand split into a
        // TF32 high part and a TF32 remainder (a b ~ a_lo b_hi + a_hi b_lo + a_hi b_hi), which keeps FP32
        // accuracy; FP32 accumulation.  Warp tile 32x32 = 2 (rows) x 4 (columns) MMA tiles, K = 32 in 4 steps.
        const int g8 = lane >> 2, tq = lane & 3;
        const int rbase = nb + ti * 32, cbase = nb + tj * 32;
        float acc[2][4][4];
#pragma unroll
        for (int mi = 0; mi < 2; ++mi)
#pragma unroll
          for (int ni = 0; ni < 4; ++ni)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[mi][ni][e] = 0.f;
#pragma unroll
        for (int k0 = 0; k0 < NB; k0 += 8) {
          uint32_t ahi[2][4], alo[2][4];
#pragma unroll
          for (int mi = 0; mi < 2; ++mi) {
            const int r0 = min(rbase + 16 * mi + g8, R - 1), r1 = min(rbase + 16 * mi + g8 + 8, R - 1);
            split_tf32(P[r0 * LD + k0 + tq], ahi[mi][0], alo[mi][0]);
            split_tf32(P[r1 * LD + k0 + tq], ahi[mi][1], alo[mi][1]);
            split_tf32(P[r0 * LD + k0 + tq + 4], ahi[mi][2], alo[mi][2]);
            split_tf32(P[r1 * LD + k0 + tq + 4], ahi[mi][3], alo[mi][3]);
          }
#pragma unroll
          for (int ni = 0; ni < 4; ++ni) {
            const int n = cbase + 8 * ni + g8;
            const bool nok = n < R;
            uint32_t bhi[2], blo[2];
            split_tf32(nok ? P[n * LD + k0 + tq] : 0.f, bhi[0], blo[0]);
            split_tf32(nok ? P[n * LD + k0 + tq + 4] : 0.f, bhi[1], blo[1]);
#pragma unroll
            for (int mi = 0; mi < 2; ++mi) {
              mma_tf32(acc[mi][ni], alo[mi], bhi);
              mma_tf32(acc[mi][ni], ahi[mi], blo);
              mma_tf32(acc[mi][ni], ahi[mi], bhi);
            }
          }
        }
        cp_async_wait_pending(0);
        __syncwarp();
        // accumulator element (mi, ni, 2h + e) is row 16 mi + g8 + 8 h, column 8 ni + 2 tq + e of the tile
#pragma unroll
        for (int mi = 0; mi < 2; ++mi)
#pragma unroll
          for (int ni = 0; ni < 4; ++ni)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const int q = 16 * mi + g8 + 8 * h, col0 = 8 * ni + 2 * tq;
              const float2 old = *reinterpret_cast<const float2 *>(cst + q * CHOL32_CST_LD + col0);
#pragma unroll
              for (int e = 0; e < 2; ++e) {
                const int col = col0 + e;
                const int il = rbase + q, jl = cbase + col;
                if (q < rows_valid && jl < R && jl <= il) tile[q * NB + col] = (e ? old.y : old.x) - acc[mi][ni][2 * h + e];
              }
            }
        __syncwarp();
      }
      if constexpr (CL == 2)
        cluster_sync_all();
      else
        __syncthreads();
    }
  }
}

// ---------------------------------------------------------------- multi-RHS solves
// One CTA per (problem, block of RB right-hand sides).  X holds the right-hand
// sides row-major (local DOF rows, ld columns) and is overwritten by the solution.
template <typename T, int NB>
__global__ void __launch_bounds__(256) k_band_solve_multi(const int *items, int n_items, const int *nloc,
                                                          const int *bwv, const long long *band_off,
                                                          const T *band, T *Xbase, const long long *x_off,
                                                          const int *x_ld) {
  constexpr int RB = 32;
  constexpr int CH = 32;  // panel rows staged per chunk
  __shared__ T Ds[NB][NB];
  __shared__ T Yb[NB][RB];
  __shared__ T Ps[CH][NB];
  __shared__ T red[8][NB][RB];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int it = blockIdx.x;
  if (it >= n_items) return;
  int k = items[2 * it], r0 = items[2 * it + 1];
  int N = nloc[k], bw = bwv[k];
  int ld = x_ld[k];
  int ncol = min(RB, ld - r0);
  const T *B = band + band_off[k];
  T *X = Xbase + x_off[k] + r0;
  const int RP = NB + bw;
  const int np = (N + NB - 1) / NB;
  bool colok = lane < ncol;
  // forward: L y = x
  for (int p = 0; p < np; ++p) {
    int k0 = p * NB, nb = min(NB, N - k0);
    for (int e = threadIdx.x; e < NB * NB; e += 256) Ds[e / NB][e % NB] = B[(long long)p * RP * NB + e];
    for (int q = wid; q < NB; q += 8) Yb[q][lane] = (q < nb && colok) ? X[(long long)(k0 + q) * ld + lane] : (T)0;
    __syncthreads();
    T y[NB / 8 + 1];
    {
      int qi = 0;
      for (int q = wid; q < NB; q += 8, ++qi) {
        T s = 0;
        for (int cc = 0; cc <= q; ++cc) s += Ds[q][cc] * Yb[cc][lane];
        y[qi] = s;
      }
    }
    __syncthreads();
    {
      int qi = 0;
      for (int q = wid; q < NB; q += 8, ++qi) {
        Yb[q][lane] = y[qi];
        if (q < nb && colok) X[(long long)(k0 + q) * ld + lane] = y[qi];
      }
    }
    __syncthreads();
    // window rows [k0+nb, min(N, k0+nb+bw)) -= Lpanel * Yb
    T yb[NB];
#pragma unroll
    for (int cc = 0; cc < NB; ++cc) yb[cc] = Yb[cc][lane];
    const T *Bp = B + (long long)p * RP * NB;
    int rend = min(N - k0, RP);
    for (int c0 = nb; c0 < rend; c0 += CH) {
      int cn = min(CH, rend - c0);
      for (int e = threadIdx.x; e < cn * NB; e += 256) Ps[e / NB][e % NB] = Bp[(long long)c0 * NB + e];
      __syncthreads();
      for (int r = wid; r < cn; r += 8) {
        T s = 0;
#pragma unroll
        for (int cc = 0; cc < NB; ++cc) s += Ps[r][cc] * yb[cc];
        if (colok) X[(long long)(k0 + c0 + r) * ld + lane] -= s;
      }
      __syncthreads();
    }
  }
  // backward: L^T x = y
  for (int p = np - 1; p >= 0; --p) {
    int k0 = p * NB, nb = min(NB, N - k0);
    for (int e = threadIdx.x; e < NB * NB; e += 256) Ds[e / NB][e % NB] = B[(long long)p * RP * NB + e];
    T acc[NB];
#pragma unroll
    for (int cc = 0; cc < NB; ++cc) acc[cc] = 0;
    const T *Bp = B + (long long)p * RP * NB;
    int rend = min(N - k0, RP);
    for (int c0 = nb; c0 < rend; c0 += CH) {
      int cn = min(CH, rend - c0);
      __syncthreads();
      for (int e = threadIdx.x; e < cn * NB; e += 256) Ps[e / NB][e % NB] = Bp[(long long)c0 * NB + e];
      __syncthreads();
      for (int r = wid; r < cn; r += 8) {
        T xv = colok ? X[(long long)(k0 + c0 + r) * ld + lane] : (T)0;
#pragma unroll
        for (int cc = 0; cc < NB; ++cc) acc[cc] += Ps[r][cc] * xv;
      }
    }
    __syncthreads();
#pragma unroll
    for (int cc = 0; cc < NB; ++cc) red[wid][cc][lane] = acc[cc];
    __syncthreads();
    for (int q = wid; q < NB; q += 8) {
      T s = 0;
      for (int w = 0; w < 8; ++w) s += red[w][q][lane];
      Yb[q][lane] = ((q < nb && colok) ? X[(long long)(k0 + q) * ld + lane] : (T)0) - s;
    }
    __syncthreads();
    for (int q = wid; q < NB; q += 8) {
      T s = 0;
      for (int cc = q; cc < NB; ++cc) s += Ds[cc][q] * Yb[cc][lane];
      if (q < nb && colok) X[(long long)(k0 + q) * ld + lane] = s;
    }
    __syncthreads();
  }
}

// FP32 multi-right-hand-side band solve, one CTA per (problem, block of 32 right-hand sides).
// The 32 right-hand-side columns of the rows inside the current band window live in a shared-memory ring
// (row i in slot i mod XR, XR >= RP + NB), so every row of X is read once and written once per sweep; the
// factor panels are streamed through a second ring in chunks of SM32_CH rows by cp.async (all threads,
// coalesced, two chunks ahead).  Per panel p (forward): Y = inv(L_pp) X_p, then X_r -= L_r Y for the window
// rows r (lane = right-hand side, its Y column in registers, the L row broadcast from shared memory).
// Backward: the window rows' column sums L_r^T X_r are accumulated per warp, reduced, and
// X_p = inv(L_pp)^T (Y_p - sum).  Rows leave the ring (written to global memory) when the window passes them.
constexpr int SM32_THREADS = 256;
constexpr int SM32_NW = SM32_THREADS / 32;
constexpr int SM32_CH = 128;  // factor rows per streamed chunk (16 KiB)
constexpr int SM32_STAGES = 3;

struct Multi32Ctx {
  const float *Bk;  // factor of the problem
  float *X;         // first right-hand-side column of the block, row stride ld
  float *Lring, *Xw;
  float (*red)[32][32];
  float (*Yb)[33];
  int N, RP, np, ld, XR;
  bool colok;
  int lane, wid;
  // chunk stream state
  int slot_issue, slot_use, ip, ic;
};

__device__ __forceinline__ int ring_slot(int i, int XR) { return i % XR; }

__device__ __forceinline__ int m32_panel_rows(const Multi32Ctx &m, int p) {
  return max(min(m.N - p * 32, m.RP), 32);
}
__device__ __forceinline__ int m32_nch(const Multi32Ctx &m, int p) {
  return (m32_panel_rows(m, p) + SM32_CH - 1) / SM32_CH;
}

template <int DIR>
__device__ __forceinline__ void m32_issue(Multi32Ctx &m) {
  if (m.ip >= 0 && m.ip < m.np) {
    const int p = m.ip;
    const int nc = m32_nch(m, p);
    const int c = DIR == 0 ? m.ic : ((m.ic + 1) % nc);  // backward: chunk 0 (inv(L_pp)) last
    const int rows = min(SM32_CH, m32_panel_rows(m, p) - c * SM32_CH);
    const float *src = m.Bk + ((long long)p * m.RP + (long long)c * SM32_CH) * 32;
    float *dst = m.Lring + (size_t)m.slot_issue * SM32_CH * 32;
    for (int piece = threadIdx.x; piece < rows * 8; piece += SM32_THREADS) cp_async16(dst + piece * 4, src + piece * 4);
    if (++m.ic >= nc) {
      m.ic = 0;
      m.ip += DIR == 0 ? 1 : -1;
    }
  }
  cp_async_commit();
  m.slot_issue = (m.slot_issue + 1) % SM32_STAGES;
}

__device__ __forceinline__ void m32_load_rows(const Multi32Ctx &m, int a, int b) {
  for (int i = a + m.wid; i < b; i += SM32_NW)
    m.Xw[(size_t)ring_slot(i, m.XR) * 32 + m.lane] = m.colok ? m.X[(long long)i * m.ld + m.lane] : 0.f;
}
__device__ __forceinline__ void m32_store_rows(const Multi32Ctx &m, int a, int b) {
  for (int i = a + m.wid; i < b; i += SM32_NW)
    if (m.colok) m.X[(long long)i * m.ld + m.lane] = m.Xw[(size_t)ring_slot(i, m.XR) * 32 + m.lane];
}

template <int DIR>
__device__ void m32_sweep(Multi32Ctx &m) {
  constexpr int NB = 32;
  const int lane = m.lane, wid = m.wid;
  m.slot_issue = 0;
  m.slot_use = 0;
  m.ip = DIR == 0 ? 0 : m.np - 1;
  m.ic = 0;
  for (int s = 0; s < SM32_STAGES - 1; ++s) m32_issue<DIR>(m);
  if (DIR == 0)
    m32_load_rows(m, 0, min(m.N, m.RP));
  else
    m32_load_rows(m, max(0, (m.np - 1) * NB), m.N);
  for (int p = DIR == 0 ? 0 : m.np - 1; DIR == 0 ? p < m.np : p >= 0; p += DIR == 0 ? 1 : -1) {
    const int k0 = p * NB, nb = min(NB, m.N - k0);
    const int R = min(m.N - k0, m.RP);
    const int nc = m32_nch(m, p);
    float vec[NB];  // forward: this lane's column of Y; backward: column sums of the window rows
#pragma unroll
    for (int e = 0; e < NB; ++e) vec[e] = 0.f;
    for (int cseq = 0; cseq < nc; ++cseq) {
      cp_async_wait_pending(SM32_STAGES - 2);
      __syncthreads();  // this chunk landed for every thread; the previous one is fully consumed
      m32_issue<DIR>(m);
      const int c = DIR == 0 ? cseq : ((cseq + 1) % nc);
      const float *Lc = m.Lring + (size_t)m.slot_use * SM32_CH * NB;
      m.slot_use = (m.slot_use + 1) % SM32_STAGES;
      const int row0 = c * SM32_CH;
      const int rows = min(SM32_CH, m32_panel_rows(m, p) - row0);
      if (DIR == 0 && c == 0) {
        // Y = inv(L_pp) X_p (row q of the block, lane = column); the ring slots of rows past the end of a
        // short last panel were never written (shared memory starts undefined), so they are masked rather
        // than multiplied by the zero columns of inv(L_pp)
        for (int q = wid; q < NB; q += SM32_NW) {
          float y = 0.f;
#pragma unroll
          for (int cc = 0; cc < NB; ++cc)
            if (cc < nb) y = fmaf(Lc[q * NB + cc], m.Xw[(size_t)ring_slot(k0 + cc, m.XR) * NB + lane], y);
          m.Yb[q][lane] = (q < nb) ? y : 0.f;
        }
        __syncthreads();
        for (int q = wid; q < nb; q += SM32_NW) m.Xw[(size_t)ring_slot(k0 + q, m.XR) * NB + lane] = m.Yb[q][lane];
#pragma unroll
        for (int cc = 0; cc < NB; ++cc) vec[cc] = m.Yb[cc][lane];
      }
      // window rows of this chunk, four per warp iteration (rows r + 8i; past the end clamped to row r and
      // masked), so that each warp has four independent rows of work in flight
      const int lo = max(row0, nb), hi = min(row0 + rows, R);
      int r = lo + wid;
      int slot = ring_slot(k0 + r, m.XR);  // advanced incrementally below
      for (; r < hi; r += 4 * SM32_NW) {
        const float *lr[4];
        float *xr[4];
        bool ok[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          ok[i] = r + i * SM32_NW < hi;
          int si = slot + i * SM32_NW;
          if (si >= m.XR) si -= m.XR;
          if (!ok[i]) si = slot;
          lr[i] = Lc + (size_t)((ok[i] ? r + i * SM32_NW : r) - row0) * NB;
          xr[i] = m.Xw + (size_t)si * NB + lane;
        }
        if (DIR == 0) {
          // X_r -= L_r . Y
          float acc[4][2];
#pragma unroll
          for (int i = 0; i < 4; ++i) acc[i][0] = acc[i][1] = 0.f;
#pragma unroll
          for (int g = 0; g < 8; ++g) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              const float4 l4 = *reinterpret_cast<const float4 *>(lr[i] + 4 * g);
              acc[i][0] = fmaf(l4.x, vec[4 * g], acc[i][0]);
              acc[i][1] = fmaf(l4.y, vec[4 * g + 1], acc[i][1]);
              acc[i][0] = fmaf(l4.z, vec[4 * g + 2], acc[i][0]);
              acc[i][1] = fmaf(l4.w, vec[4 * g + 3], acc[i][1]);
            }
          }
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const float xv = *xr[i];
            if (ok[i]) *xr[i] = xv - (acc[i][0] + acc[i][1]);
          }
        } else {
          // column sums L_r^T X_r, rows in ascending order
          float xv[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) xv[i] = ok[i] ? *xr[i] : 0.f;
#pragma unroll
          for (int g = 0; g < 8; ++g) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              const float4 l4 = *reinterpret_cast<const float4 *>(lr[i] + 4 * g);
              vec[4 * g] = fmaf(l4.x, xv[i], vec[4 * g]);
              vec[4 * g + 1] = fmaf(l4.y, xv[i], vec[4 * g + 1]);
              vec[4 * g + 2] = fmaf(l4.z, xv[i], vec[4 * g + 2]);
              vec[4 * g + 3] = fmaf(l4.w, xv[i], vec[4 * g + 3]);
            }
          }
        }
        slot += 4 * SM32_NW;
        while (slot >= m.XR) slot -= m.XR;
      }
      if (DIR == 1 && c == 0) {
        // finish the panel: t = Y_p - (sum over warps), X_p = inv(L_pp)^T t
#pragma unroll
        for (int e = 0; e < NB; ++e) m.red[wid][e][lane] = vec[e];
        __syncthreads();
        for (int q = wid; q < NB; q += SM32_NW) {
          float sum = 0.f;
#pragma unroll
          for (int w = 0; w < SM32_NW; ++w) sum += m.red[w][q][lane];
          m.Yb[q][lane] = (q < nb) ? m.Xw[(size_t)ring_slot(k0 + q, m.XR) * NB + lane] - sum : 0.f;
        }
        __syncthreads();
        for (int q = wid; q < nb; q += SM32_NW) {
          float xq = 0.f;
#pragma unroll
          for (int cc = 0; cc < NB; ++cc) xq = fmaf(Lc[cc * NB + q], m.Yb[cc][lane], xq);
          m.Xw[(size_t)ring_slot(k0 + q, m.XR) * NB + lane] = xq;
        }
      }
    }
    __syncthreads();
    // block p is final for this sweep; the next window's new rows come in
    m32_store_rows(m, k0, k0 + nb);
    if (DIR == 0) {
      if (p + 1 < m.np) m32_load_rows(m, min(m.N, k0 + m.RP), min(m.N, k0 + NB + m.RP));
    } else {
      if (p > 0) m32_load_rows(m, k0 - NB, k0);
    }
    __syncthreads();
  }
  cp_async_wait_pending(0);
  __syncthreads();
}

__global__ void __launch_bounds__(SM32_THREADS, 1) k_band_solve_multi32(const int *items, int n_items,
                                                                        const int *nloc, const int *bwv,
                                                                        const long long *band_off,
                                                                        const float *band, float *Xbase,
                                                                        const long long *x_off, const int *x_ld,
                                                                        int XR, long long bbase) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ float red[SM32_NW][32][32];
  __shared__ float Yb[32][33];
  const int it = blockIdx.x;
  if (it >= n_items) return;
  const int k = items[2 * it], r0 = items[2 * it + 1];
  const int N = nloc[k];
  if (N == 0) return;
  Multi32Ctx m;
  m.lane = threadIdx.x & 31;
  m.wid = threadIdx.x >> 5;
  m.N = N;
  m.RP = 32 + bwv[k];
  m.np = (N + 31) / 32;
  m.ld = x_ld[k];
  m.XR = XR;
  m.colok = m.lane < min(32, m.ld - r0);
  m.Bk = band + (band_off[k] - bbase);
  m.X = Xbase + x_off[k] + r0;
  m.Lring = reinterpret_cast<float *>(smraw);
  m.Xw = m.Lring + (size_t)SM32_STAGES * SM32_CH * 32;
  m.red = red;
  m.Yb = Yb;
  m32_sweep<0>(m);
  m32_sweep<1>(m);
}

// ---------------------------------------------------------------- single-RHS smoother solves
// One CTA, or a two-CTA cluster (below), per problem solves L L^T x = r for the gathered local right-hand
// side and adds (contact grids, which overlap) or stores (grain grids) x into z.
//
// Both sweeps run in steps, one per panel (forward: p = 0 .. np-1, backward: p = np-1 .. 0).  The work of a
// step is split between warps so that the short sequential chain of the triangular solve overlaps the
// bandwidth-heavy part:
//   - the leader warp handles the diagonal block of panel p and its "near" block (the next NB rows):
//       forward  y_p = inv(L_pp) (v_p - L_{p,p-1} y_{p-1}),   near product L_{p+1,p} y_p kept in registers;
//       backward x_p = inv(L_pp)^T (y_p - L_{p+1,p}^T x_{p+1} - far_p);
//   - the bulk warps handle the "far" rows (beyond the near block) of panel p-1, up to two rows per thread
//     per pass:
//       forward  v[rows] -= L_far(p-1) y_{p-1};
//       backward far_{p-1} = L_far(p-1)^T x[rows] (column sums reduced per warp);
//   - a producer warp streams the far rows of successive panels with bulk asynchronous copies
//     (cp.async.bulk) into a ring of shared-memory rows.  Chunks of up to `chunk_rows` rows are packed back
//     to back (a chunk that reaches the end of the ring is split into two copies), each guarded by a
//     full/empty mbarrier pair; a chunk is issued as soon as the rows it lands on have been released, so
//     the copies of the next one or two panels are in flight while a panel is consumed.
//   - a diagonal-chunk warp copies the leader's diagonal+near chunk of each step (2 NB rows) into a small
//     ring of its own with 16-byte cp.async (the load/store path), a few steps ahead; the leader never issues
//     or waits on a load on its chain: right-hand-side values, scratch values and output indices are fetched
//     one or two steps ahead.
// There is no per-step barrier: each role waits only for what it reads, through mbarriers.  Bulk step s
// needs leader step s-1 (y_{p-1}, or the x values above panel p-1).  In the forward sweep the rows of panel
// p are final once the first NB far rows of bulk step s-1 (warp 0 signals them as soon as its part of the
// first chunk is done) and all of bulk step s-2 are done, so the leader runs up to one step ahead of the
// bulk warps, and consecutive bulk steps may overlap (their updates of v are shared-memory atomics).  In
// the backward sweep the far sums of panel p come from bulk step s-1.  Every wait is bounded; on expiry
// the kernel records HPLMM_ERR_TIMEOUT, lets every copy in flight land and returns (z is then incomplete;
// the status tells the caller).
//
// Local vector window: only rows [p NB - 2 NB, p NB + RP + NB) of the local vector are live at step p, so
// shared memory holds a window of W >= RP + 3 NB rows (a power of two; row l lives in slot l mod W).  In the
// forward sweep the leader refills the slots of panel p-3 (last read by bulk step p-2) with the
// right-hand-side rows W further on (index and value fetched two and one steps ahead) and saves y_p to a
// global scratch
// vector; the backward sweep reads y_p back from there, keeps x in the window for the far products, and
// writes each x_p to z as soon as it is known.
//
// Two-CTA form (CL = 2, for sets with at most half as many problems as SMs): the cluster splits each
// panel's far rows, rank 0 (with the leader) the first part, at least 2 NB rows, rank 1 the rest.  Rank
// 1's rows then only update rows at least 4 NB below their panel, so it accumulates them in its own window
// and its pusher warp sends rank 0 the finished values of panel s+3 after its step s (forward), or, running
// one panel ahead in the backward sweep, the far sums of the panel it processed.  The leader sends y_p /
// x_p into rank 1's window.  Every exchange is NB values sent with st.async, completing its bytes on an
// mbarrier of the receiving CTA that an idle lane there arms (expected bytes) once the barrier's previous
// phase has completed; each side's waits on the other are therefore phase-exact, and a release-ordered
// remote arrive (which would keep its thread until the stores land) is never needed.
//
// Shared-memory bank conflicts: a factor row is 128 bytes (8 groups of 16 bytes).  A bulk thread visits its
// row's 16-byte groups starting at (thread mod 8), with its copy of y (or its column accumulators) kept in
// the same rotated order in registers; the 8 threads of one shared-memory phase therefore touch 8 different
// bank groups wherever the rows sit in the ring.
constexpr int WS_BULK_WARPS = 8;
constexpr int WS_THREADS = (3 + WS_BULK_WARPS) * 32;  // leader, far producer, diagonal-chunk producer, bulk
constexpr int WS_BULK_THREADS = WS_BULK_WARPS * 32;
// Factors are stored in S (float, double or bf16) and the arithmetic runs in T (double for FP64 factors,
// float otherwise); a stored row is NB elements of S, 128 bytes (FP32, FP64) or 64 bytes (BF16).
template <typename S> struct ComputeOf { using type = float; };
template <> struct ComputeOf<double> { using type = double; };
constexpr int WS_NSTG = 16;  // full/empty barrier pairs: far chunks in flight or buffered at once
constexpr int WS_MAX_C0 = 4;  // diagonal+near chunk stages (2 .. 4)
constexpr long long WAIT_CYCLES = 4000000000LL;  // about two seconds of SM clock


__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// potentially suspending probe of a phase: the thread sleeps until the phase completes or about
// MBAR_SUSPEND_NS nanoseconds pass, so that waiting warps leave their scheduler's issue slots to the warps
// that compute
constexpr uint32_t MBAR_SUSPEND_NS = 20000;
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.b32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity), "r"(MBAR_SUSPEND_NS)
      : "memory");
  return done != 0;
}

// the same with acquire semantics at cluster scope (phases completed by arrivals from the other CTA)
__device__ __forceinline__ bool mbar_try_wait_cluster(uint64_t *bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2, %3;\n"
      " selp.b32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity), "r"(MBAR_SUSPEND_NS)
      : "memory");
  return done != 0;
}

// bounded wait: gives up after `budget` SM cycles, or early when another warp has raised the abort flag.  The
// pipeline's waits take the caller's budget (options.wait_budget_us; about two seconds by default); the
// drains at the end (copies and remote stores still landing in this CTA's shared memory) always take
// WAIT_CYCLES, so that a CTA that gave up never leaves with data in flight towards it
template <bool CLUSTER = false>
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, const volatile int *abort_flag,
                                                  long long budget = WAIT_CYCLES) {
  const long long t0 = clock64();
  for (long long it = 0;; ++it) {
    if (CLUSTER ? mbar_try_wait_cluster(bar, parity) : mbar_try_wait(bar, parity)) return true;
    if ((it & 3) == 3) {
      if (abort_flag && *abort_flag) return false;
      if (clock64() - t0 > budget) return false;
    }
  }
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// ---- two-CTA clusters: shared-memory addresses in the other CTA, remote stores and arrivals
__device__ __forceinline__ uint32_t peer_addr(const void *p, uint32_t rank) {
  uint32_t a;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(a) : "r"(smem_u32(p)), "r"(rank));
  return a;
}
__device__ __forceinline__ void st_peer_u32(uint32_t addr, uint32_t v) {
  asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
// asynchronous store into the other CTA's shared memory that completes its bytes on an mbarrier there (the
// sender does not wait; the receiver sees the value once the barrier phase completes)
__device__ __forceinline__ void st_async_peer(uint32_t addr, float v, uint32_t bar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.f32 [%0], %1, [%2];" ::"r"(addr), "f"(v),
               "r"(bar)
               : "memory");
}
__device__ __forceinline__ void st_async_peer(uint32_t addr, double v, uint32_t bar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.f64 [%0], %1, [%2];" ::"r"(addr), "d"(v),
               "r"(bar)
               : "memory");
}
// 16-byte group loads of a stored factor row, converted to the compute type
template <typename S> struct Vec16;
template <> struct Vec16<float> {
  static __device__ __forceinline__ void load(const float *p, float *o) {
    float4 v = *reinterpret_cast<const float4 *>(p);
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
  }
};
template <> struct Vec16<double> {
  static __device__ __forceinline__ void load(const double *p, double *o) {
    double2 v = *reinterpret_cast<const double2 *>(p);
    o[0] = v.x; o[1] = v.y;
  }
};
template <> struct Vec16<__nv_bfloat16> {
  static __device__ __forceinline__ void load(const __nv_bfloat16 *p, float *o) {
    uint4 u = *reinterpret_cast<const uint4 *>(p);
    const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      o[2 * i] = __uint_as_float(w[i] << 16);             // element 2i (low half)
      o[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);  // element 2i+1 (high half)
    }
  }
};
template <typename S> __device__ __forceinline__ typename ComputeOf<S>::type ld_elem(const S *p) {
  return (typename ComputeOf<S>::type)(*p);
}
template <> __device__ __forceinline__ float ld_elem<__nv_bfloat16>(const __nv_bfloat16 *p) {
  return __bfloat162float(*p);
}

// geometry of panel p: rows of the panel inside the matrix, and its far rows [2 NB, rend)
struct PanelGeo {
  int N, NB, RP;
  __device__ int rend(int p) const { return min(N - p * NB, RP); }
  __device__ int nfar(int p) const { return max(0, rend(p) - 2 * NB); }
  __device__ int c0rows() const { return min(2 * NB, RP); }
};

// n consecutive compute-type values from shared memory with 16-byte loads (p 16-byte aligned)
template <typename T, int n> __device__ __forceinline__ void ld_vec(const T *p, T *o) {
  static_assert((n * sizeof(T)) % 16 == 0, "whole 16-byte groups");
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int u = 0; u < n / 4; ++u) {
      const float4 w = reinterpret_cast<const float4 *>(p)[u];
      o[4 * u] = w.x; o[4 * u + 1] = w.y; o[4 * u + 2] = w.z; o[4 * u + 3] = w.w;
    }
  } else {
#pragma unroll
    for (int u = 0; u < n / 2; ++u) {
      const double2 w = reinterpret_cast<const double2 *>(p)[u];
      o[2 * u] = w.x; o[2 * u + 1] = w.y;
    }
  }
}

template <typename S, int NB, int CL, int NBW>
__global__ void __launch_bounds__((3 + NBW) * 32, NBW == WS_BULK_WARPS ? 1 : NBW == 4 ? 2 : NBW == 2 ? 3 : 4) k_band_solve_ws(
    int count, const int *nloc, const int *bwv, const long long *band_off, const long long *vec_off,
    const int *gidx, const S *band, const double *r, double *z, typename ComputeOf<S>::type *yscr, int atomic,
    int ring_rows, int chunk_rows, int c0_stages, int wmask, int *status, long long wait_cycles) {
  using T = typename ComputeOf<S>::type;
  constexpr int ROWB = NB * (int)sizeof(S);  // bytes per stored row
  static_assert(ROWB == 128 || ROWB == 64, "factor rows are 128 or 64 bytes");
  constexpr int G = ROWB / 16;               // 16-byte groups per stored row
  constexpr int E = 16 / sizeof(S);          // elements per 16-byte group
  extern __shared__ __align__(128) unsigned char smdyn[];
  __shared__ __align__(8) uint64_t full_far[WS_NSTG], empty_far[WS_NSTG];
  __shared__ __align__(8) uint64_t full_c0[WS_MAX_C0], empty_c0[WS_MAX_C0];
  // step dependencies (rings of 4, event j on barrier j & 3): leader step done, first NB far rows of a bulk
  // step done (warp 0), bulk step done (every bulk warp)
  __shared__ __align__(8) uint64_t ydone[4], urg[4], bdone[4];
  // two-CTA form: rank 1's finished partial sums pushed to rank 0 (forward: the rows of panel t+3 after its
  // step t; backward: the far sums of the panel it processed), and rank 1's step-done barriers on rank 0
  __shared__ __align__(8) uint64_t pdone[4];
  __shared__ __align__(16) T v1push[5][NB];  // row 4: sink of steps with nothing to push
  __shared__ T red1[4][NB];
  // rank 1: bulk step done (every bulk warp) for its pusher warp, and its per-warp far sums (4 panels deep)
  __shared__ __align__(8) uint64_t r1done[4];
  __shared__ T red_r1[4][NBW][NB];
  __shared__ T red[2][NBW][NB];
  __shared__ __align__(16) T lbuf[NB];  // leader: the panel's right-hand side, broadcast to its lanes
  __shared__ volatile int s_abort;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int rank = (CL == 2) ? (int)cluster_rank() : 0;
  const int k = (CL == 2) ? (int)(blockIdx.x >> 1) : (int)blockIdx.x;
  if (k >= count) return;  // the same for both CTAs of a cluster
  const int N = nloc[k];
  if (N == 0) return;
  const int bw = bwv[k];
  const int RP = NB + bw;
  const int np = (N + NB - 1) / NB;
  const int W = wmask + 1;
  const PanelGeo geo{N, NB, RP};
  const S *B = band + band_off[k];
  // far rows of panel q: rank 0 takes [0, hsplit(q)), rank 1 [hsplit(q), nfar(q)).  Rank 1 gets rows only
  // when the panel has at least 4 NB far rows, and never fewer than 2 NB go to rank 0, so that rank 1's
  // updates reach rows at least 4 NB below their panel
  auto hsplit = [&](int q) {
    const int nf = geo.nfar(q);
    return (CL == 1 || nf < 4 * NB) ? nf : max(2 * NB, (nf / 2) & ~7);
  };
  auto my_lo = [&](int q) { return rank == 0 ? 0 : hsplit(q); };
  auto my_cnt = [&](int q) { return rank == 0 ? hsplit(q) : geo.nfar(q) - hsplit(q); };
  // panel whose far rows this CTA's bulk warps process at step s: p-1, and p-2 for rank 1 in the backward
  // sweep (its rows need only x values of panels p+2 and above, so it runs one panel ahead)
  auto bulk_q = [&](int s) {
    const bool fw = s < np;
    const int pp = fw ? s : (2 * np - 1 - s);
    return (rank == 1 && !fw) ? pp - 2 : pp - 1;
  };
  // far chunks: when a whole step's far rows of this CTA (at most slot_rows) fit twice in the ring, every step
  // is one copy into a slot of slot_rows rows (ring_eff a multiple of slot_rows: no copy is split);
  // otherwise chunks of chunk_rows rows packed back to back, a chunk that reaches the end of the ring split
  // into two copies
  const int nf_int = max(0, RP - 2 * NB);
  const int h_int = (CL == 1 || nf_int < 4 * NB) ? nf_int : max(2 * NB, (nf_int / 2) & ~7);
  const int slot_rows = rank == 0 ? max(h_int, min(nf_int, 4 * NB - 1)) : min(nf_int, nf_int - h_int + 8);
  const bool whole = chunk_rows >= slot_rows && slot_rows > 0 && ring_rows >= 2 * slot_rows;
  const int ring_eff = whole ? (ring_rows / slot_rows) * slot_rows : ring_rows;
  const int cr = whole ? slot_rows : chunk_rows;
  const int *gi = gidx + vec_off[k];
  T *ys = yscr + vec_off[k];
  S *ring = reinterpret_cast<S *>(smdyn);
  S *c0_ring = ring + (size_t)ring_rows * NB;
  T *v = reinterpret_cast<T *>(c0_ring + (size_t)c0_stages * 2 * NB * NB);
  const int c0rows = geo.c0rows();

  if (threadIdx.x == 0) {
    for (int i = 0; i < WS_NSTG; ++i) {
      mbar_init(&full_far[i], 1);
      mbar_init(&empty_far[i], NBW);
    }
    for (int i = 0; i < c0_stages; ++i) {
      mbar_init(&full_c0[i], 32);
      mbar_init(&empty_c0[i], 1);
    }
    for (int i = 0; i < 4; ++i) {
      // rank 0: the leader's local arrival; rank 1: its armer's arrival plus the leader's st.async bytes
      mbar_init(&ydone[i], 1);
      mbar_init(&urg[i], 1);
      mbar_init(&bdone[i], NBW);
      mbar_init(&pdone[i], 1);                   // rank 0: its armer's arrival plus the pusher's st.async bytes
      mbar_init(&r1done[i], NBW);
    }
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (rank == 0) {
    // initial window: rows 0 .. min(W, N) - 1 of the right-hand side (slots of rows >= N are never read)
    for (int l = threadIdx.x; l < min(W, N); l += ((3 + NBW) * 32)) v[l] = (T)r[gi[l]];
  } else {
    for (int l = threadIdx.x; l < W; l += ((3 + NBW) * 32)) v[l] = (T)0;  // rank 1 accumulates its own updates
  }
  if constexpr (CL == 2)
    cluster_sync_all();  // barriers initialised and windows set in both CTAs before any remote access
  else
    __syncthreads();
  const uint32_t peer = (uint32_t)(rank ^ 1);
  // the other CTA's window and step barriers, mapped once (shared::cluster addresses are linear in each CTA's
  // window, so a slot's address is the base plus its byte offset)
  const uint32_t peer_v = (CL == 2) ? peer_addr(v, peer) : 0u;
  const uint32_t peer_ydone = (CL == 2) ? peer_addr(&ydone[0], peer) : 0u;
  const uint32_t peer_pdone = (CL == 2) ? peer_addr(&pdone[0], peer) : 0u;
  const uint32_t peer_v1push = (CL == 2) ? peer_addr(&v1push[0][0], peer) : 0u;
  const uint32_t peer_red1 = (CL == 2) ? peer_addr(&red1[0][0], peer) : 0u;
  auto raise_abort = [&]() {
    s_abort = 1;
    if constexpr (CL == 2) st_peer_u32(peer_addr((const void *)&s_abort, peer), 1u);
  };

  const int nsteps = 2 * np;
  // two-CTA form: each step's exchange is NB values of T sent with st.async; the receiving CTA's armer
  // arms the step's barrier with those bytes once the barrier's previous phase (4 steps earlier) completed,
  // and finally waits for the last phases, so that no CTA exits with stores still arriving
  constexpr uint32_t XBYTES = NB * sizeof(T);
  auto armer = [&](uint64_t *bars) {
    bool ok = true;
    for (int j = 0; j < nsteps && ok; ++j) {
      if (j >= 4 && !mbar_wait_bounded<true>(&bars[j & 3], (uint32_t)(((j - 4) >> 2) & 1), &s_abort, wait_cycles)) ok = false;
      if (ok) mbar_expect_tx(&bars[j & 3], XBYTES);
    }
    if (!ok) {
      raise_abort();
      atomicCAS(status, 0, (int)HPLMM_ERR_TIMEOUT);
    }
    for (int j = max(0, nsteps - 4); j < nsteps; ++j)
      mbar_wait_bounded<true>(&bars[j & 3], (uint32_t)((j >> 2) & 1), nullptr);
  };
  if (CL == 2 && wid == 1 && lane == 1 && rank == 0) {
    armer(pdone);
  } else if (CL == 2 && wid == 2 && lane == 0 && rank == 1) {
    armer(ydone);
  } else if (wid == 1) {
    // ------------------------------------------------------------ producer
    // per step: the far rows of the bulk warps' panel
    if (lane == 0) {
      int start_tab[WS_NSTG];  // absolute ring row of each far chunk not yet known to be released
      int n = 0, rel = 0, abs_pos = 0;
      bool ok = true;
      for (int s = 0; s < nsteps && ok; ++s) {
        const int q = bulk_q(s);
        if (q < 0) continue;
        const int nf = my_cnt(q), lo = my_lo(q);
        for (int r0 = 0; r0 < nf; r0 += cr) {
          const int rows = min(cr, nf - r0);
          const int alloc = whole ? slot_rows : rows;
          // release (in order) every chunk whose barrier pair or ring rows this chunk reuses
          while (rel < n && (rel <= n - WS_NSTG || start_tab[rel % WS_NSTG] < abs_pos + alloc - ring_eff)) {
            if (!mbar_wait_bounded(&empty_far[rel % WS_NSTG], (uint32_t)((rel / WS_NSTG) & 1), &s_abort, wait_cycles)) {
              ok = false;
              break;
            }
            ++rel;
          }
          if (!ok) break;
          const int slot = n % WS_NSTG;
          start_tab[slot] = abs_pos;
          const int pos = abs_pos % ring_eff;
          const S *src = B + ((long long)q * RP + 2 * NB + lo + r0) * NB;
          const int first = min(rows, ring_eff - pos);
          mbar_expect_tx(&full_far[slot], (uint32_t)rows * (uint32_t)ROWB);
          bulk_g2s(ring + (size_t)pos * NB, src, (uint32_t)first * ROWB, &full_far[slot]);
          if (first < rows) bulk_g2s(ring, src + (size_t)first * NB, (uint32_t)(rows - first) * ROWB, &full_far[slot]);
          abs_pos += alloc;
          ++n;
        }
      }
      if (!ok) {
        raise_abort();
        atomicCAS(status, 0, (int)HPLMM_ERR_TIMEOUT);
      }
      // let every copy still in flight land before shared memory is released (no-op when all were consumed)
      for (int m = max(rel, n - WS_NSTG); m < n; ++m)
        mbar_wait_bounded(&full_far[m % WS_NSTG], (uint32_t)((m / WS_NSTG) & 1), nullptr);
    }
  } else if (wid == 2 && rank == 0) {
    // ------------------------------------------------------------ diagonal-chunk producer
    // per-thread 16-byte cp.async copies (the load/store path, leaving the bulk-copy engine to the far rows);
    // each lane's copies of a stage complete into the stage's full barrier (32 arrivals)
    for (int s = 0; s < nsteps; ++s) {
      const int p = (s < np) ? s : (2 * np - 1 - s);
      const int slot = s % c0_stages;
      if (s >= c0_stages && !mbar_wait_bounded(&empty_c0[slot], (uint32_t)((s / c0_stages - 1) & 1), &s_abort, wait_cycles)) {
        raise_abort();
        if (lane == 0) atomicCAS(status, 0, (int)HPLMM_ERR_TIMEOUT);
        break;
      }
      const unsigned char *src = reinterpret_cast<const unsigned char *>(B + (long long)p * RP * NB);
      unsigned char *dst = reinterpret_cast<unsigned char *>(c0_ring + (size_t)slot * 2 * NB * NB);
      for (int piece = lane; piece < c0rows * G; piece += 32) cp_async16(dst + piece * 16, src + piece * 16);
      asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(&full_c0[slot])) : "memory");
    }
    cp_async_wait_pending(0);
  } else if (wid == 0 && rank == 0) {
    // ------------------------------------------------------------ leader: diagonal and near blocks
    const int i = lane % NB;
    const bool own = lane < NB;  // lanes that own row i of the panel (all lanes for NB = 32)
    // rotation of the 16-byte groups of row i (distinct bank groups within each 8-lane phase)
    const int off = (G == 8) ? (i & 7) : ((i >> 1) & 3);
    // window refill of the forward sweep: at step p the slot of row (p - 3) NB + i (its last reader, bulk
    // step p - 2, has finished) takes row refill_row(p) = (p - 3) NB + W + i; its index is loaded two steps
    // and its value one step ahead
    auto refill_row = [&](int pp) { return (pp - 3) * NB + W + i; };
    int rg = -1;       // global index of refill_row(p + 1)
    double rv = 0.0;   // right-hand side of refill_row(p)
    if (own && refill_row(1) < N) rg = gi[refill_row(1)];
    T near = 0;
    T y_next = 0;      // backward: y of the panel of the next step
    int zg_next = -1;  // backward: global index of row i of the panel of the next step
    int fail = 0;
    for (int s = 0; s < nsteps; ++s) {
      const bool fwd = s < np;
      const int p = fwd ? s : (2 * np - 1 - s);
      const int k0 = p * NB, nb = min(NB, N - k0);
      // forward: the rows of panel p are final once the first NB far rows of bulk step s-1 and all of bulk
      // step s-2 are done; backward: the far sums of panel p come from bulk step s-1
      // two-CTA form: rank 1's part of panel p's rows (forward, pushed after its step s-3) or of panel p's far
      // sums (backward, pushed after its step s-2)
      if (fwd) {
        if (s >= 1 && !mbar_wait_bounded(&urg[(s - 1) & 3], (uint32_t)(((s - 1) >> 2) & 1), &s_abort, wait_cycles)) fail = 1;
        if (s >= 2 && !fail && !mbar_wait_bounded(&bdone[(s - 2) & 3], (uint32_t)(((s - 2) >> 2) & 1), &s_abort, wait_cycles))
          fail = 1;
        if (CL == 2 && p >= 3 && !fail &&
            !mbar_wait_bounded<true>(&pdone[(s - 3) & 3], (uint32_t)(((s - 3) >> 2) & 1), &s_abort, wait_cycles))
          fail = 1;
      } else {
        if (!mbar_wait_bounded(&bdone[(s - 1) & 3], (uint32_t)(((s - 1) >> 2) & 1), &s_abort, wait_cycles)) fail = 1;
        // (waited at every backward step: each completed phase frees its barrier for the bytes 4 steps later)
        if (CL == 2 && s >= 2 && !fail &&
            !mbar_wait_bounded<true>(&pdone[(s - 2) & 3], (uint32_t)(((s - 2) >> 2) & 1), &s_abort, wait_cycles))
          fail = 1;
      }
      if (fwd && !fail) {
        if (p >= 3 && own && refill_row(p) < N) v[refill_row(p) & wmask] = (T)rv;
        rv = (rg >= 0) ? r[rg] : 0.0;
        rg = -1;
        if (own && refill_row(p + 2) < N) rg = gi[refill_row(p + 2)];
      }
      const int slot = s % c0_stages;
      if (!fail && !mbar_wait_bounded(&full_c0[slot], (uint32_t)((s / c0_stages) & 1), &s_abort, wait_cycles)) fail = 1;
      if (!fail) {
        const S *c0 = c0_ring + (size_t)slot * 2 * NB * NB;
        if (fwd) {
          // y_p = inv(L_pp) x with x = v_p - near (row i of inv(L_pp) against x broadcast from shared memory)
          T vin = (lane < nb) ? v[(k0 + lane) & wmask] : (T)0;
          if (CL == 2 && p >= 3 && lane < nb) vin += v1push[p & 3][i];
          const T x = (lane < nb) ? vin - near : (T)0;
          if (own) lbuf[i] = x;
          __syncwarp();
          T a0 = 0, a1 = 0;
#pragma unroll
          for (int g = 0; g < G; ++g) {
            const int gg = (g + off) % G;
            T cf[E], xv[E];
            Vec16<S>::load(c0 + i * NB + gg * E, cf);
            ld_vec<T, E>(lbuf + gg * E, xv);
#pragma unroll
            for (int e = 0; e < E; ++e) (g & 1 ? a1 : a0) += cf[e] * xv[e];
          }
          T y = (lane < nb) ? a0 + a1 : (T)0;
          if (own) {
            v[(k0 + i) & wmask] = y;  // read by the bulk warps at the next step and by the near product
            if constexpr (CL == 2)
              st_async_peer(peer_v + (uint32_t)(((k0 + i) & wmask) * sizeof(T)), y, peer_ydone + 8u * (s & 3));
            if (lane < nb) ys[k0 + i] = y;
          }
          __syncwarp();
          // near product for the next block (rows NB .. c0rows of the chunk; the rest were not copied, their
          // coefficients are taken as zero)
          const bool nvalid = NB + i < c0rows;
          T b0 = 0, b1 = 0;
#pragma unroll
          for (int g = 0; g < G; ++g) {
            const int gg = (g + off) % G;
            T cf[E], yv[E];
            Vec16<S>::load(c0 + (NB + i) * NB + gg * E, cf);
            ld_vec<T, E>(v + ((k0 + gg * E) & wmask), yv);
#pragma unroll
            for (int e = 0; e < E; ++e) (g & 1 ? b1 : b0) += cf[e] * yv[e];
          }
          near = nvalid ? b0 + b1 : (T)0;
          if (p == np - 1) {
            // the backward sweep starts with this panel
            y_next = y;
            zg_next = -1;
            if (lane < nb) zg_next = gi[k0 + i];
          }
        } else {
          const T yv = y_next;
          const int zg = zg_next;
          if (p > 0) {
            y_next = own ? ys[k0 - NB + i] : (T)0;
            zg_next = -1;
            if (own) zg_next = gi[k0 - NB + i];
          }
          // far partial sums of panel p (bulk warps computed them in the previous step)
          T far = 0;
          if (p + 1 < np) {
#pragma unroll
            for (int w = 0; w < NBW; ++w) far += red[p & 1][w][i];
          }
          if (CL == 2 && p <= np - 3) far += red1[p & 3][i];
          // near: L_{p+1,p}^T x_{p+1} (column i of the near block; rows past the matrix contribute nothing)
          const int nrows = min(c0rows - NB, N - k0 - NB);
          T n0 = 0, n1 = 0;
          if (nrows > 0) {
            const T *xn = v + ((k0 + NB) & wmask);
#pragma unroll
            for (int g = 0; g < NB / (16 / (int)sizeof(T)); ++g) {
              constexpr int ET = 16 / sizeof(T);
              T xv[ET];
              ld_vec<T, ET>(xn + g * ET, xv);
#pragma unroll
              for (int e = 0; e < ET; ++e) {
                const int rr = g * ET + e;
                const T c = ld_elem(c0 + (NB + rr) * NB + i);
                if (rr < nrows) (e & 1 ? n1 : n0) += c * xv[e];
              }
            }
          }
          const T t = (lane < nb) ? yv - far - (n0 + n1) : (T)0;
          if (own) lbuf[i] = t;
          __syncwarp();
          // x_p = inv(L_pp)^T t (column i of inv(L_pp) against t broadcast from shared memory)
          T a0 = 0, a1 = 0;
#pragma unroll
          for (int g = 0; g < NB / (16 / (int)sizeof(T)); ++g) {
            constexpr int ET = 16 / sizeof(T);
            T tv[ET];
            ld_vec<T, ET>(lbuf + g * ET, tv);
#pragma unroll
            for (int e = 0; e < ET; ++e) (e & 1 ? a1 : a0) += ld_elem(c0 + (g * ET + e) * NB + i) * tv[e];
          }
          const T x = a0 + a1;
          // rank 1 receives a full panel every step (zeros past the matrix, in slots it never reads)
          if (CL == 2 && own)
            st_async_peer(peer_v + (uint32_t)(((k0 + i) & wmask) * sizeof(T)), lane < nb ? x : (T)0,
                          peer_ydone + 8u * (s & 3));
          if (lane < nb) {
            v[(k0 + i) & wmask] = x;
            if (atomic)
              atomicAdd(&z[zg], (double)x);
            else
              z[zg] = (double)x;
          }
        }
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(&empty_c0[slot]);
          mbar_arrive(&ydone[s & 3]);
        }
      }
      if (fail) {
        raise_abort();
        if (lane == 0) atomicCAS(status, 0, (int)HPLMM_ERR_TIMEOUT);
        break;
      }
    }
  } else if (CL == 2 && wid == 0 && rank == 1) {
    // ------------------------------------------------------------ rank 1: pusher
    // after rank 1's bulk warps finished step s it pushes to rank 0 (forward: the rows of panel s+3, final
    // now; backward: the far sums of panel q), clears the window slots of panel q (read as y_q for the last
    // time) and releases the step, one arrival per lane; the bulk warps meanwhile go on with later steps
    for (int s = 0; s < nsteps; ++s) {
      if (!mbar_wait_bounded(&r1done[s & 3], (uint32_t)((s >> 2) & 1), &s_abort, wait_cycles)) {
        raise_abort();
        if (lane == 0) atomicCAS(status, 0, (int)HPLMM_ERR_TIMEOUT);
        break;
      }
      const int q = bulk_q(s);
      // NB values every step (to the sink row when there is nothing to push)
      uint32_t dst = peer_v1push + 4u * NB * sizeof(T);
      T val = 0;
      if (s < np) {
        if (s + 3 < np) {
          dst = peer_v1push + (uint32_t)(((s + 3) & 3) * NB * sizeof(T));
          val = lane < NB ? v[((s + 3) * NB + lane) & wmask] : (T)0;
        }
        if (q >= 0 && lane < NB) v[(q * NB + lane) & wmask] = (T)0;
      } else if (q >= 0) {
        dst = peer_red1 + (uint32_t)((q & 3) * NB * sizeof(T));
        if (lane < NB) {
#pragma unroll
          for (int w = 0; w < NBW; ++w) val += red_r1[q & 3][w][lane];
        }
      }
      if (lane < NB) st_async_peer(dst + (uint32_t)(lane * sizeof(T)), val, peer_pdone + 8u * (s & 3));
    }
  } else if (wid >= 3) {
    // ------------------------------------------------------------ bulk: far rows of panel bulk_q(s)
    const int bw_id = wid - 3;
    const int tb = threadIdx.x - 96;
    // rotation of this thread's group order: rows of 8 groups use (thread mod 8); rows of 4 groups use
    // ((thread / 2) mod 4), which again spreads 8 consecutive rows over 8 distinct 16-byte bank groups
    const int off = (G == 8) ? (tb & 7) : ((tb >> 1) & 3);
    int n = 0, pos = 0;  // chunk sequence number and ring row of the next chunk
    int fail = 0;
    for (int s = 0; s < nsteps && !fail; ++s) {
      const bool fwd = s < np;
      const int q = bulk_q(s);
      bool urgent_pending = (bw_id == 0 && rank == 0);  // rank 0's warp 0 owns far rows 0 .. 31
      // y_q (forward) or the x values above panel q (backward) come from leader step s-1; rank 1 in the
      // backward sweep needs only leader step s-2
      {
        const int dep = (rank == 1 && !fwd) ? s - 2 : s - 1;
        if (dep >= 0) {
          const bool okw = rank == 0
                               ? mbar_wait_bounded(&ydone[dep & 3], (uint32_t)((dep >> 2) & 1), &s_abort, wait_cycles)
                               : mbar_wait_bounded<true>(&ydone[dep & 3], (uint32_t)((dep >> 2) & 1), &s_abort, wait_cycles);
          if (!okw) fail = 1;
        }
      }
      if (q >= 0 && !fail) {
        const int kq = q * NB;
        const int nf = my_cnt(q), lo = my_lo(q);
        T acc[NB];
        T yr[NB];
        if (fwd) {
          // y_{q} in rotated group order
#pragma unroll
          for (int g = 0; g < G; ++g) ld_vec<T, E>(v + ((kq + ((g + off) % G) * E) & wmask), yr + g * E);
        } else {
#pragma unroll
          for (int e = 0; e < NB; ++e) acc[e] = 0;
        }
        for (int r0 = 0; r0 < nf; r0 += cr) {
          const int rows = min(cr, nf - r0);
          const int slot = n % WS_NSTG;
          if (!fail && !mbar_wait_bounded(&full_far[slot], (uint32_t)((n / WS_NSTG) & 1), &s_abort, wait_cycles)) fail = 1;
          if (!fail) {
            // two rows per thread per pass (t and t + (NBW * 32)); the choice between the one- and the
            // two-row code is made per warp (a lane without a second row re-reads its first row, with no
            // update or a zero weight), so that no warp runs both
            for (int t = tb; t < rows; t += 2 * (NBW * 32)) {
              const int t2 = t + (NBW * 32);
              const bool two = t2 < rows;
              const bool warp_two = __any_sync(__activemask(), two);
              int rs = pos + t, rs2 = pos + t2;
              if (rs >= ring_eff) rs -= ring_eff;
              if (rs2 >= ring_eff) rs2 -= ring_eff;
              const S *row = ring + (size_t)rs * NB;
              const S *row2 = ring + (size_t)(two ? rs2 : rs) * NB;
              const int vrow = (kq + 2 * NB + lo + r0 + t) & wmask;
              const int vrow2 = (kq + 2 * NB + lo + r0 + t2) & wmask;
              // forward updates use shared-memory atomics: consecutive bulk steps may overlap on a row
              if (fwd) {
                if (warp_two) {
                  T s0 = 0, s1 = 0, s2 = 0, s3 = 0;
#pragma unroll
                  for (int g = 0; g < G; g += 2) {
                    T ra[E], rb[E], rc[E], rd[E];
                    Vec16<S>::load(row + ((g + off) % G) * E, ra);
                    Vec16<S>::load(row + ((g + 1 + off) % G) * E, rb);
                    Vec16<S>::load(row2 + ((g + off) % G) * E, rc);
                    Vec16<S>::load(row2 + ((g + 1 + off) % G) * E, rd);
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                      s0 += ra[e] * yr[g * E + e];
                      s1 += rb[e] * yr[(g + 1) * E + e];
                      s2 += rc[e] * yr[g * E + e];
                      s3 += rd[e] * yr[(g + 1) * E + e];
                    }
                  }
                  atomicAdd(&v[vrow], -(s0 + s1));
                  if (two) atomicAdd(&v[vrow2], -(s2 + s3));
                } else {
                  T s0 = 0, s1 = 0;
#pragma unroll
                  for (int g = 0; g < G; g += 2) {
                    T ra[E], rb[E];
                    Vec16<S>::load(row + ((g + off) % G) * E, ra);
                    Vec16<S>::load(row + ((g + 1 + off) % G) * E, rb);
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                      s0 += ra[e] * yr[g * E + e];
                      s1 += rb[e] * yr[(g + 1) * E + e];
                    }
                  }
                  atomicAdd(&v[vrow], -(s0 + s1));
                }
              } else {
                const T xv = v[vrow];
                if (warp_two) {
                  const T xv2 = two ? v[vrow2] : (T)0;
#pragma unroll
                  for (int g = 0; g < G; ++g) {
                    T ra[E], rc[E];
                    Vec16<S>::load(row + ((g + off) % G) * E, ra);
                    Vec16<S>::load(row2 + ((g + off) % G) * E, rc);
#pragma unroll
                    for (int e = 0; e < E; ++e) acc[g * E + e] += ra[e] * xv + rc[e] * xv2;
                  }
                } else {
#pragma unroll
                  for (int g = 0; g < G; ++g) {
                    T ra[E];
                    Vec16<S>::load(row + ((g + off) % G) * E, ra);
#pragma unroll
                    for (int e = 0; e < E; ++e) acc[g * E + e] += ra[e] * xv;
                  }
                }
              }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty_far[slot]);
            if (fwd && urgent_pending) {
              // warp 0's part of the first chunk covered far rows 0 .. 31: the leader may start the next panel
              if (lane == 0) mbar_arrive(&urg[s & 3]);
              urgent_pending = false;
            }
          }
          pos += whole ? slot_rows : rows;
          if (pos >= ring_eff) pos -= ring_eff;
          ++n;
        }
        if (!fwd) {
          // reduce the column sums over the lanes that share a rotation (8 groups: equal lane & 7, i.e. lane
          // bits 3 and 4 vary; 4 groups: equal (lane >> 1) & 3, i.e. bits 0, 3 and 4 vary) ...
#pragma unroll
          for (int e = 0; e < NB; ++e) {
            if (G == 4) acc[e] += __shfl_xor_sync(0xffffffffu, acc[e], 1);
            acc[e] += __shfl_xor_sync(0xffffffffu, acc[e], 8);
            acc[e] += __shfl_xor_sync(0xffffffffu, acc[e], 16);
          }
          // ... then across the rotation classes: the representative of class c collects column group c.  In
          // round d it takes, from the representative of class c - d, that lane's rotated group d, which holds
          // column group (d + c - d) = c
          const int cls = (G == 8) ? (lane & 7) : ((lane >> 1) & 3);
          T tot[E];
#pragma unroll
          for (int e = 0; e < E; ++e) tot[e] = 0;
#pragma unroll
          for (int d = 0; d < G; ++d) {
            const int src = (G == 8) ? ((cls - d) & 7) : (((cls - d) & 3) << 1);
#pragma unroll
            for (int e = 0; e < E; ++e) tot[e] += __shfl_sync(0xffffffffu, acc[d * E + e], src);
          }
          const bool rep_lane = (G == 8) ? (lane < 8) : ((lane & 0x19) == 0);
          if (rep_lane) {
#pragma unroll
            for (int e = 0; e < E; ++e) {
              if (rank == 0)
                red[q & 1][bw_id][cls * E + e] = tot[e];
              else
                red_r1[q & 3][bw_id][cls * E + e] = tot[e];
            }
          }
        }
      }
      if (fail) {
        raise_abort();
        if (lane == 0) atomicCAS(status, 0, (int)HPLMM_ERR_TIMEOUT);
        break;
      }
      __syncwarp();
      if (lane == 0) {
        if (rank == 0) {
          if (urgent_pending) mbar_arrive(&urg[s & 3]);  // no far rows in this step's first pass
          mbar_arrive(&bdone[s & 3]);
        } else {
          mbar_arrive(&r1done[s & 3]);
        }
      }
    }
  }
  if constexpr (CL == 2)
    cluster_sync_all();  // no CTA leaves while its peer may still access its shared memory
  else
    __syncthreads();
}

template <typename T>
T *band_ptr(LocalSet &S);
template <>
float *band_ptr<float>(LocalSet &S) { return S.band32.p; }
template <>
double *band_ptr<double>(LocalSet &S) { return S.band64.p; }

}  // namespace

int num_sms() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

namespace {

// band offsets of a set in the panel layout of precision T; returns the largest half bandwidth
template <typename T>
int layout_set(LocalSet &S, cudaStream_t s) {
  constexpr int NB = NBOf<T>::v;
  const int K = S.count;
  std::vector<long long> boff(K + 1, 0);
  int bwmax = 0;
  for (int k = 0; k < K; ++k) {
    const int N = S.h_n[k], bw = S.h_bw[k];
    const long long np = (N + NB - 1) / NB;
    boff[k + 1] = boff[k] + np * (NB + bw) * NB;
    if (N > 0) bwmax = std::max(bwmax, bw);
  }
  const size_t smem = (size_t)(NB + bwmax) * (NB + 16 / sizeof(T)) * sizeof(T);
  HP_REQUIRE(smem <= 200 * 1024, HPLMM_ERR_INVALID,
             "local problem half bandwidth " + std::to_string(bwmax) + " is too large; use smaller grain grids");
  S.h_band_off = boff;
  S.band_off.upload(boff, s);
  return bwmax;
}

// FP32 banded Cholesky of `count` problems listed in `order` (their bands at band + band_off[k] - bbase):
// a two-CTA cluster per problem when the problems leave at least half of the SMs idle, else one CTA per
// problem taking problems from the queue
void launch_chol32(hplmm_ctx *c, LocalSet &S, int where, cudaStream_t s, const int *order, int count, float *band,
                   long long bbase, int bwmax) {
  constexpr int NB = 32;
  const size_t smem32 =
      ((size_t)(NB + bwmax) * CHOL32_LD + (size_t)(CHOL32_THREADS / 32) * 32 * CHOL32_CST_LD) * sizeof(float);
  HP_REQUIRE(smem32 <= 216 * 1024, HPLMM_ERR_INVALID,
             "local problem half bandwidth " + std::to_string(bwmax) + " is too large; use smaller grain grids");
  S.queue.alloc(1);
  HP_CUDA(cudaMemsetAsync(S.queue.p, 0, sizeof(int), s));
  if (2 * count <= num_sms()) {
    HP_CUDA(cudaFuncSetAttribute(k_band_chol32<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem32));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(2 * count));
    cfg.blockDim = dim3(CHOL32_THREADS);
    cfg.dynamicSmemBytes = smem32;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    HP_CUDA(cudaLaunchKernelEx(&cfg, k_band_chol32<2>, order, count, S.queue.p, (const int *)S.n.p,
                               (const int *)S.bw.p, (const long long *)S.band_off.p, band, c->status.p, where,
                               bwmax, bbase));
  } else {
    const int grid = std::min(count, 2 * num_sms());
    HP_CUDA(cudaFuncSetAttribute(k_band_chol32<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem32));
    k_band_chol32<1><<<grid, CHOL32_THREADS, smem32, s>>>(order, count, S.queue.p, S.n.p, S.bw.p, S.band_off.p,
                                                          band, c->status.p, where, bwmax, bbase);
  }
  HP_CHECK_LAUNCH();
}

template <typename T>
void layout_and_factor(hplmm_ctx *c, LocalSet &S, int where, cudaStream_t s, bool sync) {
  constexpr int NB = NBOf<T>::v;
  const int K = S.count;
  const int bwmax = layout_set<T>(S, s);
  const long long total = S.h_band_off[K];
  if (sizeof(T) == 8) {
    S.band64.alloc(std::max<long long>(total, 1));
    S.band64.zero(s);
  } else {
    S.band32.alloc(std::max<long long>(total, 1));
    S.band32.zero(s);
  }
  T *band = band_ptr<T>(S);
  k_local_extract<T><<<K, 128, 0, s>>>(S.box.p, S.node_off.p, S.n.p, S.bw.p, S.band_off.p, S.lmap.p, S.lnodes.p,
                                       c->node_ijk.p, c->row_ptr.p, c->col.p, c->val64.p, c->fixed.p, band, NB,
                                       nullptr, 0LL);
  HP_CHECK_LAUNCH();
  if constexpr (sizeof(T) == 4) {
    launch_chol32(c, S, where, s, S.order.p, K, band, 0LL, bwmax);
  } else {
    const size_t smem = (size_t)(NB + bwmax) * (NB + 16 / sizeof(T)) * sizeof(T);
    S.queue.alloc(1);
    S.queue.zero(s);
    const int grid = std::min(K, 2 * num_sms());
    auto kern = k_band_chol<T, NB>;
    HP_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<grid, FACT_THREADS, smem, s>>>(S.order.p, K, S.queue.p, S.n.p, S.bw.p, S.band_off.p, band, c->status.p,
                                          where);
    HP_CHECK_LAUNCH();
  }
  if (sync) HP_CUDA(cudaStreamSynchronize(s));
}

}  // namespace

// ---------------------------------------------------------------- set construction
static void finish_set(hplmm_ctx *c, LocalSet &S, int kind, const std::vector<int> &hbox) {
  cudaStream_t s = c->stream;
  int K = S.count;
  S.box.upload(hbox, s);
  std::vector<long long> noff(K + 1, 0);
  for (int k = 0; k < K; ++k)
    noff[k + 1] = noff[k] + (long long)hbox[9 * k + 3] * hbox[9 * k + 4] * hbox[9 * k + 5];
  S.h_node_off = noff;
  S.node_total = noff[K];
  S.node_off.upload(noff, s);
  if (S.lmap.n < (size_t)std::max<long long>(noff[K], 1) || kind == 0) {
    S.lmap.alloc(std::max<long long>(noff[K], 1));
    S.lmap.zero(s);
  }
  S.lnodes.alloc(std::max<long long>(noff[K], 1));
  S.n.alloc(std::max(K, 1));
  S.bw.alloc(std::max(K, 1));
  S.bw.zero(s);
}

static void enumerate_set(hplmm_ctx *c, LocalSet &S, int kind) {
  cudaStream_t s = c->stream;
  int K = S.count;
  if (K == 0) return;
  k_local_enum<<<K, 256, 0, s>>>(kind, S.box.p, S.node_off.p, S.lmap.p, S.lnodes.p, S.n.p, c->grid_to_node.p, c->nx,
                                 c->ny, c->node_cls.p, c->fixed.p);
  HP_CHECK_LAUNCH();
  k_local_bw<<<K, 128, 0, s>>>(S.box.p, S.node_off.p, S.n.p, S.lmap.p, S.lnodes.p, c->node_ijk.p, c->row_ptr.p,
                               c->col.p, S.bw.p);
  HP_CHECK_LAUNCH();
  S.h_n = S.n.download(s, K);
  S.h_bw = S.bw.download(s, K);
  std::vector<long long> voff(K + 1, 0);
  for (int k = 0; k < K; ++k) voff[k + 1] = voff[k] + S.h_n[k];
  S.h_vec_off = voff;
  S.vec_total = voff[K];
  S.vec_off.upload(voff, s);
  S.yscr.alloc(std::max<long long>(S.vec_total, 1));
  S.gidx.alloc(std::max<long long>(S.vec_total, 1));
  k_local_gidx<<<K, 256, 0, s>>>(S.n.p, S.node_off.p, S.vec_off.p, S.lnodes.p, S.gidx.p);
  HP_CHECK_LAUNCH();
  std::vector<int> ord(K);
  std::iota(ord.begin(), ord.end(), 0);
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) {
    double ca = (double)S.h_n[a] * S.h_bw[a] * S.h_bw[a], cb = (double)S.h_n[b] * S.h_bw[b] * S.h_bw[b];
    return ca > cb;
  });
  S.order.upload(ord, s);
  HP_CUDA(cudaStreamSynchronize(s));
}

static std::vector<int> make_boxes(const std::vector<int> &bmin, const std::vector<int> &bmax, int K, int grow,
                                   int nx, int ny, int nz) {
  std::vector<int> hbox(9 * std::max(K, 1), 0);
  int lim[3] = {nx, ny, nz};
  for (int k = 0; k < K; ++k) {
    int ext[3];
    for (int a = 0; a < 3; ++a) {
      int lo = bmin[3 * k + a], hi = bmax[3 * k + a];
      if (lo > hi) {  // empty
        lo = 0;
        hi = -1;
      } else {
        lo = std::max(lo - grow, 0);
        hi = std::min(hi + grow, lim[a]);
      }
      hbox[9 * k + a] = lo;
      ext[a] = hi - lo + 1;
      hbox[9 * k + 3 + a] = std::max(ext[a], 0);
    }
    int perm[3] = {0, 1, 2};
    std::stable_sort(perm, perm + 3, [&](int a, int b) { return ext[a] < ext[b]; });
    for (int a = 0; a < 3; ++a) hbox[9 * k + 6 + a] = perm[a];
  }
  return hbox;
}

void build_local_sets(hplmm_ctx *c) {
  cudaStream_t s = c->stream;
  int G = c->n_grains;
  // grains
  {
    Buf<int> bmin, bmax;
    bmin.alloc(3 * G);
    bmax.alloc(3 * G);
    bmin.fill_bytes(0x7f, s);
    bmax.fill_bytes(0x80, s);
    k_grain_bbox<<<grid_for(c->n_nodes, 256), 256, 0, s>>>(c->node_cls.p, c->node_ijk.p, c->n_nodes, bmin.p, bmax.p);
    HP_CHECK_LAUNCH();
    auto lo = bmin.download(s), hi = bmax.download(s);
    c->grains.count = G;
    auto hbox = make_boxes(lo, hi, G, 0, c->nx, c->ny, c->nz);
    finish_set(c, c->grains, 0, hbox);
    enumerate_set(c, c->grains, 0);
  }
  // contact grids
  {
    // the ILU(0) base smoother replaces the contact-grain smoother: no contact grids then
    int C = c->opt.smoother_kind == HPLMM_SMOOTHER_ILU0 ? 0 : c->n_ifaces;
    c->contacts.count = C;
    if (C > 0) {
      Buf<int> bmin, bmax;
      bmin.alloc(3 * C);
      bmax.alloc(3 * C);
      bmin.fill_bytes(0x7f, s);
      bmax.fill_bytes(0x80, s);
      k_iface_bbox<<<grid_for(c->n_iface_nodes, 256), 256, 0, s>>>(c->iface_nodes.p, c->iface_of_node.p,
                                                                   c->n_iface_nodes, c->node_ijk.p, bmin.p, bmax.p);
      HP_CHECK_LAUNCH();
      auto lo = bmin.download(s), hi = bmax.download(s);
      int w = c->opt.contact_halfwidth;
      auto hbox = make_boxes(lo, hi, C, w, c->nx, c->ny, c->nz);
      finish_set(c, c->contacts, 1, hbox);
      c->contacts.lmap.zero(s);
      k_contact_mark<<<grid_for(c->n_iface_nodes, 128), 128, 0, s>>>(c->iface_nodes.p, c->iface_of_node.p,
                                                                     c->n_iface_nodes, c->node_ijk.p,
                                                                     c->contacts.box.p, c->contacts.node_off.p, w,
                                                                     c->contacts.lmap.p);
      HP_CHECK_LAUNCH();
      enumerate_set(c, c->contacts, 1);
    }
  }
}

__global__ void k_to_bf16(const float *src, __nv_bfloat16 *dst, long long n) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = __float2bfloat16_rn(src[i]);
}

void to_bf16(const float *src, __nv_bfloat16 *dst, long long n, cudaStream_t s) {
  if (n <= 0) return;
  k_to_bf16<<<grid_for(n, 256), 256, 0, s>>>(src, dst, n);
  HP_CHECK_LAUNCH();
}

static void bf16_copy(hplmm_ctx *c, LocalSet &S, hplmm_prec prec);

void factor_local(hplmm_ctx *c, LocalSet &S, hplmm_prec prec) {
  if (S.count == 0) return;
  int where = (&S == &c->grains) ? 1 : 2;
  ProfScope ps(c, where == 1 ? HPLMM_PH_FACTOR_GRAINS : HPLMM_PH_FACTOR_CONTACTS);
  if (prec == HPLMM_FP64)
    layout_and_factor<double>(c, S, where, c->stream, true);
  else
    layout_and_factor<float>(c, S, where, c->stream, true);
  bf16_copy(c, S, prec);
}

// Both sets at once: the grain factorisation (few large problems, one SM each) on the context's stream and
// the contact grids' on a second stream, so the contact grids fill the SMs the grains leave idle.  The phase
// timer HPLMM_PH_FACTOR_GRAINS covers both.
void factor_local_both(hplmm_ctx *c, hplmm_prec prec) {
  ProfScope ps(c, HPLMM_PH_FACTOR_GRAINS);
  if (!c->aux_stream) HP_CUDA(cudaStreamCreateWithFlags(&c->aux_stream, cudaStreamNonBlocking));
  if (!c->ev_fork) HP_CUDA(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
  if (!c->ev_join) HP_CUDA(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
  HP_CUDA(cudaEventRecord(c->ev_fork, c->stream));
  HP_CUDA(cudaStreamWaitEvent(c->aux_stream, c->ev_fork, 0));
  auto run = [&](LocalSet &S, int where, cudaStream_t st) {
    if (S.count == 0) return;
    if (prec == HPLMM_FP64)
      layout_and_factor<double>(c, S, where, st, false);
    else
      layout_and_factor<float>(c, S, where, st, false);
  };
  run(c->grains, 1, c->stream);
  run(c->contacts, 2, c->aux_stream);
  HP_CUDA(cudaEventRecord(c->ev_join, c->aux_stream));
  HP_CUDA(cudaStreamWaitEvent(c->stream, c->ev_join, 0));
  HP_CUDA(cudaStreamSynchronize(c->stream));
  bf16_copy(c, c->grains, prec);
  bf16_copy(c, c->contacts, prec);
}

static void bf16_copy(hplmm_ctx *c, LocalSet &S, hplmm_prec prec) {
  if (S.count == 0) return;
  S.prec = prec;
  // BF16 form: the apply streams a BF16 copy of the FP32 factors (FP32 arithmetic)
  S.apply_bf16 = prec == HPLMM_FP32 && c->opt.apply_prec == HPLMM_BF16;
  if (S.apply_bf16) {
    long long n = S.h_band_off.empty() ? 0 : S.h_band_off.back();
    S.band16.alloc(std::max<long long>(n, 1));
    to_bf16(S.band32.p, S.band16.p, n, c->stream);
  } else {
    S.band16.release();
  }
}

template <typename T>
static void solve_multi_t(hplmm_ctx *c, LocalSet &S, T *X, const Buf<long long> &x_off, const Buf<int> &x_ld,
                          const std::vector<int> &h_ld, const std::vector<int> *only = nullptr,
                          const T *band = nullptr, long long bbase = 0) {
  if (!band) band = band_ptr<T>(S);
  constexpr int NB = NBOf<T>::v;
  cudaStream_t s = c->stream;
  std::vector<int> items;
  std::vector<char> pick;
  if (only) {
    pick.assign(S.count, 0);
    for (int k : *only) pick[k] = 1;
  }
  // largest problems first
  auto ord = S.order.download(s, S.count);
  for (int k : ord) {
    if (S.h_n[k] == 0 || (only && !pick[k])) continue;
    for (int r0 = 0; r0 < h_ld[k]; r0 += 32) {
      items.push_back(k);
      items.push_back(r0);
    }
  }
  int n_items = (int)items.size() / 2;
  if (n_items == 0) return;
  ProfScope ps(c, HPLMM_PH_BASIS_SOLVE);
  Buf<int> it;
  it.upload(items, s);
  if constexpr (sizeof(T) == 4) {
    int rpmax = NB;
    for (int k = 0; k < S.count; ++k)
      if (S.h_n[k] > 0) rpmax = std::max(rpmax, NB + S.h_bw[k]);
    const int XR = ((rpmax + NB + NB - 1) / NB) * NB;  // ring rows >= RP + NB
    const size_t smem = ((size_t)SM32_STAGES * SM32_CH * NB + (size_t)XR * NB) * sizeof(float);
    HP_REQUIRE(smem <= 180 * 1024, HPLMM_ERR_INVALID,
               "local problem half bandwidth " + std::to_string(rpmax - NB) + " is too large for the basis solves");
    HP_CUDA(cudaFuncSetAttribute(k_band_solve_multi32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_band_solve_multi32<<<n_items, SM32_THREADS, smem, s>>>(it.p, n_items, S.n.p, S.bw.p, S.band_off.p,
                                                             band, X, x_off.p, x_ld.p, XR, bbase);
  } else {
    k_band_solve_multi<T, NB><<<n_items, 256, 0, s>>>(it.p, n_items, S.n.p, S.bw.p, S.band_off.p, band,
                                                      X, x_off.p, x_ld.p);
  }
  HP_CHECK_LAUNCH();
  HP_CUDA(cudaStreamSynchronize(s));
}

void solve_local_multi_f64(hplmm_ctx *c, LocalSet &S, double *X, const Buf<long long> &x_off, const Buf<int> &x_ld,
                           const std::vector<int> &h_ld) {
  solve_multi_t<double>(c, S, X, x_off, x_ld, h_ld);
}
void solve_local_multi_f32_subset(hplmm_ctx *c, LocalSet &S, float *X, const Buf<long long> &x_off,
                                  const Buf<int> &x_ld, const std::vector<int> &h_ld, const std::vector<int> &grains) {
  solve_multi_t<float>(c, S, X, x_off, x_ld, h_ld, &grains);
}
void solve_local_multi_f32(hplmm_ctx *c, LocalSet &S, float *X, const Buf<long long> &x_off, const Buf<int> &x_ld,
                           const std::vector<int> &h_ld) {
  solve_multi_t<float>(c, S, X, x_off, x_ld, h_ld);
}

// local right-hand-side panels of the multi-right-hand-side smoother: P[l][q] = R_q[gidx[l]] (row l of the
// set's local vectors, k columns), and back: Z_q[gidx[l]] (+)= P[l][q]
template <typename T>
__global__ void k_local_gather_multi(const int *gidx, long long n, const double *R, long long L, int k, T *P) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * k) return;
  const long long l = e / k;
  const int q = (int)(e - l * k);
  P[e] = (T)R[q * L + gidx[l]];
}
template <typename T>
__global__ void k_local_scatter_multi(const int *gidx, long long n, const T *P, long long L, int k, double *Z,
                                      int atomic) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * k) return;
  const long long l = e / k;
  const int q = (int)(e - l * k);
  double *dst = Z + q * L + gidx[l];
  if (atomic)
    atomicAdd(dst, (double)P[e]);
  else
    *dst = (double)P[e];
}

// The smoother for k right-hand sides at stride L: each local problem's right-hand sides form an N x k panel
// that the multi-right-hand-side banded solves (the basis solves' kernels) process with one read of the
// factor per 32 columns.  The BF16 form keeps no FP32 factors: it applies the one-vector solve per column.
void smoother_apply_multi(hplmm_ctx *c, LocalSet &S, const double *R, double *Z, int k, bool atomic) {
  if (S.count == 0) return;
  const long long L = 3LL * c->n_nodes;
  if (S.apply_bf16) {
    for (int q = 0; q < k; ++q) smoother_apply(c, S, R + q * L, Z + q * L, atomic);
    return;
  }
  ProfScope ps(c, (&S == &c->grains) ? HPLMM_PH_APPLY_GRAINS : HPLMM_PH_APPLY_CONTACTS);
  cudaStream_t s = c->stream;
  const long long n = S.vec_total;
  std::vector<long long> off(S.count);
  for (int p = 0; p < S.count; ++p) off[p] = S.h_vec_off[p] * k;
  Buf<long long> moff;
  Buf<int> mld;
  moff.upload(off, s);
  std::vector<int> ld(S.count, k);
  mld.upload(ld, s);
  const unsigned grid = grid_for(n * k, 256);
  if (S.prec == HPLMM_FP64) {
    c->mloc64.alloc(std::max<long long>(n * k, 1));
    k_local_gather_multi<double><<<grid, 256, 0, s>>>(S.gidx.p, n, R, L, k, c->mloc64.p);
    HP_CHECK_LAUNCH();
    solve_multi_t<double>(c, S, c->mloc64.p, moff, mld, ld);
    k_local_scatter_multi<double><<<grid, 256, 0, s>>>(S.gidx.p, n, c->mloc64.p, L, k, Z, atomic ? 1 : 0);
  } else {
    c->mloc32.alloc(std::max<long long>(n * k, 1));
    k_local_gather_multi<float><<<grid, 256, 0, s>>>(S.gidx.p, n, R, L, k, c->mloc32.p);
    HP_CHECK_LAUNCH();
    solve_multi_t<float>(c, S, c->mloc32.p, moff, mld, ld);
    k_local_scatter_multi<float><<<grid, 256, 0, s>>>(S.gidx.p, n, c->mloc32.p, L, k, Z, atomic ? 1 : 0);
  }
  HP_CHECK_LAUNCH();
}

// Staged set-up of the BF16 form: the apply streams BF16 copies of the FP32 local factors, so the FP32
// factors need not outlive the set-up.  Each set is factored in chunks of consecutive problems whose FP32
// bands fit a scratch buffer (options.stage_mb, default STAGE_ELEMS floats); a chunk of grains serves its grains' basis solves (Eqs.
// col_pk, col_cg) while it is FP32, then every chunk is rounded to BF16 into the set's BF16 band.  The
// result equals the unstaged form's (the same FP32 factors and solves); the device then holds the BF16
// bands, one FP32 chunk and the FP32 panels, instead of every FP32 band and its BF16 copy.
void factor_staged(hplmm_ctx *c, float *X, const Buf<long long> &x_off, const Buf<int> &x_ld,
                   const std::vector<int> &h_ld) {
  cudaStream_t s = c->stream;
  c->bstats = hplmm_basis_stats{};
  for (int which = 0; which < 2; ++which) {
    LocalSet &S = which == 0 ? c->grains : c->contacts;
    const int where = which == 0 ? 1 : 2;
    S.prec = HPLMM_FP32;
    S.apply_bf16 = true;
    S.band32.release();
    const int K = S.count;
    if (K == 0) continue;
    const int bwmax = layout_set<float>(S, s);
    const std::vector<long long> &boff = S.h_band_off;
    S.band16.alloc(std::max<long long>(boff[K], 1));
    long long most = 1;
    for (int k = 0; k < K; ++k) most = std::max(most, boff[k + 1] - boff[k]);
    const long long budget = c->opt.stage_mb > 0 ? ((long long)c->opt.stage_mb << 20) / 4 : STAGE_ELEMS;
    const long long cap = std::max(most, std::min<long long>(boff[K], budget));
    c->stage32.alloc(cap);
    const std::vector<int> ord = S.order.download(s, K);
    Buf<int> plist;
    for (int k0 = 0; k0 < K;) {
      int k1 = k0 + 1;
      while (k1 < K && boff[k1 + 1] - boff[k0] <= cap) ++k1;
      const long long base = boff[k0], elems = boff[k1] - boff[k0];
      std::vector<int> pl;  // the chunk's problems, most expensive first
      for (int k : ord)
        if (k >= k0 && k < k1) pl.push_back(k);
      HP_CUDA(cudaStreamSynchronize(s));  // the previous chunk's list is read until here
      plist.upload(pl, s);
      {
        ProfScope ps(c, HPLMM_PH_FACTOR_GRAINS);
        HP_CUDA(cudaMemsetAsync(c->stage32.p, 0, sizeof(float) * elems, s));
        k_local_extract<float><<<(unsigned)pl.size(), 128, 0, s>>>(
            S.box.p, S.node_off.p, S.n.p, S.bw.p, S.band_off.p, S.lmap.p, S.lnodes.p, c->node_ijk.p, c->row_ptr.p,
            c->col.p, c->val64.p, c->fixed.p, c->stage32.p, 32, plist.p, base);
        HP_CHECK_LAUNCH();
        launch_chol32(c, S, where, s, plist.p, (int)pl.size(), c->stage32.p, base, bwmax);
      }
      if (which == 0) solve_multi_t<float>(c, S, X, x_off, x_ld, h_ld, &pl, c->stage32.p, base);
      to_bf16(c->stage32.p, S.band16.p + base, elems, s);
      k0 = k1;
    }
    HP_CUDA(cudaStreamSynchronize(s));
  }
  c->stage32.release();  // the rest of the set-up and the solve need the memory more than the next set-up
}

// shared-memory plan of the smoother solve for a set: stored-row width (128 bytes for FP32/FP64 factors, 64
// bytes for BF16), one diagonal+near chunk, and the local vector window (a power of two >= RP + 3 NB rows)
struct SolvePlan {
  int rowb, W;
  size_t c0_slot, vbytes;
};
// dynamic shared-memory budgets of a smoother kernel: one CTA per SM (the opt-in maximum per block less the
// kernel's static shared memory), or two CTAs per SM (half of the SM's shared memory, less the static part
// and the per-block reservation)
struct SmemBudget {
  size_t one, pair, third, quarter;  // dynamic shared memory for one to four CTAs per SM
};
template <typename K> static SmemBudget smem_budget(K kern) {
  static std::mutex mu;
  static std::map<const void *, SmemBudget> cache;
  std::lock_guard<std::mutex> lk(mu);
  auto it = cache.find((const void *)kern);
  if (it != cache.end()) return it->second;
  cudaFuncAttributes fa{};
  HP_CUDA(cudaFuncGetAttributes(&fa, kern));
  int dev = 0, optin = 0, per_sm = 0;
  HP_CUDA(cudaGetDevice(&dev));
  HP_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  HP_CUDA(cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
  SmemBudget b;
  b.one = (size_t)optin - fa.sharedSizeBytes - 256;
  b.pair = (size_t)per_sm / 2 - fa.sharedSizeBytes - 1024 - 256;
  b.third = (size_t)per_sm / 3 - fa.sharedSizeBytes - 1024 - 256;
  b.quarter = (size_t)per_sm / 4 - fa.sharedSizeBytes - 1024 - 256;
  cache[(const void *)kern] = b;
  return b;
}

static SolvePlan solve_plan(const LocalSet &S) {
  const bool f64 = S.prec == HPLMM_FP64;
  const int NBv = f64 ? 16 : 32;
  const size_t esz = f64 ? 8 : 4;  // compute type of the local vector
  SolvePlan pl;
  pl.rowb = S.apply_bf16 ? 64 : 128;
  pl.c0_slot = (size_t)2 * NBv * pl.rowb;
  int need = 4 * NBv;  // RP + 3 NB rows
  for (int k = 0; k < S.count; ++k)
    if (S.h_n[k] > 0) need = std::max(need, S.h_bw[k] + 4 * NBv);
  pl.W = 1;
  while (pl.W < need) pl.W <<= 1;
  pl.vbytes = ((esz * (size_t)pl.W + 127) / 128) * 128;
  return pl;
}

// far chunk sizes (rows) the tuner tries: 64 KiB, and a whole step's far rows per copy
static std::vector<int> chunk_choices(const LocalSet &S) {
  return S.apply_bf16 ? std::vector<int>{1024, 4096} : std::vector<int>{512, 2048};
}

// ring rows that fit in `budget` bytes next to c0s diagonal stages and the window (a multiple of 8)
static int ring_rows_for(const SolvePlan &pl, int c0s, size_t budget) {
  const long long avail = (long long)budget - (long long)c0s * (long long)pl.c0_slot - (long long)pl.vbytes;
  return avail > 0 ? (int)((avail / pl.rowb) & ~7LL) : 0;
}

// CTAs per local problem: two (a cluster sharing each panel's far rows) when the set leaves at least half
// of the SMs idle with one CTA per problem, else one; the tuner may override
static int default_cluster(const LocalSet &S) { return 2 * S.count <= num_sms() ? 2 : 1; }

void smoother_apply(hplmm_ctx *c, LocalSet &S, const double *r_pad, double *z_pad, bool atomic) {
  if (S.count == 0) return;
  ProfScope ps(c, (&S == &c->grains) ? HPLMM_PH_APPLY_GRAINS : HPLMM_PH_APPLY_CONTACTS);
  cudaStream_t s = c->stream;
  const SolvePlan pl = solve_plan(S);
  const int fb = c->opt.smoother_bulk_warps;  // forced bulk warps, 0 if none
  const int cl = (fb > 0 && fb < WS_BULK_WARPS) ? 1
                 : c->opt.smoother_ctas > 0     ? c->opt.smoother_ctas
                                                : (S.tuned_cluster > 0 ? S.tuned_cluster : default_cluster(S));
  // depths: the tuner's choice when there is one, else 3 diagonal stages, whole-step chunks and the largest
  // ring
  const int c0s = S.tuned_c0_stages > 0 ? S.tuned_c0_stages : 3;
  // bulk warps per CTA: 8 (one CTA per SM), or, for one-CTA problems, 4, 2 or 1 with the ring sized for two,
  // three or four CTAs per SM (forced, or the tuner's choice)
  const int nbw = fb > 0 ? fb
                  : (cl == 1 && (S.tuned_bulk == 4 || S.tuned_bulk == 2 || S.tuned_bulk == 1)) ? S.tuned_bulk
                                                                                               : WS_BULK_WARPS;
  auto go = [&](auto kern, const auto *band, auto *ys) {
    const SmemBudget bud = smem_budget(kern);
    int ring = ring_rows_for(pl, c0s, nbw == WS_BULK_WARPS ? bud.one
                                      : nbw == 4            ? bud.pair
                                      : nbw == 2            ? bud.third
                                                            : bud.quarter);
    if (S.tuned_ring_rows > 0) ring = std::min(ring, S.tuned_ring_rows);
    HP_REQUIRE(ring >= 64, HPLMM_ERR_INVALID,
               "local problem too large for the smoother (window of " + std::to_string(pl.W) + " rows)");
    const int chunk = std::min(ring, S.tuned_chunk_rows > 0 ? S.tuned_chunk_rows : chunk_choices(S).back());
    const size_t smem = (size_t)ring * pl.rowb + (size_t)c0s * pl.c0_slot + pl.vbytes;
    HP_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(S.count * cl));
    cfg.blockDim = dim3((unsigned)((3 + nbw) * 32));
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)cl;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    HP_CUDA(cudaLaunchKernelEx(&cfg, kern, S.count, (const int *)S.n.p, (const int *)S.bw.p,
                               (const long long *)S.band_off.p, (const long long *)S.vec_off.p,
                               (const int *)S.gidx.p, band, (const double *)r_pad, z_pad, ys, atomic ? 1 : 0, ring,
                               chunk, c0s, pl.W - 1, c->status.p,
                               c->opt.wait_budget_us > 0 ? (long long)c->opt.wait_budget_us * 2070LL : WAIT_CYCLES));
  };
  // the kernel instance: storage type and CTAs per problem
  auto pick = [&](auto tag, auto nb, const auto *band, auto *ys) {
    using ST = decltype(tag);
    constexpr int NBv = decltype(nb)::value;
    if (cl == 2)
      go(k_band_solve_ws<ST, NBv, 2, WS_BULK_WARPS>, band, ys);
    else if (nbw == 4)
      go(k_band_solve_ws<ST, NBv, 1, 4>, band, ys);
    else if (nbw == 2)
      go(k_band_solve_ws<ST, NBv, 1, 2>, band, ys);
    else if (nbw == 1)
      go(k_band_solve_ws<ST, NBv, 1, 1>, band, ys);
    else
      go(k_band_solve_ws<ST, NBv, 1, WS_BULK_WARPS>, band, ys);
  };
  if (S.prec == HPLMM_FP64) {
    pick(double{}, std::integral_constant<int, 16>{}, (const double *)S.band64.p, S.yscr.p);
  } else if (S.apply_bf16) {
    pick(__nv_bfloat16{}, std::integral_constant<int, 32>{}, (const __nv_bfloat16 *)S.band16.p,
         reinterpret_cast<float *>(S.yscr.p));
  } else {
    pick(float{}, std::integral_constant<int, 32>{}, (const float *)S.band32.p, reinterpret_cast<float *>(S.yscr.p));
  }
  HP_CHECK_LAUNCH();
}

// ---------------------------------------------------------------- tuner of the smoother solve pipeline
// For each set of local problems, time the smoother solve under every plan (far chunk size x diagonal-chunk
// stages x ring size: the largest, or one small enough for two CTAs per SM) on the set's own factors, and
// keep the fastest.  Results are cached for the process, keyed by (count, largest local size, largest half
// bandwidth, precision), so a repeated set-up of the same size pays nothing.
namespace {
struct TuneKey {
  int count, nmax, bwmax, prec;
  bool operator<(const TuneKey &o) const {
    return std::tie(count, nmax, bwmax, prec) < std::tie(o.count, o.nmax, o.bwmax, o.prec);
  }
};
std::mutex g_tune_mu;
struct TuneChoice {
  int chunk_rows, ring_rows, c0_stages, cluster, bulk;
};
std::map<TuneKey, TuneChoice> g_tune_cache;
}  // namespace

static void tune_set(hplmm_ctx *c, LocalSet &S, bool atomic) {
  S.tuned_chunk_rows = S.tuned_ring_rows = S.tuned_c0_stages = S.tuned_cluster = S.tuned_bulk = 0;
  if (S.count == 0) return;
  TuneKey key{S.count, 0, 0,
              (int)S.prec + (S.apply_bf16 ? 8 : 0) + 16 * c->opt.smoother_ctas + 64 * c->opt.smoother_bulk_warps};
  for (int k = 0; k < S.count; ++k) {
    key.nmax = std::max(key.nmax, S.h_n[k]);
    key.bwmax = std::max(key.bwmax, S.h_bw[k]);
  }
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      S.tuned_chunk_rows = it->second.chunk_rows;
      S.tuned_ring_rows = it->second.ring_rows;
      S.tuned_c0_stages = it->second.c0_stages;
      S.tuned_cluster = it->second.cluster;
      S.tuned_bulk = it->second.bulk;
      return;
    }
  }
  const SolvePlan pl = solve_plan(S);
  cudaStream_t s = c->stream;
  cudaEvent_t e0, e1;
  HP_CUDA(cudaEventCreate(&e0));
  HP_CUDA(cudaEventCreate(&e1));
  const bool prof = c->opt.profile;
  c->opt.profile = 0;  // tuning launches are not part of any phase
  float best = 1e30f;
  TuneChoice bc{0, 0, 0, 0, 0};
  // budgets of the FP32 one-CTA kernels (the static shared memory of every instantiation is about the same;
  // smoother_apply clamps the ring to the launched kernel's own budget)
  const SmemBudget bud = S.prec == HPLMM_FP64 ? smem_budget(k_band_solve_ws<double, 16, 1, WS_BULK_WARPS>)
                                              : smem_budget(k_band_solve_ws<float, 32, 1, WS_BULK_WARPS>);
  const SmemBudget bud4 = S.prec == HPLMM_FP64 ? smem_budget(k_band_solve_ws<double, 16, 1, 4>)
                                               : smem_budget(k_band_solve_ws<float, 32, 1, 4>);
  const SmemBudget bud2 = S.prec == HPLMM_FP64 ? smem_budget(k_band_solve_ws<double, 16, 1, 2>)
                                               : smem_budget(k_band_solve_ws<float, 32, 1, 2>);
  const SmemBudget bud1 = S.prec == HPLMM_FP64 ? smem_budget(k_band_solve_ws<double, 16, 1, 1>)
                                               : smem_budget(k_band_solve_ws<float, 32, 1, 1>);
  // plans: (CTAs per problem, bulk warps, shared-memory budget); the 4-, 2- and 1-warp kernels only with the
  // two-, three- and four-per-SM budgets, which are what they are for
  struct Form {
    int cl, nbw;
    size_t budget;
  };
  const Form forms[] = {{1, WS_BULK_WARPS, bud.one}, {1, WS_BULK_WARPS, bud.pair}, {1, 4, bud4.pair}, {1, 2, bud2.third},
                        {1, 1, bud1.quarter},
                        {2, WS_BULK_WARPS, bud.one}, {2, WS_BULK_WARPS, bud.pair}};
  for (const Form &f : forms)
   for (int chunk : chunk_choices(S))
    if ((c->opt.smoother_ctas == 0 || c->opt.smoother_ctas == f.cl) &&
        (c->opt.smoother_bulk_warps == 0 || c->opt.smoother_bulk_warps == f.nbw))
    for (int c0d = 2; c0d <= 4; ++c0d) {
        const int cl = f.cl;
        const int ring = ring_rows_for(pl, c0d, f.budget);
        const int cr = std::min(chunk, ring);
        if (cr < 64) continue;
        S.tuned_chunk_rows = cr;
        S.tuned_ring_rows = ring;
        S.tuned_c0_stages = c0d;
        S.tuned_cluster = cl;
        S.tuned_bulk = f.nbw;
        smoother_apply(c, S, c->b_pad.p, c->w_zz.p, atomic);  // warm-up
        HP_CUDA(cudaEventRecord(e0, s));
        for (int rep = 0; rep < 3; ++rep) smoother_apply(c, S, c->b_pad.p, c->w_zz.p, atomic);
        HP_CUDA(cudaEventRecord(e1, s));
        HP_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        HP_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (c->opt.verbose)
          fprintf(stderr,
                  "[hplmm] tuner trial: %d problems, %d CTA(s) each, %d bulk warps, chunk %d rows, ring %d rows, "
                  "diagonal %d: %.3f ms\n",
                  S.count, cl, f.nbw, cr, ring, c0d, ms / 3);
        if (ms < best) {
          best = ms;
          bc = {cr, ring, c0d, cl, f.nbw};
        }
      }
  c->opt.profile = prof;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  S.tuned_chunk_rows = bc.chunk_rows;
  S.tuned_ring_rows = bc.ring_rows;
  S.tuned_c0_stages = bc.c0_stages;
  S.tuned_cluster = bc.cluster;
  S.tuned_bulk = bc.bulk;
  if (c->opt.verbose)
    fprintf(stderr,
            "[hplmm] tuner: %d problems (n<=%d, bw<=%d): %d CTA(s) each, %d bulk warps, chunk %d rows, ring %d "
            "rows, diagonal stages %d, %.3f ms\n",
            S.count, key.nmax, key.bwmax, bc.cluster, bc.bulk, bc.chunk_rows, bc.ring_rows, bc.c0_stages, best / 3);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache[key] = bc;
}

void tune_local(hplmm_ctx *c) {
  if (!c->opt.autotune) {
    c->grains.tuned_chunk_rows = c->grains.tuned_ring_rows = c->grains.tuned_c0_stages = c->grains.tuned_cluster = 0;
    c->contacts.tuned_chunk_rows = c->contacts.tuned_ring_rows = c->contacts.tuned_c0_stages = 0;
    c->contacts.tuned_cluster = c->grains.tuned_bulk = c->contacts.tuned_bulk = 0;
    return;
  }
  tune_set(c, c->contacts, true);
  tune_set(c, c->grains, false);
  HP_CUDA(cudaMemsetAsync(c->w_zz.p, 0, sizeof(double) * 3 * (size_t)c->n_nodes, c->stream));
  HP_CUDA(cudaStreamSynchronize(c->stream));
}

}  // namespace hp

// ---------------------------------------------------------------- algebraic mortars (Eq. algebra)
// The mortar functions of interface c solve S^c w = 0 off the mortar DOFs, with w = 1 at DOF (x_i, gamma) and
// 0 at the other mortar DOFs (the Remark after Eq. reduced_defs).  S^c stands for the interface's elasticity
// operator of Eq. algebra, built from A_hat: for every pair of distinct interface nodes {y, y'} that A_hat
// couples, the edge term (e_y - e_y')(e_y - e_y')^T (x) |B_yy'| with B_yy' = -(A_yy' + A_yy'^T)/2 and |.| the
// matrix absolute value, plus ALG_SHIFT times A_hat's diagonal.  Without the shift S^c is positive
// semidefinite and annihilates rigid translations of the interface (so the functions of one component sum
// to e_gamma); the shift makes it definite on interface pieces without a mortar node.  Each interface is a
// local problem on its own nodes (the contact-grid machinery with w = 0): S^c is extracted with the mortar and
// fixed DOFs as identity rows, factored (FP64 band), and solved for all of the interface's columns at once;
// the right-hand side of column (i, gamma) carries the unit value at its own DOF and minus the coupling to it
// on the other rows.
namespace hp {
namespace {

constexpr double ALG_SHIFT = 1e-8;  // relative to A_hat's diagonal

// P = |B| for B = -(V + V^T)/2, V a 3x3 block (row-major): cyclic Jacobi rotations (the symmetric Schur
// decomposition of Golub and Van Loan, Matrix Computations, Sec. 8.5) give B = Q L Q^T, then P = Q |L| Q^T
__device__ void abs_negsym3(const double *v, double *P) {
  double a[3][3], q[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) a[i][j] = -0.5 * (v[3 * i + j] + v[3 * j + i]);
  for (int sweep = 0; sweep < 12; ++sweep) {
    const double off = a[0][1] * a[0][1] + a[0][2] * a[0][2] + a[1][2] * a[1][2];
    const double on = a[0][0] * a[0][0] + a[1][1] * a[1][1] + a[2][2] * a[2][2];
    if (off <= 1e-36 * (on + off)) break;
    for (int pq = 0; pq < 3; ++pq) {
      const int p = pq == 2 ? 1 : 0, r = pq == 0 ? 1 : 2;
      if (a[p][r] == 0.0) continue;
      const double theta = (a[r][r] - a[p][p]) / (2.0 * a[p][r]);
      const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
      const double c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
      for (int k = 0; k < 3; ++k) {  // A J
        const double akp = a[k][p], akr = a[k][r];
        a[k][p] = c * akp - sn * akr;
        a[k][r] = sn * akp + c * akr;
      }
      for (int k = 0; k < 3; ++k) {  // J^T (A J)
        const double apk = a[p][k], ark = a[r][k];
        a[p][k] = c * apk - sn * ark;
        a[r][k] = sn * apk + c * ark;
      }
      for (int k = 0; k < 3; ++k) {  // Q J
        const double qkp = q[k][p], qkr = q[k][r];
        q[k][p] = c * qkp - sn * qkr;
        q[k][r] = sn * qkp + c * qkr;
      }
    }
  }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double sum = 0.0;
      for (int k = 0; k < 3; ++k) sum += q[i][k] * fabs(a[k][k]) * q[j][k];
      P[3 * i + j] = sum;
    }
}

// S^c of interface k into its band (lower triangle): edge terms -|B| off the diagonal, the sum of the node's
// |B| plus the shift on it; mortar and fixed DOFs as identity rows
__global__ void k_iface_extract(const int *box, const long long *node_off, const int *nloc, const int *bwv,
                                const long long *band_off, const int *lmap, const int *lnodes, const int *node_ijk,
                                const int *row_ptr, const int *col, const double *val, const uint8_t *fixed,
                                const int *mslot_of_node, double *band) {
  const int k = blockIdx.x;
  const Box b = load_box(box, k);
  const long long off = node_off[k];
  const int cnt = nloc[k] / 3, bw = bwv[k];
  double *B = band + band_off[k];
  for (int o = threadIdx.x; o < cnt; o += blockDim.x) {
    const int n = lnodes[off + o];
    const bool mo = mslot_of_node[n] >= 0;
    double dg[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, adiag[3] = {0, 0, 0};
    for (int p = row_ptr[n]; p < row_ptr[n + 1]; ++p) {
      const int m = col[p];
      const int cell = box_cell(b, node_ijk[3 * m], node_ijk[3 * m + 1], node_ijk[3 * m + 2]);
      if (cell < 0) continue;
      const int om = lmap[off + cell];
      if (om < 0) continue;
      const double *v = val + (long long)p * 9;
      if (m == n) {
        for (int d = 0; d < 3; ++d) adiag[d] = v[4 * d];
        continue;
      }
      double P[9];
      abs_negsym3(v, P);
#pragma unroll
      for (int e = 0; e < 9; ++e) dg[e] += P[e];
      if (mo || mslot_of_node[m] >= 0 || om > o) continue;
      for (int d = 0; d < 3; ++d)
        for (int d2 = 0; d2 < 3; ++d2)
          if (!fixed[3 * n + d] && !fixed[3 * m + d2]) B[panel_addr(3 * o + d, 3 * om + d2, 16, bw)] = -P[3 * d + d2];
    }
    for (int d = 0; d < 3; ++d) {
      const int i = 3 * o + d;
      if (mo || fixed[3 * n + d]) {
        B[panel_addr(i, i, 16, bw)] = 1.0;
        continue;
      }
      for (int d2 = 0; d2 < d; ++d2)
        if (!fixed[3 * n + d2]) B[panel_addr(i, 3 * o + d2, 16, bw)] = dg[3 * d + d2];
      B[panel_addr(i, i, 16, bw)] = dg[4 * d] + ALG_SHIFT * adiag[d];
    }
  }
}

// right-hand sides: row (o, d) of column (i, gamma): 1 if node o is mortar i and d = gamma; 0 on other mortar
// rows and fixed rows; otherwise minus S^c's coupling to the unit DOF, |B_{n m_i}|(d, gamma)
__global__ void k_iface_rhs(const long long *node_off, const int *nloc, const int *lnodes, const int *row_ptr,
                            const int *col, const double *val, const uint8_t *fixed, const int *iface_of_node,
                            const int *mslot_of_node, const int *mcol, const int *mfree, const long long *x_off,
                            const int *x_ld, double *X) {
  const int k = blockIdx.x;
  const int cnt = nloc[k] / 3;
  const int ld = x_ld[k];
  double *Xk = X + x_off[k];
  for (int o = threadIdx.x; o < cnt; o += blockDim.x) {
    const int n = lnodes[node_off[k] + o];
    const int ms = mslot_of_node[n];
    if (ms >= 0) {
      for (int g = 0; g < 3; ++g)
        if ((mfree[ms] >> g) & 1) Xk[(long long)(3 * o + g) * ld + mcol[ms] + __popc(mfree[ms] & ((1 << g) - 1))] = 1.0;
      continue;
    }
    for (int p = row_ptr[n]; p < row_ptr[n + 1]; ++p) {
      const int m = col[p];
      const int mm = mslot_of_node[m];
      if (mm < 0 || iface_of_node[m] != k) continue;
      double P[9];
      abs_negsym3(val + (long long)p * 9, P);
      for (int g = 0; g < 3; ++g) {
        if (!((mfree[mm] >> g) & 1)) continue;
        const int kk = mcol[mm] + __popc(mfree[mm] & ((1 << g) - 1));
        for (int d = 0; d < 3; ++d)
          if (!fixed[3 * n + d]) Xk[(long long)(3 * o + d) * ld + kk] = P[3 * d + g];
      }
    }
  }
}

// the solved columns into the interface's block of Q^o, rows (interface slot, component)
__global__ void k_iface_store(const long long *node_off, const int *nloc, const int *lnodes, const int *iface_slot,
                              const long long *x_off, const int *x_ld, const double *X, const long long *qoff,
                              double *Q) {
  const int k = blockIdx.x;
  const int cnt = nloc[k] / 3;
  const int ld = x_ld[k];
  for (int e = threadIdx.x; e < 3 * cnt * ld; e += blockDim.x) {
    const int row = e / ld, kk = e - row * ld;
    const int o = row / 3, d = row - 3 * o;
    const int slot = iface_slot[lnodes[node_off[k] + o]];
    Q[qoff[k] + (long long)(3 * slot + d) * ld + kk] = X[x_off[k] + e];
  }
}

__global__ void k_mortar_info(const int *mortar_nodes, int n_mortars, const uint8_t *fixed, int *mslot_of_node,
                              int *mfree) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n_mortars) return;
  const int n = mortar_nodes[q];
  mslot_of_node[n] = q;
  mfree[q] = (fixed[3 * n] ? 0 : 1) | (fixed[3 * n + 1] ? 0 : 2) | (fixed[3 * n + 2] ? 0 : 4);
}

}  // namespace

void build_algebraic_mortars(hplmm_ctx *c) {
  cudaStream_t s = c->stream;
  const int C = c->n_ifaces;
  if (C == 0) return;
  // columns: (mortar i, component gamma) for every free DOF of a mortar node
  c->mslot_of_node.alloc(c->n_nodes);
  c->mslot_of_node.fill_bytes(0xff, s);
  c->mfree.alloc(std::max(c->n_mortars, 1));
  k_mortar_info<<<grid_for(c->n_mortars, 256), 256, 0, s>>>(c->mortar_nodes.p, c->n_mortars, c->fixed.p,
                                                          c->mslot_of_node.p, c->mfree.p);
  HP_CHECK_LAUNCH();
  const std::vector<int> hfree = c->mfree.download(s, c->n_mortars);
  std::vector<int> hmcol(std::max(c->n_mortars, 1), 0);
  c->h_col_off.assign(C + 1, 0);
  for (int ci = 0; ci < C; ++ci) {
    int kk = 0;
    for (int q = c->h_mortar_off[ci]; q < c->h_mortar_off[ci + 1]; ++q) {
      hmcol[q] = kk;
      kk += __builtin_popcount(hfree[q]);
    }
    c->h_col_off[ci + 1] = c->h_col_off[ci] + kk;
  }
  c->mcol.upload(hmcol, s);
  layout_columns(c);
  // the interfaces as local problems on their own nodes
  LocalSet &S = c->ifsets;
  {
    Buf<int> bmin, bmax;
    bmin.alloc(3 * C);
    bmax.alloc(3 * C);
    bmin.fill_bytes(0x7f, s);
    bmax.fill_bytes(0x80, s);
    k_iface_bbox<<<grid_for(c->n_iface_nodes, 256), 256, 0, s>>>(c->iface_nodes.p, c->iface_of_node.p,
                                                                 c->n_iface_nodes, c->node_ijk.p, bmin.p, bmax.p);
    HP_CHECK_LAUNCH();
    auto lo = bmin.download(s), hi = bmax.download(s);
    S.count = C;
    auto hbox = make_boxes(lo, hi, C, 0, c->nx, c->ny, c->nz);
    finish_set(c, S, 1, hbox);
    S.lmap.zero(s);
    k_contact_mark<<<grid_for(c->n_iface_nodes, 128), 128, 0, s>>>(c->iface_nodes.p, c->iface_of_node.p,
                                                                   c->n_iface_nodes, c->node_ijk.p, S.box.p,
                                                                   S.node_off.p, 0, S.lmap.p);
    HP_CHECK_LAUNCH();
    enumerate_set(c, S, 1);
  }
  const int bwmax = layout_set<double>(S, s);
  S.band64.alloc(std::max<long long>(S.h_band_off[C], 1));
  S.band64.zero(s);
  S.prec = HPLMM_FP64;
  k_iface_extract<<<C, 128, 0, s>>>(S.box.p, S.node_off.p, S.n.p, S.bw.p, S.band_off.p, S.lmap.p, S.lnodes.p,
                                    c->node_ijk.p, c->row_ptr.p, c->col.p, c->val64.p, c->fixed.p,
                                    c->mslot_of_node.p, S.band64.p);
  HP_CHECK_LAUNCH();
  {
    const size_t smem = (size_t)(16 + bwmax) * (16 + 2) * sizeof(double);
    S.queue.alloc(1);
    S.queue.zero(s);
    auto kern = k_band_chol<double, 16>;
    HP_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<std::min(C, 2 * num_sms()), FACT_THREADS, smem, s>>>(S.order.p, C, S.queue.p, S.n.p, S.bw.p,
                                                               S.band_off.p, S.band64.p, c->status.p, 4);
    HP_CHECK_LAUNCH();
  }
  // right-hand sides, solves, and the blocks of Q^o
  std::vector<long long> xoff(C + 1, 0), qoff(C + 1, 0);
  std::vector<int> ld(C);
  for (int ci = 0; ci < C; ++ci) {
    ld[ci] = std::max(c->h_col_off[ci + 1] - c->h_col_off[ci], 1);
    xoff[ci + 1] = xoff[ci] + (long long)S.h_n[ci] * ld[ci];
    qoff[ci + 1] = qoff[ci] + 3LL * (c->h_iface_off[ci + 1] - c->h_iface_off[ci]) * ld[ci];
  }
  Buf<long long> dxoff;
  Buf<int> dld;
  dxoff.upload(xoff, s);
  dld.upload(ld, s);
  c->qoff.upload(qoff, s);
  Buf<double> X;
  X.alloc(std::max<long long>(xoff[C], 1));
  X.zero(s);
  k_iface_rhs<<<C, 128, 0, s>>>(S.node_off.p, S.n.p, S.lnodes.p, c->row_ptr.p, c->col.p, c->val64.p, c->fixed.p,
                                c->iface_of_node.p, c->mslot_of_node.p, c->mcol.p, c->mfree.p, dxoff.p, dld.p, X.p);
  HP_CHECK_LAUNCH();
  solve_multi_t<double>(c, S, X.p, dxoff, dld, ld);
  c->qblk.alloc(std::max<long long>(qoff[C], 1));
  c->qblk.zero(s);
  k_iface_store<<<C, 256, 0, s>>>(S.node_off.p, S.n.p, S.lnodes.p, c->iface_slot.p, dxoff.p, dld.p, X.p, c->qoff.p,
                                  c->qblk.p);
  HP_CHECK_LAUNCH();
  HP_CUDA(cudaStreamSynchronize(s));
  S.band64.release();  // the interface factors are not needed after the set-up
}

}  // namespace hp
