// Fine-grid assembly (paper Section 2, Eqs. stiff_iso, BC, ls_all): Q1
// hexahedra on unit voxels, the element stiffness E_e * K_ref(nu), Dirichlet
// elimination and consistent face-traction loads, stored as a node-block
// (3x3) BSR matrix over existing nodes.  Fixed components keep their slot in
// every padded vector but their rows and columns are zero, so all internal
// vectors are [n_nodes][3] with zeros on fixed slots.
#include "common.cuh"

#include <algorithm>

namespace hp {
namespace {

__device__ __forceinline__ int corner_index(int ox, int oy, int oz) { return ox + 2 * oy + 4 * oz; }

__global__ void k_node_exists(const uint8_t *mask, int nx, int ny, int nz, int *flag) {
  long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long NX = nx + 1, NY = ny + 1, NZ = nz + 1;
  if (g >= NX * NY * NZ) return;
  int i = (int)(g % NX), j = (int)((g / NX) % NY), k = (int)(g / (NX * NY));
  int any = 0;
  for (int dk = -1; dk <= 0; ++dk)
    for (int dj = -1; dj <= 0; ++dj)
      for (int di = -1; di <= 0; ++di) {
        int vi = i + di, vj = j + dj, vk = k + dk;
        if (vi < 0 || vj < 0 || vk < 0 || vi >= nx || vj >= ny || vk >= nz) continue;
        any |= mask[((long long)vk * ny + vj) * nx + vi] != 0;
      }
  flag[g] = any;
}

__global__ void k_node_finalize(const int *flag, int *ids, int *node_ijk, int nx, int ny, long long n_grid) {
  long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n_grid) return;
  long long NX = nx + 1, NY = ny + 1;
  if (flag[g]) {
    int id = ids[g];
    node_ijk[3 * id + 0] = (int)(g % NX);
    node_ijk[3 * id + 1] = (int)((g / NX) % NY);
    node_ijk[3 * id + 2] = (int)(g / (NX * NY));
  } else {
    ids[g] = -1;
  }
}

// K_ref(nu): int over the unit cube of B^T D B with 2x2x2 Gauss-Legendre points, E = 1.
// Voigt order (xx,yy,zz,yz,xz,xy), engineering shear; corner a = ax + 2 ay + 4 az.
__global__ void k_kref(double nu, double *K) {
  int r = threadIdx.x / 24, c = threadIdx.x % 24;
  if (threadIdx.x >= 576) return;
  double lam = nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  double mu = 1.0 / (2.0 * (1.0 + nu));
  double D[6][6] = {};
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) D[a][b] = lam;
  for (int a = 0; a < 3; ++a) {
    D[a][a] += 2.0 * mu;
    D[3 + a][3 + a] = mu;
  }
  const double g = 0.5 / sqrt(3.0);
  const double pts[2] = {0.5 - g, 0.5 + g};
  int na = r / 3, da = r % 3, nb = c / 3, db = c % 3;
  double acc = 0.0;
  for (int qz = 0; qz < 2; ++qz)
    for (int qy = 0; qy < 2; ++qy)
      for (int qx = 0; qx < 2; ++qx) {
        double x[3] = {pts[qx], pts[qy], pts[qz]};
        double ga[3], gb[3];
        for (int s = 0; s < 2; ++s) {
          int node = s ? nb : na;
          int o[3] = {node & 1, (node >> 1) & 1, (node >> 2) & 1};
          double f[3], sg[3];
          for (int d = 0; d < 3; ++d) {
            f[d] = o[d] ? x[d] : 1.0 - x[d];
            sg[d] = o[d] ? 1.0 : -1.0;
          }
          double *gg = s ? gb : ga;
          gg[0] = sg[0] * f[1] * f[2];
          gg[1] = f[0] * sg[1] * f[2];
          gg[2] = f[0] * f[1] * sg[2];
        }
        // Voigt strain column for (node, comp): Ba[6]
        double Ba[6] = {}, Bb[6] = {};
        for (int s = 0; s < 2; ++s) {
          double *B = s ? Bb : Ba;
          double *gg = s ? gb : ga;
          int d = s ? db : da;
          if (d == 0) { B[0] = gg[0]; B[4] = gg[2]; B[5] = gg[1]; }
          if (d == 1) { B[1] = gg[1]; B[3] = gg[2]; B[5] = gg[0]; }
          if (d == 2) { B[2] = gg[2]; B[3] = gg[1]; B[4] = gg[0]; }
        }
        double s = 0.0;
        for (int p = 0; p < 6; ++p)
          for (int q = 0; q < 6; ++q) s += Ba[p] * D[p][q] * Bb[q];
        acc += 0.125 * s;
      }
  K[r * 24 + c] = acc;
}

struct BCDev {
  uint8_t fix[6][3];
  double value[6][3];
  double traction[6][3];
};

__global__ void k_bc(const int *node_ijk, int n_nodes, int nx, int ny, int nz, const uint8_t *mask, BCDev bc,
                     uint8_t *fixed, double *uD, double *f) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= n_nodes) return;
  int p[3] = {node_ijk[3 * n], node_ijk[3 * n + 1], node_ijk[3 * n + 2]};
  int lim[3] = {nx, ny, nz};
  uint8_t fx[3] = {0, 0, 0};
  double u[3] = {0, 0, 0}, t[3] = {0, 0, 0};
  for (int face = 0; face < 6; ++face) {
    int ax = face >> 1, side = face & 1;
    int plane = side ? lim[ax] : 0;
    if (p[ax] != plane) continue;
    for (int d = 0; d < 3; ++d)
      if (bc.fix[face][d]) {
        fx[d] = 1;
        u[d] = bc.value[face][d];
      }
    double tr0 = bc.traction[face][0], tr1 = bc.traction[face][1], tr2 = bc.traction[face][2];
    if (tr0 != 0.0 || tr1 != 0.0 || tr2 != 0.0) {
      int layer = side ? lim[ax] - 1 : 0;
      int a1 = (ax + 1) % 3, a2 = (ax + 2) % 3;
      int cnt = 0;
      for (int o1 = -1; o1 <= 0; ++o1)
        for (int o2 = -1; o2 <= 0; ++o2) {
          int v[3];
          v[ax] = layer;
          v[a1] = p[a1] + o1;
          v[a2] = p[a2] + o2;
          if (v[a1] < 0 || v[a2] < 0 || v[a1] >= lim[a1] || v[a2] >= lim[a2]) continue;
          cnt += mask[((long long)v[2] * ny + v[1]) * nx + v[0]] != 0;
        }
      t[0] += 0.25 * cnt * tr0;
      t[1] += 0.25 * cnt * tr1;
      t[2] += 0.25 * cnt * tr2;
    }
  }
  for (int d = 0; d < 3; ++d) {
    fixed[3 * n + d] = fx[d];
    uD[3 * n + d] = u[d];
    f[3 * n + d] = t[d];
  }
}

// neighbour m = n + (dx,dy,dz) is coupled to n when a solid voxel has both as corners
__device__ __forceinline__ bool shares_solid(const uint8_t *mask, int nx, int ny, int nz, int i, int j, int k, int dx,
                                             int dy, int dz) {
  int x0 = max(i - 1, i + dx - 1), x1 = min(i, i + dx);
  int y0 = max(j - 1, j + dy - 1), y1 = min(j, j + dy);
  int z0 = max(k - 1, k + dz - 1), z1 = min(k, k + dz);
  for (int vz = z0; vz <= z1; ++vz)
    for (int vy = y0; vy <= y1; ++vy)
      for (int vx = x0; vx <= x1; ++vx) {
        if (vx < 0 || vy < 0 || vz < 0 || vx >= nx || vy >= ny || vz >= nz) continue;
        if (mask[((long long)vz * ny + vy) * nx + vx]) return true;
      }
  return false;
}

__global__ void k_bsr_count(const int *node_ijk, int n_nodes, const int *g2n, const uint8_t *mask, int nx, int ny,
                            int nz, int *cnt) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= n_nodes) return;
  int i = node_ijk[3 * n], j = node_ijk[3 * n + 1], k = node_ijk[3 * n + 2];
  int c = 0;
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx)
        if (shares_solid(mask, nx, ny, nz, i, j, k, dx, dy, dz)) ++c;
  cnt[n] = c;
}

__global__ void k_bsr_fill(const int *node_ijk, int n_nodes, const int *g2n, const uint8_t *mask, const float *E,
                           int nx, int ny, int nz, const double *Kref, const int *row_ptr, const uint8_t *fixed,
                           const double *uD, const double *f, int *col, double *val64, float *val32, double *b) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= n_nodes) return;
  int i = node_ijk[3 * n], j = node_ijk[3 * n + 1], k = node_ijk[3 * n + 2];
  long long NX = nx + 1, NY = ny + 1;
  int pos = row_ptr[n];
  double rhs[3] = {f[3 * n], f[3 * n + 1], f[3 * n + 2]};
  bool fr[3] = {fixed[3 * n] != 0, fixed[3 * n + 1] != 0, fixed[3 * n + 2] != 0};
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        if (!shares_solid(mask, nx, ny, nz, i, j, k, dx, dy, dz)) continue;
        int m = g2n[((long long)(k + dz) * NY + (j + dy)) * NX + (i + dx)];
        double blk[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        int x0 = max(i - 1, i + dx - 1), x1 = min(i, i + dx);
        int y0 = max(j - 1, j + dy - 1), y1 = min(j, j + dy);
        int z0 = max(k - 1, k + dz - 1), z1 = min(k, k + dz);
        for (int vz = z0; vz <= z1; ++vz)
          for (int vy = y0; vy <= y1; ++vy)
            for (int vx = x0; vx <= x1; ++vx) {
              if (vx < 0 || vy < 0 || vz < 0 || vx >= nx || vy >= ny || vz >= nz) continue;
              long long v = ((long long)vz * ny + vy) * nx + vx;
              if (!mask[v]) continue;
              double e = E[v];
              int a = corner_index(i - vx, j - vy, k - vz);
              int bb = corner_index(i + dx - vx, j + dy - vy, k + dz - vz);
              for (int d = 0; d < 3; ++d)
                for (int d2 = 0; d2 < 3; ++d2) blk[3 * d + d2] += e * Kref[(3 * a + d) * 24 + 3 * bb + d2];
            }
        bool fc[3] = {fixed[3 * m] != 0, fixed[3 * m + 1] != 0, fixed[3 * m + 2] != 0};
        for (int d = 0; d < 3; ++d)
          for (int d2 = 0; d2 < 3; ++d2)
            if (!fr[d] && fc[d2]) rhs[d] -= blk[3 * d + d2] * uD[3 * m + d2];
        for (int d = 0; d < 3; ++d)
          for (int d2 = 0; d2 < 3; ++d2)
            if (fr[d] || fc[d2]) blk[3 * d + d2] = 0.0;
        col[pos] = m;
        for (int q = 0; q < 9; ++q) {
          val64[(long long)pos * 9 + q] = blk[q];
          val32[(long long)pos * 9 + q] = (float)blk[q];
        }
        ++pos;
      }
  for (int d = 0; d < 3; ++d) b[3 * n + d] = fr[d] ? 0.0 : rhs[d];
}

__global__ void k_not_fixed(const uint8_t *fixed, int *flag, long long n) {
  long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n) flag[s] = fixed[s] ? 0 : 1;
}

__global__ void k_free_finalize(const uint8_t *fixed, int *free_index, int *dof_slot, long long n) {
  long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  if (fixed[s]) {
    free_index[s] = -1;
  } else {
    dof_slot[free_index[s]] = (int)s;
  }
}

__global__ void k_gather_free(const int *dof_slot, const double *pad, double *dof, long long n_dof) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_dof) dof[i] = pad[dof_slot[i]];
}

__global__ void k_scatter_free(const int *dof_slot, const double *dof, double *pad, long long n_dof) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_dof) pad[dof_slot[i]] = dof[i];
}

// ---------------------------------------------------------------- sliced-ELL copy of A_hat for the SpMV
// Rows are grouped in slices of 32 (one warp); a slice is padded to its longest row, and stored slot-major
// with the 9 block entries of a slot element-major, so that every load of the SpMV is one contiguous
// 128-byte (FP32) or 256-byte (FP64) access across the warp.  Padding slots point at the row's own node with
// zero values.  The rows are taken longest first within windows of SELL_SIGMA consecutive nodes (sliced ELL
// with local sorting), so that a slice's rows have nearly equal lengths: on a porous image the node degrees
// vary, and slices of 32 consecutive nodes padded about 13% of the slots, each an idle FP64 multiply-add.
constexpr int SELL_SIGMA = 1024;

// perm[window start + position] = node: a stable counting sort of each window's rows by length (longest
// first), one CTA of SELL_SIGMA threads per window; lengths above 30 share the first bucket
__global__ void __launch_bounds__(SELL_SIGMA) k_sell_sort(const int *row_ptr, int n_nodes, int *perm) {
  __shared__ int cnt[32][32];  // [key][warp]: rows of the warp with the key, then the exclusive offsets
  __shared__ int ksum[32];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const long long n = (long long)blockIdx.x * SELL_SIGMA + t;
  const int len = n < n_nodes ? row_ptr[n + 1] - row_ptr[n] : -1;
  const int key = len < 0 ? 31 : 30 - min(len, 30);  // rows past the end sort last and are not written
  cnt[w][lane] = 0;
  __syncthreads();
  const unsigned same = __match_any_sync(0xffffffffu, key);
  const int rank = __popc(same & ((1u << lane) - 1u));
  if (rank == 0) cnt[key][w] = __popc(same);
  __syncthreads();
  // exclusive scan over the entries in (key, warp) order: thread t holds entry (t / 32, t % 32)
  const int v = cnt[w][lane];
  int inc = v;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) ksum[w] = inc;
  __syncthreads();
  if (w == 0) {
    const int s0 = ksum[lane];
    int si = s0;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, si, o);
      if (lane >= o) si += y;
    }
    ksum[lane] = si - s0;
  }
  __syncthreads();
  cnt[w][lane] = inc - v + ksum[w];
  __syncthreads();
  if (len >= 0) perm[(long long)blockIdx.x * SELL_SIGMA + cnt[key][w] + rank] = (int)n;
}

__global__ void k_sell_width(const int *row_ptr, const int *perm, int n_nodes, int n_slices, int *width) {
  int sl = blockIdx.x * blockDim.x + threadIdx.x;
  if (sl >= n_slices) return;
  int w = 0;
  for (int i = sl * 32; i < min(n_nodes, sl * 32 + 32); ++i) {
    const int r = perm[i];
    w = max(w, row_ptr[r + 1] - row_ptr[r]);
  }
  width[sl] = 32 * w;  // entries of the slice
}

__global__ void k_sell_fill(const int *row_ptr, const int *col, const double *val, const int *perm, int n_nodes,
                            const int *slice_off, int *scol, double *sval64, float *sval32) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  int sl = n >> 5, lane = n & 31;
  if (sl * 32 >= n_nodes) return;
  long long base = slice_off[sl];
  int w = (slice_off[sl + 1] - slice_off[sl]) / 32;
  const int node = n < n_nodes ? perm[n] : 0;
  int b = (n < n_nodes) ? row_ptr[node] : 0, len = (n < n_nodes) ? row_ptr[node + 1] - b : 0;
  for (int j = 0; j < w; ++j) {
    long long ent = base + (long long)j * 32 + lane;
    scol[ent] = (j < len) ? col[b + j] : node;
    for (int e = 0; e < 9; ++e) {
      double v = (j < len) ? val[(long long)(b + j) * 9 + e] : 0.0;
      long long at = (base + (long long)j * 32) * 9 + (long long)e * 32 + lane;
      sval64[at] = v;
      if (sval32) sval32[at] = (float)v;
    }
  }
}

// y = A x (or y = sub - A x when sub != nullptr) on the sliced-ELL copy; one thread per row position n (node
// perm[n]).  The FP64 form is bound by the FP64 pipe; 64-thread blocks (about 23 per SM, all resident) keep the
// SMs' shares of the uneven slices close to one another.
template <typename T>
__global__ void k_spmv_sell(const int *slice_off, const int *scol, const T *sval, const int *perm, const double *x,
                            double *y, const double *sub, int n_nodes) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= n_nodes) return;
  const int node = perm[n];
  using A = typename std::conditional<std::is_same<T, double>::value, double, float>::type;
  const int sl = n >> 5, lane = n & 31;
  const long long base = slice_off[sl];
  const int w = (slice_off[sl + 1] - slice_off[sl]) >> 5;
  A s0 = 0, s1 = 0, s2 = 0;
  for (int j = 0; j < w; ++j) {
    const long long slot = base + (long long)j * 32;
    const int m = scol[slot + lane];
    const T *v = sval + slot * 9 + lane;
    A x0 = (A)x[3 * m], x1 = (A)x[3 * m + 1], x2 = (A)x[3 * m + 2];
    // one multiply-add per entry into the running sums (a product summed into a partial first would cost
    // an extra multiply and add, and the FP64 form is bound by the FP64 pipe)
    s0 += (A)v[0] * x0;
    s0 += (A)v[32] * x1;
    s0 += (A)v[64] * x2;
    s1 += (A)v[96] * x0;
    s1 += (A)v[128] * x1;
    s1 += (A)v[160] * x2;
    s2 += (A)v[192] * x0;
    s2 += (A)v[224] * x1;
    s2 += (A)v[256] * x2;
  }
  if (sub) {
    y[3 * node] = sub[3 * node] - (double)s0;
    y[3 * node + 1] = sub[3 * node + 1] - (double)s1;
    y[3 * node + 2] = sub[3 * node + 2] - (double)s2;
  } else {
    y[3 * node] = (double)s0;
    y[3 * node + 1] = (double)s1;
    y[3 * node + 2] = (double)s2;
  }
}

// y = A_hat x (or sub - A_hat x) element by element, in FP32 (the residual updates of the FP32 and BF16
// apply forms): A_hat = sum over solid voxels e of E_e K_ref, so the row block of node n is rebuilt from the
// moduli of its (up to) eight voxels and the 24 x 24 reference stiffness, which the kernel receives as a
// parameter (constant memory, read with compile-time offsets).  Thread per node: the 27 neighbours' values
// into registers (absent neighbours as zeros), then per voxel t = K_ref[corner of n][.] x_voxel and
// y += E_e t.  Vectors are zero on fixed slots (the columns of fixed DOFs drop out) and the rows of fixed
// DOFs are zero, as in the assembled A_hat.  It reads the moduli, the node map and the vectors instead of
// A_hat's 36 bytes per block.
struct KRef32 {
  float k[576];
};

// FP32 copy of a vector: each value is converted once (a node's 27 neighbours would otherwise convert it
// 27 times, and FP64 -> FP32 conversions run at the FP64 rate)
__global__ void k_vec_to_f32(const double *x, float *xf, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) xf[i] = (float)x[i];
}

__global__ void __launch_bounds__(256) k_spmv_ebe32(const int *node_ijk, int n_nodes, const int *g2n,
                                                    const uint8_t *mask, const float *E, int nx, int ny, int nz,
                                                    const __grid_constant__ KRef32 K, const uint8_t *fixed,
                                                    const float *x, double *y, const double *sub) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= n_nodes) return;
  const int i = node_ijk[3 * n], j = node_ijk[3 * n + 1], k = node_ijk[3 * n + 2];
  const long long NX = nx + 1, NY = ny + 1;
  float xv[27][3];
#pragma unroll
  for (int q = 0; q < 27; ++q) {
    const int dx = q % 3 - 1, dy = (q / 3) % 3 - 1, dz = q / 9 - 1;
    const int ii = i + dx, jj = j + dy, kk = k + dz;
    int m = -1;
    if (ii >= 0 && jj >= 0 && kk >= 0 && ii <= nx && jj <= ny && kk <= nz) m = g2n[((long long)kk * NY + jj) * NX + ii];
#pragma unroll
    for (int d = 0; d < 3; ++d) xv[q][d] = m >= 0 ? x[3LL * m + d] : 0.f;
  }
  float acc[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int oz = 0; oz < 2; ++oz)
#pragma unroll
    for (int oy = 0; oy < 2; ++oy)
#pragma unroll
      for (int ox = 0; ox < 2; ++ox) {
        // voxel (i - 1 + ox, j - 1 + oy, k - 1 + oz); node n is its corner (1 - ox, 1 - oy, 1 - oz)
        const int vx = i - 1 + ox, vy = j - 1 + oy, vz = k - 1 + oz;
        if (vx < 0 || vy < 0 || vz < 0 || vx >= nx || vy >= ny || vz >= nz) continue;
        const long long v = ((long long)vz * ny + vy) * nx + vx;
        if (!mask[v]) continue;
        const float e = E[v];
        const int a = (1 - ox) + 2 * (1 - oy) + 4 * (1 - oz);
        float t[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int bb = 0; bb < 8; ++bb) {
          const int cx = bb & 1, cy = (bb >> 1) & 1, cz = bb >> 2;
          const int q = (ox - 1 + cx + 1) + 3 * (oy - 1 + cy + 1) + 9 * (oz - 1 + cz + 1);
#pragma unroll
          for (int d = 0; d < 3; ++d)
#pragma unroll
            for (int d2 = 0; d2 < 3; ++d2) t[d] = fmaf(K.k[(3 * a + d) * 24 + 3 * bb + d2], xv[q][d2], t[d]);
        }
#pragma unroll
        for (int d = 0; d < 3; ++d) acc[d] = fmaf(e, t[d], acc[d]);
      }
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const long long r = 3LL * n + d;
    const double av = fixed[r] ? 0.0 : (double)acc[d];
    y[r] = sub ? sub[r] - av : av;
  }
}

// Y_q = A X_q (or SUB_q - A X_q) for up to four vectors q < kc, at stride L: the matrix is read once for the
// group (the multi-right-hand-side solve shares one preconditioner over several load cases)
template <typename T>
__global__ void k_spmv_sell4(const int *slice_off, const int *scol, const T *sval, const int *perm, const double *x,
                             double *y, const double *sub, int n_nodes, long long L, int kc) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= n_nodes) return;
  const int node = perm[n];
  using A = typename std::conditional<std::is_same<T, double>::value, double, float>::type;
  const int sl = n >> 5, lane = n & 31;
  const long long base = slice_off[sl];
  const int w = (slice_off[sl + 1] - slice_off[sl]) >> 5;
  A s[4][3] = {};
  for (int j = 0; j < w; ++j) {
    const long long slot = base + (long long)j * 32;
    const int m = scol[slot + lane];
    const T *v = sval + slot * 9 + lane;
    A a[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) a[e] = (A)v[32 * e];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (q < kc) {
        const double *xq = x + q * L + 3LL * m;
        const A x0 = (A)xq[0], x1 = (A)xq[1], x2 = (A)xq[2];
        s[q][0] += a[0] * x0 + a[1] * x1 + a[2] * x2;
        s[q][1] += a[3] * x0 + a[4] * x1 + a[5] * x2;
        s[q][2] += a[6] * x0 + a[7] * x1 + a[8] * x2;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (q >= kc) continue;
    double *yq = y + q * L + 3LL * node;
    if (sub) {
      const double *sq = sub + q * L + 3LL * node;
      yq[0] = sq[0] - (double)s[q][0];
      yq[1] = sq[1] - (double)s[q][1];
      yq[2] = sq[2] - (double)s[q][2];
    } else {
      yq[0] = (double)s[q][0];
      yq[1] = (double)s[q][1];
      yq[2] = (double)s[q][2];
    }
  }
}

}  // namespace

// first solid voxel whose modulus is not a positive finite number (atomic minimum of its index)
__global__ void k_bad_modulus(const uint8_t *mask, const float *E, long long nvox, long long *first) {
  long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nvox || !mask[v]) return;
  const float e = E[v];
  if (!(e > 0.f) || !isfinite(e)) atomicMin((unsigned long long *)first, (unsigned long long)v);
}

void assemble(hplmm_ctx *c, const uint8_t *mask, int nx, int ny, int nz, const float *E, double E0, double nu,
              const hplmm_bcs *bcs, double *b_out) {
  HP_REQUIRE(mask != nullptr && bcs != nullptr, HPLMM_ERR_INVALID, "assemble: mask and bcs are required");
  HP_REQUIRE(nx > 0 && ny > 0 && nz > 0, HPLMM_ERR_INVALID, "assemble: image dimensions must be positive");
  HP_REQUIRE(nu > -1.0 && nu < 0.5, HPLMM_ERR_INVALID, "assemble: Poisson ratio must lie in (-1, 0.5)");
  HP_REQUIRE((long long)(nx + 1) * (ny + 1) * (nz + 1) < (1LL << 31), HPLMM_ERR_INVALID,
             "assemble: image too large for 32-bit node indices");
  cudaStream_t s = c->stream;
  c->assembled = false;
  c->setup_done = false;
  drop_apply_graph(c);
  c->nx = nx;
  c->ny = ny;
  c->nz = nz;
  c->nu = nu;
  c->E0 = E0;
  long long nvox = (long long)nx * ny * nz;
  c->mask.alloc(nvox);
  HP_CUDA(cudaMemcpyAsync(c->mask.p, mask, nvox, cudaMemcpyDeviceToDevice, s));
  c->E.alloc(nvox);
  if (E) {
    HP_CUDA(cudaMemcpyAsync(c->E.p, E, nvox * sizeof(float), cudaMemcpyDeviceToDevice, s));
  } else {
    std::vector<float> h(nvox, (float)E0);
    HP_CUDA(cudaMemcpyAsync(c->E.p, h.data(), nvox * sizeof(float), cudaMemcpyHostToDevice, s));
    HP_CUDA(cudaStreamSynchronize(s));
  }
  {
    // a solid voxel with E <= 0, NaN or infinite would make A_hat indefinite or undefined
    Buf<long long> first;
    first.alloc(1);
    first.fill_bytes(0x7f, s);
    k_bad_modulus<<<grid_for(nvox, 256), 256, 0, s>>>(c->mask.p, c->E.p, nvox, first.p);
    HP_CHECK_LAUNCH();
    const long long v = first.download(s, 1)[0];
    HP_REQUIRE(v >= nvox, HPLMM_ERR_INVALID,
               "assemble: solid voxel (" + std::to_string(v % nx) + ", " + std::to_string((v / nx) % ny) + ", " +
                   std::to_string(v / ((long long)nx * ny)) + ") has a modulus that is not a positive finite number");
  }
  c->n_grid = (long long)(nx + 1) * (ny + 1) * (nz + 1);
  Buf<int> flag;
  flag.alloc(c->n_grid);
  c->grid_to_node.alloc(c->n_grid);
  k_node_exists<<<grid_for(c->n_grid, 256), 256, 0, s>>>(c->mask.p, nx, ny, nz, flag.p);
  HP_CHECK_LAUNCH();
  long long nn = exclusive_scan_i32(flag.p, c->grid_to_node.p, c->n_grid, s);
  HP_REQUIRE(nn > 0, HPLMM_ERR_INVALID, "assemble: the image has no solid voxel");
  c->n_nodes = (int)nn;
  c->node_ijk.alloc(3 * nn);
  k_node_finalize<<<grid_for(c->n_grid, 256), 256, 0, s>>>(flag.p, c->grid_to_node.p, c->node_ijk.p, nx, ny,
                                                           c->n_grid);
  HP_CHECK_LAUNCH();
  c->Kref.alloc(576);
  k_kref<<<1, 576, 0, s>>>(nu, c->Kref.p);
  HP_CHECK_LAUNCH();
  {
    const std::vector<double> kh = c->Kref.download(s);
    c->h_kref32.assign(kh.begin(), kh.end());  // FP32 copy for the element-by-element residual updates
  }

  BCDev bc;
  for (int f = 0; f < 6; ++f)
    for (int d = 0; d < 3; ++d) {
      bc.fix[f][d] = bcs->fix[f][d] ? 1 : 0;
      bc.value[f][d] = bcs->value[f][d];
      bc.traction[f][d] = bcs->traction[f][d];
    }
  long long nslot = 3LL * nn;
  c->fixed.alloc(nslot);
  Buf<double> uD, f;
  uD.alloc(nslot);
  f.alloc(nslot);
  k_bc<<<grid_for(nn, 256), 256, 0, s>>>(c->node_ijk.p, c->n_nodes, nx, ny, nz, c->mask.p, bc, c->fixed.p, uD.p,
                                         f.p);
  HP_CHECK_LAUNCH();

  c->row_ptr.alloc(nn + 1);
  Buf<int> cnt;
  cnt.alloc(nn + 1);
  k_bsr_count<<<grid_for(nn, 256), 256, 0, s>>>(c->node_ijk.p, c->n_nodes, c->grid_to_node.p, c->mask.p, nx, ny, nz,
                                                 cnt.p);
  HP_CHECK_LAUNCH();
  HP_CUDA(cudaMemsetAsync(cnt.p + nn, 0, sizeof(int), s));
  c->nnzb = exclusive_scan_i32(cnt.p, c->row_ptr.p, nn + 1, s);
  c->col.alloc(c->nnzb);
  c->val64.alloc(c->nnzb * 9);
  c->val32.alloc(c->nnzb * 9);
  c->b_pad.alloc(nslot);
  k_bsr_fill<<<grid_for(nn, 128), 128, 0, s>>>(c->node_ijk.p, c->n_nodes, c->grid_to_node.p, c->mask.p, c->E.p, nx,
                                               ny, nz, c->Kref.p, c->row_ptr.p, c->fixed.p, uD.p, f.p, c->col.p,
                                               c->val64.p, c->val32.p, c->b_pad.p);
  HP_CHECK_LAUNCH();

  c->free_index.alloc(nslot);
  Buf<int> freeflag;
  freeflag.alloc(nslot);
  k_not_fixed<<<grid_for(nslot, 256), 256, 0, s>>>(c->fixed.p, freeflag.p, nslot);
  HP_CHECK_LAUNCH();
  c->n_dof = exclusive_scan_i32(freeflag.p, c->free_index.p, nslot, s);
  c->dof_slot.alloc(c->n_dof);
  k_free_finalize<<<grid_for(nslot, 256), 256, 0, s>>>(c->fixed.p, c->free_index.p, c->dof_slot.p, nslot);
  HP_CHECK_LAUNCH();
  // sliced-ELL copies (FP64 and the FP32 shadow) for the SpMV; the CSR FP32 values are then dropped
  {
    int nsl = (int)((nn + 31) / 32);
    c->sell_perm.alloc(nn);
    k_sell_sort<<<grid_for(nn, SELL_SIGMA), SELL_SIGMA, 0, s>>>(c->row_ptr.p, c->n_nodes, c->sell_perm.p);
    HP_CHECK_LAUNCH();
    c->sell_off.alloc(nsl + 1);
    k_sell_width<<<grid_for(nsl, 256), 256, 0, s>>>(c->row_ptr.p, c->sell_perm.p, c->n_nodes, nsl, c->sell_off.p);
    HP_CHECK_LAUNCH();
    HP_CUDA(cudaMemsetAsync(c->sell_off.p + nsl, 0, sizeof(int), s));
    long long nent = exclusive_scan_i32(c->sell_off.p, c->sell_off.p, nsl + 1, s);
    HP_REQUIRE(nent < (1LL << 31), HPLMM_ERR_INVALID, "assemble: too many blocks for 32-bit SpMV offsets");
    c->sell_col.alloc(nent);
    c->sell_val64.alloc(nent * 9);
    // the FP32 copy serves only the assembled FP32 residual updates (matrix_free_updates = 0)
    if (c->opt.matrix_free_updates)
      c->sell_val32.release();
    else
      c->sell_val32.alloc(nent * 9);
    k_sell_fill<<<grid_for((long long)nsl * 32, 128), 128, 0, s>>>(c->row_ptr.p, c->col.p, c->val64.p,
                                                                   c->sell_perm.p, c->n_nodes, c->sell_off.p,
                                                                   c->sell_col.p, c->sell_val64.p, c->sell_val32.p);
    HP_CHECK_LAUNCH();
    c->val32.release();
  }
  // every connected solid part needs a prescribed displacement, else A_hat is singular (rigid motions)
  check_anchored(c);
  if (b_out) gather_free(c, c->b_pad.p, b_out);
  HP_CUDA(cudaStreamSynchronize(s));
  c->assembled = true;
}

void gather_free(hplmm_ctx *c, const double *pad, double *dof) {
  k_gather_free<<<grid_for(c->n_dof, 256), 256, 0, c->stream>>>(c->dof_slot.p, pad, dof, c->n_dof);
  HP_CHECK_LAUNCH();
}

void scatter_free(hplmm_ctx *c, const double *dof, double *pad) {
  HP_CUDA(cudaMemsetAsync(pad, 0, sizeof(double) * 3 * (size_t)c->n_nodes, c->stream));
  k_scatter_free<<<grid_for(c->n_dof, 256), 256, 0, c->stream>>>(c->dof_slot.p, dof, pad, c->n_dof);
  HP_CHECK_LAUNCH();
}

void spmv(hplmm_ctx *c, const double *x_pad, double *y_pad, hplmm_prec prec, const double *sub) {
  ProfScope ps(c, HPLMM_PH_SPMV);
  const unsigned grid = grid_for(c->n_nodes, 64);
  const int *off = c->sell_off.p, *col = c->sell_col.p, *perm = c->sell_perm.p;
  // the BF16 form keeps A_hat in FP32: its residual updates r - A_hat z subtract nearly equal vectors, and
  // A_hat rounded to BF16 (8-bit significand) left errors of the size of the difference on stiffness
  // contrasts of 1e4 (measured: 300 instead of 178 FGMRES iterations on a fractured 128^3 block)
  if (prec == HPLMM_FP64) {
    k_spmv_sell<double><<<grid, 64, 0, c->stream>>>(off, col, c->sell_val64.p, perm, x_pad, y_pad, sub, c->n_nodes);
  } else if (c->opt.matrix_free_updates) {
    KRef32 K;
    for (int e = 0; e < 576; ++e) K.k[e] = c->h_kref32[e];
    const long long L = 3LL * c->n_nodes;
    if ((long long)c->w_x32.n < L) c->w_x32.alloc(L);
    k_vec_to_f32<<<grid_for(L, 256), 256, 0, c->stream>>>(x_pad, c->w_x32.p, L);
    HP_CHECK_LAUNCH();
    k_spmv_ebe32<<<grid_for(c->n_nodes, 256), 256, 0, c->stream>>>(c->node_ijk.p, c->n_nodes, c->grid_to_node.p,
                                                                    c->mask.p, c->E.p, c->nx, c->ny, c->nz, K,
                                                                    c->fixed.p, c->w_x32.p, y_pad, sub);
  } else {
    k_spmv_sell<float><<<grid, 64, 0, c->stream>>>(off, col, c->sell_val32.p, perm, x_pad, y_pad, sub, c->n_nodes);
  }
  HP_CHECK_LAUNCH();
}

void spmv_multi(hplmm_ctx *c, const double *X, double *Y, int k, hplmm_prec prec, const double *SUB) {
  if (prec != HPLMM_FP64 && c->opt.matrix_free_updates) {
    // element by element there is no matrix to share between the vectors: one product per vector
    const long long L = 3LL * c->n_nodes;
    for (int q = 0; q < k; ++q) spmv(c, X + q * L, Y + q * L, prec, SUB ? SUB + q * L : nullptr);
    return;
  }
  ProfScope ps(c, HPLMM_PH_SPMV);
  const unsigned grid = grid_for(c->n_nodes, 64);
  const long long L = 3LL * c->n_nodes;
  const int *off = c->sell_off.p, *col = c->sell_col.p, *perm = c->sell_perm.p;
  for (int q0 = 0; q0 < k; q0 += 4) {
    const int kc = std::min(4, k - q0);
    const double *sub = SUB ? SUB + q0 * L : nullptr;
    if (prec == HPLMM_FP64)
      k_spmv_sell4<double><<<grid, 64, 0, c->stream>>>(off, col, c->sell_val64.p, perm, X + q0 * L, Y + q0 * L, sub,
                                                       c->n_nodes, L, kc);
    else
      k_spmv_sell4<float><<<grid, 64, 0, c->stream>>>(off, col, c->sell_val32.p, perm, X + q0 * L, Y + q0 * L, sub,
                                                      c->n_nodes, L, kc);
    HP_CHECK_LAUNCH();
  }
}

}  // namespace hp
