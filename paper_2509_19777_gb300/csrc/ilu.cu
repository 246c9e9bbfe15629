// ILU(0) base smoother M_ILU(0): the black-box alternative to the contact-grain smoother in the paper's
// smoother comparison (Section 4.1 names ILU(k) as a base smoother M_l of Eq. local_smoother; Section 5
// runs it with fill level 0 and n_st = 6 stages).
//
// The factor lives in a copy of A_hat's node-block storage (BSR, 3x3 blocks, block columns ascending in
// each row), so its pattern is the structural one: DOFs coupled when their nodes share a solid voxel.
// Elimination runs over the DOFs in slot order (node-major, nodes lexicographic with x fastest), the
// order of the free DOFs; fixed slots carry zero rows and columns and are skipped.  L (unit lower) and U
// share the storage: row (n, a) holds L left of its diagonal and U from it on.
//
// Schedule: a node's rows need only the rows of its neighbours with smaller ids.  Such a neighbour
// (dx, dy, dz) has dz < 0, or dz = 0 and dy < 0, or dz = dy = 0 and dx < 0, so the level
// lambda = i + 2 j + 4 k of node (i, j, k) is strictly smaller for it (the largest difference is
// 1 + 2 - 4 = -1), and nodes of one level are independent.  The factorisation and the forward solve run
// one launch per non-empty level in ascending order, the backward solve in descending order; one warp
// handles one node (its three rows in sequence, the entries of a row across the lanes).
#include "common.cuh"

namespace hp {
namespace {

constexpr int ILU_WARPS = 4;  // nodes per block

__global__ void k_ilu_level(const int *node_ijk, int n_nodes, int *lev) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n < n_nodes) lev[n] = node_ijk[3 * n] + 2 * node_ijk[3 * n + 1] + 4 * node_ijk[3 * n + 2];
}

// position of the diagonal block of every node row (the node shares a solid voxel with itself)
__global__ void k_ilu_diag(const int *row_ptr, const int *col, int n_nodes, int *diag) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= n_nodes) return;
  int lo = row_ptr[n], hi = row_ptr[n + 1] - 1, at = -1;
  while (lo <= hi) {
    const int mid = (lo + hi) >> 1, v = col[mid];
    if (v == n) {
      at = mid;
      break;
    }
    if (v < n)
      lo = mid + 1;
    else
      hi = mid - 1;
  }
  diag[n] = at;
}

// Row-oriented ILU(0) of the rows of one level's nodes.  For row i = (n, a), in increasing column order
// k < i within the pattern: l_ik = a_ik / u_kk, then a_ij -= l_ik u_kj for every j > k of row k that
// row i's pattern holds (updates outside it are dropped).
__global__ void __launch_bounds__(ILU_WARPS * 32)
    k_ilu0_level(const int *__restrict__ nodes, int cnt, const int *__restrict__ row_ptr,
                 const int *__restrict__ col, const int *__restrict__ diag, const uint8_t *__restrict__ fixed,
                 double *val, int *status) {
  __shared__ int s_col[ILU_WARPS][32];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = blockIdx.x * ILU_WARPS + wid;
  if (t >= cnt) return;  // uniform over the warp
  const int n = nodes[t];
  const int rb = row_ptr[n], nb = row_ptr[n + 1] - rb;  // at most 27 blocks
  const int dp = diag[n];
  int *sc = s_col[wid];
  if (lane < nb) sc[lane] = col[rb + lane];
  __syncwarp();
  for (int a = 0; a < 3; ++a) {
    if (fixed[3 * n + a]) continue;
    // with the rows of earlier nodes: blocks rb .. dp-1 in ascending node order, components 0..2
    for (int q = rb; q < dp; ++q) {
      const int m = sc[q - rb];
      const int md = diag[m], me = row_ptr[m + 1];
      for (int b = 0; b < 3; ++b) {
        if (fixed[3 * m + b]) continue;
        const double l = val[(long long)q * 9 + a * 3 + b] / val[(long long)md * 9 + b * 4];
        __syncwarp();
        if (lane == 0) val[(long long)q * 9 + a * 3 + b] = l;
        // row (m, b) right of its diagonal: entries e = 3 (block - md) + component, e > b
        const int ne = 3 * (me - md);
        for (int e = b + 1 + lane; e < ne; e += 32) {
          const int qq = md + e / 3, bb = e - 3 * (e / 3);
          const int target = col[qq];
          int lo = 0, hi = nb - 1, p = -1;
          while (lo <= hi) {
            const int mid = (lo + hi) >> 1, v = sc[mid];
            if (v == target) {
              p = rb + mid;
              break;
            }
            if (v < target)
              lo = mid + 1;
            else
              hi = mid - 1;
          }
          if (p >= 0) val[(long long)p * 9 + a * 3 + bb] -= l * val[(long long)qq * 9 + b * 3 + bb];
        }
        __syncwarp();
      }
    }
    // with the earlier rows of this node, (n, b) for b < a: same block row, so every entry is in the pattern
    for (int b = 0; b < a; ++b) {
      if (fixed[3 * n + b]) continue;
      const double l = val[(long long)dp * 9 + a * 3 + b] / val[(long long)dp * 9 + b * 4];
      __syncwarp();
      if (lane == 0) val[(long long)dp * 9 + a * 3 + b] = l;
      const int ne = 3 * (rb + nb - dp);
      for (int e = b + 1 + lane; e < ne; e += 32) {
        const int qq = dp + e / 3, bb = e - 3 * (e / 3);
        val[(long long)qq * 9 + a * 3 + bb] -= l * val[(long long)qq * 9 + b * 3 + bb];
      }
      __syncwarp();
    }
    if (lane == 0) {
      const double u = val[(long long)dp * 9 + a * 4];
      if (!(u != 0.0) || !isfinite(u)) {
        if (atomicCAS(status, 0, (int)HPLMM_ERR_SINGULAR) == 0) {
          status[1] = 5;
          status[2] = n;
          status[3] = a;
        }
      }
    }
    __syncwarp();
  }
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// y = L^{-1} r on one level's nodes (L unit lower)
__global__ void __launch_bounds__(ILU_WARPS * 32)
    k_ilu_fwd(const int *__restrict__ nodes, int cnt, const int *__restrict__ row_ptr, const int *__restrict__ col,
              const int *__restrict__ diag, const uint8_t *__restrict__ fixed, const double *__restrict__ val,
              const double *__restrict__ r, double *y) {
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = blockIdx.x * ILU_WARPS + wid;
  if (t >= cnt) return;
  const int n = nodes[t];
  const int rb = row_ptr[n], dp = diag[n];
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  const int ne = 3 * (dp - rb);
  for (int e = lane; e < ne; e += 32) {
    const int q = rb + e / 3, b = e - 3 * (e / 3);
    const double yv = y[3LL * col[q] + b];
    const double *v = val + (long long)q * 9 + b;
    s0 += v[0] * yv;
    s1 += v[3] * yv;
    s2 += v[6] * yv;
  }
  s0 = warp_sum(s0);
  s1 = warp_sum(s1);
  s2 = warp_sum(s2);
  if (lane == 0) {
    const double *d = val + (long long)dp * 9;
    const long long o = 3LL * n;
    const double y0 = fixed[o] ? 0.0 : r[o] - s0;
    const double y1 = fixed[o + 1] ? 0.0 : r[o + 1] - s1 - d[3] * y0;
    const double y2 = fixed[o + 2] ? 0.0 : r[o + 2] - s2 - d[6] * y0 - d[7] * y1;
    y[o] = y0;
    y[o + 1] = y1;
    y[o + 2] = y2;
  }
}

// z = U^{-1} y on one level's nodes, in place (z holds y on entry)
__global__ void __launch_bounds__(ILU_WARPS * 32)
    k_ilu_bwd(const int *__restrict__ nodes, int cnt, const int *__restrict__ row_ptr, const int *__restrict__ col,
              const int *__restrict__ diag, const uint8_t *__restrict__ fixed, const double *__restrict__ val,
              double *z) {
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = blockIdx.x * ILU_WARPS + wid;
  if (t >= cnt) return;
  const int n = nodes[t];
  const int re = row_ptr[n + 1], dp = diag[n];
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  const int ne = 3 * (re - dp - 1);
  for (int e = lane; e < ne; e += 32) {
    const int q = dp + 1 + e / 3, b = e - 3 * (e / 3);
    const double zv = z[3LL * col[q] + b];
    const double *v = val + (long long)q * 9 + b;
    s0 += v[0] * zv;
    s1 += v[3] * zv;
    s2 += v[6] * zv;
  }
  s0 = warp_sum(s0);
  s1 = warp_sum(s1);
  s2 = warp_sum(s2);
  if (lane == 0) {
    const double *d = val + (long long)dp * 9;
    const long long o = 3LL * n;
    const double z2 = fixed[o + 2] ? 0.0 : (z[o + 2] - s2) / d[8];
    const double z1 = fixed[o + 1] ? 0.0 : (z[o + 1] - s1 - d[5] * z2) / d[4];
    const double z0 = fixed[o] ? 0.0 : (z[o] - s0 - d[1] * z1 - d[2] * z2) / d[0];
    z[o] = z0;
    z[o + 1] = z1;
    z[o + 2] = z2;
  }
}

}  // namespace

void ilu_setup(hplmm_ctx *c) {
  ProfScope ps(c, HPLMM_PH_FACTOR_ILU);
  cudaStream_t s = c->stream;
  const int nn = c->n_nodes;
  // levels: a stable counting sort of the nodes by lambda (ascending node id inside a level)
  Buf<int> lev;
  lev.alloc(nn);
  k_ilu_level<<<grid_for(nn, 256), 256, 0, s>>>(c->node_ijk.p, nn, lev.p);
  HP_CHECK_LAUNCH();
  const std::vector<int> hl = lev.download(s);
  const int nlev = c->nx + 2 * c->ny + 4 * c->nz + 1;
  std::vector<int> start(nlev + 1, 0);
  for (int n = 0; n < nn; ++n) {
    HP_REQUIRE(hl[n] >= 0 && hl[n] < nlev, HPLMM_ERR_INVALID, "ilu_setup: node outside the image grid");
    ++start[hl[n] + 1];
  }
  for (int l = 0; l < nlev; ++l) start[l + 1] += start[l];
  std::vector<int> order(nn), fill(start.begin(), start.end() - 1);
  for (int n = 0; n < nn; ++n) order[fill[hl[n]]++] = n;
  c->h_ilu_off.clear();
  for (int l = 0; l < nlev; ++l)
    if (start[l + 1] > start[l]) c->h_ilu_off.push_back(start[l]);
  c->h_ilu_off.push_back(nn);
  c->ilu_nodes.alloc(nn);
  c->ilu_nodes.upload(order, s);
  c->ilu_diag.alloc(nn);
  k_ilu_diag<<<grid_for(nn, 256), 256, 0, s>>>(c->row_ptr.p, c->col.p, nn, c->ilu_diag.p);
  HP_CHECK_LAUNCH();
  c->ilu_val.alloc(c->nnzb * 9);
  HP_CUDA(cudaMemcpyAsync(c->ilu_val.p, c->val64.p, sizeof(double) * 9 * (size_t)c->nnzb, cudaMemcpyDeviceToDevice,
                          s));
  for (size_t l = 0; l + 1 < c->h_ilu_off.size(); ++l) {
    const int off = c->h_ilu_off[l], cnt = c->h_ilu_off[l + 1] - off;
    k_ilu0_level<<<(cnt + ILU_WARPS - 1) / ILU_WARPS, ILU_WARPS * 32, 0, s>>>(
        c->ilu_nodes.p + off, cnt, c->row_ptr.p, c->col.p, c->ilu_diag.p, c->fixed.p, c->ilu_val.p, c->status.p);
    HP_CHECK_LAUNCH();
  }
}

void ilu_stage(hplmm_ctx *c, const double *r_pad, double *z_pad) {
  ProfScope ps(c, HPLMM_PH_APPLY_ILU);
  cudaStream_t s = c->stream;
  const int nl = (int)c->h_ilu_off.size() - 1;
  HP_REQUIRE(nl >= 1, HPLMM_ERR_STATE, "ILU(0) smoother: no factor (set-up incomplete)");
  for (int l = 0; l < nl; ++l) {
    const int off = c->h_ilu_off[l], cnt = c->h_ilu_off[l + 1] - off;
    k_ilu_fwd<<<(cnt + ILU_WARPS - 1) / ILU_WARPS, ILU_WARPS * 32, 0, s>>>(
        c->ilu_nodes.p + off, cnt, c->row_ptr.p, c->col.p, c->ilu_diag.p, c->fixed.p, c->ilu_val.p, r_pad, z_pad);
    HP_CHECK_LAUNCH();
  }
  for (int l = nl - 1; l >= 0; --l) {
    const int off = c->h_ilu_off[l], cnt = c->h_ilu_off[l + 1] - off;
    k_ilu_bwd<<<(cnt + ILU_WARPS - 1) / ILU_WARPS, ILU_WARPS * 32, 0, s>>>(
        c->ilu_nodes.p + off, cnt, c->row_ptr.p, c->col.p, c->ilu_diag.p, c->fixed.p, c->ilu_val.p, z_pad);
    HP_CHECK_LAUNCH();
  }
}

}  // namespace hp
