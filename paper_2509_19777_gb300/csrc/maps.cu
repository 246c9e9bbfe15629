// Grain grids, contact interfaces, couplings and mortars (paper Sections
// 3.1-3.3, 4.2; Eqs. permute, node_init, gauss, reduced_defs).
//
// Readings of points the paper leaves open (identical to the CPU oracle's):
//  * S(node) = grains of the node's solid adjacent voxels; |S| = 1 -> interior
//    node of that grain, |S| >= 2 -> interface node of the pair (min S, second
//    smallest S), since an interface is shared by exactly two grains (Sec. 3.2).
//  * one pair may share several interfaces: its nodes are split into connected
//    components, two nodes being adjacent when a solid voxel has both as corners;
//    nodes without a free DOF belong to no class.
//  * interfaces are ordered by (pair, smallest node id); W lists grain interiors
//    then interfaces, each in node order.
//  * grain g is coupled to interface c when a node of c is a corner of a solid
//    voxel of g; in strict mode only c's two grains get nonzero shape vectors.
//  * mortar placement works in node-index units with exact integer squared
//    distances; the energy sum_j 1/||y - x_j|| is accumulated in ascending mortar
//    order with correctly rounded sqrt and division, so the choice of nodes is
//    reproducible bit for bit; ties go to the smallest node id.
#include "common.cuh"

#include <algorithm>
#include <numeric>

namespace hp {
namespace {

constexpr int BIGI = 0x7fffffff;

__global__ void k_voxel_grain(const uint8_t *mask, const int32_t *partition, int n_grains, int nx, int ny, int nz,
                              int px, int py, int pz, int *vg, int *status) {
  long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long nv = (long long)nx * ny * nz;
  if (v >= nv) return;
  if (!mask[v]) {
    vg[v] = -1;
    return;
  }
  int g;
  if (partition) {
    g = partition[v];
    if (g < 0 || g >= n_grains) {
      atomicExch(status, 1);
      g = 0;
    }
  } else {
    int i = (int)(v % nx), j = (int)((v / nx) % ny), k = (int)(v / ((long long)nx * ny));
    int gx = (int)(((long long)i * px) / nx), gy = (int)(((long long)j * py) / ny), gz = (int)(((long long)k * pz) / nz);
    g = gx + px * (gy + py * gz);
  }
  vg[v] = g;
}

// the distinct grains of a node's solid adjacent voxels, ascending; returns the count
__device__ int node_grains(const int *vg, int nx, int ny, int nz, int i, int j, int k, int *out) {
  int t[8];
  int m = 0;
  for (int dk = -1; dk <= 0; ++dk)
    for (int dj = -1; dj <= 0; ++dj)
      for (int di = -1; di <= 0; ++di) {
        int vi = i + di, vj = j + dj, vk = k + dk;
        if (vi < 0 || vj < 0 || vk < 0 || vi >= nx || vj >= ny || vk >= nz) continue;
        int g = vg[((long long)vk * ny + vj) * nx + vi];
        if (g >= 0) t[m++] = g;
      }
  for (int a = 1; a < m; ++a) {  // insertion sort
    int x = t[a], b = a - 1;
    while (b >= 0 && t[b] > x) {
      t[b + 1] = t[b];
      --b;
    }
    t[b + 1] = x;
  }
  int d = 0;
  for (int a = 0; a < m; ++a)
    if (a == 0 || t[a] != t[a - 1]) out[d++] = t[a];
  return d;
}

__global__ void k_classify(const int *node_ijk, int n_nodes, const int *vg, int nx, int ny, int nz,
                           const uint8_t *fixed, int n_grains, int *cls, long long *pairkey, int *label) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= n_nodes) return;
  int S[8];
  int ns = node_grains(vg, nx, ny, nz, node_ijk[3 * n], node_ijk[3 * n + 1], node_ijk[3 * n + 2], S);
  bool has_free = !fixed[3 * n] || !fixed[3 * n + 1] || !fixed[3 * n + 2];
  if (has_free && ns == 1) {
    cls[n] = S[0];
    pairkey[n] = -1;
    label[n] = BIGI;
  } else if (has_free && ns >= 2) {
    cls[n] = -1;
    pairkey[n] = (long long)S[0] * n_grains + S[1];
    label[n] = n;
  } else {
    cls[n] = -2;
    pairkey[n] = -1;
    label[n] = BIGI;
  }
}

// one round of min-label propagation over BSR neighbours of the same pair, with hooking
__global__ void k_cc_step(const int *row_ptr, const int *col, const long long *pairkey, int *label, int n_nodes,
                          int *changed) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= n_nodes) return;
  long long pk = pairkey[n];
  if (pk < 0) return;
  int l = label[n];
  int best = l;
  for (int p = row_ptr[n]; p < row_ptr[n + 1]; ++p) {
    int m = col[p];
    if (pairkey[m] == pk) best = min(best, label[m]);
  }
  if (best < l) {
    atomicMin(&label[n], best);
    atomicMin(&label[l], best);
    *changed = 1;
  }
}

__global__ void k_cc_jump(const long long *pairkey, int *label, int n_nodes) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= n_nodes || pairkey[n] < 0) return;
  int l = label[n];
  int ll = label[l];
  while (ll < l) {
    l = ll;
    ll = label[l];
  }
  label[n] = l;
}

__global__ void k_cc_init(int *label, long long *key, int n_nodes) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= n_nodes) return;
  label[n] = n;
  key[n] = 0;
}

// a component is anchored when one of its nodes has a prescribed displacement component
__global__ void k_anchor_mark(const uint8_t *fixed, const int *label, int n_nodes, int *anchored) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n < n_nodes && (fixed[3 * n] | fixed[3 * n + 1] | fixed[3 * n + 2])) anchored[label[n]] = 1;
}

__global__ void k_floating_first(const int *label, const int *anchored, int n_nodes, int *first) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n < n_nodes && !anchored[label[n]]) atomicMin(first, n);
}

__global__ void k_root_flags(const long long *pairkey, const int *label, int n_nodes, int *flag) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n < n_nodes) flag[n] = (pairkey[n] >= 0 && label[n] == n) ? 1 : 0;
}

__global__ void k_root_keys(const long long *pairkey, const int *flag, const int *pos, int n_nodes,
                            uint64_t *keys) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n < n_nodes && flag[n]) keys[pos[n]] = (uint64_t)pairkey[n] * (uint64_t)n_nodes + (uint64_t)n;
}

__global__ void k_iface_from_keys(const uint64_t *keys, int n_ifaces, int n_nodes, int n_grains, int *root_iface,
                                  int *iface_pair) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_ifaces) return;
  uint64_t k = keys[c];
  int root = (int)(k % (uint64_t)n_nodes);
  long long pk = (long long)(k / (uint64_t)n_nodes);
  root_iface[root] = c;
  iface_pair[2 * c] = (int)(pk / n_grains);
  iface_pair[2 * c + 1] = (int)(pk % n_grains);
}

__global__ void k_iface_of_node(const long long *pairkey, const int *label, const int *root_iface, int n_nodes,
                                int *iface_of_node, int *flag) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= n_nodes) return;
  if (pairkey[n] >= 0) {
    iface_of_node[n] = root_iface[label[n]];
    flag[n] = 1;
  } else {
    iface_of_node[n] = -1;
    flag[n] = 0;
  }
}

__global__ void k_iface_node_keys(const int *iface_of_node, const int *flag, const int *pos, int n_nodes,
                                  uint64_t *keys) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n < n_nodes && flag[n]) keys[pos[n]] = (uint64_t)iface_of_node[n] * (uint64_t)n_nodes + (uint64_t)n;
}

__global__ void k_iface_lists(const uint64_t *keys, long long count, int n_nodes, int *iface_nodes, int *iface_cnt) {
  long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= count) return;
  int node = (int)(keys[p] % (uint64_t)n_nodes);
  int c = (int)(keys[p] / (uint64_t)n_nodes);
  iface_nodes[p] = node;
  atomicAdd(&iface_cnt[c], 1);
}

__global__ void k_iface_slot(const int *iface_nodes, const int *iface_of_node, const int *iface_off, long long count,
                             int *iface_slot) {
  long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= count) return;
  int node = iface_nodes[p];
  iface_slot[node] = (int)(p - iface_off[iface_of_node[node]]);
}

__global__ void k_coupling(const int *iface_nodes, const int *iface_of_node, long long count, const int *node_ijk,
                           const int *vg, int nx, int ny, int nz, const int *iface_pair, int n_grains, int strict,
                           uint8_t *coupling, const uint8_t *fixed, int *comp_mask) {
  long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= count) return;
  int n = iface_nodes[p];
  int c = iface_of_node[n];
  int cm = (fixed[3 * n] ? 0 : 1) | (fixed[3 * n + 1] ? 0 : 2) | (fixed[3 * n + 2] ? 0 : 4);
  atomicOr(&comp_mask[c], cm);
  // the column layout always follows the touch coupling, so that the Galerkin sub-assembly sees
  // every coarse column active on a grain's voxels; strict mode only zeroes the basis right-hand
  // sides of non-pair grains (see the basis kernel)
  (void)strict;
  (void)iface_pair;
  int S[8];
  int ns = node_grains(vg, nx, ny, nz, node_ijk[3 * n], node_ijk[3 * n + 1], node_ijk[3 * n + 2], S);
  for (int a = 0; a < ns; ++a) coupling[(long long)c * n_grains + S[a]] = 1;
}

__global__ void k_grain_has_rhs(const int *cls, const double *b, int n_nodes, int *flag) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= n_nodes) return;
  int g = cls[n];
  if (g >= 0 && (b[3 * n] != 0.0 || b[3 * n + 1] != 0.0 || b[3 * n + 2] != 0.0)) flag[g] = 1;
}

// ------------------------------------------------------------ mortar placement
struct ArgMin {
  double v;
  int i;
};

__device__ __forceinline__ ArgMin better(ArgMin a, ArgMin b) {
  if (b.v < a.v || (b.v == a.v && b.i < a.i)) return b;
  return a;
}

__device__ ArgMin block_argmin(ArgMin x, ArgMin *sh) {
  for (int o = 16; o > 0; o >>= 1) {
    ArgMin y;
    y.v = __shfl_down_sync(0xffffffffu, x.v, o);
    y.i = __shfl_down_sync(0xffffffffu, x.i, o);
    x = better(x, y);
  }
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = x;
  __syncthreads();
  if (w == 0) {
    int nw = (blockDim.x + 31) >> 5;
    x = lane < nw ? sh[lane] : ArgMin{INFINITY, BIGI};
    for (int o = 16; o > 0; o >>= 1) {
      ArgMin y;
      y.v = __shfl_down_sync(0xffffffffu, x.v, o);
      y.i = __shfl_down_sync(0xffffffffu, x.i, o);
      x = better(x, y);
    }
    if (lane == 0) sh[0] = x;
  }
  __syncthreads();
  ArgMin r = sh[0];
  __syncthreads();
  return r;
}

__device__ __forceinline__ long long d2i(const int *P, int a, int b) {
  long long dx = P[3 * a] - P[3 * b], dy = P[3 * a + 1] - P[3 * b + 1], dz = P[3 * a + 2] - P[3 * b + 2];
  return dx * dx + dy * dy + dz * dz;
}

// energy of candidate y against the chosen mortars except index `skip`, ascending mortar order
__device__ __forceinline__ double energy(const int *P, int y, const int *chosen, int cnt, int skip) {
  double acc = 0.0;
  for (int j = 0; j < cnt; ++j) {
    if (j == skip) continue;
    double d = (double)d2i(P, y, chosen[j]);
    acc = __dadd_rn(acc, __ddiv_rn(1.0, __dsqrt_rn(d)));
  }
  return acc;
}

// one CTA per interface: coordinates of its nodes (P, node-list order), mortar placement, Gaussian weights
__global__ void k_mortars(const int *iface_off, const int *iface_nodes, const int *node_ijk, const int *mortar_off,
                          int *mortar_nodes, int *mortar_idx, const long long *eta_off, double *eta, double beta,
                          int *Pbuf) {
  extern __shared__ int sh_int[];
  __shared__ ArgMin red[32];
  __shared__ int best_pair[3];
  int c = blockIdx.x;
  int f0 = iface_off[c], F = iface_off[c + 1] - f0;
  int m0 = mortar_off[c], nc = mortar_off[c + 1] - m0;
  int *chosen = sh_int;  // nc entries
  int *P = Pbuf + 3LL * f0;
  for (int y = threadIdx.x; y < F; y += blockDim.x) {
    int n = iface_nodes[f0 + y];
    P[3 * y] = node_ijk[3 * n];
    P[3 * y + 1] = node_ijk[3 * n + 1];
    P[3 * y + 2] = node_ijk[3 * n + 2];
  }
  __syncthreads();
  if (nc == F) {
    for (int i = threadIdx.x; i < nc; i += blockDim.x) chosen[i] = i;
  } else if (nc == 1) {
    // nearest to the centroid: minimise ||F*y - sum||^2 in exact integers
    __shared__ long long ssum[3];
    if (threadIdx.x < 3) ssum[threadIdx.x] = 0;
    __syncthreads();
    long long sx = 0, sy = 0, sz = 0;
    for (int y = threadIdx.x; y < F; y += blockDim.x) {
      sx += P[3 * y];
      sy += P[3 * y + 1];
      sz += P[3 * y + 2];
    }
    atomicAdd((unsigned long long *)&ssum[0], (unsigned long long)sx);
    atomicAdd((unsigned long long *)&ssum[1], (unsigned long long)sy);
    atomicAdd((unsigned long long *)&ssum[2], (unsigned long long)sz);
    __syncthreads();
    ArgMin loc{INFINITY, BIGI};
    for (int y = threadIdx.x; y < F; y += blockDim.x) {
      long long dx = (long long)F * P[3 * y] - ssum[0], dy = (long long)F * P[3 * y + 1] - ssum[1],
                dz = (long long)F * P[3 * y + 2] - ssum[2];
      loc = better(loc, ArgMin{(double)(dx * dx + dy * dy + dz * dz), y});
    }
    ArgMin r = block_argmin(loc, red);
    if (threadIdx.x == 0) chosen[0] = r.i;
  } else {
    // farthest pair; ties -> smallest (a, b)
    long long bd = -1;
    int ba = BIGI, bb = BIGI;
    for (int a = threadIdx.x; a < F; a += blockDim.x)
      for (int b = a + 1; b < F; ++b) {
        long long d = d2i(P, a, b);
        if (d > bd) {
          bd = d;
          ba = a;
          bb = b;
        }
      }
    // reduce: larger distance wins, then smaller a, then smaller b (encode as argmin on -d)
    ArgMin loc{(double)(-bd), ba};
    ArgMin r = block_argmin(loc, red);
    // the winning thread is the one holding (r.v, r.i); its partner index
    if (loc.v == r.v && loc.i == r.i && ba != BIGI) {
      best_pair[0] = ba;
      best_pair[1] = bb;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      chosen[0] = best_pair[0];
      chosen[1] = best_pair[1];
    }
    __syncthreads();
    // greedy additions (Eq. node_init)
    for (int i = 2; i < nc; ++i) {
      ArgMin l2{INFINITY, BIGI};
      for (int y = threadIdx.x; y < F; y += blockDim.x) {
        bool taken = false;
        for (int j = 0; j < i; ++j) taken |= chosen[j] == y;
        if (taken) continue;
        l2 = better(l2, ArgMin{energy(P, y, chosen, i, -1), y});
      }
      ArgMin r2 = block_argmin(l2, red);
      if (threadIdx.x == 0) chosen[i] = r2.i;
      __syncthreads();
    }
    // sweeps in ascending mortar order until nothing moves (at most 100)
    for (int sweep = 0; sweep < 100; ++sweep) {
      int moved = 0;
      for (int i = 0; i < nc; ++i) {
        ArgMin l3{INFINITY, BIGI};
        for (int y = threadIdx.x; y < F; y += blockDim.x) {
          bool taken = false;
          for (int j = 0; j < nc; ++j) taken |= (j != i) && chosen[j] == y;
          if (taken) continue;
          l3 = better(l3, ArgMin{energy(P, y, chosen, nc, i), y});
        }
        ArgMin r3 = block_argmin(l3, red);
        if (r3.i != chosen[i]) moved = 1;
        __syncthreads();
        if (threadIdx.x == 0) chosen[i] = r3.i;
        __syncthreads();
      }
      if (!moved) break;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nc; i += blockDim.x) {
    mortar_idx[m0 + i] = chosen[i];
    mortar_nodes[m0 + i] = iface_nodes[f0 + chosen[i]];
  }
  // Gaussian mortars (Eq. gauss): softmax over i of -||y-x_i||^2 / (beta * min_{j!=i} ||x_i-x_j||^2)
  double *et = eta + eta_off[c];
  for (int y = threadIdx.x; y < F; y += blockDim.x) {
    if (nc == 1) {
      et[y] = 1.0;
      continue;
    }
    double amax = -INFINITY;
    for (int i = 0; i < nc; ++i) {
      long long dm = 0x7fffffffffffffffLL;
      for (int j = 0; j < nc; ++j)
        if (j != i) dm = min(dm, d2i(P, chosen[i], chosen[j]));
      double a = -(double)d2i(P, y, chosen[i]) / (beta * (double)dm);
      et[(long long)y * nc + i] = a;
      amax = fmax(amax, a);
    }
    double s = 0.0;
    for (int i = 0; i < nc; ++i) {
      double e = exp(et[(long long)y * nc + i] - amax);
      et[(long long)y * nc + i] = e;
      s += e;
    }
    for (int i = 0; i < nc; ++i) et[(long long)y * nc + i] /= s;
  }
}

__global__ void k_w_keys(const int *dof_slot, long long n_dof, const int *cls, const int *iface_of_node,
                         int n_grains, uint64_t *keys) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_dof) return;
  int node = dof_slot[i] / 3;
  long long rank = cls[node] >= 0 ? cls[node] : (long long)n_grains + iface_of_node[node];
  keys[i] = (uint64_t)rank * (uint64_t)n_dof + (uint64_t)i;
}

__global__ void k_w_out(const uint64_t *keys, long long n_dof, int64_t *W) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_dof) W[i] = (int64_t)(keys[i] % (uint64_t)n_dof);
}

}  // namespace

// Connected parts of the solid (nodes joined by a shared solid voxel, i.e. by a block of A_hat): a part with
// no prescribed displacement component can move rigidly, so A_hat is singular; report a node of it.
void check_anchored(hplmm_ctx *c) {
  cudaStream_t s = c->stream;
  const int nn = c->n_nodes;
  Buf<int> label, anchored, changed, first;
  Buf<long long> key;
  label.alloc(nn);
  key.alloc(nn);
  anchored.alloc(nn);
  anchored.zero(s);
  changed.alloc(1);
  first.alloc(1);
  first.fill_bytes(0x7f, s);
  k_cc_init<<<grid_for(nn, 256), 256, 0, s>>>(label.p, key.p, nn);
  HP_CHECK_LAUNCH();
  for (int it = 0; it < 100000; ++it) {
    changed.zero(s);
    k_cc_step<<<grid_for(nn, 256), 256, 0, s>>>(c->row_ptr.p, c->col.p, key.p, label.p, nn, changed.p);
    HP_CHECK_LAUNCH();
    k_cc_jump<<<grid_for(nn, 256), 256, 0, s>>>(key.p, label.p, nn);
    HP_CHECK_LAUNCH();
    if (changed.download(s, 1)[0] == 0) break;
  }
  k_anchor_mark<<<grid_for(nn, 256), 256, 0, s>>>(c->fixed.p, label.p, nn, anchored.p);
  HP_CHECK_LAUNCH();
  k_floating_first<<<grid_for(nn, 256), 256, 0, s>>>(label.p, anchored.p, nn, first.p);
  HP_CHECK_LAUNCH();
  const int n = first.download(s, 1)[0];
  if (n < nn) {
    int ijk[3];
    HP_CUDA(cudaMemcpyAsync(ijk, c->node_ijk.p + 3LL * n, sizeof(ijk), cudaMemcpyDeviceToHost, s));
    HP_CUDA(cudaStreamSynchronize(s));
    throw Error(HPLMM_ERR_SINGULAR, "assemble: the solid part holding node (" + std::to_string(ijk[0]) + ", " +
                                        std::to_string(ijk[1]) + ", " + std::to_string(ijk[2]) +
                                        ") has no prescribed displacement: it can move rigidly (A_hat is singular)");
  }
}

void build_maps(hplmm_ctx *c, const int32_t *partition) {
  cudaStream_t s = c->stream;
  int nn = c->n_nodes;
  long long nv = (long long)c->nx * c->ny * c->nz;
  c->status.alloc(4);
  c->status.zero(s);
  c->vgrain.alloc(nv);
  k_voxel_grain<<<grid_for(nv, 256), 256, 0, s>>>(c->mask.p, partition, c->n_grains, c->nx, c->ny, c->nz, c->px,
                                                  c->py, c->pz, c->vgrain.p, c->status.p);
  HP_CHECK_LAUNCH();
  auto st = c->status.download(s, 1);
  HP_REQUIRE(st[0] == 0, HPLMM_ERR_INVALID, "setup: partition holds a grain id outside [0, n_grains)");

  c->node_cls.alloc(nn);
  Buf<long long> pairkey;
  pairkey.alloc(nn);
  Buf<int> label, flag, pos;
  label.alloc(nn);
  flag.alloc(nn + 1);
  pos.alloc(nn + 1);
  k_classify<<<grid_for(nn, 256), 256, 0, s>>>(c->node_ijk.p, nn, c->vgrain.p, c->nx, c->ny, c->nz, c->fixed.p,
                                               c->n_grains, c->node_cls.p, pairkey.p, label.p);
  HP_CHECK_LAUNCH();
  // connected components of each pair's interface nodes
  Buf<int> changed;
  changed.alloc(1);
  for (int it = 0; it < 100000; ++it) {
    changed.zero(s);
    k_cc_step<<<grid_for(nn, 256), 256, 0, s>>>(c->row_ptr.p, c->col.p, pairkey.p, label.p, nn, changed.p);
    HP_CHECK_LAUNCH();
    k_cc_jump<<<grid_for(nn, 256), 256, 0, s>>>(pairkey.p, label.p, nn);
    HP_CHECK_LAUNCH();
    if (changed.download(s, 1)[0] == 0) break;
  }
  k_root_flags<<<grid_for(nn, 256), 256, 0, s>>>(pairkey.p, label.p, nn, flag.p);
  HP_CHECK_LAUNCH();
  long long n_if = exclusive_scan_i32(flag.p, pos.p, nn, s);
  c->n_ifaces = (int)n_if;
  Buf<uint64_t> keys;
  keys.alloc(std::max<long long>(n_if, 1));
  k_root_keys<<<grid_for(nn, 256), 256, 0, s>>>(pairkey.p, flag.p, pos.p, nn, keys.p);
  HP_CHECK_LAUNCH();
  sort_u64(keys.p, n_if, s);
  Buf<int> root_iface;
  root_iface.alloc(nn);
  c->iface_pair.alloc(2 * std::max<long long>(n_if, 1));
  k_iface_from_keys<<<grid_for(n_if, 128), 128, 0, s>>>(keys.p, c->n_ifaces, nn, c->n_grains, root_iface.p,
                                                        c->iface_pair.p);
  HP_CHECK_LAUNCH();
  c->iface_of_node.alloc(nn);
  k_iface_of_node<<<grid_for(nn, 256), 256, 0, s>>>(pairkey.p, label.p, root_iface.p, nn, c->iface_of_node.p,
                                                    flag.p);
  HP_CHECK_LAUNCH();
  long long nin = exclusive_scan_i32(flag.p, pos.p, nn, s);
  c->n_iface_nodes = nin;
  Buf<uint64_t> nkeys;
  nkeys.alloc(std::max<long long>(nin, 1));
  k_iface_node_keys<<<grid_for(nn, 256), 256, 0, s>>>(c->iface_of_node.p, flag.p, pos.p, nn, nkeys.p);
  HP_CHECK_LAUNCH();
  sort_u64(nkeys.p, nin, s);
  c->iface_nodes.alloc(std::max<long long>(nin, 1));
  Buf<int> cnt;
  cnt.alloc(n_if + 1);
  cnt.zero(s);
  k_iface_lists<<<grid_for(nin, 256), 256, 0, s>>>(nkeys.p, nin, nn, c->iface_nodes.p, cnt.p);
  HP_CHECK_LAUNCH();
  c->iface_off.alloc(n_if + 1);
  exclusive_scan_i32(cnt.p, c->iface_off.p, n_if + 1, s);
  c->h_iface_off = c->iface_off.download(s);
  c->iface_slot.alloc(nn);
  k_iface_slot<<<grid_for(nin, 256), 256, 0, s>>>(c->iface_nodes.p, c->iface_of_node.p, c->iface_off.p, nin,
                                                  c->iface_slot.p);
  HP_CHECK_LAUNCH();

  // couplings and component masks
  Buf<uint8_t> coup;
  coup.alloc((size_t)std::max<long long>(n_if, 1) * c->n_grains);
  coup.zero(s);
  c->comp_mask.alloc(std::max<long long>(n_if, 1));
  c->comp_mask.zero(s);
  k_coupling<<<grid_for(nin, 256), 256, 0, s>>>(c->iface_nodes.p, c->iface_of_node.p, nin, c->node_ijk.p,
                                                c->vgrain.p, c->nx, c->ny, c->nz, c->iface_pair.p, c->n_grains,
                                                c->opt.strict_two_grain, coup.p, c->fixed.p, c->comp_mask.p);
  HP_CHECK_LAUNCH();
  auto hc = coup.download(s);
  c->h_comp_mask = c->comp_mask.download(s, n_if);
  // mortar counts and coarse column layout
  int n = c->opt.n_mortar;
  c->h_mortar_off.assign(n_if + 1, 0);
  c->h_col_off.assign(n_if + 1, 0);
  std::vector<long long> heta(n_if + 1, 0);
  for (int ci = 0; ci < n_if; ++ci) {
    int F = c->h_iface_off[ci + 1] - c->h_iface_off[ci];
    int nc = std::min(n, F);
    int ncomp = __builtin_popcount(c->h_comp_mask[ci]);
    c->h_mortar_off[ci + 1] = c->h_mortar_off[ci] + nc;
    c->h_col_off[ci + 1] = c->h_col_off[ci] + nc * ncomp;
    heta[ci + 1] = heta[ci] + (long long)F * nc;
  }
  c->n_mortars = c->h_mortar_off[n_if];
  c->n_mortar_cols = c->h_col_off[n_if];
  c->mortar_off.upload(c->h_mortar_off, s);
  c->col_off.upload(c->h_col_off, s);
  c->eta_off.upload(heta, s);
  c->eta.alloc(std::max<long long>(heta[n_if], 1));
  c->mortar_nodes.alloc(std::max(c->n_mortars, 1));
  c->mortar_idx.alloc(std::max(c->n_mortars, 1));

  // grain -> coupled interfaces, columns per grain, kept corrections
  int G = c->n_grains;
  c->h_glists.assign(G, {});
  for (int ci = 0; ci < n_if; ++ci)
    for (int g = 0; g < G; ++g)
      if (hc[(size_t)ci * G + g]) c->h_glists[g].push_back(ci);
  Buf<int> hasb;
  hasb.alloc(G);
  hasb.zero(s);
  k_grain_has_rhs<<<grid_for(nn, 256), 256, 0, s>>>(c->node_cls.p, c->b_corr.p, nn, hasb.p);
  HP_CHECK_LAUNCH();
  c->h_grain_hasb = hasb.download(s);
  layout_columns(c);
}

// columns of every grain's panel from the interfaces' column counts (h_col_off): the coupled interfaces'
// mortar columns in ascending interface order, then the grain's correction column when b^g != 0
void layout_columns(hplmm_ctx *c) {
  cudaStream_t s = c->stream;
  const int G = c->n_grains;
  const int n_if = c->n_ifaces;
  const auto &lists = c->h_glists;
  const auto &hb = c->h_grain_hasb;
  c->n_mortar_cols = c->h_col_off[n_if];
  c->col_off.upload(c->h_col_off, s);
  c->h_gi_off.assign(G + 1, 0);
  c->h_gi_iface.clear();
  c->h_gi_colbase.clear();
  c->h_kg.assign(G, 0);
  c->h_corr_col.assign(G, -1);
  long long ncorr = 0;
  for (int g = 0; g < G; ++g) {
    c->h_gi_off[g + 1] = c->h_gi_off[g] + (int)lists[g].size();
    int base = 0;
    for (int ci : lists[g]) {
      c->h_gi_iface.push_back(ci);
      c->h_gi_colbase.push_back(base);
      base += c->h_col_off[ci + 1] - c->h_col_off[ci];
    }
    c->h_kg[g] = base;
    if (hb[g]) {
      c->h_corr_col[g] = (int)(c->n_mortar_cols + ncorr++);
      c->h_kg[g] += 1;
    }
  }
  c->n_coarse = c->n_mortar_cols + ncorr;
  if (c->h_gi_iface.empty()) {
    c->h_gi_iface.push_back(0);
    c->h_gi_colbase.push_back(0);
  }
  c->gi_off.upload(c->h_gi_off, s);
  c->gi_iface.upload(c->h_gi_iface, s);
  c->gi_colbase.upload(c->h_gi_colbase, s);
  c->kg.upload(c->h_kg, s);
  c->corr_col.upload(c->h_corr_col, s);
  HP_CUDA(cudaStreamSynchronize(s));
}

void build_mortars(hplmm_ctx *c) {
  cudaStream_t s = c->stream;
  if (c->n_ifaces == 0) return;
  Buf<int> P;
  P.alloc(3 * std::max<long long>(c->n_iface_nodes, 1));
  size_t smem = sizeof(int) * (size_t)std::max(c->opt.n_mortar, 1);
  k_mortars<<<c->n_ifaces, 256, smem, s>>>(c->iface_off.p, c->iface_nodes.p, c->node_ijk.p, c->mortar_off.p,
                                          c->mortar_nodes.p, c->mortar_idx.p, c->eta_off.p, c->eta.p, c->opt.beta,
                                          P.p);
  HP_CHECK_LAUNCH();
  HP_CUDA(cudaStreamSynchronize(s));
}

void compute_W(hplmm_ctx *c, int64_t *W) {
  cudaStream_t s = c->stream;
  Buf<uint64_t> keys;
  keys.alloc(std::max<long long>(c->n_dof, 1));
  k_w_keys<<<grid_for(c->n_dof, 256), 256, 0, s>>>(c->dof_slot.p, c->n_dof, c->node_cls.p, c->iface_of_node.p,
                                                   c->n_grains, keys.p);
  HP_CHECK_LAUNCH();
  sort_u64(keys.p, c->n_dof, s);
  k_w_out<<<grid_for(c->n_dof, 256), 256, 0, s>>>(keys.p, c->n_dof, W);
  HP_CHECK_LAUNCH();
  HP_CUDA(cudaStreamSynchronize(s));
}

}  // namespace hp
