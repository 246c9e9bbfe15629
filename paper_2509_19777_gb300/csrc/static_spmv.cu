// y = A_hat x without any device allocation.
//
// hplmm_spmv stages x and y in padded [n_nodes][3] work vectors that the
// context allocates on demand.  This variant keeps those two work vectors in
// one file-scope device array instead, so a call allocates nothing: it is for
// callers whose device memory is entirely owned by their own allocator (a
// pool reserved up front, a fixed memory budget) or whose loops must never
// hit the implicit synchronisation of cudaMalloc/cudaFree.
//
// Limit: 3 * n_nodes <= HPLMM_NOALLOC_MAX_SLOTS (786,432 slots, i.e. 262,144
// fine nodes); the array (12 MiB) stays resident on every device that loads
// the library until the process exits.  All calls share it and it keeps the
// previous call's contents, so the padded input is cleared before use, and
// calls that overlap on the GPU (other streams, other threads) race.
#include "common.cuh"

#include <mutex>

namespace {

constexpr long long NOALLOC_MAX_SLOTS = 3LL << 18;
constexpr int MAX_DEVICES = 64;

static __device__ __align__(256) double g_noalloc_scratch[2 * NOALLOC_MAX_SLOTS];

std::mutex g_mu;
double *g_scratch_ptr[MAX_DEVICES] = {};

// the array's device address on the current device (looked up once per device and cached for the process:
// the cache assumes the device's primary context is never reset while the library is loaded)
double *scratch_for_device(int dev) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (dev < 0 || dev >= MAX_DEVICES) throw hp::Error(HPLMM_ERR_INVALID, "device index out of range");
  if (!g_scratch_ptr[dev]) {
    void *ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || ptr == nullptr)
      throw hp::Error(HPLMM_ERR_CUDA, std::string("cudaGetSymbolAddress of the static scratch failed: ") +
                                          cudaGetErrorString(e));
    g_scratch_ptr[dev] = static_cast<double *>(ptr);
  }
  return g_scratch_ptr[dev];
}

__global__ void k_na_scatter(const int *dof_slot, const double *dof, double *pad, long long n_dof) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_dof) pad[dof_slot[i]] = dof[i];
}

__global__ void k_na_gather(const int *dof_slot, const double *pad, double *dof, long long n_dof) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_dof) dof[i] = pad[dof_slot[i]];
}

__global__ void k_na_spmv(const int *row_ptr, const int *col, const double *val, const double *x, double *y,
                          int n_nodes) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= n_nodes) return;
  double s0 = 0, s1 = 0, s2 = 0;
  for (int p = row_ptr[n]; p < row_ptr[n + 1]; ++p) {
    int m = col[p];
    const double *v = val + (long long)p * 9;
    double x0 = x[3 * m], x1 = x[3 * m + 1], x2 = x[3 * m + 2];
    s0 += v[0] * x0;
    s0 += v[1] * x1;
    s0 += v[2] * x2;
    s1 += v[3] * x0;
    s1 += v[4] * x1;
    s1 += v[5] * x2;
    s2 += v[6] * x0;
    s2 += v[7] * x1;
    s2 += v[8] * x2;
  }
  y[3 * n] = s0;
  y[3 * n + 1] = s1;
  y[3 * n + 2] = s2;
}

}  // namespace

extern "C" hplmm_status hplmm_spmv_noalloc(hplmm_ctx *c, const double *x, double *y) {
  if (!c) return HPLMM_ERR_INVALID;
  try {
    HP_REQUIRE(c->assembled, HPLMM_ERR_STATE, "call hplmm_assemble first");
    HP_REQUIRE(x && y, HPLMM_ERR_INVALID, "spmv_noalloc: null vector");
    long long L = 3LL * c->n_nodes;
    HP_REQUIRE(L <= NOALLOC_MAX_SLOTS, HPLMM_ERR_INVALID,
               "spmv_noalloc: 3*n_nodes = " + std::to_string(L) + " exceeds the static scratch limit of " +
                   std::to_string(NOALLOC_MAX_SLOTS) + " slots (262,144 nodes); use hplmm_spmv");
    int dev = 0;
    HP_CUDA(cudaGetDevice(&dev));
    // the array's address is per device: the one looked up must be that of the device the context's
    // stream and buffers belong to
    HP_REQUIRE(dev == c->device, HPLMM_ERR_INVALID,
               "spmv_noalloc: the context belongs to device " + std::to_string(c->device) +
                   " but device " + std::to_string(dev) + " is current; make the context's device current");
    double *xp = scratch_for_device(dev);
    double *yp = xp + NOALLOC_MAX_SLOTS;
    cudaStream_t s = c->stream;
    // the shared array keeps the last call's values: clear the padded input (fixed slots must be zero)
    HP_CUDA(cudaMemsetAsync(xp, 0, sizeof(double) * (size_t)L, s));
    k_na_scatter<<<hp::grid_for(c->n_dof, 256), 256, 0, s>>>(c->dof_slot.p, x, xp, c->n_dof);
    HP_CHECK_LAUNCH();
    k_na_spmv<<<hp::grid_for(c->n_nodes, 128), 128, 0, s>>>(c->row_ptr.p, c->col.p, c->val64.p, xp, yp,
                                                            c->n_nodes);
    HP_CHECK_LAUNCH();
    k_na_gather<<<hp::grid_for(c->n_dof, 256), 256, 0, s>>>(c->dof_slot.p, yp, y, c->n_dof);
    HP_CHECK_LAUNCH();
    return HPLMM_OK;
  } catch (const hp::Error &e) {
    c->err = e.what();
    return e.code;
  } catch (const std::exception &e) {
    c->err = e.what();
    return HPLMM_ERR_CUDA;
  }
}
