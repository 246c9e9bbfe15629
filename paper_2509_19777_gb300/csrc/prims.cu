// Device primitives used while building the index maps: an exclusive scan of
// int32 flags/counts and an in-place ascending sort of 64-bit keys.
#include "common.cuh"

namespace hp {
namespace {

constexpr int SCAN_BLOCK = 1024;

__device__ __forceinline__ int warp_incl_scan(int v) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) >= o) v += t;
  }
  return v;
}

// each block scans SCAN_BLOCK consecutive values; writes exclusive prefix and block total
__global__ void k_scan_block(const int *in, int *out, int *block_sums, long long n) {
  __shared__ int warp_tot[32];
  long long i = (long long)blockIdx.x * SCAN_BLOCK + threadIdx.x;
  int v = (i < n) ? in[i] : 0;
  int incl = warp_incl_scan(v);
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 31) warp_tot[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    int t = warp_tot[lane];
    int s = warp_incl_scan(t);
    warp_tot[lane] = s - t;
  }
  __syncthreads();
  int excl = incl - v + warp_tot[wid];
  if (i < n) out[i] = excl;
  if (threadIdx.x == SCAN_BLOCK - 1) block_sums[blockIdx.x] = excl + v;
}

__global__ void k_scan_add(int *out, const int *block_offsets, long long n) {
  long long i = (long long)blockIdx.x * SCAN_BLOCK + threadIdx.x;
  if (i < n) out[i] += block_offsets[blockIdx.x];
}

struct ScanScratch {
  std::vector<Buf<int> *> levels;
  ~ScanScratch() {
    for (auto *b : levels) delete b;
  }
  int *get(int level, size_t count) {
    while ((int)levels.size() <= level) levels.push_back(new Buf<int>());
    if (levels[level]->n < count + 1) levels[level]->alloc(count + 1);
    return levels[level]->p;
  }
};

thread_local ScanScratch g_scan;

void scan_rec(const int *in, int *out, long long n, int level, cudaStream_t s) {
  long long nb = (n + SCAN_BLOCK - 1) / SCAN_BLOCK;
  if (nb < 1) nb = 1;
  int *sums = g_scan.get(level, (size_t)nb);
  k_scan_block<<<(unsigned)nb, SCAN_BLOCK, 0, s>>>(in, out, sums, n);
  HP_CHECK_LAUNCH();
  if (nb > 1) {
    // exclusive scan of block sums in place, then add
    scan_rec(sums, sums, nb, level + 1, s);
    k_scan_add<<<(unsigned)nb, SCAN_BLOCK, 0, s>>>(out, sums, n);
    HP_CHECK_LAUNCH();
  }
}

__global__ void k_bitonic_global(uint64_t *keys, long long j, long long k) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long l = i ^ j;
  if (l > i) {
    uint64_t a = keys[i], b = keys[l];
    bool up = (i & k) == 0;
    if ((a > b) == up) {
      keys[i] = b;
      keys[l] = a;
    }
  }
}

// all steps j = jstart ... 1 of stage k inside one 2048-key tile
__global__ void k_bitonic_shared(uint64_t *keys, long long k, int jstart) {
  __shared__ uint64_t t[2048];
  long long base = (long long)blockIdx.x * 2048;
  t[threadIdx.x] = keys[base + threadIdx.x];
  t[threadIdx.x + 1024] = keys[base + threadIdx.x + 1024];
  __syncthreads();
  for (int j = jstart; j > 0; j >>= 1) {
    for (int h = 0; h < 2; ++h) {
      int i = threadIdx.x + h * 1024;
      int l = i ^ j;
      if (l > i) {
        uint64_t a = t[i], b = t[l];
        bool up = ((base + i) & k) == 0;
        if ((a > b) == up) {
          t[i] = b;
          t[l] = a;
        }
      }
    }
    __syncthreads();
  }
  keys[base + threadIdx.x] = t[threadIdx.x];
  keys[base + threadIdx.x + 1024] = t[threadIdx.x + 1024];
}

__global__ void k_fill_u64(uint64_t *p, long long from, long long to, uint64_t v) {
  long long i = from + (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < to) p[i] = v;
}

thread_local Buf<uint64_t> g_sort;

}  // namespace

long long exclusive_scan_i32(const int *in, int *out, long long n, cudaStream_t s) {
  if (n <= 0) return 0;
  int last_in = 0;
  HP_CUDA(cudaMemcpyAsync(&last_in, in + n - 1, sizeof(int), cudaMemcpyDeviceToHost, s));
  HP_CUDA(cudaStreamSynchronize(s));
  scan_rec(in, out, n, 0, s);
  int last_out = 0;
  HP_CUDA(cudaMemcpyAsync(&last_out, out + n - 1, sizeof(int), cudaMemcpyDeviceToHost, s));
  HP_CUDA(cudaStreamSynchronize(s));
  return (long long)last_out + last_in;
}

void sort_u64(uint64_t *keys, long long n, cudaStream_t s) {
  if (n <= 1) return;
  long long N = 2048;
  while (N < n) N <<= 1;
  if (g_sort.n < (size_t)N) g_sort.alloc((size_t)N);
  uint64_t *t = g_sort.p;
  HP_CUDA(cudaMemcpyAsync(t, keys, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
  k_fill_u64<<<grid_for(N - n, 256), 256, 0, s>>>(t, n, N, ~0ull);
  HP_CHECK_LAUNCH();
  for (long long k = 2; k <= N; k <<= 1) {
    long long j = k >> 1;
    for (; j >= 2048; j >>= 1) {
      k_bitonic_global<<<grid_for(N, 256), 256, 0, s>>>(t, j, k);
      HP_CHECK_LAUNCH();
    }
    k_bitonic_shared<<<(unsigned)(N / 2048), 1024, 0, s>>>(t, k, (int)j);
    HP_CHECK_LAUNCH();
  }
  HP_CUDA(cudaMemcpyAsync(keys, t, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
}

}  // namespace hp
