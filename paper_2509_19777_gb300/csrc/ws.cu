// Learned warm start of the local basis solves and the iterative basis solver it feeds.
//
// The paper solves every local basis problem exactly (Eqs. col_pk, col_cg; Section 6.3).  This file adds an
// optional iterative path: a 3-D convolutional network maps one basis problem (its grain's solid voxels,
// log moduli and right-hand side on the grain's 17^3 node grid) to an initial guess, and block-Jacobi
// preconditioned conjugate gradients, batched over every (grain, block of 32 right-hand sides) in one launch,
// refines it; columns that miss the tolerance fall back to the exact banded solve.  The network is trained
// on the GPU, from basis problems whose exact solutions the library itself computed, by the forward and
// backward kernels below and Adam.
//
// Sample of a basis problem (grain g, right-hand-side column a), on the grid whose origin is the minimum
// corner of g's solid voxels (indices [z][y][x], 17 nodes per axis):
//   channel 0: 1 on voxel (i,j,k) < 16 that is a solid voxel of g;   channel 1: its log E;
//   channels 2..4: the right-hand side's x,y,z components on g's free DOFs divided by s, the RMS of the
//   right-hand side over those DOFs;   target: the exact solution divided by its own RMS over those DOFs;
//   valid: 1 where a free DOF of g sits.   A prediction q, read at the valid positions, is the direction of
//   the initial guess: CG first scales it by the factor that minimises the A-norm error along it, so only
//   the shape of the solution has to be learned.
// Network: 3x3x3 convolutions with zero padding and dilations 1, 2, 4, 8 (an output sees inputs up to 15
// nodes away along each axis), channels 5 -> 32 -> 32 -> 32 -> 3, bias, ReLU after the first three.
// Parameters: per layer W[co][ci][tz][ty][tx] (tap reads offset ((tz-1)d, (ty-1)d, (tx-1)d) for dilation d),
// then bias[co].  Loss: masked mean squared error.  Training in FP32; inference stores weights and activations
// in BF16 (FP32 arithmetic).
#include "common.cuh"

#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

namespace hp {

namespace {

constexpr int WS_D = 17;                 // grid nodes per axis of a grain sample
constexpr int WS_D3 = WS_D * WS_D * WS_D;
constexpr int WS_NL = 4;
constexpr int WS_CH[WS_NL + 1] = {5, 32, 32, 32, 3};
constexpr int WS_DIL[WS_NL] = {1, 2, 4, 8};
constexpr int CONV_THREADS = 320;        // >= D^2 positions of one z-slice (D <= 17)
constexpr int CONV_CG = 8;               // input channels staged per pass

constexpr long long layer_w_off(int l) {
  long long o = 0;
  for (int i = 0; i < l; ++i) o += (long long)WS_CH[i + 1] * WS_CH[i] * 27 + WS_CH[i + 1];
  return o;
}
constexpr long long WS_NPARAM = layer_w_off(WS_NL);

template <typename T> __device__ __forceinline__ float to_f(T v) { return (float)v; }
template <> __device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <typename T> __device__ __forceinline__ T from_f(float v) { return (T)v; }
template <> __device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

// ---------------------------------------------------------------- convolution, forward form
// out[n][o][p] = bias[o] + sum_{i,t} W[o][i][t] in[n][i][p + (t - 1) dil] over a D^3 grid, zero padding.
// One CTA per (sample n, z-slice), one thread per (y, x) of the slice holding all CO accumulators; input
// channels are staged CONV_CG at a time as a zero-bordered halo of the 3 slices z - dil, z, z + dil (border
// width dil in y and x), the weights of the group
// transposed to [t][i][o] so that a thread reads the CO weights of one (t, i) as broadcast 16-byte loads.
// Optional: ReLU on the output, or multiplication by a mask (mask > 0) for the backward data pass.
template <int CO, typename TI, typename TO, typename TW>
__global__ void __launch_bounds__(CONV_THREADS) k_conv(const TI *in, int CI, const TW *W, const TW *bias, TO *out,
                                                       int D, int dil, int relu, const float *mask) {
  extern __shared__ __align__(16) float csm[];
  const int E = D + 2 * dil;                            // bordered extent
  float *halo = csm;                                    // [CONV_CG][3][E][E]
  float *Ws = csm + CONV_CG * 3 * E * E;                // [27][CONV_CG][CO4]
  constexpr int CO4 = (CO + 3) / 4 * 4;
  const int n = blockIdx.y, z = blockIdx.x;
  const int D2 = D * D, D3 = D2 * D;
  const int pos = threadIdx.x, y = pos / D, x = pos - y * D;
  const bool act = pos < D2;
  float acc[CO];
#pragma unroll
  for (int o = 0; o < CO; ++o) acc[o] = bias ? to_f(bias[o]) : 0.f;
  for (int ci0 = 0; ci0 < CI; ci0 += CONV_CG) {
    const int cg = min(CONV_CG, CI - ci0);
    __syncthreads();
    for (int e = threadIdx.x; e < CONV_CG * 3 * E * E; e += CONV_THREADS) {
      int i = e / (3 * E * E), r = e - i * 3 * E * E;
      int dz = r / (E * E), r2 = r - dz * E * E;
      int yy = r2 / E - dil, xx = r2 % E - dil, zz = z + (dz - 1) * dil;
      float v = 0.f;
      if (i < cg && zz >= 0 && zz < D && yy >= 0 && yy < D && xx >= 0 && xx < D)
        v = to_f(in[((long long)n * CI + ci0 + i) * D3 + (long long)zz * D2 + yy * D + xx]);
      halo[e] = v;
    }
    for (int e = threadIdx.x; e < 27 * CONV_CG * CO4; e += CONV_THREADS) {
      int t = e / (CONV_CG * CO4), r = e - t * CONV_CG * CO4;
      int i = r / CO4, o = r - i * CO4;
      Ws[e] = (i < cg && o < CO) ? to_f(W[((long long)o * CI + ci0 + i) * 27 + t]) : 0.f;
    }
    __syncthreads();
    if (act) {
      for (int i = 0; i < cg; ++i) {
#pragma unroll
        for (int t = 0; t < 27; ++t) {
          const int dz = t / 9, dy = (t / 3) % 3, dx = t % 3;
          const float xv = halo[((i * 3 + dz) * E + (y + dy * dil)) * E + (x + dx * dil)];
          const float *wr = Ws + (t * CONV_CG + i) * CO4;
#pragma unroll
          for (int o4 = 0; o4 < CO4; o4 += 4) {
            float4 w = *reinterpret_cast<const float4 *>(wr + o4);
            if (o4 + 0 < CO) acc[o4 + 0] = fmaf(w.x, xv, acc[o4 + 0]);
            if (o4 + 1 < CO) acc[o4 + 1] = fmaf(w.y, xv, acc[o4 + 1]);
            if (o4 + 2 < CO) acc[o4 + 2] = fmaf(w.z, xv, acc[o4 + 2]);
            if (o4 + 3 < CO) acc[o4 + 3] = fmaf(w.w, xv, acc[o4 + 3]);
          }
        }
      }
    }
  }
  if (act) {
    const long long p = (long long)z * D2 + pos;
#pragma unroll
    for (int o = 0; o < CO; ++o) {
      float v = acc[o];
      const long long at = ((long long)n * CO + o) * D3 + p;
      if (relu) v = fmaxf(v, 0.f);
      if (mask && !(mask[at] > 0.f)) v = 0.f;
      out[at] = from_f<TO>(v);
    }
  }
}

// W'[i][o][t] = W[o][i][26 - t]: the adjoint of a convolution is the convolution (same dilation) with these
// weights
__global__ void k_flip_weights(const float *W, int CO, int CI, float *Wt) {
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)CO * CI * 27) return;
  int o = (int)(e / (CI * 27)), r = (int)(e - (long long)o * CI * 27);
  int i = r / 27, t = r - i * 27;
  Wt[((long long)i * CO + o) * 27 + (26 - t)] = W[e];
}

// ---------------------------------------------------------------- convolution, weight gradient
// gW[o][i][t] += sum_{n,p} gy[n][o][p] in[n][i][p + (t - 1) dil];  gb[o] += sum_{n,p} gy[n][o][p].
// One CTA per (sample, input-channel group of 8), looping over the z-slices.  Warp w owns output channels
// 4w..4w+3 (its 4 gradients of a position are one broadcast 16-byte load); lane c owns the (i, t) columns
// c, c+32, ... of the group (8 x 27 = 216 columns, 7 per lane).  Sums are added to gW with atomics.
template <int CO>
__global__ void __launch_bounds__(256) k_conv_wgrad(const float *in, int CI, const float *gy, float *gW, float *gb,
                                                    int D, int dil) {
  constexpr int NQ = (CO + 3) / 4;  // warps with work
  constexpr int NCOL = CONV_CG * 27, PER = (NCOL + 31) / 32;
  extern __shared__ __align__(16) float wsm[];
  const int E = D + 2 * dil, D2 = D * D, D3 = D2 * D;
  float *halo = wsm;                          // [CONV_CG][3][E][E]
  float *gs = wsm + CONV_CG * 3 * E * E;      // [D2][NQ*4]
  const int n = blockIdx.y, ci0 = blockIdx.x * CONV_CG;
  const int cg = min(CONV_CG, CI - ci0);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float acc[4][PER];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int m = 0; m < PER; ++m) acc[a][m] = 0.f;
  float bacc[4] = {0.f, 0.f, 0.f, 0.f};
  int offm[PER];
  bool okm[PER];
#pragma unroll
  for (int m = 0; m < PER; ++m) {
    int j = lane + 32 * m;
    int i = j / 27, t = j - i * 27;
    okm[m] = j < NCOL && i < cg;
    int dz = t / 9, dy = (t / 3) % 3, dx = t % 3;
    offm[m] = okm[m] ? ((i * 3 + dz) * E + dy * dil) * E + dx * dil : 0;
  }
  for (int z = 0; z < D; ++z) {
    __syncthreads();
    for (int e = threadIdx.x; e < CONV_CG * 3 * E * E; e += blockDim.x) {
      int i = e / (3 * E * E), r = e - i * 3 * E * E;
      int dz = r / (E * E), r2 = r - dz * E * E;
      int yy = r2 / E - dil, xx = r2 % E - dil, zz = z + (dz - 1) * dil;
      float v = 0.f;
      if (i < cg && zz >= 0 && zz < D && yy >= 0 && yy < D && xx >= 0 && xx < D)
        v = in[((long long)n * CI + ci0 + i) * D3 + (long long)zz * D2 + yy * D + xx];
      halo[e] = v;
    }
    for (int e = threadIdx.x; e < D2 * NQ * 4; e += blockDim.x) {
      int p = e / (NQ * 4), o = e - p * NQ * 4;
      gs[e] = (o < CO) ? gy[((long long)n * CO + o) * D3 + (long long)z * D2 + p] : 0.f;
    }
    __syncthreads();
    if (w < NQ) {
      for (int p = 0; p < D2; ++p) {
        const int y = p / D, x = p - y * D;
        const float4 g4 = *reinterpret_cast<const float4 *>(gs + p * NQ * 4 + 4 * w);
        const int base = y * E + x;
        if (ci0 == 0) {
          bacc[0] += g4.x;
          bacc[1] += g4.y;
          bacc[2] += g4.z;
          bacc[3] += g4.w;
        }
#pragma unroll
        for (int m = 0; m < PER; ++m) {
          const float v = halo[offm[m] + base];
          acc[0][m] = fmaf(g4.x, v, acc[0][m]);
          acc[1][m] = fmaf(g4.y, v, acc[1][m]);
          acc[2][m] = fmaf(g4.z, v, acc[2][m]);
          acc[3][m] = fmaf(g4.w, v, acc[3][m]);
        }
      }
    }
  }
  if (w < NQ) {
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int o = 4 * w + a;
      if (o >= CO) continue;
#pragma unroll
      for (int m = 0; m < PER; ++m) {
        if (!okm[m]) continue;
        int j = lane + 32 * m, i = j / 27, t = j - i * 27;
        atomicAdd(&gW[((long long)o * CI + ci0 + i) * 27 + t], acc[a][m]);
      }
      if (ci0 == 0 && lane == 0) atomicAdd(&gb[o], bacc[a]);
    }
  }
}

// ---------------------------------------------------------------- loss, Adam
// masked squared error: loss_sum += sum valid (q - t)^2, count += sum valid
__global__ void k_ws_loss(const float *q, const float *t, const float *valid, long long n, double *sums) {
  __shared__ double s0[8], s1[8];
  double a = 0.0, c = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    float m = valid[i];
    double d = (double)(q[i] - t[i]) * m;
    a += d * d;
    c += m;
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    c += __shfl_down_sync(0xffffffffu, c, o);
  }
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    s0[w] = a;
    s1[w] = c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double A = 0.0, C = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
      A += s0[i];
      C += s1[i];
    }
    atomicAdd(&sums[0], A);
    atomicAdd(&sums[1], C);
  }
}

// dL/dq = 2 (q - t) valid / count
__global__ void k_ws_loss_grad(const float *q, const float *t, const float *valid, long long n, const double *sums,
                               float *g) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double cnt = sums[1] > 0.0 ? sums[1] : 1.0;
  g[i] = (float)(2.0 * (double)(q[i] - t[i]) * valid[i] / cnt);
}

__global__ void k_adam(float *th, const float *g, float *m, float *v, long long n, float lr, float c1, float c2) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  float mi = b1 * m[i] + (1.f - b1) * g[i];
  float vi = b2 * v[i] + (1.f - b2) * g[i] * g[i];
  m[i] = mi;
  v[i] = vi;
  th[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void k_f32_to_bf16(const float *a, __nv_bfloat16 *b, long long n) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = __float2bfloat16_rn(a[i]);
}

}  // namespace

// ---------------------------------------------------------------- host: network passes
namespace {

size_t conv_smem(int CO, int D, int dil) {
  const int E = D + 2 * dil, CO4 = (CO + 3) / 4 * 4;
  return sizeof(float) * ((size_t)CONV_CG * 3 * E * E + (size_t)27 * CONV_CG * CO4);
}
size_t wgrad_smem(int CO, int D, int dil) {
  const int E = D + 2 * dil, NQ = (CO + 3) / 4;
  return sizeof(float) * ((size_t)CONV_CG * 3 * E * E + (size_t)D * D * NQ * 4);
}

template <int CO, typename TI, typename TO, typename TW>
void launch_conv(const TI *in, int CI, const TW *W, const TW *b, TO *out, int B, int D, int dil, bool relu,
                 const float *mask, cudaStream_t s) {
  auto kern = k_conv<CO, TI, TO, TW>;
  size_t sm = conv_smem(CO, D, dil);
  HP_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  kern<<<dim3(D, B), CONV_THREADS, sm, s>>>(in, CI, W, b, out, D, dil, relu ? 1 : 0, mask);
  HP_CHECK_LAUNCH();
}

template <int CO>
void launch_wgrad(const float *in, int CI, const float *gy, float *gW, float *gb, int B, int D, int dil,
                  cudaStream_t s) {
  auto kern = k_conv_wgrad<CO>;
  size_t sm = wgrad_smem(CO, D, dil);
  HP_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  kern<<<dim3((CI + CONV_CG - 1) / CONV_CG, B), 256, sm, s>>>(in, CI, gy, gW, gb, D, dil);
  HP_CHECK_LAUNCH();
}

}  // namespace

long long ws_num_params() { return WS_NPARAM; }

// forward in FP32 of B samples (input [B][5][D^3]); activations a1..a3 [B][32][D^3] and q [B][3][D^3]
static void ws_forward32(hplmm_ctx *c, const float *theta, const float *x, int B, int D, float *a1, float *a2,
                         float *a3, float *q) {
  cudaStream_t s = c->stream;
  const float *W[WS_NL], *bb[WS_NL];
  for (int l = 0; l < WS_NL; ++l) {
    W[l] = theta + layer_w_off(l);
    bb[l] = W[l] + (long long)WS_CH[l + 1] * WS_CH[l] * 27;
  }
  launch_conv<32, float, float, float>(x, 5, W[0], bb[0], a1, B, D, WS_DIL[0], true, nullptr, s);
  launch_conv<32, float, float, float>(a1, 32, W[1], bb[1], a2, B, D, WS_DIL[1], true, nullptr, s);
  launch_conv<32, float, float, float>(a2, 32, W[2], bb[2], a3, B, D, WS_DIL[2], true, nullptr, s);
  launch_conv<3, float, float, float>(a3, 32, W[3], bb[3], q, B, D, WS_DIL[3], false, nullptr, s);
}

// loss and gradient (FP32) of B samples; grad has WS_NPARAM entries (overwritten); returns the loss
double ws_loss_grad(hplmm_ctx *c, const float *theta, const float *x, const float *tgt, const float *valid, int B,
                    int D, float *grad) {
  cudaStream_t s = c->stream;
  auto &w = c->ws;
  const long long D3 = (long long)D * D * D;
  const long long nact = (long long)B * 32 * D3, nq = (long long)B * 3 * D3;
  w.a1.alloc(nact);
  w.a2.alloc(nact);
  w.a3.alloc(nact);
  w.q.alloc(nq);
  w.g32a.alloc(nact);
  w.g32b.alloc(nact);
  w.gq.alloc(nq);
  w.wflip.alloc(32 * 32 * 27);
  w.sums.alloc(2);
  ws_forward32(c, theta, x, B, D, w.a1.p, w.a2.p, w.a3.p, w.q.p);
  HP_CUDA(cudaMemsetAsync(w.sums.p, 0, 2 * sizeof(double), s));
  k_ws_loss<<<std::min<long long>(grid_for(nq, 256), 1024), 256, 0, s>>>(w.q.p, tgt, valid, nq, w.sums.p);
  HP_CHECK_LAUNCH();
  k_ws_loss_grad<<<grid_for(nq, 256), 256, 0, s>>>(w.q.p, tgt, valid, nq, w.sums.p, w.gq.p);
  HP_CHECK_LAUNCH();
  HP_CUDA(cudaMemsetAsync(grad, 0, sizeof(float) * WS_NPARAM, s));
  float *gW[WS_NL], *gb[WS_NL];
  const float *W[WS_NL];
  for (int l = 0; l < WS_NL; ++l) {
    W[l] = theta + layer_w_off(l);
    gW[l] = grad + layer_w_off(l);
    gb[l] = gW[l] + (long long)WS_CH[l + 1] * WS_CH[l] * 27;
  }
  // layer 4 (32 -> 3): weight gradient, then the data gradient through the ReLU of a3
  launch_wgrad<3>(w.a3.p, 32, w.gq.p, gW[3], gb[3], B, D, WS_DIL[3], s);
  k_flip_weights<<<grid_for(3 * 32 * 27, 256), 256, 0, s>>>(W[3], 3, 32, w.wflip.p);
  HP_CHECK_LAUNCH();
  launch_conv<32, float, float, float>(w.gq.p, 3, w.wflip.p, nullptr, w.g32a.p, B, D, WS_DIL[3], false, w.a3.p, s);
  // layer 3 (32 -> 32)
  launch_wgrad<32>(w.a2.p, 32, w.g32a.p, gW[2], gb[2], B, D, WS_DIL[2], s);
  k_flip_weights<<<grid_for(32 * 32 * 27, 256), 256, 0, s>>>(W[2], 32, 32, w.wflip.p);
  HP_CHECK_LAUNCH();
  launch_conv<32, float, float, float>(w.g32a.p, 32, w.wflip.p, nullptr, w.g32b.p, B, D, WS_DIL[2], false, w.a2.p,
                                       s);
  // layer 2 (32 -> 32)
  launch_wgrad<32>(w.a1.p, 32, w.g32b.p, gW[1], gb[1], B, D, WS_DIL[1], s);
  k_flip_weights<<<grid_for(32 * 32 * 27, 256), 256, 0, s>>>(W[1], 32, 32, w.wflip.p);
  HP_CHECK_LAUNCH();
  launch_conv<32, float, float, float>(w.g32b.p, 32, w.wflip.p, nullptr, w.g32a.p, B, D, WS_DIL[1], false, w.a1.p,
                                       s);
  // layer 1 (5 -> 32): weight gradient only
  launch_wgrad<32>(x, 5, w.g32a.p, gW[0], gb[0], B, D, WS_DIL[0], s);
  double h[2];
  HP_CUDA(cudaMemcpyAsync(h, w.sums.p, sizeof(h), cudaMemcpyDeviceToHost, s));
  HP_CUDA(cudaStreamSynchronize(s));
  return h[1] > 0.0 ? h[0] / h[1] : 0.0;
}

// inference: q [B][3][WS_D3] (FP32) from x [B][5][WS_D3] with BF16 weights and activations
void ws_infer(hplmm_ctx *c, const float *x, int B, float *q) {
  cudaStream_t s = c->stream;
  auto &w = c->ws;
  const long long nact = (long long)B * 32 * WS_D3;
  w.h1.alloc(nact);
  w.h2.alloc(nact);
  const __nv_bfloat16 *W[WS_NL], *bb[WS_NL];
  for (int l = 0; l < WS_NL; ++l) {
    W[l] = w.theta16.p + layer_w_off(l);
    bb[l] = W[l] + (long long)WS_CH[l + 1] * WS_CH[l] * 27;
  }
  launch_conv<32, float, __nv_bfloat16, __nv_bfloat16>(x, 5, W[0], bb[0], w.h1.p, B, WS_D, WS_DIL[0], true, nullptr,
                                                        s);
  launch_conv<32, __nv_bfloat16, __nv_bfloat16, __nv_bfloat16>(w.h1.p, 32, W[1], bb[1], w.h2.p, B, WS_D, WS_DIL[1],
                                                                true, nullptr, s);
  launch_conv<32, __nv_bfloat16, __nv_bfloat16, __nv_bfloat16>(w.h2.p, 32, W[2], bb[2], w.h1.p, B, WS_D, WS_DIL[2],
                                                                true, nullptr, s);
  launch_conv<3, __nv_bfloat16, float, __nv_bfloat16>(w.h1.p, 32, W[3], bb[3], q, B, WS_D, WS_DIL[3], false, nullptr,
                                                      s);
}

void ws_set_params(hplmm_ctx *c, const float *theta_host) {
  auto &w = c->ws;
  w.theta.alloc(WS_NPARAM);
  w.theta16.alloc(WS_NPARAM);
  w.m.alloc(WS_NPARAM);
  w.v.alloc(WS_NPARAM);
  w.grad.alloc(WS_NPARAM);
  HP_CUDA(cudaMemcpyAsync(w.theta.p, theta_host, sizeof(float) * WS_NPARAM, cudaMemcpyHostToDevice, c->stream));
  w.m.zero(c->stream);
  w.v.zero(c->stream);
  w.adam_step = 0;
  k_f32_to_bf16<<<grid_for(WS_NPARAM, 256), 256, 0, c->stream>>>(w.theta.p, w.theta16.p, WS_NPARAM);
  HP_CHECK_LAUNCH();
  HP_CUDA(cudaStreamSynchronize(c->stream));
  w.has_params = true;
}

void ws_get_params(hplmm_ctx *c, float *theta_host) {
  HP_REQUIRE(c->ws.has_params, HPLMM_ERR_STATE, "the warm-start network has no parameters yet");
  HP_CUDA(cudaMemcpyAsync(theta_host, c->ws.theta.p, sizeof(float) * WS_NPARAM, cudaMemcpyDeviceToHost, c->stream));
  HP_CUDA(cudaStreamSynchronize(c->stream));
}

// Adam over the collected samples in the given order (minibatches of `batch`); loss of every step to host
void ws_train(hplmm_ctx *c, const int32_t *order, long long n_order, int batch, double lr, double *loss_out) {
  auto &w = c->ws;
  HP_REQUIRE(w.has_params, HPLMM_ERR_STATE, "set the warm-start network parameters first");
  HP_REQUIRE(w.n_samples > 0, HPLMM_ERR_STATE, "no training samples collected");
  HP_REQUIRE(batch >= 1 && batch <= 256, HPLMM_ERR_INVALID, "batch must lie in [1, 256]");
  for (long long i = 0; i < n_order; ++i)
    HP_REQUIRE(order[i] >= 0 && order[i] < w.n_samples, HPLMM_ERR_INVALID, "sample index out of range");
  cudaStream_t s = c->stream;
  const long long S5 = 5LL * WS_D3, S3 = 3LL * WS_D3;
  w.bx.alloc((size_t)batch * S5);
  w.bt.alloc((size_t)batch * S3);
  w.bv.alloc((size_t)batch * S3);
  const long long steps = n_order / batch;
  for (long long st = 0; st < steps; ++st) {
    // gather the minibatch (device-to-device copies of whole samples)
    for (int b = 0; b < batch; ++b) {
      long long k = order[st * batch + b];
      HP_CUDA(cudaMemcpyAsync(w.bx.p + b * S5, w.tin.p + k * S5, sizeof(float) * S5, cudaMemcpyDeviceToDevice, s));
      HP_CUDA(cudaMemcpyAsync(w.bt.p + b * S3, w.ttgt.p + k * S3, sizeof(float) * S3, cudaMemcpyDeviceToDevice, s));
      HP_CUDA(cudaMemcpyAsync(w.bv.p + b * S3, w.tvalid.p + k * S3, sizeof(float) * S3, cudaMemcpyDeviceToDevice, s));
    }
    double loss = ws_loss_grad(c, w.theta.p, w.bx.p, w.bt.p, w.bv.p, batch, WS_D, w.grad.p);
    ++w.adam_step;
    const float c1 = (float)(1.0 - std::pow(0.9, (double)w.adam_step));
    const float c2 = (float)(1.0 - std::pow(0.999, (double)w.adam_step));
    k_adam<<<grid_for(WS_NPARAM, 256), 256, 0, s>>>(w.theta.p, w.grad.p, w.m.p, w.v.p, WS_NPARAM, (float)lr, c1, c2);
    HP_CHECK_LAUNCH();
    if (loss_out) loss_out[st] = loss;
  }
  k_f32_to_bf16<<<grid_for(WS_NPARAM, 256), 256, 0, s>>>(w.theta.p, w.theta16.p, WS_NPARAM);
  HP_CHECK_LAUNCH();
  HP_CUDA(cudaStreamSynchronize(s));
}

// ---------------------------------------------------------------- samples of the current set-up
namespace {

__global__ void k_ws_vbox(const int *vg, long long nv, int nx, int ny, int *vmin, int *vmax) {
  long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nv) return;
  int g = vg[v];
  if (g < 0) return;
  int p[3] = {(int)(v % nx), (int)((v / nx) % ny), (int)(v / ((long long)nx * ny))};
  for (int a = 0; a < 3; ++a) {
    atomicMin(&vmin[3 * g + a], p[a]);
    atomicMax(&vmax[3 * g + a], p[a]);
  }
}

// free local DOFs of each grain
__global__ void k_ws_nfree(int G, const long long *node_off, const int *nloc, const int *lnodes, const uint8_t *fixed,
                           int *nfree) {
  int g = blockIdx.x;
  if (g >= G) return;
  const int *ln = lnodes + node_off[g];
  int cnt = 0;
  for (int l = threadIdx.x; l < nloc[g]; l += blockDim.x) {
    int o = l / 3, d = l - 3 * o;
    cnt += fixed[3 * ln[o] + d] ? 0 : 1;
  }
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
  __shared__ int part[32];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += part[i];
    nfree[g] = t;
  }
}

// s_j = RMS of the right-hand side of sample j over its grain's free DOFs (one warp per sample)
__global__ void k_ws_scale(int S, const int *sg, const int *sa, const long long *node_off, const int *nloc,
                           const int *lnodes, const uint8_t *fixed, const long long *panel_off, const int *kg,
                           const float *rhs, const int *nfree, float *scale) {
  int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  int lane = threadIdx.x & 31;
  if (j >= S) return;
  int g = sg[j], a = sa[j], k = kg[g];
  const int *ln = lnodes + node_off[g];
  const float *R = rhs + panel_off[g];
  double acc = 0.0;
  for (int l = lane; l < nloc[g]; l += 32) {
    int o = l / 3, d = l - 3 * o;
    if (fixed[3 * ln[o] + d]) continue;
    double v = R[(long long)l * k + a];
    acc += v * v;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) scale[j] = nfree[g] > 0 ? (float)sqrt(acc / nfree[g]) : 0.f;
}

// inputs (and optionally targets and valid masks) of samples [j0, j0 + B), one CTA per sample;
// the destination arrays are zeroed first by the caller
__global__ void k_ws_fill(int j0, const int *sg, const int *sa, const int *vmin, const float *tscale,
                          const float *scale, const int *vg, const float *E, int nx, int ny, int nz,
                          const long long *node_off, const int *nloc, const int *lnodes, const int *node_ijk,
                          const uint8_t *fixed, const long long *panel_off, const int *kg, const float *rhs,
                          const float *sol, float *xin, float *tgt, float *valid) {
  constexpr int D = WS_D, D2 = D * D, D3 = D2 * D;
  int b = blockIdx.x, j = j0 + b;
  int g = sg[j], a = sa[j], k = kg[g];
  int ox = vmin[3 * g], oy = vmin[3 * g + 1], oz = vmin[3 * g + 2];
  float *X = xin + (long long)b * 5 * D3;
  for (int e = threadIdx.x; e < 16 * 16 * 16; e += blockDim.x) {
    int i = e & 15, jj = (e >> 4) & 15, kk = e >> 8;
    int x = ox + i, y = oy + jj, z = oz + kk;
    if (x >= nx || y >= ny || z >= nz) continue;
    long long v = ((long long)z * ny + y) * nx + x;
    if (vg[v] != g) continue;
    int p = kk * D2 + jj * D + i;
    X[p] = 1.f;
    X[D3 + p] = logf(E[v]);
  }
  const float s = scale[j];
  if (!(s > 0.f)) return;
  const float inv_s = 1.f / s, tsc = (tscale && tscale[j] > 0.f) ? 1.f / tscale[j] : 0.f;
  const int *ln = lnodes + node_off[g];
  const float *R = rhs + panel_off[g];
  const float *Y = sol ? sol + panel_off[g] : nullptr;
  for (int l = threadIdx.x; l < nloc[g]; l += blockDim.x) {
    int o = l / 3, d = l - 3 * o;
    int n = ln[o];
    if (fixed[3 * n + d]) continue;
    int p = (node_ijk[3 * n + 2] - oz) * D2 + (node_ijk[3 * n + 1] - oy) * D + (node_ijk[3 * n] - ox);
    X[(2 + d) * D3 + p] = R[(long long)l * k + a] * inv_s;
    if (tgt) tgt[(long long)b * 3 * D3 + d * D3 + p] = Y[(long long)l * k + a] * tsc;
    if (valid) valid[(long long)b * 3 * D3 + d * D3 + p] = 1.f;
  }
}

// x0 of samples [j0, j0 + B) from the predictions q (the direction of the guess on free DOFs, 0 on fixed
// ones and for a zero right-hand side)
__global__ void k_ws_guess(int j0, const int *sg, const int *sa, const int *vmin, const float *scale,
                           const long long *node_off, const int *nloc, const int *lnodes,
                           const int *node_ijk, const uint8_t *fixed, const long long *panel_off, const int *kg,
                           const float *q, float *x0) {
  constexpr int D = WS_D, D2 = D * D, D3 = D2 * D;
  int b = blockIdx.x, j = j0 + b;
  int g = sg[j], a = sa[j], k = kg[g];
  int ox = vmin[3 * g], oy = vmin[3 * g + 1], oz = vmin[3 * g + 2];
  const bool on = scale[j] > 0.f;
  const int *ln = lnodes + node_off[g];
  float *X0 = x0 + panel_off[g];
  for (int l = threadIdx.x; l < nloc[g]; l += blockDim.x) {
    int o = l / 3, d = l - 3 * o;
    int n = ln[o];
    float v = 0.f;
    if (!fixed[3 * n + d] && on) {
      int p = (node_ijk[3 * n + 2] - oz) * D2 + (node_ijk[3 * n + 1] - oy) * D + (node_ijk[3 * n] - ox);
      v = q[(long long)b * 3 * D3 + d * D3 + p];
    }
    X0[(long long)l * k + a] = v;
  }
}

}  // namespace

// per-grain origin, sample -> (grain, column) maps and right-hand-side scales of a panel (and the solution
// scales of a second panel when given)
static void ws_prepare(hplmm_ctx *c, const float *rhs_panel, const float *sol_panel = nullptr) {
  auto &w = c->ws;
  cudaStream_t s = c->stream;
  const int G = c->n_grains;
  std::vector<int> sg, sa;
  for (int g = 0; g < G; ++g)
    if (c->grains.h_n[g] > 0)
      for (int a = 0; a < c->h_kg[g]; ++a) {
        sg.push_back(g);
        sa.push_back(a);
      }
  w.S = (long long)sg.size();
  if (w.S == 0) return;
  w.sg.upload(sg, s);
  w.sa.upload(sa, s);
  w.vmin.alloc(3 * G);
  w.vmax.alloc(3 * G);
  w.vmin.fill_bytes(0x7f, s);
  w.vmax.fill_bytes(0x80, s);
  long long nv = (long long)c->nx * c->ny * c->nz;
  k_ws_vbox<<<grid_for(nv, 256), 256, 0, s>>>(c->vgrain.p, nv, c->nx, c->ny, w.vmin.p, w.vmax.p);
  HP_CHECK_LAUNCH();
  auto lo = w.vmin.download(s), hi = w.vmax.download(s);
  for (int g = 0; g < G; ++g) {
    if (lo[3 * g] > hi[3 * g]) continue;  // no solid voxel
    for (int a = 0; a < 3; ++a)
      HP_REQUIRE(hi[3 * g + a] - lo[3 * g + a] + 1 <= WS_D - 1, HPLMM_ERR_INVALID,
                 "warm start: grain " + std::to_string(g) + " spans more than 16 voxels along an axis");
  }
  w.nfree.alloc(G);
  k_ws_nfree<<<G, 256, 0, s>>>(G, c->grains.node_off.p, c->grains.n.p, c->grains.lnodes.p, c->fixed.p, w.nfree.p);
  HP_CHECK_LAUNCH();
  w.scale.alloc(w.S);
  k_ws_scale<<<grid_for(w.S * 32, 256), 256, 0, s>>>((int)w.S, w.sg.p, w.sa.p, c->grains.node_off.p, c->grains.n.p,
                                                     c->grains.lnodes.p, c->fixed.p, c->panel_off.p, c->kg.p,
                                                     rhs_panel, w.nfree.p, w.scale.p);
  HP_CHECK_LAUNCH();
  if (sol_panel) {
    w.tscale.alloc(w.S);
    k_ws_scale<<<grid_for(w.S * 32, 256), 256, 0, s>>>((int)w.S, w.sg.p, w.sa.p, c->grains.node_off.p,
                                                       c->grains.n.p, c->grains.lnodes.p, c->fixed.p, c->panel_off.p,
                                                       c->kg.p, sol_panel, w.nfree.p, w.tscale.p);
    HP_CHECK_LAUNCH();
  }
}

static void ws_fill(hplmm_ctx *c, long long j0, int B, const float *rhs_panel, const float *sol_panel, float *xin,
                    float *tgt, float *valid) {
  auto &w = c->ws;
  cudaStream_t s = c->stream;
  HP_CUDA(cudaMemsetAsync(xin, 0, sizeof(float) * (size_t)B * 5 * WS_D3, s));
  if (tgt) HP_CUDA(cudaMemsetAsync(tgt, 0, sizeof(float) * (size_t)B * 3 * WS_D3, s));
  if (valid) HP_CUDA(cudaMemsetAsync(valid, 0, sizeof(float) * (size_t)B * 3 * WS_D3, s));
  k_ws_fill<<<B, 256, 0, s>>>((int)j0, w.sg.p, w.sa.p, w.vmin.p, tgt ? w.tscale.p : nullptr, w.scale.p, c->vgrain.p,
                              c->E.p, c->nx,
                              c->ny, c->nz, c->grains.node_off.p, c->grains.n.p, c->grains.lnodes.p, c->node_ijk.p,
                              c->fixed.p, c->panel_off.p, c->kg.p, rhs_panel, sol_panel, xin, tgt, valid);
  HP_CHECK_LAUNCH();
}

// append the current set-up's basis problems (right-hand sides and exact FP32 solutions) to the training set
long long ws_collect(hplmm_ctx *c) {
  auto &w = c->ws;
  HP_REQUIRE(c->setup_done, HPLMM_ERR_STATE, "call hplmm_setup first");
  HP_REQUIRE(c->opt.local_prec == HPLMM_FP32 && c->Xrhs.n > 1 && c->X32.p != nullptr, HPLMM_ERR_STATE,
             "collecting warm-start samples needs a set-up with local_prec = FP32 and keep_basis_rhs = 1");
  ws_prepare(c, c->Xrhs.p, c->X32.p);
  if (w.S == 0) return w.n_samples;
  const long long S5 = 5LL * WS_D3, S3 = 3LL * WS_D3;
  const long long need = w.n_samples + w.S;
  if (need > w.cap) {
    long long cap = std::max<long long>(need, 2 * w.cap);
    Buf<float> a, b, v;
    a.alloc(cap * S5);
    b.alloc(cap * S3);
    v.alloc(cap * S3);
    if (w.n_samples) {
      HP_CUDA(cudaMemcpyAsync(a.p, w.tin.p, sizeof(float) * w.n_samples * S5, cudaMemcpyDeviceToDevice, c->stream));
      HP_CUDA(cudaMemcpyAsync(b.p, w.ttgt.p, sizeof(float) * w.n_samples * S3, cudaMemcpyDeviceToDevice, c->stream));
      HP_CUDA(cudaMemcpyAsync(v.p, w.tvalid.p, sizeof(float) * w.n_samples * S3, cudaMemcpyDeviceToDevice, c->stream));
      HP_CUDA(cudaStreamSynchronize(c->stream));
    }
    std::swap(w.tin.p, a.p);
    std::swap(w.tin.n, a.n);
    std::swap(w.tin.cap, a.cap);
    std::swap(w.ttgt.p, b.p);
    std::swap(w.ttgt.n, b.n);
    std::swap(w.ttgt.cap, b.cap);
    std::swap(w.tvalid.p, v.p);
    std::swap(w.tvalid.n, v.n);
    std::swap(w.tvalid.cap, v.cap);
    w.cap = cap;
  }
  const int CH = 256;
  for (long long j0 = 0; j0 < w.S; j0 += CH) {
    int B = (int)std::min<long long>(CH, w.S - j0);
    long long at = w.n_samples + j0;
    ws_fill(c, j0, B, c->Xrhs.p, c->X32.p, w.tin.p + at * S5, w.ttgt.p + at * S3, w.tvalid.p + at * S3);
  }
  HP_CUDA(cudaStreamSynchronize(c->stream));
  w.n_samples = need;
  return w.n_samples;
}

// initial guesses for every basis problem of the current set-up into x0 (panel layout) from the network
void ws_guess(hplmm_ctx *c, const float *rhs_panel, float *x0) {
  auto &w = c->ws;
  HP_REQUIRE(w.has_params, HPLMM_ERR_STATE, "warm start requested but the network has no parameters");
  ws_prepare(c, rhs_panel);
  if (w.S == 0) return;
  cudaStream_t s = c->stream;
  const int CH = 256;
  w.bx.alloc((size_t)CH * 5 * WS_D3);
  w.q.alloc((size_t)CH * 3 * WS_D3);
  for (long long j0 = 0; j0 < w.S; j0 += CH) {
    int B = (int)std::min<long long>(CH, w.S - j0);
    ws_fill(c, j0, B, rhs_panel, nullptr, w.bx.p, nullptr, nullptr);
    ws_infer(c, w.bx.p, B, w.q.p);
    k_ws_guess<<<B, 256, 0, s>>>((int)j0, w.sg.p, w.sa.p, w.vmin.p, w.scale.p, c->grains.node_off.p,
                                 c->grains.n.p, c->grains.lnodes.p, c->node_ijk.p, c->fixed.p, c->panel_off.p,
                                 c->kg.p, w.q.p, x0);
    HP_CHECK_LAUNCH();
  }
}

// ---------------------------------------------------------------- batched block-Jacobi PCG basis solve
namespace {

constexpr int ELL_W = 27;  // node neighbours (3x3x3 stencil)

struct PBox {
  int lo[3], ext[3], perm[3];
};
__device__ __forceinline__ int pbox_cell(const int *box, int k, int x, int y, int z) {
  const int *b = box + 9 * k;
  int p[3] = {x - b[0], y - b[1], z - b[2]};
  for (int a = 0; a < 3; ++a)
    if (p[a] < 0 || p[a] >= b[3 + a]) return -1;
  int f = b[6], m = b[7], s = b[8];
  return (p[s] * b[3 + m] + p[m]) * b[3 + f] + p[f];
}

// local ELL of each grain problem (the principal submatrix of A_hat, fixed components as identity rows) and
// the inverse of every node's 3x3 diagonal block; one thread per local node
__global__ void k_ws_ell(int G, const int *box, const long long *node_off, const int *nloc, const int *lmap,
                         const int *lnodes, const long long *ell_off, const int *node_ijk, const int *row_ptr,
                         const int *col, const double *val, const uint8_t *fixed, int *nb, float *blk, float *dinv) {
  int g = blockIdx.y;
  int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= G || o >= nloc[g] / 3) return;
  const long long off = node_off[g];
  const int n = lnodes[off + o];
  const long long e0 = ell_off[g] + o;  // node index in the ELL arrays
  int slot = 0;
  double D[9];
  for (int q = 0; q < 9; ++q) D[q] = 0.0;
  for (int p = row_ptr[n]; p < row_ptr[n + 1] && slot < ELL_W; ++p) {
    int m = col[p];
    int cell = pbox_cell(box, g, node_ijk[3 * m], node_ijk[3 * m + 1], node_ijk[3 * m + 2]);
    int om = cell >= 0 ? lmap[off + cell] : -1;
    if (om < 0) continue;
    float b9[9];
    for (int d = 0; d < 3; ++d)
      for (int d2 = 0; d2 < 3; ++d2) {
        double v = val[(long long)p * 9 + 3 * d + d2];
        if (fixed[3 * n + d] || fixed[3 * m + d2]) v = (m == n && d == d2) ? 1.0 : 0.0;
        b9[3 * d + d2] = (float)v;
        if (m == n) D[3 * d + d2] = v;
      }
    nb[e0 * ELL_W + slot] = om;
    for (int q = 0; q < 9; ++q) blk[(e0 * ELL_W + slot) * 9 + q] = b9[q];
    ++slot;
  }
  for (; slot < ELL_W; ++slot) nb[e0 * ELL_W + slot] = -1;
  // inverse of the symmetric positive definite 3x3 diagonal block by its adjugate
  double c00 = D[4] * D[8] - D[5] * D[7], c01 = D[5] * D[6] - D[3] * D[8], c02 = D[3] * D[7] - D[4] * D[6];
  double det = D[0] * c00 + D[1] * c01 + D[2] * c02;
  double id = det != 0.0 ? 1.0 / det : 0.0;
  double inv[9] = {c00 * id, (D[2] * D[7] - D[1] * D[8]) * id, (D[1] * D[5] - D[2] * D[4]) * id,
                   c01 * id, (D[0] * D[8] - D[2] * D[6]) * id, (D[2] * D[3] - D[0] * D[5]) * id,
                   c02 * id, (D[1] * D[6] - D[0] * D[7]) * id, (D[0] * D[4] - D[1] * D[3]) * id};
  for (int q = 0; q < 9; ++q) dinv[e0 * 9 + q] = (float)inv[q];
}

constexpr int PCG_THREADS = 256;
constexpr int PCG_NW = PCG_THREADS / 32;

// sum over the CTA of one value per lane (column): returns the total of this lane's column to every thread
__device__ __forceinline__ float col_reduce(float v, float (*red)[32]) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  red[w][lane] = v;
  __syncthreads();
  float t = 0.f;
#pragma unroll
  for (int i = 0; i < PCG_NW; ++i) t += red[i][lane];
  return t;
}

// One CTA per (grain, block of 32 right-hand sides): block-Jacobi preconditioned CG on every column,
// x (the panel) holding the initial guess on entry and the solution on exit, b the right-hand sides.
// Work vectors r, p, q live in `work` ([3][rows][32] per item).  Per column: iterations to reach
// ||b - A x|| <= tol ||b|| (or -1 when max_iters ran out) and the initial relative residual.
__global__ void __launch_bounds__(PCG_THREADS) k_ws_pcg(const int *items, int n_items, const int *nloc,
                                                        const long long *ell_off, const int *nb, const float *blk,
                                                        const float *dinv, const long long *panel_off, const int *kg,
                                                        const int *col0, const float *bpanel, float *xpanel,
                                                        const long long *work_off, float *work, float tol,
                                                        int max_iters, int *iters, float *rel0, int *unconv) {
  __shared__ float red[PCG_NW][32];
  __shared__ int s_done;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int it = blockIdx.x;
  if (it >= n_items) return;
  const int g = items[2 * it], a0 = items[2 * it + 1];
  const int N = nloc[g], nn = N / 3, k = kg[g];
  const int ncol = min(32, k - a0);
  const bool colok = lane < ncol;
  const long long E0 = ell_off[g];
  const float *B = bpanel + panel_off[g] + a0;
  float *X = xpanel + panel_off[g] + a0;
  float *R = work + work_off[it], *P = R + (long long)N * 32, *Q = P + (long long)N * 32;
  auto b_at = [&](int row) -> float { return colok ? B[(long long)row * k + lane] : 0.f; };
  // the guess x0 is first scaled by the energy-optimal factor alpha0 = (x0 . b) / (x0 . A x0), which can only
  // lower the A-norm error against the zero guess; then r = b - A x, z = D^{-1} r kept in P
  float bb = 0.f, xb = 0.f, xax = 0.f;
  for (int o = wid; o < nn; o += PCG_NW) {
    float ax[3] = {0.f, 0.f, 0.f};
    for (int sl = 0; sl < ELL_W; ++sl) {
      int om = nb[(E0 + o) * ELL_W + sl];
      if (om < 0) break;
      const float *b9 = blk + ((E0 + o) * ELL_W + sl) * 9;
      float x0 = colok ? X[(long long)(3 * om) * k + lane] : 0.f;
      float x1 = colok ? X[(long long)(3 * om + 1) * k + lane] : 0.f;
      float x2 = colok ? X[(long long)(3 * om + 2) * k + lane] : 0.f;
      ax[0] += b9[0] * x0 + b9[1] * x1 + b9[2] * x2;
      ax[1] += b9[3] * x0 + b9[4] * x1 + b9[5] * x2;
      ax[2] += b9[6] * x0 + b9[7] * x1 + b9[8] * x2;
    }
    for (int d = 0; d < 3; ++d) {
      float bv = b_at(3 * o + d);
      float xv = colok ? X[(long long)(3 * o + d) * k + lane] : 0.f;
      bb += bv * bv;
      xb += xv * bv;
      xax += xv * ax[d];
      Q[(long long)(3 * o + d) * 32 + lane] = ax[d];
    }
  }
  xb = col_reduce(xb, red);
  xax = col_reduce(xax, red);
  const float alpha0 = xax > 0.f ? xb / xax : 0.f;
  float rr = 0.f, rz = 0.f;
  for (int o = wid; o < nn; o += PCG_NW) {
    float r3[3];
    for (int d = 0; d < 3; ++d) {
      long long at = (long long)(3 * o + d) * 32 + lane;
      if (colok) X[(long long)(3 * o + d) * k + lane] *= alpha0;
      r3[d] = b_at(3 * o + d) - alpha0 * Q[at];
      rr += r3[d] * r3[d];
      R[at] = r3[d];
    }
    const float *di = dinv + (E0 + o) * 9;
    for (int d = 0; d < 3; ++d) {
      float z = di[3 * d] * r3[0] + di[3 * d + 1] * r3[1] + di[3 * d + 2] * r3[2];
      P[(long long)(3 * o + d) * 32 + lane] = z;
      rz += r3[d] * z;
    }
  }
  bb = col_reduce(bb, red);
  rr = col_reduce(rr, red);
  rz = col_reduce(rz, red);
  const float tol2 = tol * tol;
  bool conv = !colok || bb == 0.f || rr <= tol2 * bb;
  int my_iters = conv ? 0 : -1;
  if (colok) rel0[col0[g] + a0 + lane] = bb > 0.f ? sqrtf(rr / bb) : 0.f;
  for (int iter = 0; iter < max_iters; ++iter) {
    // stop when every column has converged
    if (threadIdx.x == 0) s_done = 0;
    __syncthreads();
    if (wid == 0) {
      unsigned all = __ballot_sync(0xffffffffu, conv);
      if (lane == 0) s_done = (all == 0xffffffffu);
    }
    __syncthreads();
    if (s_done) break;
    // q = A p, pq = p . q
    float pq = 0.f;
    for (int o = wid; o < nn; o += PCG_NW) {
      float ax[3] = {0.f, 0.f, 0.f};
      for (int sl = 0; sl < ELL_W; ++sl) {
        int om = nb[(E0 + o) * ELL_W + sl];
        if (om < 0) break;
        const float *b9 = blk + ((E0 + o) * ELL_W + sl) * 9;
        float p0 = P[(long long)(3 * om) * 32 + lane], p1 = P[(long long)(3 * om + 1) * 32 + lane],
              p2 = P[(long long)(3 * om + 2) * 32 + lane];
        ax[0] += b9[0] * p0 + b9[1] * p1 + b9[2] * p2;
        ax[1] += b9[3] * p0 + b9[4] * p1 + b9[5] * p2;
        ax[2] += b9[6] * p0 + b9[7] * p1 + b9[8] * p2;
      }
      for (int d = 0; d < 3; ++d) {
        Q[(long long)(3 * o + d) * 32 + lane] = ax[d];
        pq += P[(long long)(3 * o + d) * 32 + lane] * ax[d];
      }
    }
    pq = col_reduce(pq, red);
    const float alpha = (!conv && pq > 0.f) ? rz / pq : 0.f;
    // x += alpha p, r -= alpha q, z = D^{-1} r
    float rz2 = 0.f, rr2 = 0.f;
    for (int o = wid; o < nn; o += PCG_NW) {
      float r3[3];
      for (int d = 0; d < 3; ++d) {
        long long at = (long long)(3 * o + d) * 32 + lane;
        if (colok) X[(long long)(3 * o + d) * k + lane] += alpha * P[at];
        r3[d] = R[at] - alpha * Q[at];
        R[at] = r3[d];
        rr2 += r3[d] * r3[d];
      }
      const float *di = dinv + (E0 + o) * 9;
      for (int d = 0; d < 3; ++d) rz2 += r3[d] * (di[3 * d] * r3[0] + di[3 * d + 1] * r3[1] + di[3 * d + 2] * r3[2]);
    }
    rz2 = col_reduce(rz2, red);
    rr2 = col_reduce(rr2, red);
    if (!conv && rr2 <= tol2 * bb) {
      conv = true;
      my_iters = iter + 1;
    }
    const float beta = (!conv && rz > 0.f) ? rz2 / rz : 0.f;
    rz = rz2;
    // p = z + beta p
    for (int o = wid; o < nn; o += PCG_NW) {
      long long at0 = (long long)(3 * o) * 32 + lane;
      float r0 = R[at0], r1 = R[at0 + 32], r2 = R[at0 + 64];
      const float *di = dinv + (E0 + o) * 9;
      for (int d = 0; d < 3; ++d) {
        float z = di[3 * d] * r0 + di[3 * d + 1] * r1 + di[3 * d + 2] * r2;
        long long at = at0 + 32 * d;
        P[at] = z + beta * P[at];
      }
    }
  }
  if (colok) {
    iters[col0[g] + a0 + lane] = my_iters;
    if (my_iters < 0) atomicExch(&unconv[g], 1);
  }
}

}  // namespace

// basis solves by PCG (cold or warm start); returns nothing, fills c->bstats; grains with an unconverged
// column are re-solved exactly by the banded factor (the fallback)
void ws_pcg_basis(hplmm_ctx *c, bool warm) {
  auto &w = c->ws;
  cudaStream_t s = c->stream;
  LocalSet &S = c->grains;
  const int G = c->n_grains;
  const long long total = c->h_panel_off.empty() ? 0 : c->h_panel_off.back();
  // keep the right-hand sides: X32 becomes the iterate
  c->Xrhs.alloc(std::max<long long>(total, 1));
  HP_CUDA(cudaMemcpyAsync(c->Xrhs.p, c->X32.p, sizeof(float) * total, cudaMemcpyDeviceToDevice, s));
  cudaEvent_t e0, e1, e2;
  HP_CUDA(cudaEventCreate(&e0));
  HP_CUDA(cudaEventCreate(&e1));
  HP_CUDA(cudaEventCreate(&e2));
  HP_CUDA(cudaEventRecord(e0, s));
  if (warm)
    ws_guess(c, c->Xrhs.p, c->X32.p);
  else
    HP_CUDA(cudaMemsetAsync(c->X32.p, 0, sizeof(float) * total, s));
  HP_CUDA(cudaEventRecord(e1, s));
  // local ELL and block-Jacobi inverses
  std::vector<long long> eoff(G + 1, 0);
  int maxnodes = 1;
  for (int g = 0; g < G; ++g) {
    eoff[g + 1] = eoff[g] + S.h_n[g] / 3;
    maxnodes = std::max(maxnodes, S.h_n[g] / 3);
  }
  w.ell_off.upload(eoff, s);
  w.nb.alloc(std::max<long long>(eoff[G], 1) * ELL_W);
  w.blk.alloc(std::max<long long>(eoff[G], 1) * ELL_W * 9);
  w.dinv.alloc(std::max<long long>(eoff[G], 1) * 9);
  k_ws_ell<<<dim3(grid_for(maxnodes, 128), G), 128, 0, s>>>(G, S.box.p, S.node_off.p, S.n.p, S.lmap.p, S.lnodes.p,
                                                            w.ell_off.p, c->node_ijk.p, c->row_ptr.p, c->col.p,
                                                            c->val64.p, c->fixed.p, w.nb.p, w.blk.p, w.dinv.p);
  HP_CHECK_LAUNCH();
  // items (grain, 32-column block) and their work vectors
  std::vector<int> items, col0(G, 0);
  std::vector<long long> woff;
  long long wtot = 0;
  int ncols = 0;
  for (int g = 0; g < G; ++g) {
    col0[g] = ncols;
    ncols += c->h_kg[g];
    if (S.h_n[g] == 0) continue;
    for (int a0 = 0; a0 < c->h_kg[g]; a0 += 32) {
      items.push_back(g);
      items.push_back(a0);
      woff.push_back(wtot);
      wtot += 3LL * S.h_n[g] * 32;
    }
  }
  const int n_items = (int)items.size() / 2;
  w.iters.alloc(std::max(ncols, 1));
  w.rel0.alloc(std::max(ncols, 1));
  w.unconv.alloc(std::max(G, 1));
  w.iters.fill_bytes(0, s);
  w.rel0.zero(s);
  w.unconv.zero(s);
  if (n_items > 0) {
    Buf<int> it, c0;
    Buf<long long> wo;
    it.upload(items, s);
    c0.upload(col0, s);
    wo.upload(woff, s);
    w.pcg_work.alloc(std::max<long long>(wtot, 1));
    k_ws_pcg<<<n_items, PCG_THREADS, 0, s>>>(it.p, n_items, S.n.p, w.ell_off.p, w.nb.p, w.blk.p, w.dinv.p,
                                             c->panel_off.p, c->kg.p, c0.p, c->Xrhs.p, c->X32.p, wo.p, w.pcg_work.p,
                                             (float)c->opt.basis_tol, c->opt.basis_max_iters, w.iters.p, w.rel0.p,
                                             w.unconv.p);
    HP_CHECK_LAUNCH();
  }
  HP_CUDA(cudaEventRecord(e2, s));
  HP_CUDA(cudaEventSynchronize(e2));
  float t_net = 0.f, t_pcg = 0.f;
  HP_CUDA(cudaEventElapsedTime(&t_net, e0, e1));
  HP_CUDA(cudaEventElapsedTime(&t_pcg, e1, e2));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaEventDestroy(e2);
  auto hi = w.iters.download(s, ncols);
  auto hr = w.rel0.download(s, ncols);
  auto hu = w.unconv.download(s, G);
  hplmm_basis_stats &bs = c->bstats;
  bs = hplmm_basis_stats{};
  bs.columns = ncols;
  double rsum = 0.0;
  for (int j = 0; j < ncols; ++j) {
    if (hi[j] < 0) {
      ++bs.fallback_columns;
      bs.iters_total += c->opt.basis_max_iters;
      bs.iters_max = std::max<long long>(bs.iters_max, c->opt.basis_max_iters);
    } else {
      bs.iters_total += hi[j];
      bs.iters_max = std::max<long long>(bs.iters_max, hi[j]);
    }
    rsum += hr[j];
  }
  bs.init_rel_res_mean = ncols ? rsum / ncols : 0.0;
  bs.t_net_ms = t_net;
  bs.t_pcg_ms = t_pcg;
  // fallback: grains with an unconverged column are solved exactly from their right-hand sides
  std::vector<int> redo;
  for (int g = 0; g < G; ++g)
    if (hu[g]) redo.push_back(g);
  if (!redo.empty()) {
    for (int g : redo)
      HP_CUDA(cudaMemcpyAsync(c->X32.p + c->h_panel_off[g], c->Xrhs.p + c->h_panel_off[g],
                              sizeof(float) * (c->h_panel_off[g + 1] - c->h_panel_off[g]), cudaMemcpyDeviceToDevice,
                              s));
    solve_local_multi_f32_subset(c, S, c->X32.p, c->panel_off, c->kg, c->h_kg, redo);
  }
  bs.fallback_grains = (long long)redo.size();
}

}  // namespace hp
