// Sparse FP64 Cholesky of the coarse matrix A^o (paper Section 4.2, Eq. mg_struct; the paper applies
// (A^o)^{-1} with a direct solver, Section 6.3) and the coarse solve of every preconditioner apply.
//
// A^o = P_hat^T A_hat P_hat is the sum over grains of dense blocks on each grain's coupled coarse columns
// (the mortar columns of the interfaces it touches and its correction column), so the grains play the
// part of finite elements and the factor is multifrontal:
//   * symbolic (host): a recursive bisection of the grain centres (longest axis, median) is a
//     nested-dissection tree; each column group is eliminated at the lowest tree node whose subtree holds
//     every grain coupled to it; nodes with fewer than CF_AMIN columns are merged into their parents;
//     front f = its p pivot columns (padded with identity columns to P, a multiple of the 64-wide tile),
//     then its b boundary columns (columns of ancestors coupled to its subtree), sorted by elimination
//     rank; the boundary row positions in the parent's front are precomputed;
//   * numeric (GPU): the Galerkin product adds A^o's entries into the fronts (cf_add); fronts are then
//     factored level by level (all fronts of one height at once): right-looking 64 x 64 tile Cholesky of
//     the pivot columns with the Schur update of the whole front, the explicit inverse of the pivot block
//     alongside, and the update block added into the parent (extend-add);
//   * solve: per level, forward y_p = inv(L_pp) t_p and t_b -= L_bp y_p (ascending levels), then backward
//     y_p -= L_bp^T x_b and x_p = inv(L_pp)^T y_p (descending levels): four launches per level, each a
//     row- or column-parallel product over all fronts of the level.
#include "common.cuh"

#include <algorithm>
#include <numeric>

namespace hp {
namespace {

constexpr int CT = 64;        // tile edge of the front factorisation
constexpr int CF_AMIN = 64;   // fronts with fewer pivot columns are merged into their parents

enum Kind {
  K_POTRF = 0, K_TRSM, K_SYRK, K_TRINV_SCALE, K_TRINV_UPDATE, K_EXTEND, K_FWD_Y, K_FWD_B, K_BWD_B, K_BWD_Y,
  K_OZ_SLICE, K_OZ_SYRK
};

inline long long rup(long long a, long long b) { return (a + b - 1) / b * b; }

// ---------------------------------------------------------------- front factorisation kernels
// Diagonal tile of a front: Cholesky factor L_kk and its inverse W = L_kk^{-1}, one CTA of 512 threads.
// The kernel is on the critical path of the factorisation and its steps are short, so it is laid out for
// latency: one block barrier per step, and the pivot's square root off the path of the updates.
//   factor, right-looking on unscaled columns (a_rc -= a_rq a_cq / d_q): warp 0 holds the diagonal (lane l:
//   rows l and l + 32); the other 15 warps hold the strictly lower triangle, numbered "column 62 first, rows
//   ascending within a column", element e in slot e / 480 of owner e mod 480.  The trailing triangle of step q
//   is then the prefix e < M(q) and column q the 63 - q elements after it, so a warp's slot is wholly busy,
//   wholly idle or on the boundary.  Phase q: the owners update the prefix with column q (published raw in
//   row q of the shared tile) and publish column q + 1, which that update completed; warp 0 updates the
//   diagonal and the lane of row q + 1 takes its pivot (1/sqrt(d) by rsqrt, d / sqrt(d), 1/d) while the
//   others work;
//   inverse, right-looking, two phases behind: step q subtracts L_rq W_qj from rows r > q (columns j <= q,
//   addressed compactly) and finishes row q + 1 with 1/L_{q+1,q+1} as it makes the last update there; it
//   reads column q scaled, written over the raw one in the phase after the factor used it.
// The shared tile holds the factor's columns transposed in its upper part (raw, then scaled) and W's strict
// lower part below; W's diagonal and L's are the pivot arrays.  Pivot tiles are always full (P is a
// multiple of 64; padding columns are identity columns).
constexpr int PT_THREADS = 512;
constexpr int PT_OFF = CT * (CT - 1) / 2;                       // strictly lower elements
constexpr int PT_OWNERS = PT_THREADS - 32;                      // threads of warps 1 ..
constexpr int PT_SLOTS = (PT_OFF + PT_OWNERS - 1) / PT_OWNERS;  // register slots per owner

// elements of the columns right of q in the owners' numbering
__device__ __forceinline__ int pt_prefix(int q) { return q >= CT - 1 ? 0 : (CT - 2 - q) * (CT - 1 - q) / 2; }

__global__ void __launch_bounds__(PT_THREADS) k_cf_potrf(const FTask *tasks, const long long *foff, const int *mv,
                                                         const long long *doff, double *Fr, double *Dr,
                                                         int *status) {
  __shared__ double S[CT][CT + 1];  // S[q][r] = column q of the factor at row r > q; S[r][j] = W_rj, r > j
  __shared__ double prd[CT], piv[CT], pl[CT];  // 1/L_qq, 1/d_q, L_qq
  const FTask tk = tasks[blockIdx.x];
  const long long N = mv[tk.f];
  double *A = Fr + foff[tk.f];
  double *Dinv = Dr + doff[tk.f] + (long long)tk.a * CT * CT;
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  const int u = t - 32, ub = (wid - 1) * 32;
  const int k0 = tk.a * CT;
  for (int e = t; e < CT * CT; e += PT_THREADS) {
    const int r = e / CT, c = e % CT;
    if (c <= r) S[r][c] = A[(long long)(k0 + r) * N + k0 + c];
  }
  __syncthreads();
  double dg[2] = {0.0, 0.0};
  double a[PT_SLOTS];
  int rs[PT_SLOTS], cs[PT_SLOTS];
#pragma unroll
  for (int k = 0; k < PT_SLOTS; ++k) {
    // column j = 62 - c (from the right) holds j + 1 elements, rows c + 1 .. 63, from offset j (j + 1) / 2
    const int e = wid > 0 ? PT_OWNERS * k + u : 0;
    int j = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
    while (j > 0 && j * (j + 1) / 2 > e) --j;
    while ((j + 1) * (j + 2) / 2 <= e) ++j;
    cs[k] = CT - 2 - j;
    rs[k] = cs[k] + 1 + e - j * (j + 1) / 2;
    a[k] = (wid > 0 && e < PT_OFF) ? S[rs[k]][cs[k]] : 0.0;
  }
  if (wid == 0) {
    dg[0] = S[lane][lane];
    dg[1] = S[lane + 32][lane + 32];
  }
  __syncthreads();
  for (int e = t; e < CT * CT; e += PT_THREADS) {
    const int r = e / CT, c = e % CT;
    if (c < r) S[r][c] = 0.0;
  }
  auto pivot = [&](int q, double d) {
    if (!(d > 0.0)) {
      if (atomicCAS(status, 0, (int)HPLMM_ERR_SINGULAR) == 0) {
        status[1] = 3;
        status[2] = tk.f;
        status[3] = k0 + q;
      }
      d = 1.0;
    }
    const double r = rsqrt(d);
    prd[q] = r;
    piv[q] = r * r;
    pl[q] = d * r;
  };
  if (wid > 0) {
    const int lo = pt_prefix(0);
#pragma unroll
    for (int k = 0; k < PT_SLOTS; ++k) {
      const int e = PT_OWNERS * k + u;
      if (e >= lo && e < lo + CT - 1) S[0][rs[k]] = a[k];
    }
  } else if (lane == 0) {
    pivot(0, dg[0]);
  }
  __syncthreads();
  for (int cc = 0; cc <= CT; ++cc) {
    if (cc < CT) {
      const double iv = piv[cc];
      if (wid == 0) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int r = lane + 32 * h;
          if (r > cc) {
            const double v = S[cc][r];
            dg[h] -= (v * iv) * v;
          }
        }
        if (cc + 1 < CT && lane == ((cc + 1) & 31)) pivot(cc + 1, cc + 1 < 32 ? dg[0] : dg[1]);
      } else {
        const int M = pt_prefix(cc), Mn = pt_prefix(cc + 1);
        const double rd = prd[cc];
#pragma unroll
        for (int k = 0; k < PT_SLOTS; ++k) {
          const int eb = PT_OWNERS * k + ub, e = eb + lane;
          if (eb < M && e < M) {
            const double p = S[cc][rs[k]] * iv;
            a[k] -= p * S[cc][cs[k]];
            if (e >= Mn) S[cc + 1][rs[k]] = a[k];  // column cc + 1 is complete: publish it raw
          }
          if (eb + 31 >= M && eb < M + CT - 1 - cc && e >= M && e < M + CT - 1 - cc) a[k] *= rd;  // column cc
        }
      }
    }
    if (wid > 0 && cc >= 1) {
      // column cc - 1 scaled, over its raw copy (read by the factor in the previous phase)
      const int q = cc - 1, lo = pt_prefix(q), hi = lo + CT - 1 - q;
#pragma unroll
      for (int k = 0; k < PT_SLOTS; ++k) {
        const int eb = PT_OWNERS * k + ub, e = eb + lane;
        if (eb + 31 >= lo && eb < hi && e >= lo && e < hi) S[q][rs[k]] = a[k];
      }
    }
    if (wid > 0 && cc >= 2) {
      // inverse step q = cc - 2
      const int q = cc - 2, ncol = q + 1, cnt = (CT - 1 - q) * ncol;
      const double rq = prd[q], rn = prd[q + 1];
      for (int e = u; e < cnt; e += PT_OWNERS) {
        const int ro = e / ncol, j = e - ro * ncol, r = q + 1 + ro;
        const double wq = (j == q) ? rq : S[q][j];
        double v = S[r][j] - S[q][r] * wq;
        if (ro == 0) v *= rn;
        S[r][j] = v;
      }
    }
    __syncthreads();
  }
  for (int e = t; e < CT * CT; e += PT_THREADS) {
    const int r = e / CT, c = e % CT;
    A[(long long)(k0 + r) * N + k0 + c] = c < r ? S[c][r] : (c == r ? pl[r] : 0.0);
    Dinv[e] = c < r ? S[r][c] : (c == r ? prd[r] : 0.0);
  }
}

// F[it][kt] <- F[it][kt] inv(L_kk)^T for the tiles below the diagonal tile; CTA (tile, slice of 16 rows)
__global__ void __launch_bounds__(256) k_cf_trsm(const FTask *tasks, const long long *foff, const int *mv,
                                                 const long long *doff, double *Fr, const double *Dr) {
  __shared__ double Di[CT][CT + 1];
  __shared__ double Bt[16][CT + 1];
  const FTask tk = tasks[blockIdx.x];
  const long long N = mv[tk.f];
  double *A = Fr + foff[tk.f];
  const double *Dinv = Dr + doff[tk.f] + (long long)tk.a * CT * CT;
  const int rs = 16 * blockIdx.y;
  const int k0 = tk.a * CT, i0 = tk.b * CT;
  const int nbi = (int)min((long long)CT, N - i0);
  for (int e = threadIdx.x; e < CT * CT; e += blockDim.x) Di[e / CT][e % CT] = Dinv[e];
  for (int e = threadIdx.x; e < 16 * CT; e += blockDim.x) {
    const int r = e / CT, cc = e % CT;
    Bt[r][cc] = (rs + r < nbi) ? A[(long long)(i0 + rs + r) * N + k0 + cc] : 0.0;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 16 * CT; e += blockDim.x) {
    const int r = e / CT, cc = e % CT;
    double s0 = 0.0, s1 = 0.0;
    int q = 0;
    for (; q + 1 <= cc; q += 2) {
      s0 += Bt[r][q] * Di[cc][q];
      s1 += Bt[r][q + 1] * Di[cc][q + 1];
    }
    if (q <= cc) s0 += Bt[r][q] * Di[cc][q];
    if (rs + r < nbi) A[(long long)(i0 + rs + r) * N + k0 + cc] = s0 + s1;
  }
}

// F[it][jt] -= F[it][kt] F[jt][kt]^T for it >= jt > kt (lower tiles only, the boundary block included)
__global__ void __launch_bounds__(256) k_cf_syrk(const FTask *tasks, const long long *foff, const int *mv,
                                                 double *Fr) {
  __shared__ double Ai[CT][CT + 1];
  __shared__ double Aj[CT][CT + 1];
  const FTask tk = tasks[blockIdx.x];
  const long long N = mv[tk.f];
  double *A = Fr + foff[tk.f];
  const int k0 = tk.a * CT, i0 = tk.b * CT, j0 = tk.c * CT;
  const int nbi = (int)min((long long)CT, N - i0), nbj = (int)min((long long)CT, N - j0);
  for (int e = threadIdx.x; e < CT * CT; e += blockDim.x) {
    const int r = e / CT, cc = e % CT;
    Ai[r][cc] = r < nbi ? A[(long long)(i0 + r) * N + k0 + cc] : 0.0;
    Aj[r][cc] = r < nbj ? A[(long long)(j0 + r) * N + k0 + cc] : 0.0;
  }
  __syncthreads();
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;  // 256 threads, 4 x 4 outputs each
  double acc[4][4] = {};
  for (int q = 0; q < CT; ++q) {
    double a[4], b[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      a[u] = Ai[ty + 16 * u][q];
      b[u] = Aj[tx + 16 * u][q];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[u][v] += a[u] * b[v];
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int r = ty + 16 * u, cc = tx + 16 * v;
      if (r < nbi && cc < nbj && (tk.b != tk.c || cc <= r)) A[(long long)(i0 + r) * N + j0 + cc] -= acc[u][v];
    }
}

// ---- the Schur update on the tensor cores, FP64 by the Ozaki splitting scheme (Ozaki, Ogita, Oishi and Rump,
// "Error-free transformations of matrix multiplication by using fast routines of matrix multiplication and
// its applications", Numer. Algorithms 59, 2012).  Each row r of the panel column block kt is scaled by
// 2^-e_r with 2^e_r above the row's largest magnitude and cut to a 56-bit fixed-point integer M (truncated:
// an error below 2^-56 of the row's largest entry), written in base 256 as M = sum_p d_p 256^(6-p) with
// d_0 in [-256, 255] and d_1 .. d_6 in [0, 255]: every digit is exact in BF16.  A digit product summed over
// the tile's 64 columns is below 2^22 in magnitude, so tcgen05.mma kind::f16 (BF16 operands, FP32
// accumulation) computes it exactly; the products of one group g = p + q are accumulated in the same 64 TMEM
// columns (exact up to g = 3; from g = 4 on the FP32 rounding lies below 2^-52 of the leading group), and
// the groups g <= 6 are kept (the dropped ones lie below 2^-53 of |L_i||L_j|).  Then
// (L_i L_j^T)_ab = 2^(e_a + e_b - 64) sum_g 256^(6-g) D_g, recombined in FP64 by Horner's rule.
// CTA = 128 rows (two tiles of the column below the diagonal) x one 64-column tile, 128 threads: all seven
// digits of both operands are staged at once in the canonical K-major no-swizzle layout (168 KB), one
// thread issues the 28 x 4 MMAs (M = 128, N = 64, K = 16), one commit; each thread then reads its row's
// seven accumulators back with tcgen05.ld.
namespace oz {
constexpr int ND = 7;                         // base-256 digits per value
constexpr int A_BYTES = 128 * CT * 2;         // one digit of the 128-row operand (16 KB)
constexpr int B_BYTES = CT * CT * 2;          // one digit of the 64-row operand (8 KB)
constexpr int SMEM = ND * (A_BYTES + B_BYTES);  // 168 KB
constexpr int TMEM_COLS = 512;                // 7 groups x 64 columns
constexpr long long WAIT_CYCLES = 2000000000LL;

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
// byte offset of BF16 element (row, k), k a multiple of 8, in a K-major no-swizzle tile of 64 columns:
// 8-row x 16-byte core matrices, 128 bytes apart along K, 8-row groups 1024 bytes apart
__device__ __forceinline__ int off8(int row, int k) { return (row >> 3) * 1024 + (k >> 3) * 128 + (row & 7) * 16; }
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  const uint64_t lbo = 128 >> 4, sbo = 1024 >> 4;
  return (uint64_t)((addr >> 4) & 0x3fff) | (lbo << 16) | (sbo << 32) | (1ull << 46);
}
// kind::f16 instruction descriptor: D F32, A and B BF16 (K-major), N = 64, M = 128
__device__ __forceinline__ uint32_t idesc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(64 >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}
__device__ __forceinline__ void mma(uint32_t dtm, uint64_t a, uint64_t b, uint32_t id, int acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtm),
      "l"(a), "l"(b), "r"(id), "r"(acc)
      : "memory");
}
}  // namespace oz

// digits of the 64 rows of panel tile (it, kt) of a front (TRSM task {f, kt, it}): slot = the task's index,
// S[slot][digit][row][64 columns] and E[slot][row]
__global__ void __launch_bounds__(256) k_cf_oz_slice(const FTask *tasks, const long long *foff, const int *mv,
                                                     const double *Fr, __nv_bfloat16 *S, int *E) {
  const FTask tk = tasks[blockIdx.x];
  const long long m = mv[tk.f];
  const double *A = Fr + foff[tk.f];
  const int i0 = tk.b * CT, k0 = tk.a * CT;
  const int r = threadIdx.x >> 2, q = threadIdx.x & 3;  // row, quarter of its 64 columns
  const long long row = i0 + r;
  double v[16];
  double mx = 0.0;
#pragma unroll
  for (int e = 0; e < 16; ++e) {
    v[e] = row < m ? A[row * m + k0 + 16 * q + e] : 0.0;
    mx = fmax(mx, fabs(v[e]));
  }
  mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
  mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, 2));
  int ex = 0;
  if (mx > 0.0) frexp(mx, &ex);  // mx < 2^ex
  if (q == 0) E[(long long)blockIdx.x * CT + r] = ex;
  __nv_bfloat16 *Sd = S + (long long)blockIdx.x * oz::ND * CT * CT;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    long long M[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) M[e] = __double2ll_rz(ldexp(v[8 * h + e], 56 - ex));
#pragma unroll
    for (int d = 0; d < oz::ND; ++d) {
      __align__(16) __nv_bfloat16 o[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int dig = d == 0 ? (int)(M[e] >> 48) : (int)((M[e] >> (8 * (6 - d))) & 255);
        o[e] = __int2bfloat16_rn(dig);
      }
      *reinterpret_cast<uint4 *>(Sd + ((long long)d * CT + r) * CT + 16 * q + 8 * h) = *reinterpret_cast<uint4 *>(o);
    }
  }
}

// F[rows of tiles it, it+1][tile jt] -= L L^T on the tensor cores (task {f, kt, it, jt, slot(it), slot(jt)});
// 256 threads: all stage (eight 16-byte loads in flight per thread), warp w reads TMEM lanes 32 (w mod 4)
// .. + 31 and columns 32 (w / 4) .. + 31 of every group.  The groups are recombined in 64-bit integers:
// sum_{g<=5} D_g 256^(5-g) + floor(D_6 / 256) stays below 2^63 (|D_0| < 2^22), and the dropped fraction is
// below 2^-62 of it; one conversion to FP64 and a scaling by 2^(e_a + e_b - 56) follow.
constexpr int OZ_THREADS = 256;
__global__ void __launch_bounds__(OZ_THREADS) k_cf_oz_syrk(const int *otask, const long long *foff, const int *mv,
                                                           double *Fr, const __nv_bfloat16 *S, const int *E,
                                                           int *status) {
  extern __shared__ __align__(1024) unsigned char osm[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
  const int *t = otask + 6LL * blockIdx.x;
  const int f = t[0], it = t[2], jt = t[3], si = t[4], sj = t[5];
  const long long m = mv[f];
  double *A = Fr + foff[f];
  const int Tf = (int)((m + CT - 1) / CT);
  const bool two = it + 1 < Tf;
  if (wid == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(oz::su32(&tmem_base)),
                 "r"(oz::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(oz::su32(&bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // stage the digits: A rows 0..63 from slot si, 64..127 from slot si + 1 (zero rows past the front), then B
  constexpr int NA = oz::ND * 128 * 8, NBC = oz::ND * 64 * 8;  // 16-byte chunks
  unsigned char *Bs = osm + oz::ND * oz::A_BYTES;
  for (int c0 = tid; c0 < NA + NBC; c0 += 8 * OZ_THREADS) {
    uint4 v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int c = c0 + u * OZ_THREADS;
      v[u] = make_uint4(0u, 0u, 0u, 0u);
      if (c < NA) {
        const int d = c >> 10, row = (c >> 3) & 127, kc = c & 7;
        if (row < 64 || two) {
          const int slot = row < 64 ? si : si + 1;
          v[u] = __ldg(reinterpret_cast<const uint4 *>(S + (((long long)slot * oz::ND + d) * CT + (row & 63)) * CT +
                                                      8 * kc));
        }
      } else if (c < NA + NBC) {
        const int cb = c - NA, d = cb >> 9, row = (cb >> 3) & 63, kc = cb & 7;
        v[u] = __ldg(reinterpret_cast<const uint4 *>(S + (((long long)sj * oz::ND + d) * CT + row) * CT + 8 * kc));
      }
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int c = c0 + u * OZ_THREADS;
      if (c < NA) {
        const int d = c >> 10, row = (c >> 3) & 127, kc = c & 7;
        *reinterpret_cast<uint4 *>(osm + d * oz::A_BYTES + oz::off8(row, 8 * kc)) = v[u];
      } else if (c < NA + NBC) {
        const int cb = c - NA, d = cb >> 9, row = (cb >> 3) & 63, kc = cb & 7;
        *reinterpret_cast<uint4 *>(Bs + d * oz::B_BYTES + oz::off8(row, 8 * kc)) = v[u];
      }
    }
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t dtm = tmem_base;
  if (tid == 0) {
    const uint32_t id = oz::idesc();
    const uint32_t abase = oz::su32(osm), bbase = oz::su32(Bs);
    for (int p = 0; p < oz::ND; ++p)
      for (int q = 0; p + q < oz::ND; ++q) {
        const int g = p + q;
        for (int ks = 0; ks < CT / 16; ++ks) {
          const uint64_t ad = oz::sdesc(abase + p * oz::A_BYTES + ks * 256);
          const uint64_t bd = oz::sdesc(bbase + q * oz::B_BYTES + ks * 256);
          // the loop meets every group first at p = 0, which starts its accumulator
          oz::mma(dtm + (uint32_t)(g * 64), ad, bd, id, (p > 0 || ks > 0) ? 1 : 0);
        }
      }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(oz::su32(&bar))
                 : "memory");
  }
  bool ok = true;
  for (int attempt = 0; attempt < 2; ++attempt) {
    // the second (longer) wait only after a timeout: the MMAs must not outlive the tensor memory
    const long long t0 = clock64(), budget = (attempt + 1) * oz::WAIT_CYCLES;
    bool done = false;
    for (;;) {
      uint32_t d;
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.b32 %0, 1, 0, p;\n}\n"
          : "=r"(d)
          : "r"(oz::su32(&bar))
          : "memory");
      if (d) {
        done = true;
        break;
      }
      if (clock64() - t0 > budget) break;
    }
    if (done) break;
    if (ok) atomicCAS(status, 0, (int)HPLMM_ERR_TIMEOUT);
    ok = false;
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const int r = 32 * (wid & 3) + lane;            // row of the 128-row block
  const int ch = wid >> 2;                         // column half
  const long long grow = (long long)it * CT + r;   // row in the front
  const int rtile = it + (r >> 6);
  const int ei = E[(long long)(r < 64 ? si : si + 1) * CT + (r & 63)];
  for (int c0 = 32 * ch; c0 < 32 * ch + 32; c0 += 16) {
    long long acc[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) acc[i] = 0;
    for (int g = 0; g < oz::ND; ++g) {
      uint32_t u[16];
      const uint32_t taddr = dtm + ((uint32_t)(32 * (wid & 3)) << 16) + (uint32_t)(g * 64 + c0);
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]),
            "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15])
          : "r"(taddr)
          : "memory");
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const long long v = (long long)__float2int_rn(__uint_as_float(u[i]));  // an integer below 2^26
        acc[i] += g < 6 ? (v << (8 * (5 - g))) : (v >> 8);
      }
    }
    if (ok && grow < m) {
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int cc = c0 + i;
        const long long col = (long long)jt * CT + cc;
        if (col < m && (rtile != jt || cc <= (r & 63)) && acc[i] != 0)
          A[grow * m + col] -= ldexp((double)acc[i], ei + E[(long long)sj * CT + cc] - 56);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (wid == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(dtm), "r"(oz::TMEM_COLS) : "memory");
}

// Explicit inverse of the pivot block, Y = inv(L_pp) (P x P, row-major), by right-looking block
// substitution of L Y = I: Y starts as the identity; step kt: Y[kt][jt] <- inv(L_kk) Y[kt][jt] (jt <= kt),
// then Y[it][jt] -= L[it][kt] Y[kt][jt] for kt < it < P / 64.
__global__ void k_cf_eye(const int *Pv, const long long *yoff, int nf, double *Yr) {
  const int f = blockIdx.y;
  if (f >= nf) return;
  const long long P = Pv[f];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < P * P; i += (long long)gridDim.x * blockDim.x)
    Yr[yoff[f] + i] = (i / P == i % P) ? 1.0 : 0.0;
}

// Y[kt][jt] <- inv(L_kk) Y[kt][jt]: one CTA owns the whole tile (it is read and written in place, so no
// other CTA may read it meanwhile); inv(L_kk) rows come through the read-only cache
__global__ void __launch_bounds__(256) k_cf_trinv_scale(const FTask *tasks, const int *Pv, const long long *yoff,
                                                        const long long *doff, double *Yr, const double *Dr) {
  __shared__ double Bt[CT][CT + 1];
  const FTask tk = tasks[blockIdx.x];
  const long long P = Pv[tk.f];
  double *Y = Yr + yoff[tk.f];
  const double *Dinv = Dr + doff[tk.f] + (long long)tk.a * CT * CT;
  const int k0 = tk.a * CT, j0 = tk.b * CT;
  for (int e = threadIdx.x; e < CT * CT; e += blockDim.x) Bt[e / CT][e % CT] = Y[(k0 + e / CT) * P + j0 + e % CT];
  __syncthreads();
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4] = {};
  for (int q = 0; q < CT; ++q) {
    double a[4], b[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      a[u] = __ldg(Dinv + (ty + 16 * u) * CT + q);
      b[u] = Bt[q][tx + 16 * u];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[u][v] += a[u] * b[v];
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) Y[(k0 + ty + 16 * u) * P + j0 + tx + 16 * v] = acc[u][v];
}

__global__ void __launch_bounds__(256) k_cf_trinv_update(const FTask *tasks, const int *mv, const int *Pv,
                                                         const long long *foff, const long long *yoff,
                                                         const double *Fr, double *Yr) {
  __shared__ double Lt[CT][CT + 1];
  __shared__ double Yt[CT][CT + 1];
  const FTask tk = tasks[blockIdx.x];
  const long long N = mv[tk.f], P = Pv[tk.f];
  const double *L = Fr + foff[tk.f];
  double *Y = Yr + yoff[tk.f];
  const int k0 = tk.a * CT, i0 = tk.b * CT, j0 = tk.c * CT;
  for (int e = threadIdx.x; e < CT * CT; e += blockDim.x) {
    const int r = e / CT, cc = e % CT;
    Lt[r][cc] = L[(long long)(i0 + r) * N + k0 + cc];
    Yt[r][cc] = Y[(k0 + r) * P + j0 + cc];
  }
  __syncthreads();
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4] = {};
  for (int q = 0; q < CT; ++q) {
    double a[4], b[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      a[u] = Lt[ty + 16 * u][q];
      b[u] = Yt[q][tx + 16 * u];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[u][v] += a[u] * b[v];
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) Y[(i0 + ty + 16 * u) * P + j0 + tx + 16 * v] -= acc[u][v];
}

// identity on the padding rows and columns of every front's pivot block (rows p .. P-1)
__global__ void k_cf_pad(const int *pv, const int *Pv, const int *mv, const long long *foff, int nf, double *Fr) {
  const int f = blockIdx.x;
  if (f >= nf) return;
  const long long m = mv[f];
  for (int i = pv[f] + threadIdx.x; i < Pv[f]; i += blockDim.x) Fr[foff[f] + (long long)i * m + i] = 1.0;
}

// F[i][j] = (F[i][j] + F[j][i]) / 2 for the entries of the pivot columns (j < P, i > j): A^o is symmetric and
// the Galerkin product added both halves; the factorisation reads the lower triangle
__global__ void k_cf_symmetrize(const int *Pv, const int *mv, const long long *foff, int nf, double *Fr) {
  const int f = blockIdx.y;
  if (f >= nf) return;
  const long long m = mv[f], P = Pv[f];
  double *A = Fr + foff[f];
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < m * P; e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / P, j = e % P;
    if (i <= j) continue;
    const double v = 0.5 * (A[i * m + j] + A[j * m + i]);
    A[i * m + j] = v;
  }
}

// extend-add: the update block of front f (its boundary x boundary lower triangle, tile (it, jt)) into the
// parent's front at the precomputed rows
__global__ void __launch_bounds__(256) k_cf_extend(const FTask *tasks, const int *mv, const int *Pv, const int *bv,
                                                   const int *parent, const long long *foff, const long long *roff,
                                                   const int *rel, double *Fr) {
  const FTask tk = tasks[blockIdx.x];
  const int f = tk.f, u = parent[f];
  const long long m = mv[f], P = Pv[f], mu = mv[u];
  const int b = bv[f];
  const double *A = Fr + foff[f];
  double *B = Fr + foff[u];
  const int *rl = rel + roff[f];
  for (int e = threadIdx.x; e < CT * CT; e += blockDim.x) {
    const int i = tk.a * CT + e / CT, j = tk.b * CT + e % CT;
    if (i >= b || j > i) continue;
    const double v = A[(P + i) * m + P + j];
    if (v != 0.0) atomicAdd(&B[(long long)rl[i] * mu + rl[j]], v);
  }
}

// ---------------------------------------------------------------- coarse solve kernels
// Forward kernels: CTA = 32 rows of one front, warp w the rows w, w + 8, w + 16, w + 24 of the block.  The
// gathered right-hand side (t or y at the front's pivot columns) is staged in shared memory in chunks of
// FW_CH values, so that each row is a contiguous stream against shared memory, the four rows' loads of a
// lane are independent (four in flight), and no load waits on an index load.
constexpr int FW_CH = 2048;

// forward, pivot rows: y[idx_i] = sum_{j <= i} Y[i][j] t[idx_j]
__global__ void __launch_bounds__(256) k_cf_fwd_y(const FTask *tasks, const int *pv, const int *Pv,
                                                  const long long *yoff, const long long *ioff, const int *idx,
                                                  const double *Yr, const double *t, double *y) {
  __shared__ double tl[FW_CH];
  const FTask tk = tasks[blockIdx.x];
  const int p = pv[tk.f];
  const long long P = Pv[tk.f];
  const double *Y = Yr + yoff[tk.f];
  const int *ix = idx + ioff[tk.f];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int rend = min(tk.a + 32, p);
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int j0 = 0; j0 < rend; j0 += FW_CH) {
    const int jn = min(FW_CH, rend - j0);
    __syncthreads();
    for (int j = threadIdx.x; j < jn; j += blockDim.x) tl[j] = t[ix[j0 + j]];
    __syncthreads();
    const double *yr[4];
    int lim[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int r = tk.a + wid + 8 * u;
      lim[u] = r < rend ? min(jn, r - j0 + 1) : 0;  // row r reads columns j <= r
      yr[u] = Y + (long long)(r < rend ? r : tk.a) * P + j0;
    }
    for (int j = lane; j < lim[0] || j < lim[1] || j < lim[2] || j < lim[3]; j += 32) {
      const double tv = tl[j];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (j < lim[u]) acc[u] = fma(yr[u][j], tv, acc[u]);
    }
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    double sum = acc[u];
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o);
    const int r = tk.a + wid + 8 * u;
    if (lane == 0 && r < rend) y[ix[r]] = sum;
  }
}

// forward, boundary rows: t[idx_i] -= sum_j L_bp[i][j] y[idx_j]; several fronts of a level may share a
// boundary column, hence the atomic update
__global__ void __launch_bounds__(256) k_cf_fwd_b(const FTask *tasks, const int *pv, const int *Pv, const int *bv,
                                                  const int *mv, const long long *foff, const long long *ioff,
                                                  const int *idx, const double *Fr, const double *y, double *t) {
  __shared__ double yl[FW_CH];
  const FTask tk = tasks[blockIdx.x];
  const int p = pv[tk.f], b = bv[tk.f];
  const long long P = Pv[tk.f], m = mv[tk.f];
  const double *L = Fr + foff[tk.f];
  const int *ix = idx + ioff[tk.f];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int rend = min(tk.a + 32, b);
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int j0 = 0; j0 < p; j0 += FW_CH) {
    const int jn = min(FW_CH, p - j0);
    __syncthreads();
    for (int j = threadIdx.x; j < jn; j += blockDim.x) yl[j] = y[ix[j0 + j]];
    __syncthreads();
    const double *lr[4];
    int lim[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int r = tk.a + wid + 8 * u;
      lim[u] = r < rend ? jn : 0;
      lr[u] = L + (P + (r < rend ? r : tk.a)) * m + j0;
    }
    for (int j = lane; j < lim[0]; j += 32) {  // lim[0] is the largest
      const double yv = yl[j];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (j < lim[u]) acc[u] = fma(lr[u][j], yv, acc[u]);
    }
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    double sum = acc[u];
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o);
    const int r = tk.a + wid + 8 * u;
    if (lane == 0 && r < rend && sum != 0.0) atomicAdd(&t[ix[P + r]], -sum);
  }
}

// backward, boundary part: y[idx_j] -= sum_i L_bp[i][j] x[idx_{P+i}]; CTA = 256 pivot columns x 64
// boundary rows of one front
__global__ void __launch_bounds__(256) k_cf_bwd_b(const FTask *tasks, const int *pv, const int *Pv, const int *bv,
                                                  const int *mv, const long long *foff, const long long *ioff,
                                                  const int *idx, const double *Fr, const double *x, double *y) {
  __shared__ double xs[64];
  const FTask tk = tasks[blockIdx.x];
  const int p = pv[tk.f], b = bv[tk.f];
  const long long P = Pv[tk.f], m = mv[tk.f];
  const double *L = Fr + foff[tk.f];
  const int *ix = idx + ioff[tk.f];
  const int nr = min(64, b - tk.b);
  if (threadIdx.x < nr) xs[threadIdx.x] = x[ix[P + tk.b + threadIdx.x]];
  __syncthreads();
  const int j = tk.a + threadIdx.x;
  if (j >= p) return;
  const double *lc = L + (P + tk.b) * m + j;
  double s0 = 0.0, s1 = 0.0;
  int i = 0;
  for (; i + 1 < nr; i += 2) {
    s0 += lc[i * m] * xs[i];
    s1 += lc[(i + 1) * m] * xs[i + 1];
  }
  if (i < nr) s0 += lc[i * m] * xs[i];
  const double s = s0 + s1;
  if (s != 0.0) atomicAdd(&y[ix[j]], -s);
}

// backward, pivot part: x[idx_i] += sum_{j >= i} Y[j][i] y[idx_j]; CTA = 256 columns x 64 rows of one front
__global__ void __launch_bounds__(256) k_cf_bwd_y(const FTask *tasks, const int *pv, const int *Pv,
                                                  const long long *yoff, const long long *ioff, const int *idx,
                                                  const double *Yr, const double *y, double *x) {
  __shared__ double ys[64];
  const FTask tk = tasks[blockIdx.x];
  const int p = pv[tk.f];
  const long long P = Pv[tk.f];
  const double *Y = Yr + yoff[tk.f];
  const int *ix = idx + ioff[tk.f];
  const int nr = min(64, p - tk.b);
  if (threadIdx.x < nr) ys[threadIdx.x] = y[ix[tk.b + threadIdx.x]];
  __syncthreads();
  const int i = tk.a + threadIdx.x;
  if (i >= p) return;
  const double *yc = Y + tk.b * P + i;
  double s0 = 0.0, s1 = 0.0;
  int q = max(0, i - tk.b);  // rows j >= i only
  for (; q + 1 < nr; q += 2) {
    s0 += yc[q * P] * ys[q];
    s1 += yc[(q + 1) * P] * ys[q + 1];
  }
  if (q < nr) s0 += yc[q * P] * ys[q];
  const double s = s0 + s1;
  if (s != 0.0) atomicAdd(&x[ix[i]], s);
}

// ---------------------------------------------------------------- symbolic analysis
struct TNode {
  int parent = -1;
  std::vector<int> kids;    // children in the (merged) tree
  std::vector<int> grains;  // grains whose leaf is this node (after merging)
  std::vector<int> groups;  // column groups eliminated here (after merging: absorbed children first)
  int depth = 0;
  bool kept = true;
};

}  // namespace

void cf_analyse(hplmm_ctx *c, const std::vector<int> &gbox) {
  cudaStream_t s = c->stream;
  CoarseFactor &F = c->cf;
  const int G = c->n_grains;
  const int nI = c->n_ifaces;
  const long long No = c->n_coarse;
  // column groups: interfaces 0..nI-1 (their mortar columns), then one group per kept correction column
  std::vector<int> grp_first, grp_count, corr_group(G, -1);
  for (int ci = 0; ci < nI; ++ci) {
    grp_first.push_back(c->h_col_off[ci]);
    grp_count.push_back(c->h_col_off[ci + 1] - c->h_col_off[ci]);
  }
  for (int g = 0; g < G; ++g)
    if (c->h_corr_col[g] >= 0) {
      corr_group[g] = (int)grp_first.size();
      grp_first.push_back(c->h_corr_col[g]);
      grp_count.push_back(1);
    }
  const int NG = (int)grp_first.size();
  // groups of every grain (its coupled interfaces, then its correction)
  auto grain_groups = [&](int g, auto &&fn) {
    for (int q = c->h_gi_off[g]; q < c->h_gi_off[g + 1]; ++q) fn(c->h_gi_iface[q]);
    if (corr_group[g] >= 0) fn(corr_group[g]);
  };

  // 1. bisection tree of the grain centres
  std::vector<TNode> T;
  std::vector<int> leaf(G, 0);
  {
    std::vector<double> ctr(3 * (size_t)G, 0.0);
    for (int g = 0; g < G; ++g)
      for (int a = 0; a < 3; ++a)
        ctr[3 * g + a] = gbox[6 * g + 3 + a] > 0 ? gbox[6 * g + a] + 0.5 * gbox[6 * g + 3 + a] : 0.0;
    struct Item {
      int node;
      std::vector<int> set;
    };
    std::vector<Item> stack;
    std::vector<int> all(G);
    std::iota(all.begin(), all.end(), 0);
    T.emplace_back();
    stack.push_back({0, all});
    while (!stack.empty()) {
      Item it = std::move(stack.back());
      stack.pop_back();
      if (it.set.size() <= 1) {
        for (int g : it.set) {
          leaf[g] = it.node;
          T[it.node].grains.push_back(g);
        }
        continue;
      }
      double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
      for (int g : it.set)
        for (int a = 0; a < 3; ++a) {
          lo[a] = std::min(lo[a], ctr[3 * g + a]);
          hi[a] = std::max(hi[a], ctr[3 * g + a]);
        }
      int ax = 0;
      for (int a = 1; a < 3; ++a)
        if (hi[a] - lo[a] > hi[ax] - lo[ax]) ax = a;
      std::stable_sort(it.set.begin(), it.set.end(),
                       [&](int a, int b) { return ctr[3 * a + ax] < ctr[3 * b + ax]; });
      const size_t half = it.set.size() / 2;
      std::vector<int> L(it.set.begin(), it.set.begin() + half), R(it.set.begin() + half, it.set.end());
      for (int side = 0; side < 2; ++side) {
        const int id = (int)T.size();
        T.emplace_back();
        T[id].parent = it.node;
        T[id].depth = T[it.node].depth + 1;
        T[it.node].kids.push_back(id);
        stack.push_back({id, side == 0 ? std::move(L) : std::move(R)});
      }
    }
  }
  // 2. every group at the lowest common ancestor of its grains
  auto lca = [&](int a, int b) {
    while (T[a].depth > T[b].depth) a = T[a].parent;
    while (T[b].depth > T[a].depth) b = T[b].parent;
    while (a != b) {
      a = T[a].parent;
      b = T[b].parent;
    }
    return a;
  };
  std::vector<int> gnode(NG, -1);
  for (int g = 0; g < G; ++g)
    grain_groups(g, [&](int q) { gnode[q] = gnode[q] < 0 ? leaf[g] : lca(gnode[q], leaf[g]); });
  for (int q = 0; q < NG; ++q) {
    if (gnode[q] < 0) gnode[q] = 0;  // coupled to no grain: its rows of A^o are zero, the root reports it
    T[gnode[q]].groups.push_back(q);
  }
  // 3. merge small nodes into their parents (children have larger ids than their parents)
  auto ncols = [&](const TNode &n) {
    long long k = 0;
    for (int q : n.groups) k += grp_count[q];
    return k;
  };
  for (int v = (int)T.size() - 1; v >= 1; --v) {
    if (ncols(T[v]) >= CF_AMIN) continue;
    const int u = T[v].parent;
    T[v].kept = false;
    std::vector<int> g2 = T[v].groups;
    g2.insert(g2.end(), T[u].groups.begin(), T[u].groups.end());
    T[u].groups.swap(g2);
    T[u].grains.insert(T[u].grains.end(), T[v].grains.begin(), T[v].grains.end());
    auto &uk = T[u].kids;
    uk.erase(std::find(uk.begin(), uk.end(), v));
    for (int k : T[v].kids) {
      T[k].parent = u;
      uk.push_back(k);
    }
  }
  // 4. post-order of the kept tree = front order; elimination ranks; heights
  std::vector<int> order;
  {
    std::vector<std::pair<int, int>> st{{0, 0}};
    while (!st.empty()) {
      auto &top = st.back();
      if (top.second < (int)T[top.first].kids.size()) {
        const int k = T[top.first].kids[top.second++];
        st.push_back({k, 0});
      } else {
        order.push_back(top.first);
        st.pop_back();
      }
    }
  }
  const int nf = (int)order.size();
  std::vector<int> front_of(T.size(), -1);
  for (int f = 0; f < nf; ++f) front_of[order[f]] = f;
  std::vector<int> h_erank(std::max<long long>(No, 1), -1), h_owner(std::max<long long>(No, 1), 0),
      h_fpos(std::max<long long>(No, 1), 0);
  std::vector<int> grp_front(NG, 0);
  F.h_p.assign(nf, 0);
  {
    int r = 0;
    for (int f = 0; f < nf; ++f) {
      int pos = 0;
      for (int q : T[order[f]].groups) {
        grp_front[q] = f;
        for (int j = 0; j < grp_count[q]; ++j) {
          const int col = grp_first[q] + j;
          h_erank[col] = r++;
          h_owner[col] = f;
          h_fpos[col] = pos++;
        }
      }
      F.h_p[f] = pos;
    }
  }
  F.nf = nf;
  F.h_parent.assign(nf, -1);
  F.h_level.assign(nf, 0);
  for (int f = 0; f < nf; ++f) {
    const int v = order[f];
    if (T[v].parent >= 0) F.h_parent[f] = front_of[T[v].parent];
    for (int k : T[v].kids) F.h_level[f] = std::max(F.h_level[f], F.h_level[front_of[k]] + 1);
  }
  F.nlev = 0;
  for (int f = 0; f < nf; ++f) F.nlev = std::max(F.nlev, F.h_level[f] + 1);
  // 5. boundary groups, bottom-up: groups of the front's own grains and its children's boundaries, less
  // its pivots
  std::vector<std::vector<int>> bnd(nf);
  {
    std::vector<int> stamp(NG, -1);
    for (int f = 0; f < nf; ++f) {
      const int v = order[f];
      std::vector<int> &B = bnd[f];
      auto take = [&](int q) {
        if (stamp[q] == f || grp_front[q] == f) return;
        stamp[q] = f;
        B.push_back(q);
      };
      for (int g : T[v].grains) grain_groups(g, take);
      for (int k : T[v].kids)
        for (int q : bnd[front_of[k]]) take(q);
      std::sort(B.begin(), B.end(), [&](int a, int b) { return grp_front[a] < grp_front[b] ||
                                                               (grp_front[a] == grp_front[b] &&
                                                                h_erank[grp_first[a]] < h_erank[grp_first[b]]); });
      for (int q : B)
        HP_REQUIRE(grp_front[q] > f, HPLMM_ERR_INVALID, "coarse factor: boundary column not owned by an ancestor");
    }
  }
  // 6. front layout, row lists, extend-add maps
  F.h_b.assign(nf, 0);
  F.h_P.assign(nf, 0);
  F.h_m.assign(nf, 0);
  F.h_foff.assign(nf + 1, 0);
  F.h_yoff.assign(nf + 1, 0);
  F.h_doff.assign(nf + 1, 0);
  F.h_ioff.assign(nf + 1, 0);
  std::vector<int> h_idx, h_rank;
  std::vector<long long> h_roff(nf + 1, 0);
  std::vector<int> h_rel;
  F.flops = 0;
  F.solve_bytes = 0;
  for (int f = 0; f < nf; ++f) {
    const int p = F.h_p[f];
    int b = 0;
    for (int q : bnd[f]) b += grp_count[q];
    const int P = (int)rup(p, CT);
    const long long m = (long long)P + b;
    F.h_b[f] = b;
    F.h_P[f] = P;
    F.h_m[f] = (int)m;
    F.h_foff[f + 1] = F.h_foff[f] + m * m;
    F.h_yoff[f + 1] = F.h_yoff[f] + (long long)P * P;
    F.h_doff[f + 1] = F.h_doff[f] + (long long)(P / CT) * CT * CT;
    F.h_ioff[f + 1] = F.h_ioff[f] + m;
    for (int q : T[order[f]].groups)
      for (int j = 0; j < grp_count[q]; ++j) {
        h_idx.push_back(grp_first[q] + j);
        h_rank.push_back(h_erank[grp_first[q] + j]);
      }
    for (int j = p; j < P; ++j) {
      h_idx.push_back(-1);
      h_rank.push_back(-1);
    }
    for (int q : bnd[f])
      for (int j = 0; j < grp_count[q]; ++j) {
        h_idx.push_back(grp_first[q] + j);
        h_rank.push_back(h_erank[grp_first[q] + j]);
      }
    F.flops += (double)p * p * p / 3.0 + (double)p * p * b + (double)p * b * b;
    F.solve_bytes += 8LL * 2 * ((long long)p * (p + 1) / 2 + (long long)p * b);
  }
  for (int f = 0; f < nf; ++f) {
    const int u = F.h_parent[f];
    if (u >= 0) {
      const int *rk = h_rank.data() + F.h_ioff[u];
      for (long long i = F.h_ioff[f] + F.h_P[f]; i < F.h_ioff[f + 1]; ++i) {
        const int col = h_idx[i];
        int row;
        if (h_owner[col] == u) {
          row = h_fpos[col];
        } else {
          const int *a = std::lower_bound(rk + F.h_P[u], rk + F.h_m[u], h_rank[i]);
          HP_REQUIRE(a < rk + F.h_m[u] && *a == h_rank[i], HPLMM_ERR_INVALID,
                     "coarse factor: a boundary column is missing from the parent front");
          row = (int)(a - rk);
        }
        h_rel.push_back(row);
      }
    } else {
      HP_REQUIRE(F.h_b[f] == 0, HPLMM_ERR_INVALID, "coarse factor: the root front has boundary columns");
    }
    h_roff[f + 1] = (long long)h_rel.size();
  }
  F.F_total = F.h_foff[nf];
  F.Y_total = F.h_yoff[nf];
  F.D_total = F.h_doff[nf];
  F.idx_total = F.h_ioff[nf];
  if (h_idx.empty()) {
    h_idx.push_back(-1);
    h_rank.push_back(-1);
  }
  if (h_rel.empty()) h_rel.push_back(0);
  F.m.upload(F.h_m, s);
  F.P.upload(F.h_P, s);
  F.p.upload(F.h_p, s);
  F.b.upload(F.h_b, s);
  F.parent.upload(F.h_parent, s);
  F.foff.upload(F.h_foff, s);
  F.yoff.upload(F.h_yoff, s);
  F.doff.upload(F.h_doff, s);
  F.ioff.upload(F.h_ioff, s);
  F.roff.upload(h_roff, s);
  F.idx.upload(h_idx, s);
  F.rank.upload(h_rank, s);
  F.rel.upload(h_rel, s);
  F.erank.upload(h_erank, s);
  F.owner.upload(h_owner, s);
  F.fpos.upload(h_fpos, s);
  F.F.alloc(std::max<long long>(F.F_total, 1));
  F.F.zero(s);
  F.Y.alloc(std::max<long long>(F.Y_total, 1));
  F.D.alloc(std::max<long long>(F.D_total, 1));

  // 7. launch schedules.  Factorisation, per level (all fronts of one height), per tile step kt:
  // diagonal tile, panel tiles below it, Schur update of the trailing tiles, inverse steps; then the
  // extend-add of the level's update blocks into their parents.
  std::vector<FTask> tk;
  std::vector<int> ot;  // tensor-core Schur update tasks, six ints each
  F.fact.clear();
  F.oz_slots = 0;
  auto push = [&](std::vector<FLaunch> &L, int kind, int kt, long long off) {
    const int cnt = (int)((long long)tk.size() - off);
    if (cnt > 0) L.push_back({kind, kt, off, cnt});
  };
  std::vector<std::vector<int>> lev(F.nlev);
  for (int f = 0; f < nf; ++f) lev[F.h_level[f]].push_back(f);
  for (int h = 0; h < F.nlev; ++h) {
    int ktmax = 0;
    for (int f : lev[h]) ktmax = std::max(ktmax, F.h_P[f] / CT);
    for (int kt = 0; kt < ktmax; ++kt) {
      long long o = (long long)tk.size();
      for (int f : lev[h])
        if (F.h_P[f] / CT > kt) tk.push_back({f, kt, 0, 0});
      push(F.fact, K_POTRF, kt, o);
      o = (long long)tk.size();
      for (int f : lev[h]) {
        if (F.h_P[f] / CT <= kt) continue;
        const int Tf = (int)((F.h_m[f] + CT - 1) / CT);
        for (int it = kt + 1; it < Tf; ++it) tk.push_back({f, kt, it, 0});
      }
      const long long o_trsm = o;
      push(F.fact, K_TRSM, kt, o);
      if (c->opt.tensor_coarse) {
        // the Schur update on the tensor cores: digits of the panel tiles (one slot per TRSM task, in the same
        // order), then one task per (pair of row tiles it, it + 1; column tile jt)
        const int nslot = (int)((long long)tk.size() - o_trsm);
        if (nslot > 0) {
          F.fact.push_back({K_OZ_SLICE, kt, o_trsm, nslot});
          F.oz_slots = std::max<long long>(F.oz_slots, nslot);
          const long long ot0 = (long long)ot.size() / 6;
          int base = 0;
          for (int f : lev[h]) {
            if (F.h_P[f] / CT <= kt) continue;
            const int Tf = (int)((F.h_m[f] + CT - 1) / CT);
            for (int jt = kt + 1; jt < Tf; ++jt)
              for (int it = jt; it < Tf; it += 2) {
                const int tsk[6] = {f, kt, it, jt, base + it - kt - 1, base + jt - kt - 1};
                ot.insert(ot.end(), tsk, tsk + 6);
              }
            base += Tf - kt - 1;
          }
          const int cnt = (int)((long long)ot.size() / 6 - ot0);
          if (cnt > 0) F.fact.push_back({K_OZ_SYRK, kt, ot0, cnt});
        }
      } else {
        o = (long long)tk.size();
        for (int f : lev[h]) {
          if (F.h_P[f] / CT <= kt) continue;
          const int Tf = (int)((F.h_m[f] + CT - 1) / CT);
          for (int it = kt + 1; it < Tf; ++it)
            for (int jt = kt + 1; jt <= it; ++jt) tk.push_back({f, kt, it, jt});
        }
        push(F.fact, K_SYRK, kt, o);
      }
      o = (long long)tk.size();
      for (int f : lev[h]) {
        if (F.h_P[f] / CT <= kt) continue;
        for (int jt = 0; jt <= kt; ++jt) tk.push_back({f, kt, jt, 0});
      }
      push(F.fact, K_TRINV_SCALE, kt, o);
      o = (long long)tk.size();
      for (int f : lev[h]) {
        const int Tp = F.h_P[f] / CT;
        if (Tp <= kt) continue;
        for (int it = kt + 1; it < Tp; ++it)
          for (int jt = 0; jt <= kt; ++jt) tk.push_back({f, kt, it, jt});
      }
      push(F.fact, K_TRINV_UPDATE, kt, o);
    }
    long long o = (long long)tk.size();
    for (int f : lev[h]) {
      if (F.h_parent[f] < 0 || F.h_b[f] == 0) continue;
      const int Tb = (F.h_b[f] + CT - 1) / CT;
      for (int it = 0; it < Tb; ++it)
        for (int jt = 0; jt <= it; ++jt) tk.push_back({f, it, jt, 0});
    }
    push(F.fact, K_EXTEND, 0, o);
  }
  // Solve, per level: forward products (rows of inv(L_pp) in blocks of 32; rows of L_bp in blocks of 32),
  // backward products (column blocks of 256 x row chunks of 64 of L_bp, then of inv(L_pp))
  F.fwd.assign(F.nlev, {});
  F.bwd.assign(F.nlev, {});
  for (int h = 0; h < F.nlev; ++h) {
    long long o = (long long)tk.size();
    for (int f : lev[h])
      for (int r0 = 0; r0 < F.h_p[f]; r0 += 32) tk.push_back({f, r0, 0, 0});
    push(F.fwd[h], K_FWD_Y, 0, o);
    o = (long long)tk.size();
    for (int f : lev[h])
      for (int r0 = 0; r0 < F.h_b[f]; r0 += 32) tk.push_back({f, r0, 0, 0});
    push(F.fwd[h], K_FWD_B, 0, o);
    o = (long long)tk.size();
    for (int f : lev[h])
      for (int c0 = 0; c0 < F.h_p[f]; c0 += 256)
        for (int r0 = 0; r0 < F.h_b[f]; r0 += 64) tk.push_back({f, c0, r0, 0});
    push(F.bwd[h], K_BWD_B, 0, o);
    o = (long long)tk.size();
    for (int f : lev[h])
      for (int c0 = 0; c0 < F.h_p[f]; c0 += 256)
        for (int r0 = (c0 / 64) * 64; r0 < F.h_p[f]; r0 += 64) tk.push_back({f, c0, r0, 0});
    push(F.bwd[h], K_BWD_Y, 0, o);
  }
  if (tk.empty()) tk.push_back({0, 0, 0, 0});
  F.tasks.upload(tk, s);
  if (ot.empty()) ot.assign(6, 0);
  F.otask.upload(ot, s);
  if (F.oz_slots > 0) {
    F.oz_S.alloc((size_t)F.oz_slots * 7 * CT * CT);
    F.oz_E.alloc((size_t)F.oz_slots * CT);
  } else {
    F.oz_S.release();
    F.oz_E.release();
  }
  HP_CUDA(cudaStreamSynchronize(s));
}

}  // namespace hp

namespace hp {

void cf_factor(hplmm_ctx *c) {
  cudaStream_t s = c->stream;
  CoarseFactor &F = c->cf;
  if (F.nf == 0 || c->n_coarse == 0) return;
  const int nf = F.nf;
  const FTask *tk = F.tasks.p;
  k_cf_symmetrize<<<dim3(64, nf), 256, 0, s>>>(F.P.p, F.m.p, F.foff.p, nf, F.F.p);
  HP_CHECK_LAUNCH();
  k_cf_pad<<<nf, 64, 0, s>>>(F.p.p, F.P.p, F.m.p, F.foff.p, nf, F.F.p);
  HP_CHECK_LAUNCH();
  k_cf_eye<<<dim3(64, nf), 256, 0, s>>>(F.P.p, F.yoff.p, nf, F.Y.p);
  HP_CHECK_LAUNCH();
  for (const FLaunch &L : F.fact) {
    const FTask *t = tk + L.off;
    switch (L.kind) {
      case K_POTRF:
        k_cf_potrf<<<L.count, PT_THREADS, 0, s>>>(t, F.foff.p, F.m.p, F.doff.p, F.F.p, F.D.p, c->status.p);
        break;
      case K_TRSM:
        k_cf_trsm<<<dim3(L.count, 4), 256, 0, s>>>(t, F.foff.p, F.m.p, F.doff.p, F.F.p, F.D.p);
        break;
      case K_SYRK:
        k_cf_syrk<<<L.count, 256, 0, s>>>(t, F.foff.p, F.m.p, F.F.p);
        break;
      case K_TRINV_SCALE:
        k_cf_trinv_scale<<<L.count, 256, 0, s>>>(t, F.P.p, F.yoff.p, F.doff.p, F.Y.p, F.D.p);
        break;
      case K_TRINV_UPDATE:
        k_cf_trinv_update<<<L.count, 256, 0, s>>>(t, F.m.p, F.P.p, F.foff.p, F.yoff.p, F.F.p, F.Y.p);
        break;
      case K_EXTEND:
        k_cf_extend<<<L.count, 256, 0, s>>>(t, F.m.p, F.P.p, F.bdev(), F.parent.p,
                                            F.foff.p, F.roff.p, F.rel.p, F.F.p);
        break;
      case K_OZ_SLICE:
        k_cf_oz_slice<<<L.count, 256, 0, s>>>(t, F.foff.p, F.m.p, F.F.p, F.oz_S.p, F.oz_E.p);
        break;
      case K_OZ_SYRK:
        HP_CUDA(cudaFuncSetAttribute(k_cf_oz_syrk, cudaFuncAttributeMaxDynamicSharedMemorySize, oz::SMEM));
        k_cf_oz_syrk<<<L.count, OZ_THREADS, oz::SMEM, s>>>(F.otask.p + 6 * L.off, F.foff.p, F.m.p, F.F.p, F.oz_S.p,
                                                     F.oz_E.p, c->status.p);
        break;
      default:
        throw Error(HPLMM_ERR_INVALID, "coarse factor: bad launch kind");
    }
    HP_CHECK_LAUNCH();
  }
}

void cf_solve(hplmm_ctx *c, double *t, double *y, double *x) {
  cudaStream_t s = c->stream;
  CoarseFactor &F = c->cf;
  HP_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * (size_t)c->n_coarse, s));
  if (F.nf == 0) return;
  const FTask *tk = F.tasks.p;
  for (int h = 0; h < F.nlev; ++h)
    for (const FLaunch &L : F.fwd[h]) {
      const FTask *tt = tk + L.off;
      if (L.kind == K_FWD_Y)
        k_cf_fwd_y<<<L.count, 256, 0, s>>>(tt, F.p.p, F.P.p, F.yoff.p, F.ioff.p, F.idx.p, F.Y.p, t, y);
      else
        k_cf_fwd_b<<<L.count, 256, 0, s>>>(tt, F.p.p, F.P.p, F.bdev(), F.m.p, F.foff.p, F.ioff.p, F.idx.p, F.F.p, y,
                                           t);
      HP_CHECK_LAUNCH();
    }
  for (int h = F.nlev - 1; h >= 0; --h)
    for (const FLaunch &L : F.bwd[h]) {
      const FTask *tt = tk + L.off;
      if (L.kind == K_BWD_B)
        k_cf_bwd_b<<<L.count, 256, 0, s>>>(tt, F.p.p, F.P.p, F.bdev(), F.m.p, F.foff.p, F.ioff.p, F.idx.p, F.F.p, x,
                                           y);
      else
        k_cf_bwd_y<<<L.count, 256, 0, s>>>(tt, F.p.p, F.P.p, F.yoff.p, F.ioff.p, F.idx.p, F.Y.p, y, x);
      HP_CHECK_LAUNCH();
    }
}

}  // namespace hp
