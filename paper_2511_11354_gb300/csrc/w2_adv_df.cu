// Characteristic shift of the sliced FP64 path (W2_F64_SLICED): the periodic
// cubic B-spline shift of k_adv in w2_f64.cu (Sec. 4.1, the A_per solve and
// the B_nu evaluation) in double-float arithmetic on the FP32 pipe, which
// runs about 76 times as many operations per clock as this GPU's FP64 pipe.
//
// Formats: the pass that reads a step's FP64 arrays (x2 lines in the step,
// x1 lines in w2_advect) splits them into double-float pairs and writes its
// outputs as pairs (one float2 per element, the same 8 bytes as a double);
// the following pass reads the pairs and writes FP64.  The conversions are
// integer bit operations (w2_df.cuh).  Per element the pair keeps about 47
// bits, so a step agrees with the FP64 shift to ~1e-14.
//
// Launch as k_adv: one CTA per (momentum row n1, fixed other coordinate), one
// thread per column n2, the slab [x][n2] of pairs in shared memory.
#include <math.h>
#include <stdint.h>

#include "w2_df.cuh"
#include "w2_internal.cuh"

namespace w2 {
namespace {

// 8-byte asynchronous copy global -> shared (all of a column's copies are in
// flight together; the thread waits for its own copies only).
__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// Normalised pair of (sh, se).
__device__ __forceinline__ float2 df_norm(float sh, float se) {
  float h, l;
  fast_two_sum(sh, se, h, l);
  return make_float2(h, l);
}

constexpr int kChunks = 2;  // independent pieces of each recursion (instruction-level parallelism)

// Start values of the recursions at positions pos[c]: the causal value
// c_m = zscale sum_{k < nterm} z^k f_{(m - k) mod n}, or the anticausal
// d_m = zscale sum_{k < nterm} z^k c_{(m + k) mod n}.  With nterm = n these
// are the exact periodic sums (zscale = 1 / (1 - z^n)); with nterm = 32 < n
// the sum stops at 26 terms (the tail is below |z|^26 / (1 - |z|) ~ 1e-15 of
// the scale, under the pairs' own rounding).  Pairs for the terms above
// 2^-26 (k < 14), FP32 for the rest (below 2^-50 of the sum's scale).
template <bool CAUSAL>
__device__ __forceinline__ void start_sums(const float2 *col, int stride, int n, const int (&pos)[kChunks],
                                           const AdvDFArgs &a, float2 (&out)[kChunks]) {
  float sh[kChunks], se[kChunks], tail[kChunks];
#pragma unroll
  for (int c = 0; c < kChunks; ++c) sh[c] = se[c] = tail[c] = 0.f;
  const int nt = a.nterm == n ? n : (a.nterm < 26 ? a.nterm : 26);
  const int kdf = nt < 14 ? nt : 14;
  for (int k = 0; k < nt; ++k) {
    const float2 zk = a.zpow[k];
#pragma unroll
    for (int c = 0; c < kChunks; ++c) {
      int idx = CAUSAL ? pos[c] - k : pos[c] + k;
      idx += CAUSAL ? (idx < 0 ? n : 0) : (idx >= n ? -n : 0);
      const float2 v = col[idx * stride];
      if (k < kdf) {
        float ph, pe;
        df_mul(zk.x, zk.y, v.x, v.y, ph, pe);
        df_acc(sh[c], se[c], ph, pe);
      } else {
        tail[c] = __fmaf_rn(zk.x, v.x, tail[c]);
      }
    }
  }
#pragma unroll
  for (int c = 0; c < kChunks; ++c) {
    const float2 sv = df_norm(sh[c], __fadd_rn(se[c], tail[c]));
    float ph, pe;
    df_mul(a.zscale.x, a.zscale.y, sv.x, sv.y, ph, pe);
    out[c] = df_norm(ph, pe);
  }
}

// One recursion step u = f + z v on pairs.
__device__ __forceinline__ float2 rec_step(float2 f, float2 v, float zh, float zl) {
  float ph, pe, s, t;
  df_mul(zh, zl, v.x, v.y, ph, pe);
  two_sum(f.x, ph, s, t);
  t = __fadd_rn(t, __fadd_rn(f.y, pe));
  return df_norm(s, t);
}

// In place on a strided column: c_i = f_i + z c_{i-1} (periodic), then
// d_i = c_i + z d_{i+1} (periodic); the -6 z factor is in the weights.  Each
// pass runs as kChunks interleaved recursions over consecutive pieces of the
// line, each started from its own exact start sum.
__device__ __forceinline__ void coeffs_df(float2 *col, int stride, int n, const AdvDFArgs &a) {
  const float zh = a.z.x, zl = a.z.y;
  int lo[kChunks], len[kChunks], hi[kChunks];
#pragma unroll
  for (int c = 0; c < kChunks; ++c) {
    lo[c] = (c * n) / kChunks;
    len[c] = ((c + 1) * n) / kChunks - lo[c];
    hi[c] = lo[c] + len[c] - 1;
  }
  const int lmax = (n + kChunks - 1) / kChunks;
  float2 cur[kChunks];
  start_sums<true>(col, stride, n, lo, a, cur);
#pragma unroll
  for (int c = 0; c < kChunks; ++c)
    if (len[c] > 0) col[lo[c] * stride] = cur[c];
  for (int j = 1; j < lmax; ++j) {
#pragma unroll
    for (int c = 0; c < kChunks; ++c) {
      if (j < len[c]) {
        const int i = lo[c] + j;
        cur[c] = rec_step(col[i * stride], cur[c], zh, zl);
        col[i * stride] = cur[c];
      }
    }
  }
  start_sums<false>(col, stride, n, hi, a, cur);
#pragma unroll
  for (int c = 0; c < kChunks; ++c)
    if (len[c] > 0) col[hi[c] * stride] = cur[c];
  for (int j = 1; j < lmax; ++j) {
#pragma unroll
    for (int c = 0; c < kChunks; ++c) {
      if (j < len[c]) {
        const int i = hi[c] - j;
        cur[c] = rec_step(col[i * stride], cur[c], zh, zl);
        col[i * stride] = cur[c];
      }
    }
  }
}

// Spline value sum_q w_q d_{p + q} from the window (d_p, d_{p+1}, d_{p+2}, d_{p+3}).
__device__ __forceinline__ float2 eval_win(const float2 (&d)[4], const float2 (&w)[4]) {
  float sh, se;
  df_mul(w[0].x, w[0].y, d[0].x, d[0].y, sh, se);
#pragma unroll
  for (int q = 1; q < 4; ++q) {
    float ph, pe;
    df_mul(w[q].x, w[q].y, d[q].x, d[q].y, ph, pe);
    df_acc(sh, se, ph, pe);
  }
  return df_norm(sh, se);
}

// u + c v for pairs u, v and a constant pair c, as FP64.
__device__ __forceinline__ double axpy_join(float2 u, float2 c, float2 v) {
  float ph, pe, s, t;
  df_mul(c.x, c.y, v.x, v.y, ph, pe);
  two_sum(u.x, ph, s, t);
  t = __fadd_rn(t, __fadd_rn(u.y, pe));
  const float2 r = df_norm(s, t);
  return df_join(r.x, r.y);
}

// DIR 0: lines along x2 at fixed (i1 = blockIdx.y, n1 = blockIdx.x), shift of column n2.
// DIR 1: lines along x1 at fixed (i2 = blockIdx.y, n1 = blockIdx.x), shift of row n1.
// Inputs are pairs when DIR == TWO (the second pass), FP64 otherwise; outputs the other way.
// TWO: shift in0 and in1, lane 2 n2 + r taking array r of column n2 (2 nk threads); DIR 1
// with TWO writes out0 = a + tau b (lane r = 0) and out1 = a + tau/2 b (lane r = 1), the
// two lanes swapping their values by shuffle.  Without TWO: one thread per column.
template <int NK, int DIR, int TWO>
__global__ void __launch_bounds__(TWO ? 2 * NK : NK) k_adv_df(AdvDFArgs a) {
  constexpr int IN_DF = (DIR == 1) == (TWO == 1);
  constexpr int S = NK + 1;
  extern __shared__ float2 smf[];
  const int nx = a.nx;
  const int n1 = blockIdx.x, fixed = blockIdx.y;
  const int t = TWO ? (int)(threadIdx.x >> 1) : (int)threadIdx.x;  // column n2
  const int r = TWO ? (int)(threadIdx.x & 1) : 0;                  // array
  float2 *A = smf + (size_t)r * (nx * S + 8);  // second buffer skewed by 16 banks (lanes 2c, 2c+1 differ)
  const void *in = r ? a.in1 : a.in0;
  const size_t lineStride = (DIR == 0) ? (size_t)NK * NK : (size_t)nx * NK * NK;
  const size_t base = (DIR == 0) ? ((size_t)fixed * nx * NK + n1) * NK : ((size_t)fixed * NK + n1) * NK;
  // stage this thread's column; FP64 inputs are split into pairs in place
  for (int i = 0; i < nx; ++i)
    cp_async8(A + i * S + t, reinterpret_cast<const double *>(in) + base + i * lineStride + t);
  cp_async_wait_all();
  if (!IN_DF)
    for (int i = 0; i < nx; ++i) A[i * S + t] = df_split(*reinterpret_cast<const double *>(A + i * S + t));
  const int sidx = (DIR == 0) ? t : n1;
  const int k0 = a.k0tab[sidx];
  const float2 w[4] = {a.wdf[4 * sidx], a.wdf[4 * sidx + 1], a.wdf[4 * sidx + 2], a.wdf[4 * sidx + 3]};
  coeffs_df(A + t, S, nx, a);
  // walk the coefficient index p of tap 0 (output x_i with i = p - jb mod nx)
  // with a sliding window of four coefficients
  int jb = (k0 - 1) % nx;
  jb += (jb < 0) ? nx : 0;
  int i = jb ? nx - jb : 0;
  float2 d[4];
#pragma unroll
  for (int q = 0; q < 3; ++q) d[q] = A[q * S + t];
  void *out = r ? a.out1 : a.out0;
  const float2 coef = r ? a.half_tau : a.tau;
#pragma unroll 4
  for (int p = 0; p < nx; ++p) {
    int p3 = p + 3;
    p3 -= (p3 >= nx) ? nx : 0;
    d[3] = A[p3 * S + t];
    const size_t o = base + i * lineStride + t;
    const float2 v = eval_win(d, w);
    if (!TWO && IN_DF) {
      reinterpret_cast<double *>(out)[o] = df_join(v.x, v.y);
    } else if (DIR == 0 || !TWO) {
      reinterpret_cast<float2 *>(out)[o] = v;
    } else {
      float2 u;  // the partner lane's value: b for lane 0, a for lane 1
      u.x = __shfl_xor_sync(0xffffffffu, v.x, 1);
      u.y = __shfl_xor_sync(0xffffffffu, v.y, 1);
      reinterpret_cast<double *>(out)[o] = r ? axpy_join(u, coef, v) : axpy_join(v, coef, u);
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) d[q] = d[q + 1];
    i = (i + 1 == nx) ? 0 : i + 1;
  }
}

template <int NK>
cudaError_t prep_adv_df() {
  cudaError_t e = cudaSuccess;
#define W2_ADVDF_ATTR(D, T2)                                                                   \
  e = cudaFuncSetAttribute(k_adv_df<NK, D, T2>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                           200 * 1024);                                                        \
  if (e != cudaSuccess) return e;
  W2_ADVDF_ATTR(0, 0) W2_ADVDF_ATTR(0, 1) W2_ADVDF_ATTR(1, 0) W2_ADVDF_ATTR(1, 1)
#undef W2_ADVDF_ATTR
  return e;
}

template <int NK>
cudaError_t run_adv_df(int dir, int two, const AdvDFArgs &a, cudaStream_t s) {
  dim3 grid(NK, a.nx), block(two ? 2 * NK : NK);
  const size_t smem = sizeof(float2) * ((size_t)(two ? 2 : 1) * a.nx * (NK + 1) + 8);
  if (dir == 0 && !two) k_adv_df<NK, 0, 0><<<grid, block, smem, s>>>(a);
  if (dir == 0 && two) k_adv_df<NK, 0, 1><<<grid, block, smem, s>>>(a);
  if (dir == 1 && !two) k_adv_df<NK, 1, 0><<<grid, block, smem, s>>>(a);
  if (dir == 1 && two) k_adv_df<NK, 1, 1><<<grid, block, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t prepare_kernels_adv_df(int nk) {
  switch (nk) {
    case 16: return prep_adv_df<16>();
    case 32: return prep_adv_df<32>();
    case 48: return prep_adv_df<48>();
    case 64: return prep_adv_df<64>();
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_adv_df(int nk, int dir, int two, const AdvDFArgs &a, cudaStream_t s) {
  if (a.nterm < 1 || a.nterm > 32) return cudaErrorInvalidValue;
  switch (nk) {
    case 16: return run_adv_df<16>(dir, two, a, s);
    case 32: return run_adv_df<32>(dir, two, a, s);
    case 48: return run_adv_df<48>(dir, two, a, s);
    case 64: return run_adv_df<64>(dir, two, a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace w2
