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

// Pieces of each line: kPieces threads per (column, array) each run both
// recursions over one piece of the line, from their own exact start sums.
constexpr int kPieces = 2;

// Start value of a recursion at position pos: the causal value
// c_m = zscale sum_{k < nterm} z^k f_{(m - k) mod n}, or the anticausal
// d_m = zscale sum_{k < nterm} z^k c_{(m + k) mod n}.  With nterm = n these
// are the exact periodic sums (zscale = 1 / (1 - z^n)); with nterm = 32 < n
// the sum stops at 26 terms (the tail is below |z|^26 / (1 - |z|) ~ 1e-15 of
// the scale, under the pairs' own rounding).  Pairs for the terms above
// 2^-26 (k < 14), FP32 for the rest (below 2^-50 of the sum's scale).
template <bool CAUSAL>
__device__ __forceinline__ float2 start_sum(const float2 *col, int stride, int n, int pos, const AdvDFArgs &a) {
  float sh = 0.f, se = 0.f, tail = 0.f;
  const int nt = a.nterm == n ? n : (a.nterm < 26 ? a.nterm : 26);
  const int kdf = nt < 14 ? nt : 14;
  for (int k = 0; k < nt; ++k) {
    const float2 zk = a.zpow[k];
    int idx = CAUSAL ? pos - k : pos + k;
    idx += CAUSAL ? (idx < 0 ? n : 0) : (idx >= n ? -n : 0);
    const float2 v = col[idx * stride];
    if (k < kdf) {
      float ph, pe;
      df_mul(zk.x, zk.y, v.x, v.y, ph, pe);
      df_acc(sh, se, ph, pe);
    } else {
      tail = __fmaf_rn(zk.x, v.x, tail);
    }
  }
  const float2 sv = df_norm(sh, __fadd_rn(se, tail));
  float ph, pe;
  df_mul(a.zscale.x, a.zscale.y, sv.x, sv.y, ph, pe);
  return df_norm(ph, pe);
}

// One recursion step u = f + z v on pairs.
__device__ __forceinline__ float2 rec_step(float2 f, float2 v, float zh, float zl) {
  float ph, pe, s, t;
  df_mul(zh, zl, v.x, v.y, ph, pe);
  two_sum(f.x, ph, s, t);
  t = __fadd_rn(t, __fadd_rn(f.y, pe));
  return df_norm(s, t);
}

// In place on a strided column, by the kPieces threads of the column (this
// thread: rows [lo, lo + len)): c_i = f_i + z c_{i-1} (periodic), then
// d_i = c_i + z d_{i+1} (periodic); the -6 z factor is in the weights.  Every
// thread of the CTA calls this: it holds the CTA barriers between the phases.
__device__ __forceinline__ void coeffs_df(float2 *col, int stride, int n, int lo, int len, const AdvDFArgs &a) {
  const float zh = a.z.x, zl = a.z.y;
  const int hi = lo + len - 1;
  float2 cur = len > 0 ? start_sum<true>(col, stride, n, lo, a) : make_float2(0.f, 0.f);
  __syncthreads();  // every start sum has read the input line
  if (len > 0) col[lo * stride] = cur;
  for (int j = 1; j < len; ++j) {
    const int i = lo + j;
    cur = rec_step(col[i * stride], cur, zh, zl);
    col[i * stride] = cur;
  }
  __syncthreads();
  cur = len > 0 ? start_sum<false>(col, stride, n, hi, a) : make_float2(0.f, 0.f);
  __syncthreads();  // every start sum has read the causal pass
  if (len > 0) col[hi * stride] = cur;
  for (int j = 1; j < len; ++j) {
    const int i = hi - j;
    cur = rec_step(col[i * stride], cur, zh, zl);
    col[i * stride] = cur;
  }
  __syncthreads();
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
// TWO: shift in0 and in1, lane 2 n2 + r taking array r of column n2; DIR 1 with TWO writes
// out0 = a + tau b (lane r = 0) and out1 = a + tau/2 b (lane r = 1), the two lanes swapping
// their values by shuffle.  Without TWO: one thread per column and piece.  Thread
// q (A NK) + A n2 + r (A = 2 with TWO, else 1) takes piece q of the line: its rows for
// the staging, the recursions and the outputs.
template <int NK, int DIR, int TWO>
__global__ void __launch_bounds__(kPieces * (TWO ? 2 : 1) * NK) k_adv_df(AdvDFArgs a) {
  constexpr int IN_DF = (DIR == 1) == (TWO == 1);
  constexpr int S = NK + 1, AR = TWO ? 2 : 1;
  extern __shared__ float2 smf[];
  const int nx = a.nx;
  const int n1 = blockIdx.x, fixed = blockIdx.y;
  const int q = threadIdx.x / (AR * NK), lt = threadIdx.x - q * (AR * NK);
  const int t = lt / AR;  // column n2
  const int r = lt % AR;  // array
  const int lo = (q * nx) / kPieces, len = ((q + 1) * nx) / kPieces - lo;
  float2 *A = smf + (size_t)r * (nx * S + 8);  // second buffer skewed by 16 banks (lanes 2c, 2c+1 differ)
  const void *in = r ? a.in1 : a.in0;
  const size_t lineStride = (DIR == 0) ? (size_t)NK * NK : (size_t)nx * NK * NK;
  const size_t base = (DIR == 0) ? ((size_t)fixed * nx * NK + n1) * NK : ((size_t)fixed * NK + n1) * NK;
  // stage this thread's rows of its column; FP64 inputs are split into pairs in place
  for (int i = lo; i < lo + len; ++i)
    cp_async8(A + i * S + t, reinterpret_cast<const double *>(in) + base + i * lineStride + t);
  cp_async_wait_all();
  if (!IN_DF)
    for (int i = lo; i < lo + len; ++i) A[i * S + t] = df_split(*reinterpret_cast<const double *>(A + i * S + t));
  __syncthreads();  // the start sums read other pieces' rows
  const int sidx = (DIR == 0) ? t : n1;
  const int k0 = a.k0tab[sidx];
  const float2 w[4] = {a.wdf[4 * sidx], a.wdf[4 * sidx + 1], a.wdf[4 * sidx + 2], a.wdf[4 * sidx + 3]};
  coeffs_df(A + t, S, nx, lo, len, a);
  // outputs x_i, i in [lo, lo + len): taps p = i + k0 - 1 + (0..3) (mod nx),
  // a sliding window of four coefficients
  int p = (lo + k0 - 1) % nx;
  p += (p < 0) ? nx : 0;
  float2 d[4];
#pragma unroll
  for (int u = 0; u < 3; ++u) {
    int pu = p + u;
    pu -= (pu >= nx) ? nx : 0;
    d[u] = A[pu * S + t];
  }
  void *out = r ? a.out1 : a.out0;
  const float2 coef = r ? a.half_tau : a.tau;
#pragma unroll 4
  for (int i = lo; i < lo + len; ++i) {
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
    for (int u = 0; u < 3; ++u) d[u] = d[u + 1];
    p = (p + 1 == nx) ? 0 : p + 1;
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
  dim3 grid(NK, a.nx), block(kPieces * (two ? 2 : 1) * NK);
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
