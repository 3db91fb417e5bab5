// Device pieces shared by the two sliced FP64 sweeps (k_theta_s on mma.sync,
// w2_f64s.cu; k_theta_t on tcgen05, w2_f64t.cu): the six-digit fixed-point
// split of FP64 values, BF16 bits of a digit, the exact per-X sum of values a
// CTA holds in registers, and the mirror block of the exchange-symmetric
// sweep.
#pragma once
#include <stdint.h>

#include "w2_blocks.cuh"
#include "w2_df.cuh"
#include "w2_internal.cuh"

namespace w2 {
namespace slice {

constexpr int kDig = 6;  // digits per operand

__device__ __forceinline__ int expo(double v) {
  return (int)(((unsigned long long)__double_as_longlong(v) >> 52) & 0x7ff);
}

// Six balanced base-256 digits of |v| 2^(48 - E), 2^E = 2^(emax - 1022) the
// block bound (emax the largest biased exponent of the block, >= 1), with v's sign:
//     round(|v| 2^(48 - E)) = sum_{s=0..5} |d_s| 256^(5-s),  d_0 in [0, 256],  d_1..d_5 in [-128, 127].
// The 48-bit integer is cut as two 24-bit halves in 32-bit arithmetic: the
// low half gives d_5..d_3 and a carry of 0 or 1 into the high half, which
// gives d_2, d_1 and d_0.
__device__ __forceinline__ void digits6(double v, int emax, int (&d)[kDig]) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const int e = (int)((b >> 52) & 0x7ff);
  const unsigned long long m = (b & 0xfffffffffffffull) | (e ? (1ull << 52) : 0ull);
  const int sh = emax - (e ? e : 1) + 5;  // >= 5
  const unsigned long long n = sh < 64 ? (m + (1ull << (sh - 1))) >> sh : 0ull;  // <= 2^48
  int lo = (int)(n & 0xffffffull), hi = (int)(n >> 24);
#pragma unroll
  for (int s = kDig - 1; s >= 3; --s) {
    const int l = lo & 255, ds = l - ((l & 128) << 1);
    d[s] = ds;
    lo = (lo - ds) >> 8;
  }
  hi += lo;
#pragma unroll
  for (int s = 2; s >= 1; --s) {
    const int l = hi & 255, ds = l - ((l & 128) << 1);
    d[s] = ds;
    hi = (hi - ds) >> 8;
  }
  d[0] = hi;
  const int sg = -(int)(b >> 63);  // 0 or -1: the sign of v on every digit
#pragma unroll
  for (int s = 0; s < kDig; ++s) d[s] = (d[s] ^ sg) - sg;
}

// BF16 bits of a small integer (|d| <= 256): exact through the FP32 magic-number sum.
__device__ __forceinline__ uint32_t bf16_int(int d) {
  return __float_as_uint(__int_as_float(0x4B400000 + d) - 12582912.0f) >> 16;
}

// Exact sum (the rule and bits of xsum_block) of the PER values each thread
// of the CTA holds, em the thread's largest biased exponent among them.
// Every thread calls this; red: 32 ints followed by 32 long longs of shared
// memory.  Thread 0 writes *out.
template <int PER>
__device__ __forceinline__ void held_exact_sum(const double (&v)[PER], int em, double *out, int *red) {
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, nw = blockDim.x >> 5;
  long long *lred = reinterpret_cast<long long *>(red + 32);
  em = __reduce_max_sync(0xffffffffu, em);
  if (lane == 0) red[w] = em;
  __syncthreads();
  em = 0;
  for (int q = 0; q < nw; ++q) em = max(em, red[q]);
  em = max(em, 1);
  long long acc = 0;
#pragma unroll
  for (int i = 0; i < PER; ++i) acc += fixed_image(v[i], em);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) lred[w] = acc;
  __syncthreads();
  if (tid == 0) {
    long long tot = 0;
    for (int q = 0; q < nw; ++q) tot += lred[q];
    *out = em == 2047 ? __longlong_as_double(0x7ff8000000000000ll) : ll_to_double_scaled(tot, em - 1071);
  }
  __syncthreads();
}

// The mirror block X' = (i2, i1) of an exchange-symmetric input: Theta at X'
// is the transpose of Theta at X (the one-body kernels of the two particles
// coincide and the pair kernel is odd in x1 - x2), so
//   MODE 0: out(X')[r][c] = C[c][r],   MODE 1: out(X')[r][c] = h(X')[r][c] + half_tau C[c][r],
// with C = Theta at X staged in shared memory at row stride NK + 1, and in the
// corrector (with xsum given) the exact per-X sum of out(X').  Every thread of
// the CTA (THREADS of them) calls this; red as for held_exact_sum.
template <int NK, int THREADS, int MODE>
__device__ __forceinline__ void mirror_block(const ThetaArgs &a, const double *C, int Xm, int *red) {
  constexpr int PER = NK * NK / THREADS;
  const int tid = threadIdx.x;
  const size_t mbase = (size_t)Xm * NK * NK;
  double v[PER];
  int em = 0;
  if (MODE == 1) {  // every load of h before the first store (the stores may alias it)
#pragma unroll
    for (int i = 0; i < PER; ++i) v[i] = a.h[mbase + tid + i * THREADS];
  }
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int e = tid + i * THREADS, r = e / NK, c = e - r * NK;
    const double t = C[c * (NK + 1) + r];
    v[i] = MODE == 0 ? t : fma(a.half_tau, t, v[i]);
    a.out[mbase + e] = v[i];
    em = max(em, expo(v[i]));
  }
  if (MODE == 1 && a.xsum) held_exact_sum<PER>(v, em, a.xsum + Xm, red);
}

}  // namespace slice
}  // namespace w2
