// Device bodies shared by the single-problem kernels and the batched
// persistent step: the kernel tables (densities -> potentials on the fine
// points -> shift kernels) and the exact per-X momentum sums.  Each
// translation unit that launches them includes this header; the bodies are
// compiled the same way everywhere, so every caller gets the same bits.
#pragma once
#include <math.h>

#include "w2_df.cuh"
#include "w2_internal.cuh"

namespace w2 {

__device__ __forceinline__ double phi_xc(int kind, double n) {
  if (kind == 1) return n;
  if (kind == 2) {  // Hedin-Lundqvist form, defined for n >= 0
    double c = cbrt(fmax(n, 0.0));
    return 0.985 * c + 0.985 * 0.034 * log1p(18.37 * c);
  }
  return 0.0;
}

// grid: (nx, 2) for one-body kernels (blockIdx.y = particle), (nx, 1) for the
// pair kernel.  Dynamic shared memory: (nx + M) doubles; 512 threads.
// compiled once (not inlined) so the single-problem and batched kernels
// run the same machine code and give identical bits
static __device__ __noinline__ void tables_block(const TabArgs &a, const int i, const int part, double *sm) {
  const int nx = a.nx, nk = a.nk, M = a.M;
  double *n = sm, *U = sm + nx;
  const int quads = blockDim.x >> 2, qd = threadIdx.x >> 2;
  const bool lead = (threadIdx.x & 3) == 0;
  const bool mf = !a.pair_mode && a.xsum && (a.c_h != 0.0 || (a.c_xc != 0.0 && a.xc_kind));
  // one quad per item; the item loops run the same number of rounds in every
  // thread (the quads' shuffles need all lanes)
  if (mf) {
    const double w = a.dx * a.dp * a.dp;
    for (int b = 0; b < nx; b += quads) {
      const int q = b + qd;
      const double s = quad_sum(q < nx, nx, [&](int k) {
        return part == 0 ? a.xsum[(size_t)q * nx + k] : a.xsum[(size_t)k * nx + q];
      });
      if (lead && q < nx) n[q] = s * w;
    }
  }
  __syncthreads();
  for (int b = 0; b < M; b += quads) {
    const int l = b + qd;
    const bool v = l < M;
    double u = 0.0;
    if (a.pair_mode) {
      if (v) u = a.gamma * a.w_fine[(size_t)i * M + l];
    } else {
      if (v) u = a.vext_fine[(size_t)i * M + l];
      if (mf && a.c_h != 0.0) {
        const double *ker = a.h_fine ? a.h_fine : a.w_fine;  // Poisson kernel, or W scaled below
        const double vh = quad_sum(v, nx, [&](int q) {
          int d = i - q;
          d += (d < 0) ? nx : 0;
          return ker[(size_t)d * M + l] * n[q];
        });
        u += a.c_h * (a.h_fine ? 1.0 : a.gamma * a.dx) * vh;
      }
      if (mf && a.c_xc != 0.0 && a.xc_kind) {
        const double ni = quad_sum(v, nx, [&](int q) {
          int d = i - q;
          d += (d < 0) ? nx : 0;
          return a.d_fine[(size_t)d * M + l] * n[q];
        });
        u += a.c_xc * phi_xc(a.xc_kind, ni);
      }
    }
    if (lead && v) U[l] = u;
  }
  __syncthreads();
  const int W = 2 * nk - 1;
  double *K = a.K + ((size_t)part * nx + i) * W;
  const double inv = 1.0 / (a.hbar * nk);
  for (int b = 0; b < nk; b += quads) {
    const int j = b + qd;
    double s = quad_sum(j < nk, nk - 1, [&](int k) {
      const int l = k + 1;
      return (U[l] - U[M - l]) * a.sintab[(l * j) % M];
    });
    if (lead && j < nk) {
      s *= inv;
      K[nk - 1 + j] = s;
      K[nk - 1 - j] = -s;
    }
  }
}

// Fixed-point image of v: round(|v| 2^(49 - E)) (FP64) or |v| 2^(48 - E)
// (FP32), with sign, where 2^E bounds the block (emax its largest biased
// exponent); the unit is 2^(emax - 1071) for FP64 and 2^(emax - 174) for FP32,
// so that up to 4096 (FP64) or 16384 (FP32) images add up below 2^62.
// Integer operations only.
__device__ __forceinline__ long long fixed_image(double v, int emax) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const int e = (int)((b >> 52) & 0x7ff);
  const unsigned long long m = (b & 0xfffffffffffffull) | (e ? (1ull << 52) : 0ull);
  const int sh = emax - (e ? e : 1) + 4;  // >= 4
  const long long q = sh < 64 ? (long long)((m + (1ull << (sh - 1))) >> sh) : 0;
  return (b >> 63) ? -q : q;
}

__device__ __forceinline__ long long fixed_image(float v, int emax) {
  const unsigned b = __float_as_uint(v);
  const int e = (int)((b >> 23) & 0xff);
  const unsigned long long m = (unsigned long long)((b & 0x7fffffu) | (e ? 0x800000u : 0u)) << 24;
  const int sh = emax - (e ? e : 1);  // >= 0
  const long long q = sh == 0 ? (long long)m : sh < 64 ? (long long)((m + (1ull << (sh - 1))) >> sh) : 0;
  return (b >> 31) ? -q : q;
}

__device__ __forceinline__ int expo_of(double v) {
  return (int)(((unsigned long long)__double_as_longlong(v) >> 52) & 0x7ff);
}
__device__ __forceinline__ int expo_of(float v) { return (int)((__float_as_uint(v) >> 23) & 0xff); }

// Block maximum exponent and exact fixed-point sum of the n values at base,
// with up to K values per thread held in registers between the two steps
// (the rest, if any, read a second time).
template <typename T, int K>
__device__ __forceinline__ void xsum_hold(const T *f, size_t base, int n, int &em_out, long long &acc_out, int *ired) {
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, nw = blockDim.x >> 5;
  T v[K];
  int em = 0;
#pragma unroll
  for (int i = 0; i < K; ++i) {
    const int e = tid + i * (int)blockDim.x;
    v[i] = e < n ? f[base + e] : (T)0;
    em = max(em, expo_of(v[i]));
  }
  for (int e = tid + K * (int)blockDim.x; e < n; e += blockDim.x) em = max(em, expo_of(f[base + e]));
  em = __reduce_max_sync(0xffffffffu, em);
  if (lane == 0) ired[w] = em;
  __syncthreads();
  em = 0;
  for (int q = 0; q < nw; ++q) em = max(em, ired[q]);
  em = max(em, 1);
  long long acc = 0;
#pragma unroll
  for (int i = 0; i < K; ++i) acc += fixed_image(v[i], em);
  for (int e = tid + K * (int)blockDim.x; e < n; e += blockDim.x) acc += fixed_image(f[base + e], em);
  em_out = em;
  acc_out = acc;
}

// xsum[X] = sum_P f(X, P), one block per X, as an exact sum of fixed-point
// images (each rounded to 2^-49 / 2^-48 of the block bound, then added
// without rounding): the result does not depend on the order of the
// additions, and neither the FP64 pipe nor a floating-point reduction tree is
// involved.  A block holding Inf or NaN gives NaN.  red: 256 doubles of
// shared memory (used as 32 ints and 32 int64).
// (The sum is exact, so every kernel that uses this gives the same bits.)
template <typename T, int K>
__device__ __forceinline__ void xsum_block(const T *f, double *xsum, int nk, int X, double *red) {
  constexpr int EMAX_NONFINITE = sizeof(T) == 8 ? 2047 : 255;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, nw = blockDim.x >> 5;
  const size_t base = (size_t)X * nk * nk;
  const int n = nk * nk;
  int *ired = reinterpret_cast<int *>(red);
  long long *lred = reinterpret_cast<long long *>(red) + 32;
  int em;
  long long acc;
  xsum_hold<T, K>(f, base, n, em, acc, ired);  // one read of the block when n <= K * blockDim
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) lred[w] = acc;
  __syncthreads();
  if (tid == 0) {
    long long tot = 0;
    for (int q = 0; q < nw; ++q) tot += lred[q];
    xsum[X] = em == EMAX_NONFINITE ? __longlong_as_double(0x7ff8000000000000ll)
                                   : ll_to_double_scaled(tot, em - (sizeof(T) == 8 ? 1071 : 174));
  }
  __syncthreads();  // red is reused by the next item of a persistent caller
}

// The same exact per-X sum for a block whose threads hold its nk^2 values in
// registers (each value held by exactly one thread; threads without values
// pass zeros): block maximum exponent, fixed-point images, integer sum.  The
// result has the bits xsum_block gives for the same values.  Every thread of
// the block calls it; red: 64 ints of shared memory, 8-byte aligned, free on
// entry.  Thread 0 writes *out.
template <typename T, int N>
__device__ __forceinline__ void block_exact_sum(const T (&v)[N], double *out, int *red) {
  constexpr int EMAX_NONFINITE = sizeof(T) == 8 ? 2047 : 255;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, nw = blockDim.x >> 5;
  long long *lred = reinterpret_cast<long long *>(red + 32);
  int em = 0;
#pragma unroll
  for (int i = 0; i < N; ++i) em = max(em, expo_of(v[i]));
  em = __reduce_max_sync(0xffffffffu, em);
  if (lane == 0) red[w] = em;
  __syncthreads();
  em = 0;
  for (int q = 0; q < nw; ++q) em = max(em, red[q]);
  em = max(em, 1);
  long long acc = 0;
#pragma unroll
  for (int i = 0; i < N; ++i) acc += fixed_image(v[i], em);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) lred[w] = acc;
  __syncthreads();
  if (tid == 0) {
    long long tot = 0;
    for (int q = 0; q < nw; ++q) tot += lred[q];
    *out = em == EMAX_NONFINITE ? __longlong_as_double(0x7ff8000000000000ll)
                                : ll_to_double_scaled(tot, em - (sizeof(T) == 8 ? 1071 : 174));
  }
  __syncthreads();  // red is free again
}

}  // namespace w2
